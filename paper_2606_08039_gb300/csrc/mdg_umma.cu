// Fused inference of the surrogate network on the 5th-generation tensor cores (sm_103a):
// tcgen05.mma with the accumulators in tensor memory, operands in shared memory.
//
// One persistent thread block per SM takes 128-row tiles of drones; its warps have fixed
// roles and hand work to each other through mbarriers:
//
//   producer warp   streams the weights, chunk by chunk, into a ring of four 32 KB shared-
//                   memory slots with bulk asynchronous copies (cp.async.bulk, completion
//                   counted in bytes on the slot's mbarrier), and copies each tile's inputs
//                   into their operand buffer one tile ahead;
//   MMA warp        one thread issues the tcgen05.mma instructions (M = 128, N = 256 or 32,
//                   K = 16 each; bf16 x bf16 -> FP32) of every layer, one 64-column K chunk
//                   at a time, and commits them to the mbarriers that free a weight slot,
//                   free the input buffer, or announce a finished accumulator;
//   16 epilogue     read an accumulator back (tcgen05.ld), add the bias, apply SiLU and
//   warps           write the bf16 activations, chunk by chunk, as the next layer's A
//                   operand; the output layer's FP32 values go to global memory.
//
// The two 256-column accumulators in tensor memory alternate between layers, so layer
// l+1's MMAs on chunk c start as soon as the epilogue of layer l has written chunk c of
// the activations, while that epilogue still reads the rest of layer l's accumulator.
// Activations never leave the SM; the weights are re-read from L2 for every tile.
//
// Shared-memory operands use the canonical K-major layout with 128-byte swizzling: a
// [rows x 64] bf16 chunk stores row r at r * 128 bytes with its 16-byte pieces permuted by
// XOR with (r mod 8); every chunk starts on a 1024-byte boundary. The weights are kept in
// global memory as an image of exactly these chunks (mlp_build_image), so each slot is
// filled by one bulk copy. Every mbarrier wait is bounded: on expiry the block records
// MDG_STATUS_TIMEOUT in the status word, every role leaves its loop, the copies and MMAs
// already issued are waited for (again with a bound), the tensor memory is freed and the
// block returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "mdg.h"
#include "mdg_internal.cuh"

namespace mdg {
namespace {

constexpr int kRows = 128;                 // tile rows (UMMA M)
constexpr int kEpiWarps = 16;              // four per TMEM lane quadrant
constexpr int kProdWarp = kEpiWarps;       // producer warp
constexpr int kMmaWarp = kEpiWarps + 1;    // MMA warp (also allocates the tensor memory)
constexpr int kThreads = (kEpiWarps + 2) * 32;
constexpr int kSlots = 4;
constexpr uint32_t kSlotBytes = 32768;     // one [256 x 64] bf16 weight chunk
constexpr uint32_t kChunkBytes = 16384;    // one [128 x 64] bf16 activation chunk
constexpr uint32_t kOffAct = 0;            // activations [128 x 256]: four chunks
constexpr uint32_t kOffX = 4 * kChunkBytes;  // inputs [128 x 64]: one chunk
constexpr uint32_t kOffSlot = kOffX + kChunkBytes;
constexpr uint32_t kDynBytes = kOffSlot + kSlots * kSlotBytes;
constexpr uint32_t kTmemCols = 512;        // two accumulators of 256 columns
constexpr int kLoadsPerTile = 10;          // W1, W2 chunks 0-3, W3 chunks 0-3, W4
constexpr uint32_t kSuspendNs = 1000;      // longest suspension of one mbarrier try_wait
constexpr int kWaitLimit = MDG_MLP_DEFAULT_TRY_WAITS;  // try_waits (at most ~0.26 s) before giving up

// Weight image: the chunks in the order the MMAs consume them, load i at i * 32 KB.
//   load 0      W1 [256 x 64]
//   loads 1-4   W2 chunk c [256 x 64]
//   loads 5-8   W3 chunk c [256 x 64]
//   load 9      W4 [32 x 256] as four [32 x 64] chunks of 4 KB (16 KB)
constexpr uint32_t kImgBytes = 9 * kSlotBytes + 16384;
static_assert(kImgBytes == 2 * (256 * 64 + 2 * 256 * 256 + 32 * 256), "the image holds every weight once");
static_assert(kDynBytes + 1024 + 4096 <= 232448, "shared memory of one block");

__device__ __forceinline__ uint32_t image_layer_base(int l)
{
    return l == 0 ? 0u : l == 1 ? kSlotBytes : l == 2 ? 5 * kSlotBytes : 9 * kSlotBytes;
}

// mbarriers
enum {
    kBarWFull = 0,                    // [kSlots] producer expect_tx; the bulk copy completes it
    kBarWEmpty = kBarWFull + kSlots,  // [kSlots] MMA commit: the slot's MMAs are done
    kBarXFull = kBarWEmpty + kSlots,  // producer: the tile's inputs have landed
    kBarXEmpty,                       // MMA commit: layer 0 is done with the inputs
    kBarAccFull,                      // [2] MMA commit: accumulator b holds a finished layer
    kBarActFull = kBarAccFull + 2,    // [4] the 16 epilogue warps: activation chunk c written
    kBarMmaDone = kBarActFull + 4,    // MMA commit at the end: nothing left in flight
    kNumBars
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address
    d |= (uint64_t)1 << 16;                           // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                           // descriptor version
    d |= (uint64_t)2 << 61;                           // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: bf16 A and B (K-major), FP32 D, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_ss(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// The mbarrier completes once every tcgen05 operation issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase of `parity` to complete: one non-blocking test, then mbarrier.try_wait,
// which suspends the thread in hardware until the phase completes or about kSuspendNs pass.
// Gives up when another role has aborted (abort != null) or after `limit` tries, which
// records the timeout and aborts the block. The work waits take the launch's limit; the
// drain waits of the exit path always take kWaitLimit, so that a block leaves only once
// every copy and MMA it issued has completed.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, volatile int* abort, uint32_t* status,
                                          int limit)
{
    if (mbar_test(mbar, parity)) return true;
    for (int i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity), "r"(kSuspendNs)
            : "memory");
        if (done) return true;
        if (abort && *abort) return false;
    }
    if (abort) *abort = 1;
    atomicOr(status, MDG_STATUS_TIMEOUT);
    return false;
}

// The same for waits on the critical path between MMAs and epilogue: poll with test_wait
// (a suspended thread wakes up later than a polling one), backing off by `sleep_ns` between
// polls (0: none), at most `limit` polls.
__device__ __forceinline__ bool mbar_spin(uint32_t mbar, uint32_t parity, volatile int* abort, uint32_t* status,
                                          int sleep_ns, int limit)
{
    for (int i = 0; i < limit; ++i) {
        if (mbar_test(mbar, parity)) return true;
        if ((i & 63) == 63 && *abort) return false;
        if (sleep_ns) __nanosleep(sleep_ns);
    }
    *abort = 1;
    atomicOr(status, MDG_STATUS_TIMEOUT);
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

// Bulk copy global -> shared; completes `bytes` of the mbarrier's transaction count.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t s, const void* g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g));
}

// 16 (x16) or 8 (x8) consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// SiLU of two pre-activations given as h = z/2: silu(z) = z / (1 + exp(-z)) = h (1 + tanh h),
// one special-function instruction each (tanh.approx.f32, relative error about 2^-11).
__device__ __forceinline__ __nv_bfloat162 silu_pair(float h0, float h1)
{
    float t0, t1;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t0) : "f"(h0));
    asm("tanh.approx.f32 %0, %1;" : "=f"(t1) : "f"(h1));
    return __floats2bfloat162_rn(fmaf(h0, t0, h0), fmaf(h1, t1, h1));
}

__global__ void __launch_bounds__(kThreads, 1)
    mlp_umma_kernel(const __nv_bfloat16* __restrict__ x, float* __restrict__ y, int n_tiles,
                    const uint8_t* __restrict__ w_img, const float* __restrict__ master, MlpView w, uint32_t* status,
                    int wait_limit, int spin_limit)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bars[kNumBars];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    // b/2 of the hidden layers (SiLU takes z/2), then the output bias
    __shared__ __align__(16) float s_hb[3 * MDG_MLP_HIDDEN + MDG_MLP_OUT_PAD];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t act_a = smem_u32(base + kOffAct), x_a = smem_u32(base + kOffX), slot_a = smem_u32(base + kOffSlot);
    const uint32_t bar0 = smem_u32(&bars[0]);
    auto bar = [bar0](int i) { return bar0 + 8u * (uint32_t)i; };
    volatile int* abort = &s_abort;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kNumBars; ++i) {
            const uint32_t count = (i >= kBarActFull && i < kBarActFull + 4) ? kEpiWarps : 1;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar(i)), "r"(count));
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_abort = 0;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
#pragma unroll
    for (int l = 0; l < 4; ++l)
        for (int i = threadIdx.x; i < (l < 3 ? MDG_MLP_HIDDEN : MDG_MLP_OUT_PAD); i += kThreads)
            s_hb[l * MDG_MLP_HIDDEN + i] = (l < 3 ? 0.5f : 1.f) * master[w.b_off[l] + i];
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;

    if (warp == kProdWarp) {
        // ---------------- producer (whole warp; lane 0 issues the bulk copies) ----------------
        int j = 0;  // weight loads issued
        int s = 0;  // tiles of this block
        bool ok = true;
        auto load_x = [&](int tile) {
            const __nv_bfloat16* src = x + (size_t)tile * kRows * MDG_MLP_IN_PAD;
#pragma unroll 4
            for (int i = lane; i < kRows * 8; i += 32) {
                const int r = i >> 3, k8 = i & 7;
                cp_async16(x_a + r * 128 + ((k8 ^ (r & 7)) << 4), src + r * MDG_MLP_IN_PAD + k8 * 8);
            }
        };
        load_x(blockIdx.x);  // the grid never exceeds the tile count
        for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++s) {
            for (int i = 0; i < kLoadsPerTile; ++i, ++j) {
                const int slot = j % kSlots, use = j / kSlots;
                if (use > 0) ok = __all_sync(0xffffffffu, mbar_wait(bar(kBarWEmpty + slot), (use - 1) & 1, abort, status, wait_limit));
                if (!ok) break;
                const uint32_t bytes = i == kLoadsPerTile - 1 ? 16384u : kSlotBytes;
                if (lane == 0) {
                    mbar_expect_tx(bar(kBarWFull + slot), bytes);
                    bulk_g2s(slot_a + slot * kSlotBytes, w_img + (size_t)i * kSlotBytes, bytes, bar(kBarWFull + slot));
                }
                __syncwarp();
                if (i == 0) {
                    // this tile's inputs (issued one tile ahead) complete before layer 0 reads them
                    asm volatile("cp.async.wait_all;\n" ::: "memory");
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar(kBarXFull));
                } else if (i == 4 && tile + (int)gridDim.x < n_tiles) {
                    // layer 0 of this tile is done with the input buffer: fetch the next tile's
                    ok = __all_sync(0xffffffffu, mbar_wait(bar(kBarXEmpty), s & 1, abort, status, wait_limit));
                    if (!ok) {
                        ++j;
                        break;
                    }
                    load_x(tile + gridDim.x);
                }
            }
        }
        // drain: every copy issued has landed before the block may exit
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        if (lane == 0)
            for (int slot = 0; slot < kSlots && slot < j; ++slot) {
                const int uses = (j - 1 - slot) / kSlots + 1;  // loads issued into this slot
                mbar_wait(bar(kBarWFull + slot), (uses - 1) & 1, nullptr, status, kWaitLimit);
            }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issue (one thread) ----------------
        if (lane == 0) {
            const uint32_t id_h = idesc_bf16(kRows, MDG_MLP_HIDDEN), id_o = idesc_bf16(kRows, MDG_MLP_OUT_PAD);
            int j = 0, s = 0;
            uint32_t n_act = 0;  // completed activation phases (one per hidden-layer epilogue)
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++s) {
                // layer 0: x [128 x 64] . W1^T -> accumulator 0
                ok = mbar_wait(bar(kBarXFull), s & 1, abort, status, wait_limit) &&
                     mbar_wait(bar(kBarWFull + j % kSlots), (j / kSlots) & 1, abort, status, wait_limit);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                {
                    const uint32_t wsl = slot_a + (j % kSlots) * kSlotBytes;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        mma_bf16_ss(tmem, sw128_desc(x_a + k * 32), sw128_desc(wsl + k * 32), id_h, k != 0);
                    mma_commit(bar(kBarWEmpty + j % kSlots));
                    mma_commit(bar(kBarXEmpty));
                    mma_commit(bar(kBarAccFull + 0));
                    ++j;
                }
                // layers 1, 2: chunk c of the activations as soon as the epilogue has written it.
                // The tensor cores take ~128 cycles per MMA and this thread can run only about
                // one MMA ahead of them, so the bookkeeping of the next group (the previous
                // group's commit, non-blocking tests of the next group's barriers) is spread
                // between the four MMAs of the current one.
                for (int l = 1; l < 3 && ok; ++l) {
                    const uint32_t d = tmem + (uint32_t)(l & 1) * 256;
                    bool act_ok = false, w_ok = false;  // the group's barriers, tested ahead
                    for (int c = 0; c < 4; ++c, ++j) {
                        ok = (act_ok || mbar_spin(bar(kBarActFull + c), n_act & 1, abort, status, 0, spin_limit)) &&
                             (w_ok || mbar_wait(bar(kBarWFull + j % kSlots), (j / kSlots) & 1, abort, status,
                                                wait_limit));
                        if (!ok) break;
                        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                        const uint32_t asl = act_a + c * kChunkBytes, wsl = slot_a + (j % kSlots) * kSlotBytes;
                        mma_bf16_ss(d, sw128_desc(asl), sw128_desc(wsl), id_h, c != 0);
                        if (c > 0) mma_commit(bar(kBarWEmpty + (j - 1) % kSlots));
                        mma_bf16_ss(d, sw128_desc(asl + 32), sw128_desc(wsl + 32), id_h, 1);
                        act_ok = c < 3 && mbar_test(bar(kBarActFull + c + 1), n_act & 1);
                        mma_bf16_ss(d, sw128_desc(asl + 64), sw128_desc(wsl + 64), id_h, 1);
                        w_ok = c < 3 && mbar_test(bar(kBarWFull + (j + 1) % kSlots), ((j + 1) / kSlots) & 1);
                        mma_bf16_ss(d, sw128_desc(asl + 96), sw128_desc(wsl + 96), id_h, 1);
                    }
                    if (!ok) break;
                    mma_commit(bar(kBarWEmpty + (j - 1) % kSlots));
                    ++n_act;
                    mma_commit(bar(kBarAccFull + (l & 1)));
                }
                if (!ok) break;
                // layer 3: W4 [32 x 256] in one slot as four [32 x 64] chunks -> accumulator 1
                ok = mbar_wait(bar(kBarWFull + j % kSlots), (j / kSlots) & 1, abort, status, wait_limit);
                const uint32_t wsl = slot_a + (j % kSlots) * kSlotBytes;
                bool act_ok = false;
                for (int c = 0; c < 4 && ok; ++c) {
                    ok = act_ok || mbar_spin(bar(kBarActFull + c), n_act & 1, abort, status, 0, spin_limit);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    const uint32_t asl = act_a + c * kChunkBytes, bsl = wsl + c * 4096;
                    mma_bf16_ss(tmem + 256, sw128_desc(asl), sw128_desc(bsl), id_o, c != 0);
                    mma_bf16_ss(tmem + 256, sw128_desc(asl + 32), sw128_desc(bsl + 32), id_o, 1);
                    act_ok = c < 3 && mbar_test(bar(kBarActFull + c + 1), n_act & 1);
                    mma_bf16_ss(tmem + 256, sw128_desc(asl + 64), sw128_desc(bsl + 64), id_o, 1);
                    mma_bf16_ss(tmem + 256, sw128_desc(asl + 96), sw128_desc(bsl + 96), id_o, 1);
                }
                if (!ok) break;
                ++n_act;
                mma_commit(bar(kBarWEmpty + j % kSlots));
                mma_commit(bar(kBarAccFull + 1));
                ++j;
            }
            // nothing in flight before the tensor memory is freed
            mma_commit(bar(kBarMmaDone));
            mbar_wait(bar(kBarMmaDone), 0, nullptr, status, kWaitLimit);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 0-15) ----------------
        const int q = warp & 3, p = warp >> 2;  // TMEM lane quadrant, column part
        const int row = q * 32 + lane;
        const uint32_t t_row = tmem + ((uint32_t)(q * 32) << 16);
        const int sw = row & 7;
        uint32_t n_acc0 = 0, n_acc1 = 0;  // completed phases of the two accumulators
        bool ok = true;
        for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
            for (int l = 0; l < 3 && ok; ++l) {
                const int b = l & 1;
                ok = __all_sync(0xffffffffu, mbar_spin(bar(kBarAccFull + b), (b ? n_acc1 : n_acc0) & 1, abort, status, 32,
                                                       spin_limit));
                if (!ok) break;
                n_acc0 += 1 - b;
                n_acc1 += b;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const float4* hb4 = reinterpret_cast<const float4*>(s_hb + l * MDG_MLP_HIDDEN);
#pragma unroll 1
                for (int c = 0; c < 4; ++c) {
                    const int col = c * 64 + p * 16;
                    float v[16];
                    tmem_ld16(t_row + (uint32_t)b * 256 + col, v);
                    float hb[16];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 t = hb4[col / 4 + i];
                        hb[4 * i] = t.x, hb[4 * i + 1] = t.y, hb[4 * i + 2] = t.z, hb[4 * i + 3] = t.w;
                    }
                    __nv_bfloat162 o[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        o[i] = silu_pair(fmaf(v[2 * i], 0.5f, hb[2 * i]), fmaf(v[2 * i + 1], 0.5f, hb[2 * i + 1]));
                    uint8_t* dst = base + kOffAct + c * kChunkBytes + row * 128;
                    *reinterpret_cast<uint4*>(dst + (((2 * p) ^ sw) << 4)) = *reinterpret_cast<const uint4*>(&o[0]);
                    *reinterpret_cast<uint4*>(dst + (((2 * p + 1) ^ sw) << 4)) = *reinterpret_cast<const uint4*>(&o[4]);
                    // generic-proxy stores -> the MMAs' async proxy; TMEM reads done before the arrive
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar(kBarActFull + c));
                }
            }
            if (!ok) break;
            // output layer: accumulator 1, 32 columns, eight per column part
            ok = __all_sync(0xffffffffu, mbar_spin(bar(kBarAccFull + 1), n_acc1 & 1, abort, status, 32, spin_limit));
            if (!ok) break;
            ++n_acc1;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            float v[8];
            tmem_ld8(t_row + 256 + p * 8, v);
            const float* b4 = s_hb + 3 * MDG_MLP_HIDDEN + p * 8;
            float4* out = reinterpret_cast<float4*>(y + ((size_t)tile * kRows + row) * MDG_MLP_OUT_PAD + p * 8);
            out[0] = make_float4(v[0] + b4[0], v[1] + b4[1], v[2] + b4[2], v[3] + b4[3]);
            out[1] = make_float4(v[4] + b4[4], v[5] + b4[5], v[6] + b4[6], v[7] + b4[7]);
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

// ---- paired inference: two 128-row tiles in flight ----
//
// The kernel above holds both 256-column TMEM accumulators for its one tile (layer l is read
// out while layer l + 1 accumulates), so its tensor cores idle while the epilogue of each
// layer's first chunk runs. Here the epilogue first moves a layer's whole accumulator into
// registers (each of the 16 epilogue threads of a row quadrant and column part holds its 64
// values) and only then computes SiLU, so the layer's 256 columns are free again at once: one
// tile needs one accumulator, and two tiles, A in columns 0-255 and B in 256-511, alternate:
// while the epilogue works on one tile's layer, the tensor cores run the other tile's. The
// MMA thread issues, per pair of tiles, A.L1, B.L1 (one W1 chunk for both), A.L2, B.L2, A.L3,
// B.L3, A.L4, B.L4 (one W4 load). The W2/W3 chunks stream through a three-slot ring: tile A
// takes K chunks 0-3 in order, tile B then takes 1, 2 and 3 while they are still resident and
// reloads 0, so a hidden layer costs five chunk loads per pair instead of eight (tile B sums
// its K chunks in the order 1, 2, 3, 0; tile A's arithmetic is the single-tile kernel's). The
// slots are released in the order they were filled, so load n of the block goes to slot n % 3.
// The inputs have no buffer of their own: each tile's [128 x 64] input is written by TMA (a
// tensor map with the 128-byte swizzle) into chunk 0 of its activation buffer once the
// previous pair's layer 4 has read that buffer (ActFree), prefetched into L2 a pair ahead.
// A layer's first MMA into a tile's accumulator waits for the epilogue to have drained the
// previous layer (AccDrained); tile A's MMA on K chunk c waits for chunk c of the previous
// layer's activations (ActFull); tile B's layer waits once for chunk 3 (each epilogue warp
// writes the chunks in order, so 3 implies all). Waits are bounded as above, with the same exit.
constexpr uint32_t kPActA = 0;                          // tile A activations: 4 chunks
constexpr uint32_t kPActB = 4 * kChunkBytes;            // tile B activations
constexpr uint32_t kPSlot = 8 * kChunkBytes;            // three weight slots
constexpr int kPSlots = 3;
constexpr uint32_t kPDynBytes = kPSlot + kPSlots * kSlotBytes;
static_assert(kPDynBytes + 1024 + 512 <= 232448, "shared memory of one paired block");
constexpr int kPLoadsPerPair = 12;  // W1, W2 c0-3, W2 c0 (B), W3 c0-3, W3 c0 (B), W4
static_assert(kPLoadsPerPair % kPSlots == 0, "every pair starts at slot 0");

enum {
    kPBarWFull = 0,                       // [3]
    kPBarWEmpty = kPBarWFull + kPSlots,   // [3]
    kPBarXFull = kPBarWEmpty + kPSlots,   // [2] TMA: tile A's, B's inputs landed
    kPBarActFree = kPBarXFull + 2,        // [2] MMA commit: layer 4 has read the tile's activations
    kPBarAccFull = kPBarActFree + 2,      // [2] MMA commit: the tile's layer is accumulated
    kPBarAccDrained = kPBarAccFull + 2,   // [2] 16 epilogue warps: the accumulator is in registers
    kPBarActFull = kPBarAccDrained + 2,   // [2][4] 16 epilogue warps: activation chunk c written
    kPBarMmaDone = kPBarActFull + 8,
    kPNumBars
};

// Image index of load k of a pair: 0 W1; 1-4 W2 c0-3, 5 W2 c0; 6-9 W3 c0-3, 10 W3 c0; 11 W4.
__device__ __forceinline__ int pair_load_image(int k) { return (int)((0x958765143210ull >> (4 * k)) & 15u); }

// TMA of one [128 x 64] bf16 input tile (rows row..row+127) into 128-byte-swizzled shared
// memory, completing on mbar; and its prefetch into L2.
__device__ __forceinline__ void tma_rows(uint32_t dst, const CUtensorMap* map, int row, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row), "r"(mbar) : "memory");
}
__device__ __forceinline__ void tma_rows_prefetch(const CUtensorMap* map, int row)
{
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];\n"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row) : "memory");
}

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t r[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

template <bool kApply>
__global__ void __launch_bounds__(kThreads, 1)
    mlp_umma_pair_kernel(const __grid_constant__ CUtensorMap xmap, float* __restrict__ y, int n_tiles,
                         const uint8_t* __restrict__ w_img, const float* __restrict__ master, MlpView w,
                         uint32_t* status, int wait_limit, int spin_limit, const MlpApply ap)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bars[kPNumBars];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t act0 = smem_u32(base + kPActA), slot_a = smem_u32(base + kPSlot);
    const uint32_t bar0 = smem_u32(&bars[0]);
    auto bar = [bar0](int i) { return bar0 + 8u * (uint32_t)i; };
    volatile int* abort = &s_abort;
    const int n_pairs = (n_tiles + 1) / 2;

    if (threadIdx.x == 0) {
        for (int i = 0; i < kPNumBars; ++i) {
            const bool epi = (i >= kPBarAccDrained && i < kPBarMmaDone);
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar(i)), "r"(epi ? kEpiWarps : 1));
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_abort = 0;
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;

    if (warp == kProdWarp) {
        // ---------------- producer (one thread) ----------------
        if (lane == 0) {
            int issued = 0, x_issued0 = 0, x_issued1 = 0;
            bool ok = true;
            auto load_x = [&](int pr, int t) {
                mbar_expect_tx(bar(kPBarXFull + t), kChunkBytes);
                tma_rows(act0 + (uint32_t)t * 4 * kChunkBytes, &xmap, (2 * pr + t) * kRows, bar(kPBarXFull + t));
                if (t) ++x_issued1; else ++x_issued0;
            };
            if (blockIdx.x < n_pairs) {  // the grid never exceeds the pair count
                load_x(blockIdx.x, 0);
                if (2 * blockIdx.x + 1 < n_tiles) load_x(blockIdx.x, 1);
            }
            int s = 0;  // pairs of this block
            for (int pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x, ++s) {
                const int next = pr + (int)gridDim.x;
                const bool hasB = 2 * pr + 1 < n_tiles;
                for (int k = 0; k < kPLoadsPerPair; ++k) {
                    const int n = kPLoadsPerPair * s + k, slot = k % kPSlots;
                    if (n >= kPSlots)
                        ok = mbar_spin(bar(kPBarWEmpty + slot), (n / kPSlots - 1) & 1, abort, status, 0, spin_limit);
                    if (!ok) break;
                    const int img = pair_load_image(k);
                    const uint32_t bytes = img == 9 ? 16384u : kSlotBytes;
                    mbar_expect_tx(bar(kPBarWFull + slot), bytes);
                    bulk_g2s(slot_a + slot * kSlotBytes, w_img + (size_t)img * kSlotBytes, bytes, bar(kPBarWFull + slot));
                    ++issued;
                    if (k == 1 && s > 0) {
                        // the previous pair's layer 4 has read tile A's (then B's) activations:
                        // this pair's inputs go into their chunk 0
                        ok = mbar_spin(bar(kPBarActFree + 0), (s - 1) & 1, abort, status, 0, spin_limit);
                        if (!ok) break;
                        load_x(pr, 0);
                        ok = mbar_spin(bar(kPBarActFree + 1), (s - 1) & 1, abort, status, 0, spin_limit);
                        if (!ok) break;
                        if (hasB) load_x(pr, 1);
                    } else if (k == 2 && next < n_pairs) {
                        tma_rows_prefetch(&xmap, 2 * next * kRows);
                        if (2 * next + 1 < n_tiles) tma_rows_prefetch(&xmap, (2 * next + 1) * kRows);
                    }
                }
            }
            // drain: every copy issued has landed before the block may exit
            for (int slot = 0; slot < kPSlots; ++slot) {
                int last = issued - 1;
                while (last >= 0 && last % kPSlots != slot) --last;
                if (last >= 0) mbar_wait(bar(kPBarWFull + slot), (last / kPSlots) & 1, nullptr, status, kWaitLimit);
            }
            if (x_issued0 > 0) mbar_wait(bar(kPBarXFull + 0), (x_issued0 - 1) & 1, nullptr, status, kWaitLimit);
            if (x_issued1 > 0) mbar_wait(bar(kPBarXFull + 1), (x_issued1 - 1) & 1, nullptr, status, kWaitLimit);
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issue (one thread) ----------------
        if (lane == 0) {
            const uint32_t id_h = idesc_bf16(kRows, MDG_MLP_HIDDEN), id_o = idesc_bf16(kRows, MDG_MLP_OUT_PAD);
            int s = 0;
            // AccDrained and ActFull phases completed per tile (kept in registers: A in the low,
            // B in the high half)
            uint32_t n_drain = 0u, n_act = 0u;
            bool ok = true;
            auto wfull = [&](int k) {
                const int n = kPLoadsPerPair * s + k;
                return mbar_spin(bar(kPBarWFull + k % kPSlots), (n / kPSlots) & 1, abort, status, 0, spin_limit);
            };
            // Shared-memory descriptors, computed once: a chunk's or slot's descriptor is the base
            // descriptor plus its byte offset / 16 in the start-address field (every address of
            // the block's shared memory is below 256 KB, so the field never carries), and the
            // K step of 16 bf16 within a 128-byte row adds 32 bytes, i.e. 2.
            const uint64_t act_desc = sw128_desc(act0), slot_desc = sw128_desc(slot_a);
            auto wslot = [&](int k) { return slot_desc + (uint64_t)((k % kPSlots) * (kSlotBytes >> 4)); };
            auto release = [&](int k) { mma_commit(bar(kPBarWEmpty + k % kPSlots)); };
            // the first MMA of a layer into tile t's accumulator: the previous layer drained
            auto drained = [&](int t) {
                const bool r = mbar_spin(bar(kPBarAccDrained + t), (n_drain >> (16 * t)) & 1, abort, status, 0, spin_limit);
                n_drain += 1u << (16 * t);
                return r;
            };
            auto act = [&](int t, int c) {
                return mbar_spin(bar(kPBarActFull + 4 * t + c), (n_act >> (16 * t)) & 1, abort, status, 0, spin_limit);
            };
            // K chunk c of tile t's activations against the weight chunk in slot ws: four MMAs
            auto chunk = [&](int t, int c, uint64_t wd, uint32_t id, bool first) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint64_t ad = act_desc + (uint64_t)((t * 4 + c) * (kChunkBytes >> 4));
                const uint32_t d = tmem + 256u * t;
                mma_bf16_ss(d, ad, wd, id, !first);
#pragma unroll
                for (int k = 1; k < 4; ++k) mma_bf16_ss(d, ad + 2 * k, wd + 2 * k, id, 1);
            };
            for (int pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x, ++s) {
                const bool hasB = 2 * pr + 1 < n_tiles;
                const int nt = hasB ? 2 : 1;
                // layer 1: the inputs in chunk 0 of each tile's activation buffer, one W1 chunk (load 0)
                ok = wfull(0);
                for (int t = 0; t < nt && ok; ++t) {
                    ok = mbar_wait(bar(kPBarXFull + t), s & 1, abort, status, wait_limit) && (s == 0 || drained(t));
                    if (!ok) break;
                    chunk(t, 0, wslot(0), id_h, true);
                    mma_commit(bar(kPBarAccFull + t));
                }
                if (!ok) break;
                release(0);
                // layers 2 and 3 (loads k0..k0+4): A chunks 0-3 in order, each as soon as the
                // epilogue has written it; B chunks 1, 2, 3 (A's loads, still resident) and 0 (reloaded)
                for (int l = 1; l < 3 && ok; ++l) {
                    const int k0 = l == 1 ? 1 : 6;
                    for (int c = 0; c < 4 && ok; ++c) {
                        ok = wfull(k0 + c) && (c != 0 || drained(0)) && act(0, c);
                        if (!ok) break;
                        chunk(0, c, wslot(k0 + c), id_h, c == 0);
                        if (c == 3) mma_commit(bar(kPBarAccFull + 0));
                        if (c == 0) release(k0);
                    }
                    if (!ok) break;
                    n_act += 1u;
                    for (int i = 0; i < 4 && ok; ++i) {
                        const int c = (i + 1) & 3;
                        const int k = i < 3 ? k0 + 1 + i : k0 + 4;
                        if (hasB) {
                            ok = (i < 3 || wfull(k)) && (i != 0 || (drained(1) && act(1, 3)));
                            if (!ok) break;
                            chunk(1, c, wslot(k), id_h, i == 0);
                            if (i == 3) mma_commit(bar(kPBarAccFull + 1));
                        } else {
                            ok = i < 3 || wfull(k);  // tile B missing: its load still lands, and is released
                            if (!ok) break;
                        }
                        release(k);
                    }
                    if (ok && hasB) n_act += 1u << 16;
                }
                if (!ok) break;
                // layer 4: W4 [32 x 256] as four [32 x 64] chunks in one slot (load 11), A then B;
                // after each, the tile's activation buffer is free for the next pair's inputs
                ok = wfull(11);
                for (int t = 0; t < nt && ok; ++t) {
                    ok = drained(t);
                    const uint64_t wsl = wslot(11);
                    for (int c = 0; c < 4 && ok; ++c) {
                        if (t == 0 || c == 0) ok = act(t, t == 0 ? c : 3);
                        if (!ok) break;
                        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                        const uint64_t ad = act_desc + (uint64_t)((t * 4 + c) * (kChunkBytes >> 4));
                        const uint64_t bd = wsl + (uint64_t)(c * (4096 >> 4));
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            mma_bf16_ss(tmem + 256u * t, ad + 2 * k, bd + 2 * k, id_o, (c | k) != 0);
                    }
                    if (!ok) break;
                    n_act += 1u << (16 * t);
                    mma_commit(bar(kPBarAccFull + t));
                    mma_commit(bar(kPBarActFree + t));
                }
                if (!ok) break;
                if (!hasB) mma_commit(bar(kPBarActFree + 1));
                release(11);
            }
            // nothing in flight before the tensor memory is freed
            mma_commit(bar(kPBarMmaDone));
            mbar_wait(bar(kPBarMmaDone), 0, nullptr, status, kWaitLimit);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 0-15) ----------------
        const int q = warp & 3, p = warp >> 2;  // TMEM lane quadrant, column part
        const int row = q * 32 + lane;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const int sw = row & 7;
        uint32_t n_acc[2] = {0u, 0u};
        bool ok = true;
        for (int pr = blockIdx.x; pr < n_pairs && ok; pr += gridDim.x) {
            const bool hasB = 2 * pr + 1 < n_tiles;
            const int nt = hasB ? 2 : 1;
            for (int l = 0; l < 3 && ok; ++l) {
                const float* bias = master + w.b_off[l];
                for (int t = 0; t < nt && ok; ++t) {
                    ok = __all_sync(0xffffffffu, mbar_spin(bar(kPBarAccFull + t), n_acc[t] & 1, abort, status, 32,
                                                           spin_limit));
                    if (!ok) break;
                    ++n_acc[t];
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    // the whole accumulator part of this thread (4 chunks x 16 columns) into registers
                    uint32_t r[4][16];
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        tmem_ld16_nowait(tmem + 256u * t + lane_off + (uint32_t)(c * 64 + p * 16), r[c]);
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar(kPBarAccDrained + t));
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int col = c * 64 + p * 16;
                        float hb[16];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float4 b4 = __ldg(reinterpret_cast<const float4*>(bias + col) + i);
                            hb[4 * i] = 0.5f * b4.x, hb[4 * i + 1] = 0.5f * b4.y, hb[4 * i + 2] = 0.5f * b4.z,
                                      hb[4 * i + 3] = 0.5f * b4.w;
                        }
                        __nv_bfloat162 o[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            o[i] = silu_pair(fmaf(__uint_as_float(r[c][2 * i]), 0.5f, hb[2 * i]),
                                             fmaf(__uint_as_float(r[c][2 * i + 1]), 0.5f, hb[2 * i + 1]));
                        uint8_t* dst = base + (t ? kPActB : kPActA) + c * kChunkBytes + row * 128;
                        *reinterpret_cast<uint4*>(dst + (((2 * p) ^ sw) << 4)) = *reinterpret_cast<const uint4*>(&o[0]);
                        *reinterpret_cast<uint4*>(dst + (((2 * p + 1) ^ sw) << 4)) = *reinterpret_cast<const uint4*>(&o[4]);
                        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                        __syncwarp();
                        if (lane == 0) mbar_arrive(bar(kPBarActFull + 4 * t + c));
                    }
                }
            }
            // output layer: 32 columns, eight per column part
            for (int t = 0; t < nt && ok; ++t) {
                ok = __all_sync(0xffffffffu, mbar_spin(bar(kPBarAccFull + t), n_acc[t] & 1, abort, status, 32,
                                                       spin_limit));
                if (!ok) break;
                ++n_acc[t];
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const int tile = 2 * pr + t;
                if constexpr (!kApply) {
                    float v[8];
                    tmem_ld8(tmem + 256u * t + lane_off + p * 8, v);
                    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bar(kPBarAccDrained + t));
                    const float* b4 = master + w.b_off[3] + p * 8;
                    float4* out = reinterpret_cast<float4*>(y + ((size_t)tile * kRows + row) * MDG_MLP_OUT_PAD + p * 8);
                    out[0] = make_float4(v[0] + b4[0], v[1] + b4[1], v[2] + b4[2], v[3] + b4[3]);
                    out[1] = make_float4(v[4] + b4[4], v[5] + b4[5], v[6] + b4[6], v[7] + b4[7]);
                    continue;
                } else {
                // the state update instead of y: the warps of column part 0 read the row's first
                // 16 columns (the 13 outputs) and update their drone; the others only release
                float v[16];
                if (p == 0) {
                    tmem_ld8(tmem + 256u * t + lane_off, v);
                    tmem_ld8(tmem + 256u * t + lane_off + 8, v + 8);
                }
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(bar(kPBarAccDrained + t));
                const long long g = (long long)tile * kRows + row;
                if (p == 0 && g < ap.n && !ap.env_flag[g / ap.uniform_N]) {
                    const float* b = master + w.b_off[3];
                    float dl[13];
#pragma unroll
                    for (int k = 0; k < 13; ++k) dl[k] = ap.out_mean[k] + ap.out_std[k] * (v[k] + b[k]);
                    float4* S = ap.state;
                    const long long n = ap.n;
                    float4 s0 = S[g], s1 = S[n + g], s2 = S[2 * n + g], s3 = S[3 * n + g];
                    s0.x += dl[0], s0.y += dl[1], s0.z += dl[2];
                    float qv[4] = {s0.w + dl[3], s1.x + dl[4], s1.y + dl[5], s1.z + dl[6]};
                    s1.w += dl[7], s2.x += dl[8], s2.y += dl[9];
                    s2.z += dl[10], s2.w += dl[11], s3.x += dl[12];
                    float qn = 0.f;
#pragma unroll
                    for (int r = 0; r < 4; ++r) qn += qv[r] * qv[r];
                    const float inv = rsqrtf(qn);
                    s0.w = qv[0] * inv, s1.x = qv[1] * inv, s1.y = qv[2] * inv, s1.z = qv[3] * inv;
                    S[g] = s0, S[n + g] = s1, S[2 * n + g] = s2, S[3 * n + g] = s3;
                }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

// ---- training GEMMs on tcgen05: C[M x N] = A[M x K] B[N x K]^T, both operands K-major ----
//
// One 128-thread block computes a 128 x BN tile of C over a range of K (split-K when
// gridDim.z > 1: the partial tiles are added to the output with atomics). Per 64-wide K chunk
// every thread copies its share of the A and B chunks into shared memory (cp.async, 16 bytes
// each, written straight into the 128-byte-swizzled K-major layout of the inference kernel's
// operands; a 32-wide last chunk is padded with zeros), one thread issues the chunk's four
// tcgen05.mma (K = 16 each) into the TMEM accumulator and commits them to the chunk's stage
// mbarrier; two stages alternate, so the next chunk's copies overlap this chunk's MMAs. The
// epilogue reads the accumulator row by row (thread = row, tcgen05.ld.32x32b) and hands every
// element (m, n, acc) to the layer's epilogue functor. Waits are bounded: on expiry the block
// records MDG_STATUS_TIMEOUT, drains its MMAs, skips its epilogue and frees its TMEM.
constexpr int kGemmThreads = 128;

template <int BN>
struct GemmShape {
    static constexpr uint32_t a_bytes = 128 * 128;                    // [128 x 64] bf16
    static constexpr uint32_t b_bytes = BN * 128;                     // [BN x 64] bf16
    static constexpr uint32_t stage_bytes = a_bytes + b_bytes;
    static constexpr uint32_t smem = 1024 + 2 * stage_bytes;          // alignment slack + two stages
    static constexpr uint32_t tmem_cols = BN < 32 ? 32 : BN;
};

// Copies rows [row0, row0 + rows) x columns [k0, k0 + kw) (kw = 64 or 32) of a K-major bf16
// matrix (leading dimension ld elements) into a swizzled [rows x 64] chunk at `dst`; columns
// beyond kw are zero.
__device__ __forceinline__ void load_chunk(uint32_t dst, const __nv_bfloat16* src, int ld, int row0, int rows, int k0,
                                           int kw, uint8_t* dst_generic)
{
    const int pieces = kw / 8;
    for (int i = threadIdx.x; i < rows * 8; i += kGemmThreads) {
        const int r = i >> 3, k8 = i & 7;
        const uint32_t off = (uint32_t)r * 128 + ((k8 ^ (r & 7)) << 4);
        if (k8 < pieces) cp_async16(dst + off, src + (size_t)(row0 + r) * ld + k0 + k8 * 8);
        else *reinterpret_cast<uint4*>(dst_generic + off) = make_uint4(0u, 0u, 0u, 0u);
    }
}

template <int BN, class Epi>
__global__ void __launch_bounds__(kGemmThreads) umma_gemm_kernel(const __nv_bfloat16* __restrict__ A, int lda,
                                                                 const __nv_bfloat16* __restrict__ B, int ldb, int K,
                                                                 int k_per_split, Epi epi, uint32_t* status)
{
    using S = GemmShape<BN>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bars[3];  // stage 0, stage 1: MMAs done with the stage; 2: accumulator done
    __shared__ uint32_t s_tmem;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * 128, n0 = blockIdx.x * BN;
    const int k_begin = blockIdx.z * k_per_split;
    const int k_end = min(K, k_begin + k_per_split);
    const uint32_t bar0 = smem_u32(&bars[0]);
    if (threadIdx.x == 0) {
        for (int i = 0; i < 3; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0 + 8u * i));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(S::tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = idesc_bf16(128, BN);

    bool ok = true;
    int c = 0;  // chunks issued
    for (int k0 = k_begin; k0 < k_end; k0 += 64, ++c) {
        const int st = c & 1;
        if (c >= 2) {  // the MMAs of chunk c - 2 have read this stage
            const bool done = mbar_wait(bar0 + 8u * st, ((c - 2) >> 1) & 1, nullptr, status, kWaitLimit);
            ok = __syncthreads_and(done);
            if (!ok) break;
        }
        const int kw = min(64, k_end - k0);
        uint8_t* sa = base + st * S::stage_bytes;
        uint8_t* sb = sa + S::a_bytes;
        load_chunk(smem_u32(sa), A, lda, m0, 128, k0, kw, sa);
        load_chunk(smem_u32(sb), B, ldb, n0, BN, k0, kw, sb);
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mma_bf16_ss(tmem, sw128_desc(smem_u32(sa) + kk * 32), sw128_desc(smem_u32(sb) + kk * 32), idesc,
                            (c > 0 || kk > 0) ? 1u : 0u);
            mma_commit(bar0 + 8u * st);
        }
    }
    // every MMA issued has completed before the accumulator is read or the TMEM freed
    if (threadIdx.x == 0) mma_commit(bar0 + 16u);
    const bool drained = mbar_wait(bar0 + 16u, 0, nullptr, status, kWaitLimit);
    ok = __syncthreads_and(ok && drained && c > 0);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
        const int row = warp * 32 + lane;
        const uint32_t t_row = tmem + ((uint32_t)(warp * 32) << 16);
        float loss = 0.f;
#pragma unroll 1
        for (int cc = 0; cc < BN; cc += 16) {
            float v[16];
            tmem_ld16(t_row + cc, v);
            loss += epi.chunk(m0 + row, n0 + cc, v);
        }
        epi.finish(loss);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(S::tmem_cols));
}

__device__ __forceinline__ float silu_train(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad_train(float z)
{
    const float sg = 1.f / (1.f + __expf(-z));
    return sg * (1.f + z * (1.f - sg));
}

// The epilogues take the 16 consecutive accumulator columns n0 .. n0 + 15 of row m (one
// thread per row): row-major outputs are written 16 bytes at a time, transposed outputs one
// element per thread, consecutive rows of a warp side by side.
__device__ __forceinline__ void store_bf16x16(__nv_bfloat16* dst, const float v[16])
{
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<const uint32_t*>(&p);
    }
    reinterpret_cast<uint4*>(dst)[0] = make_uint4(w[0], w[1], w[2], w[3]);
    reinterpret_cast<uint4*>(dst)[1] = make_uint4(w[4], w[5], w[6], w[7]);
}
__device__ __forceinline__ void store_f32x16(float* dst, const float v[16])
{
#pragma unroll
    for (int i = 0; i < 4; ++i)
        reinterpret_cast<float4*>(dst)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}
__device__ __forceinline__ void load_f32x16(const float* src, float v[16])
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 t = reinterpret_cast<const float4*>(src)[i];
        v[4 * i] = t.x, v[4 * i + 1] = t.y, v[4 * i + 2] = t.z, v[4 * i + 3] = t.w;
    }
}

// Hidden layer forward: z = acc + b[n] (FP32, kept for the backward pass), h = bf16(silu(z))
// row-major and transposed (the transposed copy is the K-major operand of the weight gradient).
struct TrainEpiHidden {
    const float* bias;
    float* z;
    __nv_bfloat16* h;
    __nv_bfloat16* hT;
    int ld, ldT;
    __device__ __forceinline__ float chunk(int m, int n0, const float acc[16]) const
    {
        float zz[16], hv[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            zz[i] = acc[i] + bias[n0 + i];
            hv[i] = silu_train(zz[i]);
        }
        store_f32x16(z + (size_t)m * ld + n0, zz);
        store_bf16x16(h + (size_t)m * ld + n0, hv);
#pragma unroll
        for (int i = 0; i < 16; ++i) hT[(size_t)(n0 + i) * ldT + m] = __float2bfloat16_rn(hv[i]);
        return 0.f;
    }
    __device__ __forceinline__ void finish(float) const {}
};

// Output layer forward with the MSE: y = acc + b[n]; on the n_valid used columns
// dy = scale (y - t) (bf16, row-major and transposed) and loss += (y - t)^2 / (rows n_valid).
struct TrainEpiOut {
    const float* bias;
    float* y;
    const float* target;
    __nv_bfloat16* dy;
    __nv_bfloat16* dyT;
    float* loss_acc;
    int ld, ldT, n_valid;
    float grad_scale, loss_scale;
    __device__ __forceinline__ float chunk(int m, int n0, const float acc[16]) const
    {
        float yy[16], tt[16], g[16];
        load_f32x16(target + (size_t)m * ld + n0, tt);
        float loss = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            yy[i] = acc[i] + bias[n0 + i];
            const float d = n0 + i < n_valid ? yy[i] - tt[i] : 0.f;
            g[i] = grad_scale * d;
            loss += d * d * loss_scale;
        }
        store_f32x16(y + (size_t)m * ld + n0, yy);
        store_bf16x16(dy + (size_t)m * ld + n0, g);
#pragma unroll
        for (int i = 0; i < 16; ++i) dyT[(size_t)(n0 + i) * ldT + m] = __float2bfloat16_rn(g[i]);
        return loss;
    }
    __device__ __forceinline__ void finish(float loss) const
    {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(loss_acc, loss);
    }
};

// Input gradient of a hidden layer: dz_prev = bf16(acc silu'(z_prev)), row-major and transposed.
struct TrainEpiDx {
    const float* zprev;
    __nv_bfloat16* dz;
    __nv_bfloat16* dzT;
    int ld, ldT;
    __device__ __forceinline__ float chunk(int m, int n0, const float acc[16]) const
    {
        float zp[16], g[16];
        load_f32x16(zprev + (size_t)m * ld + n0, zp);
#pragma unroll
        for (int i = 0; i < 16; ++i) g[i] = acc[i] * silu_grad_train(zp[i]);
        store_bf16x16(dz + (size_t)m * ld + n0, g);
#pragma unroll
        for (int i = 0; i < 16; ++i) dzT[(size_t)(n0 + i) * ldT + m] = __float2bfloat16_rn(g[i]);
        return 0.f;
    }
    __device__ __forceinline__ void finish(float) const {}
};

// Weight gradient (split over K = the batch): g[m][n] (or g[n][m] when transposed) += acc,
// four columns per vector reduction in the row-major case.
struct TrainEpiGrad {
    float* g;
    int ld;
    bool transpose;
    __device__ __forceinline__ float chunk(int m, int n0, const float acc[16]) const
    {
        if (transpose) {
#pragma unroll
            for (int i = 0; i < 16; ++i) atomicAdd(g + (size_t)(n0 + i) * ld + m, acc[i]);
        } else {
            float4* row = reinterpret_cast<float4*>(g + (size_t)m * ld + n0);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                atomicAdd(row + i, make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]));
        }
        return 0.f;
    }
    __device__ __forceinline__ void finish(float) const {}
};

// out[c][r] = in[r][c] for a [rows x cols] bf16 matrix (32 x 32 tiles through shared memory).
__global__ void __launch_bounds__(256) transpose_bf16_kernel(const __nv_bfloat16* __restrict__ in,
                                                             __nv_bfloat16* __restrict__ out, int rows, int cols)
{
    __shared__ __nv_bfloat16 tile[32][34];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < 32; i += 8)
        if (r0 + i < rows && c0 + tx < cols) tile[i][tx] = in[(size_t)(r0 + i) * cols + c0 + tx];
    __syncthreads();
    for (int i = ty; i < 32; i += 8)
        if (c0 + i < cols && r0 + tx < rows) out[(size_t)(c0 + i) * rows + r0 + tx] = tile[tx][i];
}

// One thread per 16-byte piece (8 consecutive k of one row n) of every weight matrix.
__global__ void build_image_kernel(const __nv_bfloat16* __restrict__ w16, MlpView w, uint8_t* __restrict__ img)
{
    const int dims[5] = {MDG_MLP_IN_PAD, MDG_MLP_HIDDEN, MDG_MLP_HIDDEN, MDG_MLP_HIDDEN, MDG_MLP_OUT_PAD};
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    for (int l = 0; l < 4; ++l) {
        const int K = dims[l], N = dims[l + 1], pieces = N * K / 8;
        if (i < pieces) {
            const int n = i / (K / 8), k8 = i % (K / 8);
            const int c = k8 >> 3, kk8 = k8 & 7;
            const uint32_t off = image_layer_base(l) + (uint32_t)c * N * 128 + n * 128 + ((kk8 ^ (n & 7)) << 4);
            *reinterpret_cast<uint4*>(img + off) =
                *reinterpret_cast<const uint4*>(w16 + w.w_off[l] + (size_t)n * K + k8 * 8);
            return;
        }
        i -= pieces;
    }
}

}  // namespace

constexpr size_t kUmmaSmem = 1024 + kDynBytes;

constexpr size_t kUmmaPairSmem = 1024 + kPDynBytes;

size_t mlp_image_bytes() { return kImgBytes; }

cudaError_t mlp_build_image(const MlpView& w, void* img, cudaStream_t s)
{
    const int pieces = (int)(kImgBytes / 16);
    build_image_kernel<<<(pieces + 255) / 256, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(w.w16), w,
                                                             static_cast<uint8_t*>(img));
    return cudaGetLastError();
}

namespace {
// cuTensorMapEncodeTiled, looked up through the runtime (no link against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}
}  // namespace

cudaError_t mlp_forward_umma_pairs(const MlpView& w, const void* img, const void* x, int B, float* y,
                                   uint32_t* status, int wait_limit, int spin_limit, cudaStream_t s,
                                   const MlpApply* apply)
{
    if (B % kRows) return cudaErrorInvalidValue;
    const int n_tiles = B / kRows;
    if (n_tiles == 0) return cudaSuccess;
    if (reinterpret_cast<uintptr_t>(x) % 16) return cudaErrorMisalignedAddress;  // TMA source
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_done[dev]) {
        e = cudaFuncSetAttribute(mlp_umma_pair_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kUmmaPairSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(mlp_umma_pair_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kUmmaPairSmem);
        if (e != cudaSuccess) return e;
        attr_done[dev] = true;
    }
    const EncodeTiledFn encode = encode_tiled();
    if (!encode) return cudaErrorNotSupported;
    // the inputs [B x 64] bf16, row-major: boxes of one tile (128 rows x 128 bytes), 128-byte swizzle
    CUtensorMap xmap;
    const cuuint64_t dims[2] = {MDG_MLP_IN_PAD, (cuuint64_t)B};
    const cuuint64_t strides[1] = {MDG_MLP_IN_PAD * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {MDG_MLP_IN_PAD, kRows};
    const cuuint32_t elem_strides[2] = {1, 1};
    if (encode(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(x), dims, strides, box, elem_strides,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    int n_sm = 152;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int n_pairs = (n_tiles + 1) / 2;
    const int grid = n_pairs < n_sm ? n_pairs : n_sm;
    const MlpApply ap = apply ? *apply : MlpApply{};
    if (apply)
        mlp_umma_pair_kernel<true><<<grid, kThreads, kUmmaPairSmem, s>>>(
            xmap, y, n_tiles, static_cast<const uint8_t*>(img), w.master, w, status, wait_limit, spin_limit, ap);
    else
        mlp_umma_pair_kernel<false><<<grid, kThreads, kUmmaPairSmem, s>>>(
            xmap, y, n_tiles, static_cast<const uint8_t*>(img), w.master, w, status, wait_limit, spin_limit, ap);
    return cudaGetLastError();
}

cudaError_t mlp_forward_umma(const MlpView& w, const void* img, const void* x, int B, float* y, uint32_t* status,
                             int wait_limit, int spin_limit, cudaStream_t s)
{
    if (B % kRows) return cudaErrorInvalidValue;
    const int n_tiles = B / kRows;
    if (n_tiles == 0) return cudaSuccess;
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_done[dev]) {
        e = cudaFuncSetAttribute(mlp_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUmmaSmem);
        if (e != cudaSuccess) return e;
        attr_done[dev] = true;
    }
    int n_sm = 152;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = n_tiles < n_sm ? n_tiles : n_sm;
    mlp_umma_kernel<<<grid, kThreads, kUmmaSmem, s>>>(static_cast<const __nv_bfloat16*>(x), y, n_tiles,
                                                      static_cast<const uint8_t*>(img), w.master, w, status,
                                                      wait_limit, spin_limit);
    return cudaGetLastError();
}

template <int BN, class Epi>
static cudaError_t umma_gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                             int splits, Epi epi, uint32_t* status, cudaStream_t s)
{
    if (M % 128 || N % BN || K % 32 || K <= 0 || splits < 1) return cudaErrorInvalidValue;
    using S = GemmShape<BN>;
    static bool attr_done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_done[dev]) {
        e = cudaFuncSetAttribute(umma_gemm_kernel<BN, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
        if (e != cudaSuccess) return e;
        attr_done[dev] = true;
    }
    // K per split: whole 64-wide chunks
    const int chunks = (K + 63) / 64;
    const int per = (chunks + splits - 1) / splits;
    splits = (chunks + per - 1) / per;
    dim3 grid(N / BN, M / 128, splits);
    umma_gemm_kernel<BN, Epi><<<grid, kGemmThreads, S::smem, s>>>(reinterpret_cast<const __nv_bfloat16*>(A), lda,
                                                                  reinterpret_cast<const __nv_bfloat16*>(B), ldb, K,
                                                                  per * 64, epi, status);
    return cudaGetLastError();
}

static cudaError_t transpose_bf16(const void* in, void* out, int rows, int cols, cudaStream_t s)
{
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    transpose_bf16_kernel<<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(in), static_cast<__nv_bfloat16*>(out),
                                               rows, cols);
    return cudaGetLastError();
}

cudaError_t mlp_weights_transposed(const MlpView& w, void* wT, cudaStream_t s)
{
    // W2^T, W3^T [256 x 256] and W4^T [256 x 32] (the B operands of the input gradients)
    const __nv_bfloat16* w16 = static_cast<const __nv_bfloat16*>(w.w16);
    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(wT);
    cudaError_t e = transpose_bf16(w16 + w.w_off[1], o, MDG_MLP_HIDDEN, MDG_MLP_HIDDEN, s);
    if (e == cudaSuccess) e = transpose_bf16(w16 + w.w_off[2], o + MDG_MLP_HIDDEN * MDG_MLP_HIDDEN, MDG_MLP_HIDDEN,
                                             MDG_MLP_HIDDEN, s);
    if (e == cudaSuccess) e = transpose_bf16(w16 + w.w_off[3], o + 2 * MDG_MLP_HIDDEN * MDG_MLP_HIDDEN,
                                             MDG_MLP_OUT_PAD, MDG_MLP_HIDDEN, s);
    return e;
}

size_t mlp_weights_transposed_elems() { return 2 * MDG_MLP_HIDDEN * MDG_MLP_HIDDEN + MDG_MLP_HIDDEN * MDG_MLP_OUT_PAD; }

cudaError_t mlp_grad_umma(const MlpView& w, const TrainBuffers& t, const void* x, int B, const float* target,
                          float* loss_acc, float* grad, uint32_t* status, cudaStream_t s)
{
    const int H = MDG_MLP_HIDDEN, I = MDG_MLP_IN_PAD, O = MDG_MLP_OUT_PAD;
    const __nv_bfloat16* w16 = static_cast<const __nv_bfloat16*>(w.w16);
    const __nv_bfloat16* xin = static_cast<const __nv_bfloat16*>(x);
    const __nv_bfloat16* wT = static_cast<const __nv_bfloat16*>(t.wT);
    auto bf = [](void* p) { return static_cast<__nv_bfloat16*>(p); };
    // the weight gradients are split over the batch and added up with atomics
    const int splits = B / 256 > 0 ? B / 256 : 1;
    cudaError_t e = cudaMemsetAsync(grad, 0, (size_t)MDG_MLP_PARAMS * 4, s);
    if (e == cudaSuccess) e = transpose_bf16(x, t.xT, B, I, s);
    // forward
    const __nv_bfloat16* in = xin;
    int fan_in = I;
    for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
        TrainEpiHidden ep{w.master + w.b_off[l], t.z[l], bf(t.h[l]), bf(t.hT[l]), H, B};
        e = umma_gemm<128>(in, fan_in, w16 + w.w_off[l], fan_in, B, H, fan_in, 1, ep, status, s);
        in = bf(t.h[l]);
        fan_in = H;
    }
    if (e == cudaSuccess) {
        TrainEpiOut eo{w.master + w.b_off[3], t.y, target, bf(t.dy), bf(t.dyT), loss_acc, O, B, MDG_MLP_OUT,
                       2.f / ((float)B * MDG_MLP_OUT), 1.f / ((float)B * MDG_MLP_OUT)};
        e = umma_gemm<32>(in, H, w16 + w.w_off[3], H, B, O, H, 1, eo, status, s);
    }
    // backward: output layer (dW4 as its transpose [256 x 32] = H3^T dY)
    if (e == cudaSuccess) {
        TrainEpiGrad eg{grad + w.w_off[3], H, true};
        e = umma_gemm<32>(bf(t.hT[2]), B, bf(t.dyT), B, H, O, B, splits, eg, status, s);
    }
    if (e == cudaSuccess) e = mlp_bias_grad(t.dy, B, O, grad + w.b_off[3], s);
    if (e == cudaSuccess) {  // dH3 = dY W4 (K = 32) -> dZ3
        TrainEpiDx ex{t.z[2], bf(t.dz[2]), bf(t.dzT[2]), H, B};
        e = umma_gemm<128>(bf(t.dy), O, wT + 2 * H * H, O, B, H, O, 1, ex, status, s);
    }
    // hidden layers l = 2, 1, 0 (weights W3, W2, W1)
    for (int l = 2; l >= 0 && e == cudaSuccess; --l) {
        const int fi = l == 0 ? I : H;
        const __nv_bfloat16* inT = l == 0 ? bf(t.xT) : bf(t.hT[l - 1]);
        TrainEpiGrad eg{grad + w.w_off[l], fi, false};
        if (fi == H) e = umma_gemm<128>(bf(t.dzT[l]), B, inT, B, H, fi, B, splits, eg, status, s);
        else e = umma_gemm<64>(bf(t.dzT[l]), B, inT, B, H, fi, B, splits, eg, status, s);
        if (e == cudaSuccess) e = mlp_bias_grad(t.dz[l], B, H, grad + w.b_off[l], s);
        if (e == cudaSuccess && l > 0) {  // dH_{l-1} = dZ_l W_l -> dZ_{l-1}
            TrainEpiDx ex{t.z[l - 1], bf(t.dz[l - 1]), bf(t.dzT[l - 1]), H, B};
            e = umma_gemm<128>(bf(t.dz[l]), H, wT + (size_t)(l - 1) * H * H, H, B, H, H, 1, ex, status, s);
        }
    }
    return e;
}

}  // namespace mdg
