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
constexpr int kSpinLimit = MDG_MLP_DEFAULT_POLLS;      // polls of a spinning wait (a few tenths of a second)

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

size_t mlp_image_bytes() { return kImgBytes; }

cudaError_t mlp_build_image(const MlpView& w, void* img, cudaStream_t s)
{
    const int pieces = (int)(kImgBytes / 16);
    build_image_kernel<<<(pieces + 255) / 256, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(w.w16), w,
                                                             static_cast<uint8_t*>(img));
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

}  // namespace mdg
