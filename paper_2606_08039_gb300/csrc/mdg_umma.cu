// Fused inference of the surrogate network on the 5th-generation tensor cores (sm_103a):
// tcgen05.mma with the accumulator in tensor memory, operands in shared memory.
//
// One persistent thread block (16 warps) per SM takes 128-row tiles of drones. For each of
// the four layers one thread issues the K/16 tcgen05.mma instructions (M = 128, N = 256 or
// 32, bf16 x bf16 -> FP32 in TMEM) on the shared-memory activations and weights and commits
// them to an mbarrier; once they complete, the copy of the next operands (the next layer's
// weights, or the next tile's inputs and first-layer weights) is issued, and meanwhile the
// warps read the accumulator back with tcgen05.ld, add the bias, apply SiLU and write the
// bf16 activations into the shared-memory operand of the next layer (the output layer's
// FP32 values go to global memory). Activations never leave the SM.
//
// Shared-memory operands use the canonical K-major layout with 128-byte swizzling: a
// [rows x K] bf16 matrix is stored as K/64 chunks of rows x 128 bytes; within a chunk row r
// starts at r * 128 and its 16-byte pieces are permuted by XOR with (r mod 8). Each chunk
// starts on a 1024-byte boundary. Every wait on the mbarrier is bounded: on expiry the
// block records MDG_STATUS_TIMEOUT in the status word, releases its tensor memory and
// returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "mdg.h"
#include "mdg_internal.cuh"

namespace mdg {
namespace {

constexpr int kRows = 128;         // tile rows (UMMA M)
constexpr int kThreads = 512;      // 16 warps: four per TMEM lane quadrant, 64 columns each
constexpr int kActBytes = 128 * 256 * 2;   // activations [128 x 256] bf16
constexpr int kWBytes = 256 * 256 * 2;     // largest weight matrix [256 x 256] bf16
constexpr uint32_t kTmemCols = 256;
constexpr int kWaitLimit = 1 << 22;        // mbarrier polls (with 64 ns back-off: ~0.3 s) before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(uint32_t s, const void* g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g));
}

// byte offset of the 16-byte piece (row r, piece k8) of a [rows x K] K-major SW128 matrix
__device__ __forceinline__ uint32_t sw128_offset(int r, int k8, int rows)
{
    const int chunk = k8 >> 3, piece = k8 & 7;
    return (uint32_t)(chunk * rows * 128 + r * 128 + ((piece ^ (r & 7)) << 4));
}

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

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase)
{
    for (int i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
        __nanosleep(64);
    }
    return false;
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Issue the copy of a row-major [rows x K] bf16 matrix (K contiguous) into the SW128
// K-major layout (cp.async, one commit group); cp_wait() completes it.
__device__ __forceinline__ void stage_async(uint32_t s_base, const __nv_bfloat16* g, int rows, int K)
{
    const int pieces = rows * (K >> 3);
    for (int i = threadIdx.x; i < pieces; i += kThreads) {
        const int r = i / (K >> 3), k8 = i % (K >> 3);
        cp_async16(s_base + sw128_offset(r, k8, rows), g + (size_t)r * K + k8 * 8);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// SiLU(z) = z / (1 + exp(-z)) = z/2 (1 + tanh(z/2)): one special-function instruction
// (tanh.approx.f32, relative error about 2^-11) instead of an exponential and a division.
__device__ __forceinline__ float silu_tanh(float z)
{
    const float h = 0.5f * z;
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
    return fmaf(h, t, h);
}

__device__ __forceinline__ void make_operands_visible()
{
    // generic-proxy shared-memory writes (cp.async, st.shared) -> async proxy (tcgen05.mma)
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
    mlp_umma_kernel(const __nv_bfloat16* __restrict__ x, float* __restrict__ y, int n_tiles, const float* __restrict__ master,
                    const __nv_bfloat16* __restrict__ w16, MlpView w, uint32_t* status)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte aligned operand buffers
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* s_act = base;
    uint8_t* s_w = base + kActBytes;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_tmem;
    __shared__ float s_bias[3 * MDG_MLP_HIDDEN + MDG_MLP_OUT_PAD];  // b1, b2, b3, b4

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t mbar_a = smem_u32(&mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_a));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    for (int i = threadIdx.x; i < 3 * MDG_MLP_HIDDEN + MDG_MLP_OUT_PAD; i += kThreads) {
        const int l = i < 3 * MDG_MLP_HIDDEN ? i / MDG_MLP_HIDDEN : 3;
        s_bias[i] = master[w.b_off[l] + (i - l * MDG_MLP_HIDDEN)];
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t act_a = smem_u32(s_act), w_a = smem_u32(s_w);
    const int quad = warp & 3, part = warp >> 2;  // TMEM lane quadrant, column quarter
    const int row = quad * 32 + lane;  // this thread's accumulator row (TMEM lane)
    const uint32_t t_row = tmem + ((uint32_t)(quad * 32) << 16);
    const int dims[5] = {MDG_MLP_IN_PAD, MDG_MLP_HIDDEN, MDG_MLP_HIDDEN, MDG_MLP_HIDDEN, MDG_MLP_OUT_PAD};
    uint32_t phase = 0;
    bool abort = false;  // identical in every thread (set from __syncthreads_and)

    // the first tile's inputs and first-layer weights
    if (blockIdx.x < n_tiles) {
        stage_async(act_a, x + (size_t)blockIdx.x * kRows * MDG_MLP_IN_PAD, kRows, MDG_MLP_IN_PAD);
        stage_async(w_a, w16 + w.w_off[0], dims[1], dims[0]);
    }
    for (int tile = blockIdx.x; tile < n_tiles && !abort; tile += gridDim.x) {
        for (int l = 0; l < 4; ++l) {
            const int K = dims[l], N = dims[l + 1];
            cp_wait();  // this layer's weights (and, for l = 0, the tile's inputs) have landed
            make_operands_visible();
            if (threadIdx.x == 0) {
                const uint32_t idesc = idesc_bf16(kRows, N);
                for (int k16 = 0; k16 < K / 16; ++k16) {
                    const int chunk = k16 >> 2, within = (k16 & 3) * 32;
                    const uint64_t ad = sw128_desc(act_a + chunk * kRows * 128 + within);
                    const uint64_t bd = sw128_desc(w_a + chunk * N * 128 + within);
                    mma_bf16_ss(tmem, ad, bd, idesc, k16 > 0);
                }
                mma_commit(mbar_a);
            }
            const bool ok = mbar_wait(mbar_a, phase);
            phase ^= 1;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (!__syncthreads_and(ok)) {
                if (threadIdx.x == 0) atomicOr(status, MDG_STATUS_TIMEOUT);
                abort = true;
                break;
            }
            // The MMAs have consumed their operands: start the next copies now so that they
            // overlap this layer's epilogue (the next layer's weights, or after the last layer
            // the next tile's inputs and first-layer weights).
            if (l < 3) {
                stage_async(w_a, w16 + w.w_off[l + 1], dims[l + 2], dims[l + 1]);
            } else if (tile + (int)gridDim.x < n_tiles) {
                stage_async(act_a, x + (size_t)(tile + gridDim.x) * kRows * MDG_MLP_IN_PAD, kRows, MDG_MLP_IN_PAD);
                stage_async(w_a, w16 + w.w_off[0], dims[1], dims[0]);
            }
            const float* bias = s_bias + l * MDG_MLP_HIDDEN;
            if (l < 3) {
                // bias + SiLU -> bf16 activations, this warp's quarter of the 256 columns
#pragma unroll 1
                for (int c0 = part * 64; c0 < part * 64 + 64; c0 += 32) {
                    float v[32];
                    tmem_ld32(t_row + c0, v);
                    __nv_bfloat162 o[16];
#pragma unroll
                    for (int i = 0; i < 32; i += 2)
                        o[i / 2] = __floats2bfloat162_rn(silu_tanh(v[i] + bias[c0 + i]),
                                                         silu_tanh(v[i + 1] + bias[c0 + i + 1]));
                    const uint4* o4 = reinterpret_cast<const uint4*>(o);
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const uint32_t off = sw128_offset(row, (c0 >> 3) + p, kRows);
                        *reinterpret_cast<uint4*>(s_act + off) = o4[p];
                    }
                }
            } else if (part == 0) {
                float v[32];
                tmem_ld32(t_row, v);
                float4* out = reinterpret_cast<float4*>(y + ((size_t)tile * kRows + row) * MDG_MLP_OUT_PAD);
#pragma unroll
                for (int i = 0; i < 32; i += 4)
                    out[i / 4] = make_float4(v[i] + bias[i], v[i + 1] + bias[i + 1], v[i + 2] + bias[i + 2],
                                             v[i + 3] + bias[i + 3]);
            }
            // all tensor-memory reads and activation writes done before the next MMA
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();
        }
    }
    cp_wait();  // no copy left in flight
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace

constexpr size_t kUmmaSmem = 1024 + kActBytes + kWBytes;

cudaError_t mlp_forward_umma(const MlpView& w, const void* x, int B, float* y, uint32_t* status, cudaStream_t s)
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
    mlp_umma_kernel<<<grid, kThreads, kUmmaSmem, s>>>(static_cast<const __nv_bfloat16*>(x), y, n_tiles, w.master,
                                                      static_cast<const __nv_bfloat16*>(w.w16), w, status);
    return cudaGetLastError();
}

}  // namespace mdg
