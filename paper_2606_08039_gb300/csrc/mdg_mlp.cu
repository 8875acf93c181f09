// BF16 tensor-core kernels of the learned surrogate: a tiled GEMM on mma.sync
// m16n8k16 (FP32 accumulation) with fused epilogues for the forward pass, the input
// gradient and the weight gradient, the bias-gradient reduction, Adam, and the input
// standardisation. The network is 64 -> 256 -> 256 -> 256 -> 32 (41 inputs and 13 outputs
// used, zero padded), SiLU on the hidden layers.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include "mdg.h"
#include "mdg_internal.cuh"

namespace mdg {
namespace {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z)
{
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(unsigned r[4], const void* smem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}
__device__ __forceinline__ void ldmatrix_x4_trans(unsigned r[4], const void* smem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(s));
}

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---- epilogues: called with (row m, column n, value) for every element of C ----

struct EpiHidden {  // z = acc + b[n]; h = bf16(silu(z)); z kept (FP32) for backward when non-null
    const float* bias;
    float* z;
    bf16* h;
    int ld;
    __device__ __forceinline__ void operator()(int m, int n, float acc) const
    {
        const float zz = acc + bias[n];
        if (z) z[(size_t)m * ld + n] = zz;
        h[(size_t)m * ld + n] = __float2bfloat16_rn(silu_f(zz));
    }
};

struct EpiOut {  // y = acc + b[n]; with targets: dy = scale (y - t) on valid columns, loss += (y - t)^2 / (rows * valid)
    const float* bias;
    float* y;
    int ld;
    const float* target;
    bf16* dy;
    float* loss_acc;
    int n_valid;
    float grad_scale;
    float loss_scale;
    __device__ __forceinline__ float operator()(int m, int n, float acc) const
    {
        const float yy = acc + bias[n];
        if (y) y[(size_t)m * ld + n] = yy;
        if (!target) return 0.f;
        const float d = n < n_valid ? yy - target[(size_t)m * ld + n] : 0.f;
        dy[(size_t)m * ld + n] = __float2bfloat16_rn(grad_scale * d);
        return d * d * loss_scale;
    }
};

struct EpiDx {  // dz_prev = bf16(acc * silu'(z_prev))
    const float* zprev;
    bf16* dz;
    int ld;
    __device__ __forceinline__ void operator()(int m, int n, float acc) const
    {
        dz[(size_t)m * ld + n] = __float2bfloat16_rn(acc * silu_grad_f(zprev[(size_t)m * ld + n]));
    }
};

struct EpiGrad {  // gradient store, optionally transposed
    float* g;
    int ld;
    bool transpose;
    __device__ __forceinline__ void operator()(int m, int n, float acc) const
    {
        if (transpose) g[(size_t)n * ld + m] = acc;
        else g[(size_t)m * ld + n] = acc;
    }
};

template <class E>
struct EpiReturnsLoss {
    static constexpr bool value = false;
};
template <>
struct EpiReturnsLoss<EpiOut> {
    static constexpr bool value = true;
};

// C[M x N] = op(A)[M x K] op(B)[K x N], bf16 inputs, FP32 accumulation.
//   A: kAT = false: A[m][k] at A + m lda + k;  kAT = true: stored [k][m] at A + k lda + m
//   B: kBT = false: B[k][n] = W[n][k] at B + n ldb + k;  kBT = true: stored [k][n] at B + k ldb + n
// Requires M % 128 == 0, N % BN == 0, K % 32 == 0, 16-byte aligned rows (lda, ldb % 8 == 0).
// 128 threads (4 warps), tile 128 x BN x 32, cp.async double buffering, ldmatrix(.trans).
template <int BN, bool kAT, bool kBT, class Epi>
__global__ void __launch_bounds__(128) gemm_kernel(const bf16* __restrict__ A, int lda, const bf16* __restrict__ B,
                                                   int ldb, int M, int N, int K, Epi epi)
{
    constexpr int BM = 128, BK = 32;
    constexpr int WARPS_N = BN / 32, WARPS_M = 4 / WARPS_N;
    constexpr int WM = BM / WARPS_M, WN = BN / WARPS_N;
    constexpr int MT = WM / 16, NT = WN / 8;
    constexpr int A_ROWS = kAT ? BK : BM, A_COLS = kAT ? BM : BK;
    constexpr int B_ROWS = kBT ? BK : BN, B_COLS = kBT ? BN : BK;
    constexpr int A_LD = A_COLS + 8, B_LD = B_COLS + 8;  // padded rows: conflict-free ldmatrix
    __shared__ __align__(16) bf16 sA[2][A_ROWS * A_LD];
    __shared__ __align__(16) bf16 sB[2][B_ROWS * B_LD];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp / WARPS_N, wn = warp % WARPS_N;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

    auto load_tile = [&](int buf, int k0) {
        // A tile
        for (int c = tid; c < A_ROWS * A_COLS / 8; c += 128) {
            const int r = c / (A_COLS / 8), cc = (c % (A_COLS / 8)) * 8;
            const bf16* g = kAT ? A + (size_t)(k0 + r) * lda + m0 + cc : A + (size_t)(m0 + r) * lda + k0 + cc;
            cp_async16(&sA[buf][r * A_LD + cc], g);
        }
        for (int c = tid; c < B_ROWS * B_COLS / 8; c += 128) {
            const int r = c / (B_COLS / 8), cc = (c % (B_COLS / 8)) * 8;
            const bf16* g = kBT ? B + (size_t)(k0 + r) * ldb + n0 + cc : B + (size_t)(n0 + r) * ldb + k0 + cc;
            cp_async16(&sB[buf][r * B_LD + cc], g);
        }
        cp_async_commit();
    };

    float acc[MT][NT][4];
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

    const int k_tiles = K / BK;
    load_tile(0, 0);
    for (int kt = 0; kt < k_tiles; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < k_tiles) {
            load_tile(buf ^ 1, (kt + 1) * BK);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const bf16* a_s = sA[buf];
        const bf16* b_s = sB[buf];
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[MT][4];
#pragma unroll
            for (int i = 0; i < MT; ++i) {
                const int mb = wm * WM + i * 16;
                const int mat = lane >> 3, r = lane & 7;
                if (!kAT) {
                    const int row = mb + (mat & 1) * 8 + r, col = kk + (mat >> 1) * 8;
                    ldmatrix_x4(af[i], &a_s[row * A_LD + col]);
                } else {
                    const int row = kk + (mat >> 1) * 8 + r, col = mb + (mat & 1) * 8;
                    ldmatrix_x4_trans(af[i], &a_s[row * A_LD + col]);
                }
            }
#pragma unroll
            for (int j = 0; j < NT; j += 2) {
                const int nb = wn * WN + j * 8;
                const int mat = lane >> 3, r = lane & 7;
                unsigned bfr[4];
                if (!kBT) {
                    const int row = nb + (mat >> 1) * 8 + r, col = kk + (mat & 1) * 8;
                    ldmatrix_x4(bfr, &b_s[row * B_LD + col]);
                } else {
                    const int row = kk + (mat & 1) * 8 + r, col = nb + (mat >> 1) * 8;
                    ldmatrix_x4_trans(bfr, &b_s[row * B_LD + col]);
                }
#pragma unroll
                for (int i = 0; i < MT; ++i) {
                    mma_bf16(acc[i][j], af[i], bfr[0], bfr[1]);
                    mma_bf16(acc[i][j + 1], af[i], bfr[2], bfr[3]);
                }
            }
        }
        __syncthreads();
    }

    // epilogue: c0,c1 at (row g, cols 2q, 2q+1), c2,c3 at (row g + 8, same cols)
    const int g = lane >> 2, q = lane & 3;
    float loss = 0.f;
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const int m = m0 + wm * WM + i * 16 + g, n = n0 + wn * WN + j * 8 + 2 * q;
            if constexpr (EpiReturnsLoss<Epi>::value) {
                loss += epi(m, n, acc[i][j][0]) + epi(m, n + 1, acc[i][j][1]) + epi(m + 8, n, acc[i][j][2]) +
                        epi(m + 8, n + 1, acc[i][j][3]);
            } else {
                epi(m, n, acc[i][j][0]);
                epi(m, n + 1, acc[i][j][1]);
                epi(m + 8, n, acc[i][j][2]);
                epi(m + 8, n + 1, acc[i][j][3]);
            }
        }
    if constexpr (EpiReturnsLoss<Epi>::value) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
        if (lane == 0 && epi.loss_acc) atomicAdd(epi.loss_acc, loss);
    }
}

template <int BN, bool kAT, bool kBT, class Epi>
cudaError_t gemm(const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, Epi epi, cudaStream_t s)
{
    if (M % 128 || N % BN || K % 32) return cudaErrorInvalidValue;
    dim3 grid(N / BN, M / 128);
    gemm_kernel<BN, kAT, kBT, Epi><<<grid, 128, 0, s>>>(A, lda, B, ldb, M, N, K, epi);
    return cudaGetLastError();
}

// db[n] = sum over rows of dz[m][n] (bf16 input, FP32 sums): one block per 64 columns and 256
// rows (each lane two adjacent columns, eight warps over the rows), its partial sums added to
// db (zeroed by the launcher) with atomics, so that a batch of 8192 rows spreads over 32 x N/64
// blocks instead of N/32.
constexpr int kBiasRows = 256;
__global__ void __launch_bounds__(256) bias_grad_kernel(const bf16* __restrict__ dz, int M, int N, float* db)
{
    __shared__ float2 part[8][32];
    const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
    const int n = blockIdx.x * 64 + 2 * x;
    const int m0 = blockIdx.y * kBiasRows, m1 = min(M, m0 + kBiasRows);
    float2 acc = make_float2(0.f, 0.f);
    if (n < N)
        for (int m = m0 + y; m < m1; m += 8) {
            const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(dz + (size_t)m * N + n));
            acc.x += v.x;
            acc.y += v.y;
        }
    part[y][x] = acc;
    __syncthreads();
    if (y == 0 && n < N) {
        float2 t = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 8; ++k) t.x += part[k][x].x, t.y += part[k][x].y;
        atomicAdd(db + n, t.x);
        atomicAdd(db + n + 1, t.y);
    }
}

// Adam (Kingma and Ba) on the flat FP32 master parameters; refreshes their bf16 copies.
__global__ void adam_kernel(float* __restrict__ w, bf16* __restrict__ w16, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        w16[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ w, bf16* __restrict__ w16, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        w16[i] = __float2bfloat16_rn(w[i]);
}

// x[r][k] = bf16((raw[r][k] - mean[k]) / std[k]) for k < 41, 0 for the padding up to 64.
__global__ void standardize_kernel(const float* __restrict__ raw, bf16* __restrict__ x, long long rows,
                                   const float* __restrict__ mean, const float* __restrict__ inv_std)
{
    const long long total = rows * MDG_MLP_IN_PAD;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / MDG_MLP_IN_PAD;
        const int k = (int)(i % MDG_MLP_IN_PAD);
        const float val = k < MDG_MLP_IN ? (raw[r * MDG_MLP_IN + k] - mean[k]) * inv_std[k] : 0.f;
        x[i] = __float2bfloat16_rn(val);
    }
}

}  // namespace

// ---- host-side launchers (declared in mdg_internal.cuh) ----

cudaError_t mlp_forward(const MlpView& w, const void* x, int B, float* z_hidden[3], void* h_hidden[3], float* y,
                        const float* target, void* dy, float* loss_acc, cudaStream_t s)
{
    const bf16* in = static_cast<const bf16*>(x);
    const bf16* w16 = static_cast<const bf16*>(w.w16);
    cudaError_t e;
    const int dims[5] = {MDG_MLP_IN_PAD, MDG_MLP_HIDDEN, MDG_MLP_HIDDEN, MDG_MLP_HIDDEN, MDG_MLP_OUT_PAD};
    for (int l = 0; l < 3; ++l) {
        EpiHidden epi{w.master + w.b_off[l], z_hidden[l], static_cast<bf16*>(h_hidden[l]), MDG_MLP_HIDDEN};
        e = gemm<64, false, false>(in, dims[l], w16 + w.w_off[l], dims[l], B, MDG_MLP_HIDDEN, dims[l], epi, s);
        if (e != cudaSuccess) return e;
        in = static_cast<const bf16*>(h_hidden[l]);
    }
    EpiOut epo{w.master + w.b_off[3], y, MDG_MLP_OUT_PAD, target, static_cast<bf16*>(dy), loss_acc, MDG_MLP_OUT,
               2.f / ((float)B * MDG_MLP_OUT), 1.f / ((float)B * MDG_MLP_OUT)};
    return gemm<32, false, false>(in, MDG_MLP_HIDDEN, w16 + w.w_off[3], MDG_MLP_HIDDEN, B, MDG_MLP_OUT_PAD,
                                  MDG_MLP_HIDDEN, epo, s);
}

cudaError_t mlp_backward(const MlpView& w, const void* x, int B, float* const z_hidden[3], void* const h_hidden[3],
                         void* dy, void* dz_hidden[3], float* grad, cudaStream_t s)
{
    const bf16* w16 = static_cast<const bf16*>(w.w16);
    const int dims[5] = {MDG_MLP_IN_PAD, MDG_MLP_HIDDEN, MDG_MLP_HIDDEN, MDG_MLP_HIDDEN, MDG_MLP_OUT_PAD};
    cudaError_t e;
    // output layer: dW4^T [256 x 32] = H3^T dY, db4, dH3 = dY W4 -> dZ3
    const bf16* dcur = static_cast<const bf16*>(dy);
    for (int l = 3; l >= 0; --l) {
        const bf16* hin = l == 0 ? static_cast<const bf16*>(x) : static_cast<const bf16*>(h_hidden[l - 1]);
        const int fan_in = dims[l], fan_out = dims[l + 1];
        if (l == 3) {  // transposed: M = fan_in (256), N = fan_out (32)
            EpiGrad eg{grad + w.w_off[3], fan_in, true};
            e = gemm<32, true, true>(hin, fan_in, dcur, fan_out, fan_in, fan_out, B, eg, s);
        } else {  // M = fan_out (256), N = fan_in (64 or 256)
            EpiGrad eg{grad + w.w_off[l], fan_in, false};
            e = gemm<64, true, true>(dcur, fan_out, hin, fan_in, fan_out, fan_in, B, eg, s);
        }
        if (e != cudaSuccess) return e;
        if ((e = mlp_bias_grad(dcur, B, fan_out, grad + w.b_off[l], s)) != cudaSuccess) return e;
        if (l > 0) {  // dH_{l-1} = dZ_l W_l (W_l stored [fan_out][fan_in] = [K][N]) -> dZ_{l-1}
            EpiDx ex{z_hidden[l - 1], static_cast<bf16*>(dz_hidden[l - 1]), fan_in};
            e = gemm<64, false, true>(dcur, fan_out, w16 + w.w_off[l], fan_in, B, fan_in, fan_out, ex, s);
            if (e != cudaSuccess) return e;
            dcur = static_cast<const bf16*>(dz_hidden[l - 1]);
        }
    }
    return cudaSuccess;
}

cudaError_t mlp_adam(const MlpView& w, const float* grad, float* m, float* v, float lr, int step, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<152 * 4, 256, 0, s>>>(w.master, static_cast<bf16*>(w.w16), grad, m, v, MDG_MLP_PARAMS, lr, b1, b2,
                                        eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t mlp_refresh_bf16(const MlpView& w, cudaStream_t s)
{
    to_bf16_kernel<<<152 * 4, 256, 0, s>>>(w.master, static_cast<bf16*>(w.w16), MDG_MLP_PARAMS);
    return cudaGetLastError();
}

cudaError_t mlp_bias_grad(const void* dz, int M, int N, float* db, cudaStream_t s)
{
    if (N % 2) return cudaErrorInvalidValue;  // the layer widths (256, 32) are even
    cudaError_t e = cudaMemsetAsync(db, 0, (size_t)N * sizeof(float), s);
    if (e != cudaSuccess || M == 0) return e;
    const dim3 grid((N + 63) / 64, (M + kBiasRows - 1) / kBiasRows);
    bias_grad_kernel<<<grid, 256, 0, s>>>(static_cast<const bf16*>(dz), M, N, db);
    return cudaGetLastError();
}

cudaError_t mlp_standardize(const float* raw, void* x, long long rows, const float* mean, const float* inv_std,
                            cudaStream_t s)
{
    if (rows == 0) return cudaSuccess;
    long long blocks = (rows * MDG_MLP_IN_PAD + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    standardize_kernel<<<(int)blocks, 256, 0, s>>>(raw, static_cast<bf16*>(x), rows, mean, inv_std);
    return cudaGetLastError();
}

}  // namespace mdg
