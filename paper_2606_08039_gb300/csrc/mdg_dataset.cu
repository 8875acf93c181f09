// Training data of the learned surrogate, built on the device: transitions of the plain
// integrator (the 41 network inputs of a state and its RPMs, the 13-d state change over one
// control step) and the standardisation of a set of transitions (the trimming of its tails,
// the mean and standard deviation of the kept set, the out-of-distribution box, and the
// standardised inputs and targets the training GEMMs read).
#include <cuda_bf16.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "mdg.h"
#include "mdg_internal.cuh"

namespace {

constexpr int kIn = MDG_MLP_IN, kOut = MDG_MLP_OUT, kCols = kIn + kOut;
constexpr int kScanBlock = 1024;  // elements per block of the stable compaction
constexpr int kSampleMax = 262144;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    mdg::set_last_error(buf);
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(MDG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// The 13-d state [p, q, v, w] of drone g from the state planes.
__device__ __forceinline__ void state13(const float4* S, long long n, long long g, float x[13])
{
    const float4 a = S[g], b = S[n + g], c = S[2 * n + g], d = S[3 * n + g];
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
    x[8] = c.x; x[9] = c.y; x[10] = c.z; x[11] = c.w;
    x[12] = d.x;
}

// Before the step: the applied RPMs (rpm times rpm_scale, when given) and delta = -x_before.
__global__ void transition_begin_kernel(const float4* __restrict__ S, long long n, const float4* __restrict__ rpm,
                                        const float4* __restrict__ scale, float4* __restrict__ applied,
                                        float* __restrict__ delta)
{
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
        float4 r = rpm[g];
        if (scale) {
            const float4 f = scale[g];
            r = make_float4(r.x * f.x, r.y * f.y, r.z * f.z, r.w * f.w);
        }
        applied[g] = r;
        float x[13];
        state13(S, n, g, x);
#pragma unroll
        for (int k = 0; k < 13; ++k) delta[13 * g + k] = -x[k];
    }
}

// After the step: delta += x_after.
__global__ void transition_end_kernel(const float4* __restrict__ S, long long n, float* __restrict__ delta)
{
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
        float x[13];
        state13(S, n, g, x);
#pragma unroll
        for (int k = 0; k < 13; ++k) delta[13 * g + k] += x[k];
    }
}

// Column c of row i of the transition set: the inputs, then the targets.
__device__ __forceinline__ float column(const float* raw, const float* delta, long long i, int c)
{
    return c < kIn ? raw[i * kIn + c] : delta[i * kOut + (c - kIn)];
}

// Keys that order floats as unsigned integers (finite values; -0 before +0).
__device__ __forceinline__ uint32_t float_key(float v)
{
    const uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float key_float(uint32_t k)
{
    const uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}

// flags[i] = 1 if every input and target of row i is finite.
__global__ void finite_kernel(const float* __restrict__ raw, const float* __restrict__ delta, long long N,
                              uint8_t* __restrict__ flags)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        bool ok = true;
        for (int c = 0; c < kCols; ++c) ok = ok && isfinite(column(raw, delta, i, c));
        flags[i] = ok ? 1 : 0;
    }
}

// Stable compaction of the rows whose flag is set: per block of kScanBlock rows its count,
// then (one block) the exclusive prefix sum of the counts, then every set row's index at its
// position. The order of the rows is kept.
__global__ void __launch_bounds__(kScanBlock) count_kernel(const uint8_t* __restrict__ flags, long long N,
                                                           int* __restrict__ counts)
{
    const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    const int f = i < N ? flags[i] : 0;
    const int c = __syncthreads_count(f);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

__global__ void __launch_bounds__(1024) scan_kernel(int* __restrict__ counts, int n_blocks, long long* __restrict__ total)
{
    __shared__ long long s_carry;
    __shared__ int s_part[1024];
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n_blocks; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < n_blocks ? counts[i] : 0;
        s_part[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan
            const int add = threadIdx.x >= o ? s_part[threadIdx.x - o] : 0;
            __syncthreads();
            s_part[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < n_blocks) counts[i] = (int)(s_carry + s_part[threadIdx.x] - v);  // exclusive
        __syncthreads();
        if (threadIdx.x == 1023) s_carry += s_part[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = s_carry;
}

__global__ void __launch_bounds__(kScanBlock) scatter_kernel(const uint8_t* __restrict__ flags, long long N,
                                                             const int* __restrict__ offsets, int* __restrict__ idx)
{
    __shared__ int s_warp[kScanBlock / 32];
    const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    const int f = i < N ? flags[i] : 0;
    const unsigned ballot = __ballot_sync(0xffffffffu, f);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_warp[warp] = __popc(ballot);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    if (f) idx[offsets[blockIdx.x] + before + __popc(ballot & ((1u << lane) - 1u))] = (int)i;
}

// Order statistics by bisection on the float keys: for every selection s (a column and a rank
// k_s among the sampled rows), [lo_s, hi_s] shrinks to the key of the (k_s + 1)-th smallest
// value. One pass counts, for every selection, the sampled values of its column with key <= the
// midpoint; the update halves the interval. 32 passes pin the key exactly.
struct Selections {
    int n;              // selections: kCols columns x 4 ranks
    int rank[kCols * 4];
};

__global__ void __launch_bounds__(256) select_count_kernel(const float* __restrict__ raw, const float* __restrict__ delta,
                                                           const int* __restrict__ rows, long long stride,
                                                           long long n_sample, const uint32_t* __restrict__ lo,
                                                           const uint32_t* __restrict__ hi, unsigned* __restrict__ count)
{
    __shared__ unsigned s_count[kCols * 4];
    __shared__ uint32_t s_mid[kCols * 4];
    for (int j = threadIdx.x; j < kCols * 4; j += blockDim.x) {
        s_count[j] = 0;
        s_mid[j] = lo[j] + (hi[j] - lo[j]) / 2;
    }
    __syncthreads();
    const long long total = n_sample * kCols;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long s = t / kCols;
        const int c = (int)(t % kCols);
        const long long r = rows[s * stride];
        const uint32_t key = float_key(column(raw, delta, r, c));
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (key <= s_mid[4 * c + q]) atomicAdd(&s_count[4 * c + q], 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kCols * 4; j += blockDim.x)
        if (s_count[j]) atomicAdd(&count[j], s_count[j]);
}

__global__ void select_update_kernel(Selections sel, uint32_t* lo, uint32_t* hi, unsigned* count)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= sel.n) return;
    const uint32_t mid = lo[j] + (hi[j] - lo[j]) / 2;
    if (count[j] >= (unsigned)sel.rank[j] + 1u) hi[j] = mid;
    else lo[j] = mid + 1u;
    count[j] = 0;
}

struct Stats {
    float box_lo[kCols], box_hi[kCols];  // the trim box of every column
    float mean[kCols], inv_std[kCols], std_[kCols];
    float ood_z, target_clip;
};

// keep1: finite and inside the trim box in every column.
__global__ void box_kernel(const float* __restrict__ raw, const float* __restrict__ delta, long long N,
                           const uint8_t* __restrict__ finite, const Stats* __restrict__ st, uint8_t* __restrict__ keep)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        bool ok = finite[i] != 0;
        for (int c = 0; c < kCols && ok; ++c) {
            const float v = column(raw, delta, i, c);
            ok = v >= st->box_lo[c] && v <= st->box_hi[c];
        }
        keep[i] = ok ? 1 : 0;
    }
}

// Per column over the listed rows: sum (pass 0), or the sum of squared deviations from the
// mean (pass 1), in FP64.
__global__ void __launch_bounds__(256) moments_kernel(const float* __restrict__ raw, const float* __restrict__ delta,
                                                      const int* __restrict__ rows, long long n_rows, int pass,
                                                      const double* __restrict__ mean, double* __restrict__ acc)
{
    __shared__ double s_acc[kCols];
    for (int c = threadIdx.x; c < kCols; c += blockDim.x) s_acc[c] = 0.0;
    __syncthreads();
    const long long total = n_rows * kCols;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long s = t / kCols;
        const int c = (int)(t % kCols);
        const double v = column(raw, delta, rows[s], c);
        const double x = pass == 0 ? v : (v - mean[c]) * (v - mean[c]);
        atomicAdd(&s_acc[c], x);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < kCols; c += blockDim.x) atomicAdd(&acc[c], s_acc[c]);
}

// keep2: among the keep1 rows, every standardised input within +-ood_z and every
// standardised target within +-target_clip.
__global__ void zbox_kernel(const float* __restrict__ raw, const float* __restrict__ delta, const int* __restrict__ rows,
                            long long n_rows, const Stats* __restrict__ st, uint8_t* __restrict__ keep)
{
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n_rows;
         s += (long long)gridDim.x * blockDim.x) {
        const long long i = rows[s];
        bool ok = true;
        for (int c = 0; c < kCols && ok; ++c) {
            const float z = (column(raw, delta, i, c) - st->mean[c]) / st->std_[c];
            ok = fabsf(z) <= (c < kIn ? st->ood_z : st->target_clip);
        }
        keep[s] = ok ? 1 : 0;
    }
}

// rows[j] = rows2[rows[j]]: positions among the keep1 rows to indices into the set.
__global__ void gather_rows_kernel(int* __restrict__ rows, const int* __restrict__ rows2, long long n)
{
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
        rows[j] = rows2[rows[j]];
}

// Minimum and maximum key of every input column over the listed rows.
__global__ void __launch_bounds__(256) range_kernel(const float* __restrict__ raw, const int* __restrict__ rows,
                                                    long long n_rows, uint32_t* __restrict__ kmin,
                                                    uint32_t* __restrict__ kmax)
{
    __shared__ uint32_t s_min[kIn], s_max[kIn];
    for (int c = threadIdx.x; c < kIn; c += blockDim.x) {
        s_min[c] = 0xffffffffu;
        s_max[c] = 0u;
    }
    __syncthreads();
    const long long total = n_rows * kIn;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long s = t / kIn;
        const int c = (int)(t % kIn);
        const uint32_t k = float_key(raw[(long long)rows[s] * kIn + c]);
        atomicMin(&s_min[c], k);
        atomicMax(&s_max[c], k);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < kIn; c += blockDim.x) {
        atomicMin(&kmin[c], s_min[c]);
        atomicMax(&kmax[c], s_max[c]);
    }
}

// The training set: row j of the output is listed row rows[j], inputs standardised to bf16
// (zero padded to 64), targets standardised (zero padded to 32).
__global__ void emit_kernel(const float* __restrict__ raw, const float* __restrict__ delta, const int* __restrict__ rows,
                            long long n_rows, const Stats* __restrict__ st, __nv_bfloat16* __restrict__ x,
                            float* __restrict__ t)
{
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n_rows;
         j += (long long)gridDim.x * blockDim.x) {
        const long long i = rows[j];
        for (int k = 0; k < MDG_MLP_IN_PAD; ++k)
            x[j * MDG_MLP_IN_PAD + k] =
                __float2bfloat16_rn(k < kIn ? (raw[i * kIn + k] - st->mean[k]) * st->inv_std[k] : 0.f);
        for (int k = 0; k < MDG_MLP_OUT_PAD; ++k)
            t[j * MDG_MLP_OUT_PAD + k] =
                k < kOut ? (delta[i * kOut + k] - st->mean[kIn + k]) / st->std_[kIn + k] : 0.f;
    }
}

int grid_for(long long n, int block) { return (int)std::min<long long>((n + block - 1) / block, 152 * 16); }

// Stable compaction on the device: idx[0 .. count) = the set rows in order. Returns the count.
cudaError_t compact(const uint8_t* flags, long long N, int* idx, int* counts, long long* d_total, long long* count,
                    cudaStream_t s)
{
    const int nb = (int)((N + kScanBlock - 1) / kScanBlock);
    count_kernel<<<nb, kScanBlock, 0, s>>>(flags, N, counts);
    scan_kernel<<<1, 1024, 0, s>>>(counts, nb, d_total);
    scatter_kernel<<<nb, kScanBlock, 0, s>>>(flags, N, counts, idx);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(count, d_total, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

}  // namespace

extern "C" {

int mdg_transition(mdg_handle h, float* state, const float* rpm, const float* rpm_scale, float* applied, float* raw,
                   float* delta, int32_t n_substeps, void* stream)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_transition: NULL handle");
    const long long n = mdg_num_drones(h);
    if (n == 0) return MDG_OK;
    if (!state || !rpm || !applied || !raw || !delta) return fail(MDG_ERR_ARG, "mdg_transition: NULL buffer");
    const uintptr_t a16 = reinterpret_cast<uintptr_t>(state) | reinterpret_cast<uintptr_t>(rpm) |
                          reinterpret_cast<uintptr_t>(rpm_scale) | reinterpret_cast<uintptr_t>(applied);
    if (a16 & 15u) return fail(MDG_ERR_ARG, "mdg_transition: state, rpm, rpm_scale and applied must be 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(raw) | reinterpret_cast<uintptr_t>(delta)) & 3u)
        return fail(MDG_ERR_ARG, "mdg_transition: raw and delta must be 4-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    transition_begin_kernel<<<grid_for(n, 256), 256, 0, s>>>(reinterpret_cast<const float4*>(state), n,
                                                             reinterpret_cast<const float4*>(rpm),
                                                             reinterpret_cast<const float4*>(rpm_scale),
                                                             reinterpret_cast<float4*>(applied), delta);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mdg_transition");
    int rc = mdg_features(h, state, applied, raw, stream);
    if (rc == MDG_OK) rc = mdg_step(h, state, applied, MDG_ACT_RPM, n_substeps, stream);
    if (rc != MDG_OK) return rc;
    transition_end_kernel<<<grid_for(n, 256), 256, 0, s>>>(reinterpret_cast<const float4*>(state), n, delta);
    e = cudaGetLastError();
    return e == cudaSuccess ? MDG_OK : cuda_fail(e, "mdg_transition");
}

int mdg_mlp_fit_normalization(mdg_mlp m, const float* raw, const float* delta, int64_t N, float trim_frac, float margin,
                              float ood_z, float target_clip, uint16_t* x_out, float* t_out, int64_t* n_finite,
                              int64_t* n_kept, void* stream)
{
    if (!m || !raw || !delta || !x_out || !t_out) return fail(MDG_ERR_ARG, "mdg_mlp_fit_normalization: NULL argument");
    if (N <= 0 || N > 0x7fffffffLL) return fail(MDG_ERR_ARG, "mdg_mlp_fit_normalization: N = %lld", (long long)N);
    if (!(trim_frac >= 0.f && trim_frac < 0.5f) || !(margin >= 0.f) || !(ood_z > 0.f) || !(target_clip > 0.f))
        return fail(MDG_ERR_ARG, "mdg_mlp_fit_normalization: trim_frac in [0, 0.5), margin >= 0, ood_z and "
                                 "target_clip > 0");
    if ((reinterpret_cast<uintptr_t>(x_out) & 15u) || (reinterpret_cast<uintptr_t>(t_out) & 15u))
        return fail(MDG_ERR_ARG, "mdg_mlp_fit_normalization: x_out and t_out must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((N + kScanBlock - 1) / kScanBlock);
    uint8_t *finite = nullptr, *keep = nullptr;
    int *rows = nullptr, *rows2 = nullptr, *counts = nullptr;
    long long* d_total = nullptr;
    uint32_t *lo = nullptr, *hi = nullptr, *kmin = nullptr, *kmax = nullptr;
    unsigned* cnt = nullptr;
    double *d_mean = nullptr, *d_acc = nullptr;
    Stats* d_st = nullptr;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc((void**)&finite, N);
    alloc((void**)&keep, N);
    alloc((void**)&rows, N * sizeof(int));
    alloc((void**)&rows2, N * sizeof(int));
    alloc((void**)&counts, (size_t)nb * sizeof(int));
    alloc((void**)&d_total, sizeof(long long));
    alloc((void**)&lo, kCols * 4 * 4);
    alloc((void**)&hi, kCols * 4 * 4);
    alloc((void**)&cnt, kCols * 4 * 4);
    alloc((void**)&kmin, kIn * 4);
    alloc((void**)&kmax, kIn * 4);
    alloc((void**)&d_mean, kCols * 8);
    alloc((void**)&d_acc, kCols * 8);
    alloc((void**)&d_st, sizeof(Stats));
    long long n_fin = 0, n1 = 0, n2 = 0;
    Stats st{};
    if (e == cudaSuccess) {
        finite_kernel<<<grid_for(N, 256), 256, 0, s>>>(raw, delta, N, finite);
        e = compact(finite, N, rows, counts, d_total, &n_fin, s);
    }
    if (e == cudaSuccess && n_fin == 0) {
        e = cudaErrorInvalidValue;
    }
    // the trim box: quantiles trim_frac and 1 - trim_frac of every column over an evenly
    // strided sample of at most kSampleMax finite rows (linear interpolation between order
    // statistics), widened by margin times their distance
    const long long stride = std::max<long long>(1, n_fin / kSampleMax);
    const long long n_sample = (n_fin + stride - 1) / stride;
    Selections sel{};
    sel.n = kCols * 4;
    const double hq[2] = {(n_sample - 1) * (double)trim_frac, (n_sample - 1) * (1.0 - (double)trim_frac)};
    for (int c = 0; c < kCols; ++c)
        for (int q = 0; q < 2; ++q) {
            const long long k0 = (long long)floor(hq[q]);
            sel.rank[4 * c + 2 * q] = (int)k0;
            sel.rank[4 * c + 2 * q + 1] = (int)std::min(k0 + 1, n_sample - 1);
        }
    if (e == cudaSuccess) {
        std::vector<uint32_t> h_lo(kCols * 4, 0u), h_hi(kCols * 4, 0xffffffffu);
        e = cudaMemcpyAsync(lo, h_lo.data(), h_lo.size() * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hi, h_hi.data(), h_hi.size() * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, kCols * 4 * 4, s);
        for (int it = 0; it < 32 && e == cudaSuccess; ++it) {
            select_count_kernel<<<grid_for(n_sample * kCols, 256), 256, 0, s>>>(raw, delta, rows, stride, n_sample,
                                                                               lo, hi, cnt);
            select_update_kernel<<<1, 256, 0, s>>>(sel, lo, hi, cnt);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_lo.data(), lo, h_lo.size() * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        for (int c = 0; c < kCols && e == cudaSuccess; ++c) {
            float qv[2];
            for (int q = 0; q < 2; ++q) {
                const float x0 = key_float(h_lo[4 * c + 2 * q]), x1 = key_float(h_lo[4 * c + 2 * q + 1]);
                const float w = (float)(hq[q] - floor(hq[q]));
                qv[q] = x0 + w * (x1 - x0);
            }
            const float r = qv[1] - qv[0];
            st.box_lo[c] = qv[0] - margin * r;
            st.box_hi[c] = qv[1] + margin * r;
        }
    }
    // keep1 and its mean and standard deviation (FP64; unbiased; a column whose deviation is
    // below 1e-6 max(|mean|, 1) is scaled by 1)
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_st, &st, sizeof(Stats), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        box_kernel<<<grid_for(N, 256), 256, 0, s>>>(raw, delta, N, finite, d_st, keep);
        e = compact(keep, N, rows2, counts, d_total, &n1, s);
    }
    if (e == cudaSuccess && n1 < 2) e = cudaErrorInvalidValue;
    double mean[kCols], var[kCols];
    if (e == cudaSuccess) e = cudaMemsetAsync(d_acc, 0, kCols * 8, s);
    if (e == cudaSuccess) {
        moments_kernel<<<grid_for(n1 * kCols, 256), 256, 0, s>>>(raw, delta, rows2, n1, 0, d_mean, d_acc);
        e = cudaMemcpyAsync(mean, d_acc, kCols * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        for (int c = 0; c < kCols; ++c) mean[c] /= (double)n1;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_mean, mean, kCols * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_acc, 0, kCols * 8, s);
    if (e == cudaSuccess) {
        moments_kernel<<<grid_for(n1 * kCols, 256), 256, 0, s>>>(raw, delta, rows2, n1, 1, d_mean, d_acc);
        e = cudaMemcpyAsync(var, d_acc, kCols * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e == cudaSuccess) {
        for (int c = 0; c < kCols; ++c) {
            const double sd = sqrt(var[c] / (double)(n1 - 1));
            const float sf = sd > 1e-6 * std::max(fabs(mean[c]), 1.0) ? (float)sd : 1.f;
            st.mean[c] = (float)mean[c];
            st.std_[c] = sf;
            st.inv_std[c] = 1.f / sf;
        }
        st.ood_z = ood_z;
        st.target_clip = target_clip;
        e = cudaMemcpyAsync(d_st, &st, sizeof(Stats), cudaMemcpyHostToDevice, s);
    }
    // keep2 (standardised inputs within +-ood_z, targets within +-target_clip) among keep1
    if (e == cudaSuccess) {
        zbox_kernel<<<grid_for(n1, 256), 256, 0, s>>>(raw, delta, rows2, n1, d_st, keep);
        e = compact(keep, n1, rows, counts, d_total, &n2, s);  // positions among rows2
    }
    // rows = indices of the kept rows into the set (their positions among the keep1 rows mapped)
    if (e == cudaSuccess && n2 > 0) {
        gather_rows_kernel<<<grid_for(n2, 256), 256, 0, s>>>(rows, rows2, n2);
        e = cudaGetLastError();
    }
    // the out-of-distribution box: the kept inputs' range, widened by 10% of it plus 1e-6
    float in_lo[kIn], in_hi[kIn];
    if (e == cudaSuccess && n2 > 0) {
        std::vector<uint32_t> fmin(kIn, 0xffffffffu), fmax(kIn, 0u);
        e = cudaMemcpyAsync(kmin, fmin.data(), kIn * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(kmax, fmax.data(), kIn * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            range_kernel<<<grid_for(n2 * kIn, 256), 256, 0, s>>>(raw, rows, n2, kmin, kmax);
            e = cudaMemcpyAsync(fmin.data(), kmin, kIn * 4, cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(fmax.data(), kmax, kIn * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        for (int c = 0; c < kIn; ++c) {
            const float a = key_float(fmin[c]), b = key_float(fmax[c]);
            const float pad = 0.1f * (b - a) + 1e-6f;
            in_lo[c] = a - pad;
            in_hi[c] = b + pad;
        }
    }
    const long long n_out = n2 / 128 * 128;
    if (e == cudaSuccess && n_out > 0) {
        emit_kernel<<<grid_for(n_out, 256), 256, 0, s>>>(raw, delta, rows, n_out, d_st,
                                                         reinterpret_cast<__nv_bfloat16*>(x_out), t_out);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFree(finite);
    cudaFree(keep);
    cudaFree(rows);
    cudaFree(rows2);
    cudaFree(counts);
    cudaFree(d_total);
    cudaFree(lo);
    cudaFree(hi);
    cudaFree(cnt);
    cudaFree(kmin);
    cudaFree(kmax);
    cudaFree(d_mean);
    cudaFree(d_acc);
    cudaFree(d_st);
    if (e != cudaSuccess) {
        if (e == cudaErrorInvalidValue) return fail(MDG_ERR_ARG, "mdg_mlp_fit_normalization: too few usable rows");
        return cuda_fail(e, "mdg_mlp_fit_normalization");
    }
    if (n2 == 0) return fail(MDG_ERR_ARG, "mdg_mlp_fit_normalization: no row passes the trim");
    std::vector<float> out_std(kOut), in_std(kIn);
    for (int k = 0; k < kIn; ++k) in_std[k] = st.std_[k];
    for (int k = 0; k < kOut; ++k) out_std[k] = st.std_[kIn + k];
    const int rc = mdg_mlp_set_normalization(m, st.mean, in_std.data(), st.mean + kIn, out_std.data(), in_lo, in_hi);
    if (rc != MDG_OK) return rc;
    if (n_finite) *n_finite = n_fin;
    if (n_kept) *n_kept = n_out;
    return MDG_OK;
}

}  // extern "C"
