// Host side of the learned surrogate (mdg_mlp_*, mdg_features, mdg_surrogate_step):
// parameter and scratch buffers, the training step (forward with targets, backward,
// Adam) and the per-control-step pipeline prepare -> network -> apply -> fallback.
#include <cuda_bf16.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <vector>

#include "mdg.h"
#include "mdg_internal.cuh"

namespace {

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

int cuda_fail(cudaError_t e, const char* what) { return fail(MDG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e)); }

// Offsets of W_l and b_l in the flat parameter layout of mdg.h.
constexpr int kDims[5] = {MDG_MLP_IN_PAD, MDG_MLP_HIDDEN, MDG_MLP_HIDDEN, MDG_MLP_HIDDEN, MDG_MLP_OUT_PAD};

mdg::MlpView layout(float* master, void* w16)
{
    mdg::MlpView v{};
    v.master = master;
    v.w16 = w16;
    int off = 0;
    for (int l = 0; l < 4; ++l) {
        v.w_off[l] = off;
        off += kDims[l + 1] * kDims[l];
        v.b_off[l] = off;
        off += kDims[l + 1];
    }
    return v;
}
static_assert(MDG_MLP_PARAMS == 256 * 64 + 256 + 2 * (256 * 256 + 256) + 32 * 256 + 32, "parameter count");

}  // namespace

struct mdg_mlp_s {
    int device = 0;
    int max_batch = 0;
    float* master = nullptr;
    __nv_bfloat16* w16 = nullptr;
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    int step = 0;
    float* z[3] = {};
    __nv_bfloat16* h[3] = {};
    __nv_bfloat16* dz[3] = {};
    float* y = nullptr;
    __nv_bfloat16* dy = nullptr;
    __nv_bfloat16* x = nullptr;  // inference inputs [max_batch][64]
    float* loss = nullptr;
    float* norm = nullptr;       // in_mean[41] in_inv_std[41] in_lo[41] in_hi[41] out_mean[13] out_std[13]
    bool norm_set = false;
    unsigned* env_flag = nullptr;
    int* fb_list = nullptr;
    int* fb_count = nullptr;
    uint32_t* status = nullptr;
    int path = MDG_MLP_PATH_TCGEN05_PAIRS;
    uint8_t* img = nullptr;      // weight image of the tcgen05 kernel
    bool img_stale = true;       // the bf16 weights changed since the image was built
    int wait_limit = MDG_MLP_DEFAULT_TRY_WAITS;  // bounded waits of the tcgen05 kernel
    int spin_limit = MDG_MLP_DEFAULT_POLLS;
    int train_path = MDG_MLP_PATH_TCGEN05;
    __nv_bfloat16* hT[3] = {};  // tcgen05 training: transposed activations and gradients
    __nv_bfloat16* dzT[3] = {};
    __nv_bfloat16* dyT = nullptr;
    __nv_bfloat16* xT = nullptr;
    __nv_bfloat16* wT = nullptr;  // W2^T, W3^T, W4^T
    bool wT_stale = true;
    mdg::MlpView view() const { return layout(master, w16); }
};

namespace {

void destroy_mlp(mdg_mlp m)
{
    cudaFree(m->master);
    cudaFree(m->w16);
    cudaFree(m->grad);
    cudaFree(m->m);
    cudaFree(m->v);
    for (int l = 0; l < 3; ++l) {
        cudaFree(m->z[l]);
        cudaFree(m->h[l]);
        cudaFree(m->dz[l]);
    }
    cudaFree(m->y);
    cudaFree(m->dy);
    cudaFree(m->x);
    cudaFree(m->loss);
    cudaFree(m->norm);
    cudaFree(m->env_flag);
    cudaFree(m->fb_list);
    cudaFree(m->fb_count);
    cudaFree(m->status);
    cudaFree(m->img);
    for (int l = 0; l < 3; ++l) {
        cudaFree(m->hT[l]);
        cudaFree(m->dzT[l]);
    }
    cudaFree(m->dyT);
    cudaFree(m->xT);
    cudaFree(m->wT);
    delete m;
}

// The tcgen05 kernel reads the weights from their image; rebuild it after they change.
cudaError_t forward_umma(mdg_mlp m, const void* x, int B, float* y, uint32_t* status, cudaStream_t s,
                         const mdg::MlpApply* apply = nullptr)
{
    if (m->img_stale) {
        cudaError_t e = mdg::mlp_build_image(m->view(), m->img, s);
        if (e != cudaSuccess) return e;
        m->img_stale = false;
    }
    if (m->path == MDG_MLP_PATH_TCGEN05_PAIRS)
        return mdg::mlp_forward_umma_pairs(m->view(), m->img, x, B, y, status, m->wait_limit, m->spin_limit, s, apply);
    return mdg::mlp_forward_umma(m->view(), m->img, x, B, y, status, m->wait_limit, m->spin_limit, s);
}

bool batch_ok(mdg_mlp m, int B) { return B > 0 && B % 128 == 0 && B <= m->max_batch; }

struct Guard {
    int prev = -1;
    explicit Guard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~Guard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

int mdg_mlp_create(int32_t max_batch, const float* init, mdg_mlp* out)
{
    if (!out) return fail(MDG_ERR_ARG, "mdg_mlp_create: out is NULL");
    *out = nullptr;
    if (max_batch <= 0 || max_batch % 128) return fail(MDG_ERR_ARG, "mdg_mlp_create: max_batch must be a positive multiple of 128");
    mdg_mlp m = new mdg_mlp_s();
    cudaGetDevice(&m->device);
    m->max_batch = max_batch;
    const size_t P = MDG_MLP_PARAMS, B = (size_t)max_batch, H = MDG_MLP_HIDDEN;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
    };
    alloc((void**)&m->master, P * 4);
    alloc((void**)&m->w16, P * 2);
    alloc((void**)&m->grad, P * 4);
    alloc((void**)&m->m, P * 4);
    alloc((void**)&m->v, P * 4);
    for (int l = 0; l < 3; ++l) {
        alloc((void**)&m->z[l], B * H * 4);
        alloc((void**)&m->h[l], B * H * 2);
        alloc((void**)&m->dz[l], B * H * 2);
    }
    alloc((void**)&m->y, B * MDG_MLP_OUT_PAD * 4);
    alloc((void**)&m->dy, B * MDG_MLP_OUT_PAD * 2);
    alloc((void**)&m->x, B * MDG_MLP_IN_PAD * 2);
    alloc((void**)&m->loss, 4);
    alloc((void**)&m->norm, (4 * MDG_MLP_IN + 2 * MDG_MLP_OUT) * 4);
    alloc((void**)&m->env_flag, B * 4);
    alloc((void**)&m->fb_list, B * 4);
    alloc((void**)&m->fb_count, 4);
    alloc((void**)&m->status, 8);
    alloc((void**)&m->img, mdg::mlp_image_bytes());
    for (int l = 0; l < 3; ++l) {
        alloc((void**)&m->hT[l], B * H * 2);
        alloc((void**)&m->dzT[l], B * H * 2);
    }
    alloc((void**)&m->dyT, B * MDG_MLP_OUT_PAD * 2);
    alloc((void**)&m->xT, B * MDG_MLP_IN_PAD * 2);
    alloc((void**)&m->wT, mdg::mlp_weights_transposed_elems() * 2);
    if (e == cudaSuccess && init) e = cudaMemcpy(m->master, init, P * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = mdg::mlp_refresh_bf16(m->view(), 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        destroy_mlp(m);
        return cuda_fail(e, "mdg_mlp_create");
    }
    *out = m;
    return MDG_OK;
}

int mdg_mlp_destroy(mdg_mlp m)
{
    if (!m) return MDG_OK;
    Guard g(m->device);
    cudaDeviceSynchronize();
    destroy_mlp(m);
    return MDG_OK;
}

int mdg_mlp_get_params(mdg_mlp m, float* host_out)
{
    if (!m || !host_out) return fail(MDG_ERR_ARG, "mdg_mlp_get_params: NULL argument");
    Guard g(m->device);
    cudaError_t e = cudaMemcpy(host_out, m->master, (size_t)MDG_MLP_PARAMS * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MDG_OK : cuda_fail(e, "mdg_mlp_get_params");
}

int mdg_mlp_set_params(mdg_mlp m, const float* host_in)
{
    if (!m || !host_in) return fail(MDG_ERR_ARG, "mdg_mlp_set_params: NULL argument");
    Guard g(m->device);
    cudaError_t e = cudaMemcpy(m->master, host_in, (size_t)MDG_MLP_PARAMS * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = mdg::mlp_refresh_bf16(m->view(), 0);
    m->img_stale = true;
    m->wT_stale = true;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e == cudaSuccess ? MDG_OK : cuda_fail(e, "mdg_mlp_set_params");
}

int mdg_mlp_get_grads(mdg_mlp m, float* host_out)
{
    if (!m || !host_out) return fail(MDG_ERR_ARG, "mdg_mlp_get_grads: NULL argument");
    Guard g(m->device);
    cudaError_t e = cudaMemcpy(host_out, m->grad, (size_t)MDG_MLP_PARAMS * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MDG_OK : cuda_fail(e, "mdg_mlp_get_grads");
}

int mdg_mlp_set_normalization(mdg_mlp m, const float* in_mean, const float* in_std, const float* out_mean,
                              const float* out_std, const float* in_lo, const float* in_hi)
{
    if (!m || !in_mean || !in_std || !out_mean || !out_std || !in_lo || !in_hi)
        return fail(MDG_ERR_ARG, "mdg_mlp_set_normalization: NULL argument");
    std::vector<float> h(4 * MDG_MLP_IN + 2 * MDG_MLP_OUT);
    for (int k = 0; k < MDG_MLP_IN; ++k) {
        if (!(in_std[k] > 0.f)) return fail(MDG_ERR_ARG, "mdg_mlp_set_normalization: in_std[%d] must be > 0", k);
        h[k] = in_mean[k];
        h[MDG_MLP_IN + k] = 1.f / in_std[k];
        h[2 * MDG_MLP_IN + k] = in_lo[k];
        h[3 * MDG_MLP_IN + k] = in_hi[k];
    }
    for (int k = 0; k < MDG_MLP_OUT; ++k) {
        h[4 * MDG_MLP_IN + k] = out_mean[k];
        h[4 * MDG_MLP_IN + MDG_MLP_OUT + k] = out_std[k];
    }
    Guard g(m->device);
    cudaError_t e = cudaMemcpy(m->norm, h.data(), h.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_mlp_set_normalization");
    m->norm_set = true;
    return MDG_OK;
}

int mdg_mlp_standardize(mdg_mlp m, const float* raw, uint16_t* x, int64_t rows, void* stream)
{
    if (!m) return fail(MDG_ERR_ARG, "mdg_mlp_standardize: NULL handle");
    if (!m->norm_set) return fail(MDG_ERR_ARG, "mdg_mlp_standardize: call mdg_mlp_set_normalization first");
    if (rows < 0) return fail(MDG_ERR_ARG, "mdg_mlp_standardize: rows < 0");
    if (rows > 0 && (!raw || !x)) return fail(MDG_ERR_ARG, "mdg_mlp_standardize: NULL buffer");
    Guard g(m->device);
    cudaError_t e = mdg::mlp_standardize(raw, x, rows, m->norm, m->norm + MDG_MLP_IN, (cudaStream_t)stream);
    return e == cudaSuccess ? MDG_OK : cuda_fail(e, "mdg_mlp_standardize");
}

int mdg_mlp_forward(mdg_mlp m, const uint16_t* x, float* y, int32_t B, void* stream)
{
    if (!m || !x || !y) return fail(MDG_ERR_ARG, "mdg_mlp_forward: NULL argument");
    if (!batch_ok(m, B)) return fail(MDG_ERR_ARG, "mdg_mlp_forward: B = %d must be a multiple of 128 <= %d", B, m->max_batch);
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u)
        return fail(MDG_ERR_ARG, "mdg_mlp_forward: x and y must be 16-byte aligned");
    Guard g(m->device);
    cudaError_t e;
    if (m->path != MDG_MLP_PATH_MMA_SYNC) {
        e = forward_umma(m, x, B, y, m->status, (cudaStream_t)stream);
    } else {
        float* zs[3] = {nullptr, nullptr, nullptr};
        void* hs[3] = {m->h[0], m->h[1], m->h[2]};
        e = mdg::mlp_forward(m->view(), x, B, zs, hs, y, nullptr, nullptr, nullptr, (cudaStream_t)stream);
    }
    return e == cudaSuccess ? MDG_OK : cuda_fail(e, "mdg_mlp_forward");
}

int mdg_mlp_get_normalization(mdg_mlp m, float* in_mean, float* in_std, float* out_mean, float* out_std, float* in_lo,
                              float* in_hi)
{
    if (!m) return fail(MDG_ERR_ARG, "mdg_mlp_get_normalization: NULL handle");
    if (!m->norm_set) return fail(MDG_ERR_ARG, "mdg_mlp_get_normalization: the surrogate has no normalisation");
    std::vector<float> h(4 * MDG_MLP_IN + 2 * MDG_MLP_OUT);
    Guard g(m->device);
    cudaError_t e = cudaMemcpy(h.data(), m->norm, h.size() * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_mlp_get_normalization");
    for (int k = 0; k < MDG_MLP_IN; ++k) {
        if (in_mean) in_mean[k] = h[k];
        if (in_std) in_std[k] = 1.f / h[MDG_MLP_IN + k];
        if (in_lo) in_lo[k] = h[2 * MDG_MLP_IN + k];
        if (in_hi) in_hi[k] = h[3 * MDG_MLP_IN + k];
    }
    for (int k = 0; k < MDG_MLP_OUT; ++k) {
        if (out_mean) out_mean[k] = h[4 * MDG_MLP_IN + k];
        if (out_std) out_std[k] = h[4 * MDG_MLP_IN + MDG_MLP_OUT + k];
    }
    return MDG_OK;
}

int mdg_mlp_grad(mdg_mlp m, const uint16_t* x, const float* t, int32_t B, float* loss_out, void* stream)
{
    if (!m || !x || !t) return fail(MDG_ERR_ARG, "mdg_mlp_grad: NULL argument");
    if (!batch_ok(m, B)) return fail(MDG_ERR_ARG, "mdg_mlp_grad: B = %d must be a multiple of 128 <= %d", B, m->max_batch);
    Guard g(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(m->loss, 0, 4, s);
    float* zs[3] = {m->z[0], m->z[1], m->z[2]};
    void* hs[3] = {m->h[0], m->h[1], m->h[2]};
    void* dzs[3] = {m->dz[0], m->dz[1], m->dz[2]};
    if (m->train_path == MDG_MLP_PATH_TCGEN05) {
        if (e == cudaSuccess && m->wT_stale) {
            e = mdg::mlp_weights_transposed(m->view(), m->wT, s);
            if (e == cudaSuccess) m->wT_stale = false;
        }
        mdg::TrainBuffers tb;
        for (int l = 0; l < 3; ++l) {
            tb.z[l] = m->z[l];
            tb.h[l] = m->h[l];
            tb.hT[l] = m->hT[l];
            tb.dz[l] = m->dz[l];
            tb.dzT[l] = m->dzT[l];
        }
        tb.y = m->y;
        tb.dy = m->dy;
        tb.dyT = m->dyT;
        tb.xT = m->xT;
        tb.wT = m->wT;
        if (e == cudaSuccess) e = mdg::mlp_grad_umma(m->view(), tb, x, B, t, m->loss, m->grad, m->status, s);
    } else {
        if (e == cudaSuccess) e = mdg::mlp_forward(m->view(), x, B, zs, hs, m->y, t, m->dy, m->loss, s);
        if (e == cudaSuccess) e = mdg::mlp_backward(m->view(), x, B, zs, hs, m->dy, dzs, m->grad, s);
    }
    if (e == cudaSuccess && loss_out) e = cudaMemcpyAsync(loss_out, m->loss, 4, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? MDG_OK : cuda_fail(e, "mdg_mlp_grad");
}

int mdg_mlp_adam(mdg_mlp m, float lr, void* stream)
{
    if (!m) return fail(MDG_ERR_ARG, "mdg_mlp_adam: NULL handle");
    if (!(lr > 0.f)) return fail(MDG_ERR_ARG, "mdg_mlp_adam: lr must be > 0");
    Guard g(m->device);
    m->step += 1;
    m->img_stale = true;
    m->wT_stale = true;
    cudaError_t e = mdg::mlp_adam(m->view(), m->grad, m->m, m->v, lr, m->step, (cudaStream_t)stream);
    return e == cudaSuccess ? MDG_OK : cuda_fail(e, "mdg_mlp_adam");
}

int mdg_mlp_set_path(mdg_mlp m, int32_t path)
{
    if (!m) return fail(MDG_ERR_ARG, "mdg_mlp_set_path: NULL handle");
    if (path != MDG_MLP_PATH_MMA_SYNC && path != MDG_MLP_PATH_TCGEN05 && path != MDG_MLP_PATH_TCGEN05_PAIRS)
        return fail(MDG_ERR_ARG, "mdg_mlp_set_path: unknown path %d", path);
    m->path = path;
    return MDG_OK;
}

int mdg_mlp_set_train_path(mdg_mlp m, int32_t path)
{
    if (!m) return fail(MDG_ERR_ARG, "mdg_mlp_set_train_path: NULL handle");
    if (path != MDG_MLP_PATH_MMA_SYNC && path != MDG_MLP_PATH_TCGEN05)
        return fail(MDG_ERR_ARG, "mdg_mlp_set_train_path: unknown path %d", path);
    m->train_path = path;
    return MDG_OK;
}

int mdg_mlp_set_wait_limits(mdg_mlp m, int32_t try_waits, int32_t polls)
{
    if (!m) return fail(MDG_ERR_ARG, "mdg_mlp_set_wait_limits: NULL handle");
    m->wait_limit = try_waits < 0 ? MDG_MLP_DEFAULT_TRY_WAITS : try_waits;
    m->spin_limit = polls < 0 ? MDG_MLP_DEFAULT_POLLS : polls;
    return MDG_OK;
}

int mdg_mlp_status(mdg_mlp m, void* stream, uint32_t* bits)
{
    if (!m) return fail(MDG_ERR_ARG, "mdg_mlp_status: NULL handle");
    Guard g(m->device);
    uint32_t st[2] = {0u, 0u};
    cudaError_t e = cudaMemcpyAsync(st, m->status, 8, cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, 8, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_mlp_status");
    if (bits) *bits = st[0];
    return MDG_OK;
}

int mdg_features(mdg_handle h, const float* state, const float* rpm, float* raw, void* stream)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_features: NULL handle");
    if (h->n_drones == 0) return MDG_OK;
    if (!state || !rpm || !raw) return fail(MDG_ERR_ARG, "mdg_features: NULL buffer");
    if ((reinterpret_cast<uintptr_t>(state) | reinterpret_cast<uintptr_t>(rpm)) & 15u)
        return fail(MDG_ERR_ARG, "mdg_features: state and rpm must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(raw) & 3u) return fail(MDG_ERR_ARG, "mdg_features: raw misaligned");
    Guard g(h->device);
    mdg::SurrogateArgs a{};
    a.s.state = reinterpret_cast<float4*>(const_cast<float*>(state));
    a.s.tiles = h->d_tiles;
    a.s.env_off = h->d_off;
    a.s.env_flags = h->d_flags;
    a.s.env_act = h->d_act;
    a.s.status = h->d_status;
    a.s.n = h->n_drones;
    a.s.n_envs = h->n_envs;
    a.s.uniform_N = h->uniform_N;
    a.s.envs_per_tile = h->envs_per_tile;
    a.s.uniform_bits = h->uniform_bits;
    a.s.act_type = MDG_ACT_RPM;
    a.s.c = h->dc;
    a.raw = raw;
    a.rpm = reinterpret_cast<const float4*>(rpm);
    cudaError_t e = mdg::launch_features(a, h->n_tiles, h->block, (cudaStream_t)stream);
    return e == cudaSuccess ? MDG_OK : cuda_fail(e, "mdg_features");
}

int mdg_surrogate_step(mdg_handle h, mdg_mlp m, float* state, const float* action, int32_t action_type,
                       int32_t n_substeps, float ood_z, int32_t* n_fallback, void* stream)
{
    if (!h || !m) return fail(MDG_ERR_ARG, "mdg_surrogate_step: NULL handle");
    if (h->n_drones == 0) return MDG_OK;
    if (h->uniform_N <= 0)
        return fail(MDG_ERR_UNSUPPORTED, "mdg_surrogate_step: needs environments of one size");
    if (!mdg::valid_action(action_type))
        return fail(MDG_ERR_ARG, "mdg_surrogate_step: unknown action_type %d", action_type);
    if (action_type == MDG_ACT_MIXED && !h->act_set)
        return fail(MDG_ERR_ARG, "mdg_surrogate_step: MDG_ACT_MIXED needs mdg_set_action_types first");
    if (n_substeps < 1) return fail(MDG_ERR_ARG, "mdg_surrogate_step: n_substeps < 1");
    if (h->dr)
        return fail(MDG_ERR_UNSUPPORTED, "mdg_surrogate_step: randomization is not supported (its fallback runs the plain model)");
    if (h->dc.dsl && !h->d_sp)
        return fail(MDG_ERR_ARG, "mdg_surrogate_step: the DSL controller needs mdg_set_setpoints first");
    if (!m->norm_set) return fail(MDG_ERR_ARG, "mdg_surrogate_step: the surrogate has no normalisation");
    const int n_pad = (int)((h->n_drones + 127) / 128 * 128);
    if (n_pad > m->max_batch)
        return fail(MDG_ERR_ARG, "mdg_surrogate_step: %lld drones exceed the surrogate's max_batch %d",
                    (long long)h->n_drones, m->max_batch);
    if (!state || !action) return fail(MDG_ERR_ARG, "mdg_surrogate_step: NULL buffer");
    if ((reinterpret_cast<uintptr_t>(state) | reinterpret_cast<uintptr_t>(action)) & 15u)
        return fail(MDG_ERR_ARG, "mdg_surrogate_step: state and action must be 16-byte aligned");
    Guard g(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    mdg::SurrogateArgs a{};
    a.s.state = reinterpret_cast<float4*>(state);
    a.s.action = reinterpret_cast<const float4*>(action);
    a.s.tiles = h->d_tiles;
    a.s.env_off = h->d_off;
    a.s.env_flags = h->d_flags;
    a.s.env_act = h->d_act;
    a.s.status = h->d_status;
    a.s.n = h->n_drones;
    a.s.n_sub = n_substeps;
    a.s.act_type = action_type;
    a.s.n_envs = h->n_envs;
    a.s.uniform_N = h->uniform_N;
    a.s.envs_per_tile = h->envs_per_tile;
    a.s.uniform_bits = h->uniform_bits;
    a.s.setpoints = h->d_sp;
    a.s.c = h->dc;
    a.x = m->x;
    a.y = m->y;
    a.in_mean = m->norm;
    a.in_inv_std = m->norm + MDG_MLP_IN;
    a.in_lo = m->norm + 2 * MDG_MLP_IN;
    a.in_hi = m->norm + 3 * MDG_MLP_IN;
    a.out_mean = m->norm + 4 * MDG_MLP_IN;
    a.out_std = m->norm + 4 * MDG_MLP_IN + MDG_MLP_OUT;
    a.ood_z = ood_z;
    a.env_flag = m->env_flag;
    a.fallback_list = m->fb_list;
    a.fallback_count = m->fb_count;
    cudaError_t e = cudaMemsetAsync(m->env_flag, 0, (size_t)h->n_envs * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->fb_count, 0, 4, s);
    if (e == cudaSuccess && n_pad > h->n_drones)  // padding rows of the network input
        e = cudaMemsetAsync(m->x + (size_t)h->n_drones * MDG_MLP_IN_PAD, 0,
                            (size_t)(n_pad - h->n_drones) * MDG_MLP_IN_PAD * 2, s);
    bool fused = false;
    if (e == cudaSuccess) e = mdg::launch_surrogate_prepare(a, h->n_tiles, h->block, s);
    if (e == cudaSuccess) {
        if (m->path == MDG_MLP_PATH_TCGEN05_PAIRS) {
            // the paired kernel updates the state itself (no y, no separate update launch)
            mdg::MlpApply ap{a.s.state, h->n_drones, h->uniform_N, m->env_flag, a.out_mean, a.out_std};
            e = forward_umma(m, m->x, n_pad, m->y, h->d_status, s, &ap);
            fused = true;
        } else if (m->path != MDG_MLP_PATH_MMA_SYNC) {
            e = forward_umma(m, m->x, n_pad, m->y, h->d_status, s);
        } else {
            float* zs[3] = {nullptr, nullptr, nullptr};
            void* hs[3] = {m->h[0], m->h[1], m->h[2]};
            e = mdg::mlp_forward(m->view(), m->x, n_pad, zs, hs, m->y, nullptr, nullptr, nullptr, s);
        }
    }
    if (e == cudaSuccess && !fused) e = mdg::launch_surrogate_apply(a, s);
    if (e == cudaSuccess) e = mdg::launch_surrogate_fallback(a, s);
    if (e == cudaSuccess && n_fallback) e = cudaMemcpyAsync(n_fallback, m->fb_count, 4, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? MDG_OK : cuda_fail(e, "mdg_surrogate_step");
}

}  // extern "C"
