// Host side of the C ABI declared in include/mdg.h: constants, handle lifetime,
// argument validation, launch tiles and the status word.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "mdg.h"
#include "mdg_internal.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(MDG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace


// (struct mdg_ctx is defined in mdg_internal.cuh)

// Table and constant builders shared by the handle API and the allocation-free entry point.
namespace mdg {

void set_last_error(const char* msg) { g_last_error = msg; }

bool constants_valid(const mdg_constants& c, std::string& why)
{
    const double pos[] = {c.mass, c.arm, c.thrust2weight, c.Jxx, c.Jyy, c.Jzz, c.kf, c.km, c.prop_radius,
                          c.g, c.h_clip, c.dt_sim, c.dt_ctrl, c.dw_max_xy};
    for (double v : pos)
        if (!(v > 0.0) || !isfinite(v)) {
            why = "model constants must be positive and finite";
            return false;
        }
    if (c.thrust2weight <= 1.0) {
        why = "thrust2weight must exceed 1";
        return false;
    }
    if (c.frame != MDG_FRAME_X && c.frame != MDG_FRAME_P) {
        why = "frame must be MDG_FRAME_X or MDG_FRAME_P";
        return false;
    }
    if (c.integrator != MDG_INTEGRATOR_EULER && c.integrator != MDG_INTEGRATOR_RK4) {
        why = "integrator must be MDG_INTEGRATOR_EULER or MDG_INTEGRATOR_RK4";
        return false;
    }
    if (c.gnd_heights != MDG_GND_COM && c.gnd_heights != MDG_GND_ROTOR) {
        why = "gnd_heights must be MDG_GND_COM or MDG_GND_ROTOR";
        return false;
    }
    if (c.controller != MDG_CTRL_PID && c.controller != MDG_CTRL_DSL) {
        why = "controller must be MDG_CTRL_PID or MDG_CTRL_DSL";
        return false;
    }
    if (c.controller == MDG_CTRL_DSL &&
        (!(c.sp_rate_pos > 0.0) || !isfinite(c.sp_rate_pos) || !(c.sp_rate_yaw > 0.0) || !isfinite(c.sp_rate_yaw))) {
        why = "the DSL controller needs positive, finite setpoint rates";
        return false;
    }
    return true;
}

DevConsts make_dev_consts(const mdg_constants& c)
{
    mdg::DevConsts d{};
    const double pi = 3.14159265358979323846;
    d.mass = (float)c.mass;
    d.inv_mass = (float)(1.0 / c.mass);
    d.g = (float)c.g;
    d.inv_g = (float)(1.0 / c.g);
    d.kf = (float)c.kf;
    d.km = (float)c.km;
    d.l_sqrt2 = (float)(c.arm / sqrt(2.0));
    const double J[3] = {c.Jxx, c.Jyy, c.Jzz};
    for (int i = 0; i < 3; ++i) {
        d.J[i] = (float)J[i];
        d.inv_J[i] = (float)(1.0 / J[i]);
    }
    d.gnd_k = (float)(c.c_gnd * (c.prop_radius / 4.0) * (c.prop_radius / 4.0));
    d.h_clip = (float)c.h_clip;
    d.drag_k = (float)(2.0 * pi / 60.0);
    d.c_xy = (float)c.c_xy;
    d.c_z = (float)c.c_z;
    d.c_dz = (float)(c.c_z - c.c_xy);
    d.dw_k = (float)(c.dw_c1 * (c.prop_radius / 4.0) * (c.prop_radius / 4.0));
    d.dw_c2 = (float)c.dw_c2;
    d.dw_c3 = (float)c.dw_c3;
    d.dw_max_xy2 = (float)(c.dw_max_xy * c.dw_max_xy);
    d.dw_dz_min = (float)std::max(0.0, c.dw_dz_min);
    for (int i = 0; i < 3; ++i) {
        d.pos_kp[i] = (float)c.pos_kp[i];
        d.pos_ki[i] = (float)c.pos_ki[i];
        d.pos_kd[i] = (float)c.pos_kd[i];
        d.att_kp[i] = (float)c.att_kp[i];
        d.att_ki[i] = (float)c.att_ki[i];
        d.att_kd[i] = (float)c.att_kd[i];
    }
    d.pos_iclamp = (float)c.pos_iclamp;
    d.att_iclamp = (float)c.att_iclamp;
    d.dt_sim = (float)c.dt_sim;
    d.dt_ctrl = (float)c.dt_ctrl;
    const double maxrpm = sqrt(c.thrust2weight * c.mass * c.g / (4.0 * c.kf));
    d.max_rpm = (float)maxrpm;
    d.f_max = (float)(c.kf * maxrpm * maxrpm);
    d.inv_kf = (float)(1.0 / c.kf);
    d.hover_rpm = (float)sqrt(c.mass * c.g / (4.0 * c.kf));
    d.alloc_z = (float)(c.kf / c.km);
    d.frame_p = c.frame == MDG_FRAME_P ? 1 : 0;
    d.rk4 = c.integrator == MDG_INTEGRATOR_RK4 ? 1 : 0;
    d.gnd_rotor = c.gnd_heights == MDG_GND_ROTOR ? 1 : 0;
    d.dsl = c.controller == MDG_CTRL_DSL ? 1 : 0;
    d.sp_step_pos = (float)(c.sp_rate_pos * c.dt_ctrl);
    d.sp_step_yaw = (float)(c.sp_rate_yaw * c.dt_ctrl);
    if (d.frame_p) {
        // + layout: tau_x = L (F1 - F3), tau_y = L (F2 - F0); the mixing rows [1,1,1,1],
        // [0,1,0,-1] L, [-1,0,1,0] L, [-1,1,-1,1] k_m/k_f are orthogonal with squared norms
        // 4, 2 L^2, 2 L^2, 4 (k_m/k_f)^2
        d.l_sqrt2 = (float)c.arm;
        d.alloc_xy = (float)(2.0 / c.arm);
        const float sx[4] = {0.f, 1.f, 0.f, -1.f}, sy[4] = {-1.f, 0.f, 1.f, 0.f};
        for (int i = 0; i < 4; ++i) d.mix_x[i] = sx[i], d.mix_y[i] = sy[i];
    } else {
        d.alloc_xy = (float)(sqrt(2.0) / c.arm);
        const float sx[4] = {1.f, 1.f, -1.f, -1.f}, sy[4] = {-1.f, 1.f, 1.f, -1.f};
        for (int i = 0; i < 4; ++i) d.mix_x[i] = sx[i], d.mix_y[i] = sy[i];
    }
    // rotor body positions: tau_x = sum_i y_i F_i and tau_y = -sum_i x_i F_i, so rotor i
    // sits at y_i = a mix_x[i], x_i = -a mix_y[i] with a = L/sqrt2 (X) or L (+)
    for (int i = 0; i < 4; ++i) {
        d.rotor_x[i] = -d.l_sqrt2 * d.mix_y[i];
        d.rotor_y[i] = d.l_sqrt2 * d.mix_x[i];
    }
    return d;
}

// Greedy packing of whole environments, in CSR order, into tiles of at most `block`
// drones and `block` environments, with the tile bits the kernels branch on.
std::vector<Tile> build_tiles(const std::vector<int32_t>& off, const std::vector<uint8_t>& flags, int block)
{
    std::vector<mdg::Tile> tiles;
    const int n_envs = (int)off.size() - 1;
    int e = 0;
    while (e < n_envs) {
        const int e0 = e;
        while (e < n_envs && (off[e + 1] - off[e0]) <= block && (e + 1 - e0) <= block) ++e;
        if (e == e0) break;  // an environment larger than the block: rejected before this point
        mdg::Tile t;
        t.x = off[e0];
        t.y = off[e] - off[e0];
        t.z = e0;
        t.w = e - e0;
        bool any_dw = false, warp_local = true;
        for (int k = e0; k < e; ++k) {
            const int ls = off[k] - off[e0], N = off[k + 1] - off[k];
            if (N > 0 && (flags[k] & MDG_DW)) any_dw = true;
            if (N > 0 && (ls >> 5) != ((ls + N - 1) >> 5)) warp_local = false;
        }
        if (any_dw) t.w |= mdg::kTileAnyDW;
        if (warp_local) t.w |= mdg::kTileWarpLocal;
        if (t.y > 0) tiles.push_back(t);
    }
    return tiles;
}

// Default threads per block: enough for the largest environment, and otherwise the size
// that spreads the tiles most evenly over the SMs (a block count close to a multiple of
// the SM count), preferring larger blocks on ties.
int default_block(int32_t max_env, int64_t n_drones, int n_sm)
{
    int lo = 32;
    while (lo < max_env) lo *= 2;
    if (lo >= 1024) return 1024;
    int best = std::max(lo, 128);
    double best_eff = -1.0;
    for (int b = lo; b <= 256; b *= 2) {
        const double blocks = std::ceil((double)n_drones / b);
        const double waves = std::ceil(blocks / n_sm);
        const double eff = blocks / (waves * n_sm);
        if (eff > best_eff - 1e-9) {
            best_eff = eff;
            best = b;
        }
    }
    return best;
}

}  // namespace mdg

namespace {

using mdg::build_tiles;
using mdg::constants_valid;
using mdg::default_block;
using mdg::make_dev_consts;

int set_block(mdg_ctx* h, int block)
{
    std::vector<mdg::Tile> tiles = build_tiles(h->h_off, h->h_flags, block);
    mdg::Tile* d_tiles = nullptr;
    if (!tiles.empty()) {
        cudaError_t e = cudaMalloc(&d_tiles, tiles.size() * sizeof(mdg::Tile));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(tiles)");
        e = cudaMemcpy(d_tiles, tiles.data(), tiles.size() * sizeof(mdg::Tile), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d_tiles);
            return cuda_fail(e, "cudaMemcpy(tiles)");
        }
    }
    if (h->d_tiles) {
        cudaDeviceSynchronize();
        cudaFree(h->d_tiles);
    }
    h->d_tiles = d_tiles;
    h->n_tiles = (int)tiles.size();
    h->block = block;
    // Uniform batches (all environments of one size N > 0): the kernels compute the tiles
    // arithmetically (block / N environments per block), which the greedy packing matches.
    h->uniform_N = 0;
    if (h->n_envs > 0 && h->max_env > 0) {
        const int N = h->max_env;
        bool uniform = true;
        for (int32_t e = 0; e < h->n_envs && uniform; ++e) uniform = (h->h_off[e + 1] - h->h_off[e]) == N;
        if (uniform) {
            h->uniform_N = N;
            h->envs_per_tile = block / N;
            h->uniform_bits = 0;
            for (const mdg::Tile& t : tiles) h->uniform_bits |= t.w & mdg::kTileAnyDW;
            bool all_local = true;
            for (const mdg::Tile& t : tiles) all_local = all_local && (t.w & mdg::kTileWarpLocal);
            if (all_local) h->uniform_bits |= mdg::kTileWarpLocal;
        }
    }
    return MDG_OK;
}

void free_schedule(mdg_ctx* h)
{
    cudaFree(h->d_sched_off);
    cudaFree(h->d_sched_items);
    h->d_sched_off = h->d_sched_items = nullptr;
    h->sched_grid = 0;
}

void free_rollout_tables(mdg_ctx* h)
{
    cudaFree(h->d_items);
    cudaFree(h->d_item_order);
    cudaFree(h->d_slot_env);
    cudaFree(h->d_slot_goff);
    cudaFree(h->d_slot_loff);
    h->d_items = nullptr;
    h->d_item_order = nullptr;
    h->d_slot_env = h->d_slot_goff = h->d_slot_loff = nullptr;
    h->n_items = 0;
    h->rollout_block = 0;
    h->rollout_cap = -1;
    h->item_cost.clear();
    free_schedule(h);
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& v)
{
    *dst = nullptr;
    if (v.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc(dst, v.size() * sizeof(T));
    if (e == cudaSuccess) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

// The dependent chain of one substep of an environment of N drones, in units of the
// instructions of a substep without downwash (~160), for the static schedule: the drones of
// a work item run in parallel threads, so an item lasts about as long as its longest chain.
double item_chain(int N, uint32_t flags) { return 160.0 + ((flags & MDG_DW) ? 23.0 * (N - 1) : 0.0); }

// Work items of the rollout kernel for the current block size and item cap. Uniform batches
// use the arithmetic tiles. Otherwise environments are sorted by (size descending, physics
// subset, index), so that the environments sharing a warp share their size and branches, and
// packed greedily into items of at most `cap` drones (the block size, or the handle's item
// cap when smaller; an environment larger than the cap is an item of its own) and `block`
// environments; items are handed out in decreasing cost (drones plus downwash pairs),
// longest first.
int ensure_rollout_tables(mdg_ctx* h)
{
    if (h->rollout_block == h->block && h->rollout_cap == h->item_cap && h->d_counter) return MDG_OK;
    if (h->d_item_order) cudaDeviceSynchronize();
    free_rollout_tables(h);
    cudaError_t e;
    if (!h->d_counter && (e = cudaMalloc(&h->d_counter, sizeof(int))) != cudaSuccess)
        return cuda_fail(e, "rollout: cudaMalloc(counter)");
    std::vector<int> order;
    h->item_cost.clear();
    if (h->uniform_N > 0) {
        h->n_items = h->n_tiles;
        order.resize(h->n_items);
        for (int i = 0; i < h->n_items; ++i) order[i] = i;
        bool dw = false;
        for (int32_t k = 0; k < h->n_envs; ++k) dw = dw || (h->h_flags[k] & MDG_DW);
        h->item_cost.assign(h->n_items, item_chain(h->uniform_N, dw ? MDG_DW : 0u));
    } else {
        const int cap = h->item_cap > 0 && h->item_cap < h->block ? h->item_cap : h->block;
        std::vector<int> envs;
        for (int32_t k = 0; k < h->n_envs; ++k)
            if (h->h_off[k + 1] > h->h_off[k]) envs.push_back(k);
        auto N = [&](int k) { return h->h_off[k + 1] - h->h_off[k]; };
        std::sort(envs.begin(), envs.end(), [&](int a, int b) {
            if (N(a) != N(b)) return N(a) > N(b);
            if (h->h_flags[a] != h->h_flags[b]) return h->h_flags[a] < h->h_flags[b];
            return a < b;
        });
        std::vector<int4> items;
        std::vector<int> slot_goff(envs.size()), slot_loff(envs.size());
        std::vector<double> cost;
        size_t i = 0;
        while (i < envs.size()) {
            const size_t i0 = i;
            int drones = 0;
            bool any_dw = false, local = true;
            double c = 0.0, chain = 0.0;
            while (i < envs.size() && (i == i0 || drones + N(envs[i]) <= cap) && drones + N(envs[i]) <= h->block &&
                   (int)(i + 1 - i0) <= h->block) {
                const int n = N(envs[i]);
                slot_goff[i] = h->h_off[envs[i]];
                slot_loff[i] = drones;
                if (h->h_flags[envs[i]] & MDG_DW) {
                    any_dw = true;
                    c += (double)n * n;
                }
                if ((drones >> 5) != ((drones + n - 1) >> 5)) local = false;
                c += n;
                chain = std::max(chain, item_chain(n, h->h_flags[envs[i]]));
                drones += n;
                ++i;
            }
            if (i == i0) return fail(MDG_ERR_ARG, "rollout: an environment exceeds the block size");
            int bits = (any_dw ? mdg::kTileAnyDW : 0) | (local ? mdg::kTileWarpLocal : 0);
            items.push_back(make_int4((int)i0, (int)(i - i0), drones, bits));
            cost.push_back(c);
            h->item_cost.push_back(chain);
        }
        h->n_items = (int)items.size();
        order.resize(h->n_items);
        for (int k = 0; k < h->n_items; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        if ((e = upload(&h->d_items, items)) != cudaSuccess || (e = upload(&h->d_slot_env, envs)) != cudaSuccess ||
            (e = upload(&h->d_slot_goff, slot_goff)) != cudaSuccess ||
            (e = upload(&h->d_slot_loff, slot_loff)) != cudaSuccess) {
            free_rollout_tables(h);
            return cuda_fail(e, "rollout: tables");
        }
    }
    if ((e = upload(&h->d_item_order, order)) != cudaSuccess) {
        free_rollout_tables(h);
        return cuda_fail(e, "rollout: item order");
    }
    h->rollout_block = h->block;
    h->rollout_cap = h->item_cap;
    free_schedule(h);
    return MDG_OK;
}

// The static schedule of the rollout kernel for a grid of `grid` persistent blocks: longest
// processing time first (items by decreasing chain estimate, each to the block with the least
// estimated work so far, the lower block index on ties), each block running its items in the
// order they were given to it. The same items on the same blocks every launch: the duration
// does not depend on which block happens to reach the work counter first.
int ensure_schedule(mdg_ctx* h, int grid)
{
    if (h->sched_grid == grid && h->d_sched_off) return MDG_OK;
    free_schedule(h);
    const int n = h->n_items;
    std::vector<int> by_cost(n);
    for (int i = 0; i < n; ++i) by_cost[i] = i;
    std::stable_sort(by_cost.begin(), by_cost.end(), [&](int a, int b) { return h->item_cost[a] > h->item_cost[b]; });
    std::vector<std::vector<int>> lists(grid);
    // min-heap of (load, block)
    std::vector<std::pair<double, int>> heap;
    for (int b = 0; b < grid; ++b) heap.push_back({0.0, b});
    auto later = [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
        return x.first != y.first ? x.first > y.first : x.second > y.second;
    };
    std::make_heap(heap.begin(), heap.end(), later);
    for (int it : by_cost) {
        std::pop_heap(heap.begin(), heap.end(), later);
        auto& top = heap.back();
        lists[top.second].push_back(it);
        top.first += h->item_cost[it];
        std::push_heap(heap.begin(), heap.end(), later);
    }
    std::vector<int> off(grid + 1, 0), items;
    items.reserve(n);
    for (int b = 0; b < grid; ++b) {
        items.insert(items.end(), lists[b].begin(), lists[b].end());
        off[b + 1] = (int)items.size();
    }
    cudaError_t e;
    if ((e = upload(&h->d_sched_off, off)) != cudaSuccess || (e = upload(&h->d_sched_items, items)) != cudaSuccess) {
        free_schedule(h);
        return cuda_fail(e, "rollout: static schedule");
    }
    h->sched_grid = grid;
    return MDG_OK;
}

void destroy_ctx(mdg_ctx* h)
{
    free_rollout_tables(h);
    cudaFree(h->d_counter);
    cudaFree(h->d_off);
    cudaFree(h->d_flags);
    cudaFree(h->d_act);
    cudaFree(h->d_tiles);
    cudaFree(h->d_status);
    cudaFree(h->d_rand);
    delete h;
}

int check_state_ptr(const mdg_ctx* h, const void* p, const char* name)
{
    if (h->n_drones == 0) return MDG_OK;
    if (!p) return fail(MDG_ERR_ARG, "%s is NULL", name);
    if (!aligned16(p)) return fail(MDG_ERR_ARG, "%s is not 16-byte aligned", name);
    return MDG_OK;
}

mdg::StepArgs base_args(mdg_ctx* h, float* state)
{
    mdg::StepArgs a{};
    a.state = reinterpret_cast<float4*>(state);
    a.tiles = h->d_tiles;
    a.env_off = h->d_off;
    a.env_flags = h->d_flags;
    a.env_act = h->d_act;
    a.status = h->d_status;
    a.n = h->n_drones;
    a.n_envs = h->n_envs;
    a.uniform_N = h->uniform_N;
    a.envs_per_tile = h->envs_per_tile;
    a.uniform_bits = h->uniform_bits;
    a.setpoints = h->d_sp;
    a.rand = h->dr ? h->d_rand : nullptr;
    a.c = h->dc;
    return a;
}

}  // namespace

extern "C" {

int mdg_constants_cf2x(mdg_constants* out)
{
    if (!out) return fail(MDG_ERR_ARG, "mdg_constants_cf2x: out is NULL");
    memset(out, 0, sizeof(*out));
    out->mass = 0.027;
    out->arm = 0.0397;
    out->thrust2weight = 2.25;
    out->Jxx = 1.4e-5;
    out->Jyy = 1.4e-5;
    out->Jzz = 2.17e-5;
    out->kf = 3.16e-10;
    out->km = 7.94e-12;
    out->prop_radius = 0.02325;
    out->g = 9.81;
    out->c_gnd = 11.36859;
    out->h_clip = 0.25 * out->prop_radius * sqrt(out->c_gnd / (out->thrust2weight - 1.0));
    out->c_xy = 9.1785e-7;
    out->c_z = 10.311e-7;
    out->dw_c1 = 2267.18;
    out->dw_c2 = 0.16;
    out->dw_c3 = -0.11;
    out->dw_max_xy = 10.0;
    out->dw_dz_min = 0.0;
    const double kp[3] = {0.4, 0.4, 1.0}, ki[3] = {0.01, 0.01, 0.01}, kd[3] = {0.9, 0.9, 2.0};
    const double akp[3] = {2e-3, 2e-3, 1e-3}, aki[3] = {0.0, 0.0, 1e-4}, akd[3] = {5e-4, 5e-4, 2e-4};
    for (int i = 0; i < 3; ++i) {
        out->pos_kp[i] = kp[i];
        out->pos_ki[i] = ki[i];
        out->pos_kd[i] = kd[i];
        out->att_kp[i] = akp[i];
        out->att_ki[i] = aki[i];
        out->att_kd[i] = akd[i];
    }
    out->pos_iclamp = 2.0;
    out->att_iclamp = 0.5;
    out->dt_sim = 1.0 / 240.0;
    out->dt_ctrl = 1.0 / 48.0;
    out->sp_rate_pos = 2.0;
    out->sp_rate_yaw = 3.14159265358979323846;
    out->frame = MDG_FRAME_X;
    out->integrator = MDG_INTEGRATOR_EULER;
    out->controller = MDG_CTRL_PID;
    return MDG_OK;
}

int mdg_constants_cf2p(mdg_constants* out)
{
    if (!out) return fail(MDG_ERR_ARG, "mdg_constants_cf2p: out is NULL");
    mdg_constants_cf2x(out);
    out->frame = MDG_FRAME_P;
    return MDG_OK;
}

int mdg_constants_race(mdg_constants* out)
{
    if (!out) return fail(MDG_ERR_ARG, "mdg_constants_race: out is NULL");
    mdg_constants cf;
    mdg_constants_cf2x(&cf);
    *out = cf;
    out->mass = 0.25;
    out->arm = 0.125;
    out->thrust2weight = 4.0;
    out->Jxx = 4.86e-4;
    out->Jyy = 4.86e-4;
    out->Jzz = 8.80e-4;
    out->kf = 1.28e-8;
    out->km = 5.96e-10;
    out->prop_radius = 0.0635;
    out->h_clip = 0.25 * out->prop_radius * sqrt(out->c_gnd / (out->thrust2weight - 1.0));
    const double ratio[3] = {out->Jxx / cf.Jxx, out->Jyy / cf.Jyy, out->Jzz / cf.Jzz};
    for (int i = 0; i < 3; ++i) {
        out->att_kp[i] = cf.att_kp[i] * ratio[i];
        out->att_ki[i] = cf.att_ki[i] * ratio[i];
        out->att_kd[i] = cf.att_kd[i] * ratio[i];
    }
    return MDG_OK;
}

int mdg_controller_dsl(mdg_constants* c)
{
    if (!c) return fail(MDG_ERR_ARG, "mdg_controller_dsl: c is NULL");
    const double wp[3] = {1.5, 1.5, 2.0}, zp[3] = {0.8, 0.8, 1.0};
    const double wa[3] = {20.0, 20.0, 10.0}, za = 0.9, kia[3] = {0.0, 0.0, 5.0};
    const double J[3] = {c->Jxx, c->Jyy, c->Jzz};
    for (int r = 0; r < 3; ++r) {
        c->pos_kp[r] = wp[r] * wp[r];
        c->pos_kd[r] = 2.0 * zp[r] * wp[r];
        c->pos_ki[r] = 0.05;
        c->att_kp[r] = J[r] * wa[r] * wa[r];
        c->att_kd[r] = 2.0 * za * wa[r] * J[r];
        c->att_ki[r] = J[r] * kia[r];
    }
    c->pos_iclamp *= 0.5;
    c->att_iclamp *= 0.5;
    c->controller = MDG_CTRL_DSL;
    return MDG_OK;
}

int mdg_constants_size(void) { return (int)sizeof(mdg_constants); }

double mdg_hover_rpm(const mdg_constants* c)
{
    if (!c || !(c->kf > 0.0) || !(c->mass > 0.0) || !(c->g > 0.0)) return -1.0;
    return sqrt(c->mass * c->g / (4.0 * c->kf));
}

double mdg_max_rpm(const mdg_constants* c)
{
    if (!c || !(c->kf > 0.0) || !(c->mass > 0.0) || !(c->g > 0.0) || !(c->thrust2weight > 0.0)) return -1.0;
    return sqrt(c->thrust2weight * c->mass * c->g / (4.0 * c->kf));
}

int mdg_create(int32_t n_envs, const int32_t* drones_per_env, const uint32_t* model_flags, const mdg_constants* c,
               mdg_handle* out)
{
    if (!out) return fail(MDG_ERR_ARG, "mdg_create: out is NULL");
    *out = nullptr;
    if (n_envs < 0) return fail(MDG_ERR_ARG, "mdg_create: n_envs < 0");
    if (n_envs > 0 && (!drones_per_env || !model_flags))
        return fail(MDG_ERR_ARG, "mdg_create: drones_per_env and model_flags are required");
    mdg_constants cc;
    if (c) cc = *c;
    else mdg_constants_cf2x(&cc);
    std::string why;
    if (!constants_valid(cc, why)) return fail(MDG_ERR_ARG, "mdg_create: %s", why.c_str());
    std::vector<int32_t> off(n_envs + 1, 0);
    std::vector<uint8_t> flags(n_envs, 0);
    int32_t max_env = 0;
    int64_t total = 0;
    for (int32_t e = 0; e < n_envs; ++e) {
        const int32_t N = drones_per_env[e];
        if (N < 0 || N > MDG_MAX_ENV_DRONES)
            return fail(MDG_ERR_ARG, "mdg_create: drones_per_env[%d] = %d outside [0, %d]", e, N, MDG_MAX_ENV_DRONES);
        if (model_flags[e] & ~(MDG_GND | MDG_DRAG | MDG_DW))
            return fail(MDG_ERR_ARG, "mdg_create: model_flags[%d] has unknown bits", e);
        total += N;
        if (total > 0x7fffffffLL) return fail(MDG_ERR_ARG, "mdg_create: more than 2^31 - 1 drones");
        off[e + 1] = (int32_t)total;
        flags[e] = (uint8_t)model_flags[e];
        max_env = std::max(max_env, N);
    }
    mdg_ctx* h = new mdg_ctx();
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaGetDevice");
    }
    h->n_envs = n_envs;
    h->n_drones = total;
    h->max_env = max_env;
    h->c = cc;
    h->dc = make_dev_consts(cc);
    h->cc = cc;
    h->h_off = off;
    h->h_flags = flags;
    h->uniform_flags = n_envs > 0 ? flags[0] : -1;
    for (int32_t e2 = 1; e2 < n_envs; ++e2)
        if (flags[e2] != flags[0]) h->uniform_flags = -1;
    if ((e = cudaMalloc(&h->d_off, off.size() * sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_flags, std::max<size_t>(1, flags.size()))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_act, std::max<size_t>(1, flags.size()))) != cudaSuccess ||
        (e = cudaMalloc(&h->d_status, 2 * sizeof(uint32_t))) != cudaSuccess) {
        destroy_ctx(h);
        return cuda_fail(e, "mdg_create: cudaMalloc");
    }
    const uint32_t status0[2] = {0u, 0xffffffffu};
    if ((e = cudaMemcpy(h->d_off, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (n_envs > 0 && (e = cudaMemcpy(h->d_flags, flags.data(), flags.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (e = cudaMemcpy(h->d_status, status0, sizeof(status0), cudaMemcpyHostToDevice)) != cudaSuccess) {
        destroy_ctx(h);
        return cuda_fail(e, "mdg_create: cudaMemcpy");
    }
    int n_sm = 152;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, h->device);
    int rc = set_block(h, default_block(max_env, total, n_sm > 0 ? n_sm : 152));
    if (rc != MDG_OK) {
        destroy_ctx(h);
        return rc;
    }
    *out = h;
    return MDG_OK;
}

int mdg_destroy(mdg_handle h)
{
    if (!h) return MDG_OK;
    DeviceGuard dg(h->device);
    cudaDeviceSynchronize();
    destroy_ctx(h);
    return MDG_OK;
}

int64_t mdg_num_drones(mdg_handle h)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_num_drones: NULL handle");
    return h->n_drones;
}

int mdg_set_action_types(mdg_handle h, const uint8_t* per_env)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_set_action_types: NULL handle");
    if (h->n_envs == 0) {
        h->act_set = true;
        return MDG_OK;
    }
    if (!per_env) return fail(MDG_ERR_ARG, "mdg_set_action_types: per_env is NULL");
    bool ext = false;
    for (int32_t e = 0; e < h->n_envs; ++e) {
        if (!mdg::valid_env_action(per_env[e]))
            return fail(MDG_ERR_ARG, "mdg_set_action_types: per_env[%d] = %d is not an action type", e, per_env[e]);
        ext = ext || mdg::extended_action(per_env[e]);
    }
    DeviceGuard dg(h->device);
    cudaError_t e = cudaMemcpy(h->d_act, per_env, (size_t)h->n_envs, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_set_action_types: cudaMemcpy");
    h->act_set = true;
    h->act_ext = ext;
    return MDG_OK;
}

int mdg_set_setpoints(mdg_handle h, float* setpoints)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_set_setpoints: NULL handle");
    if (setpoints && !aligned16(setpoints)) return fail(MDG_ERR_ARG, "mdg_set_setpoints: not 16-byte aligned");
    h->d_sp = reinterpret_cast<float4*>(setpoints);
    return MDG_OK;
}

int mdg_set_randomization(mdg_handle h, const float* env_params, float* motor, float* action_hist,
                          int32_t hist_depth, float* wind_state, uint64_t seed)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_set_randomization: NULL handle");
    if (!env_params) {
        h->dr = nullptr;
        h->rand_host.obs_bias = nullptr;
        return MDG_OK;
    }
    if (h->dc.rk4) return fail(MDG_ERR_UNSUPPORTED, "mdg_set_randomization: randomization integrates with Euler substeps");
    if (!motor || !action_hist || !wind_state)
        return fail(MDG_ERR_ARG, "mdg_set_randomization: motor, action_hist and wind_state are required");
    if (!aligned16(env_params) || !aligned16(motor) || !aligned16(action_hist) || !aligned16(wind_state))
        return fail(MDG_ERR_ARG, "mdg_set_randomization: buffers must be 16-byte aligned");
    if (hist_depth < 1 || hist_depth > MDG_MAX_HIST_DEPTH)
        return fail(MDG_ERR_ARG, "mdg_set_randomization: hist_depth = %d outside [1, %d]", hist_depth,
                    MDG_MAX_HIST_DEPTH);
    if (h->n_envs > 0) {
        DeviceGuard dg(h->device);
        std::vector<float> tab((size_t)h->n_envs * MDG_DR_PARAMS);
        cudaError_t e = cudaMemcpy(tab.data(), env_params, tab.size() * sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "mdg_set_randomization: reading env_params");
        for (int32_t k = 0; k < h->n_envs; ++k) {
            const float* r = tab.data() + (size_t)k * MDG_DR_PARAMS;
            for (int i = 0; i <= MDG_DR_G; ++i)
                if (!(r[i] > 0.f) || !isfinite(r[i]))
                    return fail(MDG_ERR_ARG, "mdg_set_randomization: env %d: factor %d = %g must be positive", k, i,
                                (double)r[i]);
            const float dly = r[MDG_DR_DELAY], bits = r[MDG_DR_WIND];
            bool ok = r[MDG_DR_TAU] >= 0.f && isfinite(r[MDG_DR_TAU]) && dly >= 0.f && dly == floorf(dly) &&
                      dly < (float)hist_depth && bits >= 0.f && bits == floorf(bits) && bits <= (float)MDG_WIND_COMBINED &&
                      r[MDG_DR_KDRAG] >= 0.f && r[MDG_DR_GUST_P] >= 0.f && r[MDG_DR_GUST_P] <= 1.f &&
                      r[MDG_DR_GUST_T] > 0.f && r[MDG_DR_DRY_SIGMA] >= 0.f && r[MDG_DR_DRY_V] >= 0.f &&
                      r[MDG_DR_DRY_H] > 0.f && r[MDG_DR_NOISE_P] >= 0.f && r[MDG_DR_NOISE_V] >= 0.f &&
                      r[MDG_DR_NOISE_RPY] >= 0.f && r[MDG_DR_NOISE_W] >= 0.f &&
                      (r[MDG_DR_OBS_DELAY] == 0.f || r[MDG_DR_OBS_DELAY] == 1.f);
            for (int i = MDG_DR_VWIND; i < MDG_DR_PARAMS; ++i) ok = ok && isfinite(r[i]);
            if (!ok)
                return fail(MDG_ERR_ARG, "mdg_set_randomization: env %d: invalid lag, delay, wind or sensor values", k);
        }
    }
    mdg::RandArgs ra;
    ra.dr = env_params;
    ra.motor = reinterpret_cast<float4*>(motor);
    ra.hist = reinterpret_cast<float4*>(action_hist);
    ra.wind = reinterpret_cast<float4*>(wind_state);
    ra.seed = seed;
    ra.depth = hist_depth;
    ra.obs_bias = h->dr ? h->rand_host.obs_bias : nullptr;  // an attached bias stays attached
    DeviceGuard dg(h->device);
    cudaError_t e = cudaSuccess;
    if (!h->d_rand) e = cudaMalloc(reinterpret_cast<void**>(&h->d_rand), sizeof(mdg::RandArgs));
    if (e == cudaSuccess) e = cudaMemcpy(h->d_rand, &ra, sizeof(ra), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_set_randomization: device copy of the buffers");
    h->dr = env_params;
    h->rand_host = ra;
    return MDG_OK;
}

int mdg_set_obs_bias(mdg_handle h, const float* obs_bias)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_set_obs_bias: NULL handle");
    if (!h->dr) return fail(MDG_ERR_ARG, "mdg_set_obs_bias: attach the randomization first (mdg_set_randomization)");
    if (obs_bias && !aligned16(obs_bias)) return fail(MDG_ERR_ARG, "mdg_set_obs_bias: obs_bias is not 16-byte aligned");
    mdg::RandArgs ra = h->rand_host;
    ra.obs_bias = reinterpret_cast<const float4*>(obs_bias);
    DeviceGuard dg(h->device);
    // the device copy is read by kernels already queued: replace it in stream order on the
    // legacy default stream, as mdg_set_randomization does
    const cudaError_t e = cudaMemcpy(h->d_rand, &ra, sizeof(ra), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_set_obs_bias: device copy of the buffers");
    h->rand_host = ra;
    return MDG_OK;
}

int mdg_reset(mdg_handle h, float* state, const float* nominal, const float* init_range, const float* bias_sigma,
              float* obs_bias, uint64_t seed, uint64_t episode, void* stream)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_reset: NULL handle");
    int rc;
    if ((rc = check_state_ptr(h, state, "state")) != MDG_OK) return rc;
    if ((rc = check_state_ptr(h, nominal, "nominal")) != MDG_OK) return rc;
    if (obs_bias && !aligned16(obs_bias)) return fail(MDG_ERR_ARG, "mdg_reset: obs_bias is not 16-byte aligned");
    if (obs_bias && !bias_sigma) return fail(MDG_ERR_ARG, "mdg_reset: obs_bias needs bias_sigma");
    mdg::ResetArgs r{};
    r.state = reinterpret_cast<float4*>(state);
    r.nominal = reinterpret_cast<const float4*>(nominal);
    r.obs_bias = reinterpret_cast<float4*>(obs_bias);
    r.n = h->n_drones;
    if (init_range) {
        for (int k = 0; k < 3; ++k)
            if (!(init_range[k] >= 0.f) || !isfinite(init_range[k]))
                return fail(MDG_ERR_ARG, "mdg_reset: init_range[%d] = %g must be finite and >= 0", k,
                            (double)init_range[k]);
        r.range_pos = init_range[0];
        r.range_att = init_range[1];
        r.range_vel = init_range[2];
    }
    if (obs_bias)
        for (int k = 0; k < 4; ++k) {
            if (!(bias_sigma[k] >= 0.f) || !isfinite(bias_sigma[k]))
                return fail(MDG_ERR_ARG, "mdg_reset: bias_sigma[%d] = %g must be finite and >= 0", k,
                            (double)bias_sigma[k]);
            r.sigma[k] = bias_sigma[k];
        }
    r.seed = seed;
    r.episode = episode;
    if (r.n == 0) return MDG_OK;
    DeviceGuard dg(h->device);
    const cudaError_t e = mdg::launch_reset(r, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_reset: launch");
    return MDG_OK;
}

int mdg_set_rollout_schedule(mdg_handle h, int32_t mode, int32_t item_drones)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_set_rollout_schedule: NULL handle");
    if (mode != MDG_SCHED_DYNAMIC && mode != MDG_SCHED_STATIC)
        return fail(MDG_ERR_ARG, "mdg_set_rollout_schedule: unknown mode %d", mode);
    if (item_drones < 0 || item_drones > 1024)
        return fail(MDG_ERR_ARG, "mdg_set_rollout_schedule: item_drones = %d outside [0, 1024]", item_drones);
    h->sched = mode;
    h->item_cap = item_drones;
    return MDG_OK;
}

int mdg_get_rollout_schedule(mdg_handle h, int32_t* mode, int32_t* item_drones)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_get_rollout_schedule: NULL handle");
    if (mode) *mode = h->sched;
    if (item_drones) *item_drones = h->item_cap;
    return MDG_OK;
}

int mdg_set_block_size(mdg_handle h, int32_t threads_per_block)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_set_block_size: NULL handle");
    if (threads_per_block < 32 || threads_per_block > 1024 || threads_per_block % 32 != 0)
        return fail(MDG_ERR_ARG, "mdg_set_block_size: %d is not a multiple of 32 in [32, 1024]", threads_per_block);
    if (threads_per_block < h->max_env)
        return fail(MDG_ERR_ARG, "mdg_set_block_size: %d is smaller than the largest environment (%d drones)",
                    threads_per_block, h->max_env);
    DeviceGuard dg(h->device);
    return set_block(h, threads_per_block);
}

int32_t mdg_get_block_size(mdg_handle h)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_get_block_size: NULL handle");
    return h->block;
}

// The physics-flag selector handed to the launchers: the batch's uniform flags, or 8 (the
// runtime-flag kernels) when an action type beyond RPM/PID is in use.
static int launch_flags(mdg_handle h, int32_t action_type)
{
    const bool ext = mdg::extended_action(action_type) || (action_type == MDG_ACT_MIXED && h->act_ext);
    return (ext || h->dc.dsl) ? 8 : h->uniform_flags;
}

// The DSL controller reads and writes the caller's setpoints: they must be attached.
static int check_setpoints(mdg_handle h, const char* fn)
{
    if (h->dc.dsl && !h->d_sp && h->n_drones > 0)
        return fail(MDG_ERR_ARG, "%s: the DSL controller needs mdg_set_setpoints first", fn);
    return MDG_OK;
}

static int step_common(mdg_handle h, float* state, const float* action, int32_t action_type, int32_t n_substeps,
                       float* kin, int32_t* nbr_idx, float* nbr_rel, bool with_obs, void* stream,
                       bool obs_host = false)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_step: NULL handle");
    if (!mdg::valid_action(action_type)) return fail(MDG_ERR_ARG, "mdg_step: unknown action_type %d", action_type);
    if (action_type == MDG_ACT_MIXED && !h->act_set)
        return fail(MDG_ERR_ARG, "mdg_step: MDG_ACT_MIXED needs mdg_set_action_types first");
    if (n_substeps < 1) return fail(MDG_ERR_ARG, "mdg_step: n_substeps = %d < 1", n_substeps);
    int rc;
    if ((rc = check_setpoints(h, "mdg_step")) != MDG_OK) return rc;
    if (obs_host && h->dr)
        return fail(MDG_ERR_UNSUPPORTED, "mdg_step_obs_host: not with randomization (use mdg_step_obs)");
    if ((rc = check_state_ptr(h, state, "state")) != MDG_OK) return rc;
    if ((rc = check_state_ptr(h, action, "action")) != MDG_OK) return rc;
    if (with_obs) {
        if ((rc = check_state_ptr(h, kin, "kin")) != MDG_OK) return rc;
        if ((rc = check_state_ptr(h, nbr_idx, "nbr_idx")) != MDG_OK) return rc;
        if (nbr_rel && !aligned16(nbr_rel)) return fail(MDG_ERR_ARG, "nbr_rel is not 16-byte aligned");
    }
    if (h->n_drones == 0) return MDG_OK;
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(MDG_ERR_CUDA, "mdg_step: cannot select device %d", h->device);
    mdg::StepArgs a = base_args(h, state);
    a.action = reinterpret_cast<const float4*>(action);
    a.kin = kin;
    a.nbr_idx = reinterpret_cast<int4*>(nbr_idx);
    a.nbr_rel = nbr_rel;
    a.n_sub = n_substeps;
    a.act_type = action_type;
    a.obs_host = obs_host ? 1 : 0;
    cudaError_t e =
        mdg::launch_step(a, h->n_tiles, h->block, with_obs, launch_flags(h, action_type), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_step: launch");
    return MDG_OK;
}

int mdg_step(mdg_handle h, float* state, const float* action, int32_t action_type, int32_t n_substeps, void* stream)
{
    return step_common(h, state, action, action_type, n_substeps, nullptr, nullptr, nullptr, false, stream);
}

int mdg_step_obs(mdg_handle h, float* state, const float* action, int32_t action_type, int32_t n_substeps,
                 float* kin, int32_t* nbr_idx, float* nbr_rel, void* stream)
{
    return step_common(h, state, action, action_type, n_substeps, kin, nbr_idx, nbr_rel, true, stream);
}

// The device address of page-locked, mapped host memory (NULL stays NULL).
static int mapped_ptr(const void* host, void** dev, const char* name)
{
    *dev = nullptr;
    if (!host) return MDG_OK;
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, host);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MDG_ERR_ARG, "mdg_step_obs_host: %s: %s", name, cudaGetErrorString(e));
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer)
        return fail(MDG_ERR_ARG, "mdg_step_obs_host: %s is not mapped page-locked host memory", name);
    *dev = at.devicePointer;
    return MDG_OK;
}

int mdg_sync(void* stream, int32_t timeout_ms)
{
    if (timeout_ms < 0) return fail(MDG_ERR_ARG, "mdg_sync: timeout_ms = %d < 0", timeout_ms);
    const auto t0 = std::chrono::steady_clock::now();
    const auto limit = std::chrono::milliseconds(timeout_ms);
    for (;;) {
        const cudaError_t e = cudaStreamQuery((cudaStream_t)stream);
        if (e == cudaSuccess) return MDG_OK;
        if (e != cudaErrorNotReady) return cuda_fail(e, "mdg_sync");
        if (std::chrono::steady_clock::now() - t0 >= limit)
            return fail(MDG_ERR_TIMEOUT, "mdg_sync: stream still busy after %d ms", timeout_ms);
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

int mdg_step_obs_host(mdg_handle h, float* state, const float* action_host, int32_t action_type, int32_t n_substeps,
                      float* kin_host, int32_t* nbr_idx_host, float* nbr_rel_host, void* stream)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_step_obs_host: NULL handle");
    if (h->n_drones == 0) return MDG_OK;
    if (!action_host || !kin_host || !nbr_idx_host) return fail(MDG_ERR_ARG, "mdg_step_obs_host: NULL buffer");
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(MDG_ERR_CUDA, "mdg_step_obs_host: cannot select device %d", h->device);
    void *act = nullptr, *kin = nullptr, *idx = nullptr, *rel = nullptr;
    int rc;
    if ((rc = mapped_ptr(action_host, &act, "action_host")) != MDG_OK) return rc;
    if ((rc = mapped_ptr(kin_host, &kin, "kin_host")) != MDG_OK) return rc;
    if ((rc = mapped_ptr(nbr_idx_host, &idx, "nbr_idx_host")) != MDG_OK) return rc;
    if ((rc = mapped_ptr(nbr_rel_host, &rel, "nbr_rel_host")) != MDG_OK) return rc;
    return step_common(h, state, static_cast<const float*>(act), action_type, n_substeps, static_cast<float*>(kin),
                       static_cast<int32_t*>(idx), static_cast<float*>(rel), true, stream, true);
}

int mdg_pid_ff(mdg_handle h, float* state, const float* waypoints, const float* target_acc, float* rpm_out,
               float* pos_err, float* yaw_err, void* stream)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_pid: NULL handle");
    int rc;
    if ((rc = check_state_ptr(h, state, "state")) != MDG_OK) return rc;
    if ((rc = check_state_ptr(h, waypoints, "waypoints")) != MDG_OK) return rc;
    if ((rc = check_state_ptr(h, rpm_out, "rpm_out")) != MDG_OK) return rc;
    if (target_acc && !aligned16(target_acc)) return fail(MDG_ERR_ARG, "target_acc is not 16-byte aligned");
    if (pos_err && (reinterpret_cast<uintptr_t>(pos_err) & 3u)) return fail(MDG_ERR_ARG, "pos_err misaligned");
    if (yaw_err && (reinterpret_cast<uintptr_t>(yaw_err) & 3u)) return fail(MDG_ERR_ARG, "yaw_err misaligned");
    if ((rc = check_setpoints(h, "mdg_pid")) != MDG_OK) return rc;
    if (h->n_drones == 0) return MDG_OK;
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(MDG_ERR_CUDA, "mdg_pid: cannot select device %d", h->device);
    mdg::PidArgs a{};
    a.state = reinterpret_cast<float4*>(state);
    a.waypoints = reinterpret_cast<const float4*>(waypoints);
    a.target_acc = reinterpret_cast<const float4*>(target_acc);
    a.setpoints = h->d_sp;
    a.rpm_out = reinterpret_cast<float4*>(rpm_out);
    a.pos_err = pos_err;
    a.yaw_err = yaw_err;
    a.n = h->n_drones;
    a.c = h->dc;
    cudaError_t e = mdg::launch_pid(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_pid: launch");
    return MDG_OK;
}

int mdg_pid(mdg_handle h, float* state, const float* waypoints, float* rpm_out, float* pos_err, float* yaw_err,
            void* stream)
{
    return mdg_pid_ff(h, state, waypoints, nullptr, rpm_out, pos_err, yaw_err, stream);
}

int mdg_render(mdg_handle h, const float* state, uint8_t* rgba, float* depth, int32_t* seg, void* stream)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_render: NULL handle");
    int rc;
    if ((rc = check_state_ptr(h, state, "state")) != MDG_OK) return rc;
    const void* outs[] = {rgba, depth, seg};
    for (const void* o : outs)
        if (o && (reinterpret_cast<uintptr_t>(o) & 3u)) return fail(MDG_ERR_ARG, "mdg_render: outputs must be 4-byte aligned");
    if (h->n_drones == 0 || (!rgba && !depth && !seg)) return MDG_OK;
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(MDG_ERR_CUDA, "mdg_render: cannot select device %d", h->device);
    mdg::CamArgs a{};
    a.state = reinterpret_cast<const float4*>(state);
    a.n = h->n_drones;
    a.n_envs = h->n_envs;
    a.env_off = h->d_off;
    a.uniform_N = h->uniform_N;
    a.rgba = reinterpret_cast<uchar4*>(rgba);
    a.depth = depth;
    a.seg = seg;
    a.semi_a = (float)(h->cc.arm + h->cc.prop_radius);
    a.semi_c = (float)(0.3 * (h->cc.arm + h->cc.prop_radius));
    a.max_env = h->max_env;
    a.status = h->d_status;
    cudaError_t e = mdg::launch_render(a, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_render: launch");
    return MDG_OK;
}

int mdg_obs(mdg_handle h, const float* state, float* kin, int32_t* nbr_idx, float* nbr_rel, void* stream)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_obs: NULL handle");
    int rc;
    if ((rc = check_state_ptr(h, state, "state")) != MDG_OK) return rc;
    if ((rc = check_state_ptr(h, kin, "kin")) != MDG_OK) return rc;
    if ((rc = check_state_ptr(h, nbr_idx, "nbr_idx")) != MDG_OK) return rc;
    if (nbr_rel && !aligned16(nbr_rel)) return fail(MDG_ERR_ARG, "nbr_rel is not 16-byte aligned");
    if (h->n_drones == 0) return MDG_OK;
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(MDG_ERR_CUDA, "mdg_obs: cannot select device %d", h->device);
    mdg::StepArgs a = base_args(h, const_cast<float*>(state));
    a.kin = kin;
    a.nbr_idx = reinterpret_cast<int4*>(nbr_idx);
    a.nbr_rel = nbr_rel;
    a.act_type = MDG_ACT_RPM;
    cudaError_t e = mdg::launch_obs(a, h->n_tiles, h->block, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_obs: launch");
    return MDG_OK;
}

int mdg_status(mdg_handle h, void* stream, uint32_t* bits, int64_t* first_drone)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_status: NULL handle");
    DeviceGuard dg(h->device);
    uint32_t st[2];
    cudaError_t e = cudaMemcpyAsync(st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_status: read");
    const uint32_t status0[2] = {0u, 0xffffffffu};
    e = cudaMemcpyAsync(h->d_status, status0, sizeof(status0), cudaMemcpyHostToDevice, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_status: clear");
    if (bits) *bits = st[0];
    if (first_drone) *first_drone = st[1] == 0xffffffffu ? -1 : (int64_t)st[1];
    return (st[0] & MDG_STATUS_NONFINITE) ? MDG_ERR_NONFINITE : MDG_OK;
}

// The persistent grid of a rollout: the SMs times the blocks of the kernel variant that fit
// one SM, at most one block per work item.
static int rollout_grid(mdg_handle h, const mdg::RolloutArgs& r)
{
    int n_sm = 152;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, h->device);
    int grid = n_sm * mdg::rollout_blocks_per_sm(r.s, h->block, launch_flags(h, r.s.act_type));
    if (grid <= 0 || grid > r.n_items) grid = r.n_items;
    return grid;
}

static int rollout_args(mdg_handle h, float* state, const float* actions, int32_t action_per_step, int32_t action_type,
                        int32_t n_substeps, int32_t K, int32_t obs_mode, float* kin, int32_t* nbr_idx, float* nbr_rel,
                        mdg::RolloutArgs* r)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_rollout: NULL handle");
    if (!mdg::valid_action(action_type)) return fail(MDG_ERR_ARG, "mdg_rollout: unknown action_type %d", action_type);
    if (action_type == MDG_ACT_MIXED && !h->act_set)
        return fail(MDG_ERR_ARG, "mdg_rollout: MDG_ACT_MIXED needs mdg_set_action_types first");
    if (n_substeps < 1) return fail(MDG_ERR_ARG, "mdg_rollout: n_substeps = %d < 1", n_substeps);
    if (K < 0) return fail(MDG_ERR_ARG, "mdg_rollout: K = %d < 0", K);
    if (check_setpoints(h, "mdg_rollout") != MDG_OK) return MDG_ERR_ARG;
    if (obs_mode != MDG_OBS_NONE && obs_mode != MDG_OBS_LAST && obs_mode != MDG_OBS_EVERY_STEP)
        return fail(MDG_ERR_ARG, "mdg_rollout: unknown obs_mode %d", obs_mode);
    int rc;
    if ((rc = check_state_ptr(h, state, "state")) != MDG_OK) return rc;
    if ((rc = check_state_ptr(h, actions, "actions")) != MDG_OK) return rc;
    if (obs_mode != MDG_OBS_NONE) {
        if ((rc = check_state_ptr(h, kin, "kin")) != MDG_OK) return rc;
        if ((rc = check_state_ptr(h, nbr_idx, "nbr_idx")) != MDG_OK) return rc;
        if (nbr_rel && !aligned16(nbr_rel)) return fail(MDG_ERR_ARG, "nbr_rel is not 16-byte aligned");
    }
    if ((rc = ensure_rollout_tables(h)) != MDG_OK) return rc;
    *r = mdg::RolloutArgs{};
    r->s = base_args(h, state);
    r->s.action = reinterpret_cast<const float4*>(actions);
    r->s.kin = obs_mode != MDG_OBS_NONE ? kin : nullptr;
    r->s.nbr_idx = obs_mode != MDG_OBS_NONE ? reinterpret_cast<int4*>(nbr_idx) : nullptr;
    r->s.nbr_rel = obs_mode != MDG_OBS_NONE ? nbr_rel : nullptr;
    r->s.n_sub = n_substeps;
    r->s.act_type = action_type;
    r->action_stride = action_per_step ? h->n_drones : 0;
    r->K = K;
    r->obs_mode = obs_mode;
    r->n_items = h->n_items;
    r->work_counter = h->d_counter;
    r->item_order = h->d_item_order;
    r->items = h->d_items;
    r->slot_env = h->d_slot_env;
    r->slot_goff = h->d_slot_goff;
    r->slot_loff = h->d_slot_loff;
    r->sched_off = nullptr;
    r->sched_items = nullptr;
    if (h->sched == MDG_SCHED_STATIC && h->n_items > 0) {
        if ((rc = ensure_schedule(h, rollout_grid(h, *r))) != MDG_OK) return rc;
        r->sched_off = h->d_sched_off;
        r->sched_items = h->d_sched_items;
    }
    return MDG_OK;
}

static cudaError_t enqueue_rollout(mdg_handle h, const mdg::RolloutArgs& r, cudaStream_t s)
{
    if (r.n_items == 0 || r.K == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(h->d_counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    return mdg::launch_rollout(r, h->block, launch_flags(h, r.s.act_type), rollout_grid(h, r), s);
}

int mdg_rollout(mdg_handle h, float* state, const float* actions, int32_t action_per_step, int32_t action_type,
                int32_t n_substeps, int32_t K, int32_t obs_mode, float* kin, int32_t* nbr_idx, float* nbr_rel,
                void* stream)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_rollout: NULL handle");
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(MDG_ERR_CUDA, "mdg_rollout: cannot select device %d", h->device);
    if (h->n_drones == 0) return MDG_OK;
    mdg::RolloutArgs r;
    int rc = rollout_args(h, state, actions, action_per_step, action_type, n_substeps, K, obs_mode, kin, nbr_idx,
                          nbr_rel, &r);
    if (rc != MDG_OK) return rc;
    cudaError_t e = enqueue_rollout(h, r, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_rollout: launch");
    return MDG_OK;
}

struct mdg_graph_s {
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

int mdg_rollout_graph_create(mdg_handle h, float* state, const float* actions, int32_t action_per_step,
                             int32_t action_type, int32_t n_substeps, int32_t K, int32_t obs_mode, float* kin,
                             int32_t* nbr_idx, float* nbr_rel, mdg_graph* out)
{
    if (!out) return fail(MDG_ERR_ARG, "mdg_rollout_graph_create: out is NULL");
    *out = nullptr;
    if (!h) return fail(MDG_ERR_ARG, "mdg_rollout_graph_create: NULL handle");
    DeviceGuard dg(h->device);
    if (!dg.ok) return fail(MDG_ERR_CUDA, "mdg_rollout_graph_create: cannot select device %d", h->device);
    mdg::RolloutArgs r{};
    if (h->n_drones > 0) {
        int rc = rollout_args(h, state, actions, action_per_step, action_type, n_substeps, K, obs_mode, kin, nbr_idx,
                              nbr_rel, &r);
        if (rc != MDG_OK) return rc;
    }
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_rollout_graph_create: stream");
    mdg_graph g = new mdg_graph_s();
    g->device = h->device;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = h->n_drones > 0 ? enqueue_rollout(h, r, cs) : cudaSuccess;
        e = cudaStreamEndCapture(cs, &g->graph);
        if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return cuda_fail(e, "mdg_rollout_graph_create: capture");
    }
    *out = g;
    return MDG_OK;
}

int mdg_graph_launch(mdg_graph g, void* stream)
{
    if (!g) return fail(MDG_ERR_ARG, "mdg_graph_launch: NULL graph");
    DeviceGuard dg(g->device);
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mdg_graph_launch");
    return MDG_OK;
}

int mdg_graph_destroy(mdg_graph g)
{
    if (!g) return MDG_OK;
    DeviceGuard dg(g->device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return MDG_OK;
}

int mdg_autotune(mdg_handle h, float* state, const float* actions, int32_t action_per_step, int32_t action_type,
                 int32_t n_substeps, int32_t K, void* stream, int32_t* best_block, float* best_ms)
{
    if (!h) return fail(MDG_ERR_ARG, "mdg_autotune: NULL handle");
    if (K < 0) return fail(MDG_ERR_ARG, "mdg_autotune: K = %d < 0", K);
    if (h->n_drones == 0) {
        if (best_block) *best_block = h->block;
        return MDG_OK;
    }
    int rc;
    if ((rc = check_state_ptr(h, state, "state")) != MDG_OK) return rc;
    if ((rc = check_state_ptr(h, actions, "actions")) != MDG_OK) return rc;
    DeviceGuard dg(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t state_bytes = (size_t)MDG_STATE_PLANES * 16 * h->n_drones;
    float* saved = nullptr;
    float* kin = nullptr;
    int32_t* idx = nullptr;
    float* rel = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    const int original = h->block, orig_sched = h->sched, orig_cap = h->item_cap;
    int best = original, best_sched = orig_sched, best_cap = orig_cap;
    float best_t = 1e30f;
    if ((e = cudaMalloc(&saved, state_bytes)) != cudaSuccess || (e = cudaMalloc(&kin, 80 * h->n_drones)) != cudaSuccess ||
        (e = cudaMalloc(&idx, 16 * h->n_drones)) != cudaSuccess || (e = cudaMalloc(&rel, 96 * h->n_drones)) != cudaSuccess ||
        (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess ||
        (e = cudaMemcpyAsync(saved, state, state_bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
        rc = cuda_fail(e, "mdg_autotune: scratch");
    } else {
        int lo = 32;
        while (lo < h->max_env) lo += 32;
        // candidates: block sizes; for rollouts also the schedule (work counter or static) and,
        // for uneven batches, the item cap (the block, half of it, a quarter of it; never below
        // the largest environment or one warp)
        struct Cand {
            int block, sched, cap;
        };
        std::vector<Cand> cands;
        for (int b = lo; b <= 1024; b = b < 64 ? 64 : b * 2) {
            if (K == 0) {
                cands.push_back({b, orig_sched, orig_cap});
                continue;
            }
            std::vector<int> caps = {0};
            if (h->uniform_N <= 0)
                for (int c = b / 2; c >= std::max(32, h->max_env) && c >= b / 4; c /= 2) caps.push_back(c);
            for (int c : caps)
                for (int sm : {MDG_SCHED_DYNAMIC, MDG_SCHED_STATIC}) cands.push_back({b, sm, c});
        }
        for (size_t ci = 0; ci < cands.size() && rc == MDG_OK; ++ci) {
            const int b = cands[ci].block;
            if ((rc = set_block(h, b)) != MDG_OK) break;
            h->sched = cands[ci].sched;
            h->item_cap = cands[ci].cap;
            float total = 0.f;
            for (int rep = 0; rep < 7 && rc == MDG_OK; ++rep) {
                e = cudaMemcpyAsync(state, saved, state_bytes, cudaMemcpyDeviceToDevice, s);
                if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "mdg_autotune");
                    break;
                }
                if (K == 0)
                    rc = step_common(h, state, actions, action_type, n_substeps, kin, idx, rel, true, stream);
                else
                    rc = mdg_rollout(h, state, actions, action_per_step, action_type, n_substeps, K, MDG_OBS_LAST, kin,
                                     idx, rel, stream);
                if (rc != MDG_OK) break;
                if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
                    rc = cuda_fail(e, "mdg_autotune: timing");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep >= 2) total += ms;  // two warm-up launches per candidate
            }
            if (rc == MDG_OK && total / 5 < best_t) {
                best_t = total / 5;
                best = b;
                best_sched = cands[ci].sched;
                best_cap = cands[ci].cap;
            }
        }
        if (rc == MDG_OK) {
            rc = set_block(h, best);
            h->sched = best_sched;
            h->item_cap = best_cap;
        } else {
            set_block(h, original);
            h->sched = orig_sched;
            h->item_cap = orig_cap;
        }
        cudaMemcpyAsync(state, saved, state_bytes, cudaMemcpyDeviceToDevice, s);
        cudaStreamSynchronize(s);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(saved);
    cudaFree(kin);
    cudaFree(idx);
    cudaFree(rel);
    if (rc == MDG_OK) {
        if (best_block) *best_block = best;
        if (best_ms) *best_ms = best_t;
    }
    return rc;
}

const char* mdg_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
