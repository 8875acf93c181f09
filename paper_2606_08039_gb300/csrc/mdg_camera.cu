// Camera frames by ray casting (the RGB observation of Section 3.4.4: 48 x 64 frames from
// each drone's onboard camera, 60 degree field of view, at [0.02, 0, 0] in the body frame).
// The paper renders them with MuJoCo's OpenGL renderer and the Crazyflie meshes; here every
// frame is ray cast in a kernel from primitive shapes:
//   - pinhole camera along body +x, image right = body -y, image up = body +z, 60 degrees
//     the vertical field of view, each pixel through the centre of its cell, row 0 on top;
//   - the environment's other drones as oblate ellipsoids in their body frames, semi-axes
//     (L + r_p, L + r_p, 0.3 (L + r_p)); the ground z = 0 as a 0.5 m checkerboard seen from
//     above; the camera's own drone is not drawn;
//   - Lambert shading, ambient 0.35 + diffuse 0.65 max(0, n . l), l along (0.3, 0.2, 1);
//     ground greys 0.55 / 0.35, drone k coloured by the palette entry k mod 8, sky
//     (0.55, 0.70, 0.90) unshaded; channels round(255 c), alpha 255;
//   - depth along the optical axis to the nearest hit beyond 1e-4 m (+inf: sky);
//     segmentation -1 sky, 0 ground, 1 + the global index of the drone hit.
// One 128-thread block per camera; the block first builds, in shared memory, each drone's
// ray transform (world direction -> the drone's scaled body frame), the camera origin in
// that frame, the normal transform and the drone's screen rectangle, and then for each
// 32-pixel segment (half a row: one warp's pixels) the mask of drones whose rectangles it
// meets; a pixel pays a ~25-flop ray-ellipsoid test only for the drones of its segment's
// mask (above 64 drones per environment, the rectangles are tested per drone); each thread
// renders 24 pixels, consecutive threads consecutive pixels (coalesced stores). Small blocks
// keep eight cameras in flight per SM, so that one camera's setup overlaps others' pixels.
#include "mdg_internal.cuh"

namespace mdg {
namespace {

constexpr int kCamH = 48, kCamW = 64, kCamPixels = kCamH * kCamW;
constexpr int kCamThreads = 128;
constexpr float kTMin = 1e-4f;
// unit light direction (0.3, 0.2, 1) / |(0.3, 0.2, 1)|
constexpr float kLx = 0.28221626f, kLy = 0.18814417f, kLz = 0.94072087f;

__constant__ float c_palette[8][3] = {{0.90f, 0.25f, 0.20f}, {0.20f, 0.70f, 0.30f}, {0.20f, 0.35f, 0.90f},
                                      {0.95f, 0.75f, 0.15f}, {0.70f, 0.30f, 0.80f}, {0.15f, 0.75f, 0.80f},
                                      {0.95f, 0.50f, 0.20f}, {0.60f, 0.60f, 0.65f}};

// Per drone of the environment, in shared memory, seven float4 (a ray test reads the first
// four): O = the camera origin in the drone's scaled body frame, M = diag(1/s) R^T (world
// ray -> scaled body ray, row r in float4 1 + r), C = |O|^2 - 1, Nm = R diag(1/s) (scaled
// body point -> world normal direction), its segment id, and the pixel rectangle
// [r0, r1] x [c0, c1] outside which no ray can meet it (the projection of its oriented
// bounding box, half-extents (a, a, c) along its body axes, padded by a pixel; empty when
// its bounding cube of half-width a lies behind the camera or beyond a side plane of the
// view frustum, or for the camera's own drone; the whole image when the cube straddles the
// image plane inside the frustum):
//   0: O0 O1 O2 C      1: M00 M01 M02 Nm0   2: M10 M11 M12 Nm1   3: M20 M21 M22 Nm2
//   4: Nm3 Nm4 Nm5 Nm6   5: Nm7 Nm8 id r0   6: r1 c0 c1 -
constexpr int kSceneF4 = 7;

// Square root and reciprocal of the special function unit (relative error near 2^-23): the
// hit distance of a ray-ellipsoid test, well inside the depth tolerance.
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct Rot {
    float m[9];  // row-major, body -> world
};

__device__ __forceinline__ Rot rot_of(float w, float x, float y, float z)
{
    Rot R;
    R.m[0] = 1.f - 2.f * (y * y + z * z);
    R.m[1] = 2.f * (x * y - w * z);
    R.m[2] = 2.f * (x * z + w * y);
    R.m[3] = 2.f * (x * y + w * z);
    R.m[4] = 1.f - 2.f * (x * x + z * z);
    R.m[5] = 2.f * (y * z - w * x);
    R.m[6] = 2.f * (x * z - w * y);
    R.m[7] = 2.f * (y * z + w * x);
    R.m[8] = 1.f - 2.f * (x * x + y * y);
    return R;
}

__global__ void __launch_bounds__(kCamThreads) render_kernel(const CamArgs a)
{
    extern __shared__ float4 s_scene[];  // [max_env][kSceneF4]
    __shared__ int s_env[2];             // first drone of the camera's environment, its size
    __shared__ unsigned long long s_mask[kCamPixels / 32];  // per 32-pixel segment: drones it may see (N <= 64)
    __shared__ float s_cam[3];           // camera origin
    __shared__ float s_R[9];             // the camera drone's rotation (body -> world)
    const int t = threadIdx.x;
    const float inv_a = 1.f / a.semi_a, inv_c = 1.f / a.semi_c;
    const float th = 0.57735026918962576f;  // tan(30 degrees)
    const float kInf = __int_as_float(0x7f800000);
    for (long long cam = blockIdx.x; cam < a.n; cam += gridDim.x) {
        __syncthreads();  // the previous camera's scene is no longer read
        if (t == 0) {
            int first, N;
            if (a.uniform_N > 0) {
                const long long e = cam / a.uniform_N;
                first = (int)(e * a.uniform_N);
                N = a.uniform_N;
            } else {
                int lo = 0, hi = a.n_envs - 1;  // largest env with env_off[env] <= cam
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (a.env_off[mid] <= cam) lo = mid;
                    else hi = mid - 1;
                }
                first = a.env_off[lo];
                N = a.env_off[lo + 1] - first;
            }
            if (!MDG_CHECK(N >= 1 && N <= a.max_env && cam >= first && cam < first + N, a.status)) N = 0;
            s_env[0] = first;
            s_env[1] = N;
            const float4 p0 = a.state[cam], p1 = a.state[a.n + cam];
            const Rot R = rot_of(p0.w, p1.x, p1.y, p1.z);
            for (int i = 0; i < 9; ++i) s_R[i] = R.m[i];
            s_cam[0] = p0.x + 0.02f * R.m[0];
            s_cam[1] = p0.y + 0.02f * R.m[3];
            s_cam[2] = p0.z + 0.02f * R.m[6];
        }
        __syncthreads();
        const int first = s_env[0], N = s_env[1];
        const float ox = s_cam[0], oy = s_cam[1], oz = s_cam[2];
        const int own_k = (int)(cam - first);
        for (int k = t; k < N; k += kCamThreads) {
            const long long g = first + k;
            const float4 p0 = a.state[g], p1 = a.state[a.n + g];
            const Rot R = rot_of(p0.w, p1.x, p1.y, p1.z);
            const float inv_s[3] = {inv_a, inv_a, inv_c};
            const float dx = ox - p0.x, dy = oy - p0.y, dz = oz - p0.z;
            float4* sc = s_scene + k * kSceneF4;
            float O[3], M[9], Nm[9];
            float C = -1.f;
            for (int r = 0; r < 3; ++r) {
                // row r of R^T is column r of R
                O[r] = (R.m[r] * dx + R.m[3 + r] * dy + R.m[6 + r] * dz) * inv_s[r];
                C += O[r] * O[r];
                M[3 * r + 0] = R.m[r] * inv_s[r];
                M[3 * r + 1] = R.m[3 + r] * inv_s[r];
                M[3 * r + 2] = R.m[6 + r] * inv_s[r];
            }
            for (int r = 0; r < 3; ++r)
                for (int q = 0; q < 3; ++q) Nm[3 * r + q] = R.m[3 * r + q] * inv_s[q];
            sc[0] = make_float4(O[0], O[1], O[2], C);
            sc[1] = make_float4(M[0], M[1], M[2], Nm[0]);
            sc[2] = make_float4(M[3], M[4], M[5], Nm[1]);
            sc[3] = make_float4(M[6], M[7], M[8], Nm[2]);
            sc[4] = make_float4(Nm[3], Nm[4], Nm[5], Nm[6]);
            const float seg_id = __int_as_float((int)(g + 1));
            // screen rectangle: the drone's centre in the camera drone's body frame
            const float ex = p0.x - ox, ey = p0.y - oy, ez = p0.z - oz;
            const float X = s_R[0] * ex + s_R[3] * ey + s_R[6] * ez;
            const float Y = s_R[1] * ex + s_R[4] * ey + s_R[7] * ez;
            const float Z = s_R[2] * ex + s_R[5] * ey + s_R[8] * ez;
            const float rho = a.semi_a;
            int r0 = 0, r1 = kCamH - 1, c0 = 0, c1 = kCamW - 1;
            // outside the view frustum: behind the camera, or beyond one of its four side
            // planes |nx| <= hx, |ny| <= hy (padded by two pixels); for a linear test the cube's
            // worst corner is the centre's value minus rho times the sum of |coefficients|
            const float hx = th * kCamW / kCamH * (1.f + 4.f / kCamW), hy = th * (1.f + 4.f / kCamH);
            const bool unseen = X + rho < 0.f || (-Y - hx * X) - rho * (1.f + hx) > 0.f ||
                                (Y - hx * X) - rho * (1.f + hx) > 0.f || (Z - hy * X) - rho * (1.f + hy) > 0.f ||
                                (-Z - hy * X) - rho * (1.f + hy) > 0.f;
            if (unseen) {
                r0 = 1, r1 = 0;  // empty
            } else if (X - rho > 1e-3f) {
                // the corners of the drone's own bounding box, half-extents (a, a, c) along its
                // body axes, in the camera drone's body frame: G = R_cam^T R_k (column q = the
                // drone's axis q) scaled by the half-extent
                float G[9];
                for (int r = 0; r < 3; ++r)
                    for (int q = 0; q < 3; ++q)
                        G[3 * r + q] = (s_R[r] * R.m[q] + s_R[3 + r] * R.m[3 + q] + s_R[6 + r] * R.m[6 + q]) *
                                       (q == 2 ? a.semi_c : a.semi_a);
                float nx_lo = 1e30f, nx_hi = -1e30f, ny_lo = 1e30f, ny_hi = -1e30f;
                for (int corner = 0; corner < 8; ++corner) {
                    const float sx = (corner & 1) ? 1.f : -1.f, sy = (corner & 2) ? 1.f : -1.f;
                    const float sz = (corner & 4) ? 1.f : -1.f;
                    const float cx = X + sx * G[0] + sy * G[1] + sz * G[2];
                    const float cy = Y + sx * G[3] + sy * G[4] + sz * G[5];
                    const float cz = Z + sx * G[6] + sy * G[7] + sz * G[8];
                    const float ic = __fdividef(1.f, cx);  // the rectangle's padding covers its error
                    const float nxc = -cy * ic, nyc = cz * ic;
                    nx_lo = fminf(nx_lo, nxc);
                    nx_hi = fmaxf(nx_hi, nxc);
                    ny_lo = fminf(ny_lo, nyc);
                    ny_hi = fmaxf(ny_hi, nyc);
                }
                // col = ((nx / (th W/H)) + 1) W/2 - 0.5, row = (1 - ny / th) H/2 - 0.5
                const float kx = 0.5f * kCamW / (th * kCamW / kCamH), ky = 0.5f * kCamH / th;
                c0 = max(0, (int)floorf((nx_lo * kx + 0.5f * kCamW - 0.5f)) - 1);
                c1 = min(kCamW - 1, (int)ceilf((nx_hi * kx + 0.5f * kCamW - 0.5f)) + 1);
                r0 = max(0, (int)floorf((0.5f * kCamH - ny_hi * ky - 0.5f)) - 1);
                r1 = min(kCamH - 1, (int)ceilf((0.5f * kCamH - ny_lo * ky - 0.5f)) + 1);
            }
            if (k == own_k) r0 = 1, r1 = 0;  // the camera's own drone: empty
            sc[5] = make_float4(Nm[7], Nm[8], seg_id, __int_as_float(r0));
            sc[6] = make_float4(__int_as_float(r1), __int_as_float(c0), __int_as_float(c1), 0.f);
        }
        __syncthreads();
        if (N == 0) continue;
        // per 32-pixel segment (half a row, one warp's pixels), the drones whose screen
        // rectangles it meets
        if (N <= 64) {
            for (int sgm = t; sgm < kCamPixels / 32; sgm += kCamThreads) {
                const int row = sgm >> 1, sc0 = (sgm & 1) * 32, sc1 = sc0 + 31;
                unsigned long long m = 0;
                for (int k = 0; k < N; ++k) {
                    const float4 q5 = s_scene[k * kSceneF4 + 5], q6 = s_scene[k * kSceneF4 + 6];
                    const bool meets = row >= __float_as_int(q5.w) && row <= __float_as_int(q6.x) &&
                                       sc1 >= __float_as_int(q6.y) && sc0 <= __float_as_int(q6.z);
                    m |= (unsigned long long)meets << k;
                }
                s_mask[sgm] = m;
            }
            __syncthreads();
        }
        for (int p = t; p < kCamPixels; p += kCamThreads) {
            const int row = p / kCamW, col = p % kCamW;
            const float nx = ((col + 0.5f) * (2.f / kCamW) - 1.f) * (th * kCamW / kCamH);
            const float ny = (1.f - (row + 0.5f) * (2.f / kCamH)) * th;
            // world direction of the body ray (1, -nx, ny), not normalised: its component along
            // the optical axis is 1, so the ray parameter t of a hit is its depth along the axis
            // (the minimum distance 1e-4 m is then taken along that axis)
            const float d0 = s_R[0] - nx * s_R[1] + ny * s_R[2];
            const float d1 = s_R[3] - nx * s_R[4] + ny * s_R[5];
            const float d2 = s_R[6] - nx * s_R[7] + ny * s_R[8];
            float t_best = kInf;
            int hit = -1;  // -1 sky, -2 ground, else the drone slot
            if (oz > 0.f && d2 < 0.f) {
                const float tg = -oz * __frcp_rn(d2);
                if (tg > kTMin) {
                    t_best = tg;
                    hit = -2;
                }
            }
            // a warp covers 32 pixels of one row: its candidates are the segment's mask (the same
            // for all its lanes); above 64 drones, the rectangles are tested per drone
            const int wc0 = col & ~31, wc1 = wc0 + 31;
            unsigned long long cand = N <= 64 ? s_mask[p >> 5] : ~0ull;
            for (int k = 0; k < N; ++k) {
                if (N <= 64) {
                    if (!cand) break;
                    k = __ffsll((long long)cand) - 1;
                    cand &= cand - 1;
                }
                const float4* sc = s_scene + k * kSceneF4;
                if (N > 64) {
                    const float4 q5 = sc[5], q6 = sc[6];
                    if (row < __float_as_int(q5.w) || row > __float_as_int(q6.x) || wc1 < __float_as_int(q6.y) ||
                        wc0 > __float_as_int(q6.z))
                        continue;  // outside the drone's screen rectangle (also: the camera's own drone)
                }
                const float4 o = sc[0], m0 = sc[1], m1 = sc[2], m2 = sc[3];
                const float D0 = m0.x * d0 + m0.y * d1 + m0.z * d2;
                const float D1 = m1.x * d0 + m1.y * d1 + m1.z * d2;
                const float D2 = m2.x * d0 + m2.y * d1 + m2.z * d2;
                const float A = D0 * D0 + D1 * D1 + D2 * D2;
                const float B = 2.f * (D0 * o.x + D1 * o.y + D2 * o.z);
                const float disc = B * B - 4.f * A * o.w;
                if (disc < 0.f) continue;
                const float sq = sqrt_approx(disc), i2a = 0.5f * rcp_approx(A);
                const float t1 = (-B - sq) * i2a, t2 = (-B + sq) * i2a;
                const float tk = t1 > kTMin ? t1 : (t2 > kTMin ? t2 : kInf);
                if (tk < t_best) {
                    t_best = tk;
                    hit = k;
                }
            }
            float r = 0.55f, gcol = 0.70f, b = 0.90f;  // sky
            int seg = -1;
            if (hit == -2) {
                const float px = ox + t_best * d0, py = oy + t_best * d1;
                const int par = ((int)floorf(px * 2.f) + (int)floorf(py * 2.f)) & 1;
                const float shade = 0.35f + 0.65f * kLz;  // normal +z
                const float grey = par ? 0.35f : 0.55f;
                r = gcol = b = grey * shade;
                seg = 0;
            } else if (hit >= 0) {
                const float4* sc = s_scene + hit * kSceneF4;
                const float4 o = sc[0], m0 = sc[1], m1 = sc[2], m2 = sc[3], q4 = sc[4], q5 = sc[5];
                const float D0 = m0.x * d0 + m0.y * d1 + m0.z * d2;
                const float D1 = m1.x * d0 + m1.y * d1 + m1.z * d2;
                const float D2 = m2.x * d0 + m2.y * d1 + m2.z * d2;
                const float P0 = o.x + t_best * D0, P1 = o.y + t_best * D1, P2 = o.z + t_best * D2;
                float n0 = m0.w * P0 + m1.w * P1 + m2.w * P2;
                float n1 = q4.x * P0 + q4.y * P1 + q4.z * P2;
                float n2 = q4.w * P0 + q5.x * P1 + q5.y * P2;
                const float in = rsqrtf(fmaxf(n0 * n0 + n1 * n1 + n2 * n2, 1e-30f));
                const float nl = (n0 * kLx + n1 * kLy + n2 * kLz) * in;
                const float shade = 0.35f + 0.65f * fmaxf(0.f, nl);
                const int id = __float_as_int(q5.z);
                const int pc = (id - 1) & 7;
                r = c_palette[pc][0] * shade;
                gcol = c_palette[pc][1] * shade;
                b = c_palette[pc][2] * shade;
                seg = id;
            }
            const long long o = cam * kCamPixels + p;
            if (a.rgba) {
                const int R8 = __float2int_rn(255.f * __saturatef(r));
                const int G8 = __float2int_rn(255.f * __saturatef(gcol));
                const int B8 = __float2int_rn(255.f * __saturatef(b));
                a.rgba[o] = make_uchar4((unsigned char)R8, (unsigned char)G8, (unsigned char)B8, 255);
            }
            if (a.depth) a.depth[o] = t_best;  // +inf for sky
            if (a.seg) a.seg[o] = seg;
        }
    }
}

}  // namespace

cudaError_t launch_render(const CamArgs& a, cudaStream_t s)
{
    if (a.n == 0) return cudaSuccess;
    const int smem = a.max_env * kSceneF4 * (int)sizeof(float4);
    static int opted = 0;
    if (smem > 48 * 1024 && smem > opted) {
        cudaError_t e = cudaFuncSetAttribute(render_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        opted = smem;
    }
    const long long grid = a.n < 152LL * 64 ? a.n : 152LL * 64;
    render_kernel<<<(unsigned)grid, kCamThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mdg
