// Keyframe depth fusion, Eq. 1 (Section 3 "Keyframe Fusion").
//
// Each valid, non-discontinuity pixel x of frame i is warped into the keyframe,
// p* = g(T*^-1, g(T_i, pi^-1(x, Z_i(x)))), rounded to its nearest keyframe pixel
// x*, and accumulated as sum(w_z Z*_p) and sum(w_z) with w_z = cos(theta) / Z^2.
// Applying Eq. 1 sequentially gives exactly that ratio of sums, so the kernel
// scatters both sums with float atomics (order-free up to rounding) and a second
// pass divides.  One thread per 4 pixels of a frame row; up to 64 frames per launch.
#include <cmath>
#include <mutex>
#include <vector>

#include "volume.cuh"

namespace {

constexpr int FUSE_MAX_FRAMES = 64;  // frames per launch (kernel parameter space)

// a*b - c*d with one rounding error (fma-compensated, W. Kahan): the normal's
// components cancel strongly for surfaces seen at grazing angles
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    const float w = c * d;
    const float e = fmaf(-c, d, w);
    const float f = fmaf(a, b, -w);
    return f + e;
}
constexpr int FUSE_TX = 32, FUSE_TY = 8;

struct FuseFrame {
    float R[9];  // keyframe_from_frame rotation  R*^T R_i
    float t[3];  // keyframe_from_frame translation R*^T (t_i - t*)
    int kf;      // output keyframe image
};

struct FuseArgs {
    FuseFrame f[FUSE_MAX_FRAMES];
};

// process-wide timing of the fusion launches (sc_fusion_profile)
struct FuseProf {
    std::mutex mu;
    bool on = false;
    std::vector<cudaEvent_t> ev;  // pairs around each fuse_kernel launch
    std::vector<int> frames;
    double ms = 0.0;
    int64_t launches = 0, nframes = 0;
} g_fprof;

cudaEvent_t fprof_event(cudaStream_t s) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    cudaEventRecord(e, s);
    return e;
}

struct FuseCam {
    float fx, fy, cx, cy, ifx, ify;  // ifx = 1/fx, ify = 1/fy
    int W, H;
    float disc_rel;
    float* S;     // sum w_z Z*_p (in the Z* output until normalised)
    float* Wsum;  // sum w_z (the W* output)
};

// Eq. 1 contribution of one frame pixel (u, v) with depth z and 4-neighbours.
__device__ __forceinline__ void fuse_pixel(const FuseFrame& F, const FuseCam& c, int u, int v, float z, float zl,
                                           float zr, float zu, float zd, float* S, float* Wsum) {
    if (!(z > 0.f)) return;
    if (!(zl > 0.f && zr > 0.f && zu > 0.f && zd > 0.f)) return;
    const float lim = c.disc_rel * z;
    if (fabsf(zl - z) > lim || fabsf(zr - z) > lim || fabsf(zu - z) > lim || fabsf(zd - z) > lim) return;
    // warp into the keyframe
    const float xn = (u - c.cx) * c.ifx, yn = (v - c.cy) * c.ify;
    const float P[3] = {xn * z, yn * z, z};
    float ps[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) ps[r] = fmaf(F.R[3 * r], P[0], fmaf(F.R[3 * r + 1], P[1], fmaf(F.R[3 * r + 2], P[2], F.t[r])));
    if (!(ps[2] > 0.f)) return;
    // approximate reciprocal (2 ulp): a few 1e-5 px at the nearest-pixel rounding
    const float rz = __fdividef(1.f, ps[2]);
    const float uu = fmaf(c.fx * ps[0], rz, c.cx) + 0.5f;
    const float vv = fmaf(c.fy * ps[1], rz, c.cy) + 0.5f;
    if (!(uu >= 0.f && uu < (float)c.W && vv >= 0.f && vv < (float)c.H)) return;
    const size_t q = (size_t)F.kf * c.W * c.H + (size_t)(int)vv * c.W + (int)uu;
    // w_z = cos(theta) / Z^2, theta from the central-difference normal
    // a = P(u+1,v) - P(u-1,v), b = P(u,v+1) - P(u,v-1), written as
    // x (z_r - z_l) + (z_r + z_l) / fx etc. so that no large terms cancel
    const float dzx = zr - zl, dzy = zd - zu;
    const float ax = fmaf(xn, dzx, (zr + zl) * c.ifx);
    const float ay = yn * dzx;
    const float az = dzx;
    const float bx = xn * dzy;
    const float by = fmaf(yn, dzy, (zd + zu) * c.ify);
    const float bz = dzy;
    const float nx = diff_of_products(ay, bz, az, by), ny = diff_of_products(az, bx, ax, bz),
                nz = diff_of_products(ax, by, ay, bx);
    const float n2 = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
    if (!(n2 > 0.f)) return;
    const float w = __fdividef(fabsf(nz) * rsqrtf(n2), z * z);
    atomicAdd(S + q, w * ps[2]);
    atomicAdd(Wsum + q, w);
}

// One thread per 4 consecutive pixels of a row (u0 = 4 * thread): the row and its two
// neighbour rows come in as float4 loads plus the two pixels beyond the ends.
// Border pixels have no full neighbourhood and are skipped.  Width multiple of 4.
__global__ void __launch_bounds__(FUSE_TX* FUSE_TY) fuse_kernel(const float* __restrict__ depths, FuseArgs a,
                                                                 FuseCam c) {
    const int W = c.W, H = c.H;
    const int u0 = 4 * (blockIdx.x * FUSE_TX + threadIdx.x);
    const int v = blockIdx.y * FUSE_TY + threadIdx.y;
    if (u0 >= W || v < 1 || v >= H - 1) return;
    const FuseFrame F = a.f[blockIdx.z];
    const float* Z = depths + (size_t)blockIdx.z * W * H + (size_t)v * W + u0;
    const float4 row = __ldg(reinterpret_cast<const float4*>(Z));
    const float4 up = __ldg(reinterpret_cast<const float4*>(Z - W));
    const float4 dn = __ldg(reinterpret_cast<const float4*>(Z + W));
    const float left = u0 > 0 ? __ldg(Z - 1) : 0.f;
    const float right = u0 + 4 < W ? __ldg(Z + 4) : 0.f;
    float* S = c.S;
    float* Ws = c.Wsum;
    if (u0 > 0) fuse_pixel(F, c, u0, v, row.x, left, row.y, up.x, dn.x, S, Ws);
    fuse_pixel(F, c, u0 + 1, v, row.y, row.x, row.z, up.y, dn.y, S, Ws);
    fuse_pixel(F, c, u0 + 2, v, row.z, row.y, row.w, up.z, dn.z, S, Ws);
    if (u0 + 4 < W) fuse_pixel(F, c, u0 + 3, v, row.w, row.z, right, up.w, dn.w, S, Ws);
}

// Any width: one thread per pixel.
__global__ void __launch_bounds__(FUSE_TX* FUSE_TY) fuse_kernel_any(const float* __restrict__ depths, FuseArgs a,
                                                                     FuseCam c) {
    const int u = blockIdx.x * FUSE_TX + threadIdx.x;
    const int v = blockIdx.y * FUSE_TY + threadIdx.y;
    const int W = c.W, H = c.H;
    if (u < 1 || v < 1 || u >= W - 1 || v >= H - 1) return;
    const FuseFrame& F = a.f[blockIdx.z];
    const float* Z = depths + (size_t)blockIdx.z * W * H;
    const size_t p = (size_t)v * W + u;
    fuse_pixel(F, c, u, v, __ldg(Z + p), __ldg(Z + p - 1), __ldg(Z + p + 1), __ldg(Z + p - W), __ldg(Z + p + W), c.S,
               c.Wsum);
}

__global__ void fuse_normalise_kernel(float* Z, const float* Wsum, size_t n) {
    const size_t n4 = n / 4;  // both arrays 16-byte aligned
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        const float4 w = reinterpret_cast<const float4*>(Wsum)[i];
        float4 z = reinterpret_cast<float4*>(Z)[i];
        z.x = w.x > 0.f ? z.x / w.x : 0.f;
        z.y = w.y > 0.f ? z.y / w.y : 0.f;
        z.z = w.z > 0.f ? z.z / w.z : 0.f;
        z.w = w.w > 0.f ? z.w / w.w : 0.f;
        reinterpret_cast<float4*>(Z)[i] = z;
    }
    for (size_t i = 4 * n4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float w = Wsum[i];
        Z[i] = w > 0.f ? Z[i] / w : 0.f;
    }
}

// Fuse frames [0, n) into keyframe images; frame f goes to image frame_kf[f] at pose kf_poses[frame_kf[f]].
int fuse_impl(const float* depths, const sc_pose* frame_poses, const int32_t* frame_kf, int32_t n,
              const sc_pose* kf_poses, int32_t n_kf, const sc_intrinsics* K, const sc_fusion_params* fusion,
              float* kf_depth, float* kf_weight, cudaStream_t s) {
    if (!depths || !frame_poses || n < 1 || !kf_poses || n_kf < 1 || !sc::intrinsics_ok(K) || !fusion ||
        !kf_depth || !kf_weight || !(fusion->disc_rel >= 0.f))
        return SC_ERR_INVALID_ARG;
    if (((uintptr_t)depths & 15) || ((uintptr_t)kf_depth & 15) || ((uintptr_t)kf_weight & 15))
        return SC_ERR_INVALID_ARG;
    for (int f = 0; f < n; ++f) {
        if (frame_kf && (frame_kf[f] < 0 || frame_kf[f] >= n_kf)) return SC_ERR_INVALID_ARG;
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 4; ++q)
                if (!std::isfinite(frame_poses[f].m[r][q])) return SC_ERR_INVALID_ARG;
    }
    const int W = K->width, H = K->height;
    const size_t npx = (size_t)W * H;
    SC_CUDA(cudaMemsetAsync(kf_depth, 0, n_kf * npx * sizeof(float), s));
    SC_CUDA(cudaMemsetAsync(kf_weight, 0, n_kf * npx * sizeof(float), s));
    FuseCam c{K->fx, K->fy, K->cx, K->cy, (float)(1.0 / K->fx), (float)(1.0 / K->fy), W, H, fusion->disc_rel,
              kf_depth, kf_weight};
    for (int f0 = 0; f0 < n; f0 += FUSE_MAX_FRAMES) {
        const int nf = (n - f0) < FUSE_MAX_FRAMES ? (n - f0) : FUSE_MAX_FRAMES;
        FuseArgs a;
        for (int f = 0; f < nf; ++f) {
            const sc_pose& T = frame_poses[f0 + f];
            const int kf = frame_kf ? frame_kf[f0 + f] : 0;
            const sc_pose& Tk = kf_poses[kf];
            // keyframe_from_frame, composed in double and rounded once
            for (int r = 0; r < 3; ++r) {
                for (int q = 0; q < 3; ++q) {
                    double acc = 0;
                    for (int k = 0; k < 3; ++k) acc += (double)Tk.m[k][r] * (double)T.m[k][q];
                    a.f[f].R[3 * r + q] = (float)acc;
                }
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += (double)Tk.m[k][r] * ((double)T.m[k][3] - (double)Tk.m[k][3]);
                a.f[f].t[r] = (float)acc;
            }
            a.f[f].kf = kf;
        }
        dim3 block(FUSE_TX, FUSE_TY);
        cudaEvent_t e0 = nullptr;
        {
            std::lock_guard<std::mutex> lock(g_fprof.mu);
            if (g_fprof.on) e0 = fprof_event(s);
        }
        if (W % 4 == 0) {
            dim3 grid((W / 4 + FUSE_TX - 1) / FUSE_TX, (H + FUSE_TY - 1) / FUSE_TY, nf);
            fuse_kernel<<<grid, block, 0, s>>>(depths + (size_t)f0 * npx, a, c);
        } else {
            dim3 grid((W + FUSE_TX - 1) / FUSE_TX, (H + FUSE_TY - 1) / FUSE_TY, nf);
            fuse_kernel_any<<<grid, block, 0, s>>>(depths + (size_t)f0 * npx, a, c);
        }
        if (e0) {
            std::lock_guard<std::mutex> lock(g_fprof.mu);
            g_fprof.ev.push_back(e0);
            g_fprof.ev.push_back(fprof_event(s));
            g_fprof.frames.push_back(nf);
        }
        sc::count_launches(1);
        SC_CUDA(cudaGetLastError());
    }
    int dev = 0, sms = 148;
    SC_CUDA(cudaGetDevice(&dev));
    SC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    fuse_normalise_kernel<<<sms * 8, 256, 0, s>>>(kf_depth, kf_weight, n_kf * npx);
    sc::count_launches(1);
    SC_CUDA(cudaGetLastError());
    return SC_OK;
}

}  // namespace

extern "C" int sc_fusion_profile(int32_t enable, double* ms, int64_t* launches, int64_t* frames) {
    std::lock_guard<std::mutex> lock(g_fprof.mu);
    for (size_t i = 0; i + 1 < g_fprof.ev.size(); i += 2) {
        SC_CUDA(cudaEventSynchronize(g_fprof.ev[i + 1]));
        float t = 0.f;
        if (cudaEventElapsedTime(&t, g_fprof.ev[i], g_fprof.ev[i + 1]) == cudaSuccess) {
            g_fprof.ms += t;
            g_fprof.launches += 1;
            g_fprof.nframes += g_fprof.frames[i / 2];
        }
        cudaEventDestroy(g_fprof.ev[i]);
        cudaEventDestroy(g_fprof.ev[i + 1]);
    }
    g_fprof.ev.clear();
    g_fprof.frames.clear();
    if (ms) *ms = g_fprof.ms;
    if (launches) *launches = g_fprof.launches;
    if (frames) *frames = g_fprof.nframes;
    if (enable >= 0) {  // -1: read only; 0 / 1: reset and switch off / on
        g_fprof.on = enable != 0;
        g_fprof.ms = 0.0;
        g_fprof.launches = 0;
        g_fprof.nframes = 0;
    }
    return SC_OK;
}

extern "C" int sc_fuse_frames_into_keyframe(const float* depths, const sc_pose* frame_poses, int32_t n,
                                            const sc_pose* kf_pose, const sc_intrinsics* K,
                                            const sc_fusion_params* fusion, float* kf_depth, float* kf_weight,
                                            sc_stream stream) {
    return fuse_impl(depths, frame_poses, nullptr, n, kf_pose, 1, K, fusion, kf_depth, kf_weight,
                     (cudaStream_t)stream);
}

extern "C" int sc_fuse_keyframes(const float* depths, const sc_pose* frame_poses, const int32_t* frame_kf,
                                 int32_t n_frames, const sc_pose* kf_poses, int32_t n_kf, const sc_intrinsics* K,
                                 const sc_fusion_params* fusion, float* kf_depth, float* kf_weight,
                                 sc_stream stream) {
    if (!frame_kf) return SC_ERR_INVALID_ARG;
    return fuse_impl(depths, frame_poses, frame_kf, n_frames, kf_poses, n_kf, K, fusion, kf_depth, kf_weight,
                     (cudaStream_t)stream);
}

// ------------------------------------------------------------ raw sensor depth ----

namespace {

// z = raw * scale (one float multiply, round to nearest), 0 stays 0 (invalid)
__global__ void depth_from_u16_kernel(const uint16_t* __restrict__ raw, size_t n, float scale, float* __restrict__ out) {
    const size_t n8 = n / 8;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n8; i += (size_t)gridDim.x * blockDim.x) {
        const uint4 r = __ldg(reinterpret_cast<const uint4*>(raw) + i);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
        float4* o = reinterpret_cast<float4*>(out) + 2 * i;
        o[0] = make_float4(__fmul_rn((float)(w[0] & 0xffffu), scale), __fmul_rn((float)(w[0] >> 16), scale),
                           __fmul_rn((float)(w[1] & 0xffffu), scale), __fmul_rn((float)(w[1] >> 16), scale));
        o[1] = make_float4(__fmul_rn((float)(w[2] & 0xffffu), scale), __fmul_rn((float)(w[2] >> 16), scale),
                           __fmul_rn((float)(w[3] & 0xffffu), scale), __fmul_rn((float)(w[3] >> 16), scale));
    }
    for (size_t i = n8 * 8 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __fmul_rn((float)raw[i], scale);
}

}  // namespace

extern "C" int sc_depth_from_u16(const uint16_t* raw, int64_t n, float scale, float* depth, sc_stream stream) {
    if (n < 0 || (n > 0 && (!raw || !depth)) || !(scale > 0.f) || !std::isfinite(scale)) return SC_ERR_INVALID_ARG;
    if (((uintptr_t)raw & 15) || ((uintptr_t)depth & 15)) return SC_ERR_INVALID_ARG;
    if (n == 0) return SC_OK;
    int dev = 0, sms = 0;
    SC_CUDA(cudaGetDevice(&dev));
    SC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    depth_from_u16_kernel<<<sms * 8, 256, 0, (cudaStream_t)stream>>>(raw, (size_t)n, scale, depth);
    sc::count_launches(1);
    SC_CUDA(cudaGetLastError());
    return SC_OK;
}
