// Keyframe depth fusion, Eq. 1 (Section 3 "Keyframe Fusion").
//
// Each valid, non-discontinuity pixel x of frame i is warped into the keyframe,
// p* = g(T*^-1, g(T_i, pi^-1(x, Z_i(x)))), rounded to its nearest keyframe pixel
// x*, and accumulated as sum(w_z Z*_p) and sum(w_z) with w_z = cos(theta) / Z^2.
// Applying Eq. 1 sequentially gives exactly that ratio of sums, so the kernel
// scatters both sums, interleaved per keyframe pixel, with one 8-byte vector float
// atomic per pixel (order-free up to rounding) into pooled scratch, and a second pass
// divides and writes Z* and W*.  A frame taken at the keyframe's own pose (the first
// of a KF_CONST group) maps every pixel onto itself, so it initialises the sums with
// plain stores, which also replaces zeroing them.  One thread per 4 pixels of a frame
// row; up to 576 frames per launch (fewer launches, fewer partly filled last waves:
// the 540 scattered frames of 60 keyframes take 1 launch, against 2 of up to 512 frames
// and 9 of up to 64).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "volume.cuh"

namespace {

// frames per launch: 56 B each; 576 of them and the other arguments (56 B) fill 32,312 of
// the 32,764 bytes of kernel parameters
constexpr int FUSE_MAX_FRAMES = 576;

constexpr int FUSE_TX = 32, FUSE_TY = 8;


struct FuseFrame {
    float Pr[9];  // keyframe_from_frame rotation R*^T R_i, rows 0 and 1 scaled by fx and fy
    float t[3];   // keyframe_from_frame translation R*^T (t_i - t*), scaled likewise
    int kf;       // output keyframe image
    int src;      // input frame index
};

// Frames whose pose is the keyframe's own (the first frame of a KF_CONST group, R6):
// their warp is the identity, x* = x and Z*_p = z (exactly, in float as in exact
// arithmetic), so each keyframe's first such frame initialises the sums with plain
// stores instead of a memset followed by atomics.
constexpr int FUSE_MAX_INIT = 1024;  // keyframe images per init launch (kernel parameter space)
struct FuseInit {
    int src[FUSE_MAX_INIT];  // per keyframe image: its identity frame, or -1 (the sums start at zero)
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
    float cx, cy, ifx, ify;  // ifx = 1/fx, ify = 1/fy
    float cxh, cyh;          // cx + 1/2, cy + 1/2: nearest pixel by one floor
    int W, H;
    float disc_rel;
    float2* acc;  // per keyframe pixel (sum w_z Z*_p, sum w_z), interleaved
};

// floor(x) for 0 <= x < 2^23 without a conversion instruction (adding 2^23 rounded
// down leaves floor(x) in the low mantissa bits); every other x, inf and NaN included,
// lands outside [0, 2^23), so "(unsigned) fuse_floor(x) < size" is the range test too
__device__ __forceinline__ int fuse_floor(float x) { return __float_as_int(__fadd_rd(x, 8388608.f)) - 0x4b000000; }

// Eq. 1 contribution of one frame pixel with depth z and 4-neighbours at normalised
// image coordinates xn = (u - cx) / fx, yn = (v - cy) / fy; rb[r] = Pr[r][1] yn + Pr[r][2]
// is the part of the pixel's ray that its row shares.  All tests fold into one
// predicate, so a warp takes no divergent early exits; the two sums go out as one
// 8-byte vector atomic.
// Whether pixel depth z and its 4-neighbours pass the discontinuity test of Eq. 1's
// input: z valid and every neighbour valid and within disc_rel * z of it.  With
// disc_rel < 1 (NEAR) a neighbour within disc_rel * z of a valid z is itself valid
// (>= (1 - disc_rel) z > 0, and NaN fails the comparison), so its own test is implied.
template <bool NEAR>
__device__ __forceinline__ bool fuse_smooth(float disc_rel, float z, float zl, float zr, float zu, float zd) {
    const float lim = disc_rel * z;
    bool ok = z > 0.f;
    if (!NEAR) ok = ok && zl > 0.f && zr > 0.f && zu > 0.f && zd > 0.f;
    return ok && fabsf(zl - z) <= lim && fabsf(zr - z) <= lim && fabsf(zu - z) <= lim && fabsf(zd - z) <= lim;
}

// w_z = cos(theta) / z^2 of a pixel with depth z, theta from the normal n = a x b of
// the central differences
//   a = P(u+1,v) - P(u-1,v) = dzx (xn, yn, 1) + (A, 0, 0),  A = (z_r + z_l) / fx
//   b = P(u,v+1) - P(u,v-1) = dzy (xn, yn, 1) + (0, B, 0),  B = (z_d + z_u) / fy
// whose cross product expands to n = (-dzx B, -dzy A, A B + dzx B xn + dzy A yn): the
// dzx dzy xn yn terms of a_x b_y and a_y b_x cancel algebraically, not in float.
// Returns 0 when the normal is undefined (n = 0).
__device__ __forceinline__ float fuse_weight(const FuseCam& c, float xn, float yn, float z, float zl, float zr,
                                             float zu, float zd) {
    const float A = (zr + zl) * c.ifx, B = (zd + zu) * c.ify;
    const float m1 = (zr - zl) * B, m2 = (zd - zu) * A;
    const float nz = fmaf(m1, xn, fmaf(m2, yn, A * B));
    const float n2 = fmaf(m1, m1, fmaf(m2, m2, nz * nz));
    return n2 > 0.f ? __fdividef(fabsf(nz) * rsqrtf(n2), z * z) : 0.f;
}

template <bool NEAR>
__device__ __forceinline__ void fuse_pixel(const FuseFrame& F, const FuseCam& c, float xn, float yn,
                                           const float rb[3], float z, float zl, float zr, float zu, float zd,
                                           float2* acc) {
    bool ok = fuse_smooth<NEAR>(c.disc_rel, z, zl, zr, zu, zd);
    // warp into the keyframe: (fx X*, fy Y*, Z*) = z Pr (xn, yn, 1) + t, the pixel's ray
    // Pr (xn, yn, 1) formed first (one fma per row on top of the row's share)
    const float a0 = fmaf(F.Pr[0], xn, rb[0]);
    const float a1 = fmaf(F.Pr[3], xn, rb[1]);
    const float a2 = fmaf(F.Pr[6], xn, rb[2]);
    const float X = fmaf(a0, z, F.t[0]);
    const float Y = fmaf(a1, z, F.t[1]);
    const float Zs = fmaf(a2, z, F.t[2]);
    // approximate reciprocal (2 ulp): a few 1e-5 px at the nearest-pixel rounding
    const float rz = __fdividef(1.f, Zs);
    const int iu = fuse_floor(fmaf(X, rz, c.cxh));
    const int iv = fuse_floor(fmaf(Y, rz, c.cyh));
    ok = ok && Zs > 0.f && (unsigned)iu < (unsigned)c.W && (unsigned)iv < (unsigned)c.H;
    if (ok) {
        const float w = fuse_weight(c, xn, yn, z, zl, zr, zu, zd);
        if (w > 0.f) atomicAdd(acc + (iv * c.W + iu), make_float2(w * Zs, w));
    }
}

// One thread per 4 consecutive pixels of a row (u0 = 4 * thread): the row and its two
// neighbour rows come in as float4 loads plus the two pixels beyond the ends.
// Border pixels have no full neighbourhood and are skipped.  Width multiple of 4.
template <bool NEAR>
__global__ void __launch_bounds__(FUSE_TX* FUSE_TY) fuse_kernel(const float* __restrict__ depths, FuseArgs a,
                                                                 FuseCam c) {
    const int W = c.W, H = c.H;
    const int u0 = 4 * (blockIdx.x * FUSE_TX + threadIdx.x);
    const int v = blockIdx.y * FUSE_TY + threadIdx.y;
    if (u0 >= W || v < 1 || v >= H - 1) return;
    const FuseFrame& F = a.f[blockIdx.z];
    const size_t npx = (size_t)W * H;
    const float* Z = depths + (size_t)F.src * npx + (size_t)v * W + u0;
    const float4 row = __ldg(reinterpret_cast<const float4*>(Z));
    const float4 up = __ldg(reinterpret_cast<const float4*>(Z - W));
    const float4 dn = __ldg(reinterpret_cast<const float4*>(Z + W));
    const float left = u0 > 0 ? __ldg(Z - 1) : 0.f;     // 0: the first pixel has no left neighbour
    const float right = u0 + 4 < W ? __ldg(Z + 4) : 0.f;  // 0: the last pixel has no right neighbour
    float2* acc = c.acc + (size_t)F.kf * npx;
    // pixel coordinates stepped in float (exact integers): one conversion per thread
    const float uf = (float)u0;
    const float yn = ((float)v - c.cy) * c.ify;
    const float rb[3] = {fmaf(F.Pr[1], yn, F.Pr[2]), fmaf(F.Pr[4], yn, F.Pr[5]), fmaf(F.Pr[7], yn, F.Pr[8])};
    fuse_pixel<NEAR>(F, c, (uf - c.cx) * c.ifx, yn, rb, row.x, left, row.y, up.x, dn.x, acc);
    fuse_pixel<NEAR>(F, c, ((uf + 1.f) - c.cx) * c.ifx, yn, rb, row.y, row.x, row.z, up.y, dn.y, acc);
    fuse_pixel<NEAR>(F, c, ((uf + 2.f) - c.cx) * c.ifx, yn, rb, row.z, row.y, row.w, up.z, dn.z, acc);
    fuse_pixel<NEAR>(F, c, ((uf + 3.f) - c.cx) * c.ifx, yn, rb, row.w, row.z, right, up.w, dn.w, acc);
}

// The sums of keyframe images [k0, k0 + gridDim.z) initialised from each image's
// identity frame (or zero): every pixel is written, border pixels with zero.  One
// thread per 4 pixels of a row, two 16-byte stores.  Width multiple of 4.
template <bool NEAR>
__global__ void __launch_bounds__(FUSE_TX* FUSE_TY) fuse_init_kernel(const float* __restrict__ depths, FuseInit a,
                                                                      int k0, FuseCam c) {
    const int W = c.W, H = c.H;
    const int u0 = 4 * (blockIdx.x * FUSE_TX + threadIdx.x);
    const int v = blockIdx.y * FUSE_TY + threadIdx.y;
    if (u0 >= W || v >= H) return;
    const size_t npx = (size_t)W * H;
    const int src = a.src[blockIdx.z];
    float4* out = reinterpret_cast<float4*>(c.acc + (size_t)(k0 + blockIdx.z) * npx + (size_t)v * W + u0);
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (src >= 0 && v >= 1 && v < H - 1) {
        const float* Z = depths + (size_t)src * npx + (size_t)v * W + u0;
        const float4 row = __ldg(reinterpret_cast<const float4*>(Z));
        const float4 up = __ldg(reinterpret_cast<const float4*>(Z - W));
        const float4 dn = __ldg(reinterpret_cast<const float4*>(Z + W));
        const float left = u0 > 0 ? __ldg(Z - 1) : 0.f;
        const float right = u0 + 4 < W ? __ldg(Z + 4) : 0.f;
        const float z[6] = {left, row.x, row.y, row.z, row.w, right};
        const float zu[4] = {up.x, up.y, up.z, up.w}, zd[4] = {dn.x, dn.y, dn.z, dn.w};
        const float yn = ((float)v - c.cy) * c.ify;
        const float uf = (float)u0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!fuse_smooth<NEAR>(c.disc_rel, z[j + 1], z[j], z[j + 2], zu[j], zd[j])) continue;
            const float w = fuse_weight(c, ((uf + (float)j) - c.cx) * c.ifx, yn, z[j + 1], z[j], z[j + 2], zu[j], zd[j]);
            s[2 * j] = w * z[j + 1];
            s[2 * j + 1] = w;
        }
    }
    out[0] = make_float4(s[0], s[1], s[2], s[3]);
    out[1] = make_float4(s[4], s[5], s[6], s[7]);
}

// Any width: one thread per pixel.
template <bool NEAR>
__global__ void __launch_bounds__(FUSE_TX* FUSE_TY) fuse_kernel_any(const float* __restrict__ depths, FuseArgs a,
                                                                     FuseCam c) {
    const int u = blockIdx.x * FUSE_TX + threadIdx.x;
    const int v = blockIdx.y * FUSE_TY + threadIdx.y;
    const int W = c.W, H = c.H;
    if (u < 1 || v < 1 || u >= W - 1 || v >= H - 1) return;
    const FuseFrame& F = a.f[blockIdx.z];
    const size_t npx = (size_t)W * H;
    const float* Z = depths + (size_t)F.src * npx;
    const size_t p = (size_t)v * W + u;
    const float yn = ((float)v - c.cy) * c.ify;
    const float rb[3] = {fmaf(F.Pr[1], yn, F.Pr[2]), fmaf(F.Pr[4], yn, F.Pr[5]), fmaf(F.Pr[7], yn, F.Pr[8])};
    fuse_pixel<NEAR>(F, c, ((float)u - c.cx) * c.ifx, yn, rb, __ldg(Z + p), __ldg(Z + p - 1), __ldg(Z + p + 1),
                     __ldg(Z + p - W), __ldg(Z + p + W), c.acc + (size_t)F.kf * npx);
}

// Z* = S / W* where W* > 0, else 0; W* out as is.  Two pixels' sums per 16-byte load.
__global__ void fuse_normalise_kernel(const float2* __restrict__ acc, float* __restrict__ Z, float* __restrict__ Wsum,
                                      size_t n) {
    const size_t n2 = n / 2;  // pairs of pixels: 16-byte loads, 8-byte stores
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
        const float4 sw = __ldcs(reinterpret_cast<const float4*>(acc) + i);
        reinterpret_cast<float2*>(Z)[i] =
            make_float2(sw.y > 0.f ? sw.x / sw.y : 0.f, sw.w > 0.f ? sw.z / sw.w : 0.f);
        reinterpret_cast<float2*>(Wsum)[i] = make_float2(sw.y, sw.w);
    }
    for (size_t i = 2 * n2 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 sw = acc[i];
        Z[i] = sw.y > 0.f ? sw.x / sw.y : 0.f;
        Wsum[i] = sw.y;
    }
}

// Stream-ordered scratch for the interleaved sums: a memory pool per device that keeps
// its memory between calls (release threshold at the maximum), so after the first call
// a fusion takes its scratch from memory the pool already holds; concurrent calls on
// other streams get blocks of their own.
cudaMemPool_t g_fuse_pool[64] = {};
std::mutex g_fuse_pool_mu;

cudaError_t fuse_pool(int dev, cudaMemPool_t* out) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_fuse_pool_mu);
    if (!g_fuse_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        cudaError_t e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_fuse_pool[dev] = p;
    }
    *out = g_fuse_pool[dev];
    return cudaSuccess;
}

int fuse_launch(const float* depths, const sc_pose* frame_poses, const int32_t* frame_kf, int32_t n,
                const sc_pose* kf_poses, const sc_intrinsics* K, const sc_fusion_params* fusion, float2* acc,
                size_t acc_bytes, int sms, float* kf_depth, float* kf_weight, int32_t n_kf, cudaStream_t s);

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
    int dev = 0, sms = 148;
    SC_CUDA(cudaGetDevice(&dev));
    SC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaMemPool_t pool = nullptr;
    SC_CUDA(fuse_pool(dev, &pool));
    float2* acc = nullptr;
    const size_t acc_bytes = (size_t)n_kf * npx * sizeof(float2);
    SC_CUDA(cudaMallocFromPoolAsync((void**)&acc, acc_bytes, pool, s));
    const int rc = fuse_launch(depths, frame_poses, frame_kf, n, kf_poses, K, fusion, acc, acc_bytes, sms,
                               kf_depth, kf_weight, n_kf, s);
    cudaFreeAsync(acc, s);
    return rc;
}

int fuse_launch(const float* depths, const sc_pose* frame_poses, const int32_t* frame_kf, int32_t n,
                const sc_pose* kf_poses, const sc_intrinsics* K, const sc_fusion_params* fusion, float2* acc,
                size_t acc_bytes, int sms, float* kf_depth, float* kf_weight, int32_t n_kf, cudaStream_t s) {
    const int W = K->width, H = K->height;
    const size_t npx = (size_t)W * H;
    FuseCam c{K->cx, K->cy, (float)(1.0 / K->fx), (float)(1.0 / K->fy), (float)((double)K->cx + 0.5),
              (float)((double)K->cy + 0.5), W, H, fusion->disc_rel, acc};
    const bool near = fusion->disc_rel < 1.f;
    dim3 block(FUSE_TX, FUSE_TY);
    // each keyframe image's first frame at the keyframe's own pose initialises its sums
    // (widths multiple of 4); the other frames are scattered with atomics
    std::vector<int> init_src(n_kf, -1);
    std::vector<char> is_init(n, 0);
    if (W % 4 == 0) {
        for (int f = 0; f < n; ++f) {
            const int kf = frame_kf ? frame_kf[f] : 0;
            if (init_src[kf] < 0 && !memcmp(&frame_poses[f], &kf_poses[kf], sizeof(sc_pose))) {
                init_src[kf] = f;
                is_init[f] = 1;
            }
        }
        for (int k0 = 0; k0 < n_kf; k0 += FUSE_MAX_INIT) {
            const int nk = std::min(n_kf - k0, FUSE_MAX_INIT);
            FuseInit a;
            for (int k = 0; k < nk; ++k) a.src[k] = init_src[k0 + k];
            dim3 grid((W / 4 + FUSE_TX - 1) / FUSE_TX, (H + FUSE_TY - 1) / FUSE_TY, nk);
            if (near) fuse_init_kernel<true><<<grid, block, 0, s>>>(depths, a, k0, c);
            else fuse_init_kernel<false><<<grid, block, 0, s>>>(depths, a, k0, c);
            sc::count_launches(1);
            SC_CUDA(cudaGetLastError());
        }
    } else {
        SC_CUDA(cudaMemsetAsync(acc, 0, acc_bytes, s));
    }
    std::vector<int> rest;
    rest.reserve(n);
    for (int f = 0; f < n; ++f)
        if (!is_init[f]) rest.push_back(f);
    const int n_rest = (int)rest.size();
    for (int f0 = 0; f0 < n_rest; f0 += FUSE_MAX_FRAMES) {
        const int nf = (n_rest - f0) < FUSE_MAX_FRAMES ? (n_rest - f0) : FUSE_MAX_FRAMES;
        FuseArgs a;
        for (int f = 0; f < nf; ++f) {
            const int src = rest[f0 + f];
            const sc_pose& T = frame_poses[src];
            const int kf = frame_kf ? frame_kf[src] : 0;
            const sc_pose& Tk = kf_poses[kf];
            // keyframe_from_frame with the focal lengths folded into rows 0 and 1,
            // composed in double and rounded once
            const double scale[3] = {(double)K->fx, (double)K->fy, 1.0};
            for (int r = 0; r < 3; ++r) {
                for (int q = 0; q < 3; ++q) {
                    double acc = 0;
                    for (int k = 0; k < 3; ++k) acc += (double)Tk.m[k][r] * (double)T.m[k][q];
                    a.f[f].Pr[3 * r + q] = (float)(scale[r] * acc);
                }
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += (double)Tk.m[k][r] * ((double)T.m[k][3] - (double)Tk.m[k][3]);
                a.f[f].t[r] = (float)(scale[r] * acc);
            }
            a.f[f].kf = kf;
            a.f[f].src = src;
        }
        cudaEvent_t e0 = nullptr;
        {
            std::lock_guard<std::mutex> lock(g_fprof.mu);
            if (g_fprof.on) e0 = fprof_event(s);
        }
        if (W % 4 == 0) {
            dim3 grid((W / 4 + FUSE_TX - 1) / FUSE_TX, (H + FUSE_TY - 1) / FUSE_TY, nf);
            if (near) fuse_kernel<true><<<grid, block, 0, s>>>(depths, a, c);
            else fuse_kernel<false><<<grid, block, 0, s>>>(depths, a, c);
        } else {
            dim3 grid((W + FUSE_TX - 1) / FUSE_TX, (H + FUSE_TY - 1) / FUSE_TY, nf);
            if (near) fuse_kernel_any<true><<<grid, block, 0, s>>>(depths, a, c);
            else fuse_kernel_any<false><<<grid, block, 0, s>>>(depths, a, c);
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
    fuse_normalise_kernel<<<sms * 8, 256, 0, s>>>(acc, kf_depth, kf_weight, n_kf * npx);
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

// ------------------------------------------------------------ sensor colour ----

namespace {

// 4 pixels per thread: three 32-bit words of packed RGB in, one 16-byte RGBA store out
// (little-endian: word 0 = r0 g0 b0 r1, word 1 = g1 b1 r2 g2, word 2 = b2 r3 g3 b3)
__global__ void rgba_from_rgb_kernel(const uint8_t* __restrict__ rgb, size_t n, uint8_t* __restrict__ rgba) {
    const size_t n4 = n / 4;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t* w = reinterpret_cast<const uint32_t*>(rgb) + 3 * i;
        const uint32_t w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2);
        const uint32_t a = 0xff000000u;
        reinterpret_cast<uint4*>(rgba)[i] = make_uint4((w0 & 0x00ffffffu) | a, (w0 >> 24) | ((w1 & 0xffffu) << 8) | a,
                                                       (w1 >> 16) | ((w2 & 0xffu) << 16) | a, (w2 >> 8) | a);
    }
    for (size_t i = n4 * 4 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        rgba[4 * i] = rgb[3 * i];
        rgba[4 * i + 1] = rgb[3 * i + 1];
        rgba[4 * i + 2] = rgb[3 * i + 2];
        rgba[4 * i + 3] = 255u;
    }
}

}  // namespace

extern "C" int sc_rgba_from_rgb(const uint8_t* rgb, int64_t n_pixels, uint8_t* rgba, sc_stream stream) {
    if (n_pixels < 0 || (n_pixels > 0 && (!rgb || !rgba))) return SC_ERR_INVALID_ARG;
    if (((uintptr_t)rgb & 3) || ((uintptr_t)rgba & 15)) return SC_ERR_INVALID_ARG;
    if (n_pixels == 0) return SC_OK;
    const uintptr_t a0 = (uintptr_t)rgb, a1 = a0 + 3 * (uintptr_t)n_pixels;
    const uintptr_t b0 = (uintptr_t)rgba, b1 = b0 + 4 * (uintptr_t)n_pixels;
    if (a0 < b1 && b0 < a1) return SC_ERR_INVALID_ARG;  // overlapping buffers
    int dev = 0, sms = 0;
    SC_CUDA(cudaGetDevice(&dev));
    SC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    rgba_from_rgb_kernel<<<sms * 8, 256, 0, (cudaStream_t)stream>>>(rgb, (size_t)n_pixels, rgba);
    sc::count_launches(1);
    SC_CUDA(cudaGetLastError());
    return SC_OK;
}
