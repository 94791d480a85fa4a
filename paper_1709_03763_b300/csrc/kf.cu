// Keyframe strategies (Section 4.2): the overlap ratio of KF_OVRLP on the GPU and
// the host loop that groups frames into keyframes (KF_CONST, KF_DIST, KF_OVRLP).
//
// overlap_kernel: one thread per 4 pixels of a row (one thread per pixel for widths
// not a multiple of 4) of up to 64 frames per launch (grid z = frame):
// a valid pixel (Z > 0) is warped into the keyframe (keyframe_from_frame composed in
// double on the host) and counts as overlapping when it lands in front of the
// keyframe with its nearest pixel (halves up) inside the image.  Per-CTA counts are
// reduced with warp shuffles and added with two 64-bit atomics per frame.
//
// KF_OVRLP is sequential by definition (the keyframe a frame is compared with depends
// on the earlier decisions), so the grouping loop evaluates up to the next 32 frames
// against the current keyframe in one launch (about 1.5x the last group's length),
// reads the counts back (through a pinned buffer held per device for the life of the
// process, so concurrent calls on one device take turns), starts a keyframe at the
// first frame below the threshold and continues after it.
#include <cmath>
#include <mutex>
#include <vector>

#include "volume.cuh"

namespace {

constexpr int OV_MAX_FRAMES = 64;
constexpr int OV_SPEC = 32;  // frames evaluated per step of the grouping loop
constexpr int OV_TX = 32, OV_TY = 8;

struct OvFrame {
    float R[9];  // keyframe_from_frame rotation R_k^T R_f
    float t[3];  // keyframe_from_frame translation R_k^T (t_f - t_k)
    int frame;   // depth image index
    int pad;
};

struct OvArgs {
    OvFrame f[OV_MAX_FRAMES];
};

struct OvCam {
    float fx, fy, cx, cy, ifx, ify;
    int W, H;
};



// Overlap decision of one pixel (u, v) with depth z: valid (z > 0) and, if valid,
// whether its point lands in front of the keyframe with its nearest pixel inside.
__device__ __forceinline__ void overlap_pixel(const OvFrame& F, const OvCam& c, float uf, float yn, float z,
                                              unsigned& valid, unsigned& inside) {
    if (!(z > 0.f)) return;
    ++valid;
    const float P[3] = {(uf - c.cx) * c.ifx * z, yn * z, z};
    float p[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        p[r] = fmaf(F.R[3 * r], P[0], fmaf(F.R[3 * r + 1], P[1], fmaf(F.R[3 * r + 2], P[2], F.t[r])));
    if (p[2] > 0.f) {
        const float rz = 1.f / p[2];
        const float uu = floorf(fmaf(c.fx * p[0], rz, c.cx) + 0.5f);
        const float vv = floorf(fmaf(c.fy * p[1], rz, c.cy) + 0.5f);
        inside += (uu >= 0.f && uu < (float)c.W && vv >= 0.f && vv < (float)c.H) ? 1u : 0u;
    }
}

__device__ __forceinline__ unsigned warp_add(unsigned v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-CTA counts: warp shuffles, then two 64-bit atomics per CTA.
__device__ __forceinline__ void overlap_reduce(unsigned valid, unsigned inside, unsigned long long* counts) {
    __shared__ unsigned red[2][OV_TX * OV_TY / 32];
    const int tid = threadIdx.y * OV_TX + threadIdx.x, lane = tid & 31, w = tid >> 5;
    valid = warp_add(valid);
    inside = warp_add(inside);
    if (lane == 0) {
        red[0][w] = valid;
        red[1][w] = inside;
    }
    __syncthreads();
    if (tid < 2) {
        unsigned long long s = 0;
#pragma unroll
        for (int k = 0; k < OV_TX * OV_TY / 32; ++k) s += red[tid][k];
        if (s) atomicAdd(counts + 2 * blockIdx.z + tid, s);
    }
}

// Width a multiple of 4: pixels u0 .. u0 + 3 from one 16-byte load.
__global__ void __launch_bounds__(OV_TX* OV_TY) overlap_kernel(const float* __restrict__ depths, const OvArgs a,
                                                               const OvCam c, unsigned long long* counts) {
    const OvFrame& F = a.f[blockIdx.z];
    const int u0 = 4 * (blockIdx.x * OV_TX + threadIdx.x), v = blockIdx.y * OV_TY + threadIdx.y;
    unsigned valid = 0, inside = 0;
    if (u0 < c.W && v < c.H) {
        const float4 z = __ldg(reinterpret_cast<const float4*>(depths + (size_t)F.frame * c.W * c.H +
                                                                (size_t)v * c.W + u0));
        const float uf = (float)u0, yn = ((float)v - c.cy) * c.ify;
        overlap_pixel(F, c, uf, yn, z.x, valid, inside);
        overlap_pixel(F, c, uf + 1.f, yn, z.y, valid, inside);
        overlap_pixel(F, c, uf + 2.f, yn, z.z, valid, inside);
        overlap_pixel(F, c, uf + 3.f, yn, z.w, valid, inside);
    }
    overlap_reduce(valid, inside, counts);
}

// Any width: one pixel per thread.
__global__ void __launch_bounds__(OV_TX* OV_TY) overlap_kernel_any(const float* __restrict__ depths,
                                                                   const OvArgs a, const OvCam c,
                                                                   unsigned long long* counts) {
    const OvFrame& F = a.f[blockIdx.z];
    const int u = blockIdx.x * OV_TX + threadIdx.x, v = blockIdx.y * OV_TY + threadIdx.y;
    unsigned valid = 0, inside = 0;
    if (u < c.W && v < c.H)
        overlap_pixel(F, c, (float)u, ((float)v - c.cy) * c.ify,
                      __ldg(depths + (size_t)F.frame * c.W * c.H + (size_t)v * c.W + u), valid, inside);
    overlap_reduce(valid, inside, counts);
}

// Pinned host copy of one grouping step's counts, per device (allocated on first use,
// held until exit); the mutex serialises KF_OVRLP calls that share it.
struct OvHost {
    std::mutex mu;
    unsigned long long* counts = nullptr;
} g_ov_host[64];

bool pose_ok(const sc_pose& T) {
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 4; ++q)
            if (!std::isfinite(T.m[r][q])) return false;
    return true;
}

// frames[i] against keyframe pose Tk, counts (device, zeroed here) [n][2]
int launch_overlap(const float* depths, const sc_pose* poses, const int* frames, int n, const sc_pose& Tk,
                   const sc_intrinsics* K, unsigned long long* counts, cudaStream_t s) {
    OvCam c{K->fx, K->fy, K->cx, K->cy, (float)(1.0 / K->fx), (float)(1.0 / K->fy), K->width, K->height};
    SC_CUDA(cudaMemsetAsync(counts, 0, (size_t)n * 2 * sizeof(unsigned long long), s));
    for (int i0 = 0; i0 < n; i0 += OV_MAX_FRAMES) {
        const int m = std::min(OV_MAX_FRAMES, n - i0);
        OvArgs a;
        for (int i = 0; i < m; ++i) {
            const sc_pose& T = poses[frames[i0 + i]];
            OvFrame& F = a.f[i];
            for (int r = 0; r < 3; ++r) {
                for (int q = 0; q < 3; ++q) {
                    double acc = 0;
                    for (int k = 0; k < 3; ++k) acc += (double)Tk.m[k][r] * (double)T.m[k][q];
                    F.R[3 * r + q] = (float)acc;
                }
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += (double)Tk.m[k][r] * ((double)T.m[k][3] - (double)Tk.m[k][3]);
                F.t[r] = (float)acc;
            }
            F.frame = frames[i0 + i];
            F.pad = 0;
        }
        if (K->width % 4 == 0 && ((uintptr_t)depths & 15) == 0) {
            const dim3 grid((K->width / 4 + OV_TX - 1) / OV_TX, (K->height + OV_TY - 1) / OV_TY, m);
            overlap_kernel<<<grid, dim3(OV_TX, OV_TY), 0, s>>>(depths, a, c, counts + 2 * i0);
        } else {
            const dim3 grid((K->width + OV_TX - 1) / OV_TX, (K->height + OV_TY - 1) / OV_TY, m);
            overlap_kernel_any<<<grid, dim3(OV_TX, OV_TY), 0, s>>>(depths, a, c, counts + 2 * i0);
        }
        sc::count_launches(1);
        SC_CUDA(cudaGetLastError());
    }
    return SC_OK;
}

}  // namespace

extern "C" int sc_overlap_counts(const float* depths, const sc_pose* frame_poses, int32_t n, const sc_pose* kf_pose,
                                 const sc_intrinsics* K, uint64_t* counts, sc_stream stream) {
    if (!depths || !frame_poses || n < 0 || !kf_pose || !sc::intrinsics_ok(K) || (n > 0 && !counts))
        return SC_ERR_INVALID_ARG;
    if (((uintptr_t)depths & 3) || ((uintptr_t)counts & 7) || !pose_ok(*kf_pose)) return SC_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!pose_ok(frame_poses[i])) return SC_ERR_INVALID_ARG;
    std::vector<int> frames(n);
    for (int i = 0; i < n; ++i) frames[i] = i;
    if (n == 0) return SC_OK;
    return launch_overlap(depths, frame_poses, frames.data(), n, *kf_pose, K, (unsigned long long*)counts,
                          (cudaStream_t)stream);
}

extern "C" int sc_segment_keyframes(int32_t strategy, const double* params, const float* depths,
                                    const sc_pose* poses, int32_t n, const sc_intrinsics* K, int32_t* frame_kf,
                                    int32_t* n_keyframes, sc_stream stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!params || !poses || n < 0 || (n > 0 && !frame_kf) || !n_keyframes) return SC_ERR_INVALID_ARG;
    if (strategy < SC_KF_CONST || strategy > SC_KF_OVRLP) return SC_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!pose_ok(poses[i])) return SC_ERR_INVALID_ARG;
    if (strategy == SC_KF_CONST && !(params[0] >= 1.0)) return SC_ERR_INVALID_ARG;
    if (strategy == SC_KF_DIST && !(params[0] >= 0.0 && params[1] >= 0.0)) return SC_ERR_INVALID_ARG;
    if (strategy == SC_KF_OVRLP &&
        (!depths || !sc::intrinsics_ok(K) || !(params[0] >= 0.0 && params[0] <= 1.0) || ((uintptr_t)depths & 3)))
        return SC_ERR_INVALID_ARG;
    *n_keyframes = 0;
    if (n == 0) return SC_OK;
    frame_kf[0] = 0;
    int groups = 1, kf = 0;
    if (strategy == SC_KF_CONST) {
        const int kappa = (int)params[0];
        for (int f = 1; f < n; ++f) {
            if (f % kappa == 0) ++groups;
            frame_kf[f] = groups - 1;
        }
    } else if (strategy == SC_KF_DIST) {
        const float thr_t = (float)params[0], thr_r = (float)params[1];
        for (int f = 1; f < n; ++f) {
            const sc_pose& A = poses[kf];
            const sc_pose& B = poses[f];
            double dt = 0.0, tr = 0.0;
            for (int r = 0; r < 3; ++r) {
                const double d = (double)B.m[r][3] - (double)A.m[r][3];
                dt += d * d;
                for (int q = 0; q < 3; ++q) tr += (double)A.m[r][q] * (double)B.m[r][q];
            }
            dt = std::sqrt(dt);
            const double dr = std::acos(std::fmax(-1.0, std::fmin(1.0, (tr - 1.0) / 2.0)));
            if (dt > (double)thr_t || dr > (double)thr_r) {
                kf = f;
                ++groups;
            }
            frame_kf[f] = groups - 1;
        }
    } else {
        const float thr = (float)params[0];
        int dev = 0;
        SC_CUDA(cudaGetDevice(&dev));
        OvHost& oh = g_ov_host[dev & 63];
        std::lock_guard<std::mutex> lock(oh.mu);
        if (!oh.counts) SC_CUDA(cudaMallocHost((void**)&oh.counts, OV_SPEC * 2 * sizeof(unsigned long long)));
        unsigned long long* hcounts = oh.counts;
        unsigned long long* dcounts = nullptr;
        SC_CUDA(cudaMallocAsync((void**)&dcounts, OV_SPEC * 2 * sizeof(unsigned long long), s));
        int f = 1, rc = SC_OK;
        int frames[OV_SPEC];
        // frames evaluated in the next step: half again the last group's length (groups
        // of a trajectory have similar lengths), at least 8, at most OV_SPEC; the
        // decisions do not depend on it, only how much work is speculative
        int spec = OV_SPEC;
        while (f < n && rc == SC_OK) {
            const int m = std::min(spec, n - f);
            for (int i = 0; i < m; ++i) frames[i] = f + i;
            rc = launch_overlap(depths, poses, frames, m, poses[kf], K, dcounts, s);
            if (rc != SC_OK) break;
            if (cudaMemcpyAsync(hcounts, dcounts, (size_t)m * 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                rc = SC_ERR_CUDA;
                break;
            }
            int i = 0;
            for (; i < m; ++i) {
                const unsigned long long nv = hcounts[2 * i], ni = hcounts[2 * i + 1];
                const double ratio = nv ? (double)ni / (double)nv : 0.0;
                if (ratio < (double)thr) break;
                frame_kf[f + i] = groups - 1;
            }
            if (i < m) {  // frame f + i starts a keyframe; evaluate the frames after it
                const int len = f + i - kf;
                spec = std::max(8, std::min(OV_SPEC, len + len / 2));
                kf = f + i;
                ++groups;
                frame_kf[kf] = groups - 1;
                f = kf + 1;
            } else {
                f += m;
                spec = OV_SPEC;
            }
        }
        cudaFreeAsync(dcounts, s);
        if (rc != SC_OK) return rc;
    }
    *n_keyframes = groups;
    return SC_OK;
}
