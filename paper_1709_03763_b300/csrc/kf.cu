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
// on the earlier decisions), so each step of the grouping loop evaluates up to the next
// 32 frames against the current keyframe in one launch (about 1.5x the last group's
// length), starts a keyframe at the first frame below the threshold and continues after
// it.  The loop runs on the device: a CUDA graph whose while-node body is the overlap
// launch and a one-warp decide kernel that takes the decisions, writes the groups,
// composes the next step's frame-to-keyframe poses and sets the loop condition, so a
// grouping call costs one graph launch and one read-back instead of one host round
// trip per keyframe.  The graph is built once per device (and image size); everything
// that varies between calls lives in a device state block it reads.
#include <algorithm>
#include <cmath>
#include <cstring>
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

// Per-CTA counts into this frame's pair (valid, inside): warp shuffles, then two 64-bit
// atomics per CTA.
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
        if (s) atomicAdd(counts + tid, s);
    }
}

// This CTA's share of frame F's counts.  VEC4 (width a multiple of 4, 16-byte aligned
// depths): pixels u0 .. u0 + 3 from one 16-byte load per thread; else one pixel per
// thread.  counts: this frame's pair.
template <bool VEC4>
__device__ __forceinline__ void overlap_frame(const OvFrame& F, const OvCam& c, const float* __restrict__ depths,
                                              unsigned long long* counts, int bx, int by) {
    unsigned valid = 0, inside = 0;
    const int v = by * OV_TY + threadIdx.y;
    const float* Z = depths + (size_t)F.frame * c.W * c.H;
    if (VEC4) {
        const int u0 = 4 * (bx * OV_TX + threadIdx.x);
        if (u0 < c.W && v < c.H) {
            const float4 z = __ldg(reinterpret_cast<const float4*>(Z + (size_t)v * c.W + u0));
            const float uf = (float)u0, yn = ((float)v - c.cy) * c.ify;
            overlap_pixel(F, c, uf, yn, z.x, valid, inside);
            overlap_pixel(F, c, uf + 1.f, yn, z.y, valid, inside);
            overlap_pixel(F, c, uf + 2.f, yn, z.z, valid, inside);
            overlap_pixel(F, c, uf + 3.f, yn, z.w, valid, inside);
        }
    } else {
        const int u = bx * OV_TX + threadIdx.x;
        if (u < c.W && v < c.H)
            overlap_pixel(F, c, (float)u, ((float)v - c.cy) * c.ify, __ldg(Z + (size_t)v * c.W + u), valid, inside);
    }
    overlap_reduce(valid, inside, counts);
}

template <bool VEC4>
__global__ void __launch_bounds__(OV_TX* OV_TY) overlap_kernel(const float* __restrict__ depths, const OvArgs a,
                                                               const OvCam c, unsigned long long* counts) {
    overlap_frame<VEC4>(a.f[blockIdx.z], c, depths, counts + 2 * blockIdx.z, blockIdx.x, blockIdx.y);
}

// ------------------------------------------------ the grouping loop on the device ----

// Everything a device-side KF_OVRLP grouping reads and updates (one per device,
// rewritten by each call).  Frames [f, f + step) of the current step are compared with
// keyframe kf; tab holds their keyframe_from_frame poses.
struct OvState {
    int n;                 // frames
    int kf;                // current keyframe (frame index)
    int f;                 // first frame of the step
    int step;              // frames evaluated by the step (8 .. OV_SPEC, at most n - f)
    int spec;              // the step length rule's value before clipping to n - f
    int groups;            // keyframes so far
    double thr;            // ratio threshold
    OvCam cam;
    const float* depths;   // device [n][H][W]
    const sc_pose* poses;  // device [n]
    int32_t* frame_kf;     // device [n]
    unsigned long long counts[OV_SPEC][2];
    OvFrame tab[OV_SPEC];
};

// keyframe_from_frame of pose T against keyframe pose Tk, composed in double with
// explicitly rounded operations (the same values the host composition gives) and
// rounded to float once
__host__ __device__ inline void ov_compose(const sc_pose& Tk, const sc_pose& T, int frame, OvFrame& F) {
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) {
#ifdef __CUDA_ARCH__
                acc = __dadd_rn(acc, __dmul_rn((double)Tk.m[k][r], (double)T.m[k][q]));
#else
                acc += (double)Tk.m[k][r] * (double)T.m[k][q];
#endif
            }
            F.R[3 * r + q] = (float)acc;
        }
        double acc = 0;
        for (int k = 0; k < 3; ++k) {
#ifdef __CUDA_ARCH__
            acc = __dadd_rn(acc, __dmul_rn((double)Tk.m[k][r], __dsub_rn((double)T.m[k][3], (double)Tk.m[k][3])));
#else
            acc += (double)Tk.m[k][r] * ((double)T.m[k][3] - (double)Tk.m[k][3]);
#endif
        }
        F.t[r] = (float)acc;
    }
    F.frame = frame;
    F.pad = 0;
}

// The step's overlap counts: persistent CTAs over (slot in the step, tile of the frame),
// so a short step launches no idle CTAs.
template <bool VEC4>
__global__ void __launch_bounds__(OV_TX* OV_TY) overlap_step_kernel(OvState* st, int tiles_x, int tiles) {
    const int n = st->step * tiles;
    for (int w = blockIdx.x; w < n; w += gridDim.x) {
        const int z = w / tiles, t = w - z * tiles;
        overlap_frame<VEC4>(st->tab[z], st->cam, st->depths, st->counts[z], t % tiles_x, t / tiles_x);
        __syncthreads();  // the reduction's shared partials are reused by the next tile
    }
}

// One warp: the step's decisions (ratio = inside / valid in double, below thr starts a
// keyframe; the first such frame wins), the groups of the frames decided, the next
// step (its length about 1.5x the last group's, 8 .. OV_SPEC), its poses and zeroed
// counts, and the loop condition (frames left).
__global__ void overlap_decide_kernel(OvState* st, cudaGraphConditionalHandle loop) {
    const int lane = threadIdx.x;
    const int n = st->n, f = st->f, m = st->step;
    int kf = st->kf, groups = st->groups;
    bool below = false;
    if (lane < m) {
        const unsigned long long nv = st->counts[lane][0], ni = st->counts[lane][1];
        const double ratio = nv ? (double)ni / (double)nv : 0.0;
        below = ratio < st->thr;
    }
    const unsigned b = __ballot_sync(0xffffffffu, below);
    const int first = b ? __ffs(b) - 1 : m;  // frames f .. f + first - 1 stay in the group
    if (lane < first) st->frame_kf[f + lane] = groups - 1;
    int nf, spec;
    if (first < m) {
        const int len = f + first - kf;
        spec = max(8, min(OV_SPEC, len + len / 2));
        kf = f + first;
        ++groups;
        if (lane == 0) st->frame_kf[kf] = groups - 1;
        nf = kf + 1;
    } else {
        spec = OV_SPEC;
        nf = f + m;
    }
    const int step = max(0, min(spec, n - nf));
    if (lane < OV_SPEC) {
        st->counts[lane][0] = 0ull;
        st->counts[lane][1] = 0ull;
        if (lane < step) ov_compose(st->poses[kf], st->poses[nf + lane], nf + lane, st->tab[lane]);
    }
    if (lane == 0) {
        st->kf = kf;
        st->groups = groups;
        st->f = nf;
        st->step = step;
        st->spec = spec;
        cudaGraphSetConditional(loop, nf < n ? 1u : 0u);
    }
}

// Per-device grouping graph (while node over overlap_step + decide) and its state.
struct OvGraph {
    std::mutex mu;
    OvState* st = nullptr;           // device
    OvState* st_h = nullptr;         // pinned staging of the call's initial state
    int32_t* groups_h = nullptr;     // pinned read-back
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int W = 0, H = 0;
    bool vec4 = false;
} g_ov_graph[64];

cudaError_t ov_graph_build(OvGraph& G, int W, int H, bool vec4) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G.exec = nullptr;
    G.graph = nullptr;
    cudaError_t e;
    cudaGraph_t g = nullptr;
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault)) != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cn;
    if ((e = cudaGraphAddNode(&cn, g, nullptr, nullptr, 0, &cp)) != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    OvState* st = G.st;
    int tiles_x = vec4 ? (W / 4 + OV_TX - 1) / OV_TX : (W + OV_TX - 1) / OV_TX;
    int tiles = tiles_x * ((H + OV_TY - 1) / OV_TY);
    void* a1[] = {&st, &tiles_x, &tiles};
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaKernelNodeParams k1 = {};
    k1.func = vec4 ? (void*)overlap_step_kernel<true> : (void*)overlap_step_kernel<false>;
    k1.gridDim = dim3(std::min(sms * 8, OV_SPEC * tiles));
    k1.blockDim = dim3(OV_TX, OV_TY);
    k1.kernelParams = a1;
    cudaGraphNode_t n1, n2;
    if ((e = cudaGraphAddKernelNode(&n1, body, nullptr, 0, &k1)) != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    void* a2[] = {&st, &h};
    cudaKernelNodeParams k2 = {};
    k2.func = (void*)overlap_decide_kernel;
    k2.gridDim = dim3(1);
    k2.blockDim = dim3(32);
    k2.kernelParams = a2;
    if ((e = cudaGraphAddKernelNode(&n2, body, &n1, 1, &k2)) != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    if ((e = cudaGraphInstantiate(&G.exec, g, 0)) != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
    }
    G.graph = g;
    G.W = W;
    G.H = H;
    G.vec4 = vec4;
    return cudaSuccess;
}

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
        for (int i = 0; i < m; ++i) ov_compose(Tk, poses[frames[i0 + i]], frames[i0 + i], a.f[i]);
        if (K->width % 4 == 0 && ((uintptr_t)depths & 15) == 0) {
            const dim3 grid((K->width / 4 + OV_TX - 1) / OV_TX, (K->height + OV_TY - 1) / OV_TY, m);
            overlap_kernel<true><<<grid, dim3(OV_TX, OV_TY), 0, s>>>(depths, a, c, counts + 2 * i0);
        } else {
            const dim3 grid((K->width + OV_TX - 1) / OV_TX, (K->height + OV_TY - 1) / OV_TY, m);
            overlap_kernel<false><<<grid, dim3(OV_TX, OV_TY), 0, s>>>(depths, a, c, counts + 2 * i0);
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
        if (dev < 0 || dev >= 64) return SC_ERR_INVALID_ARG;
        OvGraph& G = g_ov_graph[dev];
        std::lock_guard<std::mutex> lock(G.mu);
        if (!G.st) {
            SC_CUDA(cudaMalloc((void**)&G.st, sizeof(OvState)));
            SC_CUDA(cudaMallocHost((void**)&G.st_h, sizeof(OvState)));
            SC_CUDA(cudaMallocHost((void**)&G.groups_h, sizeof(int32_t)));
        }
        const bool vec4 = K->width % 4 == 0 && ((uintptr_t)depths & 15) == 0;
        if (!G.exec || G.W != K->width || G.H != K->height || G.vec4 != vec4)
            SC_CUDA(ov_graph_build(G, K->width, K->height, vec4));
        // per-call buffers (stream-ordered): the poses and the groups
        sc_pose* poses_d = nullptr;
        int32_t* fk_d = nullptr;
        SC_CUDA(cudaMallocAsync((void**)&poses_d, (size_t)n * sizeof(sc_pose), s));
        cudaError_t e = cudaMallocAsync((void**)&fk_d, (size_t)n * sizeof(int32_t), s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(poses_d, poses, (size_t)n * sizeof(sc_pose), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && n > 1) {
            // the first step: frames 1 .. 32 against frame 0
            OvState& h = *G.st_h;
            memset(&h, 0, sizeof(OvState));
            h.n = n;
            h.kf = 0;
            h.f = 1;
            h.spec = OV_SPEC;
            h.step = std::min(OV_SPEC, n - 1);
            h.groups = 1;
            h.thr = (double)thr;
            h.cam = OvCam{K->fx, K->fy, K->cx, K->cy, (float)(1.0 / K->fx), (float)(1.0 / K->fy), K->width, K->height};
            h.depths = depths;
            h.poses = poses_d;
            h.frame_kf = fk_d;
            for (int i = 0; i < h.step; ++i) ov_compose(poses[0], poses[1 + i], 1 + i, h.tab[i]);
            e = cudaMemcpyAsync(G.st, G.st_h, sizeof(OvState), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaGraphLaunch(G.exec, s);
            sc::count_launches(1);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(frame_kf + 1, fk_d + 1, (size_t)(n - 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(G.groups_h, &G.st->groups, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        }
        if (poses_d) cudaFreeAsync(poses_d, s);
        if (fk_d) cudaFreeAsync(fk_d, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        SC_CUDA(e);
        groups = n > 1 ? *G.groups_h : 1;
    }
    *n_keyframes = groups;
    return SC_OK;
}
