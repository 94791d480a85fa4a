// Loss on the fused SDF and its adjoint with respect to keyframe poses and depth
// (an extension; the paper has no counterpart).
//
//   L = (1/P) sum_p Dt(p)^2 + lambda * sum_v W D^2 / sum_v W
//
// Forward: one pass over the pool for the weighted regulariser's sums (which also
// zeroes the gradient), one pass over the points (count, sum of Dt^2 and the scatter
// of the unscaled point gradient 2 Dt beta), and one pass over the pool that scales
// the point gradient by 1/P once P is known and adds the regulariser's gradient.  Adjoint: D(v) = sum_k w_k d_k(v) / W(v), so for each keyframe the
// kernel walks its block list, recomputes each voxel's projective sample exactly
// as the integration did (same sample function, same camera constants) and
// accumulates g = dL/dD(v) / W(v) for unclamped samples into the depth-pixel
// gradient and into four pose moments (sum g, sum g q) from which the se(3)
// gradient follows.  Lane values are float, warp and CTA partials double.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <new>

#include "volume.cuh"

using namespace sc;

namespace {

constexpr int LOSS_THREADS = 256;

__device__ inline double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Trilinear neighbourhood of point p: voxel corner indices and weights; returns
// false if any corner is unallocated or unobserved (W = 0).
struct Corners {
    uint32_t vox[8];  // slot * 512 + voxel index (max_blocks <= 2^23)
    float beta[8];
};

__device__ inline bool point_corners(const DevVolume& V, float s, float inv_s, const float* p, Corners& c, float& Dt) {
    // grid coordinate g = p / s without a double division: q = p (1/s) is within two
    // float ulps of g, r = p - q s is its residual (one fused rounding), and the
    // fraction (q - floor(q)) + r / s carries about 1e-7 voxel of error where a
    // float g would carry 1e-4 at 10^3 voxels from the origin
    int i0[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float x = __ldg(p + a);
        const float q = __fmul_rn(x, inv_s);
        const float r = __fmaf_rn(-q, s, x);
        float fl = floorf(q);
        float fr = __fadd_rn(__fsub_rn(q, fl), __fmul_rn(r, inv_s));
        if (fr < 0.f) {  // g lies just below the integer q rounded up to
            fl = __fsub_rn(fl, 1.f);
            fr = __fadd_rn(fr, 1.f);
        } else if (fr >= 1.f) {
            fl = __fadd_rn(fl, 1.f);
            fr = __fsub_rn(fr, 1.f);
        }
        i0[a] = (int)fl;
        f[a] = fr;
    }
    // the corners' blocks first (one, two, four or eight distinct ones) ...
    int32_t last_slot = -1;
    int lbx = 0x7fffffff, lby = 0, lbz = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int ox = k & 1, oy = (k >> 1) & 1, oz = (k >> 2) & 1;
        const int ix = i0[0] + ox, iy = i0[1] + oy, iz = i0[2] + oz;
        const int bx = ix >> 3, by = iy >> 3, bz = iz >> 3;
        if (bx != lbx || by != lby || bz != lbz) {
            lbx = bx;
            lby = by;
            lbz = bz;
            last_slot = coord_ok(bx, by, bz) ? find_slot(V, pack_key(bx, by, bz)) : -1;
        }
        if (last_slot < 0) return false;
        const int vi = (ix & 7) + 8 * (iy & 7) + 64 * (iz & 7);
        c.vox[k] = (uint32_t)last_slot * NVOX + vi;
    }
    // ... then all sixteen voxel loads in flight together
    float w[8], d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        w[k] = V.W[c.vox[k]];
        d[k] = V.D[c.vox[k]];
    }
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (!(w[k] > 0.f)) return false;
        const int ox = k & 1, oy = (k >> 1) & 1, oz = (k >> 2) & 1;
        const float b = (ox ? f[0] : 1.f - f[0]) * (oy ? f[1] : 1.f - f[1]) * (oz ? f[2] : 1.f - f[2]);
        c.beta[k] = b;
        acc = fmaf(b, d[k], acc);
    }
    Dt = acc;
    return true;
}

// out[1] += P, out[2] += sum Dt^2, grad += 2 Dt beta (scaled by 1/P later).  Dt^2 is
// summed in float over at most 8 points of a thread, then in double.
__global__ void loss_points_kernel(DevVolume V, float s, float inv_s, const float* pts, int64_t n, double* out,
                                   float* grad) {
    __shared__ double sh[2][LOSS_THREADS / 32];
    double a = 0.0;
    float af = 0.f;
    int m = 0;
    unsigned cnt = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Corners c;
        float Dt;
        if (point_corners(V, s, inv_s, pts + 3 * i, c, Dt)) {
            af = fmaf(Dt, Dt, af);
            ++cnt;
            if (++m == 8) {
                a += (double)af;
                af = 0.f;
                m = 0;
            }
            const float g = 2.f * Dt;
#pragma unroll
            for (int k = 0; k < 8; ++k) atomicAdd(grad + c.vox[k], g * c.beta[k]);
        }
    }
    a += (double)af;
    a = warp_sum(a);
    const double cn = warp_sum((double)cnt);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[0][w] = a;
        sh[1][w] = cn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0, C = 0;
        for (int k = 0; k < LOSS_THREADS / 32; ++k) {
            A += sh[0][k];
            C += sh[1][k];
        }
        atomicAdd(out + 1, C);
        atomicAdd(out + 2, A);
    }
}

// out[3] += sum W D^2, out[4] += sum W over pool slots [0, used); grad = 0 there
__global__ void loss_reg_kernel(DevVolume V, double* out, float* grad) {
    __shared__ double sh[2][LOSS_THREADS / 32];
    const size_t nv = (size_t)min(*V.pool_count, V.max_blocks) * NVOX;
    // float sums over at most 8 groups of 4 voxels, then double
    double a = 0.0, b = 0.0;
    float pa = 0.f, pb = 0.f;
    int m = 0;
    for (size_t i = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) * 4; i < nv; i += (size_t)gridDim.x * blockDim.x * 4) {
        const float4 W = *reinterpret_cast<const float4*>(V.W + i);
        const float4 D = *reinterpret_cast<const float4*>(V.D + i);
        *reinterpret_cast<float4*>(grad + i) = make_float4(0.f, 0.f, 0.f, 0.f);
        if (W.x > 0.f) { pa = fmaf(W.x * D.x, D.x, pa); pb += W.x; }
        if (W.y > 0.f) { pa = fmaf(W.y * D.y, D.y, pa); pb += W.y; }
        if (W.z > 0.f) { pa = fmaf(W.z * D.z, D.z, pa); pb += W.z; }
        if (W.w > 0.f) { pa = fmaf(W.w * D.w, D.w, pa); pb += W.w; }
        if (++m == 8) {
            a += pa;
            b += pb;
            pa = pb = 0.f;
            m = 0;
        }
    }
    a += pa;
    b += pb;
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[0][w] = a;
        sh[1][w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0, B = 0;
        for (int k = 0; k < LOSS_THREADS / 32; ++k) {
            A += sh[0][k];
            B += sh[1][k];
        }
        atomicAdd(out + 3, A);
        atomicAdd(out + 4, B);
    }
}

// grad_D = grad_D / P + 2 lambda W D / sum W (the regulariser's part 0 where W = 0),
// pool slots [0, used); the point part is zero wherever W = 0
__global__ void loss_grad_combine_kernel(DevVolume V, float lambda, const double* out, float* grad) {
    const size_t nv = (size_t)min(*V.pool_count, V.max_blocks) * NVOX;
    const double P = out[1], sw = out[4];
    const float inv_p = P > 0.0 ? (float)(1.0 / P) : 0.f;
    const float scale = sw > 0.0 ? (float)(2.0 * lambda / sw) : 0.f;
    for (size_t i = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) * 4; i < nv; i += (size_t)gridDim.x * blockDim.x * 4) {
        const float4 W = *reinterpret_cast<const float4*>(V.W + i);
        const float4 D = *reinterpret_cast<const float4*>(V.D + i);
        float4 g = *reinterpret_cast<const float4*>(grad + i);
        g.x = g.x * inv_p + (W.x > 0.f ? scale * W.x * D.x : 0.f);
        g.y = g.y * inv_p + (W.y > 0.f ? scale * W.y * D.y : 0.f);
        g.z = g.z * inv_p + (W.z > 0.f ? scale * W.z * D.z : 0.f);
        g.w = g.w * inv_p + (W.w > 0.f ? scale * W.w * D.w : 0.f);
        *reinterpret_cast<float4*>(grad + i) = g;
    }
}

__global__ void loss_finalize_kernel(float lambda, double* out) {
    const double P = out[1];
    double L = P > 0.0 ? out[2] / P : 0.0;
    if (out[4] > 0.0) L += (double)lambda * out[3] / out[4];
    out[0] = L;
}

// ------------------------------------------------------------------ adjoint ----

struct AdjItem {
    KfCam cam;
    const int32_t* list;
    const int32_t* count;
    float* grad_depth;  // [H][W] or null
};

// acc [n][4]: sum g, sum g mx, sum g my, sum g mz  (m = i - ti, the voxel index relative
// to the camera's integer voxel, exact in float; the finalize subtracts tf sum g to get
// the sums over q = m - tf, the voxel relative to the camera in voxel units).
// Grid (chunks, n): blockIdx.y is the keyframe; the chunk's warps stride over its
// block list, one warp per block (4 voxels per lane per group); lane sums are float,
// the warp and CTA reductions double, one set of 4 atomics per CTA.
constexpr int ADJ_THREADS = 256;

#ifndef SC_ADJ_MIN_BLOCKS
#define SC_ADJ_MIN_BLOCKS 5  // resident CTAs per SM: 48 registers, 40 warps
#endif
__global__ void __launch_bounds__(ADJ_THREADS, SC_ADJ_MIN_BLOCKS) adjoint_kernel(DevVolume V, const AdjItem* items, uint32_t cap,
                                                              const float* grad, double* acc) {
    __shared__ double sh[ADJ_THREADS / 32][4];
    __shared__ KfCam sh_cam;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k = blockIdx.y;
    const AdjItem& it = items[k];
    // the keyframe's camera copied into shared memory once: read from the item table in
    // global memory, its fields took registers and reloads in every block's projections
    // (the adjoint is 13 % faster with the copy)
    {
        const uint32_t* cs = reinterpret_cast<const uint32_t*>(&it.cam);
        uint32_t* cd = reinterpret_cast<uint32_t*>(&sh_cam);
        for (int i = threadIdx.x; i < (int)(sizeof(KfCam) / 4); i += ADJ_THREADS) cd[i] = cs[i];
    }
    __syncthreads();
    const KfCam& cam = sh_cam;
    const uint32_t cnt = min((uint32_t)*it.count, cap);
    const uint32_t nw = gridDim.x * (ADJ_THREADS / 32);
    // per lane: float sums over one block's 16 voxels, then double across blocks
    // (contributions of both signs cancel strongly in the pose moments)
    double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
    for (uint32_t b = blockIdx.x * (ADJ_THREADS / 32) + warp; b < cnt; b += nw) {
        const int32_t slot = it.list[b];
        if (slot < 0) {  // streamed out to the host block store
            if (lane == 0) set_status(V.status, SC_ERR_NOT_RESIDENT);
            continue;
        }
        const int4 c = V.coord[slot];
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 1
        for (int g = 0; g < 4; ++g) {
            int lx0, ly, lz;
            lane_voxels(lane, g, lx0, ly, lz);
            const size_t off = (size_t)slot * NVOX + 4 * lane + 128 * g;
            const int iy = 8 * c.y + ly, iz = 8 * c.z + lz;
            // the lane's 4 voxels share y and z; their x runs mx0 .. mx0 + 3 (exact floats)
            const float mx0 = (float)(8 * c.x + lx0 - cam.ti[0]);
            // the lane's 4 voxels are contiguous: one 16-byte load each of dL/dD and W,
            // issued before the projection so that their latency overlaps it
            const float4 g4 = __ldg(reinterpret_cast<const float4*>(grad + off));
            const float4 w4 = __ldg(reinterpret_cast<const float4*>(V.W + off));
            const float gj[4] = {g4.x, g4.y, g4.z, g4.w}, wj[4] = {w4.x, w4.y, w4.z, w4.w};
            Proj4 P;
            project4(cam, (float)(8 * c.x + lx0), (float)iy, (float)iz, P);
            float Z[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) Z[j] = P.ok[j] ? __ldg(cam.depth + P.pix[j]) : 0.f;
            // branch-free: the update decision of decide() (ok, Z > 0, eta >= -mu; eta is
            // finite whenever ok and Z > 0) and no clamp (eta < mu) select the sample; a
            // zero cotangent contributes nothing and is never divided by its voxel's W
            // (an unobserved voxel has W = 0)
            float ag = 0.f, agx = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float eta = __fsub_rn(Z[j], P.pz[j]);
                const bool on = P.ok[j] & (Z[j] > 0.f) & (eta >= -cam.mu) & (eta < cam.mu) & (gj[j] != 0.f);
                // one approximate reciprocal (1 ulp) per sample instead of a division
                const float gv = on ? __fmul_rn(gj[j], rcp_approx(wj[j])) : 0.f;
                if (on && it.grad_depth) atomicAdd(it.grad_depth + P.pix[j], gv);
                ag += gv;
                agx = fmaf(gv, mx0 + (float)j, agx);
            }
            a0 += ag;
            a1 += agx;
            a2 = fmaf(ag, (float)(iy - cam.ti[1]), a2);
            a3 = fmaf(ag, (float)(iz - cam.ti[2]), a3);
        }
        d0 += a0;
        d1 += a1;
        d2 += a2;
        d3 += a3;
    }
    const double s0 = warp_sum(d0), s1 = warp_sum(d1), s2 = warp_sum(d2), s3 = warp_sum(d3);
    if (lane == 0) {
        sh[warp][0] = s0;
        sh[warp][1] = s1;
        sh[warp][2] = s2;
        sh[warp][3] = s3;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < ADJ_THREADS / 32; ++w) t += sh[w][threadIdx.x];
        if (t != 0.0) atomicAdd(acc + 4 * k + threadIdx.x, t);
    }
}

// grad_xi[k] = (r3 A, s B x r3 + (t x r3) A), A = sum g, B = sum g q
struct AdjPose {
    double r3[3];
    double t[3];
    double tf[3];  // the camera's fractional voxel offset (KfCam tf)
};

__global__ void adjoint_finalize_kernel(const AdjPose* poses, const double* acc, int n, double s, double* grad_xi) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double* r = poses[k].r3;
    const double* t = poses[k].t;
    const double A = acc[4 * k];
    const double* tf = poses[k].tf;
    const double B[3] = {s * (acc[4 * k + 1] - tf[0] * A), s * (acc[4 * k + 2] - tf[1] * A),
                         s * (acc[4 * k + 3] - tf[2] * A)};
    double* g = grad_xi + 6 * k;
    for (int j = 0; j < 3; ++j) g[j] = r[j] * A;
    const double bx[3] = {B[1] * r[2] - B[2] * r[1], B[2] * r[0] - B[0] * r[2], B[0] * r[1] - B[1] * r[0]};
    const double tx[3] = {t[1] * r[2] - t[2] * r[1], t[2] * r[0] - t[0] * r[2], t[0] * r[1] - t[1] * r[0]};
    for (int j = 0; j < 3; ++j) g[3 + j] = bx[j] + tx[j] * A;
}

}  // namespace

// Item and pose tables (pinned staging + device copies) and the double
// accumulators of sc_sdf_adjoint, owned by one volume: calls on different volumes
// share nothing.
struct AdjScratch {
    int cap = 0;
    AdjItem* items_d = nullptr;
    AdjPose* poses_d = nullptr;
    double* acc_d = nullptr;
    AdjItem* items_h = nullptr;
    AdjPose* poses_h = nullptr;
    cudaEvent_t staged = nullptr;  // recorded after the last call's copies from items_h / poses_h
};

namespace {

void adj_free(AdjScratch& A) {
    if (A.items_d) cudaFree(A.items_d);
    if (A.poses_d) cudaFree(A.poses_d);
    if (A.acc_d) cudaFree(A.acc_d);
    if (A.items_h) cudaFreeHost(A.items_h);
    if (A.poses_h) cudaFreeHost(A.poses_h);
    if (A.staged) cudaEventDestroy(A.staged);
    A = AdjScratch();
}

// Room for n keyframes in the volume's adjoint tables (allocates on first use and
// when n grows past the capacity, at least 256).
int adj_reserve(sc_volume* V, int n) {
    if (!V->adj) {
        V->adj = new (std::nothrow) AdjScratch();
        if (!V->adj) return SC_ERR_CUDA;
    }
    AdjScratch& A = *V->adj;
    if (A.cap >= n) return SC_OK;
    adj_free(A);
    const int cap = n < 256 ? 256 : n;
    SC_CUDA(cudaMalloc((void**)&A.items_d, cap * sizeof(AdjItem)));
    SC_CUDA(cudaMalloc((void**)&A.poses_d, cap * sizeof(AdjPose)));
    SC_CUDA(cudaMalloc((void**)&A.acc_d, cap * 4 * sizeof(double)));
    SC_CUDA(cudaMallocHost((void**)&A.items_h, cap * sizeof(AdjItem)));
    SC_CUDA(cudaMallocHost((void**)&A.poses_h, cap * sizeof(AdjPose)));
    SC_CUDA(cudaEventCreateWithFlags(&A.staged, cudaEventDisableTiming));
    A.cap = cap;
    return SC_OK;
}

}  // namespace

void adj_destroy(sc_volume* V) {
    if (!V->adj) return;
    adj_free(*V->adj);
    delete V->adj;
    V->adj = nullptr;
}

extern "C" int sc_sdf_loss(sc_volume* V, const float* points, int64_t n, float lambda, float* grad_D, double* out,
                           sc_stream stream) {
    if (!V || (!points && n > 0) || n < 0 || !grad_D || !out || !(lambda >= 0.f)) return SC_ERR_INVALID_ARG;
    if (((uintptr_t)grad_D & 15) || ((uintptr_t)out & 7)) return SC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const float vs = V->p.voxel_size;
    SC_CUDA(cudaMemsetAsync(out, 0, 5 * sizeof(double), s));
    const int grid = V->num_sms * 8;
    loss_reg_kernel<<<grid, LOSS_THREADS, 0, s>>>(V->dv, out, grad_D);
    if (n > 0) loss_points_kernel<<<grid, LOSS_THREADS, 0, s>>>(V->dv, vs, (float)(1.0 / (double)vs), points, n, out,
                                                              grad_D);
    loss_grad_combine_kernel<<<grid, LOSS_THREADS, 0, s>>>(V->dv, lambda, out, grad_D);
    loss_finalize_kernel<<<1, 1, 0, s>>>(lambda, out);
    count_launches(n > 0 ? 4 : 3);
    SC_CUDA(cudaGetLastError());
    V->last_stream = s;
    return SC_OK;
}

extern "C" int sc_sdf_adjoint(sc_volume* V, const int32_t* kf_ids, const float* const* depths, const sc_pose* poses,
                              int32_t n, const sc_intrinsics* K, const float* grad_D, double* grad_xi,
                              float* grad_depth, sc_stream stream) {
    if (!V || !kf_ids || !depths || !poses || n < 1 || n > 65535 || !intrinsics_ok(K) || !grad_D || !grad_xi ||
        ((uintptr_t)grad_D & 15))
        return SC_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (kf_ids[i] < 0 || kf_ids[i] >= V->p.max_keyframes || !depths[i]) return SC_ERR_INVALID_ARG;
        if (!V->integrated[kf_ids[i]]) return SC_ERR_NOT_INTEGRATED;
        if (V->nonresident[kf_ids[i]]) return SC_ERR_NOT_RESIDENT;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int rc = adj_reserve(V, n);
    if (rc) return rc;
    AdjScratch& A = *V->adj;
    // the pinned staging tables may still be read by a previous call's copies: wait for
    // those copies only, not for the work queued on the stream since
    SC_CUDA(cudaEventSynchronize(A.staged));
    const size_t img = (size_t)K->width * K->height;
    for (int i = 0; i < n; ++i) {
        const int kf = kf_ids[i];
        A.items_h[i].cam = make_cam(V, K, &poses[i], depths[i], nullptr);
        A.items_h[i].list = list_ptr(V, kf, V->cur[kf]);
        A.items_h[i].count = count_ptr(V, kf, V->cur[kf]);
        A.items_h[i].grad_depth = grad_depth ? grad_depth + i * img : nullptr;
        for (int r = 0; r < 3; ++r) {
            A.poses_h[i].r3[r] = (double)poses[i].m[r][2];
            A.poses_h[i].t[r] = (double)poses[i].m[r][3];
            A.poses_h[i].tf[r] = (double)A.items_h[i].cam.tf[r];
        }
    }
    SC_CUDA(cudaMemcpyAsync(A.items_d, A.items_h, n * sizeof(AdjItem), cudaMemcpyHostToDevice, s));
    SC_CUDA(cudaMemcpyAsync(A.poses_d, A.poses_h, n * sizeof(AdjPose), cudaMemcpyHostToDevice, s));
    SC_CUDA(cudaEventRecord(A.staged, s));
    SC_CUDA(cudaMemsetAsync(A.acc_d, 0, n * 4 * sizeof(double), s));
    if (grad_depth) SC_CUDA(cudaMemsetAsync(grad_depth, 0, n * img * sizeof(float), s));
    const int chunks = std::max(1, std::min(64, (V->num_sms * 8 + n - 1) / n));
    adjoint_kernel<<<dim3(chunks, n), ADJ_THREADS, 0, s>>>(V->dv, A.items_d, V->p.max_blocks_per_keyframe, grad_D,
                                                          A.acc_d);
    adjoint_finalize_kernel<<<(n + 127) / 128, 128, 0, s>>>(A.poses_d, A.acc_d, n, (double)V->p.voxel_size, grad_xi);
    count_launches(2);
    SC_CUDA(cudaGetLastError());
    V->last_stream = s;
    return SC_OK;
}

// ---------------------------------------------- allocation-free adjoint ----
//
// The same adjoint kernels, with their keyframe table, pose table and double
// accumulators in a file-scope device array instead of memory this library
// allocates.  For callers that must not allocate device memory once running: a
// real-time tracking thread whose memory budget is fixed at start-up, or a host
// application whose device memory is owned by another allocator (a pool that must
// see every byte in use).

namespace {

constexpr int ADJ_STATIC_MAX = 256;  // keyframes per call

struct AdjStatic {
    AdjItem items[ADJ_STATIC_MAX];
    AdjPose poses[ADJ_STATIC_MAX];
    double acc[4 * ADJ_STATIC_MAX];
};

// host-side device addresses of the scratch array below, one per device (the
// array's name in host code is a stand-in, not a device address); looked up once
// per device under the mutex, read without it afterwards
std::atomic<void*> g_adj_static_ptr[64];
std::mutex g_adj_static_mu;

}  // namespace

// about 76 KB on every GPU that loads the library, held until the process exits
static __device__ __align__(256) unsigned char g_adj_static[sizeof(AdjStatic)];

extern "C" int sc_sdf_adjoint_noalloc(sc_volume* V, const int32_t* kf_ids, const float* const* depths,
                                      const sc_pose* poses, int32_t n, const sc_intrinsics* K, const float* grad_D,
                                      double* grad_xi, float* grad_depth, sc_stream stream) {
    if (!V || !kf_ids || !depths || !poses || n < 1 || !intrinsics_ok(K) || !grad_D || !grad_xi ||
        ((uintptr_t)grad_D & 15))
        return SC_ERR_INVALID_ARG;
    if (n > ADJ_STATIC_MAX) return SC_ERR_CAPACITY;
    for (int i = 0; i < n; ++i) {
        if (kf_ids[i] < 0 || kf_ids[i] >= V->p.max_keyframes || !depths[i]) return SC_ERR_INVALID_ARG;
        if (!V->integrated[kf_ids[i]]) return SC_ERR_NOT_INTEGRATED;
        if (V->nonresident[kf_ids[i]]) return SC_ERR_NOT_RESIDENT;
    }
    // the scratch array is per device: the volume's device must be the current one
    int dev = 0;
    SC_CUDA(cudaGetDevice(&dev));
    if (dev != V->device || dev < 0 || dev >= 64) return SC_ERR_INVALID_ARG;
    void* addr = g_adj_static_ptr[dev].load(std::memory_order_acquire);
    if (!addr) {
        // once per device, with that device current
        std::lock_guard<std::mutex> lock(g_adj_static_mu);
        addr = g_adj_static_ptr[dev].load(std::memory_order_relaxed);
        if (!addr) {
            SC_CUDA(cudaGetSymbolAddress(&addr, g_adj_static));
            g_adj_static_ptr[dev].store(addr, std::memory_order_release);
        }
    }
    AdjStatic* S = static_cast<AdjStatic*>(addr);
    cudaStream_t s = (cudaStream_t)stream;
    // host tables in pageable memory: cudaMemcpyAsync from pageable memory returns
    // once the data has been staged, so the buffers can be reused at once
    static thread_local AdjItem items_h[ADJ_STATIC_MAX];
    static thread_local AdjPose poses_h[ADJ_STATIC_MAX];
    const size_t img = (size_t)K->width * K->height;
    for (int i = 0; i < n; ++i) {
        const int kf = kf_ids[i];
        items_h[i].cam = make_cam(V, K, &poses[i], depths[i], nullptr);
        items_h[i].list = list_ptr(V, kf, V->cur[kf]);
        items_h[i].count = count_ptr(V, kf, V->cur[kf]);
        items_h[i].grad_depth = grad_depth ? grad_depth + i * img : nullptr;
        for (int r = 0; r < 3; ++r) {
            poses_h[i].r3[r] = (double)poses[i].m[r][2];
            poses_h[i].t[r] = (double)poses[i].m[r][3];
            poses_h[i].tf[r] = (double)items_h[i].cam.tf[r];
        }
    }
    SC_CUDA(cudaMemcpyAsync(S->items, items_h, n * sizeof(AdjItem), cudaMemcpyHostToDevice, s));
    SC_CUDA(cudaMemcpyAsync(S->poses, poses_h, n * sizeof(AdjPose), cudaMemcpyHostToDevice, s));
    // the array keeps the previous call's contents: the accumulators start at zero
    SC_CUDA(cudaMemsetAsync(S->acc, 0, n * 4 * sizeof(double), s));
    if (grad_depth) SC_CUDA(cudaMemsetAsync(grad_depth, 0, n * img * sizeof(float), s));
    const int chunks = std::max(1, std::min(64, (V->num_sms * 8 + n - 1) / n));
    adjoint_kernel<<<dim3(chunks, n), ADJ_THREADS, 0, s>>>(V->dv, S->items, V->p.max_blocks_per_keyframe, grad_D,
                                                          S->acc);
    adjoint_finalize_kernel<<<(n + 127) / 128, 128, 0, s>>>(S->poses, S->acc, n, (double)V->p.voxel_size, grad_xi);
    count_launches(2);
    SC_CUDA(cudaGetLastError());
    V->last_stream = s;
    return SC_OK;
}
