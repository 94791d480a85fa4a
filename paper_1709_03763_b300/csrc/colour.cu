// Colour keyframe fusion (Section 3 "Keyframe Fusion", colour paragraph).
//
// Two kernels per chunk of whole keyframe groups (32 frames, or one larger group of
// at most 64):
//  * colour_prep_kernel, one CTA per 32x16 tile of a frame: unsharp masking
//    S = I + (I - G*I) with the 5x5 binomial G, computed in integers (S is a
//    multiple of 1/256 and stored exactly as three u16 in an 8-byte texel), and
//    the frame's four blurriness sums (Crete-Roffet measure on the luma
//    Y = 77 R + 150 G + 29 B, in units of 1/256): per direction sum |dY| and
//    sum max(0, 9 |dY| - |dS9|), where S9 is the 9-tap box sum, whose difference
//    between neighbours telescopes to Y(p + 4e) - Y(p - 5e).  Integer sums make
//    the weight w_b = 1 - max_e (9 sF_e - sV_e) / (9 sF_e) exact up to one division.
//  * colour_fuse_kernel, one thread per keyframe pixel x*: the Eq. 1 normal of Z*
//    at x*, then for each frame of the keyframe's group the back-warp
//    p_i = g(T_i^-1, g(T*, pi^-1(x*, Z*(x*)))), the footprint and occlusion tests,
//    the bilinear sample of S and the weight w_c = w_b cos(theta) / z_i^2; the
//    colour is the lower weighted median per channel (the smallest sample c_j with
//    sum_{c_l <= c_j} w_l >= half the total weight, by counting over the samples),
//    rounded to 8 bits.  The kernel is instantiated for the group size (N samples in
//    registers, unrolled), so its median costs about 2 N^2 instructions per channel.
#include <algorithm>
#include <cmath>
#include <vector>

#include "volume.cuh"

namespace {

constexpr int COL_MAX_FRAMES = 64;   // frames per keyframe, and workspace frames
constexpr int COL_CHUNK_FRAMES = 32; // frames per chunk unless one group is larger: 32 frames
                                     // of texels (79 MB at 640x480) stay in the 126 MB L2
                                     // between the prep and the fuse launch
constexpr int COL_TX = 32, COL_TY = 8;  // CTA shape (both kernels)
constexpr int PREP_TY = 16;             // prep tile height: two rows per thread
constexpr int HALO_LO = 5, HALO_HI = 4;  // blurriness differences reach rows/columns p-5 .. p+4
constexpr int TILE_W = COL_TX + HALO_LO + HALO_HI;
constexpr int TILE_H = PREP_TY + HALO_LO + HALO_HI;
constexpr int S_MAX = 255 * 256;  // unsharp value range in 1/256 units

struct ColFrame {
    float R[9];  // frame_from_keyframe rotation R_i^T R*
    float t[3];  // frame_from_keyframe translation R_i^T (t* - t_i)
    int frame;   // index into the caller's frame arrays
    int pad;
};

struct ColChunk {
    ColFrame f[COL_MAX_FRAMES];       // chunk frames, grouped by keyframe; texel slot = index here
    int kf_off[COL_MAX_FRAMES + 1];   // chunk keyframe k owns f[kf_off[k] .. kf_off[k+1])
    int kf_base;                      // first keyframe of the chunk
    int n_frames;
};

struct ColCam {
    float fx, fy, cx, cy, ifx, ify;
    int W, H;
    float disc_rel, occl_rel;
    const uint32_t* rgba;  // caller frames [n_frames][H][W] RGBA8
    const float* depths;   // caller frames [n_frames][H][W]
    uint2* S;              // workspace [COL_MAX_FRAMES][H][W] unsharp texels
    unsigned long long* sums;  // workspace [COL_MAX_FRAMES][4] blurriness sums
    const float* kf_depth;     // [n_kf][H][W] Z*
    uint32_t* kf_rgba;         // [n_kf][H][W] output RGBA8
    float* kf_colour;          // [n_kf][H][W][3] output medians or null
    float* frame_weight;       // [n_frames] output w_b or null
};

__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
    const float w = c * d;
    const float e = fmaf(-c, d, w);
    const float f = fmaf(a, b, -w);
    return f + e;
}

__device__ __forceinline__ unsigned warp_sum(unsigned v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(COL_TX* COL_TY) colour_prep_kernel(const ColChunk ch, const ColCam c) {
    __shared__ uint32_t tile[TILE_H][TILE_W];       // RGBA8, coordinates clamped to the image
    __shared__ int Yt[TILE_H][TILE_W];              // luma x 256
    __shared__ uint32_t hrb[PREP_TY + 4][COL_TX];   // horizontal binomial sums, R | B << 16
    __shared__ uint32_t hga[PREP_TY + 4][COL_TX];   // G | A << 16
    __shared__ unsigned red[4][COL_TX * COL_TY / 32];
    const int slot = blockIdx.z;
    const int W = c.W, H = c.H;
    const size_t npx = (size_t)W * H;
    const uint32_t* img = c.rgba + (size_t)ch.f[slot].frame * npx;
    const int x0 = blockIdx.x * COL_TX, y0 = blockIdx.y * PREP_TY;
    const int tid = threadIdx.y * COL_TX + threadIdx.x;

    for (int r = threadIdx.y; r < TILE_H; r += COL_TY) {
        const uint32_t* src = img + (size_t)min(max(y0 - HALO_LO + r, 0), H - 1) * W;
        for (int q = threadIdx.x; q < TILE_W; q += COL_TX) {
            const uint32_t p = __ldg(src + min(max(x0 - HALO_LO + q, 0), W - 1));
            tile[r][q] = p;
            Yt[r][q] = 77 * (int)(p & 255u) + 150 * (int)((p >> 8) & 255u) + 29 * (int)((p >> 16) & 255u);
        }
    }
    __syncthreads();
    // horizontal (1 4 6 4 1) on rows y0-2 .. y0+PREP_TY+1, two channels per 32-bit word:
    // each 16-bit lane stays below 16 * 255, so no carry crosses lanes
    for (int i = tid; i < (PREP_TY + 4) * COL_TX; i += COL_TX * COL_TY) {
        const int r = i / COL_TX, q = i - r * COL_TX;
        const uint32_t* row = &tile[HALO_LO - 2 + r][HALO_LO - 2 + q];
        const uint32_t p0 = row[0], p1 = row[1], p2 = row[2], p3 = row[3], p4 = row[4];
        const uint32_t m = 0x00ff00ffu;
        hrb[r][q] = (p0 & m) + 4u * (p1 & m) + 6u * (p2 & m) + 4u * (p3 & m) + (p4 & m);
        hga[r][q] = ((p0 >> 8) & m) + 4u * ((p1 >> 8) & m) + 6u * ((p2 >> 8) & m) + 4u * ((p3 >> 8) & m) +
                    ((p4 >> 8) & m);
    }
    __syncthreads();

    const int tx = threadIdx.x;
    unsigned sFv = 0, sVv = 0, sFh = 0, sVh = 0;
#pragma unroll
    for (int half = 0; half < PREP_TY / COL_TY; ++half) {
        const int ty = threadIdx.y + COL_TY * half;
        const int x = x0 + tx, y = y0 + ty;
        if (x >= W || y >= H) continue;
        // vertical (1 4 6 4 1): each 16-bit lane stays below 256 * 255
        const uint32_t Brb = hrb[ty][tx] + 4u * hrb[ty + 1][tx] + 6u * hrb[ty + 2][tx] + 4u * hrb[ty + 3][tx] +
                             hrb[ty + 4][tx];
        const uint32_t Bga = hga[ty][tx] + 4u * hga[ty + 1][tx] + 6u * hga[ty + 2][tx] + 4u * hga[ty + 3][tx] +
                             hga[ty + 4][tx];
        const uint32_t p = tile[HALO_LO + ty][HALO_LO + tx];
        // 256 * (2 I - B / 256), clamped to [0, 255 * 256]
        const int sR = min(max(512 * (int)(p & 255u) - (int)(Brb & 0xffffu), 0), S_MAX);
        const int sG = min(max(512 * (int)((p >> 8) & 255u) - (int)(Bga & 0xffffu), 0), S_MAX);
        const int sB = min(max(512 * (int)((p >> 16) & 255u) - (int)(Brb >> 16), 0), S_MAX);
        c.S[(size_t)slot * npx + (size_t)y * W + x] = make_uint2((unsigned)sR | ((unsigned)sG << 16), (unsigned)sB);
        const int Y0 = Yt[HALO_LO + ty][HALO_LO + tx];
        if (y >= 1) {
            const int dF = abs(Y0 - Yt[HALO_LO + ty - 1][HALO_LO + tx]);
            const int dB9 = abs(Yt[HALO_LO + ty + 4][HALO_LO + tx] - Yt[HALO_LO + ty - 5][HALO_LO + tx]);
            sFv += (unsigned)dF;
            sVv += (unsigned)max(0, 9 * dF - dB9);
        }
        if (x >= 1) {
            const int dF = abs(Y0 - Yt[HALO_LO + ty][HALO_LO + tx - 1]);
            const int dB9 = abs(Yt[HALO_LO + ty][HALO_LO + tx + 4] - Yt[HALO_LO + ty][HALO_LO + tx - 5]);
            sFh += (unsigned)dF;
            sVh += (unsigned)max(0, 9 * dF - dB9);
        }
    }
    // per-CTA sums fit in 32 bits (512 x 9 x 65280 < 2^32); one 64-bit atomic per sum
    sFv = warp_sum(sFv);
    sVv = warp_sum(sVv);
    sFh = warp_sum(sFh);
    sVh = warp_sum(sVh);
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) {
        red[0][warp] = sFv;
        red[1][warp] = sVv;
        red[2][warp] = sFh;
        red[3][warp] = sVh;
    }
    __syncthreads();
    if (tid < 4) {
        unsigned long long t = 0;
#pragma unroll
        for (int w = 0; w < COL_TX * COL_TY / 32; ++w) t += red[tid][w];
        if (t) atomicAdd(c.sums + 4 * slot + tid, t);
    }
}

// w_b = 1 - max over the two directions of (9 sF - sV) / (9 sF); 0 blur where sF = 0
__device__ __forceinline__ float blur_weight(const unsigned long long* s4) {
    double b = 0.0;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const unsigned long long sF = s4[2 * d], sV = s4[2 * d + 1];
        if (sF) {
            const double bd = (double)(9ull * sF - sV) / (double)(9ull * sF);
            b = bd > b ? bd : b;
        }
    }
    return (float)(1.0 - b);
}

// Lower weighted median of N samples, unused ones with value +inf and weight 0: the
// smallest sample v_j whose cumulative weight sum_{v_l <= v_j} w_l reaches half the
// total (an unused sample never qualifies with a finite value).
template <int N>
__device__ __forceinline__ float weighted_median(const float (&v)[N], const float (&w)[N], float half) {
    float best = INFINITY;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        float cw = 0.f;
#pragma unroll
        for (int l = 0; l < N; ++l) cw += (v[l] <= v[j]) ? w[l] : 0.f;
        best = (cw >= half && v[j] < best) ? v[j] : best;
    }
    return best;
}

// registers capped for 4 resident CTAs per SM up to 12 samples, 2 up to 16
template <int NMAX>
__global__ void __launch_bounds__(COL_TX* COL_TY, NMAX <= 12 ? 4 : (NMAX <= 16 ? 2 : 1))
    colour_fuse_kernel(const ColChunk ch, const ColCam c) {
    __shared__ float wb_s[COL_MAX_FRAMES];
    const int k = blockIdx.z;
    const int f0 = ch.kf_off[k], n = ch.kf_off[k + 1] - f0;
    const int tid = threadIdx.y * COL_TX + threadIdx.x;
    if (tid < n) {
        const float wb = blur_weight(c.sums + 4 * (f0 + tid));
        wb_s[tid] = wb;
        if (c.frame_weight && blockIdx.x == 0 && blockIdx.y == 0) c.frame_weight[ch.f[f0 + tid].frame] = wb;
    }
    __syncthreads();
    const int W = c.W, H = c.H;
    const int u = blockIdx.x * COL_TX + threadIdx.x, v = blockIdx.y * COL_TY + threadIdx.y;
    if (u >= W || v >= H) return;
    const size_t npx = (size_t)W * H;
    const size_t kq = (size_t)(ch.kf_base + k) * npx + (size_t)v * W + u;
    const float* Zk = c.kf_depth + (size_t)(ch.kf_base + k) * npx;

    float val[3][NMAX], wt[NMAX];
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
        wt[j] = 0.f;
        val[0][j] = val[1][j] = val[2][j] = INFINITY;
    }

    bool ok = u > 0 && v > 0 && u < W - 1 && v < H - 1;
    float z = 0.f, zl = 0.f, zr = 0.f, zu = 0.f, zd = 0.f;
    if (ok) {
        z = __ldg(Zk + (size_t)v * W + u);
        zl = __ldg(Zk + (size_t)v * W + u - 1);
        zr = __ldg(Zk + (size_t)v * W + u + 1);
        zu = __ldg(Zk + (size_t)(v - 1) * W + u);
        zd = __ldg(Zk + (size_t)(v + 1) * W + u);
        ok = z > 0.f && zl > 0.f && zr > 0.f && zu > 0.f && zd > 0.f;
        const float lim = c.disc_rel * z;
        ok = ok && !(fabsf(zl - z) > lim || fabsf(zr - z) > lim || fabsf(zu - z) > lim || fabsf(zd - z) > lim);
    }
    float P[3], nk[3], inv_nn = 0.f;
    if (ok) {
        const float xn = (u - c.cx) * c.ifx, yn = (v - c.cy) * c.ify;
        P[0] = xn * z;
        P[1] = yn * z;
        P[2] = z;
        // Eq. 1's central-difference normal in keyframe camera coordinates
        const float a0 = (u + 1 - c.cx) * c.ifx * zr - (u - 1 - c.cx) * c.ifx * zl;
        const float a1 = yn * (zr - zl), a2 = zr - zl;
        const float b0 = xn * (zd - zu);
        const float b1 = (v + 1 - c.cy) * c.ify * zd - (v - 1 - c.cy) * c.ify * zu, b2 = zd - zu;
        nk[0] = diff_of_products(a1, b2, a2, b1);
        nk[1] = diff_of_products(a2, b0, a0, b2);
        nk[2] = diff_of_products(a0, b1, a1, b0);
        const float nn2 = nk[0] * nk[0] + nk[1] * nk[1] + nk[2] * nk[2];
        ok = nn2 > 0.f;
        inv_nn = rsqrtf(nn2);
    }
    if (ok) {
        // branch-free per frame, so that the gathers of all frames can be in flight
        // together: an invalid sample reads an in-range texel and gets weight 0
        const float* dep = c.depths;
        const uint2* S = c.S + (size_t)f0 * npx;
        const float Wm = (float)(W - 1), Hm = (float)(H - 1);
#pragma unroll
        for (int j = 0; j < NMAX; ++j) {
            if (j >= n) break;
            const float wb = wb_s[j];
            const ColFrame& F = ch.f[f0 + j];
            float p[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) p[r] = fmaf(F.R[3 * r], P[0], fmaf(F.R[3 * r + 1], P[1], fmaf(F.R[3 * r + 2], P[2], F.t[r])));
            // approximate reciprocal (2 ulp): ~1e-4 px at the image border, inside the
            // pixel margin the oracle flags
            const float rz = __fdividef(1.f, p[2]);
            float us = fmaf(c.fx * p[0], rz, c.cx), vs = fmaf(c.fy * p[1], rz, c.cy);
            bool v = p[2] > 0.f && wb > 0.f && us >= 0.f && us <= Wm && vs >= 0.f && vs <= Hm;
            us = v ? us : 0.f;
            vs = v ? vs : 0.f;
            // occlusion test at the nearest pixel (halves up)
            const int xr = (int)floorf(us + 0.5f), yr = (int)floorf(vs + 0.5f);
            const float zi = __ldg(dep + (size_t)F.frame * npx + (size_t)yr * W + xr);
            // bilinear footprint of the unsharp image
            const int xa = min((int)floorf(us), W - 2), ya = min((int)floorf(vs), H - 2);
            const float ax = us - (float)xa, ay = vs - (float)ya;
            const uint2* Sj = S + (size_t)j * npx + (size_t)ya * W + xa;
            const uint2 t00 = __ldg(Sj), t01 = __ldg(Sj + 1), t10 = __ldg(Sj + W), t11 = __ldg(Sj + W + 1);
            // w_c = w_b cos(theta) / z_i^2, theta between the normal (frame coordinates) and the optical axis
            const float nz = fmaf(F.R[6], nk[0], fmaf(F.R[7], nk[1], F.R[8] * nk[2]));
            const float w = wb * fabsf(nz) * inv_nn * rz * rz;
            v = v && zi > 0.f && !(fabsf(zi - p[2]) > c.occl_rel * p[2]) && w > 0.f;
            // u16 -> float without a conversion instruction: 2^23 + q has q in its mantissa
            const float b23 = 8388608.f;
            const float q00[3] = {__uint_as_float(0x4b000000u | (t00.x & 0xffffu)) - b23,
                                  __uint_as_float(0x4b000000u | (t00.x >> 16)) - b23,
                                  __uint_as_float(0x4b000000u | t00.y) - b23};
            const float q01[3] = {__uint_as_float(0x4b000000u | (t01.x & 0xffffu)) - b23,
                                  __uint_as_float(0x4b000000u | (t01.x >> 16)) - b23,
                                  __uint_as_float(0x4b000000u | t01.y) - b23};
            const float q10[3] = {__uint_as_float(0x4b000000u | (t10.x & 0xffffu)) - b23,
                                  __uint_as_float(0x4b000000u | (t10.x >> 16)) - b23,
                                  __uint_as_float(0x4b000000u | t10.y) - b23};
            const float q11[3] = {__uint_as_float(0x4b000000u | (t11.x & 0xffffu)) - b23,
                                  __uint_as_float(0x4b000000u | (t11.x >> 16)) - b23,
                                  __uint_as_float(0x4b000000u | t11.y) - b23};
#pragma unroll
            for (int ch3 = 0; ch3 < 3; ++ch3) {
                const float top = fmaf(ax, q01[ch3] - q00[ch3], q00[ch3]);
                const float bot = fmaf(ax, q11[ch3] - q10[ch3], q10[ch3]);
                val[ch3][j] = v ? fmaf(ay, bot - top, top) : INFINITY;
            }
            wt[j] = v ? w : 0.f;
        }
    }
    float total = 0.f;
#pragma unroll
    for (int j = 0; j < NMAX; ++j) total += wt[j];
    uint32_t out = 0;
    float m[3] = {0.f, 0.f, 0.f};
    if (total > 0.f) {
        const float half = 0.5f * total;
#pragma unroll
        for (int ch3 = 0; ch3 < 3; ++ch3) m[ch3] = weighted_median<NMAX>(val[ch3], wt, half) * (1.f / 256.f);
        out = (uint32_t)floorf(m[0] + 0.5f) | ((uint32_t)floorf(m[1] + 0.5f) << 8) |
              ((uint32_t)floorf(m[2] + 0.5f) << 16) | 0xff000000u;
    }
    c.kf_rgba[kq] = out;
    if (c.kf_colour) {
        c.kf_colour[3 * kq] = m[0];
        c.kf_colour[3 * kq + 1] = m[1];
        c.kf_colour[3 * kq + 2] = m[2];
    }
}

size_t texel_bytes(int W, int H) { return ((size_t)COL_MAX_FRAMES * W * H * sizeof(uint2) + 255) & ~(size_t)255; }

}  // namespace

extern "C" uint64_t sc_colour_workspace_bytes(int32_t width, int32_t height) {
    if (width < 2 || height < 2 || width > 16384 || height > 16384) return 0;
    return texel_bytes(width, height) + COL_MAX_FRAMES * 4 * sizeof(unsigned long long);
}

extern "C" int sc_fuse_colour_keyframes(const uint8_t* rgba, const float* depths, const sc_pose* frame_poses,
                                        const int32_t* frame_kf, int32_t n_frames, const float* kf_depth,
                                        const sc_pose* kf_poses, int32_t n_kf, const sc_intrinsics* K,
                                        const sc_colour_params* prm, void* workspace, uint64_t workspace_bytes,
                                        uint8_t* kf_rgba, float* kf_colour, float* frame_weight, sc_stream stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!rgba || !depths || !frame_poses || !frame_kf || n_frames < 0 || !kf_depth || !kf_poses || n_kf < 1 ||
        !sc::intrinsics_ok(K) || !prm || !workspace || !kf_rgba)
        return SC_ERR_INVALID_ARG;
    const int W = K->width, H = K->height;
    if (W < 2 || H < 2 || !(prm->disc_rel >= 0.f) || !(prm->occl_rel >= 0.f) || !std::isfinite(prm->disc_rel) ||
        !std::isfinite(prm->occl_rel))
        return SC_ERR_INVALID_ARG;
    if (((uintptr_t)rgba & 15) || ((uintptr_t)depths & 15) || ((uintptr_t)kf_depth & 15) ||
        ((uintptr_t)kf_rgba & 15) || ((uintptr_t)workspace & 255) || ((uintptr_t)kf_colour & 3) ||
        ((uintptr_t)frame_weight & 3))
        return SC_ERR_INVALID_ARG;
    if (workspace_bytes < sc_colour_workspace_bytes(W, H)) return SC_ERR_CAPACITY;
    // frames grouped by keyframe (stable), at most COL_MAX_FRAMES each
    std::vector<std::vector<int>> group(n_kf);
    for (int f = 0; f < n_frames; ++f) {
        if (frame_kf[f] < 0 || frame_kf[f] >= n_kf) return SC_ERR_INVALID_ARG;
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 4; ++q)
                if (!std::isfinite(frame_poses[f].m[r][q])) return SC_ERR_INVALID_ARG;
        group[frame_kf[f]].push_back(f);
    }
    for (int k = 0; k < n_kf; ++k) {
        if ((int)group[k].size() > COL_MAX_FRAMES) return SC_ERR_INVALID_ARG;
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 4; ++q)
                if (!std::isfinite(kf_poses[k].m[r][q])) return SC_ERR_INVALID_ARG;
    }
    ColCam c;
    c.fx = K->fx;
    c.fy = K->fy;
    c.cx = K->cx;
    c.cy = K->cy;
    c.ifx = (float)(1.0 / K->fx);
    c.ify = (float)(1.0 / K->fy);
    c.W = W;
    c.H = H;
    c.disc_rel = prm->disc_rel;
    c.occl_rel = prm->occl_rel;
    c.rgba = (const uint32_t*)rgba;
    c.depths = depths;
    c.S = (uint2*)workspace;
    c.sums = (unsigned long long*)((char*)workspace + texel_bytes(W, H));
    c.kf_depth = kf_depth;
    c.kf_rgba = (uint32_t*)kf_rgba;
    c.kf_colour = kf_colour;
    c.frame_weight = frame_weight;
    const dim3 block(COL_TX, COL_TY);
    const int gx = (W + COL_TX - 1) / COL_TX, gy = (H + COL_TY - 1) / COL_TY;
    int k = 0;
    while (k < n_kf) {
        ColChunk ch;
        ch.kf_base = k;
        int nk = 0, nf = 0;
        ch.kf_off[0] = 0;
        while (k < n_kf && nk < COL_MAX_FRAMES &&
               (nk == 0 || nf + (int)group[k].size() <= COL_CHUNK_FRAMES)) {
            const sc_pose& Tk = kf_poses[k];
            for (int f : group[k]) {
                const sc_pose& T = frame_poses[f];
                ColFrame& F = ch.f[nf++];
                // frame_from_keyframe = T_i^-1 T*, composed in double and rounded once
                for (int r = 0; r < 3; ++r) {
                    for (int q = 0; q < 3; ++q) {
                        double acc = 0;
                        for (int i = 0; i < 3; ++i) acc += (double)T.m[i][r] * (double)Tk.m[i][q];
                        F.R[3 * r + q] = (float)acc;
                    }
                    double acc = 0;
                    for (int i = 0; i < 3; ++i) acc += (double)T.m[i][r] * ((double)Tk.m[i][3] - (double)T.m[i][3]);
                    F.t[r] = (float)acc;
                }
                F.frame = f;
                F.pad = 0;
            }
            ch.kf_off[++nk] = nf;
            ++k;
        }
        ch.n_frames = nf;
        int chunk_max = 0;
        for (int q = 0; q < nk; ++q) chunk_max = std::max(chunk_max, ch.kf_off[q + 1] - ch.kf_off[q]);
        if (nf > 0) {
            SC_CUDA(cudaMemsetAsync(c.sums, 0, (size_t)nf * 4 * sizeof(unsigned long long), s));
            colour_prep_kernel<<<dim3(gx, (H + PREP_TY - 1) / PREP_TY, nf), block, 0, s>>>(ch, c);
            sc::count_launches(1);
            SC_CUDA(cudaGetLastError());
        }
        const dim3 grid(gx, gy, nk);
        if (chunk_max <= 4)
            colour_fuse_kernel<4><<<grid, block, 0, s>>>(ch, c);
        else if (chunk_max <= 8)
            colour_fuse_kernel<8><<<grid, block, 0, s>>>(ch, c);
        else if (chunk_max <= 10)
            colour_fuse_kernel<10><<<grid, block, 0, s>>>(ch, c);
        else if (chunk_max <= 12)
            colour_fuse_kernel<12><<<grid, block, 0, s>>>(ch, c);
        else if (chunk_max <= 16)
            colour_fuse_kernel<16><<<grid, block, 0, s>>>(ch, c);
        else if (chunk_max <= 24)
            colour_fuse_kernel<24><<<grid, block, 0, s>>>(ch, c);
        else if (chunk_max <= 32)
            colour_fuse_kernel<32><<<grid, block, 0, s>>>(ch, c);
        else
            colour_fuse_kernel<64><<<grid, block, 0, s>>>(ch, c);
        sc::count_launches(1);
        SC_CUDA(cudaGetLastError());
    }
    return SC_OK;
}
