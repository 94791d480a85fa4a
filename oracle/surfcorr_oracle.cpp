// FP64 CPU oracle for keyframe surface correction (Maier, Schaller, Cremers,
// "Efficient Online Surface Correction for Real-time Large-Scale 3D
// Reconstruction", arXiv 1709.03763).
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
// benchmark's CPU-baseline leg load this library.  It shares no code, header,
// table or constant with the CUDA path, and it never reads a value the CUDA
// path produced.  It is deliberately plain and slow: one voxel, one pixel, one
// decision at a time, in double precision, in the order the paper states the
// steps.  Inputs are the same float32 depth / uint8 colour / float32 poses the
// GPU gets, promoted to double.
//
// Functions and what pins them (the pins live in tests/test_oracle_*.py):
//   or_fuse                  Eq. 1 keyframe depth fusion (Section 3 "Keyframe Fusion").
//                            Pinned: identical frames at one pose give Z* = Z and
//                            W* = sum of cos(theta)/Z^2; a fronto-parallel plane has
//                            cos(theta) = 1; x-translated views of a plane fuse to z0;
//                            Eq. 1 applied in any frame order gives the same ratio.
//   or_vol_*                 Voxel-hashed TSDF (Section 3 "SDF volume"): block
//                            allocation, running-average integration, Eq. 2
//                            de-integration, sequential re-integration batches
//                            (Section 4.3).  Pinned: closed-form truncated distance
//                            for a fronto-parallel plane and for a sphere, weights
//                            equal a brute-force observation count, integrate then
//                            de-integrate restores the volume, allocation equals a
//                            dense point-sampling of each band segment.
//   or_pose_distance,        Keyframe selection (Section 4.3, Eq. 3, Fig. 4).
//   or_select_topm,          Pinned: the Fig. 4 worked example.
//   or_select_consecutive
//   or_colour_unsharp,       Colour keyframe fusion (Section 3 "Keyframe Fusion", colour
//   or_colour_blurriness,    paragraph): unsharp masking, blurriness weight, back-warp,
//   or_weighted_median,      bilinear sampling, weighted median.  Pinned: the binomial's
//   or_fuse_colour           variance on x^2 images, linear images unchanged, the clamp;
//                            blurriness of ramp edges (width s: s/9 up to 5) and the luma
//                            weights; the weighted median as the smallest L1 minimiser;
//                            translated views of a ramp (sign and size of the warp, exact
//                            bilinear samples), w_z = cos(theta)/z^2 on a tilted plane,
//                            dropped occluded / out-of-view samples.
//   or_marching_cubes,       Marching Cubes (Section 3 "SDF volume") under a stated
//   or_mc_case               triangulation rule.  Pinned: single-corner, checkerboard and
//                            half-cube cases; a plane (vertices, area, orientation,
//                            skipped cubes); a sphere (distance bound, closed orientable
//                            genus-0 mesh, enclosed volume).
//   or_overlap, or_segment   Keyframe strategies KF_CONST / KF_DIST / KF_OVRLP (Section
//                            4.2).  Pinned: constant groups, translation and rotation
//                            steps against the distance thresholds, the closed-form
//                            overlap of sideways views of a plane.
//   or_loss, or_grad,        Loss on the fused SDF and its analytic gradient with
//   or_loss_perturbed        respect to keyframe se(3) poses and depth pixels (this
//                            extension has no counterpart in the paper).  Pinned: a
//                            plane moved along the optical axis (closed form), zero
//                            roll gradient for a fronto-parallel plane, and central
//                            finite differences of or_loss_perturbed.
//
// Readings of points the paper leaves open (pixel convention, normal estimate,
// discontinuity test, sampling weight, truncation band, the voxel set an
// integration touches, W' = 0 in Eq. 2, se(3) parameterisation) are stated
// where they are used below.
//
// Decision margins: float32 arithmetic on the GPU cannot reproduce every
// threshold decision of this double-precision reference exactly.  Each
// decision below therefore records its margin; an item whose margin is below
// tau (tau_px pixels for rounding, tau_m metres for distances) is flagged and
// the parity tests leave flagged items out of exact comparisons.

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <unordered_map>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

double g_tau_px = 5e-4;   // pixel-rounding margin (pixels)
double g_tau_m = 2e-6;    // distance margin (metres)
double g_tau_rel = 1e-6;  // relative margin for the discontinuity test

struct Intr {
    double fx, fy, cx, cy;
    int W, H;
};

// Pose T = (R, t) in SE(3), world_from_camera: g(T, p) = R p + t (Section 3
// "Preliminaries").  Stored as a row-major 3x4 matrix [R | t].
struct Pose {
    double R[3][3];
    double t[3];
};

Pose pose_from(const float* m) {
    Pose P;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) P.R[r][c] = (double)m[r * 4 + c];
        P.t[r] = (double)m[r * 4 + 3];
    }
    return P;
}

// g(T, p) = R p + t
void apply(const Pose& T, const double p[3], double out[3]) {
    for (int r = 0; r < 3; ++r) out[r] = T.R[r][0] * p[0] + T.R[r][1] * p[1] + T.R[r][2] * p[2] + T.t[r];
}

// g(T^-1, p) = R^T (p - t)
void apply_inv(const Pose& T, const double p[3], double out[3]) {
    double q[3] = {p[0] - T.t[0], p[1] - T.t[1], p[2] - T.t[2]};
    for (int r = 0; r < 3; ++r) out[r] = T.R[0][r] * q[0] + T.R[1][r] * q[1] + T.R[2][r] * q[2];
}

// pi^-1(x, Z): pixel centres at integer coordinates, Z is z-depth.
void backproject(const Intr& K, double u, double v, double Z, double out[3]) {
    out[0] = (u - K.cx) / K.fx * Z;
    out[1] = (v - K.cy) / K.fy * Z;
    out[2] = Z;
}

// Nearest pixel of a continuous image coordinate, halves rounded up:
// floor(a + 1/2).  Returns the margin: distance of a + 1/2 to the nearest
// integer (how far the coordinate is from a rounding tie).
long round_half_up(double a, double* margin) {
    double b = a + 0.5;
    double f = std::floor(b);
    double fr = b - f;
    *margin = std::min(fr, 1.0 - fr);
    return (long)f;
}

}  // namespace

// ============================================================================
// Keyframe depth fusion, Eq. 1 (Section 3 "Keyframe Fusion")
// ============================================================================
//
// For each frame i of the keyframe's group (in the given order) and each pixel
// x of Z_i (row-major):
//   * skip invalid depth (Z <= 0) and pixels close to depth discontinuities.
//     Reading: a pixel is kept only if all four 4-neighbours are valid and
//     |Z(n) - Z(x)| <= disc_rel * Z(x) for each; border pixels have no full
//     neighbourhood and are skipped.
//   * w_z(x) = cos(theta) * Z(x)^-2, theta the angle between the depth normal
//     and the camera axis.  Reading: normal = (P(u+1,v) - P(u-1,v)) x
//     (P(u,v+1) - P(u,v-1)) with P = pi^-1 in camera coordinates, and
//     cos(theta) = |n_z| / |n|.
//   * p* = g(T*^-1, g(T_i, pi^-1(x, Z_i(x)))); x* = pi(p*) rounded to the
//     nearest pixel (same rounding as the volume update); skip if Z*_p <= 0 or
//     x* falls outside the image.
//   * Eq. 1: Z*(x*) <- (W*(x*) Z*(x*) + w_z Z*_p) / (W*(x*) + w_z);
//            W*(x*) <- W*(x*) + w_z.
//     Reading: no z-test; every warped sample is averaged into its pixel.
// Z* and W* start at zero.  flag marks the target pixels a source pixel with a
// marginal decision may land in: x* and, for a marginal rounding, the pixel across
// the tie.
extern "C" int or_fuse(const float* depths, const float* poses, int n, const float* kf_pose,
                       double fx, double fy, double cx, double cy, int W, int H, double disc_rel,
                       double* Zs, double* Ws, uint8_t* flag) {
    const Intr K{fx, fy, cx, cy, W, H};
    const Pose Tk = pose_from(kf_pose);
    for (long p = 0; p < (long)W * H; ++p) {
        Zs[p] = 0.0;
        Ws[p] = 0.0;
        flag[p] = 0;
    }
    for (int f = 0; f < n; ++f) {
        const float* Z = depths + (long)f * W * H;
        const Pose Tf = pose_from(poses + 12 * f);
        for (int v = 0; v < H; ++v) {
            for (int u = 0; u < W; ++u) {
                double z = Z[(long)v * W + u];
                if (!(z > 0.0)) continue;
                if (u == 0 || v == 0 || u == W - 1 || v == H - 1) continue;
                double zn[4] = {Z[(long)v * W + u - 1], Z[(long)v * W + u + 1],
                                Z[(long)(v - 1) * W + u], Z[(long)(v + 1) * W + u]};
                if (!(zn[0] > 0.0 && zn[1] > 0.0 && zn[2] > 0.0 && zn[3] > 0.0)) continue;
                // discontinuity test (exact decision + its margin)
                bool keep = true, marginal = false;
                for (int k = 0; k < 4; ++k) {
                    double gap = std::fabs(zn[k] - z) - disc_rel * z;
                    if (std::fabs(gap) < g_tau_rel * z) marginal = true;
                    if (gap > 0.0) keep = false;
                }
                if (!keep && !marginal) continue;
                // warp into the keyframe: p* = g(T*^-1, g(T_i, pi^-1(x, Z_i(x))))
                double P[3], pw[3], ps[3];
                backproject(K, u, v, z, P);
                apply(Tf, P, pw);
                apply_inv(Tk, pw, ps);
                if (std::fabs(ps[2]) < g_tau_m) marginal = true;
                if (!(ps[2] > 0.0)) continue;
                double mu_, mv_;
                const double uf = K.fx * ps[0] / ps[2] + K.cx, vf = K.fy * ps[1] / ps[2] + K.cy;
                long xs = round_half_up(uf, &mu_);
                long ys = round_half_up(vf, &mv_);
                if (mu_ < g_tau_px || mv_ < g_tau_px) marginal = true;
                if (marginal) {
                    // the target pixels a float32 evaluation could pick: x* and, on each axis
                    // whose rounding is marginal, the neighbour across the tie
                    const long ax = mu_ < g_tau_px ? (uf + 0.5 - std::floor(uf + 0.5) < 0.5 ? xs - 1 : xs + 1) : xs;
                    const long ay = mv_ < g_tau_px ? (vf + 0.5 - std::floor(vf + 0.5) < 0.5 ? ys - 1 : ys + 1) : ys;
                    const long cxs[2] = {xs, ax}, cys[2] = {ys, ay};
                    for (int i = 0; i < 2; ++i)
                        for (int j = 0; j < 2; ++j) {
                            const long yy = cys[i], xx = cxs[j];
                            if (yy >= 0 && yy < H && xx >= 0 && xx < W) flag[yy * W + xx] = 1;
                        }
                }
                if (!keep) continue;
                if (xs < 0 || xs >= W || ys < 0 || ys >= H) continue;
                // w_z = cos(theta) / Z^2 from the central-difference depth normal
                double Pl[3], Pr[3], Pu[3], Pd[3];
                backproject(K, u - 1, v, zn[0], Pl);
                backproject(K, u + 1, v, zn[1], Pr);
                backproject(K, u, v - 1, zn[2], Pu);
                backproject(K, u, v + 1, zn[3], Pd);
                double a[3] = {Pr[0] - Pl[0], Pr[1] - Pl[1], Pr[2] - Pl[2]};
                double b[3] = {Pd[0] - Pu[0], Pd[1] - Pu[1], Pd[2] - Pu[2]};
                double nrm[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
                double nn = std::sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
                if (!(nn > 0.0)) continue;
                double cos_theta = std::fabs(nrm[2]) / nn;
                double wz = cos_theta / (z * z);
                long q = ys * W + xs;
                // Eq. 1
                Zs[q] = (Ws[q] * Zs[q] + wz * ps[2]) / (Ws[q] + wz);
                Ws[q] = Ws[q] + wz;
            }
        }
    }
    return 0;
}

// ============================================================================
// Voxel-hashed TSDF volume (Section 3 "SDF volume"; Section 4.3)
// ============================================================================
//
// Voxel i (integer 3-vector) sits at world position i * s.  Voxel blocks hold
// 8^3 voxels; block b covers voxel indices 8b .. 8b+7 on each axis and the
// closed world box [8 b s, 8 (b+1) s]^3.  Each voxel stores D (signed
// distance, metres), C (colour, RGB in 0..255) and W (integration weight).
// The block map is keyed by block coordinate; storage order is irrelevant.

namespace {

constexpr int BS = 8;
constexpr int NV = BS * BS * BS;

struct Block {
    double D[NV];
    double W[NV];
    double C[NV][3];
    uint8_t vflag[NV];
    uint8_t kflag[NV];  // clamp-kink marginal decisions among the integrated samples
    uint8_t bflag;
    Block() {
        std::memset(D, 0, sizeof(D));
        std::memset(W, 0, sizeof(W));
        std::memset(C, 0, sizeof(C));
        std::memset(vflag, 0, sizeof(vflag));
        std::memset(kflag, 0, sizeof(kflag));
        bflag = 0;
    }
};

int64_t pack(long x, long y, long z) {
    const long O = 1L << 20;
    return (int64_t)((x + O) | ((y + O) << 21) | ((z + O) << 42));
}
void unpack(int64_t k, long* x, long* y, long* z) {
    const long O = 1L << 20, M = (1L << 21) - 1;
    *x = (long)(k & M) - O;
    *y = (long)((k >> 21) & M) - O;
    *z = (long)((k >> 42) & M) - O;
}

long floor_div(long a, long b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

struct Touched {
    std::vector<int64_t> blocks;         // A(k, T): this keyframe's blocks, sorted
    std::vector<uint8_t> marginal;       // allocation decision uncertain for that block
};

struct Vol {
    double s, mu;
    int rgba8;  // 1: colour is stored as 8-bit integers (rounded after each update)
    std::unordered_map<int64_t, Block> blocks;
    std::map<int, Touched> touched;
    // blocks some integration reached only marginally (a float32 implementation
    // may allocate or update them where this reference does not)
    std::unordered_map<int64_t, uint8_t> ghosts;
    // voxel samples taken by integrations and de-integrations: projected (in front of
    // the camera) and with a value-changing marginal decision
    long n_proj = 0, n_vmarg = 0;
};

// Closed segment [q0, q1] against the closed box [lo, hi]^3 (slab test).
bool seg_box(const double q0[3], const double q1[3], const double lo[3], const double hi[3]) {
    double tmin = 0.0, tmax = 1.0;
    for (int a = 0; a < 3; ++a) {
        double d = q1[a] - q0[a];
        if (d == 0.0) {
            if (q0[a] < lo[a] || q0[a] > hi[a]) return false;
            continue;
        }
        double t0 = (lo[a] - q0[a]) / d, t1 = (hi[a] - q0[a]) / d;
        if (t0 > t1) std::swap(t0, t1);
        tmin = std::max(tmin, t0);
        tmax = std::min(tmax, t1);
        if (tmin > tmax) return false;
    }
    return true;
}

// A(k, T): allocation / visibility (Section 3 "SDF volume": blocks are first
// allocated, then voxels are updated).  Reading: for every valid pixel x the
// centre ray's band segment, camera z in [Z(x) - mu, Z(x) + mu], is taken to
// world coordinates; every block whose closed box meets that segment belongs to
// A(k, T).  Candidates are all blocks in the segment's bounding box (brute force).
// A block is "marginal" when the segment meets the box grown by tau_m but not the
// box shrunk by tau_m, for every pixel that reaches it.
void allocation_set(const Vol& V, const float* depth, const Intr& K, const Pose& T,
                    std::vector<int64_t>& out, std::vector<uint8_t>& marg) {
    const double B = BS * V.s;
    // per block: bit 0 = some pixel meets the exact box, bit 1 = some pixel meets the
    // shrunk box (robust member), bit 2 = some pixel meets the grown box
    std::map<int64_t, int> state;
    for (int v = 0; v < K.H; ++v) {
        for (int u = 0; u < K.W; ++u) {
            double z = depth[(long)v * K.W + u];
            if (!(z > 0.0)) continue;
            double c0[3], c1[3], q0[3], q1[3];
            backproject(K, u, v, z - V.mu, c0);
            backproject(K, u, v, z + V.mu, c1);
            apply(T, c0, q0);
            apply(T, c1, q1);
            long blo[3], bhi[3];
            for (int a = 0; a < 3; ++a) {
                double lo = std::min(q0[a], q1[a]), hi = std::max(q0[a], q1[a]);
                blo[a] = (long)std::ceil((lo - g_tau_m) / B) - 1;
                bhi[a] = (long)std::floor((hi + g_tau_m) / B);
            }
            for (long bz = blo[2]; bz <= bhi[2]; ++bz)
                for (long by = blo[1]; by <= bhi[1]; ++by)
                    for (long bx = blo[0]; bx <= bhi[0]; ++bx) {
                        double lo[3] = {bx * B, by * B, bz * B};
                        double hi[3] = {(bx + 1) * B, (by + 1) * B, (bz + 1) * B};
                        double lo_s[3], hi_s[3], lo_g[3], hi_g[3];
                        for (int a = 0; a < 3; ++a) {
                            lo_s[a] = lo[a] + g_tau_m;
                            hi_s[a] = hi[a] - g_tau_m;
                            lo_g[a] = lo[a] - g_tau_m;
                            hi_g[a] = hi[a] + g_tau_m;
                        }
                        int bits = (seg_box(q0, q1, lo, hi) ? 1 : 0) | (seg_box(q0, q1, lo_s, hi_s) ? 2 : 0) |
                                   (seg_box(q0, q1, lo_g, hi_g) ? 4 : 0);
                        if (bits) state[pack(bx, by, bz)] |= bits;
                    }
        }
    }
    out.clear();
    marg.clear();
    for (auto& kv : state) {
        out.push_back(kv.first);
        if (kv.second & 2) marg.push_back(0);        // robust member
        else if (kv.second & 1) marg.push_back(1);   // member by the exact test, marginal
        else marg.push_back(2);                      // marginal non-member
    }
}

// Per-voxel projective sample of keyframe (depth, colour) at pose T.
// Returns true when the voxel is updated; fills d, c and the decision margins.
struct Sample {
    bool upd;
    bool marginal;  // any decision within its margin (value-changing ones or the clamp kink)
    bool vmarg;     // a decision within its margin that can change W, D or C: the pixel
                    // rounding, the camera plane or the band edge (not the clamp kink,
                    // where d = min(eta, mu) is continuous)
    bool proj;      // in front of the camera: the nearest-pixel decision was taken
    bool kink;      // updated with eta within its margin of mu (the clamp decision)
    bool clamped;
    long pix;
    double d;
    double c[3];
    double pv[3];
    double zc;
};

Sample sample_voxel(const Vol& V, const float* depth, const uint8_t* rgba, const Intr& K, const Pose& T,
                    long ix, long iy, long iz) {
    Sample S{};
    S.upd = false;
    S.marginal = false;
    S.vmarg = false;
    S.proj = false;
    S.kink = false;
    S.pix = -1;
    S.pv[0] = ix * V.s;
    S.pv[1] = iy * V.s;
    S.pv[2] = iz * V.s;
    double pc[3];
    apply_inv(T, S.pv, pc);
    S.zc = pc[2];
    if (std::fabs(pc[2]) < g_tau_m) S.marginal = S.vmarg = true;
    if (!(pc[2] > 0.0)) return S;
    S.proj = true;
    double mu_, mv_;
    long px = round_half_up(K.fx * pc[0] / pc[2] + K.cx, &mu_);
    long py = round_half_up(K.fy * pc[1] / pc[2] + K.cy, &mv_);
    if (mu_ < g_tau_px || mv_ < g_tau_px) S.marginal = S.vmarg = true;
    S.pix = std::min(std::max(py, 0L), (long)K.H - 1) * K.W + std::min(std::max(px, 0L), (long)K.W - 1);
    if (px < 0 || px >= K.W || py < 0 || py >= K.H) return S;
    long q = py * K.W + px;
    double Z = depth[q];
    if (!(Z > 0.0)) return S;
    // projective distance along the camera z axis (Section 4.3): eta = Z(x) - z_c
    double eta = Z - pc[2];
    if (std::fabs(eta + V.mu) < g_tau_m) S.marginal = S.vmarg = true;
    if (eta < -V.mu) return S;  // far behind the observed surface: not updated
    S.upd = true;
    S.pix = q;
    S.clamped = !(eta < V.mu);
    if (std::fabs(eta - V.mu) < g_tau_m) S.marginal = S.kink = true;  // clamp kink (matters for gradients)
    S.d = std::min(eta, V.mu);
    if (rgba) {
        for (int ch = 0; ch < 3; ++ch) S.c[ch] = (double)rgba[4 * q + ch];
    } else {
        S.c[0] = S.c[1] = S.c[2] = 0.0;
    }
    return S;
}

double to_u8(double x) {
    // 8-bit storage: round half to even, saturate.
    double r = std::nearbyint(x);
    return std::min(255.0, std::max(0.0, r));
}

// Running weighted average (Section 3) with sign +1, or its inverse Eq. 2
// (Section 4.3) with sign -1.  Sampling weight w = 1 per keyframe observation
// (reading: the paper names w_i without giving its value).  When Eq. 2 brings W
// to zero the division is undefined; reading: the voxel returns to its empty
// state D = C = 0, W = 0 (the block stays allocated).
void update_blocks(Vol& V, const std::vector<int64_t>& blocks, const std::vector<uint8_t>& marg,
                   const float* depth, const uint8_t* rgba, const Intr& K, const Pose& T, int sign) {
    std::vector<Block*> ptrs(blocks.size(), nullptr);
    for (size_t b = 0; b < blocks.size(); ++b) {
        auto it = V.blocks.find(blocks[b]);
        if (it != V.blocks.end()) ptrs[b] = &it->second;
    }
    long n_proj = 0, n_vmarg = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : n_proj, n_vmarg)
    for (long b = 0; b < (long)blocks.size(); ++b) {
        Block* blk = ptrs[b];
        if (!blk) continue;
        if (marg[b]) blk->bflag = 1;
        if (marg[b] == 2) continue;  // marginal non-member: not part of A(k, T)
        long bx, by, bz;
        unpack(blocks[b], &bx, &by, &bz);
        for (int lz = 0; lz < BS; ++lz)
            for (int ly = 0; ly < BS; ++ly)
                for (int lx = 0; lx < BS; ++lx) {
                    int vi = lx + BS * ly + BS * BS * lz;
                    Sample S = sample_voxel(V, depth, rgba, K, T, bx * BS + lx, by * BS + ly, bz * BS + lz);
                    // vflag counts the value-changing marginal decisions among the
                    // samples currently integrated: Eq. 2 re-evaluates exactly the
                    // samples of the integration it undoes, so whatever a float32
                    // evaluation decided there it removes again (sticky once at 255)
                    if (S.vmarg && blk->vflag[vi] < 255) {
                        if (sign > 0) ++blk->vflag[vi];
                        else if (blk->vflag[vi] > 0) --blk->vflag[vi];
                    }
                    if (S.kink && blk->kflag[vi] < 255) {
                        if (sign > 0) ++blk->kflag[vi];
                        else if (blk->kflag[vi] > 0) --blk->kflag[vi];
                    }
                    n_proj += S.proj;
                    n_vmarg += S.vmarg;
                    if (!S.upd) continue;
                    const double w = 1.0;
                    double Wv = blk->W[vi];
                    if (sign > 0) {
                        blk->D[vi] = (blk->D[vi] * Wv + S.d * w) / (Wv + w);
                        for (int ch = 0; ch < 3; ++ch) {
                            double c = (blk->C[vi][ch] * Wv + S.c[ch] * w) / (Wv + w);
                            blk->C[vi][ch] = V.rgba8 ? to_u8(c) : c;
                        }
                        blk->W[vi] = Wv + w;
                    } else {
                        double Wn = Wv - w;  // Eq. 2
                        if (Wn == 0.0) {
                            blk->D[vi] = 0.0;
                            for (int ch = 0; ch < 3; ++ch) blk->C[vi][ch] = 0.0;
                        } else {
                            blk->D[vi] = (blk->D[vi] * Wv - S.d * w) / Wn;
                            for (int ch = 0; ch < 3; ++ch) {
                                double c = (blk->C[vi][ch] * Wv - S.c[ch] * w) / Wn;
                                blk->C[vi][ch] = V.rgba8 ? to_u8(c) : c;
                            }
                        }
                        blk->W[vi] = Wn;
                    }
                }
    }
    V.n_proj += n_proj;
    V.n_vmarg += n_vmarg;
}

}  // namespace

extern "C" void or_set_margins(double tau_px, double tau_m, double tau_rel) {
    g_tau_px = tau_px;
    g_tau_m = tau_m;
    g_tau_rel = tau_rel;
}

extern "C" void or_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

extern "C" int or_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

extern "C" void* or_vol_create(double voxel_size, double trunc, int rgba8) {
    Vol* V = new Vol();
    V->s = voxel_size;
    V->mu = trunc;
    V->rgba8 = rgba8;
    return V;
}

extern "C" void or_vol_destroy(void* vol) { delete (Vol*)vol; }

extern "C" void* or_vol_clone(void* vol) { return new Vol(*(Vol*)vol); }

// Integrate keyframe kf_id at pose T: first allocate A(k, T), then update the
// voxels of exactly those blocks (reading: an integration touches only the
// blocks its own band segments reach, so that Eq. 2 run on the same block list
// is its exact inverse).  Returns -1 if kf_id is already integrated.
extern "C" int or_integrate(void* vol, int kf_id, const float* depth, const uint8_t* rgba,
                            double fx, double fy, double cx, double cy, int W, int H, const float* pose) {
    Vol& V = *(Vol*)vol;
    if (V.touched.count(kf_id)) return -1;
    const Intr K{fx, fy, cx, cy, W, H};
    const Pose T = pose_from(pose);
    Touched tl;
    allocation_set(V, depth, K, T, tl.blocks, tl.marginal);
    for (size_t b = 0; b < tl.blocks.size(); ++b) {
        if (tl.marginal[b] != 2) V.blocks.try_emplace(tl.blocks[b]);
        if (tl.marginal[b] != 0) V.ghosts[tl.blocks[b]] = 1;
    }
    update_blocks(V, tl.blocks, tl.marginal, depth, rgba, K, T, +1);
    V.touched[kf_id] = std::move(tl);
    return 0;
}

// De-integrate keyframe kf_id, Eq. 2, with the depth, colour and pose it was
// integrated with, over its stored block list.  Returns -1 if not integrated.
extern "C" int or_deintegrate(void* vol, int kf_id, const float* depth, const uint8_t* rgba,
                              double fx, double fy, double cx, double cy, int W, int H, const float* pose) {
    Vol& V = *(Vol*)vol;
    auto it = V.touched.find(kf_id);
    if (it == V.touched.end()) return -1;
    const Intr K{fx, fy, cx, cy, W, H};
    const Pose T = pose_from(pose);
    update_blocks(V, it->second.blocks, it->second.marginal, depth, rgba, K, T, -1);
    V.touched.erase(it);
    return 0;
}

// One pose-graph update (Section 4.3 "Re-integration strategy"): de-integrate
// every item at its former pose, in item order, then integrate every item at
// its updated pose, in item order.  depths [n][H][W], rgba [n][H][W][4],
// poses [n][12].
extern "C" int or_reintegrate_batch(void* vol, int n, const int* kf_ids, const float* depths, const uint8_t* rgba,
                                    const float* old_poses, const float* new_poses,
                                    double fx, double fy, double cx, double cy, int W, int H) {
    long img = (long)W * H;
    for (int i = 0; i < n; ++i) {
        int rc = or_deintegrate(vol, kf_ids[i], depths + i * img, rgba ? rgba + 4 * i * img : nullptr,
                                fx, fy, cx, cy, W, H, old_poses + 12 * i);
        if (rc) return rc;
    }
    for (int i = 0; i < n; ++i) {
        int rc = or_integrate(vol, kf_ids[i], depths + i * img, rgba ? rgba + 4 * i * img : nullptr,
                              fx, fy, cx, cy, W, H, new_poses + 12 * i);
        if (rc) return rc;
    }
    return 0;
}

extern "C" long or_vol_num_blocks(void* vol) { return (long)((Vol*)vol)->blocks.size(); }

// Export blocks in ascending key order: coords [n][3], D/W [n][512], C [n][512][3],
// bflag [n], vflag [n][512].
extern "C" void or_vol_export(void* vol, int32_t* coords, double* D, double* Wt, double* C, uint8_t* bflag,
                              uint8_t* vflag) {
    Vol& V = *(Vol*)vol;
    std::vector<int64_t> keys;
    keys.reserve(V.blocks.size());
    for (auto& kv : V.blocks) keys.push_back(kv.first);
    std::sort(keys.begin(), keys.end());
    for (size_t i = 0; i < keys.size(); ++i) {
        long x, y, z;
        unpack(keys[i], &x, &y, &z);
        coords[3 * i] = (int32_t)x;
        coords[3 * i + 1] = (int32_t)y;
        coords[3 * i + 2] = (int32_t)z;
        const Block& b = V.blocks[keys[i]];
        if (D) std::memcpy(D + i * NV, b.D, sizeof(b.D));
        if (Wt) std::memcpy(Wt + i * NV, b.W, sizeof(b.W));
        if (C) std::memcpy(C + i * NV * 3, b.C, sizeof(b.C));
        if (bflag) bflag[i] = b.bflag | (V.ghosts.count(keys[i]) ? 1 : 0);
        if (vflag) std::memcpy(vflag + i * NV, b.vflag, NV);
    }
}

// Clamp-kink counts per voxel in the block order of or_vol_export: kflag [n][512].
// The kink leaves D, W and C alone (d = min(eta, mu) is continuous) but decides
// whether a sample has a derivative, so gradient comparisons need it.
extern "C" void or_vol_export_kink(void* vol, uint8_t* kflag) {
    Vol& V = *(Vol*)vol;
    std::vector<int64_t> keys;
    keys.reserve(V.blocks.size());
    for (auto& kv : V.blocks) keys.push_back(kv.first);
    std::sort(keys.begin(), keys.end());
    for (size_t i = 0; i < keys.size(); ++i) std::memcpy(kflag + i * NV, V.blocks[keys[i]].kflag, NV);
}

// Blocks that some integration reached only marginally and that this reference
// did not allocate: count, or fills coords [n][3].
extern "C" long or_vol_ghosts(void* vol, int32_t* coords) {
    Vol& V = *(Vol*)vol;
    std::vector<int64_t> keys;
    for (auto& kv : V.ghosts)
        if (!V.blocks.count(kv.first)) keys.push_back(kv.first);
    std::sort(keys.begin(), keys.end());
    if (coords) {
        for (size_t i = 0; i < keys.size(); ++i) {
            long x, y, z;
            unpack(keys[i], &x, &y, &z);
            coords[3 * i] = (int32_t)x;
            coords[3 * i + 1] = (int32_t)y;
            coords[3 * i + 2] = (int32_t)z;
        }
    }
    return (long)keys.size();
}

// The stored block list of kf_id: count, or fills coords [n][3] and marginal [n]
// (0 robust member, 1 marginal member, 2 marginal non-member).
extern "C" long or_vol_touched(void* vol, int kf_id, int32_t* coords, uint8_t* marginal) {
    Vol& V = *(Vol*)vol;
    auto it = V.touched.find(kf_id);
    if (it == V.touched.end()) return -1;
    const Touched& t = it->second;
    if (coords) {
        for (size_t i = 0; i < t.blocks.size(); ++i) {
            long x, y, z;
            unpack(t.blocks[i], &x, &y, &z);
            coords[3 * i] = (int32_t)x;
            coords[3 * i + 1] = (int32_t)y;
            coords[3 * i + 2] = (int32_t)z;
            if (marginal) marginal[i] = t.marginal[i];
        }
    }
    return (long)t.blocks.size();
}

// Allocation set A(k, T) alone, without touching any volume: returns the count
// or fills coords [n][3] and marginal [n] (as or_vol_touched).
extern "C" long or_allocation_set(double voxel_size, double trunc, const float* depth, double fx, double fy,
                                  double cx, double cy, int W, int H, const float* pose, int32_t* coords,
                                  uint8_t* marginal) {
    Vol V;
    V.s = voxel_size;
    V.mu = trunc;
    V.rgba8 = 0;
    const Intr K{fx, fy, cx, cy, W, H};
    std::vector<int64_t> out;
    std::vector<uint8_t> marg;
    allocation_set(V, depth, K, pose_from(pose), out, marg);
    if (coords) {
        for (size_t i = 0; i < out.size(); ++i) {
            long x, y, z;
            unpack(out[i], &x, &y, &z);
            coords[3 * i] = (int32_t)x;
            coords[3 * i + 1] = (int32_t)y;
            coords[3 * i + 2] = (int32_t)z;
            if (marginal) marginal[i] = marg[i];
        }
    }
    return (long)out.size();
}

// ============================================================================
// Keyframe selection (Section 4.3, Eq. 3, Fig. 4)
// ============================================================================

// ||s t_i - s t_i'|| with t = (Euler angles, translation), s = (2,2,2,1,1,1).
// Reading: Z-Y-X Euler angles (R = Rz(a) Ry(b) Rx(c)) of the world_from_camera
// rotation, in radians, each angle difference wrapped to (-pi, pi].
extern "C" double or_pose_distance(const float* T0, const float* T1) {
    auto euler = [](const Pose& P, double e[3]) {
        e[1] = std::asin(std::max(-1.0, std::min(1.0, -P.R[2][0])));
        e[0] = std::atan2(P.R[1][0], P.R[0][0]);
        e[2] = std::atan2(P.R[2][1], P.R[2][2]);
    };
    Pose A = pose_from(T0), B = pose_from(T1);
    double ea[3], eb[3];
    euler(A, ea);
    euler(B, eb);
    const double pi = 3.14159265358979323846;
    double acc = 0.0;
    for (int k = 0; k < 3; ++k) {
        double d = ea[k] - eb[k];
        while (d > pi) d -= 2 * pi;
        while (d <= -pi) d += 2 * pi;
        acc += (2.0 * d) * (2.0 * d);
    }
    for (int k = 0; k < 3; ++k) {
        double d = A.t[k] - B.t[k];
        acc += d * d;
    }
    return std::sqrt(acc);
}

// The m most-moved keyframes: descending distance, ties to the lower index.
extern "C" void or_select_topm(const double* dist, int K, int m, int* out) {
    std::vector<int> idx(K);
    for (int i = 0; i < K; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return dist[a] > dist[b]; });
    for (int i = 0; i < m && i < K; ++i) out[i] = idx[i];
}

// Eq. 3: first index j (0-based) of the m consecutive keyframes with the
// largest summed distance; ties to the smallest j.
extern "C" int or_select_consecutive(const double* dist, int K, int m, double* sums_out) {
    int best = -1;
    double best_sum = -1.0;
    for (int j = 0; j + m <= K; ++j) {
        double s = 0.0;
        for (int i = j; i < j + m; ++i) s += dist[i];
        if (sums_out) sums_out[j] = s;
        if (s > best_sum) {
            best_sum = s;
            best = j;
        }
    }
    return best;
}

// ============================================================================
// Loss on the fused SDF and its gradient (no counterpart in the paper)
// ============================================================================
//
// L = (1/P) sum_p Dt(p)^2 + lambda * sum_v W(v) D(v)^2 / sum_v W(v)
// Dt(p) is the trilinear interpolation of D over the 8 voxels around p (voxel i
// at i*s); points whose 8 voxels are not all observed (W > 0) are dropped and P
// counts the rest.  The second sum runs over voxels with W > 0.

namespace {

struct DOverlay {
    // optional replacement D values: block key -> D[512]
    const std::unordered_map<int64_t, std::vector<double>>* over = nullptr;
};

bool voxel_at(const Vol& V, const DOverlay& ov, long ix, long iy, long iz, double* D, double* W,
              bool* flagged = nullptr) {
    long bx = floor_div(ix, BS), by = floor_div(iy, BS), bz = floor_div(iz, BS);
    int64_t key = pack(bx, by, bz);
    auto it = V.blocks.find(key);
    if (it == V.blocks.end()) {
        if (flagged && V.ghosts.count(key)) *flagged = true;
        return false;
    }
    int vi = (int)(ix - bx * BS) + BS * (int)(iy - by * BS) + BS * BS * (int)(iz - bz * BS);
    if (flagged && (it->second.bflag || it->second.vflag[vi] || V.ghosts.count(key))) *flagged = true;
    *W = it->second.W[vi];
    *D = it->second.D[vi];
    if (ov.over) {
        auto jt = ov.over->find(key);
        if (jt != ov.over->end()) *D = jt->second[vi];
    }
    return *W > 0.0;
}

struct PointEval {
    bool valid;
    bool marginal;
    double Dt;
    long ix[8], iy[8], iz[8];
    double beta[8];
};

// marginal: the floor of a grid coordinate is within 1e-6 of a tie, or one of the
// 8 corners (up to the first unobserved one) has a marginal decision
PointEval eval_point(const Vol& V, const DOverlay& ov, const double* p) {
    PointEval E{};
    E.valid = false;
    E.marginal = false;
    double g[3], f[3];
    long i0[3];
    for (int a = 0; a < 3; ++a) {
        g[a] = p[a] / V.s;
        double fl = std::floor(g[a]);
        i0[a] = (long)fl;
        f[a] = g[a] - fl;
        if (f[a] < 1e-6 || f[a] > 1.0 - 1e-6) E.marginal = true;
    }
    double acc = 0.0;
    for (int c = 0; c < 8; ++c) {
        int ox = c & 1, oy = (c >> 1) & 1, oz = (c >> 2) & 1;
        E.ix[c] = i0[0] + ox;
        E.iy[c] = i0[1] + oy;
        E.iz[c] = i0[2] + oz;
        E.beta[c] = (ox ? f[0] : 1 - f[0]) * (oy ? f[1] : 1 - f[1]) * (oz ? f[2] : 1 - f[2]);
        double D, W;
        // a corner with a marginal decision may be observed on one side only
        if (!voxel_at(V, ov, E.ix[c], E.iy[c], E.iz[c], &D, &W, &E.marginal)) return E;
        acc += E.beta[c] * D;
    }
    E.valid = true;
    E.Dt = acc;
    return E;
}

double loss_impl(const Vol& V, const DOverlay& ov, const double* pts, long n, double lambda, long* n_valid,
                 uint8_t* pflag) {
    double s1 = 0.0;
    long P = 0;
    for (long i = 0; i < n; ++i) {
        PointEval E = eval_point(V, ov, pts + 3 * i);
        if (pflag) pflag[i] = E.marginal;
        if (!E.valid) continue;
        s1 += E.Dt * E.Dt;
        ++P;
    }
    double swd = 0.0, sw = 0.0;
    for (auto& kv : V.blocks) {
        const std::vector<double>* od = nullptr;
        if (ov.over) {
            auto jt = ov.over->find(kv.first);
            if (jt != ov.over->end()) od = &jt->second;
        }
        for (int vi = 0; vi < NV; ++vi) {
            double W = kv.second.W[vi];
            if (!(W > 0.0)) continue;
            double D = od ? (*od)[vi] : kv.second.D[vi];
            swd += W * D * D;
            sw += W;
        }
    }
    if (n_valid) *n_valid = P;
    double L = (P > 0 ? s1 / (double)P : 0.0);
    if (sw > 0.0) L += lambda * swd / sw;
    return L;
}

// T(xi) = exp(xi^) T with xi = (rho, omega) (reading: left perturbation of the
// world_from_camera pose, Rodrigues exponential).
Pose perturb(const Pose& T, const double* xi) {
    const double* rho = xi;
    const double* w = xi + 3;
    double th = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double Kx[3][3] = {{0, -w[2], w[1]}, {w[2], 0, -w[0]}, {-w[1], w[0], 0}};
    double K2[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            K2[r][c] = 0;
            for (int k = 0; k < 3; ++k) K2[r][c] += Kx[r][k] * Kx[k][c];
        }
    double A, Bc, Cc;
    if (th < 1e-8) {
        A = 1.0 - th * th / 6.0;
        Bc = 0.5 - th * th / 24.0;
        Cc = 1.0 / 6.0 - th * th / 120.0;
    } else {
        A = std::sin(th) / th;
        Bc = (1 - std::cos(th)) / (th * th);
        Cc = (th - std::sin(th)) / (th * th * th);
    }
    double Rx[3][3], Vx[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double I = (r == c) ? 1.0 : 0.0;
            Rx[r][c] = I + A * Kx[r][c] + Bc * K2[r][c];
            Vx[r][c] = I + Bc * Kx[r][c] + Cc * K2[r][c];
        }
    Pose O;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            O.R[r][c] = 0;
            for (int k = 0; k < 3; ++k) O.R[r][c] += Rx[r][k] * T.R[k][c];
        }
        O.t[r] = 0;
        for (int k = 0; k < 3; ++k) O.t[r] += Rx[r][k] * T.t[k] + Vx[r][k] * rho[k];
    }
    return O;
}

}  // namespace

extern "C" double or_loss(void* vol, const double* pts, long n, double lambda, long* n_valid, uint8_t* pflag) {
    DOverlay ov;
    return loss_impl(*(Vol*)vol, ov, pts, n, lambda, n_valid, pflag);
}

// Analytic gradient of L with respect to each listed keyframe's pose (left
// se(3) perturbation xi = (rho, omega) at xi = 0) and depth pixels.
//   D(v) = sum_k w_k d_k(v) / W(v)  =>  dD(v)/dd_k = w_k / W(v)
//   d_k = Z_k(x) - z_c  when unclamped (eta < mu), else mu (zero derivative)
//   dd/dZ_k(x) = 1;  dd/dxi = -dz_c/dxi,  p_c = R^T (p_v - t)
//   dp_c/drho = -R^T,  dp_c/domega = R^T [p_v]_x
// Pixel assignment, band membership and the clamp are piecewise constant in the
// pose and depth; they contribute no derivative.
// grad_xi [K][6] (rho then omega), grad_depth [K][H][W] (may be null).
// err_xi [K][6] and err_depth [K][H][W] (each may be null) receive an error
// budget: the summed magnitudes of the contributions whose decisions are marginal
// (a voxel's rounding, band edge, clamp kink or camera plane; every voxel of a block
// whose allocation is marginal) -- contributions a float32 evaluation may include,
// drop or move to a neighbouring pixel.  Contributions this reference does not
// make at all (marginal voxels it does not update, blocks it does not allocate)
// are bounded with the largest |dL/dD / W| of the volume.
extern "C" int or_grad(void* vol, int K_, const int* kf_ids, const float* depths, const uint8_t* rgba,
                       const float* poses, double fx, double fy, double cx, double cy, int W, int H,
                       const double* pts, long n, double lambda, double* grad_xi, double* grad_depth,
                       double* err_xi, double* err_depth) {
    Vol& V = *(Vol*)vol;
    const Intr K{fx, fy, cx, cy, W, H};
    DOverlay ov;
    // dL/dD(v)
    std::unordered_map<int64_t, std::vector<double>> G;
    double sw = 0.0;
    for (auto& kv : V.blocks)
        for (int vi = 0; vi < NV; ++vi)
            if (kv.second.W[vi] > 0.0) sw += kv.second.W[vi];
    for (auto& kv : V.blocks) {
        std::vector<double> g(NV, 0.0);
        for (int vi = 0; vi < NV; ++vi)
            if (kv.second.W[vi] > 0.0 && sw > 0.0) g[vi] = 2.0 * lambda * kv.second.W[vi] * kv.second.D[vi] / sw;
        G.emplace(kv.first, std::move(g));
    }
    std::vector<PointEval> evs;
    long P = 0;
    for (long i = 0; i < n; ++i) {
        PointEval E = eval_point(V, ov, pts + 3 * i);
        if (E.valid) {
            evs.push_back(E);
            ++P;
        }
    }
    for (const PointEval& E : evs) {
        for (int c = 0; c < 8; ++c) {
            long bx = floor_div(E.ix[c], BS), by = floor_div(E.iy[c], BS), bz = floor_div(E.iz[c], BS);
            int vi = (int)(E.ix[c] - bx * BS) + BS * (int)(E.iy[c] - by * BS) + BS * BS * (int)(E.iz[c] - bz * BS);
            G[pack(bx, by, bz)][vi] += 2.0 / (double)P * E.Dt * E.beta[c];
        }
    }
    // largest |dL/dD / W| of any observed voxel: bounds contributions this reference
    // does not make but a float32 evaluation may
    double gmax = 0.0;
    for (auto& kv : V.blocks)
        for (int vi = 0; vi < NV; ++vi)
            if (kv.second.W[vi] > 0.0) gmax = std::max(gmax, std::fabs(G.at(kv.first)[vi] / kv.second.W[vi]));
    long img = (long)W * H;
    for (int k = 0; k < K_; ++k) {
        double* gx = grad_xi + 6 * k;
        for (int j = 0; j < 6; ++j) gx[j] = 0.0;
        double* ex = err_xi ? err_xi + 6 * k : nullptr;
        if (ex)
            for (int j = 0; j < 6; ++j) ex[j] = 0.0;
        double* gd = grad_depth ? grad_depth + k * img : nullptr;
        if (gd)
            for (long q = 0; q < img; ++q) gd[q] = 0.0;
        double* ed = err_depth ? err_depth + k * img : nullptr;
        if (ed)
            for (long q = 0; q < img; ++q) ed[q] = 0.0;
        auto it = V.touched.find(kf_ids[k]);
        if (it == V.touched.end()) return -1;
        const Pose T = pose_from(poses + 12 * k);
        const float* depth = depths + k * img;
        const double r3[3] = {T.R[0][2], T.R[1][2], T.R[2][2]};  // third row of R^T
        const Touched& tl = it->second;
        auto budget = [&](const Sample& S, double gv_abs) {
            const double* p = S.pv;
            const double cx_[3] = {p[1] * r3[2] - p[2] * r3[1], p[2] * r3[0] - p[0] * r3[2],
                                   p[0] * r3[1] - p[1] * r3[0]};
            if (ex)
                for (int j = 0; j < 3; ++j) {
                    ex[j] += gv_abs * std::fabs(r3[j]);
                    ex[3 + j] += gv_abs * std::fabs(cx_[j]);
                }
            if (ed && S.pix >= 0) {
                const long px = S.pix % W, py = S.pix / W;
                for (long dy = -1; dy <= 1; ++dy)
                    for (long dx = -1; dx <= 1; ++dx) {
                        const long yy = py + dy, xx = px + dx;
                        if (yy >= 0 && yy < H && xx >= 0 && xx < W) ed[yy * W + xx] += gv_abs;
                    }
            }
        };
        for (size_t b = 0; b < tl.blocks.size(); ++b) {
            long bx, by, bz;
            unpack(tl.blocks[b], &bx, &by, &bz);
            const bool ghost = tl.marginal[b] == 2;
            const bool bmarg = tl.marginal[b] != 0;
            const Block* blk = ghost ? nullptr : &V.blocks.at(tl.blocks[b]);
            const std::vector<double>* g = ghost ? nullptr : &G.at(tl.blocks[b]);
            for (int lz = 0; lz < BS; ++lz)
                for (int ly = 0; ly < BS; ++ly)
                    for (int lx = 0; lx < BS; ++lx) {
                        int vi = lx + BS * ly + BS * BS * lz;
                        Sample S = sample_voxel(V, depth, nullptr, K, T, bx * BS + lx, by * BS + ly, bz * BS + lz);
                        if (ghost) {
                            // a block only a float32 evaluation may allocate for this keyframe
                            if (S.upd || S.marginal) budget(S, gmax);
                            continue;
                        }
                        if (!S.upd) {
                            if (S.marginal || bmarg) budget(S, gmax);
                            continue;
                        }
                        const bool marg = S.marginal || bmarg;
                        if (S.clamped && !marg) continue;
                        const double gv = (*g)[vi] * 1.0 / blk->W[vi];
                        if (!S.clamped) {
                            // -dz_c/drho = r3 ; -dz_c/domega = -(r3 x p_v) = p_v x r3
                            const double* p = S.pv;
                            const double cx_[3] = {p[1] * r3[2] - p[2] * r3[1], p[2] * r3[0] - p[0] * r3[2],
                                                   p[0] * r3[1] - p[1] * r3[0]};
                            if (gd) gd[S.pix] += gv;
                            for (int j = 0; j < 3; ++j) {
                                gx[j] += gv * r3[j];
                                gx[3 + j] += gv * cx_[j];
                            }
                        }
                        // a marginal voxel's W may differ by one on the float32 side
                        if (marg) budget(S, std::max(std::fabs(gv), gmax));
                    }
        }
    }
    (void)rgba;
    return 0;
}

// Loss with keyframe kf_ids[k_sel]'s contribution re-evaluated at the perturbed
// pose exp(xi^) T_k and depth Z_k + dz * [pixel == pix] (pix < 0: no depth
// change), with every discrete decision (pixel, band membership, clamp) frozen
// at the unperturbed state:  D'(v) = D(v) + (d_k(v; xi, dz) - d_k(v; 0)) w / W(v).
// Used for central finite differences.
extern "C" double or_loss_perturbed(void* vol, int kf_id, const float* depth, const float* pose, double fx,
                                    double fy, double cx, double cy, int W, int H, const double* xi, long pix,
                                    double dz, const double* pts, long n, double lambda) {
    Vol& V = *(Vol*)vol;
    const Intr K{fx, fy, cx, cy, W, H};
    auto it = V.touched.find(kf_id);
    if (it == V.touched.end()) return NAN;
    const Pose T = pose_from(pose);
    const Pose Tp = perturb(T, xi);
    std::unordered_map<int64_t, std::vector<double>> over;
    const Touched& tl = it->second;
    for (size_t b = 0; b < tl.blocks.size(); ++b) {
        if (tl.marginal[b] == 2) continue;
        long bx, by, bz;
        unpack(tl.blocks[b], &bx, &by, &bz);
        const Block& blk = V.blocks.at(tl.blocks[b]);
        std::vector<double> D(blk.D, blk.D + NV);
        bool any = false;
        for (int lz = 0; lz < BS; ++lz)
            for (int ly = 0; ly < BS; ++ly)
                for (int lx = 0; lx < BS; ++lx) {
                    int vi = lx + BS * ly + BS * BS * lz;
                    Sample S = sample_voxel(V, depth, nullptr, K, T, bx * BS + lx, by * BS + ly, bz * BS + lz);
                    if (!S.upd || S.clamped) continue;
                    double pc[3];
                    apply_inv(Tp, S.pv, pc);
                    double Z = (double)depth[S.pix] + (S.pix == pix ? dz : 0.0);
                    double d_new = Z - pc[2];
                    D[vi] += (d_new - S.d) * 1.0 / blk.W[vi];
                    any = true;
                }
        if (any) over.emplace(tl.blocks[b], std::move(D));
    }
    DOverlay ov;
    ov.over = &over;
    return loss_impl(V, ov, pts, n, lambda, nullptr, nullptr);
}

// Sample counts of all integrations and de-integrations so far: out[0] voxel
// samples in front of the camera, out[1] samples with a value-changing marginal
// decision (pixel rounding, camera plane, band edge).
extern "C" void or_vol_stats(void* vol, long* out) {
    const Vol& V = *(const Vol*)vol;
    out[0] = V.n_proj;
    out[1] = V.n_vmarg;
}

namespace {

// Cotangent dL/dD given per block: coords [n][3], values [n][512].
std::unordered_map<int64_t, const double*> cotangent_map(long n, const int32_t* coords, const double* vals) {
    std::unordered_map<int64_t, const double*> G;
    for (long i = 0; i < n; ++i) G[pack(coords[3 * i], coords[3 * i + 1], coords[3 * i + 2])] = vals + i * NV;
    return G;
}

// The contribution status of voxel (ix, iy, iz) sampled at pixel q of keyframe depth:
// 1 if updated without clamping (eta in [-mu, mu)), else 0.  Used for the other
// outcomes of a marginal rounding.
int status_at(const Vol& V, const float* depth, const Intr& K, double zc, long qx, long qy) {
    if (!(zc > 0.0) || qx < 0 || qx >= K.W || qy < 0 || qy >= K.H) return 0;
    const double Z = depth[qy * K.W + qx];
    if (!(Z > 0.0)) return 0;
    const double eta = Z - zc;
    return (eta >= -V.mu && eta < V.mu) ? 1 : 0;
}

}  // namespace

// Vector-Jacobian product of the keyframe integrations (the adjoint) for a given
// cotangent G = dL/dD (per voxel) on this volume:
//   D(v) = sum_k w_k d_k(v) / W(v)  =>  dL/dd_k(v) = G(v) w / W(v)  (w = 1)
//   d_k = Z_k(x) - z_c when unclamped, else mu;  dd/dZ_k(x) = 1,
//   dd/drho = r3, dd/domega = p_v x r3  (left perturbation, r3 = R e3),
// summed over the voxels of each keyframe's stored block list (marginal
// non-members excluded).  Voxels with W = 0 or G = 0 contribute nothing.
// err_xi [K][6] / err_depth [K][H][W] (may be null) bound what a float32
// evaluation may do differently: a marginal decision whose other outcome changes
// whether the sample contributes adds |G/W| times the derivative magnitudes to
// the pose budget; a contributing sample with a marginal rounding adds |G/W| to
// the depth budget at its pixel and at each pixel across the tie (the pose
// derivative does not depend on the pixel, the depth gradient does).
extern "C" int or_adjoint(void* vol, int K_, const int* kf_ids, const float* depths, const float* poses, double fx,
                          double fy, double cx, double cy, int W, int H, long n_g, const int32_t* g_coords,
                          const double* g_vals, double* grad_xi, double* grad_depth, double* err_xi,
                          double* err_depth) {
    Vol& V = *(Vol*)vol;
    const Intr K{fx, fy, cx, cy, W, H};
    const auto G = cotangent_map(n_g, g_coords, g_vals);
    const long img = (long)W * H;
    for (int k = 0; k < K_; ++k) {
        auto it = V.touched.find(kf_ids[k]);
        if (it == V.touched.end()) return -1;
        double* gx = grad_xi + 6 * k;
        double* ex = err_xi ? err_xi + 6 * k : nullptr;
        double* gd = grad_depth ? grad_depth + k * img : nullptr;
        double* ed = err_depth ? err_depth + k * img : nullptr;
        for (int j = 0; j < 6; ++j) {
            gx[j] = 0.0;
            if (ex) ex[j] = 0.0;
        }
        for (long q = 0; gd && q < img; ++q) gd[q] = 0.0;
        for (long q = 0; ed && q < img; ++q) ed[q] = 0.0;
        const Pose T = pose_from(poses + 12 * k);
        const float* depth = depths + k * img;
        const double r3[3] = {T.R[0][2], T.R[1][2], T.R[2][2]};
        const Touched& tl = it->second;
        for (size_t b = 0; b < tl.blocks.size(); ++b) {
            if (tl.marginal[b] == 2) continue;
            auto gi = G.find(tl.blocks[b]);
            if (gi == G.end()) continue;
            const Block& blk = V.blocks.at(tl.blocks[b]);
            long bx, by, bz;
            unpack(tl.blocks[b], &bx, &by, &bz);
            for (int vi = 0; vi < NV; ++vi) {
                const double g = gi->second[vi];
                if (g == 0.0 || !(blk.W[vi] > 0.0)) continue;
                const long ix = bx * BS + vi % BS, iy = by * BS + (vi / BS) % BS, iz = bz * BS + vi / (BS * BS);
                const Sample S = sample_voxel(V, depth, nullptr, K, T, ix, iy, iz);
                const double gv = g / blk.W[vi];
                const double* p = S.pv;
                const double px_[3] = {p[1] * r3[2] - p[2] * r3[1], p[2] * r3[0] - p[0] * r3[2],
                                       p[0] * r3[1] - p[1] * r3[0]};
                const int base = (S.upd && !S.clamped) ? 1 : 0;
                if (base) {
                    for (int j = 0; j < 3; ++j) {
                        gx[j] += gv * r3[j];
                        gx[3 + j] += gv * px_[j];
                    }
                    if (gd) gd[S.pix] += gv;
                }
                if (!S.marginal) continue;
                // the other outcomes a float32 evaluation may take
                bool flips = false;
                double pc[3];
                apply_inv(T, S.pv, pc);
                if (std::fabs(pc[2]) < g_tau_m) flips = true;  // camera plane
                if (S.proj) {
                    // S.pix is the nearest pixel clamped into the image; it is the
                    // sampled pixel whenever the rounding put the voxel inside
                    const double Z = depth[S.pix];
                    const double eta = Z - pc[2];
                    if (S.upd || Z > 0.0) {
                        if (std::fabs(eta + V.mu) < g_tau_m) flips = true;  // band edge
                        if (std::fabs(eta - V.mu) < g_tau_m) flips = true;  // clamp kink
                    }
                }
                std::vector<long> alts;  // pixels across a marginal rounding tie
                if (pc[2] > 0.0) {
                    const double uf = K.fx * pc[0] / pc[2] + K.cx, vf = K.fy * pc[1] / pc[2] + K.cy;
                    double mu_, mv_;
                    const long qx = round_half_up(uf, &mu_), qy = round_half_up(vf, &mv_);
                    const long ax = (uf + 0.5 - std::floor(uf + 0.5) < 0.5) ? qx - 1 : qx + 1;
                    const long ay = (vf + 0.5 - std::floor(vf + 0.5) < 0.5) ? qy - 1 : qy + 1;
                    const bool mu_m = mu_ < g_tau_px, mv_m = mv_ < g_tau_px;
                    const long cand[3][2] = {{ax, qy}, {qx, ay}, {ax, ay}};
                    const bool use[3] = {mu_m, mv_m, mu_m && mv_m};
                    for (int c = 0; c < 3; ++c) {
                        if (!use[c]) continue;
                        const int st = status_at(V, depth, K, pc[2], cand[c][0], cand[c][1]);
                        if (st != base) flips = true;
                        if (st) alts.push_back(cand[c][1] * W + cand[c][0]);
                    }
                }
                const double ag = std::fabs(gv);
                if (flips && ex)
                    for (int j = 0; j < 3; ++j) {
                        ex[j] += ag * std::fabs(r3[j]);
                        ex[3 + j] += ag * std::fabs(px_[j]);
                    }
                if (ed) {
                    if (flips && base) ed[S.pix] += ag;
                    if (!alts.empty()) {
                        if (base) ed[S.pix] += ag;
                        for (long q : alts) ed[q] += ag;
                    }
                }
            }
        }
    }
    return 0;
}

// The functional L_G(xi, dz) = sum_v G(v) D(v) with keyframe kf_id's contribution
// re-evaluated at exp(xi^) T and depth Z + dz at pixel pix (pix < 0: none), every
// discrete decision frozen at the unperturbed state; its central differences
// check or_adjoint.
extern "C" double or_adjoint_functional(void* vol, int kf_id, const float* depth, const float* pose, double fx,
                                        double fy, double cx, double cy, int W, int H, const double* xi, long pix,
                                        double dz, long n_g, const int32_t* g_coords, const double* g_vals) {
    Vol& V = *(Vol*)vol;
    const Intr K{fx, fy, cx, cy, W, H};
    auto it = V.touched.find(kf_id);
    if (it == V.touched.end()) return NAN;
    const auto G = cotangent_map(n_g, g_coords, g_vals);
    const Pose T = pose_from(pose);
    const Pose Tp = perturb(T, xi);
    // sum over the keyframe's voxels of G (d(xi) - d(0)) w / W; the other keyframes'
    // terms and this keyframe's unperturbed terms are constant and cancel in a
    // central difference, so only the change is summed
    double acc = 0.0;
    const Touched& tl = it->second;
    for (size_t b = 0; b < tl.blocks.size(); ++b) {
        if (tl.marginal[b] == 2) continue;
        auto gi = G.find(tl.blocks[b]);
        if (gi == G.end()) continue;
        const Block& blk = V.blocks.at(tl.blocks[b]);
        long bx, by, bz;
        unpack(tl.blocks[b], &bx, &by, &bz);
        for (int vi = 0; vi < NV; ++vi) {
            const double g = gi->second[vi];
            if (g == 0.0 || !(blk.W[vi] > 0.0)) continue;
            const Sample S = sample_voxel(V, depth, nullptr, K, T, bx * BS + vi % BS, by * BS + (vi / BS) % BS,
                                          bz * BS + vi / (BS * BS));
            if (!S.upd || S.clamped) continue;
            double pc[3];
            apply_inv(Tp, S.pv, pc);
            const double Z = (double)depth[S.pix] + (S.pix == pix ? dz : 0.0);
            acc += g * ((Z - pc[2]) - S.d) / blk.W[vi];
        }
    }
    return acc;
}

// ============================================================================
// Colour keyframe fusion (Section 3 "Keyframe Fusion", colour paragraph)
// ============================================================================
//
// Three steps, in the order the paper gives them:
//  1. every input colour image C_i is deblurred by unsharp masking;
//  2. a blurriness measure of C_i gives the per-frame weight w_b;
//  3. each keyframe pixel x* is warped back into every frame i of its group with
//     the keyframe depth Z*, the deblurred colour is sampled there bilinearly and
//     weighted by w_c = w_b * w_z; C*(x*) is the weighted median of the samples.
//
// Readings (the paper names the operations, not their parameters):
//  * unsharp masking: S = I + (I - G*I), G the 5x5 binomial filter (1 4 6 4 1)/16
//    on each axis (variance 1 per axis), amount 1, image borders replicated, S
//    clamped to [0, 255]; R, G, B separately.
//  * blurriness: the no-reference blur measure of Crete-Roffet et al. (2007) on the
//    luma Y = (77 R + 150 G + 29 B) / 256 of the input image.  Per direction e:
//    B = 9-tap box mean of Y along e (borders replicated), D_F = |Y(p) - Y(p - e)|,
//    D_B = |B(p) - B(p - e)|, V = max(0, D_F - D_B), summed over every pixel p whose
//    p - e is inside the image; b_e = (sum D_F - sum V) / sum D_F, and b_e = 0 when
//    sum D_F = 0 (no edge, no evidence of blur).  b = max(b_vertical, b_horizontal)
//    lies in [0, 1]; w_b = 1 - b.
//  * w_z = cos(theta) / z_i^2 as in Eq. 1: z_i the depth of the point in frame i,
//    theta the angle between frame i's optical axis and the surface normal.  The
//    normal is Eq. 1's central-difference normal of Z* at x* (same neighbour and
//    discontinuity test), rotated into frame i.  A keyframe pixel with Z* <= 0 or
//    without a valid normal gets no colour.
//  * an observation is valid if z_i > 0, the sample point (u, v) lies in
//    [0, W-1] x [0, H-1], and frame i's depth at the nearest pixel agrees with the
//    point: Z_i > 0 and |Z_i - z_i| <= occl_rel * z_i (occlusion test).  Frames with
//    w_b = 0 contribute nothing.
//  * weighted median, per channel: the smallest sample value m with
//    sum_{j : c_j <= m} w_j >= (sum_j w_j) / 2.  The colour is m rounded to the
//    nearest integer, halves up, alpha 255; no observation gives (0, 0, 0, 0).
//
// Margins: flag marks keyframe pixels where a float32 evaluation may take another
// discrete decision (normal test, z_i sign, footprint bounds, occlusion pixel or
// threshold, which sample crosses half the weight given the weights' float32
// error).  err bounds, per channel, how far an unflagged median can move when
// every sample point moves by tau_px pixels:
// bilinear sampling is Lipschitz in the position with the cell's largest
// differences, and the weighted median moves by at most the largest sample move.

namespace {

constexpr int kBinom[5] = {1, 4, 6, 4, 1};

inline long clampl(long a, long lo, long hi) { return a < lo ? lo : (a > hi ? hi : a); }

// Unsharp masking of one RGBA8 image into S[H][W][3] (double, exact: every value is
// a multiple of 1/256).  The 5x5 filter is applied as one 2-D sum.
void unsharp(const uint8_t* rgba, int W, int H, double* S) {
#pragma omp parallel for schedule(static)
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < W; ++x)
            for (int c = 0; c < 3; ++c) {
                double blur = 0.0;
                for (int b = -2; b <= 2; ++b)
                    for (int a = -2; a <= 2; ++a) {
                        const long yy = clampl(y + b, 0, H - 1), xx = clampl(x + a, 0, W - 1);
                        blur += (double)(kBinom[a + 2] * kBinom[b + 2]) * rgba[(yy * W + xx) * 4 + c];
                    }
                blur /= 256.0;
                const double I = rgba[(y * W + x) * 4 + c];
                double s = I + (I - blur);
                S[(y * W + x) * 3 + c] = s < 0.0 ? 0.0 : (s > 255.0 ? 255.0 : s);
            }
}

// Crete-Roffet blurriness of one RGBA8 image, in [0, 1].
double blurriness(const uint8_t* rgba, int W, int H) {
    std::vector<double> Y((size_t)W * H);
    for (long p = 0; p < (long)W * H; ++p)
        Y[p] = (77.0 * rgba[p * 4] + 150.0 * rgba[p * 4 + 1] + 29.0 * rgba[p * 4 + 2]) / 256.0;
    double b_dir[2];
    for (int dir = 0; dir < 2; ++dir) {  // 0: vertical (e = one row), 1: horizontal (e = one column)
        const int ex = dir == 1, ey = dir == 0;
        std::vector<double> B((size_t)W * H);
        for (long y = 0; y < H; ++y)
            for (long x = 0; x < W; ++x) {
                double s = 0.0;
                for (int k = -4; k <= 4; ++k) {
                    const long yy = clampl(y + k * ey, 0, H - 1), xx = clampl(x + k * ex, 0, W - 1);
                    s += Y[yy * W + xx];
                }
                B[y * W + x] = s / 9.0;
            }
        double sF = 0.0, sV = 0.0;
        for (long y = ey; y < H; ++y)
            for (long x = ex; x < W; ++x) {
                const long p = y * W + x, q = (y - ey) * W + (x - ex);
                const double dF = std::fabs(Y[p] - Y[q]);
                const double dB = std::fabs(B[p] - B[q]);
                sF += dF;
                sV += std::max(0.0, dF - dB);
            }
        b_dir[dir] = sF > 0.0 ? (sF - sV) / sF : 0.0;
    }
    return std::max(b_dir[0], b_dir[1]);
}

// Lower weighted median of (c_j, w_j): sort by value, walk the cumulative weight.
// near_tie reports whether some cumulative sum at a change of value lies within
// tol of half the total.
double weighted_median(std::vector<std::pair<double, double>> obs, double tol, bool* near_tie) {
    std::sort(obs.begin(), obs.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    double total = 0.0;
    for (const auto& o : obs) total += o.second;
    const double half = 0.5 * total;
    double cum = 0.0, m = obs.back().first;
    bool found = false;
    *near_tie = false;
    for (size_t k = 0; k < obs.size(); ++k) {
        cum += obs[k].second;
        const bool last_of_value = k + 1 == obs.size() || obs[k + 1].first != obs[k].first;
        if (!last_of_value) continue;
        if (k + 1 < obs.size() && std::fabs(cum - half) <= tol) *near_tie = true;
        if (!found && cum >= half) {
            m = obs[k].first;
            found = true;
        }
    }
    return m;
}

// Weight margins of the weighted median: a float32 evaluation of w_c = w_b cos(theta) / z^2
// carries a relative error (g_tau_w) and, through the normal, an absolute error in
// cos(theta) (g_tau_cos) that dominates at grazing angles.
double g_tau_w = 1e-5;
double g_tau_cos = 1e-5;

}  // namespace

extern "C" void or_colour_unsharp(const uint8_t* rgba, int W, int H, double* S) { unsharp(rgba, W, H, S); }

extern "C" double or_colour_blurriness(const uint8_t* rgba, int W, int H) { return blurriness(rgba, W, H); }

extern "C" double or_weighted_median(const double* c, const double* w, int n) {
    std::vector<std::pair<double, double>> obs;
    for (int j = 0; j < n; ++j) obs.emplace_back(c[j], w[j]);
    bool nt;
    return n > 0 ? weighted_median(obs, 0.0, &nt) : NAN;
}

extern "C" int or_fuse_colour(const uint8_t* rgba, const float* depths, const float* poses, int n,
                              const float* kf_depth, const float* kf_pose, double fx, double fy, double cx,
                              double cy, int W, int H, double disc_rel, double occl_rel, double* med, double* err,
                              uint8_t* out_rgba, int32_t* nobs, double* wsum, uint8_t* flag, double* wb_out) {
    const Intr K{fx, fy, cx, cy, W, H};
    const Pose Tk = pose_from(kf_pose);
    // steps 1 and 2, per frame
    std::vector<double> S((size_t)n * W * H * 3);
    std::vector<double> wb(n);
    for (int i = 0; i < n; ++i) {
        const uint8_t* img = rgba + (size_t)i * W * H * 4;
        unsharp(img, W, H, S.data() + (size_t)i * W * H * 3);
        wb[i] = 1.0 - blurriness(img, W, H);
        if (wb_out) wb_out[i] = wb[i];
    }
    std::vector<Pose> Tf(n);
    for (int i = 0; i < n; ++i) Tf[i] = pose_from(poses + 12 * i);
    // step 3, per keyframe pixel
#pragma omp parallel for schedule(dynamic, 4)
    for (long v = 0; v < H; ++v)
        for (long u = 0; u < W; ++u) {
            const long p = v * W + u;
            for (int c = 0; c < 3; ++c) med[p * 3 + c] = err[p * 3 + c] = 0.0;
            for (int c = 0; c < 4; ++c) out_rgba[p * 4 + c] = 0;
            nobs[p] = 0;
            wsum[p] = 0.0;
            flag[p] = 0;
            const double z = kf_depth[p];
            if (!(z > 0.0)) continue;
            if (u == 0 || v == 0 || u == W - 1 || v == H - 1) continue;
            const double zn[4] = {kf_depth[p - 1], kf_depth[p + 1], kf_depth[p - W], kf_depth[p + W]};
            if (!(zn[0] > 0.0 && zn[1] > 0.0 && zn[2] > 0.0 && zn[3] > 0.0)) continue;
            bool keep = true, marginal = false;
            for (int k = 0; k < 4; ++k) {
                const double gap = std::fabs(zn[k] - z) - disc_rel * z;
                if (std::fabs(gap) < g_tau_rel * z) marginal = true;
                if (gap > 0.0) keep = false;
            }
            if (marginal) flag[p] = 1;
            if (!keep) continue;
            // keyframe normal (camera coordinates of the keyframe), then world
            double Pl[3], Pr[3], Pu[3], Pd[3], P[3];
            backproject(K, u - 1, v, zn[0], Pl);
            backproject(K, u + 1, v, zn[1], Pr);
            backproject(K, u, v - 1, zn[2], Pu);
            backproject(K, u, v + 1, zn[3], Pd);
            backproject(K, u, v, z, P);
            const double a[3] = {Pr[0] - Pl[0], Pr[1] - Pl[1], Pr[2] - Pl[2]};
            const double b[3] = {Pd[0] - Pu[0], Pd[1] - Pu[1], Pd[2] - Pu[2]};
            const double nk[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
            const double nn = std::sqrt(nk[0] * nk[0] + nk[1] * nk[1] + nk[2] * nk[2]);
            if (!(nn > 0.0)) continue;
            double nw[3];
            for (int r = 0; r < 3; ++r) nw[r] = Tk.R[r][0] * nk[0] + Tk.R[r][1] * nk[1] + Tk.R[r][2] * nk[2];
            double pw[3];
            apply(Tk, P, pw);
            std::vector<std::pair<double, double>> obs[3];
            double e[3] = {0.0, 0.0, 0.0};
            double w_err = 0.0;  // bound on the summed weight error of all samples
            for (int i = 0; i < n; ++i) {
                if (!(wb[i] > 0.0)) continue;
                // p_i = g(T_i^-1, g(T*, pi^-1(x*, Z*(x*))))
                double pi[3];
                apply_inv(Tf[i], pw, pi);
                if (std::fabs(pi[2]) < g_tau_m) flag[p] = 1;
                if (!(pi[2] > 0.0)) continue;
                const double us = K.fx * pi[0] / pi[2] + K.cx, vs = K.fy * pi[1] / pi[2] + K.cy;
                // footprint bounds (decision + margin)
                const double mb = std::min(std::min(std::fabs(us), std::fabs(us - (W - 1))),
                                           std::min(std::fabs(vs), std::fabs(vs - (H - 1))));
                if (mb < g_tau_px) flag[p] = 1;
                if (!(us >= 0.0 && us <= W - 1 && vs >= 0.0 && vs <= H - 1)) continue;
                // occlusion test at the nearest pixel; a marginal rounding flags the pixel
                // when the neighbour across the tie decides differently
                const float* Zi = depths + (size_t)i * W * H;
                auto visible = [&](long xx, long yy, bool* thr_marg) {
                    if (xx < 0 || yy < 0 || xx >= W || yy >= H) return false;
                    const double zi = Zi[yy * W + xx];
                    if (!(zi > 0.0)) return false;
                    const double gap = std::fabs(zi - pi[2]) - occl_rel * pi[2];
                    if (std::fabs(gap) < g_tau_m + g_tau_rel * pi[2]) *thr_marg = true;
                    return gap <= 0.0;
                };
                double mu_, mv_;
                const long xr = round_half_up(us, &mu_), yr = round_half_up(vs, &mv_);
                bool thr = false;
                const bool vis = visible(xr, yr, &thr);
                if (thr) flag[p] = 1;
                if (mu_ < g_tau_px || mv_ < g_tau_px) {
                    const long ax = mu_ < g_tau_px ? (us + 0.5 - std::floor(us + 0.5) < 0.5 ? xr - 1 : xr + 1) : xr;
                    const long ay = mv_ < g_tau_px ? (vs + 0.5 - std::floor(vs + 0.5) < 0.5 ? yr - 1 : yr + 1) : yr;
                    bool t2 = false;
                    if (visible(ax, yr, &t2) != vis || visible(xr, ay, &t2) != vis || visible(ax, ay, &t2) != vis || t2)
                        flag[p] = 1;
                }
                if (!vis) continue;
                // w_c = w_b * w_z, w_z = cos(theta) / z_i^2 with the normal in frame i
                double ni[3];
                for (int r = 0; r < 3; ++r) ni[r] = Tf[i].R[0][r] * nw[0] + Tf[i].R[1][r] * nw[1] + Tf[i].R[2][r] * nw[2];
                const double cos_theta = std::fabs(ni[2]) / nn;
                const double wc = wb[i] * cos_theta / (pi[2] * pi[2]);
                if (!(wc > 0.0)) continue;
                // bilinear sample of the deblurred image
                const double* Si = S.data() + (size_t)i * W * H * 3;
                long x0 = (long)std::floor(us), y0 = (long)std::floor(vs);
                if (x0 > W - 2) x0 = W - 2;
                if (y0 > H - 2) y0 = H - 2;
                const double ax_ = us - x0, ay_ = vs - y0;
                for (int c = 0; c < 3; ++c) {
                    const double s00 = Si[(y0 * W + x0) * 3 + c], s01 = Si[(y0 * W + x0 + 1) * 3 + c];
                    const double s10 = Si[((y0 + 1) * W + x0) * 3 + c], s11 = Si[((y0 + 1) * W + x0 + 1) * 3 + c];
                    const double val = (1.0 - ay_) * ((1.0 - ax_) * s00 + ax_ * s01) + ay_ * ((1.0 - ax_) * s10 + ax_ * s11);
                    obs[c].emplace_back(val, wc);
                    const double lip = std::max(std::fabs(s01 - s00), std::fabs(s11 - s10)) +
                                       std::max(std::fabs(s10 - s00), std::fabs(s11 - s01));
                    e[c] = std::max(e[c], g_tau_px * lip);
                }
                wsum[p] += wc;
                w_err += g_tau_w * wc + wb[i] * g_tau_cos / (pi[2] * pi[2]);
            }
            nobs[p] = (int32_t)obs[0].size();
            if (obs[0].empty()) continue;
            for (int c = 0; c < 3; ++c) {
                bool nt = false;
                const double m = weighted_median(obs[c], w_err, &nt);
                if (nt) flag[p] = 1;
                med[p * 3 + c] = m;
                err[p * 3 + c] = e[c];
                out_rgba[p * 4 + c] = (uint8_t)std::floor(m + 0.5);
            }
            out_rgba[p * 4 + 3] = 255;
        }
    return 0;
}

// ============================================================================
// Marching Cubes iso-surface extraction (Section 3 "SDF volume")
// ============================================================================
//
// The paper extracts the zero level set of D with Marching Cubes.  The cube of
// voxel (x, y, z) has corners (x + i0, y + i1, z + i2), i the three bits of the
// corner number; it is meshed only if all 8 corner voxels exist and are observed
// (W > 0).  A corner is inside when D < 0.  Every cube edge whose corners differ
// carries one vertex, linearly interpolated to D = 0.
//
// Reading of the triangulation (the paper cites Marching Cubes without a case
// table; this is a rule, applied cube by cube):
//  * on each face, walking its four corners in cyclic order, the crossed edges are
//    joined by segments: two crossed edges form one segment; with four (inside
//    corners diagonal) each inside corner is cut off by the segment joining its two
//    edges, so inside corners never connect across a face;
//  * every crossed edge lies on two faces, so the segments close into loops;
//  * a loop is oriented so that its Newell normal, computed on the edge midpoints,
//    points along the sum over its edges of the edge direction from the inside
//    corner to the outside one: triangle normals point to D > 0 (free space);
//  * a loop is fanned from its smallest edge number: (e0, e_i, e_i+1); loops in
//    order of their smallest edge number.
// Edge numbering: axis a = e / 4 (x, y, z); r = e % 4 gives the corner bits of the
// two other axes (lower axis in bit 0).

namespace {

struct McEdge {
    int axis, lo, hi;
};

McEdge mc_edge(int e) {
    const int a = e / 4, r = e % 4;
    int b = -1, c = -1;
    for (int d = 0; d < 3; ++d)
        if (d != a) {
            if (b < 0) b = d;
            else c = d;
        }
    const int lo = ((r & 1) << b) | (((r >> 1) & 1) << c);
    return McEdge{a, lo, lo | (1 << a)};
}

int mc_edge_of(int c0, int c1) {
    for (int e = 0; e < 12; ++e) {
        const McEdge E = mc_edge(e);
        if ((E.lo == c0 && E.hi == c1) || (E.lo == c1 && E.hi == c0)) return e;
    }
    return -1;
}

// Triangles (edge triples) of one cube given its inside-corner bit mask.
std::vector<std::array<int, 3>> mc_cube_triangles(int inside) {
    auto in = [&](int corner) { return (inside >> corner) & 1; };
    // partner[e][0 / 1]: the crossed edges e is joined to on its two faces
    int partner[12][2];
    int np[12] = {0};
    for (int f = 0; f < 6; ++f) {
        const int a = f / 2, side = f % 2;
        int b = -1, c = -1;
        for (int d = 0; d < 3; ++d)
            if (d != a) {
                if (b < 0) b = d;
                else c = d;
            }
        const int cyc[4] = {(side << a), (side << a) | (1 << b), (side << a) | (1 << b) | (1 << c),
                            (side << a) | (1 << c)};
        int cut[4];  // cut[k]: edge between cyc[k] and cyc[k+1] if crossed, else -1
        int ncut = 0;
        for (int k = 0; k < 4; ++k) {
            const int c0 = cyc[k], c1 = cyc[(k + 1) % 4];
            cut[k] = in(c0) != in(c1) ? mc_edge_of(c0, c1) : -1;
            ncut += cut[k] >= 0;
        }
        auto join = [&](int e0, int e1) {
            partner[e0][np[e0]++] = e1;
            partner[e1][np[e1]++] = e0;
        };
        if (ncut == 2) {
            int first = -1;
            for (int k = 0; k < 4; ++k)
                if (cut[k] >= 0) {
                    if (first < 0) first = cut[k];
                    else join(first, cut[k]);
                }
        } else if (ncut == 4) {
            for (int k = 0; k < 4; ++k)
                if (in(cyc[k])) join(cut[(k + 3) % 4], cut[k]);  // the two edges at inside corner k
        }
    }
    // loops
    std::vector<std::array<int, 3>> tris;
    bool used[12] = {false};
    for (int start = 0; start < 12; ++start) {
        const McEdge S = mc_edge(start);
        if (used[start] || in(S.lo) == in(S.hi)) continue;
        std::vector<int> loop{start};
        used[start] = true;
        int prev = start, cur = partner[start][0];
        while (cur != start) {
            loop.push_back(cur);
            used[cur] = true;
            const int next = partner[cur][0] == prev ? partner[cur][1] : partner[cur][0];
            prev = cur;
            cur = next;
        }
        // orientation: Newell normal of the midpoints against the inside -> outside directions
        double N[3] = {0, 0, 0}, g[3] = {0, 0, 0};
        const size_t m = loop.size();
        std::vector<std::array<double, 3>> q(m);
        for (size_t i = 0; i < m; ++i) {
            const McEdge E = mc_edge(loop[i]);
            for (int d = 0; d < 3; ++d) q[i][d] = ((E.lo >> d) & 1) + (d == E.axis ? 0.5 : 0.0);
            g[E.axis] += in(E.lo) ? 1.0 : -1.0;
        }
        for (size_t i = 0; i < m; ++i) {
            const auto& p0 = q[i];
            const auto& p1 = q[(i + 1) % m];
            N[0] += (p0[1] - p1[1]) * (p0[2] + p1[2]);
            N[1] += (p0[2] - p1[2]) * (p0[0] + p1[0]);
            N[2] += (p0[0] - p1[0]) * (p0[1] + p1[1]);
        }
        if (N[0] * g[0] + N[1] * g[1] + N[2] * g[2] < 0.0) std::reverse(loop.begin(), loop.end());
        // loop starts at its smallest edge number, which is `start` (loops are found in edge order)
        const auto it = std::find(loop.begin(), loop.end(), start);
        std::rotate(loop.begin(), it, loop.end());
        for (size_t i = 1; i + 1 < m; ++i) tris.push_back({loop[0], loop[i], loop[i + 1]});
    }
    return tris;
}

}  // namespace

// Marching Cubes over blocks given as arrays (coords [n][3] block coordinates,
// D and W [n][512], voxel index x + 8 y + 64 z).  Writes up to cap triangles:
// tri [cap][3][3] vertex positions in metres (voxel i at i * voxel_size) and cube
// [cap][4] = (x, y, z of the cube's first corner voxel, triangle number within the
// cube).  Returns the number of triangles (which may exceed cap).
extern "C" long or_marching_cubes(const int32_t* coords, const float* D, const float* W, long n,
                                  double voxel_size, double* tri, int32_t* cube, long cap) {
    std::unordered_map<int64_t, long> index;
    for (long b = 0; b < n; ++b) index[pack(coords[3 * b], coords[3 * b + 1], coords[3 * b + 2])] = b;
    // the triangulation of every inside mask (the rule above, per cube)
    static std::vector<std::array<int, 3>> cases[256];
    static bool built = false;
    if (!built) {
        for (int m = 0; m < 256; ++m) cases[m] = mc_cube_triangles(m);
        built = true;
    }
    long count = 0;
    for (long b = 0; b < n; ++b) {
        const long bx = coords[3 * b], by = coords[3 * b + 1], bz = coords[3 * b + 2];
        for (int lz = 0; lz < BS; ++lz)
            for (int ly = 0; ly < BS; ++ly)
                for (int lx = 0; lx < BS; ++lx) {
                    double cd[8];
                    long cv[8][3];
                    bool ok = true;
                    for (int i = 0; i < 8 && ok; ++i) {
                        const long vx = bx * BS + lx + (i & 1), vy = by * BS + ly + ((i >> 1) & 1),
                                   vz = bz * BS + lz + ((i >> 2) & 1);
                        const auto f = index.find(pack(floor_div(vx, BS), floor_div(vy, BS), floor_div(vz, BS)));
                        if (f == index.end()) {
                            ok = false;
                            break;
                        }
                        const long vi = (vx - floor_div(vx, BS) * BS) + BS * (vy - floor_div(vy, BS) * BS) +
                                        BS * BS * (vz - floor_div(vz, BS) * BS);
                        if (!(W[f->second * NV + vi] > 0.0f)) ok = false;
                        cd[i] = D[f->second * NV + vi];
                        cv[i][0] = vx;
                        cv[i][1] = vy;
                        cv[i][2] = vz;
                    }
                    if (!ok) continue;
                    int inside = 0;
                    for (int i = 0; i < 8; ++i) inside |= (cd[i] < 0.0 ? 1 : 0) << i;
                    const auto& tl = cases[inside];
                    for (size_t k = 0; k < tl.size(); ++k) {
                        if (count < cap) {
                            for (int j = 0; j < 3; ++j) {
                                const McEdge E = mc_edge(tl[k][j]);
                                const double t = cd[E.lo] / (cd[E.lo] - cd[E.hi]);
                                for (int d = 0; d < 3; ++d)
                                    tri[count * 9 + 3 * j + d] =
                                        voxel_size * ((double)cv[E.lo][d] + (d == E.axis ? t : 0.0));
                            }
                            cube[count * 4] = (int32_t)(bx * BS + lx);
                            cube[count * 4 + 1] = (int32_t)(by * BS + ly);
                            cube[count * 4 + 2] = (int32_t)(bz * BS + lz);
                            cube[count * 4 + 3] = (int32_t)k;
                        }
                        ++count;
                    }
                }
    }
    return count;
}

// The triangulation rule alone: edge triples of inside mask m (for the pins).
extern "C" int or_mc_case(int m, int32_t* edges) {
    const auto t = mc_cube_triangles(m & 255);
    for (size_t k = 0; k < t.size(); ++k)
        for (int j = 0; j < 3; ++j) edges[3 * k + j] = t[k][j];
    return (int)t.size();
}

// ============================================================================
// Keyframe strategies (Section 4.2): KF_CONST, KF_DIST, KF_OVRLP
// ============================================================================
//
// Frames are taken in order; frame 0 starts the first group and the frame that
// triggers a new keyframe starts the next group (its pose is the keyframe pose).
//  * KF_CONST(kappa): a new keyframe every kappa frames.
//  * KF_DIST(thr_t, thr_r): a new keyframe when the relative pose between the current
//    frame and the current keyframe has translation norm > thr_t (metres) or rotation
//    angle > thr_r (radians).  Reading: translation norm |t_f - t_k| (of T_k^-1 T_f),
//    angle acos((trace(R_k^T R_f) - 1) / 2).
//  * KF_OVRLP(thr): a new keyframe when the overlap ratio drops below thr.  Reading of
//    "pixels visible in both": the share of the frame's valid pixels (Z > 0) whose
//    point, warped into the keyframe, is in front of it (z > 0) and has its nearest
//    pixel (halves up) inside the keyframe image.
// For the overlap ratio the oracle also counts the marginal pixels (a rounding or the
// camera plane within the margins), so that a float32 evaluation can be compared.

namespace {

void overlap_count(const float* depth, const Pose& Tf, const Pose& Tk, const Intr& K, long* valid, long* inside,
                   long* marginal) {
    long nv = 0, ni = 0, nm = 0;
    for (long v = 0; v < K.H; ++v)
        for (long u = 0; u < K.W; ++u) {
            const double z = depth[v * K.W + u];
            if (!(z > 0.0)) continue;
            ++nv;
            double P[3], pw[3], pk[3];
            backproject(K, (double)u, (double)v, z, P);
            apply(Tf, P, pw);
            apply_inv(Tk, pw, pk);
            bool marg = std::fabs(pk[2]) < g_tau_m;
            if (!(pk[2] > 0.0)) {
                nm += marg;
                continue;
            }
            double mu_, mv_;
            const double uf = K.fx * pk[0] / pk[2] + K.cx, vf = K.fy * pk[1] / pk[2] + K.cy;
            const long xs = round_half_up(uf, &mu_), ys = round_half_up(vf, &mv_);
            // a marginal rounding matters only where it can move the pixel across the border
            if ((mu_ < g_tau_px && (xs == 0 || xs == K.W || xs == -1 || xs == K.W - 1)) ||
                (mv_ < g_tau_px && (ys == 0 || ys == K.H || ys == -1 || ys == K.H - 1)))
                marg = true;
            nm += marg;
            if (xs >= 0 && xs < K.W && ys >= 0 && ys < K.H) ++ni;
        }
    *valid = nv;
    *inside = ni;
    *marginal = nm;
}

double rotation_angle(const Pose& A, const Pose& B) {
    double tr = 0.0;  // trace(R_A^T R_B)
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) tr += A.R[r][c] * B.R[r][c];
    const double x = std::max(-1.0, std::min(1.0, (tr - 1.0) / 2.0));
    return std::acos(x);
}

}  // namespace

extern "C" void or_overlap(const float* depth, const float* frame_pose, const float* kf_pose, double fx, double fy,
                           double cx, double cy, int W, int H, long* counts /*valid, inside, marginal*/) {
    const Intr K{fx, fy, cx, cy, W, H};
    overlap_count(depth, pose_from(frame_pose), pose_from(kf_pose), K, &counts[0], &counts[1], &counts[2]);
}

// strategy 0 KF_CONST (p0 = kappa), 1 KF_DIST (p0 = thr_t, p1 = thr_r), 2 KF_OVRLP (p0 = thr).
// frame_kf[f] = group of frame f; flag[f] = 1 where frame f's decision is within the
// margins (KF_OVRLP: the marginal pixels could move the ratio across thr; KF_DIST: a
// distance within 1e-6 relative of its threshold).  Returns the number of keyframes.
extern "C" int or_segment(int strategy, double p0, double p1, const float* depths, const float* poses, int n,
                          double fx, double fy, double cx, double cy, int W, int H, int32_t* frame_kf, uint8_t* flag) {
    const Intr K{fx, fy, cx, cy, W, H};
    if (n <= 0) return 0;
    int groups = 1, kf = 0;
    frame_kf[0] = 0;
    flag[0] = 0;
    for (int f = 1; f < n; ++f) {
        bool fresh = false;
        flag[f] = 0;
        const Pose Tf = pose_from(poses + 12 * f), Tk = pose_from(poses + 12 * kf);
        if (strategy == 0) {
            fresh = (f % (int)p0) == 0;
        } else if (strategy == 1) {
            double dt = 0.0;
            for (int r = 0; r < 3; ++r) dt += (Tf.t[r] - Tk.t[r]) * (Tf.t[r] - Tk.t[r]);
            dt = std::sqrt(dt);
            const double dr = rotation_angle(Tk, Tf);
            fresh = dt > p0 || dr > p1;
            if (std::fabs(dt - p0) <= 1e-6 * p0 || std::fabs(dr - p1) <= 1e-6 * p1) flag[f] = 1;
        } else {
            long nv, ni, nm;
            overlap_count(depths + (size_t)f * W * H, Tf, Tk, K, &nv, &ni, &nm);
            const double ratio = nv > 0 ? (double)ni / (double)nv : 0.0;
            fresh = ratio < p0;
            if (nv > 0 && std::fabs(ratio - p0) * (double)nv <= (double)nm) flag[f] = 1;
        }
        if (fresh) {
            kf = f;
            ++groups;
        }
        frame_kf[f] = groups - 1;
    }
    return groups;
}

// ============================================================================
// Streaming sphere (Section 3 "SDF volume"; Section 4.3 streaming order)
// ============================================================================
//
// Only voxel blocks within a sphere of constant radius around the camera stay in
// GPU memory.  Reading: a block is inside when its centre, the centre of its 8^3
// voxels ((8 b + 3.5) * voxel_size per axis), lies within radius of the camera
// position (distance <= radius).  out[b] = 1 for blocks outside; marg[b] = 1 where
// the distance is within 1e-5 m of the radius (a float32 evaluation of the squared
// distance of a block a few metres away errs by about 1e-6 m).  Streaming itself changes no voxel value; the tests check that
// invariance against the unstreamed volume.
extern "C" long or_sphere_outside(const int32_t* coords, long n, double voxel_size, const double* centre,
                                  double radius, uint8_t* out, uint8_t* marg) {
    long count = 0;
    for (long b = 0; b < n; ++b) {
        double d2 = 0.0;
        for (int r = 0; r < 3; ++r) {
            const double c = (8.0 * coords[3 * b + r] + 3.5) * voxel_size - centre[r];
            d2 += c * c;
        }
        const double d = std::sqrt(d2);
        out[b] = d > radius;
        marg[b] = std::fabs(d - radius) <= 1e-5;
        count += out[b];
    }
    return count;
}
