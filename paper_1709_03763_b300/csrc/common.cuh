// Device-side building blocks shared by the surfcorr kernels: volume layout,
// spatial hash, the per-voxel projective sample and the running-average update.
//
// Layout in HBM (all arrays indexed by pool slot, one slot per 8^3 block):
//   D      float [max_blocks][512]      signed distance, metres
//   W      float [max_blocks][512]      integration weight (integer-valued)
//   C8     uint32 [max_blocks][512]     colour RGBA8 (r | g<<8 | b<<16), or
//   Cf     float [max_blocks][3][512]   colour RGB_F32 (parity mode)
//   coord  int4 [max_blocks]            block coordinate of each slot
//   flags  uint32 [max_blocks]          bit 0: fresh (zero-initialise on first update)
// Voxel index inside a block: x + 8 y + 64 z, so a warp's 32 lanes x float4
// cover 128 consecutive voxels (four 512-byte coalesced transactions per block
// and field).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "surfcorr.h"

namespace sc {

constexpr int BLK = 8;
constexpr int NVOX = 512;
constexpr unsigned long long KEY_EMPTY = ~0ull;
constexpr int32_t SLOT_PENDING = -1;
constexpr int32_t SLOT_FAILED = -2;
constexpr uint32_t FLAG_FRESH = 1u;
constexpr int COORD_BIAS = 1 << 20;  // block coordinates in [-2^20, 2^20 - 1]
constexpr int DEFAULT_RETRY = 1 << 20;

struct __align__(16) HashEntry {
    unsigned long long key;
    int32_t slot;
    uint32_t pad;
};

__host__ __device__ inline unsigned long long pack_key(int x, int y, int z) {
    return (unsigned long long)(uint32_t)(x + COORD_BIAS) |
           ((unsigned long long)(uint32_t)(y + COORD_BIAS) << 21) |
           ((unsigned long long)(uint32_t)(z + COORD_BIAS) << 42);
}

__host__ __device__ inline bool coord_ok(int x, int y, int z) {
    return x >= -COORD_BIAS && x < COORD_BIAS && y >= -COORD_BIAS && y < COORD_BIAS && z >= -COORD_BIAS &&
           z < COORD_BIAS;
}

__device__ inline int3 unpack_key(unsigned long long k) {
    const unsigned long long M = (1ull << 21) - 1;
    return make_int3((int)(k & M) - COORD_BIAS, (int)((k >> 21) & M) - COORD_BIAS,
                     (int)((k >> 42) & M) - COORD_BIAS);
}

// 64-bit finaliser (xor-shift-multiply) -> bucket index.
__host__ __device__ inline uint32_t hash_bucket(unsigned long long k, uint32_t mask) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (uint32_t)k & mask;
}

// Everything a kernel needs to address the volume, passed by value.
struct DevVolume {
    HashEntry* table;
    uint32_t bucket_mask;
    uint32_t bucket_size;
    uint32_t max_probe;
    uint32_t max_blocks;
    float* D;
    float* W;
    uint32_t* C8;
    float* Cf;
    int4* coord;
    uint32_t* flags;
    uint32_t* stamp;
    uint32_t* pool_count;
    int32_t* status;
    int32_t retry_limit;
    int32_t colour_f32;
    unsigned long long* prof;  // device work counters when profiling, else null
};

__device__ inline void set_status(int32_t* status, int32_t code) { atomicCAS(status, 0, code); }

// Per keyframe-operation camera constants, built on the host from the float
// pose in double precision and rounded once:
//   q = (i - ti) - tf   voxel index relative to the camera position (voxel units)
//   p_c = M q           camera coordinates (metres), M = voxel_size * R^T
//   Pr = diag(fx, fy, 1) M   the projection rows: pi(p_c) = (Pr_0 q, Pr_1 q) / (Pr_2 q) + (cx, cy)
//   segment endpoint in relative voxel units: Ms * pi^-1(x, z) + tf, Ms = R / voxel_size
struct KfCam {
    float2 Pxy[3];   // the first two rows of Pr by columns, as f32x2 pairs: (Pr[q], Pr[3 + q])
    float2 cxyh;     // (cx + 1/2, cy + 1/2)
    float Pz[3];     // the third row of Pr
    float Pr[9];
    float Ms[9];
    float tf[3];
    int ti[3];
    float tiF[3];    // ti as floats (exact: |ti| < 2^21)
    float fx, fy, cx, cy;
    float cxh, cyh;  // cx + 1/2, cy + 1/2: nearest pixel = floor(u + 1/2)
    float ifx, ify;  // 1 / fx, 1 / fy
    int W, H;
    float mu;
    const float* depth;
    const uint32_t* rgba;  // RGBA8 as one 32-bit word per pixel
    const uint2* tex;      // (depth bits, RGBA8) per pixel, where a packed copy exists
};

// 1/x to about 1 ulp (the MUFU reciprocal); denormal x flushes to zero (1/x = inf).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// floor(x) for 0 <= x < 2^23 without a conversion instruction: adding 2^23 rounded
// down leaves floor(x) in the mantissa.  Any other x (negative, >= 2^23, infinite or
// NaN) gives a value outside [0, 2^23): x < 0 sums to a float below 2^23 (negative
// integer result), x >= 2^23 to one of at least 2^24, and inf / NaN keep exponent bits
// that are either far above 2^23 or negative, so one unsigned comparison against an
// image size in [1, 2^23) tests "0 <= x < size" and takes the floor together.
__device__ __forceinline__ int floor_small(float x) { return __float_as_int(__fadd_rd(x, 8388608.f)) - 0x4b000000; }

// Projection of the 4 voxels (ix0 + j, iy, iz), j = 0..3, that one thread owns,
// given as floats (exact integers).
// Every operation is an explicit round-to-nearest intrinsic (or the one approximate
// reciprocal), in one fixed order, so that integration, de-integration, the batched
// net-delta kernel and the adjoint reach bit-identical decisions and distances for
// the same keyframe and pose.  Voxel j + 1 adds the x column of Pr to voxel j's
// projective coordinates.  ok[j]: in front of the camera and the nearest pixel
// (halves rounded up) inside the image; pix[j] is only meaningful when ok[j].
// Computing all four first lets the caller issue the four depth gathers back to back.
struct Proj4 {
    float pz[4];
    int pix[4];
    bool ok[4];
};

template <typename Cam>
__device__ __forceinline__ void project4(const Cam& k, float ix0, float iy, float iz, Proj4& p) {
    // (i - ti) is exact in float, so this is the relative index (i - ti) - tf rounded once
    const float qx = __fsub_rn(__fsub_rn(ix0, k.tiF[0]), k.tf[0]);
    const float qy = __fsub_rn(__fsub_rn(iy, k.tiF[1]), k.tf[1]);
    const float qz = __fsub_rn(__fsub_rn(iz, k.tiF[2]), k.tf[2]);
    // the image-plane rows x and y as one f32x2 pair (each component the same
    // round-to-nearest operation as its scalar form), the depth row alone
    float pz = __fmaf_rn(k.Pz[2], qz, __fmaf_rn(k.Pz[1], qy, __fmul_rn(k.Pz[0], qx)));
    float2 pxy = __ffma2_rn(k.Pxy[2], make_float2(qz, qz),
                            __ffma2_rn(k.Pxy[1], make_float2(qy, qy), __fmul2_rn(k.Pxy[0], make_float2(qx, qx))));
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (j > 0) {
            pz = __fadd_rn(pz, k.Pz[0]);
            pxy = __fadd2_rn(pxy, k.Pxy[0]);
        }
        const float rz = rcp_approx(pz);
        // nearest pixel and the range test in one (floor_small on both coordinates):
        // (unsigned) floor(u + 1/2) < W holds exactly when 0 <= u + 1/2 < W (NaN / inf fail it)
        const float2 f = __fadd2_rd(__ffma2_rn(pxy, make_float2(rz, rz), k.cxyh), make_float2(8388608.f, 8388608.f));
        const int iu = __float_as_int(f.x) - 0x4b000000, iv = __float_as_int(f.y) - 0x4b000000;
        p.pz[j] = pz;
        p.ok[j] = pz > 0.f && (unsigned)iu < (unsigned)k.W && (unsigned)iv < (unsigned)k.H;
        p.pix[j] = p.ok[j] ? iv * k.W + iu : 0;
    }
}

// The update decision for one projected voxel given the keyframe depth Z at its
// pixel: updated iff Z > 0 and eta = Z - z_c >= -mu; then d = min(eta, mu).
template <typename Cam>
__device__ __forceinline__ bool decide(const Cam& k, bool ok, float Z, float pz, float& d, float& eta) {
    if (!ok || !(Z > 0.f)) return false;
    eta = __fsub_rn(Z, pz);
    if (eta < -k.mu) return false;
    d = fminf(eta, k.mu);
    return true;
}

__device__ __forceinline__ uint32_t u8_sat(float x) {
    // round half to even, saturate to [0, 255] (NaN -> 0): one conversion instruction
    uint32_t r;
    asm("cvt.rni.sat.u8.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r & 0xffu;
}

// Running weighted average with w = 1 (sign +1) or its inverse, Eq. 2 (sign -1).
// W reaching 0 resets D to 0.
__device__ __forceinline__ void update_dw(float& D, float& W, float d, int sign) {
    if (sign > 0) {
        const float Wn = __fadd_rn(W, 1.f);
        D = __fdiv_rn(__fmaf_rn(D, W, d), Wn);
        W = Wn;
    } else {
        const float Wn = __fsub_rn(W, 1.f);
        D = (Wn == 0.f) ? 0.f : __fdiv_rn(__fmaf_rn(D, W, -d), Wn);
        W = Wn;
    }
}

// Colour channel in float (RGB_F32 mode): same rule as D.  W is the weight
// before the update.
__device__ __forceinline__ float update_cf(float C, float W, float c, int sign) {
    if (sign > 0) return __fdiv_rn(__fmaf_rn(C, W, c), __fadd_rn(W, 1.f));
    const float Wn = __fsub_rn(W, 1.f);
    return (Wn == 0.f) ? 0.f : __fdiv_rn(__fmaf_rn(C, W, -c), Wn);
}

// RGBA8 word: each channel averaged in float then rounded half-to-even.
__device__ __forceinline__ uint32_t update_c8(uint32_t C, float W, uint32_t c, int sign) {
    const float Wn = sign > 0 ? __fadd_rn(W, 1.f) : __fsub_rn(W, 1.f);
    if (Wn == 0.f) return 0u;
    uint32_t out = 0;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float a = (float)((C >> (8 * ch)) & 255u);
        const float b = (float)((c >> (8 * ch)) & 255u);
        const float v = __fdiv_rn(__fmaf_rn(a, W, sign > 0 ? b : -b), Wn);
        out |= u8_sat(v) << (8 * ch);
    }
    return out;
}

// Voxel coordinates of the 4 consecutive voxels lane `lane` owns in group g
// (0..3) of a block: linear index v0 = 4 lane + 128 g.
__device__ __forceinline__ void lane_voxels(int lane, int g, int& lx0, int& ly, int& lz) {
    const int v0 = 4 * lane + 128 * g;
    lx0 = v0 & 7;
    ly = (v0 >> 3) & 7;
    lz = v0 >> 6;
}

// ---------------------------------------------------------------- hashing ----

// 16-byte load that bypasses stale L1 copies (key and slot of a hash entry).  The
// words are read individually atomically; a key that matches always comes with
// either SLOT_PENDING, SLOT_FAILED or its final slot (slots are written once).
__device__ __forceinline__ uint4 ld_volatile_u4(const void* p) {
    uint4 r;
    asm volatile("ld.volatile.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

// Lock-free insert-or-find of `key`.  Bucketed open addressing: the key's home
// bucket, then the following buckets (wrapping) up to max_probe buckets.  An
// empty entry is claimed with a 64-bit CAS on its key; the slot is published
// later (SLOT_PENDING until then).  Each entry is read with one 16-byte load, so
// for a key that exists the published slot comes back in the same round trip
// (*slot_seen, else -1).  Returns the entry index, or -1 with the status set
// (SC_ERR_HASH_FULL).  *won is set when this call created the entry.
__device__ inline int hash_claim(const DevVolume& V, unsigned long long key, bool* won, int32_t* slot_seen) {
    const uint32_t b = hash_bucket(key, V.bucket_mask);
    *won = false;
    *slot_seen = -1;
    for (uint32_t probe = 0; probe < V.max_probe; ++probe) {
        const uint32_t base = ((b + probe) & V.bucket_mask) * V.bucket_size;
        for (uint32_t e = 0; e < V.bucket_size; ++e) {
            HashEntry* ep = &V.table[base + e];
            const uint4 w = ld_volatile_u4(ep);
            unsigned long long k = (unsigned long long)w.x | ((unsigned long long)w.y << 32);
            if (k == key) {
                *slot_seen = (int32_t)w.z >= 0 ? (int32_t)w.z : -1;
                return (int)(base + e);
            }
            if (k == KEY_EMPTY) {
                k = atomicCAS(&ep->key, KEY_EMPTY, key);
                if (k == KEY_EMPTY) {
                    *won = true;
                    return (int)(base + e);
                }
                if (k == key) return (int)(base + e);
            }
        }
    }
    set_status(V.status, SC_ERR_HASH_FULL);
    return -1;
}

// Find without inserting: entry index or -1.
__device__ inline int hash_find(const DevVolume& V, unsigned long long key) {
    const uint32_t b = hash_bucket(key, V.bucket_mask);
    for (uint32_t probe = 0; probe < V.max_probe; ++probe) {
        const uint32_t base = ((b + probe) & V.bucket_mask) * V.bucket_size;
        for (uint32_t e = 0; e < V.bucket_size; ++e) {
            const unsigned long long k = V.table[base + e].key;
            if (k == key) return (int)(base + e);
            if (k == KEY_EMPTY) return -1;
        }
    }
    return -1;
}

// Slot of a claimed entry, waiting (bounded) for its publication by the CTA that
// created it.  Returns the slot or -1 (status SC_ERR_RETRY_LIMIT on give-up; a
// failed allocation returns -1 silently, its creator set the status).
__device__ inline int32_t entry_slot(const DevVolume& V, int entry) {
    volatile int32_t* sp = &V.table[entry].slot;
    for (int32_t it = 0; it < V.retry_limit; ++it) {
        const int32_t s = *sp;
        if (s >= 0) return s;
        if (s == SLOT_FAILED) return -1;
        __nanosleep(64);
    }
    set_status(V.status, SC_ERR_RETRY_LIMIT);
    return -1;
}

// Slot of voxel-block `key` for lookups: pool slot or -1.
__device__ inline int32_t find_slot(const DevVolume& V, unsigned long long key) {
    const int e = hash_find(V, key);
    if (e < 0) return -1;
    const int32_t s = V.table[e].slot;
    return s >= 0 ? s : -1;
}

}  // namespace sc
