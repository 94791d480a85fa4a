// Block allocation (Section 3 "SDF volume": blocks are allocated before the
// voxels are updated), shared by the per-keyframe path and the batched path.
//
// A(k, T): every 8^3 block whose closed box meets the band segment
// {pi^-1(x, z) : z in [Z(x) - mu, Z(x) + mu]} of a valid pixel x, in world
// coordinates.  Computed per 32x32 pixel tile by one CTA:
//   A  enumerate each pixel's blocks (a walk across block faces) into shared memory,
//      which removes the many duplicates neighbouring pixels produce: a block inside
//      the tile's window (16^3 blocks around the surface at a reference pixel) sets its
//      byte of a direct-indexed byte map with a plain store; any other block goes into a
//      set of 32-bit camera-relative keys;
//   B  claim every unique key in the global hash table (64-bit CAS); each warp's new
//      entries get consecutive pool slots from one atomic add and are published at once;
//   C  read each key's slot and let the Sink decide whether this call lists it
//      (first time for this keyframe) and, for batches, whether it joins the
//      batch's union of touched blocks; appends go through one atomic per warp;
//      B and C run warp by warp, with no barrier between them;
//   D  only if the set or the compacted key list overflowed: the blocks they miss,
//      one at a time.
#pragma once

#include <climits>

#include "common.cuh"

namespace sc {

#ifndef SC_ALLOC_CTAS_PER_SM
#define SC_ALLOC_CTAS_PER_SM 8  // resident allocation CTAs per SM (caps registers at 32)
#endif
// Pixel tiles of 32 x TY pixels, one CTA of 256 threads, TY / 8 pixels per thread (one
// column, rows r, r + 8, ...).  Batches and stream-in probes take 32 x 32 tiles (fewer
// tiles, so less per-tile work: 13 % faster than 32 x 16 over 60 images); the plain path
// allocates one keyframe per launch and takes 32 x 16, which doubles its CTAs.
constexpr int ALLOC_TX = 32;
constexpr int ALLOC_TY = 32;        // batched allocation, stream-in probe
constexpr int ALLOC_TY_PLAIN = 16;  // one keyframe per launch
constexpr int ALLOC_THREADS = 256;
template <int TY>
__host__ __device__ constexpr int alloc_ppt() { return ALLOC_TX * TY / ALLOC_THREADS; }
constexpr int SET_BITS = 10;
constexpr int SET_SIZE = 1 << SET_BITS;  // unique blocks of a tile before overflow handling
constexpr int MAX_BLOCK_WALK = 48;   // block-face crossings of one band segment
constexpr float MAX_DEPTH = 1.0e4f;  // metres; larger depth values are treated as invalid

// Blocks met by pixel (u, v)'s band segment; calls f(bx, by, bz) once per block.
// Geometry in voxel units relative to the camera's integer voxel position ti.
// The segment is walked from its start block to its end block across block
// faces (3-D DDA, exactly sum |b1 - b0| steps).  That is the set of closed boxes
// the segment meets, except where the segment passes within float error of a
// block edge, corner or face it only touches: such decisions are marginal.
template <typename F>
__device__ inline void for_each_segment_block(const KfCam& k, int u, int v, float Z, F&& f) {
    const float xn = __fmul_rn(__fsub_rn((float)u, k.cx), k.ifx);
    const float yn = __fmul_rn(__fsub_rn((float)v, k.cy), k.ify);
    const float z0 = __fsub_rn(Z, k.mu), z1 = __fadd_rn(Z, k.mu);

    float q0[3], q1[3];
    int b[3], rem[3], step[3];
    float tmax[3], tdel[3];
    int n = 0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float ray = __fmaf_rn(k.Ms[3 * r], xn, __fmaf_rn(k.Ms[3 * r + 1], yn, k.Ms[3 * r + 2]));
        q0[r] = __fmaf_rn(z0, ray, k.tf[r]);
        q1[r] = __fmaf_rn(z1, ray, k.tf[r]);
        b[r] = (__float2int_rd(q0[r]) + k.ti[r]) >> 3;
        const int e = (__float2int_rd(q1[r]) + k.ti[r]) >> 3;
        rem[r] = abs(e - b[r]);
        n += rem[r];
        const float d = __fsub_rn(q1[r], q0[r]);
        step[r] = d > 0.f ? 1 : -1;
        tmax[r] = __int_as_float(0x7f800000);  // +inf: no crossing on this axis
        tdel[r] = tmax[r];
        if (rem[r] > 0) {
            // approximate reciprocal (1 ulp): the crossing times only order the axes of
            // the walk; a different order within float error of a tie is a marginal
            // decision (a segment passing within float error of a block edge)
            const float inv = rcp_approx(d);
            const float bound = (float)(8 * (b[r] + (step[r] > 0 ? 1 : 0)) - k.ti[r]);
            tmax[r] = __fmul_rn(__fsub_rn(bound, q0[r]), inv);
            tdel[r] = __fmul_rn(8.f, fabsf(inv));
        }
    }
    // a band segment spans a handful of blocks; a longer walk comes from a
    // degenerate input and is skipped rather than followed
    if (n > MAX_BLOCK_WALK) return;
    // scalar walk state (no dynamically indexed arrays: everything stays in registers)
    int bx = b[0], by = b[1], bz = b[2];
    int rx = rem[0], ry = rem[1], rz = rem[2];
    float tx = tmax[0], ty = tmax[1], tz = tmax[2];
    f(bx, by, bz);
    for (int i = 0; i < n; ++i) {
        // axis with a crossing left and the nearest next face (x before y before z on ties)
        const bool px = rx > 0 && (ry == 0 || tx <= ty) && (rz == 0 || tx <= tz);
        const bool py = !px && ry > 0 && (rz == 0 || ty <= tz);
        if (px) {
            bx += step[0];
            --rx;
            tx = __fadd_rn(tx, tdel[0]);
        } else if (py) {
            by += step[1];
            --ry;
            ty = __fadd_rn(ty, tdel[1]);
        } else {
            bz += step[2];
            --rz;
            tz = __fadd_rn(tz, tdel[2]);
        }
        f(bx, by, bz);
    }
}

// The CTA's shared set holds 32-bit keys: each block coordinate relative to the
// camera's block, 10 bits per axis (+-512 blocks, 41 m at 1 cm voxels, beyond any
// sensor range).  A block outside that range (a depth of kilometres) is counted as an
// overflow and claimed by phase D with its full key.
constexpr uint32_t KEY32_EMPTY = 0xFFFFFFFFu;  // never a key: keys use 30 bits

__device__ __forceinline__ bool key32(int bx, int by, int bz, const int3& ref, uint32_t* k) {
    const uint32_t dx = (uint32_t)(bx - ref.x + 512), dy = (uint32_t)(by - ref.y + 512),
                   dz = (uint32_t)(bz - ref.z + 512);
    *k = dx | (dy << 10) | (dz << 20);
    return (dx | dy | dz) < 1024u;
}

__device__ __forceinline__ unsigned long long key64_of(uint32_t k, const int3& ref) {
    return pack_key((int)(k & 1023u) - 512 + ref.x, (int)((k >> 10) & 1023u) - 512 + ref.y,
                    (int)(k >> 20) - 512 + ref.z);
}

// Slot of a key in the CTA's shared set (Fibonacci hashing: one multiply).
__device__ __forceinline__ uint32_t set_hash(uint32_t key) { return (key * 0x9E3779B1u) >> (32 - SET_BITS); }

// Insert into the CTA's shared set.  Most inserts find their key already there:
// read before CAS so that those do not serialise on the shared atomic unit.
__device__ inline bool set_insert(uint32_t* set, uint32_t key) {
    uint32_t h = set_hash(key);
    for (int i = 0; i < SET_SIZE; ++i) {
        uint32_t k = ((volatile uint32_t*)set)[h];
        if (k == key) return true;
        if (k == KEY32_EMPTY) {
            k = atomicCAS(&set[h], KEY32_EMPTY, key);
            if (k == KEY32_EMPTY || k == key) return true;
        }
        h = (h + 1) & (SET_SIZE - 1);
    }
    return false;
}

__device__ inline bool set_contains(const uint32_t* set, uint32_t key) {
    uint32_t h = set_hash(key);
    for (int i = 0; i < SET_SIZE; ++i) {
        const uint32_t k = set[h];
        if (k == key) return true;
        if (k == KEY32_EMPTY) return false;
        h = (h + 1) & (SET_SIZE - 1);
    }
    return false;
}

// Publish a claimed entry: record its block coordinate, mark the slot fresh,
// then make the slot visible to other threads.
__device__ inline void publish(const DevVolume& V, int entry, unsigned long long key, uint32_t slot) {
    if (slot >= V.max_blocks) {
        set_status(V.status, SC_ERR_POOL_FULL);
        atomicExch(&V.table[entry].slot, SLOT_FAILED);
        return;
    }
    const int3 c = unpack_key(key);
    V.coord[slot] = make_int4(c.x, c.y, c.z, 0);
    V.flags[slot] = FLAG_FRESH;
    __threadfence();
    atomicExch(&V.table[entry].slot, (int32_t)slot);
}

constexpr int WIN = 16;  // tile window edge in blocks (byte map of WIN^3 entries)

struct AllocShared {
    uint4 bmap[WIN * WIN * WIN / 16];  // byte per window block (x + WIN y + WIN^2 z): 1 = met
    uint32_t set[SET_SIZE];  // open-addressing set of the tile's other block keys (key32)
    uint32_t uk[SET_SIZE];   // compacted: the unique keys (key32) of the tile
    int n_keys;    // unique keys found; uk holds the first SET_SIZE of them
    int overflow;  // 1: a key did not fit the set (its threads run phase D); 2: more unique keys
                   // than uk holds (every thread runs phase D over all its blocks)
    int3 wo;       // window origin (block coordinates); window off when wo.x == INT_MIN
    KfCam cam;     // the tile's camera, read by every pixel's walk from shared memory (4 %
                   // faster than from the batch's item table in global memory)
};

// Append the slots of the lanes with `pred` through a global counter: one atomic add
// per warp.  Called by all 32 lanes.
__device__ __forceinline__ void warp_append(const DevVolume& V, int32_t* list, int32_t* count, uint32_t cap, bool pred,
                                            int32_t slot, int32_t full_code) {
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    int b = 0;
    if (lane == 0) b = atomicAdd(count, __popc(m));
    b = __shfl_sync(0xffffffffu, b, 0);
    if (pred) {
        const uint32_t p = (uint32_t)b + (uint32_t)__popc(m & ((1u << lane) - 1u));
        if (p < cap) list[p] = slot;
        else set_status(V.status, full_code);
    }
}

// Append one slot through a global counter (used by phase D).
__device__ inline void append_one(const DevVolume& V, int32_t* list, int32_t* count, uint32_t cap, int32_t slot) {
    const uint32_t p = (uint32_t)atomicAdd(count, 1);
    if (p < cap) list[p] = slot;
    else set_status(V.status, SC_ERR_LIST_FULL);
}

// Process tile (tx, ty) of keyframe camera k.  The Sink provides
//   bool list_first(slot)  : true the first time this keyframe reaches slot
//   void mark_new(slot)    : record that this keyframe has listed a slot just created
//   bool union_first(slot) : true the first time the batch reaches slot (batches only)
//   int32_t* list, *count; uint32_t cap; int32_t* ulist, *ucount; uint32_t ucap
// Must be called by all ALLOC_THREADS threads of the CTA.
// The camera's block: 32-bit set keys are relative to it.
__device__ __forceinline__ int3 cam_block(const KfCam& k) {
    return make_int3(k.ti[0] >> 3, k.ti[1] >> 3, k.ti[2] >> 3);
}

// Window of a tile: 16^3 blocks centred on the block of the surface point (depth Z, no
// band) of a reference pixel -- the first valid one of the tile centre and eight points
// around it -- so that a smooth surface's blocks fall inside.  Off (wo.x = INT_MIN) when
// no reference pixel is valid or a window block would lie outside the 32-bit key range.
template <int TY>
__device__ inline int3 tile_window(const KfCam& k, int tx, int ty, const int3& ref, bool ref_ok) {
    const int3 off = make_int3(INT_MIN, 0, 0);
    if (!ref_ok) return off;
    // the tile centre first, then the eight points halfway to its edges and corners:
    // all nine depths requested together, the first valid one kept
    constexpr int qx[9] = {2, 1, 3, 1, 3, 2, 2, 1, 3}, qy[9] = {2, 1, 1, 3, 3, 1, 3, 2, 2};
    float Z = 0.f;
    int uz = 0, vz = 0;
#pragma unroll
    for (int c = 8; c >= 0; --c) {
        const int u = min(tx * ALLOC_TX + ALLOC_TX / 4 * qx[c], k.W - 1);
        const int v = min(ty * TY + TY / 4 * qy[c], k.H - 1);
        const float z = __ldg(k.depth + (size_t)v * k.W + u);
        const bool ok = z > 0.f && z < MAX_DEPTH;
        Z = ok ? z : Z;
        uz = ok ? u : uz;
        vz = ok ? v : vz;
    }
    if (!(Z > 0.f)) return off;
    const float xn = __fmul_rn(__fsub_rn((float)uz, k.cx), k.ifx);
    const float yn = __fmul_rn(__fsub_rn((float)vz, k.cy), k.ify);
    int b[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float ray = __fmaf_rn(k.Ms[3 * r], xn, __fmaf_rn(k.Ms[3 * r + 1], yn, k.Ms[3 * r + 2]));
        b[r] = ((__float2int_rd(__fmaf_rn(Z, ray, k.tf[r])) + k.ti[r]) >> 3) - WIN / 2;
    }
    // every window block must have a 32-bit key (|b - ref| <= 511 per axis)
    if (b[0] - ref.x < -512 || b[0] + WIN - 1 - ref.x > 511 || b[1] - ref.y < -512 || b[1] + WIN - 1 - ref.y > 511 ||
        b[2] - ref.z < -512 || b[2] + WIN - 1 - ref.z > 511)
        return off;
    return make_int3(b[0], b[1], b[2]);
}

// Phase A of a tile, shared by the allocation and the stream-in probe: clear the byte
// map and the set, insert every pixel's band-segment blocks, compact the unique keys
// into uk (its first min(n_keys, SET_SIZE) entries).  Returns this thread's overflow flag (a key that did not
// fit, or a camera so far out that its 32-bit keys could decode to invalid
// coordinates); the CTA-wide flag is sh.overflow.  Must be called by all ALLOC_THREADS
// threads.
template <int TY>
__device__ inline bool tile_collect(const KfCam& k, int tx, int ty, AllocShared& sh) {
    constexpr int PPT = alloc_ppt<TY>();
    const int tid = threadIdx.x;
    for (int i = tid; i < WIN * WIN * WIN / 16; i += ALLOC_THREADS) sh.bmap[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid; i < SET_SIZE; i += ALLOC_THREADS) sh.set[i] = KEY32_EMPTY;
    {
        const uint32_t* cs = reinterpret_cast<const uint32_t*>(&k);
        uint32_t* cd = reinterpret_cast<uint32_t*>(&sh.cam);
        for (int i = tid; i < (int)(sizeof(KfCam) / 4); i += ALLOC_THREADS) cd[i] = cs[i];
    }
    const int3 ref = cam_block(k);
    // every 32-bit key of this camera decodes to a valid block coordinate (else all its
    // blocks take the overflow path, which checks each one)
    const bool ref_ok = coord_ok(ref.x - 512, ref.y - 512, ref.z - 512) && coord_ok(ref.x + 511, ref.y + 511, ref.z + 511);
    if (tid == 0) {
        sh.n_keys = 0;
        sh.overflow = 0;
        sh.wo = tile_window<TY>(k, tx, ty, ref, ref_ok);
    }
    const int u = tx * ALLOC_TX + (tid % ALLOC_TX);
    const int v0 = ty * TY + (tid / ALLOC_TX);
    float Zp[PPT];
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        const int v = v0 + r * (ALLOC_THREADS / ALLOC_TX);
        Zp[r] = (u < k.W && v < k.H) ? __ldg(k.depth + (size_t)v * k.W + u) : 0.f;
    }
    __syncthreads();
    const int3 wo = sh.wo;
    unsigned char* bmap = reinterpret_cast<unsigned char*>(sh.bmap);
    bool my_ovf = false;
    // unrolled over the thread's pixels: their walks interleave (4.5 % faster than one
    // pixel at a time, despite the longer code)
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
        const int v = v0 + r * (ALLOC_THREADS / ALLOC_TX);
        const float Z = Zp[r];
        auto ins = [&](int bx, int by, int bz) {
            const uint32_t dx = (uint32_t)bx - (uint32_t)wo.x, dy = (uint32_t)by - (uint32_t)wo.y,
                           dz = (uint32_t)bz - (uint32_t)wo.z;
            if ((dx | dy | dz) < (uint32_t)WIN) {  // inside the window (never when it is off)
                bmap[dx + WIN * dy + WIN * WIN * dz] = 1;
                return;
            }
            uint32_t kk;
            if (!ref_ok || !key32(bx, by, bz, ref, &kk) || !set_insert(sh.set, kk)) my_ovf = true;
        };
        if (Z > 0.f && Z < MAX_DEPTH) for_each_segment_block(sh.cam, u, v, Z, ins);
    }
    if (my_ovf) sh.overflow = 1;
    __syncthreads();
    // compact the window's met blocks and the set's keys so that the global phases run
    // in one round; more unique keys than uk holds send the whole tile to phase D
    auto push = [&](uint32_t key) {
        const int p = atomicAdd(&sh.n_keys, 1);
        if (p < SET_SIZE) sh.uk[p] = key;
        else sh.overflow = 2;
    };
    if (wo.x != INT_MIN) {
        for (int i = tid; i < WIN * WIN * WIN / 16; i += ALLOC_THREADS) {
            const uint4 q = sh.bmap[i];
            const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t m = w4[j];
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= ~(0xffu << (bit & ~7));
                    const int e = 16 * i + 4 * j + (bit >> 3);
                    uint32_t kk;
                    key32(wo.x + (e % WIN), wo.y + (e / WIN) % WIN, wo.z + e / (WIN * WIN), ref, &kk);
                    push(kk);
                }
            }
        }
    }
    for (int i = tid; i < SET_SIZE; i += ALLOC_THREADS)
        if (sh.set[i] != KEY32_EMPTY) push(sh.set[i]);
    __syncthreads();
    return my_ovf;
}

// Whether block (bx, by, bz) of this tile was compacted into uk (in the window, or in
// the set); false for every block once the tile has more unique keys than uk holds.
__device__ __forceinline__ bool tile_holds(const AllocShared& sh, int bx, int by, int bz, const int3& ref,
                                           bool ref_ok) {
    if (sh.overflow == 2) return false;
    const uint32_t dx = (uint32_t)bx - (uint32_t)sh.wo.x, dy = (uint32_t)by - (uint32_t)sh.wo.y,
                   dz = (uint32_t)bz - (uint32_t)sh.wo.z;
    if ((dx | dy | dz) < (uint32_t)WIN) return true;
    uint32_t kk;
    return ref_ok && key32(bx, by, bz, ref, &kk) && set_contains(sh.set, kk);
}

// Every block of this thread's pixels that the tile did not compact (the overflow
// path): f(bx, by, bz) for each, coordinates checked.
template <int TY, typename F>
__device__ inline void tile_overflow_blocks(const DevVolume& V, const KfCam& k, int tx, int ty, const AllocShared& sh,
                                            F&& f) {
    const int tid = threadIdx.x;
    const int3 ref = cam_block(k);
    const bool ref_ok = coord_ok(ref.x - 512, ref.y - 512, ref.z - 512) && coord_ok(ref.x + 511, ref.y + 511, ref.z + 511);
    const int u = tx * ALLOC_TX + (tid % ALLOC_TX);
    const int v0 = ty * TY + (tid / ALLOC_TX);
    for (int r = 0; r < alloc_ppt<TY>(); ++r) {
        const int v = v0 + r * (ALLOC_THREADS / ALLOC_TX);
        float Z = 0.f;
        if (u < k.W && v < k.H) Z = __ldg(k.depth + (size_t)v * k.W + u);
        if (!(Z > 0.f && Z < MAX_DEPTH)) continue;
        for_each_segment_block(k, u, v, Z, [&](int bx, int by, int bz) {
            if (!coord_ok(bx, by, bz)) {
                set_status(V.status, SC_ERR_INVALID_ARG);
                return;
            }
            if (tile_holds(sh, bx, by, bz, ref, ref_ok)) return;
            f(bx, by, bz);
        });
    }
}

template <int TY, typename Sink>
__device__ inline void alloc_tile(const DevVolume& V, const KfCam& k, int tx, int ty, Sink& sk, AllocShared& sh) {
    const int tid = threadIdx.x;
    // A: every pixel's band-segment blocks into the shared set
    const bool my_ovf = tile_collect<TY>(k, tx, ty, sh);
    const int3 ref = cam_block(k);
    const int nk = min(sh.n_keys, SET_SIZE);

    // B + C, warp by warp without CTA barriers: each warp claims its keys, takes pool
    // slots for the entries it created with one atomic add, publishes them, then
    // dedupes its keys' slots and appends them with one atomic add per list.  A warp
    // publishes its own entries before it waits for anyone else's, so no wait is circular.
    const int lane = tid & 31;
    const int nk_w = (nk + 31) & ~31;  // warp-uniform trip count: the ballots see whole warps
    for (int i = tid; i < nk_w; i += ALLOC_THREADS) {
        const bool act = i < nk;
        bool won = false;
        int32_t seen = -1;
        int e = -1;
        unsigned long long key = 0;
        if (act) {
            key = key64_of(sh.uk[i], ref);
            e = hash_claim(V, key, &won, &seen);
            won = won && e >= 0;
        }
        const unsigned wm = __ballot_sync(0xffffffffu, won);
        uint32_t base = 0;
        if (wm) {
            if (lane == 0) base = atomicAdd(V.pool_count, (uint32_t)__popc(wm));
            base = __shfl_sync(0xffffffffu, base, 0);
        }
        int32_t slot = seen;
        if (won) {
            const uint32_t ns = base + (uint32_t)__popc(wm & ((1u << lane) - 1u));
            // nobody else can list a slot before it is published: mark it for this
            // keyframe, then publish (a full pool publishes a failed entry instead)
            if (ns < V.max_blocks) {
                sk.mark_new((int32_t)ns);
                slot = (int32_t)ns;
            }
            publish(V, e, key, ns);
        } else if (act && e >= 0 && slot < 0) {
            slot = entry_slot(V, e);
        }
        const bool ok = act && e >= 0 && slot >= 0;
        const bool first = ok && (won || sk.list_first(slot));
        const bool ufirst = Sink::kUnion && ok && sk.union_first(slot);
        warp_append(V, sk.list, sk.count, sk.cap, first, slot, SC_ERR_LIST_FULL);
        if (Sink::kUnion) warp_append(V, sk.ulist, sk.ucount, sk.ucap, ufirst, slot, SC_ERR_POOL_FULL);
    }

    // D: keys that did not fit in the shared set
    if (sh.overflow == 2 || (sh.overflow != 0 && my_ovf)) {
        tile_overflow_blocks<TY>(V, k, tx, ty, sh, [&](int bx, int by, int bz) {
            const unsigned long long key = pack_key(bx, by, bz);
            bool won;
            int32_t seen;
            const int e = hash_claim(V, key, &won, &seen);
            if (e < 0) return;
            if (won) publish(V, e, key, atomicAdd(V.pool_count, 1u));
            const int32_t slot = seen >= 0 ? seen : entry_slot(V, e);
            if (slot < 0) return;
            if (sk.list_first(slot)) append_one(V, sk.list, sk.count, sk.cap, slot);
            if (Sink::kUnion && sk.union_first(slot)) append_one(V, sk.ulist, sk.ucount, sk.ucap, slot);
        });
    }
    __syncthreads();  // shared state is reused by the CTA's next tile
}

struct PlainSink {
    static constexpr bool kUnion = false;
    uint32_t* stamp;
    uint32_t call_id;
    int32_t* list;
    int32_t* count;
    uint32_t cap;
    int32_t* ulist;
    int32_t* ucount;
    uint32_t ucap;
    __device__ bool list_first(int32_t slot) { return atomicExch(&stamp[slot], call_id) != call_id; }
    __device__ void mark_new(int32_t slot) { stamp[slot] = call_id; }
    __device__ bool union_first(int32_t) { return false; }
};

}  // namespace sc
