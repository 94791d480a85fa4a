// Batched re-integration of one pose-graph update (Section 4.3 "Re-integration
// strategy"): every item is de-integrated at its former pose and re-integrated
// at its updated pose.
//
// Sequential semantics (de-integrate all items in order, then integrate all
// items in order) give, per voxel, in exact arithmetic
//   W' = W - sum_old w + sum_new w,   D' = (D W - sum_old d w + sum_new d w) / W'
// (and D' = 0 when W' = 0; a voxel whose weight passes through 0 mid-sequence
// has D W - sum_old d w = 0 there, so the reset of Eq. 2 changes nothing).  The
// batch therefore computes each touched voxel's net change over all items and
// applies it with ONE read-modify-write of its D / W / C, instead of 2n.
//
// Graph (captured once per launch configuration, replayed every call, launched without
// a host synchronisation):
//   1. H2D copy of the call's header and item table (one of two alternating pinned
//      staging blocks; the node is pointed at it and resized per call)
//   2. pack: zero the counters and the items' new block-list counts; pack the depth and
//      colour of each item whose texel slot does not already hold its images into
//      8-byte texels (one gather per sample in step 5)
//   3. batched allocation of A(k, T_new) for all items (persistent over
//      (item, pixel tile)); each item's new list is deduplicated with a per-slot
//      item bit; every touched slot joins the batch's union list once
//   4. mark old footprints: set (item, old) bits on every slot of each item's
//      current list, union as above
//   5. net-delta: persistent warps take (union block, voxel group) units from a
//      queue, recompute each (voxel, item) sample for the items whose bits are set,
//      sum, and apply once
//   6. clear the union slots' item bits and fresh flags
//   7. D2H copy of the status word
// Per-slot item bitmasks: [max_blocks][mw] words, old bits then new bits; step 6
// zeroes them again, so the masks are all zero between calls.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "alloc.cuh"
#include "volume.cuh"

using namespace sc;

namespace {

struct BatchItem {
    KfCam oldc;
    KfCam newc;
    int32_t* old_list;
    int32_t* old_count;
    int32_t* new_list;
    int32_t* new_count;
    int32_t pack_item;  // items[r].pack_item, r < n_pack: the r-th item whose texels this call packs
};

struct BatchHeader {
    int32_t n;
    uint32_t call_id;
    int32_t tiles_x;
    int32_t tiles;
    int32_t n_pack;  // items whose texel slot does not already hold their images
};
constexpr size_t STAGE_HDR = 256;  // header bytes ahead of the item table in a staging block

constexpr int ALLOC_CTAS_PER_SM = SC_ALLOC_CTAS_PER_SM;  // persistent allocation CTAs per SM

struct BatchSink {
    static constexpr bool kUnion = true;
    uint32_t* masks;  // this item's new-bit word, slot stride mw
    int mw;
    uint32_t bit;
    uint32_t* stamp;
    uint32_t call_id;
    int32_t* list;
    int32_t* count;
    uint32_t cap;
    int32_t* ulist;
    int32_t* ucount;
    uint32_t ucap;
    __device__ bool list_first(int32_t slot) {
        return !(atomicOr(masks + (size_t)slot * mw, bit) & bit);
    }
    // other items may set their bits on a new slot as soon as it is published
    __device__ void mark_new(int32_t slot) { atomicOr(masks + (size_t)slot * mw, bit); }
    __device__ bool union_first(int32_t slot) { return atomicExch(&stamp[slot], call_id) != call_id; }
};

__global__ void __launch_bounds__(ALLOC_THREADS, SC_ALLOC_CTAS_PER_SM) batch_alloc_kernel(DevVolume V, const BatchItem* items,
                                                                    const BatchHeader* hdr, uint32_t* masks, int mw,
                                                                    int32_t* ulist, int32_t* counters,
                                                                    uint32_t list_cap) {
    __shared__ AllocShared sh;
    const int n = hdr->n, tiles = hdr->tiles, tiles_x = hdr->tiles_x;
    const uint32_t call_id = hdr->call_id;
    const int half = mw / 2;
    for (int w = blockIdx.x; w < n * tiles; w += gridDim.x) {
        const int i = w / tiles, t = w - i * tiles;
        const BatchItem& it = items[i];
        BatchSink sk{masks + half + (i >> 5), mw, 1u << (i & 31), V.stamp, call_id, it.new_list, it.new_count,
                     list_cap, ulist, counters, V.max_blocks};
        alloc_tile<ALLOC_TY>(V, it.newc, t % tiles_x, t / tiles_x, sk, sh);
    }
}

// grid (chunks, max_batch): blockIdx.y is the item, its chunk CTAs stride over its list
__global__ void batch_mark_old_kernel(DevVolume V, const BatchItem* items, const BatchHeader* hdr, uint32_t* masks,
                                      int mw, int32_t* ulist, int32_t* counters, uint32_t list_cap) {
    const int n = hdr->n;
    const uint32_t call_id = hdr->call_id;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.y; i < n; i += gridDim.y) {
        const uint32_t cnt = min((uint32_t)*items[i].old_count, list_cap);
        const int32_t* list = items[i].old_list;
        const uint32_t bit = 1u << (i & 31);
        // warp-uniform trip count so the ballot below sees the full warp
        for (uint32_t base = blockIdx.x * blockDim.x; base < cnt; base += stride) {
            const uint32_t j = base + threadIdx.x;
            bool first = false;
            int32_t slot = -1;
            if (j < cnt) {
                slot = list[j];
                if (slot >= 0) {
                    atomicOr(masks + (size_t)slot * mw + (i >> 5), bit);
                    first = atomicExch(&V.stamp[slot], call_id) != call_id;
                } else {
                    set_status(V.status, SC_ERR_NOT_RESIDENT);  // streamed out to the host
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, first);
            if (!m) continue;
            int b = 0;
            if (lane == 0) b = atomicAdd(counters, __popc(m));
            b = __shfl_sync(0xffffffffu, b, 0);
            if (first) {
                const uint32_t p = (uint32_t)b + __popc(m & ((1u << lane) - 1u));
                if (p < V.max_blocks) ulist[p] = slot;
                else set_status(V.status, SC_ERR_POOL_FULL);
            }
        }
    }
}

// The part of a keyframe camera the net-delta kernel samples with, kept in shared
// memory (96 bytes; old cameras of items 0..n-1, then their new cameras).
struct __align__(16) NdCam {
    float2 Pxy[3];  // as in KfCam
    float2 cxyh;
    float Pz[3];
    float tf[3];
    float tiF[3];
    float mu;
    int W, H;
    const uint2* tex;
};
static_assert(sizeof(NdCam) == 96, "camera table entry: 96 bytes");

__device__ __forceinline__ void load_ndcam(NdCam& o, const KfCam& k) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        o.Pxy[i] = k.Pxy[i];
        o.Pz[i] = k.Pz[i];
        o.tf[i] = k.tf[i];
        o.tiF[i] = k.tiF[i];
    }
    o.cxyh = k.cxyh;
    o.mu = k.mu;
    o.W = k.W;
    o.H = k.H;
    o.tex = k.tex;
}

// Packed copies of the items' keyframes, one 8-byte texel per pixel so that a sample
// reads depth and colour with one gather: x = the depth bits, with every invalid depth
// (Z <= 0 or NaN) stored as -inf; y = RGB8 with the alpha byte set to 1 (it counts the
// samples: see NdAcc).  Item i's texels start at tex + i * stride (stride = the pixel
// count rounded up to even, > npx: 16-byte aligned) and texel npx is a sentinel (-inf,
// 0) that voxels projecting outside the image read, so that eta = Z - z_c >= -mu alone
// decides a sample (-inf never passes it).
__device__ __forceinline__ uint2 pack_texel(float z, uint32_t c) {
    return make_uint2(z > 0.f ? __float_as_uint(z) : 0xff800000u, (c & 0x00ffffffu) | 0x01000000u);
}

// Only the header's n_pack listed items are packed: a slot that already holds its
// item's images is skipped without a pass over its pixels.  The first kernel of the
// batch graph, so it also zeroes the items' new-list counts and the batch counters.
__global__ void batch_pack_kernel(const BatchItem* items, const BatchHeader* hdr, uint2* tex, uint32_t npx,
                                  uint32_t stride, int32_t* counters) {
    const int n = hdr->n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) *items[i].new_count = 0;
    if (blockIdx.x == 0 && threadIdx.x < 4) counters[threadIdx.x] = 0;
    const uint32_t q = npx / 4;  // 640 x 480 and every width multiple of 4: float4 / uint4 loads
    const int n_pack = hdr->n_pack;
    const size_t total = (size_t)n_pack * q;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / q);
        const int it = items[r].pack_item;
        const uint32_t p = (uint32_t)(i - (size_t)r * q) * 4;
        const KfCam& k = items[it].newc;
        const float4 d = __ldg(reinterpret_cast<const float4*>(k.depth + p));
        const uint4 c = __ldg(reinterpret_cast<const uint4*>(k.rgba + p));
        const uint2 t0 = pack_texel(d.x, c.x), t1 = pack_texel(d.y, c.y), t2 = pack_texel(d.z, c.z),
                    t3 = pack_texel(d.w, c.w);
        uint4* o = reinterpret_cast<uint4*>(tex + (size_t)it * stride + p);
        o[0] = make_uint4(t0.x, t0.y, t1.x, t1.y);
        o[1] = make_uint4(t2.x, t2.y, t3.x, t3.y);
    }
    // remainder pixels (npx % 4) and each item's sentinel
    const uint32_t r0 = q * 4, nr = npx - r0 + 1;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)n_pack * nr;
         i += (size_t)gridDim.x * blockDim.x) {
        const int it = items[i / nr].pack_item;
        const uint32_t p = r0 + (uint32_t)(i % nr);
        const KfCam& k = items[it].newc;
        tex[(size_t)it * stride + p] = p < npx ? pack_texel(k.depth[p], k.rgba[p]) : make_uint2(0xff800000u, 0u);
    }
}

// Per-voxel net sums of one voxel group.  Colour channels and the weight are
// integers; when fewer than PACK_MAX_ITEMS item bits are set on the block they are
// kept packed, two 16-bit lanes per register biased by 2^15 (r | b << 16 and
// g | count << 16): every partial sum then stays inside [0, 2^16) -- at most
// 128 x 255 < 2^15 is added or subtracted -- so the lanes never carry or borrow into
// each other and the packed sums equal the separate integer sums exactly.
constexpr uint32_t PACK_BIAS = 0x80008000u;
constexpr int PACK_MAX_ITEMS = 128;

struct NdAcc {
    float aD[4];      // sum of signed distances (float, in item order)
    uint32_t rb[4];   // packed: r | b << 16   (packed mode)
    uint32_t gw[4];   // packed: g | count << 16
};

struct NdAccWide {
    float aD[4];
    int aW[4];
    int aC[4][3];
};

// One item's contribution to the 4 voxels, given their projection and texels.
// Branch-free: the update decision of decide() is eta >= -mu on the packed texel
// (invalid depth and voxels outside the image read -inf, in front of the camera or
// not), and it selects the contribution; a voxel that is not updated adds exactly zero
// (its distance sum is never -0, so +0 leaves it bit for bit).  The texel's bytes give
// the packed lanes directly: r | b << 16 and g | 1 << 16 (the alpha byte is the count).
template <int SIGN>
__device__ __forceinline__ void net_delta_item(const NdCam& k, const Proj4& P, const uint2 t[4], NdAcc& A,
                                               bool& touched) {
    const float mu = k.mu;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float eta = __fsub_rn(__uint_as_float(t[j].x), P.pz[j]);
        const bool up = eta >= -mu;
        const float d = up ? fminf(eta, mu) : 0.f;
        const uint32_t cw = up ? t[j].y : 0u;
        const uint32_t rb = __byte_perm(cw, 0u, 0x4240);
        const uint32_t gw = __byte_perm(cw, 0u, 0x4341);
        if (SIGN > 0) {
            A.aD[j] = __fadd_rn(A.aD[j], d);
            A.rb[j] += rb;
            A.gw[j] += gw;
        } else {
            A.aD[j] = __fsub_rn(A.aD[j], d);
            A.rb[j] -= rb;
            A.gw[j] -= gw;
        }
    }
}

// The same with separate integer sums (more than PACK_MAX_ITEMS bits on a block).
template <int SIGN>
__device__ __forceinline__ void net_delta_item(const NdCam& k, const Proj4& P, const uint2 t[4], NdAccWide& A,
                                               bool& touched) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float d, eta;
        if (decide(k, P.ok[j], __uint_as_float(t[j].x), P.pz[j], d, eta)) {
            touched = true;
            const uint32_t cw = t[j].y;
            const int s = SIGN;
            A.aD[j] = SIGN > 0 ? __fadd_rn(A.aD[j], d) : __fsub_rn(A.aD[j], d);
            A.aW[j] += s;
            A.aC[j][0] += s * (int)(cw & 255u);
            A.aC[j][1] += s * (int)((cw >> 8) & 255u);
            A.aC[j][2] += s * (int)((cw >> 16) & 255u);
        }
    }
}

// Projection of the 4 voxels into item k and the texels (depth bits, RGBA8) they sample.
__device__ __forceinline__ void net_delta_fetch(const NdCam& k, float vx, float vy, float vz, Proj4& P, uint2 t[4]) {
    project4(k, vx, vy, vz, P);
    // a voxel outside the image reads the item's sentinel texel (index W H)
    const int sentinel = k.W * k.H;
#pragma unroll
    for (int j = 0; j < 4; ++j) t[j] = __ldg(k.tex + (P.ok[j] ? P.pix[j] : sentinel));
}

// Net change of the 4 voxels (lx0..lx0+3, ly, lz) of block c over the items whose
// bits are set in mask word `word` (items ibase .. ibase + 31 of the camera table
// `cams`), with sign SIGN (-1: old bits, de-integration; +1: new bits).  Weights and
// colours are integer sums (exactly the float sums of the same integers); distances
// are summed in float in item order.
template <int SIGN, typename Acc>
__device__ __forceinline__ void net_delta_word(const NdCam* cams, uint32_t word, float vx, float vy, float vz,
                                               Acc& A, bool& touched) {
    while (word) {
        const int b0 = __ffs(word) - 1;
        word &= word - 1;
        Proj4 P0;
        uint2 t0[4];
        net_delta_fetch(cams[b0], vx, vy, vz, P0, t0);
        net_delta_item<SIGN>(cams[b0], P0, t0, A, touched);
    }
}

// All items of the slot's mask: old bits (first half of the words) subtract, new
// bits add, in item order.
template <typename Acc>
__device__ __forceinline__ void net_delta_group(const NdCam* cams, int n, const int4 c, int lx0, int ly, int lz,
                                                uint32_t mw0, uint32_t mw1, int mw, Acc& A, bool& touched) {
    const int half = mw / 2;
    const float vx = (float)(8 * c.x + lx0), vy = (float)(8 * c.y + ly), vz = (float)(8 * c.z + lz);
    // only the words with a bit set, in increasing word order (old words come first, so
    // the items keep their order); lane w holds word w, lane w - 32 word w >= 32
    unsigned long long nzw = (unsigned long long)__ballot_sync(0xffffffffu, mw0 != 0u) |
                             ((unsigned long long)__ballot_sync(0xffffffffu, mw1 != 0u) << 32);
    while (nzw) {
        const int w = __ffsll(nzw) - 1;
        nzw &= nzw - 1;
        const uint32_t word = __shfl_sync(0xffffffffu, w < 32 ? mw0 : mw1, w & 31);
        if (w < half) net_delta_word<-1>(cams + (w << 5), word, vx, vy, vz, A, touched);
        else net_delta_word<1>(cams + n + ((w - half) << 5), word, vx, vy, vz, A, touched);
    }
}

// Net weight and colour sums of voxel j as integers.
__device__ __forceinline__ void nd_unpack(const NdAcc& A, int j, int& w, int c[3]) {
    w = (int)(A.gw[j] >> 16) - 32768;
    c[0] = (int)(A.rb[j] & 0xFFFFu) - 32768;
    c[1] = (int)(A.gw[j] & 0xFFFFu) - 32768;
    c[2] = (int)(A.rb[j] >> 16) - 32768;
}
__device__ __forceinline__ void nd_unpack(const NdAccWide& A, int j, int& w, int c[3]) {
    w = A.aW[j];
    c[0] = A.aC[j][0];
    c[1] = A.aC[j][1];
    c[2] = A.aC[j][2];
}

// Whether any of the 4 voxels has a net change (the packed sums track no "touched"
// flag per sample: a voxel whose samples cancel exactly is left as it is, which is
// what the read-modify-write would write back).
__device__ __forceinline__ bool nd_changed(const NdAcc& A, bool touched) {
    bool c = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) c |= (A.aD[j] != 0.f) | (A.rb[j] != PACK_BIAS) | (A.gw[j] != PACK_BIAS);
    return c;
}
__device__ __forceinline__ bool nd_changed(const NdAccWide&, bool touched) { return touched; }

__device__ __forceinline__ void nd_init(NdAcc& A) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        A.aD[j] = 0.f;
        A.rb[j] = PACK_BIAS;
        A.gw[j] = PACK_BIAS;
    }
}
__device__ __forceinline__ void nd_init(NdAccWide& A) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        A.aD[j] = 0.f;
        A.aW[j] = 0;
        A.aC[j][0] = A.aC[j][1] = A.aC[j][2] = 0;
    }
}

// The read-modify-write of one voxel group (4 voxels per lane) with its net sums:
// D' = (D W + sum d) / W', W' = W + sum w, colour likewise (W' = 0 resets the voxel).
// RGBA8: Dv, Wv, Cv were loaded before the samples (zero for a fresh block).
template <bool F32, typename Acc>
__device__ __forceinline__ void nd_apply(const DevVolume& V, int32_t slot, size_t off, int lane, int g, bool fresh,
                                         const Acc& A, float4 Dv, float4 Wv, uint4 Cv) {
    float aW[4], aC[4][3];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int w, c[3];
        nd_unpack(A, j, w, c);
        aW[j] = (float)w;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) aC[j][ch] = (float)c[ch];
    }
    float* Dp = &Dv.x;
    float* Wp = &Wv.x;
    float Wn[4], rW[4];
    bool nz[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        Wn[j] = __fadd_rn(Wp[j], aW[j]);
        nz[j] = Wn[j] != 0.f;
        // one reciprocal per voxel for its four quotients (D and three colour channels):
        // a few ulp where a division would give 0.5 ulp -- 1e-8 m for |D| <= mu, and a
        // colour quotient moves by ~1e-5 of a level, which can only change the 8-bit
        // rounding of a quotient that lies exactly on a half level
        rW[j] = rcp_approx(Wn[j]);
    }
    if (F32) {
        const size_t cb = (size_t)slot * 3 * NVOX + 4 * lane + 128 * g;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float4 Cf = fresh ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(V.Cf + cb + ch * NVOX);
            float* Cp = &Cf.x;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (aW[j] != 0.f || aC[j][ch] != 0.f)
                    Cp[j] = nz[j] ? __fmul_rn(__fmaf_rn(Cp[j], Wp[j], aC[j][ch]), rW[j]) : 0.f;
            *reinterpret_cast<float4*>(V.Cf + cb + ch * NVOX) = Cf;
        }
    } else {
        // branch-free: every voxel's new value is computed and selected (a voxel without
        // a net change keeps its bytes; W' = 0 empties it)
        uint32_t* Cp = &Cv.x;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool ch_any = aW[j] != 0.f || aC[j][0] != 0.f || aC[j][1] != 0.f || aC[j][2] != 0.f;
            uint32_t out = 0;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float a = (float)((Cp[j] >> (8 * ch)) & 255u);
                out |= u8_sat(__fmul_rn(__fmaf_rn(a, Wp[j], aC[j][ch]), rW[j])) << (8 * ch);
            }
            Cp[j] = ch_any ? (nz[j] ? out : 0u) : Cp[j];
        }
        __stcs(reinterpret_cast<uint4*>(V.C8 + off), Cv);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool d_any = aW[j] != 0.f || A.aD[j] != 0.f;
        const float Dn = nz[j] ? __fmul_rn(__fmaf_rn(Dp[j], Wp[j], A.aD[j]), rW[j]) : 0.f;
        Dp[j] = d_any ? Dn : Dp[j];
        Wp[j] = d_any ? Wn[j] : Wp[j];
    }
    __stcs(reinterpret_cast<float4*>(V.D + off), Dv);
    __stcs(reinterpret_cast<float4*>(V.W + off), Wv);
}

// One voxel group of a block: the samples of every item with a bit on the block,
// then one read-modify-write (in RGBA8 evict-first: the state is read and written
// once).  The state is loaded after the samples: held across them, its 12 registers
// kept the kernel at 4 CTAs per SM; loaded late, it fits 48 registers and 5 CTAs
// (Kinect pose update -2 %, batching workload +4 % re-integrations/s).
template <bool F32, typename Acc>
__device__ __forceinline__ void nd_group(const DevVolume& V, const NdCam* cams, int n_items, int32_t slot, int4 c,
                                         bool fresh, uint32_t mw0, uint32_t mw1, int mw, int lane, int g) {
    int lx0, ly, lz;
    lane_voxels(lane, g, lx0, ly, lz);
    const size_t off = (size_t)slot * NVOX + 4 * lane + 128 * g;
    Acc A;
    nd_init(A);
    bool touched = false;
    net_delta_group(cams, n_items, c, lx0, ly, lz, mw0, mw1, mw, A, touched);
    if (!nd_changed(A, touched) && !fresh) return;
    float4 Dv = make_float4(0.f, 0.f, 0.f, 0.f), Wv = Dv;
    uint4 Cv = make_uint4(0u, 0u, 0u, 0u);
    if (!F32) {
        Dv = __ldcs(reinterpret_cast<const float4*>(V.D + off));
        Wv = __ldcs(reinterpret_cast<const float4*>(V.W + off));
        Cv = __ldcs(reinterpret_cast<const uint4*>(V.C8 + off));
    } else if (!fresh) {
        Dv = *reinterpret_cast<const float4*>(V.D + off);
        Wv = *reinterpret_cast<const float4*>(V.W + off);
    }
    if (fresh) {  // first update of a new block: its memory holds no prior state
        Dv = make_float4(0.f, 0.f, 0.f, 0.f);
        Wv = Dv;
        Cv = make_uint4(0u, 0u, 0u, 0u);
    }
    nd_apply<F32>(V, slot, off, lane, g, fresh, A, Dv, Wv, Cv);
}

// Work unit u = (union block u / 4, voxel group u % 4): one warp, 128 voxels, four
// per lane.  Units come from a queue in chunks of `grab`.
#ifndef SC_ND_MIN_BLOCKS
#define SC_ND_MIN_BLOCKS 5  // CTAs of 256 threads per SM the register budget must allow (48 registers)
#endif

template <bool F32>
__global__ void __launch_bounds__(256, SC_ND_MIN_BLOCKS) net_delta_kernel(DevVolume V, const BatchItem* items, const BatchHeader* hdr, uint32_t* masks,
                                 int mw, const int32_t* ulist, int32_t* counters, int grab, uint32_t list_cap) {
    extern __shared__ __align__(16) unsigned char nd_smem[];
    NdCam* cams = reinterpret_cast<NdCam*>(nd_smem);
    const int n_items = hdr->n;
    for (int i = threadIdx.x; i < 2 * n_items; i += blockDim.x)
        load_ndcam(cams[i], i < n_items ? items[i].oldc : items[i - n_items].newc);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t n_union = min((uint32_t)counters[0], V.max_blocks);
    const uint32_t n_units = 4 * n_union;
    if (V.prof && blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long pairs = 0;
        for (int i = 0; i < hdr->n; ++i)
            pairs += min((uint32_t)*items[i].old_count, list_cap) + min((uint32_t)*items[i].new_count, list_cap);
        atomicAdd(V.prof + 1, (unsigned long long)n_union);
        atomicAdd(V.prof + 2, pairs);
    }
    while (true) {
        uint32_t base = 0;
        if (lane == 0) base = (uint32_t)atomicAdd(&counters[1], grab);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_units) break;
        const uint32_t end = min(base + (uint32_t)grab, n_units);
        for (uint32_t unit = base; unit < end; ++unit) {
            const int32_t slot = ulist[unit >> 2];
            const int g = unit & 3;
            const int4 c = V.coord[slot];
            const bool fresh = (V.flags[slot] & FLAG_FRESH) != 0;
            const uint32_t* mp = masks + (size_t)slot * mw;
            const uint32_t mw0 = lane < mw ? mp[lane] : 0u;
            const uint32_t mw1 = lane + 32 < mw ? mp[lane + 32] : 0u;
            // items with a bit on this block bound every voxel's count of samples
            const int n_bits = (int)__reduce_add_sync(0xffffffffu, (unsigned)(__popc(mw0) + __popc(mw1)));
            if (n_bits <= PACK_MAX_ITEMS)
                nd_group<F32, NdAcc>(V, cams, n_items, slot, c, fresh, mw0, mw1, mw, lane, g);
            else
                nd_group<F32, NdAccWide>(V, cams, n_items, slot, c, fresh, mw0, mw1, mw, lane, g);
        }
    }
}

// After the net-delta update: zero the union slots' item bits and fresh flags, so
// the masks are all zero between calls.
__global__ void net_delta_clear_kernel(DevVolume V, uint32_t* masks, int mw, const int32_t* ulist,
                                       const int32_t* counters) {
    const uint32_t n_union = min((uint32_t)counters[0], V.max_blocks);
    const size_t n = (size_t)n_union * mw;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int32_t slot = ulist[i / mw];
        const int w = (int)(i % mw);
        masks[(size_t)slot * mw + w] = 0u;
        if (w == 0) V.flags[slot] = 0u;
    }
}

}  // namespace

struct BatchState {
    int mw = 0;
    int32_t* zero = nullptr;  // a device word holding 0: the old-list length of integrate-only items
    uint2* tex = nullptr;     // packed keyframe images [max_batch][tex_stride]
    uint32_t tex_px = 0;      // pixels per image
    uint32_t tex_stride = 0;  // texels per item: tex_px rounded up to even, plus one sentinel
    uint32_t* masks = nullptr;
    int32_t* ulist = nullptr;
    int32_t* counters = nullptr;
    // the call's header and item table travel as one block: STAGE_HDR bytes of header,
    // then the items; two pinned host copies alternate between calls, each guarded by an
    // event recorded after the launch that read it, so a call waits only for the launch
    // two calls back instead of synchronising the stream
    unsigned char* stage_d = nullptr;
    BatchHeader* hdr_d = nullptr;  // views into stage_d
    BatchItem* items_d = nullptr;
    unsigned char* stage_h[2] = {nullptr, nullptr};  // pinned
    cudaEvent_t staged[2] = {nullptr, nullptr};
    int buf = 0;  // staging copy of the next call
    // what each texel slot holds: the keyframe, its image pointers and image binding
    // count, and the image size, when a batch packed it
    struct PackedSlot {
        int32_t kf = -1;
        const float* depth = nullptr;
        const uint8_t* rgba = nullptr;
        uint32_t epoch = 0;
        uint32_t px = 0;
    };
    std::vector<PackedSlot> slots;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t items_node = nullptr;
    sc_batch_config graph_cfg{};
    DevVolume graph_dv{};
    int graph_f32 = 0;
};

void batch_destroy(sc_volume* V) {
    BatchState* B = V->batch;
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
    if (B->masks) cudaFree(B->masks);
    if (B->ulist) cudaFree(B->ulist);
    if (B->counters) cudaFree(B->counters);
    if (B->zero) cudaFree(B->zero);
    if (B->tex) cudaFree(B->tex);
    if (B->stage_d) cudaFree(B->stage_d);
    for (int k = 0; k < 2; ++k) {
        if (B->stage_h[k]) cudaFreeHost(B->stage_h[k]);
        if (B->staged[k]) cudaEventDestroy(B->staged[k]);
    }
    delete B;
    V->batch = nullptr;
}

namespace {

size_t nd_smem_bytes(sc_volume* V);

int batch_init(sc_volume* V) {
    if (V->batch) return SC_OK;
    BatchState* B = new BatchState();
    V->batch = B;
    B->mw = 2 * ((V->p.max_batch + 31) / 32);
    const size_t mbytes = (size_t)V->p.max_blocks * B->mw * sizeof(uint32_t);
    SC_CUDA(cudaMalloc((void**)&B->masks, mbytes));
    SC_CUDA(cudaMemset(B->masks, 0, mbytes));
    SC_CUDA(cudaMalloc((void**)&B->ulist, (size_t)V->p.max_blocks * sizeof(int32_t)));
    SC_CUDA(cudaMalloc((void**)&B->counters, 4 * sizeof(int32_t)));
    SC_CUDA(cudaMalloc((void**)&B->zero, sizeof(int32_t)));
    SC_CUDA(cudaMemset(B->zero, 0, sizeof(int32_t)));
    const size_t stage_bytes = STAGE_HDR + (size_t)V->p.max_batch * sizeof(BatchItem);
    SC_CUDA(cudaMalloc((void**)&B->stage_d, stage_bytes));
    B->hdr_d = reinterpret_cast<BatchHeader*>(B->stage_d);
    B->items_d = reinterpret_cast<BatchItem*>(B->stage_d + STAGE_HDR);
    for (int k = 0; k < 2; ++k) {
        SC_CUDA(cudaMallocHost((void**)&B->stage_h[k], stage_bytes));
        SC_CUDA(cudaEventCreateWithFlags(&B->staged[k], cudaEventDisableTiming));
    }
    SC_CUDA(cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
    const size_t smem = nd_smem_bytes(V);
    if (smem > 48 * 1024) {
        SC_CUDA(cudaFuncSetAttribute(net_delta_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        SC_CUDA(cudaFuncSetAttribute(net_delta_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    V->device_bytes += mbytes + (size_t)V->p.max_blocks * 4 + (size_t)V->p.max_batch * sizeof(BatchItem);
    return SC_OK;
}

size_t nd_smem_bytes(sc_volume* V) { return (size_t)2 * V->p.max_batch * sizeof(NdCam); }

int ctas_per_sm_clamped(sc_volume* V, const sc_batch_config& c) {
    int occ = 0;
    const int threads = 32 * c.warps_per_cta;
    const size_t smem = nd_smem_bytes(V);
    cudaError_t e = V->p.colour_format == SC_RGB_F32
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, net_delta_kernel<true>, threads, smem)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, net_delta_kernel<false>, threads, smem);
    if (e != cudaSuccess || occ < 1) occ = 1;
    return std::max(1, std::min(c.ctas_per_sm, occ));
}

// Enqueue steps 2-6 (and the item copy) on stream s; used for capture.
cudaError_t enqueue_batch(sc_volume* V, cudaStream_t s, cudaGraphNode_t* items_node) {
    BatchState* B = V->batch;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(B->stage_d, B->stage_h[0], STAGE_HDR + sizeof(BatchItem), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return e;
    if (items_node) {
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        if ((e = cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &ndeps)) != cudaSuccess)
            return e;
        if (ndeps != 1) return cudaErrorUnknown;
        *items_node = deps[0];
    }
    batch_pack_kernel<<<V->num_sms * 8, 256, 0, s>>>(B->items_d, B->hdr_d, B->tex, B->tex_px, B->tex_stride,
                                                     B->counters);
    if (V->prof_on) cudaEventRecordWithFlags(V->graph_ev[0], s, cudaEventRecordExternal);
    batch_alloc_kernel<<<V->num_sms * ALLOC_CTAS_PER_SM, ALLOC_THREADS, 0, s>>>(
        V->dv, B->items_d, B->hdr_d, B->masks, B->mw, B->ulist, B->counters, V->p.max_blocks_per_keyframe);
    if (V->prof_on) cudaEventRecordWithFlags(V->graph_ev[1], s, cudaEventRecordExternal);
    const int mark_y = std::min(V->p.max_batch, 1024);
    batch_mark_old_kernel<<<dim3(std::max(1, V->num_sms * 8 / mark_y), mark_y), 256, 0, s>>>(
        V->dv, B->items_d, B->hdr_d, B->masks, B->mw, B->ulist, B->counters, V->p.max_blocks_per_keyframe);
    if (V->prof_on) cudaEventRecordWithFlags(V->graph_ev[2], s, cudaEventRecordExternal);
    const sc_batch_config& c = V->bcfg;
    const int grid = V->num_sms * ctas_per_sm_clamped(V, c);
    const uint32_t cap = V->p.max_blocks_per_keyframe;
    if (V->p.colour_format == SC_RGB_F32)
        net_delta_kernel<true><<<grid, 32 * c.warps_per_cta, nd_smem_bytes(V), s>>>(
            V->dv, B->items_d, B->hdr_d, B->masks, B->mw, B->ulist, B->counters, c.blocks_per_grab, cap);
    else
        net_delta_kernel<false><<<grid, 32 * c.warps_per_cta, nd_smem_bytes(V), s>>>(
            V->dv, B->items_d, B->hdr_d, B->masks, B->mw, B->ulist, B->counters, c.blocks_per_grab, cap);
    if (V->prof_on) cudaEventRecordWithFlags(V->graph_ev[3], s, cudaEventRecordExternal);
    net_delta_clear_kernel<<<V->num_sms * 4, 256, 0, s>>>(V->dv, B->masks, B->mw, B->ulist, B->counters);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaMemcpyAsync(V->h_status, V->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
}

int ensure_graph(sc_volume* V) {
    BatchState* B = V->batch;
    const bool same = B->exec && !memcmp(&B->graph_cfg, &V->bcfg, sizeof(sc_batch_config)) &&
                      !memcmp(&B->graph_dv, &V->dv, sizeof(DevVolume));
    if (same) return SC_OK;
    // no launch of the old graph may still be in flight
    for (int k = 0; k < 2; ++k) SC_CUDA(cudaEventSynchronize(B->staged[k]));
    if (B->exec) {
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
    }
    if (B->graph) {
        cudaGraphDestroy(B->graph);
        B->graph = nullptr;
    }
    SC_CUDA(cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_batch(V, B->cap_stream, &B->items_node);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(B->cap_stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_status(e);
    }
    SC_CUDA(e2);
    B->graph = g;
    SC_CUDA(cudaGraphInstantiate(&B->exec, g, 0));
    B->graph_cfg = V->bcfg;
    B->graph_dv = V->dv;
    return SC_OK;
}

// One batch item as the host sees it; old == nullptr: integrate only (the keyframe is
// not integrated and has no old footprint).
struct ItemSpec {
    int32_t kf_id;
    const float* depth;
    const uint8_t* rgba;
    const sc_pose* oldp;
    const sc_pose* newp;
};

bool pose_finite(const sc_pose* p) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c)
            if (!std::isfinite(p->m[r][c])) return false;
    return true;
}

int prepare_specs(sc_volume* V, const ItemSpec* items, int32_t n, const sc_intrinsics* K) {
    if (!V || !items || n < 1 || n > V->p.max_batch || !intrinsics_ok(K)) return SC_ERR_INVALID_ARG;
    std::vector<uint8_t> seen(V->p.max_keyframes, 0);
    for (int i = 0; i < n; ++i) {
        const ItemSpec& it = items[i];
        if (it.kf_id < 0 || it.kf_id >= V->p.max_keyframes || seen[it.kf_id]) return SC_ERR_INVALID_ARG;
        if (!it.depth || !it.rgba || ((uintptr_t)it.depth & 15) || ((uintptr_t)it.rgba & 15))
            return SC_ERR_INVALID_ARG;
        if (!it.newp || !pose_finite(it.newp) || (it.oldp && !pose_finite(it.oldp))) return SC_ERR_INVALID_ARG;
        seen[it.kf_id] = 1;
        if (it.oldp && !V->integrated[it.kf_id]) return SC_ERR_NOT_INTEGRATED;
        if (it.oldp && V->nonresident[it.kf_id]) return SC_ERR_NOT_RESIDENT;
        if (!it.oldp && V->integrated[it.kf_id]) return SC_ERR_ALREADY_INTEGRATED;
    }
    int rc = batch_init(V);
    if (rc) return rc;
    BatchState* B = V->batch;
    const uint32_t npx = (uint32_t)K->width * (uint32_t)K->height;
    if (npx != B->tex_px) {
        // packed keyframe images for this image size; the graph captured the old buffer
        if (B->tex) cudaFree(B->tex);
        B->tex = nullptr;
        B->tex_px = 0;
        const uint32_t stride = (npx + 2) & ~1u;  // > npx, even: every item's texels 16-byte aligned
        SC_CUDA(cudaMalloc((void**)&B->tex, (size_t)V->p.max_batch * stride * sizeof(uint2)));
        B->tex_px = npx;
        B->tex_stride = stride;
        if (B->exec) {
            cudaGraphExecDestroy(B->exec);
            B->exec = nullptr;
        }
    }
    if (B->slots.size() != (size_t)V->p.max_batch) B->slots.assign(V->p.max_batch, BatchState::PackedSlot());
    // this call's staging copy: free once the launch two calls back has read it
    SC_CUDA(cudaEventSynchronize(B->staged[B->buf]));
    BatchHeader* hdr_h = reinterpret_cast<BatchHeader*>(B->stage_h[B->buf]);
    BatchItem* items_h = reinterpret_cast<BatchItem*>(B->stage_h[B->buf] + STAGE_HDR);
    int n_pack = 0;
    for (int i = 0; i < n; ++i) {
        const ItemSpec& it = items[i];
        BatchItem& b = items_h[i];
        const int cur = V->cur[it.kf_id];
        b.oldc = make_cam(V, K, it.oldp ? it.oldp : it.newp, it.depth, it.rgba);
        b.newc = make_cam(V, K, it.newp, it.depth, it.rgba);
        b.old_list = list_ptr(V, it.kf_id, cur);
        b.old_count = it.oldp ? count_ptr(V, it.kf_id, cur) : B->zero;
        b.new_list = list_ptr(V, it.kf_id, 1 - cur);
        b.new_count = count_ptr(V, it.kf_id, 1 - cur);
        b.oldc.tex = b.newc.tex = B->tex + (size_t)i * B->tex_stride;
        // a keyframe that is not integrated yet binds its images now; an integrated one
        // keeps the images of its integration (de-integration must use them), so a slot
        // packed from the same pointers under the same binding still holds them
        if (!it.oldp) ++V->img_epoch[it.kf_id];
        BatchState::PackedSlot& ps = B->slots[i];
        const bool packed = it.oldp && ps.kf == it.kf_id && ps.depth == it.depth && ps.rgba == it.rgba &&
                            ps.epoch == V->img_epoch[it.kf_id] && ps.px == B->tex_px;
        // items are written in order, so entry n_pack <= i is already filled
        if (!packed) items_h[n_pack++].pack_item = i;
        ps.kf = it.kf_id;
        ps.depth = it.depth;
        ps.rgba = it.rgba;
        ps.epoch = V->img_epoch[it.kf_id];
        ps.px = B->tex_px;
    }
    if (++V->call_id == 0) V->call_id = 1;  // (plain calls reset stamps on wrap)
    hdr_h->n = n;
    hdr_h->n_pack = n_pack;
    hdr_h->call_id = V->call_id;
    hdr_h->tiles_x = (K->width + ALLOC_TX - 1) / ALLOC_TX;
    hdr_h->tiles = hdr_h->tiles_x * ((K->height + ALLOC_TY - 1) / ALLOC_TY);
    rc = ensure_graph(V);
    if (rc) return rc;
    // point the table copy at this call's staging copy, sized to its n items
    SC_CUDA(cudaGraphExecMemcpyNodeSetParams1D(B->exec, B->items_node, B->stage_d, B->stage_h[B->buf],
                                               STAGE_HDR + (size_t)n * sizeof(BatchItem), cudaMemcpyHostToDevice));
    return SC_OK;
}

int prepare_items(sc_volume* V, const sc_reint_item* items, int32_t n, const sc_intrinsics* K) {
    if (!items || n < 1) return SC_ERR_INVALID_ARG;
    std::vector<ItemSpec> sp(n);
    for (int i = 0; i < n; ++i)
        sp[i] = ItemSpec{items[i].kf_id, items[i].depth, items[i].rgba, &items[i].old_pose, &items[i].new_pose};
    return prepare_specs(V, sp.data(), n, K);
}

constexpr int GRAPH_KERNELS = 5;  // pack (and counter reset), batched allocation, mark old, net-delta, clear

// Launch the prepared graph.  Asynchronous: device errors stay in the volume's sticky
// status word (sc_get_status); with profiling on, the call synchronises to read the
// graph's event times and returns the status as well.
int launch_batch(sc_volume* V, cudaStream_t s) {
    BatchState* B = V->batch;
    SC_CUDA(cudaGraphLaunch(B->exec, s));
    count_launches(GRAPH_KERNELS);
    SC_CUDA(cudaEventRecord(B->staged[B->buf], s));
    B->buf ^= 1;
    V->last_stream = s;
    if (!V->prof_on) return SC_OK;
    SC_CUDA(cudaStreamSynchronize(s));
    {
        float a = 0.f, b = 0.f, c = 0.f;
        if (cudaEventElapsedTime(&a, V->graph_ev[0], V->graph_ev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&b, V->graph_ev[1], V->graph_ev[2]) == cudaSuccess &&
            cudaEventElapsedTime(&c, V->graph_ev[2], V->graph_ev[3]) == cudaSuccess) {
            V->prof_ms[2] += a;
            V->prof_ms[3] += b;
            V->prof_ms[4] += c;
            V->prof_n[2] += 1;
        }
        (void)cudaGetLastError();
    }
    return *V->h_status;
}

}  // namespace

extern "C" int sc_reintegrate_batch(sc_volume* V, const sc_reint_item* items, int32_t n, const sc_intrinsics* K,
                                    sc_stream stream) {
    int rc = prepare_items(V, items, n, K);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = launch_batch(V, s);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) V->cur[items[i].kf_id] ^= 1;
    return SC_OK;
}

extern "C" int sc_integrate_keyframes(sc_volume* V, const int32_t* kf_ids, const float* const* depths,
                                      const uint8_t* const* rgbas, const sc_pose* poses, int32_t n,
                                      const sc_intrinsics* K, sc_stream stream) {
    if (!V || !kf_ids || !depths || !rgbas || !poses || n < 1) return SC_ERR_INVALID_ARG;
    std::vector<ItemSpec> sp(n);
    for (int i = 0; i < n; ++i) sp[i] = ItemSpec{kf_ids[i], depths[i], rgbas[i], nullptr, &poses[i]};
    int rc = prepare_specs(V, sp.data(), n, K);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = launch_batch(V, s);
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        V->cur[kf_ids[i]] ^= 1;
        V->integrated[kf_ids[i]] = 1;
    }
    return SC_OK;
}

extern "C" int sc_set_batch_config(sc_volume* V, const sc_batch_config* c) {
    if (!V || !c) return SC_ERR_INVALID_ARG;
    if (!(c->warps_per_cta == 2 || c->warps_per_cta == 4 || c->warps_per_cta == 8 || c->warps_per_cta == 16) ||
        c->ctas_per_sm < 1 || c->ctas_per_sm > 16 || c->blocks_per_grab < 1 || c->blocks_per_grab > 16)
        return SC_ERR_INVALID_ARG;
    V->bcfg = *c;
    return SC_OK;
}

extern "C" int sc_get_batch_config(sc_volume* V, sc_batch_config* c) {
    if (!V || !c) return SC_ERR_INVALID_ARG;
    *c = V->bcfg;
    return SC_OK;
}

// ------------------------------------------------------------------ autotune ----

namespace {

struct Snapshot {
    uint32_t used = 0;
    size_t col_bytes = 0;
    void* buf = nullptr;
    size_t bytes = 0;
};

int snapshot_take(sc_volume* V, Snapshot& S, cudaStream_t s) {
    SC_CUDA(cudaMemcpyAsync(V->h_word, V->pool_count, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    S.used = std::min(V->h_word[0], V->p.max_blocks);
    const size_t nb = S.used;
    S.col_bytes = nb * NVOX * (V->p.colour_format == SC_RGB_F32 ? 3 * sizeof(float) : sizeof(uint32_t));
    const size_t tbytes = (size_t)V->p.n_buckets * V->p.bucket_size * sizeof(HashEntry);
    S.bytes = 2 * nb * NVOX * sizeof(float) + S.col_bytes + nb * sizeof(uint32_t) + tbytes + 256;
    SC_CUDA(cudaMalloc(&S.buf, S.bytes));
    char* p = (char*)S.buf;
    SC_CUDA(cudaMemcpyAsync(p, V->D, nb * NVOX * sizeof(float), cudaMemcpyDeviceToDevice, s));
    p += nb * NVOX * sizeof(float);
    SC_CUDA(cudaMemcpyAsync(p, V->W, nb * NVOX * sizeof(float), cudaMemcpyDeviceToDevice, s));
    p += nb * NVOX * sizeof(float);
    SC_CUDA(cudaMemcpyAsync(p, V->Cf ? (void*)V->Cf : (void*)V->C8, S.col_bytes, cudaMemcpyDeviceToDevice, s));
    p += S.col_bytes;
    SC_CUDA(cudaMemcpyAsync(p, V->flags, nb * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    p += nb * sizeof(uint32_t);
    SC_CUDA(cudaMemcpyAsync(p, V->table, tbytes, cudaMemcpyDeviceToDevice, s));
    return SC_OK;
}

int snapshot_restore(sc_volume* V, const Snapshot& S, cudaStream_t s) {
    const size_t nb = S.used;
    const size_t tbytes = (size_t)V->p.n_buckets * V->p.bucket_size * sizeof(HashEntry);
    const char* p = (const char*)S.buf;
    SC_CUDA(cudaMemcpyAsync(V->D, p, nb * NVOX * sizeof(float), cudaMemcpyDeviceToDevice, s));
    p += nb * NVOX * sizeof(float);
    SC_CUDA(cudaMemcpyAsync(V->W, p, nb * NVOX * sizeof(float), cudaMemcpyDeviceToDevice, s));
    p += nb * NVOX * sizeof(float);
    SC_CUDA(cudaMemcpyAsync(V->Cf ? (void*)V->Cf : (void*)V->C8, p, S.col_bytes, cudaMemcpyDeviceToDevice, s));
    p += S.col_bytes;
    SC_CUDA(cudaMemcpyAsync(V->flags, p, nb * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    p += nb * sizeof(uint32_t);
    SC_CUDA(cudaMemcpyAsync(V->table, p, tbytes, cudaMemcpyDeviceToDevice, s));
    SC_CUDA(cudaMemcpyAsync(V->pool_count, &S.used, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    SC_CUDA(cudaMemsetAsync(V->status, 0, sizeof(int32_t), s));
    SC_CUDA(cudaStreamSynchronize(s));
    return SC_OK;
}

}  // namespace

extern "C" int sc_autotune_batch(sc_volume* V, const sc_reint_item* items, int32_t n, const sc_intrinsics* K,
                                 sc_stream stream, sc_batch_config* best, float* ms_out) {
    if (!V || !best) return SC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Snapshot S;
    int rc = snapshot_take(V, S, s);
    if (rc) {
        if (S.buf) cudaFree(S.buf);
        return rc;
    }
    const sc_batch_config orig = V->bcfg;
    std::vector<sc_batch_config> cands;
    for (int w : {4, 8})
        for (int c : {2, 4, 8})
            for (int g : {1, 4}) cands.push_back(sc_batch_config{w, c, g});
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    sc_batch_config best_cfg = orig;
    for (const sc_batch_config& c : cands) {
        V->bcfg = c;
        std::vector<float> ts;
        for (int rep = 0; rep < 4 && rc == SC_OK; ++rep) {
            rc = prepare_items(V, items, n, K);
            if (rc) break;
            cudaEventRecord(e0, s);
            rc = cuda_status(cudaGraphLaunch(V->batch->exec, s));
            count_launches(GRAPH_KERNELS);
            cudaEventRecord(e1, s);
            if (rc == SC_OK) rc = cuda_status(cudaStreamSynchronize(s));
            if (rc == SC_OK) rc = *V->h_status;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) ts.push_back(ms);  // first run warms up the graph
            const int rr = snapshot_restore(V, S, s);
            if (rc == SC_OK) rc = rr;
        }
        if (rc) break;
        std::sort(ts.begin(), ts.end());
        const float med = ts[ts.size() / 2];
        if (med < best_ms) {
            best_ms = med;
            best_cfg = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(S.buf);
    V->bcfg = rc ? orig : best_cfg;
    V->last_stream = s;
    if (rc) return rc;
    *best = best_cfg;
    if (ms_out) *ms_out = best_ms;
    return SC_OK;
}
