// The streaming sphere (Section 3 "SDF volume": only voxel blocks within a sphere
// of constant radius around the camera stay in GPU memory, the others are streamed
// to the host; Section 4.3 streams the spheres around T_j* and T'_j* in before a
// re-integration).
//
// A block is inside when its centre ((8 b + 3.5) * voxel_size per axis) is within
// the radius of the given point; the distance is computed in float, squared, with
// explicit round-to-nearest operations, the same on the device and the host.
//
// The host block store is pinned, device-mapped memory: the copy kernels read and
// write it directly (zero-copy over the host link, 16-byte accesses).
//
// Stream out: mark the resident blocks outside the sphere; copy them into the store
// (one warp per block); compact the pool (each resident block above the new pool
// size moves into a hole below it); rewrite every keyframe block list through a
// slot map (moved slot -> new slot, evicted slot -> external id -(e + 2), e the
// block's store entry); rebuild the hash table from the remaining blocks.
// Stream in: insert the stored blocks inside the sphere at new pool slots, copy them
// back, and rewrite list entries -(e + 2) to their new slots.  Keyframe lists hence
// always name each block of A(k, T) exactly once, resident or stored, and Eq. 2
// stays an exact inverse across streaming.
#include <algorithm>
#include <cmath>
#include <vector>

#include "alloc.cuh"
#include "volume.cuh"

struct sc_block_store {
    int device;
    int colour_f32;
    int64_t capacity;
    // pinned, device-mapped
    int4* coord;     // [cap]
    uint32_t* flags; // [cap]
    float* D;        // [cap][512]
    float* W;        // [cap][512]
    void* C;         // [cap][512] RGBA8 or [cap][3][512] float
    int32_t* ext;    // [cap] staging: store entries of one transfer
    int32_t* slot_out;  // [cap] staging: the pool slot each streamed-in entry got, or -1
    // device
    int32_t* ext2slot;  // [cap] store entry -> new pool slot during a stream-in, else -1
    uint32_t* mark;     // [cap] store entries named by the keyframes of one stream-in (0 between calls)
    int32_t* dlist;     // [cap] device list of those entries
    int32_t* dcount;    // [1]
    // device hash index of the stored blocks: block key -> store entry, open addressing
    // (icap = a power of two >= 2 cap entries; deleted entries become tombstones that
    // later inserts reuse)
    unsigned long long* ikey;  // [icap]
    int32_t* ival;             // [icap]
    uint32_t imask;            // icap - 1
    // host bookkeeping
    std::vector<int32_t> free_ids;
    std::vector<uint8_t> used;
    int64_t count;
};

namespace {

using namespace sc;

#define SC_CUDA_RC(call)          \
    do {                          \
        const int r_ = (call);    \
        if (r_ != SC_OK) return r_; \
    } while (0)

__host__ __device__ inline bool outside_sphere(int bx, int by, int bz, float s, float cx, float cy, float cz,
                                               float r2) {
#ifdef __CUDA_ARCH__
    const float dx = __fsub_rn(__fmul_rn(s, __fadd_rn((float)(8 * bx), 3.5f)), cx);
    const float dy = __fsub_rn(__fmul_rn(s, __fadd_rn((float)(8 * by), 3.5f)), cy);
    const float dz = __fsub_rn(__fmul_rn(s, __fadd_rn((float)(8 * bz), 3.5f)), cz);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)) > r2;
#else
    volatile float dx = s * ((float)(8 * bx) + 3.5f) - cx;  // volatile: no contraction on the host
    volatile float dy = s * ((float)(8 * by) + 3.5f) - cy;
    volatile float dz = s * ((float)(8 * bz) + 3.5f) - cz;
    volatile float xx = dx * dx, yy = dy * dy, zz = dz * dz;
    volatile float a = xx + yy;
    return a + zz > r2;
#endif
}

constexpr unsigned long long IDX_TOMB = ~1ull;  // a deleted index entry (never a block key)

// The store index's device view.
struct StoreIndex {
    unsigned long long* key;
    int32_t* val;
    uint32_t mask;
};

// Insert a stored block's key (keys are unique: a block is stored at most once).
__device__ inline void index_insert(const StoreIndex& I, unsigned long long key, int32_t e) {
    uint32_t h = hash_bucket(key, I.mask);
    for (uint32_t i = 0; i <= I.mask; ++i) {
        const unsigned long long k = I.key[h];
        if ((k == KEY_EMPTY || k == IDX_TOMB) && atomicCAS(&I.key[h], k, key) == k) {
            I.val[h] = e;
            return;
        }
        if (k != KEY_EMPTY && k != IDX_TOMB) h = (h + 1) & I.mask;  // occupied: next; lost a race: re-read
    }
}

// Store entry of a key, or -1.
__device__ inline int32_t index_find(const StoreIndex& I, unsigned long long key) {
    uint32_t h = hash_bucket(key, I.mask);
    for (uint32_t i = 0; i <= I.mask; ++i) {
        const unsigned long long k = I.key[h];
        if (k == key) return I.val[h];
        if (k == KEY_EMPTY) return -1;
        h = (h + 1) & I.mask;
    }
    return -1;
}

__device__ inline void index_remove(const StoreIndex& I, unsigned long long key) {
    uint32_t h = hash_bucket(key, I.mask);
    for (uint32_t i = 0; i <= I.mask; ++i) {
        const unsigned long long k = I.key[h];
        if (k == key) {
            I.key[h] = IDX_TOMB;
            return;
        }
        if (k == KEY_EMPTY) return;
        h = (h + 1) & I.mask;
    }
}

// copy one block's payload between two (slot-indexed) block arrays, one warp
__device__ __forceinline__ void copy_block(int lane, bool f32, const float* D0, const float* W0, const void* C0,
                                           size_t s0, float* D1, float* W1, void* C1, size_t s1) {
    for (int i = lane; i < NVOX / 4; i += 32) {
        reinterpret_cast<float4*>(D1 + s1 * NVOX)[i] = reinterpret_cast<const float4*>(D0 + s0 * NVOX)[i];
        reinterpret_cast<float4*>(W1 + s1 * NVOX)[i] = reinterpret_cast<const float4*>(W0 + s0 * NVOX)[i];
        if (f32) {
            for (int ch = 0; ch < 3; ++ch)
                reinterpret_cast<float4*>((float*)C1 + (3 * s1 + ch) * NVOX)[i] =
                    reinterpret_cast<const float4*>((const float*)C0 + (3 * s0 + ch) * NVOX)[i];
        } else {
            reinterpret_cast<uint4*>((uint32_t*)C1 + s1 * NVOX)[i] =
                reinterpret_cast<const uint4*>((const uint32_t*)C0 + s0 * NVOX)[i];
        }
    }
}

struct SoCounters {
    int32_t n_out, n_hole, n_move;
};

__global__ void so_mark_kernel(DevVolume V, uint32_t n, float s, float cx, float cy, float cz, float r2,
                               uint8_t* out, int32_t* ev, SoCounters* cnt, int32_t* remap) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int4 c = V.coord[i];
        const bool o = outside_sphere(c.x, c.y, c.z, s, cx, cy, cz, r2);
        out[i] = o;
        remap[i] = (int32_t)i;
        if (o) ev[atomicAdd(&cnt->n_out, 1)] = (int32_t)i;
    }
}

// evicted block i -> store entry ext[i]
__global__ void so_copy_out_kernel(DevVolume V, const int32_t* ev, const int32_t* ext, int32_t n_out, int4* st_coord,
                                   uint32_t* st_flags, float* st_D, float* st_W, void* st_C, int32_t* remap,
                                   StoreIndex I) {
    const int lane = threadIdx.x & 31, wpb = blockDim.x / 32;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < n_out; i += gridDim.x * wpb) {
        const int32_t slot = ev[i], e = ext[i];
        if (lane == 0) {
            const int4 c = V.coord[slot];
            st_coord[e] = c;
            st_flags[e] = V.flags[slot];
            remap[slot] = -(e + 2);
            index_insert(I, pack_key(c.x, c.y, c.z), e);
        }
        copy_block(lane, V.colour_f32 != 0, V.D, V.W, V.colour_f32 ? (const void*)V.Cf : (const void*)V.C8,
                   (size_t)slot, st_D, st_W, st_C, (size_t)e);
    }
}

// holes: evicted slots below n_live; movers: resident slots at or above n_live
__global__ void so_plan_kernel(uint32_t n, uint32_t n_live, const uint8_t* out, int32_t* holes, int32_t* movers,
                               SoCounters* cnt) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (i < n_live && out[i]) holes[atomicAdd(&cnt->n_hole, 1)] = (int32_t)i;
        if (i >= n_live && !out[i]) movers[atomicAdd(&cnt->n_move, 1)] = (int32_t)i;
    }
}

__global__ void so_move_kernel(DevVolume V, const int32_t* holes, const int32_t* movers, const SoCounters* cnt,
                               int32_t* remap) {
    const int lane = threadIdx.x & 31, wpb = blockDim.x / 32;
    const int k = cnt->n_move;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < k; i += gridDim.x * wpb) {
        const int32_t from = movers[i], to = holes[i];
        if (lane == 0) {
            V.coord[to] = V.coord[from];
            V.flags[to] = V.flags[from];
            V.stamp[to] = 0u;
            remap[from] = to;
        }
        void* C = V.colour_f32 ? (void*)V.Cf : (void*)V.C8;
        copy_block(lane, V.colour_f32 != 0, V.D, V.W, C, (size_t)from, V.D, V.W, C, (size_t)to);
    }
}

// every list entry 0 <= e < n becomes remap[e]
__global__ void remap_lists_kernel(int32_t* lists, const int32_t* counts, int n_lists, uint32_t cap,
                                   const int32_t* remap, uint32_t n) {
    for (int l = blockIdx.y; l < n_lists; l += gridDim.y) {
        const uint32_t m = min((uint32_t)counts[l], cap);
        int32_t* list = lists + (size_t)l * cap;
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
            const int32_t e = list[i];
            if (e >= 0 && (uint32_t)e < n) list[i] = remap[e];
        }
    }
}

// every list entry -(x + 2) whose store entry x was streamed in becomes its slot
__global__ void unmap_lists_kernel(int32_t* lists, const int32_t* counts, int n_lists, uint32_t cap,
                                   const int32_t* ext2slot) {
    for (int l = blockIdx.y; l < n_lists; l += gridDim.y) {
        const uint32_t m = min((uint32_t)counts[l], cap);
        int32_t* list = lists + (size_t)l * cap;
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
            const int32_t e = list[i];
            if (e <= -2) {
                const int32_t s = ext2slot[-e - 2];
                if (s >= 0) list[i] = s;
            }
        }
    }
}

__global__ void rehash_kernel(DevVolume V, uint32_t n_live) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_live; i += gridDim.x * blockDim.x) {
        const int4 c = V.coord[i];
        bool won;
        int32_t seen;
        const int e = hash_claim(V, pack_key(c.x, c.y, c.z), &won, &seen);
        if (e >= 0) atomicExch(&V.table[e].slot, (int32_t)i);
    }
}

__global__ void clear_table_kernel(HashEntry* t, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        t[i].key = KEY_EMPTY;
        t[i].slot = SLOT_PENDING;
        t[i].pad = 0;
    }
}

// stored entries ext[0..k) back into the pool
__global__ void si_copy_in_kernel(DevVolume V, const int32_t* ext, int32_t k, const int4* st_coord,
                                  const uint32_t* st_flags, const float* st_D, const float* st_W, const void* st_C,
                                  int32_t* ext2slot, int32_t* slot_out, StoreIndex I) {
    const int lane = threadIdx.x & 31, wpb = blockDim.x / 32;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < k; i += gridDim.x * wpb) {
        const int32_t e = ext[i];
        int32_t slot = -1;
        int h = -1;  // lane 0: the block's hash entry
        if (lane == 0) {
            const int4 c = st_coord[e];
            bool won;
            int32_t seen;
            h = hash_claim(V, pack_key(c.x, c.y, c.z), &won, &seen);
            if (h >= 0 && !won) {
                set_status(V.status, SC_ERR_CONFLICT);
            } else if (h >= 0) {
                const uint32_t s = atomicAdd(V.pool_count, 1u);
                if (s >= V.max_blocks) {
                    set_status(V.status, SC_ERR_POOL_FULL);
                    atomicExch(&V.table[h].slot, SLOT_FAILED);
                } else {
                    V.coord[s] = c;
                    V.flags[s] = st_flags[e];
                    V.stamp[s] = 0u;
                    slot = (int32_t)s;
                    index_remove(I, pack_key(c.x, c.y, c.z));
                }
            }
        }
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (lane == 0) slot_out[i] = slot;
        if (slot < 0) continue;
        void* C = V.colour_f32 ? (void*)V.Cf : (void*)V.C8;
        copy_block(lane, V.colour_f32 != 0, st_D, st_W, st_C, (size_t)e, V.D, V.W, C, (size_t)slot);
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            atomicExch(&V.table[h].slot, slot);  // publish only once the payload is in place
            ext2slot[e] = slot;
        }
    }
}

// flags[l] = 1 when list l names a stored block
__global__ void list_flags_kernel(const int32_t* lists, const int32_t* counts, int n_lists, uint32_t cap,
                                  uint8_t* flags) {
    for (int l = blockIdx.y; l < n_lists; l += gridDim.y) {
        const uint32_t m = min((uint32_t)counts[l], cap);
        const int32_t* list = lists + (size_t)l * cap;
        bool any = false;
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
            any |= list[i] < 0;
        if (__syncthreads_or(any) && threadIdx.x == 0) flags[l] = 1;
    }
}

// the store entries named (as -(e + 2)) by the given lists, each once
struct KfLists {
    const int32_t* list[64];
    const int32_t* count[64];
};
__global__ void collect_ext_kernel(KfLists L, int n_lists, uint32_t cap, uint32_t* mark, int32_t* out,
                                   int32_t* count) {
    for (int l = blockIdx.y; l < n_lists; l += gridDim.y) {
        const uint32_t m = min((uint32_t)*L.count[l], cap);
        for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
            const int32_t e = L.list[l][i];
            if (e <= -2 && atomicExch(&mark[-e - 2], 1u) == 0u) out[atomicAdd(count, 1)] = -e - 2;
        }
    }
}

// The stored blocks that allocating A(k, T) for cameras cams[0..n) would reach: the
// allocation's own tile walk (tile_collect), each unique key looked up in the store
// index; each entry found is listed once.  Persistent over (camera, tile).
__global__ void __launch_bounds__(ALLOC_THREADS, SC_ALLOC_CTAS_PER_SM) si_probe_kernel(
        DevVolume V, const KfCam* cams, int n, int tiles_x, int tiles, StoreIndex I, uint32_t* mark, int32_t* out,
        int32_t* count) {
    __shared__ AllocShared sh;
    for (int w = blockIdx.x; w < n * tiles; w += gridDim.x) {
        const int i = w / tiles, t = w - i * tiles;
        const KfCam& k = cams[i];
        const int tx = t % tiles_x, ty = t / tiles_x;
        const bool my_ovf = tile_collect<ALLOC_TY>(k, tx, ty, sh);
        const int3 ref = cam_block(k);
        auto hit = [&](unsigned long long key) {
            const int32_t e = index_find(I, key);
            if (e >= 0 && atomicExch(&mark[e], 1u) == 0u) out[atomicAdd(count, 1)] = e;
        };
        const int nk = min(sh.n_keys, SET_SIZE);
        for (int j = threadIdx.x; j < nk; j += ALLOC_THREADS) hit(key64_of(sh.uk[j], ref));
        if (sh.overflow == 2 || (sh.overflow != 0 && my_ovf))
            tile_overflow_blocks<ALLOC_TY>(V, k, tx, ty, sh, [&](int bx, int by, int bz) { hit(pack_key(bx, by, bz)); });
        __syncthreads();  // shared state is reused by the CTA's next tile
    }
}

__global__ void unmark_kernel(const int32_t* ext, int32_t k, uint32_t* mark) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) mark[ext[i]] = 0u;
}

__global__ void reset_ext2slot_kernel(const int32_t* ext, int32_t k, int32_t* ext2slot) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) ext2slot[ext[i]] = -1;
}

// device-side scratch of a stream-out: sized to the pool, allocated stream-ordered per call
struct SoScratch {
    uint8_t* out;
    int32_t *ev, *holes, *movers, *remap;
    SoCounters* cnt;
};

// Recompute which keyframes' current lists name stored blocks (host flags checked by
// the entry points before any launch).
int refresh_residency(sc_volume* V, cudaStream_t s) {
    const int n_lists = V->p.max_keyframes * 2;
    uint8_t* d = nullptr;
    SC_CUDA(cudaMallocAsync((void**)&d, n_lists, s));
    SC_CUDA(cudaMemsetAsync(d, 0, n_lists, s));
    dim3 grid(std::max(1, std::min(64, (int)((V->p.max_blocks_per_keyframe + 255) / 256))), std::min(n_lists, 1024));
    list_flags_kernel<<<grid, 256, 0, s>>>(V->lists, V->list_counts, n_lists, V->p.max_blocks_per_keyframe, d);
    count_launches(1);
    SC_CUDA(cudaGetLastError());
    std::vector<uint8_t> h(n_lists);
    SC_CUDA(cudaMemcpyAsync(h.data(), d, n_lists, cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    cudaFreeAsync(d, s);
    for (int k = 0; k < V->p.max_keyframes; ++k) V->nonresident[k] = V->integrated[k] && h[2 * k + V->cur[k]];
    return SC_OK;
}

int lists_launch_shape(sc_volume* V, dim3* grid) {
    const int n_lists = V->p.max_keyframes * 2;
    *grid = dim3(std::max(1, std::min(64, (int)((V->p.max_blocks_per_keyframe + 255) / 256))),
                 std::min(n_lists, 1024));
    return n_lists;
}

}  // namespace

extern "C" int sc_create_block_store(int64_t capacity, int32_t colour_format, sc_block_store** out) {
    if (!out || capacity < 1 || capacity > (1ll << 26) || (colour_format != SC_RGBA8 && colour_format != SC_RGB_F32))
        return SC_ERR_INVALID_ARG;
    *out = nullptr;
    sc_block_store* S = new (std::nothrow) sc_block_store();
    if (!S) return SC_ERR_INVALID_ARG;
    SC_CUDA(cudaGetDevice(&S->device));
    S->colour_f32 = colour_format == SC_RGB_F32;
    S->capacity = capacity;
    const size_t cap = (size_t)capacity;
    auto halloc = [&](void** p, size_t bytes) { return cudaHostAlloc(p, bytes, cudaHostAllocMapped); };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = halloc((void**)&S->coord, cap * sizeof(int4));
    if (e == cudaSuccess) e = halloc((void**)&S->flags, cap * sizeof(uint32_t));
    if (e == cudaSuccess) e = halloc((void**)&S->D, cap * NVOX * sizeof(float));
    if (e == cudaSuccess) e = halloc((void**)&S->W, cap * NVOX * sizeof(float));
    if (e == cudaSuccess) e = halloc(&S->C, cap * NVOX * (S->colour_f32 ? 3 * sizeof(float) : sizeof(uint32_t)));
    if (e == cudaSuccess) e = halloc((void**)&S->ext, cap * sizeof(int32_t));
    if (e == cudaSuccess) e = halloc((void**)&S->slot_out, cap * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&S->ext2slot, cap * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(S->ext2slot, 0xff, cap * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&S->mark, cap * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(S->mark, 0, cap * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&S->dlist, cap * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&S->dcount, sizeof(int32_t));
    size_t icap = 1024;
    while (icap < 2 * cap) icap *= 2;
    S->imask = (uint32_t)(icap - 1);
    if (e == cudaSuccess) e = cudaMalloc((void**)&S->ikey, icap * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(S->ikey, 0xff, icap * sizeof(unsigned long long));  // KEY_EMPTY
    if (e == cudaSuccess) e = cudaMalloc((void**)&S->ival, icap * sizeof(int32_t));
    if (e != cudaSuccess) {
        sc_destroy_block_store(S);
        return cuda_status(e);
    }
    S->free_ids.resize(cap);
    for (size_t i = 0; i < cap; ++i) S->free_ids[i] = (int32_t)(cap - 1 - i);  // pop_back gives 0, 1, ...
    S->used.assign(cap, 0);
    S->count = 0;
    *out = S;
    return SC_OK;
}

extern "C" int sc_destroy_block_store(sc_block_store* S) {
    if (!S) return SC_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    if (S->coord) cudaFreeHost(S->coord);
    if (S->flags) cudaFreeHost(S->flags);
    if (S->D) cudaFreeHost(S->D);
    if (S->W) cudaFreeHost(S->W);
    if (S->C) cudaFreeHost(S->C);
    if (S->ext) cudaFreeHost(S->ext);
    if (S->slot_out) cudaFreeHost(S->slot_out);
    if (S->ext2slot) cudaFree(S->ext2slot);
    if (S->mark) cudaFree(S->mark);
    if (S->dlist) cudaFree(S->dlist);
    if (S->dcount) cudaFree(S->dcount);
    if (S->ikey) cudaFree(S->ikey);
    if (S->ival) cudaFree(S->ival);
    delete S;
    return SC_OK;
}

extern "C" int64_t sc_block_store_count(const sc_block_store* S) { return S ? S->count : -1; }

extern "C" int sc_stream_out(sc_volume* V, sc_block_store* S, const float* centre, float radius, int64_t* n_moved,
                             sc_stream stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!V || !S || !centre || !(radius >= 0.f) || !n_moved) return SC_ERR_INVALID_ARG;
    if (!std::isfinite(centre[0]) || !std::isfinite(centre[1]) || !std::isfinite(centre[2])) return SC_ERR_INVALID_ARG;
    if (S->colour_f32 != (V->p.colour_format == SC_RGB_F32) || S->device != V->device) return SC_ERR_INVALID_ARG;
    SC_CUDA(cudaSetDevice(V->device));
    *n_moved = 0;
    SC_CUDA(cudaMemcpyAsync(V->h_word, V->pool_count, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    const uint32_t n = std::min(V->h_word[0], V->p.max_blocks);
    if (n == 0) return read_status(V, s);
    SoScratch X{};
    SC_CUDA(cudaMallocAsync((void**)&X.out, n, s));
    SC_CUDA(cudaMallocAsync((void**)&X.ev, (size_t)n * 4, s));
    SC_CUDA(cudaMallocAsync((void**)&X.holes, (size_t)n * 4, s));
    SC_CUDA(cudaMallocAsync((void**)&X.movers, (size_t)n * 4, s));
    SC_CUDA(cudaMallocAsync((void**)&X.remap, (size_t)n * 4, s));
    SC_CUDA(cudaMallocAsync((void**)&X.cnt, sizeof(SoCounters), s));
    SC_CUDA(cudaMemsetAsync(X.cnt, 0, sizeof(SoCounters), s));
    const float r2 = std::isinf(radius) ? INFINITY : radius * radius;
    const int grid = V->num_sms * 8;
    so_mark_kernel<<<grid, 256, 0, s>>>(V->dv, n, V->p.voxel_size, centre[0], centre[1], centre[2], r2, X.out, X.ev,
                                        X.cnt, X.remap);
    count_launches(1);
    SC_CUDA(cudaGetLastError());
    SoCounters hc;
    SC_CUDA(cudaMemcpyAsync(&hc, X.cnt, sizeof(hc), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    const int32_t n_out = hc.n_out;
    int rc = SC_OK;
    if (n_out > 0) {
        if ((size_t)n_out > S->free_ids.size()) {
            rc = SC_ERR_CAPACITY;
        } else {
            for (int32_t i = 0; i < n_out; ++i) {
                const int32_t e = S->free_ids.back();
                S->free_ids.pop_back();
                S->ext[i] = e;
                S->used[e] = 1;
            }
            S->count += n_out;
            const uint32_t n_live = n - (uint32_t)n_out;
            const int wgrid = std::min((n_out + 7) / 8, V->num_sms * 16);
            so_copy_out_kernel<<<wgrid, 256, 0, s>>>(V->dv, X.ev, S->ext, n_out, S->coord, S->flags, S->D, S->W, S->C,
                                                     X.remap, StoreIndex{S->ikey, S->ival, S->imask});
            so_plan_kernel<<<grid, 256, 0, s>>>(n, n_live, X.out, X.holes, X.movers, X.cnt);
            so_move_kernel<<<wgrid, 256, 0, s>>>(V->dv, X.holes, X.movers, X.cnt, X.remap);
            dim3 lg;
            const int n_lists = lists_launch_shape(V, &lg);
            remap_lists_kernel<<<lg, 256, 0, s>>>(V->lists, V->list_counts, n_lists, V->p.max_blocks_per_keyframe,
                                                  X.remap, n);
            const size_t nent = (size_t)V->dv.bucket_mask + 1;
            clear_table_kernel<<<grid, 256, 0, s>>>(V->table, nent * V->p.bucket_size);
            if (n_live > 0) rehash_kernel<<<grid, 256, 0, s>>>(V->dv, n_live);
            count_launches(n_live > 0 ? 6 : 5);
            SC_CUDA(cudaGetLastError());
            V->h_word[1] = n_live;
            SC_CUDA(cudaMemcpyAsync(V->pool_count, V->h_word + 1, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
            *n_moved = n_out;
        }
    }
    cudaFreeAsync(X.out, s);
    cudaFreeAsync(X.ev, s);
    cudaFreeAsync(X.holes, s);
    cudaFreeAsync(X.movers, s);
    cudaFreeAsync(X.remap, s);
    cudaFreeAsync(X.cnt, s);
    if (*n_moved > 0) SC_CUDA_RC(refresh_residency(V, s));
    const int st = read_status(V, s);
    return rc ? rc : st;
}

namespace {

// Stream in the store entries S->ext[0..k) (k > 0), then update lists, residency
// flags and the store's bookkeeping.
int stream_in_entries(sc_volume* V, sc_block_store* S, int32_t k, int64_t* n_moved, cudaStream_t s) {
    const int wgrid = std::min((k + 7) / 8, V->num_sms * 16);
    si_copy_in_kernel<<<wgrid, 256, 0, s>>>(V->dv, S->ext, k, S->coord, S->flags, S->D, S->W, S->C, S->ext2slot,
                                            S->slot_out, StoreIndex{S->ikey, S->ival, S->imask});
    dim3 lg;
    const int n_lists = lists_launch_shape(V, &lg);
    unmap_lists_kernel<<<lg, 256, 0, s>>>(V->lists, V->list_counts, n_lists, V->p.max_blocks_per_keyframe,
                                          S->ext2slot);
    reset_ext2slot_kernel<<<std::min((k + 255) / 256, 1024), 256, 0, s>>>(S->ext, k, S->ext2slot);
    count_launches(3);
    SC_CUDA(cudaGetLastError());
    SC_CUDA_RC(refresh_residency(V, s));
    const int st = read_status(V, s);  // synchronises: slot_out is final
    // entries that reached the pool leave the store; the others (a conflict, a full
    // pool) stay stored and their list entries stay external
    int64_t moved = 0;
    for (int32_t i = 0; i < k; ++i) {
        if (S->slot_out[i] < 0) continue;
        S->used[S->ext[i]] = 0;
        S->free_ids.push_back(S->ext[i]);
        ++moved;
    }
    S->count -= moved;
    *n_moved = moved;
    return st;
}

bool stream_args_ok(sc_volume* V, sc_block_store* S) {
    return V && S && S->colour_f32 == (V->p.colour_format == SC_RGB_F32) && S->device == V->device;
}

// Stream in the S->dcount entries collected in S->dlist (marked in S->mark): copy the
// list to the host staging, clear the marks, move the blocks.
int stream_in_collected(sc_volume* V, sc_block_store* S, int64_t* n_moved, cudaStream_t s) {
    int32_t k = 0;
    SC_CUDA(cudaMemcpyAsync(&k, S->dcount, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    if (k == 0) return read_status(V, s);
    SC_CUDA(cudaMemcpyAsync(S->ext, S->dlist, (size_t)k * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    unmark_kernel<<<std::min((k + 255) / 256, 1024), 256, 0, s>>>(S->dlist, k, S->mark);
    count_launches(1);
    SC_CUDA(cudaGetLastError());
    SC_CUDA(cudaStreamSynchronize(s));
    return stream_in_entries(V, S, k, n_moved, s);
}

}  // namespace

extern "C" int sc_stream_in(sc_volume* V, sc_block_store* S, const float* centre, float radius, int64_t* n_moved,
                            sc_stream stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!stream_args_ok(V, S) || !centre || !(radius >= 0.f) || !n_moved) return SC_ERR_INVALID_ARG;
    if (!std::isfinite(centre[0]) || !std::isfinite(centre[1]) || !std::isfinite(centre[2])) return SC_ERR_INVALID_ARG;
    SC_CUDA(cudaSetDevice(V->device));
    *n_moved = 0;
    SC_CUDA(cudaStreamSynchronize(s));  // the store's entries are final on the host
    const float r2 = std::isinf(radius) ? INFINITY : radius * radius;
    int32_t k = 0;
    for (int64_t e = 0; e < S->capacity; ++e) {
        if (!S->used[e]) continue;
        const int4 c = S->coord[e];
        if (!outside_sphere(c.x, c.y, c.z, V->p.voxel_size, centre[0], centre[1], centre[2], r2))
            S->ext[k++] = (int32_t)e;
    }
    if (k == 0) return read_status(V, s);
    return stream_in_entries(V, S, k, n_moved, s);
}

extern "C" int sc_stream_in_keyframes(sc_volume* V, sc_block_store* S, const int32_t* kf_ids, int32_t n,
                                      int64_t* n_moved, sc_stream stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!stream_args_ok(V, S) || !kf_ids || n < 0 || !n_moved) return SC_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (kf_ids[i] < 0 || kf_ids[i] >= V->p.max_keyframes) return SC_ERR_INVALID_ARG;
    SC_CUDA(cudaSetDevice(V->device));
    *n_moved = 0;
    SC_CUDA(cudaMemsetAsync(S->dcount, 0, sizeof(int32_t), s));
    for (int i0 = 0; i0 < n; i0 += 64) {
        KfLists L;
        int m = 0;
        for (int i = i0; i < n && i < i0 + 64; ++i) {
            const int kf = kf_ids[i];
            if (!V->integrated[kf] || !V->nonresident[kf]) continue;
            L.list[m] = list_ptr(V, kf, V->cur[kf]);
            L.count[m] = count_ptr(V, kf, V->cur[kf]);
            ++m;
        }
        if (m == 0) continue;
        const dim3 grid(std::max(1, std::min(64, (int)((V->p.max_blocks_per_keyframe + 255) / 256))), m);
        collect_ext_kernel<<<grid, 256, 0, s>>>(L, m, V->p.max_blocks_per_keyframe, S->mark, S->dlist, S->dcount);
        count_launches(1);
        SC_CUDA(cudaGetLastError());
    }
    return stream_in_collected(V, S, n_moved, s);
}

extern "C" int sc_stream_in_poses(sc_volume* V, sc_block_store* S, const float* const* depths, const sc_pose* poses,
                                  int32_t n, const sc_intrinsics* K, int64_t* n_moved, sc_stream stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!stream_args_ok(V, S) || n < 0 || (n > 0 && (!depths || !poses)) || !intrinsics_ok(K) || !n_moved)
        return SC_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (!depths[i]) return SC_ERR_INVALID_ARG;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 4; ++c)
                if (!std::isfinite(poses[i].m[r][c])) return SC_ERR_INVALID_ARG;
    }
    SC_CUDA(cudaSetDevice(V->device));
    *n_moved = 0;
    if (n == 0 || S->count == 0) return read_status(V, s);
    std::vector<KfCam> h(n);
    for (int i = 0; i < n; ++i) h[i] = make_cam(V, K, &poses[i], depths[i], nullptr);
    KfCam* d = nullptr;
    SC_CUDA(cudaMallocAsync((void**)&d, n * sizeof(KfCam), s));
    SC_CUDA(cudaMemcpyAsync(d, h.data(), n * sizeof(KfCam), cudaMemcpyHostToDevice, s));
    SC_CUDA(cudaMemsetAsync(S->dcount, 0, sizeof(int32_t), s));
    const int tiles_x = (K->width + ALLOC_TX - 1) / ALLOC_TX;
    const int tiles = tiles_x * ((K->height + ALLOC_TY - 1) / ALLOC_TY);
    si_probe_kernel<<<V->num_sms * SC_ALLOC_CTAS_PER_SM, ALLOC_THREADS, 0, s>>>(
        V->dv, d, n, tiles_x, tiles, StoreIndex{S->ikey, S->ival, S->imask}, S->mark, S->dlist, S->dcount);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(d, s);
    SC_CUDA(e);
    return stream_in_collected(V, S, n_moved, s);
}
