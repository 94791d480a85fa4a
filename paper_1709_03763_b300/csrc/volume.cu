// Voxel-hashed TSDF volume: creation, block allocation, integration (running
// weighted average, Section 3 "SDF volume"), de-integration (Eq. 2, Section 4.3)
// and block-list extraction.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>

#include "alloc.cuh"
#include "volume.cuh"

using namespace sc;

#include <atomic>

namespace {
std::atomic<uint64_t> g_launches{0};
}

extern "C" uint64_t sc_kernel_launches(void) { return g_launches.load(); }

namespace sc {

void count_launches(uint64_t n) { g_launches += n; }

int cuda_status(cudaError_t e) {
    (void)cudaGetLastError();
    return e == cudaSuccess ? SC_OK : SC_ERR_CUDA;
}

bool intrinsics_ok(const sc_intrinsics* K) {
    return K && K->width > 0 && K->height > 0 && K->width <= 16384 && K->height <= 16384 && K->fx > 0.f &&
           K->fy > 0.f && std::isfinite(K->cx) && std::isfinite(K->cy);
}

KfCam make_cam(const sc_volume* V, const sc_intrinsics* K, const sc_pose* T, const float* depth,
               const uint8_t* rgba) {
    KfCam c;
    const double s = (double)V->p.voxel_size;
    double R[3][3], t[3];
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) R[r][q] = (double)T->m[r][q];
        t[r] = (double)T->m[r][3];
    }
    const double fk[3] = {(double)K->fx, (double)K->fy, 1.0};
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            c.Pr[r * 3 + q] = (float)(fk[r] * s * R[q][r]);  // diag(fx, fy, 1) s R^T
            c.Ms[r * 3 + q] = (float)(R[r][q] / s);          // R / s
        }
    for (int a = 0; a < 3; ++a) {
        const double tv = t[a] / s;
        const double fl = std::floor(tv);
        c.ti[a] = (int)fl;
        c.tiF[a] = (float)fl;
        c.tf[a] = (float)(tv - fl);
    }
    c.fx = K->fx;
    c.fy = K->fy;
    c.cx = K->cx;
    c.cy = K->cy;
    c.cxh = (float)((double)K->cx + 0.5);
    c.cyh = (float)((double)K->cy + 0.5);
    c.cxyh = make_float2(c.cxh, c.cyh);
    for (int q = 0; q < 3; ++q) {
        c.Pxy[q] = make_float2(c.Pr[q], c.Pr[3 + q]);
        c.Pz[q] = c.Pr[6 + q];
    }
    c.ifx = (float)(1.0 / (double)K->fx);
    c.ify = (float)(1.0 / (double)K->fy);
    c.W = K->width;
    c.H = K->height;
    c.mu = V->p.trunc;
    c.depth = depth;
    c.rgba = (const uint32_t*)rgba;
    c.tex = nullptr;
    return c;
}

int read_status(sc_volume* V, cudaStream_t s) {
    SC_CUDA(cudaMemcpyAsync(V->h_status, V->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    return *V->h_status;
}

cudaEvent_t prof_mark(sc_volume* V, cudaStream_t s) {
    if (!V->prof_on) return nullptr;
    cudaEvent_t e = nullptr;
    if (!V->ev_free.empty()) {
        e = V->ev_free.back();
        V->ev_free.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return nullptr;
    }
    cudaEventRecord(e, s);
    return e;
}

void prof_pair(sc_volume* V, cudaEvent_t a, cudaEvent_t b, int kind) {
    if (a && b) V->ev_pending.push_back({a, b, kind});
}

}  // namespace sc

// =============================================================== allocation ====

namespace {

// Plain path: one CTA per 32x32 pixel tile of one keyframe.
__global__ void __launch_bounds__(ALLOC_THREADS, SC_ALLOC_CTAS_PER_SM) alloc_kernel(DevVolume V, KfCam k, PlainSink sk) {
    __shared__ AllocShared sh;
    alloc_tile<ALLOC_TY_PLAIN>(V, k, blockIdx.x, blockIdx.y, sk, sh);
}

// =================================================================== update ====

constexpr int UPD_THREADS = 128;  // one CTA (4 warps) per 8^3 block; a thread owns 4 voxels

// Thread t of the CTA owns voxels 4t .. 4t+3 of the block (one float4 of each
// field).  The four samples are computed first; the thread's D / W / C are only
// read and written when one of its voxels is updated (or the block is fresh and
// must be zero-initialised).  Persistent: CTAs stride over the list.
template <int SIGN, bool F32>
__global__ void __launch_bounds__(UPD_THREADS) update_kernel(DevVolume V, KfCam k, const int32_t* list,
                                                             const int32_t* count_ptr, uint32_t cap) {
    const int t = threadIdx.x;
    const uint32_t n = min((uint32_t)*count_ptr, cap);
    if (V.prof && blockIdx.x == 0 && t == 0) atomicAdd(V.prof, (unsigned long long)n);
    const int lx0 = (4 * t) & 7, ly = ((4 * t) >> 3) & 7, lz = (4 * t) >> 6;
    for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
        const int32_t slot = list[i];
        if (slot < 0) {  // streamed out to the host block store
            if (t == 0) set_status(V.status, SC_ERR_NOT_RESIDENT);
            continue;
        }
        const int4 c = V.coord[slot];
        bool fresh = false;
        if (SIGN > 0) {
            fresh = (V.flags[slot] & FLAG_FRESH) != 0;
            __syncthreads();  // every thread has read the flag before it is cleared
            if (fresh && t == 0) V.flags[slot] = 0;
        }
        Proj4 P;
        project4(k, (float)(8 * c.x + lx0), (float)(8 * c.y + ly), (float)(8 * c.z + lz), P);
        float Z[4], d[4], eta;
#pragma unroll
        for (int j = 0; j < 4; ++j) Z[j] = P.ok[j] ? __ldg(k.depth + P.pix[j]) : 0.f;
        bool up[4];
        bool any = false;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            up[j] = decide(k, P.ok[j], Z[j], P.pz[j], d[j], eta);
            any |= up[j];
        }
        if (!any && !fresh) continue;
        uint32_t cc[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) cc[j] = up[j] ? __ldg(k.rgba + P.pix[j]) : 0u;
        const size_t off = (size_t)slot * NVOX + 4 * t;
        float4 Dv = make_float4(0.f, 0.f, 0.f, 0.f), Wv = Dv;
        if (!fresh) {
            Dv = *reinterpret_cast<const float4*>(V.D + off);
            Wv = *reinterpret_cast<const float4*>(V.W + off);
        }
        float* Dp = &Dv.x;
        float* Wp = &Wv.x;
        if (F32) {
            const size_t cb = (size_t)slot * 3 * NVOX + 4 * t;
            float4 Cv[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch)
                Cv[ch] = fresh ? make_float4(0.f, 0.f, 0.f, 0.f)
                               : *reinterpret_cast<const float4*>(V.Cf + cb + ch * NVOX);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!up[j]) continue;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch)
                    (&Cv[ch].x)[j] = update_cf((&Cv[ch].x)[j], Wp[j], (float)((cc[j] >> (8 * ch)) & 255u), SIGN);
                update_dw(Dp[j], Wp[j], d[j], SIGN);
            }
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) *reinterpret_cast<float4*>(V.Cf + cb + ch * NVOX) = Cv[ch];
        } else {
            uint4 Cv = make_uint4(0u, 0u, 0u, 0u);
            if (!fresh) Cv = *reinterpret_cast<const uint4*>(V.C8 + off);
            uint32_t* Cp = &Cv.x;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!up[j]) continue;
                Cp[j] = update_c8(Cp[j], Wp[j], cc[j], SIGN);
                update_dw(Dp[j], Wp[j], d[j], SIGN);
            }
            *reinterpret_cast<uint4*>(V.C8 + off) = Cv;
        }
        *reinterpret_cast<float4*>(V.D + off) = Dv;
        *reinterpret_cast<float4*>(V.W + off) = Wv;
    }
}

// ============================================================== extraction ====

constexpr int EXTRACT_THREADS = 256;
constexpr int EXTRACT_PER = 4;  // hash entries per thread and round

__global__ void __launch_bounds__(EXTRACT_THREADS) extract_kernel(DevVolume V, uint32_t n_entries, int32_t* coords,
                                                                  int32_t* slots, int32_t* tmp, uint32_t* count,
                                                                  uint32_t cap) {
    // each round a CTA takes 1024 consecutive entries (warp w: 128 of them, four 16-byte
    // loads per lane, all requested before any is examined); the CTA's occupied entries
    // get their output positions from one atomic add per CTA and round
    __shared__ uint32_t wbase[EXTRACT_THREADS / 32];
    __shared__ uint32_t cta_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr uint32_t PER_CTA = EXTRACT_THREADS * EXTRACT_PER;
    const uint4* tab = reinterpret_cast<const uint4*>(V.table);
    for (uint32_t cb = blockIdx.x * PER_CTA; cb < n_entries; cb += gridDim.x * PER_CTA) {  // uniform in the CTA
        uint4 ent[EXTRACT_PER];
#pragma unroll
        for (int j = 0; j < EXTRACT_PER; ++j) {
            const uint32_t e = cb + warp * 32 * EXTRACT_PER + 32 * j + lane;
            ent[j] = e < n_entries ? __ldg(tab + e) : make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0u);
        }
        bool ok[EXTRACT_PER];
        unsigned m[EXTRACT_PER];
        uint32_t wc = 0;
#pragma unroll
        for (int j = 0; j < EXTRACT_PER; ++j) {
            const unsigned long long key = (unsigned long long)ent[j].x | ((unsigned long long)ent[j].y << 32);
            ok[j] = key != KEY_EMPTY && (int32_t)ent[j].z >= 0;
            m[j] = __ballot_sync(0xffffffffu, ok[j]);
            wc += (uint32_t)__popc(m[j]);
        }
        if (lane == 0) wbase[warp] = wc;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < EXTRACT_THREADS / 32; ++w) {
                const uint32_t c = wbase[w];
                wbase[w] = t;
                t += c;
            }
            cta_base = t ? atomicAdd(count, t) : 0u;
        }
        __syncthreads();
        uint32_t b = cta_base + wbase[warp];
#pragma unroll
        for (int j = 0; j < EXTRACT_PER; ++j) {
            const uint32_t i = b + (uint32_t)__popc(m[j] & ((1u << lane) - 1u));
            b += (uint32_t)__popc(m[j]);
            if (!ok[j] || i >= cap) continue;
            const unsigned long long key = (unsigned long long)ent[j].x | ((unsigned long long)ent[j].y << 32);
            const int3 c = unpack_key(key);
            if (coords) {
                coords[3 * i] = c.x;
                coords[3 * i + 1] = c.y;
                coords[3 * i + 2] = c.z;
            }
            const int32_t slot = (int32_t)ent[j].z;
            if (slots) slots[i] = slot;
            tmp[i] = slot;
        }
        __syncthreads();  // wbase and cta_base are rewritten by the next round
    }
}

// Copy voxel payloads of the first n extracted blocks (one warp per block).
__global__ void gather_payload_kernel(DevVolume V, const int32_t* tmp, uint32_t n, float* D, float* W, void* C) {
    const int lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const size_t src = (size_t)tmp[i] * NVOX, dst = (size_t)i * NVOX;
        for (int g = 0; g < 4; ++g) {
            const int o = 4 * lane + 128 * g;
            if (D) *reinterpret_cast<float4*>(D + dst + o) = *reinterpret_cast<const float4*>(V.D + src + o);
            if (W) *reinterpret_cast<float4*>(W + dst + o) = *reinterpret_cast<const float4*>(V.W + src + o);
            if (C) {
                if (V.colour_f32) {
                    float* Co = (float*)C + dst * 3;
                    const float* Ci = V.Cf + src * 3;
                    for (int j = 0; j < 4; ++j)
                        for (int ch = 0; ch < 3; ++ch) Co[3 * (o + j) + ch] = Ci[ch * NVOX + o + j];
                } else {
                    *reinterpret_cast<uint4*>((uint32_t*)C + dst + o) =
                        *reinterpret_cast<const uint4*>(V.C8 + src + o);
                }
            }
        }
    }
}

__global__ void reset_table_kernel(HashEntry* t, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        t[i].key = KEY_EMPTY;
        t[i].slot = SLOT_PENDING;
        t[i].pad = 0;
    }
}

int grid_for(sc_volume* V, int per_sm) { return V->num_sms * per_sm; }

}  // namespace

namespace sc {

cudaError_t launch_alloc(sc_volume* V, const KfCam& cam, int32_t* list, int32_t* count, uint32_t call_id,
                         cudaStream_t s) {
    dim3 grid((cam.W + ALLOC_TX - 1) / ALLOC_TX, (cam.H + ALLOC_TY_PLAIN - 1) / ALLOC_TY_PLAIN);
    PlainSink sk{V->stamp, call_id, list, count, V->p.max_blocks_per_keyframe, nullptr, nullptr, 0};
    alloc_kernel<<<grid, ALLOC_THREADS, 0, s>>>(V->dv, cam, sk);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_update(sc_volume* V, const KfCam& cam, const int32_t* list, const int32_t* count, int sign,
                          cudaStream_t s) {
    const int grid = grid_for(V, 16);  // 16 x 4 warps per SM, persistent over the list
    const uint32_t cap = V->p.max_blocks_per_keyframe;
    const bool f32 = V->p.colour_format == SC_RGB_F32;
    if (sign > 0) {
        if (f32) update_kernel<1, true><<<grid, UPD_THREADS, 0, s>>>(V->dv, cam, list, count, cap);
        else update_kernel<1, false><<<grid, UPD_THREADS, 0, s>>>(V->dv, cam, list, count, cap);
    } else {
        if (f32) update_kernel<-1, true><<<grid, UPD_THREADS, 0, s>>>(V->dv, cam, list, count, cap);
        else update_kernel<-1, false><<<grid, UPD_THREADS, 0, s>>>(V->dv, cam, list, count, cap);
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace sc

// ================================================================= C ABI ====

namespace {

template <typename T>
cudaError_t dalloc(sc_volume* V, T** p, size_t bytes) {
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e == cudaSuccess) V->device_bytes += bytes;
    return e;
}

void free_all(sc_volume* V) {
    void* ptrs[] = {V->table, V->D, V->W, V->C8, V->Cf, V->coord, V->flags, V->stamp, V->pool_count,
                    V->status, V->lists, V->list_counts, V->extract_slots, V->extract_count, V->prof_dev};
    for (auto& pr : V->ev_pending) {
        V->ev_free.push_back(pr.a);
        V->ev_free.push_back(pr.b);
    }
    std::sort(V->ev_free.begin(), V->ev_free.end());
    V->ev_free.erase(std::unique(V->ev_free.begin(), V->ev_free.end()), V->ev_free.end());
    for (cudaEvent_t e : V->ev_free)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : V->graph_ev)
        if (e) cudaEventDestroy(e);
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (V->h_status) cudaFreeHost(V->h_status);
    if (V->h_word) cudaFreeHost(V->h_word);
}

bool pow2(uint32_t x) { return x && !(x & (x - 1)); }

}  // namespace

void batch_destroy(sc_volume* V);  // batch.cu
void adj_destroy(sc_volume* V);    // loss.cu

extern "C" int sc_abi_version(void) { return SC_ABI_VERSION; }

extern "C" const char* sc_status_string(int s) {
    switch (s) {
        case SC_OK: return "ok";
        case SC_ERR_INVALID_ARG: return "invalid argument";
        case SC_ERR_CUDA: return "CUDA runtime error";
        case SC_ERR_HASH_FULL: return "hash table full (probe limit reached)";
        case SC_ERR_POOL_FULL: return "voxel pool full";
        case SC_ERR_RETRY_LIMIT: return "bounded device wait gave up";
        case SC_ERR_NOT_INTEGRATED: return "keyframe not integrated";
        case SC_ERR_CAPACITY: return "output capacity too small";
        case SC_ERR_ALREADY_INTEGRATED: return "keyframe already integrated";
        case SC_ERR_LIST_FULL: return "keyframe block list full";
        case SC_ERR_NOT_RESIDENT: return "keyframe block not resident (stream it in first)";
        case SC_ERR_CONFLICT: return "streamed-in block already resident";
        default: return "unknown status";
    }
}

extern "C" int sc_create_volume(const sc_volume_params* p, sc_volume** out) {
    if (!p || !out) return SC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!(p->voxel_size > 0.f) || !(p->trunc > 0.f) || !pow2(p->n_buckets) || p->bucket_size < 1 ||
        p->bucket_size > 16 || p->max_blocks < 1 || p->max_blocks > (1u << 23) || p->max_keyframes < 1 ||
        p->max_blocks_per_keyframe < 1 || p->max_batch < 1 || p->max_batch > 1024 ||
        (p->colour_format != SC_RGBA8 && p->colour_format != SC_RGB_F32))
        return SC_ERR_INVALID_ARG;
    if ((uint64_t)p->n_buckets * p->bucket_size > (1ull << 31)) return SC_ERR_INVALID_ARG;
    sc_volume* V = new (std::nothrow) sc_volume();
    if (!V) return SC_ERR_CUDA;
    V->p = *p;
    V->integrated.assign(p->max_keyframes, 0);
    V->img_epoch.assign(p->max_keyframes, 0);
    V->cur.assign(p->max_keyframes, 0);
    V->nonresident.assign(p->max_keyframes, 0);
    V->call_id = 0;
    V->last_stream = nullptr;
    V->batch = nullptr;
    V->adj = nullptr;
    V->bcfg = sc_batch_config{4, 8, 1};
    V->prof_on = false;
    V->prof_dev = nullptr;
    for (double& x : V->prof_ms) x = 0.0;
    for (int64_t& x : V->prof_n) x = 0;
    for (cudaEvent_t& e : V->graph_ev) e = nullptr;
    int rc = SC_OK;
    auto fail = [&](cudaError_t e) {
        rc = cuda_status(e);
        free_all(V);
        delete V;
        return rc;
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&V->device)) != cudaSuccess) return fail(e);
    if ((e = cudaDeviceGetAttribute(&V->num_sms, cudaDevAttrMultiProcessorCount, V->device)) != cudaSuccess)
        return fail(e);
    const size_t nent = (size_t)p->n_buckets * p->bucket_size;
    const size_t nb = p->max_blocks;
    const size_t nlist = (size_t)p->max_keyframes * 2 * p->max_blocks_per_keyframe;
    if ((e = dalloc(V, &V->table, nent * sizeof(HashEntry))) != cudaSuccess) return fail(e);
    if ((e = dalloc(V, &V->D, nb * NVOX * sizeof(float))) != cudaSuccess) return fail(e);
    if ((e = dalloc(V, &V->W, nb * NVOX * sizeof(float))) != cudaSuccess) return fail(e);
    if (p->colour_format == SC_RGB_F32) {
        if ((e = dalloc(V, &V->Cf, nb * 3 * NVOX * sizeof(float))) != cudaSuccess) return fail(e);
    } else {
        if ((e = dalloc(V, &V->C8, nb * NVOX * sizeof(uint32_t))) != cudaSuccess) return fail(e);
    }
    if ((e = dalloc(V, &V->coord, nb * sizeof(int4))) != cudaSuccess) return fail(e);
    if ((e = dalloc(V, &V->flags, nb * sizeof(uint32_t))) != cudaSuccess) return fail(e);
    if ((e = dalloc(V, &V->stamp, nb * sizeof(uint32_t))) != cudaSuccess) return fail(e);
    if ((e = dalloc(V, &V->pool_count, sizeof(uint32_t))) != cudaSuccess) return fail(e);
    if ((e = dalloc(V, &V->status, sizeof(int32_t))) != cudaSuccess) return fail(e);
    if ((e = dalloc(V, &V->lists, nlist * sizeof(int32_t))) != cudaSuccess) return fail(e);
    if ((e = dalloc(V, &V->list_counts, (size_t)p->max_keyframes * 2 * sizeof(int32_t))) != cudaSuccess)
        return fail(e);
    if ((e = dalloc(V, &V->extract_slots, nb * sizeof(int32_t))) != cudaSuccess) return fail(e);
    if ((e = dalloc(V, &V->extract_count, sizeof(unsigned long long))) != cudaSuccess) return fail(e);
    if ((e = dalloc(V, &V->prof_dev, 4 * sizeof(unsigned long long))) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(V->prof_dev, 0, 4 * sizeof(unsigned long long))) != cudaSuccess) return fail(e);
    for (cudaEvent_t& ev : V->graph_ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return fail(e);
    if ((e = cudaMallocHost((void**)&V->h_status, sizeof(int32_t))) != cudaSuccess) return fail(e);
    if ((e = cudaMallocHost((void**)&V->h_word, 64)) != cudaSuccess) return fail(e);

    // zero the pool once; afterwards blocks are zeroed lazily on first update
    if ((e = cudaMemset(V->D, 0, nb * NVOX * sizeof(float))) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(V->W, 0, nb * NVOX * sizeof(float))) != cudaSuccess) return fail(e);
    if (V->Cf && (e = cudaMemset(V->Cf, 0, nb * 3 * NVOX * sizeof(float))) != cudaSuccess) return fail(e);
    if (V->C8 && (e = cudaMemset(V->C8, 0, nb * NVOX * sizeof(uint32_t))) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(V->flags, 0, nb * sizeof(uint32_t))) != cudaSuccess) return fail(e);
    if ((e = cudaMemset(V->stamp, 0, nb * sizeof(uint32_t))) != cudaSuccess) return fail(e);

    DevVolume& d = V->dv;
    d.table = V->table;
    d.bucket_mask = p->n_buckets - 1;
    d.bucket_size = p->bucket_size;
    d.max_probe = p->n_buckets < 64 ? p->n_buckets : 64;
    d.max_blocks = p->max_blocks;
    d.D = V->D;
    d.W = V->W;
    d.C8 = V->C8;
    d.Cf = V->Cf;
    d.coord = V->coord;
    d.flags = V->flags;
    d.stamp = V->stamp;
    d.pool_count = V->pool_count;
    d.status = V->status;
    d.retry_limit = DEFAULT_RETRY;
    d.colour_f32 = p->colour_format == SC_RGB_F32;
    d.prof = nullptr;
    V->last_stream = nullptr;
    rc = sc_reset_volume(V, nullptr);
    if (rc == SC_OK) rc = cuda_status(cudaDeviceSynchronize());
    if (rc != SC_OK) {
        free_all(V);
        delete V;
        return rc;
    }
    *out = V;
    return SC_OK;
}

extern "C" int sc_destroy_volume(sc_volume* V) {
    if (!V) return SC_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    batch_destroy(V);
    adj_destroy(V);
    free_all(V);
    delete V;
    return SC_OK;
}

extern "C" int sc_reset_volume(sc_volume* V, sc_stream stream) {
    if (!V) return SC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nent = (size_t)V->p.n_buckets * V->p.bucket_size;
    reset_table_kernel<<<grid_for(V, 8), 256, 0, s>>>(V->table, nent);
    count_launches(1);
    SC_CUDA(cudaGetLastError());
    SC_CUDA(cudaMemsetAsync(V->pool_count, 0, sizeof(uint32_t), s));
    SC_CUDA(cudaMemsetAsync(V->status, 0, sizeof(int32_t), s));
    SC_CUDA(cudaMemsetAsync(V->list_counts, 0, (size_t)V->p.max_keyframes * 2 * sizeof(int32_t), s));
    std::fill(V->nonresident.begin(), V->nonresident.end(), 0);
    // pool slots are handed out again from 0: mark them fresh lazily via the allocator,
    // and forget the per-call stamps
    SC_CUDA(cudaMemsetAsync(V->stamp, 0, (size_t)V->p.max_blocks * sizeof(uint32_t), s));
    V->call_id = 0;
    std::fill(V->integrated.begin(), V->integrated.end(), 0);
    std::fill(V->cur.begin(), V->cur.end(), 0);
    V->last_stream = s;
    return SC_OK;
}

extern "C" int sc_get_status(sc_volume* V, int32_t* device_status) {
    if (!V || !device_status) return SC_ERR_INVALID_ARG;
    int st = read_status(V, V->last_stream);
    if (st > 0) return st;  // never: statuses are <= 0
    *device_status = st;
    SC_CUDA(cudaMemsetAsync(V->status, 0, sizeof(int32_t), V->last_stream));
    SC_CUDA(cudaStreamSynchronize(V->last_stream));
    return SC_OK;
}

extern "C" int sc_get_volume_info(sc_volume* V, sc_volume_info* info) {
    if (!V || !info) return SC_ERR_INVALID_ARG;
    SC_CUDA(cudaMemcpyAsync(V->h_word, V->pool_count, sizeof(uint32_t), cudaMemcpyDeviceToHost, V->last_stream));
    SC_CUDA(cudaStreamSynchronize(V->last_stream));
    const uint32_t used = V->h_word[0];
    info->allocated_blocks = used < V->p.max_blocks ? used : V->p.max_blocks;
    info->max_blocks = V->p.max_blocks;
    info->hash_entries = V->p.n_buckets * V->p.bucket_size;
    int n = 0;
    for (uint8_t b : V->integrated) n += b;
    info->integrated_keyframes = n;
    info->device_bytes = V->device_bytes;
    return SC_OK;
}

extern "C" int sc_set_retry_limit(sc_volume* V, int32_t limit) {
    if (!V || limit < 0) return SC_ERR_INVALID_ARG;
    V->dv.retry_limit = limit == 0 ? DEFAULT_RETRY : limit;
    return SC_OK;
}

static int check_kf_args(sc_volume* V, int32_t kf_id, const float* depth, const uint8_t* rgba,
                         const sc_intrinsics* K, const sc_pose* T) {
    if (!V || !depth || !rgba || !T || !intrinsics_ok(K)) return SC_ERR_INVALID_ARG;
    if (kf_id < 0 || kf_id >= V->p.max_keyframes) return SC_ERR_INVALID_ARG;
    if (((uintptr_t)depth & 15) || ((uintptr_t)rgba & 15)) return SC_ERR_INVALID_ARG;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c)
            if (!std::isfinite(T->m[r][c])) return SC_ERR_INVALID_ARG;
    return SC_OK;
}

extern "C" int sc_integrate_keyframe(sc_volume* V, int32_t kf_id, const float* depth, const uint8_t* rgba,
                                     const sc_intrinsics* K, const sc_pose* T, sc_stream stream) {
    int rc = check_kf_args(V, kf_id, depth, rgba, K, T);
    if (rc) return rc;
    if (V->integrated[kf_id]) return SC_ERR_ALREADY_INTEGRATED;
    cudaStream_t s = (cudaStream_t)stream;
    const KfCam cam = make_cam(V, K, T, depth, rgba);
    const int which = V->cur[kf_id];
    int32_t* list = list_ptr(V, kf_id, which);
    int32_t* cnt = count_ptr(V, kf_id, which);
    if (++V->call_id == 0) {  // stamps wrapped: forget them
        SC_CUDA(cudaMemsetAsync(V->stamp, 0, (size_t)V->p.max_blocks * sizeof(uint32_t), s));
        V->call_id = 1;
    }
    SC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t), s));
    cudaEvent_t e0 = prof_mark(V, s);
    SC_CUDA(launch_alloc(V, cam, list, cnt, V->call_id, s));
    cudaEvent_t e1 = prof_mark(V, s);
    SC_CUDA(launch_update(V, cam, list, cnt, +1, s));
    cudaEvent_t e2 = prof_mark(V, s);
    prof_pair(V, e0, e1, 0);
    prof_pair(V, e1 ? e1 : nullptr, e2, 1);
    V->integrated[kf_id] = 1;
    ++V->img_epoch[kf_id];
    V->last_stream = s;
    return SC_OK;
}

extern "C" int sc_deintegrate_keyframe(sc_volume* V, int32_t kf_id, const float* depth, const uint8_t* rgba,
                                       const sc_intrinsics* K, const sc_pose* T, sc_stream stream) {
    int rc = check_kf_args(V, kf_id, depth, rgba, K, T);
    if (rc) return rc;
    if (!V->integrated[kf_id]) return SC_ERR_NOT_INTEGRATED;
    if (V->nonresident[kf_id]) return SC_ERR_NOT_RESIDENT;
    cudaStream_t s = (cudaStream_t)stream;
    const KfCam cam = make_cam(V, K, T, depth, rgba);
    const int which = V->cur[kf_id];
    cudaEvent_t e0 = prof_mark(V, s);
    SC_CUDA(launch_update(V, cam, list_ptr(V, kf_id, which), count_ptr(V, kf_id, which), -1, s));
    prof_pair(V, e0, prof_mark(V, s), 1);
    V->integrated[kf_id] = 0;
    V->last_stream = s;
    return SC_OK;
}

extern "C" int sc_extract_block_list(sc_volume* V, int32_t* coords, int32_t* slots, float* D, float* W, void* C,
                                     int32_t capacity, int32_t* count, sc_stream stream) {
    if (!V || !count || capacity < 0) return SC_ERR_INVALID_ARG;
    if (capacity > 0 && !coords && !slots && !D && !W && !C) return SC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t nent = V->p.n_buckets * V->p.bucket_size;
    const uint32_t cap = (uint32_t)capacity < V->p.max_blocks ? (uint32_t)capacity : V->p.max_blocks;
    SC_CUDA(cudaMemsetAsync(V->extract_count, 0, sizeof(uint32_t), s));
    extract_kernel<<<grid_for(V, 8), EXTRACT_THREADS, 0, s>>>(V->dv, nent, coords, slots, V->extract_slots, V->extract_count,
                                                  cap);
    count_launches(1);
    SC_CUDA(cudaGetLastError());
    SC_CUDA(cudaMemcpyAsync(V->h_word, V->extract_count, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    const uint32_t n = V->h_word[0];
    *count = (int32_t)n;
    const uint32_t m = n < cap ? n : cap;
    if (m > 0 && (D || W || C)) {
        gather_payload_kernel<<<grid_for(V, 16), 128, 0, s>>>(V->dv, V->extract_slots, m, D, W, C);
        count_launches(1);
        SC_CUDA(cudaGetLastError());
    }
    V->last_stream = s;
    const int st = read_status(V, s);
    if (st) return st;
    return n > (uint32_t)capacity ? SC_ERR_CAPACITY : SC_OK;
}

extern "C" int sc_get_keyframe_blocks(sc_volume* V, int32_t kf_id, int32_t* slots, int32_t capacity,
                                      int32_t* count, sc_stream stream) {
    if (!V || !count || kf_id < 0 || kf_id >= V->p.max_keyframes || capacity < 0) return SC_ERR_INVALID_ARG;
    if (!V->integrated[kf_id]) return SC_ERR_NOT_INTEGRATED;
    cudaStream_t s = (cudaStream_t)stream;
    const int which = V->cur[kf_id];
    SC_CUDA(cudaMemcpyAsync(V->h_word, count_ptr(V, kf_id, which), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    int32_t n = (int32_t)V->h_word[0];
    if ((uint32_t)n > V->p.max_blocks_per_keyframe) n = (int32_t)V->p.max_blocks_per_keyframe;
    *count = n;
    const int32_t m = n < capacity ? n : capacity;
    if (slots && m > 0)
        SC_CUDA(cudaMemcpyAsync(slots, list_ptr(V, kf_id, which), (size_t)m * sizeof(int32_t),
                                cudaMemcpyDeviceToDevice, s));
    SC_CUDA(cudaStreamSynchronize(s));
    V->last_stream = s;
    return n > capacity ? SC_ERR_CAPACITY : SC_OK;
}

extern "C" int sc_set_profiling(sc_volume* V, int32_t enabled) {
    if (!V) return SC_ERR_INVALID_ARG;
    SC_CUDA(cudaStreamSynchronize(V->last_stream));
    for (auto& pr : V->ev_pending) {
        V->ev_free.push_back(pr.a);
        if (pr.b != pr.a) V->ev_free.push_back(pr.b);
    }
    V->ev_pending.clear();
    std::sort(V->ev_free.begin(), V->ev_free.end());
    V->ev_free.erase(std::unique(V->ev_free.begin(), V->ev_free.end()), V->ev_free.end());
    for (double& x : V->prof_ms) x = 0.0;
    for (int64_t& x : V->prof_n) x = 0;
    SC_CUDA(cudaMemset(V->prof_dev, 0, 4 * sizeof(unsigned long long)));
    V->prof_on = enabled != 0;
    V->dv.prof = V->prof_on ? V->prof_dev : nullptr;
    return SC_OK;
}

extern "C" int sc_get_profile(sc_volume* V, sc_profile* out) {
    if (!V || !out) return SC_ERR_INVALID_ARG;
    SC_CUDA(cudaStreamSynchronize(V->last_stream));
    // events are shared between consecutive pairs (end of one = start of the next)
    std::vector<cudaEvent_t> done;
    for (auto& pr : V->ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pr.a, pr.b) == cudaSuccess) {
            V->prof_ms[pr.kind] += ms;
            V->prof_n[pr.kind] += 1;
        }
        done.push_back(pr.a);
        done.push_back(pr.b);
    }
    V->ev_pending.clear();
    std::sort(done.begin(), done.end());
    done.erase(std::unique(done.begin(), done.end()), done.end());
    for (cudaEvent_t e : done) V->ev_free.push_back(e);
    unsigned long long c[4] = {0, 0, 0, 0};
    SC_CUDA(cudaMemcpy(c, V->prof_dev, sizeof(c), cudaMemcpyDeviceToHost));
    sc_profile p{};
    p.enabled = V->prof_on;
    p.alloc_ms = V->prof_ms[0];
    p.alloc_launches = V->prof_n[0];
    p.update_ms = V->prof_ms[1];
    p.update_launches = V->prof_n[1];
    p.update_blocks = (int64_t)c[0];
    p.batch_alloc_ms = V->prof_ms[2];
    p.batch_mark_ms = V->prof_ms[3];
    p.batch_net_ms = V->prof_ms[4];
    p.batch_launches = V->prof_n[2];
    p.batch_union_blocks = (int64_t)c[1];
    p.batch_pairs = (int64_t)c[2];
    p.mc_ms = V->prof_ms[5];
    p.mc_launches = V->prof_n[5];
    *out = p;
    return SC_OK;
}
