// Marching Cubes extraction of the SDF's zero level set (Section 3 "SDF volume"),
// block import and keyframe block lists set from coordinates (restoring a volume).
//
// Cube (x, y, z) has the 8 corner voxels (x + i0, y + i1, z + i2), i0..i2 the bits
// of the corner number; it is meshed when all 8 exist and are observed (W > 0).  A
// corner is inside when D < 0.  Each crossed edge carries a vertex at the linear
// zero of D.  The triangulation of an inside mask follows one rule, built into a
// 256-case table on the host at first use:
//  * around each face, every maximal run of consecutive inside corners (not the
//    whole ring) is closed off by one segment between the crossed edges at its two
//    ends; so diagonal inside corners of a face are cut off separately;
//  * a segment is directed so that, seen from outside the cube, its run of inside
//    corners lies on its right; the directed segments chain into loops, whose
//    triangles then face free space (D > 0);
//  * each loop is fanned from its smallest edge number; loops in order of their
//    smallest edge number.
// Edge e runs along axis e / 4 from the corner whose other two coordinate bits are
// e % 4 (lower axis in bit 0).
//
// mc_kernel: one CTA of 128 threads per pool slot; the block's voxels and the faces
// of its 7 upper neighbours (found in the hash) are staged in shared memory as a
// 9 x 9 x 9 tile of D (NaN where unobserved); a thread classifies 4 consecutive cubes;
// a CTA-wide scan of triangle counts and one atomic give each triangle its output
// position, and the block's triangles, listed in that order in shared memory, are
// emitted by all threads (the surface crosses few cubes, so emitting each cube's
// triangles from the thread that classified it left half the lanes idle).
#include <algorithm>
#include <mutex>
#include <vector>

#include "volume.cuh"

namespace {

using namespace sc;

constexpr int MC_THREADS = 128;
constexpr int MC_MAXT = 5;  // triangles per case under the rule (checked when the table is built)
constexpr int TILE = 9;

struct McTable {
    uint8_t ntri[256];
    uint8_t edge[256][3 * MC_MAXT];
};

// ---- host: the case table ----

struct HostCube {
    int lo[12], axis[12];  // edge -> lower corner, axis
    HostCube() {
        for (int e = 0; e < 12; ++e) {
            const int a = e >> 2, r = e & 3;
            const int o1 = (a == 0) ? 1 : 0, o2 = (a == 2) ? 1 : 2;
            lo[e] = ((r & 1) << o1) | (((r >> 1) & 1) << o2);
            axis[e] = a;
        }
    }
    int edge(int c0, int c1) const {  // the edge joining two corners one axis apart
        const int a = (c0 ^ c1) == 1 ? 0 : ((c0 ^ c1) == 2 ? 1 : 2);
        for (int e = 4 * a; e < 4 * a + 4; ++e)
            if (lo[e] == (c0 & c1)) return e;
        return -1;
    }
};

// Corners of a face ring in counter-clockwise order seen from outside the cube
// (outward normal towards the viewer).
void face_ring(int a, int side, int ring[4]) {
    const int u = (a + 1) % 3, w = (a + 2) % 3;  // (u, w, a) right-handed
    const int base = side << a;
    // counter-clockwise about +a is u, then w; about -a it is w, then u
    const int p = side ? u : w, q = side ? w : u;
    ring[0] = base;
    ring[1] = base | (1 << p);
    ring[2] = base | (1 << p) | (1 << q);
    ring[3] = base | (1 << q);
}

int build_case(const HostCube& C, int mask, uint8_t* out) {
    auto inside = [&](int c) { return (mask >> c) & 1; };
    int next[12];
    std::fill(next, next + 12, -1);
    for (int a = 0; a < 3; ++a)
        for (int side = 0; side < 2; ++side) {
            int ring[4];
            face_ring(a, side, ring);
            // each run of inside corners ring[i..j] (cyclic, not the whole ring): the ring
            // enters it across the edge (ring[i-1], ring[i]) and leaves across (ring[j],
            // ring[j+1]).  The chord from the entering to the leaving edge runs with the
            // counter-clockwise ring, whose corners are on its right (the face is on the
            // left of a counter-clockwise boundary), so the run lies on the chord's right.
            for (int i = 0; i < 4; ++i) {
                if (!inside(ring[i]) || inside(ring[(i + 3) % 4])) continue;  // i starts a run
                int j = i;
                while (inside(ring[(j + 1) % 4])) j = (j + 1) % 4;
                const int enter = C.edge(ring[(i + 3) % 4], ring[i]);
                const int leave = C.edge(ring[j], ring[(j + 1) % 4]);
                next[enter] = leave;
            }
        }
    int n = 0;
    bool seen[12] = {false};
    for (int e0 = 0; e0 < 12; ++e0) {
        if (next[e0] < 0 || seen[e0]) continue;
        std::vector<int> loop;
        for (int e = e0; !seen[e]; e = next[e]) {
            seen[e] = true;
            loop.push_back(e);
            if (next[e] < 0) return -1;  // an open chain would break the rule
        }
        if (loop.size() < 3) return -1;
        // e0 is the loop's smallest edge (smaller crossed edges belong to earlier loops)
        for (size_t i = 1; i + 1 < loop.size(); ++i) {
            if (n == MC_MAXT) return -1;
            out[3 * n] = (uint8_t)loop[0];
            out[3 * n + 1] = (uint8_t)loop[i];
            out[3 * n + 2] = (uint8_t)loop[i + 1];
            ++n;
        }
    }
    return n;
}

std::once_flag g_mc_once;
McTable g_mc_host;
bool g_mc_ok = false;
std::mutex g_mc_dev_mu;
McTable* g_mc_dev[64] = {nullptr};

void build_table() {
    HostCube C;
    g_mc_ok = true;
    for (int m = 0; m < 256; ++m) {
        const int n = build_case(C, m, g_mc_host.edge[m]);
        if (n < 0) g_mc_ok = false;
        g_mc_host.ntri[m] = (uint8_t)(n < 0 ? 0 : n);
    }
}

const McTable* device_table(int dev, cudaStream_t s) {
    std::call_once(g_mc_once, build_table);
    if (!g_mc_ok) return nullptr;
    std::lock_guard<std::mutex> lock(g_mc_dev_mu);
    McTable*& t = g_mc_dev[dev & 63];
    if (!t) {
        if (cudaMalloc((void**)&t, sizeof(McTable)) != cudaSuccess) {
            t = nullptr;
            return nullptr;
        }
        if (cudaMemcpy(t, &g_mc_host, sizeof(McTable), cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
    }
    (void)s;
    return t;
}

// ---- device ----

struct McOut {
    float* tri;         // [cap][3][3]
    int32_t* cube;      // [cap][4] or null
    unsigned long long* count;
    unsigned long long cap;
    float voxel_size;
};

__device__ __forceinline__ int tile_at(int x, int y, int z) { return x + TILE * (y + TILE * z); }

__global__ void __launch_bounds__(MC_THREADS) mc_kernel(DevVolume V, const McTable* __restrict__ T, McOut out,
                                                        uint32_t n_slots) {
    __shared__ float tD[TILE * TILE * TILE];
    __shared__ int32_t nslot[8];
    __shared__ int32_t scan[MC_THREADS / 32];
    __shared__ unsigned long long base_s;
    __shared__ uint8_t cmask[NVOX];                // case of each of the block's 512 cubes
    __shared__ uint16_t tri_ref[NVOX * MC_MAXT];   // (cube << 3 | t) of each triangle, in output order
    const uint32_t slot = blockIdx.x;
    if (slot >= n_slots) return;
    const int tid = threadIdx.x;
    const int4 bc = V.coord[slot];
    if (V.flags[slot] & FLAG_FRESH) return;  // never updated: no observed voxel
    if (tid < 8) {
        int32_t s = (int32_t)slot;
        if (tid > 0) {
            const int bx = bc.x + (tid & 1), by = bc.y + ((tid >> 1) & 1), bz = bc.z + ((tid >> 2) & 1);
            s = coord_ok(bx, by, bz) ? find_slot(V, pack_key(bx, by, bz)) : -1;
            if (s >= 0 && (V.flags[s] & FLAG_FRESH)) s = -1;
        }
        nslot[tid] = s;
    }
    __syncthreads();
    for (int i = tid; i < TILE * TILE * TILE; i += MC_THREADS) {
        const int x = i % TILE, y = (i / TILE) % TILE, z = i / (TILE * TILE);
        const int nb = (x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2);
        const int32_t s = nslot[nb];
        float d = __int_as_float(0x7fc00000);  // NaN: unobserved or missing
        if (s >= 0) {
            // W and D requested together (one round trip, not two)
            const size_t v = (size_t)s * NVOX + (x & 7) + 8 * (y & 7) + 64 * (z & 7);
            const float w = V.W[v], dv = V.D[v];
            if (w > 0.f) d = dv;
        }
        tD[i] = d;
    }
    __syncthreads();
    // 4 cubes per thread: x = lx0 .. lx0 + 3
    const int lx0 = 4 * (tid & 1), ly = (tid >> 1) & 7, lz = tid >> 4;
    int masks[4], cnt = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int m = 0;
        bool ok = true;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float d = tD[tile_at(lx0 + j + (c & 1), ly + ((c >> 1) & 1), lz + ((c >> 2) & 1))];
            ok = ok && (d == d);
            m |= (d < 0.f ? 1 : 0) << c;
        }
        masks[j] = ok ? m : 0;
        cnt += ok ? __ldg(&T->ntri[m]) : 0;
    }
    // CTA exclusive scan of the triangle counts
    const int lane = tid & 31, warp = tid >> 5;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) scan[warp] = incl;
    __syncthreads();
    int wbase = 0, total = 0;
#pragma unroll
    for (int w = 0; w < MC_THREADS / 32; ++w) {
        if (w < warp) wbase += scan[w];
        total += scan[w];
    }
    if (tid == 0) base_s = total ? atomicAdd(out.count, (unsigned long long)total) : 0ull;
    // the block's triangles in output order, (cube, t) each, so that the emission below
    // spreads them over all threads instead of leaving the threads of empty cubes idle
    int loc = wbase + incl - cnt;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int m = masks[j];
        cmask[4 * tid + j] = (uint8_t)m;
        const int nt = __ldg(&T->ntri[m]);
        for (int t = 0; t < nt; ++t) tri_ref[loc++] = (uint16_t)(((4 * tid + j) << 3) | t);
    }
    __syncthreads();
    const float s = out.voxel_size;
    for (int i = tid; i < total; i += MC_THREADS) {
        const unsigned long long k = base_s + (unsigned long long)i;
        if (k >= out.cap) break;
        const int r = tri_ref[i], cube = r >> 3, t = r & 7;
        const int owner = cube >> 2;
        const int cx = 4 * (owner & 1) + (cube & 3), cy = (owner >> 1) & 7, cz = owner >> 4;
        const int m = cmask[cube];
        const int vx = 8 * bc.x + cx, vy = 8 * bc.y + cy, vz = 8 * bc.z + cz;
        float* o = out.tri + 9 * k;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int e = __ldg(&T->edge[m][3 * t + q]);
            const int a = e >> 2, rr = e & 3;
            const int o1 = (a == 0) ? 1 : 0, o2 = (a == 2) ? 1 : 2;
            const int lo = ((rr & 1) << o1) | (((rr >> 1) & 1) << o2);
            const int hi = lo | (1 << a);
            const float d0 = tD[tile_at(cx + (lo & 1), cy + ((lo >> 1) & 1), cz + ((lo >> 2) & 1))];
            const float d1 = tD[tile_at(cx + (hi & 1), cy + ((hi >> 1) & 1), cz + ((hi >> 2) & 1))];
            const float tt = __fdiv_rn(d0, __fsub_rn(d0, d1));
            const int vc[3] = {vx + (lo & 1), vy + ((lo >> 1) & 1), vz + ((lo >> 2) & 1)};
#pragma unroll
            for (int d = 0; d < 3; ++d)
                o[3 * q + d] = __fmul_rn(s, d == a ? __fadd_rn((float)vc[d], tt) : (float)vc[d]);
        }
        if (out.cube) {
            int32_t* c = out.cube + 4 * k;
            c[0] = vx;
            c[1] = vy;
            c[2] = vz;
            c[3] = t;
        }
    }
}

// Import: one warp per input block: insert (or find) its hash entry, take a pool
// slot, copy the payload and mark the slot as holding data.
__global__ void import_kernel(DevVolume V, const int32_t* coords, const float* D, const float* W, const void* C,
                              int32_t n) {
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x / 32;
    for (int b = blockIdx.x * wpb + (threadIdx.x >> 5); b < n; b += gridDim.x * wpb) {
        int32_t slot = -1;
        if (lane == 0) {
            const int x = coords[3 * b], y = coords[3 * b + 1], z = coords[3 * b + 2];
            if (!coord_ok(x, y, z)) {
                set_status(V.status, SC_ERR_INVALID_ARG);
            } else {
                const unsigned long long key = pack_key(x, y, z);
                bool won;
                int32_t seen;
                const int e = hash_claim(V, key, &won, &seen);
                if (e >= 0) {
                    if (won) {
                        const uint32_t s = atomicAdd(V.pool_count, 1u);
                        if (s >= V.max_blocks) {
                            set_status(V.status, SC_ERR_POOL_FULL);
                            atomicExch(&V.table[e].slot, SLOT_FAILED);
                        } else {
                            V.coord[s] = make_int4(x, y, z, 0);
                            V.flags[s] = 0u;
                            __threadfence();
                            atomicExch(&V.table[e].slot, (int32_t)s);
                            slot = (int32_t)s;
                        }
                    } else {
                        slot = seen >= 0 ? seen : entry_slot(V, e);
                    }
                }
            }
        }
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot < 0) continue;
        if (lane == 0) V.flags[slot] = 0u;
        const size_t dst = (size_t)slot * NVOX, src = (size_t)b * NVOX;
        for (int i = lane; i < NVOX / 4; i += 32) {
            reinterpret_cast<float4*>(V.D + dst)[i] = __ldg(reinterpret_cast<const float4*>(D + src) + i);
            reinterpret_cast<float4*>(V.W + dst)[i] = __ldg(reinterpret_cast<const float4*>(W + src) + i);
            if (V.colour_f32) {
                for (int ch = 0; ch < 3; ++ch)
                    reinterpret_cast<float4*>(V.Cf + 3 * dst + ch * NVOX)[i] =
                        C ? __ldg(reinterpret_cast<const float4*>((const float*)C + 3 * src + ch * NVOX) + i)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                reinterpret_cast<uint4*>(V.C8 + dst)[i] =
                    C ? __ldg(reinterpret_cast<const uint4*>((const uint32_t*)C + src) + i) : make_uint4(0u, 0u, 0u, 0u);
            }
        }
    }
}

// list[i] = slot of block coords[i]; a coordinate without a resident block sets the
// status (SC_ERR_INVALID_ARG), and the caller then leaves the list empty
__global__ void set_list_kernel(DevVolume V, const int32_t* coords, int32_t n, int32_t* list) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x = coords[3 * i], y = coords[3 * i + 1], z = coords[3 * i + 2];
        const int32_t s = coord_ok(x, y, z) ? find_slot(V, pack_key(x, y, z)) : -1;
        if (s < 0) set_status(V.status, SC_ERR_INVALID_ARG);
        list[i] = s < 0 ? 0 : s;
    }
}

}  // namespace

extern "C" int sc_set_keyframe_blocks(sc_volume* V, int32_t kf_id, const int32_t* coords, int32_t n,
                                      sc_stream stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!V || kf_id < 0 || kf_id >= V->p.max_keyframes || n < 0 || (n > 0 && !coords) || ((uintptr_t)coords & 3))
        return SC_ERR_INVALID_ARG;
    if ((uint32_t)n > V->p.max_blocks_per_keyframe) return SC_ERR_LIST_FULL;
    if (V->integrated[kf_id]) return SC_ERR_ALREADY_INTEGRATED;
    SC_CUDA(cudaSetDevice(V->device));
    const int which = V->cur[kf_id];
    int32_t* list = list_ptr(V, kf_id, which);
    if (n > 0) {
        set_list_kernel<<<std::min((n + 255) / 256, V->num_sms * 8), 256, 0, s>>>(V->dv, coords, n, list);
        count_launches(1);
        SC_CUDA(cudaGetLastError());
    }
    V->h_word[3] = (uint32_t)n;
    SC_CUDA(cudaMemcpyAsync(count_ptr(V, kf_id, which), V->h_word + 3, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    const int st = read_status(V, s);
    if (st) {  // a block is missing: the keyframe stays not integrated
        V->h_word[3] = 0;
        SC_CUDA(cudaMemcpyAsync(count_ptr(V, kf_id, which), V->h_word + 3, sizeof(int32_t), cudaMemcpyHostToDevice, s));
        SC_CUDA(cudaStreamSynchronize(s));
        return st;
    }
    V->integrated[kf_id] = 1;
    ++V->img_epoch[kf_id];
    V->nonresident[kf_id] = 0;
    return SC_OK;
}

extern "C" int sc_mc_case(int32_t mask, int32_t* edges) {
    if (mask < 0 || mask > 255 || !edges) return SC_ERR_INVALID_ARG;
    std::call_once(g_mc_once, build_table);
    if (!g_mc_ok) return SC_ERR_INVALID_ARG;
    const int n = g_mc_host.ntri[mask];
    for (int i = 0; i < 3 * n; ++i) edges[i] = g_mc_host.edge[mask][i];
    return n;
}

extern "C" int sc_marching_cubes(sc_volume* V, float* triangles, int32_t* cubes, int64_t capacity, int64_t* count,
                                 sc_stream stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!V || !count || capacity < 0 || (capacity > 0 && !triangles)) return SC_ERR_INVALID_ARG;
    if (((uintptr_t)triangles & 3) || ((uintptr_t)cubes & 3)) return SC_ERR_INVALID_ARG;
    SC_CUDA(cudaSetDevice(V->device));
    const McTable* T = device_table(V->device, s);
    if (!T) return SC_ERR_CUDA;
    // the allocated slot count bounds the grid (one CTA per slot)
    SC_CUDA(cudaMemcpyAsync(V->h_word, V->pool_count, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    SC_CUDA(cudaStreamSynchronize(s));
    const uint32_t n_slots = std::min(*V->h_word, V->p.max_blocks);
    unsigned long long* dcount = reinterpret_cast<unsigned long long*>(V->extract_count);
    SC_CUDA(cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), s));
    if (n_slots > 0) {
        McOut o{triangles, cubes, dcount, (unsigned long long)capacity, V->p.voxel_size};
        cudaEvent_t e0 = prof_mark(V, s);
        mc_kernel<<<n_slots, MC_THREADS, 0, s>>>(V->dv, T, o, n_slots);
        prof_pair(V, e0, prof_mark(V, s), 5);
        count_launches(1);
        SC_CUDA(cudaGetLastError());
    }
    unsigned long long* hp = reinterpret_cast<unsigned long long*>(V->h_word + 2);  // pinned
    SC_CUDA(cudaMemcpyAsync(hp, dcount, sizeof(*hp), cudaMemcpyDeviceToHost, s));
    const int st = read_status(V, s);
    const unsigned long long h = *hp;
    *count = (int64_t)h;
    if (st) return st;
    return (int64_t)h > capacity ? SC_ERR_CAPACITY : SC_OK;
}

extern "C" int sc_import_blocks(sc_volume* V, const int32_t* coords, const float* D, const float* W, const void* C,
                                int32_t n, sc_stream stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!V || n < 0 || (n > 0 && (!coords || !D || !W))) return SC_ERR_INVALID_ARG;
    if (((uintptr_t)D & 15) || ((uintptr_t)W & 15) || ((uintptr_t)C & 15) || ((uintptr_t)coords & 3))
        return SC_ERR_INVALID_ARG;
    SC_CUDA(cudaSetDevice(V->device));
    if (n > 0) {
        const int threads = 256, wpb = threads / 32;
        const int grid = std::min((n + wpb - 1) / wpb, V->num_sms * 16);
        import_kernel<<<grid, threads, 0, s>>>(V->dv, coords, D, W, C, n);
        count_launches(1);
        SC_CUDA(cudaGetLastError());
    }
    return read_status(V, s);
}
