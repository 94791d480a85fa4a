// Host-side state of a volume and helpers shared by the .cu files.
#pragma once

#include <vector>

#include "common.cuh"

struct BatchState;  // batched re-integration state (batch.cu)
struct AdjScratch;  // adjoint item tables and accumulators (loss.cu)

struct sc_volume {
    sc_volume_params p;
    int device;
    int num_sms;
    sc::DevVolume dv;
    // device memory
    sc::HashEntry* table;
    float* D;
    float* W;
    uint32_t* C8;
    float* Cf;
    int4* coord;
    uint32_t* flags;
    uint32_t* stamp;
    uint32_t* pool_count;
    int32_t* status;
    int32_t* lists;        // [max_keyframes][2][max_blocks_per_keyframe]
    int32_t* list_counts;  // [max_keyframes][2]
    int32_t* extract_slots;  // [max_blocks] scratch for extraction
    uint32_t* extract_count;  // 8 bytes: 32-bit extraction count, 64-bit triangle count
    // host mirrors
    std::vector<uint8_t> integrated;
    std::vector<uint8_t> cur;  // which of the two list buffers holds the current list
    std::vector<uint8_t> nonresident;  // the current list names a block in a host block store
    // per keyframe, counts the times it became integrated: its images (depth, colour) are
    // bound from then until it is de-integrated, so a batch may reuse texels it packed
    // from the same images under the same count
    std::vector<uint32_t> img_epoch;
    uint32_t call_id;
    cudaStream_t last_stream;
    int32_t* h_status;  // pinned
    uint32_t* h_word;   // pinned scratch
    uint64_t device_bytes;
    BatchState* batch;
    AdjScratch* adj;  // allocated by the first sc_sdf_adjoint call, grown on demand
    sc_batch_config bcfg;
    // profiling
    bool prof_on;
    unsigned long long* prof_dev;  // [4] update blocks, batch union, batch pairs
    struct EvPair {
        cudaEvent_t a, b;
        int kind;  // 0 alloc, 1 update
    };
    std::vector<EvPair> ev_pending;
    std::vector<cudaEvent_t> ev_free;
    double prof_ms[6];  // alloc, update, batch alloc, batch mark, batch net, marching cubes
    int64_t prof_n[6];  // launches: alloc, update, batch, -, -, marching cubes
    cudaEvent_t graph_ev[4];
};

namespace sc {

// process-wide count of kernels launched by this library
void count_launches(uint64_t n);

int cuda_status(cudaError_t e);
#define SC_CUDA(call)                                 \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return sc::cuda_status(e_); \
    } while (0)

KfCam make_cam(const sc_volume* V, const sc_intrinsics* K, const sc_pose* T, const float* depth,
               const uint8_t* rgba);
bool intrinsics_ok(const sc_intrinsics* K);

inline int32_t* list_ptr(sc_volume* V, int kf, int which) {
    return V->lists + ((size_t)kf * 2 + which) * V->p.max_blocks_per_keyframe;
}
inline int32_t* count_ptr(sc_volume* V, int kf, int which) { return V->list_counts + (size_t)kf * 2 + which; }

// Allocate A(k, T) and write the keyframe's block list (plain path).
cudaError_t launch_alloc(sc_volume* V, const KfCam& cam, int32_t* list, int32_t* count, uint32_t call_id,
                         cudaStream_t s);
// Running-average update (sign +1) or Eq. 2 (sign -1) over a block list.
cudaError_t launch_update(sc_volume* V, const KfCam& cam, const int32_t* list, const int32_t* count, int sign,
                          cudaStream_t s);
// Synchronise `s` and return the device status word (without clearing it).
int read_status(sc_volume* V, cudaStream_t s);

// Profiling: an event recorded on s (null when profiling is off) and the pairing of
// two such events as one timed launch of `kind`.
cudaEvent_t prof_mark(sc_volume* V, cudaStream_t s);
void prof_pair(sc_volume* V, cudaEvent_t a, cudaEvent_t b, int kind);

}  // namespace sc
