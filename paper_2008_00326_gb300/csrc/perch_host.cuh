// Host-side internals of libperch shared by its translation units: the
// context and its records, the scoring scratch, and the helpers every entry
// point uses.  Not part of the public ABI.
#pragma once

#include "perch.h"
#include "perch_internal.cuh"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstdint>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

namespace perch_host {

// Who still reads a resident mesh or observation: queued or running served
// requests and batch graphs (users), and asynchronous calls on the callers'
// streams (an event recorded after each, dropped once it has completed).
// Releasing the object is refused (PERCH_E_BUSY) while any is outstanding.
struct UseTrack {
    int users = 0;
    std::vector<cudaEvent_t> pending;
};

struct MeshRec {
    perch::DevMesh dm{};
    void* verts = nullptr;
    void* tris = nullptr;
    UseTrack use;
};

struct SceneRec {
    perch::DevScene ds{};
    perch_params params{};
    void* depth = nullptr;
    void* labels = nullptr;
    void* lab = nullptr;
    void* pxyz = nullptr;          // per-pixel observed points (DevScene::pxyz)
    void* pts = nullptr;
    void* table = nullptr;
    void* nrm = nullptr;           // observed normals (GICP targets), made on first use
    int nrm_jump = -1;             // the normal_max_jump_units they were made with
    void* near = nullptr;          // near-cell bitmap (DevScene::near_bits)
    void* cstart = nullptr;        // dense cell index (DevScene::cell_start)
    UseTrack use;
};

// Everything one chain of scoring launches needs besides its inputs: one
// hypothesis counter per job followed by the vertex-cache slot mask (zeroed
// together before each run), the vertex-cache pool, and the side streams a
// multi-job run spreads its launches over.  Runs that share a ScoreScratch
// are ordered on the GPU through `last`.
constexpr int kSideStreams = 4;

struct ScoreScratch {
    unsigned* next = nullptr;      // device: counters, then slot mask
    size_t next_words = 0;
    void* vcache = nullptr;
    size_t vcache_bytes = 0;
    void* src = nullptr;           // GICP source clouds, one slot per resident block
    size_t src_bytes = 0;
    cudaStream_t side[kSideStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kSideStreams] = {};
    cudaEvent_t last = nullptr;
};

// An NVTX range over the rest of the enclosing scope: the host stages of
// each call show up by name in a profiler's timeline (header-only NVTX v3:
// free when no tool is attached).
class Range {
public:
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

class DeviceGuard {
public:
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
        if (prev_ != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev_ >= 0) cudaSetDevice(prev_);
    }

private:
    int prev_ = -1;
};

// Capacity of the shared-memory bitset that marks nearest neighbours inside
// the admissible box.  Boxes larger than this are processed in row bands (each
// band repeats the render and search), so the capacity only trades shared
// memory against that rare repetition.  At least one image row always fits.
// The defaults (a 7,064-word z-buffer, 32,768 mark bits, 256 threads) keep a
// scoring block at 55.6 KB of shared memory, so that four blocks of 64
// registers per thread fit an SM: 32 warps instead of 24, 11 % faster on the
// bench workload than three blocks with an 8,192-word z-buffer.
constexpr int kZbufWordsDefault = 7064;
constexpr int kMarkBitsDefault = 1 << 15;

}  // namespace perch_host

struct perch_ctx {
    int device = 0;
    uint64_t budget = 0;
    uint64_t used = 0;
    std::unordered_map<void*, size_t> allocs;
    std::map<int32_t, perch_host::MeshRec> meshes;
    std::map<int32_t, perch_host::SceneRec> scenes;
    int32_t next_id = 1;
    std::string err;
    cudaStream_t stream = nullptr;
    void* stage = nullptr;
    size_t stage_bytes = 0;
    int* d_err = nullptr;
    unsigned long long* d_best_partial = nullptr;   // 3 words per block, kBestMaxBlocks blocks
    unsigned* d_best_ticket = nullptr;
    long long* d_best_index = nullptr;
    int32_t* d_best_cost = nullptr;
    cudaEvent_t best_last = nullptr;                // the last argmin launch (they share the scratch)
    perch_host::ScoreScratch plain;                    // scratch of the context's own scoring launches
    std::map<uint64_t, perch::ScoreConfig> tuned;   // autotuner results by batch class
    perch::ScoreConfig cfg{256, perch_host::kZbufWordsDefault, perch_host::kMarkBitsDefault, 0};
    // A running server's threads share the context: they and the calls that
    // may overlap them (loading and releasing meshes and observations) hold
    // mu around the maps, the budget and the allocations.  Every other call
    // is refused while a server runs.
    std::mutex mu;
    std::atomic<int> servers{0};
};

struct perch_batch_graph {
    perch_ctx* ctx = nullptr;
    unsigned* next = nullptr;              // the graph's own counters and slot mask
    void* vcache = nullptr;                // and vertex-cache pool
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;            // recorded after each launch
    std::vector<std::pair<int32_t, int32_t>> uses;   // (scene, mesh) of its items, counted as users
};

namespace perch_host {

// Record st and a message in the context's last error (printf format).
perch_status fail(perch_ctx* c, perch_status st, const char* fmt, ...);
perch_status cuda_fail(perch_ctx* c, cudaError_t e, const char* what);
// Device allocation charged to the context's HBM budget; dfree returns it.
perch_status dalloc(perch_ctx* c, size_t bytes, void** p);
void dfree(perch_ctx* c, void* p);
// The context's device staging buffer, grown to at least bytes.
perch_status ensure_stage(perch_ctx* c, size_t bytes);
// Read and clear the device error word (synchronous).
perch_status check_device_error(perch_ctx* c);
bool finite(float x);
uint32_t next_pow2(uint64_t x);
perch_status clip_roi(perch_ctx* c, const SceneRec& s, const int32_t* roi, int out[4]);
int mark_words_for(const SceneRec& s, int label, const int roi[4], int cap_bits);
perch_status fit_config(perch_ctx* c, int mark_words, perch::ScoreConfig* cfg);
perch_status scratch_init(perch_ctx* c, ScoreScratch& X);
void scratch_free(perch_ctx* c, ScoreScratch& X);
// PERCH_E_BUSY (with a message) while a server runs on the context.
perch_status refuse_while_serving(perch_ctx* c);
// Remember an asynchronous call on stream st that reads scene_id and/or
// mesh_id (-1: none), so that releasing them waits for it to finish.
perch_status note_async_use(perch_ctx* c, int32_t scene_id, int32_t mesh_id, cudaStream_t st);
// True while the object has users or unfinished asynchronous calls.
bool in_use(UseTrack& u);
// Add d (+1 / -1) to the users of a scene and a mesh (ids that exist).
void count_users(perch_ctx* c, int32_t scene_id, int32_t mesh_id, int d);
// Build the device description of one work item.
perch_status make_job(perch_ctx* c, int32_t scene_id, int32_t mesh_id, int32_t label,
                      const int32_t* roi, const float* poses, int32_t* costs, long long n,
                      perch::Job* J, int* mark_words, const SceneRec** scene, const MeshRec** mesh);
// Called by run_jobs right after job j's launch with the stream it went to,
// to enqueue work that needs only that job (the server's per-request
// read-back).
using AfterJob = std::function<cudaError_t(size_t, cudaStream_t)>;
// Launch the persistent scorer once per job, on stream st after every earlier
// run that used X (see the definition).
perch_status run_jobs(perch_ctx* c, ScoreScratch& X, const std::vector<perch::Job>& jobs, int mark_words,
                      const perch::ScoreConfig& cfg_in, cudaStream_t st, unsigned long long* dump,
                      const AfterJob* after_job = nullptr);

}  // namespace perch_host
