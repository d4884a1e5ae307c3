// libperch host side: the C ABI declared in include/perch.h.
//
// A context owns every device allocation it makes and charges each to its HBM
// budget.  Meshes and observations are copied once and stay resident; scoring
// calls launch the fused kernel (perch_kernels.cu) on the caller's stream or,
// in synchronous mode, on the context's own stream with staging copies.
#include "perch.h"
#include "perch_internal.cuh"

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <thread>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

namespace {

struct MeshRec {
    perch::DevMesh dm{};
    void* verts = nullptr;
    void* tris = nullptr;
};

struct SceneRec {
    perch::DevScene ds{};
    perch_params params{};
    void* depth = nullptr;
    void* labels = nullptr;
    void* lab = nullptr;
    void* pts = nullptr;
    void* table = nullptr;
    void* nrm = nullptr;           // observed normals (GICP targets), made on first use
    int nrm_jump = -1;             // the normal_max_jump_units they were made with
    void* near = nullptr;          // near-cell bitmap (DevScene::near_bits)
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

}  // namespace

struct perch_ctx {
    int device = 0;
    uint64_t budget = 0;
    uint64_t used = 0;
    std::unordered_map<void*, size_t> allocs;
    std::map<int32_t, MeshRec> meshes;
    std::map<int32_t, SceneRec> scenes;
    int32_t next_id = 1;
    std::string err;
    cudaStream_t stream = nullptr;
    void* stage = nullptr;
    size_t stage_bytes = 0;
    int* d_err = nullptr;
    unsigned long long* d_best_partial = nullptr;   // 3 words per block, 1024 blocks
    unsigned* d_best_ticket = nullptr;
    long long* d_best_index = nullptr;
    int32_t* d_best_cost = nullptr;
    ScoreScratch plain;                    // scratch of the context's own scoring launches
    std::map<uint64_t, perch::ScoreConfig> tuned;   // autotuner results by batch class
    perch::ScoreConfig cfg{256, 8192, 1 << 16};
};

struct perch_batch_graph {
    perch_ctx* ctx = nullptr;
    unsigned* next = nullptr;              // the graph's own counters and slot mask
    void* vcache = nullptr;                // and vertex-cache pool
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

perch_status fail(perch_ctx* c, perch_status st, const char* fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return st;
}

perch_status cuda_fail(perch_ctx* c, cudaError_t e, const char* what)
{
    cudaGetLastError();
    return fail(c, PERCH_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

perch_status dalloc(perch_ctx* c, size_t bytes, void** p)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (c->budget && c->used + bytes > c->budget)
        return fail(c, PERCH_E_BUDGET, "allocation of %zu bytes exceeds the HBM budget (%llu of %llu used)",
                    bytes, (unsigned long long)c->used, (unsigned long long)c->budget);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, PERCH_E_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    c->allocs[*p] = bytes;
    c->used += bytes;
    return PERCH_OK;
}

void dfree(perch_ctx* c, void* p)
{
    if (!p) return;
    auto it = c->allocs.find(p);
    if (it != c->allocs.end()) {
        c->used -= it->second;
        c->allocs.erase(it);
    }
    cudaFree(p);
}

perch_status ensure_stage(perch_ctx* c, size_t bytes)
{
    if (c->stage_bytes >= bytes) return PERCH_OK;
    dfree(c, c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
    size_t want = std::max(bytes, (size_t)1 << 20);
    perch_status st = dalloc(c, want, &c->stage);
    if (st == PERCH_OK) c->stage_bytes = want;
    return st;
}

// Read and clear the device error word (synchronous).
perch_status check_device_error(perch_ctx* c)
{
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading the device error word");
    if (h == 0) return PERCH_OK;
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    cudaStreamSynchronize(c->stream);
    if (h == perch::kErrSourceCap)
        return fail(c, PERCH_E_INVALID, "a hypothesis' GICP source cloud exceeded max_source_points");
    return fail(c, PERCH_E_CUDA, "kernel invariant violated (flags 0x%x)", h);
}

bool finite(float x) { return std::isfinite(x); }

uint32_t next_pow2(uint64_t x)
{
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return (uint32_t)p;
}

perch_status clip_roi(perch_ctx* c, const SceneRec& s, const int32_t* roi, int out[4])
{
    int W = s.ds.W, H = s.ds.H;
    if (!roi) {
        out[0] = 0; out[1] = 0; out[2] = W; out[3] = H;
        return PERCH_OK;
    }
    out[0] = std::max(0, roi[0]);
    out[1] = std::max(0, roi[1]);
    out[2] = std::min(W, roi[2]);
    out[3] = std::min(H, roi[3]);
    if (out[2] < out[0]) out[2] = out[0];
    if (out[3] < out[1]) out[3] = out[1];
    (void)c;
    return PERCH_OK;
}

// Capacity of the shared-memory bitset that marks nearest neighbours inside
// the admissible box.  Boxes larger than this are processed in row bands (each
// band repeats the render and search), so the capacity only trades shared
// memory against that rare repetition.  At least one image row always fits.
constexpr int kMarkBitsDefault = 1 << 16;

int mark_words_for(const SceneRec& s, int label, const int roi[4], int cap_bits)
{
    long long bits = label >= 0 ? (long long)(roi[2] - roi[0]) * (roi[3] - roi[1])
                                : (long long)s.ds.W * s.ds.H;
    bits = std::min<long long>(bits, cap_bits);
    bits = std::max<long long>(bits, s.ds.W);
    return (int)(((bits + 31) / 32 + 2) & ~1ll);   // even: keeps the later 8-byte arrays aligned
}

// Fit the z-buffer into the opt-in shared memory limit of the device.
// Shrink the z-buffer of *cfg (the caller's launch shape) until the block's
// shared memory fits the device.
perch_status fit_config(perch_ctx* c, int mark_words, perch::ScoreConfig* cfg)
{
    int max_optin = 0;
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (max_optin <= 0) max_optin = 48 * 1024;
    while (perch::score_smem_bytes(*cfg, mark_words) > (size_t)max_optin && cfg->zcap_words > 1024)
        cfg->zcap_words /= 2;
    if (perch::score_smem_bytes(*cfg, mark_words) > (size_t)max_optin)
        return fail(c, PERCH_E_INVALID, "admissible-set bitset (%d words) does not fit in shared memory",
                    mark_words);
    return PERCH_OK;
}

perch_status scratch_init(perch_ctx* c, ScoreScratch& X)
{
    cudaError_t e = cudaEventCreateWithFlags(&X.last, cudaEventDisableTiming);
    if (!e) e = cudaEventCreateWithFlags(&X.fork, cudaEventDisableTiming);
    for (int i = 0; i < kSideStreams && !e; ++i) {
        e = cudaStreamCreateWithFlags(&X.side[i], cudaStreamNonBlocking);
        if (!e) e = cudaEventCreateWithFlags(&X.join[i], cudaEventDisableTiming);
    }
    if (!e) e = cudaEventRecord(X.last, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "scratch streams");
    return PERCH_OK;
}

void scratch_free(perch_ctx* c, ScoreScratch& X)
{
    if (X.last) cudaEventSynchronize(X.last);
    dfree(c, X.next);
    dfree(c, X.vcache);
    dfree(c, X.src);
    for (int i = 0; i < kSideStreams; ++i) {
        if (X.side[i]) cudaStreamDestroy(X.side[i]);
        if (X.join[i]) cudaEventDestroy(X.join[i]);
    }
    if (X.fork) cudaEventDestroy(X.fork);
    if (X.last) cudaEventDestroy(X.last);
    X = ScoreScratch{};
}

// Build the device description of one work item.
perch_status make_job(perch_ctx* c, int32_t scene_id, int32_t mesh_id, int32_t label,
                      const int32_t* roi, const float* poses, int32_t* costs, long long n,
                      perch::Job* J, int* mark_words, const SceneRec** scene, const MeshRec** mesh)
{
    auto si = c->scenes.find(scene_id);
    if (si == c->scenes.end()) return fail(c, PERCH_E_NOTFOUND, "unknown scene %d", scene_id);
    auto mi = c->meshes.find(mesh_id);
    if (mi == c->meshes.end()) return fail(c, PERCH_E_NOTFOUND, "unknown mesh %d", mesh_id);
    if (label < -1) return fail(c, PERCH_E_INVALID, "label must be -1 or >= 0");
    if (label >= 0 && !si->second.labels)
        return fail(c, PERCH_E_INVALID, "label %d given but the observation has no labels", label);
    if (n < 0) return fail(c, PERCH_E_INVALID, "n < 0");
    int r[4];
    clip_roi(c, si->second, roi, r);
    *J = perch::Job{};
    J->sc = si->second.ds;
    J->m = mi->second.dm;
    J->label = label;
    for (int i = 0; i < 4; ++i) J->roi[i] = r[i];
    J->poses = poses;
    J->costs = costs;
    J->n = n;
    *mark_words = mark_words_for(si->second, label, r, c->cfg.mark_bits);
    if (scene) *scene = &si->second;
    if (mesh) *mesh = &mi->second;
    return PERCH_OK;
}

// Launch the persistent scorer once per job, on stream st after every
// earlier run that used X.  Each launch gets the whole resident grid; with
// several jobs the launches go round-robin over X's side streams, so the
// blocks of job j+1 start on the SMs that job j's blocks leave at its tail,
// and every job keeps its fields in the parameter bank.
// after_job (optional) is called right after job j's launch with the stream
// it went to, to enqueue work that needs only that job (the server's
// per-request read-back).
using AfterJob = std::function<cudaError_t(size_t, cudaStream_t)>;

perch_status run_jobs(perch_ctx* c, ScoreScratch& X, const std::vector<perch::Job>& jobs,
                      int mark_words, const perch::ScoreConfig& cfg_in, cudaStream_t st,
                      unsigned long long* dump, const AfterJob* after_job = nullptr)
{
    long long total = 0;
    int max_verts = 0;
    bool small_images = true;
    for (const auto& j : jobs) {
        if (j.n > 0xFFFFFFF0ll) return fail(c, PERCH_E_INVALID, "more than 2^32 hypotheses in one item");
        total += j.n;
        max_verts = std::max(max_verts, j.m.n_verts);
        small_images = small_images && j.sc.W <= 1023 && j.sc.H <= 1023;
    }
    if (total == 0) return PERCH_OK;
    perch::ScoreConfig cfg = cfg_in;
    perch_status stt = fit_config(c, mark_words, &cfg);
    if (stt != PERCH_OK) return stt;
    const int grid = perch::score_grid(cfg, mark_words);
    if (grid <= 0) {
        cudaGetLastError();
        return fail(c, PERCH_E_CUDA, "scoring kernel does not fit on the device");
    }
    // vertex caches: a pool of one slot per resident block, used when snapped
    // coordinates fit in int16
    long long vstride = 0;
    if (small_images) {
        vstride = ((long long)max_verts + 31) / 32 * 32;
        size_t need = (size_t)grid * vstride * sizeof(unsigned long long);
        if (need > X.vcache_bytes) {
            cudaEventSynchronize(X.last);
            dfree(c, X.vcache);
            X.vcache = nullptr;
            X.vcache_bytes = 0;
            if ((stt = dalloc(c, need, &X.vcache)) != PERCH_OK) return stt;
            X.vcache_bytes = need;
        }
    }
    const size_t nj = jobs.size();
    const size_t mask_words = ((size_t)grid + 31) / 32;
    const size_t words = nj + mask_words;
    if (words > X.next_words) {
        cudaEventSynchronize(X.last);
        dfree(c, X.next);
        X.next = nullptr;
        X.next_words = 0;
        void* p = nullptr;
        if ((stt = dalloc(c, std::max<size_t>(words, 64) * sizeof(unsigned), &p)) != PERCH_OK) return stt;
        X.next = (unsigned*)p;
        X.next_words = std::max<size_t>(words, 64);
    }
    perch::ScoreArgs a{};
    a.zcap_words = cfg.zcap_words;
    a.mark_words = mark_words;
    a.dump = dump;
    a.err = c->d_err;
    a.vcache = vstride ? (unsigned long long*)X.vcache : nullptr;
    a.vstride = vstride;
    a.vmask = X.next + nj;
    a.vslots = grid;
    cudaError_t e = cudaStreamWaitEvent(st, X.last, 0);
    if (!e) e = cudaMemsetAsync(X.next, 0, words * sizeof(unsigned), st);
    const bool fan = nj > 1;
    const int nside = (int)std::min<size_t>(nj, kSideStreams);
    if (!e && fan) e = cudaEventRecord(X.fork, st);
    for (int k = 0; k < nside && fan && !e; ++k) e = cudaStreamWaitEvent(X.side[k], X.fork, 0);
    for (size_t j = 0; j < nj && !e; ++j) {
        a.job = jobs[j];
        a.n = jobs[j].n;
        a.next = X.next + j;
        cudaStream_t js = fan ? X.side[j % kSideStreams] : st;
        e = perch::launch_score(a, cfg, grid, js);
        if (!e && after_job) e = (*after_job)(j, js);
    }
    for (int k = 0; k < nside && fan && !e; ++k) {
        e = cudaEventRecord(X.join[k], X.side[k]);
        if (!e) e = cudaStreamWaitEvent(st, X.join[k], 0);
    }
    if (!e) e = cudaEventRecord(X.last, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "scoring launch");
    return PERCH_OK;
}

// Near-cell bitmap of an observation: one bit per hash cell of the observed
// points' cell box grown by one, set iff one of the cell's 27 neighbours holds
// a point.  Skipped (no filter) when the box exceeds 2^27 cells.
perch_status build_near_cells(perch_ctx* c, SceneRec& s)
{
    perch::DevScene& d = s.ds;
    d.near_bits = nullptr;
    if (d.n_pts <= 0) return PERCH_OK;
    void* bnd = nullptr;
    perch_status st = dalloc(c, 6 * sizeof(int), &bnd);
    if (st != PERCH_OK) return st;
    const int init[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
    int got[6];
    cudaError_t e = cudaMemcpyAsync(bnd, init, sizeof(init), cudaMemcpyHostToDevice, c->stream);
    if (!e) e = perch::launch_cell_bounds(d, (int*)bnd, c->stream);
    if (!e) e = cudaMemcpyAsync(got, bnd, sizeof(got), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    dfree(c, bnd);
    if (e) return cuda_fail(c, e, "near-cell bounds");
    long long cells = 1;
    for (int a = 0; a < 3; ++a) {
        d.near_lo[a] = got[a] - 1;
        d.near_n[a] = got[3 + a] - got[a] + 3;
        cells *= d.near_n[a];
    }
    if (cells > (1ll << 27)) return PERCH_OK;
    const size_t bytes = (size_t)((cells + 31) / 32) * 4;
    void* occ = nullptr;
    if ((st = dalloc(c, bytes, &s.near)) != PERCH_OK) return st;
    if ((st = dalloc(c, bytes, &occ)) != PERCH_OK) return st;
    e = cudaMemsetAsync(s.near, 0, bytes, c->stream);
    if (!e) e = cudaMemsetAsync(occ, 0, bytes, c->stream);
    if (!e) e = perch::launch_near_cells(d, (uint32_t*)occ, (uint32_t*)s.near, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    dfree(c, occ);
    if (e) return cuda_fail(c, e, "near-cell bitmap");
    d.near_bits = (const uint32_t*)s.near;
    return PERCH_OK;
}

// Grow a scratch buffer of X (after every earlier run that used X).
perch_status grow(perch_ctx* c, ScoreScratch& X, void** buf, size_t* have, size_t need)
{
    if (need <= *have) return PERCH_OK;
    cudaEventSynchronize(X.last);
    dfree(c, *buf);
    *buf = nullptr;
    *have = 0;
    perch_status st = dalloc(c, need, buf);
    if (st == PERCH_OK) *have = need;
    return st;
}

// Launch the GICP refinement of one job on stream st, after every earlier run
// that used X (they share the counter, the slot pool and the caches).
perch_status run_gicp(perch_ctx* c, ScoreScratch& X, const perch::Job& J, const perch_gicp_params& gp,
                      const float4* nrm, float* poses_out, int32_t* info, cudaStream_t st)
{
    if (J.n == 0) return PERCH_OK;
    if (J.n > 0xFFFFFFF0ll) return fail(c, PERCH_E_INVALID, "more than 2^32 hypotheses in one call");
    int dev = 0, max_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int zcap = c->cfg.zcap_words;
    while (perch::gicp_smem_bytes(zcap) > (size_t)max_optin && zcap > 1024) zcap /= 2;
    const int grid = perch::gicp_grid(zcap);
    if (grid <= 0) {
        cudaGetLastError();
        return fail(c, PERCH_E_CUDA, "refinement kernel does not fit on the device");
    }
    const long long s = J.sc.stride;
    const long long lattice = ((J.roi[2] - J.roi[0] + s - 1) / s) * ((J.roi[3] - J.roi[1] + s - 1) / s);
    long long cap = gp.max_source_points > 0 ? gp.max_source_points : 65536;
    cap = std::max(1ll, std::min(cap, lattice));
    perch_status stt = grow(c, X, &X.src, &X.src_bytes, (size_t)grid * (size_t)cap * 2 * sizeof(float4));
    if (stt != PERCH_OK) return stt;
    long long vstride = 0;
    if (J.sc.W <= 1023 && J.sc.H <= 1023) {
        vstride = ((long long)J.m.n_verts + 31) / 32 * 32;
        stt = grow(c, X, &X.vcache, &X.vcache_bytes, (size_t)grid * vstride * sizeof(unsigned long long));
        if (stt != PERCH_OK) return stt;
    }
    const size_t words = 1 + ((size_t)grid + 31) / 32;
    if (words > X.next_words) {
        size_t have = X.next_words * sizeof(unsigned);
        void* p = X.next;
        stt = grow(c, X, &p, &have, std::max<size_t>(words, 64) * sizeof(unsigned));
        X.next = (unsigned*)p;
        X.next_words = have / sizeof(unsigned);
        if (stt != PERCH_OK) return stt;
    }
    perch::GicpArgs a{};
    a.job = J;
    a.n = J.n;
    a.zcap_words = zcap;
    a.err = c->d_err;
    a.next = X.next;
    a.smask = X.next + 1;
    a.slots = grid;
    a.src = (float4*)X.src;
    a.src_cap = (int)cap;
    a.vcache = vstride ? (unsigned long long*)X.vcache : nullptr;
    a.vstride = vstride;
    a.nrm = nrm;
    a.max_iters = gp.max_iterations;
    a.min_corr = gp.min_correspondences;
    a.epsilon = gp.epsilon;
    a.stop_rot = gp.stop_rotation_rad;
    a.stop_trans = gp.stop_translation_m;
    a.poses_out = poses_out;
    a.info = info;
    cudaError_t e = cudaStreamWaitEvent(st, X.last, 0);
    if (!e) e = cudaMemsetAsync(X.next, 0, words * sizeof(unsigned), st);
    if (!e) e = perch::launch_gicp(a, grid, st);
    if (!e) e = cudaEventRecord(X.last, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "refinement launch");
    return PERCH_OK;
}

}  // namespace

extern "C" {

perch_status perch_default_params(perch_params* p)
{
    if (!p) return PERCH_E_INVALID;
    p->delta_m = 0.01f;
    p->tau_c = 12.5f;
    p->color_check = 1;
    p->stride = 1;
    p->occ_margin_units = 100;
    p->z_near_m = 0.05f;
    p->jo_mode = 0;
    return PERCH_OK;
}

perch_status perch_create(perch_ctx** out, int32_t device, uint64_t hbm_budget_bytes)
{
    if (!out) return PERCH_E_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
        cudaGetLastError();
        return PERCH_E_CUDA;
    }
    if (device < 0 || device >= ndev) return PERCH_E_INVALID;
    perch_ctx* c = new (std::nothrow) perch_ctx();
    if (!c) return PERCH_E_NOMEM;
    c->device = device;
    c->budget = hbm_budget_bytes;
    DeviceGuard g(device);
    perch_status st = PERCH_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) st = cuda_fail(c, e, "cudaStreamCreate");
    void* p = nullptr;
    if (st == PERCH_OK && (st = dalloc(c, sizeof(int), &p)) == PERCH_OK) c->d_err = (int*)p;
    if (st == PERCH_OK && (st = dalloc(c, sizeof(unsigned long long) * 3 * 1024, &p)) == PERCH_OK)
        c->d_best_partial = (unsigned long long*)p;
    if (st == PERCH_OK && (st = dalloc(c, 64, &p)) == PERCH_OK) {
        c->d_best_ticket = (unsigned*)p;
        c->d_best_index = (long long*)((char*)p + 16);
        c->d_best_cost = (int32_t*)((char*)p + 32);
    }
    if (st == PERCH_OK) st = scratch_init(c, c->plain);
    if (st == PERCH_OK) {
        cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
        cudaMemsetAsync(c->d_best_ticket, 0, 64, c->stream);
        if ((e = perch::init_device_tables(c->stream)) != cudaSuccess) st = cuda_fail(c, e, "init tables");
    }
    if (st == PERCH_OK && (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        st = cuda_fail(c, e, "perch_create");
    if (st != PERCH_OK) {
        perch_destroy(c);
        return st;
    }
    *out = c;
    return PERCH_OK;
}

perch_status perch_destroy(perch_ctx* c)
{
    if (!c) return PERCH_OK;
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    scratch_free(c, c->plain);
    for (auto& kv : c->allocs) cudaFree(kv.first);
    c->allocs.clear();
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return PERCH_OK;
}

const char* perch_last_error(const perch_ctx* c)
{
    return c ? c->err.c_str() : "null context";
}

uint64_t perch_hbm_used(const perch_ctx* c)
{
    return c ? c->used : 0;
}

perch_status perch_load_mesh(perch_ctx* c, const float* verts_xyz, const uint8_t* rgb,
                             int32_t n_verts, const int32_t* tris, int32_t n_tris,
                             float vol_radius_m, float vol_height_m, int32_t* mesh_id)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (!verts_xyz || !rgb || !tris || !mesh_id || n_verts < 1 || n_tris < 1)
        return fail(c, PERCH_E_INVALID, "perch_load_mesh: null pointer or empty mesh");
    if (!finite(vol_radius_m) || !finite(vol_height_m) || vol_radius_m < 0 || vol_height_m < 0)
        return fail(c, PERCH_E_INVALID, "perch_load_mesh: bad admissible cylinder");
    std::vector<float> v4((size_t)n_verts * 4);
    MeshRec rec;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int32_t i = 0; i < n_verts; ++i) {
        for (int k = 0; k < 3; ++k) {
            float x = verts_xyz[3 * i + k];
            if (!finite(x)) return fail(c, PERCH_E_INVALID, "perch_load_mesh: non-finite vertex %d", i);
            v4[4 * i + k] = x;
            lo[k] = std::min(lo[k], x);
            hi[k] = std::max(hi[k], x);
        }
        uint32_t packed = (uint32_t)rgb[3 * i] | ((uint32_t)rgb[3 * i + 1] << 8) |
                          ((uint32_t)rgb[3 * i + 2] << 16);
        std::memcpy(&v4[4 * i + 3], &packed, 4);
    }
    std::vector<int32_t> t4((size_t)n_tris * 4);
    for (int32_t i = 0; i < n_tris; ++i) {
        for (int k = 0; k < 3; ++k) {
            int32_t x = tris[3 * i + k];
            if (x < 0 || x >= n_verts)
                return fail(c, PERCH_E_INVALID, "perch_load_mesh: triangle %d has index %d out of range", i, x);
            t4[4 * i + k] = x;
        }
        t4[4 * i + 3] = 0;
    }
    DeviceGuard g(c->device);
    perch_status st = dalloc(c, v4.size() * sizeof(float), &rec.verts);
    if (st != PERCH_OK) return st;
    if ((st = dalloc(c, t4.size() * sizeof(int32_t), &rec.tris)) != PERCH_OK) {
        dfree(c, rec.verts);
        return st;
    }
    cudaError_t e = cudaMemcpyAsync(rec.verts, v4.data(), v4.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rec.tris, t4.data(), t4.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        dfree(c, rec.verts);
        dfree(c, rec.tris);
        return cuda_fail(c, e, "perch_load_mesh upload");
    }
    rec.dm.verts = (const float4*)rec.verts;
    rec.dm.tris = (const int4*)rec.tris;
    rec.dm.n_verts = n_verts;
    rec.dm.n_tris = n_tris;
    rec.dm.vol_r = vol_radius_m;
    rec.dm.vol_h = vol_height_m;
    for (int k = 0; k < 3; ++k) {
        rec.dm.lo[k] = lo[k];
        rec.dm.hi[k] = hi[k];
    }
    int32_t id = c->next_id++;
    c->meshes[id] = rec;
    *mesh_id = id;
    return PERCH_OK;
}

perch_status perch_release_mesh(perch_ctx* c, int32_t mesh_id)
{
    if (!c) return PERCH_E_INVALID;
    auto it = c->meshes.find(mesh_id);
    if (it == c->meshes.end()) return fail(c, PERCH_E_NOTFOUND, "unknown mesh %d", mesh_id);
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    dfree(c, it->second.verts);
    dfree(c, it->second.tris);
    c->meshes.erase(it);
    return PERCH_OK;
}

perch_status perch_set_observation(perch_ctx* c, const uint16_t* depth, const uint8_t* rgb,
                                   const int32_t* labels, int32_t W, int32_t H, float fx,
                                   float fy, float cx, float cy, const perch_params* params,
                                   int32_t* scene_id)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (!depth || !rgb || !params || !scene_id)
        return fail(c, PERCH_E_INVALID, "perch_set_observation: null pointer");
    if (W < 1 || H < 1 || (long long)W * H > 466033)
        return fail(c, PERCH_E_INVALID, "perch_set_observation: image %dx%d outside 1 <= W*H <= 466033", W, H);
    if (!finite(fx) || !finite(fy) || !finite(cx) || !finite(cy) || fx <= 0 || fy <= 0)
        return fail(c, PERCH_E_INVALID, "perch_set_observation: bad intrinsics");
    const perch_params& p = *params;
    if (!finite(p.delta_m) || p.delta_m < 1e-4f || p.delta_m > 1.0f || !finite(p.tau_c) || p.tau_c < 0 ||
        (p.color_check != 0 && p.color_check != 1) || p.stride < 1 || p.occ_margin_units < -1 ||
        !finite(p.z_near_m) || p.z_near_m <= 0 || (p.jo_mode != 0 && p.jo_mode != 1))
        return fail(c, PERCH_E_INVALID, "perch_set_observation: parameters out of range");
    const float cell = p.delta_m * perch::kCellGrow;
    const double zmax = 65535.0 / 10000.0;
    double xmax = std::max(std::fabs(0.0 - cx), std::fabs(W - 1.0 - cx)) * zmax / fx;
    double ymax = std::max(std::fabs(0.0 - cy), std::fabs(H - 1.0 - cy)) * zmax / fy;
    double lim = perch::kMaxCellCoord * (double)cell * 0.99;
    if (xmax > lim || ymax > lim || zmax > lim)
        return fail(c, PERCH_E_INVALID, "perch_set_observation: delta too small for the field of view");

    long long npx = (long long)W * H;
    long long n_valid = 0;
    for (long long i = 0; i < npx; ++i) {
        int u = (int)(i % W), v = (int)(i / W);
        if (depth[i] != 0 && u % p.stride == 0 && v % p.stride == 0) ++n_valid;
    }
    uint32_t cap = next_pow2(std::max<long long>(1024, 2 * n_valid));
    uint32_t n_tiles = (cap + 1023) / 1024;

    DeviceGuard g(c->device);
    SceneRec s;
    s.params = p;
    perch_status st = PERCH_OK;
    void *d_rgb = nullptr, *slot = nullptr, *keys = nullptr, *count = nullptr, *cursor = nullptr,
         *start = nullptr, *nvalid = nullptr, *big = nullptr;
    auto cleanup_scratch = [&]() {
        dfree(c, d_rgb); dfree(c, slot); dfree(c, keys); dfree(c, count);
        dfree(c, cursor); dfree(c, start); dfree(c, nvalid); dfree(c, big);
    };
    auto cleanup_scene = [&]() {
        dfree(c, s.depth); dfree(c, s.labels); dfree(c, s.lab); dfree(c, s.pts); dfree(c, s.table); dfree(c, s.nrm);
        dfree(c, s.near);
    };
    if ((st = dalloc(c, npx * sizeof(uint16_t), &s.depth)) ||
        (labels && (st = dalloc(c, npx * sizeof(int32_t), &s.labels))) ||
        (st = dalloc(c, npx * sizeof(float4), &s.lab)) ||
        (st = dalloc(c, std::max<long long>(1, n_valid) * sizeof(float4), &s.pts)) ||
        (st = dalloc(c, (size_t)cap * sizeof(uint4), &big)) ||
        (st = dalloc(c, npx * 3, &d_rgb)) || (st = dalloc(c, npx * sizeof(int32_t), &slot)) ||
        (st = dalloc(c, (size_t)cap * 8, &keys)) || (st = dalloc(c, (size_t)cap * 4, &count)) ||
        (st = dalloc(c, ((size_t)cap + n_tiles) * 4, &cursor)) ||
        (st = dalloc(c, (size_t)cap * 4, &start)) || (st = dalloc(c, 2 * sizeof(int), &nvalid))) {
        cleanup_scratch();
        cleanup_scene();
        return st;
    }
    cudaError_t e = cudaMemcpyAsync(s.depth, depth, npx * sizeof(uint16_t), cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync(d_rgb, rgb, npx * 3, cudaMemcpyHostToDevice, c->stream);
    if (!e && labels) e = cudaMemcpyAsync(s.labels, labels, npx * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
    perch::DevScene& d = s.ds;
    d.W = W; d.H = H; d.fx = fx; d.fy = fy; d.cx = cx; d.cy = cy;
    d.delta = p.delta_m;
    d.delta2 = p.delta_m * p.delta_m;
    d.cell = cell;
    d.tau_c = p.tau_c;
    d.z_near = p.z_near_m;
    d.color_check = p.color_check;
    d.stride = p.stride;
    d.occ_margin = p.occ_margin_units;
    d.jo_mode = p.jo_mode;
    d.depth = (const uint16_t*)s.depth;
    d.labels = (const int32_t*)s.labels;
    d.lab = (const float4*)s.lab;
    d.pts = (const float4*)s.pts;
    d.table = (const uint4*)big;
    d.table_mask = cap - 1;
    d.n_pts = (int)n_valid;
    perch::BuildBuffers b{};
    b.slot_of_pixel = (int32_t*)slot;
    b.keys = (unsigned long long*)keys;
    b.count = (uint32_t*)count;
    b.cursor = (uint32_t*)cursor;
    b.start = (uint32_t*)start;
    b.n_valid = (int*)nvalid;
    b.lab = (float4*)s.lab;
    b.pts = (float4*)s.pts;
    b.table = (uint4*)big;
    if (!e) e = perch::launch_build(d, b, cap, (const uint8_t*)d_rgb, c->d_err, c->stream);
    int got[2] = {-1, -1};
    if (!e) e = cudaMemcpyAsync(got, nvalid, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) {
        cleanup_scratch();
        cleanup_scene();
        return cuda_fail(c, e, "perch_set_observation build");
    }
    if ((st = check_device_error(c)) != PERCH_OK || got[0] != n_valid) {
        cleanup_scratch();
        cleanup_scene();
        return st != PERCH_OK ? st : fail(c, PERCH_E_CUDA, "observation build counted %d of %lld points", got[0], n_valid);
    }
    // compact the hash table to eight times its occupied cells: most of the
    // 27 lookups per query are misses, and a load factor of at most 1/8 ends
    // nearly all of them at the first slot
    uint32_t cap_small = next_pow2(std::max<long long>(64, 8ll * got[1]));
    if ((st = dalloc(c, (size_t)cap_small * sizeof(uint4), &s.table)) != PERCH_OK) {
        cleanup_scratch();
        cleanup_scene();
        return st;
    }
    e = perch::launch_compact_table((const uint4*)big, cap, (uint4*)s.table, cap_small, c->d_err, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    cleanup_scratch();
    if (e) {
        cleanup_scene();
        return cuda_fail(c, e, "perch_set_observation table");
    }
    if ((st = check_device_error(c)) != PERCH_OK) {
        cleanup_scene();
        return st;
    }
    d.table = (const uint4*)s.table;
    d.table_mask = cap_small - 1;
    if ((st = build_near_cells(c, s)) != PERCH_OK) {
        cleanup_scene();
        return st;
    }
    int32_t id = c->next_id++;
    c->scenes[id] = s;
    *scene_id = id;
    return PERCH_OK;
}

perch_status perch_release_scene(perch_ctx* c, int32_t scene_id)
{
    if (!c) return PERCH_E_INVALID;
    auto it = c->scenes.find(scene_id);
    if (it == c->scenes.end()) return fail(c, PERCH_E_NOTFOUND, "unknown scene %d", scene_id);
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    SceneRec& s = it->second;
    dfree(c, s.depth); dfree(c, s.labels); dfree(c, s.lab); dfree(c, s.pts); dfree(c, s.table); dfree(c, s.nrm);
        dfree(c, s.near);
    c->scenes.erase(it);
    return PERCH_OK;
}

perch_status perch_score_hypotheses(perch_ctx* c, int32_t scene_id, int32_t mesh_id,
                                    int32_t label, const int32_t* roi, const float* poses,
                                    int64_t n, int32_t* costs, void* cuda_stream)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (n < 0) return fail(c, PERCH_E_INVALID, "n < 0");
    if (n == 0) return PERCH_OK;
    if (!poses || !costs) return fail(c, PERCH_E_INVALID, "null poses or costs");
    DeviceGuard g(c->device);
    perch::Job J;
    int mw;
    perch_status st = make_job(c, scene_id, mesh_id, label, roi, poses, costs, n, &J, &mw, nullptr, nullptr);
    if (st != PERCH_OK) return st;
    if (cuda_stream) {
        std::vector<perch::Job> jobs(1, J);
        return run_jobs(c, c->plain, jobs, mw, c->cfg, (cudaStream_t)cuda_stream, nullptr);
    }
    const long long chunk = 1 << 20;
    if ((st = ensure_stage(c, (size_t)std::min<long long>(n, chunk) * (48 + 8))) != PERCH_OK) return st;
    float* d_poses = (float*)c->stage;
    int32_t* d_costs = (int32_t*)((char*)c->stage + (size_t)std::min<long long>(n, chunk) * 48);
    for (long long off = 0; off < n; off += chunk) {
        long long k = std::min(chunk, n - off);
        cudaError_t e = cudaMemcpyAsync(d_poses, poses + 12 * off, k * 48, cudaMemcpyHostToDevice, c->stream);
        if (e) return cuda_fail(c, e, "perch_score_hypotheses upload");
        std::vector<perch::Job> jobs(1, J);
        jobs[0].poses = d_poses;
        jobs[0].costs = d_costs;
        jobs[0].n = k;
        if ((st = run_jobs(c, c->plain, jobs, mw, c->cfg, c->stream, nullptr)) != PERCH_OK) return st;
        e = cudaMemcpyAsync(costs + 2 * off, d_costs, k * 8, cudaMemcpyDeviceToHost, c->stream);
        if (!e) e = cudaStreamSynchronize(c->stream);
        if (e) return cuda_fail(c, e, "perch_score_hypotheses");
    }
    return check_device_error(c);
}

// Validate a batch and turn it into jobs; `base_poses` / `base_costs` are the
// arrays the item offsets index.
static perch_status batch_jobs(perch_ctx* c, const perch_work_item* items, int32_t n_items,
                               const float* base_poses, int32_t* base_costs,
                               std::vector<perch::Job>* jobs, int* mark_words, long long* total)
{
    if (!items || n_items < 0) return fail(c, PERCH_E_INVALID, "bad item list");
    jobs->clear();
    *mark_words = 0;
    *total = 0;
    std::vector<std::pair<long long, long long>> spans;
    for (int32_t i = 0; i < n_items; ++i) {
        const perch_work_item& it = items[i];
        if (it.n < 0 || it.pose_offset < 0) return fail(c, PERCH_E_INVALID, "item %d: negative n or offset", i);
        if (it.n == 0) continue;
        const int32_t* roi = (it.roi[2] > it.roi[0] && it.roi[3] > it.roi[1]) ? it.roi : nullptr;
        perch::Job J;
        int mw;
        perch_status st = make_job(c, it.scene_id, it.mesh_id, it.label, roi, base_poses + 12 * it.pose_offset,
                                   base_costs + 2 * it.pose_offset, it.n, &J, &mw, nullptr, nullptr);
        if (st != PERCH_OK) return st;
        jobs->push_back(J);
        *mark_words = std::max(*mark_words, mw);
        *total += it.n;
        spans.push_back({it.pose_offset, it.pose_offset + it.n});
    }
    std::sort(spans.begin(), spans.end());
    for (size_t i = 1; i < spans.size(); ++i)
        if (spans[i].first < spans[i - 1].second) return fail(c, PERCH_E_INVALID, "batch items overlap");
    return PERCH_OK;
}

perch_status perch_score_batch(perch_ctx* c, const perch_work_item* items, int32_t n_items,
                               const float* poses, int32_t* costs, void* cuda_stream)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (!poses || !costs) return fail(c, PERCH_E_INVALID, "null poses or costs");
    DeviceGuard g(c->device);
    std::vector<perch::Job> jobs;
    int mw;
    long long total;
    long long extent = 0;
    for (int32_t i = 0; items && i < n_items; ++i) extent = std::max<long long>(extent, items[i].pose_offset + items[i].n);
    if (cuda_stream) {
        perch_status st = batch_jobs(c, items, n_items, poses, costs, &jobs, &mw, &total);
        if (st != PERCH_OK) return st;
        return run_jobs(c, c->plain, jobs, mw, c->cfg, (cudaStream_t)cuda_stream, nullptr);
    }
    perch_status st = ensure_stage(c, (size_t)std::max<long long>(1, extent) * (48 + 8));
    if (st != PERCH_OK) return st;
    float* d_poses = (float*)c->stage;
    int32_t* d_costs = (int32_t*)((char*)c->stage + (size_t)extent * 48);
    if ((st = batch_jobs(c, items, n_items, d_poses, d_costs, &jobs, &mw, &total)) != PERCH_OK) return st;
    cudaError_t e = cudaMemcpyAsync(d_poses, poses, extent * 48, cudaMemcpyHostToDevice, c->stream);
    if (e) return cuda_fail(c, e, "perch_score_batch upload");
    if ((st = run_jobs(c, c->plain, jobs, mw, c->cfg, c->stream, nullptr)) != PERCH_OK) return st;
    for (int32_t i = 0; i < n_items && !e; ++i)
        if (items[i].n > 0)
            e = cudaMemcpyAsync(costs + 2 * items[i].pose_offset, d_costs + 2 * items[i].pose_offset,
                                items[i].n * 8, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "perch_score_batch");
    return check_device_error(c);
}

perch_status perch_best(perch_ctx* c, const int32_t* costs, const uint64_t* ids, int64_t n,
                        int64_t* best_index, int32_t* best_cost, void* cuda_stream)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (!costs || !best_index || !best_cost) return fail(c, PERCH_E_INVALID, "null pointer");
    if (n < 1 || n > 0x7FFFFFFFll) return fail(c, PERCH_E_INVALID, "n out of range");
    DeviceGuard g(c->device);
    perch::BestArgs a{};
    a.n = n;
    a.partial = c->d_best_partial;
    a.ticket = c->d_best_ticket;
    cudaError_t e;
    if (cuda_stream) {
        a.costs = costs;
        a.ids = (const unsigned long long*)ids;
        a.best_index = (long long*)best_index;
        a.best_cost = best_cost;
        if ((e = perch::launch_best(a, (cudaStream_t)cuda_stream)) != cudaSuccess)
            return cuda_fail(c, e, "perch_best launch");
        return PERCH_OK;
    }
    size_t need = (size_t)n * 8 + (ids ? (size_t)n * 8 : 0);
    perch_status st = ensure_stage(c, need);
    if (st != PERCH_OK) return st;
    int32_t* d_costs = (int32_t*)c->stage;
    unsigned long long* d_ids = ids ? (unsigned long long*)((char*)c->stage + (size_t)n * 8) : nullptr;
    e = cudaMemcpyAsync(d_costs, costs, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream);
    if (!e && ids) e = cudaMemcpyAsync(d_ids, ids, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream);
    a.costs = d_costs;
    a.ids = d_ids;
    a.best_index = c->d_best_index;
    a.best_cost = c->d_best_cost;
    if (!e) e = perch::launch_best(a, c->stream);
    long long bi = -1;
    int32_t bc = 0;
    if (!e) e = cudaMemcpyAsync(&bi, c->d_best_index, 8, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaMemcpyAsync(&bc, c->d_best_cost, 4, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return cuda_fail(c, e, "perch_best");
    *best_index = bi;
    *best_cost = bc;
    return PERCH_OK;
}

perch_status perch_set_launch_config(perch_ctx* c, int32_t threads, int32_t zbuf_words,
                                     int32_t mark_bits)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (mark_bits == 0) mark_bits = kMarkBitsDefault;
    if ((threads != 128 && threads != 256 && threads != 512) || zbuf_words < 1024 ||
        zbuf_words > 49152 || mark_bits < 1024 || mark_bits > (1 << 22))
        return fail(c, PERCH_E_INVALID, "launch config (%d threads, %d words, %d bits) out of range",
                    threads, zbuf_words, mark_bits);
    c->cfg.threads = threads;
    c->cfg.zcap_words = zbuf_words & ~3;
    c->cfg.mark_bits = mark_bits;
    return PERCH_OK;
}

perch_status perch_pose_proposals(perch_ctx* c, int32_t scene_id, int32_t mesh_id, int32_t label,
                                  const int32_t* bbox, int32_t M, int32_t N, int32_t K, float* poses,
                                  int32_t* z_range, void* cuda_stream)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (!bbox || !poses) return fail(c, PERCH_E_INVALID, "null bbox or poses");
    if (M < 1 || N < 1 || K < 1 || (long long)M * N * K > (1ll << 26))
        return fail(c, PERCH_E_INVALID, "proposal counts out of range");
    auto si = c->scenes.find(scene_id);
    if (si == c->scenes.end()) return fail(c, PERCH_E_NOTFOUND, "unknown scene %d", scene_id);
    auto mi = c->meshes.find(mesh_id);
    if (mi == c->meshes.end()) return fail(c, PERCH_E_NOTFOUND, "unknown mesh %d", mesh_id);
    if (label < 0 || !si->second.labels) return fail(c, PERCH_E_INVALID, "proposals need a label and labels");
    DeviceGuard g(c->device);
    perch::ProposalArgs a{};
    a.sc = si->second.ds;
    a.label = label;
    clip_roi(c, si->second, bbox, a.box);
    a.M = M; a.N = N; a.K = K;
    for (int k = 0; k < 3; ++k) a.centre[k] = 0.5f * (mi->second.dm.lo[k] + mi->second.dm.hi[k]);
    const long long n = (long long)M * N * K;
    perch_status st = ensure_stage(c, (size_t)n * 48 + 64);
    if (st != PERCH_OK) return st;
    a.zr = (unsigned*)((char*)c->stage + (size_t)n * 48);
    if (cuda_stream) {
        a.poses = poses;
        a.z_out = z_range;
        cudaError_t e = perch::launch_proposals(a, (cudaStream_t)cuda_stream);
        return e ? cuda_fail(c, e, "perch_pose_proposals") : PERCH_OK;
    }
    a.poses = (float*)c->stage;
    a.z_out = (int32_t*)(a.zr + 2);
    cudaError_t e = perch::launch_proposals(a, c->stream);
    if (!e) e = cudaMemcpyAsync(poses, a.poses, n * 48, cudaMemcpyDeviceToHost, c->stream);
    if (!e && z_range) e = cudaMemcpyAsync(z_range, a.z_out, 8, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    return e ? cuda_fail(c, e, "perch_pose_proposals") : PERCH_OK;
}

perch_status perch_default_gicp_params(perch_gicp_params* p)
{
    if (!p) return PERCH_E_INVALID;
    p->max_iterations = 10;
    p->epsilon = 1e-3f;
    p->normal_max_jump_units = 200;
    p->min_correspondences = 6;
    p->stop_rotation_rad = 1e-5f;
    p->stop_translation_m = 1e-5f;
    p->max_source_points = 0;
    return PERCH_OK;
}

perch_status perch_refine_hypotheses(perch_ctx* c, int32_t scene_id, int32_t mesh_id, int32_t label,
                                     const int32_t* roi, const float* poses, int64_t n,
                                     const perch_gicp_params* params, float* poses_out, int32_t* info,
                                     void* cuda_stream)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (n < 0) return fail(c, PERCH_E_INVALID, "n < 0");
    if (n == 0) return PERCH_OK;
    if (!poses || !poses_out || !params) return fail(c, PERCH_E_INVALID, "null poses, poses_out or params");
    const perch_gicp_params gp = *params;
    if (gp.max_iterations < 0 || gp.max_iterations > 1000)
        return fail(c, PERCH_E_INVALID, "max_iterations must be in [0, 1000]");
    if (!finite(gp.epsilon) || !(gp.epsilon > 0.0f) || !(gp.epsilon < 1.0f))
        return fail(c, PERCH_E_INVALID, "epsilon must be in (0, 1)");
    if (gp.normal_max_jump_units < 0 || gp.min_correspondences < 1 || gp.max_source_points < 0)
        return fail(c, PERCH_E_INVALID, "normal_max_jump_units, min_correspondences or max_source_points out of range");
    if (!finite(gp.stop_rotation_rad) || !finite(gp.stop_translation_m) || gp.stop_rotation_rad < 0.0f ||
        gp.stop_translation_m < 0.0f)
        return fail(c, PERCH_E_INVALID, "stop thresholds must be finite and >= 0");
    DeviceGuard g(c->device);
    perch::Job J;
    int mw;
    perch_status st = make_job(c, scene_id, mesh_id, label, roi, poses, nullptr, n, &J, &mw, nullptr, nullptr);
    if (st != PERCH_OK) return st;
    J.sc.jo_mode = 0;
    // observed normals of the scene for this jump threshold (made once, synchronously)
    SceneRec& S = c->scenes[scene_id];
    if (!S.nrm || S.nrm_jump != gp.normal_max_jump_units) {
        cudaEventSynchronize(c->plain.last);
        if (!S.nrm && (st = dalloc(c, (size_t)S.ds.W * S.ds.H * sizeof(float4), &S.nrm)) != PERCH_OK) return st;
        cudaError_t e = perch::launch_obs_normals(S.ds, gp.normal_max_jump_units, (float4*)S.nrm, c->stream);
        if (!e) e = cudaStreamSynchronize(c->stream);
        if (e) return cuda_fail(c, e, "observed normals");
        S.nrm_jump = gp.normal_max_jump_units;
    }
    const float4* nrm = (const float4*)S.nrm;
    if (cuda_stream) return run_gicp(c, c->plain, J, gp, nrm, poses_out, info, (cudaStream_t)cuda_stream);
    const long long chunk = 1 << 18;
    const long long k0 = std::min<long long>(n, chunk);
    if ((st = ensure_stage(c, (size_t)k0 * (48 + 48 + 8))) != PERCH_OK) return st;
    float* d_in = (float*)c->stage;
    float* d_out = (float*)((char*)c->stage + (size_t)k0 * 48);
    int32_t* d_info = (int32_t*)((char*)c->stage + (size_t)k0 * 96);
    for (long long off = 0; off < n; off += chunk) {
        const long long k = std::min(chunk, n - off);
        cudaError_t e = cudaMemcpyAsync(d_in, poses + 12 * off, k * 48, cudaMemcpyHostToDevice, c->stream);
        if (e) return cuda_fail(c, e, "perch_refine_hypotheses upload");
        perch::Job Jk = J;
        Jk.poses = d_in;
        Jk.n = k;
        if ((st = run_gicp(c, c->plain, Jk, gp, nrm, d_out, d_info, c->stream)) != PERCH_OK) return st;
        e = cudaMemcpyAsync(poses_out + 12 * off, d_out, k * 48, cudaMemcpyDeviceToHost, c->stream);
        if (!e && info) e = cudaMemcpyAsync(info + 2 * off, d_info, k * 8, cudaMemcpyDeviceToHost, c->stream);
        if (!e) e = cudaStreamSynchronize(c->stream);
        if (e) return cuda_fail(c, e, "perch_refine_hypotheses");
    }
    return check_device_error(c);
}

perch_status perch_tree_search(perch_ctx* c, int32_t scene_id, const perch_tree_object* objects, int32_t K,
                               int32_t beam_width, int32_t* order, int32_t* pose_index, int64_t* level_cost,
                               int64_t* edges_scored)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (!objects || !order || !pose_index || !level_cost) return fail(c, PERCH_E_INVALID, "null argument");
    if (K < 1 || K > 64) return fail(c, PERCH_E_INVALID, "K must be in [1, 64]");
    if (beam_width < 1 || beam_width > 4096) return fail(c, PERCH_E_INVALID, "beam_width must be in [1, 4096]");
    auto si = c->scenes.find(scene_id);
    if (si == c->scenes.end()) return fail(c, PERCH_E_NOTFOUND, "unknown scene %d", scene_id);
    if (si->second.ds.jo_mode != 0) return fail(c, PERCH_E_INVALID, "the tree search needs jo_mode 0");
    DeviceGuard g(c->device);
    const perch::DevScene& ds = si->second.ds;
    const size_t npx = (size_t)ds.W * ds.H, words = (npx + 31) / 32;
    // validate the objects and lay their poses out in one device buffer
    std::vector<long long> off(K + 1, 0);
    for (int32_t j = 0; j < K; ++j) {
        if (!objects[j].poses || objects[j].n < 1) return fail(c, PERCH_E_INVALID, "object %d: no poses", j);
        off[j + 1] = off[j] + objects[j].n;
    }
    const long long total = off[K];
    // scratch: poses, per-level edge costs, 2 x beam state images
    const size_t state_bytes = npx * sizeof(uint32_t) + 2 * words * sizeof(uint32_t);
    const size_t cost_cap = (size_t)beam_width * (size_t)total;
    void *d_poses = nullptr, *d_costs = nullptr, *d_states = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(c->stream);
        dfree(c, d_poses);
        dfree(c, d_costs);
        dfree(c, d_states);
    };
    perch_status st = dalloc(c, (size_t)total * 48, &d_poses);
    if (st == PERCH_OK) st = dalloc(c, (cost_cap + 2) * 8, &d_costs);
    if (st == PERCH_OK) st = dalloc(c, 2 * (size_t)beam_width * state_bytes, &d_states);
    if (st != PERCH_OK) {
        cleanup();
        return st;
    }
    auto slot = [&](int half, int k) { return (char*)d_states + ((size_t)half * beam_width + k) * state_bytes; };
    cudaError_t e = cudaSuccess;
    for (int32_t j = 0; j < K && !e; ++j)
        e = cudaMemcpyAsync((float*)d_poses + 12 * off[j], objects[j].poses, (size_t)objects[j].n * 48,
                            cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemsetAsync(slot(0, 0), 0, state_bytes, c->stream);
    if (e) {
        cleanup();
        return cuda_fail(c, e, "perch_tree_search setup");
    }
    struct State {
        long long g;
        uint64_t placed;
        std::vector<int32_t> order, pose;
        std::vector<int64_t> cost;
    };
    std::vector<State> cur(1, State{0, 0, {}, {}, {}});
    int half = 0;
    long long edges = 0;
    std::vector<int32_t> h_costs;
    auto tree_of = [&](int half_, int k, bool out, int child_k) {
        perch::TreeState T{};
        char* base = slot(half_, k);
        T.depth = (const uint32_t*)base;
        T.mark = (const uint32_t*)(base + npx * 4);
        T.vol = (const uint32_t*)(base + npx * 4 + words * 4);
        if (out) {
            char* cb = slot(1 - half_, child_k);
            T.out_depth = (uint32_t*)cb;
            T.out_mark = (uint32_t*)(cb + npx * 4);
            T.out_vol = (uint32_t*)(cb + npx * 4 + words * 4);
        }
        T.margin = std::max(0, ds.occ_margin);
        return T;
    };
    for (int32_t level = 0; level < K; ++level) {
        // every remaining object at every pose, from every state of the level
        std::vector<perch::Job> jobs;
        std::vector<std::pair<int, int>> who;       // (state rank, object) per job
        std::vector<long long> coff;
        long long acc = 0;
        int mw = 0;
        for (size_t b = 0; b < cur.size(); ++b)
            for (int32_t j = 0; j < K; ++j) {
                if (cur[b].placed >> j & 1) continue;
                const perch_tree_object& o = objects[j];
                const int32_t* roi = (o.roi[2] > o.roi[0] && o.roi[3] > o.roi[1]) ? o.roi : nullptr;
                perch::Job J;
                int w;
                st = make_job(c, scene_id, o.mesh_id, o.label, roi, (const float*)d_poses + 12 * off[j],
                              (int32_t*)d_costs + 2 * acc, o.n, &J, &w, nullptr, nullptr);
                if (st != PERCH_OK) {
                    cleanup();
                    return st;
                }
                J.tree = tree_of(half, (int)b, false, 0);
                jobs.push_back(J);
                who.push_back({(int)b, j});
                coff.push_back(acc);
                mw = std::max(mw, w);
                acc += o.n;
            }
        if ((st = run_jobs(c, c->plain, jobs, mw, c->cfg, c->stream, nullptr)) != PERCH_OK) {
            cleanup();
            return st;
        }
        h_costs.resize(2 * (size_t)acc);
        e = cudaMemcpyAsync(h_costs.data(), d_costs, (size_t)acc * 8, cudaMemcpyDeviceToHost, c->stream);
        if (!e) e = cudaStreamSynchronize(c->stream);
        if (e) {
            cleanup();
            return cuda_fail(c, e, "perch_tree_search costs");
        }
        edges += acc;
        // (path cost, parent rank, object, pose) of every edge not refused
        struct Cand {
            long long g;
            int b, j, h;
        };
        std::vector<Cand> cands;
        for (size_t q = 0; q < jobs.size(); ++q) {
            const int b = who[q].first, j = who[q].second;
            for (int32_t h = 0; h < objects[j].n; ++h) {
                const int32_t jo = h_costs[2 * (coff[q] + h)], jr = h_costs[2 * (coff[q] + h) + 1];
                if (jo < 0) continue;
                cands.push_back({cur[b].g + jo + jr, b, j, h});
            }
        }
        if (cands.empty()) {
            cleanup();
            return fail(c, PERCH_E_NOTFOUND, "every placement at level %d is refused", level);
        }
        const size_t keep = std::min<size_t>(cands.size(), (size_t)beam_width);
        std::partial_sort(cands.begin(), cands.begin() + keep, cands.end(), [](const Cand& x, const Cand& y) {
            if (x.g != y.g) return x.g < y.g;
            if (x.b != y.b) return x.b < y.b;
            if (x.j != y.j) return x.j < y.j;
            return x.h < y.h;
        });
        // materialise the kept children's state images
        std::vector<State> nxt;
        for (size_t k = 0; k < keep && !e; ++k) {
            const Cand& cd = cands[k];
            e = cudaMemcpyAsync(slot(1 - half, (int)k), slot(half, cd.b), state_bytes, cudaMemcpyDeviceToDevice,
                                c->stream);
            if (e) break;
            const perch_tree_object& o = objects[cd.j];
            const int32_t* roi = (o.roi[2] > o.roi[0] && o.roi[3] > o.roi[1]) ? o.roi : nullptr;
            perch::Job J;
            int w;
            st = make_job(c, scene_id, o.mesh_id, o.label, roi, (const float*)d_poses + 12 * (off[cd.j] + cd.h),
                          (int32_t*)d_costs + 2 * cost_cap, 1, &J, &w, nullptr, nullptr);
            if (st == PERCH_OK) {
                J.tree = tree_of(half, cd.b, true, (int)k);
                std::vector<perch::Job> one(1, J);
                st = run_jobs(c, c->plain, one, w, c->cfg, c->stream, nullptr);
            }
            if (st != PERCH_OK) {
                cleanup();
                return st;
            }
            State s = cur[cd.b];
            s.g = cd.g;
            s.placed |= 1ull << cd.j;
            s.order.push_back(cd.j);
            s.pose.push_back(cd.h);
            s.cost.push_back(cd.g);
            nxt.push_back(std::move(s));
        }
        if (e) {
            cleanup();
            return cuda_fail(c, e, "perch_tree_search state");
        }
        cur.swap(nxt);
        half = 1 - half;
    }
    st = check_device_error(c);
    cleanup();
    if (st != PERCH_OK) return st;
    for (int32_t l = 0; l < K; ++l) {
        order[l] = cur[0].order[l];
        pose_index[l] = cur[0].pose[l];
        level_cost[l] = cur[0].cost[l];
    }
    if (edges_scored) *edges_scored = edges;
    return PERCH_OK;
}

perch_status perch_add_s(perch_ctx* c, int32_t mesh_id, const float* poses, const float* poses_true, int64_t n,
                         int32_t symmetric, double* add, void* cuda_stream)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (n < 0) return fail(c, PERCH_E_INVALID, "n < 0");
    if (n == 0) return PERCH_OK;
    if (!poses || !poses_true || !add) return fail(c, PERCH_E_INVALID, "null pointer");
    auto mi = c->meshes.find(mesh_id);
    if (mi == c->meshes.end()) return fail(c, PERCH_E_NOTFOUND, "unknown mesh %d", mesh_id);
    DeviceGuard g(c->device);
    const perch::DevMesh& m = mi->second.dm;
    if (cuda_stream) {
        cudaError_t e = perch::launch_add_s(m.verts, m.n_verts, poses, poses_true, n, symmetric ? 1 : 0, add,
                                            (cudaStream_t)cuda_stream);
        return e ? cuda_fail(c, e, "perch_add_s") : PERCH_OK;
    }
    perch_status st = ensure_stage(c, (size_t)n * (48 + 48 + 8));
    if (st != PERCH_OK) return st;
    float* dp = (float*)c->stage;
    float* dt = (float*)((char*)c->stage + (size_t)n * 48);
    double* dout = (double*)((char*)c->stage + (size_t)n * 96);
    cudaError_t e = cudaMemcpyAsync(dp, poses, (size_t)n * 48, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync(dt, poses_true, (size_t)n * 48, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = perch::launch_add_s(m.verts, m.n_verts, dp, dt, n, symmetric ? 1 : 0, dout, c->stream);
    if (!e) e = cudaMemcpyAsync(add, dout, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    return e ? cuda_fail(c, e, "perch_add_s") : PERCH_OK;
}

perch_status perch_add_s_auc(const double* add, int64_t n, double max_threshold, double* auc)
{
    if (!add || !auc || n < 1 || !(max_threshold > 0.0)) return PERCH_E_INVALID;
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += std::max(0.0, 1.0 - add[i] / max_threshold);
    *auc = s / (double)n;
    return PERCH_OK;
}

perch_status perch_debug_render_keys(perch_ctx* c, int32_t scene_id, int32_t mesh_id,
                                     const int32_t* roi, const float* pose, uint64_t* keys)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (!pose || !keys) return fail(c, PERCH_E_INVALID, "null pose or keys");
    DeviceGuard g(c->device);
    perch_status st = ensure_stage(c, 64);
    if (st != PERCH_OK) return st;
    float* d_pose = (float*)c->stage;
    int32_t* d_cost = (int32_t*)((char*)c->stage + 48);
    perch::Job J;
    int mw;
    const SceneRec* s;
    if ((st = make_job(c, scene_id, mesh_id, -1, roi, d_pose, d_cost, 1, &J, &mw, &s, nullptr)) != PERCH_OK)
        return st;
    size_t npx = (size_t)s->ds.W * s->ds.H;
    void* dump = nullptr;
    if ((st = dalloc(c, npx * 8, &dump)) != PERCH_OK) return st;
    cudaError_t e = cudaMemsetAsync(dump, 0xFF, npx * 8, c->stream);
    if (!e) e = cudaMemcpyAsync(d_pose, pose, 48, cudaMemcpyHostToDevice, c->stream);
    if (e) {
        dfree(c, dump);
        return cuda_fail(c, e, "perch_debug_render_keys");
    }
    std::vector<perch::Job> jobs(1, J);
    st = run_jobs(c, c->plain, jobs, mw, c->cfg, c->stream, (unsigned long long*)dump);
    if (st == PERCH_OK) {
        e = cudaMemcpyAsync(keys, dump, npx * 8, cudaMemcpyDeviceToHost, c->stream);
        if (!e) e = cudaStreamSynchronize(c->stream);
        if (e) st = cuda_fail(c, e, "perch_debug_render_keys");
    }
    cudaStreamSynchronize(c->stream);
    dfree(c, dump);
    if (st != PERCH_OK) return st;
    return check_device_error(c);
}

perch_status perch_batch_graph_create(perch_ctx* c, const perch_work_item* items, int32_t n_items,
                                      const float* poses, int32_t* costs, perch_batch_graph** out)
{
    if (!c || !out) return PERCH_E_INVALID;
    c->err.clear();
    *out = nullptr;
    if (!poses || !costs) return fail(c, PERCH_E_INVALID, "null poses or costs");
    DeviceGuard g(c->device);
    std::vector<perch::Job> jobs;
    int mw;
    long long total;
    perch_status st = batch_jobs(c, items, n_items, poses, costs, &jobs, &mw, &total);
    if (st != PERCH_OK) return st;
    if (total == 0) return fail(c, PERCH_E_INVALID, "empty batch");
    perch::ScoreConfig cfg = c->cfg;
    if ((st = fit_config(c, mw, &cfg)) != PERCH_OK) return st;
    const int resident = perch::score_grid(cfg, mw);
    if (resident <= 0) {
        cudaGetLastError();
        return fail(c, PERCH_E_CUDA, "scoring kernel does not fit on the device");
    }
    perch_batch_graph* G = new (std::nothrow) perch_batch_graph();
    if (!G) return fail(c, PERCH_E_NOMEM, "graph handle");
    G->ctx = c;
    // One kernel node per item, each with the whole resident grid, its own
    // counter and the shared vertex-cache pool; node j follows node j - 4,
    // mirroring the side-stream round robin of the direct launch.
    const size_t nj = jobs.size();
    int max_verts = 0;
    bool small_images = true;
    for (const auto& j : jobs) {
        max_verts = std::max(max_verts, j.m.n_verts);
        small_images = small_images && j.sc.W <= 1023 && j.sc.H <= 1023;
    }
    const long long vstride = small_images ? ((long long)max_verts + 31) / 32 * 32 : 0;
    const size_t words = nj + ((size_t)resident + 31) / 32;
    void* p = nullptr;
    if ((st = dalloc(c, words * sizeof(unsigned), &p)) == PERCH_OK) G->next = (unsigned*)p;
    if (st == PERCH_OK && vstride > 0)
        st = dalloc(c, (size_t)resident * vstride * sizeof(unsigned long long), &G->vcache);
    cudaError_t e = cudaSuccess;
    if (st == PERCH_OK) e = cudaGraphCreate(&G->graph, 0);
    cudaGraphNode_t reset = nullptr;
    if (st == PERCH_OK && !e) {
        cudaMemsetParams mp{};
        mp.dst = G->next;
        mp.value = 0;
        mp.elementSize = 4;
        mp.width = words;
        mp.height = 1;
        mp.pitch = 0;
        e = cudaGraphAddMemsetNode(&reset, G->graph, nullptr, 0, &mp);
    }
    std::vector<cudaGraphNode_t> nodes(nj, nullptr);
    for (size_t j = 0; j < nj && st == PERCH_OK && !e; ++j) {
        if (jobs[j].n == 0) {
            if (j >= 4) nodes[j] = nodes[j - 4];
            continue;
        }
        perch::ScoreArgs a{};
        a.job = jobs[j];
        a.n = jobs[j].n;
        a.zcap_words = cfg.zcap_words;
        a.mark_words = mw;
        a.err = c->d_err;
        a.next = G->next + j;
        a.vcache = vstride ? (unsigned long long*)G->vcache : nullptr;
        a.vstride = vstride;
        a.vmask = G->next + nj;
        a.vslots = resident;
        cudaGraphNode_t dep = (j >= 4 && nodes[j - 4]) ? nodes[j - 4] : reset;
        e = perch::add_score_node(G->graph, &dep, 1, a, cfg, resident, &nodes[j]);
    }
    if (st == PERCH_OK && !e) e = cudaGraphInstantiate(&G->exec, G->graph, 0);
    if (st == PERCH_OK && e) st = cuda_fail(c, e, "perch_batch_graph_create");
    if (st != PERCH_OK) {
        perch_batch_graph_destroy(G);
        return st;
    }
    *out = G;
    return PERCH_OK;
}

perch_status perch_batch_graph_launch(perch_batch_graph* G, void* cuda_stream)
{
    if (!G || !G->exec) return PERCH_E_INVALID;
    DeviceGuard g(G->ctx->device);
    cudaError_t e = cudaGraphLaunch(G->exec, (cudaStream_t)cuda_stream);
    if (e) return cuda_fail(G->ctx, e, "perch_batch_graph_launch");
    return PERCH_OK;
}

perch_status perch_batch_graph_destroy(perch_batch_graph* G)
{
    if (!G) return PERCH_OK;
    perch_ctx* c = G->ctx;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    dfree(c, G->next);
    dfree(c, G->vcache);
    delete G;
    return PERCH_OK;
}

perch_status perch_autotune(perch_ctx* c, const perch_work_item* items, int32_t n_items,
                            const float* poses, int32_t* costs, int32_t* threads, int32_t* zbuf_words)
{
    if (!c || !threads || !zbuf_words) return PERCH_E_INVALID;
    c->err.clear();
    if (!items || n_items < 1 || !poses || !costs) return fail(c, PERCH_E_INVALID, "empty batch");
    DeviceGuard g(c->device);
    // class of the batch: largest ROI area and triangle count, as powers of two
    long long max_area = 0, max_tris = 0;
    for (int32_t i = 0; i < n_items; ++i) {
        auto si = c->scenes.find(items[i].scene_id);
        auto mi = c->meshes.find(items[i].mesh_id);
        if (si == c->scenes.end() || mi == c->meshes.end()) return fail(c, PERCH_E_NOTFOUND, "item %d", i);
        long long area = (items[i].roi[2] > items[i].roi[0] && items[i].roi[3] > items[i].roi[1])
                             ? (long long)(items[i].roi[2] - items[i].roi[0]) * (items[i].roi[3] - items[i].roi[1])
                             : (long long)si->second.ds.W * si->second.ds.H;
        max_area = std::max(max_area, area);
        max_tris = std::max<long long>(max_tris, mi->second.dm.n_tris);
    }
    const uint64_t key = ((uint64_t)next_pow2(max_area) << 32) | next_pow2(max_tris);
    auto hit = c->tuned.find(key);
    if (hit != c->tuned.end()) {
        c->cfg.threads = hit->second.threads;
        c->cfg.zcap_words = hit->second.zcap_words;
        *threads = c->cfg.threads;
        *zbuf_words = c->cfg.zcap_words;
        return PERCH_OK;
    }
    // time each shape on a sample of whole items (launches of the real
    // sizes, so per-launch tails weigh the same): every 8th item in order of
    // size, which keeps the batch's mix of small and large items; batches of
    // fewer than 16 items are timed whole
    std::vector<int32_t> idx(n_items);
    for (int32_t i = 0; i < n_items; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) { return items[x].n > items[y].n; });
    std::vector<perch_work_item> sample;
    const int32_t step = n_items < 16 ? 1 : 8;
    for (int32_t k = step / 2; k < n_items; k += step) sample.push_back(items[idx[k]]);
    std::vector<perch::Job> jobs;
    int mw;
    long long total;
    perch_status st = batch_jobs(c, sample.data(), (int32_t)sample.size(), poses, costs, &jobs, &mw, &total);
    if (st != PERCH_OK) return st;
    const perch::ScoreConfig saved = c->cfg;
    perch::ScoreConfig best = saved;
    float best_ms = 3.0e38f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int th[3] = {128, 256, 512};
    const int zw[4] = {2048, 4096, 8192, 16384};
    for (int ti = 0; ti < 3 && st == PERCH_OK; ++ti) {
        for (int zi = 0; zi < 4 && st == PERCH_OK; ++zi) {
            perch::ScoreConfig cfg = saved;
            cfg.threads = th[ti];
            cfg.zcap_words = zw[zi];
            if (perch::score_smem_bytes(cfg, mw) > 200 * 1024) continue;
            float ms = 3.0e38f;
            for (int rep = 0; rep < 2 && st == PERCH_OK; ++rep) {
                cudaEventRecord(e0, c->stream);
                st = run_jobs(c, c->plain, jobs, mw, cfg, c->stream, nullptr);
                cudaEventRecord(e1, c->stream);
                cudaEventSynchronize(e1);
                float t = 0.0f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) ms = std::min(ms, t);
            }
            if (st == PERCH_OK && ms < best_ms) {
                best_ms = ms;
                best = cfg;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PERCH_OK) return st;
    c->cfg.threads = best.threads;
    c->cfg.zcap_words = best.zcap_words;
    c->tuned[key] = c->cfg;
    *threads = c->cfg.threads;
    *zbuf_words = c->cfg.zcap_words;
    return check_device_error(c);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// served form: continuous batching over launch slots
// ---------------------------------------------------------------------------

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServedRequest {
    uint64_t ticket = 0;
    perch::Job tmpl{};              // scene, mesh, label, ROI (pointers filled per launch)
    int mark_words = 0;
    std::vector<float> poses;       // copy of the caller's poses
    int32_t* user_costs = nullptr;
    int64_t n = 0;
    int64_t t_submit = 0, t_done = 0;
    perch_status status = PERCH_OK;
    bool done = false;
};

struct Slot {
    ScoreScratch X;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    float* d_poses = nullptr;
    int32_t* d_costs = nullptr;
    float* h_poses = nullptr;       // pinned
    int32_t* h_costs = nullptr;     // pinned
    std::vector<std::shared_ptr<ServedRequest>> reqs;
    std::vector<int64_t> offsets;
    std::vector<cudaEvent_t> req_done;  // per request: its costs are in h_costs
    bool busy = false;
};

}  // namespace

struct perch_server {
    perch_ctx* c = nullptr;
    perch_server_config cfg{};
    std::vector<Slot> slots;
    std::mutex mu;                  // queue, slots, tickets
    std::mutex ctx_mu;              // context state used by submit and the scheduler
    std::condition_variable cv_sched, cv_done, cv_wait;
    std::deque<std::shared_ptr<ServedRequest>> pending;
    int64_t pending_hyps = 0;
    std::deque<int> in_flight;      // slots in launch order
    std::unordered_map<uint64_t, std::shared_ptr<ServedRequest>> tickets;
    uint64_t next_ticket = 1;
    bool stopping = false;
    bool sched_done = false;
    std::thread sched, completer;
};

namespace {

void serve_schedule(perch_server* S)
{
    cudaSetDevice(S->c->device);
    for (;;) {
        std::unique_lock<std::mutex> lk(S->mu);
        auto free_slot = [&]() {
            for (size_t i = 0; i < S->slots.size(); ++i)
                if (!S->slots[i].busy) return (int)i;
            return -1;
        };
        S->cv_sched.wait(lk, [&] {
            return (S->stopping && S->pending.empty()) || (!S->pending.empty() && free_slot() >= 0);
        });
        if (S->pending.empty()) break;
        if (S->cfg.max_wait_us > 0 && !S->stopping && S->pending_hyps < S->cfg.max_batch_hypotheses)
            S->cv_sched.wait_for(lk, std::chrono::microseconds(S->cfg.max_wait_us), [&] {
                return S->stopping || S->pending_hyps >= S->cfg.max_batch_hypotheses;
            });
        const int si = free_slot();
        Slot& slot = S->slots[si];
        slot.reqs.clear();
        slot.offsets.clear();
        int64_t total = 0;
        while (!S->pending.empty() && total + S->pending.front()->n <= S->cfg.max_batch_hypotheses) {
            auto r = S->pending.front();
            S->pending.pop_front();
            S->pending_hyps -= r->n;
            slot.reqs.push_back(r);
            total += r->n;
        }
        // smallest requests first: each completes as soon as its own launch
        // and read-back are done, so short ones do not wait for long ones
        std::stable_sort(slot.reqs.begin(), slot.reqs.end(),
                         [](const std::shared_ptr<ServedRequest>& x, const std::shared_ptr<ServedRequest>& y) {
                             return x->n < y->n;
                         });
        for (size_t k = 0, off = 0; k < slot.reqs.size(); off += slot.reqs[k]->n, ++k) slot.offsets.push_back(off);
        slot.busy = true;
        lk.unlock();
        perch_status st = PERCH_OK;
        while (slot.req_done.size() < slot.reqs.size()) {
            cudaEvent_t ev = nullptr;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                st = PERCH_E_CUDA;
                break;
            }
            slot.req_done.push_back(ev);
        }

        std::vector<perch::Job> jobs;
        int mw = 0;
        for (size_t k = 0; k < slot.reqs.size(); ++k) {
            const auto& r = slot.reqs[k];
            std::memcpy(slot.h_poses + 12 * slot.offsets[k], r->poses.data(), r->poses.size() * sizeof(float));
            perch::Job J = r->tmpl;
            J.poses = slot.d_poses + 12 * slot.offsets[k];
            J.costs = slot.d_costs + 2 * slot.offsets[k];
            J.n = r->n;
            jobs.push_back(J);
            mw = std::max(mw, r->mark_words);
        }
        cudaError_t e = cudaSuccess;
        if (st == PERCH_OK) e = cudaMemcpyAsync(slot.d_poses, slot.h_poses, total * 48, cudaMemcpyHostToDevice, slot.stream);
        if (e) st = PERCH_E_CUDA;
        if (st == PERCH_OK) {
            const AfterJob readback = [&](size_t j, cudaStream_t js) {
                const int64_t off = slot.offsets[j], n = slot.reqs[j]->n;
                cudaError_t r = cudaMemcpyAsync(slot.h_costs + 2 * off, slot.d_costs + 2 * off, n * 8,
                                                cudaMemcpyDeviceToHost, js);
                return r ? r : cudaEventRecord(slot.req_done[j], js);
            };
            std::lock_guard<std::mutex> g(S->ctx_mu);
            st = run_jobs(S->c, slot.X, jobs, mw, S->c->cfg, slot.stream, nullptr, &readback);
        }
        cudaEventRecord(slot.done, slot.stream);
        if (st != PERCH_OK)
            for (auto& r : slot.reqs) r->status = st;
        lk.lock();
        // hand the slot to the completion thread only once its event is recorded
        S->in_flight.push_back(si);
        S->cv_done.notify_all();
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->sched_done = true;
    S->cv_done.notify_all();
}

void serve_complete(perch_server* S)
{
    cudaSetDevice(S->c->device);
    for (;;) {
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_done.wait(lk, [&] { return !S->in_flight.empty() || S->sched_done; });
        if (S->in_flight.empty()) break;
        const int si = S->in_flight.front();
        lk.unlock();
        Slot& slot = S->slots[si];
        // requests in launch order, each as soon as its own read-back is done
        for (size_t k = 0; k < slot.reqs.size(); ++k) {
            auto& r = slot.reqs[k];
            cudaError_t e = r->status == PERCH_OK ? cudaEventSynchronize(slot.req_done[k]) : cudaSuccess;
            if (e != cudaSuccess && r->status == PERCH_OK) r->status = PERCH_E_CUDA;
            if (r->status == PERCH_OK)
                std::memcpy(r->user_costs, slot.h_costs + 2 * slot.offsets[k], r->n * 2 * sizeof(int32_t));
            r->t_done = now_ns();
            std::lock_guard<std::mutex> g(S->mu);
            r->done = true;
            r->poses.clear();
            r->poses.shrink_to_fit();
            S->cv_wait.notify_all();
        }
        cudaEventSynchronize(slot.done);
        lk.lock();
        slot.reqs.clear();
        slot.busy = false;
        S->in_flight.pop_front();
        S->cv_sched.notify_all();
        S->cv_wait.notify_all();
    }
}

}  // namespace

extern "C" {

perch_status perch_server_start(perch_ctx* c, const perch_server_config* cfg, perch_server** out)
{
    if (!c || !cfg || !out) return PERCH_E_INVALID;
    c->err.clear();
    *out = nullptr;
    if (cfg->slots < 1 || cfg->slots > 16 || cfg->max_batch_hypotheses < 1 || cfg->max_batch_hypotheses > (1ll << 30) ||
        cfg->max_wait_us < 0)
        return fail(c, PERCH_E_INVALID, "server configuration out of range");
    DeviceGuard g(c->device);
    perch_server* S = new (std::nothrow) perch_server();
    if (!S) return fail(c, PERCH_E_NOMEM, "server");
    S->c = c;
    S->cfg = *cfg;
    S->slots.resize(cfg->slots);
    perch_status st = PERCH_OK;
    const size_t nb = (size_t)cfg->max_batch_hypotheses;
    for (auto& slot : S->slots) {
        void* p = nullptr;
        if (st == PERCH_OK) st = scratch_init(c, slot.X);
        if (st == PERCH_OK && (st = dalloc(c, nb * 48, &p)) == PERCH_OK) slot.d_poses = (float*)p;
        if (st == PERCH_OK && (st = dalloc(c, nb * 8, &p)) == PERCH_OK) slot.d_costs = (int32_t*)p;
        if (st == PERCH_OK && (cudaMallocHost(&p, nb * 48) != cudaSuccess || !(slot.h_poses = (float*)p)))
            st = fail(c, PERCH_E_NOMEM, "pinned staging");
        if (st == PERCH_OK && (cudaMallocHost(&p, nb * 8) != cudaSuccess || !(slot.h_costs = (int32_t*)p)))
            st = fail(c, PERCH_E_NOMEM, "pinned staging");
        if (st == PERCH_OK && (cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking) != cudaSuccess ||
                               cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming) != cudaSuccess))
            st = cuda_fail(c, cudaGetLastError(), "server stream");
    }
    if (st != PERCH_OK) {
        for (auto& slot : S->slots) {
            scratch_free(c, slot.X);
            dfree(c, slot.d_poses);
            dfree(c, slot.d_costs);
            if (slot.h_poses) cudaFreeHost(slot.h_poses);
            if (slot.h_costs) cudaFreeHost(slot.h_costs);
            if (slot.stream) cudaStreamDestroy(slot.stream);
            if (slot.done) cudaEventDestroy(slot.done);
            for (auto ev : slot.req_done) cudaEventDestroy(ev);
        }
        delete S;
        return st;
    }
    S->sched = std::thread(serve_schedule, S);
    S->completer = std::thread(serve_complete, S);
    *out = S;
    return PERCH_OK;
}

perch_status perch_submit(perch_server* S, const perch_request* req, uint64_t* ticket)
{
    if (!S || !req || !ticket) return PERCH_E_INVALID;
    if (!req->poses || !req->costs || req->n < 1) return PERCH_E_INVALID;
    if (req->n > S->cfg.max_batch_hypotheses) return PERCH_E_BUDGET;
    auto r = std::make_shared<ServedRequest>();
    {
        std::lock_guard<std::mutex> g(S->ctx_mu);
        const int32_t* roi = (req->roi[2] > req->roi[0] && req->roi[3] > req->roi[1]) ? req->roi : nullptr;
        perch_status st = make_job(S->c, req->scene_id, req->mesh_id, req->label, roi, nullptr, nullptr,
                                   req->n, &r->tmpl, &r->mark_words, nullptr, nullptr);
        if (st != PERCH_OK) return st;
    }
    r->poses.assign(req->poses, req->poses + 12 * req->n);
    r->user_costs = req->costs;
    r->n = req->n;
    r->t_submit = now_ns();
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return PERCH_E_BUSY;
    r->ticket = S->next_ticket++;
    S->tickets[r->ticket] = r;
    S->pending.push_back(r);
    S->pending_hyps += r->n;
    *ticket = r->ticket;
    S->cv_sched.notify_all();
    return PERCH_OK;
}

perch_status perch_poll(perch_server* S, uint64_t ticket)
{
    if (!S) return PERCH_E_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return PERCH_E_NOTFOUND;
    if (!it->second->done) return PERCH_E_BUSY;
    return it->second->status;
}

perch_status perch_wait(perch_server* S, uint64_t ticket, int64_t timeout_us)
{
    if (!S) return PERCH_E_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return PERCH_E_NOTFOUND;
    auto r = it->second;
    if (timeout_us < 0) {
        S->cv_wait.wait(lk, [&] { return r->done; });
    } else if (!S->cv_wait.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; })) {
        return PERCH_E_TIMEOUT;
    }
    return r->status;
}

perch_status perch_ticket_times(perch_server* S, uint64_t ticket, int64_t* submit_ns, int64_t* done_ns)
{
    if (!S || !submit_ns || !done_ns) return PERCH_E_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return PERCH_E_NOTFOUND;
    if (!it->second->done) return PERCH_E_BUSY;
    *submit_ns = it->second->t_submit;
    *done_ns = it->second->t_done;
    return PERCH_OK;
}

perch_status perch_server_stop(perch_server* S)
{
    if (!S) return PERCH_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        S->cv_sched.notify_all();
    }
    if (S->sched.joinable()) S->sched.join();
    if (S->completer.joinable()) S->completer.join();
    perch_ctx* c = S->c;
    DeviceGuard g(c->device);
    for (auto& slot : S->slots) {
        if (slot.stream) cudaStreamSynchronize(slot.stream);
        scratch_free(c, slot.X);
        dfree(c, slot.d_poses);
        dfree(c, slot.d_costs);
        if (slot.h_poses) cudaFreeHost(slot.h_poses);
        if (slot.h_costs) cudaFreeHost(slot.h_costs);
        if (slot.stream) cudaStreamDestroy(slot.stream);
        if (slot.done) cudaEventDestroy(slot.done);
        for (auto ev : slot.req_done) cudaEventDestroy(ev);
    }
    delete S;
    return PERCH_OK;
}

}  // extern "C"
