// libperch host side: contexts, resident meshes and observations, scoring,
// argmin, proposals, pose errors and the debug views of the C ABI declared in
// include/perch.h (batched form: perch_batch.cu; served form: perch_serve.cu;
// refinement: perch_refine.cu; tree search: perch_tree.cu).
//
// A context owns every device allocation it makes and charges each to its HBM
// budget.  Meshes and observations are copied once and stay resident; scoring
// calls launch the fused kernel (perch_kernels.cu) on the caller's stream or,
// in synchronous mode, on the context's own stream with staging copies.
#include "perch_host.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

namespace perch_host {


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

int mark_words_for(const SceneRec& s, int label, const int roi[4], int cap_bits)
{
    // jo_mode 1 keeps a 64-bit key per pixel (its nearest rendered point)
    // instead of a mark bit: four times the capacity, at least one image row
    const int per_px = s.ds.jo_mode == 1 ? 64 : 1;
    const long long cap = s.ds.jo_mode == 1 ? 4ll * cap_bits : cap_bits;
    long long bits = per_px * (label >= 0 ? (long long)(roi[2] - roi[0]) * (roi[3] - roi[1])
                                          : (long long)s.ds.W * s.ds.H);
    bits = std::min<long long>(bits, cap);
    bits = std::max<long long>(bits, (long long)per_px * s.ds.W);
    return (int)(((bits + 31) / 32 + 2) & ~1ll);   // even: keeps the later 8-byte arrays aligned
}

// Shrink the z-buffer of *cfg (the caller's launch shape) until the block's
// shared memory fits the device's opt-in limit.
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

perch_status refuse_while_serving(perch_ctx* c)
{
    if (c->servers.load() > 0)
        return fail(c, PERCH_E_BUSY, "a server is running on this context: use the server calls, or "
                                     "load and release meshes and observations, until it is stopped");
    return PERCH_OK;
}

static void drop_finished(UseTrack& u)
{
    size_t k = 0;
    for (cudaEvent_t ev : u.pending) {
        if (cudaEventQuery(ev) == cudaErrorNotReady) {
            u.pending[k++] = ev;
        } else {
            cudaGetLastError();
            cudaEventDestroy(ev);
        }
    }
    u.pending.resize(k);
}

bool in_use(UseTrack& u)
{
    drop_finished(u);
    return u.users > 0 || !u.pending.empty();
}

static perch_status track(perch_ctx* c, UseTrack& u, cudaStream_t st)
{
    drop_finished(u);
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (!e) e = cudaEventRecord(ev, st);
    if (e) {
        if (ev) cudaEventDestroy(ev);
        return cuda_fail(c, e, "recording an asynchronous use");
    }
    u.pending.push_back(ev);
    return PERCH_OK;
}

perch_status note_async_use(perch_ctx* c, int32_t scene_id, int32_t mesh_id, cudaStream_t st)
{
    perch_status r = PERCH_OK;
    auto si = c->scenes.find(scene_id);
    if (si != c->scenes.end()) r = track(c, si->second.use, st);
    auto mi = c->meshes.find(mesh_id);
    if (r == PERCH_OK && mi != c->meshes.end()) r = track(c, mi->second.use, st);
    return r;
}

void count_users(perch_ctx* c, int32_t scene_id, int32_t mesh_id, int d)
{
    auto si = c->scenes.find(scene_id);
    if (si != c->scenes.end()) si->second.use.users += d;
    auto mi = c->meshes.find(mesh_id);
    if (mi != c->meshes.end()) mi->second.use.users += d;
}

static void free_tracking(UseTrack& u)
{
    for (cudaEvent_t ev : u.pending) {
        cudaEventSynchronize(ev);
        cudaEventDestroy(ev);
    }
    u.pending.clear();
}

// Launch the persistent scorer once per job, on stream st after every
// earlier run that used X.  Each launch gets the whole resident grid; with
// several jobs the launches go round-robin over X's side streams, so the
// blocks of job j+1 start on the SMs that job j's blocks leave at its tail,
// and every job keeps its fields in the parameter bank.
// after_job (optional) is called right after job j's launch with the stream
// it went to, to enqueue work that needs only that job (the server's
// per-request read-back).
perch_status run_jobs(perch_ctx* c, ScoreScratch& X, const std::vector<perch::Job>& jobs,
                      int mark_words, const perch::ScoreConfig& cfg_in, cudaStream_t st,
                      unsigned long long* dump, const AfterJob* after_job)
{
    Range r("perch: scoring launches");
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
    // coordinates fit in int16; with tile bins each slot also holds the bins
    long long vstride = 0, bin_off = 0;
    if (small_images) {
        vstride = perch::vcache_slot_words(max_verts, cfg.bin_cap, &bin_off);
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
    a.bin_cap = vstride ? cfg.bin_cap : 0;
    a.bin_off = bin_off;
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

}  // namespace perch_host

using namespace perch_host;

namespace {

// Dense cell index over the near-cell box (at most 2^24 cells): the cloud
// re-sorted by cell (z-major, then y, then x) with each cell's start, so that
// the radius search reads a row of three cells as one run instead of probing
// the hash table for each of 27 cells.  The hash table is then no longer
// needed and is freed.  A larger box keeps the hash table.
perch_status build_dense_cells(perch_ctx* c, SceneRec& s, long long cells)
{
    perch::DevScene& d = s.ds;
    d.cell_start = nullptr;
    if (d.n_pts <= 0 || cells > (1ll << 24)) return PERCH_OK;
    const size_t n = (size_t)cells, n_tiles = (n + 1023) / 1024;
    void *count = nullptr, *cursor = nullptr, *sums = nullptr, *out = nullptr;
    auto cleanup = [&]() { dfree(c, count); dfree(c, cursor); dfree(c, sums); dfree(c, out); };
    perch_status st;
    if ((st = dalloc(c, (n + 1) * 4, &s.cstart)) || (st = dalloc(c, n * 4, &count)) ||
        (st = dalloc(c, n * 4, &cursor)) || (st = dalloc(c, n_tiles * 4, &sums)) ||
        (st = dalloc(c, (size_t)d.n_pts * sizeof(float4), &out))) {
        cleanup();
        dfree(c, s.cstart);
        s.cstart = nullptr;
        return st;
    }
    const uint32_t last = (uint32_t)d.n_pts;
    cudaError_t e = cudaMemsetAsync(count, 0, n * 4, c->stream);
    if (!e) e = cudaMemsetAsync(cursor, 0, n * 4, c->stream);
    if (!e) e = perch::launch_dense_cells(d, (uint32_t*)count, (uint32_t*)cursor, (uint32_t*)sums,
                                          (uint32_t*)s.cstart, (float4*)out, c->stream);
    if (!e) e = cudaMemcpyAsync((uint32_t*)s.cstart + n, &last, 4, cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) {
        cleanup();
        dfree(c, s.cstart);
        s.cstart = nullptr;
        return cuda_fail(c, e, "dense cell index");
    }
    dfree(c, count);
    dfree(c, cursor);
    dfree(c, sums);
    dfree(c, s.pts);
    dfree(c, s.table);
    s.pts = out;
    s.table = nullptr;
    d.pts = (const float4*)out;
    d.table = nullptr;
    d.table_mask = 0;
    d.cell_start = (const uint32_t*)s.cstart;
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
    return build_dense_cells(c, s, cells);
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
    if (st == PERCH_OK && (st = dalloc(c, sizeof(unsigned long long) * 3 * perch::kBestMaxBlocks, &p)) == PERCH_OK)
        c->d_best_partial = (unsigned long long*)p;
    if (st == PERCH_OK && (st = dalloc(c, 64, &p)) == PERCH_OK) {
        c->d_best_ticket = (unsigned*)p;
        c->d_best_index = (long long*)((char*)p + 16);
        c->d_best_cost = (int32_t*)((char*)p + 32);
    }
    if (st == PERCH_OK) st = scratch_init(c, c->plain);
    if (st == PERCH_OK && (e = cudaEventCreateWithFlags(&c->best_last, cudaEventDisableTiming)) != cudaSuccess)
        st = cuda_fail(c, e, "cudaEventCreate");
    if (st == PERCH_OK && (e = cudaEventRecord(c->best_last, c->stream)) != cudaSuccess)
        st = cuda_fail(c, e, "cudaEventRecord");
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
    if (c->servers.load() > 0) return refuse_while_serving(c);
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& kv : c->scenes) free_tracking(kv.second.use);
    for (auto& kv : c->meshes) free_tracking(kv.second.use);
    if (c->best_last) {
        cudaEventSynchronize(c->best_last);
        cudaEventDestroy(c->best_last);
    }
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
    std::lock_guard<std::mutex> lk(c->mu);
    Range r("perch: mesh upload");
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
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->meshes.find(mesh_id);
    if (it == c->meshes.end()) return fail(c, PERCH_E_NOTFOUND, "unknown mesh %d", mesh_id);
    DeviceGuard g(c->device);
    if (in_use(it->second.use))
        return fail(c, PERCH_E_BUSY, "mesh %d is in use (%d served requests or batch graphs, %zu unfinished "
                                     "asynchronous calls)", mesh_id, it->second.use.users,
                    it->second.use.pending.size());
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

    std::lock_guard<std::mutex> lk(c->mu);
    Range r("perch: observation build (cloud, CIELAB, voxel hash)");
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
        dfree(c, s.near); dfree(c, s.cstart); dfree(c, s.pxyz);
    };
    if ((st = dalloc(c, npx * sizeof(uint16_t), &s.depth)) ||
        (labels && (st = dalloc(c, npx * sizeof(int32_t), &s.labels))) ||
        (st = dalloc(c, npx * sizeof(float4), &s.lab)) || (st = dalloc(c, npx * sizeof(float4), &s.pxyz)) ||
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
    d.inv_cell = 1.0f / cell;
    d.tau_c = p.tau_c;
    d.z_near = p.z_near_m;
    d.color_check = p.color_check;
    d.stride = p.stride;
    d.occ_margin = p.occ_margin_units;
    d.jo_mode = p.jo_mode;
    d.depth = (const uint16_t*)s.depth;
    d.labels = (const int32_t*)s.labels;
    d.lab = (const float4*)s.lab;
    d.pxyz = (const float4*)s.pxyz;
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
    b.pxyz = (float4*)s.pxyz;
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
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->scenes.find(scene_id);
    if (it == c->scenes.end()) return fail(c, PERCH_E_NOTFOUND, "unknown scene %d", scene_id);
    DeviceGuard g(c->device);
    SceneRec& s = it->second;
    if (in_use(s.use))
        return fail(c, PERCH_E_BUSY, "scene %d is in use (%d served requests or batch graphs, %zu unfinished "
                                     "asynchronous calls)", scene_id, s.use.users, s.use.pending.size());
    cudaStreamSynchronize(c->stream);
    dfree(c, s.depth); dfree(c, s.labels); dfree(c, s.lab); dfree(c, s.pts); dfree(c, s.table); dfree(c, s.nrm);
    dfree(c, s.near); dfree(c, s.cstart); dfree(c, s.pxyz);
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
    perch_status st = refuse_while_serving(c);
    if (st != PERCH_OK) return st;
    DeviceGuard g(c->device);
    perch::Job J;
    int mw;
    st = make_job(c, scene_id, mesh_id, label, roi, poses, costs, n, &J, &mw, nullptr, nullptr);
    if (st != PERCH_OK) return st;
    if (cuda_stream) {
        std::vector<perch::Job> jobs(1, J);
        st = run_jobs(c, c->plain, jobs, mw, c->cfg, (cudaStream_t)cuda_stream, nullptr);
        return st != PERCH_OK ? st : note_async_use(c, scene_id, mesh_id, (cudaStream_t)cuda_stream);
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

perch_status perch_best(perch_ctx* c, const int32_t* costs, const uint64_t* ids, int64_t n,
                        int64_t* best_index, int32_t* best_cost, void* cuda_stream)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (!costs || !best_index || !best_cost) return fail(c, PERCH_E_INVALID, "null pointer");
    if (n < 1 || n > 0x7FFFFFFFll) return fail(c, PERCH_E_INVALID, "n out of range");
    perch_status rs = refuse_while_serving(c);
    if (rs != PERCH_OK) return rs;
    DeviceGuard g(c->device);
    Range r("perch: argmin");
    perch::BestArgs a{};
    a.n = n;
    a.partial = c->d_best_partial;
    a.ticket = c->d_best_ticket;
    cudaError_t e;
    if (cuda_stream) {
        // every argmin of the context shares its scratch: run after the previous one
        cudaStream_t s = (cudaStream_t)cuda_stream;
        a.costs = costs;
        a.ids = (const unsigned long long*)ids;
        a.best_index = (long long*)best_index;
        a.best_cost = best_cost;
        e = cudaStreamWaitEvent(s, c->best_last, 0);
        if (!e) e = perch::launch_best(a, s);
        if (!e) e = cudaEventRecord(c->best_last, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "perch_best launch");
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
    if (!e) e = cudaStreamWaitEvent(c->stream, c->best_last, 0);
    if (!e) e = perch::launch_best(a, c->stream);
    if (!e) e = cudaEventRecord(c->best_last, c->stream);
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

perch_status perch_best_key(perch_ctx* c, const int32_t* costs, const uint64_t* ids, int64_t n, uint64_t* key,
                            void* cuda_stream)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (!costs || !key || !cuda_stream) return fail(c, PERCH_E_INVALID, "null costs, key or stream");
    if (n < 1 || n > 0x7FFFFFFFll) return fail(c, PERCH_E_INVALID, "n out of range");
    perch_status rs = refuse_while_serving(c);
    if (rs != PERCH_OK) return rs;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    perch::BestArgs a{};
    a.costs = costs;
    a.ids = (const unsigned long long*)ids;
    a.n = n;
    a.partial = c->d_best_partial;
    a.ticket = c->d_best_ticket;
    a.key = (unsigned long long*)key;
    cudaError_t e = cudaStreamWaitEvent(s, c->best_last, 0);
    if (!e) e = perch::launch_best(a, s);
    if (!e) e = cudaEventRecord(c->best_last, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "perch_best_key launch");
    return PERCH_OK;
}

perch_status perch_sync(perch_ctx* c, void* cuda_stream)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    perch_status st = refuse_while_serving(c);
    if (st != PERCH_OK) return st;
    DeviceGuard g(c->device);
    cudaError_t e = cudaStreamSynchronize(cuda_stream ? (cudaStream_t)cuda_stream : c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "perch_sync");
    return check_device_error(c);
}

perch_status perch_set_launch_config(perch_ctx* c, int32_t threads, int32_t zbuf_words,
                                     int32_t mark_bits)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (refuse_while_serving(c) != PERCH_OK) return PERCH_E_BUSY;
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

perch_status perch_set_raster_bins(perch_ctx* c, int32_t bin_cap)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (refuse_while_serving(c) != PERCH_OK) return PERCH_E_BUSY;
    if (bin_cap != 0 && (bin_cap < 64 || bin_cap > 65536))
        return fail(c, PERCH_E_INVALID, "bin capacity %d: 0 or 64 .. 65536", bin_cap);
    c->cfg.bin_cap = bin_cap;
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
    if (refuse_while_serving(c) != PERCH_OK) return PERCH_E_BUSY;
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
        if (e) return cuda_fail(c, e, "perch_pose_proposals");
        return note_async_use(c, scene_id, -1, (cudaStream_t)cuda_stream);
    }
    a.poses = (float*)c->stage;
    a.z_out = (int32_t*)(a.zr + 2);
    cudaError_t e = perch::launch_proposals(a, c->stream);
    if (!e) e = cudaMemcpyAsync(poses, a.poses, n * 48, cudaMemcpyDeviceToHost, c->stream);
    if (!e && z_range) e = cudaMemcpyAsync(z_range, a.z_out, 8, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    return e ? cuda_fail(c, e, "perch_pose_proposals") : PERCH_OK;
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
    if (refuse_while_serving(c) != PERCH_OK) return PERCH_E_BUSY;
    DeviceGuard g(c->device);
    const perch::DevMesh& m = mi->second.dm;
    if (cuda_stream) {
        cudaError_t e = perch::launch_add_s(m.verts, m.n_verts, poses, poses_true, n, symmetric ? 1 : 0, add,
                                            (cudaStream_t)cuda_stream);
        if (e) return cuda_fail(c, e, "perch_add_s");
        return note_async_use(c, -1, mesh_id, (cudaStream_t)cuda_stream);
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
    perch_status st = refuse_while_serving(c);
    if (st != PERCH_OK) return st;
    DeviceGuard g(c->device);
    st = ensure_stage(c, 64);
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

}  // extern "C"
