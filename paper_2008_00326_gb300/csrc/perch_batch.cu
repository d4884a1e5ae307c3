// libperch batched form: many scenes' searches in one call, the same batch as
// a replayable CUDA graph, and the launch-shape autotuner (include/perch.h,
// "batched form").
#include "perch_host.cuh"

#include <algorithm>
#include <cstring>

using namespace perch_host;

namespace {

// Validate a batch and turn it into jobs; `base_poses` / `base_costs` are the
// arrays the item offsets index.
perch_status batch_jobs(perch_ctx* c, const perch_work_item* items, int32_t n_items,
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

}  // namespace

extern "C" {

perch_status perch_score_batch(perch_ctx* c, const perch_work_item* items, int32_t n_items,
                               const float* poses, int32_t* costs, void* cuda_stream)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (!poses || !costs) return fail(c, PERCH_E_INVALID, "null poses or costs");
    perch_status st = refuse_while_serving(c);
    if (st != PERCH_OK) return st;
    DeviceGuard g(c->device);
    std::vector<perch::Job> jobs;
    int mw;
    long long total;
    long long extent = 0;
    for (int32_t i = 0; items && i < n_items; ++i) extent = std::max<long long>(extent, items[i].pose_offset + items[i].n);
    if (cuda_stream) {
        st = batch_jobs(c, items, n_items, poses, costs, &jobs, &mw, &total);
        if (st != PERCH_OK) return st;
        cudaStream_t s = (cudaStream_t)cuda_stream;
        st = run_jobs(c, c->plain, jobs, mw, c->cfg, s, nullptr);
        for (int32_t i = 0; i < n_items && st == PERCH_OK; ++i)
            if (items[i].n > 0) st = note_async_use(c, items[i].scene_id, items[i].mesh_id, s);
        return st;
    }
    st = ensure_stage(c, (size_t)std::max<long long>(1, extent) * (48 + 8));
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

perch_status perch_batch_graph_create(perch_ctx* c, const perch_work_item* items, int32_t n_items,
                                      const float* poses, int32_t* costs, perch_batch_graph** out)
{
    if (!c || !out) return PERCH_E_INVALID;
    c->err.clear();
    *out = nullptr;
    if (!poses || !costs) return fail(c, PERCH_E_INVALID, "null poses or costs");
    perch_status st = refuse_while_serving(c);
    if (st != PERCH_OK) return st;
    DeviceGuard g(c->device);
    std::vector<perch::Job> jobs;
    int mw;
    long long total;
    st = batch_jobs(c, items, n_items, poses, costs, &jobs, &mw, &total);
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
    long long bin_off = 0;
    const long long vstride = small_images ? perch::vcache_slot_words(max_verts, cfg.bin_cap, &bin_off) : 0;
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
        a.bin_cap = vstride ? cfg.bin_cap : 0;
        a.bin_off = bin_off;
        a.vmask = G->next + nj;
        a.vslots = resident;
        cudaGraphNode_t dep = (j >= 4 && nodes[j - 4]) ? nodes[j - 4] : reset;
        e = perch::add_score_node(G->graph, &dep, 1, a, cfg, resident, &nodes[j]);
    }
    if (st == PERCH_OK && !e) e = cudaGraphInstantiate(&G->exec, G->graph, 0);
    if (st == PERCH_OK && !e) e = cudaEventCreateWithFlags(&G->done, cudaEventDisableTiming);
    if (st == PERCH_OK && e) st = cuda_fail(c, e, "perch_batch_graph_create");
    if (st != PERCH_OK) {
        perch_batch_graph_destroy(G);
        return st;
    }
    // the graph reads its items' scenes and meshes until it is destroyed
    for (int32_t i = 0; i < n_items; ++i)
        if (items[i].n > 0) {
            G->uses.push_back({items[i].scene_id, items[i].mesh_id});
            count_users(c, items[i].scene_id, items[i].mesh_id, +1);
        }
    *out = G;
    return PERCH_OK;
}

perch_status perch_batch_graph_launch(perch_batch_graph* G, void* cuda_stream)
{
    if (!G || !G->exec) return PERCH_E_INVALID;
    DeviceGuard g(G->ctx->device);
    cudaError_t e = cudaGraphLaunch(G->exec, (cudaStream_t)cuda_stream);
    if (!e) e = cudaEventRecord(G->done, (cudaStream_t)cuda_stream);
    if (e) return cuda_fail(G->ctx, e, "perch_batch_graph_launch");
    return PERCH_OK;
}

perch_status perch_batch_graph_destroy(perch_batch_graph* G)
{
    if (!G) return PERCH_OK;
    perch_ctx* c = G->ctx;
    DeviceGuard g(c->device);
    // waits for the graph's last launch only, not for the rest of the device
    if (G->done) {
        cudaEventSynchronize(G->done);
        cudaEventDestroy(G->done);
    }
    {
        std::lock_guard<std::mutex> lk(c->mu);
        for (const auto& u : G->uses) count_users(c, u.first, u.second, -1);
    }
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    dfree(c, G->next);
    dfree(c, G->vcache);
    delete G;
    return PERCH_OK;
}

perch_status perch_autotune(perch_ctx* c, const perch_work_item* items, int32_t n_items,
                            const float* poses, int32_t* costs, int32_t* threads, int32_t* zbuf_words,
                            int32_t* bin_cap)
{
    if (!c || !threads || !zbuf_words) return PERCH_E_INVALID;
    c->err.clear();
    if (!items || n_items < 1 || !poses || !costs) return fail(c, PERCH_E_INVALID, "empty batch");
    perch_status rs = refuse_while_serving(c);
    if (rs != PERCH_OK) return rs;
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
        c->cfg.bin_cap = hit->second.bin_cap;
        *threads = c->cfg.threads;
        *zbuf_words = c->cfg.zcap_words;
        if (bin_cap) *bin_cap = c->cfg.bin_cap;
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
    // threads x z-buffer words x tile-bin capacity; bins only where small
    // z-buffers make several tiles per hypothesis likely
    const int th[3] = {128, 256, 512};
    const int zw[5] = {2048, 4096, 7064, 8192, 16384};
    const int bc[3] = {0, 1024, 4096};
    for (int ti = 0; ti < 3 && st == PERCH_OK; ++ti) {
        for (int zi = 0; zi < 5 && st == PERCH_OK; ++zi) {
          for (int bi = 0; bi < (zw[zi] <= 4096 ? 3 : 1) && st == PERCH_OK; ++bi) {
            perch::ScoreConfig cfg = saved;
            cfg.threads = th[ti];
            cfg.zcap_words = zw[zi];
            cfg.bin_cap = bc[bi];
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
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PERCH_OK) return st;
    c->cfg.threads = best.threads;
    c->cfg.zcap_words = best.zcap_words;
    c->cfg.bin_cap = best.bin_cap;
    c->tuned[key] = c->cfg;
    *threads = c->cfg.threads;
    *zbuf_words = c->cfg.zcap_words;
    if (bin_cap) *bin_cap = c->cfg.bin_cap;
    return check_device_error(c);
}

}  // extern "C"
