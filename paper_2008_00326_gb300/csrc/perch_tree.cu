// libperch Monotone Scene Generation tree search (Sec. III, Fig. 2; variant
// 2.0-B): a level-wise beam over tree edges scored by the scorer's tree
// kernel against device state images.
#include "perch_host.cuh"

#include <algorithm>

using namespace perch_host;

extern "C" {

perch_status perch_tree_search(perch_ctx* c, int32_t scene_id, const perch_tree_object* objects, int32_t K,
                               int32_t beam_width, int32_t* order, int32_t* pose_index, int64_t* level_cost,
                               int64_t* edges_scored)
{
    if (!c) return PERCH_E_INVALID;
    c->err.clear();
    if (!objects || !order || !pose_index || !level_cost) return fail(c, PERCH_E_INVALID, "null argument");
    if (K < 1 || K > 64) return fail(c, PERCH_E_INVALID, "K must be in [1, 64]");
    if (beam_width < 1 || beam_width > 4096) return fail(c, PERCH_E_INVALID, "beam_width must be in [1, 4096]");
    if (refuse_while_serving(c) != PERCH_OK) return PERCH_E_BUSY;
    Range r("perch: tree search");
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

}  // extern "C"
