// libperch served form: a continuous-batching server over launch slots
// (include/perch.h, "served form").
#include "perch_host.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>

using namespace perch_host;


namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServedRequest {
    uint64_t ticket = 0;
    int32_t scene_id = 0, mesh_id = 0;   // counted as users of both until the request completes
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
    std::mutex mu;                  // queue, slots, tickets (the context's own state: c->mu)
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
            std::lock_guard<std::mutex> g(S->c->mu);
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
            {
                // its scene and mesh may be released from now on
                std::lock_guard<std::mutex> g(S->c->mu);
                count_users(S->c, r->scene_id, r->mesh_id, -1);
            }
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
    c->servers.fetch_add(1);
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
    r->poses.assign(req->poses, req->poses + 12 * req->n);
    r->user_costs = req->costs;
    r->n = req->n;
    r->scene_id = req->scene_id;
    r->mesh_id = req->mesh_id;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return PERCH_E_BUSY;
    {
        // validated and counted as a user of its scene and mesh under the
        // context's lock, so a concurrent release either precedes it (the
        // ids are gone: PERCH_E_NOTFOUND) or is refused (PERCH_E_BUSY)
        std::lock_guard<std::mutex> g(S->c->mu);
        const int32_t* roi = (req->roi[2] > req->roi[0] && req->roi[3] > req->roi[1]) ? req->roi : nullptr;
        perch_status st = make_job(S->c, req->scene_id, req->mesh_id, req->label, roi, nullptr, nullptr,
                                   req->n, &r->tmpl, &r->mark_words, nullptr, nullptr);
        if (st != PERCH_OK) return st;
        count_users(S->c, req->scene_id, req->mesh_id, +1);
    }
    r->t_submit = now_ns();
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

perch_status perch_ticket_release(perch_server* S, uint64_t ticket)
{
    if (!S) return PERCH_E_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return PERCH_E_NOTFOUND;
    if (!it->second->done) return PERCH_E_BUSY;
    S->tickets.erase(it);
    return PERCH_OK;
}

perch_status perch_server_tickets(perch_server* S, int64_t* held)
{
    if (!S || !held) return PERCH_E_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    *held = (int64_t)S->tickets.size();
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
    c->servers.fetch_sub(1);
    delete S;
    return PERCH_OK;
}

}  // extern "C"
