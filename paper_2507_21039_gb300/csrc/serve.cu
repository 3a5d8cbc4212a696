// Continuous-batching server for |M|^2 requests (declared in include/me_serve.h).
//
// One scheduler thread owns the queue.  It takes the oldest queued request,
// groups the queued requests of the same (process, precision) behind it into a
// batch of at most max_batch events, and starts the batch on a free lane (CUDA
// stream) as soon as the bytes of all batches in flight stay within the HBM
// budget.  A lane stages the requests' momenta into its pinned buffer, runs
// H2D copy -> |M|^2 kernel -> D2H copy (as a CUDA graph when enabled), and a
// host function queued behind the D2H copy scatters the results to the
// requests' buffers, stamps their latency and frees the lane.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "me.h"
#include "me_serve.h"

namespace {

using Clock = std::chrono::steady_clock;

enum State { QUEUED = 0, RUNNING = 1, DONE = 2, FAILED = 3, CANCELLED = 4 };

struct Request {
    uint64_t id = 0;
    std::string process;
    int precision = 0;
    int npar = 0;
    const double* mom = nullptr;
    int64_t nevt = 0;
    double* out = nullptr;
    Clock::time_point t_submit;
    int state = QUEUED;
    int status = ME_OK;
    double latency_us = 0.0;
};

struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
};

struct Lane {
    int index = 0;
    cudaStream_t stream = nullptr;
    double* d_mom = nullptr;
    double* d_me2 = nullptr;
    double* h_mom = nullptr;
    double* h_me2 = nullptr;
    bool busy = false;
    uint64_t bytes = 0;
    int64_t nevt = 0;
    std::vector<std::shared_ptr<Request>> batch;
    std::map<std::pair<std::string, int>, GraphSlot> graphs;
    struct srv_server* owner = nullptr;
};

constexpr int kMaxPar = 7;
constexpr int kMaxLanes = 16;

int npar_of(const char* process)
{
    static const std::pair<const char*, int> table[] = {
        {"ee_mumu", 4}, {"gg_ttx", 4}, {"gg_ttxg", 5}, {"gg_ttxgg", 6}, {"gg_ttxggg", 7}};
    for (auto& e : table)
        if (std::strcmp(process, e.first) == 0) return e.second;
    return 0;
}

bool is_pinned(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

}  // namespace

struct srv_server {
    srv_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work;   // scheduler: queue or lanes changed
    std::condition_variable cv_done;   // waiters: some request finished
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> tickets;
    std::map<std::pair<std::string, int>, me_handle*> handles;
    std::vector<Lane> lanes;
    uint64_t bytes_in_flight = 0;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread sched;
    // counters
    uint64_t n_requests = 0, n_batches = 0, n_events = 0, n_graph_updates = 0, n_graph_instantiations = 0,
             n_failed = 0, n_cancelled = 0, max_queue = 0, max_bytes_in_flight = 0;

    me_handle* handle_for(const std::string& proc, int prec, int* status);
    void run();
    void launch(Lane& lane, std::vector<std::shared_ptr<Request>> batch, uint64_t bytes);
    static void CUDART_CB on_done(void* arg);
};

// Resident handle per (process, precision): created and filtered on first use.
// The helicity mask comes from a fixed probe (seeded RAMBO at 2 TeV), so it does
// not depend on which request arrives first.
me_handle* srv_server::handle_for(const std::string& proc, int prec, int* status)
{
    auto key = std::make_pair(proc, prec);
    auto it = handles.find(key);
    if (it != handles.end()) return it->second;
    const int npar = npar_of(proc.c_str());
    double masses[kMaxPar] = {0};
    const bool qcd = proc != "ee_mumu";
    if (qcd) masses[2] = masses[3] = 173.0;
    me_handle* h = nullptr;
    *status = me_init(&h, proc.c_str(), masses, npar, nullptr, 0, prec);
    if (*status != ME_OK) return nullptr;
    const int64_t nprobe = 4096;
    double* d_probe = nullptr;
    if (cudaMalloc(&d_probe, sizeof(double) * 4 * npar * nprobe) != cudaSuccess) {
        me_free(h);
        *status = ME_ENOMEM;
        return nullptr;
    }
    *status = rambo_sample(20240607, 0, nprobe, qcd ? 2000.0 : 100.0, masses, npar, nullptr, d_probe, nullptr,
                           nullptr, nullptr);
    if (*status == ME_OK && cudaDeviceSynchronize() != cudaSuccess) *status = ME_ECUDA;
    if (*status == ME_OK) *status = me_filter_helicities(h, d_probe, nprobe, nullptr);
    // one direct launch outside any capture (sets kernel attributes once)
    if (*status == ME_OK) {
        double* d_out = nullptr;
        if (cudaMalloc(&d_out, sizeof(double) * nprobe) == cudaSuccess) {
            *status = me_sigmakin(h, d_probe, nprobe, d_out, nullptr);
            if (cudaDeviceSynchronize() != cudaSuccess && *status == ME_OK) *status = ME_ECUDA;
            cudaFree(d_out);
        }
    }
    cudaFree(d_probe);
    if (*status != ME_OK) {
        me_free(h);
        return nullptr;
    }
    handles[key] = h;
    return h;
}

void CUDART_CB srv_server::on_done(void* arg)
{
    Lane* lane = static_cast<Lane*>(arg);
    srv_server* s = lane->owner;
    const auto now = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        int64_t off = 0;
        for (auto& r : lane->batch) {
            if (r->state == RUNNING) {
                std::memcpy(r->out, lane->h_me2 + off, sizeof(double) * r->nevt);
                r->latency_us = std::chrono::duration<double, std::micro>(now - r->t_submit).count();
                r->state = DONE;
            }
            off += r->nevt;
        }
        lane->batch.clear();
        lane->busy = false;
        s->bytes_in_flight -= lane->bytes;
        lane->bytes = 0;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

void srv_server::launch(Lane& lane, std::vector<std::shared_ptr<Request>> batch, uint64_t bytes)
{
    const std::string proc = batch.front()->process;
    const int prec = batch.front()->precision;
    const int npar = batch.front()->npar;
    int status = ME_OK;
    me_handle* h = handle_for(proc, prec, &status);
    int64_t n = 0;
    if (h) {
        for (auto& r : batch) {  // stage into the lane's pinned buffer
            std::memcpy(lane.h_mom + n * npar * 4, r->mom, sizeof(double) * npar * 4 * r->nevt);
            n += r->nevt;
        }
    }
    auto fail = [&](int st) {
        std::lock_guard<std::mutex> lock(mu);
        for (auto& r : batch) {
            if (r->state == RUNNING) r->state = FAILED;
            r->status = st;
        }
        n_failed += batch.size();
        lane.busy = false;
        bytes_in_flight -= bytes;
        cv_done.notify_all();
        cv_work.notify_all();
    };
    if (!h) return fail(status);
    const size_t mbytes = sizeof(double) * npar * 4 * n;
    lane.batch = std::move(batch);
    lane.bytes = bytes;
    lane.nevt = n;
    cudaError_t e = cudaSuccess;
    if (cfg.use_graphs) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(lane.stream, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            cudaMemcpyAsync(lane.d_mom, lane.h_mom, mbytes, cudaMemcpyHostToDevice, lane.stream);
            status = me_sigmakin(h, lane.d_mom, n, lane.d_me2, lane.stream);
            cudaMemcpyAsync(lane.h_me2, lane.d_me2, sizeof(double) * n, cudaMemcpyDeviceToHost, lane.stream);
            e = cudaStreamEndCapture(lane.stream, &g);
        }
        if (e == cudaSuccess && status == ME_OK) {
            GraphSlot& slot = lane.graphs[std::make_pair(proc, prec)];
            bool ok = false;
            if (slot.exec) {
                cudaGraphExecUpdateResultInfo info;
                if (cudaGraphExecUpdate(slot.exec, g, &info) == cudaSuccess) {
                    ok = true;
                    ++n_graph_updates;
                } else {
                    cudaGetLastError();
                    cudaGraphExecDestroy(slot.exec);
                    slot.exec = nullptr;
                }
            }
            if (!ok) {
                e = cudaGraphInstantiate(&slot.exec, g, 0);
                ++n_graph_instantiations;
            }
            if (e == cudaSuccess) e = cudaGraphLaunch(slot.exec, lane.stream);
        }
        if (g) cudaGraphDestroy(g);
    } else {
        e = cudaMemcpyAsync(lane.d_mom, lane.h_mom, mbytes, cudaMemcpyHostToDevice, lane.stream);
        if (e == cudaSuccess) status = me_sigmakin(h, lane.d_mom, n, lane.d_me2, lane.stream);
        if (e == cudaSuccess && status == ME_OK)
            e = cudaMemcpyAsync(lane.h_me2, lane.d_me2, sizeof(double) * n, cudaMemcpyDeviceToHost, lane.stream);
    }
    if (e == cudaSuccess && status == ME_OK) e = cudaLaunchHostFunc(lane.stream, &srv_server::on_done, &lane);
    if (e != cudaSuccess || status != ME_OK) {
        cudaGetLastError();
        std::vector<std::shared_ptr<Request>> b = std::move(lane.batch);
        lane.batch.clear();
        lane.bytes = 0;
        batch = std::move(b);
        return fail(status != ME_OK ? status : ME_ECUDA);
    }
}

void srv_server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    while (true) {
        cv_work.wait(lock, [&] {
            if (stop) return true;
            if (queue.empty()) return false;
            for (auto& l : lanes)
                if (!l.busy) return true;
            return false;
        });
        if (stop) break;
        // oldest request first; same (process, precision) requests behind it join its batch
        auto head = queue.front();
        const uint64_t per_event = sizeof(double) * (4 * head->npar + 1);
        std::vector<std::shared_ptr<Request>> batch;
        int64_t n = 0;
        for (auto it = queue.begin(); it != queue.end();) {
            auto& r = *it;
            if (r->process == head->process && r->precision == head->precision && n + r->nevt <= cfg.max_batch) {
                n += r->nevt;
                batch.push_back(r);
                it = queue.erase(it);
            } else {
                ++it;
            }
        }
        const uint64_t bytes = per_event * (uint64_t)n;
        if (bytes_in_flight > 0 && bytes_in_flight + bytes > cfg.hbm_budget_bytes) {
            // not enough device memory budget yet: put the batch back, wait for a completion
            for (auto rit = batch.rbegin(); rit != batch.rend(); ++rit) queue.push_front(*rit);
            cv_work.wait(lock, [&] { return stop || bytes_in_flight + bytes <= cfg.hbm_budget_bytes; });
            continue;
        }
        Lane* lane = nullptr;
        for (auto& l : lanes)
            if (!l.busy) {
                lane = &l;
                break;
            }
        lane->busy = true;
        bytes_in_flight += bytes;
        max_bytes_in_flight = std::max(max_bytes_in_flight, bytes_in_flight);
        for (auto& r : batch) r->state = RUNNING;
        ++n_batches;
        n_events += n;
        lock.unlock();
        launch(*lane, std::move(batch), bytes);
        lock.lock();
    }
}

extern "C" {

int srv_create(srv_server** out, const srv_config* cfg)
{
    if (!out || !cfg || cfg->lanes < 1 || cfg->lanes > kMaxLanes || cfg->max_batch < 1) return ME_EINVAL;
    *out = nullptr;
    std::unique_ptr<srv_server> s(new (std::nothrow) srv_server());
    if (!s) return ME_ENOMEM;
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    s->lanes.resize(cfg->lanes);
    const size_t mom_bytes = sizeof(double) * 4 * kMaxPar * (size_t)cfg->max_batch;
    const size_t me2_bytes = sizeof(double) * (size_t)cfg->max_batch;
    int rc = ME_OK;
    for (int i = 0; i < cfg->lanes && rc == ME_OK; ++i) {
        Lane& l = s->lanes[i];
        l.index = i;
        l.owner = s.get();
        if (cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) != cudaSuccess) rc = ME_ECUDA;
        else if (cudaMalloc(&l.d_mom, mom_bytes) != cudaSuccess || cudaMalloc(&l.d_me2, me2_bytes) != cudaSuccess ||
                 cudaMallocHost(&l.h_mom, mom_bytes) != cudaSuccess ||
                 cudaMallocHost(&l.h_me2, me2_bytes) != cudaSuccess)
            rc = ME_ENOMEM;
    }
    if (rc != ME_OK) {
        cudaGetLastError();
        srv_destroy(s.release());
        return rc;
    }
    srv_server* raw = s.release();
    raw->sched = std::thread([raw] { raw->run(); });
    *out = raw;
    return ME_OK;
}

int srv_submit(srv_server* s, const char* process, int precision, const double* momenta, int64_t nevt,
               double* me2_out, uint64_t* ticket)
{
    if (!s || !process || !momenta || !me2_out || !ticket) return ME_EINVAL;
    const int npar = npar_of(process);
    if (!npar || nevt <= 0 || nevt > s->cfg.max_batch || precision < ME_PREC_FP64 || precision > ME_PREC_MIXED64)
        return ME_EINVAL;
    auto r = std::make_shared<Request>();
    r->process = process;
    r->precision = precision;
    r->npar = npar;
    r->mom = momenta;
    r->nevt = nevt;
    r->out = me2_out;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        r->id = s->next_id++;
        s->queue.push_back(r);
        s->tickets[r->id] = r;
        ++s->n_requests;
        s->max_queue = std::max<uint64_t>(s->max_queue, s->queue.size());
        *ticket = r->id;
    }
    s->cv_work.notify_all();
    return ME_OK;
}

int srv_wait(srv_server* s, uint64_t ticket, int timeout_ms, double* latency_us)
{
    if (!s) return ME_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return ME_EINVAL;
    auto r = it->second;
    auto finished = [&] { return r->state == DONE || r->state == FAILED || r->state == CANCELLED; };
    if (timeout_ms < 0) s->cv_done.wait(lock, finished);
    else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), finished)) return ME_ETIMEOUT;
    s->tickets.erase(ticket);
    if (latency_us) *latency_us = r->latency_us;
    if (r->state == DONE) return ME_OK;
    if (r->state == CANCELLED) return ME_EINVAL;
    return r->status != ME_OK ? r->status : ME_ECUDA;
}

int srv_cancel(srv_server* s, uint64_t ticket)
{
    if (!s) return ME_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return ME_EINVAL;
    auto r = it->second;
    if (r->state == QUEUED) {
        auto q = std::find(s->queue.begin(), s->queue.end(), r);
        if (q != s->queue.end()) s->queue.erase(q);
    }
    if (r->state == QUEUED || r->state == RUNNING) {
        r->state = CANCELLED;
        ++s->n_cancelled;
    }
    s->tickets.erase(it);
    s->cv_done.notify_all();
    return ME_OK;
}

int srv_stats(srv_server* s, char* buf, int cap)
{
    if (!s || !buf || cap <= 0) return ME_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    int busy = 0;
    for (auto& l : s->lanes) busy += l.busy;
    snprintf(buf, cap,
             "{\"requests\": %llu, \"batches\": %llu, \"events\": %llu, \"queue_depth\": %zu, \"max_queue_depth\": "
             "%llu, \"lanes_busy\": %d, \"bytes_in_flight\": %llu, \"graph_updates\": %llu, "
             "\"graph_instantiations\": %llu, \"failed\": %llu, \"cancelled\": %llu, \"handles\": %zu, "
             "\"max_bytes_in_flight\": %llu}",
             (unsigned long long)s->n_requests, (unsigned long long)s->n_batches, (unsigned long long)s->n_events,
             s->queue.size(), (unsigned long long)s->max_queue, busy, (unsigned long long)s->bytes_in_flight,
             (unsigned long long)s->n_graph_updates, (unsigned long long)s->n_graph_instantiations,
             (unsigned long long)s->n_failed, (unsigned long long)s->n_cancelled, s->handles.size(),
             (unsigned long long)s->max_bytes_in_flight);
    return ME_OK;
}

void srv_destroy(srv_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->queue.clear();
    }
    s->cv_work.notify_all();
    if (s->sched.joinable()) s->sched.join();
    for (auto& l : s->lanes)
        if (l.stream) cudaStreamSynchronize(l.stream);
    for (auto& l : s->lanes) {
        for (auto& kv : l.graphs)
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (l.stream) cudaStreamDestroy(l.stream);
        cudaFree(l.d_mom);
        cudaFree(l.d_me2);
        cudaFreeHost(l.h_mom);
        cudaFreeHost(l.h_me2);
    }
    for (auto& kv : s->handles) me_free(kv.second);
    delete s;
}

}  // extern "C"
