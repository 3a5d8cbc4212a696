// Continuous-batching server for |M|^2 requests (declared in include/me_serve.h).
//
// One scheduler thread owns the queue.  It takes the oldest queued request
// whose batch fits the HBM budget, groups the queued requests of the same
// (process, precision) behind it into a batch of at most max_batch events, and
// starts the batch on a free lane (CUDA stream).  A request that does not fit
// yet is passed over by later, smaller ones at most kMaxBypass times; then the
// scheduler waits for it.  A batch's device bytes are its momenta and |M|^2
// plus the global scratch its launch allocates (the FP64 colour-flow vectors of
// the largest process).  A lane stages the requests' momenta into its pinned
// buffer, runs H2D copy -> |M|^2 kernel -> D2H copy (as a CUDA graph when
// enabled) between two timing events, and a host function queued behind the
// D2H copy scatters the results to the requests' buffers, stamps their
// latency and frees the lane.  The scheduler thread reads the timing events of
// finished batches (a host function may not call CUDA) and keeps the largest
// number of batches seen running at once on the device.
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
#include "me_proc.h"
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
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;  // device time of the lane's current batch
    bool timing_pending = false;                        // a finished batch whose events are not read yet
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
constexpr int kMaxBypass = 8;        // times the oldest request may be passed over by later ones
constexpr size_t kMaxIntervals = 4096;  // device intervals of recent batches kept for the overlap count

int npar_of(const char* process)
{
    const me::ProcDesc* pd = me::find_process(process);
    return pd && pd->npar <= kMaxPar ? pd->npar : 0;
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
             n_failed = 0, n_cancelled = 0, max_queue = 0, max_bytes_in_flight = 0, n_bypass = 0;
    int max_lanes_busy = 0;           // host view: lanes holding a launched, unfinished batch at once
    int max_device_concurrency = 0;   // device view: batches whose kernels ran at overlapping times
    int head_bypassed = 0;            // times the current oldest request was passed over
    uint64_t lane_buffer_bytes = 0;   // fixed device bytes of the lanes' buffers
    cudaEvent_t ev_ref = nullptr;     // time origin of the device intervals
    std::deque<std::pair<float, float>> intervals;
    void read_timings();

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
    const me::ProcDesc* pd = me::find_process(proc.c_str());
    double masses[kMaxPar] = {0};
    const bool qcd = pd && pd->family == 1;  // g g -> t t~ + n g: massive tops
    if (qcd) masses[2] = masses[3] = 173.0;
    const double probe_sqrt_s = qcd ? 2000.0 : (pd && pd->family == 2 ? 500.0 : 100.0);
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
    *status = rambo_sample(20240607, 0, nprobe, probe_sqrt_s, masses, npar, nullptr, d_probe, nullptr, nullptr,
                           nullptr);
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
        lane->timing_pending = true;
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
            // external records: the graph records the events each time it runs
            cudaEventRecordWithFlags(lane.ev_start, lane.stream, cudaEventRecordExternal);
            cudaMemcpyAsync(lane.d_mom, lane.h_mom, mbytes, cudaMemcpyHostToDevice, lane.stream);
            status = me_sigmakin(h, lane.d_mom, n, lane.d_me2, lane.stream);
            cudaMemcpyAsync(lane.h_me2, lane.d_me2, sizeof(double) * n, cudaMemcpyDeviceToHost, lane.stream);
            cudaEventRecordWithFlags(lane.ev_end, lane.stream, cudaEventRecordExternal);
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
        e = cudaEventRecord(lane.ev_start, lane.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(lane.d_mom, lane.h_mom, mbytes, cudaMemcpyHostToDevice, lane.stream);
        if (e == cudaSuccess) status = me_sigmakin(h, lane.d_mom, n, lane.d_me2, lane.stream);
        if (e == cudaSuccess && status == ME_OK)
            e = cudaMemcpyAsync(lane.h_me2, lane.d_me2, sizeof(double) * n, cudaMemcpyDeviceToHost, lane.stream);
        if (e == cudaSuccess && status == ME_OK) e = cudaEventRecord(lane.ev_end, lane.stream);
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

// Device bytes of one batch: momenta and |M|^2 of its events in the lane's
// buffers, plus the global scratch the launch allocates (the FP64 colour-flow
// vectors of the largest process: per resident CTA, times the resident CTAs)
uint64_t batch_bytes(const std::string& process, int precision, int npar, int64_t n)
{
    uint64_t b = sizeof(double) * (4 * (uint64_t)npar + 1) * (uint64_t)n;
    if (const me::ProcDesc* pd = me::find_process(process.c_str())) {
        const size_t per = pd->jscratch_per_cta(precision);
        if (per) b += (uint64_t)per * (uint64_t)std::max(1, pd->jscratch_ctas(precision));
    }
    return b;
}

// Device intervals of the batches finished since the last call (scheduler
// thread, lock held): each new interval is compared with the recent ones to
// find the largest number of batches that ran at the same time.
void srv_server::read_timings()
{
    for (auto& l : lanes) {
        if (!l.timing_pending || l.busy) continue;
        l.timing_pending = false;
        float t0 = 0.0f, t1 = 0.0f;
        if (cudaEventElapsedTime(&t0, ev_ref, l.ev_start) != cudaSuccess ||
            cudaEventElapsedTime(&t1, ev_ref, l.ev_end) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        // largest overlap count at the start of the new interval or of any stored one inside it
        std::vector<float> points{t0};
        for (auto& iv : intervals)
            if (iv.first > t0 && iv.first < t1) points.push_back(iv.first);
        for (float p : points) {
            int c = (p >= t0 && p < t1) ? 1 : 0;
            for (auto& iv : intervals) c += (iv.first <= p && p < iv.second) ? 1 : 0;
            max_device_concurrency = std::max(max_device_concurrency, c);
        }
        intervals.emplace_back(t0, t1);
        if (intervals.size() > kMaxIntervals) intervals.pop_front();
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
        read_timings();
        // the oldest request whose batch fits the budget (the oldest one itself once
        // it has been passed over kMaxBypass times); the queued requests of the
        // same (process, precision) behind it join its batch
        std::vector<std::shared_ptr<Request>> batch;
        uint64_t bytes = 0;
        bool head = true;
        for (size_t qi = 0; qi < queue.size(); ++qi) {
            const auto cand = queue[qi];
            bool seen = false;  // a group already considered (an earlier request of the same kind)
            for (size_t j = 0; j < qi && !seen; ++j)
                seen = queue[j]->process == cand->process && queue[j]->precision == cand->precision;
            if (seen) continue;
            int64_t n = 0;
            for (auto& r : queue)
                if (r->process == cand->process && r->precision == cand->precision && n + r->nevt <= cfg.max_batch)
                    n += r->nevt;
            const uint64_t b = batch_bytes(cand->process, cand->precision, cand->npar, n);
            if (bytes_in_flight == 0 || bytes_in_flight + b <= cfg.hbm_budget_bytes) {
                bytes = b;
                for (auto it = queue.begin(); it != queue.end();) {
                    auto& r = *it;
                    if (r->process == cand->process && r->precision == cand->precision &&
                        (int64_t)(r->nevt) <= n) {
                        n -= r->nevt;
                        batch.push_back(r);
                        it = queue.erase(it);
                    } else {
                        ++it;
                    }
                }
                break;
            }
            if (head && head_bypassed >= kMaxBypass) break;  // the oldest request waits for room
            head = false;
        }
        if (batch.empty()) {  // nothing fits the budget yet: wait for a completion or a new request
            const uint64_t before = bytes_in_flight;
            const size_t queued = queue.size();
            cv_work.wait(lock, [&] { return stop || bytes_in_flight < before || queue.size() != queued; });
            continue;
        }
        if (head) {
            head_bypassed = 0;
        } else {
            ++head_bypassed;
            ++n_bypass;
        }
        Lane* lane = nullptr;
        for (auto& l : lanes)
            if (!l.busy) {
                lane = &l;
                break;
            }
        lane->busy = true;
        int busy = 0;
        for (auto& l : lanes) busy += l.busy;
        max_lanes_busy = std::max(max_lanes_busy, busy);
        bytes_in_flight += bytes;
        max_bytes_in_flight = std::max(max_bytes_in_flight, bytes_in_flight);
        int64_t n = 0;
        for (auto& r : batch) {
            r->state = RUNNING;
            n += r->nevt;
        }
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
        if (cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&l.ev_start) != cudaSuccess || cudaEventCreate(&l.ev_end) != cudaSuccess)
            rc = ME_ECUDA;
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
    if (cudaEventCreate(&s->ev_ref) != cudaSuccess || cudaEventRecord(s->ev_ref, 0) != cudaSuccess ||
        cudaEventSynchronize(s->ev_ref) != cudaSuccess) {
        cudaGetLastError();
        srv_destroy(s.release());
        return ME_ECUDA;
    }
    s->lane_buffer_bytes = (uint64_t)cfg->lanes * (mom_bytes + me2_bytes);
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
    s->read_timings();
    int busy = 0;
    for (auto& l : s->lanes) busy += l.busy;
    snprintf(buf, cap,
             "{\"requests\": %llu, \"batches\": %llu, \"events\": %llu, \"queue_depth\": %zu, \"max_queue_depth\": "
             "%llu, \"lanes_busy\": %d, \"bytes_in_flight\": %llu, \"graph_updates\": %llu, "
             "\"graph_instantiations\": %llu, \"failed\": %llu, \"cancelled\": %llu, \"handles\": %zu, "
             "\"max_bytes_in_flight\": %llu, \"max_lanes_busy\": %d, \"max_device_concurrency\": %d, "
             "\"head_bypasses\": %llu, \"lane_buffer_bytes\": %llu}",
             (unsigned long long)s->n_requests, (unsigned long long)s->n_batches, (unsigned long long)s->n_events,
             s->queue.size(), (unsigned long long)s->max_queue, busy, (unsigned long long)s->bytes_in_flight,
             (unsigned long long)s->n_graph_updates, (unsigned long long)s->n_graph_instantiations,
             (unsigned long long)s->n_failed, (unsigned long long)s->n_cancelled, s->handles.size(),
             (unsigned long long)s->max_bytes_in_flight, s->max_lanes_busy, s->max_device_concurrency,
             (unsigned long long)s->n_bypass, (unsigned long long)s->lane_buffer_bytes);
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
        if (l.ev_start) cudaEventDestroy(l.ev_start);
        if (l.ev_end) cudaEventDestroy(l.ev_end);
        cudaFree(l.d_mom);
        cudaFree(l.d_me2);
        cudaFreeHost(l.h_mom);
        cudaFreeHost(l.h_me2);
    }
    for (auto& kv : s->handles) me_free(kv.second);
    if (s->ev_ref) cudaEventDestroy(s->ev_ref);
    delete s;
}

}  // extern "C"
