// Request server: independent projections submitted by any host thread,
// admitted under a device-memory budget and run by worker threads, each with
// its own context and CUDA stream (the served workload: Poisson arrivals of
// matrices of many sizes, each projected by Alg. 2 or Alg. 3 of the paper).
//
// Built on the public C ABI only (psdproj_create / psdproj_alg1 /
// psdproj_alg2 / psdproj_sync_status).  Admission is first come, first
// served: the request at the head of the queue is admitted when its
// footprint fits under the budget together with the requests already
// admitted and not finished; later requests wait behind it, so none starves.
// A worker runs one request at a time on its stream, waits for it on a
// blocking-sync event, reads its context's status word (so a device error is
// charged to that request alone) and releases its footprint.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/psdproj.h"

namespace {

using clock_type = std::chrono::steady_clock;

enum { T_QUEUED = 0, T_READY = 1, T_RUNNING = 2, T_DONE = 3 };

struct Ticket {
    psdproj_request req;
    size_t bytes = 0;
    int state = T_QUEUED;
    int status = 0;
    clock_type::time_point t_submit, t_done;
};

// Device memory a request holds while admitted: its A, P and W, and the
// workspace and image of A that the worker context running it needs for
// this request's size, sketch width and form (a worker keeps what it grew
// to for its largest request; the charge is this request's own need).
size_t default_footprint(const psdproj_request &r, const psdproj_opts &o)
{
    size_t b = (size_t)r.n * (size_t)r.lda * sizeof(float);
    if (r.dP) b += (size_t)r.n * (size_t)r.ldp * sizeof(float);
    if (r.dW) b += (size_t)r.ldw * (size_t)(r.k + r.p) * sizeof(float);
    b += psdproj_projection_bytes(r.n, r.k, r.p, &o);
    return b;
}

int check_request(const psdproj_request &r, int out_mode)
{
    if (!r.dA || r.n < 1 || r.lda < r.n || r.k < 1 || r.p < 0 || r.q < 0 || r.q > 16) return PSDPROJ_EINVAL;
    if (r.algorithm != 1 && r.algorithm != 2) return PSDPROJ_EINVAL;
    const int64_t m = (int64_t)r.k + r.p;
    if (m > r.n || m > PSDPROJ_MAX_M) return PSDPROJ_EINVAL;
    if (out_mode != PSDPROJ_OUT_FACTOR && (!r.dP || r.ldp < r.n)) return PSDPROJ_EINVAL;
    if (r.dW && r.ldw < r.n) return PSDPROJ_EINVAL;
    return PSDPROJ_OK;
}

}  // namespace

struct psdproj_server {
    int device = 0;
    psdproj_opts opts;
    size_t admit_bytes = 0;
    std::vector<psdproj_ctx *> ctx;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done_ev;
    std::vector<std::thread> workers;

    std::mutex mu;
    std::condition_variable cv_work;   // an admitted request or stop
    std::condition_variable cv_done;   // a request finished
    std::deque<uint64_t> pending;      // submitted, waiting for admission
    std::deque<uint64_t> ready;        // admitted, waiting for a worker
    std::unordered_map<uint64_t, Ticket> tickets;
    uint64_t next_ticket = 1;
    size_t inflight = 0, inflight_peak = 0;
    int running = 0;
    uint64_t submitted = 0, completed = 0, failed = 0;
    int last_status = 0, last_cuda = 0, last_line = 0;
    bool stop = false;

    // called with mu held: admit from the head of the queue while it fits
    void admit()
    {
        bool any = false;
        while (!pending.empty()) {
            Ticket &t = tickets[pending.front()];
            if (inflight + t.bytes > admit_bytes) break;
            inflight += t.bytes;
            inflight_peak = std::max(inflight_peak, inflight);
            t.state = T_READY;
            ready.push_back(pending.front());
            pending.pop_front();
            any = true;
        }
        if (any) cv_work.notify_all();
    }

    void worker(int w)
    {
        cudaSetDevice(device);
        for (;;) {
            uint64_t id;
            psdproj_request r;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stop || !ready.empty(); });
                if (ready.empty()) return;   // stop requested and nothing admitted
                id = ready.front();
                ready.pop_front();
                Ticket &t = tickets[id];
                t.state = T_RUNNING;
                r = t.req;
                ++running;
            }
            int rc;
            if (r.algorithm == 1)
                rc = psdproj_alg1(ctx[w], r.dA, r.n, r.lda, r.k, r.p, r.q, r.seed, r.dP, r.ldp, r.dW, r.ldw,
                                  r.d_rank, &opts);
            else
                rc = psdproj_alg2(ctx[w], r.dA, r.n, r.lda, r.k, r.p, r.q, r.seed, r.alpha_in, r.d_alpha_out,
                                  r.d_info, r.dP, r.ldp, r.dW, r.ldw, r.d_rank, &opts);
            // wait without spinning, then read (and clear) this context's
            // device status: it belongs to this request alone
            cudaError_t e = cudaEventRecord(done_ev[w], streams[w]);
            if (e == cudaSuccess) e = cudaEventSynchronize(done_ev[w]);
            int cuda_err = 0, cuda_line = 0;
            if (rc != PSDPROJ_OK) cuda_err = psdproj_last_cuda_error(&cuda_line);
            const int st = psdproj_sync_status(ctx[w]);
            if (rc == PSDPROJ_OK && e != cudaSuccess) {
                rc = PSDPROJ_ECUDA;
                cuda_err = (int)e;
                cuda_line = -__LINE__;          // negative: a line of this file
            }
            if (rc == PSDPROJ_OK && st != PSDPROJ_OK) {
                rc = st;
                if (st == PSDPROJ_ECUDA) cuda_err = psdproj_last_cuda_error(&cuda_line);
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                Ticket &t = tickets[id];
                t.status = rc;
                t.state = T_DONE;
                t.t_done = clock_type::now();
                inflight -= t.bytes;
                --running;
                ++completed;
                if (rc != PSDPROJ_OK) {
                    ++failed;
                    last_status = rc;
                    last_cuda = cuda_err;
                    last_line = cuda_line;
                }
                admit();
            }
            cv_done.notify_all();
        }
    }
};

extern "C" {

int psdproj_server_create(psdproj_server **out, int device, int workers, size_t admit_bytes,
                          const psdproj_opts *opts)
{
    if (!out || workers < 1 || workers > 64 || admit_bytes == 0) return PSDPROJ_EINVAL;
    *out = nullptr;
    psdproj_server *s = new (std::nothrow) psdproj_server();
    if (!s) return PSDPROJ_ENOMEM;
    s->device = device;
    s->admit_bytes = admit_bytes;
    if (opts) s->opts = *opts; else psdproj_default_opts(&s->opts);
    if (s->opts.prec < PSDPROJ_PREC_FP32 || s->opts.prec > PSDPROJ_PREC_BF16X3 ||
        (s->opts.syrk_prec != PSDPROJ_PREC_FP32 && s->opts.syrk_prec != PSDPROJ_PREC_BF16X3) ||
        s->opts.out_mode < PSDPROJ_OUT_FULL || s->opts.out_mode > PSDPROJ_OUT_FACTOR) {
        delete s;
        return PSDPROJ_EINVAL;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        delete s;
        return PSDPROJ_EINVAL;
    }
    int rc = PSDPROJ_OK;
    for (int w = 0; w < workers && rc == PSDPROJ_OK; ++w) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { rc = PSDPROJ_ECUDA; break; }
        s->streams.push_back(st);
        if (cudaEventCreateWithFlags(&ev, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess) {
            rc = PSDPROJ_ECUDA;
            break;
        }
        s->done_ev.push_back(ev);
        psdproj_ctx *c = nullptr;
        rc = psdproj_create(&c, device, st, 0);
        if (rc == PSDPROJ_OK) s->ctx.push_back(c);
    }
    if (rc != PSDPROJ_OK) {
        psdproj_server_destroy(s);
        return rc;
    }
    for (int w = 0; w < workers; ++w) s->workers.emplace_back([s, w] { s->worker(w); });
    *out = s;
    return PSDPROJ_OK;
}

int psdproj_server_submit(psdproj_server *s, const psdproj_request *req, uint64_t *ticket)
{
    if (!s || !req || !ticket) return PSDPROJ_EINVAL;
    *ticket = 0;
    const int rc = check_request(*req, s->opts.out_mode);
    if (rc != PSDPROJ_OK) return rc;
    const size_t bytes = req->footprint_bytes > 0 ? (size_t)req->footprint_bytes : default_footprint(*req, s->opts);
    if (bytes > s->admit_bytes) return PSDPROJ_ETOOLARGE;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return PSDPROJ_EINVAL;
    const uint64_t id = s->next_ticket++;
    Ticket &t = s->tickets[id];
    t.req = *req;
    t.bytes = bytes;
    t.t_submit = clock_type::now();
    s->pending.push_back(id);
    ++s->submitted;
    s->admit();
    *ticket = id;
    return PSDPROJ_OK;
}

int psdproj_server_wait(psdproj_server *s, uint64_t ticket, double timeout_s, int *status, double *latency_ms)
{
    if (!s) return PSDPROJ_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = clock_type::now() + std::chrono::duration_cast<clock_type::duration>(
                                                  std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
    for (;;) {
        auto it = s->tickets.find(ticket);
        if (it == s->tickets.end()) return PSDPROJ_EINVAL;   // unknown, or already collected
        if (it->second.state == T_DONE) {
            if (status) *status = it->second.status;
            if (latency_ms)
                *latency_ms = std::chrono::duration<double, std::milli>(it->second.t_done - it->second.t_submit).count();
            s->tickets.erase(it);
            return PSDPROJ_OK;
        }
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto jt = s->tickets.find(ticket);
            if (jt == s->tickets.end()) return PSDPROJ_EINVAL;
            if (jt->second.state != T_DONE) return PSDPROJ_ETIMEOUT;
        }
    }
}

int psdproj_server_drain(psdproj_server *s, double timeout_s)
{
    if (!s) return PSDPROJ_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = clock_type::now() + std::chrono::duration_cast<clock_type::duration>(
                                                  std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
    while (!s->pending.empty() || !s->ready.empty() || s->running > 0) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
            (!s->pending.empty() || !s->ready.empty() || s->running > 0))
            return PSDPROJ_ETIMEOUT;
    }
    return PSDPROJ_OK;
}

int psdproj_server_get_stats(psdproj_server *s, psdproj_server_stats *out)
{
    if (!s || !out) return PSDPROJ_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->queued = (int64_t)s->pending.size();
    out->running = (int64_t)s->ready.size() + s->running;
    out->inflight_bytes = (int64_t)s->inflight;
    out->inflight_peak_bytes = (int64_t)s->inflight_peak;
    out->admit_bytes = (int64_t)s->admit_bytes;
    out->last_error_status = s->last_status;
    out->last_error_cuda = s->last_cuda;
    out->last_error_line = s->last_line;
    return PSDPROJ_OK;
}

int psdproj_server_destroy(psdproj_server *s)
{
    if (!s) return PSDPROJ_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // requests never admitted are dropped; admitted ones still run
        for (uint64_t id : s->pending) s->tickets.erase(id);
        s->pending.clear();
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers)
        if (t.joinable()) t.join();
    cudaSetDevice(s->device);
    for (psdproj_ctx *c : s->ctx) psdproj_destroy(c);
    for (cudaEvent_t e : s->done_ev) cudaEventDestroy(e);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
    return PSDPROJ_OK;
}

}  // extern "C"
