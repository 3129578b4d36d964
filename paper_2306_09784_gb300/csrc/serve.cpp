// Served form: continuous batching of imaging requests from several radars.
//
// One worker thread per server owns three CUDA streams:
//  * copy stream: host -> device copies of each admitted request (beat cube,
//    w_sar, trajectory) and the device -> host copy of finished images;
//  * range-compression stream: range compression of newly admitted requests,
//    overlapping the backprojection rounds already running;
//  * round stream: backprojection rounds.  A round is ONE batched launch over
//    the next sub-aperture chunk of every active request (chunk_pulses
//    chirps, or fewer when a work quantum per request and round is set),
//    accumulated into its device-resident image.  Requests that arrive while
//    a round runs join the next round; finished ones leave.
// Admission is bounded by slots (max_inflight) and by an HBM budget: one
// device pool allocated at creation and sub-allocated first-fit; a request
// waits in the queue until its buffers fit.  Each request's image equals its
// stand-alone backprojection up to FP32 summation order.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "sar_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// First-fit sub-allocator over one device allocation (host-side bookkeeping).
class Pool {
   public:
    bool init(size_t bytes) {
        size_ = align256(bytes);
        if (cudaMalloc((void **)&base_, size_) != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return false;
        }
        free_[0] = size_;
        return true;
    }
    void destroy() {
        if (base_) cudaFree(base_);
        base_ = nullptr;
    }
    size_t size() const { return size_; }
    char *alloc(size_t bytes) {
        bytes = align256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, sz = it->second;
                free_.erase(it);
                if (sz > bytes) free_[off + bytes] = sz - bytes;
                return base_ + off;
            }
        }
        return nullptr;
    }
    void release(char *p, size_t bytes) {
        if (!p) return;
        bytes = align256(bytes);
        size_t off = (size_t)(p - base_);
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                off = prev->first;
                bytes += prev->second;
                free_.erase(prev);
            }
        }
        free_[off] = bytes;
    }

   private:
    char *base_ = nullptr;
    size_t size_ = 0;
    std::map<size_t, size_t> free_;
};

struct Request {
    uint64_t ticket = 0;
    sar_request r{};
    Clock::time_point t_submit;
    std::atomic<int> state{SAR_REQ_QUEUED};
    std::atomic<bool> cancel{false};
    // geometry
    int n_rx = 0, n_samples = 0, n_bins = 0, fp16 = 0, max_pulses = 0;
    int64_t n_pixels = 0;
    // device buffers (pool)
    char *d_beat = nullptr, *d_waz = nullptr, *d_qtx = nullptr, *d_qrx = nullptr, *d_prof = nullptr,
         *d_img = nullptr;
    size_t b_beat = 0, b_waz = 0, b_qtx = 0, b_qrx = 0, b_prof = 0, b_img = 0;
    int next_pulse = 0;
    bool joined = false;          // took part in a round (its range compression is ordered before)
    void *img_host_dev = nullptr;  // image_host as a device address, if page-locked and mapped
    bool finishing = false;       // final round enqueued
    cudaEvent_t rc_ev = nullptr;  // range compression done
    cudaEvent_t ev = nullptr;     // last GPU work of this request
    double latency_ms = 0;
    int status = SAR_OK;

    size_t total_bytes() const { return b_beat + b_waz + b_qtx + b_qrx + b_prof + b_img; }
};

}  // namespace

struct sar_server {
    sar_server_config cfg{};
    int device = 0;
    cudaStream_t copy_s = nullptr, rc_s = nullptr, round_s = nullptr;
    sar_batch *batch[2] = {nullptr, nullptr};
    cudaEvent_t round_ev[2] = {nullptr, nullptr};
    bool round_pending[2] = {false, false};
    int parity = 0;
    Pool pool;
    std::mutex mu;
    std::condition_variable cv;        // worker wake-up
    std::condition_variable done_cv;   // request completion
    std::deque<Request *> queue;
    std::map<uint64_t, Request *> reqs;
    std::vector<Request *> active;
    std::thread worker;
    std::atomic<bool> stop{false};
    uint64_t next_ticket = 1;
    int fatal = SAR_OK;
    // statistics
    uint64_t rounds = 0, completed = 0;
};

namespace {

void free_request_buffers(sar_server *s, Request *q, bool keep_image) {
    s->pool.release(q->d_beat, q->b_beat);
    s->pool.release(q->d_waz, q->b_waz);
    s->pool.release(q->d_qtx, q->b_qtx);
    s->pool.release(q->d_qrx, q->b_qrx);
    s->pool.release(q->d_prof, q->b_prof);
    q->d_beat = q->d_waz = q->d_qtx = q->d_qrx = q->d_prof = nullptr;
    if (!keep_image) {
        s->pool.release(q->d_img, q->b_img);
        q->d_img = nullptr;
    }
}

void destroy_request(sar_server *s, Request *q) {
    free_request_buffers(s, q, false);
    if (q->rc_ev) cudaEventDestroy(q->rc_ev);
    if (q->ev) cudaEventDestroy(q->ev);
    delete q;
}

// Allocates all device buffers of q from the pool; false (nothing kept) if
// they do not fit now.  Caller holds the lock.
bool try_allocate(sar_server *s, Request *q) {
    char *p[6] = {};
    const size_t b[6] = {q->b_beat, q->b_waz, q->b_qtx, q->b_qrx, q->b_prof, q->b_img};
    for (int i = 0; i < 6; ++i) {
        p[i] = s->pool.alloc(b[i]);
        if (!p[i]) {
            for (int k = 0; k < i; ++k) s->pool.release(p[k], b[k]);
            return false;
        }
    }
    q->d_beat = p[0];
    q->d_waz = p[1];
    q->d_qtx = p[2];
    q->d_qrx = p[3];
    q->d_prof = p[4];
    q->d_img = p[5];
    return true;
}

// Copies and range compression of a newly admitted request (worker thread).
int start_request(sar_server *s, Request *q) {
    const sar_request &r = q->r;
    const int M = r.M, R = q->n_rx, N = q->n_samples;
    if (cudaEventCreateWithFlags(&q->rc_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming) != cudaSuccess)
        return SAR_ECUDA;
    if (r.image_host) {
        // a page-locked, mapped destination is written by the final round's
        // kernels themselves (besides the device image), so the image does
        // not wait for a copy behind other requests' uploads
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, r.image_host) == cudaSuccess) {
            if (pa.type == cudaMemoryTypeHost && pa.devicePointer && (uintptr_t)pa.devicePointer % 8 == 0)
                q->img_host_dev = pa.devicePointer;
        } else {
            cudaGetLastError();
        }
    }
    bool ok = cudaMemcpyAsync(q->d_beat, r.beat_host, (size_t)M * R * N * 8, cudaMemcpyHostToDevice, s->copy_s) ==
              cudaSuccess;
    if (r.w_az_host)
        ok = ok && cudaMemcpyAsync(q->d_waz, r.w_az_host, (size_t)M * 4, cudaMemcpyHostToDevice, s->copy_s) ==
                       cudaSuccess;
    ok = ok && cudaMemcpyAsync(q->d_qtx, r.q_tx_host, (size_t)M * 16, cudaMemcpyHostToDevice, s->copy_s) ==
                   cudaSuccess;
    ok = ok && cudaMemcpyAsync(q->d_qrx, r.q_rx_host, (size_t)M * R * 16, cudaMemcpyHostToDevice, s->copy_s) ==
                   cudaSuccess;
    ok = ok && cudaEventRecord(q->ev, s->copy_s) == cudaSuccess;
    ok = ok && cudaStreamWaitEvent(s->rc_s, q->ev, 0) == cudaSuccess;
    if (!ok) return SAR_ECUDA;
    int rc = sar_range_compress(r.plan, q->d_beat, M, r.w_az_host ? (const float *)q->d_waz : nullptr, q->d_prof,
                                s->rc_s);
    if (rc) return rc;
    if (cudaEventRecord(q->rc_ev, s->rc_s) != cudaSuccess) return SAR_ECUDA;
    if (cudaEventRecord(q->ev, s->rc_s) != cudaSuccess) return SAR_ECUDA;
    return SAR_OK;
}

// One backprojection round over the next chunk of every active request.
// Returns true if a round was launched.
int launch_round(sar_server *s, std::vector<Request *> &work, bool *launched) {
    *launched = false;
    std::vector<Request *> part;
    for (Request *q : work) {
        if (q->state != SAR_REQ_RUNNING || q->cancel || q->next_pulse >= q->r.M) continue;
        if (!q->joined) {
            // a request joins once its upload and range compression are done,
            // so that a round never waits on copies still in flight (requests
            // admitted together would otherwise hold the first round until
            // the last upload finished)
            const cudaError_t e = cudaEventQuery(q->rc_ev);
            if (e == cudaErrorNotReady) continue;
            if (e != cudaSuccess) return SAR_ECUDA;
        }
        part.push_back(q);
    }
    if (part.empty()) return SAR_OK;
    const int k = s->parity;
    if (s->round_pending[k]) {  // at most two rounds in flight
        if (cudaEventSynchronize(s->round_ev[k]) != cudaSuccess) return SAR_ECUDA;
        s->round_pending[k] = false;
    }
    sar_batch *b = s->batch[k];
    int rc = sar_batch_clear(b);
    if (rc) return rc;
    const int chunk = s->cfg.chunk_pulses;
    const double quantum = 1e6 * (double)s->cfg.quantum_mupdates;
    for (Request *q : part) {
        if (!q->joined) {
            if (cudaStreamWaitEvent(s->round_s, q->rc_ev, 0) != cudaSuccess) return SAR_ECUDA;
            q->joined = true;
        }
        const int m0 = q->next_pulse;
        int cnt = std::min(chunk, q->r.M - m0);
        if (quantum > 0) {
            // at most about `quantum` pixel x chirp x Rx updates of this
            // request per round: a small frame completes in its first round,
            // a large one advances by a share and leaves room for newcomers
            const double per_chirp = (double)q->n_pixels * q->n_rx;
            cnt = (int)std::min<double>(cnt, std::max(1.0, std::ceil(quantum / per_chirp)));
        }
        const int R = q->n_rx;
        const size_t rows0 = (size_t)m0 * R;
        const char *samples;
        const float *scales = nullptr;
        if (q->fp16) {
            const size_t pad = align256((size_t)q->r.M * R * 4);
            scales = (const float *)q->d_prof + rows0;
            samples = q->d_prof + pad + rows0 * q->n_bins * 4;
        } else {
            samples = q->d_prof + rows0 * q->n_bins * 8;
        }
        const bool final_round = m0 + cnt == q->r.M;
        rc = sar::batch_add_rows(b, q->r.plan, samples, scales, cnt, (const double *)q->d_qtx + 2 * m0,
                                 (const double *)q->d_qrx + 2 * rows0, q->d_img, m0 > 0 ? 1 : 0,
                                 final_round ? q->img_host_dev : nullptr);
        if (rc) return rc;
        q->next_pulse = m0 + cnt;
    }
    rc = sar_batch_commit(b, s->round_s);
    if (!rc) rc = sar_batch_launch(b, s->round_s);
    if (rc) return rc;
    if (cudaEventRecord(s->round_ev[k], s->round_s) != cudaSuccess) return SAR_ECUDA;
    // each participant's buffers are in use until this round has finished
    for (Request *q : part)
        if (cudaEventRecord(q->ev, s->round_s) != cudaSuccess) return SAR_ECUDA;
    s->round_pending[k] = true;
    s->parity ^= 1;
    s->rounds += 1;
    for (Request *q : part) {
        if (q->next_pulse < q->r.M) continue;
        // final round of q: image back to the host (if wanted), then done
        q->finishing = true;
        if (q->r.image_host && !q->img_host_dev) {
            if (cudaStreamWaitEvent(s->copy_s, s->round_ev[k], 0) != cudaSuccess) return SAR_ECUDA;
            if (cudaMemcpyAsync(q->r.image_host, q->d_img, (size_t)q->n_pixels * 8, cudaMemcpyDeviceToHost,
                                s->copy_s) != cudaSuccess)
                return SAR_ECUDA;
            if (cudaEventRecord(q->ev, s->copy_s) != cudaSuccess) return SAR_ECUDA;
        } else {
            if (cudaEventRecord(q->ev, s->round_s) != cudaSuccess) return SAR_ECUDA;
        }
    }
    *launched = true;
    return SAR_OK;
}

void fail_all(sar_server *s, int status) {
    s->fatal = status;
    for (Request *q : s->active) {
        q->state = SAR_REQ_FAILED;
        q->status = status;
    }
    s->active.clear();
    for (Request *q : s->queue) {
        q->state = SAR_REQ_FAILED;
        q->status = status;
    }
    s->queue.clear();
    s->done_cv.notify_all();
}

void worker_main(sar_server *s) {
    if (cudaSetDevice(s->device) != cudaSuccess) {
        std::lock_guard<std::mutex> lk(s->mu);
        fail_all(s, SAR_ECUDA);
        return;
    }
    while (!s->stop.load()) {
        std::vector<Request *> admitted, work;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->fatal) {
                s->cv.wait_for(lk, std::chrono::milliseconds(10));
                continue;
            }
            // admission: slots and HBM budget, in arrival order
            while (!s->queue.empty() && (int)s->active.size() < s->cfg.max_inflight) {
                Request *q = s->queue.front();
                if (q->cancel) {  // released while queued
                    s->queue.pop_front();
                    continue;
                }
                if (!try_allocate(s, q)) break;
                s->queue.pop_front();
                q->state = SAR_REQ_RUNNING;  // from here on only the worker frees it
                s->active.push_back(q);
                admitted.push_back(q);
            }
            work = s->active;
        }
        int rc = SAR_OK;
        for (Request *q : admitted) {
            rc = start_request(s, q);
            if (rc) break;
        }
        bool launched = false;
        if (!rc) rc = launch_round(s, work, &launched);
        if (rc) {
            std::lock_guard<std::mutex> lk(s->mu);
            fail_all(s, rc);
            continue;
        }
        // completions and cancellations
        {
            std::unique_lock<std::mutex> lk(s->mu);
            const auto now = Clock::now();
            bool any = false;
            for (size_t i = 0; i < s->active.size();) {
                Request *q = s->active[i];
                const bool idle_cancel = q->cancel && !q->finishing;
                if ((q->finishing || idle_cancel) && cudaEventQuery(q->ev) == cudaSuccess) {
                    if (q->cancel) {
                        s->reqs.erase(q->ticket);
                        s->active.erase(s->active.begin() + i);
                        destroy_request(s, q);
                        continue;
                    }
                    q->latency_ms = std::chrono::duration<double, std::milli>(now - q->t_submit).count();
                    q->state = SAR_REQ_DONE;
                    free_request_buffers(s, q, true);
                    s->active.erase(s->active.begin() + i);
                    s->completed += 1;
                    any = true;
                    continue;
                }
                ++i;
            }
            if (any) s->done_cv.notify_all();
            if (!launched && admitted.empty()) {
                // nothing new to launch: wait for a submission or GPU progress.
                // While requests are in flight, poll at a short interval so
                // that a range compression finishing (a request ready to join)
                // or a round completing is acted on within ~20 us.
                s->cv.wait_for(lk, std::chrono::microseconds(s->active.empty() ? 100 : 20));
            }
        }
    }
}

}  // namespace

extern "C" {

int sar_server_create(const sar_server_config *cfg, sar_server **out) {
    if (!cfg || !out) return SAR_EINVAL;
    *out = nullptr;
    if (cfg->hbm_budget_bytes < (1u << 20) || cfg->max_inflight < 1 || cfg->max_inflight > 4096 ||
        cfg->queue_capacity < 1 || cfg->chunk_pulses < 1 || cfg->quantum_mupdates < 0)
        return SAR_EINVAL;
    sar_server *s = new (std::nothrow) sar_server();
    if (!s) return SAR_ENOMEM;
    s->cfg = *cfg;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return SAR_ECUDA;
    }
    bool ok = cudaStreamCreateWithFlags(&s->copy_s, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->rc_s, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->round_s, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&s->round_ev[0], cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&s->round_ev[1], cudaEventDisableTiming) == cudaSuccess;
    if (ok) ok = sar_batch_create(cfg->max_inflight, &s->batch[0]) == SAR_OK &&
                 sar_batch_create(cfg->max_inflight, &s->batch[1]) == SAR_OK;
    if (ok) ok = s->pool.init(cfg->hbm_budget_bytes);
    if (!ok) {
        cudaGetLastError();
        sar_server_destroy(s);
        return SAR_ENOMEM;
    }
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        sar_server_destroy(s);
        return SAR_ENOMEM;
    }
    *out = s;
    return SAR_OK;
}

void sar_server_destroy(sar_server *s) {
    if (!s) return;
    s->stop.store(true);
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    int cur = -1;
    cudaGetDevice(&cur);
    cudaSetDevice(s->device);
    if (s->round_s) cudaStreamSynchronize(s->round_s);
    if (s->rc_s) cudaStreamSynchronize(s->rc_s);
    if (s->copy_s) cudaStreamSynchronize(s->copy_s);
    for (auto &kv : s->reqs) destroy_request(s, kv.second);
    s->reqs.clear();
    for (int k = 0; k < 2; ++k) {
        if (s->batch[k]) sar_batch_destroy(s->batch[k]);
        if (s->round_ev[k]) cudaEventDestroy(s->round_ev[k]);
    }
    if (s->copy_s) cudaStreamDestroy(s->copy_s);
    if (s->rc_s) cudaStreamDestroy(s->rc_s);
    if (s->round_s) cudaStreamDestroy(s->round_s);
    s->pool.destroy();
    if (cur >= 0) cudaSetDevice(cur);
    delete s;
}

int sar_submit(sar_server *s, const sar_request *req, uint64_t *ticket) {
    if (!s || !req || !ticket || !req->plan || !req->beat_host || !req->q_tx_host || !req->q_rx_host)
        return SAR_EINVAL;
    int n_rx, n_samples, n_bins, fp16, max_pulses;
    int64_t n_pixels;
    if (sar::plan_geometry(req->plan, &n_rx, &n_samples, &n_bins, &fp16, &n_pixels, &max_pulses) != SAR_OK)
        return SAR_EINVAL;
    if (req->M < 1 || req->M > max_pulses || sar::plan_device(req->plan) != s->device) return SAR_EINVAL;
    Request *q = new (std::nothrow) Request();
    if (!q) return SAR_ENOMEM;
    q->r = *req;
    q->n_rx = n_rx;
    q->n_samples = n_samples;
    q->n_bins = n_bins;
    q->fp16 = fp16;
    q->n_pixels = n_pixels;
    q->max_pulses = max_pulses;
    const size_t M = (size_t)req->M, R = (size_t)n_rx;
    q->b_beat = M * R * n_samples * 8;
    q->b_waz = M * 4;
    q->b_qtx = M * 16;
    q->b_qrx = M * R * 16;
    size_t pb = 0;
    sar_profile_bytes(req->plan, req->M, &pb);
    q->b_prof = pb;
    q->b_img = (size_t)n_pixels * 8;
    size_t need = 0;
    for (size_t b : {q->b_beat, q->b_waz, q->b_qtx, q->b_qrx, q->b_prof, q->b_img}) need += align256(b);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal) {
        delete q;
        return s->fatal;
    }
    if (need > s->pool.size()) {  // can never be admitted
        delete q;
        return SAR_ENOMEM;
    }
    if ((int)s->queue.size() >= s->cfg.queue_capacity) {
        delete q;
        return SAR_EAGAIN;
    }
    q->ticket = s->next_ticket++;
    q->t_submit = Clock::now();
    s->reqs[q->ticket] = q;
    s->queue.push_back(q);
    *ticket = q->ticket;
    s->cv.notify_all();
    return SAR_OK;
}

int sar_poll(sar_server *s, uint64_t ticket, int32_t *state, const void **image_dev, double *latency_ms) {
    if (!s) return SAR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return SAR_ENOTFOUND;
    Request *q = it->second;
    if (state) *state = q->state;
    if (image_dev) *image_dev = q->state == SAR_REQ_DONE ? q->d_img : nullptr;
    if (latency_ms) *latency_ms = q->state == SAR_REQ_DONE ? q->latency_ms : 0.0;
    if (q->state == SAR_REQ_FAILED) return q->status;
    return q->state == SAR_REQ_DONE ? SAR_OK : SAR_EAGAIN;
}

int sar_wait(sar_server *s, uint64_t ticket, double timeout_ms) {
    if (!s || !(timeout_ms >= 0)) return SAR_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = Clock::now() + std::chrono::microseconds((long long)(timeout_ms * 1000.0));
    for (;;) {
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return SAR_ENOTFOUND;
        if (it->second->state == SAR_REQ_DONE) return SAR_OK;
        if (it->second->state == SAR_REQ_FAILED) return it->second->status;
        if (s->done_cv.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto jt = s->reqs.find(ticket);
            if (jt != s->reqs.end() && jt->second->state == SAR_REQ_DONE) return SAR_OK;
            return SAR_ETIMEOUT;
        }
    }
}

int sar_release(sar_server *s, uint64_t ticket) {
    if (!s) return SAR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return SAR_ENOTFOUND;
    Request *q = it->second;
    if (q->state == SAR_REQ_QUEUED) {
        q->cancel = true;  // the worker drops it from the queue
        auto qi = std::find(s->queue.begin(), s->queue.end(), q);
        if (qi != s->queue.end()) s->queue.erase(qi);
        s->reqs.erase(it);
        delete q;
        return SAR_OK;
    }
    if (q->state == SAR_REQ_RUNNING) {
        q->cancel = true;  // freed by the worker once its GPU work has drained
        s->cv.notify_all();
        return SAR_OK;
    }
    // done or failed: its GPU work has completed
    s->reqs.erase(it);
    destroy_request(s, q);
    return SAR_OK;
}

int sar_server_get_stats(sar_server *s, sar_server_stats *st) {
    if (!s || !st) return SAR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    st->queued = (int32_t)s->queue.size();
    st->active = (int32_t)s->active.size();
    st->rounds = (int64_t)s->rounds;
    st->completed = (int64_t)s->completed;
    st->pool_bytes = s->pool.size();
    return SAR_OK;
}

}  // extern "C"
