// dope_server.cu -- request server: continuous batching of DOPE solves on one
// GPU (declared in include/dope.h).  Host code only; the GPU work is the
// batched persistent launch of dope.cu (all admitted requests' blocks in one
// cooperative kernel, each request on its own Algorithm 1).
//
// Life of a request (worker thread):
//   queued   -> admitted when its device state fits in the arena and fewer
//               than max_batch requests are admitted; context, tables and
//               input upload are issued on the set-up stream
//   set-up   -> the running launch is asked to yield (host-mapped flag read
//               at an iteration boundary) once the input copies are done;
//               the set-up kernels then run between two launches
//   running  -> part of every launch until its stop test holds or it reaches
//               max_iter (a launch also ends when any request finishes)
//   finish   -> labels and energy written (finish kernels on the compute
//               stream, label copy to the host on the copy stream)
//   done     -> result published, device memory back to the arena
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "dope.h"
#include "dope_internal.h"

namespace {

// First-fit allocator over one device allocation (worker thread only).
class Arena {
public:
    int init(size_t bytes) {
        bytes &= ~(size_t)255;
        if (bytes < 4096) return DOPE_EINVAL;
        if (cudaMalloc(&base_, bytes) != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return DOPE_ENOMEM;
        }
        size_ = bytes;
        free_[0] = bytes;
        return DOPE_OK;
    }
    void shutdown() {
        if (base_) cudaFree(base_);
        base_ = nullptr;
        free_.clear();
        used_.clear();
    }
    void* alloc(size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        if (!bytes) bytes = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, len = it->second;
            free_.erase(it);
            if (len > bytes) free_[off + bytes] = len - bytes;
            used_[off] = bytes;
            in_use_ += bytes;
            if (in_use_ > peak_) peak_ = in_use_;
            return base_ + off;
        }
        return nullptr;
    }
    void release(void* p) {
        if (!p) return;
        const size_t off = (size_t)(static_cast<char*>(p) - base_);
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t len = u->second, start = off;
        used_.erase(u);
        in_use_ -= len;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + len == nx->first) {
            len += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                start = pv->first;
                len += pv->second;
                free_.erase(pv);
            }
        }
        free_[start] = len;
    }
    size_t size() const { return size_; }
    size_t in_use() const { return in_use_; }
    size_t peak() const { return peak_; }
    static void* s_alloc(void* self, size_t b) { return static_cast<Arena*>(self)->alloc(b); }
    static void s_release(void* self, void* p) { static_cast<Arena*>(self)->release(p); }

private:
    char* base_ = nullptr;
    size_t size_ = 0, in_use_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;   // offset -> length
    std::map<size_t, size_t> used_;
};

enum JobState { J_QUEUED, J_SETUP, J_READY, J_RUNNING, J_FINISH };

struct Slot {              // pinned, one per admitted request
    int64_t energy;
    int status;
    int pad;
};

struct Job {
    uint64_t id = 0;
    dope_request r{};
    dope_image_request img{};   // the request's image source, when r.image_request is set
    double t_submit = 0, t_admit = 0;
    JobState state = J_QUEUED;
    bool cancel = false;        // dope_server_cancel: drop at the next safe point
    dope_ctx* ctx = nullptr;
    uint8_t* lab_dev = nullptr;
    bool own_lab = false;
    int slot = -1;
    cudaEvent_t ev_copied = nullptr, ev_setup = nullptr, ev_fin = nullptr, ev_done = nullptr;
    int status = 0, iters = 0, conv = 0;
};

constexpr int NSLOTS = 2 * DOPE_BATCH_MAX + 64;

}  // namespace

struct dope_server {
    dope_server_params p{};
    int dev = 0;
    Arena arena;
    dope_allocator al{};
    std::map<long long, dope_tables*> tables;
    cudaStream_t s_comp = nullptr, s_setup = nullptr, s_copy = nullptr;
    int* yield_h = nullptr;
    int* yield_d = nullptr;
    Slot* slots = nullptr;
    std::vector<int> free_slots;
    std::vector<cudaEvent_t> ev_pool;
    cudaEvent_t ev_l0 = nullptr, ev_l1 = nullptr;
    dope_batch_ws* ws = nullptr;
    std::chrono::steady_clock::time_point t0;
    // shared with the caller's threads
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job*> submitted;
    std::deque<dope_result> results;
    std::vector<uint64_t> cancels;   // ids to cancel, taken by the worker
    bool stop = false;
    uint64_t next_id = 1;
    std::atomic<int64_t> n_submitted{0}, n_admitted{0}, n_completed{0}, n_launches{0}, n_yields{0};
    std::atomic<int64_t> n_queued{0}, n_in_flight{0}, max_in_flight{0};
    std::atomic<uint64_t> bytes_in_use{0}, bytes_peak{0};
    std::atomic<double> gpu_launch_s{0.0};
    std::thread worker;
    // worker only
    std::deque<Job*> queue;
    std::vector<Job*> setup, ready, running, finishing, launched;
    bool in_launch = false;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    cudaEvent_t get_event() {
        if (!ev_pool.empty()) {
            cudaEvent_t e = ev_pool.back();
            ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return e;
    }
    void put_event(cudaEvent_t& e) {
        if (e) ev_pool.push_back(e);
        e = nullptr;
    }
    int admitted_count() const { return (int)(setup.size() + ready.size() + running.size()); }
    void update_gauges() {
        n_queued = (int64_t)queue.size();
        const int64_t f = admitted_count();
        n_in_flight = f;
        if (f > max_in_flight) max_in_flight = f;
        bytes_in_use = arena.in_use();
        bytes_peak = arena.peak();
    }
};

namespace {

bool request_ok(const dope_request* r) {
    if (!r || (r->ndim != 2 && r->ndim != 3)) return false;
    if (r->ndim == 2 && r->connectivity != 4 && r->connectivity != 8) return false;
    if (r->ndim == 3 && r->connectivity != 6) return false;
    if (!r->labels) return false;
    if (r->image_request) {
        const dope_image_request* q = static_cast<const dope_image_request*>(r->image_request);
        if (!q->image || q->channels < 1 || q->channels > DOPE_GMM_MAX_CH || !(q->clip > 0.0) ||
            !std::isfinite(q->sigma))
            return false;
    } else if (!r->unaries || !r->weights) {
        return false;
    }
    if ((r->where_inputs != DOPE_HOST && r->where_inputs != DOPE_DEVICE) ||
        (r->where_labels != DOPE_HOST && r->where_labels != DOPE_DEVICE))
        return false;
    if (!(r->lambda >= 0.0) || !std::isfinite(r->lambda)) return false;
    long long n = 1, b = 1;
    for (int i = 0; i < r->ndim; ++i) {
        if (r->grid[i] <= 0 || r->block_shape[i] <= 0 || r->grid[i] > (1LL << 30)) return false;
        n *= r->grid[i];
        b *= r->block_shape[i];
        if (n >= (1LL << 31)) return false;
    }
    return b <= 4096;
}

void publish(dope_server* s, Job* j, int status, int64_t energy) {
    dope_result res{};
    res.id = j->id;
    res.tag = j->r.tag;
    res.status = status;
    res.iterations = j->iters;
    res.converged = j->conv;
    res.energy_int = energy;
    res.t_submit = j->t_submit;
    res.t_admit = j->t_admit;
    res.t_done = s->now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->results.push_back(res);
    }
    s->n_completed++;
    s->cv_done.notify_all();
}

// Give back everything a job holds (its GPU work has drained).
void release_job(dope_server* s, Job* j) {
    if (j->ctx) dope_destroy(j->ctx);
    j->ctx = nullptr;
    if (j->own_lab && j->lab_dev) s->arena.release(j->lab_dev);
    j->lab_dev = nullptr;
    if (j->slot >= 0) s->free_slots.push_back(j->slot);
    j->slot = -1;
    s->put_event(j->ev_copied);
    s->put_event(j->ev_setup);
    s->put_event(j->ev_fin);
    s->put_event(j->ev_done);
    delete j;
}

void fail_job(dope_server* s, Job* j, int status) {
    publish(s, j, status, 0);
    release_job(s, j);
}

dope_tables* tables_for(dope_server* s, int conn, const int32_t blk[3], int* rc) {
    const long long key = ((long long)conn << 48) | ((long long)blk[0] << 32) | ((long long)blk[1] << 16) | blk[2];
    auto it = s->tables.find(key);
    if (it != s->tables.end()) return it->second;
    dope_tables* t = nullptr;
    *rc = dope_tables_create(conn, blk, &s->al, s->s_setup, &t);
    if (*rc) return nullptr;
    s->tables[key] = t;
    return t;
}

// Admit queued requests (first come, first served) while memory and slots last.
void admit(dope_server* s) {
    // mode 2: batch only as wide as the backlog (at least 2): near first come,
    // first served while the server keeps up, full batching when it does not
    int limit = s->p.max_batch;
    if (s->p.mode == 2) limit = std::min(limit, std::max(2, (int)s->queue.size()));
    while (!s->queue.empty() && s->admitted_count() < limit && !s->free_slots.empty()) {
        Job* j = s->queue.front();
        const dope_request& r = j->r;
        int32_t blk3[3] = {1, 1, 1};
        for (int i = 0; i < r.ndim; ++i) blk3[3 - r.ndim + i] = r.block_shape[i];
        int rc = DOPE_OK;
        dope_tables* tab = tables_for(s, r.connectivity, blk3, &rc);
        bool nomem = false;
        if (!tab) {
            if (rc != DOPE_ENOMEM) { s->queue.pop_front(); fail_job(s, j, rc); continue; }
            nomem = true;
        }
        dope_ctx* ctx = nullptr;
        if (!nomem) {
            rc = dope_create_ex(r.grid, r.ndim, r.connectivity, r.block_shape, r.lambda,
                                r.use_params ? &r.params : nullptr, 1, &s->al, tab, s->s_setup, &ctx);
            if (rc == DOPE_ENOMEM) nomem = true;
            else if (rc) { s->queue.pop_front(); fail_job(s, j, rc); continue; }
        }
        uint8_t* lab = nullptr;
        if (!nomem) {
            if (r.where_labels == DOPE_DEVICE) {
                lab = r.labels;
            } else {
                lab = static_cast<uint8_t*>(s->arena.alloc((size_t)dope_ctx_pixels(ctx)));
                if (!lab) nomem = true;
            }
        }
        if (!nomem) {
            j->ev_copied = s->get_event();
            j->ev_setup = s->get_event();
            rc = r.image_request
                     ? dope_image_upload_async(ctx, &j->img, r.where_inputs, s->s_setup, j->ev_copied)
                     : dope_upload_async(ctx, r.unaries, r.weights, r.where_inputs, s->s_setup, j->ev_copied);
            if (rc == DOPE_ENOMEM) nomem = true;
            else if (rc) {
                s->queue.pop_front();
                cudaStreamSynchronize(s->s_setup);
                dope_destroy(ctx);
                if (r.where_labels != DOPE_DEVICE) s->arena.release(lab);
                fail_job(s, j, rc);
                continue;
            }
        }
        if (nomem) {
            // undo; the request waits for memory unless nothing else holds any
            if (ctx || lab) cudaStreamSynchronize(s->s_setup);
            if (ctx) dope_destroy(ctx);
            if (lab && r.where_labels != DOPE_DEVICE) s->arena.release(lab);
            s->put_event(j->ev_copied);
            s->put_event(j->ev_setup);
            if (s->admitted_count() == 0 && s->finishing.empty()) {
                s->queue.pop_front();
                fail_job(s, j, DOPE_ENOMEM);
                continue;
            }
            break;
        }
        j->slot = s->free_slots.back();
        s->free_slots.pop_back();
        Slot* sl = &s->slots[j->slot];
        sl->status = 0;
        sl->energy = 0;
        dope_status_async(ctx, &sl->status, s->s_setup);
        cudaEventRecord(j->ev_setup, s->s_setup);
        j->ctx = ctx;
        j->lab_dev = lab;
        j->own_lab = (r.where_labels != DOPE_DEVICE);
        j->t_admit = s->now();
        j->state = J_SETUP;
        s->queue.pop_front();
        s->setup.push_back(j);
        s->n_admitted++;
    }
}

// Set-up done -> ready (or failed).  wait: also wait for set-ups whose input
// copies are done (their remaining work is a few short kernels).
void promote(dope_server* s, bool wait) {
    std::vector<Job*> keep;
    for (Job* j : s->setup) {
        bool done = cudaEventQuery(j->ev_setup) == cudaSuccess;
        if (!done && wait && cudaEventQuery(j->ev_copied) == cudaSuccess) {
            cudaEventSynchronize(j->ev_setup);
            done = true;
        }
        cudaGetLastError();
        if (!done) { keep.push_back(j); continue; }
        dope_release_staging(j->ctx);
        const int st = s->slots[j->slot].status;
        if (j->cancel) { fail_job(s, j, DOPE_ECANCELED); continue; }
        if (st) { fail_job(s, j, st); continue; }
        j->state = J_READY;
        s->ready.push_back(j);
    }
    s->setup.swap(keep);
}

// Labels and energy of a finished request; its result is published once the
// copies have landed.
void finish(dope_server* s, Job* j) {
    j->state = J_FINISH;
    j->ev_fin = s->get_event();
    if (j->status == DOPE_OK) {
        dope_finish_async(j->ctx, j->lab_dev, &s->slots[j->slot].energy, s->s_comp);
        cudaEventRecord(j->ev_fin, s->s_comp);
        if (j->r.where_labels == DOPE_HOST) {
            j->ev_done = s->get_event();
            cudaStreamWaitEvent(s->s_copy, j->ev_fin, 0);
            cudaMemcpyAsync(j->r.labels, j->lab_dev, (size_t)dope_ctx_pixels(j->ctx), cudaMemcpyDeviceToHost,
                            s->s_copy);
            cudaEventRecord(j->ev_done, s->s_copy);
        }
    } else {
        cudaEventRecord(j->ev_fin, s->s_comp);
    }
    s->finishing.push_back(j);
}

void retire(dope_server* s) {
    std::vector<Job*> keep;
    for (Job* j : s->finishing) {
        cudaEvent_t e = j->ev_done ? j->ev_done : j->ev_fin;
        if (cudaEventQuery(e) != cudaSuccess) {
            cudaGetLastError();
            keep.push_back(j);
            continue;
        }
        int status = j->status;
        if (status == DOPE_OK && !j->conv) status = DOPE_ENOTCONV;
        publish(s, j, status, s->slots[j->slot].energy);
        release_job(s, j);
    }
    s->finishing.swap(keep);
}

void start_launch(dope_server* s) {
    for (Job* j : s->ready) {
        j->state = J_RUNNING;
        s->running.push_back(j);
    }
    s->ready.clear();
    *(volatile int*)s->yield_h = 0;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    std::vector<dope_ctx*> cs;
    for (Job* j : s->running) cs.push_back(j->ctx);
    const int n_iter = s->p.launch_iters > 0 ? s->p.launch_iters : (1 << 30);
    cudaEventRecord(s->ev_l0, s->s_comp);
    int rc = dope_batch_launch(cs.data(), (int)cs.size(), n_iter, 1, 0, s->yield_d, s->ws, s->s_comp);
    cudaEventRecord(s->ev_l1, s->s_comp);
    if (rc) {
        cudaGetLastError();
        for (Job* j : s->running) {
            j->status = rc;
            finish(s, j);
        }
        s->running.clear();
        return;
    }
    s->launched = s->running;
    s->in_launch = true;
    s->n_launches++;
}

void end_launch(dope_server* s) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s->ev_l0, s->ev_l1) == cudaSuccess) s->gpu_launch_s = s->gpu_launch_s + ms * 1e-3;
    cudaGetLastError();
    const int n = (int)s->launched.size();
    std::vector<dope_ctx*> cs;
    for (Job* j : s->launched) cs.push_back(j->ctx);
    std::vector<int> t((size_t)n), conv((size_t)n), st((size_t)n);
    const int rc = dope_batch_collect(cs.data(), n, s->ws, t.data(), conv.data(), st.data());
    std::vector<Job*> keep;
    for (int i = 0; i < n; ++i) {
        Job* j = s->launched[(size_t)i];
        j->iters = t[(size_t)i];
        j->conv = conv[(size_t)i];
        j->status = rc ? rc : st[(size_t)i];
        if (j->cancel && !j->status && !j->conv && j->iters < dope_ctx_max_iter(j->ctx)) j->status = DOPE_ECANCELED;
        if (j->status || j->conv || j->iters >= dope_ctx_max_iter(j->ctx)) finish(s, j);
        else keep.push_back(j);
    }
    s->running.swap(keep);
    s->launched.clear();
    s->in_launch = false;
}

// One request through the single-problem path (mode 1).
void run_one(dope_server* s) {
    Job* j = s->ready.front();
    s->ready.erase(s->ready.begin());
    j->state = J_RUNNING;
    cudaEventRecord(s->ev_l0, s->s_comp);
    int t = 0, conv = 0;
    const int rc = dope_run_single(j->ctx, s->s_comp, &t, &conv);
    cudaEventRecord(s->ev_l1, s->s_comp);
    cudaEventSynchronize(s->ev_l1);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s->ev_l0, s->ev_l1) == cudaSuccess) s->gpu_launch_s = s->gpu_launch_s + ms * 1e-3;
    cudaGetLastError();
    s->n_launches++;
    j->iters = t;
    j->conv = conv;
    j->status = rc;
    finish(s, j);
}

// Requests cancelled since the last pass: queued and ready ones go at once,
// set-ups once their work has drained (promote), running ones at the end of
// the launch, which is asked to yield (end_launch); finishing ones keep their
// result.
void apply_cancels(dope_server* s, const std::vector<uint64_t>& ids) {
    for (uint64_t id : ids) {
        bool found = false;
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
            if ((*it)->id == id) {
                Job* j = *it;
                s->queue.erase(it);
                fail_job(s, j, DOPE_ECANCELED);
                found = true;
                break;
            }
        if (found) continue;
        for (auto it = s->ready.begin(); it != s->ready.end(); ++it)
            if ((*it)->id == id) {
                Job* j = *it;
                s->ready.erase(it);
                fail_job(s, j, DOPE_ECANCELED);
                found = true;
                break;
            }
        if (found) continue;
        for (Job* j : s->setup)
            if (j->id == id) { j->cancel = true; found = true; }
        if (found) continue;
        for (auto it = s->running.begin(); it != s->running.end(); ++it)
            if ((*it)->id == id) {
                Job* j = *it;
                j->cancel = true;
                if (s->in_launch) {
                    if (!*(volatile int*)s->yield_h) {
                        *(volatile int*)s->yield_h = 1;
                        s->n_yields++;
                    }
                } else {            // between launches: finish it now
                    s->running.erase(it);
                    j->status = DOPE_ECANCELED;
                    finish(s, j);
                }
                break;
            }
    }
}

void worker_main(dope_server* s) {
    cudaSetDevice(s->dev);
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->stop) break;
            while (!s->submitted.empty()) {
                s->queue.push_back(s->submitted.front());
                s->submitted.pop_front();
            }
        }
        std::vector<uint64_t> cancel_now;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            cancel_now.swap(s->cancels);
        }
        if (!cancel_now.empty()) apply_cancels(s, cancel_now);
        admit(s);
        promote(s, false);
        retire(s);
        if (s->in_launch) {
            if (cudaEventQuery(s->ev_l1) == cudaSuccess) {
                end_launch(s);
                promote(s, true);
            } else {
                cudaGetLastError();
                bool want = !s->ready.empty();
                for (Job* j : s->setup)
                    if (cudaEventQuery(j->ev_copied) == cudaSuccess) want = true;
                cudaGetLastError();
                if (want && !*(volatile int*)s->yield_h) {
                    *(volatile int*)s->yield_h = 1;
                    s->n_yields++;
                }
            }
        }
        bool busy = s->in_launch;
        if (!s->in_launch) {
            if (s->p.mode != 1 && (!s->running.empty() || !s->ready.empty())) {
                start_launch(s);
                busy = true;
            } else if (s->p.mode == 1 && !s->ready.empty()) {
                run_one(s);
                busy = true;
            }
        }
        s->update_gauges();
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->stop) break;
        if (!s->submitted.empty()) continue;
        const bool pending = busy || !s->setup.empty() || !s->finishing.empty() || !s->ready.empty();
        s->cv_work.wait_for(lk, pending ? std::chrono::microseconds(20) : std::chrono::milliseconds(5));
    }
    // shut down: let the GPU drain, then give everything back
    cudaStreamSynchronize(s->s_comp);
    cudaStreamSynchronize(s->s_setup);
    cudaStreamSynchronize(s->s_copy);
    cudaGetLastError();
    if (s->in_launch) {            // give the launch's constant table back
        std::vector<dope_ctx*> cs;
        for (Job* j : s->launched) cs.push_back(j->ctx);
        dope_batch_collect(cs.data(), (int)cs.size(), s->ws, nullptr, nullptr, nullptr);
        s->in_launch = false;
        s->launched.clear();
    }
    std::vector<Job*> all;
    for (Job* j : s->queue) all.push_back(j);
    for (auto* v : {&s->setup, &s->ready, &s->running, &s->finishing})
        for (Job* j : *v) all.push_back(j);
    s->queue.clear();
    s->setup.clear(); s->ready.clear(); s->running.clear(); s->finishing.clear();
    for (Job* j : all) release_job(s, j);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (Job* j : s->submitted) delete j;
        s->submitted.clear();
    }
}

}  // namespace

extern "C" {

int dope_server_create(const dope_server_params* p, dope_server** out) {
    if (!out) return DOPE_EINVAL;
    *out = nullptr;
    dope_server_params prm{};
    if (p) prm = *p;
    if (prm.max_batch <= 0 || prm.max_batch > DOPE_BATCH_MAX) prm.max_batch = DOPE_BATCH_MAX;
    if (prm.mode < 0 || prm.mode > 2) return DOPE_EINVAL;
    if (prm.launch_iters < 0) return DOPE_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return DOPE_ECUDA;
    }
    dope_server* s = new (std::nothrow) dope_server();
    if (!s) return DOPE_ENOMEM;
    s->p = prm;
    cudaGetDevice(&s->dev);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return DOPE_ECUDA;
    }
    size_t bytes = prm.hbm_bytes ? (size_t)prm.hbm_bytes : fr / 4 * 3;
    int rc = s->arena.init(bytes);
    if (rc) { delete s; return rc; }
    s->p.hbm_bytes = s->arena.size();
    s->al.self = &s->arena;
    s->al.alloc = Arena::s_alloc;
    s->al.release = Arena::s_release;
    bool ok = cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->s_setup, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking) == cudaSuccess &&
              cudaHostAlloc(&s->yield_h, sizeof(int), cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer((void**)&s->yield_d, s->yield_h, 0) == cudaSuccess &&
              cudaMallocHost(&s->slots, sizeof(Slot) * NSLOTS) == cudaSuccess &&
              cudaEventCreate(&s->ev_l0) == cudaSuccess && cudaEventCreate(&s->ev_l1) == cudaSuccess;
    if (ok) ok = dope_batch_ws_create(&s->ws) == DOPE_OK;
    if (!ok) {
        cudaGetLastError();
        dope_server_destroy(s);
        return DOPE_ECUDA;
    }
    *s->yield_h = 0;
    for (int i = NSLOTS - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->t0 = std::chrono::steady_clock::now();
    s->worker = std::thread(worker_main, s);
    *out = s;
    return DOPE_OK;
}

int dope_server_submit(dope_server* s, const dope_request* r, uint64_t* id) {
    if (!s || !request_ok(r)) return DOPE_EINVAL;
    Job* j = new (std::nothrow) Job();
    if (!j) return DOPE_ENOMEM;
    j->r = *r;
    if (r->image_request) {
        j->img = *static_cast<const dope_image_request*>(r->image_request);
        j->r.image_request = &j->img;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) { delete j; return DOPE_EINVAL; }
        j->id = s->next_id++;
        j->t_submit = s->now();
        s->submitted.push_back(j);
    }
    s->n_submitted++;
    s->cv_work.notify_one();
    if (id) *id = j->id;
    return DOPE_OK;
}

int dope_server_cancel(dope_server* s, uint64_t id) {
    if (!s) return DOPE_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (id == 0 || id >= s->next_id) return DOPE_EINVAL;
        s->cancels.push_back(id);
    }
    s->cv_work.notify_one();
    return DOPE_OK;
}

int dope_server_poll(dope_server* s, dope_result* out, int cap, int* count, double timeout_s) {
    if (!s || !count || cap < 0 || (cap > 0 && !out)) return DOPE_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->results.empty() && timeout_s > 0)
        s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [s] { return !s->results.empty(); });
    int n = 0;
    while (n < cap && !s->results.empty()) {
        out[n++] = s->results.front();
        s->results.pop_front();
    }
    *count = n;
    return DOPE_OK;
}

double dope_server_clock(const dope_server* s) { return s ? s->now() : 0.0; }

int dope_server_get_stats(dope_server* s, dope_server_stats* st) {
    if (!s || !st) return DOPE_EINVAL;
    memset(st, 0, sizeof(*st));
    st->submitted = s->n_submitted;
    st->admitted = s->n_admitted;
    st->completed = s->n_completed;
    st->launches = s->n_launches;
    st->yields = s->n_yields;
    st->queued = s->n_queued;
    st->in_flight = s->n_in_flight;
    st->max_in_flight = s->max_in_flight;
    st->bytes_limit = s->p.hbm_bytes;
    st->bytes_in_use = s->bytes_in_use;
    st->bytes_peak = s->bytes_peak;
    st->gpu_launch_s = s->gpu_launch_s;
    return DOPE_OK;
}

void dope_server_destroy(dope_server* s) {
    if (!s) return;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    for (auto& kv : s->tables) dope_tables_destroy(kv.second);
    s->tables.clear();
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    s->ev_pool.clear();
    if (s->ev_l0) cudaEventDestroy(s->ev_l0);
    if (s->ev_l1) cudaEventDestroy(s->ev_l1);
    if (s->ws) dope_batch_ws_destroy(s->ws);
    if (s->slots) cudaFreeHost(s->slots);
    if (s->yield_h) cudaFreeHost(s->yield_h);
    if (s->s_comp) cudaStreamDestroy(s->s_comp);
    if (s->s_setup) cudaStreamDestroy(s->s_setup);
    if (s->s_copy) cudaStreamDestroy(s->s_copy);
    s->arena.shutdown();
    delete s;
}

}  // extern "C"
