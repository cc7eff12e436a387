// dope.cu -- C-ABI of the GB300 DOPE ADMM hot path (declared in include/dope.h).
//
// Algorithm 1 of Dolz, Ben Ayed, Desrosiers (arXiv 1704.03116) on one GPU:
// per iteration one launch of k_block_solve (all blocks' Eq. 8 min-cuts,
// "in parallel") followed by one launch of k_face_update (Eq. 10, Eq. 11 and
// the per-block stop quantity).  Iterations are issued in batches; every
// kernel checks the device-side stop flag first, so launches past
// convergence return at once and the host synchronises once per batch.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "dope.h"
#include "dope_internal.h"
#include "dope_kernels.cuh"
#include "dope_overlap.cuh"
#include "dope_nsm.cuh"
#include "dope_big.h"

using namespace dope;

struct dope_ctx {
    Geo g;
    int ndim, conn;
    double lambda;
    dope_allocator al{};          // device memory source (null alloc: cudaMalloc)
    dope_tables* own_tab = nullptr;   // tables built for this context (else shared)
    dope_params p;
    int threads, smem;
    int persist_grid = 0;     // CTAs of the persistent launch (0: not possible)
    int pthreads = 0;         // threads per CTA of the persistent launch (256-wide or 512-wide kernel)
    int resident = 0;         // 1: the resident persistent kernel (K CTAs, one block each)
    int resident_smem = 0;
    int resident_threads = 0;
    // device state
    int32_t* U = nullptr;
    int32_t* Wl = nullptr;
    uint8_t* yhat = nullptr;
    double* yF = nullptr;
    double* aF = nullptr;
    double* r2blk = nullptr;
    int16_t* faceIndex = nullptr;
    int16_t* faceLocal = nullptr;
    int* halo = nullptr;
    int16_t* hslot = nullptr;   // [conn][F] halo pixel index of (direction, face slot)
    int* hinfo = nullptr;       // [NH] halo_entry of each distinct halo pixel
    int NH = 0;
    int window_ok = 0;          // the resident kernel fits with its run-ahead window arrays
    // overlapping partition (grow != 0): image-order U / Wl / q / y, box-major a / yhat
    int ov = 0;
    OvArgs oa{};
    int nsm = 0;                // non-submodular: LSA-TR block solves (k_nsm_solve)
    int nsm_smem = 0;
    int ov_threads = 0, ov_smem = 0;
    Ctrl* ctrl = nullptr;
    size_t ctrl_bytes = 0;
    unsigned char* sched = nullptr;   // block worklists of the persistent / batched kernels (sched_bytes)
    unsigned long long* wslot = nullptr;   // run-ahead windows of the persistent kernel: [K][F] entry slots,
    unsigned long long* wtag = nullptr;    // [K] block tags,
    unsigned* wmask = nullptr;             // [K][CHUNK_WORDS] entry chunks,
    double* wst = nullptr;                 // [K][F][4] states after a window's last two iterations
    unsigned sched_epoch = 0;         // launches issued with them
    int sched_t = -1;                 // the lists are valid for iteration sched_t + 1 (-1: not valid)
    bool sched_launch = false;        // the launch in flight uses the lists
    Ctrl* hctrl = nullptr;      // pinned host copy of the whole control block (dope_solve's single read)
    // staging (lazily allocated)
    void* stage = nullptr;
    size_t stage_bytes = 0;
    void* stage2 = nullptr;
    size_t stage2_bytes = 0;
    // host state
    int have_u = 0, have_w = 0;
    bool pending = false;     // an asynchronous upload's status word not read yet
    long long spin_limit = 4000000000LL;   // grid-barrier wait bound in SM cycles (about 2 s)
    int begun = 0;            // dope_solve_begin: 1 launch issued, 2 solved synchronously
    bool begun_pend = false;  // the issued launch carries an upload's status word
    int sync_rc = 0, sync_iters = 0;
    int64_t sync_energy = 0;
    int t = 0;          // iterations done since reset
    double mu = 0.0;    // mu the next iteration uses
    dope_stats stats{};
    long long launches = 0;   // kernels launched since the last stats reset
    // profiling
    int profiling = 0;
    std::vector<cudaEvent_t> ev;   // 3 per iteration: before solve, between, after update
    dope_profile prof{};
};

int dope_sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    if (dev >= 0 && dev < 64) {
        const int v = cache[dev].load(std::memory_order_relaxed);
        if (v > 0) return v;
    }
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
        cudaGetLastError();
        return 1;
    }
    if (dev >= 0 && dev < 64) cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

namespace {

#define CK(x)                                  \
    do {                                       \
        cudaError_t _e = (x);                  \
        if (_e != cudaSuccess) return DOPE_ECUDA; \
    } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// CTAs for n elements: one per element group, at most 32 per SM (the
// kernels stride over the rest).
int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    const long long cap = 32LL * dope_sm_count();
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

void* dalloc(const dope_allocator& al, size_t bytes) {
    if (!bytes) bytes = 16;
    if (al.alloc) return al.alloc(al.self, bytes);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dfree(const dope_allocator& al, void* p) {
    if (!p) return;
    if (al.alloc) al.release(al.self, p);
    else cudaFree(p);
}

// Width of the persistent / batched solver CTA for a block of B nodes
// (threads: the context's solver width): the 256-wide kernel (3 CTAs per SM)
// up to 1024 nodes, else the 512-wide one (2 CTAs per SM).
int solver_width(int B, int threads) {
    if (threads <= 256) return threads;
    return B <= 1024 ? 256 : threads;
}

// The persistent kernel for a connectivity and CTA width; win: its form with
// run-ahead windows (launched after the plain form, see k_admm_persistent).
const void* persistent_fn(int conn, int nt, bool win = false) {
    if (win) {
        if (nt <= 256)
            return conn == 4 ? (const void*)k_admm_persistent<4, 256, true>
                 : conn == 8 ? (const void*)k_admm_persistent<8, 256, true> : (const void*)k_admm_persistent<6, 256, true>;
        return conn == 4 ? (const void*)k_admm_persistent<4, 512, true>
             : conn == 8 ? (const void*)k_admm_persistent<8, 512, true> : (const void*)k_admm_persistent<6, 512, true>;
    }
    if (nt <= 256)
        return conn == 4 ? (const void*)k_admm_persistent<4, 256, false>
             : conn == 8 ? (const void*)k_admm_persistent<8, 256, false> : (const void*)k_admm_persistent<6, 256, false>;
    return conn == 4 ? (const void*)k_admm_persistent<4, 512, false>
         : conn == 8 ? (const void*)k_admm_persistent<8, 512, false> : (const void*)k_admm_persistent<6, 512, false>;
}

const void* batch_fn(int nt) {
    return nt <= 256 ? (const void*)k_admm_batch<256> : (const void*)k_admm_batch<512>;
}

int ensure_stage(dope_ctx* c, size_t bytes, int which) {
    void** p = which ? &c->stage2 : &c->stage;
    size_t* sz = which ? &c->stage2_bytes : &c->stage_bytes;
    if (*sz >= bytes) return DOPE_OK;
    dfree(c->al, *p);
    *p = nullptr;
    *sz = 0;
    *p = dalloc(c->al, bytes);
    if (!*p) return DOPE_ENOMEM;
    *sz = bytes;
    return DOPE_OK;
}

// Read the control header (conv_t, status, stats) after synchronising.
int read_ctrl(dope_ctx* c, Ctrl* h, cudaStream_t st) {
    CK(cudaMemcpyAsync(h, c->ctrl, sizeof(Ctrl) - sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return DOPE_OK;
}

int clear_status(dope_ctx* c, cudaStream_t st) {
    CK(cudaMemsetAsync(c->ctrl, 0, sizeof(Ctrl) - sizeof(unsigned long long), st));
    return DOPE_OK;
}

// Settle an asynchronous upload (dope_set_inputs, dope_set_image without
// sigma_used): read the status word its quantisers wrote (one
// synchronisation).  An input error invalidates both inputs and is returned.
int settle_inputs(dope_ctx* c, cudaStream_t st) {
    if (!c->pending) return DOPE_OK;
    c->pending = false;
    Ctrl h{};
    int rc = read_ctrl(c, &h, st);
    if (rc) return rc;
    if (h.status) {
        c->have_u = c->have_w = 0;
        return h.status;
    }
    return DOPE_OK;
}

template <int CONN>
void launch_solve(dope_ctx* c, const SolveArgs& a, cudaStream_t st) {
    k_block_solve<CONN><<<c->g.K, c->threads, c->smem, st>>>(a);
}

void solve_launch(dope_ctx* c, const SolveArgs& a, cudaStream_t st) {
    c->launches++;
    if (c->nsm) {
        if (c->conn == 4) k_nsm_solve<4><<<c->g.K, c->threads, c->nsm_smem, st>>>(a, c->p.lsa_steps);
        else if (c->conn == 8) k_nsm_solve<8><<<c->g.K, c->threads, c->nsm_smem, st>>>(a, c->p.lsa_steps);
        else k_nsm_solve<6><<<c->g.K, c->threads, c->nsm_smem, st>>>(a, c->p.lsa_steps);
        return;
    }
    if (c->conn == 4) launch_solve<4>(c, a, st);
    else if (c->conn == 8) launch_solve<8>(c, a, st);
    else launch_solve<6>(c, a, st);
}

void update_launch(dope_ctx* c, const UpdArgs& a, cudaStream_t st) {
    c->launches++;
    const int threads = face_update_threads(c->g.F);
    if (c->conn == 4) k_face_update<4><<<c->g.K, threads, 0, st>>>(a);
    else if (c->conn == 8) k_face_update<8><<<c->g.K, threads, 0, st>>>(a);
    else k_face_update<6><<<c->g.K, threads, 0, st>>>(a);
}

// Iteration-dependent solver arguments: mu and the integer forced-test bound.
void set_mu(SolveArgs& a, double mu) {
    a.mu = mu;
    const double h = (1024.0 * mu) * 0.5;
    a.int_test = (h < 4503599627370496.0) ? 1 : 0;   // 2^52
    a.H = a.int_test ? (long long)std::floor(h) : 0;
}

SolveArgs solve_args(dope_ctx* c) {
    SolveArgs a;
    a.g = c->g;
    a.U = c->U;
    a.Wl = c->Wl;
    a.yhat = c->yhat;
    a.yF = c->yF;
    a.aF = c->aF;
    a.faceIndex = c->faceIndex;
    a.halo = c->halo;
    a.faceLocal = c->faceLocal;
    a.Cgiven = nullptr;
    a.ctrl = c->ctrl;
    a.mu = c->mu;
    a.eps = c->p.eps;
    a.t = c->t + 1;
    a.first = (c->t == 0);
    a.check_prev = 0;
    a.relabel_period = c->p.relabel_period;
    a.max_pulses = c->p.max_pulses;
    a.fold_rounds = c->p.fold_rounds;
    set_mu(a, c->mu);
    return a;
}

UpdArgs update_args(dope_ctx* c) {
    UpdArgs a;
    a.g = c->g;
    a.Wl = c->Wl;
    a.yhat = c->yhat;
    a.yF = c->yF;
    a.aF = c->aF;
    a.r2blk = c->r2blk;
    a.faceLocal = c->faceLocal;
    a.faceIndex = c->faceIndex;
    a.halo = c->halo;
    a.ctrl = c->ctrl;
    a.mu = c->mu;
    a.t = c->t + 1;
    return a;
}

void fill_stats(dope_ctx* c, const Ctrl& h) {
    c->stats.pulses_total = (int64_t)h.pulses_total;
    c->stats.pulses_max = h.pulses_max;
    c->stats.free_nodes_total = (int64_t)h.free_total;
    c->stats.bfs_levels_total = (int64_t)h.bfs_levels;
    c->stats.bfs_levels_max = h.bfs_levels_max;
    c->stats.fold_rounds_max = h.fold_rounds_max;
    for (int i = 0; i < 4; ++i) c->stats.phase_cycles[i] = (double)h.cyc[i];
    for (int i = 0; i < 4; ++i) c->stats.loop_cycles[i] = (double)h.pcyc[i];
    for (int i = 0; i < 8; ++i) c->stats.window_cycles[i] = (double)h.wcyc[i];
    c->stats.blocks_solved = (int64_t)h.sched_work[0];
    c->stats.blocks_updated = (int64_t)h.sched_work[1];
    c->stats.blocks_solved_partial = (int64_t)h.sched_part;
}

int read_r2max(dope_ctx* c, int t, double* r2, cudaStream_t st) {
    unsigned long long bits = 0;
    CK(cudaMemcpyAsync(&bits, &c->ctrl->r2max[t], sizeof(bits), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    memcpy(r2, &bits, sizeof(*r2));
    return DOPE_OK;
}

int ov_run(dope_ctx* c, int n, cudaStream_t st);
int ov_reset_async(dope_ctx* c, cudaStream_t st);
int ov_finish(dope_ctx* c, uint8_t* labels_dev, int64_t* energy, cudaStream_t st);

// Issue up to n iterations as one cooperative launch (k_admm_resident when
// every block has its own co-resident CTA, else k_admm_persistent).
int persistent_issue(dope_ctx* c, int n, cudaStream_t st, uint8_t* out_labels = nullptr, int out_energy = 0) {
    const int t0 = c->t;
    PersistArgs P;
    P.out_labels = out_labels;
    P.out_energy = out_energy;
    P.s = solve_args(c);
    P.u = update_args(c);
    P.t0 = t0;
    P.n = n;
    P.mu_start = c->mu;
    P.mu_fact = c->p.mu_fact;
    P.spin_limit = c->spin_limit;
    P.dynamic = c->persist_grid < c->g.K;
    P.window = c->window_ok && c->p.launch_mode == 0;
    P.NH = c->NH;
    P.hslot = c->hslot;
    P.hinfo = c->hinfo;
    P.wl_cont = 0;
    P.lwin = 0;
    P.lwcap = 0;
    P.wslot = c->wslot;
    P.wtag = c->wtag;
    P.wmask = c->wmask;
    P.wst = c->wst;
    c->sched_launch = false;
    if (c->sched && !c->resident && c->p.mu_fact >= 1.0) {
        // worklists: valid while mu does not decrease (the forced test's bound
        // only grows); each launch's marks carry a new epoch.  A launch that
        // continues the previous list launch of this context from the state it
        // left (nothing changed since) starts from its lists.
        ++c->sched_epoch;
        P.s.sched = P.u.sched = c->sched;
        P.s.epoch = P.u.epoch = c->sched_epoch;
        P.wl_cont = (c->t > 0 && c->sched_t == c->t) ? 1 : 0;
        c->sched_launch = true;
        // run-ahead windows over the lists (launch_mode 0): per-chunk partial
        // sums of a piece of up to MB blocks, LWMAX iterations at most
        if (c->wslot && P.dynamic && c->p.launch_mode == 0) {
            // chunk sums of a piece (MB blocks) in at most half of it, the list
            // of moving slots in the rest
            const long long per_it = (long long)MB * ((c->g.F + 31) / 32) * 8;
            const long long cap = ((long long)c->smem / 2 - (long long)MB * ((c->g.F + 31) / 32) * 8) / per_it;
            P.lwcap = (int)(cap < LWMAX ? cap : LWMAX);
            P.lwin = P.lwcap >= 2 ? 1 : 0;
        }
    }
    c->sched_t = -1;
    void* args[] = {&P};
    if (c->profiling) {
        if (c->ev.size() < 2) {
            c->ev.resize(2);
            for (auto& e : c->ev) CK(cudaEventCreate(&e));
        }
        CK(cudaEventRecord(c->ev[0], st));
    }
    cudaError_t e;
    if (c->resident) {
        const void* fn = c->conn == 4 ? (const void*)k_admm_resident<4>
                       : c->conn == 8 ? (const void*)k_admm_resident<8> : (const void*)k_admm_resident<6>;
        e = cudaLaunchCooperativeKernel(fn, c->g.K, c->resident_threads, args, c->resident_smem, st);
    } else {
        e = cudaLaunchCooperativeKernel(persistent_fn(c->conn, c->pthreads), c->persist_grid, c->pthreads, args,
                                        c->smem, st);
        if (e == cudaSuccess && P.lwin) {
            // the windowed form continues where the plain one handed off (it
            // returns at once when the plain one ended the launch)
            c->launches++;
            e = cudaLaunchCooperativeKernel(persistent_fn(c->conn, c->pthreads, true), c->persist_grid, c->pthreads,
                                            args, c->smem, st);
        }
    }
    if (e != cudaSuccess) return DOPE_ECUDA;
    c->launches++;
    if (c->profiling) CK(cudaEventRecord(c->ev[1], st));
    return DOPE_OK;
}

// Fold a finished persistent launch (control header h, and the per-iteration
// r2 trace when the caller copied it) into the context state and statistics.
int persistent_collect(dope_ctx* c, int t0, const Ctrl& h, const unsigned long long* r2trace, cudaStream_t st) {
    if (h.status) return h.status;
    const int done = h.iters_done - t0;
    c->sched_t = c->sched_launch ? t0 + done : -1;
    const int converged = h.conv_t != 0;
    if (c->profiling) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
        c->prof.launches[0]++;
        c->prof.ms[0] += ms;
        c->prof.iterations += done;
        if (t0 == 0) c->prof.first_iteration_launches++;
    }
    double mu = c->mu;
    for (int j = 0; j < done; ++j) mu = mu * c->p.mu_fact;
    c->t = t0 + done;
    c->mu = mu;
    c->stats.iterations = c->t;
    c->stats.converged = converged;
    fill_stats(c, h);
    c->stats.windows = h.windows;
    c->stats.window_iterations = h.window_iters;
    c->stats.solver_kernel = c->resident ? 2 : 1;
    double r2 = 0.0;
    if (r2trace) {
        memcpy(&r2, &r2trace[c->t], sizeof(r2));
    } else {
        int rc = read_r2max(c, c->t, &r2, st);
        if (rc) return rc;
    }
    c->stats.rmax_last = std::sqrt(r2);
    c->stats.kernel_launches = c->launches;
    return DOPE_OK;
}

// Up to n iterations in one cooperative launch of k_admm_persistent.
int run_persistent(dope_ctx* c, int n, cudaStream_t st) {
    const int t0 = c->t;
    int rc = persistent_issue(c, n, st);
    if (rc) return rc;
    Ctrl h{};
    rc = read_ctrl(c, &h, st);
    if (rc) return rc;
    return persistent_collect(c, t0, h, nullptr, st);
}

// Up to n iterations of Algorithm 1 from the current state.
int run_iterations(dope_ctx* c, int n, cudaStream_t st) {
    {
        const int rc = settle_inputs(c, st);
        if (rc) return rc;
    }
    if (!c->have_u || !c->have_w) return DOPE_EINVAL;
    const int t0 = c->t;
    if (n > c->p.max_iter - t0) n = c->p.max_iter - t0;
    memset(&c->stats, 0, sizeof(c->stats));
    if (n <= 0) {
        c->stats.iterations = c->t;
        return DOPE_OK;
    }
    int rc = clear_status(c, st);
    if (rc) return rc;
    CK(cudaMemsetAsync(&c->ctrl->r2max[t0 + 1], 0, sizeof(unsigned long long) * (size_t)n, st));
    if (c->ov) return ov_run(c, n, st);
    if (c->p.launch_mode != 1 && c->persist_grid > 0) return run_persistent(c, n, st);
    if (c->profiling && c->ev.size() < 3 * (size_t)n) {
        size_t have = c->ev.size();
        c->ev.resize(3 * (size_t)n);
        for (size_t i = have; i < c->ev.size(); ++i) CK(cudaEventCreate(&c->ev[i]));
    }
    std::vector<double> mus((size_t)n + 1);
    mus[0] = c->mu;
    for (int j = 1; j <= n; ++j) mus[j] = mus[j - 1] * c->p.mu_fact;
    Ctrl h{};
    int launched = 0, batch = 4;
    while (launched < n) {
        const int nb = (n - launched < batch) ? n - launched : batch;
        for (int j = 0; j < nb; ++j) {
            const int idx = launched + j;
            SolveArgs sa = solve_args(c);
            sa.t = t0 + idx + 1;
            set_mu(sa, mus[idx]);
            sa.first = (t0 + idx == 0);
            sa.check_prev = (idx > 0);
            if (c->profiling) CK(cudaEventRecord(c->ev[3 * idx], st));
            solve_launch(c, sa, st);
            if (c->profiling) CK(cudaEventRecord(c->ev[3 * idx + 1], st));
            UpdArgs ua = update_args(c);
            ua.t = t0 + idx + 1;
            ua.mu = mus[idx];
            update_launch(c, ua, st);
            if (c->profiling) CK(cudaEventRecord(c->ev[3 * idx + 2], st));
        }
        CK(cudaGetLastError());
        launched += nb;
        rc = read_ctrl(c, &h, st);
        if (rc) return rc;
        if (h.status) return h.status;
        if (h.conv_t) break;
        if (batch < 32) batch *= 2;
    }
    int done, converged;
    if (h.conv_t) {
        done = h.conv_t - t0;
        converged = 1;
    } else {
        done = launched;
        unsigned long long bits = 0;
        CK(cudaMemcpyAsync(&bits, &c->ctrl->r2max[t0 + done], sizeof(bits), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        double r2;
        memcpy(&r2, &bits, sizeof(r2));
        converged = !(std::sqrt(r2) > c->p.eps);
    }
    if (c->profiling) {
        for (int idx = 0; idx < done; ++idx) {
            float a = 0.f, b = 0.f;
            CK(cudaEventElapsedTime(&a, c->ev[3 * idx], c->ev[3 * idx + 1]));
            CK(cudaEventElapsedTime(&b, c->ev[3 * idx + 1], c->ev[3 * idx + 2]));
            c->prof.launches[0]++;
            c->prof.ms[0] += a;
            c->prof.launches[1]++;
            c->prof.ms[1] += b;
            c->prof.iterations++;
            if (t0 + idx == 0) {
                c->prof.first_iteration_launches++;
                c->prof.first_iteration_ms += a;
            }
        }
    }
    c->t = t0 + done;
    c->mu = mus[done];
    c->sched_t = -1;
    c->stats.iterations = c->t;
    c->stats.converged = converged;
    fill_stats(c, h);
    {
        unsigned long long bits = 0;
        CK(cudaMemcpyAsync(&bits, &c->ctrl->r2max[c->t], sizeof(bits), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        double r2;
        memcpy(&r2, &bits, sizeof(r2));
        c->stats.rmax_last = std::sqrt(r2);
    }
    c->stats.kernel_launches = c->launches;
    return DOPE_OK;
}

int energy_of(dope_ctx* c, const uint8_t* lab_bm, int64_t* out, cudaStream_t st) {
    CK(cudaMemsetAsync(&c->ctrl->energy, 0, sizeof(unsigned long long), st));
    c->launches++;
    const int threads = 256;
    const int blocks = grid_for(c->g.N, threads);
    if (c->conn == 4) k_energy<4><<<blocks, threads, 0, st>>>(c->g, c->U, c->Wl, lab_bm, c->ctrl);
    else if (c->conn == 8) k_energy<8><<<blocks, threads, 0, st>>>(c->g, c->U, c->Wl, lab_bm, c->ctrl);
    else k_energy<6><<<blocks, threads, 0, st>>>(c->g, c->U, c->Wl, lab_bm, c->ctrl);
    CK(cudaGetLastError());
    unsigned long long v = 0;
    CK(cudaMemcpyAsync(&v, &c->ctrl->energy, sizeof(v), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (out) *out = (int64_t)v;
    return DOPE_OK;
}

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum.
// The limit is a per-function, process-wide setting: setting it to one
// context's own size would lower it under another context's launches.
void raise_smem_limit(const void* fn) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess && optin > (int)fa.sharedSizeBytes)
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaGetLastError();
}

template <int CONN>
void raise_smem_limits() {
    raise_smem_limit((const void*)k_block_solve<CONN>);
    raise_smem_limit((const void*)k_admm_persistent<CONN, 256, false>);
    raise_smem_limit((const void*)k_admm_persistent<CONN, 512, false>);
    raise_smem_limit((const void*)k_admm_persistent<CONN, 256, true>);
    raise_smem_limit((const void*)k_admm_persistent<CONN, 512, true>);
    raise_smem_limit((const void*)k_admm_resident<CONN>);
    raise_smem_limit((const void*)k_nsm_solve<CONN>);
}

// Algorithm 1 initialisation (y = 1/2, a = 0, mu = mu0), stream-ordered.
int reset_state_async(dope_ctx* c, cudaStream_t st) {
    c->t = 0;
    c->mu = c->p.mu0;
    c->sched_t = -1;
    const int threads = 256;
    k_init_state<<<grid_for((long long)c->g.K * c->g.F, threads), threads, 0, st>>>(c->g, c->yF, c->aF);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(c->yhat, 0, (size_t)c->g.N, st));
    return DOPE_OK;
}

int reset_state(dope_ctx* c) {
    int rc = c->ov ? ov_reset_async(c, 0) : reset_state_async(c, 0);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    return DOPE_OK;
}


// Persistent-launch choices of a context: CTAs of k_admm_persistent, and
// whether the resident kernel (one CTA per block, with or without its
// run-ahead window arrays) fits co-resident.
void choose_launch(dope_ctx* c) {
    const Geo& g = c->g;
    const int connectivity = c->conn;
    const long long B = g.B;
    c->pthreads = solver_width(g.B, c->p.threads > 0 ? c->p.threads : c->threads);
    if (c->p.threads > 0) c->pthreads = c->threads;
    int dev = 0, sms = 0, coop = 0, per_sm = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // co-resident CTAs of both forms (plain and windowed): the grid fits either
    per_sm = 1 << 30;
    for (int win = 0; win < 2; ++win) {
        const void* fn = persistent_fn(connectivity, c->pthreads, win != 0);
        cudaFuncAttributes fa0;
        int n = 0;
        if (cudaFuncGetAttributes(&fa0, fn) != cudaSuccess ||
            (size_t)c->smem + fa0.sharedSizeBytes > (size_t)optin ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, c->pthreads, c->smem) != cudaSuccess)
            n = 0;
        if (n < per_sm) per_sm = n;
    }
    cudaGetLastError();
    long long cap = (long long)per_sm * sms;
    c->persist_grid = (coop && cap > 0) ? (int)(cap < g.K ? cap : g.K) : 0;
    const void* fr = connectivity == 4 ? (const void*)k_admm_resident<4>
                   : connectivity == 8 ? (const void*)k_admm_resident<8>
                                       : (const void*)k_admm_resident<6>;
    int rt = (int)((B + 31) / 32 * 32);
    if (rt > 256) rt = 256;
    cudaFuncAttributes fa;
    size_t static_smem = 0;
    if (cudaFuncGetAttributes(&fa, fr) == cudaSuccess) static_smem = fa.sharedSizeBytes;
    else optin = 0;
    for (int with_window = 1; with_window >= 0 && !c->resident; --with_window) {
        const size_t rs = with_window ? window_smem_bytes(connectivity, (int)B, g.F, c->NH)
                                      : resident_smem_bytes(connectivity, (int)B, g.F);
        int per_sm_r = 0;
        if (coop && rs + static_smem <= (size_t)optin && (long long)rt * NPTMAX >= B &&
            c->p.threads == 0 && g.F <= 128 * 32) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_r, fr, rt, rs) != cudaSuccess)
                per_sm_r = 0;
        }
        cudaGetLastError();
        if (per_sm_r > 0 && (long long)per_sm_r * sms >= g.K) {
            c->resident = 1;
            c->resident_smem = (int)rs;
            c->resident_threads = rt;
            c->window_ok = with_window;
        }
    }
}

// ---------------------------------------------------------------------------
// Overlapping partition (grow != 0): set-up, iterations, finish.
// ---------------------------------------------------------------------------
// Tiles along one axis whose grown range [t b - g, (t+1) b + g) holds c.
int ov_axis_q(long long c, int b, int gr, int nb) {
    long long lo = c - gr >= 0 ? (c - gr) / b : -((gr - c + b - 1) / b);
    long long hi = (c + gr) / b;
    if (lo < 0) lo = 0;
    if (hi > nb - 1) hi = nb - 1;
    return (int)(hi - lo + 1);
}

// Calls f(std::integral_constant<int, CONN>) for the connectivities the
// overlapping-partition kernels are built for (the 3x3 ones and the larger
// kernels of Section 3); false for any other.
template <class F>
bool ov_dispatch(int conn, F&& f) {
    switch (conn) {
        case 4: f(std::integral_constant<int, 4>{}); return true;
        case 8: f(std::integral_constant<int, 8>{}); return true;
        case 6: f(std::integral_constant<int, 6>{}); return true;
        default: return false;   // the larger kernels: dope_big.cu's launchers
    }
}

template <int CONN>
void ov_raise_smem() {
    static std::once_flag once;
    std::call_once(once, []() { raise_smem_limit((const void*)k_ov_solve<CONN>); });
}

int ov_reset_async(dope_ctx* c, cudaStream_t st) {
    c->t = 0;
    c->mu = c->p.mu0;
    c->sched_t = -1;
    const OvArgs& A = c->oa;
    const int threads = 256;
    // y = 1/2 (Algorithm 1 initialisation), a = 0, yhat = 0
    k_init_state<<<grid_for(A.N, threads), threads, 0, st>>>(Geo{1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1,
                                                                   (int)A.N, A.N, 1, 1, 1, A.N}, A.y, A.a);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(A.a, 0, sizeof(double) * (size_t)A.g.K * A.g.B, st));
    CK(cudaMemsetAsync(A.yhat, 0, (size_t)A.g.K * A.g.B, st));
    return DOPE_OK;
}

int create_overlap(dope_ctx* c, const int64_t dims[3], const int32_t blk[3], const int grow3[3],
                   cudaStream_t st) {
    for (int i = 0; i < 3; ++i)
        if (grow3[i] < 0 || 2 * grow3[i] > blk[i]) return DOPE_EINVAL;
    const long long box = (long long)(blk[0] + 2 * grow3[0]) * (blk[1] + 2 * grow3[1]) * (blk[2] + 2 * grow3[2]);
    if (box > 4096) return DOPE_EINVAL;
    const long long N = dims[0] * dims[1] * dims[2];
    c->ov = 1;
    // flat geometry: the whole grid as one "block", so the set-up kernels keep image order
    Geo& g = c->g;
    g.D = (int)dims[0]; g.H = (int)dims[1]; g.W = (int)dims[2];
    g.bd = g.D; g.bh = g.H; g.bw = g.W;
    g.B = (int)(N < (1LL << 30) ? N : (1LL << 30));
    g.nbz = g.nby = g.nbx = 1;
    g.K = 1;
    g.F = 0;
    g.N = N;
    g.Du = g.D; g.Hu = g.H; g.Wu = g.W;
    g.Nu = N;
    OvArgs& A = c->oa;
    A.D = g.D; A.H = g.H; A.W = g.W;
    A.tbd = blk[0]; A.tbh = blk[1]; A.tbw = blk[2];
    A.gd = grow3[0]; A.gh = grow3[1]; A.gw = grow3[2];
    A.nbz = (int)(dims[0] / blk[0]); A.nby = (int)(dims[1] / blk[1]); A.nbx = (int)(dims[2] / blk[2]);
    const int qmax = (A.gd ? 2 : 1) * (A.gh ? 2 : 1) * (A.gw ? 2 : 1);
    A.M = qmax * qmax;
    A.N = N;
    Geo& b = A.g;
    memset(&b, 0, sizeof(b));
    b.bd = blk[0] + 2 * A.gd; b.bh = blk[1] + 2 * A.gh; b.bw = blk[2] + 2 * A.gw;
    b.B = (int)box;
    b.D = b.bd; b.H = b.bh; b.W = b.bw;
    b.nbz = A.nbz; b.nby = A.nby; b.nbx = A.nbx;
    b.K = A.nbz * A.nby * A.nbx;
    b.N = (long long)b.K * b.B;
    A.eps = c->p.eps;
    A.relabel_period = c->p.relabel_period;
    A.max_pulses = c->p.max_pulses;
    A.fold_rounds = c->p.fold_rounds;
    int t = (int)((box + 31) / 32 * 32);
    if (t > 512) t = 512;
    if (t < 32) t = 32;
    c->ov_threads = t;
    c->ov_smem = (int)solver_smem_bytes(c->conn, (int)box);
    c->threads = t;
    c->smem = c->ov_smem;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (c->ov_smem > optin) return DOPE_EINVAL;
    if (!ov_dispatch(c->conn, [](auto cc) { ov_raise_smem<decltype(cc)::value>(); })) big_raise_smem(c->conn);
    const int nh = c->conn / 2;
    const size_t KB = (size_t)b.K * b.B;
    int rc = DOPE_OK;
    auto Al = [&](void** ptr, size_t bytes) {
        if (rc == DOPE_OK) {
            *ptr = dalloc(c->al, bytes);
            if (!*ptr) rc = DOPE_ENOMEM;
        }
    };
    Al((void**)&c->U, sizeof(int32_t) * (size_t)N);
    Al((void**)&c->Wl, sizeof(int32_t) * (size_t)N * nh);
    Al((void**)&A.q, (size_t)N);
    Al((void**)&A.y, sizeof(double) * (size_t)N);
    Al((void**)&A.a, sizeof(double) * KB);
    Al((void**)&A.yhat, KB);
    Al((void**)&c->r2blk, sizeof(double) * (size_t)b.K);
    c->ctrl_bytes = sizeof(Ctrl) + sizeof(unsigned long long) * ((size_t)c->p.max_iter + 2);
    Al((void**)&c->ctrl, c->ctrl_bytes);
    if (rc) return rc;
    A.U = c->U;
    A.Wl = c->Wl;
    A.r2blk = c->r2blk;
    A.ctrl = c->ctrl;
    // q: blocks holding each pixel (Proposition 1's q_ii), per-axis counts multiplied
    std::vector<uint8_t> q((size_t)N);
    for (long long z = 0; z < dims[0]; ++z) {
        const int qz = ov_axis_q(z, blk[0], A.gd, A.nbz);
        for (long long y = 0; y < dims[1]; ++y) {
            const int qy = ov_axis_q(y, blk[1], A.gh, A.nby);
            for (long long x = 0; x < dims[2]; ++x)
                q[(size_t)((z * dims[1] + y) * dims[2] + x)] = (uint8_t)(qz * qy * ov_axis_q(x, blk[2], A.gw, A.nbx));
        }
    }
    if (cudaMemcpy(const_cast<uint8_t*>(A.q), q.data(), (size_t)N, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemsetAsync(c->ctrl, 0, c->ctrl_bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return DOPE_ECUDA;
    }
    if (A.gd | A.gh | A.gw) {
        // Eq. 10's two pixel lists: "inner" pixels are held, with every pixel
        // within the kernel radius, by one block only; along each axis the
        // holding range [lo, hi] is monotone in the coordinate, so that is
        // lo(c - R) == hi(c + R) per axis
        const int R = c->conn == 24 || c->conn == 32 ? 2 : (c->conn == 48 ? 3 : (c->conn == 80 ? 4 : 1));
        const bool three_d = c->conn == 6 || c->conn == 32;
        auto axis = [&](long long n, int b, int gr, int nb, int r) {
            std::vector<uint8_t> v((size_t)n);
            auto fdiv = [](long long a, long long d) { return a >= 0 ? a / d : -((-a + d - 1) / d); };
            for (long long x = 0; x < n; ++x) {
                long long lo = fdiv(x - r - gr, b), hi = fdiv(x + r + gr, b);
                if (lo < 0) lo = 0;
                if (hi > nb - 1) hi = nb - 1;
                v[(size_t)x] = lo == hi;
            }
            return v;
        };
        const auto iz = axis(dims[0], blk[0], A.gd, A.nbz, three_d ? R : 0);
        const auto iy = axis(dims[1], blk[1], A.gh, A.nby, R);
        const auto ix = axis(dims[2], blk[2], A.gw, A.nbx, R);
        std::vector<int> inner, band;
        inner.reserve((size_t)N);
        for (long long z = 0; z < dims[0]; ++z)
            for (long long y = 0; y < dims[1]; ++y)
                for (long long x = 0; x < dims[2]; ++x) {
                    const int j = (int)((z * dims[1] + y) * dims[2] + x);
                    if (iz[(size_t)z] && iy[(size_t)y] && ix[(size_t)x]) inner.push_back(j);
                    else band.push_back(j);
                }
        int* di = (int*)dalloc(c->al, sizeof(int) * (inner.size() + 1));
        int* db = (int*)dalloc(c->al, sizeof(int) * (band.size() + 1));
        if (!di || !db) {
            dfree(c->al, di);
            dfree(c->al, db);
            return DOPE_ENOMEM;
        }
        A.inner = di;
        A.band = db;
        A.n_inner = (long long)inner.size();
        A.n_band = (long long)band.size();
        if ((!inner.empty() && cudaMemcpy(di, inner.data(), sizeof(int) * inner.size(), cudaMemcpyHostToDevice) != cudaSuccess) ||
            (!band.empty() && cudaMemcpy(db, band.data(), sizeof(int) * band.size(), cudaMemcpyHostToDevice) != cudaSuccess)) {
            cudaGetLastError();
            return DOPE_ECUDA;
        }
    }
    return ov_reset_async(c, st);
}

template <int CONN>
void ov_launch_iteration(dope_ctx* c, int t, double mu, int check_prev, cudaStream_t st, cudaEvent_t mid) {
    const OvArgs& A = c->oa;
    k_ov_solve<CONN><<<A.g.K, c->ov_threads, c->ov_smem, st>>>(A, mu, t, check_prev);
    if (mid) cudaEventRecord(mid, st);
    if ((A.gd | A.gh | A.gw) == 0) {
        k_ov_y_q1<CONN><<<grid_for(A.N, 256), 256, 0, st>>>(A, mu);
    } else if (A.inner) {
        k_ov_y_inner<CONN><<<grid_for(A.n_inner, 256), 256, 0, st>>>(A, mu);
        k_ov_y_band<CONN><<<grid_for(A.n_band, 256), 256, 0, st>>>(A, mu);
        c->launches++;
    } else {
        k_ov_y<CONN><<<grid_for(A.N, 256), 256, 0, st>>>(A, mu);
    }
    k_ov_a<CONN><<<A.g.K, 256, 0, st>>>(A, t);
    c->launches += 3;
}

// Up to n iterations of Algorithm 1 on the overlapping partition (three
// launches per iteration, issued in batches; the stop test of iteration t is
// read by iteration t + 1's solve launch, as in launch mode 1).
int ov_run(dope_ctx* c, int n, cudaStream_t st) {
    const int t0 = c->t;
    std::vector<double> mus((size_t)n + 1);
    mus[0] = c->mu;
    for (int j = 1; j <= n; ++j) mus[j] = mus[j - 1] * c->p.mu_fact;
    if (c->profiling && c->ev.size() < 3 * (size_t)n) {
        const size_t have = c->ev.size();
        c->ev.resize(3 * (size_t)n);
        for (size_t i = have; i < c->ev.size(); ++i) CK(cudaEventCreate(&c->ev[i]));
    }
    Ctrl h{};
    int launched = 0, batch = 4;
    while (launched < n) {
        const int nb = (n - launched < batch) ? n - launched : batch;
        for (int j = 0; j < nb; ++j) {
            const int idx = launched + j;
            if (c->profiling) CK(cudaEventRecord(c->ev[3 * idx], st));
            cudaEvent_t mid = c->profiling ? c->ev[3 * idx + 1] : nullptr;
            if (!ov_dispatch(c->conn, [&](auto cc) {
                    ov_launch_iteration<decltype(cc)::value>(c, t0 + idx + 1, mus[idx], idx > 0, st, mid);
                })) {
                big_ov_iteration(c->conn, c->oa, c->ov_threads, c->ov_smem, mus[idx], t0 + idx + 1, idx > 0, st, mid);
                c->launches += 3;
            }
            if (c->profiling) CK(cudaEventRecord(c->ev[3 * idx + 2], st));
        }
        CK(cudaGetLastError());
        launched += nb;
        int rc = read_ctrl(c, &h, st);
        if (rc) return rc;
        if (h.status) return h.status;
        if (h.conv_t) break;
        if (batch < 32) batch *= 2;
    }
    int done, converged;
    if (h.conv_t) {
        done = h.conv_t - t0;
        converged = 1;
    } else {
        done = launched;
        double r2 = 0.0;
        int rc = read_r2max(c, t0 + done, &r2, st);
        if (rc) return rc;
        converged = !(std::sqrt(r2) > c->p.eps);
    }
    if (c->profiling) {
        for (int idx = 0; idx < done; ++idx) {
            float ms_a = 0.f, ms_b = 0.f;
            CK(cudaEventElapsedTime(&ms_a, c->ev[3 * idx], c->ev[3 * idx + 1]));
            CK(cudaEventElapsedTime(&ms_b, c->ev[3 * idx + 1], c->ev[3 * idx + 2]));
            c->prof.launches[0]++;
            c->prof.ms[0] += ms_a;
            c->prof.launches[1]++;
            c->prof.ms[1] += ms_b;
            c->prof.iterations++;
            if (t0 + idx == 0) {
                c->prof.first_iteration_launches++;
                c->prof.first_iteration_ms += ms_a;
            }
        }
    }
    c->t = t0 + done;
    c->mu = mus[done];
    c->sched_t = -1;
    c->stats.iterations = c->t;
    c->stats.converged = converged;
    fill_stats(c, h);
    double r2 = 0.0;
    int rc = read_r2max(c, c->t, &r2, st);
    if (rc) return rc;
    c->stats.rmax_last = std::sqrt(r2);
    c->stats.kernel_launches = c->launches;
    c->stats.solver_kernel = 0;
    return DOPE_OK;
}

// Proposition 1 labels (image order, device) and, if asked, their E_int.
int ov_finish(dope_ctx* c, uint8_t* labels_dev, int64_t* energy, cudaStream_t st) {
    const OvArgs& A = c->oa;
    k_ov_labels<<<grid_for(A.N, 256), 256, 0, st>>>(A, labels_dev);
    c->launches++;
    CK(cudaGetLastError());
    if (energy) {
        CK(cudaMemsetAsync(&c->ctrl->energy, 0, sizeof(unsigned long long), st));
        const int blocks = grid_for(A.N, 256);
        if (!ov_dispatch(c->conn, [&](auto cc) {
                k_energy_img<decltype(cc)::value><<<blocks, 256, 0, st>>>(A.D, A.H, A.W, c->U, c->Wl, labels_dev, c->ctrl);
            }))
            big_energy_img(c->conn, A.D, A.H, A.W, c->U, c->Wl, labels_dev, c->ctrl, blocks, 256, st);
        c->launches++;
        CK(cudaGetLastError());
        unsigned long long v = 0;
        CK(cudaMemcpyAsync(&v, &c->ctrl->energy, sizeof(v), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        *energy = (int64_t)v;
    }
    return DOPE_OK;
}

std::once_flag g_smem_once[3];

void raise_all_smem_limits(int conn) {
    const int ci = conn == 4 ? 0 : (conn == 8 ? 1 : 2);
    std::call_once(g_smem_once[ci], [conn]() {
        if (conn == 4) raise_smem_limits<4>();
        else if (conn == 8) raise_smem_limits<8>();
        else raise_smem_limits<6>();
        raise_smem_limit((const void*)k_admm_batch<256>);
        raise_smem_limit((const void*)k_admm_batch<512>);
    });
}

}  // namespace

int dope_tables_create(int connectivity, const int32_t blk3[3], const dope_allocator* alp,
                       cudaStream_t st, dope_tables** out) {
    if (!out || !blk3) return DOPE_EINVAL;
    *out = nullptr;
    if (connectivity != 4 && connectivity != 8 && connectivity != 6) return DOPE_EINVAL;
    const int bd = blk3[0], bh = blk3[1], bw = blk3[2];
    if (bd <= 0 || bh <= 0 || bw <= 0 || (long long)bd * bh * bw > 4096) return DOPE_EINVAL;
    const int B = bd * bh * bw;
    // face slots: pixels with a neighbour outside their block (any direction)
    static const int OFF[3][4][3] = {
        {{0, 0, 1}, {0, 1, 0}, {0, 0, 0}, {0, 0, 0}},
        {{0, 0, 1}, {0, 1, 0}, {0, 1, 1}, {0, 1, -1}},
        {{0, 0, 1}, {0, 1, 0}, {1, 0, 0}, {0, 0, 0}}};
    const int ci = connectivity == 4 ? 0 : (connectivity == 8 ? 1 : 2);
    const int nh = connectivity / 2;
    std::vector<int16_t> fidx((size_t)B, -1), floc;
    for (int l = 0; l < B; ++l) {
        int lx = l % bw, ly = (l / bw) % bh, lz = l / (bw * bh);
        bool face = false;
        for (int o = 0; o < nh && !face; ++o)
            for (int sg = -1; sg <= 1; sg += 2) {
                int z = lz + sg * OFF[ci][o][0], y = ly + sg * OFF[ci][o][1], x = lx + sg * OFF[ci][o][2];
                if (z < 0 || z >= bd || y < 0 || y >= bh || x < 0 || x >= bw) face = true;
            }
        if (face) {
            fidx[(size_t)l] = (int16_t)floc.size();
            floc.push_back((int16_t)l);
        }
    }
    const int F = (int)floc.size();
    // halo table [conn][F]: the cross-block neighbour of every face slot
    std::vector<int> halo((size_t)connectivity * (F ? F : 1), -1);
    for (int f = 0; f < F; ++f) {
        const int l = floc[(size_t)f];
        const int lx = l % bw, ly = (l / bw) % bh, lz = l / (bw * bh);
        for (int d = 0; d < connectivity; ++d) {
            const int o = d < nh ? d : d - nh, sg = d < nh ? 1 : -1;
            int z = lz + sg * OFF[ci][o][0], y = ly + sg * OFF[ci][o][1], x = lx + sg * OFF[ci][o][2];
            if (z >= 0 && z < bd && y >= 0 && y < bh && x >= 0 && x < bw) continue;
            const int dkz = z < 0 ? -1 : (z >= bd ? 1 : 0);
            const int dky = y < 0 ? -1 : (y >= bh ? 1 : 0);
            const int dkx = x < 0 ? -1 : (x >= bw ? 1 : 0);
            z -= dkz * bd; y -= dky * bh; x -= dkx * bw;
            const int ln = (z * bh + y) * bw + x;
            halo[(size_t)d * F + f] = halo_entry((dkz + 1) * 9 + (dky + 1) * 3 + (dkx + 1), ln,
                                                 fidx[(size_t)ln]);
        }
    }
    // distinct halo pixels (first-seen order over face slots, then directions)
    std::vector<int16_t> hslot((size_t)connectivity * (F ? F : 1), -1);
    std::vector<int> hinfo;
    for (int f = 0; f < F; ++f)
        for (int d = 0; d < connectivity; ++d) {
            const int e = halo[(size_t)d * F + f];
            if (e < 0) continue;
            int slot = -1;
            for (size_t h = 0; h < hinfo.size(); ++h)
                if (hinfo[h] == e) { slot = (int)h; break; }
            if (slot < 0) { slot = (int)hinfo.size(); hinfo.push_back(e); }
            hslot[(size_t)d * F + f] = (int16_t)slot;
        }
    const int NH = (int)hinfo.size();
    if (hinfo.empty()) hinfo.push_back(-1);

    dope_tables* t = new (std::nothrow) dope_tables();
    if (!t) return DOPE_ENOMEM;
    t->conn = connectivity;
    t->blk[0] = bd; t->blk[1] = bh; t->blk[2] = bw;
    t->F = F;
    t->NH = NH;
    t->al = alp ? *alp : dope_allocator{nullptr, nullptr, nullptr};
    const size_t b_fi = sizeof(int16_t) * (size_t)B, b_fl = sizeof(int16_t) * (size_t)(F ? F : 1);
    const size_t b_ha = sizeof(int) * halo.size(), b_hs = sizeof(int16_t) * hslot.size();
    const size_t b_hi = sizeof(int) * hinfo.size();
    t->faceIndex = (int16_t*)dalloc(t->al, b_fi);
    t->faceLocal = (int16_t*)dalloc(t->al, b_fl);
    t->halo = (int*)dalloc(t->al, b_ha);
    t->hslot = (int16_t*)dalloc(t->al, b_hs);
    t->hinfo = (int*)dalloc(t->al, b_hi);
    t->bytes = b_fi + b_fl + b_ha + b_hs + b_hi;
    if (!t->faceIndex || !t->faceLocal || !t->halo || !t->hslot || !t->hinfo) {
        dope_tables_destroy(t);
        return DOPE_ENOMEM;
    }
    if (cudaMemcpyAsync(t->faceIndex, fidx.data(), b_fi, cudaMemcpyHostToDevice, st) ||
        (F && cudaMemcpyAsync(t->faceLocal, floc.data(), sizeof(int16_t) * (size_t)F, cudaMemcpyHostToDevice, st)) ||
        cudaMemcpyAsync(t->halo, halo.data(), b_ha, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(t->hslot, hslot.data(), b_hs, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(t->hinfo, hinfo.data(), b_hi, cudaMemcpyHostToDevice, st)) {
        cudaGetLastError();
        dope_tables_destroy(t);
        return DOPE_ECUDA;
    }
    // pageable sources: the copies above are staged before they return
    *out = t;
    return DOPE_OK;
}

void dope_tables_destroy(dope_tables* t) {
    if (!t) return;
    dfree(t->al, t->faceIndex);
    dfree(t->al, t->faceLocal);
    dfree(t->al, t->halo);
    dfree(t->al, t->hslot);
    dfree(t->al, t->hinfo);
    delete t;
}

int dope_create_ex(const int64_t* grid, int ndim, int connectivity, const int32_t* block_shape,
                   double lambda, const dope_params* p, int pad, const dope_allocator* alp,
                   dope_tables* tab, cudaStream_t st, dope_ctx** out) {
    if (!out) return DOPE_EINVAL;
    *out = nullptr;
    if (!grid || !block_shape || (ndim != 2 && ndim != 3)) return DOPE_EINVAL;
    const bool big_kernel = (ndim == 2 && (connectivity == 24 || connectivity == 48 || connectivity == 80)) ||
                            (ndim == 3 && connectivity == 32);
    if (ndim == 2 && connectivity != 4 && connectivity != 8 && !big_kernel) return DOPE_EINVAL;
    if (ndim == 3 && connectivity != 6 && !big_kernel) return DOPE_EINVAL;
    if (!(lambda >= 0.0) || !std::isfinite(lambda)) return DOPE_EINVAL;
    int64_t dims[3] = {1, 1, 1}, udims[3] = {1, 1, 1};
    int32_t blk[3] = {1, 1, 1};
    for (int i = 0; i < ndim; ++i) {
        dims[3 - ndim + i] = grid[i];
        blk[3 - ndim + i] = block_shape[i];
    }
    for (int i = 0; i < 3; ++i) {
        if (dims[i] <= 0 || blk[i] <= 0 || dims[i] > (1LL << 30)) return DOPE_EINVAL;
        udims[i] = dims[i];
        if (dims[i] % blk[i]) {
            if (!pad) return DOPE_EINVAL;
            dims[i] = (dims[i] + blk[i] - 1) / blk[i] * blk[i];
        }
    }
    const long long N = dims[0] * dims[1] * dims[2];
    const long long B = (long long)blk[0] * blk[1] * blk[2];
    if (N >= (1LL << 31) || B > 4096) return DOPE_EINVAL;
    if (p && (p->threads < 0 || p->threads > 512 || p->threads % 32 ||
              (p->threads > 0 && (long long)p->threads * NPTMAX < B)))
        return DOPE_EINVAL;
    if (tab && (tab->conn != connectivity || tab->blk[0] != blk[0] || tab->blk[1] != blk[1] ||
                tab->blk[2] != blk[2]))
        return DOPE_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return DOPE_ECUDA;
    }

    dope_ctx* c = new (std::nothrow) dope_ctx();
    if (!c) return DOPE_ENOMEM;
    c->al = alp ? *alp : dope_allocator{nullptr, nullptr, nullptr};
    c->ndim = ndim;
    c->conn = connectivity;
    c->lambda = lambda;
    dope_default_params(&c->p);
    if (p) c->p = *p;
    if (!(c->p.mu0 > 0.0)) c->p.mu0 = (ndim == 3) ? 500.0 : 100.0;
    if (!(c->p.mu_fact > 0.0)) c->p.mu_fact = 1.05;
    if (!(c->p.eps >= 0.0)) c->p.eps = 1e-3;
    if (c->p.max_iter <= 0) c->p.max_iter = 1000;
    if (c->p.relabel_period <= 0) c->p.relabel_period = 8;
    if (c->p.max_pulses <= 0) c->p.max_pulses = (int)(64 * B + 4096);
    if (c->p.fold_rounds <= 0) c->p.fold_rounds = MAX_FOLD_ROUNDS;
    if (c->p.barrier_timeout_us > 0) {
        // SM cycles from the device's clock rate (kHz)
        int dev = 0, khz = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess ||
            khz <= 0) {
            cudaGetLastError();
            khz = 2070000;
        }
        c->spin_limit = (long long)c->p.barrier_timeout_us * (long long)khz / 1000LL + 1;
    }
    {
        int grow3[3] = {0, 0, 0};
        bool any = false;
        for (int i = 0; i < ndim; ++i) {
            grow3[3 - ndim + i] = c->p.grow[i];
            any = any || c->p.grow[i] != 0;
        }
        if (any || big_kernel) {
            // overlapping partitions, and the larger kernels (at zero growth the
            // overlap kernels compute exactly the Q = I iteration)
            int rc = (pad || c->p.lsa_steps > 0) ? DOPE_EINVAL : create_overlap(c, dims, blk, grow3, st);
            if (rc) { dope_destroy(c); return rc; }
            *out = c;
            return DOPE_OK;
        }
    }

    Geo& g = c->g;
    g.D = (int)dims[0]; g.H = (int)dims[1]; g.W = (int)dims[2];
    g.bd = blk[0]; g.bh = blk[1]; g.bw = blk[2];
    g.B = (int)B;
    g.nbz = g.D / g.bd; g.nby = g.H / g.bh; g.nbx = g.W / g.bw;
    g.K = g.nbz * g.nby * g.nbx;
    g.N = N;
    g.Du = (int)udims[0]; g.Hu = (int)udims[1]; g.Wu = (int)udims[2];
    g.Nu = udims[0] * udims[1] * udims[2];

    int rc = DOPE_OK;
    if (!tab) {
        rc = dope_tables_create(connectivity, blk, alp, st, &c->own_tab);
        if (rc) { delete c; return rc; }
        tab = c->own_tab;
    }
    g.F = tab->F;
    c->NH = tab->NH;
    c->faceIndex = tab->faceIndex;
    c->faceLocal = tab->faceLocal;
    c->halo = tab->halo;
    c->hslot = tab->hslot;
    c->hinfo = tab->hinfo;

    int threads = c->p.threads;
    if (threads <= 0) {
        threads = (int)((B + 31) / 32 * 32);
        if (threads > 512) threads = 512;
        if (threads < 32) threads = 32;
    }
    if (threads % 32 || threads > 512 || (long long)threads * NPTMAX < B) {
        dope_destroy(c);
        return DOPE_EINVAL;
    }
    c->threads = threads;
    c->smem = (int)solver_smem_bytes(connectivity, (int)B);
    const int nh = connectivity / 2;

    auto A = [&](void** ptr, size_t bytes) {
        if (rc == DOPE_OK) {
            *ptr = dalloc(c->al, bytes);
            if (!*ptr) rc = DOPE_ENOMEM;
        }
    };
    A((void**)&c->U, sizeof(int32_t) * (size_t)N);
    A((void**)&c->Wl, sizeof(int32_t) * (size_t)N * nh);
    A((void**)&c->yhat, (size_t)N);
    A((void**)&c->yF, sizeof(double) * (size_t)g.K * g.F);
    A((void**)&c->aF, sizeof(double) * (size_t)g.K * g.F);
    A((void**)&c->r2blk, sizeof(double) * (size_t)g.K);
    c->ctrl_bytes = sizeof(Ctrl) + sizeof(unsigned long long) * ((size_t)c->p.max_iter + 2);
    A((void**)&c->ctrl, c->ctrl_bytes);
    if (rc) { dope_destroy(c); return rc; }
    if (cudaMemsetAsync(c->ctrl, 0, c->ctrl_bytes, st) != cudaSuccess) {
        cudaGetLastError();
        dope_destroy(c);
        return DOPE_ECUDA;
    }
    raise_all_smem_limits(connectivity);
    {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (c->smem > optin) { dope_destroy(c); return DOPE_EINVAL; }
    }
    choose_launch(c);
    if (c->p.lsa_steps > 0) {
        // non-submodular: LSA-TR block solves, two launches per iteration
        c->nsm = 1;
        c->persist_grid = 0;
        c->resident = 0;
        if (c->p.threads <= 0) {
            // narrower CTAs: a block's LSA-TR steps are barrier-bound, so more
            // blocks in flight per SM pay more than more threads per block
            // (16x16 blocks: 64 threads solve 1.6x faster than 256)
            int t = (int)(((B + 3) / 4 + 31) / 32 * 32);
            if (t > 512) t = 512;
            if (t < 32) t = 32;
            if ((long long)t * NPTMAX >= B) c->threads = t;
        }
        c->nsm_smem = (int)(((solver_smem_bytes(connectivity, (int)B) + 15) & ~(size_t)15) + nsm_extra_bytes((int)B));
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (c->nsm_smem > optin || pad) { dope_destroy(c); return DOPE_EINVAL; }
    }
    if (!c->nsm) {
        // worklists of the persistent and batched kernels; marks start below
        // every launch's
        const size_t sb = sched_bytes(g.K, g.F);
        A((void**)&c->sched, sb);
        if (rc) { dope_destroy(c); return rc; }
        if (cudaMemsetAsync(c->sched, 0, sb, st) != cudaSuccess) {
            cudaGetLastError();
            dope_destroy(c);
            return DOPE_ECUDA;
        }
        // run-ahead windows of the persistent kernel (list launches that are
        // not resident); tags start below every launch's
        if (!c->resident && c->persist_grid > 0 && c->persist_grid < g.K) {
            A((void**)&c->wslot, sizeof(unsigned long long) * (size_t)g.K * g.F);
            A((void**)&c->wtag, sizeof(unsigned long long) * (size_t)g.K);
            A((void**)&c->wmask, sizeof(unsigned) * CHUNK_WORDS * (size_t)g.K);
            A((void**)&c->wst, 4 * sizeof(double) * (size_t)g.K * g.F);
            if (rc) { dope_destroy(c); return rc; }
            if (cudaMemsetAsync(c->wtag, 0, sizeof(unsigned long long) * (size_t)g.K, st) != cudaSuccess) {
                cudaGetLastError();
                dope_destroy(c);
                return DOPE_ECUDA;
            }
        }
    }
    rc = reset_state_async(c, st);
    if (rc) { dope_destroy(c); return rc; }
    *out = c;
    return DOPE_OK;
}

namespace {
}  // namespace

extern "C" {

void dope_default_params(dope_params* p) {
    if (!p) return;
    p->mu0 = 0.0;
    p->mu_fact = 1.05;
    p->eps = 1e-3;
    p->max_iter = 1000;
    p->relabel_period = 0;
    p->threads = 0;
    p->max_pulses = 0;
    p->fold_rounds = 0;
    p->launch_mode = 0;
    p->grow[0] = p->grow[1] = p->grow[2] = 0;
    p->lsa_steps = 0;
}

const char* dope_strerror(int s) {
    switch (s) {
        case DOPE_OK: return "ok";
        case DOPE_EINVAL: return "invalid argument";
        case DOPE_EUNSUPPORTED: return "unsupported input (negative pairwise weight)";
        case DOPE_ENOMEM: return "out of memory";
        case DOPE_EOVERFLOW: return "capacity out of range";
        case DOPE_ENOTCONV: return "max_iter reached before convergence";
        case DOPE_ETIMEOUT: return "a bounded device loop or wait ran out";
        case DOPE_ECUDA: return "CUDA runtime error";
        case DOPE_ECANCELED: return "request cancelled";
        default: return "unknown status";
    }
}

int dope_check_status(uint64_t* first_bad, int clear) {
    if (!first_bad) return DOPE_EINVAL;
    *first_bad = 0;
#ifdef DOPE_CHECKED
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return DOPE_ECUDA;
    }
    unsigned long long w = 0, wb = 0;
    if (cudaMemcpyFromSymbol(&w, dope::dope_check_word, sizeof(w)) != cudaSuccess) {
        cudaGetLastError();
        return DOPE_ECUDA;
    }
    if (clear) {
        const unsigned long long z = 0;
        if (cudaMemcpyToSymbol(dope::dope_check_word, &z, sizeof(z)) != cudaSuccess) {
            cudaGetLastError();
            return DOPE_ECUDA;
        }
    }
    const int rc = dope_big_check_word(&wb, clear);
    if (rc) return rc;
    *first_bad = (uint64_t)(w ? w : wb);
    return DOPE_OK;
#else
    (void)clear;
    return DOPE_EUNSUPPORTED;
#endif
}

void dope_destroy(dope_ctx* c) {
    if (!c) return;
    const dope_allocator al = c->al;
    dfree(al, c->U);
    dfree(al, c->Wl);
    dfree(al, c->yhat);
    dfree(al, c->yF);
    dfree(al, c->aF);
    dfree(al, c->r2blk);
    dfree(al, c->ctrl);
    dfree(al, c->sched);
    dfree(al, c->wslot);
    dfree(al, c->wtag);
    dfree(al, c->wmask);
    dfree(al, c->wst);
    dfree(al, c->stage);
    dfree(al, c->stage2);
    dfree(al, const_cast<uint8_t*>(c->oa.q));
    dfree(al, const_cast<int*>(c->oa.inner));
    dfree(al, const_cast<int*>(c->oa.band));
    dfree(al, c->oa.y);
    dfree(al, c->oa.a);
    dfree(al, c->oa.yhat);
    if (c->own_tab) dope_tables_destroy(c->own_tab);
    if (c->hctrl) cudaFreeHost(c->hctrl);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    delete c;
}

int dope_create(const int64_t* grid, int ndim, int connectivity, const int32_t* block_shape,
                double lambda, const dope_params* p, dope_ctx** out) {
    int rc = dope_create_ex(grid, ndim, connectivity, block_shape, lambda, p, 0, nullptr, nullptr, 0, out);
    if (rc) return rc;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        dope_destroy(*out);
        *out = nullptr;
        return DOPE_ECUDA;
    }
    return DOPE_OK;
}

// Quantise device unaries (user order) into the context (stream-ordered).
static int issue_set_unaries(dope_ctx* c, const float* src, cudaStream_t st) {
    if (c) c->sched_t = -1;   // inputs or labels change: the worklists no longer hold
    const int threads = 256;
    k_set_unaries<<<grid_for(c->g.N, threads), threads, 0, st>>>(c->g, src, c->U, c->ctrl);
    CK(cudaGetLastError());
    return DOPE_OK;
}

int dope_set_unaries(dope_ctx* c, const float* u, int64_t n, int where, void* stream) {
    if (!c || !u || n != c->g.Nu || (where != DOPE_HOST && where != DOPE_DEVICE)) return DOPE_EINVAL;
    cudaStream_t st = S(stream);
    settle_inputs(c, st);   // an earlier asynchronous upload's error leaves both inputs unset
    const float* src = u;
    if (where == DOPE_HOST) {
        int rc = ensure_stage(c, sizeof(float) * (size_t)n, 0);
        if (rc) return rc;
        CK(cudaMemcpyAsync(c->stage, u, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, st));
        src = (const float*)c->stage;
    }
    int rc = clear_status(c, st);
    if (rc) return rc;
    rc = issue_set_unaries(c, src, st);
    if (rc) return rc;
    Ctrl h{};
    rc = read_ctrl(c, &h, st);
    if (rc) return rc;
    c->have_u = (h.status == 0);
    return h.status;
}

// Quantise device weights (user order, [conn/2][Nu]) into the context.
static int issue_set_weights(dope_ctx* c, const int32_t* src, cudaStream_t st) {
    if (c) c->sched_t = -1;   // inputs or labels change: the worklists no longer hold
    const int threads = 256;
    const int blocks = grid_for(c->g.N, threads);
    if (c->ov) {
        const int nh = c->conn / 2;
        if (!ov_dispatch(c->conn, [&](auto cc) {
                k_set_weights<decltype(cc)::value><<<blocks, threads, 0, st>>>(c->g, src, c->Wl, c->lambda, c->ctrl, 0);
            }))
            big_set_weights(c->conn, c->g, src, c->Wl, c->lambda, c->ctrl, blocks, threads, st);
        const long long scale = (long long)c->oa.M * (c->conn > 8 ? c->conn / 8 : 1);
        k_ov_wcheck<<<grid_for(c->g.N * nh, threads), threads, 0, st>>>(c->Wl, c->g.N * nh, scale, c->ctrl);
    } else if (c->conn == 4) k_set_weights<4><<<blocks, threads, 0, st>>>(c->g, src, c->Wl, c->lambda, c->ctrl, c->nsm);
    else if (c->conn == 8) k_set_weights<8><<<blocks, threads, 0, st>>>(c->g, src, c->Wl, c->lambda, c->ctrl, c->nsm);
    else k_set_weights<6><<<blocks, threads, 0, st>>>(c->g, src, c->Wl, c->lambda, c->ctrl, c->nsm);
    CK(cudaGetLastError());
    return DOPE_OK;
}

int dope_set_weights(dope_ctx* c, const int32_t* wq, int64_t n, int where, void* stream) {
    if (!c || !wq || n != c->g.Nu || (where != DOPE_HOST && where != DOPE_DEVICE)) return DOPE_EINVAL;
    cudaStream_t st = S(stream);
    settle_inputs(c, st);   // an earlier asynchronous upload's error leaves both inputs unset
    const int nh = c->conn / 2;
    const int32_t* src = wq;
    if (where == DOPE_HOST) {
        int rc = ensure_stage(c, sizeof(int32_t) * (size_t)n * nh, 0);
        if (rc) return rc;
        CK(cudaMemcpyAsync(c->stage, wq, sizeof(int32_t) * (size_t)n * nh, cudaMemcpyHostToDevice, st));
        src = (const int32_t*)c->stage;
    }
    int rc = clear_status(c, st);
    if (rc) return rc;
    rc = issue_set_weights(c, src, st);
    if (rc) return rc;
    Ctrl h{};
    rc = read_ctrl(c, &h, st);
    if (rc) return rc;
    c->have_w = (h.status == 0);
    return h.status;
}

int dope_set_inputs(dope_ctx* c, const float* u, const int32_t* wq, int64_t n, int where, void* stream) {
    if (!c || !u || !wq || n != c->g.Nu || (where != DOPE_HOST && where != DOPE_DEVICE)) return DOPE_EINVAL;
    cudaStream_t st = S(stream);
    c->pending = false;   // both inputs are replaced
    const size_t nu = (size_t)n, nh = (size_t)(c->conn / 2);
    const float* su = u;
    const int32_t* sw = wq;
    if (where == DOPE_HOST) {
        const size_t off_w = (sizeof(float) * nu + 255) & ~(size_t)255;
        int rc = ensure_stage(c, off_w + sizeof(int32_t) * nu * nh, 0);
        if (rc) return rc;
        char* base = (char*)c->stage;
        CK(cudaMemcpyAsync(base, u, sizeof(float) * nu, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(base + off_w, wq, sizeof(int32_t) * nu * nh, cudaMemcpyHostToDevice, st));
        su = (const float*)base;
        sw = (const int32_t*)(base + off_w);
    }
    int rc = clear_status(c, st);
    if (!rc) rc = issue_set_unaries(c, su, st);
    if (!rc) rc = issue_set_weights(c, sw, st);
    if (rc) return rc;
    c->have_u = c->have_w = 1;   // provisional: the status is read by the next synchronising call
    c->pending = true;
    return DOPE_OK;
}

// Potentials of an image into the context's staging memory, then the
// quantisers (stream-ordered, no synchronisation).  *ws_out: the device
// scratch whose second double holds the sigma used.
static int image_issue(dope_ctx* c, const float* image, int channels, const dope_gmm* fg, const dope_gmm* bg, double clip,
                double sigma, int inv_dist, int where, cudaStream_t st, cudaEvent_t after_copies, double** ws_out) {
    if (c) c->sched_t = -1;   // inputs change: the worklists no longer hold
    if (!c || !image || channels < 1 || channels > DOPE_GMM_MAX_CH || (where != DOPE_HOST && where != DOPE_DEVICE))
        return DOPE_EINVAL;
    const size_t n = (size_t)c->g.Nu;
    const int nh = c->conn / 2;
    // scratch: [sigma workspace 64 B][u: n floats][wq: nh * n int32][image if on the host]
    const size_t off_u = 64, off_w = off_u + ((sizeof(float) * n + 255) & ~(size_t)255);
    const size_t off_i = off_w + ((sizeof(int32_t) * n * nh + 255) & ~(size_t)255);
    const size_t bytes = off_i + (where == DOPE_HOST ? sizeof(float) * n * channels : 0);
    int rc = ensure_stage(c, bytes, 0);
    if (rc) return rc;
    char* base = (char*)c->stage;
    double* ws = (double*)base;
    float* u = (float*)(base + off_u);
    int32_t* wq = (int32_t*)(base + off_w);
    const float* img = image;
    if (where == DOPE_HOST) {
        CK(cudaMemcpyAsync(base + off_i, image, sizeof(float) * n * channels, cudaMemcpyHostToDevice, st));
        img = (const float*)(base + off_i);
    }
    if (after_copies) CK(cudaEventRecord(after_copies, st));
    rc = pot_unaries_issue(img, (long long)n, channels, fg, bg, clip, u, st);
    if (rc) return rc;
    const int64_t dims[3] = {c->g.Du, c->g.Hu, c->g.Wu};
    rc = pot_weights_issue(img, dims, c->ndim, channels, c->conn, sigma, inv_dist, wq, ws, st);
    if (rc) return rc;
    rc = clear_status(c, st);
    if (!rc) rc = issue_set_unaries(c, u, st);
    if (!rc) rc = issue_set_weights(c, wq, st);
    if (ws_out) *ws_out = ws;
    return rc;
}

int dope_set_image(dope_ctx* c, const float* image, int channels, const dope_gmm* fg, const dope_gmm* bg,
                   double clip, double sigma, int inv_dist, int where, double* sigma_used, void* stream) {
    cudaStream_t st = S(stream);
    double* ws = nullptr;
    if (c) c->pending = false;   // both inputs are replaced
    int rc = image_issue(c, image, channels, fg, bg, clip, sigma, inv_dist, where, st, nullptr, &ws);
    if (rc) return rc;
    if (!sigma_used) {
        // asynchronous: the status is read by the next synchronising call
        c->have_u = c->have_w = 1;
        c->pending = true;
        return DOPE_OK;
    }
    double sig = sigma;
    if (!(sigma > 0.0)) CK(cudaMemcpyAsync(&sig, ws + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    Ctrl h{};
    rc = read_ctrl(c, &h, st);
    if (rc) return rc;
    if (sigma_used) *sigma_used = sig;
    c->have_u = c->have_w = (h.status == 0);
    return h.status;
}


int dope_reset(dope_ctx* c) {
    if (!c) return DOPE_EINVAL;
    return reset_state(c);
}

int dope_iterate(dope_ctx* c, int n_iter, int* iterations_done, int* converged, void* stream) {
    if (!c || n_iter < 0 || c->begun) return DOPE_EINVAL;
    c->launches = 0;
    int rc = run_iterations(c, n_iter, S(stream));
    if (rc) return rc;
    if (iterations_done) *iterations_done = c->t;
    if (converged) *converged = c->stats.converged;
    return DOPE_OK;
}

// A solve of this context is one persistent launch (the resident or the
// persistent kernel runs Algorithm 1 from its initial state to the labels).
static bool single_launch(const dope_ctx* c) {
    return !c->ov && !c->nsm && c->p.launch_mode != 1 && c->persist_grid > 0 && c->p.max_iter > 0;
}

// First half of a single-launch solve: clear the control block (keeping an
// asynchronous upload's status word), the launch, the labels copied out and
// the control block copied to pinned host memory.  No synchronisation.
static int solve_issue(dope_ctx* c, uint8_t* labels, int where, int want_energy, cudaStream_t st) {
    if (!c->hctrl && cudaMallocHost(&c->hctrl, c->ctrl_bytes) != cudaSuccess) {
        cudaGetLastError();
        c->hctrl = nullptr;
        return DOPE_ENOMEM;
    }
    c->t = 0;
    c->mu = c->p.mu0;
    c->sched_t = -1;
    const int n = c->p.max_iter;
    memset(&c->stats, 0, sizeof(c->stats));
    const bool pend = c->pending;
    c->begun_pend = pend;
    // on any failure below, a pending upload's status stays pending
    auto fail = [&](int rc) { c->pending = pend; c->begun_pend = false; return rc; };
    if (pend) {
        static_assert(offsetof(Ctrl, status) == sizeof(int), "status follows conv_t");
        if (cudaMemsetAsync(c->ctrl, 0, sizeof(int), st) != cudaSuccess ||
            cudaMemsetAsync((char*)c->ctrl + 2 * sizeof(int), 0,
                            sizeof(Ctrl) - sizeof(unsigned long long) - 2 * sizeof(int), st) != cudaSuccess) {
            cudaGetLastError();
            return fail(DOPE_ECUDA);
        }
    } else {
        const int rc0 = clear_status(c, st);
        if (rc0) return fail(rc0);
    }
    if (cudaMemsetAsync(&c->ctrl->r2max[1], 0, sizeof(unsigned long long) * (size_t)n, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(DOPE_ECUDA);
    }
    uint8_t* dst = labels;
    if (where == DOPE_HOST) {
        const int rc = ensure_stage(c, (size_t)c->g.Nu, 1);
        if (rc) return fail(rc);
        dst = (uint8_t*)c->stage2;
    }
    c->launches = 0;
    const int rc = persistent_issue(c, n, st, dst, want_energy);
    if (rc) return fail(rc);
    if ((where == DOPE_HOST &&
         cudaMemcpyAsync(labels, dst, (size_t)c->g.Nu, cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
        cudaMemcpyAsync(c->hctrl, c->ctrl, c->ctrl_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(DOPE_ECUDA);
    }
    c->pending = false;   // its status word is now read with the control block
    return DOPE_OK;
}

// Second half, once the stream has passed the copies: the results from the
// pinned control block.
static int solve_collect(dope_ctx* c, int64_t* energy_int, int* iterations, cudaStream_t st) {
    const bool pend = c->begun_pend;
    c->begun_pend = false;
    const int rc = persistent_collect(c, 0, *c->hctrl, c->hctrl->r2max, st);
    if (rc) {
        if (pend && (rc == DOPE_EINVAL || rc == DOPE_EUNSUPPORTED || rc == DOPE_EOVERFLOW))
            c->have_u = c->have_w = 0;   // the upload's error: its inputs are not usable
        return rc;
    }
    if (energy_int) *energy_int = (int64_t)c->hctrl->energy;
    c->stats.kernel_launches = c->launches;
    if (iterations) *iterations = c->t;
    return c->stats.converged ? DOPE_OK : DOPE_ENOTCONV;
}

int dope_solve(dope_ctx* c, uint8_t* labels, int where, int64_t* energy_int, int* iterations,
               void* stream) {
    if (!c || !labels || (where != DOPE_HOST && where != DOPE_DEVICE)) return DOPE_EINVAL;
    if (c->begun) return DOPE_EINVAL;   // a dope_solve_begin awaits its dope_solve_end
    if (!c->have_u || !c->have_w) return DOPE_EINVAL;
    cudaStream_t st = S(stream);
    if (c->ov) {
        c->launches = 0;
        int rc = ov_reset_async(c, st);
        if (!rc) rc = run_iterations(c, c->p.max_iter, st);
        uint8_t* dst = labels;
        if (!rc && where == DOPE_HOST) {
            rc = ensure_stage(c, (size_t)c->g.Nu, 1);
            dst = (uint8_t*)c->stage2;
        }
        if (!rc) rc = ov_finish(c, dst, energy_int, st);
        if (rc) return rc;
        if (where == DOPE_HOST) CK(cudaMemcpyAsync(labels, dst, (size_t)c->g.Nu, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        c->stats.kernel_launches = c->launches;
        if (iterations) *iterations = c->t;
        return c->stats.converged ? DOPE_OK : DOPE_ENOTCONV;
    }
    // Algorithm 1 initialisation: y = 1/2, a = 0, mu = mu0 (stream-ordered)
    c->t = 0;
    c->mu = c->p.mu0;
    c->sched_t = -1;
    c->launches = 1;
    const int threads = 256;
    if (single_launch(c)) {
        // one persistent launch that also starts from y = 1/2, a = 0 and
        // finishes with the labels and their energy, then one read of the whole
        // control block: a single launch and a single synchronisation per solve
        int rc = solve_issue(c, labels, where, energy_int ? 1 : 0, st);
        if (rc) return rc;
        CK(cudaStreamSynchronize(st));
        return solve_collect(c, energy_int, iterations, st);
    }
    k_init_state<<<grid_for((long long)c->g.K * c->g.F, threads), threads, 0, st>>>(c->g, c->yF, c->aF);
    CK(cudaGetLastError());
    int rc = run_iterations(c, c->p.max_iter, st);
    if (rc) return rc;
    if (energy_int) {
        rc = energy_of(c, c->yhat, energy_int, st);
        if (rc) return rc;
    }
    uint8_t* dst = labels;
    if (where == DOPE_HOST) {
        rc = ensure_stage(c, (size_t)c->g.Nu, 1);
        if (rc) return rc;
        dst = (uint8_t*)c->stage2;
    }
    k_unpermute_u8<<<grid_for(c->g.Nu, threads), threads, 0, st>>>(c->g, c->yhat, dst);
    c->launches++;
    CK(cudaGetLastError());
    if (where == DOPE_HOST) CK(cudaMemcpyAsync(labels, dst, (size_t)c->g.Nu, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    c->stats.kernel_launches = c->launches;
    if (iterations) *iterations = c->t;
    return c->stats.converged ? DOPE_OK : DOPE_ENOTCONV;
}

int dope_solve_begin(dope_ctx* c, uint8_t* labels, int where, void* stream) {
    if (!c || !labels || (where != DOPE_HOST && where != DOPE_DEVICE)) return DOPE_EINVAL;
    if (c->begun) return DOPE_EINVAL;
    if (!c->have_u || !c->have_w) return DOPE_EINVAL;
    cudaStream_t st = S(stream);
    if (single_launch(c)) {
        const int rc = solve_issue(c, labels, where, 1, st);
        if (rc) return rc;
        c->begun = 1;
        return DOPE_OK;
    }
    // other contexts solve here; dope_solve_end returns the outcome
    int64_t e = 0;
    int it = 0;
    c->sync_rc = dope_solve(c, labels, where, &e, &it, stream);
    c->sync_energy = e;
    c->sync_iters = it;
    c->begun = 2;
    return DOPE_OK;
}

int dope_solve_end(dope_ctx* c, int64_t* energy_int, int* iterations, void* stream) {
    if (!c || !c->begun) return DOPE_EINVAL;
    const int how = c->begun;
    c->begun = 0;
    if (how == 2) {
        if (energy_int) *energy_int = c->sync_energy;
        if (iterations) *iterations = c->sync_iters;
        return c->sync_rc;
    }
    cudaStream_t st = S(stream);
    CK(cudaStreamSynchronize(st));
    return solve_collect(c, energy_int, iterations, st);
}

int dope_get_state(dope_ctx* c, double* y, double* a, uint8_t* yhat, double* mu, int* t, void* stream) {
    if (!c) return DOPE_EINVAL;
    cudaStream_t st = S(stream);
    if (c->ov) {
        if (a || yhat) return DOPE_EINVAL;
        if (y) CK(cudaMemcpyAsync(y, c->oa.y, sizeof(double) * (size_t)c->oa.N, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (mu) *mu = c->mu;
        if (t) *t = c->t;
        return DOPE_OK;
    }
    const size_t N = (size_t)c->g.N;
    int rc = ensure_stage(c, N * 17, 1);
    if (rc) return rc;
    double* dy = (double*)c->stage2;
    double* da = dy + N;
    uint8_t* dh = (uint8_t*)(da + N);
    const int threads = 256;
    k_get_state<<<grid_for(c->g.N, threads), threads, 0, st>>>(c->g, c->yF, c->aF, c->yhat, c->faceIndex,
                                                               c->t, dy, da, dh);
    CK(cudaGetLastError());
    if (y) CK(cudaMemcpyAsync(y, dy, N * 8, cudaMemcpyDeviceToHost, st));
    if (a) CK(cudaMemcpyAsync(a, da, N * 8, cudaMemcpyDeviceToHost, st));
    if (yhat) CK(cudaMemcpyAsync(yhat, dh, N, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (mu) *mu = c->mu;
    if (t) *t = c->t;
    return DOPE_OK;
}

int dope_set_state(dope_ctx* c, const double* y, const double* a, const uint8_t* yhat, double mu,
                   int t, void* stream) {
    if (!c || !y || !a || !yhat || t < 0 || t > c->p.max_iter || !(mu > 0.0)) return DOPE_EINVAL;
    if (c->ov) return DOPE_EINVAL;
    cudaStream_t st = S(stream);
    settle_inputs(c, st);
    const size_t N = (size_t)c->g.N;
    int rc = ensure_stage(c, N * 17, 1);
    if (rc) return rc;
    double* dy = (double*)c->stage2;
    double* da = dy + N;
    uint8_t* dh = (uint8_t*)(da + N);
    CK(cudaMemcpyAsync(dy, y, N * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(da, a, N * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dh, yhat, N, cudaMemcpyHostToDevice, st));
    rc = clear_status(c, st);
    if (rc) return rc;
    const int threads = 256;
    k_set_state<<<grid_for(c->g.N, threads), threads, 0, st>>>(c->g, dy, da, dh, c->faceIndex, t, c->yF,
                                                               c->aF, c->yhat, c->ctrl);
    CK(cudaGetLastError());
    Ctrl h{};
    rc = read_ctrl(c, &h, st);
    if (rc) return rc;
    if (h.status) {
        reset_state(c);
        return h.status;
    }
    c->t = t;
    c->mu = mu;
    c->sched_t = -1;
    return DOPE_OK;
}

int dope_shifted_caps(dope_ctx* c, int64_t* C, void* stream) {
    if (!c || !C || !c->have_u || !c->have_w) return DOPE_EINVAL;
    if (c->ov) return DOPE_EINVAL;
    cudaStream_t st = S(stream);
    {
        const int rs = settle_inputs(c, st);
        if (rs) return rs;
    }
    const size_t N = (size_t)c->g.N;
    int rc = ensure_stage(c, N * 8, 1);
    if (rc) return rc;
    long long* d = (long long*)c->stage2;
    const int threads = 256;
    const int blocks = grid_for(c->g.N, threads);
    const int first = c->t == 0;
    if (c->conn == 4)
        k_shifted_caps<4><<<blocks, threads, 0, st>>>(c->g, c->U, c->Wl, c->yhat, c->yF, c->aF, c->faceIndex, first, c->mu, d);
    else if (c->conn == 8)
        k_shifted_caps<8><<<blocks, threads, 0, st>>>(c->g, c->U, c->Wl, c->yhat, c->yF, c->aF, c->faceIndex, first, c->mu, d);
    else
        k_shifted_caps<6><<<blocks, threads, 0, st>>>(c->g, c->U, c->Wl, c->yhat, c->yF, c->aF, c->faceIndex, first, c->mu, d);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(C, d, N * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return DOPE_OK;
}

int dope_block_cuts(dope_ctx* c, const int64_t* C, uint8_t* yhat, void* stream) {
    if (c) c->sched_t = -1;   // inputs or labels change: the worklists no longer hold
    if (!c || !C || !yhat || !c->have_w) return DOPE_EINVAL;
    if (c->ov || c->nsm) return DOPE_EINVAL;
    cudaStream_t st = S(stream);
    {
        const int rs = settle_inputs(c, st);
        if (rs) return rs;
    }
    const size_t N = (size_t)c->g.N;
    int rc = ensure_stage(c, N * 17, 1);
    if (rc) return rc;
    long long* cimg = (long long*)c->stage2;
    long long* cbm = cimg + N;
    uint8_t* lab = (uint8_t*)(cbm + N);
    // labels land in a scratch slab; the ADMM state is left untouched
    rc = ensure_stage(c, N, 0);
    if (rc) return rc;
    uint8_t* ybm = (uint8_t*)c->stage;
    CK(cudaMemcpyAsync(cimg, C, N * 8, cudaMemcpyHostToDevice, st));
    const int threads = 256;
    k_permute_i64<<<grid_for(c->g.N, threads), threads, 0, st>>>(c->g, cimg, cbm);
    rc = clear_status(c, st);
    if (rc) return rc;
    SolveArgs a = solve_args(c);
    a.Cgiven = cbm;
    a.yhat = ybm;
    a.check_prev = 0;
    solve_launch(c, a, st);
    k_unpermute_u8<<<grid_for(c->g.N, threads), threads, 0, st>>>(c->g, ybm, lab);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(yhat, lab, N, cudaMemcpyDeviceToHost, st));
    Ctrl h{};
    rc = read_ctrl(c, &h, st);
    if (rc) return rc;
    c->stats.pulses_total = (int64_t)h.pulses_total;
    c->stats.pulses_max = h.pulses_max;
    c->stats.free_nodes_total = (int64_t)h.free_total;
    return h.status;
}

int dope_energy(dope_ctx* c, const uint8_t* labels, int where, int64_t* energy_int, void* stream) {
    if (!c || !labels || !energy_int || !c->have_u || !c->have_w) return DOPE_EINVAL;
    cudaStream_t st = S(stream);
    {
        const int rs = settle_inputs(c, st);
        if (rs) return rs;
    }
    const size_t N = (size_t)c->g.N;
    int rc = ensure_stage(c, 2 * N, 1);
    if (rc) return rc;
    uint8_t* img = (uint8_t*)c->stage2;
    uint8_t* bm = img + N;
    const uint8_t* src = labels;
    if (where == DOPE_HOST) {
        CK(cudaMemcpyAsync(img, labels, N, cudaMemcpyHostToDevice, st));
        src = img;
    }
    const int threads = 256;
    if (c->ov) {
        CK(cudaMemsetAsync(&c->ctrl->energy, 0, sizeof(unsigned long long), st));
        const int blocks = grid_for(c->g.N, threads);
        const OvArgs& A = c->oa;
        if (!ov_dispatch(c->conn, [&](auto cc) {
                k_energy_img<decltype(cc)::value><<<blocks, threads, 0, st>>>(A.D, A.H, A.W, c->U, c->Wl, src, c->ctrl);
            }))
            big_energy_img(c->conn, A.D, A.H, A.W, c->U, c->Wl, src, c->ctrl, blocks, threads, st);
        CK(cudaGetLastError());
        unsigned long long v = 0;
        CK(cudaMemcpyAsync(&v, &c->ctrl->energy, sizeof(v), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        *energy_int = (int64_t)v;
        return DOPE_OK;
    }
    k_permute_u8<<<grid_for(c->g.N, threads), threads, 0, st>>>(c->g, src, bm);
    CK(cudaGetLastError());
    return energy_of(c, bm, energy_int, st);
}

int dope_trace(dope_ctx* c, double* rmax, int cap, int* count) {
    if (!c || (!rmax && cap > 0)) return DOPE_EINVAL;
    int n = c->t < cap ? c->t : cap;
    std::vector<unsigned long long> bits((size_t)n + 1);
    if (n > 0) {
        CK(cudaMemcpy(bits.data(), &c->ctrl->r2max[1], sizeof(unsigned long long) * (size_t)n,
                      cudaMemcpyDeviceToHost));
        for (int i = 0; i < n; ++i) {
            double r2;
            memcpy(&r2, &bits[(size_t)i], sizeof(r2));
            rmax[i] = std::sqrt(r2);
        }
    }
    if (count) *count = n;
    return DOPE_OK;
}

int dope_get_stats(dope_ctx* c, dope_stats* st) {
    if (!c || !st) return DOPE_EINVAL;
    *st = c->stats;
    return DOPE_OK;
}

int dope_set_profiling(dope_ctx* c, int enable) {
    if (!c) return DOPE_EINVAL;
    c->profiling = enable ? 1 : 0;
    memset(&c->prof, 0, sizeof(c->prof));
    return DOPE_OK;
}

int dope_get_profile(dope_ctx* c, dope_profile* out) {
    if (!c || !out) return DOPE_EINVAL;
    *out = c->prof;
    return DOPE_OK;
}

int dope_get_geometry(dope_ctx* c, int64_t* n_pixels, int64_t* n_blocks, int* block_volume, int* face_size) {
    if (!c) return DOPE_EINVAL;
    const Geo& g = c->ov ? c->oa.g : c->g;
    if (n_pixels) *n_pixels = c->g.N;
    if (n_blocks) *n_blocks = g.K;
    if (block_volume) *block_volume = g.B;
    if (face_size) *face_size = c->ov ? 0 : g.F;
    return DOPE_OK;
}

}  // extern "C"

int dope_image_upload_async(dope_ctx* c, const dope_image_request* q, int where, cudaStream_t st,
                            cudaEvent_t after_copies) {
    if (c) c->sched_t = -1;   // inputs change: the worklists no longer hold
    if (!c || !q) return DOPE_EINVAL;
    int rc = image_issue(c, q->image, q->channels, &q->fg, &q->bg, q->clip, q->sigma, q->inv_dist, where, st,
                         after_copies, nullptr);
    if (rc) return rc;
    c->have_u = c->have_w = 1;   // provisional until dope_ctx_status has read the status word
    return DOPE_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free solve (dope_solve_noalloc).
//
// For callers that must not allocate device memory: code that runs while a
// framework's caching allocator has reserved the GPU's memory, plugins whose
// host application forbids cudaMalloc after start-up, or latency-critical
// loops where an allocation (and the implicit synchronisation of cudaFree)
// is not acceptable.  All device state of one solve lives in the file-scope
// array below; every GPU that loads this library holds it until the process
// exits.  In host code `dope_noalloc_scratch` is only a host-side stand-in
// for the symbol: its device address is taken once per device with
// cudaGetSymbolAddress and passed to the kernels.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char dope_noalloc_scratch[DOPE_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES];     // device address of the array, once looked up

// Face slots of a block: pixels with a neighbour outside the block, numbered
// in increasing local index (same tables as dope_create builds on the host).
template <int CONN>
__global__ void k_face_tables(int bd, int bh, int bw, int16_t* faceIndex, int16_t* faceLocal,
                              int* halo) {
    __shared__ int warp_tot[32];
    __shared__ int running;
    const int B = bd * bh * bw;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) running = 0;
    __syncthreads();
    for (int base = 0; base < B; base += blockDim.x) {
        const int l = base + tid;
        bool face = false;
        if (l < B) {
            const int lx = l % bw, ly = (l / bw) % bh, lz = l / (bw * bh);
#pragma unroll
            for (int d = 0; d < CONN; ++d) {
                int dz, dy, dx;
                dir_off<CONN>(d, dz, dy, dx);
                const int z = lz + dz, y = ly + dy, x = lx + dx;
                if (z < 0 || z >= bd || y < 0 || y >= bh || x < 0 || x >= bw) face = true;
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, face);
        if (lane == 0) warp_tot[wid] = __popc(m);
        __syncthreads();
        int off = running;
        for (int w = 0; w < wid; ++w) off += warp_tot[w];
        if (l < B) {
            if (face) {
                const int slot = off + __popc(m & ((1u << lane) - 1u));
                faceIndex[l] = (int16_t)slot;
                faceLocal[slot] = (int16_t)l;
            } else {
                faceIndex[l] = -1;
            }
        }
        __syncthreads();
        if (tid == 0) {
            int tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += warp_tot[w];
            running += tot;
        }
        __syncthreads();
    }
    // halo table [CONN][F]
    const int F = running;
    for (int i = tid; i < CONN * F; i += blockDim.x) {
        const int d = i / F, f = i % F;
        const int l = faceLocal[f];
        const int lx = l % bw, ly = (l / bw) % bh, lz = l / (bw * bh);
        int dz, dy, dx;
        dir_off<CONN>(d, dz, dy, dx);
        int z = lz + dz, y = ly + dy, x = lx + dx;
        int e = -1;
        if (!(z >= 0 && z < bd && y >= 0 && y < bh && x >= 0 && x < bw)) {
            const int dkz = z < 0 ? -1 : (z >= bd ? 1 : 0);
            const int dky = y < 0 ? -1 : (y >= bh ? 1 : 0);
            const int dkx = x < 0 ? -1 : (x >= bw ? 1 : 0);
            z -= dkz * bd; y -= dky * bh; x -= dkx * bw;
            const int ln = (z * bh + y) * bw + x;
            e = halo_entry((dkz + 1) * 9 + (dky + 1) * 3 + (dkx + 1), ln, faceIndex[ln]);
        }
        halo[i] = e;
    }
}

// Per-device set-up: device address of the scratch array, with the device
// current.  Only a successful lookup is kept; a failed one (the module could
// not be loaded, e.g. no memory left for the array) clears the error state
// and is retried by the next call.
int noalloc_setup(int* dev_out, void** ptr_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return DOPE_ECUDA;
    }
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return DOPE_EINVAL;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, dope_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return DOPE_ECUDA;
        }
        g_noalloc_ptr[dev] = ptr;
    }
    *dev_out = dev;
    *ptr_out = g_noalloc_ptr[dev];
    return DOPE_OK;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// off += align256(bytes), false if that passes `limit` (every term is checked
// against the space left, so the sum cannot wrap)
inline bool take(size_t& off, size_t bytes, size_t limit) {
    if (off > limit || bytes > limit - off) return false;
    const size_t a = align256(bytes);
    if (a > limit - off) return false;
    off += a;
    return true;
}

}  // namespace

extern "C" int dope_solve_noalloc(const int64_t* grid, int ndim, int connectivity,
                                  const int32_t* block_shape, double lambda, const dope_params* p,
                                  const float* u, const int32_t* wq, uint8_t* labels,
                                  int64_t* energy_int, int* iterations, void* stream) {
    if (!grid || !block_shape || !u || !wq || !labels) return DOPE_EINVAL;
    if (ndim != 2 && ndim != 3) return DOPE_EINVAL;
    if (ndim == 2 && connectivity != 4 && connectivity != 8) return DOPE_EINVAL;
    if (ndim == 3 && connectivity != 6) return DOPE_EINVAL;
    if (!(lambda >= 0.0) || !std::isfinite(lambda)) return DOPE_EINVAL;
    int64_t dims[3] = {1, 1, 1};
    int32_t blk[3] = {1, 1, 1};
    for (int i = 0; i < ndim; ++i) {
        dims[3 - ndim + i] = grid[i];
        blk[3 - ndim + i] = block_shape[i];
    }
    for (int i = 0; i < 3; ++i) {
        if (dims[i] <= 0 || blk[i] <= 0 || dims[i] % blk[i] || dims[i] > (1LL << 30)) return DOPE_EINVAL;
    }
    const long long N = dims[0] * dims[1] * dims[2];
    const long long B = (long long)blk[0] * blk[1] * blk[2];
    if (N >= (1LL << 31) || B > 4096) return DOPE_EINVAL;
    dope_params prm;
    dope_default_params(&prm);
    if (p) prm = *p;
    if (!(prm.mu0 > 0.0)) prm.mu0 = (ndim == 3) ? 500.0 : 100.0;
    if (!(prm.mu_fact > 0.0)) prm.mu_fact = 1.05;
    if (!(prm.eps >= 0.0)) prm.eps = 1e-3;
    if (prm.max_iter <= 0) prm.max_iter = 1000;
    if (prm.relabel_period <= 0) prm.relabel_period = 8;
    if (prm.max_pulses <= 0) prm.max_pulses = (int)(64 * B + 4096);
    if (prm.fold_rounds <= 0) prm.fold_rounds = MAX_FOLD_ROUNDS;
    int threads = prm.threads;
    if (threads <= 0) {
        threads = (int)((B + 31) / 32 * 32);
        if (threads > 512) threads = 512;
        if (threads < 32) threads = 32;
    }
    if (threads % 32 || threads > 512 || (long long)threads * NPTMAX < B) return DOPE_EINVAL;

    Geo g;
    g.D = (int)dims[0]; g.H = (int)dims[1]; g.W = (int)dims[2];
    g.bd = blk[0]; g.bh = blk[1]; g.bw = blk[2];
    g.B = (int)B;
    g.nbz = g.D / g.bd; g.nby = g.H / g.bh; g.nbx = g.W / g.bw;
    g.K = g.nbz * g.nby * g.nbx;
    g.N = N;
    g.Du = g.D; g.Hu = g.H; g.Wu = g.W;
    g.Nu = N;
    {   // face count (interior = (bd-2)(bh-2)(bw-2)-style box of the connectivity)
        const int iz = (connectivity == 6) ? (g.bd > 2 ? g.bd - 2 : 0) : g.bd;
        const int iy = g.bh > 2 ? g.bh - 2 : 0, ix = g.bw > 2 ? g.bw - 2 : 0;
        g.F = (int)(B - (long long)iz * iy * ix);
    }
    const int nh = connectivity / 2;

    // scratch layout (every term checked against the space left)
    const size_t LIM = (size_t)DOPE_NOALLOC_SCRATCH_BYTES;
    if ((size_t)prm.max_iter > LIM / sizeof(unsigned long long)) return DOPE_EINVAL;
    const size_t ctrl_bytes = sizeof(Ctrl) + sizeof(unsigned long long) * ((size_t)prm.max_iter + 2);
    size_t off = 0;
    const size_t o_ctrl = off;  if (!take(off, ctrl_bytes, LIM)) return DOPE_EINVAL;
    const size_t o_U = off;     if (!take(off, sizeof(int32_t) * (size_t)N, LIM)) return DOPE_EINVAL;
    const size_t o_Wl = off;    if (!take(off, sizeof(int32_t) * (size_t)N * nh, LIM)) return DOPE_EINVAL;
    const size_t o_yhat = off;  if (!take(off, (size_t)N, LIM)) return DOPE_EINVAL;
    const size_t o_yF = off;    if (!take(off, sizeof(double) * (size_t)g.K * g.F, LIM)) return DOPE_EINVAL;
    const size_t o_aF = off;    if (!take(off, sizeof(double) * (size_t)g.K * g.F, LIM)) return DOPE_EINVAL;
    const size_t o_r2 = off;    if (!take(off, sizeof(double) * (size_t)g.K, LIM)) return DOPE_EINVAL;
    const size_t o_fi = off;    if (!take(off, sizeof(int16_t) * (size_t)B, LIM)) return DOPE_EINVAL;
    const size_t o_fl = off;    if (!take(off, sizeof(int16_t) * (size_t)(g.F ? g.F : 1), LIM)) return DOPE_EINVAL;
    const size_t o_halo = off;
    if (!take(off, sizeof(int) * (size_t)connectivity * (g.F ? g.F : 1), LIM)) return DOPE_EINVAL;

    int dev = 0;
    void* base = nullptr;
    int rc = noalloc_setup(&dev, &base);
    if (rc) return rc;
    unsigned char* sb = static_cast<unsigned char*>(base);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(sb + o_ctrl);
    int32_t* U = reinterpret_cast<int32_t*>(sb + o_U);
    int32_t* Wl = reinterpret_cast<int32_t*>(sb + o_Wl);
    uint8_t* yhat = sb + o_yhat;
    double* yF = reinterpret_cast<double*>(sb + o_yF);
    double* aF = reinterpret_cast<double*>(sb + o_aF);
    double* r2blk = reinterpret_cast<double*>(sb + o_r2);
    int16_t* faceIndex = reinterpret_cast<int16_t*>(sb + o_fi);
    int16_t* faceLocal = reinterpret_cast<int16_t*>(sb + o_fl);
    int* halo = reinterpret_cast<int*>(sb + o_halo);
    cudaStream_t st = S(stream);
    const int smem = (int)solver_smem_bytes(connectivity, (int)B);

    // everything that must start at zero: the control word and the trace
    CK(cudaMemsetAsync(ctrl, 0, ctrl_bytes, st));
    if (connectivity == 4) {
        raise_smem_limits<4>();
        k_face_tables<4><<<1, 1024, 0, st>>>(g.bd, g.bh, g.bw, faceIndex, faceLocal, halo);
    } else if (connectivity == 8) {
        raise_smem_limits<8>();
        k_face_tables<8><<<1, 1024, 0, st>>>(g.bd, g.bh, g.bw, faceIndex, faceLocal, halo);
    } else {
        raise_smem_limits<6>();
        k_face_tables<6><<<1, 1024, 0, st>>>(g.bd, g.bh, g.bw, faceIndex, faceLocal, halo);
    }
    const int tpb = 256;
    k_set_unaries<<<grid_for(N, tpb), tpb, 0, st>>>(g, u, U, ctrl);
    if (connectivity == 4) k_set_weights<4><<<grid_for(N, tpb), tpb, 0, st>>>(g, wq, Wl, lambda, ctrl, 0);
    else if (connectivity == 8) k_set_weights<8><<<grid_for(N, tpb), tpb, 0, st>>>(g, wq, Wl, lambda, ctrl, 0);
    else k_set_weights<6><<<grid_for(N, tpb), tpb, 0, st>>>(g, wq, Wl, lambda, ctrl, 0);
    k_init_state<<<grid_for((long long)g.K * g.F, tpb), tpb, 0, st>>>(g, yF, aF);
    CK(cudaGetLastError());
    Ctrl h{};
    CK(cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl) - sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h.status) return h.status;

    // Algorithm 1, batches of iterations with the device-side stop test
    SolveArgs sa;
    sa.g = g; sa.U = U; sa.Wl = Wl; sa.yhat = yhat; sa.yF = yF; sa.aF = aF;
    sa.faceIndex = faceIndex; sa.halo = halo; sa.faceLocal = faceLocal; sa.Cgiven = nullptr; sa.ctrl = ctrl; sa.eps = prm.eps;
    sa.relabel_period = prm.relabel_period; sa.max_pulses = prm.max_pulses;
    sa.fold_rounds = prm.fold_rounds;
    UpdArgs ua;
    ua.g = g; ua.Wl = Wl; ua.yhat = yhat; ua.yF = yF; ua.aF = aF; ua.r2blk = r2blk;
    ua.faceLocal = faceLocal; ua.faceIndex = faceIndex; ua.halo = halo; ua.ctrl = ctrl;
    const int uthreads = face_update_threads(g.F);
    double mu = prm.mu0;
    int launched = 0, batch = 4;
    while (launched < prm.max_iter) {
        const int nb = (prm.max_iter - launched < batch) ? prm.max_iter - launched : batch;
        for (int j = 0; j < nb; ++j) {
            const int t = launched + j + 1;
            sa.t = t; set_mu(sa, mu); sa.first = (t == 1); sa.check_prev = (t > 1);
            ua.t = t; ua.mu = mu;
            if (connectivity == 4) {
                k_block_solve<4><<<g.K, threads, smem, st>>>(sa);
                k_face_update<4><<<g.K, uthreads, 0, st>>>(ua);
            } else if (connectivity == 8) {
                k_block_solve<8><<<g.K, threads, smem, st>>>(sa);
                k_face_update<8><<<g.K, uthreads, 0, st>>>(ua);
            } else {
                k_block_solve<6><<<g.K, threads, smem, st>>>(sa);
                k_face_update<6><<<g.K, uthreads, 0, st>>>(ua);
            }
            mu = mu * prm.mu_fact;
        }
        CK(cudaGetLastError());
        launched += nb;
        CK(cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl) - sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (h.status) return h.status;
        if (h.conv_t) break;
        if (batch < 32) batch *= 2;
    }
    int done = launched, converged = 0;
    if (h.conv_t) {
        done = h.conv_t;
        converged = 1;
    } else {
        unsigned long long bits = 0;
        CK(cudaMemcpyAsync(&bits, &ctrl->r2max[done], sizeof(bits), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        double r2;
        memcpy(&r2, &bits, sizeof(r2));
        converged = !(std::sqrt(r2) > prm.eps);
    }
    if (energy_int) {
        CK(cudaMemsetAsync(&ctrl->energy, 0, sizeof(unsigned long long), st));
        if (connectivity == 4) k_energy<4><<<grid_for(N, tpb), tpb, 0, st>>>(g, U, Wl, yhat, ctrl);
        else if (connectivity == 8) k_energy<8><<<grid_for(N, tpb), tpb, 0, st>>>(g, U, Wl, yhat, ctrl);
        else k_energy<6><<<grid_for(N, tpb), tpb, 0, st>>>(g, U, Wl, yhat, ctrl);
    }
    k_unpermute_u8<<<grid_for(N, tpb), tpb, 0, st>>>(g, yhat, labels);
    CK(cudaGetLastError());
    unsigned long long e = 0;
    if (energy_int) CK(cudaMemcpyAsync(&e, &ctrl->energy, sizeof(e), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (energy_int) *energy_int = (int64_t)e;
    if (iterations) *iterations = done;
    return converged ? DOPE_OK : DOPE_ENOTCONV;
}

// ---------------------------------------------------------------------------
// Stream-ordered pieces used by the request server, and the batched launch.
// ---------------------------------------------------------------------------
int dope_upload_async(dope_ctx* c, const float* u, const int32_t* wq, int where, cudaStream_t st,
                      cudaEvent_t after_copies) {
    if (c) c->sched_t = -1;   // inputs or labels change: the worklists no longer hold
    if (!c || !u || !wq || (where != DOPE_HOST && where != DOPE_DEVICE)) return DOPE_EINVAL;
    const size_t n = (size_t)c->g.Nu;
    const int nh = c->conn / 2;
    const float* su = u;
    const int32_t* sw = wq;
    if (where == DOPE_HOST) {
        int rc = ensure_stage(c, sizeof(float) * n + sizeof(int32_t) * n * nh, 0);
        if (rc) return rc;
        float* du = (float*)c->stage;
        int32_t* dw = (int32_t*)(du + n);
        CK(cudaMemcpyAsync(du, u, sizeof(float) * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dw, wq, sizeof(int32_t) * n * nh, cudaMemcpyHostToDevice, st));
        su = du;
        sw = dw;
    }
    if (after_copies) CK(cudaEventRecord(after_copies, st));
    int rc = clear_status(c, st);
    if (rc) return rc;
    const int threads = 256;
    const int blocks = grid_for(c->g.N, threads);
    k_set_unaries<<<blocks, threads, 0, st>>>(c->g, su, c->U, c->ctrl);
    if (c->conn == 4) k_set_weights<4><<<blocks, threads, 0, st>>>(c->g, sw, c->Wl, c->lambda, c->ctrl, c->nsm);
    else if (c->conn == 8) k_set_weights<8><<<blocks, threads, 0, st>>>(c->g, sw, c->Wl, c->lambda, c->ctrl, c->nsm);
    else k_set_weights<6><<<blocks, threads, 0, st>>>(c->g, sw, c->Wl, c->lambda, c->ctrl, c->nsm);
    CK(cudaGetLastError());
    c->have_u = c->have_w = 1;   // provisional until dope_ctx_status has read the status word
    return DOPE_OK;
}

int dope_ctx_status(dope_ctx* c, int* status, cudaStream_t st) {
    if (!c || !status) return DOPE_EINVAL;
    Ctrl h{};
    int rc = read_ctrl(c, &h, st);
    if (rc) return rc;
    *status = h.status;
    if (h.status) c->have_u = c->have_w = 0;
    return DOPE_OK;
}

int dope_status_async(dope_ctx* c, int* status_pinned, cudaStream_t st) {
    if (!c || !status_pinned) return DOPE_EINVAL;
    CK(cudaMemcpyAsync(status_pinned, &c->ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    return DOPE_OK;
}

int dope_ctx_max_iter(const dope_ctx* c) { return c ? c->p.max_iter : 0; }

void dope_release_staging(dope_ctx* c) {
    if (!c) return;
    dfree(c->al, c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
}

size_t dope_ctx_device_bytes(const dope_ctx* c) {
    if (!c) return 0;
    const size_t N = (size_t)c->g.N, KF = (size_t)c->g.K * c->g.F;
    return N * 4 + N * 4 * (size_t)(c->conn / 2) + N + 16 * KF + 8 * (size_t)c->g.K + c->ctrl_bytes +
           (c->sched ? sched_bytes(c->g.K, c->g.F) : 0) + c->stage_bytes + c->stage2_bytes +
           (c->wslot ? (40 * KF + 8 * (size_t)c->g.K + 4 * CHUNK_WORDS * (size_t)c->g.K) : 0);
}

int64_t dope_ctx_pixels(const dope_ctx* c) { return c ? (int64_t)c->g.Nu : 0; }

int dope_iterations(const dope_ctx* c, int* t, int* converged) {
    if (!c) return DOPE_EINVAL;
    if (t) *t = c->t;
    if (converged) *converged = c->stats.converged;
    return DOPE_OK;
}

int dope_finish_async(dope_ctx* c, uint8_t* labels_dev, int64_t* energy_pinned, cudaStream_t st) {
    if (!c || !labels_dev) return DOPE_EINVAL;
    const int threads = 256;
    if (energy_pinned) {
        CK(cudaMemsetAsync(&c->ctrl->energy, 0, sizeof(unsigned long long), st));
        const int blocks = grid_for(c->g.N, threads);
        if (c->conn == 4) k_energy<4><<<blocks, threads, 0, st>>>(c->g, c->U, c->Wl, c->yhat, c->ctrl);
        else if (c->conn == 8) k_energy<8><<<blocks, threads, 0, st>>>(c->g, c->U, c->Wl, c->yhat, c->ctrl);
        else k_energy<6><<<blocks, threads, 0, st>>>(c->g, c->U, c->Wl, c->yhat, c->ctrl);
        CK(cudaMemcpyAsync(energy_pinned, &c->ctrl->energy, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    }
    k_unpermute_u8<<<grid_for(c->g.Nu, threads), threads, 0, st>>>(c->g, c->yhat, labels_dev);
    CK(cudaGetLastError());
    return DOPE_OK;
}

struct dope_batch_ws {
    BatchDesc* hdesc = nullptr;   // pinned; copied to the constant table c_batch
    BatchProb* hprob = nullptr;   // pinned
    BatchProb* dprob = nullptr;
    BatchOut* hout = nullptr;     // pinned
    BatchOut* dout = nullptr;
    Ctrl* bc = nullptr;
    int* hstatus = nullptr;       // pinned copy of the launch's status word
    int n = 0;                    // problems of the launch in flight
    int threads = 0, smem = 0, grid = 0;
    bool holds_table = false;     // this workspace's launch owns c_batch until collected
};

namespace {
// c_batch is one table per process: one batched launch in flight at a time.
// Taken by dope_batch_launch, given back by dope_batch_collect (or when the
// workspace is destroyed), possibly from another thread: a binary semaphore.
std::mutex g_table_m;
std::condition_variable g_table_cv;
bool g_table_busy = false;

void table_acquire() {
    std::unique_lock<std::mutex> lk(g_table_m);
    g_table_cv.wait(lk, [] { return !g_table_busy; });
    g_table_busy = true;
}

void table_release() {
    {
        std::lock_guard<std::mutex> lk(g_table_m);
        g_table_busy = false;
    }
    g_table_cv.notify_one();
}
}  // namespace

int dope_batch_ws_create(dope_batch_ws** out) {
    if (!out) return DOPE_EINVAL;
    *out = nullptr;
    dope_batch_ws* w = new (std::nothrow) dope_batch_ws();
    if (!w) return DOPE_ENOMEM;
    if (cudaMallocHost(&w->hdesc, sizeof(BatchDesc) * BATCH_MAX) != cudaSuccess ||
        cudaMallocHost(&w->hprob, sizeof(BatchProb) * BATCH_MAX) != cudaSuccess ||
        cudaMalloc(&w->dprob, sizeof(BatchProb) * BATCH_MAX) != cudaSuccess ||
        cudaMallocHost(&w->hout, sizeof(BatchOut) * BATCH_MAX) != cudaSuccess ||
        cudaMalloc(&w->dout, sizeof(BatchOut) * BATCH_MAX) != cudaSuccess ||
        cudaMalloc(&w->bc, sizeof(Ctrl)) != cudaSuccess ||
        cudaMallocHost(&w->hstatus, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        dope_batch_ws_destroy(w);
        return DOPE_ENOMEM;
    }
    *out = w;
    return DOPE_OK;
}

void dope_batch_ws_destroy(dope_batch_ws* w) {
    if (!w) return;
    if (w->holds_table) {
        w->holds_table = false;
        table_release();
    }
    cudaFreeHost(w->hdesc);
    cudaFreeHost(w->hprob);
    cudaFree(w->dprob);
    cudaFreeHost(w->hout);
    cudaFree(w->dout);
    cudaFree(w->bc);
    cudaFreeHost(w->hstatus);
    delete w;
}

namespace {

// Co-resident CTAs per SM of k_admm_batch for (threads, dynamic smem), cached.
int batch_per_sm(int threads, int smem) {
    static std::mutex mu;
    static std::vector<int> keys, vals;
    std::lock_guard<std::mutex> lk(mu);
    const int key = threads * (1 << 20) + smem;
    for (size_t i = 0; i < keys.size(); ++i)
        if (keys[i] == key) return vals[i];
    int dev = 0, optin = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, batch_fn(threads)) != cudaSuccess ||
        (size_t)smem + fa.sharedSizeBytes > (size_t)optin ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_fn(threads), threads, smem) !=
            cudaSuccess)
        per_sm = 0;
    cudaGetLastError();
    keys.push_back(key);
    vals.push_back(per_sm);
    return per_sm;
}

}  // namespace

int dope_batch_launch(dope_ctx* const* cs, int n, int n_iter, int exit_on_done, int clear_status,
                      const int* yield_flag, dope_batch_ws* w, cudaStream_t st) {
    if (!cs || n < 1 || n > BATCH_MAX || !w || n_iter < 0) return DOPE_EINVAL;
    int threads = 32, smem = 0;
    long long total = 0;
    for (int i = 0; i < n; ++i) {
        dope_ctx* c = cs[i];
        if (!c || !c->have_u || !c->have_w || c->ov || c->nsm) return DOPE_EINVAL;
        for (int j = 0; j < i; ++j)
            if (cs[j] == c) return DOPE_EINVAL;
        const int width = solver_width(c->g.B, c->threads);
        if (width > threads) threads = width;
        if (c->smem > smem) smem = c->smem;
        total += c->g.K;
        BatchDesc& d = w->hdesc[i];
        d.g = c->g;
        d.U = c->U;
        d.Wl = c->Wl;
        d.yhat = c->yhat;
        d.yF = c->yF;
        d.aF = c->aF;
        d.r2blk = c->r2blk;
        d.faceIndex = c->faceIndex;
        d.halo = c->halo;
        d.faceLocal = c->faceLocal;
        d.Cgiven = nullptr;
        d.ctrl = c->ctrl;
        d.eps = c->p.eps;
        d.relabel_period = c->p.relabel_period;
        d.max_pulses = c->p.max_pulses;
        d.fold_rounds = c->p.fold_rounds;
        d.conn = c->conn;
        d.sched = nullptr;
        d.epoch = 0;
        BatchProb& b = w->hprob[i];
        b.cont = 0;
        c->sched_launch = false;
        if (c->sched && c->p.mu_fact >= 1.0) {
            // worklists (see k_admm_batch); each launch's marks carry a new
            // epoch, and a launch that continues this context's previous list
            // launch from the state it left starts from its lists
            d.sched = c->sched;
            d.epoch = ++c->sched_epoch;
            b.cont = (c->t > 0 && c->sched_t == c->t) ? 1 : 0;
            c->sched_launch = true;
        }
        c->sched_t = -1;
        b.t0 = c->t;
        const int left = c->p.max_iter - c->t;
        b.n = n_iter < left ? n_iter : left;
        if (b.n < 0) b.n = 0;
        b.K = c->g.K;
        b.mu = c->mu;
        b.mu_fact = c->p.mu_fact;
    }
    raise_all_smem_limits(cs[0]->conn);
    int dev = 0, sms = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    const int per_sm = batch_per_sm(threads, smem);
    if (!coop || per_sm <= 0) return DOPE_EUNSUPPORTED;
    long long grid = (long long)per_sm * sms;
    if (grid > total) grid = total;
    if (grid < 1) grid = 1;
    BatchArgs P;
    P.probs = w->dprob;
    P.out = w->dout;
    P.nprob = n;
    P.exit_on_done = exit_on_done ? 1 : 0;
    P.yield_flag = yield_flag;
    P.bc = w->bc;
    P.spin_limit = 4000000000LL;   // about 2 s at the GB300 clock
    if (w->holds_table) return DOPE_EINVAL;   // previous launch not collected
    table_acquire();
    w->holds_table = true;
    cudaError_t e = cudaMemcpyToSymbolAsync(c_batch, w->hdesc, sizeof(BatchDesc) * (size_t)n, 0,
                                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w->dprob, w->hprob, sizeof(BatchProb) * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_batch_prep<<<n, 128, 0, st>>>(P, clear_status ? 1 : 0);
        e = cudaGetLastError();
    }
    void* args[] = {&P};
    if (e == cudaSuccess) e = cudaLaunchCooperativeKernel(batch_fn(threads), (int)grid, threads, args, smem, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w->hout, w->dout, sizeof(BatchOut) * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w->hstatus, &w->bc->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(st);   // nothing may still read the table
        w->holds_table = false;
        table_release();
        return DOPE_ECUDA;
    }
    for (int i = 0; i < n; ++i) cs[i]->launches += 2;
    w->n = n;
    w->threads = threads;
    w->smem = smem;
    w->grid = (int)grid;
    return DOPE_OK;
}

int dope_batch_collect(dope_ctx* const* cs, int n, dope_batch_ws* w, int* t, int* conv, int* status) {
    if (!cs || !w || n != w->n) return DOPE_EINVAL;
    if (w->holds_table) {
        w->holds_table = false;
        table_release();
    }
    const int launch_status = *w->hstatus;
    for (int i = 0; i < n; ++i) {
        dope_ctx* c = cs[i];
        const BatchOut& o = w->hout[i];
        c->t = o.t;
        c->mu = o.mu;
        c->sched_t = (c->sched_launch && o.status == 0 && launch_status == 0) ? o.t : -1;
        memset(&c->stats, 0, sizeof(c->stats));
        c->stats.iterations = o.t;
        c->stats.converged = o.conv;
        c->stats.rmax_last = std::sqrt(o.r2);
        c->stats.kernel_launches = c->launches;
        c->stats.solver_kernel = 3;
        c->stats.blocks_solved = (int64_t)o.work[0];
        c->stats.blocks_updated = (int64_t)o.work[1];
        if (t) t[i] = o.t;
        if (conv) conv[i] = o.conv;
        if (status) status[i] = o.status;
    }
    w->n = 0;
    return *w->hstatus;
}

namespace {
std::mutex g_batch_mu;
dope_batch_ws* g_batch_ws[NOALLOC_MAX_DEVICES];
}  // namespace

extern "C" int dope_iterate_batch(dope_ctx* const* ctxs, int n, int n_iter, int* iterations,
                                  int* converged, int* status, void* stream) {
    if (!ctxs || n < 1 || n > DOPE_BATCH_MAX || n_iter < 0) return DOPE_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return DOPE_ECUDA;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    if (!g_batch_ws[dev]) {
        int rc = dope_batch_ws_create(&g_batch_ws[dev]);
        if (rc) return rc;
    }
    dope_batch_ws* w = g_batch_ws[dev];
    cudaStream_t st = S(stream);
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) continue;
        const int rs = settle_inputs(ctxs[i], st);
        if (rs) return rs;
        ctxs[i]->launches = 0;
    }
    int rc = dope_batch_launch(ctxs, n, n_iter, 0, 1, nullptr, w, st);
    if (rc) return rc;
    CK(cudaStreamSynchronize(st));
    std::vector<int> sts((size_t)n, 0);
    rc = dope_batch_collect(ctxs, n, w, iterations, converged, sts.data());
    if (status)
        for (int i = 0; i < n; ++i) status[i] = sts[(size_t)i];
    if (rc) return rc;
    for (int i = 0; i < n; ++i)
        if (sts[(size_t)i]) return sts[(size_t)i];
    return DOPE_OK;
}

extern "C" int dope_labels(dope_ctx* c, uint8_t* labels, int where, int64_t* energy_int, void* stream) {
    if (!c || !labels || (where != DOPE_HOST && where != DOPE_DEVICE)) return DOPE_EINVAL;
    cudaStream_t st = S(stream);
    int rc = settle_inputs(c, st);
    if (rc) return rc;
    if (!c->have_u || !c->have_w) return DOPE_EINVAL;
    if (c->ov) {
        uint8_t* dst = labels;
        if (where == DOPE_HOST) {
            rc = ensure_stage(c, (size_t)c->g.Nu, 1);
            if (rc) return rc;
            dst = (uint8_t*)c->stage2;
        }
        rc = ov_finish(c, dst, energy_int, st);
        if (rc) return rc;
        if (where == DOPE_HOST) CK(cudaMemcpyAsync(labels, dst, (size_t)c->g.Nu, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return DOPE_OK;
    }
    if (energy_int) {
        rc = energy_of(c, c->yhat, energy_int, st);
        if (rc) return rc;
    }
    uint8_t* dst = labels;
    if (where == DOPE_HOST) {
        rc = ensure_stage(c, (size_t)c->g.Nu, 1);
        if (rc) return rc;
        dst = (uint8_t*)c->stage2;
    }
    const int threads = 256;
    k_unpermute_u8<<<grid_for(c->g.Nu, threads), threads, 0, st>>>(c->g, c->yhat, dst);
    CK(cudaGetLastError());
    if (where == DOPE_HOST) CK(cudaMemcpyAsync(labels, dst, (size_t)c->g.Nu, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return DOPE_OK;
}

int dope_run_single(dope_ctx* c, cudaStream_t st, int* t, int* conv) {
    if (!c) return DOPE_EINVAL;
    c->launches = 0;
    int rc = run_iterations(c, c->p.max_iter - c->t, st);
    if (t) *t = c->t;
    if (conv) *conv = c->stats.converged;
    return rc;
}

// ---------------------------------------------------------------------------
// Autotuner (dope_autotune): stage-wise search over solver settings.
// ---------------------------------------------------------------------------
namespace {

struct TuneRun {
    const int64_t* grid;
    int ndim, conn;
    double lambda;
    const float* u;          // device
    const int32_t* wq;       // device
    int reps;
    cudaStream_t st;
    uint8_t* lab;            // device, N
    cudaEvent_t e0, e1;
};

// One candidate: create, load, warm up, time `reps` solves.
void tune_one(const TuneRun& R, const int32_t* blk, const dope_params& prm, dope_tune_result* r) {
    memset(r, 0, sizeof(*r));
    for (int i = 0; i < R.ndim; ++i) r->block_shape[i] = blk[i];
    r->params = prm;
    r->ms = -1.0;
    dope_ctx* c = nullptr;
    int rc = dope_create(R.grid, R.ndim, R.conn, blk, R.lambda, &prm, &c);
    if (!rc) rc = dope_set_unaries(c, R.u, c->g.Nu, DOPE_DEVICE, R.st);
    if (!rc) rc = dope_set_weights(c, R.wq, c->g.Nu, DOPE_DEVICE, R.st);
    int64_t e = 0;
    int it = 0;
    if (!rc) {
        rc = dope_solve(c, R.lab, DOPE_DEVICE, &e, &it, R.st);
        if (rc == DOPE_ENOTCONV) rc = DOPE_OK;
    }
    double best = -1.0;
    for (int k = 0; !rc && k < R.reps; ++k) {
        cudaEventRecord(R.e0, R.st);
        rc = dope_solve(c, R.lab, DOPE_DEVICE, &e, &it, R.st);
        cudaEventRecord(R.e1, R.st);
        cudaEventSynchronize(R.e1);
        if (rc == DOPE_ENOTCONV) rc = DOPE_OK;
        float ms = 0.f;
        if (!rc && cudaEventElapsedTime(&ms, R.e0, R.e1) == cudaSuccess && (best < 0 || ms < best)) best = ms;
    }
    cudaGetLastError();
    if (c) {
        r->converged = c->stats.converged;
        dope_destroy(c);
    }
    r->status = rc;
    r->ms = best;
    r->iterations = it;
    r->energy_int = e;
}

bool tune_better(const dope_tune_result& a, const dope_tune_result& b) {
    if (a.status || !a.converged || a.ms < 0) return false;
    if (b.status || !b.converged || b.ms < 0) return true;
    return a.ms < b.ms;
}

}  // namespace

extern "C" int dope_autotune(const int64_t* grid, int ndim, int connectivity, const int32_t* block_shape,
                             double lambda, const dope_params* base, const float* u, const int32_t* wq,
                             int where, int flags, int reps, dope_tune_result* out, int cap, int* count,
                             dope_tune_result* best, void* stream) {
    if (!grid || !block_shape || !u || !wq || !best || (where != DOPE_HOST && where != DOPE_DEVICE) ||
        (ndim != 2 && ndim != 3) || reps < 1 || cap < 0 || (cap > 0 && !out))
        return DOPE_EINVAL;
    long long n = 1;
    for (int i = 0; i < ndim; ++i) {
        if (grid[i] <= 0) return DOPE_EINVAL;
        n *= grid[i];
    }
    const int nh = connectivity / 2;
    if (nh < 2 || nh > 4) return DOPE_EINVAL;
    dope_params prm0;
    dope_default_params(&prm0);
    if (base) prm0 = *base;
    cudaStream_t st = S(stream);
    TuneRun R;
    R.grid = grid;
    R.ndim = ndim;
    R.conn = connectivity;
    R.lambda = lambda;
    R.reps = reps;
    R.st = st;
    void* du = nullptr;
    void* dw = nullptr;
    void* dl = nullptr;
    if (cudaMalloc(&dl, (size_t)n) != cudaSuccess) { cudaGetLastError(); return DOPE_ENOMEM; }
    R.lab = (uint8_t*)dl;
    if (where == DOPE_HOST) {
        if (cudaMalloc(&du, sizeof(float) * (size_t)n) != cudaSuccess ||
            cudaMalloc(&dw, sizeof(int32_t) * (size_t)n * nh) != cudaSuccess ||
            cudaMemcpyAsync(du, u, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(dw, wq, sizeof(int32_t) * (size_t)n * nh, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(du); cudaFree(dw); cudaFree(dl);
            return DOPE_ENOMEM;
        }
        R.u = (const float*)du;
        R.wq = (const int32_t*)dw;
    } else {
        R.u = u;
        R.wq = wq;
    }
    cudaEventCreate(&R.e0);
    cudaEventCreate(&R.e1);
    int nout = 0;
    auto record = [&](const dope_tune_result& r) {
        if (nout < cap) out[nout] = r;
        ++nout;
    };
    int32_t blk[3] = {1, 1, 1};
    for (int i = 0; i < ndim; ++i) blk[i] = block_shape[i];
    dope_tune_result cur;
    tune_one(R, blk, prm0, &cur);
    record(cur);
    // stage 1: block shapes tiling the grid
    if (flags & DOPE_TUNE_BLOCK) {
        static const int S2[] = {8, 16, 32, 64};
        static const int S3[] = {4, 8, 16, 32};
        std::vector<std::vector<int32_t>> cands;
        if (ndim == 2) {
            for (int by : S2)
                for (int bx : S2)
                    if (by * bx >= 64 && by * bx <= 4096 && grid[0] % by == 0 && grid[1] % bx == 0)
                        cands.push_back({by, bx, 1});
        } else {
            for (int bz : S3)
                for (int by : S3)
                    for (int bx : S3)
                        if (bz * by * bx >= 256 && bz * by * bx <= 4096 && grid[0] % bz == 0 &&
                            grid[1] % by == 0 && grid[2] % bx == 0)
                            cands.push_back({bz, by, bx});
        }
        for (auto& b : cands) {
            bool same = true;
            for (int i = 0; i < ndim; ++i) same = same && b[(size_t)i] == blk[i];
            if (same) continue;
            dope_tune_result r;
            tune_one(R, b.data(), prm0, &r);
            record(r);
            if (tune_better(r, cur)) cur = r;
        }
        for (int i = 0; i < ndim; ++i) blk[i] = cur.block_shape[i];
    }
    // stages 2-5: settings that leave the labels unchanged
    const int relabels[] = {2, 4, 8, 16, 32};
    const int widths[] = {0, 256, 512};
    const int folds[] = {1, 2, 3, 4};
    const int modes[] = {0, 2};
    for (int stage = 0; stage < 4; ++stage) {
        const int* vals = stage == 0 ? relabels : stage == 1 ? widths : stage == 2 ? folds : modes;
        const int nv = stage == 0 ? 5 : stage == 1 ? 3 : stage == 2 ? 4 : 2;
        const dope_params start = cur.params;
        for (int v = 0; v < nv; ++v) {
            dope_params q = start;
            if (stage == 0) { if (q.relabel_period == vals[v] || (q.relabel_period == 0 && vals[v] == 8)) continue; q.relabel_period = vals[v]; }
            if (stage == 1) { if (q.threads == vals[v]) continue; q.threads = vals[v]; }
            if (stage == 2) { if (q.fold_rounds == vals[v] || (q.fold_rounds == 0 && vals[v] == 3)) continue; q.fold_rounds = vals[v]; }
            if (stage == 3) { if (q.launch_mode == vals[v]) continue; q.launch_mode = vals[v]; }
            if (stage == 1 && vals[v] > 0) {
                long long B = 1;
                for (int i = 0; i < ndim; ++i) B *= blk[i];
                if ((long long)vals[v] * NPTMAX < B) continue;
            }
            dope_tune_result r;
            tune_one(R, blk, q, &r);
            record(r);
            if (tune_better(r, cur)) cur = r;
        }
    }
    *best = cur;
    if (count) *count = nout < cap ? nout : cap;
    cudaEventDestroy(R.e0);
    cudaEventDestroy(R.e1);
    cudaFree(du);
    cudaFree(dw);
    cudaFree(dl);
    cudaGetLastError();
    return cur.status;
}

extern "C" int dope_get_block_state(dope_ctx* c, double* a, uint8_t* yhat, int64_t cap, int64_t* count,
                                    void* stream) {
    if (!c || !c->ov) return DOPE_EINVAL;
    const int64_t n = (int64_t)c->oa.g.K * c->oa.g.B;
    if (count) *count = n;
    if ((a || yhat) && cap < n) return DOPE_EINVAL;
    cudaStream_t st = S(stream);
    if (a) CK(cudaMemcpyAsync(a, c->oa.a, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st));
    if (yhat) CK(cudaMemcpyAsync(yhat, c->oa.yhat, (size_t)n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return DOPE_OK;
}
