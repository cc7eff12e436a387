// dope_kernels.cuh -- device code of the DOPE ADMM hot path (sm_103a).
//
// Layout in HBM (all "block-major": pixel (z,y,x) of block k = (kz,ky,kx) at
// local index l = (lz*bh + ly)*bw + lx lives at k*B + l, so one CTA reads one
// contiguous slab):
//   U    int32 [N]            quantised unaries, rne(1024 u)
//   Wl   int32 [conn/2][N]    quantised forward-edge weights, rne(lambda wq)
//   yhat uint8 [N]            block labels of the last iteration
//   yF   f64   [K][F]         y of the F face pixels of every block (Eq. 10)
//   aF   f64   [K][F]         a of the face pixels (Eq. 11)
// Pixels with no neighbour in another block ("interior") always have
// y = yhat and a = 0 once an iteration has run (Eq. 10 / 11 with Q = I give
// y = yhat + a - 0 and a = a + 0 starting from a = 0), so only the face is
// stored; this is exact, not an approximation.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda/atomic>

namespace dope {

// ---------------------------------------------------------------------------
// Shared-memory arrays of the block solver and the resident kernel are used
// through SArr, a pointer with the array's length.  In the ordinary build it
// is the pointer alone.  In the checked build (DOPE_CHECKED, libdope_checked)
// every index is tested against the length first: an index outside the array
// is recorded in dope_check_word (the first one wins: (length << 32 | index) + 1)
// and the access goes to a scratch cell instead, so a wrong index neither
// faults nor writes outside the array; the host reads the word with
// dope_check_status.  Each translation unit has its own word.
// ---------------------------------------------------------------------------
#ifdef DOPE_CHECKED
static __device__ unsigned long long dope_check_word;
static __device__ __align__(16) unsigned char dope_check_cell[16];
#endif

template <class T>
struct SArr {
    T* p;
#ifdef DOPE_CHECKED
    long long n;
    __device__ __forceinline__ SArr(T* ptr, long long len) : p(ptr), n(len) {}
    __device__ __forceinline__ T& operator[](long long i) const {
        if (i < 0 || i >= n) {
            atomicCAS(&dope_check_word, 0ull,
                      ((unsigned long long)(n & 0xffffffffLL) << 32 | (unsigned long long)(i & 0xffffffffLL)) + 1ull);
            return *reinterpret_cast<T*>(dope_check_cell);
        }
        return p[i];
    }
    __device__ __forceinline__ SArr sub(long long off, long long len) const {
        if (off < 0 || off + len > n) {
            atomicCAS(&dope_check_word, 0ull,
                      ((unsigned long long)(n & 0xffffffffLL) << 32 | (unsigned long long)(off & 0xffffffffLL)) + 1ull);
            return SArr(reinterpret_cast<T*>(dope_check_cell), 0);
        }
        return SArr(p + off, len);
    }
#else
    __device__ __forceinline__ SArr(T* ptr, long long) : p(ptr) {}
    __device__ __forceinline__ T& operator[](long long i) const { return p[i]; }
    __device__ __forceinline__ SArr sub(long long off, long long len) const { return SArr(p + off, len); }
#endif
    __device__ __forceinline__ explicit operator bool() const { return p != nullptr; }
};

constexpr int NPTMAX = 8;          // nodes per thread in the block solver
constexpr int FREE = 0, FIX0 = 1, FIX1 = 2;
constexpr int MAX_FOLD_ROUNDS = 3;    // default bound on exact-folding rounds
constexpr double CLAMP62 = 4611686018427387904.0;   // 2^62

// Block-solver shared memory: res int32 [conn][B], R1 8 B [B], R2 4 B [B],
// st uint8 [B], then (aligned to 4 B) the bit-parallel BFS words: per-direction
// residual masks [conn][W], seeds / frontier buffers [3][W], W = ceil(B / 32),
// then the free-node list int16 [B].
__host__ __device__ inline size_t solver_bits_offset(int conn, int B) {
    return ((size_t)(conn + 3) * 4 * B + B + 3) & ~(size_t)3;
}
// After the bit words: the list of nodes left free by the first folding round
// (int16 [B]), so later rounds and the push-relabel pulses visit only those.
__host__ __device__ inline size_t solver_list_offset(int conn, int B) {
    return solver_bits_offset(conn, B) + 4 * (size_t)(conn + 3) * ((B + 31) / 32);
}
__host__ __device__ inline size_t solver_smem_bytes(int conn, int B) {
    return solver_list_offset(conn, B) + 2 * (size_t)B;
}

struct Geo {
    int D, H, W;            // grid (D = 1 for 2-D), a whole number of blocks
    int bd, bh, bw, B;      // block shape and volume
    int nbz, nby, nbx, K;   // block grid
    int F;                  // face pixels per block
    long long N;
    // caller's grid, <= (D, H, W); pixels beyond it are padding with zero
    // unary and zero n-links (isolated, so they change no other pixel's
    // iterates and add nothing to the energy)
    int Du, Hu, Wu;
    long long Nu;
};

constexpr int LWMAX = 64;   // most iterations per run-ahead window of the persistent kernel

struct Ctrl {
    int conv_t;             // iteration whose stop test held (0 = not yet)
    int status;             // first DOPE_* error raised by a kernel
    int pulses_max;
    int pad;
    unsigned long long pulses_total;
    unsigned long long free_total;
    unsigned long long energy;      // k_energy accumulator (two's complement)
    unsigned long long cyc[4];      // SM cycles of CTA thread 0: build, fold, pulses, BFS
    unsigned long long bfs_levels;  // BFS levels summed over all BFS runs
    int bfs_levels_max;
    int fold_rounds_max;
    unsigned bar_count;             // grid barrier of the persistent kernel: arrivals
    unsigned yield;                 // batched launch: the host's request to end it, as read by CTA 0
    int abort;                      // set when a barrier wait gave up
    int iters_done;                 // last iteration the persistent kernel ran
    int thaw;                       // earliest iteration of a window whose labels moved
    int windows;                    // run-ahead windows run (statistics)
    int window_iters;               // iterations done inside windows (statistics)
    unsigned work[2];               // block counters of the persistent kernel (solve, update)
    unsigned long long wcyc[8];     // run-ahead windows, thread 0 of each CTA: build, cut,
                                    // label check, own update, halo update, set-up,
                                    // wait at the closing barrier, rest of the resolution
    unsigned long long pcyc[4];     // persistent kernel, thread 0 of each CTA: solve phase,
                                    // first barrier wait, update phase, second barrier wait
    unsigned long long sched_work[2];   // blocks solved / updated from the worklists (statistics)
    unsigned long long sched_part;      // of those solves, the ones that evaluated only some chunks
    unsigned cuts[2];               // persistent kernel: blocks solved by a cut, by iteration parity
    int handoff;                    // persistent kernel: the plain launch stopped at a frozen iteration,
    unsigned bar_handoff;           // ... the grid barriers it had passed (bar_count goes on from there)
    double mu_next;                 // ... and mu of the iteration after it
    unsigned wwork[3];              // persistent kernel's windows: piece counters of the three phases
    int lthaw[2];                   // persistent kernel's windows: earliest iteration not proven, by window parity
    unsigned long long r2w[2][LWMAX];   // persistent kernel's windows: bits of max_k r2_k, by window parity
    unsigned long long r2max[1];    // [max_iter + 2]: bits of max_k r2_k per iteration
};

// ---------------------------------------------------------------------------
// Block worklists (persistent kernels).  A block is *quiet* for iteration t+1
// when its Eq. 8 problem provably keeps its labels and its Eq. 10 / 11 update
// provably changes nothing:
//   * every face pixel i of the block has a_i = +0 and y_i = yhat_i, and every
//     cross-block neighbour j has y_j = y_i and yhat_j = yhat_i; so every cross
//     term of Eq. 8 is exactly zero and the pixel's unary is that of an
//     interior pixel, U_i +- 512 mu;
//   * every pixel passes the integer forced test (|U_i +- H| beyond its n-link
//     sum, H = floor(512 mu)), so every minimiser of Eq. 8 keeps its label.
// With the labels fixed, G_i = 0 for every face pixel, Eq. 10 gives y = yhat
// and Eq. 11 a = +0: the state does not move.  Because mu only grows (H is
// monotone), a quiet block stays quiet until its own state or a cross
// neighbour's state (y, a or label) changes.  The kernel therefore solves, in
// iteration t+1, only the blocks on a solve list: the non-quiet blocks and
// the blocks next to a face pixel whose state changed in iteration t; and it
// updates, in iteration t, only the blocks on an update list: the non-quiet
// blocks and the blocks next to a face pixel whose label changed.  Everything
// else is skipped, exactly: the skipped work would have reproduced the state
// bit for bit.  The first iteration of every launch solves and updates every
// block and evaluates nothing (so a state set from outside is never trusted).
//
// Per-context buffer (sched_bytes), K blocks, F face slots per block:
//   sq_n, uq_n  u32 [2]    lengths of the lists below (kept here, not in the
//                          control block, so they outlive its clearing)
//   smark, umark u64 [K]   last (epoch << 32 | t) a block was put on the
//                          solve / update list (one entry per list)
//   sq, uq      int32 [2][K]  the lists, by parity of their iteration
//   qs          uint8 [K]     1: the block was found quiet at its last solve
//   yhF         uint8 [K][F]  label of each face slot as of its block's last update
// ---------------------------------------------------------------------------
struct SchedView {
    unsigned* sq_n;
    unsigned* uq_n;
    unsigned long long* smark;
    unsigned long long* umark;
    int* sq;
    int* uq;
    unsigned* act;      // [K][4] chunks (32 face slots each) holding a slot that is not trivial
    unsigned* dsc;      // [K][4] chunks whose slots' Eq. 8 inputs changed since the block's last solve
    unsigned* duc;      // [K][4] chunks whose slots' cross-neighbour labels changed in this solve phase
    uint8_t* qs;        // [K] 0 not forced, 1 quiet, 2 forced with active chunks, 3 not evaluated (a launch's first iteration)
    uint8_t* yhF;
};

// Chunk masks hold up to 128 chunks of 32 face slots (F <= B <= 4096).
constexpr int CHUNK_WORDS = 4;

__host__ __device__ inline size_t sched_bytes(int K, int F) {
    return 16 + 16 * (size_t)K + 16 * (size_t)K + 48 * (size_t)K + (size_t)K + (size_t)K * F;
}

__device__ __forceinline__ SchedView sched_view(unsigned char* base, int K) {
    SchedView s;
    s.sq_n = reinterpret_cast<unsigned*>(base);
    s.uq_n = s.sq_n + 2;
    s.smark = reinterpret_cast<unsigned long long*>(base + 16);
    s.umark = s.smark + K;
    s.sq = reinterpret_cast<int*>(s.umark + K);
    s.uq = s.sq + 2 * (size_t)K;
    s.act = reinterpret_cast<unsigned*>(s.uq + 2 * (size_t)K);
    s.dsc = s.act + CHUNK_WORDS * (size_t)K;
    s.duc = s.dsc + CHUNK_WORDS * (size_t)K;
    s.qs = reinterpret_cast<uint8_t*>(s.duc + CHUNK_WORDS * (size_t)K);
    s.yhF = s.qs + K;
    return s;
}

// Mark face slot fn of block kn in a chunk mask.
__device__ __forceinline__ void chunk_mark(unsigned* masks, int kn, int fn) {
    const int ch = fn >> 5;
    atomicOr(&masks[(size_t)kn * CHUNK_WORDS + (ch >> 5)], 1u << (ch & 31));
}

// Put block kn on a list for the iteration whose mark is m, unless it is on
// it already.
__device__ __forceinline__ void wl_push(unsigned long long* mark, int* list, unsigned* count, int kn,
                                        unsigned long long m) {
    if (atomicMax(&mark[kn], m) < m) list[atomicAdd(count, 1u)] = kn;
}

// Threads 0..26 of the CTA: put every block of the 3x3(x3) neighbourhood of
// block k whose offset code ((dkz+1)*9 + (dky+1)*3 + dkx+1, 13 = k itself) is
// set in `mask` on the list.
template <class GEO>
__device__ __forceinline__ void wl_push_mask(const GEO& g, int k, unsigned mask, unsigned long long* mark,
                                             int* list, unsigned* count, unsigned long long m) {
    const int j = threadIdx.x;
    if (j >= 27 || !((mask >> j) & 1u)) return;
    const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
    const int nkz = kz + j / 9 - 1, nky = ky + (j / 3) % 3 - 1, nkx = kx + j % 3 - 1;
    if (nkz < 0 || nkz >= g.nbz || nky < 0 || nky >= g.nby || nkx < 0 || nkx >= g.nbx) return;
    wl_push(mark, list, count, (nkz * g.nby + nky) * g.nbx + nkx, m);
}

__device__ __forceinline__ unsigned long long wl_mark(unsigned epoch, int t) {
    return ((unsigned long long)epoch << 32) | (unsigned)t;
}

struct SolveArgs {
    Geo g;
    const int32_t* U;
    const int32_t* Wl;
    uint8_t* yhat;
    const double* yF;
    const double* aF;
    const int16_t* faceIndex;       // [B] face slot of local pixel, -1 if interior
    const int* halo;                // [CONN][F] cross-block neighbour of face slot (halo_entry)
    const int16_t* faceLocal;       // [F] local pixel of face slot
    const long long* Cgiven;        // block-major int64 unaries (test hook) or null
    Ctrl* ctrl;
    double mu, eps;
    int t, first, check_prev;
    int relabel_period, max_pulses;
    int fold_rounds;                // bound on exact-folding rounds
    int int_test;                   // interior forced test in integers (needs 512 mu < 2^52)
    long long H;                    // floor(512 mu)
    unsigned char* sched = nullptr; // block worklists (persistent kernel), or null
    unsigned epoch = 0;             // launch number for the worklists' marks
};

struct UpdArgs {
    Geo g;
    const int32_t* Wl;
    const uint8_t* yhat;
    double* yF;
    double* aF;
    double* r2blk;
    const int16_t* faceLocal;       // [F] local pixel of face slot
    const int16_t* faceIndex;
    const int* halo;
    Ctrl* ctrl;
    double mu;
    int t;
    unsigned char* sched = nullptr; // block worklists (persistent kernel), or null
    unsigned epoch = 0;
};

// Values of one iteration t that the block solver and the face update need:
// mu, and the integer forced-node test bound H = floor(512 mu) when
// 512 mu < 2^52 (int_test).
struct IterArgs {
    double mu;
    long long H;
    int t, first, int_test;
    int qeval;      // evaluate quiet blocks and fill the worklists (needs A.sched)
};

__device__ __forceinline__ IterArgs iter_args(int t, double mu) {
    IterArgs it;
    it.mu = mu;
    it.t = t;
    it.first = (t == 1);
    const double h = __dmul_rn(__dmul_rn(1024.0, mu), 0.5);
    it.int_test = h < 4503599627370496.0 ? 1 : 0;   // 2^52
    it.H = it.int_test ? (long long)floor(h) : 0;
    it.qeval = 0;
    return it;
}

// The iteration values a SolveArgs carries (k_block_solve, test hooks).
__device__ __forceinline__ IterArgs iter_of(const SolveArgs& A) {
    IterArgs it;
    it.mu = A.mu;
    it.H = A.H;
    it.t = A.t;
    it.first = A.first;
    it.int_test = A.int_test;
    it.qeval = 0;
    return it;
}

// Halo table entry of (face slot f, direction d): -1 if the neighbour is in
// the same block, else (block-offset code << 24) | (ln << 12) | fn with the
// neighbour's local index ln, its face slot fn and code = (dkz+1)*9 +
// (dky+1)*3 + (dkx+1) for the block offset (dkz, dky, dkx) in {-1,0,1}^3.
__host__ __device__ inline int halo_entry(int code, int ln, int fn) {
    return (code << 24) | (ln << 12) | fn;
}

// Decode a halo entry for block (kz,ky,kx); false if the neighbour block is
// outside the block grid (the pixel lies on the grid border).
__device__ __forceinline__ bool halo_decode(const Geo& g, int e, int kz, int ky, int kx, int& kn,
                                            int& ln, int& fn) {
    if (e < 0) return false;
    const int code = e >> 24;
    const int nkz = kz + code / 9 - 1, nky = ky + (code / 3) % 3 - 1, nkx = kx + code % 3 - 1;
    if (nkz < 0 || nkz >= g.nbz || nky < 0 || nky >= g.nby || nkx < 0 || nkx >= g.nbx) return false;
    kn = (nkz * g.nby + nky) * g.nbx + nkx;
    ln = (e >> 12) & 0xfff;
    fn = e & 0xfff;
    return true;
}

// Direction k of connectivity CONN: k < CONN/2 is forward offset k, k >= CONN/2
// the backward offset k - CONN/2.  Forward offsets (dz,dy,dx):
// 4: (0,0,1) (0,1,0); 8: + (0,1,1) (0,1,-1); 6: (0,0,1) (0,1,0) (1,0,0).
template <int CONN>
__device__ __forceinline__ void dir_off(int k, int& dz, int& dy, int& dx) {
    constexpr int nh = CONN / 2;
    const int o = k < nh ? k : k - nh;
    const int s = k < nh ? 1 : -1;
    if (CONN == 6) {
        dz = (o == 2); dy = (o == 1); dx = (o == 0);
    } else if (CONN == 4 || CONN == 8) {
        dz = 0; dy = (o >= 1); dx = (o == 0) ? 1 : (o == 1 ? 0 : (o == 2 ? 1 : -1));
    } else if (CONN == 32) {
        // radius-2 ball, forward offsets ordered by (dz, dy, dx)
        dz = o < 6 ? 0 : (o < 15 ? 1 : 2);
        if (o < 6) {
            dy = o < 2 ? 0 : (o < 5 ? 1 : 2);
            dx = o < 2 ? o + 1 : (o < 5 ? o - 3 : 0);
        } else if (o < 15) {
            dy = (o - 6) / 3 - 1;
            dx = (o - 6) % 3 - 1;
        } else {
            dy = 0;
            dx = 0;
        }
    } else {
        // (2r+1)^2 - 1 square kernel: row dy = 0 with dx = 1..r, then rows
        // dy = 1..r with dx = -r..r
        constexpr int r = CONN == 24 ? 2 : (CONN == 48 ? 3 : 4);
        dz = 0;
        if (o < r) {
            dy = 0;
            dx = o + 1;
        } else {
            dy = 1 + (o - r) / (2 * r + 1);
            dx = (o - r) % (2 * r + 1) - r;
        }
    }
    dz *= s; dy *= s; dx *= s;
}

// Largest coordinate offset of the neighbourhood of connectivity CONN.
template <int CONN>
__host__ __device__ constexpr int kernel_radius() {
    return CONN == 24 || CONN == 32 ? 2 : (CONN == 48 ? 3 : (CONN == 80 ? 4 : 1));
}

// Local-index offset of direction d inside a block with row pitch bw and
// plane size pl (= bh * bw); the direction is a compile-time constant in the
// unrolled loops, so this folds to one or two integer operations.
template <int CONN>
__device__ __forceinline__ int dir_lofs(int d, int bw, int pl) {
    int dz, dy, dx;
    dir_off<CONN>(d, dz, dy, dx);
    return dz * pl + dy * bw + dx;
}

template <int CONN>
__device__ __forceinline__ int opp_dir(int k) {
    constexpr int nh = CONN / 2;
    return k < nh ? k + nh : k - nh;
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies global -> shared (cp.async.bulk, the 1-D form of
// the tensor memory accelerator), completed on an mbarrier in shared memory.
// Source and destination 16-byte aligned, sizes multiples of 16.  The CTA is
// its own cluster, so its shared::cluster addresses are its own.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Order this thread's earlier generic-proxy accesses of shared memory before
// later asynchronous-proxy writes to it (the bulk copies).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void set_status(Ctrl* c, int code) {
    atomicCAS(&c->status, 0, code);
}

// Cross-block neighbour of local pixel (lz,ly,lx) of block (kz,ky,kx) along
// direction d.  Returns false if the neighbour is inside the same block or
// outside the grid; else the neighbour's block kn and local index ln.
template <int CONN>
__device__ __forceinline__ bool cross_nbr(const Geo& g, int kz, int ky, int kx, int lz, int ly,
                                          int lx, int d, int& kn, int& ln) {
    int dz, dy, dx;
    dir_off<CONN>(d, dz, dy, dx);
    int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
    if (nlz >= 0 && nlz < g.bd && nly >= 0 && nly < g.bh && nlx >= 0 && nlx < g.bw) return false;
    int gz = kz * g.bd + nlz, gy = ky * g.bh + nly, gx = kx * g.bw + nlx;
    if (gz < 0 || gz >= g.D || gy < 0 || gy >= g.H || gx < 0 || gx >= g.W) return false;
    int nkz = kz + (nlz < 0 ? -1 : (nlz >= g.bd ? 1 : 0));
    int nky = ky + (nly < 0 ? -1 : (nly >= g.bh ? 1 : 0));
    int nkx = kx + (nlx < 0 ? -1 : (nlx >= g.bw ? 1 : 0));
    nlz -= (nkz - kz) * g.bd; nly -= (nky - ky) * g.bh; nlx -= (nkx - kx) * g.bw;
    kn = (nkz * g.nby + nky) * g.nbx + nkx;
    ln = (nlz * g.bh + nly) * g.bw + nlx;
    return true;
}

// Eq. 8 unary of pixel v of block k, x1024, rounded half-to-even (step a4):
//   s = U_i; s += Wl_ij * (y_i - y_j) for cross-block j in direction order;
//   s += (1024 mu) * ((a_i - y_i) + 1/2)
// Every double operation is one IEEE round-to-nearest op (explicit
// intrinsics, so nothing is contracted into an FMA).  At the first iteration
// y = 1/2 and a = 0 make every shift vanish and s = U_i exactly.
template <int CONN>
__device__ __forceinline__ long long shifted_cap(const Geo& g, const int32_t* __restrict__ U,
                                                 const int32_t* __restrict__ Wl,
                                                 const uint8_t* __restrict__ yhat,
                                                 const double* __restrict__ yF,
                                                 const double* __restrict__ aF,
                                                 const int16_t* __restrict__ faceIndex, int k,
                                                 int kz, int ky, int kx, int v, int lz, int ly,
                                                 int lx, int first, double m1024) {
    constexpr int nh = CONN / 2;
    const long long gi = (long long)k * g.B + v;
    const int Ui = U[gi];
    if (first) return (long long)Ui;
    const int f = faceIndex[v];
    double s = (double)Ui;
    double yv, av;
    if (f < 0) {
        yv = (double)__ldcg(&yhat[gi]);
        av = 0.0;
    } else {
        yv = __ldcg(&yF[(long long)k * g.F + f]);
        av = __ldcg(&aF[(long long)k * g.F + f]);
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            int kn, ln;
            if (!cross_nbr<CONN>(g, kz, ky, kx, lz, ly, lx, d, kn, ln)) continue;
            const int fn = faceIndex[ln];
            const double yj = __ldcg(&yF[(long long)kn * g.F + fn]);
            const int w = (d < nh) ? Wl[(long long)d * g.N + gi]
                                   : Wl[(long long)(d - nh) * g.N + (long long)kn * g.B + ln];
            s = __dadd_rn(s, __dmul_rn((double)w, __dsub_rn(yv, yj)));
        }
    }
    s = __dadd_rn(s, __dmul_rn(m1024, __dadd_rn(__dsub_rn(av, yv), 0.5)));
    s = fmin(fmax(s, -CLAMP62), CLAMP62);
    return __double2ll_rn(s);
}

// The unaries the block solver works with.  For a pixel with no cross-block
// neighbour at iteration t >= 2, y = yhat and a = 0, so s = U + h with
// h = +-512 mu exactly (sign + for yhat = 0).  With H = floor(512 mu) and
// U + H, U - H exact integers below 2^53, round-to-nearest is monotone and
// C = rne(s) lies in {U + H, U + H + 1} (yhat = 0) or {U - H - 1, U - H}
// (yhat = 1).  If U + H >= cs (resp. U - H < -cs), where cs is the node's
// n-link sum, the node is forced to keep its label whatever C is exactly,
// and U +- H (forced the same way) stands in for C; the pointwise-minimal
// minimiser does not change.  Every other pixel gets the exact FP64 value.
//
// face_cap: the exact value for face slot f (pixel v) -- the operations of
// shifted_cap in the same order, with the neighbours found through the halo
// table and every load issued before the FP64 chain.
template <int CONN>
__device__ __forceinline__ long long face_cap_from(long long Ui, double yv, double av, const double* yj,
                                                   const int* wj, unsigned ok, double m1024) {
    double s = (double)Ui;
#pragma unroll
    for (int d = 0; d < CONN; ++d)
        if ((ok >> d) & 1) s = __dadd_rn(s, __dmul_rn((double)wj[d], __dsub_rn(yv, yj[d])));
    s = __dadd_rn(s, __dmul_rn(m1024, __dadd_rn(__dsub_rn(av, yv), 0.5)));
    s = fmin(fmax(s, -CLAMP62), CLAMP62);
    return __double2ll_rn(s);
}

template <int CONN>
__device__ __forceinline__ long long face_cap_core(const Geo& g, long long Ui, double yv, double av,
                                                   const int32_t* __restrict__ Wl,
                                                   const double* __restrict__ yF,
                                                   const int* __restrict__ halo, int k, int kz,
                                                   int ky, int kx, int v, int f, double m1024) {
    constexpr int nh = CONN / 2;
    const long long gi = (long long)k * g.B + v;
    double yj[CONN];
    int wj[CONN];
    unsigned ok = 0;
#pragma unroll
    for (int d = 0; d < CONN; ++d) {
        int kn, ln, fn;
        yj[d] = 0.0;
        wj[d] = 0;
        if (halo_decode(g, halo[d * g.F + f], kz, ky, kx, kn, ln, fn)) {
            ok |= 1u << d;
            yj[d] = __ldcg(&yF[(long long)kn * g.F + fn]);
            wj[d] = (d < nh) ? Wl[(long long)d * g.N + gi]
                             : Wl[(long long)(d - nh) * g.N + (long long)kn * g.B + ln];
        }
    }
    return face_cap_from<CONN>(Ui, yv, av, yj, wj, ok, m1024);
}

template <int CONN>
__device__ __forceinline__ long long face_cap(const Geo& g, const int32_t* __restrict__ U,
                                              const int32_t* __restrict__ Wl,
                                              const double* __restrict__ yF,
                                              const double* __restrict__ aF,
                                              const int* __restrict__ halo, int k, int kz, int ky,
                                              int kx, int v, int f, double m1024) {
    const double yv = __ldcg(&yF[(long long)k * g.F + f]);
    const double av = __ldcg(&aF[(long long)k * g.F + f]);
    return face_cap_core<CONN>(g, (long long)U[(long long)k * g.B + v], yv, av, Wl, yF, halo, k, kz,
                               ky, kx, v, f, m1024);
}

// Eq. 8 unary of an interior pixel (y = yhat, a = 0), the operations of
// shifted_cap's interior branch.
__device__ __forceinline__ long long interior_cap(long long Ui, int yh, double m1024) {
    double s = (double)Ui;
    s = __dadd_rn(s, __dmul_rn(m1024, __dadd_rn(__dsub_rn(0.0, (double)yh), 0.5)));
    s = fmin(fmax(s, -CLAMP62), CLAMP62);
    return __double2ll_rn(s);
}

// ---------------------------------------------------------------------------
// Block solver: one CTA per block (steps a4, a5, a6).
//
// Shared memory (B = block volume):
//   res   int32 [CONN][B]   residual capacity of edge v -> v + off(d)
//   R1    8 B  [B]          int64 unary during folding; then e[B], ein[B]
//   R2    4 B  [B]          int32 n-link sum during folding; then h0[B], h1[B] (int16)
//   st    uint8 [B]         FREE / FIX0 / FIX1
//
// 1. Capacity build: res = Wl on intra-block edges, C64 = Eq. 8 unary.
// 2. Exact folding: a free node with C >= sum of its remaining n-links takes
//    label 0 in the pointwise-minimal minimiser, one with C < -sum takes 1;
//    it is fixed and its n-links are folded into the neighbours' unaries
//    (+w if fixed to 0, -w if fixed to 1).  Repeated until nothing changes.
//    After this every free node has |C| < 2^28, so int32 is exact.
// 3. Push-relabel on the free nodes (implicit terminals: e > 0 excess,
//    e < 0 remaining capacity to t), synchronous pulses: push along admissible
//    edges with heights fixed for the pulse, then relabel with double-buffered
//    heights; global relabel (BFS from t) every relabel_period pulses.
// 4. Canonical cut: after the max-preflow, the nodes that reach t in the
//    residual graph (backward BFS from the nodes with e < 0) form the minimal
//    sink side, i.e. the pointwise-minimal minimiser; label 1 = sink side.
// ---------------------------------------------------------------------------

// Backward BFS from t, bit-parallel.  Every node is a bit of W = ceil(B/32)
// words; each direction's residual edges (res > 0) become a mask built with
// warp ballots, and one warp expands the frontier level by level: the nodes
// that can step into the frontier along direction d are E_d & (F shifted by
// the direction's local offset).  The distances are the exact BFS distances
// (1 = residual capacity to t, HMAX = cannot reach t), the same heights the
// level-synchronous search gives, at one warp-synchronisation per level
// instead of a block barrier.  Returns whether a free node with excess can
// still reach t.
template <int CONN>
__device__ __forceinline__ int bfs_bits(const SArr<int> res, const SArr<int> e, const SArr<int16_t> h,
                                        const SArr<uint8_t> st, const SArr<uint32_t> bits, int bw, int pl, int B,
                                        int HMAX, int tid, int NT, int& levels) {
    const int W = (B + 31) >> 5;
    const SArr<uint32_t> E = bits.sub(0, (long long)CONN * W);          // [CONN][W]
    const SArr<uint32_t> Fa = bits.sub((long long)CONN * W, W);         // frontier, two buffers
    const SArr<uint32_t> Fb = bits.sub((long long)(CONN + 1) * W, W);
    const int lane = tid & 31;
    for (int base = 0; base < B; base += NT) {
        const int v = base + tid;
        const bool in = v < B;
        const int wi = v >> 5;
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            const unsigned m = __ballot_sync(0xffffffffu, in && res[d * B + v] > 0);
            if (lane == 0 && wi < W) E[d * W + wi] = m;
        }
        const bool seed = in && st[v] == FREE && e[v] < 0;
        const unsigned ms = __ballot_sync(0xffffffffu, seed);
        if (lane == 0 && wi < W) Fa[wi] = ms;
        if (in) h[v] = seed ? (int16_t)1 : (int16_t)HMAX;
    }
    __syncthreads();
    int lv = 1;
    if (tid < 32) {
        constexpr int MAXW = 4;          // W <= 128 (B <= 4096)
        uint32_t vis[MAXW];
#pragma unroll
        for (int s2 = 0; s2 < MAXW; ++s2) {
            const int i = lane + 32 * s2;
            vis[s2] = i < W ? Fa[i] : 0u;
        }
        SArr<uint32_t> F = Fa;
        SArr<uint32_t> Nf = Fb;
        while (lv < HMAX - 1) {
            unsigned any = 0;
#pragma unroll
            for (int s2 = 0; s2 < MAXW; ++s2) {
                const int i = lane + 32 * s2;
                if (i >= W) continue;
                uint32_t nw = 0;
#pragma unroll
                for (int d = 0; d < CONN; ++d) {
                    const int o = dir_lofs<CONN>(d, bw, pl);   // G[v] = F[v + o]
                    const int a = o >> 5, b = o & 31;
                    const int i0 = i + a, i1 = i + a + 1;
                    const uint32_t lo = (i0 >= 0 && i0 < W) ? F[i0] : 0u;
                    const uint32_t hi = (b != 0 && i1 >= 0 && i1 < W) ? F[i1] : 0u;
                    const uint32_t G = b ? ((lo >> b) | (hi << (32 - b))) : lo;
                    nw |= E[d * W + i] & G;
                }
                nw &= ~vis[s2];
                Nf[i] = nw;
                vis[s2] |= nw;
                any |= nw;
                uint32_t m = nw;
                while (m) {
                    const int j = __ffs(m) - 1;
                    h[32 * i + j] = (int16_t)(lv + 1);
                    m &= m - 1;
                }
            }
            if (!__any_sync(0xffffffffu, any != 0)) break;
            ++lv;
            __syncwarp();
            const SArr<uint32_t> tmp = F; F = Nf; Nf = tmp;
        }
    }
    levels += lv;
    __syncthreads();
    int act = 0;
#pragma unroll 1
    for (int q = 0; q < NPTMAX; ++q) {
        int v = tid + q * NT;
        if (v < B && st[v] == FREE && e[v] > 0 && h[v] < HMAX) act = 1;
    }
    return __syncthreads_or(act);
}

// The block solver and the face update are templates over the argument
// block (SolveArgs / UpdArgs, or a batched launch's per-problem descriptor):
// any type with the fields they read.
template <int CONN, class SA>
__device__ __forceinline__ void cut_block(const SA& __restrict__ A, int k, unsigned char* smem, int bw, int pl,
                                       unsigned long long imask, long long c_start, uint8_t* lab_smem,
                                       bool to_global = true);

// Two floats bracketing a double, from its bits alone (no FP64 operation):
// lo <= x <= hi.  The double's mantissa is cut to 23 bits (toward zero) and,
// if anything was cut, the other bound is the next float away from zero.
// Magnitudes below 2^-126 get [-2^-126, 2^-126] (0 stays exact), magnitudes
// of 2^128 and above an infinite bound.
__device__ __forceinline__ void dbl_bounds(double x, float& lo, float& hi) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const bool neg = (b >> 63) != 0;
    const int e = (int)((b >> 52) & 0x7ff);
    float tlo, thi;                      // bounds of |x|
    if ((b << 1) == 0) {
        tlo = thi = 0.f;
    } else if (e < 1023 - 126) {
        tlo = 0.f;
        thi = 1.1754943508222875e-38f;   // 2^-126
    } else if (e > 1023 + 127) {
        tlo = 3.4028234663852886e38f;    // largest float
        thi = __int_as_float(0x7f800000);
    } else {
        const unsigned fb = ((unsigned)(e - 1023 + 127) << 23) | (unsigned)((b >> 29) & 0x7fffff);
        tlo = __uint_as_float(fb);
        thi = (b & 0x1fffffffull) ? __uint_as_float(fb + 1u) : tlo;   // fb + 1: next float up (inf at the top)
    }
    lo = neg ? -thi : tlo;
    hi = neg ? -tlo : thi;
}

// Certificate for the Eq. 8 unary of a face pixel without FP64 work: an
// interval [s_lo, s_hi] holding the exact real value of
//   s = U + sum_d w_d (y - y_d) + m1024 ((a - y) + 1/2)
// from FP32 interval arithmetic with directed rounding on the bounds of each
// double, widened by 2^-48 M for the roundings of the FP64 evaluation the
// exact path does: at most 3 CONN + 4 <= 28 round-to-nearest steps, each of
// which moves the result by at most 2^-53 M, where M = |U| + sum_d w_d (|y| +
// |y_d|) + m1024 (|a| + |y| + 1/2) bounds every intermediate value (an error
// in y - y_d or a - y enters multiplied by w_d or m1024, still within M).
// Returns 0 if s provably rounds to C >= cs (label 0 in
// every minimiser), 1 if to C < -cs (label 1), -1 if the interval decides
// nothing (the exact value must be computed).  w_d >= 0 (submodular).
template <int CONN>
__device__ __forceinline__ int face_cert(long long Ui, double yv, double av, const double* yj, const int* wj,
                                         unsigned ok, double m1024, long long cs) {
    float ylo, yhi, alo, ahi, mlo, mhi;
    dbl_bounds(yv, ylo, yhi);
    dbl_bounds(av, alo, ahi);
    dbl_bounds(m1024, mlo, mhi);
    float slo = __ll2float_rd(Ui), shi = __ll2float_ru(Ui);
    float M = fabsf(shi) > fabsf(slo) ? fabsf(shi) : fabsf(slo);
    const float ymag = fmaxf(fabsf(ylo), fabsf(yhi));
#pragma unroll
    for (int d = 0; d < CONN; ++d) {
        if (!((ok >> d) & 1)) continue;
        float jlo, jhi;
        dbl_bounds(yj[d], jlo, jhi);
        const float w = (float)wj[d];                 // exact: n-links are below 2^24
        slo = __fadd_rd(slo, __fmul_rd(w, __fsub_rd(ylo, jhi)));
        shi = __fadd_ru(shi, __fmul_ru(w, __fsub_ru(yhi, jlo)));
        M = __fadd_ru(M, __fmul_ru(w, __fadd_ru(ymag, fmaxf(fabsf(jlo), fabsf(jhi)))));
    }
    const float qlo = __fadd_rd(__fsub_rd(alo, yhi), 0.5f);
    const float qhi = __fadd_ru(__fsub_ru(ahi, ylo), 0.5f);
    slo = __fadd_rd(slo, qlo >= 0.f ? __fmul_rd(mlo, qlo) : __fmul_rd(mhi, qlo));
    shi = __fadd_ru(shi, qhi >= 0.f ? __fmul_ru(mhi, qhi) : __fmul_ru(mlo, qhi));
    M = __fadd_ru(M, __fmul_ru(mhi, __fadd_ru(__fadd_ru(fmaxf(fabsf(alo), fabsf(ahi)), ymag), 0.5f)));
    static_assert(CONN <= 8, "the rounding count above assumes at most 8 neighbours");
    const float dl = __fmul_ru(M, 3.552713678800501e-15f);      // 2^-48 M
    if (__fsub_rd(slo, dl) >= __ll2float_ru(cs)) return 0;      // s >= cs: C >= cs
    if (__fadd_ru(shi, dl) <= __ll2float_rd(-cs - 1)) return 1; // s <= -cs - 1: C < -cs
    return -1;
}

// Eq. 8 unary of face slot f (local pixel v, label yh, unary Ui, intra-block
// n-link sum cs) of block k.  A slot in the trivial state (a = +0, y = yhat)
// whose cross neighbours all have y_j = y_i gets the interior unary (every
// cross term is +-0) and the integer forced test; every other slot the exact
// FP64 value.  Returns C (the exact value, or U +- H where the integer test
// holds); `uni`: trivial with equal cross neighbours, labels included (the
// neighbours' labels as of their blocks' last update); `forced`: forced to
// its own label yh (C >= cs for 0, C < -cs for 1) in every minimiser.
template <int CONN, class SA>
__device__ __forceinline__ long long face_slot_cap(const SA& __restrict__ A, const IterArgs& it, const SchedView& sv,
                                                   int k, int kz, int ky, int kx, int f, int v, long long Ui,
                                                   int yh, long long cs, double m1024, bool& uni, bool& forced) {
    const Geo& g = A.g;
    constexpr int nh = CONN / 2;
    const long long gi = (long long)k * g.B + v;
    const long long sidx = (long long)k * g.F + f;
    const double yv = __ldcg(&A.yF[sidx]);
    const double av = __ldcg(&A.aF[sidx]);
    double yj[CONN];
    int wj[CONN];
    unsigned ok = 0;
    bool lab_same = true;
#pragma unroll
    for (int d = 0; d < CONN; ++d) {
        int kn, ln, fn;
        yj[d] = 0.0;
        wj[d] = 0;
        if (halo_decode(g, A.halo[d * g.F + f], kz, ky, kx, kn, ln, fn)) {
            ok |= 1u << d;
            yj[d] = __ldcg(&A.yF[(long long)kn * g.F + fn]);
            wj[d] = (d < nh) ? A.Wl[(long long)d * g.N + gi]
                             : A.Wl[(long long)(d - nh) * g.N + (long long)kn * g.B + ln];
            if (it.qeval) lab_same = lab_same && (int)__ldcg(&sv.yhF[(long long)kn * g.F + fn]) == yh;
        }
    }
    // equality tests on the bits (no FP64 work): y = +0 or 1.0 exactly, and a
    // neighbour's y with the same bits as this pixel's
    const long long yb = __double_as_longlong(yv);
    bool u = __double_as_longlong(av) == 0 && yb == (yh ? 0x3ff0000000000000LL : 0LL);
#pragma unroll
    for (int d = 0; d < CONN; ++d)
        if ((ok >> d) & 1) u = u && __double_as_longlong(yj[d]) == yb;
    long long C;
    if (u) {
        const long long T = yh ? Ui - it.H : Ui + it.H;
        if (it.int_test && (yh ? (T < -cs) : (T >= cs))) C = T;
        else C = interior_cap(Ui, yh, m1024);
    } else {
        // a certified label needs no exact value: any C beyond the n-link
        // sum on that side gives the same minimisers (the folding fixes the
        // node either way)
        const int lab = face_cert<CONN>(Ui, yv, av, yj, wj, ok, m1024, cs);
        if (lab == 0) C = cs;
        else if (lab == 1) C = -cs - 1;
        else C = face_cap_from<CONN>(Ui, yv, av, yj, wj, ok, m1024);
    }
    uni = u && lab_same;
    forced = yh ? (C < -cs) : (C >= cs);
    return C;
}

// Intra-block n-link sum of local pixel v (the value the capacity build puts
// in capsum), read from the forward weight planes.
template <int CONN>
__device__ __forceinline__ long long nlink_sum(const Geo& g, const int32_t* __restrict__ Wl, int k, int v) {
    constexpr int nh = CONN / 2;
    const int lx = v % g.bw, ly = (v / g.bw) % g.bh, lz = v / (g.bw * g.bh);
    const long long gi = (long long)k * g.B + v;
    long long cs = 0;
#pragma unroll
    for (int d = 0; d < CONN; ++d) {
        int dz, dy, dx;
        dir_off<CONN>(d, dz, dy, dx);
        const int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
        if (nlz < 0 || nlz >= g.bd || nly < 0 || nly >= g.bh || nlx < 0 || nlx >= g.bw) continue;
        cs += (d < nh) ? Wl[(long long)d * g.N + gi]
                       : Wl[(long long)(d - nh) * g.N + gi + (dz * g.bh + dy) * g.bw + dx];
    }
    return cs;
}

// One warp: re-evaluate chunk ch of forced block k (a partial solve).  Returns
// through the warp: forced (every slot still forced to its label) and uni
// (every slot trivial with equal neighbours).
template <int CONN, class SA>
__device__ __forceinline__ void eval_chunk(const SA& __restrict__ A, const IterArgs& it, const SchedView& sv, int k,
                                           int ch, double m1024, bool& all_forced, bool& all_uni) {
    const Geo& g = A.g;
    const int lane = threadIdx.x & 31;
    const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
    const int f = ch * 32 + lane;
    bool uni = true, forced = true;
    if (f < g.F) {
        const int v = A.faceLocal[f];
        const long long gi = (long long)k * g.B + v;
        const int yh = __ldcg(&A.yhat[gi]);
        const long long cs = nlink_sum<CONN>(g, A.Wl, k, v);
        face_slot_cap<CONN>(A, it, sv, k, kz, ky, kx, f, v, (long long)A.U[gi], yh, cs, m1024, uni, forced);
    }
    all_forced = __all_sync(0xffffffffu, forced);
    all_uni = __all_sync(0xffffffffu, uni);
}

// Partial solves of up to MB forced blocks at once (their nodes were all
// forced to their labels at their last solve; see solve_block): the chunks
// to evaluate of all of them are spread over the CTA's warps, so their load
// latencies overlap.  ok[j] = 1 if block j's labels stand (its masks and
// state are updated and it is put on the update list if still active); 0 if
// a slot is no longer forced, and then nothing was written for it.
constexpr int MB = 4;

// Shared scratch of the update and partial-solve helpers.  They are templates
// over the connectivity, and a batched launch instantiates each of them three
// times; taking their arrays from one non-template accessor keeps a single
// copy per kernel (static shared variables of a template exist once per
// instantiation).  The helpers never run at the same time in a CTA.
struct UpdSmem {
    double part[MB][128];        // per block and chunk: sum of (yhat - y)^2
    unsigned pm[MB][128];        // per block and chunk: offset codes to push
    unsigned dom[MB][CHUNK_WORDS];   // chunks updated / evaluated
    unsigned act[MB][CHUNK_WORDS];   // chunks found active
    unsigned mm[MB];             // per block: push mask
    int okb[MB];                 // per block: labels stand
    int qb[MB];                  // per block: list state (0 not forced, 1 quiet, 2 forced and active)
    int tot;
    int ecnt;                    // run-ahead window: moving slots listed
    int ovf;                     // run-ahead window: the list did not fit
};
__device__ __forceinline__ UpdSmem& upd_smem() {
    __shared__ UpdSmem u;
    return u;
}

template <int CONN, class SA>
__device__ void partial_solve_multi(const SA& __restrict__ A, const IterArgs it, const int* kk, int nb, int* ok) {
    const Geo& g = A.g;
    const int tid = threadIdx.x, wid = tid >> 5, nw = blockDim.x >> 5;
    const SchedView sv = sched_view(A.sched, g.K);
    const double m1024 = __dmul_rn(1024.0, it.mu);
    UpdSmem& us = upd_smem();
    unsigned (&s_ev)[MB][CHUNK_WORDS] = us.dom;
    unsigned (&s_act)[MB][CHUNK_WORDS] = us.act;
    int (&s_okb)[MB] = us.okb;
    int& s_tot = us.tot;
    const int nchunks = (g.F + 31) >> 5;
    if (tid < nb * CHUNK_WORDS) {
        const int j = tid / CHUNK_WORDS, w = tid % CHUNK_WORDS;
        const size_t o = (size_t)kk[j] * CHUNK_WORDS + w;
        const int q = __ldcg(&sv.qs[kk[j]]);
        if (q == 3) {
            // not evaluated since the launch's first iteration: every chunk,
            // and every interior pixel below
            const int hi = nchunks - w * 32;
            s_ev[j][w] = hi <= 0 ? 0u : (hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u));
        } else {
            s_ev[j][w] = __ldcg(&sv.act[o]) | __ldcg(&sv.dsc[o]);     // every active chunk is among them
        }
        s_act[j][w] = 0u;
        if (w == 0) us.qb[j] = q;
    }
    if (tid < MB) s_okb[tid] = 1;
    __syncthreads();
    if (tid == 0) {
        int tot = 0;
        for (int j = 0; j < nb; ++j)
            for (int w = 0; w < CHUNK_WORDS; ++w) tot += __popc(s_ev[j][w]);
        s_tot = tot;
    }
    __syncthreads();
    const int tot = s_tot;
    // task t -> (block j, chunk ch): the t-th set bit over the blocks' masks
    for (int t = wid; t < tot; t += nw) {
        int r = t, j = 0, w = 0;
        for (;;) {
            const int c = __popc(s_ev[j][w]);
            if (r < c) break;
            r -= c;
            if (++w == CHUNK_WORDS) { w = 0; ++j; }
        }
        unsigned m = s_ev[j][w];
        for (int i = 0; i < r; ++i) m &= m - 1;
        const int ch = w * 32 + __ffs(m) - 1;
        bool fo, un;
        eval_chunk<CONN>(A, it, sv, kk[j], ch, m1024, fo, un);
        if ((threadIdx.x & 31) == 0) {
            if (!fo) s_okb[j] = 0;
            if (!un) atomicOr(&s_act[j][ch >> 5], 1u << (ch & 31));
        }
    }
    // interior pixels of the blocks not evaluated since the launch's first
    // iteration: the forced test of the capacity build (the integer bound,
    // else the exact interior unary) against the intra-block n-link sum
    const int B = g.B;
    for (int q = tid; q < nb * B; q += blockDim.x) {
        const int j = q / B, v = q - j * B;
        if (us.qb[j] != 3 || A.faceIndex[v] >= 0) continue;
        const int k = kk[j];
        const long long gi = (long long)k * B + v;
        const int yh = __ldcg(&A.yhat[gi]);
        const long long Ui = A.U[gi];
        const long long cs = nlink_sum<CONN>(g, A.Wl, k, v);
        const long long T = yh ? Ui - it.H : Ui + it.H;
        bool forced = it.int_test && (yh ? (T < -cs) : (T >= cs));
        if (!forced) {
            const long long C = interior_cap(Ui, yh, m1024);
            forced = yh ? (C < -cs) : (C >= cs);
        }
        if (!forced) s_okb[j] = 0;
    }
    __syncthreads();
    // blocks whose labels stand: masks, state, and the update list (threads
    // 32 j .. 32 j + 26 push block j)
    if (tid < nb * CHUNK_WORDS) {
        const int j = tid / CHUNK_WORDS, w = tid % CHUNK_WORDS;
        if (s_okb[j]) {
            const size_t o = (size_t)kk[j] * CHUNK_WORDS + w;
            sv.act[o] = s_act[j][w];
            sv.dsc[o] = 0u;
        }
    }
    {
        const int j = tid >> 5;
        if (j < nb && s_okb[j]) {
            int any = 0;
#pragma unroll
            for (int w = 0; w < CHUNK_WORDS; ++w) any |= s_act[j][w] != 0;
            if ((tid & 31) == 0) {
                sv.qs[kk[j]] = any ? 2 : 1;
                atomicAdd(&A.ctrl->sched_part, 1ull);
            }
            const int lane = tid & 31;
            if (any && lane == 13) {
                // this block itself (offset code 13) on the update list
                wl_push(sv.umark, sv.uq + (size_t)(it.t & 1) * g.K, &sv.uq_n[it.t & 1], kk[j],
                        wl_mark(A.epoch, it.t));
            }
        }
    }
    if (tid < nb) ok[tid] = s_okb[tid];
    __syncthreads();
}

template <int CONN, class SA>
__device__ void solve_block(const SA& __restrict__ A, const IterArgs it, int k, unsigned char* smem,
                            bool try_partial = true) {
    const Geo& g = A.g;
    const int B = g.B;
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = NT >> 5;
    int* res_p = reinterpret_cast<int*>(smem);
    long long* C64_p = reinterpret_cast<long long*>(res_p + CONN * B);
    int* capsum_p = reinterpret_cast<int*>(C64_p + B);
    const SArr<int> res(res_p, (long long)CONN * B);
    const SArr<long long> C64(C64_p, B);
    const SArr<int> capsum(capsum_p, B);
    const SArr<uint8_t> st(reinterpret_cast<uint8_t*>(capsum_p + B), B);
    const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
    const int bw = g.bw, pl = g.bh * g.bw;
    constexpr int nh = CONN / 2;
    const double m1024 = __dmul_rn(1024.0, it.mu);
    const SchedView sv = sched_view(A.sched, g.K);
    const int nchunks = (g.F + 31) >> 5;
    unsigned long long imask = 0;        // 8 bits per own node: intra-block directions
    unsigned oldlab = 0;                 // bit q: label of own node tid + q NT before this solve
    int allf = 1;                        // every own node forced to its own label
    int allu = 1;                        // every face slot trivial with equal cross neighbours
    __shared__ unsigned s_pm;            // neighbour blocks to put on the update list
    __shared__ unsigned s_act[CHUNK_WORDS];
    __shared__ unsigned s_ev[CHUNK_WORDS];
    __shared__ int s_ok;
    const long long c_start = clock64();

    if (try_partial && it.qeval && (unsigned)(__ldcg(&sv.qs[k]) - 1) < 2u) {
        // Every node of the block was forced to its label at its last solve.
        // Nodes in chunks that are neither active nor marked dirty still are
        // (their inputs did not change, and the integer test's bound only
        // grows), so only those chunks are evaluated again; if all their slots
        // are still forced to their labels, the labels stand.
        if (tid < CHUNK_WORDS) {
            const unsigned a = __ldcg(&sv.act[(size_t)k * CHUNK_WORDS + tid]);
            const unsigned d = __ldcg(&sv.dsc[(size_t)k * CHUNK_WORDS + tid]);
            s_ev[tid] = a | d;       // every active chunk is among them
            s_act[tid] = 0u;
        }
        if (tid == 0) s_ok = 1;
        __syncthreads();
        int ok = 1;
        // the evaluated chunks in increasing order, one per warp
        int seen = 0;
        for (int w = 0; w < CHUNK_WORDS; ++w) {
            unsigned m = s_ev[w];
            while (m) {
                const int ch = w * 32 + __ffs(m) - 1;
                m &= m - 1;
                if ((seen++ % nw) != wid) continue;
                const int f = ch * 32 + lane;
                bool uni = true, forced = true;
                if (f < g.F) {
                    const int v = A.faceLocal[f];
                    const long long gi = (long long)k * B + v;
                    const int yh = __ldcg(&A.yhat[gi]);
                    const long long cs = nlink_sum<CONN>(g, A.Wl, k, v);
                    face_slot_cap<CONN>(A, it, sv, k, kz, ky, kx, f, v, (long long)A.U[gi], yh, cs, m1024, uni,
                                        forced);
                }
                ok &= __all_sync(0xffffffffu, forced) ? 1 : 0;
                if (!__all_sync(0xffffffffu, uni) && lane == 0) atomicOr(&s_act[w], 1u << (ch & 31));
            }
        }
        if (!__syncthreads_and(ok)) {
            if (tid == 0) s_ok = 0;
        }
        __syncthreads();
        if (s_ok) {
            // labels stand; the block stays forced (quiet if no chunk is active)
            int any = 0;
#pragma unroll
            for (int w = 0; w < CHUNK_WORDS; ++w) any |= s_act[w] != 0;
            if (tid < CHUNK_WORDS) {
                sv.act[(size_t)k * CHUNK_WORDS + tid] = s_act[tid];
                sv.dsc[(size_t)k * CHUNK_WORDS + tid] = 0u;
            }
            if (tid == 0) {
                sv.qs[k] = any ? 2 : 1;
                atomicAdd(&A.ctrl->sched_part, 1ull);
            }
            wl_push_mask(g, k, any ? (1u << 13) : 0u, sv.umark, sv.uq + (size_t)(it.t & 1) * g.K,
                         &sv.uq_n[it.t & 1], wl_mark(A.epoch, it.t));
            __syncthreads();
            return;
        }
        // a slot is no longer forced to its label: the full solve below
    }

    // 1a. capacity build: forward intra-block n-links, U and yhat.  The block's
    // slabs are contiguous (block-major layout), so when the block volume is a
    // multiple of 16 one thread stages them into shared memory with bulk
    // asynchronous copies (the forward weight planes straight into res, U
    // into the capsum array, the labels into st), completed on an mbarrier;
    // the nodes then zero the out-of-block n-links and widen U in place.
    const bool bulk = !A.Cgiven && (B & 15) == 0;
    if (bulk) {
        __shared__ unsigned long long s_bar;
        if (tid == 0) mbar_init(&s_bar, 1);
        __syncthreads();
        if (tid == 0) {
            fence_proxy_async_smem();     // earlier generic accesses of this smem come first
            const unsigned plane = 4u * (unsigned)B;
            const unsigned bytes = (unsigned)nh * plane + plane + (it.first ? 0u : (unsigned)B);
            mbar_expect_tx(&s_bar, bytes);
            const long long base = (long long)k * B;
#pragma unroll
            for (int d = 0; d < nh; ++d) bulk_g2s(res_p + (size_t)d * B, A.Wl + (long long)d * g.N + base, plane, &s_bar);
            bulk_g2s(capsum_p, A.U + base, plane, &s_bar);
            if (!it.first) bulk_g2s(&st[0], A.yhat + base, (unsigned)B, &s_bar);
        }
        {
            // every thread waits for the copies (bounded, about 2 s: they come
            // from this GPU's memory); a wait that runs out sets the status,
            // then waits as long again for the copies still in flight
            const long long t0 = clock64();
            bool late = false;
            while (!mbar_try_wait(&s_bar, 0)) {
                if (!late && clock64() - t0 > 4000000000LL) {
                    if (tid == 0) set_status(A.ctrl, 6 /* DOPE_ETIMEOUT */);
                    late = true;
                }
                if (clock64() - t0 > 8000000000LL) break;
            }
        }
        __syncthreads();
#pragma unroll 1
        for (int q = 0; q < NPTMAX; ++q) {
            int v = tid + q * NT;
            if (v >= B) continue;
            const int lx = v % g.bw, ly = (v / g.bw) % g.bh, lz = v / (g.bw * g.bh);
            uint8_t m = 0;
#pragma unroll
            for (int d = 0; d < CONN; ++d) {
                int dz, dy, dx;
                dir_off<CONN>(d, dz, dy, dx);
                const int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
                const bool in = nlz >= 0 && nlz < g.bd && nly >= 0 && nly < g.bh && nlx >= 0 && nlx < g.bw;
                if (in) m |= (uint8_t)(1u << d);
                else if (d < nh) res[d * B + v] = 0;
            }
            imask |= (unsigned long long)m << (8 * q);
            if (it.first) st[v] = 0;
        }
        // U: int32 in capsum -> int64 in C64 (different arrays; capsum is
        // rewritten only in step 1b, after the barrier below)
#pragma unroll 1
        for (int q = 0; q < NPTMAX; ++q) {
            int v = tid + q * NT;
            if (v < B) C64[v] = (long long)capsum[v];
        }
        __syncthreads();
        if (tid == 0) mbar_inval(&s_bar);
    } else {
#pragma unroll 1
        for (int q = 0; q < NPTMAX; ++q) {
            int v = tid + q * NT;
            if (v >= B) continue;
            const int lx = v % g.bw, ly = (v / g.bw) % g.bh, lz = v / (g.bw * g.bh);
            const long long gi = (long long)k * B + v;
            uint8_t m = 0;
#pragma unroll
            for (int d = 0; d < CONN; ++d) {
                int dz, dy, dx;
                dir_off<CONN>(d, dz, dy, dx);
                const int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
                const bool in = nlz >= 0 && nlz < g.bd && nly >= 0 && nly < g.bh && nlx >= 0 && nlx < g.bw;
                if (in) m |= (uint8_t)(1u << d);
                if (d < nh) res[d * B + v] = in ? A.Wl[(long long)d * g.N + gi] : 0;
            }
            imask |= (unsigned long long)m << (8 * q);
            C64[v] = A.Cgiven ? A.Cgiven[gi] : (long long)A.U[gi];
            st[v] = it.first ? 0 : __ldcg(&A.yhat[gi]);
        }
    }
    if (tid < CHUNK_WORDS) s_act[tid] = 0u;
    __syncthreads();
    // 1b. backward n-links from shared memory, n-link sums, interior unaries
    const bool need_caps = !A.Cgiven && !it.first;
#pragma unroll 1
    for (int q = 0; q < NPTMAX; ++q) {
        int v = tid + q * NT;
        if (v >= B) continue;
        const unsigned m = (unsigned)(imask >> (8 * q)) & 0xffu;
        int cs = 0;
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            if (d < nh) {
                cs += res[d * B + v];
            } else {
                const int w = ((m >> d) & 1) ? res[(d - nh) * B + v + dir_lofs<CONN>(d, bw, pl)] : 0;
                res[d * B + v] = w;
                cs += w;
            }
        }
        capsum[v] = cs;
        const int yh = st[v];
        oldlab |= (unsigned)yh << q;
        if (need_caps && A.faceIndex[v] < 0) {
            st[v] = FREE;
            // interior pixel: y = yhat, a = 0 (see the note above face_cap)
            const long long Ui = C64[v];
            const long long T = yh ? Ui - it.H : Ui + it.H;
            if (it.int_test && (yh ? (T < -(long long)cs) : (T >= (long long)cs))) {
                C64[v] = T;
            } else {
                const int lx = v % g.bw, ly = (v / g.bw) % g.bh, lz = v / (g.bw * g.bh);
                const long long C = shifted_cap<CONN>(g, A.U, A.Wl, A.yhat, A.yF, A.aF, A.faceIndex, k, kz, ky,
                                                      kx, v, lz, ly, lx, 0, m1024);
                C64[v] = C;
                if (!(yh ? (C < -(long long)cs) : (C >= (long long)cs))) allf = 0;
            }
        } else if (!need_caps) {
            st[v] = FREE;
        }
    }
    // 1c. face pixels, in chunks of 32 slots per warp (after the n-link sums are in)
    if (need_caps) {
        __syncthreads();
        for (int ch = wid; ch < nchunks; ch += nw) {
            const int f = ch * 32 + lane;
            bool uni = true, forced = true;
            if (f < g.F) {
                const int v = A.faceLocal[f];
                C64[v] = face_slot_cap<CONN>(A, it, sv, k, kz, ky, kx, f, v, C64[v], st[v], capsum[v], m1024, uni,
                                             forced);
                st[v] = FREE;
            }
            allf &= forced ? 1 : 0;
            allu &= uni ? 1 : 0;
            if (it.qeval && !__all_sync(0xffffffffu, uni) && lane == 0) atomicOr(&s_act[ch >> 5], 1u << (ch & 31));
        }
    }
    // Every node forced to its own label: the labels stand (the cut would
    // reproduce them), so the cut is skipped.
    allf = need_caps ? __syncthreads_and(allf) : (__syncthreads(), 0);
    if (A.sched) {
        const int quiet = __syncthreads_and(allu) && allf;
        if (tid == 0) {
            // 0: not forced; 1: quiet; 2: forced with active chunks.  The
            // first iteration of a launch (no evaluation) leaves 3.
            sv.qs[k] = (uint8_t)(!it.qeval ? 3 : (quiet ? 1 : (allf ? 2 : 0)));
            s_pm = quiet ? 0u : (1u << 13);      // a block that is not quiet is updated
        }
        if (tid < CHUNK_WORDS) {
            sv.act[(size_t)k * CHUNK_WORDS + tid] = s_act[tid];
            sv.dsc[(size_t)k * CHUNK_WORDS + tid] = 0u;
            if (!it.qeval) sv.duc[(size_t)k * CHUNK_WORDS + tid] = 0u;
        }
    }
    if (allf) {
        if (it.qeval) {
            __syncthreads();
            wl_push_mask(g, k, s_pm, sv.umark, sv.uq + (size_t)(it.t & 1) * g.K, &sv.uq_n[it.t & 1],
                         wl_mark(A.epoch, it.t));
            __syncthreads();
        }
        return;
    }
    cut_block<CONN, SA>(A, k, smem, bw, pl, imask, c_start, nullptr);
    if (A.sched && tid == 0) atomicAdd(&A.ctrl->cuts[it.t & 1], 1u);
    if (it.qeval) {
        // blocks next to a face pixel whose label changed get updated too, and
        // the chunks of those neighbours are marked for their update
        unsigned pm = 0;
#pragma unroll 1
        for (int q = 0; q < NPTMAX; ++q) {
            const int v = tid + q * NT;
            if (v >= B) continue;
            const int nl = __ldcg(&A.yhat[(long long)k * B + v]);
            const int f = A.faceIndex[v];
            if (nl != (int)((oldlab >> q) & 1u) && f >= 0) {
#pragma unroll
                for (int d = 0; d < CONN; ++d) {
                    int kn, ln, fn;
                    const int e = A.halo[d * g.F + f];
                    if (halo_decode(g, e, kz, ky, kx, kn, ln, fn)) {
                        pm |= 1u << (e >> 24);
                        chunk_mark(sv.duc, kn, fn);
                    }
                }
            }
        }
        pm = __reduce_or_sync(0xffffffffu, pm);
        if ((tid & 31) == 0 && pm) atomicOr(&s_pm, pm);
        __syncthreads();
        wl_push_mask(g, k, s_pm, sv.umark, sv.uq + (size_t)(it.t & 1) * g.K, &sv.uq_n[it.t & 1],
                     wl_mark(A.epoch, it.t));
        __syncthreads();
    }
}

// Steps a5-a6 on the graph the build left in shared memory (res, C64, capsum,
// st): exact folding, push-relabel, canonical cut, labels to A.yhat (and to
// lab_smem when given), statistics.
template <int CONN, class SA>
__device__ __forceinline__ void cut_block(const SA& __restrict__ A, int k, unsigned char* smem, int bw, int pl,
                                       unsigned long long imask, long long c_start, uint8_t* lab_smem,
                                       bool to_global) {
    const Geo& g = A.g;
    const int B = g.B;
    const int tid = threadIdx.x, NT = blockDim.x;
    int* res_p = reinterpret_cast<int*>(smem);
    long long* C64_p = reinterpret_cast<long long*>(res_p + CONN * B);
    int* capsum_p = reinterpret_cast<int*>(C64_p + B);
    const SArr<int> res(res_p, (long long)CONN * B);
    const SArr<long long> C64(C64_p, B);
    const SArr<int> e(reinterpret_cast<int*>(C64_p), B);
    const SArr<int> ein(reinterpret_cast<int*>(C64_p) + B, B);
    const SArr<int> capsum(capsum_p, B);
    const SArr<int16_t> hA(reinterpret_cast<int16_t*>(capsum_p), B);
    const SArr<int16_t> hB(reinterpret_cast<int16_t*>(capsum_p) + B, B);
    const SArr<uint8_t> st(reinterpret_cast<uint8_t*>(capsum_p + B), B);
    const SArr<uint32_t> bits(reinterpret_cast<uint32_t*>(smem + solver_bits_offset(CONN, B)),
                              (long long)(CONN + 3) * ((B + 31) / 32));
    const SArr<int16_t> flist(reinterpret_cast<int16_t*>(smem + solver_list_offset(CONN, B)), B);
    __shared__ int s_nf;
    const long long c_built = clock64();
    long long c_bfs = 0;
    int levels = 0, bfs_max = 0;

    // 2. exact folding of forced nodes.  The first round scans every node and
    // lists the nodes it leaves free (flist, s_nf of them, in no particular
    // order: every pass below decides each node from values fixed for the
    // pass, so the order does not matter); later rounds, the unary
    // conversion and the push-relabel pulses visit only the list.  Nodes fixed
    // by later rounds stay in the list and are skipped by their state.
    if (tid == 0) s_nf = 0;
    __syncthreads();             // the count starts at 0 before any warp appends
    int round = 0;
    const int rounds = A.fold_rounds > 0 ? A.fold_rounds : 1;   // the first round builds the list
    for (; round < rounds; ++round) {
        int changed = 0;
        if (round == 0) {
#pragma unroll 1
            for (int q = 0; q < NPTMAX; ++q) {
                int v = tid + q * NT;
                bool fr = false;
                if (v < B && st[v] == FREE) {
                    const long long c = C64[v];
                    const long long cs = capsum[v];
                    int ns = (c >= cs) ? FIX0 : (c < -cs ? FIX1 : FREE);
                    if (ns != FREE) {
                        st[v] = (uint8_t)ns;
#pragma unroll
                        for (int d = 0; d < CONN; ++d) res[d * B + v] = 0;
                        changed = 1;
                    } else {
                        fr = true;
                    }
                }
                // warp-aggregated append to the free-node list
                const unsigned m = __ballot_sync(0xffffffffu, fr);
                int base = 0;
                if ((tid & 31) == 0 && m) base = atomicAdd(&s_nf, __popc(m));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (fr) flist[base + __popc(m & ((1u << (tid & 31)) - 1u))] = (int16_t)v;
            }
        } else {
            const int nf0 = s_nf;
#pragma unroll 1
            for (int i = tid; i < nf0; i += NT) {
                const int v = flist[i];
                if (st[v] != FREE) continue;
                const long long c = C64[v];
                const long long cs = capsum[v];
                int ns = (c >= cs) ? FIX0 : (c < -cs ? FIX1 : FREE);
                if (ns != FREE) {
                    st[v] = (uint8_t)ns;
#pragma unroll
                    for (int d = 0; d < CONN; ++d) res[d * B + v] = 0;
                    changed = 1;
                }
            }
        }
        // stop when nothing changed, or when no node is left free
        __syncthreads();
        const int nfl = s_nf;
        int left = 0;
#pragma unroll 1
        for (int i = tid; i < nfl; i += NT) left |= st[flist[i]] == FREE;
        const int any_changed = __syncthreads_or(changed);
        if (!any_changed || !__syncthreads_or(left)) { round += any_changed; break; }
#pragma unroll 1
        for (int i = tid; i < nfl; i += NT) {
            const int v = flist[i];
            if (st[v] == FREE) {
                long long c = C64[v];
                int cs = capsum[v];
#pragma unroll
                for (int d = 0; d < CONN; ++d) {
                    const int r = res[d * B + v];
                    if (r > 0) {
                        const int su = st[v + dir_lofs<CONN>(d, bw, pl)];
                        if (su != FREE) {
                            c += (su == FIX0) ? r : -r;
                            cs -= r;
                            res[d * B + v] = 0;
                        }
                    }
                }
                C64[v] = c;
                capsum[v] = cs;
            }
        }
        __syncthreads();
    }
    __syncthreads();
    const int nlist = s_nf;

    // unaries of free nodes (|C| < 2^28) -> R2 as int32, then R1 becomes e / ein
    // and R2 the heights (only the free nodes' entries are used from here on)
    int nfree = 0;
#pragma unroll 1
    for (int i = tid; i < nlist; i += NT) {
        const int v = flist[i];
        const bool fr = st[v] == FREE;
        capsum[v] = fr ? (int)C64[v] : 0;
        nfree += fr;
    }
    __syncthreads();
#pragma unroll 1
    for (int i = tid; i < nlist; i += NT) {
        const int v = flist[i];
        e[v] = capsum[v];
        ein[v] = 0;
    }
    const long long c_folded = clock64();
    const int HMAX = B + 1;
    int pulses = 0;
    SArr<int16_t> hc = hA;
    SArr<int16_t> hn = hB;
    if (__syncthreads_or(nfree)) {
        // 3. push-relabel (phase 1: maximum preflow)
        long long cb = clock64();
        int lv0 = levels;
        int active = bfs_bits<CONN>(res, e, hc, st, bits, bw, pl, B, HMAX, tid, NT, levels);
        bfs_max = max(bfs_max, levels - lv0);
        c_bfs += clock64() - cb;
        const int period = A.relabel_period;
        while (active) {
            if (pulses >= A.max_pulses) {
                if (tid == 0) set_status(A.ctrl, 6 /* DOPE_ETIMEOUT */);
                break;
            }
            // push: heights hc fixed for the whole phase (free nodes only: a
            // free node's residual edges all lead to free nodes)
#pragma unroll 1
            for (int i = tid; i < nlist; i += NT) {
                const int v = flist[i];
                if (st[v] == FREE) {
                    int ev = e[v];
                    const int hv = hc[v];
                    if (ev > 0 && hv < HMAX) {
#pragma unroll
                        for (int d = 0; d < CONN; ++d) {
                            if (ev == 0) break;
                            const int r = res[d * B + v];
                            if (r > 0) {
                                const int u = v + dir_lofs<CONN>(d, bw, pl);
                                if (hc[u] == hv - 1) {
                                    const int dl = min(ev, r);
                                    res[d * B + v] = r - dl;
                                    res[opp_dir<CONN>(d) * B + u] += dl;
                                    atomicAdd(&ein[u], dl);
                                    ev -= dl;
                                }
                            }
                        }
                        e[v] = ev;
                    }
                }
            }
            __syncthreads();
            // merge incoming flow, relabel into hn (a fixed node's height is
            // never read: no residual edge leads to it)
            int act = 0;
#pragma unroll 1
            for (int i = tid; i < nlist; i += NT) {
                const int v = flist[i];
                int hv = hc[v];
                if (st[v] == FREE) {
                    const int ev = e[v] + ein[v];
                    ein[v] = 0;
                    e[v] = ev;
                    if (ev > 0 && hv < HMAX) {
                        int mn = HMAX;
                        bool adm = false;
#pragma unroll
                        for (int d = 0; d < CONN; ++d) {
                            if (res[d * B + v] > 0) {
                                const int hu = hc[v + dir_lofs<CONN>(d, bw, pl)];
                                adm |= (hu == hv - 1);
                                mn = min(mn, hu);
                            }
                        }
                        if (!adm) hv = min(mn + 1, HMAX);
                        if (hv < HMAX) act = 1;
                    }
                }
                hn[v] = (int16_t)hv;
            }
            active = __syncthreads_or(act);
            const SArr<int16_t> tmp = hc; hc = hn; hn = tmp;
            ++pulses;
            if (active && period > 0 && (pulses % period) == 0) {
                cb = clock64();
                lv0 = levels;
                active = bfs_bits<CONN>(res, e, hc, st, bits, bw, pl, B, HMAX, tid, NT, levels);
                bfs_max = max(bfs_max, levels - lv0);
                c_bfs += clock64() - cb;
            }
        }
        // 4. canonical cut
        cb = clock64();
        lv0 = levels;
        bfs_bits<CONN>(res, e, hc, st, bits, bw, pl, B, HMAX, tid, NT, levels);
        bfs_max = max(bfs_max, levels - lv0);
        c_bfs += clock64() - cb;
    }
    const long long c_end = clock64();

    // 6. labels
#pragma unroll 1
    for (int q = 0; q < NPTMAX; ++q) {
        int v = tid + q * NT;
        if (v >= B) continue;
        uint8_t lab;
        if (st[v] == FIX0) lab = 0;
        else if (st[v] == FIX1) lab = 1;
        else lab = (hc[v] < HMAX) ? 1 : 0;
        if (to_global) A.yhat[(long long)k * B + v] = lab;
        if (lab_smem) lab_smem[v] = lab;
    }
    int nf = 0;
#pragma unroll 1
    for (int q = 0; q < NPTMAX; ++q) {
        int v = tid + q * NT;
        if (v < B && st[v] == FREE) nf++;
    }
    // statistics
    for (int o = 16; o > 0; o >>= 1) nf += __shfl_xor_sync(0xffffffffu, nf, o);
    if ((tid & 31) == 0 && nf) atomicAdd(&A.ctrl->free_total, (unsigned long long)nf);
    if (tid == 0) {
        if (pulses) {
            atomicAdd(&A.ctrl->pulses_total, (unsigned long long)pulses);
            atomicMax(&A.ctrl->pulses_max, pulses);
        }
        atomicAdd(&A.ctrl->cyc[0], (unsigned long long)(c_built - c_start));
        atomicAdd(&A.ctrl->cyc[1], (unsigned long long)(c_folded - c_built));
        atomicAdd(&A.ctrl->cyc[2], (unsigned long long)(c_end - c_folded - c_bfs));
        atomicAdd(&A.ctrl->cyc[3], (unsigned long long)c_bfs);
        if (levels) atomicAdd(&A.ctrl->bfs_levels, (unsigned long long)levels);
        atomicMax(&A.ctrl->bfs_levels_max, bfs_max);
        atomicMax(&A.ctrl->fold_rounds_max, round);
    }
    __syncthreads();   // shared memory is reused by the next block / phase
}

// One launch = one iteration's block solves (steps a4-a6), one CTA per block.
// With check_prev, the CTA first evaluates the stop test of the previous
// iteration (Algorithm 1's loop condition) and returns if it holds.
template <int CONN>
__global__ void __launch_bounds__(512, 2) k_block_solve(SolveArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_skip;
    if (threadIdx.x == 0) {
        int skip = 0;
        if (A.check_prev) {
            if (*(volatile int*)&A.ctrl->conv_t) {
                skip = 1;
            } else {
                double r2 = __longlong_as_double((long long)__ldcg(&A.ctrl->r2max[A.t - 1]));
                if (!(__dsqrt_rn(r2) > A.eps)) {
                    skip = 1;
                    if (blockIdx.x == 0) atomicCAS(&A.ctrl->conv_t, 0, A.t - 1);
                }
            }
        }
        s_skip = skip;
    }
    __syncthreads();
    if (s_skip) return;
    solve_block<CONN>(A, iter_of(A), blockIdx.x, smem);
}

// ---------------------------------------------------------------------------
// Steps a2 + a3: Eq. 10 / Eq. 11 on the face pixels and the per-block stop
// quantity r2_k = sum_{i in block k} (yhat_i - y_i)^2 (interior pixels add
// exactly 0).  One CTA per block; face slots strided over its threads.
//   G_i = sum_{j in X(i)} Wl_ij (yhat_i - yhat_j)        (exact, integer)
//   y_i = (yhat_i + a_i) - (G_i / 1024) / mu               (Eq. 10)
//   a_i = a_i + (yhat_i - y_i)                             (Eq. 11)
// ---------------------------------------------------------------------------
// One warp: Eq. 10 / Eq. 11 on chunk ch (32 face slots) of block k.  Returns
// the chunk's sum of (yhat - y)^2 (every lane: the butterfly's result) and the
// offset codes of the blocks to solve next iteration (OR over the warp).
template <int CONN, class UA>
__device__ __forceinline__ void update_chunk(const UA& __restrict__ A, double mu, int t, int k, int ch, int selfpush,
                                             const SchedView& sv, double& d2_out, unsigned& pm_out) {
    const Geo& g = A.g;
    const int lane = threadIdx.x & 31;
    constexpr int nh = CONN / 2;
    const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
    const bool wl = A.sched != nullptr;
    const int f = ch * 32 + lane;
    double d2 = 0.0;
    unsigned pm = 0;
    int fj[CONN], kj[CONN];   // face slot and block of each cross neighbour (block -1: none)
#pragma unroll
    for (int d = 0; d < CONN; ++d) {
        kj[d] = -1;
        fj[d] = 0;
    }
    if (f < g.F) {
        const int v = A.faceLocal[f];
        const long long gi = (long long)k * g.B + v;
        int wj[CONN], yj[CONN];
        unsigned cm = 0;      // offset codes of the blocks holding this pixel's cross neighbours
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            int kn, ln, fn;
            wj[d] = 0;
            yj[d] = 0;
            const int e = A.halo[d * g.F + f];
            if (halo_decode(g, e, kz, ky, kx, kn, ln, fn)) {
                const long long gj = (long long)kn * g.B + ln;
                wj[d] = (d < nh) ? A.Wl[(long long)d * g.N + gi] : A.Wl[(long long)(d - nh) * g.N + gj];
                yj[d] = __ldcg(&A.yhat[gj]);
                cm |= 1u << (e >> 24);
                kj[d] = kn;
                fj[d] = fn;
            }
        }
        const int yh = __ldcg(&A.yhat[gi]);
        int G = 0;
#pragma unroll
        for (int d = 0; d < CONN; ++d) G += wj[d] * (yh - yj[d]);
        const long long s = (long long)k * g.F + f;
        const double yo = __ldcg(&A.yF[s]);
        const double ao = __ldcg(&A.aF[s]);
        const double aa = t == 1 ? 0.0 : ao;   // a = 0 before iteration 1
        double yn, an;
        if (G == 0 && __double_as_longlong(aa) == 0) {
            // the operations below with G = 0 and a = +0: y = yhat + (+0) = yhat,
            // a = +0 + (yhat - y) = +0, (yhat - y)^2 = +0
            yn = (double)yh;
            an = 0.0;
        } else {
            const double gq = __dmul_rn((double)G, 0.0009765625);   // G / 1024, exact
            // G = 0: (G/1024)/mu = +0 and x - (+0) = x exactly, so the division is skipped
            const double ya = __dadd_rn((double)yh, aa);
            yn = G ? __dsub_rn(ya, __ddiv_rn(gq, mu)) : ya;
            an = __dadd_rn(aa, __dsub_rn((double)yh, yn));
            const double dd = __dsub_rn((double)yh, yn);
            d2 = __dmul_rn(dd, dd);
        }
        // only what changed is written back
        bool changed = __double_as_longlong(yn) != __double_as_longlong(yo) ||
                       __double_as_longlong(an) != __double_as_longlong(ao);
        if (changed) {
            A.yF[s] = yn;
            A.aF[s] = an;
        }
        if (wl) {
            if ((int)__ldcg(&sv.yhF[s]) != yh) {
                sv.yhF[s] = (uint8_t)yh;
                changed = true;
            }
            if (changed) pm = cm | (1u << 13);
        }
    }
    if (wl && !selfpush) {
        // this slot's and its cross neighbours' Eq. 8 inputs changed: their
        // blocks are solved next iteration and these chunks evaluated (one
        // atomic per distinct chunk of the warp; the first iteration of a
        // launch needs none, every block's next solve is a full one)
        const bool ch_me = pm != 0;
        const unsigned lanes = __ballot_sync(0xffffffffu, ch_me);
        if (ch_me && lane == __ffs(lanes) - 1) chunk_mark(sv.dsc, k, f);
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            const bool mk = ch_me && kj[d] >= 0;
            const unsigned key = mk ? (unsigned)kj[d] * 128u + (unsigned)(fj[d] >> 5) : 0xffffffffu;
            const unsigned grp = __match_any_sync(0xffffffffu, key);
            if (mk && lane == __ffs(grp) - 1) chunk_mark(sv.dsc, kj[d], fj[d]);
        }
    }
    if (__any_sync(0xffffffffu, d2 != 0.0))
        for (int o = 16; o > 0; o >>= 1) d2 = __dadd_rn(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    if (wl) pm = __reduce_or_sync(0xffffffffu, pm);
    d2_out = d2;
    pm_out = pm;
}

// Eq. 10 / Eq. 11 on up to MB blocks kk[0..nb) of one problem.  Each block's
// chunks to update are chosen first: every chunk in a full iteration (full !=
// 0: the first of a launch, or no worklists) or of a block that is not
// forced; a forced block's active chunks and those holding a slot whose cross
// neighbour's label changed otherwise (every other slot is trivial with G =
// 0: its update is the identity and adds +0 to r_k^2).  The chunks of all the
// blocks are spread over the CTA's warps, so their load latencies overlap;
// each block's r_k^2 is then summed in a fixed order, whatever the CTA shape
// (slots in chunks of 32, each chunk by the same butterfly, chunks in
// increasing order), and its pushes made by its own warp.
template <int CONN, class UA>
__device__ void update_blocks(const UA& __restrict__ A, double mu, int t, const int* kk, int nb, int full) {
    const Geo& g = A.g;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const bool wl = A.sched != nullptr;
    const SchedView sv = sched_view(A.sched, g.K);
    UpdSmem& us = upd_smem();
    double (&partm)[MB][128] = us.part;
    unsigned (&pmm)[MB][128] = us.pm;
    unsigned (&s_dom)[MB][CHUNK_WORDS] = us.dom;
    const int nchunks = (g.F + 31) >> 5;
    if (tid < nb * CHUNK_WORDS) {
        const int j = tid / CHUNK_WORDS, w = tid % CHUNK_WORDS;
        const int hi = nchunks - w * 32;
        const unsigned all = hi <= 0 ? 0u : (hi >= 32 ? 0xffffffffu : ((1u << hi) - 1u));
        unsigned m = all;
        int q = 0;
        if (wl && !full) {   // (a full iteration reads no list state)
            const size_t o = (size_t)kk[j] * CHUNK_WORDS + w;
            q = __ldcg(&sv.qs[kk[j]]);
            const unsigned du = __ldcg(&sv.duc[o]);
            if (q == 1 || q == 2) m = (__ldcg(&sv.act[o]) | du) & all;
            if (du) sv.duc[o] = 0u;
        }
        s_dom[j][w] = m;
        if (w == 0) us.qb[j] = q;
    }
    __syncthreads();
    if (tid == 0) {
        int tot = 0;
        for (int j = 0; j < nb; ++j)
            for (int w = 0; w < CHUNK_WORDS; ++w) tot += __popc(s_dom[j][w]);
        us.tot = tot;
    }
    __syncthreads();
    const int tot = us.tot;
    for (int tk = wid; tk < tot; tk += nw) {
        int r = tk, j = 0, w = 0;
        for (;;) {
            const int c = __popc(s_dom[j][w]);
            if (r < c) break;
            r -= c;
            if (++w == CHUNK_WORDS) { w = 0; ++j; }
        }
        unsigned m = s_dom[j][w];
        for (int i = 0; i < r; ++i) m &= m - 1;
        const int ch = w * 32 + __ffs(m) - 1;
        double d2;
        unsigned pm;
        update_chunk<CONN>(A, mu, t, kk[j], ch, full, sv, d2, pm);
        if (lane == 0) {
            partm[j][ch] = d2;
            pmm[j][ch] = pm;
        }
    }
    __syncthreads();
    if (wid < nb && lane == 0) {
        const int j = wid, k = kk[j];
        double r2 = 0.0;
        unsigned m = 0;
        for (int ch = 0; ch < nchunks; ++ch) {
            if (!((s_dom[j][ch >> 5] >> (ch & 31)) & 1u)) continue;   // +0: adds nothing
            r2 = __dadd_rn(r2, partm[j][ch]);
            m |= pmm[j][ch];
        }
        A.r2blk[k] = r2;
        if (r2 != 0.0) atomicMax(&A.ctrl->r2max[t], (unsigned long long)__double_as_longlong(r2));
        // the blocks next to a face pixel whose state changed (and this block,
        // if it changed or is not quiet) are solved next iteration
        if (full || us.qb[j] != 1) m |= 1u << 13;
        us.mm[j] = m;
    }
    __syncthreads();
    if (wl && wid < nb && lane < 27) {
        const int j = wid, k = kk[j];
        const unsigned m = us.mm[j];
        if ((m >> lane) & 1u) {
            const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
            const int nkz = kz + lane / 9 - 1, nky = ky + (lane / 3) % 3 - 1, nkx = kx + lane % 3 - 1;
            if (nkz >= 0 && nkz < g.nbz && nky >= 0 && nky < g.nby && nkx >= 0 && nkx < g.nbx)
                wl_push(sv.smark, sv.sq + (size_t)((t + 1) & 1) * g.K, &sv.sq_n[(t + 1) & 1],
                        (nkz * g.nby + nky) * g.nbx + nkx, wl_mark(A.epoch, t + 1));
        }
    }
    __syncthreads();
}

// One block's update (see update_blocks).
template <int CONN, class UA>
__device__ __forceinline__ void update_block(const UA& __restrict__ A, double mu, int t, int k, int full) {
    const int kk[1] = {k};
    update_blocks<CONN>(A, mu, t, kk, 1, full);
}

// One launch = one iteration's Eq. 10 / Eq. 11 update, one CTA per block.
template <int CONN>
__global__ void __launch_bounds__(256) k_face_update(UpdArgs A) {
    if (*(volatile int*)&A.ctrl->conv_t) return;
    update_block<CONN>(A, A.mu, A.t, blockIdx.x, 0);
}

// Threads of a k_face_update CTA (one CTA per block) for F face slots.
inline int face_update_threads(int F) {
    int t = (F + 31) / 32 * 32;
    return t < 32 ? 32 : (t > 256 ? 256 : t);
}

// ---------------------------------------------------------------------------
// Set-up, finish and test-hook kernels (image order <-> block-major)
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long bm_index(const Geo& g, long long i) {
    const int x = (int)(i % g.W);
    const long long r = i / g.W;
    const int y = (int)(r % g.H);
    const int z = (int)(r / g.H);
    const int k = ((z / g.bd) * g.nby + (y / g.bh)) * g.nbx + (x / g.bw);
    const int l = ((z % g.bd) * g.bh + (y % g.bh)) * g.bw + (x % g.bw);
    return (long long)k * g.B + l;
}

// Caller-grid index of padded pixel (z, y, x), or -1 for a padding pixel.
__device__ __forceinline__ long long user_index(const Geo& g, int z, int y, int x) {
    if (z >= g.Du || y >= g.Hu || x >= g.Wu) return -1;
    return ((long long)z * g.Hu + y) * g.Wu + x;
}

// U = rne(1024 u); |U| < 2^30 and u finite, else DOPE_EOVERFLOW.  Padding
// pixels get 0.
#ifndef DOPE_KERNEL_TEMPLATES_ONLY
__global__ void k_set_unaries(Geo g, const float* __restrict__ u, int32_t* __restrict__ U, Ctrl* c) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.W);
        const long long r = i / g.W;
        const int y = (int)(r % g.H);
        const int z = (int)(r / g.H);
        const long long iu = user_index(g, z, y, x);
        int q = 0;
        if (iu >= 0) {
            const double v = __dmul_rn(1024.0, (double)u[iu]);
            if (!(fabs(v) < 1073741823.5)) set_status(c, 4);
            else q = (int)__double2ll_rn(v);
        }
        U[bm_index(g, i)] = q;
    }
}
#endif

// Wl = rne(lambda wq); wq >= 0 (else DOPE_EUNSUPPORTED), zero toward the
// outside of the grid (else DOPE_EINVAL), Wl < 2^24 (else DOPE_EOVERFLOW).
template <int CONN>
__global__ void k_set_weights(Geo g, const int32_t* __restrict__ wq, int32_t* __restrict__ Wl,
                              double lambda, Ctrl* c, int allow_negative) {
    constexpr int nh = CONN / 2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.W);
        const long long r = i / g.W;
        const int y = (int)(r % g.H);
        const int z = (int)(r / g.H);
        const long long b = bm_index(g, i);
        const long long iu = user_index(g, z, y, x);
#pragma unroll
        for (int d = 0; d < nh; ++d) {
            int dz, dy, dx;
            dir_off<CONN>(d, dz, dy, dx);
            if (iu < 0) {           // padding pixel: no n-links
                Wl[(long long)d * g.N + b] = 0;
                continue;
            }
            const int w = wq[(long long)d * g.Nu + iu];
            int q = 0;
            const bool inside = (z + dz >= 0) && (z + dz < g.Du) && (y + dy >= 0) && (y + dy < g.Hu) &&
                                (x + dx >= 0) && (x + dx < g.Wu);
            if (w < 0 && !allow_negative) set_status(c, 2);
            else if (!inside && w != 0) set_status(c, 1);
            else {
                const double v = __dmul_rn(lambda, (double)w);
                if (!(fabs(v) < 16777215.5)) set_status(c, 4);
                else q = (int)__double2ll_rn(v);
            }
            Wl[(long long)d * g.N + b] = q;
        }
    }
}

#ifndef DOPE_KERNEL_TEMPLATES_ONLY
__global__ void k_init_state(Geo g, double* yF, double* aF) {
    const long long n = (long long)g.K * g.F;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        yF[i] = 0.5;
        aF[i] = 0.0;
    }
}
#endif

// labels (caller's image order, padding dropped) <- yhat (block-major)
#ifndef DOPE_KERNEL_TEMPLATES_ONLY
__global__ void k_unpermute_u8(Geo g, const uint8_t* __restrict__ src, uint8_t* __restrict__ dst) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.Nu;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.Wu);
        const long long r = i / g.Wu;
        const int y = (int)(r % g.Hu);
        const int z = (int)(r / g.Hu);
        dst[i] = src[bm_index(g, ((long long)z * g.H + y) * g.W + x)];
    }
}
#endif

#ifndef DOPE_KERNEL_TEMPLATES_ONLY
__global__ void k_permute_u8(Geo g, const uint8_t* __restrict__ src, uint8_t* __restrict__ dst) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
         i += (long long)gridDim.x * blockDim.x)
        dst[bm_index(g, i)] = src[i];
}
#endif

#ifndef DOPE_KERNEL_TEMPLATES_ONLY
__global__ void k_permute_i64(Geo g, const long long* __restrict__ src, long long* __restrict__ dst) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
         i += (long long)gridDim.x * blockDim.x)
        dst[bm_index(g, i)] = src[i];
}
#endif

// E_int of block-major labels (Eq. 1, each undirected edge once), int64.
template <int CONN>
__global__ void k_energy(Geo g, const int32_t* __restrict__ U, const int32_t* __restrict__ Wl,
                         const uint8_t* __restrict__ lab, Ctrl* c) {
    constexpr int nh = CONN / 2;
    long long acc = 0;
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < g.N;
         gi += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(gi / g.B), v = (int)(gi % g.B);
        const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
        const int lx = v % g.bw, ly = (v / g.bw) % g.bh, lz = v / (g.bw * g.bh);
        const int yi = lab[gi];
        acc += (long long)U[gi] * yi;
#pragma unroll
        for (int d = 0; d < nh; ++d) {
            int dz, dy, dx;
            dir_off<CONN>(d, dz, dy, dx);
            const int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
            long long gj;
            if (nlz < g.bd && nly < g.bh && nlx >= 0 && nlx < g.bw) {
                gj = gi + (dz * g.bh + dy) * g.bw + dx;
            } else {
                int kn, ln;
                if (!cross_nbr<CONN>(g, kz, ky, kx, lz, ly, lx, d, kn, ln)) continue;
                gj = (long long)kn * g.B + ln;
            }
            if (yi != lab[gj]) acc += Wl[(long long)d * g.N + gi];
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&c->energy, (unsigned long long)acc);
}

// Dense state (image order) from the face state.
#ifndef DOPE_KERNEL_TEMPLATES_ONLY
__global__ void k_get_state(Geo g, const double* yF, const double* aF, const uint8_t* yhat,
                            const int16_t* faceIndex, int t, double* y, double* a, uint8_t* yh) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = bm_index(g, i);
        const int k = (int)(b / g.B), v = (int)(b % g.B);
        const int f = faceIndex[v];
        const uint8_t lab = yhat[b];
        double yv, av;
        if (f >= 0) { yv = yF[(long long)k * g.F + f]; av = aF[(long long)k * g.F + f]; }
        else { yv = t == 0 ? 0.5 : (double)lab; av = 0.0; }
        if (y) y[i] = yv;
        if (a) a[i] = av;
        if (yh) yh[i] = t == 0 ? 0 : lab;
    }
}
#endif

// Face state from a dense state; checks the interior invariant.
#ifndef DOPE_KERNEL_TEMPLATES_ONLY
__global__ void k_set_state(Geo g, const double* y, const double* a, const uint8_t* yh,
                            const int16_t* faceIndex, int t, double* yF, double* aF,
                            uint8_t* yhat, Ctrl* c) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = bm_index(g, i);
        const int k = (int)(b / g.B), v = (int)(b % g.B);
        const int f = faceIndex[v];
        const uint8_t lab = yh[i];
        if (lab > 1) set_status(c, 1);
        yhat[b] = lab;
        if (t == 0) {
            if (y[i] != 0.5 || a[i] != 0.0) set_status(c, 1);
        } else if (f < 0) {
            if (y[i] != (double)lab || a[i] != 0.0) set_status(c, 1);
        }
        if (f >= 0) { yF[(long long)k * g.F + f] = y[i]; aF[(long long)k * g.F + f] = a[i]; }
    }
}
#endif

// Step a4 alone: Eq. 8 unaries of every pixel (image order) for the state.
template <int CONN>
__global__ void k_shifted_caps(Geo g, const int32_t* U, const int32_t* Wl, const uint8_t* yhat,
                               const double* yF, const double* aF, const int16_t* faceIndex,
                               int first, double mu, long long* out) {
    const double m1024 = __dmul_rn(1024.0, mu);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = bm_index(g, i);
        const int k = (int)(b / g.B), v = (int)(b % g.B);
        const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
        const int lx = v % g.bw, ly = (v / g.bw) % g.bh, lz = v / (g.bw * g.bh);
        out[i] = shifted_cap<CONN>(g, U, Wl, yhat, yF, aF, faceIndex, k, kz, ky, kx, v, lz, ly, lx,
                                   first, m1024);
    }
}


// ---------------------------------------------------------------------------
// Persistent path: all of Algorithm 1 in one cooperative launch.
//
// Every CTA owns blocks k = blockIdx.x, blockIdx.x + gridDim.x, ...  Each
// iteration: solve the owned blocks (a4-a6), grid barrier, update their face
// state (a2-a3), grid barrier, then every CTA reads the same max_k r_k^2 and
// takes the same decision (a3); mu <- mu * mu_fact (a7) on the device, the
// same double multiplication as the host sequence.  Mutable state is read
// with L2 loads (__ldcg) since it is written by other CTAs within the launch.
// ---------------------------------------------------------------------------
struct PersistArgs {
    SolveArgs s;
    UpdArgs u;
    int t0, n;              // run iterations t0+1 .. t0+n
    double mu_start, mu_fact;
    long long spin_limit;   // SM cycles a barrier wait may take before giving up
    int dynamic;            // blocks handed out by an atomic counter (K > grid)
    int window;             // resident kernel: run-ahead windows of frozen iterations
    int NH;                 // halo pixels of a block (distinct cross-block neighbours)
    const int16_t* hslot;   // [CONN][F] halo pixel of (direction, face slot), -1 if none
    const int* hinfo;       // [NH] halo_entry of each halo pixel
    int wl_cont;            // 1: the worklists left by the previous launch hold (first iteration uses them)
    uint8_t* out_labels;    // finish (a8) in the launch: labels in the caller's image order (or null)
    int out_energy;         // finish (a8) in the launch: E_int of the labels into ctrl->energy
    int lwin;               // persistent kernel: run-ahead windows over the worklists
    int lwcap;              // their longest window the dynamic shared memory holds
    unsigned long long* wslot;   // [K][F] window entry slots: G (low 32 bits), bound (high, float)
    unsigned long long* wtag;    // [K] tag of the last window that had the block on its list
    unsigned* wmask;             // [K][4] that window's entry chunks of the block
    double* wst;                 // [K][F][4] states (y, a) after a window's last two iterations
};

// Step a8 for block k at the end of a persistent launch (after a grid
// barrier, so every block's final labels are in yhat): the block's labels in
// the caller's image order, and the block's share of E_int (its unaries and
// the edges leaving its pixels forward, each undirected edge once) added to
// ctrl->energy.  Every thread of the CTA calls it.
template <int CONN>
__device__ void finish_block(const PersistArgs& P, int k, long long* red) {
    const Geo& g = P.s.g;
    constexpr int nh = CONN / 2;
    const int B = g.B;
    const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
    long long acc = 0;
    for (int v = threadIdx.x; v < B; v += blockDim.x) {
        const int lx = v % g.bw, ly = (v / g.bw) % g.bh, lz = v / (g.bw * g.bh);
        const long long gi = (long long)k * B + v;
        const int yi = __ldcg(&P.s.yhat[gi]);
        if (P.out_labels) {
            const int z = kz * g.bd + lz, y = ky * g.bh + ly, x = kx * g.bw + lx;
            if (z < g.Du && y < g.Hu && x < g.Wu) P.out_labels[((long long)z * g.Hu + y) * g.Wu + x] = (uint8_t)yi;
        }
        if (P.out_energy) {
            acc += (long long)P.s.U[gi] * yi;
#pragma unroll
            for (int d = 0; d < nh; ++d) {
                int dz, dy, dx;
                dir_off<CONN>(d, dz, dy, dx);
                const int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
                long long gj;
                if (nlz < g.bd && nly < g.bh && nlx >= 0 && nlx < g.bw) {
                    gj = gi + (dz * g.bh + dy) * g.bw + dx;
                } else {
                    int kn, ln;
                    if (!cross_nbr<CONN>(g, kz, ky, kx, lz, ly, lx, d, kn, ln)) continue;
                    gj = (long long)kn * B + ln;
                }
                if (yi != __ldcg(&P.s.yhat[gj])) acc += P.s.Wl[(long long)d * g.N + gi];
            }
        }
    }
    if (!P.out_energy) return;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        if (t) atomicAdd(&P.s.ctrl->energy, (unsigned long long)t);
    }
    __syncthreads();
}

// Step a8 over the whole grid at the end of a persistent launch, as a flat
// grid-stride loop over the block-major pixel index (coalesced reads of the
// labels, unaries and weight planes; no per-block barriers): labels in the
// caller's image order and E_int (unaries of the labelled pixels plus every
// cut forward edge, each undirected edge once) into ctrl->energy.  The sum is
// in int64 and so exact in any order.  Every thread of every CTA calls it.
template <int CONN>
__device__ void finish_flat(const PersistArgs& P, long long* red) {
    const Geo& g = P.s.g;
    constexpr int nh = CONN / 2;
    const int B = g.B;
    long long acc = 0;
    // N < 2^31 (the context checks it), so the index arithmetic stays in 32 bits
    const unsigned stride = gridDim.x * blockDim.x, n = (unsigned)g.N, ub = (unsigned)B;
    for (unsigned gu = blockIdx.x * blockDim.x + threadIdx.x; gu < n; gu += stride) {
        const long long gi = gu;
        const int k = (int)(gu / ub), v = (int)(gu - (unsigned)k * ub);
        const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
        const int lx = v % g.bw, ly = (v / g.bw) % g.bh, lz = v / (g.bw * g.bh);
        const int yi = __ldcg(&P.s.yhat[gi]);
        if (P.out_labels) {
            const int z = kz * g.bd + lz, y = ky * g.bh + ly, x = kx * g.bw + lx;
            if (z < g.Du && y < g.Hu && x < g.Wu) P.out_labels[((long long)z * g.Hu + y) * g.Wu + x] = (uint8_t)yi;
        }
        if (P.out_energy) {
            acc += (long long)P.s.U[gi] * yi;
#pragma unroll
            for (int d = 0; d < nh; ++d) {
                int dz, dy, dx;
                dir_off<CONN>(d, dz, dy, dx);
                const int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
                long long gj;
                if (nlz < g.bd && nly < g.bh && nlx >= 0 && nlx < g.bw) {
                    gj = gi + (dz * g.bh + dy) * g.bw + dx;
                } else {
                    int kn, ln;
                    if (!cross_nbr<CONN>(g, kz, ky, kx, lz, ly, lx, d, kn, ln)) continue;
                    gj = (long long)kn * B + ln;
                }
                if (yi != __ldcg(&P.s.yhat[gj])) acc += P.s.Wl[(long long)d * g.N + gi];
            }
        }
    }
    if (!P.out_energy) return;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        if (t) atomicAdd(&P.s.ctrl->energy, (unsigned long long)t);
    }
}

// Next block for this CTA: static stride, or the phase's atomic counter.
__device__ __forceinline__ int next_block(int dynamic, unsigned* counter, int k_prev, int* s_k) {
    if (!dynamic) return k_prev < 0 ? (int)blockIdx.x : k_prev + (int)gridDim.x;
    __syncthreads();
    if (threadIdx.x == 0) *s_k = (int)atomicAdd(counter, 1u);
    __syncthreads();
    return *s_k;
}

// Hands out entries [0, n) of a list to the CTAs in pieces of at most MB:
// when n <= MB x grid, one even piece per CTA (n / grid or one more; no
// atomics, so no CTA takes a second piece while others idle); otherwise
// pieces of MB grabbed from *counter (zeroed beforehand) until none is left.
// f(i0, nb) runs with the whole CTA; pieces are separated by __syncthreads.
template <class Fn>
__device__ __forceinline__ void list_pieces(int n, unsigned* counter, int* s_i, Fn&& f) {
    const int G = (int)gridDim.x;
    if (n <= MB * G) {
        const int i0 = (int)((long long)blockIdx.x * n / G);
        const int i1 = (int)((long long)(blockIdx.x + 1) * n / G);
        if (i1 > i0) f(i0, i1 - i0);
        return;
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) *s_i = (int)atomicAdd(counter, (unsigned)MB);
        __syncthreads();
        const int i0 = *s_i;
        if (i0 >= n) break;
        f(i0, n - i0 < MB ? n - i0 : MB);
    }
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  The
// arrival counter only grows: barrier number b of the launch completes when
// it reaches b * nblocks.  Thread 0 arrives with a release RMW (the CTA's
// earlier writes are ordered before it through __syncthreads) and waits with
// acquire loads, so writes made before the barrier by any CTA are visible
// after it.  A wait that exceeds spin_limit sets DOPE_ETIMEOUT and the abort
// flag; every CTA then returns false from this and from later barriers.
// Split form of the barrier: arrive (release) now, wait (acquire) later;
// work placed between the two must not read other CTAs' writes.
__device__ __forceinline__ void grid_arrive(Ctrl* c, unsigned& nbar) {
    __syncthreads();
    ++nbar;
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(c->bar_count);
        cnt.fetch_add(1u, cuda::memory_order_release);
    }
}

__device__ __forceinline__ bool grid_wait(Ctrl* c, unsigned nblocks, unsigned nbar, long long spin_limit) {
    __shared__ int s_okw;
    if (threadIdx.x == 0) {
        int ok = 1;
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(c->bar_count);
        const unsigned target = nbar * nblocks;
        const long long t0 = clock64();
        while (cnt.load(cuda::memory_order_acquire) < target) {
            if (*(volatile int*)&c->abort) { ok = 0; break; }
            if (clock64() - t0 > spin_limit) {
                set_status(c, 6 /* DOPE_ETIMEOUT */);
                atomicExch(&c->abort, 1);
                ok = 0;
                break;
            }
        }
        s_okw = ok;
    }
    __syncthreads();
    return s_okw != 0;
}

__device__ __forceinline__ bool grid_sync(Ctrl* c, unsigned nblocks, unsigned& nbar,
                                          long long spin_limit) {
    __shared__ int s_ok;
    __syncthreads();
    ++nbar;
    if (threadIdx.x == 0) {
        int ok = 1;
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(c->bar_count);
        const unsigned target = nbar * nblocks;
        if (cnt.fetch_add(1u, cuda::memory_order_release) + 1u != target) {
            const long long t0 = clock64();
            while (cnt.load(cuda::memory_order_acquire) < target) {
                if (*(volatile int*)&c->abort) { ok = 0; break; }
                if (clock64() - t0 > spin_limit) {
                    set_status(c, 6 /* DOPE_ETIMEOUT */);
                    atomicExch(&c->abort, 1);
                    ok = 0;
                    break;
                }
            }
        } else {
            cuda::atomic_thread_fence(cuda::memory_order_acquire, cuda::thread_scope_device);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// One Eq. 10 / Eq. 11 step of a face pixel with fixed label yh and cross sum G
// (the operations of update_block, in the same order).
__device__ __forceinline__ double face_step(int yh, int G, double mu, double& y, double& a) {
    const double gq = __dmul_rn((double)G, 0.0009765625);
    const double ya = __dadd_rn((double)yh, a);
    const double yn = G ? __dsub_rn(ya, __ddiv_rn(gq, mu)) : ya;
    a = __dadd_rn(a, __dsub_rn((double)yh, yn));
    y = yn;
    const double dd = __dsub_rn((double)yh, yn);
    return __dmul_rn(dd, dd);
}

// Bytes of dynamic shared memory of the running launch.
__device__ __forceinline__ int dyn_smem_bytes() {
    unsigned r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return (int)r;
}

// ---------------------------------------------------------------------------
// Run-ahead windows of the persistent kernel.  Once an iteration solves no
// block by a cut (every block on the list kept its labels by the forced
// tests), the labels are expected to stay frozen, and then each face slot's
// y and a follow Eq. 10 / Eq. 11 with a constant cross sum G, independently of
// every other slot.  A window advances Wn iterations at once over the blocks
// S on the current solve list, in three phases separated by grid barriers:
//
//  1. traj: for each chunk of S holding a slot that is not trivial or whose
//     Eq. 8 inputs changed (act | dsc, the entry chunks), G and the state at
//     the window start; the slot's (G, bound B) go to wslot, where B bounds
//     |a| and |y - yhat| for every state of the window (with labels frozen,
//     a_t = g / mu_t and y_t - yhat = a_{t-1} - g / mu_t in exact arithmetic,
//     g = G / 1024, each computed step adding a few ulps and no accumulation,
//     so B = |a_tw| + |y_tw - yhat| + 2 |g| / mu_{tw+1} + 2^-40).  The slot's
//     states are stepped through the window with the update's operations and
//     each block's r2 summed per iteration in the update's fixed order, its
//     maximum over S kept per iteration.
//  2. cert: for each face slot of S whose state or a cross neighbour's state
//     may move (an entry slot, or next to one), the Eq. 8 forced test of
//     every window iteration from an interval certificate built on the
//     bounds (at the window's first iteration, the exact unary where the
//     certificate is too weak).  Every other pixel of a block of S
//     is forced by the integer test or its exact interior unary at the
//     block's last solve, and stays so while mu grows.  The first iteration
//     with a slot not proven forced (or a block of S not forced at its last
//     solve) ends the valid run.
//  3. commit: the first valid iteration whose stop test holds, else the last
//     valid one, is the end of the window: every entry slot's state there is
//     replayed from the window start and written, the r2 maxima of the
//     committed iterations copied to the trace, and the worklists left as the
//     iteration after the end expects (the list S, its chunks marked dirty).
//
// Every committed state, residual and stop decision is the one the ordinary
// iterations compute, bit for bit: the labels of the window's iterations are
// those the ordinary solves would keep (every node proven forced), and the
// states are computed by the same operations in the same order.
// ---------------------------------------------------------------------------
struct LWin {
    int tw;                    // last iteration before the window
    int Wn;                    // window iterations tw+1 .. tw+Wn
    double mu;                 // mu of iteration tw+1
    unsigned long long tag;    // tag of this window's blocks (wtag)
    unsigned long long* r2w;   // [LWMAX] bits of max over S of r2_k, by window iteration
    int* thaw;                 // earliest iteration not proven (atomicMin)
};

// One window step of the state (y, a) of a slot with label yh and cross sum G
// from the window start, n steps with mu = mu0, mu0 * f, ... (the states the
// ordinary iterations compute).
__device__ __forceinline__ void lwin_replay(int yh, int G, double mu0, double fct, int n, double& y, double& a) {
    double m = mu0;
    for (int i = 0; i < n; ++i) {
        face_step(yh, G, m, y, a);
        m = __dmul_rn(m, fct);
    }
}

// Sum of 32 values in the order of the warp butterfly used for a chunk's
// (yhat - y)^2 (levels pairing lanes i and i ^ 16, then ^ 8, ^ 4, ^ 2, ^ 1),
// by one thread: m marks the lanes whose value is not +0, v[r * stride] is
// the value of the r-th marked lane.  Adding +0 to a value x >= +0 gives x
// exactly, so only the pairs of two marked values are added, and the result
// is the butterfly's, bit for bit.
__device__ __forceinline__ double bfly_sum(unsigned m, const double* v, int stride) {
    if (m == 0u) return 0.0;
    if ((m & (m - 1u)) == 0u) return v[0];
    double w[16];
    unsigned p = 0u;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const bool lo = (m >> i) & 1u, hi = (m >> (i + 16)) & 1u;
        const int rl = __popc(m & ((1u << i) - 1u));
        const int rh = __popc(m & ((1u << (i + 16)) - 1u));
        double x = 0.0;
        if (lo && hi) x = __dadd_rn(v[rl * stride], v[rh * stride]);
        else if (lo) x = v[rl * stride];
        else if (hi) x = v[rh * stride];
        w[i] = x;
        if (lo || hi) p |= 1u << i;
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const bool a = (p >> i) & 1u, b = (p >> (i + o)) & 1u;
            if (a && b) w[i] = __dadd_rn(w[i], w[i + o]);
            else if (b) w[i] = w[i + o];
        }
        p = (p | (p >> o)) & ((1u << o) - 1u);
    }
    return w[0];
}

// Window iterations whose chunk sums one pass of phase 1 keeps in shared
// memory, and entries (slots that move) a thread carries through the window.
constexpr int LW_WB = 8;
constexpr int LW_RMAX = 4;

// Phase 1 for a piece kk[0..nb) of S.  scr / scr_bytes: dynamic shared memory.
template <int CONN>
__device__ __noinline__ void lwin_traj(const PersistArgs& P, const LWin& W, const int* kk, int nb,
                                       unsigned char* scr, int scr_bytes) {
    const UpdArgs& A = P.u;
    const Geo& g = A.g;
    constexpr int nh = CONN / 2;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5, NT = blockDim.x;
    const SchedView sv = sched_view(A.sched, g.K);
    UpdSmem& us = upd_smem();
    unsigned (&s_dom)[MB][CHUNK_WORDS] = us.dom;
    double* mus = us.part[0];            // mu of each window iteration
    const int Wn = W.Wn;
    if (tid < nb * CHUNK_WORDS) {
        const int j = tid / CHUNK_WORDS, w = tid % CHUNK_WORDS;
        const int k = kk[j];
        const size_t o = (size_t)k * CHUNK_WORDS + w;
        const unsigned m = __ldcg(&sv.act[o]) | __ldcg(&sv.dsc[o]);
        s_dom[j][w] = m;
        P.wmask[o] = m;
        if (w == 0) {
            P.wtag[k] = W.tag;
            const int q = __ldcg(&sv.qs[k]);
            if (q == 0 || q == 3) atomicMin(W.thaw, W.tw + 1);   // not proven forced: its next solve may cut
        }
    }
    if (tid == 0) {
        double m = W.mu;
        for (int i = 0; i < Wn; ++i) {
            mus[i] = m;
            m = __dmul_rn(m, P.mu_fact);
        }
        us.ecnt = 0;
        us.ovf = 0;
    }
    __syncthreads();
    if (tid == 0) {
        int tot = 0;
        for (int j = 0; j < nb; ++j) {
            us.okb[j] = tot;
            for (int w = 0; w < CHUNK_WORDS; ++w) tot += __popc(s_dom[j][w]);
        }
        us.tot = tot;
    }
    __syncthreads();
    const int tot = us.tot;
    // scratch: chunk sums part[tot][Wn], per chunk its moving lanes and their
    // first entry, per entry its slot (x2, + label) and G, and the entries'
    // (yhat - y)^2 for LW_WB iterations at a time
    double* part = reinterpret_cast<double*>(scr);
    unsigned* t_mask = reinterpret_cast<unsigned*>(part + (size_t)tot * Wn);
    int* t_base = reinterpret_cast<int*>(t_mask + tot);
    const size_t head = ((size_t)tot * Wn * 8 + (size_t)tot * 8 + 15) & ~(size_t)15;
    const int ecap = scr_bytes > (long long)head ? (int)(((size_t)scr_bytes - head) / (8 + 4 + 8 * LW_WB)) : 0;
    long long* e_s = reinterpret_cast<long long*>(scr + head);
    double* e_d = reinterpret_cast<double*>(e_s + ecap);
    int* e_G = reinterpret_cast<int*>(e_d + (size_t)ecap * LW_WB);
    // pass A, a warp per chunk: G, the bound and the entry list
    for (int tk = wid; tk < tot; tk += nw) {
        int r = tk, j = 0, w = 0;
        for (;;) {
            const int c = __popc(s_dom[j][w]);
            if (r < c) break;
            r -= c;
            if (++w == CHUNK_WORDS) { w = 0; ++j; }
        }
        unsigned mm = s_dom[j][w];
        for (int i = 0; i < r; ++i) mm &= mm - 1;
        const int ch = w * 32 + __ffs(mm) - 1;
        const int k = kk[j];
        const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
        const int f = ch * 32 + lane;
        bool mv = false;
        int G = 0, yh = 0;
        long long s = 0;
        if (f < g.F) {
            const int v = A.faceLocal[f];
            const long long gi = (long long)k * g.B + v;
            int wj[CONN], yj[CONN];
#pragma unroll
            for (int d = 0; d < CONN; ++d) {
                int kn, ln, fn;
                wj[d] = 0;
                yj[d] = 0;
                if (halo_decode(g, A.halo[d * g.F + f], kz, ky, kx, kn, ln, fn)) {
                    const long long gj = (long long)kn * g.B + ln;
                    wj[d] = (d < nh) ? A.Wl[(long long)d * g.N + gi] : A.Wl[(long long)(d - nh) * g.N + gj];
                    yj[d] = __ldcg(&A.yhat[gj]);
                }
            }
            yh = __ldcg(&A.yhat[gi]);
#pragma unroll
            for (int d = 0; d < CONN; ++d) G += wj[d] * (yh - yj[d]);
            s = (long long)k * g.F + f;
            const double y = __ldcg(&A.yF[s]), a = __ldcg(&A.aF[s]);
            // a slot with G = 0, a = +0 and y = yhat keeps its state and adds +0
            mv = !(G == 0 && __double_as_longlong(a) == 0 &&
                   __double_as_longlong(y) == __double_as_longlong((double)yh));
            float bf = 9.094947017729282e-13f;   // 2^-40
            if (mv) {
                bf = __double2float_ru(fabs(a) + fabs(y - (double)yh) +
                                       2.0 * fabs((double)G) * 0.0009765625 * (1.0 / W.mu) * (1.0 + 1e-12) +
                                       9.094947017729282e-13);
                // above 2^-40 for every moving slot (2^-40 with G = 0 marks a still one)
                if (__float_as_uint(bf) <= 0x2b800000u) bf = __uint_as_float(0x2b800001u);
            }
            P.wslot[s] = ((unsigned long long)__float_as_uint(bf) << 32) | (unsigned)G;
        }
        const unsigned ntm = __ballot_sync(0xffffffffu, mv);
        int base = 0;
        if (ntm) {
            if (lane == 0) base = atomicAdd(&us.ecnt, __popc(ntm));
            base = __shfl_sync(0xffffffffu, base, 0);
        }
        if (base + __popc(ntm) > ecap) {
            if (lane == 0) us.ovf = 1;
        } else if (mv) {
            const int e = base + __popc(ntm & ((1u << lane) - 1u));
            e_s[e] = (s << 1) | yh;
            e_G[e] = G;
        }
        if (lane == 0) {
            t_mask[tk] = ntm;
            t_base[tk] = base;
        }
    }
    __syncthreads();
    const int ne = us.ecnt;
    if (us.ovf || ne > LW_RMAX * NT) {
        // more moving slots than the scratch holds: no window this time
        if (tid == 0) atomicMin(W.thaw, W.tw + 1);
        __syncthreads();
        return;
    }
    // the entries a thread carries: e = tid + r NT
    double ey[LW_RMAX], ea[LW_RMAX];
#pragma unroll
    for (int r = 0; r < LW_RMAX; ++r) {
        const int e = tid + r * NT;
        ey[r] = 0.0;
        ea[r] = 0.0;
        if (e < ne) {
            const long long s = e_s[e] >> 1;
            ey[r] = __ldcg(&A.yF[s]);
            ea[r] = __ldcg(&A.aF[s]);
        }
    }
    for (int i0 = 0; i0 < Wn; i0 += LW_WB) {
        const int nb8 = Wn - i0 < LW_WB ? Wn - i0 : LW_WB;
#pragma unroll
        for (int r = 0; r < LW_RMAX; ++r) {
            const int e = tid + r * NT;
            if (e >= ne) continue;
            const int yh = (int)(e_s[e] & 1), G = e_G[e];
            for (int ii = 0; ii < nb8; ++ii) {
                e_d[(size_t)e * LW_WB + ii] = face_step(yh, G, mus[i0 + ii], ey[r], ea[r]);
                if (i0 + ii == Wn - 2 || i0 + ii == Wn - 1) {
                    // the states after the window's last two iterations
                    const long long s = e_s[e] >> 1;
                    const int q = i0 + ii == Wn - 1 ? 1 : 0;
                    P.wst[(size_t)s * 4 + 2 * q] = ey[r];
                    P.wst[(size_t)s * 4 + 2 * q + 1] = ea[r];
                }
            }
        }
        __syncthreads();
        // chunk sums, the lanes of a warp on the same chunk where they can
        for (int q = tid; q < tot * nb8; q += NT) {
            const int tk = q / nb8, ii = q - tk * nb8;
            part[(size_t)tk * Wn + i0 + ii] = bfly_sum(t_mask[tk], e_d + (size_t)t_base[tk] * LW_WB + ii, LW_WB);
        }
        __syncthreads();
    }
    // each block's r2 per iteration: its chunks' sums in increasing chunk order
    // (the other chunks' slots are trivial and add +0)
    for (int q = tid; q < nb * Wn; q += NT) {
        const int j = q / Wn, i = q % Wn;
        const int t0 = us.okb[j], t1 = j + 1 < nb ? us.okb[j + 1] : tot;
        double r2 = 0.0;
        for (int tk = t0; tk < t1; ++tk) r2 = __dadd_rn(r2, part[(size_t)tk * Wn + i]);
        if (r2 != 0.0) atomicMax(&W.r2w[i], (unsigned long long)__double_as_longlong(r2));
    }
    __syncthreads();
}

// The exact Eq. 8 forced test of face slot f of block k at window iteration
// i (the unary of iteration tw+i from the states after iteration tw+i-1,
// replayed from the window start where they move; mv: some state around the
// slot moves, eo / em: the slot / its cross neighbours are entry slots).
// Phase 2 calls it for the window's first iteration only, where nothing is
// replayed.
template <int CONN>
__device__ __noinline__ bool lwin_exact(const PersistArgs& P, const LWin& W, int k, int f, int i, bool mv, bool eo,
                                        unsigned em, double m1024, long long Ui, int lab, long long cs) {
    const SolveArgs& A = P.s;
    const Geo& g = A.g;
    constexpr int nh = CONN / 2;
    const int F = g.F;
    const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
    const long long gi = (long long)k * g.B + A.faceLocal[f];
    const long long s = (long long)k * F + f;
    double yv = __ldcg(&A.yF[s]), av = __ldcg(&A.aF[s]);
    if (eo && mv) lwin_replay(lab, (int)(unsigned)__ldcg(&P.wslot[s]), W.mu, P.mu_fact, i - 1, yv, av);
    double yjv[CONN];
    int wj[CONN];
    unsigned okm = 0;
#pragma unroll
    for (int d = 0; d < CONN; ++d) {
        yjv[d] = 0.0;
        wj[d] = 0;
        int kn, ln, fn;
        if (!halo_decode(g, A.halo[d * F + f], kz, ky, kx, kn, ln, fn)) continue;
        okm |= 1u << d;
        wj[d] = (d < nh) ? A.Wl[(long long)d * g.N + gi] : A.Wl[(long long)(d - nh) * g.N + (long long)kn * g.B + ln];
        const long long sj = (long long)kn * F + fn;
        yjv[d] = __ldcg(&A.yF[sj]);
        if (mv && ((em >> d) & 1u)) {
            double aj = __ldcg(&A.aF[sj]);
            const int lj = __ldcg(&A.yhat[(long long)kn * g.B + ln]);
            lwin_replay(lj, (int)(unsigned)__ldcg(&P.wslot[sj]), W.mu, P.mu_fact, i - 1, yjv[d], aj);
        }
    }
    const long long C = face_cap_from<CONN>(Ui, yv, av, yjv, wj, okm, m1024);
    return lab ? (C < -cs) : (C >= cs);
}

// Phase 2 for a piece kk[0..nb) of S.
template <int CONN>
__device__ __noinline__ void lwin_cert(const PersistArgs& P, const LWin& W, const int* kk, int nb) {
    const SolveArgs& A = P.s;
    const Geo& g = A.g;
    constexpr int nh = CONN / 2;
    const int F = g.F;
    const int tid = threadIdx.x;
    // entry chunks of the 27 blocks around each block of the piece (0 outside
    // the grid or S), and the window iterations' constants
    __shared__ unsigned s_nm[MB][27][CHUNK_WORDS];
    __shared__ double s_mu[LWMAX], s_m1024[LWMAX];
    __shared__ long long s_H[LWMAX];
    __shared__ float s_mf[LWMAX], s_e2h[LWMAX];
    __shared__ int s_it[LWMAX];
    for (int q = tid; q < nb * 27; q += blockDim.x) {
        const int j = q / 27, code = q % 27, k = kk[j];
        const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
        const int nz = kz + code / 9 - 1, ny = ky + (code / 3) % 3 - 1, nx = kx + code % 3 - 1;
        bool in = nz >= 0 && nz < g.nbz && ny >= 0 && ny < g.nby && nx >= 0 && nx < g.nbx;
        const int kn = in ? (nz * g.nby + ny) * g.nbx + nx : 0;
        in = in && __ldcg(&P.wtag[kn]) == W.tag;
        for (int w = 0; w < CHUNK_WORDS; ++w)
            s_nm[j][code][w] = in ? __ldcg(&P.wmask[(size_t)kn * CHUNK_WORDS + w]) : 0u;
    }
    if (tid == 0) {
        double m = W.mu;
        for (int i = 0; i < W.Wn; ++i) {
            s_mu[i] = m;
            m = __dmul_rn(m, P.mu_fact);
        }
    }
    __syncthreads();
    if (tid < W.Wn) {
        // iteration tw+1+tid: m1024 and H as iter_args computes them
        const double m1024 = __dmul_rn(1024.0, s_mu[tid]);
        const double h = __dmul_rn(m1024, 0.5);
        s_m1024[tid] = m1024;
        s_it[tid] = h < 4503599627370496.0 ? 1 : 0;   // 2^52
        s_H[tid] = s_it[tid] ? (long long)floor(h) : 0;
        s_mf[tid] = __double2float_ru(m1024);
        s_e2h[tid] = __fmul_ru(1.8189894035458565e-12f, __double2float_ru(h));   // 2^-40 * 2h
    }
    __syncthreads();
    int fail = 0x7fffffff;   // earliest window iteration (1-based) found not forced
    unsigned ncert = 0, nexact = 0;
    // an entry slot that does not move has G = 0 and the bound 2^-40
    constexpr unsigned long long STILL = 0x2b80000000000000ull;
    for (int q = tid; q < nb * F; q += blockDim.x) {
        const int j = q / F, f = q - j * F, k = kk[j];
        const bool eo = (s_nm[j][13][f >> 10] >> ((f >> 5) & 31)) & 1u;
        unsigned em = 0;
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            const int he = A.halo[d * F + f];
            if (he >= 0) {
                const int code = he >> 24, fn = he & 0xfff;
                if ((s_nm[j][code][fn >> 10] >> ((fn >> 5) & 31)) & 1u) em |= 1u << d;
            }
        }
        // neither the slot nor a cross neighbour can move: its unary keeps the
        // interior form of its last solve, forced while mu grows
        if (!eo && em == 0) continue;
        ++ncert;
        const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
        const int v = A.faceLocal[f];
        const long long gi = (long long)k * g.B + v;
        const long long s = (long long)k * F + f;
        const int lab = __ldcg(&A.yhat[gi]);
        const long long Ui = A.U[gi];
        const long long cs = nlink_sum<CONN>(g, A.Wl, k, v);
        float bo = 0.f;
        bool mv = false;   // the slot's or a cross neighbour's state moves in the window
        if (eo) {
            const unsigned long long e = __ldcg(&P.wslot[s]);
            bo = __uint_as_float((unsigned)(e >> 32));
            mv = e != STILL;
        }
        // the certificate's integer part and bounds, one direction at a time
        long long I = Ui, wtot = 0;
        float wsum = 0.f;
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            int kn, ln, fn;
            if (!halo_decode(g, A.halo[d * F + f], kz, ky, kx, kn, ln, fn)) continue;
            const int w = (d < nh) ? A.Wl[(long long)d * g.N + gi] : A.Wl[(long long)(d - nh) * g.N + (long long)kn * g.B + ln];
            const int lj = __ldcg(&A.yhat[(long long)kn * g.B + ln]);
            const long long sj = (long long)kn * F + fn;
            float bj;
            if ((em >> d) & 1u) {
                const unsigned long long e = __ldcg(&P.wslot[sj]);
                bj = __uint_as_float((unsigned)(e >> 32));
                mv = mv || e != STILL;
            } else {
                bj = __double2float_ru(fabs(__ldcg(&A.yF[sj]) - (double)lj));   // constant in the window
            }
            I += (long long)w * (lab - lj);
            wsum = __fadd_ru(wsum, __fmul_ru((float)w, __fadd_ru(bo, bj)));
            wtot += w;
        }
        // allowance for the computed value vs the exact one: 2^-40 (|I| + 3 sum w),
        // plus 2^-40 * 2h per iteration below
        const float cE = __double2float_ru(9.094947017729282e-13 * ((double)llabs(I) + 3.0 * (double)wtot) *
                                           (1.0 + 1e-12));
        const float base = __fadd_ru(wsum, cE);
        const float bo2 = __fmul_ru(2.f, bo);
        // With no state around the slot moving, its unary is U + (a constant)
        // + m1024 (1/2 - yhat), which only moves away from the cut as mu
        // grows: the first window iteration decides for all.
        const int imax = mv ? W.Wn : 1;
        for (int i = 1; i <= imax && i < fail; ++i) {
            if (!s_it[i - 1]) { fail = i; break; }   // no integer bound
            const long long H = s_H[i - 1];
            const float dl = __fadd_ru(__fadd_ru(base, __fmul_ru(s_mf[i - 1], bo2)), s_e2h[i - 1]);
            bool ok = false;
            if (dl < 4.0e18f) {
                const long long D = (dl < 2.0e9f ? (long long)(int)ceilf(dl) : (long long)ceilf(dl)) + 1;
                ok = lab ? (I - H + D + 1 <= -cs) : (I + H - D - 1 >= cs);
            }
            if (!ok && i == 1) {
                // no certificate at the window's first iteration: the exact unary
                // from the states at the window start decides.  Later iterations
                // have none (their states would have to be replayed, quadratic
                // in the window's length where certificates are weak): the
                // window ends there.
                ++nexact;
                ok = lwin_exact<CONN>(P, W, k, f, i, mv, eo, em, s_m1024[i - 1], Ui, lab, cs);
            }
            if (!ok) { fail = i; break; }
        }
    }
    if (fail != 0x7fffffff) atomicMin(W.thaw, W.tw + fail);
    // statistics: slots certified, exact unaries evaluated
    ncert = __reduce_add_sync(0xffffffffu, ncert);
    nexact = __reduce_add_sync(0xffffffffu, nexact);
    if ((tid & 31) == 0) {
        if (ncert) atomicAdd(&A.ctrl->wcyc[6], (unsigned long long)ncert);
        if (nexact) atomicAdd(&A.ctrl->wcyc[7], (unsigned long long)nexact);
    }
    __syncthreads();
}

// Phase 3 for a piece kk[0..nb) (entries i0.. of the list S): the state after
// n window iterations for every moving slot (kept by phase 1 for the last two
// iterations, else replayed), the chunk marks the ordinary updates would have
// made, and (list_to != null) the piece's entries copied to the list of the
// iteration after the window.
template <int CONN>
__device__ __noinline__ void lwin_commit(const PersistArgs& P, const LWin& W, const int* kk, int nb, int n,
                                         int* list_to, int i0) {
    const UpdArgs& A = P.u;
    const Geo& g = A.g;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const SchedView sv = sched_view(A.sched, g.K);
    UpdSmem& us = upd_smem();
    unsigned (&s_dom)[MB][CHUNK_WORDS] = us.dom;
    if (list_to && tid < nb) list_to[i0 + tid] = kk[tid];
    if (tid < nb * CHUNK_WORDS) {
        const int j = tid / CHUNK_WORDS, w = tid % CHUNK_WORDS;
        const size_t o = (size_t)kk[j] * CHUNK_WORDS + w;
        const unsigned m = __ldcg(&P.wmask[o]);
        s_dom[j][w] = m;
        // the entry chunks are evaluated at the next solve
        if (n > 0 && m) atomicOr(&sv.dsc[o], m);
    }
    __syncthreads();
    if (tid == 0) {
        int tot = 0;
        for (int j = 0; j < nb; ++j)
            for (int w = 0; w < CHUNK_WORDS; ++w) tot += __popc(s_dom[j][w]);
        us.tot = tot;
    }
    __syncthreads();
    const int tot = n > 0 ? us.tot : 0;
    const int q = n == W.Wn ? 1 : (n == W.Wn - 1 ? 0 : -1);   // kept state, or replay
    for (int tk = wid; tk < tot; tk += nw) {
        int r = tk, j = 0, w = 0;
        for (;;) {
            const int c = __popc(s_dom[j][w]);
            if (r < c) break;
            r -= c;
            if (++w == CHUNK_WORDS) { w = 0; ++j; }
        }
        unsigned mm = s_dom[j][w];
        for (int i = 0; i < r; ++i) mm &= mm - 1;
        const int ch = w * 32 + __ffs(mm) - 1;
        const int k = kk[j];
        const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
        const int f = ch * 32 + lane;
        bool changed = false;
        if (f < g.F) {
            const long long s = (long long)k * g.F + f;
            const int yh = __ldcg(&A.yhat[(long long)k * g.B + A.faceLocal[f]]);
            const int G = (int)(unsigned)__ldcg(&P.wslot[s]);
            const double y0 = __ldcg(&A.yF[s]), a0 = __ldcg(&A.aF[s]);
            const bool mv = !(G == 0 && __double_as_longlong(a0) == 0 &&
                              __double_as_longlong(y0) == __double_as_longlong((double)yh));
            if (mv) {
                double y = y0, a = a0;
                if (q >= 0) {
                    y = __ldcg(&P.wst[(size_t)s * 4 + 2 * q]);
                    a = __ldcg(&P.wst[(size_t)s * 4 + 2 * q + 1]);
                } else {
                    lwin_replay(yh, G, W.mu, P.mu_fact, n, y, a);
                }
                if (__double_as_longlong(y) != __double_as_longlong(y0) ||
                    __double_as_longlong(a) != __double_as_longlong(a0)) {
                    A.yF[s] = y;
                    A.aF[s] = a;
                    changed = true;
                }
            }
        }
        // a changed slot's cross neighbours' chunks are evaluated at the next
        // solve (its own chunk is an entry chunk, marked above)
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            int kn = -1, ln, fn = 0;
            bool mk = false;
            if (changed) mk = halo_decode(g, A.halo[d * g.F + f], kz, ky, kx, kn, ln, fn);
            const unsigned key = mk ? (unsigned)kn * 128u + (unsigned)(fn >> 5) : 0xffffffffu;
            const unsigned grp = __match_any_sync(0xffffffffu, key);
            if (mk && lane == __ffs(grp) - 1) chunk_mark(sv.dsc, kn, fn);
        }
    }
    __syncthreads();
}

// Length of a window from iteration tw (launch ends after tlimit).  Once
// labels are frozen every block residual shrinks by 1/mu_fact per iteration,
// so the stop test is expected about ln(r/eps)/ln(mu_fact) iterations on; the
// window is cut there (plus one).  This only sizes the window; what is
// committed is decided by the exact stop test.
static __device__ __noinline__ int lwin_size(const PersistArgs& P, int tw, int tlimit) {
    const Ctrl* c = P.s.ctrl;
    int Wn = min(min(LWMAX, P.lwcap), tlimit - tw);
    const double r_tw = __dsqrt_rn(__longlong_as_double((long long)__ldcg(&c->r2max[tw])));
    const double r_pr = tw >= 2 ? __dsqrt_rn(__longlong_as_double((long long)__ldcg(&c->r2max[tw - 1]))) : 0.0;
    const bool geometric = r_pr > 0.0 && fabs(r_tw * P.mu_fact / r_pr - 1.0) < 1e-3;
    if (r_tw > P.s.eps && P.mu_fact > 1.0) {
        const double n_pred = ceil(log(r_tw / P.s.eps) / log(P.mu_fact));
        if (n_pred + 1.0 < (double)Wn) Wn = max(1, (int)n_pred + 1);
    }
    if (!geometric) Wn = min(Wn, 16);
    return Wn;
}

struct LWRes {
    int tend;        // last iteration committed
    int stop;        // its stop test held
    int ran_out;     // every window iteration was proven (labels still frozen)
    int failed;      // a grid barrier gave up
    unsigned nbar;   // barriers passed so far in the launch
};

// One window from iteration tw with mu of iteration tw+1 (every CTA, uniform
// arguments): the three phases and their barriers (see LWin).
template <int CONN>
__device__ __noinline__ LWRes lwin_run(const PersistArgs& P, int tw, double mu, int Wn, int nwin, unsigned nbar,
                                       unsigned char* smem, int* s_kk, int* s_k) {
    Ctrl* c = P.s.ctrl;
    const int K = P.s.g.K;
    const SchedView sv = sched_view(P.s.sched, K);
    __shared__ int s_tend, s_stop;
    LWRes R;
    R.failed = 0;
    LWin W;
    W.tw = tw;
    W.Wn = Wn;
    W.mu = mu;
    W.tag = ((unsigned long long)P.s.epoch << 32) | (unsigned)(nwin + 1);
    W.r2w = c->r2w[nwin & 1];
    W.thaw = &c->lthaw[nwin & 1];
    const int ns = (int)__ldcg(&sv.sq_n[(tw + 1) & 1]);
    const int* Sl = sv.sq + (size_t)((tw + 1) & 1) * K;
    const long long w0 = clock64();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->wwork[1] = 0u;
        c->wwork[2] = 0u;
    }
    auto load_piece = [&](int i0, int nb) {
        if (threadIdx.x < nb) s_kk[threadIdx.x] = __ldcg(&Sl[i0 + threadIdx.x]);
        __syncthreads();
    };
    const int scr_bytes = dyn_smem_bytes();
    auto p1 = [&](int i0, int nb) { load_piece(i0, nb); lwin_traj<CONN>(P, W, s_kk, nb, smem, scr_bytes); };
    list_pieces(ns, &c->wwork[0], s_k, p1);
    const long long w1 = clock64();
    if (!grid_sync(c, gridDim.x, nbar, P.spin_limit)) { R.failed = 1; R.nbar = nbar; return R; }
    const long long w2 = clock64();
    auto p2 = [&](int i0, int nb) { load_piece(i0, nb); lwin_cert<CONN>(P, W, s_kk, nb); };
    list_pieces(ns, &c->wwork[1], s_k, p2);
    const long long w3 = clock64();
    if (!grid_sync(c, gridDim.x, nbar, P.spin_limit)) { R.failed = 1; R.nbar = nbar; return R; }
    const long long w4 = clock64();
    // resolution (the same in every CTA): the valid run ends before the
    // earliest iteration not proven; the window ends at the first valid
    // iteration whose stop test holds, else at the valid end
    const int tstar = __ldcg(W.thaw);
    const int tvalid = min(tstar - 1, tw + Wn);
    if (threadIdx.x == 0) {
        int tend = tvalid, stop = 0;
        for (int tt = tw + 1; tt <= tvalid; ++tt) {
            const double r2 = __longlong_as_double((long long)__ldcg(&W.r2w[tt - tw - 1]));
            if (!(__dsqrt_rn(r2) > P.s.eps)) { tend = tt; stop = 1; break; }
        }
        s_tend = tend;
        s_stop = stop;
    }
    __syncthreads();
    const int tend = s_tend, stop = s_stop;
    const int n = tend - tw;
    int* list_to = (((tend + 1) ^ (tw + 1)) & 1) ? sv.sq + (size_t)((tend + 1) & 1) * K : nullptr;
    auto p3 = [&](int i0, int nb) {
        load_piece(i0, nb);
        lwin_commit<CONN>(P, W, s_kk, nb, n, list_to, i0);
    };
    list_pieces(ns, &c->wwork[2], s_k, p3);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int tt = tw + 1; tt <= tend; ++tt) c->r2max[tt] = __ldcg(&W.r2w[tt - tw - 1]);
        if (list_to) {
            sv.sq_n[(tend + 1) & 1] = (unsigned)ns;
            sv.uq_n[(tend + 1) & 1] = 0u;
        }
        c->windows += 1;
        c->window_iters += n;
        c->cuts[(tend + 1) & 1] = 0u;
        // the next window's phase-1 counter, residuals and thaw
        c->wwork[0] = 0u;
        for (int i = 0; i < LWMAX; ++i) c->r2w[(nwin + 1) & 1][i] = 0ull;
        c->lthaw[(nwin + 1) & 1] = 0x7fffffff;
    }
    const long long w5 = clock64();
    if (!grid_sync(c, gridDim.x, nbar, P.spin_limit)) { R.failed = 1; R.nbar = nbar; return R; }
    if (threadIdx.x == 0) {
        const long long w6 = clock64();
        atomicAdd(&c->wcyc[0], (unsigned long long)(w1 - w0));
        atomicAdd(&c->wcyc[1], (unsigned long long)(w2 - w1));
        atomicAdd(&c->wcyc[2], (unsigned long long)(w3 - w2));
        atomicAdd(&c->wcyc[3], (unsigned long long)(w4 - w3));
        atomicAdd(&c->wcyc[4], (unsigned long long)(w5 - w4));
        atomicAdd(&c->wcyc[5], (unsigned long long)(w6 - w5));
    }
    R.tend = tend;
    R.stop = stop;
    R.ran_out = tstar > tw + Wn;
    R.nbar = nbar;
    return R;
}

// Occupancy of the block-solver kernels by CTA width: 256 threads (up to
// 2048 nodes, 4 per thread for 32x32 blocks) run 3 CTAs per SM with 80
// registers; 512 threads (blocks up to 4096 nodes) run 2 CTAs per SM with 64.
template <int NT>
struct SolverOcc { static constexpr int min_blocks = NT <= 256 ? 3 : 2; };

// WIN: the form with run-ahead windows.  A solve with windows (lwin) is two
// launches back to back: the plain form runs the ordinary iterations and, at
// the first one that solves no block by a cut, records its iteration and mu
// in the control block and returns (handoff, no finish); the windowed form
// then continues from there to the end of the launch's iterations and does
// the finish, or returns at once if the plain form already ended.  The
// ordinary iterations thus run in a kernel with no window code (the calls
// into it cost the iteration path registers); the windowed form runs only
// the frozen tail.
template <int CONN, int NT, bool WIN>
__global__ void __launch_bounds__(NT, SolverOcc<NT>::min_blocks) k_admm_persistent(const __grid_constant__ PersistArgs P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_k;
    __shared__ int s_kk[MB], s_qq[MB], s_pk[MB], s_pok[MB], s_np;   // a grab of list entries
    __shared__ long long s_red[32];
    Ctrl* c = P.s.ctrl;
    const int K = P.s.g.K;
    double mu = P.mu_start;
    int t = P.t0, conv = 0;
    bool failed = false;
    unsigned nbar = 0;
    const bool wl = P.s.sched != nullptr;
    // Window state, the same in every thread of the CTA, kept in shared memory
    // (thread 0 writes it after the last barrier of an iteration or window,
    // every thread reads it after the loop's __syncthreads): the last
    // iteration solved no block by a cut, iterations to wait before the next
    // try, the current wait after failed tries, windows run.  The window code
    // reads the launch arguments from a shared copy.
    __shared__ int s_ws[4];
    if (threadIdx.x < 4) s_ws[threadIdx.x] = 0;
    if (WIN) {
        // the plain form's launch ended the solve (or the launch): nothing to do
        if (!__ldcg(&c->handoff)) return;
        t = __ldcg(&c->iters_done);
        mu = __ldcg(&c->mu_next);
        // the barrier's arrival counter only grows: continue its numbering
        nbar = __ldcg(&c->bar_handoff);
        if (threadIdx.x == 0) s_ws[0] = 1;
    }
    __shared__ __align__(16) unsigned char s_Pbuf[WIN ? sizeof(PersistArgs) : 16];
    if (WIN)
        for (int i = threadIdx.x; i < (int)(sizeof(PersistArgs) / 4); i += blockDim.x)
            reinterpret_cast<int*>(s_Pbuf)[i] = reinterpret_cast<const int*>(&P)[i];
    const PersistArgs& SP = *reinterpret_cast<const PersistArgs*>(s_Pbuf);
    while (t < P.t0 + P.n) {
        __syncthreads();
        if (WIN && s_ws[0] && s_ws[1] == 0 && P.t0 + P.n - t >= 2) {
            const int Wn = lwin_size(SP, t, P.t0 + P.n);
            if (Wn >= 2) {
                const LWRes R = lwin_run<CONN>(SP, t, mu, Wn, s_ws[3], nbar, smem, s_kk, &s_k);
                nbar = R.nbar;
                if (R.failed) { failed = true; break; }
                for (int i = t; i < R.tend; ++i) mu = __dmul_rn(mu, P.mu_fact);
                const int n = R.tend - t;
                t = R.tend;
                if (R.stop) { conv = 1; break; }
                if (threadIdx.x == 0) {
                    // a window that ran to its end leaves the labels frozen; one
                    // cut short waits for a frozen ordinary iteration, and one
                    // that committed next to nothing backs off before the next try
                    s_ws[3] += 1;
                    s_ws[0] = R.ran_out;
                    if (n < 2) {
                        s_ws[2] = s_ws[2] ? min(2 * s_ws[2], 16) : 1;
                        s_ws[1] = s_ws[2];
                    } else {
                        s_ws[2] = 0;
                    }
                }
                continue;
            }
        }
        ++t;
        // (the list pointers are derived here, not kept across the window call)
        const SchedView sv = sched_view(P.s.sched, K);
        IterArgs it = iter_args(t, mu);
        // with worklists, the launch's first iteration does every block;
        // later ones the blocks on the lists (see sched_view)
        const bool full = !wl || (!WIN && t == P.t0 + 1 && !P.wl_cont);
        it.qeval = !full;
        // the update counter is idle during the solve phase and vice versa,
        // so each is reset in the other phase; likewise the list counts
        const long long c0 = clock64();
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            c->work[1] = 0u;
            if (wl) sv.sq_n[(t + 1) & 1] = 0u;
        }
        const int ns = full ? K : (int)__ldcg(&sv.sq_n[t & 1]);
        if (full || !P.dynamic) {
            for (int i = next_block(P.dynamic, &c->work[0], -1, &s_k); i < ns;
                 i = next_block(P.dynamic, &c->work[0], i, &s_k))
                solve_block<CONN>(P.s, it, full ? i : __ldcg(&sv.sq[(t & 1) * (size_t)K + i]), smem);
        } else {
            // from the list, a few entries at a time: the forced blocks among
            // them are re-evaluated together (partial_solve_multi), the others
            // (and any whose partial solve fails) solved one by one
            auto piece = [&](int i0, int nb) {
                if (threadIdx.x < nb) {
                    const int kb = __ldcg(&sv.sq[(t & 1) * (size_t)K + i0 + threadIdx.x]);
                    s_kk[threadIdx.x] = kb;
                    s_qq[threadIdx.x] = __ldcg(&sv.qs[kb]);
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    int np = 0;
                    for (int j = 0; j < nb; ++j)
                        if (s_qq[j]) s_pk[np++] = s_kk[j];
                    s_np = np;
                }
                __syncthreads();
                const int np = s_np;
                if (np) partial_solve_multi<CONN>(P.s, it, s_pk, np, s_pok);
                for (int j = 0, jp = 0; j < nb; ++j) {
                    bool done = false;
                    if (s_qq[j]) done = s_pok[jp++] != 0;
                    if (!done) solve_block<CONN>(P.s, it, s_kk[j], smem, false);
                }
                __syncthreads();
            };
            list_pieces(ns, &c->work[0], &s_k, piece);
        }
        const long long c1 = clock64();
        if (!grid_sync(c, gridDim.x, nbar, P.spin_limit)) { failed = true; break; }
        const long long c2 = clock64();
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            c->work[0] = 0u;
            // (every CTA read the cut count of iteration t-1 before the barrier)
            c->cuts[(t + 1) & 1] = 0u;
            if (wl) sv.uq_n[(t + 1) & 1] = 0u;
        }
        const int nu = full ? K : (int)__ldcg(&sv.uq_n[t & 1]);
        if (!wl || !P.dynamic) {
            for (int i = next_block(P.dynamic, &c->work[1], -1, &s_k); i < nu;
                 i = next_block(P.dynamic, &c->work[1], i, &s_k))
                update_block<CONN>(P.u, mu, t, full ? i : __ldcg(&sv.uq[(t & 1) * (size_t)K + i]), full ? 1 : 0);
        } else {
            // from the list (or every block, in a full iteration), a few
            // entries at a time, updated together
            auto piece = [&](int i0, int nb) {
                if (threadIdx.x < nb)
                    s_kk[threadIdx.x] = full ? i0 + (int)threadIdx.x
                                             : __ldcg(&sv.uq[(t & 1) * (size_t)K + i0 + threadIdx.x]);
                __syncthreads();
                update_blocks<CONN>(P.u, mu, t, s_kk, nb, full ? 1 : 0);
            };
            list_pieces(nu, &c->work[1], &s_k, piece);
        }
        if (wl && !full && blockIdx.x == 0 && threadIdx.x == 0) {
            atomicAdd(&c->sched_work[0], (unsigned long long)ns);
            atomicAdd(&c->sched_work[1], (unsigned long long)nu);
        }
        const long long c3 = clock64();
        if (!grid_sync(c, gridDim.x, nbar, P.spin_limit)) { failed = true; break; }
        if (threadIdx.x == 0) {
            const long long c4 = clock64();
            atomicAdd(&c->pcyc[0], (unsigned long long)(c1 - c0));
            atomicAdd(&c->pcyc[1], (unsigned long long)(c2 - c1));
            atomicAdd(&c->pcyc[2], (unsigned long long)(c3 - c2));
            atomicAdd(&c->pcyc[3], (unsigned long long)(c4 - c3));
        }
        mu = __dmul_rn(mu, P.mu_fact);
        if (threadIdx.x == 0) {
            s_ws[0] = wl && !full && __ldcg(&c->cuts[t & 1]) == 0u;
            if (s_ws[1] > 0) --s_ws[1];
        }
        const double r2 = __longlong_as_double((long long)__ldcg(&c->r2max[t]));
        if (!(__dsqrt_rn(r2) > P.s.eps)) { conv = 1; break; }
        if (!WIN && P.lwin) {
            // labels frozen: the windowed form continues from here
            __syncthreads();
            if (s_ws[0] && P.t0 + P.n - t >= 2) {
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    c->iters_done = t;
                    c->mu_next = mu;
                    c->bar_handoff = nbar;
                    c->lthaw[0] = c->lthaw[1] = 0x7fffffff;   // for the windows
                    c->conv_t = 0;
                    c->handoff = 1;
                }
                return;
            }
        }
    }
    if (!WIN && blockIdx.x == 0 && threadIdx.x == 0) c->handoff = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->iters_done = t;
        c->conv_t = conv ? t : 0;
    }
    // every exit above follows the last iteration's second barrier, and its
    // labels were written before the first: the finish can read them all
    if (!failed && (P.out_labels || P.out_energy))
        finish_flat<CONN>(P, s_red);
}

// ---------------------------------------------------------------------------
// Resident persistent path (K <= co-resident CTAs): CTA k owns block k for
// the whole launch and keeps its intra-block n-links, n-link sums, unaries,
// labels and face state in shared memory, so a light iteration reads only the
// neighbours' halo (face y, labels) from L2.  Arithmetic is the same as in
// solve_block / update_block, operation for operation.
//
// Extra shared memory after the solver's (aligned to 16 B):
//   yS, aS  f64 [F]          face y and a of the owned block
//   resW    int32 [CONN/2][B] intra-block n-link capacities, forward directions
//   cs0     int32 [B]        their sums
//   Us      int32 [B]        unaries
//   lab     uint8 [B]        labels
// ---------------------------------------------------------------------------
// Byte offsets of the resident kernel's shared-memory arrays.  The host sizes
// the launch with `.resident_end` / `.window_end` and the kernel takes every
// pointer from here, so the two cannot disagree.
struct ResidentLayout {
    size_t yS, aS, resW, cs0, Us, fl, lab, resident_end;                 // always present
    size_t yS0, aS0, hy, ha, rloc, Gf, hG, hw, hs, hl, labw;              // run-ahead windows
    size_t cI, cB, cW, cE, hB;                                             // window certificates
    size_t ring, window_end;                                               // last RING own states
};

constexpr int RING = 4;    // own face states kept for short rollbacks

constexpr int WMAX = 64;   // most iterations per run-ahead window

__host__ __device__ inline ResidentLayout resident_layout(int conn, int B, int F, int NH) {
    ResidentLayout L;
    size_t o = (solver_smem_bytes(conn, B) + 15) & ~(size_t)15;
    L.yS = o;   o += 8 * (size_t)F;
    L.aS = o;   o += 8 * (size_t)F;
    L.resW = o; o += 4 * (size_t)(conn / 2) * B;     // forward planes only
    L.cs0 = o;  o += 4 * (size_t)B;
    L.Us = o;   o += 4 * (size_t)B;
    L.fl = o;   o += 2 * (size_t)F;
    L.lab = o;  o += (size_t)B;
    L.resident_end = o;
    o = (o + 15) & ~(size_t)15;
    L.yS0 = o;  o += 8 * (size_t)F;
    L.aS0 = o;  o += 8 * (size_t)F;
    L.hy = o;   o += 8 * (size_t)NH;
    L.ha = o;   o += 8 * (size_t)NH;
    L.rloc = o; o += 8 * (size_t)WMAX;
    L.Gf = o;   o += 4 * (size_t)F;
    L.hG = o;   o += 4 * (size_t)NH;
    L.hw = o;   o += 4 * (size_t)conn * F;
    L.hs = o;   o += 2 * (size_t)conn * F;
    L.hl = o;   o += (size_t)NH;
    L.labw = o; o += (size_t)B;
    o = (o + 7) & ~(size_t)7;
    L.cI = o;   o += 8 * (size_t)F;
    L.cB = o;   o += 4 * (size_t)F;
    L.cW = o;   o += 4 * (size_t)F;
    L.cE = o;   o += 4 * (size_t)F;
    L.hB = o;   o += 4 * (size_t)NH;
    o = (o + 7) & ~(size_t)7;
    L.ring = o; o += 16 * (size_t)RING * F;
    L.window_end = o;
    return L;
}
__host__ __device__ inline size_t resident_smem_bytes(int conn, int B, int F) {
    return resident_layout(conn, B, F, 0).resident_end;
}

template <int CONN>
__device__ __forceinline__ void update_block_resident(const UpdArgs& A, int k, int t, double mu,
                                                      const SArr<uint8_t> lab, const SArr<double> yS,
                                                      const SArr<double> aS) {
    const Geo& g = A.g;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    constexpr int nh = CONN / 2;
    const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
    __shared__ double part[128];
    const int nchunks = (g.F + 31) >> 5;
    for (int ch = wid; ch < nchunks; ch += nw) {
        const int f = ch * 32 + lane;
        double d2 = 0.0;
        if (f < g.F) {
            const int v = A.faceLocal[f];
            const long long gi = (long long)k * g.B + v;
            int wj[CONN], yj[CONN];
#pragma unroll
            for (int d = 0; d < CONN; ++d) {
                int kn, ln, fn;
                wj[d] = 0;
                yj[d] = 0;
                if (halo_decode(g, A.halo[d * g.F + f], kz, ky, kx, kn, ln, fn)) {
                    const long long gj = (long long)kn * g.B + ln;
                    wj[d] = (d < nh) ? A.Wl[(long long)d * g.N + gi] : A.Wl[(long long)(d - nh) * g.N + gj];
                    yj[d] = __ldcg(&A.yhat[gj]);
                }
            }
            const int yh = lab[v];
            int G = 0;
#pragma unroll
            for (int d = 0; d < CONN; ++d) G += wj[d] * (yh - yj[d]);
            const long long sidx = (long long)k * g.F + f;
            const double gq = __dmul_rn((double)G, 0.0009765625);   // G / 1024, exact
            const double aa = aS[f];
            const double ya = __dadd_rn((double)yh, aa);
            const double yn = G ? __dsub_rn(ya, __ddiv_rn(gq, mu)) : ya;
            const double an = __dadd_rn(aa, __dsub_rn((double)yh, yn));
            yS[f] = yn;
            aS[f] = an;
            A.yF[sidx] = yn;
            A.aF[sidx] = an;
            const double dd = __dsub_rn((double)yh, yn);
            d2 = __dmul_rn(dd, dd);
        }
        for (int o = 16; o > 0; o >>= 1) d2 = __dadd_rn(d2, __shfl_xor_sync(0xffffffffu, d2, o));
        if (lane == 0) part[ch] = d2;
    }
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int ch = 0; ch < nchunks; ++ch) sum = __dadd_rn(sum, part[ch]);
        A.r2blk[k] = sum;
        atomicMax(&A.ctrl->r2max[t], (unsigned long long)__double_as_longlong(sum));
    }
    __syncthreads();
}


__host__ __device__ inline size_t window_smem_bytes(int conn, int B, int F, int NH) {
    return resident_layout(conn, B, F, NH).window_end;
}

// ---------------------------------------------------------------------------
// Run-ahead windows (resident kernel).  Once labels stop moving, a face
// pixel's y and a follow Eq. 10 / 11 with a constant cross sum G, and the Eq. 8
// unaries of the next iteration depend only on the block's own state and on
// its halo pixels' y.  A CTA can therefore run iterations ahead on its own:
// it keeps its halo pixels' y, a, label and G in shared memory, advances them
// with the same operations their owner uses, solves its block exactly each
// iteration and checks that the labels did not move.  The first iteration in
// which any block's labels moved (or the window end) bounds the valid run;
// iterations are only committed up to it, and the stop test is evaluated on
// the committed ones in order.  Every committed state is the one the ordinary
// iteration computes, bit for bit.
// ---------------------------------------------------------------------------
template <int CONN>
__global__ void __launch_bounds__(256, 2) k_admm_resident(PersistArgs P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Geo& g = P.s.g;
    const int B = g.B, F = g.F, NH = P.NH;
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = NT >> 5;
    const int k = blockIdx.x;                  // gridDim.x == K
    constexpr int nh = CONN / 2;
    Ctrl* c = P.s.ctrl;
    int* res_p = reinterpret_cast<int*>(smem);
    long long* C64_p = reinterpret_cast<long long*>(res_p + CONN * B);
    int* capsum_p = reinterpret_cast<int*>(C64_p + B);
    const SArr<int> res(res_p, (long long)CONN * B);
    const SArr<long long> C64(C64_p, B);
    const SArr<int> capsum(capsum_p, B);
    const SArr<uint8_t> st(reinterpret_cast<uint8_t*>(capsum_p + B), B);
    const ResidentLayout L = resident_layout(CONN, B, F, NH);
    const SArr<double> yS(reinterpret_cast<double*>(smem + L.yS), F);
    const SArr<double> aS(reinterpret_cast<double*>(smem + L.aS), F);
    const SArr<int> resW(reinterpret_cast<int*>(smem + L.resW), (long long)nh * B);
    const SArr<int> cs0(reinterpret_cast<int*>(smem + L.cs0), B);
    const SArr<int> Us(reinterpret_cast<int*>(smem + L.Us), B);
    const SArr<int16_t> fl(reinterpret_cast<int16_t*>(smem + L.fl), F);   // face slot -> local pixel
    const SArr<uint8_t> lab(smem + L.lab, B);
    // run-ahead window arrays: allocated (and touched) only when P.window
    const SArr<double> yS0(reinterpret_cast<double*>(smem + L.yS0), F);
    const SArr<double> aS0(reinterpret_cast<double*>(smem + L.aS0), F);
    const SArr<double> hy(reinterpret_cast<double*>(smem + L.hy), NH);
    const SArr<double> ha(reinterpret_cast<double*>(smem + L.ha), NH);
    const SArr<double> rloc(reinterpret_cast<double*>(smem + L.rloc), WMAX);
    const SArr<int> Gf(reinterpret_cast<int*>(smem + L.Gf), F);
    const SArr<int> hG(reinterpret_cast<int*>(smem + L.hG), NH);
    const SArr<int> hw(reinterpret_cast<int*>(smem + L.hw), (long long)CONN * F);
    const SArr<int16_t> hs(reinterpret_cast<int16_t*>(smem + L.hs), (long long)CONN * F);
    const SArr<uint8_t> hl(smem + L.hl, NH);
    const SArr<uint8_t> labw(smem + L.labw, B);
    const SArr<long long> cI(reinterpret_cast<long long*>(smem + L.cI), F);   // certificate: exact integer part
    const SArr<float> cB(reinterpret_cast<float*>(smem + L.cB), F);            // bound on |a|, |y - yhat|
    const SArr<float> cW(reinterpret_cast<float*>(smem + L.cW), F);            // sum_j w_j (B_i + B_j)
    const SArr<float> cE(reinterpret_cast<float*>(smem + L.cE), F);            // rounding allowance
    const SArr<float> hB(reinterpret_cast<float*>(smem + L.hB), NH);            // bound for halo pixels
    const SArr<double> ring(reinterpret_cast<double*>(smem + L.ring), (long long)RING * 2 * F);      // [RING][2][F] own y, a
    __shared__ long long s_tau;                                   // max interior |U| + n-link sum
    __shared__ double part[128];

    const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
    const int bw = g.bw, pl = g.bh * g.bw;
    unsigned long long imask = 0;
    unsigned fmask = 0;                          // bit q: own node q is a face pixel
    // one-time load of the owned block
#pragma unroll 1
    for (int q = 0; q < NPTMAX; ++q) {
        int v = tid + q * NT;
        if (v >= B) continue;
        const int lx = v % g.bw, ly = (v / g.bw) % g.bh, lz = v / (g.bw * g.bh);
        const long long gi = (long long)k * B + v;
        uint8_t m = 0;
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            int dz, dy, dx;
            dir_off<CONN>(d, dz, dy, dx);
            const int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
            const bool in = nlz >= 0 && nlz < g.bd && nly >= 0 && nly < g.bh && nlx >= 0 && nlx < g.bw;
            if (in) m |= (uint8_t)(1u << d);
            if (d < nh) resW[d * B + v] = in ? P.s.Wl[(long long)d * g.N + gi] : 0;
        }
        imask |= (unsigned long long)m << (8 * q);
        if (P.s.faceIndex[v] >= 0) fmask |= 1u << q;
        Us[v] = P.s.U[gi];
        lab[v] = P.t0 == 0 ? 0 : __ldcg(&P.s.yhat[gi]);
    }
    for (int f = tid; f < F; f += NT) {
        // Algorithm 1 starts from y = 1/2, a = 0
        yS[f] = P.t0 == 0 ? 0.5 : __ldcg(&P.s.yF[(long long)k * F + f]);
        aS[f] = P.t0 == 0 ? 0.0 : __ldcg(&P.s.aF[(long long)k * F + f]);
        fl[f] = P.s.faceLocal[f];
    }
    if (P.window) {
        // cross-edge weights and halo slots of the face slots, -1 where the
        // neighbour lies outside the grid
        for (int i = tid; i < CONN * F; i += NT) {
            const int d = i / F, f = i % F;
            int kn, ln, fn;
            int w = 0, slot = -1;
            if (halo_decode(g, P.s.halo[i], kz, ky, kx, kn, ln, fn)) {
                const long long gi = (long long)k * B + P.s.faceLocal[f];
                w = (d < nh) ? P.s.Wl[(long long)d * g.N + gi]
                             : P.s.Wl[(long long)(d - nh) * g.N + (long long)kn * B + ln];
                slot = P.hslot[i];
            }
            hw[i] = w;
            hs[i] = (int16_t)slot;
        }
    }
    if (blockIdx.x == 0 && tid == 0) c->thaw = 0x7fffffff;
    __syncthreads();
#pragma unroll 1
    for (int q = 0; q < NPTMAX; ++q) {
        int v = tid + q * NT;
        if (v >= B) continue;
        const unsigned m = (unsigned)(imask >> (8 * q)) & 0xffu;
        int cs = 0;
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            if (d < nh) cs += resW[d * B + v];
            else if ((m >> d) & 1) cs += resW[(d - nh) * B + v + dir_lofs<CONN>(d, bw, pl)];
        }
        cs0[v] = cs;
    }
    if (tid == 0) s_tau = 0;
    __syncthreads();
    {   // interior pixels are forced to keep their label once 512 mu exceeds this
        long long tmax = 0;
#pragma unroll 1
        for (int q = 0; q < NPTMAX; ++q) {
            int v = tid + q * NT;
            if (v < B && !((fmask >> q) & 1u)) {
                const long long u = Us[v];
                const long long x = (u < 0 ? -u : u) + cs0[v] + 2;
                tmax = x > tmax ? x : tmax;
            }
        }
        if (tmax) atomicMax(&s_tau, tmax);
    }
    __syncthreads();
    const long long tau_int = s_tau;

    // Eq. 8 unary of face slot f with the halo y from the window's halo copy
    // (the operations of face_cap_core, in the same order).
    auto local_face_cap = [&](int f, int v, double m1024) -> long long {
        const double yv = yS[f], av = aS[f];
        double sv = (double)Us[v];
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            const int hsl = hs[d * F + f];
            if (hsl >= 0) sv = __dadd_rn(sv, __dmul_rn((double)hw[d * F + f], __dsub_rn(yv, hy[hsl])));
        }
        sv = __dadd_rn(sv, __dmul_rn(m1024, __dadd_rn(__dsub_rn(av, yv), 0.5)));
        sv = fmin(fmax(sv, -CLAMP62), CLAMP62);
        return __double2ll_rn(sv);
    };
    // Build of iteration t (first = t is 1): n-links and interior unaries from
    // shared memory; face unaries with the halo y from L2 (hy == nullptr) or
    // from the window's halo copy.
    auto build = [&](bool first, double m1024, int int_test, long long H, bool local) {
#pragma unroll 1
        for (int q = 0; q < NPTMAX; ++q) {
            int v = tid + q * NT;
            if (v >= B) continue;
            const int cs = cs0[v];
            capsum[v] = cs;
            st[v] = FREE;
            const long long Ui = Us[v];
            long long cv = Ui;
            if (!first && !((fmask >> q) & 1u)) {
                const int yh = lab[v];
                const long long T = yh ? Ui - H : Ui + H;
                if (int_test && (yh ? (T < -(long long)cs) : (T >= (long long)cs))) cv = T;
                else cv = interior_cap(Ui, yh, m1024);
            }
            C64[v] = cv;
        }
        if (!first) {
            for (int f = tid; f < F; f += NT) {
                const int v = fl[f];
                long long cv;
                if (!local) {
                    cv = face_cap_core<CONN>(g, (long long)Us[v], yS[f], aS[f], P.s.Wl, P.s.yF, P.s.halo, k,
                                             kz, ky, kx, v, f, m1024);
                } else {
                    cv = local_face_cap(f, v, m1024);
                }
                C64[v] = cv;
            }
        }
        __syncthreads();
    };
    // Intra-block n-links into the solver's residual array (needed only when
    // some node is not forced).
    auto copy_res = [&]() {
#pragma unroll 1
        for (int q = 0; q < NPTMAX; ++q) {
            int v = tid + q * NT;
            if (v >= B) continue;
            const unsigned m = (unsigned)(imask >> (8 * q)) & 0xffu;
#pragma unroll
            for (int d = 0; d < CONN; ++d)
                res[d * B + v] = d < nh ? resW[d * B + v]
                               : (((m >> d) & 1) ? resW[(d - nh) * B + v + dir_lofs<CONN>(d, bw, pl)] : 0);
        }
        __syncthreads();
    };
    // When every node is forced in the first folding round (C >= its n-link
    // sum: label 0; C < minus it: label 1) the labels are those cut_block
    // returns, without the max-flow; out receives them.  false: some node is
    // free and cut_block must run.
    auto fast_forced = [&](const SArr<uint8_t> out) -> bool {
        int fr = 0;
#pragma unroll 1
        for (int q = 0; q < NPTMAX; ++q) {
            int v = tid + q * NT;
            if (v >= B) continue;
            const long long cv = C64[v], cs = cs0[v];
            if (!(cv >= cs) && !(cv < -cs)) fr = 1;
        }
        if (__syncthreads_or(fr)) return false;
#pragma unroll 1
        for (int q = 0; q < NPTMAX; ++q) {
            int v = tid + q * NT;
            if (v >= B) continue;
            out[v] = C64[v] >= (long long)cs0[v] ? 0 : 1;
        }
        return true;
    };
    // Fixed-order block sum of per-face-slot values computed by fn(f) (the
    // order update_block uses for r_k^2).
    auto face_sum = [&](auto fn) -> double {
        const int nchunks = (F + 31) >> 5;
        for (int ch = wid; ch < nchunks; ch += nw) {
            const int f = ch * 32 + lane;
            double d2 = f < F ? fn(f) : 0.0;
            for (int o = 16; o > 0; o >>= 1) d2 = __dadd_rn(d2, __shfl_xor_sync(0xffffffffu, d2, o));
            if (lane == 0) part[ch] = d2;
        }
        __syncthreads();
        double t2 = 0.0;
        if (tid == 0)
            for (int ch = 0; ch < nchunks; ++ch) t2 = __dadd_rn(t2, part[ch]);
        __syncthreads();
        return t2;   // valid in thread 0
    };
    auto iter_consts = [&](double mu, double& m1024, int& int_test, long long& H) {
        m1024 = __dmul_rn(1024.0, mu);
        const double h = __dmul_rn(m1024, 0.5);
        int_test = h < 4503599627370496.0 ? 1 : 0;   // 2^52
        H = int_test ? (long long)floor(h) : 0;
    };

    const int tlimit = P.t0 + P.n;
    double mu = P.mu_start;
    int t = P.t0, conv = 0;
    unsigned nbar = 0;
    bool need_normal = true, failed = false;
    while (t < tlimit && !failed) {
        if (need_normal || !P.window) {
            // ordinary iteration t+1
            ++t;
            double m1024; int int_test; long long H;
            iter_consts(mu, m1024, int_test, H);
            const long long c0 = clock64();
            build(t == 1, m1024, int_test, H, false);
            if (t > 1 && fast_forced(lab)) {
#pragma unroll 1
                for (int q = 0; q < NPTMAX; ++q) {
                    int v = tid + q * NT;
                    if (v < B) P.s.yhat[(long long)k * B + v] = lab[v];
                }
            } else {
                copy_res();
                cut_block<CONN>(P.s, k, smem, bw, pl, imask, c0, lab.p);
            }
            const long long c1 = clock64();
            if (!grid_sync(c, gridDim.x, nbar, P.spin_limit)) { failed = true; break; }
            const long long c2 = clock64();
            update_block_resident<CONN>(P.u, k, t, mu, lab, yS, aS);
            const long long c3 = clock64();
            mu = __dmul_rn(mu, P.mu_fact);
            if (!grid_sync(c, gridDim.x, nbar, P.spin_limit)) { failed = true; break; }
            if (tid == 0) {
                atomicAdd(&c->pcyc[0], (unsigned long long)(c1 - c0));
                atomicAdd(&c->pcyc[1], (unsigned long long)(c2 - c1));
                atomicAdd(&c->pcyc[2], (unsigned long long)(c3 - c2));
            }
            const double r2 = __longlong_as_double((long long)__ldcg(&c->r2max[t]));
            if (!(__dsqrt_rn(r2) > P.s.eps)) { conv = 1; break; }
            need_normal = (t == 1);
            continue;
        }
        // ---- run-ahead window from iteration tw = t ----
        const int tw = t;
        // Once labels are frozen every block residual shrinks by 1/mu_fact per
        // iteration, so the stop test is expected about ln(r/eps)/ln(mu_fact)
        // iterations on; the window is cut there (plus one) instead of running
        // WMAX iterations past the stop.  This only sizes the window; what is
        // committed is decided by the exact stop test below.
        int Wn = min(WMAX, tlimit - tw);
        {
            const double r_tw = __dsqrt_rn(__longlong_as_double((long long)__ldcg(&c->r2max[tw])));
            const double r_pr = tw >= 2 ? __dsqrt_rn(__longlong_as_double((long long)__ldcg(&c->r2max[tw - 1])))
                                        : 0.0;
            // the geometric regime shows as r_tw / r_{tw-1} = 1 / mu_fact
            const bool geometric = r_pr > 0.0 && fabs(r_tw * P.mu_fact / r_pr - 1.0) < 1e-3;
            if (r_tw > P.s.eps && P.mu_fact > 1.0) {
                const double n_pred = ceil(log(r_tw / P.s.eps) / log(P.mu_fact));
                if (n_pred + 1.0 < (double)Wn) Wn = max(1, (int)n_pred + 1);
            }
            if (!geometric) Wn = min(Wn, 16);
        }
        const long long c0 = clock64();
        for (int f = tid; f < F; f += NT) { yS0[f] = yS[f]; aS0[f] = aS[f]; }
        // own cross sums G (constant while labels do not move)
        for (int f = tid; f < F; f += NT) {
            const int v = fl[f];
            int G = 0;
#pragma unroll
            for (int d = 0; d < CONN; ++d) {
                int kn, ln, fn;
                if (hs[d * F + f] >= 0 && halo_decode(g, P.s.halo[d * F + f], kz, ky, kx, kn, ln, fn))
                    G += hw[d * F + f] * ((int)lab[v] - (int)__ldcg(&P.s.yhat[(long long)kn * B + ln]));
            }
            Gf[f] = G;
        }
        // halo pixels: state, label and their own cross sums
        for (int h = tid; h < NH; h += NT) {
            int kn, ln, fn;
            if (!halo_decode(g, P.hinfo[h], kz, ky, kx, kn, ln, fn)) continue;
            const int knz = kn / (g.nby * g.nbx), kny = (kn / g.nbx) % g.nby, knx = kn % g.nbx;
            hy[h] = __ldcg(&P.s.yF[(long long)kn * F + fn]);
            ha[h] = __ldcg(&P.s.aF[(long long)kn * F + fn]);
            const int yh = __ldcg(&P.s.yhat[(long long)kn * B + ln]);
            hl[h] = (uint8_t)yh;
            int G = 0;
#pragma unroll
            for (int d = 0; d < CONN; ++d) {
                int km, lm, fm;
                if (halo_decode(g, P.s.halo[d * F + fn], knz, kny, knx, km, lm, fm)) {
                    const long long gj = (long long)kn * B + ln;
                    const int w = (d < nh) ? P.s.Wl[(long long)d * g.N + gj]
                                           : P.s.Wl[(long long)(d - nh) * g.N + (long long)km * B + lm];
                    G += w * (yh - (int)__ldcg(&P.s.yhat[(long long)km * B + lm]));
                }
            }
            hG[h] = G;
        }
        __syncthreads();
        // Certificates (see the note on the frozen regime above the loop): with
        // labels frozen, a_t = g / mu_t and y_t - yhat = a_{t-1} - g / mu_t in
        // exact arithmetic (g = G / 1024), each computed step adding at most a
        // few ulps (no accumulation, since a is reset to g / mu every step), so
        //   B = |a_tw| + |y_tw - yhat| + 2 |g| / mu_tw + 2^-40
        // bounds |a| and |y - yhat| for every state of the window.
        const double inv_mu_tw = 1.0 / mu;   // 1 / mu of the window's first iteration (bounds only)
        for (int h = tid; h < NH; h += NT) {
            const double b = fabs(ha[h]) + fabs(hy[h] - (double)hl[h]) +
                             2.0 * fabs((double)hG[h]) * 0.0009765625 * inv_mu_tw * (1.0 + 1e-12) +
                             9.094947017729282e-13;   // 2^-40
            hB[h] = __double2float_ru(b);
        }
        __syncthreads();
        for (int f = tid; f < F; f += NT) {
            const int v = fl[f];
            const double b = fabs(aS[f]) + fabs(yS[f] - (double)lab[v]) +
                             2.0 * fabs((double)Gf[f]) * 0.0009765625 * inv_mu_tw * (1.0 + 1e-12) +
                             9.094947017729282e-13;
            const float bf = __double2float_ru(b);
            long long I = Us[v], wtot = 0;
            float wsum = 0.f;
#pragma unroll
            for (int d = 0; d < CONN; ++d) {
                const int hsl = hs[d * F + f];
                if (hsl < 0) continue;
                const int w = hw[d * F + f];
                I += (long long)w * ((int)lab[v] - (int)hl[hsl]);
                wsum = __fadd_ru(wsum, __fmul_ru((float)w, __fadd_ru(bf, hB[hsl])));
                wtot += w;
            }
            cI[f] = I;
            cB[f] = bf;
            cW[f] = wsum;
            // allowance for the computed value vs the exact one: 2^-40 (|I| + 3 sum w)
            // here, plus 2^-40 * 2h per iteration below
            cE[f] = __double2float_ru(9.094947017729282e-13 * ((double)llabs(I) + 3.0 * (double)wtot) *
                                      (1.0 + 1e-12));
        }
        __syncthreads();
        double muw = mu;
        int thaw_s = Wn + 1;
        long long wc[5] = {0, 0, 0, 0, 0};
        const long long cs_start = clock64();
        for (int sidx = 1; sidx <= Wn; ++sidx) {
            double m1024; int int_test; long long H;
            iter_consts(muw, m1024, int_test, H);
            long long ta = clock64();
            // Certified frozen iteration: every interior pixel forced by the
            // integer bound, every face pixel forced (to its own label) by
            // its certificate -> the labels do not move; no unaries needed.
            bool cert = int_test && P.mu_fact >= 1.0;
            if (cert) {
                const float mf = __double2float_ru(m1024);
                const float e2h = __fmul_ru(1.8189894035458565e-12f, __double2float_ru(__dmul_rn(m1024, 0.5)));  // 2^-40 * 2h
                int okc = 1;
                if (H < tau_int) {
                    // interior pixels one by one: the integer bound, else the exact unary
#pragma unroll 1
                    for (int q = 0; q < NPTMAX; ++q) {
                        int v = tid + q * NT;
                        if (v >= B || ((fmask >> q) & 1u)) continue;
                        const int yh = lab[v];
                        const long long Ui = Us[v], cs = cs0[v];
                        const long long T = yh ? Ui - H : Ui + H;
                        bool ok = yh ? (T < -cs) : (T >= cs);
                        if (!ok) {
                            const long long C = interior_cap(Ui, yh, m1024);
                            ok = yh ? (C < -cs) : (C >= cs);
                        }
                        okc &= ok ? 1 : 0;
                    }
                }
                for (int f = tid; f < F; f += NT) {
                    const int v = fl[f];
                    const float dl = __fadd_ru(__fadd_ru(cW[f], __fmul_ru(__fmul_ru(2.f, mf), cB[f])),
                                               __fadd_ru(cE[f], e2h));
                    if (!(dl < 4.0e18f)) { okc = 0; continue; }
                    const long long D = (long long)ceilf(dl) + 1;
                    const long long cs = cs0[v];
                    bool ok = lab[v] ? (cI[f] - H + D + 1 <= -cs) : (cI[f] + H - D - 1 >= cs);
                    if (!ok) {
                        // no certificate: the exact unary decides for this pixel
                        const long long C = local_face_cap(f, v, m1024);
                        ok = lab[v] ? (C < -cs) : (C >= cs);
                    }
                    okc &= ok ? 1 : 0;
                }
                cert = __syncthreads_and(okc) != 0;
            }
            long long tb = ta, tc = ta;
            if (!cert) {
                build(false, m1024, int_test, H, true);
                tb = clock64();
                if (!fast_forced(labw)) {
                    copy_res();
                    cut_block<CONN>(P.s, k, smem, bw, pl, imask, clock64(), labw.p, false);
                }
                tc = clock64();
                int moved = 0;
#pragma unroll 1
                for (int q = 0; q < NPTMAX; ++q) {
                    int v = tid + q * NT;
                    if (v < B && labw[v] != lab[v]) moved = 1;
                }
                if (__syncthreads_or(moved)) { thaw_s = sidx; break; }
            }
            long long td = clock64();
            const double r2 = face_sum([&](int f) {
                return face_step(lab[fl[f]], Gf[f], muw, yS[f], aS[f]);
            });
            if (tid == 0) rloc[sidx - 1] = r2;
            {
                const SArr<double> rs = ring.sub((long long)(sidx % RING) * 2 * F, 2LL * F);
                for (int f = tid; f < F; f += NT) { rs[f] = yS[f]; rs[F + f] = aS[f]; }
            }
            long long te = clock64();
            for (int h = tid; h < NH; h += NT) {
                double yv = hy[h], av = ha[h];
                face_step(hl[h], hG[h], muw, yv, av);
                hy[h] = yv;
                ha[h] = av;
            }
            muw = __dmul_rn(muw, P.mu_fact);
            __syncthreads();
            long long tf = clock64();
            wc[0] += tb - ta; wc[1] += tc - tb; wc[2] += td - tc; wc[3] += te - td; wc[4] += tf - te;
        }
        if (tid == 0) {
            for (int i = 0; i < 5; ++i) atomicAdd(&c->wcyc[i], (unsigned long long)wc[i]);
            atomicAdd(&c->wcyc[5], (unsigned long long)(cs_start - c0));
        }
        // resolution: earliest moved iteration over all blocks, committed residuals
        if (tid == 0) atomicMin(&c->thaw, tw + thaw_s);
        const long long cr0 = clock64();
        if (!grid_sync(c, gridDim.x, nbar, P.spin_limit)) { failed = true; break; }
        const long long cr1 = clock64();
        const int tstar = __ldcg(&c->thaw);
        const int tvalid = min(tstar - 1, tw + Wn);
        if (tid == 0)
            for (int tt = tw + 1; tt <= tvalid; ++tt)
                atomicMax(&c->r2max[tt], (unsigned long long)__double_as_longlong(rloc[tt - tw - 1]));
        if (!grid_sync(c, gridDim.x, nbar, P.spin_limit)) { failed = true; break; }
        if (blockIdx.x == 0 && tid == 0) {
            c->thaw = 0x7fffffff;
            c->windows += 1;
            c->window_iters += tvalid - tw;
        }
        // first committed iteration whose stop test holds (all candidates read at once)
        __shared__ int s_stop;
        if (tid == 0) s_stop = 0x7fffffff;
        __syncthreads();
        for (int tt = tw + 1 + tid; tt <= tvalid; tt += NT) {
            const double r2 = __longlong_as_double((long long)__ldcg(&c->r2max[tt]));
            if (!(__dsqrt_rn(r2) > P.s.eps)) atomicMin(&s_stop, tt);
        }
        __syncthreads();
        int tend = tvalid;
        if (s_stop <= tvalid) { tend = s_stop; conv = 1; }
        // own face state at tend: the current one, one kept in the ring, or a
        // replay of the committed iterations from the window start
        const int sdone = thaw_s - 1;                  // iterations this CTA advanced
        const int back = (tw + sdone) - tend;          // iterations to undo
        if (back > 0 && back < RING && tend > tw) {
            const SArr<double> rs = ring.sub((long long)((tend - tw) % RING) * 2 * F, 2LL * F);
            for (int f = tid; f < F; f += NT) { yS[f] = rs[f]; aS[f] = rs[F + f]; }
        } else if (back > 0) {
            for (int f = tid; f < F; f += NT) {
                double yv = yS0[f], av = aS0[f];
                double m = mu;
                const int yh = lab[fl[f]];
                for (int tt = tw + 1; tt <= tend; ++tt) {
                    face_step(yh, Gf[f], m, yv, av);
                    m = __dmul_rn(m, P.mu_fact);
                }
                yS[f] = yv;
                aS[f] = av;
            }
        }
        __syncthreads();
        for (int f = tid; f < F; f += NT) {
            P.u.yF[(long long)k * F + f] = yS[f];
            P.u.aF[(long long)k * F + f] = aS[f];
        }
        for (int tt = tw + 1; tt <= tend; ++tt) mu = __dmul_rn(mu, P.mu_fact);
        t = tend;
        const long long c1 = clock64();
        if (tid == 0) {
            atomicAdd(&c->pcyc[3], (unsigned long long)(c1 - c0));
            atomicAdd(&c->wcyc[6], (unsigned long long)(cr1 - cr0));
            atomicAdd(&c->wcyc[7], (unsigned long long)(c1 - cr1));
        }
        if (conv) break;
        if (!grid_sync(c, gridDim.x, nbar, P.spin_limit)) { failed = true; break; }
        need_normal = (tstar <= tw + Wn);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->iters_done = t;
        c->conv_t = conv ? t : 0;
    }
    if (!failed && (P.out_labels || P.out_energy)) {
        __shared__ long long s_red[32];
        if (grid_sync(c, gridDim.x, nbar, P.spin_limit)) finish_block<CONN>(P, k, s_red);
    }
}

#ifndef DOPE_KERNEL_TEMPLATES_ONLY   // the batched launch and its constant table live in one translation unit
// ---------------------------------------------------------------------------
// Batched path: many problems (contexts) advanced in one cooperative launch.
// Every iteration the blocks of all live problems form one list (live problem
// q owns entries base_q .. base_q + K_q - 1) handed out by an atomic counter,
// in the solve phase and again in the update phase.  Each problem keeps its
// own iteration count, mu and stop test (Algorithm 1 per problem, unchanged),
// and the per-block arithmetic is that of the single-problem kernels, so a
// problem's iterates are bit-identical whatever it is batched with.  A problem
// leaves the list when its stop test holds or its allowance of iterations is
// used up.  The launch ends when no problem is left, when the host's yield
// flag is set (read at an iteration boundary) or, if asked, at the first
// boundary where a problem finished while others go on.
// ---------------------------------------------------------------------------
constexpr int BATCH_MAX = 256;   // problems per launch

// Per-problem arguments of the block solver and the face update, in constant
// memory: every CTA reads the same problem's fields, which the constant cache
// broadcasts, as the single-problem kernels read theirs from the kernel
// parameters.  Written by the host before each batched launch (one batched
// launch in flight per process at a time).
struct BatchDesc {
    Geo g;
    const int32_t* U;
    const int32_t* Wl;
    uint8_t* yhat;
    double* yF;
    double* aF;
    double* r2blk;
    const int16_t* faceIndex;
    const int* halo;
    const int16_t* faceLocal;
    const long long* Cgiven;        // always null here
    Ctrl* ctrl;
    double eps;
    int relabel_period, max_pulses, fold_rounds, conn;
    unsigned char* sched;           // always null here (no worklists in the batched launch)
    unsigned epoch;
};

__constant__ BatchDesc c_batch[BATCH_MAX];

// Per-problem loop state of a batched launch (device memory).
struct BatchProb {
    int t0;                 // iterations done before the launch
    int n;                  // iterations allowed in this launch
    int K;                  // blocks
    int cont;               // 1: the worklists left by this problem's previous launch hold
    double mu;              // mu of iteration t0 + 1
    double mu_fact;
};

// Per-problem result of a batched launch (written by CTA 0 at its end).
struct BatchOut {
    int t;                  // iterations done
    int conv;               // the stop test held at iteration t
    int status;             // the problem's status word
    int pad;
    double mu;              // mu of iteration t + 1
    double r2;              // max_k r2_k of iteration t (0 if t = 0)
    unsigned long long work[2];   // the problem's block solves / updates run from its worklists so far
};

struct BatchArgs {
    const BatchProb* probs; // [nprob], device memory
    BatchOut* out;          // [nprob]
    int nprob;              // 1 .. BATCH_MAX
    int exit_on_done;
    const int* yield_flag;  // host-mapped or device int; nonzero ends the launch (may be null)
    Ctrl* bc;               // barrier and block counters of the launch (zeroed by the host)
    long long spin_limit;
};

// Live problem owning list entry gk (binary search over the live bases).
__device__ __forceinline__ int batch_owner(const int* lbase, int nlive, int gk) {
    int lo = 0, hi = nlive - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (lbase[mid] <= gk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Warp 0: exclusive prefix sums of s_cnt[0 .. nlive) into s_lbase, the total
// into *s_total (ballot-free shuffle scan in chunks of 32).
__device__ __forceinline__ void batch_scan(const int* s_cnt, int* s_lbase, int nlive, int* s_total) {
    const int lane = threadIdx.x & 31;
    int run = 0;
    for (int c0 = 0; c0 < nlive; c0 += 32) {
        const int q = c0 + lane;
        const int kp = q < nlive ? s_cnt[q] : 0;
        int v = kp;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (q < nlive) s_lbase[q] = run + v - kp;
        run += __shfl_sync(0xffffffffu, v, 31);
    }
    if (lane == 0) *s_total = run;
}

template <int NT>
__global__ void __launch_bounds__(NT, SolverOcc<NT>::min_blocks) k_admm_batch(BatchArgs P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double s_mu[BATCH_MAX];
    __shared__ int s_t[BATCH_MAX];
    __shared__ int s_K[BATCH_MAX];
    __shared__ int s_list[BATCH_MAX];     // live problems, in problem order
    __shared__ int s_lbase[BATCH_MAX];    // their first entries in the phase's list
    __shared__ int s_cnt[BATCH_MAX];      // their entries in the phase's list
    __shared__ unsigned char s_alive[BATCH_MAX];
    __shared__ unsigned char s_conv[BATCH_MAX];
    __shared__ unsigned char s_full[BATCH_MAX];   // 1: this iteration does every block of the problem
    __shared__ int s_nlive, s_total, s_k, s_any, s_done;
    __shared__ int s_gp[MB], s_gk[MB], s_gq[MB], s_gpk[MB], s_gok[MB], s_gnp;   // a piece of list entries
    const int np = P.nprob;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    Ctrl* bc = P.bc;
    for (int p = tid; p < np; p += blockDim.x) {
        const BatchProb bp = P.probs[p];
        s_t[p] = bp.t0;
        s_mu[p] = bp.mu;
        s_K[p] = bp.K;
        s_alive[p] = (bp.n > 0 && __ldcg(&c_batch[p].ctrl->status) == 0) ? 1 : 0;
        s_conv[p] = 0;
    }
    __syncthreads();
    unsigned nbar = 0;
    for (;;) {
        // live list (warp 0, ballot compaction)
        if (wid == 0) {
            int cnt = 0;
            for (int c0 = 0; c0 < np; c0 += 32) {
                const int p = c0 + lane;
                const bool al = p < np && s_alive[p];
                const unsigned m = __ballot_sync(0xffffffffu, al);
                if (al) s_list[cnt + __popc(m & ((1u << lane) - 1u))] = p;
                cnt += __popc(m);
            }
            if (lane == 0) s_nlive = cnt;
        }
        __syncthreads();
        const int nlive = s_nlive;
        if (nlive == 0) break;
        // with worklists, a problem's first iteration in the launch does every
        // block, later ones the blocks on its lists (see sched_view)
        for (int q = tid; q < nlive; q += blockDim.x) {
            const int p = s_list[q];
            const int t = s_t[p] + 1;
            const bool full = c_batch[p].sched == nullptr || (s_t[p] == P.probs[p].t0 && !P.probs[p].cont);
            s_full[p] = full ? 1 : 0;
            s_cnt[q] = full ? s_K[p] : (int)__ldcg(&sched_view(c_batch[p].sched, s_K[p]).sq_n[t & 1]);
        }
        __syncthreads();
        if (wid == 0) batch_scan(s_cnt, s_lbase, nlive, &s_total);
        __syncthreads();
        int total = s_total;
        // solve phase (the update counter is idle now and is reset here, as are
        // the next iteration's solve-list counts)
        if (blockIdx.x == 0) {
            if (tid == 0) bc->work[1] = 0u;
            for (int q = tid; q < nlive; q += blockDim.x) {
                const int p = s_list[q];
                if (c_batch[p].sched) sched_view(c_batch[p].sched, s_K[p]).sq_n[(s_t[p] + 2) & 1] = 0u;
            }
        }
        // a few entries at a time; the forced blocks of one problem among them
        // are re-evaluated together (partial_solve_multi), the others one by one
        auto solve_piece = [&](int g0, int nb) {
            if (tid < nb) {
                const int q = batch_owner(s_lbase, nlive, g0 + tid);
                const int p = s_list[q];
                const int i = g0 + tid - s_lbase[q];
                const int t = s_t[p] + 1;
                const int kb = s_full[p] ? i
                                         : __ldcg(&sched_view(c_batch[p].sched, s_K[p]).sq[(size_t)(t & 1) * s_K[p] + i]);
                s_gp[tid] = p;
                s_gk[tid] = kb;
                s_gq[tid] = s_full[p] ? 0 : __ldcg(&sched_view(c_batch[p].sched, s_K[p]).qs[kb]);
            }
            __syncthreads();
            for (int j0 = 0; j0 < nb;) {
                const int p = s_gp[j0];
                int j1 = j0 + 1;
                while (j1 < nb && s_gp[j1] == p) ++j1;
                const int t = s_t[p] + 1;
                IterArgs it = iter_args(t, s_mu[p]);
                it.qeval = !s_full[p];
                const int conn = c_batch[p].conn;
                if (tid == 0) {
                    int np = 0;
                    for (int j = j0; j < j1; ++j)
                        if (s_gq[j]) s_gpk[np++] = s_gk[j];
                    s_gnp = np;
                }
                __syncthreads();
                if (s_gnp) {
                    if (conn == 4) partial_solve_multi<4>(c_batch[p], it, s_gpk, s_gnp, s_gok);
                    else if (conn == 8) partial_solve_multi<8>(c_batch[p], it, s_gpk, s_gnp, s_gok);
                    else partial_solve_multi<6>(c_batch[p], it, s_gpk, s_gnp, s_gok);
                }
                for (int j = j0, jp = 0; j < j1; ++j) {
                    bool done = false;
                    if (s_gq[j]) done = s_gok[jp++] != 0;
                    if (done) continue;
                    if (conn == 4) solve_block<4>(c_batch[p], it, s_gk[j], smem, false);
                    else if (conn == 8) solve_block<8>(c_batch[p], it, s_gk[j], smem, false);
                    else solve_block<6>(c_batch[p], it, s_gk[j], smem, false);
                }
                __syncthreads();
                j0 = j1;
            }
        };
        list_pieces(total, &bc->work[0], &s_k, solve_piece);
        if (!grid_sync(bc, gridDim.x, nbar, P.spin_limit)) break;
        // update phase
        for (int q = tid; q < nlive; q += blockDim.x) {
            const int p = s_list[q];
            const int t = s_t[p] + 1;
            if (!s_full[p] && blockIdx.x == 0) {
                atomicAdd(&c_batch[p].ctrl->sched_work[0], (unsigned long long)s_cnt[q]);
            }
            s_cnt[q] = s_full[p] ? s_K[p] : (int)__ldcg(&sched_view(c_batch[p].sched, s_K[p]).uq_n[t & 1]);
        }
        __syncthreads();
        if (wid == 0) batch_scan(s_cnt, s_lbase, nlive, &s_total);
        __syncthreads();
        total = s_total;
        if (blockIdx.x == 0) {
            if (tid == 0) bc->work[0] = 0u;
            for (int q = tid; q < nlive; q += blockDim.x) {
                const int p = s_list[q];
                if (c_batch[p].sched) {
                    sched_view(c_batch[p].sched, s_K[p]).uq_n[(s_t[p] + 2) & 1] = 0u;
                    if (!s_full[p]) atomicAdd(&c_batch[p].ctrl->sched_work[1], (unsigned long long)s_cnt[q]);
                }
            }
        }
        // a few entries at a time; the blocks of one problem among them are
        // updated together
        auto update_piece = [&](int g0, int nb) {
            if (tid < nb) {
                const int q = batch_owner(s_lbase, nlive, g0 + tid);
                const int p = s_list[q];
                const int i = g0 + tid - s_lbase[q];
                const int t = s_t[p] + 1;
                const int kb = s_full[p] ? i
                                         : __ldcg(&sched_view(c_batch[p].sched, s_K[p]).uq[(size_t)(t & 1) * s_K[p] + i]);
                s_gp[tid] = p;
                s_gk[tid] = kb;
            }
            __syncthreads();
            for (int j0 = 0; j0 < nb;) {
                const int p = s_gp[j0];
                int j1 = j0 + 1;
                while (j1 < nb && s_gp[j1] == p) ++j1;
                const int t = s_t[p] + 1;
                const int conn = c_batch[p].conn;
                if (conn == 4) update_blocks<4>(c_batch[p], s_mu[p], t, s_gk + j0, j1 - j0, s_full[p]);
                else if (conn == 8) update_blocks<8>(c_batch[p], s_mu[p], t, s_gk + j0, j1 - j0, s_full[p]);
                else update_blocks<6>(c_batch[p], s_mu[p], t, s_gk + j0, j1 - j0, s_full[p]);
                j0 = j1;
            }
        };
        list_pieces(total, &bc->work[1], &s_k, update_piece);
        if (blockIdx.x == 0 && tid == 0) {
            unsigned y = 0;
            if (P.yield_flag) {
                cuda::atomic_ref<const int, cuda::thread_scope_system> f(*P.yield_flag);
                y = f.load(cuda::memory_order_relaxed) != 0 ? 1u : 0u;
            }
            bc->yield = y;
        }
        if (!grid_sync(bc, gridDim.x, nbar, P.spin_limit)) break;
        // per-problem stop tests; every CTA takes the same decisions
        if (tid == 0) { s_any = 0; s_done = 0; }
        __syncthreads();
        for (int q = tid; q < nlive; q += blockDim.x) {
            const int p = s_list[q];
            const int t = s_t[p] + 1;
            const double r2 = __longlong_as_double((long long)__ldcg(&c_batch[p].ctrl->r2max[t]));
            const bool conv = !(__dsqrt_rn(r2) > c_batch[p].eps);
            s_t[p] = t;
            s_mu[p] = __dmul_rn(s_mu[p], P.probs[p].mu_fact);
            if (conv || t - P.probs[p].t0 >= P.probs[p].n) {
                s_alive[p] = 0;
                s_conv[p] = conv ? 1 : 0;
                s_done = 1;
            } else {
                s_any = 1;
            }
        }
        __syncthreads();
        const unsigned yield = __ldcg(&bc->yield);
        if (!s_any || yield || (P.exit_on_done && s_done)) break;
    }
    if (blockIdx.x == 0) {
        for (int p = tid; p < np; p += blockDim.x) {
            const Ctrl* c = c_batch[p].ctrl;
            BatchOut o;
            o.t = s_t[p];
            o.conv = s_conv[p];
            o.status = __ldcg(&c->status);
            o.pad = 0;
            o.mu = s_mu[p];
            o.r2 = o.t > 0 ? __longlong_as_double((long long)__ldcg(&c->r2max[o.t])) : 0.0;
            o.work[0] = __ldcg(&c->sched_work[0]);
            o.work[1] = __ldcg(&c->sched_work[1]);
            P.out[p] = o;
        }
    }
}

// Before a batched launch (one CTA per problem): zero the launch's barrier
// and block counters, the trace slots the launch will fill and, if asked,
// each problem's status word.
__global__ void k_batch_prep(BatchArgs P, int clear_status) {
    const int p = blockIdx.x;
    if (p == 0 && threadIdx.x == 0) {
        Ctrl* bc = P.bc;
        bc->status = 0;
        bc->bar_count = 0u;
        bc->abort = 0;
        bc->yield = 0u;
        bc->work[0] = 0u;
        bc->work[1] = 0u;
    }
    if (p >= P.nprob) return;
    const BatchProb bp = P.probs[p];
    Ctrl* c = c_batch[p].ctrl;
    if (threadIdx.x == 0 && clear_status) {
        c->status = 0;
        c->conv_t = 0;
    }
    for (int j = threadIdx.x; j < bp.n; j += blockDim.x) c->r2max[bp.t0 + 1 + j] = 0ull;
}
#endif  // DOPE_KERNEL_TEMPLATES_ONLY

}  // namespace dope
