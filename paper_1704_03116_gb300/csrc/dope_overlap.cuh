// dope_overlap.cuh -- device code of the overlapping-block path (Q != I,
// the paper's Size10 / Size25 partitions).  Included by dope.cu after
// dope_kernels.cuh; reuses its block cut (cut_block).
//
// Partition: the regular tiling by (tbd, tbh, tbw) with every tile grown by
// (gd, gh, gw) pixels on each side, clipped to the grid; 2 g <= tile side per
// axis, so a pixel lies in at most two blocks per axis and q_i (Proposition 1:
// the number of blocks holding i) is 1, 2, 4 or 8.  Block k is stored as the
// full box of (tile + 2 grow) pixels around tile k ("box-major": node l of
// block k at k * B + l); box nodes outside the grid are phantoms (no unary, no
// n-links, label 0).
//
// Theorem 1 per pixel, for i in Omega_k, phi_kj = 1 - [j in Omega_k] / q_j:
//   Eq. 8 unary (x1024):  s = (U_i + sum_d (Wl_ij phi_kj)(y_i - y_j)) / q_i
//                             + (1024 mu)((a_ki - y_i) + 1/2)
//   Eq. 8 n-links:        Wl_ij / (q_i q_j)  (i, j in Omega_k)
// Every block objective is multiplied by M = qmax^2 (a positive constant, so
// the minimisers do not change): n-links M Wl_ij / (q_i q_j) are integers and
// the unary is rne(M s).  Eq. 10's cross term
//   [(C_k + R_k S_k)^T yhat_k]_j = [j in Omega_k] (1/q_j) sum_{i in N(j)} w_ij phi_ki yhat_kj
//                                  - phi_kj sum_{i in N(j), i in Omega_k} (w_ij / q_i) yhat_ki
// is an integer G in units of lambda / (1024 M), so
//   y_j = A_j / q_j - ((G_j / (1024 M)) / mu) / q_j,   A_j = sum_{k holding j} (yhat_kj + a_kj)
// (A summed in increasing k) and Eq. 11 is a_kl = a_kl + (yhat_kl - y_i).
// With zero growth every formula is, operation for operation, the Q = I one.
#pragma once

namespace dope {

struct OvArgs {
    Geo g;                     // box geometry: bd/bh/bw = box extent, B = box volume, K = blocks
    int D, H, W;               // grid
    int tbd, tbh, tbw;         // tile
    int gd, gh, gw;            // growth per side
    int nbz, nby, nbx;         // tiles per axis
    int M;                     // objective scale qmax^2
    long long N;
    const int32_t* U;          // [N] image order
    const int32_t* Wl;         // [conn/2][N] image order
    const uint8_t* q;          // [N] blocks holding each pixel
    double* y;                 // [N] Eq. 10 state
    double* a;                 // [K][B] Eq. 11 multipliers, box-major
    uint8_t* yhat;             // [K][B] block labels, box-major
    double* r2blk;             // [K]
    // with growth: the pixels held, together with every neighbour, by one
    // block only (their Eq. 10 cross term is 0) and all the others
    const int* inner;          // [n_inner] image indices, or null
    const int* band;           // [n_band]
    long long n_inner, n_band;
    Ctrl* ctrl;
    double eps;
    int relabel_period, max_pulses, fold_rounds;
};

// Grid coordinates of box node l of block k; false for a phantom.
__device__ __forceinline__ bool ov_node(const OvArgs& A, int k, int l, int& z, int& y, int& x) {
    const int kz = k / (A.nby * A.nbx), ky = (k / A.nbx) % A.nby, kx = k % A.nbx;
    const int lz = l / (A.g.bh * A.g.bw), ly = (l / A.g.bw) % A.g.bh, lx = l % A.g.bw;
    z = kz * A.tbd - A.gd + lz;
    y = ky * A.tbh - A.gh + ly;
    x = kx * A.tbw - A.gw + lx;
    return z >= 0 && z < A.D && y >= 0 && y < A.H && x >= 0 && x < A.W;
}

// Box-local index of grid pixel (z, y, x) in block (kz, ky, kx), or -1.
__device__ __forceinline__ int ov_local(const OvArgs& A, int kz, int ky, int kx, int z, int y, int x) {
    const int lz = z - (kz * A.tbd - A.gd), ly = y - (ky * A.tbh - A.gh), lx = x - (kx * A.tbw - A.gw);
    if (lz < 0 || lz >= A.g.bd || ly < 0 || ly >= A.g.bh || lx < 0 || lx >= A.g.bw) return -1;
    return (lz * A.g.bh + ly) * A.g.bw + lx;
}

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// 1 / q for the block counts q in {1, 2, 4, 8} (Proposition 1's q_ii with
// 2 g <= tile side), exactly: dividing by q and multiplying by this are the
// same correctly rounded operation on the same exact value, so x * inv_q(q)
// has the bits of x / q (and avoids the FP64 divide).
__device__ __forceinline__ double inv_q(int q) {
    return q == 1 ? 1.0 : (q == 2 ? 0.5 : (q == 4 ? 0.25 : (q == 8 ? 0.125 : __ddiv_rn(1.0, (double)q))));
}

// num * M / (qa * qb) for the powers of two q in {1, 2, 4, 8} and M = qmax^2
// (qa * qb divides M, so the shift is exact).
__device__ __forceinline__ int ov_frac(int num, int M, int qa, int qb) {
    return (num * M) >> ((__ffs(qa) - 1) + (__ffs(qb) - 1));
}

// Step a4 + a5 for one block of the overlapping partition: box graph in shared
// memory (same layout as solve_block), then the exact canonical cut.
template <int CONN>
__global__ void __launch_bounds__(512) k_ov_solve(OvArgs A, double mu, int t, int check_prev) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int k = blockIdx.x;
    if (check_prev) {            // the previous iteration's stop test (as k_block_solve)
        if (*(volatile int*)&A.ctrl->conv_t) return;
        const double r2 = __longlong_as_double((long long)__ldcg(&A.ctrl->r2max[t - 1]));
        if (!(__dsqrt_rn(r2) > A.eps)) {
            if (k == 0 && threadIdx.x == 0) atomicCAS(&A.ctrl->conv_t, 0, t - 1);
            return;
        }
    }
    const Geo& g = A.g;
    const int B = g.B;
    const int tid = threadIdx.x, NT = blockDim.x;
    constexpr int nh = CONN / 2;
    int* res = reinterpret_cast<int*>(smem);
    long long* C64 = reinterpret_cast<long long*>(res + CONN * B);
    int* capsum = reinterpret_cast<int*>(C64 + B);
    uint8_t* st = reinterpret_cast<uint8_t*>(capsum + B);
    const int bw = g.bw, pl = g.bh * g.bw;
    const double m1024 = __dmul_rn(1024.0, mu);
    const long long c_start = clock64();
    // zero growth: every q is 1 and M is 1 (Q = I), so in-box neighbours only
    // give their forward n-link and need neither q nor the backward weight
    const bool q1 = (A.gd | A.gh | A.gw) == 0;
    // forward n-links and unaries
#pragma unroll 1
    for (int v = tid; v < B; v += NT) {
        int z, y, x;
        const bool real = ov_node(A, k, v, z, y, x);
        const int lz = v / pl, ly = (v / bw) % g.bh, lx = v % bw;
        if (!real) {
#pragma unroll
            for (int d = 0; d < nh; ++d) res[d * B + v] = 0;
            C64[v] = 0;
            continue;
        }
        const long long i = ((long long)z * A.H + y) * A.W + x;
        const int qi = A.q[i];
        const double yi = A.y[i];
        double s = (double)A.U[i];
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            int dz, dy, dx;
            dir_off<CONN>(d, dz, dy, dx);
            const int nz = z + dz, ny = y + dy, nx = x + dx;
            const bool in_grid = nz >= 0 && nz < A.D && ny >= 0 && ny < A.H && nx >= 0 && nx < A.W;
            const int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
            const bool in_box = nlz >= 0 && nlz < g.bd && nly >= 0 && nly < g.bh && nlx >= 0 && nlx < g.bw;
            if (d < nh) res[d * B + v] = 0;
            if (!in_grid) continue;
            const long long j = ((long long)nz * A.H + ny) * A.W + nx;
            if (q1 && in_box) {
                if (d < nh) res[d * B + v] = A.Wl[(long long)d * A.N + i];
                continue;
            }
            const int w = (d < nh) ? A.Wl[(long long)d * A.N + i] : A.Wl[(long long)(d - nh) * A.N + j];
            const int qj = A.q[j];
            if (d < nh && in_box) res[d * B + v] = w * ov_frac(1, A.M, qi, qj);
            double phi = 1.0;
            if (in_box) {
                if (qj == 1) continue;
                phi = __dsub_rn(1.0, inv_q(qj));
            }
            const double wf = __dmul_rn((double)w, phi);
            const double t_ = __dmul_rn(wf, __dsub_rn(yi, A.y[j]));
            s = __dadd_rn(s, t_);
        }
        s = __dmul_rn(s, inv_q(qi));
        const double vv = __dadd_rn(__dsub_rn(A.a[(long long)k * B + v], yi), 0.5);
        s = __dadd_rn(s, __dmul_rn(m1024, vv));
        double ms = __dmul_rn((double)A.M, s);
        if (ms > 4611686018427387904.0) ms = 4611686018427387904.0;
        if (ms < -4611686018427387904.0) ms = -4611686018427387904.0;
        C64[v] = __double2ll_rn(ms);
    }
    __syncthreads();
    // backward n-links from shared memory, n-link sums
#pragma unroll 1
    for (int v = tid; v < B; v += NT) {
        const int lz = v / pl, ly = (v / bw) % g.bh, lx = v % bw;
        int cs = 0;
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            if (d < nh) {
                cs += res[d * B + v];
            } else {
                int dz, dy, dx;
                dir_off<CONN>(d, dz, dy, dx);
                const int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
                const bool in_box = nlz >= 0 && nlz < g.bd && nly >= 0 && nly < g.bh && nlx >= 0 && nlx < g.bw;
                const int w = in_box ? res[(d - nh) * B + v + dir_lofs<CONN>(d, bw, pl)] : 0;
                res[d * B + v] = w;
                cs += w;
            }
        }
        capsum[v] = cs;
        st[v] = FREE;
    }
    __syncthreads();
    cut_block<CONN, OvArgs>(A, k, smem, bw, pl, 0ull, c_start, nullptr);
}

// Tiles whose box holds coordinate c along one axis: [lo, hi] (at most two).
__device__ __forceinline__ void ov_tiles(int c, int gr, int tb, int nb, int& lo, int& hi) {
    lo = max(0, floordiv(c - gr, tb));
    hi = min(nb - 1, floordiv(c + gr, tb));
}

// Eq. 10 for pixel j.  A_j runs over the blocks holding j in increasing
// block order; the integer G_j over the blocks holding j (first term) and,
// per neighbour i, over the blocks holding i (second term).
template <int CONN>
__device__ __forceinline__ void ov_y_pixel(const OvArgs& A, double mu, long long j, double inv) {
    constexpr int nh = CONN / 2;
    const int x = (int)(j % A.W);
    const int y = (int)((j / A.W) % A.H);
    const int z = (int)(j / ((long long)A.W * A.H));
    const int qj = A.q[j];
    int kz0, kz1, ky0, ky1, kx0, kx1;
    ov_tiles(z, A.gd, A.tbd, A.nbz, kz0, kz1);
    ov_tiles(y, A.gh, A.tbh, A.nby, ky0, ky1);
    ov_tiles(x, A.gw, A.tbw, A.nbx, kx0, kx1);
    double Asum = 0.0;
    long long G = 0;
    // blocks holding j: A_j and the first term
    for (int kz = kz0; kz <= kz1; ++kz)
        for (int ky = ky0; ky <= ky1; ++ky)
            for (int kx = kx0; kx <= kx1; ++kx) {
                const long long kb = (long long)((kz * A.nby + ky) * A.nbx + kx) * A.g.B;
                const int lj = ov_local(A, kz, ky, kx, z, y, x);
                const int yj = A.yhat[kb + lj];
                Asum = __dadd_rn(Asum, __dadd_rn((double)yj, A.a[kb + lj]));
                if (!yj) continue;
#pragma unroll 4
                for (int d = 0; d < CONN; ++d) {
                    int dz, dy, dx;
                    dir_off<CONN>(d, dz, dy, dx);
                    const int iz = z + dz, iy = y + dy, ix = x + dx;
                    if (iz < 0 || iz >= A.D || iy < 0 || iy >= A.H || ix < 0 || ix >= A.W) continue;
                    const long long i = ((long long)iz * A.H + iy) * A.W + ix;
                    const long long w = (d < nh) ? A.Wl[(long long)d * A.N + j] : A.Wl[(long long)(d - nh) * A.N + i];
                    if (!w) continue;
                    const int qi = A.q[i];
                    const int li = ov_local(A, kz, ky, kx, iz, iy, ix);
                    G += w * ov_frac(qi - (li >= 0), A.M, qi, qj);
                }
            }
    // second term: per neighbour i, the blocks holding i whose label of i is 1
#pragma unroll 4
    for (int d = 0; d < CONN; ++d) {
        int dz, dy, dx;
        dir_off<CONN>(d, dz, dy, dx);
        const int iz = z + dz, iy = y + dy, ix = x + dx;
        if (iz < 0 || iz >= A.D || iy < 0 || iy >= A.H || ix < 0 || ix >= A.W) continue;
        const long long i = ((long long)iz * A.H + iy) * A.W + ix;
        const long long w = (d < nh) ? A.Wl[(long long)d * A.N + j] : A.Wl[(long long)(d - nh) * A.N + i];
        if (!w) continue;
        const int qi = A.q[i];
        int iz0, iz1, iy0, iy1, ix0, ix1;
        ov_tiles(iz, A.gd, A.tbd, A.nbz, iz0, iz1);
        ov_tiles(iy, A.gh, A.tbh, A.nby, iy0, iy1);
        ov_tiles(ix, A.gw, A.tbw, A.nbx, ix0, ix1);
        for (int kz = iz0; kz <= iz1; ++kz)
            for (int ky = iy0; ky <= iy1; ++ky)
                for (int kx = ix0; kx <= ix1; ++kx) {
                    const long long kb = (long long)((kz * A.nby + ky) * A.nbx + kx) * A.g.B;
                    if (!A.yhat[kb + ov_local(A, kz, ky, kx, iz, iy, ix)]) continue;
                    const int lj = ov_local(A, kz, ky, kx, z, y, x);
                    G -= w * ov_frac(qj - (lj >= 0), A.M, qj, qi);
                }
    }
    const double yv = __dmul_rn(Asum, inv_q(qj));
    const double gq = __dmul_rn((double)G, inv);
    const double tq = __dmul_rn(__ddiv_rn(gq, mu), inv_q(qj));
    A.y[j] = __dsub_rn(yv, tq);
}

// Eq. 10 for every pixel (one thread per pixel).
template <int CONN>
__global__ void k_ov_y(OvArgs A, double mu) {
    if (*(volatile int*)&A.ctrl->conv_t) return;
    const double inv = 1.0 / (1024.0 * (double)A.M);   // exact: a power of two
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < A.N;
         j += (long long)gridDim.x * blockDim.x)
        ov_y_pixel<CONN>(A, mu, j, inv);
}

// Eq. 10 for the pixels of A.band (the general form, warps of band pixels only).
template <int CONN>
__global__ void k_ov_y_band(OvArgs A, double mu) {
    if (*(volatile int*)&A.ctrl->conv_t) return;
    const double inv = 1.0 / (1024.0 * (double)A.M);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < A.n_band;
         t += (long long)gridDim.x * blockDim.x)
        ov_y_pixel<CONN>(A, mu, (long long)A.band[t], inv);
}

// Eq. 10 for the pixels of A.inner: held, with every neighbour, by one block
// k only, so phi_ki = 0 in the first term and [j in Omega_k] = 1 in the
// second, G_j = 0, and y_j = (yhat_kj + a_kj) / q_j - ((0 / (1024 M)) / mu) / q_j
// with the general form's operations.  (A template only so that each
// translation unit that launches it has its own instance.)
template <int CONN>
__global__ void k_ov_y_inner(OvArgs A, double mu) {
    if (*(volatile int*)&A.ctrl->conv_t) return;
    const double inv = 1.0 / (1024.0 * (double)A.M);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < A.n_inner;
         t += (long long)gridDim.x * blockDim.x) {
        const long long j = A.inner[t];
        const int x = (int)(j % A.W);
        const int y = (int)((j / A.W) % A.H);
        const int z = (int)(j / ((long long)A.W * A.H));
        int kz, ky, kx, hi;
        ov_tiles(z, A.gd, A.tbd, A.nbz, kz, hi);
        ov_tiles(y, A.gh, A.tbh, A.nby, ky, hi);
        ov_tiles(x, A.gw, A.tbw, A.nbx, kx, hi);
        const long long kb = (long long)((kz * A.nby + ky) * A.nbx + kx) * A.g.B;
        const int lj = ov_local(A, kz, ky, kx, z, y, x);
        const int qj = A.q[j];
        const double As = __dadd_rn(0.0, __dadd_rn((double)A.yhat[kb + lj], A.a[kb + lj]));
        const double yv = __dmul_rn(As, inv_q(qj));
        const double gq = __dmul_rn(0.0, inv);
        const double tq = __dmul_rn(__ddiv_rn(gq, mu), inv_q(qj));
        A.y[j] = __dsub_rn(yv, tq);
    }
}

// Eq. 10 at zero growth (Q = I, M = 1): G_j = sum over the neighbours i of j
// in other blocks of Wl_ij (yhat_j - yhat_i), the same integer the general
// form gives, and y_j = (yhat_j + a_j) - (G_j / 1024) / mu with the general
// form's operations.  Pixels farther than the kernel radius from their
// block's faces have no such neighbour and skip the neighbourhood.
template <int CONN>
__global__ void k_ov_y_q1(OvArgs A, double mu) {
    if (*(volatile int*)&A.ctrl->conv_t) return;
    constexpr int nh = CONN / 2;
    constexpr int R = kernel_radius<CONN>();
    constexpr bool three_d = CONN == 6 || CONN == 32;
    const double inv = 1.0 / 1024.0;
    const int bd = A.g.bd, bh = A.g.bh, bw = A.g.bw;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < A.N;
         j += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(j % A.W);
        const int y = (int)((j / A.W) % A.H);
        const int z = (int)(j / ((long long)A.W * A.H));
        const int kz = z / bd, ky = y / bh, kx = x / bw;
        const int lz = z - kz * bd, ly = y - ky * bh, lx = x - kx * bw;
        const long long kl = (long long)((kz * A.nby + ky) * A.nbx + kx) * A.g.B + (lz * bh + ly) * bw + lx;
        const int yj = A.yhat[kl];
        const double Asum = __dadd_rn(0.0, __dadd_rn((double)yj, A.a[kl]));
        long long G = 0;
        const bool edge = lx < R || lx >= bw - R || ly < R || ly >= bh - R || (three_d && (lz < R || lz >= bd - R));
        if (edge) {
#pragma unroll 4
            for (int d = 0; d < CONN; ++d) {
                int dz, dy, dx;
                dir_off<CONN>(d, dz, dy, dx);
                const int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
                if (nlz >= 0 && nlz < bd && nly >= 0 && nly < bh && nlx >= 0 && nlx < bw) continue;   // same block
                const int iz = z + dz, iy = y + dy, ix = x + dx;
                if (iz < 0 || iz >= A.D || iy < 0 || iy >= A.H || ix < 0 || ix >= A.W) continue;
                const long long i = ((long long)iz * A.H + iy) * A.W + ix;
                const long long w = (d < nh) ? A.Wl[(long long)d * A.N + j] : A.Wl[(long long)(d - nh) * A.N + i];
                if (!w) continue;
                const int kzi = iz / bd, kyi = iy / bh, kxi = ix / bw;
                const long long ki = (long long)((kzi * A.nby + kyi) * A.nbx + kxi) * A.g.B +
                                     ((iz - kzi * bd) * bh + (iy - kyi * bh)) * bw + (ix - kxi * bw);
                G += w * (long long)(yj - (int)A.yhat[ki]);
            }
        }
        const double yv = Asum;                                    // x / 1 = x
        const double gq = __dmul_rn((double)G, inv);
        const double tq = __ddiv_rn(gq, mu);
        A.y[j] = __dsub_rn(yv, tq);
    }
}

// Eq. 11 for every box node and the per-block stop quantity (one CTA per
// block; r2 summed in fixed chunks of 32 whatever the CTA shape).
template <int CONN>
__global__ void __launch_bounds__(256) k_ov_a(OvArgs A, int t) {
    if (*(volatile int*)&A.ctrl->conv_t) return;
    __shared__ double part[128];
    const int k = blockIdx.x;
    const int B = A.g.B;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int nchunks = (B + 31) >> 5;
    for (int ch = wid; ch < nchunks; ch += nw) {
        const int l = ch * 32 + lane;
        double d2 = 0.0;
        int z, y, x;
        if (l < B && ov_node(A, k, l, z, y, x)) {
            const long long i = ((long long)z * A.H + y) * A.W + x;
            const long long kl = (long long)k * B + l;
            const double yh = (double)A.yhat[kl];
            const double yi = A.y[i];
            A.a[kl] = __dadd_rn(A.a[kl], __dsub_rn(yh, yi));
            const double dd = __dsub_rn(yh, yi);
            d2 = __dmul_rn(dd, dd);
        }
        for (int o = 16; o > 0; o >>= 1) d2 = __dadd_rn(d2, __shfl_xor_sync(0xffffffffu, d2, o));
        if (lane == 0) part[ch] = d2;
    }
    __syncthreads();
    if (tid == 0) {
        double r2 = 0.0;
        for (int ch = 0; ch < nchunks; ++ch) r2 = __dadd_rn(r2, part[ch]);
        A.r2blk[k] = r2;
        atomicMax(&A.ctrl->r2max[t], (unsigned long long)__double_as_longlong(r2));
    }
}

#ifndef DOPE_KERNEL_TEMPLATES_ONLY
// Proposition 1 output: label 1 iff the block copies vote 1 by a strict majority.
__global__ void k_ov_labels(OvArgs A, uint8_t* labels) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < A.N;
         j += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(j % A.W);
        const int y = (int)((j / A.W) % A.H);
        const int z = (int)(j / ((long long)A.W * A.H));
        const int kz0 = max(0, floordiv(z - A.gd, A.tbd)), kz1 = min(A.nbz - 1, floordiv(z + A.gd, A.tbd));
        const int ky0 = max(0, floordiv(y - A.gh, A.tbh)), ky1 = min(A.nby - 1, floordiv(y + A.gh, A.tbh));
        const int kx0 = max(0, floordiv(x - A.gw, A.tbw)), kx1 = min(A.nbx - 1, floordiv(x + A.gw, A.tbw));
        int votes = 0;
        for (int kz = kz0; kz <= kz1; ++kz)
            for (int ky = ky0; ky <= ky1; ++ky)
                for (int kx = kx0; kx <= kx1; ++kx) {
                    const int l = ov_local(A, kz, ky, kx, z, y, x);
                    if (l >= 0) votes += A.yhat[(long long)((kz * A.nby + ky) * A.nbx + kx) * A.g.B + l];
                }
        labels[j] = (uint8_t)(2 * votes > (int)A.q[j]);
    }
}
#endif

#ifndef DOPE_KERNEL_TEMPLATES_ONLY
// Rejects n-links whose scaled capacity would break the block cut's int32
// bound: M |Wl| * max(1, conn / 8) must stay below 2^24 (so a node's n-link
// sum stays below 2^27, as for the 3x3 kernels).
__global__ void k_ov_wcheck(const int32_t* Wl, long long n, long long scale, Ctrl* c) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long w = Wl[i] < 0 ? -(long long)Wl[i] : (long long)Wl[i];
        if (w * scale >= 16777216LL) set_status(c, 4 /* DOPE_EOVERFLOW */);
    }
}
#endif

// E_int of image-order labels on image-order U / Wl (Eq. 1, each edge once).
template <int CONN>
__global__ void k_energy_img(int D, int H, int W, const int32_t* __restrict__ U, const int32_t* __restrict__ Wl,
                             const uint8_t* __restrict__ lab, Ctrl* c) {
    constexpr int nh = CONN / 2;
    const long long N = (long long)D * H * W;
    long long acc = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % W), y = (int)((i / W) % H), z = (int)(i / ((long long)W * H));
        const int yi = lab[i];
        acc += (long long)U[i] * yi;
#pragma unroll
        for (int d = 0; d < nh; ++d) {
            int dz, dy, dx;
            dir_off<CONN>(d, dz, dy, dx);
            const int nz = z + dz, ny = y + dy, nx = x + dx;
            if (nz < 0 || nz >= D || ny < 0 || ny >= H || nx < 0 || nx >= W) continue;
            const long long j = ((long long)nz * H + ny) * W + nx;
            if (yi != lab[j]) acc += Wl[(long long)d * N + i];
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&c->energy, (unsigned long long)acc);
}

}  // namespace dope
