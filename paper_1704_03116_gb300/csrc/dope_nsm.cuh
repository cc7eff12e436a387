// dope_nsm.cuh -- non-submodular blocks: every block's Eq. 8 (Q = I) solved
// by LSA-TR, the trust-region local submodular approximation the paper
// distributes in its curvature experiment.  Included by dope.cu after
// dope_kernels.cuh; reuses its exact block cut (cut_block) for every step.
//
// Block objective, weights of any sign:
//   E(x) = sum_i C_i x_i + sum_{edges ij in the block} Wl_ij |x_i - x_j|.
// An edge with Wl_ij = -w < 0 equals -w x_i - w x_j + 2 w x_i x_j; the product
// is replaced by its tangent at the current labelling x^s,
// x_i^s x_j + x_j^s x_i - x_i^s x_j^s, so the approximation is submodular and
// exact at x^s.  A step minimises approximation + lam * |x - x^s|_1 exactly
// (canonical minimal cut) and keeps the minimiser x* iff E(x*) < E(x^s).
// Trust region (integers): lam starts at 1024; x* = x^s: lam /= 4 (stop at
// lam = 0); accepted with actual decrease R >= 3/4 of the predicted P:
// lam /= 4; rejected: lam = max(4 lam, 1) (capped at 2^50).  At most `steps`
// steps per block and ADMM iteration, starting from the block's labels of the
// previous iteration (0 at iteration 1).
#pragma once

namespace dope {

constexpr long long LSA_LAM0 = 1024;

// Sum of one int64 per thread over the CTA; every thread gets the total.
__device__ __forceinline__ long long block_sum_ll(long long v, long long* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    long long t = 0;
    for (int w = 0; w < nw; ++w) t += red[w];
    __syncthreads();
    return t;
}

// Bytes of shared memory k_nsm_solve needs beyond the block solver's.
__host__ __device__ inline size_t nsm_extra_bytes(int B) { return ((18 * (size_t)B + 7) & ~(size_t)7) + 8 * 32; }

template <int CONN>
__global__ void __launch_bounds__(512) k_nsm_solve(SolveArgs A, int steps) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_skip;
    const int k = blockIdx.x;
    const int tid = threadIdx.x, NT = blockDim.x;
    if (tid == 0) {
        int skip = 0;
        if (A.check_prev) {
            if (*(volatile int*)&A.ctrl->conv_t) {
                skip = 1;
            } else {
                const double r2 = __longlong_as_double((long long)__ldcg(&A.ctrl->r2max[A.t - 1]));
                if (!(__dsqrt_rn(r2) > A.eps)) {
                    skip = 1;
                    if (k == 0) atomicCAS(&A.ctrl->conv_t, 0, A.t - 1);
                }
            }
        }
        s_skip = skip;
    }
    __syncthreads();
    if (s_skip) return;
    const Geo& g = A.g;
    const int B = g.B;
    constexpr int nh = CONN / 2;
    int* res = reinterpret_cast<int*>(smem);
    long long* C64 = reinterpret_cast<long long*>(res + CONN * B);
    int* capsum = reinterpret_cast<int*>(C64 + B);
    uint8_t* st = reinterpret_cast<uint8_t*>(capsum + B);
    unsigned char* ext = smem + ((solver_smem_bytes(CONN, B) + 15) & ~(size_t)15);
    long long* Cb = reinterpret_cast<long long*>(ext);          // exact Eq. 8 unaries
    long long* un = Cb + B;                                     // approximation's unaries
    uint8_t* x = reinterpret_cast<uint8_t*>(un + B);            // current labels
    uint8_t* xs = x + B;                                        // step minimiser
    long long* red = reinterpret_cast<long long*>(ext + ((18 * (size_t)B + 7) & ~(size_t)7));
    const int kz = k / (g.nby * g.nbx), ky = (k / g.nbx) % g.nby, kx = k % g.nbx;
    const int bw = g.bw, pl = g.bh * g.bw;
    const double m1024 = __dmul_rn(1024.0, A.mu);
    // exact unaries of every node, start labels
    for (int v = tid; v < B; v += NT) {
        const int lx = v % bw, ly = (v / bw) % g.bh, lz = v / pl;
        const int f = A.faceIndex[v];
        long long c;
        if (A.first) c = (long long)A.U[(long long)k * B + v];
        else if (f >= 0) c = face_cap<CONN>(g, A.U, A.Wl, A.yF, A.aF, A.halo, k, kz, ky, kx, v, f, m1024);
        else c = shifted_cap<CONN>(g, A.U, A.Wl, A.yhat, A.yF, A.aF, A.faceIndex, k, kz, ky, kx, v, lz, ly, lx, 0, m1024);
        Cb[v] = c;
        x[v] = A.first ? 0 : A.yhat[(long long)k * B + v];
    }
    __syncthreads();
    // E(x) over the block's own edges (each once, along the forward directions)
    auto energy = [&](const uint8_t* lab) -> long long {
        long long e = 0;
        for (int v = tid; v < B; v += NT) {
            const int lx = v % bw, ly = (v / bw) % g.bh, lz = v / pl;
            if (lab[v]) e += Cb[v];
#pragma unroll
            for (int d = 0; d < nh; ++d) {
                int dz, dy, dx;
                dir_off<CONN>(d, dz, dy, dx);
                const int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
                if (nlz >= g.bd || nly >= g.bh || nlx < 0 || nlx >= bw) continue;
                const int u = v + dir_lofs<CONN>(d, bw, pl);
                if (lab[v] != lab[u]) e += A.Wl[(long long)d * g.N + (long long)k * B + v];
            }
        }
        return block_sum_ll(e, red);
    };
    long long e_cur = energy(x);
    long long lam = LSA_LAM0;
    for (int s = 0; s < steps; ++s) {
        // approximation around x: submodular n-links, unaries, constant
        long long cst = 0;
        for (int v = tid; v < B; v += NT) un[v] = Cb[v];
        __syncthreads();
        for (int v = tid; v < B; v += NT) {
            const int lx = v % bw, ly = (v / bw) % g.bh, lz = v / pl;
#pragma unroll
            for (int d = 0; d < nh; ++d) {
                int dz, dy, dx;
                dir_off<CONN>(d, dz, dy, dx);
                const int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
                int r = 0;
                if (nlz < g.bd && nly < g.bh && nlx >= 0 && nlx < bw) {
                    const int u = v + dir_lofs<CONN>(d, bw, pl);
                    const int w = A.Wl[(long long)d * g.N + (long long)k * B + v];
                    if (w > 0) {
                        r = w;
                    } else if (w < 0) {
                        const long long m = -(long long)w;
                        atomicAdd(reinterpret_cast<unsigned long long*>(&un[v]), (unsigned long long)(-m + 2 * m * x[u]));
                        atomicAdd(reinterpret_cast<unsigned long long*>(&un[u]), (unsigned long long)(-m + 2 * m * x[v]));
                        cst -= 2 * m * x[v] * x[u];
                    }
                }
                res[d * B + v] = r;
            }
        }
        cst = block_sum_ll(cst, red);
        for (int v = tid; v < B; v += NT) {
            const int lx = v % bw, ly = (v / bw) % g.bh, lz = v / pl;
            int cs = 0;
#pragma unroll
            for (int d = 0; d < CONN; ++d) {
                if (d < nh) {
                    cs += res[d * B + v];
                } else {
                    int dz, dy, dx;
                    dir_off<CONN>(d, dz, dy, dx);
                    const int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
                    const bool in = nlz >= 0 && nlz < g.bd && nly >= 0 && nly < g.bh && nlx >= 0 && nlx < bw;
                    const int w = in ? res[(d - nh) * B + v + dir_lofs<CONN>(d, bw, pl)] : 0;
                    res[d * B + v] = w;
                    cs += w;
                }
            }
            capsum[v] = cs;
            st[v] = FREE;
            C64[v] = un[v] + lam * (1 - 2 * (long long)x[v]);
        }
        __syncthreads();
        cut_block<CONN>(A, k, smem, bw, pl, 0ull, clock64(), xs, false);
        __syncthreads();
        int diff = 0;
        for (int v = tid; v < B; v += NT) diff |= (xs[v] != x[v]);
        if (!__syncthreads_or(diff)) {
            if (lam == 0) break;
            lam /= 4;
            continue;
        }
        // predicted value of the approximation at x* (it equals E at x)
        long long ap = 0;
        for (int v = tid; v < B; v += NT) {
            const int lx = v % bw, ly = (v / bw) % g.bh, lz = v / pl;
            if (xs[v]) ap += un[v];
#pragma unroll
            for (int d = 0; d < nh; ++d) {
                int dz, dy, dx;
                dir_off<CONN>(d, dz, dy, dx);
                const int nlz = lz + dz, nly = ly + dy, nlx = lx + dx;
                if (nlz >= g.bd || nly >= g.bh || nlx < 0 || nlx >= bw) continue;
                const int u = v + dir_lofs<CONN>(d, bw, pl);
                const int w = A.Wl[(long long)d * g.N + (long long)k * B + v];
                if (w > 0 && xs[v] != xs[u]) ap += w;
            }
        }
        ap = cst + block_sum_ll(ap, red);
        const long long e_new = energy(xs);
        const long long R = e_cur - e_new, P = e_cur - ap;
        if (R > 0) {
            for (int v = tid; v < B; v += NT) x[v] = xs[v];
            e_cur = e_new;
            if (4 * R >= 3 * P) lam /= 4;
        } else {
            lam = lam * 4 > 0 ? lam * 4 : 1;
            if (lam > (1LL << 50)) lam = 1LL << 50;
        }
        __syncthreads();
    }
    for (int v = tid; v < B; v += NT) A.yhat[(long long)k * B + v] = x[v];
}

}  // namespace dope
