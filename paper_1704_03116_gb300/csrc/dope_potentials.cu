// dope_potentials.cu -- whole-image potentials on the device: the Gaussian
// mixture data term and the contrast-sensitive Potts weights that Algorithm 1
// computes before its loop (its first step; Section 4 reports that this step
// costs the same for every partition and weighs heavily in the run times).
//
//   u_i   = clip(log p_bg(x_i) - log p_fg(x_i)),  p = sum_j pi_j N(m_j, S_j)
//   wq_ij = rne(1024 exp(-|x_i - x_j|^2 / (2 sigma^2)) [/ |p_i - p_j|])
//
// Both are elementwise over the image: 12 B read per RGB pixel, 4 B written
// for u and 4 B per forward offset for wq; at these sizes the kernels are
// bound by instruction issue as much as by HBM.  The mixture constants are
// formed once on the host in FP64 (Cholesky factor L of each S_j, its
// inverse, log-determinant and log-weight, all in log2 units) and passed by
// value; the device evaluates each component as c_j - |L'_j (x - m_j)|^2 in
// FP32 and combines them with the hardware base-2 exponential and logarithm.
// The weights take their rounding decision in FP32 with one correctly
// rounded operation at a time (no contraction), in the order the header
// lists, so that only the exponential differs from an FP32 restatement.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "dope_internal.h"
#include "dope_potentials.h"

namespace {

#define PCK(x)                                          \
    do {                                                \
        if ((x) != cudaSuccess) {                       \
            cudaGetLastError();                         \
            return DOPE_ECUDA;                          \
        }                                               \
    } while (0)

constexpr int MAXC = DOPE_GMM_MAX_COMP;
constexpr int MAXF = DOPE_GMM_MAX_CH;
constexpr int MAXOFF = 40;   // forward offsets of the 9x9 square

// One mixture, ready for the device: component j's log2-density is
//   c[j] - sum_r ( sum_{c <= r} Li[j][r(r+1)/2 + c] (x_c - mean[j][c]) )^2
// (the inverse Cholesky factor scaled by sqrt(log2(e) / 2), the constant in
// log2 units).
struct GmmDev {
    int K;
    float mean[MAXC][MAXF];
    float Li[MAXC][MAXF * (MAXF + 1) / 2];
    float c[MAXC];
};

struct GmmPair {
    GmmDev fg, bg;
};

// Host: validate one model and form its device constants in FP64.
int gmm_prepare(const dope_gmm* g, int C, GmmDev* out) {
    if (!g || g->n_comp < 1 || g->n_comp > MAXC || g->channels != C) return DOPE_EINVAL;
    memset(out, 0, sizeof(*out));
    out->K = g->n_comp;
    for (int j = g->n_comp; j < MAXC; ++j) out->c[j] = -INFINITY;   // padding: exp(-inf) = 0
    for (int j = 0; j < g->n_comp; ++j) {
        const double w = g->weight[j];
        if (!(w > 0.0) || !isfinite(w)) return DOPE_EINVAL;
        double L[MAXF][MAXF] = {};
        for (int r = 0; r < C; ++r) {
            for (int c = 0; c <= r; ++c) {
                double s = g->cov[j][r][c];
                if (!isfinite(s)) return DOPE_EINVAL;
                for (int k = 0; k < c; ++k) s -= L[r][k] * L[c][k];
                if (r == c) {
                    if (!(s > 0.0)) return DOPE_EINVAL;   // not positive definite
                    L[r][r] = sqrt(s);
                } else {
                    L[r][c] = s / L[c][c];
                }
            }
        }
        // inverse of the lower-triangular factor, column by column
        double Li[MAXF][MAXF] = {};
        for (int c = 0; c < C; ++c) {
            Li[c][c] = 1.0 / L[c][c];
            for (int r = c + 1; r < C; ++r) {
                double s = 0.0;
                for (int k = c; k < r; ++k) s += L[r][k] * Li[k][c];
                Li[r][c] = -s / L[r][r];
            }
        }
        // log2 units: log2 N_j(x) = c[j] - |Li'_j (x - m_j)|^2 with
        // Li' = Li sqrt(log2(e) / 2) and c[j] = log2(e) (log w_j - log det L_j - C/2 log 2 pi)
        const double log2e = 1.4426950408889634, sc = sqrt(0.5 * log2e);
        double half_logdet = 0.0;
        for (int r = 0; r < C; ++r) half_logdet += log(L[r][r]);
        out->c[j] = (float)(log2e * (log(w) - half_logdet - 0.5 * C * log(2.0 * M_PI)));
        for (int r = 0; r < C; ++r) {
            const double m = g->mean[j][r];
            if (!isfinite(m)) return DOPE_EINVAL;
            out->mean[j][r] = (float)m;
            for (int c = 0; c <= r; ++c) out->Li[j][r * (r + 1) / 2 + c] = (float)(Li[r][c] * sc);
        }
    }
    return DOPE_OK;
}

// Hardware base-2 exponential and logarithm (MUFU; relative error of
// ex2 and absolute error of lg2 near 2^-22 on the ranges used here).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// log2 sum_j 2^(l_j) over K components (l_j the log2-densities): the largest
// term as the shift, then one ex2 per component.  K is a template constant
// (the larger of the two models' counts; the smaller model's extra
// components have c = -inf and add exactly 0), so every constant is an
// immediate operand of the parameter bank.
template <int C, int K>
__device__ __forceinline__ float mixture_ll2(const GmmDev& g, const float* x) {
    float nl[K];   // -l_j
    float lo = INFINITY;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        float d[C];
#pragma unroll
        for (int c = 0; c < C; ++c) d[c] = x[c] - g.mean[j][c];
        float q = -g.c[j];
#pragma unroll
        for (int r = 0; r < C; ++r) {
            float z = 0.f;
#pragma unroll
            for (int c = 0; c <= r; ++c) z = fmaf(g.Li[j][r * (r + 1) / 2 + c], d[c], z);
            q = fmaf(z, z, q);
        }
        nl[j] = q;
        lo = fminf(lo, q);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < K; ++j) s += ex2_approx(lo - nl[j]);
    return lg2_approx(s) - lo;
}

constexpr int GMM_TILE = 256;   // pixels per CTA tile (one per thread)

// Each CTA stages a tile of GMM_TILE pixels (GMM_TILE * C consecutive floats)
// through shared memory with coalesced loads, then evaluates one pixel per
// thread; grid-stride over tiles.  Plain (L2-allocating) loads and stores:
// the image is read again by the contrast kernels and u by the quantiser.
template <int C, int K>
__global__ void __launch_bounds__(GMM_TILE) k_gmm_unaries(const float* __restrict__ img, long long n, GmmPair P,
                                                           float clip, float* __restrict__ u) {
    __shared__ float tile[GMM_TILE * C];
    const long long ntiles = (n + GMM_TILE - 1) / GMM_TILE;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long p0 = t * GMM_TILE;
        const int cnt = (int)min((long long)GMM_TILE, n - p0);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt * C; e += GMM_TILE) tile[e] = img[p0 * C + e];
        __syncthreads();
        if (threadIdx.x < cnt) {
            float x[C];
#pragma unroll
            for (int c = 0; c < C; ++c) x[c] = tile[threadIdx.x * C + c];
            float v = 0.6931471805599453f * (mixture_ll2<C, K>(P.bg, x) - mixture_ll2<C, K>(P.fg, x));
            v = v < -clip ? -clip : (v > clip ? clip : v);   // NaN stays NaN
            u[p0 + threadIdx.x] = v;
        }
    }
}

template <int C, int K>
void launch_gmm(int blocks, const float* img, long long n, const GmmPair& P, float clip, float* u, cudaStream_t st) {
    k_gmm_unaries<C, K><<<blocks, GMM_TILE, 0, st>>>(img, n, P, clip, u);
}

template <int C>
void launch_gmm_k(int K, int blocks, const float* img, long long n, const GmmPair& P, float clip, float* u,
                  cudaStream_t st) {
    switch (K) {
        case 1: launch_gmm<C, 1>(blocks, img, n, P, clip, u, st); break;
        case 2: launch_gmm<C, 2>(blocks, img, n, P, clip, u, st); break;
        case 3: launch_gmm<C, 3>(blocks, img, n, P, clip, u, st); break;
        case 4: launch_gmm<C, 4>(blocks, img, n, P, clip, u, st); break;
        case 5: launch_gmm<C, 5>(blocks, img, n, P, clip, u, st); break;
        case 6: launch_gmm<C, 6>(blocks, img, n, P, clip, u, st); break;
        case 7: launch_gmm<C, 7>(blocks, img, n, P, clip, u, st); break;
        default: launch_gmm<C, 8>(blocks, img, n, P, clip, u, st); break;
    }
}

// Grid and neighbourhood of the contrast kernels.
struct ContrastGeo {
    int D, H, W, C, nh;
    long long N;
    signed char off[MAXOFF][3];   // (dz, dy, dx)
    float invdist[MAXOFF];        // fp32(1 / |offset|) or 1
};

// Forward offsets of a connectivity, in the order of the weight layout.
int fwd_offsets(int ndim, int conn, signed char (*off)[3]) {
    static const signed char o4[2][3] = {{0, 0, 1}, {0, 1, 0}};
    static const signed char o8[4][3] = {{0, 0, 1}, {0, 1, 0}, {0, 1, 1}, {0, 1, -1}};
    static const signed char o6[3][3] = {{0, 0, 1}, {0, 1, 0}, {1, 0, 0}};
    if (ndim == 2 && conn == 4) { memcpy(off, o4, sizeof(o4)); return 2; }
    if (ndim == 2 && conn == 8) { memcpy(off, o8, sizeof(o8)); return 4; }
    if (ndim == 3 && conn == 6) { memcpy(off, o6, sizeof(o6)); return 3; }
    int r = 0;
    bool ball = false;
    if (ndim == 2 && (conn == 24 || conn == 48 || conn == 80)) r = conn == 24 ? 2 : (conn == 48 ? 3 : 4);
    else if (ndim == 3 && conn == 32) { r = 2; ball = true; }
    else return 0;
    int n = 0;
    for (int dz = 0; dz <= (ball ? r : 0); ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx) {
                const bool positive = dz > 0 || (dz == 0 && (dy > 0 || (dy == 0 && dx > 0)));
                if (!positive || (ball && dz * dz + dy * dy + dx * dx > r * r)) continue;
                off[n][0] = (signed char)dz;
                off[n][1] = (signed char)dy;
                off[n][2] = (signed char)dx;
                ++n;
            }
    return n == conn / 2 ? n : 0;
}

// |x_i - x_j|^2 in FP32: squares in channel order, summed left to right,
// every operation rounded on its own.
template <int C>
__device__ __forceinline__ float contrast_d2(const float* xi, const float* __restrict__ xj) {
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float d = __fsub_rn(xi[c], __ldg(&xj[c]));
        s = c == 0 ? __fmul_rn(d, d) : __fadd_rn(s, __fmul_rn(d, d));
    }
    return s;
}

// Pixel traversal of the contrast kernels: a CTA of (bx, by) threads covers
// bx consecutive pixels of by consecutive rows; blockIdx.x picks the column
// segment and blockIdx.y strides over the D * ceil(H / by) row groups, so no
// per-pixel division is needed and the grid stays a few CTAs per SM.
template <typename Fn>
__device__ __forceinline__ void for_each_pixel(const ContrastGeo& G, int hb, Fn&& fn) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const long long groups = (long long)G.D * hb;
    for (long long r = blockIdx.y; r < groups; r += gridDim.y) {
        const int z = (int)(r / hb), y = (int)(r % hb) * blockDim.y + threadIdx.y;
        if (x < G.W && y < G.H) fn(z, y, x, ((long long)z * G.H + y) * G.W + x);
    }
}

// Offsets of the contrast kernels: compile-time for connectivity 4, 8 and 6
// (the weight layout's order), from the geometry's table otherwise (CONN 0).
template <int CONN>
__device__ __forceinline__ void pair_off(const ContrastGeo& G, int d, int& dz, int& dy, int& dx) {
    if constexpr (CONN == 4) {
        dz = 0; dy = d; dx = 1 - d;
    } else if constexpr (CONN == 8) {
        dz = 0; dy = d >= 1; dx = d == 0 ? 1 : (d == 1 ? 0 : (d == 2 ? 1 : -1));
    } else if constexpr (CONN == 6) {
        dz = d == 2; dy = d == 1; dx = d == 0;
    } else {
        dz = G.off[d][0]; dy = G.off[d][1]; dx = G.off[d][2];
    }
}

template <int CONN>
__host__ __device__ constexpr int pair_count() { return CONN == 4 ? 2 : (CONN == 8 ? 4 : (CONN == 6 ? 3 : 0)); }

// Visit every forward pair (d, neighbour features) of pixel (z, y, x) in
// offset order; fn(d, xj) gets xj = nullptr where the partner is outside the
// grid.  For the radius-1 neighbourhoods an interior pixel skips the bounds
// checks and finds its partners at fixed index offsets.
template <int C, int CONN, typename Fn>
__device__ __forceinline__ void for_each_pair(const ContrastGeo& G, const float* __restrict__ img, int z, int y,
                                              int x, long long i, Fn&& fn) {
    if constexpr (CONN != 0) {
        constexpr int NH = pair_count<CONN>();
        const bool interior = x >= 1 && x + 1 < G.W && y + 1 < G.H && (CONN != 6 || z + 1 < G.D);
        if (interior) {
#pragma unroll
            for (int d = 0; d < NH; ++d) {
                int dz, dy, dx;
                pair_off<CONN>(G, d, dz, dy, dx);
                const long long o = ((long long)dz * G.H + dy) * G.W + dx;
                fn(d, img + (i + o) * C);
            }
            return;
        }
#pragma unroll
        for (int d = 0; d < NH; ++d) {
            int dz, dy, dx;
            pair_off<CONN>(G, d, dz, dy, dx);
            const int zz = z + dz, yy = y + dy, xx = x + dx;
            const bool in = zz < G.D && yy < G.H && xx >= 0 && xx < G.W;
            fn(d, in ? img + (((long long)zz * G.H + yy) * G.W + xx) * C : nullptr);
        }
    } else {
        for (int d = 0; d < G.nh; ++d) {
            int dz, dy, dx;
            pair_off<0>(G, d, dz, dy, dx);
            const int zz = z + dz, yy = y + dy, xx = x + dx;
            const bool in = zz < G.D && yy >= 0 && yy < G.H && xx >= 0 && xx < G.W;
            fn(d, in ? img + (((long long)zz * G.H + yy) * G.W + xx) * C : nullptr);
        }
    }
}

// Sum over every neighbour pair of |x_i - x_j|: per pixel in FP32 (offset
// order), over pixels in FP64; one double atomic per CTA into acc.
template <int C, int CONN>
__global__ void __launch_bounds__(256) k_contrast_sum(const float* __restrict__ img, const __grid_constant__ ContrastGeo G,
                                                      int hb, double* __restrict__ acc) {
    __shared__ double red[8];
    double part = 0.0;
    for_each_pixel(G, hb, [&](int z, int y, int x, long long i) {
        float xi[C];
#pragma unroll
        for (int c = 0; c < C; ++c) xi[c] = __ldg(&img[i * C + c]);
        float s = 0.f;
        for_each_pair<C, CONN>(G, img, z, y, x, i, [&](int, const float* xj) {
            if (xj) s = __fadd_rn(s, __fsqrt_rn(contrast_d2<C>(xi, xj)));
        });
        part += (double)s;
    });
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const int t = threadIdx.y * blockDim.x + threadIdx.x, nw = (blockDim.x * blockDim.y) >> 5;
    if ((t & 31) == 0) red[t >> 5] = part;
    __syncthreads();
    if (t == 0) {
        double tot = 0.0;
        for (int w = 0; w < nw; ++w) tot += red[w];
        if (tot != 0.0) atomicAdd(acc, tot);
    }
}

// wq[d][i] for every pixel and forward offset.  sigma_given > 0 is used as
// is; otherwise sigma = max(acc[0] / pairs, 1e-6).  Thread 0 of CTA 0 stores
// the sigma used in acc[1].
template <int C, int CONN>
__global__ void __launch_bounds__(256) k_contrast_weights(const float* __restrict__ img, const __grid_constant__ ContrastGeo G,
                                                          int hb, double sigma_given, double pairs,
                                                          double* __restrict__ acc, int32_t* __restrict__ wq) {
    double sigma = sigma_given;
    if (!(sigma > 0.0)) {
        sigma = pairs > 0.0 ? __ddiv_rn(acc[0], pairs) : 0.0;
        if (!(sigma >= 1e-6)) sigma = 1e-6;
    }
    const float k = __double2float_rn(__ddiv_rn(1.0, __dmul_rn(__dmul_rn(2.0, sigma), sigma)));
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0 && acc) acc[1] = sigma;
    for_each_pixel(G, hb, [&](int z, int y, int x, long long i) {
        float xi[C];
#pragma unroll
        for (int c = 0; c < C; ++c) xi[c] = __ldg(&img[i * C + c]);
        for_each_pair<C, CONN>(G, img, z, y, x, i, [&](int d, const float* xj) {
            int32_t q = 0;
            if (xj) {
                const float a = __fmul_rn(contrast_d2<C>(xi, xj), k);
                float e = expf(-a);
                e = __fmul_rn(e, G.invdist[d]);
                q = __float2int_rn(__fmul_rn(1024.f, e));
            }
            wq[(long long)d * G.N + i] = q;
        });
    });
}

template <int C, int CONN>
void launch_contrast(bool sum, dim3 grid, dim3 block, const float* img, const ContrastGeo& G, int hb, double sigma,
                     double pairs, double* ws, int32_t* wq, cudaStream_t st) {
    if (sum) k_contrast_sum<C, CONN><<<grid, block, 0, st>>>(img, G, hb, ws);
    else k_contrast_weights<C, CONN><<<grid, block, 0, st>>>(img, G, hb, sigma, pairs, ws, wq);
}

template <int C>
void launch_contrast_c(int conn, bool sum, dim3 grid, dim3 block, const float* img, const ContrastGeo& G, int hb,
                       double sigma, double pairs, double* ws, int32_t* wq, cudaStream_t st) {
    if (conn == 4) launch_contrast<C, 4>(sum, grid, block, img, G, hb, sigma, pairs, ws, wq, st);
    else if (conn == 8) launch_contrast<C, 8>(sum, grid, block, img, G, hb, sigma, pairs, ws, wq, st);
    else if (conn == 6) launch_contrast<C, 6>(sum, grid, block, img, G, hb, sigma, pairs, ws, wq, st);
    else launch_contrast<C, 0>(sum, grid, block, img, G, hb, sigma, pairs, ws, wq, st);
}

void launch_contrast_any(int C, int conn, bool sum, dim3 grid, dim3 block, const float* img, const ContrastGeo& G,
                         int hb, double sigma, double pairs, double* ws, int32_t* wq, cudaStream_t st) {
    switch (C) {
        case 1: launch_contrast_c<1>(conn, sum, grid, block, img, G, hb, sigma, pairs, ws, wq, st); break;
        case 2: launch_contrast_c<2>(conn, sum, grid, block, img, G, hb, sigma, pairs, ws, wq, st); break;
        case 3: launch_contrast_c<3>(conn, sum, grid, block, img, G, hb, sigma, pairs, ws, wq, st); break;
        default: launch_contrast_c<4>(conn, sum, grid, block, img, G, hb, sigma, pairs, ws, wq, st); break;
    }
}

// A few CTAs per SM for the grid-stride kernels: the SM count of the device
// current at the call (the kernels stride, so any grid is correct; a failed
// query only makes the grid small).
int grid_cap() { return dope_sm_count() * 8; }

int blocks_for(long long n, int per_block) {
    const long long b = (n + per_block - 1) / per_block;
    const int cap = grid_cap();
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

int pot_unaries_issue(const float* img, long long n, int C, const dope_gmm* fg, const dope_gmm* bg, double clip,
                      float* u, cudaStream_t st) {
    if (n < 0 || C < 1 || C > MAXF || !(clip > 0.0) || (n > 0 && (!img || !u))) return DOPE_EINVAL;
    GmmPair P;
    int rc = gmm_prepare(fg, C, &P.fg);
    if (!rc) rc = gmm_prepare(bg, C, &P.bg);
    if (rc) return rc;
    if (n == 0) return DOPE_OK;
    const float cl = clip > 3.0e38 ? 3.0e38f : (float)clip;
    const int blocks = blocks_for(n, GMM_TILE);
    const int K = P.fg.K > P.bg.K ? P.fg.K : P.bg.K;
    switch (C) {
        case 1: launch_gmm_k<1>(K, blocks, img, n, P, cl, u, st); break;
        case 2: launch_gmm_k<2>(K, blocks, img, n, P, cl, u, st); break;
        case 3: launch_gmm_k<3>(K, blocks, img, n, P, cl, u, st); break;
        default: launch_gmm_k<4>(K, blocks, img, n, P, cl, u, st); break;
    }
    PCK(cudaGetLastError());
    return DOPE_OK;
}

int pot_weights_issue(const float* img, const int64_t dims[3], int ndim, int C, int conn, double sigma,
                      int inv_dist, int32_t* wq, double* ws, cudaStream_t st) {
    if (C < 1 || C > MAXF || !dims || (ndim != 2 && ndim != 3)) return DOPE_EINVAL;
    ContrastGeo G;
    memset(&G, 0, sizeof(G));
    G.nh = fwd_offsets(ndim, conn, G.off);
    if (!G.nh) return DOPE_EINVAL;
    long long N = 1;
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || dims[a] > (1 << 30)) return DOPE_EINVAL;
        N *= dims[a];                       // < 2^31 * 2^30 at every step
        if (N >= (1LL << 31)) return DOPE_EINVAL;
    }
    if (ndim == 2 && dims[0] != 1) return DOPE_EINVAL;
    if (!img || !wq || (!(sigma > 0.0) && !ws) || !isfinite(sigma)) return DOPE_EINVAL;
    G.D = (int)dims[0];
    G.H = (int)dims[1];
    G.W = (int)dims[2];
    G.C = C;
    G.N = N;
    double pairs = 0.0;
    for (int d = 0; d < G.nh; ++d) {
        const int dz = G.off[d][0], dy = G.off[d][1], dx = G.off[d][2];
        G.invdist[d] = inv_dist ? (float)(1.0 / sqrt((double)(dz * dz + dy * dy + dx * dx))) : 1.0f;
        const long long ez = G.D - (dz < 0 ? -dz : dz), ey = G.H - (dy < 0 ? -dy : dy), ex = G.W - (dx < 0 ? -dx : dx);
        if (ez > 0 && ey > 0 && ex > 0) pairs += (double)(ez * ey * ex);
    }
    // CTA shape: bx = the power of two in [32, 256] that covers a row (or
    // 256), by = 256 / bx rows; grid.x column segments, grid.y row groups
    int bx = 32;
    while (bx < 256 && bx < G.W) bx <<= 1;
    const int by = 256 / bx;
    const int hb = (G.H + by - 1) / by;
    const long long gx = (G.W + bx - 1) / bx, groups = (long long)G.D * hb;
    if (gx > 0x7fffffffLL) return DOPE_EINVAL;
    const long long want = grid_cap() / gx > 0 ? grid_cap() / gx : 1;
    const dim3 grid((unsigned)gx, (unsigned)(groups < want ? groups : (want < 65535 ? want : 65535)));
    const dim3 block(bx, by);
    if (!(sigma > 0.0)) {
        PCK(cudaMemsetAsync(ws, 0, 2 * sizeof(double), st));
        launch_contrast_any(C, conn, true, grid, block, img, G, hb, sigma, pairs, ws, wq, st);
        PCK(cudaGetLastError());
    }
    launch_contrast_any(C, conn, false, grid, block, img, G, hb, sigma, pairs, ws, wq, st);
    PCK(cudaGetLastError());
    return DOPE_OK;
}

extern "C" int dope_gmm_unaries(const float* image_dev, int64_t n, int channels, const dope_gmm* fg,
                                const dope_gmm* bg, double clip, float* u_dev, void* stream) {
    return pot_unaries_issue(image_dev, (long long)n, channels, fg, bg, clip, u_dev, (cudaStream_t)stream);
}

extern "C" int dope_contrast_weights(const float* image_dev, const int64_t* grid, int ndim, int channels,
                                     int connectivity, double sigma, int inv_dist, int32_t* wq_dev,
                                     void* workspace_dev, double* sigma_used, void* stream) {
    if (!grid || (ndim != 2 && ndim != 3)) return DOPE_EINVAL;
    if (workspace_dev && ((uintptr_t)workspace_dev & 7)) return DOPE_EINVAL;
    const int64_t dims[3] = {ndim == 3 ? grid[0] : 1, grid[ndim - 2], grid[ndim - 1]};
    cudaStream_t st = (cudaStream_t)stream;
    double* ws = (double*)workspace_dev;
    const bool given = sigma > 0.0;
    // with a given sigma and no workspace, the kernel has nowhere to record it
    int rc = pot_weights_issue(image_dev, dims, ndim, channels, connectivity, sigma, inv_dist, wq_dev,
                               given ? nullptr : ws, st);
    if (rc) return rc;
    if (sigma_used) {
        if (given) {
            *sigma_used = sigma;
        } else {
            PCK(cudaMemcpyAsync(sigma_used, ws + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
            PCK(cudaStreamSynchronize(st));
        }
    }
    return DOPE_OK;
}
