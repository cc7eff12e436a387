// dope_potentials.cu -- whole-image potentials on the device: the Gaussian
// mixture data term and the contrast-sensitive Potts weights that Algorithm 1
// computes before its loop (its first step; Section 4 reports that this step
// costs the same for every partition and weighs heavily in the run times).
//
//   u_i   = clip(log p_bg(x_i) - log p_fg(x_i)),  p = sum_j pi_j N(m_j, S_j)
//   wq_ij = rne(1024 exp(-|x_i - x_j|^2 / (2 sigma^2)) [/ |p_i - p_j|])
//
// Both are elementwise over the image and bound by HBM traffic (12 B read per
// RGB pixel; 4 B written for u, 4 B per forward offset for wq).  The mixture
// constants are formed once on the host in FP64 (Cholesky factor L of each
// S_j, its inverse, log-determinant and log-weight) and passed by value; the
// device evaluates each component as c_j - |L_j^-1 (x - m_j)|^2 / 2 in FP32.
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

// One mixture, ready for the device: component j's log-density is
//   c[j] - 0.5 * sum_r ( sum_{c <= r} Li[j][r(r+1)/2 + c] (x_c - mean[j][c]) )^2
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
        double half_logdet = 0.0;
        for (int r = 0; r < C; ++r) half_logdet += log(L[r][r]);
        out->c[j] = (float)(log(w) - half_logdet - 0.5 * C * log(2.0 * M_PI));
        for (int r = 0; r < C; ++r) {
            const double m = g->mean[j][r];
            if (!isfinite(m)) return DOPE_EINVAL;
            out->mean[j][r] = (float)m;
            for (int c = 0; c <= r; ++c) out->Li[j][r * (r + 1) / 2 + c] = (float)Li[r][c];
        }
    }
    return DOPE_OK;
}

template <int C>
__device__ __forceinline__ float mixture_ll(const GmmDev& g, const float* x) {
    float l[MAXC];
    float top = -INFINITY;
#pragma unroll
    for (int j = 0; j < MAXC; ++j) {
        if (j < g.K) {
            float q = 0.f;
#pragma unroll
            for (int r = 0; r < C; ++r) {
                float z = 0.f;
#pragma unroll
                for (int c = 0; c <= r; ++c) z = fmaf(g.Li[j][r * (r + 1) / 2 + c], x[c] - g.mean[j][c], z);
                q = fmaf(z, z, q);
            }
            l[j] = fmaf(-0.5f, q, g.c[j]);
            top = fmaxf(top, l[j]);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < MAXC; ++j)
        if (j < g.K) s += expf(l[j] - top);
    return top + logf(s);
}

constexpr int GMM_TILE = 256;   // pixels per CTA tile (one per thread)

// Each CTA stages a tile of GMM_TILE pixels (GMM_TILE * C consecutive floats)
// through shared memory with coalesced loads, then evaluates one pixel per
// thread; grid-stride over tiles.  Plain (L2-allocating) loads and stores:
// the image is read again by the contrast kernels and u by the quantiser.
template <int C>
__global__ void __launch_bounds__(GMM_TILE) k_gmm_unaries(const float* __restrict__ img, long long n,
                                                           GmmPair P, float clip, float* __restrict__ u) {
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
            float v = mixture_ll<C>(P.bg, x) - mixture_ll<C>(P.fg, x);
            v = v < -clip ? -clip : (v > clip ? clip : v);   // NaN stays NaN
            u[p0 + threadIdx.x] = v;
        }
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

// Sum over every neighbour pair of |x_i - x_j|: per pixel in FP32 (offset
// order), over pixels in FP64; one double atomic per warp into acc.
template <int C>
__global__ void __launch_bounds__(256) k_contrast_sum(const float* __restrict__ img, ContrastGeo G,
                                                      double* __restrict__ acc) {
    double part = 0.0;
    const unsigned HW = (unsigned)G.H * (unsigned)G.W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < G.N;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned ii = (unsigned)i;   // N < 2^31
        const int x = (int)(ii % (unsigned)G.W), y = (int)((ii / (unsigned)G.W) % (unsigned)G.H),
                  z = (int)(ii / (unsigned)HW);
        float xi[C];
#pragma unroll
        for (int c = 0; c < C; ++c) xi[c] = __ldg(&img[i * C + c]);
        float s = 0.f;
        for (int d = 0; d < G.nh; ++d) {
            const int zz = z + G.off[d][0], yy = y + G.off[d][1], xx = x + G.off[d][2];
            if (zz >= G.D || yy < 0 || yy >= G.H || xx < 0 || xx >= G.W) continue;
            const long long j = ((long long)zz * G.H + yy) * G.W + xx;
            s = __fadd_rn(s, __fsqrt_rn(contrast_d2<C>(xi, &img[j * C])));
        }
        part += (double)s;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && part != 0.0) atomicAdd(acc, part);
}

// wq[d][i] for every pixel and forward offset.  sigma_given > 0 is used as
// is; otherwise sigma = max(acc[0] / pairs, 1e-6).  Thread 0 of CTA 0 stores
// the sigma used in acc[1].
template <int C>
__global__ void __launch_bounds__(256) k_contrast_weights(const float* __restrict__ img, ContrastGeo G,
                                                          double sigma_given, double pairs,
                                                          double* __restrict__ acc, int32_t* __restrict__ wq) {
    double sigma = sigma_given;
    if (!(sigma > 0.0)) {
        sigma = pairs > 0.0 ? __ddiv_rn(acc[0], pairs) : 0.0;
        if (!(sigma >= 1e-6)) sigma = 1e-6;
    }
    const float k = __double2float_rn(__ddiv_rn(1.0, __dmul_rn(__dmul_rn(2.0, sigma), sigma)));
    if (blockIdx.x == 0 && threadIdx.x == 0 && acc) acc[1] = sigma;
    const unsigned HW = (unsigned)G.H * (unsigned)G.W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < G.N;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned ii = (unsigned)i;   // N < 2^31
        const int x = (int)(ii % (unsigned)G.W), y = (int)((ii / (unsigned)G.W) % (unsigned)G.H),
                  z = (int)(ii / (unsigned)HW);
        float xi[C];
#pragma unroll
        for (int c = 0; c < C; ++c) xi[c] = __ldg(&img[i * C + c]);
        for (int d = 0; d < G.nh; ++d) {
            const int zz = z + G.off[d][0], yy = y + G.off[d][1], xx = x + G.off[d][2];
            int32_t q = 0;
            if (zz < G.D && yy >= 0 && yy < G.H && xx >= 0 && xx < G.W) {
                const long long j = ((long long)zz * G.H + yy) * G.W + xx;
                const float a = __fmul_rn(contrast_d2<C>(xi, &img[j * C]), k);
                float e = expf(-a);
                e = __fmul_rn(e, G.invdist[d]);
                q = __float2int_rn(__fmul_rn(1024.f, e));
            }
            wq[(long long)d * G.N + i] = q;
        }
    }
}

int grid_cap() {
    static int sms = 0;
    if (!sms) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            sms = v;
        else {
            cudaGetLastError();
            sms = 152;
        }
    }
    return sms * 8;
}

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
    switch (C) {
        case 1: k_gmm_unaries<1><<<blocks, GMM_TILE, 0, st>>>(img, n, P, cl, u); break;
        case 2: k_gmm_unaries<2><<<blocks, GMM_TILE, 0, st>>>(img, n, P, cl, u); break;
        case 3: k_gmm_unaries<3><<<blocks, GMM_TILE, 0, st>>>(img, n, P, cl, u); break;
        default: k_gmm_unaries<4><<<blocks, GMM_TILE, 0, st>>>(img, n, P, cl, u); break;
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
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > (1 << 30)) return DOPE_EINVAL;
    if (ndim == 2 && dims[0] != 1) return DOPE_EINVAL;
    const long long N = dims[0] * dims[1] * dims[2];
    if (N >= (1LL << 31)) return DOPE_EINVAL;
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
    const int blocks = blocks_for(N, 256);
    if (!(sigma > 0.0)) {
        PCK(cudaMemsetAsync(ws, 0, 2 * sizeof(double), st));
        switch (C) {
            case 1: k_contrast_sum<1><<<blocks, 256, 0, st>>>(img, G, ws); break;
            case 2: k_contrast_sum<2><<<blocks, 256, 0, st>>>(img, G, ws); break;
            case 3: k_contrast_sum<3><<<blocks, 256, 0, st>>>(img, G, ws); break;
            default: k_contrast_sum<4><<<blocks, 256, 0, st>>>(img, G, ws); break;
        }
        PCK(cudaGetLastError());
    }
    switch (C) {
        case 1: k_contrast_weights<1><<<blocks, 256, 0, st>>>(img, G, sigma, pairs, ws, wq); break;
        case 2: k_contrast_weights<2><<<blocks, 256, 0, st>>>(img, G, sigma, pairs, ws, wq); break;
        case 3: k_contrast_weights<3><<<blocks, 256, 0, st>>>(img, G, sigma, pairs, ws, wq); break;
        default: k_contrast_weights<4><<<blocks, 256, 0, st>>>(img, G, sigma, pairs, ws, wq); break;
    }
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
