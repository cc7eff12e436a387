/*
 * dope_potentials.h -- C-ABI of the whole-image potentials on the GPU.
 *
 * Algorithm 1 begins by computing the unary and pairwise potentials of the
 * whole image (its first step, before the partition); Section 4 reports that
 * this step, which every partition pays in full, takes a large share of the
 * paper's run times.  These calls compute both from the image on the device,
 * so a solve can start from pixels instead of from potentials copied in:
 *
 *   data term (Eq. 1, the negative log-likelihood form of Section 2):
 *     u_i = clip( log p_bg(x_i) - log p_fg(x_i) ),
 *     p(x) = sum_j pi_j N(x; m_j, S_j)          (Gaussian mixture colour model;
 *                                                Section 4 draws its colour
 *                                                models from clusters of seeds)
 *   pairwise term (Eq. 1 with the contrast-sensitive Potts weights of
 *   Section 2), for every forward offset of the neighbourhood:
 *     w_ij = exp( -|x_i - x_j|^2 / (2 sigma^2) ) [ / |p_i - p_j| ],
 *     wq_ij = rne(1024 w_ij), 0 where the partner lies outside the grid;
 *     sigma = the given value, or (sigma <= 0) the mean of |x_i - x_j| over
 *     every neighbour pair of the grid, each pair once, floored at 1e-6.
 *
 * Conventions (as in dope.h): pixel index i = (z*H + y)*W + x; images are
 * float32, pixel-major with the channels interleaved ([N][C], C = 1..4);
 * forward offsets in the order dope.h lists for connectivity 4 / 8 / 6, and
 * for the larger kernels (24, 48, 80: 5x5, 7x7, 9x9 squares in 2-D; 32: the
 * radius-2 ball in 3-D) every offset (dz, dy, dx) of the kernel whose first
 * non-zero coordinate is positive, in increasing (dz, dy, dx) order.
 *
 * Precision: FP32 arithmetic on the device, with the mixture constants
 * (Cholesky factors, log-determinants, log-weights) formed on the host in
 * FP64; the data term combines its components with the hardware base-2
 * exponential and logarithm (errors near 2^-22), and the weights use one
 * FP32 exp per pair.  The quantised weight of a pair whose 1024 w lies
 * within a few FP32 ulp of a rounding tie can differ by one from the FP64
 * definition; every other weight is the FP64 definition's rne(1024 w).
 *
 * All pointers named *_dev are device pointers of the current device; the
 * caller owns them.  Work is ordered on `stream` (a cudaStream_t, NULL = the
 * legacy default stream).  Returns DOPE_* status codes (dope.h).
 */
#ifndef DOPE_POTENTIALS_H
#define DOPE_POTENTIALS_H

#include <stdint.h>

#include "dope.h"

#ifdef __cplusplus
extern "C" {
#endif

#define DOPE_GMM_MAX_COMP 8
#define DOPE_GMM_MAX_CH 4

/* One colour model: a mixture of n_comp Gaussians over `channels` features.
 * weight[j] > 0 is used as given (not renormalised); cov[j] must be symmetric
 * positive definite -- only its lower triangle (r >= c) is read. */
typedef struct {
    int n_comp;                                             /* 1..8 */
    int channels;                                           /* 1..4 */
    double weight[DOPE_GMM_MAX_COMP];
    double mean[DOPE_GMM_MAX_COMP][DOPE_GMM_MAX_CH];
    double cov[DOPE_GMM_MAX_COMP][DOPE_GMM_MAX_CH][DOPE_GMM_MAX_CH];
} dope_gmm;

/* Bytes of device workspace dope_contrast_weights needs (8-byte aligned). */
#define DOPE_CONTRAST_WS_BYTES 64

/* Data term of n pixels: u_dev[i] = clip(log p_bg(x_i) - log p_fg(x_i)) in
 * [-clip, clip] (clip > 0), from image_dev [n][channels].  fg and bg are host
 * structs with the same channel count as the image.  Asynchronous on
 * `stream`.  DOPE_EINVAL for a bad argument or a covariance that is not
 * positive definite (checked on the host before any GPU work); n = 0 is a
 * no-op. */
int dope_gmm_unaries(const float* image_dev, int64_t n, int channels, const dope_gmm* fg,
                     const dope_gmm* bg, double clip, float* u_dev, void* stream);

/* Contrast weights of an image on a grid (ndim 2: (H, W), 3: (D, H, W)):
 * wq_dev[k][i] = rne(1024 w) as above, int32 [conn/2][N].  sigma > 0 is used
 * as given; sigma <= 0 computes the mean contrast on the device first (one
 * extra pass over the image).  inv_dist != 0 divides by the pixel distance.
 * workspace_dev: DOPE_CONTRAST_WS_BYTES of device memory owned by the caller,
 * used only when sigma <= 0.  sigma_used (host, may be NULL) receives the
 * sigma applied; passing it synchronises `stream`, otherwise the call is
 * asynchronous.  DOPE_EINVAL for a bad shape / connectivity / channel count
 * / pointer. */
int dope_contrast_weights(const float* image_dev, const int64_t* grid, int ndim, int channels,
                          int connectivity, double sigma, int inv_dist, int32_t* wq_dev,
                          void* workspace_dev, double* sigma_used, void* stream);

/* Both potentials straight into a context (the context's grid and
 * connectivity; the unaries then quantised as by dope_set_unaries, the
 * weights as by dope_set_weights): the image (host or device, `where`) goes
 * through the two calls above into the context's own scratch memory, then
 * into its solver state.  With sigma_used != NULL the call synchronises once
 * at the end and returns the status of dope_set_unaries / dope_set_weights
 * (DOPE_EOVERFLOW when a quantised unary or weight leaves its range); with
 * sigma_used == NULL it does not synchronise, and that status is reported by
 * the next synchronising call on the context, as for dope_set_inputs
 * (dope.h). */
int dope_set_image(dope_ctx* ctx, const float* image, int channels, const dope_gmm* fg,
                   const dope_gmm* bg, double clip, double sigma, int inv_dist, int where,
                   double* sigma_used, void* stream);

/* A request's inputs given as an image, for dope_server_submit
 * (dope_request.image_request): the server computes the potentials on the
 * GPU in the request's set-up, as dope_set_image does, into memory it charges
 * to its arena.  The struct is copied at submit; the image (host or device,
 * dope_request.where_inputs) must stay valid and unchanged until the result
 * has been polled.  A model that is not valid fails the request with
 * DOPE_EINVAL. */
typedef struct {
    const float *image;       /* [N][channels], image order */
    int channels;             /* 1..4, the models' channel count */
    int inv_dist;             /* divide the weights by the pixel distance */
    double clip;              /* > 0 */
    double sigma;             /* > 0: given; <= 0: the mean contrast */
    dope_gmm fg, bg;
} dope_image_request;

#ifdef __cplusplus
}
#endif

#endif /* DOPE_POTENTIALS_H */
