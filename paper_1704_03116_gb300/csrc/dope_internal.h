// dope_internal.h -- C++ interface between the solver library (dope.cu) and
// the request server (dope_server.cu).  Not part of the C-ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "dope.h"
#include "dope_potentials.h"

// SM count of the current device (queried once per device and cached;
// 1 if the query fails).  Grid-stride kernels size their grids from it.
int dope_sm_count();

// Source of device memory for a context.  alloc returns 256-byte aligned
// device memory or null; release gives it back.  A null alloc means
// cudaMalloc / cudaFree.
struct dope_allocator {
    void* self;
    void* (*alloc)(void* self, size_t bytes);
    void (*release)(void* self, void* ptr);
};

// Face and halo tables of one (connectivity, block shape), in device memory.
// They depend on nothing else, so every context of that kind can share one.
struct dope_tables {
    int conn;
    int32_t blk[3];          // (bd, bh, bw)
    int F, NH;
    int16_t* faceIndex;      // [B]
    int16_t* faceLocal;      // [F]
    int* halo;               // [conn][F]
    int16_t* hslot;          // [conn][F]
    int* hinfo;              // [NH]
    size_t bytes;            // device bytes held
    dope_allocator al;
};

// Build the tables (host computation, stream-ordered copies).
int dope_tables_create(int conn, const int32_t blk3[3], const dope_allocator* al, cudaStream_t st,
                       dope_tables** out);
void dope_tables_destroy(dope_tables* t);

// dope_create with three extensions: pad != 0 rounds the grid up to whole
// blocks (the extra pixels are padding: zero unary, no n-links); device memory
// comes from `al` (null: cudaMalloc); `tab` (null: built here) supplies the
// tables.  All device work is issued on `st` and nothing synchronises: the
// context is ready once `st` has drained.
int dope_create_ex(const int64_t* grid, int ndim, int connectivity, const int32_t* block_shape,
                   double lambda, const dope_params* p, int pad, const dope_allocator* al,
                   dope_tables* tab, cudaStream_t st, dope_ctx** out);

// Stream-ordered upload of unaries and weights in the caller's grid order
// (where = DOPE_HOST: through a staging buffer taken from the context's
// allocator).  Errors found by the device land in the context's status word;
// read it with dope_ctx_status once `st` has drained.
// after_copies (may be null) is recorded on `st` once the host copies are
// issued, before the set-up kernels.
int dope_upload_async(dope_ctx* c, const float* u, const int32_t* wq, int where, cudaStream_t st,
                      cudaEvent_t after_copies);
int dope_ctx_status(dope_ctx* c, int* status, cudaStream_t st);   // synchronises `st`
// Stream-ordered copy of the status word into pinned host memory.
int dope_status_async(dope_ctx* c, int* status_pinned, cudaStream_t st);
int dope_ctx_max_iter(const dope_ctx* c);
void dope_release_staging(dope_ctx* c);                           // after `st` drained
size_t dope_ctx_device_bytes(const dope_ctx* c);
int64_t dope_ctx_pixels(const dope_ctx* c);                      // caller's grid

// Finish (step a8) of a context, stream-ordered: labels of the last iteration
// in the caller's grid order into `labels_dev` (device memory) and E_int.
// energy_pinned (pinned host memory, may be null) receives E_int once `st` drains.
int dope_finish_async(dope_ctx* c, uint8_t* labels_dev, int64_t* energy_pinned, cudaStream_t st);
int dope_iterations(const dope_ctx* c, int* t, int* converged);

// Batched launch: all contexts advance together in one cooperative launch.
struct dope_batch_ws;
int dope_batch_ws_create(dope_batch_ws** out);
void dope_batch_ws_destroy(dope_batch_ws* w);

// Issue one batched launch (asynchronous).  Each context runs up to
// min(n_iter, max_iter - t) more iterations.  exit_on_done ends the launch at
// the first iteration boundary where a context finished and others remain;
// yield_flag (device-readable, may be null) ends it at the next boundary once
// nonzero.  clear_status clears each context's status word first (else a
// context with a nonzero status does not iterate).
int dope_batch_launch(dope_ctx* const* cs, int n, int n_iter, int exit_on_done, int clear_status,
                      const int* yield_flag, dope_batch_ws* w, cudaStream_t st);
// After `st` drained: fold the launch's results into the contexts; per
// context iterations done so far, stop test held, status.  Returns the
// launch's own status (barrier timeout) or DOPE_OK.
int dope_batch_collect(dope_ctx* const* cs, int n, dope_batch_ws* w, int* t, int* conv, int* status);

// The single-problem path (what dope_solve runs) from the context's current
// state to its stop test or max_iter; synchronises `st`.
int dope_run_single(dope_ctx* c, cudaStream_t st, int* t, int* conv);

// dope_upload_async for a request given as an image: the image (host copy
// staged first; after_copies, if not null, is recorded once the caller's
// image is no longer read) goes through the potentials kernels into the
// context's staging memory and then through the quantisers.  Stream-ordered;
// the status word is read later (dope_ctx_status / dope_status_async).
int dope_image_upload_async(dope_ctx* c, const dope_image_request* q, int where, cudaStream_t st,
                            cudaEvent_t after_copies);

// Whole-image potentials (dope_potentials.cu), stream-ordered, no
// synchronisation.  pot_unaries_issue: u[i] of n pixels of a [n][C] image.
// pot_weights_issue: wq [conn/2][N] of a (D, H, W) grid (D = 1 for ndim 2);
// ws = 2 doubles of device scratch (sum of contrasts, sigma used), needed
// only when sigma <= 0.  Both validate their arguments (DOPE_EINVAL) before
// any GPU work.
int pot_unaries_issue(const float* img, long long n, int C, const dope_gmm* fg, const dope_gmm* bg, double clip,
                      float* u, cudaStream_t st);
int pot_weights_issue(const float* img, const int64_t dims[3], int ndim, int C, int conn, double sigma,
                      int inv_dist, int32_t* wq, double* ws, cudaStream_t st);
