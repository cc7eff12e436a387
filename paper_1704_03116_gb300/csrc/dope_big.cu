// dope_big.cu -- the larger-kernel instantiations (Section 3's kernel sizes
// 5, 7 and 9) of the overlapping-partition kernels, in a translation unit of
// their own so the library builds in parallel.  Only templates are
// instantiated here; every non-template kernel and the batched launch's
// constant table are defined once, in dope.cu.
#include <cuda_runtime.h>

#include <mutex>

#include "dope.h"
#define DOPE_KERNEL_TEMPLATES_ONLY
#include "dope_kernels.cuh"
#include "dope_overlap.cuh"
#include "dope_big.h"

int dope_sm_count();   // dope.cu: SM count of the current device (cached)

namespace dope {

namespace {

template <class F>
void big_dispatch(int conn, F&& f) {
    switch (conn) {
        case 24: f(std::integral_constant<int, 24>{}); break;
        case 48: f(std::integral_constant<int, 48>{}); break;
        case 80: f(std::integral_constant<int, 80>{}); break;
        case 32: f(std::integral_constant<int, 32>{}); break;
        default: break;
    }
}

// Dynamic shared memory limit of a kernel raised to the device's opt-in maximum.
void raise_limit(const void* fn) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess && optin > (int)fa.sharedSizeBytes)
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaGetLastError();
}

// CTAs for n elements: one per element group, at most 32 per SM of the
// current device (the kernels stride over the rest).
int grid_for_n(long long n, int threads) {
    const int sms = dope_sm_count();
    long long b = (n + threads - 1) / threads;
    if (b > 32LL * sms) b = 32LL * sms;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

bool big_conn(int conn) { return conn == 24 || conn == 48 || conn == 80 || conn == 32; }

void big_raise_smem(int conn) {
    static std::once_flag once[4];
    const int i = conn == 24 ? 0 : (conn == 48 ? 1 : (conn == 80 ? 2 : 3));
    big_dispatch(conn, [&](auto cc) {
        std::call_once(once[i], []() { raise_limit((const void*)k_ov_solve<decltype(cc)::value>); });
    });
}

void big_ov_iteration(int conn, const OvArgs& A, int threads, int smem, double mu, int t, int check_prev,
                      cudaStream_t st, cudaEvent_t mid) {
    big_dispatch(conn, [&](auto cc) {
        constexpr int C = decltype(cc)::value;
        k_ov_solve<C><<<A.g.K, threads, smem, st>>>(A, mu, t, check_prev);
        if (mid) cudaEventRecord(mid, st);
        if ((A.gd | A.gh | A.gw) == 0) {
            k_ov_y_q1<C><<<grid_for_n(A.N, 256), 256, 0, st>>>(A, mu);
        } else if (A.inner) {
            k_ov_y_inner<C><<<grid_for_n(A.n_inner, 256), 256, 0, st>>>(A, mu);
            k_ov_y_band<C><<<grid_for_n(A.n_band, 256), 256, 0, st>>>(A, mu);
        } else {
            k_ov_y<C><<<grid_for_n(A.N, 256), 256, 0, st>>>(A, mu);
        }
        k_ov_a<C><<<A.g.K, 256, 0, st>>>(A, t);
    });
}

void big_set_weights(int conn, const Geo& g, const int32_t* src, int32_t* Wl, double lambda, Ctrl* ctrl,
                     int blocks, int threads, cudaStream_t st) {
    big_dispatch(conn, [&](auto cc) {
        k_set_weights<decltype(cc)::value><<<blocks, threads, 0, st>>>(g, src, Wl, lambda, ctrl, 0);
    });
}

void big_energy_img(int conn, int D, int H, int W, const int32_t* U, const int32_t* Wl, const uint8_t* lab,
                    Ctrl* ctrl, int blocks, int threads, cudaStream_t st) {
    big_dispatch(conn, [&](auto cc) {
        k_energy_img<decltype(cc)::value><<<blocks, threads, 0, st>>>(D, H, W, U, Wl, lab, ctrl);
    });
}

}  // namespace dope

// The checked build's index record of this translation unit (the larger-kernel
// instantiations): read, and cleared if asked.  0 on the ordinary build.
int dope_big_check_word(unsigned long long* w, int clear) {
#ifdef DOPE_CHECKED
    if (cudaMemcpyFromSymbol(w, dope::dope_check_word, sizeof(*w)) != cudaSuccess) {
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
#else
    (void)clear;
    *w = 0;
#endif
    return DOPE_OK;
}

