// dope_big.h -- launchers of the larger-kernel instantiations (5x5, 7x7, 9x9
// squares: conn 24, 48, 80; radius-2 ball: conn 32) of the overlapping-
// partition kernels.  They are compiled in their own translation unit
// (dope_big.cu) so that the build stays parallel; dope.cu calls them for
// those connectivities.  Internal to the library.
#pragma once

namespace dope {

bool big_conn(int conn);
void big_raise_smem(int conn);
// One Algorithm 1 iteration on the overlapping partition: block solves, Eq. 10,
// Eq. 11 (mid, if not null, is recorded between the solve and the updates).
void big_ov_iteration(int conn, const OvArgs& A, int threads, int smem, double mu, int t, int check_prev,
                      cudaStream_t st, cudaEvent_t mid);
void big_set_weights(int conn, const Geo& g, const int32_t* src, int32_t* Wl, double lambda, Ctrl* ctrl,
                     int blocks, int threads, cudaStream_t st);
void big_energy_img(int conn, int D, int H, int W, const int32_t* U, const int32_t* Wl, const uint8_t* lab,
                    Ctrl* ctrl, int blocks, int threads, cudaStream_t st);

}  // namespace dope

// The checked build's shared-memory index record of dope_big.cu (0 on the
// ordinary build); clear != 0 resets it.
int dope_big_check_word(unsigned long long* w, int clear);
