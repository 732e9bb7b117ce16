// Launchers of the Fourier-space kernels (initial fields, spectra).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tl_internal.cuh"

namespace tl {

// Half-spectrum [N][N][N/2+1] of Hermitian Gaussian modes (see tl_init_spec).
cudaError_t launch_fill_modes(double2 *modes, int N, double kIR, double A, double m2, int pi_spectrum,
                              int fixed_modulus, uint64_t seed, uint64_t stream, int sm_count, cudaStream_t s);
// dst[pitched(i)] = (T)(base + scale * delta[i]) (delta may be NULL; delta dense).
cudaError_t launch_assemble(int dtype, void *dst, const double *delta, size_t n, double base, double scale, int N,
                            long long P, long long PP, int sm_count, cudaStream_t s);
// dst[i] = (double)src[pitched(i)] (dst dense).
cudaError_t launch_widen(int dtype, double *dst, const void *src, size_t n, int N, long long P, long long PP,
                         int sm_count, cudaStream_t s);
// Shell sums of |d|^2 / N^6, |n| and mode counts (accumulated with atomics).
cudaError_t launch_bin(const double2 *modes, int N, int nbins, double *Psum, double *rsum, unsigned long long *cnt,
                       int sm_count, cudaStream_t s);

}  // namespace tl
