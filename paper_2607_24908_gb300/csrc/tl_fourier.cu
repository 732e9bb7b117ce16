// Initial Gaussian random fields and binned power spectra (off the per-step
// loop).  The paper prepares states and measures in Fourier space through its
// automatic Fourier views (Sec. 2) with Philox-2x64 random numbers (Sec. 2);
// here the mode draw, the field assembly and the shell binning are kernels
// of this library and the transforms are cuFFT library calls (FP64).
#include <math.h>

#include "tl_fourier.cuh"
#include "tl_philox.cuh"

namespace tl {


__device__ __forceinline__ int signed_mode(int i, int N) { return (i < N / 2) ? i : i - N; }

// One entry of the half spectrum [iz][iy][ix], ix in [0, N/2].
__global__ void fill_modes_kernel(double2 *modes, int N, double kIR, double A, double m2, int pi_spectrum,
                                  int fixed_modulus, uint64_t seed, uint64_t stream)
{
    const int NH = N / 2 + 1;
    const size_t total = (size_t)N * N * NH;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % NH);
        const int iy = (int)((i / NH) % N);
        const int iz = (int)(i / ((size_t)NH * N));
        const long nx = ix, ny = signed_mode(iy, N), nz = signed_mode(iz, N);
        const long r2 = nx * nx + ny * ny + nz * nz;
        double2 out = make_double2(0.0, 0.0);
        if (r2 > 0 && 4 * r2 < (long)N * N) {
            const bool canon = nx > 0 || (nx == 0 && (ny > 0 || (ny == 0 && nz > 0)));
            const uint64_t own = ((uint64_t)iz * N + (uint64_t)iy) * N + (uint64_t)ix;
            const uint64_t pz = (uint64_t)((N - iz) % N), py = (uint64_t)((N - iy) % N), px = (uint64_t)((N - ix) % N);
            const uint64_t partner = (pz * N + py) * N + px;
            uint64_t w0, w1;
            philox2x64_10(canon ? own : partner, stream, seed, w0, w1);
            const double two53 = 9007199254740992.0;
            const double u1 = ((double)(w0 >> 11) + 1.0) / two53;
            const double u2 = (double)(w1 >> 11) / two53;
            const double k = kIR * sqrt((double)r2);
            const double om = sqrt(k * k + m2);
            const double P = pi_spectrum ? A * om / 2.0 : A / (2.0 * om);
            const double L = 2.0 * M_PI / kIR;
            const double amp = sqrt(P / (L * L * L)) * (fixed_modulus ? 1.0 : sqrt(-log(u1)));
            double s, c;
            sincos(2.0 * M_PI * u2, &s, &c);
            out = make_double2(amp * c, canon ? amp * s : -amp * s);
        }
        modes[i] = out;
    }
}

// dense index i = (z N + y) N + x  <->  pitched offset z PP + y P + x
__device__ __forceinline__ long long pitched(size_t i, int N, long long P, long long PP)
{
    const long long x = (long long)(i % N), y = (long long)((i / N) % N), z = (long long)(i / ((size_t)N * N));
    return z * PP + y * P + x;
}

template <typename T>
__global__ void assemble_kernel(T *dst, const double *delta, size_t n, double base, double scale, int N, long long P,
                                long long PP)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[pitched(i, N, P, PP)] = (T)(base + (delta ? scale * delta[i] : 0.0));
}

template <typename T>
__global__ void widen_kernel(double *dst, const T *src, size_t n, int N, long long P, long long PP)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[pitched(i, N, P, PP)];
}

// bin(s) = floor(sqrt(s) + 1/2) for an integer s >= 0, decided in integers:
// m is the bin iff m (m - 1) < s <= m (m + 1).
__device__ __forceinline__ int shell_bin(long s)
{
    long m = (long)floor(sqrt((double)s) + 0.5);
    while (m > 0 && m * (m - 1) >= s) --m;
    while ((m + 1) * m < s) ++m;
    return (int)m;
}

__global__ void bin_kernel(const double2 *modes, int N, int nbins, double *Psum, double *rsum,
                           unsigned long long *cnt)
{
    extern __shared__ double sh[];
    double *sP = sh;
    double *sR = sh + nbins;
    unsigned long long *sC = reinterpret_cast<unsigned long long *>(sh + 2 * nbins);
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        sP[b] = 0.0;
        sR[b] = 0.0;
        sC[b] = 0ull;
    }
    __syncthreads();
    const int NH = N / 2 + 1;
    const size_t total = (size_t)N * N * NH;
    const double inv_n6 = 1.0 / ((double)N * N * N) / ((double)N * N * N);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % NH);
        const int iy = (int)((i / NH) % N);
        const int iz = (int)(i / ((size_t)NH * N));
        const long nx = ix, ny = signed_mode(iy, N), nz = signed_mode(iz, N);
        const long r2 = nx * nx + ny * ny + nz * nz;
        const int w = (ix == 0 || 2 * ix == N) ? 1 : 2;  // r2c keeps one of each (n, -n) pair for 0 < nx < N/2
        const double2 d = modes[i];
        const int b = shell_bin(r2);
        atomicAdd(&sP[b], w * (d.x * d.x + d.y * d.y) * inv_n6);
        atomicAdd(&sR[b], w * sqrt((double)r2));
        atomicAdd(&sC[b], (unsigned long long)w);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        if (sC[b]) {
            atomicAdd(&Psum[b], sP[b]);
            atomicAdd(&rsum[b], sR[b]);
            atomicAdd(&cnt[b], sC[b]);
        }
    }
}

static unsigned grid_for(size_t n, int sm_count)
{
    size_t g = (n + 255) / 256;
    size_t cap = (size_t)(sm_count > 0 ? sm_count : 152) * 16;
    return (unsigned)(g < cap ? (g > 0 ? g : 1) : cap);
}

cudaError_t launch_fill_modes(double2 *modes, int N, double kIR, double A, double m2, int pi_spectrum,
                              int fixed_modulus, uint64_t seed, uint64_t stream, int sm_count, cudaStream_t s)
{
    size_t total = (size_t)N * N * (N / 2 + 1);
    fill_modes_kernel<<<grid_for(total, sm_count), 256, 0, s>>>(modes, N, kIR, A, m2, pi_spectrum, fixed_modulus,
                                                                seed, stream);
    return cudaGetLastError();
}

cudaError_t launch_assemble(int dtype, void *dst, const double *delta, size_t n, double base, double scale, int N,
                            long long P, long long PP, int sm_count, cudaStream_t s)
{
    if (dtype == TL_F32)
        assemble_kernel<float><<<grid_for(n, sm_count), 256, 0, s>>>(static_cast<float *>(dst), delta, n, base, scale,
                                                                     N, P, PP);
    else
        assemble_kernel<double><<<grid_for(n, sm_count), 256, 0, s>>>(static_cast<double *>(dst), delta, n, base,
                                                                      scale, N, P, PP);
    return cudaGetLastError();
}

cudaError_t launch_widen(int dtype, double *dst, const void *src, size_t n, int N, long long P, long long PP,
                         int sm_count, cudaStream_t s)
{
    if (dtype == TL_F32)
        widen_kernel<float><<<grid_for(n, sm_count), 256, 0, s>>>(dst, static_cast<const float *>(src), n, N, P, PP);
    else
        widen_kernel<double><<<grid_for(n, sm_count), 256, 0, s>>>(dst, static_cast<const double *>(src), n, N, P, PP);
    return cudaGetLastError();
}

cudaError_t launch_bin(const double2 *modes, int N, int nbins, double *Psum, double *rsum, unsigned long long *cnt,
                       int sm_count, cudaStream_t s)
{
    size_t total = (size_t)N * N * (N / 2 + 1);
    size_t shmem = (size_t)nbins * (2 * sizeof(double) + sizeof(unsigned long long));
    bin_kernel<<<grid_for(total, sm_count), 256, shmem, s>>>(modes, N, nbins, Psum, rsum, cnt);
    return cudaGetLastError();
}

}  // namespace tl
