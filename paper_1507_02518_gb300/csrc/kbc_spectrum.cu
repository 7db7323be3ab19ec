// kbc_spectrum.cu -- shell-summed kinetic-energy spectrum E(kappa) of a velocity field on a
// periodic N^3 grid (Sec. "Numerical Simulations": k = integral of E(kappa) d kappa,
// D(kappa) = 2 nu kappa^2 E(kappa)).
//
// Per component, a copy to an aligned real buffer and a real-to-complex 3D FFT (cuFFT,
// library step) in the caller's work buffer, then shell_kernel bins 1/2 |u_hat|^2 / P^2 by m = rint(|n|) of the integer wave
// vector n in a per-block shared-memory histogram (FP64), and shell_final_kernel adds the
// block histograms in a fixed order. The n = 0 mode (the mean flow) is left out.
#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include "kbc_ops.h"

namespace kbc {
namespace {

constexpr int kSpecBlocks = 608;  // 4 per SM on 152 SMs
constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

template <typename C> __device__ __forceinline__ double norm2(const C& c) {
  return (double)c.x * (double)c.x + (double)c.y * (double)c.y;
}

template <typename C>
__global__ void __launch_bounds__(256) shell_kernel(const C* X, uint32_t n, int nbins,
                                                    double scale, double* partials) {
  extern __shared__ double hist[];
  for (int m = threadIdx.x; m < nbins; m += blockDim.x) hist[m] = 0.0;
  __syncthreads();
  const uint32_t nh = n / 2 + 1;
  const uint64_t total = (uint64_t)n * n * nh;
  for (uint64_t idx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t kx = (uint32_t)(idx % nh);
    const uint64_t r = idx / nh;
    const uint32_t ky = (uint32_t)(r % n), kz = (uint32_t)(r / n);
    const int ix = (int)kx;
    const int iy = ky <= n / 2 ? (int)ky : (int)ky - (int)n;
    const int iz = kz <= n / 2 ? (int)kz : (int)kz - (int)n;
    if (ix == 0 && iy == 0 && iz == 0) continue;
    // the half spectrum holds one of each pair (n, -n), whose two halves |u_hat|^2 / 2 are
    // equal, except on the kx = 0 and kx = n/2 planes, which hold both members
    const double w = (kx == 0 || (n % 2 == 0 && kx == n / 2)) ? 1.0 : 2.0;
    const int m = (int)rint(sqrt((double)(ix * ix + iy * iy + iz * iz)));
    if (m < nbins) atomicAdd(&hist[m], w * scale * norm2(X[idx]));
  }
  __syncthreads();
  for (int m = threadIdx.x; m < nbins; m += blockDim.x)
    partials[(uint64_t)blockIdx.x * nbins + m] = hist[m];
}

__global__ void shell_final_kernel(const double* partials, int nblocks, int nbins,
                                   double* bins) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < nbins; m += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < nblocks; ++b) acc += partials[(uint64_t)b * nbins + m];
    bins[m] += acc;
  }
}

struct Plan {
  cufftHandle h = 0;
  bool ok = false;
  ~Plan() {
    if (ok) cufftDestroy(h);
  }
};

// plan without its own work area; *ws receives the work-area bytes
cufftResult make_plan(Plan* p, uint32_t n, bool fp64, size_t* ws) {
  cufftResult r = cufftCreate(&p->h);
  if (r != CUFFT_SUCCESS) return r;
  p->ok = true;
  r = cufftSetAutoAllocation(p->h, 0);
  if (r != CUFFT_SUCCESS) return r;
  return cufftMakePlan3d(p->h, (int)n, (int)n, (int)n, fp64 ? CUFFT_D2Z : CUFFT_R2C, ws);
}

struct WorkLayout {
  size_t real, spec, fft, partials, bins, total;
};
WorkLayout layout(uint32_t n, bool fp64, int nbins, size_t fft_ws) {
  WorkLayout L;
  size_t off = 0;
  // one velocity component, copied to a 256-byte aligned start (the components of the
  // velocity field start at multiples of n^3 values, which cuFFT does not accept for odd n)
  L.real = off;
  off += align_up((size_t)n * n * n * (fp64 ? 8 : 4));
  L.spec = off;
  off += align_up((size_t)n * n * (n / 2 + 1) * (fp64 ? 16 : 8));
  L.fft = off;
  off += align_up(fft_ws);
  L.partials = off;
  off += align_up(sizeof(double) * (size_t)kSpecBlocks * nbins);
  L.bins = off;
  off += align_up(sizeof(double) * (size_t)nbins);
  L.total = off;
  return L;
}

}  // namespace

size_t spectrum_work_bytes(uint32_t n, bool fp64, int nbins) {
  Plan p;
  size_t ws = 0;
  if (make_plan(&p, n, fp64, &ws) != CUFFT_SUCCESS) return 0;
  return layout(n, fp64, nbins, ws).total;
}

// ufield: [3][n^3] velocity in FP64 (fp64) or FP32; bins_host receives nbins values
int spectrum(const void* ufield, uint32_t n, bool fp64, int nbins, void* work, size_t work_bytes,
             double* bins_host, cudaStream_t st, const char** why) {
  Plan p;
  size_t ws = 0;
  if (make_plan(&p, n, fp64, &ws) != CUFFT_SUCCESS) {
    *why = "cuFFT plan creation failed";
    return 3;
  }
  const WorkLayout L = layout(n, fp64, nbins, ws);
  if (work_bytes < L.total) {
    *why = "work buffer smaller than lb_spectrum_work_bytes";
    return 2;
  }
  char* base = (char*)work;
  if (cufftSetWorkArea(p.h, base + L.fft) != CUFFT_SUCCESS ||
      cufftSetStream(p.h, st) != CUFFT_SUCCESS) {
    *why = "cuFFT work area or stream";
    return 3;
  }
  double* bins = (double*)(base + L.bins);
  double* partials = (double*)(base + L.partials);
  cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(double) * nbins, st);
  const uint64_t P = (uint64_t)n * n * n;
  const double scale = 0.5 / ((double)P * (double)P);
  const size_t shm = sizeof(double) * nbins;
  const size_t esz = fp64 ? 8 : 4;
  for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
    e = cudaMemcpyAsync(base + L.real, (const char*)ufield + a * P * esz, P * esz,
                        cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) break;
    cufftResult r;
    if (fp64) {
      r = cufftExecD2Z(p.h, (cufftDoubleReal*)(base + L.real),
                       (cufftDoubleComplex*)(base + L.spec));
    } else {
      r = cufftExecR2C(p.h, (cufftReal*)(base + L.real), (cufftComplex*)(base + L.spec));
    }
    if (r != CUFFT_SUCCESS) {
      *why = "cuFFT execution failed";
      return 3;
    }
    if (fp64)
      shell_kernel<cufftDoubleComplex><<<kSpecBlocks, 256, shm, st>>>(
          (const cufftDoubleComplex*)(base + L.spec), n, nbins, scale, partials);
    else
      shell_kernel<cufftComplex><<<kSpecBlocks, 256, shm, st>>>(
          (const cufftComplex*)(base + L.spec), n, nbins, scale, partials);
    shell_final_kernel<<<(nbins + 255) / 256, 256, 0, st>>>(partials, kSpecBlocks, nbins, bins);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bins_host, bins, sizeof(double) * nbins, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return 3;
  }
  return 0;
}

}  // namespace kbc
