// lb_noalloc.cu -- diagnostics of a population field without any memory allocation.
//
// Some callers cannot allocate device memory at the moment they want diagnostics:
//   * extensions running inside a host framework that reserves the device's memory through
//     its own pool allocator: a cudaMalloc behind the pool's back can fail once the pool has
//     taken the GPU's free memory, and memory the pool does not know about breaks its
//     accounting;
//   * monitoring hooks of long jobs whose populations were sized to fill the GPU's memory:
//     there is no room left for a diagnostics work buffer, and the hook must not change the
//     job's footprint between steps;
//   * latency-sensitive loops: cudaMalloc and cudaFree can synchronise the whole device and
//     stall the work of other streams.
// For them this file offers lb_diagnostics_noalloc: the caller passes the populations (device
// memory it already holds) and a host struct for the result, and the work space comes from
// one file-scope __device__ array that the library image carries on every GPU that loads it.
//
// Limits and behaviour, stated for users:
//   * at most kNoallocMaxNodes = 65,536 lattice nodes per call (e.g. 40^3 or 64x32x32); larger
//     boxes are rejected with LB_ERR_INVALID_ARG before any GPU work;
//   * the array (about 1.6 MB) stays resident on each GPU that loaded the library until the
//     process exits;
//   * the first call on a device does a one-time set-up: it looks up the array's device
//     address (cudaGetSymbolAddress) with that device current; make that first call before
//     any stream capture begins;
//   * every call shares the one array per device and keeps the last call's contents (the
//     call clears the sums it accumulates before using them), so calls that overlap on the
//     GPU (different streams, or different host threads) race on it; issue them one after
//     another;
//   * the call enqueues its kernels on the given stream and synchronises that stream before
//     it returns.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "kbc_lb.h"

// message for lb_last_error(NULL) (defined with the other thread-local errors in lb_api.cu)
void kbc_set_thread_error(const std::string& msg);

namespace {

constexpr int kNoallocMaxNodes = 65536;
constexpr int kNaBlocks = 256;     // fixed grid of the reduction kernels
constexpr int kNaThreads = 256;
constexpr int kNaSums = 16;
constexpr int kMaxDevices = 64;

// u field (3 planes) + per-block partial sums + final sums, FP64
constexpr size_t kScratchDoubles =
    (size_t)3 * kNoallocMaxNodes + (size_t)kNaBlocks * kNaSums + kNaSums;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

struct NaGeo {
  uint32_t nx, ny, nz, nxy;
  uint32_t P;
};

__device__ __forceinline__ void na_coords(const NaGeo& g, uint32_t n, uint32_t& x, uint32_t& y,
                                          uint32_t& z) {
  z = n / g.nxy;
  const uint32_t r = n - z * g.nxy;
  y = r / g.nx;
  x = r - y * g.nx;
}

__device__ __forceinline__ uint32_t na_wrap(int v, uint32_t n) {
  return v < 0 ? n - 1 : ((uint32_t)v == n ? 0 : (uint32_t)v);
}

template <int N>
__device__ __forceinline__ void na_block_sum(double (&v)[N], double* dst) {
  __shared__ double sh[kNaThreads / 32][N];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
  if (lane == 0)
    for (int j = 0; j < N; ++j) sh[warp][j] = v[j];
  __syncthreads();
  if (threadIdx.x < N) {
    double acc = 0.0;
    for (int w = 0; w < kNaThreads / 32; ++w) acc += sh[w][threadIdx.x];
    dst[threadIdx.x] = acc;
  }
}

// rho, rho u and u of every node of the canonical field f[27][P]; partial sums per block over
// the nodes whose rho and u are finite: 0 sum rho, 1-3 sum rho u, 4-6 sum u, 7 sum |u|^2,
// and 10 the number of non-finite nodes
__global__ void __launch_bounds__(kNaThreads) na_fields_kernel(const double* __restrict__ f,
                                                               NaGeo g, double* scratch) {
  double* uf = scratch;
  double* partials = scratch + 3 * (size_t)kNoallocMaxNodes;
  double v[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < g.P; n += gridDim.x * blockDim.x) {
    double rho = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
    for (int i = 0; i < 27; ++i) {
      const double fi = f[(size_t)i * g.P + n];
      rho += fi;
      mx += (i % 3 - 1) * fi;
      my += ((i / 3) % 3 - 1) * fi;
      mz += (i / 9 - 1) * fi;
    }
    const double ux = mx / rho, uy = my / rho, uz = mz / rho;
    uf[n] = ux;
    uf[g.P + n] = uy;
    uf[2 * (size_t)g.P + n] = uz;
    if (!isfinite(rho) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz)) {
      v[10] += 1.0;
      continue;
    }
    v[0] += rho;
    v[1] += mx;
    v[2] += my;
    v[3] += mz;
    v[4] += ux;
    v[5] += uy;
    v[6] += uz;
    v[7] += ux * ux + uy * uy + uz * uz;
  }
  na_block_sum<11>(v, partials + blockIdx.x * kNaSums);
}

// Second pass, after the first pass's sums are reduced: second-order central differences of
// u over the nodes whose gradients are finite, 11 sum |curl u|^2, 12 sum (d_b u_a + d_a u_b)^2,
// 13 their number; and 14 sum |u - <u>|^2 over the finite nodes, <u> from the first pass.
__global__ void __launch_bounds__(kNaThreads) na_grad_kernel(NaGeo g, double* scratch) {
  const double* uf = scratch;
  double* partials = scratch + 3 * (size_t)kNoallocMaxNodes;
  const double* sums = partials + (size_t)kNaBlocks * kNaSums;
  const double nfin = (double)g.P - sums[10];
  const double mean[3] = {sums[4] / nfin, sums[5] / nfin, sums[6] / nfin};
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (uint32_t n = blockIdx.x * blockDim.x + threadIdx.x; n < g.P; n += gridDim.x * blockDim.x) {
    uint32_t x, y, z;
    na_coords(g, n, x, y, z);
    const uint32_t xp = na_wrap((int)x + 1, g.nx), xm = na_wrap((int)x - 1, g.nx);
    const uint32_t yp = na_wrap((int)y + 1, g.ny), ym = na_wrap((int)y - 1, g.ny);
    const uint32_t zp = na_wrap((int)z + 1, g.nz), zm = na_wrap((int)z - 1, g.nz);
    const uint32_t row = y * g.nx + z * g.nxy;
    const uint32_t np[3] = {xp + row, x + yp * g.nx + z * g.nxy, x + y * g.nx + zp * g.nxy};
    const uint32_t nm[3] = {xm + row, x + ym * g.nx + z * g.nxy, x + y * g.nx + zm * g.nxy};
    double gr[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        gr[a][b] = 0.5 * (uf[(size_t)a * g.P + np[b]] - uf[(size_t)a * g.P + nm[b]]);
    const double wx = gr[2][1] - gr[1][2], wy = gr[0][2] - gr[2][0], wz = gr[1][0] - gr[0][1];
    const double ww = wx * wx + wy * wy + wz * wz;
    double ss = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const double s = gr[a][b] + gr[b][a];
        ss += s * s;
      }
    if (isfinite(ww) && isfinite(ss)) {
      v[0] += ww;
      v[1] += ss;
      v[2] += 1.0;
    }
    const double d0 = uf[n] - mean[0], d1 = uf[g.P + n] - mean[1];
    const double d2 = uf[2 * (size_t)g.P + n] - mean[2];
    const double dd = d0 * d0 + d1 * d1 + d2 * d2;
    if (isfinite(dd)) v[3] += dd;
  }
  na_block_sum<4>(v, partials + blockIdx.x * kNaSums + 11);
}

__global__ void na_final_kernel(double* scratch) {
  const double* partials = scratch + 3 * (size_t)kNoallocMaxNodes;
  double* sums = scratch + 3 * (size_t)kNoallocMaxNodes + (size_t)kNaBlocks * kNaSums;
  const int j = threadIdx.x;
  if (j >= kNaSums) return;
  double acc = 0.0;
  for (int b = 0; b < kNaBlocks; ++b) acc += partials[b * kNaSums + j];
  sums[j] = acc;
}

// Device address of the scratch array on the current device, looked up once per device.
lb_status scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    kbc_set_thread_error(std::string("no current CUDA device: ") + cudaGetErrorString(e));
    return LB_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    kbc_set_thread_error("device index out of range for the static scratch table");
    return LB_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      kbc_set_thread_error(std::string("cudaGetSymbolAddress of the diagnostics scratch failed: ") +
                        cudaGetErrorString(e));
      return LB_ERR_CUDA;
    }
    g_scratch_ptr[dev] = (double*)p;
  }
  *out = g_scratch_ptr[dev];
  return LB_OK;
}

}  // namespace

extern "C" {

lb_status lb_diagnostics_noalloc(int32_t nx, int32_t ny, int32_t nz, double nu, const double* f,
                                 void* stream, lb_diag* out) {
  if (!out || !f) {
    kbc_set_thread_error("f and out must not be NULL");
    return LB_ERR_INVALID_ARG;
  }
  if (nx < 3 || ny < 3 || nz < 3) {
    kbc_set_thread_error("every box edge must be >= 3");
    return LB_ERR_INVALID_ARG;
  }
  const uint64_t P = (uint64_t)nx * ny * nz;
  if (P > (uint64_t)kNoallocMaxNodes) {
    char buf[160];
    snprintf(buf, sizeof buf,
             "box of %llu nodes exceeds the %d-node limit of the static diagnostics scratch",
             (unsigned long long)P, kNoallocMaxNodes);
    kbc_set_thread_error(buf);
    return LB_ERR_INVALID_ARG;
  }
  if (!(nu > 0.0) || !std::isfinite(nu)) {
    kbc_set_thread_error("nu must be finite and > 0");
    return LB_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  lb_status s = scratch_for_current_device(&scratch);
  if (s != LB_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  NaGeo g;
  g.nx = (uint32_t)nx;
  g.ny = (uint32_t)ny;
  g.nz = (uint32_t)nz;
  g.nxy = g.nx * g.ny;
  g.P = (uint32_t)P;
  double* partials = scratch + 3 * (size_t)kNoallocMaxNodes;
  double* sums = partials + (size_t)kNaBlocks * kNaSums;
  // the array keeps the previous call's contents: the partial sums must start from zero
  cudaError_t e = cudaMemsetAsync(partials, 0, sizeof(double) * (kNaBlocks * kNaSums + kNaSums), st);
  if (e == cudaSuccess) {
    na_fields_kernel<<<kNaBlocks, kNaThreads, 0, st>>>(f, g, scratch);
    na_final_kernel<<<1, 32, 0, st>>>(scratch);  // <u> for the second pass
    na_grad_kernel<<<kNaBlocks, kNaThreads, 0, st>>>(g, scratch);
    na_final_kernel<<<1, 32, 0, st>>>(scratch);
    e = cudaGetLastError();
  }
  double h[kNaSums];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, sums, sizeof h, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    kbc_set_thread_error(std::string("diagnostics without allocation: ") + cudaGetErrorString(e));
    return LB_ERR_CUDA;
  }
  // averages over the nodes whose moments (Pf) or velocity gradients (Pg) are finite
  const double Pf = (double)P - h[10], Pg = h[13];
  memset(out, 0, sizeof *out);
  out->step = -1;
  out->nodes = (int64_t)P;
  out->mass = h[0];
  for (int a = 0; a < 3; ++a) out->momentum[a] = h[1 + a];
  out->kinetic_energy = 0.5 * h[14] / Pf;  // k = 1/2 <|u - <u>|^2>, two passes
  out->enstrophy = 0.5 * h[11] / Pg;
  out->dissipation = 0.5 * nu * h[12] / Pg;
  out->gamma_mean = NAN;
  out->gamma_std = NAN;
  out->nonfinite_count = (int64_t)h[10];
  out->den_guard_count = 0;
  out->grad_order = 2;
  out->reserved = 0;
  out->dudx2 = NAN;  // the longitudinal-derivative moments are not computed here
  for (int m = 0; m < 4; ++m) out->skewness[m] = NAN;
  if (out->nonfinite_count > 0) {
    kbc_set_thread_error("the population field holds NaN/Inf");
    return LB_ERR_NONFINITE;
  }
  return LB_OK;
}

}  // extern "C"
