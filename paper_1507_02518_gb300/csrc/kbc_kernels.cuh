// kbc_kernels.cuh -- CUDA kernels of the D3Q27 KBC step and its host-transfer helpers.
//
// Included once per storage type by kbc_f64.cu / kbc_f32.cu / kbc_f16.cu, which instantiate
// kbc::Ops<S>. Hot path: step_kernel (one fused stream + KBC collide per node, eq:Egeneral)
// and batch_kernel (the same update over a work list of boxes).
#pragma once

#include <type_traits>

#include "kbc_device.cuh"
#include "kbc_ops.h"
#include "kbc_staged.cuh"

namespace kbc {

// FP64 arithmetic needs more than 128 registers per thread: cap its blocks at 256 threads
template <typename S> struct MaxThreads { static constexpr int value = 512; };
template <> struct MaxThreads<double> { static constexpr int value = 256; };

template <typename S, int MODE, bool RECORD, bool CENTRAL, bool EXACT = false>
__global__ void __launch_bounds__(MaxThreads<S>::value) step_kernel(const S* src, S* dst, Geo g, CollideParams cp,
                                                   float* gamma_out, StepCounters* ctr) {
  const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t y = blockIdx.y * blockDim.y + threadIdx.y;
  const uint32_t z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  node_update<S, MODE, RECORD, CENTRAL, EXACT>(src, dst, g, x, y, z, cp, gamma_out, ctr);
}

// Two nodes per thread with packed FP32x2 arithmetic: a block of 128 threads covers 256
// consecutive x nodes of one row, each warp 64 of them as (x, x + 32) pairs.
template <typename S, int MODE, bool RECORD, bool CENTRAL>
__global__ void __launch_bounds__(128, 3) pair_step_kernel(const S* src, S* dst, Geo g,
                                                        CollideParams cp, float* gamma_out,
                                                        StepCounters* ctr) {
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t xa = blockIdx.x * 256 + warp * 64 + lane;
  const uint32_t xb = xa + 32;
  if (xa >= g.nx) return;
  node_update2<S, MODE, RECORD, CENTRAL>(src, dst, g, xa, xb, xb < g.nx, blockIdx.y, blockIdx.z,
                                         cp, gamma_out, ctr);
}

// one block per 256-node row segment (a persistent grid measured slower on GB300)
template <typename S, int MODE, bool RECORD, bool CENTRAL>
static cudaError_t launch_pair(const S* src, S* dst, const Geo& g, const CollideParams& cp,
                               float* gamma_out, StepCounters* ctr, cudaStream_t st) {
  const dim3 grid((g.nx + 255) / 256, g.ny, g.nz);
  pair_step_kernel<S, MODE, RECORD, CENTRAL><<<grid, 128, 0, st>>>(src, dst, g, cp, gamma_out,
                                                                   ctr);
  return cudaGetLastError();
}

// Batched ensemble: a persistent grid walks the work list; item k covers rows
// [row0, row0 + nrows) (row = y + ny z) of one box.
template <typename S, int MODE, bool RECORD, bool CENTRAL>
__global__ void __launch_bounds__(MaxThreads<S>::value) batch_kernel(const BoxDesc* __restrict__ boxes,
                                                    const WorkItem* __restrict__ items,
                                                    int nitems, int parity, int with_t,
                                                    int with_q, int gamma_mode) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const WorkItem w = items[it];
    const BoxDesc bd = boxes[w.box];
    Geo g;
    g.nx = bd.nx;
    g.ny = bd.ny;
    g.nz = bd.nz;
    g.nxy = bd.nxy;
    g.P = (uint64_t)bd.nxy * bd.nz;
    CollideParams cp;
    cp.beta = bd.beta;
    cp.two_beta = bd.two_beta;
    cp.inv_beta = bd.inv_beta;
    cp.betaf = (float)bd.beta;
    cp.two_betaf = (float)bd.two_beta;
    cp.inv_betaf = (float)bd.inv_beta;
    cp.with_t = with_t;
    cp.with_q = with_q;
    cp.gamma_mode = gamma_mode;
    const S* src = (const S*)bd.pop[MODE == MODE_PULL ? parity : 0];
    S* dst = (S*)bd.pop[MODE == MODE_PULL ? (parity ^ 1) : 0];
    const uint32_t nodes = bd.nx * (uint32_t)w.nrows;
    for (uint32_t k = threadIdx.x; k < nodes; k += blockDim.x) {
      const uint32_t row = (uint32_t)w.row0 + k / bd.nx;
      const uint32_t x = k - (k / bd.nx) * bd.nx;
      const uint32_t z = row / bd.ny;
      const uint32_t y = row - z * bd.ny;
      node_update<S, MODE, RECORD, CENTRAL>(src, dst, g, x, y, z, cp, bd.gamma, bd.ctr);
    }
  }
}

// The packed form of batch_kernel: 128 threads, each item's rows cut into 64-node chunks,
// each thread two nodes (x, x + 32) of a chunk with the FP32x2 collision.
template <typename S, int MODE, bool RECORD, bool CENTRAL>
__global__ void __launch_bounds__(128, 3) batch_pair_kernel(const BoxDesc* __restrict__ boxes,
                                                           const WorkItem* __restrict__ items,
                                                           int nitems, int parity, int with_t,
                                                           int with_q, int gamma_mode) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const WorkItem w = items[it];
    const BoxDesc bd = boxes[w.box];
    Geo g;
    g.nx = bd.nx;
    g.ny = bd.ny;
    g.nz = bd.nz;
    g.nxy = bd.nxy;
    g.P = (uint64_t)bd.nxy * bd.nz;
    CollideParams cp;
    cp.beta = bd.beta;
    cp.two_beta = bd.two_beta;
    cp.inv_beta = bd.inv_beta;
    cp.betaf = (float)bd.beta;
    cp.two_betaf = (float)bd.two_beta;
    cp.inv_betaf = (float)bd.inv_beta;
    cp.with_t = with_t;
    cp.with_q = with_q;
    cp.gamma_mode = gamma_mode;
    const S* src = (const S*)bd.pop[MODE == MODE_PULL ? parity : 0];
    S* dst = (S*)bd.pop[MODE == MODE_PULL ? (parity ^ 1) : 0];
    const uint32_t nchunk = (bd.nx + 63) / 64;
    const uint32_t units = (uint32_t)w.nrows * nchunk * 32;
    for (uint32_t u = threadIdx.x; u < units; u += blockDim.x) {
      const uint32_t slot = u & 31, q = u >> 5;
      const uint32_t rr = q / nchunk, chunk = q - rr * nchunk;
      const uint32_t row = (uint32_t)w.row0 + rr;
      const uint32_t z = row / bd.ny, y = row - z * bd.ny;
      const uint32_t xa = chunk * 64 + slot, xb = xa + 32;
      if (xa < bd.nx)
        node_update2<S, MODE, RECORD, CENTRAL>(src, dst, g, xa, xb, xb < bd.nx, y, z, cp,
                                               bd.gamma, bd.ctr);
    }
  }
}

// ------------------------------------------------------------------ canonical addressing
// Address of canonical population i of node (x, y, z) at a time of the given parity.
template <typename S>
__device__ __forceinline__ S* canon_addr(S* b0, S* b1, const Geo& g, const Nbr& nb, int scheme,
                                         int parity, int i) {
  const uint32_t back = nb.ox[1 - cx(i)] + nb.oy[1 - cy(i)] + nb.oz[1 - cz(i)];
  const uint32_t here = nb.ox[1] + nb.oy[1] + nb.oz[1];
  if (scheme == 0) return (parity ? b1 : b0) + (uint64_t)i * g.P + back;
  if (parity == 0) return b0 + (uint64_t)i * g.P + here;
  return b0 + (uint64_t)(26 - i) * g.P + back;
}

__device__ __forceinline__ void node_coords(const Geo& g, uint64_t n, uint32_t& x, uint32_t& y,
                                            uint32_t& z) {
  z = (uint32_t)(n / g.nxy);
  const uint32_t r = (uint32_t)(n - (uint64_t)z * g.nxy);
  y = r / g.nx;
  x = r - y * g.nx;
}

template <typename S>
__global__ void init_kernel(S* b0, S* b1, Geo g, int scheme, int parity, const double* rho,
                            const double* u, uint64_t n0, uint64_t cnt, uint64_t ld) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < cnt;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x, y, z;
    node_coords(g, n0 + k, x, y, z);
    Nbr nb;
    nb.init(g, x, y, z);
    double dq[27];
    equilibrium_shift<double>(rho ? rho[k] : 1.0, u[k], u[ld + k], u[2 * ld + k], dq);
#pragma unroll
    for (int i = 0; i < 27; ++i)
      *canon_addr<S>(b0, b1, g, nb, scheme, parity, i) = Codec<S>::from_delta(dq[i], i);
  }
}

template <typename S>
__global__ void get_kernel(const S* b0, const S* b1, Geo g, int scheme, int parity, double* out,
                           uint64_t n0, uint64_t cnt, uint64_t ld) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < cnt;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x, y, z;
    node_coords(g, n0 + k, x, y, z);
    Nbr nb;
    nb.init(g, x, y, z);
#pragma unroll
    for (int i = 0; i < 27; ++i) {
      const S v = *canon_addr<S>((S*)b0, (S*)b1, g, nb, scheme, parity, i);
      out[i * ld + k] = wgt(i) + Codec<S>::to_delta(v, i);
    }
  }
}

template <typename S>
__global__ void set_kernel(S* b0, S* b1, Geo g, int scheme, int parity, const double* in,
                           uint64_t n0, uint64_t cnt, uint64_t ld) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < cnt;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x, y, z;
    node_coords(g, n0 + k, x, y, z);
    Nbr nb;
    nb.init(g, x, y, z);
#pragma unroll
    for (int i = 0; i < 27; ++i)
      *canon_addr<S>(b0, b1, g, nb, scheme, parity, i) =
          Codec<S>::from_delta(in[i * ld + k] - wgt(i), i);
  }
}

// rho and rho u of canonical f(t) at one node, accumulated in FP64 from the shifts
template <typename S>
__device__ __forceinline__ void node_moments(const S* b0, const S* b1, const Geo& g,
                                             const Nbr& nb, int scheme, int parity, double& rho,
                                             double (&m)[3]) {
  double s = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
#pragma unroll
  for (int i = 0; i < 27; ++i) {
    const double dv = Codec<S>::to_delta(*canon_addr<S>((S*)b0, (S*)b1, g, nb, scheme, parity, i), i);
    s += dv;
    if (cx(i)) mx += cx(i) * dv;
    if (cy(i)) my += cy(i) * dv;
    if (cz(i)) mz += cz(i) * dv;
  }
  rho = 1.0 + s;
  m[0] = mx;
  m[1] = my;
  m[2] = mz;
}

template <typename S>
__global__ void moments_kernel(const S* b0, const S* b1, Geo g, int scheme, int parity,
                               double* rho_out, double* u_out, uint64_t n0, uint64_t cnt,
                               uint64_t ld) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < cnt;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x, y, z;
    node_coords(g, n0 + k, x, y, z);
    Nbr nb;
    nb.init(g, x, y, z);
    double rho, m[3];
    node_moments<S>(b0, b1, g, nb, scheme, parity, rho, m);
    if (rho_out) rho_out[k] = rho;
    for (int a = 0; a < 3; ++a) u_out[a * ld + k] = m[a] / rho;
  }
}

// ------------------------------------------------------------------ diagnostics
// Sums (FP64) in partials[block * kDiagSums + j]:
//  0 sum rho, 1-3 sum rho u, 4-6 sum u, 7 sum |u|^2, 8 sum gamma, 9 sum gamma^2,
//  10 non-finite nodes, 11 sum |curl u|^2, 12 sum (d_b u_a + d_a u_b)^2,
//  13-17 sum (d u_x / d x)^n for n = 2..6
template <int N>
__device__ __forceinline__ void block_reduce_store(double (&v)[N], double* dst) {
  __shared__ double sh[32][N];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < N; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
  }
  if (lane == 0)
    for (int j = 0; j < N; ++j) sh[warp][j] = v[j];
  __syncthreads();
  if (threadIdx.x < N) {
    double acc = 0.0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) acc += sh[w][threadIdx.x];
    dst[threadIdx.x] = acc;
  }
}

// rho and rho u of canonical f(t) at one node in the arithmetic type of the storage
template <typename S>
__device__ __forceinline__ void node_moments_r(const S* b0, const S* b1, const Geo& g,
                                               const Nbr& nb, int scheme, int parity,
                                               typename Codec<S>::R& rho,
                                               typename Codec<S>::R (&m)[3]) {
  using R = typename Codec<S>::R;
  R s = R(0), mx = R(0), my = R(0), mz = R(0);
#pragma unroll
  for (int i = 0; i < 27; ++i) {
    const R dv = (R)Codec<S>::to_delta(*canon_addr<S>((S*)b0, (S*)b1, g, nb, scheme, parity, i), i);
    s += dv;
    if (cx(i)) mx += cx(i) * dv;
    if (cy(i)) my += cy(i) * dv;
    if (cz(i)) mz += cz(i) * dv;
  }
  rho = R(1) + s;
  m[0] = mx;
  m[1] = my;
  m[2] = mz;
}

// Per-node quantities in the storage's arithmetic type; per-thread and global sums in FP64.
template <typename S>
__global__ void __launch_bounds__(256) diag_fields_kernel(const S* b0, const S* b1, Geo g,
                                                          int scheme, int parity,
                                                          const float* gamma, int with_gamma,
                                                          typename Codec<S>::R* uf,
                                                          double* partials) {
  using R = typename Codec<S>::R;
  double v[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (uint64_t n = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; n < g.P;
       n += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x, y, z;
    node_coords(g, n, x, y, z);
    Nbr nb;
    nb.init(g, x, y, z);
    R rho, m[3];
    node_moments_r<S>(b0, b1, g, nb, scheme, parity, rho, m);
    const R ir = R(1) / rho;
    const R ux = m[0] * ir, uy = m[1] * ir, uz = m[2] * ir;
    uf[n] = ux;
    uf[g.P + n] = uy;
    uf[2 * g.P + n] = uz;
    if (!isfinite(rho) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz)) {
      v[10] += 1.0;
      continue;
    }
    v[0] += (double)rho;
    v[1] += (double)m[0];
    v[2] += (double)m[1];
    v[3] += (double)m[2];
    v[4] += (double)ux;
    v[5] += (double)uy;
    v[6] += (double)uz;
    v[7] += (double)(ux * ux + uy * uy + uz * uz);
    if (with_gamma) {
      const double gm = gamma[n];
      v[8] += gm;
      v[9] += gm * gm;
    }
  }
  block_reduce_store<11>(v, partials + blockIdx.x * kDiagSums);
}

// central-difference coefficients c_k of d u / d x = sum_k c_k (u(x + k) - u(x - k)):
// second order (K = 1) and eighth order (K = 4)
template <int K> struct FdCoef;
template <> struct FdCoef<1> {
  static __device__ __forceinline__ double c(int) { return 0.5; }
};
template <> struct FdCoef<4> {
  static __device__ __forceinline__ double c(int k) {
    return k == 1 ? 4.0 / 5.0 : k == 2 ? -1.0 / 5.0 : k == 3 ? 4.0 / 105.0 : -1.0 / 280.0;
  }
};

template <typename R, int K>
__global__ void __launch_bounds__(256) diag_grad_kernel(Geo g, const R* uf, double* partials) {
  double v[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const uint32_t dims[3] = {g.nx, g.ny, g.nz};
  for (uint64_t n = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; n < g.P;
       n += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t c[3];
    node_coords(g, n, c[0], c[1], c[2]);
    R gr[3][3];  // gr[a][b] = d u_a / d x_b
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) gr[a][b] = R(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const uint64_t stride = b == 0 ? 1 : b == 1 ? g.nx : g.nxy;
#pragma unroll
      for (int k = 1; k <= K; ++k) {
        // periodic neighbours c_b + k and c_b - k (k <= 4 may wrap more than once for tiny boxes)
        const uint32_t cp = (c[b] + k) % dims[b];
        const uint32_t cm = (c[b] + 4u * dims[b] - k) % dims[b];
        const uint64_t np = n + ((int64_t)cp - (int64_t)c[b]) * (int64_t)stride;
        const uint64_t nm = n + ((int64_t)cm - (int64_t)c[b]) * (int64_t)stride;
        const R ck = (R)FdCoef<K>::c(k);
#pragma unroll
        for (int a = 0; a < 3; ++a) gr[a][b] += ck * (uf[a * g.P + np] - uf[a * g.P + nm]);
      }
    }
    const R wx = gr[2][1] - gr[1][2], wy = gr[0][2] - gr[2][0], wz = gr[1][0] - gr[0][1];
    const R ww = wx * wx + wy * wy + wz * wz;
    R ss = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const R s = gr[a][b] + gr[b][a];
        ss += s * s;
      }
    if (isfinite(ww) && isfinite(ss)) {
      v[0] += (double)ww;
      v[1] += (double)ss;
      const double q = (double)gr[0][0];
      double qn = q * q;
#pragma unroll
      for (int m = 2; m <= 6; ++m) {
        v[m] += qn;
        qn *= q;
      }
    }
  }
  block_reduce_store<7>(v, partials + blockIdx.x * kDiagSums + 11);
}

// fixed-order final reduction: sums[j] = sum over blocks of partials[block][j]
static __global__ void diag_final_kernel(const double* partials, int nblocks, double* sums) {
  const int j = threadIdx.x;
  if (j >= kDiagSums) return;
  double acc = 0.0;
  for (int b = 0; b < nblocks; ++b) acc += partials[b * kDiagSums + j];
  sums[j] = acc;
}

// Stabilizer gap on canonical f(t): per node the estimate eq:result21 and the root of
// eq:result1 from the same collision inputs. Partial sums per block: [0] nodes evaluated,
// [1] sum |gamma_est - gamma*|, [2] sum gamma_est, [3] sum gamma*, [4] nodes where the Newton
// iteration did not converge, [5] nodes skipped (guarded or non-finite), [6] max |difference|.
constexpr int kGapSums = 7;
template <typename S, bool CENTRAL>
__global__ void __launch_bounds__(256) gap_kernel(const S* b0, const S* b1, Geo g, int scheme,
                                                  int parity, CollideParams cp,
                                                  double* partials) {
  using R = typename Codec<S>::R;
  double v[6] = {0, 0, 0, 0, 0, 0};
  double vmax = 0.0;
  for (uint64_t n = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; n < g.P;
       n += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x, y, z;
    node_coords(g, n, x, y, z);
    Nbr nb;
    nb.init(g, x, y, z);
    R d[27];
    Unroll<0, 27>::run([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      d[I] = Codec<S>::template load<I>(canon_addr<S>((S*)b0, (S*)b1, g, nb, scheme, parity, I));
    });
    int guarded, status = 1;
    R gest = R(0);
    const R gex = collide<R, CENTRAL, true>(d, cp, &guarded, &gest, &status);
    if (guarded || !(gex == gex) || !(gest == gest)) {
      v[5] += 1.0;
      continue;
    }
    const double diff = fabs((double)gex - (double)gest);
    v[0] += 1.0;
    v[1] += diff;
    v[2] += (double)gest;
    v[3] += (double)gex;
    if (status != 0) v[4] += 1.0;
    vmax = fmax(vmax, diff);
  }
  block_reduce_store<6>(v, partials + blockIdx.x * kDiagSums);
  // block maximum
  __shared__ double shm[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) shm[warp] = vmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) m = fmax(m, shm[w]);
    partials[blockIdx.x * kDiagSums + 6] = m;
  }
}

// fixed-order final reduction of the gap partials (slot 6 by maximum)
static __global__ void gap_final_kernel(const double* partials, int nblocks, double* sums) {
  const int j = threadIdx.x;
  if (j >= kGapSums) return;
  double acc = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    const double p = partials[b * kDiagSums + j];
    acc = j == 6 ? fmax(acc, p) : acc + p;
  }
  sums[j] = acc;
}

// ------------------------------------------------------------------ density pre-solve
// One iteration of the consistent-initialisation loop (Sec. "Numerical Simulations", after
// Mei et al.): f' = f - 2 beta_pre (f - f_eq(rho(f), u0(x))) with the velocity held at u0,
// streamed by the pattern of MODE. u0 is [3][P] in the collision precision. With `store`
// set, rho - 1 of the loaded state is kept in rho_prev (FP32) for rho_change_kernel.
template <typename S, int MODE>
__global__ void __launch_bounds__(MaxThreads<S>::value) presolve_kernel(
    const S* src, S* dst, Geo g, typename Codec<S>::R beta2, const typename Codec<S>::R* u0,
    float* rho_prev, int store) {
  using C = Codec<S>;
  using R = typename C::R;
  using Pat = Pattern<MODE>;
  const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t y = blockIdx.y * blockDim.y + threadIdx.y;
  const uint32_t z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  Nbr nb;
  nb.init(g, x, y, z);
  R d[27];
  Unroll<0, 27>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    d[I] = C::template load<I>(src + (uint64_t)Pat::load_plane(I) * g.P +
                               nb.template at<I, Pat::load_shift>());
  });
  R s = R(0);
#pragma unroll
  for (int i = 0; i < 27; ++i) s += d[i];
  const uint32_t n = nb.ox[1] + nb.oy[1] + nb.oz[1];
  R eq[27];
  equilibrium_shift<R>(R(1) + s, u0[n], u0[g.P + n], u0[2 * g.P + n], eq);
#pragma unroll
  for (int i = 0; i < 27; ++i) d[i] -= beta2 * (d[i] - eq[i]);
  Unroll<0, 27>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    C::template store<I>(dst + (uint64_t)Pat::store_plane(I) * g.P +
                             nb.template at<I, Pat::store_shift>(),
                         d[I]);
  });
  if (store) rho_prev[n] = (float)s;
}

// *resid = max over nodes of |(rho - 1) of canonical f(t) - rho_prev| in FP32 (as the bits of
// a non-negative float, so that atomicMax orders them); NaN is raised to +Inf.
template <typename S>
__global__ void __launch_bounds__(256) rho_change_kernel(const S* b0, const S* b1, Geo g,
                                                          int scheme, int parity,
                                                          const float* rho_prev,
                                                          unsigned int* resid) {
  using R = typename Codec<S>::R;
  float m = 0.0f;
  for (uint64_t n = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; n < g.P;
       n += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x, y, z;
    node_coords(g, n, x, y, z);
    Nbr nb;
    nb.init(g, x, y, z);
    // rho - 1 summed as presolve_kernel sums it, so that a fixed point gives exactly 0
    R d[27];
    Unroll<0, 27>::run([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      d[I] = Codec<S>::template load<I>(canon_addr<S>((S*)b0, (S*)b1, g, nb, scheme, parity, I));
    });
    R s = R(0);
#pragma unroll
    for (int i = 0; i < 27; ++i) s += d[i];
    float ch = fabsf((float)s - rho_prev[n]);
    if (!(ch == ch)) ch = INFINITY;
    m = fmaxf(m, ch);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(resid, __float_as_uint(m));
}

// ufield[a * P + n0 + k] = (R) u[a * ld + k]
template <typename R>
__global__ void convert_u_kernel(const double* u, R* ufield, uint64_t n0, uint64_t cnt,
                                 uint64_t ld, uint64_t P) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < cnt;
       k += (uint64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < 3; ++a) ufield[a * P + n0 + k] = (R)u[a * ld + k];
  }
}

// ------------------------------------------------------------------ host launchers
inline Geo make_geo(const BoxView& b) {
  Geo g;
  g.nx = b.nx;
  g.ny = b.ny;
  g.nz = b.nz;
  g.nxy = b.nx * b.ny;
  g.P = b.P;
  return g;
}

inline CollideParams make_cp(double beta, int with_t, int with_q, int gamma_mode) {
  CollideParams cp;
  cp.beta = beta;
  cp.two_beta = 2.0 * beta;
  cp.inv_beta = 1.0 / beta;
  cp.betaf = (float)cp.beta;
  cp.two_betaf = (float)cp.two_beta;
  cp.inv_betaf = (float)cp.inv_beta;
  cp.with_t = with_t;
  cp.with_q = with_q;
  cp.gamma_mode = gamma_mode;
  return cp;
}

inline int grid_for(uint64_t cnt, int threads) {
  uint64_t blocks = (cnt + threads - 1) / threads;
  const uint64_t cap = 152ull * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

template <typename S, int MODE, bool RECORD, bool CENTRAL>
static cudaError_t launch_step_c(const BoxView& b, const S* src, S* dst, const Geo& g,
                                 const CollideParams& cp, const StepOpts& o, StepCounters* ctr,
                                 cudaStream_t st) {
  if (cp.gamma_mode == GAMMA_EXACT) {  // one node per thread, whatever kernel was chosen
    const dim3 block(o.bx, o.by, 1);
    const dim3 grid((b.nx + o.bx - 1) / o.bx, (b.ny + o.by - 1) / o.by, b.nz);
    step_kernel<S, MODE, RECORD, CENTRAL, true><<<grid, block, 0, st>>>(src, dst, g, cp, b.gamma,
                                                                        ctr);
    return cudaGetLastError();
  }
  if constexpr (!CENTRAL) {
    if (o.kernel == KERNEL_STAGED)
      return launch_staged<S, MODE, RECORD>(src, dst, g, cp, b.gamma, ctr, o.budget, o.stall, st);
    if (o.kernel == KERNEL_PERSISTENT)
      return launch_persistent<S, MODE, RECORD>(src, dst, g, cp, b.gamma, ctr,
                                                (uint32_t)o.prefetch, st);
  }
  if constexpr (!std::is_same<S, double>::value) {
    if (o.kernel == KERNEL_PACKED || o.kernel == KERNEL_AUTO)
      return launch_pair<S, MODE, RECORD, CENTRAL>(src, dst, g, cp, b.gamma, ctr, st);
  }
  const dim3 block(o.bx, o.by, 1);
  const dim3 grid((b.nx + o.bx - 1) / o.bx, (b.ny + o.by - 1) / o.by, b.nz);
  step_kernel<S, MODE, RECORD, CENTRAL><<<grid, block, 0, st>>>(src, dst, g, cp, b.gamma, ctr);
  return cudaGetLastError();
}

template <typename S, int MODE, bool RECORD>
static cudaError_t launch_step(const BoxView& b, const S* src, S* dst, const Geo& g,
                               const CollideParams& cp, const StepOpts& o, StepCounters* ctr,
                               cudaStream_t st) {
  if (b.central)
    return launch_step_c<S, MODE, RECORD, true>(b, src, dst, g, cp, o, ctr, st);
  return launch_step_c<S, MODE, RECORD, false>(b, src, dst, g, cp, o, ctr, st);
}

template <typename S>
bool Ops<S>::staged_ok(uint32_t nx) {
  return staged_supported<S>(nx);
}

template <typename S>
cudaError_t Ops<S>::step(const BoxView& b, int64_t t, bool record, const StepOpts& o,
                         StepCounters* counters, cudaStream_t st) {
  const Geo g = make_geo(b);
  const CollideParams cp = make_cp(b.beta, b.with_t, b.with_q, b.gamma_mode);
  const int parity = (int)(t & 1);
  if (b.scheme == 0) {
    const S* src = (const S*)b.pop[parity];
    S* dst = (S*)b.pop[parity ^ 1];
    return record ? launch_step<S, MODE_PULL, true>(b, src, dst, g, cp, o, counters, st)
                  : launch_step<S, MODE_PULL, false>(b, src, dst, g, cp, o, counters, st);
  }
  S* buf = (S*)b.pop[0];
  if (parity == 0)
    return record ? launch_step<S, MODE_AA_EVEN, true>(b, buf, buf, g, cp, o, counters, st)
                  : launch_step<S, MODE_AA_EVEN, false>(b, buf, buf, g, cp, o, counters, st);
  return record ? launch_step<S, MODE_AA_ODD, true>(b, buf, buf, g, cp, o, counters, st)
                : launch_step<S, MODE_AA_ODD, false>(b, buf, buf, g, cp, o, counters, st);
}

template <typename S>
cudaError_t Ops<S>::init(const BoxView& b, int64_t t, const double* rho, const double* u,
                         uint64_t n0, uint64_t cnt, uint64_t ld, cudaStream_t st) {
  init_kernel<S><<<grid_for(cnt, 256), 256, 0, st>>>((S*)b.pop[0], (S*)b.pop[1], make_geo(b),
                                                     b.scheme, (int)(t & 1), rho, u, n0, cnt, ld);
  return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::get(const BoxView& b, int64_t t, double* out, uint64_t n0, uint64_t cnt,
                        uint64_t ld, cudaStream_t st) {
  get_kernel<S><<<grid_for(cnt, 256), 256, 0, st>>>((const S*)b.pop[0], (const S*)b.pop[1],
                                                    make_geo(b), b.scheme, (int)(t & 1), out, n0,
                                                    cnt, ld);
  return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::set(const BoxView& b, int64_t t, const double* in, uint64_t n0,
                        uint64_t cnt, uint64_t ld, cudaStream_t st) {
  set_kernel<S><<<grid_for(cnt, 256), 256, 0, st>>>((S*)b.pop[0], (S*)b.pop[1], make_geo(b),
                                                    b.scheme, (int)(t & 1), in, n0, cnt, ld);
  return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::moments(const BoxView& b, int64_t t, double* rho, double* u, uint64_t n0,
                            uint64_t cnt, uint64_t ld, cudaStream_t st) {
  moments_kernel<S><<<grid_for(cnt, 256), 256, 0, st>>>((const S*)b.pop[0], (const S*)b.pop[1],
                                                        make_geo(b), b.scheme, (int)(t & 1), rho,
                                                        u, n0, cnt, ld);
  return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::presolve_step(const BoxView& b, int64_t t, double beta_pre, const void* u0,
                                  bool store, const StepOpts& o, cudaStream_t st) {
  using R = typename Codec<S>::R;
  const Geo g = make_geo(b);
  const R beta2 = (R)(2.0 * beta_pre);
  const dim3 block(o.bx, o.by, 1);
  const dim3 grid((b.nx + o.bx - 1) / o.bx, (b.ny + o.by - 1) / o.by, b.nz);
  const int parity = (int)(t & 1);
  const R* u = (const R*)u0;
  if (b.scheme == 0)
    presolve_kernel<S, MODE_PULL><<<grid, block, 0, st>>>(
        (const S*)b.pop[parity], (S*)b.pop[parity ^ 1], g, beta2, u, b.gamma, store ? 1 : 0);
  else if (parity == 0)
    presolve_kernel<S, MODE_AA_EVEN><<<grid, block, 0, st>>>(
        (const S*)b.pop[0], (S*)b.pop[0], g, beta2, u, b.gamma, store ? 1 : 0);
  else
    presolve_kernel<S, MODE_AA_ODD><<<grid, block, 0, st>>>(
        (const S*)b.pop[0], (S*)b.pop[0], g, beta2, u, b.gamma, store ? 1 : 0);
  return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::rho_change(const BoxView& b, int64_t t, unsigned int* resid, int nblocks,
                               cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(resid, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  rho_change_kernel<S><<<nblocks, 256, 0, st>>>((const S*)b.pop[0], (const S*)b.pop[1],
                                                make_geo(b), b.scheme, (int)(t & 1), b.gamma,
                                                resid);
  return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::convert_u(const double* u, void* ufield, uint64_t n0, uint64_t cnt,
                              uint64_t ld, uint64_t P, cudaStream_t st) {
  using R = typename Codec<S>::R;
  convert_u_kernel<R><<<grid_for(cnt, 256), 256, 0, st>>>(u, (R*)ufield, n0, cnt, ld, P);
  return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::gamma_gap(const BoxView& b, int64_t t, double* partials, int nblocks,
                              double* sums, cudaStream_t st) {
  const Geo g = make_geo(b);
  CollideParams cp = make_cp(b.beta, b.with_t, b.with_q, GAMMA_EXACT);
  if (b.central)
    gap_kernel<S, true><<<nblocks, 256, 0, st>>>((const S*)b.pop[0], (const S*)b.pop[1], g,
                                                 b.scheme, (int)(t & 1), cp, partials);
  else
    gap_kernel<S, false><<<nblocks, 256, 0, st>>>((const S*)b.pop[0], (const S*)b.pop[1], g,
                                                  b.scheme, (int)(t & 1), cp, partials);
  gap_final_kernel<<<1, 32, 0, st>>>(partials, nblocks, sums);
  return cudaGetLastError();
}

template <typename S>
cudaError_t Ops<S>::diag(const BoxView& b, int64_t t, bool with_gamma, int order, void* ufield,
                         double* partials, int nblocks, double* sums, cudaStream_t st) {
  using R = typename Codec<S>::R;
  const Geo g = make_geo(b);
  cudaMemsetAsync(partials, 0, sizeof(double) * kDiagSums * nblocks, st);
  diag_fields_kernel<S><<<nblocks, 256, 0, st>>>((const S*)b.pop[0], (const S*)b.pop[1], g,
                                                 b.scheme, (int)(t & 1), b.gamma,
                                                 with_gamma ? 1 : 0, (R*)ufield, partials);
  if (order == 8)
    diag_grad_kernel<R, 4><<<nblocks, 256, 0, st>>>(g, (const R*)ufield, partials);
  else
    diag_grad_kernel<R, 1><<<nblocks, 256, 0, st>>>(g, (const R*)ufield, partials);
  diag_final_kernel<<<1, 32, 0, st>>>(partials, nblocks, sums);
  return cudaGetLastError();
}

template <typename S, int MODE, bool CENTRAL>
static void launch_batch_c(const BoxDesc* boxes, const WorkItem* items, int nitems, int parity,
                           bool record, bool packed, int with_t, int with_q, int gamma_mode,
                           int threads, int grid, cudaStream_t st) {
  if constexpr (!std::is_same<S, double>::value) {
    if (packed) {
      if (record)
        batch_pair_kernel<S, MODE, true, CENTRAL><<<grid, 128, 0, st>>>(
            boxes, items, nitems, parity, with_t, with_q, gamma_mode);
      else
        batch_pair_kernel<S, MODE, false, CENTRAL><<<grid, 128, 0, st>>>(
            boxes, items, nitems, parity, with_t, with_q, gamma_mode);
      return;
    }
  }
  if (record)
    batch_kernel<S, MODE, true, CENTRAL><<<grid, threads, 0, st>>>(boxes, items, nitems, parity,
                                                                   with_t, with_q, gamma_mode);
  else
    batch_kernel<S, MODE, false, CENTRAL><<<grid, threads, 0, st>>>(boxes, items, nitems, parity,
                                                                    with_t, with_q, gamma_mode);
}

template <typename S, int MODE>
static void launch_batch(const BoxDesc* boxes, const WorkItem* items, int nitems, int parity,
                         bool record, bool packed, bool central, int with_t, int with_q,
                         int gamma_mode, int threads, int grid, cudaStream_t st) {
  if (central)
    launch_batch_c<S, MODE, true>(boxes, items, nitems, parity, record, packed, with_t, with_q,
                                  gamma_mode, threads, grid, st);
  else
    launch_batch_c<S, MODE, false>(boxes, items, nitems, parity, record, packed, with_t, with_q,
                                   gamma_mode, threads, grid, st);
}

template <typename S>
cudaError_t Ops<S>::batch_step(const BoxDesc* boxes, const WorkItem* items, int nitems,
                               int64_t t, bool record, bool packed, int scheme, int with_t,
                               int with_q, int central, int gamma_mode, int threads, int grid,
                               cudaStream_t st) {
  const int parity = (int)(t & 1);
  if (scheme == 0)
    launch_batch<S, MODE_PULL>(boxes, items, nitems, parity, record, packed, central, with_t,
                               with_q, gamma_mode, threads, grid, st);
  else if (parity == 0)
    launch_batch<S, MODE_AA_EVEN>(boxes, items, nitems, parity, record, packed, central, with_t,
                                  with_q, gamma_mode, threads, grid, st);
  else
    launch_batch<S, MODE_AA_ODD>(boxes, items, nitems, parity, record, packed, central, with_t,
                                 with_q, gamma_mode, threads, grid, st);
  return cudaGetLastError();
}

template <typename S>
int Ops<S>::batch_occupancy(int threads, int scheme, bool packed) {
  int blocks = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if constexpr (!std::is_same<S, double>::value) {
    if (packed) {
      if (scheme == 0)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &blocks, batch_pair_kernel<S, MODE_PULL, false, false>, 128, 0);
      else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &blocks, batch_pair_kernel<S, MODE_AA_ODD, false, false>, 128, 0);
      if (e != cudaSuccess || blocks < 1) blocks = 1;
      return blocks;
    }
  }
  if (scheme == 0)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, batch_kernel<S, MODE_PULL, false, false>,
                                                      threads, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks,
                                                      batch_kernel<S, MODE_AA_ODD, false, false>,
                                                      threads, 0);
  if (e != cudaSuccess || blocks < 1) blocks = 1;
  return blocks;
}

}  // namespace kbc
