// kbc_aux.cuh -- kernels around the step: canonical-state transfer (init, get, set, moments),
// diagnostics, the stabilizer gap and the density pre-solve, with their Ops<S> launchers.
//
// Included at the end of kbc_kernels.cuh (it uses the step kernels' device code and host
// helpers); kept apart so that the step kernels' sources stay separate from these.
#pragma once

namespace kbc {
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

// (32-bit arithmetic: a box holds fewer than 2^31 nodes; a 64-bit division would be a long
// software sequence)
__device__ __forceinline__ void node_coords(const Geo& g, uint64_t n, uint32_t& x, uint32_t& y,
                                            uint32_t& z) {
  const uint32_t m = (uint32_t)n;
  z = m / g.nxy;
  const uint32_t r = m - z * g.nxy;
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
// Sums (FP64) in partials[block * kDiagSums + j], over the nodes whose rho and u are finite
// (0-10) or whose velocity gradients are finite (11-19):
//  0 sum (rho - 1), 1-3 sum rho u, 4-6 sum u, 7 sum |u|^2, 8 sum gamma, 9 sum gamma^2,
//  10 non-finite nodes, 11 sum |curl u|^2, 12 sum (d_b u_a + d_a u_b)^2,
//  13-17 sum (d u_x / d x)^n for n = 2..6, 18 sum |u - <u>|^2 (second pass, with <u> from the
//  first), 19 nodes with finite gradients
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

// Address of canonical f_I(node, t) for a compile-time layout: KIND 0 pull (buf = the buffer
// of parity t), 1 AA at even t, 2 AA at odd t (buf = the one AA buffer).
template <int KIND, int I, typename S>
__device__ __forceinline__ const S* canon_ptr(const S* buf, const Geo& g, const Nbr& nb) {
  if constexpr (KIND == 1) return buf + (uint64_t)I * g.P + nb.template at<I, 0>();
  else if constexpr (KIND == 0) return buf + (uint64_t)I * g.P + nb.template at<I, -1>();
  else return buf + (uint64_t)(26 - I) * g.P + nb.template at<I, -1>();
}

// rho - 1 and rho u of canonical f(t) at one node, in the arithmetic type of the storage
template <typename S, int KIND>
__device__ __forceinline__ void node_moments_r(const S* buf, const Geo& g, const Nbr& nb,
                                               typename Codec<S>::R& drho,
                                               typename Codec<S>::R (&m)[3]) {
  using R = typename Codec<S>::R;
  R s = R(0), mx = R(0), my = R(0), mz = R(0);
  Unroll<0, 27>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    const R dv = Codec<S>::template load<I>(canon_ptr<KIND, I>(buf, g, nb));
    s += dv;
    if constexpr (cx(I) != 0) mx += R(cx(I)) * dv;
    if constexpr (cy(I) != 0) my += R(cy(I)) * dv;
    if constexpr (cz(I) != 0) mz += R(cz(I)) * dv;
  });
  drho = s;
  m[0] = mx;
  m[1] = my;
  m[2] = mz;
}

// Per-node quantities in the storage's arithmetic type; block and global sums in FP64.
// 4 blocks of 256 threads per SM: the fixed grid of 608 blocks is then resident in one wave
template <typename S, int KIND>
__global__ void __launch_bounds__(256, 4) diag_fields_kernel(const S* buf, Geo g,
                                                          const float* gamma, int with_gamma,
                                                          typename Codec<S>::R* uf,
                                                          double* partials) {
  using R = typename Codec<S>::R;
  // per-thread sums in R (FP64 arithmetic per node would saturate GB300's FP64 pipe); the
  // density enters as rho - 1 so that FP32 sums keep their relative accuracy
  R acc[11] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
  for (uint64_t n = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; n < g.P;
       n += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x, y, z;
    node_coords(g, n, x, y, z);
    Nbr nb;
    nb.init(g, x, y, z);
    R drho, m[3];
    node_moments_r<S, KIND>(buf, g, nb, drho, m);
    const R rho = R(1) + drho;
    const R ir = R(1) / rho;
    const R ux = m[0] * ir, uy = m[1] * ir, uz = m[2] * ir;
    uf[n] = ux;
    uf[g.P + n] = uy;
    uf[2 * g.P + n] = uz;
    if (!isfinite(rho) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz)) {
      acc[10] += R(1);
      continue;
    }
    acc[0] += drho;
    acc[1] += m[0];
    acc[2] += m[1];
    acc[3] += m[2];
    acc[4] += ux;
    acc[5] += uy;
    acc[6] += uz;
    acc[7] += ux * ux + uy * uy + uz * uz;
    if (with_gamma) {
      const R gm = (R)gamma[n];
      acc[8] += gm;
      acc[9] += gm * gm;
    }
  }
  double v[11];
#pragma unroll
  for (int j = 0; j < 11; ++j) v[j] = (double)acc[j];
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

// Per-thread sums in the arithmetic type R (a thread covers about P / 155,648 nodes, ~100 at
// 256^3; FP64 arithmetic per node would saturate GB300's FP64 pipe), then FP64 from the
// block reduction on.
template <typename R, int K>
__global__ void __launch_bounds__(256) diag_grad_kernel(Geo g, const R* uf, const double* sums,
                                                        double* partials) {
  R acc[9] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
  const uint32_t dims[3] = {g.nx, g.ny, g.nz};
  // <u> over the finite nodes, from the sums of the first pass
  const double nfin = (double)g.P - sums[10];
  const R mean[3] = {(R)(sums[4] / nfin), (R)(sums[5] / nfin), (R)(sums[6] / nfin)};
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
      const int64_t stride = b == 0 ? 1 : b == 1 ? (int64_t)g.nx : (int64_t)g.nxy;
      const int64_t dim = dims[b];
      // periodic neighbours c_b + k and c_b - k, stepped one node at a time so that each
      // step wraps at most once (the stencil may go round a 3-node box more than once)
      int64_t cp = c[b], cm = c[b];
#pragma unroll
      for (int k = 1; k <= K; ++k) {
        ++cp;
        if (cp >= dim) cp -= dim;
        --cm;
        if (cm < 0) cm += dim;
        const uint64_t np = n + (cp - (int64_t)c[b]) * stride;
        const uint64_t nm = n + (cm - (int64_t)c[b]) * stride;
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
      acc[0] += ww;
      acc[1] += ss;
      const R q = gr[0][0];
      R qn = q * q;
#pragma unroll
      for (int m = 2; m <= 6; ++m) {
        acc[m] += qn;
        qn *= q;
      }
      acc[8] += R(1);
    }
    const R d0 = uf[n] - mean[0], d1 = uf[g.P + n] - mean[1], d2 = uf[2 * g.P + n] - mean[2];
    const R dd = d0 * d0 + d1 * d1 + d2 * d2;
    if (isfinite(dd)) acc[7] += dd;
  }
  double v[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) v[j] = (double)acc[j];
  block_reduce_store<9>(v, partials + blockIdx.x * kDiagSums + 11);
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
  const int parity = (int)(t & 1);
  const int wg = with_gamma ? 1 : 0;
  if (b.scheme == 0)
    diag_fields_kernel<S, 0><<<nblocks, 256, 0, st>>>((const S*)b.pop[parity], g, b.gamma, wg,
                                                      (R*)ufield, partials);
  else if (parity == 0)
    diag_fields_kernel<S, 1><<<nblocks, 256, 0, st>>>((const S*)b.pop[0], g, b.gamma, wg,
                                                      (R*)ufield, partials);
  else
    diag_fields_kernel<S, 2><<<nblocks, 256, 0, st>>>((const S*)b.pop[0], g, b.gamma, wg,
                                                      (R*)ufield, partials);
  diag_final_kernel<<<1, 32, 0, st>>>(partials, nblocks, sums);  // <u> for the second pass
  if (order == 8)
    diag_grad_kernel<R, 4><<<nblocks, 256, 0, st>>>(g, (const R*)ufield, sums, partials);
  else
    diag_grad_kernel<R, 1><<<nblocks, 256, 0, st>>>(g, (const R*)ufield, sums, partials);
  diag_final_kernel<<<1, 32, 0, st>>>(partials, nblocks, sums);
  return cudaGetLastError();
}

}  // namespace kbc
