// kbc_device.cuh -- device-side building blocks of the D3Q27 KBC step (sm_103a).
//
// Method: arXiv:1507.02518, Sec. KBC (eq:Egeneral with eq:ksh-mirror, Table 1, eq:result21) with the
// product-form equilibrium eq:entropic_eq and the natural moments eq:natmoments.
//
// Register-level design (one thread = one lattice node):
//   * the 27 populations are held as the shift delta_i = f_i - W_i (storage codec below);
//   * natural moments come from a factorised x -> y -> z reduction of delta;
//   * the equilibrium is carried per axis: phi(v) = W_v (1 + e_v) with e_0 = -(R-1),
//     e_{+-1} = 2(R-1) +- 3u, R = sqrt(1 + 3u^2) -- the 1D closed form of eq:entropic_eq
//     (W_1 A(u) B(u) = (2R - 1 + 3u)/6, W_0 A(u) = 2(2 - R)/3), so f_eq - W and 1/f_eq are
//     built from 9 per-axis factors without cancellation;
//   * Table 1 is applied to the moment deviations M - M_eq (M_eq_pqr = m_p(ux) m_q(uy) m_r(uz),
//     m_0 = 1, m_1 = u, m_2 = (2R - 1)/3), scaled by rho;
//   * the entropic scalar products (Sec. KBC) use the factorised weights 1/f_eq_i =
//     rx(a) ry(b) rz(c).
#pragma once

#include <cuda_fp16.h>
#include <string.h>
#include <stdint.h>

#include <type_traits>

#include "kbc_ops.h"

namespace kbc {

// ------------------------------------------------------------------ lattice constants
// i = (vx+1) + 3(vy+1) + 9(vz+1); weights W_i = W_vx W_vy W_vz, W_0 = 2/3, W_+-1 = 1/6
// (eq:weights, eq:sound).
__host__ __device__ constexpr int cx(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy(int i) { return (i / 3) % 3 - 1; }
__host__ __device__ constexpr int cz(int i) { return i / 9 - 1; }
__host__ __device__ constexpr double w1(int v) { return v == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
__host__ __device__ constexpr double wgt(int i) { return w1(cx(i)) * w1(cy(i)) * w1(cz(i)); }
// 1/W_i is exact in binary: 27/8, 27/2, 54, 216
__host__ __device__ constexpr double inv_wgt(int i) {
  return (1.0 / w1(cx(i))) * (1.0 / w1(cy(i))) * (1.0 / w1(cz(i)));
}
__host__ __device__ constexpr int opp(int i) { return 26 - i; }

// ------------------------------------------------------------------ storage codecs
// Each storage type S maps to an arithmetic type R and encodes the shift delta = f - W.
// load/store give and take the shift itself (diagnostics, transfers, pre-solve). The step
// kernels use load_raw/store_raw, whose unit is the collision's: the shift for FP64 and FP32,
// and the shift relative to the weight, (f - W)/W, for FP16 (rel = true), so that no
// per-population scaling sits between the stored halves and the collision (the collision
// folds the weights into its constants).
template <typename S> struct Codec;

template <> struct Codec<double> {
  using R = double;
  static constexpr bool rel = false;
  template <int I> __device__ static __forceinline__ R load(const double* p) { return *p; }
  template <int I> __device__ static __forceinline__ R load_ro(const double* p) { return __ldg(p); }
  template <int I> __device__ static __forceinline__ void store(double* p, R d) { *p = d; }
  template <int I> __device__ static __forceinline__ R load_raw(const double* p) { return *p; }
  template <int I> __device__ static __forceinline__ R load_raw_ro(const double* p) {
    return __ldg(p);
  }
  template <int I> __device__ static __forceinline__ void store_raw(double* p, R d) { *p = d; }
  __host__ __device__ static double to_delta(double s, int) { return s; }
  __host__ __device__ static double from_delta(double d, int) { return d; }
};

template <> struct Codec<float> {
  using R = float;
  static constexpr bool rel = false;
  template <int I> __device__ static __forceinline__ R load(const float* p) { return *p; }
  template <int I> __device__ static __forceinline__ R load_ro(const float* p) { return __ldg(p); }
  template <int I> __device__ static __forceinline__ void store(float* p, R d) { *p = d; }
  template <int I> __device__ static __forceinline__ R load_raw(const float* p) { return *p; }
  template <int I> __device__ static __forceinline__ R load_raw_ro(const float* p) {
    return __ldg(p);
  }
  template <int I> __device__ static __forceinline__ void store_raw(float* p, R d) { *p = d; }
  __device__ static double to_delta(float s, int) { return (double)s; }
  __device__ static float from_delta(double d, int) { return (float)d; }
};

// FP16: the stored half is (f_i - W_i) / W_i, rounded to nearest even. Keeping the value
// relative to W_i keeps every direction clear of the half subnormal range.
template <> struct Codec<uint16_t> {
  using R = float;
  static constexpr bool rel = true;
  template <int I> __device__ static __forceinline__ R load(const uint16_t* p) {
    return __fmul_rn((float)wgt(I), __half2float(__ushort_as_half(*p)));
  }
  template <int I> __device__ static __forceinline__ R load_ro(const uint16_t* p) {
    return __fmul_rn((float)wgt(I), __half2float(__ushort_as_half(__ldg(p))));
  }
  template <int I> __device__ static __forceinline__ void store(uint16_t* p, R d) {
    *p = __half_as_ushort(__float2half_rn(__fmul_rn(d, (float)inv_wgt(I))));
  }
  template <int I> __device__ static __forceinline__ R load_raw(const uint16_t* p) {
    return __half2float(__ushort_as_half(*p));
  }
  template <int I> __device__ static __forceinline__ R load_raw_ro(const uint16_t* p) {
    return __half2float(__ushort_as_half(__ldg(p)));
  }
  template <int I> __device__ static __forceinline__ void store_raw(uint16_t* p, R d) {
    *p = __half_as_ushort(__float2half_rn(d));
  }
  __device__ static double to_delta(uint16_t s, int i) {
    return wgt(i) * (double)__half2float(__ushort_as_half(s));
  }
  __device__ static uint16_t from_delta(double d, int i) {
    return __half_as_ushort(__double2half(d * inv_wgt(i)));
  }
};

// Two values of one plane (nodes a and b) at a time in the collision's unit (load_raw /
// store_raw above), for the packed kernels.
template <typename S> struct Codec2;
template <> struct Codec2<float> {
  template <int I, bool RO>
  __device__ static __forceinline__ float2 load(const float* pa, const float* pb) {
    return RO ? make_float2(__ldg(pa), __ldg(pb)) : make_float2(*pa, *pb);
  }
  template <int I> __device__ static __forceinline__ void store(float* pa, float* pb, bool va,
                                                              bool vb, float2 v) {
    if (va) *pa = v.x;
    if (vb) *pb = v.y;
  }
};
template <> struct Codec2<uint16_t> {
  template <int I, bool RO>
  __device__ static __forceinline__ float2 load(const uint16_t* pa, const uint16_t* pb) {
    const uint16_t a = RO ? __ldg(pa) : *pa, b = RO ? __ldg(pb) : *pb;
    return __half22float2(__halves2half2(__ushort_as_half(a), __ushort_as_half(b)));
  }
  template <int I> __device__ static __forceinline__ void store(uint16_t* pa, uint16_t* pb,
                                                              bool va, bool vb, float2 v) {
    const __half2 h = __float22half2_rn(v);
    if (va) *pa = __half_as_ushort(__low2half(h));
    if (vb) *pb = __half_as_ushort(__high2half(h));
  }
};

// Two adjacent nodes (x, x + 1) of one plane in the collision's unit, for the kernels that
// give a thread two neighbouring nodes of a row: v0, vl and vr point at the values of nodes x,
// x - 1 and x + 2 (row neighbours, periodic wrap already applied); SX selects the pair read,
// nodes (x + SX, x + 1 + SX). The unshifted pair is one 32-bit (FP16) or 64-bit (FP32) access
// (x even, rows of even length); a shifted pair is two scalar accesses. RO: read-only path.
template <typename S> struct PairIO;
template <> struct PairIO<uint16_t> {
  template <bool RO> __device__ static __forceinline__ uint16_t ld1(const uint16_t* p) {
    return RO ? __ldg(p) : *p;
  }
  template <int SX, bool RO>
  __device__ static __forceinline__ float2 get(const uint16_t* v0, const uint16_t* vl,
                                               const uint16_t* vr) {
    if constexpr (SX == 0) {
      const unsigned int w = RO ? __ldg(reinterpret_cast<const unsigned int*>(v0))
                                : *reinterpret_cast<const unsigned int*>(v0);
      __half2 h;
      memcpy(&h, &w, sizeof h);
      return __half22float2(h);
    } else if constexpr (SX < 0) {
      return __half22float2(
          __halves2half2(__ushort_as_half(ld1<RO>(vl)), __ushort_as_half(ld1<RO>(v0))));
    } else {
      return __half22float2(
          __halves2half2(__ushort_as_half(ld1<RO>(v0 + 1)), __ushort_as_half(ld1<RO>(vr))));
    }
  }
  __device__ static __forceinline__ void put2(uint16_t* p, float2 v) {
    *reinterpret_cast<__half2*>(p) = __float22half2_rn(v);
  }
  __device__ static __forceinline__ void put1(uint16_t* p, float v) {
    *p = __half_as_ushort(__float2half_rn(v));
  }
};
template <> struct PairIO<float> {
  template <bool RO> __device__ static __forceinline__ float ld1(const float* p) {
    return RO ? __ldg(p) : *p;
  }
  template <int SX, bool RO>
  __device__ static __forceinline__ float2 get(const float* v0, const float* vl,
                                               const float* vr) {
    if constexpr (SX == 0) {
      return RO ? __ldg(reinterpret_cast<const float2*>(v0))
                : *reinterpret_cast<const float2*>(v0);
    } else if constexpr (SX < 0) {
      return make_float2(ld1<RO>(vl), ld1<RO>(v0));
    } else {
      return make_float2(ld1<RO>(v0 + 1), ld1<RO>(vr));
    }
  }
  __device__ static __forceinline__ void put2(float* p, float2 v) {
    *reinterpret_cast<float2*>(p) = v;
  }
  __device__ static __forceinline__ void put1(float* p, float v) { *p = v; }
};

// guard on <dh|dh> (the paper is silent when it vanishes; gamma falls back to 2, LBGK)
template <typename R> struct Guard;
template <> struct Guard<double> { static constexpr double den = 1e-300; };
template <> struct Guard<float> { static constexpr float den = 1e-30f; };

// With FP32 storage, an FP32 collision whose <dh|dh> falls under kDenFp64 is not used: the
// lane is flagged (*fp64 bit k), the node's bit is set in the box's mask (flag_fp64), and a
// pass launched after the step kernel (fp64_pass_kernel) collides the node again in FP64
// from its inputs (fp64_node_update), with the FP64 guard of the oracle. The inputs are still
// in memory then: the pull step reads src only and stores the flagged node's FP32 outputs
// anyway (the pass overwrites them), the AA step does not store a flagged node (each AA node
// alone reads and writes its slots). The step kernels hold no call of the FP64 path, which
// would cost them registers. FP16 storage takes no FP64 path: its rounding of the stored
// populations (the step's output) exceeds the FP32 error of gamma near equilibrium. The
// FP32 dh carries an absolute error of about 1e-8 (relative to W_i): the round-off of the
// O(0.1) shifts it is the difference of. At <dh|dh> = 1e-13, |dh / W| ~ 3e-7, so the FP32
// denominator -- and the ratio of eq:result21 -- would be off by a few per cent below it, while
// at 1e-9 they are still good to 1e-3 (smooth fields at 512^3 have many nodes there, and
// collide them in FP32). An accurate denominator needs dh, and so the node's moments and
// equilibrium, in FP64.
constexpr float kDenFp64 = 1e-13f;

enum { GAMMA_ESTIMATE = 0, GAMMA_LBGK = 1, GAMMA_RLB = 2, GAMMA_EXACT = 3 };

struct CollideParams {
  double beta;      // relaxation parameter of eq:Egeneral
  double two_beta;  // 2 beta
  double inv_beta;  // 1 / beta
  float betaf, two_betaf, inv_betaf;  // the same, rounded once on the host for FP32 kernels
  int with_t;       // shear part includes t (Table 1)
  int with_q;       // shear part includes q (Table 1)
  int gamma_mode;   // GAMMA_*
};

// the parameter in the arithmetic precision (no FP64 conversion inside FP32 kernels)
template <typename T> __device__ __forceinline__ T prec(double d, float f);
template <> __device__ __forceinline__ double prec<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float prec<float>(double, float f) { return f; }

// Explicitly rounded arithmetic. Every operation of the collision goes through these, so the
// compiler does not contract them: the scalar kernels that inline collide<float|double>()
// (direct, staged, persistent, batched; pull and AA) produce bit-identical populations from
// identical inputs, which the tests check. Ar<float2> holds two nodes and uses the packed
// FP32x2 instructions of sm_100+; its results agree with the scalar path to FP32 round-off but
// not bit for bit (measured on GB300; both are equally close to an FP64 collision).

// single MUFU approximations (relative error about 2^-22 for normal inputs)
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <typename R> struct Ar;
template <> struct Ar<float> {
  using Scalar = float;
  static constexpr int lanes = 1;
  static __device__ __forceinline__ float c(double v) { return (float)v; }
  static __device__ __forceinline__ float bc(float v) { return v; }
  static __device__ __forceinline__ float neg(float a) { return -a; }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) {
    return __fmaf_rn(a, b, c);
  }
  // hardware-approximate forms (one MUFU instruction, then an explicitly rounded multiply)
  // where FP32 round-off is not the limit: the reciprocal weights of the entropic products,
  // 1/rho, R = sqrt(1 + 3u^2) >= 1, and the ratio of eq:result21
  static __device__ __forceinline__ float div_fast(float a, float b) {
    return __fmul_rn(a, rcp_approx(b));
  }
  static __device__ __forceinline__ float sqrt_fast(float a) {
    return __fmul_rn(a, rsqrt_approx(a));
  }
  static __device__ __forceinline__ float rcp_fast(float a) { return rcp_approx(a); }
  static __device__ __forceinline__ float lane(float a, int) { return a; }
  static __device__ __forceinline__ void set_lane(float& a, int, float v) { a = v; }
};
template <> struct Ar<float2> {
  using Scalar = float;
  static constexpr int lanes = 2;
  static __device__ __forceinline__ float2 c(double v) { return make_float2((float)v, (float)v); }
  static __device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }
  static __device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ float2 sub(float2 a, float2 b) {
    return __fadd2_rn(a, neg(b));
  }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) {
    return __ffma2_rn(a, b, c);
  }
  static __device__ __forceinline__ float2 div_fast(float2 a, float2 b) {
    return __fmul2_rn(a, make_float2(rcp_approx(b.x), rcp_approx(b.y)));
  }
  static __device__ __forceinline__ float2 sqrt_fast(float2 a) {
    return __fmul2_rn(a, make_float2(rsqrt_approx(a.x), rsqrt_approx(a.y)));
  }
  static __device__ __forceinline__ float2 rcp_fast(float2 a) {
    return make_float2(rcp_approx(a.x), rcp_approx(a.y));
  }
  static __device__ __forceinline__ float lane(float2 a, int k) { return k ? a.y : a.x; }
  static __device__ __forceinline__ void set_lane(float2& a, int k, float v) {
    if (k) a.y = v; else a.x = v;
  }
};
template <> struct Ar<double> {
  using Scalar = double;
  static constexpr int lanes = 1;
  static __device__ __forceinline__ double c(double v) { return v; }
  static __device__ __forceinline__ double bc(double v) { return v; }
  static __device__ __forceinline__ double neg(double a) { return -a; }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) {
    return __fma_rn(a, b, c);
  }
  // FP64 keeps IEEE division and square root everywhere
  static __device__ __forceinline__ double div_fast(double a, double b) { return __ddiv_rn(a, b); }
  static __device__ __forceinline__ double sqrt_fast(double a) { return __dsqrt_rn(a); }
  static __device__ __forceinline__ double lane(double a, int) { return a; }
  static __device__ __forceinline__ void set_lane(double& a, int, double v) { a = v; }
};

// ------------------------------------------------------------------ exact stabilizer
// The root gamma* of eq:result1,
//   g(gamma) = sum_i dh_i ln(1 + ((1 - beta gamma) dh_i - (2 beta - 1) ds_i) / f_eq_i) = 0,
// the critical point of the post-collision entropy along gamma (Sec. KBC). g is strictly
// decreasing where every logarithm is defined: g'(gamma) = -beta sum_i dh_i^2 / (f_eq_i (1+x_i)).
// Newton's method from the estimate eq:result21, each step halved until every argument
// 1 + x_i stays positive; bounded iteration counts. With a_i = dh_i - (2 beta - 1) ds_i,
// x_i = (a_i - beta gamma dh_i) / f_eq_i and 1/f_eq_i = rx[a] ry[b] rz[c].
template <typename T> struct NewtonLimits;
template <> struct NewtonLimits<double> {
  static constexpr int iters = 50;
  static constexpr double tol = 1e-15;  // |step| <= tol (1 + |gamma|)
};
template <> struct NewtonLimits<float> {
  static constexpr int iters = 20;
  static constexpr float tol = 1e-6f;
};
__device__ __forceinline__ double log1p_t(double x) { return log1p(x); }
__device__ __forceinline__ float log1p_t(float x) { return log1pf(x); }

// status: 0 converged, 1 stopped where g is undefined or flat (gamma kept), 2 iteration cap
template <typename T>
__device__ __noinline__ T newton_gamma(const T (&dh)[27], const T (&av)[27], const T (&rx)[3],
                                       const T (&ry)[3], const T (&rz)[3], T beta, T g,
                                       int* status) {
  *status = 2;
#pragma unroll 1
  for (int it = 0; it < NewtonLimits<T>::iters; ++it) {
    T val = T(0), der = T(0);
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 27; ++i) {
      const T r = rx[i % 3] * ry[(i / 3) % 3] * rz[i / 9];
      const T x = (av[i] - beta * g * dh[i]) * r;
      if (!(T(1) + x > T(0))) ok = false;
      val += dh[i] * log1p_t(x);
      der -= beta * dh[i] * dh[i] * r / (T(1) + x);
    }
    if (!ok || der == T(0)) {
      *status = 1;
      break;
    }
    T step = -val / der;
#pragma unroll 1
    for (int tries = 0; tries < 60; ++tries) {
      bool pos = true;
#pragma unroll
      for (int i = 0; i < 27; ++i) {
        const T r = rx[i % 3] * ry[(i / 3) % 3] * rz[i / 9];
        if (!(T(1) + (av[i] - beta * (g + step) * dh[i]) * r > T(0))) pos = false;
      }
      if (pos) break;
      step *= T(0.5);
    }
    g += step;
    if (fabs(step) <= NewtonLimits<T>::tol * (T(1) + fabs(g))) {
      *status = 0;
      break;
    }
  }
  return g;
}

// One KBC collision on the shifted populations d[i] = f_i - W_i, in place: the post-collision
// state of eq:Egeneral with the mirror state eq:ksh-mirror, f' = f - beta (2 ds + gamma dh),
// ds = s - s_eq by Table 1, dh = f - f_eq - ds, gamma by eq:result21 (Sec. KBC); R holds one
// node (float, double) or two (float2). Returns gamma; bit k of *guarded is set when lane k's
// <dh|dh> fell under the guard. fp64 (FP32 arithmetic only): if given, bit k is set when
// lane k's <dh|dh> fell under kDenFp64 (its outputs are then to be replaced in FP64).
// EXACT (one node per thread only): gamma is the root of eq:result1 found by newton_gamma()
// from the estimate; *gamma_est receives the estimate and *newton the solver's status.
// POLY: the equilibrium is the second-order polynomial eq:polynomial2 instead of the product
// form eq:entropic_eq (its moments, the populations for dh, and the entropic weights).
template <typename R, bool CENTRAL = false, bool EXACT = false, bool POLY = false>
__device__ __forceinline__ R collide(R (&d)[27], const CollideParams& cp, int* guarded,
                                     typename Ar<R>::Scalar* gamma_est = nullptr,
                                     int* newton = nullptr, int* fp64 = nullptr) {
  using O = Ar<R>;
  using T = typename O::Scalar;
  static_assert(!(EXACT && POLY), "the exact stabilizer is built for the product form only");
  // ---- natural moments of delta by a factorised x -> y -> z reduction (eq:natmoments)
  // row r = (vy+1) + 3(vz+1); X0 = sum over vx, X1 = sum vx, X2 = sum vx^2
  R X0[9], X1[9], X2[9];
#pragma unroll
  for (int r = 0; r < 9; ++r) {
    const R m = d[3 * r + 0], z = d[3 * r + 1], p = d[3 * r + 2];
    X2[r] = O::add(p, m);
    X1[r] = O::sub(p, m);
    X0[r] = O::add(X2[r], z);
  }
  // y stage: Yp_q[c] = sum over vy of Xp * vy^q, c = vz+1
  auto ystage = [](const R (&X)[9], R (&Y0)[3], R (&Y1)[3], R (&Y2)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R m = X[3 * c + 0], z = X[3 * c + 1], p = X[3 * c + 2];
      Y2[c] = O::add(p, m);
      Y1[c] = O::sub(p, m);
      Y0[c] = O::add(Y2[c], z);
    }
  };
  R Y00[3], Y01[3], Y02[3], Y10[3], Y11[3], Y12[3], Y20[3], Y21[3], Y22[3];
  ystage(X0, Y00, Y01, Y02);
  ystage(X1, Y10, Y11, Y12);
  ystage(X2, Y20, Y21, Y22);
  (void)Y22;
  // z stage: D_pqr = sum over vz of Ypq * vz^r
  auto zsum = [](const R (&Y)[3]) { return O::add(O::add(Y[0], Y[2]), Y[1]); };
  const R D000 = zsum(Y00), D001 = O::sub(Y00[2], Y00[0]), D002 = O::add(Y00[2], Y00[0]);
  const R D100 = zsum(Y10), D101 = O::sub(Y10[2], Y10[0]), D102 = O::add(Y10[2], Y10[0]);
  const R D010 = zsum(Y01), D011 = O::sub(Y01[2], Y01[0]), D012 = O::add(Y01[2], Y01[0]);
  const R D200 = zsum(Y20), D201 = O::sub(Y20[2], Y20[0]);
  const R D020 = zsum(Y02), D021 = O::sub(Y02[2], Y02[0]);
  const R D110 = zsum(Y11), D111 = O::sub(Y11[2], Y11[0]);
  const R D120 = zsum(Y12);
  const R D210 = zsum(Y21);

  // ---- conserved quantities rho, u (eq:natmoments); sum W = 1, sum W v = 0
  const R one = O::c(1.0), three = O::c(3.0);
  const R drho = D000;
  const R rho = O::add(one, drho);
  const R ir = O::div_fast(one, rho);
  const R ux = O::mul(D100, ir), uy = O::mul(D010, ir), uz = O::mul(D001, ir);

  // ---- per-axis factors of the equilibrium eq:entropic_eq: e = R - 1 = 3u^2 / (1 + R)
  // FP32: 3u^2/(1 + R) avoids the cancellation of R - 1 at small u. FP64: R - 1 directly
  // (exact subtraction, absolute error ~1e-16, far below what the populations resolve),
  // which saves a division on GB300's narrow FP64 pipe.
  auto axis_e = [&](R u) {
    const R u3 = O::mul(three, O::mul(u, u));
    const R Rr = O::sqrt_fast(O::add(one, u3));
    if constexpr (std::is_same<T, double>::value)
      return O::sub(Rr, one);
    else
      return O::div_fast(u3, O::add(one, Rr));
  };
  const R c23 = O::c(2.0 / 3.0), c13 = O::c(1.0 / 3.0);
  // product form: e = R - 1 and the per-axis second moment m_2(u) = (2R - 1)/3 = 1/3 + 2e/3,
  // which also scales the third moments (rho M_eq,120 = rho u_x m_2(u_y)).
  // eq:polynomial2: e = 3u^2/2 gives the second moment 1/3 + u^2; its third moments are
  // rho u_a / 3 (a, b, b) and 0 (x, y, z), so m3 = 1/3 there.
  R ex, ey, ez, m3x, m3y, m3z;
  if constexpr (POLY) {
    const R c32 = O::c(1.5);
    ex = O::mul(c32, O::mul(ux, ux));
    ey = O::mul(c32, O::mul(uy, uy));
    ez = O::mul(c32, O::mul(uz, uz));
    m3x = m3y = m3z = c13;
  } else {
    ex = axis_e(ux);
    ey = axis_e(uy);
    ez = axis_e(uz);
    m3x = O::fma(c23, ex, c13);
    m3y = O::fma(c23, ey, c13);
    m3z = O::fma(c23, ez, c13);
  }

  // ---- rho-scaled moment deviations rho (M - M_eq), the inputs of Table 1 for ds = s - s_eq
  const R nrc23 = O::neg(O::mul(rho, c23));
  const R nd3 = O::mul(drho, O::c(-1.0 / 3.0));
  const R A200 = O::fma(nrc23, ex, O::add(D200, nd3));
  const R A020 = O::fma(nrc23, ey, O::add(D020, nd3));
  const R A002 = O::fma(nrc23, ez, O::add(D002, nd3));
  const R ANxz = O::sub(A200, A002), ANyz = O::sub(A020, A002);
  const R ATfull = O::add(O::add(A200, A020), A002);
  const R AT = cp.with_t ? ATfull : O::c(0.0);
  const R nD100 = O::neg(D100), nD010 = O::neg(D010), nD001 = O::neg(D001);
  const R APxy = O::fma(nD100, uy, D110), APxz = O::fma(nD100, uz, D101);
  const R APyz = O::fma(nD010, uz, D011);
  const R qs = O::c(cp.with_q ? 1.0 : 0.0);
  // third-order natural deviations rho (M - M_eq), before the variant mask
  const R RQxyy = O::fma(nD100, m3y, D120), RQxzz = O::fma(nD100, m3z, D102);
  const R RQxxy = O::fma(nD010, m3x, D210), RQyzz = O::fma(nD010, m3z, D012);
  const R RQxxz = O::fma(nD001, m3x, D201), RQyyz = O::fma(nD001, m3y, D021);
  const R RQxyz = POLY ? D111 : O::fma(O::neg(O::mul(D100, uy)), uz, D111);
  const R AQxyy = O::mul(qs, RQxyy), AQxzz = O::mul(qs, RQxzz);
  const R AQxxy = O::mul(qs, RQxxy), AQyzz = O::mul(qs, RQyzz);
  const R AQxxz = O::mul(qs, RQxxz), AQyyz = O::mul(qs, RQyyz);
  const R AQxyz = O::mul(qs, RQxyz);

  // Table 1 per velocity class: ds = d + t + q evaluated on the deviations
  const R c16 = O::c(1.0 / 6.0), half = O::c(0.5), quarter = O::c(0.25);
  const R s0 = O::neg(AT);
  const R Fx = O::mul(O::add(O::sub(O::add(ANxz, ANxz), ANyz), AT), c16);
  const R Fy = O::mul(O::add(O::sub(O::add(ANyz, ANyz), ANxz), AT), c16);
  const R Fz = O::mul(O::sub(O::sub(AT, ANxz), ANyz), c16);
  const R Gx = O::mul(O::add(AQxyy, AQxzz), half);
  const R Gy = O::mul(O::add(AQxxy, AQyzz), half);
  const R Gz = O::mul(O::add(AQxxz, AQyyz), half);
  const R Pxy4 = O::mul(quarter, APxy), Pxz4 = O::mul(quarter, APxz);
  const R Pyz4 = O::mul(quarter, APyz);
  const R Qxxy4 = O::mul(quarter, AQxxy), Qxyy4 = O::mul(quarter, AQxyy);
  const R Qxxz4 = O::mul(quarter, AQxxz), Qxzz4 = O::mul(quarter, AQxzz);
  const R Qyyz4 = O::mul(quarter, AQyyz), Qyzz4 = O::mul(quarter, AQyzz);
  const R Qxyz8 = O::mul(O::c(0.125), AQxyz);
  auto sg = [](int s, R v) { return s > 0 ? v : O::neg(v); };
  // (s1 P) + (s2 Q1) + (s3 Q2) for an edge class; signs are compile-time after unrolling
  auto edge = [&](int sp, R P4, int s1, R Q1, int s2, R Q2) {
    return O::add(O::add(sg(sp, P4), sg(s1, Q1)), sg(s2, Q2));
  };
  auto ds_of = [&](int a, int b, int c) -> R {
    const int nnz = (a != 0) + (b != 0) + (c != 0);
    if (nnz == 0) return s0;
    if (nnz == 1) {
      if (a != 0) return a > 0 ? O::sub(Fx, Gx) : O::add(Fx, Gx);
      if (b != 0) return b > 0 ? O::sub(Fy, Gy) : O::add(Fy, Gy);
      return c > 0 ? O::sub(Fz, Gz) : O::add(Fz, Gz);
    }
    if (nnz == 2) {
      if (c == 0) return edge(a * b, Pxy4, b, Qxxy4, a, Qxyy4);
      if (b == 0) return edge(a * c, Pxz4, c, Qxxz4, a, Qxzz4);
      return edge(b * c, Pyz4, c, Qyyz4, b, Qyzz4);
    }
    return sg(a * b * c, Qxyz8);
  };

  // equilibrium factors: rho phi_x(a) = W_a (1 + gx_a), phi_y(b) = W_b (1 + fy_b), ...
  // with e_0 = -e, e_{+-1} = 2e +- 3u; the x factor carries rho: gx = drho + rho e_x
  // (product form only; eq:polynomial2 is evaluated per direction in the loop below)
  R gx[3], fy[3], fz[3];
  // reciprocal weights of the entropic scalar product, 1/f_eq_i = rx[a] ry[b] rz[c]
  R rx[3], ry[3], rz[3];
  if constexpr (!POLY) {
    const R tex = O::add(ex, ex), tey = O::add(ey, ey), tez = O::add(ez, ez);
    const R ux3 = O::mul(three, ux), uy3 = O::mul(three, uy), uz3 = O::mul(three, uz);
    gx[0] = O::fma(rho, O::sub(tex, ux3), drho);
    gx[1] = O::fma(O::neg(rho), ex, drho);
    gx[2] = O::fma(rho, O::add(tex, ux3), drho);
    fy[0] = O::sub(tey, uy3);
    fy[1] = O::neg(ey);
    fy[2] = O::add(tey, uy3);
    fz[0] = O::sub(tez, uz3);
    fz[1] = O::neg(ez);
    fz[2] = O::add(tez, uz3);
    // per axis: q = 1 / (p0 p1 p2) gives the three reciprocals 1/p_a by products. FP32 takes
    // one MUFU reciprocal per axis; FP64 shares one IEEE division among the three axes.
    R px[3], py[3], pz[3], Q[3];
    auto axis_p = [&](const R (&e)[3], R (&p)[3], R& q) {
      p[0] = O::mul(c16, O::add(one, e[0]));
      p[1] = O::mul(c23, O::add(one, e[1]));
      p[2] = O::mul(c16, O::add(one, e[2]));
      q = O::mul(p[0], O::mul(p[1], p[2]));
    };
    axis_p(gx, px, Q[0]);
    axis_p(fy, py, Q[1]);
    axis_p(fz, pz, Q[2]);
    R iq[3];
    if constexpr (std::is_same<T, double>::value) {
      const R Q12 = O::mul(Q[1], Q[2]);
      const R inv = O::div_fast(one, O::mul(Q[0], Q12));
      const R invQ0 = O::mul(inv, Q[0]);
      iq[0] = O::mul(inv, Q12);
      iq[1] = O::mul(invQ0, Q[2]);
      iq[2] = O::mul(invQ0, Q[1]);
    } else {
      iq[0] = O::div_fast(one, Q[0]);
      iq[1] = O::div_fast(one, Q[1]);
      iq[2] = O::div_fast(one, Q[2]);
    }
    auto recip_axis = [&](const R (&p)[3], R q, R (&r)[3]) {
      const R qp0 = O::mul(q, p[0]);
      r[0] = O::mul(O::mul(p[1], p[2]), q);
      r[1] = O::mul(p[2], qp0);
      r[2] = O::mul(p[1], qp0);
    };
    recip_axis(px, iq[0], rx);
    recip_axis(py, iq[1], ry);
    recip_axis(pz, iq[2], rz);
  }
  // eq:polynomial2 with c_s^2 = 1/3: (f_eq_i - W_i)/W_i = drho + rho (3 s + 9/2 s^2 - 3/2 u.u),
  // s = u.v_i
  [[maybe_unused]] const R nu15 =
      POLY ? O::mul(O::c(-1.5), O::fma(ux, ux, O::fma(uy, uy, O::mul(uz, uz)))) : O::c(0.0);

  // ---- dh, the two entropic products, and the part of the relaxation known before gamma
  // (Sec. KBC: dh = f - f_eq - ds; <X|Y> = sum X_i Y_i / f_eq_i): d <- d - 2 beta ds, dh kept
  // for the gamma-dependent part
  const R nb2 = O::bc(-prec<T>(cp.two_beta, cp.two_betaf));
  R dh[27];
  // a_i = dh_i - (2 beta - 1) ds_i, kept for the exact stabilizer only
  [[maybe_unused]] R av[EXACT ? 27 : 1];
  [[maybe_unused]] const R nc2 = O::sub(O::c(1.0), O::bc(prec<T>(cp.two_beta, cp.two_betaf)));
  R num = O::c(0.0), den = O::c(0.0);
  // (1 + gx)(1 + fy) - 1 for the 9 (a, b) pairs, shared by the three z levels
  R Pab[9];
  if constexpr (!POLY) {
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) Pab[a + 3 * b] = O::fma(gx[a], fy[b], O::add(gx[a], fy[b]));
  }
  // Central-moment variants (appendix): the shear part is built on the central moments.
  // Their deviations follow from the natural ones because rho and u are conserved: second
  // order unchanged, third order rho dMc_120 = rho dM_120 - 2 uy rho dM_110 - ux rho dM_020
  // and its permutations, rho dMc_111 = rho dM_111 - ux rho dM_011 - uy rho dM_101 - uz rho dM_110.
  // ds_i = sum over the s moments of cx(a;p) cy(b;q) cz(c;r) rho dMc_pqr with the 1D central
  // inverse c(0) = [1 - u^2, -2u, -1], c(+-1) = [u(u +- 1)/2, u +- 1/2, 1/2].
  R B200, B020, B002, Bc[7], cxv[3][3], cyv[3][3], czv[3][3];
  if constexpr (CENTRAL) {
    const R tr = cp.with_t ? O::c(0.0) : O::mul(ATfull, O::c(1.0 / 3.0));
    B200 = O::sub(A200, tr);
    B020 = O::sub(A020, tr);
    B002 = O::sub(A002, tr);
    const R two = O::c(2.0);
    Bc[0] = O::mul(qs, O::fma(O::neg(ux), A020, O::fma(O::neg(O::mul(two, uy)), APxy, RQxyy)));  // 120
    Bc[1] = O::mul(qs, O::fma(O::neg(ux), A002, O::fma(O::neg(O::mul(two, uz)), APxz, RQxzz)));  // 102
    Bc[2] = O::mul(qs, O::fma(O::neg(uy), A200, O::fma(O::neg(O::mul(two, ux)), APxy, RQxxy)));  // 210
    Bc[3] = O::mul(qs, O::fma(O::neg(uy), A002, O::fma(O::neg(O::mul(two, uz)), APyz, RQyzz)));  // 012
    Bc[4] = O::mul(qs, O::fma(O::neg(uz), A200, O::fma(O::neg(O::mul(two, ux)), APxz, RQxxz)));  // 201
    Bc[5] = O::mul(qs, O::fma(O::neg(uz), A020, O::fma(O::neg(O::mul(two, uy)), APyz, RQyyz)));  // 021
    Bc[6] = O::mul(qs, O::fma(O::neg(uz), APxy,
                              O::fma(O::neg(uy), APxz, O::fma(O::neg(ux), APyz, RQxyz))));   // 111
    auto coef = [&](R u, R (&cv)[3][3]) {  // cv[v+1][p]
      const R hu = O::mul(O::c(0.5), u);
      const R uu = O::mul(u, u);
      cv[0][0] = O::sub(O::mul(hu, u), hu);          // u(u - 1)/2
      cv[1][0] = O::sub(one, uu);                    // 1 - u^2
      cv[2][0] = O::add(O::mul(hu, u), hu);          // u(u + 1)/2
      cv[0][1] = O::sub(u, O::c(0.5));
      cv[1][1] = O::mul(O::c(-2.0), u);
      cv[2][1] = O::add(u, O::c(0.5));
      cv[0][2] = O::c(0.5);
      cv[1][2] = O::c(-1.0);
      cv[2][2] = O::c(0.5);
    };
    coef(ux, cxv);
    coef(uy, cyv);
    coef(uz, czv);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R cn = O::c(0.0), cd = O::c(0.0);
    // z stage of the central shear part: Zpq = sum_r cz(c;r) rho dMc_pqr
    R Z00, Z01, Z02, Z10, Z11, Z12, Z20, Z21;
    if constexpr (CENTRAL) {
      const R* cz = czv[c];
      Z20 = O::fma(cz[1], Bc[4], O::mul(cz[0], B200));
      Z02 = O::fma(cz[1], Bc[5], O::mul(cz[0], B020));
      Z00 = O::mul(cz[2], B002);
      Z11 = O::fma(cz[1], Bc[6], O::mul(cz[0], APxy));
      Z10 = O::fma(cz[2], Bc[1], O::mul(cz[1], APxz));
      Z01 = O::fma(cz[2], Bc[3], O::mul(cz[1], APyz));
      Z12 = O::mul(cz[0], Bc[0]);
      Z21 = O::mul(cz[0], Bc[2]);
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      R rn = O::c(0.0), rd = O::c(0.0);
      R Y0, Y1, Y2;  // y stage: Yp = sum_q cy(b;q) Zpq
      if constexpr (CENTRAL) {
        const R* cy = cyv[b];
        Y0 = O::fma(cy[2], Z02, O::fma(cy[1], Z01, O::mul(cy[0], Z00)));
        Y1 = O::fma(cy[2], Z12, O::fma(cy[1], Z11, O::mul(cy[0], Z10)));
        Y2 = O::fma(cy[1], Z21, O::mul(cy[0], Z20));
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int i = a + 3 * b + 9 * c;
        R G, wi;  // (f_eq_i - W_i)/W_i, and the x weight (product) or 1/f_eq_i (polynomial)
        if constexpr (POLY) {
          R sv = O::c(0.0);
          if (a != 1) sv = a == 2 ? O::add(sv, ux) : O::sub(sv, ux);
          if (b != 1) sv = b == 2 ? O::add(sv, uy) : O::sub(sv, uy);
          if (c != 1) sv = c == 2 ? O::add(sv, uz) : O::sub(sv, uz);
          G = O::fma(rho, O::fma(sv, O::fma(O::c(4.5), sv, three), nu15), drho);
          wi = O::mul(O::c(inv_wgt(i)), O::div_fast(one, O::add(one, G)));
        } else {
          // (1 + gx)(1 + fy)(1 + fz) - 1 without cancellation
          const R P = Pab[a + 3 * b];
          G = O::fma(P, fz[c], O::add(P, fz[c]));
          wi = rx[a];
        }
        R dsi;
        if constexpr (CENTRAL) {
          const R* cx = cxv[a];
          dsi = O::fma(cx[2], Y2, O::fma(cx[1], Y1, O::mul(cx[0], Y0)));
        } else {
          dsi = ds_of(a - 1, b - 1, c - 1);
        }
        const R dhi = O::sub(O::fma(O::c(-wgt(i)), G, d[i]), dsi);
        const R t1 = O::mul(wi, dhi);
        rn = O::fma(t1, dsi, rn);
        rd = O::fma(t1, dhi, rd);
        dh[i] = dhi;
        if constexpr (EXACT) av[i] = O::fma(nc2, dsi, dhi);
        d[i] = O::fma(nb2, dsi, d[i]);
      }
      if constexpr (POLY) {
        cn = O::add(rn, cn);
        cd = O::add(rd, cd);
      } else {
        cn = O::fma(ry[b], rn, cn);
        cd = O::fma(ry[b], rd, cd);
      }
    }
    if constexpr (POLY) {
      num = O::add(cn, num);
      den = O::add(cd, den);
    } else {
      num = O::fma(rz[c], cn, num);
      den = O::fma(rz[c], cd, den);
    }
  }

  // ---- stabilizer (eq:result21) and the rest of the relaxation f' = f - beta(2 ds + gamma dh)
  const T ib = prec<T>(cp.inv_beta, cp.inv_betaf);
  R gamma = O::c(0.0);
  int gmask = 0;
#pragma unroll
  for (int k = 0; k < O::lanes; ++k) {
    const T nk = O::lane(num, k), dk = O::lane(den, k);
    T gk;
    if (cp.gamma_mode == GAMMA_LBGK) {
      gk = T(2);
    } else if (cp.gamma_mode == GAMMA_RLB) {
      gk = ib;
    } else if (std::is_same<T, float>::value && !EXACT && fp64 && dk < T(kDenFp64) &&
               dk == dk) {
      gk = T(2);  // replaced by the FP64 collision of this node
      *fp64 |= 1 << k;
    } else if (dk > Guard<T>::den) {
      gk = Ar<T>::fma(-Ar<T>::sub(T(2), ib), Ar<T>::div_fast(nk, dk), ib);
    } else if (dk == dk) {
      gk = T(2);
      gmask |= 1 << k;
    } else {
      gk = dk;  // NaN propagates to the populations and to the diagnostics
    }
    O::set_lane(gamma, k, gk);
  }
  *guarded = gmask;
  if constexpr (EXACT) {
    static_assert(O::lanes == 1, "the exact stabilizer runs one node per thread");
    if (gamma_est) *gamma_est = gamma;
    int status = 1;
    // guarded (<dh|dh> ~ 0) and non-finite nodes keep the estimate's value
    if (!gmask && gamma == gamma && cp.gamma_mode == GAMMA_EXACT)
      gamma = newton_gamma<T>(dh, av, rx, ry, rz, prec<T>(cp.beta, cp.betaf), gamma, &status);
    if (newton) *newton = status;
  }
  const R nbg = O::neg(O::mul(O::bc(prec<T>(cp.beta, cp.betaf)), gamma));
#pragma unroll
  for (int i = 0; i < 27; ++i) d[i] = O::fma(nbg, dh[i], d[i]);
  return gamma;
}

// ------------------------------------------------------------------ lean FP32 collision
// The collision of collide() for the product-form equilibrium and the natural-moment shear
// parts, in FP32 arithmetic (R = float or float2), arranged for the fewest FP32 operations per
// node (every FP32 step kernel of these variants runs it):
//   * REL (FP16 storage): the data are h_i = (f_i - W_i) / W_i. Each moment stage weights the
//     velocities -1, 0, +1 as 1 : 4 : 1 (that is 6 W_v), so the moments come out 216 times
//     their value; that factor and the 1/W_i of the outputs sit in the constants of Table 1's
//     class values, and dh/W = h - G - ds/W needs no weight per population;
//   * the entropic weights (W_i/f_eq_i for REL, 1/f_eq_i otherwise) are products of one MUFU
//     reciprocal per axis and velocity component;
//   * the q part's switch multiplies three class constants, not the seven third moments;
//   * 3u^2 reuses 3u, and the first term of each entropic sum is a product, not an FMA on 0.
template <typename R, bool REL>
__device__ __forceinline__ R collide_lean(R (&d)[27], const CollideParams& cp, int* guarded,
                                          int* fp64) {
  using O = Ar<R>;
  using T = float;
  static_assert(std::is_same<typename O::Scalar, float>::value, "FP32 arithmetic only");
  const R one = O::c(1.0), three = O::c(3.0);
  // ---- moments (eq:natmoments) by a factorised x -> y -> z reduction; REL weights 1 : 4 : 1
  auto stage0 = [&](R m, R z, R p) {
    const R s = O::add(p, m);
    if constexpr (REL) return O::fma(O::c(4.0), z, s);
    else return O::add(s, z);
  };
  R X0[9], X1[9], X2[9];
#pragma unroll
  for (int r = 0; r < 9; ++r) {
    const R m = d[3 * r + 0], z = d[3 * r + 1], p = d[3 * r + 2];
    X2[r] = O::add(p, m);
    X1[r] = O::sub(p, m);
    X0[r] = stage0(m, z, p);
  }
  auto ystage = [&](const R (&X)[9], R (&Y0)[3], R (&Y1)[3], R (&Y2)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R m = X[3 * c + 0], z = X[3 * c + 1], p = X[3 * c + 2];
      Y2[c] = O::add(p, m);
      Y1[c] = O::sub(p, m);
      Y0[c] = stage0(m, z, p);
    }
  };
  R Y00[3], Y01[3], Y02[3], Y10[3], Y11[3], Y12[3], Y20[3], Y21[3], Y22[3];
  ystage(X0, Y00, Y01, Y02);
  ystage(X1, Y10, Y11, Y12);
  ystage(X2, Y20, Y21, Y22);
  (void)Y22;
  auto zsum = [&](const R (&Y)[3]) { return stage0(Y[0], Y[1], Y[2]); };
  // E_pqr = D_pqr / K: the moment sums of the data, K = 1/216 for REL
  const R E000 = zsum(Y00), E001 = O::sub(Y00[2], Y00[0]), E002 = O::add(Y00[2], Y00[0]);
  const R E100 = zsum(Y10), E101 = O::sub(Y10[2], Y10[0]), E102 = O::add(Y10[2], Y10[0]);
  const R E010 = zsum(Y01), E011 = O::sub(Y01[2], Y01[0]), E012 = O::add(Y01[2], Y01[0]);
  const R E200 = zsum(Y20), E201 = O::sub(Y20[2], Y20[0]);
  const R E020 = zsum(Y02), E021 = O::sub(Y02[2], Y02[0]);
  const R E110 = zsum(Y11), E111 = O::sub(Y11[2], Y11[0]);
  const R E120 = zsum(Y12);
  const R E210 = zsum(Y21);
  constexpr double K = REL ? 1.0 / 216.0 : 1.0;

  // ---- conserved quantities rho, u; kir = K / rho
  R drho, rho, kir;
  if constexpr (REL) {
    drho = O::mul(E000, O::c(K));
    rho = O::add(one, drho);
    kir = O::rcp_fast(O::add(O::c(216.0), E000));
  } else {
    drho = E000;
    rho = O::add(one, drho);
    kir = O::rcp_fast(rho);
  }
  const R ux = O::mul(E100, kir), uy = O::mul(E010, kir), uz = O::mul(E001, kir);

  // ---- per-axis factors of eq:entropic_eq: e = R - 1 = 3u^2 / (1 + R), R = sqrt(1 + 3u^2)
  R ux3, uy3, uz3, ex, ey, ez;
  auto axis = [&](R u, R& u3, R& e) {
    u3 = O::mul(three, u);
    const R uu3 = O::mul(u3, u);
    const R Rr = O::sqrt_fast(O::add(one, uu3));
    e = O::mul(uu3, O::rcp_fast(O::add(one, Rr)));
  };
  axis(ux, ux3, ex);
  axis(uy, uy3, ey);
  axis(uz, uz3, ez);
  const R c23 = O::c(2.0 / 3.0), c13 = O::c(1.0 / 3.0);
  const R m3x = O::fma(c23, ex, c13), m3y = O::fma(c23, ey, c13), m3z = O::fma(c23, ez, c13);

  // ---- rho (M - M_eq): second moments at their value, the others at 1/K of it
  const R nrc23 = O::mul(rho, O::c(-2.0 / 3.0));
  const R nd3 = O::mul(drho, O::c(-1.0 / 3.0));
  auto second = [&](R E, R e) {
    if constexpr (REL) return O::fma(nrc23, e, O::fma(E, O::c(K), nd3));
    else return O::fma(nrc23, e, O::add(E, nd3));
  };
  const R A200 = second(E200, ex), A020 = second(E020, ey), A002 = second(E002, ez);
  const R ANxz = O::sub(A200, A002), ANyz = O::sub(A020, A002);
  const R ATfull = O::add(O::add(A200, A020), A002);
  const R AT = cp.with_t ? ATfull : O::c(0.0);
  const R nE100 = O::neg(E100), nE010 = O::neg(E010), nE001 = O::neg(E001);
  const R APxy = O::fma(nE100, uy, E110), APxz = O::fma(nE100, uz, E101);
  const R APyz = O::fma(nE010, uz, E011);
  const R RQxyy = O::fma(nE100, m3y, E120), RQxzz = O::fma(nE100, m3z, E102);
  const R RQxxy = O::fma(nE010, m3x, E210), RQyzz = O::fma(nE010, m3z, E012);
  const R RQxxz = O::fma(nE001, m3x, E201), RQyyz = O::fma(nE001, m3y, E021);
  const R RQxyz = O::fma(O::mul(nE100, uy), uz, E111);

  // ---- Table 1 class values of ds in the data's unit (REL: ds_i / W_i)
  constexpr double wR = REL ? 27.0 / 8.0 : 1.0, wF = REL ? 13.5 : 1.0;
  constexpr double wE = REL ? 54.0 : 1.0, wC = REL ? 216.0 : 1.0;
  const T qf = cp.with_q ? 1.0f : 0.0f;
  const R cG = O::bc(qf * (float)(K * wF / 2.0));
  const R cQ4 = O::bc(qf * (float)(K * wE / 4.0));
  const R cQ8 = O::bc(qf * (float)(K * wC / 8.0));
  const R s0 = O::mul(AT, O::c(-wR));
  const R cF = O::c(wF / 6.0);
  const R Fx = O::mul(O::add(O::sub(O::add(ANxz, ANxz), ANyz), AT), cF);
  const R Fy = O::mul(O::add(O::sub(O::add(ANyz, ANyz), ANxz), AT), cF);
  const R Fz = O::mul(O::sub(O::sub(AT, ANxz), ANyz), cF);
  const R Gx = O::mul(O::add(RQxyy, RQxzz), cG);
  const R Gy = O::mul(O::add(RQxxy, RQyzz), cG);
  const R Gz = O::mul(O::add(RQxxz, RQyyz), cG);
  const R cP = O::c(K * wE / 4.0);
  const R Pxy4 = O::mul(APxy, cP), Pxz4 = O::mul(APxz, cP), Pyz4 = O::mul(APyz, cP);
  const R Qxxy4 = O::mul(RQxxy, cQ4), Qxyy4 = O::mul(RQxyy, cQ4);
  const R Qxxz4 = O::mul(RQxxz, cQ4), Qxzz4 = O::mul(RQxzz, cQ4);
  const R Qyyz4 = O::mul(RQyyz, cQ4), Qyzz4 = O::mul(RQyzz, cQ4);
  const R Qxyz8 = O::mul(RQxyz, cQ8);
  auto sg = [](int s, R v) { return s > 0 ? v : O::neg(v); };
  auto edge = [&](int sp, R P4, int s1, R Q1, int s2, R Q2) {
    return O::add(O::add(sg(sp, P4), sg(s1, Q1)), sg(s2, Q2));
  };
  auto ds_of = [&](int a, int b, int c) -> R {
    const int nnz = (a != 0) + (b != 0) + (c != 0);
    if (nnz == 0) return s0;
    if (nnz == 1) {
      if (a != 0) return a > 0 ? O::sub(Fx, Gx) : O::add(Fx, Gx);
      if (b != 0) return b > 0 ? O::sub(Fy, Gy) : O::add(Fy, Gy);
      return c > 0 ? O::sub(Fz, Gz) : O::add(Fz, Gz);
    }
    if (nnz == 2) {
      if (c == 0) return edge(a * b, Pxy4, b, Qxxy4, a, Qxyy4);
      if (b == 0) return edge(a * c, Pxz4, c, Qxxz4, a, Qxzz4);
      return edge(b * c, Pyz4, c, Qyyz4, b, Qyzz4);
    }
    return sg(a * b * c, Qxyz8);
  };

  // ---- equilibrium: f_eq_i / W_i = X_a Y_b Z_c with X_a = 1 + gx_a (carrying rho),
  // Y_b = 1 + fy_b, Z_c = 1 + fz_c, e_0 = -e, e_{+-1} = 2e +- 3u
  const R tex = O::add(ex, ex), tey = O::add(ey, ey), tez = O::add(ez, ez);
  R gx[3], fy[3], fz[3];
  gx[0] = O::fma(rho, O::sub(tex, ux3), drho);
  gx[1] = O::fma(O::neg(rho), ex, drho);
  gx[2] = O::fma(rho, O::add(tex, ux3), drho);
  fy[0] = O::sub(tey, uy3);
  fy[1] = O::neg(ey);
  fy[2] = O::add(tey, uy3);
  fz[0] = O::sub(tez, uz3);
  fz[1] = O::neg(ez);
  fz[2] = O::add(tez, uz3);
  // entropic weights per axis: REL W_a / X_a, otherwise 1 / (W_a X_a)
  R wx[3], wy[3], wz[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double Wa = a == 1 ? 2.0 / 3.0 : 1.0 / 6.0;
    const R cw = O::c(REL ? 1.0 / Wa : Wa);
    wx[a] = O::rcp_fast(O::fma(cw, gx[a], cw));
    wy[a] = O::rcp_fast(O::fma(cw, fy[a], cw));
    wz[a] = O::rcp_fast(O::fma(cw, fz[a], cw));
  }
  // X_a Y_b - 1 for the 9 (a, b) pairs, without cancellation
  R Pab[9];
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) Pab[a + 3 * b] = O::fma(gx[a], fy[b], O::add(gx[a], fy[b]));

  // ---- dh (Sec. KBC: dh = f - f_eq - ds), the entropic products <ds|dh>, <dh|dh>, and the
  // part of f' = f - beta (2 ds + gamma dh) known before gamma
  const R nb2 = O::bc(-cp.two_betaf);
  R dh[27];
  R num, den;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R cn, cd;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      R rn, rd;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int i = a + 3 * b + 9 * c;
        const R P = Pab[a + 3 * b];
        const R G = O::fma(P, fz[c], O::add(P, fz[c]));  // X_a Y_b Z_c - 1
        const R dsi = ds_of(a - 1, b - 1, c - 1);
        R dhi;
        if constexpr (REL) dhi = O::sub(O::sub(d[i], G), dsi);
        else dhi = O::sub(O::fma(O::c(-wgt(i)), G, d[i]), dsi);
        const R t1 = O::mul(wx[a], dhi);
        if (a == 0) {
          rn = O::mul(t1, dsi);
          rd = O::mul(t1, dhi);
        } else {
          rn = O::fma(t1, dsi, rn);
          rd = O::fma(t1, dhi, rd);
        }
        dh[i] = dhi;
        d[i] = O::fma(nb2, dsi, d[i]);
      }
      if (b == 0) {
        cn = O::mul(wy[b], rn);
        cd = O::mul(wy[b], rd);
      } else {
        cn = O::fma(wy[b], rn, cn);
        cd = O::fma(wy[b], rd, cd);
      }
    }
    if (c == 0) {
      num = O::mul(wz[c], cn);
      den = O::mul(wz[c], cd);
    } else {
      num = O::fma(wz[c], cn, num);
      den = O::fma(wz[c], cd, den);
    }
  }

  // ---- stabilizer (eq:result21) and the rest of the relaxation
  const T ib = cp.inv_betaf;
  R gamma = O::c(0.0);
  int gmask = 0;
#pragma unroll
  for (int k = 0; k < O::lanes; ++k) {
    const T nk = O::lane(num, k), dk = O::lane(den, k);
    T gk;
    if (cp.gamma_mode == GAMMA_LBGK) {
      gk = T(2);
    } else if (cp.gamma_mode == GAMMA_RLB) {
      gk = ib;
    } else if (fp64 && dk < kDenFp64 && dk == dk) {
      gk = T(2);  // replaced by the FP64 collision of this node
      *fp64 |= 1 << k;
    } else if (dk > Guard<T>::den) {
      gk = Ar<T>::fma(-Ar<T>::sub(T(2), ib), Ar<T>::div_fast(nk, dk), ib);
    } else if (dk == dk) {
      gk = T(2);
      gmask |= 1 << k;
    } else {
      gk = dk;  // NaN propagates to the populations and to the diagnostics
    }
    O::set_lane(gamma, k, gk);
  }
  *guarded = gmask;
  const R nbg = O::mul(O::bc(-cp.betaf), gamma);
#pragma unroll
  for (int i = 0; i < 27; ++i) d[i] = O::fma(nbg, dh[i], d[i]);
  return gamma;
}

// The collision of a step kernel on data in the storage's collision unit (REL: relative to
// W_i, the FP16 codec): the lean form for FP32 arithmetic, product-form equilibrium and
// natural moments; collide() otherwise.
template <typename R, bool CENTRAL, bool EXACT, bool POLY, bool REL>
__device__ __forceinline__ R collide_step(R (&d)[27], const CollideParams& cp, int* guarded,
                                          int* fp64) {
  using O = Ar<R>;
  using T = typename O::Scalar;
  if constexpr (!CENTRAL && !EXACT && !POLY && std::is_same<T, float>::value) {
    if constexpr (std::is_same<R, float>::value) {
      // One node: the FP32x2 collision with the node in both lanes. Every FP32 step kernel
      // then runs the same compiled arithmetic and gives the same bits; the scalar (float)
      // instantiation rounds differently (the compiler places the approximate MUFU reciprocal
      // and square root differently in the two code shapes).
      float2 d2[27];
#pragma unroll
      for (int i = 0; i < 27; ++i) d2[i] = make_float2(d[i], d[i]);
      int g2 = 0, f2 = 0;
      const float2 gam = collide_lean<float2, REL>(d2, cp, &g2, fp64 ? &f2 : nullptr);
#pragma unroll
      for (int i = 0; i < 27; ++i) d[i] = d2[i].x;
      *guarded = g2 & 1;
      if (fp64) *fp64 = f2 & 1;
      return gam.x;
    } else {
      return collide_lean<R, REL>(d, cp, guarded, fp64);
    }
  } else {
    if constexpr (REL) {
#pragma unroll
      for (int i = 0; i < 27; ++i) d[i] = O::mul(O::c(wgt(i)), d[i]);
    }
    const R g = collide<R, CENTRAL, EXACT, POLY>(d, cp, guarded, nullptr, nullptr, fp64);
    if constexpr (REL) {
#pragma unroll
      for (int i = 0; i < 27; ++i) d[i] = O::mul(O::c(inv_wgt(i)), d[i]);
    }
    return g;
  }
}


// Equilibrium shift f_eq_i(rho, u) - W_i by the same per-axis closed form, in the precision T
// of the arguments (FP64 for initialisation, the collision precision for the pre-solve).
template <typename T>
__device__ __forceinline__ void equilibrium_shift(T rho, T ux, T uy, T uz, T (&out)[27]) {
  const T one = T(1), two = T(2), three = T(3);
  const T drho = rho - one;
  const T Rx = sqrt(one + three * ux * ux), Ry = sqrt(one + three * uy * uy),
          Rz = sqrt(one + three * uz * uz);
  const T ex = three * ux * ux / (one + Rx), ey = three * uy * uy / (one + Ry),
          ez = three * uz * uz / (one + Rz);
  const T gx[3] = {drho + (two * ex - three * ux) * rho, drho - ex * rho,
                   drho + (two * ex + three * ux) * rho};
  const T fy[3] = {two * ey - three * uy, -ey, two * ey + three * uy};
  const T fz[3] = {two * ez - three * uz, -ez, two * ez + three * uz};
#pragma unroll
  for (int i = 0; i < 27; ++i) {
    const T gxa = gx[cx(i) + 1], fyb = fy[cy(i) + 1], fzc = fz[cz(i) + 1];
    const T P = gxa + fyb + gxa * fyb;
    out[i] = T(wgt(i)) * (P + fzc + P * fzc);
  }
}

// ------------------------------------------------------------------ addressing
// The canonical state at time t is the pre-collision field f(x, t). Where population i of
// node y lives in memory:
//   pull            buffer t&1, plane i,     node y - v_i   (post-collision of t-1 at the source)
//   AA, t even      buffer 0,   plane i,     node y
//   AA, t odd       buffer 0,   plane 26-i,  node y - v_i
// A step at node x loads canon(t, i, x) and stores f'_i(x) at canon(t+1, i, x + v_i), which
// is: pull -> (plane i, node x) of the other buffer; AA even -> (plane 26-i, node x);
// AA odd -> (plane i, node x + v_i).
enum { MODE_PULL = 0, MODE_AA_EVEN = 1, MODE_AA_ODD = 2 };

struct Geo {
  uint32_t nx, ny, nz, nxy;
  uint64_t P;
  uint32_t zb, ze;         // the step kernels update the planes zb <= z < ze (all: 0, nz)
  uint32_t* fbmask;        // one bit per node (linear index): collide again in FP64
  unsigned int* fb_any;    // set to 1 with any bit of fbmask
  unsigned int* fb_batch;  // the batch-wide flag, set as well (null outside a batch)
};

// Marks node n (linear index x + nx y + nx ny z) for the FP64 re-collision pass; the caller
// has not stored its FP32 outputs.
__device__ __forceinline__ void flag_fp64(const Geo& g, uint32_t n) {
  atomicOr(g.fbmask + (n >> 5), 1u << (n & 31));
  *g.fb_any = 1u;
  if (g.fb_batch) *g.fb_batch = 1u;
}

// in-plane offsets of the 3x3x3 neighbourhood of (x, y, z) on the periodic box
struct Nbr {
  uint32_t ox[3], oy[3], oz[3];
  __device__ __forceinline__ void init(const Geo& g, uint32_t x, uint32_t y, uint32_t z) {
    ox[0] = x == 0 ? g.nx - 1 : x - 1;
    ox[1] = x;
    ox[2] = x + 1 == g.nx ? 0 : x + 1;
    oy[0] = (y == 0 ? g.ny - 1 : y - 1) * g.nx;
    oy[1] = y * g.nx;
    oy[2] = (y + 1 == g.ny ? 0 : y + 1) * g.nx;
    oz[0] = (z == 0 ? g.nz - 1 : z - 1) * g.nxy;
    oz[1] = z * g.nxy;
    oz[2] = (z + 1 == g.nz ? 0 : z + 1) * g.nxy;
  }
  // node x + s * v_i, s in {-1, 0, +1}
  template <int I, int SHIFT> __device__ __forceinline__ uint32_t at() const {
    return ox[SHIFT * cx(I) + 1] + oy[SHIFT * cy(I) + 1] + oz[SHIFT * cz(I) + 1];
  }
};

// where canon(t, i, node + LOADSHIFT v_i) lives, for a given step mode
template <int MODE> struct Pattern;
template <> struct Pattern<MODE_PULL> {
  static constexpr int load_shift = -1, store_shift = 0;
  __host__ __device__ static constexpr int load_plane(int i) { return i; }
  __host__ __device__ static constexpr int store_plane(int i) { return i; }
};
template <> struct Pattern<MODE_AA_EVEN> {
  static constexpr int load_shift = 0, store_shift = 0;
  __host__ __device__ static constexpr int load_plane(int i) { return i; }
  __host__ __device__ static constexpr int store_plane(int i) { return 26 - i; }
};
template <> struct Pattern<MODE_AA_ODD> {
  static constexpr int load_shift = -1, store_shift = 1;
  __host__ __device__ static constexpr int load_plane(int i) { return 26 - i; }
  __host__ __device__ static constexpr int store_plane(int i) { return i; }
};

// compile-time loop over the 27 velocities
template <int I, int N> struct Unroll {
  template <typename F> __device__ __forceinline__ static void run(F&& f) {
    f(std::integral_constant<int, I>{});
    Unroll<I + 1, N>::run(f);
  }
};
template <int N> struct Unroll<N, N> {
  template <typename F> __device__ __forceinline__ static void run(F&&) {}
};

// FP64 collision of one node whose FP32 <dh|dh> fell under kDenFp64, after the step kernel:
// loads the node's inputs where the step's pattern keeps them (pull: src, which the step
// does not write; AA: the node's own slots, which the step left alone), collides them in
// FP64 (collide<double>, with the oracle's guard) and stores the outputs in the storage type.
// Returns gamma; *guarded is set when <dh|dh> fell under the FP64 guard.
template <typename S, int MODE, bool CENTRAL, bool POLY>
__device__ __noinline__ float fp64_node_update(const S* src, S* dst, Geo g, uint32_t x,
                                               uint32_t y, uint32_t z, CollideParams cp,
                                               int* guarded) {
  using C = Codec<S>;
  using Pat = Pattern<MODE>;
  Nbr nb;
  nb.init(g, x, y, z);
  double d[27];
  Unroll<0, 27>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    d[I] = C::to_delta(
        src[(uint64_t)Pat::load_plane(I) * g.P + nb.template at<I, Pat::load_shift>()], I);
  });
  int gd = 0;
  const double gam = collide<double, CENTRAL, false, POLY>(d, cp, &gd);
  Unroll<0, 27>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    dst[(uint64_t)Pat::store_plane(I) * g.P + nb.template at<I, Pat::store_shift>()] =
        C::from_delta(d[I], I);
  });
  *guarded = gd;
  return (float)gam;
}

// ------------------------------------------------------------------ the fused node update
// Loads f(x, t) of node (x, y, z) by the pattern of MODE, collides, stores f'(x) where
// f(t+1) expects it. src and dst are the same buffer in the AA modes.
template <typename S, int MODE, bool RECORD, bool CENTRAL = false, bool EXACT = false,
          bool POLY = false>
__device__ __forceinline__ void node_update(const S* src, S* dst, const Geo& g, uint32_t x,
                                            uint32_t y, uint32_t z, const CollideParams& cp,
                                            float* gamma_out, StepCounters* ctr) {
  using C = Codec<S>;
  using R = typename C::R;
  using Pat = Pattern<MODE>;
  Nbr nb;
  nb.init(g, x, y, z);
  R d[27];
  Unroll<0, 27>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    const S* p = src + (uint64_t)Pat::load_plane(I) * g.P + nb.template at<I, Pat::load_shift>();
    if constexpr (MODE == MODE_PULL) {
      d[I] = C::template load_raw_ro<I>(p);
    } else {
      d[I] = C::template load_raw<I>(p);
    }
  });
  int guarded, fp64 = 0;
  R gamma = collide_step<R, CENTRAL, EXACT, POLY, C::rel>(
      d, cp, &guarded, std::is_same<S, float>::value ? &fp64 : nullptr);
  if (MODE == MODE_PULL || !fp64) {  // a flagged node is left to the FP64 pass (AA: not stored)
    Unroll<0, 27>::run([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      S* p = dst + (uint64_t)Pat::store_plane(I) * g.P + nb.template at<I, Pat::store_shift>();
      C::template store_raw<I>(p, d[I]);
    });
  }
  if (fp64) flag_fp64(g, nb.ox[1] + nb.oy[1] + nb.oz[1]);
  if constexpr (RECORD) {
    gamma_out[nb.ox[1] + nb.oy[1] + nb.oz[1]] = (float)gamma;
    if (guarded) atomicAdd(&ctr->guarded, 1ull);
  }
}

// Two nodes per thread, a = (xa, ya, za) and b = (xb, yb, zb), laid out so that every load
// and store instruction of a warp stays coalesced (b = a + 32 in the node order); the
// collision runs once on float2 lanes with packed FP32x2 instructions. When b is outside the
// box or the work unit (vb false) the caller passes b = a: lane 1 recomputes node a and is
// not stored. SAME_ROW: b lies in a's row (yb = ya, zb = za), which keeps fewer coordinates
// live. FP32 arithmetic only (S = float or uint16_t).
template <typename S, int MODE, bool RECORD, bool CENTRAL = false, bool POLY = false,
          bool SAME_ROW = true>
__device__ __forceinline__ void node_update2(const S* src, S* dst, const Geo& g, uint32_t xa,
                                             uint32_t ya, uint32_t za, uint32_t xb,
                                             uint32_t yb, uint32_t zb, bool vb,
                                             const CollideParams& cp, float* gamma_out,
                                             StepCounters* ctr) {
  using C = Codec<S>;
  using Pat = Pattern<MODE>;
  static_assert(std::is_same<typename C::R, float>::value, "FP32 arithmetic only");
  if constexpr (SAME_ROW) {
    yb = ya;
    zb = za;
  }
  Nbr na, nb;
  na.init(g, xa, ya, za);
  nb.init(g, xb, yb, zb);
  float2 d[27];
  Unroll<0, 27>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    const S* base = src + (uint64_t)Pat::load_plane(I) * g.P;
    d[I] = Codec2<S>::template load<I, MODE == MODE_PULL>(
        base + na.template at<I, Pat::load_shift>(), base + nb.template at<I, Pat::load_shift>());
  });
  int guarded, fp64 = 0;
  float2 gamma = collide_step<float2, CENTRAL, false, POLY, C::rel>(
      d, cp, &guarded, std::is_same<S, float>::value ? &fp64 : nullptr);
  // flagged lanes are left to the FP64 pass (AA: not stored)
  const bool va = MODE == MODE_PULL || !(fp64 & 1);
  const bool vbs = vb && (MODE == MODE_PULL || !(fp64 & 2));
  // In the AA modes the stores reuse the load addresses' planes; opaque copies of P and dst
  // make the compiler recompute the store addresses instead of keeping 27 64-bit addresses
  // live across the collision (which spilled at 3 blocks per SM).
  // The odd AA step also stores to the 27 neighbours: its neighbour offsets are rebuilt from
  // opaque copies of the coordinates rather than kept live across the collision.
  uint64_t Ps = g.P;
  S* dsts = dst;
  if constexpr (MODE != MODE_PULL) asm volatile("" : "+l"(Ps), "+l"(dsts));
  Nbr sa = na, sb = nb;
  if constexpr (MODE == MODE_AA_ODD) {
    if constexpr (SAME_ROW) {
      uint32_t xa2 = xa, xb2 = xb, y2 = ya, z2 = za;
      asm volatile("" : "+r"(xa2), "+r"(xb2), "+r"(y2), "+r"(z2));
      sa.init(g, xa2, y2, z2);
      sb.init(g, xb2, y2, z2);
    } else {
      uint32_t xa2 = xa, xb2 = xb, ya2 = ya, za2 = za, yb2 = yb, zb2 = zb;
      asm volatile("" : "+r"(xa2), "+r"(xb2), "+r"(ya2), "+r"(za2), "+r"(yb2), "+r"(zb2));
      sa.init(g, xa2, ya2, za2);
      sb.init(g, xb2, yb2, zb2);
    }
  }
  Unroll<0, 27>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    S* base = dsts + (uint64_t)Pat::store_plane(I) * Ps;
    Codec2<S>::template store<I>(base + sa.template at<I, Pat::store_shift>(),
                                 base + sb.template at<I, Pat::store_shift>(), va, vbs, d[I]);
  });
  if (fp64) {
    if (fp64 & 1) flag_fp64(g, na.ox[1] + na.oy[1] + na.oz[1]);
    if ((fp64 & 2) && vb) flag_fp64(g, nb.ox[1] + nb.oy[1] + nb.oz[1]);
  }
  if constexpr (RECORD) {
    gamma_out[na.ox[1] + na.oy[1] + na.oz[1]] = gamma.x;
    if (vb) gamma_out[nb.ox[1] + nb.oy[1] + nb.oz[1]] = gamma.y;
    const int n = __popc(guarded & (vb ? 3 : 1));
    if (n) atomicAdd(&ctr->guarded, (unsigned long long)n);
  }
}

// Two adjacent nodes (x, x + 1) of one row per thread (x even, nx even), the collision on
// FP32x2 lanes: the planes the pattern does not shift in x are read and, for the pull and the
// even AA step, written as one 32/64-bit access per plane; the x-shifted ones as two scalar
// accesses. The 9 neighbour rows are addressed from 3 + 3 row offsets and 3 x positions,
// which keeps fewer registers live than two full neighbourhoods. FP32 arithmetic only.
template <typename S, int MODE, bool RECORD>
__device__ __forceinline__ void node_update_adj(const S* src, S* dst, const Geo& g, uint32_t x,
                                                uint32_t y, uint32_t z, const CollideParams& cp,
                                                float* gamma_out, StepCounters* ctr) {
  using C = Codec<S>;
  using Pat = Pattern<MODE>;
  using IO = PairIO<S>;
  static_assert(std::is_same<typename C::R, float>::value, "FP32 arithmetic only");
  uint32_t oy[3], oz[3];
  oy[0] = (y == 0 ? g.ny - 1 : y - 1) * g.nx;
  oy[1] = y * g.nx;
  oy[2] = (y + 1 == g.ny ? 0 : y + 1) * g.nx;
  oz[0] = (z == 0 ? g.nz - 1 : z - 1) * g.nxy;
  oz[1] = z * g.nxy;
  oz[2] = (z + 1 == g.nz ? 0 : z + 1) * g.nxy;
  uint32_t xm = x == 0 ? g.nx - 1 : x - 1;
  uint32_t xp2 = x + 2 == g.nx ? 0 : x + 2;
  float2 d[27];
  Unroll<0, 27>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    constexpr int LS = Pat::load_shift;
    const S* row = src + (uint64_t)Pat::load_plane(I) * g.P + oy[LS * cy(I) + 1] +
                   oz[LS * cz(I) + 1];
    d[I] = IO::template get<LS * cx(I), MODE == MODE_PULL>(row + x, row + xm, row + xp2);
  });
  int guarded, fp64 = 0;
  float2 gamma = collide_step<float2, false, false, false, C::rel>(
      d, cp, &guarded, std::is_same<S, float>::value ? &fp64 : nullptr);
  // flagged lanes are left to the FP64 pass; the pull step stores them anyway (the pass
  // overwrites them from src), the AA step does not
  const int skip = MODE == MODE_PULL ? 0 : fp64;
  const bool wa = !(skip & 1), wb = !(skip & 2);
  // AA: opaque copies of P and dst keep the compiler from holding 27 addresses across the
  // collision
  uint64_t Ps = g.P;
  S* dsts = dst;
  if constexpr (MODE != MODE_PULL) asm volatile("" : "+l"(Ps), "+l"(dsts));
  if constexpr (MODE == MODE_AA_ODD) {
    // the odd step stores to the neighbours: their row offsets and x positions are rebuilt
    // from opaque copies of the coordinates rather than kept live across the collision
    uint32_t x2 = x, y2 = y, z2 = z;
    asm volatile("" : "+r"(x2), "+r"(y2), "+r"(z2));
    oy[0] = (y2 == 0 ? g.ny - 1 : y2 - 1) * g.nx;
    oy[1] = y2 * g.nx;
    oy[2] = (y2 + 1 == g.ny ? 0 : y2 + 1) * g.nx;
    oz[0] = (z2 == 0 ? g.nz - 1 : z2 - 1) * g.nxy;
    oz[1] = z2 * g.nxy;
    oz[2] = (z2 + 1 == g.nz ? 0 : z2 + 1) * g.nxy;
    xm = x2 == 0 ? g.nx - 1 : x2 - 1;
    xp2 = x2 + 2 == g.nx ? 0 : x2 + 2;
  }
  Unroll<0, 27>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    constexpr int SS = Pat::store_shift;
    S* row = dsts + (uint64_t)Pat::store_plane(I) * Ps + oy[SS * cy(I) + 1] + oz[SS * cz(I) + 1];
    constexpr int SX = SS * cx(I);
    if constexpr (SX == 0) {
      if (!skip) {
        IO::put2(row + x, d[I]);
      } else {
        if (wa) IO::put1(row + x, d[I].x);
        if (wb) IO::put1(row + x + 1, d[I].y);
      }
    } else if constexpr (SX > 0) {
      if (wa) IO::put1(row + x + 1, d[I].x);
      if (wb) IO::put1(row + xp2, d[I].y);
    } else {
      if (wa) IO::put1(row + xm, d[I].x);
      if (wb) IO::put1(row + x, d[I].y);
    }
  });
  if (fp64) {
    if (fp64 & 1) flag_fp64(g, oy[1] + oz[1] + x);
    if (fp64 & 2) flag_fp64(g, oy[1] + oz[1] + x + 1);
  }
  if constexpr (RECORD) {
    *reinterpret_cast<float2*>(gamma_out + oy[1] + oz[1] + x) = gamma;
    const int n = __popc(guarded & 3);
    if (n) atomicAdd(&ctr->guarded, (unsigned long long)n);
  }
}

}  // namespace kbc
