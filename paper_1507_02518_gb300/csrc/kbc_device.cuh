// kbc_device.cuh -- device-side building blocks of the D3Q27 KBC step (sm_103a).
//
// Method: arXiv:1507.02518, Sec. KBC (collision listing, Table 1, eq:result21) with the
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
#include <stdint.h>

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
template <typename S> struct Codec;

template <> struct Codec<double> {
  using R = double;
  template <int I> __device__ static __forceinline__ R load(const double* p) { return *p; }
  template <int I> __device__ static __forceinline__ R load_ro(const double* p) { return __ldg(p); }
  template <int I> __device__ static __forceinline__ void store(double* p, R d) { *p = d; }
  __host__ __device__ static double to_delta(double s, int) { return s; }
  __host__ __device__ static double from_delta(double d, int) { return d; }
};

template <> struct Codec<float> {
  using R = float;
  template <int I> __device__ static __forceinline__ R load(const float* p) { return *p; }
  template <int I> __device__ static __forceinline__ R load_ro(const float* p) { return __ldg(p); }
  template <int I> __device__ static __forceinline__ void store(float* p, R d) { *p = d; }
  __device__ static double to_delta(float s, int) { return (double)s; }
  __device__ static float from_delta(double d, int) { return (float)d; }
};

// FP16: the stored half is (f_i - W_i) / W_i, rounded to nearest even. Keeping the value
// relative to W_i keeps every direction clear of the half subnormal range.
template <> struct Codec<uint16_t> {
  using R = float;
  template <int I> __device__ static __forceinline__ R load(const uint16_t* p) {
    return (float)wgt(I) * __half2float(__ushort_as_half(*p));
  }
  template <int I> __device__ static __forceinline__ R load_ro(const uint16_t* p) {
    return (float)wgt(I) * __half2float(__ushort_as_half(__ldg(p)));
  }
  template <int I> __device__ static __forceinline__ void store(uint16_t* p, R d) {
    *p = __half_as_ushort(__float2half_rn(d * (float)inv_wgt(I)));
  }
  __device__ static double to_delta(uint16_t s, int i) {
    return wgt(i) * (double)__half2float(__ushort_as_half(s));
  }
  __device__ static uint16_t from_delta(double d, int i) {
    return __half_as_ushort(__double2half(d * inv_wgt(i)));
  }
};

// ------------------------------------------------------------------ numeric helpers
template <typename R> __device__ __forceinline__ R rsq(R x);
template <> __device__ __forceinline__ float rsq<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double rsq<double>(double x) { return sqrt(x); }

// three reciprocals with one division: 1/p0 = p1 p2 / (p0 p1 p2), ...
template <typename R>
__device__ __forceinline__ void recip3(R p0, R p1, R p2, R& r0, R& r1, R& r2) {
  const R p12 = p1 * p2;
  const R q = R(1) / (p0 * p12);
  r0 = p12 * q;
  const R qp0 = q * p0;
  r1 = p2 * qp0;
  r2 = p1 * qp0;
}

// guard on <dh|dh> (the paper is silent when it vanishes; gamma falls back to 2, LBGK)
template <typename R> struct Guard;
template <> struct Guard<double> { static constexpr double den = 1e-300; };
template <> struct Guard<float> { static constexpr float den = 1e-30f; };

enum { GAMMA_ESTIMATE = 0, GAMMA_LBGK = 1, GAMMA_RLB = 2 };

struct CollideParams {
  double beta;      // relaxation parameter of eq:Egeneral
  double two_beta;  // 2 beta
  double inv_beta;  // 1 / beta
  int with_t;       // shear part includes t (Table 1)
  int with_q;       // shear part includes q (Table 1)
  int gamma_mode;   // GAMMA_*
};

// One KBC collision on the shifted populations d[i] = f_i - W_i, in place (collision
// listing of Sec. KBC). Returns gamma; *guarded is set when <dh|dh> fell under the guard.
template <typename R>
__device__ __forceinline__ R collide(R (&d)[27], const CollideParams& cp, bool* guarded) {
  // ---- natural moments of delta by a factorised x -> y -> z reduction (eq:natmoments)
  // row r = (vy+1) + 3(vz+1); X0 = sum over vx, X1 = sum vx, X2 = sum vx^2
  R X0[9], X1[9], X2[9];
#pragma unroll
  for (int r = 0; r < 9; ++r) {
    const R m = d[3 * r + 0], z = d[3 * r + 1], p = d[3 * r + 2];
    X2[r] = p + m;
    X1[r] = p - m;
    X0[r] = X2[r] + z;
  }
  // y stage: Yp_q[c] = sum over vy of Xp * vy^q, c = vz+1
  auto ystage = [](const R (&X)[9], R (&Y0)[3], R (&Y1)[3], R (&Y2)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R m = X[3 * c + 0], z = X[3 * c + 1], p = X[3 * c + 2];
      Y2[c] = p + m;
      Y1[c] = p - m;
      Y0[c] = Y2[c] + z;
    }
  };
  R Y00[3], Y01[3], Y02[3], Y10[3], Y11[3], Y12[3], Y20[3], Y21[3], Y22[3];
  ystage(X0, Y00, Y01, Y02);
  ystage(X1, Y10, Y11, Y12);
  ystage(X2, Y20, Y21, Y22);
  (void)Y22;
  // z stage: D_pqr = sum over vz of Ypq * vz^r
  const R D000 = Y00[0] + Y00[1] + Y00[2], D001 = Y00[2] - Y00[0], D002 = Y00[2] + Y00[0];
  const R D100 = Y10[0] + Y10[1] + Y10[2], D101 = Y10[2] - Y10[0], D102 = Y10[2] + Y10[0];
  const R D010 = Y01[0] + Y01[1] + Y01[2], D011 = Y01[2] - Y01[0], D012 = Y01[2] + Y01[0];
  const R D200 = Y20[0] + Y20[1] + Y20[2], D201 = Y20[2] - Y20[0];
  const R D020 = Y02[0] + Y02[1] + Y02[2], D021 = Y02[2] - Y02[0];
  const R D110 = Y11[0] + Y11[1] + Y11[2], D111 = Y11[2] - Y11[0];
  const R D120 = Y12[0] + Y12[1] + Y12[2];
  const R D210 = Y21[0] + Y21[1] + Y21[2];

  // ---- conserved quantities (listing step 1); sum W = 1, sum W v = 0
  const R drho = D000;
  const R rho = R(1) + drho;
  const R ir = R(1) / rho;
  const R ux = D100 * ir, uy = D010 * ir, uz = D001 * ir;

  // ---- per-axis equilibrium factors (listing step 2)
  const R Rx = rsq<R>(R(1) + R(3) * ux * ux);
  const R Ry = rsq<R>(R(1) + R(3) * uy * uy);
  const R Rz = rsq<R>(R(1) + R(3) * uz * uz);
  const R ex = R(3) * ux * ux / (R(1) + Rx);   // R - 1 without cancellation
  const R ey = R(3) * uy * uy / (R(1) + Ry);
  const R ez = R(3) * uz * uz / (R(1) + Rz);
  const R m2x = R(1.0 / 3.0) + R(2.0 / 3.0) * ex;  // m_2(u) = (2R - 1)/3
  const R m2y = R(1.0 / 3.0) + R(2.0 / 3.0) * ey;
  const R m2z = R(1.0 / 3.0) + R(2.0 / 3.0) * ez;

  // ---- rho-scaled moment deviations rho (M - M_eq) (listing steps 3-4)
  const R d3 = drho * R(1.0 / 3.0);
  const R A200 = (D200 - d3) - rho * (R(2.0 / 3.0) * ex);
  const R A020 = (D020 - d3) - rho * (R(2.0 / 3.0) * ey);
  const R A002 = (D002 - d3) - rho * (R(2.0 / 3.0) * ez);
  const R ANxz = A200 - A002, ANyz = A020 - A002;
  const R AT = cp.with_t ? (A200 + A020 + A002) : R(0);
  const R APxy = D110 - D100 * uy, APxz = D101 - D100 * uz, APyz = D011 - D010 * uz;
  const R qs = cp.with_q ? R(1) : R(0);
  const R AQxyy = qs * (D120 - D100 * m2y), AQxzz = qs * (D102 - D100 * m2z);
  const R AQxxy = qs * (D210 - D010 * m2x), AQyzz = qs * (D012 - D010 * m2z);
  const R AQxxz = qs * (D201 - D001 * m2x), AQyyz = qs * (D021 - D001 * m2y);
  const R AQxyz = qs * (D111 - D100 * uy * uz);

  // Table 1 per velocity class: ds = d + t + q evaluated on the deviations
  const R s0 = -AT;
  const R Fx = (R(2) * ANxz - ANyz + AT) * R(1.0 / 6.0), Gx = (AQxyy + AQxzz) * R(0.5);
  const R Fy = (R(2) * ANyz - ANxz + AT) * R(1.0 / 6.0), Gy = (AQxxy + AQyzz) * R(0.5);
  const R Fz = (AT - ANxz - ANyz) * R(1.0 / 6.0), Gz = (AQxxz + AQyyz) * R(0.5);
  const R Pxy4 = R(0.25) * APxy, Pxz4 = R(0.25) * APxz, Pyz4 = R(0.25) * APyz;
  const R Qxxy4 = R(0.25) * AQxxy, Qxyy4 = R(0.25) * AQxyy, Qxxz4 = R(0.25) * AQxxz;
  const R Qxzz4 = R(0.25) * AQxzz, Qyyz4 = R(0.25) * AQyyz, Qyzz4 = R(0.25) * AQyzz;
  const R Qxyz8 = R(0.125) * AQxyz;
  auto ds_of = [&](int a, int b, int c) -> R {
    const int nnz = (a != 0) + (b != 0) + (c != 0);
    if (nnz == 0) return s0;
    if (nnz == 1) {
      if (a != 0) return a > 0 ? Fx - Gx : Fx + Gx;
      if (b != 0) return b > 0 ? Fy - Gy : Fy + Gy;
      return c > 0 ? Fz - Gz : Fz + Gz;
    }
    if (nnz == 2) {
      if (c == 0) return R(a * b) * Pxy4 + R(b) * Qxxy4 + R(a) * Qxyy4;
      if (b == 0) return R(a * c) * Pxz4 + R(c) * Qxxz4 + R(a) * Qxzz4;
      return R(b * c) * Pyz4 + R(c) * Qyyz4 + R(b) * Qyzz4;
    }
    return R(a * b * c) * Qxyz8;
  };

  // equilibrium factors: rho phi_x(a) = W_a (1 + gx_a), phi_y(b) = W_b (1 + ey_b), ...
  const R gx[3] = {drho + (R(2) * ex - R(3) * ux) * rho, drho - ex * rho,
                   drho + (R(2) * ex + R(3) * ux) * rho};
  const R fy[3] = {R(2) * ey - R(3) * uy, -ey, R(2) * ey + R(3) * uy};
  const R fz[3] = {R(2) * ez - R(3) * uz, -ez, R(2) * ez + R(3) * uz};
  // reciprocal weights of the entropic scalar product, 1/f_eq_i = rx[a] ry[b] rz[c]
  R rx[3], ry[3], rz[3];
  recip3<R>(R(1.0 / 6.0) * (R(1) + gx[0]), R(2.0 / 3.0) * (R(1) + gx[1]),
            R(1.0 / 6.0) * (R(1) + gx[2]), rx[0], rx[1], rx[2]);
  recip3<R>(R(1.0 / 6.0) * (R(1) + fy[0]), R(2.0 / 3.0) * (R(1) + fy[1]),
            R(1.0 / 6.0) * (R(1) + fy[2]), ry[0], ry[1], ry[2]);
  recip3<R>(R(1.0 / 6.0) * (R(1) + fz[0]), R(2.0 / 3.0) * (R(1) + fz[1]),
            R(1.0 / 6.0) * (R(1) + fz[2]), rz[0], rz[1], rz[2]);

  // ---- dh, the two entropic products, and the part of the relaxation known before gamma
  // (listing steps 5-6): d <- d - 2 beta ds, dh kept for the gamma-dependent part
  const R b2 = R(cp.two_beta);
  R dh[27];
  R num = R(0), den = R(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R cn = R(0), cd = R(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const R Pab0 = gx[0] + fy[b] + gx[0] * fy[b];
      const R Pab1 = gx[1] + fy[b] + gx[1] * fy[b];
      const R Pab2 = gx[2] + fy[b] + gx[2] * fy[b];
      const R Pab[3] = {Pab0, Pab1, Pab2};
      R rn = R(0), rd = R(0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int i = a + 3 * b + 9 * c;
        const R G = Pab[a] + fz[c] + Pab[a] * fz[c];      // (f_eq_i - W_i) / W_i
        const R dsi = ds_of(a - 1, b - 1, c - 1);
        const R dhi = d[i] - R(wgt(i)) * G - dsi;
        const R t1 = rx[a] * dhi;
        rn += t1 * dsi;
        rd += t1 * dhi;
        dh[i] = dhi;
        d[i] -= b2 * dsi;
      }
      cn += ry[b] * rn;
      cd += ry[b] * rd;
    }
    num += rz[c] * cn;
    den += rz[c] * cd;
  }

  // ---- stabilizer (eq:result21) and the rest of the relaxation (listing step 7)
  const R ib = R(cp.inv_beta);
  R gamma;
  *guarded = false;
  if (cp.gamma_mode == GAMMA_LBGK) {
    gamma = R(2);
  } else if (cp.gamma_mode == GAMMA_RLB) {
    gamma = ib;
  } else if (den > Guard<R>::den) {
    gamma = ib - (R(2) - ib) * (num / den);
  } else if (den == den) {
    gamma = R(2);
    *guarded = true;
  } else {
    gamma = den;  // NaN propagates to the populations and to the diagnostics
  }
  const R bg = R(cp.beta) * gamma;
#pragma unroll
  for (int i = 0; i < 27; ++i) d[i] -= bg * dh[i];
  return gamma;
}

// Equilibrium shift f_eq_i(rho, u) - W_i by the same per-axis closed form, in FP64.
__device__ __forceinline__ void equilibrium_shift(double rho, double ux, double uy, double uz,
                                                  double (&out)[27]) {
  const double drho = rho - 1.0;
  const double Rx = sqrt(1.0 + 3.0 * ux * ux), Ry = sqrt(1.0 + 3.0 * uy * uy),
               Rz = sqrt(1.0 + 3.0 * uz * uz);
  const double ex = 3.0 * ux * ux / (1.0 + Rx), ey = 3.0 * uy * uy / (1.0 + Ry),
               ez = 3.0 * uz * uz / (1.0 + Rz);
  const double gx[3] = {drho + (2.0 * ex - 3.0 * ux) * rho, drho - ex * rho,
                        drho + (2.0 * ex + 3.0 * ux) * rho};
  const double fy[3] = {2.0 * ey - 3.0 * uy, -ey, 2.0 * ey + 3.0 * uy};
  const double fz[3] = {2.0 * ez - 3.0 * uz, -ez, 2.0 * ez + 3.0 * uz};
#pragma unroll
  for (int i = 0; i < 27; ++i) {
    const double gxa = gx[cx(i) + 1], fyb = fy[cy(i) + 1], fzc = fz[cz(i) + 1];
    const double P = gxa + fyb + gxa * fyb;
    out[i] = wgt(i) * (P + fzc + P * fzc);
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
};

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

}  // namespace kbc
