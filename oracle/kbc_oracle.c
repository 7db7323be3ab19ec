/*
 * kbc_oracle.c -- plain FP64 CPU oracle of the D3Q27 KBC lattice Boltzmann step.
 *
 * TEST INFRASTRUCTURE ONLY: called by tests, by the package smoke check and by the
 * benchmark's CPU-baseline leg. The product (CUDA) path never links or calls it, and it
 * shares no code, header, table or constant with that path.
 *
 * Every function follows the paper (arXiv:1507.02518) in its own order and notation,
 * without factorisation or fusion:
 *   lattice, weights, sound speed ....... Sec. "Equilibrium on the standard lattice" (eq:D1Q3,
 *                                           eq:D3Q27vel, eq:weights, eq:sound)
 *   product-form equilibrium ............ eq:entropic_eq with A(u), B(u), Psi(u)
 *   natural moments ..................... eq:natmoments (straight sums over 27 velocities)
 *   moment representation of f .......... eq:moment_rep (Q labels read by counting powers)
 *   k / d / t / q parts ................. Table 1 (tab:s_parts)
 *   central moments and central parts ... Sec. "Moment System" and the appendix (eq:cm1-eq:cm23,
 *                                           eq:cmf000-eq:cmfxyz), as tensor products of the
 *                                           one-dimensional central inverse
 *   collision ........................... eq:Egeneral with the mirror state eq:ksh-mirror
 *                                           (Sec. KBC): with ds = s - s_eq and
 *                                           dh = h - h_eq = f - f_eq - ds (k = k_eq, since k
 *                                           depends on the conserved fields only),
 *                                           f' = (1 - beta) f + beta f_mirr
 *                                              = f - beta (2 ds + gamma dh),
 *                                           gamma from eq:result21
 *   mirror form ......................... eq:Egeneral with eq:ksh-mirror (second route)
 *   exact stabilizer .................... root of eq:result1 (Newton iteration)
 *   streaming ........................... left-hand side of eq:Egeneral, periodic box
 *   diagnostics ......................... Sec. "Numerical Simulations": k, Omega, epsilon
 *
 * Readings where the paper is silent: gamma = 2 when <dh|dh> <= ORC_DEN_GUARD; no clipping
 * of gamma. Compiled -O2 -ffp-contract=off, no fast-math.
 */
#include "kbc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* one-dimensional weights W_{-1}, W_0, W_{+1} (eq:sound and the line after it) */
static const double W1D[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};

/* component a (0=x,1=y,2=z) of velocity i, with i = (vx+1) + 3(vy+1) + 9(vz+1) */
static int vcomp(int i, int a) {
  if (a == 0) return i % 3 - 1;
  if (a == 1) return (i / 3) % 3 - 1;
  return i / 9 - 1;
}

/* integer power v^p for v in {-1,0,1}, p in {0,1,2}; 0^0 = 1 */
static double ipw(int v, int p) {
  double r = 1.0;
  for (int k = 0; k < p; ++k) r *= (double)v;
  return r;
}

static double weight(int i) {
  return W1D[vcomp(i, 0) + 1] * W1D[vcomp(i, 1) + 1] * W1D[vcomp(i, 2) + 1]; /* eq:weights */
}

void orc_lattice(int32_t *v, double *w) {
  for (int i = 0; i < 27; ++i) {
    for (int a = 0; a < 3; ++a) v[3 * i + a] = vcomp(i, a);
    w[i] = weight(i);
  }
}

/* eq:viscosity with c_s^2 = 1/3 (eq:sound): nu = (1/3)(1/(2 beta) - 1/2) => beta = 1/(6 nu + 1) */
double orc_beta(double nu) { return 1.0 / (6.0 * nu + 1.0); }

static double fA(double u) { return 2.0 - sqrt(1.0 + 3.0 * u * u); }
static double fB(double u) { return (2.0 * u + sqrt(1.0 + 3.0 * u * u)) / (1.0 - u); }
static double bpow(double b, int e) { return e == 0 ? 1.0 : (e > 0 ? b : 1.0 / b); }

/* eq:entropic_eq: f_i = rho W_i Psi B(ux)^vix B(uy)^viy B(uz)^viz, Psi = A(ux)A(uy)A(uz) */
void orc_equilibrium(double rho, const double *u, double *feq) {
  const double psi = fA(u[0]) * fA(u[1]) * fA(u[2]);
  const double bx = fB(u[0]), by = fB(u[1]), bz = fB(u[2]);
  for (int i = 0; i < 27; ++i) {
    feq[i] = rho * weight(i) * psi * bpow(bx, vcomp(i, 0)) * bpow(by, vcomp(i, 1)) *
             bpow(bz, vcomp(i, 2));
  }
}

/* eq:polynomial2 with c_s^2 = 1/3 (eq:sound):
 * rho W_i (1 + (u.v_i)/c_s^2 + ((u.v_i)^2 - c_s^2 u.u) / (2 c_s^4)) */
void orc_equilibrium_poly2(double rho, const double *u, double *feq) {
  const double cs2 = 1.0 / 3.0;
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < 27; ++i) {
    const double uv = u[0] * vcomp(i, 0) + u[1] * vcomp(i, 1) + u[2] * vcomp(i, 2);
    feq[i] = rho * weight(i) * (1.0 + uv / cs2 + (uv * uv - cs2 * uu) / (2.0 * cs2 * cs2));
  }
}

static void equilibrium_of(int variant, double rho, const double *u, double *feq) {
  if (variant & ORC_EQ_POLY2)
    orc_equilibrium_poly2(rho, u, feq);
  else
    orc_equilibrium(rho, u, feq);
}

/* eq:natmoments: rho M_pqr = sum_i f_i vix^p viy^q viz^r; M stored at [p*9 + q*3 + r] */
void orc_moments(const double *f, double *rho, double *M) {
  double r = 0.0;
  for (int i = 0; i < 27; ++i) r += f[i];
  *rho = r;
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q)
      for (int s = 0; s < 3; ++s) {
        double acc = 0.0;
        for (int i = 0; i < 27; ++i)
          acc += f[i] * ipw(vcomp(i, 0), p) * ipw(vcomp(i, 1), q) * ipw(vcomp(i, 2), s);
        M[p * 9 + q * 3 + s] = acc / r;
      }
}

#define MM(p, q, r) M[(p) * 9 + (q) * 3 + (r)]

/* Table 1: kinematic part k and the shear-part groups d, t, q for every velocity. */
void orc_table1(const double *M, double rho, double *k, double *d, double *t, double *q) {
  const double ux = MM(1, 0, 0), uy = MM(0, 1, 0), uz = MM(0, 0, 1);
  /* renamed moments (Sec. "Moment System for D3Q27") */
  const double T = MM(2, 0, 0) + MM(0, 2, 0) + MM(0, 0, 2);
  const double Nxz = MM(2, 0, 0) - MM(0, 0, 2);
  const double Nyz = MM(0, 2, 0) - MM(0, 0, 2);
  const double Pxy = MM(1, 1, 0), Pxz = MM(1, 0, 1), Pyz = MM(0, 1, 1);
  const double Qxyy = MM(1, 2, 0), Qxzz = MM(1, 0, 2), Qxxy = MM(2, 1, 0);
  const double Qyzz = MM(0, 1, 2), Qxxz = MM(2, 0, 1), Qyyz = MM(0, 2, 1);
  const double Qxyz = MM(1, 1, 1);
  for (int i = 0; i < 27; ++i) {
    const int sx = vcomp(i, 0), sy = vcomp(i, 1), sz = vcomp(i, 2);
    double kk = 0.0, dd = 0.0, tt = 0.0, qq = 0.0;
    if (sx == 0 && sy == 0 && sz == 0) {               /* (0,0,0) */
      kk = 1.0;
      tt = -T;
    } else if (sy == 0 && sz == 0) {                   /* (sigma,0,0) */
      kk = sx * ux / 2.0;
      dd = (2.0 * Nxz - Nyz) / 6.0;
      tt = T / 6.0;
      qq = -sx * (Qxyy + Qxzz) / 2.0;
    } else if (sx == 0 && sz == 0) {                   /* (0,lambda,0) */
      kk = sy * uy / 2.0;
      dd = (-Nxz + 2.0 * Nyz) / 6.0;
      tt = T / 6.0;
      qq = -sy * (Qxxy + Qyzz) / 2.0;
    } else if (sx == 0 && sy == 0) {                   /* (0,0,delta) */
      kk = sz * uz / 2.0;
      dd = (-Nxz - Nyz) / 6.0;
      tt = T / 6.0;
      qq = -sz * (Qxxz + Qyyz) / 2.0;
    } else if (sz == 0) {                              /* (sigma,lambda,0) */
      dd = sx * sy * Pxy / 4.0;
      qq = (sy * Qxxy + sx * Qxyy) / 4.0;
    } else if (sy == 0) {                              /* (sigma,0,delta) */
      dd = sx * sz * Pxz / 4.0;
      qq = (sz * Qxxz + sx * Qxzz) / 4.0;
    } else if (sx == 0) {                              /* (0,lambda,delta) */
      dd = sy * sz * Pyz / 4.0;
      qq = (sz * Qyyz + sy * Qyzz) / 4.0;
    } else {                                           /* (sigma,lambda,delta) */
      qq = sx * sy * sz * Qxyz / 8.0;
    }
    k[i] = rho * kk;
    d[i] = rho * dd;
    t[i] = rho * tt;
    q[i] = rho * qq;
  }
}

/* eq:moment_rep: the 27 populations written in the natural-moment basis. */
void orc_moment_rep(const double *M, double rho, double *f) {
  const double ux = MM(1, 0, 0), uy = MM(0, 1, 0), uz = MM(0, 0, 1);
  const double T = MM(2, 0, 0) + MM(0, 2, 0) + MM(0, 0, 2);
  const double Nxz = MM(2, 0, 0) - MM(0, 0, 2);
  const double Nyz = MM(0, 2, 0) - MM(0, 0, 2);
  const double Pxy = MM(1, 1, 0), Pxz = MM(1, 0, 1), Pyz = MM(0, 1, 1);
  const double Qxyy = MM(1, 2, 0), Qxzz = MM(1, 0, 2), Qxxy = MM(2, 1, 0);
  const double Qyzz = MM(0, 1, 2), Qxxz = MM(2, 0, 1), Qyyz = MM(0, 2, 1);
  const double Qxyz = MM(1, 1, 1);
  const double M022 = MM(0, 2, 2), M202 = MM(2, 0, 2), M220 = MM(2, 2, 0), M222 = MM(2, 2, 2);
  const double M122 = MM(1, 2, 2), M212 = MM(2, 1, 2), M221 = MM(2, 2, 1);
  const double M112 = MM(1, 1, 2), M121 = MM(1, 2, 1), M211 = MM(2, 1, 1);
  for (int i = 0; i < 27; ++i) {
    const double s = vcomp(i, 0), l = vcomp(i, 1), d = vcomp(i, 2);
    double v;
    if (s == 0 && l == 0 && d == 0) {
      v = 1.0 - T + M022 + M202 + M220 - M222;
    } else if (l == 0 && d == 0) {
      v = (3 * s * ux + 2 * Nxz - Nyz + T - 3 * s * Qxyy - 3 * s * Qxzz + 3 * s * M122 -
           3 * M202 - 3 * M220 + 3 * M222) / 6.0;
    } else if (s == 0 && d == 0) {
      v = (3 * l * uy - Nxz + 2 * Nyz + T - 3 * l * Qxxy - 3 * l * Qyzz + 3 * l * M212 -
           3 * M022 - 3 * M220 + 3 * M222) / 6.0;
    } else if (s == 0 && l == 0) {
      v = (3 * d * uz - Nxz - Nyz + T - 3 * d * Qxxz - 3 * d * Qyyz + 3 * d * M221 -
           3 * M022 - 3 * M202 + 3 * M222) / 6.0;
    } else if (d == 0) {
      v = (s * l * Pxy + l * Qxxy + s * Qxyy + M220 - s * M122 - l * M212 - s * l * M112 -
           M222) / 4.0;
    } else if (l == 0) {
      v = (s * d * Pxz + d * Qxxz + s * Qxzz + M202 - s * M122 - d * M221 - s * d * M121 -
           M222) / 4.0;
    } else if (s == 0) {
      v = (l * d * Pyz + d * Qyyz + l * Qyzz + M022 - l * M212 - d * M221 - l * d * M211 -
           M222) / 4.0;
    } else {
      v = (s * l * d * Qxyz + s * M122 + l * M212 + d * M221 + s * l * M112 + s * d * M121 +
           l * d * M211 + M222) / 8.0;
    }
    f[i] = rho * v;
  }
}
#undef MM

/* Central moments (Sec. "Moment System for D3Q27"):
 * rho Mc_pqr = sum_i f_i (vix - ux)^p (viy - uy)^q (viz - uz)^r, stored at [p*9 + q*3 + r]. */
void orc_central_moments(const double *f, double *rho, double *u, double *Mc) {
  double r = 0.0, m[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < 27; ++i) {
    r += f[i];
    for (int a = 0; a < 3; ++a) m[a] += vcomp(i, a) * f[i];
  }
  *rho = r;
  for (int a = 0; a < 3; ++a) u[a] = m[a] / r;
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q)
      for (int s = 0; s < 3; ++s) {
        double acc = 0.0;
        for (int i = 0; i < 27; ++i) {
          double w = f[i];
          for (int k = 0; k < p; ++k) w *= vcomp(i, 0) - u[0];
          for (int k = 0; k < q; ++k) w *= vcomp(i, 1) - u[1];
          for (int k = 0; k < s; ++k) w *= vcomp(i, 2) - u[2];
          acc += w;
        }
        Mc[p * 9 + q * 3 + s] = acc / r;
      }
}

/* One-dimensional central inverse: coefficient of the p-th central moment in the population of
 * velocity v, i.e. the inverse of the 3x3 matrix ((v - u)^p). The populations of
 * eq:cmf000-eq:cmfxyz are its tensor products: f_abc = rho sum_pqr c(a;p) c(b;q) c(c;r) Mc_pqr. */
static double cinv(int v, int p, double u) {
  if (v == 0) return p == 0 ? 1.0 - u * u : (p == 1 ? -2.0 * u : -1.0);
  const double s = (double)v;
  return p == 0 ? u * (u + s) / 2.0 : (p == 1 ? (s + 2.0 * u) / 2.0 : 0.5);
}

/* Central-basis groups of every population (Sec. KBC, appendix): k~ from Mc_000 (the first
 * central moments vanish), d~ from the deviatoric stress (Pi~, N~), t~ from the trace T~,
 * q~ from the third-order Q~, h~ the remaining higher moments. With
 * Mc_200 = (T + 2Nxz - Nyz)/3, Mc_020 = (T - Nxz + 2Nyz)/3, Mc_002 = (T - Nxz - Nyz)/3. */
void orc_central_parts(const double *Mc, double rho, const double *u, double *k, double *d,
                       double *t, double *q, double *h) {
#define MC(p, q, r) Mc[(p) * 9 + (q) * 3 + (r)]
  const double T = MC(2, 0, 0) + MC(0, 2, 0) + MC(0, 0, 2);
  const double Nxz = MC(2, 0, 0) - MC(0, 0, 2), Nyz = MC(0, 2, 0) - MC(0, 0, 2);
  for (int i = 0; i < 27; ++i) {
    const int a = vcomp(i, 0), b = vcomp(i, 1), c = vcomp(i, 2);
    double C[27];
    for (int p = 0; p < 3; ++p)
      for (int qq = 0; qq < 3; ++qq)
        for (int r = 0; r < 3; ++r)
          C[p * 9 + qq * 3 + r] = cinv(a, p, u[0]) * cinv(b, qq, u[1]) * cinv(c, r, u[2]);
    const double c200 = C[18], c020 = C[6], c002 = C[2];
    k[i] = rho * (C[0] * MC(0, 0, 0) + C[9] * MC(1, 0, 0) + C[3] * MC(0, 1, 0) + C[1] * MC(0, 0, 1));
    t[i] = rho * T * (c200 + c020 + c002) / 3.0;
    d[i] = rho * (Nxz * (2.0 * c200 - c020 - c002) / 3.0 + Nyz * (-c200 + 2.0 * c020 - c002) / 3.0 +
                  C[12] * MC(1, 1, 0) + C[10] * MC(1, 0, 1) + C[4] * MC(0, 1, 1));
    q[i] = rho * (C[15] * MC(1, 2, 0) + C[11] * MC(1, 0, 2) + C[21] * MC(2, 1, 0) +
                  C[5] * MC(0, 1, 2) + C[19] * MC(2, 0, 1) + C[7] * MC(0, 2, 1) +
                  C[13] * MC(1, 1, 1));
    double rest = 0.0;
    const int hm[8] = {2 * 3 + 2, 2 * 9 + 2, 2 * 9 + 2 * 3, 1 * 9 + 2 * 3 + 2, 2 * 9 + 1 * 3 + 2,
                       2 * 9 + 2 * 3 + 1, 1 * 9 + 1 * 3 + 2, 1 * 9 + 2 * 3 + 1};
    for (int j = 0; j < 8; ++j) rest += C[hm[j]] * Mc[hm[j]];
    rest += C[2 * 9 + 1 * 3 + 1] * MC(2, 1, 1) + C[26] * MC(2, 2, 2);
    h[i] = rho * rest;
  }
#undef MC
}

static void shear_part(const double *d, const double *t, const double *q, int variant,
                       double *s) {
  const int v = variant & 3;
  const int with_t = (v == ORC_S_DT || v == ORC_S_DTQ);
  const int with_q = (v == ORC_S_DQ || v == ORC_S_DTQ);
  for (int i = 0; i < 27; ++i) s[i] = d[i] + (with_t ? t[i] : 0.0) + (with_q ? q[i] : 0.0);
}

/* k and the s groups of a population vector in the basis the variant names */
static void groups(const double *f, int variant, double *rho, double *u, double *k, double *d,
                   double *t, double *q) {
  if ((variant & 15) >= ORC_S_CD) {
    double Mc[27], h[27];
    orc_central_moments(f, rho, u, Mc);
    orc_central_parts(Mc, *rho, u, k, d, t, q, h);
  } else {
    double M[27];
    orc_moments(f, rho, M);
    u[0] = M[9];
    u[1] = M[3];
    u[2] = M[1];
    orc_table1(M, *rho, k, d, t, q);
  }
}

/* The deviations of Sec. KBC: f_eq(rho, u) (eq:entropic_eq, or eq:polynomial2), the shear
 * deviation ds = s - s_eq (s from Table 1 on the moments of f, s_eq from Table 1 on the moments
 * of f_eq), and dh = h - h_eq = f - f_eq - ds (eq:ksh-representation with k = k_eq). */
void orc_deltas(const double *f, int variant, double *feq, double *ds, double *dh) {
  double rho, u[3], rho_eq, u_eq[3];
  double k[27], d[27], t[27], q[27], s[27];
  double keq[27], deq[27], teq[27], qeq[27], seq[27];
  groups(f, variant, &rho, u, k, d, t, q);           /* rho, u and the groups of f */
  equilibrium_of(variant, rho, u, feq);
  groups(feq, variant, &rho_eq, u_eq, keq, deq, teq, qeq);  /* s_eq from the moments of f_eq */
  shear_part(d, t, q, variant, s);
  shear_part(deq, teq, qeq, variant, seq);
  for (int i = 0; i < 27; ++i) {
    ds[i] = s[i] - seq[i];
    dh[i] = f[i] - feq[i] - ds[i];
  }
}

/* entropic scalar product <X|Y> = sum_i X_i Y_i / f_eq_i (Sec. KBC) */
static double esp(const double *x, const double *y, const double *feq) {
  double acc = 0.0;
  for (int i = 0; i < 27; ++i) acc += x[i] * y[i] / feq[i];
  return acc;
}

int orc_collide(const double *f, double beta, int variant, int gamma_mode, double *fout,
                double *gamma_out) {
  double feq[27], ds[27], dh[27];
  orc_deltas(f, variant, feq, ds, dh);
  int guarded = 0;
  double gamma;
  if (gamma_mode == ORC_GAMMA_LBGK) {
    gamma = 2.0;
  } else if (gamma_mode == ORC_GAMMA_RLB) {
    gamma = 1.0 / beta;
  } else {
    const double num = esp(ds, dh, feq), den = esp(dh, dh, feq);
    if (den <= ORC_DEN_GUARD) {
      gamma = 2.0;
      guarded = 1;
    } else {
      gamma = 1.0 / beta - (2.0 - 1.0 / beta) * num / den;   /* eq:result21 */
      if (gamma_mode == ORC_GAMMA_EXACT) gamma = orc_gamma_exact(feq, ds, dh, beta, gamma);
    }
  }
  /* eq:Egeneral with eq:ksh-mirror: (1 - beta) f + beta f_mirr = f - beta (2 ds + gamma dh) */
  for (int i = 0; i < 27; ++i) fout[i] = f[i] - beta * (2.0 * ds[i] + gamma * dh[i]);
  if (gamma_out) *gamma_out = gamma;
  return guarded;
}

/* eq:Egeneral with the mirror state eq:ksh-mirror, built from explicit k, s, h parts */
void orc_collide_mirror(const double *f, double beta, int variant, double gamma, double *fout) {
  double rho, u[3], feq[27], rho_eq, u_eq[3];
  double k[27], d[27], t[27], q[27], s[27], keq[27], deq[27], teq[27], qeq[27], seq[27];
  groups(f, variant, &rho, u, k, d, t, q);
  equilibrium_of(variant, rho, u, feq);
  groups(feq, variant, &rho_eq, u_eq, keq, deq, teq, qeq);
  shear_part(d, t, q, variant, s);
  shear_part(deq, teq, qeq, variant, seq);
  for (int i = 0; i < 27; ++i) {
    const double h = f[i] - k[i] - s[i];
    const double heq = feq[i] - keq[i] - seq[i];
    const double mirr = k[i] + (2.0 * seq[i] - s[i]) + ((1.0 - gamma) * h + gamma * heq);
    fout[i] = (1.0 - beta) * f[i] + beta * mirr;
  }
}

/* root of eq:result1, g(gamma) = sum dh_i ln(1 + ((1-beta gamma) dh_i - (2beta-1) ds_i)/f_eq_i),
 * by damped Newton iteration from gamma0. g is strictly decreasing where it is defined. */
double orc_gamma_exact(const double *feq, const double *ds, const double *dh, double beta,
                       double gamma0) {
  double g = gamma0;
  for (int it = 0; it < 100; ++it) {
    double val = 0.0, der = 0.0;
    int ok = 1;
    for (int i = 0; i < 27; ++i) {
      const double arg = feq[i] + (1.0 - beta * g) * dh[i] - (2.0 * beta - 1.0) * ds[i];
      if (arg <= 0.0) { ok = 0; break; }
      val += dh[i] * log(arg / feq[i]);
      der += dh[i] * (-beta * dh[i]) / arg;
    }
    if (!ok || der == 0.0) break;
    double step = -val / der;
    /* keep every post-collision population positive */
    for (int tries = 0; tries < 60; ++tries) {
      int pos = 1;
      for (int i = 0; i < 27; ++i)
        if (feq[i] + (1.0 - beta * (g + step)) * dh[i] - (2.0 * beta - 1.0) * ds[i] <= 0.0) pos = 0;
      if (pos) break;
      step *= 0.5;
    }
    g += step;
    if (fabs(step) <= 1e-15 * (1.0 + fabs(g))) break;
  }
  return g;
}

/* eq:S */
double orc_entropy(const double *f) {
  double s = 0.0;
  for (int i = 0; i < 27; ++i) s -= f[i] * log(f[i] / weight(i));
  return s;
}

static int64_t wrap(int64_t a, int64_t n) { return ((a % n) + n) % n; }

/* propagation, left-hand side of eq:Egeneral: dst_i(x) = src_i(x - v_i), periodic */
void orc_stream(int32_t nx, int32_t ny, int32_t nz, const double *src, double *dst) {
  const int64_t P = (int64_t)nx * ny * nz;
  for (int i = 0; i < 27; ++i) {
    const int vx = vcomp(i, 0), vy = vcomp(i, 1), vz = vcomp(i, 2);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t z = 0; z < nz; ++z)
      for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
          const int64_t sx = wrap(x - vx, nx), sy = wrap(y - vy, ny), sz = wrap(z - vz, nz);
          dst[i * P + x + nx * (y + ny * z)] = src[i * P + sx + nx * (sy + ny * sz)];
        }
  }
}

int64_t orc_collide_field(int32_t nx, int32_t ny, int32_t nz, double *f, double beta,
                          int variant, int gamma_mode, double *gamma_field) {
  const int64_t P = (int64_t)nx * ny * nz;
  int64_t guarded = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(+ : guarded)
#endif
  for (int64_t n = 0; n < P; ++n) {
    double fl[27], fo[27], g;
    for (int i = 0; i < 27; ++i) fl[i] = f[i * P + n];
    guarded += orc_collide(fl, beta, variant, gamma_mode, fo, &g);
    for (int i = 0; i < 27; ++i) f[i * P + n] = fo[i];
    if (gamma_field) gamma_field[n] = g;
  }
  return guarded;
}

void orc_init_equilibrium(int32_t nx, int32_t ny, int32_t nz, const double *rho,
                          const double *u, double *f) {
  const int64_t P = (int64_t)nx * ny * nz;
  for (int64_t n = 0; n < P; ++n) {
    double feq[27];
    const double un[3] = {u[n], u[P + n], u[2 * P + n]};
    orc_equilibrium(rho[n], un, feq);
    for (int i = 0; i < 27; ++i) f[i * P + n] = feq[i];
  }
}

/* rho = sum f_i, rho u = sum v_i f_i (Sec. "Introduction") */
void orc_macroscopic(int32_t nx, int32_t ny, int32_t nz, const double *f, double *rho,
                     double *u) {
  const int64_t P = (int64_t)nx * ny * nz;
  for (int64_t n = 0; n < P; ++n) {
    double r = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 27; ++i) {
      const double fi = f[i * P + n];
      r += fi;
      for (int a = 0; a < 3; ++a) m[a] += vcomp(i, a) * fi;
    }
    rho[n] = r;
    for (int a = 0; a < 3; ++a) u[a * P + n] = m[a] / r;
  }
}

/* Diagnostics of Sec. "Numerical Simulations" on the macroscopic fields:
 * out[0] = sum rho, out[1..3] = sum rho u,
 * out[4] = k = 1/2 <u'.u'>,  u' = u - <u>,
 * out[5] = Omega = 1/2 <|curl u'|^2>,
 * out[6] = epsilon = 1/2 nu <(d_b u'_a + d_a u'_b)^2>,
 * out[7] = P, out[8] = <(d u'_x / d x)^2>,
 * out[9..12] = longitudinal skewness factors S_11^n, n = 3..6:
 *              (-1)^n <(d u'_x/d x)^n> <(d u'_x/d x)^2>^(-n/2),
 * derivatives by central differences of order 2 (the figures) or 8 (Table 2) on the periodic
 * grid: d u / d x = sum_k c_k (u(x + k) - u(x - k)),
 * order 2: c_1 = 1/2;  order 8: c = 4/5, -1/5, 4/105, -1/280. */
void orc_diagnostics(int32_t nx, int32_t ny, int32_t nz, const double *rho, const double *u,
                     double nu, int order, double *out) {
  static const double c2[1] = {0.5};
  static const double c8[4] = {4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0};
  const double *coef = order == 8 ? c8 : c2;
  const int K = order == 8 ? 4 : 1;
  const int64_t P = (int64_t)nx * ny * nz;
  double mass = 0.0, mom[3] = {0, 0, 0}, mean[3] = {0, 0, 0};
  for (int64_t n = 0; n < P; ++n) {
    mass += rho[n];
    for (int a = 0; a < 3; ++a) {
      mom[a] += rho[n] * u[a * P + n];
      mean[a] += u[a * P + n];
    }
  }
  for (int a = 0; a < 3; ++a) mean[a] /= (double)P;
  double ke = 0.0, ens = 0.0, dis = 0.0, pw[7] = {0, 0, 0, 0, 0, 0, 0};
  const int64_t dims[3] = {nx, ny, nz};
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        const int64_t n = x + nx * (y + ny * z);
        const int64_t c[3] = {x, y, z};
        double g[3][3]; /* g[a][b] = d u_a / d x_b */
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) g[a][b] = 0.0;
        for (int b = 0; b < 3; ++b)
          for (int k = 1; k <= K; ++k) {
            int64_t cp[3] = {c[0], c[1], c[2]}, cm[3] = {c[0], c[1], c[2]};
            cp[b] = wrap(c[b] + k, dims[b]);
            cm[b] = wrap(c[b] - k, dims[b]);
            const int64_t np = cp[0] + nx * (cp[1] + ny * cp[2]);
            const int64_t nm = cm[0] + nx * (cm[1] + ny * cm[2]);
            for (int a = 0; a < 3; ++a) g[a][b] += coef[k - 1] * (u[a * P + np] - u[a * P + nm]);
          }
        for (int a = 0; a < 3; ++a) {
          const double up = u[a * P + n] - mean[a];
          ke += up * up;
        }
        const double wx = g[2][1] - g[1][2], wy = g[0][2] - g[2][0], wz = g[1][0] - g[0][1];
        ens += wx * wx + wy * wy + wz * wz;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            const double sab = g[a][b] + g[b][a];
            dis += sab * sab;
          }
        double q = 1.0;
        for (int m = 1; m <= 6; ++m) {
          q *= g[0][0];
          pw[m] += q;
        }
      }
  out[0] = mass;
  for (int a = 0; a < 3; ++a) out[1 + a] = mom[a];
  out[4] = 0.5 * ke / (double)P;
  out[5] = 0.5 * ens / (double)P;
  out[6] = 0.5 * nu * dis / (double)P;
  out[7] = (double)P;
  const double m2 = pw[2] / (double)P;
  out[8] = m2;
  for (int m = 3; m <= 6; ++m)
    out[9 + m - 3] = (m % 2 ? -1.0 : 1.0) * (pw[m] / (double)P) / pow(m2, 0.5 * m);
}

/* nsteps of eq:Egeneral on the pre-collision field f(t): collide every node (right-hand
 * side), then propagate (left-hand side). The result f(t + nsteps) is left in fa; fb is
 * scratch. gamma_field, if given, receives the stabilizer of the last collision.
 * Returns the number of guarded nodes over all steps. */
int64_t orc_run(int32_t nx, int32_t ny, int32_t nz, double *fa, double *fb, int64_t nsteps,
                double beta, int variant, int gamma_mode, double *gamma_field) {
  const int64_t P = (int64_t)nx * ny * nz;
  int64_t guarded = 0;
  double *a = fa, *b = fb;
  for (int64_t s = 0; s < nsteps; ++s) {
    guarded += orc_collide_field(nx, ny, nz, a, beta, variant, gamma_mode, gamma_field);
    orc_stream(nx, ny, nz, a, b);
    double *tmp = a;
    a = b;
    b = tmp;
  }
  if (a != fa) memcpy(fa, a, (size_t)(27 * P) * sizeof(double));
  return guarded;
}

/* Consistent initial density and higher moments (Sec. "Numerical Simulations", following
 * Mei et al.): the lattice Boltzmann iteration with the velocity held at the prescribed u0,
 *   f <- S[ f - 2 beta_pre (f - f_eq(rho(f), u0)) ],   S = propagation (orc_stream),
 * whose density relaxes to the steady state of its mass balance. After each iteration the
 * change max_x |rho^{n+1}(x) - rho^n(x)| is measured; the loop stops after the first
 * iteration whose change is <= tol, or after max_iters. Returns the iterations run, or -1
 * when its work array cannot be allocated; *residual = the last change (NaN when none was
 * run). fb is scratch of the size of f. */
int64_t orc_presolve(int32_t nx, int32_t ny, int32_t nz, double *f, double *fb, const double *u0,
                     double beta_pre, int64_t max_iters, double tol, double *residual) {
  const int64_t P = (int64_t)nx * ny * nz;
  double *rho_old = (double *)malloc((size_t)P * sizeof(double));
  double res = NAN;
  int64_t it = 0;
  if (!rho_old) {
    if (residual) *residual = NAN;
    return -1;
  }
  for (int64_t n = 0; n < P; ++n) {
    double r = 0.0;
    for (int i = 0; i < 27; ++i) r += f[i * P + n];
    rho_old[n] = r;
  }
  while (it < max_iters) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t n = 0; n < P; ++n) {
      double rho = 0.0, feq[27];
      for (int i = 0; i < 27; ++i) rho += f[i * P + n];
      const double un[3] = {u0[n], u0[P + n], u0[2 * P + n]};
      orc_equilibrium(rho, un, feq);
      for (int i = 0; i < 27; ++i) f[i * P + n] -= 2.0 * beta_pre * (f[i * P + n] - feq[i]);
    }
    orc_stream(nx, ny, nz, f, fb);
    memcpy(f, fb, (size_t)(27 * P) * sizeof(double));
    ++it;
    res = 0.0;
    for (int64_t n = 0; n < P; ++n) {
      double r = 0.0;
      for (int i = 0; i < 27; ++i) r += f[i * P + n];
      const double ch = fabs(r - rho_old[n]);
      if (!(ch <= res)) res = ch;    /* NaN propagates */
      rho_old[n] = r;
    }
    if (res <= tol) break;
  }
  free(rho_old);
  if (residual) *residual = res;
  return it;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
