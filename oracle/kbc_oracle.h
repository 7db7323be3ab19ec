/*
 * kbc_oracle.h -- plain FP64 CPU oracle of the D3Q27 KBC lattice Boltzmann step.
 *
 * TEST INFRASTRUCTURE ONLY. This code exists to check the CUDA path; it is called by
 * tests, by the package smoke check and by the benchmark's CPU-baseline leg, never by
 * the product path. It shares no code, header, table or constant with the CUDA library.
 *
 * Paper: Boesch, Chikatamarla, Karlin, "Entropic multi-relaxation lattice Boltzmann
 * scheme for turbulent flows" (arXiv:1507.02518).
 *
 * Conventions (shared with the CUDA library only by documentation, not by code):
 *   velocity index  i = (vx+1) + 3*(vy+1) + 9*(vz+1),  v in {-1,0,1}^3  (eq:D3Q27vel)
 *   field layout    f[i*P + n],  P = nx*ny*nz,  n = x + nx*(y + ny*z)   (x fastest)
 *   populations are plain (unshifted) f_i.
 */
#ifndef KBC_ORACLE_H
#define KBC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* choice of the shear part s (Sec. KBC): natural-moment groups of Table 1, or the same groups
 * in the central-moment basis (appendix, eq:cmf000-eq:cmfxyz) */
enum {
  ORC_S_D = 0, ORC_S_DT = 1, ORC_S_DQ = 2, ORC_S_DTQ = 3,
  ORC_S_CD = 4, ORC_S_CDT = 5, ORC_S_CDQ = 6, ORC_S_CDTQ = 7
};
/* OR'ed into a variant argument: collide with the second-order polynomial equilibrium
 * eq:polynomial2 instead of the product form eq:entropic_eq */
#define ORC_EQ_POLY2 16

/* how the stabilizer gamma is chosen */
enum {
  ORC_GAMMA_ESTIMATE = 0, /* eq:result21 (the method) */
  ORC_GAMMA_LBGK = 1,     /* gamma = 2 (LBGK special case, Sec. KBC) */
  ORC_GAMMA_RLB = 2,      /* gamma = 1/beta (regularized special case, Sec. KBC) */
  ORC_GAMMA_EXACT = 3     /* root of eq:result1 by Newton iteration */
};

/* den <= this => gamma = 2 (paper is silent on <dh|dh> -> 0; see the oracle notes) */
#define ORC_DEN_GUARD 1e-300

void   orc_lattice(int32_t *v /*27x3*/, double *w /*27*/);
double orc_beta(double nu);
void   orc_equilibrium(double rho, const double *u /*3*/, double *feq /*27*/);
void   orc_equilibrium_poly2(double rho, const double *u /*3*/, double *feq /*27*/);
void   orc_moments(const double *f /*27*/, double *rho, double *M /*27: M[p*9+q*3+r]*/);
void   orc_table1(const double *M, double rho, double *k, double *d, double *t, double *q);
void   orc_moment_rep(const double *M, double rho, double *f /*27*/);
void   orc_central_moments(const double *f, double *rho, double *u /*3*/, double *Mc /*27*/);
void   orc_central_parts(const double *Mc, double rho, const double *u, double *k, double *d,
                         double *t, double *q, double *h);
int    orc_collide(const double *f, double beta, int variant, int gamma_mode,
                   double *fout, double *gamma_out);
void   orc_collide_mirror(const double *f, double beta, int variant, double gamma, double *fout);
void   orc_deltas(const double *f, int variant, double *feq, double *ds, double *dh);
double orc_gamma_exact(const double *feq, const double *ds, const double *dh, double beta,
                       double gamma0);
double orc_entropy(const double *f);

void   orc_stream(int32_t nx, int32_t ny, int32_t nz, const double *src, double *dst);
int64_t orc_collide_field(int32_t nx, int32_t ny, int32_t nz, double *f, double beta,
                          int variant, int gamma_mode, double *gamma_field);
void   orc_init_equilibrium(int32_t nx, int32_t ny, int32_t nz, const double *rho,
                            const double *u, double *f);
void   orc_macroscopic(int32_t nx, int32_t ny, int32_t nz, const double *f, double *rho,
                       double *u);
void   orc_diagnostics(int32_t nx, int32_t ny, int32_t nz, const double *rho, const double *u,
                       double nu, int order, double *out /*13*/);
int64_t orc_run(int32_t nx, int32_t ny, int32_t nz, double *fa, double *fb, int64_t nsteps,
                double beta, int variant, int gamma_mode, double *gamma_field);
int64_t orc_presolve(int32_t nx, int32_t ny, int32_t nz, double *f, double *fb,
                     const double *u0, double beta_pre, int64_t max_iters, double tol,
                     double *residual);
int    orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
