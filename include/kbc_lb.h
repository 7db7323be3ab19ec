/*
 * kbc_lb.h -- C ABI of the GB300 (sm_103a) D3Q27 KBC lattice Boltzmann library.
 *
 * Method: Boesch, Chikatamarla, Karlin, "Entropic multi-relaxation lattice Boltzmann scheme
 * for turbulent flows" (arXiv:1507.02518). One time step is eq:Egeneral on a periodic box:
 * every node collides with the KBC operator (Sec. KBC: the mirror state eq:ksh-mirror in
 * eq:Egeneral, i.e. f' = f - beta(2 ds + gamma dh) with ds = s - s_eq from Table 1 and the
 * product-form equilibrium eq:entropic_eq, dh = f - f_eq - ds, and the stabilizer gamma of
 * eq:result21) and the post-collision populations propagate along the 27 links.
 *
 * Conventions
 *   velocities   i = (vx+1) + 3*(vy+1) + 9*(vz+1), v in {-1,0,1}^3 (eq:D3Q27vel); the opposite
 *                of i is 26 - i.
 *   node index   n = x + nx*(y + ny*z) (x fastest).
 *   canonical    a population field f[27][P] (P = nx*ny*nz, plane i contiguous) of FP64
 *                values holding the PRE-collision populations f_i(x, t) of the current time
 *                t. Both streaming schemes expose exactly this state.
 *   memory       the library allocates no device memory. The caller passes one device buffer
 *                of at least lb_required_bytes() bytes and keeps it alive until lb_destroy;
 *                the library never frees it. "on_device" arguments say whether a pointer is
 *                device (1) or host (0) memory. Host memory may be pageable (copied through
 *                the staging area in chunks) or page-locked (cudaHostAlloc, cudaHostRegister:
 *                the kernels read or write it in place over the host-device link, no
 *                staging copies); either way the call has finished with it on return.
 *   streams      all work is enqueued on the CUDA stream given to lb_create (NULL = legacy
 *                default stream). lb_step and lb_batch_step never synchronise; lb_moments,
 *                lb_diagnostics, lb_get_populations, lb_set_populations, lb_presolve and
 *                lb_init_field from host memory synchronise the stream.
 *   errors       every call returns lb_status; no exception crosses the ABI. Errors of
 *                asynchronous kernels surface at the next synchronising call as
 *                LB_ERR_CUDA. lb_last_error() gives a message. A context is used by one host
 *                thread at a time.
 */
#ifndef KBC_LB_H
#define KBC_LB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t lb_status;
enum {
  LB_OK = 0,
  LB_ERR_INVALID_ARG = 1,  /* bad size, parameter, pointer or enum value */
  LB_ERR_OOM = 2,          /* a caller buffer is smaller than required, or host memory ran out */
  LB_ERR_CUDA = 3,         /* a CUDA call or kernel failed (message in lb_last_error) */
  LB_ERR_NONFINITE = 4,    /* lb_diagnostics found NaN/Inf populations */
  LB_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out */
  LB_ERR_UNSUPPORTED = 6   /* valid but not built (e.g. no sm_103a device) */
};

/* Shear part s (Sec. KBC): s in {d, d+t, d+q, d+t+q} built on the natural moments (Table 1),
 * or the same groups d~, t~, q~ built on the central moments (appendix, eq:cmf000 ff.). */
enum {
  LB_S_D = 0, LB_S_DT = 1, LB_S_DQ = 2, LB_S_DTQ = 3,
  LB_S_CD = 4, LB_S_CDT = 5, LB_S_CDQ = 6, LB_S_CDTQ = 7
};
/* Stabilizer: eq:result21 (the method), the fixed special cases named in Sec. KBC
 * (gamma = 2, LBGK; gamma = 1/beta, regularized LB), or LB_GAMMA_EXACT: per node the root
 * gamma* of the entropy condition eq:result1, by a damped Newton iteration started from
 * eq:result21 (at most 50 iterations in FP64, 20 in FP32; each step halved until every
 * logarithm's argument stays positive; nodes where <dh|dh> falls under the guard keep
 * gamma = 2). LB_GAMMA_EXACT runs in the one-node-per-thread direct kernel only and is not
 * available to batches. */
enum { LB_GAMMA_ESTIMATE = 0, LB_GAMMA_LBGK = 1, LB_GAMMA_RLB = 2, LB_GAMMA_EXACT = 3 };
/* Storage of the populations in device memory; collision arithmetic is FP64 for LB_F64 and
 * FP32 otherwise. All three store the shift f_i - W_i; LB_F16 stores (f_i - W_i)/W_i in
 * IEEE half precision, rounded to nearest even. */
enum { LB_F64 = 0, LB_F32 = 1, LB_F16 = 2 };
/* Streaming: LB_PULL keeps two population arrays (gather, collide, write);
 * LB_AA keeps one array updated in place with alternating even/odd steps. */
enum { LB_PULL = 0, LB_AA = 1 };
/* Equilibrium of the collision: the product form eq:entropic_eq (the method), or the
 * second-order polynomial eq:polynomial2 (the standard LB equilibrium, a comparison mode; not
 * with LB_GAMMA_EXACT, the batch kernels or the staged/persistent kernels). Initialisation
 * (lb_init_field, lb_presolve) always uses the product form. */
enum { LB_EQ_PRODUCT = 0, LB_EQ_POLY2 = 1 };

typedef struct {
  int32_t nx, ny, nz;   /* periodic box, each >= 3, nx*ny*nz < 2^31 */
  double nu;            /* kinematic viscosity > 0; beta = 1/(6 nu + 1) (eq:viscosity, c_s^2 = 1/3) */
  int32_t variant;      /* LB_S_* */
  int32_t gamma_mode;   /* LB_GAMMA_* */
  int32_t storage;      /* LB_F64 / LB_F32 / LB_F16 */
  int32_t scheme;       /* LB_PULL / LB_AA */
  int32_t equilibrium;  /* LB_EQ_PRODUCT (0) / LB_EQ_POLY2 */
} lb_config;

/* Diagnostics of Sec. "Numerical Simulations" at the current time t. Averages <.> are over
 * nodes; u' = u - <u> (k is summed in a second pass over the field, after <u>); gradients
 * are central differences of order grad_order: 2 (the default, as for the paper's enstrophy
 * curves) or 8 (Table 2), see lb_set_diag_order. In a field holding NaN/Inf the averages
 * run over the nodes whose rho and u (k, <u>, gamma) or velocity gradients (Omega, epsilon,
 * dudx2, skewness) are finite, and the call returns LB_ERR_NONFINITE. */
typedef struct {
  int64_t step;             /* t */
  int64_t nodes;            /* P */
  double mass;              /* sum rho */
  double momentum[3];       /* sum rho u */
  double kinetic_energy;    /* k = 1/2 <u'.u'> */
  double enstrophy;         /* Omega = 1/2 <|curl u'|^2> */
  double dissipation;       /* epsilon = 1/2 nu <(d_b u'_a + d_a u'_b)^2> */
  double gamma_mean;        /* <gamma> of the collision that produced the state at t */
  double gamma_std;         /* its standard deviation over nodes */
  int64_t nonfinite_count;  /* nodes whose rho or u is NaN/Inf */
  int64_t den_guard_count;  /* nodes where <dh|dh> fell under the guard (gamma set to 2),
                               counted over the same collision as gamma_mean */
  int32_t grad_order;       /* 2 or 8 */
  int32_t reserved;
  double dudx2;             /* <(d u'_x / d x)^2> */
  double skewness[4];       /* longitudinal skewness factors S_11^n, n = 3..6 (Table 2):
                               (-1)^n <(d u'_x/d x)^n> <(d u'_x/d x)^2>^(-n/2);
                               NaN when dudx2 is 0 (no x-gradient, e.g. at rest) */
} lb_diag;

/* Gap between the stabilizer estimate eq:result21 and the exact root gamma* of eq:result1,
 * both evaluated on the collision inputs of the current state f(t) (Sec. KBC). Averages are
 * over the evaluated nodes; nodes under the <dh|dh> guard or holding NaN/Inf are skipped. */
typedef struct {
  int64_t step;          /* t */
  int64_t nodes;         /* nodes evaluated */
  double mean_abs;       /* <|gamma_est - gamma*|> */
  double max_abs;        /* max |gamma_est - gamma*| */
  double mean_estimate;  /* <gamma_est> */
  double mean_exact;     /* <gamma*> */
  int64_t unconverged;   /* nodes where the Newton iteration stopped before converging */
  int64_t skipped;       /* nodes skipped (guard or non-finite) */
} lb_gap;

typedef struct lb_ctx lb_ctx;

/* Bytes of device memory a context with this configuration needs (populations, diagnostics
 * fields and a bounded host-transfer staging area), or 0 if the configuration is invalid. */
size_t lb_required_bytes(const lb_config *cfg);

/* Create a context on the current CUDA device.
 *   dev_buf  device buffer of `bytes` bytes, 256-byte aligned, owned by the caller.
 *   stream   cudaStream_t to enqueue on (NULL = default stream).
 * The populations start at rest (f_i = W_i, t = 0) until lb_init_field or
 * lb_set_populations. On failure *out is NULL and lb_last_error(NULL) explains. */
lb_status lb_create(const lb_config *cfg, void *dev_buf, size_t bytes, void *stream,
                    lb_ctx **out);
lb_status lb_destroy(lb_ctx *ctx);

/* Message of the last failed call on ctx (ctx NULL: of the last failed lb_create or
 * lb_batch_create on this thread). Never NULL; valid until the next call on ctx. */
const char *lb_last_error(const lb_ctx *ctx);

/* Set f(x, 0) = f_eq(rho(x), u(x)) by eq:entropic_eq and t = 0.
 *   rho  FP64 [P] (NULL: rho = 1 everywhere);  u  FP64 [3][P] (u_x plane, u_y, u_z).
 * Pageable host inputs are copied through the staging area in chunks, page-locked ones are
 * read in place; |u_a| < 1 is required. Host inputs: synchronises. */
lb_status lb_init_field(lb_ctx *ctx, const double *rho, const double *u, int on_device);

/* Consistent initial state (Sec. "Numerical Simulations": the initial density and higher
 * moments come from an iteration run to steady state beforehand, after Mei et al.). Sets
 * f = f_eq(1, u0) (unless from_current), then iterates
 *     f <- S[ f - 2 beta_pre (f - f_eq(rho(f), u0)) ],   beta_pre = 1/(6 nu_pre + 1),
 * (S: propagation) with the velocity of the equilibrium held at u0 while the density evolves.
 * Every 32 iterations (and after the last) the largest change of rho over the last iteration
 * is measured, on rho - 1 rounded to FP32; the loop stops when it is <= tol (a negative tol
 * runs max_iters) or after max_iters iterations, rounded up to an even count. The result is
 * the state at t = 0; lb_diagnostics has no gamma until the next lb_step.
 *   u0            FP64 [3][P], host (pageable: copied in chunks; page-locked: read in
 *                 place) or device (on_device != 0)
 *   nu_pre        > 0, the pre-solve's own relaxation (1/6 relaxes fully to f_eq each
 *                 iteration)
 *   from_current  nonzero: start from the current state instead of f_eq(1, u0), e.g. from
 *                 lb_init_field(rho_guess, u0) with a density interpolated from a coarser
 *                 pre-solve; requires t = 0 (LB_ERR_INVALID_ARG otherwise)
 *   iters         iterations run (may be NULL);  residual  the last measured change (may be
 *                 NULL; NaN if max_iters is 0)
 * Uses the diagnostics work area and the gamma field as scratch. Synchronises. Returns
 * LB_ERR_NONFINITE if the iteration produced NaN/Inf. */
lb_status lb_presolve(lb_ctx *ctx, const double *u0, int on_device, double nu_pre,
                      int64_t max_iters, double tol, int32_t from_current, int64_t *iters,
                      double *residual);

/* Advance n >= 0 time steps (eq:Egeneral with the KBC collision). Asynchronous. The last of
 * the n collisions also records gamma per node for lb_diagnostics. */
lb_status lb_step(lb_ctx *ctx, int64_t n);

/* rho [P] and u [3][P] (FP64, caller-owned) of the current state. Synchronises. */
lb_status lb_moments(lb_ctx *ctx, double *rho, double *u, int on_device);

/* Fill *out for the current state. Synchronises. Returns LB_ERR_NONFINITE (with *out filled)
 * if any node is NaN/Inf. */
lb_status lb_diagnostics(lb_ctx *ctx, lb_diag *out);

/* Order (2 or 8) of the central differences lb_diagnostics uses for velocity gradients:
 * du/dx = sum_k c_k (u(x + k) - u(x - k)), c = 1/2 (order 2) or 4/5, -1/5, 4/105, -1/280
 * (order 8). Default 2. */
lb_status lb_set_diag_order(lb_ctx *ctx, int32_t order);

/* Kinetic-energy spectrum of the current state (Sec. "Numerical Simulations": E(kappa) with
 * k = integral of E; D(kappa) = 2 nu kappa^2 E(kappa)). Cubic boxes (nx = ny = nz = N) only.
 *   E[m], m = 0..nbins-1 (host, caller-owned): the sum over integer wave vectors n != 0 with
 *        rint(|n|) = m of 1/2 |u_hat(n)|^2, u_hat(n) = (1/P) sum_x u(x) e^{-2 pi i n.x/N}; shell m
 *        holds kappa = 2 pi m / N, sum_m E[m] = k when nbins > sqrt(3) N / 2 (higher shells are
 *        dropped otherwise). E[0] = 0 (the mean flow is not part of u').
 *   work  device buffer of lb_spectrum_work_bytes(ctx, nbins) bytes, 256-byte aligned, owned
 *         by the caller (FFT of one velocity component, the FFT work area, block histograms).
 * The velocity is the one lb_diagnostics uses (collision precision); the 3D real-to-complex
 * FFTs are cuFFT's (its plan holds a small internal allocation for the duration of the call).
 * 1 <= nbins <= 6144. Synchronises. LB_ERR_UNSUPPORTED for non-cubic boxes. */
size_t lb_spectrum_work_bytes(lb_ctx *ctx, int32_t nbins);
lb_status lb_spectrum(lb_ctx *ctx, void *work, size_t work_bytes, int32_t nbins, double *E);

/* Fill *out with the stabilizer gap of the current state (NaN averages when no node was
 * evaluated). Does not advance t or touch the populations; uses the diagnostics work area.
 * Synchronises. Arithmetic in the collision precision of the storage (FP64 for LB_F64).
 * LB_ERR_UNSUPPORTED for LB_EQ_POLY2 contexts. */
lb_status lb_stabilizer_gap(lb_ctx *ctx, lb_gap *out);

/* Canonical pre-collision populations f[27][P] (FP64, caller-owned) at the current time t,
 * whatever the scheme and step parity. Synchronises. */
lb_status lb_get_populations(lb_ctx *ctx, double *f, int on_device);

/* The stabilizer gamma of every node from the last collision of the last lb_step call
 * (eq:result21, or 2 / 1/beta in the LBGK / RLB modes; 2 where <dh|dh> fell under the guard;
 * FP32, caller-owned gamma[P], node order). With LB_F32 storage, a node whose FP32 <dh|dh>
 * fell under 1e-13 is collided again in FP64 from its inputs (a second kernel after each
 * step kernel) and takes that gamma and those populations; LB_F16 storage keeps the FP32
 * collision there. LB_ERR_INVALID_ARG when no step has run since the state was set.
 * Synchronises. */
lb_status lb_get_gamma(lb_ctx *ctx, float *gamma, int on_device);

/* Overwrite the state with canonical populations f[27][P] at the current time t (checkpoint
 * resume, test seeding). Values are rounded to the storage precision. Synchronises. */
lb_status lb_set_populations(lb_ctx *ctx, const double *f, int on_device);

/* Current time t and the relaxation parameter beta of the context. */
int64_t lb_time(const lb_ctx *ctx);
double lb_beta(const lb_ctx *ctx);
/* Reset t (e.g. after loading a checkpoint written at time t; call before
 * lb_set_populations). t >= 0. */
lb_status lb_set_time(lb_ctx *ctx, int64_t t);

/* Which step kernel runs. All kernels give bit-identical populations for a given storage
 * (the FP32 kernels of one node per thread run the FP32x2 collision with the node in both
 * lanes, so every FP32 kernel executes the same compiled arithmetic). FP64 storage runs the
 * direct kernel.
 *   LB_KERNEL_ROWS        two adjacent nodes per thread on packed FP32x2 instructions; a
 *                         persistent grid walks tiles of whole rows (nx <= 256) or 256-node
 *                         row segments (nx a multiple of 256), whose 27 source rows the
 *                         bulk-copy engine stages in shared memory ahead of the collision
 *                         (mbarrier pipeline, bounded waits). Needs LB_F32 / LB_F16, the
 *                         product-form equilibrium, a natural-moment variant, nx even with
 *                         nx * sizeof(stored value) % 16 == 0, and for nx <= 256 a tile of R
 *                         rows (R dividing ny) with R * nx a multiple of 64 in [128, 256];
 *                         else LB_ERR_UNSUPPORTED.
 *   LB_KERNEL_ADJ         two adjacent nodes (x, x+1) per thread on packed FP32x2
 *                         instructions, straight from global memory: the planes not shifted
 *                         in x are one 32/64-bit access per plane. Needs LB_F32 / LB_F16, the
 *                         product-form equilibrium, a natural-moment variant and an even nx.
 *   LB_KERNEL_PACKED      two nodes per thread, (x, x+32) of one row, the collision on
 *                         packed FP32x2 instructions; LB_F32 / LB_F16 only.
 *   LB_KERNEL_PERSISTENT  a persistent grid walks 128-node row segments, one thread per node,
 *                         loading from global memory; the bulk-copy engine prefetches into L2
 *                         the source rows of segments a few items ahead (lb_set_prefetch) when
 *                         rows are whole multiples of 16 bytes.
 *   LB_KERNEL_STAGED      the same items with the 27 source rows staged in shared memory by
 *                         asynchronous bulk copies in an mbarrier pipeline; needs
 *                         nx * sizeof(stored value) % 16 == 0 (else LB_ERR_UNSUPPORTED).
 *                         Staged and persistent run the natural-moment variants only.
 *   LB_KERNEL_DIRECT      one thread per node over a full grid (lb_set_block), any nx.
 *   LB_KERNEL_AUTO        (default) for FP32 arithmetic adjacent pairs where that kernel
 *                         applies (even nx, product form, natural moments), packed
 *                         otherwise; direct for LB_F64. */
enum {
  LB_KERNEL_AUTO = 0,
  LB_KERNEL_DIRECT = 1,
  LB_KERNEL_STAGED = 2,
  LB_KERNEL_PERSISTENT = 3,
  LB_KERNEL_PACKED = 4,
  LB_KERNEL_ROWS = 5,
  LB_KERNEL_ADJ = 6
};
lb_status lb_set_kernel(lb_ctx *ctx, int32_t kind);

/* L2 prefetch distance of the persistent kernel, in work items per CTA (0 = off, at most 8;
 * default 2). */
lb_status lb_set_prefetch(lb_ctx *ctx, int32_t items_ahead);

/* Launch shape of the direct kernel: threads per block along x (bx) and y (by), with
 * bx*by in {64, 128, 256, 512} (at most 256 for LB_F64) and bx a multiple of 32. */
lb_status lb_set_block(lb_ctx *ctx, int32_t bx, int32_t by);

/* Bound on every device-side wait of the staged kernels, in SM clock cycles (default 2e9,
 * about one second). When a wait runs out the kernel sets a flag, waits (with the same bound)
 * for the copies it has issued, and returns; the next synchronising call returns
 * LB_ERR_TIMEOUT and the state is not valid: lb_step, lb_moments, lb_diagnostics,
 * lb_get_populations, lb_spectrum and lb_stabilizer_gap then return LB_ERR_TIMEOUT until
 * lb_set_populations, lb_init_field or lb_presolve rewrites the state. stall_copies != 0
 * is a test hook of that path: the staged kernel then issues no copies, so its first wait
 * runs out (use a small budget). */
lb_status lb_set_wait_budget(lb_ctx *ctx, uint64_t cycles, int32_t stall_copies);

/* Diagnostics of a canonical population field with no memory allocation of any kind.
 * The paper has no counterpart: this entry point exists for callers that cannot allocate
 * device memory when they need diagnostics -- extensions inside a host framework whose pool
 * allocator has reserved the device's memory (a cudaMalloc behind its back can fail or
 * break its accounting), monitors of jobs sized to fill the GPU's memory that must not
 * change the footprint, and latency-sensitive loops where cudaMalloc/cudaFree would
 * synchronise the device. It computes the fields of lb_diag that depend on the populations
 * alone (mass, momentum, kinetic_energy, enstrophy, dissipation, nonfinite_count, nodes),
 * with the averages of lb_diagnostics at grad_order 2; gamma_mean and gamma_std are NaN,
 * den_guard_count is 0, dudx2 and skewness are NaN and step is -1.
 *   f       device pointer to FP64 canonical populations f[27][P] (the layout of
 *           lb_get_populations), P = nx*ny*nz <= 65536 nodes; larger boxes return
 *           LB_ERR_INVALID_ARG before any GPU work.
 *   nu      the kinematic viscosity in the dissipation, > 0.
 *   stream  cudaStream_t the work is enqueued on; the call synchronises it before returning.
 *   out     host struct, filled on LB_OK and LB_ERR_NONFINITE.
 * The work space is one file-scope __device__ array (about 1.6 MB) that stays on every GPU that
 * loaded the library until the process exits. The first call on a device does a one-time
 * set-up, looking up that array's address with the device current; make that first call
 * before any stream capture begins. All calls share the array and it keeps the last call's
 * contents (each call clears what it accumulates): calls that overlap on the GPU race and
 * must be serialised by the caller. Errors: LB_ERR_INVALID_ARG, LB_ERR_CUDA,
 * LB_ERR_NONFINITE; lb_last_error(NULL) explains. */
lb_status lb_diagnostics_noalloc(int32_t nx, int32_t ny, int32_t nz, double nu, const double *f,
                                 void *stream, lb_diag *out);

/* ---------------------------------------------------------------- slabs of one box split along z
 * One periodic box (eq:Egeneral's propagation wraps in x, y and z) split into slabs of whole
 * z-planes, one per GPU (the multi-GPU form of a single box). A slab context holds planes
 * z0 .. z0 + nz_local - 1 of the global nx x ny x nz box plus one halo plane on each side; the
 * collision is local, and after each step the 9 populations that cross each face (v_z = +1
 * through the top, v_z = -1 through the bottom) travel to the neighbouring slab: per face and
 * step 9 nx ny stored values. The caller moves them (NCCL send/recv, a peer copy, or a device
 * copy when the slabs share a GPU): the library packs them into contiguous face buffers and
 * unpacks what the caller delivered. One step is
 *   lb_slab_step_faces(ctx, record)   steps the two boundary planes and packs send_up /
 *                                     send_down (enqueue the sends after this call),
 *   lb_slab_step_interior(ctx)        steps the other planes (overlaps the transfer), t += 1,
 *   lb_slab_unpack(ctx)               after recv_below / recv_above hold the neighbours'
 *                                     send_up / send_down of the same step.
 * The slab below the global plane 0 is the one holding plane nz - 1 (periodic); a single slab
 * holding the whole box is its own neighbour on both sides. Everything is enqueued on the
 * context's stream; nothing synchronises. lb_init_field, lb_set_populations,
 * lb_get_populations, lb_moments and lb_get_gamma work on a slab context with the slab's own
 * nx*ny*nz_local nodes (local z = global z - z0) once its step is complete; lb_step,
 * lb_diagnostics, lb_spectrum, lb_stabilizer_gap and lb_presolve are whole-box calls
 * (LB_ERR_INVALID_ARG / LB_ERR_UNSUPPORTED). lb_destroy releases it. */
size_t lb_slab_required_bytes(const lb_config *global, int32_t nz_local);
lb_status lb_slab_create(const lb_config *global, int32_t z0, int32_t nz_local, void *dev_buf,
                         size_t bytes, void *stream, lb_ctx **out);
/* Device addresses of the four face buffers (inside the context's buffer) and their size,
 * 9 * nx * ny * sizeof(stored value) bytes each. Any pointer may be NULL. */
lb_status lb_slab_faces(lb_ctx *ctx, void **send_up, void **send_down, void **recv_below,
                        void **recv_above, size_t *face_bytes);
/* record != 0: the collision records gamma and the guard count (lb_get_gamma). */
lb_status lb_slab_step_faces(lb_ctx *ctx, int32_t record);
lb_status lb_slab_step_interior(lb_ctx *ctx);
lb_status lb_slab_unpack(lb_ctx *ctx);

/* ---------------------------------------------------------------- batched ensemble
 * Many independent periodic boxes of uneven sizes and viscosities, stepped together: one
 * kernel launch per time step walks a work list of (box, row-tile) items, and n steps are
 * captured once in a CUDA graph and replayed. All boxes share storage, scheme, variant and
 * gamma_mode (taken from cfgs[0]); nx/ny/nz/nu are per box. */
typedef struct lb_batch lb_batch;

size_t lb_batch_required_bytes(const lb_config *cfgs, int32_t nbox);
lb_status lb_batch_create(const lb_config *cfgs, int32_t nbox, void *dev_buf, size_t bytes,
                          void *stream, lb_batch **out);
lb_status lb_batch_destroy(lb_batch *b);
const char *lb_batch_last_error(const lb_batch *b);
/* Per-box view: a context that aliases box `box` of the batch (init, moments, diagnostics,
 * populations). Valid until lb_batch_destroy; do not lb_destroy it. Its lb_step steps that
 * box alone. */
lb_ctx *lb_batch_box(lb_batch *b, int32_t box);
/* Advance every box n >= 0 steps by replaying CUDA graphs of at most 64 steps each (each
 * captured on first use for its length and step parity, so at most 130 graphs are kept).
 * Asynchronous. LB_ERR_OOM if host memory runs out while capturing. */
lb_status lb_batch_step(lb_batch *b, int64_t n);
/* Diagnostics of every box into out[nbox]. Synchronises. */
lb_status lb_batch_diagnostics(lb_batch *b, lb_diag *out);
/* Kernel of the batched step, all with the same bits per storage type: LB_KERNEL_ADJ (two
 * adjacent nodes (x, x+1) per thread on FP32x2 instructions, 128 threads per block; LB_F32 /
 * LB_F16, every box with an even nx, natural moments; else LB_ERR_UNSUPPORTED),
 * LB_KERNEL_PACKED (nodes (n, n+32) of an item per thread on FP32x2 instructions, 128 threads
 * per block; LB_F32 / LB_F16), LB_KERNEL_DIRECT (one node per thread), or LB_KERNEL_AUTO
 * (default: ADJ where it applies, else PACKED when the arithmetic is FP32, else DIRECT). */
lb_status lb_batch_set_kernel(lb_batch *b, int32_t kind);
/* Launch shape of the batched step: `threads` per block (multiple of 32, <= 512; 128 for the
 * ADJ and PACKED kernels) and `tile`,
 * the target number of nodes per work item (an item is ceil(tile / nx) whole x-rows of one
 * box). The grid is persistent: SMs x resident blocks, clamped to the number of items. */
lb_status lb_batch_set_tile(lb_batch *b, int32_t threads, int32_t tile);
/* Time each candidate (threads in {128, 256, 512}) x (tile in {256 .. 4096}) for
 * `trial_steps` steps on the current state and keep the fastest. The state advances by the
 * trial steps, so call it on a throw-away state like the one to be run (e.g. the initial
 * fields) and initialise again afterwards. Not on the rest state with LB_F32 storage: there
 * every node's <dh|dh> is 0 and takes the FP64 re-collision, which would be timed instead.
 * Outputs may be NULL; best_ms is the best time per step. Synchronises. */
lb_status lb_batch_autotune(lb_batch *b, int32_t trial_steps, int32_t *best_threads,
                            int32_t *best_tile, double *best_ms);

#ifdef __cplusplus
}
#endif
#endif /* KBC_LB_H */
