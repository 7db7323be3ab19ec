// kbc_ops.h -- host-side launch interface of the per-storage kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kbc {

struct BoxView {
  uint32_t nx, ny, nz;
  uint64_t P;          // nx * ny * nz
  void* pop[2];        // population buffers (pull: two; AA: pop[1] == pop[0])
  float* gamma;        // [P] stabilizer of the last recorded collision
  uint32_t* fbmask;    // [ceil(P / 32)] nodes flagged for the FP64 re-collision (zero between
                       // steps)
  double beta;
  int with_t, with_q, gamma_mode;
  int central;         // shear part in the central-moment basis
  int poly;            // polynomial equilibrium eq:polynomial2 instead of the product form
  int scheme;          // 0 pull, 1 AA
  uint32_t zb, ze;     // planes zb <= z < ze are stepped (a whole box: 0, nz)
};

// counters written by the step kernels: guard events of the recorded collision, a flag set
// when a bounded device-side wait ran out, and the state of the FP64 re-collision pass
// (fb_any: a step kernel flagged a node in fbmask; fb_done: blocks of the pass that finished)
struct StepCounters {
  unsigned long long guarded;
  unsigned int timeout;
  unsigned int fb_any;
  unsigned int fb_done;
  unsigned int pad;
};

// the batch-wide flag of the FP64 re-collision pass (some box flagged a node) and its count
// of finished blocks
struct BatchFlags {
  unsigned int any;
  unsigned int done;
};

// kernel choice and test hooks of one step launch
enum {
  KERNEL_AUTO = 0,
  KERNEL_DIRECT = 1,
  KERNEL_STAGED = 2,
  KERNEL_PERSISTENT = 3,
  KERNEL_PACKED = 4,
  KERNEL_ROWS = 5,
  KERNEL_ADJ = 6
};
struct StepOpts {
  int bx, by;                 // block of the direct kernel
  int kernel;                 // KERNEL_*
  int prefetch;               // L2 prefetch distance of the persistent kernel (items)
  unsigned long long budget;  // wait budget (SM cycles) of the staged kernel
  int stall;                  // test hook: the staged kernel issues no copies
};

// one item of the batched work list: rows [row0, row0 + nrows) of box `box`
// (row = y + ny * z)
struct WorkItem {
  int32_t box;
  int32_t row0;
  int32_t nrows;
  int32_t pad;
};

// device-side description of one box of a batch
struct BoxDesc {
  uint32_t nx, ny, nz, nxy;
  void* pop[2];
  float* gamma;
  uint32_t* fbmask;
  StepCounters* ctr;
  double beta, two_beta, inv_beta;
};

template <typename S> struct Ops {
  // one time step t -> t+1 of one box; `record` writes gamma and counts guards
  static cudaError_t step(const BoxView& b, int64_t t, bool record, const StepOpts& o,
                          StepCounters* counters, cudaStream_t st);
  // whether the staged (bulk-copy pipelined) kernel supports this row length
  static bool staged_ok(uint32_t nx);
  // whether the row-staged pair kernel (KERNEL_ROWS) takes this box
  static bool rows_ok(uint32_t nx, uint32_t ny, uint32_t nz);
  // canonical f(t) = f_eq(rho, u) for nodes [n0, n0 + cnt) (rho may be null: 1)
  static cudaError_t init(const BoxView& b, int64_t t, const double* rho, const double* u,
                          uint64_t n0, uint64_t cnt, uint64_t ld, cudaStream_t st);
  // out[i * ld + (n - n0)] = canonical f_i(n, t) for n in [n0, n0 + cnt)
  static cudaError_t get(const BoxView& b, int64_t t, double* out, uint64_t n0, uint64_t cnt,
                         uint64_t ld, cudaStream_t st);
  static cudaError_t set(const BoxView& b, int64_t t, const double* in, uint64_t n0,
                         uint64_t cnt, uint64_t ld, cudaStream_t st);
  // rho[n - n0], u[a * ld + (n - n0)] of f(t)
  static cudaError_t moments(const BoxView& b, int64_t t, double* rho, double* u, uint64_t n0,
                             uint64_t cnt, uint64_t ld, cudaStream_t st);
  // diagnostics: writes u (arithmetic type of S) to ufield[3][P] and per-block partial sums
  // order: 2 or 8, the order of the central differences of the velocity gradients
  static cudaError_t diag(const BoxView& b, int64_t t, bool with_gamma, int order, void* ufield,
                          double* partials, int nblocks, double* sums, cudaStream_t st);
  // one density pre-solve iteration t -> t+1 with the velocity held at u0 ([3][P], collision
  // precision); `store` keeps rho - 1 of f(t) in b.gamma for rho_change
  static cudaError_t presolve_step(const BoxView& b, int64_t t, double beta_pre, const void* u0,
                                   bool store, const StepOpts& o, cudaStream_t st);
  // *resid = FP32 bits of max |rho(f(t)) - 1 - b.gamma| (zeroed first)
  static cudaError_t rho_change(const BoxView& b, int64_t t, unsigned int* resid, int nblocks,
                                cudaStream_t st);
  // ufield[a][n0 + k] = u[a * ld + k] in the collision precision
  static cudaError_t convert_u(const double* u, void* ufield, uint64_t n0, uint64_t cnt,
                               uint64_t ld, uint64_t P, cudaStream_t st);
  // stabilizer gap of canonical f(t): sums[0..6] as laid out by gap_kernel
  static cudaError_t gamma_gap(const BoxView& b, int64_t t, double* partials, int nblocks,
                               double* sums, cudaStream_t st);
  // one time step of every box of a batch over a work list
  // (packed: 0 one node per thread; 1 the FP32x2 (n, n + 32) pairs, 128 threads; 2 the FP32x2
  // adjacent pairs (x, x + 1), 128 threads, every nx even, natural moments; FP32 arithmetic)
  // (flags: the batch's FP64 re-collision flag; nbox boxes)
  static cudaError_t batch_step(const BoxDesc* boxes, int nbox, BatchFlags* flags,
                                const WorkItem* items, int nitems,
                                int64_t t, bool record, int packed, int scheme, int with_t,
                                int with_q, int central, int gamma_mode, int threads, int grid,
                                cudaStream_t st);
  // resident blocks per SM of the batch kernel at this block size
  static int batch_occupancy(int threads, int scheme, int packed);
};

// kinetic-energy spectrum (kbc_spectrum.cu): work bytes for an n^3 velocity field in FP64 or
// FP32 with nbins shells (0 if cuFFT cannot plan it), and the spectrum itself; returns 0, or
// 2 (work too small) / 3 (cuFFT or CUDA failure) with *why set
size_t spectrum_work_bytes(uint32_t n, bool fp64, int nbins);
int spectrum(const void* ufield, uint32_t n, bool fp64, int nbins, void* work, size_t work_bytes,
             double* bins_host, cudaStream_t st, const char** why);

constexpr int kDiagSums = 24;   // layout of the diagnostics sums, see kbc_kernels.cuh
constexpr int kDiagBlocks = 608;  // fixed grid of the reduction kernels (4 per SM on 152 SMs)

}  // namespace kbc
