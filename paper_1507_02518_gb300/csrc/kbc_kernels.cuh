// kbc_kernels.cuh -- CUDA kernels of the D3Q27 KBC step and their launchers.
//
// Included once per storage type by kbc_f64.cu / kbc_f32.cu / kbc_f16.cu, which instantiate
// kbc::Ops<S>. Hot path: step_kernel / pair_step_kernel (one fused stream + KBC collide per
// node, eq:Egeneral) and batch_kernel / batch_pair_kernel (the same update over a work list of
// boxes). Transfer, diagnostics and pre-solve kernels are in kbc_aux.cuh.
#pragma once

#include <type_traits>

#include "kbc_device.cuh"
#include "kbc_ops.h"
#include "kbc_staged.cuh"
#include "kbc_tma.cuh"

namespace kbc {

// FP64 arithmetic needs more than 128 registers per thread: cap its blocks at 256 threads
template <typename S> struct MaxThreads { static constexpr int value = 512; };
template <> struct MaxThreads<double> { static constexpr int value = 256; };

template <typename S, int MODE, bool RECORD, bool CENTRAL, bool EXACT = false,
          bool POLY = false>
__global__ void __launch_bounds__(MaxThreads<S>::value) step_kernel(const S* src, S* dst, Geo g, CollideParams cp,
                                                   float* gamma_out, StepCounters* ctr) {
  const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t y = blockIdx.y * blockDim.y + threadIdx.y;
  const uint32_t z = blockIdx.z + g.zb;
  if (x >= g.nx || y >= g.ny) return;
  node_update<S, MODE, RECORD, CENTRAL, EXACT, POLY>(src, dst, g, x, y, z, cp, gamma_out, ctr);
}

// Moves node (x, y, z) of a box with rows of nx nodes and planes of ny rows k nodes forward in
// the node order (x fastest); x may start at or beyond nx (it is reduced first).
__device__ __forceinline__ void advance_node(uint32_t& x, uint32_t& y, uint32_t& z, uint32_t k,
                                             uint32_t nx, uint32_t ny) {
  x += k;
  if (x >= nx) {
    const uint32_t r = x / nx;
    x -= r * nx;
    y += r;
    if (y >= ny) {
      const uint32_t p = y / ny;
      y -= p * ny;
      z += p;
    }
  }
}

// Two nodes per thread with packed FP32x2 arithmetic: a block of up to 128 threads covers
// 2 x blockDim.x consecutive x nodes of one row, each warp 64 of them as (x, x + 32) pairs.
template <typename S, int MODE, bool RECORD, bool CENTRAL, bool POLY = false>
__global__ void __launch_bounds__(128, 3) pair_step_kernel(const S* src, S* dst, Geo g,
                                                        CollideParams cp, float* gamma_out,
                                                        StepCounters* ctr) {
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t xa = blockIdx.x * (2 * blockDim.x) + warp * 64 + lane;
  if (xa >= g.nx) return;
  const bool vb = xa + 32 < g.nx;
  const uint32_t z = blockIdx.z + g.zb;
  node_update2<S, MODE, RECORD, CENTRAL, POLY>(src, dst, g, xa, blockIdx.y, z,
                                               vb ? xa + 32 : xa, blockIdx.y, z, vb,
                                               cp, gamma_out, ctr);
}

// Two adjacent nodes per thread, (x, x + 1) with x even: a block of blockDim.x threads covers
// 2 blockDim.x consecutive nodes of one row (nx even).
template <typename S, int MODE, bool RECORD>
__global__ void __launch_bounds__(128, 3) adj_step_kernel(const S* src, S* dst, Geo g,
                                                       CollideParams cp, float* gamma_out,
                                                       StepCounters* ctr) {
  const uint32_t x = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (x >= g.nx) return;
  node_update_adj<S, MODE, RECORD>(src, dst, g, x, blockIdx.y, blockIdx.z + g.zb, cp,
                                   gamma_out, ctr);
}

template <typename S, int MODE, bool RECORD>
static cudaError_t launch_adj(const S* src, S* dst, const Geo& g, const CollideParams& cp,
                              float* gamma_out, StepCounters* ctr, cudaStream_t st) {
  const uint32_t pairs = g.nx / 2;
  const uint32_t threads = pairs >= 128 ? 128 : (pairs + 31) / 32 * 32;
  const dim3 grid((pairs + threads - 1) / threads, g.ny, g.ze - g.zb);
  adj_step_kernel<S, MODE, RECORD><<<grid, threads, 0, st>>>(src, dst, g, cp, gamma_out, ctr);
  return cudaGetLastError();
}

// The same update over the box's node order instead of rows: block k covers nodes
// [256 k, 256 k + 256), each warp 64 of them as pairs (n, n + 32), which may straddle rows.
// For row lengths that are not a multiple of 64 this keeps every lane busy, at the price of
// two divisions per thread for the coordinates and of two coordinate triples kept live.
template <typename S, int MODE, bool RECORD, bool CENTRAL, bool POLY = false>
__global__ void __launch_bounds__(128, 3) pair_linear_kernel(const S* src, S* dst, Geo g,
                                                          CollideParams cp, float* gamma_out,
                                                          StepCounters* ctr) {
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t nend = g.ze * g.nxy;  // P < 2^31
  const uint32_t n = g.zb * g.nxy + blockIdx.x * 256 + warp * 64 + lane;
  if (n >= nend) return;
  const uint32_t row = n / g.nx;
  const uint32_t xa = n - row * g.nx;
  const uint32_t za = row / g.ny;
  const uint32_t ya = row - za * g.ny;
  uint32_t xb = xa, yb = ya, zb = za;
  const bool vb = n + 32 < nend;
  if (vb) advance_node(xb, yb, zb, 32, g.nx, g.ny);
  node_update2<S, MODE, RECORD, CENTRAL, POLY, false>(src, dst, g, xa, ya, za, xb, yb, zb, vb,
                                                      cp, gamma_out, ctr);
}

// Warps per block of the pair kernel: a row needs ceil(nx / 64) warps; blocks of w <= 4 warps
// launch ceil(rows' warps / w) w warps per row, so take the w with the fewest warps left
// without nodes (the larger w on a tie): nx = 100 -> 2, 256 -> 4, 400 -> 1, 600 -> 2.
inline uint32_t pair_block_warps(uint32_t nx) {
  const uint32_t need = (nx + 63) / 64;
  uint32_t best = 4, best_idle = (need + 3) / 4 * 4 - need;
  for (uint32_t w = 3; w >= 1; --w) {
    const uint32_t idle = (need + w - 1) / w * w - need;
    if (idle < best_idle) {
      best = w;
      best_idle = idle;
    }
  }
  return best;
}

// Blocks of whole row segments (a persistent grid measured slower on GB300), sized by
// pair_block_warps; when that leaves more than 5 % of the lanes without a node (rows that are
// not close to a multiple of 64 nodes long), blocks of 256 consecutive nodes instead.
template <typename S, int MODE, bool RECORD, bool CENTRAL, bool POLY = false>
static cudaError_t launch_pair(const S* src, S* dst, const Geo& g, const CollideParams& cp,
                               float* gamma_out, StepCounters* ctr, cudaStream_t st) {
  const uint32_t warps = pair_block_warps(g.nx);
  const uint32_t row_blocks = (g.nx + 64 * warps - 1) / (64 * warps);
  const uint64_t nodes = (uint64_t)(g.ze - g.zb) * g.nxy;
  if (20 * (uint64_t)g.nx < 19 * (uint64_t)row_blocks * 64 * warps) {
    pair_linear_kernel<S, MODE, RECORD, CENTRAL, POLY>
        <<<(unsigned)((nodes + 255) / 256), 128, 0, st>>>(src, dst, g, cp, gamma_out, ctr);
    return cudaGetLastError();
  }
  const dim3 grid(row_blocks, g.ny, g.ze - g.zb);
  pair_step_kernel<S, MODE, RECORD, CENTRAL, POLY><<<grid, 32 * warps, 0, st>>>(
      src, dst, g, cp, gamma_out, ctr);
  return cudaGetLastError();
}

// the geometry and collision parameters of box `bd` of a batch (the whole box is stepped;
// flagged nodes also set the batch-wide flag fb_batch)
__device__ __forceinline__ Geo box_geo(const BoxDesc& bd, unsigned int* fb_batch) {
  Geo g;
  g.nx = bd.nx;
  g.ny = bd.ny;
  g.nz = bd.nz;
  g.nxy = bd.nxy;
  g.P = (uint64_t)bd.nxy * bd.nz;
  g.zb = 0;
  g.ze = bd.nz;
  g.fbmask = bd.fbmask;
  g.fb_any = &bd.ctr->fb_any;
  g.fb_batch = fb_batch;
  return g;
}

__device__ __forceinline__ CollideParams box_cp(const BoxDesc& bd, int with_t, int with_q,
                                                int gamma_mode) {
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
  return cp;
}

// Batched ensemble: a persistent grid walks the work list; item k covers rows
// [row0, row0 + nrows) (row = y + ny z) of one box.
template <typename S, int MODE, bool RECORD, bool CENTRAL>
__global__ void __launch_bounds__(MaxThreads<S>::value) batch_kernel(const BoxDesc* __restrict__ boxes,
                                                    const WorkItem* __restrict__ items,
                                                    int nitems, BatchFlags* flags, int parity,
                                                    int with_t, int with_q, int gamma_mode) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const WorkItem w = items[it];
    const BoxDesc bd = boxes[w.box];
    const Geo g = box_geo(bd, &flags->any);
    const CollideParams cp = box_cp(bd, with_t, with_q, gamma_mode);
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
                                                           int nitems, BatchFlags* flags, int parity,
                                                           int with_t, int with_q, int gamma_mode) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const WorkItem w = items[it];
    const BoxDesc bd = boxes[w.box];
    const Geo g = box_geo(bd, &flags->any);
    const CollideParams cp = box_cp(bd, with_t, with_q, gamma_mode);
    const S* src = (const S*)bd.pop[MODE == MODE_PULL ? parity : 0];
    S* dst = (S*)bd.pop[MODE == MODE_PULL ? (parity ^ 1) : 0];
    // The item's rows are one contiguous range of nodes: warp q handles its nodes
    // [64 q, 64 q + 64) as pairs (n, n + 32), so rows of any length keep every lane busy
    // (rows shorter or longer than a multiple of 64 nodes share warps). The coordinates of
    // a advance by the block's 256 nodes per iteration, those of b are a's plus 32; a row
    // crossing costs one division, none otherwise. blockDim.x is 128 for this kernel.
    const uint32_t nodes = bd.nx * (uint32_t)w.nrows;
    const uint32_t wstep = blockDim.x >> 5, slot = threadIdx.x & 31;
    const uint32_t stride = 64 * wstep;
    uint32_t la = 64 * (threadIdx.x >> 5) + slot;
    uint32_t za = (uint32_t)w.row0 / bd.ny;
    uint32_t ya = (uint32_t)w.row0 - za * bd.ny, xa = 0;
    advance_node(xa, ya, za, la, bd.nx, bd.ny);
    for (; la < nodes; la += stride) {
      uint32_t xb = xa, yb = ya, zb = za;
      const bool vb = la + 32 < nodes;
      if (vb) advance_node(xb, yb, zb, 32, bd.nx, bd.ny);
      node_update2<S, MODE, RECORD, CENTRAL, false, false>(src, dst, g, xa, ya, za, xb, yb, zb,
                                                           vb, cp, bd.gamma, bd.ctr);
      advance_node(xa, ya, za, stride, bd.nx, bd.ny);
    }
  }
}

// The adjacent-pair form of the batched step (every box of the batch has an even nx; product
// form, natural moments): each thread takes nodes (x, x + 1) of a row, x even, walking the
// item's node range 256 nodes per block pass (coordinates advance incrementally).
template <typename S, int MODE, bool RECORD>
__global__ void __launch_bounds__(128, 3) batch_adj_kernel(const BoxDesc* __restrict__ boxes,
                                                          const WorkItem* __restrict__ items,
                                                          int nitems, BatchFlags* flags, int parity,
                                                          int with_t, int with_q, int gamma_mode) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const WorkItem w = items[it];
    const BoxDesc bd = boxes[w.box];
    const Geo g = box_geo(bd, &flags->any);
    const CollideParams cp = box_cp(bd, with_t, with_q, gamma_mode);
    const S* src = (const S*)bd.pop[MODE == MODE_PULL ? parity : 0];
    S* dst = (S*)bd.pop[MODE == MODE_PULL ? (parity ^ 1) : 0];
    const uint32_t nodes = bd.nx * (uint32_t)w.nrows;
    const uint32_t stride = 2 * blockDim.x;
    uint32_t n = 2 * threadIdx.x;
    uint32_t z = (uint32_t)w.row0 / bd.ny;
    uint32_t y = (uint32_t)w.row0 - z * bd.ny, x = 0;
    advance_node(x, y, z, n, bd.nx, bd.ny);
    for (; n < nodes; n += stride) {
      node_update_adj<S, MODE, RECORD>(src, dst, g, x, y, z, cp, bd.gamma, bd.ctr);
      advance_node(x, y, z, stride, bd.nx, bd.ny);
    }
  }
}

// ------------------------------------------------------------------ FP64 re-collision pass
// A step kernel (FP32 storage) that meets a node whose FP32 <dh|dh> fell under kDenFp64 sets
// its bit in the box's mask (flag_fp64) and, in AA, does not store it. The pass launched
// after it collides every flagged node again in FP64 from its inputs (fp64_node_update) and
// clears the mask. When nothing was flagged (the usual case) it
// reads one flag and exits. The last of its blocks to finish clears the flags; all blocks
// have read them by then.
constexpr int kPassThreads = 256;
constexpr int kPassBlocks = 152;  // one wave: the pass kernels run one block per SM

// the flagged nodes among mask words w = w0, w0 + stride, ...; returns the guard events
template <typename S, int MODE, bool CENTRAL, bool POLY>
__device__ unsigned long long fp64_pass_words(const S* src, S* dst, const Geo& g,
                                              const CollideParams& cp,
                                              float* gamma_out, int record, uint32_t w0,
                                              uint32_t stride) {
  const uint32_t words = (uint32_t)((g.P + 31) >> 5);
  unsigned long long guards = 0;
  for (uint32_t w = w0; w < words; w += stride) {
    uint32_t m = g.fbmask[w];
    if (m == 0) continue;
    g.fbmask[w] = 0;
    while (m) {
      const uint32_t n = 32 * w + (uint32_t)(__ffs(m) - 1);
      m &= m - 1;
      const uint32_t z = n / g.nxy, r = n - z * g.nxy;
      const uint32_t y = r / g.nx, x = r - y * g.nx;
      int gd = 0;
      const float gam = fp64_node_update<S, MODE, CENTRAL, POLY>(src, dst, g, x, y, z, cp, &gd);
      if (record) {
        gamma_out[n] = gam;
        guards += (unsigned long long)gd;
      }
    }
  }
  return guards;
}

// true in thread 0 of the last block of the grid to get here (after __syncthreads)
__device__ __forceinline__ bool pass_last_block(unsigned int* done) {
  __syncthreads();
  if (threadIdx.x != 0) return false;
  __threadfence();
  return atomicAdd(done, 1u) == gridDim.x - 1;
}

template <typename S, int MODE, bool CENTRAL, bool POLY>
__global__ void __launch_bounds__(kPassThreads) fp64_pass_kernel(const S* src, S* dst, Geo g,
                                                                 CollideParams cp,
                                                                 float* gamma_out,
                                                                 StepCounters* ctr, int record) {
  if (*(volatile unsigned int*)&ctr->fb_any == 0) return;
  const unsigned long long guards =
      fp64_pass_words<S, MODE, CENTRAL, POLY>(src, dst, g, cp, gamma_out, record,
                                              blockIdx.x * blockDim.x + threadIdx.x,
                                              gridDim.x * blockDim.x);
  if (guards) atomicAdd(&ctr->guarded, guards);
  if (pass_last_block(&ctr->fb_done)) {
    ctr->fb_any = 0;
    ctr->fb_done = 0;
  }
}

// the same over the boxes of a batch (boxes that flagged nothing are skipped)
template <typename S, int MODE, bool CENTRAL>
__global__ void __launch_bounds__(kPassThreads) batch_fp64_pass_kernel(
    const BoxDesc* __restrict__ boxes, int nbox, BatchFlags* flags, int parity, int with_t,
    int with_q, int gamma_mode, int record) {
  if (*(volatile unsigned int*)&flags->any == 0) return;
  for (int k = 0; k < nbox; ++k) {
    const BoxDesc bd = boxes[k];
    if (*(volatile unsigned int*)&bd.ctr->fb_any == 0) continue;
    const Geo g = box_geo(bd, nullptr);
    const CollideParams cp = box_cp(bd, with_t, with_q, gamma_mode);
    const S* src = (const S*)bd.pop[MODE == MODE_PULL ? parity : 0];
    S* dst = (S*)bd.pop[MODE == MODE_PULL ? (parity ^ 1) : 0];
    const unsigned long long guards =
        fp64_pass_words<S, MODE, CENTRAL, false>(src, dst, g, cp, bd.gamma, record,
                                                 blockIdx.x * blockDim.x + threadIdx.x,
                                                 gridDim.x * blockDim.x);
    if (guards) atomicAdd(&bd.ctr->guarded, guards);
  }
  if (pass_last_block(&flags->done)) {
    for (int k = 0; k < nbox; ++k) boxes[k].ctr->fb_any = 0;
    flags->any = 0;
    flags->done = 0;
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
  g.zb = b.zb;
  g.ze = b.ze;
  g.fbmask = b.fbmask;
  g.fb_any = nullptr;
  g.fb_batch = nullptr;
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

template <typename S, int MODE, bool RECORD, bool CENTRAL, bool POLY>
static cudaError_t launch_step_c(const BoxView& b, const S* src, S* dst, const Geo& g,
                                 const CollideParams& cp, const StepOpts& o, StepCounters* ctr,
                                 cudaStream_t st) {
  if constexpr (!POLY) {
    if (cp.gamma_mode == GAMMA_EXACT) {  // one node per thread, whatever kernel was chosen
      const dim3 block(o.bx, o.by, 1);
      const dim3 grid((b.nx + o.bx - 1) / o.bx, (b.ny + o.by - 1) / o.by, g.ze - g.zb);
      step_kernel<S, MODE, RECORD, CENTRAL, true><<<grid, block, 0, st>>>(src, dst, g, cp,
                                                                          b.gamma, ctr);
      return cudaGetLastError();
    }
  }
  if constexpr (!CENTRAL && !POLY) {
    if (o.kernel == KERNEL_STAGED)
      return launch_staged<S, MODE, RECORD>(src, dst, g, cp, b.gamma, ctr, o.budget, o.stall, st);
    if (o.kernel == KERNEL_PERSISTENT)
      return launch_persistent<S, MODE, RECORD>(src, dst, g, cp, b.gamma, ctr,
                                                (uint32_t)o.prefetch, st);
  }
  if constexpr (!std::is_same<S, double>::value) {
    if constexpr (!CENTRAL && !POLY) {
      if (o.kernel == KERNEL_ROWS)
        return launch_rows<S, MODE, RECORD>(src, dst, g, cp, b.gamma, ctr, o.budget, o.stall, st);
      // the default for even rows: adjacent pairs (measured faster than (x, x + 32) pairs at
      // 256^3: FP32 AA 0.549 vs 0.630 ms, FP16 AA 0.446 vs 0.504 ms, pull equal or better)
      if ((o.kernel == KERNEL_ADJ || o.kernel == KERNEL_AUTO) && g.nx % 2 == 0)
        return launch_adj<S, MODE, RECORD>(src, dst, g, cp, b.gamma, ctr, st);
    }
    if (o.kernel == KERNEL_PACKED || o.kernel == KERNEL_AUTO || o.kernel == KERNEL_ROWS)
      return launch_pair<S, MODE, RECORD, CENTRAL, POLY>(src, dst, g, cp, b.gamma, ctr, st);
  }
  const dim3 block(o.bx, o.by, 1);
  const dim3 grid((b.nx + o.bx - 1) / o.bx, (b.ny + o.by - 1) / o.by, g.ze - g.zb);
  step_kernel<S, MODE, RECORD, CENTRAL, false, POLY><<<grid, block, 0, st>>>(src, dst, g, cp,
                                                                             b.gamma, ctr);
  return cudaGetLastError();
}

// the step kernel, then (FP32 storage, the estimate of eq:result21: the only case that
// flags nodes) the FP64 re-collision pass over the nodes it flagged
template <typename S, int MODE, bool RECORD, bool CENTRAL, bool POLY>
static cudaError_t launch_step_p(const BoxView& b, const S* src, S* dst, const Geo& g,
                                 const CollideParams& cp, const StepOpts& o, StepCounters* ctr,
                                 cudaStream_t st) {
  cudaError_t e = launch_step_c<S, MODE, RECORD, CENTRAL, POLY>(b, src, dst, g, cp, o, ctr, st);
  if constexpr (std::is_same<S, float>::value) {
    if (e == cudaSuccess && cp.gamma_mode == GAMMA_ESTIMATE) {
      const uint64_t words = (g.P + 31) / 32;
      uint64_t blocks = (words + kPassThreads - 1) / kPassThreads;
      if (blocks > (uint64_t)kPassBlocks) blocks = kPassBlocks;
      fp64_pass_kernel<S, MODE, CENTRAL, POLY><<<(unsigned)blocks, kPassThreads, 0, st>>>(
          src, dst, g, cp, b.gamma, ctr, RECORD ? 1 : 0);
      e = cudaGetLastError();
    }
  }
  return e;
}

template <typename S, int MODE, bool RECORD>
static cudaError_t launch_step(const BoxView& b, const S* src, S* dst, const Geo& g,
                               const CollideParams& cp, const StepOpts& o, StepCounters* ctr,
                               cudaStream_t st) {
  if (b.poly) {
    if (b.central)
      return launch_step_p<S, MODE, RECORD, true, true>(b, src, dst, g, cp, o, ctr, st);
    return launch_step_p<S, MODE, RECORD, false, true>(b, src, dst, g, cp, o, ctr, st);
  }
  if (b.central)
    return launch_step_p<S, MODE, RECORD, true, false>(b, src, dst, g, cp, o, ctr, st);
  return launch_step_p<S, MODE, RECORD, false, false>(b, src, dst, g, cp, o, ctr, st);
}

template <typename S>
bool Ops<S>::staged_ok(uint32_t nx) {
  return staged_supported<S>(nx);
}

template <typename S>
bool Ops<S>::rows_ok(uint32_t nx, uint32_t ny, uint32_t nz) {
  if constexpr (std::is_same<S, double>::value) {
    return false;
  } else {
    Geo g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.nxy = nx * ny;
    g.P = (uint64_t)nx * ny * nz;
    g.zb = 0;
    g.ze = nz;
    g.fbmask = nullptr;
    g.fb_any = g.fb_batch = nullptr;
    RowsArgs a;
    return rows_shape<S>(g, &a);
  }
}

template <typename S>
cudaError_t Ops<S>::step(const BoxView& b, int64_t t, bool record, const StepOpts& o,
                         StepCounters* counters, cudaStream_t st) {
  Geo g = make_geo(b);
  g.fb_any = &counters->fb_any;
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

// Launch arguments shared by the batch kernels.
struct BatchArgs {
  const BoxDesc* boxes;
  int nbox;
  BatchFlags* flags;
  const WorkItem* items;
  int nitems, parity, with_t, with_q, gamma_mode, threads, grid;
};

template <typename S, int MODE, bool CENTRAL>
static void launch_batch_c(const BatchArgs& a, bool record, int packed, cudaStream_t st) {
  if constexpr (!std::is_same<S, double>::value) {
    if constexpr (!CENTRAL) {
      if (packed == 2) {
        if (record)
          batch_adj_kernel<S, MODE, true><<<a.grid, 128, 0, st>>>(
              a.boxes, a.items, a.nitems, a.flags, a.parity, a.with_t, a.with_q, a.gamma_mode);
        else
          batch_adj_kernel<S, MODE, false><<<a.grid, 128, 0, st>>>(
              a.boxes, a.items, a.nitems, a.flags, a.parity, a.with_t, a.with_q, a.gamma_mode);
        return;
      }
    }
    if (packed) {
      if (record)
        batch_pair_kernel<S, MODE, true, CENTRAL><<<a.grid, 128, 0, st>>>(
            a.boxes, a.items, a.nitems, a.flags, a.parity, a.with_t, a.with_q, a.gamma_mode);
      else
        batch_pair_kernel<S, MODE, false, CENTRAL><<<a.grid, 128, 0, st>>>(
            a.boxes, a.items, a.nitems, a.flags, a.parity, a.with_t, a.with_q, a.gamma_mode);
      return;
    }
  }
  if (record)
    batch_kernel<S, MODE, true, CENTRAL><<<a.grid, a.threads, 0, st>>>(
        a.boxes, a.items, a.nitems, a.flags, a.parity, a.with_t, a.with_q, a.gamma_mode);
  else
    batch_kernel<S, MODE, false, CENTRAL><<<a.grid, a.threads, 0, st>>>(
        a.boxes, a.items, a.nitems, a.flags, a.parity, a.with_t, a.with_q, a.gamma_mode);
}

template <typename S, int MODE>
static void launch_batch(const BatchArgs& a, bool record, int packed, bool central,
                         cudaStream_t st) {
  if (central)
    launch_batch_c<S, MODE, true>(a, record, packed, st);
  else
    launch_batch_c<S, MODE, false>(a, record, packed, st);
  if constexpr (std::is_same<S, float>::value) {
    if (a.gamma_mode == GAMMA_ESTIMATE) {  // the FP32 kernels' flagged nodes, in FP64
      if (central)
        batch_fp64_pass_kernel<S, MODE, true><<<kPassBlocks, kPassThreads, 0, st>>>(
            a.boxes, a.nbox, a.flags, a.parity, a.with_t, a.with_q, a.gamma_mode, record);
      else
        batch_fp64_pass_kernel<S, MODE, false><<<kPassBlocks, kPassThreads, 0, st>>>(
            a.boxes, a.nbox, a.flags, a.parity, a.with_t, a.with_q, a.gamma_mode, record);
    }
  }
}

template <typename S>
cudaError_t Ops<S>::batch_step(const BoxDesc* boxes, int nbox, BatchFlags* flags,
                               const WorkItem* items, int nitems, int64_t t, bool record,
                               int packed, int scheme, int with_t, int with_q, int central,
                               int gamma_mode, int threads, int grid, cudaStream_t st) {
  BatchArgs a;
  a.boxes = boxes;
  a.nbox = nbox;
  a.flags = flags;
  a.items = items;
  a.nitems = nitems;
  a.parity = (int)(t & 1);
  a.with_t = with_t;
  a.with_q = with_q;
  a.gamma_mode = gamma_mode;
  a.threads = threads;
  a.grid = grid;
  if (scheme == 0)
    launch_batch<S, MODE_PULL>(a, record, packed, central != 0, st);
  else if (a.parity == 0)
    launch_batch<S, MODE_AA_EVEN>(a, record, packed, central != 0, st);
  else
    launch_batch<S, MODE_AA_ODD>(a, record, packed, central != 0, st);
  return cudaGetLastError();
}

template <typename S>
int Ops<S>::batch_occupancy(int threads, int scheme, int packed) {
  int blocks = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if constexpr (!std::is_same<S, double>::value) {
    if (packed == 2) {
      if (scheme == 0)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &blocks, batch_adj_kernel<S, MODE_PULL, false>, 128, 0);
      else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &blocks, batch_adj_kernel<S, MODE_AA_ODD, false>, 128, 0);
      if (e != cudaSuccess || blocks < 1) blocks = 1;
      return blocks;
    }
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

#include "kbc_aux.cuh"
