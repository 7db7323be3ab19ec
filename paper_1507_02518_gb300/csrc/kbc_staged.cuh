// kbc_staged.cuh -- the KBC step with its loads staged through shared memory by the bulk-copy
// (TMA) engine in a multi-stage mbarrier pipeline (sm_90+ PTX, built for sm_103a).
//
// Work item = one x-segment of kSeg nodes of one (y, z) row. For each of the 27 populations the
// source row segment (shifted by the streaming pattern in y and z) plus a 16-byte halo on each
// side is copied into shared memory with cp.async.bulk; the +-1 shifts in x and the periodic
// wrap at the row ends are then plain shared-memory indexing. A persistent grid walks the items;
// each CTA keeps kStages items in flight, so the bytes in flight no longer depend on registers
// or occupancy. Stores go straight from registers to global memory (coalesced).
//
// Every wait on an mbarrier is bounded by a clock64 budget; on expiry the CTA sets the
// context's timeout flag and exits (no copies are left in flight: a stage is only waited on
// after its copies were issued, and nothing is issued after a timeout).
#pragma once

#include "kbc_device.cuh"
#include "kbc_ops.h"

namespace kbc {

constexpr int kSeg = 128;  // nodes per work item (= threads per CTA)

template <typename S> struct StagedCfg;
// pipeline depth and the minimum resident CTAs per SM the register budget is fitted to
template <> struct StagedCfg<float> { static constexpr int stages = 3, min_blocks = 4; };
template <> struct StagedCfg<uint16_t> { static constexpr int stages = 4, min_blocks = 4; };
template <> struct StagedCfg<double> { static constexpr int stages = 2, min_blocks = 2; };

template <typename S> struct StagedLayout {
  static constexpr int H = 16 / (int)sizeof(S);  // halo elements = 16 bytes
  static constexpr int ROW = kSeg + 2 * H;       // elements per staged row
  static constexpr int STAGES = StagedCfg<S>::stages;
  static constexpr size_t stage_bytes = (size_t)27 * ROW * sizeof(S);
  static constexpr size_t bar_offset = (STAGES * stage_bytes + 15) / 16 * 16;
  static constexpr size_t smem_bytes = bar_offset + STAGES * sizeof(uint64_t);
};

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the phase with the given parity to complete, for at most `budget` SM cycles
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long budget) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((unsigned long long)(clock64() - t0) > budget) return false;
  }
}

struct StagedArgs {
  uint32_t nseg;     // x-segments per row
  uint32_t nitems;   // nseg * ny * (ze - zb)
  unsigned long long budget;  // wait budget in SM cycles
  int stall;         // test hook: issue no copies, so every wait runs out
};

// Issue the bulk copies of one work item into one stage (called by all 32 lanes of warp 0).
template <typename S, int MODE>
__device__ __forceinline__ void staged_issue(const S* src, const Geo& g, const StagedArgs& a,
                                             uint32_t item, S* stage_buf, uint64_t* bar) {
  using L = StagedLayout<S>;
  using Pat = Pattern<MODE>;
  constexpr int H = L::H;
  const int lane = threadIdx.x & 31;
  const uint32_t seg = item % a.nseg;
  const uint32_t row = item / a.nseg + g.zb * g.ny;
  const uint32_t y = row % g.ny, z = row / g.ny;
  const uint32_t x0 = seg * kSeg;
  const uint32_t cnt = min((uint32_t)kSeg, g.nx - x0);
  if (a.stall) return;
  if (lane == 0) mbar_arrive_expect_tx(bar, 27u * (cnt + 2 * H) * (uint32_t)sizeof(S));
  __syncwarp();
  if (lane < 27) {
    const int i = lane;
    const int sy = Pat::load_shift * cy(i), sz = Pat::load_shift * cz(i);
    const uint32_t ys = sy < 0 ? (y == 0 ? g.ny - 1 : y - 1) : (sy > 0 ? (y + 1 == g.ny ? 0 : y + 1) : y);
    const uint32_t zs = sz < 0 ? (z == 0 ? g.nz - 1 : z - 1) : (sz > 0 ? (z + 1 == g.nz ? 0 : z + 1) : z);
    const S* rowp = src + (uint64_t)Pat::load_plane(i) * g.P + ((uint64_t)zs * g.ny + ys) * g.nx;
    S* dst = stage_buf + i * L::ROW;
    const uint32_t lo = x0 == 0 ? 0 : x0 - H;
    const uint32_t hi = min(x0 + cnt + H, g.nx);
    if (x0 == 0) bulk_g2s(dst, rowp + (g.nx - H), H * sizeof(S), bar);          // left wrap
    bulk_g2s(dst + H + lo - x0, rowp + lo, (hi - lo) * (uint32_t)sizeof(S), bar);  // segment
    if (x0 + cnt == g.nx) bulk_g2s(dst + H + cnt, rowp, H * sizeof(S), bar);     // right wrap
  }
}

template <typename S, int MODE, bool RECORD>
__global__ void __launch_bounds__(kSeg, StagedCfg<S>::min_blocks) staged_step_kernel(const S* src, S* dst, Geo g,
                                                           CollideParams cp, float* gamma_out,
                                                           StepCounters* ctr, StagedArgs a) {
  using C = Codec<S>;
  using R = typename C::R;
  using L = StagedLayout<S>;
  using Pat = Pattern<MODE>;
  constexpr int H = L::H;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S* sbuf = reinterpret_cast<S*>(smem_raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + L::bar_offset);
  const int tid = threadIdx.x;
  const bool producer = tid < 32;

  if (tid == 0) {
    for (int s = 0; s < L::STAGES; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (producer) {
    for (int s = 0; s < L::STAGES; ++s) {
      const uint32_t item = blockIdx.x + (uint32_t)s * gridDim.x;
      if (item < a.nitems)
        staged_issue<S, MODE>(src, g, a, item, sbuf + (size_t)s * 27 * L::ROW, &bars[s]);
    }
  }

  uint32_t k = 0;
  for (uint32_t item = blockIdx.x; item < a.nitems; item += gridDim.x, ++k) {
    const int stage = (int)(k % L::STAGES);
    const uint32_t parity = (k / L::STAGES) & 1u;
    const bool ok = mbar_wait_bounded(&bars[stage], parity, a.budget);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(&ctr->timeout, 1u);
        // let the copies already issued for the following items land (bounded) before the
        // CTA's shared memory is released
        for (int j = 1; j < L::STAGES; ++j) {
          const uint32_t later = item + (uint32_t)j * gridDim.x;
          if (later >= a.nitems || a.stall) break;
          const uint32_t kk = k + (uint32_t)j;
          mbar_wait_bounded(&bars[kk % L::STAGES], (kk / L::STAGES) & 1u, a.budget);
        }
      }
      return;
    }
    const uint32_t seg = item % a.nseg;
    const uint32_t row = item / a.nseg + g.zb * g.ny;
    const uint32_t y = row % g.ny, z = row / g.ny;
    const uint32_t x0 = seg * kSeg;
    const uint32_t cnt = min((uint32_t)kSeg, g.nx - x0);
    if ((uint32_t)tid < cnt) {
      const S* sb = sbuf + (size_t)stage * 27 * L::ROW;
      R d[27];
      Unroll<0, 27>::run([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        d[I] = C::template load_raw<I>(sb + I * L::ROW + H + tid + Pat::load_shift * cx(I));
      });
      int guarded, fp64 = 0;
      const uint32_t x = x0 + tid;
      R gamma = collide_step<R, false, false, false, C::rel>(
          d, cp, &guarded, std::is_same<S, float>::value ? &fp64 : nullptr);
      Nbr nb;
      nb.init(g, x, y, z);
      if (MODE == MODE_PULL || !fp64) {  // a flagged node is left to the FP64 pass (AA: not
                                         // stored)
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
    __syncthreads();  // every thread is done with this stage
    if (producer) {
      const uint32_t next = item + (uint32_t)L::STAGES * gridDim.x;
      if (next < a.nitems) {
        fence_proxy_async_smem();
        staged_issue<S, MODE>(src, g, a, next, sbuf + (size_t)stage * 27 * L::ROW, &bars[stage]);
      }
    }
  }
}

// ------------------------------------------------------------------ persistent + L2 prefetch
// The same 128-node row-segment items, walked by a persistent grid without shared memory:
// each thread loads its node's 27 values straight from global memory, while lanes 0..26 of
// warp 0 ask the bulk-copy engine to prefetch into L2 the 27 source row segments of the item
// `prefetch` steps ahead (cp.async.bulk.prefetch.L2: no destination, no barrier, no wait).
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

template <typename S> struct PersistCfg { static constexpr int min_blocks = 4; };
template <> struct PersistCfg<double> { static constexpr int min_blocks = 2; };

struct PersistArgs {
  uint32_t nseg, nitems;
  uint32_t prefetch;  // items ahead (0: off; needs rows of whole 16-byte multiples)
};

template <typename S, int MODE>
__device__ __forceinline__ void prefetch_item(const S* src, const Geo& g, const PersistArgs& a,
                                              uint32_t item, int lane) {
  using Pat = Pattern<MODE>;
  const uint32_t seg = item % a.nseg;
  const uint32_t row = item / a.nseg + g.zb * g.ny;
  const uint32_t y = row % g.ny, z = row / g.ny;
  const uint32_t x0 = seg * kSeg;
  const uint32_t cnt = min((uint32_t)kSeg, g.nx - x0);
  const int i = lane;
  const int sy = Pat::load_shift * cy(i), sz = Pat::load_shift * cz(i);
  const uint32_t ys = sy < 0 ? (y == 0 ? g.ny - 1 : y - 1) : (sy > 0 ? (y + 1 == g.ny ? 0 : y + 1) : y);
  const uint32_t zs = sz < 0 ? (z == 0 ? g.nz - 1 : z - 1) : (sz > 0 ? (z + 1 == g.nz ? 0 : z + 1) : z);
  const S* rowp = src + (uint64_t)Pat::load_plane(i) * g.P + ((uint64_t)zs * g.ny + ys) * g.nx;
  bulk_prefetch_l2(rowp + x0, cnt * (uint32_t)sizeof(S));
}

template <typename S, int MODE, bool RECORD>
__global__ void __launch_bounds__(kSeg, PersistCfg<S>::min_blocks)
    persistent_step_kernel(const S* src, S* dst, Geo g, CollideParams cp, float* gamma_out,
                           StepCounters* ctr, PersistArgs a) {
  const int tid = threadIdx.x;
  if (a.prefetch && tid < 27)
    for (uint32_t d = 0; d < a.prefetch; ++d) {
      const uint32_t item = blockIdx.x + d * gridDim.x;
      if (item < a.nitems) prefetch_item<S, MODE>(src, g, a, item, tid);
    }
  for (uint32_t item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    if (a.prefetch && tid < 27) {
      const uint32_t ahead = item + a.prefetch * gridDim.x;
      if (ahead < a.nitems) prefetch_item<S, MODE>(src, g, a, ahead, tid);
    }
    const uint32_t seg = item % a.nseg;
    const uint32_t row = item / a.nseg + g.zb * g.ny;
    const uint32_t y = row % g.ny, z = row / g.ny;
    const uint32_t x = seg * kSeg + tid;
    if (x < g.nx) node_update<S, MODE, RECORD>(src, dst, g, x, y, z, cp, gamma_out, ctr);
  }
}

template <typename S, int MODE, bool RECORD>
cudaError_t launch_persistent(const S* src, S* dst, const Geo& g, const CollideParams& cp,
                              float* gamma_out, StepCounters* ctr, uint32_t prefetch,
                              cudaStream_t st) {
  static int blocks_per_sm = 0;
  static int sms = 0;
  auto kern = persistent_step_kernel<S, MODE, RECORD>;
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, kSeg, 0);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  PersistArgs a;
  a.nseg = (g.nx + kSeg - 1) / kSeg;
  a.nitems = a.nseg * g.ny * (g.ze - g.zb);
  a.prefetch = (((uint64_t)g.nx * sizeof(S)) % 16 == 0) ? prefetch : 0;
  const uint32_t cap = (uint32_t)(sms * blocks_per_sm);
  const uint32_t grid = a.nitems < cap ? a.nitems : cap;
  kern<<<grid, kSeg, 0, st>>>(src, dst, g, cp, gamma_out, ctr, a);
  return cudaGetLastError();
}

// true if the staged kernel can run this box: rows are whole multiples of 16 bytes
template <typename S> inline bool staged_supported(uint32_t nx) {
  return ((uint64_t)nx * sizeof(S)) % 16 == 0;
}

template <typename S, int MODE, bool RECORD>
cudaError_t launch_staged(const S* src, S* dst, const Geo& g, const CollideParams& cp,
                          float* gamma_out, StepCounters* ctr, unsigned long long budget,
                          int stall, cudaStream_t st) {
  using L = StagedLayout<S>;
  static int blocks_per_sm = 0;
  static int sms = 0;
  auto kern = staged_step_kernel<S, MODE, RECORD>;
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L::smem_bytes);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, kSeg, L::smem_bytes);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  StagedArgs a;
  a.nseg = (g.nx + kSeg - 1) / kSeg;
  a.nitems = a.nseg * g.ny * (g.ze - g.zb);
  a.budget = budget;
  a.stall = stall;
  const uint32_t cap = (uint32_t)(sms * blocks_per_sm);
  const uint32_t grid = a.nitems < cap ? a.nitems : cap;
  kern<<<grid, kSeg, L::smem_bytes, st>>>(src, dst, g, cp, gamma_out, ctr, a);
  return cudaGetLastError();
}

}  // namespace kbc
