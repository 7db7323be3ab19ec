// kbc_tma.cuh -- the KBC step (eq:Egeneral, Sec. KBC) with its source rows staged in shared
// memory by the bulk-copy (TMA) engine, two adjacent nodes per thread on the FP32x2 collision.
//
// Design (FP32 and FP16 storage; sm_103a):
//   * work unit = a tile: R whole rows (x = 0 .. nx-1) of one z-plane when nx <= 256 (R nx <=
//     256 nodes), or one 256-node x-segment of a row when nx is a multiple of 256 above 256;
//   * for each of the 27 planes the tile's source rows -- shifted by the streaming pattern in
//     y and z -- are copied into shared memory with cp.async.bulk (1D, 16-byte aligned, up to
//     two copies per plane for a periodic wrap in y, or halo copies at the row ends of a
//     segment); the +-1 shift in x and its periodic wrap become shared-memory indices that
//     are fixed per thread;
//   * a persistent grid walks the tiles; warp 0 issues the copies of tile k + S into stage
//     k mod S as soon as every warp has read tile k out of it (mbarrier "empty"), so S tiles
//     are in flight while the collision runs from registers -- the bytes in flight no longer
//     depend on how many warps the collision's registers leave resident;
//   * thread j of a row holds nodes x = 2j and 2j + 1: the unshifted planes are one 32-bit
//     (FP16) or 64-bit (FP32) shared load, the x-shifted planes two scalar loads, and the pull
//     and even-AA stores are one 32/64-bit global store per plane (the pair is adjacent);
//   * every mbarrier wait is bounded (clock64 budget); a wait that runs out sets the context's
//     timeout flag, stops further copies, and warp 0 waits (bounded) for the copies it issued
//     before the CTA exits.
// The in-place AA step is safe with prefetching: a node's slots are read and written by that
// node only, so the copies of later tiles never see a slot that an earlier tile rewrote.
#pragma once

#include "kbc_device.cuh"
#include "kbc_ops.h"
#include "kbc_staged.cuh"

namespace kbc {

constexpr int kRowsNodes = 256;   // nodes per tile (at most)
constexpr int kRowsThreads = 128;  // threads per CTA (two nodes each)

template <typename S> struct RowsCfg;
template <> struct RowsCfg<uint16_t> { static constexpr int stages = 3; };
template <> struct RowsCfg<float> { static constexpr int stages = 2; };

template <typename S> struct RowsLayout {
  static constexpr int H = 16 / (int)sizeof(S);         // segment halo: 16 bytes
  static constexpr int PS = kRowsNodes + 2 * H;         // elements per staged plane
  static constexpr int STAGES = RowsCfg<S>::stages;
  static constexpr uint32_t stage_elems = 27u * PS;
  static constexpr size_t bar_offset = ((size_t)STAGES * stage_elems * sizeof(S) + 15) / 16 * 16;
  static constexpr size_t smem_bytes = bar_offset + 2 * STAGES * sizeof(uint64_t);
};

struct RowsArgs {
  uint32_t R;        // rows per tile
  uint32_t seg;      // nodes per tile along x (nx, or 256 in segment mode)
  uint32_t nseg;     // tiles per row (1, or nx / 256)
  uint32_t halo;     // 0 (whole rows: the x wrap is an index) or H (segments)
  uint32_t ygroups;  // ny / R
  uint32_t ntiles;   // nseg * ygroups * (ze - zb)
  unsigned long long budget;  // wait budget in SM cycles
  int stall;         // test hook: issue no copies, so every wait runs out
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Issue the copies of tile t into one stage (all lanes of warp 0 call it).
template <typename S, int MODE>
__device__ __forceinline__ void rows_issue(const S* src, const Geo& g, const RowsArgs& a,
                                           uint32_t t, S* stage, uint64_t* full) {
  using L = RowsLayout<S>;
  using Pat = Pattern<MODE>;
  constexpr uint32_t es = sizeof(S);
  const int lane = threadIdx.x & 31;
  const uint32_t sg = t % a.nseg;
  const uint32_t rest = t / a.nseg;
  const uint32_t yg = rest % a.ygroups, z = g.zb + rest / a.ygroups;
  const uint32_t y0 = yg * a.R, x0 = sg * a.seg;
  const uint32_t row_elems = a.seg + 2 * a.halo;
  if (lane == 0) mbar_arrive_expect_tx(full, 27u * a.R * row_elems * es);
  __syncwarp();
  if (lane >= 27) return;
  const int i = lane;
  const int sy = Pat::load_shift * cy(i), sz = Pat::load_shift * cz(i);
  const uint32_t zs = sz < 0 ? (z == 0 ? g.nz - 1 : z - 1)
                             : (sz > 0 ? (z + 1 == g.nz ? 0 : z + 1) : z);
  const S* plane = src + (uint64_t)Pat::load_plane(i) * g.P + (uint64_t)zs * g.nxy;
  S* dst = stage + i * L::PS;
  if (a.halo == 0) {
    // R whole rows: source rows y0 + r + sy (mod ny), r = 0 .. R-1, in at most two runs
    const uint32_t ys = sy < 0 ? (y0 == 0 ? g.ny - 1 : y0 - 1) : (y0 + sy) % g.ny;
    const uint32_t run = min(a.R, g.ny - ys);
    bulk_g2s(dst, plane + (uint64_t)ys * g.nx, run * g.nx * es, full);
    if (run < a.R) bulk_g2s(dst + run * g.nx, plane, (a.R - run) * g.nx * es, full);
  } else {
    // one segment [x0, x0 + seg) of row y0 + sy with H elements of halo on each side
    const uint32_t ys = sy < 0 ? (y0 == 0 ? g.ny - 1 : y0 - 1)
                               : (sy > 0 ? (y0 + 1 == g.ny ? 0 : y0 + 1) : y0);
    const S* row = plane + (uint64_t)ys * g.nx;
    const uint32_t H = a.halo;
    if (x0 == 0) {
      bulk_g2s(dst, row + (g.nx - H), H * es, full);
      bulk_g2s(dst + H, row, (a.seg + H) * es, full);
    } else if (x0 + a.seg == g.nx) {
      bulk_g2s(dst, row + (x0 - H), (a.seg + H) * es, full);
      bulk_g2s(dst + a.seg + H, row, H * es, full);
    } else {
      bulk_g2s(dst, row + (x0 - H), (a.seg + 2 * H) * es, full);
    }
  }
}

template <typename S, int MODE, bool RECORD>
__global__ void __launch_bounds__(kRowsThreads, 3)
    rows_step_kernel(const S* src, S* dst, Geo g, CollideParams cp, float* gamma_out,
                     StepCounters* ctr, RowsArgs a) {
  using C = Codec<S>;
  using L = RowsLayout<S>;
  using Pat = Pattern<MODE>;
  using LD = PairIO<S>;
  static_assert(std::is_same<typename C::R, float>::value, "FP32 arithmetic only");
  constexpr int ST = L::STAGES;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  S* sbuf = reinterpret_cast<S*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + L::bar_offset);
  uint64_t* empty = full + ST;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;

  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], (uint32_t)nwarps);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  // tiles of this CTA: t_k = blockIdx.x + k * gridDim.x
  const uint32_t ntile_cta =
      blockIdx.x < a.ntiles ? (a.ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  uint32_t issued = 0;  // tiles whose copies warp 0 has issued
  if (warp == 0 && !a.stall) {
    for (; issued < (uint32_t)ST && issued < ntile_cta; ++issued)
      rows_issue<S, MODE>(src, g, a, blockIdx.x + issued * gridDim.x,
                          sbuf + issued * L::stage_elems, &full[issued]);
  }

  // the thread's place in a tile: row r, node pair x = x0 + 2j, 2j + 1
  const uint32_t half_seg = a.seg >> 1;
  const uint32_t r = (uint32_t)tid / half_seg, j = (uint32_t)tid % half_seg;
  const bool active = r < a.R;
  // staged-row indices of nodes x, x - 1 and x + 2 (whole rows wrap by index)
  uint32_t i0, il, ir;
  if (a.halo == 0) {
    i0 = 2 * j;
    il = j == 0 ? a.seg - 1 : 2 * j - 1;
    ir = 2 * j + 2 == a.seg ? 0 : 2 * j + 2;
  } else {
    i0 = a.halo + 2 * j;
    il = i0 - 1;
    ir = i0 + 2;
  }
  const uint32_t rowoff = r * (a.seg + 2 * a.halo);

  uint32_t k = 0;
  for (; k < ntile_cta; ++k) {
    const uint32_t s = k % ST, ph = (k / ST) & 1u;
    if (*(volatile int*)&abort_flag) break;
    if (!mbar_wait_bounded(&full[s], ph, a.budget)) {
      atomicExch(&ctr->timeout, 1u);
      *(volatile int*)&abort_flag = 1;
      break;
    }
    const uint32_t t = blockIdx.x + k * gridDim.x;
    const uint32_t sg = t % a.nseg, rest = t / a.nseg;
    const uint32_t yg = rest % a.ygroups, z = g.zb + rest / a.ygroups;
    const uint32_t x = sg * a.seg + 2 * j, y = yg * a.R + r;
    float2 d[27];
    if (active) {
      const S* st = sbuf + s * L::stage_elems + rowoff;
      const S* v0 = st + i0;
      const S* vl = st + il;
      const S* vr = st + ir;
      Unroll<0, 27>::run([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        constexpr int SX = Pat::load_shift * cx(I);
        d[I] = LD::template get<SX, false>(v0 + I * L::PS, vl + I * L::PS, vr + I * L::PS);
      });
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    // warp 0 refills this stage with tile k + ST once every warp has read it
    if (warp == 0 && !a.stall && issued < ntile_cta && issued == k + ST) {
      bool ok = true;
      if (lane == 0) {
        ok = mbar_wait_bounded(&empty[s], ph, a.budget);
        if (ok) fence_proxy_async_smem();
      }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      if (!ok) {
        if (lane == 0) {
          atomicExch(&ctr->timeout, 1u);
          *(volatile int*)&abort_flag = 1;
        }
      } else {
        rows_issue<S, MODE>(src, g, a, blockIdx.x + issued * gridDim.x,
                            sbuf + s * L::stage_elems, &full[s]);
        ++issued;
      }
    }
    if (!active) continue;

    int guarded, fp64 = 0;
    float2 gamma = collide_step<float2, false, false, false, C::rel>(
        d, cp, &guarded, std::is_same<S, float>::value ? &fp64 : nullptr);

    // stores where f(t+1) expects them (Pattern<MODE>); flagged lanes are left to the FP64
    // pass (pull: stored anyway, the pass overwrites them from src; AA: not stored)
    const uint64_t n = (uint64_t)x + (uint64_t)g.nx * (y + (uint64_t)g.ny * z);
    const int skip = MODE == MODE_PULL ? 0 : fp64;
    if constexpr (MODE != MODE_AA_ODD) {
      S* p = dst + n;
      if (!skip) {
        Unroll<0, 27>::run([&](auto ic) {
          constexpr int I = decltype(ic)::value;
          LD::put2(p + (uint64_t)Pat::store_plane(I) * g.P, d[I]);
        });
      } else {
        Unroll<0, 27>::run([&](auto ic) {
          constexpr int I = decltype(ic)::value;
          S* q = p + (uint64_t)Pat::store_plane(I) * g.P;
          if (!(skip & 1)) LD::put1(q, d[I].x);
          if (!(skip & 2)) LD::put1(q + 1, d[I].y);
        });
      }
    } else {
      // odd AA step: f'_i of node x goes to plane i at node x + v_i
      const uint32_t xm = x == 0 ? g.nx - 1 : x - 1;
      const uint32_t xp2 = x + 2 == g.nx ? 0 : x + 2;
      const uint32_t oy[3] = {(y == 0 ? g.ny - 1 : y - 1) * g.nx, y * g.nx,
                              (y + 1 == g.ny ? 0 : y + 1) * g.nx};
      const uint32_t oz[3] = {(z == 0 ? g.nz - 1 : z - 1) * g.nxy, z * g.nxy,
                              (z + 1 == g.nz ? 0 : z + 1) * g.nxy};
      const bool wa = !(skip & 1), wb = !(skip & 2);
      Unroll<0, 27>::run([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        S* rowp = dst + (uint64_t)I * g.P + oy[cy(I) + 1] + oz[cz(I) + 1];
        if constexpr (cx(I) == 0) {
          if (!skip) {
            LD::put2(rowp + x, d[I]);
          } else {
            if (wa) LD::put1(rowp + x, d[I].x);
            if (wb) LD::put1(rowp + x + 1, d[I].y);
          }
        } else if constexpr (cx(I) > 0) {
          if (wa) LD::put1(rowp + x + 1, d[I].x);
          if (wb) LD::put1(rowp + xp2, d[I].y);
        } else {
          if (wa) LD::put1(rowp + xm, d[I].x);
          if (wb) LD::put1(rowp + x, d[I].y);
        }
      });
    }
    if (fp64) {
      if (fp64 & 1) flag_fp64(g, (uint32_t)n);
      if (fp64 & 2) flag_fp64(g, (uint32_t)n + 1);
    }
    if constexpr (RECORD) {
      *reinterpret_cast<float2*>(gamma_out + n) = gamma;
      const int cnt = __popc(guarded & 3);
      if (cnt) atomicAdd(&ctr->guarded, (unsigned long long)cnt);
    }
  }
  // warp 0 lets the copies it issued and nobody consumed land before the CTA can exit
  // (bounded; only after a wait ran out can there be any)
  if (warp == 0 && lane == 0) {
    for (uint32_t kk = k; kk < issued; ++kk)
      mbar_wait_bounded(&full[kk % ST], (kk / ST) & 1u, a.budget);
  }
}

// Tile shape for a box, or false when the kernel does not take it: rows must be whole
// multiples of 16 bytes (bulk-copy alignment) and of 2 nodes; nx <= 256 needs R rows per tile
// with R nx a multiple of 64 nodes in [128, 256] and R dividing ny; larger nx must be a
// multiple of 256.
template <typename S> inline bool rows_shape(const Geo& g, RowsArgs* a) {
  if (((uint64_t)g.nx * sizeof(S)) % 16 != 0 || g.nx % 2 != 0) return false;
  uint32_t R = 1, seg, halo;
  if (g.nx <= (uint32_t)kRowsNodes) {
    R = 0;
    for (uint32_t r = 1; r * g.nx <= (uint32_t)kRowsNodes; ++r)
      if ((r * g.nx) % 64 == 0 && r * g.nx >= 128 && g.ny % r == 0) R = r;
    if (R == 0) return false;
    seg = g.nx;
    halo = 0;
  } else {
    if (g.nx % kRowsNodes != 0) return false;
    seg = kRowsNodes;
    halo = RowsLayout<S>::H;
  }
  a->R = R;
  a->seg = seg;
  a->nseg = g.nx / seg;
  a->halo = halo;
  a->ygroups = g.ny / R;
  a->ntiles = a->nseg * a->ygroups * (g.ze - g.zb);
  return true;
}

template <typename S, int MODE, bool RECORD>
cudaError_t launch_rows(const S* src, S* dst, const Geo& g, const CollideParams& cp,
                        float* gamma_out, StepCounters* ctr, unsigned long long budget,
                        int stall, cudaStream_t st) {
  using L = RowsLayout<S>;
  static int blocks_per_sm = 0;
  static int sms = 0;
  auto kern = rows_step_kernel<S, MODE, RECORD>;
  RowsArgs a;
  if (!rows_shape<S>(g, &a)) return cudaErrorInvalidValue;
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L::smem_bytes);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, kRowsThreads,
                                                      L::smem_bytes);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
  }
  a.budget = budget;
  a.stall = stall;
  const uint32_t threads = a.R * (a.seg / 2);
  const uint32_t cap = (uint32_t)(sms * blocks_per_sm);
  const uint32_t grid = a.ntiles < cap ? a.ntiles : cap;
  kern<<<grid, threads, L::smem_bytes, st>>>(src, dst, g, cp, gamma_out, ctr, a);
  return cudaGetLastError();
}

}  // namespace kbc
