// lb_api.cu -- C ABI of the KBC library (see include/kbc_lb.h): context management, bounded
// host staging, diagnostics assembly and the batched ensemble with its CUDA graphs and
// launch-shape autotuner. The library allocates no device memory: every region below is
// carved out of the caller's buffer.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "kbc_lb.h"
#include "kbc_ops.h"

namespace {
// NVTX range over one library call (host-side span; a profiler that records NVTX shows the
// kernels it enqueued under it; without one attached the calls cost a few nanoseconds)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};
}  // namespace

namespace {

thread_local std::string g_create_error;

constexpr size_t kAlign = 256;
constexpr uint64_t kStageNodes = 1ull << 20;  // host-transfer chunk (nodes)
constexpr int32_t kMaxSpectrumBins = 6144;     // shared-memory histogram of 48 KB
constexpr int64_t kGraphSteps = 64;  // steps per captured batch graph (even: the chunks of one
                                     // call then share the parity of their first step)

// Runs f(), turning a host allocation failure into LB_ERR_OOM so that no C++ exception
// crosses the C ABI.
template <typename F> lb_status no_throw(F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    try {
      g_create_error = "host memory allocation failed";
    } catch (...) {
    }
    return LB_ERR_OOM;
  }
}

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t elem_size(int storage) { return storage == LB_F64 ? 8 : (storage == LB_F32 ? 4 : 2); }
// the FP64 re-collision mask of P nodes: one bit per node, whole 32-bit words
size_t fbmask_bytes(uint64_t P) { return (size_t)((P + 31) / 32) * 4; }
size_t arith_size(int storage) { return storage == LB_F64 ? 8 : 4; }

bool valid_config(const lb_config* c, std::string* why) {
  char buf[256];
  if (!c) {
    *why = "config is NULL";
    return false;
  }
  if (c->nx < 3 || c->ny < 3 || c->nz < 3) {
    snprintf(buf, sizeof buf, "box %d x %d x %d: every edge must be >= 3", c->nx, c->ny, c->nz);
    *why = buf;
    return false;
  }
  const uint64_t P = (uint64_t)c->nx * c->ny * c->nz;
  if (P >= (1ull << 31)) {
    *why = "nx*ny*nz must be < 2^31";
    return false;
  }
  if (!(c->nu > 0.0) || !std::isfinite(c->nu)) {
    *why = "nu must be finite and > 0";
    return false;
  }
  if (c->variant < LB_S_D || c->variant > LB_S_CDTQ) {
    *why = "variant must be LB_S_D..LB_S_DTQ or LB_S_CD..LB_S_CDTQ";
    return false;
  }
  if (c->gamma_mode < LB_GAMMA_ESTIMATE || c->gamma_mode > LB_GAMMA_EXACT) {
    *why = "gamma_mode must be LB_GAMMA_ESTIMATE, LB_GAMMA_LBGK, LB_GAMMA_RLB or LB_GAMMA_EXACT";
    return false;
  }
  if (c->storage < LB_F64 || c->storage > LB_F16) {
    *why = "storage must be LB_F64, LB_F32 or LB_F16";
    return false;
  }
  if (c->scheme != LB_PULL && c->scheme != LB_AA) {
    *why = "scheme must be LB_PULL or LB_AA";
    return false;
  }
  if (c->equilibrium != LB_EQ_PRODUCT && c->equilibrium != LB_EQ_POLY2) {
    *why = "equilibrium must be LB_EQ_PRODUCT or LB_EQ_POLY2";
    return false;
  }
  return true;
}

// per-box region: populations (1 or 2 arrays), gamma field, step counters, the mask of nodes
// flagged for the FP64 re-collision (one bit per node)
struct BoxLayout {
  size_t pop0, pop1, gamma, counters, fbmask, total;
};
BoxLayout box_layout(const lb_config* c, size_t off) {
  const uint64_t P = (uint64_t)c->nx * c->ny * c->nz;
  BoxLayout L;
  L.pop0 = off = align_up(off);
  off += 27 * P * elem_size(c->storage);
  if (c->scheme == LB_PULL) {
    L.pop1 = off = align_up(off);
    off += 27 * P * elem_size(c->storage);
  } else {
    L.pop1 = L.pop0;
  }
  L.gamma = off = align_up(off);
  off += P * sizeof(float);
  L.counters = off = align_up(off);
  off += sizeof(kbc::StepCounters);
  L.fbmask = off = align_up(off);
  off += fbmask_bytes(P);
  L.total = align_up(off);
  return L;
}

// shared work region: diagnostics velocity field, partial sums, staging
struct SharedLayout {
  size_t ufield, partials, sums, staging, total;
  uint64_t stage_nodes;
};
SharedLayout shared_layout(int storage, uint64_t maxP, size_t off) {
  SharedLayout L;
  L.ufield = off = align_up(off);
  off += 3 * maxP * arith_size(storage);
  L.partials = off = align_up(off);
  off += sizeof(double) * kbc::kDiagSums * kbc::kDiagBlocks;
  L.sums = off = align_up(off);
  off += sizeof(double) * kbc::kDiagSums;
  L.stage_nodes = maxP < kStageNodes ? maxP : kStageNodes;
  L.staging = off = align_up(off);
  off += L.stage_nodes * 27 * sizeof(double);
  L.total = align_up(off);
  return L;
}

lb_status check_device(std::string* why) {
  int dev = 0, major = 0, minor = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (e != cudaSuccess) {
    *why = std::string("no usable CUDA device: ") + cudaGetErrorString(e);
    return LB_ERR_CUDA;
  }
  if (major != 10 || minor != 3) {
    char buf[128];
    snprintf(buf, sizeof buf, "kernels are built for sm_103a only; device is sm_%d%d", major,
             minor);
    *why = buf;
    return LB_ERR_UNSUPPORTED;
  }
  return LB_OK;
}

// The device address of a host pointer into page-locked memory (cudaHostAlloc, or registered
// with cudaHostRegister), which kernels can read and write directly over the host-device link;
// NULL for pageable memory or when the platform maps no such address.
const void* mapped_host(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost) ? a.devicePointer : nullptr;
}


// ---------------------------------------------------------------- slab faces
// A face is 9 population planes (plane0 .. plane0 + 8: the velocities with v_z = -1 or +1) of
// one z-plane of a slab's local box; each is a contiguous run of nx ny values, the runs P
// values apart. face_kernel copies two faces between the population array and two contiguous
// buffers [9][nx ny] (to_buffer: pack; otherwise unpack), in units of U (16 bytes when every
// run is a multiple of 16 bytes, else 2 bytes).
struct FaceSpec {
  uint32_t plane0, z;
};

template <typename U>
__global__ void face_kernel(char* pops, uint64_t plane_bytes, uint64_t zplane_bytes,
                            FaceSpec f0, FaceSpec f1, char* buf0, char* buf1, int to_buffer) {
  const uint64_t run = zplane_bytes / sizeof(U);  // units per population plane of a face
  const uint64_t per_face = 9 * run;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < 2 * per_face;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const int which = k >= per_face;
    const uint64_t q = which ? k - per_face : k;
    const FaceSpec f = which ? f1 : f0;
    const uint64_t j = q / run, e = q - j * run;
    U* p = reinterpret_cast<U*>(pops + (f.plane0 + j) * plane_bytes + f.z * zplane_bytes) + e;
    U* b = reinterpret_cast<U*>(which ? buf1 : buf0) + q;
    if (to_buffer)
      *b = *p;
    else
      *p = *b;
  }
}

// Which faces a slab sends and receives after a step (local planes: 0 and nz + 1 are the halo
// planes, 1 .. nz the slab's own). Pull: the outgoing populations of the boundary planes of
// the buffer just written go to the neighbours' halos. AA, even step: the boundary planes'
// slots that the neighbours' odd step reads. AA, odd step: the halo slots this slab's odd step
// wrote, which belong to the neighbours' boundary planes.
struct SlabFaces {
  FaceSpec send_up, send_down, recv_below, recv_above;
};
SlabFaces slab_faces(int scase, uint32_t nz) {
  const uint32_t m = 0, p = 18;  // first plane of v_z = -1, of v_z = +1
  SlabFaces f;
  if (scase == 0) {           // pull
    f.send_up = {p, nz};
    f.send_down = {m, 1};
    f.recv_below = {p, 0};
    f.recv_above = {m, nz + 1};
  } else if (scase == 1) {    // AA, after an even step
    f.send_up = {m, nz};
    f.send_down = {p, 1};
    f.recv_below = {m, 0};
    f.recv_above = {p, nz + 1};
  } else {                    // AA, after an odd step
    f.send_up = {p, nz + 1};
    f.send_down = {m, 0};
    f.recv_below = {p, 1};
    f.recv_above = {m, nz};
  }
  return f;
}

}  // namespace

void kbc_set_thread_error(const std::string& msg) { g_create_error = msg; }

struct lb_ctx {
  lb_config cfg;
  kbc::BoxView box;
  int64_t t = 0;
  cudaStream_t stream = nullptr;
  void* ufield = nullptr;
  double* partials = nullptr;
  double* sums = nullptr;
  kbc::StepCounters* counters = nullptr;
  double* staging = nullptr;
  uint64_t stage_nodes = 0;
  int bx = 128, by = 1;
  int kernel = kbc::KERNEL_AUTO;
  int prefetch = 2;
  unsigned long long wait_budget = 2000000000ull;  // about 1 s at the SM clock
  int stall = 0;
  int diag_order = 2;
  bool gamma_valid = false;
  bool batch_view = false;
  // set when a step kernel's bounded wait ran out: the populations are not a valid state
  // until lb_set_populations, lb_init_field or lb_presolve rewrites them
  bool needs_reset = false;
  // nodes the transfer calls expose, in the context's node numbering: the whole box, or a
  // slab's own planes (between its halo planes)
  uint64_t n_first = 0, n_count = 0;
  // slab of a box split along z (lb_slab_create): its first global plane and plane count, the
  // face buffers (send up, send down, receive from below, receive from above), the exchange
  // pattern of the step whose faces were packed, and where the step stands (0 stepped and
  // unpacked, 1 faces stepped and packed, 2 stepped, faces not yet unpacked)
  bool slab = false;
  int32_t slab_z0 = 0, slab_nz = 0, slab_nz_total = 0;
  void* face[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t face_bytes = 0;
  int slab_case = 0;
  int slab_phase = 0;
  bool slab_record = false;
  std::string err;
};

namespace {

lb_status fail(lb_ctx* c, lb_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

lb_status cuda_fail(lb_ctx* c, cudaError_t e, const char* what) {
  return fail(c, LB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void default_block(lb_ctx* c) {
  int bx = 128;
  while (bx > 32 && bx / 2 >= c->cfg.nx) bx /= 2;
  c->bx = bx;
  c->by = 128 / bx;
}

void setup_ctx(lb_ctx* c, const lb_config* cfg, char* base, const BoxLayout& B,
               const SharedLayout& S, cudaStream_t st) {
  c->cfg = *cfg;
  c->box.nx = cfg->nx;
  c->box.ny = cfg->ny;
  c->box.nz = cfg->nz;
  c->box.P = (uint64_t)cfg->nx * cfg->ny * cfg->nz;
  c->box.pop[0] = base + B.pop0;
  c->box.pop[1] = base + B.pop1;
  c->box.gamma = (float*)(base + B.gamma);
  c->box.beta = 1.0 / (6.0 * cfg->nu + 1.0);  // eq:viscosity with c_s^2 = 1/3
  const int v = cfg->variant & 3;  // the central variants repeat the natural groups
  c->box.with_t = (v == LB_S_DT || v == LB_S_DTQ);
  c->box.with_q = (v == LB_S_DQ || v == LB_S_DTQ);
  c->box.central = cfg->variant >= LB_S_CD;
  c->box.poly = cfg->equilibrium == LB_EQ_POLY2;
  c->box.gamma_mode = cfg->gamma_mode;
  c->box.scheme = cfg->scheme;
  c->box.zb = 0;
  c->box.ze = (uint32_t)cfg->nz;
  c->n_first = 0;
  c->n_count = c->box.P;
  c->counters = (kbc::StepCounters*)(base + B.counters);
  c->box.fbmask = (uint32_t*)(base + B.fbmask);
  c->stream = st;
  c->ufield = base + S.ufield;
  c->partials = (double*)(base + S.partials);
  c->sums = (double*)(base + S.sums);
  c->staging = (double*)(base + S.staging);
  c->stage_nodes = S.stage_nodes;
  default_block(c);
}

// dispatch a member of Ops<S> on the context's storage type
template <typename F> cudaError_t dispatch(const lb_ctx* c, F&& f) {
  switch (c->cfg.storage) {
    case LB_F64: return f(kbc::Ops<double>{});
    case LB_F32: return f(kbc::Ops<float>{});
    default: return f(kbc::Ops<uint16_t>{});
  }
}

lb_status zero_state(lb_ctx* c) {
  const size_t bytes = 27 * c->box.P * elem_size(c->cfg.storage);
  cudaError_t e = cudaMemsetAsync(c->box.pop[0], 0, bytes, c->stream);
  if (e == cudaSuccess && c->box.pop[1] != c->box.pop[0])
    e = cudaMemsetAsync(c->box.pop[1], 0, bytes, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->counters, 0, sizeof(kbc::StepCounters), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->box.fbmask, 0, fbmask_bytes(c->box.P), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "clearing populations");
  c->t = 0;
  c->gamma_valid = false;
  return LB_OK;
}

// Synchronise the stream, then surface a bounded-wait timeout flagged by a step kernel.
lb_status sync(lb_ctx* c, const char* what) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  unsigned int flag = 0;
  e = cudaMemcpyAsync(&flag, &c->counters->timeout, sizeof flag, cudaMemcpyDeviceToHost,
                      c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  if (flag) {
    cudaMemsetAsync(&c->counters->timeout, 0, sizeof flag, c->stream);
    cudaStreamSynchronize(c->stream);
    c->needs_reset = true;
    return fail(c, LB_ERR_TIMEOUT, std::string(what) + ": a step kernel's bounded wait for its "
                                   "staged loads ran out; the state is not valid until "
                                   "lb_set_populations, lb_init_field or lb_presolve");
  }
  return LB_OK;
}

// Calls that read or advance the state refuse to run on a state left invalid by a timeout.
lb_status check_state(lb_ctx* c, const char* what) {
  if (c->slab && c->slab_phase != 0)
    return fail(c, LB_ERR_INVALID_ARG, std::string(what) + ": the slab's step is not complete "
                                       "(lb_slab_step_interior, then lb_slab_unpack)");
  if (!c->needs_reset) return LB_OK;
  return fail(c, LB_ERR_TIMEOUT, std::string(what) + ": the state is not valid after a timed-"
                                 "out step; call lb_set_populations, lb_init_field or "
                                 "lb_presolve first");
}

cudaError_t launch_faces(lb_ctx* c, char* pops, FaceSpec f0, FaceSpec f1, void* b0, void* b1,
                         int to_buffer) {
  const uint64_t es = elem_size(c->cfg.storage);
  const uint64_t zplane = (uint64_t)c->box.nx * c->box.ny * es;
  const uint64_t plane = c->box.P * es;
  const uint64_t units16 = 2 * 9 * (zplane / 16);
  if (zplane % 16 == 0) {
    const int grid = (int)std::min<uint64_t>((units16 + 255) / 256, 152ull * 8);
    face_kernel<uint4><<<grid, 256, 0, c->stream>>>(pops, plane, zplane, f0, f1, (char*)b0,
                                                    (char*)b1, to_buffer);
  } else {
    const uint64_t units2 = 2 * 9 * (zplane / 2);
    const int grid = (int)std::min<uint64_t>((units2 + 255) / 256, 152ull * 8);
    face_kernel<uint16_t><<<grid, 256, 0, c->stream>>>(pops, plane, zplane, f0, f1, (char*)b0,
                                                       (char*)b1, to_buffer);
  }
  return cudaGetLastError();
}

lb_status slab_only(lb_ctx* c, const char* what) {
  if (!c) return LB_ERR_INVALID_ARG;
  if (!c->slab) return fail(c, LB_ERR_INVALID_ARG, std::string(what) + " needs a slab context");
  return LB_OK;
}

kbc::StepOpts step_opts(const lb_ctx* c) {
  kbc::StepOpts o;
  o.bx = c->bx;
  o.by = c->by;
  o.kernel = c->kernel;
  o.prefetch = c->prefetch;
  o.budget = c->wait_budget;
  o.stall = c->stall;
  return o;
}

}  // namespace

extern "C" {

size_t lb_required_bytes(const lb_config* cfg) {
  std::string why;
  if (!valid_config(cfg, &why)) return 0;
  const BoxLayout B = box_layout(cfg, 0);
  const SharedLayout S = shared_layout(cfg->storage, (uint64_t)cfg->nx * cfg->ny * cfg->nz, B.total);
  return S.total;
}

lb_status lb_create(const lb_config* cfg, void* dev_buf, size_t bytes, void* stream,
                    lb_ctx** out) {
  return no_throw([&]() -> lb_status {
    if (!out) {
      g_create_error = "out is NULL";
      return LB_ERR_INVALID_ARG;
    }
    *out = nullptr;
    std::string why;
    if (!valid_config(cfg, &why)) {
      g_create_error = why;
      return LB_ERR_INVALID_ARG;
    }
    if (cfg->equilibrium == LB_EQ_POLY2 && cfg->gamma_mode == LB_GAMMA_EXACT) {
      g_create_error = "the exact stabilizer is built for the product-form equilibrium only";
      return LB_ERR_UNSUPPORTED;
    }
    if (!dev_buf || ((uintptr_t)dev_buf % kAlign) != 0) {
      g_create_error = "dev_buf must be a non-NULL 256-byte aligned device pointer";
      return LB_ERR_INVALID_ARG;
    }
    const size_t need = lb_required_bytes(cfg);
    if (bytes < need) {
      char buf[160];
      snprintf(buf, sizeof buf, "buffer of %zu bytes is smaller than the %zu bytes required", bytes,
               need);
      g_create_error = buf;
      return LB_ERR_OOM;
    }
    lb_status s = check_device(&why);
    if (s != LB_OK) {
      g_create_error = why;
      return s;
    }
    lb_ctx* c = new lb_ctx();
    char* base = (char*)dev_buf;
    const BoxLayout B = box_layout(cfg, 0);
    const SharedLayout S = shared_layout(cfg->storage, (uint64_t)cfg->nx * cfg->ny * cfg->nz, B.total);
    setup_ctx(c, cfg, base, B, S, (cudaStream_t)stream);
    s = zero_state(c);
    if (s != LB_OK) {
      g_create_error = c->err;
      delete c;
      return s;
    }
    *out = c;
    return LB_OK;
  });
}

lb_status lb_destroy(lb_ctx* c) {
  if (!c) return LB_ERR_INVALID_ARG;
  if (c->batch_view) return fail(c, LB_ERR_INVALID_ARG, "a batch box view is owned by its batch");
  delete c;
  return LB_OK;
}

const char* lb_last_error(const lb_ctx* c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

lb_status lb_init_field(lb_ctx* c, const double* rho, const double* u, int on_device) {
  Range range_("lb_init_field");
  if (!c) return LB_ERR_INVALID_ARG;
  if (!u) return fail(c, LB_ERR_INVALID_ARG, "u is NULL");
  c->needs_reset = false;  // the state is rewritten
  c->slab_phase = 0;
  const uint64_t P = c->n_count, nb = c->n_first;  // nodes exposed through the API
  c->t = 0;
  c->gamma_valid = false;
  cudaError_t e;
  if (on_device) {
    e = dispatch(c, [&](auto ops) { return ops.init(c->box, 0, rho, u, nb, P, P, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    return LB_OK;
  }
  const double* mu = (const double*)mapped_host(u);
  const double* mrho = (const double*)mapped_host(rho);
  if (mu && (!rho || mrho)) {  // page-locked inputs: the kernel reads them in place
    e = dispatch(c, [&](auto ops) { return ops.init(c->box, 0, mrho, mu, nb, P, P, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    return sync(c, "init");
  }
  for (uint64_t n0 = 0; n0 < P; n0 += c->stage_nodes) {
    const uint64_t cnt = (P - n0 < c->stage_nodes) ? P - n0 : c->stage_nodes;
    double* srho = c->staging;
    double* su = c->staging + cnt;
    e = cudaSuccess;
    if (rho) e = cudaMemcpyAsync(srho, rho + n0, cnt * 8, cudaMemcpyHostToDevice, c->stream);
    for (int a = 0; a < 3 && e == cudaSuccess; ++a)
      e = cudaMemcpyAsync(su + a * cnt, u + a * P + n0, cnt * 8, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "copying initial fields");
    e = dispatch(c, [&](auto ops) {
      return ops.init(c->box, 0, rho ? srho : nullptr, su, nb + n0, cnt, cnt, c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
  }
  return sync(c, "init");
}

lb_status lb_presolve(lb_ctx* c, const double* u0, int on_device, double nu_pre,
                      int64_t max_iters, double tol, int32_t from_current, int64_t* iters,
                      double* residual) {
  Range range_("lb_presolve");
  if (!c) return LB_ERR_INVALID_ARG;
  if (!u0) return fail(c, LB_ERR_INVALID_ARG, "u0 is NULL");
  if (!(nu_pre > 0.0) || !std::isfinite(nu_pre))
    return fail(c, LB_ERR_INVALID_ARG, "nu_pre must be finite and > 0");
  if (c->slab) return fail(c, LB_ERR_UNSUPPORTED, "the pre-solve runs on whole boxes");
  if (max_iters < 0) return fail(c, LB_ERR_INVALID_ARG, "max_iters must be >= 0");
  if (std::isnan(tol)) return fail(c, LB_ERR_INVALID_ARG, "tol is NaN");
  if (from_current && c->t != 0)
    return fail(c, LB_ERR_INVALID_ARG, "from_current needs the state at t = 0");
  if (from_current) {
    if (lb_status cs = check_state(c, "presolve"); cs != LB_OK) return cs;
  }
  c->needs_reset = false;  // the state is rewritten
  c->slab_phase = 0;
  const uint64_t P = c->box.P;
  const double beta_pre = 1.0 / (6.0 * nu_pre + 1.0);
  c->t = 0;
  c->gamma_valid = false;
  cudaError_t e = cudaSuccess;
  // u0 into the diagnostics velocity field (collision precision); unless continuing from the
  // current state, f = f_eq(1, u0) at t = 0
  if (!on_device && mapped_host(u0)) {  // page-locked input: read in place
    u0 = (const double*)mapped_host(u0);
    on_device = 1;
  }
  if (on_device) {
    e = dispatch(c, [&](auto ops) { return ops.convert_u(u0, c->ufield, 0, P, P, P, c->stream); });
    if (e == cudaSuccess && !from_current)
      e = dispatch(c, [&](auto ops) { return ops.init(c->box, 0, nullptr, u0, 0, P, P, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "pre-solve set-up");
  } else {
    for (uint64_t n0 = 0; n0 < P; n0 += c->stage_nodes) {
      const uint64_t cnt = (P - n0 < c->stage_nodes) ? P - n0 : c->stage_nodes;
      double* su = c->staging;
      for (int a = 0; a < 3 && e == cudaSuccess; ++a)
        e = cudaMemcpyAsync(su + a * cnt, u0 + a * P + n0, cnt * 8, cudaMemcpyHostToDevice,
                            c->stream);
      if (e == cudaSuccess)
        e = dispatch(c, [&](auto ops) {
          return ops.convert_u(su, c->ufield, n0, cnt, cnt, P, c->stream);
        });
      if (e == cudaSuccess && !from_current)
        e = dispatch(c, [&](auto ops) { return ops.init(c->box, 0, nullptr, su, n0, cnt, cnt, c->stream); });
      if (e != cudaSuccess) return cuda_fail(c, e, "pre-solve set-up");
    }
  }
  // iterations in chunks of kCheck; an even total keeps the state at an even time, where
  // both schemes store it in the layout of t = 0
  const int64_t kCheck = 32;
  const int64_t total = max_iters + (max_iters & 1);
  const kbc::StepOpts o = step_opts(c);
  int64_t done = 0;
  double res = NAN;
  unsigned int* d_res = (unsigned int*)c->sums;
  while (done < total) {
    const int64_t chunk = (total - done < kCheck) ? total - done : kCheck;
    for (int64_t j = 0; j < chunk && e == cudaSuccess; ++j) {
      const bool store = (j == chunk - 1);
      e = dispatch(c, [&](auto ops) {
        return ops.presolve_step(c->box, c->t, beta_pre, c->ufield, store, o, c->stream);
      });
      c->t += 1;
    }
    if (e == cudaSuccess)
      e = dispatch(c, [&](auto ops) {
        return ops.rho_change(c->box, c->t, d_res, kbc::kDiagBlocks, c->stream);
      });
    unsigned int bits = 0;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&bits, d_res, sizeof bits, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) {
      c->t = 0;
      return cuda_fail(c, e, "pre-solve iteration");
    }
    lb_status st = sync(c, "pre-solve");
    if (st != LB_OK) {
      c->t = 0;
      return st;
    }
    float r;
    memcpy(&r, &bits, sizeof r);
    res = (double)r;
    done += chunk;
    if (std::isinf(res)) {
      c->t = 0;
      if (iters) *iters = done;
      if (residual) *residual = res;
      return fail(c, LB_ERR_NONFINITE, "the pre-solve produced NaN/Inf populations");
    }
    if (res <= tol) break;
  }
  if (done == 0) {  // no iteration ran: the set-up kernels still read u0
    lb_status st = sync(c, "pre-solve set-up");
    if (st != LB_OK) return st;
  }
  c->t = 0;
  if (iters) *iters = done;
  if (residual) *residual = res;
  return LB_OK;
}

lb_status lb_step(lb_ctx* c, int64_t n) {
  Range range_("lb_step");
  if (!c) return LB_ERR_INVALID_ARG;
  if (n < 0) return fail(c, LB_ERR_INVALID_ARG, "n must be >= 0");
  if (c->slab)
    return fail(c, LB_ERR_INVALID_ARG, "a slab context steps with lb_slab_step_faces, "
                                       "lb_slab_step_interior and lb_slab_unpack");
  if (lb_status cs = check_state(c, "step"); cs != LB_OK) return cs;
  for (int64_t k = 0; k < n; ++k) {
    const bool record = (k == n - 1);
    cudaError_t e = cudaSuccess;
    if (record) e = cudaMemsetAsync(&c->counters->guarded, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess)
      e = dispatch(c, [&](auto ops) {
        return ops.step(c->box, c->t, record, step_opts(c), c->counters, c->stream);
      });
    if (e != cudaSuccess) return cuda_fail(c, e, "step kernel");
    c->t += 1;
  }
  if (n > 0) c->gamma_valid = true;
  return LB_OK;
}

lb_status lb_moments(lb_ctx* c, double* rho, double* u, int on_device) {
  Range range_("lb_moments");
  if (!c) return LB_ERR_INVALID_ARG;
  if (!u) return fail(c, LB_ERR_INVALID_ARG, "u is NULL");
  if (lb_status cs = check_state(c, "moments"); cs != LB_OK) return cs;
  const uint64_t P = c->n_count, nb = c->n_first;  // nodes exposed through the API
  cudaError_t e;
  if (!on_device) {  // page-locked outputs: the kernel writes them in place
    double* mu = (double*)mapped_host(u);
    double* mrho = (double*)mapped_host(rho);
    if (mu && (!rho || mrho)) {
      rho = mrho;
      u = mu;
      on_device = 1;
    }
  }
  if (on_device) {
    e = dispatch(c, [&](auto ops) { return ops.moments(c->box, c->t, rho, u, nb, P, P, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel");
    return sync(c, "moments");
  }
  for (uint64_t n0 = 0; n0 < P; n0 += c->stage_nodes) {
    const uint64_t cnt = (P - n0 < c->stage_nodes) ? P - n0 : c->stage_nodes;
    double* srho = c->staging;
    double* su = c->staging + cnt;
    e = dispatch(c, [&](auto ops) {
      return ops.moments(c->box, c->t, srho, su, nb + n0, cnt, cnt, c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel");
    if (rho) e = cudaMemcpyAsync(rho + n0, srho, cnt * 8, cudaMemcpyDeviceToHost, c->stream);
    for (int a = 0; a < 3 && e == cudaSuccess; ++a)
      e = cudaMemcpyAsync(u + a * P + n0, su + a * cnt, cnt * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "copying moments");
  }
  return sync(c, "moments");
}

lb_status lb_diagnostics(lb_ctx* c, lb_diag* out) {
  Range range_("lb_diagnostics");
  if (!c || !out) return c ? fail(c, LB_ERR_INVALID_ARG, "out is NULL") : LB_ERR_INVALID_ARG;
  if (c->slab)
    return fail(c, LB_ERR_UNSUPPORTED, "diagnostics of a slab need its neighbours' velocities; "
                                       "gather the slabs' moments instead");
  if (lb_status cs = check_state(c, "diagnostics"); cs != LB_OK) return cs;
  cudaError_t e = dispatch(c, [&](auto ops) {
    return ops.diag(c->box, c->t, c->gamma_valid, c->diag_order, c->ufield, c->partials,
                    kbc::kDiagBlocks,
                    c->sums, c->stream);
  });
  if (e != cudaSuccess) return cuda_fail(c, e, "diagnostics kernels");
  double s[kbc::kDiagSums];
  kbc::StepCounters ctr;
  e = cudaMemcpyAsync(s, c->sums, sizeof s, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&ctr, c->counters, sizeof ctr, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "copying diagnostics");
  lb_status st = sync(c, "diagnostics");
  if (st != LB_OK) return st;
  // averages over the nodes whose moments (Pf) or velocity gradients (Pg) are finite; with a
  // field free of NaN/Inf both are P
  const double P = (double)c->box.P;
  const double Pf = P - s[10], Pg = s[19];
  out->step = c->t;
  out->nodes = (int64_t)c->box.P;
  out->mass = Pf + s[0];  // finite nodes: their count plus the sum of rho - 1
  for (int a = 0; a < 3; ++a) out->momentum[a] = s[1 + a];
  out->kinetic_energy = 0.5 * s[18] / Pf;  // k = 1/2 <|u - <u>|^2>, two passes
  out->enstrophy = 0.5 * s[11] / Pg;
  out->dissipation = 0.5 * c->cfg.nu * s[12] / Pg;
  if (c->gamma_valid) {
    const double gm = s[8] / Pf;
    const double var = s[9] / Pf - gm * gm;
    out->gamma_mean = gm;
    out->gamma_std = var > 0.0 ? std::sqrt(var) : 0.0;
    out->den_guard_count = (int64_t)ctr.guarded;
  } else {
    out->gamma_mean = NAN;
    out->gamma_std = NAN;
    out->den_guard_count = 0;
  }
  out->grad_order = c->diag_order;
  out->reserved = 0;
  const double m2 = s[13] / Pg;
  out->dudx2 = m2;
  for (int m = 3; m <= 6; ++m)
    out->skewness[m - 3] = (m % 2 ? -1.0 : 1.0) * (s[13 + m - 2] / Pg) / std::pow(m2, 0.5 * m);
  out->nonfinite_count = (int64_t)s[10];
  if (out->nonfinite_count > 0) {
    char buf[96];
    snprintf(buf, sizeof buf, "%lld nodes hold NaN/Inf at step %lld",
             (long long)out->nonfinite_count, (long long)c->t);
    return fail(c, LB_ERR_NONFINITE, buf);
  }
  return LB_OK;
}

static bool spectrum_args(lb_ctx* c, int32_t nbins, lb_status* st) {
  if (c->box.nx != c->box.ny || c->box.nx != c->box.nz) {
    *st = fail(c, LB_ERR_UNSUPPORTED, "the spectrum is defined on cubic boxes only");
    return false;
  }
  if (nbins < 1 || nbins > kMaxSpectrumBins) {
    *st = fail(c, LB_ERR_INVALID_ARG, "nbins must be in 1..6144");
    return false;
  }
  return true;
}

size_t lb_spectrum_work_bytes(lb_ctx* c, int32_t nbins) {
  lb_status st;
  if (!c || !spectrum_args(c, nbins, &st)) return 0;
  return kbc::spectrum_work_bytes(c->box.nx, c->cfg.storage == LB_F64, nbins);
}

lb_status lb_spectrum(lb_ctx* c, void* work, size_t work_bytes, int32_t nbins, double* E) {
  Range range_("lb_spectrum");
  if (!c) return LB_ERR_INVALID_ARG;
  if (!work || !E) return fail(c, LB_ERR_INVALID_ARG, "work or E is NULL");
  if (c->slab) return fail(c, LB_ERR_UNSUPPORTED, "the spectrum needs the whole box");
  if (lb_status cs = check_state(c, "spectrum"); cs != LB_OK) return cs;
  lb_status st;
  if (!spectrum_args(c, nbins, &st)) return st;
  if (((uintptr_t)work % kAlign) != 0)
    return fail(c, LB_ERR_INVALID_ARG, "work must be 256-byte aligned");
  // the velocity field of the current state, as lb_diagnostics computes it
  cudaError_t e = dispatch(c, [&](auto ops) {
    return ops.diag(c->box, c->t, c->gamma_valid, c->diag_order, c->ufield, c->partials,
                    kbc::kDiagBlocks, c->sums, c->stream);
  });
  if (e != cudaSuccess) return cuda_fail(c, e, "velocity field");
  const char* why = "";
  const int r = kbc::spectrum(c->ufield, c->box.nx, c->cfg.storage == LB_F64, nbins, work,
                              work_bytes, E, c->stream, &why);
  if (r == 2) return fail(c, LB_ERR_INVALID_ARG, why);
  if (r != 0) return fail(c, LB_ERR_CUDA, std::string("spectrum: ") + why);
  return sync(c, "spectrum");
}

lb_status lb_set_diag_order(lb_ctx* c, int32_t order) {
  if (!c) return LB_ERR_INVALID_ARG;
  if (order != 2 && order != 8) return fail(c, LB_ERR_INVALID_ARG, "order must be 2 or 8");
  c->diag_order = order;
  return LB_OK;
}

lb_status lb_stabilizer_gap(lb_ctx* c, lb_gap* out) {
  Range range_("lb_stabilizer_gap");
  if (!c || !out) return c ? fail(c, LB_ERR_INVALID_ARG, "out is NULL") : LB_ERR_INVALID_ARG;
  if (c->slab) return fail(c, LB_ERR_UNSUPPORTED, "the stabilizer gap runs on whole boxes");
  if (lb_status cs = check_state(c, "stabilizer gap"); cs != LB_OK) return cs;
  if (c->box.poly)
    return fail(c, LB_ERR_UNSUPPORTED, "the stabilizer gap is built for the product-form "
                                       "equilibrium only");
  cudaError_t e = dispatch(c, [&](auto ops) {
    return ops.gamma_gap(c->box, c->t, c->partials, kbc::kDiagBlocks, c->sums, c->stream);
  });
  if (e != cudaSuccess) return cuda_fail(c, e, "stabilizer gap kernels");
  double s[7];
  e = cudaMemcpyAsync(s, c->sums, sizeof s, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "copying the stabilizer gap");
  lb_status st = sync(c, "stabilizer gap");
  if (st != LB_OK) return st;
  const double n = s[0];
  out->step = c->t;
  out->nodes = (int64_t)n;
  out->mean_abs = n > 0 ? s[1] / n : NAN;
  out->max_abs = n > 0 ? s[6] : NAN;
  out->mean_estimate = n > 0 ? s[2] / n : NAN;
  out->mean_exact = n > 0 ? s[3] / n : NAN;
  out->unconverged = (int64_t)s[4];
  out->skipped = (int64_t)s[5];
  return LB_OK;
}

lb_status lb_get_populations(lb_ctx* c, double* f, int on_device) {
  Range range_("lb_get_populations");
  if (!c) return LB_ERR_INVALID_ARG;
  if (!f) return fail(c, LB_ERR_INVALID_ARG, "f is NULL");
  if (lb_status cs = check_state(c, "get_populations"); cs != LB_OK) return cs;
  const uint64_t P = c->n_count, nb = c->n_first;  // nodes exposed through the API
  cudaError_t e;
  if (!on_device && mapped_host(f)) {  // page-locked output: written in place
    f = (double*)mapped_host(f);
    on_device = 1;
  }
  if (on_device) {
    e = dispatch(c, [&](auto ops) { return ops.get(c->box, c->t, f, nb, P, P, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "export kernel");
    return sync(c, "get_populations");
  }
  for (uint64_t n0 = 0; n0 < P; n0 += c->stage_nodes) {
    const uint64_t cnt = (P - n0 < c->stage_nodes) ? P - n0 : c->stage_nodes;
    e = dispatch(c, [&](auto ops) { return ops.get(c->box, c->t, c->staging, nb + n0, cnt, cnt, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "export kernel");
    for (int i = 0; i < 27 && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(f + i * P + n0, c->staging + i * cnt, cnt * 8, cudaMemcpyDeviceToHost,
                          c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "copying populations");
  }
  return sync(c, "get_populations");
}

lb_status lb_get_gamma(lb_ctx* c, float* gamma, int on_device) {
  Range range_("lb_get_gamma");
  if (!c) return LB_ERR_INVALID_ARG;
  if (!gamma) return fail(c, LB_ERR_INVALID_ARG, "gamma is NULL");
  if (lb_status cs = check_state(c, "get_gamma"); cs != LB_OK) return cs;
  if (!c->gamma_valid)
    return fail(c, LB_ERR_INVALID_ARG, "no collision has been recorded since the state was set");
  cudaError_t e = cudaMemcpyAsync(gamma, c->box.gamma + c->n_first, c->n_count * sizeof(float),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "copying the gamma field");
  return sync(c, "get_gamma");
}

lb_status lb_set_populations(lb_ctx* c, const double* f, int on_device) {
  Range range_("lb_set_populations");
  if (!c) return LB_ERR_INVALID_ARG;
  if (!f) return fail(c, LB_ERR_INVALID_ARG, "f is NULL");
  c->needs_reset = false;  // the state is rewritten
  c->slab_phase = 0;
  const uint64_t P = c->n_count, nb = c->n_first;  // nodes exposed through the API
  c->gamma_valid = false;
  cudaError_t e;
  if (!on_device && mapped_host(f)) {  // page-locked input: read in place
    f = (const double*)mapped_host(f);
    on_device = 1;
  }
  if (on_device) {
    e = dispatch(c, [&](auto ops) { return ops.set(c->box, c->t, f, nb, P, P, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "import kernel");
    return sync(c, "set_populations");
  }
  for (uint64_t n0 = 0; n0 < P; n0 += c->stage_nodes) {
    const uint64_t cnt = (P - n0 < c->stage_nodes) ? P - n0 : c->stage_nodes;
    e = cudaSuccess;
    for (int i = 0; i < 27 && e == cudaSuccess; ++i)
      e = cudaMemcpyAsync(c->staging + i * cnt, f + i * P + n0, cnt * 8, cudaMemcpyHostToDevice,
                          c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "copying populations");
    e = dispatch(c, [&](auto ops) { return ops.set(c->box, c->t, c->staging, nb + n0, cnt, cnt, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "import kernel");
  }
  return sync(c, "set_populations");
}

int64_t lb_time(const lb_ctx* c) { return c ? c->t : -1; }
double lb_beta(const lb_ctx* c) { return c ? c->box.beta : NAN; }

lb_status lb_set_time(lb_ctx* c, int64_t t) {
  if (!c) return LB_ERR_INVALID_ARG;
  if (t < 0) return fail(c, LB_ERR_INVALID_ARG, "t must be >= 0");
  c->t = t;
  c->gamma_valid = false;
  return LB_OK;
}

lb_status lb_set_kernel(lb_ctx* c, int32_t kind) {
  if (!c) return LB_ERR_INVALID_ARG;
  if (kind < LB_KERNEL_AUTO || kind > LB_KERNEL_ADJ)
    return fail(c, LB_ERR_INVALID_ARG, "kind must be LB_KERNEL_AUTO, _DIRECT, _STAGED, "
                                       "_PERSISTENT, _PACKED, _ROWS or _ADJ");
  if (kind == LB_KERNEL_ADJ) {
    if (c->cfg.storage == LB_F64)
      return fail(c, LB_ERR_UNSUPPORTED, "the adjacent-pair kernel needs FP32 arithmetic "
                                         "(LB_F32 or LB_F16 storage)");
    if (c->box.poly || c->box.central)
      return fail(c, LB_ERR_UNSUPPORTED, "the adjacent-pair kernel implements the product-form "
                                         "equilibrium and the natural-moment variants only");
    if (c->box.nx % 2 != 0)
      return fail(c, LB_ERR_UNSUPPORTED, "the adjacent-pair kernel needs an even nx");
  }
  if (kind == LB_KERNEL_ROWS) {
    if (c->cfg.storage == LB_F64)
      return fail(c, LB_ERR_UNSUPPORTED, "the rows kernel needs FP32 arithmetic (LB_F32 or "
                                         "LB_F16 storage)");
    if (c->box.poly || c->box.central)
      return fail(c, LB_ERR_UNSUPPORTED, "the rows kernel implements the product-form "
                                         "equilibrium and the natural-moment variants only");
    bool ok = false;
    dispatch(c, [&](auto ops) {
      ok = ops.rows_ok(c->box.nx, c->box.ny, c->box.nz);
      return cudaSuccess;
    });
    if (!ok)
      return fail(c, LB_ERR_UNSUPPORTED, "the rows kernel does not take this box shape (nx even, "
                                         "nx * sizeof(value) % 16 == 0, nx <= 256 with a tile of "
                                         "R rows, R | ny, R * nx a multiple of 64 in [128, 256], "
                                         "or nx a multiple of 256)");
  }
  if ((kind == LB_KERNEL_STAGED || kind == LB_KERNEL_PERSISTENT) && c->box.poly)
    return fail(c, LB_ERR_UNSUPPORTED, "the staged and persistent kernels implement the "
                                       "product-form equilibrium only");
  if ((kind == LB_KERNEL_STAGED || kind == LB_KERNEL_PERSISTENT) && c->box.central)
    return fail(c, LB_ERR_UNSUPPORTED, "the staged and persistent kernels implement the natural-"
                                       "moment variants only");
  if (c->cfg.gamma_mode == LB_GAMMA_EXACT && kind != LB_KERNEL_AUTO && kind != LB_KERNEL_DIRECT)
    return fail(c, LB_ERR_UNSUPPORTED, "the exact stabilizer runs in the direct kernel only");
  if (kind == LB_KERNEL_PACKED && c->cfg.storage == LB_F64)
    return fail(c, LB_ERR_UNSUPPORTED, "the packed FP32x2 kernel needs FP32 arithmetic "
                                       "(LB_F32 or LB_F16 storage)");
  if (kind == LB_KERNEL_STAGED) {
    bool ok = false;
    dispatch(c, [&](auto ops) {
      ok = ops.staged_ok(c->box.nx);
      return cudaSuccess;
    });
    if (!ok)
      return fail(c, LB_ERR_UNSUPPORTED, "the staged kernel needs nx * sizeof(value) to be a "
                                         "multiple of 16 bytes");
  }
  c->kernel = kind;
  return LB_OK;
}

lb_status lb_set_prefetch(lb_ctx* c, int32_t items_ahead) {
  if (!c) return LB_ERR_INVALID_ARG;
  if (items_ahead < 0 || items_ahead > 8)
    return fail(c, LB_ERR_INVALID_ARG, "items_ahead must be in [0, 8]");
  c->prefetch = items_ahead;
  return LB_OK;
}

lb_status lb_set_wait_budget(lb_ctx* c, uint64_t cycles, int32_t stall_copies) {
  if (!c) return LB_ERR_INVALID_ARG;
  if (cycles == 0) return fail(c, LB_ERR_INVALID_ARG, "cycles must be > 0");
  c->wait_budget = cycles;
  c->stall = stall_copies ? 1 : 0;
  return LB_OK;
}

lb_status lb_set_block(lb_ctx* c, int32_t bx, int32_t by) {
  if (!c) return LB_ERR_INVALID_ARG;
  if (bx < 32 || bx > 512 || bx % 32 != 0 || by < 1 || by > 16)
    return fail(c, LB_ERR_INVALID_ARG, "block must be bx*by in {64,128,256,512}, bx % 32 == 0");
  const int n = bx * by;
  if (n != 64 && n != 128 && n != 256 && n != 512)
    return fail(c, LB_ERR_INVALID_ARG, "block must be bx*by in {64,128,256,512}, bx % 32 == 0");
  if (c->cfg.storage == LB_F64 && n > 256)
    return fail(c, LB_ERR_INVALID_ARG, "FP64 storage allows at most 256 threads per block");
  c->bx = bx;
  c->by = by;
  return LB_OK;
}


// ---------------------------------------------------------------- slabs of a box split along z

size_t lb_slab_required_bytes(const lb_config* global, int32_t nz_local) {
  std::string why;
  if (!valid_config(global, &why) || nz_local < 1 || nz_local > global->nz) return 0;
  lb_config lc = *global;
  lc.nz = nz_local + 2;
  if (!valid_config(&lc, &why)) return 0;
  const BoxLayout B = box_layout(&lc, 0);
  const SharedLayout S = shared_layout(lc.storage, (uint64_t)lc.nx * lc.ny * lc.nz, B.total);
  const size_t fb = align_up((size_t)9 * lc.nx * lc.ny * elem_size(lc.storage));
  return S.total + 4 * fb;
}

lb_status lb_slab_create(const lb_config* global, int32_t z0, int32_t nz_local, void* dev_buf,
                         size_t bytes, void* stream, lb_ctx** out) {
  return no_throw([&]() -> lb_status {
    if (!out) {
      g_create_error = "out is NULL";
      return LB_ERR_INVALID_ARG;
    }
    *out = nullptr;
    std::string why;
    if (!valid_config(global, &why)) {
      g_create_error = why;
      return LB_ERR_INVALID_ARG;
    }
    if (nz_local < 1 || z0 < 0 || z0 >= global->nz || nz_local > global->nz - z0) {
      g_create_error = "need 0 <= z0 and 1 <= nz_local with z0 + nz_local <= nz";
      return LB_ERR_INVALID_ARG;
    }
    if (global->equilibrium == LB_EQ_POLY2 && global->gamma_mode == LB_GAMMA_EXACT) {
      g_create_error = "the exact stabilizer is built for the product-form equilibrium only";
      return LB_ERR_UNSUPPORTED;
    }
    lb_config lc = *global;
    lc.nz = nz_local + 2;
    if (!valid_config(&lc, &why)) {
      g_create_error = "slab: " + why;
      return LB_ERR_INVALID_ARG;
    }
    if (!dev_buf || ((uintptr_t)dev_buf % kAlign) != 0) {
      g_create_error = "dev_buf must be a non-NULL 256-byte aligned device pointer";
      return LB_ERR_INVALID_ARG;
    }
    const size_t need = lb_slab_required_bytes(global, nz_local);
    if (bytes < need) {
      char buf[160];
      snprintf(buf, sizeof buf, "buffer of %zu bytes is smaller than the %zu bytes required",
               bytes, need);
      g_create_error = buf;
      return LB_ERR_OOM;
    }
    lb_status s = check_device(&why);
    if (s != LB_OK) {
      g_create_error = why;
      return s;
    }
    lb_ctx* c = new lb_ctx();
    char* base = (char*)dev_buf;
    const BoxLayout B = box_layout(&lc, 0);
    const SharedLayout S = shared_layout(lc.storage, (uint64_t)lc.nx * lc.ny * lc.nz, B.total);
    setup_ctx(c, &lc, base, B, S, (cudaStream_t)stream);
    c->slab = true;
    c->slab_z0 = z0;
    c->slab_nz = nz_local;
    c->slab_nz_total = global->nz;
    const uint64_t nxy = (uint64_t)lc.nx * lc.ny;
    c->n_first = nxy;
    c->n_count = nxy * (uint64_t)nz_local;
    c->box.zb = 1;
    c->box.ze = (uint32_t)nz_local + 1;
    c->face_bytes = (size_t)9 * nxy * elem_size(lc.storage);
    const size_t fb = align_up(c->face_bytes);
    for (int k = 0; k < 4; ++k) c->face[k] = base + S.total + k * fb;
    s = zero_state(c);
    if (s != LB_OK) {
      g_create_error = c->err;
      delete c;
      return s;
    }
    *out = c;
    return LB_OK;
  });
}

lb_status lb_slab_faces(lb_ctx* c, void** send_up, void** send_down, void** recv_below,
                        void** recv_above, size_t* face_bytes) {
  if (lb_status s = slab_only(c, "lb_slab_faces"); s != LB_OK) return s;
  if (send_up) *send_up = c->face[0];
  if (send_down) *send_down = c->face[1];
  if (recv_below) *recv_below = c->face[2];
  if (recv_above) *recv_above = c->face[3];
  if (face_bytes) *face_bytes = c->face_bytes;
  return LB_OK;
}

lb_status lb_slab_step_faces(lb_ctx* c, int32_t record) {
  Range range_("lb_slab_step_faces");
  if (lb_status s = slab_only(c, "lb_slab_step_faces"); s != LB_OK) return s;
  if (lb_status cs = check_state(c, "slab step"); cs != LB_OK) return cs;
  if (c->slab_phase != 0)
    return fail(c, LB_ERR_INVALID_ARG, "the previous step's faces are not unpacked yet "
                                       "(lb_slab_step_interior, then lb_slab_unpack)");
  cudaError_t e = cudaSuccess;
  if (record)
    e = cudaMemsetAsync(&c->counters->guarded, 0, sizeof(unsigned long long), c->stream);
  const uint32_t nz = (uint32_t)c->slab_nz;
  // the boundary planes (local 1 and nz) first, so that their faces can travel while the
  // interior planes are stepped
  for (int k = 0; k < (nz > 1 ? 2 : 1) && e == cudaSuccess; ++k) {
    const uint32_t z = k == 0 ? 1 : nz;
    c->box.zb = z;
    c->box.ze = z + 1;
    e = dispatch(c, [&](auto ops) {
      return ops.step(c->box, c->t, record != 0, step_opts(c), c->counters, c->stream);
    });
  }
  c->box.zb = 1;
  c->box.ze = nz + 1;
  if (e != cudaSuccess) return cuda_fail(c, e, "slab boundary step");
  const int scase = c->cfg.scheme == LB_PULL ? 0 : ((c->t & 1) == 0 ? 1 : 2);
  char* pops = (char*)c->box.pop[c->cfg.scheme == LB_PULL ? ((c->t + 1) & 1) : 0];
  const SlabFaces f = slab_faces(scase, nz);
  e = launch_faces(c, pops, f.send_up, f.send_down, c->face[0], c->face[1], 1);
  if (e != cudaSuccess) return cuda_fail(c, e, "packing slab faces");
  c->slab_case = scase;
  c->slab_phase = 1;
  c->slab_record = record != 0;
  return LB_OK;
}

lb_status lb_slab_step_interior(lb_ctx* c) {
  Range range_("lb_slab_step_interior");
  if (lb_status s = slab_only(c, "lb_slab_step_interior"); s != LB_OK) return s;
  if (c->slab_phase != 1)
    return fail(c, LB_ERR_INVALID_ARG, "call lb_slab_step_faces first");
  const uint32_t nz = (uint32_t)c->slab_nz;
  cudaError_t e = cudaSuccess;
  if (nz > 2) {
    c->box.zb = 2;
    c->box.ze = nz;
    e = dispatch(c, [&](auto ops) {
      return ops.step(c->box, c->t, c->slab_record, step_opts(c), c->counters, c->stream);
    });
    c->box.zb = 1;
    c->box.ze = nz + 1;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "slab interior step");
  c->t += 1;
  c->gamma_valid = c->slab_record;
  c->slab_phase = 2;
  return LB_OK;
}

lb_status lb_slab_unpack(lb_ctx* c) {
  Range range_("lb_slab_unpack");
  if (lb_status s = slab_only(c, "lb_slab_unpack"); s != LB_OK) return s;
  if (c->slab_phase != 2)
    return fail(c, LB_ERR_INVALID_ARG, "call lb_slab_step_faces and lb_slab_step_interior first");
  char* pops = (char*)c->box.pop[c->cfg.scheme == LB_PULL ? (c->t & 1) : 0];
  const SlabFaces f = slab_faces(c->slab_case, (uint32_t)c->slab_nz);
  cudaError_t e = launch_faces(c, pops, f.recv_below, f.recv_above, c->face[2], c->face[3], 0);
  if (e != cudaSuccess) return cuda_fail(c, e, "unpacking slab faces");
  c->slab_phase = 0;
  return LB_OK;
}

}  // extern "C"

// ====================================================================== batched ensemble

struct lb_batch {
  int nbox = 0;
  lb_config base_cfg;
  std::vector<lb_ctx*> views;
  std::vector<lb_config> cfgs;
  kbc::BoxDesc* d_boxes = nullptr;
  kbc::WorkItem* d_items = nullptr;
  kbc::BatchFlags* d_flags = nullptr;  // the batch-wide flag of the FP64 re-collision pass
  size_t max_items = 0;
  int nitems = 0;
  int threads = 256;
  int tile = 512;  // target nodes per work item
  // 0 one node per thread; FP32 arithmetic only: 1 FP32x2 pairs (n, n + 32), 2 FP32x2 adjacent
  // pairs (x, x + 1) (every box with an even nx, natural moments)
  int packed = 0;
  int grid = 1;
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  std::map<std::pair<int64_t, int>, cudaGraphExec_t> graphs;
  int64_t t = 0;
  std::string err;
};

namespace {

lb_status bfail(lb_batch* b, lb_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}

// The batch kernel a kernel request selects: 0 one node per thread (FP64 arithmetic, or
// LB_KERNEL_DIRECT), 1 the FP32x2 (n, n + 32) pairs, 2 the FP32x2 adjacent pairs, which AUTO
// takes whenever every box has an even nx and the moments are natural (as for one box).
int batch_kind(const lb_config* cfgs, int nbox, int32_t kind) {
  if (cfgs[0].storage == LB_F64 || kind == LB_KERNEL_DIRECT) return 0;
  if (kind == LB_KERNEL_PACKED) return 1;
  bool even = cfgs[0].variant < LB_S_CD;
  for (int k = 0; k < nbox && even; ++k) even = cfgs[k].nx % 2 == 0;
  return even ? 2 : 1;
}

struct BatchLayout {
  size_t boxes, items, flags, shared_off, total;
  size_t max_items;
  std::vector<BoxLayout> box;
  SharedLayout shared;
};

bool batch_layout(const lb_config* cfgs, int32_t nbox, BatchLayout* L, std::string* why) {
  if (!cfgs || nbox < 1) {
    *why = "need at least one box";
    return false;
  }
  uint64_t maxP = 0;
  size_t rows = 0;
  for (int b = 0; b < nbox; ++b) {
    lb_config c = cfgs[b];
    c.variant = cfgs[0].variant;
    c.gamma_mode = cfgs[0].gamma_mode;
    c.storage = cfgs[0].storage;
    c.scheme = cfgs[0].scheme;
    c.equilibrium = cfgs[0].equilibrium;
    if (!valid_config(&c, why)) {
      *why = "box " + std::to_string(b) + ": " + *why;
      return false;
    }
    const uint64_t P = (uint64_t)c.nx * c.ny * c.nz;
    if (P > maxP) maxP = P;
    rows += (size_t)c.ny * c.nz;
  }
  size_t off = 0;
  L->boxes = off;
  off = align_up(off + sizeof(kbc::BoxDesc) * nbox);
  L->items = off;
  L->max_items = rows;
  off = align_up(off + sizeof(kbc::WorkItem) * rows);
  L->flags = off;
  off = align_up(off + sizeof(kbc::BatchFlags));
  L->box.clear();
  for (int b = 0; b < nbox; ++b) {
    lb_config c = cfgs[b];
    c.storage = cfgs[0].storage;
    c.scheme = cfgs[0].scheme;
    c.equilibrium = cfgs[0].equilibrium;
    BoxLayout B = box_layout(&c, off);
    L->box.push_back(B);
    off = B.total;
  }
  L->shared = shared_layout(cfgs[0].storage, maxP, off);
  L->total = L->shared.total;
  return true;
}

void clear_graphs(lb_batch* b) {
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// rebuild the work list for the current tile and upload it
lb_status build_items(lb_batch* b) {
  std::vector<kbc::WorkItem> items;
  items.reserve(b->max_items);
  for (int k = 0; k < b->nbox; ++k) {
    const lb_config& c = b->cfgs[k];
    int rows_per = b->tile / c.nx;
    if (rows_per < 1) rows_per = 1;
    const int rows = c.ny * c.nz;
    for (int r = 0; r < rows; r += rows_per) {
      kbc::WorkItem w;
      w.box = k;
      w.row0 = r;
      w.nrows = (rows - r < rows_per) ? rows - r : rows_per;
      w.pad = 0;
      items.push_back(w);
    }
  }
  b->nitems = (int)items.size();
  cudaError_t e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(kbc::WorkItem) * items.size(),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string("uploading work list: ") + cudaGetErrorString(e));
  int occ = 1;
  switch (b->base_cfg.storage) {
    case LB_F64:
      occ = kbc::Ops<double>::batch_occupancy(b->threads, b->base_cfg.scheme, false);
      break;
    case LB_F32:
      occ = kbc::Ops<float>::batch_occupancy(b->threads, b->base_cfg.scheme, b->packed);
      break;
    default:
      occ = kbc::Ops<uint16_t>::batch_occupancy(b->threads, b->base_cfg.scheme, b->packed);
      break;
  }
  const int cap = num_sms() * occ;
  b->grid = b->nitems < cap ? b->nitems : cap;
  clear_graphs(b);
  return LB_OK;
}

cudaError_t enqueue_batch_step(lb_batch* b, int64_t t, bool record, cudaStream_t st) {
  const lb_config& c = b->base_cfg;
  const int v = c.variant & 3;
  const int wt = (v == LB_S_DT || v == LB_S_DTQ);
  const int wq = (v == LB_S_DQ || v == LB_S_DTQ);
  const int central = c.variant >= LB_S_CD;
  switch (c.storage) {
    case LB_F64:
      return kbc::Ops<double>::batch_step(b->d_boxes, b->nbox, b->d_flags, b->d_items,
                                          b->nitems, t, record, 0,
                                          c.scheme, wt, wq, central, c.gamma_mode, b->threads,
                                          b->grid, st);
    case LB_F32:
      return kbc::Ops<float>::batch_step(b->d_boxes, b->nbox, b->d_flags, b->d_items,
                                         b->nitems, t, record,
                                         b->packed, c.scheme, wt, wq, central, c.gamma_mode,
                                         b->threads, b->grid, st);
    default:
      return kbc::Ops<uint16_t>::batch_step(b->d_boxes, b->nbox, b->d_flags, b->d_items,
                                            b->nitems, t, record,
                                            b->packed, c.scheme, wt, wq, central, c.gamma_mode,
                                            b->threads, b->grid, st);
  }
}

// The instantiated graph of `len` batch steps from the batch's current time (only its parity
// matters to the kernels); `record` makes the last of them record gamma and the guard count.
// Captured on first use and cached.
lb_status batch_graph(lb_batch* b, int64_t len, bool record, cudaGraphExec_t* out) {
  const auto key = std::make_pair(len, (int)(b->t & 1) | (record ? 2 : 0));
  auto it = b->graphs.find(key);
  if (it != b->graphs.end()) {
    *out = it->second;
    return LB_OK;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess)
    return bfail(b, LB_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
  cudaError_t le = cudaSuccess;
  for (int64_t k = 0; k < len; ++k) {
    const bool rec = record && (k == len - 1);
    if (rec) {
      for (lb_ctx* v : b->views)
        if (le == cudaSuccess)
          le = cudaMemsetAsync(&v->counters->guarded, 0, sizeof(unsigned long long),
                               b->capture_stream);
    }
    if (le == cudaSuccess) le = enqueue_batch_step(b, b->t + k, rec, b->capture_stream);
  }
  e = cudaStreamEndCapture(b->capture_stream, &graph);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return bfail(b, LB_ERR_CUDA, std::string("capturing batch steps: ") +
                                     cudaGetErrorString(le != cudaSuccess ? le : e));
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess)
    return bfail(b, LB_ERR_CUDA, std::string("instantiating graph: ") + cudaGetErrorString(e));
  try {
    b->graphs.emplace(key, exec);
  } catch (...) {
    cudaGraphExecDestroy(exec);
    throw;
  }
  *out = exec;
  return LB_OK;
}

}  // namespace

extern "C" {

size_t lb_batch_required_bytes(const lb_config* cfgs, int32_t nbox) {
  BatchLayout L;
  std::string why;
  if (!batch_layout(cfgs, nbox, &L, &why)) return 0;
  return L.total;
}

lb_status lb_batch_create(const lb_config* cfgs, int32_t nbox, void* dev_buf, size_t bytes,
                          void* stream, lb_batch** out) {
  return no_throw([&]() -> lb_status {
    if (!out) {
      g_create_error = "out is NULL";
      return LB_ERR_INVALID_ARG;
    }
    *out = nullptr;
    BatchLayout L;
    std::string why;
    if (!batch_layout(cfgs, nbox, &L, &why)) {
      g_create_error = why;
      return LB_ERR_INVALID_ARG;
    }
    if (cfgs[0].gamma_mode == LB_GAMMA_EXACT) {
      g_create_error = "the batch kernels do not implement the exact stabilizer";
      return LB_ERR_UNSUPPORTED;
    }
    if (cfgs[0].equilibrium == LB_EQ_POLY2) {
      g_create_error = "the batch kernels implement the product-form equilibrium only";
      return LB_ERR_UNSUPPORTED;
    }
    if (!dev_buf || ((uintptr_t)dev_buf % kAlign) != 0) {
      g_create_error = "dev_buf must be a non-NULL 256-byte aligned device pointer";
      return LB_ERR_INVALID_ARG;
    }
    if (bytes < L.total) {
      char buf[160];
      snprintf(buf, sizeof buf, "buffer of %zu bytes is smaller than the %zu bytes required", bytes,
               L.total);
      g_create_error = buf;
      return LB_ERR_OOM;
    }
    lb_status s = check_device(&why);
    if (s != LB_OK) {
      g_create_error = why;
      return s;
    }
    // owned by `guard` until the batch is complete: every early return (and a host allocation
    // failure below) releases what was built so far
    std::unique_ptr<lb_batch, lb_status (*)(lb_batch*)> guard(new lb_batch(), lb_batch_destroy);
    lb_batch* b = guard.get();
    char* base = (char*)dev_buf;
    b->nbox = nbox;
    b->base_cfg = cfgs[0];
    b->stream = (cudaStream_t)stream;
    b->d_boxes = (kbc::BoxDesc*)(base + L.boxes);
    b->d_items = (kbc::WorkItem*)(base + L.items);
    b->d_flags = (kbc::BatchFlags*)(base + L.flags);
    b->max_items = L.max_items;
    b->packed = batch_kind(cfgs, nbox, LB_KERNEL_AUTO);
    if (b->packed) b->threads = 128;
    cudaError_t e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      g_create_error = std::string("creating capture stream: ") + cudaGetErrorString(e);
      return LB_ERR_CUDA;
    }
    std::vector<kbc::BoxDesc> descs(nbox);
    b->cfgs.reserve(nbox);
    b->views.reserve(nbox);
    for (int k = 0; k < nbox; ++k) {
      lb_config c = cfgs[k];
      c.variant = cfgs[0].variant;
      c.gamma_mode = cfgs[0].gamma_mode;
      c.storage = cfgs[0].storage;
      c.scheme = cfgs[0].scheme;
      c.equilibrium = cfgs[0].equilibrium;
      b->cfgs.push_back(c);
      b->views.push_back(new lb_ctx());
      lb_ctx* v = b->views.back();
      setup_ctx(v, &c, base, L.box[k], L.shared, b->stream);
      v->batch_view = true;
      s = zero_state(v);
      if (s != LB_OK) {
        g_create_error = "initialising box " + std::to_string(k) + ": " + v->err;
        return s;
      }
      kbc::BoxDesc& d = descs[k];
      d.nx = c.nx;
      d.ny = c.ny;
      d.nz = c.nz;
      d.nxy = (uint32_t)c.nx * c.ny;
      d.pop[0] = v->box.pop[0];
      d.pop[1] = v->box.pop[1];
      d.gamma = v->box.gamma;
      d.fbmask = v->box.fbmask;
      d.ctr = v->counters;
      d.beta = v->box.beta;
      d.two_beta = 2.0 * v->box.beta;
      d.inv_beta = 1.0 / v->box.beta;
    }
    e = cudaMemcpyAsync(b->d_boxes, descs.data(), sizeof(kbc::BoxDesc) * nbox,
                        cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_flags, 0, sizeof(kbc::BatchFlags), b->stream);
    if (e != cudaSuccess) {
      g_create_error = "uploading box descriptors: " + std::string(cudaGetErrorString(e));
      return LB_ERR_CUDA;
    }
    s = build_items(b);
    if (s != LB_OK) {
      g_create_error = b->err;
      return s;
    }
    guard.release();
    *out = b;
    return LB_OK;
  });
}

lb_status lb_batch_destroy(lb_batch* b) {
  if (!b) return LB_ERR_INVALID_ARG;
  clear_graphs(b);
  for (lb_ctx* v : b->views) delete v;
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  delete b;
  return LB_OK;
}

const char* lb_batch_last_error(const lb_batch* b) {
  return b ? b->err.c_str() : g_create_error.c_str();
}

lb_ctx* lb_batch_box(lb_batch* b, int32_t box) {
  if (!b || box < 0 || box >= b->nbox) return nullptr;
  return b->views[box];
}

lb_status lb_batch_step(lb_batch* b, int64_t n) {
  return no_throw([&]() -> lb_status {
    Range range_("lb_batch_step");
    if (!b) return LB_ERR_INVALID_ARG;
    if (n < 0) return bfail(b, LB_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return LB_OK;
    // all boxes must share one time (initialising a box resets its t to 0)
    for (lb_ctx* v : b->views)
      if (v->t != b->views[0]->t)
        return bfail(b, LB_ERR_INVALID_ARG, "boxes of a batch are at different times; step, "
                                            "initialise or re-time all of them together");
    b->t = b->views[0]->t;
    // replay graphs of at most kGraphSteps steps, so that the cache stays bounded (one graph of
    // kGraphSteps steps and one tail per length, per parity) whatever n the caller passes
    lb_status st = LB_OK;
    for (int64_t done = 0; done < n && st == LB_OK;) {
      const int64_t len = (n - done > kGraphSteps) ? kGraphSteps : n - done;
      const bool record = (done + len == n);
      cudaGraphExec_t exec = nullptr;
      st = batch_graph(b, len, record, &exec);
      if (st != LB_OK) break;
      cudaError_t e = cudaGraphLaunch(exec, b->stream);
      if (e != cudaSuccess) {
        st = bfail(b, LB_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
        break;
      }
      b->t += len;
      done += len;
    }
    for (lb_ctx* v : b->views) {
      v->t = b->t;
      v->gamma_valid = (st == LB_OK);
    }
    return st;
  });
}

lb_status lb_batch_diagnostics(lb_batch* b, lb_diag* out) {
  return no_throw([&]() -> lb_status {
    if (!b || !out) return b ? bfail(b, LB_ERR_INVALID_ARG, "out is NULL") : LB_ERR_INVALID_ARG;
    lb_status worst = LB_OK;
    for (int k = 0; k < b->nbox; ++k) {
      lb_status s = lb_diagnostics(b->views[k], &out[k]);
      if (s == LB_ERR_NONFINITE) {
        worst = s;
        b->err = "box " + std::to_string(k) + ": " + b->views[k]->err;
      } else if (s != LB_OK) {
        b->err = "box " + std::to_string(k) + ": " + b->views[k]->err;
        return s;
      }
    }
    return worst;
  });
}

lb_status lb_batch_set_kernel(lb_batch* b, int32_t kind) {
  return no_throw([&]() -> lb_status {
    if (!b) return LB_ERR_INVALID_ARG;
    if (kind != LB_KERNEL_AUTO && kind != LB_KERNEL_DIRECT && kind != LB_KERNEL_PACKED &&
        kind != LB_KERNEL_ADJ)
      return bfail(b, LB_ERR_INVALID_ARG,
                   "batch kernel must be LB_KERNEL_AUTO, _DIRECT, _PACKED or _ADJ");
    const bool fp32 = b->base_cfg.storage != LB_F64;
    if ((kind == LB_KERNEL_PACKED || kind == LB_KERNEL_ADJ) && !fp32)
      return bfail(b, LB_ERR_UNSUPPORTED, "the packed kernels need FP32 arithmetic");
    const int k = batch_kind(b->cfgs.data(), b->nbox, kind);
    if (kind == LB_KERNEL_ADJ && k != 2)
      return bfail(b, LB_ERR_UNSUPPORTED,
                   "the adjacent-pair kernel needs an even nx in every box and natural moments");
    b->packed = k;
    b->threads = b->packed ? 128 : 256;
    return build_items(b);
  });
}

lb_status lb_batch_set_tile(lb_batch* b, int32_t threads, int32_t tile) {
  return no_throw([&]() -> lb_status {
    if (!b) return LB_ERR_INVALID_ARG;
    const int maxt = b->base_cfg.storage == LB_F64 ? 256 : 512;
    if (b->packed && threads != 128)
      return bfail(b, LB_ERR_INVALID_ARG, "the packed batch kernel runs 128 threads per block");
    if (threads < 32 || threads > maxt || threads % 32 != 0 || tile < 32)
      return bfail(b, LB_ERR_INVALID_ARG, "threads must be a multiple of 32 in [32, 512] (256 for "
                                          "FP64); tile >= 32");
    b->threads = threads;
    b->tile = tile;
    return build_items(b);
  });
}

lb_status lb_batch_autotune(lb_batch* b, int32_t trial_steps, int32_t* best_threads,
                            int32_t* best_tile, double* best_ms) {
  return no_throw([&]() -> lb_status {
    if (!b) return LB_ERR_INVALID_ARG;
    if (trial_steps < 1) return bfail(b, LB_ERR_INVALID_ARG, "trial_steps must be >= 1");
    const int cand_threads[] = {128, 256, 512};
    const int maxt = b->base_cfg.storage == LB_F64 ? 256 : 512;
    const int cand_tile[] = {256, 512, 1024, 2048, 4096};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
      return bfail(b, LB_ERR_CUDA, "creating timing events");
    double best = 1e300;
    int bt = b->threads, bl = b->tile;
    b->t = b->views[0]->t;
    lb_status st = LB_OK;
    for (int th : cand_threads) {
      if (th > maxt || (b->packed && th != 128)) continue;
      for (int tl : cand_tile) {
        b->threads = th;
        b->tile = tl;
        st = build_items(b);
        if (st != LB_OK) break;
        cudaError_t e = enqueue_batch_step(b, b->t, false, b->stream);  // warm-up
        b->t += 1;
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        for (int k = 0; k < trial_steps && e == cudaSuccess; ++k) {
          e = enqueue_batch_step(b, b->t, false, b->stream);
          b->t += 1;
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
          st = bfail(b, LB_ERR_CUDA, std::string("autotune trial: ") + cudaGetErrorString(e));
          break;
        }
        const double per = ms / trial_steps;
        if (per < best) {
          best = per;
          bt = th;
          bl = tl;
        }
      }
      if (st != LB_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (lb_ctx* v : b->views) {
      v->t = b->t;
      v->gamma_valid = false;
    }
    if (st != LB_OK) return st;
    b->threads = bt;
    b->tile = bl;
    st = build_items(b);
    if (st != LB_OK) return st;
    if (best_threads) *best_threads = bt;
    if (best_tile) *best_tile = bl;
    if (best_ms) *best_ms = best;
    return LB_OK;
  });
}

}  // extern "C"
