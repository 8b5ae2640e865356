// lb_capi.cu -- the C ABI declared in include/lb.h: argument validation,
// context lifetime, device memory, staging of host buffers and dispatch to
// the kernels.  No function lets a C++ exception or a CUDA error escape: each
// returns an LB_* status code.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>

#include "lb_dispatch.cuh"
#include "lb_internal.h"

namespace lbgb {
size_t reduce_scratch_doubles();
}

using namespace lbgb;

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LB_OK;
  if (e == cudaErrorMemoryAllocation) return LB_E_NOMEM;
  return LB_E_CUDA;
}

#define LB_TRY_CUDA(expr)                     \
  do {                                        \
    cudaError_t _e = (expr);                  \
    if (_e != cudaSuccess) return cuda_status(_e); \
  } while (0)

int lattice_q(int lattice) { return lattice == LB_D2Q9 ? 9 : lattice == LB_D3Q19 ? 19 : lattice == LB_D3Q27 ? 27 : -1; }
int lattice_d(int lattice) { return lattice == LB_D2Q9 ? 2 : 3; }

size_t storage_bytes(int s) {
  switch (s) {
    case LB_F64: return 8;
    case LB_F32: return 4;
    case LB_F16S:
    case LB_BF16S: return 2;
    default: return 0;
  }
}

// Build a 4-D TMA descriptor (x, y, z, direction) of the population array;
// box = one plane of one brick for all directions.
int make_tensor_map(lb_ctx* ctx) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return LB_E_CUDA;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  CUtensorMapDataType dt;
  switch (ctx->storage) {
    case LB_F64: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; break;
    case LB_F32: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
    case LB_F16S: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
    default: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
  }
  const Geometry& g = ctx->g;
  const cuuint64_t es = ctx->elem_bytes;
  cuuint64_t dims[4] = {cuuint64_t(g.nx), cuuint64_t(g.ny), cuuint64_t(g.nz), cuuint64_t(g.q)};
  cuuint64_t strides[3] = {cuuint64_t(g.pitch) * es, cuuint64_t(g.pitch) * g.ny * es, cuuint64_t(g.vol) * es};
  cuuint32_t box[4] = {cuuint32_t(ctx->plan.bx), cuuint32_t(ctx->plan.by), 1u, cuuint32_t(g.q)};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = encode(&ctx->tmap, dt, 4, ctx->f, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? LB_OK : LB_E_CUDA;
}

// Host moment fields cross to and from the device through a buffer of at
// most this size, in two halves: while the context stream converts the chunk
// in one half, a copy stream moves the next (or previous) chunk through the
// other.
constexpr size_t kChunkBytes = size_t(512) << 20;

// The copy stream and the per-half events of one host transfer.  Every
// operation on the copy stream is waited for by the context stream before
// the transfer returns, so destroying them afterwards is safe.
struct CopyLane {
  cudaStream_t s = nullptr;
  cudaEvent_t ready[2] = {nullptr, nullptr};  // half filled (in) / emptied (out)
  cudaEvent_t done[2] = {nullptr, nullptr};   // half consumed (in) / filled (out)
  cudaError_t init() {
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&ready[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming);
    }
    return e;
  }
  ~CopyLane() {
    if (s) cudaStreamSynchronize(s);
    for (int k = 0; k < 2; ++k) {
      if (ready[k]) cudaEventDestroy(ready[k]);
      if (done[k]) cudaEventDestroy(done[k]);
    }
    if (s) cudaStreamDestroy(s);
  }
};

// Stage a host (or device) FP64 input to device memory on the context stream.
struct Staged {
  double* ptr = nullptr;
  bool owned = false;
};

int stage_in(lb_ctx* ctx, const double* src, size_t count, int on_device, Staged* out) {
  out->ptr = nullptr;
  out->owned = false;
  if (!src) return LB_OK;
  if (on_device) {
    out->ptr = const_cast<double*>(src);
    return LB_OK;
  }
  LB_TRY_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&out->ptr), count * sizeof(double), ctx->stream));
  out->owned = true;
  LB_TRY_CUDA(cudaMemcpyAsync(out->ptr, src, count * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  return LB_OK;
}

void unstage(lb_ctx* ctx, Staged* s) {
  if (s->owned && s->ptr) cudaFreeAsync(s->ptr, ctx->stream);
  s->ptr = nullptr;
  s->owned = false;
}

// a state set from outside makes the context usable again after a timeout or
// a refused halo message; an abandoned kernel's status stays
__global__ void clear_status_kernel(int* status) {
  if (*status != LB_E_ABANDONED) *status = 0;
}

int after_state_change(lb_ctx* ctx) {
  if (ctx->scheme == LB_SCHEME_FUSED) LB_TRY_CUDA(k1_bootstrap(ctx));
  if (ctx->d_uprev) ctx->have_uprev = false;
  if (ctx->d_status) {
    clear_status_kernel<<<1, 1, 0, ctx->stream>>>(ctx->d_status);
    LB_TRY_CUDA(cudaGetLastError());
  }
  return LB_OK;
}

int read_status(lb_ctx* ctx) {
  int st = 0;
  LB_TRY_CUDA(cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  LB_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
  return st;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

namespace lbgb {

void drop_step_graph(lb_ctx* ctx) {
  if (ctx->step_graph) cudaGraphExecDestroy(ctx->step_graph);
  ctx->step_graph = nullptr;
}

int ctx_replan(lb_ctx* ctx, const void* variant, int bz) {
  if (!ctx || ctx->scheme != LB_SCHEME_FUSED) return LB_E_INVAL;
  FusedPlan p;
  if (!k1_plan_variant(ctx->g, variant, bz, &p)) return LB_E_INVAL;
  DeviceGuard guard(ctx->device);
  LB_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
  // a captured step pair holds the old shell buffers and brick plan
  drop_step_graph(ctx);
  const size_t aux_bytes = size_t(2) * size_t(p.parity_elems) * ctx->real_bytes;
  void* aux = nullptr;
  LB_TRY_CUDA(cudaMalloc(&aux, aux_bytes));
  cudaError_t e = cudaMemsetAsync(aux, 0, aux_bytes, ctx->stream);
  if (e != cudaSuccess) {
    cudaFree(aux);
    return cuda_status(e);
  }
  const FusedPlan old_plan = ctx->plan;
  void* old_aux = ctx->aux;
  const size_t old_bytes = ctx->aux_bytes;
  ctx->plan = p;
  ctx->aux = aux;
  ctx->aux_bytes = aux_bytes;
  int rc = make_tensor_map(ctx);
  if (rc == LB_OK) rc = cuda_status(k1_configure(ctx));
  if (rc == LB_OK) rc = after_state_change(ctx);  // rebuild the shell from the populations
  if (rc == LB_OK) rc = cuda_status(cudaStreamSynchronize(ctx->stream));
  if (rc != LB_OK) {
    ctx->plan = old_plan;
    ctx->aux = old_aux;
    ctx->aux_bytes = old_bytes;
    make_tensor_map(ctx);
    cudaFree(aux);
    return rc;
  }
  cudaFree(old_aux);
  return LB_OK;
}

}  // namespace lbgb

extern "C" {

int lb_abi_version(void) { return LB_ABI_VERSION; }

const char* lb_status_string(int code) {
  switch (code) {
    case LB_OK: return "ok";
    case LB_E_INVAL: return "invalid argument";
    case LB_E_NOMEM: return "out of memory";
    case LB_E_CUDA: return "CUDA error";
    case LB_E_DIVERGED: return "non-finite state (diverged)";
    case LB_E_TIMEOUT: return "kernel wait timed out";
    case LB_E_UNSUPPORTED: return "unsupported by this build";
    case LB_E_TOO_LARGE: return "grid exceeds the no-allocation scratch size";
    case LB_E_ABANDONED: return "kernel timed out and its copies were not confirmed finished";
    default: return "unknown status";
  }
}

void lb_default_options(lb_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->storage = LB_F32;
  opt->scheme = LB_SCHEME_FUSED;
  opt->rho0 = 1.0;
  opt->stream = nullptr;
  opt->device = -1;
}

int lb_lattice_table(int32_t lattice, int32_t* c, double* w, int32_t* opp) {
  int q = -1;
  dispatch_lattice(lattice, [&](auto Lt) {
    using L = decltype(Lt);
    q = L::Q;
    for (int a = 0; a < L::Q; ++a) {
      // user-facing components: in 2D the internal z axis is the user's y
      const int ux = L::cx(a);
      const int uy = L::D == 2 ? L::cz(a) : L::cy(a);
      const int uz = L::D == 2 ? 0 : L::cz(a);
      if (c) {
        c[3 * a] = ux;
        c[3 * a + 1] = uy;
        c[3 * a + 2] = uz;
      }
      if (w) w[a] = weight<L>(a);
      if (opp) opp[a] = L::opp(a);
    }
  });
  return q < 0 ? LB_E_INVAL : q;
}

int lb_memory_plan(int32_t lattice, int32_t bytes_per_value, lb_memory_plan_t* out) {
  const int q = lattice_q(lattice);
  if (q < 0 || !out || bytes_per_value <= 0) return LB_E_INVAL;
  const int d = lattice_d(lattice);
  lb_memory_plan_t p;
  p.q = q;
  p.m = 1 + d + d * (d + 1) / 2;
  p.arrays_moment_scheme = q + p.m;
  p.arrays_flip_flop = 2 * q + d + 1;
  p.arrays_single = q;
  p.bytes_per_node_moment_scheme = double(p.arrays_moment_scheme) * bytes_per_value;
  p.bytes_per_node_flip_flop = double(p.arrays_flip_flop) * bytes_per_value;
  p.bytes_per_node_single = double(p.arrays_single) * bytes_per_value;
  *out = p;
  return LB_OK;
}

int lb_plan_fused(int32_t lattice, int32_t storage, const int64_t dims[3], const int32_t tile[3], int32_t sms,
                  lb_plan_t* out) {
  if (!out || !dims || sms < 0) return LB_E_INVAL;
  const int q = lattice_q(lattice);
  if (q < 0 || storage_bytes(storage) == 0) return LB_E_INVAL;
  const int d = lattice_d(lattice);
  for (int k = 0; k < 3; ++k)
    if (dims[k] < 1 || dims[k] > (int64_t(1) << 30)) return LB_E_INVAL;
  if (d == 2 && dims[2] != 1) return LB_E_INVAL;
  // the internal axes of lb_create: 2D (x, y) -> (x, z)
  Geometry g{};
  g.lattice = lattice;
  g.q = q;
  g.d = d;
  g.nx = int(dims[0]);
  g.ny = d == 2 ? 1 : int(dims[1]);
  g.nz = d == 2 ? int(dims[1]) : int(dims[2]);
  FusedPlan p{};
  if (!k1_plan(g, storage, tile, &p, sms)) return LB_E_UNSUPPORTED;
  out->bx = p.bx;
  out->by = p.by;
  out->bz = p.bz;
  out->nbx = p.nbx;
  out->nby = p.nby;
  out->nbz = p.nbz;
  out->bricks = int64_t(p.nbx) * p.nby * p.nbz;
  out->tma_slots = p.slots;
  out->nodes_per_thread = p.npt;
  out->export_warps = p.xwarps;
  out->shared_bytes = int64_t(p.smem_bytes);
  out->shell_elems_per_parity = p.sx_elems + p.sy_elems + p.sz_elems;
  return LB_OK;
}

int lb_create(int32_t lattice, const int64_t dims[3], double tau, const lb_boundary* bnd, const lb_options* opt_in,
              lb_ctx** out) {
  if (!out) return LB_E_INVAL;
  *out = nullptr;
  const int q = lattice_q(lattice);
  if (q < 0 || !dims) return LB_E_INVAL;
  const int d = lattice_d(lattice);
  for (int k = 0; k < 3; ++k)
    if (dims[k] < 1 || dims[k] > (int64_t(1) << 30)) return LB_E_INVAL;
  if (d == 2 && dims[2] != 1) return LB_E_INVAL;
  if (!(tau > 0.5) || !(tau < 1e6)) return LB_E_INVAL;
  lb_options opt;
  if (opt_in) opt = *opt_in;
  else lb_default_options(&opt);
  if (!(opt.rho0 > 0.0)) return LB_E_INVAL;
  if (storage_bytes(opt.storage) == 0) return LB_E_INVAL;
  if (opt.scheme != LB_SCHEME_FUSED && opt.scheme != LB_SCHEME_TWO_PASS) return LB_E_INVAL;
  lb_boundary b;
  if (bnd) b = *bnd;
  else std::memset(&b, 0, sizeof(b));
  for (int ax = 0; ax < 3; ++ax) {
    const int lo = b.kind[2 * ax], hi = b.kind[2 * ax + 1];
    if (lo < 0 || lo > LB_LINK || hi < 0 || hi > LB_LINK) return LB_E_INVAL;
    if ((lo == LB_PERIODIC) != (hi == LB_PERIODIC)) return LB_E_INVAL;
  }
  if (d == 2 && (b.kind[4] != LB_PERIODIC || b.kind[5] != LB_PERIODIC)) {
    // the z faces of a 2D grid carry no velocities; accept any kind but ignore it
    b.kind[4] = b.kind[5] = LB_PERIODIC;
  }
  // link faces: only the two faces of the slowest axis (z in 3D, y in 2D),
  // and only with the fused scheme
  bool any_link = false;
  for (int f = 0; f < 6; ++f) {
    if (b.kind[f] != LB_LINK) continue;
    if (f / 2 != d - 1) return LB_E_INVAL;
    any_link = true;
  }
  if (any_link && opt.scheme != LB_SCHEME_FUSED) return LB_E_UNSUPPORTED;

  lb_ctx* ctx = new (std::nothrow) lb_ctx();
  if (!ctx) return LB_E_NOMEM;
  ctx->bnd_user = b;
  ctx->opt_user = opt;
  ctx->tau_user = tau;
  ctx->lattice = lattice;
  ctx->storage = opt.storage;
  ctx->scheme = opt.scheme;
  for (int k = 0; k < 3; ++k) ctx->dims[k] = dims[k];
  ctx->n_nodes = dims[0] * dims[1] * dims[2];
  ctx->elem_bytes = storage_bytes(opt.storage);
  ctx->real_bytes = opt.storage == LB_F64 ? 8 : 4;

  Geometry& g = ctx->g;
  g.lattice = lattice;
  g.q = q;
  g.d = d;
  g.tau = tau;
  g.rho0 = opt.rho0;
  // internal axes: 3D identity; 2D (x, y) -> (x, z) with an internal y of 1
  const int ax_of_user[3] = {0, d == 2 ? 2 : 1, d == 2 ? 1 : 2};
  int n_int[3] = {1, 1, 1};
  for (int k = 0; k < d; ++k) n_int[ax_of_user[k]] = int(dims[k]);
  if (d == 3) n_int[2] = int(dims[2]);
  g.nx = n_int[0];
  g.ny = n_int[1];
  g.nz = n_int[2];
  for (int f = 0; f < 6; ++f) {
    g.face_kind[f] = LB_PERIODIC;
    for (int k = 0; k < 3; ++k) g.wall_u[f][k] = 0.0;
  }
  for (int k = 0; k < 3; ++k) g.force[k] = 0.0;
  for (int uk = 0; uk < d; ++uk) {
    const int ia = ax_of_user[uk];
    g.face_kind[2 * ia] = b.kind[2 * uk];
    g.face_kind[2 * ia + 1] = b.kind[2 * uk + 1];
    g.force[ia] = opt.force[uk];
  }
  for (int f = 0; f < 2 * d; ++f) {
    const int uk = f / 2, side = f % 2;
    const int ifc = 2 * ax_of_user[uk] + side;
    for (int k = 0; k < d; ++k) g.wall_u[ifc][ax_of_user[k]] = b.wall_u[f][k];
  }
  g.has_force = g.force[0] != 0.0 || g.force[1] != 0.0 || g.force[2] != 0.0;
  for (int ax = 0; ax < 3; ++ax) g.per[ax] = g.face_kind[2 * ax] == LB_PERIODIC ? 1 : 0;
  for (int k = 0; k < 2; ++k) g.zlink[k] = g.face_kind[4 + k] == LB_LINK ? 1 : 0;
  g.pitch = (int64_t(g.nx) + 31) / 32 * 32;
  g.vol = g.pitch * g.ny * g.nz;

  ctx->stream = nullptr;
  ctx->own_stream = false;
  int dev = opt.device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
    delete ctx;
    return LB_E_CUDA;
  }
  ctx->device = dev;
  DeviceGuard guard(dev);
  int rc = LB_OK;
  do {
    if (opt.stream) {
      ctx->stream = static_cast<cudaStream_t>(opt.stream);
    } else {
      if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { rc = LB_E_CUDA; break; }
      ctx->own_stream = true;
    }
    if (ctx->scheme == LB_SCHEME_FUSED) {
      if (!k1_plan(g, ctx->storage, opt.tile, &ctx->plan)) { rc = LB_E_UNSUPPORTED; break; }
      ctx->aux_bytes = size_t(2) * size_t(ctx->plan.parity_elems) * ctx->real_bytes;
    } else {
      if (g.ny > 65535 || g.nz > 65535) { rc = LB_E_UNSUPPORTED; break; }
      ctx->aux_bytes = k0_aux_bytes(g, ctx->storage);
    }
    ctx->f_bytes = size_t(q) * size_t(g.vol) * ctx->elem_bytes;
    cudaError_t e = cudaMalloc(&ctx->f, ctx->f_bytes);
    if (e != cudaSuccess) { rc = cuda_status(e); break; }
    if (ctx->aux_bytes) {
      e = cudaMalloc(&ctx->aux, ctx->aux_bytes);
      if (e != cudaSuccess) { rc = cuda_status(e); break; }
      e = cudaMemsetAsync(ctx->aux, 0, ctx->aux_bytes, ctx->stream);
      if (e != cudaSuccess) { rc = cuda_status(e); break; }
    }
    e = cudaMalloc(reinterpret_cast<void**>(&ctx->d_status), sizeof(int));
    if (e != cudaSuccess) { rc = cuda_status(e); break; }
    e = cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) { rc = cuda_status(e); break; }
    e = cudaMalloc(reinterpret_cast<void**>(&ctx->d_red), reduce_scratch_doubles() * sizeof(double));
    if (e != cudaSuccess) { rc = cuda_status(e); break; }
    // pitch padding stays zero forever
    e = cudaMemsetAsync(ctx->f, 0, ctx->f_bytes, ctx->stream);
    if (e != cudaSuccess) { rc = cuda_status(e); break; }
    if (ctx->scheme == LB_SCHEME_FUSED) {
      rc = make_tensor_map(ctx);
      if (rc != LB_OK) break;
      e = k1_configure(ctx);
      if (e != cudaSuccess) { rc = cuda_status(e); break; }
    }
    const double zero[3] = {0, 0, 0};
    e = aux_init_uniform(ctx, g.rho0, zero);
    if (e != cudaSuccess) { rc = cuda_status(e); break; }
    rc = after_state_change(ctx);
    if (rc != LB_OK) break;
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { rc = cuda_status(e); break; }
  } while (false);
  if (rc != LB_OK) {
    lb_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return LB_OK;
}

void lb_destroy(lb_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard guard(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  drop_step_graph(ctx);
  if (ctx->f) cudaFree(ctx->f);
  if (ctx->aux) cudaFree(ctx->aux);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_red) cudaFree(ctx->d_red);
  if (ctx->d_uprev) cudaFree(ctx->d_uprev);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

int lb_init_moments(lb_ctx* ctx, const double* rho, const double* u, const double* pineq, int32_t on_device) {
  if (!ctx || !rho || !u) return LB_E_INVAL;
  DeviceGuard guard(ctx->device);
  const size_t N = size_t(ctx->n_nodes);
  const int d = ctx->g.d;
  const int np = d == 2 ? 3 : 6;
  if (!on_device) {
    // host fields: chunks of nodes through the two halves of one bounded
    // device buffer (one copy per component on the copy stream), each chunk
    // converted on the context stream as it lands
    const int ncomp = 1 + d + (pineq ? np : 0);
    const size_t C = std::max<size_t>(1, std::min(N, kChunkBytes / (2 * size_t(ncomp) * sizeof(double))));
    CopyLane lane;
    LB_TRY_CUDA(lane.init());
    double* buf = nullptr;
    LB_TRY_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&buf), 2 * C * ncomp * sizeof(double), ctx->stream));
    // the copy stream starts after the allocation (and after the work
    // already queued on the context stream)
    int rc = cuda_status(cudaEventRecord(lane.done[1], ctx->stream));
    if (rc == LB_OK) rc = cuda_status(cudaStreamWaitEvent(lane.s, lane.done[1], 0));
    size_t k = 0;
    for (size_t n0 = 0; n0 < N && rc == LB_OK; n0 += C, ++k) {
      const size_t cnt = std::min(C, N - n0);
      const int h = int(k & 1);
      double* br = buf + size_t(h) * C * ncomp;
      double* bu = br + C;
      double* bp = br + C * (1 + d);
      // the conversion of the chunk two back has left this half
      if (k >= 2) rc = cuda_status(cudaStreamWaitEvent(lane.s, lane.done[h], 0));
      if (rc == LB_OK)
        rc = cuda_status(cudaMemcpyAsync(br, rho + n0, cnt * sizeof(double), cudaMemcpyHostToDevice, lane.s));
      for (int c = 0; c < d && rc == LB_OK; ++c)
        rc = cuda_status(cudaMemcpyAsync(bu + c * C, u + c * N + n0, cnt * sizeof(double), cudaMemcpyHostToDevice,
                                         lane.s));
      for (int c = 0; pineq && c < np && rc == LB_OK; ++c)
        rc = cuda_status(cudaMemcpyAsync(bp + c * C, pineq + c * N + n0, cnt * sizeof(double),
                                         cudaMemcpyHostToDevice, lane.s));
      if (rc == LB_OK) rc = cuda_status(cudaEventRecord(lane.ready[h], lane.s));
      if (rc == LB_OK) rc = cuda_status(cudaStreamWaitEvent(ctx->stream, lane.ready[h], 0));
      if (rc == LB_OK)
        rc = cuda_status(aux_init_moments_range(ctx, br, bu, pineq ? bp : nullptr, int64_t(n0), int64_t(n0 + cnt),
                                                int64_t(C)));
      if (rc == LB_OK) rc = cuda_status(cudaEventRecord(lane.done[h], ctx->stream));
    }
    // nothing on the copy stream may outlive the buffer
    if (cudaEventRecord(lane.ready[0], lane.s) == cudaSuccess) cudaStreamWaitEvent(ctx->stream, lane.ready[0], 0);
    cudaFreeAsync(buf, ctx->stream);
    if (rc == LB_OK) rc = after_state_change(ctx);
    const int rc2 = cuda_status(cudaStreamSynchronize(ctx->stream));
    return rc != LB_OK ? rc : rc2;
  }
  Staged sr, su, sp;
  int rc = stage_in(ctx, rho, N, on_device, &sr);
  if (rc == LB_OK) rc = stage_in(ctx, u, N * d, on_device, &su);
  if (rc == LB_OK) rc = stage_in(ctx, pineq, N * np, on_device, &sp);
  if (rc == LB_OK) rc = cuda_status(aux_init_moments(ctx, sr.ptr, su.ptr, sp.ptr));
  if (rc == LB_OK) rc = after_state_change(ctx);
  unstage(ctx, &sr);
  unstage(ctx, &su);
  unstage(ctx, &sp);
  if (rc == LB_OK) rc = cuda_status(cudaStreamSynchronize(ctx->stream));
  return rc;
}

int lb_init_uniform(lb_ctx* ctx, double rho, const double u[3]) {
  if (!ctx || !u) return LB_E_INVAL;
  DeviceGuard guard(ctx->device);
  double uu[3] = {u[0], u[1], ctx->g.d == 3 ? u[2] : 0.0};
  int rc = cuda_status(aux_init_uniform(ctx, rho, uu));
  if (rc == LB_OK) rc = after_state_change(ctx);
  if (rc == LB_OK) rc = cuda_status(cudaStreamSynchronize(ctx->stream));
  return rc;
}

int lb_set_populations(lb_ctx* ctx, const double* f, int32_t on_device) {
  if (!ctx || !f) return LB_E_INVAL;
  DeviceGuard guard(ctx->device);
  Staged sf;
  int rc = stage_in(ctx, f, size_t(ctx->g.q) * size_t(ctx->n_nodes), on_device, &sf);
  if (rc == LB_OK) rc = cuda_status(aux_set_populations(ctx, sf.ptr));
  if (rc == LB_OK) rc = after_state_change(ctx);
  unstage(ctx, &sf);
  if (rc == LB_OK) rc = cuda_status(cudaStreamSynchronize(ctx->stream));
  return rc;
}

static int copy_out(lb_ctx* ctx, double* dst, size_t count, int on_device,
                    cudaError_t (*fill)(lb_ctx*, double*, void*), void* arg) {
  if (on_device) {
    int rc = cuda_status(fill(ctx, dst, arg));
    if (rc == LB_OK) rc = cuda_status(cudaStreamSynchronize(ctx->stream));
    return rc;
  }
  double* tmp = nullptr;
  LB_TRY_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&tmp), count * sizeof(double), ctx->stream));
  int rc = cuda_status(fill(ctx, tmp, arg));
  if (rc == LB_OK)
    rc = cuda_status(cudaMemcpyAsync(dst, tmp, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  cudaFreeAsync(tmp, ctx->stream);
  const int rc2 = cuda_status(cudaStreamSynchronize(ctx->stream));
  return rc != LB_OK ? rc : rc2;
}

int lb_get_populations(lb_ctx* ctx, double* f, int32_t on_device) {
  if (!ctx || !f) return LB_E_INVAL;
  DeviceGuard guard(ctx->device);
  return copy_out(ctx, f, size_t(ctx->g.q) * size_t(ctx->n_nodes), on_device,
                  [](lb_ctx* c, double* p, void*) { return aux_get_populations(c, p); }, nullptr);
}

struct RegionArg {
  const int64_t* lo;
  const int64_t* size;
};

int lb_get_region(lb_ctx* ctx, const int64_t lo[3], const int64_t size[3], double* f_host) {
  if (!ctx || !lo || !size || !f_host) return LB_E_INVAL;
  for (int k = 0; k < 3; ++k)
    if (lo[k] < 0 || size[k] < 1 || lo[k] + size[k] > ctx->dims[k]) return LB_E_INVAL;
  DeviceGuard guard(ctx->device);
  RegionArg ra{lo, size};
  const size_t count = size_t(ctx->g.q) * size_t(size[0] * size[1] * size[2]);
  return copy_out(ctx, f_host, count, 0,
                  [](lb_ctx* c, double* p, void* a) {
                    const RegionArg* r = static_cast<const RegionArg*>(a);
                    return aux_get_region(c, r->lo, r->size, p);
                  },
                  &ra);
}

// Record two fused steps, from the current shell parity, as a CUDA graph on
// the context stream (nothing runs).  Returns false, leaving no error set,
// where the stream cannot be captured (it is already being captured, e.g. by
// the caller) or capture fails; lb_step then launches step by step.
static bool capture_step_pair(lb_ctx* ctx) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return false;
  }
  const int p0 = ctx->parity;
  if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaError_t e = k1_step(ctx);
  if (e == cudaSuccess) e = k1_step(ctx);
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(ctx->stream, &graph);
  ctx->parity = p0;  // the pair was only recorded
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess && ee == cudaSuccess && graph) e = cudaGraphInstantiate(&exec, graph, 0);
  else e = cudaErrorStreamCaptureInvalidated;
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  if (e != cudaSuccess || !exec) return false;
  ctx->step_graph = exec;
  ctx->graph_parity = p0;
  return true;
}

int lb_step(lb_ctx* ctx, int64_t n) {
  if (!ctx || n < 0) return LB_E_INVAL;
  // a slab bordering others takes one step between two halo exchanges
  if (n > 1 && (ctx->g.zlink[0] || ctx->g.zlink[1])) return LB_E_INVAL;
  DeviceGuard guard(ctx->device);
  int64_t i = 0;
  // long runs of the fused scheme replay a captured pair of steps: one graph
  // launch per two steps instead of two launches, each with its host-side
  // argument set-up (what dominates the step of a small domain)
  constexpr int64_t kGraphMinSteps = 4;
  if (ctx->scheme == LB_SCHEME_FUSED && n >= kGraphMinSteps) {
    if (ctx->step_graph && ctx->parity != ctx->graph_parity) {
      // the pair starts from the other parity: one plain step first
      cudaError_t e = k1_step(ctx);
      if (e != cudaSuccess) return cuda_status(e);
      ctx->steps_done++;
      ++i;
    }
    if (ctx->step_graph || capture_step_pair(ctx)) {
      for (; i + 2 <= n; i += 2) {
        cudaError_t e = cudaGraphLaunch(ctx->step_graph, ctx->stream);
        if (e != cudaSuccess) return cuda_status(e);
        ctx->steps_done += 2;
      }
    }
  }
  for (; i < n; ++i) {
    cudaError_t e = ctx->scheme == LB_SCHEME_FUSED ? k1_step(ctx) : k0_step(ctx);
    if (e != cudaSuccess) return cuda_status(e);
    ctx->steps_done++;
  }
  return LB_OK;
}

struct MomArg {
  double* rho;
  double* u;
};

int lb_moments(lb_ctx* ctx, double* rho, double* u, int32_t on_device) {
  if (!ctx || (!rho && !u)) return LB_E_INVAL;
  DeviceGuard guard(ctx->device);
  const size_t N = size_t(ctx->n_nodes);
  const int d = ctx->g.d;
  if (on_device) {
    int rc = cuda_status(aux_moments(ctx, rho, u));
    if (rc == LB_OK) rc = cuda_status(cudaStreamSynchronize(ctx->stream));
    return rc;
  }
  // chunks of nodes through the two halves of one bounded device buffer:
  // the context stream fills a half, the copy stream empties it to the host
  const size_t C = std::max<size_t>(1, std::min(N, kChunkBytes / (2 * (1 + d) * sizeof(double))));
  CopyLane lane;
  LB_TRY_CUDA(lane.init());
  double* tmp = nullptr;
  LB_TRY_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&tmp), 2 * (1 + d) * C * sizeof(double), ctx->stream));
  int rc = LB_OK;
  size_t k = 0;
  for (size_t n0 = 0; n0 < N && rc == LB_OK; n0 += C, ++k) {
    const size_t cnt = std::min(C, N - n0);
    const int h = int(k & 1);
    double* half = tmp + size_t(h) * (1 + d) * C;
    // the copy of the chunk two back has left this half
    if (k >= 2) rc = cuda_status(cudaStreamWaitEvent(ctx->stream, lane.ready[h], 0));
    if (rc == LB_OK)
      rc = cuda_status(aux_moments_range(ctx, rho ? half : nullptr, u ? half + C : nullptr, int64_t(n0),
                                         int64_t(n0 + cnt), int64_t(C)));
    if (rc == LB_OK) rc = cuda_status(cudaEventRecord(lane.done[h], ctx->stream));
    if (rc == LB_OK) rc = cuda_status(cudaStreamWaitEvent(lane.s, lane.done[h], 0));
    if (rc == LB_OK && rho)
      rc = cuda_status(cudaMemcpyAsync(rho + n0, half, cnt * sizeof(double), cudaMemcpyDeviceToHost, lane.s));
    for (int c = 0; u && c < d && rc == LB_OK; ++c)
      rc = cuda_status(cudaMemcpyAsync(u + c * N + n0, half + C + c * C, cnt * sizeof(double),
                                       cudaMemcpyDeviceToHost, lane.s));
    if (rc == LB_OK) rc = cuda_status(cudaEventRecord(lane.ready[h], lane.s));
  }
  // the context stream (and so the caller's synchronisation) waits for the
  // last copies; the buffer is freed after them
  if (cudaEventRecord(lane.ready[0], lane.s) == cudaSuccess) cudaStreamWaitEvent(ctx->stream, lane.ready[0], 0);
  cudaFreeAsync(tmp, ctx->stream);
  const int rc2 = cuda_status(cudaStreamSynchronize(ctx->stream));
  return rc != LB_OK ? rc : rc2;
}

int lb_reduce(lb_ctx* ctx, double* mass, double mom[3], double* residual) {
  if (!ctx) return LB_E_INVAL;
  DeviceGuard guard(ctx->device);
  double out[7];
  const bool want_res = residual != nullptr;
  int rc = cuda_status(aux_reduce(ctx, out, want_res));
  if (rc != LB_OK) return rc;
  return reduce_finish(ctx, out, want_res, mass, mom, residual);
}

}  // extern "C"

int lbgb::reduce_finish(lb_ctx* ctx, const double* out, bool want_res, double* mass, double mom[3],
                        double* residual) {
  const int d = ctx->g.d;
  if (mass) *mass = out[0];
  if (mom) {
    // internal (x, y, z) -> user axes
    const double ji[3] = {out[1], out[2], out[3]};
    mom[0] = ji[0];
    mom[1] = d == 2 ? ji[2] : ji[1];
    mom[2] = d == 2 ? 0.0 : ji[2];
  }
  if (want_res) {
    *residual = (ctx->have_uprev && out[5] > 0.0) ? std::sqrt(out[4] / out[5]) : 1.0;
    ctx->have_uprev = true;
  }
  if (out[6] != 0.0 || !std::isfinite(out[0])) return LB_E_DIVERGED;
  return LB_OK;
}

extern "C" {

int lb_sync(lb_ctx* ctx) {
  if (!ctx) return LB_E_INVAL;
  DeviceGuard guard(ctx->device);
  LB_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
  LB_TRY_CUDA(cudaGetLastError());
  const int st = read_status(ctx);
  return st == 0 ? LB_OK : st;
}

int lb_info(const lb_ctx* ctx, lb_info_t* info) {
  if (!ctx || !info) return LB_E_INVAL;
  std::memset(info, 0, sizeof(*info));
  info->lattice = ctx->lattice;
  info->q = ctx->g.q;
  info->d = ctx->g.d;
  info->storage = ctx->storage;
  info->scheme = ctx->scheme;
  for (int k = 0; k < 3; ++k) info->dims[k] = ctx->dims[k];
  info->steps_done = ctx->steps_done;
  if (ctx->scheme == LB_SCHEME_FUSED) {
    info->tile[0] = ctx->plan.bx;
    info->tile[1] = ctx->plan.by;
    info->tile[2] = ctx->plan.bz;
    info->nodes_per_thread = ctx->plan.npt;
    info->tma_slots = ctx->plan.slots;
  }
  info->population_bytes = ctx->f_bytes;
  info->aux_bytes = ctx->aux_bytes;
  info->algorithmic_bytes_per_update = uint64_t(2) * ctx->g.q * ctx->elem_bytes;
  return LB_OK;
}

}  // extern "C"
