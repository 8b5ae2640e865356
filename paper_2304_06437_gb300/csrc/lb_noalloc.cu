// lb_noalloc.cu -- lb_step_noalloc(): the two-pass step for callers that must
// not allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: their device memory is
// owned by another allocator (a framework's caching pool or a fixed memory
// budget that leaves nothing to spare), or they run latency-sensitive loops
// that must not enter the driver's allocator.  This entry point allocates
// nothing.  The caller passes the population array; the per-node moment
// arrays of the two-pass schedule, which lb_create would allocate, live in a
// fixed file-scope device array instead.
//
// Scratch rules:
//  * g_lb_noalloc_scratch holds LB_NOALLOC_SCRATCH_BYTES; once this entry point
//    has been used on a device (with lazy module loading: from first use,
//    otherwise from library load), that device keeps the array until the
//    process exits;
//  * host code never passes the array's name to a kernel (on the host it is
//    only a stand-in symbol): the first call in each CUDA context (normally
//    the device's primary context), with that context current, looks up its
//    device address with cudaGetSymbolAddress and caches it under the
//    context's unique id, so make that first call before any stream capture;
//    a context created later (after cudaDeviceReset, or a driver-API context
//    made current by the caller) has a new id and gets its own look-up, never
//    a stale address;
//  * every call on a device shares the same array and leaves its last
//    contents behind; the moments kernel overwrites every entry it later
//    reads, so nothing needs clearing, but calls that overlap on the GPU
//    (different streams, no ordering) race on the array.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "lb_dispatch.cuh"
#include "lb_internal.h"

namespace {

constexpr size_t kScratchDoubles = LB_NOALLOC_SCRATCH_BYTES / sizeof(double);
constexpr int kCacheEntries = 64;

static __device__ __align__(256) double g_lb_noalloc_scratch[kScratchDoubles];

std::mutex g_setup_mutex;

// cache of the array's device address per CUDA context, keyed by the
// context's process-unique id (cuCtxGetId; a handle value can be reused after
// a context is destroyed, an id cannot)
struct ScratchEntry {
  unsigned long long ctx_id;
  double* addr;
};
ScratchEntry g_scratch_cache[kCacheEntries] = {};
int g_scratch_used = 0, g_scratch_next = 0;

typedef CUresult (*PFN_ctx_get_current)(CUcontext*);
typedef CUresult (*PFN_ctx_get_id)(CUcontext, unsigned long long*);

template <class F>
cudaError_t driver_fn(const char* name, unsigned version, F* out) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion(name, &fn, version, cudaEnableDefault, &q);
  if (e != cudaSuccess) return e;
  if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorSymbolNotFound;
  *out = reinterpret_cast<F>(fn);
  return cudaSuccess;
}

// device address of the scratch array in the current context (set-up once per
// context)
cudaError_t scratch_address(double** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  static PFN_ctx_get_current get_current = nullptr;
  static PFN_ctx_get_id get_id = nullptr;
  cudaError_t e;
  if (!get_current && (e = driver_fn("cuCtxGetCurrent", 4000, &get_current)) != cudaSuccess) return e;
  if (!get_id && (e = driver_fn("cuCtxGetId", 12000, &get_id)) != cudaSuccess) return e;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  void* p = nullptr;
  if (!ctx) {
    // no context current yet: the runtime call below makes the device's
    // primary context current
    e = cudaGetSymbolAddress(&p, g_lb_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  }
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  for (int k = 0; k < g_scratch_used; ++k)
    if (g_scratch_cache[k].ctx_id == id) {
      *out = g_scratch_cache[k].addr;
      return cudaSuccess;
    }
  if (!p) {
    e = cudaGetSymbolAddress(&p, g_lb_noalloc_scratch);
    if (e != cudaSuccess) return e;
  }
  // a full table recycles its oldest entry: that context only looks its
  // address up again on its next call
  ScratchEntry& slot = g_scratch_cache[g_scratch_used < kCacheEntries ? g_scratch_used++ : g_scratch_next];
  if (g_scratch_used == kCacheEntries) g_scratch_next = (g_scratch_next + 1) % kCacheEntries;
  slot.ctx_id = id;
  slot.addr = static_cast<double*>(p);
  *out = slot.addr;
  return cudaSuccess;
}

// in-place conversion between f and the shifted ft = f - t_a rho0, the same
// arithmetic as lb_set_populations / lb_get_populations
template <class L>
__global__ void shift_kernel(double* __restrict__ f, int64_t n, double rho0, int to_shifted) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    lbgb::static_for<0, L::Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      const double v = f[a * n + i];
      f[a * n + i] = to_shifted ? v - lbgb::weight<L>(a) * rho0 : v + lbgb::weight<L>(a) * rho0;
    });
  }
}

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return LB_OK;
  if (e == cudaErrorMemoryAllocation) return LB_E_NOMEM;
  return LB_E_CUDA;
}

}  // namespace

extern "C" int lb_step_noalloc(int32_t lattice, const int64_t dims[3], double tau, const lb_boundary* bnd,
                               double rho0, const double force[3], double* f, int64_t n, void* stream) {
  using namespace lbgb;
  const int q = lattice == LB_D2Q9 ? 9 : lattice == LB_D3Q19 ? 19 : lattice == LB_D3Q27 ? 27 : -1;
  if (q < 0 || !dims || !f || n < 0) return LB_E_INVAL;
  const int d = lattice == LB_D2Q9 ? 2 : 3;
  for (int k = 0; k < 3; ++k)
    if (dims[k] < 1 || dims[k] > (int64_t(1) << 30)) return LB_E_INVAL;
  if (d == 2 && dims[2] != 1) return LB_E_INVAL;
  if (!(tau > 0.5) || !(tau < 1e6) || !(rho0 > 0.0)) return LB_E_INVAL;
  lb_boundary b;
  if (bnd) b = *bnd;
  else b = lb_boundary{};
  for (int ax = 0; ax < 3; ++ax) {
    const int lo = b.kind[2 * ax], hi = b.kind[2 * ax + 1];
    if (lo < 0 || lo > 2 || hi < 0 || hi > 2) return LB_E_INVAL;
    if ((lo == LB_PERIODIC) != (hi == LB_PERIODIC)) return LB_E_INVAL;
  }
  const int m = 1 + d + d * (d + 1) / 2;
  const int64_t N = dims[0] * dims[1] * dims[2];
  if (N > int64_t(kScratchDoubles / size_t(m))) return LB_E_TOO_LARGE;

  // geometry in internal axes (2D: the user's y is the internal z axis)
  Geometry g{};
  g.lattice = lattice;
  g.q = q;
  g.d = d;
  g.tau = tau;
  g.rho0 = rho0;
  const int ax_of_user[3] = {0, d == 2 ? 2 : 1, d == 2 ? 1 : 2};
  int n_int[3] = {1, 1, 1};
  for (int k = 0; k < d; ++k) n_int[ax_of_user[k]] = int(dims[k]);
  g.nx = n_int[0];
  g.ny = n_int[1];
  g.nz = n_int[2];
  for (int fc = 0; fc < 6; ++fc) g.face_kind[fc] = LB_PERIODIC;
  for (int uk = 0; uk < d; ++uk) {
    const int ia = ax_of_user[uk];
    g.face_kind[2 * ia] = b.kind[2 * uk];
    g.face_kind[2 * ia + 1] = b.kind[2 * uk + 1];
    g.force[ia] = force ? force[uk] : 0.0;
  }
  for (int fc = 0; fc < 2 * d; ++fc) {
    const int ifc = 2 * ax_of_user[fc / 2] + fc % 2;
    for (int k = 0; k < d; ++k) g.wall_u[ifc][ax_of_user[k]] = b.wall_u[fc][k];
  }
  g.has_force = g.force[0] != 0.0 || g.force[1] != 0.0 || g.force[2] != 0.0;
  for (int ax = 0; ax < 3; ++ax) g.per[ax] = g.face_kind[2 * ax] == LB_PERIODIC ? 1 : 0;
  g.pitch = g.nx;  // the caller's canonical layout: no row padding
  g.vol = N;
  if (g.ny > 65535 || g.nz > 65535) return LB_E_UNSUPPORTED;

  double* mom = nullptr;
  cudaError_t e = scratch_address(&mom);
  if (e != cudaSuccess) return status_of(e);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int64_t blocks = (N + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  dispatch_lattice(lattice, [&](auto Lt) {
    using L = decltype(Lt);
    shift_kernel<L><<<int(blocks), 256, 0, st>>>(f, N, rho0, 1);
  });
  e = cudaGetLastError();
  if (e != cudaSuccess) return status_of(e);
  for (int64_t i = 0; i < n && e == cudaSuccess; ++i) e = k0_step_buffers(g, f, mom, st);
  // shift back even when a step failed to launch, so that f holds unshifted
  // populations after however many steps did complete
  dispatch_lattice(lattice, [&](auto Lt) {
    using L = decltype(Lt);
    shift_kernel<L><<<int(blocks), 256, 0, st>>>(f, N, rho0, 0);
  });
  const cudaError_t e2 = cudaGetLastError();
  return status_of(e != cudaSuccess ? e : e2);
}
