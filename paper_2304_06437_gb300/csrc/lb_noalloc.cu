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
//    only a stand-in symbol): the first call on each device, with that device
//    current, looks up its device address with cudaGetSymbolAddress and caches
//    it, so make that first call before any stream capture;
//  * every call on a device shares the same array and leaves its last
//    contents behind; the moments kernel overwrites every entry it later
//    reads, so nothing needs clearing, but calls that overlap on the GPU
//    (different streams, no ordering) race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "lb_dispatch.cuh"
#include "lb_internal.h"

namespace {

constexpr size_t kScratchDoubles = LB_NOALLOC_SCRATCH_BYTES / sizeof(double);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_lb_noalloc_scratch[kScratchDoubles];

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (set-up once)
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_lb_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
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
  for (int64_t i = 0; i < n && e == cudaSuccess; ++i) e = k0_step_buffers(g, f, mom, st);
  if (e == cudaSuccess) {
    dispatch_lattice(lattice, [&](auto Lt) {
      using L = decltype(Lt);
      shift_kernel<L><<<int(blocks), 256, 0, st>>>(f, N, rho0, 0);
    });
    e = cudaGetLastError();
  }
  return status_of(e);
}
