// lb_cg.cu -- two-component colour-gradient step (paper section 2.1) in the
// thread-safe form of section 4: moments are taken in one launch, the phase
// field gradient in a second, and a third rebuilds each colour's populations
// at every node by pulling the post-collision set of the upstream node from
// those moment fields.  No launch reads and writes the same population, so
// each colour keeps ONE population array.
//
// Per node x (moments launch), from the two colours f_R, f_B:
//   rho_R = sum f_R, rho_B = sum f_B, g = f_R + f_B, and the regularized
//   relaxation coefficients of g (lb_collide.cuh: A, B, C, the order-2
//   Hermite form of Eq. LBexp / Eq. hermite), phi = (rho_R - rho_B) / rho,
//   c_R = rho_R / rho and c_RB = beta rho_R rho_B / rho;
// (gradient launch) grad phi = (1/cs2) sum_a t_a c_a phi(x + c_a), stored as
//   |grad phi| and the unit normal n;
// (rebuild launch) for every direction a and upstream node x = y - c_a:
//   g*_a = t_a (A + B.c_a + c_a.C.c_a) + (9/4) sigma omega |grad phi|
//          [t_a (c_a.n)^2 - B_a]                          (perturbation)
//   f_R(y)_a = c_R g*_a + c_RB t_a (c_a.n)/|c_a|,  f_B(y)_a = g*_a - f_R(y)_a
//                                                         (recolouring)
// Each colour is stored shifted by half the rest population, t_a rho0 / 2,
// so that g is stored shifted by t_a rho0 as in the single-component path.
// Periodic box only; D2Q9 and D3Q19; FP64 or FP32 storage and arithmetic.
//
// Near-contact interactions (section 2.2), when switched on: the gradient
// launch also flags node y if, for some direction a, the node y - h c_a is
// bulk (phi < -1 + eps) and both y and y - 2h c_a are not -- the paper's test
// from the bulk node, written from the flagged node so that every thread
// writes only its own node -- and a flagged node's relaxation coefficients
// are recomputed from its own populations with the body force
// F = A rho_R grad phi / |grad phi| (the forcing of the single-component
// step).  No thread reads coefficients in that launch, and populations are
// only written by the rebuild launch after it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "lb_dispatch.cuh"

namespace lbgb {
namespace {

constexpr int kCgThreads = 256;
// per-node fields of the moments launch: 10 relaxation coefficients, c_R,
// c_RB, phi; of the gradient launch: |grad phi| and n (3)
constexpr int kCgFields = 17;
enum { F_COEF = 0, F_CR = 10, F_CRB = 11, F_PHI = 12, F_GN = 13, F_N = 14 };

struct CgGeom {
  int nx, ny, nz;  // internal axes (2D: nx x 1 x ny)
  int64_t n;
};

__device__ __forceinline__ int64_t cg_wrap_index(const CgGeom& g, int x, int y, int z) {
  x = x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x);
  y = y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
  z = z < 0 ? z + g.nz : (z >= g.nz ? z - g.nz : z);
  return x + int64_t(g.nx) * (y + int64_t(g.ny) * z);
}

// perturbation weights B_a by |c|^2 shell; sum B = cs2, sum B c c = cs2 I
template <class L>
__host__ __device__ constexpr double cg_B(int a) {
  const int c2 = L::cx(a) * L::cx(a) + L::cy(a) * L::cy(a) + L::cz(a) * L::cz(a);
  if (L::ID == LB_D2Q9) return c2 == 0 ? -4.0 / 27.0 : (c2 == 1 ? 2.0 / 27.0 : 5.0 / 108.0);
  return c2 == 0 ? -2.0 / 9.0 : (c2 == 1 ? 1.0 / 54.0 : 1.0 / 27.0);
}

template <class L, class S, class R>
__global__ void __launch_bounds__(kCgThreads) cg_moments_kernel(CgGeom g, const S* __restrict__ fr,
                                                                  const S* __restrict__ fb, Phys<R> ph, R half_rho0,
                                                                  R beta, R* __restrict__ fld) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < g.n; i += int64_t(gridDim.x) * blockDim.x) {
    R gt[L::Q];
    R sr = R(0), sb = R(0);
    static_for<0, L::Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      const R r = load_as<S, R>(fr[a * g.n + i]), b = load_as<S, R>(fb[a * g.n + i]);
      sr = sr + r;
      sb = sb + b;
      gt[a] = r + b;
    });
    Mom<R> m;
    moments<L, R, false>(gt, ph, m);
    Coef<R> k;
    coeffs<L, R, false>(m, ph, k);
    fld[(F_COEF + 0) * g.n + i] = k.A;
    for (int al = 0; al < 3; ++al) {
      fld[(F_COEF + 1 + al) * g.n + i] = k.B[al];
      fld[(F_COEF + 4 + al) * g.n + i] = k.C[al];
      fld[(F_COEF + 7 + al) * g.n + i] = k.C2[al];
    }
    const R rr = sr + half_rho0, rb = sb + half_rho0, rho = rr + rb;
    fld[F_CR * g.n + i] = rr / rho;
    fld[F_CRB * g.n + i] = beta * rr * rb / rho;
    fld[F_PHI * g.n + i] = (rr - rb) / rho;
  }
}

// near-contact parameters of the gradient launch
template <class R>
struct CgNci {
  R amp, bulk, half_rho0;  // A, -1 + eps, rho0 / 2
  int h;
};

template <class L, class S, class R, bool NCI>
__global__ void __launch_bounds__(kCgThreads) cg_gradient_kernel(CgGeom g, R* __restrict__ fld,
                                                                  const S* __restrict__ fr,
                                                                  const S* __restrict__ fb, Phys<R> ph,
                                                                  CgNci<R> nci) {
  const R* phi = fld + F_PHI * g.n;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < g.n; i += int64_t(gridDim.x) * blockDim.x) {
    const int x = int(i % g.nx), y = int((i / g.nx) % g.ny), z = int(i / (int64_t(g.nx) * g.ny));
    R gv[3] = {R(0), R(0), R(0)};
    static_for<1, L::Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      const R p = phi[cg_wrap_index(g, x + L::cx(a), y + L::cy(a), z + L::cz(a))];
      constexpr R w = R(weight<L>(a));
      if constexpr (L::cx(a) != 0) gv[0] = fma_r(R(L::cx(a)) * w, p, gv[0]);
      if constexpr (L::cy(a) != 0) gv[1] = fma_r(R(L::cy(a)) * w, p, gv[1]);
      if constexpr (L::cz(a) != 0) gv[2] = fma_r(R(L::cz(a)) * w, p, gv[2]);
    });
    R g2 = R(0);
    for (int al = 0; al < 3; ++al) {
      gv[al] = gv[al] * R(3);  // 1 / cs2
      g2 = fma_r(gv[al], gv[al], g2);
    }
    const R gn = sqrt(g2);
    fld[F_GN * g.n + i] = gn;
    for (int al = 0; al < 3; ++al) fld[(F_N + al) * g.n + i] = gn > R(0) ? gv[al] / gn : R(0);
    if constexpr (NCI) {
      bool flag = false;
      if (phi[i] > nci.bulk) {
        const int h = nci.h;
        static_for<1, L::Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          constexpr int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
          const R p1 = phi[cg_wrap_index(g, x - h * cx, y - h * cy, z - h * cz)];
          const R p2 = phi[cg_wrap_index(g, x - 2 * h * cx, y - 2 * h * cy, z - 2 * h * cz)];
          flag = flag || (p1 < nci.bulk && p2 > nci.bulk);
        });
      }
      if (flag && gn > R(0)) {
        R gt[L::Q];
        R sr = R(0);
        static_for<0, L::Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          const R r = load_as<S, R>(fr[a * g.n + i]), b = load_as<S, R>(fb[a * g.n + i]);
          sr = sr + r;
          gt[a] = r + b;
        });
        const R rr = sr + nci.half_rho0;  // rho_R
        Phys<R> pf = ph;
        for (int al = 0; al < 3; ++al) {
          pf.F[al] = nci.amp * rr * (gv[al] / gn);
          pf.hF[al] = R(0.5) * pf.F[al];
        }
        Mom<R> m;
        moments<L, R, true>(gt, pf, m);
        Coef<R> k;
        coeffs<L, R, true>(m, pf, k);
        fld[(F_COEF + 0) * g.n + i] = k.A;
        for (int al = 0; al < 3; ++al) {
          fld[(F_COEF + 1 + al) * g.n + i] = k.B[al];
          fld[(F_COEF + 4 + al) * g.n + i] = k.C[al];
          fld[(F_COEF + 7 + al) * g.n + i] = k.C2[al];
        }
      }
    }
  }
}

template <class L, class S, class R>
__global__ void __launch_bounds__(kCgThreads) cg_rebuild_kernel(CgGeom g, const R* __restrict__ fld, R pert_k,
                                                                 R half_rho0, S* __restrict__ fr,
                                                                 S* __restrict__ fb) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < g.n; i += int64_t(gridDim.x) * blockDim.x) {
    const int x = int(i % g.nx), y = int((i / g.nx) % g.ny), z = int(i / (int64_t(g.nx) * g.ny));
    static_for<0, L::Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      constexpr int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
      const int64_t s = cg_wrap_index(g, x - cx, y - cy, z - cz);  // upstream node
      Coef<R> k;
      k.A = fld[(F_COEF + 0) * g.n + s];
      for (int al = 0; al < 3; ++al) {
        k.B[al] = fld[(F_COEF + 1 + al) * g.n + s];
        k.C[al] = fld[(F_COEF + 4 + al) * g.n + s];
        k.C2[al] = fld[(F_COEF + 7 + al) * g.n + s];
      }
      constexpr R w = R(weight<L>(a));
      const R gpost = post<L, R, a>(k) + w * (R(2) * half_rho0);  // unshifted relaxed total population
      const R gn = fld[F_GN * g.n + s];
      R cn = R(0);  // c_a . n
      if constexpr (cx != 0) cn = fma_r(R(cx), fld[(F_N + 0) * g.n + s], cn);
      if constexpr (cy != 0) cn = fma_r(R(cy), fld[(F_N + 1) * g.n + s], cn);
      if constexpr (cz != 0) cn = fma_r(R(cz), fld[(F_N + 2) * g.n + s], cn);
      constexpr R B = R(cg_B<L>(a));
      const R gstar = fma_r(pert_k * gn, fma_r(w * cn, cn, -B), gpost);
      constexpr int c2 = cx * cx + cy * cy + cz * cz;
      constexpr R inv_len = c2 == 0 ? R(0) : (c2 == 1 ? R(1) : (c2 == 2 ? R(0.70710678118654752440) :
                                                                     R(0.57735026918962576451)));
      const R rec = fld[F_CRB * g.n + s] * (w * (cn * inv_len));
      const R fred = fma_r(fld[F_CR * g.n + s], gstar, rec);
      const R fblue = gstar - fred;
      fr[a * g.n + i] = store_as<S, R>(fred - w * half_rho0);
      fb[a * g.n + i] = store_as<S, R>(fblue - w * half_rho0);
    });
  }
}

// f_k = (rho_k / rho) f^eq(rho, u) (FP64), stored shifted by t_a rho0 / 2
template <class L, class S>
__global__ void cg_init_kernel(CgGeom g, const double* __restrict__ rr, const double* __restrict__ rb,
                               const double* __restrict__ u, int d, double rho0, S* __restrict__ fr,
                               S* __restrict__ fb) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < g.n; i += int64_t(gridDim.x) * blockDim.x) {
    double uu[3] = {0, 0, 0};
    if (u) {
      uu[0] = u[i];
      if (d == 2) uu[2] = u[g.n + i];  // user y is internal z in 2D
      else {
        uu[1] = u[g.n + i];
        uu[2] = u[2 * g.n + i];
      }
    }
    const double rho = rr[i] + rb[i], usq = uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2];
    static_for<0, L::Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      const double cu = L::cx(a) * uu[0] + L::cy(a) * uu[1] + L::cz(a) * uu[2];
      const double w = weight<L>(a);
      const double feq = w * (rho + rho0 * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
      // S is float or double here: the conversion rounds to nearest
      fr[a * g.n + i] = static_cast<S>(rr[i] / rho * feq - 0.5 * w * rho0);
      fb[a * g.n + i] = static_cast<S>(rb[i] / rho * feq - 0.5 * w * rho0);
    });
  }
}

template <class L, class S, class R>
__global__ void cg_get_kernel(CgGeom g, const S* __restrict__ fs, double rho0, double* __restrict__ f) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < g.n; i += int64_t(gridDim.x) * blockDim.x)
    static_for<0, L::Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      f[a * g.n + i] = double(load_as<S, R>(fs[a * g.n + i])) + 0.5 * weight<L>(a) * rho0;
    });
}

template <class L, class S, class R>
__global__ void cg_set_kernel(CgGeom g, const double* __restrict__ f, double rho0, S* __restrict__ fs) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < g.n; i += int64_t(gridDim.x) * blockDim.x)
    static_for<0, L::Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      fs[a * g.n + i] = store_as<S, R>(R(f[a * g.n + i] - 0.5 * weight<L>(a) * rho0));
    });
}

template <class L, class S, class R>
__global__ void cg_fields_kernel(CgGeom g, const S* __restrict__ fr, const S* __restrict__ fb, double rho0,
                                 int d, double* __restrict__ rr, double* __restrict__ rb, double* __restrict__ u) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < g.n; i += int64_t(gridDim.x) * blockDim.x) {
    double sr = 0.0, sb = 0.0, j[3] = {0, 0, 0};
    static_for<0, L::Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      const double r = double(load_as<S, R>(fr[a * g.n + i])), b = double(load_as<S, R>(fb[a * g.n + i]));
      sr += r;
      sb += b;
      j[0] += L::cx(a) * (r + b);
      j[1] += L::cy(a) * (r + b);
      j[2] += L::cz(a) * (r + b);
    });
    if (rr) rr[i] = sr + 0.5 * rho0;
    if (rb) rb[i] = sb + 0.5 * rho0;
    if (u) {
      u[i] = j[0] / rho0;
      if (d == 2) u[g.n + i] = j[2] / rho0;
      else {
        u[g.n + i] = j[1] / rho0;
        u[2 * g.n + i] = j[2] / rho0;
      }
    }
  }
}

int grid_of(int64_t n) {
  int64_t b = (n + kCgThreads - 1) / kCgThreads;
  return int(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

int rc_of(cudaError_t e) { return e == cudaSuccess ? LB_OK : (e == cudaErrorMemoryAllocation ? LB_E_NOMEM : LB_E_CUDA); }

template <class F>
bool cg_dispatch(int lattice, int storage, F&& f) {
  if (lattice != LB_D2Q9 && lattice != LB_D3Q19) return false;
  if (storage != LB_F64 && storage != LB_F32) return false;
  return dispatch_lattice(lattice, [&](auto Lt) {
    if (storage == LB_F64) f(Lt, type_tag<double>{}, type_tag<double>{});
    else f(Lt, type_tag<float>{}, type_tag<float>{});
  });
}

}  // namespace
}  // namespace lbgb

struct lb_cg {
  int lattice, q, d, storage;
  int64_t dims[3];
  lbgb::CgGeom g;
  double tau, sigma, beta, rho0;
  cudaStream_t stream;
  bool own_stream;
  int device;
  size_t es, rs;  // storage and arithmetic element sizes
  void* fr;
  void* fb;
  void* fld;
  int64_t steps_done;
  double nci_amp, nci_eps;  // near-contact interactions: off while nci_amp == 0
  int nci_h;
};

using namespace lbgb;

namespace {

struct CgDev {
  int prev = -1;
  explicit CgDev(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) cudaSetDevice(dev);
  }
  ~CgDev() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// stage an FP64 buffer to the device (host input) or use it (device input)
int cg_stage(lb_cg* c, const double* src, size_t count, int on_device, double** out, bool* owned) {
  *out = nullptr;
  *owned = false;
  if (!src) return LB_OK;
  if (on_device) {
    *out = const_cast<double*>(src);
    return LB_OK;
  }
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(out), count * sizeof(double), c->stream);
  if (e != cudaSuccess) return rc_of(e);
  *owned = true;
  return rc_of(cudaMemcpyAsync(*out, src, count * sizeof(double), cudaMemcpyHostToDevice, c->stream));
}

}  // namespace

extern "C" {

int lb_cg_create(int32_t lattice, const int64_t dims[3], double tau, double sigma, double beta, int32_t storage,
                 void* stream, lb_cg** out) {
  if (!out || !dims) return LB_E_INVAL;
  *out = nullptr;
  if (lattice != LB_D2Q9 && lattice != LB_D3Q19) return LB_E_UNSUPPORTED;
  if (storage != LB_F64 && storage != LB_F32) return LB_E_UNSUPPORTED;
  const int d = lattice == LB_D2Q9 ? 2 : 3;
  for (int k = 0; k < 3; ++k)
    if (dims[k] < 1 || dims[k] > (int64_t(1) << 30)) return LB_E_INVAL;
  if (d == 2 && dims[2] != 1) return LB_E_INVAL;
  if (!(tau > 0.5) || !(tau < 1e6) || !(sigma >= 0.0) || !(beta >= 0.0) || !(beta <= 1.0)) return LB_E_INVAL;
  lb_cg* c = new (std::nothrow) lb_cg();
  if (!c) return LB_E_NOMEM;
  c->lattice = lattice;
  c->q = lattice == LB_D2Q9 ? 9 : 19;
  c->d = d;
  c->storage = storage;
  for (int k = 0; k < 3; ++k) c->dims[k] = dims[k];
  c->g.nx = int(dims[0]);
  c->g.ny = d == 2 ? 1 : int(dims[1]);
  c->g.nz = d == 2 ? int(dims[1]) : int(dims[2]);
  c->g.n = dims[0] * dims[1] * dims[2];
  c->tau = tau;
  c->sigma = sigma;
  c->beta = beta;
  c->rho0 = 1.0;
  c->es = c->rs = storage == LB_F64 ? 8 : 4;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return LB_E_CUDA;
  }
  int rc = LB_OK;
  do {
    if (stream) {
      c->stream = static_cast<cudaStream_t>(stream);
    } else {
      if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { rc = LB_E_CUDA; break; }
      c->own_stream = true;
    }
    const size_t pop = size_t(c->q) * size_t(c->g.n) * c->es;
    if ((rc = rc_of(cudaMalloc(&c->fr, pop))) != LB_OK) break;
    if ((rc = rc_of(cudaMalloc(&c->fb, pop))) != LB_OK) break;
    if ((rc = rc_of(cudaMalloc(&c->fld, size_t(kCgFields) * size_t(c->g.n) * c->rs))) != LB_OK) break;
    // an even mixture at rest: each colour t_a rho0 / 2, i.e. zero shifted values
    if ((rc = rc_of(cudaMemsetAsync(c->fr, 0, pop, c->stream))) != LB_OK) break;
    if ((rc = rc_of(cudaMemsetAsync(c->fb, 0, pop, c->stream))) != LB_OK) break;
    rc = rc_of(cudaStreamSynchronize(c->stream));
  } while (false);
  if (rc != LB_OK) {
    lb_cg_destroy(c);
    return rc;
  }
  *out = c;
  return LB_OK;
}

int lb_cg_init(lb_cg* c, const double* rho_r, const double* rho_b, const double* u, int32_t on_device) {
  if (!c || !rho_r || !rho_b) return LB_E_INVAL;
  CgDev guard(c->device);
  double *dr, *db, *du;
  bool o1, o2, o3;
  const size_t N = size_t(c->g.n);
  int rc = cg_stage(c, rho_r, N, on_device, &dr, &o1);
  if (rc == LB_OK) rc = cg_stage(c, rho_b, N, on_device, &db, &o2);
  else o2 = false, db = nullptr;
  if (rc == LB_OK) rc = cg_stage(c, u, N * c->d, on_device, &du, &o3);
  else o3 = false, du = nullptr;
  if (rc == LB_OK) {
    cg_dispatch(c->lattice, c->storage, [&](auto Lt, auto St, auto) {
      using L = decltype(Lt);
      using S = typename decltype(St)::type;
      cg_init_kernel<L, S><<<grid_of(c->g.n), kCgThreads, 0, c->stream>>>(
          c->g, dr, db, du, c->d, c->rho0, static_cast<S*>(c->fr), static_cast<S*>(c->fb));
    });
    rc = rc_of(cudaGetLastError());
  }
  if (o1) cudaFreeAsync(dr, c->stream);
  if (o2) cudaFreeAsync(db, c->stream);
  if (o3) cudaFreeAsync(du, c->stream);
  const int rc2 = rc_of(cudaStreamSynchronize(c->stream));
  return rc != LB_OK ? rc : rc2;
}

int lb_cg_set_populations(lb_cg* c, const double* fr, const double* fb, int32_t on_device) {
  if (!c || !fr || !fb) return LB_E_INVAL;
  CgDev guard(c->device);
  const size_t cnt = size_t(c->q) * size_t(c->g.n);
  int rc = LB_OK;
  for (int k = 0; k < 2 && rc == LB_OK; ++k) {
    double* d;
    bool owned;
    rc = cg_stage(c, k == 0 ? fr : fb, cnt, on_device, &d, &owned);
    if (rc != LB_OK) break;
    cg_dispatch(c->lattice, c->storage, [&](auto Lt, auto St, auto Rt) {
      using L = decltype(Lt);
      using S = typename decltype(St)::type;
      using R = typename decltype(Rt)::type;
      cg_set_kernel<L, S, R><<<grid_of(c->g.n), kCgThreads, 0, c->stream>>>(c->g, d, c->rho0,
                                                                            static_cast<S*>(k == 0 ? c->fr : c->fb));
    });
    rc = rc_of(cudaGetLastError());
    if (owned) cudaFreeAsync(d, c->stream);
  }
  const int rc2 = rc_of(cudaStreamSynchronize(c->stream));
  return rc != LB_OK ? rc : rc2;
}

int lb_cg_get_populations(lb_cg* c, double* fr, double* fb, int32_t on_device) {
  if (!c || (!fr && !fb)) return LB_E_INVAL;
  CgDev guard(c->device);
  const size_t cnt = size_t(c->q) * size_t(c->g.n);
  int rc = LB_OK;
  for (int k = 0; k < 2 && rc == LB_OK; ++k) {
    double* dst = k == 0 ? fr : fb;
    if (!dst) continue;
    double* d = dst;
    if (!on_device) {
      rc = rc_of(cudaMallocAsync(reinterpret_cast<void**>(&d), cnt * sizeof(double), c->stream));
      if (rc != LB_OK) break;
    }
    cg_dispatch(c->lattice, c->storage, [&](auto Lt, auto St, auto Rt) {
      using L = decltype(Lt);
      using S = typename decltype(St)::type;
      using R = typename decltype(Rt)::type;
      cg_get_kernel<L, S, R><<<grid_of(c->g.n), kCgThreads, 0, c->stream>>>(
          c->g, static_cast<const S*>(k == 0 ? c->fr : c->fb), c->rho0, d);
    });
    rc = rc_of(cudaGetLastError());
    if (!on_device) {
      if (rc == LB_OK) rc = rc_of(cudaMemcpyAsync(dst, d, cnt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      cudaFreeAsync(d, c->stream);
    }
  }
  const int rc2 = rc_of(cudaStreamSynchronize(c->stream));
  return rc != LB_OK ? rc : rc2;
}

int lb_cg_step(lb_cg* c, int64_t n) {
  if (!c || n < 0) return LB_E_INVAL;
  CgDev guard(c->device);
  Geometry geo{};
  geo.tau = c->tau;
  geo.rho0 = c->rho0;
  bool ok = true;
  for (int64_t s = 0; s < n && ok; ++s) {
    ok = cg_dispatch(c->lattice, c->storage, [&](auto Lt, auto St, auto Rt) {
      using L = decltype(Lt);
      using S = typename decltype(St)::type;
      using R = typename decltype(Rt)::type;
      const Phys<R> ph = make_phys<R>(geo);
      R* fld = static_cast<R*>(c->fld);
      const int grid = grid_of(c->g.n);
      cg_moments_kernel<L, S, R><<<grid, kCgThreads, 0, c->stream>>>(
          c->g, static_cast<const S*>(c->fr), static_cast<const S*>(c->fb), ph, R(0.5 * c->rho0), R(c->beta), fld);
      const CgNci<R> nci{R(c->nci_amp), R(-1.0 + c->nci_eps), R(0.5 * c->rho0), c->nci_h};
      if (c->nci_amp != 0.0)
        cg_gradient_kernel<L, S, R, true><<<grid, kCgThreads, 0, c->stream>>>(
            c->g, fld, static_cast<const S*>(c->fr), static_cast<const S*>(c->fb), ph, nci);
      else
        cg_gradient_kernel<L, S, R, false><<<grid, kCgThreads, 0, c->stream>>>(c->g, fld, nullptr, nullptr, ph, nci);
      cg_rebuild_kernel<L, S, R><<<grid, kCgThreads, 0, c->stream>>>(
          c->g, fld, R(2.25 * c->sigma / c->tau), R(0.5 * c->rho0), static_cast<S*>(c->fr), static_cast<S*>(c->fb));
    });
    if (cudaGetLastError() != cudaSuccess) return LB_E_CUDA;
    c->steps_done++;
  }
  return LB_OK;
}

int lb_cg_fields(lb_cg* c, double* rho_r, double* rho_b, double* u, int32_t on_device) {
  if (!c || (!rho_r && !rho_b && !u)) return LB_E_INVAL;
  CgDev guard(c->device);
  const size_t N = size_t(c->g.n);
  double* tmp = nullptr;
  double *dr = rho_r, *db = rho_b, *du = u;
  if (!on_device) {
    int rc = rc_of(cudaMallocAsync(reinterpret_cast<void**>(&tmp), (2 + c->d) * N * sizeof(double), c->stream));
    if (rc != LB_OK) return rc;
    dr = rho_r ? tmp : nullptr;
    db = rho_b ? tmp + N : nullptr;
    du = u ? tmp + 2 * N : nullptr;
  }
  cg_dispatch(c->lattice, c->storage, [&](auto Lt, auto St, auto Rt) {
    using L = decltype(Lt);
    using S = typename decltype(St)::type;
    using R = typename decltype(Rt)::type;
    cg_fields_kernel<L, S, R><<<grid_of(c->g.n), kCgThreads, 0, c->stream>>>(
        c->g, static_cast<const S*>(c->fr), static_cast<const S*>(c->fb), c->rho0, c->d, dr, db, du);
  });
  int rc = rc_of(cudaGetLastError());
  if (!on_device) {
    if (rc == LB_OK && rho_r) rc = rc_of(cudaMemcpyAsync(rho_r, dr, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (rc == LB_OK && rho_b) rc = rc_of(cudaMemcpyAsync(rho_b, db, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (rc == LB_OK && u)
      rc = rc_of(cudaMemcpyAsync(u, du, c->d * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    cudaFreeAsync(tmp, c->stream);
  }
  const int rc2 = rc_of(cudaStreamSynchronize(c->stream));
  return rc != LB_OK ? rc : rc2;
}

int lb_cg_set_nci(lb_cg* c, double amplitude, double eps, int32_t h) {
  if (!c || !std::isfinite(amplitude) || amplitude < 0.0 || !(eps > 0.0) || !(eps < 2.0) || h < 1) return LB_E_INVAL;
  // the sampled points lie up to 2h nodes away along every moving axis: one
  // periodic wrap must reach them
  const int lim = c->d == 2 ? std::min(c->g.nx, c->g.nz) : std::min(c->g.nx, std::min(c->g.ny, c->g.nz));
  if (2 * int64_t(h) > lim) return LB_E_INVAL;
  c->nci_amp = amplitude;
  c->nci_eps = eps;
  c->nci_h = h;
  return LB_OK;
}

int lb_cg_sync(lb_cg* c) {
  if (!c) return LB_E_INVAL;
  CgDev guard(c->device);
  return rc_of(cudaStreamSynchronize(c->stream));
}

void lb_cg_destroy(lb_cg* c) {
  if (!c) return;
  CgDev guard(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->fr) cudaFree(c->fr);
  if (c->fb) cudaFree(c->fb);
  if (c->fld) cudaFree(c->fld);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // extern "C"
