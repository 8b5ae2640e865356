// lb_aux.cu -- state conversion, readout and FP64 reductions.
//
// These kernels move data between the caller's canonical FP64 arrays and the
// internal shifted population array ft_a = f_a - t_a rho0 (row pitch padded to
// a multiple of 32 elements), and compute the diagnostics of the ABI.  Every
// node is handled by one thread; 64-bit indices throughout.
#include <cuda_runtime.h>

#include <type_traits>

#include "lb_dispatch.cuh"

namespace lbgb {
namespace {

constexpr int kThreads = 256;
constexpr int kRedBlocks = 1024;  // fixed: the reduction order never depends on the GPU

struct Layout {
  int nx;          // internal x extent (= user x extent)
  int64_t rows;    // ny * nz internal rows
  int64_t pitch;
  int64_t vol;
  int64_t n;       // nx * rows
};

inline Layout layout_of(const Geometry& g) {
  Layout l;
  l.nx = g.nx;
  l.rows = static_cast<int64_t>(g.ny) * g.nz;
  l.pitch = g.pitch;
  l.vol = g.vol;
  l.n = static_cast<int64_t>(g.nx) * l.rows;
  return l;
}

__device__ __forceinline__ int64_t ioff(const Layout& l, int64_t idx) {
  const int64_t x = idx % l.nx;
  const int64_t r = idx / l.nx;
  return x + r * l.pitch;
}

// user vector component k -> internal axis
template <class L>
__device__ __forceinline__ constexpr int user_axis(int k) {
  return (L::D == 2 && k == 1) ? 2 : k;
}

template <class L, class S, class R>
__global__ void set_pop_kernel(Layout l, const double* __restrict__ f, S* __restrict__ ft, double rho0) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < l.n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = ioff(l, idx);
    static_for<0, L::Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      const double v = f[a * l.n + idx] - weight<L>(a) * rho0;
      ft[a * l.vol + o] = store_as<S, R>(static_cast<R>(v));
    });
  }
}

template <class L, class S, class R>
__global__ void get_pop_kernel(Layout l, const S* __restrict__ ft, double* __restrict__ f, double rho0) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < l.n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = ioff(l, idx);
    static_for<0, L::Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      f[a * l.n + idx] = static_cast<double>(load_as<S, R>(ft[a * l.vol + o])) + weight<L>(a) * rho0;
    });
  }
}

// f = f^eq(rho, u) + t_a (cc - cs2 I):Pi/(2 cs2^2) - t_a c.F/(2 cs2), stored
// shifted.  rho may be null (uniform rho_u), u may be null (uniform u_u).
template <class L, class S, class R>
// nodes [n0, n1); input node idx is element idx - n0 of each component, and
// components lie cs elements apart
__global__ void init_kernel(Layout l, S* __restrict__ ft, double rho0, const double* __restrict__ rho,
                            const double* __restrict__ u, const double* __restrict__ pineq, double rho_u,
                            double ux_u, double uy_u, double uz_u, double Fx, double Fy, double Fz, int64_t n0,
                            int64_t n1, int64_t cs) {
  for (int64_t idx = n0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n1;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = ioff(l, idx);
    const int64_t k0 = idx - n0;
    const double r = rho ? rho[k0] : rho_u;
    double ui[3] = {0.0, 0.0, 0.0};
    const double uu[3] = {ux_u, uy_u, uz_u};
    for (int k = 0; k < L::D; ++k) ui[user_axis<L>(k)] = u ? u[k * cs + k0] : uu[k];
    double P[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (pineq) {
      if (L::D == 2) {
        P[0][0] = pineq[0 * cs + k0];
        P[2][2] = pineq[1 * cs + k0];
        P[0][2] = P[2][0] = pineq[2 * cs + k0];
      } else {
        P[0][0] = pineq[0 * cs + k0];
        P[1][1] = pineq[1 * cs + k0];
        P[2][2] = pineq[2 * cs + k0];
        P[0][1] = P[1][0] = pineq[3 * cs + k0];
        P[0][2] = P[2][0] = pineq[4 * cs + k0];
        P[1][2] = P[2][1] = pineq[5 * cs + k0];
      }
    }
    // the shifted populations are computed in the kernels' arithmetic type
    // R (FP32 for FP32 / FP16 / BF16 storage, FP64 for FP64): they are
    // deviations of order u, so R's rounding is that of the storage; the
    // density deviation is formed in FP64 first
    using T = R;
    const T drho = static_cast<T>(r - rho0);
    const T rho0t = static_cast<T>(rho0);
    const T Fi[3] = {static_cast<T>(Fx), static_cast<T>(Fy), static_cast<T>(Fz)};
    T ut[3], Pt[3][3];
    for (int k = 0; k < 3; ++k) {
      ut[k] = static_cast<T>(ui[k]);
      for (int m = 0; m < 3; ++m) Pt[k][m] = static_cast<T>(P[k][m]);
    }
    T usq = T(0), trP = T(0);
    for (int k = 0; k < 3; ++k) {
      usq += ut[k] * ut[k];
      trP += Pt[k][k];
    }
    // f_a = t_a [drho + rho0 (3 c.u + 4.5 (c.u)^2 - 1.5 u.u) + 4.5 (c.P.c - tr P / 3)
    //           - 1.5 c.F]: a velocity pair {a, abar} shares the even part
    // and takes the odd part (c.u, c.F) with opposite signs
    const T ev0 = drho - T(1.5) * rho0t * usq - T(1.5) * trP;
    ft[0 * l.vol + o] = store_as<S, R>(static_cast<R>(T(weight<L>(0)) * ev0));
    static_for<0, n_pairs<L>()>([&](auto P_) {
      constexpr int a = pair_first<L>(decltype(P_)::value);
      constexpr int b = L::opp(a);
      // c.u, c.F and c.P.c with the components of c (0 or +-1) applied at
      // compile time
      T cu = T(0), cF = T(0), cPc = T(0);
      static_for<0, 3>([&](auto I_) {
        constexpr int i = decltype(I_)::value;
        constexpr int ci = comp<L>(i, a);
        if constexpr (ci != 0) {
          cu += ci > 0 ? ut[i] : -ut[i];
          cF += ci > 0 ? Fi[i] : -Fi[i];
        }
        static_for<0, 3>([&](auto J_) {
          constexpr int j = decltype(J_)::value;
          constexpr int cc = ci * comp<L>(j, a);
          if constexpr (cc != 0) cPc += cc > 0 ? Pt[i][j] : -Pt[i][j];
        });
      });
      const T w = T(weight<L>(a));
      const T even = w * (ev0 + T(4.5) * (rho0t * cu * cu + cPc));
      const T odd = w * (T(3) * rho0t * cu - T(1.5) * cF);
      ft[a * l.vol + o] = store_as<S, R>(static_cast<R>(even + odd));
      ft[b * l.vol + o] = store_as<S, R>(static_cast<R>(even - odd));
    });
  }
}

// Per-node sums drho = sum ft_a and j = sum ft_a c_a of the stored state,
// returned in FP64.  FP64 storage adds in FP64.  The FP32 arithmetic types
// (FP32, FP16, BF16 storage) add in FP32 and carry the rounding error of
// every addition in a second FP32 accumulator (the error-free two-sum; the
// cascaded summation of Ogita, Rump and Oishi), so that hi + lo is the sum to
// about twice FP32's precision; only the final pairs are converted to FP64.
// GB300 converts and adds FP64 at a small fraction of its FP32 rate, which
// made the plain FP64 path the bound of these kernels.
struct Sum2 {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
  }
  __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

template <class L, class S, class R>
__device__ __forceinline__ void node_sums(const S* __restrict__ ft, int64_t vol, int64_t o, double& dr, double (&j)[3],
                                          bool& bad) {
  if constexpr (std::is_same<R, double>::value) {
    dr = 0.0;
    j[0] = j[1] = j[2] = 0.0;
    static_for<0, L::Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      const double v = load_as<S, R>(ft[a * vol + o]);
      bad |= !isfinite(v);
      constexpr int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
      dr += v;
      if constexpr (cx != 0) j[0] += cx > 0 ? v : -v;  // zero terms skipped: the sums are unchanged
      if constexpr (cy != 0) j[1] += cy > 0 ? v : -v;
      if constexpr (cz != 0) j[2] += cz > 0 ? v : -v;
    });
  } else {
    Sum2 sr, sj[3];
    static_for<0, L::Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      const float v = load_as<S, R>(ft[a * vol + o]);
      bad |= !isfinite(v);
      constexpr int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
      sr.add(v);
      if constexpr (cx != 0) sj[0].add(cx > 0 ? v : -v);
      if constexpr (cy != 0) sj[1].add(cy > 0 ? v : -v);
      if constexpr (cz != 0) sj[2].add(cz > 0 ? v : -v);
    });
    dr = sr.value();
    for (int k = 0; k < 3; ++k) j[k] = sj[k].value();
  }
}

template <class L, class S, class R>
// nodes [n0, n1) into element idx - n0 of each output component (cs apart)
__global__ void moments_kernel(Layout l, const S* __restrict__ ft, double rho0, double Fx, double Fy, double Fz,
                               double* __restrict__ rho, double* __restrict__ u, int64_t n0, int64_t n1,
                               int64_t cs) {
  for (int64_t idx = n0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n1;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = ioff(l, idx);
    double dr, j[3];
    bool bad = false;
    node_sums<L, S, R>(ft, l.vol, o, dr, j, bad);
    if (rho) rho[idx - n0] = rho0 + dr;
    if (u) {
      const double Fi[3] = {Fx, Fy, Fz};
      for (int k = 0; k < L::D; ++k) {
        const int ax = user_axis<L>(k);
        // x / 1 is x exactly: the common rho0 = 1 skips the FP64 division
        const double v = j[ax] + 0.5 * Fi[ax];
        u[k * cs + (idx - n0)] = rho0 == 1.0 ? v : v / rho0;
      }
    }
  }
}

// region [lo, lo + size) in internal coordinates -> out [q][sz][sy][sx]
template <class L, class S, class R>
__global__ void region_kernel(Layout l, int ny, const S* __restrict__ ft, double rho0, int64_t x0, int64_t y0,
                              int64_t z0, int64_t sx, int64_t sy, int64_t sz, double* __restrict__ out) {
  const int64_t n = sx * sy * sz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = x0 + i % sx;
    const int64_t y = y0 + (i / sx) % sy;
    const int64_t z = z0 + i / (sx * sy);
    const int64_t o = x + l.pitch * (y + (int64_t)ny * z);
    static_for<0, L::Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      out[a * n + i] = static_cast<double>(load_as<S, R>(ft[a * l.vol + o])) + weight<L>(a) * rho0;
    });
  }
}

// Per-block FP64 partials: [mass, jx, jy, jz, sum |u - u_prev|^2, sum |u|^2,
// non-finite count]; u in internal axes.  Fixed grid + tree order.
constexpr int kRedFields = 7;

template <class L, class S, class R>
__global__ void __launch_bounds__(kThreads) reduce_kernel(Layout l, const S* __restrict__ ft, double rho0,
                                                          double Fx, double Fy, double Fz,
                                                          float* __restrict__ uprev, int residual,
                                                          double* __restrict__ partial) {
  double acc[kRedFields] = {0, 0, 0, 0, 0, 0, 0};
  const double Fi[3] = {Fx, Fy, Fz};
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < l.n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = ioff(l, idx);
    double dr, j[3];
    bool bad = false;
    node_sums<L, S, R>(ft, l.vol, o, dr, j, bad);
    acc[0] += rho0 + dr;
    acc[1] += j[0];
    acc[2] += j[1];
    acc[3] += j[2];
    acc[6] += bad ? 1.0 : 0.0;
    if (residual) {
      for (int k = 0; k < 3; ++k) {
        const double vk = j[k] + 0.5 * Fi[k];
        const double uk = rho0 == 1.0 ? vk : vk / rho0;  // x / 1 is x exactly
        const double prev = static_cast<double>(uprev[k * l.n + idx]);
        acc[4] += (uk - prev) * (uk - prev);
        acc[5] += uk * uk;
        uprev[k * l.n + idx] = static_cast<float>(uk);
      }
    }
  }
  __shared__ double sh[kRedFields][kThreads];
  for (int k = 0; k < kRedFields; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < kRedFields; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < kRedFields; ++k) partial[k * kRedBlocks + blockIdx.x] = sh[k][0];
}

__global__ void reduce_final_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  // one block: fixed-order tree over the block partials
  __shared__ double sh[kThreads];
  for (int k = 0; k < kRedFields; ++k) {
    double a = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) a += partial[k * kRedBlocks + i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
    __syncthreads();
  }
}

int grid_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b > 152 * 64) b = 152 * 64;
  if (b < 1) b = 1;
  return static_cast<int>(b);
}

}  // namespace

cudaError_t aux_set_populations(lb_ctx* ctx, const double* f_dev) {
  const Layout l = layout_of(ctx->g);
  dispatch_lattice(ctx->lattice, [&](auto Lt) {
    using L = decltype(Lt);
    dispatch_storage(ctx->storage, [&](auto St, auto Rt) {
      using S = typename decltype(St)::type;
      using R = typename decltype(Rt)::type;
      set_pop_kernel<L, S, R><<<grid_for(l.n), kThreads, 0, ctx->stream>>>(l, f_dev, static_cast<S*>(ctx->f),
                                                                           ctx->g.rho0);
    });
  });
  return cudaGetLastError();
}

cudaError_t aux_get_populations(lb_ctx* ctx, double* f_dev) {
  const Layout l = layout_of(ctx->g);
  dispatch_lattice(ctx->lattice, [&](auto Lt) {
    using L = decltype(Lt);
    dispatch_storage(ctx->storage, [&](auto St, auto Rt) {
      using S = typename decltype(St)::type;
      using R = typename decltype(Rt)::type;
      get_pop_kernel<L, S, R><<<grid_for(l.n), kThreads, 0, ctx->stream>>>(
          l, static_cast<const S*>(ctx->f), f_dev, ctx->g.rho0);
    });
  });
  return cudaGetLastError();
}

static cudaError_t launch_init(lb_ctx* ctx, const double* rho, const double* u, const double* pineq, double rho_u,
                               const double uu[3], int64_t n0 = 0, int64_t n1 = -1, int64_t cs = -1) {
  const Layout l = layout_of(ctx->g);
  if (n1 < 0) n1 = l.n;
  if (cs < 0) cs = l.n;
  // the force is applied in internal axes inside the kernel
  const double* F = ctx->g.force;
  dispatch_lattice(ctx->lattice, [&](auto Lt) {
    using L = decltype(Lt);
    dispatch_storage(ctx->storage, [&](auto St, auto Rt) {
      using S = typename decltype(St)::type;
      using R = typename decltype(Rt)::type;
      init_kernel<L, S, R><<<grid_for(n1 - n0), kThreads, 0, ctx->stream>>>(
          l, static_cast<S*>(ctx->f), ctx->g.rho0, rho, u, pineq, rho_u, uu[0], uu[1], uu[2], F[0], F[1], F[2], n0,
          n1, cs);
    });
  });
  return cudaGetLastError();
}

cudaError_t aux_init_moments(lb_ctx* ctx, const double* rho, const double* u, const double* pineq) {
  const double zero[3] = {0, 0, 0};
  return launch_init(ctx, rho, u, pineq, ctx->g.rho0, zero);
}

cudaError_t aux_init_uniform(lb_ctx* ctx, double rho, const double u_user[3]) {
  return launch_init(ctx, nullptr, nullptr, nullptr, rho, u_user);
}

cudaError_t aux_init_moments_range(lb_ctx* ctx, const double* rho, const double* u, const double* pineq, int64_t n0,
                                   int64_t n1, int64_t cs) {
  const double zero[3] = {0, 0, 0};
  return launch_init(ctx, rho, u, pineq, ctx->g.rho0, zero, n0, n1, cs);
}

cudaError_t aux_moments(lb_ctx* ctx, double* rho, double* u) {
  return aux_moments_range(ctx, rho, u, 0, int64_t(ctx->g.nx) * ctx->g.ny * ctx->g.nz,
                           int64_t(ctx->g.nx) * ctx->g.ny * ctx->g.nz);
}

cudaError_t aux_moments_range(lb_ctx* ctx, double* rho, double* u, int64_t n0, int64_t n1, int64_t cs) {
  const Layout l = layout_of(ctx->g);
  const double* F = ctx->g.force;
  dispatch_lattice(ctx->lattice, [&](auto Lt) {
    using L = decltype(Lt);
    dispatch_storage(ctx->storage, [&](auto St, auto Rt) {
      using S = typename decltype(St)::type;
      using R = typename decltype(Rt)::type;
      moments_kernel<L, S, R><<<grid_for(n1 - n0), kThreads, 0, ctx->stream>>>(
          l, static_cast<const S*>(ctx->f), ctx->g.rho0, F[0], F[1], F[2], rho, u, n0, n1, cs);
    });
  });
  return cudaGetLastError();
}

cudaError_t aux_get_region(lb_ctx* ctx, const int64_t lo[3], const int64_t size[3], double* f_dev) {
  const Layout l = layout_of(ctx->g);
  // user box -> internal box (2D: user y is internal z)
  int64_t x0 = lo[0], y0 = lo[1], z0 = lo[2], sx = size[0], sy = size[1], sz = size[2];
  if (ctx->g.d == 2) {
    z0 = lo[1];
    sz = size[1];
    y0 = 0;
    sy = 1;
  }
  const int64_t n = sx * sy * sz;
  const int ny = ctx->g.ny;
  dispatch_lattice(ctx->lattice, [&](auto Lt) {
    using L = decltype(Lt);
    dispatch_storage(ctx->storage, [&](auto St, auto Rt) {
      using S = typename decltype(St)::type;
      using R = typename decltype(Rt)::type;
      region_kernel<L, S, R><<<grid_for(n), kThreads, 0, ctx->stream>>>(
          l, ny, static_cast<const S*>(ctx->f), ctx->g.rho0, x0, y0, z0, sx, sy, sz, f_dev);
    });
  });
  return cudaGetLastError();
}

cudaError_t aux_reduce_enqueue(lb_ctx* ctx, cudaStream_t stream, double* dev_out, bool residual) {
  const Layout l = layout_of(ctx->g);
  const double* F = ctx->g.force;
  cudaError_t err = cudaSuccess;
  if (residual && !ctx->d_uprev) {
    err = cudaMallocAsync(reinterpret_cast<void**>(&ctx->d_uprev), sizeof(float) * 3 * l.n, stream);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(ctx->d_uprev, 0, sizeof(float) * 3 * l.n, stream);
    if (err != cudaSuccess) return err;
  }
  dispatch_lattice(ctx->lattice, [&](auto Lt) {
    using L = decltype(Lt);
    dispatch_storage(ctx->storage, [&](auto St, auto Rt) {
      using S = typename decltype(St)::type;
      using R = typename decltype(Rt)::type;
      reduce_kernel<L, S, R><<<kRedBlocks, kThreads, 0, stream>>>(
          l, static_cast<const S*>(ctx->f), ctx->g.rho0, F[0], F[1], F[2], ctx->d_uprev, residual ? 1 : 0,
          ctx->d_red);
    });
  });
  reduce_final_kernel<<<1, kThreads, 0, stream>>>(ctx->d_red, kRedBlocks, dev_out);
  return cudaGetLastError();
}

cudaError_t aux_reduce(lb_ctx* ctx, double* host_out, bool residual) {
  double* dev_out = ctx->d_red + kRedFields * kRedBlocks;
  cudaError_t err = aux_reduce_enqueue(ctx, ctx->stream, dev_out, residual);
  if (err != cudaSuccess) return err;
  err = cudaMemcpyAsync(host_out, dev_out, sizeof(double) * kRedFields, cudaMemcpyDeviceToHost, ctx->stream);
  if (err != cudaSuccess) return err;
  return cudaStreamSynchronize(ctx->stream);
}

size_t reduce_scratch_doubles() { return static_cast<size_t>(kRedFields) * (kRedBlocks + 1); }

}  // namespace lbgb
