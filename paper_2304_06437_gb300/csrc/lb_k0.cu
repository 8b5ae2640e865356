// lb_k0.cu -- the paper's own two-kernel schedule (section 4), in pull form.
//
//   k0_moments : per node, read the populations and write the m = 1 + d +
//                d(d+1)/2 moment arrays (drho, u, Pi^neq) -- the "moments"
//                kernel of the paper's CUDA Fortran port.
//   k0_rebuild : per node y and direction a, rebuild the post-collision
//                population of the upstream node y - c_a from its moments
//                (Eq. LBexp with the Hermite-projected non-equilibrium part)
//                and write it to y -- the paper's "streamcoll" kernel written
//                as a pull, with its "bcs" kernel (halfway bounce-back, moving
//                wall term) fused in.
// The rebuild kernel never reads populations, so writing the single
// population array in place is race free.  Traffic per update is (2q + 2m)
// values (the paper's memory model); the fused scheme (lb_k1) removes the 2m.
#include <cuda_runtime.h>

#include "lb_dispatch.cuh"

namespace lbgb {
namespace {

template <class L>
constexpr int n_moments() { return 1 + L::D + L::D * (L::D + 1) / 2; }

// moment array slot -> field of Mom (internal axes; 2D uses x and z)
template <class L, class R>
__device__ __forceinline__ R& mom_field(Mom<R>& m, int k) {
  if constexpr (L::D == 3) {
    return k == 0 ? m.drho : k <= 3 ? m.u[k - 1] : m.pi[k - 4];
  } else {
    // drho, ux, uz, pi_xx, pi_zz, pi_xz
    return k == 0 ? m.drho : k == 1 ? m.u[0] : k == 2 ? m.u[2] : k == 3 ? m.pi[0] : k == 4 ? m.pi[2] : m.pi[4];
  }
}

template <class R>
struct K0Args {
  Phys<R> ph;
  int nx, ny, nz;
  int64_t pitch, vol;
  int per[3];
  R bb[27][8];
};

template <class L, class S, class R, bool FORCE>
__global__ void __launch_bounds__(256) k0_moments(K0Args<R> args, const S* __restrict__ ft, R* __restrict__ mom) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int z = blockIdx.z;
  if (x >= args.nx) return;
  const int64_t o = x + args.pitch * (y + (int64_t)args.ny * z);
  R f[L::Q];
  static_for<0, L::Q>([&](auto A_) {
    constexpr int a = decltype(A_)::value;
    f[a] = load_as<S, R>(ft[a * args.vol + o]);
  });
  Mom<R> m;
  moments<L, R, FORCE>(f, args.ph, m);
  static_for<0, n_moments<L>()>([&](auto K_) {
    constexpr int k = decltype(K_)::value;
    mom[k * args.vol + o] = mom_field<L, R>(m, k);
  });
}

template <class L, class S, class R, bool FORCE>
__global__ void __launch_bounds__(256) k0_rebuild(K0Args<R> args, const R* __restrict__ mom, S* __restrict__ ft) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int z = blockIdx.z;
  if (x >= args.nx) return;
  const int n[3] = {args.nx, args.ny, args.nz};
  const int p[3] = {x, y, z};
  const int64_t o = x + args.pitch * (y + (int64_t)args.ny * z);

  auto load_coef = [&](int64_t off, Coef<R>& k) {
    Mom<R> m;
    m.drho = R(0);
    for (int i = 0; i < 3; ++i) m.u[i] = R(0);
    for (int i = 0; i < 6; ++i) m.pi[i] = R(0);
    static_for<0, n_moments<L>()>([&](auto K_) {
      constexpr int kk = decltype(K_)::value;
      mom_field<L, R>(m, kk) = mom[kk * args.vol + off];
    });
    coeffs<L, R, FORCE>(m, args.ph, k);
  };

  Coef<R> own;
  load_coef(o, own);

  static_for<0, L::Q>([&](auto A_) {
    constexpr int a = decltype(A_)::value;
    constexpr int c[3] = {L::cx(a), L::cy(a), L::cz(a)};
    int s[3];
    int combo = 0;
    for (int ax = 0; ax < 3; ++ax) {
      s[ax] = p[ax] - c[ax];
      if (s[ax] < 0 || s[ax] >= n[ax]) {
        if (args.per[ax]) s[ax] = (s[ax] + n[ax]) % n[ax];
        else combo |= 1 << ax;
      }
    }
    R v;
    if (combo) {
      v = post<L, R, L::opp(a)>(own) + args.bb[a][combo];
    } else {
      Coef<R> k;
      load_coef(s[0] + args.pitch * (s[1] + (int64_t)args.ny * s[2]), k);
      v = post<L, R, a>(k);
    }
    ft[a * args.vol + o] = store_as<S, R>(v);
  });
}

template <class L, class S, class R, bool FORCE>
cudaError_t launch(lb_ctx* ctx) {
  const Geometry& g = ctx->g;
  K0Args<R> args;
  args.ph = make_phys<R>(g);
  args.nx = g.nx;
  args.ny = g.ny;
  args.nz = g.nz;
  args.pitch = g.pitch;
  args.vol = g.vol;
  for (int k = 0; k < 3; ++k) args.per[k] = g.per[k];
  make_bounce_terms<L, R>(g, args.bb);
  dim3 block(256);
  dim3 grid(div_up(g.nx, 256), g.ny, g.nz);
  R* mom = static_cast<R*>(ctx->aux);
  k0_moments<L, S, R, FORCE><<<grid, block, 0, ctx->stream>>>(args, static_cast<const S*>(ctx->f), mom);
  k0_rebuild<L, S, R, FORCE><<<grid, block, 0, ctx->stream>>>(args, mom, static_cast<S*>(ctx->f));
  return cudaGetLastError();
}

}  // namespace

size_t k0_aux_bytes(const Geometry& g, int storage) {
  const int m = 1 + g.d + g.d * (g.d + 1) / 2;
  const size_t rb = storage == LB_F64 ? sizeof(double) : sizeof(float);
  return static_cast<size_t>(m) * static_cast<size_t>(g.vol) * rb;
}

// The same two kernels on caller-provided FP64 buffers (shifted populations
// and moment arrays, both laid out with g.pitch / g.vol) on a given stream.
cudaError_t k0_step_buffers(const Geometry& g, double* ft, double* mom, cudaStream_t stream) {
  if (g.ny > 65535 || g.nz > 65535) return cudaErrorInvalidConfiguration;
  cudaError_t err = cudaErrorInvalidValue;
  dispatch_lattice(g.lattice, [&](auto Lt) {
    using L = decltype(Lt);
    auto go = [&](auto force_tag) {
      constexpr bool FORCE = decltype(force_tag)::value;
      K0Args<double> args;
      args.ph = make_phys<double>(g);
      args.nx = g.nx;
      args.ny = g.ny;
      args.nz = g.nz;
      args.pitch = g.pitch;
      args.vol = g.vol;
      for (int k = 0; k < 3; ++k) args.per[k] = g.per[k];
      make_bounce_terms<L, double>(g, args.bb);
      dim3 grid(div_up(g.nx, 256), g.ny, g.nz);
      k0_moments<L, double, double, FORCE><<<grid, 256, 0, stream>>>(args, ft, mom);
      k0_rebuild<L, double, double, FORCE><<<grid, 256, 0, stream>>>(args, mom, ft);
      err = cudaGetLastError();
    };
    if (g.has_force) go(std::true_type{});
    else go(std::false_type{});
  });
  return err;
}

cudaError_t k0_step(lb_ctx* ctx) {
  cudaError_t err = cudaErrorInvalidValue;
  if (ctx->g.ny > 65535 || ctx->g.nz > 65535) return cudaErrorInvalidConfiguration;
  dispatch_lattice(ctx->lattice, [&](auto Lt) {
    using L = decltype(Lt);
    dispatch_storage(ctx->storage, [&](auto St, auto Rt) {
      using S = typename decltype(St)::type;
      using R = typename decltype(Rt)::type;
      err = ctx->g.has_force ? launch<L, S, R, true>(ctx) : launch<L, S, R, false>(ctx);
    });
  });
  return err;
}

}  // namespace lbgb
