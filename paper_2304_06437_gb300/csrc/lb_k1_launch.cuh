// lb_k1_launch.cuh -- host-side launchers of the fused step, one set per
// compiled brick shape (lattice x storage x bx x by x pipeline depth).
#pragma once

#include "lb_k1.cuh"

namespace lbgb {

struct K1Variant {
  int lattice, storage, bx, by, ns, wb, nxw;
  size_t smem;
  cudaError_t (*configure)();
  cudaError_t (*step)(lb_ctx*);
  cudaError_t (*bootstrap)(lb_ctx*);
};

template <class R>
K1Args<R> k1_make_args(lb_ctx* ctx, int cur_parity, int next_parity) {
  const Geometry& g = ctx->g;
  const FusedPlan& p = ctx->plan;
  K1Args<R> a;
  a.ph = make_phys<R>(g);
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.nz;
  a.pitch = g.pitch;
  a.vol = g.vol;
  for (int k = 0; k < 3; ++k) a.per[k] = g.per[k];
  a.bz = p.bz;
  a.nbx = p.nbx;
  a.nby = p.nby;
  a.nbz = p.nbz;
  a.f = ctx->f;
  R* base = static_cast<R*>(ctx->aux);
  a.sh_cur = base + int64_t(cur_parity) * p.parity_elems;
  a.sh_next = base + int64_t(next_parity) * p.parity_elems;
  a.sx_off = 0;
  a.sy_off = p.sx_elems;
  a.sz_off = p.sx_elems + p.sy_elems;
  a.status = ctx->d_status;
  for (int i = 0; i < 27; ++i)
    for (int j = 0; j < 8; ++j) a.bb[i][j] = R(0);
  return a;
}

template <class L, class S, class R, int BX, int BY, int NS, int WB, int NXW>
struct K1Impl {
  using Sh = K1Shape<L, S, R, BX, BY, NS, WB, NXW>;

  static cudaError_t configure() {
    cudaError_t e = cudaFuncSetAttribute(k1_fused_step<L, S, R, BX, BY, NS, WB, NXW, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::SMEM));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k1_fused_step<L, S, R, BX, BY, NS, WB, NXW, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::SMEM));
  }

  static cudaError_t step(lb_ctx* ctx) {
    K1Args<R> a = k1_make_args<R>(ctx, ctx->parity, 1 - ctx->parity);
    make_bounce_terms<L, R>(ctx->g, a.bb);
    const int grid = ctx->plan.nbx * ctx->plan.nby * ctx->plan.nbz;
    if (ctx->g.has_force)
      k1_fused_step<L, S, R, BX, BY, NS, WB, NXW, true><<<grid, Sh::NT, Sh::SMEM, ctx->stream>>>(ctx->tmap, a);
    else
      k1_fused_step<L, S, R, BX, BY, NS, WB, NXW, false><<<grid, Sh::NT, Sh::SMEM, ctx->stream>>>(ctx->tmap, a);
    return cudaGetLastError();
  }

  static cudaError_t bootstrap(lb_ctx* ctx) {
    // fill the parity the next step reads
    K1Args<R> a = k1_make_args<R>(ctx, 1 - ctx->parity, ctx->parity);
    const int64_t n = int64_t(ctx->g.nx) * ctx->g.ny * ctx->g.nz;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (ctx->g.has_force)
      k1_bootstrap<L, S, R, BX, BY, true><<<int(blocks), 256, 0, ctx->stream>>>(a);
    else
      k1_bootstrap<L, S, R, BX, BY, false><<<int(blocks), 256, 0, ctx->stream>>>(a);
    return cudaGetLastError();
  }

  static constexpr K1Variant variant(int lattice, int storage) {
    return K1Variant{lattice, storage, BX, BY, NS, WB, NXW, Sh::SMEM, &configure, &step, &bootstrap};
  }
};

}  // namespace lbgb
