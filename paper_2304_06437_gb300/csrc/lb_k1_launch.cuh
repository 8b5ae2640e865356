// lb_k1_launch.cuh -- host-side launchers of the fused step, one set per
// compiled brick shape (lattice x storage x bx x by x pipeline depth).
#pragma once

#include "lb_k1.cuh"

namespace lbgb {

// Device-side description of one batched launch (see lb_batch.cu): the
// per-domain arguments at both shell parities, TMA descriptors, the static
// work list of brick items and each CTA's slice of it.
struct BatchLaunch {
  const void* args;  // K1Args<R>[2][n_dom], R the arithmetic type of the variant
  int n_dom;
  const CUtensorMap* tmaps;
  const int4* items;
  const int* starts;
  const int* dom_par;
  int grid;
  int k;      // step within the captured pair (0 or 1)
  bool force;
};

struct K1Variant {
  int lattice, storage, bx, by, ns, wb, nxw;
  size_t smem;
  cudaError_t (*configure)();
  cudaError_t (*step)(lb_ctx*);
  cudaError_t (*bootstrap)(lb_ctx*);
  int npt;  // nodes per thread: 1 = scalar kernel (lb_k1.cuh), 2 = paired kernel (lb_k2.cuh)
  // batched persistent launch (paired kernels only; null otherwise) and the
  // number of its CTAs that fit on one SM
  cudaError_t (*batched)(const BatchLaunch&, cudaStream_t);
  int (*batched_occupancy)();
  int ts;  // 1: completed planes leave through a TMA store (scalar kernel only)
  int minb;  // CTAs per SM the shape is compiled for
};

// the compiled shape a fused-scheme context runs (lb_k1_plan.cu)
const K1Variant* k1_ctx_variant(lb_ctx* ctx);
int k1_sm_count();

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
  a.vol32 = uint32_t(g.vol / 32);
  for (int k = 0; k < 3; ++k) a.per[k] = g.per[k];
  a.zlink[0] = g.zlink[0];
  a.zlink[1] = g.zlink[1];
  a.zg = p.zg;
  a.nzs = g.nz + 2 * p.zg;
  a.nbzs = p.nbz + 2 * p.zg;
  a.zwl = (!g.per[2] && !g.zlink[0]) ? 0 : -1;
  a.zwh = (!g.per[2] && !g.zlink[1]) ? g.nz - 1 : -1;
  a.zwrap = g.per[2] ? g.nz : 0;
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

template <class L, class S, class R, int BX, int BY, int NS, int WB, int NXW, int TS = 0, int MINB = 1>
struct K1Impl {
  using Sh = K1Shape<L, S, R, BX, BY, NS, WB, NXW, TS, MINB>;

  static cudaError_t configure() {
    const int sm = int(Sh::SMEM);
    cudaError_t e = cudaFuncSetAttribute(k1_fused_step<L, S, R, BX, BY, NS, WB, NXW, false, TS, false, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k1_fused_step<L, S, R, BX, BY, NS, WB, NXW, true, TS, false, MINB>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k1_fused_step<L, S, R, BX, BY, NS, WB, NXW, false, TS, true, MINB>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k1_fused_step<L, S, R, BX, BY, NS, WB, NXW, true, TS, true, MINB>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    return e;
  }

  static cudaError_t step(lb_ctx* ctx) {
    K1Args<R> a = k1_make_args<R>(ctx, ctx->parity, 1 - ctx->parity);
    make_bounce_terms<L, R>(ctx->g, a.bb);
    const int grid = ctx->plan.nbx * ctx->plan.nby * ctx->plan.nbz;
    const bool link = ctx->g.zlink[0] || ctx->g.zlink[1];
    cudaStream_t st = ctx->stream;
    if (link) {
      if (ctx->g.has_force)
        k1_fused_step<L, S, R, BX, BY, NS, WB, NXW, true, TS, true, MINB><<<grid, Sh::NT, Sh::SMEM, st>>>(ctx->tmap, a);
      else
        k1_fused_step<L, S, R, BX, BY, NS, WB, NXW, false, TS, true, MINB><<<grid, Sh::NT, Sh::SMEM, st>>>(ctx->tmap, a);
    } else if (ctx->g.has_force) {
      k1_fused_step<L, S, R, BX, BY, NS, WB, NXW, true, TS, false, MINB><<<grid, Sh::NT, Sh::SMEM, st>>>(ctx->tmap, a);
    } else {
      k1_fused_step<L, S, R, BX, BY, NS, WB, NXW, false, TS, false, MINB><<<grid, Sh::NT, Sh::SMEM, st>>>(ctx->tmap, a);
    }
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

  static constexpr size_t SMEM_B = K1BatchSmem<Sh, R>::BYTES;

  static cudaError_t batched(const BatchLaunch& b, cudaStream_t stream) {
    const K1Args<R>* args = static_cast<const K1Args<R>*>(b.args);
    if (b.force)
      k1_batched_step<L, S, R, BX, BY, NS, WB, NXW, true, TS, MINB><<<b.grid, Sh::NT, SMEM_B, stream>>>(
          args, b.n_dom, b.tmaps, b.items, b.starts, b.dom_par, b.k);
    else
      k1_batched_step<L, S, R, BX, BY, NS, WB, NXW, false, TS, MINB><<<b.grid, Sh::NT, SMEM_B, stream>>>(
          args, b.n_dom, b.tmaps, b.items, b.starts, b.dom_par, b.k);
    return cudaGetLastError();
  }

  static int batched_occupancy() {
    const int sm = int(SMEM_B);
    if (configure() != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(k1_batched_step<L, S, R, BX, BY, NS, WB, NXW, false, TS, MINB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess ||
        cudaFuncSetAttribute(k1_batched_step<L, S, R, BX, BY, NS, WB, NXW, true, TS, MINB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess)
      return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k1_batched_step<L, S, R, BX, BY, NS, WB, NXW, true, TS, MINB>, Sh::NT,
                                                      SMEM_B) != cudaSuccess)
      return 0;
    return n;
  }

  static constexpr K1Variant variant(int lattice, int storage) {
    return K1Variant{lattice, storage, BX, BY, NS, WB, NXW, Sh::SMEM, &configure, &step, &bootstrap, 1, &batched,
                     &batched_occupancy, TS, MINB};
  }
};

}  // namespace lbgb
