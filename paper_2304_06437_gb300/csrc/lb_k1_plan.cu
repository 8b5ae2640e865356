// lb_k1_plan.cu -- brick decomposition of the fused step: picks a compiled
// brick shape, the sweep length bz, and lays out the shell buffers.
#include <cstdio>
#include <cstdlib>

#include "lb_k1_launch.cuh"

namespace lbgb {

extern const K1Variant k1_variants_d2q9[];
extern const int k1_n_variants_d2q9;
extern const K1Variant k1_variants_d3q19[];
extern const int k1_n_variants_d3q19;
extern const K1Variant k1_variants_d3q27[];
extern const int k1_n_variants_d3q27;
extern const K1Variant k2_variants_d2q9[];
extern const int k2_n_variants_d2q9;
extern const K1Variant k2_variants_d3q19[];
extern const int k2_n_variants_d3q19;
extern const K1Variant k2_variants_d3q27[];
extern const int k2_n_variants_d3q27;

// The compiled brick shapes of a lattice in the planner's order of
// preference: for D2Q9 the paired kernels (two nodes per thread, FP32x2) come
// first, for D3Q19 / D3Q27 the scalar ones, which measure faster there (the
// paired 3D kernels need ~230 registers per thread and run 8 warps per SM).
static int variant_lists(int lattice, const K1Variant* lists[2], int counts[2]) {
  switch (lattice) {
    case LB_D2Q9:
      lists[0] = k2_variants_d2q9; counts[0] = k2_n_variants_d2q9;
      lists[1] = k1_variants_d2q9; counts[1] = k1_n_variants_d2q9;
      return 2;
    case LB_D3Q19:
      lists[0] = k1_variants_d3q19; counts[0] = k1_n_variants_d3q19;
      lists[1] = k2_variants_d3q19; counts[1] = k2_n_variants_d3q19;
      return 2;
    case LB_D3Q27:
      lists[0] = k1_variants_d3q27; counts[0] = k1_n_variants_d3q27;
      lists[1] = k2_variants_d3q27; counts[1] = k2_n_variants_d3q27;
      return 2;
    default: return 0;
  }
}

// The first compiled shape that matches (lattice, storage, bx, by, ns, wb,
// nxw, npt, ts, minb); zero fields (-1 for nxw and ts) match anything.
static const K1Variant* find_variant(int lattice, int storage, int bx, int by, int ns, int wb, int nxw, int npt,
                                     int ts, int minb = 0) {
  const K1Variant* lists[2];
  int counts[2];
  const int nl = variant_lists(lattice, lists, counts);
  for (int l = 0; l < nl; ++l) {
    for (int i = 0; i < counts[l]; ++i) {
      const K1Variant& v = lists[l][i];
      if (v.storage != storage) continue;
      if (bx > 0 && v.bx != bx) continue;
      if (by > 0 && v.by != by) continue;
      if (ns > 0 && v.ns != ns) continue;
      if (wb > 0 && v.wb != wb) continue;
      if (nxw != -1 && v.nxw != nxw) continue;
      if (npt > 0 && v.npt != npt) continue;
      if (ts >= 0 && v.ts != ts) continue;
      if (minb > 0 && v.minb != minb) continue;
      return &v;
    }
  }
  return nullptr;
}

// Optional pipeline request from the environment,
// "NS,WB[,NXW[,NPT[,TS[,MINB]]]]" (TMA slots, window buffers, dedicated
// export warps (negative: warps inside the per-plane barrier), nodes per
// thread, TMA store of completed planes, CTAs per SM), used to compare the
// compiled alternatives of a brick shape; 0 (-1 for NXW and TS) = any.
static void pipeline_request(int* ns, int* wb, int* nxw, int* npt, int* ts, int* minb) {
  *ns = 0;
  *wb = 0;
  *nxw = -1;
  *npt = 0;
  *ts = -1;
  *minb = 0;
  const char* e = std::getenv("LB_FUSED_PIPELINE");
  if (e) std::sscanf(e, "%d,%d,%d,%d,%d,%d", ns, wb, nxw, npt, ts, minb);
}

static int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 152;
  return n;
}

// Sweep length: bricks per wave fill the SMs evenly (one CTA per SM), while
// each brick stays long enough that its pipeline fill/drain (about NS + 2
// planes) and its z-shell traffic stay small.
static int choose_bz(int nz, int columns, int slots, int sms) {
  int best_bz = nz;
  double best = -1.0;
  for (int nbz = 1; nbz <= 64; ++nbz) {
    const int bz = (nz + nbz - 1) / nbz;
    if (bz < 8 && nbz > 1) break;
    const int nbz_eff = (nz + bz - 1) / bz;
    const double bricks = double(columns) * nbz_eff;
    const double waves = bricks / sms;
    const double fill = waves / std::ceil(waves);
    const double pipe = double(bz) / double(bz + slots + 2);
    const double score = fill * pipe;
    if (score > best + 1e-9) {
      best = score;
      best_bz = bz;
    }
  }
  return best_bz;
}

static void fill_plan(const Geometry& g, const K1Variant* v, int req_bz, FusedPlan* plan, int sms = 0) {
  FusedPlan p{};
  p.bx = v->bx;
  p.by = v->by;
  p.slots = v->ns;
  p.wbuf = v->wb;
  p.xwarps = v->nxw;
  p.npt = v->npt;
  p.ts = v->ts;
  p.minb = v->minb;
  p.smem_bytes = v->smem;
  p.nbx = (g.nx + p.bx - 1) / p.bx;
  p.nby = (g.ny + p.by - 1) / p.by;
  const int columns = p.nbx * p.nby;
  // resident CTAs: the SMs times the CTAs one SM holds of this shape
  const int slots_gpu = (sms > 0 ? sms : sm_count()) * (v->minb > 0 ? v->minb : 1);
  p.bz = req_bz > 0 ? (req_bz < g.nz ? req_bz : g.nz) : choose_bz(g.nz, columns, p.slots, slots_gpu);
  p.nbz = (g.nz + p.bz - 1) / p.bz;
  int nxf = 0, nyf = 0, nzf = 0;
  dispatch_lattice(g.lattice, [&](auto Lt) {
    using L = decltype(Lt);
    nxf = count_dirs<L>(0, 1);
    nyf = count_dirs<L>(1, 1);
    nzf = count_dirs<L>(2, 1);
  });
  p.nxf = nxf;
  p.nyf = nyf;
  p.nzf = nzf;
  // a link face's incoming records sit in one ghost plane (x / y records)
  // and one ghost brick row (z records) on each side of the shell
  p.zg = (g.zlink[0] || g.zlink[1]) ? 1 : 0;
  p.sx_elems = 2LL * p.nbx * nxf * int64_t(g.nz + 2 * p.zg) * g.ny;
  p.sy_elems = 2LL * p.nby * nyf * int64_t(g.nz + 2 * p.zg) * g.nx;
  p.sz_elems = 2LL * (p.nbz + 2 * p.zg) * nzf * int64_t(g.ny) * g.nx;
  p.parity_elems = ((p.sx_elems + p.sy_elems + p.sz_elems) + 31) / 32 * 32;
  *plan = p;
}

bool k1_plan(const Geometry& g, int storage, const int32_t tile_req[3], FusedPlan* plan, int sms) {
  const int rbx = tile_req ? tile_req[0] : 0;
  const int rby = tile_req ? tile_req[1] : 0;
  int rns, rwb, rnxw, rnpt, rts, rminb;
  pipeline_request(&rns, &rwb, &rnxw, &rnpt, &rts, &rminb);
  const K1Variant* v = find_variant(g.lattice, storage, rbx, rby, rns, rwb, rnxw, rnpt, rts, rminb);
  if (!v) return false;
  fill_plan(g, v, tile_req ? tile_req[2] : 0, plan, sms);
  return true;
}

bool k1_plan_variant(const Geometry& g, const void* variant, int bz, FusedPlan* plan) {
  const K1Variant* v = static_cast<const K1Variant*>(variant);
  if (!v || v->lattice != g.lattice) return false;
  fill_plan(g, v, bz, plan);
  return true;
}

int k1_variants_for(int lattice, int storage, const void** out, int cap) {
  const K1Variant* lists[2];
  int counts[2];
  const int nl = variant_lists(lattice, lists, counts);
  int n = 0;
  for (int l = 0; l < nl; ++l)
    for (int i = 0; i < counts[l]; ++i)
      if (lists[l][i].storage == storage) {
        if (n < cap) out[n] = &lists[l][i];
        ++n;
      }
  return n;
}

static const K1Variant* ctx_variant(lb_ctx* ctx) {
  return find_variant(ctx->lattice, ctx->storage, ctx->plan.bx, ctx->plan.by, ctx->plan.slots, ctx->plan.wbuf,
                      ctx->plan.xwarps, ctx->plan.npt, ctx->plan.ts, ctx->plan.minb);
}

const K1Variant* k1_ctx_variant(lb_ctx* ctx) { return ctx_variant(ctx); }

int k1_sm_count() { return sm_count(); }

cudaError_t k1_configure(lb_ctx* ctx) {
  const K1Variant* v = ctx_variant(ctx);
  if (!v) return cudaErrorInvalidValue;
  return v->configure();
}

cudaError_t k1_step(lb_ctx* ctx) {
  const K1Variant* v = ctx_variant(ctx);
  if (!v) return cudaErrorInvalidValue;
  cudaError_t e = v->step(ctx);
  if (e == cudaSuccess) ctx->parity = 1 - ctx->parity;
  return e;
}

cudaError_t k1_bootstrap(lb_ctx* ctx) {
  const K1Variant* v = ctx_variant(ctx);
  if (!v) return cudaErrorInvalidValue;
  return v->bootstrap(ctx);
}

}  // namespace lbgb
