// lb_tune.cu -- autotuner of the fused step's brick shape.
//
// Every compiled shape of the context's lattice and storage (brick bx x by,
// TMA pipeline depth, one or two nodes per thread) is timed on a proxy
// domain: the same cross-section, boundaries, tau and force, with the sweep
// axis shortened so the proxy holds at most kProxyBytes of populations.  The
// fastest shape per node update is then applied to the context (new shells
// and TMA descriptor, shell rebuilt from the current populations; the
// populations are untouched, and every shape gives the same bits).  Results
// are cached per (lattice, storage, cross-section, sweep-length class,
// boundary kinds, forcing), so domains of one kind are timed once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "lb_k1_launch.cuh"

namespace lbgb {
namespace {

constexpr double kProxyBytes = 4.0e9;

using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int>;
std::mutex g_mu;
std::map<TuneKey, const void*> g_cache;

TuneKey key_of(const lb_ctx* ctx) {
  const Geometry& g = ctx->g;
  int kinds = 0;
  for (int f = 0; f < 6; ++f) kinds = kinds * 3 + g.face_kind[f];
  // sweep-length class: the number of planes rounded to a power of two
  int nzc = 1;
  while (nzc < g.nz) nzc *= 2;
  return TuneKey{ctx->lattice, ctx->storage, g.nx, g.ny, nzc, kinds, g.has_force ? 1 : 0, 0, 0};
}

// time `steps` fused steps of one shape on a proxy; ms per node update x 1e6
int time_variant(const lb_ctx* ctx, const void* v, int steps, double* ns_per_update, int32_t tile[3]) {
  const Geometry& g = ctx->g;
  int64_t dims[3] = {ctx->dims[0], ctx->dims[1], ctx->dims[2]};
  const int slow = g.d == 2 ? 1 : 2;  // user axis that is the internal sweep axis
  const double per_plane = double(g.q) * ctx->elem_bytes * double(dims[0]) * (g.d == 2 ? 1.0 : double(dims[1]));
  const int64_t max_planes = std::max<int64_t>(8, int64_t(kProxyBytes / per_plane));
  dims[slow] = std::min<int64_t>(dims[slow], max_planes);
  lb_options opt = ctx->opt_user;
  opt.stream = nullptr;
  opt.device = ctx->device;
  opt.tile[0] = opt.tile[1] = opt.tile[2] = 0;
  lb_ctx* p = nullptr;
  int rc = lb_create(ctx->lattice, dims, ctx->tau_user, &ctx->bnd_user, &opt, &p);
  if (rc != LB_OK) return rc;
  rc = ctx_replan(p, v);
  const double u[3] = {0.01, 0.005, 0.0};
  if (rc == LB_OK) rc = lb_init_uniform(p, ctx->g.rho0, u);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rc == LB_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = LB_E_CUDA;
  if (rc == LB_OK) rc = lb_step(p, 2);
  if (rc == LB_OK && cudaEventRecord(e0, p->stream) != cudaSuccess) rc = LB_E_CUDA;
  if (rc == LB_OK) rc = lb_step(p, steps);
  if (rc == LB_OK && cudaEventRecord(e1, p->stream) != cudaSuccess) rc = LB_E_CUDA;
  if (rc == LB_OK) rc = lb_sync(p);
  float ms = 0.0f;
  if (rc == LB_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = LB_E_CUDA;
  if (rc == LB_OK) {
    *ns_per_update = double(ms) * 1e6 / (double(steps) * double(p->n_nodes));
    tile[0] = p->plan.bx;
    tile[1] = p->plan.by;
    tile[2] = p->plan.bz;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  lb_destroy(p);
  return rc;
}

}  // namespace
}  // namespace lbgb

using namespace lbgb;

extern "C" {

int lb_autotune(lb_ctx* ctx, int32_t steps, lb_tune_entry* table, int32_t cap, int32_t* n_entries) {
  if (!ctx || steps < 1) return LB_E_INVAL;
  if (n_entries) *n_entries = 0;
  if (ctx->scheme != LB_SCHEME_FUSED) return LB_E_UNSUPPORTED;
  // a slab's brick cross-section must stay that of its neighbours
  if (ctx->g.zlink[0] || ctx->g.zlink[1]) return LB_E_UNSUPPORTED;
  const TuneKey key = key_of(ctx);
  const void* best = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) best = it->second;
  }
  if (!best) {
    const void* vs[64];
    const int nv = std::min(k1_variants_for(ctx->lattice, ctx->storage, vs, 64), 64);
    double best_t = 1e300;
    int n = 0;
    for (int i = 0; i < nv; ++i) {
      double t = 0.0;
      int32_t tile[3] = {0, 0, 0};
      const int rc = time_variant(ctx, vs[i], steps, &t, tile);
      const K1Variant* v = static_cast<const K1Variant*>(vs[i]);
      if (table && n < cap) {
        lb_tune_entry& e = table[n];
        std::memset(&e, 0, sizeof(e));
        e.bx = v->bx;
        e.by = v->by;
        e.bz = tile[2];
        e.slots = v->ns;
        e.nodes_per_thread = v->npt;
        e.export_warps = v->nxw;
        e.status = rc;
        e.ns_per_update = rc == LB_OK ? t : -1.0;
      }
      ++n;
      if (rc == LB_OK && t < best_t) {
        best_t = t;
        best = vs[i];
      }
    }
    if (n_entries) *n_entries = std::min(n, cap);
    if (!best) return LB_E_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = best;
  }
  if (best == static_cast<const void*>(k1_ctx_variant(ctx))) return LB_OK;
  return ctx_replan(ctx, best);
}

}  // extern "C"
