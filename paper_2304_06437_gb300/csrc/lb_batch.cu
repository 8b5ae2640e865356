// lb_batch.cu -- many independent domains stepped together.
//
// Contexts of the fused scheme are grouped into classes that share one
// compiled brick shape (lattice, storage, brick, pipeline) and the forcing
// switch.  Per time step each class runs ONE persistent launch: a grid of as
// many CTAs as fit on the GPU at once, each sweeping a fixed slice of a work
// list that holds every brick column of every domain of the class.  The list
// is balanced once, on the host, by greedy longest-processing-time assignment
// of the bricks (cost = nodes x planes incl. pipeline fill) to the CTAs.  The
// launches of two consecutive steps of all classes are captured in a CUDA
// graph and replayed, so a long run costs one graph launch per two steps.
//
// The per-node arithmetic, the bricks and the shells are exactly those of
// the domain's own single-domain launches: every domain's populations are bit
// for bit those of stepping it alone.
#include <algorithm>
#include <cstring>
#include <new>
#include <queue>
#include <vector>

#include "lb_k1_launch.cuh"

struct lb_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<lb_ctx*> ctxs;
  struct Class {
    const lbgb::K1Variant* v = nullptr;
    bool force = false;
    std::vector<int> members;  // indices into ctxs
    void* d_args = nullptr;    // K1Args<R>[2][n]
    CUtensorMap* d_tmaps = nullptr;
    int4* d_items = nullptr;
    int* d_starts = nullptr;
    int* d_par = nullptr;
    int* h_par = nullptr;  // pinned mirror of d_par
    int n_items = 0, grid = 0;
  };
  std::vector<Class> classes;
  int* d_status = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t done = nullptr;
  cudaEvent_t fork = nullptr;          // class branches of one step
  std::vector<cudaStream_t> side;      // one per class after the first
  std::vector<cudaEvent_t> join;
  std::vector<cudaEvent_t> ctx_ev;
  int64_t steps_done = 0;
  int64_t total_nodes = 0;
  double* d_sums = nullptr;  // lb_batch_reduce: seven sums per member (device)
  double* h_sums = nullptr;  // and their pinned host copy
};

namespace lbgb {
namespace {

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? LB_OK : (e == cudaErrorMemoryAllocation ? LB_E_NOMEM : LB_E_CUDA); }

#define LB_BTRY(x)                      \
  do {                                  \
    cudaError_t e_ = (x);               \
    if (e_ != cudaSuccess) return cuda_rc(e_); \
  } while (0)

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

void free_class(lb_batch::Class& c) {
  if (c.d_args) cudaFree(c.d_args);
  if (c.d_tmaps) cudaFree(c.d_tmaps);
  if (c.d_items) cudaFree(c.d_items);
  if (c.d_starts) cudaFree(c.d_starts);
  if (c.d_par) cudaFree(c.d_par);
  if (c.h_par) cudaFreeHost(c.h_par);
  c = lb_batch::Class{};
}

// Static balance: bricks by decreasing cost, each to the least-loaded CTA.
// A brick costs its full cross-section times its planes plus the pipeline
// fill: the warps of a ragged brick issue for their idle lanes too.
void build_work_list(const lb_batch& b, const lb_batch::Class& c, int grid, std::vector<int4>& items,
                     std::vector<int>& starts) {
  struct Brick {
    double cost;
    int4 it;
  };
  std::vector<Brick> all;
  for (int m = 0; m < int(c.members.size()); ++m) {
    const lb_ctx* x = b.ctxs[c.members[m]];
    const FusedPlan& p = x->plan;
    for (int k = 0; k < p.nbz; ++k)
      for (int j = 0; j < p.nby; ++j)
        for (int i = 0; i < p.nbx; ++i) {
          const int bz = std::min(p.bz, x->g.nz - k * p.bz);
          all.push_back({double(p.bx) * p.by * (bz + p.slots + 2), make_int4(m, i, j, k)});
        }
  }
  std::stable_sort(all.begin(), all.end(), [](const Brick& a, const Brick& b2) { return a.cost > b2.cost; });
  using Load = std::pair<double, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int g = 0; g < grid; ++g) heap.push({0.0, g});
  std::vector<std::vector<int4>> per(grid);
  for (const Brick& br : all) {
    Load l = heap.top();
    heap.pop();
    per[l.second].push_back(br.it);
    l.first += br.cost;
    heap.push(l);
  }
  items.clear();
  starts.assign(grid + 1, 0);
  for (int g = 0; g < grid; ++g) {
    starts[g] = int(items.size());
    items.insert(items.end(), per[g].begin(), per[g].end());
  }
  starts[grid] = int(items.size());
}

int setup_class(lb_batch& b, lb_batch::Class& c) {
  const int n = int(c.members.size());
  const int occ = c.v->batched_occupancy();
  if (occ <= 0) return LB_E_CUDA;
  std::vector<int4> items;
  std::vector<int> starts;
  int64_t bricks = 0;
  for (int m : c.members) {
    const FusedPlan& p = b.ctxs[m]->plan;
    bricks += int64_t(p.nbx) * p.nby * p.nbz;
  }
  const int grid = int(std::min<int64_t>(bricks, int64_t(k1_sm_count()) * occ));
  build_work_list(b, c, grid, items, starts);
  c.grid = grid;
  c.n_items = int(items.size());
  // arguments of every member at both shell parities, pointing at the batch's status word
  const bool dbl = b.ctxs[c.members[0]]->real_bytes == 8;
  std::vector<K1Args<float>> argsf;
  std::vector<K1Args<double>> argsd;
  (dbl ? argsd.resize(2 * size_t(n)) : argsf.resize(2 * size_t(n)));
  std::vector<CUtensorMap> maps(n);
  for (int m = 0; m < n; ++m) {
    lb_ctx* x = b.ctxs[c.members[m]];
    for (int p = 0; p < 2; ++p) {
      if (dbl) {
        K1Args<double> a = k1_make_args<double>(x, p, 1 - p);
        dispatch_lattice(x->lattice, [&](auto Lt) { make_bounce_terms<decltype(Lt), double>(x->g, a.bb); });
        a.status = b.d_status;
        argsd[size_t(p) * n + m] = a;
      } else {
        K1Args<float> a = k1_make_args<float>(x, p, 1 - p);
        dispatch_lattice(x->lattice, [&](auto Lt) { make_bounce_terms<decltype(Lt), float>(x->g, a.bb); });
        a.status = b.d_status;
        argsf[size_t(p) * n + m] = a;
      }
    }
    maps[m] = x->tmap;
  }
  const size_t args_bytes = dbl ? argsd.size() * sizeof(K1Args<double>) : argsf.size() * sizeof(K1Args<float>);
  const void* args_src = dbl ? static_cast<const void*>(argsd.data()) : static_cast<const void*>(argsf.data());
  LB_BTRY(cudaMalloc(&c.d_args, args_bytes));
  LB_BTRY(cudaMalloc(reinterpret_cast<void**>(&c.d_tmaps), maps.size() * sizeof(CUtensorMap)));
  LB_BTRY(cudaMalloc(reinterpret_cast<void**>(&c.d_items), std::max<size_t>(1, items.size()) * sizeof(int4)));
  LB_BTRY(cudaMalloc(reinterpret_cast<void**>(&c.d_starts), starts.size() * sizeof(int)));
  LB_BTRY(cudaMalloc(reinterpret_cast<void**>(&c.d_par), n * sizeof(int)));
  LB_BTRY(cudaHostAlloc(reinterpret_cast<void**>(&c.h_par), n * sizeof(int), cudaHostAllocDefault));
  LB_BTRY(cudaMemcpyAsync(c.d_args, args_src, args_bytes, cudaMemcpyHostToDevice, b.stream));
  LB_BTRY(cudaMemcpyAsync(c.d_tmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice,
                          b.stream));
  if (!items.empty())
    LB_BTRY(cudaMemcpyAsync(c.d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, b.stream));
  LB_BTRY(cudaMemcpyAsync(c.d_starts, starts.data(), starts.size() * sizeof(int), cudaMemcpyHostToDevice, b.stream));
  for (int m = 0; m < n; ++m) c.h_par[m] = -1;  // forces an upload before the first step
  return LB_OK;
}

// Re-plan a member for batched throughput: the first plain compiled shape (in
// the planner's order) whose bricks pad the cross-section by at most 25 %, else
// the least padded one; and, for sweeps of up to 256 planes, one brick per
// column, so that small domains do not pay the pipeline fill (slots + 2
// planes) and the z-shell of short bricks.  Bits are unchanged.
int batch_replan(lb_ctx* x) {
  const void* vs[64];
  const int nv = std::min(k1_variants_for(x->lattice, x->storage, vs, 64), 64);
  const K1Variant* pick = nullptr;
  const K1Variant* least = nullptr;
  double least_waste = 1e300;
  for (int i = 0; i < nv; ++i) {
    const K1Variant* v = static_cast<const K1Variant*>(vs[i]);
    // plain shapes only: the decoupled-export and TMA-store alternatives
    // measure slower on the large domains they were tried on
    if (!v->batched || v->nxw != 0 || v->ts != 0) continue;
    const double px = double((x->g.nx + v->bx - 1) / v->bx) * v->bx;
    const double py = double((x->g.ny + v->by - 1) / v->by) * v->by;
    const double waste = px * py / (double(x->g.nx) * double(x->g.ny));
    if (!pick && waste <= 1.25) pick = v;
    if (waste < least_waste) {
      least_waste = waste;
      least = v;
    }
  }
  if (!pick) pick = least;
  if (!pick) return LB_E_UNSUPPORTED;
  const int bz = x->g.nz <= 256 ? x->g.nz : 0;
  FusedPlan want;
  if (!k1_plan_variant(x->g, pick, bz, &want)) return LB_E_UNSUPPORTED;
  if (pick == k1_ctx_variant(x) && want.bz == x->plan.bz) return LB_OK;
  return ctx_replan(x, pick, bz);
}

// Split the bricks of a class that would not give each of its persistent
// CTAs at least two: halving its members' sweep length (down to 64 planes)
// doubles their bricks, so that the static work list balances, at the price
// of one more pipeline fill (slots + 2 planes) per added brick.  Bits are
// unchanged.
int split_for_balance(lb_batch& b, lb_batch::Class& c) {
  const int occ = c.v->batched_occupancy();
  if (occ <= 0) return LB_E_CUDA;
  const int64_t cap = int64_t(k1_sm_count()) * occ;
  for (int round = 0; round < 8; ++round) {
    int64_t bricks = 0;
    for (int m : c.members) {
      const FusedPlan& p = b.ctxs[m]->plan;
      bricks += int64_t(p.nbx) * p.nby * p.nbz;
    }
    if (bricks >= 2 * cap) return LB_OK;
    bool changed = false;
    for (int m : c.members) {
      lb_ctx* x = b.ctxs[m];
      if (x->plan.bz <= 64) continue;
      const int rc = ctx_replan(x, c.v, std::max(64, (x->plan.bz + 1) / 2));
      if (rc != LB_OK) return rc;
      changed = true;
    }
    if (!changed) return LB_OK;
  }
  return LB_OK;
}

// One step (k = 0 or 1 of the captured pair) of every class.  Classes are
// independent domains: each runs on its own branch (the batch stream for the
// first, a side stream forked from it for the others) and all join back.
int launch_classes(lb_batch& b, int k) {
  const int nc = int(b.classes.size());
  if (nc > 1) {
    LB_BTRY(cudaEventRecord(b.fork, b.stream));
    for (int i = 1; i < nc; ++i) LB_BTRY(cudaStreamWaitEvent(b.side[i - 1], b.fork, 0));
  }
  for (int i = 0; i < nc; ++i) {
    auto& c = b.classes[i];
    const BatchLaunch L{c.d_args, int(c.members.size()), c.d_tmaps, c.d_items, c.d_starts, c.d_par,
                        c.grid, k, c.force};
    LB_BTRY(c.v->batched(L, i == 0 ? b.stream : b.side[i - 1]));
  }
  for (int i = 1; i < nc; ++i) {
    LB_BTRY(cudaEventRecord(b.join[i - 1], b.side[i - 1]));
    LB_BTRY(cudaStreamWaitEvent(b.stream, b.join[i - 1], 0));
  }
  return LB_OK;
}

// upload each member's current shell parity if it changed since the last step
int sync_parities(lb_batch& b) {
  for (auto& c : b.classes) {
    bool changed = false;
    for (size_t m = 0; m < c.members.size(); ++m) {
      const int p = b.ctxs[c.members[m]]->parity;
      if (c.h_par[m] != p) changed = true;
    }
    if (!changed) continue;
    // the previous upload may still be in flight: wait before rewriting the pinned mirror
    LB_BTRY(cudaStreamSynchronize(b.stream));
    for (size_t m = 0; m < c.members.size(); ++m) c.h_par[m] = b.ctxs[c.members[m]]->parity;
    LB_BTRY(cudaMemcpyAsync(c.d_par, c.h_par, c.members.size() * sizeof(int), cudaMemcpyHostToDevice, b.stream));
  }
  return LB_OK;
}

}  // namespace
}  // namespace lbgb

using namespace lbgb;

extern "C" {

int lb_batch_create(lb_ctx* const* ctxs, int32_t n, void* stream, lb_batch** out) {
  if (!out || !ctxs || n < 1) return LB_E_INVAL;
  *out = nullptr;
  const int dev = ctxs[0] ? ctxs[0]->device : -1;
  for (int i = 0; i < n; ++i) {
    lb_ctx* x = ctxs[i];
    if (!x || x->device != dev) return LB_E_INVAL;
    if (x->scheme != LB_SCHEME_FUSED) return LB_E_UNSUPPORTED;
    // a slab bordering others steps between halo exchanges, not in a batch
    if (x->g.zlink[0] || x->g.zlink[1]) return LB_E_UNSUPPORTED;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == x) return LB_E_INVAL;
    const K1Variant* v = k1_ctx_variant(x);
    if (!v || !v->batched) return LB_E_UNSUPPORTED;
  }
  DevGuard guard(dev);
  lb_batch* b = new (std::nothrow) lb_batch();
  if (!b) return LB_E_NOMEM;
  b->device = dev;
  int rc = LB_OK;
  do {
    if (stream) {
      b->stream = static_cast<cudaStream_t>(stream);
    } else {
      if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) { rc = LB_E_CUDA; break; }
      b->own_stream = true;
    }
    b->ctxs.assign(ctxs, ctxs + n);
    for (int i = 0; i < n && rc == LB_OK; ++i) {
      // the domain's own stream must be done before the batch reads its state
      if (cudaStreamSynchronize(ctxs[i]->stream) != cudaSuccess) rc = LB_E_CUDA;
      else rc = batch_replan(ctxs[i]);
    }
    if (rc != LB_OK) break;
    for (int i = 0; i < n; ++i) {
      lb_ctx* x = ctxs[i];
      b->total_nodes += x->n_nodes;
      const K1Variant* v = k1_ctx_variant(x);
      const bool force = x->g.has_force;
      auto it = std::find_if(b->classes.begin(), b->classes.end(),
                             [&](const lb_batch::Class& c) { return c.v == v && c.force == force; });
      if (it == b->classes.end()) {
        b->classes.emplace_back();
        b->classes.back().v = v;
        b->classes.back().force = force;
        it = b->classes.end() - 1;
      }
      it->members.push_back(i);
    }
    if (rc != LB_OK) break;
    for (auto& c : b->classes) {
      rc = split_for_balance(*b, c);
      if (rc != LB_OK) break;
    }
    if (rc != LB_OK) break;
    if (cudaMalloc(reinterpret_cast<void**>(&b->d_status), sizeof(int)) != cudaSuccess) { rc = LB_E_NOMEM; break; }
    if (cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream) != cudaSuccess) { rc = LB_E_CUDA; break; }
    for (auto& c : b->classes) {
      rc = setup_class(*b, c);
      if (rc != LB_OK) break;
    }
    if (rc != LB_OK) break;
    if (cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) { rc = LB_E_CUDA; break; }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) { rc = LB_E_CUDA; break; }
    for (size_t i = 1; i < b->classes.size() && rc == LB_OK; ++i) {
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = LB_E_CUDA;
      else b->side.push_back(st);
      if (rc == LB_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) rc = LB_E_CUDA;
      else if (rc == LB_OK) b->join.push_back(ev);
    }
    if (rc != LB_OK) break;
    b->ctx_ev.resize(n, nullptr);
    for (int i = 0; i < n && rc == LB_OK; ++i)
      if (cudaEventCreateWithFlags(&b->ctx_ev[i], cudaEventDisableTiming) != cudaSuccess) rc = LB_E_CUDA;
    if (rc != LB_OK) break;
    // capture two consecutive steps of every class
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = LB_E_CUDA; break; }
    int rc0 = launch_classes(*b, 0);
    int rc1 = rc0 == LB_OK ? launch_classes(*b, 1) : rc0;
    cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
    if (rc1 != LB_OK || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      rc = rc1 != LB_OK ? rc1 : LB_E_CUDA;
      break;
    }
    ee = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (ee != cudaSuccess) { rc = LB_E_CUDA; break; }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) { rc = LB_E_CUDA; break; }
  } while (false);
  if (rc != LB_OK) {
    lb_batch_destroy(b);
    return rc;
  }
  *out = b;
  return LB_OK;
}

int lb_batch_step(lb_batch* b, int64_t n) {
  if (!b || n < 0) return LB_E_INVAL;
  if (n == 0) return LB_OK;
  DevGuard guard(b->device);
  // order after work queued on the members' own streams
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    LB_BTRY(cudaEventRecord(b->ctx_ev[i], b->ctxs[i]->stream));
    LB_BTRY(cudaStreamWaitEvent(b->stream, b->ctx_ev[i], 0));
  }
  int rc = sync_parities(*b);
  if (rc != LB_OK) return rc;
  for (int64_t s = 0; s + 1 < n; s += 2) LB_BTRY(cudaGraphLaunch(b->graph, b->stream));
  if (n & 1) {
    rc = launch_classes(*b, 0);
    if (rc != LB_OK) return rc;
  }
  for (lb_ctx* x : b->ctxs) {
    if (n & 1) x->parity = 1 - x->parity;
    x->steps_done += n;
  }
  b->steps_done += n;
  // later work on a member's stream sees the batch's steps
  LB_BTRY(cudaEventRecord(b->done, b->stream));
  for (lb_ctx* x : b->ctxs) LB_BTRY(cudaStreamWaitEvent(x->stream, b->done, 0));
  return LB_OK;
}

int lb_batch_sync(lb_batch* b) {
  if (!b) return LB_E_INVAL;
  DevGuard guard(b->device);
  int st = 0;
  LB_BTRY(cudaMemcpyAsync(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  LB_BTRY(cudaStreamSynchronize(b->stream));
  return st != 0 ? st : LB_OK;
}

int lb_batch_reduce(lb_batch* b, int32_t want_residual, double* out) {
  if (!b || !out) return LB_E_INVAL;
  DevGuard guard(b->device);
  const size_t n = b->ctxs.size();
  if (!b->d_sums) {
    LB_BTRY(cudaMalloc(reinterpret_cast<void**>(&b->d_sums), n * kReduceFields * sizeof(double)));
    LB_BTRY(cudaMallocHost(reinterpret_cast<void**>(&b->h_sums), n * kReduceFields * sizeof(double)));
  }
  // after the work queued on the members' own streams and the batch's steps
  for (size_t i = 0; i < n; ++i) {
    LB_BTRY(cudaEventRecord(b->ctx_ev[i], b->ctxs[i]->stream));
    LB_BTRY(cudaStreamWaitEvent(b->stream, b->ctx_ev[i], 0));
  }
  for (size_t i = 0; i < n; ++i)
    LB_BTRY(aux_reduce_enqueue(b->ctxs[i], b->stream, b->d_sums + i * kReduceFields, want_residual != 0));
  LB_BTRY(cudaMemcpyAsync(b->h_sums, b->d_sums, n * kReduceFields * sizeof(double), cudaMemcpyDeviceToHost,
                          b->stream));
  // the members' reduction buffers and residual snapshots were used on the
  // batch stream: later work on a member's stream comes after
  LB_BTRY(cudaEventRecord(b->done, b->stream));
  for (lb_ctx* x : b->ctxs) LB_BTRY(cudaStreamWaitEvent(x->stream, b->done, 0));
  LB_BTRY(cudaStreamSynchronize(b->stream));
  for (size_t i = 0; i < n; ++i) {
    double* o = out + 6 * i;
    double mom[3] = {0, 0, 0}, res = 0.0;
    const int rc = reduce_finish(b->ctxs[i], b->h_sums + i * kReduceFields, want_residual != 0, &o[0], mom,
                                 want_residual ? &res : nullptr);
    o[1] = mom[0];
    o[2] = mom[1];
    o[3] = mom[2];
    o[4] = res;
    o[5] = rc == LB_OK ? 0.0 : double(rc);
  }
  return LB_OK;
}

int lb_batch_info(const lb_batch* b, lb_batch_info_t* info) {
  if (!b || !info) return LB_E_INVAL;
  std::memset(info, 0, sizeof(*info));
  info->n_domains = int32_t(b->ctxs.size());
  info->n_classes = int32_t(b->classes.size());
  info->total_nodes = b->total_nodes;
  info->steps_done = b->steps_done;
  for (const auto& c : b->classes) {
    info->work_items += c.n_items;
    info->launches_per_step += 1;
    info->ctas += c.grid;
  }
  return LB_OK;
}

void lb_batch_destroy(lb_batch* b) {
  if (!b) return;
  DevGuard guard(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (auto& c : b->classes) free_class(c);
  if (b->d_status) cudaFree(b->d_status);
  if (b->done) cudaEventDestroy(b->done);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t st : b->side)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t e : b->ctx_ev)
    if (e) cudaEventDestroy(e);
  if (b->d_sums) cudaFree(b->d_sums);
  if (b->h_sums) cudaFreeHost(b->h_sums);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

}  // extern "C"
