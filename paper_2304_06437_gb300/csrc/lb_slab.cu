// lb_slab.cu -- slab decomposition along the slowest axis: halo messages of
// link faces (lb_halo_*) and an in-process slab group (lb_group_*).
//
// A rank boundary is a brick face of the fused scheme (lb_k1.cuh).  What a
// slab's boundary bricks read across it in launch t + 1 is what the bricks on
// the other side exported in launch t:
//   * the z-face records SZ[side][K][ia][y][x] of the neighbour's outermost
//     brick row (its populations that cross the face), and
//   * the x- and y-face records SX[side][I][ia][z][y] / SY[side][J][ia][z][x]
//     of the neighbour's outermost plane: the ring of the virtual plane just
//     outside the slab, which carries the diagonal links that cross the face
//     and a lateral brick face at once.
// A linked context keeps one ghost plane (x / y records) and one ghost brick
// row (z records) per link face in each shell parity; the message fills them.
// Message = 64-byte header | x records | y records | z records, all of the
// shell's element type (FP64 for FP64 storage, FP32 otherwise).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "lb_internal.h"

using namespace lbgb;

namespace {

constexpr int64_t kMagic = 0x4C42534C41420001LL;  // "LBSLAB" + layout version
constexpr int kHeaderWords = 8;                    // 64 bytes

// One copy between the shell of one parity and a message: three strided
// regions (rows of the x records, rows of the y records, the z record).
struct HaloMap {
  int64_t rows[3];   // rows per region
  int64_t len[3];    // elements per row
  int64_t pitch[3];  // shell elements between consecutive rows
  int64_t src[3];    // shell offset of row 0
  int64_t base[3];   // message element offset of the region (after the header)
  int64_t total;     // elements in the message body
  int64_t header[kHeaderWords];
};

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LB_OK;
  if (e == cudaErrorMemoryAllocation) return LB_E_NOMEM;
  return LB_E_CUDA;
}

// The shell regions of face `side`: outgoing (to_msg) or the ghost slots
// (incoming).  Internal axes: the slowest axis is internal z in 2D and 3D.
HaloMap halo_map(const lb_ctx* ctx, int side, bool outgoing) {
  const Geometry& g = ctx->g;
  const FusedPlan& p = ctx->plan;
  const int64_t nzs = g.nz + 2 * p.zg, nbzs = p.nbz + 2 * p.zg;
  // plane of the x / y records (shell index, ghost offset included)
  int64_t plane;
  if (outgoing) plane = (side == 0 ? 0 : g.nz - 1) + p.zg;
  else plane = side == 0 ? 0 : g.nz + 1;  // ghost planes -1 and nz
  // z records: outgoing low face = the down-exports (side 0) of brick row 0;
  // outgoing high face = the up-exports (side 1) of the top row; the ghost
  // of the low face holds the up-exports of the row below (side 1, row -1),
  // that of the high face the down-exports of the row above (side 0, row nbz)
  int64_t zside, zrow;
  if (outgoing) {
    zside = side;
    zrow = (side == 0 ? 0 : p.nbz - 1) + p.zg;
  } else {
    zside = side == 0 ? 1 : 0;
    zrow = side == 0 ? 0 : p.nbz + 1;
  }
  HaloMap m{};
  const int64_t sx_off = 0, sy_off = p.sx_elems, sz_off = p.sx_elems + p.sy_elems;
  m.rows[0] = 2LL * p.nbx * p.nxf;
  m.len[0] = g.ny;
  m.pitch[0] = nzs * g.ny;
  m.src[0] = sx_off + plane * g.ny;
  m.rows[1] = 2LL * p.nby * p.nyf;
  m.len[1] = g.nx;
  m.pitch[1] = nzs * g.nx;
  m.src[1] = sy_off + plane * g.nx;
  m.rows[2] = 1;
  m.len[2] = int64_t(p.nzf) * g.ny * g.nx;
  m.pitch[2] = 0;
  m.src[2] = sz_off + (zside * nbzs + zrow) * int64_t(p.nzf) * g.ny * g.nx;
  m.base[0] = 0;
  m.base[1] = m.rows[0] * m.len[0];
  m.base[2] = m.base[1] + m.rows[1] * m.len[1];
  m.total = m.base[2] + m.len[2];
  // the header names the layout; the sender's face is part of it, so that
  // an unpack can tell a message packed for the wrong side
  const int64_t h[kHeaderWords] = {kMagic, ctx->lattice, int64_t(ctx->real_bytes), g.nx, g.ny,
                                   int64_t(p.bx) << 32 | p.by, m.total, outgoing ? side : 1 - side};
  for (int k = 0; k < kHeaderWords; ++k) m.header[k] = h[k];
  return m;
}

// header + body, rounded up to 16 bytes so that messages laid out back to
// back in one buffer stay aligned
int64_t message_bytes(const lb_ctx* ctx) {
  const HaloMap m = halo_map(ctx, 0, true);
  return (int64_t(kHeaderWords) * 8 + m.total * int64_t(ctx->real_bytes) + 15) / 16 * 16;
}

// Grid-stride copy of the three regions; blockIdx.y selects the region.  On
// unpack every block first compares the message header with the expected
// one and copies nothing (recording LB_E_INVAL) on a mismatch.
template <class R>
__global__ void halo_copy_kernel(R* __restrict__ shell, unsigned char* __restrict__ msg, const __grid_constant__ HaloMap m,
                                 int to_msg, int* __restrict__ status) {
  int64_t* hdr = reinterpret_cast<int64_t*>(msg);
  R* body = reinterpret_cast<R*>(msg + kHeaderWords * 8);
  if (!to_msg) {
    bool ok = true;
    for (int k = 0; k < kHeaderWords; ++k) ok &= hdr[k] == m.header[k];
    if (!ok) {
      if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) atomicExch(status, LB_E_INVAL);
      return;
    }
  } else if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < kHeaderWords) {
    hdr[threadIdx.x] = m.header[threadIdx.x];
  }
  const int r = blockIdx.y;
  const int64_t n = m.rows[r] * m.len[r];
  const int64_t len = m.len[r];
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t row = i / len, col = i - row * len;
    const int64_t s = m.src[r] + row * m.pitch[r] + col;
    if (to_msg) body[m.base[r] + i] = shell[s];
    else shell[s] = body[m.base[r] + i];
  }
}

bool linked(const lb_ctx* ctx, int side) { return ctx->g.zlink[side] != 0; }

int halo_copy(lb_ctx* ctx, int side, void* buf, bool to_msg) {
  if (!ctx || !buf || side < 0 || side > 1) return LB_E_INVAL;
  if (ctx->scheme != LB_SCHEME_FUSED || !linked(ctx, side)) return LB_E_INVAL;
  if (reinterpret_cast<uintptr_t>(buf) % 16 != 0) return LB_E_INVAL;
  const HaloMap m = halo_map(ctx, side, to_msg);
  int64_t most = 0;
  for (int r = 0; r < 3; ++r) most = std::max(most, m.rows[r] * m.len[r]);
  const int bx = int(std::min<int64_t>(std::max<int64_t>((most + 255) / 256, 1), 152 * 8));
  const dim3 grid(unsigned(bx), 3);
  if (ctx->real_bytes == 8) {
    double* shell = static_cast<double*>(ctx->aux) + int64_t(ctx->parity) * ctx->plan.parity_elems;
    halo_copy_kernel<double><<<grid, 256, 0, ctx->stream>>>(shell, static_cast<unsigned char*>(buf), m,
                                                            to_msg ? 1 : 0, ctx->d_status);
  } else {
    float* shell = static_cast<float*>(ctx->aux) + int64_t(ctx->parity) * ctx->plan.parity_elems;
    halo_copy_kernel<float><<<grid, 256, 0, ctx->stream>>>(shell, static_cast<unsigned char*>(buf), m,
                                                           to_msg ? 1 : 0, ctx->d_status);
  }
  return cuda_status(cudaGetLastError());
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

struct lb_group {
  int nranks = 0;
  int device = 0;
  int slow = 2;  // user axis that is cut (z in 3D, y in 2D)
  std::vector<lb_ctx*> ctx;
  std::vector<int64_t> offset;
  // per rank and face: message buffer (device), neighbour rank (-1: none)
  std::vector<void*> buf[2];
  std::vector<int> nbr[2];
  std::vector<cudaEvent_t> packed, unpacked;
};

extern "C" {

int lb_halo_bytes(const lb_ctx* ctx, int64_t* bytes) {
  if (!ctx || !bytes || ctx->scheme != LB_SCHEME_FUSED) return LB_E_INVAL;
  *bytes = message_bytes(ctx);
  return LB_OK;
}

int lb_halo_pack(lb_ctx* ctx, int32_t side, void* buf) {
  if (!ctx) return LB_E_INVAL;
  DeviceGuard guard(ctx->device);
  return halo_copy(ctx, side, buf, true);
}

int lb_halo_unpack(lb_ctx* ctx, int32_t side, const void* buf) {
  if (!ctx) return LB_E_INVAL;
  DeviceGuard guard(ctx->device);
  return halo_copy(ctx, side, const_cast<void*>(buf), false);
}

void lb_group_destroy(lb_group* grp) {
  if (!grp) return;
  DeviceGuard guard(grp->device);
  for (lb_ctx* c : grp->ctx)
    if (c) lb_sync(c);
  for (int s = 0; s < 2; ++s)
    for (void* b : grp->buf[s])
      if (b) cudaFree(b);
  for (cudaEvent_t e : grp->packed)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : grp->unpacked)
    if (e) cudaEventDestroy(e);
  for (lb_ctx* c : grp->ctx) lb_destroy(c);
  delete grp;
}

int lb_group_create(int32_t lattice, const int64_t dims[3], double tau, const lb_boundary* bnd,
                    const lb_options* opt_in, int32_t nranks, const int64_t* counts, lb_group** out) {
  if (!out || !dims || nranks < 1) return LB_E_INVAL;
  *out = nullptr;
  if (lattice < LB_D2Q9 || lattice > LB_D3Q27) return LB_E_INVAL;
  const int d = lattice == LB_D2Q9 ? 2 : 3;
  const int slow = d - 1;
  const int64_t extent = dims[slow];
  if (extent < nranks) return LB_E_INVAL;
  std::vector<int64_t> cnt(size_t(nranks), 0);
  if (counts) {
    int64_t sum = 0;
    for (int r = 0; r < nranks; ++r) {
      if (counts[r] < 1) return LB_E_INVAL;
      cnt[size_t(r)] = counts[r];
      sum += counts[r];
    }
    if (sum != extent) return LB_E_INVAL;
  } else {
    for (int r = 0; r < nranks; ++r) cnt[size_t(r)] = extent / nranks + (r < extent % nranks ? 1 : 0);
  }
  lb_boundary b;
  if (bnd) b = *bnd;
  else std::memset(&b, 0, sizeof(b));
  for (int f = 0; f < 6; ++f)
    if (b.kind[f] == LB_LINK) return LB_E_INVAL;  // the group places the links
  lb_options opt;
  if (opt_in) opt = *opt_in;
  else lb_default_options(&opt);
  opt.stream = nullptr;
  if (opt.scheme != LB_SCHEME_FUSED) return LB_E_UNSUPPORTED;
  const bool periodic = b.kind[2 * slow] == LB_PERIODIC;

  lb_group* grp = new (std::nothrow) lb_group();
  if (!grp) return LB_E_NOMEM;
  grp->nranks = nranks;
  grp->slow = slow;
  int rc = LB_OK;
  int64_t off = 0;
  for (int r = 0; r < nranks && rc == LB_OK; ++r) {
    int64_t rd[3] = {dims[0], dims[1], dims[2]};
    rd[slow] = cnt[size_t(r)];
    lb_boundary rb = b;
    const bool lo_link = r > 0 || periodic, hi_link = r < nranks - 1 || periodic;
    rb.kind[2 * slow] = lo_link ? LB_LINK : b.kind[2 * slow];
    rb.kind[2 * slow + 1] = hi_link ? LB_LINK : b.kind[2 * slow + 1];
    lb_ctx* c = nullptr;
    rc = lb_create(lattice, rd, tau, &rb, &opt, &c);
    if (rc != LB_OK) break;
    grp->ctx.push_back(c);
    grp->offset.push_back(off);
    off += cnt[size_t(r)];
    if (r == 0) {
      // every rank shares rank 0's brick cross-section (the halo layout)
      opt.tile[0] = c->plan.bx;
      opt.tile[1] = c->plan.by;
      grp->device = c->device;
    } else if (c->plan.bx != grp->ctx[0]->plan.bx || c->plan.by != grp->ctx[0]->plan.by ||
               c->plan.npt != grp->ctx[0]->plan.npt) {
      rc = LB_E_UNSUPPORTED;
    }
  }
  DeviceGuard guard(grp->device);
  for (int s = 0; s < 2; ++s) {
    grp->buf[s].assign(size_t(nranks), nullptr);
    grp->nbr[s].assign(size_t(nranks), -1);
  }
  grp->packed.assign(size_t(nranks), nullptr);
  grp->unpacked.assign(size_t(nranks), nullptr);
  for (int r = 0; r < nranks && rc == LB_OK; ++r) {
    lb_ctx* c = grp->ctx[size_t(r)];
    for (int s = 0; s < 2 && rc == LB_OK; ++s) {
      if (!c->g.zlink[s]) continue;
      grp->nbr[s][size_t(r)] = s == 0 ? (r + nranks - 1) % nranks : (r + 1) % nranks;
      rc = cuda_status(cudaMalloc(&grp->buf[s][size_t(r)], size_t(message_bytes(c))));
    }
    if (rc == LB_OK) rc = cuda_status(cudaEventCreateWithFlags(&grp->packed[size_t(r)], cudaEventDisableTiming));
    if (rc == LB_OK) rc = cuda_status(cudaEventCreateWithFlags(&grp->unpacked[size_t(r)], cudaEventDisableTiming));
  }
  if (rc != LB_OK) {
    lb_group_destroy(grp);
    return rc;
  }
  *out = grp;
  return LB_OK;
}

int lb_group_rank(lb_group* grp, int32_t rank, lb_ctx** ctx, int64_t* offset) {
  if (!grp || rank < 0 || rank >= grp->nranks) return LB_E_INVAL;
  if (ctx) *ctx = grp->ctx[size_t(rank)];
  if (offset) *offset = grp->offset[size_t(rank)];
  return LB_OK;
}

int lb_group_step(lb_group* grp, int64_t n) {
  if (!grp || n < 0) return LB_E_INVAL;
  DeviceGuard guard(grp->device);
  const int R = grp->nranks;
  for (int64_t t = 0; t < n; ++t) {
    // pack: after the neighbours consumed this rank's previous messages
    for (int r = 0; r < R; ++r) {
      lb_ctx* c = grp->ctx[size_t(r)];
      bool any = false;
      for (int s = 0; s < 2; ++s) {
        const int nb = grp->nbr[s][size_t(r)];
        if (nb < 0) continue;
        any = true;
        if (nb != r) {
          const cudaError_t e = cudaStreamWaitEvent(c->stream, grp->unpacked[size_t(nb)], 0);
          if (e != cudaSuccess) return cuda_status(e);
        }
        const int rc = halo_copy(c, s, grp->buf[s][size_t(r)], true);
        if (rc != LB_OK) return rc;
      }
      if (any) {
        const cudaError_t e = cudaEventRecord(grp->packed[size_t(r)], c->stream);
        if (e != cudaSuccess) return cuda_status(e);
      }
    }
    // unpack the neighbours' messages, then step
    for (int r = 0; r < R; ++r) {
      lb_ctx* c = grp->ctx[size_t(r)];
      bool any = false;
      for (int s = 0; s < 2; ++s) {
        const int nb = grp->nbr[s][size_t(r)];
        if (nb < 0) continue;
        any = true;
        if (nb != r) {
          const cudaError_t e = cudaStreamWaitEvent(c->stream, grp->packed[size_t(nb)], 0);
          if (e != cudaSuccess) return cuda_status(e);
        }
        // the low face receives the neighbour's high-face message and back
        const int rc = halo_copy(c, s, grp->buf[1 - s][size_t(nb)], false);
        if (rc != LB_OK) return rc;
      }
      if (any) {
        const cudaError_t e = cudaEventRecord(grp->unpacked[size_t(r)], c->stream);
        if (e != cudaSuccess) return cuda_status(e);
      }
      const int rc = lb_step(c, 1);
      if (rc != LB_OK) return rc;
    }
  }
  return LB_OK;
}

int lb_group_sync(lb_group* grp) {
  if (!grp) return LB_E_INVAL;
  int first = LB_OK;
  for (lb_ctx* c : grp->ctx) {
    const int rc = lb_sync(c);
    if (first == LB_OK && rc != LB_OK) first = rc;
  }
  return first;
}

}  // extern "C"
