// lb_k1.cuh -- the fused single-array step: pull-stream + regularized
// collision + bounce-back in one launch per time step.
//
// The paper (section 3) observes that the post-collision set of a node is a
// function of its moments alone, so a step can rebuild every population from
// the upstream node's state (the multline step equation; Eq. pushLB as a
// pull).  The paper realises this with two launches and full-size moment
// arrays (section 4).  Here the same rebuild runs in ONE launch over the one
// population array:
//
//   * the grid is cut into brick columns of bx x by nodes and bz planes; a CTA
//     owns one brick and is the only reader and writer of its populations in
//     a launch, so the in-place update is race free;
//   * the CTA sweeps its planes along z.  TMA streams plane z + NS of the
//     population array into a ring of shared-memory slots (mbarrier
//     complete-tx); every thread collides its node of plane z
//     (lb_collide.cuh) into a padded shared window whose one-node ring holds
//     the collided populations of the neighbouring bricks (from the shell, see
//     below); each thread then gathers, for each direction a, the value of
//     its upstream neighbour x - c_a with no branches.  The value belongs to
//     destination plane z + c_az, so three destination planes live in
//     registers and plane z - 1 is stored once complete.  Populations that do
//     not move laterally (rest, +-z) never leave the registers;
//   * cross-brick exchange: after finishing a boundary node, its owner
//     collides the new state once more and exports the populations whose c_a
//     points out of the brick into the other parity of a small "shell"
//     buffer, which neighbouring bricks read in the NEXT launch.  The lateral
//     boundary nodes of a plane are staged in shared memory and exported by a
//     few whole warps, so no warp diverges on its edge lanes; the bottom and
//     top planes of a brick export along z with every thread;
//   * halfway bounce-back (and the moving-wall term) overwrites the gathered
//     value where the upstream point lies outside a non-periodic face, in a
//     pass that only threads next to a wall take.
// Every wait is bounded; on timeout the CTA records LB_E_TIMEOUT in a status
// word, drains its own outstanding copies (bounded) and exits.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "lb_dispatch.cuh"
#include "lb_ptx.cuh"

namespace lbgb {

template <class R>
struct K1Args {
  Phys<R> ph;
  int nx, ny, nz;
  int64_t pitch, vol;
  int per[3];
  // z faces that border another context's slab (a rank boundary): their
  // incoming shell records sit in ghost slots -- plane -1 / nz of the x and
  // y records, brick row -1 / nbz of the z records -- filled between
  // launches by lb_halo_unpack.  zg = 1 when a context has ghost slots (the
  // shell's planes and brick rows are then shifted by one), nzs = nz + 2 zg
  // planes per x / y record, nbzs = nbz + 2 zg brick rows per z-record side.
  int zlink[2];
  int zg, nzs, nbzs;
  // per-plane tests read from the parameter bank (no registers in the
  // sweep): the plane of a wall at the -z / +z face (0 / nz - 1; -1 where
  // that face is periodic or a link), and nz where z wraps (periodic), else 0
  int zwl, zwh, zwrap;
  int bz, nbx, nby, nbz;
  void* f;
  const R* sh_cur;
  R* sh_next;
  int64_t sx_off, sy_off, sz_off;
  int* status;
  R bb[27][8];
  uint32_t vol32;  // vol / 32 (rows are padded to 32 elements)
};

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

__host__ __device__ constexpr size_t align128(size_t v) { return (v + 127) & ~size_t(127); }

// lateral directions (moving along x or y) get a plane of the shared window
template <class L>
LB_HD constexpr bool is_lateral(int a) { return L::cx(a) != 0 || L::cy(a) != 0; }
template <class L>
LB_HD constexpr int n_lateral() {
  int n = 0;
  for (int a = 0; a < L::Q; ++a) n += is_lateral<L>(a) ? 1 : 0;
  return n;
}
template <class L>
LB_HD constexpr int lat_index(int a) {
  int n = 0;
  for (int b = 0; b < a; ++b) n += is_lateral<L>(b) ? 1 : 0;
  return n;
}
// lateral window slot of the ia-th direction whose component along axis is
// sign, for a run-time ia: a chain of compile-time candidates, so that no
// lattice table is laid out in local memory
template <class L, int axis, int sign>
__device__ __forceinline__ int lat_slot_of_sub(int ia) {
  int r = 0;
  static_for<0, L::Q>([&](auto A_) {
    constexpr int a = decltype(A_)::value;
    if constexpr (comp<L>(axis, a) == sign) {
      if (ia == sub_index<L>(axis, sign, a)) r = lat_index<L>(a);
    }
  });
  return r;
}

// MINB: CTAs the shape is compiled to keep resident on one SM (registers
// capped at 64K / (MINB x threads), shared memory within 228 KB / MINB)
template <class L, class S, class R, int BX, int BY, int NS, int WB, int NXW, int TS = 0, int MINB = 1>
struct K1Shape {
  static constexpr int Q = L::Q;
  static constexpr int NTM = BX * BY;  // threads that own a node
  // dedicated export warps after the node warps: NXW > 0 of them decoupled
  // from the node warps' per-plane barrier, or -NXW (NXW < 0) that pass the
  // same barrier and own no node
  static constexpr int XW = NXW < 0 ? -NXW : NXW;
  static constexpr int NT = NTM + 32 * XW;
  static constexpr int NW = NTM / 32;  // node warps
  static constexpr int NXF = count_dirs<L>(0, 1);
  static constexpr int NYF = count_dirs<L>(1, 1);
  static constexpr int NZF = count_dirs<L>(2, 1);
  static constexpr int NLAT = n_lateral<L>();
  static constexpr int PY = NYF > 0 ? 1 : 0;  // window padding rows (none without y motion)
  static constexpr int WX = BX + 2;
  static constexpr int WY = BY + 2 * PY;
  static constexpr int WPLANE = WY * WX;
  static constexpr int HW = NXF * WY;  // west (and east) ring entries
  static constexpr int HS = NYF * BX;  // south (and north) ring entries
  static constexpr int H = 2 * HW + 2 * HS;
  static constexpr int HPT = (H + NTM - 1) / NTM;
  static constexpr int PMAX = NYF > 0 ? 2 * BX + 2 * (BY - 2) : 2;  // lateral perimeter nodes
  // lateral export entries, one per (perimeter node, face): segments W, E,
  // S, N, each starting on a warp boundary in 3D so that every export warp
  // writes a single face (a corner node has an entry in two segments)
  static constexpr int SEGY = NYF > 0 ? (BY + 31) / 32 * 32 : 1;
  static constexpr int SEGX = NYF > 0 ? (BX + 31) / 32 * 32 : 0;
  static constexpr int PE = 2 * SEGY + 2 * SEGX;
  // export warps: NEXW node-owning warps, or the XW dedicated ones
  static constexpr int NEXW = NXW != 0 ? XW : (PE + 31) / 32;
  // shared export warps start at warp EXW0: past the first brick row, whose
  // warps also stage a whole row of perimeter nodes every plane
  static constexpr int EXW0 = (NTM / 32 >= NEXW + 4 && BY >= 4) ? 2 : 0;
  // Which warps export (bit w: warp w).  Shared export warps are spread over
  // the four schedulers of the SM (warp w issues on scheduler w % 4): each
  // goes to the scheduler with the least work so far, counting a node warp
  // as 2 and an export warp's extra work as 1, ties to the lowest free warp.
  // A CTA of 14 node warps (4, 4, 3, 3 per scheduler) thus puts its four
  // export warps on the two lighter schedulers.
  static constexpr uint64_t shared_export_mask() {
    int load[4] = {0, 0, 0, 0};
    for (int w = 0; w < NW; ++w) load[w % 4] += 2;
    uint64_t m = 0;
    for (int k = 0; k < NEXW; ++k) {
      int best = -1;
      for (int w = EXW0; w < NW; ++w) {
        if ((m >> w) & 1) continue;
        if (best < 0 || load[w % 4] < load[best % 4]) best = w;
      }
      if (best < 0) break;
      m |= uint64_t(1) << best;
      load[best % 4] += 1;
    }
    return m;
  }
  static constexpr uint64_t EXMASK =
      NXW != 0 ? (((uint64_t(1) << XW) - 1) << NW) : shared_export_mask();
  // the lowest export warp, and whether the export warps are consecutive
  static constexpr int EXFIRST = [] {
    int w = 0;
    while (w < 63 && !((EXMASK >> w) & 1)) ++w;
    return w;
  }();
  static constexpr bool EXCONTIG = (EXMASK >> EXFIRST) == (uint64_t(1) << NEXW) - 1;
  // stage row of one perimeter node: Q values padded so that the row is a
  // whole, odd number of 16-byte units (vector stores, conflict-free loads)
  static constexpr int VEC = 16 / int(sizeof(R));
  static constexpr int QP = ((Q + VEC - 1) / VEC) % 2 == 1 ? (Q + VEC - 1) / VEC * VEC : ((Q + VEC - 1) / VEC + 1) * VEC;
  static constexpr size_t SLOT = size_t(Q) * BY * BX * sizeof(S);
  static constexpr size_t WIN = size_t(NLAT) * WPLANE * sizeof(R);
  static constexpr size_t STAGE = size_t(QP) * PMAX * sizeof(R);
  static constexpr size_t OFF_WIN = align128(NS * SLOT);
  // with dedicated export warps the lateral export runs decoupled from the
  // node warps' per-plane barrier, through a ring of SR staged planes
  // guarded by full / empty mbarriers; otherwise two staged planes suffice
  static constexpr bool DEC = NXW > 0;
  static constexpr int SR = DEC ? 4 : 2;
  static constexpr size_t OFF_STAGE = OFF_WIN + WB * align128(WIN);
  static constexpr size_t OFF_DESC = OFF_STAGE + align128(SR * STAGE);
  static constexpr size_t OFF_BAR = OFF_DESC + align128(size_t(PE) * 12);
  // TS: the completed plane leaves through a shared-memory output buffer and
  // one TMA store instead of per-thread global stores
  static constexpr size_t OFF_OUT = OFF_BAR + align128((NS + 2 * SR + 1) * sizeof(uint64_t));
  static constexpr size_t SMEM0 = OFF_OUT + (TS ? align128(SLOT) : 0);
  // halo-ring entries: with room in shared memory, each thread keeps its
  // entries' global pointer and z stride there (16 B per entry, read once
  // per plane) instead of in registers -- for up to 19 velocities (measured:
  // FP16 D3Q19 2 % faster, D3Q27 with three entries per thread 1 % slower)
  static constexpr size_t HDESC = size_t(HPT) * NT * 16;
  static constexpr size_t SMEM_CAP = (size_t(228) * 1024) / MINB - 1024;
  static constexpr bool HSMEM = SMEM0 + HDESC <= SMEM_CAP && Q <= 19;
  static constexpr size_t OFF_HDESC = SMEM0;
  static constexpr size_t SMEM = SMEM0 + (HSMEM ? HDESC : 0);
  // the plane sweep runs three planes per loop trip (the three gathered
  // sets change roles at compile time instead of being copied every plane)
  // where the three copies of the body still fit the registers: up to 19
  // FP32 arithmetic values per node, or 27 in a CTA of at most 256 threads
  static constexpr bool UNROLL3 = (Q * sizeof(R) <= 76 || (Q * sizeof(R) <= 108 && NT * MINB <= 256));
  // 16-bit storage addresses each population store as one wide multiply-add
  // of vol / 32 by a constant; the others walk one pointer along the
  // directions.  Measured at 1024^3 on one GPU, multiply-add against pointer
  // walk: D3Q27 FP16 30.3 / 28.8, D3Q19 BF16 37.5 / 36.5, but D3Q19 FP16
  // 39.5 / 40.4 and D3Q19 FP32 35.3 / 36.1 GLUPS, so those keep the walk
  static constexpr bool WIDE_STORE = sizeof(S) == 2 && !(Q == 19 && std::is_same<S, __half>::value);
  static_assert(SMEM <= SMEM_CAP, "shared memory of the shape exceeds its share of the SM");
  static_assert(BY == 1 || NYF > 0, "a 2D brick has one internal row");
  static_assert(NXW != 0 || 32 * NEXW <= NTM, "export entries need more warps than the CTA has");
  static_assert(NTM % 32 == 0 && NW + XW <= 32, "node threads fill whole warps");
  static_assert(WB == 1 || WB == 2, "one or two window buffers");
};

// index of the lateral perimeter node (tx, ty) of an active bxa x bya brick
template <int NYF>
__device__ __forceinline__ int perimeter_index(int tx, int ty, int bxa, int bya) {
  if (NYF == 0) return (tx == 0) ? 0 : (tx == bxa - 1 ? 1 : -1);
  const int m = bxa >= 2 ? 2 : 1;
  if (ty == 0) return tx;
  if (ty == bya - 1) return bxa + tx;
  if (tx == 0) return bxa * 2 + (ty - 1) * m;
  if (tx == bxa - 1) return bxa * 2 + (ty - 1) * m + 1;
  return -1;
}
template <int NYF>
__device__ __forceinline__ int perimeter_count(int bxa, int bya) {
  if (NYF == 0) return bxa >= 2 ? 2 : 1;
  const int m = bxa >= 2 ? 2 : 1;
  return bxa * (bya >= 2 ? 2 : 1) + (bya > 2 ? bya - 2 : 0) * m;
}
template <int NYF>
__device__ __forceinline__ void perimeter_node(int p, int bxa, int bya, int& tx, int& ty) {
  if (NYF == 0) {
    tx = (p == 0) ? 0 : bxa - 1;
    ty = 0;
    return;
  }
  const int m = bxa >= 2 ? 2 : 1;
  if (p < bxa) {
    tx = p;
    ty = 0;
  } else if (bya >= 2 && p < 2 * bxa) {
    tx = p - bxa;
    ty = bya - 1;
  } else {
    const int q = p - bxa * (bya >= 2 ? 2 : 1);
    ty = 1 + q / m;
    tx = (q % m == 0) ? 0 : bxa - 1;
  }
}

// Faces of a brick through which a boundary node exports (bit flags).
enum : unsigned { kFaceW = 1, kFaceE = 2, kFaceS = 4, kFaceN = 8, kFaceD = 16, kFaceU = 32 };

// Shell offsets of one node, hoisted out of the per-direction stores: the
// ia-th exported direction of a face lands at base + ia * stride.
template <class R>
struct ShellSpot {
  R* base;
  int64_t stride;
};

// Write the directions of one face: those whose component along `axis` is
// `sign` (the populations leaving through that face).
template <class L, class R, int axis, int sign>
__device__ __forceinline__ void export_face(const Coef<R>& kc, ShellSpot<R> s) {
  static_for<0, L::Q>([&](auto A_) {
    constexpr int a = decltype(A_)::value;
    if constexpr (comp<L>(axis, a) == sign) {
      constexpr int ia = sub_index<L>(axis, sign, a);
      s.base[ia * s.stride] = post<L, R, a>(kc);
    }
  });
}

// Collide the completed (rounded) state of one node once more and export the
// populations that leave the brick through the flagged faces.
template <class L, class S, class R, bool FORCE, bool LINK = false>
__device__ __forceinline__ void export_node(const K1Args<R>& args, const R (&fin)[L::Q], int x, int y, int zd,
                                            unsigned faces, int bI, int bJ, int bK) {
  constexpr int NXF = count_dirs<L>(0, 1), NYF = count_dirs<L>(1, 1), NZF = count_dirs<L>(2, 1);
  R fr[L::Q];
  static_for<0, L::Q>([&](auto A_) {
    constexpr int a = decltype(A_)::value;
    fr[a] = round_to_storage<S, R>(fin[a]);
  });
  Mom<R> m;
  moments<L, R, FORCE>(fr, args.ph, m);
  Coef<R> kc;
  coeffs<L, R, FORCE>(m, args.ph, kc);
  R* shn = args.sh_next;
  // LINK: the shell of a slab context, with ghost planes / brick rows
  const int zg = LINK ? args.zg : 0;
  const int64_t nzy = int64_t(LINK ? args.nzs : args.nz) * args.ny;
  const int64_t nzx = int64_t(LINK ? args.nzs : args.nz) * args.nx;
  const int64_t nyx = int64_t(args.ny) * args.nx;
  if (faces & (kFaceW | kFaceE)) {
    // SX[side][I][ia][z + zg][y]
    const int64_t row = int64_t(zd + zg) * args.ny + y;
    if (faces & kFaceW)
      export_face<L, R, 0, -1>(kc, {shn + args.sx_off + (int64_t(bI) * NXF) * nzy + row, nzy});
    if (faces & kFaceE)
      export_face<L, R, 0, 1>(kc, {shn + args.sx_off + ((int64_t(args.nbx) + bI) * NXF) * nzy + row, nzy});
  }
  if constexpr (NYF > 0) {
    if (faces & (kFaceS | kFaceN)) {
      // SY[side][J][ia][z + zg][x]
      const int64_t row = int64_t(zd + zg) * args.nx + x;
      if (faces & kFaceS)
        export_face<L, R, 1, -1>(kc, {shn + args.sy_off + (int64_t(bJ) * NYF) * nzx + row, nzx});
      if (faces & kFaceN)
        export_face<L, R, 1, 1>(kc, {shn + args.sy_off + ((int64_t(args.nby) + bJ) * NYF) * nzx + row, nzx});
    }
  }
  if (faces & (kFaceD | kFaceU)) {
    // SZ[side][K + zg][ia][y][x]
    const int64_t row = int64_t(y) * args.nx + x;
    if (faces & kFaceD)
      export_face<L, R, 2, -1>(kc, {shn + args.sz_off + (int64_t(bK + zg) * NZF) * nyx + row, nyx});
    if (faces & kFaceU)
      export_face<L, R, 2, 1>(
          kc, {shn + args.sz_off + ((int64_t(LINK ? args.nbzs : args.nbz) + bK + zg) * NZF) * nyx + row, nyx});
  }
}

// Export entry e of a brick shape: its face (0 W, 1 E, 2 S, 3 N) and the
// first entry of that face's segment.
template <class Sh>
__device__ __forceinline__ int export_face_of(int e) {
  if (e < Sh::SEGY) return 0;
  if (e < 2 * Sh::SEGY) return 1;
  return e < 2 * Sh::SEGY + Sh::SEGX ? 2 : 3;
}
template <class Sh>
__device__ __forceinline__ int export_seg_start(int face) {
  return face < 2 ? face * Sh::SEGY : 2 * Sh::SEGY + (face - 2) * Sh::SEGX;
}

// Collide the completed (rounded) state of a lateral perimeter node once more
// and export the populations that leave through one face; dst is the node's
// record of that face in this plane, stride the distance between directions.
template <class L, class S, class R, bool FORCE>
__device__ __forceinline__ void export_one_face(const Phys<R>& ph, const R (&fin)[L::Q], int face, R* dst,
                                                int64_t stride) {
  R fr[L::Q];
  static_for<0, L::Q>([&](auto A_) {
    constexpr int a = decltype(A_)::value;
    fr[a] = round_to_storage<S, R>(fin[a]);
  });
  Mom<R> m;
  moments<L, R, FORCE>(fr, ph, m);
  Coef<R> kc;
  coeffs<L, R, FORCE>(m, ph, kc);
  if (face == 0) export_face<L, R, 0, -1>(kc, {dst, stride});
  else if (face == 1) export_face<L, R, 0, 1>(kc, {dst, stride});
  if constexpr (count_dirs<L>(1, 1) > 0) {
    if (face == 2) export_face<L, R, 1, -1>(kc, {dst, stride});
    else if (face == 3) export_face<L, R, 1, 1>(kc, {dst, stride});
  }
}

// The sweep of one brick column (bI, bJ, bK) of one domain by the whole CTA.
// tmap_p is the domain's TMA descriptor (kernel-parameter or global memory).
// Returns false if a TMA wait timed out (the CTA recorded LB_E_TIMEOUT and
// must stop).  On return every copy the brick issued has completed and the
// mbarriers are invalidated, so the CTA may start another brick.
//
// LINK: compiled for contexts with a link face (slab decomposition); the
// other instantiations compile the plain form, whose shell has no ghosts.
//
// PHPLANE: the arguments sit in shared memory (batched sweeps); the collision
// then reads its physical constants as one block copy at the start of each
// use (loads issued ahead of the collision, not one per operand inside it).
template <class L, class S, class R, int BX, int BY, int NS, int WB, int NXW, bool FORCE, int TS = 0,
          bool LINK = false, int MINB = 1, bool PHPLANE = false>
__device__ __forceinline__ bool k1_brick(const CUtensorMap* tmap_p, const K1Args<R>& args, const int bI,
                                         const int bJ, const int bK) {
  using Sh = K1Shape<L, S, R, BX, BY, NS, WB, NXW, TS, MINB>;
  static_assert(WB == 2, "the pipelined sweep needs two window buffers");
  constexpr int Q = L::Q;
  constexpr int NTM = Sh::NTM;
  constexpr int NXF = Sh::NXF, NYF = Sh::NYF, NZF = Sh::NZF;
  constexpr int PY = Sh::PY, WX = Sh::WX, WPLANE = Sh::WPLANE;
  constexpr int HW = Sh::HW, HS = Sh::HS, H = Sh::H, HPT = Sh::HPT;
  constexpr int PMAX = Sh::PMAX, NEXW = Sh::NEXW, QP = Sh::QP, VEC = Sh::VEC, PE = Sh::PE;
  constexpr int WY = Sh::WY;
  constexpr int WSTRIDE = int(align128(Sh::WIN) / sizeof(R));  // between window buffers
  using Vec = typename std::conditional<sizeof(R) == 4, float4, double2>::type;

  extern __shared__ __align__(128) unsigned char smem[];
  S* slots = reinterpret_cast<S*>(smem);
  R* win0 = reinterpret_cast<R*>(smem + Sh::OFF_WIN);
  R* stage = reinterpret_cast<R*>(smem + Sh::OFF_STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR);
  // per export entry: shell offset (plane 0) of the face record, and the
  // stage row of the node (-1: no neighbour across that face)
  int64_t* desc_off = reinterpret_cast<int64_t*>(smem + Sh::OFF_DESC);
  int* desc_p = reinterpret_cast<int*>(smem + Sh::OFF_DESC + size_t(PE) * 8);

  const int tid = threadIdx.x;
  // owns node (tx, ty); the rest only export (all threads without dedicated
  // export warps: the launch has exactly NTM threads then)
  const bool is_main = NXW == 0 || tid < NTM;
  const int tx = tid % BX;
  const int ty = is_main ? tid / BX : BY;
  const int warp = tid / 32, lane = tid % 32;
  const int nx = args.nx, ny = args.ny, nz = args.nz;
  const int nbx = args.nbx, nby = args.nby, nbz = args.nbz;
  const int x0 = bI * BX, y0 = bJ * BY, z0 = bK * args.bz;
  const int bxa = min(BX, nx - x0), bya = min(BY, ny - y0);
  const int z1 = min(z0 + args.bz, nz);
  const int x = x0 + tx, y = y0 + ty;
  const bool active = tx < bxa && ty < bya;

  // which neighbouring bricks exist (periodic wrap counts)
  const bool nbW = x0 > 0 || args.per[0];
  const bool nbE = x0 + bxa < nx || args.per[0];
  const bool nbS = y0 > 0 || args.per[1];
  const bool nbN = y0 + bya < ny || args.per[1];
  const bool nbD = z0 > 0 || args.per[2] || (LINK && args.zlink[0]);
  const bool nbU = z1 < nz || args.per[2] || (LINK && args.zlink[1]);
  const int bIw = (bI + nbx - 1) % nbx, bIe = (bI + 1) % nbx;
  const int bJs = (bJ + nby - 1) % nby, bJn = (bJ + 1) % nby;
  // the brick rows below / above (a link face's ghost row is -1 / nbz)
  const int bKd = (LINK && !args.per[2]) ? bK - 1 : (bK + nbz - 1) % nbz;
  const int bKu = (LINK && !args.per[2]) ? bK + 1 : (bK + 1) % nbz;
  // shell planes per x / y record and brick rows per z-record side
  const int nzs = LINK ? args.nzs : nz;
  const int nbzs = LINK ? args.nbzs : nbz;
  const int zg = LINK ? args.zg : 0;

  // bounce-back predicates of this node along x and y: the upstream point of
  // a direction with c = +1 is x - 1, which leaves a non-periodic low face at x = 0
  const bool bxlo = active && (x == 0) && !args.per[0];
  const bool bxhi = active && (x == nx - 1) && !args.per[0];
  const bool bylo = active && (y == 0) && !args.per[1];
  const bool byhi = active && (y == ny - 1) && !args.per[1];
  const bool xy_wall = bxlo || bxhi || bylo || byhi;
  const bool z_walls = !args.per[2];

  S* __restrict__ fglob = static_cast<S*>(args.f);
  const R* __restrict__ shc = args.sh_cur;

  // ---------------------------------------------------------------- setup
  constexpr bool DEC = Sh::DEC;
  constexpr int SR = Sh::SR;
  uint64_t* sfull = bars + NS;        // staged plane ready (node threads arrive)
  uint64_t* sempty = bars + NS + SR;  // staged plane exported (export threads arrive)
  uint64_t* outfree = bars + NS + 2 * SR;  // output buffer read by the last TMA store
  S* outbuf = reinterpret_cast<S*>(smem + Sh::OFF_OUT);
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    if constexpr (TS != 0) mbar_init(outfree, 1);
    if constexpr (DEC) {
      for (int s = 0; s < SR; ++s) {
        mbar_init(&sfull[s], NTM);
        mbar_init(&sempty[s], 32 * NXW);
      }
    }
    fence_barrier_init();
    prefetch_tmap(tmap_p);
  }
  __syncthreads();
  // the node threads' per-plane barrier: the whole CTA, or only the node
  // warps when dedicated export warps run decoupled
  auto node_sync_or = [&](bool pred) -> bool {
    if constexpr (DEC) return bar_red_or(1, NTM, pred);
    else return __syncthreads_or(pred);
  };
  int issued = 0;  // real planes whose load was issued (thread 0's view)
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      const int zz = z0 + s;
      if (zz < z1) {
        mbar_arrive_expect_tx(&bars[s], static_cast<uint32_t>(Sh::SLOT));
        tma_load_4d(slots + size_t(s) * Q * BY * BX, tmap_p, x0, y0, zz, 0, &bars[s]);
        ++issued;
      }
    }
  }

  // ring entries of the window: entry h -> (global base, z stride, window index)
  int64_t hbase[HPT];
  int hzs[HPT];
  int hsm[HPT];
  bool hval[HPT];
  struct HaloDesc {
    const R* ptr;  // plane-0 element of the entry's shell record; null: no entry
    int64_t zs;    // elements between consecutive planes
  };
  HaloDesc* hdesc = reinterpret_cast<HaloDesc*>(smem + Sh::OFF_HDESC);
#pragma unroll
  for (int e = 0; e < HPT; ++e) {
    // later rounds of ring entries go to the last threads, away from the
    // export warps at the front of the CTA
    const int h = is_main ? (e == 0 ? tid : (NTM - 1 - tid) + e * NTM) : H;
    hval[e] = false;
    hbase[e] = 0;
    hzs[e] = 1;
    hsm[e] = 0;
    if (h < H) {
      if (h < 2 * HW) {
        const bool west = h < HW;
        const int hh = west ? h : h - HW;
        const int ia = hh / WY;
        const int r = hh % WY;  // window row; source y = y0 - PY + r
        int sy = y0 - PY + r;
        bool ok = (west ? nbW : nbE) && r < bya + 2 * PY;
        if (sy < 0 || sy >= ny) {
          if (args.per[1]) sy = (sy + ny) % ny;
          else ok = false;
        }
        const int col = west ? 0 : bxa + 1;
        // the west ring holds the high-face export (side 1) of the west brick
        const int side = west ? 1 : 0;
        const int bb = west ? bIw : bIe;
        hval[e] = ok;
        hbase[e] = args.sx_off + ((int64_t(side) * nbx + bb) * NXF + ia) * int64_t(nzs) * ny + int64_t(zg) * ny + sy;
        hzs[e] = ny;
        hsm[e] = (west ? lat_slot_of_sub<L, 0, 1>(ia) : lat_slot_of_sub<L, 0, -1>(ia)) * WPLANE + r * WX + col;
      } else {
        const int h2 = h - 2 * HW;
        const bool south = h2 < HS;
        const int hh = south ? h2 : h2 - HS;
        const int ia = hh / BX;
        const int i = hh % BX;
        const bool ok = (south ? nbS : nbN) && i < bxa;
        const int row = south ? 0 : bya + 1;
        const int side = south ? 1 : 0;
        const int bb = south ? bJs : bJn;
        hval[e] = ok;
        hbase[e] = args.sy_off + ((int64_t(side) * nby + bb) * NYF + ia) * int64_t(nzs) * nx + int64_t(zg) * nx + x0 + i;
        hzs[e] = nx;
        hsm[e] = (south ? lat_slot_of_sub<L, 1, 1>(ia) : lat_slot_of_sub<L, 1, -1>(ia)) * WPLANE + row * WX + 1 + i;
      }
    }
  }

  auto plane_needed = [&](int z) -> bool {
    if (z >= z0 && z < z1) return true;
    if (z == z0 - 1) return nbD;
    if (z == z1) return nbU;
    return false;
  };

  // ring values of two planes ahead in registers: ha = plane being produced,
  // hb = the next one (loads in flight for about two planes).  The entry
  // pointers walk up one plane per call; planes below 0 or above nz - 1 only
  // occur for periodic z, and wrap, or at a link face, where they are the
  // ghost planes -1 / nz.
  R ha[HPT], hb[HPT];
  const R* hptr[HPT];
#pragma unroll
  for (int e = 0; e < HPT; ++e) {
    hptr[e] = shc + hbase[e];
    if constexpr (Sh::HSMEM) {
      hdesc[e * Sh::NT + tid] = HaloDesc{hval[e] ? hptr[e] : nullptr, int64_t(hzs[e])};
      if (!hval[e]) hsm[e] = -1;
    }
  }
  auto halo_fetch = [&](R(&dst)[HPT], int z) {
    const bool ok = z <= z1 && plane_needed(z);
    const int zw = LINK ? (z < 0 ? z + args.zwrap : (z >= nz ? z - args.zwrap : z))
                        : (z < 0 ? z + nz : (z >= nz ? z - nz : z));
#pragma unroll
    for (int e = 0; e < HPT; ++e) {
      if constexpr (Sh::HSMEM) {
        const HaloDesc d = hdesc[e * Sh::NT + tid];
        dst[e] = (ok && d.ptr) ? d.ptr[int64_t(zw) * d.zs] : R(0);
      } else {
        dst[e] = (ok && hval[e]) ? hptr[e][int64_t(zw) * hzs[e]] : R(0);
      }
    }
  };
  halo_fetch(ha, z0 - 1);
  halo_fetch(hb, z0);

  // perimeter (lateral boundary) slot of this node, and export-warp work
  const int pidx = active ? perimeter_index<NYF>(tx, ty, bxa, bya) : -1;
  const bool any_lateral_export = nbW || nbE || (NYF > 0 && (nbS || nbN));
  // export warps take the entries in warp order; exp_lane is this lane's first
  bool exp_warp;
  int exp_lane;
  if constexpr (NXW > 0) {
    exp_warp = any_lateral_export && !is_main;
    exp_lane = tid - NTM;
  } else if constexpr (Sh::EXCONTIG) {
    exp_warp = any_lateral_export && warp >= Sh::EXFIRST && warp < Sh::EXFIRST + NEXW;
    exp_lane = (warp - Sh::EXFIRST) * 32 + lane;
  } else {
    exp_warp = any_lateral_export && ((Sh::EXMASK >> warp) & 1);
    exp_lane = __popcll(Sh::EXMASK & ((uint64_t(1) << warp) - 1)) * 32 + lane;
  }

  // this thread's own cell in the window (interior of the padding ring)
  const int wbase = (ty + PY) * WX + (tx + 1);

  // export of the staged lateral perimeter of plane zx (whole warps)
  // resolve each perimeter node's shell records once per brick
  const int64_t nzy = int64_t(nzs) * ny, nzx = int64_t(nzs) * nx;
  if (exp_warp) {
#pragma unroll 1
    for (int e = exp_lane; e < PE; e += 32 * Sh::NEXW) {
      const int face = export_face_of<Sh>(e);
      const int k = e - export_seg_start<Sh>(face);  // position along the face
      const bool xface = face < 2;
      const int ptx = xface ? (face == 0 ? 0 : bxa - 1) : k;
      const int pty = xface ? k : (face == 2 ? 0 : bya - 1);
      const bool nb = face == 0 ? nbW : (face == 1 ? nbE : (face == 2 ? nbS : nbN));
      const bool ok = nb && (xface ? pty < bya : ptx < bxa) && k < (xface ? Sh::SEGY : Sh::SEGX);
      // SX[side][I][ia][z][y], SY[side][J][ia][z][x]; the high face (E, N)
      // is the side-1 record, a brick-uniform distance further
      desc_off[e] = xface ? args.sx_off + ((int64_t(face == 1 ? nbx : 0) + bI) * NXF) * nzy + int64_t(zg) * ny +
                                (y0 + pty)
                          : args.sy_off + ((int64_t(face == 3 ? nby : 0) + bJ) * NYF) * nzx + int64_t(zg) * nx +
                                (x0 + ptx);
      desc_p[e] = ok ? perimeter_index<NYF>(ptx, pty, bxa, bya) : -1;
    }
  }
  // (the first barrier of the sweep orders these writes before their use)

  auto export_staged = [&](int zx, int sslot) {
    if (exp_warp && zx >= z0 && zx < z1) {
      R* shn = args.sh_next;
#pragma unroll 1
      for (int e = exp_lane; e < PE; e += 32 * Sh::NEXW) {
        const int p = desc_p[e];
        if (p < 0) continue;
        const Vec* st = reinterpret_cast<const Vec*>(stage + sslot * (QP * PMAX) + p * QP);
        R fin[QP];
#pragma unroll
        for (int v = 0; v < QP / VEC; ++v) *reinterpret_cast<Vec*>(&fin[v * VEC]) = st[v];
        R fq[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) fq[a] = fin[a];
        const int face = export_face_of<Sh>(e);
        const bool xface = face < 2;
        if constexpr (PHPLANE) {
          const Phys<R> phl = args.ph;
          export_one_face<L, S, R, FORCE>(phl, fq, face, shn + desc_off[e] + int64_t(zx) * (xface ? ny : nx),
                                          xface ? nzy : nzx);
        } else {
          export_one_face<L, S, R, FORCE>(args.ph, fq, face, shn + desc_off[e] + int64_t(zx) * (xface ? ny : nx),
                                          xface ? nzy : nzx);
        }
      }
    }
  };

  // Produce the window of plane c: collide a real plane (TMA slot) or copy a
  // virtual plane from the shell; the populations that do not move laterally
  // stay in onl (rest, +z, -z).  Returns false if the TMA wait timed out.
  auto produce = [&](int c, R* win, R (&onl)[3]) -> bool {
    if (!is_main) return true;
    const bool real = c >= z0 && c < z1;
    if (real) {
      const int k = c - z0;
      const int slot = k % NS;
      Phys<R> phl;
      if constexpr (PHPLANE) phl = args.ph;  // loads in flight during the wait
      if (!mbar_wait_bounded(&bars[slot], (k / NS) & 1, kWaitLimitNs)) return false;
      if (active) {
        const S* sl = slots + size_t(slot) * Q * BY * BX + ty * BX + tx;
        R fl[Q], own[Q];
        static_for<0, Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          fl[a] = load_as<S, R>(sl[a * BY * BX]);
        });
        collide<L, R, FORCE>(fl, PHPLANE ? phl : args.ph, own);
        static_for<0, Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          if constexpr (is_lateral<L>(a)) win[lat_index<L>(a) * WPLANE + wbase] = own[a];
          else onl[a == 0 ? 0 : (L::cz(a) == 1 ? 1 : 2)] = own[a];
        });
      }
    } else if (plane_needed(c) && active) {
      // virtual plane just outside the brick: the neighbouring brick's export
      const bool low = (c == z0 - 1);
      const int side = low ? 1 : 0;
      const int bb = low ? bKd : bKu;
      const int64_t base =
          args.sz_off + (int64_t(side) * nbzs + bb + zg) * NZF * int64_t(ny) * nx + int64_t(y) * nx + x;
      onl[0] = onl[1] = onl[2] = R(0);
      static_for<0, Q>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int cz = L::cz(a);
        if constexpr (cz != 0) {
          if ((cz == 1) == low) {
            constexpr int iz = sub_index<L>(2, cz, a);
            const R v = shc[base + int64_t(iz) * ny * nx];
            if constexpr (is_lateral<L>(a)) win[lat_index<L>(a) * WPLANE + wbase] = v;
            else onl[cz == 1 ? 1 : 2] = v;
          }
        }
      });
    }
    return true;
  };
  // the ring of the window of plane c (values fetched two planes ahead); kept
  // out of the lambda above so the ring arrays stay in registers.  Only valid
  // entries: an invalid north/south entry of a ragged brick would alias the
  // east ring's corner cell of a diagonal direction.
#define LB_RING_PUT(win_, c_)                                          \
  if (plane_needed(c_)) {                                              \
    _Pragma("unroll") for (int e = 0; e < HPT; ++e)                    \
      if (Sh::HSMEM ? hsm[e] >= 0 : hval[e]) (win_)[hsm[e]] = ha[e];   \
  }

  // three destination planes of gathered populations
  // (the sweep below runs three planes per loop trip and permutes the roles
  // of the three sets at compile time instead of copying them every plane;
  // an entry is always gathered, or set by a bounce-back, before it is stored)
  R G[3][Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    G[0][a] = R(0);
    G[1][a] = R(0);
    G[2][a] = R(0);
  }
  // bounce-back values of the z-descending directions of the previous plane;
  // applied after the next gather, which would otherwise overwrite them
  constexpr int NDN = count_dirs<L>(2, -1);
  R bdn[NDN];
  unsigned bdn_mask = 0;
#pragma unroll
  for (int i = 0; i < NDN; ++i) bdn[i] = R(0);

  auto abort_cta = [&](int k) {
    if (tid == 0) {
      if constexpr (TS != 0) bulk_wait_all();
      atomicExch(args.status, LB_E_TIMEOUT);
      // drain this CTA's own copies still in flight (bounded); a copy that
      // does not land in time may still write this CTA's shared memory
      bool drained = true;
      for (int kk = (k < 0 ? 0 : k); kk < issued; ++kk)
        drained &= mbar_wait_bounded(&bars[kk % NS], (kk / NS) & 1, kWaitLimitNs);
      if (!drained) atomicExch(args.status, LB_E_ABANDONED);
    }
  };

  if (DEC && !is_main) {
    // dedicated export warps: export each staged plane as soon as the node
    // threads mark it ready, then hand the ring slot back
#pragma unroll 1
    for (int zx = z0; zx < z1; ++zx) {
      const int sl = (zx - z0) % SR;
      if (!mbar_wait_bounded(&sfull[sl], ((zx - z0) / SR) & 1, kWaitLimitNs)) {
        atomicExch(args.status, LB_E_TIMEOUT);
        return false;
      }
      export_staged(zx, sl);
      mbar_arrive(&sempty[sl]);
    }
  } else {
    // ------------------------------------------------ prologue: plane z0 - 1
    R onl_g[3] = {R(0), R(0), R(0)};  // non-lateral populations of the gathered plane
    {
      bool ok = produce(z0 - 1, win0 + ((z0 - 1) & 1) * WSTRIDE, onl_g);
      if (is_main) LB_RING_PUT(win0 + ((z0 - 1) & 1) * WSTRIDE, z0 - 1);
      if (node_sync_or(!ok)) {
        abort_cta(0);
        return false;
      }
    }
  #pragma unroll
    for (int e = 0; e < HPT; ++e) ha[e] = hb[e];
    halo_fetch(hb, z0 + 1);

    // ------------------------------------------------ sweep: gather plane g,
    // produce plane g + 1 in the same barrier interval (independent work)
    auto sweep_plane = [&](const int g, auto K) -> bool {
      constexpr int k = decltype(K)::value;
      R(&G0)[Q] = G[k % 3];        // plane g - 1
      R(&G1)[Q] = G[(k + 1) % 3];  // plane g
      R(&G2)[Q] = G[(k + 2) % 3];  // plane g + 1
      const int c = g + 1;
      R* win_g = win0 + (g & 1) * WSTRIDE;
      R* win_c = win0 + (c & 1) * WSTRIDE;
      const bool real_g = g >= z0 && g < z1;
      const bool need_g = plane_needed(g);

      // exports of plane g - 2 (staged one iteration ago) first: they need
      // no TMA data, so they overlap the wait for plane c's load
      if constexpr (!DEC) export_staged(g - 2, (g - 2) & 1);

      R onl_c[3] = {R(0), R(0), R(0)};
      bool ok = true;
      if (c <= z1) {
        ok = produce(c, win_c, onl_c);
        if (is_main) LB_RING_PUT(win_c, c);
      }

      // gather plane g (window complete since the previous barrier)
      if (active && need_g) {
        static_for<0, Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          constexpr int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
          R v;
          if constexpr (is_lateral<L>(a)) v = win_g[lat_index<L>(a) * WPLANE + wbase - cy * WX - cx];
          else v = onl_g[a == 0 ? 0 : (cz == 1 ? 1 : 2)];
          if constexpr (cz == -1) G0[a] = v;
          if constexpr (cz == 0) G1[a] = v;
          if constexpr (cz == 1) G2[a] = v;
        });
      }

      // z-descending bounce-backs of plane g - 1, saved one plane ago
      if (bdn_mask) {
        static_for<0, Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          if constexpr (L::cz(a) == -1) {
            constexpr int i = sub_index<L>(2, -1, a);
            if (bdn_mask >> i & 1) G0[a] = bdn[i];
          }
        });
        bdn_mask = 0;
      }
      // halfway bounce-back for destination plane g (threads next to a wall)
      if (real_g && active &&
          (xy_wall || (LINK ? (g == args.zwl || g == args.zwh) : (z_walls && (g == 0 || g == nz - 1))))) {
        const bool bzlo = LINK ? g == args.zwl : z_walls && g == 0;
        const bool bzhi = LINK ? g == args.zwh : z_walls && g == nz - 1;
        static_for<0, Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          constexpr int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
          int cb = 0;
          if constexpr (cx == 1) cb |= bxlo ? 1 : 0;
          if constexpr (cx == -1) cb |= bxhi ? 1 : 0;
          if constexpr (cy == 1) cb |= bylo ? 2 : 0;
          if constexpr (cy == -1) cb |= byhi ? 2 : 0;
          if constexpr (cz == 1) cb |= bzlo ? 4 : 0;
          if constexpr (cz == -1) cb |= bzhi ? 4 : 0;
          if (cb != 0) {
            constexpr int oa = L::opp(a);
            R back;
            if constexpr (is_lateral<L>(oa)) back = win_g[lat_index<L>(oa) * WPLANE + wbase];
            else back = onl_g[oa == 0 ? 0 : (L::cz(oa) == 1 ? 1 : 2)];
            const R v = back + args.bb[a][cb];
            if constexpr (cz == -1) {
              constexpr int i = sub_index<L>(2, -1, a);
              bdn[i] = v;
              bdn_mask |= 1u << i;
            } else {
              G1[a] = v;
            }
          }
        });
      }

      // plane g - 1 is complete: store, stage its perimeter, export along z
      const int zd = g - 1;
      if constexpr (TS != 0) {
        // the output buffer is free once the TMA store of plane zd - 1 has read it
        if (zd > z0 && zd < z1) {
          if (tid == 0) {
            bulk_wait_read_all();
            mbar_arrive(outfree);
          }
          if (!mbar_wait_bounded(outfree, (zd - z0 - 1) & 1, kWaitLimitNs)) ok = false;
        }
      }
      if (active && zd >= z0 && zd < z1) {
        if constexpr (TS != 0) {
          S* o = outbuf + ty * BX + tx;
          static_for<0, Q>([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            o[a * BY * BX] = store_as<S, R>(G0[a]);
          });
        } else {
          if constexpr (Sh::WIDE_STORE) {
            // direction a lies a * vol elements further (vol is a multiple
            // of 32: rows are padded to 32 elements)
            char* p = reinterpret_cast<char*>(fglob + (x + args.pitch * (y + int64_t(ny) * zd)));
            const uint32_t v32 = args.vol32;
            static_for<0, Q>([&](auto A_) {
              constexpr int a = decltype(A_)::value;
              *reinterpret_cast<S*>(p + uint64_t(v32) * uint32_t(a * 32 * sizeof(S))) = store_as<S, R>(G0[a]);
            });
          } else {
            S* p = fglob + (x + args.pitch * (y + int64_t(ny) * zd));
            static_for<0, Q>([&](auto A_) {
              constexpr int a = decltype(A_)::value;
              *p = store_as<S, R>(G0[a]);
              p += args.vol;
            });
          }
        }
        if (pidx >= 0 && any_lateral_export) {
          const int sslot = DEC ? (zd - z0) % SR : (zd & 1);
          // the export warps must be done with this ring slot's previous plane
          if (DEC && zd - z0 >= SR && !mbar_wait_bounded(&sempty[sslot], (((zd - z0) / SR) - 1) & 1, kWaitLimitNs))
            ok = false;
          Vec* st = reinterpret_cast<Vec*>(stage + sslot * (QP * PMAX) + pidx * QP);
  #pragma unroll
          for (int v = 0; v < QP / VEC; ++v) {
            R tmp[VEC];
  #pragma unroll
            for (int j = 0; j < VEC; ++j) tmp[j] = (v * VEC + j < Q) ? G0[(v * VEC + j) < Q ? v * VEC + j : 0] : R(0);
            st[v] = *reinterpret_cast<const Vec*>(tmp);
          }
        }
        const bool eD = zd == z0 && nbD, eU = zd == z1 - 1 && nbU;
        if (eD || eU)
          export_node<L, S, R, FORCE, LINK>(args, G0, x, y, zd, (eD ? kFaceD : 0u) | (eU ? kFaceU : 0u), bI, bJ, bK);
      }
      // every node thread (staging or not) marks the staged plane ready
      if (DEC && zd >= z0 && zd < z1) mbar_arrive(&sfull[(zd - z0) % SR]);

      // the output buffer's generic-proxy writes must be visible to the TMA
      if (TS != 0 && zd >= z0 && zd < z1) fence_proxy_async_smem();

      // ring values move up one plane; start the loads two planes ahead
  #pragma unroll
      for (int e = 0; e < HPT; ++e) ha[e] = hb[e];
      halo_fetch(hb, c + 2);

      onl_g[0] = onl_c[0];
      onl_g[1] = onl_c[1];
      onl_g[2] = onl_c[2];

      // the only barrier of the iteration: plane c's window is complete and
      // every thread has left plane g's buffers, which plane c + 1 reuses
      if (node_sync_or(!ok)) {
        abort_cta(c - z0);
        return false;
      }
      // plane zd is complete in the output buffer: one TMA store writes it
      if (TS != 0 && tid == 0 && zd >= z0 && zd < z1) {
        tma_store_4d(tmap_p, x0, y0, zd, 0, outbuf);
        bulk_commit();
      }
      // refill the slot consumed by plane c with plane c + NS
      if (tid == 0 && c >= z0 && c < z1 && c + NS < z1) {
        const int slot = (c - z0) % NS;
        mbar_arrive_expect_tx(&bars[slot], static_cast<uint32_t>(Sh::SLOT));
        tma_load_4d(slots + size_t(slot) * Q * BY * BX, tmap_p, x0, y0, c + NS, 0, &bars[slot]);
        ++issued;
      }
      return true;
    };
    // planes z0 - 1 .. z1 + 1 (the last trips only export the staged top
    // plane and pass the barrier; every thread runs the same trips)
    if constexpr (Sh::UNROLL3) {
      for (int g = z0 - 1; g <= z1 + 1; g += 3) {
        if (!sweep_plane(g, std::integral_constant<int, 0>{})) return false;
        if (!sweep_plane(g + 1, std::integral_constant<int, 1>{})) return false;
        if (!sweep_plane(g + 2, std::integral_constant<int, 2>{})) return false;
      }
    } else {
      for (int g = z0 - 1; g <= z1 + 1; ++g) {
        if (!sweep_plane(g, std::integral_constant<int, 0>{})) return false;
        // plane g's partial set becomes the previous plane's
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          G[0][a] = G[1][a];
          G[1][a] = G[2][a];
        }
      }
    }
  }
  // every issued plane has been waited for: retire the barriers so that the
  // next brick of a persistent CTA can initialise them again
  if (TS != 0 && tid == 0) bulk_wait_all();  // the last plane's store has landed
  __syncthreads();
  if (tid == 0) {
    for (int s = 0; s < NS + (DEC ? 2 * SR : 0); ++s) mbar_inval(&bars[s]);
    if constexpr (TS != 0) mbar_inval(outfree);
  }
  __syncthreads();
  return true;
#undef LB_RING_PUT
}

// One launch per time step of one domain: one CTA per brick column.
template <class L, class S, class R, int BX, int BY, int NS, int WB, int NXW, bool FORCE, int TS = 0,
          bool LINK = false, int MINB = 1>
__global__ void __launch_bounds__(K1Shape<L, S, R, BX, BY, NS, WB, NXW, TS, MINB>::NT, MINB)
    k1_fused_step(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ K1Args<R> args) {
  const int nbx = args.nbx, nby = args.nby;
  const int b = blockIdx.x;
  k1_brick<L, S, R, BX, BY, NS, WB, NXW, FORCE, TS, LINK, MINB>(&tmap, args, b % nbx, (b / nbx) % nby,
                                                                b / (nbx * nby));
}

// One launch per time step of many domains (a batch): a persistent grid whose
// CTA i sweeps the bricks items[starts[i] .. starts[i+1]) in turn.  An item is
// (domain, bI, bJ, bK); the arguments of domain d at shell parity p are
// args[p * n_dom + d], and domain d's parity at this launch is
// (dom_par[d] + k) & 1.
// dynamic shared memory of the batched launch: the brick's own buffers, then
// the current member's arguments where they fit (else read from global memory)
template <class Sh, class R>
struct K1BatchSmem {
  static constexpr size_t ARGS = (sizeof(K1Args<R>) + 15) / 16 * 16;
  static constexpr bool STAGED = Sh::SMEM + ARGS <= Sh::SMEM_CAP;
  static constexpr size_t BYTES = Sh::SMEM + (STAGED ? ARGS : 0);
};

template <class L, class S, class R, int BX, int BY, int NS, int WB, int NXW, bool FORCE, int TS = 0,
          int MINB = 1>
__global__ void __launch_bounds__(K1Shape<L, S, R, BX, BY, NS, WB, NXW, TS, MINB>::NT, MINB)
    k1_batched_step(const K1Args<R>* __restrict__ args, int n_dom, const CUtensorMap* __restrict__ tmaps,
                    const int4* __restrict__ items, const int* __restrict__ starts, const int* __restrict__ dom_par,
                    int k) {
  using Sh = K1Shape<L, S, R, BX, BY, NS, WB, NXW, TS, MINB>;
  using BS = K1BatchSmem<Sh, R>;
  extern __shared__ __align__(128) unsigned char smem[];
  K1Args<R>* sa = reinterpret_cast<K1Args<R>*>(smem + Sh::SMEM);
  const int i1 = starts[blockIdx.x + 1];
  for (int i = starts[blockIdx.x]; i < i1; ++i) {
    const int4 it = items[i];
    const int p = (dom_par[it.x] + k) & 1;
    const K1Args<R>& ga = args[size_t(p) * n_dom + it.x];
    if constexpr (BS::STAGED) {
      // the sweep reads its arguments (physical constants, strides, shell
      // offsets) every plane: from shared memory they are plain shared loads
      // instead of global loads the compiler cannot keep in registers.  The
      // previous brick ended on a CTA barrier, so no thread still reads sa.
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&ga);
      uint32_t* dst = reinterpret_cast<uint32_t*>(sa);
      for (int w = threadIdx.x; w < int(sizeof(K1Args<R>) / 4); w += blockDim.x) dst[w] = src[w];
      __syncthreads();
      if (!k1_brick<L, S, R, BX, BY, NS, WB, NXW, FORCE, TS, false, MINB, true>(tmaps + it.x, *sa, it.y, it.z,
                                                                                it.w))
        return;
    } else {
      if (!k1_brick<L, S, R, BX, BY, NS, WB, NXW, FORCE, TS, false, MINB>(tmaps + it.x, ga, it.y, it.z, it.w))
        return;
    }
  }
}

// Shell bootstrap: collide every brick-boundary node of the current state and
// export its outgoing populations into shell parity `sh_next` (used once after
// the state is set from outside; the steps keep the shell current).
template <class L, class S, class R, int BX, int BY, bool FORCE>
__global__ void __launch_bounds__(256) k1_bootstrap(const __grid_constant__ K1Args<R> args) {
  constexpr int Q = L::Q;
  const int64_t n = int64_t(args.nx) * args.ny * args.nz;
  for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < n; idx += int64_t(gridDim.x) * blockDim.x) {
    const int x = int(idx % args.nx);
    const int y = int((idx / args.nx) % args.ny);
    const int z = int(idx / (int64_t(args.nx) * args.ny));
    const int bI = x / BX, bJ = y / BY, bK = z / args.bz;
    const int x0 = bI * BX, y0 = bJ * BY, z0 = bK * args.bz;
    const int bxa = min(BX, args.nx - x0), bya = min(BY, args.ny - y0), z1 = min(z0 + args.bz, args.nz);
    const bool eW = x == x0 && (x0 > 0 || args.per[0]);
    const bool eE = x == x0 + bxa - 1 && (x0 + bxa < args.nx || args.per[0]);
    const bool eS = y == y0 && (y0 > 0 || args.per[1]);
    const bool eN = y == y0 + bya - 1 && (y0 + bya < args.ny || args.per[1]);
    const bool eD = z == z0 && (z0 > 0 || args.per[2] || args.zlink[0]);
    const bool eU = z == z1 - 1 && (z1 < args.nz || args.per[2] || args.zlink[1]);
    if (!(eW || eE || eS || eN || eD || eU)) continue;
    const int64_t o = x + args.pitch * (y + int64_t(args.ny) * z);
    const S* fg = static_cast<const S*>(args.f);
    R fr[Q];
    static_for<0, Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      fr[a] = load_as<S, R>(fg[a * args.vol + o]);
    });
    const unsigned faces = (eW ? kFaceW : 0u) | (eE ? kFaceE : 0u) | (eS ? kFaceS : 0u) | (eN ? kFaceN : 0u) |
                           (eD ? kFaceD : 0u) | (eU ? kFaceU : 0u);
    export_node<L, S, R, FORCE, true>(args, fr, x, y, z, faces, bI, bJ, bK);
  }
}

}  // namespace lbgb
