// lb_k2.cuh -- the fused single-array step with two nodes per thread.
//
// Same schedule, shell format and results as the fused step of lb_k1.cuh (a
// CTA owns a brick column, sweeps it along z with a TMA ring of planes, pulls
// every population from a padded shared window and exchanges post-collision
// boundary populations with neighbouring bricks through a double-buffered
// shell), but each thread owns the pair of x-adjacent nodes (x, x + 1) and
// evaluates the collision of both with the packed FP32x2 instructions
// (lb_pair.cuh).  That halves the issue slots of the arithmetic and of the
// per-node bookkeeping (addresses, predicates, loop control), loads and
// stores the pair as one 64-bit (FP32) or 32-bit (FP16/BF16) access, and lets
// each lane of an export warp export two perimeter nodes at once.  Lane by
// lane the arithmetic is the scalar FP32 sequence, so the populations are bit
// for bit those of the scalar kernels.
//
// FP32 arithmetic only (FP32, shifted FP16 and shifted BF16 storage); FP64
// storage keeps the scalar kernel.
#pragma once

#include "lb_k1_launch.cuh"
#include "lb_pair.cuh"

namespace lbgb {

template <class L, class S, int BX, int BY, int NS>
struct K2Shape {
  using R = float;
  static constexpr int Q = L::Q;
  static constexpr int NP = BX / 2;          // node pairs per brick row
  static constexpr int NT = NP * BY;         // threads: one per pair
  static constexpr int NXF = count_dirs<L>(0, 1);
  static constexpr int NYF = count_dirs<L>(1, 1);
  static constexpr int NZF = count_dirs<L>(2, 1);
  static constexpr int NLAT = n_lateral<L>();
  static constexpr int PY = NYF > 0 ? 1 : 0;
  static constexpr int WX = BX + 2;
  static constexpr int WY = BY + 2 * PY;
  static constexpr int WPLANE = WY * WX;
  static constexpr int HW = NXF * WY;
  static constexpr int HS = NYF * BX;
  static constexpr int H = 2 * HW + 2 * HS;
  static constexpr int HPT = (H + NT - 1) / NT;
  static constexpr int PMAX = NYF > 0 ? 2 * BX + 2 * (BY - 2) : 2;
  static constexpr int NEXW = ((PMAX + 1) / 2 + 31) / 32;  // export warps, two nodes per lane
  static constexpr int VEC = 4;
  static constexpr int QP = ((Q + VEC - 1) / VEC) % 2 == 1 ? (Q + VEC - 1) / VEC * VEC : ((Q + VEC - 1) / VEC + 1) * VEC;
  static constexpr size_t SLOT = size_t(Q) * BY * BX * sizeof(S);
  // the window is addressed from base + 1 so that the pair cell of an even
  // node column is 8-byte aligned (WX and WPLANE are even)
  static constexpr size_t WIN = (size_t(NLAT) * WPLANE + 2) * sizeof(R);
  static constexpr size_t STAGE = size_t(QP) * PMAX * sizeof(R);
  static constexpr size_t OFF_WIN = align128(NS * SLOT);
  static constexpr size_t OFF_STAGE = OFF_WIN + 2 * align128(WIN);
  static constexpr size_t OFF_DESC = OFF_STAGE + align128(2 * STAGE);
  static constexpr size_t OFF_BAR = OFF_DESC + align128(size_t(PMAX) * 24);
  static constexpr size_t SMEM = OFF_BAR + align128(NS * sizeof(uint64_t));
  static constexpr size_t SMEM_CAP = size_t(228) * 1024 - 1024;
  static_assert(BX % 2 == 0, "pairs need an even brick width");
  static_assert(WX % 2 == 0 && WPLANE % 2 == 0, "pair cells must stay 8-byte aligned");
  static_assert(BY == 1 || NYF > 0, "a 2D brick has one internal row");
  static_assert(NEXW * 32 <= NT, "export warps exceed the CTA");
};

// Export of two staged lateral perimeter nodes (lane .x = node p0, lane .y =
// node p1) whose shell records were resolved once per brick.
template <class L, class S, bool FORCE>
__device__ __forceinline__ void export_lateral_pair(const K1Args<float>& args, const f32x2 (&fin)[L::Q],
                                                    unsigned faces0, unsigned faces1, float* pw0, float* ps0,
                                                    float* pw1, float* ps1, int64_t dxe, int64_t dyn, int64_t sxs,
                                                    int64_t sys, const Phys<f32x2>& ph2) {
  using V = f32x2;
  V fr[L::Q];
  static_for<0, L::Q>([&](auto A_) {
    constexpr int a = decltype(A_)::value;
    fr[a] = V(round_to_storage<S, float>(fin[a].x), round_to_storage<S, float>(fin[a].y));
  });
  Mom<V> m;
  moments<L, V, FORCE>(fr, ph2, m);
  Coef<V> kc;
  coeffs<L, V, FORCE>(m, ph2, kc);
  auto face = [&](auto AX, auto SG, float* b0, float* b1, int64_t stride, unsigned f0, unsigned f1) {
    constexpr int axis = decltype(AX)::value, sign = decltype(SG)::value;
    static_for<0, L::Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      if constexpr (comp<L>(axis, a) == sign) {
        constexpr int ia = sub_index<L>(axis, sign, a);
        const V v = post<L, V, a>(kc);
        if (f0) b0[ia * stride] = v.x;
        if (f1) b1[ia * stride] = v.y;
      }
    });
  };
  using I0 = std::integral_constant<int, 0>;
  using I1 = std::integral_constant<int, 1>;
  using IM = std::integral_constant<int, -1>;
  if ((faces0 | faces1) & kFaceW) face(I0{}, IM{}, pw0, pw1, sxs, faces0 & kFaceW, faces1 & kFaceW);
  if ((faces0 | faces1) & kFaceE) face(I0{}, I1{}, pw0 + dxe, pw1 + dxe, sxs, faces0 & kFaceE, faces1 & kFaceE);
  if constexpr (count_dirs<L>(1, 1) > 0) {
    if ((faces0 | faces1) & kFaceS) face(I1{}, IM{}, ps0, ps1, sys, faces0 & kFaceS, faces1 & kFaceS);
    if ((faces0 | faces1) & kFaceN) face(I1{}, I1{}, ps0 + dyn, ps1 + dyn, sys, faces0 & kFaceN, faces1 & kFaceN);
  }
}

// The sweep of one brick column (bI, bJ, bK) of one domain by the whole CTA.
// tmap is the domain's TMA descriptor (kernel-parameter or global memory).
// Returns false if a TMA wait timed out (the CTA recorded LB_E_TIMEOUT and
// must stop).  On return every copy the brick issued has completed and the
// mbarriers are invalidated, so the CTA may start another brick.
// LINK: compiled for contexts with a link face (slab decomposition); the
// other instantiations compile the plain form, whose shell has no ghosts.
template <class L, class S, int BX, int BY, int NS, bool FORCE, bool UNROLL3 = false, bool LINK = false>
__device__ __forceinline__ bool k2_brick(const CUtensorMap* tmap_p, const K1Args<float>& args, const int bI,
                                         const int bJ, const int bK) {
  using R = float;
  using V = f32x2;
  using Sh = K2Shape<L, S, BX, BY, NS>;
  constexpr int Q = L::Q;
  constexpr int NT = Sh::NT, NP = Sh::NP;
  constexpr int NXF = Sh::NXF, NYF = Sh::NYF, NZF = Sh::NZF;
  constexpr int PY = Sh::PY, WX = Sh::WX, WPLANE = Sh::WPLANE;
  constexpr int HW = Sh::HW, HS = Sh::HS, H = Sh::H, HPT = Sh::HPT;
  constexpr int PMAX = Sh::PMAX, NEXW = Sh::NEXW, QP = Sh::QP, VEC = Sh::VEC;
  constexpr int WY = Sh::WY;
  constexpr int WSTRIDE = int(align128(Sh::WIN) / sizeof(R));

  extern __shared__ __align__(128) unsigned char smem[];
  S* slots = reinterpret_cast<S*>(smem);
  R* win0 = reinterpret_cast<R*>(smem + Sh::OFF_WIN) + 1;  // shifted base, see K2Shape::WIN
  R* stage = reinterpret_cast<R*>(smem + Sh::OFF_STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR);
  int64_t* desc_off = reinterpret_cast<int64_t*>(smem + Sh::OFF_DESC);
  unsigned* desc_faces = reinterpret_cast<unsigned*>(smem + Sh::OFF_DESC + size_t(PMAX) * 16);

  Phys<V> ph2;
  {
    const Phys<R>& p = args.ph;
    ph2.rho0 = V(p.rho0);
    ph2.inv_rho0 = V(p.inv_rho0);
    ph2.om1 = V(p.om1);
    ph2.g = V(p.g);
    for (int k = 0; k < 3; ++k) {
      ph2.F[k] = V(p.F[k]);
      ph2.hF[k] = V(p.hF[k]);
    }
    ph2.cs2 = V(p.cs2);
    ph2.c15rho0 = V(p.c15rho0);
    ph2.c15om1 = V(p.c15om1);
    ph2.c3rho0 = V(p.c3rho0);
    ph2.c45rho0 = V(p.c45rho0);
    ph2.c45om1 = V(p.c45om1);
    ph2.c9rho0 = V(p.c9rho0);
    ph2.c9om1 = V(p.c9om1);
    ph2.c3g = V(p.c3g);
    ph2.c9g = V(p.c9g);
  }

  const int tid = threadIdx.x;
  const int txp = tid % NP;
  const int ty = tid / NP;
  const int tx0 = 2 * txp;
  const int warp = tid / 32, lane = tid % 32;
  const int nx = args.nx, ny = args.ny, nz = args.nz;
  const int nbx = args.nbx, nby = args.nby, nbz = args.nbz;
  const int x0 = bI * BX, y0 = bJ * BY, z0 = bK * args.bz;
  const int bxa = min(BX, nx - x0), bya = min(BY, ny - y0);
  const int z1 = min(z0 + args.bz, nz);
  const int x = x0 + tx0, y = y0 + ty;
  const bool act0 = tx0 < bxa && ty < bya;      // node x
  const bool act1 = tx0 + 1 < bxa && ty < bya;  // node x + 1

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

  // bounce-back predicates per lane (x is even, so only lane .x can sit on x = 0)
  const bool bxlo0 = act0 && (x == 0) && !args.per[0];
  const bool bxhi0 = act0 && (x == nx - 1) && !args.per[0];
  const bool bxhi1 = act1 && (x + 1 == nx - 1) && !args.per[0];
  const bool bylo = act0 && (y == 0) && !args.per[1];
  const bool byhi = act0 && (y == ny - 1) && !args.per[1];
  const bool xy_wall = bxlo0 || bxhi0 || bxhi1 || bylo || byhi;
  const bool z_walls = !args.per[2];

  S* __restrict__ fglob = static_cast<S*>(args.f);
  const R* __restrict__ shc = args.sh_cur;

  // ---------------------------------------------------------------- setup
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
    prefetch_tmap(tmap_p);
  }
  __syncthreads();
  int issued = 0;
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

  // ring entries of the window (as in the scalar kernel)
  int64_t hbase[HPT];
  int hzs[HPT];
  int hsm[HPT];
  bool hval[HPT];
#pragma unroll
  for (int e = 0; e < HPT; ++e) {
    const int h = tid + e * NT;
    hval[e] = false;
    hbase[e] = 0;
    hzs[e] = 1;
    hsm[e] = 0;
    if (h < H) {
      if (h < 2 * HW) {
        const bool west = h < HW;
        const int hh = west ? h : h - HW;
        const int ia = hh / WY;
        const int r = hh % WY;
        int sy = y0 - PY + r;
        bool ok = (west ? nbW : nbE) && r < bya + 2 * PY;
        if (sy < 0 || sy >= ny) {
          if (args.per[1]) sy = (sy + ny) % ny;
          else ok = false;
        }
        const int col = west ? 0 : bxa + 1;
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

  R ha[HPT], hb[HPT];
  const R* hptr[HPT];
#pragma unroll
  for (int e = 0; e < HPT; ++e) hptr[e] = shc + hbase[e];
  auto halo_fetch = [&](R(&dst)[HPT], int z) {
    const bool ok = z <= z1 && plane_needed(z);
    const int zw = LINK ? (z < 0 ? z + args.zwrap : (z >= nz ? z - args.zwrap : z))
                        : (z < 0 ? z + nz : (z >= nz ? z - nz : z));
#pragma unroll
    for (int e = 0; e < HPT; ++e) dst[e] = (ok && hval[e]) ? hptr[e][int64_t(zw) * hzs[e]] : R(0);
  };
  halo_fetch(ha, z0 - 1);
  halo_fetch(hb, z0);

  // perimeter slots of the two nodes, export-warp work
  const int pidx0 = act0 ? perimeter_index<NYF>(tx0, ty, bxa, bya) : -1;
  const int pidx1 = act1 ? perimeter_index<NYF>(tx0 + 1, ty, bxa, bya) : -1;
  const int pcount = perimeter_count<NYF>(bxa, bya);
  const bool any_lateral_export = nbW || nbE || (NYF > 0 && (nbS || nbN));
  const bool exp_warp = any_lateral_export && warp < NEXW;
  const int exp_lane = warp * 32 + lane;  // first pair of perimeter nodes of this lane

  const int wbase = (ty + PY) * WX + (tx0 + 1);  // odd; win0 is shifted by one

  const int64_t nzy = int64_t(nzs) * ny, nzx = int64_t(nzs) * nx;
  if (exp_warp) {
#pragma unroll 1
    for (int p = exp_lane; p < pcount; p += 32 * NEXW) {
      // descriptors for every perimeter node (the export below pairs p, p + step)
      int ptx, pty;
      perimeter_node<NYF>(p, bxa, bya, ptx, pty);
      const unsigned faces = (ptx == 0 && nbW ? kFaceW : 0u) | (ptx == bxa - 1 && nbE ? kFaceE : 0u) |
                             (NYF > 0 && pty == 0 && nbS ? kFaceS : 0u) |
                             (NYF > 0 && pty == bya - 1 && nbN ? kFaceN : 0u);
      desc_off[2 * p] = args.sx_off + (int64_t(bI) * NXF) * nzy + int64_t(zg) * ny + (y0 + pty);
      desc_off[2 * p + 1] = NYF > 0 ? args.sy_off + (int64_t(bJ) * NYF) * nzx + int64_t(zg) * nx + (x0 + ptx) : 0;
      desc_faces[p] = faces;
    }
  }

  // lanes of the export warps take perimeter nodes p and p + half, half =
  // ceil(pcount / 2), so that every lane has two nodes (one at the odd end)
  const int half = (pcount + 1) / 2;
  auto export_staged = [&](int zx) {
    if (exp_warp && zx >= z0 && zx < z1) {
      R* shn = args.sh_next;
#pragma unroll 1
      for (int p0 = exp_lane; p0 < half; p0 += 32 * NEXW) {
        const int p1 = p0 + half;
        const bool two = p1 < pcount;
        const int p1r = two ? p1 : p0;
        const float4* st0 = reinterpret_cast<const float4*>(stage + (zx & 1) * (QP * PMAX) + p0 * QP);
        const float4* st1 = reinterpret_cast<const float4*>(stage + (zx & 1) * (QP * PMAX) + p1r * QP);
        V fin[Q];
#pragma unroll
        for (int v = 0; v < QP / VEC; ++v) {
          const float4 a4 = st0[v], b4 = st1[v];
          const float av[4] = {a4.x, a4.y, a4.z, a4.w};
          const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
          for (int j = 0; j < VEC; ++j)
            if (v * VEC + j < Q) fin[v * VEC + j] = V(av[j], bv[j]);
        }
        const unsigned f0 = desc_faces[p0], f1 = two ? desc_faces[p1r] : 0u;
        export_lateral_pair<L, S, FORCE>(args, fin, f0, f1, shn + desc_off[2 * p0] + int64_t(zx) * ny,
                                         shn + desc_off[2 * p0 + 1] + int64_t(zx) * nx,
                                         shn + desc_off[2 * p1r] + int64_t(zx) * ny,
                                         shn + desc_off[2 * p1r + 1] + int64_t(zx) * nx, int64_t(nbx) * NXF * nzy,
                                         int64_t(nby) * NYF * nzx, nzy, nzx, ph2);
      }
    }
  };

  // write the pair value of the own cell (only the active nodes: the cell
  // right of an inactive node belongs to the east ring of a ragged brick)
  auto put_own = [&](R* cell, V v) {
    if (act1) store_pair<float>(cell, v);
    else if (act0) cell[0] = v.x;
  };

  auto produce = [&](int c, R* win, V(&onl)[3]) -> bool {
    const bool real = c >= z0 && c < z1;
    if (real) {
      const int k = c - z0;
      const int slot = k % NS;
      if (!mbar_wait_bounded(&bars[slot], (k / NS) & 1, kWaitLimitNs)) return false;
      if (act0) {
        const S* sl = slots + size_t(slot) * Q * BY * BX + ty * BX + tx0;
        V fl[Q], own[Q];
        static_for<0, Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          fl[a] = load_pair<S>(sl + a * BY * BX);
        });
        collide<L, V, FORCE>(fl, ph2, own);
        static_for<0, Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          if constexpr (is_lateral<L>(a)) put_own(win + lat_index<L>(a) * WPLANE + wbase, own[a]);
          else onl[a == 0 ? 0 : (L::cz(a) == 1 ? 1 : 2)] = own[a];
        });
      }
    } else if (plane_needed(c) && act0) {
      const bool low = (c == z0 - 1);
      const int side = low ? 1 : 0;
      const int bb = low ? bKd : bKu;
      const int64_t base =
          args.sz_off + (int64_t(side) * nbzs + bb + zg) * NZF * int64_t(ny) * nx + int64_t(y) * nx + x;
      onl[0] = onl[1] = onl[2] = V(0);
      static_for<0, Q>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int cz = L::cz(a);
        if constexpr (cz != 0) {
          if ((cz == 1) == low) {
            constexpr int iz = sub_index<L>(2, cz, a);
            const R* src = shc + base + int64_t(iz) * ny * nx;
            const V v(src[0], act1 ? src[1] : R(0));
            if constexpr (is_lateral<L>(a)) put_own(win + lat_index<L>(a) * WPLANE + wbase, v);
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
#define LB_RING_PUT(win_, c_)                          \
  if (plane_needed(c_)) {                              \
    _Pragma("unroll") for (int e = 0; e < HPT; ++e)    \
      if (hval[e]) (win_)[hsm[e]] = ha[e];             \
  }

  // three destination planes of gathered pairs; with UNROLL3 the sweep
  // permutes their roles at compile time (three copies of its body),
  // otherwise it copies them every plane
  V G[3][Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    G[0][a] = V(0);
    G[1][a] = V(0);
    G[2][a] = V(0);
  }
  constexpr int NDN = count_dirs<L>(2, -1);
  V bdn[NDN];
  unsigned bdn_mask0 = 0, bdn_mask1 = 0;
#pragma unroll
  for (int i = 0; i < NDN; ++i) bdn[i] = V(0);

  auto abort_cta = [&](int k) {
    if (tid == 0) {
      atomicExch(args.status, LB_E_TIMEOUT);
      // drain this CTA's own copies still in flight (bounded); a copy that
      // does not land in time may still write this CTA's shared memory
      bool drained = true;
      for (int kk = (k < 0 ? 0 : k); kk < issued; ++kk)
        drained &= mbar_wait_bounded(&bars[kk % NS], (kk / NS) & 1, kWaitLimitNs);
      if (!drained) atomicExch(args.status, LB_E_ABANDONED);
    }
  };

  V onl_g[3] = {V(0), V(0), V(0)};
  {
    bool ok = produce(z0 - 1, win0 + ((z0 - 1) & 1) * WSTRIDE, onl_g);
    LB_RING_PUT(win0 + ((z0 - 1) & 1) * WSTRIDE, z0 - 1);
    if (__syncthreads_or(!ok)) {
      abort_cta(0);
      return false;
    }
  }
#pragma unroll
  for (int e = 0; e < HPT; ++e) ha[e] = hb[e];
  halo_fetch(hb, z0 + 1);

  auto sweep_plane = [&](const int g, auto K) -> bool {
    constexpr int k = decltype(K)::value;
    V(&G0)[Q] = G[k % 3];        // plane g - 1
    V(&G1)[Q] = G[(k + 1) % 3];  // plane g
    V(&G2)[Q] = G[(k + 2) % 3];  // plane g + 1
    const int c = g + 1;
    R* win_g = win0 + (g & 1) * WSTRIDE;
    R* win_c = win0 + (c & 1) * WSTRIDE;
    const bool real_g = g >= z0 && g < z1;
    const bool need_g = plane_needed(g);

    V onl_c[3] = {V(0), V(0), V(0)};
    bool ok = true;
    if (c <= z1) {
      ok = produce(c, win_c, onl_c);
      LB_RING_PUT(win_c, c);
    }

    // gather plane g
    if (act0 && need_g) {
      static_for<0, Q>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
        V v;
        if constexpr (is_lateral<L>(a)) {
          const R* cell = win_g + lat_index<L>(a) * WPLANE + wbase - cy * WX;
          if constexpr (cx == 0) v = load_pair<float>(cell);
          else v = V(cell[-cx], cell[1 - cx]);
        } else {
          v = onl_g[a == 0 ? 0 : (cz == 1 ? 1 : 2)];
        }
        if constexpr (cz == -1) G0[a] = v;
        if constexpr (cz == 0) G1[a] = v;
        if constexpr (cz == 1) G2[a] = v;
      });
    }
    export_staged(g - 2);

    if (bdn_mask0 | bdn_mask1) {
      static_for<0, Q>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        if constexpr (L::cz(a) == -1) {
          constexpr int i = sub_index<L>(2, -1, a);
          if (bdn_mask0 >> i & 1) G0[a].x = bdn[i].x;
          if (bdn_mask1 >> i & 1) G0[a].y = bdn[i].y;
        }
      });
      bdn_mask0 = bdn_mask1 = 0;
    }
    // halfway bounce-back for destination plane g, lane by lane
    if (real_g && act0 &&
        (xy_wall || (LINK ? (g == args.zwl || g == args.zwh) : (z_walls && (g == 0 || g == nz - 1))))) {
      const bool bzlo = LINK ? g == args.zwl : z_walls && g == 0;
      const bool bzhi = LINK ? g == args.zwh : z_walls && g == nz - 1;
      static_for<0, Q>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
        int cb0 = 0, cb1 = 0;
        if constexpr (cx == 1) cb0 |= bxlo0 ? 1 : 0;
        if constexpr (cx == -1) {
          cb0 |= bxhi0 ? 1 : 0;
          cb1 |= bxhi1 ? 1 : 0;
        }
        if constexpr (cy == 1) {
          cb0 |= bylo ? 2 : 0;
          cb1 |= bylo ? 2 : 0;
        }
        if constexpr (cy == -1) {
          cb0 |= byhi ? 2 : 0;
          cb1 |= byhi ? 2 : 0;
        }
        if constexpr (cz == 1) {
          cb0 |= bzlo ? 4 : 0;
          cb1 |= bzlo ? 4 : 0;
        }
        if constexpr (cz == -1) {
          cb0 |= bzhi ? 4 : 0;
          cb1 |= bzhi ? 4 : 0;
        }
        if (!act1) cb1 = 0;
        if ((cb0 | cb1) != 0) {
          constexpr int oa = L::opp(a);
          V back;
          if constexpr (is_lateral<L>(oa)) {
            const R* cell = win_g + lat_index<L>(oa) * WPLANE + wbase;
            back = V(cell[0], cell[1]);
          } else {
            back = onl_g[oa == 0 ? 0 : (L::cz(oa) == 1 ? 1 : 2)];
          }
          if constexpr (cz == -1) {
            constexpr int i = sub_index<L>(2, -1, a);
            if (cb0) {
              bdn[i].x = back.x + args.bb[a][cb0];
              bdn_mask0 |= 1u << i;
            }
            if (cb1) {
              bdn[i].y = back.y + args.bb[a][cb1];
              bdn_mask1 |= 1u << i;
            }
          } else {
            if (cb0) G1[a].x = back.x + args.bb[a][cb0];
            if (cb1) G1[a].y = back.y + args.bb[a][cb1];
          }
        }
      });
    }

    // plane g - 1 is complete: store, stage its perimeter, export along z
    const int zd = g - 1;
    if (act0 && zd >= z0 && zd < z1) {
      if constexpr (sizeof(S) == 2) {
        // 16-bit storage: direction a lies a * vol elements further, one wide
        // multiply-add of vol / 32 (rows are padded to 32 elements) per store
        char* p = reinterpret_cast<char*>(fglob + (x + args.pitch * (y + int64_t(ny) * zd)));
        const uint32_t v32 = args.vol32;
        if (act1) {
          static_for<0, Q>([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            store_pair<S>(reinterpret_cast<S*>(p + uint64_t(v32) * uint32_t(a * 32 * sizeof(S))), G0[a]);
          });
        } else {
          static_for<0, Q>([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            *reinterpret_cast<S*>(p + uint64_t(v32) * uint32_t(a * 32 * sizeof(S))) = store_as<S, R>(G0[a].x);
          });
        }
      } else {
        S* p = fglob + (x + args.pitch * (y + int64_t(ny) * zd));
        if (act1) {
          static_for<0, Q>([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            store_pair<S>(p, G0[a]);
            p += args.vol;
          });
        } else {
          static_for<0, Q>([&](auto A_) {
            constexpr int a = decltype(A_)::value;
            *p = store_as<S, R>(G0[a].x);
            p += args.vol;
          });
        }
      }
      if (any_lateral_export) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int pidx = k == 0 ? pidx0 : pidx1;
          if (pidx >= 0) {
            float4* st = reinterpret_cast<float4*>(stage + (zd & 1) * (QP * PMAX) + pidx * QP);
#pragma unroll
            for (int v = 0; v < QP / VEC; ++v) {
              float t[VEC];
#pragma unroll
              for (int j = 0; j < VEC; ++j) {
                const int a = v * VEC + j;
                t[j] = a < Q ? (k == 0 ? G0[a < Q ? a : 0].x : G0[a < Q ? a : 0].y) : R(0);
              }
              st[v] = make_float4(t[0], t[1], t[2], t[3]);
            }
          }
        }
      }
      const bool eD = zd == z0 && nbD, eU = zd == z1 - 1 && nbU;
      if (eD || eU) {
        const unsigned fz = (eD ? kFaceD : 0u) | (eU ? kFaceU : 0u);
        R fs[Q];
#pragma unroll
        for (int a = 0; a < Q; ++a) fs[a] = G0[a].x;
        export_node<L, S, R, FORCE, LINK>(args, fs, x, y, zd, fz, bI, bJ, bK);
        if (act1) {
#pragma unroll
          for (int a = 0; a < Q; ++a) fs[a] = G0[a].y;
          export_node<L, S, R, FORCE, LINK>(args, fs, x + 1, y, zd, fz, bI, bJ, bK);
        }
      }
    }

#pragma unroll
    for (int e = 0; e < HPT; ++e) ha[e] = hb[e];
    halo_fetch(hb, c + 2);

    onl_g[0] = onl_c[0];
    onl_g[1] = onl_c[1];
    onl_g[2] = onl_c[2];

    if (__syncthreads_or(!ok)) {
      abort_cta(c - z0);
      return false;
    }
    if (tid == 0 && c >= z0 && c < z1 && c + NS < z1) {
      const int slot = (c - z0) % NS;
      mbar_arrive_expect_tx(&bars[slot], static_cast<uint32_t>(Sh::SLOT));
      tma_load_4d(slots + size_t(slot) * Q * BY * BX, tmap_p, x0, y0, c + NS, 0, &bars[slot]);
      ++issued;
    }
    return true;
  };
  // planes z0 - 1 .. z1 + 1 (the last trips only export the staged top plane
  // and pass the barrier; every thread runs the same trips)
  if constexpr (UNROLL3) {
    for (int g = z0 - 1; g <= z1 + 1; g += 3) {
      if (!sweep_plane(g, std::integral_constant<int, 0>{})) return false;
      if (!sweep_plane(g + 1, std::integral_constant<int, 1>{})) return false;
      if (!sweep_plane(g + 2, std::integral_constant<int, 2>{})) return false;
    }
  } else {
    for (int g = z0 - 1; g <= z1 + 1; ++g) {
      if (!sweep_plane(g, std::integral_constant<int, 0>{})) return false;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        G[0][a] = G[1][a];
        G[1][a] = G[2][a];
      }
    }
  }
  // every issued plane has been waited for: retire the barriers so that the
  // next brick of a persistent CTA can initialise them again
  __syncthreads();
  if (tid == 0)
    for (int s = 0; s < NS; ++s) mbar_inval(&bars[s]);
  __syncthreads();
  return true;
#undef LB_RING_PUT
}

// One launch per time step of one domain: one CTA per brick column.  D2Q9
// sweeps three planes per loop trip and keeps three CTAs per SM (the register
// cap that this implies holds the unrolled body without spills).
template <class L, class S, int BX, int BY, int NS, bool FORCE, bool LINK = false>
__global__ void __launch_bounds__(BX* BY / 2, (L::Q == 9 ? 3 : 1))
    k2_fused_step(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ K1Args<float> args) {
  const int nbx = args.nbx, nby = args.nby;
  const int b = blockIdx.x;
  k2_brick<L, S, BX, BY, NS, FORCE, L::Q == 9, LINK>(&tmap, args, b % nbx, (b / nbx) % nby, b / (nbx * nby));
}

// One launch per time step of many domains (a batch): a persistent grid whose
// CTA i sweeps the bricks items[starts[i] .. starts[i+1]) in turn.  An item is
// (domain, bI, bJ, bK); the arguments of domain d at shell parity p are
// args[p * n_dom + d], and domain d's parity at this launch is
// (dom_par[d] + k) & 1.
template <class L, class S, int BX, int BY, int NS, bool FORCE>
__global__ void __launch_bounds__(BX* BY / 2, 1)
    k2_batched_step(const K1Args<float>* __restrict__ args, int n_dom, const CUtensorMap* __restrict__ tmaps,
                    const int4* __restrict__ items, const int* __restrict__ starts, const int* __restrict__ dom_par,
                    int k) {
  using Sh = K2Shape<L, S, BX, BY, NS>;
  using BS = K1BatchSmem<Sh, float>;
  extern __shared__ __align__(128) unsigned char smem[];
  K1Args<float>* sa = reinterpret_cast<K1Args<float>*>(smem + Sh::SMEM);
  const int i1 = starts[blockIdx.x + 1];
  for (int i = starts[blockIdx.x]; i < i1; ++i) {
    const int4 it = items[i];
    const int p = (dom_par[it.x] + k) & 1;
    const K1Args<float>& ga = args[size_t(p) * n_dom + it.x];
    if constexpr (BS::STAGED) {
      // the member's arguments as shared loads in the sweep (see
      // k1_batched_step); the previous brick ended on a CTA barrier
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&ga);
      uint32_t* dst = reinterpret_cast<uint32_t*>(sa);
      for (int w = threadIdx.x; w < int(sizeof(K1Args<float>) / 4); w += blockDim.x) dst[w] = src[w];
      __syncthreads();
      if (!k2_brick<L, S, BX, BY, NS, FORCE>(tmaps + it.x, *sa, it.y, it.z, it.w)) return;
    } else {
      if (!k2_brick<L, S, BX, BY, NS, FORCE>(tmaps + it.x, ga, it.y, it.z, it.w)) return;
    }
  }
}

// host side: one compiled paired brick shape
template <class L, class S, int BX, int BY, int NS>
struct K2Impl {
  using Sh = K2Shape<L, S, BX, BY, NS>;
  static constexpr size_t SMEM_B = K1BatchSmem<Sh, float>::BYTES;

  static cudaError_t configure() {
    const int sm = int(Sh::SMEM);
    cudaError_t e;
    e = cudaFuncSetAttribute(k2_fused_step<L, S, BX, BY, NS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k2_fused_step<L, S, BX, BY, NS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k2_fused_step<L, S, BX, BY, NS, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k2_fused_step<L, S, BX, BY, NS, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             sm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k2_batched_step<L, S, BX, BY, NS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(SMEM_B));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k2_batched_step<L, S, BX, BY, NS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(SMEM_B));
  }

  static cudaError_t step(lb_ctx* ctx) {
    K1Args<float> a = k1_make_args<float>(ctx, ctx->parity, 1 - ctx->parity);
    make_bounce_terms<L, float>(ctx->g, a.bb);
    const int grid = ctx->plan.nbx * ctx->plan.nby * ctx->plan.nbz;
    cudaStream_t st = ctx->stream;
    if (ctx->g.zlink[0] || ctx->g.zlink[1]) {
      if (ctx->g.has_force)
        k2_fused_step<L, S, BX, BY, NS, true, true><<<grid, Sh::NT, Sh::SMEM, st>>>(ctx->tmap, a);
      else
        k2_fused_step<L, S, BX, BY, NS, false, true><<<grid, Sh::NT, Sh::SMEM, st>>>(ctx->tmap, a);
    } else if (ctx->g.has_force) {
      k2_fused_step<L, S, BX, BY, NS, true><<<grid, Sh::NT, Sh::SMEM, st>>>(ctx->tmap, a);
    } else {
      k2_fused_step<L, S, BX, BY, NS, false><<<grid, Sh::NT, Sh::SMEM, st>>>(ctx->tmap, a);
    }
    return cudaGetLastError();
  }

  static cudaError_t batched(const BatchLaunch& b, cudaStream_t stream) {
    const K1Args<float>* args = static_cast<const K1Args<float>*>(b.args);
    if (b.force)
      k2_batched_step<L, S, BX, BY, NS, true><<<b.grid, Sh::NT, SMEM_B, stream>>>(args, b.n_dom, b.tmaps, b.items,
                                                                                 b.starts, b.dom_par, b.k);
    else
      k2_batched_step<L, S, BX, BY, NS, false><<<b.grid, Sh::NT, SMEM_B, stream>>>(args, b.n_dom, b.tmaps, b.items,
                                                                                  b.starts, b.dom_par, b.k);
    return cudaGetLastError();
  }

  static int batched_occupancy() {
    int n = 0;
    if (configure() != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k2_batched_step<L, S, BX, BY, NS, true>, Sh::NT,
                                                      SMEM_B) != cudaSuccess)
      return 0;
    return n;
  }

  static constexpr K1Variant variant(int lattice, int storage) {
    // the shell format is the scalar kernel's, so its bootstrap is reused
    return K1Variant{lattice, storage, BX, BY, NS, 2, 0, Sh::SMEM, &configure, &step,
                     &K1Impl<L, S, float, BX, BY, NS, 2, 0>::bootstrap, 2, &batched, &batched_occupancy, 0, 1};
  }
};

}  // namespace lbgb
