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

#include "lb_dispatch.cuh"
#include "lb_ptx.cuh"

namespace lbgb {

template <class R>
struct K1Args {
  Phys<R> ph;
  int nx, ny, nz;
  int64_t pitch, vol;
  int per[3];
  int bz, nbx, nby, nbz;
  void* f;
  const R* sh_cur;
  R* sh_next;
  int64_t sx_off, sy_off, sz_off;
  int* status;
  R bb[27][8];
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
// the ia-th direction whose component along axis is sign
template <class L>
LB_HD constexpr int dir_of_sub(int axis, int sign, int ia) {
  for (int a = 0; a < L::Q; ++a)
    if (comp<L>(axis, a) == sign) {
      if (ia == 0) return a;
      --ia;
    }
  return -1;
}

template <class L, class S, class R, int BX, int BY, int NS>
struct K1Shape {
  static constexpr int Q = L::Q;
  static constexpr int NT = BX * BY;
  static constexpr int NXF = count_dirs<L>(0, 1);
  static constexpr int NYF = count_dirs<L>(1, 1);
  static constexpr int NZF = count_dirs<L>(2, 1);
  static constexpr int NLAT = n_lateral<L>();
  static constexpr int PY = NYF > 0 ? 1 : 0;  // window padding rows (none without y motion)
  static constexpr int WX = BX + 2;
  static constexpr int WY = BY + 2 * PY;
  static constexpr int HW = NXF * WY;  // west (and east) ring entries
  static constexpr int HS = NYF * BX;  // south (and north) ring entries
  static constexpr int H = 2 * HW + 2 * HS;
  static constexpr int HPT = (H + NT - 1) / NT;
  static constexpr int PMAX = NYF > 0 ? 2 * BX + 2 * (BY - 2) : 2;  // lateral perimeter nodes
  static constexpr int NEXW = (PMAX + 31) / 32;                     // export warps
  static constexpr size_t SLOT = size_t(Q) * BY * BX * sizeof(S);
  static constexpr size_t WIN = size_t(NLAT) * WY * WX * sizeof(R);
  static constexpr size_t STAGE = size_t(Q) * PMAX * sizeof(R);
  static constexpr size_t OFF_WIN = align128(NS * SLOT);
  static constexpr size_t OFF_STAGE = OFF_WIN + align128(WIN);
  static constexpr size_t OFF_BAR = OFF_STAGE + align128(2 * STAGE);
  static constexpr size_t SMEM = OFF_BAR + align128(NS * sizeof(uint64_t));
  static_assert(BY == 1 || NYF > 0, "a 2D brick has one internal row");
  static_assert(PMAX <= NT, "perimeter larger than the CTA");
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

// Collide the completed (rounded) state of one node once more and export the
// populations that leave the brick through the flagged faces.
template <class L, class S, class R, bool FORCE>
__device__ __forceinline__ void export_node(const K1Args<R>& args, const R (&fin)[L::Q], int x, int y, int zd,
                                            bool eW, bool eE, bool eS, bool eN, bool eD, bool eU, int bI, int bJ,
                                            int bK) {
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
  const int nx = args.nx, ny = args.ny, nz = args.nz;
  static_for<0, L::Q>([&](auto A_) {
    constexpr int a = decltype(A_)::value;
    constexpr int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
    const bool wx = (cx == -1 && eW) || (cx == 1 && eE);
    const bool wy = (cy == -1 && eS) || (cy == 1 && eN);
    const bool wz = (cz == -1 && eD) || (cz == 1 && eU);
    if (wx || wy || wz) {
      const R v = post<L, R, a>(kc);
      if constexpr (cx != 0) {
        if (wx) {
          constexpr int side = cx == 1 ? 1 : 0;
          constexpr int ia = sub_index<L>(0, cx, a);
          shn[args.sx_off + ((int64_t(side) * args.nbx + bI) * NXF + ia) * int64_t(nz) * ny + int64_t(zd) * ny + y] = v;
        }
      }
      if constexpr (cy != 0) {
        if (wy) {
          constexpr int side = cy == 1 ? 1 : 0;
          constexpr int ia = sub_index<L>(1, cy, a);
          shn[args.sy_off + ((int64_t(side) * args.nby + bJ) * NYF + ia) * int64_t(nz) * nx + int64_t(zd) * nx + x] = v;
        }
      }
      if constexpr (cz != 0) {
        if (wz) {
          constexpr int side = cz == 1 ? 1 : 0;
          constexpr int ia = sub_index<L>(2, cz, a);
          shn[args.sz_off + ((int64_t(side) * args.nbz + bK) * NZF + ia) * int64_t(ny) * nx + int64_t(y) * nx + x] = v;
        }
      }
    }
  });
}

template <class L, class S, class R, int BX, int BY, int NS, bool FORCE>
__global__ void __launch_bounds__(BX* BY, 1)
    k1_fused_step(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ K1Args<R> args) {
  using Sh = K1Shape<L, S, R, BX, BY, NS>;
  constexpr int Q = L::Q;
  constexpr int NT = Sh::NT;
  constexpr int NXF = Sh::NXF, NYF = Sh::NYF, NZF = Sh::NZF;
  constexpr int PY = Sh::PY, WX = Sh::WX, WY = Sh::WY;
  constexpr int HW = Sh::HW, HS = Sh::HS, H = Sh::H, HPT = Sh::HPT;
  constexpr int PMAX = Sh::PMAX, NEXW = Sh::NEXW;
  constexpr int WPLANE = WY * WX;

  extern __shared__ __align__(128) unsigned char smem[];
  S* slots = reinterpret_cast<S*>(smem);
  R* win = reinterpret_cast<R*>(smem + Sh::OFF_WIN);
  R* stage = reinterpret_cast<R*>(smem + Sh::OFF_STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR);

  const int tid = threadIdx.x;
  const int tx = tid % BX;
  const int ty = tid / BX;
  const int warp = tid / 32, lane = tid % 32;
  const int nx = args.nx, ny = args.ny, nz = args.nz;
  const int nbx = args.nbx, nby = args.nby, nbz = args.nbz;
  const int bI = blockIdx.x % nbx;
  const int bJ = (blockIdx.x / nbx) % nby;
  const int bK = blockIdx.x / (nbx * nby);
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
  const bool nbD = z0 > 0 || args.per[2];
  const bool nbU = z1 < nz || args.per[2];
  const int bIw = (bI + nbx - 1) % nbx, bIe = (bI + 1) % nbx;
  const int bJs = (bJ + nby - 1) % nby, bJn = (bJ + 1) % nby;
  const int bKd = (bK + nbz - 1) % nbz, bKu = (bK + 1) % nbz;

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
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
    prefetch_tmap(&tmap);
  }
  __syncthreads();
  int issued = 0;  // real planes whose load was issued (thread 0's view)
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      const int zz = z0 + s;
      if (zz < z1) {
        mbar_arrive_expect_tx(&bars[s], static_cast<uint32_t>(Sh::SLOT));
        tma_load_4d(slots + size_t(s) * Q * BY * BX, &tmap, x0, y0, zz, 0, &bars[s]);
        ++issued;
      }
    }
  }

  // ring entries of the window: entry h -> (global base, z stride, window index)
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
        const int r = hh % WY;  // window row; source y = y0 - PY + r
        int sy = y0 - PY + r;
        bool ok = (west ? nbW : nbE) && r < bya + 2 * PY;
        if (sy < 0 || sy >= ny) {
          if (args.per[1]) sy = (sy + ny) % ny;
          else ok = false;
        }
        const int a = dir_of_sub<L>(0, west ? 1 : -1, ia);
        const int col = west ? 0 : bxa + 1;
        // the west ring holds the high-face export (side 1) of the west brick
        const int side = west ? 1 : 0;
        const int bb = west ? bIw : bIe;
        hval[e] = ok;
        hbase[e] = args.sx_off + ((int64_t(side) * nbx + bb) * NXF + ia) * int64_t(nz) * ny + sy;
        hzs[e] = ny;
        hsm[e] = lat_index<L>(a) * WPLANE + r * WX + col;
      } else {
        const int h2 = h - 2 * HW;
        const bool south = h2 < HS;
        const int hh = south ? h2 : h2 - HS;
        const int ia = hh / BX;
        const int i = hh % BX;
        const bool ok = (south ? nbS : nbN) && i < bxa;
        const int a = dir_of_sub<L>(1, south ? 1 : -1, ia);
        const int row = south ? 0 : bya + 1;
        const int side = south ? 1 : 0;
        const int bb = south ? bJs : bJn;
        hval[e] = ok;
        hbase[e] = args.sy_off + ((int64_t(side) * nby + bb) * NYF + ia) * int64_t(nz) * nx + x0 + i;
        hzs[e] = nx;
        hsm[e] = lat_index<L>(a) * WPLANE + row * WX + 1 + i;
      }
    }
  }

  auto plane_needed = [&](int z) -> bool {
    if (z >= z0 && z < z1) return true;
    if (z == z0 - 1) return nbD;
    if (z == z1) return nbU;
    return false;
  };

  R hreg[HPT];
  auto halo_fetch = [&](int z) {
    const int zw = (z + nz) % nz;
#pragma unroll
    for (int e = 0; e < HPT; ++e) hreg[e] = hval[e] ? shc[hbase[e] + int64_t(zw) * hzs[e]] : R(0);
  };
  if (plane_needed(z0 - 1)) halo_fetch(z0 - 1);

  // perimeter (lateral boundary) slot of this node, and export-warp work
  const int pidx = active ? perimeter_index<NYF>(tx, ty, bxa, bya) : -1;
  const int pcount = perimeter_count<NYF>(bxa, bya);
  const bool any_lateral_export = nbW || nbE || (NYF > 0 && (nbS || nbN));

  // this thread's own cell in the window (interior of the padding ring)
  const int wbase = (ty + PY) * WX + (tx + 1);

  // three destination planes of gathered populations
  R G0[Q], G1[Q], G2[Q];  // planes z-1, z, z+1
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    G0[a] = R(0);
    G1[a] = R(0);
    G2[a] = R(0);
  }
  // bounce-back values of the z-descending directions of the previous plane;
  // applied after the next gather, which would otherwise overwrite them
  constexpr int NDN = count_dirs<L>(2, -1);
  R bdn[NDN];
  unsigned bdn_mask = 0;
#pragma unroll
  for (int i = 0; i < NDN; ++i) bdn[i] = R(0);

  const int n_it = (z1 - z0) + 2;
  for (int it = 0; it < n_it; ++it) {
    const int z = z0 - 1 + it;
    const bool real = z >= z0 && z < z1;
    const bool need = plane_needed(z);
    const int k = z - z0;
    const int slot = real ? (k % NS) : 0;
    bool timeout = false;
    R own[Q];  // this node's collided populations (real planes)

    // ---------------------------------------------- phase 1: window of plane z
    if (real) {
      if (!mbar_wait_bounded(&bars[slot], (k / NS) & 1, kWaitLimitNs)) timeout = true;
      if (!timeout && active) {
        const S* sl = slots + size_t(slot) * Q * BY * BX + ty * BX + tx;
        R fl[Q];
        static_for<0, Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          fl[a] = load_as<S, R>(sl[a * BY * BX]);
        });
        collide<L, R, FORCE>(fl, args.ph, own);
        static_for<0, Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          if constexpr (is_lateral<L>(a)) win[lat_index<L>(a) * WPLANE + wbase] = own[a];
        });
      }
    } else if (need && active) {
      // virtual plane just outside the brick: the neighbouring brick's export
      const bool low = (z == z0 - 1);
      const int side = low ? 1 : 0;
      const int bb = low ? bKd : bKu;
      const int64_t base = args.sz_off + (int64_t(side) * nbz + bb) * NZF * int64_t(ny) * nx + int64_t(y) * nx + x;
      static_for<0, Q>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int cz = L::cz(a);
        own[a] = R(0);
        if constexpr (cz != 0) {
          if ((cz == 1) == low) {
            constexpr int iz = sub_index<L>(2, cz, a);
            const R v = shc[base + int64_t(iz) * ny * nx];
            if constexpr (is_lateral<L>(a)) win[lat_index<L>(a) * WPLANE + wbase] = v;
            else own[a] = v;
          }
        }
      });
    }
    if (need) {
      // only valid entries: an invalid north/south entry of a ragged brick
      // would alias the east ring's corner cell of a diagonal direction
#pragma unroll
      for (int e = 0; e < HPT; ++e)
        if (hval[e]) win[hsm[e]] = hreg[e];
    }
    if (z + 1 <= z1 && plane_needed(z + 1)) halo_fetch(z + 1);

    if (__syncthreads_or(timeout)) {
      if (tid == 0) {
        atomicExch(args.status, LB_E_TIMEOUT);
        // drain this CTA's own copies still in flight (bounded)
        for (int kk = (k < 0 ? 0 : k); kk < issued; ++kk)
          mbar_wait_bounded(&bars[kk % NS], (kk / NS) & 1, kWaitLimitNs);
      }
      return;
    }

    // refill the slot just consumed with plane z + NS
    if (real && tid == 0) {
      const int zz = z + NS;
      if (zz < z1) {
        mbar_arrive_expect_tx(&bars[slot], static_cast<uint32_t>(Sh::SLOT));
        tma_load_4d(slots + size_t(slot) * Q * BY * BX, &tmap, x0, y0, zz, 0, &bars[slot]);
        ++issued;
      }
    }

    // ---------------------------------------------- phase 2: gather (no branches)
    if (active && need) {
      static_for<0, Q>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
        R v;
        if constexpr (is_lateral<L>(a)) v = win[lat_index<L>(a) * WPLANE + wbase - cy * WX - cx];
        else v = own[a];
        if constexpr (cz == -1) G0[a] = v;
        if constexpr (cz == 0) G1[a] = v;
        if constexpr (cz == 1) G2[a] = v;
      });
    }
    // z-descending bounce-backs of plane z - 1, saved one plane ago
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
    // halfway bounce-back for destination plane z (threads next to a wall)
    if (real && active && (xy_wall || (z_walls && (z == 0 || z == nz - 1)))) {
      const bool bzlo = z_walls && z == 0, bzhi = z_walls && z == nz - 1;
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
          if constexpr (is_lateral<L>(oa)) back = win[lat_index<L>(oa) * WPLANE + wbase];
          else back = own[oa];
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

    // ---------------------------------------------- exports of plane z - 2
    const int zx = z - 2;  // staged one iteration ago
    if (any_lateral_export && warp < NEXW && zx >= z0 && zx < z1) {
      const int p = warp * 32 + lane;
      if (p < pcount) {
        int ptx, pty;
        perimeter_node<NYF>(p, bxa, bya, ptx, pty);
        const R* st = stage + (zx & 1) * (Q * PMAX) + p;
        R fin[Q];
        static_for<0, Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          fin[a] = st[a * PMAX];
        });
        export_node<L, S, R, FORCE>(args, fin, x0 + ptx, y0 + pty, zx, ptx == 0 && nbW, ptx == bxa - 1 && nbE,
                                    pty == 0 && nbS, pty == bya - 1 && nbN, false, false, bI, bJ, bK);
      }
    }

    // ---------------------------------------------- plane z - 1 is complete
    const int zd = z - 1;
    if (active && zd >= z0 && zd < z1) {
      const int64_t o = x + args.pitch * (y + int64_t(ny) * zd);
      static_for<0, Q>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        fglob[a * args.vol + o] = store_as<S, R>(G0[a]);
      });
      if (pidx >= 0 && any_lateral_export) {
        R* st = stage + (zd & 1) * (Q * PMAX) + pidx;
        static_for<0, Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          st[a * PMAX] = G0[a];
        });
      }
      const bool eD = zd == z0 && nbD, eU = zd == z1 - 1 && nbU;
      if (eD || eU) export_node<L, S, R, FORCE>(args, G0, x, y, zd, false, false, false, false, eD, eU, bI, bJ, bK);
    }
    // rotate the destination planes
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      G0[a] = G1[a];
      G1[a] = G2[a];
    }
    __syncthreads();
  }

  // exports of the last plane (staged in the final iteration)
  const int zx = z1 - 1;
  if (any_lateral_export && warp < NEXW && zx >= z0) {
    const int p = warp * 32 + lane;
    if (p < pcount) {
      int ptx, pty;
      perimeter_node<NYF>(p, bxa, bya, ptx, pty);
      const R* st = stage + (zx & 1) * (Q * PMAX) + p;
      R fin[Q];
      static_for<0, Q>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        fin[a] = st[a * PMAX];
      });
      export_node<L, S, R, FORCE>(args, fin, x0 + ptx, y0 + pty, zx, ptx == 0 && nbW, ptx == bxa - 1 && nbE,
                                  pty == 0 && nbS, pty == bya - 1 && nbN, false, false, bI, bJ, bK);
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
    const bool eD = z == z0 && (z0 > 0 || args.per[2]);
    const bool eU = z == z1 - 1 && (z1 < args.nz || args.per[2]);
    if (!(eW || eE || eS || eN || eD || eU)) continue;
    const int64_t o = x + args.pitch * (y + int64_t(args.ny) * z);
    const S* fg = static_cast<const S*>(args.f);
    R fr[Q];
    static_for<0, Q>([&](auto A_) {
      constexpr int a = decltype(A_)::value;
      fr[a] = load_as<S, R>(fg[a * args.vol + o]);
    });
    export_node<L, S, R, FORCE>(args, fr, x, y, z, eW, eE, eS, eN, eD, eU, bI, bJ, bK);
  }
}

}  // namespace lbgb
