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
//     a launch, so in-place update is race free;
//   * the CTA sweeps its planes along z.  TMA streams plane z + NS of the
//     population array into a ring of shared-memory slots (mbarrier complete-
//     tx), every thread collides its node of plane z (lb_collide.cuh) into a
//     shared window, and then gathers, for each direction a, the collided
//     value of its upstream neighbour (x - c_a) from the window.  The value
//     belongs to destination plane z + c_az, so each thread keeps three planes
//     of partially gathered populations in registers and writes plane z - 1
//     once it is complete;
//   * populations whose upstream node lies in another brick come from a small
//     "shell" buffer: after finishing a boundary node, its owner collides the
//     new state once more and exports the outgoing populations (those whose
//     c_a points out of the brick) into the other parity of the shell, which
//     neighbouring bricks read in the NEXT launch.  Only boundary populations
//     travel through the shell; there is no second population array and no
//     full-size moment array;
//   * halfway bounce-back (and the moving-wall term) is applied where the
//     upstream point lies outside a non-periodic face.
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

template <class L, class S, class R, int BX, int BY, int NS>
struct K1Shape {
  static constexpr int Q = L::Q;
  static constexpr int NT = BX * BY;
  static constexpr int NXF = count_dirs<L>(0, 1);
  static constexpr int NYF = count_dirs<L>(1, 1);
  static constexpr int NZF = count_dirs<L>(2, 1);
  static constexpr int HW = NXF * (BY + 2);  // west (and east) halo entries
  static constexpr int HS = NYF * BX;        // south (and north) halo entries
  static constexpr int H = 2 * HW + 2 * HS;
  static constexpr int HPT = (H + NT - 1) / NT;
  static constexpr size_t SLOT = size_t(Q) * BY * BX * sizeof(S);
  static constexpr size_t OFF_WIN = align128(NS * SLOT);
  static constexpr size_t OFF_HALO = OFF_WIN + align128(size_t(Q) * BY * BX * sizeof(R));
  static constexpr size_t OFF_BAR = OFF_HALO + align128(size_t(H > 0 ? H : 1) * sizeof(R));
  static constexpr size_t SMEM = OFF_BAR + align128(NS * sizeof(uint64_t));
};

template <class L, class S, class R, int BX, int BY, int NS, bool FORCE>
__global__ void __launch_bounds__(BX* BY, 1)
    k1_fused_step(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ K1Args<R> args) {
  using Sh = K1Shape<L, S, R, BX, BY, NS>;
  constexpr int Q = L::Q;
  constexpr int NT = Sh::NT;
  constexpr int NXF = Sh::NXF, NYF = Sh::NYF, NZF = Sh::NZF;
  constexpr int HW = Sh::HW, HS = Sh::HS, H = Sh::H, HPT = Sh::HPT;

  extern __shared__ __align__(128) unsigned char smem[];
  S* slots = reinterpret_cast<S*>(smem);
  R* win = reinterpret_cast<R*>(smem + Sh::OFF_WIN);
  R* halo = reinterpret_cast<R*>(smem + Sh::OFF_HALO);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR);

  const int tid = threadIdx.x;
  const int tx = tid % BX;
  const int ty = tid / BX;
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

  // bounce-back predicates of this node (x, y axes): the upstream point of a
  // direction with c = +1 is x - 1, which leaves a non-periodic low face at x = 0
  const bool bxlo = (x == 0) && !args.per[0];
  const bool bxhi = (x == nx - 1) && !args.per[0];
  const bool bylo = (y == 0) && !args.per[1];
  const bool byhi = (y == ny - 1) && !args.per[1];

  S* __restrict__ fglob = static_cast<S*>(args.f);
  const R* __restrict__ shc = args.sh_cur;
  R* __restrict__ shn = args.sh_next;

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

  // halo descriptors: entry h -> (global base offset, z stride, smem index)
  int64_t hbase[HPT];
  int64_t hzs[HPT];
  bool hval[HPT];
#pragma unroll
  for (int e = 0; e < HPT; ++e) {
    const int h = tid + e * NT;
    hval[e] = false;
    hbase[e] = 0;
    hzs[e] = 1;
    if (h < H) {
      if (h < 2 * HW) {
        const bool west = h < HW;
        const int hh = west ? h : h - HW;
        const int ia = hh / (BY + 2);
        const int j = hh % (BY + 2);
        int sy = y0 - 1 + j;
        bool ok = west ? nbW : nbE;
        if (sy < 0 || sy >= ny) {
          if (args.per[1]) sy = (sy + ny) % ny;
          else ok = false;
        }
        // west halo reads the high-face export (side 1) of the west brick
        const int side = west ? 1 : 0;
        const int bb = west ? bIw : bIe;
        hval[e] = ok;
        hbase[e] = args.sx_off + ((int64_t(side) * nbx + bb) * NXF + ia) * int64_t(nz) * ny + sy;
        hzs[e] = ny;
      } else {
        const int h2 = h - 2 * HW;
        const bool south = h2 < HS;
        const int hh = south ? h2 : h2 - HS;
        const int ia = hh / BX;
        const int i = hh % BX;
        const bool ok = (south ? nbS : nbN) && i < bxa;
        const int side = south ? 1 : 0;
        const int bb = south ? bJs : bJn;
        hval[e] = ok;
        hbase[e] = args.sy_off + ((int64_t(side) * nby + bb) * NYF + ia) * int64_t(nz) * nx + x0 + i;
        hzs[e] = nx;
      }
    }
  }
  (void)HS;
  (void)NZF;

  auto plane_needed = [&](int z) -> bool {
    if (z >= z0 && z < z1) return true;
    if (z == z0 - 1) return nbD;
    if (z == z1) return nbU;
    return false;
  };
  auto wrap_z = [&](int z) -> int { return (z + nz) % nz; };

  R hreg[HPT];
  auto halo_fetch = [&](int z) {
    const int zw = wrap_z(z);
#pragma unroll
    for (int e = 0; e < HPT; ++e) hreg[e] = hval[e] ? shc[hbase[e] + int64_t(zw) * hzs[e]] : R(0);
  };
  if (plane_needed(z0 - 1)) halo_fetch(z0 - 1);

  // three destination planes of partially gathered populations
  R G0[Q], G1[Q], G2[Q];  // planes z-1, z, z+1
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    G0[a] = R(0);
    G1[a] = R(0);
    G2[a] = R(0);
  }

  const int n_it = (z1 - z0) + 2;
  for (int it = 0; it < n_it; ++it) {
    const int z = z0 - 1 + it;
    const bool real = z >= z0 && z < z1;
    const bool need = plane_needed(z);
    const int k = z - z0;
    const int slot = real ? (k % NS) : 0;
    bool timeout = false;

    // ---------------------------------------------- phase 1: window of plane z
    if (real) {
      if (!mbar_wait_bounded(&bars[slot], (k / NS) & 1, kWaitLimitNs)) timeout = true;
      if (!timeout && active) {
        const S* sl = slots + size_t(slot) * Q * BY * BX + ty * BX + tx;
        R fl[Q], fs[Q];
        static_for<0, Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          fl[a] = load_as<S, R>(sl[a * BY * BX]);
        });
        collide<L, R, FORCE>(fl, args.ph, fs);
        static_for<0, Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          win[(a * BY + ty) * BX + tx] = fs[a];
        });
      }
    } else if (need && active) {
      // virtual plane just outside the brick: the neighbouring brick's export
      const bool low = (z == z0 - 1);
      const int side = low ? 1 : 0;
      const int bb = low ? bKd : bKu;
      static_for<0, Q>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int cz = L::cz(a);
        if constexpr (cz != 0) {
          if ((cz == 1) == low) {
            constexpr int iz = sub_index<L>(2, cz, a);
            win[(a * BY + ty) * BX + tx] =
                shc[args.sz_off + ((int64_t(side) * nbz + bb) * NZF + iz) * int64_t(ny) * nx + int64_t(y) * nx + x];
          }
        }
      });
    }
    if (need) {
#pragma unroll
      for (int e = 0; e < HPT; ++e)
        if (tid + e * NT < H) halo[tid + e * NT] = hreg[e];
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

    // ---------------------------------------------- phase 2: gather
    if (active && need) {
      const bool bzlo_z = (z == 0) && !args.per[2];
      const bool bzhi_z = (z == nz - 1) && !args.per[2];
      static_for<0, Q>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        constexpr int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
        // x / y part of the bounce-back combo of direction a at this node
        int cxy = 0;
        if constexpr (cx == 1) cxy |= bxlo ? 1 : 0;
        if constexpr (cx == -1) cxy |= bxhi ? 1 : 0;
        if constexpr (cy == 1) cxy |= bylo ? 2 : 0;
        if constexpr (cy == -1) cxy |= byhi ? 2 : 0;
        // pull for destination plane zd = z + cz from the window of plane z
        const int zd = z + cz;
        if (zd >= z0 && zd < z1) {
          int cb = cxy;
          if constexpr (cz == 1) cb |= ((zd == 0) && !args.per[2]) ? 4 : 0;
          if constexpr (cz == -1) cb |= ((zd == nz - 1) && !args.per[2]) ? 4 : 0;
          if (cb == 0) {
            R v;
            bool done = false;
            if constexpr (cx == 1) {
              if (tx == 0) {
                v = halo[sub_index<L>(0, 1, a) * (BY + 2) + (ty - cy + 1)];
                done = true;
              }
            }
            if constexpr (cx == -1) {
              if (tx == bxa - 1) {
                v = halo[HW + sub_index<L>(0, -1, a) * (BY + 2) + (ty - cy + 1)];
                done = true;
              }
            }
            if constexpr (cy == 1) {
              if (!done && ty == 0) {
                v = halo[2 * HW + sub_index<L>(1, 1, a) * BX + (tx - cx)];
                done = true;
              }
            }
            if constexpr (cy == -1) {
              if (!done && ty == bya - 1) {
                v = halo[2 * HW + HS + sub_index<L>(1, -1, a) * BX + (tx - cx)];
                done = true;
              }
            }
            if (!done) v = win[(a * BY + (ty - cy)) * BX + (tx - cx)];
            if constexpr (cz == -1) G0[a] = v;
            if constexpr (cz == 0) G1[a] = v;
            if constexpr (cz == 1) G2[a] = v;
          }
        }
        // halfway bounce-back into plane z (own node, real planes only)
        if (real) {
          int cb = cxy;
          if constexpr (cz == 1) cb |= bzlo_z ? 4 : 0;
          if constexpr (cz == -1) cb |= bzhi_z ? 4 : 0;
          constexpr int oa = L::opp(a);
          if (cb != 0) G1[a] = win[(oa * BY + ty) * BX + tx] + args.bb[a][cb];
        }
      });
    }

    // ---------------------------------------------- plane z - 1 is complete
    const int zd = z - 1;
    if (active && zd >= z0 && zd < z1) {
      const int64_t o = x + args.pitch * (y + int64_t(ny) * zd);
      S st[Q];
      static_for<0, Q>([&](auto A_) {
        constexpr int a = decltype(A_)::value;
        st[a] = store_as<S, R>(G0[a]);
        fglob[a * args.vol + o] = st[a];
      });
      const bool eW = tx == 0 && nbW, eE = tx == bxa - 1 && nbE;
      const bool eS = ty == 0 && nbS, eN = ty == bya - 1 && nbN;
      const bool eD = zd == z0 && nbD, eU = zd == z1 - 1 && nbU;
      if (eW || eE || eS || eN || eD || eU) {
        // collide the stored (rounded) state once more and export the
        // populations that leave the brick; the next launch reads them
        R fr[Q];
        static_for<0, Q>([&](auto A_) {
          constexpr int a = decltype(A_)::value;
          fr[a] = load_as<S, R>(st[a]);
        });
        Mom<R> m;
        moments<L, R, FORCE>(fr, args.ph, m);
        Coef<R> kc;
        coeffs<L, R, FORCE>(m, args.ph, kc);
        static_for<0, Q>([&](auto A_) {
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
                shn[args.sx_off + ((int64_t(side) * nbx + bI) * NXF + ia) * int64_t(nz) * ny + int64_t(zd) * ny + y] = v;
              }
            }
            if constexpr (cy != 0) {
              if (wy) {
                constexpr int side = cy == 1 ? 1 : 0;
                constexpr int ia = sub_index<L>(1, cy, a);
                shn[args.sy_off + ((int64_t(side) * nby + bJ) * NYF + ia) * int64_t(nz) * nx + int64_t(zd) * nx + x] = v;
              }
            }
            if constexpr (cz != 0) {
              if (wz) {
                constexpr int side = cz == 1 ? 1 : 0;
                constexpr int ia = sub_index<L>(2, cz, a);
                shn[args.sz_off + ((int64_t(side) * nbz + bK) * NZF + ia) * int64_t(ny) * nx + int64_t(y) * nx + x] = v;
              }
            }
          }
        });
      }
    }
    // rotate the destination planes
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      G0[a] = G1[a];
      G1[a] = G2[a];
    }
    __syncthreads();
  }
}

// Shell bootstrap: collide every brick-boundary node of the current state and
// export its outgoing populations into shell parity `sh_next` (used once after
// the state is set from outside; the steps keep the shell current).
template <class L, class S, class R, int BX, int BY, bool FORCE>
__global__ void __launch_bounds__(256) k1_bootstrap(const __grid_constant__ K1Args<R> args) {
  constexpr int Q = L::Q;
  constexpr int NXF = count_dirs<L>(0, 1), NYF = count_dirs<L>(1, 1), NZF = count_dirs<L>(2, 1);
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
    Mom<R> m;
    moments<L, R, FORCE>(fr, args.ph, m);
    Coef<R> kc;
    coeffs<L, R, FORCE>(m, args.ph, kc);
    R* shn = args.sh_next;
    const int nx = args.nx, ny = args.ny, nz = args.nz;
    static_for<0, Q>([&](auto A_) {
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
            shn[args.sx_off + ((int64_t(side) * args.nbx + bI) * NXF + ia) * int64_t(nz) * ny + int64_t(z) * ny + y] = v;
          }
        }
        if constexpr (cy != 0) {
          if (wy) {
            constexpr int side = cy == 1 ? 1 : 0;
            constexpr int ia = sub_index<L>(1, cy, a);
            shn[args.sy_off + ((int64_t(side) * args.nby + bJ) * NYF + ia) * int64_t(nz) * nx + int64_t(z) * nx + x] = v;
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
}

}  // namespace lbgb
