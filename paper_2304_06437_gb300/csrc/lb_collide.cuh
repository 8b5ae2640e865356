// lb_collide.cuh -- the per-node arithmetic of the regularized step, shared by
// every kernel so that all schedules produce bit-identical populations.
//
// All quantities are deviations: the stored population is ft_a = f_a - t_a rho0
// and the density is drho = rho - rho0.  With cs^2 = 1/3:
//
//   moments (section 4, moment reconstruction):
//     drho = sum ft_a,  j = sum ft_a c_a,  P = sum ft_a c_a c_a
//     u = (j + F/2) / rho0                       (He-Luo reading, forcing shift)
//     Pi^neq = P - drho cs2 I - rho0 u u          (= sum (f - f^eq) c c)
//   post-collision set (Eq. LBexp with f^neq -> fhat^neq of Eq. hermite, plus
//   the second-order forcing term):
//     ft*_a = t_a [ A + B.c_a + c_a.C.c_a ]
//     A = drho - 3/2 rho0 u.u - 3/2 (1-omega) tr Pi^neq - 3 (1 - omega/2) u.F
//     B = 3 rho0 u + 3/2 F
//     C = 9/2 [ rho0 u u + (1-omega) Pi^neq + (1 - omega/2)(u F + F u) ]
//   (kept as the diagonal C_aa and the doubled off-diagonal 2 C_ab)
//   This is t_a [drho + rho0 (c.u/cs2 + (cc - cs2 I):uu/(2 cs2^2))]
//   + (1-omega) t_a [c.j^neq/cs2 + (cc - cs2 I):Pi^neq/(2 cs2^2)] + S_a with
//   j^neq = -F/2, written as a quadratic form in c_a.
//
// Every operation is written out explicitly (fused multiply-adds through
// fma_r) and the library is compiled with -fmad=false, so the rounding
// sequence is fixed by this source: the fused kernel, the two-pass kernel and
// the shell exporter evaluate the same instructions on the same inputs and
// agree bit for bit.
#pragma once

#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <type_traits>
#include <utility>

#include "lb_lattice.cuh"

#define LB_DEV __device__ __forceinline__

namespace lbgb {

// compile-time loop: f(std::integral_constant<int, I>) for I in [B, E)
template <int B, int E, class F>
LB_DEV void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(std::forward<F>(f));
  }
}

// ------------------------------------------------------------ storage types
template <class S, class R> LB_DEV R load_as(const S v);
template <> LB_DEV float load_as<float, float>(const float v) { return v; }
template <> LB_DEV double load_as<double, double>(const double v) { return v; }
template <> LB_DEV float load_as<__half, float>(const __half v) { return __half2float(v); }
template <> LB_DEV float load_as<__nv_bfloat16, float>(const __nv_bfloat16 v) { return __bfloat162float(v); }

template <class S, class R> LB_DEV S store_as(const R v);
template <> LB_DEV float store_as<float, float>(const float v) { return v; }
template <> LB_DEV double store_as<double, double>(const double v) { return v; }
template <> LB_DEV __half store_as<__half, float>(const float v) { return __float2half_rn(v); }
template <> LB_DEV __nv_bfloat16 store_as<__nv_bfloat16, float>(const float v) { return __float2bfloat16_rn(v); }

// round a value to the storage precision and back (identity for FP32/FP64)
template <class S, class R>
LB_DEV R round_to_storage(const R v) {
  return load_as<S, R>(store_as<S, R>(v));
}

// ------------------------------------------------------------ parameters
template <class R>
struct Phys {
  R rho0, inv_rho0;
  R om1;     // 1 - omega
  R g;       // 1 - omega / 2
  R F[3];    // body force (internal axes)
  R hF[3];   // F / 2
  R cs2;     // 1/3 rounded to R
  // products of the constants above, formed once in FP64 on the host
  R c15rho0, c15om1, c3rho0, c45rho0, c45om1, c9rho0, c9om1, c3g, c9g;
};

LB_DEV float fma_r(float a, float b, float c) { return fmaf(a, b, c); }
LB_DEV double fma_r(double a, double b, double c) { return fma(a, b, c); }

template <class R>
struct Mom {
  R drho;
  R u[3];
  R pi[6];  // Pi^neq: xx, yy, zz, xy, xz, yz (internal axes)
};

template <class R>
struct Coef {
  R A;
  R B[3];
  R C[3];   // diagonal xx, yy, zz
  R C2[3];  // doubled off-diagonal: xy, xz, yz
};

// pair index helpers: the unordered pairs {a, opp(a)} with a < opp(a)
template <class L>
LB_HD constexpr int n_pairs() { return (L::Q - 1) / 2; }
template <class L>
LB_HD constexpr int pair_first(int p) {
  int n = 0;
  for (int a = 1; a < L::Q; ++a)
    if (a < L::opp(a)) {
      if (n == p) return a;
      ++n;
    }
  return -1;
}

// off-diagonal slot of an axis pair (0,1)->0, (0,2)->1, (1,2)->2
LB_HD constexpr int od(int al, int be) { return al + be - 1; }

// pairs whose velocity has a nonzero component along axis al, and the k-th
template <class L>
LB_HD constexpr int axis_pair_count(int al) {
  int n = 0;
  for (int p = 0; p < n_pairs<L>(); ++p) n += comp<L>(al, pair_first<L>(p)) != 0 ? 1 : 0;
  return n;
}
template <class L>
LB_HD constexpr int axis_pair(int al, int k) {
  for (int p = 0; p < n_pairs<L>(); ++p)
    if (comp<L>(al, pair_first<L>(p)) != 0) {
      if (k == 0) return p;
      --k;
    }
  return -1;
}
// pairs with nonzero components along both al and be, and the k-th
template <class L>
LB_HD constexpr int od_pair_count(int al, int be) {
  int n = 0;
  for (int p = 0; p < n_pairs<L>(); ++p) n += comp<L>(al, pair_first<L>(p)) * comp<L>(be, pair_first<L>(p)) != 0;
  return n;
}
template <class L>
LB_HD constexpr int od_pair(int al, int be, int k) {
  for (int p = 0; p < n_pairs<L>(); ++p)
    if (comp<L>(al, pair_first<L>(p)) * comp<L>(be, pair_first<L>(p)) != 0) {
      if (k == 0) return p;
      --k;
    }
  return -1;
}

// balanced pairwise sum of term(k), k in [Lo, Hi)
template <int Lo, int Hi, class R, class F>
LB_DEV R tree_sum(F&& term) {
  if constexpr (Hi - Lo == 1) {
    return term(std::integral_constant<int, Lo>{});
  } else {
    constexpr int Mid = Lo + (Hi - Lo) / 2;
    return tree_sum<Lo, Mid, R>(term) + tree_sum<Mid, Hi, R>(term);
  }
}

// ------------------------------------------------------------ moments
template <class L, class R, bool FORCE>
LB_DEV void moments(const R (&f)[L::Q], const Phys<R>& ph, Mom<R>& m) {
  // even and odd pair sums: s = f_a + f_abar, t = f_a - f_abar
  R s[n_pairs<L>()], t[n_pairs<L>()];
  static_for<0, n_pairs<L>()>([&](auto P) {
    constexpr int p = decltype(P)::value;
    constexpr int a = pair_first<L>(p);
    constexpr int b = L::opp(a);
    s[p] = f[a] + f[b];
    t[p] = f[a] - f[b];
  });
  // the sums run as balanced trees (short dependency chains for the FMA
  // pipe); every kernel evaluates this same order, so the schedules agree
  // bit for bit
  constexpr int NP = n_pairs<L>();
  const R drho = tree_sum<0, NP + 1, R>([&](auto K) -> R {
    constexpr int k = decltype(K)::value;
    if constexpr (k == 0) return f[0];
    else return s[k - 1];
  });
  R j[3] = {R(0), R(0), R(0)};
  R Pd[3] = {R(0), R(0), R(0)};
  R Po[3] = {R(0), R(0), R(0)};
  static_for<0, 3>([&](auto AL) {
    constexpr int al = decltype(AL)::value;
    constexpr int n = axis_pair_count<L>(al);
    if constexpr (n > 0) {
      j[al] = tree_sum<0, n, R>([&](auto K) -> R {
        constexpr int p = axis_pair<L>(al, decltype(K)::value);
        if constexpr (comp<L>(al, pair_first<L>(p)) == 1) return t[p];
        else return -t[p];
      });
      Pd[al] = tree_sum<0, n, R>([&](auto K) -> R { return s[axis_pair<L>(al, decltype(K)::value)]; });
    }
    static_for<al + 1, 3>([&](auto BE) {
      constexpr int be = decltype(BE)::value;
      constexpr int no = od_pair_count<L>(al, be);
      if constexpr (no > 0) {
        Po[od(al, be)] = tree_sum<0, no, R>([&](auto K) -> R {
          constexpr int p = od_pair<L>(al, be, decltype(K)::value);
          if constexpr (comp<L>(al, pair_first<L>(p)) * comp<L>(be, pair_first<L>(p)) == 1) return s[p];
          else return -s[p];
        });
      }
    });
  });
  m.drho = drho;
  R ru[3];
  static_for<0, 3>([&](auto AL) {
    constexpr int al = decltype(AL)::value;
    if constexpr (L::axis(al)) {
      if constexpr (FORCE) m.u[al] = (j[al] + ph.hF[al]) * ph.inv_rho0;
      else m.u[al] = j[al] * ph.inv_rho0;
    } else {
      m.u[al] = R(0);
    }
    ru[al] = ph.rho0 * m.u[al];
  });
  static_for<0, 3>([&](auto AL) {
    constexpr int al = decltype(AL)::value;
    if constexpr (L::axis(al)) m.pi[al] = fma_r(-ru[al], m.u[al], fma_r(-ph.cs2, drho, Pd[al]));
    else m.pi[al] = R(0);
  });
  static_for<0, 3>([&](auto AL) {
    constexpr int al = decltype(AL)::value;
    static_for<al + 1, 3>([&](auto BE) {
      constexpr int be = decltype(BE)::value;
      if constexpr (L::axis(al) && L::axis(be)) m.pi[3 + od(al, be)] = fma_r(-ru[al], m.u[be], Po[od(al, be)]);
      else m.pi[3 + od(al, be)] = R(0);
    });
  });
}

// ------------------------------------------------------------ coefficients
template <class L, class R, bool FORCE>
LB_DEV void coeffs(const Mom<R>& m, const Phys<R>& ph, Coef<R>& k) {
  R usq = R(0), tr = R(0), uF = R(0);
  static_for<0, 3>([&](auto AL) {
    constexpr int al = decltype(AL)::value;
    if constexpr (L::axis(al)) {
      usq = fma_r(m.u[al], m.u[al], usq);
      tr = tr + m.pi[al];
      if constexpr (FORCE) uF = fma_r(m.u[al], ph.F[al], uF);
    }
  });
  R A = fma_r(-ph.c15om1, tr, fma_r(-ph.c15rho0, usq, m.drho));
  if constexpr (FORCE) A = fma_r(-ph.c3g, uF, A);
  k.A = A;
  static_for<0, 3>([&](auto AL) {
    constexpr int al = decltype(AL)::value;
    R b = ph.c3rho0 * m.u[al];
    R c = fma_r(ph.c45om1, m.pi[al], (ph.c45rho0 * m.u[al]) * m.u[al]);
    if constexpr (FORCE) {
      b = fma_r(R(1.5), ph.F[al], b);
      c = fma_r(ph.c9g, m.u[al] * ph.F[al], c);
    }
    k.B[al] = b;
    k.C[al] = c;
  });
  static_for<0, 3>([&](auto AL) {
    constexpr int al = decltype(AL)::value;
    static_for<al + 1, 3>([&](auto BE) {
      constexpr int be = decltype(BE)::value;
      R c = fma_r(ph.c9om1, m.pi[3 + od(al, be)], (ph.c9rho0 * m.u[al]) * m.u[be]);
      if constexpr (FORCE) c = fma_r(ph.c9g, fma_r(m.u[al], ph.F[be], ph.F[al] * m.u[be]), c);
      k.C2[od(al, be)] = c;
    });
  });
}

// ------------------------------------------------------------ one population
// ft*_a = t_a (even + odd), even = A + sum_{c_al != 0} C_alal + sum c_al c_be C2,
// odd = sum c_al B_al; evaluated as fma(t_a, even, t_a odd).  post_parts
// returns even and t_a odd; opp(a) has the same even part and exactly the
// negated odd part (every term of its sum is negated)
template <class L, class R, int a>
LB_DEV void post_parts(const Coef<R>& k, R& even, R& wodd) {
  even = k.A;
  static_for<0, 3>([&](auto AL) {
    constexpr int al = decltype(AL)::value;
    if constexpr (comp<L>(al, a) != 0) even = even + k.C[al];
  });
  static_for<0, 3>([&](auto AL) {
    constexpr int al = decltype(AL)::value;
    static_for<al + 1, 3>([&](auto BE) {
      constexpr int be = decltype(BE)::value;
      constexpr int cc = comp<L>(al, a) * comp<L>(be, a);
      if constexpr (cc == 1) even = even + k.C2[od(al, be)];
      if constexpr (cc == -1) even = even - k.C2[od(al, be)];
    });
  });
  // odd part: the sum of the signed B components in axis order
  R odd = R(0);
  bool first = true;
  static_for<0, 3>([&](auto AL) {
    constexpr int al = decltype(AL)::value;
    constexpr int ca = comp<L>(al, a);
    if constexpr (ca != 0) {
      const R term = (ca == 1) ? k.B[al] : -k.B[al];
      odd = first ? term : odd + term;
      first = false;
    }
  });
  wodd = R(weight<L>(a)) * odd;
}

template <class L, class R, int a>
LB_DEV R post(const Coef<R>& k) {
  constexpr R w = R(weight<L>(a));
  R even, wodd;
  post_parts<L, R, a>(k, even, wodd);
  if constexpr (a == 0) return w * even;  // rest population: no odd part
  else return fma_r(w, even, wodd);
}

// full regularized collision of one node: ft -> ft*; the two members of a
// velocity pair share the even part and take -/+ the odd part
template <class L, class R, bool FORCE>
LB_DEV void collide(const R (&f)[L::Q], const Phys<R>& ph, R (&out)[L::Q]) {
  Mom<R> m;
  moments<L, R, FORCE>(f, ph, m);
  Coef<R> k;
  coeffs<L, R, FORCE>(m, ph, k);
  static_assert(L::cx(0) == 0 && L::cy(0) == 0 && L::cz(0) == 0, "direction 0 is the rest population");
  out[0] = post<L, R, 0>(k);
  static_for<0, n_pairs<L>()>([&](auto P) {
    constexpr int p = decltype(P)::value;
    constexpr int a = pair_first<L>(p);
    constexpr int b = L::opp(a);
    constexpr R w = R(weight<L>(a));
    R even, wodd;
    post_parts<L, R, a>(k, even, wodd);
    out[a] = fma_r(w, even, wodd);
    out[b] = fma_r(w, even, -wodd);
  });
}

}  // namespace lbgb
