// lb_dispatch.cuh -- compile-time dispatch on lattice / storage precision and
// the host-side construction of the per-launch physical constants.
#pragma once

#include <cmath>

#include "lb_collide.cuh"
#include "lb_internal.h"

namespace lbgb {

template <class T>
struct type_tag {
  using type = T;
};

template <class F>
bool dispatch_lattice(int lattice, F&& f) {
  switch (lattice) {
    case LB_D2Q9: f(D2Q9{}); return true;
    case LB_D3Q19: f(D3Q19{}); return true;
    case LB_D3Q27: f(D3Q27{}); return true;
    default: return false;
  }
}

// f(type_tag<S>, type_tag<R>): S = storage type, R = arithmetic type
template <class F>
bool dispatch_storage(int storage, F&& f) {
  switch (storage) {
    case LB_F64: f(type_tag<double>{}, type_tag<double>{}); return true;
    case LB_F32: f(type_tag<float>{}, type_tag<float>{}); return true;
    case LB_F16S: f(type_tag<__half>{}, type_tag<float>{}); return true;
    case LB_BF16S: f(type_tag<__nv_bfloat16>{}, type_tag<float>{}); return true;
    default: return false;
  }
}

template <class R>
Phys<R> make_phys(const Geometry& g) {
  Phys<R> p;
  const double omega = 1.0 / g.tau;
  p.rho0 = R(g.rho0);
  p.inv_rho0 = R(1.0 / g.rho0);
  p.om1 = R(1.0 - omega);
  p.g = R(1.0 - 0.5 * omega);
  for (int k = 0; k < 3; ++k) {
    p.F[k] = R(g.force[k]);
    p.hF[k] = R(0.5 * g.force[k]);
  }
  p.cs2 = R(1.0 / 3.0);
  const double om1 = 1.0 - omega, gg = 1.0 - 0.5 * omega, r0 = g.rho0;
  p.c15rho0 = R(1.5 * r0);
  p.c15om1 = R(1.5 * om1);
  p.c3rho0 = R(3.0 * r0);
  p.c45rho0 = R(4.5 * r0);
  p.c45om1 = R(4.5 * om1);
  p.c9rho0 = R(9.0 * r0);
  p.c9om1 = R(9.0 * om1);
  p.c3g = R(3.0 * gg);
  p.c9g = R(9.0 * gg);
  return p;
}

// Halfway bounce-back term 2 t_a rho0 (c_a . u_w) / cs2 for direction a when
// the upstream point leaves the domain through the faces named by `combo`
// (bit 0: x, bit 1: y, bit 2: z; the side follows the sign of c_a).  A link
// leaving through several non-periodic faces uses a stationary wall if any
// crossed face is stationary, else the first crossed face in the order
// -x,+x,-y,+y,-z,+z (the corner reading of the paper's wall rule).
template <class L, class R>
void make_bounce_terms(const Geometry& g, R (*bb)[8]) {
  for (int a = 0; a < L::Q; ++a) {
    const int c[3] = {L::cx(a), L::cy(a), L::cz(a)};
    for (int combo = 0; combo < 8; ++combo) {
      bool any_stationary = false;
      int first = -1;
      bool valid = true;
      for (int ax = 0; ax < 3; ++ax) {
        if (!(combo >> ax & 1)) continue;
        if (c[ax] == 0) { valid = false; break; }
        // pulling from y - c: c > 0 leaves through the low face
        const int face = 2 * ax + (c[ax] > 0 ? 0 : 1);
        const int kind = g.face_kind[face];
        if (kind == LB_WALL) any_stationary = true;
        if (first < 0) first = face;
      }
      double term = 0.0;
      if (valid && combo != 0 && !any_stationary && first >= 0) {
        double cu = 0.0;
        for (int ax = 0; ax < 3; ++ax) cu += c[ax] * g.wall_u[first][ax];
        term = 2.0 * weight<L>(a) * g.rho0 * cu * 3.0;
      }
      bb[a][combo] = R(term);
    }
  }
}

inline int div_up(int64_t a, int64_t b) { return static_cast<int>((a + b - 1) / b); }

}  // namespace lbgb
