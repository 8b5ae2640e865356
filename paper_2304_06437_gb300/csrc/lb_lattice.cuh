// lb_lattice.cuh -- compile-time velocity sets for the CUDA path.
//
// The kernels work in "internal" 3D coordinates.  3D lattices use (x, y, z)
// directly.  D2Q9 is mapped onto the internal (x, z) plane with an internal y
// extent of 1, so that every kernel sweeps its slowest storage axis: for a 2D
// grid of nx x ny the internal grid is nx x 1 x ny and the 2D velocity
// (cx, cy) becomes (cx, 0, cy).  Storage index x + nx*(y + ny*z) is unchanged
// by this mapping.
//
// Velocity order is canonical (rest, then |c|^2, then lexicographic on the
// user-facing (cx, cy, cz) with -1 < 0 < 1), so population a of the ABI is
// population a of the kernels.  Weights: D2Q9 4/9, 1/9, 1/36; D3Q19 1/3,
// 1/18, 1/36; D3Q27 8/27, 2/27, 1/54, 1/216 (textbook values, cs^2 = 1/3,
// paper section 2).
#pragma once

#ifdef __CUDACC__
#define LB_HD __host__ __device__
#else
#define LB_HD
#endif

namespace lbgb {

struct D2Q9 {
  static constexpr int Q = 9;
  static constexpr int D = 2;
  static constexpr int ID = 0;
  // internal components; the 2D cy lives on the internal z axis
  LB_HD static constexpr int cx(int a) {
    constexpr int t[Q] = {0, -1, 0, 0, 1, -1, -1, 1, 1};
    return t[a];
  }
  LB_HD static constexpr int cy(int a) {
    constexpr int t[Q] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    return t[a];
  }
  LB_HD static constexpr int cz(int a) {
    constexpr int t[Q] = {0, 0, -1, 1, 0, -1, 1, -1, 1};
    return t[a];
  }
  LB_HD static constexpr int opp(int a) {
    constexpr int t[Q] = {0, 4, 3, 2, 1, 8, 7, 6, 5};
    return t[a];
  }
  LB_HD static constexpr int shell(int a) {
    constexpr int t[Q] = {0, 1, 1, 1, 1, 2, 2, 2, 2};
    return t[a];
  }
  // lattice axes (the internal y axis carries no velocities in 2D)
  LB_HD static constexpr bool axis(int k) { return k != 1; }
};

struct D3Q19 {
  static constexpr int Q = 19;
  static constexpr int D = 3;
  static constexpr int ID = 1;
  LB_HD static constexpr int cx(int a) {
    constexpr int t[Q] = {0, -1, 0, 0, 0, 0, 1, -1, -1, -1, -1, 0, 0, 0, 0, 1, 1, 1, 1};
    return t[a];
  }
  LB_HD static constexpr int cy(int a) {
    constexpr int t[Q] = {0, 0, -1, 0, 0, 1, 0, -1, 0, 0, 1, -1, -1, 1, 1, -1, 0, 0, 1};
    return t[a];
  }
  LB_HD static constexpr int cz(int a) {
    constexpr int t[Q] = {0, 0, 0, -1, 1, 0, 0, 0, -1, 1, 0, -1, 1, -1, 1, 0, -1, 1, 0};
    return t[a];
  }
  LB_HD static constexpr int opp(int a) {
    constexpr int t[Q] = {0, 6, 5, 4, 3, 2, 1, 18, 17, 16, 15, 14, 13, 12, 11, 10, 9, 8, 7};
    return t[a];
  }
  LB_HD static constexpr int shell(int a) {
    constexpr int t[Q] = {0, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2};
    return t[a];
  }
  LB_HD static constexpr bool axis(int) { return true; }
};

struct D3Q27 {
  static constexpr int Q = 27;
  static constexpr int D = 3;
  static constexpr int ID = 2;
  LB_HD static constexpr int cx(int a) {
    constexpr int t[Q] = {0, -1, 0, 0, 0, 0, 1, -1, -1, -1, -1, 0, 0, 0, 0, 1, 1, 1, 1,
                                -1, -1, -1, -1, 1, 1, 1, 1};
    return t[a];
  }
  LB_HD static constexpr int cy(int a) {
    constexpr int t[Q] = {0, 0, -1, 0, 0, 1, 0, -1, 0, 0, 1, -1, -1, 1, 1, -1, 0, 0, 1,
                                -1, -1, 1, 1, -1, -1, 1, 1};
    return t[a];
  }
  LB_HD static constexpr int cz(int a) {
    constexpr int t[Q] = {0, 0, 0, -1, 1, 0, 0, 0, -1, 1, 0, -1, 1, -1, 1, 0, -1, 1, 0,
                                -1, 1, -1, 1, -1, 1, -1, 1};
    return t[a];
  }
  LB_HD static constexpr int opp(int a) {
    constexpr int t[Q] = {0, 6, 5, 4, 3, 2, 1, 18, 17, 16, 15, 14, 13, 12, 11, 10, 9, 8, 7,
                                 26, 25, 24, 23, 22, 21, 20, 19};
    return t[a];
  }
  LB_HD static constexpr int shell(int a) {
    constexpr int t[Q] = {0, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2,
                                   3, 3, 3, 3, 3, 3, 3, 3};
    return t[a];
  }
  LB_HD static constexpr bool axis(int) { return true; }
};

// lattice weight of a shell, as an exact-as-possible double
template <class L>
LB_HD constexpr double weight_of_shell(int s) {
  return L::ID == 0   ? (s == 0 ? 4.0 / 9.0 : s == 1 ? 1.0 / 9.0 : 1.0 / 36.0)
         : L::ID == 1 ? (s == 0 ? 1.0 / 3.0 : s == 1 ? 1.0 / 18.0 : 1.0 / 36.0)
                      : (s == 0   ? 8.0 / 27.0
                         : s == 1 ? 2.0 / 27.0
                         : s == 2 ? 1.0 / 54.0
                                  : 1.0 / 216.0);
}

template <class L>
LB_HD constexpr double weight(int a) {
  return weight_of_shell<L>(L::shell(a));
}

// number of directions with component c along an axis (0 = x, 1 = y, 2 = z)
template <class L>
LB_HD constexpr int comp(int axis, int a) {
  return axis == 0 ? L::cx(a) : axis == 1 ? L::cy(a) : L::cz(a);
}

template <class L>
LB_HD constexpr int count_dirs(int axis, int sign) {
  int n = 0;
  for (int a = 0; a < L::Q; ++a) n += (comp<L>(axis, a) == sign) ? 1 : 0;
  return n;
}

// position of direction a among the directions whose component along axis is sign
template <class L>
LB_HD constexpr int sub_index(int axis, int sign, int a) {
  int n = 0;
  for (int b = 0; b < a; ++b) n += (comp<L>(axis, b) == sign) ? 1 : 0;
  return n;
}

}  // namespace lbgb
