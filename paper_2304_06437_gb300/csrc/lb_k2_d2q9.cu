// lb_k2_d2q9.cu -- compiled brick shapes of the paired (two nodes per thread,
// FP32x2 arithmetic) fused step for D2Q9.  Each entry: storage type, brick
// bx x by, TMA pipeline depth.  For D2Q9 these come first in the planner's
// order (the default), before the scalar shapes of lb_k1_d2q9.cu.
#include "lb_k2.cuh"

namespace lbgb {

extern const K1Variant k2_variants_d2q9[] = {
    K2Impl<D2Q9, float, 256, 1, 4>::variant(LB_D2Q9, LB_F32),
    K2Impl<D2Q9, __half, 256, 1, 4>::variant(LB_D2Q9, LB_F16S),
    K2Impl<D2Q9, __nv_bfloat16, 256, 1, 4>::variant(LB_D2Q9, LB_BF16S),
};
extern const int k2_n_variants_d2q9 = sizeof(k2_variants_d2q9) / sizeof(k2_variants_d2q9[0]);

}  // namespace lbgb
