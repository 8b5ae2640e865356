// lb_k1_d2q9.cu -- compiled brick shapes of the fused step for D2Q9.
// Each entry: storage / arithmetic type, brick bx x by, TMA pipeline depth,
// window buffers, dedicated export warps.  For D2Q9 the paired shapes of
// lb_k2_d2q9.cu come first in the planner's order; these are alternatives
// (the narrow 64 x 1 brick serves small domains in batches).
#include "lb_k1_launch.cuh"

namespace lbgb {

extern const K1Variant k1_variants_d2q9[] = {
    K1Impl<D2Q9, float, float, 256,1,4,2,0>::variant(LB_D2Q9, LB_F32),
    K1Impl<D2Q9, float, float, 64,1,4,2,0,0,8>::variant(LB_D2Q9, LB_F32),   // narrow domains (batches), 8 CTAs / SM
    K1Impl<D2Q9, float, float, 64,1,4,2,0>::variant(LB_D2Q9, LB_F32),   // narrow domains (batches)
    K1Impl<D2Q9, double, double, 256,1,3,2,0>::variant(LB_D2Q9, LB_F64),
    K1Impl<D2Q9, __half, float, 256,1,4,2,0>::variant(LB_D2Q9, LB_F16S),
    K1Impl<D2Q9, __half, float, 64,1,4,2,0>::variant(LB_D2Q9, LB_F16S),
    K1Impl<D2Q9, __nv_bfloat16, float, 256,1,4,2,0>::variant(LB_D2Q9, LB_BF16S),
};
extern const int k1_n_variants_d2q9 = sizeof(k1_variants_d2q9) / sizeof(k1_variants_d2q9[0]);

}  // namespace lbgb
