// lb_k2_d3q27.cu -- compiled brick shapes of the paired (two nodes per thread,
// FP32x2 arithmetic) fused step for D3Q27.  Each entry: storage type, brick
// bx x by, TMA pipeline depth.  Alternatives: the planner prefers the scalar
// shapes of lb_k1_d3q27.cu for D3Q27, which measure faster.
#include "lb_k2.cuh"

namespace lbgb {

extern const K1Variant k2_variants_d3q27[] = {
    K2Impl<D3Q27, float, 32, 12, 2>::variant(LB_D3Q27, LB_F32),
    K2Impl<D3Q27, float, 64, 6, 2>::variant(LB_D3Q27, LB_F32),
    K2Impl<D3Q27, __half, 32, 12, 3>::variant(LB_D3Q27, LB_F16S),
    K2Impl<D3Q27, __nv_bfloat16, 32, 12, 3>::variant(LB_D3Q27, LB_BF16S),
};
extern const int k2_n_variants_d3q27 = sizeof(k2_variants_d3q27) / sizeof(k2_variants_d3q27[0]);

}  // namespace lbgb
