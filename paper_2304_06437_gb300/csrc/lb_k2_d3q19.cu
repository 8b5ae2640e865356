// lb_k2_d3q19.cu -- compiled brick shapes of the paired (two nodes per thread,
// FP32x2 arithmetic) fused step for D3Q19.  Each entry: storage type, brick
// bx x by, TMA pipeline depth.  Alternatives: the planner prefers the scalar
// shapes of lb_k1_d3q19.cu for D3Q19, which measure faster.
#include "lb_k2.cuh"

namespace lbgb {

extern const K1Variant k2_variants_d3q19[] = {
    K2Impl<D3Q19, float, 64, 8, 3>::variant(LB_D3Q19, LB_F32),
    K2Impl<D3Q19, __half, 64, 8, 4>::variant(LB_D3Q19, LB_F16S),
    K2Impl<D3Q19, __nv_bfloat16, 64, 8, 4>::variant(LB_D3Q19, LB_BF16S),
};
extern const int k2_n_variants_d3q19 = sizeof(k2_variants_d3q19) / sizeof(k2_variants_d3q19[0]);

}  // namespace lbgb
