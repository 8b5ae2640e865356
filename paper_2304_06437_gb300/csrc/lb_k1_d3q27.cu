// lb_k1_d3q27.cu -- compiled brick shapes of the fused step for D3Q27.
// Shapes: bx, by, pipeline depth; chosen so one CTA fills an SM's shared
// memory (TMA slots + collided window + halo) with 512 (3D) or 256 (2D) threads.
#include "lb_k1_launch.cuh"

namespace lbgb {

extern const K1Variant k1_variants_d3q27[] = {
    K1Impl<D3Q27, float, float, 32,12,3>::variant(LB_D3Q27, LB_F32),
    K1Impl<D3Q27, double, double, 32,8,2>::variant(LB_D3Q27, LB_F64),
    K1Impl<D3Q27, __half, float, 32,16,4>::variant(LB_D3Q27, LB_F16S),
    K1Impl<D3Q27, __nv_bfloat16, float, 32,16,4>::variant(LB_D3Q27, LB_BF16S),
};
extern const int k1_n_variants_d3q27 = sizeof(k1_variants_d3q27) / sizeof(k1_variants_d3q27[0]);

}  // namespace lbgb
