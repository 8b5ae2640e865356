// lb_k1_d3q19.cu -- compiled brick shapes of the fused step for D3Q19.
// Each entry: storage / arithmetic type, brick bx x by, TMA pipeline depth,
// window buffers, dedicated export warps (negative: -n warps that pass the
// node warps' per-plane barrier; positive: decoupled through a staged ring).  The first entry of a storage type
// is the default; the others are alternatives the planner can be asked for
// (by brick shape, LB_FUSED_PIPELINE, the autotuner or a batch).
#include "lb_k1_launch.cuh"

namespace lbgb {

extern const K1Variant k1_variants_d3q19[] = {
    K1Impl<D3Q19, float, float, 64,8,3,2,0>::variant(LB_D3Q19, LB_F32),
    K1Impl<D3Q19, float, float, 32,16,3,2,0>::variant(LB_D3Q19, LB_F32),   // less shell traffic, equal rate
    K1Impl<D3Q19, float, float, 64,7,3,2,2>::variant(LB_D3Q19, LB_F32),    // + 2 decoupled export warps
    K1Impl<D3Q19, float, float, 64,6,3,2,4>::variant(LB_D3Q19, LB_F32),    // + 4 decoupled export warps
    K1Impl<D3Q19, float, float, 32,14,3,2,-2>::variant(LB_D3Q19, LB_F32),  // + 2 export warps in the barrier
    K1Impl<D3Q19, float, float, 64,8,2,2,0,1>::variant(LB_D3Q19, LB_F32),  // planes stored by TMA
    K1Impl<D3Q19, float, float, 32,8,2,2,0,0,2>::variant(LB_D3Q19, LB_F32),  // small domains (batches), 2 CTAs / SM
    K1Impl<D3Q19, float, float, 32,8,2,2,0>::variant(LB_D3Q19, LB_F32),  // small domains (batches)
    K1Impl<D3Q19, double, double, 32,8,2,2,0>::variant(LB_D3Q19, LB_F64),
    K1Impl<D3Q19, __half, float, 64,8,4,2,0>::variant(LB_D3Q19, LB_F16S),
    K1Impl<D3Q19, __half, float, 32,8,3,2,0>::variant(LB_D3Q19, LB_F16S),
    K1Impl<D3Q19, __half, float, 64,7,4,2,2>::variant(LB_D3Q19, LB_F16S),
    K1Impl<D3Q19, __half, float, 64,7,4,2,-2>::variant(LB_D3Q19, LB_F16S),  // + 2 export warps in the barrier
    K1Impl<D3Q19, __nv_bfloat16, float, 64,8,4,2,0>::variant(LB_D3Q19, LB_BF16S),
};
extern const int k1_n_variants_d3q19 = sizeof(k1_variants_d3q19) / sizeof(k1_variants_d3q19[0]);

}  // namespace lbgb
