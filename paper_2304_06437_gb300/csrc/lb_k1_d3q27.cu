// lb_k1_d3q27.cu -- compiled brick shapes of the fused step for D3Q27.
// Each entry: storage / arithmetic type, brick bx x by, TMA pipeline depth,
// window buffers, dedicated export warps (negative: -n warps that pass the
// node warps' per-plane barrier; positive: decoupled through a staged ring).  The first entry of a storage type
// is the default; the others are alternatives the planner can be asked for
// (by brick shape, LB_FUSED_PIPELINE, the autotuner or a batch).
#include "lb_k1_launch.cuh"

namespace lbgb {

extern const K1Variant k1_variants_d3q27[] = {
    // 14 node warps + 2 export warps in the barrier, 128 registers
    K1Impl<D3Q27, float, float, 32,14,2,2,-2>::variant(LB_D3Q27, LB_F32),
    K1Impl<D3Q27, float, float, 32,14,2,2,0>::variant(LB_D3Q27, LB_F32),  // node warps export
    K1Impl<D3Q27, float, float, 32,12,2,2,0>::variant(LB_D3Q27, LB_F32),
    K1Impl<D3Q27, float, float, 32,10,2,2,2>::variant(LB_D3Q27, LB_F32),  // + 2 decoupled export warps
    K1Impl<D3Q27, float, float, 32,10,3,2,0>::variant(LB_D3Q27, LB_F32),  // deeper TMA ring
    K1Impl<D3Q27, float, float, 32,8,3,2,0>::variant(LB_D3Q27, LB_F32),
    K1Impl<D3Q27, double, double, 32,4,2,2,0>::variant(LB_D3Q27, LB_F64),
    K1Impl<D3Q27, __half, float, 32,16,3,2,0>::variant(LB_D3Q27, LB_F16S),  // 16 warps at 128 registers
    K1Impl<D3Q27, __half, float, 32,12,3,2,0>::variant(LB_D3Q27, LB_F16S),
    K1Impl<D3Q27, __half, float, 32,10,3,2,2>::variant(LB_D3Q27, LB_F16S),
    K1Impl<D3Q27, __nv_bfloat16, float, 32,16,3,2,0>::variant(LB_D3Q27, LB_BF16S),
    K1Impl<D3Q27, __nv_bfloat16, float, 32,12,3,2,0>::variant(LB_D3Q27, LB_BF16S),
};
extern const int k1_n_variants_d3q27 = sizeof(k1_variants_d3q27) / sizeof(k1_variants_d3q27[0]);

}  // namespace lbgb
