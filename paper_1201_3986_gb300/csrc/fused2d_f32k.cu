// Instantiations of the fused 2D evaluator in FP32 with compensated sums.
#include "fused2d.cuh"

QDVM_FUSED2D_INSTANTIATE(f32k, float, true)
