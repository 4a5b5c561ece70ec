// Instantiations of the fused 2D evaluator in FP32.
#include "fused2d.cuh"

QDVM_FUSED2D_INSTANTIATE(f32, float, false)
