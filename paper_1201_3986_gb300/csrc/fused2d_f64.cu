// Instantiations of the fused 2D evaluator in FP64.
#include "fused2d.cuh"

QDVM_FUSED2D_INSTANTIATE(f64, double, false)
