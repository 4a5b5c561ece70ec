// Generic engine, mode FWD (see engine.cuh).
#include "engine.cuh"

#define EMODE FWD
#define EFN(name) name##_fwd
#include "engine_mode.inc"
