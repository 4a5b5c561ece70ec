// Generic engine, mode VJP (see engine.cuh).
#include "engine.cuh"

#define EMODE VJP
#define EFN(name) name##_vjp
#include "engine_mode.inc"
