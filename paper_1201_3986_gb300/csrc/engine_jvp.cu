// Generic engine, mode JVP (see engine.cuh).
#include "engine.cuh"

#define EMODE JVP
#define EFN(name) name##_jvp
#include "engine_mode.inc"
