// Compile-time n3 transforms, float instances (see zpass_fast_impl.cuh).
#include "zpass_fast_impl.cuh"

WDF_ZFAST_INST(float)
