// Compile-time n3 transforms, df64 instances (see zpass_fast_impl.cuh).
#include "zpass_fast_impl.cuh"

WDF_ZFAST_INST(wdf::df64)
