// Compile-time n3 transforms for the common sizes, float instances (see zpass_fast_impl.cuh).
#include "zpass_fast_impl.cuh"

WDF_ZFAST_DEFINE(zpass_fast, WDF_ZFAST_LIST)
WDF_ZFAST_INSTANTIATE(float, zpass_fast)
