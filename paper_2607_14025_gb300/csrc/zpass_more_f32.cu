// Compile-time n3 transforms for the further sizes, float instances (see zpass_fast_impl.cuh).
#include "zpass_fast_impl.cuh"

WDF_ZFAST_DEFINE(zpass_more, WDF_ZMORE_LIST)
WDF_ZFAST_INSTANTIATE(float, zpass_more)
