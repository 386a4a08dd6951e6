// Compile-time n3 transforms for the further sizes, df64 instances (see zpass_fast_impl.cuh).
#include "zpass_fast_impl.cuh"

WDF_ZFAST_DEFINE(zpass_more, WDF_ZMORE_LIST)
WDF_ZFAST_INSTANTIATE(wdf::df64, zpass_more)
