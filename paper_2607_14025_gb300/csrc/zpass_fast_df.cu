// Compile-time n3 transforms for the common sizes, df64 instances (see zpass_fast_impl.cuh).
#include "zpass_fast_impl.cuh"

WDF_ZFAST_DEFINE(zpass_fast, WDF_ZFAST_LIST)
WDF_ZFAST_INSTANTIATE(wdf::df64, zpass_fast)
