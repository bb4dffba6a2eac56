// dtypes.cuh -- reading stored (prepared) rows back as FP32.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace tpuknn {

__device__ __forceinline__ float e4m3_code_to_float(uint8_t c) {
  __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)c, __NV_E4M3);
  return __half2float(__half(h));
}

// Element d of stored row r (row pitch `pitch` elements) as FP32; E4M3
// elements are multiplied by the row's scale.
__device__ __forceinline__ float load_stored(const void* lp, int dtype, int64_t r, int pitch, int d,
                                             const float* scale) {
  if (dtype == KNN_F32) return reinterpret_cast<const float*>(lp)[r * pitch + d];
  if (dtype == KNN_BF16)
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(lp)[r * pitch + d]);
  return e4m3_code_to_float(reinterpret_cast<const uint8_t*>(lp)[r * pitch + d]) * scale[r];
}

}  // namespace tpuknn
