// prep.cu -- row preparation for the contraction (database once, queries per
// call): optional cosine normalisation (Sec. 2), conversion to the stored
// element type (FP32 / BF16 / E4M3 with a per-row scale), half squared norms
// for L2 (App. A.2, Eq. 19), zero padding of each row to the row pitch.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "dtypes.cuh"
#include "kernels.h"

namespace tpuknn {

// One thread per row: the row-wise reductions that decide a rounded code
// (the E4M3 scale, the cosine norm) run sequentially in index order so that
// the result is defined bit for bit.
template <int DT>
__global__ void prep_rows_kernel(const float* __restrict__ x, int64_t rows, int D, int pitch,
                                 int metric, void* __restrict__ out_lp,
                                 float* __restrict__ out_scale, float* __restrict__ out_hnorm,
                                 float* __restrict__ out_f32) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const float* xr = x + r * (int64_t)D;
  double inv = 1.0;
  bool zero_row = false;
  if (metric == KNN_COS) {
    double n2 = 0.0;
    for (int d = 0; d < D; ++d) {
      double t = (double)xr[d];
      n2 = __dadd_rn(n2, __dmul_rn(t, t));
    }
    if (n2 == 0.0) zero_row = true;
    else inv = __ddiv_rn(1.0, __dsqrt_rn(n2));
  }
  auto yval = [&](int d) -> float {
    if (metric != KNN_COS) return xr[d];
    if (zero_row) return 0.0f;
    return __double2float_rn(__dmul_rn((double)xr[d], inv));
  };
  float s = 1.0f;
  if (DT == KNN_E4M3) {
    float mx = 0.0f;
    for (int d = 0; d < D; ++d) mx = fmaxf(mx, fabsf(yval(d)));
    s = mx > 0.0f ? __fdiv_rn(mx, 448.0f) : 1.0f;
    if (out_scale) out_scale[r] = s;
  }
  double h2 = 0.0;
  for (int d = 0; d < pitch; ++d) {
    float y = d < D ? yval(d) : 0.0f;
    float stored;
    if (DT == KNN_F32) {
      reinterpret_cast<float*>(out_lp)[r * pitch + d] = y;
      stored = y;
    } else if (DT == KNN_BF16) {
      __nv_bfloat16 b = __float2bfloat16_rn(y);
      reinterpret_cast<__nv_bfloat16*>(out_lp)[r * pitch + d] = b;
      stored = __bfloat162float(b);
    } else {
      __nv_fp8_storage_t c = __nv_cvt_float_to_fp8(__fdiv_rn(y, s), __NV_SATFINITE, __NV_E4M3);
      reinterpret_cast<uint8_t*>(out_lp)[r * pitch + d] = (uint8_t)c;
      stored = e4m3_code_to_float((uint8_t)c) * s;
    }
    h2 += (double)stored * (double)stored;
    if (out_f32 && d < D) out_f32[r * (int64_t)D + d] = y;
  }
  if (out_hnorm) out_hnorm[r] = (float)(0.5 * h2);
}

cudaError_t launch_prep(const float* x, int64_t rows, int D, int pitch, int metric, int dtype,
                        void* out_lp, float* out_scale, float* out_hnorm, float* out_f32,
                        cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  int threads = 128;
  unsigned blocks = (unsigned)cdiv(rows, threads);
  float* h = metric == KNN_L2 ? out_hnorm : nullptr;
  float* f = metric == KNN_COS ? out_f32 : nullptr;
  switch (dtype) {
    case KNN_F32:
      prep_rows_kernel<KNN_F32><<<blocks, threads, 0, st>>>(x, rows, D, pitch, metric, out_lp,
                                                            nullptr, h, f);
      break;
    case KNN_BF16:
      prep_rows_kernel<KNN_BF16><<<blocks, threads, 0, st>>>(x, rows, D, pitch, metric, out_lp,
                                                             nullptr, h, f);
      break;
    default:
      prep_rows_kernel<KNN_E4M3><<<blocks, threads, 0, st>>>(x, rows, D, pitch, metric, out_lp,
                                                             out_scale, h, f);
      break;
  }
  return cudaGetLastError();
}

}  // namespace tpuknn
