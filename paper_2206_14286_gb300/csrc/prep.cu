// prep.cu -- row preparation for the contraction (database once, queries per
// call): optional cosine normalisation (Sec. 2), conversion to the stored
// element type (FP32 / BF16 / E4M3 with a per-row scale or with one scale for
// the whole database), half squared norms
// for L2 (App. A.2, Eq. 19), zero padding of each row to the row pitch.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "dtypes.cuh"
#include "kernels.h"

namespace tpuknn {

// A row as it is quantised: the row itself, or for COS the row scaled to
// unit length. The only order-dependent reduction that decides rounded codes,
// the cosine norm, is summed by lane 0 in index order in FP64, so y is
// defined bit for bit.
struct PrepRow {
  const float* xr;
  int D, metric;
  double inv;
  bool zero_row;
  __device__ float y(int d) const {
    if (d >= D) return 0.0f;
    if (metric != KNN_COS) return xr[d];
    if (zero_row) return 0.0f;
    return __double2float_rn(__dmul_rn((double)xr[d], inv));
  }
};

__device__ __forceinline__ PrepRow prep_row(const float* x, int64_t r, int D, int metric,
                                            int lane) {
  PrepRow p{x + r * (int64_t)D, D, metric, 1.0, false};
  if (metric == KNN_COS) {
    double n2 = 0.0;
    if (lane == 0) {
      for (int d = 0; d < D; ++d) {
        const double t = (double)p.xr[d];
        n2 = __dadd_rn(n2, __dmul_rn(t, t));
      }
    }
    n2 = __shfl_sync(0xffffffffu, n2, 0);
    if (n2 == 0.0) p.zero_row = true;
    else p.inv = __ddiv_rn(1.0, __dsqrt_rn(n2));
  }
  return p;
}

// The largest |y| over all rows (one warp per row), merged into *mx_bits as
// the bits of a non-negative float (their integer order is the float order).
__global__ void __launch_bounds__(256)
rows_absmax_kernel(const float* __restrict__ x, int64_t rows, int D, int metric,
                   unsigned* __restrict__ mx_bits) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= rows) return;
  const PrepRow p = prep_row(x, r, D, metric, lane);
  float mx = 0.0f;
  for (int d = lane; d < D; d += 32) mx = fmaxf(mx, fabsf(p.y(d)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0 && mx > 0.0f) atomicMax(mx_bits, __float_as_uint(mx));
}

__device__ __forceinline__ float e4m3_scale_of(float mx) {
  return mx > 0.0f ? __fdiv_rn(mx, 448.0f) : 1.0f;
}

__global__ void set_word_kernel(unsigned* p, unsigned v) { *p = v; }
// the database-wide scale into the first row's slot, from the maximum held there
__global__ void tensor_scale_kernel(float* scale) {
  scale[0] = e4m3_scale_of(__uint_as_float(*reinterpret_cast<const unsigned*>(scale)));
}

// One warp per row; lanes split the row. The E4M3 scale uses a maximum
// (order-free): the row's own (KNN_E4M3) or, when gmax_bits is given, the
// database-wide one (KNN_E4M3_T; then row 0's scale slot holds that maximum
// during this kernel and is written afterwards). The half norm (tolerance-
// level only) is a warp sum. If zero_buf is given, the CTAs also clear zero_n
// 32-bit words of it.
template <int DT>
__global__ void __launch_bounds__(256)
prep_rows_kernel(const float* __restrict__ x, int64_t rows, int D, int pitch, int metric,
                 void* __restrict__ out_lp, float* __restrict__ out_scale,
                 float* __restrict__ out_hnorm, float* __restrict__ out_f32,
                 uint32_t* __restrict__ zero_buf, int64_t zero_n,
                 const unsigned* __restrict__ gmax_bits) {
  // Launched behind whatever the stream ran before: wait for it (its output
  // may be these rows, or it may still read the buffers written here), then
  // let the contraction launch and run its prologue.
  pdl_wait();
  pdl_trigger();
  if (zero_buf) {
    // 16-byte stores where the buffer allows, then the odd words
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t done = 0;
    if ((reinterpret_cast<uintptr_t>(zero_buf) & 15) == 0) {
      const int64_t n4 = zero_n / 4;
      for (int64_t t = t0; t < n4; t += stride)
        reinterpret_cast<uint4*>(zero_buf)[t] = make_uint4(0u, 0u, 0u, 0u);
      done = n4 * 4;
    }
    for (int64_t t = done + t0; t < zero_n; t += stride) zero_buf[t] = 0u;
  }
  const int lane = threadIdx.x & 31;
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= rows) return;
  const PrepRow pr = prep_row(x, r, D, metric, lane);
  auto yval = [&](int d) -> float { return pr.y(d); };
  float s = 1.0f;
  if (DT == KNN_E4M3) {
    if (gmax_bits) {
      s = e4m3_scale_of(__uint_as_float(*gmax_bits));
      if (out_scale && lane == 0 && r > 0) out_scale[r] = s;
    } else {
      float mx = 0.0f;
      for (int d = lane; d < D; d += 32) mx = fmaxf(mx, fabsf(yval(d)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      s = e4m3_scale_of(mx);
      if (out_scale && lane == 0) out_scale[r] = s;
    }
  }
  double h2 = 0.0;
  for (int d = lane; d < pitch; d += 32) {
    const float y = yval(d);
    float stored;
    if (DT == KNN_F32) {
      reinterpret_cast<float*>(out_lp)[r * pitch + d] = y;
      stored = y;
    } else if (DT == KNN_BF16) {
      const __nv_bfloat16 b = __float2bfloat16_rn(y);
      reinterpret_cast<__nv_bfloat16*>(out_lp)[r * pitch + d] = b;
      stored = __bfloat162float(b);
    } else {
      const __nv_fp8_storage_t c =
          __nv_cvt_float_to_fp8(__fdiv_rn(y, s), __NV_SATFINITE, __NV_E4M3);
      reinterpret_cast<uint8_t*>(out_lp)[r * pitch + d] = (uint8_t)c;
      stored = e4m3_code_to_float((uint8_t)c) * s;
    }
    h2 += (double)stored * (double)stored;
    if (out_f32 && d < D) out_f32[r * (int64_t)D + d] = y;
  }
  if (out_hnorm) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h2 += __shfl_xor_sync(0xffffffffu, h2, o);
    if (lane == 0) out_hnorm[r] = (float)(0.5 * h2);
  }
}

cudaError_t launch_prep(const float* x, int64_t rows, int D, int pitch, int metric, int dtype,
                        void* out_lp, float* out_scale, float* out_hnorm, float* out_f32,
                        cudaStream_t st, uint32_t* zero_buf, int64_t zero_n) {
  if (rows <= 0 && zero_n <= 0) return cudaSuccess;
  const int threads = 256;
  int64_t blocks = cdiv(rows * 32, threads);
  if (zero_buf && blocks < 64) blocks = 64;
  if (blocks < 1) blocks = 1;
  float* h = metric == KNN_L2 ? out_hnorm : nullptr;
  float* f = metric == KNN_COS ? out_f32 : nullptr;
  switch (dtype) {
    case KNN_F32:
      return launch_pdl(prep_rows_kernel<KNN_F32>, dim3((unsigned)blocks), dim3(threads), 0, st, x,
                        rows, D, pitch, metric, out_lp, (float*)nullptr, h, f, zero_buf, zero_n,
                        (const unsigned*)nullptr);
    case KNN_BF16:
      return launch_pdl(prep_rows_kernel<KNN_BF16>, dim3((unsigned)blocks), dim3(threads), 0, st, x,
                        rows, D, pitch, metric, out_lp, (float*)nullptr, h, f, zero_buf, zero_n,
                        (const unsigned*)nullptr);
    case KNN_E4M3_T: {
      // the database-wide maximum, accumulated in row 0's scale slot
      if (rows <= 0 || !out_scale) return cudaErrorInvalidValue;
      unsigned* mx = reinterpret_cast<unsigned*>(out_scale);
      set_word_kernel<<<1, 1, 0, st>>>(mx, 0u);
      cudaError_t e = launch_pdl(rows_absmax_kernel, dim3((unsigned)cdiv(rows * 32, threads)),
                                 dim3(threads), 0, st, x, rows, D, metric, mx);
      if (e != cudaSuccess) return e;
      e = launch_pdl(prep_rows_kernel<KNN_E4M3>, dim3((unsigned)blocks), dim3(threads), 0, st, x,
                     rows, D, pitch, metric, out_lp, out_scale, h, f, zero_buf, zero_n,
                     (const unsigned*)mx);
      if (e != cudaSuccess) return e;
      tensor_scale_kernel<<<1, 1, 0, st>>>(out_scale);
      return cudaGetLastError();
    }
    default:
      return launch_pdl(prep_rows_kernel<KNN_E4M3>, dim3((unsigned)blocks), dim3(threads), 0, st, x,
                        rows, D, pitch, metric, out_lp, out_scale, h, f, zero_buf, zero_n,
                        (const unsigned*)nullptr);
  }
}

}  // namespace tpuknn
