// FP64 product g = A x for one point x and an FP64 projected gradient step, used by the dual
// certificate (the paper's section on the dual certificate): with y = ybar large enough that
// L(., y) is convex on the box, any box point x gives the lower bound L(x) + min over the box of
// <grad L(x), z - x> on min F.  The point from the fast path (whose operand may be BF16) is
// polished by FP64 steps, and the bound is formed on the host in FP64 from g; A is exact in its
// storage type, so the only rounding left is FP64's.  One warp per row: dense rows are read with the lanes striding over the columns, sparse
// rows with the lanes striding over the row's entries; a warp-shuffle sum closes each row.
#include <algorithm>

#include "sbo_internal.h"

namespace sbo {
namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_matvec_dense_f64(const void* __restrict__ A, int a_type, int64_t lda, int n,
                                   const double* __restrict__ x, double* g) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = warp0; i < n; i += nw) {
    double acc = 0.0;
    for (int64_t j = lane; j < n; j += 32) {
      const float a = a_type == OP_F32 ? static_cast<const float*>(A)[i * lda + j]
                                       : __bfloat162float(static_cast<const __nv_bfloat16*>(A)[i * lda + j]);
      acc = fma((double)a, x[j], acc);
    }
    acc = warp_sum_d(acc);
    if (lane == 0) g[i] = acc;
  }
}

__global__ void k_matvec_csr_f64(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const void* __restrict__ val, int vt, int n, const double* __restrict__ x, double* g) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = warp0; i < n; i += nw) {
    double acc = 0.0;
    for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
      float w;
      if (vt == 0) {
        w = static_cast<const float*>(val)[e];
      } else if (vt == 1) {
        w = __bfloat162float(static_cast<const __nv_bfloat16*>(val)[e]);
      } else {
        __nv_fp8_e4m3 q;
        q.__x = static_cast<const __nv_fp8_storage_t*>(val)[e];
        w = static_cast<float>(q);
      }
      acc = fma((double)w, x[col[e]], acc);
    }
    acc = warp_sum_d(acc);
    if (lane == 0) g[i] = acc;
  }
}

// One FP64 projected gradient step on L(., ybar) given g = A x: x <- clip(x - alpha grad, 0, 1).
__global__ void k_pgd_step_f64(double* x, const double* __restrict__ g, const int64_t* __restrict__ cp, int n,
                               double ybar, double alpha) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double xi = x[i];
    const double grad = g[i] + (double)cp[i] + ybar * (2.0 * xi - 1.0);
    x[i] = fmin(1.0, fmax(0.0, xi - alpha * grad));
  }
}

}  // namespace

cudaError_t launch_pgd_step_f64(double* x, const double* g, const int64_t* cp, int n, double ybar, double alpha,
                                cudaStream_t s) {
  const unsigned blocks = (unsigned)std::min<int64_t>(((int64_t)n + 255) / 256, 152 * 8);
  k_pgd_step_f64<<<blocks, 256, 0, s>>>(x, g, cp, n, ybar, alpha);
  return cudaGetLastError();
}

cudaError_t launch_matvec_f64(const DenseView* dense, const int32_t* rowptr, const int32_t* col, const void* val,
                              int val_type, int n, const double* x, double* g, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::min<int64_t>(((int64_t)n + 7) / 8, 152 * 16);
  if (dense) {
    const int a_type = dense->prec == SBO_FP32 ? OP_F32 : OP_BF16;
    k_matvec_dense_f64<<<blocks, 256, 0, s>>>(dense->A, a_type, dense->lda, n, x, g);
  } else {
    k_matvec_csr_f64<<<blocks, 256, 0, s>>>(rowptr, col, val, val_type, n, x, g);
  }
  return cudaGetLastError();
}

}  // namespace sbo
