// Sparse form: CSR SpMM G = A X fused with the PDBO epilogue, for graphs (Max-Cut, MIS).
//
// State is variable-major: element (i, r) at [i * ld + r], so the B restarts of one variable
// are contiguous.  One warp owns one row i of A and a chunk of 32*V restarts: lane l handles
// restarts rbase + l + 32 v (v < V), so every gather X[j][...] of a neighbour j is a run of
// 32 consecutive elements per v (one 128-byte line for FP32, 64 bytes for BF16).  Column
// indices and weights are warp-uniform loads.  Warps stride over rows; in EPI_EVAL each lane
// keeps per-restart int64 partial sums of 2F across its rows and adds them once at the end.
#include "sbo_internal.h"

namespace sbo {

enum ValType : int { VAL_F32 = 0, VAL_BF16 = 1, VAL_E4M3 = 2 };

__device__ __forceinline__ float load_val(const void* val, int64_t e, int vt) {
  if (vt == VAL_F32) return __ldg(static_cast<const float*>(val) + e);
  if (vt == VAL_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(val)[e]);
  __nv_fp8_e4m3 q;
  q.__x = static_cast<const __nv_fp8_storage_t*>(val)[e];
  return static_cast<float>(q);
}

template <int MODE, int V, int OPT>
__global__ void __launch_bounds__(256) k_csr(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                             const void* __restrict__ val, int vt, EpiArgs a) {
  const int lane = threadIdx.x & 31;
  const int warps_per_block = blockDim.x >> 5;
  const int64_t warp0 = (int64_t)blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * warps_per_block;
  const int64_t rbase = (int64_t)blockIdx.y * 32 * V;
  const int n = a.n, B = a.B;
  const int64_t ld = a.ld;
  const void* Xin = a.Xin;
  long long f2[V];
#pragma unroll
  for (int v = 0; v < V; ++v) f2[v] = 0;

  for (int64_t i = warp0; i < n; i += nwarps) {
    float acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.0f;
    const int e0 = rowptr[i], e1 = rowptr[i + 1];
    for (int e = e0; e < e1; ++e) {
      const int64_t j = __ldg(col + e);
      const float w = load_val(val, e, vt);
      const int64_t base = j * ld + rbase + lane;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        if (rbase + lane + 32 * v < B) {
          const float xv = OPT == OP_F32 ? __ldg(static_cast<const float*>(Xin) + base + 32 * v)
                                         : __bfloat162float(static_cast<const __nv_bfloat16*>(Xin)[base + 32 * v]);
          acc[v] = fmaf(w, xv, acc[v]);
        }
      }
    }
    const float cpi = a.cp[i];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int64_t r = rbase + lane + 32 * v;
      if (r >= B) continue;
      const int64_t idx = i * ld + r;
      if (MODE == EPI_UPDATE) {
        const float x = a.Xm ? a.Xm[idx] : static_cast<const float*>(Xin)[idx];
        const float y = a.Y[idx];
        const float d = acc[v] + cpi + y * (2.0f * x - 1.0f);
        float yn;
        const float xn = pdbo_update(x, y, d, a.alpha, a.beta, a.delta, a.grad_tol, &yn);
        if (a.Xm) a.Xm[idx] = xn;
        op_store(a.Xout, idx, xn, OPT);
        a.Y[idx] = yn;
        if (a.bits_out) op_store(a.bits_out, idx, xn > 0.5f ? 1.0f : 0.0f, OPT);
      } else if (MODE == EPI_EVAL) {
        const float b = op_load(Xin, idx, OPT);
        if (b != 0.0f) f2[v] += (long long)acc[v] + 2 * a.cp64[i];
      }
    }
  }
  if (MODE == EPI_EVAL) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int64_t r = rbase + lane + 32 * v;
      if (r < B && f2[v] != 0) atomicAdd(&a.F2[r], (unsigned long long)f2[v]);
    }
  }
}

template <int MODE, int OPT>
static cudaError_t launch_csr_v(const int32_t* rowptr, const int32_t* col, const void* val, int vt,
                                const EpiArgs& a, cudaStream_t s) {
  int V = 1;
  while (V < 8 && 32 * V < a.B) V *= 2;
  const int64_t chunks = (a.B + 32 * V - 1) / (32 * V);
  const int warps_per_block = 8;
  int64_t want = (a.n + warps_per_block - 1) / warps_per_block;
  const int64_t cap = (int64_t)152 * 16 / (chunks > 0 ? chunks : 1) + 1;  // EVAL: bound atomics
  if (MODE == EPI_EVAL && want > cap) want = cap;
  if (want > 65535 * 8) want = 65535 * 8;
  dim3 grid((unsigned)want, (unsigned)chunks);
  switch (V) {
    case 1: k_csr<MODE, 1, OPT><<<grid, 256, 0, s>>>(rowptr, col, val, vt, a); break;
    case 2: k_csr<MODE, 2, OPT><<<grid, 256, 0, s>>>(rowptr, col, val, vt, a); break;
    case 4: k_csr<MODE, 4, OPT><<<grid, 256, 0, s>>>(rowptr, col, val, vt, a); break;
    default: k_csr<MODE, 8, OPT><<<grid, 256, 0, s>>>(rowptr, col, val, vt, a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_csr(const int32_t* rowptr, const int32_t* col, const void* val, int val_type,
                       const EpiArgs& a, int op_type, int mode, cudaStream_t s) {
  if (mode == EPI_UPDATE) {
    return op_type == OP_F32 ? launch_csr_v<EPI_UPDATE, OP_F32>(rowptr, col, val, val_type, a, s)
                             : launch_csr_v<EPI_UPDATE, OP_BF16>(rowptr, col, val, val_type, a, s);
  }
  if (mode == EPI_EVAL) {
    return op_type == OP_F32 ? launch_csr_v<EPI_EVAL, OP_F32>(rowptr, col, val, val_type, a, s)
                             : launch_csr_v<EPI_EVAL, OP_BF16>(rowptr, col, val, val_type, a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sbo
