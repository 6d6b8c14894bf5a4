// Best-candidate bookkeeping of the multi-start run (section 4.2: B restarts, best retained).
//
// After an evaluation kernel has accumulated 2F(b_r) for every restart r:
//   k_eval_compare   F_r = 2F/2; strict improvement of restart r's best keeps (F, t) and flags
//                    the restart, so equal values keep the earliest t
//   k_copy_best      copies the candidate bits of flagged restarts
//   k_eval_finalize  min_r F_r into the trace, clears the accumulators, advances t_last
// k_best_select returns the lexicographic minimum of (F, t, r) over the per-restart bests,
// which equals the minimum over every evaluation so far.
#include "sbo_internal.h"

namespace sbo {

__global__ void k_eval_compare(const unsigned long long* __restrict__ F2, long long* bestF, long long* bestT,
                               uint8_t* improved, long long* evalF, int B, const long long* t_last,
                               long long add) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B) return;
  const long long F = (long long)F2[r] / 2;
  const long long t = *t_last + add;
  evalF[r] = F;
  const bool better = F < bestF[r];
  if (better) {
    bestF[r] = F;
    bestT[r] = t;
  }
  improved[r] = better ? 1 : 0;
}

// 2-D grid: x runs along the contiguous dimension of the layout (4 elements per thread; ld is a
// multiple of 8 and `improved` is padded to a multiple of 8), y over the other dimension.
__device__ __forceinline__ float4 op_load4(const void* p, int64_t idx, int type) {
  if (type == OP_F32) return *reinterpret_cast<const float4*>(static_cast<const float*>(p) + idx);
  const uint2 raw = *reinterpret_cast<const uint2*>(static_cast<const __nv_bfloat16*>(p) + idx);
  const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
  const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
  return make_float4(__low2float(lo), __high2float(lo), __low2float(hi), __high2float(hi));
}

__global__ void k_copy_best(const void* __restrict__ bits, int op_type, uint8_t* bestBits,
                            const uint8_t* __restrict__ improved, int n, int B, int64_t ld, int layout) {
  const int64_t inner = layout == LAYOUT_RN ? n : B;
  const int64_t outer = layout == LAYOUT_RN ? B : n;
  for (int64_t o = blockIdx.y; o < outer; o += gridDim.y) {
    if (layout == LAYOUT_RN && !improved[o]) continue;   // whole restart row unchanged
    for (int64_t q = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); q < inner;
         q += 4 * (int64_t)gridDim.x * blockDim.x) {
      const int64_t idx = o * ld + q;
      const float4 v = op_load4(bits, idx, op_type);
      uchar4 nb = make_uchar4(v.x != 0.f, v.y != 0.f, v.z != 0.f, v.w != 0.f);
      if (layout == LAYOUT_NR) {
        const uchar4 imp = *reinterpret_cast<const uchar4*>(improved + q);
        const uchar4 old = *reinterpret_cast<const uchar4*>(bestBits + idx);
        nb.x = imp.x ? nb.x : old.x;
        nb.y = imp.y ? nb.y : old.y;
        nb.z = imp.z ? nb.z : old.z;
        nb.w = imp.w ? nb.w : old.w;
      }
      *reinterpret_cast<uchar4*>(bestBits + idx) = nb;   // padding columns stay consistent
    }
  }
}

__global__ void __launch_bounds__(1024) k_eval_finalize(unsigned long long* F2, const long long* __restrict__ evalF,
                                                        long long* trace, long long* n_evals, long long trace_cap,
                                                        int B, long long* t_last, long long add) {
  __shared__ long long red[32];
  long long m = LLONG_MAX;
  for (int r = threadIdx.x; r < B; r += blockDim.x) {
    m = min(m, evalF[r]);
    F2[r] = 0ull;
  }
  for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : LLONG_MAX;
    for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) {
      const long long e = *n_evals;
      if (e < trace_cap) trace[e] = m;
      *n_evals = e + 1;
      *t_last += add;
    }
  }
}

__global__ void __launch_bounds__(1024) k_best_select(const long long* __restrict__ bestF,
                                                      const long long* __restrict__ bestT, int B, long long* out3) {
  __shared__ long long sF[32], sT[32], sR[32];
  long long F = LLONG_MAX, T = LLONG_MAX, R = LLONG_MAX;
  for (int r = threadIdx.x; r < B; r += blockDim.x) {
    const long long f = bestF[r], t = bestT[r];
    if (t < 0) continue;
    if (f < F || (f == F && (t < T || (t == T && r < R)))) { F = f; T = t; R = r; }
  }
  auto better = [](long long f, long long t, long long r, long long F0, long long T0, long long R0) {
    return f < F0 || (f == F0 && (t < T0 || (t == T0 && r < R0)));
  };
  for (int o = 16; o > 0; o >>= 1) {
    const long long f = __shfl_xor_sync(0xffffffffu, F, o);
    const long long t = __shfl_xor_sync(0xffffffffu, T, o);
    const long long r = __shfl_xor_sync(0xffffffffu, R, o);
    if (better(f, t, r, F, T, R)) { F = f; T = t; R = r; }
  }
  if ((threadIdx.x & 31) == 0) { sF[threadIdx.x >> 5] = F; sT[threadIdx.x >> 5] = T; sR[threadIdx.x >> 5] = R; }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool have = threadIdx.x < (blockDim.x >> 5);
    F = have ? sF[threadIdx.x] : LLONG_MAX;
    T = have ? sT[threadIdx.x] : LLONG_MAX;
    R = have ? sR[threadIdx.x] : LLONG_MAX;
    for (int o = 16; o > 0; o >>= 1) {
      const long long f = __shfl_xor_sync(0xffffffffu, F, o);
      const long long t = __shfl_xor_sync(0xffffffffu, T, o);
      const long long r = __shfl_xor_sync(0xffffffffu, R, o);
      if (better(f, t, r, F, T, R)) { F = f; T = t; R = r; }
    }
    if (threadIdx.x == 0) { out3[0] = F; out3[1] = T; out3[2] = R; }
  }
}

cudaError_t launch_eval_compare(const unsigned long long* F2, long long* bestF, long long* bestT,
                                uint8_t* improved, long long* evalF, int B, long long* t_last, int64_t add,
                                cudaStream_t s) {
  k_eval_compare<<<(B + 255) / 256, 256, 0, s>>>(F2, bestF, bestT, improved, evalF, B, t_last, add);
  return cudaGetLastError();
}

cudaError_t launch_copy_best(const void* bits_op, int op_type, uint8_t* bestBits, const uint8_t* improved,
                             int n, int B, int64_t ld, int layout, cudaStream_t s) {
  const int64_t inner = layout == LAYOUT_RN ? n : B;
  const int64_t outer = layout == LAYOUT_RN ? B : n;
  const int64_t bx = (inner + 1023) / 1024;
  dim3 grid((unsigned)(bx < 64 ? bx : 64), (unsigned)(outer < 65535 ? outer : 65535));
  k_copy_best<<<grid, 256, 0, s>>>(bits_op, op_type, bestBits, improved, n, B, ld, layout);
  return cudaGetLastError();
}

cudaError_t launch_eval_finalize(unsigned long long* F2, const long long* evalF, long long* trace,
                                 long long* n_evals, int64_t trace_cap, int B, long long* t_last, int64_t add,
                                 cudaStream_t s) {
  k_eval_finalize<<<1, 1024, 0, s>>>(F2, evalF, trace, n_evals, trace_cap, B, t_last, add);
  return cudaGetLastError();
}

cudaError_t launch_best_select(const long long* bestF, const long long* bestT, int B, long long* out3,
                               cudaStream_t s) {
  k_best_select<<<1, 1024, 0, s>>>(bestF, bestT, B, out3);
  return cudaGetLastError();
}

}  // namespace sbo
