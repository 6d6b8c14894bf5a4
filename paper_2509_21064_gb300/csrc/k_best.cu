// Best-candidate bookkeeping of the multi-start run (section 4.2: B restarts, best retained).
//
// After an evaluation kernel has accumulated 2F(b_r) for every restart r, k_eval_commit (one
// launch) keeps the bits, F and t of every restart whose F strictly improves on its best, so equal
// values keep the earliest t, appends min_r F_r to the trace, clears the accumulators and advances
// t_last.  k_best_select returns the lexicographic minimum of (F, t, r) over the per-restart bests,
// which equals the minimum over every evaluation so far.
#include <algorithm>
#include <cstring>

#include "sbo_internal.h"

namespace sbo {

__device__ __forceinline__ float4 op_load4(const void* p, int64_t idx, int type) {
  if (type == OP_F32) return *reinterpret_cast<const float4*>(static_cast<const float*>(p) + idx);
  if (type == OP_U8) {
    const uchar4 b = *reinterpret_cast<const uchar4*>(static_cast<const uint8_t*>(p) + idx);
    return make_float4((float)b.x, (float)b.y, (float)b.z, (float)b.w);
  }
  const uint2 raw = *reinterpret_cast<const uint2*>(static_cast<const __nv_bfloat16*>(p) + idx);
  const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
  const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
  return make_float4(__low2float(lo), __high2float(lo), __low2float(hi), __high2float(hi));
}

__device__ __forceinline__ bool improves(const CommitArgs& a, int64_t r) {
  return r < a.B && (long long)a.F2[r] / 2 < a.bestF[r];
}

// One launch per evaluation (per group member along z).  Every block copies the candidate bits of
// the restarts that improve on their best, deciding from F2 and the best records as they were
// before this evaluation (nothing writes them until every block is done).  The last block to
// finish (arrival counter, no waiting) then commits: F_r = 2F/2 into evalF, strict improvements
// into (bestF, bestT) so that equal values keep the earliest t, min_r F_r into the trace, F2 back
// to zero, t_last advanced, counter back to zero.
//
// Threads: `tpr` (a power of two) consecutive threads cover 4·tpr consecutive elements of the
// contiguous dimension (restarts in the variable-major layout, variables in the restart-major
// one); a block covers 256 / tpr lines of the other dimension at a time.
__global__ void __launch_bounds__(256) k_eval_commit(CommitArgs one, const CommitArgs* __restrict__ tab, int tpr,
                                                     long long add) {
  const CommitArgs& a = tab ? tab[blockIdx.z] : one;
  const bool rn = a.layout == LAYOUT_RN;
  const int64_t inner = rn ? a.n : a.B;
  const int64_t outer = rn ? a.B : a.n;
  const int64_t V = (inner + 3) / 4;
  const int lq = threadIdx.x & (tpr - 1);
  const int lr = threadIdx.x / tpr;
  const int rpb = blockDim.x / tpr;
  if (rn) {
    for (int64_t o = (int64_t)blockIdx.y * rpb + lr; o < outer; o += (int64_t)gridDim.y * rpb) {
      if (!improves(a, o)) continue;   // whole restart row unchanged
      for (int64_t qv = (int64_t)blockIdx.x * tpr + lq; qv < V; qv += (int64_t)gridDim.x * tpr) {
        const int64_t idx = o * a.ld + 4 * qv;
        const float4 v = op_load4(a.bits, idx, a.op_type);
        *reinterpret_cast<uchar4*>(a.bestBits + idx) =
            make_uchar4((unsigned char)v.x, (unsigned char)v.y, (unsigned char)v.z, (unsigned char)v.w);
      }
    }
  } else {
    for (int64_t qv = (int64_t)blockIdx.x * tpr + lq; qv < V; qv += (int64_t)gridDim.x * tpr) {
      const int64_t q = 4 * qv;
      const bool i0 = improves(a, q), i1 = improves(a, q + 1), i2 = improves(a, q + 2), i3 = improves(a, q + 3);
      if (!(i0 || i1 || i2 || i3)) continue;
      // four lines per pass, their loads issued before any store; the old best bits are read only
      // where some of the four restarts keep theirs (padding restarts keep theirs too)
      const bool all4 = i0 && i1 && i2 && i3;
      const int64_t step = (int64_t)gridDim.y * rpb;
      for (int64_t o0 = (int64_t)blockIdx.y * rpb + lr; o0 < outer; o0 += 4 * step) {
        float4 v[4];
        uchar4 nb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t o = o0 + u * step;
          if (o < outer) {
            v[u] = op_load4(a.bits, o * a.ld + q, a.op_type);
            if (!all4) nb[u] = *reinterpret_cast<const uchar4*>(a.bestBits + o * a.ld + q);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t o = o0 + u * step;
          if (o >= outer) continue;
          if (all4) nb[u] = make_uchar4(0, 0, 0, 0);
          if (i0) nb[u].x = (unsigned char)v[u].x;   // 0/1 bits, or the part index of Max-k-Cut
          if (i1) nb[u].y = (unsigned char)v[u].y;
          if (i2) nb[u].z = (unsigned char)v[u].z;
          if (i3) nb[u].w = (unsigned char)v[u].w;
          *reinterpret_cast<uchar4*>(a.bestBits + o * a.ld + q) = nb[u];
        }
      }
    }
  }
  // last-block-done: the block that completes the count commits the evaluation
  __shared__ int s_last;
  __shared__ long long red[8];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(a.ctr, 1u) == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const long long t = *a.t_last + add;
  long long m = LLONG_MAX;
  for (int r = threadIdx.x; r < a.B; r += blockDim.x) {
    const long long F = (long long)a.F2[r] / 2;
    a.evalF[r] = F;
    if (F < a.bestF[r]) {
      a.bestF[r] = F;
      a.bestT[r] = t;
    }
    a.F2[r] = 0ull;
    m = min(m, F);
  }
  for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = min(m, red[w]);
    m = min(m, red[0]);
    const long long e = *a.n_evals;
    if (e < a.trace_cap) a.trace[e] = m;
    *a.n_evals = e + 1;
    *a.t_last = t;
    *a.ctr = 0u;
  }
}

// Dual step of the single-constraint form (one dual per restart): mu_r += beta * sum_k
// gpart[k][r], the rows of partial sums of g(x^t) written by the update kernel.  A block covers 32
// restarts (lane = restart); warp w adds rows w, w + 32, ... (eight loads in flight, added in row
// order); the 32 warp sums are then added in warp order, so the result does not depend on
// scheduling.
__global__ void __launch_bounds__(1024) k_dual_single(float* mu, const float* __restrict__ gpart, int P, int64_t ldg,
                                                      int B, float beta) {
  __shared__ float part[32][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = blockIdx.x * 32 + lane;
  float sum = 0.0f;
  if (r < B) {
    int k = w;
    for (; k + 7 * 32 < P; k += 8 * 32) {
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = gpart[(int64_t)(k + 32 * q) * ldg + r];
#pragma unroll
      for (int q = 0; q < 8; ++q) sum += v[q];
    }
    for (; k < P; k += 32) sum += gpart[(int64_t)k * ldg + r];
  }
  part[w][lane] = sum;
  __syncthreads();
  if (w == 0 && r < B) {
    float tot = 0.0f;
#pragma unroll 8
    for (int q = 0; q < 32; ++q) tot += part[q][lane];
    mu[r] += beta * tot;
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

// Grid of the commit kernel: the contiguous dimension in runs of 4·tpr elements (tpr the smallest
// power of two >= its 4-vectors, at most 256), about four blocks per SM in all (one per SM measured
// slower: the copies of the evaluations where many restarts improve lose memory parallelism --
// 45 -> 128 us per commit at n = 20,000, B = 1,024 -- more than the arrival counter gains).
static void commit_grid(int64_t inner, int64_t outer, int& tpr, dim3& grid) {
  const int64_t V = (inner + 3) / 4;
  tpr = 1;
  while (tpr < 256 && tpr < V) tpr *= 2;
  const int rpb = 256 / tpr;
  int64_t bx = (V + tpr - 1) / tpr;
  if (bx > 64) bx = 64;
  int64_t by = (outer + rpb - 1) / rpb;
  const int64_t cap = std::max<int64_t>(1, 608 / bx);
  if (by > cap) by = cap;
  if (by > 65535) by = 65535;
  grid = dim3((unsigned)bx, (unsigned)std::max<int64_t>(by, 1));
}

cudaError_t launch_eval_commit(const CommitArgs& a, int64_t add, cudaStream_t s) {
  int tpr;
  dim3 grid;
  commit_grid(a.layout == LAYOUT_RN ? a.n : a.B, a.layout == LAYOUT_RN ? a.B : a.n, tpr, grid);
  k_eval_commit<<<grid, 256, 0, s>>>(a, nullptr, tpr, (long long)add);
  return cudaGetLastError();
}

cudaError_t launch_eval_commit_group(const CommitArgs* d_tab, int members, int64_t max_inner, int64_t max_outer,
                                     int64_t add, cudaStream_t s) {
  int tpr;
  dim3 grid;
  commit_grid(max_inner, max_outer, tpr, grid);
  grid.z = (unsigned)members;
  CommitArgs none;
  std::memset(&none, 0, sizeof(none));
  k_eval_commit<<<grid, 256, 0, s>>>(none, d_tab, tpr, (long long)add);
  return cudaGetLastError();
}

cudaError_t launch_dual_single(float* mu, const float* gpart, int P, int64_t ldg, int B, float beta, cudaStream_t s) {
  k_dual_single<<<(B + 31) / 32, 1024, 0, s>>>(mu, gpart, P, ldg, B, beta);
  return cudaGetLastError();
}

cudaError_t launch_best_select(const long long* bestF, const long long* bestT, int B, long long* out3,
                               cudaStream_t s) {
  k_best_select<<<1, 1024, 0, s>>>(bestF, bestT, B, out3);
  return cudaGetLastError();
}

}  // namespace sbo
