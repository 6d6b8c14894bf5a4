// Tiny-n form (n <= 64): the whole run -- every iteration of Algorithm 1, the rounding, the
// exact objective and the best tracking -- in one launch, with A and the iterates of a group
// of restarts held in shared memory.  One thread owns one (restart, coordinate) pair.
// FP32 arithmetic; state restart-major ([r * ld + i]).
#include <algorithm>

#include "sbo_internal.h"

namespace sbo {

constexpr int TINY_MAX_N = 64;

__global__ void __launch_bounds__(1024) k_tiny(TinyArgs a) {
  __shared__ float As[TINY_MAX_N * TINY_MAX_N];
  __shared__ float cps[TINY_MAX_N];
  __shared__ long long cp64s[TINY_MAX_N];
  extern __shared__ float dyn[];           // xs[RB][n], bs[RB][n]
  __shared__ unsigned long long f2s[1024 / 1];
  const int n = a.n;
  const int RB = max(1, 1024 / n);         // restarts per block
  const int r0 = blockIdx.x * RB;
  const int nrb = min(RB, a.B - r0);
  const int e = threadIdx.x;
  const bool active = e < nrb * n;
  const int rr = active ? e / n : 0, i = active ? e % n : 0;
  const int64_t r = r0 + rr;
  float* xs = dyn;
  float* bs = dyn + RB * n;

  for (int k = threadIdx.x; k < n * n; k += blockDim.x) As[k] = a.A[(int64_t)(k / n) * a.lda + (k % n)];
  for (int k = threadIdx.x; k < n; k += blockDim.x) { cps[k] = a.cp[k]; cp64s[k] = a.cp64[k]; }
  float x = 0.f, y = 0.f;
  if (active) {
    x = a.X[r * a.ld + i];
    y = a.Y[r * a.ld + i];
    xs[rr * n + i] = x;
  }
  __syncthreads();

  int64_t e_idx = a.e0;
  for (int64_t s = 1; s <= a.steps; ++s) {
    const int64_t t = a.t0 + s;
    float xn = x, yn = y;
    if (active) {
      float g = 0.f;
      const float* xr = xs + rr * n;
      const float* Ai = As + i * n;
      for (int k = 0; k < n; ++k) g = fmaf(Ai[k], xr[k], g);
      const float d = g + cps[i] + y * g_der(x, a.gkind);
      xn = pdbo_update(x, y, d, g_val(x, a.gkind), a.alpha, a.beta, a.delta, a.grad_tol, &yn);
      if (a.G) a.G[r * a.ld + i] = d;
    }
    __syncthreads();
    if (active) xs[rr * n + i] = xn;
    x = xn;
    y = yn;
    const bool is_eval = (t % a.K == 0) || (t == a.T);
    if (is_eval) {
      const float b = x > 0.5f ? 1.0f : 0.0f;
      if (active) bs[rr * n + i] = b;
      if (threadIdx.x < RB) f2s[threadIdx.x] = 0ull;
      __syncthreads();
      if (active && b != 0.f) {
        float g = 0.f;
        const float* br = bs + rr * n;
        const float* Ai = As + i * n;
        for (int k = 0; k < n; ++k) g = fmaf(Ai[k], br[k], g);
        atomicAdd(&f2s[rr], (unsigned long long)((long long)g + 2 * cp64s[i]));
      }
      __syncthreads();
      const long long F = (long long)f2s[rr] / 2;
      const bool improved = F < a.bestF[r];
      __syncthreads();
      if (active) {
        if (improved) a.bestBits[r * a.ld + i] = (uint8_t)(b != 0.f);
        if (i == 0) {
          if (improved) { a.bestF[r] = F; a.bestT[r] = t; }
          if (e_idx < a.trace_cap) atomicMin(&a.trace[e_idx], F);
        }
      }
      ++e_idx;
      __syncthreads();
    }
  }
  if (active) {
    a.X[r * a.ld + i] = x;
    a.Y[r * a.ld + i] = y;
  }
}

cudaError_t launch_tiny(const TinyArgs& a, cudaStream_t s) {
  if (a.n > TINY_MAX_N || a.n < 1) return cudaErrorInvalidValue;
  const int RB = std::max(1, 1024 / a.n);
  const int blocks = (a.B + RB - 1) / RB;
  const int threads = ((std::min(RB, a.B) * a.n + 31) / 32) * 32;
  const size_t dyn = sizeof(float) * 2 * RB * a.n;
  k_tiny<<<blocks, threads, dyn, s>>>(a);
  return cudaGetLastError();
}

}  // namespace sbo
