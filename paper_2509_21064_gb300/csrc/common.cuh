// Shared device-side definitions of libsbo (GB300, sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

namespace sbo {

// Device error word bits (written with atomicOr, read and cleared by sbo_sync).
enum : uint32_t { ERR_TIMEOUT = 1u, ERR_BOUNDS = 2u };

// Constraint function g of the Lagrangian (section 3.1): the quadratic x^2 - x (the default) or
// the entropy x log x + (1 - x) log(1 - x) named among the paper's choices.
enum GKind : int { G_QUAD = 0, G_ENTROPY = 1 };
// The entropy's derivative log(x / (1 - x)) is unbounded at 0 and 1: it is taken at x clamped to
// [G_ENT_EPS, 1 - G_ENT_EPS] (g itself is continuous there, with g(0) = g(1) = 0).
constexpr float G_ENT_EPS = 1e-6f;

// Epilogue modes shared by the contraction kernels.
enum EpiMode : int { EPI_UPDATE = 0, EPI_EVAL = 1, EPI_LAGR = 2 };

// Operand element types of the contraction.
// OP_U8: 0/1 candidate bytes (the sparse path's candidates; never a contraction operand of the
// tensor cores).
enum OpType : int { OP_F32 = 0, OP_BF16 = 1, OP_U8 = 2 };

// Arguments of the fused GDA / evaluation / Lagrangian epilogue.  Every state array is
// addressed as [r * ld + i] (dense, restart-major) or [i * ld + r] (CSR, variable-major);
// the kernels document which.
struct EpiArgs {
  int n, B;
  int64_t ld;              // leading dimension of every state array (elements)
  float alpha, beta, delta, grad_tol;
  const float* cp;         // c' (FP32) [n]
  const int64_t* cp64;     // c' (exact) [n]  (EPI_EVAL)
  float* Xm;               // FP32 master x, updated in place; null when the operand is FP32
  float* Y;                // y, updated in place
  const void* Xin;         // contraction operand x^t (FP32 or BF16), read by every tile
  void* Xout;              // operand x^{t+1} (ping-pong partner of Xin)
  void* bits_out;          // if non-null: b = [x^{t+1} > 1/2] in the operand type (bytes for the sparse kernel)
  unsigned long long* F2;  // EPI_EVAL: 2F(b) accumulators per restart (two's complement)
  const float* Xl;         // EPI_LAGR: x (FP32)
  const float* Yl;         // EPI_LAGR: y (FP32)
  float* L;                // EPI_LAGR: value per restart (accumulated with atomics), may be null
  float* GX;               // EPI_LAGR: dL/dx, may be null
  float* GY;               // EPI_LAGR: dL/dy, may be null
  const float* gout;       // EPI_LAGR: per-restart scale of GX, GY (upstream gradient), may be null
  uint32_t* err;           // device error word
  // Single-constraint variant (PDBO-s): one dual per restart instead of y.  When mu is non-null
  // the update reads mu[r] in place of y, leaves Y alone and writes partial sums of g(x^t) over
  // its rows into gpart[row of partials][r] (row stride gpart_ld); a separate kernel then sums
  // the rows in order and takes the dual step.
  const float* mu;
  float* gpart;
  int64_t gpart_ld;
  int gkind;               // constraint function g (GKind)
  // EPI_UPDATE: when non-null, the gradient d = dL/dx at (x^t, y^t) that the step used, written at
  // the state index of every element (the loop's own gradient, kept for parity checks)
  float* Gd;
};

__device__ __forceinline__ float g_val(float x, int kind) {
  if (kind == G_QUAD) return x * x - x;
  const float a = x > 0.0f ? x * logf(x) : 0.0f;
  const float b = x < 1.0f ? (1.0f - x) * log1pf(-x) : 0.0f;
  return a + b;
}
// log(x / (1 - x)) at x clamped to [eps, 1 - eps], formed from u = min(x, 1 - x) clamped to
// [eps, 1/2] (1 - x is exact in FP32 for x >= 1/2, so the clamp near 1 loses nothing to 1 - eps
// being unrepresentable) and g'(x) = -g'(1 - x).
__device__ __forceinline__ float g_der(float x, int kind) {
  if (kind == G_QUAD) return 2.0f * x - 1.0f;
  const bool upper = x > 0.5f;
  const float u = fmaxf(upper ? 1.0f - x : x, G_ENT_EPS);
  const float v = logf(u) - log1pf(-u);
  return upper ? -v : v;
}

// Sum of v[j] over the 32 lanes of a warp for each j = 0..31 at once (31 shuffles): lane l
// returns the sum of v[l].  Step k halves the values a lane holds: the lane keeps the half
// selected by bit (4-k) of its lane id and adds its partner's copy of that half.
__device__ __forceinline__ float warp_transpose_sum32(float (&v)[32], int lane) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int half = 16 >> k;
    const bool upper = (lane & half) != 0;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const float keep = upper ? v[j + half] : v[j];
      const float send = upper ? v[j] : v[j + half];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, half);
    }
  }
  return v[0];
}

__device__ __forceinline__ float op_load(const void* p, int64_t idx, int type) {
  if (type == OP_F32) return static_cast<const float*>(p)[idx];
  if (type == OP_U8) return (float)static_cast<const uint8_t*>(p)[idx];
  return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[idx]);
}
__device__ __forceinline__ void op_store(void* p, int64_t idx, float v, int type) {
  if (type == OP_F32) static_cast<float*>(p)[idx] = v;
  else if (type == OP_U8) static_cast<uint8_t*>(p)[idx] = (uint8_t)v;
  else static_cast<__nv_bfloat16*>(p)[idx] = __float2bfloat16_rn(v);
}

// One coordinate of Algorithm 1.  d is dL/dx at (x, y) and gx = g(x); returns x^{t+1}, writes
// y^{t+1} = y + beta g(x).
__device__ __forceinline__ float pdbo_update(float x, float y, float d, float gx, float alpha, float beta,
                                             float delta, float grad_tol, float* y_next) {
  const bool stagnating = fabsf(x - 0.5f) <= delta && fabsf(d) <= grad_tol && y <= 0.0f;
  float xn;
  if (stagnating) {
    xn = (x <= 0.5f) ? 0.5f - delta : 0.5f + delta;
  } else {
    xn = fminf(fmaxf(x - alpha * d, 0.0f), 1.0f);
  }
  *y_next = y + beta * gx;
  return xn;
}

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator: output number k of the
// stream seeded with `seed` is mix(seed + (k+1) * 0x9E3779B97F4A7C15).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ float uniform24(uint64_t seed, uint64_t r, uint64_t i) {
  const uint64_t z = splitmix64_at(seed, (r << 32) | i);
  return static_cast<float>(static_cast<uint32_t>(z >> 40)) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---- grid barrier between the iterations of one launch (cluster split-K and resident sparse kernels)
// Every CTA of the launch is resident at once (the launch is one cooperative wave), so CTAs may
// wait for one another.  Arrivals only grow within a launch: barrier k (before iteration k) is
// passed once k * gridDim.x arrivals are counted.  The last CTA to leave the kernel sets the
// words back to zero for the next launch.  A CTA that gives up waiting raises the abort word,
// which ends every other CTA's waits too.
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Orders this thread's earlier generic-proxy stores before later async-proxy (TMA) reads of other
// CTAs, then before the release that publishes them.
__device__ __forceinline__ void fence_stores_for_tma() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __threadfence();
}
__device__ __forceinline__ bool grid_wait(const unsigned int* gbar, unsigned int target, uint64_t deadline) {
  uint32_t spins = 0;
  while (ld_acquire_gpu(gbar) < target) {
    if (ld_acquire_gpu(gbar + 2) != 0u) return false;
    if ((++spins & 15u) == 0u && globaltimer_ns() > deadline) return false;
    __nanosleep(64);
  }
  return true;
}

}  // namespace sbo
