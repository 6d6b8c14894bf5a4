// Plain FP32 form of the contraction (CUDA cores) with the fused PDBO epilogue.
//
// Computes G[r][i] = sum_k X[r][k] A[k][i] (= (A x_r)_i, A symmetric) for a 64 (restarts) x
// 64 (variables) tile per CTA, whole K per tile, then applies one of three epilogues:
//   EPI_UPDATE  one iteration of Algorithm 1 (d = G + c' + y(2x-1), perturbation rule,
//               projection, dual step with the old x); writes x^{t+1} into the other
//               ping-pong buffer, y in place and optionally b = [x^{t+1} > 1/2]
//   EPI_EVAL    X holds 0/1 candidates b: accumulates 2F(b) = sum_i b_i (G_i + 2 c'_i) per
//               restart in int64 (G is an exact integer because row sums of |A| < 2^24)
//   EPI_LAGR    value and gradients of the Lagrangian (section 3.1)
// State arrays are restart-major: element (r, i) at [r * ld + i].  In the single-constraint form
// (a.mu set) the update reads mu[r] for y and writes, per 64-variable tile (blockIdx.x), the sum
// of g(x^t) of each restart into row blockIdx.x of the partial sums.
#include "sbo_internal.h"

namespace sbo {

constexpr int SM_BM = 64;   // restarts per tile
constexpr int SM_BN = 64;   // variables per tile
constexpr int SM_BK = 16;

template <int MODE>
__global__ void __launch_bounds__(256) k_simt(const float* __restrict__ A, int64_t lda, EpiArgs a) {
  __shared__ float As[2][SM_BK][SM_BN];
  __shared__ float Xs[2][SM_BK][SM_BM + 4];
  const int n = a.n, B = a.B;
  const int64_t ld = a.ld;
  const float* __restrict__ X = static_cast<const float*>(MODE == EPI_LAGR ? (const void*)a.Xl : a.Xin);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * SM_BN;
  const int64_t r0 = (int64_t)blockIdx.y * SM_BM;

  float acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.0f;

  // loader coordinates
  const int a_kk = tid >> 4, a_ii = (tid & 15) * 4;   // A tile: 16 rows (k) x 64 cols (i)
  const int x_rr = tid >> 2, x_kq = (tid & 3) * 4;    // X tile: 64 rows (r) x 16 cols (k)
  float4 ra, rx;
  auto load_regs = [&](int64_t k0) {
    const int64_t ka = k0 + a_kk;
    const int64_t ia = i0 + a_ii;
    if (ka < n && ia < lda) ra = *reinterpret_cast<const float4*>(A + ka * lda + ia);
    else ra = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t r = r0 + x_rr;
    const int64_t kx = k0 + x_kq;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (r < B) {
      const float* src = X + r * ld + kx;
      if (kx + 3 < n && (((uintptr_t)src & 15) == 0)) {
        const float4 t = *reinterpret_cast<const float4*>(src);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = (kx + j < n) ? src[j] : 0.f;
      }
    }
    rx = make_float4(v[0], v[1], v[2], v[3]);
  };
  auto store_smem = [&](int buf) {
    *reinterpret_cast<float4*>(&As[buf][a_kk][a_ii]) = ra;
    Xs[buf][x_kq + 0][x_rr] = rx.x;
    Xs[buf][x_kq + 1][x_rr] = rx.y;
    Xs[buf][x_kq + 2][x_rr] = rx.z;
    Xs[buf][x_kq + 3][x_rr] = rx.w;
  };

  const int64_t nk = (n + SM_BK - 1) / SM_BK;
  load_regs(0);
  store_smem(0);
  __syncthreads();
  for (int64_t kb = 0; kb < nk; ++kb) {
    const int buf = (int)(kb & 1);
    if (kb + 1 < nk) load_regs((kb + 1) * SM_BK);
#pragma unroll
    for (int kk = 0; kk < SM_BK; ++kk) {
      float av[4], xv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) av[q] = As[buf][kk][tx + 16 * q];
#pragma unroll
      for (int p = 0; p < 4; ++p) xv[p] = Xs[buf][kk][ty + 16 * p];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(xv[p], av[q], acc[p][q]);
    }
    if (kb + 1 < nk) store_smem(buf ^ 1);
    __syncthreads();
  }

  // ---- epilogue ---------------------------------------------------------------------------
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int64_t r = r0 + ty + 16 * p;
    long long f2 = 0;
    float lsum = 0.0f, gsum = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = i0 + tx + 16 * q;
      if (r >= B || i >= n) continue;
      const int64_t idx = r * ld + i;
      const float g = acc[p][q];
      if (MODE == EPI_UPDATE) {
        const float x = a.Xm ? a.Xm[idx] : static_cast<const float*>(a.Xin)[idx];
        const float y = a.mu ? a.mu[r] : a.Y[idx];   // single-constraint form: the restart's dual
        const float gx = g_val(x, a.gkind);
        const float d = g + a.cp[i] + y * g_der(x, a.gkind);
        float yn;
        const float xn = pdbo_update(x, y, d, gx, a.alpha, a.beta, a.delta, a.grad_tol, &yn);
        if (a.Gd) a.Gd[idx] = d;
        if (a.Xm) a.Xm[idx] = xn;
        static_cast<float*>(a.Xout)[idx] = xn;
        if (a.mu) gsum += gx;
        else a.Y[idx] = yn;
        if (a.bits_out) static_cast<float*>(a.bits_out)[idx] = xn > 0.5f ? 1.0f : 0.0f;
      } else if (MODE == EPI_EVAL) {
        const float b = X[idx];
        if (b != 0.0f) f2 += (long long)g + 2 * (long long)a.cp64[i];
      } else {
        const float x = a.Xl[idx], y = a.Yl[idx];
        const float gx = g_val(x, a.gkind);
        const float sc = a.gout ? a.gout[r] : 1.0f;
        if (a.GX) a.GX[idx] = sc * (g + a.cp[i] + y * g_der(x, a.gkind));
        if (a.GY) a.GY[idx] = sc * gx;
        lsum += 0.5f * x * g + a.cp[i] * x + y * gx;
      }
    }
    if (MODE == EPI_EVAL) {
      // lanes 0-15 and 16-31 of a warp hold two different restarts: reduce within each half
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) f2 += __shfl_xor_sync(0xffffffffu, f2, o);
      if (tx == 0 && r < B && f2 != 0) atomicAdd(&a.F2[r], (unsigned long long)f2);
    }
    if (MODE == EPI_UPDATE && a.mu) {
      // this tile's 64 variables: the 16 lanes of a half warp hold one restart
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) gsum += __shfl_xor_sync(0xffffffffu, gsum, o);
      if (tx == 0 && r < B) a.gpart[(int64_t)blockIdx.x * a.gpart_ld + r] = gsum;
    }
    if (MODE == EPI_LAGR && a.L) {
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
      if (tx == 0 && r < B) atomicAdd(&a.L[r], lsum);
    }
  }
}

cudaError_t launch_simt(const float* A, int64_t lda, const EpiArgs& a, int mode, cudaStream_t s) {
  dim3 grid((unsigned)((a.n + SM_BN - 1) / SM_BN), (unsigned)((a.B + SM_BM - 1) / SM_BM));
  if (mode == EPI_UPDATE) k_simt<EPI_UPDATE><<<grid, 256, 0, s>>>(A, lda, a);
  else if (mode == EPI_EVAL) k_simt<EPI_EVAL><<<grid, 256, 0, s>>>(A, lda, a);
  else k_simt<EPI_LAGR><<<grid, 256, 0, s>>>(A, lda, a);
  return cudaGetLastError();
}

}  // namespace sbo
