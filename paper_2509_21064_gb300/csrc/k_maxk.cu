// Max-k-Cut (the appendix on Max-k-Cut): every vertex i of restart r carries logits Z_:,i (k of
// them) and the point X_:,i = softmax(Z_:,i) of the simplex.  One iteration of the simultaneous
// GDA on L(X, y) = Tr(X W X^T) + sum_i y_i (|X_:,i|^2 - 1):
//
//   G = W X (sparse W, both edge directions stored)          h_j = 2 (G_j + y s_j),  s = X_:,i
//   Z_j <- Z_j - alpha s_j (h_j - <s, h>)                     y <- y + beta (|s|^2 - 1)
//   X'_:,i = softmax(Z'_:,i); candidate part = argmax_j X'_ji (ties to the smallest j)
//
// State is variable-major like the sparse QUBO kernel: Z and the operand X at [(i k + j) ld + r],
// y and the candidate parts (as floats) at [i ld + r], ld a multiple of 8.  One warp owns one row
// i and 128 restarts; lane l holds restarts 4l .. 4l+3 of the chunk (16-byte vectors), so the
// gather of neighbour l's k rows of X is k coalesced 512-byte runs.  Neighbour indices and weights
// are loaded 32 at a time and broadcast with shuffles.  The evaluation mode accumulates
// -w [p_i != p_l] over the stored (i, l) entries, i.e. 2F with F = -cut, in int64.
#include <algorithm>

#include "sbo_internal.h"

namespace sbo {
namespace {

__device__ __forceinline__ float cmp4(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
__device__ __forceinline__ void set4(float4& v, int k, float s) {
  if (k == 0) v.x = s; else if (k == 1) v.y = s; else if (k == 2) v.z = s; else v.w = s;
}

template <int MODE, int KP>
__global__ void __launch_bounds__(256) k_maxk(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                              const float* __restrict__ wv, EpiArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t r0 = (int64_t)blockIdx.y * 128 + 4 * lane;
  const int n = a.n, B = a.B;
  const int64_t ld = a.ld;
  const float* __restrict__ Xin = static_cast<const float*>(a.Xin);
  long long f2[4] = {0, 0, 0, 0};
  const bool lane_live = r0 < B;

  for (int64_t i = warp0; i < n; i += nwarps) {
    float4 acc[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (MODE == EPI_EVAL && lane_live) pi = *reinterpret_cast<const float4*>(Xin + i * ld + r0);
    const int e0 = __ldg(rowptr + i), e1 = __ldg(rowptr + i + 1);
    for (int eb = e0; eb < e1; eb += 32) {
      const int k = eb + lane;
      const int mycol = k < e1 ? __ldg(col + k) : 0;
      const float myw = k < e1 ? __ldg(wv + k) : 0.0f;
      const int cnt = min(32, e1 - eb);
      for (int q = 0; q < cnt; ++q) {
        const int64_t l = __shfl_sync(0xffffffffu, mycol, q);
        const float w = __shfl_sync(0xffffffffu, myw, q);
        if (!lane_live) continue;
        if (MODE == EPI_UPDATE) {
#pragma unroll
          for (int j = 0; j < KP; ++j) {
            const float4 xv = *reinterpret_cast<const float4*>(Xin + (l * KP + j) * ld + r0);
            acc[j].x = fmaf(w, xv.x, acc[j].x);
            acc[j].y = fmaf(w, xv.y, acc[j].y);
            acc[j].z = fmaf(w, xv.z, acc[j].z);
            acc[j].w = fmaf(w, xv.w, acc[j].w);
          }
        } else {
          const float4 pl = *reinterpret_cast<const float4*>(Xin + l * ld + r0);
          const long long wi = (long long)w;
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (cmp4(pi, c) != cmp4(pl, c)) f2[c] -= wi;
        }
      }
    }
    if (MODE == EPI_UPDATE && lane_live) {
      float4 z[KP], s[KP];
#pragma unroll
      for (int j = 0; j < KP; ++j) {
        z[j] = *reinterpret_cast<const float4*>(a.Xm + (i * KP + j) * ld + r0);
        s[j] = *reinterpret_cast<const float4*>(Xin + (i * KP + j) * ld + r0);
      }
      const float4 y4 = *reinterpret_cast<const float4*>(a.Y + i * ld + r0);
      float4 yn4 = make_float4(0.f, 0.f, 0.f, 0.f), part4 = yn4;
      float4 zn[KP], xn[KP];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const bool live = r0 + c < B;   // padding restarts keep their zeros
        const float y = cmp4(y4, c);
        float h[KP], dot = 0.0f, ss = 0.0f;
#pragma unroll
        for (int j = 0; j < KP; ++j) {
          const float sj = cmp4(s[j], c);
          h[j] = 2.0f * (cmp4(acc[j], c) + y * sj);
          dot = fmaf(sj, h[j], dot);
          ss = fmaf(sj, sj, ss);
        }
        float zmax = -INFINITY, znew[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) {
          const float sj = cmp4(s[j], c);
          znew[j] = cmp4(z[j], c) - a.alpha * (sj * (h[j] - dot));
          zmax = fmaxf(zmax, znew[j]);
        }
        float den = 0.0f, e[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) {
          e[j] = expf(znew[j] - zmax);
          den += e[j];
        }
        const float inv = 1.0f / den;
        int best = 0;
        float bx = -1.0f;
#pragma unroll
        for (int j = 0; j < KP; ++j) {
          const float xj = e[j] * inv;
          if (xj > bx) { bx = xj; best = j; }
          set4(zn[j], c, live ? znew[j] : 0.0f);
          set4(xn[j], c, live ? xj : 0.0f);
        }
        set4(yn4, c, live ? y + a.beta * (ss - 1.0f) : 0.0f);
        set4(part4, c, live ? (float)best : 0.0f);
      }
#pragma unroll
      for (int j = 0; j < KP; ++j) {
        *reinterpret_cast<float4*>(a.Xm + (i * KP + j) * ld + r0) = zn[j];
        *reinterpret_cast<float4*>(static_cast<float*>(a.Xout) + (i * KP + j) * ld + r0) = xn[j];
      }
      *reinterpret_cast<float4*>(a.Y + i * ld + r0) = yn4;
      if (a.bits_out) *reinterpret_cast<float4*>(static_cast<float*>(a.bits_out) + i * ld + r0) = part4;
    }
  }
  if (MODE == EPI_EVAL) {
    __shared__ unsigned long long red[128];
    for (int t = threadIdx.x; t < 128; t += blockDim.x) red[t] = 0ull;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (f2[c] != 0) atomicAdd(&red[4 * lane + c], (unsigned long long)f2[c]);
    __syncthreads();
    const int64_t rb = (int64_t)blockIdx.y * 128;
    for (int t = threadIdx.x; t < 128; t += blockDim.x)
      if (rb + t < B && red[t] != 0ull) atomicAdd(&a.F2[rb + t], red[t]);
  }
}

// Z^0_{(i k + j) ld + r} = U(seed, r, i k + j), y^0 = ybar, X^0 = softmax(Z^0); padding zero.
template <int KP>
__global__ void k_maxk_init(int n, int B, int64_t ld, uint64_t seed, float ybar, float* Z, float* Y, float* X) {
  const int64_t total = (int64_t)n * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ld, r = e % ld;
    const bool live = r < B;
    float z[KP], zmax = -INFINITY;
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      z[j] = live ? uniform24(seed, (uint64_t)r, (uint64_t)(i * KP + j)) : 0.0f;
      zmax = fmaxf(zmax, z[j]);
    }
    float den = 0.0f;
#pragma unroll
    for (int j = 0; j < KP; ++j) den += expf(z[j] - zmax);
    const float inv = 1.0f / den;
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      Z[(i * KP + j) * ld + r] = z[j];
      X[(i * KP + j) * ld + r] = live ? expf(z[j] - zmax) * inv : 0.0f;
    }
    Y[i * ld + r] = live ? ybar : 0.0f;
  }
}

// [r][i][j] view of a [(i k + j) ld + r] array (state read-back).
__global__ void k_maxk_gather(const float* __restrict__ src, int n, int kp, int B, int64_t ld, float* dst) {
  const int64_t total = (int64_t)B * n * kp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ((int64_t)n * kp), q = e % ((int64_t)n * kp);
    dst[e] = src[q * ld + r];
  }
}

template <int MODE>
cudaError_t launch_mode(const int32_t* rowptr, const int32_t* col, const float* w, const EpiArgs& a, int kp,
                        cudaStream_t s) {
  const int64_t chunks = (a.B + 127) / 128;
  int64_t want = (a.n + 7) / 8;
  if (MODE == EPI_EVAL) {
    const int64_t cap = (int64_t)152 * 8 / chunks + 1;   // bounds the closing atomics
    if (want > cap) want = cap;
  }
  if (want > 65535) want = 65535;
  const dim3 grid((unsigned)want, (unsigned)chunks);
  switch (kp) {
    case 2: k_maxk<MODE, 2><<<grid, 256, 0, s>>>(rowptr, col, w, a); break;
    case 3: k_maxk<MODE, 3><<<grid, 256, 0, s>>>(rowptr, col, w, a); break;
    case 4: k_maxk<MODE, 4><<<grid, 256, 0, s>>>(rowptr, col, w, a); break;
    case 5: k_maxk<MODE, 5><<<grid, 256, 0, s>>>(rowptr, col, w, a); break;
    case 6: k_maxk<MODE, 6><<<grid, 256, 0, s>>>(rowptr, col, w, a); break;
    case 7: k_maxk<MODE, 7><<<grid, 256, 0, s>>>(rowptr, col, w, a); break;
    case 8: k_maxk<MODE, 8><<<grid, 256, 0, s>>>(rowptr, col, w, a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_maxk(const int32_t* rowptr, const int32_t* col, const float* w, const EpiArgs& a, int kp, int mode,
                        cudaStream_t s) {
  if (a.ld % 8 != 0 || kp < 2 || kp > 8) return cudaErrorInvalidValue;
  if (mode == EPI_UPDATE) return launch_mode<EPI_UPDATE>(rowptr, col, w, a, kp, s);
  if (mode == EPI_EVAL) return launch_mode<EPI_EVAL>(rowptr, col, w, a, kp, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_maxk_init(int n, int B, int64_t ld, int kp, uint64_t seed, float ybar, float* Z, float* Y, float* X,
                             cudaStream_t s) {
  const int64_t total = (int64_t)n * ld;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
  switch (kp) {
    case 2: k_maxk_init<2><<<blocks, 256, 0, s>>>(n, B, ld, seed, ybar, Z, Y, X); break;
    case 3: k_maxk_init<3><<<blocks, 256, 0, s>>>(n, B, ld, seed, ybar, Z, Y, X); break;
    case 4: k_maxk_init<4><<<blocks, 256, 0, s>>>(n, B, ld, seed, ybar, Z, Y, X); break;
    case 5: k_maxk_init<5><<<blocks, 256, 0, s>>>(n, B, ld, seed, ybar, Z, Y, X); break;
    case 6: k_maxk_init<6><<<blocks, 256, 0, s>>>(n, B, ld, seed, ybar, Z, Y, X); break;
    case 7: k_maxk_init<7><<<blocks, 256, 0, s>>>(n, B, ld, seed, ybar, Z, Y, X); break;
    case 8: k_maxk_init<8><<<blocks, 256, 0, s>>>(n, B, ld, seed, ybar, Z, Y, X); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_maxk_gather(const float* src, int n, int kp, int B, int64_t ld, float* dst, cudaStream_t s) {
  const int64_t total = (int64_t)B * n * kp;
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 64);
  k_maxk_gather<<<blocks, 256, 0, s>>>(src, n, kp, B, ld, dst);
  return cudaGetLastError();
}

}  // namespace sbo
