// Set-up kernels: canonicalisation of a dense integer QUBO (Prop. 2.4), the x^0 / y^0
// initialisation (App. C.1) and layout/type conversions of iterates.
#include "sbo_internal.h"

namespace sbo {

// A_ij = Q_ij + Q_ji (i != j), A_ii = 0, written as FP32 or BF16 with leading dimension lda
// (columns n .. lda-1 zero).  A block owns the pair of 64 x 64 tiles (I, J) and (J, I), I <= J,
// of the tile columns J in [j0, j1) (pairs numbered down each column: (0, J), (1, J) .. (J, J)),
// which needs Q's rows of tiles up to j1 only: it reads both tiles of Q once into shared memory and
// writes both tiles of A (A(J, I) is A(I, J) transposed), so Q is read once in all and every
// global access runs along rows.  Row sums of |A_ij| (exactness of A b in FP32) are formed per
// tile row from shared memory and added with one atomic per row per tile; entries whose magnitude
// exceeds a_limit (not exact in the storage type) raise a flag.
constexpr int CANON_T = 64;

__device__ __forceinline__ int64_t tri(int64_t J) { return J * (J + 1) / 2; }   // pairs in columns < J

template <typename TQ>   // int32_t or int8_t entries of Q
__global__ void __launch_bounds__(256) k_canon_dense(const TQ* __restrict__ Q, int64_t n, int64_t j0, void* A,
                                                     int64_t lda, int a_type, unsigned long long* rowsum,
                                                     uint32_t* range_err, int64_t a_limit) {
  __shared__ int32_t s1[CANON_T][CANON_T + 1];   // Q(I, J)
  __shared__ int32_t s2[CANON_T][CANON_T + 1];   // Q(J, I)
  // pair index -> (I, J): q = tri(J) + I with 0 <= I <= J
  const int64_t q = tri(j0) + (int64_t)blockIdx.x;
  int64_t J = (int64_t)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
  if (J < 0) J = 0;
  while (J > 0 && tri(J) > q) --J;
  while (tri(J + 1) <= q) ++J;
  const int64_t I = q - tri(J);
  const int64_t r0 = I * CANON_T, c0 = J * CANON_T;
  const int tid = threadIdx.x;
  // both tiles, rows of 64 entries: a warp reads two rows' 4-entry groups, thread t columns 4(t%16)..+3
#pragma unroll 4
  for (int e = tid; e < CANON_T * CANON_T / 4; e += 256) {
    const int r = e >> 4, q = (e & 15) * 4;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t gi = r0 + r, gj = c0 + q + u;
      s1[r][q + u] = (gi < n && gj < n) ? (int32_t)Q[gi * n + gj] : 0;
      const int64_t hi = c0 + r, hj = r0 + q + u;
      s2[r][q + u] = (hi < n && hj < n) ? (int32_t)Q[hi * n + hj] : 0;
    }
  }
  __syncthreads();
  bool over = false;
  // A(I, J)[r][q] = s1[r][q] + s2[q][r];  A(J, I)[r][q] = s2[r][q] + s1[q][r]
#pragma unroll 2
  for (int e = tid; e < CANON_T * CANON_T / 4; e += 256) {
    const int r = e >> 4, q = (e & 15) * 4;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      if (side == 1 && I == J) break;
      const int64_t gi = (side ? c0 : r0) + r, gj0 = (side ? r0 : c0) + q;
      if (gi >= n || gj0 >= lda) continue;   // rows beyond n are not stored; lda - gj0 >= 4
      int64_t v[4];   // int32 entries: the sum of two can leave int32
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        v[u] = side ? (int64_t)s2[r][q + u] + s1[q + u][r] : (int64_t)s1[r][q + u] + s2[q + u][r];
        if (gi == gj0 + u) v[u] = 0;
        over |= (v[u] < 0 ? -v[u] : v[u]) > a_limit;
      }
      if (a_type == OP_F32) {
        *reinterpret_cast<float4*>(static_cast<float*>(A) + gi * lda + gj0) =
            make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
      } else {
        __nv_bfloat162 lo = __floats2bfloat162_rn((float)v[0], (float)v[1]);
        __nv_bfloat162 hi = __floats2bfloat162_rn((float)v[2], (float)v[3]);
        uint2 raw;
        raw.x = *reinterpret_cast<uint32_t*>(&lo);
        raw.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(A) + gi * lda + gj0) = raw;
      }
    }
  }
  if (over) atomicOr(range_err, 1u);
  // row sums: threads 0..63 the rows of A(I, J), threads 64..127 the rows of A(J, I)
  if (tid < 2 * CANON_T && !(tid >= CANON_T && I == J)) {
    const bool side = tid >= CANON_T;
    const int r = tid & (CANON_T - 1);
    const int64_t gi = (side ? c0 : r0) + r;
    if (gi < n) {
      unsigned long long sum = 0ull;
      for (int q = 0; q < CANON_T; ++q) {
        const int64_t gj = (side ? r0 : c0) + q;
        const int64_t v = (gj == gi) ? 0 : (side ? (int64_t)s2[r][q] + s1[q][r] : (int64_t)s1[r][q] + s2[q][r]);
        sum += (unsigned long long)(v < 0 ? -v : v);
      }
      if (sum) atomicAdd(&rowsum[gi], sum);
    }
  }
}

// c'_i = c_i + Q_ii, exact in int64, and its FP32 value.
template <typename TQ>
__global__ void k_canon_linear(const TQ* __restrict__ Q, const int32_t* __restrict__ c, int64_t n,
                               float* cp, int64_t* cp64) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t v = (int64_t)Q[i * n + i] + (c ? (int64_t)c[i] : 0);
  cp64[i] = v;
  cp[i] = (float)v;
}

__global__ void k_rowsum_check(const unsigned long long* rowsum, const int64_t* cp64, int64_t n,
                               uint32_t* range_err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (rowsum[i] >= (1ull << 24)) atomicOr(range_err, 2u);
  const int64_t c = cp64[i];
  if (c >= (1ll << 31) || c <= -(1ll << 31)) atomicOr(range_err, 4u);
}

cudaError_t launch_canon_dense(const void* Qd, int q_bytes, int64_t n, int64_t j0, int64_t j1, void* A, int64_t lda,
                               int a_type, unsigned long long* rowsum, uint32_t* range_err, int64_t a_limit,
                               cudaStream_t s) {
  if (lda % 4 != 0 || lda < n || j0 < 0 || j1 < j0) return cudaErrorInvalidValue;   // 4-entry stores along rows
  const int64_t pairs = j1 * (j1 + 1) / 2 - j0 * (j0 + 1) / 2;
  if (pairs == 0) return cudaSuccess;
  if (pairs > 0x7fffffffLL) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)pairs), block(256);
  if (q_bytes == 1)
    k_canon_dense<int8_t><<<grid, block, 0, s>>>(static_cast<const int8_t*>(Qd), n, j0, A, lda, a_type, rowsum,
                                                 range_err, a_limit);
  else
    k_canon_dense<int32_t><<<grid, block, 0, s>>>(static_cast<const int32_t*>(Qd), n, j0, A, lda, a_type, rowsum,
                                                  range_err, a_limit);
  return cudaGetLastError();
}

cudaError_t launch_canon_linear(const void* Qd, int q_bytes, const int32_t* cd, int64_t n, float* cp, int64_t* cp64,
                                cudaStream_t s) {
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (q_bytes == 1)
    k_canon_linear<int8_t><<<blocks, 256, 0, s>>>(static_cast<const int8_t*>(Qd), cd, n, cp, cp64);
  else
    k_canon_linear<int32_t><<<blocks, 256, 0, s>>>(static_cast<const int32_t*>(Qd), cd, n, cp, cp64);
  return cudaGetLastError();
}

cudaError_t launch_rowsum_check(const unsigned long long* rowsum, const int64_t* cp64, int64_t n,
                                uint32_t* range_err, cudaStream_t s) {
  k_rowsum_check<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rowsum, cp64, n, range_err);
  return cudaGetLastError();
}

// x^0 from the caller (host-provided, copied to the device as FP32 [B][n]) or from SplitMix64;
// y^0 from the caller or ybar.  Writes the FP32 master (if any), the contraction operand and y in `layout`.
__global__ void k_init_state(int n, int B, int64_t ld, int layout, uint64_t seed, float ybar,
                             const float* __restrict__ x0, const float* __restrict__ y0, float* Xm, void* Xop,
                             int op_type, float* Y, uint32_t* err) {
  const int64_t total = (int64_t)n * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r, i;
    if (layout == LAYOUT_RN) { r = e / n; i = e % n; } else { i = e / B; r = e % B; }
    float x = x0 ? x0[r * n + i] : uniform24(seed, (uint64_t)r, (uint64_t)i);
    if (!(x >= 0.0f && x <= 1.0f)) {  // also rejects NaN
      atomicOr(err, ERR_BOUNDS);
      x = 0.5f;
    }
    const int64_t idx = layout == LAYOUT_RN ? r * ld + i : i * ld + r;
    if (Xm) Xm[idx] = x;
    op_store(Xop, idx, x, op_type);
    Y[idx] = y0 ? y0[r * n + i] : ybar;
  }
}

cudaError_t launch_init_state(int n, int B, int64_t ld, int layout, uint64_t seed, float ybar,
                              const float* x0, const float* y0, float* Xm, void* Xop, int op_type, float* Y,
                              uint32_t* err, cudaStream_t s) {
  const int64_t total = (int64_t)n * B;
  const int64_t blocks = (total + 255) / 256;
  k_init_state<<<(unsigned)(blocks < 152 * 64 ? blocks : 152 * 64), 256, 0, s>>>(
      n, B, ld, layout, seed, ybar, x0, y0, Xm, Xop, op_type, Y, err);
  return cudaGetLastError();
}

// FP32 [B][n] (ld_in) -> operand type, restart-major (ld_out).
__global__ void k_to_operand(const float* __restrict__ X, int n, int B, int64_t ld_in, void* out,
                             int64_t ld_out, int op_type) {
  const int64_t total = (int64_t)n * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / n, i = e % n;
    op_store(out, r * ld_out + i, X[r * ld_in + i], op_type);
  }
}

cudaError_t launch_to_operand(const float* X, int n, int B, int64_t ld_in, void* out, int64_t ld_out,
                              int op_type, cudaStream_t s) {
  const int64_t total = (int64_t)n * B;
  const int64_t blocks = (total + 255) / 256;
  k_to_operand<<<(unsigned)(blocks < 152 * 64 ? blocks : 152 * 64), 256, 0, s>>>(X, n, B, ld_in, out, ld_out,
                                                                                 op_type);
  return cudaGetLastError();
}

// The same conversion into the variable-major layout of the sparse kernels: out[i * ld_out + r].
__global__ void k_to_operand_t(const float* __restrict__ X, int n, int B, int64_t ld_in, void* out,
                               int64_t ld_out, int op_type) {
  const int64_t total = (int64_t)n * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / n, i = e % n;
    op_store(out, i * ld_out + r, X[r * ld_in + i], op_type);
  }
}

cudaError_t launch_to_operand_t(const float* X, int n, int B, int64_t ld_in, void* out, int64_t ld_out,
                                int op_type, cudaStream_t s) {
  const int64_t total = (int64_t)n * B;
  const int64_t blocks = (total + 255) / 256;
  k_to_operand_t<<<(unsigned)(blocks < 152 * 64 ? blocks : 152 * 64), 256, 0, s>>>(X, n, B, ld_in, out, ld_out,
                                                                                   op_type);
  return cudaGetLastError();
}

// 0/1 bytes [count][n] -> operand (0.0 / 1.0) in `layout`.
__global__ void k_bits_to_operand(const uint8_t* __restrict__ bits, int n, int count, void* out,
                                  int64_t ld_out, int layout, int op_type) {
  const int64_t total = (int64_t)n * count;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / n, i = e % n;
    const int64_t idx = layout == LAYOUT_RN ? r * ld_out + i : i * ld_out + r;
    op_store(out, idx, (float)bits[e], op_type);   // 0/1, or a Max-k-Cut part index
  }
}

cudaError_t launch_bits_to_operand(const uint8_t* bits, int n, int count, void* out, int64_t ld_out,
                                   int layout, int op_type, cudaStream_t s) {
  const int64_t total = (int64_t)n * count;
  const int64_t blocks = (total + 255) / 256;
  k_bits_to_operand<<<(unsigned)(blocks < 152 * 64 ? blocks : 152 * 64), 256, 0, s>>>(bits, n, count, out,
                                                                                      ld_out, layout, op_type);
  return cudaGetLastError();
}

__global__ void k_fill_i64(long long* p, int64_t count, long long v) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
    p[e] = v;
}

cudaError_t launch_fill_i64(long long* p, int64_t count, long long v, cudaStream_t s) {
  const int64_t blocks = (count + 255) / 256;
  k_fill_i64<<<(unsigned)(blocks < 1024 ? (blocks > 0 ? blocks : 1) : 1024), 256, 0, s>>>(p, count, v);
  return cudaGetLastError();
}

// state in `layout` -> dense [B][n] FP32 (for host read-back).
__global__ void k_gather_state(const float* __restrict__ src, int n, int B, int64_t ld, int layout,
                               float* dst) {
  const int64_t total = (int64_t)n * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / n, i = e % n;
    dst[e] = layout == LAYOUT_RN ? src[r * ld + i] : src[i * ld + r];
  }
}

cudaError_t launch_gather_state(const float* src, int n, int B, int64_t ld, int layout, float* dst,
                                cudaStream_t s) {
  const int64_t total = (int64_t)n * B;
  const int64_t blocks = (total + 255) / 256;
  k_gather_state<<<(unsigned)(blocks < 152 * 64 ? blocks : 152 * 64), 256, 0, s>>>(src, n, B, ld, layout,
                                                                                   dst);
  return cudaGetLastError();
}

}  // namespace sbo
