// Set-up kernels: canonicalisation of a dense integer QUBO (Prop. 2.4), the x^0 / y^0
// initialisation (App. C.1) and layout/type conversions of iterates.
#include "sbo_internal.h"

namespace sbo {

// A_ij = Q_ij + Q_ji (i != j), A_ii = 0, written as FP32 or BF16 with leading dimension lda.
// A block owns 32 rows and CANON_TJ consecutive 32x32 column tiles; each tile's transpose is
// staged through shared memory so both reads coalesce.  Row sums of |A_ij| (exactness of A b in
// FP32) accumulate in registers over the block's tiles and are added with one atomic per row per
// block; entries whose magnitude exceeds a_limit (not exact in the storage type) raise a flag.
constexpr int CANON_TJ = 16;

template <typename TQ>   // int32_t or int8_t entries of Q
__global__ void __launch_bounds__(256) k_canon_dense(const TQ* __restrict__ Q, int64_t n, void* A,
                                                     int64_t lda, int a_type, unsigned long long* rowsum,
                                                     uint32_t* range_err, int64_t a_limit) {
  __shared__ int32_t tT[32][33];
  const int64_t i0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  unsigned long long rs[4] = {0ull, 0ull, 0ull, 0ull};
  bool over = false;
  for (int t = 0; t < CANON_TJ; ++t) {
    const int64_t j0 = ((int64_t)blockIdx.x * CANON_TJ + t) * 32;
    if (j0 >= lda) break;
    // transposed tile: tT[a][b] = Q[j0 + a][i0 + b]
    for (int a = ty; a < 32; a += 8) {
      const int64_t r = j0 + a, cidx = i0 + tx;
      tT[a][tx] = (r < n && cidx < n) ? Q[r * n + cidx] : 0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int a = ty + 8 * k;
      const int64_t i = i0 + a, j = j0 + tx;
      int64_t v = 0;
      if (i < n && j < n && i != j) v = (int64_t)Q[i * n + j] + (int64_t)tT[tx][a];
      const int64_t av = v < 0 ? -v : v;
      over |= av > a_limit;
      if (i < n && j < lda) {
        if (a_type == OP_F32) static_cast<float*>(A)[i * lda + j] = (float)v;
        else static_cast<__nv_bfloat16*>(A)[i * lda + j] = __float2bfloat16_rn((float)v);
      }
      rs[k] += (unsigned long long)av;
    }
    __syncthreads();
  }
  if (over) atomicOr(range_err, 1u);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    unsigned long long s2 = rs[k];
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    const int64_t i = i0 + ty + 8 * k;
    if (tx == 0 && i < n && s2) atomicAdd(&rowsum[i], s2);
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

cudaError_t launch_canon_dense(const void* Qd, int q_bytes, const int32_t* cd, int64_t n, void* A, int64_t lda,
                               int a_type, float* cp, int64_t* cp64, unsigned long long* rowsum,
                               uint32_t* range_err, int64_t a_limit, cudaStream_t s) {
  const int64_t nb = (n + 31) / 32;
  const int64_t nbx = (lda + 32 * CANON_TJ - 1) / (32 * CANON_TJ);
  dim3 grid((unsigned)nbx, (unsigned)nb), block(32, 8);
  if (q_bytes == 1) {
    const int8_t* Q8 = static_cast<const int8_t*>(Qd);
    k_canon_dense<int8_t><<<grid, block, 0, s>>>(Q8, n, A, lda, a_type, rowsum, range_err, a_limit);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_canon_linear<int8_t><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Q8, cd, n, cp, cp64);
  } else {
    const int32_t* Q32 = static_cast<const int32_t*>(Qd);
    k_canon_dense<int32_t><<<grid, block, 0, s>>>(Q32, n, A, lda, a_type, rowsum, range_err, a_limit);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_canon_linear<int32_t><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Q32, cd, n, cp, cp64);
  }
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
