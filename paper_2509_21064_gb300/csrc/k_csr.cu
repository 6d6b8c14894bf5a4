// Sparse form: CSR SpMM G = A X fused with the PDBO epilogue, for graphs (Max-Cut, MIS).
//
// State is variable-major: element (i, r) at [i * ld + r] (ld a multiple of 8), so the B
// restarts of one variable are contiguous.  One warp owns one row i of A and a chunk of 128*NV
// restarts; lane l holds the 4 consecutive restarts rbase + 128 v + 4 l .. +3 (v < NV), so each
// gather X[j][...] of a neighbour j is one 512-byte (FP32) or 256-byte (BF16) run per v (128
// bytes of candidates in EPI_EVAL, which reads one byte per (vertex, restart)).  The row's column
// indices and weights are loaded 32 at a time, one per lane, and broadcast with shuffles, so the
// gathers of consecutive neighbours do not wait on each other; the row's own x and y are loaded
// before the gathers.  Warps stride over rows; in EPI_EVAL every lane keeps per-restart int64
// partial sums of 2F over its rows; a block sums its warps' partials in shared memory, in warp
// order, and adds one value per restart to the global accumulator.
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "sbo_internal.h"

namespace sbo {

enum ValType : int { VAL_F32 = 0, VAL_BF16 = 1, VAL_E4M3 = 2 };

constexpr int64_t CSR_WAVES = 1;   // resident waves of blocks per launch

__device__ __forceinline__ float load_val(const void* val, int64_t e, int vt) {
  if (vt == VAL_F32) return __ldg(static_cast<const float*>(val) + e);
  if (vt == VAL_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(val)[e]);
  __nv_fp8_e4m3 q;
  q.__x = static_cast<const __nv_fp8_storage_t*>(val)[e];
  return static_cast<float>(q);
}

// 4 consecutive operand values (FP32: one 16-byte load; BF16: one 8-byte load; candidate bytes:
// one 4-byte load).
template <int OPT>
__device__ __forceinline__ float4 load4(const void* p, int64_t idx) {
  if (OPT == OP_U8) {
    const uchar4 b = __ldg(reinterpret_cast<const uchar4*>(static_cast<const uint8_t*>(p) + idx));
    return make_float4((float)b.x, (float)b.y, (float)b.z, (float)b.w);
  }
  if (OPT == OP_F32) return __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(p) + idx));
  const uint2 raw = __ldg(reinterpret_cast<const uint2*>(static_cast<const __nv_bfloat16*>(p) + idx));
  const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
  const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
  return make_float4(__low2float(lo), __high2float(lo), __low2float(hi), __high2float(hi));
}
template <int OPT>
__device__ __forceinline__ void store4(void* p, int64_t idx, float4 v) {
  if (OPT == OP_U8) {
    *reinterpret_cast<uchar4*>(static_cast<uint8_t*>(p) + idx) =
        make_uchar4((unsigned char)v.x, (unsigned char)v.y, (unsigned char)v.z, (unsigned char)v.w);
  } else if (OPT == OP_F32) {
    *reinterpret_cast<float4*>(static_cast<float*>(p) + idx) = v;
  } else {
    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
    uint2 raw;
    raw.x = *reinterpret_cast<uint32_t*>(&lo);
    raw.y = *reinterpret_cast<uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(p) + idx) = raw;
  }
}
// L2 eviction priorities for the update's own-state traffic (the "streaming" forms): x and y of a
// row are read and written once per iteration, while the operand rows are gathered by every
// neighbour, so when the state overflows L2 the former are marked evict-first and the operand
// written for the next iteration evict-last.
__device__ __forceinline__ uint64_t l2_policy_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float4 ld_policy4(const float* ptr, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(ptr), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_policy4(float* ptr, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(ptr), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ float comp(const float4& v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
__device__ __forceinline__ void set_comp(float4& v, int k, float s) {
  if (k == 0) v.x = s; else if (k == 1) v.y = s; else if (k == 2) v.z = s; else v.w = s;
}

// GK: constraint function g; SINGLE: one dual per restart (both uniform per launch, so each
// combination is its own instantiation and the per-element code carries no test of them).
// HINT: the streaming forms (L2 eviction priorities on the update's own x and y, see above).
template <int MODE, int NV, int OPT, int GK, bool SINGLE, bool PIPE, bool HINT>
__global__ void __launch_bounds__(256) k_csr(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                             const void* __restrict__ val, int vt, EpiArgs a) {
  constexpr bool UPD = MODE == EPI_UPDATE;
  constexpr bool OBJ = MODE == EPI_EVAL;     // accumulates 2F per restart
  const uint64_t pol_first = HINT ? l2_policy_first() : 0ull;
  const uint64_t pol_last = HINT ? l2_policy_last() : 0ull;
  const int lane = threadIdx.x & 31;
  const int warps_per_block = blockDim.x >> 5;
  const int64_t warp0 = (int64_t)blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const int64_t nwarps = (int64_t)gridDim.x * warps_per_block;
  const int64_t rbase = (int64_t)blockIdx.y * 128 * NV + 4 * lane;
  const int n = a.n, B = a.B;
  const int64_t ld = a.ld;
  const void* Xin = a.Xin;
  long long f2[NV][4];
  float4 gs[NV];   // single-constraint form: sum of g(x^t) over this warp's rows, per restart
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    gs[v] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 4; ++k) f2[v][k] = 0;
  }

  // PIPE: the grid is one wave of resident blocks and each warp strides over several rows,
  // software-pipelined: while row i is processed, the column indices and weights of row
  // i + nwarps (whose extent arrived during the previous row) and the extent of row i + 2 nwarps
  // are in flight, so a row waits only on its gathers.  The evaluation always runs so (its grid
  // is bounded anyway: one closing atomic per restart per block); the update does when its x and
  // y stream from DRAM.  Otherwise a warp takes one row (a grid of ceil(n / 8) blocks per chunk of
  // restarts), which measured faster on L2-resident state than striding at the lower occupancy
  // the pipeline's registers allow.  The structure is constant for the whole run, so the first
  // rows' is read before waiting on the previous kernel and overlaps its tail under programmatic
  // dependent launch.
  int64_t i = warp0;
  int e0 = 0, e1 = 0, col0 = 0, f0 = 0, f1 = 0;
  float val0 = 0.0f, cpi = 0.0f;
  long long cp2 = 0;
  if (i < n) {
    e0 = __ldg(rowptr + i);
    e1 = __ldg(rowptr + i + 1);
    if (PIPE && i + nwarps < n) {
      f0 = __ldg(rowptr + i + nwarps);
      f1 = __ldg(rowptr + i + nwarps + 1);
    }
    const int k = e0 + lane;
    col0 = k < e1 ? __ldg(col + k) : 0;
    val0 = k < e1 ? load_val(val, k, vt) : 0.0f;
    cpi = a.cp[i];
    if (OBJ) cp2 = 2 * (long long)a.cp64[i];
  }
  // Programmatic dependent launch (a no-op when launched without it): wait until the previous
  // kernel of the stream has completed and its writes are visible, then let the next one be
  // scheduled, so that its launch overlaps this kernel instead of following it.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  for (; i < n; i += nwarps) {
    if (!PIPE && i != warp0) {
      e0 = __ldg(rowptr + i);
      e1 = __ldg(rowptr + i + 1);
      const int k = e0 + lane;
      col0 = k < e1 ? __ldg(col + k) : 0;
      val0 = k < e1 ? load_val(val, k, vt) : 0.0f;
      cpi = a.cp[i];
    }
    const int64_t i1 = i + nwarps, i2 = i1 + nwarps;
    int ncol = 0, g0 = 0, g1 = 0;
    float nval = 0.0f, ncpi = 0.0f;
    long long ncp2 = 0;
    if (PIPE && i1 < n) {
      const int k = f0 + lane;
      ncol = k < f1 ? __ldg(col + k) : 0;
      nval = k < f1 ? load_val(val, k, vt) : 0.0f;
      ncpi = a.cp[i1];
      if (OBJ) ncp2 = 2 * (long long)a.cp64[i1];
      if (i2 < n) {
        g0 = __ldg(rowptr + i2);
        g1 = __ldg(rowptr + i2 + 1);
      }
    }
    // the row's own state first: independent of the gathers
    float4 xo[NV], yo[NV];
    uint32_t own_bits[NV];   // EPI_EVAL: the row's own candidate bytes, four restarts per word
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int64_t r0 = rbase + 128 * v;
      xo[v] = make_float4(0.f, 0.f, 0.f, 0.f);
      yo[v] = xo[v];
      own_bits[v] = 0u;
      if (r0 < B) {
        const int64_t idx = i * ld + r0;
        if (UPD) {
          if (HINT) {
            xo[v] = a.Xm ? ld_policy4(a.Xm + idx, pol_first) : load4<OP_F32>(Xin, idx);
            yo[v] = SINGLE ? *reinterpret_cast<const float4*>(a.mu + r0) : ld_policy4(a.Y + idx, pol_first);
          } else {
            xo[v] = a.Xm ? *reinterpret_cast<const float4*>(a.Xm + idx) : load4<OP_F32>(Xin, idx);
            yo[v] = SINGLE ? *reinterpret_cast<const float4*>(a.mu + r0)    // the restarts' duals
                         : *reinterpret_cast<const float4*>(a.Y + idx);
          }
        } else if (MODE == EPI_EVAL) {
          own_bits[v] = __ldg(reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(Xin) + idx));
        } else {
          // EPI_LAGR: the caller's restart-major FP32 x and y, [r][n]
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const bool ok = r0 + k < B;
            set_comp(xo[v], k, ok ? a.Xl[(r0 + k) * (int64_t)n + i] : 0.0f);
            set_comp(yo[v], k, ok ? a.Yl[(r0 + k) * (int64_t)n + i] : 0.0f);
          }
        }
      }
    }
    float4 acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    if constexpr (MODE == EPI_EVAL) {
      // exact objective of 0/1 candidates: (A b)_i in integers -- the weights are integers (exact in
      // their storage type) and the candidate bytes are unpacked with shifts, four restarts per
      // 32-bit word, so no value is converted between float and integer per element
      int ai[NV][4];
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int k = 0; k < 4; ++k) ai[v][k] = 0;
      for (int eb = e0; eb < e1; eb += 32) {
        int mycol = col0;
        float myval = val0;
        if (eb != e0) {
          const int k = eb + lane;
          mycol = k < e1 ? __ldg(col + k) : 0;
          myval = k < e1 ? load_val(val, k, vt) : 0.0f;
        }
        const int wint = __float2int_rn(myval);
        const int cnt = min(32, e1 - eb);
#pragma unroll 4
        for (int q = 0; q < cnt; ++q) {
          const int64_t j = __shfl_sync(0xffffffffu, mycol, q);
          const int w = __shfl_sync(0xffffffffu, wint, q);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const int64_t r0 = rbase + 128 * v;
            if (r0 < B) {
              const uint32_t word =
                  __ldg(reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(Xin) + j * ld + r0));
#pragma unroll
              for (int k = 0; k < 4; ++k) ai[v][k] += w * (int)((word >> (8 * k)) & 1u);
            }
          }
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int64_t r0 = rbase + 128 * v;
        if (r0 >= B) continue;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (r0 + k < B && ((own_bits[v] >> (8 * k)) & 1u)) f2[v][k] += (long long)ai[v][k] + cp2;
      }
    } else {
    for (int eb = e0; eb < e1; eb += 32) {
      int mycol = col0;
      float myval = val0;
      if (eb != e0) {
        const int k = eb + lane;
        mycol = k < e1 ? __ldg(col + k) : 0;
        myval = k < e1 ? load_val(val, k, vt) : 0.0f;
      }
      const int cnt = min(32, e1 - eb);
#pragma unroll 4
      for (int q = 0; q < cnt; ++q) {
        const int64_t j = __shfl_sync(0xffffffffu, mycol, q);
        const float w = __shfl_sync(0xffffffffu, myval, q);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const int64_t r0 = rbase + 128 * v;
          if (r0 < B) {
            const float4 xv = load4<OPT>(Xin, j * ld + r0);
            acc[v].x = fmaf(w, xv.x, acc[v].x);
            acc[v].y = fmaf(w, xv.y, acc[v].y);
            acc[v].z = fmaf(w, xv.z, acc[v].z);
            acc[v].w = fmaf(w, xv.w, acc[v].w);
          }
        }
      }
    }
    }
#pragma unroll
    for (int v = 0; v < NV && MODE != EPI_EVAL; ++v) {
      const int64_t r0 = rbase + 128 * v;
      if (r0 >= B) continue;
      const int64_t idx = i * ld + r0;
      if (UPD) {
        float4 xn4, yn4;
        uint32_t bw = 0u;   // candidate bytes b = [x^{t+1} > 1/2], four restarts per word
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float x = comp(xo[v], k), y = comp(yo[v], k);
          const float gx = g_val(x, GK);
          const float d = comp(acc[v], k) + cpi + y * g_der(x, GK);
          float yn;
          const float xn = pdbo_update(x, y, d, gx, a.alpha, a.beta, a.delta, a.grad_tol, &yn);
          const bool live = r0 + k < B;   // padding restarts keep their zeros
          if (a.Gd) a.Gd[idx + k] = live ? d : 0.0f;
          set_comp(xn4, k, live ? xn : 0.0f);
          set_comp(yn4, k, live ? yn : 0.0f);
          bw |= (uint32_t)(live && xn > 0.5f) << (8 * k);
          if (SINGLE) set_comp(gs[v], k, comp(gs[v], k) + (live ? gx : 0.0f));
        }
        if (HINT) {
          if (a.Xm) st_policy4(a.Xm + idx, xn4, pol_first);
          if (OPT == OP_F32) st_policy4(static_cast<float*>(a.Xout) + idx, xn4, pol_last);
          else store4<OPT>(a.Xout, idx, xn4);
          if (!SINGLE) st_policy4(a.Y + idx, yn4, pol_first);
        } else {
          if (a.Xm) *reinterpret_cast<float4*>(a.Xm + idx) = xn4;
          store4<OPT>(a.Xout, idx, xn4);
          if (!SINGLE) *reinterpret_cast<float4*>(a.Y + idx) = yn4;
        }
        if (a.bits_out) *reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(a.bits_out) + idx) = bw;
      } else if (MODE == EPI_LAGR) {
        // Lagrangian of section 3.1: dL/dx = A x + c' + y (2x - 1), dL/dy = g(x), and the row's
        // share 1/2 x (A x) + c' x + y g(x) of L, summed per restart below
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int64_t r = r0 + k;
          if (r >= B) continue;
          const float x = comp(xo[v], k), y = comp(yo[v], k), g = comp(acc[v], k);
          const float gx = g_val(x, GK);
          const float sc = a.gout ? a.gout[r] : 1.0f;
          if (a.GX) a.GX[r * n + i] = sc * (g + cpi + y * g_der(x, GK));
          if (a.GY) a.GY[r * n + i] = sc * gx;
          set_comp(gs[v], k, comp(gs[v], k) + 0.5f * x * g + cpi * x + y * gx);
        }
      }
    }
    if (PIPE) {
      e0 = f0;
      e1 = f1;
      col0 = ncol;
      val0 = nval;
      cpi = ncpi;
      cp2 = ncp2;
      f0 = g0;
      f1 = g1;
    }
  }
  if ((UPD && SINGLE) || (MODE == EPI_LAGR && a.L)) {
    // single-constraint form: the block's warps cover the same restarts; their sums of g go to
    // shared memory and are added in warp order into this block's row of partial sums.
    // Lagrangian: the same per-block sums of the rows' shares of L, added to L[r] atomically
    __shared__ float redf[8][128 * NV];
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) *reinterpret_cast<float4*>(&redf[w][128 * v + 4 * lane]) = gs[v];
    __syncthreads();
    const int64_t rb = (int64_t)blockIdx.y * 128 * NV;
    for (int t = threadIdx.x; t < 128 * NV; t += blockDim.x) {
      float sum = 0.0f;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) sum += redf[q][t];
      if (rb + t >= B) continue;
      if (MODE == EPI_LAGR) atomicAdd(&a.L[rb + t], sum);
      else a.gpart[(int64_t)blockIdx.x * a.gpart_ld + rb + t] = sum;
    }
  }
  if (OBJ) {
    // the block's warps cover the same restarts: each warp's sums go to its row of shared
    // memory, a thread per restart adds the rows, then one atomic per restart per block
    __shared__ long long red[8][128 * NV];
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int k = 0; k < 4; ++k) red[w][128 * v + 4 * lane + k] = f2[v][k];
    __syncthreads();
    const int64_t rb = (int64_t)blockIdx.y * 128 * NV;
    for (int t = threadIdx.x; t < 128 * NV; t += blockDim.x) {
      long long sum = 0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) sum += red[q][t];
      if (rb + t < B && sum != 0) atomicAdd(&a.F2[rb + t], (unsigned long long)sum);
    }
  }
}

// Restarts per lane group: 256 per warp (NV = 2) when there are more than 128 restarts and the
// grid still holds two full waves of resident warps (152 SMs x 32 warps at 64 registers per
// thread), else 128 (NV = 1), which doubles the warps of a small graph.  Fewer registers and more
// warps in flight matter because this kernel is bound by memory latency.
static int csr_nv(int64_t n, int B) {
  if (B <= 128) return 1;
  const int64_t chunks2 = (B + 255) / 256;
  return n * chunks2 >= 2 * 152 * 32 ? 2 : 1;
}

int csr_partial_rows(int64_t n, int B) {
  const int NV = csr_nv(n, B);
  const int chunks = (B + 128 * NV - 1) / (128 * NV);
  return 152 * 8 / (chunks > 0 ? chunks : 1) + 1;
}

using CsrKernel = void (*)(const int32_t*, const int32_t*, const void*, int, EpiArgs);

template <int MODE, int NV, int OPT, bool PIPE, bool HINT = false>
static CsrKernel csr_kernel(bool single, bool ent) {
  if constexpr (HINT) {   // never with the single-constraint form
    return ent ? k_csr<MODE, NV, OPT, G_ENTROPY, false, PIPE, HINT> : k_csr<MODE, NV, OPT, G_QUAD, false, PIPE, HINT>;
  } else {
    if (single)
      return ent ? k_csr<MODE, NV, OPT, G_ENTROPY, true, PIPE, false> : k_csr<MODE, NV, OPT, G_QUAD, true, PIPE, false>;
    return ent ? k_csr<MODE, NV, OPT, G_ENTROPY, false, PIPE, false> : k_csr<MODE, NV, OPT, G_QUAD, false, PIPE, false>;
  }
}

// L2 capacity of the current device (queried once per device).
static int64_t device_l2_bytes() {
  static std::mutex mu;
  static std::vector<std::pair<int, int64_t>> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(mu);
  for (const auto& e : cache)
    if (e.first == dev) return e.second;
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  cache.push_back({dev, (int64_t)l2});
  return l2;
}

// Blocks of 256 threads of kernel k resident on the current device at once (queried once per
// kernel and device).
static int64_t csr_resident_blocks(CsrKernel k) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void*, int>, int64_t>> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152 * 4;
  std::lock_guard<std::mutex> lock(mu);
  for (const auto& e : cache)
    if (e.first.first == (const void*)k && e.first.second == dev) return e.second;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, 0) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return 152 * 4;
  }
  const int64_t r = std::max<int64_t>(1, (int64_t)per_sm * sms);
  cache.push_back({{(const void*)k, dev}, r});
  return r;
}

template <int MODE, int OPT>
static cudaError_t launch_csr_v(const int32_t* rowptr, const int32_t* col, const void* val, int vt,
                                const EpiArgs& a, int form, bool pdl, cudaStream_t s) {
  const bool single = MODE == EPI_UPDATE && a.mu != nullptr;
  const bool ent = MODE != EPI_EVAL && a.gkind == G_ENTROPY;
  // the update's form: chosen by the autotuner (CSR_FORM_*), or by the rule below.  The rule
  // strides pipelined rows when x and y (16 B per element) overflow three quarters of L2: measured
  // on a 4-regular graph, n = 20,000, B = 512, 44.1 -> 41.9 us per iteration, while the
  // L2-resident torus (n = 10,000) went 17.7 -> 18.2 us.  The single-constraint form keeps the
  // rule (its rows of partial sums are sized by it).
  // The streaming forms (CSR_FORM_*_STREAM) are the same with the L2 eviction priorities (HINT)
  // on the own state.
  const bool hint = MODE == EPI_UPDATE && !single && csr_form_streams(form);
  const int base = csr_form_base(form);
  const bool forced = MODE == EPI_UPDATE && !single && base >= CSR_FORM_ROW1 && base <= CSR_FORM_PIPE2;
  const int NV = forced ? (base == CSR_FORM_ROW1 ? 1 : 2) : csr_nv(a.n, a.B);
  const int64_t l2 = device_l2_bytes();
  const bool pipe = MODE == EPI_EVAL ||
                    (MODE == EPI_UPDATE && (forced ? base == CSR_FORM_PIPE2
                                                   : NV == 2 && l2 > 0 && (int64_t)a.n * a.B * 16 * 4 > l2 * 3));
  CsrKernel kern;
  if constexpr (MODE == EPI_EVAL) {
    // pipelined rows over one resident wave: the grid, and with it the closing atomics, stays bounded
    kern = NV == 1 ? csr_kernel<MODE, 1, OPT, true>(single, ent) : csr_kernel<MODE, 2, OPT, true>(single, ent);
  } else if constexpr (MODE == EPI_UPDATE) {
    if (hint)
      kern = pipe ? csr_kernel<MODE, 2, OPT, true, true>(single, ent)
                  : NV == 1 ? csr_kernel<MODE, 1, OPT, false, true>(single, ent)
                            : csr_kernel<MODE, 2, OPT, false, true>(single, ent);
    else
      kern = pipe ? csr_kernel<MODE, 2, OPT, true>(single, ent)
                  : NV == 1 ? csr_kernel<MODE, 1, OPT, false>(single, ent) : csr_kernel<MODE, 2, OPT, false>(single, ent);
  } else {
    kern = NV == 1 ? csr_kernel<MODE, 1, OPT, false>(single, ent) : csr_kernel<MODE, 2, OPT, false>(single, ent);
  }
  const int64_t chunks = (a.B + 128 * NV - 1) / (128 * NV);
  // the one-row update in blocks of four warps (finer-grained scheduling of its single wave:
  // 100 x 100 torus, B = 512, 16.48 -> 16.1 us per iteration); everything else in blocks of eight
  const int warps_per_block = (MODE == EPI_UPDATE && !pipe && !single) ? 4 : 8;
  int64_t want = (a.n + warps_per_block - 1) / warps_per_block;
  if (pipe) {
    // one wave of resident blocks: each warp strides over rows with its next rows' structure in
    // flight
    const int64_t wave = std::max<int64_t>(1, CSR_WAVES * csr_resident_blocks(kern) / chunks);
    if (want > wave) want = wave;
    // beside the resident form's cooperative launch, the evaluation keeps to about the eighth of
    // the SMs that launch leaves free
    if (MODE == EPI_EVAL && form == CSR_FORM_RESIDENT) want = std::min<int64_t>(want, std::max<int64_t>(1, wave / 8));
  }
  if (MODE != EPI_UPDATE || a.mu) {
    // bounds the closing atomics (evaluation) or the rows of partial sums (single-constraint form)
    const int64_t cap = csr_partial_rows(a.n, a.B);
    if (want > cap) want = cap;
  }
  if (want > 65535) want = 65535;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)want, (unsigned)chunks);
  cfg.blockDim = dim3(32 * warps_per_block);
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, rowptr, col, val, vt, a);
}

cudaError_t launch_csr(const int32_t* rowptr, const int32_t* col, const void* val, int val_type,
                       const EpiArgs& a, int op_type, int mode, bool pdl, cudaStream_t s, int form) {
  if (a.ld % 8 != 0) return cudaErrorInvalidValue;  // vector accesses need 16-byte rows
  if (mode == EPI_UPDATE) {
    return op_type == OP_F32 ? launch_csr_v<EPI_UPDATE, OP_F32>(rowptr, col, val, val_type, a, form, pdl, s)
                             : launch_csr_v<EPI_UPDATE, OP_BF16>(rowptr, col, val, val_type, a, form, pdl, s);
  }
  if (mode == EPI_EVAL) {
    return launch_csr_v<EPI_EVAL, OP_U8>(rowptr, col, val, val_type, a, form, pdl, s);   // candidate bytes
  }
  if (mode == EPI_LAGR) {
    return op_type == OP_F32 ? launch_csr_v<EPI_LAGR, OP_F32>(rowptr, col, val, val_type, a, 0, pdl, s)
                             : launch_csr_v<EPI_LAGR, OP_BF16>(rowptr, col, val, val_type, a, 0, pdl, s);
  }
  return cudaErrorInvalidValue;
}

// ---- resident form (CSR_FORM_RESIDENT) -----------------------------------------------------------
// Small graphs whose state fits in the SMs' shared memory: G = csr_res_grid(n, SMs) cooperative
// CTAs, one per SM (an eighth of the SMs stays free, for the previous block's evaluation on a graph
// branch beside the launch); CTA b owns the contiguous rows [b n / G, (b+1) n / G) and keeps their
// x, y and structure (local row offsets, columns, weights) in shared memory for all the iterations
// of a launch.  An iteration gathers the
// neighbours' operand x^t from L2 (bypassing L1: the two operand buffers alternate within the
// launch), applies the same fused update as k_csr in the same order of operations (bit-identical),
// writes the rows' x^{t+1} operand to global memory and meets the other CTAs at the grid barrier.
// x and y go back to global memory at the end of the launch.  What it saves against one launch
// per iteration is the kernel boundary and every load and store of the own state.
constexpr int RES_THREADS = 1024;

struct ResParams {
  const int32_t* rowptr;
  const int32_t* col;
  const void* val;
  int vt;
  EpiArgs a;               // Xin / Xout / bits_out are taken from xop / bits_last
  void* xop[2];            // iteration j reads xop[(x0 + j) & 1] and writes the other one
  void* bits_last;         // candidate bytes written by the last iteration (null: none)
  unsigned int* gbar;      // grid barrier [arrivals, exits, abort] (iters > 1)
  int x0, iters;
  int rows_max, nnz_max, Bp;   // shared-memory extents: rows, nonzeros per CTA, restarts per row
  int eval_last;           // after the last iteration: the exact objective of its candidates into a.F2
  uint64_t timeout_ns;     // per iteration
};

template <int OPT>
__device__ __forceinline__ float4 ldcg4(const void* p, int64_t idx) {
  if (OPT == OP_F32) return __ldcg(reinterpret_cast<const float4*>(static_cast<const float*>(p) + idx));
  const uint2 raw = __ldcg(reinterpret_cast<const uint2*>(static_cast<const __nv_bfloat16*>(p) + idx));
  const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
  const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
  return make_float4(__low2float(lo), __high2float(lo), __low2float(hi), __high2float(hi));
}

size_t res_smem_bytes(int rows_max, int nnz_max, int Bp) {
  // x, y [rows][Bp] FP32; 2F per restart (int64) for the fused evaluation; row offsets, columns,
  // weights
  return (size_t)rows_max * Bp * 8 + (size_t)Bp * 8 + (size_t)(rows_max + 1) * 4 + (size_t)nnz_max * 8 + 16;
}

template <int OPT, int GK>
__global__ void __launch_bounds__(RES_THREADS, 1) k_csr_res(const __grid_constant__ ResParams P) {
  extern __shared__ __align__(16) uint8_t res_smem[];
  __shared__ int s_stop;
  const EpiArgs& a = P.a;
  const int n = a.n, B = a.B, Bp = P.Bp;
  const int64_t ld = a.ld;
  const int G = (int)gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (int)(blockDim.x >> 5);
  const int r_begin = (int)((int64_t)blockIdx.x * n / G), r_end = (int)((int64_t)(blockIdx.x + 1) * n / G);
  const int R = r_end - r_begin;
  float* xs = reinterpret_cast<float*>(res_smem);                 // [rows_max][Bp]
  float* ys = xs + (size_t)P.rows_max * Bp;                       // [rows_max][Bp]
  long long* f2s = reinterpret_cast<long long*>(ys + (size_t)P.rows_max * Bp);   // [Bp]
  int* rp = reinterpret_cast<int*>(f2s + Bp);                     // [rows_max + 1]
  int* cs = rp + P.rows_max + 1;                                  // [nnz_max]
  float* wv = reinterpret_cast<float*>(cs + P.nnz_max);           // [nnz_max]

  // structure and state of the owned rows
  const int e_begin = __ldg(P.rowptr + r_begin);
  const int e_count = __ldg(P.rowptr + r_end) - e_begin;
  for (int t = tid; t <= R; t += blockDim.x) rp[t] = __ldg(P.rowptr + r_begin + t) - e_begin;
  for (int t = tid; t < e_count; t += blockDim.x) {
    cs[t] = __ldg(P.col + e_begin + t);
    wv[t] = load_val(P.val, e_begin + t, P.vt);
  }
  const float* xsrc = a.Xm ? a.Xm : static_cast<const float*>(P.xop[P.x0]);   // FP32 operand: x itself
  const int q4 = Bp / 4;
  for (int t = tid; t < R * q4; t += blockDim.x) {
    const int il = t / q4, r = 4 * (t % q4);
    const int64_t idx = (int64_t)(r_begin + il) * ld + r;
    *reinterpret_cast<float4*>(xs + (size_t)il * Bp + r) = __ldcg(reinterpret_cast<const float4*>(xsrc + idx));
    *reinterpret_cast<float4*>(ys + (size_t)il * Bp + r) = __ldcg(reinterpret_cast<const float4*>(a.Y + idx));
  }
  if (tid == 0) s_stop = 0;
  __syncthreads();

  const int chunks = (B + 127) / 128;
  const int items = R * chunks;
  for (int it = 0; it < P.iters; ++it) {
    const int w = (P.x0 + it) & 1;
    const void* xin = P.xop[w];
    void* xout = P.xop[w ^ 1];
    uint8_t* bits = it + 1 == P.iters ? static_cast<uint8_t*>(P.bits_last) : nullptr;
    if (it > 0) {
      // x^{it} is complete once every CTA has arrived after iteration it - 1
      if (tid == 0) {
        const bool ok = grid_wait(P.gbar, (unsigned int)it * (unsigned int)G, globaltimer_ns() + P.timeout_ns);
        if (!ok) {
          atomicOr(a.err, ERR_TIMEOUT);
          atomicExch(P.gbar + 2, 1u);
        }
        s_stop = ok ? 0 : 1;
      }
      __syncthreads();
      if (s_stop) break;
    }
    for (int item = warp; item < items; item += nw) {
      const int il = item / chunks;
      const int r0 = (item % chunks) * 128 + 4 * lane;
      if (r0 >= B) continue;
      const int64_t i = r_begin + il;
      const float cpi = a.cp[i];
      const int eb = rp[il], ee = rp[il + 1];
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
      for (int e = eb; e < ee; ++e) {
        const int64_t j = cs[e];
        const float wgt = wv[e];
        const float4 xv = ldcg4<OPT>(xin, j * ld + r0);
        acc.x = fmaf(wgt, xv.x, acc.x);
        acc.y = fmaf(wgt, xv.y, acc.y);
        acc.z = fmaf(wgt, xv.z, acc.z);
        acc.w = fmaf(wgt, xv.w, acc.w);
      }
      float* xp = xs + (size_t)il * Bp + r0;
      float* yp = ys + (size_t)il * Bp + r0;
      const float4 xo = *reinterpret_cast<const float4*>(xp);
      const float4 yo = *reinterpret_cast<const float4*>(yp);
      const int64_t idx = i * ld + r0;
      float4 xn4, yn4;
      uint32_t bw = 0u;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float x = comp(xo, k), y = comp(yo, k);
        const float gx = g_val(x, GK);
        const float d = comp(acc, k) + cpi + y * g_der(x, GK);
        float yn;
        const float xn = pdbo_update(x, y, d, gx, a.alpha, a.beta, a.delta, a.grad_tol, &yn);
        const bool live = r0 + k < B;   // padding restarts keep their zeros
        if (a.Gd) a.Gd[idx + k] = live ? d : 0.0f;
        set_comp(xn4, k, live ? xn : 0.0f);
        set_comp(yn4, k, live ? yn : 0.0f);
        bw |= (uint32_t)(live && xn > 0.5f) << (8 * k);
      }
      *reinterpret_cast<float4*>(xp) = xn4;
      *reinterpret_cast<float4*>(yp) = yn4;
      store4<OPT>(xout, idx, xn4);
      if (bits) *reinterpret_cast<uint32_t*>(bits + idx) = bw;
    }
    if (it + 1 < P.iters) {
      // publish this CTA's rows of x^{it+1}: the barrier orders every thread's stores before
      // thread 0's release
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        red_release_gpu_add(P.gbar, 1u);
      }
    }
  }
  if (P.eval_last) {
    // The exact objective of the last iteration's candidates, as the evaluation kernel computes it
    // (integer weights times candidate bytes, 2F = sum_i b_i (sum_j A_ij b_j + 2 c'_i)), once every
    // CTA's candidates are written: one more arrival at the grid barrier.
    __syncthreads();
    if (tid == 0) {
      bool ok = s_stop == 0;
      if (ok) {
        __threadfence();
        red_release_gpu_add(P.gbar, 1u);
        ok = grid_wait(P.gbar, (unsigned int)P.iters * (unsigned int)G, globaltimer_ns() + P.timeout_ns);
        if (!ok) {
          atomicOr(a.err, ERR_TIMEOUT);
          atomicExch(P.gbar + 2, 1u);
        }
      }
      s_stop = ok ? 0 : 1;
    }
    for (int t = tid; t < Bp; t += blockDim.x) f2s[t] = 0;
    __syncthreads();
    if (!s_stop) {
      const uint8_t* cand = static_cast<const uint8_t*>(P.bits_last);
      for (int item = warp; item < items; item += nw) {
        const int il = item / chunks;
        const int r0 = (item % chunks) * 128 + 4 * lane;
        if (r0 >= B) continue;
        const int64_t i = r_begin + il;
        const long long cp2 = 2 * (long long)a.cp64[i];
        int ai[4] = {0, 0, 0, 0};
        for (int e = rp[il]; e < rp[il + 1]; ++e) {
          const int64_t j = cs[e];
          const int wint = __float2int_rn(wv[e]);
          const uint32_t word = __ldcg(reinterpret_cast<const unsigned int*>(cand + j * ld + r0));
#pragma unroll
          for (int k = 0; k < 4; ++k) ai[k] += wint * (int)((word >> (8 * k)) & 1u);
        }
        const float* xp = xs + (size_t)il * Bp + r0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (r0 + k < B && xp[k] > 0.5f) {   // the row's own candidate, as the update wrote it
            const long long v = (long long)ai[k] + cp2;
            if (v != 0) atomicAdd(reinterpret_cast<unsigned long long*>(&f2s[r0 + k]), (unsigned long long)v);
          }
        }
      }
      __syncthreads();
      for (int t = tid; t < B; t += blockDim.x)
        if (f2s[t] != 0) atomicAdd(&a.F2[t], (unsigned long long)f2s[t]);
    }
  }
  // the state goes back to global memory (x in the FP32 operand buffer already when there is no
  // master copy)
  __syncthreads();
  for (int t = tid; t < R * q4; t += blockDim.x) {
    const int il = t / q4, r = 4 * (t % q4);
    const int64_t idx = (int64_t)(r_begin + il) * ld + r;
    if (a.Xm) *reinterpret_cast<float4*>(a.Xm + idx) = *reinterpret_cast<const float4*>(xs + (size_t)il * Bp + r);
    *reinterpret_cast<float4*>(a.Y + idx) = *reinterpret_cast<const float4*>(ys + (size_t)il * Bp + r);
  }
  if ((P.iters > 1 || P.eval_last) && tid == 0) {
    // the last CTA out restores the barrier words for the next launch (the abort word stays
    // raised after a failure; the host clears it when it reads the error)
    if (atomicAdd(P.gbar + 1, 1u) == gridDim.x - 1) {
      atomicExch(P.gbar, 0u);
      atomicExch(P.gbar + 1, 0u);
    }
  }
}

// Whether the resident form serves this problem: the update with one dual per coordinate, and
// the largest CTA's rows and nonzeros fit in shared memory.  grid: CTAs (one per SM, at most n).
int csr_res_grid(int64_t n, int sms) {
  const int64_t g = std::max(1, sms - sms / 8);   // an eighth of the SMs stays free for the evaluation beside it
  return (int)std::max<int64_t>(1, std::min<int64_t>(n, g));
}

bool csr_res_shape(int64_t n, int B, int sms, int nnz_max, int* grid, size_t* smem) {
  if (n < 1 || sms < 1) return false;
  const int G = csr_res_grid(n, sms);
  const int rows_max = (int)((n + G - 1) / G);
  const int Bp = (B + 3) / 4 * 4;
  const size_t bytes = res_smem_bytes(rows_max, nnz_max, Bp);
  if (bytes > 200 * 1024 + 16) return false;
  *grid = G;
  *smem = bytes;
  return true;
}

cudaError_t launch_csr_res(const int32_t* rowptr, const int32_t* col, const void* val, int val_type, const EpiArgs& a,
                           int op_type, int which_x, void* const xop[2], int iters, bool eval_last, int nnz_max,
                           int sms, unsigned int* gbar, uint64_t timeout_ns, cudaStream_t s) {
  int G = 0;
  size_t smem = 0;
  if (a.mu || a.ld % 8 != 0 || iters < 1 || ((iters > 1 || eval_last) && !gbar) || which_x < 0 || which_x > 1 ||
      (eval_last && (!a.bits_out || !a.F2 || !a.cp64)) || !csr_res_shape(a.n, a.B, sms, nnz_max, &G, &smem))
    return cudaErrorInvalidValue;
  ResParams P;
  memset(&P, 0, sizeof(P));
  P.rowptr = rowptr;
  P.col = col;
  P.val = val;
  P.vt = val_type;
  P.a = a;
  P.xop[0] = xop[0];
  P.xop[1] = xop[1];
  P.bits_last = a.bits_out;
  P.gbar = gbar;
  P.x0 = which_x;
  P.iters = iters;
  P.rows_max = (int)((a.n + G - 1) / G);
  P.nnz_max = nnz_max;
  P.Bp = (a.B + 3) / 4 * 4;
  P.eval_last = eval_last ? 1 : 0;
  P.timeout_ns = timeout_ns;
  const bool ent = a.gkind == G_ENTROPY;
  void (*kern)(const ResParams) = op_type == OP_F32 ? (ent ? k_csr_res<OP_F32, G_ENTROPY> : k_csr_res<OP_F32, G_QUAD>)
                                                    : (ent ? k_csr_res<OP_BF16, G_ENTROPY> : k_csr_res<OP_BF16, G_QUAD>);
  static PerDevice per_device;   // the shared-memory limit of the four kernels, once per device
  const cudaError_t e = per_device.once([] {
    const int lim = 200 * 1024 + 16;
    cudaError_t r = cudaFuncSetAttribute(k_csr_res<OP_F32, G_QUAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_csr_res<OP_F32, G_ENTROPY>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_csr_res<OP_BF16, G_QUAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_csr_res<OP_BF16, G_ENTROPY>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    return r;
  });
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G);
  cfg.blockDim = dim3(RES_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  // cooperative: the CTAs wait for one another at the grid barrier, so the launch must be
  // scheduled whole
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeCooperative;
  attr.val.cooperative = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = (iters > 1 || eval_last) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, P);
}

}  // namespace sbo
