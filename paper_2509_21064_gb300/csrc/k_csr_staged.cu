// Sparse form, staged: the CSR SpMM G = A X fused with the PDBO update (Algorithm 1), with every
// row's operands brought into shared memory by 1-D bulk copies (cp.async.bulk, the TMA engine)
// instead of register loads, so that many rows' worth of bytes are in flight per SM at once.
//
// State is variable-major ([i * ld + r], ld a multiple of 8), as for k_csr.  A CTA owns a
// contiguous range of rows and a chunk of up to CS_RC restarts (blockIdx.y).  Warp 0 produces:
// for each row, in order, it claims a stage of the shared-memory ring and copies the row's own
// x and y (FP32, cnt restarts each) and the operand rows x_j of up to D neighbours j into it,
// completing on the stage's mbarrier; a row with more than D neighbours continues in the next
// stage(s).  The column indices and weights of 32 rows at a time are read by the warp's lanes
// (one row each) into shared memory before their stages are issued.  Warps 1..4 consume: 128
// threads x 4 consecutive restarts cover the chunk; each thread sums w_j x_j over the stage's
// neighbours into registers, releases the stage, and after a row's last stage applies the update
// and writes x^{t+1} (FP32 master and / or operand), y, the candidate bytes and, when asked, the
// gradient, with coalesced 16-byte (FP32) stores.
// Every mbarrier wait is bounded by a globaltimer budget: on expiry the kernel raises
// ERR_TIMEOUT, waits (bounded) for the copies it issued and returns.
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "tc_common.cuh"

namespace sbo {
namespace {

constexpr int CS_CONS_WARPS = 4;                    // consumer warps
constexpr int CS_THREADS = 32 * (1 + CS_CONS_WARPS);
constexpr int CS_RC = 4 * 32 * CS_CONS_WARPS;       // restarts per chunk: 4 per consumer thread (512)
constexpr int CS_DMAX = 16;                         // neighbour slots per stage at most
constexpr int CS_BATCH = 32;                        // rows whose structure the producer reads at once
constexpr int CS_SMEM_BUDGET = 110 * 1024;          // two CTAs per SM

struct StageHdr {
  int row;
  int nnb;       // neighbours in this stage
  int flags;     // 1: first stage of the row (own x, y present), 2: last stage of the row
  float cp;      // c'_row
  float w[CS_DMAX];
};

struct CsParams {
  const int32_t* rowptr;
  const int32_t* col;
  const void* val;
  int vt;            // weight type: 0 FP32, 1 BF16, 2 E4M3
  EpiArgs a;
  int rows_per_cta;
  int D;             // neighbour slots per stage
  int S;             // stages
  int rc;            // chunk width used for the stage layout (<= CS_RC, multiple of 8)
  uint32_t stage_bytes;
  uint64_t timeout_ns;
};

__device__ __forceinline__ float cs_weight(const void* val, int64_t e, int vt) {
  if (vt == 0) return __ldg(static_cast<const float*>(val) + e);
  if (vt == 1) return __bfloat162float(static_cast<const __nv_bfloat16*>(val)[e]);
  __nv_fp8_e4m3 q;
  q.__x = static_cast<const __nv_fp8_storage_t*>(val)[e];
  return static_cast<float>(q);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

template <int OPT>
__device__ __forceinline__ float4 lds_op4(const uint8_t* p) {
  if (OPT == OP_F32) return *reinterpret_cast<const float4*>(p);
  const uint2 raw = *reinterpret_cast<const uint2*>(p);
  const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
  const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
  return make_float4(__low2float(lo), __high2float(lo), __low2float(hi), __high2float(hi));
}

template <int OPT, int GK>
__global__ void __launch_bounds__(CS_THREADS, 2) k_csr_staged(CsParams P) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  const int S = P.S;
  uint64_t* full_bar = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty_bar = full_bar + S;
  int* abort_flag = reinterpret_cast<int*>(empty_bar + S);
  int* scol = abort_flag + 4;                                     // [CS_BATCH][CS_DMAX]
  float* sval = reinterpret_cast<float*>(scol + CS_BATCH * CS_DMAX);
  float* scp = sval + CS_BATCH * CS_DMAX;                         // [CS_BATCH]
  StageHdr* hdr = reinterpret_cast<StageHdr*>(scp + CS_BATCH);
  uint8_t* data = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(hdr + S) + 127) & ~uintptr_t(127));

  const EpiArgs& a = P.a;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ld = a.ld;
  const int64_t r0 = (int64_t)blockIdx.y * CS_RC;
  const int cnt = (int)(ld - r0 < CS_RC ? ld - r0 : (int64_t)CS_RC);              // restarts copied per row (multiple of 8)
  constexpr int OPB = OPT == OP_F32 ? 4 : 2;
  const uint32_t own_bytes = (uint32_t)cnt * 4u;
  const uint32_t nb_bytes = (uint32_t)cnt * OPB;
  const uint32_t off_y = (uint32_t)P.rc * 4u, off_nb = 2u * (uint32_t)P.rc * 4u, nb_pitch = (uint32_t)P.rc * OPB;
  const int64_t i_begin = (int64_t)blockIdx.x * P.rows_per_cta;
  const int64_t i_end = i_begin + P.rows_per_cta < (int64_t)a.n ? i_begin + P.rows_per_cta : (int64_t)a.n;
  const uint64_t deadline = globaltimer_ns() + P.timeout_ns;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), CS_CONS_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  const volatile int* vabort = abort_flag;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    const float* xown_src = a.Xm ? a.Xm : static_cast<const float*>(a.Xin);
    const uint8_t* xop = static_cast<const uint8_t*>(a.Xin);
    int stage = 0;
    uint32_t phase = 0;
    uint32_t issued_lo = 0, issued_par = 0;        // stages with copies issued (for the drain), < 32 stages
    bool ok = true;
    // the structure is constant over the run: the first batch is read before waiting on the
    // previous kernel (programmatic dependent launch), the state after the wait
    int e0 = 0, e1 = 0;
    auto load_batch = [&](int64_t ib) {
      const int64_t i = ib + lane;
      e0 = e1 = 0;
      if (i < i_end) {
        e0 = __ldg(P.rowptr + i);
        e1 = __ldg(P.rowptr + i + 1);
        scp[lane] = a.cp[i];
      }
      const int deg = e1 - e0;
#pragma unroll 4
      for (int m = 0; m < CS_DMAX; ++m) {
        if (m < deg) {
          scol[lane * CS_DMAX + m] = __ldg(P.col + e0 + m);
          sval[lane * CS_DMAX + m] = cs_weight(P.val, e0 + m, P.vt);
        }
      }
      __syncwarp();
    };
    if (i_begin < i_end) load_batch(i_begin);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    for (int64_t ib = i_begin; ok && ib < i_end; ib += CS_BATCH) {
      if (ib != i_begin) load_batch(ib);
      const int rows = (int)(i_end - ib < CS_BATCH ? i_end - ib : (int64_t)CS_BATCH);
      for (int j = 0; ok && j < rows; ++j) {
        const int64_t i = ib + j;
        const int rj0 = __shfl_sync(0xffffffffu, e0, j);
        const int deg = __shfl_sync(0xffffffffu, e1, j) - rj0;
        for (int kb = 0; kb == 0 || kb < deg; kb += P.D) {
          const int nnb = max(0, min(P.D, deg - kb));
          const bool first = kb == 0, last = kb + P.D >= deg;
          int got = 1;
          if (lane == 0) got = mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1u, deadline, vabort) ? 1 : 0;
          if (!__shfl_sync(0xffffffffu, got, 0)) { ok = false; break; }
          StageHdr& h = hdr[stage];
          int c = 0;
          if (lane < nnb) {
            const int m = kb + lane;
            float wv;
            if (m < CS_DMAX) {
              c = scol[j * CS_DMAX + m];
              wv = sval[j * CS_DMAX + m];
            } else {                         // beyond the registers' share: read directly
              c = __ldg(P.col + rj0 + m);
              wv = cs_weight(P.val, rj0 + m, P.vt);
            }
            h.w[lane] = wv;
          }
          if (lane == 0) {
            h.row = (int)i;
            h.nnb = nnb;
            h.flags = (first ? 1 : 0) | (last ? 2 : 0);
            h.cp = scp[j];
          }
          __syncwarp();
          const uint32_t fb = smem_u32(&full_bar[stage]);
          uint8_t* sd = data + (size_t)stage * P.stage_bytes;
          if (lane == 0) mbar_expect_tx(fb, (first ? 2u * own_bytes : 0u) + (uint32_t)nnb * nb_bytes);
          __syncwarp();
          if (lane < nnb)
            bulk_g2s(smem_u32(sd + off_nb + lane * nb_pitch), xop + ((int64_t)c * ld + r0) * OPB, nb_bytes, fb);
          if (first && lane == 30) bulk_g2s(smem_u32(sd), xown_src + i * ld + r0, own_bytes, fb);
          if (first && lane == 31) bulk_g2s(smem_u32(sd + off_y), a.Y + i * ld + r0, own_bytes, fb);
          issued_lo |= 1u << stage;
          issued_par = (issued_par & ~(1u << stage)) | (phase << stage);
          if (++stage == S) { stage = 0; phase ^= 1u; }
        }
      }
      __syncwarp();
    }
    if (lane == 0) {
      if (!ok) {
        atomicOr(a.err, ERR_TIMEOUT);
        *abort_flag = 1;
      }
      // every copy issued completes on its full barrier before the CTA may exit (the consumers
      // wait for them too, unless they gave up)
      const uint64_t dl2 = globaltimer_ns() + 200000000ull;
      const int zero = 0;
      for (int s = 0; s < S; ++s)
        if (issued_lo & (1u << s)) mbar_wait(smem_u32(&full_bar[s]), (issued_par >> s) & 1u, dl2, &zero);
    }
  } else {
    // ---------------------------------------------------------------- consumers
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int t = threadIdx.x - 32;                  // 0..127: restarts r0 + 4t .. +3
    const bool act = 4 * t < cnt;
    int stage = 0;
    uint32_t phase = 0;
    float4 xo = make_float4(0.f, 0.f, 0.f, 0.f), yo = xo, acc = xo;
    int64_t done = 0;
    const int64_t rows_total = i_end > i_begin ? i_end - i_begin : 0;
    while (done < rows_total) {
      if (!mbar_wait_warp(smem_u32(&full_bar[stage]), phase, deadline, vabort, lane)) {
        if (lane == 0) {
          atomicOr(a.err, ERR_TIMEOUT);
          *abort_flag = 1;
        }
        break;
      }
      const StageHdr& h = hdr[stage];
      const int flags = h.flags, nnb = h.nnb;
      const int64_t i = h.row;
      const float cpi = h.cp;
      const uint8_t* sd = data + (size_t)stage * P.stage_bytes;
      // a stage row holds cnt restarts (rc slots): threads past cnt read nothing
      if (act && (flags & 1)) {
        xo = *reinterpret_cast<const float4*>(sd + 16 * t);
        yo = *reinterpret_cast<const float4*>(sd + off_y + 16 * t);
        acc = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      for (int k = 0; act && k < nnb; ++k) {
        const float w = h.w[k];
        const float4 v = lds_op4<OPT>(sd + off_nb + k * nb_pitch + 4 * OPB * t);
        acc.x = fmaf(w, v.x, acc.x);
        acc.y = fmaf(w, v.y, acc.y);
        acc.z = fmaf(w, v.z, acc.z);
        acc.w = fmaf(w, v.w, acc.w);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty_bar[stage]));
      if (++stage == S) { stage = 0; phase ^= 1u; }
      if (!(flags & 2)) continue;
      ++done;
      if (!act) continue;
      const int64_t r = r0 + 4 * t;
      const int64_t idx = i * ld + r;
      float4 xn4, yn4, b4, d4;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float x = k == 0 ? xo.x : k == 1 ? xo.y : k == 2 ? xo.z : xo.w;
        const float y = k == 0 ? yo.x : k == 1 ? yo.y : k == 2 ? yo.z : yo.w;
        const float g = k == 0 ? acc.x : k == 1 ? acc.y : k == 2 ? acc.z : acc.w;
        const float d = g + cpi + y * g_der(x, GK);
        float yn;
        const float xn = pdbo_update(x, y, d, g_val(x, GK), a.alpha, a.beta, a.delta, a.grad_tol, &yn);
        const bool live = r + k < a.B;                 // padding restarts keep their zeros
        const float xv = live ? xn : 0.0f, yv = live ? yn : 0.0f, bv = (live && xn > 0.5f) ? 1.0f : 0.0f;
        const float dv = live ? d : 0.0f;
        if (k == 0) { xn4.x = xv; yn4.x = yv; b4.x = bv; d4.x = dv; }
        else if (k == 1) { xn4.y = xv; yn4.y = yv; b4.y = bv; d4.y = dv; }
        else if (k == 2) { xn4.z = xv; yn4.z = yv; b4.z = bv; d4.z = dv; }
        else { xn4.w = xv; yn4.w = yv; b4.w = bv; d4.w = dv; }
      }
      if (a.Xm) *reinterpret_cast<float4*>(a.Xm + idx) = xn4;
      if (OPT == OP_F32) {
        *reinterpret_cast<float4*>(static_cast<float*>(a.Xout) + idx) = xn4;
      } else {
        __nv_bfloat162 lo = __floats2bfloat162_rn(xn4.x, xn4.y), hi = __floats2bfloat162_rn(xn4.z, xn4.w);
        uint2 raw;
        raw.x = *reinterpret_cast<uint32_t*>(&lo);
        raw.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(a.Xout) + idx) = raw;
      }
      *reinterpret_cast<float4*>(a.Y + idx) = yn4;
      if (a.bits_out)
        *reinterpret_cast<uchar4*>(static_cast<uint8_t*>(a.bits_out) + idx) =
            make_uchar4((unsigned char)b4.x, (unsigned char)b4.y, (unsigned char)b4.z, (unsigned char)b4.w);
      if (a.Gd) *reinterpret_cast<float4*>(a.Gd + idx) = d4;
    }
  }
}

using CsKernel = void (*)(CsParams);

CsKernel cs_kernel(int op_type, int gkind) {
  if (op_type == OP_F32) return gkind == G_ENTROPY ? k_csr_staged<OP_F32, G_ENTROPY> : k_csr_staged<OP_F32, G_QUAD>;
  return gkind == G_ENTROPY ? k_csr_staged<OP_BF16, G_ENTROPY> : k_csr_staged<OP_BF16, G_QUAD>;
}

}  // namespace

// Shape of the staged form for a graph whose largest row has max_deg neighbours: neighbour slots
// per stage (D), stages (S), chunk width (rc) and shared-memory bytes; false when fewer than four
// stages fit the budget.
bool csr_staged_shape(int64_t ld, int op_type, int max_deg, int* D, int* S, int* rc, size_t* smem) {
  const int w = (int)std::min<int64_t>(CS_RC, ld);
  const int opb = op_type == OP_F32 ? 4 : 2;
  const int d = std::max(1, std::min(max_deg, 8));
  const size_t stage = ((size_t)2 * w * 4 + (size_t)d * w * opb + 127) / 128 * 128;
  const size_t fixed = 16 * 32 /* two barrier arrays, at most 32 stages */ + 16 + (size_t)CS_BATCH * (CS_DMAX * 8 + 4) +
                       32 * sizeof(StageHdr) + 128;
  const int s = (int)std::min<size_t>(16, (CS_SMEM_BUDGET - fixed) / stage);
  if (s < 4) return false;
  *D = d;
  *S = s;
  *rc = w;
  *smem = 2 * 8 * (size_t)s + 16 + (size_t)CS_BATCH * (CS_DMAX * 8 + 4) + (size_t)s * sizeof(StageHdr) + 128 +
          (size_t)s * stage;
  return true;
}

cudaError_t launch_csr_staged(const int32_t* rowptr, const int32_t* col, const void* val, int val_type,
                              const EpiArgs& a, int op_type, int max_deg, int sms, bool pdl, uint64_t timeout_ns,
                              cudaStream_t s) {
  if (a.ld % 8 != 0 || a.mu != nullptr) return cudaErrorInvalidValue;
  int D = 0, S = 0, rc = 0;
  size_t smem = 0;
  if (!csr_staged_shape(a.ld, op_type, max_deg, &D, &S, &rc, &smem)) return cudaErrorInvalidValue;
  CsKernel kern = cs_kernel(op_type, a.gkind);
  static PerDevice attrs[4];
  const int which = (op_type == OP_F32 ? 0 : 2) + (a.gkind == G_ENTROPY ? 1 : 0);
  cudaError_t e = attrs[which].once([&] {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CS_SMEM_BUDGET);
  });
  if (e != cudaSuccess) return e;
  const int64_t chunks = (a.ld + CS_RC - 1) / CS_RC;
  // two resident CTAs per SM in total, the rows split evenly over the CTAs of a chunk
  int64_t ctas = std::max<int64_t>(1, 2 * (int64_t)sms / chunks);
  ctas = std::min<int64_t>(ctas, (a.n + 7) / 8);
  const int64_t rows_per = (a.n + ctas - 1) / ctas;
  ctas = (a.n + rows_per - 1) / rows_per;
  CsParams P;
  P.rowptr = rowptr;
  P.col = col;
  P.val = val;
  P.vt = val_type;
  P.a = a;
  P.rows_per_cta = (int)rows_per;
  P.D = D;
  P.S = S;
  P.rc = rc;
  P.stage_bytes = (uint32_t)(((size_t)2 * rc * 4 + (size_t)D * rc * (op_type == OP_F32 ? 4 : 2) + 127) / 128 * 128);
  P.timeout_ns = timeout_ns;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas, (unsigned)chunks);
  cfg.blockDim = dim3(CS_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, P);
}

}  // namespace sbo
