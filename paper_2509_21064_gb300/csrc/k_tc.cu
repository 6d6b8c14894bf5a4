// Dense contraction on the 5th-generation tensor cores (tcgen05, sm_103a) with the PDBO
// epilogue fused onto the accumulator tile.
//
//   D[i][r] = sum_k A[i][k] * Xb[r][k]           (= (A x_r)_i; A is n x n, Xb is B x n, BF16)
//
// A and Xb are both K-major, so one 128-byte swizzle row holds 64 consecutive k of one row
// (TMA box 64 x rows, SWIZZLE_128B), which is the canonical K-major SW128 layout of a UMMA
// shared-memory descriptor (8-row atoms of 1024 B, SBO = 1024 B).
//
// Persistent, warp-specialised CTA (one per SM, 384 threads):
//   warp 0      TMA producer: A tile 128 x 64 and X tile tile_n x 64 per stage, mbarrier ring
//   warp 1      TMEM allocator and single-thread MMA issuer (tcgen05.mma.cta_group::1.kind::f16,
//               M=128, N=tile_n, K=16, FP32 accumulation in TMEM)
//   warps 4-11  two epilogue warpgroups (half of the columns each): tcgen05.ld of the
//               128 x tile_n accumulator (lane = row i), one PDBO iteration / exact objective /
//               Lagrangian per element, loads batched per 32-column chunk, coalesced along i
// TMEM holds two accumulators (2 x tile_n columns) so the epilogue of one tile overlaps the
// main loop of the next.  Tiles are visited m-major with the restart tiles of one row block
// adjacent, so CTAs that share an A row block run together and A is read from HBM ~once.
// Every mbarrier wait is bounded by a globaltimer budget: on expiry the kernel raises
// ERR_TIMEOUT, drains its own copies and MMAs (bounded too), frees TMEM and returns.
#include <cudaTypedefs.h>

#include <mutex>

#include "tc_common.cuh"

namespace sbo {

constexpr int TC_SMEM_BUDGET = 196 * 1024;
constexpr int TC_MIN_KB_PER_SPLIT = 8;  // a split-K unit covers at least 8 k-blocks (512 of K)
constexpr int TC_THREADS = 384;   // warps 0-3: producer, MMA, 2 idle; warps 4-11: epilogue

struct TcParams {
  CUtensorMap mapA;
  CUtensorMap mapX;
  EpiArgs epi;
  int n, m_tiles, n_tiles, num_tiles, kblocks;
  int dp_tiles;    // tiles computed whole, round-robin over the grid
  int splits;      // split-K factor of the remaining (tail) tiles
  int sk_units;    // (num_tiles - dp_tiles) * splits, one per CTA
  float* ws;       // split-K partial tiles [sk_units][BN][128] (scratch)
  int* counters;   // arrivals per (tail tile, epilogue warp slice), zero between launches (scratch)
  uint64_t timeout_ns;
  // grouped launch over several instances (the maps and epi above are then unused)
  const TcInst* insts;
  int n_insts;
  int epi_variant;  // index into TcInst::epi for this launch
};

template <int BN>
struct TcCfg {
  static constexpr int A_BYTES = TC_BM * TC_BK * 2;
  static constexpr int B_BYTES = BN * TC_BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = (TC_SMEM_BUDGET - 2048) / STAGE_BYTES > 8 ? 8 : (TC_SMEM_BUDGET - 2048) / STAGE_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /* align */ + 1024 /* barriers */;
  static constexpr int TMEM_COLS = 2 * BN;
  // instruction descriptor: D=F32 (bit 4), A=BF16 (bits 7-9), B=BF16 (bits 10-12),
  // both K-major (bits 15, 16 clear), N>>3 at bit 17, M>>4 at bit 24
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                    ((uint32_t)(TC_BM >> 4) << 24);
};

// Work list of one CTA: data-parallel tiles blockIdx.x, blockIdx.x + G, ... below dp_tiles
// (whole K each), then at most one split-K unit of the tail tiles (unit u = blockIdx.x covers
// k-blocks [s KB/S, (s+1) KB/S) of tail tile u / S, s = u % S).
struct TcWork {
  int tile, kb0, kb1, unit;  // unit < 0: whole tile
  int inst;                  // grouped launch: instance of the tile; tile is then local to it
};
template <bool GROUPED>
__device__ __forceinline__ bool tc_work(const TcParams& P, int j, TcWork& w) {
  const int G = gridDim.x, c = blockIdx.x;
  if (GROUPED) {
    // tiles of all instances in one list (instances ordered by decreasing n), round-robin
    const int t = c + j * G;
    if (t >= P.num_tiles) return false;
    int k = 0;
    while (k + 1 < P.n_insts && P.insts[k + 1].tile_begin <= t) ++k;
    w.inst = k;
    w.tile = t - P.insts[k].tile_begin;
    w.kb0 = 0;
    w.kb1 = P.insts[k].kblocks;
    w.unit = -1;
    return true;
  }
  w.inst = 0;
  const int ndp = c < P.dp_tiles ? (P.dp_tiles - c + G - 1) / G : 0;
  if (j < ndp) {
    w.tile = c + j * G;
    w.kb0 = 0;
    w.kb1 = P.kblocks;
    w.unit = -1;
    return true;
  }
  if (j == ndp && c < P.sk_units) {
    const int s = c % P.splits;
    w.tile = P.dp_tiles + c / P.splits;
    w.kb0 = (int)((int64_t)s * P.kblocks / P.splits);
    w.kb1 = (int)((int64_t)(s + 1) * P.kblocks / P.splits);
    w.unit = c;
    return true;
  }
  return false;
}

template <int BN, int MODE, bool GROUPED>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc(const __grid_constant__ TcParams P) {
  using C = TcCfg<BN>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte aligned tile area (SWIZZLE_128B atoms), barriers after it
  uint8_t* tiles = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(tiles + C::STAGES * C::STAGE_BYTES);
  uint64_t* full_bar = bars;                      // [STAGES]
  uint64_t* empty_bar = bars + C::STAGES;         // [STAGES]
  uint64_t* tfull_bar = bars + 2 * C::STAGES;     // [2]
  uint64_t* tempty_bar = bars + 2 * C::STAGES + 2;  // [2]
  uint64_t* drain_bar = bars + 2 * C::STAGES + 4;   // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * C::STAGES + 5);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint64_t deadline = globaltimer_ns() + P.timeout_ns;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&tfull_bar[a]), 1);
      mbar_init(smem_u32(&tempty_bar[a]), 256);
    }
    mbar_init(smem_u32(drain_bar), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!GROUPED) {
      tma_prefetch_map(&P.mapA);
      tma_prefetch_map(&P.mapX);
    }
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const volatile int* vabort = abort_flag;

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, issued_parity = 0;
      bool ok = true;
      TcWork w;
      for (int j = 0; ok && tc_work<GROUPED>(P, j, w); ++j) {
        const int nt = GROUPED ? P.insts[w.inst].n_tiles : P.n_tiles;
        const CUtensorMap* mapA = GROUPED ? &P.insts[w.inst].mapA : &P.mapA;
        const CUtensorMap* mapX =
            GROUPED ? &P.insts[w.inst].mapX[MODE == EPI_EVAL ? 2 : (P.epi_variant >> 1)] : &P.mapX;
        const int m_tile = w.tile / nt, n_tile = w.tile % nt;
        for (int kb = w.kb0; kb < w.kb1; ++kb) {
          if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1u, deadline, vabort)) { ok = false; break; }
          const uint32_t fb = smem_u32(&full_bar[stage]);
          mbar_expect_tx(fb, (uint32_t)C::STAGE_BYTES);
          uint8_t* sa = tiles + stage * C::STAGE_BYTES;
          tma_load_2d(smem_u32(sa), mapA, fb, kb * TC_BK, m_tile * TC_BM);
          tma_load_2d(smem_u32(sa + C::A_BYTES), mapX, fb, kb * TC_BK, n_tile * BN);
          issued_mask |= 1u << stage;
          issued_parity = (issued_parity & ~(1u << stage)) | (phase << stage);
          if (++stage == C::STAGES) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) {
        atomicOr(GROUPED ? P.insts[0].epi[0].err : P.epi.err, ERR_TIMEOUT);
        *abort_flag = 1;
        // drain: every copy this thread issued completes on its full barrier
        const uint64_t dl2 = globaltimer_ns() + 200000000ull;
        const int zero = 0;
        for (int s = 0; s < C::STAGES; ++s)
          if (issued_mask & (1u << s)) mbar_wait(smem_u32(&full_bar[s]), (issued_parity >> s) & 1u, dl2, &zero);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true, issued_any = false;
      TcWork w;
      for (int j = 0; ok && tc_work<GROUPED>(P, j, w); ++j) {
        if (!mbar_wait(smem_u32(&tempty_bar[acc]), acc_phase ^ 1u, deadline, vabort)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * BN);
        for (int kb = w.kb0; kb < w.kb1; ++kb) {
          if (!mbar_wait(smem_u32(&full_bar[stage]), phase, deadline, vabort)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(tiles + stage * C::STAGE_BYTES);
          const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk) {
            tc_mma(d_tmem, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), C::IDESC,
                   (kb > w.kb0 || kk > 0) ? 1u : 0u);
          }
          issued_any = true;
          tc_commit(smem_u32(&empty_bar[stage]));
          if (++stage == C::STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        tc_commit(smem_u32(&tfull_bar[acc]));
        if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
      }
      if (!ok) {
        atomicOr(GROUPED ? P.insts[0].epi[0].err : P.epi.err, ERR_TIMEOUT);
        *abort_flag = 1;
        if (issued_any) {
          tc_commit(smem_u32(drain_bar));
          const int zero = 0;
          mbar_wait(smem_u32(drain_bar), 0, globaltimer_ns() + 200000000ull, &zero);
        }
      }
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------------ epilogue warpgroups
    // Two warpgroups split the tile's columns; inside a warpgroup, warp w reads TMEM lanes
    // 32*(w%4) .. +31, i.e. rows i of the tile.  Each 32-column chunk first issues every global
    // load it needs (so their latencies overlap), then reads the accumulator, then computes and
    // stores.  A split-K unit writes its partial tile to the workspace instead.  Each warp owns
    // one slice of the tile (its 32 rows x its warpgroup's columns); the warp that completes a
    // slice last, over all splits of the tile, sums the slice's partials in split order (the
    // result does not depend on arrival order) and runs the epilogue on it.  All waits are
    // warp-uniform and no barrier spans more than one warp, so a timeout cannot strand a warp.
    constexpr int HALF = BN / 2;
    const int wg = (warp - 4) >> 2;
    const int wq = warp & 3;
    const int slice = wg * 4 + wq;
    int acc = 0;
    uint32_t acc_phase = 0;
    TcWork w;
    for (int jw = 0; tc_work<GROUPED>(P, jw, w); ++jw) {
      const EpiArgs& a = GROUPED ? P.insts[w.inst].epi[P.epi_variant] : P.epi;
      const int nt = GROUPED ? P.insts[w.inst].n_tiles : P.n_tiles;
      const int m_tile = w.tile / nt, n_tile = w.tile % nt;
      const int row = wq * 32 + lane;
      const int64_t i = (int64_t)m_tile * TC_BM + row;
      const bool row_ok = i < a.n;
      const float cpi = row_ok ? a.cp[i] : 0.0f;
      const long long cp2 = (MODE == EPI_EVAL && row_ok) ? 2 * (long long)a.cp64[i] : 0;
      float u[32], v[32], g[32];
      bool ok = true;
      if (w.unit < 0) {
        bool waited = false;
        for (int c0 = wg * HALF; c0 < (wg + 1) * HALF; c0 += 32) {
          const int64_t rbase = (int64_t)n_tile * BN + c0;
          epi_load<MODE>(a, i, row_ok, rbase, u, v);
          if (!waited) {
            ok = mbar_wait_warp(smem_u32(&tfull_bar[acc]), acc_phase, deadline, vabort, lane);
            if (!ok) break;
            tc_fence_after();
            waited = true;
          }
          tmem_ld32(tmem_base + ((uint32_t)(wq * 32) << 16) + (uint32_t)(acc * BN + c0), g);
          epi_apply<MODE>(a, i, row_ok, cpi, cp2, rbase, lane, g, u, v, m_tile * 4 + wq);
        }
      } else {
        ok = mbar_wait_warp(smem_u32(&tfull_bar[acc]), acc_phase, deadline, vabort, lane);
        if (ok) {
          tc_fence_after();
          float* part = P.ws + (size_t)w.unit * BN * TC_BM;  // [column][row]
          for (int c0 = wg * HALF; c0 < (wg + 1) * HALF; c0 += 32) {
            tmem_ld32(tmem_base + ((uint32_t)(wq * 32) << 16) + (uint32_t)(acc * BN + c0), g);
#pragma unroll
            for (int j = 0; j < 32; ++j) __stcg(part + (size_t)(c0 + j) * TC_BM + row, g[j]);
          }
        }
      }
      if (!ok) {
        if (lane == 0) {
          atomicOr(a.err, ERR_TIMEOUT);
          *abort_flag = 1;
        }
        break;
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&tempty_bar[acc]));
      if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
      if (w.unit >= 0) {
        const int tail = w.tile - P.dp_tiles;
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0) {
          int* ctr = P.counters + tail * 8 + slice;
          last = atomicAdd(ctr, 1) == P.splits - 1;
          if (last) *ctr = 0;  // ready for the next launch
          __threadfence();
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        __syncwarp();
        if (last) {
          __threadfence();
          for (int c0 = wg * HALF; c0 < (wg + 1) * HALF; c0 += 32) {
            const int64_t rbase = (int64_t)n_tile * BN + c0;
            epi_load<MODE>(a, i, row_ok, rbase, u, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) g[j] = 0.0f;
            for (int sp = 0; sp < P.splits; ++sp) {
              const float* ps = P.ws + (size_t)(tail * P.splits + sp) * BN * TC_BM;
#pragma unroll
              for (int j = 0; j < 32; ++j) g[j] += __ldcg(ps + (size_t)(c0 + j) * TC_BM + row);
            }
            epi_apply<MODE>(a, i, row_ok, cpi, cp2, rbase, lane, g, u, v, m_tile * 4 + wq);
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
  }
}

// ---- host side ---------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool tc_supported() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && get_encode() != nullptr;
}

static cudaError_t encode_bf16_2d(CUtensorMap* m, const void* ptr, uint64_t inner, uint64_t rows, uint64_t ld_elems,
                                  uint32_t box_rows, std::string* why) {
  auto fn = get_encode();
  if (!fn) {
    if (why) *why = "cuTensorMapEncodeTiled unavailable";
    return cudaErrorNotSupported;
  }
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) || ((ld_elems * 2) & 15)) {
    if (why) *why = "TMA needs a 16-byte aligned base and row pitch";
    return cudaErrorInvalidValue;
  }
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {ld_elems * 2};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (why) *why = "cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r);
    return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t tc_make_operand_map(CUtensorMap* m, const void* X, int64_t ldx, int n, int B, int tile_n,
                                std::string* why) {
  return encode_bf16_2d(m, X, (uint64_t)n, (uint64_t)B, (uint64_t)ldx, (uint32_t)tile_n, why);
}

template <int BN, int MODE>
static cudaError_t set_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_tc<BN, MODE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       TcCfg<BN>::SMEM);
  if (e == cudaSuccess && MODE != EPI_LAGR)
    e = cudaFuncSetAttribute(k_tc<BN, MODE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<BN>::SMEM);
  return e;
}

static cudaError_t ensure_attrs();

cudaError_t tc_make_plan(TcPlan* plan, const void* A, int64_t lda, int n, const void* X0, const void* X1,
                         const void* Xbits, int64_t ldx, int B, int tile_n, std::string* why) {
  plan->ready = false;
  if (tile_n != 64 && tile_n != 128 && tile_n != 256) {
    if (why) *why = "tile_n must be 64, 128 or 256";
    return cudaErrorInvalidValue;
  }
  cudaError_t e = encode_bf16_2d(&plan->mapA, A, (uint64_t)n, (uint64_t)n, (uint64_t)lda, TC_BM, why);
  if (e != cudaSuccess) return e;
  const void* xs[3] = {X0, X1, Xbits};
  for (int k = 0; k < 3; ++k) {
    if (!xs[k]) continue;
    e = tc_make_operand_map(&plan->mapX[k], xs[k], ldx, n, B, tile_n, why);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  plan->tile_n = tile_n;
  plan->m_tiles = (n + TC_BM - 1) / TC_BM;
  plan->n_tiles = (B + tile_n - 1) / tile_n;
  plan->num_tiles = plan->m_tiles * plan->n_tiles;
  plan->grid = plan->num_tiles < sms ? plan->num_tiles : sms;
  plan->sms = sms;
  plan->ws = nullptr;
  plan->counters = nullptr;
  plan->max_splits = 0;
  plan->pair = false;
  plan->csk = 0;
  const cudaError_t attr_err = ensure_attrs();
  if (attr_err != cudaSuccess) {
    if (why) *why = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(attr_err);
    return attr_err;
  }
  plan->ready = true;
  return cudaSuccess;
}

template <int BN, int MODE>
static cudaError_t launch_tc_t(const TcParams& P, int grid, cudaStream_t s) {
  k_tc<BN, MODE, false><<<grid, TC_THREADS, TcCfg<BN>::SMEM, s>>>(P);
  return cudaGetLastError();
}

template <int BN>
static cudaError_t launch_tc_bn(const TcParams& P, int grid, int mode, cudaStream_t s) {
  if (mode == EPI_UPDATE) return launch_tc_t<BN, EPI_UPDATE>(P, grid, s);
  if (mode == EPI_EVAL) return launch_tc_t<BN, EPI_EVAL>(P, grid, s);
  return launch_tc_t<BN, EPI_LAGR>(P, grid, s);
}

TcSchedule tc_schedule(int num_tiles, int kblocks, int sms, bool can_split, int max_splits) {
  TcSchedule r;
  r.dp_tiles = num_tiles;
  r.splits = 1;
  r.sk_units = 0;
  r.grid = num_tiles < sms ? num_tiles : sms;
  const int tail = num_tiles % sms;
  if (!can_split || tail == 0) return r;
  int S = sms / tail;
  const int kcap = kblocks / TC_MIN_KB_PER_SPLIT;
  if (S > kcap) S = kcap;
  if (S > max_splits) S = max_splits;
  if (S < 2) return r;
  r.dp_tiles = num_tiles - tail;
  r.splits = S;
  r.sk_units = tail * S;
  r.grid = r.dp_tiles > 0 ? sms : r.sk_units;
  return r;
}

cudaError_t launch_tc(const TcPlan& plan, int which_x, const CUtensorMap* map_override, const EpiArgs& a,
                      int mode, uint64_t timeout_ns, cudaStream_t s) {
  if (!plan.ready) return cudaErrorInvalidValue;
  if (plan.pair && !map_override && (mode == EPI_UPDATE || mode == EPI_EVAL))
    return launch_tc_pair(plan, which_x, a, mode, timeout_ns, s);
  if (plan.csk >= 2 && !map_override && (mode == EPI_UPDATE || mode == EPI_EVAL))
    return launch_tc_csk(plan, which_x, a, mode, 1, timeout_ns, s);
  TcParams P;
  P.mapA = plan.mapA;
  P.mapX = map_override ? *map_override : plan.mapX[which_x];
  P.epi = a;
  P.n = a.n;
  P.m_tiles = (a.n + TC_BM - 1) / TC_BM;
  P.n_tiles = (a.B + plan.tile_n - 1) / plan.tile_n;
  P.num_tiles = P.m_tiles * P.n_tiles;
  P.kblocks = (a.n + TC_BK - 1) / TC_BK;
  P.timeout_ns = timeout_ns;
  const TcSchedule sch = tc_schedule(P.num_tiles, P.kblocks, plan.sms, plan.ws != nullptr && plan.counters != nullptr,
                                     plan.max_splits);
  P.dp_tiles = sch.dp_tiles;
  P.splits = sch.splits;
  P.sk_units = sch.sk_units;
  P.ws = plan.ws;
  P.counters = plan.counters;
  const int grid = sch.grid;
  switch (plan.tile_n) {
    case 64: return launch_tc_bn<64>(P, grid, mode, s);
    case 128: return launch_tc_bn<128>(P, grid, mode, s);
    default: return launch_tc_bn<256>(P, grid, mode, s);
  }
}

static cudaError_t ensure_attrs() {
  static PerDevice per_device;
  return per_device.once([] {
    cudaError_t r = cudaSuccess;
    r = r == cudaSuccess ? set_attr<64, EPI_UPDATE>() : r;
    r = r == cudaSuccess ? set_attr<64, EPI_EVAL>() : r;
    r = r == cudaSuccess ? set_attr<64, EPI_LAGR>() : r;
    r = r == cudaSuccess ? set_attr<128, EPI_UPDATE>() : r;
    r = r == cudaSuccess ? set_attr<128, EPI_EVAL>() : r;
    r = r == cudaSuccess ? set_attr<128, EPI_LAGR>() : r;
    r = r == cudaSuccess ? set_attr<256, EPI_UPDATE>() : r;
    r = r == cudaSuccess ? set_attr<256, EPI_EVAL>() : r;
    r = r == cudaSuccess ? set_attr<256, EPI_LAGR>() : r;
    return r;
  });
}

cudaError_t launch_tc_group(const TcInst* d_insts, int n_insts, int num_tiles, int tile_n, int mode, int epi_variant,
                            uint64_t timeout_ns, cudaStream_t s) {
  if (mode != EPI_UPDATE && mode != EPI_EVAL) return cudaErrorInvalidValue;
  cudaError_t e = ensure_attrs();
  if (e != cudaSuccess) return e;
  TcParams P;
  memset(&P, 0, sizeof(P));
  P.num_tiles = num_tiles;
  P.dp_tiles = num_tiles;
  P.splits = 1;
  P.timeout_ns = timeout_ns;
  P.insts = d_insts;
  P.n_insts = n_insts;
  P.epi_variant = epi_variant;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = num_tiles < sms ? num_tiles : sms;
  if (grid < 1) return cudaSuccess;
#define SBO_GROUP_LAUNCH(BNV)                                                                            \
  if (mode == EPI_UPDATE) k_tc<BNV, EPI_UPDATE, true><<<grid, TC_THREADS, TcCfg<BNV>::SMEM, s>>>(P);     \
  else k_tc<BNV, EPI_EVAL, true><<<grid, TC_THREADS, TcCfg<BNV>::SMEM, s>>>(P);
  switch (tile_n) {
    case 64: SBO_GROUP_LAUNCH(64); break;
    case 128: SBO_GROUP_LAUNCH(128); break;
    default: SBO_GROUP_LAUNCH(256); break;
  }
#undef SBO_GROUP_LAUNCH
  return cudaGetLastError();
}

}  // namespace sbo
