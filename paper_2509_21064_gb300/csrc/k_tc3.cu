// Dense contraction for problems with fewer output tiles than SMs: split-K inside a thread-block
// cluster, several GDA iterations per launch.
//
// With B restarts and n rows there are ceil(n/128) * ceil(B/BN) tiles of the accumulator; when
// that is well below the SM count (n = 5,000 with B = 256 gives 40 tiles of 128 x 256 on 152
// SMs), one CTA per tile leaves most SMs idle and runs its epilogue with nothing to overlap.
// Here a cluster of S CTAs shares one tile:
//   * CTA s of the cluster runs k-blocks [s KB/S, (s+1) KB/S) with the same warp-specialised
//     TMA / tcgen05.mma pipeline as k_tc.cu (one accumulator of BN TMEM columns);
//   * CTA s owns the 32-column chunks [s NC/S, (s+1) NC/S) of the tile (NC = BN/32).  Its
//     epilogue warps copy the partial accumulator, column-major [column][row], into its own (now
//     idle) stage buffers for the columns it owns and into its slice of a workspace in L2 for the
//     others;
//   * after a cluster barrier, CTA s sums the S partials of its columns in split order 0..S-1
//     (so the sum does not depend on timing) and applies the PDBO update / exact objective to
//     them.  Each warp takes whole restart columns (all 128 rows, four consecutive rows per
//     lane): every partial read, state load and state store of a warp is one contiguous 512-byte
//     run of 16-byte accesses, and a batch of columns issues all its loads before any is used.
//     No CTA reads another's shared memory, so one cluster barrier per iteration suffices.
// Pulling the partials from the peers' shared memory (ld.shared::cluster.v4, the same pipelined
// rounds) measured slower than the L2 path: 6.5 against 5.2 us of epilogue per iteration at
// n = 5,000, B = 256, and 5.0 against 3.0 us at n = 2,000.
//
// An update launch runs `iters` GDA iterations: between two iterations every CTA publishes its
// part of x^{t+1} (stores fenced for the TMA loads of other CTAs) and meets the others at a grid
// barrier in global memory; the launch is one wave of clusters, so all CTAs are resident and may
// wait for one another.  That removes the launch gap, the set-up of TMEM and barriers, and the
// cold instruction cache of one launch per iteration.
//
// Every wait is bounded (globaltimer budget per iteration).  A CTA that gives up sets
// ERR_TIMEOUT, raises the launch's abort word, drains its own copies and MMAs and skips the
// reduction; the CTAs of a cluster decide together at each iteration's cluster barrier, from
// votes pushed into every CTA's shared memory before it, whether to stop, so the cluster barriers
// stay matched and every CTA returns in bounded time.
#include <cudaTypedefs.h>

#include <array>
#include <mutex>
#include <utility>
#include <vector>

#include "tc_common.cuh"

namespace sbo {
namespace {

constexpr int CSK_THREADS = 384;   // warp 0 TMA, warp 1 TMEM + MMA, warps 4-11 partial tile; all in the reduction
constexpr int CSK_SMEM_BUDGET = 196 * 1024;
constexpr int CSK_MIN_KB = 4;      // k-blocks per CTA at least

// BN restarts per tile.  PAIR: the tile is 256 rows x BN restarts on a CTA pair (cta_group::2):
// each CTA stages its own 128 rows of A and BN / 2 restarts of x per k-block.
template <int BN, bool PAIR>
struct CskCfg {
  static constexpr int H = PAIR ? 2 : 1;                  // CTAs per split
  static constexpr int A_BYTES = TC_BM * TC_BK * 2;
  static constexpr int B_BYTES = (BN / H) * TC_BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES =
      (CSK_SMEM_BUDGET - 2048) / STAGE_BYTES > 8 ? 8 : (CSK_SMEM_BUDGET - 2048) / STAGE_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /* align */ + 1024 /* barriers */;
  static constexpr int TMEM_COLS = BN;
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                    ((uint32_t)((TC_BM * H) >> 4) << 24);
  static_assert(STAGES * STAGE_BYTES >= BN * TC_BM * 4, "the partial tile must fit in the stage buffers");
};

struct CskParams {
  CUtensorMap mapA;
  CUtensorMap mapX[2];     // operand of an iteration by parity (EVAL: mapX[0] is the candidates' map)
  EpiArgs epi;             // Xout and bits_out are taken from xop / bits_last below
  void* xop[2];            // operand buffers: iteration j reads xop[w] and writes xop[w ^ 1], w = (x0 + j) & 1
  void* bits_last;         // candidates written by the last iteration (null: none)
  unsigned int* gbar;      // grid barrier [arrivals, exits, abort], zero between launches (iters > 1)
  float* ws;               // partials [tile][split][CTA of the pair][column][row] (one BN x 128 slice per CTA)
  int x0, iters;
  int n_tiles, kblocks, S; // S: K splits per tile (CTA pairs when paired; the cluster holds S CTAs or pairs)
  uint64_t timeout_ns;     // per iteration
};

__device__ __forceinline__ uint32_t csk_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void csk_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t csk_mapa(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ float f4_at(const float4& v, int k) {
  return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

constexpr int CSK_WARPS = CSK_THREADS / 32;
constexpr int CSK_CB = 4;   // restart columns per warp whose loads are in flight together

// Reduction and epilogue of tile columns [c_begin, c_end) (restarts r0 + c) of the 128 rows of
// block row_block (variables 128 row_block ..).  Warp w takes the columns c_begin + w + CSK_WARPS t;
// lane l holds rows 4l .. 4l+3 of the block (variables i0 .. i0+3).
// The S partials of a column are summed in split order.  The state rows are padded to a multiple
// of 8 elements, so the 16-byte loads at i0 < n stay inside the row; stores of the last, partial
// group of four rows go element by element.
template <int BN, int MODE, int GK, bool SINGLE>
__device__ __forceinline__ void csk_columns(const EpiArgs& a, void* xout, void* bits, const float* part,
                                            const float* ws_tile, int64_t split_stride, int s, int S, int row_block,
                                            int64_t r0, int c_begin, int c_end, int warp, int lane) {
  const int row0 = 4 * lane;
  const int64_t i0 = (int64_t)row_block * TC_BM + row0;
  const int64_t left = (int64_t)a.n - i0;
  const int nv = left <= 0 ? 0 : left >= 4 ? 4 : (int)left;   // valid rows of this lane
  float cpv[4];
  long long cp2v[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    cpv[k] = k < nv ? a.cp[i0 + k] : 0.0f;
    cp2v[k] = (MODE == EPI_EVAL && k < nv) ? 2 * (long long)a.cp64[i0 + k] : 0;
  }
  for (int cb = c_begin + warp; cb < c_end; cb += CSK_WARPS * CSK_CB) {
    float4 xv[CSK_CB], yv[CSK_CB], g[CSK_CB];
    uint2 xb[CSK_CB];
#pragma unroll
    for (int t = 0; t < CSK_CB; ++t) {   // state loads (warp-uniform column tests)
      const int c = cb + CSK_WARPS * t;
      const int64_t r = r0 + c;
      const bool ok = c < c_end && r < a.B && nv > 0;
      const int64_t idx = r * a.ld + i0;
      xv[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      yv[t] = xv[t];
      xb[t] = make_uint2(0u, 0u);
      if (ok) {
        if (MODE == EPI_UPDATE) {
          xv[t] = *reinterpret_cast<const float4*>(a.Xm + idx);
          if (SINGLE) {
            const float m = a.mu[r];
            yv[t] = make_float4(m, m, m, m);
          } else {
            yv[t] = *reinterpret_cast<const float4*>(a.Y + idx);
          }
        } else {
          xb[t] = *reinterpret_cast<const uint2*>(static_cast<const __nv_bfloat16*>(a.Xin) + idx);
        }
      }
      g[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // The S partials of the batch's columns, summed in split order (the sum does not depend on
    // timing).  One round of loads per split, issued without a branch between them (columns past
    // c_end read a valid column and are never used) and pipelined two deep, so that a warp waits
    // for about one load latency per two splits instead of one per load.
    int col[CSK_CB];
#pragma unroll
    for (int t = 0; t < CSK_CB; ++t) col[t] = min(cb + CSK_WARPS * t, c_end - 1);
    auto load_round = [&](int sp, float4 (&pv)[CSK_CB]) {
      // this CTA's own partial of a column is in its shared memory, the others' in L2
      if (sp == s) {
#pragma unroll
        for (int t = 0; t < CSK_CB; ++t) pv[t] = *reinterpret_cast<const float4*>(part + col[t] * TC_BM + row0);
      } else {
        const float* wsp = ws_tile + (size_t)sp * split_stride + row0;
#pragma unroll
        for (int t = 0; t < CSK_CB; ++t) pv[t] = __ldcg(reinterpret_cast<const float4*>(wsp + (size_t)col[t] * TC_BM));
      }
    };
    auto add_round = [&](const float4 (&pv)[CSK_CB]) {
#pragma unroll
      for (int t = 0; t < CSK_CB; ++t) {
        g[t].x += pv[t].x;
        g[t].y += pv[t].y;
        g[t].z += pv[t].z;
        g[t].w += pv[t].w;
      }
    };
    float4 pa[CSK_CB], pb[CSK_CB];
    load_round(0, pa);
    for (int sp = 0; sp < S; sp += 2) {
      if (sp + 1 < S) load_round(sp + 1, pb);
      add_round(pa);
      if (sp + 1 < S) {
        if (sp + 2 < S) load_round(sp + 2, pa);
        add_round(pb);
      }
    }
#pragma unroll
    for (int t = 0; t < CSK_CB; ++t) {
      const int c = cb + CSK_WARPS * t;
      const int64_t r = r0 + c;
      const bool col_ok = c < c_end && r < a.B;   // warp-uniform
      if (!col_ok) continue;
      const int64_t idx = r * a.ld + i0;
      if (MODE == EPI_EVAL) {
        const float xk[4] = {bf16_lo(xb[t].x), bf16_hi(xb[t].x), bf16_lo(xb[t].y), bf16_hi(xb[t].y)};
        long long w = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (k < nv && xk[k] != 0.0f) w += (long long)f4_at(g[t], k) + cp2v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0 && w != 0) atomicAdd(&a.F2[r], (unsigned long long)w);
      } else {
        float xn[4], yn[4], dd[4], gsum = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float x = f4_at(xv[t], k), y = f4_at(yv[t], k);
          const float gx = g_val(x, GK);
          dd[k] = f4_at(g[t], k) + cpv[k] + y * g_der(x, GK);
          xn[k] = pdbo_update(x, y, dd[k], gx, a.alpha, a.beta, a.delta, a.grad_tol, &yn[k]);
          if (SINGLE && k < nv) gsum += gx;
        }
        if (nv == 4) {
          if (a.Gd) *reinterpret_cast<float4*>(a.Gd + idx) = make_float4(dd[0], dd[1], dd[2], dd[3]);
          *reinterpret_cast<float4*>(a.Xm + idx) = make_float4(xn[0], xn[1], xn[2], xn[3]);
          if (!SINGLE) *reinterpret_cast<float4*>(a.Y + idx) = make_float4(yn[0], yn[1], yn[2], yn[3]);
          *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(xout) + idx) =
              make_uint2(pack_bf16x2(xn[0], xn[1]), pack_bf16x2(xn[2], xn[3]));
          if (bits) {
            float b[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) b[k] = xn[k] > 0.5f ? 1.0f : 0.0f;
            *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(bits) + idx) =
                make_uint2(pack_bf16x2(b[0], b[1]), pack_bf16x2(b[2], b[3]));
          }
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (k < nv) {
              if (a.Gd) a.Gd[idx + k] = dd[k];
              a.Xm[idx + k] = xn[k];
              if (!SINGLE) a.Y[idx + k] = yn[k];
              static_cast<__nv_bfloat16*>(xout)[idx + k] = __float2bfloat16_rn(xn[k]);
              if (bits) static_cast<__nv_bfloat16*>(bits)[idx + k] = __float2bfloat16_rn(xn[k] > 0.5f ? 1.0f : 0.0f);
            }
          }
        }
        if (SINGLE) {
          // partial sums of g(x^t) over 32 rows (eight lanes), one row of partials per 32 rows
#pragma unroll
          for (int o = 1; o < 8; o <<= 1) gsum += __shfl_xor_sync(0xffffffffu, gsum, o);
          if ((lane & 7) == 0) a.gpart[(int64_t)(row_block * 4 + (lane >> 3)) * a.gpart_ld + r] = gsum;
        }
      }
    }
  }
}

template <int BN, int MODE>
__device__ __forceinline__ void csk_epilogue(const EpiArgs& a, void* xout, void* bits, const float* part,
                                             const float* ws_tile, int64_t split_stride, int s, int S, int row_block,
                                             int64_t r0, int c_begin, int c_end, int warp, int lane) {
#define CSK_COLUMNS(M, G, SG)                                                                                    \
  csk_columns<BN, M, G, SG>(a, xout, bits, part, ws_tile, split_stride, s, S, row_block, r0, c_begin, c_end, warp, \
                            lane)
  if (MODE == EPI_EVAL) {
    CSK_COLUMNS(EPI_EVAL, G_QUAD, false);
  } else if (a.gkind == G_ENTROPY) {
    if (a.mu) CSK_COLUMNS(EPI_UPDATE, G_ENTROPY, true);
    else CSK_COLUMNS(EPI_UPDATE, G_ENTROPY, false);
  } else {
    if (a.mu) CSK_COLUMNS(EPI_UPDATE, G_QUAD, true);
    else CSK_COLUMNS(EPI_UPDATE, G_QUAD, false);
  }
#undef CSK_COLUMNS
}

template <int BN, int MODE, bool PAIR>
__global__ void __launch_bounds__(CSK_THREADS, 1) k_tc_csk(const __grid_constant__ CskParams P) {
  using C = CskCfg<BN, PAIR>;
  constexpr int H = C::H;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* tiles = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(tiles + C::STAGES * C::STAGE_BYTES);
  uint64_t* full_bar = bars;                   // [STAGES] (paired: the leader's counts both CTAs' copies)
  uint64_t* empty_bar = bars + C::STAGES;      // [STAGES]
  uint64_t* tfull_bar = bars + 2 * C::STAGES;  // accumulator complete (one phase per iteration)
  uint64_t* drain_bar = tfull_bar + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain_bar + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  int* stop_vote = abort_flag + 1;             // [2] the cluster's votes to stop, by iteration parity
  int* stop_all = abort_flag + 3;              // the cluster's decision, broadcast in the CTA

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int S = P.S;
  const int CL = S * H;                        // CTAs per cluster
  const uint32_t rank = csk_rank();
  const int sp_me = (int)rank / H;             // this CTA's K split
  const int h = (int)rank % H;                 // half of the pair (0: leader, issues the MMAs)
  const uint32_t lead = rank - (uint32_t)h;
  const uint16_t pair_mask = (uint16_t)(0x3u << lead);
  const int tile = (int)(blockIdx.x / (unsigned)CL);
  const int m_tile = tile / P.n_tiles, n_tile = tile % P.n_tiles;
  const int mb = m_tile * H + h;               // 128-row block of A this CTA accumulates
  const int kb0 = (int)((int64_t)sp_me * P.kblocks / S);
  const int kb1 = (int)((int64_t)(sp_me + 1) * P.kblocks / S);
  const int nk = kb1 - kb0;
  // restart columns [c_begin, c_end) of the tile (its rows of this CTA) are this CTA's:
  // 32-column chunks sp NC/S .. (sp+1) NC/S - 1
  constexpr int NC = BN / 32;
  const int c_begin = (int)(sp_me * NC / S) * 32, c_end = (int)((sp_me + 1) * NC / S) * 32;
  const EpiArgs& a = P.epi;
  const bool multi = P.iters > 1;

  if (threadIdx.x == 0) {
    for (int q = 0; q < C::STAGES; ++q) {
      mbar_init(smem_u32(&full_bar[q]), 1);
      mbar_init(smem_u32(&empty_bar[q]), 1);
    }
    mbar_init(smem_u32(tfull_bar), 1);
    mbar_init(smem_u32(drain_bar), 1);
    *abort_flag = 0;
    stop_vote[0] = stop_vote[1] = 0;
    *stop_all = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tma_prefetch_map(&P.mapA);
    tma_prefetch_map(&P.mapX[0]);
    if (multi) tma_prefetch_map(&P.mapX[1]);
  }
  if (warp == 1) {
    if (PAIR) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"((uint32_t)C::TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"((uint32_t)C::TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  if (PAIR) csk_cluster_sync();   // the pair's barriers are initialised and TMEM allocated in both CTAs
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const volatile int* vabort = abort_flag;
  auto bwait = [&](uint64_t* bar, uint32_t parity, uint64_t dl) {
    return PAIR ? mbar_wait_cl(smem_u32(bar), parity, dl, vabort) : mbar_wait(smem_u32(bar), parity, dl, vabort);
  };

  // pipeline positions carried across iterations by the producer and the MMA issuer
  int stage = 0;
  uint32_t phase = 0;
  uint32_t issued_mask = 0, issued_parity = 0;   // producer: stages with a copy issued, and its phase
  bool issued_any = false;                       // MMA issuer: an MMA may be in flight

  for (int it = 0; it < P.iters; ++it) {
    const int w = (P.x0 + it) & 1;
    const uint64_t deadline = globaltimer_ns() + P.timeout_ns;
    if (warp == 0) {
      // ---------------------------------------------------------------- TMA producer
      if (lane == 0 && *vabort == 0) {
        // iteration it reads x^{it}, written by every CTA in iteration it - 1
        bool ok = it == 0 || grid_wait(P.gbar, (unsigned int)it * gridDim.x, deadline);
        if (ok && it > 0) asm volatile("fence.proxy.async.global;" ::: "memory");
        for (int jk = 0; ok && jk < nk; ++jk) {
          const int kb = kb0 + jk;
          if (!bwait(&empty_bar[stage], phase ^ 1u, deadline)) { ok = false; break; }
          uint8_t* sa = tiles + stage * C::STAGE_BYTES;
          if (PAIR) {
            // both CTAs' copies complete on the leader's barrier, which the leader arms for both
            const uint32_t fb = map_to_rank(smem_u32(&full_bar[stage]), lead);
            if (h == 0) mbar_expect_tx(smem_u32(&full_bar[stage]), (uint32_t)(2 * C::STAGE_BYTES));
            tma_load_2d_pair(smem_u32(sa), &P.mapA, fb, kb * TC_BK, m_tile * 2 * TC_BM + h * TC_BM);
            tma_load_2d_pair(smem_u32(sa + C::A_BYTES), &P.mapX[w], fb, kb * TC_BK, n_tile * BN + h * (BN / 2));
          } else {
            const uint32_t fb = smem_u32(&full_bar[stage]);
            mbar_expect_tx(fb, (uint32_t)C::STAGE_BYTES);
            tma_load_2d(smem_u32(sa), &P.mapA, fb, kb * TC_BK, m_tile * TC_BM);
            tma_load_2d(smem_u32(sa + C::A_BYTES), &P.mapX[w], fb, kb * TC_BK, n_tile * BN);
          }
          issued_mask |= 1u << stage;
          issued_parity = (issued_parity & ~(1u << stage)) | (phase << stage);
          if (++stage == C::STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) {
          atomicOr(a.err, ERR_TIMEOUT);
          *abort_flag = 1;
          if (multi) atomicExch(P.gbar + 2, 1u);
          if (PAIR) {
            // a pair's copies are counted on the leader's barriers, so neither CTA can watch its own
            // land: give every copy in flight a generous fixed time instead
            if (issued_mask) {
              const uint64_t until = globaltimer_ns() + 2000000ull;
              while (globaltimer_ns() < until) {
              }
            }
          } else {
            const uint64_t dl2 = globaltimer_ns() + 200000000ull;
            const int zero = 0;
            for (int q = 0; q < C::STAGES; ++q)
              if (issued_mask & (1u << q)) mbar_wait(smem_u32(&full_bar[q]), (issued_parity >> q) & 1u, dl2, &zero);
          }
        }
      }
    } else if (warp == 1) {
      // ---------------------------------------------------------------- MMA issuer (pair: the leader)
      if (lane == 0 && h == 0 && *vabort == 0) {
        bool ok = true;
        for (int jk = 0; jk < nk; ++jk) {
          if (!bwait(&full_bar[stage], phase, deadline)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(tiles + stage * C::STAGE_BYTES);
          const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk) {
            if (PAIR)
              mma_pair(tmem_base, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), C::IDESC,
                       (jk > 0 || kk > 0) ? 1u : 0u);
            else
              tc_mma(tmem_base, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), C::IDESC,
                     (jk > 0 || kk > 0) ? 1u : 0u);
          }
          issued_any = true;
          if (PAIR) commit_pair_multicast(smem_u32(&empty_bar[stage]), pair_mask);
          else tc_commit(smem_u32(&empty_bar[stage]));
          if (++stage == C::STAGES) { stage = 0; phase ^= 1u; }
        }
        if (ok) {
          if (PAIR) commit_pair_multicast(smem_u32(tfull_bar), pair_mask);
          else tc_commit(smem_u32(tfull_bar));
        } else {
          atomicOr(a.err, ERR_TIMEOUT);
          *abort_flag = 1;
          if (multi) atomicExch(P.gbar + 2, 1u);
          if (issued_any) {
            if (PAIR) commit_pair_local(smem_u32(drain_bar));
            else tc_commit(smem_u32(drain_bar));
            const int zero = 0;
            mbar_wait(smem_u32(drain_bar), 0, globaltimer_ns() + 200000000ull, &zero);
          }
        }
      }
    } else if (warp >= 4) {
      // ---------------------------------------------------------------- partial tile out
      // Every MMA of this CTA's iteration has completed when tfull fires, so the stage buffers are
      // idle: the accumulator (lane = row) goes out column-major, [column][row], to the stage
      // buffers for the columns this CTA owns and to its workspace slice in L2 for the others.
      const int wg = (warp - 4) >> 2;
      const int wq = warp & 3;
      const int row = wq * 32 + lane;
      if (*vabort == 0) {
        const bool ready = PAIR ? mbar_wait_cl_warp(smem_u32(tfull_bar), (uint32_t)(it & 1), deadline, vabort, lane)
                                : mbar_wait_warp(smem_u32(tfull_bar), (uint32_t)(it & 1), deadline, vabort, lane);
        if (ready) {
          tc_fence_after();
          // columns this CTA owns stay in its shared memory, the others go to its slice of the
          // workspace in L2, where their owners read them
          float* part = reinterpret_cast<float*>(tiles);
          float* mine = P.ws + (((size_t)tile * S + sp_me) * H + h) * BN * TC_BM;
          float g[32];
          for (int c0 = wg * (BN / 2); c0 < (wg + 1) * (BN / 2); c0 += 32) {
            tmem_ld32(tmem_base + ((uint32_t)(wq * 32) << 16) + (uint32_t)c0, g);
            float* dst = (c0 >= c_begin && c0 < c_end) ? part : mine;
#pragma unroll
            for (int j = 0; j < 32; ++j) dst[(c0 + j) * TC_BM + row] = g[j];
          }
        } else if (lane == 0) {
          atomicOr(a.err, ERR_TIMEOUT);
          *abort_flag = 1;
          if (multi) atomicExch(P.gbar + 2, 1u);
        }
      }
    }

    // Stop together: a CTA that must stop ORs its vote into the vote word of this parity in every
    // CTA of the cluster before the barrier below, so that after it every CTA reads the same
    // decision from its own word (rewritten two iterations later, after two more cluster
    // barriers) and the cluster barriers stay matched.  Nothing is sent when no CTA stops.
    if (threadIdx.x == 0 && (*vabort != 0 || (multi && ld_acquire_gpu(P.gbar + 2) != 0u))) {
      for (int r = 0; r < CL; ++r)
        asm volatile("red.shared::cluster.or.b32 [%0], 1;" ::"r"(csk_mapa(smem_u32(&stop_vote[it & 1]), (uint32_t)r))
                     : "memory");
    }

    __syncwarp();
    tc_fence_before();
    csk_cluster_sync();   // every CTA's partial tile is out; the votes are in
    tc_fence_after();
    if (threadIdx.x == 0) {
      volatile int* vote = stop_vote + (it & 1);
      *stop_all = *vote;
      *vote = 0;   // ready for iteration it + 2
    }
    __syncthreads();
    if (*stop_all) break;   // every CTA of the cluster leaves here, before any later cluster barrier

    // ---------------------------------------------------------------- reduction + epilogue
    // All twelve warps take part (the producer and MMA warps are idle by now); the partials come
    // from shared memory and L2, not TMEM, so any warp may take any columns.  No CTA reads
    // another's shared memory from here on: the next cluster barrier is the next iteration's.
    void* bits = it + 1 == P.iters ? P.bits_last : nullptr;
    csk_epilogue<BN, MODE>(a, P.xop[w ^ 1], bits, reinterpret_cast<const float*>(tiles),
                           P.ws + ((size_t)tile * S * H + h) * BN * TC_BM, (int64_t)H * BN * TC_BM, sp_me, S, mb,
                           (int64_t)n_tile * BN, c_begin, c_end, warp, lane);
    if (it + 1 == P.iters) break;
    fence_stores_for_tma();
    // this CTA's part of x^{it+1} is written: every thread fenced its stores before this barrier,
    // which orders them before thread 0's release; its own shared-memory partials are read
    __syncthreads();
    if (threadIdx.x == 0) red_release_gpu_add(P.gbar, 1u);
  }

  if (multi) {
    __syncthreads();
    if (threadIdx.x == 0) {
      // the last CTA out restores the words for the next launch (the abort word stays raised
      // after a failure; the host clears it when it reads the error)
      if (atomicAdd(P.gbar + 1, 1u) == gridDim.x - 1) {
        atomicExch(P.gbar, 0u);
        atomicExch(P.gbar + 1, 0u);
      }
    }
  }
  if (warp == 1) {
    tc_fence_after();
    if (PAIR)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                   "r"((uint32_t)C::TMEM_COLS)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                   "r"((uint32_t)C::TMEM_COLS)
                   : "memory");
  }
}

template <int BN, int MODE, bool PAIR>
cudaError_t csk_set_attr() {
  return cudaFuncSetAttribute(k_tc_csk<BN, MODE, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              CskCfg<BN, PAIR>::SMEM);
}

template <int BN, bool PAIR>
cudaError_t csk_set_attrs() {
  const cudaError_t e = csk_set_attr<BN, EPI_UPDATE, PAIR>();
  return e == cudaSuccess ? csk_set_attr<BN, EPI_EVAL, PAIR>() : e;
}

// cluster: CTAs per cluster (S, or 2 S for pairs)
template <int BN, bool PAIR>
cudaLaunchConfig_t csk_config(int grid, int cluster, cudaLaunchAttribute* attr, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(CSK_THREADS);
  cfg.dynamicSmemBytes = CskCfg<BN, PAIR>::SMEM;
  cfg.stream = s;
  attr->id = cudaLaunchAttributeClusterDimension;
  attr->val.clusterDim.x = (unsigned)cluster;
  attr->val.clusterDim.y = 1;
  attr->val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Clusters of `cluster` CTAs of this kernel that fit on the current device at once (0 if none),
// queried once per (device, cluster size): the attributes and the occupancy answer belong to the
// device's context.
template <int BN, bool PAIR>
int csk_max_clusters(int cluster) {
  static std::mutex mu;
  static std::vector<std::pair<int, std::array<int, 9>>> cache;   // (device, answer per cluster size)
  if (cluster < 2 || cluster > 8) return 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(mu);
  std::array<int, 9>* row = nullptr;
  for (auto& c : cache)
    if (c.first == dev) row = &c.second;
  if (!row) {
    std::array<int, 9> fresh;
    fresh.fill(-1);
    cache.push_back({dev, fresh});
    row = &cache.back().second;
  }
  int& slot = (*row)[cluster];
  if (slot >= 0) return slot;
  slot = 0;
  if (csk_set_attrs<BN, PAIR>() != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchAttribute attr;
  cudaLaunchConfig_t cfg = csk_config<BN, PAIR>(cluster * 16, cluster, &attr, nullptr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_tc_csk<BN, EPI_UPDATE, PAIR>, &cfg) == cudaSuccess) slot = n;
  cudaGetLastError();
  return slot;
}

// Whether the current device takes cooperative launches of clusters: 1 yes, 0 no, -1 not known yet.
std::mutex coop_mu;
std::vector<std::pair<int, int>> coop_answer;
int coop_state(int dev) {
  std::lock_guard<std::mutex> lock(coop_mu);
  for (const auto& d : coop_answer)
    if (d.first == dev) return d.second;
  return -1;
}
void coop_record(int dev, int ok) {
  std::lock_guard<std::mutex> lock(coop_mu);
  for (auto& d : coop_answer)
    if (d.first == dev) { d.second = ok; return; }
  coop_answer.push_back({dev, ok});
}

// A launch of several iterations asks to be cooperative: its CTAs wait for one another at the
// grid barrier, and a cooperative launch is scheduled only when all of them can be resident at
// once, also beside kernels of other streams that hold SMs.  A device that refuses the attribute
// together with clusters is remembered and launched plainly (the launch is one wave of clusters
// either way).  The first attempt is never made during stream capture, where a refused launch
// would end the capture.
template <int BN, int MODE, bool PAIR>
cudaError_t csk_launch(const CskParams& P, int tiles, cudaStream_t s) {
  const int cluster = P.S * (PAIR ? 2 : 1);
  cudaLaunchAttribute attrs[2];
  cudaLaunchConfig_t cfg = csk_config<BN, PAIR>(tiles * cluster, cluster, &attrs[0], s);
  if (P.iters > 1) {
    int dev = 0;
    cudaGetDevice(&dev);
    int known = coop_state(dev);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (known < 0 && (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)) {
      cudaGetLastError();
      known = 0;   // decide outside capture; this launch goes plain
    } else if (known != 0) {
      attrs[1].id = cudaLaunchAttributeCooperative;
      attrs[1].val.cooperative = 1;
      cfg.numAttrs = 2;
      const cudaError_t e = cudaLaunchKernelEx(&cfg, k_tc_csk<BN, MODE, PAIR>, P);
      if (known < 0) coop_record(dev, e == cudaSuccess ? 1 : 0);
      if (e == cudaSuccess || known > 0) return e;
      cudaGetLastError();
      cfg.numAttrs = 1;
    }
  }
  return cudaLaunchKernelEx(&cfg, k_tc_csk<BN, MODE, PAIR>, P);
}

}  // namespace

int tc_csk_cooperative() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  return coop_state(dev);
}

namespace {

}  // namespace

int tc_csk_factor(int tile_n, int num_tiles, int kblocks, int sms) {
  if (tile_n != 64 && tile_n != 128 && tile_n != 256) return 0;
  if (num_tiles < 1 || 2 * num_tiles > sms) return 0;
  for (int S = 8; S >= 2; --S) {
    if (kblocks / S < CSK_MIN_KB || num_tiles * S > sms) continue;
    const int fit = tile_n == 64    ? csk_max_clusters<64, false>(S)
                    : tile_n == 128 ? csk_max_clusters<128, false>(S)
                                    : csk_max_clusters<256, false>(S);
    if (fit >= num_tiles) return S;   // every cluster resident at once: one wave
  }
  return 0;
}

int tc_cskp_factor(int bn, int pair_tiles, int kblocks, int sms) {
  if (bn != 128 && bn != 256) return 0;
  if (pair_tiles < 1 || 4 * pair_tiles > sms) return 0;
  for (int S = 4; S >= 2; --S) {   // clusters of 2 S <= 8 CTAs (portable size)
    if (kblocks / S < CSK_MIN_KB || pair_tiles * 2 * S > sms) continue;
    const int fit = bn == 128 ? csk_max_clusters<128, true>(2 * S) : csk_max_clusters<256, true>(2 * S);
    if (fit >= pair_tiles) return S;
  }
  return 0;
}

cudaError_t launch_tc_csk(const TcPlan& plan, int which_x, const EpiArgs& a, int mode, int iters, uint64_t timeout_ns,
                          cudaStream_t s) {
  if (!plan.ready || plan.csk < 2 || plan.csk > 8 || plan.pair || !plan.csk_ws) return cudaErrorInvalidValue;
  if (plan.csk_pair && (plan.csk > 4 || (plan.tile_n != 64 && plan.tile_n != 128))) return cudaErrorInvalidValue;
  if (mode != EPI_UPDATE && mode != EPI_EVAL) return cudaErrorInvalidValue;
  if (iters < 1 || (iters > 1 && (mode != EPI_UPDATE || !plan.gbar || which_x > 1 || a.mu))) return cudaErrorInvalidValue;
  // shared-memory attributes (also set by the occupancy query, which a cached decision skips)
  static PerDevice per_device;
  const cudaError_t attr_err = per_device.once([] {
    cudaError_t r = csk_set_attrs<64, false>();
    r = r == cudaSuccess ? csk_set_attrs<128, false>() : r;
    r = r == cudaSuccess ? csk_set_attrs<256, false>() : r;
    r = r == cudaSuccess ? csk_set_attrs<128, true>() : r;
    r = r == cudaSuccess ? csk_set_attrs<256, true>() : r;
    return r;
  });
  if (attr_err != cudaSuccess) return attr_err;
  CskParams P;
  memset(&P, 0, sizeof(P));
  P.mapA = plan.mapA;
  if (mode == EPI_UPDATE) {
    // iteration j reads operand buffer (which_x + j) & 1 and writes the other one
    P.mapX[0] = plan.mapX[0];
    P.mapX[1] = plan.mapX[1];
    P.x0 = which_x & 1;
    P.xop[which_x & 1] = const_cast<void*>(a.Xin);
    P.xop[(which_x & 1) ^ 1] = a.Xout;
    P.bits_last = a.bits_out;
  } else {
    P.mapX[0] = plan.mapX[which_x];
    P.x0 = 0;
  }
  P.epi = a;
  P.iters = iters;
  P.gbar = plan.gbar;
  P.ws = plan.csk_ws;
  P.kblocks = (a.n + TC_BK - 1) / TC_BK;
  P.S = plan.csk;
  P.timeout_ns = timeout_ns;
  if (plan.csk_pair) {
    // tiles of 256 rows x 2 tile_n restarts (the operand map's box holds one CTA's half)
    const int bn = 2 * plan.tile_n;
    P.n_tiles = (a.B + bn - 1) / bn;
    const int tiles = ((a.n + 2 * TC_BM - 1) / (2 * TC_BM)) * P.n_tiles;
    if (bn == 128)
      return mode == EPI_UPDATE ? csk_launch<128, EPI_UPDATE, true>(P, tiles, s) : csk_launch<128, EPI_EVAL, true>(P, tiles, s);
    return mode == EPI_UPDATE ? csk_launch<256, EPI_UPDATE, true>(P, tiles, s) : csk_launch<256, EPI_EVAL, true>(P, tiles, s);
  }
  P.n_tiles = (a.B + plan.tile_n - 1) / plan.tile_n;
  const int tiles = ((a.n + TC_BM - 1) / TC_BM) * P.n_tiles;
  switch (plan.tile_n) {
    case 64:
      return mode == EPI_UPDATE ? csk_launch<64, EPI_UPDATE, false>(P, tiles, s) : csk_launch<64, EPI_EVAL, false>(P, tiles, s);
    case 128:
      return mode == EPI_UPDATE ? csk_launch<128, EPI_UPDATE, false>(P, tiles, s)
                                : csk_launch<128, EPI_EVAL, false>(P, tiles, s);
    default:
      return mode == EPI_UPDATE ? csk_launch<256, EPI_UPDATE, false>(P, tiles, s)
                                : csk_launch<256, EPI_EVAL, false>(P, tiles, s);
  }
}

}  // namespace sbo
