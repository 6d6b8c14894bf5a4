// Dense contraction on CTA pairs (tcgen05.mma.cta_group::2): each pair of SMs computes a
// 256 (rows of A) x 256 (restarts) tile with the PDBO epilogue fused, as k_tc.cu does for one
// SM and 128 x tile_n.
//
//   D[i][r] = sum_k A[i][k] * Xb[r][k]      (A: n x n BF16, Xb: B x n BF16, both K-major)
//
// Why pairs: the kernel is fed from L2 by TMA.  A single SM computing 128 x 256 needs 48 KB of
// operands per 4.2 MFLOP; in a pair every SM stages only its own 128 rows of A and its own 128
// restarts of X (32 KB per stage) while each MMA instruction covers 256 x 256, so the bytes each
// SM must bring in per flop drop by a third and six stages fit in shared memory instead of four.
//
// Roles (384 threads per CTA, cluster of 2; rank 0 = leader, rank 1 = peer):
//   warp 0 (both)    TMA producer of the CTA's own halves: A rows m*256 + 128*rank .. +127,
//                    X rows n*256 + 128*rank .. +127; the copies of both CTAs complete on the
//                    leader's full barrier (cta_group::2 copies), which the leader arms for both
//   warp 1 (leader)  single-thread MMA issuer, M=256 N=256 K=16; its commits are multicast to
//                    the empty / accumulator-full barriers of both CTAs
//   warps 4-11 (both) epilogue of the CTA's 128 rows x 256 restarts (same code as k_tc.cu); every
//                    warp then arrives on the leader's accumulator-empty barrier
// TMEM (512 columns, two 256-column accumulators) is allocated by both CTAs with cta_group::2.
// Every wait is bounded; cross-CTA synchronisation uses cluster-scope release/acquire.
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "tc_common.cuh"

namespace sbo {

namespace {

constexpr int P_THREADS = 384;
constexpr int P_BN = 256;          // restarts per pair tile
constexpr int P_HALF = 128;        // restarts staged per CTA
constexpr int P_A_BYTES = TC_BM * TC_BK * 2;
constexpr int P_B_BYTES = P_HALF * TC_BK * 2;
constexpr int P_STAGE_BYTES = P_A_BYTES + P_B_BYTES;  // 32 KB
constexpr int P_STAGES = 6;
constexpr int P_SMEM = P_STAGES * P_STAGE_BYTES + 1024 /* align */ + 1024 /* barriers */;
constexpr int P_TMEM_COLS = 2 * P_BN;
constexpr uint32_t P_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(P_BN >> 3) << 17) |
                             ((uint32_t)(256 >> 4) << 24);

struct PairParams {
  CUtensorMap mapA;   // box 64 x 128
  CUtensorMap mapX;   // box 64 x 128
  EpiArgs epi;
  int n, m_tiles, n_tiles, num_tiles, kblocks;
  int dp_tiles, splits, sk_units;
  float* ws;          // split-K partials [unit][rank][256 cols][128 rows]
  int* counters;      // [tail tile][rank][8 slices]
  uint64_t timeout_ns;
};

struct PairWork {
  int tile, kb0, kb1, unit;
};
__device__ __forceinline__ bool pair_work(const PairParams& P, int j, PairWork& w) {
  const int G = gridDim.x >> 1, c = blockIdx.x >> 1;
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

template <int MODE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(P_THREADS, 1) k_tc_pair(const __grid_constant__ PairParams P) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* tiles = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(tiles + P_STAGES * P_STAGE_BYTES);
  uint64_t* full_bar = bars;                       // [STAGES]
  uint64_t* empty_bar = bars + P_STAGES;           // [STAGES]
  uint64_t* tfull_bar = bars + 2 * P_STAGES;       // [2]
  uint64_t* tempty_bar = bars + 2 * P_STAGES + 2;  // [2] (used in the leader)
  uint64_t* drain_bar = bars + 2 * P_STAGES + 4;   // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * P_STAGES + 5);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const uint64_t deadline = globaltimer_ns() + P.timeout_ns;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);  // leader: its arrive.expect_tx covers both CTAs' copies
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&tfull_bar[a]), 1);
      mbar_init(smem_u32(&tempty_bar[a]), 16);  // 8 epilogue warps in each of the two CTAs
    }
    mbar_init(smem_u32(drain_bar), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tma_prefetch_map(&P.mapA);
    tma_prefetch_map(&P.mapX);
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)P_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync_all();   // barriers of both CTAs initialised, TMEM allocated in both
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const volatile int* vabort = abort_flag;

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer (both CTAs)
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, issued_parity = 0;
      bool ok = true;
      PairWork w;
      for (int j = 0; ok && pair_work(P, j, w); ++j) {
        const int m_tile = w.tile / P.n_tiles, n_tile = w.tile % P.n_tiles;
        for (int kb = w.kb0; kb < w.kb1; ++kb) {
          if (!mbar_wait_cl(smem_u32(&empty_bar[stage]), phase ^ 1u, deadline, vabort)) { ok = false; break; }
          // both CTAs' copies complete on the leader's full barrier; the leader arms it for both
          const uint32_t fb = map_to_rank(smem_u32(&full_bar[stage]), 0);
          if (leader) mbar_expect_tx(smem_u32(&full_bar[stage]), (uint32_t)(2 * P_STAGE_BYTES));
          uint8_t* sa = tiles + stage * P_STAGE_BYTES;
          tma_load_2d_pair(smem_u32(sa), &P.mapA, fb, kb * TC_BK, m_tile * 256 + (int)rank * TC_BM);
          tma_load_2d_pair(smem_u32(sa + P_A_BYTES), &P.mapX, fb, kb * TC_BK, n_tile * P_BN + (int)rank * P_HALF);
          issued_mask |= 1u << stage;
          issued_parity = (issued_parity & ~(1u << stage)) | (phase << stage);
          if (++stage == P_STAGES) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) {
        atomicOr(P.epi.err, ERR_TIMEOUT);
        *abort_flag = 1;
        // copies of both CTAs are counted on the leader's barriers, so neither CTA can observe
        // its own copies land: give every copy in flight a generous fixed time instead
        if (issued_mask) {
          const uint64_t until = globaltimer_ns() + 2000000ull;
          while (globaltimer_ns() < until) {
          }
        }
        (void)issued_parity;
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer (leader)
    if (leader && lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true, issued_any = false;
      PairWork w;
      for (int j = 0; ok && pair_work(P, j, w); ++j) {
        if (!mbar_wait_cl(smem_u32(&tempty_bar[acc]), acc_phase ^ 1u, deadline, vabort)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * P_BN);
        for (int kb = w.kb0; kb < w.kb1; ++kb) {
          if (!mbar_wait_cl(smem_u32(&full_bar[stage]), phase, deadline, vabort)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(tiles + stage * P_STAGE_BYTES);
          const uint32_t sb = sa + P_A_BYTES;
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk)
            mma_pair(d_tmem, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), P_IDESC,
                     (kb > w.kb0 || kk > 0) ? 1u : 0u);
          issued_any = true;
          commit_pair_multicast(smem_u32(&empty_bar[stage]));
          if (++stage == P_STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        commit_pair_multicast(smem_u32(&tfull_bar[acc]));
        if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
      }
      if (!ok) {
        atomicOr(P.epi.err, ERR_TIMEOUT);
        *abort_flag = 1;
        if (issued_any) {
          commit_pair_local(smem_u32(drain_bar));
          const int zero = 0;
          mbar_wait_cl(smem_u32(drain_bar), 0, globaltimer_ns() + 200000000ull, &zero);
        }
      }
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------------ epilogue (both CTAs)
    constexpr int HALF = P_BN / 2;   // columns per epilogue warpgroup
    const int wg = (warp - 4) >> 2;
    const int wq = warp & 3;
    const int slice = wg * 4 + wq;
    const EpiArgs& a = P.epi;
    int acc = 0;
    uint32_t acc_phase = 0;
    PairWork w;
    for (int jw = 0; pair_work(P, jw, w); ++jw) {
      const int m_tile = w.tile / P.n_tiles, n_tile = w.tile % P.n_tiles;
      const int row = wq * 32 + lane;
      const int64_t i = (int64_t)m_tile * 256 + (int64_t)rank * TC_BM + row;
      const bool row_ok = i < a.n;
      const float cpi = row_ok ? a.cp[i] : 0.0f;
      const long long cp2 = (MODE == EPI_EVAL && row_ok) ? 2 * (long long)a.cp64[i] : 0;
      float u[32], v[32], g[32];
      bool ok = true;
      if (w.unit < 0) {
        bool waited = false;
        for (int c0 = wg * HALF; c0 < (wg + 1) * HALF; c0 += 32) {
          const int64_t rbase = (int64_t)n_tile * P_BN + c0;
          epi_load<MODE>(a, i, row_ok, rbase, u, v);
          if (!waited) {
            ok = mbar_wait_cl_warp(smem_u32(&tfull_bar[acc]), acc_phase, deadline, vabort, lane);
            if (!ok) break;
            tc_fence_after();
            waited = true;
          }
          tmem_ld32(tmem_base + ((uint32_t)(wq * 32) << 16) + (uint32_t)(acc * P_BN + c0), g);
          epi_apply<MODE>(a, i, row_ok, cpi, cp2, rbase, lane, g, u, v, (m_tile * 2 + (int)rank) * 4 + wq);
        }
      } else {
        ok = mbar_wait_cl_warp(smem_u32(&tfull_bar[acc]), acc_phase, deadline, vabort, lane);
        if (ok) {
          tc_fence_after();
          float* part = P.ws + ((size_t)w.unit * 2 + rank) * P_BN * TC_BM;  // [column][row]
          for (int c0 = wg * HALF; c0 < (wg + 1) * HALF; c0 += 32) {
            tmem_ld32(tmem_base + ((uint32_t)(wq * 32) << 16) + (uint32_t)(acc * P_BN + c0), g);
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
      // release the accumulator: one arrival per warp on the leader's barrier
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        const uint32_t tb = smem_u32(&tempty_bar[acc]);
        if (leader) mbar_arrive(tb);
        else mbar_arrive_remote(map_to_rank(tb, 0));
      }
      if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
      if (w.unit >= 0) {
        const int tail = w.tile - P.dp_tiles;
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0) {
          int* ctr = P.counters + tail * 16 + rank * 8 + slice;
          last = atomicAdd(ctr, 1) == P.splits - 1;
          if (last) *ctr = 0;  // ready for the next launch
          __threadfence();
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        __syncwarp();
        if (last) {
          __threadfence();
          for (int c0 = wg * HALF; c0 < (wg + 1) * HALF; c0 += 32) {
            const int64_t rbase = (int64_t)n_tile * P_BN + c0;
            epi_load<MODE>(a, i, row_ok, rbase, u, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) g[j] = 0.0f;
            for (int sp = 0; sp < P.splits; ++sp) {
              const float* ps = P.ws + ((size_t)(tail * P.splits + sp) * 2 + rank) * P_BN * TC_BM;
#pragma unroll
              for (int j = 0; j < 32; ++j) g[j] += __ldcg(ps + (size_t)(c0 + j) * TC_BM + row);
            }
            epi_apply<MODE>(a, i, row_ok, cpi, cp2, rbase, lane, g, u, v, (m_tile * 2 + (int)rank) * 4 + wq);
          }
        }
      }
    }
  }

  // both CTAs: every MMA into either CTA's TMEM has completed (its accumulator was consumed, or
  // the leader drained it) before TMEM is released
  tc_fence_before();
  cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"((uint32_t)P_TMEM_COLS)
                 : "memory");
  }
}

template <int MODE>
cudaError_t set_pair_attr() {
  return cudaFuncSetAttribute(k_tc_pair<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM);
}

}  // namespace

// Resident clusters of two CTAs on device `dev` (the current one), after setting the kernels'
// shared-memory attributes; 0 when the kernel cannot run there.
static int query_pair_clusters(int dev) {
  if (set_pair_attr<EPI_UPDATE>() != cudaSuccess || set_pair_attr<EPI_EVAL>() != cudaSuccess) return 0;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(sms & ~1));
  cfg.blockDim = dim3(P_THREADS);
  cfg.dynamicSmemBytes = P_SMEM;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = 2;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_tc_pair<EPI_UPDATE>, &cfg) != cudaSuccess) n = 0;
  cudaGetLastError();
  return n;
}

bool tc_pair_supported(int* max_clusters) {
  // per device: the attributes and the occupancy query belong to the current device's context
  static std::mutex mu;
  static std::vector<std::pair<int, int>> cache;   // (device, resident clusters)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lock(mu);
  int clusters = -1;
  for (const auto& c : cache)
    if (c.first == dev) clusters = c.second;
  if (clusters < 0) {
    clusters = query_pair_clusters(dev);
    cache.push_back({dev, clusters});
  }
  if (max_clusters) *max_clusters = clusters;
  return clusters > 0;
}

cudaError_t launch_tc_pair(const TcPlan& plan, int which_x, const EpiArgs& a, int mode, uint64_t timeout_ns,
                           cudaStream_t s) {
  int clusters = 0;
  if (!plan.ready || plan.tile_n != P_HALF || !tc_pair_supported(&clusters)) return cudaErrorInvalidValue;
  if (mode != EPI_UPDATE && mode != EPI_EVAL) return cudaErrorInvalidValue;
  PairParams P;
  memset(&P, 0, sizeof(P));
  P.mapA = plan.mapA;
  P.mapX = plan.mapX[which_x];
  P.epi = a;
  P.n = a.n;
  P.m_tiles = (a.n + 255) / 256;
  P.n_tiles = (a.B + P_BN - 1) / P_BN;
  P.num_tiles = P.m_tiles * P.n_tiles;
  P.kblocks = (a.n + TC_BK - 1) / TC_BK;
  P.timeout_ns = timeout_ns;
  // whole rounds over the clusters, the leftover tiles split along K (as for single CTAs)
  const TcSchedule sch = tc_schedule(P.num_tiles, P.kblocks, clusters, plan.ws != nullptr && plan.counters != nullptr,
                                     plan.max_splits);
  P.dp_tiles = sch.dp_tiles;
  P.splits = sch.splits;
  P.sk_units = sch.sk_units;
  P.ws = plan.ws;
  P.counters = plan.counters;
  const int grid = 2 * sch.grid;
  if (grid < 2) return cudaSuccess;
  if (mode == EPI_UPDATE) k_tc_pair<EPI_UPDATE><<<grid, P_THREADS, P_SMEM, s>>>(P);
  else k_tc_pair<EPI_EVAL><<<grid, P_THREADS, P_SMEM, s>>>(P);
  return cudaGetLastError();
}

}  // namespace sbo
