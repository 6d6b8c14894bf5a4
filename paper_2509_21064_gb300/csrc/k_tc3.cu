// Dense contraction for problems with fewer output tiles than SMs: split-K inside a thread-block
// cluster, reduced through distributed shared memory.
//
// With B restarts and n rows there are ceil(n/128) * ceil(B/BN) tiles of the accumulator; when
// that is well below the SM count (n = 5,000 with B = 256 gives 40 tiles of 128 x 256 on 152
// SMs), one CTA per tile leaves most SMs idle and runs its epilogue with nothing to overlap.
// Here a cluster of S CTAs shares one tile:
//   * CTA s of the cluster runs k-blocks [s KB/S, (s+1) KB/S) with the same warp-specialised
//     TMA / tcgen05.mma pipeline as k_tc.cu (one accumulator of BN TMEM columns);
//   * its epilogue warps copy the partial accumulator into the CTA's own (now idle) stage
//     buffers, column-major [column][row];
//   * after a cluster barrier, CTA s owns the 32-column chunks [s NC/S, (s+1) NC/S) of the tile
//     (NC = BN/32): it sums the S partials of those columns in split order 0..S-1, reading every
//     CTA's shared memory with ld.shared::cluster (lane = row, so each load of a warp is one
//     contiguous 128-byte run), so the sum does not depend on timing, and applies the PDBO
//     update / exact objective to them;
//   * a second cluster barrier keeps every CTA's shared memory alive until all reads are done.
// The epilogue is thereby spread over S SMs instead of one, and no partial tile goes through
// global memory.  (Measured against two alternatives on n = 2,000-5,000, B = 256: pushing the
// partials to their owners with st.shared::cluster, and 16-byte row-major pulls, were both
// slower than these one-word pulls.)  Every mbarrier wait is bounded (globaltimer budget); a CTA
// that gives up sets ERR_TIMEOUT, drains its own copies and MMAs, skips the reduction and still
// reaches both cluster barriers, which all CTAs therefore reach in bounded time.
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

template <int BN>
struct CskCfg {
  static constexpr int A_BYTES = TC_BM * TC_BK * 2;
  static constexpr int B_BYTES = BN * TC_BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES =
      (CSK_SMEM_BUDGET - 2048) / STAGE_BYTES > 8 ? 8 : (CSK_SMEM_BUDGET - 2048) / STAGE_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /* align */ + 1024 /* barriers */;
  static constexpr int TMEM_COLS = BN;
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                    ((uint32_t)(TC_BM >> 4) << 24);
  static_assert(STAGES * STAGE_BYTES >= BN * TC_BM * 4, "the partial tile must fit in the stage buffers");
};

struct CskParams {
  CUtensorMap mapA;
  CUtensorMap mapX;
  EpiArgs epi;
  int n_tiles, kblocks, S;
  uint64_t timeout_ns;
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
// One word of a cluster peer's shared memory.
__device__ __forceinline__ float csk_ld_remote(uint32_t cluster_addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(cluster_addr) : "memory");
  return v;
}
template <int BN, int MODE>
__global__ void __launch_bounds__(CSK_THREADS, 1) k_tc_csk(const __grid_constant__ CskParams P) {
  using C = CskCfg<BN>;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* tiles = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(tiles + C::STAGES * C::STAGE_BYTES);
  uint64_t* full_bar = bars;                   // [STAGES]
  uint64_t* empty_bar = bars + C::STAGES;      // [STAGES]
  uint64_t* tfull_bar = bars + 2 * C::STAGES;  // accumulator complete
  uint64_t* drain_bar = tfull_bar + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain_bar + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int S = P.S;
  const uint32_t s = csk_rank();
  const int tile = (int)(blockIdx.x / (unsigned)S);
  const int m_tile = tile / P.n_tiles, n_tile = tile % P.n_tiles;
  const int kb0 = (int)((int64_t)s * P.kblocks / S);
  const int kb1 = (int)((int64_t)(s + 1) * P.kblocks / S);
  const int nk = kb1 - kb0;
  const EpiArgs& a = P.epi;
  const uint64_t deadline = globaltimer_ns() + P.timeout_ns;

  if (threadIdx.x == 0) {
    for (int q = 0; q < C::STAGES; ++q) {
      mbar_init(smem_u32(&full_bar[q]), 1);
      mbar_init(smem_u32(&empty_bar[q]), 1);
    }
    mbar_init(smem_u32(tfull_bar), 1);
    mbar_init(smem_u32(drain_bar), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tma_prefetch_map(&P.mapA);
    tma_prefetch_map(&P.mapX);
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
      for (int jk = 0; jk < nk; ++jk) {
        const int kb = kb0 + jk;
        if (!mbar_wait(smem_u32(&empty_bar[stage]), phase ^ 1u, deadline, vabort)) { ok = false; break; }
        const uint32_t fb = smem_u32(&full_bar[stage]);
        mbar_expect_tx(fb, (uint32_t)C::STAGE_BYTES);
        uint8_t* sa = tiles + stage * C::STAGE_BYTES;
        tma_load_2d(smem_u32(sa), &P.mapA, fb, kb * TC_BK, m_tile * TC_BM);
        tma_load_2d(smem_u32(sa + C::A_BYTES), &P.mapX, fb, kb * TC_BK, n_tile * BN);
        issued_mask |= 1u << stage;
        issued_parity = (issued_parity & ~(1u << stage)) | (phase << stage);
        if (++stage == C::STAGES) { stage = 0; phase ^= 1u; }
      }
      if (!ok) {
        atomicOr(a.err, ERR_TIMEOUT);
        *abort_flag = 1;
        const uint64_t dl2 = globaltimer_ns() + 200000000ull;
        const int zero = 0;
        for (int q = 0; q < C::STAGES; ++q)
          if (issued_mask & (1u << q)) mbar_wait(smem_u32(&full_bar[q]), (issued_parity >> q) & 1u, dl2, &zero);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true, issued_any = false;
      for (int jk = 0; jk < nk; ++jk) {
        if (!mbar_wait(smem_u32(&full_bar[stage]), phase, deadline, vabort)) { ok = false; break; }
        tc_fence_after();
        const uint32_t sa = smem_u32(tiles + stage * C::STAGE_BYTES);
        const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk)
          tc_mma(tmem_base, sw128_desc(sa + kk * 32), sw128_desc(sb + kk * 32), C::IDESC,
                 (jk > 0 || kk > 0) ? 1u : 0u);
        issued_any = true;
        tc_commit(smem_u32(&empty_bar[stage]));
        if (++stage == C::STAGES) { stage = 0; phase ^= 1u; }
      }
      if (ok) {
        tc_commit(smem_u32(tfull_bar));
      } else {
        atomicOr(a.err, ERR_TIMEOUT);
        *abort_flag = 1;
        if (issued_any) {
          tc_commit(smem_u32(drain_bar));
          const int zero = 0;
          mbar_wait(smem_u32(drain_bar), 0, globaltimer_ns() + 200000000ull, &zero);
        }
      }
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------------ partial tile -> smem
    // Every MMA of this CTA has completed when tfull fires, so the stage buffers are idle: the
    // accumulator (lane = row) goes to part[column][row].
    const int wg = (warp - 4) >> 2;
    const int wq = warp & 3;
    const int row = wq * 32 + lane;
    if (mbar_wait_warp(smem_u32(tfull_bar), 0, deadline, vabort, lane)) {
      tc_fence_after();
      float* part = reinterpret_cast<float*>(tiles);
      float g[32];
      for (int c0 = wg * (BN / 2); c0 < (wg + 1) * (BN / 2); c0 += 32) {
        tmem_ld32(tmem_base + ((uint32_t)(wq * 32) << 16) + (uint32_t)c0, g);
#pragma unroll
        for (int j = 0; j < 32; ++j) part[(c0 + j) * TC_BM + row] = g[j];
      }
    } else if (lane == 0) {
      atomicOr(a.err, ERR_TIMEOUT);
      *abort_flag = 1;
    }
  }

  __syncwarp();
  tc_fence_before();
  csk_cluster_sync();   // every CTA's partial tile is in its shared memory
  tc_fence_after();

  if (*vabort == 0) {
    // ------------------------------------------------------------------ reduction + epilogue
    // All twelve warps take part (the producer and MMA warps are idle by now): three groups of
    // four warps, each over the tile's 128 rows, share the CTA's chunks round-robin.  The rows
    // come from shared memory, not TMEM, so any warp may take any rows.
    const int wg = warp >> 2;
    const int wq = warp & 3;
    const int row = wq * 32 + lane;
    const int64_t i = (int64_t)m_tile * TC_BM + row;
    const bool row_ok = i < a.n;
    const float cpi = row_ok ? a.cp[i] : 0.0f;
    const long long cp2 = (MODE == EPI_EVAL && row_ok) ? 2 * (long long)a.cp64[i] : 0;
    constexpr int NC = BN / 32;
    const int q0 = (int)((int)s * NC / S), q1 = (int)(((int)s + 1) * NC / S);
    const uint32_t part_local = smem_u32(tiles);
    float u[32], v[32], g[32];
    for (int q = q0 + wg; q < q1; q += CSK_THREADS / 128) {
      const int c0 = q * 32;
      const int64_t rbase = (int64_t)n_tile * BN + c0;
      epi_load<MODE>(a, i, row_ok, rbase, u, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) g[j] = 0.0f;
      for (int sp = 0; sp < S; ++sp) {      // split order: the sum does not depend on timing
        const uint32_t base = csk_mapa(part_local, (uint32_t)sp) + (uint32_t)((c0 * TC_BM + row) * 4);
#pragma unroll
        for (int j = 0; j < 32; ++j) g[j] += csk_ld_remote(base + (uint32_t)(j * TC_BM * 4));
      }
      epi_apply<MODE>(a, i, row_ok, cpi, cp2, rbase, lane, g, u, v, m_tile * 4 + wq);
    }
  }

  __syncwarp();
  tc_fence_before();
  csk_cluster_sync();   // no CTA leaves while another may still read its shared memory
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
  }
}

template <int BN, int MODE>
cudaError_t csk_set_attr() {
  return cudaFuncSetAttribute(k_tc_csk<BN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, CskCfg<BN>::SMEM);
}

template <int BN>
cudaLaunchConfig_t csk_config(int grid, int S, cudaLaunchAttribute* attr, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(CSK_THREADS);
  cfg.dynamicSmemBytes = CskCfg<BN>::SMEM;
  cfg.stream = s;
  attr->id = cudaLaunchAttributeClusterDimension;
  attr->val.clusterDim.x = (unsigned)S;
  attr->val.clusterDim.y = 1;
  attr->val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Clusters of S CTAs of this kernel that fit on the current device at once (0 if none), queried
// once per (device, S): the attributes and the occupancy answer belong to the device's context.
template <int BN>
int csk_max_clusters(int S) {
  static std::mutex mu;
  static std::vector<std::pair<int, std::array<int, 9>>> cache;   // (device, answer per S)
  if (S < 2 || S > 8) return 0;
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
  int& slot = (*row)[S];
  if (slot >= 0) return slot;
  slot = 0;
  if (csk_set_attr<BN, EPI_UPDATE>() != cudaSuccess || csk_set_attr<BN, EPI_EVAL>() != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchAttribute attr;
  cudaLaunchConfig_t cfg = csk_config<BN>(S * 16, S, &attr, nullptr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_tc_csk<BN, EPI_UPDATE>, &cfg) == cudaSuccess) slot = n;
  cudaGetLastError();
  return slot;
}

template <int BN, int MODE>
cudaError_t csk_launch(const CskParams& P, int tiles, cudaStream_t s) {
  cudaLaunchAttribute attr;
  cudaLaunchConfig_t cfg = csk_config<BN>(tiles * P.S, P.S, &attr, s);
  return cudaLaunchKernelEx(&cfg, k_tc_csk<BN, MODE>, P);
}

}  // namespace

int tc_csk_factor(int tile_n, int num_tiles, int kblocks, int sms) {
  if (tile_n != 64 && tile_n != 128 && tile_n != 256) return 0;
  if (num_tiles < 1 || 2 * num_tiles > sms) return 0;
  for (int S = 8; S >= 2; --S) {
    if (kblocks / S < CSK_MIN_KB || num_tiles * S > sms) continue;
    const int fit = tile_n == 64 ? csk_max_clusters<64>(S) : tile_n == 128 ? csk_max_clusters<128>(S)
                                                                           : csk_max_clusters<256>(S);
    if (fit >= num_tiles) return S;   // every cluster resident at once: one wave
  }
  return 0;
}

cudaError_t launch_tc_csk(const TcPlan& plan, int which_x, const EpiArgs& a, int mode, uint64_t timeout_ns,
                          cudaStream_t s) {
  if (!plan.ready || plan.csk < 2 || plan.csk > 8 || plan.pair) return cudaErrorInvalidValue;
  if (mode != EPI_UPDATE && mode != EPI_EVAL) return cudaErrorInvalidValue;
  // shared-memory attributes (also set by the occupancy query, which a cached decision skips)
  static PerDevice per_device;
  const cudaError_t attr_err = per_device.once([] {
    cudaError_t r = cudaSuccess;
    r = r == cudaSuccess ? csk_set_attr<64, EPI_UPDATE>() : r;
    r = r == cudaSuccess ? csk_set_attr<64, EPI_EVAL>() : r;
    r = r == cudaSuccess ? csk_set_attr<128, EPI_UPDATE>() : r;
    r = r == cudaSuccess ? csk_set_attr<128, EPI_EVAL>() : r;
    r = r == cudaSuccess ? csk_set_attr<256, EPI_UPDATE>() : r;
    r = r == cudaSuccess ? csk_set_attr<256, EPI_EVAL>() : r;
    return r;
  });
  if (attr_err != cudaSuccess) return attr_err;
  CskParams P;
  memset(&P, 0, sizeof(P));
  P.mapA = plan.mapA;
  P.mapX = plan.mapX[which_x];
  P.epi = a;
  P.n_tiles = (a.B + plan.tile_n - 1) / plan.tile_n;
  P.kblocks = (a.n + TC_BK - 1) / TC_BK;
  P.S = plan.csk;
  P.timeout_ns = timeout_ns;
  const int tiles = ((a.n + TC_BM - 1) / TC_BM) * P.n_tiles;
  switch (plan.tile_n) {
    case 64: return mode == EPI_UPDATE ? csk_launch<64, EPI_UPDATE>(P, tiles, s) : csk_launch<64, EPI_EVAL>(P, tiles, s);
    case 128:
      return mode == EPI_UPDATE ? csk_launch<128, EPI_UPDATE>(P, tiles, s) : csk_launch<128, EPI_EVAL>(P, tiles, s);
    default:
      return mode == EPI_UPDATE ? csk_launch<256, EPI_UPDATE>(P, tiles, s) : csk_launch<256, EPI_EVAL>(P, tiles, s);
  }
}

}  // namespace sbo
