// Device helpers shared by the tcgen05 kernels (k_tc.cu: one CTA per tile; k_tc2.cu: CTA
// pairs): mbarrier / TMA / tcgen05 PTX wrappers and the PDBO epilogue on accumulator chunks.
#pragma once
#include "sbo_internal.h"

namespace sbo {

constexpr int TC_BM = 128;   // accumulator rows per CTA (TMEM lanes)
constexpr int TC_BK = 64;    // BF16 values per 128-byte swizzle row = one k-block

// ---- PTX wrappers ----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the deadline passed or another role aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t deadline,
                                          const volatile int* abort_flag) {
  uint32_t spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++spins & 31u) == 0u) {
      if (*abort_flag) return false;
      if (globaltimer_ns() > deadline) return false;
    }
  }
  return true;
}
// Warp-uniform bounded wait: lane 0 polls, the outcome is broadcast to the whole warp.
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, uint64_t deadline,
                                               const volatile int* abort_flag, int lane) {
  int ok = 1;
  if (lane == 0) ok = mbar_wait(bar, parity, deadline, abort_flag) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"(map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// K-major operand tile with 128-byte swizzle: rows of 128 B, 8-row atoms 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                   // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                   // SWIZZLE_128B
  return d;
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// ---- CTA pairs and clusters (tcgen05 cta_group::2) ----------------------------------------------
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared::cluster address of the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cl(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cl(uint32_t bar, uint32_t parity, uint64_t deadline,
                                             const volatile int* abort_flag) {
  uint32_t spins = 0;
  while (!mbar_try_wait_cl(bar, parity)) {
    if ((++spins & 31u) == 0u) {
      if (*abort_flag) return false;
      if (globaltimer_ns() > deadline) return false;
    }
  }
  return true;
}
__device__ __forceinline__ bool mbar_wait_cl_warp(uint32_t bar, uint32_t parity, uint64_t deadline,
                                                  const volatile int* abort_flag, int lane) {
  int ok = 1;
  if (lane == 0) ok = mbar_wait_cl(bar, parity, deadline, abort_flag) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}
__device__ __forceinline__ void mma_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive (once) on the barrier at this shared-memory offset in the CTAs of `mask` (cluster ranks;
// both CTAs of the issuing pair: 0x3 in a cluster of two, 0x3 << rank in a larger one)
__device__ __forceinline__ void commit_pair_multicast(uint32_t bar, uint16_t mask = 0x3) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}
__device__ __forceinline__ void commit_pair_local(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// TMA load whose completion is counted on an mbarrier of either CTA of the pair
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, uint32_t cluster_bar, int x,
                                                 int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(dst),
      "l"(map), "r"(cluster_bar), "r"(x), "r"(y)
      : "memory");
}

// ---- epilogue pieces --------------------------------------------------------------------------
// Global loads one 32-column chunk needs before the accumulator is read.
template <int MODE>
__device__ __forceinline__ void epi_load(const EpiArgs& a, int64_t i, bool row_ok, int64_t rbase, float (&u)[32],
                                         float (&v)[32]) {
  if (MODE == EPI_UPDATE) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int64_t r = rbase + j;
      const bool ok = row_ok && r < a.B;
      const int64_t idx = r * a.ld + i;
      u[j] = ok ? a.Xm[idx] : 0.0f;
      v[j] = ok ? (a.mu ? a.mu[r] : a.Y[idx]) : 0.0f;   // single-constraint form: the restart's dual
    }
  } else if (MODE == EPI_EVAL) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int64_t r = rbase + j;
      const bool ok = row_ok && r < a.B;
      u[j] = ok ? __bfloat162float(static_cast<const __nv_bfloat16*>(a.Xin)[r * a.ld + i]) : 0.0f;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int64_t r = rbase + j;
      const bool ok = row_ok && r < a.B;
      const int64_t idx = r * a.ld + i;
      u[j] = ok ? a.Xl[idx] : 0.0f;
      v[j] = ok ? a.Yl[idx] : 0.0f;
    }
  }
}

// One chunk of the PDBO update for a compile-time constraint function GK, with one dual per
// coordinate (SINGLE false) or per restart (SINGLE true: the warp's 32 rows also add up g(x^t) per
// restart into row `prow` of the partial sums).  The kind and the form are uniform per launch, so
// epi_apply picks one specialisation per chunk instead of testing them per element.
template <int GK, bool SINGLE>
__device__ __forceinline__ void epi_update(const EpiArgs& a, int64_t i, bool row_ok, float cpi, int64_t rbase,
                                           int lane, const float (&g)[32], const float (&u)[32], const float (&v)[32],
                                           int prow) {
  if (SINGLE) {
    float gv[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int64_t r = rbase + j;
      gv[j] = 0.0f;
      if (row_ok && r < a.B) {
        const int64_t idx = r * a.ld + i;
        const float x = u[j], y = v[j];
        const float gx = g_val(x, GK);
        const float d = g[j] + cpi + y * g_der(x, GK);
        float yn;
        const float xn = pdbo_update(x, y, d, gx, a.alpha, a.beta, a.delta, a.grad_tol, &yn);
        if (a.Gd) a.Gd[idx] = d;
        a.Xm[idx] = xn;
        static_cast<__nv_bfloat16*>(a.Xout)[idx] = __float2bfloat16_rn(xn);
        if (a.bits_out)
          static_cast<__nv_bfloat16*>(a.bits_out)[idx] = __float2bfloat16_rn(xn > 0.5f ? 1.0f : 0.0f);
        gv[j] = gx;
      }
    }
    const float sum = warp_transpose_sum32(gv, lane);
    if (rbase + lane < a.B) a.gpart[(int64_t)prow * a.gpart_ld + rbase + lane] = sum;
  } else if (row_ok) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int64_t r = rbase + j;
      if (r < a.B) {
        const int64_t idx = r * a.ld + i;
        const float x = u[j], y = v[j];
        const float d = g[j] + cpi + y * g_der(x, GK);
        float yn;
        const float xn = pdbo_update(x, y, d, g_val(x, GK), a.alpha, a.beta, a.delta, a.grad_tol, &yn);
        if (a.Gd) a.Gd[idx] = d;
        a.Xm[idx] = xn;
        a.Y[idx] = yn;
        static_cast<__nv_bfloat16*>(a.Xout)[idx] = __float2bfloat16_rn(xn);
        if (a.bits_out)
          static_cast<__nv_bfloat16*>(a.bits_out)[idx] = __float2bfloat16_rn(xn > 0.5f ? 1.0f : 0.0f);
      }
    }
  }
}

// One chunk of the epilogue given the accumulator values g (= (A x_r)_i for 32 restarts r).  In
// the single-constraint form (a.mu set) the warp's 32 rows also add up g(x^t) per restart into
// row `prow` of the partial sums.
template <int MODE>
__device__ __forceinline__ void epi_apply(const EpiArgs& a, int64_t i, bool row_ok, float cpi, long long cp2,
                                          int64_t rbase, int lane, const float (&g)[32], const float (&u)[32],
                                          const float (&v)[32], int prow = 0) {
  if (MODE == EPI_UPDATE) {
    if (a.gkind == G_ENTROPY) {
      if (a.mu) epi_update<G_ENTROPY, true>(a, i, row_ok, cpi, rbase, lane, g, u, v, prow);
      else epi_update<G_ENTROPY, false>(a, i, row_ok, cpi, rbase, lane, g, u, v, prow);
    } else {
      if (a.mu) epi_update<G_QUAD, true>(a, i, row_ok, cpi, rbase, lane, g, u, v, prow);
      else epi_update<G_QUAD, false>(a, i, row_ok, cpi, rbase, lane, g, u, v, prow);
    }
  } else if (MODE == EPI_EVAL) {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int64_t r = rbase + j;
      long long w = (u[j] != 0.0f) ? (long long)g[j] + cp2 : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      if (lane == 0 && r < a.B && w != 0) atomicAdd(&a.F2[r], (unsigned long long)w);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int64_t r = rbase + j;
      float lv = 0.0f;
      if (row_ok && r < a.B) {
        const int64_t idx = r * a.ld + i;
        const float x = u[j], y = v[j];
        const float gx = g_val(x, a.gkind);
        const float sc = a.gout ? a.gout[r] : 1.0f;
        if (a.GX) a.GX[idx] = sc * (g[j] + cpi + y * g_der(x, a.gkind));
        if (a.GY) a.GY[idx] = sc * gx;
        lv = 0.5f * x * g[j] + cpi * x + y * gx;
      }
      if (a.L) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lv += __shfl_xor_sync(0xffffffffu, lv, o);
        if (lane == 0 && r < a.B) atomicAdd(&a.L[r], lv);
      }
    }
  }
}

}  // namespace sbo
