// Internal declarations of libsbo: the problem handle and the kernel launchers.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/sbo.h"
#include "common.cuh"

namespace sbo {

// Runs a set-up step once per device: function attributes and memory-pool settings belong to the
// context of the device that was current when they were set, so a process that uses several GPUs
// needs them on each.  The first result on a device is returned to every later caller on it.
class PerDevice {
 public:
  template <class F>
  cudaError_t once(F&& f) {
    int dev = 0;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu_);
    for (const auto& d : done_)
      if (d.first == dev) return d.second;
    const cudaError_t r = f();
    done_.push_back({dev, r});
    return r;
  }

 private:
  std::mutex mu_;
  std::vector<std::pair<int, cudaError_t>> done_;
};

enum Format : int { FMT_DENSE = 0, FMT_CSR = 1, FMT_MAXK = 2 };
enum Kernel : int { KER_AUTO = 0, KER_SIMT = 1, KER_TC = 2, KER_TINY = 3, KER_CSR = 4, KER_MAXK = 5 };
enum Layout : int { LAYOUT_RN = 0 /* [r][i] */, LAYOUT_NR = 1 /* [i][r] */ };

// ---- launchers (each returns the launch's cudaError_t) -----------------------------------
// k_setup.cu
// canonical A for the 64 x 64 tile pairs (I, J), I <= J, of tile columns [j0, j1) (rows of Q up
// to tile j1 must be present); c' = c + diag Q once all of Q is present
cudaError_t launch_canon_dense(const void* Qd, int q_bytes, int64_t n, int64_t j0, int64_t j1, void* A, int64_t lda,
                               int a_type, unsigned long long* rowsum, uint32_t* range_err, int64_t a_limit,
                               cudaStream_t s);
cudaError_t launch_canon_linear(const void* Qd, int q_bytes, const int32_t* cd, int64_t n, float* cp, int64_t* cp64,
                                cudaStream_t s);
cudaError_t launch_rowsum_check(const unsigned long long* rowsum, const int64_t* cp64, int64_t n,
                                uint32_t* range_err, cudaStream_t s);
cudaError_t launch_init_state(int n, int B, int64_t ld, int layout, uint64_t seed, float ybar,
                              const float* x0, const float* y0, float* Xm, void* Xop, int op_type, float* Y,
                              uint32_t* err, cudaStream_t s);
cudaError_t launch_to_operand(const float* X, int n, int B, int64_t ld_in, void* out, int64_t ld_out,
                              int op_type, cudaStream_t s);
cudaError_t launch_to_operand_t(const float* X, int n, int B, int64_t ld_in, void* out, int64_t ld_out,
                                int op_type, cudaStream_t s);
cudaError_t launch_bits_to_operand(const uint8_t* bits, int n, int count, void* out, int64_t ld_out,
                                   int layout, int op_type, cudaStream_t s);
cudaError_t launch_fill_i64(long long* p, int64_t count, long long v, cudaStream_t s);
cudaError_t launch_gather_state(const float* src, int n, int B, int64_t ld, int layout, float* dst_rn,
                                cudaStream_t s);
// k_simt.cu  (FP32 A, restart-major state)
cudaError_t launch_simt(const float* A, int64_t lda, const EpiArgs& a, int mode, cudaStream_t s);
// k_tiny.cu  (whole run in one launch for n <= 64)
struct TinyArgs {
  int n, B;
  int gkind;               // constraint function g (GKind)
  int64_t ld;
  const float* A;          // FP32 [n][lda]
  int64_t lda;
  const float* cp;
  const int64_t* cp64;
  float* X;                // FP32 [B][ld] master, in place
  float* Y;
  float alpha, beta, delta, grad_tol;
  int64_t t0, steps, K, T; // iterations t0+1 .. t0+steps; evaluate at multiples of K and at T
  long long* bestF;
  long long* bestT;
  uint8_t* bestBits;       // [B][ld]
  long long* trace;        // min_r F per evaluation, written at trace[e0 + e]
  int64_t e0, trace_cap;
  long long* evalF;        // scratch [B], F of the current evaluation
  float* G;                // if non-null: dL/dx of the latest iteration, [B][ld]
};
cudaError_t launch_tiny(const TinyArgs& a, cudaStream_t s);
// k_csr.cu  (variable-major state); pdl: launch as a programmatic dependent of the previous kernel.
// csr_partial_rows: blocks along the rows (= rows of single-constraint partial sums) at most.
// form (update only): CSR_FORM_RULE picks restarts per warp and the pipelined rows from n, B and
// L2; the others force one: one row per warp with 128 / 256 restarts, pipelined rows of 256, rows
// staged in shared memory; the *_STREAM forms are the first three with L2 eviction priorities on
// the own state (evict-first x and y, evict-last operand), for state that overflows L2.
enum CsrForm : int { CSR_FORM_RULE = 0, CSR_FORM_ROW1 = 1, CSR_FORM_ROW2 = 2, CSR_FORM_PIPE2 = 3, CSR_FORM_STAGED = 4,
                     CSR_FORM_ROW1_STREAM = 5, CSR_FORM_ROW2_STREAM = 6, CSR_FORM_PIPE2_STREAM = 7,
                     CSR_FORM_RESIDENT = 8 };
inline bool csr_form_streams(int form) { return form >= CSR_FORM_ROW1_STREAM && form <= CSR_FORM_PIPE2_STREAM; }
inline int csr_form_base(int form) { return csr_form_streams(form) ? form - 4 : form; }
cudaError_t launch_csr(const int32_t* rowptr, const int32_t* col, const void* val, int val_type,
                       const EpiArgs& a, int op_type, int mode, bool pdl, cudaStream_t s, int form = CSR_FORM_RULE);
// Resident form of the sparse update (k_csr.cu): the state of each CTA's rows stays in shared
// memory for `iters` iterations (one cooperative CTA per SM, grid barrier between iterations;
// operand buffers xop alternate from which_x, candidate bytes written by the last iteration when
// a.bits_out is set).  csr_res_shape: whether a graph with n rows, B restarts and at most nnz_max
// nonzeros in any CTA's rows (rows split evenly over min(n, sms) CTAs) fits, with its grid and
// shared memory.
bool csr_res_shape(int64_t n, int B, int sms, int nnz_max, int* grid, size_t* smem);
// CTAs of the resident form: min(n, sms - sms / 8), so that an evaluation can run beside it.
int csr_res_grid(int64_t n, int sms);
// eval_last: after the last iteration, the exact objective of its candidates (a.bits_out) is added
// into a.F2 as the evaluation kernel would add it (the commit kernel then reads and clears F2).
cudaError_t launch_csr_res(const int32_t* rowptr, const int32_t* col, const void* val, int val_type, const EpiArgs& a,
                           int op_type, int which_x, void* const xop[2], int iters, bool eval_last, int nnz_max,
                           int sms, unsigned int* gbar, uint64_t timeout_ns, cudaStream_t s);
int csr_partial_rows(int64_t n, int B);
// k_csr_staged.cu: the update with every row's operands staged in shared memory by bulk copies
// (CSR_FORM_STAGED); max_deg is the largest row length of A.  csr_staged_shape reports its stage
// layout and false when it does not apply (fewer than four stages fit).
bool csr_staged_shape(int64_t ld, int op_type, int max_deg, int* D, int* S, int* rc, size_t* smem);
cudaError_t launch_csr_staged(const int32_t* rowptr, const int32_t* col, const void* val, int val_type,
                              const EpiArgs& a, int op_type, int max_deg, int sms, bool pdl, uint64_t timeout_ns,
                              cudaStream_t s);
// k_maxk.cu  (Max-k-Cut: Z, X as [(i k + j) ld + r], y and parts as [i ld + r]; Z in EpiArgs::Xm)
cudaError_t launch_maxk(const int32_t* rowptr, const int32_t* col, const float* w, const EpiArgs& a, int kp, int mode,
                        cudaStream_t s);
cudaError_t launch_maxk_init(int n, int B, int64_t ld, int kp, uint64_t seed, float ybar, float* Z, float* Y, float* X,
                             cudaStream_t s);
cudaError_t launch_maxk_gather(const float* src, int n, int kp, int B, int64_t ld, float* dst, cudaStream_t s);
// k_best.cu
struct CommitArgs {
  const void* bits;              // candidate bits of this evaluation (operand type, state layout)
  int op_type, layout, n, B;
  int64_t ld;
  uint8_t* bestBits;             // per-restart best bits, state layout
  unsigned long long* F2;        // [B] 2F of the candidates (zeroed by the commit)
  long long *bestF, *bestT, *evalF, *trace, *n_evals, *t_last;
  long long trace_cap;
  unsigned int* ctr;             // arrival counter, zero between launches
};
cudaError_t launch_eval_commit(const CommitArgs& a, int64_t add, cudaStream_t s);
cudaError_t launch_eval_commit_group(const CommitArgs* d_tab, int members, int64_t max_inner, int64_t max_outer,
                                     int64_t add, cudaStream_t s);
// single-constraint form: mu[r] += beta * sum over the P rows of partial sums gpart[k][r]
cudaError_t launch_dual_single(float* mu, const float* gpart, int P, int64_t ldg, int B, float beta, cudaStream_t s);
cudaError_t launch_best_select(const long long* bestF, const long long* bestT, int B,
                               long long* out3, cudaStream_t s);
// k_tc.cu  (tcgen05 BF16 contraction with fused epilogue, restart-major state)
struct TcPlan {
  CUtensorMap mapA;        // A [n][lda] BF16, box 64 x 128, 128B swizzle
  CUtensorMap mapX[3];     // operand buffers [B][ld] BF16 (ping, pong, bits), box 64 x tile_n
  int tile_n;
  int num_tiles, m_tiles, n_tiles, grid, sms;
  // split-K of the tiles left over after whole rounds (optional; both null = no splitting)
  float* ws;               // >= sms * tile_n * 128 floats
  int* counters;           // >= sms * 8 ints, zero before the first launch
  int max_splits;
  bool pair;               // CTA-pair kernel (k_tc2.cu): 256 x 256 tiles; tile_n is then 128
  int csk;                 // >= 2: split-K over a cluster of csk CTAs (csk_pair: CTA pairs) per tile (k_tc3.cu)
  bool csk_pair;           // csk on CTA pairs: tiles of 256 rows x 2 tile_n restarts
  unsigned int* gbar;      // csk: grid barrier words of the multi-iteration launch (3, zero between launches)
  float* csk_ws;           // csk: partial tiles exchanged through L2 (>= sms * 256 * 128 floats)
  bool ready;
};
// One instance of a grouped launch (several dense problems in one persistent launch).  The
// table lives in device memory; instances are ordered by decreasing n.
struct TcInst {
  CUtensorMap mapA;        // A of this instance
  CUtensorMap mapX[3];     // operand buffers: ping, pong, bits (box rows = tile_n)
  EpiArgs epi[5];          // epilogue arguments: [2*cur + write_bits] for updates, [4] evaluations
  int n_tiles, kblocks;    // restart tiles, k-blocks
  int tile_begin;          // first tile of this instance in the launch's tile list
  int pad;
};
cudaError_t launch_tc_group(const TcInst* d_insts, int n_insts, int num_tiles, int tile_n, int mode, int epi_variant,
                            uint64_t timeout_ns, cudaStream_t s);

// Work split of one launch: dp_tiles whole tiles round-robin, then the remaining tiles in
// `splits` K-ranges each (sk_units = tail * splits units, one per CTA).
struct TcSchedule {
  int dp_tiles, splits, sk_units, grid;
};
TcSchedule tc_schedule(int num_tiles, int kblocks, int sms, bool can_split, int max_splits);
constexpr int TC_WS_COUNTERS_PER_TILE = 8;
bool tc_supported();
cudaError_t tc_make_plan(TcPlan* plan, const void* A, int64_t lda, int n, const void* X0, const void* X1,
                         const void* Xbits, int64_t ldx, int B, int tile_n, std::string* why);
cudaError_t tc_make_operand_map(CUtensorMap* m, const void* X, int64_t ldx, int n, int B, int tile_n,
                                std::string* why);
cudaError_t launch_tc(const TcPlan& plan, int which_x, const CUtensorMap* map_override, const EpiArgs& a,
                      int mode, uint64_t timeout_ns, cudaStream_t s);
// k_tc2.cu: CTA-pair variant (update and evaluation epilogues)
bool tc_pair_supported(int* max_clusters);
// k_tc3.cu: cluster split-K factor for num_tiles tiles of width tile_n (0: not applicable), and
// its launch (EPI_UPDATE / EPI_EVAL).  An update launch may run `iters` > 1 iterations (operand
// buffers alternating from which_x, candidates written by the last one when a.bits_out is set),
// with a grid barrier between iterations (plan.gbar); not with the single-constraint dual.
int tc_csk_factor(int tile_n, int num_tiles, int kblocks, int sms);
// CTA pairs: K splits (pairs per cluster, 2-4) for pair_tiles tiles of 256 rows x bn restarts
int tc_cskp_factor(int bn, int pair_tiles, int kblocks, int sms);
// Whether multi-iteration cluster launches on the current device are cooperative (1), plain (0) or
// not launched yet (-1).
int tc_csk_cooperative();
cudaError_t launch_tc_csk(const TcPlan& plan, int which_x, const EpiArgs& a, int mode, int iters, uint64_t timeout_ns,
                          cudaStream_t s);
cudaError_t launch_tc_pair(const TcPlan& plan, int which_x, const EpiArgs& a, int mode, uint64_t timeout_ns,
                           cudaStream_t s);

// api.cu: read-only view of a dense problem and the thread-local error message, for entry
// points defined outside api.cu.
struct DenseView {
  int64_t n;
  int prec;
  const void* A;
  int64_t lda;
  const float* cp;
  const int64_t* cp64;
  uint32_t* err;
  uint64_t timeout_ns;
  int gkind;
  int sms;
  int64_t* launches;
};
// k_cert.cu: g = A x in FP64 for one point (dense: pass the problem's view; sparse: view NULL)
cudaError_t launch_matvec_f64(const DenseView* dense, const int32_t* rowptr, const int32_t* col, const void* val,
                              int val_type, int n, const double* x, double* g, cudaStream_t s);
cudaError_t launch_pgd_step_f64(double* x, const double* g, const int64_t* cp, int n, double ybar, double alpha,
                                cudaStream_t s);
bool dense_view(sbo_problem* p, DenseView* v);
void set_last_error(const std::string& msg);

}  // namespace sbo
