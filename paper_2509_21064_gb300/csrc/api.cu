// C ABI of libsbo (declared in include/sbo.h): validation, device memory, kernel selection,
// the iteration schedule with its evaluation points, CUDA-graph replay of evaluation blocks,
// and result read-back.  Every entry point catches its own failures and returns a status.
#include <algorithm>
#include <climits>
#include <sys/stat.h>

#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <tuple>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sbo_internal.h"

using namespace sbo;

namespace {

thread_local std::string g_last_error;

sbo_status fail(sbo_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}
sbo_status cuda_fail(cudaError_t e, const char* what) {
  return fail(SBO_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SBO_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the problem's stream) from
// the device's default pool, which keeps up to SBO_POOL_RETAIN_MB (default 8192) of freed memory
// for reuse, so creating and destroying problems in a loop does not pay for fresh allocations.
void configure_pool_once() {
  static PerDevice per_device;
  per_device.once([] {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (e == cudaSuccess) e = cudaDeviceGetDefaultMemPool(&pool, dev);
    if (e != cudaSuccess) return e;
    uint64_t mb = 8192;
    if (const char* v = std::getenv("SBO_POOL_RETAIN_MB")) mb = std::strtoull(v, nullptr, 10);
    uint64_t thr = mb << 20;
    return cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  });
}

template <typename T>
cudaError_t dalloc(T** p, size_t count, cudaStream_t s) {
  *p = nullptr;
  if (count == 0) count = 1;
  configure_pool_once();
  return cudaMallocAsync(reinterpret_cast<void**>(p), count * sizeof(T), s);
}
template <typename T>
void dfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
}

}  // namespace

struct sbo_problem {
  int64_t n = 0;
  int fmt = FMT_DENSE;
  int prec = SBO_FP32;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream for graph capture
  cudaStream_t cap_side = nullptr;    // second capture stream: evaluations beside the steps
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int sms = 0;
  int64_t l2_bytes = 0;
  // dense
  void* A = nullptr;
  int64_t lda = 0;
  int a_type = OP_F32;
  // CSR
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  void* val = nullptr;
  int val_type = 0;
  int64_t nnz = 0;
  int max_deg = 0;             // longest row of A (CSR)
  int res_nnz_max = 0;         // most nonzeros of A in one CTA's rows of the resident sparse form
  int kparts = 0;              // Max-k-Cut: parts per vertex (FMT_MAXK)
  // linear term
  float* cp = nullptr;
  int64_t* cp64 = nullptr;
  uint32_t* err = nullptr;
  // options
  int opt_kernel = KER_AUTO, opt_graph = 1, opt_tile_n = 0, opt_split_k = 16, opt_autotune = 1, opt_pdl = 1;
  int opt_dual = 0;           // 0: one dual per coordinate (PDBO); 1: one per restart (PDBO-s)
  int opt_g = G_QUAD;         // constraint function g (SBO_OPT_G)
  int opt_keep_grad = 0;      // SBO_OPT_KEEP_GRAD: keep dL/dx of the latest iteration
  int opt_csr_form = 0;       // SBO_OPT_CSR_FORM: 0 autotuned (or the rule), else a CsrForm
  int opt_eval_mode = 0;      // SBO_OPT_EVAL_MODE: 0 the rule (beside), 1 in line, 2 beside
  int64_t opt_timeout_us = 4000000;
  int64_t opt_steps_per_launch = 0;   // cluster split-K iterations per launch (0: 4,096)
  // run
  bool started = false;
  sbo_gda_params prm{};
  int kernel = KER_AUTO, layout = LAYOUT_RN, op_type = OP_F32, tile_n = 0;
  int csr_form = CSR_FORM_RULE;   // form of the sparse update in this run
  int B = 0;
  int64_t ld = 0;
  int64_t t = 0;          // iterations completed
  int64_t t_last_eval = 0;
  int cur = 0;            // operand buffer holding x^t
  float* Xm = nullptr;    // FP32 master (null when the operand is the FP32 master)
  float* Y = nullptr;
  float* Gd = nullptr;    // dL/dx of the latest iteration (SBO_OPT_KEEP_GRAD), state layout
  void* Xop[2] = {nullptr, nullptr};
  void* bits = nullptr;
  long long *bestF = nullptr, *bestT = nullptr, *evalF = nullptr, *trace = nullptr, *n_evals = nullptr,
            *t_last = nullptr, *sel = nullptr;
  unsigned long long* F2 = nullptr;
  uint8_t* bestBits = nullptr;
  unsigned int* commit_ctr = nullptr;   // arrival counter of the evaluation commit (zero between launches)
  // single-constraint form: one dual per restart and the update's rows of partial sums of g
  bool single = false;
  float* mu = nullptr;
  float* gpart = nullptr;
  int64_t gpart_rows = 0, gpart_ld = 0;
  int64_t trace_cap = 0;
  int64_t n_evals_host = 0;
  TcPlan plan{};
  float* tc_ws = nullptr;      // split-K partial tiles of the tcgen05 contraction
  int* tc_ctr = nullptr;       // split-K arrival counters (zero between launches)
  unsigned int* tc_gbar = nullptr;   // grid barrier of multi-iteration launches (zero between launches)
  float* csk_ws = nullptr;           // partial tiles of the cluster split-K kernel
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  // Deferred evaluation (sparse and Max-k-Cut runs with K >= 2): a replayed block leaves the
  // candidates of its last iteration unevaluated (eval_pending; they are those of iteration t), and
  // the next block evaluates them on a branch of its graph beside its first K - 1 steps, which
  // neither read nor write what the evaluation touches.  Every call that reads results first
  // evaluates what is pending (flush_pending).
  cudaGraphExec_t gexec_nv[2] = {nullptr, nullptr};   // K steps, no evaluation
  cudaGraphExec_t gexec_ov[2] = {nullptr, nullptr};   // pending evaluation beside K steps
  int64_t graph_launches[3][2] = {{0, 0}, {0, 0}, {0, 0}};   // kernel launches of each captured block
  bool eval_pending = false;
  bool eval_fused = false;   // the last update launch also added the candidates' objective into F2
  int64_t graph_blocks_seen = 0;   // eligible K-blocks so far: a graph is captured for the second
  // Lagrangian scratch (BF16 operand)
  void* lag_op = nullptr;
  size_t lag_cap = 0;
  int64_t launches = 0;
};

namespace {

void free_run(sbo_problem* p) {
  for (auto* set : {p->gexec, p->gexec_nv, p->gexec_ov})
    for (int k = 0; k < 2; ++k)
      if (set[k]) { cudaGraphExecDestroy(set[k]); set[k] = nullptr; }
  p->eval_pending = false;
  p->eval_fused = false;
  dfree(p->Xm, p->stream);
  dfree(p->Y, p->stream);
  dfree(p->Gd, p->stream);
  dfree(p->Xop[0], p->stream);
  dfree(p->Xop[1], p->stream);
  dfree(p->bits, p->stream);
  dfree(p->bestF, p->stream);
  dfree(p->bestT, p->stream);
  dfree(p->evalF, p->stream);
  dfree(p->trace, p->stream);
  dfree(p->n_evals, p->stream);
  dfree(p->t_last, p->stream);
  dfree(p->sel, p->stream);
  dfree(p->F2, p->stream);
  dfree(p->bestBits, p->stream);
  dfree(p->commit_ctr, p->stream);
  dfree(p->mu, p->stream);
  dfree(p->gpart, p->stream);
  p->single = false;
  dfree(p->tc_ws, p->stream);
  dfree(p->tc_ctr, p->stream);
  dfree(p->tc_gbar, p->stream);
  dfree(p->csk_ws, p->stream);
  p->started = false;
}

void free_all(sbo_problem* p) {
  free_run(p);
  dfree(p->A, p->stream);
  dfree(p->rowptr, p->stream);
  dfree(p->col, p->stream);
  dfree(p->val, p->stream);
  dfree(p->cp, p->stream);
  dfree(p->cp64, p->stream);
  dfree(p->err, p->stream);
  if (p->lag_op) cudaFree(p->lag_op);   // allocated with cudaMalloc: used on callers' streams
  p->lag_op = nullptr;
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  p->cap_stream = nullptr;
  if (p->cap_side) cudaStreamDestroy(p->cap_side);
  p->cap_side = nullptr;
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  p->ev_fork = p->ev_join = nullptr;
}

sbo_status init_common(sbo_problem* p, void* stream) {
  p->stream = static_cast<cudaStream_t>(stream);
  int dev = 0;
  SBO_CUDA(cudaGetDevice(&dev));
  SBO_CUDA(cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, dev));
  int l2 = 0;
  SBO_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
  p->l2_bytes = l2;
  SBO_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
  SBO_CUDA(cudaStreamCreateWithFlags(&p->cap_side, cudaStreamNonBlocking));
  SBO_CUDA(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
  SBO_CUDA(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
  SBO_CUDA(dalloc(&p->err, 1, p->stream));
  SBO_CUDA(cudaMemsetAsync(p->err, 0, sizeof(uint32_t), p->stream));
  return SBO_OK;
}

EpiArgs base_args(const sbo_problem* p) {
  EpiArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = (int)p->n;
  a.B = p->B;
  a.ld = p->ld;
  a.alpha = (float)p->prm.alpha;
  a.beta = (float)p->prm.beta;
  a.delta = (float)p->prm.delta;
  a.grad_tol = (float)p->prm.grad_tol;
  a.cp = p->cp;
  a.cp64 = p->cp64;
  a.Xm = p->Xm;
  a.Y = p->Y;
  a.F2 = p->F2;
  a.err = p->err;
  a.gkind = p->opt_g;
  a.Gd = p->Gd;
  if (p->single) {
    a.mu = p->mu;
    a.gpart = p->gpart;
    a.gpart_ld = p->gpart_ld;
  }
  return a;
}

uint64_t timeout_ns(const sbo_problem* p) { return (uint64_t)p->opt_timeout_us * 1000ull; }

// One contraction launch with the given epilogue on the run's kernel.
// pdl: the sparse kernel may launch as a programmatic dependent of the stream's previous kernel
// (off on a graph branch, whose first kernel follows an event, not a kernel of its stream).
cudaError_t contract(sbo_problem* p, const EpiArgs& a, int mode, int which_x, cudaStream_t s, bool pdl = true) {
  ++p->launches;
  switch (p->kernel) {
    case KER_SIMT: return launch_simt(static_cast<const float*>(p->A), p->lda, a, mode, s);
    case KER_TC: return launch_tc(p->plan, which_x, nullptr, a, mode, timeout_ns(p), s);
    case KER_CSR:
      if (mode == EPI_UPDATE && p->csr_form == CSR_FORM_RESIDENT && !a.mu)
        return launch_csr_res(p->rowptr, p->col, p->val, p->val_type, a, p->op_type, which_x, p->Xop, 1, false,
                              p->res_nnz_max, p->sms, p->tc_gbar, timeout_ns(p), s);
      if (mode == EPI_UPDATE && p->csr_form == CSR_FORM_STAGED && !a.mu)
        return launch_csr_staged(p->rowptr, p->col, p->val, p->val_type, a, p->op_type, p->max_deg, p->sms,
                                 pdl && p->opt_pdl != 0, timeout_ns(p), s);
      return launch_csr(p->rowptr, p->col, p->val, p->val_type, a, p->op_type, mode, pdl && p->opt_pdl != 0, s,
                        p->csr_form);
    case KER_MAXK: return launch_maxk(p->rowptr, p->col, static_cast<const float*>(p->val), a, p->kparts, mode, s);
    default: return cudaErrorInvalidValue;
  }
}

// x^t -> x^{t+1}; optionally writes the candidate bits of x^{t+1}.
cudaError_t enqueue_step(sbo_problem* p, bool write_bits, cudaStream_t s) {
  EpiArgs a = base_args(p);
  a.Xin = p->Xop[p->cur];
  a.Xout = p->Xop[p->cur ^ 1];
  a.bits_out = write_bits ? p->bits : nullptr;
  cudaError_t e = contract(p, a, EPI_UPDATE, p->cur, s);
  p->cur ^= 1;
  if (e == cudaSuccess && p->single) {
    e = launch_dual_single(p->mu, p->gpart, (int)p->gpart_rows, p->gpart_ld, p->B, (float)p->prm.beta, s);
    ++p->launches;
  }
  return e;
}

// Iterations one launch may run: several for the cluster split-K kernel with per-coordinate
// duals (grid barrier between them), else one.
int64_t steps_per_launch(const sbo_problem* p) {
  const bool csk = p->kernel == KER_TC && p->plan.csk >= 2 && !p->plan.pair;
  const bool res = p->kernel == KER_CSR && p->csr_form == CSR_FORM_RESIDENT;
  if (!(csk || res) || p->single || !p->tc_gbar) return 1;
  return p->opt_steps_per_launch == 0 ? 4096 : p->opt_steps_per_launch;
}

// `steps` iterations; the last one writes the candidate bits when write_bits.  fuse_eval: the
// evaluation follows on this stream, so the resident sparse form may compute it in its launch.
cudaError_t enqueue_steps(sbo_problem* p, int64_t steps, bool write_bits, cudaStream_t s, bool fuse_eval = false) {
  const int64_t per = steps_per_launch(p);
  if (per <= 1) {
    for (int64_t k = 0; k < steps; ++k) {
      cudaError_t e = enqueue_step(p, write_bits && k + 1 == steps, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  for (int64_t done = 0; done < steps;) {
    const int64_t chunk = std::min(per, steps - done);
    done += chunk;
    EpiArgs a = base_args(p);
    a.Xin = p->Xop[p->cur];
    a.Xout = p->Xop[p->cur ^ 1];
    a.bits_out = write_bits && done == steps ? p->bits : nullptr;
    // the resident sparse form evaluates the candidates it writes inside the same launch; the
    // evaluation that follows then only commits them
    const bool fuse = fuse_eval && p->kernel == KER_CSR && a.bits_out != nullptr;
    ++p->launches;
    cudaError_t e = p->kernel == KER_CSR
                        ? launch_csr_res(p->rowptr, p->col, p->val, p->val_type, a, p->op_type, p->cur, p->Xop,
                                         (int)chunk, fuse, p->res_nnz_max, p->sms, p->tc_gbar, timeout_ns(p), s)
                        : launch_tc_csk(p->plan, p->cur, a, EPI_UPDATE, (int)chunk, timeout_ns(p), s);
    if (e != cudaSuccess) return e;
    if (fuse) p->eval_fused = true;
    if (chunk & 1) p->cur ^= 1;
  }
  return cudaSuccess;
}

CommitArgs commit_args(const sbo_problem* p) {
  CommitArgs c;
  std::memset(&c, 0, sizeof(c));
  c.bits = p->bits;
  c.op_type = p->kernel == KER_CSR ? OP_U8 : p->op_type;
  c.layout = p->layout;
  c.n = (int)p->n;
  c.B = p->B;
  c.ld = p->ld;
  c.bestBits = p->bestBits;
  c.F2 = p->F2;
  c.bestF = p->bestF;
  c.bestT = p->bestT;
  c.evalF = p->evalF;
  c.trace = p->trace;
  c.n_evals = p->n_evals;
  c.t_last = p->t_last;
  c.trace_cap = p->trace_cap;
  c.ctr = p->commit_ctr;
  return c;
}

// Exact objective of the bits written by the last step, then best bookkeeping.
cudaError_t enqueue_eval(sbo_problem* p, int64_t add, cudaStream_t s, bool pdl = true) {
  cudaError_t e = cudaSuccess;
  if (p->eval_fused) {
    p->eval_fused = false;   // the objective was computed by the launch that wrote the candidates
  } else {
    EpiArgs a = base_args(p);
    a.Xin = p->bits;
    e = contract(p, a, EPI_EVAL, 2, s, pdl);
    if (e != cudaSuccess) return e;
  }
  e = launch_eval_commit(commit_args(p), add, s);
  ++p->launches;
  return e;
}

int64_t next_eval_after(const sbo_problem* p, int64_t t) {
  const int64_t K = p->prm.eval_every;
  int64_t nx = (t / K + 1) * K;
  if (p->prm.iters > t && p->prm.iters < nx) nx = p->prm.iters;
  return nx;
}

// Evaluations are deferred across blocks only where every step leaves the bits alone (K >= 2) and
// the evaluation runs well beside the steps: sparse and Max-k-Cut runs replayed from graphs.  A
// block then leaves its last iteration's candidates pending and the next block evaluates them on
// a second graph branch beside its first K - 1 steps.  Measured per iteration with K = 10 (FP32):
// Max-Cut ER n = 2,000, B = 256 5.76 -> 5.14 us and the 100 x 100 torus, B = 512 16.99 -> 16.41 us;
// the 4-regular graph n = 20,000, B = 512, whose x and y stream from DRAM, 40.85 -> 39.98 us (E4M3
// 40.03 -> 39.28) with the streaming update forms.  Evaluating inside the next block's first update
// instead (one pass over the graph for both) measured slower on every graph (4-regular E4M3 41.4,
// torus 17.5 us): the fused kernel's registers cost it occupancy.  SBO_OPT_EVAL_MODE 1 forces the
// evaluation in line.
bool defer_evals(const sbo_problem* p) {
  // (the resident sparse form's cooperative launch leaves an eighth of the SMs to the evaluation)
  return (p->kernel == KER_CSR || p->kernel == KER_MAXK) && p->prm.eval_every >= 2 && p->opt_graph &&
         p->opt_eval_mode != 1;
}

// Evaluate the deferred candidates (those of iteration t) on the problem's stream.
sbo_status flush_pending(sbo_problem* p) {
  if (!p->eval_pending) return SBO_OK;
  p->eval_pending = false;
  cudaError_t e = enqueue_eval(p, p->t - p->t_last_eval, p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "evaluation launch");
  p->t_last_eval = p->t;
  ++p->n_evals_host;
  return SBO_OK;
}

sbo_status run_direct(sbo_problem* p, int64_t steps, bool eval_at_end) {
  sbo_status st = flush_pending(p);
  if (st != SBO_OK) return st;
  cudaError_t e0 = enqueue_steps(p, steps, eval_at_end, p->stream, eval_at_end);
  if (e0 != cudaSuccess) return cuda_fail(e0, "GDA step launch");
  p->t += steps;
  if (eval_at_end) {
    cudaError_t e = enqueue_eval(p, p->t - p->t_last_eval, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "evaluation launch");
    p->t_last_eval = p->t;
    ++p->n_evals_host;
  }
  return SBO_OK;
}

// Capture one block of K iterations starting from operand buffer `parity` into a graph.
// BLOCK_EVAL: the steps, then the evaluation of the last one's candidates.  BLOCK_DEFER: the steps
// only (the last one's candidates stay pending).  BLOCK_BESIDE: the pending candidates of the
// block's first iteration are evaluated on a second branch beside the first K - 1 steps (which
// read and write neither the candidates nor the records), joined before the last step writes new
// candidates; those stay pending.
enum { BLOCK_EVAL = 0, BLOCK_DEFER = 1, BLOCK_BESIDE = 2 };
sbo_status capture_block(sbo_problem* p, int parity, int kind) {
  const int64_t K = p->prm.eval_every;
  const int saved_cur = p->cur;
  const int64_t saved_launches = p->launches;
  p->cur = parity;
  cudaGraph_t g = nullptr;
  SBO_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  if (kind == BLOCK_BESIDE) {
    err = cudaEventRecord(p->ev_fork, p->cap_stream);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(p->cap_side, p->ev_fork, 0);
    if (err == cudaSuccess) err = enqueue_eval(p, K, p->cap_side, false);
    if (err == cudaSuccess) err = cudaEventRecord(p->ev_join, p->cap_side);
  }
  if (kind == BLOCK_BESIDE) {
    // the first K - 1 steps beside the evaluation, the last one (which writes new candidates) after it
    if (err == cudaSuccess) err = enqueue_steps(p, K - 1, false, p->cap_stream);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(p->cap_stream, p->ev_join, 0);
    if (err == cudaSuccess) err = enqueue_steps(p, 1, true, p->cap_stream);
  } else if (err == cudaSuccess) {
    err = enqueue_steps(p, K, true, p->cap_stream, kind == BLOCK_EVAL);
  }
  if (err == cudaSuccess && kind == BLOCK_EVAL) err = enqueue_eval(p, K, p->cap_stream);
  cudaError_t e2 = cudaStreamEndCapture(p->cap_stream, &g);
  p->cur = saved_cur;
  p->graph_launches[kind][parity] = p->launches - saved_launches;   // counted again at every replay
  p->launches = saved_launches;
  if (err != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(err, "launch during graph capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  cudaGraphExec_t* slot = kind == BLOCK_EVAL ? p->gexec : kind == BLOCK_DEFER ? p->gexec_nv : p->gexec_ov;
  cudaError_t e3 = cudaGraphInstantiate(&slot[parity], g, 0);
  cudaGraphDestroy(g);
  if (e3 != cudaSuccess) return cuda_fail(e3, "cudaGraphInstantiate");
  return SBO_OK;
}

sbo_status run_tiny(sbo_problem* p, int64_t steps) {
  TinyArgs a;
  a.n = (int)p->n;
  a.B = p->B;
  a.ld = p->ld;
  a.A = static_cast<const float*>(p->A);
  a.lda = p->lda;
  a.cp = p->cp;
  a.cp64 = p->cp64;
  a.X = p->Xm;
  a.Y = p->Y;
  a.alpha = (float)p->prm.alpha;
  a.gkind = p->opt_g;
  a.beta = (float)p->prm.beta;
  a.delta = (float)p->prm.delta;
  a.grad_tol = (float)p->prm.grad_tol;
  a.t0 = p->t;
  a.steps = steps;
  a.K = p->prm.eval_every;
  a.T = p->prm.iters;
  a.bestF = p->bestF;
  a.bestT = p->bestT;
  a.bestBits = p->bestBits;
  a.trace = p->trace;
  a.e0 = p->n_evals_host;
  a.trace_cap = p->trace_cap;
  a.evalF = p->evalF;
  a.G = p->Gd;
  cudaError_t e = launch_tiny(a, p->stream);
  ++p->launches;
  if (e != cudaSuccess) return cuda_fail(e, "tiny-n launch");
  int64_t ne = 0;
  for (int64_t t = p->t + 1; t <= p->t + steps; ++t)
    if (t % p->prm.eval_every == 0 || t == p->prm.iters) { ++ne; p->t_last_eval = t; }
  p->n_evals_host += ne;
  p->t += steps;
  long long ne_dev = (long long)p->n_evals_host, tl = (long long)p->t_last_eval;
  SBO_CUDA(cudaMemcpyAsync(p->n_evals, &ne_dev, sizeof(long long), cudaMemcpyHostToDevice, p->stream));
  SBO_CUDA(cudaMemcpyAsync(p->t_last, &tl, sizeof(long long), cudaMemcpyHostToDevice, p->stream));
  SBO_CUDA(cudaStreamSynchronize(p->stream));  // the host values above must outlive the copies
  return SBO_OK;
}

sbo_status read_err(sbo_problem* p);

// Widest tile that still gives every SM a tile (else the widest), never wider than needed.
// Tile codes: 64, 128, 256 restarts per single-CTA tile; 512 CTA pairs (256 x 256 tiles);
// 1000 + w: width w with split-K over a thread-block cluster (small problems).
// Restarts per CTA that the operand map of a tile code stages (its box height).
int tile_width(int code) {
  return code == 512 ? 128 : code >= 2000 ? (code - 2000) / 2 : code >= 1000 ? code - 1000 : code;
}

// Restarts per tile of a tile code.
int tile_restarts(int code) { return code == 512 ? 256 : code >= 2000 ? code - 2000 : tile_width(code); }

// K splits of the cluster split-K codes for this problem (0: not applicable); plan built for the code.
int csk_factor_for(const sbo_problem* p, int code, const TcPlan& pl) {
  if (!p->csk_ws || code < 1000) return 0;
  const int kblocks = (int)((p->n + 63) / 64);
  if (code >= 2000) {
    const int bn = code - 2000;
    const int pair_tiles = (int)((p->n + 255) / 256) * ((p->B + bn - 1) / bn);
    return tc_cskp_factor(bn, pair_tiles, kblocks, p->sms);
  }
  return tc_csk_factor(tile_width(code), pl.num_tiles, kblocks, p->sms);
}

int heuristic_tile(const sbo_problem* p) {
  int tn = 256;
  while (tn > 64 && (int64_t)((p->n + 127) / 128) * ((p->B + tn - 1) / tn) < p->sms) tn /= 2;
  while (tn > 64 && tn / 2 >= p->B) tn /= 2;
  return tn;
}

void attach_workspace(sbo_problem* p, TcPlan* plan) {
  plan->gbar = p->tc_gbar;
  plan->csk_ws = p->csk_ws;
  if (p->tc_ws && p->tc_ctr && p->opt_split_k >= 2) {
    plan->ws = p->tc_ws;
    plan->counters = p->tc_ctr;
    plan->max_splits = p->opt_split_k;
  }
}

// Persistent record of autotuner decisions: one line "<key> <tile>" per tuned shape, in the file
// named by SBO_TUNE_CACHE ("off" disables it), by default ~/.cache/sbo/tile_tuning.txt.  A
// later process -- for instance the same program under a profiler, whose per-launch overhead
// would swamp the trial timings -- then reuses the decision instead of re-measuring.
std::string tune_cache_path() {
  const char* e = std::getenv("SBO_TUNE_CACHE");
  if (e) return (!*e || std::string(e) == "off") ? std::string() : std::string(e);
  const char* home = std::getenv("HOME");
  return home && *home ? std::string(home) + "/.cache/sbo/tile_tuning.txt" : std::string();
}

std::string tune_key(const sbo_problem* p) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  std::string name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "unknown";
  for (auto& ch : name)
    if (ch == ' ') ch = '_';
  std::ostringstream k;
  k << "v5:" << name << ":sms" << p->sms << ":n" << p->n << ":B" << p->B << ":split" << p->opt_split_k
    << (p->opt_steps_per_launch == 1 ? ":one" : "");
  return k.str();
}

// A tile decision is the tile code, plus 10000 x the cluster size for the cluster split-K codes.
bool valid_tile_code(int t) {
  const int code = t % 10000;
  return code == 64 || code == 128 || code == 256 || code == 512 ||
         ((code == 1064 || code == 1128 || code == 1256) && t / 10000 >= 2 && t / 10000 <= 8) ||
         ((code == 2128 || code == 2256) && t / 10000 >= 2 && t / 10000 <= 4);
}

bool tune_cache_lookup(const std::string& key, int* tile, bool (*valid)(int) = valid_tile_code) {
  const std::string path = tune_cache_path();
  if (path.empty()) return false;
  std::ifstream f(path);
  std::string k;
  int t = 0;
  bool found = false;
  while (f >> k >> t) {
    if (k == key && valid(t)) {
      *tile = t;
      found = true;
    }
  }
  return found;
}

void tune_cache_store(const std::string& key, int tile) {
  const std::string path = tune_cache_path();
  if (path.empty()) return;
  // create the parent directories (best effort)
  for (size_t pos = path.find('/', 1); pos != std::string::npos; pos = path.find('/', pos + 1))
    mkdir(path.substr(0, pos).c_str(), 0755);
  std::ofstream f(path, std::ios::app);
  if (f) f << key << " " << tile << "\n";
}

// Autotuner of the tensor-core tile width: times the update kernel for every candidate width on
// this run's own buffers (called before x^0 is written, so the trial launches only overwrite
// state that initialisation rewrites) and keeps the fastest.  Decisions are kept for the life of
// the process and in the persistent record above; a cluster split-K choice is returned (and
// kept) as code + 10000 x its cluster size, so that a later process, where the occupancy query
// behind the cluster size may answer differently (under a profiler), launches the same kernel.
sbo_status tune_tile(sbo_problem* p, int* out) {
  static std::mutex mu;
  static std::map<std::string, int> cache;
  const std::string key = tune_key(p);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) { *out = it->second; return SBO_OK; }
    int t = 0;
    if (tune_cache_lookup(key, &t)) {
      if (t != 512 || tc_pair_supported(nullptr)) {
        cache[key] = t;
        *out = t;
        return SBO_OK;
      }
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SBO_CUDA(cudaEventCreate(&e0));
  SBO_CUDA(cudaEventCreate(&e1));
  int best = heuristic_tile(p);
  float best_ms = 1e30f;
  EpiArgs a = base_args(p);
  a.Xin = p->Xop[0];
  a.Xout = p->Xop[1];
  a.bits_out = nullptr;
  sbo_status st = SBO_OK;
  for (int tn : {64, 128, 256, 512, 1128, 1256, 2128, 2256}) {
    const int width = tile_width(tn);
    if (tile_restarts(tn) > 64 && tile_restarts(tn) / 2 >= p->B) continue;
    if (tn == 512 && !tc_pair_supported(nullptr)) continue;
    TcPlan pl{};
    std::string why;
    if (tc_make_plan(&pl, p->A, p->lda, (int)p->n, p->Xop[0], p->Xop[1], p->bits, p->ld, p->B, width, &why) !=
        cudaSuccess)
      continue;
    pl.pair = tn == 512;
    if (tn >= 1000) {
      pl.csk_pair = tn >= 2000;
      pl.csk = csk_factor_for(p, tn, pl);
      if (pl.csk < 2) continue;
    }
    attach_workspace(p, &pl);
    // `reps` iterations the way the run would take them: one launch of the cluster kernel when
    // its iterations share a launch, else one launch each
    const int reps = 4;
    const bool multi = pl.csk >= 2 && !p->single && pl.gbar && p->opt_steps_per_launch != 1;
    cudaError_t e = launch_tc(pl, 0, nullptr, a, EPI_UPDATE, timeout_ns(p), p->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, p->stream);
    if (multi) {
      if (e == cudaSuccess) e = launch_tc_csk(pl, 0, a, EPI_UPDATE, reps, timeout_ns(p), p->stream);
    } else {
      for (int k = 0; k < reps && e == cudaSuccess; ++k) e = launch_tc(pl, 0, nullptr, a, EPI_UPDATE, timeout_ns(p), p->stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    p->launches += multi ? 2 : reps + 1;
    if (e != cudaSuccess) { st = cuda_fail(e, "autotuner launch"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) { best_ms = ms; best = tn >= 1000 ? tn + 10000 * pl.csk : tn; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SBO_OK) return st;
  st = read_err(p);
  if (st != SBO_OK) return st;
  {
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = best;
    tune_cache_store(key, best);
  }
  *out = best;
  return SBO_OK;
}

// Autotuner of the sparse update's form: times the update launch in every form (one row per warp
// with 128 or 256 restarts, pipelined rows of 256, each with and without the L2 eviction
// priorities) on this run's own buffers, before x^0 is written, and keeps the fastest.  Kept per (device, graph
// size, restarts, precision, g) for the process and in the persistent record of tune_tile.
sbo_status tune_csr_form(sbo_problem* p, int* out) {
  static std::mutex mu;
  static std::map<std::string, int> cache;
  std::string key;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    std::string name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "unknown";
    for (auto& ch : name)
      if (ch == ' ') ch = '_';
    std::ostringstream k;
    k << "csr5:" << name << ":sms" << p->sms << ":n" << p->n << ":nnz" << p->nnz << ":deg" << p->max_deg << ":B"
      << p->B << ":op" << p->op_type << ":g" << p->opt_g;
    key = k.str();
  }
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) { *out = it->second; return SBO_OK; }
    int t = 0;
    if (tune_cache_lookup(key, &t, [](int v) { return v >= CSR_FORM_ROW1 && v <= CSR_FORM_PIPE2_STREAM; })) {
      cache[key] = t;
      *out = t;
      return SBO_OK;
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SBO_CUDA(cudaEventCreate(&e0));
  SBO_CUDA(cudaEventCreate(&e1));
  EpiArgs a = base_args(p);
  a.Xin = p->Xop[0];
  a.Xout = p->Xop[1];
  a.bits_out = nullptr;   // the run writes candidates in one iteration of K
  int best = CSR_FORM_RULE;
  float best_ms = 1e30f;
  sbo_status st = SBO_OK;
  // (the staged form, measured two to three times slower than these on every graph here, is not a
  // candidate: it stays available through SBO_OPT_CSR_FORM).  The streaming forms are candidates
  // only when x and y (16 B per element) overflow three quarters of L2: on L2-resident state their
  // evict-first loads and stores send the next iteration's state to DRAM (100 x 100 torus, B = 512,
  // E4M3: 15.9 -> 18.4 us per iteration), which launches timed back to back on one buffer do not
  // always show.
  const bool streams = p->n * (int64_t)p->B * 16 * 4 > p->l2_bytes * 3;
  // Two rounds over the forms, each form's best round counting, so that a clock or cache transient
  // during one form's timing does not decide.
  // The resident form (CSR_FORM_RESIDENT) is not a candidate: its updates alone are faster (Max-Cut
  // ER n = 2,000, B = 256: 3.8 against about 4.8 us per iteration), which is what these trials time,
  // but over a run with an evaluation every 10 iterations it measured slower in FP32 (5.8 against
  // 5.45 us per iteration with form 1) and faster in BF16 (5.0-5.2 against about 5.4).
  const int forms[] = {CSR_FORM_ROW1, CSR_FORM_ROW2, CSR_FORM_PIPE2, CSR_FORM_ROW1_STREAM, CSR_FORM_ROW2_STREAM,
                       CSR_FORM_PIPE2_STREAM};
  float form_ms[8];
  for (float& v : form_ms) v = 1e30f;
  for (int round = 0; round < 2 && st == SBO_OK; ++round)
  for (int f : forms) {
    if (csr_form_streams(f) && !streams) continue;
    int D, S, rc;
    size_t sm;
    if (f == CSR_FORM_STAGED && !csr_staged_shape(p->ld, p->op_type, p->max_deg, &D, &S, &rc, &sm)) continue;
    // the launches alternate the operand buffers as the run does, so that what one launch writes
    // (with its L2 priority) is what the next one gathers
    int par = 0;
    auto launch = [&]() {
      EpiArgs b = a;
      b.Xin = p->Xop[par];
      b.Xout = p->Xop[par ^ 1];
      par ^= 1;
      return f == CSR_FORM_STAGED
                 ? launch_csr_staged(p->rowptr, p->col, p->val, p->val_type, b, p->op_type, p->max_deg, p->sms,
                                     p->opt_pdl != 0, timeout_ns(p), p->stream)
                 : launch_csr(p->rowptr, p->col, p->val, p->val_type, b, p->op_type, EPI_UPDATE, p->opt_pdl != 0,
                              p->stream, f);
    };
    const int reps = 10;
    cudaError_t e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e0, p->stream);
    for (int k = 0; k < reps && e == cudaSuccess; ++k) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    p->launches += reps + 1;
    if (e != cudaSuccess) { st = cuda_fail(e, "sparse autotuner launch"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    form_ms[f] = std::min(form_ms[f], ms);
  }
  for (int f : forms)
    if (form_ms[f] < best_ms) { best_ms = form_ms[f]; best = f; }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SBO_OK) return st;
  st = read_err(p);
  if (st != SBO_OK) return st;
  {
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = best;
    tune_cache_store(key, best);
  }
  *out = best;
  return SBO_OK;
}

sbo_status check_params(const sbo_gda_params* q) {
  if (!q) return fail(SBO_EINVAL, "params is NULL");
  if (q->restarts < 1) return fail(SBO_EINVAL, "restarts must be >= 1");
  if (q->eval_every < 1) return fail(SBO_EINVAL, "eval_every must be >= 1");
  if (q->iters < 0) return fail(SBO_EINVAL, "iters must be >= 0");
  if (!std::isfinite(q->alpha) || q->alpha <= 0) return fail(SBO_EINVAL, "alpha must be finite and > 0");
  if (!std::isfinite(q->beta) || q->beta < 0) return fail(SBO_EINVAL, "beta must be finite and >= 0");
  if (!std::isfinite(q->ybar)) return fail(SBO_EINVAL, "ybar must be finite");
  if (!std::isfinite(q->delta) || q->delta < 0 || q->delta >= 0.5) return fail(SBO_EINVAL, "delta must be in [0, 0.5)");
  if (!std::isfinite(q->grad_tol) || q->grad_tol < 0) return fail(SBO_EINVAL, "grad_tol must be finite and >= 0");
  return SBO_OK;
}

sbo_status read_err(sbo_problem* p) {
  uint32_t w = 0;
  SBO_CUDA(cudaMemcpy(&w, p->err, sizeof(w), cudaMemcpyDeviceToHost));
  if (w) {
    SBO_CUDA(cudaMemset(p->err, 0, sizeof(uint32_t)));
    // a launch that gave up may have left the grid barrier's words raised
    if (p->tc_gbar) SBO_CUDA(cudaMemset(p->tc_gbar, 0, 3 * sizeof(unsigned int)));
    if (w & ERR_TIMEOUT) return fail(SBO_ETIMEOUT, "a bounded device-side wait expired; the kernel returned early");
    return fail(SBO_EDEVICE, "a device-side bounds check failed (input out of range)");
  }
  return SBO_OK;
}

}  // namespace

// =============================================================================================
extern "C" {

const char* sbo_last_error(void) { return g_last_error.c_str(); }
const char* sbo_version(void) { return "sbo 0.1 (sm_103a)"; }

// A second stream for host-to-device copies that the problem's stream consumes piecewise: each
// copy is ordered after the work already on the problem's stream (the destination's stream-ordered
// allocation), and the problem's stream waits for it before its next launch.  The stream and
// events are released when the lane goes out of scope (work in flight completes first).
struct CopyLane {
  cudaStream_t cs = nullptr;
  std::vector<cudaEvent_t> evs;
  cudaError_t open(cudaStream_t s) {
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) { cs = nullptr; return e; }
    return mark(s, cs);
  }
  // event on `from`, waited on by `to`
  cudaError_t mark(cudaStream_t from, cudaStream_t to) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    evs.push_back(ev);
    if ((e = cudaEventRecord(ev, from)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(to, ev, 0);
  }
  cudaError_t copy(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return e;
    return mark(cs, s);
  }
  void drain() {   // error paths: no copy may still write memory that is about to be freed
    if (cs) cudaStreamSynchronize(cs);
  }
  ~CopyLane() {
    for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
  }
};

// Dense set-up shared by the int32 and int8 entry points (q_bytes: size of one entry of Q).
static sbo_status create_dense_impl(int64_t n, const void* Q, int q_bytes, const int32_t* c, int32_t precision,
                                    void* stream, sbo_problem** out) {
  g_last_error.clear();
  if (!out) return fail(SBO_EINVAL, "out is NULL");
  *out = nullptr;
  if (!Q) return fail(SBO_EINVAL, "Q is NULL");
  if (n < 1 || n > 65536) return fail(SBO_EINVAL, "dense n must be in [1, 65536]");
  if (precision != SBO_FP32 && precision != SBO_BF16)
    return fail(SBO_EINVAL, "dense problems take SBO_FP32 or SBO_BF16 (an FP8 contraction would need FP8 x)");
  sbo_problem* p = new (std::nothrow) sbo_problem();
  if (!p) return fail(SBO_ENOMEM, "host allocation failed");
  sbo_status st = init_common(p, stream);
  if (st != SBO_OK) { free_all(p); delete p; return st; }
  p->n = n;
  p->fmt = FMT_DENSE;
  p->prec = precision;
  p->a_type = precision == SBO_FP32 ? OP_F32 : OP_BF16;
  p->lda = round_up(n, 8);
  void* Qd = nullptr;
  int32_t* cd = nullptr;
  unsigned long long* rowsum = nullptr;
  uint32_t* rerr = nullptr;
  cudaStream_t s = p->stream;
  auto cleanup_tmp = [&]() {
    if (Qd) cudaFreeAsync(Qd, s);
    Qd = nullptr;
    dfree(cd, s); dfree(rowsum, s); dfree(rerr, s);
  };
  auto bail = [&](sbo_status s) { cleanup_tmp(); free_all(p); delete p; return s; };
  cudaError_t e;
  const size_t a_elt = p->a_type == OP_F32 ? 4 : 2;
  configure_pool_once();
  if ((e = cudaMallocAsync(&p->A, (size_t)n * p->lda * a_elt, s)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc A"));
  if ((e = dalloc(&p->cp, n, s)) != cudaSuccess || (e = dalloc(&p->cp64, n, s)) != cudaSuccess ||
      (e = cudaMallocAsync(&Qd, (size_t)n * n * q_bytes, s)) != cudaSuccess || (e = dalloc(&rowsum, n, s)) != cudaSuccess ||
      (e = dalloc(&rerr, 1, s)) != cudaSuccess || (c && (e = dalloc(&cd, n, s)) != cudaSuccess))
    return bail(e == cudaErrorMemoryAllocation ? fail(SBO_ENOMEM, "device allocation failed") : cuda_fail(e, "cudaMalloc"));
  if (c && (e = cudaMemcpyAsync(cd, c, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return bail(cuda_fail(e, "copy c"));
  cudaMemsetAsync(rowsum, 0, sizeof(unsigned long long) * n, s);
  cudaMemsetAsync(rerr, 0, sizeof(uint32_t), s);
  const int64_t limit = p->a_type == OP_F32 ? (1ll << 24) : 256;
  // Q crosses in up to 16 panels of whole 64-row tiles on a second stream; as each lands, the
  // problem's stream canonicalises the tile pairs whose rows have all arrived (the panel's tile
  // columns), so the copy and the canonicalisation overlap.
  {
    CopyLane lane;
    if ((e = lane.open(s)) != cudaSuccess) return bail(cuda_fail(e, "copy stream"));
    const int64_t nt = (p->lda + 63) / 64;
    const int64_t per = (nt + 15) / 16;
    for (int64_t j0 = 0; j0 < nt; j0 += per) {
      const int64_t j1 = std::min(nt, j0 + per);
      const int64_t r0 = 64 * j0, r1 = std::min<int64_t>(n, 64 * j1);
      if (r1 > r0) {
        const size_t off = (size_t)r0 * n * q_bytes, bytes = (size_t)(r1 - r0) * n * q_bytes;
        if ((e = lane.copy(static_cast<char*>(Qd) + off, static_cast<const char*>(Q) + off, bytes, s)) != cudaSuccess) {
          lane.drain();
          return bail(cuda_fail(e, "copy Q"));
        }
      }
      if ((e = launch_canon_dense(Qd, q_bytes, n, j0, j1, p->A, p->lda, p->a_type, rowsum, rerr, limit, s)) !=
          cudaSuccess) {
        lane.drain();
        return bail(cuda_fail(e, "canonicalisation launch"));
      }
      ++p->launches;
    }
  }
  if ((e = launch_canon_linear(Qd, q_bytes, cd, n, p->cp, p->cp64, s)) != cudaSuccess)
    return bail(cuda_fail(e, "canonicalisation launch"));
  if ((e = launch_rowsum_check(rowsum, p->cp64, n, rerr, s)) != cudaSuccess) return bail(cuda_fail(e, "row-sum check"));
  p->launches += 2;
  uint32_t flags = 0;
  if ((e = cudaMemcpyAsync(&flags, rerr, sizeof(flags), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return bail(cuda_fail(e, "canonicalisation"));
  cleanup_tmp();
  if (flags & 1u) {
    free_all(p); delete p;
    return fail(SBO_ERANGE, precision == SBO_BF16 ? "|Q_ij + Q_ji| > 256 is not exact in BF16"
                                                  : "|Q_ij + Q_ji| > 2^24 is not exact in FP32");
  }
  if (flags & 2u) { free_all(p); delete p; return fail(SBO_ERANGE, "a row sum of |A_ij| reaches 2^24 (objective not exact)"); }
  if (flags & 4u) { free_all(p); delete p; return fail(SBO_ERANGE, "c_i + Q_ii outside the int32 range"); }
  *out = p;
  return SBO_OK;
}

sbo_status sbo_create_dense(int64_t n, const int32_t* Q, const int32_t* c, int32_t precision, void* stream,
                            sbo_problem** out) {
  return create_dense_impl(n, Q, 4, c, precision, stream, out);
}

sbo_status sbo_create_dense_i8(int64_t n, const int8_t* Q, const int32_t* c, int32_t precision, void* stream,
                               sbo_problem** out) {
  return create_dense_impl(n, Q, 1, c, precision, stream, out);
}

sbo_status sbo_create_csr(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col, const int32_t* val,
                          const int32_t* c, int32_t precision, void* stream, sbo_problem** out) {
  g_last_error.clear();
  if (!out) return fail(SBO_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || n >= (1ll << 31)) return fail(SBO_EINVAL, "n must be in [1, 2^31)");
  if (nnz < 0) return fail(SBO_EINVAL, "nnz must be >= 0");
  if (!rowptr || (nnz > 0 && (!col || !val))) return fail(SBO_EINVAL, "rowptr/col/val is NULL");
  if (precision != SBO_FP32 && precision != SBO_BF16 && precision != SBO_FP8_E4M3)
    return fail(SBO_EINVAL, "unknown precision");
  if (rowptr[0] != 0 || rowptr[n] != nnz) return fail(SBO_EINVAL, "rowptr[0] must be 0 and rowptr[n] must be nnz");
  for (int64_t i = 0; i < n; ++i)
    if (rowptr[i + 1] < rowptr[i]) return fail(SBO_EINVAL, "rowptr is not non-decreasing");
  // A = Q + Q^T off the diagonal, c' = c + diag(Q)  (Prop. 2.4), built as sorted triples
  std::vector<int64_t> cp(n, 0);
  if (c)
    for (int64_t i = 0; i < n; ++i) cp[i] = c[i];
  struct Trip { int32_t i, j; int64_t v; };
  std::vector<Trip> tr;
  tr.reserve((size_t)2 * nnz);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int32_t j = col[e];
      if (j < 0 || j >= n) return fail(SBO_EINVAL, "column index out of range");
      if (j == i) { cp[i] += val[e]; continue; }
      tr.push_back({(int32_t)i, j, (int64_t)val[e]});
      tr.push_back({j, (int32_t)i, (int64_t)val[e]});
    }
  std::sort(tr.begin(), tr.end(), [](const Trip& a, const Trip& b) { return a.i != b.i ? a.i < b.i : a.j < b.j; });
  std::vector<int32_t> rp(n + 1, 0), cc;
  std::vector<int64_t> vv;
  cc.reserve(tr.size());
  vv.reserve(tr.size());
  for (size_t k = 0; k < tr.size();) {
    size_t m = k;
    int64_t s = 0;
    while (m < tr.size() && tr[m].i == tr[k].i && tr[m].j == tr[k].j) s += tr[m++].v;
    if (s != 0) { cc.push_back(tr[k].j); vv.push_back(s); rp[tr[k].i + 1]++; }
    k = m;
  }
  if (cc.size() >= (size_t)INT32_MAX) return fail(SBO_EINVAL, "too many non-zeros");
  for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  const int64_t limit = precision == SBO_FP32 ? (1ll << 24) : precision == SBO_BF16 ? 256 : 16;
  std::vector<int64_t> rowabs(n, 0);
  for (int64_t i = 0; i < n; ++i)
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
      const int64_t a = vv[e] < 0 ? -vv[e] : vv[e];
      if (a > limit) return fail(SBO_ERANGE, "an entry of Q + Q^T is not exact at the requested precision");
      rowabs[i] += a;
    }
  for (int64_t i = 0; i < n; ++i) {
    if (rowabs[i] >= (1ll << 24)) return fail(SBO_ERANGE, "a row sum of |A_ij| reaches 2^24 (objective not exact)");
    if (cp[i] >= (1ll << 31) || cp[i] <= -(1ll << 31)) return fail(SBO_ERANGE, "c_i + Q_ii outside the int32 range");
  }
  sbo_problem* p = new (std::nothrow) sbo_problem();
  if (!p) return fail(SBO_ENOMEM, "host allocation failed");
  sbo_status st = init_common(p, stream);
  if (st != SBO_OK) { free_all(p); delete p; return st; }
  p->n = n;
  p->fmt = FMT_CSR;
  p->prec = precision;
  p->nnz = (int64_t)cc.size();
  for (int64_t i = 0; i < n; ++i) p->max_deg = std::max<int>(p->max_deg, rp[i + 1] - rp[i]);
  {
    const int64_t G = csr_res_grid(n, p->sms);   // rows split as k_csr_res splits them
    for (int64_t b = 0; b < G; ++b)
      p->res_nnz_max = std::max<int>(p->res_nnz_max, rp[(b + 1) * n / G] - rp[b * n / G]);
  }
  auto bail = [&](sbo_status s) { free_all(p); delete p; return s; };
  // weights in the storage type (exact by the checks above)
  std::vector<uint8_t> vbytes;
  size_t velt = 4;
  if (precision == SBO_FP32) {
    p->val_type = 0;
    vbytes.resize(cc.size() * 4);
    for (size_t k = 0; k < cc.size(); ++k) { float f = (float)vv[k]; std::memcpy(&vbytes[4 * k], &f, 4); }
  } else if (precision == SBO_BF16) {
    p->val_type = 1;
    velt = 2;
    vbytes.resize(cc.size() * 2);
    for (size_t k = 0; k < cc.size(); ++k) {
      __nv_bfloat16 h = __float2bfloat16_rn((float)vv[k]);
      std::memcpy(&vbytes[2 * k], &h, 2);
    }
  } else {
    p->val_type = 2;
    velt = 1;
    vbytes.resize(cc.size());
    for (size_t k = 0; k < cc.size(); ++k) {
      __nv_fp8_e4m3 q((float)vv[k]);
      vbytes[k] = q.__x;
    }
  }
  std::vector<float> cpf(n);
  for (int64_t i = 0; i < n; ++i) cpf[i] = (float)cp[i];
  cudaError_t e;
  cudaStream_t cs = p->stream;
  if ((e = dalloc(&p->rowptr, n + 1, cs)) != cudaSuccess || (e = dalloc(&p->col, cc.size(), cs)) != cudaSuccess ||
      (e = cudaMallocAsync(&p->val, std::max<size_t>(1, cc.size() * velt), cs)) != cudaSuccess ||
      (e = dalloc(&p->cp, n, cs)) != cudaSuccess || (e = dalloc(&p->cp64, n, cs)) != cudaSuccess)
    return bail(e == cudaErrorMemoryAllocation ? fail(SBO_ENOMEM, "device allocation failed") : cuda_fail(e, "cudaMalloc"));
  if ((e = cudaStreamSynchronize(cs)) != cudaSuccess ||
      (e = cudaMemcpy(p->rowptr, rp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (!cc.empty() && (e = cudaMemcpy(p->col, cc.data(), sizeof(int32_t) * cc.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (!cc.empty() && (e = cudaMemcpy(p->val, vbytes.data(), vbytes.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (e = cudaMemcpy(p->cp, cpf.data(), sizeof(float) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->cp64, cp.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(cuda_fail(e, "upload CSR"));
  *out = p;
  return SBO_OK;
}

sbo_status sbo_create_maxkcut(int64_t n, int64_t m, const int32_t* ei, const int32_t* ej, const int32_t* w, int32_t k,
                              void* stream, sbo_problem** out) {
  g_last_error.clear();
  if (!out) return fail(SBO_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || n >= (1ll << 31)) return fail(SBO_EINVAL, "n must be in [1, 2^31)");
  if (m < 0 || (m > 0 && (!ei || !ej || !w))) return fail(SBO_EINVAL, "m must be >= 0 and the edge arrays non-NULL");
  if (k < 2 || k > 8) return fail(SBO_EINVAL, "k must be in [2, 8]");
  // W symmetric: both directions of every edge, duplicates summed, zero sums dropped
  struct Trip { int32_t i, j; int64_t v; };
  std::vector<Trip> tr;
  tr.reserve((size_t)2 * m);
  for (int64_t e = 0; e < m; ++e) {
    const int32_t a = ei[e], b = ej[e];
    if (a < 0 || a >= n || b < 0 || b >= n) return fail(SBO_EINVAL, "edge end out of range");
    if (a == b) return fail(SBO_EINVAL, "self-loops are not allowed");
    tr.push_back({a, b, (int64_t)w[e]});
    tr.push_back({b, a, (int64_t)w[e]});
  }
  std::sort(tr.begin(), tr.end(), [](const Trip& x, const Trip& y) { return x.i != y.i ? x.i < y.i : x.j < y.j; });
  std::vector<int32_t> rp(n + 1, 0), cc;
  std::vector<float> vv;
  std::vector<int64_t> rowabs(n, 0);
  for (size_t q = 0; q < tr.size();) {
    size_t r = q;
    int64_t sum = 0;
    while (r < tr.size() && tr[r].i == tr[q].i && tr[r].j == tr[q].j) sum += tr[r++].v;
    if (sum != 0) {
      const int64_t a = sum < 0 ? -sum : sum;
      if (a > (1ll << 24)) return fail(SBO_ERANGE, "an edge weight is not exact in FP32");
      rowabs[tr[q].i] += a;
      cc.push_back(tr[q].j);
      vv.push_back((float)sum);
      rp[tr[q].i + 1]++;
    }
    q = r;
  }
  for (int64_t i = 0; i < n; ++i)
    if (rowabs[i] >= (1ll << 24)) return fail(SBO_ERANGE, "a row sum of |W_ij| reaches 2^24 (objective not exact)");
  if (cc.size() >= (size_t)INT32_MAX) return fail(SBO_EINVAL, "too many edges");
  for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  sbo_problem* p = new (std::nothrow) sbo_problem();
  if (!p) return fail(SBO_ENOMEM, "host allocation failed");
  sbo_status st = init_common(p, stream);
  auto bail = [&](sbo_status s2) { free_all(p); delete p; return s2; };
  if (st != SBO_OK) return bail(st);
  p->n = n;
  p->fmt = FMT_MAXK;
  p->prec = SBO_FP32;
  p->kparts = k;
  p->nnz = (int64_t)cc.size();
  p->val_type = 0;
  cudaError_t e;
  cudaStream_t cs = p->stream;
  if ((e = dalloc(&p->rowptr, n + 1, cs)) != cudaSuccess || (e = dalloc(&p->col, cc.size(), cs)) != cudaSuccess ||
      (e = cudaMallocAsync(&p->val, std::max<size_t>(1, vv.size() * 4), cs)) != cudaSuccess ||
      (e = dalloc(&p->cp, n, cs)) != cudaSuccess || (e = dalloc(&p->cp64, n, cs)) != cudaSuccess)
    return bail(e == cudaErrorMemoryAllocation ? fail(SBO_ENOMEM, "device allocation failed") : cuda_fail(e, "cudaMalloc"));
  if ((e = cudaStreamSynchronize(cs)) != cudaSuccess ||
      (e = cudaMemcpy(p->rowptr, rp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (!cc.empty() && (e = cudaMemcpy(p->col, cc.data(), sizeof(int32_t) * cc.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (!vv.empty() && (e = cudaMemcpy(p->val, vv.data(), sizeof(float) * vv.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (e = cudaMemset(p->cp, 0, sizeof(float) * n)) != cudaSuccess ||
      (e = cudaMemset(p->cp64, 0, sizeof(int64_t) * n)) != cudaSuccess)
    return bail(cuda_fail(e, "upload graph"));
  *out = p;
  return SBO_OK;
}

sbo_status sbo_set_option(sbo_problem* p, int32_t option, int64_t value) {
  g_last_error.clear();
  if (!p) return fail(SBO_EINVAL, "problem is NULL");
  switch (option) {
    case SBO_OPT_KERNEL:
      if (value < 0 || value > 3) return fail(SBO_EINVAL, "kernel option must be 0..3");
      p->opt_kernel = (int)value;
      return SBO_OK;
    case SBO_OPT_USE_GRAPH: p->opt_graph = value != 0; return SBO_OK;
    case SBO_OPT_TILE_N:
      if (value != 0 && value != 64 && value != 128 && value != 256 && value != 512 && value != 1064 &&
          value != 1128 && value != 1256 && value != 2128 && value != 2256)
        return fail(SBO_EINVAL,
                    "tile_n must be 0, 64, 128, 256, 512 (CTA pairs), 1064, 1128, 1256 (cluster split-K) or 2128, 2256 "
                    "(cluster split-K on CTA pairs)");
      p->opt_tile_n = (int)value;
      return SBO_OK;
    case SBO_OPT_AUTOTUNE: p->opt_autotune = value != 0; return SBO_OK;
    case SBO_OPT_PDL: p->opt_pdl = value != 0; return SBO_OK;
    case SBO_OPT_G:
      if (value != G_QUAD && value != G_ENTROPY) return fail(SBO_EINVAL, "g must be 0 (quadratic) or 1 (entropy)");
      p->opt_g = (int)value;
      return SBO_OK;
    case SBO_OPT_DUAL:
      if (value != 0 && value != 1) return fail(SBO_EINVAL, "dual form must be 0 (per coordinate) or 1 (per restart)");
      p->opt_dual = (int)value;
      return SBO_OK;
    case SBO_OPT_SPLIT_K:
      if (value < 0 || value > 64) return fail(SBO_EINVAL, "split-K factor must be in [0, 64]");
      p->opt_split_k = (int)value;
      return SBO_OK;
    case SBO_OPT_KEEP_GRAD: p->opt_keep_grad = value != 0; return SBO_OK;
    case SBO_OPT_EVAL_MODE:
      if (value < 0 || value > 2) return fail(SBO_EINVAL, "evaluation mode must be 0..2");
      p->opt_eval_mode = (int)value;
      return SBO_OK;
    case SBO_OPT_CSR_FORM:
      if (value < 0 || value > CSR_FORM_RESIDENT) return fail(SBO_EINVAL, "sparse form must be 0..8");
      p->opt_csr_form = (int)value;
      return SBO_OK;
    case SBO_OPT_STEPS_PER_LAUNCH:
      if (value < 0 || value > (1 << 20)) return fail(SBO_EINVAL, "steps per launch must be in [0, 2^20]");
      p->opt_steps_per_launch = value;
      return SBO_OK;
    case SBO_OPT_TIMEOUT_US:
      if (value < 1) return fail(SBO_EINVAL, "timeout must be >= 1 us");
      p->opt_timeout_us = value;
      return SBO_OK;
    default: return fail(SBO_EINVAL, "unknown option");
  }
}

sbo_status sbo_gda_start(sbo_problem* p, const sbo_gda_params* prm, const float* x0) {
  return sbo_gda_start_xy(p, prm, x0, nullptr);
}

sbo_status sbo_gda_start_xy(sbo_problem* p, const sbo_gda_params* prm, const float* x0, const float* y0) {
  g_last_error.clear();
  if (!p) return fail(SBO_EINVAL, "problem is NULL");
  sbo_status st = check_params(prm);
  if (st != SBO_OK) return st;
  // kernel selection
  int ker;
  if (p->fmt == FMT_MAXK) {
    if (p->opt_kernel != KER_AUTO) return fail(SBO_EINVAL, "Max-k-Cut problems use their own kernel only");
    if (p->opt_dual != 0) return fail(SBO_EINVAL, "Max-k-Cut runs the per-vertex dual");
    if (x0 || y0) return fail(SBO_EINVAL, "Max-k-Cut starts from its own random logits (x0, y0 must be NULL)");
    if (p->opt_g != G_QUAD) return fail(SBO_EINVAL, "Max-k-Cut uses the quadratic constraint function");
    if (p->opt_keep_grad) return fail(SBO_EINVAL, "Max-k-Cut runs do not keep the gradient");
    ker = KER_MAXK;
  } else if (p->fmt == FMT_CSR) {
    if (p->opt_kernel != KER_AUTO) return fail(SBO_EINVAL, "CSR problems use the CSR kernel only");
    ker = KER_CSR;
  } else if (p->opt_kernel != KER_AUTO) {
    ker = p->opt_kernel;
    if (ker == KER_TC && p->prec != SBO_BF16) return fail(SBO_EINVAL, "the tcgen05 kernel needs a BF16 problem");
    if ((ker == KER_SIMT || ker == KER_TINY) && p->prec != SBO_FP32)
      return fail(SBO_EINVAL, "the SIMT and tiny kernels need an FP32 problem");
    if (ker == KER_TINY && p->n > 64) return fail(SBO_EINVAL, "the tiny kernel needs n <= 64");
    if (ker == KER_TINY && p->opt_dual == 1)
      return fail(SBO_EINVAL, "the tiny kernel runs the per-coordinate dual only; use the SIMT kernel");
  } else if (p->prec == SBO_BF16) {
    ker = KER_TC;
  } else {
    ker = p->n <= 64 && p->opt_dual == 0 ? KER_TINY : KER_SIMT;
  }
  if (ker == KER_TC && !tc_supported()) return fail(SBO_ECUDA, "tcgen05 path needs a compute capability 10.3 device");
  free_run(p);
  p->prm = *prm;
  p->kernel = ker;
  p->B = prm->restarts;
  p->layout = (ker == KER_CSR || ker == KER_MAXK) ? LAYOUT_NR : LAYOUT_RN;
  p->op_type = (p->prec == SBO_FP32) ? OP_F32 : OP_BF16;
  p->ld = p->layout == LAYOUT_RN ? round_up(p->n, 8) : round_up(p->B, 8);
  p->t = 0;
  p->t_last_eval = 0;
  p->n_evals_host = 0;
  p->cur = 0;
  p->graph_blocks_seen = 0;
  const int64_t rows = p->layout == LAYOUT_RN ? p->B : p->n;
  const size_t elems = (size_t)rows * p->ld;
  const size_t op_elt = p->op_type == OP_F32 ? 4 : 2;
  cudaError_t e = cudaSuccess;
  const bool need_master = ker == KER_TINY || ker == KER_MAXK || p->op_type != OP_F32;
  const size_t xelems = elems * (ker == KER_MAXK ? (size_t)p->kparts : 1);   // Max-k-Cut: k logits
  // min-F trace: one entry per evaluation up to T, plus slack for runs continued beyond T
  const int64_t evals_T = prm->iters / prm->eval_every + 2;
  p->trace_cap = std::min<int64_t>(evals_T, 1 << 20) + 4096;
  auto al = [&](void** q, size_t bytes) {
    if (e == cudaSuccess) e = cudaMallocAsync(q, bytes ? bytes : 1, p->stream);
  };
  if (need_master) al((void**)&p->Xm, xelems * 4);
  al((void**)&p->Y, elems * 4);
  if (p->opt_keep_grad) al((void**)&p->Gd, elems * 4);
  if (ker != KER_TINY) {
    al(&p->Xop[0], xelems * op_elt);
    al(&p->Xop[1], xelems * op_elt);
    al(&p->bits, elems * (ker == KER_CSR ? 1 : op_elt));   // the sparse path keeps candidates as bytes
  }
  al((void**)&p->bestF, sizeof(long long) * p->B);
  al((void**)&p->bestT, sizeof(long long) * p->B);
  al((void**)&p->evalF, sizeof(long long) * p->B);
  al((void**)&p->F2, sizeof(unsigned long long) * p->B);
  al((void**)&p->commit_ctr, sizeof(unsigned int));
  p->single = p->opt_dual == 1;
  if (p->single) {
    // rows of partial sums the update kernel writes: 4 per 128 variables (tcgen05 kernels; CTA
    // pairs round up to 256), 1 per 64 variables (SIMT), 1 per block along the rows (CSR)
    p->gpart_rows = ker == KER_TC ? (p->n + 255) / 256 * 8 : ker == KER_SIMT ? (p->n + 63) / 64
                                                                             : csr_partial_rows(p->n, p->B);
    p->gpart_ld = round_up(p->B, 8);
    al((void**)&p->mu, sizeof(float) * p->gpart_ld);
    al((void**)&p->gpart, sizeof(float) * p->gpart_rows * p->gpart_ld);
  }
  al((void**)&p->bestBits, elems);
  al((void**)&p->trace, sizeof(long long) * p->trace_cap);
  al((void**)&p->n_evals, sizeof(long long));
  al((void**)&p->t_last, sizeof(long long));
  al((void**)&p->sel, sizeof(long long) * 3);
  if (e != cudaSuccess) {
    free_run(p);
    return e == cudaErrorMemoryAllocation ? fail(SBO_ENOMEM, "device allocation of the run state failed")
                                          : cuda_fail(e, "cudaMalloc");
  }
  cudaStream_t s = p->stream;
  // zero every buffer so padding never holds stale values; sentinels for bests and trace
  if (p->Xm) cudaMemsetAsync(p->Xm, 0, xelems * 4, s);
  cudaMemsetAsync(p->Y, 0, elems * 4, s);
  if (p->Gd) cudaMemsetAsync(p->Gd, 0, elems * 4, s);
  for (void* b : {p->Xop[0], p->Xop[1]})
    if (b) cudaMemsetAsync(b, 0, xelems * op_elt, s);
  if (p->bits) cudaMemsetAsync(p->bits, 0, elems * (ker == KER_CSR ? 1 : op_elt), s);
  launch_fill_i64(p->bestF, p->B, LLONG_MAX, s);
  launch_fill_i64(p->bestT, p->B, -1, s);
  launch_fill_i64(p->trace, p->trace_cap, LLONG_MAX, s);
  p->launches += 3;
  cudaMemsetAsync(p->F2, 0, sizeof(unsigned long long) * p->B, s);
  cudaMemsetAsync(p->commit_ctr, 0, sizeof(unsigned int), s);
  cudaMemsetAsync(p->bestBits, 0, elems, s);
  cudaMemsetAsync(p->n_evals, 0, sizeof(long long), s);
  cudaMemsetAsync(p->t_last, 0, sizeof(long long), s);
  if (ker == KER_TC) {
    // split-K workspace (sized for the widest tile): one partial tile per CTA, arrival counters
    // per tail tile slice
    if (p->opt_split_k >= 2) {
      if ((e = dalloc(&p->tc_ws, (size_t)p->sms * 256 * 128, s)) != cudaSuccess ||
          (e = dalloc(&p->tc_ctr, (size_t)p->sms * TC_WS_COUNTERS_PER_TILE, s)) != cudaSuccess) {
        free_run(p);
        return e == cudaErrorMemoryAllocation ? fail(SBO_ENOMEM, "device allocation of the split-K workspace failed")
                                              : cuda_fail(e, "cudaMalloc");
      }
      cudaMemsetAsync(p->tc_ctr, 0, sizeof(int) * p->sms * TC_WS_COUNTERS_PER_TILE, s);
    }
    if ((e = dalloc(&p->tc_gbar, 3, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->tc_gbar, 0, 3 * sizeof(unsigned int), s)) != cudaSuccess) {
      free_run(p);
      return cuda_fail(e, "grid barrier words");
    }
    // the cluster split-K kernel serves problems with at most sms / 2 tiles (fewest at width 256),
    // on CTA pairs at most sms / 4 tiles of 256 x 256
    if ((p->opt_tile_n == 0 || p->opt_tile_n >= 1000) &&
        ((int64_t)((p->n + 127) / 128) * ((p->B + 255) / 256) * 2 <= p->sms ||
         (int64_t)((p->n + 255) / 256) * ((p->B + 255) / 256) * 4 <= p->sms) &&
        (e = dalloc(&p->csk_ws, (size_t)p->sms * 256 * 128, s)) != cudaSuccess) {
      free_run(p);
      return e == cudaErrorMemoryAllocation ? fail(SBO_ENOMEM, "device allocation of the cluster workspace failed")
                                            : cuda_fail(e, "cudaMalloc");
    }
    int tn = p->opt_tile_n;
    std::string why;
    if (tn == 0 && p->opt_autotune) {
      sbo_status st2 = tune_tile(p, &tn);   // runs on the zeroed state, before x^0 is written
      if (st2 != SBO_OK) { free_run(p); return st2; }
    } else if (tn == 0) {
      tn = heuristic_tile(p);
    }
    const int tuned_csk = tn / 10000;   // cluster size decided by the autotuner (0: none)
    tn %= 10000;
    if (tn == 512 && !tc_pair_supported(nullptr)) tn = 256;
    e = tc_make_plan(&p->plan, p->A, p->lda, (int)p->n, p->Xop[0], p->Xop[1], p->bits, p->ld, p->B,
                     tile_width(tn), &why);
    if (e != cudaSuccess) { free_run(p); return fail(SBO_ECUDA, "tensor-core plan: " + why); }
    p->plan.pair = tn == 512;
    p->plan.csk = 0;
    p->plan.csk_pair = false;
    if (tn >= 1000) {
      p->plan.csk_pair = tn >= 2000;
      p->plan.csk = !p->csk_ws ? 0 : tuned_csk >= 2 ? tuned_csk : csk_factor_for(p, tn, p->plan);
      if (p->plan.csk < 2) {   // too many tiles for clusters: plain tiles of the same width per CTA
        p->plan.csk = 0;
        p->plan.csk_pair = false;
        tn = tile_width(tn);
      }
    }
    p->tile_n = tn;
    attach_workspace(p, &p->plan);
  } else {
    p->tile_n = 0;
  }
  p->csr_form = CSR_FORM_RULE;
  if (ker == KER_CSR && !p->single) {
    // grid barrier words of the resident form (allocated before the autotuner, which times it)
    if ((e = dalloc(&p->tc_gbar, 3, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->tc_gbar, 0, 3 * sizeof(unsigned int), s)) != cudaSuccess) {
      free_run(p);
      return cuda_fail(e, "grid barrier words");
    }
    if (p->opt_csr_form != 0) {
      p->csr_form = p->opt_csr_form;
    } else if (p->opt_autotune) {
      int f = CSR_FORM_RULE;
      sbo_status st2 = tune_csr_form(p, &f);   // on the zeroed state, before x^0 is written
      if (st2 != SBO_OK) { free_run(p); return st2; }
      p->csr_form = f;
    }
    int D, S, rc;
    size_t sm;
    if (p->csr_form == CSR_FORM_STAGED && !csr_staged_shape(p->ld, p->op_type, p->max_deg, &D, &S, &rc, &sm))
      p->csr_form = CSR_FORM_RULE;
    int rg;
    if (p->csr_form == CSR_FORM_RESIDENT && !csr_res_shape(p->n, p->B, p->sms, p->res_nnz_max, &rg, &sm))
      p->csr_form = CSR_FORM_RULE;   // the state does not fit in shared memory
    p->tile_n = p->csr_form;   // reported by sbo_info
  }
  float* x0d = nullptr;
  float* y0d = nullptr;
  if (y0) {
    for (int64_t k = 0; k < (int64_t)p->B * p->n; ++k)
      if (!std::isfinite(y0[k])) { free_run(p); return fail(SBO_EINVAL, "y0 holds a non-finite value"); }
  }
  for (int q = 0; q < 2; ++q) {
    const float* src = q == 0 ? x0 : y0;
    float** dst = q == 0 ? &x0d : &y0d;
    if (!src) continue;
    if ((e = dalloc(dst, (size_t)p->B * p->n, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(*dst, src, sizeof(float) * p->B * p->n, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
      dfree(x0d, s); dfree(y0d, s); free_run(p); return cuda_fail(e, "upload of x0 / y0");
    }
  }
  if (p->single) {
    // after the autotuner, whose trial launches may write rows the chosen kernel does not
    std::vector<float> mu0((size_t)p->gpart_ld, 0.0f);
    for (int r = 0; r < p->B; ++r) mu0[r] = y0 ? y0[(size_t)r * p->n] : (float)prm->ybar;
    if ((e = cudaMemsetAsync(p->gpart, 0, sizeof(float) * p->gpart_rows * p->gpart_ld, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(p->mu, mu0.data(), sizeof(float) * p->gpart_ld, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
      dfree(x0d, s); dfree(y0d, s); free_run(p); return cuda_fail(e, "single-constraint dual set-up");
    }
  }
  if (ker == KER_MAXK)
    e = launch_maxk_init((int)p->n, p->B, p->ld, p->kparts, prm->seed, (float)prm->ybar, p->Xm, p->Y,
                         static_cast<float*>(p->Xop[0]), s);
  else
    e = launch_init_state((int)p->n, p->B, p->ld, p->layout, prm->seed, (float)prm->ybar, x0d, y0d, p->Xm,
                          ker == KER_TINY ? (void*)p->Xm : p->Xop[0], ker == KER_TINY ? OP_F32 : p->op_type, p->Y,
                          p->err, s);
  ++p->launches;
  if (x0d || y0d) { cudaStreamSynchronize(s); dfree(x0d, s); dfree(y0d, s); }
  if (e != cudaSuccess) { free_run(p); return cuda_fail(e, "init launch"); }
  p->started = true;
  return SBO_OK;
}

sbo_status sbo_gda_run(sbo_problem* p, int64_t iters) {
  g_last_error.clear();
  if (!p) return fail(SBO_EINVAL, "problem is NULL");
  if (!p->started) return fail(SBO_ENOTREADY, "sbo_gda_start has not been called");
  if (iters < 0) return fail(SBO_EINVAL, "iters must be >= 0");
  if (iters == 0) return SBO_OK;
  if (p->kernel == KER_TINY) return run_tiny(p, iters);
  const int64_t K = p->prm.eval_every;
  const int64_t t_end = p->t + iters;
  while (p->t < t_end) {
    if (p->eval_pending && !defer_evals(p)) {   // deferral switched off (graphs): evaluate in line
      sbo_status st = flush_pending(p);
      if (st != SBO_OK) return st;
    }
    const int64_t nx = next_eval_after(p, p->t);
    const int64_t stop = std::min(nx, t_end);
    const int64_t steps = stop - p->t;
    const bool eval_here = stop == nx;
    // the records are current up to t, or the candidates of t are pending and the records up to
    // t - K (the graphs bake the evaluation's distance K)
    const bool aligned = p->t_last_eval == p->t || (p->eval_pending && p->t_last_eval + K == p->t);
    const bool eligible = p->opt_graph && eval_here && steps == K && p->t % K == 0 && aligned;
    // a captured block pays off only when it is replayed: the first eligible block of a run is
    // launched directly, later ones are replayed from graphs
    if (eligible && p->graph_blocks_seen++ >= 1) {
      const int par = p->cur;
      const bool defer = defer_evals(p);
      const int kind = !defer ? BLOCK_EVAL : p->eval_pending ? BLOCK_BESIDE : BLOCK_DEFER;
      cudaGraphExec_t* slot = kind == BLOCK_EVAL ? p->gexec : kind == BLOCK_DEFER ? p->gexec_nv : p->gexec_ov;
      if (!slot[par]) {
        sbo_status st = capture_block(p, par, kind);
        if (st != SBO_OK) return st;
      }
      cudaError_t e = cudaGraphLaunch(slot[par], p->stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
      p->launches += p->graph_launches[kind][par];
      if (K & 1) p->cur ^= 1;
      if (kind == BLOCK_BESIDE) {   // the pending candidates of the block's first iteration
        p->t_last_eval = p->t;
        ++p->n_evals_host;
      }
      p->t += K;
      if (kind == BLOCK_EVAL) {
        p->t_last_eval = p->t;
        ++p->n_evals_host;
      }
      p->eval_pending = kind != BLOCK_EVAL;
    } else {
      sbo_status st = run_direct(p, steps, eval_here);
      if (st != SBO_OK) return st;
    }
  }
  return SBO_OK;
}

sbo_status sbo_sync(sbo_problem* p) {
  g_last_error.clear();
  if (!p) return fail(SBO_EINVAL, "problem is NULL");
  sbo_status st = flush_pending(p);
  if (st != SBO_OK) return st;
  SBO_CUDA(cudaStreamSynchronize(p->stream));
  return read_err(p);
}

sbo_status sbo_gda(sbo_problem* p, const sbo_gda_params* prm) {
  sbo_status st = sbo_gda_start(p, prm, nullptr);
  if (st != SBO_OK) return st;
  st = sbo_gda_run(p, prm->iters);
  if (st != SBO_OK) return st;
  return sbo_sync(p);
}

sbo_status sbo_eval(sbo_problem* p, int64_t count, const uint8_t* bits, int64_t* F) {
  g_last_error.clear();
  if (!p) return fail(SBO_EINVAL, "problem is NULL");
  if (count < 0 || (count > 0 && (!bits || !F))) return fail(SBO_EINVAL, "bad count or NULL arrays");
  if (count == 0) return SBO_OK;
  if (count > (1 << 20)) return fail(SBO_EINVAL, "count too large");
  const int vmax = p->fmt == FMT_MAXK ? p->kparts - 1 : 1;
  for (int64_t k = 0; k < count * p->n; ++k)
    if (bits[k] > vmax) return fail(SBO_EINVAL, p->fmt == FMT_MAXK ? "parts must be < k" : "bits must be 0 or 1");
  cudaStream_t s = p->stream;
  const int layout = p->fmt == FMT_DENSE ? LAYOUT_RN : LAYOUT_NR;
  const int op = p->fmt == FMT_CSR ? OP_U8 : p->prec == SBO_FP32 ? OP_F32 : OP_BF16;
  const int64_t ld = layout == LAYOUT_RN ? round_up(p->n, 8) : round_up(count, 8);
  const int64_t rows = layout == LAYOUT_RN ? count : p->n;
  uint8_t* bd = nullptr;
  void* opd = nullptr;
  unsigned long long* f2 = nullptr;
  auto cleanup = [&]() { dfree(bd, s); if (opd) cudaFreeAsync(opd, s); opd = nullptr; dfree(f2, s); };
  cudaError_t e;
  if ((e = dalloc(&bd, (size_t)count * p->n, s)) != cudaSuccess ||
      (e = cudaMallocAsync(&opd, (size_t)rows * ld * (op == OP_F32 ? 4 : op == OP_U8 ? 1 : 2), s)) != cudaSuccess ||
      (e = dalloc(&f2, count, s)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "cudaMalloc (eval)");
  }
  cudaMemsetAsync(opd, 0, (size_t)rows * ld * (op == OP_F32 ? 4 : op == OP_U8 ? 1 : 2), s);
  cudaMemsetAsync(f2, 0, sizeof(unsigned long long) * count, s);
  if ((e = cudaMemcpyAsync(bd, bits, (size_t)count * p->n, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "copy bits");
  }
  e = launch_bits_to_operand(bd, (int)p->n, (int)count, opd, ld, layout, op, s);
  ++p->launches;
  EpiArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = (int)p->n;
  a.B = (int)count;
  a.ld = ld;
  a.cp = p->cp;
  a.cp64 = p->cp64;
  a.Xin = opd;
  a.F2 = f2;
  a.err = p->err;
  if (e == cudaSuccess) {
    ++p->launches;
    if (p->fmt == FMT_MAXK) {
      e = launch_maxk(p->rowptr, p->col, static_cast<const float*>(p->val), a, p->kparts, EPI_EVAL, s);
    } else if (p->fmt == FMT_CSR) {
      e = launch_csr(p->rowptr, p->col, p->val, p->val_type, a, op, EPI_EVAL, false, s);
    } else if (p->prec == SBO_FP32) {
      e = launch_simt(static_cast<const float*>(p->A), p->lda, a, EPI_EVAL, s);
    } else {
      TcPlan plan{};
      std::string why;
      const int tn = 64;
      e = tc_make_plan(&plan, p->A, p->lda, (int)p->n, opd, nullptr, nullptr, ld, (int)count, tn, &why);
      if (e != cudaSuccess) { cleanup(); return fail(SBO_ECUDA, "tensor-core plan: " + why); }
      e = launch_tc(plan, 0, nullptr, a, EPI_EVAL, timeout_ns(p), s);
    }
  }
  std::vector<unsigned long long> h(count);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), f2, sizeof(unsigned long long) * count, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "evaluation");
  sbo_status st = read_err(p);
  if (st != SBO_OK) return st;
  for (int64_t k = 0; k < count; ++k) F[k] = (int64_t)(long long)h[k] / 2;
  return SBO_OK;
}

sbo_status sbo_best(sbo_problem* p, uint8_t* x_out, int64_t* F_out, int64_t* iter_out, int32_t* restart_out) {
  g_last_error.clear();
  if (!p) return fail(SBO_EINVAL, "problem is NULL");
  if (p->started) {
    sbo_status st = flush_pending(p);
    if (st != SBO_OK) return st;
  }
  if (!p->started || p->n_evals_host == 0) return fail(SBO_ENOTREADY, "no evaluation has taken place yet");
  cudaStream_t s = p->stream;
  cudaError_t e = launch_best_select(p->bestF, p->bestT, p->B, p->sel, s);
  ++p->launches;
  if (e != cudaSuccess) return cuda_fail(e, "best selection");
  long long h[3];
  SBO_CUDA(cudaMemcpyAsync(h, p->sel, sizeof(h), cudaMemcpyDeviceToHost, s));
  SBO_CUDA(cudaStreamSynchronize(s));
  sbo_status st = read_err(p);
  if (st != SBO_OK) return st;
  if (h[1] < 0 || h[2] < 0 || h[2] >= p->B) return fail(SBO_EDEVICE, "inconsistent best record");
  if (F_out) *F_out = h[0];
  if (iter_out) *iter_out = h[1];
  if (restart_out) *restart_out = (int32_t)h[2];
  if (x_out) {
    const int64_t r = h[2];
    if (p->layout == LAYOUT_RN) {
      SBO_CUDA(cudaMemcpy(x_out, p->bestBits + r * p->ld, (size_t)p->n, cudaMemcpyDeviceToHost));
    } else {
      SBO_CUDA(cudaMemcpy2D(x_out, 1, p->bestBits + r, (size_t)p->ld, 1, (size_t)p->n, cudaMemcpyDeviceToHost));
    }
  }
  return SBO_OK;
}

sbo_status sbo_restart_best(sbo_problem* p, int64_t* F, int64_t* t) {
  g_last_error.clear();
  if (!p) return fail(SBO_EINVAL, "problem is NULL");
  if (!p->started) return fail(SBO_ENOTREADY, "sbo_gda_start has not been called");
  sbo_status st = flush_pending(p);
  if (st != SBO_OK) return st;
  SBO_CUDA(cudaStreamSynchronize(p->stream));
  if (F) SBO_CUDA(cudaMemcpy(F, p->bestF, sizeof(int64_t) * p->B, cudaMemcpyDeviceToHost));
  if (t) SBO_CUDA(cudaMemcpy(t, p->bestT, sizeof(int64_t) * p->B, cudaMemcpyDeviceToHost));
  return read_err(p);
}

sbo_status sbo_state(sbo_problem* p, float* X, float* Y) {
  g_last_error.clear();
  if (!p) return fail(SBO_EINVAL, "problem is NULL");
  if (!p->started) return fail(SBO_ENOTREADY, "sbo_gda_start has not been called");
  cudaStream_t s = p->stream;
  float* tmp = nullptr;
  const int kx = p->kernel == KER_MAXK ? p->kparts : 1;   // Max-k-Cut: X_:,i has k entries
  SBO_CUDA(dalloc(&tmp, (size_t)p->B * p->n * kx, s));
  const float* xsrc = p->Xm ? p->Xm : static_cast<const float*>(p->Xop[p->cur]);
  cudaError_t e = cudaSuccess;
  if (X) {
    if (p->kernel == KER_MAXK)
      e = launch_maxk_gather(static_cast<const float*>(p->Xop[p->cur]), (int)p->n, kx, p->B, p->ld, tmp, s);
    else
      e = launch_gather_state(xsrc, (int)p->n, p->B, p->ld, p->layout, tmp, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(X, tmp, sizeof(float) * p->B * p->n * kx, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (Y && e == cudaSuccess && p->single) {
    // one dual per restart: every coordinate of restart r reports mu_r
    std::vector<float> mu((size_t)p->B);
    e = cudaMemcpyAsync(mu.data(), p->mu, sizeof(float) * p->B, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int64_t r = 0; r < p->B && e == cudaSuccess; ++r) std::fill(Y + r * p->n, Y + (r + 1) * p->n, mu[r]);
  } else if (Y && e == cudaSuccess) {
    e = launch_gather_state(p->Y, (int)p->n, p->B, p->ld, p->layout, tmp, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Y, tmp, sizeof(float) * p->B * p->n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  dfree(tmp, s);
  if (e != cudaSuccess) return cuda_fail(e, "state read-back");
  return read_err(p);
}

sbo_status sbo_gradient(sbo_problem* p, float* G) {
  g_last_error.clear();
  if (!p || !G) return fail(SBO_EINVAL, "problem or G is NULL");
  if (!p->started) return fail(SBO_ENOTREADY, "sbo_gda_start has not been called");
  if (!p->Gd) return fail(SBO_ENOTREADY, "the run was started without SBO_OPT_KEEP_GRAD");
  if (p->t < 1) return fail(SBO_ENOTREADY, "no iteration has run yet");
  cudaStream_t s = p->stream;
  float* tmp = nullptr;
  SBO_CUDA(dalloc(&tmp, (size_t)p->B * p->n, s));
  cudaError_t e = launch_gather_state(p->Gd, (int)p->n, p->B, p->ld, p->layout, tmp, s);
  ++p->launches;
  if (e == cudaSuccess) e = cudaMemcpyAsync(G, tmp, sizeof(float) * p->B * p->n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dfree(tmp, s);
  if (e != cudaSuccess) return cuda_fail(e, "gradient read-back");
  return read_err(p);
}

sbo_status sbo_trace(sbo_problem* p, int64_t* minF, int64_t cap, int64_t* count) {
  g_last_error.clear();
  if (!p) return fail(SBO_EINVAL, "problem is NULL");
  if (!p->started) return fail(SBO_ENOTREADY, "sbo_gda_start has not been called");
  sbo_status st = flush_pending(p);
  if (st != SBO_OK) return st;
  SBO_CUDA(cudaStreamSynchronize(p->stream));
  long long ne = 0;
  SBO_CUDA(cudaMemcpy(&ne, p->n_evals, sizeof(ne), cudaMemcpyDeviceToHost));
  if (count) *count = ne;
  const int64_t m = std::min<int64_t>(std::min<int64_t>(ne, cap), p->trace_cap);
  if (minF && m > 0) SBO_CUDA(cudaMemcpy(minF, p->trace, sizeof(int64_t) * m, cudaMemcpyDeviceToHost));
  return read_err(p);
}

sbo_status sbo_lagrangian(sbo_problem* p, int32_t B, const float* X_dev, const float* Y_dev, const float* gout_dev,
                          float* L_dev, float* GX_dev, float* GY_dev, void* stream) {
  g_last_error.clear();
  if (!p) return fail(SBO_EINVAL, "problem is NULL");
  if (B < 1 || !X_dev || !Y_dev) return fail(SBO_EINVAL, "B must be >= 1 and X, Y non-NULL");
  if (p->fmt == FMT_MAXK) return fail(SBO_EINVAL, "sbo_lagrangian supports QUBO problems (dense or CSR)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  EpiArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = (int)p->n;
  a.B = B;
  a.ld = p->n;
  a.cp = p->cp;
  a.cp64 = p->cp64;
  a.Xl = X_dev;
  a.Yl = Y_dev;
  a.L = L_dev;
  a.GX = GX_dev;
  a.GY = GY_dev;
  a.gout = gout_dev;
  a.err = p->err;
  a.gkind = p->opt_g;
  if (L_dev) SBO_CUDA(cudaMemsetAsync(L_dev, 0, sizeof(float) * B, s));
  cudaError_t e;
  if (p->fmt == FMT_CSR) {
    // sparse form: x goes to the variable-major operand of the sparse kernel (FP32, or BF16 for
    // BF16 / E4M3 weights), the epilogue reads the caller's FP32 x and y
    const int op = p->prec == SBO_FP32 ? OP_F32 : OP_BF16;
    const int64_t ldx = round_up(B, 8);
    const size_t need = (size_t)p->n * ldx * (op == OP_F32 ? 4 : 2);
    if (need > p->lag_cap) {
      if (p->lag_op) { cudaStreamSynchronize(s); cudaFree(p->lag_op); p->lag_op = nullptr; p->lag_cap = 0; }
      SBO_CUDA(cudaMalloc(&p->lag_op, need));   // used on the caller's stream: not stream-ordered
      p->lag_cap = need;
    }
    SBO_CUDA(cudaMemsetAsync(p->lag_op, 0, need, s));
    e = launch_to_operand_t(X_dev, (int)p->n, B, p->n, p->lag_op, ldx, op, s);
    if (e != cudaSuccess) return cuda_fail(e, "operand conversion");
    a.Xin = p->lag_op;
    a.ld = ldx;
    e = launch_csr(p->rowptr, p->col, p->val, p->val_type, a, op, EPI_LAGR, false, s);
    p->launches += 2;
  } else if (p->prec == SBO_FP32) {
    a.Xin = X_dev;
    e = launch_simt(static_cast<const float*>(p->A), p->lda, a, EPI_LAGR, s);
    ++p->launches;
  } else {
    const int64_t ldx = round_up(p->n, 8);
    const size_t need = (size_t)B * ldx * 2;
    if (need > p->lag_cap) {
      if (p->lag_op) { cudaStreamSynchronize(s); cudaFree(p->lag_op); p->lag_op = nullptr; p->lag_cap = 0; }
      SBO_CUDA(cudaMalloc(&p->lag_op, need));   // used on the caller's stream: not stream-ordered
      SBO_CUDA(cudaMemsetAsync(p->lag_op, 0, need, s));
      p->lag_cap = need;
    }
    e = launch_to_operand(X_dev, (int)p->n, B, p->n, p->lag_op, ldx, OP_BF16, s);
    if (e != cudaSuccess) return cuda_fail(e, "operand conversion");
    TcPlan plan{};
    std::string why;
    int tn = 256;
    while (tn > 64 && (int64_t)((p->n + 127) / 128) * ((B + tn - 1) / tn) < p->sms) tn /= 2;
    e = tc_make_plan(&plan, p->A, p->lda, (int)p->n, p->lag_op, nullptr, nullptr, ldx, B, tn, &why);
    if (e != cudaSuccess) return fail(SBO_ECUDA, "tensor-core plan: " + why);
    e = launch_tc(plan, 0, nullptr, a, EPI_LAGR, timeout_ns(p), s);
    p->launches += 2;
  }
  if (e != cudaSuccess) return cuda_fail(e, "Lagrangian launch");
  return SBO_OK;
}

sbo_status sbo_dual_bound(sbo_problem* p, double ybar, double alpha, int64_t iters, double* lower_bound,
                          double* value) {
  g_last_error.clear();
  if (!p) return fail(SBO_EINVAL, "problem is NULL");
  if (p->fmt == FMT_MAXK) return fail(SBO_EINVAL, "the dual certificate is offered for QUBO problems");
  if (!lower_bound) return fail(SBO_EINVAL, "lower_bound is NULL");
  if (!std::isfinite(ybar) || ybar <= 0 || !std::isfinite(alpha) || alpha <= 0 || iters < 0)
    return fail(SBO_EINVAL, "ybar and alpha must be finite and > 0, iters >= 0");
  // projected gradient descent on L(., ybar): GDA with beta = 0 (y stays ybar > 0, so the
  // perturbation rule never fires), one restart
  sbo_gda_params prm{};
  prm.restarts = 1;
  prm.iters = iters > 0 ? iters : 1;
  prm.eval_every = (int32_t)std::min<int64_t>(prm.iters, INT32_MAX);
  prm.alpha = alpha;
  prm.beta = 0.0;
  prm.ybar = ybar;
  prm.delta = 0.0;
  prm.grad_tol = 0.0;
  prm.seed = 0;
  const int saved_dual = p->opt_dual, saved_g = p->opt_g;
  p->opt_dual = 0;
  p->opt_g = G_QUAD;   // the bound below is formed for the quadratic g
  sbo_status st = sbo_gda_start(p, &prm, nullptr);
  p->opt_dual = saved_dual;
  p->opt_g = saved_g;
  if (st != SBO_OK) return st;
  if (iters > 0 && (st = sbo_gda_run(p, iters)) != SBO_OK) return st;
  if ((st = sbo_sync(p)) != SBO_OK) return st;
  const int64_t n = p->n;
  cudaStream_t s = p->stream;
  std::vector<float> xf((size_t)n);
  std::vector<double> xd((size_t)n), g((size_t)n);
  std::vector<int64_t> cp((size_t)n);
  float* tmp = nullptr;
  double *xdev = nullptr, *gdev = nullptr;
  cudaError_t e = cudaSuccess;
  if ((e = dalloc(&tmp, (size_t)n, s)) != cudaSuccess || (e = dalloc(&xdev, (size_t)n, s)) != cudaSuccess ||
      (e = dalloc(&gdev, (size_t)n, s)) != cudaSuccess) {
    dfree(tmp, s); dfree(xdev, s); dfree(gdev, s);
    return cuda_fail(e, "cudaMalloc (dual bound)");
  }
  const float* xsrc = p->Xm ? p->Xm : static_cast<const float*>(p->Xop[p->cur]);
  e = launch_gather_state(xsrc, (int)n, 1, p->ld, p->layout, tmp, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(xf.data(), tmp, sizeof(float) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cp.data(), p->cp64, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (int64_t i = 0; i < n; ++i) xd[i] = (double)xf[i];
  if (e == cudaSuccess) e = cudaMemcpyAsync(xdev, xd.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s);
  DenseView v{};
  const bool dense = dense_view(p, &v);
  // FP64 polish of the point (the fast path's operand may be BF16), then g = A x at the final point
  const int64_t polish = std::min<int64_t>(iters, 500);
  for (int64_t k = 0; k < polish && e == cudaSuccess; ++k) {
    e = launch_matvec_f64(dense ? &v : nullptr, p->rowptr, p->col, p->val, p->val_type, (int)n, xdev, gdev, s);
    if (e == cudaSuccess) e = launch_pgd_step_f64(xdev, gdev, p->cp64, (int)n, ybar, alpha, s);
    p->launches += 2;
  }
  if (e == cudaSuccess) {
    e = launch_matvec_f64(dense ? &v : nullptr, p->rowptr, p->col, p->val, p->val_type, (int)n, xdev, gdev, s);
    ++p->launches;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(xd.data(), xdev, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g.data(), gdev, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dfree(tmp, s); dfree(xdev, s); dfree(gdev, s);
  if (e != cudaSuccess) return cuda_fail(e, "dual bound");
  // L(x) and the linearisation bound min over the box of L(x) + <grad, z - x> (valid when L(., ybar)
  // is convex on the box), in FP64
  double L = 0.0, gap = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const double x = xd[i], c = (double)cp[i];
    L += 0.5 * x * g[i] + c * x + ybar * (x * x - x);
    const double grad = g[i] + c + ybar * (2.0 * x - 1.0);
    gap += grad * x - std::min(0.0, grad);
  }
  *lower_bound = L - gap;
  if (value) *value = L;
  return read_err(p);
}

sbo_status sbo_info(const sbo_problem* p, int64_t* n, int32_t* restarts, int32_t* kernel, int32_t* tile_n, int64_t* t) {
  g_last_error.clear();
  if (!p) return fail(SBO_EINVAL, "problem is NULL");
  if (n) *n = p->n;
  if (restarts) *restarts = p->B;
  if (kernel) *kernel = p->kernel;
  if (tile_n) *tile_n = p->tile_n;
  if (t) *t = p->t;
  return SBO_OK;
}

int64_t sbo_launch_count(const sbo_problem* p) { return p ? p->launches : 0; }

void sbo_destroy(sbo_problem* p) {
  if (!p) return;
  cudaStreamSynchronize(p->stream);
  free_all(p);
  delete p;
}

}  // extern "C"

// ---- internal accessors for entry points defined in other translation units ---------------
namespace sbo {

bool dense_view(sbo_problem* p, DenseView* v) {
  if (!p || p->fmt != FMT_DENSE) return false;
  v->n = p->n;
  v->prec = p->prec;
  v->A = p->A;
  v->lda = p->lda;
  v->cp = p->cp;
  v->cp64 = p->cp64;
  v->err = p->err;
  v->timeout_ns = timeout_ns(p);
  v->gkind = p->opt_g;
  v->sms = p->sms;
  v->launches = &p->launches;
  return true;
}

void set_last_error(const std::string& msg) { g_last_error = msg; }

}  // namespace sbo

// =============================================================================================
// Grouped runs: several dense BF16 problems advanced together, one persistent tcgen05 launch
// per iteration over the tiles of every instance.
struct sbo_group {
  std::vector<sbo_problem*> members;  // not owned
  std::vector<int> order;             // member indices by decreasing n (instance table order)
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int tile_n = 128;           // width in use
  int opt_tile_n = 0;         // requested width; 0 = autotune at start
  TcInst* d_insts = nullptr;
  CommitArgs* d_commit = nullptr;     // per-member evaluation commit arguments
  int64_t max_n = 0, max_B = 0;
  int num_tiles = 0;
  bool started = false;
  int64_t T = 0, K = 1;
  int64_t t = 0, t_last_eval = 0, n_evals_host = 0;
  int cur = 0;
  int opt_graph = 1;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  int64_t launches = 0;
};

namespace {

void group_free_graphs(sbo_group* g) {
  for (auto& x : g->gexec)
    if (x) { cudaGraphExecDestroy(x); x = nullptr; }
}

cudaError_t group_step(sbo_group* g, bool write_bits, cudaStream_t s) {
  ++g->launches;
  const int variant = 2 * g->cur + (write_bits ? 1 : 0);
  cudaError_t e = launch_tc_group(g->d_insts, (int)g->members.size(), g->num_tiles, g->tile_n, EPI_UPDATE, variant,
                                  timeout_ns(g->members[0]), s);
  g->cur ^= 1;
  return e;
}

cudaError_t group_eval(sbo_group* g, int64_t add, cudaStream_t s) {
  cudaError_t e = launch_tc_group(g->d_insts, (int)g->members.size(), g->num_tiles, g->tile_n, EPI_EVAL, 4,
                                  timeout_ns(g->members[0]), s);
  ++g->launches;
  if (e != cudaSuccess) return e;
  // members are restart-major: rows are restarts, the contiguous dimension is the variables
  e = launch_eval_commit_group(g->d_commit, (int)g->members.size(), g->max_n, g->max_B, add, s);
  ++g->launches;
  return e;
}

sbo_status group_capture(sbo_group* g, int parity) {
  const int saved = g->cur;
  const int64_t saved_l = g->launches;
  g->cur = parity;
  cudaGraph_t gr = nullptr;
  SBO_CUDA(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  for (int64_t s = 0; s < g->K && err == cudaSuccess; ++s) err = group_step(g, s + 1 == g->K, g->cap_stream);
  if (err == cudaSuccess) err = group_eval(g, g->K, g->cap_stream);
  cudaError_t e2 = cudaStreamEndCapture(g->cap_stream, &gr);
  g->cur = saved;
  g->launches = saved_l;
  if (err != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    return cuda_fail(err, "launch during graph capture");
  }
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  cudaError_t e3 = cudaGraphInstantiate(&g->gexec[parity], gr, 0);
  cudaGraphDestroy(gr);
  if (e3 != cudaSuccess) return cuda_fail(e3, "cudaGraphInstantiate");
  return SBO_OK;
}

// Keep every member's own counters in step with the group's (so sbo_best, sbo_state, ... and
// later single-problem runs see a consistent state).
void group_sync_members(sbo_group* g) {
  for (sbo_problem* p : g->members) {
    p->t = g->t;
    p->t_last_eval = g->t_last_eval;
    p->n_evals_host = g->n_evals_host;
    p->cur = g->cur;
  }
}

sbo_status group_start_tile(sbo_group* g, const sbo_gda_params* prms, int tile_n) {
  const size_t cnt = g->members.size();
  for (size_t k = 0; k < cnt; ++k) {
    sbo_status st = check_params(&prms[k]);
    if (st != SBO_OK) return st;
    if (prms[k].iters != prms[0].iters || prms[k].eval_every != prms[0].eval_every)
      return fail(SBO_EINVAL, "members of a group share iters and eval_every");
  }
  group_free_graphs(g);
  if (g->d_insts || g->d_commit) cudaStreamSynchronize(g->stream);
  if (g->d_insts) { cudaFree(g->d_insts); g->d_insts = nullptr; }
  if (g->d_commit) { cudaFree(g->d_commit); g->d_commit = nullptr; }
  g->started = false;
  // start every member on the group's tile width, then build the instance table
  for (size_t k = 0; k < cnt; ++k) {
    sbo_problem* p = g->members[k];
    if (p->opt_dual != 0) return fail(SBO_EINVAL, "grouped runs use the per-coordinate dual");
    p->opt_kernel = KER_TC;
    p->opt_tile_n = tile_n;
    p->opt_split_k = 0;
    sbo_status st = sbo_gda_start(p, &prms[k], nullptr);
    if (st != SBO_OK) return st;
    SBO_CUDA(cudaStreamSynchronize(p->stream));
  }
  g->order.resize(cnt);
  for (size_t k = 0; k < cnt; ++k) g->order[k] = (int)k;
  std::stable_sort(g->order.begin(), g->order.end(),
                   [&](int a, int b) { return g->members[a]->n > g->members[b]->n; });
  std::vector<TcInst> tab(cnt);
  int tiles = 0;
  for (size_t q = 0; q < cnt; ++q) {
    sbo_problem* p = g->members[g->order[q]];
    TcInst& I = tab[q];
    std::memset(&I, 0, sizeof(I));
    I.mapA = p->plan.mapA;
    for (int k = 0; k < 3; ++k) I.mapX[k] = p->plan.mapX[k];
    for (int cur = 0; cur < 2; ++cur)
      for (int wb = 0; wb < 2; ++wb) {
        EpiArgs a = base_args(p);
        a.Xin = p->Xop[cur];
        a.Xout = p->Xop[cur ^ 1];
        a.bits_out = wb ? p->bits : nullptr;
        I.epi[2 * cur + wb] = a;
      }
    EpiArgs ev = base_args(p);
    ev.Xin = p->bits;
    I.epi[4] = ev;
    I.n_tiles = (p->B + tile_n - 1) / tile_n;
    I.kblocks = (int)((p->n + 63) / 64);
    I.tile_begin = tiles;
    tiles += (int)((p->n + 127) / 128) * I.n_tiles;
  }
  g->num_tiles = tiles;
  g->tile_n = tile_n;
  SBO_CUDA(cudaMalloc(&g->d_insts, sizeof(TcInst) * cnt));
  SBO_CUDA(cudaMemcpy(g->d_insts, tab.data(), sizeof(TcInst) * cnt, cudaMemcpyHostToDevice));
  std::vector<CommitArgs> ctab(cnt);
  g->max_n = g->max_B = 0;
  for (size_t k = 0; k < cnt; ++k) {
    ctab[k] = commit_args(g->members[k]);
    g->max_n = std::max<int64_t>(g->max_n, g->members[k]->n);
    g->max_B = std::max<int64_t>(g->max_B, g->members[k]->B);
  }
  SBO_CUDA(cudaMalloc(&g->d_commit, sizeof(CommitArgs) * cnt));
  SBO_CUDA(cudaMemcpy(g->d_commit, ctab.data(), sizeof(CommitArgs) * cnt, cudaMemcpyHostToDevice));
  g->T = prms[0].iters;
  g->K = prms[0].eval_every;
  g->t = g->t_last_eval = g->n_evals_host = 0;
  g->cur = 0;
  g->started = true;
  group_sync_members(g);
  return SBO_OK;
}

}  // namespace

extern "C" {

sbo_status sbo_group_create(int32_t count, sbo_problem* const* problems, void* stream, sbo_group** out) {
  g_last_error.clear();
  if (!out) return fail(SBO_EINVAL, "out is NULL");
  *out = nullptr;
  if (count < 1 || !problems) return fail(SBO_EINVAL, "count must be >= 1 and problems non-NULL");
  for (int32_t k = 0; k < count; ++k) {
    if (!problems[k]) return fail(SBO_EINVAL, "a member problem is NULL");
    if (problems[k]->fmt != FMT_DENSE || problems[k]->prec != SBO_BF16)
      return fail(SBO_EINVAL, "grouped runs take dense BF16 problems");
    for (int32_t q = 0; q < k; ++q)
      if (problems[q] == problems[k]) return fail(SBO_EINVAL, "a problem appears twice in the group");
  }
  if (!tc_supported()) return fail(SBO_ECUDA, "grouped runs need a compute capability 10.3 device");
  sbo_group* g = new (std::nothrow) sbo_group();
  if (!g) return fail(SBO_ENOMEM, "host allocation failed");
  g->members.assign(problems, problems + count);
  g->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { delete g; return cuda_fail(e, "cudaStreamCreate"); }
  *out = g;
  return SBO_OK;
}

// Tile width of a group: the one given, or (0) the fastest of the candidates, each timed on the
// group's own instance table over a few grouped update launches.
sbo_status sbo_group_start(sbo_group* g, const sbo_gda_params* prms) {
  g_last_error.clear();
  if (!g || !prms) return fail(SBO_EINVAL, "group or params is NULL");
  if (g->opt_tile_n != 0) return group_start_tile(g, prms, g->opt_tile_n);
  int max_B = 1;
  for (size_t k = 0; k < g->members.size(); ++k) max_B = std::max(max_B, prms[k].restarts);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SBO_CUDA(cudaEventCreate(&e0));
  SBO_CUDA(cudaEventCreate(&e1));
  int best = 128;
  float best_ms = 1e30f;
  sbo_status st = SBO_OK;
  for (int tn : {64, 128, 256}) {
    if (tn > 64 && tn / 2 >= max_B) continue;
    st = group_start_tile(g, prms, tn);
    if (st != SBO_OK) break;
    const int reps = 3;
    cudaError_t e = group_step(g, false, g->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, g->stream);
    for (int k = 0; k < reps && e == cudaSuccess; ++k) e = group_step(g, false, g->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, g->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) { st = cuda_fail(e, "group autotuner launch"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) { best_ms = ms; best = tn; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SBO_OK) return st;
  st = read_err(g->members[0]);
  if (st != SBO_OK) return st;
  return group_start_tile(g, prms, best);   // fresh state on the chosen width
}

sbo_status sbo_group_run(sbo_group* g, int64_t iters) {
  g_last_error.clear();
  if (!g) return fail(SBO_EINVAL, "group is NULL");
  if (!g->started) return fail(SBO_ENOTREADY, "sbo_group_start has not been called");
  if (iters < 0) return fail(SBO_EINVAL, "iters must be >= 0");
  const int64_t t_end = g->t + iters;
  while (g->t < t_end) {
    int64_t nx = (g->t / g->K + 1) * g->K;
    if (g->T > g->t && g->T < nx) nx = g->T;
    const int64_t stop = std::min(nx, t_end);
    const int64_t steps = stop - g->t;
    const bool eval_here = stop == nx;
    if (g->opt_graph && eval_here && steps == g->K && g->t % g->K == 0 && g->t_last_eval == g->t) {
      const int par = g->cur;
      if (!g->gexec[par]) {
        sbo_status st = group_capture(g, par);
        if (st != SBO_OK) return st;
      }
      cudaError_t e = cudaGraphLaunch(g->gexec[par], g->stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
      g->launches += g->K + 2;
      if (g->K & 1) g->cur ^= 1;
      g->t += g->K;
      g->t_last_eval = g->t;
      ++g->n_evals_host;
    } else {
      for (int64_t s = 0; s < steps; ++s) {
        cudaError_t e = group_step(g, eval_here && s + 1 == steps, g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "grouped step launch");
      }
      g->t += steps;
      if (eval_here) {
        cudaError_t e = group_eval(g, g->t - g->t_last_eval, g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "grouped evaluation launch");
        g->t_last_eval = g->t;
        ++g->n_evals_host;
      }
    }
  }
  group_sync_members(g);
  return SBO_OK;
}

sbo_status sbo_group_sync(sbo_group* g) {
  g_last_error.clear();
  if (!g) return fail(SBO_EINVAL, "group is NULL");
  SBO_CUDA(cudaStreamSynchronize(g->stream));
  for (sbo_problem* p : g->members) {
    sbo_status st = read_err(p);
    if (st != SBO_OK) return st;
  }
  return SBO_OK;
}

sbo_status sbo_group_set_option(sbo_group* g, int32_t option, int64_t value) {
  g_last_error.clear();
  if (!g) return fail(SBO_EINVAL, "group is NULL");
  if (option == SBO_OPT_USE_GRAPH) { g->opt_graph = value != 0; return SBO_OK; }
  if (option == SBO_OPT_TILE_N) {
    if (value != 0 && value != 64 && value != 128 && value != 256)
      return fail(SBO_EINVAL, "tile_n must be 0 (autotune), 64, 128 or 256");
    g->opt_tile_n = (int)value;
    return SBO_OK;
  }
  return fail(SBO_EINVAL, "groups take SBO_OPT_USE_GRAPH and SBO_OPT_TILE_N");
}

int64_t sbo_group_launch_count(const sbo_group* g) { return g ? g->launches : 0; }

void sbo_group_destroy(sbo_group* g) {
  if (!g) return;
  cudaStreamSynchronize(g->stream);
  group_free_graphs(g);
  if (g->d_insts) cudaFree(g->d_insts);
  if (g->d_commit) cudaFree(g->d_commit);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  delete g;
}

}  // extern "C"
