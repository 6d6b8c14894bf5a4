// sbo_lagrangian_noalloc: the Lagrangian value/gradient entry point for callers that must not
// allocate device memory.
//
// Who needs it: processes whose device memory is owned by a framework's pool or a fixed budget
// (an allocation behind the pool's back breaks its accounting, or fails once the budget is
// spent), and latency-bound loops that cannot afford the implicit synchronisation of
// cudaMalloc/cudaFree.  sbo_lagrangian keeps a growing BF16 operand buffer per handle and may
// allocate it on any call; this variant uses a fixed scratch array instead and never allocates.
// Dense problems only (FP32 or BF16).
//
// The scratch is a file-scope __device__ array of SCRATCH_BYTES.  Every GPU that loads the
// library holds it until the process exits.  Host code cannot use the array's name as a device
// address, so the first call on each device (with that device current) looks the address up
// with cudaGetSymbolAddress and caches it; make that first call before any stream capture.
// All calls on a device share the array and it keeps the last call's contents: calls whose
// work overlaps on the GPU (different streams, or different threads) race on it.
#include <cstring>
#include <mutex>
#include <string>

#include "sbo_internal.h"

namespace {

constexpr size_t SCRATCH_BYTES = size_t(16) << 20;  // 16 MiB: B * round_up(n, 8) BF16 values
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

std::mutex g_scratch_mutex;
void* g_scratch_addr[MAX_DEVICES] = {};

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

sbo_status fail(sbo_status s, const std::string& msg) {
  sbo::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" sbo_status sbo_lagrangian_noalloc(sbo_problem* p, int32_t B, const float* X_dev, const float* Y_dev,
                                             const float* gout_dev, float* L_dev, float* GX_dev, float* GY_dev,
                                             void* stream) {
  using namespace sbo;
  set_last_error("");
  DenseView v;
  if (!p) return fail(SBO_EINVAL, "problem is NULL");
  if (B < 1 || !X_dev || !Y_dev) return fail(SBO_EINVAL, "B must be >= 1 and X, Y non-NULL");
  if (!dense_view(p, &v)) return fail(SBO_EINVAL, "sbo_lagrangian_noalloc supports dense problems");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t ldx = (v.n + 7) / 8 * 8;
  const size_t need = (size_t)B * (size_t)ldx * 2;
  if (v.prec == SBO_BF16 && need > SCRATCH_BYTES)
    return fail(SBO_EINVAL, "sbo_lagrangian_noalloc: B * round_up(n, 8) * 2 = " + std::to_string(need) +
                                " bytes exceeds its fixed scratch of " + std::to_string(SCRATCH_BYTES) +
                                " bytes; split the batch or use sbo_lagrangian");
  EpiArgs a;
  memset(&a, 0, sizeof(a));
  a.n = (int)v.n;
  a.B = B;
  a.ld = v.n;
  a.cp = v.cp;
  a.cp64 = v.cp64;
  a.gkind = v.gkind;
  a.Xl = X_dev;
  a.Yl = Y_dev;
  a.L = L_dev;
  a.GX = GX_dev;
  a.GY = GY_dev;
  a.gout = gout_dev;
  a.err = v.err;
  cudaError_t e;
  if (L_dev && (e = cudaMemsetAsync(L_dev, 0, sizeof(float) * B, s)) != cudaSuccess)
    return fail(SBO_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  if (v.prec == SBO_FP32) {
    // the FP32 contraction reads X directly: no scratch involved
    a.Xin = X_dev;
    e = launch_simt(static_cast<const float*>(v.A), v.lda, a, EPI_LAGR, s);
    *v.launches += 1;
  } else {
    void* scratch = nullptr;
    if ((e = scratch_address(&scratch)) != cudaSuccess)
      return fail(SBO_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    e = launch_to_operand(X_dev, (int)v.n, B, v.n, scratch, ldx, OP_BF16, s);
    if (e != cudaSuccess) return fail(SBO_ECUDA, std::string("operand conversion: ") + cudaGetErrorString(e));
    TcPlan plan{};
    std::string why;
    int tn = 256;
    while (tn > 64 && (int64_t)((v.n + 127) / 128) * ((B + tn - 1) / tn) < v.sms) tn /= 2;
    e = tc_make_plan(&plan, v.A, v.lda, (int)v.n, scratch, nullptr, nullptr, ldx, B, tn, &why);
    if (e != cudaSuccess) return fail(SBO_ECUDA, "tensor-core plan: " + why);
    e = launch_tc(plan, 0, nullptr, a, EPI_LAGR, v.timeout_ns, s);
    *v.launches += 2;
  }
  if (e != cudaSuccess) return fail(SBO_ECUDA, std::string("Lagrangian launch: ") + cudaGetErrorString(e));
  return SBO_OK;
}
