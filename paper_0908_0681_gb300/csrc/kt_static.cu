// Allocation-free trace ratio.
//
// kt_trace_ratio needs a device workspace from its caller. Some callers cannot
// provide one: code that must not call cudaMalloc after start-up (a real-time
// loop, a host runtime that hands out all device memory itself and forbids
// other allocations, or a caller whose only memory is the inputs and outputs
// another component already owns). kt_trace_ratio_static serves them: it runs
// the same pipeline with its scratch in a fixed-size array that lives in the
// library's device image, and it allocates nothing.
//
// The array holds KT_STATIC_SCRATCH_BYTES on every GPU that loads the library,
// until the process exits. All calls share it and it keeps the last call's
// contents: the pipeline itself resets the counters that must start at zero,
// and every other scratch entry is written before it is read. Calls whose
// kernels overlap on the GPU (for example on two streams) race on the array;
// serialise them.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "kt_internal.h"

namespace {

static __device__ __align__(256) unsigned char kt_static_scratch[KT_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};
std::mutex g_scratch_mu;

// The driver's current context (through the runtime's entry-point lookup, so that the
// library needs no link against the driver library); nullptr if unavailable.
CUcontext current_context() {
  using Fn = CUresult (*)(CUcontext *);
  static Fn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<Fn>(p);
    cudaGetLastError();
  }
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

// Device address of the scratch array on the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached together with the context it
// belongs to: after a device reset the runtime creates a new context and loads the
// library's device image again, so a context other than the cached one looks the
// address up afresh.
kt_status scratch_address(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return KT_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  const CUcontext ctx = current_context();
  if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, kt_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return KT_ECUDA;
    }
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = current_context();  // the lookup may have made the primary context current
  }
  *out = g_scratch_addr[dev];
  return KT_OK;
}

}  // namespace

extern "C" kt_status kt_trace_ratio_static(kt_model *m, const kt_seq_batch *cur, const int8_t *cur_sign,
                                           const double *cur_logabs, const kt_move_batch *moves, int8_t *sign,
                                           double *logratio, int32_t *status, kt_stats *stats, void *stream) {
  if (!m || !cur || !moves || cur->n < 0) return KT_EINVAL;
  const kt::ModelView v = kt::model_view(m);
  if (v.host_only) return KT_EINVAL;
  if (cur->n == 0) return KT_OK;
  if (!sign || !logratio || !status || !cur->offsets || !cur_sign || !cur_logabs || !moves->kind || !moves->flavor ||
      !moves->t_dag || !moves->t_ann || !moves->rem_idx)
    return KT_EINVAL;
  if (kt::workspace_bytes(cur->n, v.dev->n_kept, v.dev->d_max) > (size_t)KT_STATIC_SCRATCH_BYTES) return KT_ENOMEM;
  // the scratch array of the current device must sit beside the model's tables
  if (!kt::on_model_device(v)) return KT_EINVAL;
  void *scratch = nullptr;
  const kt_status rc = scratch_address(&scratch);
  if (rc != KT_OK) return rc;
  kt::SeqView sv{cur->n, cur->offsets, cur->tau, cur->flavor, cur->dagger};
  kt::MoveView mv{moves->kind, moves->flavor, moves->t_dag, moves->t_ann, moves->rem_idx};
  const kt::Workspace w = kt::carve_workspace(scratch, cur->n, v.dev->n_kept, v.dev->d_max);
  const int e = kt::launch_pipeline(*v.dev, v.precision, v.kernel_dmax, v.group_lanes, sv, &mv, cur_sign, cur_logabs,
                                    sign, logratio, status, stats, w, stream, nullptr);
  return e == 0 ? KT_OK : KT_ECUDA;
}
