// Trace ratios from cached partial states: the kt_ratio_cache_* entry points of
// include/kt.h. The cache stores, for fixed current configurations, the forward
// and backward states of Sec. III step 3 at every operator; a ratio then
// propagates only the window of the sequence that its update edits.
#include <cuda_runtime.h>

#include <new>

#include "kt_internal.h"

struct kt_ratio_cache {
  kt_model *model = nullptr;
  kt::ModelView mv{};
  int n = 0;
  kt::CacheView C{};
  void *mem = nullptr;
  void *ws = nullptr;
  int words = 0;  // 32-bit words per cached vector
};

namespace {

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" {

kt_status kt_ratio_cache_create(kt_model *m, int32_t n_walkers, int32_t max_ops, kt_ratio_cache **out) {
  if (!m || !out || n_walkers < 1 || max_ops < 1) return KT_EINVAL;
  *out = nullptr;
  const kt::ModelView mv = kt::model_view(m);
  if (mv.host_only) return KT_EINVAL;
  const kt::DevModel &M = *mv.dev;
  kt_ratio_cache *c = new (std::nothrow) kt_ratio_cache();
  if (!c) return KT_ENOMEM;
  c->model = m;
  c->mv = mv;
  c->n = n_walkers;
  const size_t items = (size_t)n_walkers * M.n_kept, slots = items * ((size_t)max_ops + 1);
  const size_t esz = mv.precision == KT_FP64 ? 8 : 4, dv = (size_t)M.d_max;
  size_t b = 0;
  auto take = [&](size_t bytes) {
    const size_t at = b;
    b += up256(bytes);
    return at;
  };
  // cache and scratch (the tentative window states of kt_ratio_cache_propose)
  size_t o_vec[4], o_log[4], o_blk[4];
  for (int k = 0; k < 4; ++k) {
    o_vec[k] = take(slots * dv * esz);
    o_log[k] = take(slots * 16);
    o_blk[k] = take(slots * 4);
  }
  const size_t o_f = take(items * 4), o_gr = take(items * 4), o_plan = take(items * 16);
  kt_status rc = KT_OK;
  if (cudaMalloc(&c->mem, b) != cudaSuccess) {
    c->mem = nullptr;
    rc = KT_ENOMEM;
  } else if (cudaMemset(c->mem, 0, b) != cudaSuccess) {
    rc = KT_ECUDA;
  }
  const size_t wsb = kt::workspace_bytes(n_walkers, M.n_kept, M.d_max, 0);
  if (rc == KT_OK && cudaMalloc(&c->ws, wsb) != cudaSuccess) {
    c->ws = nullptr;
    rc = KT_ENOMEM;
  }
  if (rc != KT_OK) {
    cudaGetLastError();
    kt_ratio_cache_destroy(c);
    return rc;
  }
  char *p = (char *)c->mem;
  kt::CacheView &C = c->C;
  C.P = max_ops;
  C.dv = (int)dv;
  C.fvec = p + o_vec[0];
  C.bvec = p + o_vec[1];
  C.sfvec = p + o_vec[2];
  C.sbvec = p + o_vec[3];
  C.flog = (double2 *)(p + o_log[0]);
  C.blog = (double2 *)(p + o_log[1]);
  C.sflog = (double2 *)(p + o_log[2]);
  C.sblog = (double2 *)(p + o_log[3]);
  C.fblk = (int32_t *)(p + o_blk[0]);
  C.bblk = (int32_t *)(p + o_blk[1]);
  C.sfblk = (int32_t *)(p + o_blk[2]);
  C.sbblk = (int32_t *)(p + o_blk[3]);
  C.f = (int32_t *)(p + o_f);
  C.gr = (int32_t *)(p + o_gr);
  C.plan = (int4 *)(p + o_plan);
  c->words = (int)(dv * esz / 4);
  *out = c;
  return KT_OK;
}

kt_status kt_ratio_cache_build(kt_ratio_cache *c, const kt_seq_batch *b, void *stream) {
  if (!c || !b || b->n != c->n || !b->offsets || !b->tau || !b->flavor || !b->dagger) return KT_EINVAL;
  const kt::DevModel &M = *c->mv.dev;
  const kt::SeqView sv{b->n, b->offsets, b->tau, b->flavor, b->dagger};
  const kt::Workspace w = kt::carve_workspace(c->ws, c->n, M.n_kept, M.d_max, 0);
  return kt::launch_cache_build(M, c->mv.precision, c->mv.kernel_dmax, sv, w, c->C, stream) == 0 ? KT_OK : KT_ECUDA;
}

static kt_status cached_ratio(kt_ratio_cache *c, const kt_seq_batch *cur, const int8_t *cur_sign,
                              const double *cur_logabs, const kt_move_batch *moves, int8_t *sign, double *logratio,
                              int32_t *status, kt_stats *stats, void *stream, bool keep) {
  if (!c || !cur || cur->n != c->n || !cur->offsets || !cur->tau || !cur->flavor || !cur->dagger || !moves ||
      !moves->kind || !moves->flavor || !moves->t_dag || !moves->t_ann || !moves->rem_idx || !cur_sign || !cur_logabs ||
      !sign || !logratio || !status)
    return KT_EINVAL;
  const kt::DevModel &M = *c->mv.dev;
  const kt::SeqView sv{cur->n, cur->offsets, cur->tau, cur->flavor, cur->dagger};
  const kt::MoveView mv{moves->kind, moves->flavor, moves->t_dag, moves->t_ann, moves->rem_idx};
  const kt::Workspace w = kt::carve_workspace(c->ws, c->n, M.n_kept, M.d_max, 0);
  const int rc = kt::launch_cached_pipeline(M, c->mv.precision, c->mv.kernel_dmax, sv, mv, cur_sign, cur_logabs, sign,
                                            logratio, status, w, c->C, keep, stats, stream);
  return rc == 0 ? KT_OK : KT_ECUDA;
}

kt_status kt_trace_ratio_cached(kt_ratio_cache *c, const kt_seq_batch *cur, const int8_t *cur_sign,
                                const double *cur_logabs, const kt_move_batch *moves, int8_t *sign, double *logratio,
                                int32_t *status, kt_stats *stats, void *stream) {
  return cached_ratio(c, cur, cur_sign, cur_logabs, moves, sign, logratio, status, stats, stream, false);
}

kt_status kt_ratio_cache_propose(kt_ratio_cache *c, const kt_seq_batch *cur, const int8_t *cur_sign,
                                 const double *cur_logabs, const kt_move_batch *moves, int8_t *sign, double *logratio,
                                 int32_t *status, kt_stats *stats, void *stream) {
  return cached_ratio(c, cur, cur_sign, cur_logabs, moves, sign, logratio, status, stats, stream, true);
}

kt_status kt_ratio_cache_commit(kt_ratio_cache *c, const int8_t *accepted, const int32_t *status, void *stream) {
  if (!c || !accepted || !status) return KT_EINVAL;
  const kt::DevModel &M = *c->mv.dev;
  const kt::Workspace w = kt::carve_workspace(c->ws, c->n, M.n_kept, M.d_max, 0);
  return kt::launch_cache_commit(c->C, c->n, M.n_kept, w.desc, w.wstatus, accepted, status, c->words, stream) == 0
             ? KT_OK
             : KT_ECUDA;
}

void kt_ratio_cache_destroy(kt_ratio_cache *c) {
  if (!c) return;
  if (c->ws) cudaFree(c->ws);
  if (c->mem) cudaFree(c->mem);
  delete c;
}

}  // extern "C"
