// FP64 instances of the Krylov items kernels without options; the instances with the
// observables at beta/2 are in kt_items_f64_opt.cu, those with the work counters in
// kt_items_f64_stats.cu, compiled alongside.
#include "kt_items.cuh"

namespace kt {

int dispatch_items_f64_opt(int kd, const DevModel &M, const SeqView &S, const MoveView &mv, int has_moves,
                           const Workspace &ws, kt_stats *stats, cudaStream_t st);
int dispatch_items_cached_f64_opt(int kd, const DevModel &M, const SeqView &S, const MoveView &mv,
                                  const Workspace &ws, const CacheView &C, kt_stats *stats, cudaStream_t st);
int dispatch_items_f64_stats(int kd, int opt, const DevModel &M, const SeqView &S, const MoveView &mv, int has_moves,
                             const Workspace &ws, kt_stats *stats, cudaStream_t st);
int dispatch_items_cached_f64_stats(int kd, int opt, const DevModel &M, const SeqView &S, const MoveView &mv,
                                    const Workspace &ws, const CacheView &C, kt_stats *stats, cudaStream_t st);

int dispatch_items_f64(int kd, int G, const DevModel &M, const SeqView &S, const MoveView &mv, int has_moves,
                       const Workspace &ws, kt_stats *stats, cudaStream_t st) {
  const int opt = dev::items_options<double>(kd, M, ws, stats);
  if (opt & dev::KT_OPT_STATS) return dispatch_items_f64_stats(kd, opt, M, S, mv, has_moves, ws, stats, st);
  if (opt) return dispatch_items_f64_opt(kd, M, S, mv, has_moves, ws, stats, st);
  return dev::dispatch_items<double>(kd, G, M, S, mv, has_moves, ws, stats, st);
}

// Cached-mode items (the sweep's partial-state cache) at the default lane-group size
// of each row capacity.
int dispatch_items_cached_f64(int kd, const DevModel &M, const SeqView &S, const MoveView &mv, const Workspace &ws,
                              const CacheView &C, kt_stats *stats, cudaStream_t st) {
  const int opt = dev::items_options<double>(kd, M, ws, stats);
  if (opt & dev::KT_OPT_STATS) return dispatch_items_cached_f64_stats(kd, opt, M, S, mv, ws, C, stats, st);
  if (opt) return dispatch_items_cached_f64_opt(kd, M, S, mv, ws, C, stats, st);
  switch (kd) {
    case 10: return dev::launch_items_cached<double, 4, 10, 10, 0>(M, S, mv, ws, C, stats, st);
    case 36: return dev::launch_items_cached<double, 16, 36, 24, 0>(M, S, mv, ws, C, stats, st);
    case 128: return dev::launch_items_cached<double, 32, 128, 40, 0>(M, S, mv, ws, C, stats, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace kt
