// FP64 instantiations of the Krylov items kernel.
#include "kt_items.cuh"

namespace kt {

int dispatch_items_f64(int kd, int G, const DevModel &M, const SeqView &S, const MoveView &mv, int has_moves,
                       const Workspace &ws, kt_stats *stats, cudaStream_t st) {
  return dev::dispatch_items<double>(kd, G, M, S, mv, has_moves, ws, stats, st);
}

// Cached-mode items (the sweep's partial-state cache) at the default lane-group size
// of each row capacity.
int dispatch_items_cached_f64(int kd, const DevModel &M, const SeqView &S, const MoveView &mv, const Workspace &ws,
                              const CacheView &C, kt_stats *stats, cudaStream_t st) {
  switch (kd) {
    case 10: return dev::launch_items_cached<double, 4, 10, 10>(M, S, mv, ws, C, stats, st);
    case 36: return dev::launch_items_cached<double, 16, 36, 24>(M, S, mv, ws, C, stats, st);
    case 128: return dev::launch_items_cached<double, 32, 128, 40>(M, S, mv, ws, C, stats, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace kt
