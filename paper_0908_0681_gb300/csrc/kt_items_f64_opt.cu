// FP64 instances of the Krylov items kernels with the observables at beta/2 (KT_OPT_MEAS), at
// the default lane-group size of each row capacity (the results do not depend on the tiling).
#include "kt_items.cuh"

namespace kt {

int dispatch_items_f64_opt(int kd, const DevModel &M, const SeqView &S, const MoveView &mv, int has_moves,
                           const Workspace &ws, kt_stats *stats, cudaStream_t st) {
  using namespace dev;
  constexpr int MS = KT_OPT_MEAS;
  switch (kd) {
    case 10: return launch_items<double, 4, 10, 10, MS>(M, S, mv, has_moves, ws, stats, st);
    case 36: return launch_items<double, 16, 36, 24, MS>(M, S, mv, has_moves, ws, stats, st);
    case 128: return launch_items<double, 32, 128, 40, MS>(M, S, mv, has_moves, ws, stats, st);
  }
  return (int)cudaErrorInvalidValue;
}

int dispatch_items_cached_f64_opt(int kd, const DevModel &M, const SeqView &S, const MoveView &mv,
                                  const Workspace &ws, const CacheView &C, kt_stats *stats, cudaStream_t st) {
  using namespace dev;
  constexpr int MS = KT_OPT_MEAS;
  switch (kd) {
    case 10: return launch_items_cached<double, 4, 10, 10, MS>(M, S, mv, ws, C, stats, st);
    case 36: return launch_items_cached<double, 16, 36, 24, MS>(M, S, mv, ws, C, stats, st);
    case 128: return launch_items_cached<double, 32, 128, 40, MS>(M, S, mv, ws, C, stats, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace kt
