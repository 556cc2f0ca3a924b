// FP64 instances of the Krylov items kernels that count the work into kt_stats (KT_OPT_STATS,
// with KT_OPT_MEAS as asked), at the default lane-group size of each row capacity (the counts
// and the results do not depend on the tiling).
#include "kt_items.cuh"

namespace kt {

int dispatch_items_f64_stats(int kd, int opt, const DevModel &M, const SeqView &S, const MoveView &mv, int has_moves,
                             const Workspace &ws, kt_stats *stats, cudaStream_t st) {
  using namespace dev;
  constexpr int MS = KT_OPT_MEAS, SC = KT_OPT_STATS;
  const bool m = (opt & MS) != 0;
  switch (kd) {
    case 10:
      return m ? launch_items<double, 4, 10, 10, SC | MS>(M, S, mv, has_moves, ws, stats, st)
               : launch_items<double, 4, 10, 10, SC>(M, S, mv, has_moves, ws, stats, st);
    case 36:
      return m ? launch_items<double, 16, 36, 24, SC | MS>(M, S, mv, has_moves, ws, stats, st)
               : launch_items<double, 16, 36, 24, SC>(M, S, mv, has_moves, ws, stats, st);
    case 128:
      return m ? launch_items<double, 32, 128, 40, SC | MS>(M, S, mv, has_moves, ws, stats, st)
               : launch_items<double, 32, 128, 40, SC>(M, S, mv, has_moves, ws, stats, st);
  }
  return (int)cudaErrorInvalidValue;
}

int dispatch_items_cached_f64_stats(int kd, int opt, const DevModel &M, const SeqView &S, const MoveView &mv,
                                    const Workspace &ws, const CacheView &C, kt_stats *stats, cudaStream_t st) {
  using namespace dev;
  constexpr int MS = KT_OPT_MEAS, SC = KT_OPT_STATS;
  const bool m = (opt & MS) != 0;
  switch (kd) {
    case 10:
      return m ? launch_items_cached<double, 4, 10, 10, SC | MS>(M, S, mv, ws, C, stats, st)
               : launch_items_cached<double, 4, 10, 10, SC>(M, S, mv, ws, C, stats, st);
    case 36:
      return m ? launch_items_cached<double, 16, 36, 24, SC | MS>(M, S, mv, ws, C, stats, st)
               : launch_items_cached<double, 16, 36, 24, SC>(M, S, mv, ws, C, stats, st);
    case 128:
      return m ? launch_items_cached<double, 32, 128, 40, SC | MS>(M, S, mv, ws, C, stats, st)
               : launch_items_cached<double, 32, 128, 40, SC>(M, S, mv, ws, C, stats, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace kt
