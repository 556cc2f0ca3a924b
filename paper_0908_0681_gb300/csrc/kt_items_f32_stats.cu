// FP32-Krylov instances of the Krylov items kernels that count the work into kt_stats
// (KT_OPT_STATS, with KT_OPT_TRI64 and KT_OPT_MEAS as asked), at the default lane-group size of
// each row capacity: a counted launch takes that size whatever the model's tiling (the counts
// and the results do not depend on it).
#include "kt_items.cuh"

namespace kt {

int dispatch_items_f32_stats(int kd, int opt, const DevModel &M, const SeqView &S, const MoveView &mv, int has_moves,
                             const Workspace &ws, kt_stats *stats, cudaStream_t st) {
  using namespace dev;
  constexpr int T = KT_OPT_TRI64, MS = KT_OPT_MEAS, SC = KT_OPT_STATS;
  switch (kd) {
    case 10:
      switch (opt) {
        case SC: return launch_items<float, 8, 10, 10, SC>(M, S, mv, has_moves, ws, stats, st);
        case SC | MS: return launch_items<float, 8, 10, 10, SC | MS>(M, S, mv, has_moves, ws, stats, st);
        case SC | T: return launch_items<float, 8, 10, 10, SC | T>(M, S, mv, has_moves, ws, stats, st);
        case SC | T | MS: return launch_items<float, 8, 10, 10, SC | T | MS>(M, S, mv, has_moves, ws, stats, st);
      }
      break;
    case 36:
      if (opt == SC) return launch_items<float, 16, 36, 24, SC>(M, S, mv, has_moves, ws, stats, st);
      if (opt == (SC | MS)) return launch_items<float, 16, 36, 24, SC | MS>(M, S, mv, has_moves, ws, stats, st);
      break;
    case 128:
      if (opt == SC) return launch_items<float, 32, 128, 40, SC>(M, S, mv, has_moves, ws, stats, st);
      if (opt == (SC | MS)) return launch_items<float, 32, 128, 40, SC | MS>(M, S, mv, has_moves, ws, stats, st);
      break;
  }
  return (int)cudaErrorInvalidValue;
}

int dispatch_items_cached_f32_stats(int kd, int opt, const DevModel &M, const SeqView &S, const MoveView &mv,
                                    const Workspace &ws, const CacheView &C, kt_stats *stats, cudaStream_t st) {
  using namespace dev;
  constexpr int T = KT_OPT_TRI64, MS = KT_OPT_MEAS, SC = KT_OPT_STATS;
  switch (kd) {
    case 10:
      switch (opt) {
        case SC: return launch_items_cached<float, 8, 10, 10, SC>(M, S, mv, ws, C, stats, st);
        case SC | MS: return launch_items_cached<float, 8, 10, 10, SC | MS>(M, S, mv, ws, C, stats, st);
        case SC | T: return launch_items_cached<float, 8, 10, 10, SC | T>(M, S, mv, ws, C, stats, st);
        case SC | T | MS: return launch_items_cached<float, 8, 10, 10, SC | T | MS>(M, S, mv, ws, C, stats, st);
      }
      break;
    case 36:
      if (opt == SC) return launch_items_cached<float, 16, 36, 24, SC>(M, S, mv, ws, C, stats, st);
      if (opt == (SC | MS)) return launch_items_cached<float, 16, 36, 24, SC | MS>(M, S, mv, ws, C, stats, st);
      break;
    case 128:
      if (opt == SC) return launch_items_cached<float, 32, 128, 40, SC>(M, S, mv, ws, C, stats, st);
      if (opt == (SC | MS)) return launch_items_cached<float, 32, 128, 40, SC | MS>(M, S, mv, ws, C, stats, st);
      break;
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace kt
