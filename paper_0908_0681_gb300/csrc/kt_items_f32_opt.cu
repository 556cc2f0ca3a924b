// FP32-Krylov instances of the Krylov items kernels with options: KT_OPT_TRI64 (models created
// with KT_FP32_TRIDIAG64; blocks of at most 16 rows) at every lane-group size of that row
// capacity, and KT_OPT_MEAS (observables at beta/2) at the default lane-group size of each row
// capacity. A measurement launch takes that size whatever the model's tiling: its results do
// not depend on the tiling.
#include "kt_items.cuh"

namespace kt {

int dispatch_items_f32_opt(int kd, int G, int opt, const DevModel &M, const SeqView &S, const MoveView &mv,
                           int has_moves, const Workspace &ws, kt_stats *stats, cudaStream_t st) {
  using namespace dev;
  constexpr int T = KT_OPT_TRI64, MS = KT_OPT_MEAS;
  if (opt == T && kd == 10) {
    switch (G) {
      case 4: return launch_items<float, 4, 10, 10, T>(M, S, mv, has_moves, ws, stats, st);
      case 8: return launch_items<float, 8, 10, 10, T>(M, S, mv, has_moves, ws, stats, st);
      case 16: return launch_items<float, 16, 10, 10, T>(M, S, mv, has_moves, ws, stats, st);
      case 32: return launch_items<float, 32, 10, 10, T>(M, S, mv, has_moves, ws, stats, st);
    }
    return (int)cudaErrorInvalidValue;
  }
  if (opt == (T | MS) && kd == 10) return launch_items<float, 8, 10, 10, T | MS>(M, S, mv, has_moves, ws, stats, st);
  if (opt == MS) {
    switch (kd) {
      case 10: return launch_items<float, 8, 10, 10, MS>(M, S, mv, has_moves, ws, stats, st);
      case 36: return launch_items<float, 16, 36, 24, MS>(M, S, mv, has_moves, ws, stats, st);
      case 128: return launch_items<float, 32, 128, 40, MS>(M, S, mv, has_moves, ws, stats, st);
    }
  }
  return (int)cudaErrorInvalidValue;
}

int dispatch_items_cached_f32_opt(int kd, int opt, const DevModel &M, const SeqView &S, const MoveView &mv,
                                  const Workspace &ws, const CacheView &C, kt_stats *stats, cudaStream_t st) {
  using namespace dev;
  constexpr int T = KT_OPT_TRI64, MS = KT_OPT_MEAS;
  if (kd == 10) {
    switch (opt) {
      case T: return launch_items_cached<float, 8, 10, 10, T>(M, S, mv, ws, C, stats, st);
      case MS: return launch_items_cached<float, 8, 10, 10, MS>(M, S, mv, ws, C, stats, st);
      case T | MS: return launch_items_cached<float, 8, 10, 10, T | MS>(M, S, mv, ws, C, stats, st);
    }
    return (int)cudaErrorInvalidValue;
  }
  if (opt == MS) {
    switch (kd) {
      case 36: return launch_items_cached<float, 16, 36, 24, MS>(M, S, mv, ws, C, stats, st);
      case 128: return launch_items_cached<float, 32, 128, 40, MS>(M, S, mv, ws, C, stats, st);
    }
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace kt
