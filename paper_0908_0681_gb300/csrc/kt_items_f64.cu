// FP64 instantiations of the Krylov items kernel.
#include "kt_items.cuh"

namespace kt {

int dispatch_items_f64(int kd, int G, const DevModel &M, const SeqView &S, const MoveView &mv, int has_moves,
                       const Workspace &ws, kt_stats *stats, cudaStream_t st) {
  return dev::dispatch_items<double>(kd, G, M, S, mv, has_moves, ws, stats, st);
}

}  // namespace kt
