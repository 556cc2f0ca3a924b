// FP32-Krylov instantiations of the Krylov items kernel.
#include "kt_items.cuh"

namespace kt {

int dispatch_items_f32(int kd, int G, const DevModel &M, const SeqView &S, const MoveView &mv, int has_moves,
                       const Workspace &ws, kt_stats *stats, cudaStream_t st) {
  return dev::dispatch_items<float>(kd, G, M, S, mv, has_moves, ws, stats, st);
}

}  // namespace kt
