// Internal declarations shared by the host setup (kt_model.cpp) and the CUDA
// kernels (kt_kernels.cu). Not part of the public ABI.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "../../include/kt.h"

namespace kt {

// Device tables of one model (plain pointers into a single device allocation).
//
// Blocks: H_loc is block diagonal in the occupation basis. A block is the set
// of bitstrings with the same (n_up, n_dn) and, unless KT_SECTOR_BLOCKS is
// set, the same mask of singly occupied orbitals (spin flip and pair hopping
// of Eq. (H_loc) never change which orbitals hold exactly one electron).
// Inside a block, rows are the bitstrings in ascending order.
struct DevModel {
  int n_orb, nf, n_states, n_blocks, n_kept, d_max, pmax;
  int tri64;  // FP32 path: final tridiagonal exponential in FP64 (KT_FP32_TRIDIAG64)
  double beta, E0, tol, brk_rel;

  const int32_t *blk_off;     // [n_blocks] first global row of the block
  const int32_t *blk_dim;     // [n_blocks]
  const int32_t *blk_nnz;     // [n_blocks] ELL width (max off-diagonal entries per row)
  const int32_t *blk_ell;     // [n_blocks] first ELL slot of the block (row-major rows x width)
  const double *blk_shift;    // [n_blocks] lowest eigenvalue s_b of the block
  const double *blk_norm;     // [n_blocks] 1-norm of H_b - s_b
  const int32_t *blk_target;  // [n_blocks * nf * 2] block reached by c_f (dag 0) / c_f^+ (dag 1), -1 if none

  const uint16_t *st_bits;    // [n_states] bitstring of each global row
  const double *st_diag64;    // [n_states] diagonal of H - s_b
  const float *st_diag32;
  const int16_t *ell_col;     // [n_ell] column inside the block, -1 = padding
  const double *ell_val64;    // [n_ell] off-diagonal values
  const float *ell_val32;
  const uint16_t *partner;    // [n_states * nf] rank of (x ^ 1<<f) in its block | 0x8000 if the
                              //   Jordan-Wigner sign of c_f / c_f^+ on x is negative

  // S^2 inside each block (measurement at beta/2): diagonal per global row, ELL slot-major
  // entries rank | 0x8000 for -1 (0xFFFF padding), width and first slot per block
  const float *s2_diag;
  const uint16_t *s2_ell;
  const int32_t *blk_s2w, *blk_s2ell;

  // eigendecomposition of every block (setup's FP64 Jacobi): eigenvalue k of block b minus its
  // shift at global row blk_off[b] + k (ascending within the block), and its eigenvector at
  // blk_evec32[blk_evoff[b] + k * d_b + r], r = 0 .. d_b - 1 (blk_evec32lo: fl32(v - fl32(v))
  // of the FP64 component v, the low part of a double-float copy)
  const double *st_eval64;
  const float *st_eval32;
  const int32_t *blk_evoff;
  const float *blk_evec32;
  const float *blk_evec32lo;

  const int32_t *kept_blk;    // [n_kept]
  const double *kept_e;       // [n_kept] E - E0
  const int32_t *kept_off;    // [n_kept] offset into kept_vec (block dimension entries)
  const double *kept_vec64;
  const float *kept_vec32;
};

// Operator sequences: walker i owns entries offsets[i] .. offsets[i] + K_i - 1 with
// K_i = lens[i] when lens is set (fixed-capacity slots of the sweep state) and
// offsets[i+1] - offsets[i] otherwise (the CSR batches of the ABI).
struct SeqView {
  int n;
  const int32_t *offsets;
  const double *tau;
  const uint8_t *flavor;
  const uint8_t *dagger;
  const int32_t *lens = nullptr;
  bool trusted = false;  // sequences built by the library itself (the sweep): skip the O(K) validation
};

struct MoveView {
  const uint8_t *kind;
  const uint8_t *flavor;
  const double *t_dag;
  const double *t_ann;
  const int32_t *rem_idx;
};

// Workspace layout (device), sized for n walkers and n_kept kept states.
struct Workspace {
  int32_t *counters;   // [4]: 0 = number of alive items, 1 = next unit to claim, 2-3 spare
  int4 *desc;          // [n] per-walker edit descriptor {kind, p1, p2, K_new}
  int32_t *wstatus;    // [n] per-walker status from validation
  int32_t *worklist;   // [n * n_kept] alive items (walker * n_kept + kept)
  int8_t *item_sign;   // [n * n_kept]
  double *item_log;    // [n * n_kept] log|contribution| (relative to exp(-beta E0))
  int32_t *item_status;// [n * n_kept]
  int32_t *pair_flag;  // [n * n_kept] halves of the item published so far
  double *half_log;    // [2 * n * n_kept] log-weight of each half
  int32_t *half_info;  // [2 * n * n_kept] block | status << 24, or -1 if the half vanished
  void *half_vec;      // [2 * n * n_kept][d_max] final vector of each half (FP32 or FP64)
  // measurement at tau = beta/2 only (nullptr otherwise)
  double *item_obs;    // [n * n_kept][nf + n_orb + 1] <O> of each item: n_f, n_{a up} n_{a dn}, S^2
  int32_t *item_blk;   // [n * n_kept] block of the item at tau = beta/2
};

// Partial-state cache of the sweep: for every (walker, kept state) item of the
// current configuration (K operators), forward states at slot i = position i (the
// state right after operator i-1, at its time; position 0 is the kept state at
// tau = 0 and is not stored) and backward states at reverse slot K - e (the bra
// including operators e .. K-1, at the time of operator e; reverse slot 0 is the kept
// state at beta). Entries are normalised vectors with a log-weight and their block
// (-1: the state is zero). f[item] and gr[item] bound the valid forward slots
// [0, f] and reverse slots [0, gr]. The scratch arrays hold one step's tentative
// states (inside the edited window) until the accept decision.
struct CacheView {
  int P;              // positions per direction; walkers with more operators are not cached
  int dv;             // vector stride (rows) of an entry
  void *fvec, *bvec;  // [n_items][P + 1][dv] elements of the model's precision
  double2 *flog, *blog;  // log-weight = x - log(y) (y: mantissa of the normalisation product)
  int32_t *fblk, *bblk;
  void *sfvec, *sbvec;
  double2 *sflog, *sblog;
  int32_t *sfblk, *sbblk;
  int32_t *f, *gr;    // [n_items]
  int4 *plan;         // [n_items] this step: {y, x_new, m, flags}: bit 0 store states, bit 1 unit run,
                      // bit 2 cache build (both units cover the whole sequence), bit 3 the halves
                      // meet at beta/2 (measurement)
};

// Edited window of a move in the new sequence: positions [lo, hi_new) differ from
// the old sequence, positions < lo equal it, positions >= hi_new are old ones shifted
// by K_new - K_old.
__host__ __device__ inline void edit_window(int4 d, int &lo, int &hi_new) {
  lo = d.y;
  hi_new = d.x == 0 ? d.z + 2 : d.z - 1;
}

// n_obs_item = 0: trace and ratio calls; nf + n_orb + 1: measurement calls.
size_t workspace_bytes(int n_walkers, int n_kept, int d_max, int n_obs_item = 0);
Workspace carve_workspace(void *base, int n_walkers, int n_kept, int d_max, int n_obs_item = 0);

// Compiled variants of the Krylov items kernel: (row capacity DMAX, Krylov cap
// PMAX, lanes per item G).
#define KT_FOR_VARIANTS(X) \
  X(10, 10, 4) X(10, 10, 8) X(10, 10, 16) X(10, 10, 32) X(36, 24, 8) X(36, 24, 16) X(36, 24, 32) X(128, 40, 32)

// Kernel variants compiled for sm_103a: rows per block (DMAX) and Krylov cap (PMAX).
int kernel_dmax_for(int d_max);    // 0 if no variant fits
int kernel_pmax_for(int kernel_dmax);
int kernel_groups_for(int kernel_dmax, int *out, int cap);  // lane-group sizes compiled for this row capacity
int default_group_for(int kernel_dmax, int precision);

// Optional CUDA events recorded at the 5 stage boundaries of one pipeline call.
struct StageEvents {
  void *ev[5];  // cudaEvent_t
};

// Launch the full pipeline (validation/edit, pruning, Krylov items, reduction).
// moves == nullptr: plain traces. obs != nullptr (plain traces only, with the
// measurement regions of the workspace carved): also the local observables at
// tau = beta/2, [n][KT_MEASURE_NOBS(n_orb)]. Returns a CUDA error code (0 = success).
int launch_pipeline(const DevModel &m, int precision, int kernel_dmax, int group_lanes, const SeqView &seq,
                    const MoveView *moves,
                    const int8_t *cur_sign, const double *cur_logabs, int8_t *sign, double *logv, int32_t *status,
                    kt_stats *stats, const Workspace &ws, void *stream, const StageEvents *timing,
                    double *obs = nullptr);

// The trace-ratio pipeline of the sweep's cached mode: validation and edit, the
// per-item plan (pruning, the stretch between valid cached states), the cached
// Krylov items and the reduction. The items use the default lane-group size.
int launch_cached_pipeline(const DevModel &m, int precision, int kernel_dmax, const SeqView &seq,
                           const MoveView &moves, const int8_t *cur_sign, const double *cur_logabs, int8_t *sign,
                           double *logv, int32_t *status, const Workspace &ws, const CacheView &cache, bool write,
                           kt_stats *stats, void *stream);
// After the accept decision of a step with stored states: accepted moves (accepted[w]
// nonzero) take their tentative window states into the cache, rejected ones extend the
// valid ranges (rstatus: the ratio statuses of the step). words = 32-bit words per vector.
int launch_cache_commit(const CacheView &C, int n, int nk, const int4 *desc, const int32_t *wstatus,
                        const int8_t *accepted, const int32_t *rstatus, int words, void *stream);
// Traces and observables at beta/2 of the current configurations (the kt_measure
// layout of the workspace and of obs) from the cache, extending it (plan flag 8).
int launch_cached_measure(const DevModel &m, int precision, int kernel_dmax, const SeqView &seq, int8_t *sign,
                          double *logv, int32_t *status, double *obs, const Workspace &ws, const CacheView &cache,
                          void *stream);
// Store every forward and backward state of the current configurations (plan flags
// bit 2: whole sequences, no overlap) and mark them valid.
int launch_cache_build(const DevModel &m, int precision, int kernel_dmax, const SeqView &seq, const Workspace &ws,
                       const CacheView &cache, void *stream);

// Tensor-core GEMM C = A . B^T (BF16 in, FP32 out) and the surrogate network's
// forward pass (kt_mlp.cu), for the delayed-acceptance sweep.
int gemm_bf16(const void *A, int lda, const void *B, int ldb, float *C, int ldc, int M, int N, int K, int *err,
              void *st_, int splits = 1);
// Number of K slices gemm_bf16 uses for `splits` (each slice a multiple of 64 columns); with
// more than one, slice z writes its partial product to C + z * M * ldc.
int gemm_splits(int K, int splits);
int mlp_forward(kt_mlp *n, const void *X, int B, float *y, bool train, void *st_);
int mlp_inputs(const kt_mlp *n);
int mlp_max_batch(const kt_mlp *n);

// Launch parameters of a model, for entry points that live outside kt_model.cpp.
struct ModelView {
  const DevModel *dev;
  int precision, kernel_dmax, group_lanes;
  bool host_only;
  int device;  // CUDA device holding the model's tables
};
ModelView model_view(const kt_model *m);
// True when the current CUDA device is the one that holds the model's tables.
bool on_model_device(const ModelView &v);

}  // namespace kt
