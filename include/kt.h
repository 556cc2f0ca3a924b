/*
 * kt.h - C ABI of the GB300 Krylov local-trace engine for the hybridization
 * expansion (Laeuchli & Werner, "Krylov-implementation of the hybridization
 * expansion impurity solver and application to 5-orbital models").
 *
 * The engine evaluates, for a batch of Monte Carlo walkers, the local trace of
 * Eq. (weight_strong) truncated to the low-energy eigenstates of H_loc
 * (Sec. II, truncation type (i); Sec. III, steps 3-8):
 *
 *   T = sum_{n kept} <n| e^{-(beta-tau_K) H} O_K e^{-(tau_K - tau_{K-1}) H} ... O_1 e^{-tau_1 H} |n>
 *
 * with H = H_loc of Eq. (H_loc) (Sec. IV.A), O_k = c_f or c_f^+, every inner
 * interval propagated by a Lanczos approximation of exp(-dtau H) v (Sec. III,
 * step 5), and the trace ratio of a local update (insertion or removal of a
 * c^+/c pair, Sec. II) against the walker's current trace.
 *
 * Conventions fixed by this library (the paper leaves them open):
 *   - flavor f = 2a + s for orbital a in [0, n_orb) and spin s (0 up, 1 down);
 *     bit f of a Fock bitstring is the occupation n_f;
 *   - c_f and c_f^+ carry the Jordan-Wigner sign (-1)^popcount(x & ((1<<f)-1));
 *   - a sequence is sorted by time (non-decreasing), tau in [0, beta), and its
 *     operators act in increasing array index; at equal times array order
 *     decides and a zero-length interval is the identity;
 *   - the spin-flip and pair-hopping terms of Eq. (H_loc) are read with each
 *     ordered orbital pair a != b counted once (this keeps H_loc SU(2)
 *     invariant at U' = U - 2J);
 *   - results are (sign, log|T|); internally every propagation is shifted by
 *     the global ground energy E0 so that log|T| = log|T~| - beta E0 with
 *     |T~| <= N_tr.
 *
 * Memory and streams: every batch, move and output pointer below is a DEVICE
 * pointer owned by the caller. The model's tables are device memory owned by
 * the model (allocated by kt_model_create on the current device, freed by
 * kt_model_destroy). Per-call scratch is a caller-owned device workspace of
 * at least kt_workspace_size() bytes. Trace calls enqueue kernels on the given
 * cudaStream_t (NULL = legacy default stream) and return without
 * synchronising; their return value reports only argument and launch errors,
 * while per-walker outcomes land in the device array `status`.
 * No call throws; no call falls back to the CPU.
 */
#ifndef KT_H
#define KT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KT_OK = 0,
  KT_EINVAL = 1,       /* malformed argument, sequence or move */
  KT_ENOMEM = 2,       /* host or device allocation failed, or workspace too small */
  KT_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  KT_ENOCONV = 4,      /* a Krylov propagation reached its dimension cap unconverged */
  KT_ENUMERIC = 5,     /* NaN or Inf met in a log-weight */
  KT_EZEROWEIGHT = 6,  /* trace ratio requested against a current weight of 0 */
  KT_ETIMEOUT = 7,     /* a bounded device-side wait gave up */
  KT_EUNSUPPORTED = 8  /* model outside what the compiled kernels handle */
} kt_status;

/* precision */
#define KT_FP64 0         /* FP64 Krylov vectors and scalars (plain FP64 path) */
#define KT_FP32_KRYLOV 1  /* FP32 SpMV and Krylov vectors; FP64-accurate (double-float)
                             Lanczos scalars, norms and Ritz values; FP64 log-weights */

/* flags */
#define KT_DENSITY_ONLY 1u   /* drop spin-flip and pair-hopping (density-density H_loc) */
#define KT_SECTOR_BLOCKS 2u  /* propagate in whole (n_up, n_dn) sectors instead of the
                                finer blocks that also fix the set of singly occupied orbitals */
#define KT_FP32_TRIDIAG64 4u /* FP32 path only: the final exponential of the small tridiagonal T_p of
                                every propagation to FP64 accuracy, rounded to FP32 once, instead
                                of FP32 Ritz vectors with double-float Ritz values. FP32 Ritz
                                vectors are off by about u ||T_p|| / gap, and these errors neither
                                average out nor cancel between the halves of a sequence; with this
                                flag the Krylov vectors carry the only FP32 rounding. p = 2: the
                                closed form in FP64. p >= 3: the FP32 Ritz vectors refined by one
                                step of Ogita and Aishima's iteration (Japan J. Indust. Appl. Math.
                                35, 2018) in double-float, Ritz values recomputed from them and FP64
                                weights; a T_p with Ritz values too close to refine takes a full
                                FP64 QL. Exact stops: double-float sums over the block
                                eigendecomposition. Slower than the default (the FP64 pipe of
                                GB300 is 1/64 of the FP32 one) */
#define KT_HOST_ONLY 256u    /* build and check the model on the host only: no device upload;
                                trace calls on such a model return KT_EINVAL */

/* Model parameters of Eq. (H_loc) (Sec. IV.A) and of the trace truncation
 * (Sec. III, setup steps 1-2). */
typedef struct {
  int32_t n_orb;        /* orbitals, 1..7 (2*n_orb flavors, 4^n_orb Fock states) */
  double U;             /* intra-orbital repulsion */
  double J;             /* Hund coupling (spin-flip and pair hopping carry -J) */
  double Up;            /* inter-orbital U'; NaN selects U - 2J */
  double mu;            /* chemical potential, enters as -(mu + delta_a) n_{a,s} */
  const double *delta;  /* HOST pointer, [n_orb] crystal-field shifts, or NULL for zeros */
  double beta;          /* inverse temperature */
  double trunc_eps;     /* keep whole multiplets with exp(-beta (E - E0)) >= trunc_eps;
                           <= 0 keeps every eigenstate (untruncated trace) */
  double deg_tol;       /* eigenvalues within deg_tol * max(1, |E|) form one multiplet */
  double krylov_tol;    /* relative a-posteriori error target per propagation */
  int32_t krylov_pmax;  /* cap on the Krylov dimension (<= 0: the compiled maximum) */
  int32_t precision;    /* KT_FP64 or KT_FP32_KRYLOV */
  uint32_t flags;       /* KT_DENSITY_ONLY | KT_SECTOR_BLOCKS | KT_FP32_TRIDIAG64 */
} kt_model_params;

typedef struct kt_model kt_model;

typedef struct {
  int32_t n_orb, n_flavors, n_states;
  int32_t n_blocks;     /* invariant blocks of H_loc used for propagation */
  int32_t d_max;        /* largest block dimension */
  int32_t nnz_max;      /* most off-diagonal entries in one row */
  int32_t n_kept;       /* N_tr: kept eigenstates in the outer trace */
  int32_t precision;
  int32_t krylov_pmax;  /* effective Krylov cap */
  int32_t kernel_dmax;  /* row capacity of the kernel variant chosen for this model */
  int32_t group_lanes;  /* lanes that cooperate on one (walker, kept state) item (1..32) */
  double E0;            /* global ground energy of H_loc */
  double e_kept_max;    /* highest kept energy minus E0 */
  size_t device_bytes;  /* device memory held by the model's tables */
} kt_model_info;

#define KT_P_HIST 32

/* Per-call counters, accumulated on the device with atomics into a caller-owned
 * DEVICE struct (zero it before the call; pass NULL to skip counting). */
typedef struct {
  unsigned long long walkers;        /* walkers evaluated */
  unsigned long long items;          /* (walker, kept state) pairs */
  unsigned long long items_alive;    /* pairs that survived structural pruning */
  unsigned long long items_vanished; /* alive pairs whose vector became exactly zero */
  unsigned long long ops_applied;    /* c / c^+ applications */
  unsigned long long intervals;      /* Krylov propagations */
  unsigned long long krylov_iters;   /* sum of Krylov dimensions p */
  unsigned long long p_max;          /* largest p seen */
  unsigned long long noconv;         /* propagations that stopped at the cap unconverged */
  unsigned long long flops_vec;      /* algorithmic vector flops (SpMV, dots, axpys, assembly) */
  unsigned long long flops_tri;      /* FP64 flops of the small tridiagonal exponentials */
  unsigned long long bytes_apply;    /* bytes moved by c / c^+ gathers */
  unsigned long long flops_alg;      /* algorithmic Krylov flops: sum over intervals of
                                        p (2 nnz(H_b) + 11 d_b) + 2 p d_b (nnz with the diagonal;
                                        the three-term update, dots, norm and scaling; Q_p y) */
  unsigned long long flops_reorth;   /* FP32 path: reorthogonalisation, sum of 2 p (p - 1) d_b */
  unsigned long long p_hist[KT_P_HIST]; /* propagations by stopping Krylov dimension p:
                                            bin p for p < KT_P_HIST - 1, the last bin p >= KT_P_HIST - 1 */
} kt_stats;

/* CSR batch of operator sequences (Eq. (weight_strong): the time-ordered
 * product of hybridization events). All DEVICE pointers. */
typedef struct {
  int32_t n;               /* walkers */
  const int32_t *offsets;  /* [n+1], offsets[0] = 0; ops of walker i: offsets[i] .. offsets[i+1]-1 */
  const double *tau;       /* [offsets[n]] times in [0, beta), non-decreasing per walker */
  const uint8_t *flavor;   /* [offsets[n]] flavor f in [0, 2 n_orb) */
  const uint8_t *dagger;   /* [offsets[n]] 1 = c_f^+, 0 = c_f */
} kt_seq_batch;

/* One proposed local update per walker (Sec. II: insertion or removal of a
 * pair of c^+ and c). All DEVICE pointers, [n] each. */
typedef struct {
  const uint8_t *kind;     /* 0 insert, 1 remove */
  const uint8_t *flavor;   /* flavor of the pair */
  const double *t_dag;     /* insert: time of the new c^+ */
  const double *t_ann;     /* insert: time of the new c; each new operator goes after all
                              existing operators at an equal time; if t_dag == t_ann the c
                              is placed first */
  const int32_t *rem_idx;  /* remove: index (inside the walker's sequence) of an operator of
                              this flavor to drop; the next operator of the same flavor after
                              it, cyclically, must be of the other type (the c closing a
                              segment, or the c^+ closing an anti-segment) and is dropped
                              with it */
} kt_move_batch;

/* Human-readable name of a status code (static storage). */
const char *kt_status_string(kt_status s);

/* Sec. III, setup steps 1-2: enumerate the Fock space, build the blocks of
 * H_loc (Eq. (H_loc)) and the c / c^+ maps with Jordan-Wigner signs,
 * diagonalise every block, pick the kept multiplets, and upload the tables to
 * the current CUDA device. *out is owned by the caller and released with
 * kt_model_destroy. Errors: KT_EINVAL (parameters), KT_ENOMEM, KT_ECUDA,
 * KT_EUNSUPPORTED (a block larger than every compiled kernel variant). */
kt_status kt_model_create(const kt_model_params *params, kt_model **out);

/* Sizes and energies of a model (host struct). */
kt_status kt_model_query(const kt_model *m, kt_model_info *out);

/* Kept eigenstates (HOST arrays of length n_kept, any may be NULL): energy
 * E - E0, and the (n_up, n_dn) and singly-occupied-orbital mask of the block
 * that holds each one. */
kt_status kt_model_kept(const kt_model *m, double *e_minus_e0, int32_t *n_up, int32_t *n_dn,
                        int32_t *single_mask);

/* All eigenvalues of H_loc (HOST array of length n_states), ascending: the
 * spectrum of Sec. III setup step 1. */
kt_status kt_model_spectrum(const kt_model *m, double *energies);

/* Free the model and its device tables (no-op on NULL). Not stream-ordered:
 * call it after all work using the model has completed. */
void kt_model_destroy(kt_model *m);

/* Device workspace (bytes) that kt_trace / kt_trace_ratio need for n walkers. */
kt_status kt_workspace_size(const kt_model *m, int32_t n_walkers, size_t *bytes);

/* Sec. III steps 3-8 for every walker of the batch: the truncated local trace.
 * Outputs (DEVICE, [n] each): sign in {-1, 0, +1}; logabs = log|T| (-inf when
 * sign = 0); status = kt_status of that walker (KT_EINVAL for an unsorted
 * sequence, a flavor out of range or a time outside [0, beta); KT_ENOCONV if a
 * propagation stopped at the Krylov cap; KT_ENUMERIC for a NaN/Inf weight).
 * stats may be NULL. workspace: DEVICE, >= kt_workspace_size(m, batch->n).
 * stream: a cudaStream_t. Returns KT_EINVAL/KT_ENOMEM/KT_ECUDA on bad
 * arguments or launch failure, else KT_OK (asynchronous). */
kt_status kt_trace(kt_model *m, const kt_seq_batch *batch, int8_t *sign, double *logabs, int32_t *status,
                   kt_stats *stats, void *workspace, size_t workspace_bytes, void *stream);

/* Trace ratio of one local update per walker (Sec. II local updates; the
 * trace factor of the Metropolis ratio of Eq. (weight_strong)): the trace of
 * the edited sequence divided by the caller's current trace (cur_sign,
 * cur_logabs, DEVICE, [n]), as sign = sign_new * cur_sign and
 * logratio = log|T_new| - cur_logabs (-inf when the new trace is 0).
 * A walker with cur_sign == 0 gets status KT_EZEROWEIGHT, sign 0 and logratio
 * NaN; a malformed move gets KT_EINVAL. Other arguments as kt_trace. */
kt_status kt_trace_ratio(kt_model *m, const kt_seq_batch *cur, const int8_t *cur_sign, const double *cur_logabs,
                         const kt_move_batch *moves, int8_t *sign, double *logratio, int32_t *status,
                         kt_stats *stats, void *workspace, size_t workspace_bytes, void *stream);

/* Local observables at tau = beta/2 (Sec. III: with the trace truncated at
 * tau = 0 and beta, measure in the middle of the interval; the kept state is
 * propagated forward from tau = 0 and backward from beta, Sec. III step 3, and
 * the two meet at beta/2). For each walker and each diagonal operator O of the
 * occupation basis, <O> = Tr[... O(beta/2) ...] / Tr[...] with O inserted after
 * every operator with tau < beta/2 (S^2 is not diagonal: it is applied to one of the
 * two half vectors). Layout of obs (DEVICE, [n][KT_MEASURE_NOBS]):
 *   [0, 2 n_orb)              n_f, flavor f = 2a + s
 *   [2 n_orb, 3 n_orb)        n_{a up} n_{a dn} (double occupancy of orbital a)
 *   3 n_orb                   total spin S^2 (Sec. V: = S_z^2 + S_z + S- S+, whose
 *                             exchange terms stay inside each block)
 *   [3 n_orb + 1, +(n_orb+1)^2) projector on the (n_up, n_dn) sector, index
 *                             n_up * (n_orb + 1) + n_dn (a histogram summing to 1)
 * Walkers whose trace is 0 (sign 0) get NaN. sign, logabs, status as kt_trace.
 * The workspace must hold kt_measure_workspace_size(m, n) bytes. */
#define KT_MEASURE_NOBS(n_orb) (3 * (n_orb) + 1 + ((n_orb) + 1) * ((n_orb) + 1))
kt_status kt_measure_workspace_size(const kt_model *m, int32_t n_walkers, size_t *bytes);
kt_status kt_measure(kt_model *m, const kt_seq_batch *batch, int8_t *sign, double *logabs, double *obs,
                     int32_t *status, kt_stats *stats, void *workspace, size_t workspace_bytes, void *stream);

/* Allocation-free variant of kt_trace_ratio for callers that cannot allocate
 * device memory (for example code that may not call cudaMalloc after start-up,
 * or that is handed only its input and output buffers). The paper has no
 * counterpart: this is an interface convenience. Same arguments, results and
 * per-walker statuses as kt_trace_ratio, but no workspace: the scratch lives in
 * a fixed array of KT_STATIC_SCRATCH_BYTES inside the library's device image,
 * held on every GPU that loads the library until the process exits. Batches
 * whose scratch would exceed it (kt_workspace_size(m, n) > KT_STATIC_SCRATCH_BYTES,
 * about 6,700 walkers of the five-orbital model) are rejected with KT_ENOMEM
 * before any work.
 * The call allocates nothing. Its first call on each device looks up the
 * array's device address with that device current; make that first call
 * before any stream capture. All calls share the array: calls whose kernels
 * overlap on the GPU race, so serialise them. */
#define KT_STATIC_SCRATCH_BYTES (8u << 20)
kt_status kt_trace_ratio_static(kt_model *m, const kt_seq_batch *cur, const int8_t *cur_sign,
                                const double *cur_logabs, const kt_move_batch *moves, int8_t *sign,
                                double *logratio, int32_t *status, kt_stats *stats, void *stream);

/* ------------------------------------------------------------------------ */
/* Trace ratios from cached partial states (Sec. III step 3: the forward and */
/* backward propagation, kept between calls).                                */
/* ------------------------------------------------------------------------ */
/*
 * For fixed current configurations evaluated against many proposed updates,
 * kt_ratio_cache_build stores, for every walker and kept state, the normalised
 * forward state after each operator and the backward state from beta down to each
 * operator, with their log-weights. kt_trace_ratio_cached then propagates only the
 * window that an update edits: from the cached forward state before its first
 * changed operator to the cached backward state after its last one, split in the
 * middle. Results, per-walker statuses and tolerances are those of kt_trace_ratio
 * (the values differ by rounding only); the cache is only read. The batch passed to
 * kt_trace_ratio_cached must hold the configurations of the last build: the library
 * evaluates from scratch a walker whose length differs from the build, but cannot see
 * other changes. Walkers longer than max_ops operators, before or after their update,
 * are evaluated from scratch too.
 * Device memory: 4 * n_walkers * n_kept * (max_ops + 1) * (d_max * element size + 20)
 * bytes (the cache and the tentative states of kt_ratio_cache_propose) plus a kt_trace
 * workspace; errors KT_EINVAL (bad arguments, n != n_walkers),
 * KT_ENOMEM, KT_ECUDA. Calls are enqueued on the stream; build and ratio calls on one
 * cache must not overlap.
 */
typedef struct kt_ratio_cache kt_ratio_cache;
kt_status kt_ratio_cache_create(kt_model *m, int32_t n_walkers, int32_t max_ops, kt_ratio_cache **out);
/* DEVICE batch of n_walkers current configurations, layout and validation as kt_trace. */
kt_status kt_ratio_cache_build(kt_ratio_cache *c, const kt_seq_batch *cur, void *stream);
kt_status kt_trace_ratio_cached(kt_ratio_cache *c, const kt_seq_batch *cur, const int8_t *cur_sign,
                                const double *cur_logabs, const kt_move_batch *moves, int8_t *sign,
                                double *logratio, int32_t *status, kt_stats *stats, void *stream);
/* For external Markov chains on the cached configurations: kt_ratio_cache_propose gives
 * kt_trace_ratio_cached's results and also keeps the states inside each update's window
 * aside (the states outside it, valid for both configurations, extend the cache at
 * once). Then kt_ratio_cache_commit, with accepted (DEVICE int8 [n], nonzero = the
 * walker's update was accepted) and the status array of that propose call, makes the
 * cache describe the edited configuration of every accepted walker and the unchanged one
 * of the others. The caller edits its sequences the same way before the next call: an
 * insertion places c^+ at t_dag and c at t_ann, each after the operators at equal times
 * (if t_dag == t_ann the c goes first); a removal drops the operator at rem_idx and the
 * next operator of its flavor, cyclically. One propose, then one commit, per step. */
kt_status kt_ratio_cache_propose(kt_ratio_cache *c, const kt_seq_batch *cur, const int8_t *cur_sign,
                                 const double *cur_logabs, const kt_move_batch *moves, int8_t *sign,
                                 double *logratio, int32_t *status, kt_stats *stats, void *stream);
kt_status kt_ratio_cache_commit(kt_ratio_cache *c, const int8_t *accepted, const int32_t *status, void *stream);
/* No-op on NULL. Not stream-ordered: call it after the cache's work has completed. */
void kt_ratio_cache_destroy(kt_ratio_cache *c);

/* ------------------------------------------------------------------------ */
/* Batched CT-HYB Markov chains (Sec. II): Metropolis insertion and removal  */
/* of c^+/c pairs with the weight of Eq. (weight_strong) for a hybridization */
/* that is diagonal in the flavors.                                          */
/* ------------------------------------------------------------------------ */
/*
 * Weight of a configuration: w = s_P * T * prod_f det G_f, with T the truncated
 * local trace of this library, G_f[i][j] = Fh_f(tau'_i - tau_j) over the creator
 * times tau'_i and annihilator times tau_j of flavor f, Fh_f(x) = F_f(x) for
 * x >= 0 and -F_f(x + beta) for x < 0, F_f(tau) = -Delta_f(tau) >= 0 the bath
 * correlator (linear interpolation of the caller's table), and s_P the sign of
 * the permutation taking the bath operators, written flavor by flavor as
 * a(tau'_1) a^+(tau_1) a(tau'_2) a^+(tau_2) ..., into descending time order.
 *
 * Each step proposes one move per walker from six caller-supplied uniforms
 * u[0..5] in [0, 1) (DEVICE, [n_steps][n_walkers][6]):
 *   u0 < 1/2 insert, else remove; flavor f = floor(u1 * n_flavors);
 *   insert: t1 = u2 beta; with no f operators a coin u4 < 1/2 picks a segment
 *     (c^+ at t1, c at t2) or an anti-segment (c at t1, c^+ at t2) and l = beta;
 *     otherwise the next f operator after t1 (cyclically) decides (a c^+ next: a
 *     segment; a c next: an anti-segment) and l is the distance to it;
 *     t2 = t1 + u3 l (mod beta); proposal factor beta^2 (k_f = 0) or
 *     beta l / (2 (k_f + 1));
 *   remove: the floor(u2 * 2 k_f)-th f operator in time order and the next f
 *     operator after it (cyclically); proposal factor 1 / beta^2 (k_f = 1) or
 *     2 k_f / (beta l'), l' the distance from the first removed operator to the
 *     f operator that follows the pair;
 *   accept when log(u5) < log|w_new / w_old| + log(proposal factor).
 * Null moves (nothing changes): removal from an empty flavor, insertion past
 * k_cap pairs, t1 >= beta after rounding, t2 == t1.
 * The trace ratio is this library's pipeline (the model's precision); the
 * determinant ratio and the inverse matrices use O(k^2) updates in FP64 (the
 * bordered-matrix inverse for an insertion, the Schur complement for a removal).
 * Measurements, every meas_every steps, weighted by the sign of w:
 *   G_f(tau): sum over pairs of M_ji dh(tau, tau_j - tau'_i), M = G_f^{-1},
 *     dh = +1 in the bin of x > 0, -1 in the bin of x + beta for x < 0, binned on
 *     n_bins bins of [0, beta); G_f(tau_b) = n_bins / beta^2 * g_tau[b] / sign_sum;
 *   the expansion order of every flavor;
 *   optionally the observables of kt_measure at beta/2.
 * Every chain starts from the empty configuration.
 *
 * Partial-state cache (cache_ops > 0; Sec. III's forward and backward propagation,
 * kept between steps). For every walker and kept state the sweep stores, for its
 * current configuration of K operators, the normalised forward states after each
 * operator (times their log-weights) and the backward states from beta down to each
 * operator, each over a valid prefix and suffix of positions. A proposal edits the
 * window between its first and last changed operator; its trace ratio propagates
 * only from the last valid forward state before the window to the first valid
 * backward state after it (split in the middle, forward and backward concurrently),
 * writing the states it passes: positions outside the window extend the valid
 * prefix or suffix at once, positions inside it are kept aside and committed only if
 * the move is accepted. The observables at beta/2 (measure_obs) start from the cached
 * states nearest beta/2 and extend the cache. The Markov chain and its uniforms are
 * unchanged; the ratios and observables differ from the full evaluation by rounding only. Memory: 4 * n_walkers * n_kept *
 * (cache_ops + 1) * (d_max * element size + 20) bytes.
 */
typedef struct kt_sweep kt_sweep;

typedef struct {
  int32_t n_walkers;    /* independent chains */
  int32_t k_cap;        /* pairs per flavor and walker, 1..128 */
  int32_t n_tau;        /* intervals of the bath table (>= 1) */
  const double *hyb;    /* HOST [n_flavors][n_tau + 1]: F_f(i beta / n_tau) */
  int32_t n_bins;       /* G(tau) bins (>= 1) */
  int32_t measure_obs;  /* nonzero: accumulate the kt_measure observables at each measurement */
  int32_t cache_ops;    /* 0: every trace ratio is evaluated from scratch, split at the middle
                           operator. > 0: partial-state cache (see below) for walkers of up to
                           cache_ops operators (longer ones fall back to the full evaluation) */
} kt_sweep_params;

/* Caller-owned DEVICE destinations for kt_sweep_get_state; NULL entries are skipped. */
typedef struct {
  int32_t *lens;          /* [n_walkers] operators per walker */
  double *tau;            /* [n_walkers][capacity] capacity = 2 * n_flavors * k_cap */
  uint8_t *flavor;        /* [n_walkers][capacity] */
  uint8_t *dagger;        /* [n_walkers][capacity] */
  int8_t *sign;           /* [n_walkers] sign of w */
  int8_t *trace_sign;     /* [n_walkers] */
  double *trace_logabs;   /* [n_walkers] log|T| */
  double *det_logabs;     /* [n_walkers] sum over flavors of log|det G_f| (updated incrementally) */
  int32_t *order;         /* [n_walkers][n_flavors] pairs per flavor */
} kt_sweep_state;

/* Caller-owned DEVICE destinations for kt_sweep_get_accumulators; NULL entries are skipped. */
typedef struct {
  double *g_tau;          /* [n_walkers][n_flavors][n_bins] */
  double *sign_sum;       /* [n_walkers] */
  double *order_sum;      /* [n_walkers][n_flavors] sign-weighted */
  double *obs_sum;        /* [n_walkers][KT_MEASURE_NOBS(n_orb)] sign-weighted */
} kt_sweep_accum;

/* Counters of kt_sweep_counters (HOST [10]): 0 insertions proposed, 1 accepted,
 * 2 removals proposed, 3 accepted, 4 null moves, 5 insertions refused at k_cap,
 * 6 proposals rejected because the trace pipeline reported an error, 7 measurements,
 * 8 proposals rejected at stage 1 of delayed acceptance, 9 trace ratios evaluated. */
#define KT_SWEEP_NCOUNTERS 10

/* Allocate the chains of a model (device state on the current device; the model
 * must outlive the sweep) and set every walker to the empty configuration.
 * Synchronises. Errors: KT_EINVAL, KT_ENOMEM, KT_ECUDA. */
kt_status kt_sweep_create(kt_model *m, const kt_sweep_params *p, kt_sweep **out);
/* Device bytes that kt_sweep_create(m, p) allocates, computed on the host from the same
 * layouts, without touching the device. The total covers the chains (configurations,
 * inverse bath matrices, about n_walkers * n_flavors * k_cap * (8 k_cap + 36) bytes),
 * the partial-state cache when p->cache_ops > 0, and the trace-pipeline workspace. With
 * tries > 0 it adds the proposal slots that kt_sweep_run_da_multi with that many tries
 * allocates on its first call. p->hyb is not read; m may be a KT_HOST_ONLY model. Callers
 * size k_cap, cache_ops and n_walkers from the device's free memory with it. KT_EINVAL for
 * parameters kt_sweep_create would reject or tries outside 0 .. KT_DA_MAX_TRIES. */
kt_status kt_sweep_memory_bytes(const kt_model *m, const kt_sweep_params *p, int32_t tries, size_t *bytes);
/* n_steps Metropolis steps of every walker, measuring after every meas_every-th
 * step (0: never). Enqueued on the stream; returns launch errors only. */
kt_status kt_sweep_run(kt_sweep *s, int32_t n_steps, const double *uniforms, int32_t meas_every, void *stream);
/* Replace every walker's configuration (a restart from kt_sweep_get_state, or a
 * chosen starting point). HOST batch with n == n_walkers, same layout rules as
 * kt_trace. Each sequence must hold, for every flavor, as many c^+ as c (at most
 * k_cap pairs) alternating in time, and have a nonzero weight. The inverse bath
 * matrices and log-determinants are computed from scratch in FP64 on the host
 * (Gauss-Jordan elimination with partial pivoting), the traces on the device.
 * Synchronises. On KT_EINVAL (a malformed sequence, too many pairs, a singular
 * bath matrix or a zero trace) every walker is back at the empty configuration. */
kt_status kt_sweep_set_configs(kt_sweep *s, const kt_seq_batch *host_batch);
/* Count the trace pipeline's work of the following steps into a caller-owned DEVICE
 * kt_stats (as kt_trace_ratio does; zero it first). NULL stops counting. */
kt_status kt_sweep_set_stats(kt_sweep *s, kt_stats *stats);
kt_status kt_sweep_get_state(kt_sweep *s, const kt_sweep_state *dst, void *stream);
kt_status kt_sweep_get_accumulators(kt_sweep *s, const kt_sweep_accum *dst, void *stream);
/* Drift guard: recompute, for every walker, everything the chain tracks incrementally, from
 * its current configuration and from scratch, and replace the tracked values: the inverse
 * bath matrices M = G_f^{-1} and log|det G_f| in FP64 on the device (Gauss-Jordan elimination
 * with partial pivoting, one warp per walker and flavor), the sign of the bath permutation,
 * and the local trace (this library's pipeline at the model's precision). The determinant
 * fast updates of Sec. II and the products of accepted trace ratios accumulate rounding over
 * a long chain; calling this every few hundred steps bounds that drift. A walker whose fresh
 * evaluation fails (a singular G_f, a trace error) keeps its tracked values. Enqueued on the
 * stream; with max_dev (HOST [4], or NULL) it synchronises the stream and writes the largest
 * |tracked - fresh| of log|T| and of sum_f log|det G_f| over the walkers, the number of walkers
 * whose tracked sign of w or of T differed, and the number left unchanged. */
kt_status kt_sweep_refresh(kt_sweep *s, double *max_dev, void *stream);
/* Synchronises the device and copies the counters to out[KT_SWEEP_NCOUNTERS]. */
kt_status kt_sweep_counters(kt_sweep *s, unsigned long long *out);
/* Zero the accumulators and counters (the configurations are kept). */
kt_status kt_sweep_reset_accumulators(kt_sweep *s, void *stream);
void kt_sweep_destroy(kt_sweep *s);

/* ------------------------------------------------------------------------ */
/* Tensor-core GEMM (tcgen05, BF16 operands, FP32 accumulator in TMEM), the  */
/* building block of the learned delayed-acceptance filter.                  */
/* ------------------------------------------------------------------------ */
/* C[M][N] = A[M][K] . B[N][K]^T. A, B: DEVICE BF16, row-major with leading
 * dimensions lda, ldb (elements, multiples of 8, >= K), 16-byte aligned; C:
 * DEVICE FP32 row-major, ldc >= N. N and K multiples of 16 (N >= 16, K >= 16;
 * pad with zeros), any M >= 1. *err (DEVICE int32) is set to 1 if a bounded
 * wait of the kernel on the tensor core timed out (the tile is then not
 * written); the caller zeroes it. Asynchronous on the stream. */
kt_status kt_gemm_bf16(const void *A, int32_t lda, const void *B, int32_t ldb, float *C, int32_t ldc, int32_t M,
                       int32_t N, int32_t K, int32_t *err, void *stream);

/* ------------------------------------------------------------------------ */
/* Learned delayed acceptance: a surrogate network predicts log|T_new/T_old| */
/* of a proposed move; stage 1 of a two-stage Metropolis test (Christen &    */
/* Fox) uses it, and only moves that pass stage 1 get their true trace.      */
/* ------------------------------------------------------------------------ */
/*
 * Network: y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 with 256 hidden units,
 * input size n_in (a multiple of 16). BF16 operands on the tensor cores
 * (kt_gemm_bf16), FP32 accumulation; FP32 master weights, biases, output layer
 * and Adam state. Parameters are packed FP32 in the order W1 [256][n_in],
 * b1 [256], W2 [256][256], b2 [256], w3 [256], b3 [1].
 * Training minimises the mean squared error (1/B) sum (y - t)^2 with Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 */
typedef struct kt_mlp kt_mlp;
#define KT_MLP_HIDDEN 256
/* max_batch: largest batch of kt_mlp_forward / kt_mlp_backward (multiple of 16). */
kt_status kt_mlp_create(int32_t n_in, int32_t max_batch, kt_mlp **out);
kt_status kt_mlp_num_params(const kt_mlp *n, int64_t *count);
/* HOST packed FP32 parameters in and out (set also resets the Adam state); synchronous. */
kt_status kt_mlp_set_params(kt_mlp *n, const float *host_params);
kt_status kt_mlp_get_params(kt_mlp *n, float *host_params_out);
/* y[B] (DEVICE FP32) for inputs X (DEVICE BF16 [B][n_in], 16-byte aligned), B <= max_batch. */
kt_status kt_mlp_forward(kt_mlp *n, const void *X, int32_t B, float *y, void *stream);
/* Forward and backward pass on a batch (B a multiple of 16) with targets t (DEVICE FP32 [B]);
 * keeps the gradients in the object and writes the loss to *loss (DEVICE FP32, may be NULL). */
kt_status kt_mlp_backward(kt_mlp *n, const void *X, const float *t, int32_t B, float *loss, void *stream);
/* HOST copy of the packed gradients of the last kt_mlp_backward; synchronous. */
kt_status kt_mlp_get_grads(kt_mlp *n, float *host_grads_out);
/* The intermediate values of the last kt_mlp_backward (batch of B rows; KT_EINVAL if B
 * differs), copied to HOST arrays (any may be NULL; synchronous), so that every stage of the
 * gradient can be checked on its own inputs:
 *   z1  [B][256] FP32         X W1^T, before the bias;
 *   h1  [B][256] BF16 bits    relu(z1 + b1) rounded to nearest even;
 *   z2  [B][256] FP32         h1 W2^T, before the bias;
 *   dy  [B]      FP32         2 (y - t) / B;
 *   dz2 [B][256] BF16 bits    dy w3 where z2 + b2 > 0, else 0, rounded;
 *   dh1 [B][256] FP32         dz2 W2 (W2 in BF16);
 *   dz1 [256][B] BF16 bits    dh1 where z1 + b1 > 0, else 0, rounded (transposed layout). */
kt_status kt_mlp_get_tape(kt_mlp *n, int32_t B, float *z1, uint16_t *h1, float *z2, float *dy, uint16_t *dz2,
                          float *dh1, uint16_t *dz1);
/* One Adam step with the stored gradients. */
kt_status kt_mlp_adam(kt_mlp *n, float lr, void *stream);
/* Synchronises; *out = 1 if a tensor-core wait of any call timed out so far. */
kt_status kt_mlp_error(kt_mlp *n, int32_t *out);
void kt_mlp_destroy(kt_mlp *n);

/* Feature vector of a proposal (the surrogate's input; n_in = 35 n_flavors + 3 rounded
 * up to a multiple of 16). It describes the base (the configuration without the move's
 * pair: the current one for an insertion, the current one minus the pair for a
 * removal) and the pair, so that a move and its reverse share it:
 *   x[f] = k_f / 8 (pairs of flavor f in the base);
 *   x[nf + 32 f + b] += 1/4 for every segment of f in the base (a c^+ to the next c of
 *     f, cyclically) of length l with b = min(floor(32 l / beta), 31);
 *   x[33 nf] = 0; x[33 nf + 1 + f_move] = 1;
 *   x[34 nf + 1] = ((t_second - t_first) mod beta) / beta (t_first: t1 of an insertion,
 *     the chosen operator of a removal; t_second its partner);
 *   x[34 nf + 2] = +1 if the first operator is a c^+, else -1;
 *   x[34 nf + 3 + g] = fraction of the pair's interval (first operator to partner,
 *     cyclically) during which flavor g is occupied in the base; zero padding.
 * The network's output y predicts the log trace ratio of inserting the pair into the
 * base; the prediction for the move is y for an insertion and -y for a removal. */
kt_status kt_sweep_feature_size(const kt_sweep *s, int32_t *n_in);
/* n_steps plain Metropolis steps (uniforms as kt_sweep_run) that also record, for
 * every proposal whose trace ratio was evaluated and is nonzero, its features
 * (DEVICE BF16 [capacity][n_in]) and the insertion log trace ratio (log|T_new / T_old|
 * for an insertion, its negative for a removal; DEVICE FP32 [capacity]) at
 * slot atomicAdd(count, 1) while the slot is below capacity (*count, DEVICE int32,
 * keeps counting past it). */
kt_status kt_sweep_collect(kt_sweep *s, int32_t n_steps, const double *uniforms, void *features, float *targets,
                           int32_t *count, int32_t capacity, void *stream);
/* Attach a trained network (n_in must match, max_batch >= n_walkers) or detach (NULL). */
kt_status kt_sweep_set_surrogate(kt_sweep *s, kt_mlp *net);
/* Steps with delayed acceptance: uniforms DEVICE [n_steps][n_walkers][7]; u[0..5] as
 * kt_sweep_run, u6 decides stage 1: accept when log(u6) < r + log|det ratio| +
 * log(proposal factor) with r the signed prediction (+y insertion, -y removal); stage 2
 * accepts when log(u5) < log|T_new / T_old| - r. Because r is antisymmetric, this is
 * the exact two-stage rule of Christen and Fox. Only stage-1 survivors reach the trace
 * pipeline.
 * Counters 8 (stage-1 rejections) and 9 (trace ratios evaluated) count them. */
kt_status kt_sweep_run_da(kt_sweep *s, int32_t n_steps, const double *uniforms, int32_t meas_every, void *stream);

/* Multi-try delayed acceptance (the two-stage rule of kt_sweep_run_da, Christen & Fox).
 * A proposal rejected at stage 1 is a Metropolis step that leaves the configuration as it
 * is, so the next proposal starts from the same configuration. Each call step therefore
 * draws up to `tries` proposals per walker from its current configuration (uniforms DEVICE
 * [n_steps][n_walkers][tries][7], each try laid out as kt_sweep_run_da's seven), scores all
 * of them with one surrogate inference, and takes the first that passes stage 1 through the
 * trace pipeline and stage 2. The tries before it are stage-1 rejections (or null moves);
 * the tries after it are not taken. A call step is thus 1 to `tries` Metropolis steps of
 * the walker, every one judged by the exact two-stage rule.
 *
 * Measurement: because the number of Metropolis steps in a call step depends on the
 * configuration, a measurement per call step would weight configurations by the inverse of
 * their expected number of tries. Every meas_every-th call step therefore measures the
 * configuration the walker starts it in (after stage 1, before stage 2) with the weight n,
 * the number of tries the walker takes in that call step: the accumulators of
 * kt_sweep_get_accumulators hold sums of n * sign * O, and sign_sum the sum of n * sign,
 * whose ratio estimates <O> without that bias. With tries == 1, n == 1.
 *
 * Counters: 0/2 count the tries taken (proposals), 8 the stage-1 rejections among them.
 * The surrogate (kt_sweep_set_surrogate) must accept batches of tries * n_walkers rows
 * (KT_EINVAL otherwise); 1 <= tries <= KT_DA_MAX_TRIES. The first call with a larger
 * `tries` than before allocates the proposal slots (about tries * n_walkers *
 * (16 k_cap + 2 n_in + 120) bytes, plus 2 bytes per operator slot of every walker for a
 * next-same-flavor table) and synchronises; KT_ENOMEM if that fails. */
#define KT_DA_MAX_TRIES 16
kt_status kt_sweep_run_da_multi(kt_sweep *s, int32_t n_steps, int32_t tries, const double *uniforms,
                                int32_t meas_every, void *stream);

/* Kernel tiling: every (walker, kept state) item of the Krylov stage is
 * processed by a group of group_lanes lanes of one warp (32 / group_lanes items
 * per warp). kt_model_set_tiling picks one of the compiled group sizes
 * (KT_EINVAL if it is not compiled for this model's block size).
 * kt_autotune times kt_trace on the caller's batch (DEVICE buffers as in
 * kt_trace) for every compiled group size, keeps the fastest and writes it to
 * *group_lanes. It synchronises on the stream. */
kt_status kt_model_set_tiling(kt_model *m, int32_t group_lanes);
kt_status kt_autotune(kt_model *m, const kt_seq_batch *batch, int8_t *sign, double *logabs, int32_t *status,
                      void *workspace, size_t workspace_bytes, void *stream, int32_t *group_lanes);

/* Per-stage timing with CUDA events (profiling aid, not part of the method).
 * After kt_timing_begin(m, max_launches), each of the next max_launches trace
 * or trace-ratio calls on m records CUDA events on its own stream around its
 * four stages: 0 validation/edit, 1 structural pruning and the ordering of the
 * surviving items by length (two kernels), 2 Krylov items, 3 reduction. kt_timing_end waits for those events, writes the summed
 * durations in milliseconds to ms_per_stage[4] and the number of recorded calls
 * to *launches, and stops recording. Calls beyond max_launches run untimed.
 * Not thread-safe: do not share a model between host threads while timing. */
kt_status kt_timing_begin(kt_model *m, int32_t max_launches);
kt_status kt_timing_end(kt_model *m, double *ms_per_stage, int32_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* KT_H */
