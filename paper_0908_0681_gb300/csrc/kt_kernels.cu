// CUDA kernels (sm_103a) of the Krylov local-trace engine.
//
// Pipeline per call (all on the caller's stream):
//   1. prep    - one thread per walker: validate the sequence (sorted, times in
//                [0, beta), flavors in range) and, for a trace ratio, turn the
//                proposed local update (Sec. II) into an edit descriptor.
//   2. prune   - one thread per (walker, kept state): follow the block of the
//                state through the edited sequence with integer table lookups
//                only; pairs whose block path breaks are exact zeros ("the sum
//                runs over the sectors compatible with the operator
//                sequence", Sec. II). Survivors go to a worklist.
//   3. items   - persistent warps, one (walker, kept state) item at a time:
//                Sec. III steps 3-7. The kept eigenstate takes the scalar
//                first-interval factor, each c / c^+ is a gather with a
//                Jordan-Wigner sign, and every inner interval is a Lanczos
//                approximation of exp(-dtau (H - E0)) v (Sec. III step 5):
//                matrix-free SpMV on the block, FP64-accurate dot products and
//                norms (FP64, or double-float on the FP32 path), a three-term
//                recurrence, and the exponential of the small tridiagonal
//                matrix, with the Krylov dimension chosen per interval by an
//                a-posteriori error estimate.
//   4. reduce  - one thread per walker: signed log-sum-exp over kept states
//                (step 7-8) and, for a ratio, division by the current trace.
//
// Cached pipelines (the partial-state cache, CacheView): plan_kernel replaces
// prune for ratios (the stretch between valid cached states), build_plan_kernel
// fills the cache for fixed configurations, measure_plan_kernel prepares the
// observables at beta/2 from the cache; items_cached_kernel runs their units.
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>

#include "kt_internal.h"

#include "kt_device.cuh"

namespace kt {

int dispatch_items_f32(int kd, int G, const DevModel &M, const SeqView &S, const MoveView &mv, int has_moves,
                       const Workspace &ws, kt_stats *stats, cudaStream_t st);
int dispatch_items_f64(int kd, int G, const DevModel &M, const SeqView &S, const MoveView &mv, int has_moves,
                       const Workspace &ws, kt_stats *stats, cudaStream_t st);
int dispatch_items_cached_f32(int kd, const DevModel &M, const SeqView &S, const MoveView &mv, const Workspace &ws,
                              const CacheView &C, kt_stats *stats, cudaStream_t st);
int dispatch_items_cached_f64(int kd, const DevModel &M, const SeqView &S, const MoveView &mv, const Workspace &ws,
                              const CacheView &C, kt_stats *stats, cudaStream_t st);

namespace {
using namespace dev;

// ---------------------------------------------------------------------------
// 1. validation and move editing
// ---------------------------------------------------------------------------
__global__ void prep_kernel(DevModel M, SeqView S, MoveView mv, int has_moves, const int8_t *cur_sign, Workspace ws,
                            kt_stats *stats) {
  // one warp per walker: the lanes read consecutive operators (coalesced) and decide by ballot
  const int lane = threadIdx.x & 31;
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ws.counters[0] = 0;
    ws.counters[1] = 0;
    ws.counters[2] = 0;
    ws.counters[3] = 0;
  }
  if (w >= S.n) return;
  const int o = S.offsets[w], K = S.lens ? S.lens[w] : S.offsets[w + 1] - o;
  int st = KT_OK;
  int4 d = make_int4(-1, 0, 0, K);
  if (K < 0) {
    st = KT_EINVAL;
  } else if (!S.trusted) {
    // times non-decreasing from 0 and below beta, flavors and daggers in range
    double carry = 0.0;
    for (int base = 0; base < K; base += 32) {
      const int i = base + lane;
      double t = 0.0;
      int f = 0, g = 0;
      if (i < K) {
        t = __ldg(S.tau + o + i);
        f = __ldg(S.flavor + o + i);
        g = __ldg(S.dagger + o + i);
      }
      double prev = __shfl_up_sync(FULL, t, 1);
      if (lane == 0) prev = carry;
      const bool bad = i < K && (!(t >= prev) || !(t < M.beta) || f >= M.nf || g > 1);
      if (__any_sync(FULL, bad)) {
        st = KT_EINVAL;
        break;
      }
      carry = __shfl_sync(FULL, t, 31);
    }
  }
  if (has_moves && st == KT_OK) {
    const int kind = mv.kind[w], f = mv.flavor[w];
    if (f >= M.nf) {
      st = KT_EINVAL;
    } else if (kind == 0) {
      const double td = mv.t_dag[w], ta = mv.t_ann[w];
      if (!(td >= 0.0 && td < M.beta && ta >= 0.0 && ta < M.beta)) {
        st = KT_EINVAL;
      } else {
        // insertion points: the number of operators at or before each new time (the sorted
        // sequence's upper bound)
        const double tA = td < ta ? td : ta, tB = td < ta ? ta : td;
        int pa = 0, pb = 0;
        for (int base = 0; base < K; base += 32) {
          const int i = base + lane;
          const double t = i < K ? __ldg(S.tau + o + i) : 0.0;
          pa += __popc(__ballot_sync(FULL, i < K && t <= tA));
          pb += __popc(__ballot_sync(FULL, i < K && t <= tB));
        }
        d = make_int4(0, pa, pb, K + 2);
      }
    } else if (kind == 1) {
      const int r = mv.rem_idx[w];
      if (r < 0 || r >= K || S.flavor[o + r] != f) {
        st = KT_EINVAL;
      } else {
        // its partner: the next operator of the flavor after r, cyclically
        int j = -1;
        for (int base = r + 1; base < K && j < 0; base += 32) {
          const int i = base + lane;
          const unsigned m = __ballot_sync(FULL, i < K && __ldg(S.flavor + o + i) == f);
          if (m) j = base + __ffs(m) - 1;
        }
        for (int base = 0; base < r && j < 0; base += 32) {
          const int i = base + lane;
          const unsigned m = __ballot_sync(FULL, i < r && __ldg(S.flavor + o + i) == f);
          if (m) j = base + __ffs(m) - 1;
        }
        if (j < 0 || S.dagger[o + j] == S.dagger[o + r]) {
          st = KT_EINVAL;
        } else {
          d = make_int4(1, r < j ? r : j, r < j ? j : r, K - 2);
        }
      }
    } else {
      st = KT_EINVAL;
    }
    if (st == KT_OK && cur_sign[w] == 0) st = KT_EZEROWEIGHT;
  }
  if (lane == 0) {
    ws.desc[w] = d;
    ws.wstatus[w] = st;
    if (stats) atomicAdd(&stats->walkers, 1ull);
  }
}

// ---------------------------------------------------------------------------
// 2. structural pruning
// ---------------------------------------------------------------------------
// Structural pruning of one walker by one warp: the block of each lane's kept state after the
// first Kn operators of the walker's sequence, get(i) giving operator i (b = -1: a lane
// without an item). 32 operators are read at a time, one per lane (coalesced), and operator
// j reaches every lane by shuffle; a zero (b = -1) stays zero.
template <typename Get>
__device__ __forceinline__ int warp_block_walk(const DevModel &M, int b, int Kn, int lane, const Get &get) {
  const size_t row = (size_t)2 * M.nf;
  for (int base = 0; base < Kn; base += 32) {
    int code = 0;
    if (base + lane < Kn) {
      const Op op = get(base + lane);
      code = 2 * op.f + op.dag;
    }
    const int n = Kn - base < 32 ? Kn - base : 32;
    for (int j = 0; j < n; ++j) {
      const int cj = __shfl_sync(FULL, code, j);
      if (b >= 0) b = __ldg(M.blk_target + (size_t)b * row + cj);
    }
  }
  return b;
}

__global__ void prune_kernel(DevModel M, SeqView S, MoveView mv, int has_moves, Workspace ws, kt_stats *stats) {
  // one warp per walker: 32 operators of the edited sequence are read at a time, one per
  // lane, and every lane follows its kept states' blocks through them (operator j by shuffle)
  const int lane = threadIdx.x & 31;
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (w >= S.n) return;
  const int nk = M.n_kept;
  for (int q = lane; q < nk; q += 32) {
    const int item = w * nk + q;
    ws.item_sign[item] = 0;
    ws.item_status[item] = KT_OK;
    ws.item_log[item] = -INFINITY;
    ws.pair_flag[item] = 0;
  }
  if (ws.wstatus[w] != KT_OK) return;
  const Cursor c = make_cursor(S, mv, has_moves != 0, ws.desc, w);
  const int Kn = c.d.w;
  int n_alive = 0;
  for (int q0 = 0; q0 < nk; q0 += 32) {
    const int q = q0 + lane;
    const int b0 = q < nk ? __ldg(M.kept_blk + q) : -1;
    const int b = warp_block_walk(M, b0, Kn, lane, [&](int i) { return c.get(i); });
    const bool alive = q < nk && b == b0;
    if (alive) {
      const int slot = atomicAdd(&ws.counters[0], 1);
      ws.worklist[slot] = w * nk + q;
    }
    n_alive += __popc(__ballot_sync(FULL, alive));
  }
  if (stats && lane == 0) {
    atomicAdd(&stats->items, (unsigned long long)nk);
    atomicAdd(&stats->items_alive, (unsigned long long)n_alive);
  }
}

// Cached mode: structural pruning as above, and for the surviving items the
// stretch of the edited sequence that the partial-state cache does not cover: the
// forward unit starts after op y-1 with y = min(lo, f) (the last valid forward state
// before the window), the backward unit at op x with x the first position at or
// after the window whose backward state is valid; they meet at m, the middle of
// [y, x]. Walkers longer than the cache (before or after the edit) use y = 0,
// x = K_new without writing states. write = 0: the cache is only read (no state of
// this call is stored).
__global__ void plan_kernel(DevModel M, SeqView S, MoveView mv, Workspace ws, CacheView C, int write,
                            kt_stats *stats) {
  // one warp per walker, lanes over its kept states (the walk of prune_kernel)
  const int lane = threadIdx.x & 31;
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (w >= S.n) return;
  const int nk = M.n_kept;
  for (int q = lane; q < nk; q += 32) {
    const int item = w * nk + q;
    ws.item_sign[item] = 0;
    ws.item_status[item] = KT_OK;
    ws.item_log[item] = -INFINITY;
    ws.pair_flag[item] = 0;
    C.plan[item] = make_int4(0, 0, 0, 0);
  }
  if (ws.wstatus[w] != KT_OK) return;
  const Cursor c = make_cursor(S, mv, true, ws.desc, w);
  const int Kn = c.d.w, Ko = c.d.x == 0 ? Kn - 2 : Kn + 2;
  int lo, hi;
  edit_window(c.d, lo, hi);
  int n_alive = 0;
  for (int q0 = 0; q0 < nk; q0 += 32) {
    const int q = q0 + lane;
    const int b0 = q < nk ? __ldg(M.kept_blk + q) : -1;
    const int b = warp_block_walk(M, b0, Kn, lane, [&](int i) { return c.get(i); });
    const bool alive = q < nk && b == b0;
    n_alive += __popc(__ballot_sync(FULL, alive));
    if (q >= nk) continue;
    const int item = w * nk + q;
    // read-only use (fixed configurations): the cache was built for every operator of the
    // current sequence, so a walker whose length differs from the build is evaluated in full
    const bool cached = Kn <= C.P && Ko <= C.P && (write || C.f[item] == Ko);
    int y = 0, x = Kn;
    if (cached) {
      const int f = C.f[item], gr = C.gr[item];
      y = lo < f ? lo : f;
      const int x_old = max(hi - (Kn - Ko), Ko - gr);
      x = x_old + (Kn - Ko);
    }
    const int m = y + (x - y) / 2;
    C.plan[item] = make_int4(y, x, m, (cached && write ? 1 : 0) | (alive ? 2 : 0));
    if (alive) ws.worklist[atomicAdd(&ws.counters[0], 1)] = item;
  }
  if (stats && lane == 0) {
    atomicAdd(&stats->items, (unsigned long long)nk);
    atomicAdd(&stats->items_alive, (unsigned long long)n_alive);
  }
}

// Cache build for the current configurations: every (walker, kept state) item of a
// walker within the cache length gets a forward unit over all its operators and a
// backward unit over all of them, storing every state (zero states included, so that
// a later edit that revives the item finds its prefix and suffix).
__global__ void build_plan_kernel(DevModel M, SeqView S, Workspace ws, CacheView C) {
  const int item = blockIdx.x * blockDim.x + threadIdx.x;
  const int nk = M.n_kept;
  if (item >= S.n * nk) return;
  const int w = item / nk;
  ws.pair_flag[item] = 0;
  const int K = ws.desc[w].w;
  const bool ok = ws.wstatus[w] == KT_OK && K <= C.P;
  C.f[item] = ok ? K : 0;
  C.gr[item] = ok ? K : 0;
  C.plan[item] = make_int4(0, K, 0, ok ? 1 | 2 | 4 : 0);
  if (ok) ws.worklist[atomicAdd(&ws.counters[0], 1)] = item;
}

// Observables at beta/2 of the current configurations from the cache: the forward half
// of an item covers the operators before beta/2 from its last valid cached state, the
// backward half those after it from its first valid cached state, and they meet at
// beta/2 (flag 8); the states they pass are stored (they belong to the current
// configuration) and extend the valid ranges.
__global__ void measure_plan_kernel(DevModel M, SeqView S, Workspace ws, CacheView C, kt_stats *stats) {
  // one warp per walker, lanes over its kept states (the walk of prune_kernel)
  const int lane = threadIdx.x & 31;
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (w >= S.n) return;
  const int nk = M.n_kept;
  for (int q = lane; q < nk; q += 32) {
    const int item = w * nk + q;
    ws.item_sign[item] = 0;
    ws.item_status[item] = KT_OK;
    ws.item_log[item] = -INFINITY;
    ws.pair_flag[item] = 0;
    C.plan[item] = make_int4(0, 0, 0, 0);
  }
  if (ws.wstatus[w] != KT_OK) return;
  const int o = __ldg(S.offsets + w), K = ws.desc[w].w;
  // m: the operators before beta/2 (the lower bound of the sorted times)
  int m = 0;
  for (int base = 0; base < K; base += 32) {
    const int i = base + lane;
    m += __popc(__ballot_sync(FULL, i < K && __ldg(S.tau + o + i) < 0.5 * M.beta));
  }
  const bool cached = K <= C.P;
  int n_alive = 0;
  for (int q0 = 0; q0 < nk; q0 += 32) {
    const int q = q0 + lane;
    const int b0 = q < nk ? __ldg(M.kept_blk + q) : -1;
    const int b = warp_block_walk(M, b0, K, lane, [&](int i) { return load_op(S, o + i); });
    const bool alive = q < nk && b == b0;
    n_alive += __popc(__ballot_sync(FULL, alive));
    if (q >= nk) continue;
    const int item = w * nk + q;
    int y = 0, x = K;
    if (cached) {
      const int f = C.f[item], gr = C.gr[item];
      y = m < f ? m : f;
      x = max(m, K - gr);
    }
    C.plan[item] = make_int4(y, x, m, (cached ? 1 : 0) | (alive ? 2 : 0) | 8);
    if (alive) ws.worklist[atomicAdd(&ws.counters[0], 1)] = item;
  }
  if (stats && lane == 0) {
    atomicAdd(&stats->items, (unsigned long long)nk);
    atomicAdd(&stats->items_alive, (unsigned long long)n_alive);
  }
}

// After the accept decision of a cached step, one warp per (walker, kept state)
// item: an accepted move makes its tentative states (scratch) the cache's and the
// valid ranges meet at m; a rejected one keeps the cache and only extends the valid
// ranges by the states written outside the window; a pruned item (zero in the new
// configuration) keeps the unchanged prefix and suffix if the move is accepted.
__global__ void cache_commit_kernel(CacheView C, int n, int nk, const int4 *__restrict__ desc,
                                    const int32_t *__restrict__ wstatus, const int8_t *__restrict__ accepted,
                                    const int32_t *__restrict__ rstatus, int words) {
  const int lane = threadIdx.x & 31;
  const int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (item >= n * nk) return;
  const int w = item / nk;
  if (wstatus[w] != KT_OK) return;  // no update evaluated (a null or invalid move)
  const int4 pl = C.plan[item];
  const bool acc = accepted[w] != 0;
  if (!(pl.w & 1)) {
    if (acc && lane == 0) {
      C.f[item] = 0;
      C.gr[item] = 0;
    }
    return;
  }
  const int4 d = desc[w];
  int lo, hi;
  edit_window(d, lo, hi);
  const int Kn = d.w, Ko = d.x == 0 ? Kn - 2 : Kn + 2;
  const int y = pl.x, x = pl.y, m = pl.z;
  if (!(pl.w & 2)) {
    if (acc && lane == 0) {
      C.f[item] = min(C.f[item], lo);
      C.gr[item] = min(C.gr[item], Ko - (hi - (Kn - Ko)));
    }
    return;
  }
  if (!acc) {
    if (lane == 0 && rstatus[w] == KT_OK) {
      C.f[item] = max(C.f[item], min(m, lo));
      C.gr[item] = max(C.gr[item], Kn - max(m, hi));
    }
    return;
  }
  const size_t eb = (size_t)item * ((size_t)C.P + 1);
  const uint32_t *sfv = (const uint32_t *)C.sfvec, *sbv = (const uint32_t *)C.sbvec;
  uint32_t *fv = (uint32_t *)C.fvec, *bv = (uint32_t *)C.bvec;
  // forward slots (max(y, lo), m] and backward reverse slots of positions [m, min(x, hi))
  const int f0 = max(y, lo) + 1, nfw = m - f0 + 1;
  const int r0 = Kn - min(x, hi) + 1, nbw = (Kn - m) - r0 + 1;
  for (int k = lane; k < nfw * words; k += 32) {
    const size_t e = eb + f0 + k / words;
    fv[e * words + k % words] = sfv[e * words + k % words];
  }
  for (int k = lane; k < nbw * words; k += 32) {
    const size_t e = eb + r0 + k / words;
    bv[e * words + k % words] = sbv[e * words + k % words];
  }
  for (int k = lane; k < nfw; k += 32) {
    C.fblk[eb + f0 + k] = C.sfblk[eb + f0 + k];
    C.flog[eb + f0 + k] = C.sflog[eb + f0 + k];
  }
  for (int k = lane; k < nbw; k += 32) {
    C.bblk[eb + r0 + k] = C.sbblk[eb + r0 + k];
    C.blog[eb + r0 + k] = C.sblog[eb + r0 + k];
  }
  if (lane == 0) {
    C.f[item] = m;
    C.gr[item] = Kn - m;
  }
}

// Alive items ordered by the operators their two units propagate, longest first: the
// length of the walker's (edited) sequence, or with a cache plan the stretch [y, x) between
// valid cached states. A counting sort in one block, using the half-item info array as
// scratch (the items kernels write it only later). The items kernels then hand every group
// of four claims one unit from the long end and three from the short end, so that a long
// unit shares its warp with short ones, which finish early and leave it alone.
__global__ void __launch_bounds__(1024) order_kernel(DevModel M, Workspace ws, const int4 *__restrict__ plan) {
  constexpr int NB = 1024;
  __shared__ int cnt[NB];
  const int t = threadIdx.x, nk = M.n_kept;
  const int n = ws.counters[0];
  int32_t *tmp = ws.half_info;
  cnt[t] = 0;
  __syncthreads();
  // bin of an item (bin 0 = the longest); keys are >= 0 by construction, clamped anyway
  auto bin = [&](int item) {
    int k;
    if (plan) {
      const int4 p = plan[item];
      k = p.y - p.x;
    } else {
      k = ws.desc[item / nk].w;
    }
    return NB - 1 - min(max(k, 0) >> 2, NB - 1);
  };
  for (int i = t; i < n; i += NB) atomicAdd(&cnt[bin(ws.worklist[i])], 1);
  __syncthreads();
  // exclusive scan of the bin counts (bin 0 = the longest sequences)
  const int c = cnt[t];
  __syncthreads();
  for (int o = 1; o < NB; o <<= 1) {
    const int v = t >= o ? cnt[t - o] : 0;
    __syncthreads();
    cnt[t] += v;
    __syncthreads();
  }
  cnt[t] -= c;
  __syncthreads();
  for (int i = t; i < n; i += NB) {
    const int item = ws.worklist[i];
    tmp[atomicAdd(&cnt[bin(item)], 1)] = item;
  }
  __syncthreads();
  for (int i = t; i < n; i += NB) ws.worklist[i] = tmp[i];
}

// ---------------------------------------------------------------------------
// 4. reduction over kept states, ratio
// ---------------------------------------------------------------------------
__global__ void reduce_kernel(DevModel M, int n, int has_moves, const int8_t *cur_sign, const double *cur_logabs,
                              Workspace ws, int8_t *sign, double *logv, int32_t *status) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n) return;
  const int nk = M.n_kept;
  int st = ws.wstatus[w];
  if (st != KT_OK) {
    sign[w] = 0;
    logv[w] = (st == KT_EZEROWEIGHT || st == KT_EINVAL) ? NAN : -INFINITY;
    status[w] = st;
    return;
  }
  double mx = -INFINITY;
  for (int q = 0; q < nk; ++q) {
    const int it = w * nk + q;
    if (ws.item_sign[it] != 0) mx = fmax(mx, ws.item_log[it]);
    const int is = ws.item_status[it];
    if (is != KT_OK && (st == KT_OK || is == KT_ENUMERIC)) st = is;
  }
  double acc = 0.0;
  if (mx > -INFINITY)
    for (int q = 0; q < nk; ++q) {
      const int it = w * nk + q;
      if (ws.item_sign[it] != 0) acc += (double)ws.item_sign[it] * exp(ws.item_log[it] - mx);
    }
  int sg = 0;
  double la = -INFINITY;
  if (acc != 0.0 && isfinite(mx)) {
    sg = acc > 0.0 ? 1 : -1;
    la = mx + log(fabs(acc)) - M.beta * M.E0;
  }
  if (has_moves) {
    const int cs = cur_sign[w];
    sign[w] = (int8_t)(sg * cs);
    logv[w] = sg != 0 ? la - cur_logabs[w] : -INFINITY;
  } else {
    sign[w] = (int8_t)sg;
    logv[w] = la;
  }
  if (sg != 0 && !isfinite(la)) st = KT_ENUMERIC;
  status[w] = st;
}

// Observables at tau = beta/2: per walker, the kept-state items weighted by
// their share of the trace (same signed log-sum-exp as reduce_kernel).
__global__ void measure_reduce_kernel(DevModel M, int n, Workspace ws, double *obs) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n) return;
  const int nk = M.n_kept, nf = M.nf, no = M.n_orb, nl = nf + no + 1;
  const int nsec = (no + 1) * (no + 1), ntot = nl + nsec;
  double *out = obs + (size_t)w * ntot;
  double mx = -INFINITY;
  if (ws.wstatus[w] == KT_OK)
    for (int q = 0; q < nk; ++q) {
      const int it = w * nk + q;
      if (ws.item_sign[it] != 0) mx = fmax(mx, ws.item_log[it]);
    }
  for (int k = 0; k < ntot; ++k) out[k] = 0.0;
  double den = 0.0;
  if (mx > -INFINITY)
    for (int q = 0; q < nk; ++q) {
      const int it = w * nk + q;
      if (ws.item_sign[it] == 0) continue;
      const double c = (double)ws.item_sign[it] * exp(ws.item_log[it] - mx);
      den += c;
      for (int k = 0; k < nl; ++k) out[k] += c * ws.item_obs[(size_t)it * nl + k];
      const int x = __ldg(M.st_bits + __ldg(M.blk_off + ws.item_blk[it]));
      const int nup = __popc(x & 0x5555), ndn = __popc(x & 0xaaaa);
      out[nl + nup * (no + 1) + ndn] += c;
    }
  const double inv = (den != 0.0 && isfinite(mx)) ? 1.0 / den : NAN;
  for (int k = 0; k < ntot; ++k) out[k] *= inv;
}

}  // namespace


int kernel_dmax_for(int d_max) {
  if (d_max <= 10) return 10;
  if (d_max <= 36) return 36;
  if (d_max <= 128) return 128;
  return 0;
}

int kernel_pmax_for(int kd) {
  switch (kd) {
    case 10: return 10;
    case 36: return 24;
    case 128: return 40;
  }
  return 0;
}

int kernel_groups_for(int kd, int *out, int cap) {
  int n = 0;
#define KT_LIST(D, P, GG) \
  if (kd == D && n < cap) out[n++] = GG;
  KT_FOR_VARIANTS(KT_LIST)
#undef KT_LIST
  return n;
}

// Lane-group size before any autotuning: the sizes kt_autotune picked on GB300 for the
// five-orbital batch (10-row blocks: 8 lanes FP32, 4 lanes FP64) and the seven-orbital
// batch (36-row blocks: 16 lanes).
int default_group_for(int kd, int precision) {
  switch (kd) {
    case 10: return precision == KT_FP64 ? 4 : 8;
    case 36: return 16;
    case 128: return 32;
  }
  return 32;
}

int launch_pipeline(const DevModel &M, int precision, int kd, int G, const SeqView &S, const MoveView *moves,
                    const int8_t *cur_sign, const double *cur_logabs, int8_t *sign, double *logv, int32_t *status,
                    kt_stats *stats, const Workspace &ws, void *stream, const StageEvents *timing, double *obs) {
  cudaStream_t st = (cudaStream_t)stream;
  auto mark = [&](int i) {
    if (timing) cudaEventRecord((cudaEvent_t)timing->ev[i], st);
  };
  const int n = S.n;
  const int has_moves = moves ? 1 : 0;
  MoveView mv = moves ? *moves : MoveView{};
  cudaGetLastError();
  mark(0);
  prep_kernel<<<(n + 7) / 8, 256, 0, st>>>(M, S, mv, has_moves, cur_sign, ws, stats);
  mark(1);
  const long long items = (long long)n * M.n_kept;
  if (items > 0) {
    prune_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(M, S, mv, has_moves, ws, stats);
    order_kernel<<<1, 1024, 0, st>>>(M, ws, nullptr);
  }
  mark(2);
  int rc = (int)cudaGetLastError();
  if (rc) return rc;
  if (items > 0) {
    rc = (precision == KT_FP64) ? dispatch_items_f64(kd, G, M, S, mv, has_moves, ws, stats, st)
                                : dispatch_items_f32(kd, G, M, S, mv, has_moves, ws, stats, st);
    if (rc) return rc;
  }
  mark(3);
  reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(M, n, has_moves, cur_sign, cur_logabs, ws, sign, logv, status);
  if (obs) measure_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(M, n, ws, obs);
  mark(4);
  return (int)cudaGetLastError();
}

int launch_cached_pipeline(const DevModel &M, int precision, int kd, const SeqView &S, const MoveView &mv,
                           const int8_t *cur_sign, const double *cur_logabs, int8_t *sign, double *logv,
                           int32_t *status, const Workspace &ws, const CacheView &C, bool write, kt_stats *stats,
                           void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int n = S.n;
  cudaGetLastError();
  prep_kernel<<<(n + 7) / 8, 256, 0, st>>>(M, S, mv, 1, cur_sign, ws, stats);
  const long long items = (long long)n * M.n_kept;
  if (items > 0) {
    plan_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(M, S, mv, ws, C, write ? 1 : 0, stats);
    order_kernel<<<1, 1024, 0, st>>>(M, ws, C.plan);
  }
  int rc = (int)cudaGetLastError();
  if (rc) return rc;
  if (items > 0) {
    rc = (precision == KT_FP64) ? dispatch_items_cached_f64(kd, M, S, mv, ws, C, stats, st)
                                : dispatch_items_cached_f32(kd, M, S, mv, ws, C, stats, st);
    if (rc) return rc;
  }
  reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(M, n, 1, cur_sign, cur_logabs, ws, sign, logv, status);
  return (int)cudaGetLastError();
}

int launch_cache_build(const DevModel &M, int precision, int kd, const SeqView &S, const Workspace &ws,
                       const CacheView &C, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int n = S.n;
  cudaGetLastError();
  prep_kernel<<<(n + 7) / 8, 256, 0, st>>>(M, S, MoveView{}, 0, nullptr, ws, nullptr);
  const long long items = (long long)n * M.n_kept;
  if (items == 0) return (int)cudaGetLastError();
  build_plan_kernel<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(M, S, ws, C);
  order_kernel<<<1, 1024, 0, st>>>(M, ws, C.plan);
  int rc = (int)cudaGetLastError();
  if (rc) return rc;
  rc = (precision == KT_FP64) ? dispatch_items_cached_f64(kd, M, S, MoveView{}, ws, C, nullptr, st)
                              : dispatch_items_cached_f32(kd, M, S, MoveView{}, ws, C, nullptr, st);
  if (rc) return rc;
  return (int)cudaGetLastError();
}

int launch_cached_measure(const DevModel &M, int precision, int kd, const SeqView &S, int8_t *sign, double *logv,
                          int32_t *status, double *obs, const Workspace &ws, const CacheView &C, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int n = S.n;
  cudaGetLastError();
  prep_kernel<<<(n + 7) / 8, 256, 0, st>>>(M, S, MoveView{}, 0, nullptr, ws, nullptr);
  const long long items = (long long)n * M.n_kept;
  if (items > 0) {
    measure_plan_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(M, S, ws, C, nullptr);
    order_kernel<<<1, 1024, 0, st>>>(M, ws, C.plan);
    int rc = (int)cudaGetLastError();
    if (rc) return rc;
    rc = (precision == KT_FP64) ? dispatch_items_cached_f64(kd, M, S, MoveView{}, ws, C, nullptr, st)
                                : dispatch_items_cached_f32(kd, M, S, MoveView{}, ws, C, nullptr, st);
    if (rc) return rc;
  }
  reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(M, n, 0, nullptr, nullptr, ws, sign, logv, status);
  measure_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(M, n, ws, obs);
  return (int)cudaGetLastError();
}

int launch_cache_commit(const CacheView &C, int n, int nk, const int4 *desc, const int32_t *wstatus,
                        const int8_t *accepted, const int32_t *rstatus, int words, void *stream) {
  const long long nitems = (long long)n * nk;
  if (nitems == 0) return 0;
  cache_commit_kernel<<<(unsigned)((nitems * 32 + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      C, n, nk, desc, wstatus, accepted, rstatus, words);
  return (int)cudaGetLastError();
}

}  // namespace kt
