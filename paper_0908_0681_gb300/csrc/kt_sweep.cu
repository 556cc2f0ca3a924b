// Batched CT-HYB Markov chains (Sec. II): one Metropolis step per walker and
// launch group, with the weight of Eq. (weight_strong) for a flavor-diagonal
// hybridization, w = s_P * T * prod_f det G_f.
//
// Per step (all on the caller's stream, no host synchronisation):
//   propose  - one warp per walker: the move from its six uniforms, the
//              proposal factor, and the FP64 determinant ratio with the
//              permutation sign. Insertion borders G_f with a new creator row
//              and annihilator column: ratio lambda = d - R M C (M = G_f^{-1}),
//              and the vectors M C and R M are kept for the update. Removal of
//              the pair in storage row i / column j: ratio M_ji.
//   trace    - the trace-ratio pipeline of the library on the proposed edits.
//   accept   - one warp per walker: Metropolis test on the product of the
//              ratios; an accepted move edits the walker's sequence in place and
//              updates M in O(k^2) (bordered inverse, or Schur complement after
//              moving the removed row and column to the end).
//   measure  - every meas_every steps: G_f(tau) from M, the expansion orders,
//              and optionally the observables at beta/2 (kt_measure pipeline).
//
// Storage of flavor f of walker w: creator times row_t[0..k), annihilator times
// col_t[0..k) in insertion order (not sorted), and M = G_f^{-1} row-major with
// rows indexed by annihilators and columns by creators, M[j * k_cap + i].
// The weight's sign is s_P * sign(T) * prod sign(det G_f); it is independent of
// how rows and columns are ordered (a row or column swap flips det G_f and the
// permutation sign together), so an insertion appends its pair at the end of the
// flavor's block of the bath-operator sequence and
//   s_P(new) / s_P(old) = (-1)^X,  X = sum over the two new times t of
//     #{old ops x : flavor(x) <= f, tau_x < t} + #{old ops x : flavor(x) > f, tau_x > t}
//   plus 1 if tau'_new < tau_new,
// and a removal is the inverse of inserting its pair into the reduced configuration.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "kt_internal.h"

#include "kt_device.cuh"

namespace kt {
namespace {
using namespace dev;

enum { C_INS_PROP, C_INS_ACC, C_REM_PROP, C_REM_ACC, C_NULL, C_CAP, C_TRACE_ERR, C_MEAS, C_STAGE1, C_TRACE_EVAL };

struct SweepView {
  int nw, nf, kcap, cap, n_tau, n_bins, nobs;
  double beta;
  const int32_t *offsets;
  int32_t *lens;
  double *tau;
  uint8_t *flv, *dag;
  int32_t *kf;        // [nw][nf]
  double *row_t;      // [nw][nf][kcap]
  double *col_t;      // [nw][nf][kcap]
  double *M;          // [nw][nf][kcap][kcap]
  const double *hyb;  // [nf][n_tau + 1]
  int8_t *tr_sign;
  double *tr_log;
  int8_t *w_sign;
  double *det_log;
  // proposal
  uint8_t *mv_kind, *mv_flv;
  double *mv_tdag, *mv_tann;
  int32_t *mv_rem;
  int8_t *p_valid;    // 1 move to test, 0 null
  int8_t *p_sign;     // sign of the determinant ratio times (-1)^X
  double *p_lprop;    // log proposal factor
  double *p_ldet;     // log |determinant ratio|
  double *p_lambda;   // insertion: lambda
  int32_t *p_ij;      // removal: [2] storage row i (creator), column j (annihilator)
  double *p_vec;      // insertion: [nw][2 kcap]: M C (by annihilator), R M (by creator)
  int8_t *p_kind;     // 0 insertion, 1 removal (also for null moves)
  double *p_t1, *p_t2;  // the move's first operator time and its partner's
  int8_t *p_seg;      // 1 if the first operator is a c^+
  int32_t *p_pair;    // [2 nw] sequence indices of a removal's pair (-1 for insertions)
  int8_t *p_acc;      // 1 if this step's move was accepted
  // delayed acceptance
  int n_in;           // feature length
  __nv_bfloat16 *X;   // [nw][n_in] features of the proposals
  float *ytil;        // [nw] predicted log|T_new / T_old|
  // trace ratio outputs
  int8_t *r_sign;
  double *r_log;
  int32_t *r_status;
  // measurement
  double *g_acc, *sign_sum, *order_sum, *obs_sum, *obs_tmp;
  int8_t *m_sign;
  double *m_log;
  int32_t *m_status;
  unsigned long long *counters;
  // refresh from scratch (kt_sweep_refresh)
  double *f_detlog;   // [nw][nf] log|det G_f| recomputed
  int8_t *f_detsign;  // [nw][nf] its sign (0: singular)
  int8_t *f_tsign;    // [nw] trace recomputed
  double *f_tlog;
  int32_t *f_tstat;
  unsigned long long *f_dev;  // [4] max |d log T| and max |d log det| (bits of non-negative doubles),
                              //     sign mismatches, walkers left unchanged
};

// Fh_f(x): linear interpolation of F_f on tau_i = i beta / n_tau, antiperiodic for x < 0.
__device__ __forceinline__ double hyb_F(const SweepView &S, int f, double t) {
  const double pos = t / S.beta * S.n_tau;
  int i = (int)floor(pos);
  i = i < 0 ? 0 : (i > S.n_tau - 1 ? S.n_tau - 1 : i);
  const double fr = pos - i;
  const double *tab = S.hyb + (size_t)f * (S.n_tau + 1);
  const double a = __ldg(tab + i), b = __ldg(tab + i + 1);
  return a + fr * (b - a);
}
__device__ __forceinline__ double hyb_Fh(const SweepView &S, int f, double x) {
  return x >= 0.0 ? hyb_F(S, f, x) : -hyb_F(S, f, x + S.beta);
}

__device__ __forceinline__ int warp_sum(int v) { return __reduce_add_sync(FULL, (unsigned)v); }
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Index of the m-th (0-based) operator of flavor f among ops[0 .. K), or -1.
__device__ int nth_of_flavor(const uint8_t *fl, int K, int f, int m, int lane) {
  int cnt = 0;
  for (int base = 0; base < K; base += 32) {
    const int idx = base + lane;
    unsigned msk = __ballot_sync(FULL, idx < K && fl[idx] == f);
    const int c = __popc(msk);
    if (cnt + c > m) {
      for (int r = m - cnt; r > 0; --r) msk &= msk - 1;
      return base + __ffs(msk) - 1;
    }
    cnt += c;
  }
  return -1;
}

// Parity count X of the permutation sign change for a pair (tdag, tann) of flavor f
// appended at the end of its flavor block, over the ops of [0, K) except skip1, skip2.
__device__ int perm_count(const double *tau, const uint8_t *fl, int K, int f, double tdag, double tann, int skip1,
                          int skip2, int lane) {
  int c = 0;
  for (int idx = lane; idx < K; idx += 32) {
    if (idx == skip1 || idx == skip2) continue;
    const double t = tau[idx];
    const int g = fl[idx];
    if (g <= f) c += (t < tdag) + (t < tann);
    else c += (t > tdag) + (t > tann);
  }
  c = warp_sum(c);
  return c + (tdag < tann ? 1 : 0);
}

// Multi-try delayed acceptance: per walker and step, T proposals drawn from the same
// configuration, each with its own seven uniforms, stored slot by slot (slot t * nw + w).
struct TryView {
  int T;
  int8_t *p_kind, *p_seg, *p_valid, *p_sign, *p_acc;
  double *p_t1, *p_t2, *mv_tdag, *mv_tann, *p_lprop, *p_ldet, *p_lambda, *p_vec;
  int32_t *p_pair, *mv_rem, *p_ij;
  uint8_t *mv_kind, *mv_flv;
  __nv_bfloat16 *X;
  float *ytil;
  unsigned long long *scratch_counters;  // the propose kernel's counters land here; the select kernel counts
  int32_t *n_tries;   // [nw] Metropolis steps the walker took this step (tries up to and including the selected one)
  int16_t *nxt;       // [nw][cap] next operator of the same flavor (sweep_next_flavor_kernel)
  double *u5;         // [nw] stage-2 uniform of the selected try
};

// The view of try t: the walker state of S, the proposal arrays of slot t.
__host__ __device__ inline SweepView try_view(const SweepView &S, const TryView &Tv, int t) {
  SweepView v = S;
  const size_t o = (size_t)t * S.nw;
  v.p_kind = Tv.p_kind + o; v.p_seg = Tv.p_seg + o; v.p_valid = Tv.p_valid + o; v.p_sign = Tv.p_sign + o;
  v.p_acc = Tv.p_acc + o; v.p_t1 = Tv.p_t1 + o; v.p_t2 = Tv.p_t2 + o; v.mv_tdag = Tv.mv_tdag + o;
  v.mv_tann = Tv.mv_tann + o; v.p_lprop = Tv.p_lprop + o; v.p_ldet = Tv.p_ldet + o; v.p_lambda = Tv.p_lambda + o;
  v.p_vec = Tv.p_vec + o * 2 * S.kcap; v.p_pair = Tv.p_pair + 2 * o; v.mv_rem = Tv.mv_rem + o;
  v.p_ij = Tv.p_ij + 2 * o; v.mv_kind = Tv.mv_kind + o; v.mv_flv = Tv.mv_flv + o;
  v.X = Tv.X + o * S.n_in; v.ytil = Tv.ytil + o;
  v.counters = Tv.scratch_counters;
  return v;
}

// Tv.T > 0: multi-try launch, blockIdx.y = try (uniforms of try t at uni + 7 t).
__global__ void sweep_propose_kernel(SweepView S0, const double *__restrict__ uni, int ustride, TryView Tv) {
  extern __shared__ double sh[];
  const SweepView S = Tv.T ? try_view(S0, Tv, blockIdx.y) : S0;
  if (Tv.T) uni += 7 * blockIdx.y;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int w = blockIdx.x * (blockDim.x >> 5) + wib;
  if (w >= S.nw) return;
  double *Cv = sh + (size_t)wib * 2 * S.kcap;  // new column C (by creator) / row R (by annihilator)
  double *Rv = Cv + S.kcap;
  const double *u = uni + (size_t)w * ustride;
  const int nf = S.nf;
  const double beta = S.beta;
  const int o = S.offsets[w], K = S.lens[w];
  if (lane == 0) {
    S.p_kind[w] = u[0] < 0.5 ? 0 : 1;
    S.p_t1[w] = 0.0;
    S.p_t2[w] = 0.0;
    S.p_seg[w] = 0;
    S.p_pair[2 * w] = -1;
    S.p_pair[2 * w + 1] = -1;
    S.p_acc[w] = 0;
  }
  const double *tau = S.tau + o;
  const uint8_t *fl = S.flv + o, *dg = S.dag + o;
  int f = (int)(u[1] * nf);
  f = f > nf - 1 ? nf - 1 : (f < 0 ? 0 : f);
  const int kf = S.kf[w * nf + f];
  const size_t fb = (size_t)w * nf + f;
  const double *Mf = S.M + fb * S.kcap * S.kcap;
  const double *rt = S.row_t + fb * S.kcap, *ct = S.col_t + fb * S.kcap;
  int valid = 0;
  if (u[0] < 0.5) {
    // ---- insertion ----
    if (lane == 0) atomicAdd(&S.counters[C_INS_PROP], 1ull);
    const double t1 = u[2] * beta;
    bool null_move = false;
    if (kf >= S.kcap) {
      null_move = true;
      if (lane == 0) atomicAdd(&S.counters[C_CAP], 1ull);
    }
    if (!(t1 < beta)) null_move = true;
    bool seg = true;
    double lmax = beta;
    if (!null_move && kf > 0) {
      int first_any = -1, found = -1;
      for (int base = 0; base < K && found < 0; base += 32) {
        const int idx = base + lane;
        const bool isf = idx < K && fl[idx] == f;
        const unsigned m_any = __ballot_sync(FULL, isf);
        const unsigned m_after = __ballot_sync(FULL, isf && tau[idx] > t1);
        if (first_any < 0 && m_any) first_any = base + __ffs(m_any) - 1;
        if (m_after) found = base + __ffs(m_after) - 1;
      }
      const int j = found >= 0 ? found : first_any;
      if (j < 0) {  // the operator counts always match k_f; the guard only keeps reads in bounds
        null_move = true;
      } else {
        seg = dg[j] == 1;
        const double tn = tau[j];
        lmax = tn > t1 ? tn - t1 : tn + beta - t1;
      }
    } else if (!null_move) {
      seg = u[4] < 0.5;
    }
    // separate multiply and add (no contraction): the proposal times are rounded as
    // written, so chains driven by the same uniforms visit bit-identical times
    double t2 = __dadd_rn(t1, __dmul_rn(u[3], lmax));
    if (t2 >= beta) t2 -= beta;
    if (t2 == t1) null_move = true;
    if (!null_move) {
      const double td = seg ? t1 : t2, ta = seg ? t2 : t1;
      const double lp = kf == 0 ? 2.0 * log(beta) : log(beta * lmax / (2.0 * (kf + 1)));
      // bordered matrix: C_i = Fh(tau'_i - ta), R_j = Fh(td - tau_j), d = Fh(td - ta)
      for (int i = lane; i < kf; i += 32) {
        Cv[i] = hyb_Fh(S, f, rt[i] - ta);
        Rv[i] = hyb_Fh(S, f, td - ct[i]);
      }
      __syncwarp();
      double *mc = S.p_vec + (size_t)w * 2 * S.kcap, *rm = mc + S.kcap;
      double part = 0.0;
      for (int j = lane; j < kf; j += 32) {  // (M C)_j
        double a = 0.0;
        for (int i = 0; i < kf; ++i) a = fma(Mf[(size_t)j * S.kcap + i], Cv[i], a);
        mc[j] = a;
        part = fma(Rv[j], a, part);
      }
      for (int i = lane; i < kf; i += 32) {  // (R M)_i
        double a = 0.0;
        for (int j = 0; j < kf; ++j) a = fma(Rv[j], Mf[(size_t)j * S.kcap + i], a);
        rm[i] = a;
      }
      const double lambda = hyb_Fh(S, f, td - ta) - warp_sum(part);
      const int X = perm_count(tau, fl, K, f, td, ta, -1, -1, lane);
      if (lane == 0) {
        S.p_t1[w] = t1;
        S.p_t2[w] = t2;
        S.p_seg[w] = seg ? 1 : 0;
        S.mv_kind[w] = 0;
        S.mv_tdag[w] = td;
        S.mv_tann[w] = ta;
        S.p_lprop[w] = lp;
        S.p_ldet[w] = log(fabs(lambda));
        S.p_sign[w] = (int8_t)((lambda > 0.0 ? 1 : (lambda < 0.0 ? -1 : 0)) * ((X & 1) ? -1 : 1));
        S.p_lambda[w] = lambda;
      }
      valid = lambda != 0.0 ? 1 : 0;
    }
  } else {
    // ---- removal ----
    if (lane == 0) atomicAdd(&S.counters[C_REM_PROP], 1ull);
    if (kf > 0) {
      int jsel = (int)(u[2] * 2 * kf);
      jsel = jsel > 2 * kf - 1 ? 2 * kf - 1 : jsel;
      const int a = nth_of_flavor(fl, K, f, jsel, lane);
      const int b = nth_of_flavor(fl, K, f, (jsel + 1) % (2 * kf), lane);
      const int c = kf > 1 ? nth_of_flavor(fl, K, f, (jsel + 2) % (2 * kf), lane) : a;
      // the operator counts always match k_f; the guard only keeps every read in bounds
      const bool found = a >= 0 && b >= 0 && c >= 0;
      const double t1 = found ? tau[a] : 0.0, t2 = found ? tau[b] : 0.0;
      double lp;
      if (kf == 1) {
        lp = -2.0 * log(beta);
      } else {
        const double tc = found ? tau[c] : 0.0;
        const double lmax = tc > t1 ? tc - t1 : tc + beta - t1;
        lp = log(2.0 * kf / (beta * lmax));
      }
      const int da = found ? dg[a] : 0, db = found ? dg[b] : 0;
      const double td = da == 1 ? t1 : t2, ta = da == 1 ? t2 : t1;
      int ri = -1, cj = -1;
      for (int base = 0; base < kf; base += 32) {
        const int idx = base + lane;
        const unsigned mr = __ballot_sync(FULL, idx < kf && rt[idx] == td);
        const unsigned mcn = __ballot_sync(FULL, idx < kf && ct[idx] == ta);
        if (ri < 0 && mr) ri = base + __ffs(mr) - 1;
        if (cj < 0 && mcn) cj = base + __ffs(mcn) - 1;
      }
      if (found && ri >= 0 && cj >= 0 && da != db) {
        const double ratio = Mf[(size_t)cj * S.kcap + ri];
        const int X = perm_count(tau, fl, K, f, td, ta, a, b, lane);
        if (lane == 0) {
          S.p_t1[w] = t1;
          S.p_t2[w] = t2;
          S.p_seg[w] = da == 1 ? 1 : 0;
          S.p_pair[2 * w] = a;
          S.p_pair[2 * w + 1] = b;
          S.mv_kind[w] = 1;
          S.mv_rem[w] = a;
          S.p_lprop[w] = lp;
          S.p_ldet[w] = log(fabs(ratio));
          S.p_sign[w] = (int8_t)((ratio > 0.0 ? 1 : (ratio < 0.0 ? -1 : 0)) * ((X & 1) ? -1 : 1));
          S.p_ij[2 * w] = ri;
          S.p_ij[2 * w + 1] = cj;
        }
        valid = ratio != 0.0 ? 1 : 0;
      }
    }
  }
  if (lane == 0) {
    S.mv_flv[w] = (uint8_t)f;
    S.p_valid[w] = (int8_t)valid;
    if (!valid) {
      // a move the trace stage skips (structural zero of the pipeline is avoided:
      // kind 2 is rejected by its validation without any work)
      S.mv_kind[w] = 2;
      atomicAdd(&S.counters[C_NULL], 1ull);
    }
  }
}

__global__ void sweep_accept_kernel(SweepView S, const double *__restrict__ u5s, int u5stride,
                                    const int4 *__restrict__ desc, bool delayed) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= S.nw) return;
  if (!S.p_valid[w]) return;
  if (lane == 0) atomicAdd(&S.counters[C_TRACE_EVAL], 1ull);
  const int st = S.r_status[w];
  if (st != KT_OK) {
    if (lane == 0) atomicAdd(&S.counters[C_TRACE_ERR], 1ull);
    return;
  }
  const int tsg = S.r_sign[w];
  if (tsg == 0) return;  // the new trace is zero
  // plain Metropolis: the whole ratio; delayed acceptance, stage 2: true over predicted trace ratio
  const double logR = delayed ? S.r_log[w] - (double)S.ytil[w] : S.r_log[w] + S.p_ldet[w] + S.p_lprop[w];
  const double u5 = u5s[(size_t)w * u5stride];
  const bool accept = (u5 > 0.0 ? log(u5) : -INFINITY) < logR;
  if (!accept) return;
  if (lane == 0) S.p_acc[w] = 1;
  const int nf = S.nf, f = S.mv_flv[w], kind = S.mv_kind[w];
  const int o = S.offsets[w];
  double *tau = S.tau + o;
  uint8_t *fl = S.flv + o, *dg = S.dag + o;
  const int4 d = desc[w];
  // 1. the walker's sequence, edited in place (same index map as the trace pipeline)
  if (kind == 0) {
    const double td = S.mv_tdag[w], ta = S.mv_tann[w];
    const double tA = td < ta ? td : ta, tB = td < ta ? ta : td;
    const int dA = td < ta ? 1 : 0, dB = 1 - dA;
    // new index i: i < p1 old i; i == p1 A; p1 < i <= p2 old i-1; i == p2+1 B; else old i-2.
    // Chunks from the top: every source index is <= i, read before any write of the chunk.
    const int Kn = d.w;
    for (int top = Kn - 1; top >= 0; top -= 32) {
      const int i = top - lane;
      double t = 0.0;
      int g = 0, h = 0;
      if (i >= 0) {
        int src = -1;
        if (i < d.y) src = i;
        else if (i == d.y) { t = tA; g = f; h = dA; }
        else if (i <= d.z) src = i - 1;
        else if (i == d.z + 1) { t = tB; g = f; h = dB; }
        else src = i - 2;
        if (src >= 0) { t = tau[src]; g = fl[src]; h = dg[src]; }
      }
      __syncwarp();
      if (i >= 0) { tau[i] = t; fl[i] = (uint8_t)g; dg[i] = (uint8_t)h; }
      __syncwarp();
    }
  } else {
    // new index i: i < p1 old i; p1 <= i < p2 - 1 old i+1; else old i+2. Chunks from the bottom.
    const int Kn = d.w;
    for (int base = 0; base < Kn; base += 32) {
      const int i = base + lane;
      double t = 0.0;
      int g = 0, h = 0;
      if (i < Kn) {
        const int src = i < d.y ? i : (i < d.z - 1 ? i + 1 : i + 2);
        t = tau[src]; g = fl[src]; h = dg[src];
      }
      __syncwarp();
      if (i < Kn) { tau[i] = t; fl[i] = (uint8_t)g; dg[i] = (uint8_t)h; }
      __syncwarp();
    }
  }
  // 2. the inverse bath matrix of flavor f
  const size_t fb = (size_t)w * nf + f;
  const int kc = S.kcap;
  double *Mf = S.M + fb * kc * kc;
  double *rt = S.row_t + fb * kc, *ct = S.col_t + fb * kc;
  const int k = S.kf[fb];
  if (kind == 0) {
    const double lam = S.p_lambda[w], il = 1.0 / lam;
    const double *mc = S.p_vec + (size_t)w * 2 * kc, *rm = mc + kc;
    for (int e = lane; e < k * k; e += 32) {
      const int j = e / k, i = e - j * k;
      Mf[(size_t)j * kc + i] = fma(mc[j] * il, rm[i], Mf[(size_t)j * kc + i]);
    }
    for (int e = lane; e < k; e += 32) {
      Mf[(size_t)e * kc + k] = -mc[e] * il;   // new creator column
      Mf[(size_t)k * kc + e] = -rm[e] * il;   // new annihilator row
    }
    if (lane == 0) {
      Mf[(size_t)k * kc + k] = il;
      rt[k] = S.mv_tdag[w];
      ct[k] = S.mv_tann[w];
      S.kf[fb] = k + 1;
    }
  } else {
    const int i = S.p_ij[2 * w], j = S.p_ij[2 * w + 1], L = k - 1;
    // creator i <-> L: columns of M; annihilator j <-> L: rows of M
    if (i != L)
      for (int r = lane; r < k; r += 32) {
        const double x = Mf[(size_t)r * kc + i];
        Mf[(size_t)r * kc + i] = Mf[(size_t)r * kc + L];
        Mf[(size_t)r * kc + L] = x;
      }
    __syncwarp();
    if (j != L)
      for (int c = lane; c < k; c += 32) {
        const double x = Mf[(size_t)j * kc + c];
        Mf[(size_t)j * kc + c] = Mf[(size_t)L * kc + c];
        Mf[(size_t)L * kc + c] = x;
      }
    __syncwarp();
    const double is = 1.0 / Mf[(size_t)L * kc + L];
    for (int e = lane; e < L * L; e += 32) {
      const int r = e / L, c = e - r * L;
      Mf[(size_t)r * kc + c] -= Mf[(size_t)r * kc + L] * Mf[(size_t)L * kc + c] * is;
    }
    if (lane == 0) {
      rt[i] = rt[L];
      ct[j] = ct[L];
      S.kf[fb] = L;
    }
  }
  if (lane == 0) {
    S.lens[w] = d.w;
    S.tr_sign[w] = (int8_t)(tsg * S.tr_sign[w]);
    S.tr_log[w] += S.r_log[w];
    S.w_sign[w] = (int8_t)(S.w_sign[w] * tsg * S.p_sign[w]);
    S.det_log[w] += S.p_ldet[w];
    atomicAdd(&S.counters[kind == 0 ? C_INS_ACC : C_REM_ACC], 1ull);
  }
}

// Feature vector of each proposal (see kt_sweep_feature_size): the configuration without
// the move's pair (the base) and the pair. A removal's base skips the pair's operators.
__global__ void sweep_features_kernel(SweepView S0, TryView Tv) {
  extern __shared__ float hsm[];
  const SweepView S = Tv.T ? try_view(S0, Tv, blockIdx.y) : S0;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int w = blockIdx.x * (blockDim.x >> 5) + wib;
  if (w >= S.nw) return;
  const int nf = S.nf;
  const double beta = S.beta;
  // per warp: nf x 32 histogram bins (float), then nf occupied lengths (double)
  float *hist = hsm + (size_t)wib * nf * 34;
  double *occ = reinterpret_cast<double *>(hist + nf * 32);
  for (int i = lane; i < nf * 32; i += 32) hist[i] = 0.f;
  for (int i = lane; i < nf; i += 32) occ[i] = 0.0;
  __syncwarp();
  const double m0 = S.p_t1[w];
  double md = S.p_t2[w] - m0;
  if (md < 0.0) md += beta;
  const int o = S.offsets[w], K = S.lens[w];
  const double *tau = S.tau + o;
  const uint8_t *fl = S.flv + o, *dg = S.dag + o;
  const int pa = S.p_pair[2 * w], pb = S.p_pair[2 * w + 1];
  for (int i = lane; i < K; i += 32) {
    if (dg[i] != 1 || i == pa || i == pb) continue;
    const int f = fl[i];
    int j = -1;
    for (int s2 = 1; s2 < K; ++s2) {
      const int c = i + s2 < K ? i + s2 : i + s2 - K;
      if (fl[c] == f && c != pa && c != pb) {
        j = c;
        break;
      }
    }
    if (j < 0) continue;
    const double l = tau[j] > tau[i] ? tau[j] - tau[i] : tau[j] + beta - tau[i];
    int b = (int)(l / beta * 32);
    b = b > 31 ? 31 : b;
    atomicAdd(&hist[f * 32 + b], 0.25f);
    // overlap of the segment [tau_i, tau_i + l) with the pair's interval [m0, m0 + md), cyclically
    double ov = 0.0;
    for (int k = -1; k <= 1; ++k) {
      const double lo = fmax(tau[i], m0 + k * beta), hi = fmin(tau[i] + l, m0 + md + k * beta);
      ov += fmax(0.0, hi - lo);
    }
    if (ov > 0.0) atomicAdd(&occ[f], ov);
  }
  __syncwarp();
  __nv_bfloat16 *row = S.X + (size_t)w * S.n_in;
  const int fm = S.mv_flv[w];
  for (int i = lane; i < S.n_in; i += 32) {
    float x = 0.f;
    if (i < nf) {
      x = (float)(S.kf[(size_t)w * nf + i] - (pa >= 0 && i == fm ? 1 : 0)) / 8.f;
    } else if (i < 33 * nf) {
      x = hist[i - nf];
    } else if (i == 33 * nf) {
      x = 0.f;
    } else if (i <= 34 * nf) {
      x = (i - 33 * nf - 1 == fm) ? 1.f : 0.f;
    } else if (i == 34 * nf + 1) {
      double d = S.p_t2[w] - S.p_t1[w];
      if (d < 0.0) d += beta;
      x = (float)(d / beta);
    } else if (i == 34 * nf + 2) {
      x = S.p_seg[w] ? 1.f : -1.f;
    } else if (i < 35 * nf + 3) {
      x = md > 0.0 ? (float)(occ[i - 34 * nf - 3] / md) : 0.f;
    }
    row[i] = __float2bfloat16_rn(x);
  }
}

// Multi-try delayed acceptance, before the features: for every operator i of a walker, the
// next operator of the same flavor after it, cyclically (-1 if i is its flavor's only one),
// one warp per walker. The tries of a call step share the configuration, so this table is
// built once and every try's features take O(K) instead of O(K^2 / n_flavors).
__global__ void sweep_next_flavor_kernel(SweepView S, TryView Tv) {
  const int lane = threadIdx.x & 31;
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (w >= S.nw) return;
  const int o = S.offsets[w], K = S.lens[w];
  const uint8_t *fl = S.flv + o;
  int16_t *nxt = Tv.nxt + (size_t)w * S.cap;
  for (int i = lane; i < K; i += 32) {
    const int f = fl[i];
    int j = -1;
    for (int s2 = 1; s2 < K; ++s2) {
      const int c = i + s2 < K ? i + s2 : i + s2 - K;
      if (fl[c] == f) {
        j = c;
        break;
      }
    }
    nxt[i] = (int16_t)j;
  }
}

// Features of the tries (one warp per walker and try), with the values of
// sweep_features_kernel: a removal try's base skips its own pair by following the walker's
// next-same-flavor table past the pair's two operators.
__global__ void sweep_features_multi_kernel(SweepView S, TryView Tv) {
  extern __shared__ float hsm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int w = blockIdx.x * (blockDim.x >> 5) + wib;
  if (w >= S.nw) return;
  const int nf = S.nf;
  const double beta = S.beta;
  const size_t sl = (size_t)blockIdx.y * S.nw + w;
  float *hist = hsm + (size_t)wib * nf * 34;
  double *occ = reinterpret_cast<double *>(hist + nf * 32);
  for (int i = lane; i < nf * 32; i += 32) hist[i] = 0.f;
  for (int i = lane; i < nf; i += 32) occ[i] = 0.0;
  __syncwarp();
  const double m0 = Tv.p_t1[sl];
  double md = Tv.p_t2[sl] - m0;
  if (md < 0.0) md += beta;
  const int o = S.offsets[w], K = S.lens[w];
  const double *tau = S.tau + o;
  const uint8_t *fl = S.flv + o, *dg = S.dag + o;
  const int16_t *nxt = Tv.nxt + (size_t)w * S.cap;
  const int pa = Tv.p_pair[2 * sl], pb = Tv.p_pair[2 * sl + 1];
  for (int i = lane; i < K; i += 32) {
    if (dg[i] != 1 || i == pa || i == pb) continue;
    const int f = fl[i];
    int j = nxt[i];
    while (j >= 0 && (j == pa || j == pb)) j = nxt[j];
    if (j == i) j = -1;
    if (j < 0) continue;
    const double ti = tau[i], tj = tau[j];
    const double l = tj > ti ? tj - ti : tj + beta - ti;
    int b = (int)(l / beta * 32);
    b = b > 31 ? 31 : b;
    atomicAdd(&hist[f * 32 + b], 0.25f);
    double ov = 0.0;
    for (int k = -1; k <= 1; ++k) {
      const double lo = fmax(ti, m0 + k * beta), hi = fmin(ti + l, m0 + md + k * beta);
      ov += fmax(0.0, hi - lo);
    }
    if (ov > 0.0) atomicAdd(&occ[f], ov);
  }
  __syncwarp();
  __nv_bfloat16 *row = Tv.X + sl * S.n_in;
  const int fm = Tv.mv_flv[sl];
  for (int i = lane; i < S.n_in; i += 32) {
    float x = 0.f;
    if (i < nf) {
      x = (float)(S.kf[(size_t)w * nf + i] - (pa >= 0 && i == fm ? 1 : 0)) / 8.f;
    } else if (i < 33 * nf) {
      x = hist[i - nf];
    } else if (i == 33 * nf) {
      x = 0.f;
    } else if (i <= 34 * nf) {
      x = (i - 33 * nf - 1 == fm) ? 1.f : 0.f;
    } else if (i == 34 * nf + 1) {
      x = (float)(md / beta);
    } else if (i == 34 * nf + 2) {
      x = Tv.p_seg[sl] ? 1.f : -1.f;
    } else if (i < 35 * nf + 3) {
      x = md > 0.0 ? (float)(occ[i - 34 * nf - 3] / md) : 0.f;
    }
    row[i] = __float2bfloat16_rn(x);
  }
}

// Stage 1 of delayed acceptance: the surrogate's ratio decides whether the trace is computed.
// The network predicts the insertion of the pair into the base; a removal takes minus
// that, so a move and its reverse get opposite predictions (antisymmetric surrogate).
__global__ void sweep_stage1_kernel(SweepView S, const double *__restrict__ uni) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= S.nw) return;
  if (S.p_kind[w] != 0) S.ytil[w] = -S.ytil[w];
  if (!S.p_valid[w]) return;
  const double lt = (double)S.ytil[w] + S.p_ldet[w] + S.p_lprop[w];
  const double u6 = uni[(size_t)w * 7 + 6];
  if (!((u6 > 0.0 ? log(u6) : -INFINITY) < lt)) {
    S.p_valid[w] = 0;
    S.mv_kind[w] = 2;  // skipped by the trace pipeline (rejected by its validation without work)
    atomicAdd(&S.counters[C_STAGE1], 1ull);
  }
}

// Stage 1 over the tries in order (one warp per walker): the first try that passes becomes
// the step's move, copied into the walker's proposal arrays for the trace pipeline and the
// accept kernel. Every try before it is a Metropolis step that leaves the configuration as
// it is (rejected at stage 1, or a null move); the tries after it are never taken. A walker
// none of whose tries passes keeps its configuration for T steps. Counters of the tries taken.
__global__ void sweep_select_kernel(SweepView S, TryView Tv, const double *__restrict__ uni) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= S.nw) return;
  const int nw = S.nw, T = Tv.T;
  int sel = -1;
  float ysel = 0.f;
  if (lane == 0) {
    unsigned long long c_ins = 0, c_rem = 0, c_null = 0, c_cap = 0, c_st1 = 0;
    for (int t = 0; t < T; ++t) {
      const size_t sl = (size_t)t * nw + w;
      const int kind = Tv.p_kind[sl];
      if (kind == 0) ++c_ins;
      else ++c_rem;
      if (!Tv.p_valid[sl]) {
        ++c_null;
        if (kind == 0 && S.kf[(size_t)w * S.nf + Tv.mv_flv[sl]] >= S.kcap) ++c_cap;
        continue;
      }
      const float y = kind != 0 ? -Tv.ytil[sl] : Tv.ytil[sl];
      const double lt = (double)y + Tv.p_ldet[sl] + Tv.p_lprop[sl];
      const double u6 = uni[((size_t)w * T + t) * 7 + 6];
      if ((u6 > 0.0 ? log(u6) : -INFINITY) < lt) {
        sel = t;
        ysel = y;
        break;
      }
      ++c_st1;
    }
    Tv.n_tries[w] = sel < 0 ? T : sel + 1;
    S.p_acc[w] = 0;
    if (c_ins) atomicAdd(&S.counters[C_INS_PROP], c_ins);
    if (c_rem) atomicAdd(&S.counters[C_REM_PROP], c_rem);
    if (c_null) atomicAdd(&S.counters[C_NULL], c_null);
    if (c_cap) atomicAdd(&S.counters[C_CAP], c_cap);
    if (c_st1) atomicAdd(&S.counters[C_STAGE1], c_st1);
  }
  sel = __shfl_sync(FULL, sel, 0);
  if (sel < 0) {
    if (lane == 0) {
      S.p_valid[w] = 0;
      S.mv_kind[w] = 2;  // skipped by the trace pipeline
    }
    return;
  }
  const size_t sl = (size_t)sel * nw + w;
  if (lane == 0) {
    S.p_kind[w] = Tv.p_kind[sl];
    S.p_t1[w] = Tv.p_t1[sl];
    S.p_t2[w] = Tv.p_t2[sl];
    S.p_seg[w] = Tv.p_seg[sl];
    S.p_pair[2 * w] = Tv.p_pair[2 * sl];
    S.p_pair[2 * w + 1] = Tv.p_pair[2 * sl + 1];
    S.mv_kind[w] = Tv.mv_kind[sl];
    S.mv_flv[w] = Tv.mv_flv[sl];
    S.mv_tdag[w] = Tv.mv_tdag[sl];
    S.mv_tann[w] = Tv.mv_tann[sl];
    S.mv_rem[w] = Tv.mv_rem[sl];
    S.p_valid[w] = 1;
    S.p_sign[w] = Tv.p_sign[sl];
    S.p_lprop[w] = Tv.p_lprop[sl];
    S.p_ldet[w] = Tv.p_ldet[sl];
    S.p_lambda[w] = Tv.p_lambda[sl];
    S.p_ij[2 * w] = Tv.p_ij[2 * sl];
    S.p_ij[2 * w + 1] = Tv.p_ij[2 * sl + 1];
    S.ytil[w] = ysel;
    Tv.u5[w] = uni[((size_t)w * T + sel) * 7 + 5];
  }
  if (Tv.p_kind[sl] == 0) {
    const double *src = Tv.p_vec + sl * 2 * S.kcap;
    double *dst = S.p_vec + (size_t)w * 2 * S.kcap;
    for (int i = lane; i < 2 * S.kcap; i += 32) dst[i] = src[i];
  }
}

// Training data: features and the insertion log trace ratio of every evaluated nonzero
// ratio (log|T_new / T_old| for an insertion, its negative for a removal).
__global__ void sweep_record_kernel(SweepView S, __nv_bfloat16 *feat, float *targ, int *count, int cap) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= S.nw) return;
  if (!S.p_valid[w] || S.r_status[w] != KT_OK || S.r_sign[w] == 0) return;
  int slot = 0;
  if (lane == 0) slot = atomicAdd(count, 1);
  slot = __shfl_sync(FULL, slot, 0);
  if (slot >= cap) return;
  const __nv_bfloat16 *src = S.X + (size_t)w * S.n_in;
  __nv_bfloat16 *dst = feat + (size_t)slot * S.n_in;
  for (int i = lane; i < S.n_in; i += 32) dst[i] = src[i];
  if (lane == 0) targ[slot] = (float)(S.p_kind[w] == 0 ? S.r_log[w] : -S.r_log[w]);
}

// wt: per-walker weight of the measurement (NULL: 1), the Metropolis steps the walker spends
// in the measured configuration in multi-try delayed acceptance
__global__ void sweep_measure_kernel(SweepView S, const int32_t *__restrict__ wt) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= S.nw) return;
  const double s = (double)S.w_sign[w] * (wt ? (double)wt[w] : 1.0);
  const int nf = S.nf, kc = S.kcap, nb = S.n_bins;
  const double beta = S.beta;
  if (lane == 0) {
    S.sign_sum[w] += s;
    if (w == 0) atomicAdd(&S.counters[C_MEAS], 1ull);
  }
  for (int f = 0; f < nf; ++f) {
    const size_t fb = (size_t)w * nf + f;
    const int k = S.kf[fb];
    if (lane == 0) S.order_sum[fb] += s * k;
    const double *Mf = S.M + fb * kc * kc;
    const double *rt = S.row_t + fb * kc, *ct = S.col_t + fb * kc;
    double *g = S.g_acc + fb * nb;
    for (int e = lane; e < k * k; e += 32) {
      const int j = e / k, i = e - j * k;
      double x = ct[j] - rt[i], v = Mf[(size_t)j * kc + i];
      if (x < 0.0) {
        x += beta;
        v = -v;
      }
      int b = (int)(x / beta * nb);
      b = b > nb - 1 ? nb - 1 : (b < 0 ? 0 : b);
      atomicAdd(g + b, s * v);
    }
  }
}

__global__ void sweep_obs_accumulate_kernel(SweepView S, const int32_t *__restrict__ wt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= S.nw * S.nobs) return;
  const int w = t / S.nobs;
  const double v = S.obs_tmp[t];
  if (isfinite(v)) S.obs_sum[t] += (double)S.w_sign[w] * (wt ? (double)wt[w] : 1.0) * v;
}

// Refresh, step 1 (one warp per (walker, flavor)): G_f[i][j] = Fh_f(tau'_i - tau_j) over the
// stored creator and annihilator times, built in the slot of M and inverted there by
// Gauss-Jordan elimination with partial pivoting in FP64 (a lane owns whole rows, so every
// row update reads only the finished pivot row); log|det G_f| and its sign are recorded.
// The inverse keeps M's layout: M[j][i] = (G_f^{-1})_{ji}, rows indexed by annihilators.
__global__ void sweep_refresh_det_kernel(SweepView S) {
  extern __shared__ int piv_sh[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int wf = blockIdx.x * (blockDim.x >> 5) + wib;
  if (wf >= S.nw * S.nf) return;
  const int f = wf % S.nf, kc = S.kcap, k = S.kf[wf];
  int *perm = piv_sh + wib * kc;
  double *A = S.M + (size_t)wf * kc * kc;
  const double *rt = S.row_t + (size_t)wf * kc, *ct = S.col_t + (size_t)wf * kc;
  for (int idx = lane; idx < k * k; idx += 32) {
    const int i = idx / k, j = idx - i * k;
    A[(size_t)i * kc + j] = hyb_Fh(S, f, rt[i] - ct[j]);
  }
  __syncwarp();
  double ld = 0.0;
  int sg = 1;
  for (int c = 0; c < k && sg != 0; ++c) {
    double best = -1.0;
    int pr = c;
    for (int r = c + lane; r < k; r += 32) {
      const double a = fabs(A[(size_t)r * kc + c]);
      if (a > best) {
        best = a;
        pr = r;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(FULL, best, o);
      const int opr = __shfl_xor_sync(FULL, pr, o);
      if (ob > best || (ob == best && opr < pr)) {
        best = ob;
        pr = opr;
      }
    }
    if (!(best > 0.0) || !isfinite(best)) {
      sg = 0;
      break;
    }
    if (lane == 0) perm[c] = pr;
    if (pr != c) {
      for (int j = lane; j < k; j += 32) {
        const double t = A[(size_t)c * kc + j];
        A[(size_t)c * kc + j] = A[(size_t)pr * kc + j];
        A[(size_t)pr * kc + j] = t;
      }
      sg = -sg;
    }
    __syncwarp();
    const double pv = A[(size_t)c * kc + c];
    ld += log(fabs(pv));
    if (pv < 0.0) sg = -sg;
    const double inv = 1.0 / pv;
    __syncwarp();
    for (int j = lane; j < k; j += 32) A[(size_t)c * kc + j] = (j == c) ? inv : A[(size_t)c * kc + j] * inv;
    __syncwarp();
    for (int r = lane; r < k; r += 32) {
      if (r == c) continue;
      double *Ar = A + (size_t)r * kc;
      const double fct = Ar[c];
      if (fct == 0.0) continue;
      const double *Ac = A + (size_t)c * kc;
      for (int j = 0; j < k; ++j) Ar[j] = (j == c) ? -fct * Ac[c] : fma(-fct, Ac[j], Ar[j]);
    }
    __syncwarp();
  }
  if (sg != 0) {
    // the row interchanges of the elimination become column interchanges of the inverse
    for (int c = k - 1; c >= 0; --c) {
      const int pr = perm[c];
      if (pr == c) continue;
      for (int r = lane; r < k; r += 32) {
        const double t = A[(size_t)r * kc + c];
        A[(size_t)r * kc + c] = A[(size_t)r * kc + pr];
        A[(size_t)r * kc + pr] = t;
      }
      __syncwarp();
    }
  }
  if (lane == 0) {
    S.f_detlog[wf] = ld;
    S.f_detsign[wf] = (int8_t)sg;
  }
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v) {
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// Refresh, step 2 (one warp per walker): the sign s_P of the bath permutation counted from
// scratch (the bath operators flavor by flavor in storage order, tau'_1 tau_1 tau'_2 tau_2 ...,
// against descending time), the recomputed determinants and trace replace the tracked ones,
// and the deviations of the tracked values are recorded. A walker whose fresh evaluation
// failed (a singular G_f or a trace error) keeps its tracked values.
__global__ void sweep_refresh_apply_kernel(SweepView S) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= S.nw) return;
  const int nf = S.nf, kc = S.kcap;
  // operator a of the flavor-by-flavor sequence: flavor block, pair index, creator or annihilator
  int total = 0;
  for (int f = 0; f < nf; ++f) total += 2 * S.kf[w * nf + f];
  auto op_time = [&](int a) {
    int f = 0;
    while (a >= 2 * S.kf[w * nf + f]) {
      a -= 2 * S.kf[w * nf + f];
      ++f;
    }
    const size_t b = ((size_t)w * nf + f) * kc + (a >> 1);
    return (a & 1) ? S.col_t[b] : S.row_t[b];
  };
  long long inv = 0;
  for (int a = lane; a < total; a += 32) {
    const double ta = op_time(a);
    for (int c = a + 1; c < total; ++c) inv += ta < op_time(c);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) inv += __shfl_xor_sync(FULL, inv, o);
  if (lane != 0) return;
  double dl = 0.0;
  int ds = 1;
  for (int f = 0; f < nf; ++f) {
    if (S.kf[w * nf + f] == 0) continue;
    dl += S.f_detlog[w * nf + f];
    ds *= S.f_detsign[w * nf + f];
  }
  const int ts = S.f_tsign[w];
  if (ds == 0 || ts == 0 || S.f_tstat[w] != KT_OK) {
    atomicAdd(&S.f_dev[3], 1ull);
    return;
  }
  const int sp = (inv & 1) ? -1 : 1;
  const int ws = ts * sp * ds;
  if (ws != S.w_sign[w] || ts != S.tr_sign[w]) atomicAdd(&S.f_dev[2], 1ull);
  atomic_max_nonneg(&S.f_dev[0], fabs(S.tr_log[w] - S.f_tlog[w]));
  atomic_max_nonneg(&S.f_dev[1], fabs(S.det_log[w] - dl));
  S.tr_sign[w] = (int8_t)ts;
  S.tr_log[w] = S.f_tlog[w];
  S.det_log[w] = dl;
  S.w_sign[w] = (int8_t)ws;
}

__global__ void sweep_init_kernel(SweepView S, const int8_t *sg, const double *lg) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= S.nw) return;
  S.tr_sign[w] = sg[w];
  S.tr_log[w] = lg[w];
  S.w_sign[w] = sg[w];
  S.det_log[w] = 0.0;
}

template <typename T>
__global__ void gather_padded_kernel(const T *src, T *dst, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = src[t];
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace kt

struct kt_sweep {
  kt_model *model = nullptr;
  kt::ModelView mv{};
  kt::SweepView v{};
  void *mem = nullptr;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  bool measure_obs = false;
  std::vector<double> hyb_host;
  kt_mlp *net = nullptr;
  kt::CacheView cache{};  // partial-state cache (cache.P == 0: off)
  kt_stats *stats = nullptr;  // device counters of the trace pipeline (kt_sweep_set_stats)
  void *cache_mem = nullptr;
  int cache_words = 0;    // 32-bit words per cached vector
  void *try_mem = nullptr;  // proposal slots of multi-try delayed acceptance
  kt::TryView tv{};         // tv.T == 0: not allocated
};

namespace {

// dry != NULL: only the size of the allocation, in *dry.
kt_status carve_and_alloc(kt_sweep *s, size_t *dry = nullptr) {
  kt::SweepView &v = s->v;
  const size_t nw = v.nw, nf = v.nf, kc = v.kcap, cap = v.cap;
  size_t b = 0;
  auto take = [&](size_t bytes) {
    const size_t at = b;
    b += kt::up256(bytes);
    return at;
  };
  const size_t o_off = take((nw + 1) * 4), o_len = take(nw * 4), o_tau = take(nw * cap * 8), o_flv = take(nw * cap),
               o_dag = take(nw * cap), o_kf = take(nw * nf * 4), o_rt = take(nw * nf * kc * 8),
               o_ct = take(nw * nf * kc * 8), o_M = take(nw * nf * kc * kc * 8), o_hyb = take(nf * (v.n_tau + 1) * 8),
               o_trs = take(nw), o_trl = take(nw * 8), o_ws = take(nw), o_dl = take(nw * 8), o_mk = take(nw),
               o_mf = take(nw), o_md = take(nw * 8), o_ma = take(nw * 8), o_mr = take(nw * 4), o_pv = take(nw),
               o_ps = take(nw), o_plp = take(nw * 8), o_pld = take(nw * 8), o_plam = take(nw * 8),
               o_pij = take(nw * 2 * 4), o_pvec = take(nw * 2 * kc * 8), o_rs = take(nw), o_rl = take(nw * 8),
               o_rst = take(nw * 4), o_g = take(nw * nf * v.n_bins * 8), o_ss = take(nw * 8), o_os = take(nw * nf * 8),
               o_obs = take(nw * v.nobs * 8), o_obt = take(nw * v.nobs * 8), o_msg = take(nw), o_mlg = take(nw * 8),
               o_mst = take(nw * 4), o_cnt = take(KT_SWEEP_NCOUNTERS * 8), o_pk = take(nw), o_pt1 = take(nw * 8),
               o_pt2 = take(nw * 8), o_pseg = take(nw), o_X = take(nw * (size_t)v.n_in * 2), o_yt = take(nw * 4),
               o_ppair = take(nw * 2 * 4), o_pacc = take(nw), o_fdl = take(nw * nf * 8), o_fds = take(nw * nf),
               o_fts = take(nw), o_ftl = take(nw * 8), o_fst = take(nw * 4), o_fdev = take(4 * 8);
  if (dry) {
    *dry = b;
    return KT_OK;
  }
  if (cudaMalloc(&s->mem, b) != cudaSuccess) {
    cudaGetLastError();
    s->mem = nullptr;
    return KT_ENOMEM;
  }
  if (cudaMemset(s->mem, 0, b) != cudaSuccess) return KT_ECUDA;
  char *p = (char *)s->mem;
  v.offsets = (int32_t *)(p + o_off);
  v.lens = (int32_t *)(p + o_len);
  v.tau = (double *)(p + o_tau);
  v.flv = (uint8_t *)(p + o_flv);
  v.dag = (uint8_t *)(p + o_dag);
  v.kf = (int32_t *)(p + o_kf);
  v.row_t = (double *)(p + o_rt);
  v.col_t = (double *)(p + o_ct);
  v.M = (double *)(p + o_M);
  v.hyb = (const double *)(p + o_hyb);
  v.tr_sign = (int8_t *)(p + o_trs);
  v.tr_log = (double *)(p + o_trl);
  v.w_sign = (int8_t *)(p + o_ws);
  v.det_log = (double *)(p + o_dl);
  v.mv_kind = (uint8_t *)(p + o_mk);
  v.mv_flv = (uint8_t *)(p + o_mf);
  v.mv_tdag = (double *)(p + o_md);
  v.mv_tann = (double *)(p + o_ma);
  v.mv_rem = (int32_t *)(p + o_mr);
  v.p_valid = (int8_t *)(p + o_pv);
  v.p_sign = (int8_t *)(p + o_ps);
  v.p_lprop = (double *)(p + o_plp);
  v.p_ldet = (double *)(p + o_pld);
  v.p_lambda = (double *)(p + o_plam);
  v.p_ij = (int32_t *)(p + o_pij);
  v.p_vec = (double *)(p + o_pvec);
  v.r_sign = (int8_t *)(p + o_rs);
  v.r_log = (double *)(p + o_rl);
  v.r_status = (int32_t *)(p + o_rst);
  v.g_acc = (double *)(p + o_g);
  v.sign_sum = (double *)(p + o_ss);
  v.order_sum = (double *)(p + o_os);
  v.obs_sum = (double *)(p + o_obs);
  v.obs_tmp = (double *)(p + o_obt);
  v.m_sign = (int8_t *)(p + o_msg);
  v.m_log = (double *)(p + o_mlg);
  v.m_status = (int32_t *)(p + o_mst);
  v.counters = (unsigned long long *)(p + o_cnt);
  v.p_kind = (int8_t *)(p + o_pk);
  v.p_t1 = (double *)(p + o_pt1);
  v.p_t2 = (double *)(p + o_pt2);
  v.p_seg = (int8_t *)(p + o_pseg);
  v.X = (__nv_bfloat16 *)(p + o_X);
  v.ytil = (float *)(p + o_yt);
  v.p_pair = (int32_t *)(p + o_ppair);
  v.p_acc = (int8_t *)(p + o_pacc);
  v.f_detlog = (double *)(p + o_fdl);
  v.f_detsign = (int8_t *)(p + o_fds);
  v.f_tsign = (int8_t *)(p + o_fts);
  v.f_tlog = (double *)(p + o_ftl);
  v.f_tstat = (int32_t *)(p + o_fst);
  v.f_dev = (unsigned long long *)(p + o_fdev);
  return KT_OK;
}

// The partial-state cache: P + 1 slots per direction for every (walker, kept state)
// item, cache and scratch, plus the valid ranges and the per-step plan.
kt_status alloc_cache(kt_sweep *s, int P, size_t *dry = nullptr) {
  const kt::DevModel &M = *s->mv.dev;
  const size_t items = (size_t)s->v.nw * M.n_kept, slots = items * ((size_t)P + 1);
  const size_t esz = s->mv.precision == KT_FP64 ? 8 : 4, dv = (size_t)M.d_max;
  size_t b = 0;
  auto take = [&](size_t bytes) {
    const size_t at = b;
    b += kt::up256(bytes);
    return at;
  };
  size_t o_vec[4], o_log[4], o_blk[4];
  for (int k = 0; k < 4; ++k) {
    o_vec[k] = take(slots * dv * esz);
    o_log[k] = take(slots * 16);
    o_blk[k] = take(slots * 4);
  }
  const size_t o_f = take(items * 4), o_gr = take(items * 4), o_plan = take(items * 16);
  if (dry) {
    *dry = b;
    return KT_OK;
  }
  if (cudaMalloc(&s->cache_mem, b) != cudaSuccess) {
    cudaGetLastError();
    s->cache_mem = nullptr;
    return KT_ENOMEM;
  }
  char *p = (char *)s->cache_mem;
  kt::CacheView &C = s->cache;
  C.P = P;
  C.dv = (int)dv;
  C.fvec = p + o_vec[0];
  C.bvec = p + o_vec[1];
  C.sfvec = p + o_vec[2];
  C.sbvec = p + o_vec[3];
  C.flog = (double2 *)(p + o_log[0]);
  C.blog = (double2 *)(p + o_log[1]);
  C.sflog = (double2 *)(p + o_log[2]);
  C.sblog = (double2 *)(p + o_log[3]);
  C.fblk = (int32_t *)(p + o_blk[0]);
  C.bblk = (int32_t *)(p + o_blk[1]);
  C.sfblk = (int32_t *)(p + o_blk[2]);
  C.sbblk = (int32_t *)(p + o_blk[3]);
  C.f = (int32_t *)(p + o_f);
  C.gr = (int32_t *)(p + o_gr);
  C.plan = (int4 *)(p + o_plan);
  s->cache_words = (int)(dv * esz / 4);
  return cudaMemset(s->cache_mem, 0, b) == cudaSuccess ? KT_OK : KT_ECUDA;
}

// Nothing cached is valid for new configurations.
kt_status invalidate_cache(kt_sweep *s) {
  if (!s->cache_mem) return KT_OK;
  const size_t items = (size_t)s->v.nw * s->mv.dev->n_kept;
  if (cudaMemset(s->cache.f, 0, items * 4) != cudaSuccess || cudaMemset(s->cache.gr, 0, items * 4) != cudaSuccess)
    return KT_ECUDA;
  return KT_OK;
}

kt::SeqView seq_view(const kt_sweep *s) {
  kt::SeqView sv{s->v.nw, s->v.offsets, s->v.tau, s->v.flv, s->v.dag};
  sv.lens = s->v.lens;
  sv.trusted = true;  // validated by kt_sweep_set_configs and edited only by the sweep's kernels
  return sv;
}

// the trace pipeline on the current configurations, with the observables at beta/2 when obs != nullptr
int current_traces(kt_sweep *s, int8_t *sg, double *lg, int32_t *st, double *obs, cudaStream_t stream) {
  const kt::DevModel &M = *s->mv.dev;
  const kt::Workspace w = kt::carve_workspace(s->ws, s->v.nw, M.n_kept, M.d_max, obs ? M.nf + M.n_orb + 1 : 0);
  // measurements of a cached sweep start from the cached states nearest to beta/2
  if (obs && s->cache_mem)
    return kt::launch_cached_measure(M, s->mv.precision, s->mv.kernel_dmax, seq_view(s), sg, lg, st, obs, w, s->cache,
                                     stream);
  return kt::launch_pipeline(M, s->mv.precision, s->mv.kernel_dmax, s->mv.group_lanes, seq_view(s), nullptr, nullptr,
                             nullptr, sg, lg, st, nullptr, w, stream, nullptr, obs);
}

// Proposal slots for T tries per walker (kt_sweep_run_da_multi); grown on demand.
kt_status alloc_tries(kt_sweep *s, int T, size_t *dry = nullptr) {
  if (!dry && s->tv.T >= T) return KT_OK;
  if (!dry && s->try_mem) {
    cudaFree(s->try_mem);
    s->try_mem = nullptr;
    s->tv = kt::TryView{};
  }
  const size_t n = (size_t)T * s->v.nw, kc = s->v.kcap, nw = s->v.nw;
  size_t b = 0;
  auto take = [&](size_t bytes) {
    const size_t at = b;
    b += kt::up256(bytes);
    return at;
  };
  const size_t o_kind = take(n), o_seg = take(n), o_valid = take(n), o_sign = take(n), o_acc = take(n),
               o_t1 = take(n * 8), o_t2 = take(n * 8), o_td = take(n * 8), o_ta = take(n * 8), o_lp = take(n * 8),
               o_ld = take(n * 8), o_lam = take(n * 8), o_vec = take(n * 2 * kc * 8), o_pair = take(n * 2 * 4),
               o_rem = take(n * 4), o_ij = take(n * 2 * 4), o_mk = take(n), o_mf = take(n),
               o_X = take(n * (size_t)s->v.n_in * 2), o_y = take(n * 4), o_cnt = take(KT_SWEEP_NCOUNTERS * 8),
               o_nt = take(nw * 4), o_u5 = take(nw * 8), o_nxt = take(nw * (size_t)s->v.cap * 2);
  if (dry) {
    *dry = b;
    return KT_OK;
  }
  if (cudaMalloc(&s->try_mem, b) != cudaSuccess) {
    cudaGetLastError();
    s->try_mem = nullptr;
    return KT_ENOMEM;
  }
  if (cudaMemset(s->try_mem, 0, b) != cudaSuccess) return KT_ECUDA;
  char *p = (char *)s->try_mem;
  kt::TryView &t = s->tv;
  t.p_kind = (int8_t *)(p + o_kind); t.p_seg = (int8_t *)(p + o_seg); t.p_valid = (int8_t *)(p + o_valid);
  t.p_sign = (int8_t *)(p + o_sign); t.p_acc = (int8_t *)(p + o_acc);
  t.p_t1 = (double *)(p + o_t1); t.p_t2 = (double *)(p + o_t2); t.mv_tdag = (double *)(p + o_td);
  t.mv_tann = (double *)(p + o_ta); t.p_lprop = (double *)(p + o_lp); t.p_ldet = (double *)(p + o_ld);
  t.p_lambda = (double *)(p + o_lam); t.p_vec = (double *)(p + o_vec); t.p_pair = (int32_t *)(p + o_pair);
  t.mv_rem = (int32_t *)(p + o_rem); t.p_ij = (int32_t *)(p + o_ij); t.mv_kind = (uint8_t *)(p + o_mk);
  t.mv_flv = (uint8_t *)(p + o_mf); t.X = (__nv_bfloat16 *)(p + o_X); t.ytil = (float *)(p + o_y);
  t.scratch_counters = (unsigned long long *)(p + o_cnt); t.n_tries = (int32_t *)(p + o_nt);
  t.u5 = (double *)(p + o_u5);
  t.nxt = (int16_t *)(p + o_nxt);
  t.T = T;
  return KT_OK;
}

// Every walker to the empty configuration: weight = trace of the empty sequence.
kt_status reset_empty(kt_sweep *s) {
  kt::SweepView &v = s->v;
  const size_t nw = v.nw, nf = v.nf;
  if (cudaMemset(v.lens, 0, nw * 4) != cudaSuccess || cudaMemset(v.kf, 0, nw * nf * 4) != cudaSuccess) return KT_ECUDA;
  if (invalidate_cache(s) != KT_OK) return KT_ECUDA;
  if (current_traces(s, v.m_sign, v.m_log, v.m_status, nullptr, 0) != 0) return KT_ECUDA;
  kt::sweep_init_kernel<<<(v.nw + 255) / 256, 256>>>(v, v.m_sign, v.m_log);
  return cudaDeviceSynchronize() == cudaSuccess ? KT_OK : KT_ECUDA;
}

// Host copy of the device interpolation of Fh_f.
double host_Fh(const std::vector<double> &hyb, int n_tau, double beta, int f, double x) {
  double t = x >= 0.0 ? x : x + beta;
  const double pos = t / beta * n_tau;
  int i = (int)std::floor(pos);
  i = i < 0 ? 0 : (i > n_tau - 1 ? n_tau - 1 : i);
  const double fr = pos - i;
  const double a = hyb[(size_t)f * (n_tau + 1) + i], b = hyb[(size_t)f * (n_tau + 1) + i + 1];
  const double v = a + fr * (b - a);
  return x >= 0.0 ? v : -v;
}

// Inverse of the k x k matrix A (row-major) by Gauss-Jordan elimination with partial
// pivoting; writes inv (row-major), log|det A| and its sign. False if singular.
bool gauss_jordan(int k, std::vector<double> A, std::vector<double> &inv, double &logdet, int &sgn) {
  inv.assign((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) inv[(size_t)i * k + i] = 1.0;
  logdet = 0.0;
  sgn = 1;
  for (int c = 0; c < k; ++c) {
    int p = c;
    for (int r = c + 1; r < k; ++r)
      if (std::fabs(A[(size_t)r * k + c]) > std::fabs(A[(size_t)p * k + c])) p = r;
    const double piv = A[(size_t)p * k + c];
    if (piv == 0.0 || !std::isfinite(piv)) return false;
    if (p != c) {
      for (int j = 0; j < k; ++j) {
        std::swap(A[(size_t)p * k + j], A[(size_t)c * k + j]);
        std::swap(inv[(size_t)p * k + j], inv[(size_t)c * k + j]);
      }
      sgn = -sgn;
    }
    logdet += std::log(std::fabs(piv));
    if (piv < 0) sgn = -sgn;
    const double ip = 1.0 / piv;
    for (int j = 0; j < k; ++j) {
      A[(size_t)c * k + j] *= ip;
      inv[(size_t)c * k + j] *= ip;
    }
    for (int r = 0; r < k; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * k + c];
      if (f == 0.0) continue;
      for (int j = 0; j < k; ++j) {
        A[(size_t)r * k + j] -= f * A[(size_t)c * k + j];
        inv[(size_t)r * k + j] -= f * inv[(size_t)c * k + j];
      }
    }
  }
  return true;
}

}  // namespace

extern "C" {

static bool sweep_params_ok(const kt_sweep_params *p) {
  return p->n_walkers >= 1 && p->k_cap >= 1 && p->k_cap <= 128 && p->n_tau >= 1 && p->n_bins >= 1 && p->cache_ops >= 0;
}

// The sizes and the model of a sweep, before any allocation.
static void sweep_init_view(kt_sweep *s, kt_model *m, const kt_sweep_params *p) {
  const kt::ModelView mv = kt::model_view(m);
  s->model = m;
  s->mv = mv;
  s->measure_obs = p->measure_obs != 0;
  kt::SweepView &v = s->v;
  v.nw = p->n_walkers;
  v.nf = mv.dev->nf;
  v.kcap = p->k_cap;
  v.cap = 2 * v.nf * p->k_cap;
  v.n_tau = p->n_tau;
  v.n_bins = p->n_bins;
  v.nobs = KT_MEASURE_NOBS(mv.dev->n_orb);
  v.n_in = (35 * v.nf + 3 + 15) / 16 * 16;
  v.beta = mv.dev->beta;
}

kt_status kt_sweep_memory_bytes(const kt_model *m, const kt_sweep_params *p, int32_t tries, size_t *bytes) {
  if (!m || !p || !bytes || tries < 0 || tries > KT_DA_MAX_TRIES || !sweep_params_ok(p)) return KT_EINVAL;
  kt_sweep tmp;
  sweep_init_view(&tmp, const_cast<kt_model *>(m), p);
  const kt::DevModel &D = *tmp.mv.dev;
  size_t a = 0, c = 0, t = 0;
  carve_and_alloc(&tmp, &a);
  if (p->cache_ops > 0) alloc_cache(&tmp, std::min(p->cache_ops, tmp.v.cap), &c);
  if (tries > 0) alloc_tries(&tmp, tries, &t);
  *bytes = a + c + t + kt::workspace_bytes(tmp.v.nw, D.n_kept, D.d_max, D.nf + D.n_orb + 1);
  return KT_OK;
}

kt_status kt_sweep_create(kt_model *m, const kt_sweep_params *p, kt_sweep **out) {
  if (!m || !p || !out || !p->hyb) return KT_EINVAL;
  *out = nullptr;
  const kt::ModelView mv = kt::model_view(m);
  if (mv.host_only) return KT_EINVAL;
  if (!sweep_params_ok(p)) return KT_EINVAL;
  const int nf = mv.dev->nf;
  for (long long i = 0; i < (long long)nf * (p->n_tau + 1); ++i)
    if (!std::isfinite(p->hyb[i])) return KT_EINVAL;
  kt_sweep *s = new (std::nothrow) kt_sweep();
  if (!s) return KT_ENOMEM;
  sweep_init_view(s, m, p);
  kt::SweepView &v = s->v;
  kt_status rc = carve_and_alloc(s);
  if (rc == KT_OK && p->cache_ops > 0) rc = alloc_cache(s, std::min(p->cache_ops, v.cap));
  if (rc == KT_OK) {
    s->ws_bytes = kt::workspace_bytes(v.nw, mv.dev->n_kept, mv.dev->d_max, nf + mv.dev->n_orb + 1);
    if (cudaMalloc(&s->ws, s->ws_bytes) != cudaSuccess) {
      cudaGetLastError();
      s->ws = nullptr;
      rc = KT_ENOMEM;
    }
  }
  if (rc == KT_OK) {
    int32_t *offs = (int32_t *)malloc(sizeof(int32_t) * (v.nw + 1));
    if (!offs) rc = KT_ENOMEM;
    if (rc == KT_OK) {
      for (int w = 0; w <= v.nw; ++w) offs[w] = w * v.cap;
      if (cudaMemcpy((void *)v.offsets, offs, sizeof(int32_t) * (v.nw + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy((void *)v.hyb, p->hyb, sizeof(double) * nf * (p->n_tau + 1), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = KT_ECUDA;
      free(offs);
    }
  }
  if (rc == KT_OK) {
    s->hyb_host.assign(p->hyb, p->hyb + (size_t)nf * (p->n_tau + 1));
    rc = reset_empty(s);
  }
  if (rc != KT_OK) {
    cudaGetLastError();
    kt_sweep_destroy(s);
    return rc;
  }
  *out = s;
  return KT_OK;
}

// Shared step loop of kt_sweep_run (mode 0), kt_sweep_run_da (1) and kt_sweep_collect (2).
static kt_status run_steps(kt_sweep *s, int32_t n_steps, const double *uniforms, int32_t meas_every, void *stream,
                           int mode, __nv_bfloat16 *feat, float *targ, int *count, int cap) {
  if (!s || n_steps < 0 || meas_every < 0) return KT_EINVAL;
  if (n_steps == 0) return KT_OK;
  if (!uniforms) return KT_EINVAL;
  const int ustride = mode == 1 ? 7 : 6;
  cudaStream_t st = (cudaStream_t)stream;
  kt::SweepView &v = s->v;
  const kt::DevModel &M = *s->mv.dev;
  // ratios: the plain layout (no measurement regions, so the items split at the middle operator)
  const kt::Workspace w = kt::carve_workspace(s->ws, v.nw, M.n_kept, M.d_max, 0);
  const kt::MoveView mvv{v.mv_kind, v.mv_flv, v.mv_tdag, v.mv_tann, v.mv_rem};
  const kt::SeqView sv = seq_view(s);
  const int wpb = 8;
  const unsigned grid = (unsigned)((v.nw + wpb - 1) / wpb);
  const size_t shm = (size_t)wpb * 2 * v.kcap * sizeof(double);
  cudaGetLastError();
  const size_t shf = (size_t)wpb * v.nf * 34 * sizeof(float);
  for (int step = 0; step < n_steps; ++step) {
    const double *u = uniforms + (size_t)step * v.nw * ustride;
    kt::sweep_propose_kernel<<<grid, wpb * 32, shm, st>>>(v, u, ustride, kt::TryView{});
    if (mode != 0) kt::sweep_features_kernel<<<grid, wpb * 32, shf, st>>>(v, kt::TryView{});
    if (mode == 1) {
      if (kt::mlp_forward(s->net, v.X, v.nw, v.ytil, false, st) != 0) return KT_ECUDA;
      kt::sweep_stage1_kernel<<<(v.nw + 255) / 256, 256, 0, st>>>(v, u);
    }
    if (s->cache_mem) {
      if (kt::launch_cached_pipeline(M, s->mv.precision, s->mv.kernel_dmax, sv, mvv, v.tr_sign, v.tr_log, v.r_sign,
                                     v.r_log, v.r_status, w, s->cache, true, s->stats, st) != 0)
        return KT_ECUDA;
    } else if (kt::launch_pipeline(M, s->mv.precision, s->mv.kernel_dmax, s->mv.group_lanes, sv, &mvv, v.tr_sign,
                                   v.tr_log, v.r_sign, v.r_log, v.r_status, s->stats, w, st, nullptr) != 0) {
      return KT_ECUDA;
    }
    if (mode == 2) kt::sweep_record_kernel<<<grid, wpb * 32, 0, st>>>(v, feat, targ, count, cap);
    kt::sweep_accept_kernel<<<grid, wpb * 32, 0, st>>>(v, u + 5, ustride, w.desc, mode == 1);
    if (s->cache_mem) {
      kt::launch_cache_commit(s->cache, v.nw, M.n_kept, w.desc, w.wstatus, v.p_acc, v.r_status, s->cache_words, st);
    }
    if (meas_every > 0 && (step + 1) % meas_every == 0) {
      kt::sweep_measure_kernel<<<grid, wpb * 32, 0, st>>>(v, nullptr);
      if (s->measure_obs) {
        if (current_traces(s, v.m_sign, v.m_log, v.m_status, v.obs_tmp, st) != 0) return KT_ECUDA;
        const int n = v.nw * v.nobs;
        kt::sweep_obs_accumulate_kernel<<<(n + 255) / 256, 256, 0, st>>>(v, nullptr);
      }
    }
  }
  return cudaGetLastError() == cudaSuccess ? KT_OK : KT_ECUDA;
}

kt_status kt_sweep_run(kt_sweep *s, int32_t n_steps, const double *uniforms, int32_t meas_every, void *stream) {
  return run_steps(s, n_steps, uniforms, meas_every, stream, 0, nullptr, nullptr, nullptr, 0);
}

kt_status kt_sweep_run_da(kt_sweep *s, int32_t n_steps, const double *uniforms, int32_t meas_every, void *stream) {
  if (!s || !s->net) return KT_EINVAL;
  return run_steps(s, n_steps, uniforms, meas_every, stream, 1, nullptr, nullptr, nullptr, 0);
}

kt_status kt_sweep_run_da_multi(kt_sweep *s, int32_t n_steps, int32_t tries, const double *uniforms,
                                int32_t meas_every, void *stream) {
  if (!s || !s->net || n_steps < 0 || meas_every < 0 || tries < 1 || tries > KT_DA_MAX_TRIES) return KT_EINVAL;
  if ((long long)kt::mlp_max_batch(s->net) < (long long)tries * s->v.nw) return KT_EINVAL;
  if (n_steps == 0) return KT_OK;
  if (!uniforms) return KT_EINVAL;
  const kt_status ra = alloc_tries(s, tries);
  if (ra != KT_OK) return ra;
  cudaStream_t st = (cudaStream_t)stream;
  kt::SweepView &v = s->v;
  kt::TryView tv = s->tv;
  tv.T = tries;
  const kt::DevModel &M = *s->mv.dev;
  const kt::Workspace w = kt::carve_workspace(s->ws, v.nw, M.n_kept, M.d_max, 0);
  const kt::MoveView mvv{v.mv_kind, v.mv_flv, v.mv_tdag, v.mv_tann, v.mv_rem};
  const kt::SeqView sv = seq_view(s);
  const int wpb = 8;
  const unsigned grid = (unsigned)((v.nw + wpb - 1) / wpb);
  const size_t shm = (size_t)wpb * 2 * v.kcap * sizeof(double);
  const size_t shf = (size_t)wpb * v.nf * 34 * sizeof(float);
  const int ustride = 7 * tries;
  cudaGetLastError();
  for (int step = 0; step < n_steps; ++step) {
    const double *u = uniforms + (size_t)step * v.nw * ustride;
    // every try from the walker's current configuration (the configuration only changes at
    // the end of the step), all scored by one surrogate inference
    const dim3 grid_t(grid, (unsigned)tries);
    kt::sweep_propose_kernel<<<grid_t, wpb * 32, shm, st>>>(v, u, ustride, tv);
    kt::sweep_next_flavor_kernel<<<grid, wpb * 32, 0, st>>>(v, tv);
    kt::sweep_features_multi_kernel<<<grid_t, wpb * 32, shf, st>>>(v, tv);
    if (kt::mlp_forward(s->net, tv.X, tries * v.nw, tv.ytil, false, st) != 0) return KT_ECUDA;
    kt::sweep_select_kernel<<<grid, wpb * 32, 0, st>>>(v, tv, u);
    // measurement of the configuration the walker spent this step's tries in, weighted by them
    if (meas_every > 0 && (step + 1) % meas_every == 0) {
      kt::sweep_measure_kernel<<<grid, wpb * 32, 0, st>>>(v, tv.n_tries);
      if (s->measure_obs) {
        if (current_traces(s, v.m_sign, v.m_log, v.m_status, v.obs_tmp, st) != 0) return KT_ECUDA;
        const int n = v.nw * v.nobs;
        kt::sweep_obs_accumulate_kernel<<<(n + 255) / 256, 256, 0, st>>>(v, tv.n_tries);
      }
    }
    if (s->cache_mem) {
      if (kt::launch_cached_pipeline(M, s->mv.precision, s->mv.kernel_dmax, sv, mvv, v.tr_sign, v.tr_log, v.r_sign,
                                     v.r_log, v.r_status, w, s->cache, true, s->stats, st) != 0)
        return KT_ECUDA;
    } else if (kt::launch_pipeline(M, s->mv.precision, s->mv.kernel_dmax, s->mv.group_lanes, sv, &mvv, v.tr_sign,
                                   v.tr_log, v.r_sign, v.r_log, v.r_status, s->stats, w, st, nullptr) != 0) {
      return KT_ECUDA;
    }
    kt::sweep_accept_kernel<<<grid, wpb * 32, 0, st>>>(v, tv.u5, 1, w.desc, true);
    if (s->cache_mem) {
      kt::launch_cache_commit(s->cache, v.nw, M.n_kept, w.desc, w.wstatus, v.p_acc, v.r_status, s->cache_words, st);
    }
  }
  return cudaGetLastError() == cudaSuccess ? KT_OK : KT_ECUDA;
}

kt_status kt_sweep_collect(kt_sweep *s, int32_t n_steps, const double *uniforms, void *features, float *targets,
                           int32_t *count, int32_t capacity, void *stream) {
  if (!s || !features || !targets || !count || capacity < 0) return KT_EINVAL;
  return run_steps(s, n_steps, uniforms, 0, stream, 2, (__nv_bfloat16 *)features, targets, count, capacity);
}

kt_status kt_sweep_set_stats(kt_sweep *s, kt_stats *stats) {
  if (!s) return KT_EINVAL;
  s->stats = stats;
  return KT_OK;
}

kt_status kt_sweep_feature_size(const kt_sweep *s, int32_t *n_in) {
  if (!s || !n_in) return KT_EINVAL;
  *n_in = s->v.n_in;
  return KT_OK;
}

kt_status kt_sweep_set_surrogate(kt_sweep *s, kt_mlp *net) {
  if (!s) return KT_EINVAL;
  if (net && kt::mlp_inputs(net) != s->v.n_in) return KT_EINVAL;
  if (net && kt::mlp_max_batch(net) < s->v.nw) return KT_EINVAL;
  s->net = net;
  return KT_OK;
}

static kt_status set_configs_impl(kt_sweep *s, const kt_seq_batch *b);

kt_status kt_sweep_set_configs(kt_sweep *s, const kt_seq_batch *b) {
  if (!s) return KT_EINVAL;
  const kt_status rc = set_configs_impl(s, b);
  if (rc != KT_OK) {
    cudaGetLastError();
    reset_empty(s);
  }
  return rc;
}

static kt_status set_configs_impl(kt_sweep *s, const kt_seq_batch *b) {
  if (!b || b->n != s->v.nw || !b->offsets) return KT_EINVAL;
  kt::SweepView &v = s->v;
  const int nw = v.nw, nf = v.nf, kc = v.kcap, cap = v.cap;
  const double beta = v.beta;
  if (b->offsets[0] != 0) return KT_EINVAL;
  for (int w = 0; w < nw; ++w) {
    const int K = b->offsets[w + 1] - b->offsets[w];
    if (K < 0 || K > cap) return KT_EINVAL;
  }
  const size_t total = (size_t)b->offsets[nw];
  if (total > 0 && (!b->tau || !b->flavor || !b->dagger)) return KT_EINVAL;
  std::vector<int32_t> lens(nw), kf((size_t)nw * nf, 0);
  std::vector<double> tau((size_t)nw * cap, 0.0), rt((size_t)nw * nf * kc, 0.0), ct((size_t)nw * nf * kc, 0.0);
  std::vector<uint8_t> flv((size_t)nw * cap, 0), dag((size_t)nw * cap, 0);
  std::vector<double> detlog(nw, 0.0);
  std::vector<int> detsign(nw, 1);
  // pass 1: validation, times, determinants' signs and logs (M uploaded in pass 2)
  for (int w = 0; w < nw; ++w) {
    const int o = b->offsets[w], K = b->offsets[w + 1] - o;
    lens[w] = K;
    std::vector<int> last(nf, -1);
    for (int k = 0; k < K; ++k) {
      const double t = b->tau[o + k];
      const int f = b->flavor[o + k], d = b->dagger[o + k];
      if (!(t >= 0.0) || !(t < beta) || f >= nf || d > 1 || (k > 0 && t < b->tau[o + k - 1])) return KT_EINVAL;
      if (last[f] >= 0 && last[f] == d) return KT_EINVAL;  // types of one flavor alternate
      last[f] = d;
      tau[(size_t)w * cap + k] = t;
      flv[(size_t)w * cap + k] = (uint8_t)f;
      dag[(size_t)w * cap + k] = (uint8_t)d;
      if (d == 1) {
        const int i = kf[(size_t)w * nf + f]++;
        if (i >= kc) return KT_EINVAL;
        rt[((size_t)w * nf + f) * kc + i] = t;
      }
    }
    std::vector<int> na(nf, 0);
    for (int k = 0; k < K; ++k)
      if (b->dagger[o + k] == 0) {
        const int f = b->flavor[o + k];
        const int j = na[f]++;
        if (j >= kc) return KT_EINVAL;
        ct[((size_t)w * nf + f) * kc + j] = b->tau[o + k];
      }
    for (int f = 0; f < nf; ++f)
      if (na[f] != kf[(size_t)w * nf + f]) return KT_EINVAL;
  }
  // pass 2: inverses (chunks of walkers staged on the host), signs of the bath permutation
  const int chunk = 16;
  std::vector<double> Mh((size_t)chunk * nf * kc * kc);
  std::vector<int> sP(nw, 1);
  kt_status rc = KT_OK;
  for (int w0 = 0; w0 < nw && rc == KT_OK; w0 += chunk) {
    const int w1 = std::min(nw, w0 + chunk);
    std::fill(Mh.begin(), Mh.end(), 0.0);
    for (int w = w0; w < w1 && rc == KT_OK; ++w) {
      std::vector<double> seq;  // bath operators flavor by flavor: tau'_1 tau_1 tau'_2 tau_2 ...
      for (int f = 0; f < nf && rc == KT_OK; ++f) {
        const size_t fb = (size_t)w * nf + f;
        const int k = kf[fb];
        for (int i = 0; i < k; ++i) {
          seq.push_back(rt[fb * kc + i]);
          seq.push_back(ct[fb * kc + i]);
        }
        if (k == 0) continue;
        std::vector<double> A((size_t)k * k), inv;
        for (int i = 0; i < k; ++i)
          for (int j = 0; j < k; ++j) A[(size_t)i * k + j] = host_Fh(s->hyb_host, v.n_tau, beta, f, rt[fb * kc + i] - ct[fb * kc + j]);
        double ld;
        int sg;
        if (!gauss_jordan(k, A, inv, ld, sg)) {
          rc = KT_EINVAL;
          break;
        }
        detlog[w] += ld;
        detsign[w] *= sg;
        double *Mw = Mh.data() + ((size_t)(w - w0) * nf + f) * kc * kc;
        for (int j = 0; j < k; ++j)
          for (int i = 0; i < k; ++i) Mw[(size_t)j * kc + i] = inv[(size_t)j * k + i];
      }
      long long inv_count = 0;
      for (size_t a = 0; a < seq.size(); ++a)
        for (size_t c = a + 1; c < seq.size(); ++c) inv_count += seq[a] < seq[c];
      sP[w] = (inv_count & 1) ? -1 : 1;
    }
    if (rc == KT_OK &&
        cudaMemcpy(v.M + (size_t)w0 * nf * kc * kc, Mh.data(), sizeof(double) * (w1 - w0) * nf * kc * kc,
                   cudaMemcpyHostToDevice) != cudaSuccess)
      rc = KT_ECUDA;
  }
  if (rc != KT_OK) {
    return rc;
  }
  cudaError_t e = cudaMemcpy(v.lens, lens.data(), nw * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(v.tau, tau.data(), tau.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(v.flv, flv.data(), flv.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(v.dag, dag.data(), dag.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(v.kf, kf.data(), kf.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(v.row_t, rt.data(), rt.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(v.col_t, ct.data(), ct.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(v.det_log, detlog.data(), nw * 8, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    return KT_ECUDA;
  }
  if (current_traces(s, v.tr_sign, v.tr_log, v.m_status, nullptr, 0) != 0 || cudaDeviceSynchronize() != cudaSuccess) {
    return KT_ECUDA;
  }
  std::vector<int8_t> ts(nw);
  std::vector<int32_t> tst(nw);
  if (cudaMemcpy(ts.data(), v.tr_sign, nw, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(tst.data(), v.m_status, nw * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
    return KT_ECUDA;
  }
  std::vector<int8_t> ws(nw);
  for (int w = 0; w < nw; ++w) {
    if (ts[w] == 0 || tst[w] != KT_OK) {
      return KT_EINVAL;
    }
    ws[w] = (int8_t)(ts[w] * sP[w] * detsign[w]);
  }
  if (cudaMemcpy(v.w_sign, ws.data(), nw, cudaMemcpyHostToDevice) != cudaSuccess) {
    return KT_ECUDA;
  }
  return invalidate_cache(s);
}

kt_status kt_sweep_refresh(kt_sweep *s, double *max_dev, void *stream) {
  if (!s) return KT_EINVAL;
  kt::SweepView &v = s->v;
  cudaStream_t st = (cudaStream_t)stream;
  cudaGetLastError();
  if (cudaMemsetAsync(v.f_dev, 0, 4 * 8, st) != cudaSuccess) return KT_ECUDA;
  const int wpb = 8;
  const long long nmat = (long long)v.nw * v.nf;
  kt::sweep_refresh_det_kernel<<<(unsigned)((nmat + wpb - 1) / wpb), wpb * 32, wpb * v.kcap * sizeof(int), st>>>(v);
  if (current_traces(s, v.f_tsign, v.f_tlog, v.f_tstat, nullptr, st) != 0) return KT_ECUDA;
  kt::sweep_refresh_apply_kernel<<<(unsigned)(((long long)v.nw * 32 + 255) / 256), 256, 0, st>>>(v);
  if (cudaGetLastError() != cudaSuccess) return KT_ECUDA;
  if (max_dev) {
    unsigned long long h[4];
    if (cudaMemcpyAsync(h, v.f_dev, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return KT_ECUDA;
    double d0, d1;
    memcpy(&d0, &h[0], 8);
    memcpy(&d1, &h[1], 8);
    max_dev[0] = d0;
    max_dev[1] = d1;
    max_dev[2] = (double)h[2];
    max_dev[3] = (double)h[3];
  }
  return KT_OK;
}

kt_status kt_sweep_get_state(kt_sweep *s, const kt_sweep_state *d, void *stream) {
  if (!s || !d) return KT_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const kt::SweepView &v = s->v;
  const size_t nw = v.nw, cap = v.cap, nf = v.nf;
  auto cp = [&](void *dst, const void *src, size_t bytes) {
    return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st) : cudaSuccess;
  };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cp(d->lens, v.lens, nw * 4);
  if (e == cudaSuccess) e = cp(d->tau, v.tau, nw * cap * 8);
  if (e == cudaSuccess) e = cp(d->flavor, v.flv, nw * cap);
  if (e == cudaSuccess) e = cp(d->dagger, v.dag, nw * cap);
  if (e == cudaSuccess) e = cp(d->sign, v.w_sign, nw);
  if (e == cudaSuccess) e = cp(d->trace_sign, v.tr_sign, nw);
  if (e == cudaSuccess) e = cp(d->trace_logabs, v.tr_log, nw * 8);
  if (e == cudaSuccess) e = cp(d->det_logabs, v.det_log, nw * 8);
  if (e == cudaSuccess) e = cp(d->order, v.kf, nw * nf * 4);
  return e == cudaSuccess ? KT_OK : KT_ECUDA;
}

kt_status kt_sweep_get_accumulators(kt_sweep *s, const kt_sweep_accum *d, void *stream) {
  if (!s || !d) return KT_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const kt::SweepView &v = s->v;
  const size_t nw = v.nw, nf = v.nf;
  auto cp = [&](void *dst, const void *src, size_t bytes) {
    return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st) : cudaSuccess;
  };
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cp(d->g_tau, v.g_acc, nw * nf * v.n_bins * 8);
  if (e == cudaSuccess) e = cp(d->sign_sum, v.sign_sum, nw * 8);
  if (e == cudaSuccess) e = cp(d->order_sum, v.order_sum, nw * nf * 8);
  if (e == cudaSuccess) e = cp(d->obs_sum, v.obs_sum, nw * v.nobs * 8);
  return e == cudaSuccess ? KT_OK : KT_ECUDA;
}

kt_status kt_sweep_counters(kt_sweep *s, unsigned long long *out) {
  if (!s || !out) return KT_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return KT_ECUDA;
  if (cudaMemcpy(out, s->v.counters, KT_SWEEP_NCOUNTERS * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return KT_ECUDA;
  return KT_OK;
}

kt_status kt_sweep_reset_accumulators(kt_sweep *s, void *stream) {
  if (!s) return KT_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const kt::SweepView &v = s->v;
  const size_t nw = v.nw, nf = v.nf;
  cudaError_t e = cudaMemsetAsync(v.g_acc, 0, nw * nf * v.n_bins * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(v.sign_sum, 0, nw * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(v.order_sum, 0, nw * nf * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(v.obs_sum, 0, nw * v.nobs * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(v.counters, 0, KT_SWEEP_NCOUNTERS * 8, st);
  return e == cudaSuccess ? KT_OK : KT_ECUDA;
}

void kt_sweep_destroy(kt_sweep *s) {
  if (!s) return;
  if (s->try_mem) cudaFree(s->try_mem);
  if (s->ws) cudaFree(s->ws);
  if (s->mem) cudaFree(s->mem);
  if (s->cache_mem) cudaFree(s->cache_mem);
  delete s;
}

}  // extern "C"
