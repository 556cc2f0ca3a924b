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
//                matrix-free SpMV on the block, FP64 dot products and norms,
//                a three-term recurrence, and the FP64 exponential of the
//                small tridiagonal matrix, with the Krylov dimension chosen
//                per interval by an a-posteriori error estimate.
//   4. reduce  - one thread per walker: signed log-sum-exp over kept states
//                (step 7-8) and, for a ratio, division by the current trace.
#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>

#include "kt_internal.h"

namespace kt {

namespace {

constexpr unsigned FULL = 0xffffffffu;

struct Op {
  double t;
  int f, dag;
};

__device__ __forceinline__ Op load_op(const SeqView &S, int i) {
  return Op{__ldg(S.tau + i), (int)__ldg(S.flavor + i), (int)__ldg(S.dagger + i)};
}

// Operator i of the (possibly edited) sequence of one walker.
// desc = {kind, p1, p2, K_new}: kind -1 none, 0 insert (op A at new index p1,
// op B at new index p2 + 1), 1 remove (old indices p1 < p2 dropped).
struct Cursor {
  SeqView S;
  int o;
  int4 d;
  Op A, B;
  __device__ __forceinline__ Op get(int i) const {
    if (d.x == 0) {
      if (i < d.y) return load_op(S, o + i);
      if (i == d.y) return A;
      if (i <= d.z) return load_op(S, o + i - 1);
      if (i == d.z + 1) return B;
      return load_op(S, o + i - 2);
    }
    if (d.x == 1) {
      if (i < d.y) return load_op(S, o + i);
      if (i < d.z - 1) return load_op(S, o + i + 1);
      return load_op(S, o + i + 2);
    }
    return load_op(S, o + i);
  }
};

__device__ __forceinline__ Cursor make_cursor(const SeqView &S, const MoveView &mv, bool has_moves, const int4 *desc,
                                              int w) {
  Cursor c;
  c.S = S;
  c.o = __ldg(S.offsets + w);
  c.d = desc[w];
  if (has_moves && c.d.x == 0) {
    const int f = mv.flavor[w];
    const double td = mv.t_dag[w], ta = mv.t_ann[w];
    if (td < ta) {
      c.A = Op{td, f, 1};
      c.B = Op{ta, f, 0};
    } else {
      c.A = Op{ta, f, 0};
      c.B = Op{td, f, 1};
    }
  }
  return c;
}

__device__ __forceinline__ int upper_bound(const double *t, int K, double x) {
  int lo = 0, hi = K;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (t[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void stat_add(unsigned long long *p, unsigned long long v) {
  if (v) atomicAdd(p, v);
}

// ---------------------------------------------------------------------------
// 1. validation and move editing
// ---------------------------------------------------------------------------
__global__ void prep_kernel(DevModel M, SeqView S, MoveView mv, int has_moves, const int8_t *cur_sign, Workspace ws,
                            kt_stats *stats) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w == 0) {
    ws.counters[0] = 0;
    ws.counters[1] = 0;
  }
  if (w >= S.n) return;
  const int o = S.offsets[w], K = S.offsets[w + 1] - o;
  int st = KT_OK;
  int4 d = make_int4(-1, 0, 0, K);
  if (K < 0) {
    st = KT_EINVAL;
  } else {
    double prev = 0.0;
    for (int k = 0; k < K; ++k) {
      const double t = S.tau[o + k];
      if (!(t >= prev) || !(t < M.beta) || S.flavor[o + k] >= M.nf || S.dagger[o + k] > 1) {
        st = KT_EINVAL;
        break;
      }
      prev = t;
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
        const double tA = td < ta ? td : ta, tB = td < ta ? ta : td;
        const int pa = upper_bound(S.tau + o, K, tA), pb = upper_bound(S.tau + o, K, tB);
        d = make_int4(0, pa, pb, K + 2);
      }
    } else if (kind == 1) {
      const int r = mv.rem_idx[w];
      if (r < 0 || r >= K || S.flavor[o + r] != f || S.dagger[o + r] != 1) {
        st = KT_EINVAL;
      } else {
        int j = -1;
        for (int s = 1; s < K; ++s) {
          const int c = (r + s) % K;
          if (S.flavor[o + c] == f) {
            j = c;
            break;
          }
        }
        if (j < 0 || S.dagger[o + j] != 0) {
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
  ws.desc[w] = d;
  ws.wstatus[w] = st;
  if (stats) atomicAdd(&stats->walkers, 1ull);
}

// ---------------------------------------------------------------------------
// 2. structural pruning
// ---------------------------------------------------------------------------
__global__ void prune_kernel(DevModel M, SeqView S, MoveView mv, int has_moves, Workspace ws, kt_stats *stats) {
  const int item = blockIdx.x * blockDim.x + threadIdx.x;
  const int nk = M.n_kept;
  if (item >= S.n * nk) return;
  const int w = item / nk, q = item - w * nk;
  ws.item_sign[item] = 0;
  ws.item_status[item] = KT_OK;
  ws.item_log[item] = -INFINITY;
  if (ws.wstatus[w] != KT_OK) return;
  const Cursor c = make_cursor(S, mv, has_moves != 0, ws.desc, w);
  const int b0 = __ldg(M.kept_blk + q);
  int b = b0;
  for (int i = 0; i < c.d.w && b >= 0; ++i) {
    const Op op = c.get(i);
    b = __ldg(M.blk_target + ((size_t)b * M.nf + op.f) * 2 + op.dag);
  }
  const bool alive = (b == b0);
  if (alive) {
    const int slot = atomicAdd(&ws.counters[0], 1);
    ws.worklist[slot] = item;
  }
  if (stats) {
    atomicAdd(&stats->items, 1ull);
    if (alive) atomicAdd(&stats->items_alive, 1ull);
  }
}

// ---------------------------------------------------------------------------
// 3. Krylov items
// ---------------------------------------------------------------------------
template <typename VT, int DMAX, int PMAX>
struct WarpSmem {
  VT q[PMAX + 1][DMAX];  // Lanczos basis; q[0] carries the state between intervals
  VT t[DMAX];            // gather target
  double alpha[PMAX], beta[PMAX];
  double dd[PMAX], ee[PMAX];  // tridiagonal working copy -> Ritz values
  double ex[PMAX];            // exp(-dtau (lambda_k - lambda_min))
  double y[PMAX];             // exp(-dtau T) e_1 (scaled)
  double S[PMAX][PMAX];       // S[k][i]: component i of Ritz vector k
};

template <typename VT>
struct Tab;
template <>
struct Tab<float> {
  static __device__ __forceinline__ const float *diag(const DevModel &M) { return M.st_diag32; }
  static __device__ __forceinline__ const float *val(const DevModel &M) { return M.ell_val32; }
  static __device__ __forceinline__ const float *kept(const DevModel &M) { return M.kept_vec32; }
};
template <>
struct Tab<double> {
  static __device__ __forceinline__ const double *diag(const DevModel &M) { return M.st_diag64; }
  static __device__ __forceinline__ const double *val(const DevModel &M) { return M.ell_val64; }
  static __device__ __forceinline__ const double *kept(const DevModel &M) { return M.kept_vec64; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// y = exp(-dt T_p) e_1 / exp(-dt lambda_min) for the symmetric tridiagonal T_p
// (diagonal alpha[0..p), off-diagonal beta[0..p-1)). Writes y to smem and
// returns log of the factor taken out (-dt lambda_min). p = 1 and p = 2 use
// closed forms; p >= 3 an implicit QL iteration with shifts from the leading
// 2x2 block, the Ritz vectors kept one component per lane. All FP64.
// Returns false if the QL iteration did not converge.
template <typename VT, int DMAX, int PMAX>
__device__ bool tri_exp(WarpSmem<VT, DMAX, PMAX> &s, int p, double dt, int lane, double &logfac) {
  if (p == 1) {
    if (lane == 0) s.y[0] = 1.0;
    logfac = -dt * s.alpha[0];
    __syncwarp();
    return true;
  }
  if (p == 2) {
    const double a = s.alpha[0], c = s.alpha[1], b = s.beta[0];
    const double m = 0.5 * (a + c), h = 0.5 * (a - c);
    const double r = hypot(h, b);
    const double E = exp(-2.0 * dt * r);
    const double g = (r > 0.0) ? -expm1(-2.0 * dt * r) / (2.0 * r) : dt;
    if (lane == 0) {
      s.y[0] = 0.5 * (1.0 + E) - g * h;
      s.y[1] = -g * b;
    }
    logfac = -dt * (m - r);
    __syncwarp();
    return true;
  }
  // ---- p >= 3: implicit QL ----
  for (int i = lane; i < p; i += 32) {
    s.dd[i] = s.alpha[i];
    s.ee[i] = (i + 1 < p) ? s.beta[i] : 0.0;
    for (int k = 0; k < p; ++k) s.S[k][i] = (i == k) ? 1.0 : 0.0;
  }
  __syncwarp();
  const double eps = 2.3e-16;
  int lo = 0, guard = 0;
  bool ok = true;
  while (lo < p - 1) {
    // deflate from the top
    if (fabs(s.ee[lo]) <= eps * (fabs(s.dd[lo]) + fabs(s.dd[lo + 1]))) {
      ++lo;
      continue;
    }
    int hi = lo + 1;
    while (hi < p - 1 && fabs(s.ee[hi]) > eps * (fabs(s.dd[hi]) + fabs(s.dd[hi + 1]))) ++hi;
    if (++guard > 40 * p) {
      ok = false;
      break;
    }
    // shift: eigenvalue of the leading 2x2 of [lo, hi] closest to dd[lo]
    const double b0 = s.ee[lo];
    const double dm = 0.5 * (s.dd[lo + 1] - s.dd[lo]);
    const double mu = s.dd[lo] - b0 * b0 / (dm + copysign(hypot(dm, b0), dm));
    double x = s.dd[hi] - mu, z = s.ee[hi - 1];
    for (int k = hi; k > lo; --k) {
      // rotation in the (k-1, k) plane that zeroes z against x
      const double r = hypot(x, z);
      const double c = (r == 0.0) ? 1.0 : x / r, sn = (r == 0.0) ? 0.0 : -z / r;
      const double a11 = s.dd[k], a22 = s.dd[k - 1], a12 = s.ee[k - 1];
      const double ek2 = (k - 1 > lo) ? s.ee[k - 2] : 0.0;
      __syncwarp();
      if (lane == 0) {
        if (k < hi) s.ee[k] = r;
        s.dd[k] = c * c * a11 - 2.0 * c * sn * a12 + sn * sn * a22;
        s.dd[k - 1] = sn * sn * a11 + 2.0 * c * sn * a12 + c * c * a22;
        s.ee[k - 1] = c * sn * (a11 - a22) + (c * c - sn * sn) * a12;
        if (k - 1 > lo) s.ee[k - 2] = c * ek2;
      }
      for (int i = lane; i < p; i += 32) {
        const double vk = s.S[k][i], vk1 = s.S[k - 1][i];
        s.S[k][i] = c * vk - sn * vk1;
        s.S[k - 1][i] = sn * vk + c * vk1;
      }
      __syncwarp();
      if (k - 1 > lo) {
        x = s.ee[k - 1];
        z = -sn * ek2;
      }
    }
  }
  __syncwarp();
  double lmin = s.dd[0];
  for (int k = 1; k < p; ++k) lmin = fmin(lmin, s.dd[k]);
  for (int k = lane; k < p; k += 32) s.ex[k] = exp(-dt * (s.dd[k] - lmin)) * s.S[k][0];
  __syncwarp();
  for (int i = lane; i < p; i += 32) {
    double acc = 0.0;
    for (int k = 0; k < p; ++k) acc += s.S[k][i] * s.ex[k];
    s.y[i] = acc;
  }
  logfac = -dt * lmin;
  __syncwarp();
  return ok;
}

struct ItemAcc {
  unsigned long long ops, intervals, iters, pmax, noconv, flops_vec, flops_tri, bytes_apply;
};

template <typename VT, int DMAX, int PMAX>
__global__ void __launch_bounds__(256) items_kernel(DevModel M, SeqView S, MoveView mv, int has_moves, Workspace ws,
                                                    kt_stats *stats, int warps_per_block) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int R = (DMAX + 31) / 32;  // rows per lane
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  WarpSmem<VT, DMAX, PMAX> &s = reinterpret_cast<WarpSmem<VT, DMAX, PMAX> *>(smem_raw)[wib];
  const VT *__restrict__ tdiag = Tab<VT>::diag(M);
  const VT *__restrict__ tval = Tab<VT>::val(M);
  const VT *__restrict__ tkept = Tab<VT>::kept(M);
  const int n_alive = ws.counters[0];
  const int nk = M.n_kept, nf = M.nf;

  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(&ws.counters[1], 1);
    it = __shfl_sync(FULL, it, 0);
    if (it >= n_alive) break;
    const int item = ws.worklist[it];
    const int w = item / nk, q = item - w * nk;
    const Cursor cur = make_cursor(S, mv, has_moves != 0, ws.desc, w);
    const int Kn = cur.d.w;
    int b = __ldg(M.kept_blk + q);
    const int b_kept = b;
    int dim = __ldg(M.blk_dim + b);
    const double Ek = __ldg(M.kept_e + q);
    const int koff = __ldg(M.kept_off + q);
    ItemAcc acc{};
    int status = KT_OK;
    bool vanished = false;
    double L = 0.0;
    int sgn = 1;

    if (Kn == 0) {
      L = -M.beta * Ek;
    } else {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int r = lane + 32 * j;
        if (r < dim) s.q[0][r] = __ldg(tkept + koff + r);
      }
      __syncwarp();
      Op op = cur.get(0);
      L = -op.t * Ek;
      for (int i = 0; i < Kn; ++i) {
        // ---- step 4: apply c_f / c_f^+ (gather with Jordan-Wigner sign) ----
        const int b2 = __ldg(M.blk_target + ((size_t)b * nf + op.f) * 2 + op.dag);
        if (b2 < 0) {
          vanished = true;
          break;
        }
        const int off2 = __ldg(M.blk_off + b2), dim2 = __ldg(M.blk_dim + b2);
        double nrm2 = 0.0;
        VT tv[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int r = lane + 32 * j;
          VT v = VT(0);
          if (r < dim2) {
            const int g = off2 + r;
            const int x = __ldg(M.st_bits + g);
            if (((x >> op.f) & 1) == op.dag) {
              const unsigned pe = __ldg(M.partner + (size_t)g * nf + op.f);
              v = s.q[0][pe & 0x7fffu];
              if (pe & 0x8000u) v = -v;
            }
            nrm2 += (double)v * (double)v;
          }
          tv[j] = v;
        }
        nrm2 = warp_sum(nrm2);
        acc.ops += 1;
        acc.flops_vec += 3ull * dim2;
        acc.bytes_apply += (unsigned long long)dim2 * (2 * sizeof(VT) + 4);
        if (!(nrm2 > 0.0)) {
          vanished = true;
          break;
        }
        const double nrm = sqrt(nrm2);
        L += log(nrm);
        const VT inv = VT(1.0 / nrm);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int r = lane + 32 * j;
          if (r < dim2) s.q[0][r] = tv[j] * inv;
        }
        __syncwarp();
        b = b2;
        dim = dim2;
        if (i + 1 >= Kn) break;
        const Op nx = cur.get(i + 1);
        const double dt = nx.t - op.t;
        op = nx;
        if (!(dt > 0.0)) continue;
        // ---- step 5: Lanczos approximation of exp(-dt (H_b - E0)) q0 ----
        const int off = __ldg(M.blk_off + b), wid = __ldg(M.blk_nnz + b), ell = __ldg(M.blk_ell + b);
        const double shift = __ldg(M.blk_shift + b);
        const double brk = M.brk_rel * fmax(__ldg(M.blk_norm + b), 1e-300);
        const int pcap = min(dim, M.pmax);
        VT qc[R], qp[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int r = lane + 32 * j;
          qc[j] = (r < dim) ? s.q[0][r] : VT(0);
          qp[j] = VT(0);
        }
        double bprev = 0.0, logfac = 0.0;
        int p = 0;
        bool conv = false;
        unsigned long long nnz_row_sum = 0;
        for (int jj = 0; jj < pcap; ++jj) {
          // w = (H_b - s_b) q_jj
          VT wv[R];
          double al = 0.0;
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const int r = lane + 32 * j;
            VT a = VT(0);
            if (r < dim) {
              a = __ldg(tdiag + off + r) * qc[j];
              for (int k = 0; k < wid; ++k) {
                const int col = __ldg(M.ell_col + ell + k * dim + r);
                if (col >= 0) a += __ldg(tval + ell + k * dim + r) * s.q[jj][col];
              }
              al += (double)a * (double)qc[j];
            }
            wv[j] = a;
          }
          al = warp_sum(al);
          double bb = 0.0;
          const VT alv = VT(al), bpv = VT(bprev);
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const int r = lane + 32 * j;
            if (r < dim) {
              wv[j] = wv[j] - alv * qc[j] - bpv * qp[j];
              bb += (double)wv[j] * (double)wv[j];
            }
          }
          bb = sqrt(warp_sum(bb));
          p = jj + 1;
          if (lane == 0) {
            s.alpha[jj] = al;
            s.beta[jj] = bb;
          }
          __syncwarp();
          const bool exact = (p == dim) || !(bb > brk);
          const bool okq = tri_exp(s, p, dt, lane, logfac);
          acc.flops_tri += (p <= 2) ? 30ull : (unsigned long long)(12 * p * p * p + 40 * p);
          if (!okq) status = KT_ENUMERIC;
          if (exact) {
            conv = true;
            break;
          }
          double yn = 0.0;
          for (int k = lane; k < p; k += 32) yn += s.y[k] * s.y[k];
          yn = sqrt(warp_sum(yn));
          const double err = bb * fabs(s.y[p - 1]);
          if (err <= M.tol * yn) {
            conv = true;
            break;
          }
          if (p == pcap) break;
          // q_{jj+1} = w / beta
          const VT ib = VT(1.0 / bb);
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const int r = lane + 32 * j;
            qp[j] = qc[j];
            qc[j] = wv[j] * ib;
            if (r < dim) s.q[jj + 1][r] = qc[j];
          }
          bprev = bb;
          __syncwarp();
        }
        (void)nnz_row_sum;
        if (!conv) {
          acc.noconv += 1;
          if (status == KT_OK) status = KT_ENOCONV;
        }
        // v = sum_j y_j q_j, renormalised; log of everything taken out goes to L
        double vn = 0.0;
        VT vv[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int r = lane + 32 * j;
          VT a = VT(0);
          if (r < dim)
            for (int k = 0; k < p; ++k) a += VT(s.y[k]) * s.q[k][r];
          vv[j] = a;
          vn += (double)a * (double)a;
        }
        vn = warp_sum(vn);
        if (!(vn > 0.0)) {
          vanished = true;
          break;
        }
        vn = sqrt(vn);
        L += logfac + log(vn) - dt * (shift - M.E0);
        const VT ivn = VT(1.0 / vn);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int r = lane + 32 * j;
          if (r < dim) s.q[0][r] = vv[j] * ivn;
        }
        __syncwarp();
        // algorithmic flops of this propagation
        int nnz_blk = 0;
        {
          // nnz of the block (diagonal + stored off-diagonals), counted from the ELL columns
          int cnt = 0;
          for (int j = 0; j < R; ++j) {
            const int r = lane + 32 * j;
            if (r < dim) {
              cnt += 1;
              for (int k = 0; k < wid; ++k) cnt += (__ldg(M.ell_col + ell + k * dim + r) >= 0);
            }
          }
          nnz_blk = (int)warp_sum((double)cnt);
        }
        acc.intervals += 1;
        acc.iters += p;
        acc.pmax = acc.pmax > (unsigned long long)p ? acc.pmax : (unsigned long long)p;
        acc.flops_vec += (unsigned long long)p * (2ull * nnz_blk + 9ull * dim) + 2ull * p * dim + 3ull * dim;
      }
    }
    if (!vanished && Kn > 0) {
      if (b != b_kept) {
        vanished = true;
      } else {
        double ov = 0.0;
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int r = lane + 32 * j;
          if (r < dim) ov += (double)__ldg(tkept + koff + r) * (double)s.q[0][r];
        }
        ov = warp_sum(ov);
        if (ov == 0.0) {
          vanished = true;
        } else {
          sgn = ov > 0.0 ? 1 : -1;
          L += log(fabs(ov)) - (M.beta - cur.get(Kn - 1).t) * Ek;
        }
      }
    }
    if (!vanished && !isfinite(L)) status = KT_ENUMERIC;
    if (lane == 0) {
      ws.item_sign[item] = vanished ? 0 : (int8_t)sgn;
      ws.item_log[item] = vanished ? -INFINITY : L;
      ws.item_status[item] = status;
      if (stats) {
        if (vanished) atomicAdd(&stats->items_vanished, 1ull);
        stat_add(&stats->ops_applied, acc.ops);
        stat_add(&stats->intervals, acc.intervals);
        stat_add(&stats->krylov_iters, acc.iters);
        if (acc.pmax) atomicMax(&stats->p_max, acc.pmax);
        stat_add(&stats->noconv, acc.noconv);
        stat_add(&stats->flops_vec, acc.flops_vec);
        stat_add(&stats->flops_tri, acc.flops_tri);
        stat_add(&stats->bytes_apply, acc.bytes_apply);
      }
    }
    __syncwarp();
  }
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

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
template <typename VT, int DMAX, int PMAX>
int launch_items(const DevModel &M, const SeqView &S, const MoveView &mv, int has_moves, const Workspace &ws,
                 kt_stats *stats, cudaStream_t st) {
  using Sm = WarpSmem<VT, DMAX, PMAX>;
  static int cached_grid = 0, cached_wpb = 0;
  if (cached_grid == 0) {
    int wpb = (int)((48 * 1024) / sizeof(Sm));
    wpb = wpb < 1 ? 1 : (wpb > 8 ? 8 : wpb);
    const size_t smem = (size_t)wpb * sizeof(Sm);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(items_kernel<VT, DMAX, PMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, items_kernel<VT, DMAX, PMAX>, wpb * 32, smem);
    if (per_sm < 1) per_sm = 1;
    cached_wpb = wpb;
    cached_grid = sms * per_sm;
  }
  const size_t smem = (size_t)cached_wpb * sizeof(Sm);
  items_kernel<VT, DMAX, PMAX><<<cached_grid, cached_wpb * 32, smem, st>>>(M, S, mv, has_moves, ws, stats, cached_wpb);
  return (int)cudaGetLastError();
}

}  // namespace

int kernel_dmax_for(int d_max) {
  if (d_max <= 16) return 16;
  if (d_max <= 32) return 32;
  if (d_max <= 64) return 64;
  if (d_max <= 128) return 128;
  return 0;
}

int kernel_pmax_for(int kd) {
  switch (kd) {
    case 16: return 16;
    case 32: return 32;
    case 64: return 32;
    case 128: return 40;
  }
  return 0;
}

int launch_pipeline(const DevModel &M, int precision, int kd, const SeqView &S, const MoveView *moves,
                    const int8_t *cur_sign, const double *cur_logabs, int8_t *sign, double *logv, int32_t *status,
                    kt_stats *stats, const Workspace &ws, void *stream, const StageEvents *timing) {
  cudaStream_t st = (cudaStream_t)stream;
  auto mark = [&](int i) {
    if (timing) cudaEventRecord((cudaEvent_t)timing->ev[i], st);
  };
  const int n = S.n;
  const int has_moves = moves ? 1 : 0;
  MoveView mv = moves ? *moves : MoveView{};
  cudaGetLastError();
  mark(0);
  prep_kernel<<<(n + 255) / 256, 256, 0, st>>>(M, S, mv, has_moves, cur_sign, ws, stats);
  mark(1);
  const long long items = (long long)n * M.n_kept;
  if (items > 0) prune_kernel<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(M, S, mv, has_moves, ws, stats);
  mark(2);
  int rc = (int)cudaGetLastError();
  if (rc) return rc;
  if (items > 0) {
    if (precision == KT_FP64) {
      switch (kd) {
        case 16: rc = launch_items<double, 16, 16>(M, S, mv, has_moves, ws, stats, st); break;
        case 32: rc = launch_items<double, 32, 32>(M, S, mv, has_moves, ws, stats, st); break;
        case 64: rc = launch_items<double, 64, 32>(M, S, mv, has_moves, ws, stats, st); break;
        case 128: rc = launch_items<double, 128, 40>(M, S, mv, has_moves, ws, stats, st); break;
        default: return (int)cudaErrorInvalidValue;
      }
    } else {
      switch (kd) {
        case 16: rc = launch_items<float, 16, 16>(M, S, mv, has_moves, ws, stats, st); break;
        case 32: rc = launch_items<float, 32, 32>(M, S, mv, has_moves, ws, stats, st); break;
        case 64: rc = launch_items<float, 64, 32>(M, S, mv, has_moves, ws, stats, st); break;
        case 128: rc = launch_items<float, 128, 40>(M, S, mv, has_moves, ws, stats, st); break;
        default: return (int)cudaErrorInvalidValue;
      }
    }
    if (rc) return rc;
  }
  mark(3);
  reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(M, n, has_moves, cur_sign, cur_logabs, ws, sign, logv, status);
  mark(4);
  return (int)cudaGetLastError();
}

}  // namespace kt
