// Host side of the engine: model setup (Sec. III, setup steps 1-2) and the
// C ABI entry points declared in include/kt.h.
//
// Setup enumerates the 4^n_orb Fock bitstrings, groups them into invariant
// blocks of H_loc (Eq. (H_loc)), builds per block the shifted diagonal and an
// ELL list of the spin-flip / pair-hopping entries, the c / c^+ maps with
// Jordan-Wigner signs, diagonalises each block with cyclic Jacobi rotations,
// selects the kept multiplets (whole multiplets with
// exp(-beta (E - E0)) >= trunc_eps) and uploads everything in one device
// allocation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "kt_internal.h"

namespace {

int popcount32(uint32_t x) { return __builtin_popcount(x); }

// c_f (dag = false) or c_f^+ (dag = true) on bitstring x. Returns false when
// the state is annihilated; otherwise the image and the Jordan-Wigner sign.
bool flip(uint32_t x, int f, bool dag, uint32_t &y, int &sgn) {
  const uint32_t bit = 1u << f;
  const bool occ = (x & bit) != 0;
  if (occ == dag) return false;
  sgn = (popcount32(x & (bit - 1u)) & 1) ? -1 : 1;
  y = x ^ bit;
  return true;
}

// Cyclic Jacobi eigensolver for a small dense symmetric matrix (row-major).
// On return w is ascending and column j of V is the eigenvector of w[j].
void jacobi_eigh(int d, std::vector<double> A, std::vector<double> &w, std::vector<double> &V) {
  V.assign((size_t)d * d, 0.0);
  for (int i = 0; i < d; ++i) V[(size_t)i * d + i] = 1.0;
  double fro = 0.0;
  for (double a : A) fro += a * a;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < d; ++p)
      for (int q = p + 1; q < d; ++q) off += A[(size_t)p * d + q] * A[(size_t)p * d + q];
    if (off <= 1e-34 * fro || off == 0.0) break;
    for (int p = 0; p < d; ++p)
      for (int q = p + 1; q < d; ++q) {
        const double apq = A[(size_t)p * d + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)p * d + p], aqq = A[(size_t)q * d + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        // A <- R^T A R with R the rotation in the (p, q) plane
        for (int k = 0; k < d; ++k) {
          const double akp = A[(size_t)k * d + p], akq = A[(size_t)k * d + q];
          A[(size_t)k * d + p] = c * akp - s * akq;
          A[(size_t)k * d + q] = s * akp + c * akq;
        }
        for (int k = 0; k < d; ++k) {
          const double apk = A[(size_t)p * d + k], aqk = A[(size_t)q * d + k];
          A[(size_t)p * d + k] = c * apk - s * aqk;
          A[(size_t)q * d + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < d; ++k) {
          const double vkp = V[(size_t)k * d + p], vkq = V[(size_t)k * d + q];
          V[(size_t)k * d + p] = c * vkp - s * vkq;
          V[(size_t)k * d + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> idx(d);
  for (int i = 0; i < d; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return A[(size_t)a * d + a] < A[(size_t)b * d + b]; });
  w.resize(d);
  std::vector<double> Vs((size_t)d * d);
  for (int j = 0; j < d; ++j) {
    w[j] = A[(size_t)idx[j] * d + idx[j]];
    for (int i = 0; i < d; ++i) Vs[(size_t)i * d + j] = V[(size_t)i * d + idx[j]];
  }
  V.swap(Vs);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct kt_model {
  kt_model_params params{};
  std::vector<double> delta;
  kt::DevModel dev{};
  void *dev_mem = nullptr;
  size_t dev_bytes = 0;
  int kernel_dmax = 0;
  int group_lanes = 32;
  int nnz_max = 0;
  // host copies for kt_model_kept
  std::vector<double> kept_e;
  std::vector<int32_t> kept_nup, kept_ndn, kept_mask;
  std::vector<double> spectrum;
  double e_kept_max = 0.0;
  bool host_only = false;
  int device = -1;  // CUDA device that holds the tables (current at kt_model_create)
  // per-stage timing (kt_timing_begin / kt_timing_end)
  std::vector<kt::StageEvents> timing;
  int timing_used = 0;
  bool timing_on = false;
};

static void timing_release(kt_model *m) {
  for (auto &t : m->timing)
    for (void *e : t.ev)
      if (e) cudaEventDestroy((cudaEvent_t)e);
  m->timing.clear();
  m->timing_used = 0;
  m->timing_on = false;
}

namespace kt {

size_t workspace_bytes(int n, int n_kept, int d_max, int n_obs_item) {
  const size_t items = (size_t)n * (size_t)n_kept;
  size_t b = 0;
  b += align_up(4 * sizeof(int32_t), 256);
  b += align_up((size_t)n * sizeof(int4), 256);
  b += align_up((size_t)n * sizeof(int32_t), 256);
  b += align_up(items * sizeof(int32_t), 256);
  b += align_up(items * sizeof(int8_t), 256);
  b += align_up(items * sizeof(double), 256);
  b += align_up(items * sizeof(int32_t), 256);
  b += align_up(items * sizeof(int32_t), 256);
  b += align_up(2 * items * sizeof(double), 256);
  b += align_up(2 * items * sizeof(int32_t), 256);
  b += align_up(2 * items * (size_t)d_max * sizeof(double), 256);
  if (n_obs_item > 0) {
    b += align_up(items * (size_t)n_obs_item * sizeof(double), 256);
    b += align_up(items * sizeof(int32_t), 256);
  }
  return b;
}

Workspace carve_workspace(void *base, int n, int n_kept, int d_max, int n_obs_item) {
  const size_t items = (size_t)n * (size_t)n_kept;
  char *p = (char *)base;
  Workspace w;
  w.counters = (int32_t *)p; p += align_up(4 * sizeof(int32_t), 256);
  w.desc = (int4 *)p; p += align_up((size_t)n * sizeof(int4), 256);
  w.wstatus = (int32_t *)p; p += align_up((size_t)n * sizeof(int32_t), 256);
  w.worklist = (int32_t *)p; p += align_up(items * sizeof(int32_t), 256);
  w.item_sign = (int8_t *)p; p += align_up(items * sizeof(int8_t), 256);
  w.item_log = (double *)p; p += align_up(items * sizeof(double), 256);
  w.item_status = (int32_t *)p; p += align_up(items * sizeof(int32_t), 256);
  w.pair_flag = (int32_t *)p; p += align_up(items * sizeof(int32_t), 256);
  w.half_log = (double *)p; p += align_up(2 * items * sizeof(double), 256);
  w.half_info = (int32_t *)p; p += align_up(2 * items * sizeof(int32_t), 256);
  w.half_vec = (void *)p; p += align_up(2 * items * (size_t)d_max * sizeof(double), 256);
  w.item_obs = nullptr;
  w.item_blk = nullptr;
  if (n_obs_item > 0) {
    w.item_obs = (double *)p; p += align_up(items * (size_t)n_obs_item * sizeof(double), 256);
    w.item_blk = (int32_t *)p;
  }
  return w;
}

}  // namespace kt

namespace kt {

bool on_model_device(const ModelView &v) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return dev == v.device;
}

ModelView model_view(const kt_model *m) {
  return ModelView{&m->dev, m->params.precision, m->kernel_dmax, m->group_lanes, m->host_only, m->device};
}

}  // namespace kt

extern "C" {

const char *kt_status_string(kt_status s) {
  switch (s) {
    case KT_OK: return "ok";
    case KT_EINVAL: return "invalid argument, sequence or move";
    case KT_ENOMEM: return "out of memory or workspace too small";
    case KT_ECUDA: return "CUDA error";
    case KT_ENOCONV: return "Krylov propagation did not converge within the dimension cap";
    case KT_ENUMERIC: return "non-finite log-weight";
    case KT_EZEROWEIGHT: return "current weight is zero";
    case KT_ETIMEOUT: return "device wait timed out";
    case KT_EUNSUPPORTED: return "model not supported by the compiled kernels";
  }
  return "unknown status";
}

kt_status kt_model_create(const kt_model_params *pp, kt_model **out) {
  if (!pp || !out) return KT_EINVAL;
  *out = nullptr;
  const kt_model_params P = *pp;
  if (P.n_orb < 1 || P.n_orb > 7 || !(P.beta > 0) || !std::isfinite(P.U) || !std::isfinite(P.J) ||
      !std::isfinite(P.mu) || !(P.deg_tol >= 0) || !(P.krylov_tol > 0) ||
      (P.precision != KT_FP64 && P.precision != KT_FP32_KRYLOV))
    return KT_EINVAL;
  kt_model *M = new (std::nothrow) kt_model();
  if (!M) return KT_ENOMEM;
  M->params = P;
  const int n = P.n_orb, nf = 2 * n, N = 1 << nf;
  M->delta.assign(n, 0.0);
  if (P.delta)
    for (int a = 0; a < n; ++a) M->delta[a] = P.delta[a];
  M->params.delta = nullptr;
  const double U = P.U, J = P.J, Up = std::isnan(P.Up) ? P.U - 2.0 * P.J : P.Up, mu = P.mu;
  const bool sector_blocks = (P.flags & KT_SECTOR_BLOCKS) != 0;
  const bool density_only = (P.flags & KT_DENSITY_ONLY) != 0;

  // ---- blocks: key (n_up, n_dn, singly-occupied mask) ----
  std::map<std::tuple<int, int, int>, int> key2blk;
  std::vector<int> blk_of(N), rank_of(N);
  std::vector<std::vector<uint32_t>> members;
  for (uint32_t x = 0; x < (uint32_t)N; ++x) {
    int nu = 0, nd = 0, mask = 0;
    for (int a = 0; a < n; ++a) {
      const int u = (x >> (2 * a)) & 1, dn = (x >> (2 * a + 1)) & 1;
      nu += u; nd += dn;
      if (u != dn) mask |= 1 << a;
    }
    auto key = std::make_tuple(nu, nd, sector_blocks ? 0 : mask);
    auto it = key2blk.find(key);
    if (it == key2blk.end()) it = key2blk.emplace(key, 0).first;
    (void)it;
  }
  {
    int b = 0;
    for (auto &kv : key2blk) kv.second = b++;
    members.resize(b);
  }
  for (uint32_t x = 0; x < (uint32_t)N; ++x) {
    int nu = 0, nd = 0, mask = 0;
    for (int a = 0; a < n; ++a) {
      const int u = (x >> (2 * a)) & 1, dn = (x >> (2 * a + 1)) & 1;
      nu += u; nd += dn;
      if (u != dn) mask |= 1 << a;
    }
    const int b = key2blk[std::make_tuple(nu, nd, sector_blocks ? 0 : mask)];
    blk_of[x] = b;
    rank_of[x] = (int)members[b].size();
    members[b].push_back(x);
  }
  const int B = (int)members.size();
  std::vector<int32_t> blk_off(B), blk_dim(B), blk_nnz(B), blk_ell(B);
  int d_max = 0;
  for (int b = 0, off = 0; b < B; ++b) {
    blk_off[b] = off;
    blk_dim[b] = (int)members[b].size();
    off += blk_dim[b];
    d_max = std::max(d_max, blk_dim[b]);
  }

  // ---- H_loc rows: diagonal + off-diagonal (spin flip, pair hop) ----
  std::vector<double> diag(N);
  std::vector<std::vector<std::pair<int, double>>> offd(N);  // (global row of target y, value) for column x
  for (uint32_t x = 0; x < (uint32_t)N; ++x) {
    double e = 0.0;
    for (int a = 0; a < n; ++a) {
      const int u = (x >> (2 * a)) & 1, dn = (x >> (2 * a + 1)) & 1;
      e += -(mu + M->delta[a]) * (u + dn) + U * (u * dn);
      for (int b = 0; b < a; ++b) {
        const int bu = (x >> (2 * b)) & 1, bd = (x >> (2 * b + 1)) & 1;
        e += Up * (u * bd + dn * bu) + (Up - J) * (u * bu + dn * bd);
      }
    }
    diag[x] = e;
    if (density_only) continue;
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        if (a == b) continue;
        // spin flip: psi+_{a dn} psi+_{b up} psi_{b dn} psi_{a up}
        // pair hop : psi+_{b up} psi+_{b dn} psi_{a up} psi_{a dn}
        const int seqs[2][4][2] = {{{2 * a, 0}, {2 * b + 1, 0}, {2 * b, 1}, {2 * a + 1, 1}},
                                   {{2 * a + 1, 0}, {2 * a, 0}, {2 * b + 1, 1}, {2 * b, 1}}};
        for (int t = 0; t < 2; ++t) {
          uint32_t y = x;
          int sg = 1;
          bool ok = true;
          for (int k = 0; k < 4 && ok; ++k) {
            int s1;
            ok = flip(y, seqs[t][k][0], seqs[t][k][1] != 0, y, s1);
            sg *= s1;
          }
          if (ok) offd[x].push_back({(int)y, -J * sg});
        }
      }
  }
  // closure: every off-diagonal entry stays inside its block
  for (uint32_t x = 0; x < (uint32_t)N; ++x)
    for (auto &e : offd[x])
      if (blk_of[e.first] != blk_of[x]) { delete M; return KT_EUNSUPPORTED; }

  M->kernel_dmax = kt::kernel_dmax_for(d_max);
  if (M->kernel_dmax == 0) { delete M; return KT_EUNSUPPORTED; }
  M->group_lanes = kt::default_group_for(M->kernel_dmax, P.precision);

  // ---- per block: dense H, Jacobi spectrum, shift, ELL rows ----
  std::vector<std::vector<double>> evals(B), evecs(B);
  std::vector<double> blk_shift(B), blk_norm(B);
  std::vector<std::vector<std::pair<int, double>>> rows(N);  // row r of global state: (col rank, value)
  for (uint32_t x = 0; x < (uint32_t)N; ++x)
    for (auto &e : offd[x]) {  // H[y][x]; two terms reaching the same column share its entry
      auto &row = rows[e.first];
      const int col = rank_of[x];
      bool merged = false;
      for (auto &f : row)
        if (f.first == col) {
          f.second += e.second;
          merged = true;
          break;
        }
      if (!merged) row.push_back({col, e.second});
    }
  int nnz_max = 0, n_ell = 0;
  for (int b = 0; b < B; ++b) {
    const int d = blk_dim[b];
    std::vector<double> A((size_t)d * d, 0.0);
    int w = 0;
    for (int r = 0; r < d; ++r) {
      const uint32_t x = members[b][r];
      A[(size_t)r * d + r] += diag[x];
      for (auto &e : rows[x]) A[(size_t)r * d + e.first] += e.second;
      w = std::max(w, (int)rows[x].size());
    }
    jacobi_eigh(d, A, evals[b], evecs[b]);
    blk_shift[b] = evals[b][0];
    double nrm = 0.0;
    for (int c = 0; c < d; ++c) {
      double s = 0.0;
      for (int r = 0; r < d; ++r) s += std::fabs(A[(size_t)r * d + c] - (r == c ? blk_shift[b] : 0.0));
      nrm = std::max(nrm, s);
    }
    blk_norm[b] = nrm;
    blk_nnz[b] = w;
    blk_ell[b] = n_ell;
    n_ell += w * d;
    nnz_max = std::max(nnz_max, w);
  }
  M->nnz_max = nnz_max;
  std::vector<int16_t> ell_col(std::max(n_ell, 1), (int16_t)-1);
  std::vector<double> ell_val64(std::max(n_ell, 1), 0.0);
  std::vector<uint16_t> st_bits(N);
  std::vector<double> st_diag64(N);
  for (int b = 0; b < B; ++b) {
    const int d = blk_dim[b];
    for (int r = 0; r < d; ++r) {
      const uint32_t x = members[b][r];
      st_bits[blk_off[b] + r] = (uint16_t)x;
      st_diag64[blk_off[b] + r] = diag[x] - blk_shift[b];
      int k = 0;
      for (auto &e : rows[x]) {
        ell_col[blk_ell[b] + k * d + r] = (int16_t)e.first;  // slot-major: lanes read consecutive rows
        ell_val64[blk_ell[b] + k * d + r] = e.second;
        ++k;
      }
    }
  }
  // ---- S^2 per block (measurement at beta/2): diagonal S_z^2 + S_z + sum_a n_{a dn}(1 - n_{a up});
  //      off-diagonal S-_a S+_b = psi+_{a dn} psi+_{b up} psi_{b dn} psi_{a up} (a != b), the
  //      spin-flip string of H_loc with coefficient +1; it keeps the block ----
  std::vector<float> s2_diag(N);
  std::vector<std::vector<std::pair<int, int>>> s2rows(N);  // global row y: (column rank, sign)
  for (uint32_t x = 0; x < (uint32_t)N; ++x) {
    int nu = 0, nd = 0, flip_diag = 0;
    for (int a = 0; a < n; ++a) {
      const int u = (x >> (2 * a)) & 1, dn = (x >> (2 * a + 1)) & 1;
      nu += u;
      nd += dn;
      flip_diag += dn * (1 - u);
    }
    const double sz = 0.5 * (nu - nd);
    s2_diag[x] = (float)(sz * sz + sz + flip_diag);
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        if (a == b) continue;
        const int seq[4][2] = {{2 * a, 0}, {2 * b + 1, 0}, {2 * b, 1}, {2 * a + 1, 1}};
        uint32_t y = x;
        int sg = 1;
        bool ok = true;
        for (int k = 0; k < 4 && ok; ++k) {
          int s1;
          ok = flip(y, seq[k][0], seq[k][1] != 0, y, s1);
          sg *= s1;
        }
        if (ok) {
          if (blk_of[y] != blk_of[x]) { delete M; return KT_EUNSUPPORTED; }
          s2rows[y].push_back({rank_of[x], sg});
        }
      }
  }
  std::vector<int32_t> blk_s2w(B), blk_s2ell(B);
  int n_s2 = 0;
  for (int b = 0; b < B; ++b) {
    int w = 0;
    for (int r = 0; r < blk_dim[b]; ++r) w = std::max(w, (int)s2rows[members[b][r]].size());
    blk_s2w[b] = w;
    blk_s2ell[b] = n_s2;
    n_s2 += w * blk_dim[b];
  }
  std::vector<uint16_t> s2_ell(std::max(n_s2, 1), (uint16_t)0xFFFF);
  std::vector<float> s2_diag_blk(N);
  for (int b = 0; b < B; ++b) {
    const int d = blk_dim[b];
    for (int r = 0; r < d; ++r) {
      const uint32_t x = members[b][r];
      s2_diag_blk[blk_off[b] + r] = s2_diag[x];
      int k = 0;
      for (auto &e : s2rows[x]) {
        s2_ell[blk_s2ell[b] + k * d + r] = (uint16_t)(e.first | (e.second < 0 ? 0x8000 : 0));
        ++k;
      }
    }
  }

  // ---- c / c^+ block maps and partner table ----
  std::vector<int32_t> blk_target((size_t)B * nf * 2, -1);
  std::vector<uint16_t> partner((size_t)N * nf);
  for (int b = 0; b < B; ++b)
    for (int f = 0; f < nf; ++f)
      for (int dg = 0; dg < 2; ++dg) {
        int tgt = -1;
        for (uint32_t x : members[b]) {
          uint32_t y;
          int sg;
          if (!flip(x, f, dg != 0, y, sg)) continue;
          if (tgt < 0) tgt = blk_of[y];
          else if (tgt != blk_of[y]) { delete M; return KT_EUNSUPPORTED; }
        }
        blk_target[((size_t)b * nf + f) * 2 + dg] = tgt;
      }
  for (int b = 0; b < B; ++b)
    for (int r = 0; r < blk_dim[b]; ++r) {
      const uint32_t x = members[b][r];
      for (int f = 0; f < nf; ++f) {
        const uint32_t y = x ^ (1u << f);
        const int neg = popcount32(x & ((1u << f) - 1u)) & 1;
        partner[(size_t)(blk_off[b] + r) * nf + f] = (uint16_t)(rank_of[y] | (neg ? 0x8000 : 0));
      }
    }

  // ---- spectrum, E0, kept multiplets ----
  struct Lv { double e; int b, j; };
  std::vector<Lv> lv;
  lv.reserve(N);
  for (int b = 0; b < B; ++b)
    for (int j = 0; j < blk_dim[b]; ++j) lv.push_back({evals[b][j], b, j});
  std::stable_sort(lv.begin(), lv.end(), [](const Lv &a, const Lv &b) { return a.e < b.e; });
  const double E0 = lv.front().e;
  M->spectrum.reserve(lv.size());
  for (auto &l : lv) M->spectrum.push_back(l.e);
  std::vector<Lv> kept;
  for (size_t i = 0; i < lv.size();) {
    size_t j = i + 1;
    while (j < lv.size() && lv[j].e - lv[j - 1].e <= P.deg_tol * std::max(1.0, std::fabs(lv[j].e))) ++j;
    const bool keep = (P.trunc_eps <= 0) || (std::exp(-P.beta * (lv[i].e - E0)) >= P.trunc_eps);
    if (!keep) break;
    for (size_t k = i; k < j; ++k) kept.push_back(lv[k]);
    i = j;
  }
  const int NK = (int)kept.size();
  std::vector<int32_t> kept_blk(NK), kept_off(NK);
  std::vector<double> kept_e(NK), kept_vec64;
  for (int k = 0; k < NK; ++k) {
    const int b = kept[k].b, d = blk_dim[b];
    kept_blk[k] = b;
    kept_e[k] = kept[k].e - E0;
    kept_off[k] = (int32_t)kept_vec64.size();
    for (int r = 0; r < d; ++r) kept_vec64.push_back(evecs[b][(size_t)r * d + kept[k].j]);
    M->kept_e.push_back(kept_e[k]);
    const uint32_t x = members[b][0];
    int nu = 0, nd = 0, mask = 0;
    for (int a = 0; a < n; ++a) {
      const int u = (x >> (2 * a)) & 1, dn = (x >> (2 * a + 1)) & 1;
      nu += u; nd += dn;
      if (u != dn) mask |= 1 << a;
    }
    M->kept_nup.push_back(nu);
    M->kept_ndn.push_back(nd);
    M->kept_mask.push_back(sector_blocks ? -1 : mask);
    M->e_kept_max = std::max(M->e_kept_max, kept_e[k]);
  }
  if (kept_vec64.empty()) kept_vec64.push_back(0.0);

  M->host_only = (P.flags & KT_HOST_ONLY) != 0;
  {
    kt::DevModel &D = M->dev;
    D.n_orb = n; D.nf = nf; D.n_states = N; D.n_blocks = B; D.n_kept = NK; D.d_max = d_max;
    const int pcap = kt::kernel_pmax_for(M->kernel_dmax);
    D.pmax = (P.krylov_pmax > 0) ? std::min(P.krylov_pmax, pcap) : pcap;
    D.beta = P.beta; D.E0 = E0;
  }
  if (M->host_only) { *out = M; return KT_OK; }

  // ---- upload: one device allocation ----
  std::vector<float> st_diag32(st_diag64.begin(), st_diag64.end());
  std::vector<float> ell_val32(ell_val64.begin(), ell_val64.end());
  std::vector<float> kept_vec32(kept_vec64.begin(), kept_vec64.end());
  // every block's eigendecomposition (exact Krylov stops of the FP32 path): eigenvalues
  // minus the block shift per global row, eigenvectors one after another (vector k of block b
  // at blk_evoff[b] + k d, component r at + r)
  std::vector<double> st_eval64(N);
  std::vector<float> st_eval32(N), blk_evec32, blk_evec32lo;
  std::vector<int32_t> blk_evoff(B);
  for (int b = 0; b < B; ++b) {
    const int d = blk_dim[b];
    blk_evoff[b] = (int32_t)blk_evec32.size();
    for (int k = 0; k < d; ++k) {
      st_eval64[blk_off[b] + k] = evals[b][k] - blk_shift[b];
      st_eval32[blk_off[b] + k] = (float)st_eval64[blk_off[b] + k];
      for (int r = 0; r < d; ++r) {
        const double x = evecs[b][(size_t)r * d + k];
        blk_evec32.push_back((float)x);
        blk_evec32lo.push_back((float)(x - (double)(float)x));
      }
    }
  }
  struct Piece { const void *src; size_t bytes; size_t off; };
  std::vector<Piece> pieces;
  size_t total = 0;
  auto add = [&](const void *src, size_t bytes) {
    pieces.push_back({src, bytes, total});
    total += align_up(std::max<size_t>(bytes, 1), 256);
    return pieces.size() - 1;
  };
  const size_t i_off = add(blk_off.data(), B * 4), i_dim = add(blk_dim.data(), B * 4), i_nnz = add(blk_nnz.data(), B * 4),
               i_ell = add(blk_ell.data(), B * 4), i_shift = add(blk_shift.data(), B * 8), i_norm = add(blk_norm.data(), B * 8),
               i_tgt = add(blk_target.data(), blk_target.size() * 4), i_bits = add(st_bits.data(), N * 2),
               i_d64 = add(st_diag64.data(), N * 8), i_d32 = add(st_diag32.data(), N * 4),
               i_ecol = add(ell_col.data(), ell_col.size() * 2), i_ev64 = add(ell_val64.data(), ell_val64.size() * 8),
               i_ev32 = add(ell_val32.data(), ell_val32.size() * 4), i_part = add(partner.data(), partner.size() * 2),
               i_kb = add(kept_blk.data(), NK * 4), i_ke = add(kept_e.data(), NK * 8), i_ko = add(kept_off.data(), NK * 4),
               i_kv64 = add(kept_vec64.data(), kept_vec64.size() * 8), i_kv32 = add(kept_vec32.data(), kept_vec32.size() * 4),
               i_s2d = add(s2_diag_blk.data(), N * 4), i_s2e = add(s2_ell.data(), s2_ell.size() * 2),
               i_s2w = add(blk_s2w.data(), B * 4), i_s2o = add(blk_s2ell.data(), B * 4),
               i_sev64 = add(st_eval64.data(), N * 8), i_sev32 = add(st_eval32.data(), N * 4),
               i_evo = add(blk_evoff.data(), B * 4), i_evv = add(blk_evec32.data(), blk_evec32.size() * 4),
               i_evvlo = add(blk_evec32lo.data(), blk_evec32lo.size() * 4);
  void *dmem = nullptr;
  if (cudaMalloc(&dmem, total) != cudaSuccess) { cudaGetLastError(); delete M; return KT_ENOMEM; }
  std::vector<char> host(total, 0);
  for (auto &pc : pieces)
    if (pc.bytes) std::memcpy(host.data() + pc.off, pc.src, pc.bytes);
  if (cudaMemcpy(dmem, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dmem);
    delete M;
    return KT_ECUDA;
  }
  M->dev_mem = dmem;
  M->dev_bytes = total;
  if (cudaGetDevice(&M->device) != cudaSuccess) { cudaGetLastError(); M->device = -1; }
  char *base = (char *)dmem;
  auto at = [&](size_t i) { return (void *)(base + pieces[i].off); };
  kt::DevModel &D = M->dev;
  D.n_orb = n; D.nf = nf; D.n_states = N; D.n_blocks = B; D.n_kept = NK; D.d_max = d_max;
  const int pcap = kt::kernel_pmax_for(M->kernel_dmax);
  D.pmax = (P.krylov_pmax > 0) ? std::min(P.krylov_pmax, pcap) : pcap;
  D.beta = P.beta; D.E0 = E0;
  D.tol = P.krylov_tol;
  D.tri64 = (P.precision == KT_FP32_KRYLOV && (P.flags & KT_FP32_TRIDIAG64)) ? 1 : 0;
  D.brk_rel = (P.precision == KT_FP64) ? 1e-14 : 8.0 * std::ldexp(1.0, -24);
  if (P.precision == KT_FP32_KRYLOV) D.tol = std::max(D.tol, 8.0 * std::ldexp(1.0, -24));
  D.blk_off = (const int32_t *)at(i_off); D.blk_dim = (const int32_t *)at(i_dim); D.blk_nnz = (const int32_t *)at(i_nnz);
  D.blk_ell = (const int32_t *)at(i_ell); D.blk_shift = (const double *)at(i_shift); D.blk_norm = (const double *)at(i_norm);
  D.blk_target = (const int32_t *)at(i_tgt); D.st_bits = (const uint16_t *)at(i_bits);
  D.st_diag64 = (const double *)at(i_d64); D.st_diag32 = (const float *)at(i_d32);
  D.ell_col = (const int16_t *)at(i_ecol); D.ell_val64 = (const double *)at(i_ev64); D.ell_val32 = (const float *)at(i_ev32);
  D.partner = (const uint16_t *)at(i_part);
  D.kept_blk = (const int32_t *)at(i_kb); D.kept_e = (const double *)at(i_ke); D.kept_off = (const int32_t *)at(i_ko);
  D.kept_vec64 = (const double *)at(i_kv64); D.kept_vec32 = (const float *)at(i_kv32);
  D.st_eval64 = (const double *)at(i_sev64); D.st_eval32 = (const float *)at(i_sev32);
  D.blk_evoff = (const int32_t *)at(i_evo); D.blk_evec32 = (const float *)at(i_evv);
  D.blk_evec32lo = (const float *)at(i_evvlo);
  D.s2_diag = (const float *)at(i_s2d); D.s2_ell = (const uint16_t *)at(i_s2e);
  D.blk_s2w = (const int32_t *)at(i_s2w); D.blk_s2ell = (const int32_t *)at(i_s2o);
  *out = M;
  return KT_OK;
}

kt_status kt_model_query(const kt_model *m, kt_model_info *o) {
  if (!m || !o) return KT_EINVAL;
  o->n_orb = m->dev.n_orb; o->n_flavors = m->dev.nf; o->n_states = m->dev.n_states;
  o->n_blocks = m->dev.n_blocks; o->d_max = m->dev.d_max; o->nnz_max = m->nnz_max;
  o->n_kept = m->dev.n_kept; o->precision = m->params.precision; o->krylov_pmax = m->dev.pmax;
  o->kernel_dmax = m->kernel_dmax; o->group_lanes = m->group_lanes; o->E0 = m->dev.E0; o->e_kept_max = m->e_kept_max;
  o->device_bytes = m->dev_bytes;
  return KT_OK;
}

kt_status kt_model_spectrum(const kt_model *m, double *e) {
  if (!m || !e) return KT_EINVAL;
  for (size_t i = 0; i < m->spectrum.size(); ++i) e[i] = m->spectrum[i];
  return KT_OK;
}

kt_status kt_model_kept(const kt_model *m, double *e, int32_t *nu, int32_t *nd, int32_t *mask) {
  if (!m) return KT_EINVAL;
  for (int k = 0; k < m->dev.n_kept; ++k) {
    if (e) e[k] = m->kept_e[k];
    if (nu) nu[k] = m->kept_nup[k];
    if (nd) nd[k] = m->kept_ndn[k];
    if (mask) mask[k] = m->kept_mask[k];
  }
  return KT_OK;
}

void kt_model_destroy(kt_model *m) {
  if (!m) return;
  timing_release(m);
  if (m->dev_mem) cudaFree(m->dev_mem);
  delete m;
}

kt_status kt_workspace_size(const kt_model *m, int32_t n, size_t *bytes) {
  if (!m || !bytes || n < 0) return KT_EINVAL;
  *bytes = kt::workspace_bytes(n, m->dev.n_kept, m->dev.d_max);
  return KT_OK;
}

static kt_status run(kt_model *m, const kt_seq_batch *b, const kt_move_batch *mv, const int8_t *cur_sign,
                     const double *cur_logabs, int8_t *sign, double *logv, int32_t *status, kt_stats *stats,
                     void *ws, size_t ws_bytes, void *stream, double *obs = nullptr) {
  if (!m || !b || b->n < 0 || m->host_only) return KT_EINVAL;
  if (b->n == 0) return KT_OK;
  if (!sign || !logv || !status || !b->offsets || !ws) return KT_EINVAL;
  if (mv && (!mv->kind || !mv->flavor || !mv->t_dag || !mv->t_ann || !mv->rem_idx || !cur_sign || !cur_logabs))
    return KT_EINVAL;
  const int nobs_item = obs ? m->dev.nf + m->dev.n_orb + 1 : 0;
  if (ws_bytes < kt::workspace_bytes(b->n, m->dev.n_kept, m->dev.d_max, nobs_item)) return KT_ENOMEM;
  if (!kt::on_model_device(kt::model_view(m))) return KT_EINVAL;  // tables on another GPU
  kt::SeqView sv{b->n, b->offsets, b->tau, b->flavor, b->dagger};
  kt::MoveView mvv{};
  if (mv) mvv = kt::MoveView{mv->kind, mv->flavor, mv->t_dag, mv->t_ann, mv->rem_idx};
  kt::Workspace w = kt::carve_workspace(ws, b->n, m->dev.n_kept, m->dev.d_max, nobs_item);
  const kt::StageEvents *tev = nullptr;
  if (m->timing_on && m->timing_used < (int)m->timing.size()) tev = &m->timing[m->timing_used++];
  const int rc = kt::launch_pipeline(m->dev, m->params.precision, m->kernel_dmax, m->group_lanes, sv,
                                     mv ? &mvv : nullptr, cur_sign, cur_logabs, sign, logv, status, stats, w, stream, tev,
                                     obs);
  return rc == 0 ? KT_OK : KT_ECUDA;
}

kt_status kt_model_set_tiling(kt_model *m, int32_t g) {
  if (!m) return KT_EINVAL;
  int gs[8];
  const int n = kt::kernel_groups_for(m->kernel_dmax, gs, 8);
  for (int i = 0; i < n; ++i)
    if (gs[i] == g) {
      m->group_lanes = g;
      return KT_OK;
    }
  return KT_EINVAL;
}

kt_status kt_autotune(kt_model *m, const kt_seq_batch *b, int8_t *sign, double *logabs, int32_t *status, void *ws,
                      size_t ws_bytes, void *stream, int32_t *chosen) {
  if (!m || !b || m->host_only || !chosen) return KT_EINVAL;
  int gs[8];
  const int n = kt::kernel_groups_for(m->kernel_dmax, gs, 8);
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return KT_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return KT_ECUDA; }
  const int keep = m->group_lanes;
  const bool timing = m->timing_on;
  m->timing_on = false;
  float best = 1e30f;
  int best_g = keep;
  kt_status rc = KT_OK;
  for (int i = 0; i < n && rc == KT_OK; ++i) {
    m->group_lanes = gs[i];
    rc = kt_trace(m, b, sign, logabs, status, nullptr, ws, ws_bytes, stream);  // warm-up (also caches launch shape)
    float tmin = 1e30f;
    for (int rep = 0; rep < 3 && rc == KT_OK; ++rep) {
      cudaEventRecord(e0, st);
      rc = kt_trace(m, b, sign, logabs, status, nullptr, ws, ws_bytes, stream);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = KT_ECUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      tmin = ms < tmin ? ms : tmin;
    }
    if (rc == KT_OK && tmin < best) { best = tmin; best_g = gs[i]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  m->timing_on = timing;
  m->group_lanes = (rc == KT_OK) ? best_g : keep;
  *chosen = m->group_lanes;
  return rc;
}

kt_status kt_timing_begin(kt_model *m, int32_t max_launches) {
  if (!m || m->host_only || max_launches < 1) return KT_EINVAL;
  timing_release(m);
  m->timing.resize((size_t)max_launches);
  for (auto &t : m->timing)
    for (void *&e : t.ev) {
      cudaEvent_t ev;
      if (cudaEventCreate(&ev) != cudaSuccess) {
        e = nullptr;
        timing_release(m);
        return KT_ECUDA;
      }
      e = (void *)ev;
    }
  m->timing_on = true;
  return KT_OK;
}

kt_status kt_timing_end(kt_model *m, double *ms, int32_t *launches) {
  if (!m || !ms || !launches) return KT_EINVAL;
  for (int s = 0; s < 4; ++s) ms[s] = 0.0;
  *launches = m->timing_used;
  kt_status rc = KT_OK;
  for (int i = 0; i < m->timing_used; ++i) {
    auto &t = m->timing[i];
    if (cudaEventSynchronize((cudaEvent_t)t.ev[4]) != cudaSuccess) { rc = KT_ECUDA; break; }
    for (int s = 0; s < 4; ++s) {
      float f = 0.f;
      if (cudaEventElapsedTime(&f, (cudaEvent_t)t.ev[s], (cudaEvent_t)t.ev[s + 1]) != cudaSuccess) { rc = KT_ECUDA; break; }
      ms[s] += f;
    }
  }
  timing_release(m);
  cudaGetLastError();
  return rc;
}

kt_status kt_trace(kt_model *m, const kt_seq_batch *b, int8_t *sign, double *logabs, int32_t *status, kt_stats *stats,
                   void *ws, size_t ws_bytes, void *stream) {
  return run(m, b, nullptr, nullptr, nullptr, sign, logabs, status, stats, ws, ws_bytes, stream);
}

kt_status kt_measure_workspace_size(const kt_model *m, int32_t n, size_t *bytes) {
  if (!m || !bytes || n < 0) return KT_EINVAL;
  *bytes = kt::workspace_bytes(n, m->dev.n_kept, m->dev.d_max, m->dev.nf + m->dev.n_orb + 1);
  return KT_OK;
}

kt_status kt_measure(kt_model *m, const kt_seq_batch *b, int8_t *sign, double *logabs, double *obs, int32_t *status,
                     kt_stats *stats, void *ws, size_t ws_bytes, void *stream) {
  if (!obs && b && b->n > 0) return KT_EINVAL;
  return run(m, b, nullptr, nullptr, nullptr, sign, logabs, status, stats, ws, ws_bytes, stream, obs);
}

kt_status kt_trace_ratio(kt_model *m, const kt_seq_batch *cur, const int8_t *cur_sign, const double *cur_logabs,
                         const kt_move_batch *moves, int8_t *sign, double *logratio, int32_t *status, kt_stats *stats,
                         void *ws, size_t ws_bytes, void *stream) {
  if (!moves) return KT_EINVAL;
  return run(m, cur, moves, cur_sign, cur_logabs, sign, logratio, status, stats, ws, ws_bytes, stream);
}

}  // extern "C"
