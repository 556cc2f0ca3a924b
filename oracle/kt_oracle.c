/*
 * Plain CPU oracle for the Krylov CT-HYB local trace (test infrastructure only).
 *
 * This file is test infrastructure: only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark load it. The product library never links
 * it, includes it, or calls it, and it shares no code with the product.
 *
 * What it computes is the plain definition, written out the slow and obvious
 * way, in the occupation-number basis blocked by (n_up, n_dn) sectors:
 *
 *  - H_loc of Sec. IV.A, Eq. (H_loc): chemical potential and crystal field,
 *    intra-orbital U, inter-orbital U' (opposite spin) and U'-J (same spin)
 *    summed over a>b, and the spin-flip and pair-hopping terms with
 *    coefficient -J, each ordered pair a != b counted once (the "+h.c." is
 *    read as already contained in the sum over ordered pairs; that reading
 *    keeps H_loc SU(2) invariant for U' = U - 2J, as the text states).
 *  - A dense symmetric eigendecomposition of every sector block
 *    (Householder reduction to tridiagonal form, then implicit symmetric QR
 *    with Wilkinson shifts; Golub & Van Loan, Sec. 8.3), used for the
 *    low-energy spectrum (Sec. III, setup step 1) and for exact block
 *    exponentials V diag(exp(-dtau (w - E0))) V^T. Each sector is
 *    diagonalised one connected component of H's nonzero pattern at a time
 *    (H is exactly block diagonal in them, so this is the same exponential),
 *    which keeps rounding from coupling subspaces that H never couples.
 *  - Truncation of the outer trace to whole multiplets with
 *    exp(-beta (E - E0)) >= trunc_eps (Sec. II, truncation type (i);
 *    Sec. III, setup step 2).
 *  - The truncated trace Sec. III steps 3-8 / Eq. (weight_strong):
 *    T~ = sum over kept |n> of <n| e^{-(beta-tau_K)(H-E0)} O_K ...
 *         O_1 e^{-tau_1 (H-E0)} |n>,
 *    with O_k = c_f or c_f^dagger applied in increasing array index, the
 *    first and last intervals as scalars (|n> is an eigenstate) and every
 *    inner interval as an exact block exponential. Results are reported as
 *    (sign, log|T|) with log|T| = log|T~| - beta E0.
 *  - The same trace with a diagonal operator of the occupation basis inserted
 *    at one time (Sec. III: local observables measured at tau = beta/2 in the
 *    truncated trace), evaluated right to left as written.
 *
 * Conventions (the paper is silent on these): flavor f = 2a + s with orbital
 * a and spin s (0 = up, 1 = down); bit f of the state is n_f; c_f and c_f^+
 * carry the Jordan-Wigner sign (-1)^popcount(x & ((1<<f)-1)).
 *
 * The same source is compiled twice: with OR_REAL = double (the oracle
 * proper) and with OR_REAL = long double (a higher-precision twin used only
 * to tell traces whose exact value is zero from regular ones). <tgmath.h>
 * dispatches every math call on the argument type.
 */
#include <tgmath.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef OR_REAL
#define OR_REAL double
#endif
#ifndef OR_PREFIX
#define OR_PREFIX or64_
#endif
#define OR_CAT_(a, b) a##b
#define OR_CAT(a, b) OR_CAT_(a, b)
#define FN(name) OR_CAT(OR_PREFIX, name)

typedef OR_REAL real;

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2 };

typedef struct {
  int n, nf, nstates, nsec;
  int *sec_of;   /* [nstates] sector of each bitstring */
  int *rank;     /* [nstates] position inside its sector (ascending bitstring) */
  int *sec_dim;  /* [nsec] */
  int *sec_off;  /* [nsec+1] offsets into states[] */
  int *states;   /* [nstates] bitstrings grouped by sector, ascending inside */
  real **H;      /* [nsec] dense d x d, row-major */
  real **V;      /* [nsec] eigenvectors, column j = eigenvector j, row-major */
  real **w;      /* [nsec] eigenvalues ascending */
  /* per sector: connected components of H's nonzero pattern; V is block
   * diagonal in them. Component c owns rows comp_rows[s][crow_off[s][c] ..]
   * and eigenvector columns comp_cols[s][crow_off[s][c] ..]. */
  int *ncomp;
  int **crow_off, **comp_rows, **comp_cols;
  real E0, beta;
  int nkept;
  int *kept_sec, *kept_col; /* kept eigenstates: sector and eigenvector column */
  real *kept_E;
} or_model;

static int popc(uint32_t x) {
  int c = 0;
  while (x) { x &= x - 1; ++c; }
  return c;
}

/* Apply c_f (dag = 0) or c_f^+ (dag = 1) to the basis state x.
 * Returns 0 if the result vanishes, else the new state in *y and the sign. */
static int apply_op(uint32_t x, int f, int dag, uint32_t *y, int *sign) {
  uint32_t bit = 1u << f;
  if (dag ? (x & bit) : !(x & bit)) return 0;
  *sign = (popc(x & (bit - 1u)) & 1) ? -1 : 1;
  *y = x ^ bit;
  return 1;
}

/* Apply the operator string ops[3] ops[2] ops[1] ops[0] with ops[0] acting
 * first (rightmost factor of the written product). */
static int apply_string(uint32_t x, const int *fl, const int *dg, int len, uint32_t *y, int *sign) {
  int s = 1;
  for (int i = 0; i < len; ++i) {
    int si;
    if (!apply_op(x, fl[i], dg[i], &x, &si)) return 0;
    s *= si;
  }
  *y = x;
  *sign = s;
  return 1;
}

/* Diagonal (density-density) part of Eq. (H_loc). */
static real diag_energy(uint32_t x, int n, real U, real J, real Up, real mu, const double *delta) {
  real e = 0;
  for (int a = 0; a < n; ++a) {
    int nu = (x >> (2 * a)) & 1, nd = (x >> (2 * a + 1)) & 1;
    e -= (mu + (real)delta[a]) * (real)(nu + nd);
    e += U * (real)(nu * nd);
  }
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < a; ++b)
      for (int s = 0; s < 2; ++s) {
        int nas = (x >> (2 * a + s)) & 1;
        int nbo = (x >> (2 * b + 1 - s)) & 1;
        int nbs = (x >> (2 * b + s)) & 1;
        e += Up * (real)(nas * nbo) + (Up - J) * (real)(nas * nbs);
      }
  return e;
}

/* ---------------------------------------------------------------------- */
/* Dense symmetric eigensolver: Householder tridiagonalisation followed by */
/* implicit symmetric QR steps with Wilkinson shift (Golub & Van Loan,     */
/* Algorithms 8.3.1 and 8.3.2). A is d x d row-major, destroyed. On exit  */
/* w holds the eigenvalues ascending and Q the eigenvectors as columns.    */
/* ---------------------------------------------------------------------- */
static int sym_eig(int d, real *A, real *w, real *Q) {
  real *v = (real *)malloc(sizeof(real) * (size_t)(d > 0 ? d : 1));
  real *p = (real *)malloc(sizeof(real) * (size_t)(d > 0 ? d : 1));
  real *e = (real *)calloc((size_t)(d > 0 ? d : 1), sizeof(real));
  int *perm = (int *)malloc(sizeof(int) * (size_t)(d > 0 ? d : 1));
  real *Qs = (real *)malloc(sizeof(real) * (size_t)(d > 0 ? d * d : 1));
  if (!v || !p || !e || !perm || !Qs) {
    free(v); free(p); free(e); free(perm); free(Qs);
    return OR_ENOMEM;
  }
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) Q[i * d + j] = (i == j) ? 1 : 0;

  /* Householder: annihilate A[k+2:, k] for k = 0..d-3. */
  for (int k = 0; k + 2 < d; ++k) {
    int m = d - k - 1; /* length of x = A[k+1:, k] */
    real alpha = 0;
    for (int i = 0; i < m; ++i) alpha += A[(k + 1 + i) * d + k] * A[(k + 1 + i) * d + k];
    alpha = sqrt(alpha);
    if (alpha == 0) continue;
    real x0 = A[(k + 1) * d + k];
    real sgn = (x0 >= 0) ? 1 : -1;
    /* v = x + sgn*alpha*e1, P = I - 2 v v^T / (v^T v) */
    for (int i = 0; i < m; ++i) v[i] = A[(k + 1 + i) * d + k];
    v[0] += sgn * alpha;
    real vv = 0;
    for (int i = 0; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0) continue;
    real beta = 2 / vv;
    /* A <- P A P on the full matrix (rows/cols k+1..d-1 affected). */
    /* left: A[k+1+i, j] -= beta v_i (v^T A[k+1:, j]) */
    for (int j = 0; j < d; ++j) {
      real s = 0;
      for (int i = 0; i < m; ++i) s += v[i] * A[(k + 1 + i) * d + j];
      s *= beta;
      for (int i = 0; i < m; ++i) A[(k + 1 + i) * d + j] -= s * v[i];
    }
    /* right: A[i, k+1+j] -= beta (A[i, k+1:] v) v_j */
    for (int i = 0; i < d; ++i) {
      real s = 0;
      for (int j = 0; j < m; ++j) s += A[i * d + k + 1 + j] * v[j];
      s *= beta;
      for (int j = 0; j < m; ++j) A[i * d + k + 1 + j] -= s * v[j];
    }
    /* accumulate Q <- Q P (columns k+1..d-1) */
    for (int i = 0; i < d; ++i) {
      real s = 0;
      for (int j = 0; j < m; ++j) s += Q[i * d + k + 1 + j] * v[j];
      s *= beta;
      for (int j = 0; j < m; ++j) Q[i * d + k + 1 + j] -= s * v[j];
    }
  }
  /* tridiagonal: diagonal in w, off-diagonal e[i] = T[i+1, i] */
  for (int i = 0; i < d; ++i) w[i] = A[i * d + i];
  for (int i = 0; i + 1 < d; ++i) e[i] = A[(i + 1) * d + i];

  /* implicit symmetric QR with Wilkinson shift */
  const real eps = (sizeof(real) > sizeof(double)) ? (real)1e-19 : (real)2.3e-16;
  int hi = d - 1;
  int guard = 0;
  while (hi > 0) {
    /* deflate negligible off-diagonals */
    for (int i = 0; i < hi; ++i)
      if (fabs(e[i]) <= eps * (fabs(w[i]) + fabs(w[i + 1]))) e[i] = 0;
    while (hi > 0 && e[hi - 1] == 0) --hi;
    if (hi == 0) break;
    int lo = hi - 1;
    while (lo > 0 && e[lo - 1] != 0) --lo;
    if (++guard > 100 * d + 1000) break;
    /* Wilkinson shift from trailing 2x2 of the block [lo, hi] */
    real dd = (w[hi - 1] - w[hi]) / 2;
    real b2 = e[hi - 1] * e[hi - 1];
    real sg = (dd >= 0) ? 1 : -1;
    real mu = w[hi] - b2 / (dd + sg * sqrt(dd * dd + b2));
    real x = w[lo] - mu, z = e[lo];
    for (int k = lo; k < hi; ++k) {
      /* Givens rotation zeroing z against x */
      real r = hypot(x, z);
      real c = (r == 0) ? 1 : x / r, s = (r == 0) ? 0 : -z / r;
      if (k > lo) e[k - 1] = r;
      /* apply G^T T G on rows/cols k, k+1 */
      real a11 = w[k], a22 = w[k + 1], a12 = e[k];
      real t11 = c * c * a11 - 2 * c * s * a12 + s * s * a22;
      real t22 = s * s * a11 + 2 * c * s * a12 + c * c * a22;
      real t12 = c * s * (a11 - a22) + (c * c - s * s) * a12;
      w[k] = t11; w[k + 1] = t22; e[k] = t12;
      if (k + 1 < hi) {
        x = e[k];
        z = -s * e[k + 1];
        e[k + 1] = c * e[k + 1];
      }
      /* accumulate eigenvectors: columns k, k+1 */
      for (int i = 0; i < d; ++i) {
        real qk = Q[i * d + k], qk1 = Q[i * d + k + 1];
        Q[i * d + k] = c * qk - s * qk1;
        Q[i * d + k + 1] = s * qk + c * qk1;
      }
    }
  }
  /* sort ascending */
  for (int i = 0; i < d; ++i) perm[i] = i;
  for (int i = 1; i < d; ++i) {
    int t = perm[i], j = i;
    while (j > 0 && w[perm[j - 1]] > w[t]) { perm[j] = perm[j - 1]; --j; }
    perm[j] = t;
  }
  memcpy(Qs, Q, sizeof(real) * (size_t)d * (size_t)d);
  for (int j = 0; j < d; ++j) v[j] = w[perm[j]];
  for (int j = 0; j < d; ++j) {
    w[j] = v[j];
    for (int i = 0; i < d; ++i) Q[i * d + j] = Qs[i * d + perm[j]];
  }
  free(v); free(p); free(e); free(perm); free(Qs);
  return OR_OK;
}

/* Eigendecomposition of one sector matrix H (d x d) into w (ascending) and
 * the columns of V. The sector is first split into the connected components
 * of the graph of H's nonzero entries: H is exactly block diagonal in them,
 * so each component is diagonalised on its own and V is zero across
 * components. (A joint FP64 decomposition would couple the decoupled
 * components at rounding level, and exp(dtau dE) growth over an imaginary-time
 * path can amplify that coupling beyond the true trace.) */
static int sector_eig(int d, const real *H, real *w, real *V, int *ncomp_out, int **off_out, int **rows_out,
                      int **cols_out) {
  int *comp = (int *)malloc(sizeof(int) * (size_t)(d > 0 ? d : 1));
  int *stack = (int *)malloc(sizeof(int) * (size_t)(d > 0 ? d : 1));
  int *idx = (int *)malloc(sizeof(int) * (size_t)(d > 0 ? d : 1));
  real *wv = (real *)malloc(sizeof(real) * (size_t)(d > 0 ? d : 1));
  real *A = (real *)malloc(sizeof(real) * (size_t)(d * d > 0 ? d * d : 1));
  real *Q = (real *)malloc(sizeof(real) * (size_t)(d * d > 0 ? d * d : 1));
  int *perm = (int *)malloc(sizeof(int) * (size_t)(d > 0 ? d : 1));
  real *Vt = (real *)malloc(sizeof(real) * (size_t)(d * d > 0 ? d * d : 1));
  int *col_comp = (int *)malloc(sizeof(int) * (size_t)(d > 0 ? d : 1));
  int *off = (int *)calloc((size_t)d + 2, sizeof(int));
  int *rows = (int *)malloc(sizeof(int) * (size_t)(d > 0 ? d : 1));
  int *cols = (int *)malloc(sizeof(int) * (size_t)(d > 0 ? d : 1));
  int rc = OR_OK;
  if (!comp || !stack || !idx || !wv || !A || !Q || !perm || !Vt || !col_comp || !off || !rows || !cols) rc = OR_ENOMEM;
  int ncomp = 0, col = 0;
  if (rc == OR_OK) {
    for (int i = 0; i < d; ++i) comp[i] = -1;
    for (int i = 0; i < d * d; ++i) Vt[i] = 0;
    for (int i0 = 0; i0 < d && rc == OR_OK; ++i0) {
      if (comp[i0] >= 0) continue;
      /* depth-first search over nonzero couplings */
      int top = 0, n = 0;
      stack[top++] = i0;
      comp[i0] = ncomp;
      while (top > 0) {
        int i = stack[--top];
        idx[n++] = i;
        for (int j = 0; j < d; ++j)
          if (comp[j] < 0 && (H[i * d + j] != 0 || H[j * d + i] != 0)) { comp[j] = ncomp; stack[top++] = j; }
      }
      for (int a = 1; a < n; ++a) { /* ascending row order inside the component */
        int t = idx[a], b = a;
        while (b > 0 && idx[b - 1] > t) { idx[b] = idx[b - 1]; --b; }
        idx[b] = t;
      }
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) A[a * n + b] = H[idx[a] * d + idx[b]];
      rc = sym_eig(n, A, wv, Q);
      for (int k = 0; k < n && rc == OR_OK; ++k, ++col) {
        w[col] = wv[k];
        col_comp[col] = ncomp;
        for (int a = 0; a < n; ++a) Vt[idx[a] * d + col] = Q[a * n + k];
      }
      ++ncomp;
    }
  }
  if (rc == OR_OK) { /* order all columns by eigenvalue */
    for (int i = 0; i < d; ++i) perm[i] = i;
    for (int i = 1; i < d; ++i) {
      int t = perm[i], j = i;
      while (j > 0 && w[perm[j - 1]] > w[t]) { perm[j] = perm[j - 1]; --j; }
      perm[j] = t;
    }
    for (int j = 0; j < d; ++j) wv[j] = w[perm[j]];
    for (int j = 0; j < d; ++j) {
      w[j] = wv[j];
      for (int i = 0; i < d; ++i) V[i * d + j] = Vt[i * d + perm[j]];
    }
    /* component CSR: rows in ascending order, columns in eigenvalue order */
    for (int i = 0; i < d; ++i) off[comp[i] + 1]++;
    for (int c = 0; c < ncomp; ++c) off[c + 1] += off[c];
    int *fill = stack; /* reuse as a cursor array */
    for (int c = 0; c < ncomp; ++c) fill[c] = off[c];
    for (int i = 0; i < d; ++i) rows[fill[comp[i]]++] = i;
    for (int c = 0; c < ncomp; ++c) fill[c] = off[c];
    for (int j = 0; j < d; ++j) cols[fill[col_comp[perm[j]]]++] = j;
  }
  free(comp); free(stack); free(idx); free(wv); free(A); free(Q); free(perm); free(Vt); free(col_comp);
  if (rc == OR_OK) {
    *ncomp_out = ncomp; *off_out = off; *rows_out = rows; *cols_out = cols;
  } else {
    free(off); free(rows); free(cols);
  }
  return rc;
}

/* ---------------------------------------------------------------------- */

void FN(model_free)(void *hm) {
  or_model *m = (or_model *)hm;
  if (!m) return;
  if (m->H) for (int s = 0; s < m->nsec; ++s) { free(m->H[s]); free(m->V[s]); free(m->w[s]); }
  free(m->H); free(m->V); free(m->w);
  if (m->crow_off)
    for (int s = 0; s < m->nsec; ++s) { free(m->crow_off[s]); free(m->comp_rows[s]); free(m->comp_cols[s]); }
  free(m->ncomp); free(m->crow_off); free(m->comp_rows); free(m->comp_cols);
  free(m->sec_of); free(m->rank); free(m->sec_dim); free(m->sec_off); free(m->states);
  free(m->kept_sec); free(m->kept_col); free(m->kept_E);
  free(m);
}

/* Build the model: sectors, dense H per sector, spectrum, kept multiplets.
 * flags bit 0: density-density only (spin-flip and pair-hopping dropped).
 * trunc_eps <= 0 keeps every eigenstate (untruncated trace). */
int FN(model_create)(int n, double U_, double J_, double Up_, double mu_, const double *delta,
                     double beta_, double trunc_eps, double deg_tol, int flags, void **out) {
  *out = NULL;
  if (n < 1 || n > 7) return OR_EINVAL;
  or_model *m = (or_model *)calloc(1, sizeof(or_model));
  if (!m) return OR_ENOMEM;
  real U = U_, J = J_, Up = Up_, mu = mu_;
  m->n = n; m->nf = 2 * n; m->nstates = 1 << (2 * n); m->nsec = (n + 1) * (n + 1);
  m->beta = beta_;
  m->sec_of = (int *)malloc(sizeof(int) * (size_t)m->nstates);
  m->rank = (int *)malloc(sizeof(int) * (size_t)m->nstates);
  m->states = (int *)malloc(sizeof(int) * (size_t)m->nstates);
  m->sec_dim = (int *)calloc((size_t)m->nsec, sizeof(int));
  m->sec_off = (int *)calloc((size_t)m->nsec + 1, sizeof(int));
  m->H = (real **)calloc((size_t)m->nsec, sizeof(real *));
  m->V = (real **)calloc((size_t)m->nsec, sizeof(real *));
  m->w = (real **)calloc((size_t)m->nsec, sizeof(real *));
  m->ncomp = (int *)calloc((size_t)m->nsec, sizeof(int));
  m->crow_off = (int **)calloc((size_t)m->nsec, sizeof(int *));
  m->comp_rows = (int **)calloc((size_t)m->nsec, sizeof(int *));
  m->comp_cols = (int **)calloc((size_t)m->nsec, sizeof(int *));
  if (!m->sec_of || !m->rank || !m->states || !m->sec_dim || !m->sec_off || !m->H || !m->V || !m->w || !m->ncomp ||
      !m->crow_off || !m->comp_rows || !m->comp_cols) {
    FN(model_free)(m);
    return OR_ENOMEM;
  }
  /* sector index = n_up * (n+1) + n_dn */
  for (int x = 0; x < m->nstates; ++x) {
    int nu = 0, nd = 0;
    for (int a = 0; a < n; ++a) { nu += (x >> (2 * a)) & 1; nd += (x >> (2 * a + 1)) & 1; }
    int s = nu * (n + 1) + nd;
    m->sec_of[x] = s;
    m->rank[x] = m->sec_dim[s]++;
  }
  for (int s = 0; s < m->nsec; ++s) m->sec_off[s + 1] = m->sec_off[s] + m->sec_dim[s];
  for (int x = 0; x < m->nstates; ++x) m->states[m->sec_off[m->sec_of[x]] + m->rank[x]] = x;

  for (int s = 0; s < m->nsec; ++s) {
    int d = m->sec_dim[s];
    m->H[s] = (real *)calloc((size_t)d * (size_t)d, sizeof(real));
    m->V[s] = (real *)calloc((size_t)d * (size_t)d, sizeof(real));
    m->w[s] = (real *)calloc((size_t)d, sizeof(real));
    if (!m->H[s] || !m->V[s] || !m->w[s]) { FN(model_free)(m); return OR_ENOMEM; }
    real *H = m->H[s];
    for (int i = 0; i < d; ++i) {
      uint32_t x = (uint32_t)m->states[m->sec_off[s] + i];
      H[i * d + i] += diag_energy(x, n, U, J, Up, mu, delta);
      if (flags & 1) continue;
      for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
          if (a == b) continue;
          uint32_t y;
          int sg;
          /* spin flip  psi+_{a dn} psi+_{b up} psi_{b dn} psi_{a up}  (rightmost acts first) */
          int f1[4] = {2 * a, 2 * b + 1, 2 * b, 2 * a + 1};
          int g1[4] = {0, 0, 1, 1};
          if (apply_string(x, f1, g1, 4, &y, &sg)) H[m->rank[y] * d + i] += -J * (real)sg;
          /* pair hop   psi+_{b up} psi+_{b dn} psi_{a up} psi_{a dn} */
          int f2[4] = {2 * a + 1, 2 * a, 2 * b + 1, 2 * b};
          int g2[4] = {0, 0, 1, 1};
          if (apply_string(x, f2, g2, 4, &y, &sg)) H[m->rank[y] * d + i] += -J * (real)sg;
        }
    }
    int rc = sector_eig(d, H, m->w[s], m->V[s], &m->ncomp[s], &m->crow_off[s], &m->comp_rows[s], &m->comp_cols[s]);
    if (rc) { FN(model_free)(m); return rc; }
  }
  /* global ground energy */
  m->E0 = INFINITY;
  for (int s = 0; s < m->nsec; ++s)
    if (m->sec_dim[s] > 0 && m->w[s][0] < m->E0) m->E0 = m->w[s][0];

  /* kept multiplets: sort all eigenvalues, group neighbours within deg_tol,
   * keep whole groups whose lowest member passes exp(-beta(E-E0)) >= eps */
  int N = m->nstates;
  int *idx = (int *)malloc(sizeof(int) * (size_t)N);
  int *isec = (int *)malloc(sizeof(int) * (size_t)N);
  int *icol = (int *)malloc(sizeof(int) * (size_t)N);
  real *ev = (real *)malloc(sizeof(real) * (size_t)N);
  if (!idx || !isec || !icol || !ev) { free(idx); free(isec); free(icol); free(ev); FN(model_free)(m); return OR_ENOMEM; }
  int c = 0;
  for (int s = 0; s < m->nsec; ++s)
    for (int j = 0; j < m->sec_dim[s]; ++j) { isec[c] = s; icol[c] = j; ev[c] = m->w[s][j]; idx[c] = c; ++c; }
  for (int i = 1; i < N; ++i) { /* insertion sort by energy (stable) */
    int t = idx[i], j = i;
    while (j > 0 && ev[idx[j - 1]] > ev[t]) { idx[j] = idx[j - 1]; --j; }
    idx[j] = t;
  }
  m->kept_sec = (int *)malloc(sizeof(int) * (size_t)N);
  m->kept_col = (int *)malloc(sizeof(int) * (size_t)N);
  m->kept_E = (real *)malloc(sizeof(real) * (size_t)N);
  if (!m->kept_sec || !m->kept_col || !m->kept_E) { free(idx); free(isec); free(icol); free(ev); FN(model_free)(m); return OR_ENOMEM; }
  m->nkept = 0;
  int i = 0;
  while (i < N) {
    int j = i + 1;
    while (j < N) {
      real a = ev[idx[j - 1]], b = ev[idx[j]];
      real scale = fabs(b) > 1 ? fabs(b) : 1;
      if (b - a <= (real)deg_tol * scale) ++j; else break;
    }
    real elow = ev[idx[i]];
    int keep = (trunc_eps <= 0) || (exp(-m->beta * (elow - m->E0)) >= (real)trunc_eps);
    if (!keep) break; /* energies ascend: nothing further passes */
    for (int k = i; k < j; ++k) {
      m->kept_sec[m->nkept] = isec[idx[k]];
      m->kept_col[m->nkept] = icol[idx[k]];
      m->kept_E[m->nkept] = ev[idx[k]];
      ++m->nkept;
    }
    i = j;
  }
  free(idx); free(isec); free(icol); free(ev);
  *out = m;
  return OR_OK;
}

int FN(model_dims)(void *hm, int *nstates, int *nsec, int *nkept, double *E0) {
  or_model *m = (or_model *)hm;
  *nstates = m->nstates; *nsec = m->nsec; *nkept = m->nkept; *E0 = (double)m->E0;
  return OR_OK;
}

/* Sector dims and the bitstrings in oracle order. */
int FN(model_sectors)(void *hm, int *sec_dim, int *states) {
  or_model *m = (or_model *)hm;
  for (int s = 0; s < m->nsec; ++s) sec_dim[s] = m->sec_dim[s];
  for (int x = 0; x < m->nstates; ++x) states[x] = m->states[x];
  return OR_OK;
}

/* Dense H, eigenvalues and eigenvectors of one sector (as double). */
int FN(model_block)(void *hm, int s, double *H, double *w, double *V) {
  or_model *m = (or_model *)hm;
  if (s < 0 || s >= m->nsec) return OR_EINVAL;
  int d = m->sec_dim[s];
  for (int i = 0; i < d * d; ++i) { if (H) H[i] = (double)m->H[s][i]; if (V) V[i] = (double)m->V[s][i]; }
  for (int i = 0; i < d; ++i) if (w) w[i] = (double)m->w[s][i];
  return OR_OK;
}

int FN(model_kept)(void *hm, int *sec, int *col, double *E) {
  or_model *m = (or_model *)hm;
  for (int k = 0; k < m->nkept; ++k) { sec[k] = m->kept_sec[k]; col[k] = m->kept_col[k]; E[k] = (double)m->kept_E[k]; }
  return OR_OK;
}

/* ---------------------------------------------------------------------- */
/* Trace of one sequence (Sec. III steps 3-8 with exact block exponentials) */
/* ---------------------------------------------------------------------- */

/* Apply c_f / c_f^+ to a vector living in sector s. Returns the target
 * sector, or -1 if the image is the zero vector. */
static int apply_vec(const or_model *m, int s, const real *v, int f, int dag, real *out) {
  int d = m->sec_dim[s];
  int t = -1;
  for (int i = 0; i < d; ++i) {
    uint32_t x = (uint32_t)m->states[m->sec_off[s] + i], y;
    int sg;
    if (!apply_op(x, f, dag, &y, &sg)) continue;
    if (t < 0) {
      t = m->sec_of[y];
      for (int j = 0; j < m->sec_dim[t]; ++j) out[j] = 0;
    }
    out[m->rank[y]] = (real)sg * v[i];
  }
  return t;
}

/* v <- exp(-dtau (H_s - w_ref)) v through the eigenbasis, where w_ref is
 * the lowest eigenvalue whose eigenvector overlaps v; returns the log of the
 * scalar exp(-dtau (w_ref - E0)) taken out. Eigenvectors without overlap
 * contribute exactly nothing. */
static real propagate(const or_model *m, int s, real dtau, real *v, real *tmp) {
  int d = m->sec_dim[s];
  const real *V = m->V[s], *w = m->w[s];
  const int *off = m->crow_off[s], *rows = m->comp_rows[s], *cols = m->comp_cols[s];
  /* V is block diagonal in the components: u = V^T v one component at a time */
  real wref = INFINITY;
  for (int c = 0; c < m->ncomp[s]; ++c)
    for (int b = off[c]; b < off[c + 1]; ++b) {
      int j = cols[b];
      real u = 0;
      for (int a = off[c]; a < off[c + 1]; ++a) u += V[rows[a] * d + j] * v[rows[a]];
      tmp[j] = u;
      if (u != 0 && w[j] < wref) wref = w[j];
    }
  if (!(wref < INFINITY)) return 0;
  for (int j = 0; j < d; ++j) tmp[j] = (tmp[j] != 0) ? tmp[j] * exp(-dtau * (w[j] - wref)) : 0;
  for (int c = 0; c < m->ncomp[s]; ++c)
    for (int a = off[c]; a < off[c + 1]; ++a) {
      int i = rows[a];
      real u = 0;
      for (int b = off[c]; b < off[c + 1]; ++b) u += V[i * d + cols[b]] * tmp[cols[b]];
      v[i] = u;
    }
  return -dtau * (wref - m->E0);
}

/* One sequence. Writes sign (-1, 0, +1), log|T| and log|T~|. */
static int trace_one(const or_model *m, int K, const double *tau, const uint8_t *flv, const uint8_t *dag,
                     real *va, real *vb, real *tmp, real *lg, int *sg, int *sign, double *logabs, double *logtt) {
  const real beta = m->beta;
  for (int k = 0; k < K; ++k) {
    if (flv[k] >= m->nf || !(tau[k] >= 0) || !(tau[k] < (double)beta)) return OR_EINVAL;
    if (k > 0 && tau[k] < tau[k - 1]) return OR_EINVAL;
  }
  int nalive = 0;
  for (int q = 0; q < m->nkept; ++q) {
    int s0 = m->kept_sec[q], col = m->kept_col[q];
    real En = m->kept_E[q];
    int d0 = m->sec_dim[s0];
    for (int i = 0; i < d0; ++i) va[i] = m->V[s0][i * d0 + col];
    real L = 0;
    int s = s0, alive = 1;
    if (K == 0) {
      L = -beta * (En - m->E0);
      lg[q] = L; sg[q] = 1; ++nalive;
      continue;
    }
    L += -(real)tau[0] * (En - m->E0);
    for (int k = 0; k < K; ++k) {
      int t = apply_vec(m, s, va, flv[k], dag[k], vb);
      if (t < 0) { alive = 0; break; }
      s = t;
      int d = m->sec_dim[s];
      real nrm = 0;
      for (int i = 0; i < d; ++i) nrm += vb[i] * vb[i];
      nrm = sqrt(nrm);
      if (nrm == 0) { alive = 0; break; }
      L += log(nrm);
      for (int i = 0; i < d; ++i) va[i] = vb[i] / nrm;
      if (k + 1 < K) {
        real dt = (real)tau[k + 1] - (real)tau[k];
        L += propagate(m, s, dt, va, tmp);
        nrm = 0;
        for (int i = 0; i < d; ++i) nrm += va[i] * va[i];
        nrm = sqrt(nrm);
        if (nrm == 0) { alive = 0; break; }
        L += log(nrm);
        for (int i = 0; i < d; ++i) va[i] /= nrm;
      }
    }
    if (!alive || s != s0) { sg[q] = 0; continue; }
    real ov = 0;
    for (int i = 0; i < d0; ++i) ov += m->V[s0][i * d0 + col] * va[i];
    if (ov == 0) { sg[q] = 0; continue; }
    L += log(fabs(ov)) - (beta - (real)tau[K - 1]) * (En - m->E0);
    lg[q] = L; sg[q] = (ov > 0) ? 1 : -1;
    ++nalive;
  }
  /* signed log-sum-exp over kept states */
  if (nalive == 0) { *sign = 0; *logabs = -INFINITY; *logtt = -INFINITY; return OR_OK; }
  real mx = -INFINITY;
  for (int q = 0; q < m->nkept; ++q) if (sg[q] && lg[q] > mx) mx = lg[q];
  real acc = 0;
  for (int q = 0; q < m->nkept; ++q) if (sg[q]) acc += (real)sg[q] * exp(lg[q] - mx);
  if (acc == 0) { *sign = 0; *logabs = -INFINITY; *logtt = -INFINITY; return OR_OK; }
  *sign = (acc > 0) ? 1 : -1;
  real lt = mx + log(fabs(acc));
  *logtt = (double)lt;
  *logabs = (double)(lt - beta * m->E0);
  return OR_OK;
}

/* Batch of sequences in CSR layout (offsets[nseq+1]); OpenMP over sequences.
 * status[i] = 0 or OR_EINVAL. Returns the number of threads used. */
int FN(trace_batch)(void *hm, int nseq, const int *offsets, const double *tau, const uint8_t *flavor,
                    const uint8_t *dagger, int *sign, double *logabs, double *logtt, int *status, int nthreads) {
  or_model *m = (or_model *)hm;
  int dmax = 1;
  for (int s = 0; s < m->nsec; ++s) if (m->sec_dim[s] > dmax) dmax = m->sec_dim[s];
  int used = 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
  {
#pragma omp single
    used = omp_get_num_threads();
#endif
    real *va = (real *)malloc(sizeof(real) * (size_t)dmax);
    real *vb = (real *)malloc(sizeof(real) * (size_t)dmax);
    real *tmp = (real *)malloc(sizeof(real) * (size_t)dmax);
    real *lg = (real *)malloc(sizeof(real) * (size_t)(m->nkept + 1));
    int *sg = (int *)malloc(sizeof(int) * (size_t)(m->nkept + 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int i = 0; i < nseq; ++i) {
      int o = offsets[i], K = offsets[i + 1] - offsets[i];
      double la = 0, lt = 0;
      int sgn = 0;
      int rc = (va && vb && tmp && lg && sg) ? trace_one(m, K, tau + o, flavor + o, dagger + o, va, vb, tmp, lg, sg, &sgn, &la, &lt)
                                             : OR_ENOMEM;
      sign[i] = sgn; logabs[i] = la; if (logtt) logtt[i] = lt; status[i] = rc;
    }
    free(va); free(vb); free(tmp); free(lg); free(sg);
#ifdef _OPENMP
  }
#endif
  return used;
}

/* ---------------------------------------------------------------------- */
/* Diagonal observables inserted at tau = t_obs (Sec. III: measurements at  */
/* beta/2 in the truncated trace)                                          */
/* ---------------------------------------------------------------------- */

/* T_O = sum over kept |n> of <n| e^{-(beta-tau_K)(H-E0)} O_K ... O(t_obs) ...
 * O_1 e^{-tau_1 (H-E0)} |n>, with the diagonal operator O (values obs[x] on
 * bitstring x) placed after every operator with tau < t_obs. The product is
 * evaluated right to left as written: every interval that starts from a
 * vector other than the kept eigenstate is an exact block exponential. */
static int trace_obs_one(const or_model *m, int K, const double *tau, const uint8_t *flv, const uint8_t *dag,
                         real t_obs, const double *obs, real *va, real *vb, real *tmp, real *lg, int *sg,
                         int *sign, double *logabs) {
  const real beta = m->beta;
  for (int k = 0; k < K; ++k) {
    if (flv[k] >= m->nf || !(tau[k] >= 0) || !(tau[k] < (double)beta)) return OR_EINVAL;
    if (k > 0 && tau[k] < tau[k - 1]) return OR_EINVAL;
  }
  if (!(t_obs >= 0) || !(t_obs <= beta)) return OR_EINVAL;
  int mcut = 0;
  while (mcut < K && (real)tau[mcut] < t_obs) ++mcut;
  int nalive = 0;
  for (int q = 0; q < m->nkept; ++q) {
    int s0 = m->kept_sec[q], col = m->kept_col[q];
    real En = m->kept_E[q];
    int d0 = m->sec_dim[s0];
    for (int i = 0; i < d0; ++i) va[i] = m->V[s0][i * d0 + col];
    real L = 0, t = 0;
    int s = s0, alive = 1, eig = 1;
    /* events: ops 0 .. mcut-1, the observable, ops mcut .. K-1 */
    for (int e = 0; e <= K && alive; ++e) {
      const int is_obs = (e == mcut);
      const int k = e < mcut ? e : e - 1;
      const real te = is_obs ? t_obs : (real)tau[k];
      if (te > t) {
        if (eig) {
          L += -(te - t) * (En - m->E0);
        } else {
          L += propagate(m, s, te - t, va, tmp);
        }
      }
      t = te;
      int d = m->sec_dim[s];
      if (is_obs) {
        for (int i = 0; i < d; ++i) vb[i] = va[i] * (real)obs[m->states[m->sec_off[s] + i]];
      } else {
        int tg = apply_vec(m, s, va, flv[k], dag[k], vb);
        if (tg < 0) { alive = 0; break; }
        s = tg;
        d = m->sec_dim[s];
      }
      eig = 0;
      real nrm = 0;
      for (int i = 0; i < d; ++i) nrm += vb[i] * vb[i];
      nrm = sqrt(nrm);
      if (nrm == 0) { alive = 0; break; }
      L += log(nrm);
      for (int i = 0; i < d; ++i) va[i] = vb[i] / nrm;
    }
    if (!alive || s != s0) { sg[q] = 0; continue; }
    /* last interval: <n| e^{-(beta - t)(H - E0)} = e^{-(beta - t)(E_n - E0)} <n| */
    real ov = 0;
    for (int i = 0; i < d0; ++i) ov += m->V[s0][i * d0 + col] * va[i];
    if (ov == 0) { sg[q] = 0; continue; }
    L += log(fabs(ov)) - (beta - t) * (En - m->E0);
    lg[q] = L; sg[q] = (ov > 0) ? 1 : -1;
    ++nalive;
  }
  if (nalive == 0) { *sign = 0; *logabs = -INFINITY; return OR_OK; }
  real mx = -INFINITY;
  for (int q = 0; q < m->nkept; ++q) if (sg[q] && lg[q] > mx) mx = lg[q];
  real acc = 0;
  for (int q = 0; q < m->nkept; ++q) if (sg[q]) acc += (real)sg[q] * exp(lg[q] - mx);
  if (acc == 0) { *sign = 0; *logabs = -INFINITY; return OR_OK; }
  *sign = (acc > 0) ? 1 : -1;
  *logabs = (double)(mx + log(fabs(acc)) - beta * m->E0);
  return OR_OK;
}

/* Batch: for every sequence i and observable j (obs[j * nstates + x]),
 * sign[i * nobs + j] and logabs[i * nobs + j] of T_O. status[i] as
 * trace_batch. Returns the number of threads used. */
int FN(trace_obs_batch)(void *hm, int nseq, const int *offsets, const double *tau, const uint8_t *flavor,
                        const uint8_t *dagger, double t_obs, int nobs, const double *obs, int *sign, double *logabs,
                        int *status, int nthreads) {
  or_model *m = (or_model *)hm;
  int dmax = 1;
  for (int s = 0; s < m->nsec; ++s) if (m->sec_dim[s] > dmax) dmax = m->sec_dim[s];
  int used = 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
  {
#pragma omp single
    used = omp_get_num_threads();
#endif
    real *va = (real *)malloc(sizeof(real) * (size_t)dmax);
    real *vb = (real *)malloc(sizeof(real) * (size_t)dmax);
    real *tmp = (real *)malloc(sizeof(real) * (size_t)dmax);
    real *lg = (real *)malloc(sizeof(real) * (size_t)(m->nkept + 1));
    int *sg = (int *)malloc(sizeof(int) * (size_t)(m->nkept + 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1) collapse(2)
#endif
    for (int i = 0; i < nseq; ++i)
      for (int j = 0; j < nobs; ++j) {
        int o = offsets[i], K = offsets[i + 1] - offsets[i];
        double la = 0;
        int sgn = 0;
        int rc = (va && vb && tmp && lg && sg)
                     ? trace_obs_one(m, K, tau + o, flavor + o, dagger + o, (real)t_obs, obs + (size_t)j * m->nstates,
                                     va, vb, tmp, lg, sg, &sgn, &la)
                     : OR_ENOMEM;
        sign[(size_t)i * nobs + j] = sgn;
        logabs[(size_t)i * nobs + j] = la;
        if (j == 0) status[i] = rc;
      }
    free(va); free(vb); free(tmp); free(lg); free(sg);
#ifdef _OPENMP
  }
#endif
  return used;
}

/* ---------------------------------------------------------------------- */
/* A general operator that conserves (n_up, n_dn), inserted at tau = t_obs  */
/* ---------------------------------------------------------------------- */

/* As trace_obs_one, with the operator given as a dense matrix over all
 * bitstrings (op[y * nstates + x] = <y|O|x>) that maps each (n_up, n_dn)
 * sector into itself. */
static int trace_op_one(const or_model *m, int K, const double *tau, const uint8_t *flv, const uint8_t *dag,
                        real t_obs, const double *op, real *va, real *vb, real *tmp, real *lg, int *sg, int *sign,
                        double *logabs) {
  const real beta = m->beta;
  for (int k = 0; k < K; ++k) {
    if (flv[k] >= m->nf || !(tau[k] >= 0) || !(tau[k] < (double)beta)) return OR_EINVAL;
    if (k > 0 && tau[k] < tau[k - 1]) return OR_EINVAL;
  }
  if (!(t_obs >= 0) || !(t_obs <= beta)) return OR_EINVAL;
  int mcut = 0;
  while (mcut < K && (real)tau[mcut] < t_obs) ++mcut;
  int nalive = 0;
  for (int q = 0; q < m->nkept; ++q) {
    int s0 = m->kept_sec[q], col = m->kept_col[q];
    real En = m->kept_E[q];
    int d0 = m->sec_dim[s0];
    for (int i = 0; i < d0; ++i) va[i] = m->V[s0][i * d0 + col];
    real L = 0, t = 0;
    int s = s0, alive = 1, eig = 1;
    for (int e = 0; e <= K && alive; ++e) {
      const int is_obs = (e == mcut);
      const int k = e < mcut ? e : e - 1;
      const real te = is_obs ? t_obs : (real)tau[k];
      if (te > t) {
        if (eig) L += -(te - t) * (En - m->E0);
        else L += propagate(m, s, te - t, va, tmp);
      }
      t = te;
      int d = m->sec_dim[s];
      if (is_obs) {
        const int *st = m->states + m->sec_off[s];
        for (int i = 0; i < d; ++i) {
          real acc = 0;
          for (int j = 0; j < d; ++j) acc += (real)op[(size_t)st[i] * m->nstates + st[j]] * va[j];
          vb[i] = acc;
        }
      } else {
        int tg = apply_vec(m, s, va, flv[k], dag[k], vb);
        if (tg < 0) { alive = 0; break; }
        s = tg;
        d = m->sec_dim[s];
      }
      eig = 0;
      real nrm = 0;
      for (int i = 0; i < d; ++i) nrm += vb[i] * vb[i];
      nrm = sqrt(nrm);
      if (nrm == 0) { alive = 0; break; }
      L += log(nrm);
      for (int i = 0; i < d; ++i) va[i] = vb[i] / nrm;
    }
    if (!alive || s != s0) { sg[q] = 0; continue; }
    real ov = 0;
    for (int i = 0; i < d0; ++i) ov += m->V[s0][i * d0 + col] * va[i];
    if (ov == 0) { sg[q] = 0; continue; }
    L += log(fabs(ov)) - (beta - t) * (En - m->E0);
    lg[q] = L; sg[q] = (ov > 0) ? 1 : -1;
    ++nalive;
  }
  if (nalive == 0) { *sign = 0; *logabs = -INFINITY; return OR_OK; }
  real mx = -INFINITY;
  for (int q = 0; q < m->nkept; ++q) if (sg[q] && lg[q] > mx) mx = lg[q];
  real acc = 0;
  for (int q = 0; q < m->nkept; ++q) if (sg[q]) acc += (real)sg[q] * exp(lg[q] - mx);
  if (acc == 0) { *sign = 0; *logabs = -INFINITY; return OR_OK; }
  *sign = (acc > 0) ? 1 : -1;
  *logabs = (double)(mx + log(fabs(acc)) - beta * m->E0);
  return OR_OK;
}

int FN(trace_op_batch)(void *hm, int nseq, const int *offsets, const double *tau, const uint8_t *flavor,
                       const uint8_t *dagger, double t_obs, const double *op, int *sign, double *logabs, int *status,
                       int nthreads) {
  or_model *m = (or_model *)hm;
  int dmax = 1;
  for (int s = 0; s < m->nsec; ++s) if (m->sec_dim[s] > dmax) dmax = m->sec_dim[s];
  int used = 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
  {
#pragma omp single
    used = omp_get_num_threads();
#endif
    real *va = (real *)malloc(sizeof(real) * (size_t)dmax);
    real *vb = (real *)malloc(sizeof(real) * (size_t)dmax);
    real *tmp = (real *)malloc(sizeof(real) * (size_t)dmax);
    real *lg = (real *)malloc(sizeof(real) * (size_t)(m->nkept + 1));
    int *sg = (int *)malloc(sizeof(int) * (size_t)(m->nkept + 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int i = 0; i < nseq; ++i) {
      int o = offsets[i], K = offsets[i + 1] - offsets[i];
      double la = 0;
      int sgn = 0;
      int rc = (va && vb && tmp && lg && sg)
                   ? trace_op_one(m, K, tau + o, flavor + o, dagger + o, (real)t_obs, op, va, vb, tmp, lg, sg, &sgn, &la)
                   : OR_ENOMEM;
      sign[i] = sgn; logabs[i] = la; status[i] = rc;
    }
    free(va); free(vb); free(tmp); free(lg); free(sg);
#ifdef _OPENMP
  }
#endif
  return used;
}
