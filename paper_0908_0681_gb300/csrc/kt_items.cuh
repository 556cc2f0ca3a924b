// Krylov items kernel templates (internal; instantiated per precision in
// kt_items_f32.cu and kt_items_f64.cu so the two compile in parallel).
#pragma once

#include "kt_device.cuh"

namespace kt {
namespace dev {

// ---------------------------------------------------------------------------
// 3. Krylov items
//
// G lanes cooperate on one (walker, kept state) item; a warp holds 32/G items.
// Vector rows are spread over the G lanes of the item (row r on lane r % G).
// With small G every FP64 instruction of the scalar part (tridiagonal
// exponential, norms, log-weights) serves several items at once, which
// matters on GB300 where an FP64 warp instruction occupies the SM's FP64 pipe
// for 16 cycles however many lanes are active.
// Shared memory is interleaved item-minor: element e of item g of a warp lives
// at e * IPW + g, so lanes of different items touch consecutive words.
// ---------------------------------------------------------------------------
template <typename VT, int G, int DMAX, int PMAX>
struct WarpTile {
  static constexpr int IPW = 32 / G;
  VT q[(PMAX + 1) * DMAX * IPW];  // Lanczos basis; basis vector 0 carries the state between intervals
  double a[PMAX * IPW], b[PMAX * IPW];            // T_p: diagonal alpha, off-diagonal beta (FP64)
  double dd[PMAX * IPW], ee[PMAX * IPW];          // FP64 QL workspace -> Ritz values
  double ex[PMAX * IPW], y[PMAX * IPW];           // exp(-dt T_p) e_1 (scaled) and helpers
  double S[PMAX * PMAX * IPW];                     // FP64 Ritz vectors (FP64 path)
  float d32[PMAX * IPW], e32[PMAX * IPW], y32[PMAX * IPW], x32[PMAX * IPW];
  float S32[PMAX * PMAX * IPW];                   // FP32 Ritz vectors (FP32 path)
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

// Register budget of the items kernels: the FP32 warp tiles let two 256-thread CTAs share an
// SM (at most 128 registers a thread); the FP64 tiles take more than half of the shared
// memory, so one CTA per SM runs anyway and its threads may use the registers of two
#define KT_MIN_CTAS(VT) (sizeof(VT) == 8 ? 1 : 2)

// Compile-time options of the items kernels (OPT): the code a launch does not need is not in
// its instance, which keeps the hot loop's instructions together (a smaller kernel, fewer
// instruction-fetch stalls). KT_OPT_TRI64: the FP64 tridiagonal steps of KT_FP32_TRIDIAG64
// (FP32 path, blocks of at most 16 rows); KT_OPT_MEAS: the observables at beta/2;
// KT_OPT_STATS: the work counters of kt_stats.
constexpr int KT_OPT_TRI64 = 1, KT_OPT_MEAS = 2, KT_OPT_STATS = 4;

template <int G, typename T>
__device__ __forceinline__ T gsum(T v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

// Error-free transformations on the FP32 pipe (Knuth TwoSum, TwoProduct via
// fmaf). A value hi + lo carries about 48 significant bits.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
struct DF {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_prod(float x, float y) {
    const float p = x * y, pe = fmaf(x, y, -p);
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo += e + pe;
  }
  __device__ __forceinline__ void add(const DF &o) {
    float s, e;
    two_sum(hi, o.hi, s, e);
    hi = s;
    lo += e + o.lo;
  }
};
template <int G>
__device__ __forceinline__ DF gsum_df(DF v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    DF w;
    w.hi = __shfl_xor_sync(mask, v.hi, o);
    w.lo = __shfl_xor_sync(mask, v.lo, o);
    v.add(w);
  }
  return v;
}
// sqrt of a double-float, one Newton correction on the FP32 pipe.
__device__ __forceinline__ DF sqrt_df(DF v) {
  DF r;
  if (!(v.hi > 0.f)) return r;
  const float s = sqrtf(v.hi);
  const float s2 = s * s, s2e = fmaf(s, s, -s2);
  r.hi = s;
  r.lo = ((v.hi - s2) - s2e + v.lo) / (2.f * s);
  return r;
}
__device__ __forceinline__ double df_value(const DF &v) { return (double)v.hi + (double)v.lo; }

// Double-float arithmetic (Dekker / Knuth; about 44 significant bits), used on the FP32
// path for the tridiagonal scalars so that no FP64 instruction sits in the interval loop.
__device__ __forceinline__ DF df_norm(float hi, float lo) {  // fast two-sum, |hi| >= |lo|
  DF r;
  r.hi = hi + lo;
  r.lo = lo - (r.hi - hi);
  return r;
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return df_norm(s, e + a.lo + b.lo);
}
__device__ __forceinline__ DF df_neg(DF a) {
  a.hi = -a.hi;
  a.lo = -a.lo;
  return a;
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.hi * b.hi;
  return df_norm(p, fmaf(a.hi, b.hi, -p) + fmaf(a.hi, b.lo, a.lo * b.hi));
}
__device__ __forceinline__ DF df_mulf(DF a, float b) {
  const float p = a.hi * b;
  return df_norm(p, fmaf(a.hi, b, -p) + a.lo * b);
}
__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float q1 = a.hi / b.hi;
  const DF r = df_add(a, df_neg(df_mulf(b, q1)));
  return df_norm(q1, r.hi / b.hi);
}
__device__ __forceinline__ bool df_lt(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// Group-reduced dot product with FP64 accuracy: double-float on the FP32 pipe
// for FP32 vectors, FP64 FMA for FP64 vectors.
template <typename VT, int G>
struct GroupDot;
template <int G>
struct GroupDot<float, G> {
  DF acc;
  __device__ __forceinline__ void add(float x, float y) { acc.add_prod(x, y); }
  __device__ __forceinline__ double value(unsigned gm) { return df_value(gsum_df<G>(acc, gm)); }
  __device__ __forceinline__ double norm(unsigned gm) { return df_value(sqrt_df(gsum_df<G>(acc, gm))); }
  __device__ __forceinline__ DF value_df(unsigned gm) {
    const DF v = gsum_df<G>(acc, gm);
    return df_norm(v.hi, v.lo);
  }
  __device__ __forceinline__ DF norm_df(unsigned gm) {
    const DF v = sqrt_df(gsum_df<G>(acc, gm));
    return df_norm(v.hi, v.lo);
  }
};
template <int G>
struct GroupDot<double, G> {
  double acc = 0.0;
  __device__ __forceinline__ void add(double x, double y) { acc = fma(x, y, acc); }
  __device__ __forceinline__ double value(unsigned gm) { return gsum<G>(acc, gm); }
  __device__ __forceinline__ double norm(unsigned gm) { return sqrt(gsum<G>(acc, gm)); }
};

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

// Rotation (c, s) with c x - s z = r, s x + c z = 0.
template <typename R>
__device__ __forceinline__ void givens(R x, R z, R &c, R &s, R &r) {
  const R r2 = x * x + z * z;
  if (r2 == R(0)) {
    c = R(1); s = R(0); r = R(0);
    return;
  }
  const R inv = rsq(r2);
  c = x * inv;
  s = -z * inv;
  r = r2 * inv;
}

// Product of positive factors kept as mantissa * 2^exponent (no log per step).
// The mantissa is renormalised into [1, 2) by editing its exponent bits.
struct LogScale {
  double m = 1.0;
  int e = 0;
  __device__ __forceinline__ void mul(double f) {
    const long long bits = __double_as_longlong(m * f);
    e += (int)((bits >> 52) & 0x7ff) - 1023;
    m = __longlong_as_double((bits & 0x800fffffffffffffLL) | 0x3ff0000000000000LL);
  }
  __device__ __forceinline__ double log_value() const { return log(m) + (double)e * 0.69314718055994530942; }
};

// Exact power of two 2^-floor(log2 m) for a positive finite m (normal or not).
__device__ __forceinline__ float pow2_inv(float m) {
  if (m >= 1.17549435e-38f) return __int_as_float((254 - ((__float_as_int(m) >> 23) & 0xff)) << 23);
  return scalbnf(1.f, -ilogbf(m));
}
__device__ __forceinline__ double pow2_inv(double m) { return scalbn(1.0, -ilogb(m)); }

// Scale the item's rows v to unit norm and multiply the factor actually applied into
// `applied`. Usually one group reduction of the sum of squares and an rsqrt; when that
// sum is tiny or huge, an exact power-of-two prescale first brings the largest entry to
// [1, 2). False if all rows are zero.
template <typename VT, int G, int R>
__device__ __forceinline__ bool normalize_rows(VT (&v)[R], int gl, int dim, unsigned gm, LogScale &applied) {
  constexpr VT lo = sizeof(VT) == 4 ? VT(1e-30) : VT(1e-290), hi = sizeof(VT) == 4 ? VT(1e30) : VT(1e290);
  VT n2 = VT(0);
#pragma unroll
  for (int j = 0; j < R; ++j)
    if (gl + G * j < dim) n2 += v[j] * v[j];
  n2 = gsum<G>(n2, gm);
  VT sc;
  if (n2 > lo && n2 < hi) {
    sc = rsq(n2);
  } else {
    VT m = VT(0);
#pragma unroll
    for (int j = 0; j < R; ++j)
      if (gl + G * j < dim) m = fmax(m, fabs(v[j]));
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(gm, m, o));
    if (!(m > VT(0))) return false;
    const VT s1 = pow2_inv(m);
    n2 = VT(0);
#pragma unroll
    for (int j = 0; j < R; ++j)
      if (gl + G * j < dim) {
        const VT t = v[j] * s1;
        n2 += t * t;
      }
    n2 = gsum<G>(n2, gm);
    sc = s1 * rsq(n2);
  }
#pragma unroll
  for (int j = 0; j < R; ++j) v[j] *= sc;
  applied.mul((double)sc);
  return true;
}

// Symmetric tridiagonal eigensolver of one item, precision R: implicit QL
// sweeps with the shift from the leading 2x2 block. On entry d holds the
// diagonal and e the off-diagonal (e[p-1] = 0); on exit d holds the Ritz
// values and S(k, i) component i of Ritz vector k (spread over the group's
// lanes). Arrays are item-interleaved with stride IPW. False if it did not
// converge.
template <typename R, int G, int PMAX>
__device__ bool tri_eig(R *d, R *e, R *S, int grp, int gl, unsigned gm, int p) {
  constexpr int IPW = 32 / G;
#define D_(k) d[(k) * IPW + grp]
#define E_(k) e[(k) * IPW + grp]
#define S_(k, i) S[((k) * PMAX + (i)) * IPW + grp]
  for (int i = gl; i < p; i += G)
    for (int k = 0; k < p; ++k) S_(k, i) = (i == k) ? R(1) : R(0);
  __syncwarp(gm);
  const R eps = sizeof(R) == 8 ? R(2.3e-16) : R(1.2e-7);
  int lo = 0, guard = 0;
  bool ok = true;
  while (lo < p - 1) {
    if (fabs(E_(lo)) <= eps * (fabs(D_(lo)) + fabs(D_(lo + 1)))) {
      ++lo;
      continue;
    }
    int hi = lo + 1;
    while (hi < p - 1 && fabs(E_(hi)) > eps * (fabs(D_(hi)) + fabs(D_(hi + 1)))) ++hi;
    if (++guard > 40 * p) {
      ok = false;
      break;
    }
    const R b0 = E_(lo);
    const R dm = R(0.5) * (D_(lo + 1) - D_(lo));
    const R mu = D_(lo) - b0 * b0 / (dm + copysign(sqrt(dm * dm + b0 * b0), dm));
    R x = D_(hi) - mu, z = E_(hi - 1);
    for (int k = hi; k > lo; --k) {
      R c, sn, r;
      givens(x, z, c, sn, r);
      const R a11 = D_(k), a22 = D_(k - 1), a12 = E_(k - 1);
      const R ek2 = (k - 1 > lo) ? E_(k - 2) : R(0);
      const R cc = c * c, ss = sn * sn, cs = c * sn;
      const R n11 = cc * a11 - R(2) * cs * a12 + ss * a22;
      const R n22 = ss * a11 + R(2) * cs * a12 + cc * a22;
      const R n12 = cs * (a11 - a22) + (cc - ss) * a12;
      __syncwarp(gm);
      if (gl == 0) {
        if (k < hi) E_(k) = r;
        D_(k) = n11;
        D_(k - 1) = n22;
        E_(k - 1) = n12;
        if (k - 1 > lo) E_(k - 2) = c * ek2;
      }
      for (int i = gl; i < p; i += G) {
        const R vk = S_(k, i), vk1 = S_(k - 1, i);
        S_(k, i) = c * vk - sn * vk1;
        S_(k - 1, i) = sn * vk + c * vk1;
      }
      __syncwarp(gm);
      if (k - 1 > lo) {
        x = n12;
        z = -sn * ek2;
      }
    }
  }
  __syncwarp(gm);
  return ok;
#undef D_
#undef E_
#undef S_
}

// 2x2 symmetric [[a, b], [b, c]]: y = exp(-dt T) e_1 / exp(-dt lambda_min),
// returns -dt lambda_min.
template <typename R>
__device__ __forceinline__ R exp2x2(R a, R c, R b, R dt, R &y0, R &y1) {
  const R m = R(0.5) * (a + c), h = R(0.5) * (a - c);
  const R r = sqrt(h * h + b * b);
  const R E = exp(R(-2) * dt * r);
  const R g = (r > R(0)) ? -expm1(R(-2) * dt * r) / (R(2) * r) : dt;
  y0 = R(0.5) * (R(1) + E) - g * h;
  y1 = -g * b;
  return -dt * (m - r);
}

// FP32 path, p <= 2. The Ritz values and the scale exp(-dt lambda_min) (kept
// in log space) are FP64; the relative weights exp(-dt (lambda - lambda_min))
// in (0, 1] and y are formed in FP32, the precision of the Krylov vectors they
// multiply. y lands in y32.
template <typename VT, int G, int DMAX, int PMAX>
__device__ __forceinline__ void tri_small_f32(WarpTile<VT, G, DMAX, PMAX> &s, int grp, int gl, unsigned gm, int p,
                                              double dt, double &logfac) {
  constexpr int IPW = 32 / G;
  const float2 *af = reinterpret_cast<const float2 *>(s.a), *bf = reinterpret_cast<const float2 *>(s.b);
  float y0 = 1.f, y1 = 0.f;
  if (p == 1) {
    logfac = -dt * ((double)af[grp].x + (double)af[grp].y);
  } else {
    DF a, c, b;
    a.hi = af[grp].x; a.lo = af[grp].y;
    c.hi = af[IPW + grp].x; c.lo = af[IPW + grp].y;
    b.hi = bf[grp].x; b.lo = bf[grp].y;
    const DF m = df_mulf(df_add(a, c), 0.5f), h = df_mulf(df_add(a, df_neg(c)), 0.5f);
    const DF r = sqrt_df(df_add(df_mul(h, h), df_mul(b, b)));
    const DF lmin = df_add(m, df_neg(r));
    logfac = -dt * ((double)lmin.hi + (double)lmin.lo);
    const float x = 2.f * (float)dt * r.hi;  // dt (lambda_+ - lambda_-)
    const float E = expf(-x);
    const float g = (x > 1e-3f) ? (1.f - E) / (2.f * r.hi) : (float)dt * (1.f - 0.5f * x);
    y0 = 0.5f * (1.f + E) - g * h.hi;
    y1 = -g * b.hi;
  }
  if (gl == 0) {
    s.y32[grp] = y0;
    s.y32[IPW + grp] = y1;
  }
  __syncwarp(gm);
}

// FP64 y = exp(-dt T_p) e_1 / exp(-dt lambda_min) from a full FP64 QL (FP64 path).
template <typename VT, int G, int DMAX, int PMAX>
__device__ bool tri_exp64(WarpTile<VT, G, DMAX, PMAX> &s, int grp, int gl, unsigned gm, int p, double dt,
                          double &logfac) {
  constexpr int IPW = 32 / G;
#define A_(k) s.a[(k) * IPW + grp]
#define B_(k) s.b[(k) * IPW + grp]
#define D_(k) s.dd[(k) * IPW + grp]
#define E_(k) s.ee[(k) * IPW + grp]
#define X_(k) s.ex[(k) * IPW + grp]
#define Y_(k) s.y[(k) * IPW + grp]
#define S_(k, i) s.S[((k) * PMAX + (i)) * IPW + grp]
  if (p == 1) {
    if (gl == 0) Y_(0) = 1.0;
    logfac = -dt * A_(0);
    __syncwarp(gm);
    return true;
  }
  if (p == 2) {
    double y0, y1;
    logfac = exp2x2(A_(0), A_(1), B_(0), dt, y0, y1);
    if (gl == 0) {
      Y_(0) = y0;
      Y_(1) = y1;
    }
    __syncwarp(gm);
    return true;
  }
  for (int i = gl; i < p; i += G) {
    D_(i) = A_(i);
    E_(i) = (i + 1 < p) ? B_(i) : 0.0;
  }
  __syncwarp(gm);
  const bool ok = tri_eig<double, G, PMAX>(s.dd, s.ee, s.S, grp, gl, gm, p);
  double lmin = D_(0);
  for (int k = 1; k < p; ++k) lmin = fmin(lmin, D_(k));
  for (int k = gl; k < p; k += G) X_(k) = exp(-dt * (D_(k) - lmin)) * S_(k, 0);
  __syncwarp(gm);
  for (int i = gl; i < p; i += G) {
    double acc = 0.0;
    for (int k = 0; k < p; ++k) acc = fma(S_(k, i), X_(k), acc);
    Y_(i) = acc;
  }
  logfac = -dt * lmin;
  __syncwarp(gm);
  return ok;
#undef A_
#undef B_
#undef D_
#undef E_
#undef X_
#undef Y_
#undef S_
}

// FP32-path convergence estimate: ||y|| and |y_{p-1}| of exp(-dt T_p) e_1 from
// an FP32 eigendecomposition (the estimate needs about one significant digit).
// For p >= 3 the FP32 Ritz pairs are left in d32 / S32 for the final step.
template <typename VT, int G, int DMAX, int PMAX>
__device__ void tri_check32(WarpTile<VT, G, DMAX, PMAX> &s, int grp, int gl, unsigned gm, int p, double dt,
                            float &ynorm, float &ylast) {
  constexpr int IPW = 32 / G;
#define AF_(k) reinterpret_cast<float2 *>(s.a)[(k) * IPW + grp]
#define BF_(k) reinterpret_cast<float2 *>(s.b)[(k) * IPW + grp]
#define D_(k) s.d32[(k) * IPW + grp]
#define E_(k) s.e32[(k) * IPW + grp]
#define X_(k) s.x32[(k) * IPW + grp]
#define Y_(k) s.y32[(k) * IPW + grp]
#define S_(k, i) s.S32[((k) * PMAX + (i)) * IPW + grp]
  if (p == 1) {
    ynorm = 1.f;
    ylast = 1.f;
    return;
  }
  if (p == 2) {
    float y0, y1;
    exp2x2(AF_(0).x, AF_(1).x, BF_(0).x, (float)dt, y0, y1);
    ynorm = sqrtf(y0 * y0 + y1 * y1);
    ylast = fabsf(y1);
    return;
  }
  for (int i = gl; i < p; i += G) {
    D_(i) = AF_(i).x;
    E_(i) = (i + 1 < p) ? BF_(i).x : 0.f;
  }
  __syncwarp(gm);
  tri_eig<float, G, PMAX>(s.d32, s.e32, s.S32, grp, gl, gm, p);
  float lmin = D_(0);
  for (int k = 1; k < p; ++k) lmin = fminf(lmin, D_(k));
  for (int k = gl; k < p; k += G) X_(k) = expf(-(float)dt * (D_(k) - lmin)) * S_(k, 0);
  __syncwarp(gm);
  float yn = 0.f;
  for (int i = gl; i < p; i += G) {
    float acc = 0.f;
    for (int k = 0; k < p; ++k) acc = fmaf(S_(k, i), X_(k), acc);
    Y_(i) = acc;
    yn += acc * acc;
  }
  ynorm = sqrtf(gsum<G>(yn, gm));
  __syncwarp(gm);
  ylast = fabsf(Y_(p - 1));
#undef AF_
#undef BF_
#undef D_
#undef E_
#undef X_
#undef Y_
#undef S_
}

// exp(-x) for a double-float argument x = hi + lo (|lo| <= u |hi|): exp(-hi) (1 - lo), whose
// relative error is that of expf, where expf of the rounded argument alone would carry u |x|.
__device__ __forceinline__ float exp_neg_df(DF x) { return expf(-x.hi) * (1.f - x.lo); }
__device__ __forceinline__ DF df_from(double v) {
  DF r;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}

// FP32-path final step (p >= 3): every Ritz value is recomputed in double-float
// arithmetic (about 44 bits, on the FP32 pipe) as the Rayleigh quotient of its FP32 Ritz
// vector with the double-float T_p (the error is quadratic in the vector's, ~1e-14);
// lambda_min enters the log-weight. The relative weights exp(-dt (lambda_k - lambda_min))
// in (0, 1] and y = sum_k s_k s_k[0] w_k / |s_k|^2 are formed in FP32 (one Ritz pair per
// lane), the precision of the Krylov vectors they multiply. y lands in y32.
//
// REFINE (models created with KT_FP32_TRIDIAG64): the FP32 Ritz vectors X first take one
// step of Ogita and Aishima's refinement of a symmetric eigendecomposition (Japan J. Indust.
// Appl. Math. 35 (2018) 1007): with R = I - X^T X and S = X^T T_p X in double-float,
// X <- X (I + E), E_kk = R_kk / 2 and, for k != l, E_kl = (S_kl + lambda_l R_kl) /
// (lambda_l - lambda_k). That reduces the vectors' error from u |T_p| / gap to its square.
// The Ritz values are then recomputed from the refined vectors, the weights x_l[0] w_l
// formed in FP64, and y = sum_l x_l x_l[0] w_l summed in double-float, so that y is rounded
// to FP32 once, as from an FP64 eigensolve (weights rounded to FP32 first put a few ulps into
// y, which the cancellations of a trace can amplify a hundredfold). A pair whose correction
// would exceed 1e-4 (a gap within about 1e-3 |T_p|) is not refined by this step: its FP32
// mixing angle u |T_p| / gap times the weights' difference dt gap leaves an error u |T_p| dt
// in y whatever the gap, so an item with such a pair returns false without writing y, and
// the caller takes the FP64 eigensolve instead.
// Scratch: the FP64 Ritz-vector tile S, as float pairs. Without REFINE: always true.
template <bool REFINE, typename VT, int G, int DMAX, int PMAX>
__device__ bool tri_final32(WarpTile<VT, G, DMAX, PMAX> &s, int grp, int gl, unsigned gm, int p, double dt,
                            double &logfac) {
  constexpr int IPW = 32 / G;
#define AF_(k) reinterpret_cast<const float2 *>(s.a)[(k) * IPW + grp]
#define BF_(k) reinterpret_cast<const float2 *>(s.b)[(k) * IPW + grp]
#define DF_(k) reinterpret_cast<float2 *>(s.dd)[(k) * IPW + grp]
#define X_(k) s.x32[(k) * IPW + grp]
#define Y_(k) s.y32[(k) * IPW + grp]
#define S_(k, i) s.S32[((k) * PMAX + (i)) * IPW + grp]
#define W_(l, i) reinterpret_cast<float2 *>(s.S)[((l) * PMAX + (i)) * IPW + grp]
  // lane-local Ritz pair k: double-float Rayleigh quotient (and, to refine, T_p s_k)
  DF lmin;
  lmin.hi = INFINITY;
  int kmin = 0;
  for (int k = gl; k < p; k += G) {
    DF num, den;
    float sprev = 0.f, scur = S_(k, 0);
    for (int i = 0; i < p; ++i) {
      const float snext = (i + 1 < p) ? S_(k, i + 1) : 0.f;
      DF a, ti;
      a.hi = AF_(i).x;
      a.lo = AF_(i).y;
      ti = df_mulf(a, scur);
      if (i > 0) {
        DF b;
        b.hi = BF_(i - 1).x;
        b.lo = BF_(i - 1).y;
        ti = df_add(ti, df_mulf(b, sprev));
      }
      if (i + 1 < p) {
        DF b;
        b.hi = BF_(i).x;
        b.lo = BF_(i).y;
        ti = df_add(ti, df_mulf(b, snext));
      }
      if (REFINE) W_(k, i) = make_float2(ti.hi, ti.lo);
      num = df_add(num, df_mulf(ti, scur));
      den.add_prod(scur, scur);
      sprev = scur;
      scur = snext;
    }
    den = df_norm(den.hi, den.lo);
    const DF lam = df_div(num, den);
    DF_(k) = make_float2(lam.hi, lam.lo);
    X_(k) = 1.f / den.hi;
    if (df_lt(lam, lmin)) {
      lmin = lam;
      kmin = k;
    }
  }
  // smallest Ritz value over the group
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    DF ol;
    ol.hi = __shfl_xor_sync(gm, lmin.hi, o);
    ol.lo = __shfl_xor_sync(gm, lmin.lo, o);
    const int ok = __shfl_xor_sync(gm, kmin, o);
    if (df_lt(ol, lmin) || (ol.hi == lmin.hi && ol.lo == lmin.lo && ok < kmin)) {
      lmin = ol;
      kmin = ok;
    }
  }
  __syncwarp(gm);
  const float dtf = (float)dt;
  if constexpr (REFINE) {
    bool close = false;
    for (int l = gl; l < p; l += G) {
      DF t[PMAX];  // T_p x_l
#pragma unroll
      for (int i = 0; i < PMAX; ++i)
        if (i < p) {
          const float2 v = W_(l, i);
          t[i].hi = v.x;
          t[i].lo = v.y;
        }
      // column l of S and R (float: the off-diagonal entries are O(u), their sums exact)
      for (int k = 0; k < p; ++k) {
        DF sa, ra;
#pragma unroll
        for (int i = 0; i < PMAX; ++i)
          if (i < p) {
            const float x = S_(k, i);
            sa.add_prod(x, t[i].hi);
            sa.lo = fmaf(x, t[i].lo, sa.lo);
            ra.add_prod(x, S_(l, i));
          }
        const float rkl = (k == l) ? (1.f - ra.hi) - ra.lo : -(ra.hi + ra.lo);
        W_(l, k) = make_float2(k == l ? 0.f : sa.hi + sa.lo, rkl);
      }
      const float2 ll = DF_(l);
      DF lam_l;
      lam_l.hi = ll.x;
      lam_l.lo = ll.y;
      for (int k = 0; k < p; ++k) {
        const float2 sr = W_(l, k);
        float e = 0.5f * sr.y;
        if (k != l) {
          const float2 kk = DF_(k);
          DF lam_k;
          lam_k.hi = kk.x;
          lam_k.lo = kk.y;
          const DF gap = df_add(lam_l, df_neg(lam_k));
          const float num = fmaf(lam_l.hi, sr.y, sr.x), dl = gap.hi + gap.lo;
          // the same decision for E_kl and E_lk
          if (fmaxf(fabsf(num), fabsf(fmaf(lam_k.hi, sr.y, sr.x))) <= 1e-4f * fabsf(dl))
            e = num / dl;
          else
            close = true;
        }
        W_(l, k).x = e;
      }
      // correction c_l = X E[:, l] into W(l, .).y
      for (int i = 0; i < p; ++i) {
        float c = 0.f;
        for (int k = 0; k < p; ++k) c = fmaf(S_(k, i), W_(l, k).x, c);
        W_(l, i).y = c;
      }
      // Ritz value of the refined vector x' = x + c: the Rayleigh quotient of x is biased by
      // about gap |x - v|^2 (upwards for the lowest), a bias that adds up over the intervals
      // of a sequence. With r = T x - lambda x (exact in double-float) and |x'| = 1 + O(u^2),
      // lambda' - lambda = 2 c^T r + c^T (T - lambda) c, in X(l) until every lane is done
      float dlam = 0.f, cprev = 0.f, ccur = W_(l, 0).y;
#pragma unroll
      for (int i = 0; i < PMAX; ++i)
        if (i < p) {
          const float cnext = (i + 1 < p) ? W_(l, i + 1).y : 0.f;
          const DF ri = df_add(t[i], df_neg(df_mulf(lam_l, S_(l, i))));
          float tc = (AF_(i).x - lam_l.hi) * ccur;
          if (i > 0) tc = fmaf(BF_(i - 1).x, cprev, tc);
          if (i + 1 < p) tc = fmaf(BF_(i).x, cnext, tc);
          dlam = fmaf(ccur, fmaf(2.f, ri.hi + ri.lo, tc), dlam);
          cprev = ccur;
          ccur = cnext;
        }
      X_(l) = dlam;
    }
    if (__any_sync(gm, close)) return false;
    // lowest refined Ritz value over the group, then x'_l[0] w_l
    DF lmin2;
    lmin2.hi = INFINITY;
    for (int l = gl; l < p; l += G) {
      DF lam;
      lam.hi = DF_(l).x;
      lam.lo = DF_(l).y;
      lam = df_add(lam, df_norm(X_(l), 0.f));
      if (df_lt(lam, lmin2)) lmin2 = lam;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      DF ol;
      ol.hi = __shfl_xor_sync(gm, lmin2.hi, o);
      ol.lo = __shfl_xor_sync(gm, lmin2.lo, o);
      if (df_lt(ol, lmin2)) lmin2 = ol;
    }
    lmin = lmin2;
    // x'_l[0] w_l in FP64 (one exp per Ritz pair), kept as a double-float pair in x32 / e32
    for (int l = gl; l < p; l += G) {
      DF lam;
      lam.hi = DF_(l).x;
      lam.lo = DF_(l).y;
      lam = df_add(lam, df_norm(X_(l), 0.f));
      const DF diff = df_add(lam, df_neg(lmin));
      const double zw = ((double)S_(l, 0) + (double)W_(l, 0).y) * exp(-dt * ((double)diff.hi + (double)diff.lo));
      const float hi = (float)zw;
      X_(l) = hi;
      s.e32[l * IPW + grp] = (float)(zw - (double)hi);
    }
    __syncwarp(gm);
    for (int i = gl; i < p; i += G) {
      DF acc;
      for (int l = 0; l < p; ++l) {
        const float wh = X_(l), wl = s.e32[l * IPW + grp], x = S_(l, i);
        acc.add_prod(x, wh);
        acc.lo = fmaf(x, wl, fmaf(W_(l, i).y, wh, acc.lo));
      }
      Y_(i) = acc.hi + acc.lo;
    }
  } else {
    for (int k = gl; k < p; k += G) {
      DF lk;
      lk.hi = DF_(k).x;
      lk.lo = DF_(k).y;
      const DF diff = df_add(lk, df_neg(lmin));
      X_(k) = expf(-dtf * diff.hi) * S_(k, 0) * X_(k);
    }
    __syncwarp(gm);
    for (int i = gl; i < p; i += G) {
      float acc = 0.f;
      for (int k = 0; k < p; ++k) acc = fmaf(S_(k, i), X_(k), acc);
      Y_(i) = acc;
    }
  }
  logfac = -dt * ((double)lmin.hi + (double)lmin.lo);
  __syncwarp(gm);
  return true;
#undef AF_
#undef BF_
#undef DF_
#undef X_
#undef Y_
#undef S_
#undef W_
}

struct ItemAcc {
  unsigned long long ops, intervals, iters, pmax, noconv, flops_vec, flops_tri, bytes_apply, flops_alg, flops_reorth;
};

// Per-group context of one work unit (half of a (walker, kept state) item).
template <typename VT, int G, int DMAX, int PMAX>
struct Unit {
  static constexpr int IPW = 32 / G;
  static constexpr int R = (DMAX + G - 1) / G;  // rows per lane
  WarpTile<VT, G, DMAX, PMAX> &s;
  int grp, gl;
  unsigned gm;
  int b, dim;
  double Ladd;    // additive part of the log-weight
  LogScale Linv;  // product of the normalisation factors applied
  int status;
  ItemAcc acc;
  __device__ __forceinline__ VT &Q(int j, int r) { return s.q[((j) * DMAX + (r)) * IPW + grp]; }
};

// Step 4: apply c_f (dag = 0) or c_f^+ (dag = 1) to the unit's vector q_0:
// a gather with the Jordan-Wigner sign into the target block, then
// normalisation. False if the result is exactly zero.
template <typename VT, int G, int DMAX, int PMAX>
__device__ bool apply_op(const DevModel &M, Unit<VT, G, DMAX, PMAX> &u, int f, int dag) {
  constexpr int R = Unit<VT, G, DMAX, PMAX>::R;
  const int nf = M.nf;
  const int b2 = __ldg(M.blk_target + ((size_t)u.b * nf + f) * 2 + dag);
  if (b2 < 0) return false;
  const int off2 = __ldg(M.blk_off + b2), dim2 = __ldg(M.blk_dim + b2);
  VT tv[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int r = u.gl + G * j;
    VT v = VT(0);
    if (r < dim2) {
      const int g = off2 + r;
      const int x = __ldg(M.st_bits + g);
      if (((x >> f) & 1) == dag) {
        const unsigned pe = __ldg(M.partner + (size_t)g * nf + f);
        v = u.Q(0, pe & 0x7fffu);
        if (pe & 0x8000u) v = -v;
      }
    }
    tv[j] = v;
  }
  u.acc.ops += 1;
  u.acc.flops_vec += 3ull * dim2;
  u.acc.bytes_apply += (unsigned long long)dim2 * (2 * sizeof(VT) + 4);
  if (!normalize_rows<VT, G, R>(tv, u.gl, dim2, u.gm, u.Linv)) return false;
  __syncwarp(u.gm);
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int r = u.gl + G * j;
    if (r < dim2) u.Q(0, r) = tv[j];
  }
  __syncwarp(u.gm);
  u.b = b2;
  u.dim = dim2;
  return true;
}

// FP32 path, exact Krylov stop (p = d_b, or an invariant subspace found by breakdown): the
// Krylov space holds q_0 and is invariant under H_b, so the Lanczos result
// V_p exp(-dt T_p) e_1 is exp(-dt (H_b - s_b)) q_0 itself. It is formed here from the block's
// eigendecomposition (setup's FP64 Jacobi), which needs no eigensolve of T_p:
// c_k = <v_k | q_0>, weights exp(-dt (lambda_k - lambda_min)) with lambda_min the lowest
// eigenvalue whose component exceeds 4 u |q_0| (smaller components are rounding noise of
// exact zeros, which the propagator would otherwise amplify, and are dropped), and
// v = sum_k v_k c_k w_k into vv, all in FP32 (exact_propagate_df: the same with double-float
// sums). Returns -dt (lambda_min - s_b), the scale taken out, in FP64.
template <typename VT, int G, int DMAX, int PMAX>
__device__ __forceinline__ double exact_propagate32(const DevModel &M, Unit<VT, G, DMAX, PMAX> &u, int off, double dt,
                                                    VT (&vv)[Unit<VT, G, DMAX, PMAX>::R]) {
  constexpr int R = Unit<VT, G, DMAX, PMAX>::R;
  const int gl = u.gl, dim = u.dim;
  const unsigned gm = u.gm;
  const float *__restrict__ V = M.blk_evec32 + __ldg(M.blk_evoff + u.b);
  float c[R];
  float n2 = 0.f;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int k = gl + G * j;
    float a = 0.f;
    if (k < dim)
      for (int r = 0; r < dim; ++r) a = fmaf(__ldg(V + k * dim + r), u.Q(0, r), a);
    c[j] = a;
    n2 = fmaf(a, a, n2);
  }
  n2 = gsum<G>(n2, gm);
  // lowest significant eigenvalue: eigenvalues ascend within the block
  const float thr = n2 * (float)((4 * 5.9604645e-8) * (4 * 5.9604645e-8));
  int kmin = dim;
#pragma unroll
  for (int j = R - 1; j >= 0; --j) {
    const int k = gl + G * j;
    if (k < dim && c[j] * c[j] > thr) kmin = k;
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) kmin = min(kmin, __shfl_xor_sync(gm, kmin, o));
  if (kmin >= dim) kmin = 0;
  const double lmin = __ldg(M.st_eval64 + off + kmin);
  const float dtf = (float)dt;
  __syncwarp(gm);
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int k = gl + G * j;
    if (k < dim) {
      const float dl = (float)(__ldg(M.st_eval64 + off + k) - lmin);
      u.Q(1, k) = (c[j] * c[j] > thr) ? c[j] * expf(-dtf * dl) : 0.f;
    }
  }
  __syncwarp(gm);
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int r = gl + G * j;
    float a = 0.f;
    if (r < dim)
      for (int k = 0; k < dim; ++k) a = fmaf(__ldg(V + k * dim + r), u.Q(1, k), a);
    vv[j] = a;
  }
  return -dt * lmin;
}

// The exact stop of exact_propagate32 with both eigenvector sums in double-float on the FP32
// pipe (eigenvectors as fl32 pairs, products exact by FMA; about 44 significant bits, the
// accuracy of FP64 sums at a fraction of their cost on GB300, whose FP64 pipe is 1/64 of the
// FP32 one) and double-float weight arguments: models created with KT_FP32_TRIDIAG64.
template <typename VT, int G, int DMAX, int PMAX>
__device__ __forceinline__ double exact_propagate_df(const DevModel &M, Unit<VT, G, DMAX, PMAX> &u, int off, double dt,
                                                     VT (&vv)[Unit<VT, G, DMAX, PMAX>::R]) {
  constexpr int R = Unit<VT, G, DMAX, PMAX>::R;
  const int gl = u.gl, dim = u.dim;
  const unsigned gm = u.gm;
  const int eo = __ldg(M.blk_evoff + u.b);
  const float *__restrict__ Vh = M.blk_evec32 + eo;
  const float *__restrict__ Vl = M.blk_evec32lo + eo;
  float c[R];
  float n2 = 0.f;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int k = gl + G * j;
    DF a;
    if (k < dim)
      for (int r = 0; r < dim; ++r) {
        const float q = u.Q(0, r);
        a.add_prod(__ldg(Vh + k * dim + r), q);
        a.lo = fmaf(__ldg(Vl + k * dim + r), q, a.lo);
      }
    c[j] = a.hi + a.lo;
    n2 = fmaf(c[j], c[j], n2);
  }
  n2 = gsum<G>(n2, gm);
  const float thr = n2 * (float)((4 * 5.9604645e-8) * (4 * 5.9604645e-8));
  int kmin = dim;
#pragma unroll
  for (int j = R - 1; j >= 0; --j) {
    const int k = gl + G * j;
    if (k < dim && c[j] * c[j] > thr) kmin = k;
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) kmin = min(kmin, __shfl_xor_sync(gm, kmin, o));
  if (kmin >= dim) kmin = 0;
  const double lmin = __ldg(M.st_eval64 + off + kmin);
  const DF dtd = df_from(dt);
  __syncwarp(gm);
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int k = gl + G * j;
    if (k < dim) {
      const DF x = df_mul(dtd, df_from(__ldg(M.st_eval64 + off + k) - lmin));
      u.Q(1, k) = (c[j] * c[j] > thr) ? c[j] * exp_neg_df(x) : 0.f;
    }
  }
  __syncwarp(gm);
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int r = gl + G * j;
    DF a;
    if (r < dim)
      for (int k = 0; k < dim; ++k) {
        const float w = u.Q(1, k);
        a.add_prod(__ldg(Vh + k * dim + r), w);
        a.lo = fmaf(__ldg(Vl + k * dim + r), w, a.lo);
      }
    vv[j] = a.hi + a.lo;
  }
  return -dt * lmin;
}

// Step 5: q_0 <- exp(-dt (H_b - E0)) q_0 by Lanczos on H_b - s_b with the
// a-posteriori stop; the scalars taken out go to the log-weight.
// False if the propagated vector is exactly zero.
template <int OPT, typename VT, int G, int DMAX, int PMAX>
__device__ bool propagate(const DevModel &M, Unit<VT, G, DMAX, PMAX> &u, double dt, kt_stats *stats) {
  constexpr bool F32 = sizeof(VT) == 4;
  constexpr bool TRI64 = (OPT & KT_OPT_TRI64) != 0;
  const bool with_stats = (OPT & KT_OPT_STATS) && stats != nullptr;
  constexpr int R = Unit<VT, G, DMAX, PMAX>::R;
  constexpr int IPW = 32 / G;
  auto &s = u.s;
  const int grp = u.grp, gl = u.gl;
  const unsigned gm = u.gm;
#define A_(k) s.a[(k) * IPW + grp]
#define B_(k) s.b[(k) * IPW + grp]
#define Y_(k) s.y[(k) * IPW + grp]
  const VT *__restrict__ tdiag = Tab<VT>::diag(M);
  const VT *__restrict__ tval = Tab<VT>::val(M);
  const int b = u.b, dim = u.dim;
  const int off = __ldg(M.blk_off + b), wid = __ldg(M.blk_nnz + b), ell = __ldg(M.blk_ell + b);
  const double shift = __ldg(M.blk_shift + b);
  const double brk = M.brk_rel * fmax(__ldg(M.blk_norm + b), 1e-300);
  const int pcap = min(dim, M.pmax);
  const float tol32 = F32 ? (float)(0.5 * M.tol) : 0.f;  // safety factor 2 on FP32 estimates
  const float brk32 = F32 ? (float)brk : 0.f;
  VT qc[R], qp[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int r = gl + G * j;
    qc[j] = (r < dim) ? u.Q(0, r) : VT(0);
    qp[j] = VT(0);
  }
  // Blocks of at most 16 rows: the ELL column indices of the lane's rows, read once per
  // interval rather than at every Lanczos step (a block's pattern is the same at every step;
  // setup merges repeated columns, so a row has at most d_b - 1 < DMAX entries), as col + 1
  // in bytes, four to a register. The load that heads each product's chain is then gone.
  constexpr bool PACK = DMAX <= 16;
  constexpr int NW = PACK ? (DMAX + 2) / 4 : 1;
  uint32_t cpk[R][NW];
  if constexpr (PACK) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int r = gl + G * j;
#pragma unroll
      for (int w = 0; w < NW; ++w) cpk[j][w] = 0u;
      if (r < dim)
#pragma unroll
        for (int k = 0; k < DMAX - 1; ++k)
          if (k < wid) cpk[j][k >> 2] |= (uint32_t)(__ldg(M.ell_col + ell + k * dim + r) + 1) << (8 * (k & 3));
    }
  }
  double logfac = 0.0;
  VT bprev = VT(0);
  int p = 0;
  bool conv = false, exact = false;
  for (int jj = 0; jj < pcap; ++jj) {
    VT wv[R];
    GroupDot<VT, G> da;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int r = gl + G * j;
      VT a = VT(0);
      if (r < dim) {
        a = __ldg(tdiag + off + r) * qc[j];
        if constexpr (PACK) {
#pragma unroll
          for (int k = 0; k < DMAX - 1; ++k)
            if (k < wid) {
              const int col = (int)((cpk[j][k >> 2] >> (8 * (k & 3))) & 0xffu) - 1;
              if (col >= 0) a += __ldg(tval + ell + k * dim + r) * u.Q(jj, col);
            }
        } else {
          for (int k = 0; k < wid; ++k) {
            const int col = __ldg(M.ell_col + ell + k * dim + r);
            if (col >= 0) a += __ldg(tval + ell + k * dim + r) * u.Q(jj, col);
          }
        }
        da.add(a, qc[j]);
      }
      wv[j] = a;
    }
    double al = 0.0;
    DF al_df;
    if constexpr (F32) {
      al_df = da.value_df(gm);
    } else {
      al = da.value(gm);
    }
    const VT alv = F32 ? VT(al_df.hi) : VT(al), bpv = bprev;
#pragma unroll
    for (int j = 0; j < R; ++j)
      if (gl + G * j < dim) wv[j] = wv[j] - alv * qc[j] - bpv * qp[j];
    if constexpr (F32) {
      // one pass of full reorthogonalisation against q_0 .. q_jj
      for (int k = 0; k <= jj && jj > 0; ++k) {
        VT h = VT(0);
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int r = gl + G * j;
          if (r < dim) h += u.Q(k, r) * wv[j];
        }
        h = gsum<G>(h, gm);
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int r = gl + G * j;
          if (r < dim) wv[j] -= h * u.Q(k, r);
        }
      }
    }
    GroupDot<VT, G> db;
#pragma unroll
    for (int j = 0; j < R; ++j)
      if (gl + G * j < dim) db.add(wv[j], wv[j]);
    double bb = 0.0;
    DF bb_df;
    if constexpr (F32) {
      bb_df = db.norm_df(gm);
    } else {
      bb = db.norm(gm);
    }
    p = jj + 1;
    if (gl == 0) {
      if constexpr (F32) {  // double-float alpha, beta in the slots of the FP64 ones
        reinterpret_cast<float2 *>(s.a)[jj * IPW + grp] = make_float2(al_df.hi, al_df.lo);
        reinterpret_cast<float2 *>(s.b)[jj * IPW + grp] = make_float2(bb_df.hi, bb_df.lo);
      } else {
        A_(jj) = al;
        B_(jj) = bb;
      }
    }
    __syncwarp(gm);
    exact = (p == dim) || !(F32 ? (bb_df.hi > brk32) : (bb > brk));
    bool stop = exact;
    // a-posteriori checks at every p up to 4, then on a geometric schedule
    // (6, 8, 11, 15, 20, 27): each check costs an eigendecomposition of T_p
    // FP32 path, blocks of at most 16 rows: an interval two steps or less from exhausting its
    // block is not checked; the exact stop that follows costs less than the eigensolve of a check
    const bool near_exact = F32 && DMAX <= 16 && p >= 3 && dim <= pcap && dim - p <= 2;
    const bool check = !near_exact &&
                       (p <= 4 || p == 6 || p == 8 || p == 11 || p == 15 || p == 20 || p == 27 || p == pcap);
    if (!exact && check) {
      if constexpr (F32) {
        float yn, yl;
        tri_check32(s, grp, gl, gm, p, dt, yn, yl);
        stop = bb_df.hi * yl <= tol32 * yn;
      } else {
        if (!tri_exp64(s, grp, gl, gm, p, dt, logfac)) u.status = KT_ENUMERIC;
        double yn = 0.0;
        for (int k = gl; k < p; k += G) yn = fma(Y_(k), Y_(k), yn);
        yn = sqrt(gsum<G>(yn, gm));
        stop = bb * fabs(Y_(p - 1)) <= M.tol * yn;
      }
    }
    if (stop) {
      conv = true;
      break;
    }
    if (p == pcap) break;
    const VT ib = F32 ? VT(1) / VT(bb_df.hi) : VT(1) / VT(bb);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int r = gl + G * j;
      qp[j] = qc[j];
      qc[j] = wv[j] * ib;
      if (r < dim) u.Q(jj + 1, r) = qc[j];
    }
    bprev = F32 ? VT(bb_df.hi) : VT(bb);
    __syncwarp(gm);
  }
  if (!conv) {
    u.acc.noconv += 1;
    if (u.status == KT_OK) u.status = KT_ENOCONV;
  }
  // final exp(-dt T_p) e_1 at the stopping p, and v = sum_j y_j q_j (renormalised below;
  // what is taken out goes to the log-weight)
  VT vv[R];
  bool dense = false;
  // exact stops of blocks beyond 16 rows (seven orbitals) keep the Lanczos final step: formed
  // from the eigendecomposition there, their FP32 traces came out less accurate, not more
  if constexpr (F32 && DMAX <= 16) dense = exact && p >= 2;
  if (dense) {
    if (TRI64)
      logfac = exact_propagate_df(M, u, off, dt, vv);
    else
      logfac = exact_propagate32(M, u, off, dt, vv);
  } else {
    // final exp(-dt T_p) e_1 at the stopping p
    if constexpr (F32) {
      if (p == 2 && (DMAX > 16 || TRI64)) {
        // the 2x2 closed form in FP64 from the double-float alpha, beta: with KT_FP32_TRIDIAG64,
        // and in the instances for blocks beyond 16 rows (seven orbitals), where the FP32
        // eigenvector components of the 2x2 step (error u ||T_2|| / gap) were the largest
        // contribution to the trace error
        const float2 a0 = reinterpret_cast<float2 *>(s.a)[grp], a1 = reinterpret_cast<float2 *>(s.a)[IPW + grp];
        const float2 b0 = reinterpret_cast<float2 *>(s.b)[grp];
        double y0, y1;
        logfac = exp2x2((double)a0.x + (double)a0.y, (double)a1.x + (double)a1.y, (double)b0.x + (double)b0.y, dt, y0,
                        y1);
        if (gl == 0) {
          s.y32[grp] = (float)y0;
          s.y32[IPW + grp] = (float)y1;
        }
        __syncwarp(gm);
      } else if (p <= 2) {
        tri_small_f32(s, grp, gl, gm, p, dt, logfac);
      } else {
        // Ritz pairs from the check that stopped at p; refined with KT_FP32_TRIDIAG64
        bool done = false;
        if constexpr (DMAX <= 16) done = tri_final32<TRI64>(s, grp, gl, gm, p, dt, logfac);
        if (!(DMAX <= 16 && !TRI64) && !done) {
          // FP32 Ritz vectors are off by about u ||T_p|| / gap, an error that does not average
          // out over the intervals of a sequence; blocks beyond 16 rows (seven orbitals), and
          // the items with close Ritz values that KT_FP32_TRIDIAG64 does not refine, therefore
          // take the full FP64 eigensolve at the final p (alpha, beta first widened in place
          // from double-float to FP64). Exact stops beyond 16 rows come without a check at p,
          // so there are no FP32 Ritz pairs to refine.
          for (int k = gl; k < p; k += G) {
            const float2 av = reinterpret_cast<float2 *>(s.a)[k * IPW + grp];
            const float2 bv = reinterpret_cast<float2 *>(s.b)[k * IPW + grp];
            A_(k) = (double)av.x + (double)av.y;
            B_(k) = (double)bv.x + (double)bv.y;
          }
          __syncwarp(gm);
          if (!tri_exp64(s, grp, gl, gm, p, dt, logfac)) u.status = KT_ENUMERIC;
          for (int k = gl; k < p; k += G) s.y32[k * IPW + grp] = (float)Y_(k);
          __syncwarp(gm);
        }
      }
    } else {
      if (exact && !tri_exp64(s, grp, gl, gm, p, dt, logfac)) u.status = KT_ENUMERIC;
    }
    // v = sum_j y_j q_j
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int r = gl + G * j;
      VT a = VT(0);
      if (r < dim) {
        if constexpr (F32) {
          for (int k = 0; k < p; ++k) a += s.y32[k * IPW + grp] * u.Q(k, r);
        } else {
          for (int k = 0; k < p; ++k) a += Y_(k) * u.Q(k, r);
        }
      }
      vv[j] = a;
    }
  }
  if (!normalize_rows<VT, G, R>(vv, gl, dim, gm, u.Linv)) return false;
  u.Ladd += logfac - dt * (shift - M.E0);
  __syncwarp(gm);
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int r = gl + G * j;
    if (r < dim) u.Q(0, r) = vv[j];
  }
  __syncwarp(gm);
  u.acc.intervals += 1;
  u.acc.iters += p;
  u.acc.pmax = u.acc.pmax > (unsigned long long)p ? u.acc.pmax : (unsigned long long)p;
  if (with_stats) {
    if (gl == 0) atomicAdd(&stats->p_hist[p < KT_P_HIST - 1 ? p : KT_P_HIST - 1], 1ull);
    u.acc.flops_tri += (p <= 2) ? 30ull : (unsigned long long)(12 * p * p * p + 40 * p);
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int r = gl + G * j;
      if (r < dim) {
        cnt += 1;
        for (int k = 0; k < wid; ++k) cnt += (__ldg(M.ell_col + ell + k * dim + r) >= 0);
      }
    }
    const int nnz_blk = gsum<G>(cnt, gm);
    u.acc.flops_vec += (unsigned long long)p * (2ull * nnz_blk + 9ull * dim) + 2ull * p * dim + 3ull * dim;
    u.acc.flops_alg += (unsigned long long)p * (2ull * nnz_blk + 11ull * dim) + 2ull * p * dim;
    if (F32) {  // reorthogonalisation
      u.acc.flops_vec += (unsigned long long)p * (p - 1) * 2ull * dim;
      u.acc.flops_reorth += (unsigned long long)p * (p - 1) * 2ull * dim;
    }
  }
  return true;
#undef A_
#undef B_
#undef Y_
}

// Observables of one item at the meeting time beta/2, from this unit's vector (shared
// memory) and the other half's (global, `other`): <O> = sum_r o(x_r) bwd_r fwd_r /
// sum_r bwd_r fwd_r for the diagonal observables (n_f, double occupancy), and S^2 applied
// to this unit's vector dotted with the other half.
template <typename VT, int G, int DMAX, int PMAX>
__device__ __forceinline__ void measure_epilogue(const DevModel &M, Unit<VT, G, DMAX, PMAX> &u, const Workspace &ws,
                                                 int item, const VT *other, double ov) {
  constexpr int R = Unit<VT, G, DMAX, PMAX>::R;
  const int gl = u.gl;
  const unsigned gm = u.gm;
  const int nf = M.nf, nl = nf + M.n_orb + 1;
  const int off = __ldg(M.blk_off + u.b);
  VT pr[R];
  int xr[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int r = gl + G * j;
    pr[j] = VT(0);
    xr[j] = 0;
    if (r < u.dim) {
      pr[j] = u.Q(0, r) * __ldcg(other + r);
      xr[j] = __ldg(M.st_bits + off + r);
    }
  }
  const double iov = 1.0 / ov;
  for (int k = 0; k < nl - 1; ++k) {
    const int sh = k < nf ? k : 2 * (k - nf);
    const int msk = k < nf ? 1 : 3;
    GroupDot<VT, G> d;
#pragma unroll
    for (int j = 0; j < R; ++j)
      if (((xr[j] >> sh) & msk) == msk) d.add(pr[j], VT(1));
    const double v = d.value(gm) * iov;
    if (gl == 0) ws.item_obs[(size_t)item * nl + k] = v;
  }
  {
    // S^2: sum_r other_r (S^2 own)_r, S^2 applied to this unit's vector in shared memory
    const int s2w = __ldg(M.blk_s2w + u.b), s2o = __ldg(M.blk_s2ell + u.b);
    GroupDot<VT, G> d;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int r = gl + G * j;
      if (r < u.dim) {
        VT a = VT(__ldg(M.s2_diag + off + r)) * u.Q(0, r);
        for (int k = 0; k < s2w; ++k) {
          const unsigned e = __ldg(M.s2_ell + s2o + k * u.dim + r);
          if (e != 0xFFFFu) a += (e & 0x8000u) ? -u.Q(0, e & 0x7fffu) : u.Q(0, e & 0x7fffu);
        }
        d.add(a, __ldcg(other + r));
      }
    }
    const double v = d.value(gm) * iov;
    if (gl == 0) ws.item_obs[(size_t)item * nl + nl - 1] = v;
  }
  if (gl == 0) ws.item_blk[item] = u.b;
}

// Work units: every alive (walker, kept state) item is split at the middle of
// its sequence into a forward unit (ops 0 .. m-1 acting on |n>, Sec. III step 3
// "forward") and a backward unit (the adjoints of ops K-1 .. m acting on <n|,
// "backward", including the interval between ops m-1 and m). Each unit
// publishes its normalised vector and log-weight to the workspace; whichever
// finishes second forms the overlap <backward|forward>. No unit ever waits.
template <typename VT, int G, int DMAX, int PMAX, int OPT>
__global__ void __launch_bounds__(256, KT_MIN_CTAS(VT)) items_kernel(DevModel M, SeqView S, MoveView mv, int has_moves, Workspace ws,
                                                    kt_stats *stats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int R = (DMAX + G - 1) / G;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane % G;
  const unsigned gm = (G == 32) ? FULL : (((1u << G) - 1u) << (grp * G));
  WarpTile<VT, G, DMAX, PMAX> &tile = reinterpret_cast<WarpTile<VT, G, DMAX, PMAX> *>(smem_raw)[wib];
  const VT *__restrict__ tkept = Tab<VT>::kept(M);
  const int n_units = 2 * ws.counters[0];
  const int nk = M.n_kept;
  const int vstride = M.d_max;
  VT *__restrict__ hvec = reinterpret_cast<VT *>(ws.half_vec);
  constexpr bool meas = (OPT & KT_OPT_MEAS) != 0;  // ws.item_obs is set

  // claim numbers: every lane group's first one is fixed, dealing consecutive numbers to
  // warp 0 of every CTA, then warp 1 of every CTA, and so on, so that the longest units
  // (the lowest numbers) land on different SMs; later ones come from the queue
  const int slots = (int)(gridDim.x * blockDim.x) / G;
  int first = (wib * (int)gridDim.x + (int)blockIdx.x) * (32 / G) + grp;
  for (;;) {
    int c = first;
    first = -1;
    if (c < 0) {
      if (gl == 0) c = slots + atomicAdd(&ws.counters[1], 1);
      c = __shfl_sync(gm, c, grp * G);
    }
    if (c >= n_units) break;
    // units in the worklist order (longest sequences first): of every four consecutive
    // claim numbers, one takes the next unit from the long end and three from the short end
    const int b = c >> 2, j = c & 3;
    const int uix = j == 0 ? b : n_units - 1 - (3 * b + j - 1);
    const int it = uix >> 1, half = uix & 1;
    const int item = ws.worklist[it];
    const int w = item / nk, q = item - w * nk;
    const Cursor cur = make_cursor(S, mv, has_moves != 0, ws.desc, w);
    const int Kn = cur.d.w;
    const int b_kept = __ldg(M.kept_blk + q);
    const double Ek = __ldg(M.kept_e + q);
    const int koff = __ldg(M.kept_off + q);
    if (Kn == 0 && !meas) {  // empty sequence: the kept state alone, no split
      if (half == 0 && gl == 0) {
        ws.item_sign[item] = 1;
        ws.item_log[item] = -M.beta * Ek;
        ws.item_status[item] = KT_OK;
      }
      continue;
    }
    Unit<VT, G, DMAX, PMAX> u{tile, grp, gl, gm, b_kept, __ldg(M.blk_dim + b_kept), 0.0, LogScale(), KT_OK, ItemAcc{}};
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int r = gl + G * j;
      if (r < u.dim) u.Q(0, r) = __ldg(tkept + koff + r);
    }
    __syncwarp(gm);
    // Split: ops 0 .. m-1 go forward from tau = 0, ops m .. K-1 backward from
    // beta; the halves meet at t_s. Traces and ratios split at the middle
    // operator (t_s = tau_{m-1}); measurements at t_s = beta/2, with m the
    // number of operators before beta/2 (possibly 0 or K).
    int m;
    double t_s;
    if (meas) {
      t_s = 0.5 * M.beta;
      m = lower_bound(S.tau + cur.o, Kn, t_s);
    } else {
      m = Kn / 2 > 1 ? Kn / 2 : 1;
      t_s = cur.get(m - 1).t;
    }
    bool vanished = false;
    // forward: ops 0 .. m-1 in order; backward: adjoints of ops K-1 .. m; each
    // op is followed by the interval to the next op of its half, the last one
    // by the interval to t_s
    const int nsteps = half == 0 ? m : Kn - m;
    if (nsteps == 0) {
      u.Ladd = half == 0 ? -t_s * Ek : -(M.beta - t_s) * Ek;  // |n> is an eigenstate
    } else {
      Op op = cur.get(half == 0 ? 0 : Kn - 1);
      u.Ladd = half == 0 ? -op.t * Ek : -(M.beta - op.t) * Ek;  // |n> is an eigenstate at both ends
      for (int s = 0; s < nsteps; ++s) {
        const int idx = half == 0 ? s : Kn - 1 - s;
        if (!apply_op(M, u, op.f, half == 0 ? op.dag : 1 - op.dag)) {
          vanished = true;
          break;
        }
        const bool last = s + 1 == nsteps;
        Op nx;
        if (!last) nx = cur.get(half == 0 ? idx + 1 : idx - 1);
        const double tn = last ? t_s : nx.t;
        const double dt = half == 0 ? tn - op.t : op.t - tn;
        if (!last) op = nx;
        if (dt > 0.0 && !propagate<OPT>(M, u, dt, stats)) {
          vanished = true;
          break;
        }
      }
    }
    // publish this half
    const int hslot = 2 * item + half;
    if (!vanished) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int r = gl + G * j;
        if (r < u.dim) hvec[(size_t)hslot * vstride + r] = u.Q(0, r);
      }
    }
    const double Lh = vanished ? 0.0 : u.Ladd - u.Linv.log_value();
    if (gl == 0) {
      ws.half_log[hslot] = Lh;
      ws.half_info[hslot] = vanished ? -1 : (u.b | (u.status << 24));
    }
    __threadfence();
    __syncwarp(gm);
    int old = 0;
    if (gl == 0) old = atomicAdd(&ws.pair_flag[item], 1);
    old = __shfl_sync(gm, old, grp * G);
    if (old == 1) {
      // the other half is published: form the overlap
      __threadfence();
      const int oslot = 2 * item + (1 - half);
      const int oinfo = __ldcg(ws.half_info + oslot);
      const double Lo = __ldcg(ws.half_log + oslot);
      bool zero = vanished || oinfo < 0 || (oinfo & 0xffffff) != u.b;
      double ov = 0.0;
      if (!zero) {
        GroupDot<VT, G> d;
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int r = gl + G * j;
          if (r < u.dim) d.add(u.Q(0, r), __ldcg(hvec + (size_t)oslot * vstride + r));
        }
        ov = d.value(gm);
        zero = (ov == 0.0);
      }
      int st = u.status;
      if (oinfo >= 0 && (oinfo >> 24) > st) st = oinfo >> 24;
      const double L = Lh + Lo + (zero ? 0.0 : log(fabs(ov)));
      if (!zero && !isfinite(L)) st = KT_ENUMERIC;
      if (meas && !zero) measure_epilogue(M, u, ws, item, hvec + (size_t)oslot * vstride, ov);
      if (gl == 0) {
        ws.item_sign[item] = zero ? 0 : (ov > 0.0 ? 1 : -1);
        ws.item_log[item] = zero ? -INFINITY : L;
        ws.item_status[item] = st;
      }
    }
    if ((OPT & KT_OPT_STATS) && gl == 0 && stats) {
      if (old == 1 && ws.item_sign[item] == 0) atomicAdd(&stats->items_vanished, 1ull);
      stat_add(&stats->ops_applied, u.acc.ops);
      stat_add(&stats->intervals, u.acc.intervals);
      stat_add(&stats->krylov_iters, u.acc.iters);
      if (u.acc.pmax) atomicMax(&stats->p_max, u.acc.pmax);
      stat_add(&stats->noconv, u.acc.noconv);
      stat_add(&stats->flops_vec, u.acc.flops_vec);
      stat_add(&stats->flops_tri, u.acc.flops_tri);
      stat_add(&stats->bytes_apply, u.acc.bytes_apply);
      stat_add(&stats->flops_alg, u.acc.flops_alg);
      stat_add(&stats->flops_reorth, u.acc.flops_reorth);
    }
    __syncwarp(gm);
  }
}

// One cache entry: the unit's normalised vector, its log-weight as (additive part
// less the binary exponent of the normalisation product, mantissa of that product)
// so that no logarithm is taken per operator, and its block (-1: the state is zero).
template <typename VT, int G, int DMAX, int PMAX>
__device__ __forceinline__ void store_entry(VT *vec, double2 *lg, int32_t *bk, size_t e, int dv,
                                            Unit<VT, G, DMAX, PMAX> &u, bool zero) {
  constexpr int R = Unit<VT, G, DMAX, PMAX>::R;
  if (!zero) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int r = u.gl + G * j;
      if (r < u.dim) vec[e * dv + r] = u.Q(0, r);
    }
  }
  if (u.gl == 0) {
    bk[e] = zero ? -1 : u.b;
    lg[e] = zero ? make_double2(0.0, 1.0) : make_double2(fma(-(double)u.Linv.e, 0.69314718055994530942, u.Ladd), u.Linv.m);
  }
}

template <typename VT, int G, int DMAX, int PMAX>
__device__ __forceinline__ bool load_entry(const DevModel &M, const VT *vec, const double2 *lg, const int32_t *bk,
                                           size_t e, int dv, Unit<VT, G, DMAX, PMAX> &u) {
  constexpr int R = Unit<VT, G, DMAX, PMAX>::R;
  const int b = __ldcg(bk + e);
  if (b < 0) return false;
  u.b = b;
  u.dim = __ldg(M.blk_dim + b);
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int r = u.gl + G * j;
    if (r < u.dim) u.Q(0, r) = __ldcg(vec + e * dv + r);
  }
  const double2 l = __ldcg(lg + e);
  u.Ladd = l.x;
  u.Linv.m = l.y;
  u.Linv.e = 0;
  __syncwarp(u.gm);
  return true;
}

// Cached-mode work units (the sweep's partial-state cache). Every planned item
// has a forward unit, ops y .. m-1 of the edited sequence starting from the cached
// state after op y-1 (the kept state at tau = 0 when y = 0), and a backward unit,
// the adjoints of ops x-1 .. m starting from the cached bra at op x (the kept state
// at beta when x = K) and then the interval down to op m-1 (Sec. III step 3, over
// the stretch that the cache does not cover). Each state passed is written to the
// cache when its position lies outside the edited window, else to the scratch
// arrays. The halves meet as in items_kernel.
template <typename VT, int G, int DMAX, int PMAX, int OPT>
__global__ void __launch_bounds__(256, KT_MIN_CTAS(VT)) items_cached_kernel(DevModel M, SeqView S, MoveView mv, Workspace ws,
                                                           CacheView C, kt_stats *stats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int R = (DMAX + G - 1) / G;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int grp = lane / G, gl = lane % G;
  const unsigned gm = (G == 32) ? FULL : (((1u << G) - 1u) << (grp * G));
  WarpTile<VT, G, DMAX, PMAX> &tile = reinterpret_cast<WarpTile<VT, G, DMAX, PMAX> *>(smem_raw)[wib];
  const VT *__restrict__ tkept = Tab<VT>::kept(M);
  const int n_units = 2 * ws.counters[0];
  const int nk = M.n_kept;
  const int vstride = M.d_max, dv = C.dv;
  VT *__restrict__ hvec = reinterpret_cast<VT *>(ws.half_vec);
  const size_t P1 = (size_t)C.P + 1;
  constexpr bool meas = (OPT & KT_OPT_MEAS) != 0;  // observables at beta/2 (plans with flag 8)

  // claim numbers as in items_kernel: a fixed first one per lane group, then the queue
  const int slots = (int)(gridDim.x * blockDim.x) / G;
  int first = (wib * (int)gridDim.x + (int)blockIdx.x) * (32 / G) + grp;
  for (;;) {
    int c = first;
    first = -1;
    if (c < 0) {
      if (gl == 0) c = slots + atomicAdd(&ws.counters[1], 1);
      c = __shfl_sync(gm, c, grp * G);
    }
    if (c >= n_units) break;
    // the worklist is ordered longest stretch first: one unit of every four consecutive
    // claim numbers from the long end, three from the short end
    const int b = c >> 2, j = c & 3;
    const int uix = j == 0 ? b : n_units - 1 - (3 * b + j - 1);
    const int it = uix >> 1, half = uix & 1;
    const int item = ws.worklist[it];
    const int w = item / nk, q = item - w * nk;
    const Cursor cur = make_cursor(S, mv, true, ws.desc, w);
    const int Kn = cur.d.w;
    const int4 pl = C.plan[item];
    const bool cached = (pl.w & 1) != 0;
    int lo, hi;
    edit_window(cur.d, lo, hi);
    const int b_kept = __ldg(M.kept_blk + q);
    const double Ek = __ldg(M.kept_e + q);
    const int koff = __ldg(M.kept_off + q);
    Unit<VT, G, DMAX, PMAX> u{tile, grp, gl, gm, b_kept, __ldg(M.blk_dim + b_kept), 0.0, LogScale(), KT_OK, ItemAcc{}};
    const size_t eb = (size_t)item * P1;
    const int y = pl.x, x = pl.y, m = pl.z;
    // One loop for both halves (a single inlined copy of propagate and apply_op):
    // forward, steps s = 0 .. m-y-1 take op i = y+s: the interval up to it, then the op;
    // backward, steps s = 0 .. x-m-1 take op i = x-1-s: the interval down to it, then
    // its adjoint; a last step without op takes the interval down to op m-1.
    const bool fwd = half == 0;
    const bool build = (pl.w & 4) != 0;  // cache build: each half covers the whole sequence
    const bool at_half = (pl.w & 8) != 0;  // measurement: the halves meet at beta/2
    const int start = fwd ? y : x;
    const bool from_kept = fwd ? (y == 0) : (x == Kn);
    double t = fwd ? (y == 0 ? 0.0 : cur.get(y - 1).t) : (x == Kn ? M.beta : cur.get(x).t);
    bool eigen = from_kept, vanished = false;
    if (from_kept) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int r = gl + G * j;
        if (r < u.dim) u.Q(0, r) = __ldg(tkept + koff + r);
      }
      __syncwarp(gm);
    } else {
      vanished = !load_entry(M, (const VT *)(fwd ? C.fvec : C.bvec), fwd ? C.flog : C.blog, fwd ? C.fblk : C.bblk,
                             eb + (fwd ? start : Kn - start), dv, u);
    }
    const int n_ops = build ? Kn : (fwd ? m - y : x - m);
    // the last step of a half without an operator: the interval to the meeting time
    const int n_steps = build ? n_ops : (fwd && !at_half ? n_ops : n_ops + 1);
    const double tf = at_half ? 0.5 * M.beta : (m >= 1 ? cur.get(m - 1).t : 0.0);
    for (int s = 0; s < n_steps; ++s) {
      const bool has_op = s < n_ops;
      const int i = fwd ? y + s : x - 1 - s;
      Op op{tf, 0, 0};
      if (has_op) op = cur.get(i);
      if (!vanished) {
        const double dt = fwd ? op.t - t : t - op.t;
        if (eigen) u.Ladd -= dt * Ek;
        else if (dt > 0.0 && !propagate<OPT>(M, u, dt, stats)) vanished = true;
        if (has_op) {
          if (!vanished && !apply_op(M, u, op.f, fwd ? op.dag : 1 - op.dag)) vanished = true;
          eigen = false;
        }
      }
      t = op.t;
      if (has_op && cached) {
        // forward slot i+1 / backward reverse slot K-i; outside the window the state is
        // valid for the current configuration too and goes to the cache itself
        const bool out = build || at_half || (fwd ? i + 1 <= lo : i >= hi);
        const size_t e = eb + (fwd ? i + 1 : Kn - i);
        VT *vec = (VT *)(fwd ? (out ? C.fvec : C.sfvec) : (out ? C.bvec : C.sbvec));
        double2 *lg = fwd ? (out ? C.flog : C.sflog) : (out ? C.blog : C.sblog);
        int32_t *bk = fwd ? (out ? C.fblk : C.sfblk) : (out ? C.bblk : C.sbblk);
        store_entry(vec, lg, bk, e, dv, u, vanished);
      }
    }
    // a measurement stores states of the current configuration: the valid range grows
    if (at_half && cached && gl == 0 && u.status == KT_OK) {
      if (fwd) C.f[item] = max(C.f[item], m);
      else C.gr[item] = max(C.gr[item], Kn - m);
    }
    // publish this half; the second to finish forms the overlap (not for a build)
    if (!build) {
      const int hslot = 2 * item + half;
      if (!vanished) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int r = gl + G * j;
          if (r < u.dim) hvec[(size_t)hslot * vstride + r] = u.Q(0, r);
        }
      }
      const double Lh = vanished ? 0.0 : u.Ladd - u.Linv.log_value();
      if (gl == 0) {
        ws.half_log[hslot] = Lh;
        ws.half_info[hslot] = vanished ? -1 : (u.b | (u.status << 24));
      }
      __threadfence();
      __syncwarp(gm);
      int old = 0;
      if (gl == 0) old = atomicAdd(&ws.pair_flag[item], 1);
      old = __shfl_sync(gm, old, grp * G);
      if (old == 1) {
        __threadfence();
        const int oslot = 2 * item + (1 - half);
        const int oinfo = __ldcg(ws.half_info + oslot);
        const double Lo = __ldcg(ws.half_log + oslot);
        bool zero = vanished || oinfo < 0 || (oinfo & 0xffffff) != u.b;
        double ov = 0.0;
        if (!zero) {
          GroupDot<VT, G> d;
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const int r = gl + G * j;
            if (r < u.dim) d.add(u.Q(0, r), __ldcg(hvec + (size_t)oslot * vstride + r));
          }
          ov = d.value(gm);
          zero = (ov == 0.0);
        }
        int st = u.status;
        if (oinfo >= 0 && (oinfo >> 24) > st) st = oinfo >> 24;
        const double L = Lh + Lo + (zero ? 0.0 : log(fabs(ov)));
        if (!zero && !isfinite(L)) st = KT_ENUMERIC;
        if (meas && !zero) measure_epilogue(M, u, ws, item, hvec + (size_t)oslot * vstride, ov);
        if (gl == 0) {
          ws.item_sign[item] = zero ? 0 : (ov > 0.0 ? 1 : -1);
          ws.item_log[item] = zero ? -INFINITY : L;
          ws.item_status[item] = st;
        }
      }
    }
    if ((OPT & KT_OPT_STATS) && gl == 0 && stats) {
      stat_add(&stats->ops_applied, u.acc.ops);
      stat_add(&stats->intervals, u.acc.intervals);
      stat_add(&stats->krylov_iters, u.acc.iters);
      if (u.acc.pmax) atomicMax(&stats->p_max, u.acc.pmax);
      stat_add(&stats->noconv, u.acc.noconv);
      stat_add(&stats->flops_vec, u.acc.flops_vec);
      stat_add(&stats->flops_tri, u.acc.flops_tri);
      stat_add(&stats->bytes_apply, u.acc.bytes_apply);
      stat_add(&stats->flops_alg, u.acc.flops_alg);
      stat_add(&stats->flops_reorth, u.acc.flops_reorth);
    }
    __syncwarp(gm);
  }
}

// launch helpers
template <typename VT, int G, int DMAX, int PMAX, int OPT>
int launch_items(const DevModel &M, const SeqView &S, const MoveView &mv, int has_moves, const Workspace &ws,
                 kt_stats *stats, cudaStream_t st) {
  using Tile = WarpTile<VT, G, DMAX, PMAX>;
  static int cached_grid = 0, cached_wpb = 0;
  if (cached_grid == 0) {
    int wpb = (int)((200 * 1024) / sizeof(Tile));
    wpb = wpb < 1 ? 1 : (wpb > 8 ? 8 : wpb);
    const size_t smem = (size_t)wpb * sizeof(Tile);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(items_kernel<VT, G, DMAX, PMAX, OPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, items_kernel<VT, G, DMAX, PMAX, OPT>, wpb * 32, smem);
    if (per_sm < 1) per_sm = 1;
    cached_wpb = wpb;
    cached_grid = sms * per_sm;
  }
  const size_t smem = (size_t)cached_wpb * sizeof(Tile);
  items_kernel<VT, G, DMAX, PMAX, OPT><<<cached_grid, cached_wpb * 32, smem, st>>>(M, S, mv, has_moves, ws, stats);
  return (int)cudaGetLastError();
}


template <typename VT, int G, int DMAX, int PMAX, int OPT>
int launch_items_cached(const DevModel &M, const SeqView &S, const MoveView &mv, const Workspace &ws,
                        const CacheView &C, kt_stats *stats, cudaStream_t st) {
  using Tile = WarpTile<VT, G, DMAX, PMAX>;
  static int cached_grid = 0, cached_wpb = 0;
  if (cached_grid == 0) {
    int wpb = (int)((200 * 1024) / sizeof(Tile));
    wpb = wpb < 1 ? 1 : (wpb > 8 ? 8 : wpb);
    const size_t smem = (size_t)wpb * sizeof(Tile);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(items_cached_kernel<VT, G, DMAX, PMAX, OPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, items_cached_kernel<VT, G, DMAX, PMAX, OPT>, wpb * 32, smem);
    if (per_sm < 1) per_sm = 1;
    cached_wpb = wpb;
    cached_grid = sms * per_sm;
  }
  const size_t smem = (size_t)cached_wpb * sizeof(Tile);
  items_cached_kernel<VT, G, DMAX, PMAX, OPT><<<cached_grid, cached_wpb * 32, smem, st>>>(M, S, mv, ws, C, stats);
  return (int)cudaGetLastError();
}

// The options a launch needs: KT_OPT_TRI64 only where the FP32 path's blocks have at most 16
// rows (larger ones always take the FP64 steps), KT_OPT_MEAS when the observables are asked for,
// KT_OPT_STATS when the work is counted.
template <typename VT>
int items_options(int kd, const DevModel &M, const Workspace &ws, const kt_stats *stats) {
  return (sizeof(VT) == 4 && kd <= 16 && M.tri64 ? KT_OPT_TRI64 : 0) | (ws.item_obs ? KT_OPT_MEAS : 0) |
         (stats ? KT_OPT_STATS : 0);
}

// Launches without options: every compiled (rows, lane group) variant.
template <typename VT>
int dispatch_items(int kd, int G, const DevModel &M, const SeqView &S, const MoveView &mv, int has_moves,
                   const Workspace &ws, kt_stats *stats, cudaStream_t st) {
#define KT_CASE(D, P, GG) \
  if (kd == D && G == GG) return launch_items<VT, GG, D, P, 0>(M, S, mv, has_moves, ws, stats, st);
  KT_FOR_VARIANTS(KT_CASE)
#undef KT_CASE
  return (int)cudaErrorInvalidValue;
}

}  // namespace dev
}  // namespace kt
