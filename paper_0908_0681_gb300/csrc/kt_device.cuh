// Device helpers shared by the kernels of the engine (internal).
#pragma once

#include <cuda_runtime.h>

#include <math.h>
#include <stdint.h>

#include "kt_internal.h"

namespace kt {
namespace dev {


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

// Number of entries of the sorted t[0 .. K) that are < x.
__device__ __forceinline__ int lower_bound(const double *t, int K, double x) {
  int lo = 0, hi = K;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (t[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void stat_add(unsigned long long *p, unsigned long long v) {
  if (v) atomicAdd(p, v);
}

}  // namespace dev
}  // namespace kt
