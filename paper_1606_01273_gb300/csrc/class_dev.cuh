// Classes A-G (internal): index helpers shared by the solve (class_ag.cu) and the
// densities (density_ag.cu).
#pragma once
#include <algorithm>
#include <cmath>

#include "class_ag.cuh"

namespace caspt2 {

__device__ __forceinline__ long ipow(int a, int k) {
  long r = 1;
  for (int i = 0; i < k; ++i) r *= a;
  return r;
}

// <M~|..|N~> RDM element of rank `rank` at the indices vals[idx[0..2 rank)].
__device__ __forceinline__ double rdm_at(const double* const* g, int rank, int n, int a, int M,
                                         int N, const int* vals, const int8_t* idx) {
  if (rank == 0) return M == N ? 1.0 : 0.0;
  long off = 0;
  for (int j = 0; j < 2 * rank; ++j) off = off * a + vals[idx[j]];
  return g[rank][((long)M * n + N) * ipow(a, 2 * rank) + off];
}

__device__ __forceinline__ void tri_decode(long t, int R, bool strict, int& x, int& y) {
  // enumerate x <= y (or x < y) row-major by x over [0, R)
  const int w = strict ? R - 1 : R;
  double b = 2.0 * w + 1.0;
  int xx = (int)floor((b - sqrt(b * b - 8.0 * (double)t)) * 0.5);
  if (xx < 0) xx = 0;
  auto start = [&](int q) { return (long)q * w - (long)q * (q - 1) / 2; };
  while (xx > 0 && start(xx) > t) --xx;
  while (start(xx + 1) <= t) ++xx;
  x = xx;
  y = (int)(t - start(xx)) + xx + (strict ? 1 : 0);
}

// Sector tuple -> coordinates of the external slots (output order of C.ext) and the
// partner tuple with the pair swapped.
__device__ __forceinline__ void sector_tuple(const DevClass& C, const int* extdim, int sector,
                                             long t, int* co, int* co_sw) {
  if (C.pair0 < 0) {
    for (int k = C.next - 1; k >= 0; --k) {
      co[k] = t % extdim[k];
      t /= extdim[k];
      co_sw[k] = co[k];
    }
    return;
  }
  int ip = -1, jp = -1;
  for (int k = 0; k < C.next; ++k) {
    if (C.ext[k] == C.pair0) ip = k;
    if (C.ext[k] == C.pair1) jp = k;
  }
  const int R = extdim[ip];
  const bool strict = sector == 1;
  const long npairs = strict ? (long)R * (R - 1) / 2 : (long)R * (R + 1) / 2;
  const long pidx = t % npairs;
  t /= npairs;
  for (int k = C.next - 1; k >= 0; --k) {
    if (k == ip || k == jp) continue;
    co[k] = t % extdim[k];
    t /= extdim[k];
  }
  int x, y;
  tri_decode(pidx, R, strict, x, y);
  co[ip] = x;
  co[jp] = y;
  for (int k = 0; k < C.next; ++k) co_sw[k] = co[k];
  co_sw[ip] = y;
  co_sw[jp] = x;
}

// Row-major index of an external tuple over all tuples (slots in C.ext order).
__device__ __forceinline__ long tuple_index(const DevClass& C, const int* extdim, const int* co) {
  long t = 0;
  for (int k = 0; k < C.next; ++k) t = t * extdim[k] + co[k];
  return t;
}

inline long ipow_host(int a, int k) {
  long r = 1;
  for (int i = 0; i < k; ++i) r *= a;
  return r;
}

inline int launch_blocks(long total, int threads = 256) {
  long b = (total + threads - 1) / threads;
  return (int)std::max<long>(1, std::min<long>(b, 152L * 32));
}
inline int space_dim(const Dims& d, int sp) { return sp == SP_C ? d.c : (sp == SP_A ? d.a : d.v); }
inline int space_off(const Dims& d, int sp) {
  return sp == SP_C ? 0 : (sp == SP_A ? d.c : d.c + d.a);
}

// Number of tuples of a sector (0: identity or symmetric, 1: antisymmetric).
inline long sector_tuples(const ClassWork& w, int sector) {
  const DevClass& C = w.dc;
  if (C.pair0 < 0) {
    long t = 1;
    for (int k = 0; k < C.next; ++k) t *= w.ed.d[k];
    return sector == 0 ? t : 0;
  }
  long t = 1, R = 0;
  for (int k = 0; k < C.next; ++k) {
    if (C.ext[k] == C.pair0) R = w.ed.d[k];
    else if (C.ext[k] != C.pair1) t *= w.ed.d[k];
  }
  return t * (sector == 0 ? R * (R + 1) / 2 : R * (R - 1) / 2);
}

// All external tuples of a class (product of the external dimensions).
inline long all_tuples(const ClassWork& w) {
  long t = 1;
  for (int k = 0; k < w.dc.next; ++k) t *= w.ed.d[k];
  return t;
}

}  // namespace caspt2
