// FP64 symmetric eigensolver for the per-class overlap and Fock matrices
// (Sec. II.B: eigenvalues of the overlap below the threshold are truncated):
//   1. Householder reduction to tridiagonal form, T = Q^T A Q (one reflector per step:
//      p = tau A22 v, w = p - (tau/2)(p.v) v, A22 -= v w^T + w v^T);
//   2. every eigenvalue of T by bisection on Sturm counts (one thread per eigenvalue,
//      absolute accuracy ~ eps ||T||);
//   3. every eigenvector of T by inverse iteration on the pivoted tridiagonal LU
//      (one thread per eigenvalue), Gram-Schmidt inside clusters of equal eigenvalues;
//   4. one Newton-Schulz step Z <- Z (3 - Z^T Z) / 2 to restore orthogonality to
//      rounding level;
//   5. back-transformation V = Q Z by applying the reflectors in reverse order.
#include <vector>

#include "linalg.cuh"

namespace caspt2 {

namespace {

constexpr int kT = 256;

int nblocks(long total, int threads = kT) {
  long b = (total + threads - 1) / threads;
  return (int)std::max<long>(1, std::min<long>(b, 152L * 32));
}

}  // namespace

// Reflector for column k: x = A[k][k+1..m-1] (row k, symmetric storage).
// v is stored in vbuf[k*m + k+1 ..] with v[k+1] = 1; tau[k]; d[k] = A[k][k]; e[k] = beta.
__global__ void k_house(double* __restrict__ A, int m, int k, double* __restrict__ vbuf,
                        double* __restrict__ tau, double* __restrict__ d, double* __restrict__ e) {
  __shared__ double red[32];
  __shared__ double sh[2];
  const double* x = A + (long)k * m + k + 1;
  const int n1 = m - k - 1;
  double s = 0.0;
  for (int i = 1 + threadIdx.x; i < n1; i += blockDim.x) s += x[i] * x[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    const double alpha = x[0];
    double beta, t, scale;
    if (s == 0.0) {
      beta = alpha;
      t = 0.0;
      scale = 0.0;
    } else {
      beta = -copysign(sqrt(alpha * alpha + s), alpha);
      t = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    sh[0] = t;
    sh[1] = scale;
    tau[k] = t;
    d[k] = A[(long)k * m + k];
    e[k] = beta;
  }
  __syncthreads();
  const double scale = sh[1];
  double* v = vbuf + (long)k * m + k + 1;
  for (int i = threadIdx.x; i < n1; i += blockDim.x) v[i] = (i == 0) ? 1.0 : x[i] * scale;
}

// p[i] = tau * sum_j A22[i][j] v[j], one warp per row of the trailing block
__global__ void k_symv(const double* __restrict__ A, int m, int k, const double* __restrict__ vbuf,
                       const double* __restrict__ tau, double* __restrict__ p) {
  const int n1 = m - k - 1;
  const double* v = vbuf + (long)k * m + k + 1;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const double t = tau[k];
  for (int i = warp; i < n1; i += nw) {
    const double* row = A + (long)(k + 1 + i) * m + k + 1;
    double s = 0.0;
    for (int j = lane; j < n1; j += 32) s += row[j] * v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) p[i] = t * s;
  }
}

// A22 -= v w^T + w v^T with w = p - (tau/2)(p.v) v  (each block recomputes p.v)
__global__ void k_rank2(double* __restrict__ A, int m, int k, const double* __restrict__ vbuf,
                        const double* __restrict__ tau, const double* __restrict__ p) {
  __shared__ double red[32];
  __shared__ double sg;
  const int n1 = m - k - 1;
  const double* v = vbuf + (long)k * m + k + 1;
  double s = 0.0;
  for (int i = threadIdx.x; i < n1; i += blockDim.x) s += p[i] * v[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) sg = 0.5 * tau[k] * s;
  __syncthreads();
  const double g = sg;
  const long total = (long)n1 * n1;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const int i = t / n1, j = t % n1;
    const double wi = p[i] - g * v[i], wj = p[j] - g * v[j];
    A[(long)(k + 1 + i) * m + k + 1 + j] -= v[i] * wj + wi * v[j];
  }
}

// Grid-wide barrier for a cooperative launch, bounded: after kSpinLimit polls it sets
// *err and returns false so that every block can leave the kernel.
constexpr long kSpinLimit = 1L << 24;

__device__ bool grid_sync_bounded(unsigned* count, volatile unsigned* gen, int* err) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      *count = 0;
      __threadfence();
      atomicAdd((unsigned*)gen, 1u);
      ok = 1;
    } else {
      long it = 0;
      while (*gen == g && *(volatile int*)err == 0) {
        if (++it > kSpinLimit) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(64);
      }
      ok = (*(volatile int*)err == 0);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Reflector of row k from its trailing part (one block): tau, d[k], e[k] = beta, v.
__device__ void house_row(double* __restrict__ A, int m, int k, double* __restrict__ vbuf,
                          double* __restrict__ tau, double* __restrict__ d,
                          double* __restrict__ e, double* red, double* sh) {
  const int n1 = m - k - 1;
  const double* x = A + (long)k * m + k + 1;
  double s = 0.0;
  for (int i = 1 + threadIdx.x; i < n1; i += blockDim.x) s += __ldcg(x + i) * __ldcg(x + i);
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    const double alpha = __ldcg(x);
    double beta, t, scale;
    if (s == 0.0) { beta = alpha; t = 0.0; scale = 0.0; }
    else {
      beta = -copysign(sqrt(alpha * alpha + s), alpha);
      t = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    sh[1] = scale;
    tau[k] = t;
    d[k] = __ldcg(A + (long)k * m + k);
    e[k] = beta;
  }
  __syncthreads();
  const double scale = sh[1];
  double* v = vbuf + (long)k * m + k + 1;
  for (int i = threadIdx.x; i < n1; i += blockDim.x) v[i] = (i == 0) ? 1.0 : __ldcg(x + i) * scale;
  __syncthreads();
}

// Householder reduction in one cooperative launch, two bounded grid barriers per step:
//   p = tau A22 v (warps over rows)                              | barrier
//   A22 -= v w^T + w v^T; block 0 then forms the next reflector   | barrier
// from row k+1, which its warp 0 has just finished updating.
// sync[0..1] barrier state (zeroed by the host), sync[2] error flag.
__global__ void __launch_bounds__(512)
k_tridiag(double* __restrict__ A, int m, double* __restrict__ vbuf, double* __restrict__ tau,
          double* __restrict__ d, double* __restrict__ e, double* __restrict__ p,
          unsigned* sync) {
  __shared__ double red[32];
  __shared__ double sh[2];
  int* err = reinterpret_cast<int*>(sync + 2);
  if (blockIdx.x == 0) house_row(A, m, 0, vbuf, tau, d, e, red, sh);
  if (!grid_sync_bounded(sync, sync + 1, err)) return;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int k = 0; k + 2 < m; ++k) {
    const int n1 = m - k - 1;
    const double* v = vbuf + (long)k * m + k + 1;
    const double t = __ldcg(tau + k);
    for (int i = warp; i < n1; i += nw) {
      const double* row = A + (long)(k + 1 + i) * m + k + 1;
      double s = 0.0;
      for (int j = lane; j < n1; j += 32) s += __ldcg(row + j) * __ldcg(v + j);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) p[i] = t * s;
    }
    if (!grid_sync_bounded(sync, sync + 1, err)) return;
    double s = 0.0;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) s += __ldcg(p + i) * __ldcg(v + i);
    s = block_sum(s, red);
    if (threadIdx.x == 0) sh[0] = 0.5 * t * s;
    __syncthreads();
    const double g = sh[0];
    for (int i = warp; i < n1; i += nw) {
      const double vi = __ldcg(v + i), wi = __ldcg(p + i) - g * vi;
      double* row = A + (long)(k + 1 + i) * m + k + 1;
      for (int j = lane; j < n1; j += 32) {
        const double vj = __ldcg(v + j), wj = __ldcg(p + j) - g * vj;
        row[j] = __ldcg(row + j) - (vi * wj + wi * vj);
      }
    }
    if (blockIdx.x == 0 && k + 3 < m) {
      __syncthreads();
      house_row(A, m, k + 1, vbuf, tau, d, e, red, sh);
    }
    if (!grid_sync_bounded(sync, sync + 1, err)) return;
  }
}

// Householder reflector of x[0..n1) (x[0] = alpha): tau, beta and v (v[0] = 1) written
// by every calling block; the reduction order is fixed, so all blocks obtain bitwise
// identical results from identical x.
__device__ void house_vec(const double* __restrict__ x, int n1, double* __restrict__ v,
                          double* red, double* sh) {
  double s = 0.0;
  for (int i = 1 + threadIdx.x; i < n1; i += blockDim.x) s += x[i] * x[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    const double alpha = x[0];
    double beta, t, scale;
    if (s == 0.0) { beta = alpha; t = 0.0; scale = 0.0; }
    else {
      beta = -copysign(sqrt(alpha * alpha + s), alpha);
      t = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    sh[0] = t;
    sh[1] = scale;
    sh[2] = beta;
  }
  __syncthreads();
  const double scale = sh[1];
  for (int i = threadIdx.x; i < n1; i += blockDim.x) v[i] = (i == 0) ? 1.0 : x[i] * scale;
  __syncthreads();
}

// Householder reduction with the matrix resident in shared memory: block b owns the
// rows r = b (mod gridDim.x).  One bounded grid barrier per step:
//   p_i = tau sum_j A_ij v_j for owned rows (published)                | barrier
//   every block: w = p - (tau/2)(p.v) v, update of its rows, and — redundantly — the
//   update of row k+1 (published by its owner after the previous step) and the next
//   reflector, so no second barrier is needed; the owner of row k+2 publishes it.
// Shared layout: rows [nloc][m], v[m], w[m], r[m] (all indexed by absolute column).
// pbuf[2][m], rowbuf[2][m] are double-buffered by step parity; sync[0..1] barrier state,
// sync[2] error flag.
__global__ void __launch_bounds__(512)
k_tridiag_smem(const double* __restrict__ A, int m, double* __restrict__ vbuf,
               double* __restrict__ tau, double* __restrict__ d, double* __restrict__ e,
               double* __restrict__ pbuf, double* __restrict__ rowbuf, unsigned* sync) {
  extern __shared__ double smem[];
  __shared__ double red[32];
  __shared__ double sh[4];
  int* err = reinterpret_cast<int*>(sync + 2);
  const int G = gridDim.x, b = blockIdx.x;
  const int nloc = (m - b + G - 1) / G;            // rows b, b+G, ...
  double* rows = smem;
  double* v = rows + (long)((m + G - 1) / G) * m;
  double* w = v + m;
  double* r = w + m;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (long q = threadIdx.x; q < (long)nloc * m; q += blockDim.x) {
    const int li = q / m, j = q % m;
    rows[q] = A[(long)(b + li * G) * m + j];
  }
  // reflector of row 0 (every block from the input)
  for (int j = threadIdx.x; j < m; j += blockDim.x) r[j] = A[j];
  __syncthreads();
  house_vec(r + 1, m - 1, v + 1, red, sh);
  double t = sh[0];
  if (b == 0) {
    for (int i = threadIdx.x; i < m - 1; i += blockDim.x) vbuf[1 + i] = v[1 + i];
    if (threadIdx.x == 0) { tau[0] = t; d[0] = r[0]; e[0] = sh[2]; }
  }
  for (int k = 0; k + 2 < m; ++k) {
    const int k1 = k + 1;
    // p for the owned trailing rows
    const int lfirst = (k1 - b + G - 1) / G;       // first owned row index >= k+1
    for (int li = lfirst + warp; li < nloc; li += nwarp) {
      const double* row = rows + (long)li * m;
      double s = 0.0;
      for (int j = k1 + lane; j < m; j += 32) s += row[j] * v[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) pbuf[(long)(k & 1) * m + b + li * G] = t * s;
    }
    if (!grid_sync_bounded(sync, sync + 1, err)) return;
    // w = p - (tau/2)(p.v) v
    double s = 0.0;
    for (int j = k1 + threadIdx.x; j < m; j += blockDim.x) {
      const double pj = __ldcg(pbuf + (long)(k & 1) * m + j);
      w[j] = pj;
      s += pj * v[j];
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) sh[3] = 0.5 * t * s;
    __syncthreads();
    const double g = sh[3];
    for (int j = k1 + threadIdx.x; j < m; j += blockDim.x) w[j] -= g * v[j];
    __syncthreads();
    // update of the owned rows
    const long nq = (long)(nloc - lfirst) * (m - k1);
    for (long q = threadIdx.x; q < nq; q += blockDim.x) {
      const int li = lfirst + (int)(q / (m - k1));
      const int j = k1 + (int)(q % (m - k1));
      const int i = b + li * G;
      rows[(long)li * m + j] -= v[i] * w[j] + w[i] * v[j];
    }
    // row k+1 after this step (every block, from the copy published before the barrier)
    const double* old = (k == 0) ? A + (long)k1 * m : rowbuf + (long)(k1 & 1) * m;
    for (int j = k1 + threadIdx.x; j < m; j += blockDim.x)
      r[j] = __ldcg(old + j) - (v[k1] * w[j] + w[k1] * v[j]);
    __syncthreads();
    // the owner of row k+2 publishes it for the next step
    const int k2 = k + 2;
    if (k2 < m && (k2 % G) == b) {
      const double* row = rows + (long)(k2 / G) * m;
      for (int j = k2 + threadIdx.x; j < m; j += blockDim.x)
        rowbuf[(long)(k2 & 1) * m + j] = row[j];
    }
    if (k + 3 < m) {
      // next reflector from row k+1's trailing part (v is free again)
      house_vec(r + k2, m - k2, v + k2, red, sh);
      t = sh[0];
      if (b == 0) {
        for (int i = threadIdx.x; i < m - k2; i += blockDim.x)
          vbuf[(long)k1 * m + k2 + i] = v[k2 + i];
        if (threadIdx.x == 0) { tau[k1] = t; d[k1] = r[k1]; e[k1] = sh[2]; }
      }
    } else if (b == 0 && threadIdx.x == 0) {
      d[m - 2] = r[m - 2];
      e[m - 2] = r[m - 1];
    }
    __syncthreads();
  }
  // last diagonal element from its owner
  if (m >= 2 && ((m - 1) % G) == b && threadIdx.x == 0)
    d[m - 1] = rows[(long)((m - 1) / G) * m + m - 1];
}

// Shared memory of k_tridiag_smem for m columns on G blocks (0 if it does not fit).
constexpr size_t kTridiagSmemMax = 200ull * 1024;
constexpr size_t kBisectSmemMax = 200ull * 1024;    // d and e^2 of the tridiagonal matrix
size_t tridiag_smem_bytes(int m, int G) {
  const size_t b = 8ull * ((size_t)((m + G - 1) / G) * m + 3ull * m);
  return b <= kTridiagSmemMax ? b : 0;
}

__global__ void k_tail(const double* __restrict__ A, int m, double* d, double* e) {
  if (threadIdx.x != 0) return;
  if (m >= 2) {
    d[m - 2] = A[(long)(m - 2) * m + m - 2];
    e[m - 2] = A[(long)(m - 2) * m + m - 1];
  }
  d[m - 1] = A[(long)(m - 1) * m + m - 1];
  e[m - 1] = 0.0;
}

// Sturm count: number of eigenvalues of T below x
__device__ int sturm(const double* __restrict__ d, const double* __restrict__ e2, int m, double x,
                     double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < 0.0) ++cnt;
  for (int i = 1; i < m; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

__global__ void k_e2(const double* __restrict__ e, int m, double* __restrict__ e2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) e2[i] = (i < m - 1) ? e[i] * e[i] : 0.0;
}

// Number of eigenvalues of T below x from the sign changes of the leading principal
// minors p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (p_{-1} = 1): three FP64 operations
// per step and no division.  Signs, exact zeros (which take the sign opposite to their
// predecessor) and the range check are integer operations on the bit patterns; the pair
// (p_i, p_{i-1}) is rescaled by 2^(-+500) when |p_i| leaves [2^-600, 2^600], checked every
// 4 steps (|p| grows by at most (2||T|| + ||T||^2) per step, far inside the FP64 range).
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }

__device__ int sturm_nodiv(const double* __restrict__ d, const double* __restrict__ e2, int m,
                           double x) {
  double pm = 1.0, pc = d[0] - x;
  if ((dbits(pc) << 1) == 0) pc = -1e-300;
  int cnt = (int)((unsigned long long)dbits(pc) >> 63);
  for (int i = 1; i < m; ++i) {
    double pn = fma(d[i] - x, pc, -e2[i - 1] * pm);
    const long long bn = dbits(pn), bc = dbits(pc);
    if ((bn << 1) == 0) pn = bc < 0 ? 1e-300 : -1e-300;
    cnt += (int)((unsigned long long)(dbits(pn) ^ bc) >> 63);
    pm = pc;
    pc = pn;
    if ((i & 3) == 0) {
      const int ex = (int)((dbits(pc) >> 52) & 0x7FF);
      const int exm = (int)((dbits(pm) >> 52) & 0x7FF);
      if (ex > 1023 + 600) { pc *= 0x1p-500; pm *= 0x1p-500; }
      else if (ex < 1023 - 600 && exm < 1023 - 600) { pc *= 0x1p500; pm *= 0x1p500; }
    }
  }
  return cnt;
}

// j-th smallest eigenvalue by 4-way multisection inside the Gershgorin interval: four
// lanes per eigenvalue evaluate the Sturm count at the three interior quarter points
// (lane 3 idles), so each step removes two bits; stop at an absolute width of tol.
__global__ void k_bisect(const double* __restrict__ dg, const double* __restrict__ e,
                         const double* __restrict__ e2g, int m, double glo, double ghi, double tol,
                         double* __restrict__ w) {
  extern __shared__ double sde[];      // d[m], e2[m] staged per block
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    sde[i] = dg[i];
    sde[m + i] = e2g[i];
  }
  __syncthreads();
  const double* d = sde;
  const double* e2 = sde + m;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = gid >> 2, q = gid & 3;
  const unsigned grp = 0xFu << (threadIdx.x & 28);
  if ((gid & ~3) >= ((m + 0) << 2)) return;          // whole group beyond m
  const bool live = j < m;
  double lo = glo, hi = ghi;
  for (int it = 0; it < 80; ++it) {
    if (hi - lo <= tol) break;
    const double h = 0.25 * (hi - lo);
    const double x = lo + h * (q + 1);
    const bool above = live && q < 3 && x > lo && x < hi && sturm_nodiv(d, e2, m, x) > j;
    const unsigned b = (__ballot_sync(grp, above) >> (threadIdx.x & 28)) & 0x7u;
    const int first = b ? (__ffs(b) - 1) : 3;           // first quarter point above j
    const double nhi = first < 3 ? lo + h * (first + 1) : hi;
    const double nlo = first > 0 ? lo + h * first : lo;
    if (!(nhi < hi || nlo > lo)) break;
    lo = nlo;
    hi = nhi;
  }
  if (live && q == 0) w[j] = 0.5 * (lo + hi);
}

__device__ __forceinline__ double hash_unit(unsigned a, unsigned b) {
  unsigned h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
  return (double)(h & 0xFFFFFF) / 16777216.0 + 0.5;   // in [0.5, 1.5)
}

// Inverse iteration for eigenvalue j (thread j).  Scratch arrays are laid out
// [i][j] so that threads access consecutive addresses.  Z[i][j] = component i of vector j.
__global__ void k_inviter(const double* __restrict__ d, const double* __restrict__ e,
                          const double* __restrict__ w, int m, double tnorm,
                          double* __restrict__ u0, double* __restrict__ u1,
                          double* __restrict__ u2, double* __restrict__ lm,
                          double* __restrict__ pv, double* __restrict__ Z) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const double lam = w[j];
  const double tiny = 2.2e-16 * (tnorm > 0 ? tnorm : 1.0);
#define IX(i) ((long)(i) * m + j)
  // factor T - lam I = P L U, U with two superdiagonals
  for (int i = 0; i < m; ++i) {
    u0[IX(i)] = d[i] - lam;
    u1[IX(i)] = (i < m - 1) ? e[i] : 0.0;
    u2[IX(i)] = 0.0;
  }
  for (int i = 0; i < m - 1; ++i) {
    const double c = e[i];          // subdiagonal element of row i+1
    const double a = u0[IX(i)];
    if (fabs(a) >= fabs(c)) {
      const double piv = (a == 0.0) ? tiny : a;
      u0[IX(i)] = piv;
      const double l = c / piv;
      lm[IX(i)] = l;
      pv[IX(i)] = 0.0;
      u0[IX(i + 1)] -= l * u1[IX(i)];
    } else {
      const double l = a / c;
      lm[IX(i)] = l;
      pv[IX(i)] = 1.0;
      const double b_i = u1[IX(i)];
      const double a_n = u0[IX(i + 1)], b_n = u1[IX(i + 1)];
      u0[IX(i)] = c;
      u1[IX(i)] = a_n;
      u2[IX(i)] = b_n;
      u0[IX(i + 1)] = b_i - l * a_n;
      u1[IX(i + 1)] = -l * b_n;
    }
  }
  if (u0[IX(m - 1)] == 0.0) u0[IX(m - 1)] = tiny;
  // pivots -> reciprocals (|pivot| raised to tiny), so the solves below multiply
  for (int i = 0; i < m; ++i) {
    double piv = u0[IX(i)];
    if (fabs(piv) < tiny) piv = copysign(tiny, piv == 0.0 ? 1.0 : piv);
    u0[IX(i)] = 1.0 / piv;
  }
  // start vector
  for (int i = 0; i < m; ++i) Z[IX(i)] = hash_unit(i, j);
  for (int iter = 0; iter < 3; ++iter) {
    // apply L^-1 with the row interchanges
    for (int i = 0; i < m - 1; ++i) {
      double yi = Z[IX(i)], yn = Z[IX(i + 1)];
      if (pv[IX(i)] != 0.0) {
        const double t = yi; yi = yn; yn = t;
      }
      Z[IX(i)] = yi;
      Z[IX(i + 1)] = yn - lm[IX(i)] * yi;
    }
    // U^-1 with overflow guard
    double big = 0.0;
    for (int i = m - 1; i >= 0; --i) {
      double x = Z[IX(i)];
      if (i + 1 < m) x -= u1[IX(i)] * Z[IX(i + 1)];
      if (i + 2 < m) x -= u2[IX(i)] * Z[IX(i + 2)];
      x *= u0[IX(i)];
      Z[IX(i)] = x;
      big = fmax(big, fabs(x));
      if (big > 1e100) {  // rescale the partial solution
        for (int k2 = i; k2 < m; ++k2) Z[IX(k2)] *= 1e-100;
        big *= 1e-100;
      }
    }
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += Z[IX(i)] * Z[IX(i)];
    nrm = 1.0 / sqrt(nrm);
    for (int i = 0; i < m; ++i) Z[IX(i)] *= nrm;
  }
#undef IX
}

// Modified Gram-Schmidt inside each cluster of (numerically) equal eigenvalues.
// One block per eigenvalue index; only cluster starts do work.
__global__ void k_cluster_mgs(const double* __restrict__ w, int m, double tol,
                              double* __restrict__ Z) {
  __shared__ double red[32];
  __shared__ double sc;
  const int j0 = blockIdx.x;
  if (j0 > 0 && w[j0] - w[j0 - 1] <= tol) return;            // not a start
  if (j0 + 1 >= m || w[j0 + 1] - w[j0] > tol) return;         // singleton
  int j1 = j0 + 1;
  while (j1 + 1 < m && w[j1 + 1] - w[j1] <= tol) ++j1;
  for (int j = j0; j <= j1; ++j) {
    for (int k = j0; k < j; ++k) {
      double s = 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) s += Z[(long)i * m + k] * Z[(long)i * m + j];
      s = block_sum(s, red);
      if (threadIdx.x == 0) sc = s;
      __syncthreads();
      const double proj = sc;
      for (int i = threadIdx.x; i < m; i += blockDim.x) Z[(long)i * m + j] -= proj * Z[(long)i * m + k];
      __syncthreads();
    }
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s += Z[(long)i * m + j] * Z[(long)i * m + j];
    s = block_sum(s, red);
    if (threadIdx.x == 0) sc = (s > 0.0) ? 1.0 / sqrt(s) : 0.0;
    __syncthreads();
    const double nr = sc;
    for (int i = threadIdx.x; i < m; i += blockDim.x) Z[(long)i * m + j] *= nr;
    __syncthreads();
  }
}

// G = 1.5 I - 0.5 G (in place)
__global__ void k_ns_coef(double* __restrict__ G, int m) {
  const long total = (long)m * m;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x)
    G[t] = ((t / m == t % m) ? 1.5 : 0.0) - 0.5 * G[t];
}

// r[c] = sum_i v[i] Z[k+1+i][c]: 32 columns x 8 row groups per block (coalesced rows),
// fixed-order reduction over the row groups in shared memory.
__global__ void __launch_bounds__(256)
k_vtz(const double* __restrict__ vbuf, int m, int k, const double* __restrict__ Z,
      double* __restrict__ r) {
  __shared__ double part[8][33];
  const int n1 = m - k - 1;
  const double* v = vbuf + (long)k * m + k + 1;
  const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + cx;
  double s = 0.0;
  if (c < m) {
#pragma unroll 4
    for (int i = ry; i < n1; i += 8) s += v[i] * Z[(long)(k + 1 + i) * m + c];
  }
  part[ry][cx] = s;
  __syncthreads();
  if (ry == 0 && c < m) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += part[q][cx];
    r[c] = t;
  }
}

// Back-transformation V = H_0 ... H_{m-3} Z with each block owning cb consecutive columns
// (cb = 8 with 32 row groups of 256 threads): for every reflector (in reverse order) the block
// forms r_c = v . Z[k+1.., c] for its columns over rg = blockDim / cb row groups and
// applies Z[k+1+i][c] -= tau v_i r_c.  Columns are independent, so no grid-wide
// synchronisation is needed.
__global__ void __launch_bounds__(256)
k_backtransform(const double* __restrict__ vbuf, const double* __restrict__ tau, int m, int cb,
                double* __restrict__ Z) {
  __shared__ double part[256];
  __shared__ double rc[32];
  const int rg = blockDim.x / cb;
  const int cx = threadIdx.x % cb, ry = threadIdx.x / cb;
  const bool act = ry < rg;
  const int c = blockIdx.x * cb + cx;
  for (int k = m - 3; k >= 0; --k) {
    const int n1 = m - k - 1;
    const double* v = vbuf + (long)k * m + k + 1;
    double s = 0.0;
    if (act && c < m)
      for (int i = ry; i < n1; i += rg) s += v[i] * Z[(long)(k + 1 + i) * m + c];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < cb) {
      double t = 0.0;
      for (int q = 0; q < rg; ++q) t += part[q * cb + threadIdx.x];
      rc[threadIdx.x] = t * tau[k];
    }
    __syncthreads();
    if (act && c < m) {
      const double r = rc[cx];
      for (int i = ry; i < n1; i += rg) Z[(long)(k + 1 + i) * m + c] -= v[i] * r;
    }
    __syncthreads();
  }
}

// Z[k+1+i][c] -= tau v[i] r[c]
__global__ void k_zupd(const double* __restrict__ vbuf, int m, int k,
                       const double* __restrict__ tau, const double* __restrict__ r,
                       double* __restrict__ Z) {
  const int n1 = m - k - 1;
  const double* v = vbuf + (long)k * m + k + 1;
  const double t = tau[k];
  const long total = (long)n1 * m;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total;
       q += (long)gridDim.x * blockDim.x) {
    const int i = q / m, c = q % m;
    Z[(long)(k + 1 + i) * m + c] -= t * v[i] * r[c];
  }
}

size_t sym_eig_tridiag_work(int m) { return (size_t)m * m * 9 + (size_t)m * 8 + 64; }

int sym_eig_tridiag(double* A, int m, double* w, double* V, double* work, cudaStream_t s,
                    KernelTimer* tm) {
  if (m <= 0) return CASPT2_OK;
  const long mm = (long)m * m;
  double* vbuf = work;            // m*m reflectors
  double* Z = vbuf + mm;          // m*m eigenvectors of T
  double* G = Z + mm;             // m*m Gram / scratch
  double* u0 = G + mm;            // 5*m*m inverse-iteration scratch
  double* u1 = u0 + mm;
  double* u2 = u1 + mm;
  double* lm = u2 + mm;
  double* pv = lm + mm;
  double* d = pv + mm;
  double* e = d + m;
  double* e2 = e + m;
  double* tau = e2 + m;
  double* p = tau + m;
  double* r = p + m;
  // 1. tridiagonalise (one cooperative launch for large matrices: rows resident in
  //    shared memory when they fit, else streamed through L2)
  int dev = 0, nsm = 0;
  CASPT2_CUDA_TRY(cudaGetDevice(&dev));
  CASPT2_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int Gs = std::max(1, std::min(nsm, m));
  const size_t smem_b = m > 64 ? tridiag_smem_bytes(m, Gs) : 0;
  if (smem_b > 0) {
    unsigned* sync = reinterpret_cast<unsigned*>(r);   // r is free until the back-transform
    double* pbuf = u0;                                 // u0.. are free until inverse iteration
    double* rowbuf = u0 + 2 * (long)m;
    // the attribute is global to the kernel: set the fixed maximum (never a per-launch
    // size) so that concurrent solves of different sizes cannot lower it under each other
    CASPT2_CUDA_TRY(cudaFuncSetAttribute(k_tridiag_smem,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTridiagSmemMax));
    CASPT2_CUDA_TRY(cudaMemsetAsync(sync, 0, 4 * sizeof(unsigned), s));
    const double* Ac = A;
    void* args[] = {&Ac, (void*)&m, &vbuf, &tau, &d, &e, &pbuf, &rowbuf, &sync};
    ++launch_counter();
    if (tm && tm->e0) CASPT2_CUDA_TRY(cudaEventRecord(tm->e0, s));
    CASPT2_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_tridiag_smem, Gs, 512, args, smem_b, s));
    if (tm && tm->e1) CASPT2_CUDA_TRY(cudaEventRecord(tm->e1, s));
    int herr = 0;
    CASPT2_CUDA_TRY(cudaMemcpyAsync(&herr, sync + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
    if (herr != 0) return CASPT2_ETIMEOUT;
    if (tm && tm->e0) {
      float ms = 0.f;
      CASPT2_CUDA_TRY(cudaEventElapsedTime(&ms, tm->e0, tm->e1));
      tm->ms += ms;
      tm->flops += 4.0 / 3.0 * (double)m * m * m;   // Householder tridiagonalisation
      ++tm->launches;
    }
  } else if (m > 64) {
    int per = 0;
    CASPT2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tridiag, 512, 0));
    const int grid = std::max(1, std::min(nsm * std::max(per, 1), nsm));
    unsigned* sync = reinterpret_cast<unsigned*>(r);   // r is free until the back-transform
    CASPT2_CUDA_TRY(cudaMemsetAsync(sync, 0, 4 * sizeof(unsigned), s));
    void* args[] = {&A, (void*)&m, &vbuf, &tau, &d, &e, &p, &sync};
    ++launch_counter();
    if (tm && tm->e0) CASPT2_CUDA_TRY(cudaEventRecord(tm->e0, s));
    CASPT2_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_tridiag, grid, 512, args, 0, s));
    if (tm && tm->e1) CASPT2_CUDA_TRY(cudaEventRecord(tm->e1, s));
    int herr = 0;
    CASPT2_CUDA_TRY(cudaMemcpyAsync(&herr, sync + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
    if (herr != 0) return CASPT2_ETIMEOUT;
    if (tm && tm->e0) {
      float ms = 0.f;
      CASPT2_CUDA_TRY(cudaEventElapsedTime(&ms, tm->e0, tm->e1));
      tm->ms += ms;
      tm->flops += 4.0 / 3.0 * (double)m * m * m;   // Householder tridiagonalisation
      ++tm->launches;
    }
  } else {
    for (int k = 0; k + 2 < m; ++k) {
      const int n1 = m - k - 1;
      ++launch_counter();
      k_house<<<1, 256, 0, s>>>(A, m, k, vbuf, tau, d, e);
      ++launch_counter();
      k_symv<<<std::max(1, std::min((n1 + 7) / 8, 152 * 8)), 256, 0, s>>>(A, m, k, vbuf, tau, p);
      ++launch_counter();
      k_rank2<<<nblocks((long)n1 * n1), kT, 0, s>>>(A, m, k, vbuf, tau, p);
    }
  }
  if (smem_b == 0) {
    ++launch_counter();
    k_tail<<<1, 32, 0, s>>>(A, m, d, e);
  }
  CASPT2_CUDA_TRY(cudaGetLastError());
  // Gershgorin interval and pivmin on the host (small vectors)
  std::vector<double> hd(m), he(m);
  CASPT2_CUDA_TRY(cudaMemcpyAsync(hd.data(), d, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(he.data(), e, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
  double glo = 1e300, ghi = -1e300, emax2 = 0.0, tnorm = 0.0;
  for (int i = 0; i < m; ++i) {
    const double r0 = (i > 0 ? fabs(he[i - 1]) : 0.0) + (i < m - 1 ? fabs(he[i]) : 0.0);
    glo = std::min(glo, hd[i] - r0);
    ghi = std::max(ghi, hd[i] + r0);
    if (i < m - 1) emax2 = std::max(emax2, he[i] * he[i]);
    tnorm = std::max(tnorm, fabs(hd[i]) + r0);
    if (!(hd[i] == hd[i]) || !(he[i] == he[i])) return CASPT2_ENAN;
  }
  const double pad = 2.2e-16 * std::max(1.0, tnorm) * 4.0 + 1e-300;
  glo -= pad;
  ghi += pad;
  const double pivmin = std::max(1e-300, 1e-290 * std::max(1.0, emax2));
  // 2. eigenvalues
  ++launch_counter();
  k_e2<<<(m + 255) / 256, 256, 0, s>>>(e, m, e2);
  ++launch_counter();
  if (2 * sizeof(double) * (size_t)m > kBisectSmemMax) return CASPT2_EINVAL;
  CASPT2_CUDA_TRY(cudaFuncSetAttribute(k_bisect, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kBisectSmemMax));
  k_bisect<<<(4 * m + 127) / 128, 128, 2 * sizeof(double) * m, s>>>(
      d, e, e2, m, glo, ghi, 4.0 * 2.2e-16 * std::max(1.0, tnorm), w);
  // 3. eigenvectors of T
  ++launch_counter();
  k_inviter<<<(m + 127) / 128, 128, 0, s>>>(d, e, w, m, tnorm, u0, u1, u2, lm, pv, Z);
  ++launch_counter();
  k_cluster_mgs<<<m, 256, 0, s>>>(w, m, 1e-12 * std::max(1.0, tnorm), Z);
  CASPT2_CUDA_TRY(cudaGetLastError());
  // 4. Newton-Schulz: Z <- Z (1.5 I - 0.5 Z^T Z)
  CASPT2_CUDA_TRY(dgemm(m, m, m, 1.0, Z, m, true, Z, m, false, 0.0, G, m, s));
  ++launch_counter();
  k_ns_coef<<<nblocks(mm), kT, 0, s>>>(G, m);
  CASPT2_CUDA_TRY(dgemm(m, m, m, 1.0, Z, m, false, G, m, false, 0.0, V, m, s));
  // 5. back-transformation V = H_0 ... H_{m-3} Z (column-owned, one launch)
  if (m >= 3) {
    ++launch_counter();
    const int cb = 8;       // 8 columns x 32 row groups per block
    k_backtransform<<<(m + cb - 1) / cb, 256, 0, s>>>(vbuf, tau, m, cb, V);
  }
  CASPT2_CUDA_TRY(cudaGetLastError());
  return CASPT2_OK;
}

}  // namespace caspt2
