// FP64 symmetric eigensolver for the per-class overlap and Fock matrices
// (Sec. II.B: eigenvalues of the overlap below the threshold are truncated):
//   1. Householder reduction to tridiagonal form, T = Q^T A Q (one reflector per step:
//      p = tau A22 v, w = p - (tau/2)(p.v) v, A22 -= v w^T + w v^T);
//   2. every eigenvalue of T by bisection on Sturm counts (one thread per eigenvalue,
//      absolute accuracy ~ eps ||T||);
//   3. every eigenvector of T by inverse iteration on the pivoted tridiagonal LU
//      (one thread per eigenvalue), Gram-Schmidt inside clusters of equal eigenvalues;
//   4. one Newton-Schulz step Z <- Z (3 - Z^T Z) / 2 to restore orthogonality to
//      rounding level (skipped when Z^T Z is already within 1e-13 of the identity);
//   5. back-transformation V = Q Z by applying the reflectors in reverse order.
#include <cstring>
#include <vector>

#include "class_ag.cuh"
#include "ozaki.cuh"
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
    unsigned g;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(gen) : "memory");
    unsigned prev;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
                 : "=r"(prev) : "l"(count) : "memory");
    if (prev == gridDim.x - 1) {
      *count = 0;
      asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(gen), "r"(g + 1u) : "memory");
      ok = 1;
    } else {
      long it = 0;
      unsigned cur;
      for (;;) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(gen) : "memory");
        if (cur != g) break;
        if (*(volatile int*)err != 0) break;
        if (++it > kSpinLimit) {
          atomicExch(err, 1);
          break;
        }
        if (it > 64) __nanosleep(32);
      }
      ok = (*(volatile int*)err == 0);
    }
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

// Blocked Householder reduction, one cooperative launch per panel of b columns
// k0 .. k0+b-1 (the LAPACK dlatrd scheme, written from its definition): the trailing
// matrix is left as it stands during the panel and its true value is
// A22 - V W^T - W V^T, with V the panel's reflectors and W the vectors
// w = p - (tau/2)(p.v) v, p = tau (A22 - V W^T - W V^T) v.  After the panel the host
// applies A22 -= V W^T + W V^T as two FP64 GEMMs.  Per column k = k0 + j, three bounded
// grid barriers; blocks own contiguous runs of the rows (and of the columns of row k+1):
//   A: every block forms the reflector of row k from the row (already up to date) into
//      shared memory -- the reductions run in a fixed order, so every copy is the same;
//      block 0 stores it (vbuf row k, column j of Vr, tau, d, e);
//   B: p_raw = A22 v (a warp per half row, eight loads in flight per lane) and partial
//      sums of W^T v and V^T v;                                          | barrier
//   C: p = tau (p_raw - V (W^T v) - W (V^T v)) (a warp per owned row, lanes over the
//      panel columns) and partial sums of p.v;                           | barrier
//   D: alpha = (tau/2) p.v, W[:, j] = p - alpha v, and the owned columns of row k+1
//      brought up to date with the panel's columns 0..j.                 | barrier
// W and Vr are [m][nb] row-major (Vr holds the panel's reflectors by row, so that a row's
// panel entries are contiguous); p [m]; pr [2][m]; part [grid][2 nb + 1]; sync[0..1] barrier,
// [2] error.  Dynamic shared memory: v [m].
constexpr int kLatrdPanel = 64;
constexpr int kLatrdMin = 1024;     // sizes at which the blocked reduction is used (when
                                    // the rows do not fit in shared memory)
__global__ void __launch_bounds__(512, 2)
k_latrd(double* __restrict__ A, int m, int k0, int b, double* __restrict__ vbuf,
        double* __restrict__ tau, double* __restrict__ d, double* __restrict__ e,
        double* __restrict__ W, double* __restrict__ Vr, double* __restrict__ p,
        double* __restrict__ pr, double* __restrict__ part, unsigned* sync) {
  constexpr int nb = kLatrdPanel;
  extern __shared__ double vs[];                      // v of the current column, by row
  __shared__ double red[32];
  __shared__ double sh[4];
  __shared__ double xy[2 * nb];
  __shared__ double rk[2 * nb];                       // row k+1 of V and W (panel columns)
  int* err = reinterpret_cast<int*>(sync + 2);
  const int G = gridDim.x, bid = blockIdx.x;
  const int warp = (bid * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nw = (G * blockDim.x) >> 5;
  const int wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  for (int j = 0; j < b; ++j) {
    const int k = k0 + j;
    const int n1 = m - k - 1;
    // ---- A: reflector of row k (every block; block 0 stores it)
    {
      const double* x = A + (long)k * m + k + 1;
      double s2 = 0.0;
      for (int i = 1 + threadIdx.x; i < n1; i += blockDim.x) {
        const double xi = __ldcg(x + i);
        s2 = fma(xi, xi, s2);
      }
      s2 = block_sum(s2, red);
      if (threadIdx.x == 0) {
        const double alpha = __ldcg(x);
        double beta, t, scale;
        if (s2 == 0.0) { beta = alpha; t = 0.0; scale = 0.0; }
        else {
          beta = -copysign(sqrt(alpha * alpha + s2), alpha);
          t = (beta - alpha) / beta;
          scale = 1.0 / (alpha - beta);
        }
        sh[0] = t;
        sh[1] = scale;
        if (bid == 0) {
          tau[k] = t;
          d[k] = __ldcg(A + (long)k * m + k);
          e[k] = beta;
        }
      }
      __syncthreads();
      const double scale = sh[1];
      for (int i = threadIdx.x; i < n1; i += blockDim.x) {
        const double vi = (i == 0) ? 1.0 : __ldcg(x + i) * scale;
        vs[k + 1 + i] = vi;
        if (bid == 0) {
          vbuf[(long)k * m + k + 1 + i] = vi;
          Vr[(long)(k + 1 + i) * nb + j] = vi;
        }
      }
      __syncthreads();
    }
    const double t = sh[0];
    const int R = (n1 + G - 1) / G;                   // rows (and row-k+1 columns) owned
    const int r0 = k + 1 + bid * R, r1 = min(m, r0 + R);
    // ---- B: p_raw = A22 v over rows >= k+1 as two half-row items per row (a warp per
    //      item, eight loads in flight per lane; pr holds the halves, [0, m) and [m, 2m));
    //      partials of W^T v, V^T v (columns l < j)
    {
      const int n1h = ((n1 + 1) / 2 + 31) / 32 * 32;
      for (int it = warp; it < 2 * n1; it += nw) {
        const int i = it >> 1, half = it & 1;
        const double* row = A + (long)(k + 1 + i) * m;
        const int qe = half ? m : min(m, k + 1 + n1h);
        double sa[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) sa[u] = 0.0;
        int q = k + 1 + (half ? n1h : 0) + lane;
        for (; q + 7 * 32 < qe; q += 8 * 32) {
          double av[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) av[u] = __ldcg(row + q + 32 * u);
#pragma unroll
          for (int u = 0; u < 8; ++u) sa[u] = fma(av[u], vs[q + 32 * u], sa[u]);
        }
        for (; q < qe; q += 32) sa[0] = fma(__ldcg(row + q), vs[q], sa[0]);
        double sum = ((sa[0] + sa[1]) + (sa[2] + sa[3])) + ((sa[4] + sa[5]) + (sa[6] + sa[7]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
        if (lane == 0) pr[half * m + k + 1 + i] = sum;
      }
    }
    if (threadIdx.x < 2 * j) {
      const int tq = threadIdx.x;
      const double* src = tq < j ? W + tq : Vr + (tq - j);
      double acc = 0.0;
      for (int i = r0; i < r1; ++i) acc = fma(__ldcg(src + (long)i * nb), vs[i], acc);
      part[(long)bid * (2 * nb + 1) + tq] = acc;
    }
    if (!grid_sync_bounded(sync, sync + 1, err)) return;
    // ---- C: p = tau (p_raw - V x - W y), x = W^T v, y = V^T v; partials of p . v
    //      (each x, y entry summed over the blocks' partials by one warp: lanes stride the
    //      blocks, then a fixed shuffle tree)
    for (int q = wib; q < 2 * j; q += wpb) {
      double acc = 0.0;
      for (int g = lane; g < G; g += 32) acc += __ldcg(part + (long)g * (2 * nb + 1) + q);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) xy[q] = acc;
    }
    __syncthreads();
    {
      double sp = 0.0;
      for (int i = r0 + wib; i < r1; i += wpb) {
        double c = 0.0;
        for (int l = lane; l < j; l += 32)
          c = fma(__ldcg(Vr + (long)i * nb + l), xy[l], fma(__ldcg(W + (long)i * nb + l), xy[j + l], c));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        const double pv = t * ((__ldcg(pr + i) + __ldcg(pr + m + i)) - c);
        if (lane == 0) p[i] = pv;
        sp = fma(pv, vs[i], sp);
      }
      sp = block_sum(lane == 0 ? sp : 0.0, red);
      if (threadIdx.x == 0) part[(long)bid * (2 * nb + 1) + 2 * nb] = sp;
    }
    if (!grid_sync_bounded(sync, sync + 1, err)) return;
    // ---- D: alpha = (tau/2) p.v (fixed order over the blocks), W[:, j] = p - alpha v;
    //         the owned columns of row k+1 brought up to date (not after the panel's last
    //         column: the trailing GEMM update takes over there)
    if (wib == 0) {
      double sum = 0.0;
      for (int g = lane; g < G; g += 32) sum += __ldcg(part + (long)g * (2 * nb + 1) + 2 * nb);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) sh[2] = 0.5 * t * sum;
    }
    __syncthreads();
    const double alpha = sh[2];
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x)
      W[(long)i * nb + j] = __ldcg(p + i) - alpha * vs[i];
    if (bid == 0)
      for (int i = threadIdx.x; i <= k; i += blockDim.x) W[(long)i * nb + j] = 0.0;
    if (j + 1 < b) {
      const int k1 = k + 1;
      // row k1 of V and W over l <= j (W[k1][j] formed here; p[k1] is visible)
      for (int l = threadIdx.x; l <= j; l += blockDim.x) {
        rk[l] = (l == j) ? vs[k1] : __ldcg(Vr + (long)k1 * nb + l);
        rk[nb + l] = (l == j) ? __ldcg(p + k1) - alpha * vs[k1] : __ldcg(W + (long)k1 * nb + l);
      }
      __syncthreads();
      for (int i = r0 + wib; i < r1; i += wpb) {
        double c = 0.0;
        for (int l = lane; l < j; l += 32)
          c = fma(rk[l], __ldcg(W + (long)i * nb + l), fma(rk[nb + l], __ldcg(Vr + (long)i * nb + l), c));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) {
          const double wij = __ldcg(p + i) - alpha * vs[i];
          A[(long)k1 * m + i] = __ldcg(A + (long)k1 * m + i) - c - (rk[j] * wij + rk[nb + j] * vs[i]);
        }
      }
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
  double* w = v + m;                               // p of this step (all rows)
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
    // p = tau A v for the owned trailing rows (one warp per row, four partial sums)
    const int lfirst = (k1 - b + G - 1) / G;       // first owned row index >= k+1
    for (int li = lfirst + warp; li < nloc; li += nwarp) {
      const double* row = rows + (long)li * m;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int j = k1 + lane;
      for (; j + 96 < m; j += 128) {
        s0 += row[j] * v[j];
        s1 += row[j + 32] * v[j + 32];
        s2 += row[j + 64] * v[j + 64];
        s3 += row[j + 96] * v[j + 96];
      }
      for (; j < m; j += 32) s0 += row[j] * v[j];
      double s = (s0 + s1) + (s2 + s3);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) pbuf[(long)(k & 1) * m + b + li * G] = t * s;
    }
    if (!grid_sync_bounded(sync, sync + 1, err)) return;
    // g = (tau/2) p.v; with w = p - g v the update A -= v w^T + w v^T reads
    // A_ij -= v_i p_j + (p_i - 2 g v_i) v_j  (two FMAs per element)
    double s = 0.0;
    for (int j = k1 + threadIdx.x; j < m; j += blockDim.x) {
      const double pj = __ldcg(pbuf + (long)(k & 1) * m + j);
      w[j] = pj;
      s += pj * v[j];
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) sh[3] = t * s;             // 2 g
    __syncthreads();
    const double g2 = sh[3];
    // update of the owned rows
    for (int li = lfirst; li < nloc; ++li) {
      const int i = b + li * G;
      const double vi = v[i], bi = fma(-g2, vi, w[i]);
      double* row = rows + (long)li * m;
      for (int j = k1 + threadIdx.x; j < m; j += blockDim.x)
        row[j] = fma(-bi, v[j], fma(-vi, w[j], row[j]));
    }
    // row k+1 after this step (every block, from the copy published before the barrier)
    const double* old = (k == 0) ? A + (long)k1 * m : rowbuf + (long)(k1 & 1) * m;
    {
      const double vi = v[k1], bi = fma(-g2, vi, w[k1]);
      for (int j = k1 + threadIdx.x; j < m; j += blockDim.x)
        r[j] = fma(-bi, v[j], fma(-vi, w[j], __ldcg(old + j)));
    }
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
constexpr size_t kBackSmemMax = 200ull * 1024;      // resident columns of the back-transform
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

// Sturm count in single precision by the ratio recurrence q_i = d_i - x - e_(i-1)^2 / q_(i-1)
// (q raised to -pivmin where it vanishes): the count is exact for a tridiagonal matrix whose
// elements carry relative errors of a few float roundings, so it brackets every eigenvalue
// to within a few 2^-24 tnorm.
__device__ int sturm_f32(const float* __restrict__ d, const float* __restrict__ e2, int m, float x,
                         float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int cnt = q < 0.f ? 1 : 0;
  for (int i = 1; i < m; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += q < 0.f ? 1 : 0;
  }
  return cnt;
}

// j-th smallest eigenvalue by 4-way multisection inside the Gershgorin interval: four
// lanes per eigenvalue evaluate the Sturm count at the three interior quarter points
// (lane 3 idles), so each step removes two bits; stop at an absolute width of tol.
__global__ void k_bisect(const double* __restrict__ dg, const double* __restrict__ e,
                         const double* __restrict__ e2g, int m, double glo, double ghi, double tol,
                         double* __restrict__ w) {
  extern __shared__ double sde[];      // d[m], e2[m] staged per block (and float copies)
  float* sdf = reinterpret_cast<float*>(sde + 2 * m);
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    sde[i] = dg[i];
    sde[m + i] = e2g[i];
    sdf[i] = (float)dg[i];
    sdf[m + i] = (float)e2g[i];
  }
  __syncthreads();
  const double* d = sde;
  const double* e2 = sde + m;
  // eight lanes per eigenvalue: lanes 0..6 count at the seven interior eighth points of
  // the bracket (three bits per pass); one Sturm chain per lane, many warps, so that every
  // SM sub-partition's FP64 unit has work
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = gid >> 3, q = gid & 7;
  const unsigned sh = threadIdx.x & 24;
  const unsigned grp = 0xFFu << sh;
  if ((gid & ~7) >= (m << 3)) return;          // whole group beyond m
  const bool live = j < m;
  double lo = glo, hi = ghi;
  // single-precision phase (the float units run many times the FP64 rate): octasection to
  // a width of 64 float roundings of the norm, then the bracket widened by as much and
  // checked with two FP64 counts (the full interval again if it fails)
  const double span = fmax(fabs(glo), fabs(ghi));
  const double fgap = 64.0 * 0x1p-24 * span;
  if (span > 0.0 && span < 1e30 && ghi - glo > 4.0 * fgap) {
    const float pivmin = (float)fmax(1e-30, 0x1p-24 * 1e-8 * span);
    float flo = (float)glo, fhi = (float)ghi;
    for (int it = 0; it < 40; ++it) {
      if ((double)fhi - (double)flo <= fgap) break;
      const float h = 0.125f * (fhi - flo);
      const float x = flo + h * (float)(q + 1);
      const bool above = live && q < 7 && x > flo && x < fhi &&
                         sturm_f32(sdf, sdf + m, m, x, pivmin) > j;
      const unsigned b = (__ballot_sync(grp, above) >> sh) & 0x7Fu;
      const int first = b ? (__ffs(b) - 1) : 7;
      const float nhi = first < 7 ? flo + h * (float)(first + 1) : fhi;
      const float nlo = first > 0 ? flo + h * (float)first : flo;
      if (!(nhi < fhi || nlo > flo)) break;
      flo = nlo;
      fhi = nhi;
    }
    const double clo = fmax(glo, (double)flo - fgap), chi = fmin(ghi, (double)fhi + fgap);
    // lane 0 checks count(clo) <= j, lane 1 count(chi) > j
    bool good = true;
    if (live && q < 2) {
      const int cnt = sturm_nodiv(d, e2, m, q == 0 ? clo : chi);
      good = q == 0 ? (clo <= glo || cnt <= j) : (chi >= ghi || cnt > j);
    }
    const unsigned bad = (__ballot_sync(grp, !good) >> sh) & 0x3u;
    if (!bad) {
      lo = clo;
      hi = chi;
    }
  }
  for (int it = 0; it < 60; ++it) {
    if (hi - lo <= tol) break;
    const double h = 0.125 * (hi - lo);
    const double x = lo + h * (q + 1);
    const bool above = live && q < 7 && x > lo && x < hi && sturm_nodiv(d, e2, m, x) > j;
    const unsigned b = (__ballot_sync(grp, above) >> sh) & 0x7Fu;
    const int first = b ? (__ffs(b) - 1) : 7;           // first eighth point above j
    const double nhi = first < 7 ? lo + h * (first + 1) : hi;
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
__global__ void k_inviter(const double* __restrict__ dg, const double* __restrict__ eg,
                          const double* __restrict__ w, int m, double tnorm,
                          double* __restrict__ u0, double* __restrict__ u1,
                          double* __restrict__ u2, double* __restrict__ lm,
                          double* __restrict__ pv, double* __restrict__ Z) {
  extern __shared__ double sde[];      // d[m], e[m] staged per block
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    sde[i] = dg[i];
    sde[m + i] = eg[i];
  }
  __syncthreads();
  const double* d = sde;
  const double* e = sde + m;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const double lam = w[j];
  const double tiny = 2.2e-16 * (tnorm > 0 ? tnorm : 1.0);
#define IX(i) ((long)(i) * m + j)
  // Factor T - lam I = P L U (U with two superdiagonals), the current row carried in
  // registers; rows are final once passed, so their pivots are stored as reciprocals
  // (|pivot| raised to tiny) and the solves below multiply.
  auto raise = [&](double piv, double rp) {   // reciprocal of the pivot raised to tiny
    return fabs(piv) < tiny ? 1.0 / copysign(tiny, piv == 0.0 ? 1.0 : piv) : rp;
  };
  double a = d[0] - lam, b = m > 1 ? e[0] : 0.0;
  for (int i = 0; i < m - 1; ++i) {
    const double c = e[i];          // subdiagonal element of row i+1
    const double an = d[i + 1] - lam, bn = (i + 1 < m - 1) ? e[i + 1] : 0.0;
    if (fabs(a) >= fabs(c)) {
      const double piv = (a == 0.0) ? tiny : a;
      const double rp = 1.0 / piv;
      const double l = c * rp;
      u0[IX(i)] = raise(piv, rp);
      u1[IX(i)] = b;
      u2[IX(i)] = 0.0;
      lm[IX(i)] = l;
      pv[IX(i)] = 0.0;
      a = an - l * b;
      b = bn;
    } else {
      const double rp = 1.0 / c;
      const double l = a * rp;
      u0[IX(i)] = raise(c, rp);
      u1[IX(i)] = an;
      u2[IX(i)] = bn;
      lm[IX(i)] = l;
      pv[IX(i)] = 1.0;
      a = b - l * an;
      b = -l * bn;
    }
  }
  {
    const double piv = a == 0.0 ? tiny : a;
    u0[IX(m - 1)] = raise(piv, 1.0 / piv);
  }
  u1[IX(m - 1)] = 0.0;
  u2[IX(m - 1)] = 0.0;
  // three inverse iterations from a fixed start vector; the normalisation of each
  // iterate is folded into the next forward pass.  Both passes go in chunks of eight
  // rows whose operands are loaded before the dependent chain runs through them.
  constexpr int CH = 8;
  double scale = 1.0;
  for (int iter = 0; iter < 3; ++iter) {
    // apply L^-1 with the row interchanges
    double cur = iter == 0 ? hash_unit(0, j) : Z[IX(0)] * scale;
    for (int i0 = 0; i0 < m - 1; i0 += CH) {
      const int cnt = min(CH, m - 1 - i0);
      double yv[CH], lv[CH], pq[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        if (u < cnt) {
          const int i = i0 + u;
          yv[u] = iter == 0 ? hash_unit(i + 1, j) : Z[IX(i + 1)] * scale;
          lv[u] = lm[IX(i)];
          pq[u] = pv[IX(i)];
        }
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        if (u < cnt) {
          double yn = yv[u];
          if (pq[u] != 0.0) {
            const double t = cur; cur = yn; yn = t;
          }
          Z[IX(i0 + u)] = cur;
          cur = yn - lv[u] * cur;
        }
      }
    }
    // U^-1 with overflow guard (x1 = x_{i+1}, x2 = x_{i+2})
    double big = 0.0, nrm = 0.0, x1 = 0.0, x2 = 0.0;
    for (int i0 = m - 1; i0 >= 0; i0 -= CH) {
      const int cnt = min(CH, i0 + 1);
      double zv[CH], a0[CH], a1[CH], a2[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        if (u < cnt) {
          const int i = i0 - u;
          zv[u] = i == m - 1 ? cur : Z[IX(i)];
          a0[u] = u0[IX(i)];
          a1[u] = u1[IX(i)];
          a2[u] = u2[IX(i)];
        }
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        if (u < cnt) {
          const int i = i0 - u;
          double x = zv[u];
          x -= a1[u] * x1;
          x -= a2[u] * x2;
          x *= a0[u];
          Z[IX(i)] = x;
          nrm += x * x;
          x2 = x1;
          x1 = x;
          big = fmax(big, fabs(x));
          if (big > 1e100) {  // rescale the partial solution
            for (int k2 = i; k2 < m; ++k2) Z[IX(k2)] *= 1e-100;
            big *= 1e-100;
            nrm *= 1e-200;
            x1 *= 1e-100;
            x2 *= 1e-100;
          }
        }
      }
    }
    scale = 1.0 / sqrt(nrm);
  }
  for (int i = 0; i < m; ++i) Z[IX(i)] *= scale;
#undef IX
}

// Modified Gram-Schmidt inside each cluster of (numerically) equal eigenvalues.
// One block per eigenvalue index; only cluster starts do work.
// Orthonormalise each cluster of close eigenvalues (w sorted): the block of the cluster's
// first index takes the cluster's columns, in shared memory when they fit (else in place
// in Z), and applies classical Gram-Schmidt twice per vector (each pass projects the
// vector on all earlier cluster vectors at once), then normalises it.
__global__ void __launch_bounds__(256)
k_cluster_cgs2(const double* __restrict__ w, int m, double tol, int smem_bytes,
               double* __restrict__ Z) {
  extern __shared__ double cs[];
  __shared__ double part[8][33];
  __shared__ double red[32];
  __shared__ double sc;
  const int j0 = blockIdx.x;
  if (j0 > 0 && w[j0] - w[j0 - 1] <= tol) return;            // not a start
  if (j0 + 1 >= m || w[j0 + 1] - w[j0] > tol) return;         // singleton
  int j1 = j0 + 1;
  while (j1 + 1 < m && w[j1 + 1] - w[j1] <= tol) ++j1;
  const int c = j1 - j0 + 1;
  const bool in_smem = ((long)m * c + c) * 8 <= smem_bytes;
  double* Zb = in_smem ? cs : Z + j0;          // column q of the cluster: Zb[i * ld + q]
  const long ld = in_smem ? c : m;
  double* pk = in_smem ? cs + (long)m * c : cs;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  if (in_smem) {
    for (long t = threadIdx.x; t < (long)m * c; t += blockDim.x)
      cs[t] = Z[(t / c) * m + j0 + t % c];
    __syncthreads();
  }
  for (int q = 0; q < c; ++q) {
    for (int pass = 0; pass < 2 && q > 0; ++pass) {
      // pk[r] = sum_i Zb[i][r] Zb[i][q] for r < q: lanes over 32 columns, warps over rows
      // (four independent partial sums each), fixed-order sums over the warps
      for (int r0 = 0; r0 < q; r0 += 32) {
        const int r = r0 + lane;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        if (r < q) {
          int i = wp;
          for (; i + 24 < m; i += 32) {
            a0 += Zb[i * ld + r] * Zb[i * ld + q];
            a1 += Zb[(i + 8) * ld + r] * Zb[(i + 8) * ld + q];
            a2 += Zb[(i + 16) * ld + r] * Zb[(i + 16) * ld + q];
            a3 += Zb[(i + 24) * ld + r] * Zb[(i + 24) * ld + q];
          }
          for (; i < m; i += 8) a0 += Zb[i * ld + r] * Zb[i * ld + q];
        }
        part[wp][lane] = (a0 + a1) + (a2 + a3);
        __syncthreads();
        if (wp == 0 && r < q) {
          double t = 0.0;
#pragma unroll
          for (int g = 0; g < 8; ++g) t += part[g][lane];
          pk[r] = t;
        }
        __syncthreads();
      }
      // Zb[i][q] -= sum_r pk[r] Zb[i][r]: one thread per row
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double* zr = Zb + i * ld;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int r = 0;
        for (; r + 3 < q; r += 4) {
          a0 += pk[r] * zr[r];
          a1 += pk[r + 1] * zr[r + 1];
          a2 += pk[r + 2] * zr[r + 2];
          a3 += pk[r + 3] * zr[r + 3];
        }
        for (; r < q; ++r) a0 += pk[r] * zr[r];
        Zb[i * ld + q] -= (a0 + a1) + (a2 + a3);
      }
      __syncthreads();
    }
    double s2 = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s2 += Zb[i * ld + q] * Zb[i * ld + q];
    s2 = block_sum(s2, red);
    if (threadIdx.x == 0) sc = (s2 > 0.0) ? 1.0 / sqrt(s2) : 0.0;
    __syncthreads();
    const double nr = sc;
    for (int i = threadIdx.x; i < m; i += blockDim.x) Zb[i * ld + q] *= nr;
    __syncthreads();
  }
  if (in_smem)
    for (long t = threadIdx.x; t < (long)m * c; t += blockDim.x)
      Z[(t / c) * m + j0 + t % c] = cs[t];
}

// G[i][i] -= x
__global__ void k_sub_diag(double* __restrict__ G, int m, double x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) G[(long)i * m + i] -= x;
}

// G = 1.5 I - 0.5 G (in place)
// and dev = max |G - I| (order-independent integer maximum of the bit patterns)
__global__ void k_ns_coef(double* __restrict__ G, int m, unsigned long long* __restrict__ dev) {
  const long total = (long)m * m;
  unsigned long long mx = 0;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total;
       t += (long)gridDim.x * blockDim.x) {
    const bool diag = t / m == t % m;
    const double g = G[t];
    const unsigned long long b =
        (unsigned long long)__double_as_longlong(g - (diag ? 1.0 : 0.0)) & 0x7FFFFFFFFFFFFFFFull;
    mx = b > mx ? b : mx;
    G[t] = (diag ? 1.5 : 0.0) - 0.5 * g;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(dev, mx);
}

// Orthonormality probe of the eigenvector matrix Z (columns): with two fixed +-1 vectors
// r1, r2, dev = max_k |(Z^T Z r)_k - r_k| over both (two passes over Z instead of the m^3
// Gram product).  A column set orthonormal to within e gives dev <~ e sqrt(m); a larger
// dev sends the caller to the full Gram matrix.
__device__ __forceinline__ double probe_sign(int k, int which) {
  const unsigned h = (unsigned)k * 2654435761u + (which ? 0x9E3779B9u : 0x7F4A7C15u);
  return ((h >> 13) & 1u) ? 1.0 : -1.0;
}
// u[q][i] = sum_k Z[i][k] r_q[k]: a warp per row
__global__ void __launch_bounds__(256)
k_ortho_probe1(const double* __restrict__ Z, int m, double* __restrict__ u) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = warp; i < m; i += nw) {
    const double* row = Z + (long)i * m;
    double s1 = 0.0, s2 = 0.0;
    for (int k = lane; k < m; k += 32) {
      const double z = row[k];
      s1 = fma(z, probe_sign(k, 0), s1);
      s2 = fma(z, probe_sign(k, 1), s2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_down_sync(0xffffffffu, s1, o);
      s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
      u[i] = s1;
      u[m + i] = s2;
    }
  }
}
// w_q[c] = sum_i Z[i][c] u_q[i] (32 columns x 8 row groups per block, fixed-order sum over
// the groups) and dev = max |w_q[c] - r_q[c]| (integer maximum of the bit patterns)
__global__ void __launch_bounds__(256)
k_ortho_probe2(const double* __restrict__ Z, int m, const double* __restrict__ u,
               unsigned long long* __restrict__ dev) {
  __shared__ double part[2][8][33];
  const int cx = threadIdx.x & 31, rg = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + cx;
  double s1 = 0.0, s2 = 0.0;
  if (c < m)
    for (int i = rg; i < m; i += 8) {
      const double z = Z[(long)i * m + c];
      s1 = fma(z, u[i], s1);
      s2 = fma(z, u[m + i], s2);
    }
  part[0][rg][cx] = s1;
  part[1][rg][cx] = s2;
  __syncthreads();
  if (rg == 0 && c < m) {
    double w1 = 0.0, w2 = 0.0;
    for (int g = 0; g < 8; ++g) {
      w1 += part[0][g][cx];
      w2 += part[1][g][cx];
    }
    const double e = fmax(fabs(w1 - probe_sign(c, 0)), fabs(w2 - probe_sign(c, 1)));
    const unsigned long long b = (unsigned long long)__double_as_longlong(e);
    if (e == e) atomicMax(dev, b);
    else atomicMax(dev, 0x7FF8000000000000ull);
  }
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

// Same back-transformation with the block's cb columns of Z resident in shared memory
// (column-major, zs[c][i]) for the whole reflector loop and one warp per column: the warp
// forms v . z_c with a shuffle reduction and updates its column, so the block synchronises
// once per reflector, when the next reflector (double-buffered in shared memory by
// 8-byte cp.async copies) has landed.  Z is read and written once.
__global__ void __launch_bounds__(512)
k_backtransform_smem(const double* __restrict__ vbuf, const double* __restrict__ tau, int m,
                     int cb, double* __restrict__ Z) {
  extern __shared__ double zs[];                 // zs[cb][m], then vs[2][m]
  double* vs = zs + (long)cb * m;
  const int c0 = blockIdx.x * cb;
  const int ncol = min(cb, m - c0);
  const int lane = threadIdx.x & 31, wc = threadIdx.x >> 5;
  const int nth = blockDim.x;
  for (long q = threadIdx.x; q < (long)m * cb; q += nth) {
    const int i = q / cb, c = q % cb;            // row-major walk of Z (coalesced per row)
    zs[(long)c * m + i] = c < ncol ? Z[(long)i * m + c0 + c] : 0.0;
  }
  auto prefetch = [&](int k) {                   // v_k -> vs[k & 1]
    const int n1 = m - k - 1;
    const double* v = vbuf + (long)k * m + k + 1;
    double* dst = vs + (long)(k & 1) * m;
    for (int i = threadIdx.x; i < n1; i += nth) {
      const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + i);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(v + i) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  if (m >= 3) prefetch(m - 3);
  const bool act = wc < ncol;
  double* zc = zs + (long)wc * m;
  for (int k = m - 3; k >= 0; --k) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();                             // v_k visible; step k+1 done with vs[(k+1)&1]
    if (k > 0) prefetch(k - 1);
    if (!act) continue;
    const int n1 = m - k - 1;
    const double* v = vs + (long)(k & 1) * m;
    double* z = zc + k + 1;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = lane;
    for (; i + 96 < n1; i += 128) {
      s0 += v[i] * z[i];
      s1 += v[i + 32] * z[i + 32];
      s2 += v[i + 64] * z[i + 64];
      s3 += v[i + 96] * z[i + 96];
    }
    for (; i < n1; i += 32) s0 += v[i] * z[i];
    double sum = (s0 + s1) + (s2 + s3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    const double r = sum * tau[k];
    for (int i2 = lane; i2 < n1; i2 += 32) z[i2] -= v[i2] * r;
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  for (long q = threadIdx.x; q < (long)m * cb; q += nth) {
    const int i = q / cb, c = q % cb;
    if (c < ncol) Z[(long)i * m + c0 + c] = zs[(long)c * m + i];
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

// Compact WY form of a panel of reflectors (Schreiber and Van Loan): H_k0 ... H_k0+b-1 =
// I - Vp T Vp^T with T upper triangular, T_ii = tau_i and
// T_{j,i} = -tau_i sum_{l = j..i-1} T_{j,l} (v_l . v_i) (j < i).  One block of b threads;
// Gp[l][i] = v_{k0+l} . v_{k0+i}.
__global__ void k_wy_T(const double* __restrict__ Gp, const double* __restrict__ tau, int k0,
                       int b, double* __restrict__ T) {
  const int j = threadIdx.x;
  for (int i = 0; i < b; ++i) {
    double acc = 0.0;
    if (j < i)
      for (int l = j; l < i; ++l) acc = fma(T[j * b + l], Gp[l * b + i], acc);
    __syncthreads();
    if (j < i) T[j * b + i] = -tau[k0 + i] * acc;
    else if (j == i) T[j * b + i] = tau[k0 + i];
    else if (j < b) T[j * b + i] = 0.0;
    __syncthreads();
  }
}

size_t sym_eig_tridiag_work(int m) { return (size_t)m * m * 9 + (size_t)m * 8 + 64; }

namespace {
constexpr int kWyPanel = 128;       // reflectors per compact-WY panel
constexpr int kWyMinSize = 1024;    // blocked back-transformation from this size up

// V <- H_0 H_1 ... H_{m-3} V as panels P_j = I - Vp T Vp^T applied last panel first:
// W = Vp^T V (rows below the panel start), W <- T W, V -= Vp W, three FP64 GEMMs per
// panel.  vbuf rows hold the reflectors with zeros left of their first entry, so a panel's
// rows of vbuf are Vp^T as it stands.  scratch >= 2 b m + 2 b^2 + part doubles.
int backtransform_wy(const double* vbuf, const double* tau, int m, double* V, double* scratch,
                     long scratch_size, cudaStream_t s, OzWork* oz) {
  const int nref = m - 2;
  const int nb = kWyPanel;
  double* W = scratch;
  double* W2 = W + (long)nb * m;
  double* Gp = W2 + (long)nb * m;
  double* T = Gp + (long)nb * nb;
  double* part = T + (long)nb * nb;
  const long partmax = scratch_size - (part - scratch);
  if (partmax < (long)nb * nb) return CASPT2_EINVAL;
  for (int k0 = ((nref - 1) / nb) * nb; k0 >= 0; k0 -= nb) {
    const int b = std::min(nb, nref - k0);
    const int r = m - k0 - 1;                            // rows k0+1 .. m-1
    const double* Vt = vbuf + (long)k0 * m;              // b x m, zeros left of each v
    int st = gram_product(Vt, Vt, 1, b, m, 0, Gp, b, 0, part, partmax, s, nullptr);
    if (st != CASPT2_OK) return st;
    ++launch_counter();
    k_wy_T<<<1, b, 0, s>>>(Gp, tau, k0, b, T);
    CASPT2_CUDA_TRY(cudaGetLastError());
    if (oz && oz->on) {
      // precision form: the two large products as FP64-accurate split products (the
      // eigenvalues are fixed before this step; only the vectors pass through it)
      const OzView va{Vt + k0 + 1, m, 1, r, 0};                  // rows l, K = row i
      const OzView vb{V + (long)(k0 + 1) * m, 1, m, r, 0};       // rows col, K = row i
      CASPT2_CUDA_TRY(oz_matmul(*oz, va, vb, false, b, m, r, 1.0, 0.0, W, m, s));
      CASPT2_CUDA_TRY(dgemm(b, m, b, 1.0, T, b, false, W, m, false, 0.0, W2, m, s));
      const OzView vp{Vt + k0 + 1, 1, m, b, 0};                  // rows i, K = l
      const OzView vw{W2, 1, m, b, 0};                           // rows col, K = l
      CASPT2_CUDA_TRY(oz_matmul(*oz, vp, vw, false, r, m, b, -1.0, 1.0, V + (long)(k0 + 1) * m,
                                m, s));
    } else {
      CASPT2_CUDA_TRY(dgemm(b, m, r, 1.0, Vt + k0 + 1, m, false, V + (long)(k0 + 1) * m, m,
                            false, 0.0, W, m, s));
      CASPT2_CUDA_TRY(dgemm(b, m, b, 1.0, T, b, false, W, m, false, 0.0, W2, m, s));
      CASPT2_CUDA_TRY(dgemm(r, m, b, -1.0, Vt + k0 + 1, m, true, W2, m, false, 1.0,
                            V + (long)(k0 + 1) * m, m, s));
    }
  }
  return CASPT2_OK;
}
}  // namespace

int sym_eig_tridiag(double* A, int m, double* w, double* V, double* work, cudaStream_t s,
                    KernelTimer* tm, OzWork* oz) {
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
  // reflector rows are read whole by the blocked back-transformation: zero them first
  if (m >= kWyMinSize) CASPT2_CUDA_TRY(cudaMemsetAsync(vbuf, 0, sizeof(double) * mm, s));
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
      // the matrix read once and the reflectors (lower triangle) written once
      tm->bytes += 8.0 * m * m + 4.0 * m * (m - 1.0);
      ++tm->launches;
    }
  } else if (m > 64 && m >= kLatrdMin) {
    // blocked reduction: panels of kLatrdPanel columns (one cooperative launch each) and
    // the trailing update as two FP64 GEMMs per panel
    unsigned* sync = reinterpret_cast<unsigned*>(r);   // r is free until the back-transform
    double* Wp = u0;                                   // [m][kLatrdPanel]
    double* pp = u1;
    double* pr = u1 + m;                               // [2][m] (the two row halves)
    double* part = u1 + 3 * (long)m;                   // [grid][2 panel + 1]
    double* Vr = u2;                                   // [m][kLatrdPanel]
    if (sizeof(double) * (size_t)m > kBisectSmemMax) return CASPT2_EINVAL;
    CASPT2_CUDA_TRY(cudaFuncSetAttribute(k_latrd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kBisectSmemMax));
    int per = 0;
    CASPT2_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_latrd, 512,
                                                                  sizeof(double) * (size_t)m));
    // two blocks per SM when they fit (more warps in flight for the latency-bound
    // matrix-vector products), one otherwise
    const int grid = std::max(1, nsm * std::max(1, std::min(per, 2)));
    if ((long)grid * (2 * kLatrdPanel + 1) > mm - 3 * (long)m) return CASPT2_EINVAL;
    CASPT2_CUDA_TRY(cudaMemsetAsync(sync, 0, 4 * sizeof(unsigned), s));
    const int npanel = (m - 2 + kLatrdPanel - 1) / kLatrdPanel;
    if (tm && tm->e0) {
      while ((int)tm->pev.size() < 2 * npanel) {
        cudaEvent_t ev = nullptr;
        CASPT2_CUDA_TRY(cudaEventCreate(&ev));
        tm->pev.push_back(ev);
      }
      CASPT2_CUDA_TRY(cudaEventRecord(tm->e0, s));
    }
    std::vector<double> pbytes;
    for (int k0 = 0; k0 < m - 2; k0 += kLatrdPanel) {
      const int b = std::min(kLatrdPanel, m - 2 - k0);
      void* args[] = {&A, (void*)&m, (void*)&k0, (void*)&b, &vbuf, &tau, &d, &e, &Wp, &Vr, &pp,
                      &pr, &part, &sync};
      const int pi = k0 / kLatrdPanel;
      if (tm && tm->e0) {
        CASPT2_CUDA_TRY(cudaEventRecord(tm->pev[2 * pi], s));
        double by = 0.0;
        for (int j = 0; j < b; ++j) {
          const double n1 = (double)(m - k0 - j - 1);
          by += 8.0 * n1 * n1;
        }
        pbytes.push_back(by);
      }
      ++launch_counter();
      CASPT2_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_latrd, grid, 512, args,
                                                  sizeof(double) * (size_t)m, s));
      if (tm && tm->e0) CASPT2_CUDA_TRY(cudaEventRecord(tm->pev[2 * pi + 1], s));
      const int rr = m - k0 - b;
      if (rr > 0) {
        double* A22 = A + (long)(k0 + b) * m + k0 + b;
        const double* Vp = vbuf + (long)k0 * m + k0 + b;
        const double* Wr = Wp + (long)(k0 + b) * kLatrdPanel;
        CASPT2_CUDA_TRY(dgemm(rr, rr, b, -1.0, Vp, m, true, Wr, kLatrdPanel, true, 1.0, A22, m, s));
        CASPT2_CUDA_TRY(dgemm(rr, rr, b, -1.0, Wr, kLatrdPanel, false, Vp, m, false, 1.0, A22, m,
                              s));
      }
    }
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
      tm->bytes += 8.0 * m * m + 4.0 * m * (m - 1.0);
      for (size_t q = 0; q < pbytes.size(); ++q) {
        float pm = 0.f;
        CASPT2_CUDA_TRY(cudaEventElapsedTime(&pm, tm->pev[2 * q], tm->pev[2 * q + 1]));
        tm->pms += pm;
        tm->pbytes += pbytes[q];
        ++tm->plaunches;
      }
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
      // the matrix read once and the reflectors (lower triangle) written once
      tm->bytes += 8.0 * m * m + 4.0 * m * (m - 1.0);
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
  if (3 * sizeof(double) * (size_t)m > kBisectSmemMax) return CASPT2_EINVAL;
  CASPT2_CUDA_TRY(cudaFuncSetAttribute(k_bisect, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kBisectSmemMax));
  // blocks sized so that one wave covers all 8m lanes (the staged copy of the tridiagonal
  // matrix limits residency to one block per SM at the largest sizes)
  const int bis_t = (int)std::min<long>(1024, std::max<long>(32, ((8L * m + nsm - 1) / nsm + 31) / 32 * 32));
  k_bisect<<<(unsigned)((8L * m + bis_t - 1) / bis_t), bis_t, 3 * sizeof(double) * m, s>>>(
      d, e, e2, m, glo, ghi, 4.0 * 2.2e-16 * std::max(1.0, tnorm), w);
  // 3. eigenvectors of T
  ++launch_counter();
  // one warp per block so that the m independent LU chains spread over the SMs
  CASPT2_CUDA_TRY(cudaFuncSetAttribute(k_inviter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kBisectSmemMax));
  k_inviter<<<(m + 31) / 32, 32, 2 * sizeof(double) * m, s>>>(d, e, w, m, tnorm, u0, u1, u2, lm,
                                                               pv, Z);
  ++launch_counter();
  CASPT2_CUDA_TRY(cudaFuncSetAttribute(k_cluster_cgs2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kBisectSmemMax));
  {
    const int cbytes = (int)std::min<size_t>(kBisectSmemMax, 8ull * ((size_t)m * m + m));
    k_cluster_cgs2<<<m, 256, cbytes, s>>>(w, m, 1e-12 * std::max(1.0, tnorm), cbytes, Z);
  }
  CASPT2_CUDA_TRY(cudaGetLastError());
  // 4. Newton-Schulz: Z <- Z (1.5 I - 0.5 Z^T Z), skipped when Z is already orthonormal to
  //    1e-13 (the step would change it by less than that)
  //    The probe Z^T Z r (two passes over Z) decides first; only when it is above 1e-13 is
  //    the m^3 Gram matrix formed and the element-wise test applied.
  unsigned long long* ns_dev = reinterpret_cast<unsigned long long*>(r + m);
  CASPT2_CUDA_TRY(cudaMemsetAsync(ns_dev, 0, sizeof(unsigned long long), s));
  ++launch_counter();
  k_ortho_probe1<<<nblocks(32L * m), kT, 0, s>>>(Z, m, G);
  ++launch_counter();
  k_ortho_probe2<<<(m + 31) / 32, 256, 0, s>>>(Z, m, G, ns_dev);
  CASPT2_CUDA_TRY(cudaGetLastError());
  unsigned long long hdev = 0;
  CASPT2_CUDA_TRY(cudaMemcpyAsync(&hdev, ns_dev, sizeof(hdev), cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
  double dev_probe;
  std::memcpy(&dev_probe, &hdev, sizeof(double));
  if (!(dev_probe == dev_probe)) return CASPT2_ENAN;
  if (dev_probe <= 1e-13) {
    CASPT2_CUDA_TRY(cudaMemcpyAsync(V, Z, sizeof(double) * mm, cudaMemcpyDeviceToDevice, s));
  } else {
    CASPT2_CUDA_TRY(cudaMemsetAsync(ns_dev, 0, sizeof(unsigned long long), s));
    CASPT2_CUDA_TRY(dgemm_sym(m, m, 1.0, Z, m, true, Z, m, false, 0.0, G, m, s));
    ++launch_counter();
    k_ns_coef<<<nblocks(mm), kT, 0, s>>>(G, m, ns_dev);
    CASPT2_CUDA_TRY(cudaGetLastError());
    CASPT2_CUDA_TRY(cudaMemcpyAsync(&hdev, ns_dev, sizeof(hdev), cudaMemcpyDeviceToHost, s));
    CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
    double dev_ortho;
    std::memcpy(&dev_ortho, &hdev, sizeof(double));
    if (!(dev_ortho == dev_ortho)) return CASPT2_ENAN;
    if (dev_ortho <= 1e-13) {
      CASPT2_CUDA_TRY(cudaMemcpyAsync(V, Z, sizeof(double) * mm, cudaMemcpyDeviceToDevice, s));
    } else if (oz && oz->on) {
      // V = Z + Z Ec, Ec = (1/2)(I - Z^T Z) (G - I): the correction is of the size of the
      // orthogonality error, so a split product with S slices (error below about
      // 2^(1-7S) m max|Z| max|Ec|) is kept under 1e-17 with S = ceil((57 + log2(m dev/2)) / 7)
      ++launch_counter();
      k_sub_diag<<<(m + 255) / 256, 256, 0, s>>>(G, m, 1.0);
      CASPT2_CUDA_TRY(cudaGetLastError());
      CASPT2_CUDA_TRY(cudaMemcpyAsync(V, Z, sizeof(double) * mm, cudaMemcpyDeviceToDevice, s));
      const double lg = std::log2(std::max(1e-300, 0.5 * (double)m * dev_ortho));
      const int S = std::max(2, std::min(kOzMaxSlices, (int)std::ceil((57.0 + lg) / 7.0)));
      const int S0 = oz->S;
      oz->S = S;
      const OzView vz{Z, m, 1, m, 0}, vg{G, m, 1, m, 0};   // G symmetric: B(j, k) = G[j][k]
      const cudaError_t e = oz_matmul(*oz, vz, vg, false, m, m, m, 1.0, 1.0, V, m, s);
      oz->S = S0;
      CASPT2_CUDA_TRY(e);
    } else {
      CASPT2_CUDA_TRY(dgemm(m, m, m, 1.0, Z, m, false, G, m, false, 0.0, V, m, s));
    }
  }
  // 5. back-transformation V = H_0 ... H_{m-3} Z: blocked (compact WY panels as FP64
  //    GEMMs) for large matrices, else column-owned in one launch.  Z, G and the
  //    inverse-iteration scratch are free here.
  if (m >= kWyMinSize) {
    const int st = backtransform_wy(vbuf, tau, m, V, Z, 7 * mm, s, oz);
    if (st != CASPT2_OK) return st;
  } else if (m >= 3) {
    ++launch_counter();
    // columns resident in shared memory: ceil(m / SMs) per block (one block per SM, the
    // FP64 work spread evenly, one warp per column), fewer per block when they do not fit
    const long fit = (long)(kBackSmemMax / (8ull * m)) - 2;      // minus the v buffers
    const int cbs = (int)std::min<long>(std::min<long>(16, (m + nsm - 1) / nsm), fit);
    if (cbs >= 1) {
      CASPT2_CUDA_TRY(cudaFuncSetAttribute(k_backtransform_smem,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kBackSmemMax));
      k_backtransform_smem<<<(m + cbs - 1) / cbs, 32 * cbs, sizeof(double) * (size_t)m * (cbs + 2),
                             s>>>(vbuf, tau, m, cbs, V);
    } else {
      const int cb = 8;     // 8 columns x 32 row groups per block
      k_backtransform<<<(m + cb - 1) / cb, 256, 0, s>>>(vbuf, tau, m, cb, V);
    }
  }
  CASPT2_CUDA_TRY(cudaGetLastError());
  return CASPT2_OK;
}

}  // namespace caspt2
