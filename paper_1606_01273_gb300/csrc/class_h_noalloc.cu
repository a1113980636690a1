// Class-H energy pieces through an entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running inside another framework's
// memory pool or a pre-sized arena, plugins loaded into a host that forbids
// allocations after start-up, and latency-critical loops that must never hit the
// allocator's synchronisation.  caspt2_classH_noalloc serves them: the caller
// passes device inputs and device outputs, and every intermediate lives in one
// fixed file-scope device array, g_scratch, of kScratchBytes (4 MiB).  Every GPU
// that loads this library holds that array until the process exits.
//
// In host code, g_scratch names a host-side stand-in, not the device array, so
// its device address is looked up once per device with cudaGetSymbolAddress (the
// first call on each device does this, with that device current) and passed to
// the kernels.  That first call should therefore be made before any stream
// capture begins.  All calls share the array and it keeps the previous call's
// contents: the values that must start from a known state (the smallest
// denominator and the status word) are reset on every call, and everything else
// is fully overwritten before it is read.  Calls whose work overlaps on the GPU
// (other threads, other streams) race on the array and must be serialised by the
// caller.
//
// The kernel is a persistent-grid variant of the direct class-H kernel: it reads
// the DF factors in place (no packed copy) and each CTA keeps its running sums in
// shared memory, so the scratch needed is bounded by the grid size rather than by
// the problem size.
#include <mutex>
#include <vector>

#include "kernels.cuh"

namespace caspt2 {
namespace {

constexpr size_t kScratchBytes = CASPT2_NOALLOC_SCRATCH_BYTES;
constexpr size_t kScratchDoubles = kScratchBytes / sizeof(double);
constexpr int kMaxDevices = 64;
constexpr int kNaGrid = 152 * 4;     // persistent CTAs (4 per SM)
constexpr int kNaT = 64, kNaK = 16, kNaThreads = 256;
constexpr int kNaMaxShift = kMaxStates * kMaxStates;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

std::mutex g_scratch_mu;
double* g_scratch_dev[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CASPT2_ECUDA;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return CASPT2_ECUDA;
    g_scratch_dev[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_dev[dev];
  return CASPT2_OK;
}

struct Layout {  // offsets (in doubles) into the scratch array
  size_t fref, U, Etil, Ftil, E0, W, omega, shifts, sums, mindenom, status, eps, partial, total;
};

Layout layout(const Dims& d, int nshift, int grid) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t n) { size_t r = o; o += (n + 31) & ~size_t(31); return r; };  // 256 B
  const size_t n2 = (size_t)d.n * d.n;
  L.fref = take(n2); L.U = take(n2); L.Etil = take(d.n); L.Ftil = take(n2); L.E0 = take(d.n);
  L.W = take(n2); L.omega = take(d.n); L.shifts = take(nshift);
  L.sums = take(2 * nshift + 1); L.mindenom = take(1); L.status = take(1);
  L.eps = take((size_t)d.c + d.v);
  L.partial = take((size_t)grid * (2 * nshift + 1));
  L.total = o;
  return L;
}

// Pair index p -> (x, y), x <= y < R, enumerated row-major by x (64-bit, closed form
// with an exact integer correction).
__device__ __forceinline__ void tri_pair(long p, int R, int& x, int& y) {
  const double b = 2.0 * R + 1.0;
  long xx = (long)floor(0.5 * (b - sqrt(fmax(b * b - 8.0 * (double)p, 0.0))));
  if (xx < 0) xx = 0;
  if (xx > R - 1) xx = R - 1;
  auto start = [&](long q) { return q * R - q * (q - 1) / 2; };
  while (xx > 0 && start(xx) > p) --xx;
  while (xx + 1 < R && start(xx + 1) <= p) ++xx;
  x = (int)xx;
  y = (int)(p - start(xx) + xx);
}

__global__ void k_na_prepare(const double* __restrict__ f, int nmo, int c, int a, int v,
                             double* eps, double* mindenom, int* status) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < c) eps[x] = f[(long)x * nmo + x];
  else if (x < c + v) eps[x] = f[(long)(x + a) * nmo + x + a];
  if (x == 0) { *mindenom = 1e300; *status = 0; }
}

__global__ void k_na_shifts(const double* __restrict__ omega, const double* __restrict__ E0,
                            double shift, int n, int scheme, double* shifts) {
  int k = threadIdx.x;
  if (scheme == CASPT2_SSSR) {
    if (k == 0) shifts[0] = shift;
    return;
  }
  if (k < n * n) shifts[k] = omega[k / n] - E0[k % n] + shift;
}

// Persistent variant: CTA b handles tiles b, b + grid, ...; the DF factors are
// read in place, B[P][i][vo + a].
__global__ void __launch_bounds__(kNaThreads)
k_na_classH(const double* __restrict__ B, const double* __restrict__ eps,
            const double* __restrict__ shifts, int nshift, int c, int v, int X, int nmo,
            int vo, int ntile, long ntask, double* __restrict__ partial) {
  __shared__ double sAi[kNaK][kNaT], sBj[kNaK][kNaT], sAj[kNaK][kNaT], sBi[kNaK][kNaT];
  __shared__ double sEa[kNaT], sEb[kNaT];
  __shared__ double sShift[kNaMaxShift];
  __shared__ double sAcc[2 * kNaMaxShift + 1];
  __shared__ double red[32];
  const int ncol = 2 * nshift + 1;
  for (int k = threadIdx.x; k < nshift; k += kNaThreads) sShift[k] = shifts[k];
  for (int k = threadIdx.x; k < ncol; k += kNaThreads) sAcc[k] = (k == ncol - 1) ? 1e300 : 0.0;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const long strideP = (long)nmo * nmo;

  const long ntp = (long)ntile * (ntile + 1) / 2;   // tile pairs ta <= tb
  for (long task = blockIdx.x; task < ntask; task += gridDim.x) {
    int ta, tb, i, j;
    tri_pair(task % ntp, ntile, ta, tb);
    tri_pair(task / ntp, c, i, j);
    const bool same = (i == j);
    // (a, b) and (b, a) give equal terms (K(a,b) of the pair ij is K'(b,a)), so a
    // tile pair ta < tb stands for both orders
    const double wt = (ta == tb) ? 1.0 : 2.0;
    const int a0 = ta * kNaT, b0 = tb * kNaT;
    const double* bi = B + (long)i * nmo + vo;
    const double* bj = B + (long)j * nmo + vo;
    __syncthreads();
    for (int k = threadIdx.x; k < kNaT; k += kNaThreads) {
      sEa[k] = (a0 + k < v) ? eps[c + a0 + k] : 0.0;
      sEb[k] = (b0 + k < v) ? eps[c + b0 + k] : 0.0;
    }
    double t1[4][4], t2[4][4];
#pragma unroll
    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) t1[ii][jj] = t2[ii][jj] = 0.0;
    for (int P0 = 0; P0 < X; P0 += kNaK) {
      __syncthreads();
      for (int l = threadIdx.x; l < kNaK * kNaT; l += kNaThreads) {
        const int kk = l / kNaT, col = l % kNaT;
        const int P = P0 + kk;
        const bool okP = P < X;
        const int a = a0 + col, b = b0 + col;
        sAi[kk][col] = (okP && a < v) ? bi[P * strideP + a] : 0.0;
        sBj[kk][col] = (okP && b < v) ? bj[P * strideP + b] : 0.0;
        if (!same) {
          sAj[kk][col] = (okP && a < v) ? bj[P * strideP + a] : 0.0;
          sBi[kk][col] = (okP && b < v) ? bi[P * strideP + b] : 0.0;
        }
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < kNaK; ++kk) {
        double ra[4], rb[4];
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) ra[ii] = sAi[kk][ty + 16 * ii];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) rb[jj] = sBj[kk][tx + 16 * jj];
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) t1[ii][jj] = fma(ra[ii], rb[jj], t1[ii][jj]);
        if (!same) {
#pragma unroll
          for (int ii = 0; ii < 4; ++ii) ra[ii] = sAj[kk][ty + 16 * ii];
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) rb[jj] = sBi[kk][tx + 16 * jj];
#pragma unroll
          for (int ii = 0; ii < 4; ++ii)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) t2[ii][jj] = fma(ra[ii], rb[jj], t2[ii][jj]);
        }
      }
    }
    const double ei = eps[i], ej = eps[j];
    double num[16], d0[16];
#pragma unroll
    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int la = ty + 16 * ii, lb = tx + 16 * jj;
        const bool ok = (a0 + la < v) && (b0 + lb < v);
        const double k1 = t1[ii][jj];
        const double k2 = same ? k1 : t2[ii][jj];
        double nm = k1 * (2.0 * k1 - k2);
        if (!same) nm += k2 * (2.0 * k2 - k1);
        num[ii * 4 + jj] = ok ? wt * nm : 0.0;
        d0[ii * 4 + jj] = ok ? (sEa[la] + sEb[lb] - ei - ej) : 1.0;
      }
    double dmin = 1e300;
    for (int k = 0; k < nshift; ++k) {
      const double sh = sShift[k];
      double e = 0.0, nr = 0.0;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const double inv = 1.0 / (d0[q] + sh);
        e = fma(num[q], inv, e);
        nr = fma(num[q] * inv, inv, nr);
        if (num[q] != 0.0) dmin = fmin(dmin, fabs(d0[q] + sh));
      }
      e = block_sum(e, red);
      if (threadIdx.x == 0) sAcc[k] += e;
      nr = block_sum(nr, red);
      if (threadIdx.x == 0) sAcc[nshift + k] += nr;
    }
    dmin = block_min(dmin, red);
    if (threadIdx.x == 0) sAcc[ncol - 1] = fmin(sAcc[ncol - 1], dmin);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < ncol; k += kNaThreads) partial[(long)blockIdx.x * ncol + k] = sAcc[k];
}

__global__ void k_na_reduce(const double* __restrict__ partial, int nblocks, int ncol,
                            double* __restrict__ sums) {
  __shared__ double red[32];
  const int col = blockIdx.x;
  const bool is_min = (col == ncol - 1);
  double acc = is_min ? 1e300 : 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
    double x = partial[(long)b * ncol + col];
    acc = is_min ? fmin(acc, x) : acc + x;
  }
  acc = is_min ? block_min(acc, red) : block_sum(acc, red);
  if (threadIdx.x == 0) sums[col] = acc;
}

__global__ void k_na_combine(const double* __restrict__ sums, const double* __restrict__ W,
                             int n, int scheme, double* e_out, double* n_out, double* mindenom,
                             int* status) {
  const int idx = threadIdx.x;
  const int nshift = (scheme == CASPT2_SSSR) ? 1 : n * n;
  if (idx < n * n) {
    const int L = idx / n, Lp = idx % n;
    double e = 0.0;
    if (scheme == CASPT2_SSSR) {
      e = (L == Lp) ? -sums[0] : 0.0;
    } else {
      for (int nu = 0; nu < n; ++nu) e -= W[L * n + nu] * W[Lp * n + nu] * sums[nu * n + L];
    }
    if (e_out) e_out[idx] = e;
  }
  if (idx < n && n_out) {
    double nr = 0.0;
    if (scheme == CASPT2_SSSR) {
      nr = sums[nshift];
    } else {
      for (int nu = 0; nu < n; ++nu) nr += W[idx * n + nu] * W[idx * n + nu] * sums[nshift + nu * n + idx];
    }
    n_out[idx] = nr;
  }
  if (idx == 0) {
    const double dm = sums[2 * nshift];
    *mindenom = dm;
    if (!(dm == dm)) atomicExch(status, CASPT2_ENAN);
  }
}

}  // namespace
}  // namespace caspt2

using namespace caspt2;

extern "C" int caspt2_classH_noalloc(const caspt2_dims* dims, const caspt2_options* opt,
                                     const double* fock, const double* dfB, const double* rdm1,
                                     double* e, double* norm, void* cuda_stream) {
  if (!dims || !opt) return CASPT2_EINVAL;
  const Dims d{dims->nclosed, dims->nact, dims->nvirt, dims->naux, dims->nstate};
  if (d.c < 0 || d.a < 0 || d.v < 0 || d.X <= 0 || d.n <= 0 || d.n > kMaxStates)
    return CASPT2_EINVAL;
  if (opt->scheme != CASPT2_MSMR && opt->scheme != CASPT2_SSSR) return CASPT2_EINVAL;
  if (!(opt->shift >= 0.0)) return CASPT2_EINVAL;
  const int nshift = classH_nshift(d, opt->scheme);
  const Layout L = layout(d, nshift, kNaGrid);
  if (L.total > kScratchDoubles) return CASPT2_ESCRATCH;
  if (!fock || !dfB || !e || !norm || (d.a > 0 && !rdm1)) return CASPT2_EINVAL;

  double* s0 = nullptr;
  int st = scratch_address(&s0);
  if (st != CASPT2_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int n = d.n, nmo = d.nmo();
  int* status = reinterpret_cast<int*>(s0 + L.status);
  {
    // the class-H pieces use only the diagonal of f's closed and virtual blocks and its
    // active block: refuse an f with inter-class coupling (host copy, no device memory)
    std::vector<double> hf((size_t)nmo * nmo);
    CASPT2_CUDA_TRY(cudaMemcpyAsync(hf.data(), fock, sizeof(double) * hf.size(),
                                    cudaMemcpyDeviceToHost, s));
    CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
    st = check_block_diagonal_fock(hf.data(), d);
    if (st != CASPT2_OK) return st;
  }

  k_na_prepare<<<(d.c + d.v + 127) / 128 + 1, 128, 0, s>>>(fock, nmo, d.c, d.a, d.v, s0 + L.eps,
                                                         s0 + L.mindenom, status);
  CASPT2_CUDA_TRY(cudaGetLastError());
  if (d.a > 0) {
    CASPT2_CUDA_TRY(launch_fref(fock, rdm1, d, s0 + L.fref, s));
  } else {
    CASPT2_CUDA_TRY(cudaMemsetAsync(s0 + L.fref, 0, sizeof(double) * n * n, s));
  }
  CASPT2_CUDA_TRY(launch_sym_eig(s0 + L.fref, n, s0 + L.U, s0 + L.Etil, opt->xms ? 0 : 1, status, s));
  CASPT2_CUDA_TRY(launch_congruence(s0 + L.fref, s0 + L.U, n, s0 + L.Ftil, s));
  CASPT2_CUDA_TRY(launch_diag(s0 + L.Ftil, n, s0 + L.E0, s));
  if (d.c == 0 || d.v == 0) {
    CASPT2_CUDA_TRY(cudaMemsetAsync(e, 0, sizeof(double) * n * n, s));
    CASPT2_CUDA_TRY(cudaMemsetAsync(norm, 0, sizeof(double) * n, s));
    int hst0 = 0;   // the XMS eigensolve may have set ENOTCONV or ENAN
    CASPT2_CUDA_TRY(cudaMemcpyAsync(&hst0, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
    return hst0;
  }
  CASPT2_CUDA_TRY(launch_sym_eig(s0 + L.Ftil, n, s0 + L.W, s0 + L.omega, 0, status, s));
  k_na_shifts<<<1, kNaMaxShift, 0, s>>>(s0 + L.omega, s0 + L.E0, opt->shift, n, opt->scheme,
                                       s0 + L.shifts);
  const int ntile = (d.v + kNaT - 1) / kNaT;
  const long ntask = (long)d.c * (d.c + 1) / 2 * ((long)ntile * (ntile + 1) / 2);
  const int grid = (int)(ntask < kNaGrid ? ntask : kNaGrid);
  k_na_classH<<<grid, kNaThreads, 0, s>>>(dfB, s0 + L.eps, s0 + L.shifts, nshift, d.c, d.v, d.X,
                                         nmo, d.c + d.a, ntile, ntask, s0 + L.partial);
  const int ncol = 2 * nshift + 1;
  k_na_reduce<<<ncol, 256, 0, s>>>(s0 + L.partial, grid, ncol, s0 + L.sums);
  k_na_combine<<<1, kNaMaxShift, 0, s>>>(s0 + L.sums, s0 + L.W, n, opt->scheme, e, norm,
                                        s0 + L.mindenom, status);
  CASPT2_CUDA_TRY(cudaGetLastError());
  int hst = 0;
  double hmin = 0.0;
  CASPT2_CUDA_TRY(cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaMemcpyAsync(&hmin, s0 + L.mindenom, sizeof(double), cudaMemcpyDeviceToHost, s));
  CASPT2_CUDA_TRY(cudaStreamSynchronize(s));
  if (hst != 0) return hst;
  if (hmin < 1e-3) return CASPT2_WINTRUDER;
  return CASPT2_OK;
}
