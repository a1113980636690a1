// FP64-accurate GEMM from exact BF16 slices on the tcgen05 tensor cores (see ozaki.cuh).
//
// One CTA computes a 128 x 64 tile of C.  Its K loop runs over stages of 16: all 256
// threads copy (cp.async, 16 bytes each, all in flight together) the S slices of the A
// and B tiles into a ring of four shared-memory buffers, two stages ahead of the MMAs
// (canonical K-major layout without swizzle: core matrices of 8 rows x 16 bytes, K-adjacent
// core matrices 128 bytes apart, row groups 256 bytes apart), one thread issues the
// tcgen05.mma instructions of every slice pair (s, t) with s + t < S into the TMEM
// accumulator of level s + t (128 lanes x 64 FP32 columns per level) and commits them to
// that buffer's mbarrier; a buffer is refilled once its stage's MMAs have completed.  After each
// K chunk of 256 the eight warps read the S levels from TMEM (warp w: lanes 32 (w % 4).., 32
// columns at 32 (w / 4)); the level sums (exact integers) are added, shifted, into two
// int64 accumulators per output, converted to FP64 once at the end.  Every mbarrier wait
// is bounded; on timeout the CTA records the error, stops issuing work, waits (bounded)
// for its committed MMAs and frees its TMEM.
#include <algorithm>
#include <cstdint>

#include "ozaki.cuh"

namespace caspt2 {

namespace {

constexpr int kOzM = 128, kOzN = 64;
constexpr int kOzThreads = 256;
constexpr long kOzSpin = 1L << 22;
constexpr int kOzKs = 16;                           // K per shared-memory stage (one MMA)
constexpr int kOzBufs = 4;                          // stage ring; copies run 2 stages ahead
constexpr int kOzASlice = kOzM * kOzKs * 2;         // bytes of one A slice tile per stage
constexpr int kOzBSlice = kOzN * kOzKs * 2;
constexpr int kOzSbo = (kOzKs / 8) * 128;           // row-group stride (bytes)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading byte offset
// >> 4 (bits 16-29, between core matrices adjacent in K), stride byte offset >> 4
// (bits 32-45, between core matrices adjacent in M/N), version 1 (bit 46), no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B BF16 (bits 7-9 and
// 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                            ((uint32_t)(kOzN >> 3) << 17) | ((uint32_t)(kOzM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_u32(bar)));
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long it = 0; it < kOzSpin; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kOzThreads, 1)
k_oz_gemm(const __nv_bfloat16* __restrict__ As, const double* __restrict__ sa,
          const __nv_bfloat16* __restrict__ Bs, const double* __restrict__ sb, int M, int N,
          int Kp, int S, int chunks_per_split, double alpha, double beta, double* __restrict__ C,
          long ldc, double* __restrict__ part, int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t bars[kOzBufs];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kOzM, n0 = blockIdx.x * kOzN;
  const long sliceA = (long)M * Kp, sliceB = (long)N * Kp;
  const int stage_bytes = S * (kOzASlice + kOzBSlice);
  const uint32_t tcols = 512;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < kOzBufs; ++q)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[q])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = tmem_base;

  // exact integer accumulation of the level sums: hi = sum_(l<3) L_l 2^(7(2-l)),
  // lo = sum_(l>=3) L_l 2^(7(S-1-l)); value = hi 2^-28 + lo 2^(-7(S+1))
  long long hi[32], lo[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0;

  const int spc = kOzKChunk / kOzKs;              // stages per exact chunk
  // stages of this split (blockIdx.z): exact chunks [z cps, (z + 1) cps)
  const int gbeg = blockIdx.z * chunks_per_split * spc;
  const int nst = max(0, min(Kp / kOzKs, gbeg + chunks_per_split * spc) - gbeg);

  // copy of stage g into ring buffer g % kOzBufs: S slices of A (128 rows) and B (64 rows),
  // 16-byte pieces of 8 K values, all in flight together; one commit group per stage
  auto issue_copy = [&](int g) {
    uint8_t* buf = smem + (long)(g % kOzBufs) * stage_bytes;
    const int nA = S * kOzM * (kOzKs / 8), nB = S * kOzN * (kOzKs / 8);
    const int k0 = (gbeg + g) * kOzKs;
    for (int q = tid; q < nA + nB; q += kOzThreads) {
      const bool isA = q < nA;
      const int qq = isA ? q : q - nA;
      const int c = qq % (kOzKs / 8);
      const int rr = (qq / (kOzKs / 8)) % (isA ? kOzM : kOzN);
      const int s = qq / ((kOzKs / 8) * (isA ? kOzM : kOzN));
      const int grow = (isA ? m0 : n0) + rr;
      const bool ok = grow < (isA ? M : N);
      // rows past the edge read nothing (source size 0) and are zero-filled
      const __nv_bfloat16* src =
          ok ? (isA ? As + s * sliceA : Bs + s * sliceB) + (long)grow * Kp + k0 + 8 * c : As;
      uint8_t* dst = buf + (isA ? s * kOzASlice : S * kOzASlice + s * kOzBSlice) +
                     (rr >> 3) * kOzSbo + c * 128 + (rr & 7) * 16;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)),
                   "l"(src), "r"(ok ? 16 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // MMAs of stage g complete the (g / kOzBufs)-th phase of bars[g % kOzBufs]
  auto stage_parity = [](int g) { return (uint32_t)((g / kOzBufs) & 1); };

  for (int g = 0; g < 2 && g < nst; ++g) issue_copy(g);
  int committed = 0;                              // stages whose MMAs were committed
  for (int g = 0; g < nst; ++g) {
    // copy of stage g done (the copy of g + 1 may still be in flight)
    if (g + 1 < nst) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (abort_flag) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const bool first = (g % spc) == 0;
      const uint32_t ab = smem_u32(smem + (long)(g % kOzBufs) * stage_bytes);
      const uint32_t bb = ab + S * kOzASlice;
      for (int s = 0; s < S; ++s)
        for (int t = 0; t < S - s; ++t) {
          const uint64_t ad = sdesc(ab + s * kOzASlice, 128, kOzSbo);
          const uint64_t bd = sdesc(bb + t * kOzBSlice, 128, kOzSbo);
          const uint32_t accf = (first && s == 0) ? 0u : 1u;
          mma_bf16(tbase + (uint32_t)((s + t) * kOzN), ad, bd, accf);
        }
      mma_commit(&bars[g % kOzBufs]);
    }
    committed = g + 1;
    // prefetch stage g + 2 into the buffer of stage g - 2 once its MMAs are done
    if (g + 2 < nst) {
      if (g >= 2 && !bar_wait(&bars[(g + 2) % kOzBufs], stage_parity(g - 2))) abort_flag = 1;
      issue_copy(g + 2);
    }
    if ((g % spc) == spc - 1 || g == nst - 1) {
      // end of an exact chunk: add the S level sums into the integer accumulators
      if (!bar_wait(&bars[g % kOzBufs], stage_parity(g))) abort_flag = 1;
      __syncthreads();
      if (abort_flag) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t lb = (uint32_t)(32 * (warp & 3)) << 16;
      const uint32_t cb = (uint32_t)(32 * (warp >> 2));
      for (int l = 0; l < S; ++l) {
        uint32_t r[32];
        tmem_ld32(tbase + lb + (uint32_t)(l * kOzN) + cb, r);
        // each level sum is an integer below 2^24: exact in FP32 and in int32
        if (l < 3) {
          const int sh = 7 * (2 - l);
#pragma unroll
          for (int j = 0; j < 32; ++j)
            hi[j] += (long long)__float2int_rn(__uint_as_float(r[j])) << sh;
        } else {
          const int sh = 7 * (S - 1 - l);
#pragma unroll
          for (int j = 0; j < 32; ++j)
            lo[j] += (long long)__float2int_rn(__uint_as_float(r[j])) << sh;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // drain: the MMAs of the last committed stages must finish before TMEM is freed
  if (abort_flag) {
    if (tid == 0) atomicExch(err, 1);
    for (int g = committed - kOzBufs; g < committed; ++g)
      if (g >= 0) bar_wait(&bars[g % kOzBufs], (uint32_t)((g / kOzBufs) & 1));
  } else {
    const int row = m0 + 32 * (warp & 3) + lane;
    double acc[32];
    const double wlo = ldexp(1.0, -7 * (S + 1));
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = (double)hi[j] * 0x1p-28 + (double)lo[j] * wlo;
    if (row < M) {
      const double sr = alpha * sa[row];
      if (part) {   // split K: this split's share, summed in a fixed order afterwards
        double* prow = part + ((long)blockIdx.z * M + row) * N;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + 32 * (warp >> 2) + j;
          if (col < N) prow[col] = sr * sb[col] * acc[j];
        }
      } else {
        double* crow = C + (long)row * ldc;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = n0 + 32 * (warp >> 2) + j;
          if (col < N) {
            const double v = sr * sb[col] * acc[j];
            crow[col] = beta == 0.0 ? v : v + beta * crow[col];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(tcols));
  }
}

// C[i][j] = sum_z part[z][i][j] (fixed order) + beta C[i][j]
__global__ void k_oz_reduce(const double* __restrict__ part, int nsplit, int M, int N,
                            double beta, double* __restrict__ C, long ldc) {
  const long total = (long)M * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int z = 0; z < nsplit; ++z) v += part[(long)z * total + e];
    double* c = C + (e / N) * ldc + e % N;
    *c = beta == 0.0 ? v : v + beta * *c;
  }
}

// Element (r, k) of a view; k = (k / kin, k % kin) in 32-bit arithmetic (k, kin < 2^31).
__device__ __forceinline__ double oz_at(const OzView& v, long r, unsigned k, bool split_k) {
  if (!split_k) return v.X[r * v.rs + (long)k * v.cs];
  const unsigned kin = (unsigned)v.kin, p = k / kin, q = k - p * kin;
  return v.X[r * v.rs + (long)p * v.kout + (long)q * v.cs];
}

// 32 x 32 tiles (rows x K) staged in shared memory: global reads run along the unit stride
// of the view (rows when rs == 1, else K), then row maxima or slices are formed per tile.
constexpr int kOzTile = 32;

__device__ __forceinline__ void oz_load_tile(const OzView& v, int R, int K, int r0, int k0,
                                             bool split_k, double (*t)[kOzTile + 1]) {
  const bool rows_fast = v.rs == 1 && v.cs != 1;
  for (int q = threadIdx.x; q < kOzTile * kOzTile; q += blockDim.x) {
    const int a = q % kOzTile, b = q / kOzTile;     // a runs along the fast index
    const int rr = rows_fast ? a : b, kk = rows_fast ? b : a;
    const int r = r0 + rr, k = k0 + kk;
    t[rr][kk] = (r < R && k < K) ? oz_at(v, r, (unsigned)k, split_k) : 0.0;
  }
}

// Row maxima of |x| as the bit patterns of non-negative doubles (order-independent
// atomicMax on integers, so the result does not depend on the schedule and no FP64
// instruction is spent).  grid (K tiles, row tiles).
__global__ void k_oz_rowmax(OzView v, int R, int K, bool split_k,
                            unsigned long long* __restrict__ mx) {
  __shared__ double t[kOzTile][kOzTile + 1];
  const int k0 = blockIdx.x * kOzTile;
  for (int r0 = blockIdx.y * kOzTile; r0 < R; r0 += gridDim.y * kOzTile) {
    oz_load_tile(v, R, K, r0, k0, split_k, t);
    __syncthreads();
    if (threadIdx.x < kOzTile && r0 + (int)threadIdx.x < R) {
      unsigned long long m = 0;
      for (int kk = 0; kk < kOzTile; ++kk) {
        const unsigned long long b =
            (unsigned long long)__double_as_longlong(t[threadIdx.x][kk]) & 0x7FFFFFFFFFFFFFFFull;
        m = b > m ? b : m;
      }
      if (m) atomicMax(mx + r0 + threadIdx.x, m);
    }
    __syncthreads();
  }
}

// sigma_r = 2^(floor(log2 max|x_r|) + 1) (1 for a zero row).
__global__ void k_oz_scale(const unsigned long long* __restrict__ mx, int R,
                           double* __restrict__ scale) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const double m = __longlong_as_double((long long)mx[r]);
  scale[r] = m > 0.0 ? ldexp(1.0, ilogb(m) + 1) : 1.0;
}

// S slices of x / sigma_r into out[s][r][Kp] (zeros for K <= k < Kp); grid (Kp tiles,
// row tiles), writes along K.
__global__ void k_oz_split(OzView v, int R, int K, int Kp, int S, bool split_k,
                           const double* __restrict__ scale, __nv_bfloat16* __restrict__ out) {
  __shared__ double t[kOzTile][kOzTile + 1];
  __shared__ int er[kOzTile];
  const int k0 = blockIdx.x * kOzTile;
  const long plane = (long)R * Kp;
  for (int r0 = blockIdx.y * kOzTile; r0 < R; r0 += gridDim.y * kOzTile) {
    oz_load_tile(v, R, K, r0, k0, split_k, t);
    if (threadIdx.x < kOzTile)
      er[threadIdx.x] = r0 + (int)threadIdx.x < R ? ilogb(scale[r0 + threadIdx.x]) : 0;
    __syncthreads();
    for (int q = threadIdx.x; q < kOzTile * kOzTile; q += blockDim.x) {
      const int kk = q % kOzTile, rr = q / kOzTile;
      const int r = r0 + rr, k = k0 + kk;
      if (r >= R || k >= Kp) continue;
      // x / sigma_r (|.| < 1) as a 2^56 fixed-point integer, taken from the bits of x: the
      // 53-bit significand shifted by (exponent - 52 + 56 - log2 sigma_r), rounded to nearest
      const long long bits = __double_as_longlong(t[rr][kk]);
      const int ex = (int)((bits >> 52) & 0x7FF);
      long long X = 0;
      if (ex != 0) {
        const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
        const int sh = ex - 1023 + 4 - er[rr];
        if (sh >= 0) X = mant << sh;
        else if (sh > -60) X = (mant + (1LL << (-sh - 1))) >> (-sh);
        if (bits < 0) X = -X;
      }
      // slice s: the signed 7-bit digit of weight 2^(49 - 7 s), rounded to nearest, so
      // |a_0| <= 128 and |a_s| <= 64
      const long e = (long)r * Kp + k;
      for (int s = 0; s < S; ++s) {
        const int sh = 49 - 7 * s;
        const long long a = (X + (1LL << (sh - 1))) >> sh;
        X -= a << sh;
        out[(long)s * plane + e] = __float2bfloat16_rn((float)a);
      }
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t oz_split(const OzView& v, int R, int K, int Kp, int S, __nv_bfloat16* out,
                     double* scale, cudaStream_t s) {
  if (R <= 0) return cudaSuccess;
  if ((long)Kp >= (1L << 31)) return cudaErrorInvalidValue;
  const bool split_k = v.kin < K;
  // the row maxima are staged in the scale array itself (same size, 8 bytes each)
  unsigned long long* mx = reinterpret_cast<unsigned long long*>(scale);
  cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * R, s);
  if (e != cudaSuccess) return e;
  const unsigned rt = std::min<unsigned>((R + kOzTile - 1) / kOzTile, 65535u);
  ++launch_counter();
  k_oz_rowmax<<<dim3((K + kOzTile - 1) / kOzTile, rt), 256, 0, s>>>(v, R, K, split_k, mx);
  ++launch_counter();
  k_oz_scale<<<(R + 255) / 256, 256, 0, s>>>(mx, R, scale);
  ++launch_counter();
  k_oz_split<<<dim3((Kp + kOzTile - 1) / kOzTile, rt), 256, 0, s>>>(v, R, K, Kp, S, split_k,
                                                                    scale, out);
  return cudaGetLastError();
}

cudaError_t oz_gemm(const __nv_bfloat16* As, const double* sa, const __nv_bfloat16* Bs,
                    const double* sb, int M, int N, int Kp, int S, double alpha, double beta,
                    double* C, long ldc, int* err, cudaStream_t s, int nsplit, double* part) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (S < 1 || S > kOzMaxSlices || Kp % kOzKStage != 0) return cudaErrorInvalidValue;
  // at least 116 KB so that one CTA (holding all 512 TMEM columns) runs per SM; the
  // attribute is global to the kernel, so it is set to the fixed maximum (7 slices)
  const int smem = std::max(kOzBufs * S * (kOzASlice + kOzBSlice), 116 * 1024);
  const int smem_max = std::max(kOzBufs * kOzMaxSlices * (kOzASlice + kOzBSlice), 116 * 1024);
  cudaError_t e =
      cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e != cudaSuccess) return e;
  const int nchunk = (Kp + kOzKChunk - 1) / kOzKChunk;
  nsplit = std::max(1, std::min(nsplit, nchunk));
  const int cps = (nchunk + nsplit - 1) / nsplit;
  nsplit = (nchunk + cps - 1) / cps;
  if (nsplit > 1 && !part) return cudaErrorInvalidValue;
  dim3 grid((N + kOzN - 1) / kOzN, (M + kOzM - 1) / kOzM, nsplit);
  ++launch_counter();
  k_oz_gemm<<<grid, kOzThreads, smem, s>>>(As, sa, Bs, sb, M, N, Kp, S, cps, alpha, beta, C, ldc,
                                           nsplit > 1 ? part : nullptr, err);
  if (nsplit > 1) {
    const long total = (long)M * N;
    ++launch_counter();
    k_oz_reduce<<<(int)std::max<long>(1, std::min<long>((total + 255) / 256, 152L * 8)), 256, 0, s>>>(
        part, nsplit, M, N, beta, C, ldc);
  }
  return cudaGetLastError();
}

void oz_release(OzWork& w) {
  if (w.sl) cudaFree(w.sl);
  if (w.sc) cudaFree(w.sc);
  if (w.err) cudaFree(w.err);
  if (w.part) cudaFree(w.part);
  w.part = nullptr;
  w.part_n = 0;
  w.sl = nullptr;
  w.sc = nullptr;
  w.err = nullptr;
  w.sl_bytes = w.sc_n = 0;
}

namespace {
cudaError_t oz_reserve(OzWork& w, size_t bytes, size_t nsc) {
  cudaError_t e = cudaSuccess;
  if (!w.err) {
    if ((e = cudaMalloc(&w.err, sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMemset(w.err, 0, sizeof(int))) != cudaSuccess) return e;
  }
  if (bytes > w.sl_bytes) {
    if (w.sl) cudaFree(w.sl);
    w.sl = nullptr;
    w.sl_bytes = 0;
    if ((e = cudaMalloc(&w.sl, bytes)) != cudaSuccess) return e;
    w.sl_bytes = bytes;
  }
  if (nsc > w.sc_n) {
    if (w.sc) cudaFree(w.sc);
    w.sc = nullptr;
    w.sc_n = 0;
    if ((e = cudaMalloc(&w.sc, nsc * sizeof(double))) != cudaSuccess) return e;
    w.sc_n = nsc;
  }
  return cudaSuccess;
}
}  // namespace

cudaError_t oz_matmul(OzWork& w, const OzView& A, const OzView& B, bool same, int M, int N,
                      int K, double alpha, double beta, double* C, long ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int Kp = oz_kpad(std::max(K, 1));
  const size_t a_bytes = oz_slice_bytes(M, std::max(K, 1), w.S);
  const size_t b_bytes = same ? 0 : oz_slice_bytes(N, std::max(K, 1), w.S);
  cudaError_t e = oz_reserve(w, a_bytes + b_bytes, (size_t)M + (same ? 0 : N));
  if (e != cudaSuccess) return e;
  __nv_bfloat16* as = w.sl;
  __nv_bfloat16* bs = same ? w.sl : w.sl + a_bytes / sizeof(__nv_bfloat16);
  double* sa = w.sc;
  double* sb = same ? w.sc : w.sc + M;
  if ((e = oz_split(A, M, K, Kp, w.S, as, sa, s)) != cudaSuccess) return e;
  if (!same && (e = oz_split(B, N, K, Kp, w.S, bs, sb, s)) != cudaSuccess) return e;
  // split K over CTAs when the output has few tiles (about two waves of 152 SMs)
  const long tiles = (long)((M + 127) / 128) * ((N + 63) / 64);
  const int nchunk = (Kp + kOzKChunk - 1) / kOzKChunk;
  int nsplit = (int)std::max<long>(1, std::min<long>(nchunk, (304 + tiles - 1) / tiles));
  if (nsplit > 1) {
    const size_t need = (size_t)nsplit * M * N;
    if (need > w.part_n) {
      if (w.part) cudaFree(w.part);
      w.part = nullptr;
      w.part_n = 0;
      if ((e = cudaMalloc(&w.part, need * sizeof(double))) != cudaSuccess) return e;
      w.part_n = need;
    }
  }
  return oz_gemm(as, sa, bs, sb, M, N, Kp, w.S, alpha, beta, C, ldc, w.err, s, nsplit, w.part);
}

}  // namespace caspt2
