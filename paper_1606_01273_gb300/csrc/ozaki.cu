// FP64-accurate GEMM from exact BF16 slices on the tcgen05 tensor cores (see ozaki.cuh).
//
// Persistent CTAs (one per SM) walk the 128 x 64 tiles of C (and K splits) with
// warp-specialised roles and a ring of five shared-memory stages of K = 16 that runs on
// across tiles:
//   warp 0 (one thread)  TMA producer: per stage four bulk-tensor copies (two K groups of 8
//                        for A and for B, each box holding all S slices: {8 K, rows, S}),
//                        completing the stage's `full` mbarrier by transaction bytes;
//   warp 1 (one thread)  MMA issuer: per stage, for every A slice s, the tcgen05.mma of
//                        slice s with the B slices t < S - s (stacked along N, up to four
//                        per instruction) into the TMEM accumulators of levels s + t (128
//                        lanes x 64 FP32 columns per level), committed to the stage's `empty`
//                        mbarrier, and at the end of every exact K chunk of 256 to `tfull`;
//   warps 2-9            epilogue: after each chunk they read the S levels from TMEM (warp w:
//                        lanes 32 (w % 4).., 32 columns at 32 ((w - 2) / 4)), add the exact
//                        integer level sums, shifted, into two int64 accumulators per output
//                        and release TMEM through `tempty`; FP64 conversion once at the end.
// The shared-memory layout is the canonical K-major one without swizzle: core matrices of
// 8 rows x 16 bytes, M/N-adjacent core matrices 128 bytes apart (the TMA box rows), K-adjacent
// ones one box apart.  Every mbarrier wait is bounded; on timeout the CTA records the error,
// stops issuing work, waits (bounded) for its copies and MMAs in flight and frees its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "ozaki.cuh"

namespace caspt2 {

namespace {

constexpr int kOzM = 128, kOzN = 64;
constexpr int kOzThreads = 320;                     // warps: TMA, MMA, eight epilogue
constexpr long kOzSpin = 1L << 22;
constexpr int kOzKs = 16;                           // K per shared-memory stage (one MMA)
constexpr int kOzStages = 5;                        // stage ring
constexpr int kOzABox = kOzM * 8 * 2;               // bytes of one slice of an A box (8 K)
constexpr int kOzBBox = kOzN * 8 * 2;
__host__ __device__ inline int oz_stage_bytes(int S) { return 2 * S * (kOzABox + kOzBBox); }

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
__host__ __device__ constexpr uint32_t oz_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kOzM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
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

__device__ __forceinline__ void bar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                          int c2, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__global__ void __launch_bounds__(kOzThreads, 1)
k_oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          const double* __restrict__ sa, const double* __restrict__ sb, int M, int N, int Kp,
          int S, int chunks_per_split, int nsplit, double alpha, double beta,
          double* __restrict__ C, long ldc, double* __restrict__ part, int* err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[kOzStages], empty[kOzStages], tfull, tempty;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, n_issued, n_committed;
  volatile int* abort_v = &abort_flag;
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int stage_bytes = oz_stage_bytes(S);
  const uint32_t tcols = 512;

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < kOzStages; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[q])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tfull)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_u32(&tempty)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
    n_issued = n_committed = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = tmem_base;

  // tiles (n tile, m tile, K split) in a persistent loop; every role walks the same
  // sequence, and the stage ring and barrier phases run on across tiles
  const int ntn = (N + kOzN - 1) / kOzN, ntm = (M + kOzM - 1) / kOzM;
  const long ntiles = (long)ntn * ntm * nsplit;
  const int spc = kOzKChunk / kOzKs;              // stages per exact chunk
  auto tile_of = [&](long ti, int& m0, int& n0, int& z, int& gbeg, int& nst) {
    n0 = (int)(ti % ntn) * kOzN;
    m0 = (int)((ti / ntn) % ntm) * kOzM;
    z = (int)(ti / ((long)ntn * ntm));
    gbeg = z * chunks_per_split * spc;            // stages of K split z
    nst = max(0, min(Kp / kOzKs, gbeg + chunks_per_split * spc) - gbeg);
  };

  if (warp == 0) {
    if (lane == 0) {
      int G = 0;                                  // stages issued by this CTA
      for (long ti = blockIdx.x; ti < ntiles && !*abort_v; ti += gridDim.x) {
        int m0, n0, z, gbeg, nst;
        tile_of(ti, m0, n0, z, gbeg, nst);
        for (int g = 0; g < nst; ++g, ++G) {
          const int b = G % kOzStages;
          if (G >= kOzStages && !bar_wait(&empty[b], (uint32_t)(((G / kOzStages) - 1) & 1))) {
            *abort_v = 1;
            break;
          }
          if (*abort_v) break;
          bar_arrive_tx(&full[b], (uint32_t)stage_bytes);
          const uint32_t da = smem_u32(smem + (long)b * stage_bytes);
          const uint32_t db = da + 2 * S * kOzABox;
          const int k0 = (gbeg + g) * kOzKs;
          tma_load3(da, &tmA, k0, m0, 0, &full[b]);
          tma_load3(da + S * kOzABox, &tmA, k0 + 8, m0, 0, &full[b]);
          tma_load3(db, &tmB, k0, n0, 0, &full[b]);
          tma_load3(db + S * kOzBBox, &tmB, k0 + 8, n0, 0, &full[b]);
          n_issued = G + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint64_t adesc0 = sdesc(smem_u32(smem), S * kOzABox, 128);
      const uint64_t bdesc0 = sdesc(smem_u32(smem) + 2 * S * kOzABox, S * kOzBBox, 128);
      int G = 0, Cc = 0;                          // stages and chunks of this CTA
      for (long ti = blockIdx.x; ti < ntiles && !*abort_v; ti += gridDim.x) {
        int m0, n0, z, gbeg, nst;
        tile_of(ti, m0, n0, z, gbeg, nst);
        for (int g = 0; g < nst; ++g, ++G) {
          const int b = G % kOzStages;
          const bool first = (g % spc) == 0;
          if (first && Cc > 0 && !bar_wait(&tempty, (uint32_t)((Cc - 1) & 1))) {
            *abort_v = 1;
            break;
          }
          if (!bar_wait(&full[b], (uint32_t)((G / kOzStages) & 1))) {
            *abort_v = 1;
            break;
          }
          if (*abort_v) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint64_t soff = (uint64_t)((b * stage_bytes) >> 4);
          // the B slices of a stage are stacked along N (slice t at rows 64 t..), so one MMA
          // multiplies A slice s by B slices t0 .. t0 + cnt - 1 into the TMEM column blocks
          // s + t0 .. (levels), up to four slices (N = 256) per instruction
          for (int s = 0; s < S; ++s) {
            const uint64_t ad = adesc0 + soff + (uint64_t)((s * kOzABox) >> 4);
            for (int t0 = 0; t0 < S - s; t0 += 4) {
              const int cnt = min(4, S - s - t0);
              const uint64_t bd = bdesc0 + soff + (uint64_t)((t0 * kOzBBox) >> 4);
              mma_bf16(tbase + (uint32_t)((s + t0) * kOzN), ad, bd, oz_idesc(kOzN * cnt),
                       (first && s == 0) ? 0u : 1u);
            }
          }
          mma_commit(&empty[b]);
          if ((g % spc) == spc - 1 || g == nst - 1) {
            mma_commit(&tfull);
            ++Cc;
          }
          n_committed = G + 1;
        }
      }
    }
  } else {
    // epilogue: per tile, one chunk of S levels at a time; TMEM is released as soon as the
    // levels are in registers, so the next chunk's (or tile's) MMAs overlap the stores
    const int q = warp & 3, h = (warp - 2) >> 2;
    const uint32_t lb = (uint32_t)(32 * q) << 16;
    int Cc = 0;
    for (long ti = blockIdx.x; ti < ntiles && !*abort_v; ti += gridDim.x) {
      int m0, n0, z, gbeg, nst;
      tile_of(ti, m0, n0, z, gbeg, nst);
      const int nchunk = (nst + spc - 1) / spc;
      // exact integer accumulation of the level sums: hi = sum_(l<3) L_l 2^(7(2-l)),
      // lo = sum_(l>=3) L_l 2^(7(S-1-l)); value = hi 2^-28 + lo 2^(-7(S+1))
      long long hi[32], lo[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0;
      bool ok = true;
      for (int c = 0; c < nchunk; ++c, ++Cc) {
        if (!bar_wait(&tfull, (uint32_t)(Cc & 1))) {
          *abort_v = 1;
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int l = 0; l < S; ++l) {
          uint32_t r[32];
          tmem_ld32(tbase + lb + (uint32_t)(l * kOzN + 32 * h), r);
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
        __syncwarp();
        if (lane == 0) bar_arrive(&tempty);
      }
      if (!ok) break;
      const int row = m0 + 32 * q + lane;
      double acc[32];
      const double wlo = ldexp(1.0, -7 * (S + 1));
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = (double)hi[j] * 0x1p-28 + (double)lo[j] * wlo;
      if (row < M) {
        const double sr = alpha * sa[row];
        if (part) {   // split K: this split's share, summed in a fixed order afterwards
          double* prow = part + ((long)z * M + row) * N;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + 32 * h + j;
            if (col < N) prow[col] = sr * sb[col] * acc[j];
          }
        } else {
          double* crow = C + (long)row * ldc;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + 32 * h + j;
            if (col < N) {
              const double v = sr * sb[col] * acc[j];
              crow[col] = beta == 0.0 ? v : v + beta * crow[col];
            }
          }
        }
      }
    }
  }
  __syncthreads();
  if (*abort_v) {
    // drain: copies in flight must land and committed MMAs finish before the CTA leaves
    if (tid == 0) atomicExch(err, 1);
    if (tid == 0)
      for (int g = max(0, n_issued - kOzStages); g < n_issued; ++g)
        bar_wait(&full[g % kOzStages], (uint32_t)((g / kOzStages) & 1));
    if (tid == 32)
      for (int g = max(0, n_committed - kOzStages); g < n_committed; ++g)
        bar_wait(&empty[g % kOzStages], (uint32_t)((g / kOzStages) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 1) {
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

namespace {
// cuTensorMapEncodeTiled through the runtime's driver entry point (resolved once)
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 3-D map of slices out[s][r][Kp] (BF16): dims (Kp, R, S), box (8 K, rows, S).
bool slice_map(CUtensorMap* map, const __nv_bfloat16* X, int R, int Kp, int S, int rows) {
  auto enc = tmap_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)R, (cuuint64_t)S};
  const cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)R * Kp * 2};
  const cuuint32_t box[3] = {8u, (cuuint32_t)rows, (cuuint32_t)S};
  const cuuint32_t es[3] = {1u, 1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(X), dims,
             strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

cudaError_t oz_gemm(const __nv_bfloat16* As, const double* sa, const __nv_bfloat16* Bs,
                    const double* sb, int M, int N, int Kp, int S, double alpha, double beta,
                    double* C, long ldc, int* err, cudaStream_t s, int nsplit, double* part) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (S < 1 || S > kOzMaxSlices || Kp % kOzKStage != 0) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(As) | reinterpret_cast<uintptr_t>(Bs)) & 15)
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!slice_map(&ma, As, M, Kp, S, kOzM) || !slice_map(&mb, Bs, N, Kp, S, kOzN))
    return cudaErrorInvalidValue;
  // the ring of five stages (1 KB alignment slack); the attribute is global to the kernel,
  // so it is set to the fixed maximum (7 slices)
  const int smem = kOzStages * oz_stage_bytes(S) + 1024;
  const int smem_max = kOzStages * oz_stage_bytes(kOzMaxSlices) + 1024;
  cudaError_t e =
      cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
  if (e != cudaSuccess) return e;
  const int nchunk = (Kp + kOzKChunk - 1) / kOzKChunk;
  nsplit = std::max(1, std::min(nsplit, nchunk));
  const int cps = (nchunk + nsplit - 1) / nsplit;
  nsplit = (nchunk + cps - 1) / cps;
  if (nsplit > 1 && !part) return cudaErrorInvalidValue;
  // persistent CTAs (one per SM: the ring and all 512 TMEM columns) over the tiles
  const long ntiles = (long)((N + kOzN - 1) / kOzN) * ((M + kOzM - 1) / kOzM) * nsplit;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<long>(ntiles, nsm);
  ++launch_counter();
  k_oz_gemm<<<grid, kOzThreads, smem, s>>>(ma, mb, sa, sb, M, N, Kp, S, cps, nsplit, alpha, beta,
                                           C, ldc, nsplit > 1 ? part : nullptr, err);
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
