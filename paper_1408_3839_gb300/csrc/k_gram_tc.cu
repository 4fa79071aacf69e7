// k_gram_tc.cu -- step a3 on the tensor cores (LHF_MIXED): the weighted 1D Gram contraction
// C_r[row] = sum_c V_r(c) Q_row(c) of the folded products Q (rows = (window block, mu, nu))
// with the potential factors V, from the exact base-2^7 digit planes written by k_gram_slice /
// k_vslice (k_gram.cu).  Only the rows whose functions overlap somewhere (gram_row_cells > 0;
// 41% of tube_256's direction-0 rows) are contracted, in the compact order of k_gram_rowmap; the
// results go to their rows through its map, the other rows' factors are zeros.
//
// With row = 2^e_row sum_a alpha_a 2^(-7(a+1)) and V_r = 2^e_r sum_b beta_b 2^(-7(b+1)) (digits
// alpha, beta integers with |.| <= 128), the contraction is
//   C_r[row] = 2^(e_row + e_r) sum_s 2^(-7(s+2)) D_s,   D_s = sum_c sum_{a+b=s} alpha_a(c) beta_b(c),
// the splitting of Ozaki et al. ("Error-free transformations of matrix multiplication by using
// fast routines of matrix multiplication", 2012) with the 28 digit pairs a + b <= 6 kept
// (relative truncation ~2^-48 of sum |Q| |V|).  Each D_s is an integer below 2^24 for K <= 448, so
// BF16 x BF16 products accumulated in FP32 are exact; the recombination runs in 64-bit integers
// (its one rounding, 2^-53 of the scale, is far below the truncation of the dropped pairs) and is
// converted to FP64 once.
//
// Jobs are (system, direction, 128-row tile, 64-column tile); a persistent grid of one CTA per SM
// takes every gridDim.x-th job, warp 0 running the loads and MMAs one chunk ahead across its tiles
// while warps 1 .. 8 drain the previous tile's accumulators (mbarriers tmem_full / tmem_empty):
//   * TMA (cp.async.bulk.tensor.2d, 64-byte swizzle, no multicast) brings, per 32-wide K chunk,
//     the 7 digit planes of the A tile (7 x 128 x 32 BF16) and of the B tile (7 x 64 x 32) into
//     one of two shared-memory stages (84 KB each): the load of chunk k + 1 runs while the MMAs
//     of chunk k execute;
//   * one thread issues tcgen05.mma.cta_group::1.kind::f16 (M = 128, K = 16) for every pair
//     (a, b) into the TMEM accumulator of its diagonal s = a + b (7 x 64 columns of the 512
//     allocated) -- the B planes of consecutive b side by side in shared memory, so that one MMA
//     of N = 64 nb takes plane a against nb of them -- then tcgen05.commit to the stage's
//     mbarrier, which frees the stage;
//   * warps 1 .. 8 read the accumulators back with tcgen05.ld (32x32b; warp w reads TMEM lanes
//     32 (w % 4) .. + 31, half of the columns each), release them, recombine the 7 diagonals and
//     store the FP64 results in the layout of the FP64 route.
// Every mbarrier wait is bounded (~1 s of clock cycles); on time-out the CTA sets kFlagTimeout,
// waits (bounded) for its outstanding operations, frees its TMEM and returns.
#include <cuda.h>
#include <algorithm>
#include <mutex>
#include <string.h>

#include <vector>

#include "lhf_internal.cuh"

namespace lhf {
namespace {

constexpr int kEpiWarps = 8;  // warps 1 .. 8 read TMEM lane quadrant w % 4, half the columns each
constexpr int kTcThreads = 32 * (1 + kEpiWarps);
constexpr int kTileM = 128;
constexpr int kTileN = 64;
constexpr int kChunkK = kPlaneChunk;  // one 64-byte swizzle atom of BF16
constexpr int kStages = 2;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kABytes = kTileM * kChunkK * 2;  // 8 KB per digit plane
constexpr uint32_t kBBytes = kTileN * kChunkK * 2;  // 4 KB per digit plane
constexpr uint32_t kStageBytes = kSlices * (kABytes + kBBytes);
constexpr size_t kSmemBytes = kStages * kStageBytes + 1024;  // + alignment slack for the swizzle base
constexpr long long kWaitCycles = 2000000000ll;    // ~1 s at 2 GHz

struct TcJob {
  int sys, l, row0, n0;
};

struct TcArgs {  // per (system, direction)
  CUtensorMap mapA;
  CUtensorMap mapB;
  double *C;
  const int *rowexp;
  const int *colexp;
  const int *c2f;   // compact row -> row of the contracted window (rows with overlap only)
  int rows_full;    // rows of the contracted window, Jc m0^2
  int rows, Kpad, Rt, m0;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Bounded wait on an mbarrier phase; also gives up once *ok (if given) drops to 0.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const int *ok) {
  const long long t0 = clock64();
  for (unsigned spin = 0;; ++spin) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((spin & 15u) == 15u && ok && *(volatile const int *)ok == 0) return false;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

// Shared-memory matrix descriptor: K-major tile of 64-byte rows, 64-byte swizzle, 8-row groups
// 512 bytes apart (start >> 4 in bits 0-13, leading offset 16 B (unused) in 16-29, stride 512 B
// in 32-45, descriptor version 1 in 46-48, swizzle mode 4 = 64B in 61-63).
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9, 10-12 = 1),
// both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

// x 2^e for an integer x, |x| < 2^63: x rounded to 53 bits (to nearest, ties to even) and scaled,
// the value of scale_pow2((double)x, e), formed with integer operations (on this GPU an FP64
// instruction costs a warp 16 cycles of the FP64 unit, whatever its active lanes); results outside
// the normal range take scale_pow2 itself.
__device__ __forceinline__ double int_times_pow2(long long x, int e) {
  if (x == 0) return 0.0;
  const unsigned long long sgn = x < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long u = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
  const int lz = __clzll(u);
  const unsigned long long m = u << lz;  // leading bit at 63
  unsigned long long mant = m >> 11;     // 53 bits
  const unsigned long long rem = m & 0x7ffull;
  int top = 63 - lz;  // exponent of the leading bit of x
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
    ++mant;
    if (mant == (1ull << 53)) {
      mant >>= 1;
      ++top;
    }
  }
  const int be = top + e + 1023;
  if (be < 1 || be > 2046) return scale_pow2((double)x, e);
  return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | (mant & ((1ull << 52) - 1))));
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(const TcJob *__restrict__ jobs, int njobs,
                                                           const TcArgs *__restrict__ args, unsigned *flags) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[kStages], bar_free[kStages], tmem_full, tmem_empty;
  __shared__ uint32_t tmem_slot;
  __shared__ int ok_sh;
  unsigned char *tiles =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t s0 = smem_u32(tiles);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    for (int st = 0; st < kStages; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_full[st])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_free[st])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tmem_full)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tmem_empty)), "r"(kEpiWarps) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    ok_sh = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    // ---- control (one thread): the loads run one chunk ahead of the MMAs, across tiles -------
    if (lane == 0) {
      // chunk cursor over this CTA's tiles (jobs blockIdx.x, blockIdx.x + gridDim.x, ..)
      struct Cur {
        int job, ch, nch;
      };
      auto first = [&](int job) {
        return Cur{job, 0, job < njobs ? args[jobs[job].sys * 3 + jobs[job].l].Kpad / kChunkK : 0};
      };
      auto next = [&](Cur c) { return ++c.ch < c.nch ? c : first(c.job + (int)gridDim.x); };
      // global chunk g uses stage g % 2 for the (g / 2)-th time: its barriers complete with parity
      // (g / 2) & 1
      auto load = [&](const Cur &c, int g) {
        const TcJob jb = jobs[c.job];
        const TcArgs &P = args[jb.sys * 3 + jb.l];
        if (c.ch == 0) {
          asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.mapA)) : "memory");
          asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.mapB)) : "memory");
        }
        const int st = g & 1;
        const uint32_t sA = s0 + st * kStageBytes, sB = sA + kSlices * kABytes, bf = smem_u32(&bar_full[st]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bf), "r"(kStageBytes) : "memory");
        // chunk-major planes: rows (k * nchunks + ch) * rows + row0 .. of a 32-wide 2D view
        for (int a = 0; a < kSlices; ++a)
          tma_load_2d(sA + a * kABytes, &P.mapA, 0, (a * c.nch + c.ch) * P.rows + jb.row0, bf);
        for (int b = 0; b < kSlices; ++b)
          tma_load_2d(sB + b * kBBytes, &P.mapB, 0, (b * c.nch + c.ch) * P.Rt + jb.n0, bf);
      };
      bool ok = true;
      int last_commit = -1, last_load = -1, last_arrived = -1, ntile = 0;
      Cur cur = first(blockIdx.x), ahead = cur;
      if (cur.nch > 0) {
        load(cur, 0);
        last_load = 0;
      }
      for (int g = 0; cur.nch > 0 && ok; ++g) {
        const int st = g & 1;
        ahead = next(ahead);
        if (ahead.nch > 0) {
          // stage (g + 1) % 2 is free once the MMAs of chunk g - 1 are done
          if (g >= 1 && !mbar_wait(smem_u32(&bar_free[st ^ 1]), ((g - 1) >> 1) & 1, &ok_sh)) {
            ok = false;
            break;
          }
          load(ahead, g + 1);
          last_load = g + 1;
        }
        if (!mbar_wait(smem_u32(&bar_full[st]), (g >> 1) & 1, &ok_sh)) {
          ok = false;
          break;
        }
        last_arrived = g;
        // a tile's first MMAs overwrite the accumulators: the previous tile's epilogue must be done
        if (cur.ch == 0 && ntile > 0 && !mbar_wait(smem_u32(&tmem_empty), (ntile - 1) & 1, &ok_sh)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // digit plane a of A against the B planes b0 .. b0 + nb - 1 (consecutive 64-row tiles in
        // shared memory: one B operand of N = 64 nb rows) lands in the accumulators of the
        // diagonals a + b0 .. a + b0 + nb - 1 (consecutive 64-column TMEM ranges): the 28 pairs
        // a + b <= 6 as 10 MMAs of N <= 256 per K step (a = 0 first: it initialises every
        // diagonal)
        const uint32_t sA = s0 + st * kStageBytes, sB = sA + kSlices * kABytes;
        for (int kk = 0; kk < kChunkK / 16; ++kk)
          for (int a = 0; a < kSlices; ++a)
            for (int b0 = 0; b0 < kSlices - a; b0 += 4) {
              const int nb = min(4, kSlices - a - b0);
              const uint64_t ad = sw64_desc(sA + a * kABytes + kk * 32);
              const uint64_t bd = sw64_desc(sB + b0 * kBBytes + kk * 32);
              mma_bf16(tmem + (uint32_t)((a + b0) * kTileN), ad, bd, idesc_n(nb * kTileN),
                       (cur.ch > 0 || a > 0 || kk > 0) ? 1u : 0u);
            }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&bar_free[st]))
                     : "memory");
        last_commit = g;
        if (cur.ch == cur.nch - 1) {
          // the tile's accumulators are complete once these MMAs are
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           smem_u32(&tmem_full))
                       : "memory");
          ++ntile;
        }
        cur = next(cur);
      }
      if (!ok) {
        atomicOr(flags, kFlagTimeout);
        ok_sh = 0;
        // bounded: the MMAs and loads still in flight complete before the CTA exits
        if (last_commit >= 0) mbar_wait(smem_u32(&bar_free[last_commit & 1]), (last_commit >> 1) & 1, nullptr);
        for (int g = last_arrived + 1; g <= last_load; ++g)
          mbar_wait(smem_u32(&bar_full[g & 1]), (g >> 1) & 1, nullptr);
      }
    }
  } else {
    // ---- epilogue warps 1 .. 8: TMEM lanes 32 quad .. 32 quad + 31, one half of the columns ----
    const int quad = warp & 3, half = (warp - 1) >> 2;
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    int ntile = 0;
    for (int job = blockIdx.x; job < njobs; job += gridDim.x, ++ntile) {
      bool ready = false;
      if (lane == 0) ready = mbar_wait(smem_u32(&tmem_full), ntile & 1, &ok_sh);
      if (!__shfl_sync(0xffffffffu, ready ? 1 : 0, 0)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const TcJob jb = jobs[job];
      const TcArgs &P = args[jb.sys * 3 + jb.l];
      const int row = jb.row0 + quad * 32 + lane;  // compact row
      const int mm = P.m0 * P.m0;
      const int er = row < P.rows ? P.rowexp[row] : 0;
      int frow = row < P.rows ? P.c2f[row] : -1;
      if (frow < 0 || frow >= P.rows_full) frow = -1;  // (a map entry out of range writes nothing)
      double *Crow = P.C + (int64_t)(frow < 0 ? 0 : frow / mm) * (P.Rt + 2) * mm + (frow < 0 ? 0 : frow % mm);
      for (int cc = half * (kTileN / 32); cc < (half + 1) * (kTileN / 32); ++cc) {
        uint32_t v[kSlices][16];
#pragma unroll
        for (int s = 0; s < kSlices; ++s) tmem_ld16(tmem + lane_base + (uint32_t)(s * kTileN + cc * 16), v[s]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (cc == (half + 1) * (kTileN / 32) - 1) {
          // every read of this warp's accumulators is done: the next tile's MMAs may start
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tmem_empty)) : "memory");
        }
        if (frow >= 0) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int n = jb.n0 + cc * 16 + t;
            if (n >= P.Rt) continue;
            // D_s are integers below 2^24 held exactly in FP32: converted to int32 and combined in
            // 64-bit integers, hi < 2^39 (weights 2^-14 .. 2^-28) and lo < 2^46 (2^-35 .. 2^-56),
            // then T = hi 2^24 + round(lo / 16) (< 2^63; the rounding, 2^-53 of the scale 2^E, is
            // far below the 2^-48 truncation of the dropped digit pairs) converted and scaled once
            long long d[kSlices];
#pragma unroll
            for (int s = 0; s < kSlices; ++s) d[s] = (long long)__float2int_rn(__uint_as_float(v[s][t]));
            const long long hi = (d[0] << 14) + (d[1] << 7) + d[2];
            const long long lo = (d[3] << 21) + (d[4] << 14) + (d[5] << 7) + d[6];
            const long long T = (hi << 24) + ((lo + 8) >> 4);
            const int E = er + P.colexp[n];
            Crow[(int64_t)n * mm] = int_times_pow2(T, E - 52);
          }
        }
      }
    }
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ---- host side ---------------------------------------------------------------------------

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// The chunk-major planes [kSlices][K / 32][rows][32] as a 2D tensor of 32-wide rows: a box of
// box_rows rows at y = (k K / 32 + ch) rows + row0 is one contiguous block.
bool encode_planes(CUtensorMap *map, void *base, int K, int rows, int box_rows) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)kPlaneChunk, (cuuint64_t)kSlices * (K / kPlaneChunk) * rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kPlaneChunk * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kChunkK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

size_t gram_tc_args_bytes(const SysDev *host_sys, int nsys) {
  size_t jobs = 0;
  for (int i = 0; i < nsys; ++i)
    for (int l = 0; l < 3; ++l) {
      const DirDev &D = host_sys[i].d[l];
      const size_t rows = (size_t)D.rows_c;
      jobs += ((rows + kTileM - 1) / kTileM) * ((host_sys[i].Rt + kTileN - 1) / kTileN);
    }
  return (size_t)nsys * 3 * sizeof(TcArgs) + jobs * sizeof(TcJob) + 256;
}

cudaError_t gram_tc_prepare(const SysDev *host_sys, int nsys, void *host_buf, size_t host_bytes, int *njobs,
                            size_t *jobs_off) {
  std::vector<TcArgs> args((size_t)nsys * 3);
  std::vector<TcJob> jobs;
  memset(args.data(), 0, args.size() * sizeof(TcArgs));
  for (int i = 0; i < nsys; ++i) {
    const SysDev &s = host_sys[i];
    for (int l = 0; l < 3; ++l) {
      const DirDev &D = s.d[l];
      // the rows with overlap of the contracted window blocks cw0 .. cw0 + Jc - 1 (the others'
      // factors are zeros, written by k_gram_slice)
      const int rows = D.rows_c;
      if (D.Jc < 1) return cudaErrorNotSupported;
      if (rows < 1) continue;
      if (D.Kpad % kChunkK != 0 || D.Kpad > 448) return cudaErrorNotSupported;
      TcArgs &a = args[(size_t)i * 3 + l];
      if (!encode_planes(&a.mapA, s.ws + D.offA, D.Kpad, rows, kTileM) ||
          !encode_planes(&a.mapB, s.ws + D.offB, D.Kpad, s.Rt, kTileN))
        return cudaErrorInvalidValue;
      a.C = s.ws + D.offC + (size_t)D.cw0 * (s.Rt + 2) * s.m0 * s.m0;
      a.rowexp = reinterpret_cast<const int *>(s.ws + D.offRE);
      a.colexp = reinterpret_cast<const int *>(s.ws + D.offCE);
      a.c2f = reinterpret_cast<const int *>(s.ws + D.offRM) + (size_t)D.Jc * s.m0 * s.m0;
      a.rows_full = D.Jc * s.m0 * s.m0;
      a.rows = rows;
      a.Kpad = D.Kpad;
      a.Rt = s.Rt;
      a.m0 = s.m0;
      for (int r0 = 0; r0 < rows; r0 += kTileM)
        for (int n0 = 0; n0 < s.Rt; n0 += kTileN) jobs.push_back({i, l, r0, n0});
    }
  }
  const size_t abytes = args.size() * sizeof(TcArgs);
  const size_t need = abytes + jobs.size() * sizeof(TcJob);
  if (need > host_bytes) return cudaErrorMemoryAllocation;
  unsigned char *h = static_cast<unsigned char *>(host_buf);
  memcpy(h, args.data(), abytes);
  memcpy(h + abytes, jobs.data(), jobs.size() * sizeof(TcJob));
  *njobs = (int)jobs.size();
  *jobs_off = abytes;
  return cudaSuccess;
}

cudaError_t gram_tc_launch(const void *dev_buf, int njobs, size_t jobs_off, unsigned *flags, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e != cudaSuccess) return e;
  // persistent: one CTA per SM (shared memory and TMEM admit one), each taking every
  // gridDim.x-th job
  int dev = 0, nsm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min(njobs, nsm));
  const unsigned char *d = static_cast<const unsigned char *>(dev_buf);
  kmark(LHF_K_GRAM_TC, 1, st);
  k_gram_tc<<<(unsigned)grid, kTcThreads, kSmemBytes, st>>>(reinterpret_cast<const TcJob *>(d + jobs_off), njobs,
                                                            reinterpret_cast<const TcArgs *>(d), flags);
  kmark(LHF_K_GRAM_TC, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_gram_tc_impl(const SysDev *host_sys, int nsys, void *dev_buf, size_t dev_bytes,
                                void *host_buf, size_t host_bytes, unsigned *flags, cudaStream_t st) {
  int njobs = 0;
  size_t jobs_off = 0;
  cudaError_t e = gram_tc_prepare(host_sys, nsys, host_buf, host_bytes, &njobs, &jobs_off);
  if (e != cudaSuccess) return e;
  const size_t need = jobs_off + (size_t)njobs * sizeof(TcJob);
  if (need > dev_bytes) return cudaErrorMemoryAllocation;
  // host_buf is pinned and owned by the caller: it must stay untouched until the copy has run
  e = cudaMemcpyAsync(dev_buf, host_buf, need, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return gram_tc_launch(dev_buf, njobs, jobs_off, flags, st);
}

}  // namespace lhf
