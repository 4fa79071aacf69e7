// k_dense.cu -- step a9, eigensolve: generalized symmetric-definite eigenvalues H x = lambda S x
// of one dense N x N pencil (the open box of Table 4.1's full eigensolver), FP64.
//
// One cooperative launch (all CTAs resident); CTA b owns the rows i = b mod G of every work
// matrix and is the only CTA that writes them; rows of other CTAs are read with ld.global.cg
// (from L2, never from a stale L1 line) after a grid barrier.
//   0. diagonal scaling D = diag(S)^{-1/2}: S~ = D S D, H~ = D H D (same eigenvalues)
//   1. Cholesky S~ = L L^T, right-looking by columns: every CTA forms column j of L from the
//      updated matrix, then updates its own rows of the trailing part (one grid barrier per j).
//      Column j is read by every CTA during step j, so L is written where nobody reads it in
//      that step: the diagonal to a separate array, L_ij (i > j) to the upper triangle at (j, i)
//   2. Y = H~ L^{-T}: every row y solves y L^T = h by forward substitution (rows independent)
//   3. C = L^{-1} H~ L^{-T} = Y^T L^{-T}: the own rows of Y^T, then step 2 again; symmetrised
//   4. Householder tridiagonalisation C = Q T Q^T: for column k every CTA forms v from
//      C[k+1:, k] (alpha = -sign(x0) |x|, v = x - alpha e1, tau = 1 / (|x|^2 - alpha x0)),
//      p = tau C v on its own rows, w = p - (tau/2)(p.v) v, C <- C - v w^T - w v^T on its own
//      rows (two grid barriers per column); T = tridiag(te, td, te)
//   5. eigenvalue t of T by multisection on the Sturm count (the number of negative pivots of
//      the LDL^T factorisation of T - sigma I equals the number of eigenvalues below sigma):
//      8 lanes evaluate 8 equally spaced sigmas per round, 18 rounds shrink the Gershgorin
//      interval by 9^18.  Eigenvalues come out ascending by construction.
// The grid barrier is a counter and a generation word in global memory with a bounded wait: a
// CTA that waits longer than wait_cycles SM clock cycles (default 2e9, about a second) raises
// kFlagTimeout and an abort word that makes every CTA return.  The barrier completes when
// `arrivals` CTAs have arrived: gridDim.x, or one more for the failure-detection test, whose
// waits then run out.
#include <math.h>

#include "lhf_internal.cuh"

namespace lhf {
namespace {

constexpr int kDenseThreads = 256;
constexpr int kSturmLanes = 8;   // sigmas per eigenvalue and round
constexpr int kSturmRounds = 18; // interval shrinks by (kSturmLanes + 1)^kSturmRounds

struct GridBar {
  unsigned count;
  unsigned gen;
  unsigned abort;
  unsigned bad;  // non-positive pivot seen
};

// Bounded grid-wide barrier; returns false if it (or another CTA's barrier) gave up.
__device__ bool grid_barrier(GridBar *bar, unsigned nblocks, unsigned *flags, int *ok_sh, long long wait_cycles) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = atomicAdd(&bar->gen, 0u);
    __threadfence();
    if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const long long t0 = clock64();
      unsigned spins = 0;
      // poll with plain volatile loads (atomics on the word would contend with the arrivals)
      const volatile unsigned *gen = &bar->gen;
      const volatile unsigned *abort_word = &bar->abort;
      while (*gen == g) {
        if ((++spins & 255u) == 0 && (clock64() - t0 > wait_cycles || *abort_word)) {
          atomicOr(flags, kFlagTimeout);
          atomicExch(&bar->abort, 1u);
          ok = 0;
          break;
        }
        __nanosleep(20);
      }
    }
    if (atomicAdd(&bar->abort, 0u)) ok = 0;
    __threadfence();
    *ok_sh = ok;
  }
  __syncthreads();
  return *ok_sh != 0;
}

// Block-wide sum (fixed order: per-warp shuffle tree, then one warp over the partials).
__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < kDenseThreads / 32 ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// The own rows x of X become x L^{-T} (solve L z = x^T by forward substitution, right-looking
// over k with one __syncthreads per k).  L_mk (m > k) is read from the strict upper triangle of
// Lt (row k, contiguous in m), L_kk from ld; both from L2.
__device__ void rows_times_inv_lt(double *X, const double *Lt, const double *ld, int N, int G) {
  for (int k = 0; k < N; ++k) {
    const double lkk = __ldcg(ld + k);
    if (threadIdx.x == 0)
      for (int i = blockIdx.x; i < N; i += G) X[(int64_t)i * N + k] /= lkk;
    __syncthreads();
    const double *lrow = Lt + (int64_t)k * N;
    for (int i = blockIdx.x; i < N; i += G) {
      double *row = X + (int64_t)i * N;
      const double zk = row[k];
      for (int m = k + 1 + threadIdx.x; m < N; m += kDenseThreads) row[m] -= __ldcg(lrow + m) * zk;
    }
    __syncthreads();
  }
}

// Number of eigenvalues of T = tridiag(e, d, e) below sigma: the sign changes of the Sturm
// sequence of leading principal minors p_i = (d_i - sigma) p_(i-1) - e_(i-1)^2 p_(i-2), p_0 = 1
// (a sign change where p_i / p_(i-1) < 0, the LDL^T pivot of T - sigma I), without divisions; the
// pair (p_(i-1), p_i) is rescaled by an exact power of two when it leaves [2^-500, 2^500], and an
// exact zero takes the sign that counts it (the pivot -0 of the LDL^T form).
__device__ int sturm_count(const double *td, const double *te2, int N, double sigma) {
  int cnt = 0;
  double p0 = 1.0, p1 = __ldcg(td) - sigma;
  if (p1 == 0.0) p1 = -1e-300;
  cnt += p1 < 0.0;
  for (int i = 1; i < N; ++i) {
    double p2 = fma(__ldcg(td + i) - sigma, p1, -__ldcg(te2 + i - 1) * p0);
    if (p2 == 0.0) p2 = p1 > 0.0 ? -1e-300 : 1e-300;
    cnt += (p2 < 0.0) != (p1 < 0.0);
    p0 = p1;
    p1 = p2;
    const double a = fabs(p1);
    if (a > 0x1p500) {
      p0 *= 0x1p-500;
      p1 *= 0x1p-500;
    } else if (a < 0x1p-500 && fabs(p0) < 0x1p-500) {
      p0 *= 0x1p500;
      p1 *= 0x1p500;
    }
  }
  return cnt;
}

__global__ void __launch_bounds__(kDenseThreads) k_dense_eig(const double *__restrict__ H,
                                                            const double *__restrict__ S, int N,
                                                            double *eig, double *work, GridBar *bar,
                                                            unsigned *flags, long long wait_cycles,
                                                            unsigned arrivals) {
  extern __shared__ double sm[];
  double *vec = sm;      // [N] scales, column of L, Householder vector
  double *wv = sm + N;   // [N] w
  __shared__ double red[33];
  __shared__ int ok_sh;
  const int G = gridDim.x, tid = threadIdx.x;
  const int64_t NN = (int64_t)N * N;
  double *Lm = work;            // [N][N] scaled S (lower triangle updated), L^T (strict upper)
  double *C = work + NN;        // [N][N] scaled H, then Y, then C
  double *Yt = work + 2 * NN;   // [N][N] Y^T, then C before symmetrisation
  double *pv = work + 3 * NN;   // [N] p of the current Householder step
  double *td = pv + N;          // [N] diagonal of T
  double *te = td + N;          // [N] off-diagonal of T (te[k] = T[k+1][k])
  double *te2 = te + N;         // [N] te^2
  double *ld = te2 + N;         // [N] diagonal of L
  bool bad = false;

  // 0. scaling (every CTA forms all scales; each writes its own rows)
  for (int i = tid; i < N; i += kDenseThreads) {
    const double sii = S[(int64_t)i * N + i];
    vec[i] = sii > 0.0 ? 1.0 / sqrt(sii) : 0.0;
    if (!(sii > 0.0)) bar->bad = 1u;
  }
  __syncthreads();
  for (int i = blockIdx.x; i < N; i += G)
    for (int j = tid; j < N; j += kDenseThreads) {
      const double sc = vec[i] * vec[j];
      Lm[(int64_t)i * N + j] = S[(int64_t)i * N + j] * sc;
      C[(int64_t)i * N + j] = H[(int64_t)i * N + j] * sc;
    }
  if (!grid_barrier(bar, arrivals, flags, &ok_sh, wait_cycles)) return;
  bad = __ldcg(&bar->bad) != 0u;

  // 1. Cholesky (lower triangle of Lm)
  for (int j = 0; j < N && !bad; ++j) {
    const double ajj = __ldcg(Lm + (int64_t)j * N + j);
    if (!(ajj > 0.0)) {  // every CTA reads the same pivot and stops here
      bad = true;
      break;
    }
    const double ljj = sqrt(ajj), inv = 1.0 / ljj;
    for (int k = j + 1 + tid; k < N; k += kDenseThreads) vec[k] = __ldcg(Lm + (int64_t)k * N + j) * inv;
    __syncthreads();
    for (int i = blockIdx.x; i < N; i += G) {
      if (i < j) continue;
      double *row = Lm + (int64_t)i * N;
      if (i == j) {  // row j: L_jj and L_kj (k > j) into the strict upper part of row j
        if (tid == 0) ld[j] = ljj;
        for (int k = j + 1 + tid; k < N; k += kDenseThreads) row[k] = vec[k];
        continue;
      }
      const double li = vec[i];
      for (int k = j + 1 + tid; k <= i; k += kDenseThreads) row[k] -= li * vec[k];
    }
    if (!grid_barrier(bar, arrivals, flags, &ok_sh, wait_cycles)) return;
  }
  if (bad) {
    if (blockIdx.x == 0 && tid == 0) atomicOr(flags, kFlagNotSpd);
    for (int t = blockIdx.x * kDenseThreads + tid; t < N; t += G * kDenseThreads) eig[t] = NAN;
    return;
  }

  // 2. Y = H~ L^{-T} on the own rows of C
  rows_times_inv_lt(C, Lm, ld, N, G);
  if (!grid_barrier(bar, arrivals, flags, &ok_sh, wait_cycles)) return;
  // 3. own rows of Y^T, times L^{-T}, then C = (X + X^T) / 2 on the own rows
  for (int i = blockIdx.x; i < N; i += G)
    for (int j = tid; j < N; j += kDenseThreads) Yt[(int64_t)i * N + j] = __ldcg(C + (int64_t)j * N + i);
  __syncthreads();
  rows_times_inv_lt(Yt, Lm, ld, N, G);
  if (!grid_barrier(bar, arrivals, flags, &ok_sh, wait_cycles)) return;
  for (int i = blockIdx.x; i < N; i += G)
    for (int j = tid; j < N; j += kDenseThreads)
      C[(int64_t)i * N + j] = 0.5 * (Yt[(int64_t)i * N + j] + __ldcg(Yt + (int64_t)j * N + i));
  if (!grid_barrier(bar, arrivals, flags, &ok_sh, wait_cycles)) return;

  // 4. Householder tridiagonalisation of C
  for (int k = 0; k + 2 < N; ++k) {
    double part = 0.0;
    for (int i = k + 1 + tid; i < N; i += kDenseThreads) {
      const double x = __ldcg(C + (int64_t)i * N + k);
      vec[i] = x;
      part += x * x;
    }
    const double sig = block_sum(part, red);  // synchronises: vec is complete
    const double x0 = vec[k + 1];
    const double alpha = sig > 0.0 ? (x0 >= 0.0 ? -sqrt(sig) : sqrt(sig)) : 0.0;
    const double tau = sig > 0.0 ? 1.0 / (sig - alpha * x0) : 0.0;
    __syncthreads();
    if (tid == 0) vec[k + 1] = x0 - alpha;
    if (blockIdx.x == 0 && tid == 0) {
      td[k] = __ldcg(C + (int64_t)k * N + k);
      te[k] = sig > 0.0 ? alpha : x0;
    }
    __syncthreads();
    if (tau != 0.0) {
      // p = tau C v on the own rows, one warp per row (shuffle reduction, no block barrier)
      const int warp = tid >> 5, lane = tid & 31;
      for (int q = warp; blockIdx.x + (int64_t)q * G < N; q += kDenseThreads / 32) {
        const int i = blockIdx.x + q * G;
        if (i <= k) continue;
        const double *row = C + (int64_t)i * N;
        double acc = 0.0;
        for (int j = k + 1 + lane; j < N; j += 32) acc += row[j] * vec[j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) pv[i] = tau * acc;
      }
    }
    if (!grid_barrier(bar, arrivals, flags, &ok_sh, wait_cycles)) return;
    if (tau != 0.0) {
      double pd = 0.0;
      for (int i = k + 1 + tid; i < N; i += kDenseThreads) {
        const double p = __ldcg(pv + i);
        wv[i] = p;
        pd += p * vec[i];
      }
      const double Kf = 0.5 * tau * block_sum(pd, red);
      for (int i = k + 1 + tid; i < N; i += kDenseThreads) wv[i] -= Kf * vec[i];
      __syncthreads();
      for (int i = blockIdx.x; i < N; i += G) {  // C <- C - v w^T - w v^T, own rows
        if (i <= k) continue;
        double *row = C + (int64_t)i * N;
        const double vi = vec[i], wi = wv[i];
        for (int j = k + 1 + tid; j < N; j += kDenseThreads) row[j] -= vi * wv[j] + wi * vec[j];
      }
    }
    if (!grid_barrier(bar, arrivals, flags, &ok_sh, wait_cycles)) return;
  }
  if (blockIdx.x == 0 && tid == 0) {
    if (N >= 2) {
      td[N - 2] = __ldcg(C + (int64_t)(N - 2) * N + N - 2);
      te[N - 2] = __ldcg(C + (int64_t)(N - 1) * N + N - 2);
    }
    td[N - 1] = __ldcg(C + (int64_t)(N - 1) * N + N - 1);
    for (int i = 0; i + 1 < N; ++i) te2[i] = te[i] * te[i];
  }
  if (!grid_barrier(bar, arrivals, flags, &ok_sh, wait_cycles)) return;

  // 5. multisection on the Sturm count; every CTA forms the Gershgorin interval itself
  double glo = INFINITY, ghi = -INFINITY, emax2 = 0.0;
  for (int i = tid; i < N; i += kDenseThreads) {
    const double di = __ldcg(td + i);
    const double r = (i > 0 ? fabs(__ldcg(te + i - 1)) : 0.0) + (i + 1 < N ? fabs(__ldcg(te + i)) : 0.0);
    glo = fmin(glo, di - r);
    ghi = fmax(ghi, di + r);
    if (i + 1 < N) emax2 = fmax(emax2, __ldcg(te2 + i));
  }
  for (int o = 16; o > 0; o >>= 1) {
    glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
    emax2 = fmax(emax2, __shfl_xor_sync(0xffffffffu, emax2, o));
  }
  __syncthreads();
  if ((tid & 31) == 0) {
    red[tid >> 5] = glo;
    red[8 + (tid >> 5)] = ghi;
    red[16 + (tid >> 5)] = emax2;
  }
  __syncthreads();
  glo = red[0];
  ghi = red[8];
  emax2 = red[16];
  for (int w = 1; w < kDenseThreads / 32; ++w) {
    glo = fmin(glo, red[w]);
    ghi = fmax(ghi, red[8 + w]);
    emax2 = fmax(emax2, red[16 + w]);
  }
  const double span = fmax(fabs(glo), fabs(ghi));
  const double pivmin = 2.2250738585072014e-308 * fmax(1.0, emax2);
  glo -= 4.0 * 2.220446049250313e-16 * span + pivmin;
  ghi += 4.0 * 2.220446049250313e-16 * span + pivmin;
  // eigenvalue t per group of kSturmLanes lanes, spread over the CTAs: t = b + G u
  const int groups = kDenseThreads / kSturmLanes, grp = tid / kSturmLanes, gl = tid % kSturmLanes;
  const unsigned gmask = ((1u << kSturmLanes) - 1u) << ((tid & 31) / kSturmLanes * kSturmLanes);
  for (int u0 = 0; u0 * G < N; u0 += groups) {
    const int t = blockIdx.x + G * (u0 + grp);
    const bool live = t < N;
    double lo = glo, hi = ghi;
    for (int rd = 0; rd < kSturmRounds; ++rd) {
      const double step = (hi - lo) / (kSturmLanes + 1);
      const double sg = lo + (gl + 1) * step;
      const bool above = live && sturm_count(td, te2, N, sg) > t;  // lambda_t < sg
      const unsigned bal = __ballot_sync(0xffffffffu, above) & gmask;
      // first lane (of the group) whose sigma has lambda_t below it
      const int first = bal ? __ffs(bal) - 1 - (tid & 31) / kSturmLanes * kSturmLanes : kSturmLanes;
      const double nlo = first == 0 ? lo : lo + first * step;
      const double nhi = first == kSturmLanes ? hi : lo + (first + 1) * step;
      lo = nlo;
      hi = nhi;
    }
    if (live && gl == 0) eig[t] = 0.5 * (lo + hi);
  }
}

}  // namespace

size_t dense_eig_workspace_doubles(int N) { return (size_t)3 * N * N + 5 * (size_t)N + 64; }

cudaError_t launch_dense_eig(const double *H, const double *S, int N, double *eig, double *work,
                             unsigned *flags, cudaStream_t st, long long wait_cycles, int stall) {
  if (N <= 0) return cudaSuccess;
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
  if (!coop) return cudaErrorNotSupported;
  const size_t smem = (size_t)2 * N * sizeof(double);
  if (smem > 48 * 1024) {
    if ((e = cudaFuncSetAttribute(k_dense_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
  }
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_eig, kDenseThreads, smem)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorNotSupported;
  const int G = sms < N ? sms : N;  // one CTA per SM, all resident
  GridBar *bar = reinterpret_cast<GridBar *>(work + 3 * (size_t)N * N + 5 * (size_t)N);
  if ((e = cudaMemsetAsync(bar, 0, sizeof(GridBar), st)) != cudaSuccess) return e;
  if (wait_cycles <= 0) wait_cycles = kDefaultWaitCycles;
  unsigned arrivals = (unsigned)G + (stall ? 1u : 0u);
  void *args[] = {(void *)&H,    (void *)&S,     (void *)&N,           (void *)&eig,     (void *)&work,
                  (void *)&bar,  (void *)&flags, (void *)&wait_cycles, (void *)&arrivals};
  kmark(LHF_K_DENSE_EIG, 1, st);
  e = cudaLaunchCooperativeKernel((const void *)k_dense_eig, dim3(G), dim3(kDenseThreads), args, smem, st);
  kmark(LHF_K_DENSE_EIG, 0, st);
  return e;
}

}  // namespace lhf
