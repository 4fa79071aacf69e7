// k_eig.cu -- step a8: generalized Hermitian eigenvalues at every k-point, one warp per matrix.
//
// Hbar_kappa u = lambda Sbar_kappa u (eq. (4.7)); the spectrum of the lattice matrix is the
// union over kappa (Prop. 6.1, eq. (6.7)).  Per k-point, in FP64 and in shared memory:
//   1. Cholesky Sbar = L L^H                      (column by column, lanes over rows)
//   2. C = L^{-1} Hbar L^{-H}                      (two forward substitutions, lanes over columns;
//                                                  C^H = L^{-1} (L^{-1} Hbar)^H and C = C^H)
//   3. cyclic complex Jacobi on C: sweeps of m-1 steps; each step applies m/2 disjoint plane
//      rotations at once (round-robin ordering), first to columns, then to rows.  The rotation
//      for the pair (p, q) with C_pq = |g| e^{i phi} is J = [[c, s e^{i phi}], [-s e^{-i phi}, c]]
//      with t = s/c the smaller root of t^2 + 2 tau t - 1 = 0, tau = (C_qq - C_pp) / (2 |g|);
//      it zeroes C_pq.  Sweeps stop when the off-diagonal Frobenius norm is below 1e-16 of the
//      total.
//   4. eigenvalues = diag(C), sorted ascending by a warp bitonic sort.
// Real blocks give Hbar_{-kappa} = conj(Hbar_kappa): only one k-point of each conjugate pair is
// solved and its eigenvalues are written to both.
#include <math.h>

#include "lhf_internal.cuh"

namespace lhf {
namespace {

constexpr int kEigWarps = 4;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // a * conj(b)
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

__host__ __device__ inline size_t eig_warp_bytes(int m) {
  return (size_t)2 * m * m * sizeof(double2) + 16 * (3 * sizeof(double) + 2 * sizeof(int));
}

__global__ void __launch_bounds__(kEigWarps * 32) k_eig(const SysDev *__restrict__ sysv,
                                                        unsigned *flags, unsigned long long *counters,
                                                        int max_m0) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kap = blockIdx.x * kEigWarps + warp;
  if (kap >= s.nblocks) return;
  const int L0 = s.d[0].L, L1 = s.d[1].L, L2 = s.d[2].L;
  const int k0 = kap / (L1 * L2), k1 = (kap / L2) % L1, k2 = kap % L2;
  const int mk = (((L0 - k0) % L0) * L1 + (L1 - k1) % L1) * L2 + (L2 - k2) % L2;
  if (mk < kap) return;  // the conjugate partner solves this pair
  const int m = s.m0, mm = m * m;
  extern __shared__ unsigned char smraw[];
  unsigned char *base = smraw + (size_t)warp * eig_warp_bytes(max_m0);
  double2 *A = reinterpret_cast<double2 *>(base);
  double2 *B = A + mm;
  double *rc = reinterpret_cast<double *>(B + mm);
  double *rsr = rc + 16, *rsi = rsr + 16;
  int *rp = reinterpret_cast<int *>(rsi + 16), *rq = rp + 16;

  const double2 *Hb = reinterpret_cast<const double2 *>(s.Hbar) + (int64_t)kap * mm;
  const double2 *Sb = reinterpret_cast<const double2 *>(s.Sbar) + (int64_t)kap * mm;
  for (int e = lane; e < mm; e += 32) {
    A[e] = Hb[e];
    B[e] = Sb[e];
  }
  __syncwarp();

  // 1. Cholesky of Sbar (lower triangle, in place in B)
  bool ok = true;
  for (int j = 0; j < m; ++j) {
    if (lane == 0) {
      double d = B[j * m + j].x;
      for (int k = 0; k < j; ++k) {
        const double2 v = B[j * m + k];
        d -= v.x * v.x + v.y * v.y;
      }
      B[j * m + j] = make_double2(d > 0.0 ? sqrt(d) : -1.0, 0.0);
    }
    __syncwarp();
    const double dj = B[j * m + j].x;
    if (!(dj > 0.0)) {
      ok = false;
      break;
    }
    const double inv = 1.0 / dj;
    for (int i = j + 1 + lane; i < m; i += 32) {
      double2 v = B[i * m + j];
      for (int k = 0; k < j; ++k) v = csub(v, cmulc(B[i * m + k], B[j * m + k]));
      B[i * m + j] = cscale(v, inv);
    }
    __syncwarp();
  }

  if (ok) {
    // 2. C = L^{-1} Hbar L^{-H}
    for (int pass = 0; pass < 2; ++pass) {
      for (int c = lane; c < m; c += 32) {
        for (int i = 0; i < m; ++i) {
          double2 v = A[i * m + c];
          for (int k = 0; k < i; ++k) v = csub(v, cmul(B[i * m + k], A[k * m + c]));
          A[i * m + c] = cscale(v, 1.0 / B[i * m + i].x);
        }
      }
      __syncwarp();
      if (pass == 0) {  // A <- A^H
        for (int e = lane; e < mm; e += 32) {
          const int i = e / m, j = e - (e / m) * m;
          if (i < j) {
            const double2 x = A[i * m + j], y = A[j * m + i];
            A[i * m + j] = make_double2(y.x, -y.y);
            A[j * m + i] = make_double2(x.x, -x.y);
          } else if (i == j) {
            A[e].y = -A[e].y;
          }
        }
        __syncwarp();
      }
    }
    for (int e = lane; e < mm; e += 32) {  // Hermitian part of the rounding
      const int i = e / m, j = e - (e / m) * m;
      if (i < j) {
        const double2 x = A[i * m + j], y = A[j * m + i];
        const double2 a = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
        A[i * m + j] = a;
        A[j * m + i] = make_double2(a.x, -a.y);
      } else if (i == j) {
        A[e].y = 0.0;
      }
    }
    __syncwarp();

    // 3. cyclic Jacobi, round-robin parallel ordering
    const int mp = m + (m & 1), npair = mp / 2;
    int sweep = 0;
    for (; sweep < 40; ++sweep) {
      double off = 0.0, tot = 0.0;
      for (int e = lane; e < mm; e += 32) {
        const double v = A[e].x * A[e].x + A[e].y * A[e].y;
        tot += v;
        if (e / m != e - (e / m) * m) off += v;
      }
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
      }
      if (off <= 1e-32 * tot) break;
      for (int step = 0; step < mp - 1; ++step) {
        if (lane < npair) {
          const int pa = lane, pb = mp - 1 - lane;
          int p = pa == 0 ? 0 : ((pa - 1 + step) % (mp - 1)) + 1;
          int q = pb == 0 ? 0 : ((pb - 1 + step) % (mp - 1)) + 1;
          if (p > q) {
            const int t = p;
            p = q;
            q = t;
          }
          double c = 1.0, sr = 0.0, si = 0.0;
          if (q < m) {
            const double2 g = A[p * m + q];
            const double ag = hypot(g.x, g.y);
            const double app = A[p * m + p].x, aqq = A[q * m + q].x;
            if (ag > 1e-300 && ag > 1e-18 * sqrt(fabs(app * aqq))) {
              const double tau = (aqq - app) / (2.0 * ag);
              const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
              c = 1.0 / sqrt(1.0 + t * t);
              const double sn = t * c;
              sr = sn * g.x / ag;
              si = sn * g.y / ag;
            }
          }
          rp[lane] = p;
          rq[lane] = q;
          rc[lane] = c;
          rsr[lane] = sr;
          rsi[lane] = si;
        }
        __syncwarp();
        const int work = npair * m;
        for (int it = lane; it < work; it += 32) {  // columns: A <- A J
          const int k = it / m, r = it - (it / m) * m;
          const int p = rp[k], q = rq[k];
          if (q >= m || (rsr[k] == 0.0 && rsi[k] == 0.0)) continue;
          const double c = rc[k];
          const double2 se = make_double2(rsr[k], rsi[k]), sec = make_double2(rsr[k], -rsi[k]);
          const double2 x = A[r * m + p], y = A[r * m + q];
          const double2 sy = cmul(sec, y), sx = cmul(se, x);
          A[r * m + p] = make_double2(c * x.x - sy.x, c * x.y - sy.y);
          A[r * m + q] = make_double2(sx.x + c * y.x, sx.y + c * y.y);
        }
        __syncwarp();
        for (int it = lane; it < work; it += 32) {  // rows: A <- J^H A
          const int k = it / m, r = it - (it / m) * m;
          const int p = rp[k], q = rq[k];
          if (q >= m || (rsr[k] == 0.0 && rsi[k] == 0.0)) continue;
          const double c = rc[k];
          const double2 se = make_double2(rsr[k], rsi[k]), sec = make_double2(rsr[k], -rsi[k]);
          const double2 x = A[p * m + r], y = A[q * m + r];
          const double2 sy = cmul(se, y), sx = cmul(sec, x);
          A[p * m + r] = make_double2(c * x.x - sy.x, c * x.y - sy.y);
          A[q * m + r] = make_double2(sx.x + c * y.x, sx.y + c * y.y);
        }
        __syncwarp();
        if (lane < npair && rq[lane] < m && !(rsr[lane] == 0.0 && rsi[lane] == 0.0)) {
          A[rp[lane] * m + rq[lane]] = make_double2(0.0, 0.0);
          A[rq[lane] * m + rp[lane]] = make_double2(0.0, 0.0);
        }
        __syncwarp();
      }
    }
    if (lane == 0 && counters) {
      atomicAdd(counters, (unsigned long long)sweep);
      atomicAdd(counters + 1, 1ull);
    }
  }

  // 4. sort and store
  double v = (ok && lane < m) ? A[lane * m + lane].x : INFINITY;
  for (int k = 2; k <= 32; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      const double o = __shfl_xor_sync(0xffffffffu, v, j);
      const bool up = (lane & k) == 0, lower = (lane & j) == 0;
      v = (lower == up) ? fmin(v, o) : fmax(v, o);
    }
  if (!ok) v = NAN;
  if (lane < m) {
    s.eig[(int64_t)kap * m + lane] = v;
    s.eig[(int64_t)mk * m + lane] = v;
  }
  if (lane == 0) {
    if (s.kstat) {
      s.kstat[kap] = ok ? 0 : (int)LHF_ERR_NOT_SPD;
      s.kstat[mk] = ok ? 0 : (int)LHF_ERR_NOT_SPD;
    }
    if (!ok) atomicOr(flags, kFlagNotSpd);
  }
}

}  // namespace

cudaError_t launch_eig(const SysDev *sys, int nsys, int max_k, int max_m0, unsigned *flags,
                       unsigned long long *counters, cudaStream_t st) {
  if (max_k <= 0 || nsys <= 0) return cudaSuccess;
  const size_t smem = kEigWarps * eig_warp_bytes(max_m0);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((max_k + kEigWarps - 1) / kEigWarps, nsys);
  k_eig<<<grid, kEigWarps * 32, smem, st>>>(sys, flags, counters, max_m0);
  return cudaGetLastError();
}

}  // namespace lhf
