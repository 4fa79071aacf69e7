// k_eig.cu -- step a8: generalized Hermitian eigenvalues at every k-point, one warp per matrix.
//
// Hbar_kappa u = lambda Sbar_kappa u (eq. (4.7)); the spectrum of the lattice matrix is the
// union over kappa (Prop. 6.1, eq. (6.7)).  Per k-point, in FP64 and in shared memory:
//   0. functions whose overlap diagonal cancelled to rounding level (Re Sbar_ii <= tau s0_i,
//      s0_i the cell-periodic norm = mean over kappa of Re Sbar_ii) are numerically absent and
//      dropped; the kept m' x m' pencil is gathered and scaled by D = diag(Sbar)^{-1/2}
//   1. Cholesky S = L L^H                         (column by column, lanes over rows)
//   2. C = L^{-1} H L^{-H}                         (two forward substitutions, lanes over columns;
//                                                  C^H = L^{-1} (L^{-1} H)^H and C = C^H)
//      or, when a scaled pivot falls below kCholTol (near-linear dependence), canonical
//      orthogonalisation: Jacobi with vectors S = V diag(sigma) V^H, directions with sigma below
//      kLindepTol dropped, X = V_kept diag(sigma)^{-1/2}, C = X^H H X
//   3. cyclic complex Jacobi on C: sweeps of m'-1 steps; each step applies m'/2 disjoint plane
//      rotations at once (round-robin ordering) as 2x2 block updates R1^H X R2.  The rotation
//      for the pair (p, q) with C_pq = |g| e^{i phi} is J = [[c, s e^{i phi}], [-s e^{-i phi}, c]]
//      with t = s/c the smaller root of t^2 + 2 tau t - 1 = 0, tau = (C_qq - C_pp) / (2 |g|);
//      it zeroes C_pq.  Sweeps stop when the off-diagonal Frobenius norm is below 1e-16 of the
//      total.
//   4. eigenvalues = diag(C) and +inf for dropped functions/directions, sorted by a warp bitonic
//      sort.
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

// per warp: A, B, V (m^2 complex each), rotation table (16 x {c, sr, si, p, q}), kept index
// map, scales and overlap eigenvalues (32 each), and the (k1 < k2) pair-block table (120 x 2)
__host__ __device__ inline size_t eig_warp_bytes(int m) {
  return (size_t)3 * m * m * sizeof(double2) + 16 * (3 * sizeof(double) + 2 * sizeof(int)) +
         32 * (2 * sizeof(double) + 2 * sizeof(int)) + 288;
}

struct RotTab {
  double *c, *sr, *si;
  int *p, *q;
  const unsigned char *blk;  // [nblk][2] pair indices (k1, k2), k1 < k2
};

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }

// Cyclic Jacobi on the Hermitian m x m matrix A (shared memory, row-major), one warp.  Each sweep
// is m'-1 steps (m' = m rounded up to even) of m'/2 disjoint rotations (round-robin ordering);
// a step applies A <- J^H A J for the product J of its rotations.  R = [[c, s e^{i phi}],
// [-s e^{-i phi}, c]] with t = s / c the smaller root of t^2 + 2 tau t - 1 = 0,
// tau = (A_qq - A_pp) / (2 |A_pq|), zeroes A_pq; written with u = t / |A_pq| =
// 2 sign(d) / (|d| + sqrt(d^2 + 4 |A_pq|^2)), d = A_qq - A_pp, so that one square root, one
// division and one reciprocal square root give the rotation.  The lane of a pair updates its
// own diagonal block in closed form (A_pp - t |A_pq|, A_qq + t |A_pq|, zero off-diagonal); the
// blocks A[{p1,q1}, {p2,q2}] of two different pairs k1 < k2 are then updated as X <- R1^H X R2
// by one lane each, and the mirrored block written as the conjugate transpose.  With V
// non-null the rotations are also accumulated into V's columns (V <- V J).  Stops when the
// off-diagonal Frobenius norm falls below 1e-16 of the total.  Returns the sweeps.
__device__ int jacobi_herm(double2 *A, double2 *V, int m, int lane, const RotTab &R) {
  const int mm = m * m, mp = m + (m & 1), npair = mp / 2;
  const int nblk = npair * (npair - 1) / 2;
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
          const double a = A[p * m + p].x, b = A[q * m + q].x;
          const double ag2 = g.x * g.x + g.y * g.y;
          if (ag2 > 1e-290 && ag2 > 1e-36 * fabs(a * b)) {
            const double d = b - a;
            const double u = copysign(2.0, d) / (fabs(d) + sqrt(fma(d, d, 4.0 * ag2)));
            const double tg = u * ag2;  // t |A_pq|
            c = rsqrt(fma(tg, u, 1.0));  // 1 / sqrt(1 + t^2)
            const double uc = u * c;
            sr = uc * g.x;
            si = uc * g.y;
            A[p * m + p] = make_double2(a - tg, 0.0);
            A[q * m + q] = make_double2(b + tg, 0.0);
            A[p * m + q] = make_double2(0.0, 0.0);
            A[q * m + p] = make_double2(0.0, 0.0);
          }
        }
        R.p[lane] = p;
        R.q[lane] = q;
        R.c[lane] = c;
        R.sr[lane] = sr;
        R.si[lane] = si;
      }
      __syncwarp();
      for (int bi = lane; bi < nblk; bi += 32) {
        const int k1 = R.blk[2 * bi], k2 = R.blk[2 * bi + 1];
        const bool r1 = !(R.sr[k1] == 0.0 && R.si[k1] == 0.0), r2 = !(R.sr[k2] == 0.0 && R.si[k2] == 0.0);
        if (!r1 && !r2) continue;
        const int p1 = R.p[k1], q1 = R.q[k1], p2 = R.p[k2], q2 = R.q[k2];
        const bool v1 = q1 < m, v2 = q2 < m;  // q = m is the dummy of an odd order
        const double c1 = R.c[k1], c2 = R.c[k2];
        const double2 s1 = make_double2(R.sr[k1], R.si[k1]), s2 = make_double2(R.sr[k2], R.si[k2]);
        const double2 z = make_double2(0.0, 0.0);
        const double2 x11 = A[p1 * m + p2], x12 = v2 ? A[p1 * m + q2] : z;
        const double2 x21 = v1 ? A[q1 * m + p2] : z, x22 = (v1 && v2) ? A[q1 * m + q2] : z;
        // Y = X R2: Y[:,0] = c2 X[:,0] - conj(s2) X[:,1], Y[:,1] = s2 X[:,0] + c2 X[:,1]
        const double2 y11 = csub(cscale(x11, c2), cmul(conjd(s2), x12));
        const double2 y21 = csub(cscale(x21, c2), cmul(conjd(s2), x22));
        const double2 y12 = cadd(cmul(s2, x11), cscale(x12, c2));
        const double2 y22 = cadd(cmul(s2, x21), cscale(x22, c2));
        // X' = R1^H Y: row 0 = c1 Y0 - s1 Y1, row 1 = conj(s1) Y0 + c1 Y1
        const double2 n11 = csub(cscale(y11, c1), cmul(s1, y21));
        const double2 n12 = csub(cscale(y12, c1), cmul(s1, y22));
        const double2 n21 = cadd(cmul(conjd(s1), y11), cscale(y21, c1));
        const double2 n22 = cadd(cmul(conjd(s1), y12), cscale(y22, c1));
        A[p1 * m + p2] = n11;
        A[p2 * m + p1] = conjd(n11);
        if (v2) {
          A[p1 * m + q2] = n12;
          A[q2 * m + p1] = conjd(n12);
        }
        if (v1) {
          A[q1 * m + p2] = n21;
          A[p2 * m + q1] = conjd(n21);
        }
        if (v1 && v2) {
          A[q1 * m + q2] = n22;
          A[q2 * m + q1] = conjd(n22);
        }
      }
      if (V) {
        const int work = npair * m;
        for (int it = lane; it < work; it += 32) {  // V <- V J
          const int k = it / m, r = it - (it / m) * m;
          const int p = R.p[k], q = R.q[k];
          if (q >= m || (R.sr[k] == 0.0 && R.si[k] == 0.0)) continue;
          const double c = R.c[k];
          const double2 se = make_double2(R.sr[k], R.si[k]);
          const double2 x = V[r * m + p], y = V[r * m + q];
          V[r * m + p] = csub(cscale(x, c), cmul(conjd(se), y));
          V[r * m + q] = cadd(cmul(se, x), cscale(y, c));
        }
      }
      __syncwarp();
    }
  }
  return sweep;
}

// Hermitian part of a matrix that is Hermitian up to rounding.
__device__ void hermitian_part(double2 *A, int m, int lane) {
  for (int e = lane; e < m * m; e += 32) {
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
}

// s0_i = (1/K) sum_kappa Re Sbar_kappa[i][i], one CTA per system, fixed-order reduction.
__global__ void __launch_bounds__(256) k_overlap_norms(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box || !s.s0) return;
  __shared__ double part[256];
  const int m = s.m0, K = s.nblocks, tid = threadIdx.x;
  const double2 *Sb = reinterpret_cast<const double2 *>(s.Sbar);
  for (int i = 0; i < m; ++i) {
    double acc = 0.0;
    for (int k = tid; k < K; k += 256) acc += Sb[(int64_t)k * m * m + i * m + i].x;
    part[tid] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (tid < w) part[tid] += part[tid + w];
      __syncthreads();
    }
    if (tid == 0) s.s0[i] = part[0] / K;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kEigWarps * 32) k_eig(const SysDev *__restrict__ sysv,
                                                        unsigned *flags, unsigned long long *counters,
                                                        int max_m0) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // k-point of this warp: the i-th entry of the list of solved k-points (one per conjugate pair)
  // when the system has one, otherwise warp i takes k-point i and leaves it to its partner if
  // the partner's index is lower
  const int widx = blockIdx.x * kEigWarps + warp;
  int kap;
  if (s.klist) {
    if (widx >= s.nkhalf) return;
    kap = s.klist[widx];
  } else {
    kap = widx;
    if (kap >= s.nblocks) return;
  }
  const int L0 = s.d[0].L, L1 = s.d[1].L, L2 = s.d[2].L;
  const int k0 = kap / (L1 * L2), k1 = (kap / L2) % L1, k2 = kap % L2;
  const int mk = (((L0 - k0) % L0) * L1 + (L1 - k1) % L1) * L2 + (L2 - k2) % L2;
  if (!s.klist && mk < kap) return;  // the conjugate partner solves this pair
  const int m0 = s.m0;
  extern __shared__ unsigned char smraw[];
  unsigned char *base = smraw + (size_t)warp * eig_warp_bytes(max_m0);
  double2 *A = reinterpret_cast<double2 *>(base);
  double2 *B = A + max_m0 * max_m0;
  double2 *V = B + max_m0 * max_m0;
  double *rc = reinterpret_cast<double *>(V + max_m0 * max_m0);
  double *rsr = rc + 16, *rsi = rsr + 16;
  double *dsc = rsi + 16;   // [32] scale of kept function a
  double *sg = dsc + 32;    // [32] eigenvalues of the scaled overlap (canonical path)
  int *rp = reinterpret_cast<int *>(sg + 32), *rq = rp + 16;
  int *kidx = rq + 16;      // [32] original index of kept function a
  int *kidx2 = kidx + 32;   // [32] kept overlap eigen-directions (canonical path)
  unsigned char *blk = reinterpret_cast<unsigned char *>(kidx2 + 32);  // [<= 120][2]
  {
    // pairs k1 < k2 ordered by k2, so that the first n (n - 1) / 2 entries are those of n pairs
    const int np = (m0 + 1) / 2;  // pairs of the largest order this warp may rotate
    for (int bi = lane; bi < np * (np - 1) / 2; bi += 32) {
      int k2 = 1, rem = bi;
      while (rem >= k2) {
        rem -= k2;
        ++k2;
      }
      blk[2 * bi] = (unsigned char)rem;
      blk[2 * bi + 1] = (unsigned char)k2;
    }
    __syncwarp();
  }
  const RotTab R{rc, rsr, rsi, rp, rq, blk};

  const double2 *Hb = reinterpret_cast<const double2 *>(s.Hbar) + (int64_t)kap * m0 * m0;
  const double2 *Sb = reinterpret_cast<const double2 *>(s.Sbar) + (int64_t)kap * m0 * m0;

  // 0. numerically absent Bloch functions; gather and scale the kept pencil
  bool ok = true;
  double dii = 0.0;
  bool keep = false;
  if (lane < m0) {
    dii = Sb[lane * m0 + lane].x;
    const double norm = s.s0[lane];
    if (!(norm > 0.0)) ok = false;
    keep = dii > kDropTol * norm;
  }
  ok = __all_sync(0xffffffffu, ok);
  const unsigned kmask = __ballot_sync(0xffffffffu, keep);
  int m = __popc(kmask);
  if (keep) {
    const int a = __popc(kmask & ((1u << lane) - 1u));
    kidx[a] = lane;
    dsc[a] = 1.0 / sqrt(dii);
  }
  __syncwarp();
  for (int e = lane; e < m * m; e += 32) {
    const int a = e / m, b = e - (e / m) * m;
    const int ia = kidx[a], ib = kidx[b];
    const double sc = dsc[a] * dsc[b];
    A[e] = cscale(Hb[ia * m0 + ib], sc);
    B[e] = cscale(Sb[ia * m0 + ib], sc);
  }
  __syncwarp();

  // 1. Cholesky of the scaled overlap (lower triangle, in place in B); a pivot below kCholTol
  //    sends the k-point to canonical orthogonalisation
  bool chol = ok;
  for (int j = 0; chol && j < m; ++j) {
    if (lane == 0) {
      double d = B[j * m + j].x;
      for (int k = 0; k < j; ++k) {
        const double2 v = B[j * m + k];
        d -= v.x * v.x + v.y * v.y;
      }
      B[j * m + j] = make_double2(d >= kCholTol ? sqrt(d) : -1.0, 0.0);
    }
    __syncwarp();
    const double dj = B[j * m + j].x;
    if (!(dj > 0.0)) {
      chol = false;
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

  int sweeps = 0;
  if (ok && chol) {
    // 2. C = L^{-1} H L^{-H}
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
        for (int e = lane; e < m * m; e += 32) {
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
    hermitian_part(A, m, lane);
  } else if (ok) {
    // 2'. canonical orthogonalisation: S~ = V diag(sigma) V^H, keep sigma >= kLindepTol,
    //     X = V_kept diag(sigma)^{-1/2}, C = X^H H~ X
    for (int e = lane; e < m * m; e += 32) {
      const int a = e / m, b = e - (e / m) * m;
      B[e] = cscale(Sb[kidx[a] * m0 + kidx[b]], dsc[a] * dsc[b]);
      V[e] = make_double2(a == b ? 1.0 : 0.0, 0.0);
    }
    __syncwarp();
    hermitian_part(B, m, lane);
    sweeps += jacobi_herm(B, V, m, lane, R);
    const bool kp = lane < m && B[lane * m + lane].x >= kLindepTol;
    const unsigned m2mask = __ballot_sync(0xffffffffu, kp);
    const int m2 = __popc(m2mask);
    if (kp) {
      const int b = __popc(m2mask & ((1u << lane) - 1u));
      kidx2[b] = lane;
      sg[b] = 1.0 / sqrt(B[lane * m + lane].x);
    }
    __syncwarp();
    for (int e = lane; e < m * m2; e += 32) {  // X (m x m2) into B
      const int i = e / m2, b = e - (e / m2) * m2;
      B[e] = cscale(V[i * m + kidx2[b]], sg[b]);
    }
    __syncwarp();
    for (int e = lane; e < m * m2; e += 32) {  // W = H~ X (m x m2) into V
      const int i = e / m2, b = e - (e / m2) * m2;
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < m; ++k) {
        const double2 t = cmul(A[i * m + k], B[k * m2 + b]);
        acc.x += t.x;
        acc.y += t.y;
      }
      V[e] = acc;
    }
    __syncwarp();
    for (int e = lane; e < m2 * m2; e += 32) {  // C = X^H W (m2 x m2) into A
      const int a = e / m2, b = e - (e / m2) * m2;
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < m; ++k) {
        const double2 x = B[k * m2 + a], w = V[k * m2 + b];
        acc.x += x.x * w.x + x.y * w.y;  // conj(x) w
        acc.y += x.x * w.y - x.y * w.x;
      }
      A[e] = acc;
    }
    __syncwarp();
    m = m2;
    hermitian_part(A, m, lane);
  }

  if (ok) {
    // 3. cyclic Jacobi on C
    sweeps += jacobi_herm(A, nullptr, m, lane, R);
    if (lane == 0 && counters) {
      atomicAdd(counters, (unsigned long long)sweeps);
      atomicAdd(counters + 1, 1ull);
      if (!chol) atomicAdd(counters + 2, 1ull);
    }
  }

  // 4. sort and store (dropped functions and directions: +inf, last)
  double v = (ok && lane < m) ? A[lane * m + lane].x : INFINITY;
  for (int k = 2; k <= 32; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      const double o = __shfl_xor_sync(0xffffffffu, v, j);
      const bool up = (lane & k) == 0, lower = (lane & j) == 0;
      v = (lower == up) ? fmin(v, o) : fmax(v, o);
    }
  if (!ok) v = NAN;
  if (lane < m0) {
    s.eig[(int64_t)kap * m0 + lane] = v;
    s.eig[(int64_t)mk * m0 + lane] = v;
  }
  if (lane == 0) {
    const int st = ok ? m0 - m : (int)LHF_ERR_NOT_SPD;
    if (s.kstat) {
      s.kstat[kap] = st;
      s.kstat[mk] = st;
    }
    if (!ok) atomicOr(flags, kFlagNotSpd);
  }
}

}  // namespace

cudaError_t launch_overlap_norms(const SysDev *sys, int nsys, cudaStream_t st) {
  if (nsys <= 0) return cudaSuccess;
  k_overlap_norms<<<dim3(1, nsys), 256, 0, st>>>(sys);
  return cudaGetLastError();
}

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
