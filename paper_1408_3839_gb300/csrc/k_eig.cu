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
#include "lhf_pairs.cuh"

namespace lhf {
namespace {

constexpr int kEigMaxWarps = 8;  // warps (k-points) per CTA: blockDim.x / 32, set by the launcher

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// acc + a b and acc - a conj(b) as four FMAs each
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ double2 cfms_conj(double2 a, double2 b, double2 acc) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(-a.y, b.x, acc.y);
  acc.y = fma(a.x, b.y, acc.y);
  return acc;
}

// The lanes that solve one matrix: G = 32 (a whole warp) or G = 16 (half a warp, two matrices
// per warp, used when every order is at most 16: the scalar steps of a factorisation -- pivots,
// norms, reciprocals -- then cost one FP64 warp instruction per two matrices).  Every
// collective (shuffle, ballot, vote, syncwarp) runs over the group's own lanes only, so the two
// groups of a warp may follow different paths.
template <int G>
struct Grp {
  unsigned mask;  // the group's lanes within the warp
  int lane;       // lane within the group
  int base;       // first warp lane of the group
  __device__ Grp() {
    const int wl = (int)(threadIdx.x & 31);
    base = wl & ~(G - 1);
    lane = wl - base;
    mask = G == 32 ? 0xffffffffu : (0xffffu << base);
  }
  __device__ __forceinline__ void sync() const { __syncwarp(mask); }
  __device__ __forceinline__ double sum(double v) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
  }
  __device__ __forceinline__ unsigned ballot(bool p) const { return __ballot_sync(mask, p) >> base; }
};

// per warp: A, B, V (m^2 complex each; V in the system's per-k-point scratch SysDev::evs instead
// when vglob), rotation table (16 x {c, sr, si, p, q}), kept index map, scales and overlap
// eigenvalues (32 each), the (k1 < k2) pair-block table (120 x 2) and the Householder vectors
// (2 x 32 complex).  V is touched only by the canonical route, the FP64 trace test and the
// eigenvector path: out of shared memory it leaves room for a third more resident matrices.
__host__ __device__ inline size_t eig_warp_core_bytes(int m, bool vglob) {
  return (size_t)(vglob ? 2 : 3) * m * m * sizeof(double2) + 16 * (3 * sizeof(double) + 2 * sizeof(int)) +
         32 * (2 * sizeof(double) + 2 * sizeof(int)) + 288;
}
// + 64 complex of Householder scratch (v and w), except with vglob from order 8 on: then the
// vectors take B's space, free once C is formed on the tridiagonal route
__host__ __device__ inline bool eig_hh_in_b(int m, bool vglob) { return vglob && m >= 8; }
__host__ __device__ inline size_t eig_warp_bytes(int m, bool vglob) {
  return eig_warp_core_bytes(m, vglob) + (eig_hh_in_b(m, vglob) ? 0 : 64 * sizeof(double2));
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
template <int G>
__device__ int jacobi_herm(double2 *A, double2 *V, int m, const Grp<G> &g, const RotTab &R) {
  const int lane = g.lane;
  const int mm = m * m, mp = m + (m & 1), npair = mp / 2;
  const int nblk = npair * (npair - 1) / 2;
  int sweep = 0;
  for (; sweep < 40; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = lane; e < mm; e += G) {
      const double v = A[e].x * A[e].x + A[e].y * A[e].y;
      tot += v;
      if (e / m != e - (e / m) * m) off += v;
    }
    for (int o = G / 2; o > 0; o >>= 1) {
      off += __shfl_xor_sync(g.mask, off, o);
      tot += __shfl_xor_sync(g.mask, tot, o);
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
      g.sync();
      for (int bi = lane; bi < nblk; bi += G) {
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
        for (int it = lane; it < work; it += G) {  // V <- V J
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
      g.sync();
    }
  }
  return sweep;
}

// Householder reduction of the Hermitian m x m matrix A (shared memory, destroyed) to a real
// symmetric tridiagonal matrix with the same eigenvalues, one warp.  Column k: x = A[k+1:, k],
// alpha = -e^{i arg x0} |x|, v = x - alpha e1, H = I - tau v v^H with tau = 1 / (|x|^2 + |x| |x0|);
// A <- H A H as p = tau A v, w = p - (tau/2)(v^H p) v, A <- A - v w^H - w v^H on the trailing
// block.  Only the lower triangle of the trailing block is kept (the upper one is its conjugate);
// the matrix-vector product takes two lanes per row.  The off-diagonal alpha_k is replaced by
// |alpha_k| (a diagonal unitary similarity).  td[0..m), te[0..m-1) receive the diagonal and
// off-diagonal.  vw: 2 x 32 complex scratch.
template <int G>
__device__ void householder_tridiag(double2 *A, int m, const Grp<G> &g, double2 *vw, double *td, double *te) {
  const int lane = g.lane;
  double2 *vec = vw, *wv = vw + 32;
  for (int k = 0; k + 2 < m; ++k) {
    const int n = m - k - 1;
    double2 xi = make_double2(0.0, 0.0);
    if (lane < n) xi = A[(k + 1 + lane) * m + k];
    double part = xi.x * xi.x + xi.y * xi.y;
    for (int o = G / 2; o > 0; o >>= 1) part += __shfl_xor_sync(g.mask, part, o);
    const double sig = part;
    const double2 x0 = A[(k + 1) * m + k];
    const double akk = A[k * m + k].x;
    if (!(sig > 0.0)) {  // column already reduced
      if (lane == 0) {
        td[k] = akk;
        te[k] = 0.0;
      }
      continue;
    }
    // |x| and |x0| from reciprocal square roots (the scaled entries are far inside the FP64
    // range), e^{i arg x0} = x0 / |x0|
    const double nrm = sig * rsqrt(sig);
    const double a2 = fma(x0.x, x0.x, x0.y * x0.y);
    const double ra = a2 > 0.0 ? rsqrt(a2) : 0.0, ax0 = a2 * ra;
    const double2 ph = a2 > 0.0 ? make_double2(x0.x * ra, x0.y * ra) : make_double2(1.0, 0.0);
    const double tau = 1.0 / fma(nrm, ax0, sig);
    if (lane < n) vec[lane] = lane == 0 ? make_double2(x0.x + ph.x * nrm, x0.y + ph.y * nrm) : xi;
    g.sync();
    // p = tau B v, B = A[k+1:, k+1:] from its lower triangle, RL = G / 16 lanes per row
    constexpr int RL = G / 16;
    const double2 *Bt = A + (k + 1) * m + (k + 1);
    double kp = 0.0;
    for (int r0 = 0; r0 < n; r0 += 16) {
      const int r = r0 + lane / RL;
      double2 pi = make_double2(0.0, 0.0);
      if (r < n) {
        for (int j = lane % RL; j < n; j += RL) {
          double2 b = j <= r ? Bt[r * m + j] : Bt[j * m + r];
          if (j > r) b.y = -b.y;
          pi = cfma(b, vec[j], pi);
        }
      }
      if (RL == 2) {
        pi.x += __shfl_xor_sync(g.mask, pi.x, 1);
        pi.y += __shfl_xor_sync(g.mask, pi.y, 1);
      }
      if (r < n && lane % RL == 0) {
        pi = cscale(pi, tau);
        wv[r] = pi;
        kp += vec[r].x * pi.x + vec[r].y * pi.y;  // Re(conj(v_r) p_r)
      }
    }
    // K = (tau / 2) Re(v^H p)
    for (int o = G / 2; o > 0; o >>= 1) kp += __shfl_xor_sync(g.mask, kp, o);
    const double Kf = 0.5 * tau * kp;
    g.sync();
    if (lane < n) wv[lane] = make_double2(wv[lane].x - Kf * vec[lane].x, wv[lane].y - Kf * vec[lane].y);
    g.sync();
    // lower triangle (i >= j) of the trailing block: a -= v_i conj(w_j) + w_i conj(v_j)
    for (int t = lane; t < n * (n + 1) / 2; t += G) {
      int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= t) ++i;
      while (i * (i + 1) / 2 > t) --i;
      const int j = t - i * (i + 1) / 2;
      const double2 vi = vec[i], wi = wv[i], vj = vec[j], wj = wv[j];
      double2 &a = A[(k + 1 + i) * m + (k + 1 + j)];
      a = cfms_conj(wi, vj, cfms_conj(vi, wj, a));
    }
    if (lane == 0) {
      td[k] = akk;
      te[k] = nrm;
    }
    g.sync();
  }
  if (lane == 0) {
    if (m >= 2) {
      td[m - 2] = A[(m - 2) * m + (m - 2)].x;
      const double2 b = A[(m - 1) * m + (m - 2)];
      te[m - 2] = hypot(b.x, b.y);
    }
    td[m - 1] = A[(m - 1) * m + (m - 1)].x;
  }
  g.sync();
}

// Hermitian part of a matrix that is Hermitian up to rounding.
template <int G>
__device__ void hermitian_part(double2 *A, int m, const Grp<G> &g) {
  const int lane = g.lane;
  for (int e = lane; e < m * m; e += G) {
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
  g.sync();
}

// ---- compensated FP32 pairs for the mixed route's reduction ---------------------------------
// GB300 runs FP64 at 1/64 of the FP32 rate and charges the FP64 unit per warp instruction, so
// the mixed route (whose eigenvalue target is 1e-6 Ha) takes the Cholesky-route reduction --
// Cholesky, the two triangular solves, Householder -- in pairs of FP32 words: a real value is
// h + l with |l| <= ulp(h) / 2 (48 significant bits), a complex entry a float4 {re_h, re_l, im_h,
// im_l} in the 16 bytes of the double2 it replaces.  Sums of products are compensated dot
// products (Ogita, Rump and Oishi 2005): each product's rounding error comes from an FMA, each
// sum's from Knuth's TwoSum, and both are gathered in a second FP32 word, so that a sum of n
// products is as accurate as if computed with twice the FP32 precision.  Square roots and
// reciprocals take the FP32 approximation and one Newton step in pair arithmetic.  __fadd_rn and
// __fmul_rn keep the compiler from contracting the error-free transforms into FMAs.
struct Cacc {
  float rs, rc, is, ic;  // real part rs + rc, imaginary part is + ic
};

// 1 / a, 1 / sqrt(a), sqrt(a): the FP32 value and one Newton step in pair arithmetic
__device__ __forceinline__ float2 df_recip(float2 a) {
  const float h = __frcp_rn(a.x);
  const float2 e = df_add(make_float2(1.0f, 0.0f), df_mul(make_float2(-h, 0.0f), a));  // 1 - h a
  return df_norm(h, __fmul_rn(h, e.x));
}
__device__ __forceinline__ float2 df_rsqrt(float2 a) {
  const float h = rsqrtf(a.x);
  const float2 e = df_add(make_float2(1.0f, 0.0f), df_neg(df_mul(a, df_mul(make_float2(h, 0.0f), make_float2(h, 0.0f)))));
  return df_norm(h, __fmul_rn(0.5f * h, e.x));  // h (1 + (1 - a h^2) / 2)
}
__device__ __forceinline__ float2 df_sqrt(float2 a) {
  if (!(a.x > 0.0f)) return make_float2(0.0f, 0.0f);
  const float h = __fsqrt_rn(a.x);
  const float2 r = df_add(a, df_neg(df_mul(make_float2(h, 0.0f), make_float2(h, 0.0f))));  // a - h^2
  return df_norm(h, __fdiv_rn(r.x, 2.0f * h));
}
// x as a pair from its bits, without FP64 instructions (this GPU issues them at 1/64 of the FP32
// rate): h = the leading 24 significant bits, l = the remaining 29 bits rounded to 24, then
// renormalised (|x - (h + l)| <= 2^-48 |x|).  Zero and subnormal x give 0; an exponent outside
// h's and l's normal range (|x| < 2^-74, |x| >= 2^128, inf, NaN) takes the FP64 conversion.
__device__ __forceinline__ float2 pair_from_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ffu);
  if (E == 0) return make_float2(0.0f, 0.0f);
  const int fe = E - 896;  // h's biased FP32 exponent (E - 1023 + 127)
  if (fe < 53 || fe > 254) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
  }
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const float h = __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)((b >> 29) & 0x7fffffu));
  // x - h = +-(low 29 bits) 2^(E - 1075), the power of two an FP32 normal (fe - 52 >= 1)
  const float lm = __fmul_rn((float)(unsigned)(b & 0x1fffffffu), __uint_as_float((unsigned)(fe - 52) << 23));
  return df_norm(h, sign ? -lm : lm);
}
__device__ __forceinline__ float4 df_from(double2 v) {
  const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
  return make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
}
__device__ __forceinline__ double2 df_to(float4 v) {
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}
// A += a b and A -= a conj(b) (complex)
__device__ __forceinline__ void cacc_mad(Cacc &A, float4 a, float4 b) {
  acc_prod(A.rs, A.rc, a.x, a.y, b.x, b.y);
  acc_prod(A.rs, A.rc, -a.z, -a.w, b.z, b.w);
  acc_prod(A.is, A.ic, a.x, a.y, b.z, b.w);
  acc_prod(A.is, A.ic, a.z, a.w, b.x, b.y);
}
__device__ __forceinline__ void cacc_msub_conj(Cacc &A, float4 a, float4 b) {
  acc_prod(A.rs, A.rc, -a.x, -a.y, b.x, b.y);
  acc_prod(A.rs, A.rc, -a.z, -a.w, b.z, b.w);
  acc_prod(A.is, A.ic, -a.z, -a.w, b.x, b.y);
  acc_prod(A.is, A.ic, a.x, a.y, b.z, b.w);
}
__device__ __forceinline__ Cacc cacc_from(float4 v) { return Cacc{v.x, v.y, v.z, v.w}; }
__device__ __forceinline__ float4 cacc_value(const Cacc &A) {
  const float2 r = df_norm(A.rs, A.rc), i = df_norm(A.is, A.ic);
  return make_float4(r.x, r.y, i.x, i.y);
}
__device__ __forceinline__ float4 df_cscale(float4 v, float2 t) {
  const float2 r = df_mul(make_float2(v.x, v.y), t), i = df_mul(make_float2(v.z, v.w), t);
  return make_float4(r.x, r.y, i.x, i.y);
}
__device__ __forceinline__ float4 df_conj(float4 v) { return make_float4(v.x, v.y, -v.z, -v.w); }
__device__ __forceinline__ float2 df_abs2(float4 v) {  // |v|^2
  float s = 0.0f, c = 0.0f;
  acc_prod(s, c, v.x, v.y, v.x, v.y);
  acc_prod(s, c, v.z, v.w, v.z, v.w);
  return df_norm(s, c);
}
// sum of a pair over the group's lanes (pairwise compensated)
template <int G>
__device__ __forceinline__ float2 df_group_sum(float2 v, const Grp<G> &g) {
  for (int o = G / 2; o > 0; o >>= 1) {
    const float h = __shfl_xor_sync(g.mask, v.x, o), l = __shfl_xor_sync(g.mask, v.y, o);
    v = df_add(v, make_float2(h, l));
  }
  return v;
}

// Hermitian part (X + X^H) / 2 in pairs.
template <int G>
__device__ void df_hermitian_part(float4 *A, int m, const Grp<G> &g) {
  for (int e = g.lane; e < m * m; e += G) {
    const int i = e / m, j = e - (e / m) * m;
    if (i < j) {
      const float4 x = A[i * m + j], y = A[j * m + i];
      const float2 re = df_add(make_float2(x.x, x.y), make_float2(y.x, y.y));
      const float2 im = df_add(make_float2(x.z, x.w), make_float2(-y.z, -y.w));
      const float4 a = make_float4(0.5f * re.x, 0.5f * re.y, 0.5f * im.x, 0.5f * im.y);
      A[i * m + j] = a;
      A[j * m + i] = df_conj(a);
    } else if (i == j) {
      A[e].z = 0.0f;
      A[e].w = 0.0f;
    }
  }
  g.sync();
}

// FP32 copy of the Cholesky factor's entry (i, j), i > j, for the trace estimate: stored in the
// first 8 bytes of the (16-byte) element (j, i) of the factorised matrix, whose strict upper
// triangle neither the factorisation nor the triangular solves read.
__device__ __forceinline__ float2 *l32_at(void *B, int m, int i, int j) {
  return reinterpret_cast<float2 *>(static_cast<unsigned char *>(B) + (size_t)(j * m + i) * 16);
}

// Cholesky of the scaled overlap in pairs, as the FP64 loop of k_eig: the FP32 copy of the
// off-diagonal factor in the free strict upper triangle of B (l32_at) and the inverse pivots sgf
// (pairs) for the triangular solves.  False when a scaled pivot falls below kCholTol.
template <int G>
__device__ bool df_cholesky(float4 *B, int m, const Grp<G> &g, float2 *sgf) {
  const int lane = g.lane;
  for (int j = 0; j < m; ++j) {
    const float2 d = make_float2(B[j * m + j].x, B[j * m + j].y);
    if (!(d.x + d.y >= (float)kCholTol)) return false;  // group-uniform
    const float2 inv = df_rsqrt(d), ljj = df_mul(d, inv);
    g.sync();
    for (int i = j + 1 + lane; i < m; i += G) {
      const float4 lij = df_cscale(B[i * m + j], inv);
      B[i * m + j] = lij;
      *l32_at(B, m, i, j) = make_float2(lij.x, lij.z);
    }
    g.sync();
    if (lane == 0) {
      B[j * m + j] = make_float4(ljj.x, ljj.y, 0.0f, 0.0f);
      sgf[j] = inv;
    }
    const int n = m - j - 1;
    for (int t = lane; t < n * (n + 1) / 2; t += G) {
      int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= t) ++i;
      while (i * (i + 1) / 2 > t) --i;
      const int k = t - i * (i + 1) / 2;
      const int ri = j + 1 + i, rk = j + 1 + k;
      Cacc acc = cacc_from(B[ri * m + rk]);
      cacc_msub_conj(acc, B[ri * m + j], B[rk * m + j]);
      B[ri * m + rk] = cacc_value(acc);
    }
    g.sync();
  }
  return true;
}

// Forward substitution in pairs, as the FP64 pass of k_eig: columns cc < ncol of X (A for cc < m,
// V for the identity columns m .. 2m - 1) become L^{-1} X, lanes over columns (two lanes per
// column when 16 columns or fewer fill a whole warp).
template <int G>
__device__ void df_forward(float4 *A, float4 *V, const float4 *B, const float2 *sgf, int m, int ncol, const Grp<G> &g) {
  const int lane = g.lane;
  const int q = (G == 32 && ncol <= 16) ? 2 : 1;
  for (int cc0 = 0; cc0 < ncol; cc0 += G / q) {
    const int cc = cc0 + lane / q, part = lane % q;
    const bool act = cc < ncol;
    float4 *X = cc < m ? A : V;
    const int c = act ? (cc < m ? cc : cc - m) : 0;
    float4 z[kMaxM0];
    for (int i = 0; i < m; ++i) {
      Cacc acc{0.0f, 0.0f, 0.0f, 0.0f};
      if (act)
        for (int k = part; k < i; k += q) cacc_mad(acc, B[i * m + k], z[k]);
      if (q == 2) {
        const float rs = __shfl_xor_sync(g.mask, acc.rs, 1), rc = __shfl_xor_sync(g.mask, acc.rc, 1);
        const float is = __shfl_xor_sync(g.mask, acc.is, 1), ic = __shfl_xor_sync(g.mask, acc.ic, 1);
        acc_add(acc.rs, acc.rc, rs, rc);
        acc_add(acc.is, acc.ic, is, ic);
      }
      const float4 xi = act ? X[i * m + c] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      Cacc d = cacc_from(xi);
      acc_add(d.rs, d.rc, -acc.rs, -acc.rc);
      acc_add(d.is, d.ic, -acc.is, -acc.ic);
      z[i] = df_cscale(cacc_value(d), sgf[i]);
      if (act && part == 0) X[i * m + c] = z[i];
    }
  }
  g.sync();
}

// A += c x (c a real pair, x a complex pair)
__device__ __forceinline__ void cacc_rmad(Cacc &A, float2 c, float4 x) {
  acc_prod(A.rs, A.rc, c.x, c.y, x.x, x.y);
  acc_prod(A.is, A.ic, c.x, c.y, x.z, x.w);
}

// Cyclic Jacobi in pairs, as jacobi_herm (same ordering, rotations and block updates; the
// rotation table's c, s_r, s_i hold pairs in their doubles' bytes): the rotation from
// u = 2 sign(d) / (|d| + sqrt(d^2 + 4 |A_pq|^2)) with the square root and the reciprocals in
// pair arithmetic, the 2 x 2 block updates as compensated sums.  Pairs resolve about 2^-46 of
// an entry, so the sweeps stop once the off-diagonal Frobenius norm falls below 2^-42 of the
// total (squared: 2^-84), a margin above the rounding noise of the updates; the off-diagonal
// left moves an eigenvalue by its square over the gap.  Returns the sweeps.
template <int G>
__device__ int df_jacobi_herm(float4 *A, float4 *V, int m, const Grp<G> &g, const RotTab &R) {
  const int lane = g.lane;
  const int mm = m * m, mp = m + (m & 1), npair = mp / 2;
  const int nblk = npair * (npair - 1) / 2;
  float2 *Rc = reinterpret_cast<float2 *>(R.c), *Rr = reinterpret_cast<float2 *>(R.sr);
  float2 *Ri = reinterpret_cast<float2 *>(R.si);
  int sweep = 0;
  for (; sweep < 40; ++sweep) {
    float off = 0.0f, tot = 0.0f;
    for (int e = lane; e < mm; e += G) {
      const float v = fmaf(A[e].x, A[e].x, A[e].z * A[e].z);
      tot += v;
      if (e / m != e - (e / m) * m) off += v;
    }
    for (int o = G / 2; o > 0; o >>= 1) {
      off += __shfl_xor_sync(g.mask, off, o);
      tot += __shfl_xor_sync(g.mask, tot, o);
    }
    if (off <= 0x1p-84f * tot) break;
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
        float2 c = make_float2(1.0f, 0.0f), sr = make_float2(0.0f, 0.0f), si = make_float2(0.0f, 0.0f);
        if (q < m) {
          const float4 gq = A[p * m + q];
          const float2 a = make_float2(A[p * m + p].x, A[p * m + p].y), b = make_float2(A[q * m + q].x, A[q * m + q].y);
          const float2 ag2 = df_abs2(gq);
          if (ag2.x > 1e-37f && ag2.x > 1e-30f * fabsf(a.x * b.x)) {
            const float2 d = df_add(b, df_neg(a));
            const float2 r = df_sqrt(df_add(df_mul(d, d), df_mul(make_float2(4.0f, 0.0f), ag2)));
            const float2 ad = d.x < 0.0f ? df_neg(d) : d;
            float2 u = df_recip(df_add(ad, r));
            u = make_float2(2.0f * (d.x < 0.0f ? -u.x : u.x), 2.0f * (d.x < 0.0f ? -u.y : u.y));
            const float2 tg = df_mul(u, ag2);  // t |A_pq|
            c = df_rsqrt(df_add(make_float2(1.0f, 0.0f), df_mul(tg, u)));  // 1 / sqrt(1 + t^2)
            const float2 uc = df_mul(u, c);
            sr = df_mul(uc, make_float2(gq.x, gq.y));
            si = df_mul(uc, make_float2(gq.z, gq.w));
            const float2 na = df_add(a, df_neg(tg)), nb = df_add(b, tg);
            A[p * m + p] = make_float4(na.x, na.y, 0.0f, 0.0f);
            A[q * m + q] = make_float4(nb.x, nb.y, 0.0f, 0.0f);
            A[p * m + q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            A[q * m + p] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          }
        }
        R.p[lane] = p;
        R.q[lane] = q;
        Rc[lane] = c;
        Rr[lane] = sr;
        Ri[lane] = si;
      }
      g.sync();
      for (int bi = lane; bi < nblk; bi += G) {
        const int k1 = R.blk[2 * bi], k2 = R.blk[2 * bi + 1];
        const bool r1 = !(Rr[k1].x == 0.0f && Ri[k1].x == 0.0f), r2 = !(Rr[k2].x == 0.0f && Ri[k2].x == 0.0f);
        if (!r1 && !r2) continue;
        const int p1 = R.p[k1], q1 = R.q[k1], p2 = R.p[k2], q2 = R.q[k2];
        const bool v1 = q1 < m, v2 = q2 < m;  // q = m is the dummy of an odd order
        const float2 c1 = Rc[k1], c2 = Rc[k2];
        const float4 s1 = make_float4(Rr[k1].x, Rr[k1].y, Ri[k1].x, Ri[k1].y);
        const float4 s2 = make_float4(Rr[k2].x, Rr[k2].y, Ri[k2].x, Ri[k2].y);
        const float4 ms2c = make_float4(-s2.x, -s2.y, s2.z, s2.w);  // -conj(s2)
        const float4 ms1 = make_float4(-s1.x, -s1.y, -s1.z, -s1.w);  // -s1
        const float4 s1c = df_conj(s1);
        const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float4 x11 = A[p1 * m + p2], x12 = v2 ? A[p1 * m + q2] : z;
        const float4 x21 = v1 ? A[q1 * m + p2] : z, x22 = (v1 && v2) ? A[q1 * m + q2] : z;
        // Y = X R2: Y[:,0] = c2 X[:,0] - conj(s2) X[:,1], Y[:,1] = s2 X[:,0] + c2 X[:,1]
        Cacc t11{}, t21{}, t12{}, t22{};
        cacc_rmad(t11, c2, x11);
        cacc_mad(t11, ms2c, x12);
        cacc_rmad(t21, c2, x21);
        cacc_mad(t21, ms2c, x22);
        cacc_mad(t12, s2, x11);
        cacc_rmad(t12, c2, x12);
        cacc_mad(t22, s2, x21);
        cacc_rmad(t22, c2, x22);
        const float4 y11 = cacc_value(t11), y21 = cacc_value(t21), y12 = cacc_value(t12), y22 = cacc_value(t22);
        // X' = R1^H Y: row 0 = c1 Y0 - s1 Y1, row 1 = conj(s1) Y0 + c1 Y1
        Cacc u11{}, u12{}, u21{}, u22{};
        cacc_rmad(u11, c1, y11);
        cacc_mad(u11, ms1, y21);
        cacc_rmad(u12, c1, y12);
        cacc_mad(u12, ms1, y22);
        cacc_mad(u21, s1c, y11);
        cacc_rmad(u21, c1, y21);
        cacc_mad(u22, s1c, y12);
        cacc_rmad(u22, c1, y22);
        const float4 n11 = cacc_value(u11), n12 = cacc_value(u12), n21 = cacc_value(u21), n22 = cacc_value(u22);
        A[p1 * m + p2] = n11;
        A[p2 * m + p1] = df_conj(n11);
        if (v2) {
          A[p1 * m + q2] = n12;
          A[q2 * m + p1] = df_conj(n12);
        }
        if (v1) {
          A[q1 * m + p2] = n21;
          A[p2 * m + q1] = df_conj(n21);
        }
        if (v1 && v2) {
          A[q1 * m + q2] = n22;
          A[q2 * m + q1] = df_conj(n22);
        }
      }
      if (V) {
        const int work = npair * m;
        for (int it = lane; it < work; it += G) {  // V <- V J
          const int k = it / m, r = it - (it / m) * m;
          const int p = R.p[k], q = R.q[k];
          if (q >= m || (Rr[k].x == 0.0f && Ri[k].x == 0.0f)) continue;
          const float2 c = Rc[k];
          const float4 se = make_float4(Rr[k].x, Rr[k].y, Ri[k].x, Ri[k].y);
          const float4 mse = make_float4(-se.x, -se.y, se.z, se.w);  // -conj(se)
          const float4 x = V[r * m + p], y = V[r * m + q];
          Cacc a{}, b{};
          cacc_rmad(a, c, x);
          cacc_mad(a, mse, y);
          cacc_mad(b, se, x);
          cacc_rmad(b, c, y);
          V[r * m + p] = cacc_value(a);
          V[r * m + q] = cacc_value(b);
        }
      }
      g.sync();
    }
  }
  return sweep;
}

// Householder reduction to real tridiagonal form in pairs, as householder_tridiag (same steps and
// lane layout); td, te receive the diagonal and off-diagonal in FP64.  vw: 2 x 32 pair scratch.
template <int G>
__device__ void df_householder_tridiag(float4 *A, int m, const Grp<G> &g, float4 *vw, double *td, double *te) {
  const int lane = g.lane;
  float4 *vec = vw, *wv = vw + 32;
  for (int k = 0; k + 2 < m; ++k) {
    const int n = m - k - 1;
    float4 xi = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (lane < n) xi = A[(k + 1 + lane) * m + k];
    const float2 sig = df_group_sum(df_abs2(xi), g);
    const float4 x0 = A[(k + 1) * m + k];
    const float2 akk = make_float2(A[k * m + k].x, A[k * m + k].y);
    if (!(sig.x > 0.0f)) {  // column already reduced
      if (lane == 0) {
        td[k] = (double)akk.x + (double)akk.y;
        te[k] = 0.0;
      }
      continue;
    }
    const float2 nrm = df_sqrt(sig);
    const float2 a2 = df_abs2(x0);
    const bool nz = a2.x > 0.0f;
    const float2 ra = nz ? df_rsqrt(a2) : make_float2(0.0f, 0.0f), ax0 = df_mul(a2, ra);
    const float2 phr = nz ? df_mul(make_float2(x0.x, x0.y), ra) : make_float2(1.0f, 0.0f);
    const float2 phi = nz ? df_mul(make_float2(x0.z, x0.w), ra) : make_float2(0.0f, 0.0f);
    const float2 tau = df_recip(df_add(df_mul(nrm, ax0), sig));
    if (lane < n) {
      if (lane == 0) {
        const float2 r = df_add(make_float2(x0.x, x0.y), df_mul(phr, nrm));
        const float2 i = df_add(make_float2(x0.z, x0.w), df_mul(phi, nrm));
        vec[0] = make_float4(r.x, r.y, i.x, i.y);
      } else {
        vec[lane] = xi;
      }
    }
    g.sync();
    constexpr int RL = G / 16;
    const float4 *Bt = A + (k + 1) * m + (k + 1);
    float kps = 0.0f, kpc = 0.0f;
    for (int r0 = 0; r0 < n; r0 += 16) {
      const int r = r0 + lane / RL;
      Cacc pi{0.0f, 0.0f, 0.0f, 0.0f};
      if (r < n) {
        for (int j = lane % RL; j < n; j += RL) {
          const float4 b = j <= r ? Bt[r * m + j] : df_conj(Bt[j * m + r]);
          cacc_mad(pi, b, vec[j]);
        }
      }
      if (RL == 2) {
        const float rs = __shfl_xor_sync(g.mask, pi.rs, 1), rc = __shfl_xor_sync(g.mask, pi.rc, 1);
        const float is = __shfl_xor_sync(g.mask, pi.is, 1), ic = __shfl_xor_sync(g.mask, pi.ic, 1);
        acc_add(pi.rs, pi.rc, rs, rc);
        acc_add(pi.is, pi.ic, is, ic);
      }
      if (r < n && lane % RL == 0) {
        const float4 p = df_cscale(cacc_value(pi), tau);
        wv[r] = p;
        const float4 v = vec[r];  // Re(conj(v_r) p_r)
        acc_prod(kps, kpc, v.x, v.y, p.x, p.y);
        acc_prod(kps, kpc, v.z, v.w, p.z, p.w);
      }
    }
    const float2 kp = df_group_sum(df_norm(kps, kpc), g);
    const float2 Kf = df_mul(make_float2(0.5f * tau.x, 0.5f * tau.y), kp);  // (tau / 2) Re(v^H p)
    g.sync();
    if (lane < n) {
      const float4 v = vec[lane], w = wv[lane];
      Cacc acc = cacc_from(w);
      acc_prod(acc.rs, acc.rc, -Kf.x, -Kf.y, v.x, v.y);
      acc_prod(acc.is, acc.ic, -Kf.x, -Kf.y, v.z, v.w);
      wv[lane] = cacc_value(acc);
    }
    g.sync();
    for (int t = lane; t < n * (n + 1) / 2; t += G) {
      int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
      while ((i + 1) * (i + 2) / 2 <= t) ++i;
      while (i * (i + 1) / 2 > t) --i;
      const int j = t - i * (i + 1) / 2;
      float4 &a = A[(k + 1 + i) * m + (k + 1 + j)];
      Cacc acc = cacc_from(a);
      cacc_msub_conj(acc, vec[i], wv[j]);
      cacc_msub_conj(acc, wv[i], vec[j]);
      a = cacc_value(acc);
    }
    if (lane == 0) {
      td[k] = (double)akk.x + (double)akk.y;
      te[k] = (double)nrm.x + (double)nrm.y;
    }
    g.sync();
  }
  if (lane == 0) {
    if (m >= 2) {
      td[m - 2] = (double)A[(m - 2) * m + (m - 2)].x + (double)A[(m - 2) * m + (m - 2)].y;
      const double2 b = df_to(A[(m - 1) * m + (m - 2)]);
      te[m - 2] = hypot(b.x, b.y);
    }
    td[m - 1] = (double)A[(m - 1) * m + (m - 1)].x + (double)A[(m - 1) * m + (m - 1)].y;
  }
  g.sync();
}

// Eigenvectors of the pencil at k-point kap (and, conjugated, at its partner mk) from the
// eigenvectors W of C (columns of V after Jacobi, sorted order given by vid per lane):
//   Cholesky route:  y = L^{-H} w (back substitution, lanes over columns), S~-orthonormal;
//   canonical route: y = X w with X = V_kept diag(sigma)^{-1/2} (in B, m x m2 by rows);
// then u = D y on the kept functions (D = diag(Sbar)^{-1/2}) and zero on the removed ones, so
// that u^H Sbar u = 1 on the kept block.  Each eigenvector's phase is fixed by making its first
// component of largest magnitude real and positive.  Row r of vecs[kap] is the eigenvector of
// the r-th smallest eigenvalue; dropped slots and failed k-points hold zero / NaN rows.
template <int G>
__device__ void bloch_vectors(const SysDev &s, int kap, int mk, bool ok, bool chol, int m, int mkept, const Grp<G> &g,
                              int vid, double2 *A, const double2 *B, double2 *V, const double *sg, const double *dsc,
                              const int *kidx) {
  const int lane = g.lane;
  const int m0 = s.m0;
  const double2 *U = V;  // back-transformed columns, row stride m
  if (ok && chol) {
    const int q = (G == 32 && m <= 16) ? 2 : 1;
    const int cc = lane / q, part = lane % q;
    const bool act = cc < m;
    double2 z[kMaxM0];
    for (int i = m - 1; i >= 0; --i) {
      double2 acc = make_double2(0.0, 0.0);
      if (act)
        for (int k = i + 1 + part; k < m; k += q) {
          const double2 l = B[k * m + i];  // conj(L[k][i]) z[k]
          acc.x = fma(l.x, z[k].x, fma(l.y, z[k].y, acc.x));
          acc.y = fma(l.x, z[k].y, fma(-l.y, z[k].x, acc.y));
        }
      if (q == 2) {
        acc.x += __shfl_xor_sync(g.mask, acc.x, 1);
        acc.y += __shfl_xor_sync(g.mask, acc.y, 1);
      }
      const double2 w = act ? V[i * m + cc] : make_double2(0.0, 0.0);
      z[i] = cscale(csub(w, acc), sg[i]);
    }
    g.sync();
    if (act && part == 0)
      for (int i = 0; i < m; ++i) V[i * m + cc] = z[i];
    g.sync();
  } else if (ok) {
    // U = X W (mkept x m) into A (its diagonal, the eigenvalues, is already in registers)
    g.sync();
    for (int e = lane; e < mkept * m; e += G) {
      const int a = e / m, c = e - (e / m) * m;
      double2 acc = make_double2(0.0, 0.0);
      for (int b = 0; b < m; ++b) acc = cfma(B[a * m + b], V[b * m + c], acc);
      A[e] = acc;
    }
    g.sync();
    U = A;
  }
  if (lane >= m0) return;
  double2 *out = reinterpret_cast<double2 *>(s.vecs) + ((int64_t)kap * m0 + lane) * m0;
  double2 *outc = reinterpret_cast<double2 *>(s.vecs) + ((int64_t)mk * m0 + lane) * m0;
  if (!ok || lane >= m) {
    const double2 fill = ok ? make_double2(0.0, 0.0) : make_double2(NAN, NAN);
    for (int mu = 0; mu < m0; ++mu) {
      out[mu] = fill;
      if (mk != kap) outc[mu] = fill;
    }
    return;
  }
  // phase: the first component of largest magnitude becomes real and positive
  double big = -1.0;
  int abig = 0;
  double2 ph = make_double2(1.0, 0.0);
  for (int a = 0; a < mkept; ++a) {
    const double2 u = cscale(U[a * m + vid], dsc[a]);
    const double mag = u.x * u.x + u.y * u.y;
    if (mag > big) {
      big = mag;
      abig = a;
      ph = u;
    }
  }
  const double amag = sqrt(big);
  ph = big > 0.0 ? make_double2(ph.x / amag, -ph.y / amag) : make_double2(1.0, 0.0);  // conj(u_max) / |u_max|
  for (int mu = 0; mu < m0; ++mu) {
    double2 u = make_double2(0.0, 0.0);
    for (int a = 0; a < mkept; ++a)
      if (kidx[a] == mu) u = a == abig ? make_double2(amag, 0.0) : cmul(cscale(U[a * m + vid], dsc[a]), ph);
    out[mu] = u;
    if (mk != kap) outc[mu] = make_double2(u.x, -u.y);
  }
}

// s0_i = (1/K) sum_kappa Re Sbar_kappa[i][i], one CTA per system, fixed-order reduction.
__global__ void __launch_bounds__(256) k_overlap_norms(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box || !s.s0) return;
  // every diagonal entry at once: a group of P lanes (16, or 8 when m0 > 16) per entry i, each
  // lane summing every P-th k-point, then a fixed shuffle tree within the group
  const int m = s.m0, K = s.nblocks, tid = threadIdx.x;
  const int P = m <= 16 ? 16 : 8;
  const int i = tid / P, sub = tid % P;
  const double2 *Sb = reinterpret_cast<const double2 *>(s.Sbar);
  double acc = 0.0;
  if (i < m)
    for (int k = sub; k < K; k += P) acc += Sb[(int64_t)k * m * m + i * m + i].x;
  for (int o = P / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (i < m && sub == 0) s.s0[i] = acc / K;
}

template <int G>
__global__ void __maxnreg__(80) k_eig(const SysDev *__restrict__ sysv,
                                                        unsigned *flags, unsigned long long *counters,
                                                        int max_m0, int vglob) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box) return;
  const Grp<G> g;
  const int lane = g.lane;
  // matrix slot of this group in the CTA (32 / G groups per warp)
  const int slotm = (int)(threadIdx.x >> 5) * (32 / G) + (int)((threadIdx.x & 31) / G);
  // k-point of this group: the i-th entry of the list of solved k-points (one per conjugate
  // pair) when the system has one, otherwise group i takes k-point i and leaves it to its
  // partner if the partner's index is lower
  const int widx = blockIdx.x * (int)((blockDim.x >> 5) * (32 / G)) + slotm;
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
  unsigned char *base = smraw + (size_t)slotm * eig_warp_bytes(max_m0, vglob != 0);
  double2 *A = reinterpret_cast<double2 *>(base);
  double2 *B = A + max_m0 * max_m0;
  double2 *V = vglob ? reinterpret_cast<double2 *>(s.evs) + (int64_t)widx * m0 * m0 : B + max_m0 * max_m0;
  double *rc = reinterpret_cast<double *>(B + (vglob ? 1 : 2) * max_m0 * max_m0);
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
    for (int bi = lane; bi < np * (np - 1) / 2; bi += G) {
      int k2 = 1, rem = bi;
      while (rem >= k2) {
        rem -= k2;
        ++k2;
      }
      blk[2 * bi] = (unsigned char)rem;
      blk[2 * bi + 1] = (unsigned char)k2;
    }
    g.sync();
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
  ok = __all_sync(g.mask, ok);
  const unsigned kmask = g.ballot(keep);
  int m = __popc(kmask);
  // mixed route, eigenvalues only: the reduction in compensated FP32 pairs (A, B and V then hold
  // float4 pairs in the same bytes): Cholesky route, canonical route and Jacobi
  const bool dfp = s.eig_df != 0 && s.tri != nullptr && s.vecs == nullptr;
  float4 *Af = reinterpret_cast<float4 *>(A), *Bf = reinterpret_cast<float4 *>(B), *Vf = reinterpret_cast<float4 *>(V);
  float2 *sgf = reinterpret_cast<float2 *>(sg);  // inverse pivots as pairs (in sg's doubles)
  float2 *dscf = reinterpret_cast<float2 *>(rc);  // the scales as pairs (rotation-table space, free until Jacobi)
  bool a_df = false;                            // A holds pairs
  if (keep) {
    const int a = __popc(kmask & ((1u << lane) - 1u));
    kidx[a] = lane;
    dsc[a] = 1.0 / sqrt(dii);
    if (dfp) dscf[a] = fp32_pair(dsc[a]);
  }
  g.sync();
  double hf2 = 0.0;  // ||H~||_F^2
  if (dfp) {
    // the pair route gathers straight from the FP64 blocks: the entries split into pairs by their
    // bits and scaled in pairs (no FP64 instruction per entry); ||H~||_F^2 in FP32 (it only
    // chooses between the tridiagonal and the Jacobi route, by a factor of 4)
    float hf = 0.0f;
    for (int e = lane; e < m * m; e += G) {
      const int a = e / m, b = e - (e / m) * m;
      const int ia = kidx[a], ib = kidx[b];
      const float2 sc = df_mul(dscf[a], dscf[b]);
      const double2 hv = Hb[ia * m0 + ib], sv = Sb[ia * m0 + ib];
      const float2 hr = pair_from_bits(hv.x), hi = pair_from_bits(hv.y);
      const float2 sr = pair_from_bits(sv.x), si = pair_from_bits(sv.y);
      const float4 x = df_cscale(make_float4(hr.x, hr.y, hi.x, hi.y), sc);
      Af[e] = x;
      Bf[e] = df_cscale(make_float4(sr.x, sr.y, si.x, si.y), sc);
      hf = fmaf(x.x, x.x, fmaf(x.z, x.z, hf));
    }
    for (int o = G / 2; o > 0; o >>= 1) hf += __shfl_xor_sync(g.mask, hf, o);
    hf2 = (double)hf;
  } else {
    for (int e = lane; e < m * m; e += G) {
      const int a = e / m, b = e - (e / m) * m;
      const int ia = kidx[a], ib = kidx[b];
      const double sc = dsc[a] * dsc[b];
      A[e] = cscale(Hb[ia * m0 + ib], sc);
      B[e] = cscale(Sb[ia * m0 + ib], sc);
      hf2 += A[e].x * A[e].x + A[e].y * A[e].y;
    }
    for (int o = G / 2; o > 0; o >>= 1) hf2 += __shfl_xor_sync(g.mask, hf2, o);
  }
  g.sync();
  // the blocks are Hermitian up to the rounding of the transform: solve their Hermitian parts
  if (dfp) {
    df_hermitian_part(Af, m, g);
    df_hermitian_part(Bf, m, g);
    a_df = true;
  } else {
    hermitian_part(A, m, g);
    hermitian_part(B, m, g);
  }

  // 1. Cholesky of the scaled overlap (lower triangle, in place in B), right-looking: column j
  //    is scaled by its pivot, then the trailing lower triangle is updated by every lane (no
  //    serial sums); a pivot below kCholTol sends the k-point to canonical orthogonalisation
  bool chol = ok;
  if (dfp && chol) chol = df_cholesky(Bf, m, g, sgf);
  for (int j = 0; !dfp && chol && j < m; ++j) {
    const double d = B[j * m + j].x;
    if (!(d >= kCholTol)) {  // warp-uniform: every lane reads the same pivot
      chol = false;
      break;
    }
    const double inv = rsqrt(d), ljj = d * inv;  // 1 / L_jj and L_jj
    g.sync();
    for (int i = j + 1 + lane; i < m; i += G) {
      const double2 lij = cscale(B[i * m + j], inv);
      B[i * m + j] = lij;
      *l32_at(B, m, i, j) = make_float2((float)lij.x, (float)lij.y);
    }
    g.sync();
    if (lane == 0) {
      B[j * m + j] = make_double2(ljj, 0.0);
      sg[j] = inv;
    }
    // B[i][k] -= L[i][j] conj(L[k][j]) for j < k <= i < m: the n (n + 1) / 2 entries of the
    // trailing lower triangle, n = m - j - 1, row by row
    const int n = m - j - 1;
    for (int t = lane; t < n * (n + 1) / 2; t += G) {
      int i = (int)((sqrt(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);  // row of the t-th entry
      while ((i + 1) * (i + 2) / 2 <= t) ++i;
      while (i * (i + 1) / 2 > t) --i;
      const int k = t - i * (i + 1) / 2;
      const int ri = j + 1 + i, rk = j + 1 + k;
      B[ri * m + rk] = cfms_conj(B[ri * m + j], B[rk * m + j], B[ri * m + rk]);
    }
    g.sync();
  }

  int sweeps = 0;
  // 2a. trace(S~^{-1}) = ||L^{-1}||_F^2 >= 1 / lambda_min decides whether the Cholesky route may
  //     be taken: 1 / trace >= kLindepTol proves that no overlap direction falls below
  //     kLindepTol, so that it solves the same pencil as canonical orthogonalisation.  First an
  //     FP32 estimate from the FP32 copy of L (forward substitution of L Z = I, two lanes per
  //     column when m <= 16): wherever trace <= 1e8 the FP32 solve is accurate to a few percent
  //     (kappa(L) <= 4e4), so an estimate below 1e6 accepts and one above 1e10 (or not finite)
  //     rejects with a factor 100 to spare; in between the exact FP64 solve decides (step 2).
  bool need64 = false;
  if (ok && chol) {
    const int q = (G == 32 && m <= 16) ? 2 : 1;
    const int cc = lane / q, part = lane % q;
    const bool act = cc < m;
    float2 z[kMaxM0];
    float tr = 0.0f;
    for (int i = 0; i < m; ++i) {
      float2 acc = make_float2(0.0f, 0.0f);
      if (act)
        for (int k = part; k < i; k += q) {
          const float2 l = *l32_at(B, m, i, k);
          acc.x = fmaf(l.x, z[k].x, acc.x);
          acc.x = fmaf(-l.y, z[k].y, acc.x);
          acc.y = fmaf(l.x, z[k].y, acc.y);
          acc.y = fmaf(l.y, z[k].x, acc.y);
        }
      if (q == 2) {
        acc.x += __shfl_xor_sync(g.mask, acc.x, 1);
        acc.y += __shfl_xor_sync(g.mask, acc.y, 1);
      }
      const float di = dfp ? sgf[i].x : (float)sg[i];  // 1 / L_ii
      z[i] = make_float2(((i == cc ? 1.0f : 0.0f) - acc.x) * di, -acc.y * di);
      if (act && part == 0) tr = fmaf(z[i].x, z[i].x, fmaf(z[i].y, z[i].y, tr));
    }
    for (int o = G / 2; o > 0; o >>= 1) tr += __shfl_xor_sync(g.mask, tr, o);
    if (!(tr <= 1e6f)) {
      if (tr <= 1e10f)
        need64 = true;
      else
        chol = false;  // also when not finite
    }
    g.sync();
  }
  if (ok && chol && dfp) {
    // 2 (pairs).  The same two passes as below: W = L^{-1} H (with the identity columns m .. 2m - 1
    // when the trace test is open), A <- W^H, C = L^{-1} A, its Hermitian part
    if (need64)
      for (int e = lane; e < m * m; e += G) {
        const int i = e / m, j = e - (e / m) * m;
        Vf[e] = make_float4(i == j ? 1.0f : 0.0f, 0.0f, 0.0f, 0.0f);
      }
    g.sync();
    df_forward(Af, Vf, Bf, sgf, m, need64 ? 2 * m : m, g);
    if (need64) {
      double tr = 0.0;
      for (int e = lane; e < m * m; e += G) {
        const double2 v = df_to(Vf[e]);
        tr += v.x * v.x + v.y * v.y;
      }
      for (int o = G / 2; o > 0; o >>= 1) tr += __shfl_xor_sync(g.mask, tr, o);
      if (!(tr * kLindepTol <= 1.0)) chol = false;  // a direction may lie below kLindepTol
    }
    if (chol) {
      for (int e = lane; e < m * m; e += G) {  // A <- A^H
        const int i = e / m, j = e - (e / m) * m;
        if (i < j) {
          const float4 x = Af[i * m + j], y = Af[j * m + i];
          Af[i * m + j] = df_conj(y);
          Af[j * m + i] = df_conj(x);
        } else if (i == j) {
          Af[e] = df_conj(Af[e]);
        }
      }
      g.sync();
      df_forward(Af, Vf, Bf, sgf, m, m, g);
      df_hermitian_part(Af, m, g);
    }
  }
  if (ok && chol && !dfp) {
    // 2. C = L^{-1} H L^{-H}.  When the FP32 estimate left the decision open, the first pass also
    //    solves L Z = I in FP64 in the columns m .. 2m-1 and ||Z||_F^2 decides: 1 / ||Z||_F^2 >=
    //    kLindepTol keeps the Cholesky route, otherwise the k-point goes to the canonical route.
    if (need64) {
      for (int e = lane; e < m * m; e += G) {
        const int i = e / m, j = e - (e / m) * m;
        V[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
      }
    }
    g.sync();  // sg[i] = 1 / L_ii from the factorisation
    for (int pass = 0; pass < 2; ++pass) {
      // forward substitution per column; with 16 columns or fewer two lanes share a column
      // (even and odd k of each inner sum, combined by a shuffle)
      const int ncol = (pass == 0 && need64) ? 2 * m : m;
      const int q = (G == 32 && ncol <= 16) ? 2 : 1;
      for (int cc0 = 0; cc0 < ncol; cc0 += G / q) {
        const int cc = cc0 + lane / q, part = lane % q;
        const bool act = cc < ncol;
        double2 *X = cc < m ? A : V;
        const int c = act ? (cc < m ? cc : cc - m) : 0;
        double2 z[kMaxM0];
        for (int i = 0; i < m; ++i) {
          double2 acc = make_double2(0.0, 0.0);
          if (act)
            for (int k = part; k < i; k += q) acc = cfma(B[i * m + k], z[k], acc);
          if (q == 2) {
            acc.x += __shfl_xor_sync(g.mask, acc.x, 1);
            acc.y += __shfl_xor_sync(g.mask, acc.y, 1);
          }
          const double2 xi = act ? X[i * m + c] : make_double2(0.0, 0.0);
          z[i] = cscale(csub(xi, acc), sg[i]);
          if (act && part == 0) X[i * m + c] = z[i];
        }
      }
      g.sync();
      if (pass == 0) {
        if (need64) {
          double tr = 0.0;
          for (int e = lane; e < m * m; e += G) tr += V[e].x * V[e].x + V[e].y * V[e].y;
          for (int o = G / 2; o > 0; o >>= 1) tr += __shfl_xor_sync(g.mask, tr, o);
          if (!(tr * kLindepTol <= 1.0)) {  // a direction may lie below kLindepTol
            chol = false;
            break;
          }
        }
        // A <- A^H
        for (int e = lane; e < m * m; e += G) {
          const int i = e / m, j = e - (e / m) * m;
          if (i < j) {
            const double2 x = A[i * m + j], y = A[j * m + i];
            A[i * m + j] = make_double2(y.x, -y.y);
            A[j * m + i] = make_double2(x.x, -x.y);
          } else if (i == j) {
            A[e].y = -A[e].y;
          }
        }
        g.sync();
      }
    }
    if (chol) {
      hermitian_part(A, m, g);
    } else {  // the scaled H again for the canonical route
      for (int e = lane; e < m * m; e += G) {
        const int a = e / m, b = e - (e / m) * m;
        A[e] = cscale(Hb[kidx[a] * m0 + kidx[b]], dsc[a] * dsc[b]);
      }
      g.sync();
      hermitian_part(A, m, g);
    }
  }
  const int mkept = m;  // kept functions (rows of the back-transformation)
  bool canon64 = ok && !chol;  // canonical route in FP64
  if (ok && !chol && dfp) {
    // 2' (pairs).  Canonical orthogonalisation as below, in compensated FP32 pairs: the scaled
    //     pencil again from the FP64 blocks (the Cholesky attempt overwrote B, the solves A),
    //     the overlap's eigen-decomposition by Jacobi, X = V_kept diag(sigma)^{-1/2},
    //     C = X^H H~ X.  An eigenvalue sigma within 1e-3 of kLindepTol leaves the decision to
    //     the FP64 route, whose rounding is 2^-7 of the pairs'.
    for (int e = lane; e < m * m; e += G) {
      const int a = e / m, b = e - (e / m) * m;
      const double sc = dsc[a] * dsc[b];
      Af[e] = df_from(cscale(Hb[kidx[a] * m0 + kidx[b]], sc));
      Bf[e] = df_from(cscale(Sb[kidx[a] * m0 + kidx[b]], sc));
      Vf[e] = make_float4(a == b ? 1.0f : 0.0f, 0.0f, 0.0f, 0.0f);
    }
    g.sync();
    df_hermitian_part(Af, m, g);
    df_hermitian_part(Bf, m, g);
    sweeps += df_jacobi_herm(Bf, Vf, m, g, R);
    double sig = 0.0;
    if (lane < m) sig = (double)Bf[lane * m + lane].x + (double)Bf[lane * m + lane].y;
    const bool near = lane < m && fabs(sig - kLindepTol) < 1e-3 * kLindepTol;
    if (!g.ballot(near)) {
      canon64 = false;
      const bool kp = lane < m && sig >= kLindepTol;
      const unsigned m2mask = g.ballot(kp);
      const int m2 = __popc(m2mask);
      if (kp) {
        const int b = __popc(m2mask & ((1u << lane) - 1u));
        kidx2[b] = lane;
        sgf[b] = df_rsqrt(make_float2(Bf[lane * m + lane].x, Bf[lane * m + lane].y));
      }
      g.sync();
      for (int e = lane; e < m * m2; e += G) {  // X (m x m2) into B
        const int i = e / m2, b = e - (e / m2) * m2;
        Bf[e] = df_cscale(Vf[i * m + kidx2[b]], sgf[b]);
      }
      g.sync();
      for (int e = lane; e < m * m2; e += G) {  // W = H~ X (m x m2) into V
        const int i = e / m2, b = e - (e / m2) * m2;
        Cacc acc{};
        for (int k = 0; k < m; ++k) cacc_mad(acc, Af[i * m + k], Bf[k * m2 + b]);
        Vf[e] = cacc_value(acc);
      }
      g.sync();
      for (int e = lane; e < m2 * m2; e += G) {  // C = X^H W (m2 x m2) into A
        const int a = e / m2, b = e - (e / m2) * m2;
        Cacc acc{};
        for (int k = 0; k < m; ++k) cacc_mad(acc, df_conj(Bf[k * m2 + a]), Vf[k * m2 + b]);
        Af[e] = cacc_value(acc);
      }
      g.sync();
      m = m2;
      df_hermitian_part(Af, m, g);
    } else {
      a_df = false;
      for (int e = lane; e < m * m; e += G) {  // the scaled H again in FP64
        const int a = e / m, b = e - (e / m) * m;
        A[e] = cscale(Hb[kidx[a] * m0 + kidx[b]], dsc[a] * dsc[b]);
      }
      g.sync();
      hermitian_part(A, m, g);
    }
  }
  if (canon64) {
    // 2'. canonical orthogonalisation: S~ = V diag(sigma) V^H, keep sigma >= kLindepTol,
    //     X = V_kept diag(sigma)^{-1/2}, C = X^H H~ X
    for (int e = lane; e < m * m; e += G) {
      const int a = e / m, b = e - (e / m) * m;
      B[e] = cscale(Sb[kidx[a] * m0 + kidx[b]], dsc[a] * dsc[b]);
      V[e] = make_double2(a == b ? 1.0 : 0.0, 0.0);
    }
    g.sync();
    hermitian_part(B, m, g);
    sweeps += jacobi_herm(B, V, m, g, R);
    const bool kp = lane < m && B[lane * m + lane].x >= kLindepTol;
    const unsigned m2mask = g.ballot(kp);
    const int m2 = __popc(m2mask);
    if (kp) {
      const int b = __popc(m2mask & ((1u << lane) - 1u));
      kidx2[b] = lane;
      sg[b] = 1.0 / sqrt(B[lane * m + lane].x);
    }
    g.sync();
    for (int e = lane; e < m * m2; e += G) {  // X (m x m2) into B
      const int i = e / m2, b = e - (e / m2) * m2;
      B[e] = cscale(V[i * m + kidx2[b]], sg[b]);
    }
    g.sync();
    for (int e = lane; e < m * m2; e += G) {  // W = H~ X (m x m2) into V
      const int i = e / m2, b = e - (e / m2) * m2;
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < m; ++k) {
        const double2 t = cmul(A[i * m + k], B[k * m2 + b]);
        acc.x += t.x;
        acc.y += t.y;
      }
      V[e] = acc;
    }
    g.sync();
    for (int e = lane; e < m2 * m2; e += G) {  // C = X^H W (m2 x m2) into A
      const int a = e / m2, b = e - (e / m2) * m2;
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < m; ++k) {
        const double2 x = B[k * m2 + a], w = V[k * m2 + b];
        acc.x += x.x * w.x + x.y * w.y;  // conj(x) w
        acc.y += x.x * w.y - x.y * w.x;
      }
      A[e] = acc;
    }
    g.sync();
    m = m2;
    hermitian_part(A, m, g);
  }

  bool tri = s.tri != nullptr;
  if (tri && ok) {
    // The tridiagonal route (Householder + QR) is accurate to ~m eps ||C|| absolute for every
    // eigenvalue; Jacobi keeps the accuracy of the small eigenvalues of graded matrices (nearly
    // singular overlaps, nearly cancelled Bloch functions with large scaled entries), so such
    // k-points stay on Jacobi: tridiagonal only if ||C||_F <= 2 ||H~||_F
    double cf2 = 0.0;
    if (a_df) {
      float c2 = 0.0f;
      for (int e = lane; e < m * m; e += G) c2 = fmaf(Af[e].x, Af[e].x, fmaf(Af[e].z, Af[e].z, c2));
      cf2 = (double)c2;
    } else {
      for (int e = lane; e < m * m; e += G) cf2 += A[e].x * A[e].x + A[e].y * A[e].y;
    }
    for (int o = G / 2; o > 0; o >>= 1) cf2 += __shfl_xor_sync(g.mask, cf2, o);
    // and only if its absolute error stays below half the 1e-10 Ha floor: m eps ||C||_F <= 5e-11
    const double cmax = 5e-11 / (m * 2.220446049250313e-16);
    if (!(cf2 <= 4.0 * hf2) || !(cf2 <= cmax * cmax)) {
      tri = false;
      if (lane == 0) s.tri[(int64_t)widx * (2 * m0 + 1)] = -2.0;  // solved here
    }
  }
  bool jac_done = false;
  if (a_df && !tri) {  // Jacobi in pairs; the eigenvalues (C's diagonal) back to FP64
    sweeps += df_jacobi_herm(Af, nullptr, m, g, R);
    for (int e = lane; e < m; e += G) {
      const float4 d = Af[e * m + e];
      A[e * m + e] = make_double2((double)d.x + (double)d.y, 0.0);
    }
    g.sync();
    a_df = false;
    jac_done = true;
  }
  if (tri) {
    // 3'. tridiagonal route: Householder reduction here, the tridiagonal eigenvalues by
    //     k_tridiag_eig (one thread per matrix); slot widx = [m | d[m0] | e[m0]]
    double *slot = s.tri + (int64_t)widx * (2 * m0 + 1);
    unsigned char *hh = eig_hh_in_b(max_m0, vglob != 0) ? reinterpret_cast<unsigned char *>(B)
                                                         : base + eig_warp_core_bytes(max_m0, vglob != 0);
    if (ok && m > 0) {
      if (a_df)
        df_householder_tridiag(Af, m, g, reinterpret_cast<float4 *>(hh), slot + 1,
                               slot + 1 + m0);
      else
        householder_tridiag(A, m, g, reinterpret_cast<double2 *>(hh), slot + 1,
                            slot + 1 + m0);
    }
    if (lane == 0) {
      slot[0] = ok ? (double)m : -1.0;
      if (counters && ok) {
        atomicAdd(counters + 1, 1ull);
        if (!chol) atomicAdd(counters + 2, 1ull);
      }
      const int st = ok ? m0 - m : (int)LHF_ERR_NOT_SPD;
      if (s.kstat) {
        s.kstat[kap] = st;
        s.kstat[mk] = st;
      }
      if (!ok) atomicOr(flags, kFlagNotSpd);
    }
    if (!ok && lane < m0) {
      s.eig[(int64_t)kap * m0 + lane] = NAN;
      s.eig[(int64_t)mk * m0 + lane] = NAN;
    }
    return;
  }

  if (ok) {
    // 3. cyclic Jacobi on C (with the eigenvectors of C accumulated in V when requested: V is
    //    free on both routes once C is formed)
    if (s.vecs) {
      for (int e = lane; e < m * m; e += G) {
        const int i = e / m, j = e - (e / m) * m;
        V[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
      }
      g.sync();
    }
    if (!jac_done) sweeps += jacobi_herm(A, s.vecs ? V : nullptr, m, g, R);
    if (lane == 0 && counters) {
      if (!s.tri) atomicAdd(counters, (unsigned long long)sweeps);  // tridiagonal mode counts QR rotations
      atomicAdd(counters + 1, 1ull);
      if (!chol) atomicAdd(counters + 2, 1ull);
    }
  }

  // 4. sort and store (dropped functions and directions: +inf, last); the sort carries the
  //    column of each eigenvalue (ties keep the lower column first)
  double v = (ok && lane < m) ? A[lane * m + lane].x : INFINITY;
  int vid = lane;
  for (int k = 2; k <= G; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      const double o = __shfl_xor_sync(g.mask, v, j);
      const int oid = __shfl_xor_sync(g.mask, vid, j);
      const bool up = (lane & k) == 0, lower = (lane & j) == 0;
      const bool o_less = o < v || (o == v && oid < vid);
      if ((lower == up) == o_less) {
        v = o;
        vid = oid;
      }
    }
  if (!ok) v = NAN;
  if (s.vecs) bloch_vectors(s, kap, mk, ok, chol, m, mkept, g, vid, A, B, V, sg, dsc, kidx);
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

// Eigenvalues of the real symmetric tridiagonal matrices left by k_eig (diagonal d, off-diagonal
// e, order m): G lanes per matrix, lane i finds the i-th smallest eigenvalue, so that the results
// come out sorted and every lane runs the same short recurrence (a one-thread QR iteration per
// matrix is a long serial chain that leaves the GPU idle).
//   * Scaling: T / 2^s with 2^s >= max(|d|, |e|) (exact); the eigenvalues lie in the Gershgorin
//     interval [lo, hi] of the scaled matrix, |lo|, |hi| <= 3 + 2^-20.
//   * Sturm counts: the number of eigenvalues below x is the number of negative pivots of
//     T - x I = L D L^T, r_0 = d_0 - x, r_j = (d_j - x) - e_(j-1)^2 / r_(j-1) (Sylvester's law of
//     inertia).  In FP32 the computed count is the exact count of a matrix within
//     eta ~ 6 eps_32 max|T| < 2^-21 of T (rounding of the recurrence as backward perturbations
//     of the entries), so count32(y) lies between #(lambda < y - eta) and #(lambda < y + eta).
//   * FP32 quadrisection: 12 steps, each shrinking [lo, hi] by 4 with three counts evaluated
//     together (24 halvings), give [a, b] with count32(a) <= i < count32(b);
//     with delta = 2^-19 > 4 eta, count32(a - 2 delta) = i and count32(b + 2 delta) = i + 1 prove
//     that [A, B] = [a - delta, b + delta] holds lambda_i alone, at least delta - eta from either
//     end, and that det(T - x I) has the sign (-1)^i at A.
//   * FP64 Newton's iteration on q_m(x) = det(T - x I) from the leading-minor recurrence
//     q_j = (d_j - x) q_(j-1) - e_(j-1)^2 q_(j-2) and its derivative, kept inside the bracket
//     (bisecting when a step leaves it), stopped once a step is below 2^-40 (with the other
//     eigenvalues at least delta - eta away, the quadratic error of the last step is far below
//     the rounding of q_m).
//   * Otherwise (a cluster closer than 2 delta, or no convergence in 12 steps) bisection on FP64
//     minor counts until lambda_i is alone in the bracket (then Newton again) or the bracket is
//     two adjacent doubles.
// counters[0] accumulates the FP64 recurrence passes (one pass: m steps).
constexpr int kTriMaxThreads = 256;  // threads per CTA: blockDim.x (a multiple of G), set by the launcher
constexpr int kTriMax = kMaxM0;

// q_m(x) = det(T - x I) and its derivative (dn, e2: scaled diagonal and squared off-diagonal,
// |entries| <= 1, |x| <= 4: no overflow; the minors are rescaled by 2^400 every fourth step when
// they have fallen below 2^-400, which leaves the ratio q / q' and the signs unchanged).
__device__ __forceinline__ void tri_det(const double *dn, const double *e2, int m, double x, double &q_out,
                                        double &dq_out) {
  double qm1 = 1.0, q = dn[0] - x, dqm1 = 0.0, dq = -1.0;
  for (int j = 1; j < m; ++j) {
    const double t = dn[j] - x, b = e2[j - 1];
    const double qn = fma(t, q, -b * qm1);
    const double dqn = fma(t, dq, fma(-b, dqm1, -q));
    qm1 = q;
    q = qn;
    dqm1 = dq;
    dq = dqn;
    if ((j & 3) == 3 && fabs(q) < 0x1p-400) {
      q *= 0x1p400;
      qm1 *= 0x1p400;
      dq *= 0x1p400;
      dqm1 *= 0x1p400;
    }
  }
  q_out = q;
  dq_out = dq;
}

// Eigenvalues below x from the signs of the FP64 leading minors (an exact zero minor takes the
// sign opposite to its predecessor; a minor below 2^-400 is rescaled with its predecessor by
// 2^400).  Signs and the range test read the bit patterns (integer operations).
__device__ int tri_count64(const double *dn, const double *e2, int m, double x) {
  double qm1 = 1.0, q = dn[0] - x;
  if (q == 0.0) q = -1e-290;
  int neg = __double_as_longlong(q) < 0 ? 1 : 0;
  int c = neg;
  for (int j = 1; j < m; ++j) {
    double qn = fma(dn[j] - x, q, -e2[j - 1] * qm1);
    if (((__double_as_longlong(qn) >> 52) & 0x7ff) < 1023 - 400) {  // |qn| < 2^-400
      if (qn == 0.0) {
        qn = neg ? 1e-290 : -1e-290;
      } else {
        qn *= 0x1p400;
        q *= 0x1p400;
      }
    }
    const int nn = __double_as_longlong(qn) < 0 ? 1 : 0;
    c += nn ^ neg;
    neg = nn;
    qm1 = q;
    q = qn;
  }
  return c;
}

// Newton's iteration on q_m inside [A, B], which holds lambda_i alone (sign of q_m at A:
// (-1)^i), from x0; bisects when a step leaves the bracket.  True with *x once a step is below
// tol (or q_m vanishes), false after 12 steps.  The error after a step dx is about
// |q''/(2 q')| dx^2 ~ dx^2 / gap: tol = 2^-40 needs a gap of at least ~2^-18 to the other
// eigenvalues, tol = 2^-50 serves any gap.
__device__ bool tri_newton(const double *dn, const double *e2, int m, int i, double A, double B, double x0,
                           double tol, double *x, int *passes) {
  const bool negA = (i & 1) != 0;
  double xc = x0;
  for (int it = 0; it < 12; ++it) {
    double q, dq;
    tri_det(dn, e2, m, xc, q, dq);
    ++*passes;
    if (q == 0.0) {
      *x = xc;
      return true;
    }
    if ((q < 0.0) == negA)
      A = xc;
    else
      B = xc;
    const double dx = dq != 0.0 ? q / dq : INFINITY;
    const double xn = xc - dx;
    if (fabs(dx) <= tol) {
      *x = fmin(fmax(xn, A), B);
      return true;
    }
    xc = (xn > A && xn < B) ? xn : 0.5 * (A + B);
  }
  return false;
}

// Negative pivots of the FP32 L D L^T factorisation of T - x I (an exact zero pivot is taken as
// a tiny negative one).
__device__ int tri_count32(const float *df, const float *e2f, int m, float x) {
  float r = df[0] - x;
  if (r == 0.0f) r = -1e-30f;
  int c = r < 0.0f ? 1 : 0;
  for (int j = 1; j < m; ++j) {
    r = (df[j] - x) - __fdividef(e2f[j - 1], r);
    if (r == 0.0f) r = -1e-30f;
    c += r < 0.0f ? 1 : 0;
  }
  return c;
}

// The same counts at three points at once: three independent recurrences in one loop, so that
// each hides the others' latency (the reciprocals dominate a single chain).
__device__ __forceinline__ void tri_count32x3(const float *df, const float *e2f, int m, float x0, float x1, float x2,
                                              int &c0, int &c1, int &c2) {
  float r0 = df[0] - x0, r1 = df[0] - x1, r2 = df[0] - x2;
  if (r0 == 0.0f) r0 = -1e-30f;
  if (r1 == 0.0f) r1 = -1e-30f;
  if (r2 == 0.0f) r2 = -1e-30f;
  c0 = r0 < 0.0f ? 1 : 0;
  c1 = r1 < 0.0f ? 1 : 0;
  c2 = r2 < 0.0f ? 1 : 0;
  for (int j = 1; j < m; ++j) {
    const float d = df[j], e = e2f[j - 1];
    r0 = (d - x0) - __fdividef(e, r0);
    r1 = (d - x1) - __fdividef(e, r1);
    r2 = (d - x2) - __fdividef(e, r2);
    if (r0 == 0.0f) r0 = -1e-30f;
    if (r1 == 0.0f) r1 = -1e-30f;
    if (r2 == 0.0f) r2 = -1e-30f;
    c0 += r0 < 0.0f ? 1 : 0;
    c1 += r1 < 0.0f ? 1 : 0;
    c2 += r2 < 0.0f ? 1 : 0;
  }
}

template <int G>
__global__ void __launch_bounds__(kTriMaxThreads) k_tridiag_eig(const SysDev *__restrict__ sysv, unsigned *flags,
                                                              unsigned long long *counters) {
  (void)flags;
  const SysDev &s = sysv[blockIdx.y];
  if (s.box || !s.tri || !s.klist) return;
  const int gi = threadIdx.x / G, i = threadIdx.x % G;  // group (matrix) in the CTA, eigenvalue index
  const int widx = blockIdx.x * (int)(blockDim.x / G) + gi;
  if (widx >= s.nkhalf) return;  // uniform over the group
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  const int m0 = s.m0;
  const double *slot = s.tri + (int64_t)widx * (2 * m0 + 1);
  const int m = (int)slot[0];
  if (m < 0) return;  // -1: not positive definite (NaN written by k_eig); -2: solved by k_eig
  // per matrix of the CTA: d and e^2 in FP64 and FP32 (shared memory sized by the launch, so
  // that small CTAs keep many matrices resident: the kernel is bound by its dependent chains)
  extern __shared__ double trsm[];
  const int groups = (int)(blockDim.x / G);
  double *dn = trsm + (size_t)gi * kTriMax, *e2 = trsm + (size_t)(groups + gi) * kTriMax;
  float *df = reinterpret_cast<float *>(trsm + (size_t)2 * groups * kTriMax) + (size_t)gi * kTriMax;
  float *e2f = reinterpret_cast<float *>(trsm + (size_t)2 * groups * kTriMax) + (size_t)(groups + gi) * kTriMax;
  // scale 2^ex >= max |entries|
  const double di = i < m ? slot[1 + i] : 0.0;
  const double ei = i + 1 < m ? slot[1 + m0 + i] : 0.0;
  double mx = fmax(fabs(di), fabs(ei));
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(gmask, mx, o));
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);
  const double dni = scale_pow2(di, -ex), eni = scale_pow2(ei, -ex);
  if (i < m) {
    dn[i] = dni;
    e2[i] = eni * eni;
    df[i] = (float)dni;
    e2f[i] = (float)(eni * eni);
  }
  // Gershgorin interval of the scaled matrix
  const double eprev = __shfl_up_sync(gmask, eni, 1, G);
  const double rad = fabs(eni) + (i > 0 ? fabs(eprev) : 0.0);
  double lo = i < m ? dni - rad : 1e300, hi = i < m ? dni + rad : -1e300;
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(gmask, lo, o));
    hi = fmax(hi, __shfl_xor_sync(gmask, hi, o));
  }
  lo -= 0x1p-20;
  hi += 0x1p-20;
  __syncwarp(gmask);
  double x = INFINITY;
  int passes = 0;
  if (i < m) {
    // FP32 quadrisection on the pivot counts (count(a) <= i < count(b) throughout): three points
    // per step, the bracket shrinks by 4, 12 steps as 24 of bisection
    float a = (float)lo, b = (float)hi;
    for (int it = 0; it < 12; ++it) {
      const float w = b - a;
      const float p1 = a + 0.25f * w, p2 = a + 0.5f * w, p3 = a + 0.75f * w;
      int c1, c2, c3;
      tri_count32x3(df, e2f, m, p1, p2, p3, c1, c2, c3);
      if (c1 > i) {
        b = p1;
      } else if (c2 > i) {
        a = p1;
        b = p2;
      } else if (c3 > i) {
        a = p2;
        b = p3;
      } else {
        a = p3;
      }
    }
    // isolation margin delta = 2^-19 > 4 eta (eta: the FP32 counts' backward error, above);
    // eigenvalues closer than ~2 delta go to the cluster path below
    const double delta = 0x1p-19;
    bool done = false;
    if (tri_count32(df, e2f, m, (float)((double)a - 2.0 * delta)) == i &&
        tri_count32(df, e2f, m, (float)((double)b + 2.0 * delta)) == i + 1)
      done = tri_newton(dn, e2, m, i, (double)a - delta, (double)b + delta, 0.5 * ((double)a + (double)b), 0x1p-40,
                        &x, &passes);
    if (!done) {
      // a cluster: bisection on FP64 minor counts, count(A) <= i < count(B), from the FP32
      // bracket when the FP64 counts confirm it, until lambda_i is alone in [A, B] (then
      // Newton) or the bracket is two adjacent doubles
      double A = (double)a - 2.0 * delta, B = (double)b + 2.0 * delta;
      int cA = tri_count64(dn, e2, m, A), cB = tri_count64(dn, e2, m, B);
      passes += 2;
      if (cA > i) {
        A = lo;
        cA = 0;
      }
      if (cB <= i) {
        B = hi;
        cB = m;
      }
      bool newton_tried = false;
      for (int it = 0; it < 120; ++it) {
        if (!newton_tried && cA == i && cB == i + 1) {
          newton_tried = true;
          if (tri_newton(dn, e2, m, i, A, B, 0.5 * (A + B), 0x1p-50, &x, &passes)) {
            done = true;
            break;
          }
        }
        const double mid = 0.5 * (A + B);
        if (!(mid > A && mid < B)) break;
        const int c = tri_count64(dn, e2, m, mid);
        ++passes;
        if (c <= i) {
          A = mid;
          cA = c;
        } else {
          B = mid;
          cB = c;
        }
      }
      if (!done) x = 0.5 * (A + B);
    }
    x = scale_pow2(x, ex);
  }
  const int kap = s.klist[widx];
  const int L0 = s.d[0].L, L1 = s.d[1].L, L2 = s.d[2].L;
  const int k0 = kap / (L1 * L2), k1 = (kap / L2) % L1, k2 = kap % L2;
  const int mk = (((L0 - k0) % L0) * L1 + (L1 - k1) % L1) * L2 + (L2 - k2) % L2;
  if (i < m0) {
    s.eig[(int64_t)kap * m0 + i] = x;  // +inf in the removed slots i >= m
    s.eig[(int64_t)mk * m0 + i] = x;
  }
  if (counters) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) passes += __shfl_xor_sync(gmask, passes, o);
    if (i == 0) atomicAdd(counters, (unsigned long long)passes);
  }
}

}  // namespace

cudaError_t launch_overlap_norms(const SysDev *sys, int nsys, cudaStream_t st) {
  if (nsys <= 0) return cudaSuccess;
  kmark(LHF_K_OVERLAP_NORMS, 1, st);
  k_overlap_norms<<<dim3(1, nsys), 256, 0, st>>>(sys);
  kmark(LHF_K_OVERLAP_NORMS, 0, st);
  return cudaGetLastError();
}

// Lanes per matrix: half a warp up to order 16 (the FP64 scalar steps then cost one warp
// instruction per two matrices), a whole warp otherwise or when `full` (the pair arithmetic of the
// mixed route, whose scalar steps are FP32: a warp per matrix halves the shared memory per warp and
// gives two lanes to each column of the triangular solves).
static inline int eig_group(int max_m0, bool full) { return (max_m0 <= 16 && !full) ? 16 : 32; }

int eig_max_warps(int max_m0, bool full, bool vglob) {
  const int per_warp = 32 / eig_group(max_m0, full);
  int w = kEigMaxWarps;
  while (w > 1 && (size_t)w * per_warp * eig_warp_bytes(max_m0, vglob) > 227 * 1024) --w;
  return w;
}

template <int G>
static cudaError_t launch_k_eig(const SysDev *sys, int nsys, int max_k, int max_m0, unsigned *flags,
                                unsigned long long *counters, cudaStream_t st, int warps, bool vglob) {
  const int per_cta = warps * (32 / G);
  const size_t smem = (size_t)per_cta * eig_warp_bytes(max_m0, vglob);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_eig<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((max_k + per_cta - 1) / per_cta, nsys);
  kmark(LHF_K_EIG, 1, st);
  k_eig<G><<<grid, warps * 32, smem, st>>>(sys, flags, counters, max_m0, vglob ? 1 : 0);
  kmark(LHF_K_EIG, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_eig_reduce(const SysDev *sys, int nsys, int max_k, int max_m0, unsigned *flags,
                              unsigned long long *counters, cudaStream_t st, int warps, bool full, bool vglob) {
  if (max_k <= 0 || nsys <= 0) return cudaSuccess;
  if (warps < 1 || warps > eig_max_warps(max_m0, full, vglob)) return cudaErrorInvalidValue;
  return eig_group(max_m0, full) == 16 ? launch_k_eig<16>(sys, nsys, max_k, max_m0, flags, counters, st, warps, vglob)
                                       : launch_k_eig<32>(sys, nsys, max_k, max_m0, flags, counters, st, warps, vglob);
}

cudaError_t launch_tridiag(const SysDev *sys, int nsys, int max_k, int max_m0, unsigned *flags,
                           unsigned long long *counters, cudaStream_t st, int threads) {
  if (max_k <= 0 || nsys <= 0) return cudaSuccess;
  // G lanes per matrix (one per eigenvalue): 16 when every order fits, else 32
  const int G = max_m0 <= 16 ? 16 : 32;
  if (threads < G || threads > kTriMaxThreads || threads % G != 0) return cudaErrorInvalidValue;
  const int per = threads / G;
  const size_t smem = (size_t)per * kTriMax * (2 * sizeof(double) + 2 * sizeof(float));  // <= 6 KB
  kmark(LHF_K_TRIDIAG_EIG, 1, st);
  if (G == 16)
    k_tridiag_eig<16><<<dim3((max_k + per - 1) / per, nsys), threads, smem, st>>>(sys, flags, counters);
  else
    k_tridiag_eig<32><<<dim3((max_k + per - 1) / per, nsys), threads, smem, st>>>(sys, flags, counters);
  kmark(LHF_K_TRIDIAG_EIG, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_eig(const SysDev *sys, int nsys, int max_k, int max_m0, unsigned *flags,
                       unsigned long long *counters, cudaStream_t st, bool tri, int eig_warps, int tri_threads,
                       bool full, bool vglob) {
  cudaError_t e = launch_eig_reduce(sys, nsys, max_k, max_m0, flags, counters, st, eig_warps, full, vglob);
  if (e != cudaSuccess || !tri) return e;
  return launch_tridiag(sys, nsys, max_k, max_m0, flags, counters, st, tri_threads);
}

}  // namespace lhf
