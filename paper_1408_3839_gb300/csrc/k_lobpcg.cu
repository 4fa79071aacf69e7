// k_lobpcg.cu -- step a9 for large open boxes: the lowest eigenvalues of the (L,1,1) box without a
// dense eigensolve.
//
// In the box (Sec. 3.3, eqs. (3.8)-(3.10)) the Galerkin matrices are block-banded: the block of
// cells (p, q) vanishes unless the supports of the two cells' functions meet, |q - p| inside the
// overlap window (Lemma 3.1).  Their overlap and kinetic parts are block-Toeplitz (they depend on
// q - p only) and the nuclear part differs from a Toeplitz one only through the finite set of
// nuclei; a block-Toeplitz matrix embeds into a block-circulant one of larger size (Remark 2.4),
// which the DFT along the cells block-diagonalises (Lemma 2.2).  The solver:
//   * band: H and S as [L][bJ][m0][m0] blocks, row cell p, column cell p + d, d = bjlo + dd;
//   * matvec: Y_H = H X and Y_S = S X for a block of vectors, O(L bJ m0^2) per vector;
//   * preconditioner: the block-circulant matrix of M >= L + bJ cells (M a power of two) whose
//     blocks are the box's band blocks averaged over the rows (each block diagonal replaced by its
//     mean, the optimal circulant of a Toeplitz-like matrix), P_d = Havg_d - sigma Savg_d; in k-space it is
//     the m0 x m0 Hermitian block Pbar_kappa = Hbar_kappa - sigma Sbar_kappa per kappa (Prop. 6.1),
//     positive definite for sigma below the bulk spectrum, applied as zero padding to M cells,
//     DFT, Cholesky solves per kappa, inverse DFT, restriction to the L box cells;
//   * LOBPCG: Rayleigh-Ritz on span[X, W, P] (iterates, preconditioned residuals, previous
//     directions), the small pencil solved in one CTA by canonical orthogonalisation (cyclic
//     Jacobi with vectors on the scaled Gram matrix, directions below a threshold dropped) and
//     cyclic Jacobi on the projected matrix.
// Everything runs in FP64.  Vectors are stored [k][N] (one vector contiguous), N = L m0, row
// (p, mu) = p m0 + mu.
#include <math.h>

#include "lhf_internal.cuh"

namespace lhf {
namespace {

// ---- band assembly ------------------------------------------------------------------------
// H, S band blocks of one box from its factors (the rank sum of k_box_assemble, band layout).
__global__ void __launch_bounds__(256) k_box_band(const SysDev *__restrict__ sysv, double *Hband,
                                                 double *Sband) {
  const SysDev &s = sysv[0];
  const int m0 = s.m0, mm = m0 * m0, Rt = s.Rt, slots = Rt + 2, L0 = s.d[0].L;
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= (int64_t)L0 * s.bJ * mm) return;
  const int e = (int)(item % mm);
  const int64_t pd = item / mm;
  const int dd = (int)(pd % s.bJ), p = (int)(pd / s.bJ);
  const int q = p + s.bjlo + dd;
  double h = 0.0, sv = 0.0;
  if (q >= 0 && q < L0) {
    const double *F0 = s.ws + s.offCb + ((int64_t)p * s.bJ + dd) * slots * mm + e;
    const double *F1 = s.ws + s.d[1].offC + e;
    const double *F2 = s.ws + s.d[2].offC + e;
    double v = 0.0;
    for (int r = 0; r < Rt; ++r) {
      const int64_t o = (int64_t)r * mm;
      v += s.c[r] * F0[o] * F1[o] * F2[o];
    }
    const int64_t ok = (int64_t)Rt * mm, om = (int64_t)(Rt + 1) * mm;
    const double K0 = F0[ok], K1 = F1[ok], K2 = F2[ok];
    const double M0 = F0[om], M1 = F1[om], M2 = F2[om];
    sv = M0 * M1 * M2;
    h = 0.5 * (K0 * M1 * M2 + M0 * K1 * M2 + M0 * M1 * K2) - v;
  }
  Hband[item] = h;
  Sband[item] = sv;
}

// ---- banded matvec ------------------------------------------------------------------------
// One CTA per cell row p, one thread per (vector c, function mu): YH = H X, YS = S X.
__global__ void k_band_mv(const double *__restrict__ Hb, const double *__restrict__ Sb,
                          const double *__restrict__ X, double *YH, double *YS, int L, int bJ, int bjlo,
                          int m0, int kv, int64_t N) {
  const int p = blockIdx.x;
  const int mm = m0 * m0;
  for (int t = threadIdx.x; t < kv * m0; t += blockDim.x) {
    const int c = t / m0, mu = t - (t / m0) * m0;
    const double *x = X + (int64_t)c * N;
    double ah = 0.0, as = 0.0;
    for (int dd = 0; dd < bJ; ++dd) {
      const int q = p + bjlo + dd;
      if (q < 0 || q >= L) continue;
      const double *hrow = Hb + ((int64_t)p * bJ + dd) * mm + mu * m0;
      const double *srow = Sb + ((int64_t)p * bJ + dd) * mm + mu * m0;
      const double *xq = x + (int64_t)q * m0;
      for (int nu = 0; nu < m0; ++nu) {
        const double xv = xq[nu];
        ah = fma(__ldg(hrow + nu), xv, ah);
        as = fma(__ldg(srow + nu), xv, as);
      }
    }
    YH[(int64_t)c * N + (int64_t)p * m0 + mu] = ah;
    YS[(int64_t)c * N + (int64_t)p * m0 + mu] = as;
  }
}

// ---- preconditioner -----------------------------------------------------------------------
// Averages of the band blocks over the rows where they exist (the blocks of the optimal
// circulant approximation of a Toeplitz-like matrix: each diagonal replaced by its mean), thread
// per (dd, entry): out [bJ][m0][m0].
__global__ void k_band_average(const double *__restrict__ Hb, const double *__restrict__ Sb, int L, int bJ,
                               int bjlo, int m0, double *Ha, double *Sa) {
  const int mm = m0 * m0;
  const int item = blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= bJ * mm) return;
  const int dd = item / mm, e = item - (item / mm) * mm;
  const int d = bjlo + dd;
  double h = 0.0, sv = 0.0;
  int cnt = 0;
  for (int p = 0; p < L; ++p) {
    if (p + d < 0 || p + d >= L) continue;
    h += Hb[((int64_t)p * bJ + dd) * mm + e];
    sv += Sb[((int64_t)p * bJ + dd) * mm + e];
    ++cnt;
  }
  Ha[item] = cnt ? h / cnt : 0.0;
  Sa[item] = cnt ? sv / cnt : 0.0;
}

// Hbar_kappa, Sbar_kappa of the middle row's blocks on the circulant of M cells, whose row p holds
// the block X_mid,d in column p + d: with the forward DFT xhat_kappa = sum_p exp(-2 pi i kappa p / M)
// x_p, the product becomes yhat_kappa = Xbar_kappa xhat_kappa with
// Xbar_kappa[mu][nu] = sum_d exp(+2 pi i kappa d / M) X_mid,d[mu][nu] (thread per (kappa, mu, nu)).
__global__ void k_prec_blocks(const double *__restrict__ Hb, const double *__restrict__ Sb, int mid, int bJ,
                              int bjlo, int m0, int M, double2 *Hk, double2 *Sk) {
  const int mm = m0 * m0;
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= (int64_t)M * mm) return;
  const int kap = (int)(item / mm), e = (int)(item % mm);
  double hr = 0.0, hi = 0.0, sr = 0.0, si = 0.0;
  for (int dd = 0; dd < bJ; ++dd) {
    const int d = bjlo + dd;
    // exp(+2 pi i kappa d / M) with the phase reduced mod M exactly in integers
    long long ph = ((long long)kap * d) % M;
    if (ph < 0) ph += M;
    double sn, cs;
    sincospi(2.0 * (double)ph / (double)M, &sn, &cs);
    const double h = Hb[((int64_t)mid * bJ + dd) * mm + e], sv = Sb[((int64_t)mid * bJ + dd) * mm + e];
    hr = fma(cs, h, hr);
    hi = fma(sn, h, hi);
    sr = fma(cs, sv, sr);
    si = fma(sn, sv, si);
  }
  Hk[item] = make_double2(hr, hi);
  Sk[item] = make_double2(sr, si);
}

// Cholesky of the Hermitian part of Pbar_kappa = Hbar - sigma Sbar per kappa (thread per kappa),
// lower factor in Lk with 1 / L_jj on the diagonal; a non-positive pivot raises *bad.
__global__ void k_prec_factor(const double2 *__restrict__ Hk, const double2 *__restrict__ Sk, double sigma,
                              int m0, int M, double2 *Lk, unsigned *bad) {
  const int kap = blockIdx.x * blockDim.x + threadIdx.x;
  if (kap >= M) return;
  const int mm = m0 * m0;
  const double2 *H = Hk + (int64_t)kap * mm;
  const double2 *S = Sk + (int64_t)kap * mm;
  double2 *A = Lk + (int64_t)kap * mm;
  // lower triangle of the Hermitian part
  for (int i = 0; i < m0; ++i)
    for (int j = 0; j <= i; ++j) {
      const double2 a = H[i * m0 + j], b = H[j * m0 + i], c = S[i * m0 + j], d = S[j * m0 + i];
      const double re = 0.5 * (a.x + b.x) - sigma * 0.5 * (c.x + d.x);
      const double im = (i == j) ? 0.0 : 0.5 * (a.y - b.y) - sigma * 0.5 * (c.y - d.y);
      A[i * m0 + j] = make_double2(re, im);
    }
  bool ok = true;
  for (int j = 0; j < m0 && ok; ++j) {
    double dj = A[j * m0 + j].x;
    for (int k = 0; k < j; ++k) dj -= A[j * m0 + k].x * A[j * m0 + k].x + A[j * m0 + k].y * A[j * m0 + k].y;
    if (!(dj > 0.0)) {
      ok = false;
      break;
    }
    const double ljj = sqrt(dj), inv = 1.0 / ljj;
    A[j * m0 + j] = make_double2(inv, 0.0);
    for (int i = j + 1; i < m0; ++i) {
      double2 v = A[i * m0 + j];
      for (int k = 0; k < j; ++k) {  // v -= L_ik conj(L_jk)
        const double2 a = A[i * m0 + k], b = A[j * m0 + k];
        v.x -= a.x * b.x + a.y * b.y;
        v.y -= a.y * b.x - a.x * b.y;
      }
      A[i * m0 + j] = make_double2(v.x * inv, v.y * inv);
    }
  }
  if (!ok) atomicOr(bad, 1u);
}

// In-place radix-2 FFT of M = 2^bits complex values in shared memory (sign -1: forward).
__device__ void fft_shared(double2 *x, int M, int bits, double sign) {
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const int j = (int)(__brev((unsigned)i) >> (32 - bits));
    if (j > i) {
      const double2 t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
  __syncthreads();
  for (int hs = 1; hs < M; hs <<= 1) {
    for (int k = threadIdx.x; k < M / 2; k += blockDim.x) {
      const int kk = k % hs, top = (k / hs) * 2 * hs + kk, bot = top + hs;
      double sn, cs;
      sincospi((double)kk / (double)hs, &sn, &cs);  // exp(sign i pi kk / hs)
      const double wr = cs, wi = sign * sn;
      const double2 u = x[top], v = x[bot];
      const double2 wv = make_double2(wr * v.x - wi * v.y, wr * v.y + wi * v.x);
      x[top] = make_double2(u.x + wv.x, u.y + wv.y);
      x[bot] = make_double2(u.x - wv.x, u.y - wv.y);
    }
    __syncthreads();
  }
}

// Forward: the series of vector c, component nu over the box cells, zero-padded to M cells,
// transformed (CTA per (c, nu)); out [c][kappa][nu].
__global__ void k_vec_fft_fwd(const double *__restrict__ X, double2 *out, int L, int m0, int M, int bits,
                              int64_t N) {
  extern __shared__ double2 xs[];
  const int c = blockIdx.x / m0, nu = blockIdx.x % m0;
  for (int p = threadIdx.x; p < M; p += blockDim.x)
    xs[p] = make_double2(p < L ? X[(int64_t)c * N + (int64_t)p * m0 + nu] : 0.0, 0.0);
  __syncthreads();
  fft_shared(xs, M, bits, -1.0);
  for (int k = threadIdx.x; k < M; k += blockDim.x) out[((int64_t)c * M + k) * m0 + nu] = xs[k];
}

// Inverse: back to cell space (scaled by 1 / M), real part on the box cells.
__global__ void k_vec_fft_inv(const double2 *__restrict__ in, double *Y, int L, int m0, int M, int bits,
                              int64_t N) {
  extern __shared__ double2 xs[];
  const int c = blockIdx.x / m0, nu = blockIdx.x % m0;
  for (int k = threadIdx.x; k < M; k += blockDim.x) xs[k] = in[((int64_t)c * M + k) * m0 + nu];
  __syncthreads();
  fft_shared(xs, M, bits, 1.0);
  const double inv = 1.0 / (double)M;
  for (int p = threadIdx.x; p < L; p += blockDim.x) Y[(int64_t)c * N + (int64_t)p * m0 + nu] = xs[p].x * inv;
}

// y = Pbar_kappa^{-1} x per (vector, kappa): forward and back substitution with the Cholesky factor.
__global__ void k_prec_solve(const double2 *__restrict__ Lk, double2 *V, int m0, int M, int kv) {
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= (int64_t)kv * M) return;
  const int kap = (int)(item % M);
  const double2 *A = Lk + (int64_t)kap * m0 * m0;
  double2 *x = V + item * m0;
  double2 z[kMaxM0];
  for (int i = 0; i < m0; ++i) {  // L z = x
    double2 v = x[i];
    for (int k = 0; k < i; ++k) {
      const double2 a = A[i * m0 + k];
      v.x -= a.x * z[k].x - a.y * z[k].y;
      v.y -= a.x * z[k].y + a.y * z[k].x;
    }
    const double d = A[i * m0 + i].x;
    z[i] = make_double2(v.x * d, v.y * d);
  }
  for (int i = m0 - 1; i >= 0; --i) {  // L^H y = z
    double2 v = z[i];
    for (int k = i + 1; k < m0; ++k) {  // conj(L_ki) y_k
      const double2 a = A[k * m0 + i];
      v.x -= a.x * z[k].x + a.y * z[k].y;
      v.y -= a.x * z[k].y - a.y * z[k].x;
    }
    const double d = A[i * m0 + i].x;
    z[i] = make_double2(v.x * d, v.y * d);
  }
  for (int i = 0; i < m0; ++i) x[i] = z[i];
}

// ---- exact shifted factorisation (block-tridiagonal Cholesky) ------------------------------
// Cells grouped into super-cells of g cells (g >= the band's reach in cells) make H - sigma S
// block-tridiagonal with blocks of B = g m0 rows; nb = ceil(L / g) blocks, the last one padded
// with identity rows.  D[i] = the diagonal block i, E[i] = the block (i, i - 1) (i >= 1).
__global__ void k_tri_blocks(const double *__restrict__ Hb, const double *__restrict__ Sb, double sigma, int L,
                             int bJ, int bjlo, int m0, int g, int nb, double *D, double *E) {
  const int B = g * m0;
  const int64_t BB = (int64_t)B * B;
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= 2 * (int64_t)nb * BB) return;
  const int which = (int)(item / ((int64_t)nb * BB));  // 0: D, 1: E
  const int64_t rest = item - (int64_t)which * nb * BB;
  const int i = (int)(rest / BB);
  const int r = (int)((rest % BB) / B), col = (int)(rest % B);
  const int p = i * g + r / m0, mu = r % m0;
  const int q = (which == 0 ? i : i - 1) * g + col / m0, nu = col % m0;
  double v = 0.0;
  if (which == 0 && p >= L) {
    v = (r == col) ? 1.0 : 0.0;  // padding rows of the last block
  } else if (p < L && q >= 0 && q < L) {
    const int dd = q - p - bjlo;
    if (dd >= 0 && dd < bJ) {
      const int64_t o = ((int64_t)p * bJ + dd) * m0 * m0 + mu * m0 + nu;
      v = Hb[o] - sigma * Sb[o];
    }
  }
  (which == 0 ? D : E)[rest] = v;
}

// Block-tridiagonal Cholesky in place, one CTA, block rows in order: E[i] <- E[i] L[i-1]^-T,
// D[i] <- D[i] - E[i] E[i]^T, D[i] <- chol(D[i]) (lower, the diagonal holding 1 / L_jj).  A
// non-positive pivot sets *bad and stops (sigma is not below the spectrum).
__global__ void __launch_bounds__(1024) k_tri_factor(double *D, double *E, int B, int nb, unsigned *bad) {
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int i = 0; i < nb; ++i) {
    double *Di = D + (int64_t)i * B * B;
    if (i > 0) {
      const double *Lp = D + (int64_t)(i - 1) * B * B;
      double *Ei = E + (int64_t)i * B * B;
      // rows of E[i]: solve L_{i-1} f = e (forward, per row; thread per row)
      for (int r = threadIdx.x; r < B; r += blockDim.x) {
        double *e = Ei + (int64_t)r * B;
        for (int j = 0; j < B; ++j) {
          double v = e[j];
          for (int k = 0; k < j; ++k) v -= Lp[(int64_t)j * B + k] * e[k];
          e[j] = v * Lp[(int64_t)j * B + j];
        }
      }
      __syncthreads();
      // D[i] -= E[i] E[i]^T on the lower triangle
      for (int64_t t = threadIdx.x; t < (int64_t)B * B; t += blockDim.x) {
        const int r = (int)(t / B), cc = (int)(t % B);
        if (cc > r) continue;
        const double *er = Ei + (int64_t)r * B, *ec = Ei + (int64_t)cc * B;
        double acc = 0.0;
        for (int k = 0; k < B; ++k) acc = fma(er[k], ec[k], acc);
        Di[t] -= acc;
      }
      __syncthreads();
    }
    // Cholesky of D[i], right-looking, column by column
    for (int j = 0; j < B; ++j) {
      const double d = Di[(int64_t)j * B + j];
      if (!(d > 0.0)) {
        if (threadIdx.x == 0) {
          fail = 1;
          atomicOr(bad, 1u);
        }
      }
      __syncthreads();
      if (fail) return;
      const double inv = rsqrt(d);
      for (int r = j + 1 + threadIdx.x; r < B; r += blockDim.x) Di[(int64_t)r * B + j] *= inv;
      __syncthreads();
      if (threadIdx.x == 0) Di[(int64_t)j * B + j] = inv;
      // trailing lower triangle: D[r][c] -= L[r][j] L[c][j], j < c <= r
      const int n = B - j - 1;
      for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
        const int r = j + 1 + (int)(t / n), cc = j + 1 + (int)(t % n);
        if (cc > r) continue;
        Di[(int64_t)r * B + cc] -= Di[(int64_t)r * B + j] * Di[(int64_t)cc * B + j];
      }
      __syncthreads();
    }
  }
}

// x = (H - sigma S)^{-1} b for kv vectors with the block-tridiagonal factor (CTA per vector):
// forward y_i = L_ii^{-1} (b_i - L_{i,i-1} y_{i-1}), backward x_i = L_ii^{-T} (y_i - L_{i+1,i}^T x_{i+1}).
// Y [kv][N] holds b on entry and x on exit; scratch V [kv][nb B].
__global__ void __launch_bounds__(256) k_tri_solve(const double *__restrict__ D, const double *__restrict__ E,
                                                   int B, int nb, int64_t N, double *Y, double *V) {
  const int c = blockIdx.x;
  double *y = V + (int64_t)c * nb * B;
  double *out = Y + (int64_t)c * N;
  for (int64_t t = threadIdx.x; t < (int64_t)nb * B; t += blockDim.x) y[t] = t < N ? out[t] : 0.0;
  __syncthreads();
  for (int i = 0; i < nb; ++i) {
    double *yi = y + (int64_t)i * B;
    const double *Li = D + (int64_t)i * B * B;
    if (i > 0) {
      const double *Ei = E + (int64_t)i * B * B, *yp = y + (int64_t)(i - 1) * B;
      for (int r = threadIdx.x; r < B; r += blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < B; ++k) acc = fma(Ei[(int64_t)r * B + k], yp[k], acc);
        yi[r] -= acc;
      }
      __syncthreads();
    }
    for (int j = 0; j < B; ++j) {  // column-oriented forward substitution
      if (threadIdx.x == 0) yi[j] *= Li[(int64_t)j * B + j];
      __syncthreads();
      const double yj = yi[j];
      for (int r = j + 1 + threadIdx.x; r < B; r += blockDim.x) yi[r] -= Li[(int64_t)r * B + j] * yj;
      __syncthreads();
    }
  }
  for (int i = nb - 1; i >= 0; --i) {
    double *yi = y + (int64_t)i * B;
    const double *Li = D + (int64_t)i * B * B;
    if (i < nb - 1) {
      const double *En = E + (int64_t)(i + 1) * B * B, *xn = y + (int64_t)(i + 1) * B;
      for (int r = threadIdx.x; r < B; r += blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < B; ++k) acc = fma(En[(int64_t)k * B + r], xn[k], acc);
        yi[r] -= acc;
      }
      __syncthreads();
    }
    for (int j = B - 1; j >= 0; --j) {  // L_ii^T x = y, row j of L^T is column j of L
      if (threadIdx.x == 0) yi[j] *= Li[(int64_t)j * B + j];
      __syncthreads();
      const double xj = yi[j];
      for (int r = threadIdx.x; r < j; r += blockDim.x) yi[r] -= Li[(int64_t)j * B + r] * xj;
      __syncthreads();
    }
  }
  for (int64_t t = threadIdx.x; t < N; t += blockDim.x) out[t] = y[t];
}

// ---- Gram matrices and linear combinations ------------------------------------------------
// G[i][j] = sum_n Z[i][n] Y[j][n] for i, j < n (CTA per pair i <= j, fixed-order reduction;
// both triangles written).
__global__ void __launch_bounds__(256) k_gram_vec(const double *__restrict__ Z, const double *__restrict__ Y,
                                                  int nz, int64_t N, double *G, int ldg) {
  const int i = blockIdx.y, j = blockIdx.x;
  if (j < i || j >= nz || i >= nz) return;
  const double *a = Z + (int64_t)i * N, *b = Y + (int64_t)j * N;
  const double *a2 = Z + (int64_t)j * N, *b2 = Y + (int64_t)i * N;
  double acc = 0.0, acc2 = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += 256) {
    acc = fma(a[n], b[n], acc);
    acc2 = fma(a2[n], b2[n], acc2);
  }
  __shared__ double red[2][8];
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = acc;
    red[1][threadIdx.x >> 5] = acc2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0, s2 = 0.0;
    for (int w = 0; w < 8; ++w) {
      s += red[0][w];
      s2 += red[1][w];
    }
    // the symmetrised value (Z^T Y is symmetric in exact arithmetic for Y = H Z, S Z)
    const double v = 0.5 * (s + s2);
    G[i * ldg + j] = v;
    G[j * ldg + i] = v;
  }
}

// out[c][n] = sum_{j = j0}^{j1 - 1} C[j][c] Z[j][n], c < kv (thread per (c, n)).
__global__ void k_lincomb(const double *__restrict__ Z, const double *__restrict__ C, int ldc, int j0, int j1,
                          int kv, int64_t N, double *out) {
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= (int64_t)kv * N) return;
  const int c = (int)(item / N);
  const int64_t n = item - (int64_t)c * N;
  double acc = 0.0;
  for (int j = j0; j < j1; ++j) acc = fma(C[j * ldc + c], Z[(int64_t)j * N + n], acc);
  out[item] = acc;
}

// R[c] = YH[c] - theta_c YS[c]; rnorm[c] = ||R[c]|| (CTA per vector).
__global__ void __launch_bounds__(256) k_residual(const double *__restrict__ YH, const double *__restrict__ YS,
                                                  const double *__restrict__ theta, int64_t N, double *R,
                                                  double *rnorm) {
  const int c = blockIdx.x;
  const double th = theta[c];
  double acc = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += 256) {
    const double r = YH[(int64_t)c * N + n] - th * YS[(int64_t)c * N + n];
    R[(int64_t)c * N + n] = r;
    acc = fma(r, r, acc);
  }
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    rnorm[c] = sqrt(s);
  }
}

// Seeded start vectors: a counter-based hash of (seed, c, n) mapped to [-1, 1).
__global__ void k_start_vectors(double *X, int kv, int64_t N, unsigned long long seed) {
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= (int64_t)kv * N) return;
  unsigned long long z = seed + 0x9e3779b97f4a7c15ull * (unsigned long long)(item + 1);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  X[item] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// ---- the small Rayleigh-Ritz pencil --------------------------------------------------------
constexpr int kRRMax = 72;  // largest subspace (3 x 24 vectors)

// Cyclic Jacobi with vectors on the symmetric n x n matrix A (shared, row-major, lda = kRRMax),
// one CTA: each step rotates n'/2 disjoint pairs (round-robin); A <- J^T A J, V <- V J.
__device__ void jacobi_sym(double *A, double *V, int n, double *rc, double *rs, int *rp, int *rq) {
  const int np = (n + 1) / 2 * 2, half = np / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    // off-diagonal norm against the total
    __shared__ double offs, tot;
    if (threadIdx.x == 0) {
      offs = 0.0;
      tot = 0.0;
    }
    __syncthreads();
    double o = 0.0, t = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e - (e / n) * n;
      const double v = A[i * kRRMax + j];
      t += v * v;
      if (i != j) o += v * v;
    }
    atomicAdd(&offs, o);
    atomicAdd(&tot, t);
    __syncthreads();
    if (!(offs > 1e-30 * tot)) break;
    for (int step = 0; step < np - 1; ++step) {
      // pair k: positions k and np - 1 - k of the round-robin ring (player np-1 fixed)
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        // circle method: player np - 1 fixed, the others rotate by one per step
        int a, b;
        if (k == 0) {
          a = step;
          b = np - 1;
        } else {
          a = (step + k) % (np - 1);
          b = (step - k + (np - 1)) % (np - 1);
        }
        int p = min(a, b), q = max(a, b);
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = A[p * kRRMax + q];
          if (fabs(apq) > 1e-300) {
            const double th = (A[q * kRRMax + q] - A[p * kRRMax + p]) / (2.0 * apq);
            const double tt = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(tt * tt + 1.0);
            s = tt * c;
          }
        } else {
          q = p;  // idle pair
        }
        rc[k] = c;
        rs[k] = s;
        rp[k] = p;
        rq[k] = q;
      }
      __syncthreads();
      // columns: A[:, p], A[:, q]
      for (int e = threadIdx.x; e < half * n; e += blockDim.x) {
        const int k = e / n, i = e - (e / n) * n;
        const int p = rp[k], q = rq[k];
        if (p == q) continue;
        const double c = rc[k], s = rs[k];
        const double ap = A[i * kRRMax + p], aq = A[i * kRRMax + q];
        A[i * kRRMax + p] = c * ap - s * aq;
        A[i * kRRMax + q] = s * ap + c * aq;
        const double vp = V[i * kRRMax + p], vq = V[i * kRRMax + q];
        V[i * kRRMax + p] = c * vp - s * vq;
        V[i * kRRMax + q] = s * vp + c * vq;
      }
      __syncthreads();
      // rows: A[p, :], A[q, :]
      for (int e = threadIdx.x; e < half * n; e += blockDim.x) {
        const int k = e / n, j = e - (e / n) * n;
        const int p = rp[k], q = rq[k];
        if (p == q) continue;
        const double c = rc[k], s = rs[k];
        const double ap = A[p * kRRMax + j], aq = A[q * kRRMax + j];
        A[p * kRRMax + j] = c * ap - s * aq;
        A[q * kRRMax + j] = s * ap + c * aq;
      }
      __syncthreads();
    }
  }
}

// Rayleigh-Ritz of the pencil (A, B), n x n (ld = n): scaling to unit diagonal of B, canonical
// orthogonalisation of B (directions below cut x max dropped), Jacobi on the projected A;
// theta[0..kv) the kv smallest Ritz values, C (n x kv, ld kv) their coefficients (B-orthonormal
// Ritz vectors Z C).  info[0] = number of kept directions.
__global__ void __launch_bounds__(256) k_rayleigh_ritz(const double *__restrict__ Ag, const double *__restrict__ Bg,
                                                       int n, int kv, double cut, double *theta, double *C,
                                                       int *info) {
  extern __shared__ double sm[];
  double *A = sm;                   // [kRRMax][kRRMax]
  double *V = A + kRRMax * kRRMax;  // [kRRMax][kRRMax]
  double *X = V + kRRMax * kRRMax;  // [kRRMax][kRRMax]
  __shared__ double dsc[kRRMax], sg[kRRMax], rc[kRRMax / 2], rs[kRRMax / 2];
  __shared__ int rp[kRRMax / 2], rq[kRRMax / 2], kept[kRRMax], nk_sh;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double b = Bg[i * n + i];
    dsc[i] = b > 0.0 ? 1.0 / sqrt(b) : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    A[i * kRRMax + j] = Bg[e] * dsc[i] * dsc[j];
    V[i * kRRMax + j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  jacobi_sym(A, V, n, rc, rs, rp, rq);
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int i = 0; i < n; ++i) mx = fmax(mx, A[i * kRRMax + i]);
    int nk = 0;
    for (int i = 0; i < n; ++i)
      if (A[i * kRRMax + i] > cut * mx) {
        sg[nk] = 1.0 / sqrt(A[i * kRRMax + i]);
        kept[nk++] = i;
      }
    nk_sh = nk;
  }
  __syncthreads();
  const int nk = nk_sh;
  // X = D V_kept diag(sigma)^{-1/2}  (n x nk)
  for (int e = threadIdx.x; e < n * nk; e += blockDim.x) {
    const int i = e / nk, a = e - (e / nk) * nk;
    X[i * kRRMax + a] = dsc[i] * V[i * kRRMax + kept[a]] * sg[a];
  }
  __syncthreads();
  // W = A_g X into V (n x nk), then A = X^T W (nk x nk)
  for (int e = threadIdx.x; e < n * nk; e += blockDim.x) {
    const int i = e / nk, a = e - (e / nk) * nk;
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc = fma(Ag[i * n + k], X[k * kRRMax + a], acc);
    V[i * kRRMax + a] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nk * nk; e += blockDim.x) {
    const int a = e / nk, b = e - (e / nk) * nk;
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc = fma(X[k * kRRMax + a], V[k * kRRMax + b], acc);
    A[a * kRRMax + b] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nk * nk; e += blockDim.x) {
    const int a = e / nk, b = e - (e / nk) * nk;
    if (a < b) {
      const double v = 0.5 * (A[a * kRRMax + b] + A[b * kRRMax + a]);
      A[a * kRRMax + b] = v;
      A[b * kRRMax + a] = v;
    }
    V[a * kRRMax + b] = a == b ? 1.0 : 0.0;
  }
  __syncthreads();
  jacobi_sym(A, V, nk, rc, rs, rp, rq);
  // order the Ritz values ascending (selection by rank; ties by index)
  for (int a = threadIdx.x; a < nk; a += blockDim.x) {
    const double va = A[a * kRRMax + a];
    int rank = 0;
    for (int b = 0; b < nk; ++b) {
      const double vb = A[b * kRRMax + b];
      if (vb < va || (vb == va && b < a)) ++rank;
    }
    if (rank < kv) {
      theta[rank] = va;
      for (int i = 0; i < n; ++i) {  // C[:, rank] = X y_a
        double acc = 0.0;
        for (int k = 0; k < nk; ++k) acc = fma(X[i * kRRMax + k], V[k * kRRMax + a], acc);
        C[i * kv + rank] = acc;
      }
    }
  }
  if (threadIdx.x == 0) info[0] = nk;
}

}  // namespace

// ---- launchers ----------------------------------------------------------------------------

cudaError_t launch_box_band(const SysDev *sys, long long items, double *Hband, double *Sband, cudaStream_t st) {
  if (items <= 0) return cudaSuccess;
  kmark(LHF_K_BOX_ASSEMBLE, 1, st);
  k_box_band<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(sys, Hband, Sband);
  kmark(LHF_K_BOX_ASSEMBLE, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_band_mv(const double *Hb, const double *Sb, const double *X, double *YH, double *YS, int L,
                           int bJ, int bjlo, int m0, int kv, cudaStream_t st) {
  const int threads = ((kv * m0 + 31) / 32) * 32;
  kmark(LHF_K_BOX_SOLVE, 1, st);
  k_band_mv<<<L, threads > 512 ? 512 : threads, 0, st>>>(Hb, Sb, X, YH, YS, L, bJ, bjlo, m0, kv,
                                                          (int64_t)L * m0);
  kmark(LHF_K_BOX_SOLVE, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_band_average(const double *Hb, const double *Sb, int L, int bJ, int bjlo, int m0, double *Ha,
                                double *Sa, cudaStream_t st) {
  const int items = bJ * m0 * m0;
  kmark(LHF_K_BOX_SOLVE, 1, st);
  k_band_average<<<(items + 127) / 128, 128, 0, st>>>(Hb, Sb, L, bJ, bjlo, m0, Ha, Sa);
  kmark(LHF_K_BOX_SOLVE, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_prec_blocks(const double *Hb, const double *Sb, int mid, int bJ, int bjlo, int m0, int M,
                               double2 *Hk, double2 *Sk, cudaStream_t st) {
  const long long items = (long long)M * m0 * m0;
  kmark(LHF_K_BOX_SOLVE, 1, st);
  k_prec_blocks<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(Hb, Sb, mid, bJ, bjlo, m0, M, Hk, Sk);
  kmark(LHF_K_BOX_SOLVE, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_prec_factor(const double2 *Hk, const double2 *Sk, double sigma, int m0, int M, double2 *Lk,
                               unsigned *bad, cudaStream_t st) {
  kmark(LHF_K_BOX_SOLVE, 1, st);
  k_prec_factor<<<(M + 127) / 128, 128, 0, st>>>(Hk, Sk, sigma, m0, M, Lk, bad);
  kmark(LHF_K_BOX_SOLVE, 0, st);
  return cudaGetLastError();
}

// Y = T X: zero padding to M cells, DFT, Pbar_kappa^{-1}, inverse DFT, restriction (Vk: kv M m0
// complex scratch).
cudaError_t launch_prec_apply(const double2 *Lk, const double *X, double *Y, double2 *Vk, int L, int m0, int M,
                              int kv, cudaStream_t st) {
  int bits = 0;
  while ((1 << bits) < M) ++bits;
  const size_t smem = (size_t)M * sizeof(double2);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_vec_fft_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_vec_fft_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  const int64_t N = (int64_t)L * m0;
  kmark(LHF_K_BOX_SOLVE, 1, st);
  k_vec_fft_fwd<<<kv * m0, 256, smem, st>>>(X, Vk, L, m0, M, bits, N);
  const long long items = (long long)kv * M;
  k_prec_solve<<<(unsigned)((items + 127) / 128), 128, 0, st>>>(Lk, Vk, m0, M, kv);
  k_vec_fft_inv<<<kv * m0, 256, smem, st>>>(Vk, Y, L, m0, M, bits, N);
  kmark(LHF_K_BOX_SOLVE, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_tri_factor(const double *Hb, const double *Sb, double sigma, int L, int bJ, int bjlo, int m0,
                              int g, int nb, double *D, double *E, unsigned *bad, cudaStream_t st) {
  const int B = g * m0;
  const long long items = 2ll * nb * B * B;
  kmark(LHF_K_BOX_SOLVE, 1, st);
  k_tri_blocks<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(Hb, Sb, sigma, L, bJ, bjlo, m0, g, nb, D, E);
  k_tri_factor<<<1, 1024, 0, st>>>(D, E, B, nb, bad);
  kmark(LHF_K_BOX_SOLVE, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_tri_solve(const double *D, const double *E, int B, int nb, long long N, int kv, double *Y,
                             double *V, cudaStream_t st) {
  kmark(LHF_K_BOX_SOLVE, 1, st);
  k_tri_solve<<<kv, 256, 0, st>>>(D, E, B, nb, N, Y, V);
  kmark(LHF_K_BOX_SOLVE, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_gram_vec(const double *Z, const double *Y, int nz, long long N, double *G, cudaStream_t st) {
  kmark(LHF_K_BOX_SOLVE, 1, st);
  k_gram_vec<<<dim3(nz, nz), 256, 0, st>>>(Z, Y, nz, N, G, nz);
  kmark(LHF_K_BOX_SOLVE, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_lincomb(const double *Z, const double *C, int ldc, int j0, int j1, int kv, long long N,
                           double *out, cudaStream_t st) {
  const long long items = (long long)kv * N;
  kmark(LHF_K_BOX_SOLVE, 1, st);
  k_lincomb<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(Z, C, ldc, j0, j1, kv, N, out);
  kmark(LHF_K_BOX_SOLVE, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_residual(const double *YH, const double *YS, const double *theta, int kv, long long N,
                            double *R, double *rnorm, cudaStream_t st) {
  kmark(LHF_K_BOX_SOLVE, 1, st);
  k_residual<<<kv, 256, 0, st>>>(YH, YS, theta, N, R, rnorm);
  kmark(LHF_K_BOX_SOLVE, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_start_vectors(double *X, int kv, long long N, unsigned long long seed, cudaStream_t st) {
  const long long items = (long long)kv * N;
  k_start_vectors<<<(unsigned)((items + 255) / 256), 256, 0, st>>>(X, kv, N, seed);
  return cudaGetLastError();
}

int rayleigh_ritz_max() { return kRRMax; }

cudaError_t launch_rayleigh_ritz(const double *A, const double *B, int n, int kv, double cut, double *theta,
                                 double *C, int *info, cudaStream_t st) {
  if (n > kRRMax || kv > n) return cudaErrorInvalidValue;
  const size_t smem = (size_t)3 * kRRMax * kRRMax * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_rayleigh_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kmark(LHF_K_BOX_SOLVE, 1, st);
  k_rayleigh_ritz<<<1, 256, smem, st>>>(A, B, n, kv, cut, theta, C, info);
  kmark(LHF_K_BOX_SOLVE, 0, st);
  return cudaGetLastError();
}

}  // namespace lhf
