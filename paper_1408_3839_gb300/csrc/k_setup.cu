// k_setup.cu -- steps a1 and a2: 1D basis samples and 1D potential factors, FP64.
//
// a1 (Sec. 3.4, eq. (3.14)): g_mu^(l)(x_i) for the cell-0 copy of every basis function at every
//    grid node of direction l, periodised over the supercell L b in periodic directions.
// a2 (Sec. 3.2 eqs. (3.5), (3.6), (3.9); Sec. 4.1 eq. (4.1)): for rank term r = (nu, q),
//    v_r^(l)(i) = sum_k w_k int_{cell i} exp(-t_q^2 (x - a_nu,l - k b)^2) dx over the lattice
//    images k of nucleus nu (periodic: window centred on cell 0, evaluated for the cell-0 nodes;
//    open box: the L actual cells weighted by their charges; single open cell: k = 0).
//
// Layout: systems on blockIdx.y; a1 one CTA per chunk of 512 samples of a row (a thread per run of
// 8 consecutive samples), a2 the row constants once per (direction, sinc node) and then one CTA
// per chunk of 512 cells of a row (see k_basis, k_pot_rows, k_potential).
#include <math.h>

#include "lhf_internal.cuh"
#include "lhf_pairs.cuh"

namespace lhf {
namespace {

__device__ __forceinline__ double gto_factor(double d, double alpha, double cut, bool pdir,
                                             double pnorm) {
  if (fabs(d) > cut) return 0.0;
  double g = exp(-alpha * d * d);
  if (pdir) g *= pnorm * d;
  return g;
}

// Sample e (node i = e - gext) of the cell-0 copy of mu in direction l; exact zero outside the
// widened cut range without floating-point work.
__device__ double basis_sample(const SysDev &s, int l, int mu, int e) {
  const DirDev &D = s.d[l];
  int rel = e - s.node_lo[l][mu];
  const int wrapped = (D.periodic && rel < 0) ? 1 : 0;
  if (wrapped) rel += D.n;
  if (rel < 0 || rel >= s.node_span[l][mu]) return 0.0;
  const double x = D.x0 + (e - D.gext + 0.5) * D.h;
  const double A = s.centre[mu][l];
  const double cut = s.cut[mu];
  const double al = s.alpha[mu];
  const bool pdir = (s.kind[mu] == 1 + l);
  const double pn = s.pnorm[mu];
  if (!D.periodic) return gto_factor(x - A, al, cut, pdir, pn);
  const double P = D.L * D.b;
  const double d0 = x - A;
  if (s.node_span[l][mu] < D.n) {
    // the window is shorter than the period: the one image within the cut is the one that puts
    // node e at its unwrapped index (node_lo + node_wrap n) + rel, image m = -(node_wrap + wrapped)
    // (the others contribute exact zeros to the sum below)
    const int m = -(s.node_wrap[l][mu] + wrapped);
    return gto_factor(d0 - m * P, al, cut, pdir, pn);
  }
  // images m with |d0 - m P| <= cut (the bracket is widened by one on each side; the cut test
  // inside gto_factor decides)
  const int mlo = (int)floor((d0 - cut) * D.invP) - 1;
  const int mhi = (int)ceil((d0 + cut) * D.invP) + 1;
  double g = 0.0;
  for (int m = mlo; m <= mhi; ++m) g += gto_factor(d0 - m * P, al, cut, pdir, pn);
  return g;
}

// Samples and their forward differences D_e = g_e - g_(e+1) (periodic directions wrap; open
// ones take g_n = 0; not formed for the extended samples of an open box), and on the mixed route
// both also as FP32 pairs: one CTA per (system,
// direction, function mu, chunk of kBasisChunk samples of the row), so that the long rows of a
// periodic lattice direction are spread over several CTAs.  In a periodic lattice direction
// only the nodes of the support cells cell_lo .. cell_hi of the cell-0 copy (mod L, at most L
// cells) are written -- the Gram kernels read nothing else, and every node outside them lies
// beyond the cut (zero sample); other directions write the whole row (basis_row_samples).
//
// A thread takes a run of kBasisRun consecutive samples.  Along a run the distance to the
// centre advances by h, d_j = d_0 + j h (continuous across the periodic wrap of the node index:
// the image changes with it), so that
//   exp(-alpha d_j^2) = exp(-alpha d_0^2) E^j T_j,  E = exp(-2 alpha d_0 h),  T_j = exp(-alpha h^2 j^2)
// with T from a per-CTA table: two exponentials per run instead of one per sample, within a few
// ulps of the direct value (the rounding of the direct argument alpha d^2 near the cut is of the
// same size).  Runs whose ends lie where exp(-alpha d^2) could underflow (alpha d^2 > 600, far
// beyond the cut), and rows whose support window covers the whole period (several images per
// node), take the direct per-sample evaluation.  The neighbour of a run's last sample is the
// next lane's first sample, or is evaluated where the next lane holds none.
constexpr int kBasisRun = 8;
constexpr int kBasisThreads = kBasisChunk / kBasisRun;  // one run per thread and chunk
static_assert(kBasisThreads % 32 == 0, "chunks end on warp boundaries");

__global__ void __launch_bounds__(kBasisThreads) k_basis(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  const int m0 = s.m0;
  int b = blockIdx.x, l = 0, mu = 0, count = 0;
  for (int r = 0; r < 3 * m0; ++r) {
    const int cnt = basis_row_samples(s, r / m0, r % m0);
    const int nch = (cnt + kBasisChunk - 1) / kBasisChunk;
    if (b < nch) {
      l = r / m0;
      mu = r % m0;
      count = cnt;
      break;
    }
    b -= nch;
  }
  if (count == 0) return;  // surplus CTA of a smaller system
  const DirDev &D = s.d[l];
  const int nx = D.n + D.gext;
  int start = 0;
  if (D.periodic) {
    start = (s.cell_lo[l][mu] % D.L) * D.nc;
    if (start < 0) start += D.n;
  }
  const double al = s.alpha[mu], h = D.h, cut = s.cut[mu], pn = s.pnorm[mu];
  const bool pdir = (s.kind[mu] == 1 + l);
  __shared__ double T[kBasisRun];
  if (threadIdx.x < kBasisRun) {
    const double u = h * (double)threadIdx.x;
    T[threadIdx.x] = exp(-al * (u * u));
  }
  __syncthreads();
  // several images per node: direct evaluation (row-uniform)
  const bool direct_row = D.periodic && s.node_span[l][mu] >= D.n;
  const int lane = threadIdx.x & 31;
  const int kend = min(count, (b + 1) * kBasisChunk);
  const int k0 = b * kBasisChunk + (int)threadIdx.x * kBasisRun;
  const bool has = k0 < kend;
  int e0 = start + k0;
  if (e0 >= nx) e0 -= nx;  // periodic wrap (start < n = nx there)
  double g[kBasisRun];
  if (has) {
    // offset of the run's first sample in the support window and its distance to the centre of
    // the image that holds it (as basis_sample); the recurrence needs the window offset not to
    // wrap inside the run (the image changes there)
    int rel = e0 - s.node_lo[l][mu];
    const int wrapped = (D.periodic && rel < 0) ? 1 : 0;
    if (wrapped) rel += D.n;
    double d0 = D.x0 + (e0 - D.gext + 0.5) * h - s.centre[mu][l];
    if (D.periodic) d0 += (double)(s.node_wrap[l][mu] + wrapped) * (D.L * D.b);
    const double dl = d0 + (kBasisRun - 1) * h;
    const bool direct = direct_row || (D.periodic && rel + kBasisRun - 1 >= D.n) || al * (d0 * d0) > 600.0 ||
                        al * (dl * dl) > 600.0;
    if (direct) {
#pragma unroll
      for (int j = 0; j < kBasisRun; ++j) {
        int e = e0 + j;
        if (e >= nx) e -= nx;
        g[j] = k0 + j < kend ? basis_sample(s, l, mu, e) : 0.0;
      }
    } else {
      const double g0 = exp(-al * (d0 * d0)), E = exp(-2.0 * al * d0 * h);
      double P = 1.0;
#pragma unroll
      for (int j = 0; j < kBasisRun; ++j) {
        // the widened window (exact zeros outside it) and the cut, as basis_sample
        const int rj = rel + j;
        const double dj = d0 + j * h;
        double v = g0 * P * T[j];
        if (pdir) v *= pn * dj;
        g[j] = (k0 + j < kend && rj >= 0 && rj < s.node_span[l][mu] && fabs(dj) <= cut) ? v : 0.0;
        P *= E;
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < kBasisRun; ++j) g[j] = 0.0;
  }
  // the whole warp takes part in the shuffle: the next run's first sample
  double gn = __shfl_down_sync(0xffffffffu, g[0], 1);
  if (!has) return;
#pragma unroll
  for (int j = 0; j < kBasisRun; ++j) {
    if (k0 + j >= kend) break;
    int e = e0 + j;
    if (e >= nx) e -= nx;
    s.ws[D.offG + (int64_t)mu * nx + e] = g[j];
    if (D.offD < 0) continue;
    double nxt;
    if (e + 1 == D.n)
      nxt = D.periodic ? basis_sample(s, l, mu, 0) : 0.0;
    else if (j + 1 < kBasisRun)
      nxt = k0 + j + 1 < kend ? g[j + 1] : basis_sample(s, l, mu, e + 1);
    else
      nxt = (lane == 31 || k0 + kBasisRun >= kend) ? basis_sample(s, l, mu, e + 1) : gn;
    const double dif = g[j] - nxt;
    s.ws[D.offD + (int64_t)mu * D.n + e] = dif;
    if (D.offGD >= 0) {
      const float2 gp = fp32_pair(g[j]), dp = fp32_pair(dif);
      reinterpret_cast<float4 *>(s.ws + D.offGD)[(int64_t)mu * D.n + e] = make_float4(gp.x, gp.y, dp.x, dp.y);
    }
  }
}

// int_{-d}^{d} exp(-(m + u)^2) du = exp(-m^2) sum_k H_2k(m) 2 d^(2k+1) / (2k+1)!  (Taylor series
// of the Gaussian about the cell centre; H_n are the physicists' Hermite polynomials, whose
// recurrence H_{n+1} = 2 m H_n - 2 n H_{n-1} gives the derivatives).  Used for narrow cells
// where the erf difference would cancel.
__constant__ double kRecip[64] = {
    1.0 / 1,  1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,  1.0 / 7,  1.0 / 8,  1.0 / 9,  1.0 / 10, 1.0 / 11,
    1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17, 1.0 / 18, 1.0 / 19, 1.0 / 20, 1.0 / 21, 1.0 / 22,
    1.0 / 23, 1.0 / 24, 1.0 / 25, 1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29, 1.0 / 30, 1.0 / 31, 1.0 / 32, 1.0 / 33,
    1.0 / 34, 1.0 / 35, 1.0 / 36, 1.0 / 37, 1.0 / 38, 1.0 / 39, 1.0 / 40, 1.0 / 41, 1.0 / 42, 1.0 / 43, 1.0 / 44,
    1.0 / 45, 1.0 / 46, 1.0 / 47, 1.0 / 48, 1.0 / 49, 1.0 / 50, 1.0 / 51, 1.0 / 52, 1.0 / 53, 1.0 / 54, 1.0 / 55,
    1.0 / 56, 1.0 / 57, 1.0 / 58, 1.0 / 59, 1.0 / 60, 1.0 / 61, 1.0 / 62, 1.0 / 63, 1.0 / 64};

__device__ double gauss_cell_series(double m, double d) {
  double hm1 = 1.0, h0 = 2.0 * m;   // H_0, H_1
  double p = d;                     // d^(n+1) / (n+1)!  for n = 0
  double sum = 2.0 * p;             // k = 0 term: H_0 * 2 d
  int small = 0;                    // consecutive negligible terms (a Hermite root may zero one)
  for (int n = 1; n < 60; ++n) {
    p = p * d * kRecip[n];  // d^(n+1) / (n+1)!
    if (!(n & 1)) {
      double term = 2.0 * h0 * p;
      sum += term;
      small = (fabs(term) <= 1e-18 * fabs(sum)) ? small + 1 : 0;
      if (small == 2) break;
    }
    double hn = 2.0 * m * h0 - 2.0 * n * hm1;  // H_{n+1}
    hm1 = h0;
    h0 = hn;
  }
  return exp(-m * m) * sum;
}

// Exact integral of exp(-t^2 (x - c)^2) over [lo, hi]  (eq. (3.5) with one term of eq. (3.6)).
// invt = 1 / t (divisions are FP64 instruction sequences on this GPU: the row's reciprocals are
// formed once).
__device__ double gauss_cell_integral(double t, double invt, double lo, double hi, double c) {
  const double A = t * (lo - c), B = t * (hi - c);
  const double f = 0.88622692545275801365 * invt;  // sqrt(pi) / (2 t)
  if (A < 0.0 && B > 0.0) return f * (erf(B) + erf(-A));
  const double delta = B - A;
  const double m = 0.5 * (A + B);
  if (delta <= 0.25 && fabs(m) * delta <= 1.0) return gauss_cell_series(m, 0.5 * delta) * invt;
  if (A >= 0.0) return f * (erfc(A) - erfc(B));
  return f * (erfc(-B) - erfc(-A));
}

// Cell integrals by Taylor series about the cell centre.  For a cell of width h centred at
// distance xc from a Gaussian exp(-t^2 x^2), m = t xc, delta = t h and d = delta / 2:
//   int_cell exp(-t^2 x^2) dx = exp(-m^2) S(m^2) / t,
//   S = sum_j a_j H_2j(m) = sum_j b_j y^j,  y = m^2,  a_j = 2 d^(2j+1) / (2j+1)!
// (the odd terms integrate to zero; H_n are the physicists' Hermite polynomials), and with
// H_2j(m) = sum_i (2j)! (-1)^(j-i) 4^i / ((j-i)! (2i)!) y^i
//   b_i = 4^i / (2i)! sum_{l >= 0} (-1)^l 2 d^(2(i+l)+1) / ((2(i+l)+1) l!).
// The series is cut after degree J, the first j with (22 d)^(2j+2) / (2j+3)! < 1e-18 (|m| <= 11
// within the reach of a Gaussian).  The b_i depend on t and h only: one set per potential row.
constexpr double kTaylorMaxDelta = 0.25;
constexpr int kTaylorMaxJ = 16;

__device__ int taylor_degree(double d) {
  const double x22 = (22.0 * d) * (22.0 * d);
  int J = 1;
  double bound = x22 * x22 * kRecip[0] * kRecip[1] * kRecip[2] * kRecip[3] * kRecip[4];  // j = 1
  while (bound >= 1e-18 && J < kTaylorMaxJ) {
    ++J;
    bound *= x22 * kRecip[2 * J + 1] * kRecip[2 * J + 2];
  }
  return J;
}

__device__ double taylor_coef(int i, int J, double d) {
  const double d2 = d * d;
  double dp = 2.0 * d;  // 2 d^(2(i+l)+1), l = 0
  for (int u = 0; u < i; ++u) dp *= d2;
  double sum = 0.0, lf = 1.0;  // lf = 1 / l!
  for (int l = 0; i + l <= J; ++l) {
    const double term = dp * kRecip[2 * (i + l)] * lf;  // / (2(i+l)+1)
    sum += (l & 1) ? -term : term;
    dp *= d2;
    lf *= kRecip[l];  // 1 / (l+1)!
  }
  double f = sum;  // * 4^i / (2i)!
  for (int u = 1; u <= 2 * i; ++u) f *= kRecip[u - 1];
  for (int u = 0; u < i; ++u) f *= 4.0;
  return f;
}

__device__ __forceinline__ double taylor_S(const double *bc, int J, double y) {
  double S = bc[J];
  for (int j = J - 1; j >= 0; --j) S = fma(S, y, bc[j]);
  return S;
}

// Wide Gaussians (s = t b <= 0.1) over many images: the image sum is a trapezoidal rule of
// phi(k) = psi(m0 - k s), psi(m) = exp(-m^2) S(m^2), and the Euler-Maclaurin formula gives it in
// closed form:
//   sum_{k=a..c} w_k phi(k) = (1/s) int_{m_c}^{m_a} psi + sum_{j=1..7} B_2j/(2j)! s^(2j-1)
//                              (psi^(2j-1)(m_a) - psi^(2j-1)(m_c)) + (w_a - 1/2) phi(a) + (w_c - 1/2) phi(c)
// with m_a = m0 - a s, m_c = m0 - c s.  The integral is sum_j b_j (G_2j(m_a) - G_2j(m_c)),
// G_0 = (sqrt(pi)/2) erf, G_2j = (2j-1)/2 G_2j-2 - m^(2j-1) exp(-m^2) / 2.  The derivatives are
// psi^(n) = exp(-m^2) P_n(m) with P_0(m) = S(m^2) and P_(n+1) = P_n' - 2 m P_n, so the whole
// correction is exp(-m^2) C(m) at each end, C = sum_j B_2j/(2j)! s^(2j-1) P_(2j-1): a polynomial
// of degree <= 2 kEmJ + 2 kEmP - 1 whose coefficients depend on the row (t, h, b) only.  The
// remainder after 7 terms is below 1e-17 of the sum for s <= 0.1 (the terms fall like
// (s / 2 pi)^(2j) sqrt((2j)!)), and S has degree <= 2 kEmJ.
constexpr int kEmJ = 3;
constexpr int kEmP = 7;
constexpr int kEmDeg = 2 * kEmJ + 2 * kEmP - 1;
constexpr double kEmMaxS = 0.1;
__constant__ double kEmB[kEmP] = {1.0 / 12.0,         -1.0 / 720.0,     1.0 / 30240.0,
                                  -1.0 / 1209600.0,   1.0 / 47900160.0, -691.0 / 1307674368000.0,
                                  1.0 / 74724249600.0};

// Coefficients of C (C[k] of m^k, k <= kEmDeg) by one warp, lane k holding the coefficient of
// m^k: P_0 = S(m^2) from the series coefficients, P_(n+1) = P_n' - 2 m P_n (coefficients
// (k + 1) P_n[k + 1] - 2 P_n[k - 1], neighbours by shuffles), C accumulating
// B_2j / (2j)! s^(2j-1) P_(2j-1).
__device__ void em_poly_warp(const double *bc, int J, double s, double *C) {
  const int k = threadIdx.x & 31;
  double P = ((k & 1) == 0 && k / 2 <= J) ? bc[k / 2] : 0.0;
  double acc = 0.0, sp = s;  // s^(2j-1)
  for (int n = 0; n < 2 * kEmP - 1; ++n) {
    const double up = __shfl_down_sync(0xffffffffu, P, 1);  // coefficient of m^(k+1)
    const double dn = __shfl_up_sync(0xffffffffu, P, 1);    // coefficient of m^(k-1)
    P = (double)(k + 1) * (k < 31 ? up : 0.0) - 2.0 * (k > 0 ? dn : 0.0);
    if (((n + 1) & 1) != 0) {
      acc = fma(kEmB[n / 2] * sp, P, acc);  // j = (n + 2) / 2
      sp *= s * s;
    }
  }
  if (k <= kEmDeg) C[k] = acc;
}

// (sqrt(pi)/2) (erf(x) - erf(y)) for x >= y, without cancellation when both are far out on one
// side.
__device__ double half_sqrtpi_erf_diff(double x, double y) {
  const double f = 0.88622692545275801365;
  if (y >= 0.0) return f * (erfc(y) - erfc(x));
  if (x <= 0.0) return f * (erfc(-x) - erfc(-y));
  return f * (erf(x) - erf(y));
}

__device__ double image_sum_em(double t, double xc, double b, double invs, const double *bc, int J, const double *C,
                               int klo, int khi, int kmax, bool even) {
  const double s = t * b, m0 = t * xc;
  const double ma = m0 - klo * s, mc = m0 - khi * s;
  const double ea = exp(-ma * ma), ec = exp(-mc * mc);
  // integral of psi over [m_c, m_a]
  double ga = 0.0, gc = 0.0;  // G_2j(m_a) - G_2j(m_c) built by the recurrence from G_0
  double g_diff = half_sqrtpi_erf_diff(ma, mc);
  double integ = bc[0] * g_diff;
  double pa = ma, pc = mc;  // m^(2j-1)
  for (int j = 1; j <= J; ++j) {
    ga = pa * ea;
    gc = pc * ec;
    g_diff = 0.5 * (2 * j - 1) * g_diff - 0.5 * (ga - gc);
    integ = fma(bc[j], g_diff, integ);
    pa *= ma * ma;
    pc *= mc * mc;
  }
  integ *= invs;
  double ca = C[kEmDeg], cc = C[kEmDeg];
#pragma unroll
  for (int k = kEmDeg - 1; k >= 0; --k) {
    ca = fma(ca, ma, C[k]);
    cc = fma(cc, mc, C[k]);
  }
  const double wa = (even && (klo == kmax || klo == -kmax)) ? 0.5 : 1.0;
  const double wc = (even && (khi == kmax || khi == -kmax)) ? 0.5 : 1.0;
  return integ + (ea * ca - ec * cc) + (wa - 0.5) * ea * taylor_S(bc, J, ma * ma) +
         (wc - 0.5) * ec * taylor_S(bc, J, mc * mc);
}

// Sum over the images k = klo .. khi (weight 1/2 on k = +-kmax when the window is even) of
// t int_{cell} exp(-t^2 (x - c0 - k b)^2) dx for a narrow cell (delta <= kTaylorMaxDelta) centred
// at c0 + xc: sum_k w_k exp(-m_k^2) S(m_k^2), m_k = t (xc - k b).  exp(-m_k^2) follows the images
// by exp(-m_{k+-1}^2) = exp(-m_k^2) R, R = exp(-+2 m_k s - s^2), s = t b, R <- R exp(-2 s^2),
// walking outward from the image nearest to the cell and restarted from exp every 8 images, so
// that the dominant terms come from small exponents and the product's rounding stays within a
// few tens of ulp.
__device__ double image_sum_taylor(double t, double xc, double b, double invb, const double *bc, int J, int klo,
                                   int khi, int kmax, bool even) {
  if (klo > khi) return 0.0;  // no image within reach
  const double sb = t * b;
  const double Q = exp(-2.0 * sb * sb);
  // the image nearest to the cell, clamped to the window
  int kc = (int)rint(xc * invb);
  kc = kc < klo ? klo : (kc > khi ? khi : kc);
  double v = 0.0;
  // outward: dir = +1 (k = kc .. khi, m decreasing), dir = -1 (k = kc-1 .. klo, m increasing)
  for (int dir = 1; dir >= -1; dir -= 2) {
    const int kbeg = dir > 0 ? kc : kc - 1;
    const int kend = dir > 0 ? khi + 1 : klo - 1;
    for (int k0 = kbeg; k0 != kend;) {
      double m = t * (xc - k0 * b);
      double e = exp(-m * m);
      double R = exp(dir * 2.0 * m * sb - sb * sb);
      const int steps = dir > 0 ? min(8, kend - k0) : min(8, k0 - kend);
      for (int u = 0; u < steps; ++u) {
        const int k = k0 + dir * u;
        const double S = taylor_S(bc, J, m * m);
        const double w = (even && (k == kmax || k == -kmax)) ? 0.5 * e : e;
        v = fma(w, S, v);
        e *= R;
        R *= Q;
        m -= dir * sb;
      }
      k0 += dir * steps;
    }
  }
  return v;
}

// The same recurrence over the actual nuclei of an open box, k = klo .. khi, each image weighted
// by its cell's charge over the row's reference charge (zc[k M0] / Z; weight 1 without zc).
__device__ __noinline__ double image_sum_taylor_box(double t, double xc, double b, double invb, const double *bc, int J, int klo,
                                       int khi, const double *zc, int M0, double invZ) {
  if (klo > khi) return 0.0;  // no nucleus within reach
  const double sb = t * b;
  const double Q = exp(-2.0 * sb * sb);
  int kc = (int)rint(xc * invb);
  kc = kc < klo ? klo : (kc > khi ? khi : kc);
  double v = 0.0;
  for (int dir = 1; dir >= -1; dir -= 2) {
    const int kbeg = dir > 0 ? kc : kc - 1;
    const int kend = dir > 0 ? khi + 1 : klo - 1;
    for (int k0 = kbeg; k0 != kend;) {
      double m = t * (xc - k0 * b);
      double e = exp(-m * m);
      double R = exp(dir * 2.0 * m * sb - sb * sb);
      const int steps = dir > 0 ? min(8, kend - k0) : min(8, k0 - kend);
      for (int u = 0; u < steps; ++u) {
        const int k = k0 + dir * u;
        const double S = taylor_S(bc, J, m * m);
        const double w = zc ? e * (zc[(int64_t)k * M0] * invZ) : e;
        v = fma(w, S, v);
        e *= R;
        R *= Q;
        m -= dir * sb;
      }
      k0 += dir * steps;
    }
  }
  return v;
}

// Image sums whose window holds every image within reach (the images beyond the window lie
// beyond exp(-100) of the nearest one): the lattice sum of the Gaussian is periodic in x and its
// Fourier series (Poisson summation) integrates over the cell in closed form,
//   sum_k int_cell exp(-t^2 (x - c0 - k b)^2) dx
//     = sqrt(pi) / (t b) [h + sum_{n>=1} exp(-pi^2 n^2 / s^2) (2 b / (pi n)) cos(2 pi n (x_m - c0) / b)
//                             sin(pi n h / b)],   s = t b, x_m the cell midpoint,
// cut after the first n with exp(-pi^2 n^2 / s^2) below 1e-20 (n > 2.16 s): a few terms where
// the direct sum would take ~20 / s images.  The weights of the cosines depend on the row only;
// cos(n theta) follows from cos(theta) by the Chebyshev recurrence (terms n >= 2 carry weights
// below exp(-4 pi^2 / s^2) < 3e-8, far below the recurrence's rounding growth).
constexpr double kPoissonMaxS = 1.5;
constexpr int kPoissonMaxN = 5;  // ceil(2.16 s) + 1 for s < 1.5
constexpr double kPi = 3.14159265358979323846;

__device__ double poisson_weight(int n, double s, double h, double b) {
  const double g = exp(-(kPi * n / s) * (kPi * n / s));
  if (g == 0.0) return 0.0;
  return g * (2.0 * b / (kPi * n)) * sinpi(n * h / b);
}

__device__ double image_sum_poisson(double pref, double h, double xc, double invb, const double *pw, int N) {
  const double c1 = cospi(2.0 * xc * invb);  // xc: cell midpoint minus c0
  double acc = h, cm = 1.0, cn = c1;  // cos((n-1) theta), cos(n theta)
  for (int n = 1; n <= N; ++n) {
    acc = fma(pw[n], cn, acc);
    const double nx = 2.0 * c1 * cn - cm;
    cm = cn;
    cn = nx;
  }
  return pref * acc;  // pref = sqrt(pi) / (t b)
}

// Row constants per (system, direction l, sinc node q), a warp each (they depend on t_q, h_l and
// b_l only, not on the nucleus): PC[0] = J, PC[1 + i] = b_i (i <= J), PC[18 + k] = the
// Euler-Maclaurin coefficients (k <= kEmDeg), PC[38 + n] = the Poisson weights (n <= NP), then
// the row's scalars (t, 1/t, the reach 10/t, delta = t h, s = t b, 1/b, 1/h, 1/(t b), the
// Poisson prefactor sqrt(pi)/(t b)) and its branch flags as an integer bit pattern: formed once
// here instead of by every thread of every row of k_potential (an FP64 division is a sequence of
// FP64 instructions, and this GPU charges each per warp).
constexpr int kPcBc = 1, kPcEm = kPcBc + kTaylorMaxJ + 1, kPcPw = kPcEm + kEmDeg + 1;
constexpr int kPcT = kPcPw + kPoissonMaxN + 1, kPcInvT = kPcT + 1, kPcReach = kPcT + 2, kPcDelta = kPcT + 3,
              kPcSb = kPcT + 4, kPcInvB = kPcT + 5, kPcInvH = kPcT + 6, kPcInvS = kPcT + 7, kPcPref = kPcT + 8,
              kPcFlags = kPcT + 9;
static_assert(kPcFlags < kPotConst, "row constants");
// flags: bit 0 Taylor cells, bit 1 Euler-Maclaurin row, bit 2 Poisson row, bits 8.. NP, bits 16.. J
__device__ __forceinline__ double pot_flags(bool taylor, bool em_row, bool poisson_row, int NP, int J) {
  return __longlong_as_double((long long)taylor | ((long long)em_row << 1) | ((long long)poisson_row << 2) |
                              ((long long)NP << 8) | ((long long)J << 16));
}

__global__ void __launch_bounds__(64) k_pot_rows(const SysDev *__restrict__ sysv) {
  // a warp per row (lane i: series coefficient i, Euler-Maclaurin coefficient i, Poisson weight i)
  const SysDev &s = sysv[blockIdx.y];
  const int idx = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (idx >= 3 * s.R) return;  // warp-uniform
  const int l = idx / s.R, q = idx - l * s.R;
  const DirDev &D = s.d[l];
  double *pc = s.ws + s.offPC + (int64_t)idx * kPotConst;
  const double t = s.t[q], delta = t * D.h, sb = t * D.b;
  const bool taylor = delta <= kTaylorMaxDelta;
  const int J = taylor ? taylor_degree(0.5 * delta) : 0;
  const bool em_row = D.periodic && taylor && sb <= kEmMaxS && J <= kEmJ;
  const bool poisson_row = D.periodic && sb < kPoissonMaxS;
  const int NP = poisson_row ? min((int)ceil(2.16 * sb) + 1, kPoissonMaxN) : 0;
  __shared__ double bcs[2][kTaylorMaxJ + 1];
  double *bc = bcs[threadIdx.x >> 5];
  if (lane <= kTaylorMaxJ) bc[lane] = (taylor && lane <= J) ? taylor_coef(lane, J, 0.5 * delta) : 0.0;
  __syncwarp();
  if (lane == 0) {
    pc[0] = (double)J;
    const double invt = 1.0 / t, invb = 1.0 / D.b;
    pc[kPcT] = t;
    pc[kPcInvT] = invt;
    pc[kPcReach] = 10.0 * invt;
    pc[kPcDelta] = delta;
    pc[kPcSb] = sb;
    pc[kPcInvB] = invb;
    pc[kPcInvH] = 1.0 / D.h;
    pc[kPcInvS] = invt * invb;
    pc[kPcPref] = 1.7724538509055160273 * invt * invb;
    pc[kPcFlags] = pot_flags(taylor, em_row, poisson_row, NP, J);
  }
  if (lane <= kTaylorMaxJ) pc[kPcBc + lane] = bc[lane];
  if (em_row) {
    em_poly_warp(bc, J, sb, pc + kPcEm);
  } else if (lane <= kEmDeg) {
    pc[kPcEm + lane] = 0.0;
  }
  if (lane <= kPoissonMaxN) pc[kPcPw + lane] = (lane >= 1 && lane <= NP) ? poisson_weight(lane, sb, D.h, D.b) : 0.0;
}

// One CTA per (system, direction, rank term r = (nucleus nu, sinc node q)): the row constants
// (series coefficients, Euler-Maclaurin polynomial, Poisson weights, formed by k_pot_rows) in
// shared memory, then a thread per cell i of the row.  Cells farther than 10 / t from every image within the window
// get exactly zero (their integrals are below exp(-100) of the nearest image's).
constexpr int kPotThreads = 128;
constexpr int kPotRun = 4;  // cells per thread on the single open cell rows

__global__ void __launch_bounds__(kPotThreads) k_potential(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  const int Rt = s.Rt;
  // CTA -> (direction l, rank term r, chunk of cells)
  int bidx = blockIdx.x, l = 0;
  for (; l < 3; ++l) {
    const int cnt = Rt * ((s.d[l].nv + kPotChunk - 1) / kPotChunk);
    if (bidx < cnt) break;
    bidx -= cnt;
  }
  if (l == 3) return;
  const DirDev &D = s.d[l];
  const int nch = (D.nv + kPotChunk - 1) / kPotChunk;
  const int r = bidx / nch, chunk = bidx - r * nch;
  const int nu = r / s.R, q = r - nu * s.R;
  const double c0 = s.a[nu][l];
  const double *pc = s.ws + s.offPC + (int64_t)(l * s.R + q) * kPotConst;
  const int tid = threadIdx.x;
  const int ibeg = chunk * kPotChunk, iend = min(D.nv, ibeg + kPotChunk);
  const double base = D.periodic ? D.cell0 : D.x0;  // left edge of cell 0
  // Per-row scalars in shared memory.  Thread 0 forms the few that depend on the nucleus, in
  // FP64 once per CTA: the cell midpoints relative to c0, xc_i = xc0 + i h; the image range of
  // cell i (images k with c0 + k b within the reach of the cell) as FP32 affine functions of i,
  // k in [ceil(flo + i fst), floor(fhi + i fst)] -- an image whose distance rounds across the
  // reach lies exp(-100) below the nearest one, so its inclusion does not matter; a single open
  // cell row's cells within reach of c0, ilo .. ihi.  Threads 1 .. kPotRun form the run table of
  // the single open cell rows, U_j = exp(-(delta j)^2).
  __shared__ double rowc[kPotConst];
  __shared__ double xc0_sh, invZ_sh, U[kPotRun];
  __shared__ float flo_sh, fhi_sh, fst_sh;
  __shared__ int ilo_sh, ihi_sh;
  if (tid < kPotConst) rowc[tid] = pc[tid];
  if (tid == 0) {
    const double reach = pc[kPcReach], invb = pc[kPcInvB], invh = pc[kPcInvH];
    xc0_sh = (base - c0) + 0.5 * D.h;
    flo_sh = (float)((base - reach - c0) * invb);
    fhi_sh = (float)((base + D.h + reach - c0) * invb);
    fst_sh = (float)(D.h * invb);
    // cell i within reach: base + i h - reach <= c0 <= base + (i + 1) h + reach
    const double lo_f = ceil((c0 - reach - base) * invh - 1.0), hi_f = floor((c0 + reach - base) * invh);
    ilo_sh = lo_f < (double)ibeg ? ibeg : (lo_f > (double)iend ? iend : (int)lo_f);
    ihi_sh = hi_f >= (double)iend ? iend - 1 : (hi_f < (double)ibeg - 1.0 ? ibeg - 1 : (int)hi_f);
    invZ_sh = D.lattice ? 1.0 / s.Z[nu] : 1.0;
  } else if (tid <= kPotRun && !D.periodic && !D.lattice) {
    const double dj = pc[kPcDelta] * (tid - 1);
    U[tid - 1] = exp(-dj * dj);
  }
  __syncthreads();
  const double *bc = rowc + kPcBc, *emc = rowc + kPcEm, *pw = rowc + kPcPw;
  const double t = rowc[kPcT], invt = rowc[kPcInvT], invb = rowc[kPcInvB];
  const long long fl = __double_as_longlong(rowc[kPcFlags]);
  const bool taylor = (fl & 1) != 0, em_row = (fl & 2) != 0, poisson_row = (fl & 4) != 0;
  const int NP = (int)((fl >> 8) & 0xff), J = (int)((fl >> 16) & 0xff);
  const int ilo = ilo_sh, ihi = ihi_sh;
  const double xc0 = xc0_sh;
  const float flo = flo_sh, fhi = fhi_sh, fst = fst_sh;

  double *out = s.ws + D.offV + (int64_t)r * D.nv;
  if (!D.periodic && !D.lattice) {
    // a single open cell row: cells ilo .. ihi within reach, exact zeros elsewhere
    for (int i = ibeg + tid; i < iend; i += kPotThreads)
      if (i < ilo || i > ihi) out[i] = 0.0;
    if (!taylor) {
      for (int i = ilo + tid; i <= ihi; i += kPotThreads) {
        const double lo = D.x0 + i * D.h;
        out[i] = gauss_cell_integral(t, invt, lo, lo + D.h, c0);
      }
      return;
    }
    // narrow cells: exp(-m^2) S(m^2) / t at the cell centres, m_j = m_0 + j delta along a run of
    // kPotRun cells, exp(-m_j^2) = exp(-m_0^2) E^j U_j with E = exp(-2 m_0 delta) (|m| <= 10 +
    // kPotRun delta within reach: no underflow)
    const double delta = rowc[kPcDelta];
    for (int i0 = ilo + kPotRun * tid; i0 <= ihi; i0 += kPotRun * kPotThreads) {
      const double m0 = t * (xc0 + i0 * D.h);
      const double g0 = exp(-m0 * m0), E = exp(-2.0 * m0 * delta);
      const double gt = g0 * invt;
      double P = 1.0;
#pragma unroll
      for (int j = 0; j < kPotRun; ++j) {
        const int i = i0 + j;
        if (i > ihi) break;
        const double m = fma((double)j, delta, m0);
        out[i] = gt * P * U[j] * taylor_S(bc, J, m * m);
        P *= E;
      }
    }
    return;
  }
  for (int i = ibeg + tid; i < iend; i += kPotThreads) {
    double v = 0.0;
    const double xc = fma((double)i, D.h, xc0);  // cell midpoint - c0
    const float fi = (float)i;
    const float kf_lo = ceilf(fmaf(fi, fst, flo)), kf_hi = floorf(fmaf(fi, fst, fhi));
    if (D.periodic) {
      const int kmax = D.K / 2;
      const bool even = (D.K % 2) == 0;
      // (clamped on both sides before the conversion: an empty range stays empty)
      const int klo = kf_lo < (float)-kmax ? -kmax : (kf_lo > (float)(kmax + 1) ? kmax + 1 : (int)kf_lo);
      const int khi = kf_hi > (float)kmax ? kmax : (kf_hi < (float)(-kmax - 1) ? -kmax - 1 : (int)kf_hi);
      if (poisson_row && klo > -kmax && khi < kmax) {
        v = image_sum_poisson(rowc[kPcPref], D.h, xc, invb, pw, NP);
      } else if (em_row && khi - klo >= 16) {
        v = image_sum_em(t, xc, D.b, rowc[kPcInvS], bc, J, emc, klo, khi, kmax, even) * invt;
      } else if (taylor) {
        v = image_sum_taylor(t, xc, D.b, invb, bc, J, klo, khi, kmax, even) * invt;
      } else {
        const double lo = D.cell0 + i * D.h, hi = lo + D.h;
        for (int k = klo; k <= khi; ++k) {
          const double wk = (even && (k == kmax || k == -kmax)) ? 0.5 : 1.0;
          v += wk * gauss_cell_integral(t, invt, lo, hi, c0 + k * D.b);
        }
      }
    } else {
      // open box: the L actual cells, weighted by their charges
      const int klo = kf_lo < 0.0f ? 0 : (kf_lo > (float)D.L ? D.L : (int)kf_lo);
      const int khi = kf_hi > (float)(D.L - 1) ? D.L - 1 : (kf_hi < -1.0f ? -1 : (int)kf_hi);
      const double invZ = invZ_sh;
      if (taylor) {
        v = image_sum_taylor_box(t, xc, D.b, invb, bc, J, klo, khi, s.zcell ? s.zcell + nu : nullptr, s.M0, invZ) *
            invt;
      } else {
        const double lo = D.x0 + i * D.h, hi = lo + D.h;
        for (int k = klo; k <= khi; ++k) {
          const double wk = s.zcell ? s.zcell[k * s.M0 + nu] * invZ : 1.0;
          v += wk * gauss_cell_integral(t, invt, lo, hi, c0 + k * D.b);
        }
      }
    }
    out[i] = v;
  }
}

}  // namespace

cudaError_t launch_basis(const SysDev *sys, int nsys, int max_rows, cudaStream_t st) {
  if (max_rows <= 0 || nsys <= 0) return cudaSuccess;
  dim3 grid(max_rows, nsys);
  kmark(LHF_K_BASIS, 1, st);
  k_basis<<<grid, kBasisThreads, 0, st>>>(sys);
  kmark(LHF_K_BASIS, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_potential(const SysDev *sys, int nsys, int max_rows, cudaStream_t st) {
  if (max_rows <= 0 || nsys <= 0) return cudaSuccess;
  // the row constants (3 R rows per system, a warp each), then the rows
  kmark(LHF_K_POTENTIAL, 1, st);
  k_pot_rows<<<dim3((3 * kMaxR + 1) / 2, nsys), 64, 0, st>>>(sys);
  kmark(LHF_K_POTENTIAL, 0, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dim3 grid(max_rows, nsys);
  kmark(LHF_K_POTENTIAL, 1, st);
  k_potential<<<grid, kPotThreads, 0, st>>>(sys);
  kmark(LHF_K_POTENTIAL, 0, st);
  return cudaGetLastError();
}

}  // namespace lhf
