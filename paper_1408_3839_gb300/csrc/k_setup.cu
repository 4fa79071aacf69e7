// k_setup.cu -- steps a1 and a2: 1D basis samples and 1D potential factors, FP64.
//
// a1 (Sec. 3.4, eq. (3.14)): g_mu^(l)(x_i) for the cell-0 copy of every basis function at every
//    grid node of direction l, periodised over the supercell L b in periodic directions.
// a2 (Sec. 3.2 eqs. (3.5), (3.6), (3.9); Sec. 4.1 eq. (4.1)): for rank term r = (nu, q),
//    v_r^(l)(i) = sum_k w_k int_{cell i} exp(-t_q^2 (x - a_nu,l - k b)^2) dx over the lattice
//    images k of nucleus nu (periodic: window centred on cell 0, evaluated for the cell-0 nodes;
//    open box: the L actual cells weighted by their charges; single open cell: k = 0).
//
// Layout: thread per output element, systems on blockIdx.y, elements flattened over
// (direction, row, node) so that consecutive threads write consecutive nodes (coalesced).
#include <math.h>

#include "lhf_internal.cuh"

namespace lhf {
namespace {

__device__ __forceinline__ double gto_factor(double d, double alpha, double cut, bool pdir,
                                             double pnorm) {
  if (fabs(d) > cut) return 0.0;
  double g = exp(-alpha * d * d);
  if (pdir) g *= pnorm * d;
  return g;
}

__global__ void __launch_bounds__(256) k_basis(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int m0 = s.m0;
  int l = 0;
  for (; l < 3; ++l) {
    int64_t cnt = (int64_t)m0 * s.d[l].n;
    if (item < cnt) break;
    item -= cnt;
  }
  if (l == 3) return;
  const DirDev &D = s.d[l];
  const int mu = (int)(item / D.n);
  const int i = (int)(item - (int64_t)mu * D.n);
  const double x = D.x0 + (i + 0.5) * D.h;
  const double A = s.centre[mu][l];
  const double cut = s.cut[mu];
  const double al = s.alpha[mu];
  const bool pdir = (s.kind[mu] == 1 + l);
  const double pn = s.pnorm[mu];
  double g = 0.0;
  if (D.periodic) {
    const double P = D.L * D.b;
    const double d0 = x - A;
    // images m with |d0 - m P| <= cut (the bracket is widened by one on each side; the cut
    // test inside gto_factor decides)
    const int mlo = (int)floor((d0 - cut) * D.invP) - 1;
    const int mhi = (int)ceil((d0 + cut) * D.invP) + 1;
    for (int m = mlo; m <= mhi; ++m) g += gto_factor(d0 - m * P, al, cut, pdir, pn);
  } else {
    g = gto_factor(x - A, al, cut, pdir, pn);
  }
  s.ws[D.offG + (int64_t)mu * D.n + i] = g;
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
__device__ double gauss_cell_integral(double t, double lo, double hi, double c) {
  const double A = t * (lo - c), B = t * (hi - c);
  const double f = 0.88622692545275801365 / t;  // sqrt(pi) / (2 t)
  if (A < 0.0 && B > 0.0) return f * (erf(B) + erf(-A));
  const double delta = B - A;
  const double m = 0.5 * (A + B);
  if (delta <= 0.25 && fabs(m) * delta <= 1.0) return gauss_cell_series(m, 0.5 * delta) / t;
  if (A >= 0.0) return f * (erfc(A) - erfc(B));
  return f * (erfc(-B) - erfc(-A));
}

__global__ void __launch_bounds__(256) k_potential(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int Rt = s.Rt;
  int l = 0;
  for (; l < 3; ++l) {
    int64_t cnt = (int64_t)Rt * s.d[l].nv;
    if (item < cnt) break;
    item -= cnt;
  }
  if (l == 3) return;
  const DirDev &D = s.d[l];
  const int r = (int)(item / D.nv);
  const int i = (int)(item - (int64_t)r * D.nv);
  const int nu = r / s.R, q = r - nu * s.R;
  const double t = s.t[q];
  const double c0 = s.a[nu][l];
  double v = 0.0;
  // images farther than 10/t from the cell contribute below exp(-100) of the nearest one
  const double reach = 10.0 / t;
  if (D.periodic) {
    const double lo = D.cell0 + i * D.h, hi = lo + D.h;
    const int kmax = D.K / 2;
    const bool even = (D.K % 2) == 0;
    double klo_f = ceil((lo - reach - c0) / D.b), khi_f = floor((hi + reach - c0) / D.b);
    int klo = (klo_f < -kmax) ? -kmax : (int)klo_f;
    int khi = (khi_f > kmax) ? kmax : (int)khi_f;
    const double delta = t * D.h, sb = t * D.b;
    if (delta <= 1e-3 && sb <= 0.1) {
      // Wide Gaussian: with m_k = t (x_mid - c0 - k b), the cell integral is
      // h exp(-m_k^2) [1 + (2 m^2 - 1) delta^2 / 12 + (4 m^4 - 12 m^2 + 3) delta^4 / 480] up to
      // O(delta^6) (the Taylor series about the cell centre), and exp(-m_k^2) follows k by
      // exp(-m_{k+1}^2) = exp(-m_k^2) R_k, R_{k+1} = R_k exp(-2 s^2), s = t b, restarted from exp
      // every 8 images so that the product's rounding stays within 32 ulp.
      const double xm = 0.5 * (lo + hi);
      const double d2 = delta * delta, c2 = d2 * (1.0 / 12.0), c4 = d2 * d2 * (1.0 / 480.0);
      const double Q = exp(-2.0 * sb * sb);
      for (int k0 = klo; k0 <= khi; k0 += 8) {
        double mk = t * (xm - c0 - k0 * D.b);
        double e = exp(-mk * mk);
        double R = exp(2.0 * mk * sb - sb * sb);
        const int kend = min(k0 + 8, khi + 1);
        for (int k = k0; k < kend; ++k) {
          const double m2 = mk * mk;
          const double corr = 1.0 + (2.0 * m2 - 1.0) * c2 + ((4.0 * m2 - 12.0) * m2 + 3.0) * c4;
          const double wk = (even && (k == kmax || k == -kmax)) ? 0.5 : 1.0;
          v += wk * e * corr;
          e *= R;
          R *= Q;
          mk = t * (xm - c0 - (k + 1) * D.b);
        }
      }
      v *= D.h;
    } else {
      for (int k = klo; k <= khi; ++k) {
        const double wk = (even && (k == kmax || k == -kmax)) ? 0.5 : 1.0;
        v += wk * gauss_cell_integral(t, lo, hi, c0 + k * D.b);
      }
    }
  } else {
    const double lo = D.x0 + i * D.h, hi = lo + D.h;
    if (D.lattice) {
      double klo_f = ceil((lo - reach - c0) / D.b), khi_f = floor((hi + reach - c0) / D.b);
      int klo = (klo_f < 0.0) ? 0 : (int)klo_f;
      int khi = (khi_f > D.L - 1) ? D.L - 1 : (int)khi_f;
      for (int k = klo; k <= khi; ++k) {
        const double wk = s.zcell ? s.zcell[k * s.M0 + nu] / s.Z[nu] : 1.0;
        v += wk * gauss_cell_integral(t, lo, hi, c0 + k * D.b);
      }
    } else {
      v = gauss_cell_integral(t, lo, hi, c0);
    }
  }
  s.ws[D.offV + (int64_t)r * D.nv + i] = v;
}

}  // namespace

cudaError_t launch_basis(const SysDev *sys, int nsys, int max_items, cudaStream_t st) {
  if (max_items <= 0 || nsys <= 0) return cudaSuccess;
  dim3 grid((max_items + 255) / 256, nsys);
  k_basis<<<grid, 256, 0, st>>>(sys);
  return cudaGetLastError();
}

cudaError_t launch_potential(const SysDev *sys, int nsys, int max_items, cudaStream_t st) {
  if (max_items <= 0 || nsys <= 0) return cudaSuccess;
  dim3 grid((max_items + 255) / 256, nsys);
  k_potential<<<grid, 256, 0, st>>>(sys);
  return cudaGetLastError();
}

}  // namespace lhf
