// k_orbital.cu -- Bloch orbitals on the grid (eq. (6.8) expanded in the basis; Sec. 3.4).
//
// The eigenvector of the lattice matrix for k-point kappa with Bloch vector u (eq. (6.8)) is the
// function
//   psi(x) = N^{-1/2} sum_p exp(2 pi i kappa . p / L) sum_mu u_mu phi_mu(x - p b),  N = L0 L1 L2,
// over the lattice cells p, with phi_mu(x - p b) = prod_l g_mu^l(x_l - p_l b_l) separable
// (eq. (3.14); periodised along periodic directions).  Summing the phases direction by
// direction gives a rank-m0 separable form on the grid:
//   psi(i0, i1, i2) = N^{-1/2} sum_mu u_mu B0_mu(i0) B1_mu(i1) B2_mu(i2),
//   Bl_mu(i) = sum_{p=0}^{L_l - 1} exp(2 pi i kappa_l p / L_l) g_mu^l(i - p n_c)   (node i - p n_c mod n
//   in a periodic direction; a single cell otherwise).
// k_bloch_factors: thread per (direction, mu, node of the requested window): Bl_mu(i), the cell
//   phases tabulated per CTA in shared memory.
// k_orbital_values: thread per (orbital, grid point of the window): the rank-m0 sum.
#include "lhf_internal.cuh"

namespace lhf {
namespace {

constexpr int kOrbThreads = 256;

struct OrbArgs {
  int kappa[3], lo[3], cnt[3];
  int norb;
  const double2 *coef;  // [norb][m0]
  double2 *B;           // [3][m0][max cnt] Bloch-summed factors
  double2 *out;         // [norb][cnt0][cnt1][cnt2]
  int ldB;              // max cnt
};

__global__ void __launch_bounds__(kOrbThreads) k_bloch_factors(const SysDev *__restrict__ sysv, OrbArgs a) {
  const SysDev &s = sysv[0];
  const int m0 = s.m0;
  extern __shared__ double2 phase[];  // [L_l] exp(2 pi i kappa_l p / L_l)
  const int l = blockIdx.y;
  const DirDev &D = s.d[l];
  const int Ll = D.L;
  for (int p = threadIdx.x; p < Ll; p += blockDim.x) {
    long long t = ((long long)a.kappa[l] * p) % Ll;
    if (t < 0) t += Ll;
    double sn, cs;
    sincospi(2.0 * (double)t / (double)Ll, &sn, &cs);
    phase[p] = make_double2(cs, sn);
  }
  __syncthreads();
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= (int64_t)m0 * a.cnt[l]) return;
  const int mu = (int)(item / a.cnt[l]), k = (int)(item - (int64_t)mu * a.cnt[l]);
  const int i = a.lo[l] + k;
  const double *G = s.ws + D.offG + (int64_t)mu * (D.n + D.gext) + D.gext;
  double2 acc = make_double2(0.0, 0.0);
  if (D.periodic) {
    for (int p = 0; p < Ll; ++p) {  // the rows are zero outside the support windows (filled first)
      int e = i - p * D.nc;
      e %= D.n;
      if (e < 0) e += D.n;
      const double g = G[e];
      if (g == 0.0) continue;
      acc.x = fma(g, phase[p].x, acc.x);
      acc.y = fma(g, phase[p].y, acc.y);
    }
  } else {
    acc.x = G[i];  // a single cell
  }
  a.B[((int64_t)l * m0 + mu) * a.ldB + k] = acc;
}

__global__ void __launch_bounds__(kOrbThreads) k_orbital_values(const SysDev *__restrict__ sysv, OrbArgs a) {
  const SysDev &s = sysv[0];
  const int m0 = s.m0;
  const int64_t npts = (int64_t)a.cnt[0] * a.cnt[1] * a.cnt[2];
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= npts * a.norb) return;
  const int o = (int)(item / npts);
  const int64_t pt = item - (int64_t)o * npts;
  const int k2 = (int)(pt % a.cnt[2]), k1 = (int)((pt / a.cnt[2]) % a.cnt[1]), k0 = (int)(pt / ((int64_t)a.cnt[1] * a.cnt[2]));
  const double2 *u = a.coef + (int64_t)o * m0;
  const double2 *B0 = a.B + k0, *B1 = a.B + (int64_t)m0 * a.ldB + k1, *B2 = a.B + (int64_t)2 * m0 * a.ldB + k2;
  double2 acc = make_double2(0.0, 0.0);
  for (int mu = 0; mu < m0; ++mu) {
    const double2 x = B0[(int64_t)mu * a.ldB], y = B1[(int64_t)mu * a.ldB], z = B2[(int64_t)mu * a.ldB];
    const double2 xy = make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
    const double2 w = make_double2(xy.x * z.x - xy.y * z.y, xy.x * z.y + xy.y * z.x);
    const double2 c = u[mu];
    acc.x += c.x * w.x - c.y * w.y;
    acc.y += c.x * w.y + c.y * w.x;
  }
  const double nrm = rsqrt((double)s.d[0].L * s.d[1].L * s.d[2].L);
  a.out[item] = make_double2(acc.x * nrm, acc.y * nrm);
}

}  // namespace

cudaError_t launch_orbitals(const SysDev *sys, const int *kappa, const int *lo, const int *cnt, int norb,
                            const double *coef, double *B, double *out, int m0, int maxL, cudaStream_t st) {
  OrbArgs a;
  int ld = 0;
  for (int l = 0; l < 3; ++l) {
    a.kappa[l] = kappa[l];
    a.lo[l] = lo[l];
    a.cnt[l] = cnt[l];
    ld = cnt[l] > ld ? cnt[l] : ld;
  }
  a.norb = norb;
  a.coef = reinterpret_cast<const double2 *>(coef);
  a.B = reinterpret_cast<double2 *>(B);
  a.out = reinterpret_cast<double2 *>(out);
  a.ldB = ld;
  const size_t smem = sizeof(double2) * (size_t)maxL;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_bloch_factors, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int64_t items = (int64_t)m0 * ld;
  k_bloch_factors<<<dim3((unsigned)((items + kOrbThreads - 1) / kOrbThreads), 3), kOrbThreads, smem, st>>>(sys, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t n = (int64_t)cnt[0] * cnt[1] * cnt[2] * norb;
  k_orbital_values<<<(unsigned)((n + kOrbThreads - 1) / kOrbThreads), kOrbThreads, 0, st>>>(sys, a);
  return cudaGetLastError();
}

}  // namespace lhf
