// k_kspace.cu -- the separable k-space route to the k-point blocks (Theorem 2.5; Prop. 4.2).
//
// The blocks of the first block column are sums of Hadamard products of per-direction factors
// (Lemma 4.1): X_j = sum_r c_r C0_r[j0] o C1_r[j1] o C2_r[j2] (and the rank-1 / rank-3 forms of
// the overlap and the P1 Laplacian).  Since omega^{kappa . j} = prod_l omega_l^{kappa_l j_l}, the
// DFT over the lattice of such a sum is the same sum of Hadamard products of the 1D DFTs of the
// factors:
//   Xbar_kappa = sum_r c_r F0_r(kappa_0) o F1_r(kappa_1) o F2_r(kappa_2),
//   Fl_r(kappa_l) = sum_{j_l in window} omega_l^{kappa_l j_l} Cl_r[j_l],  omega_l = exp(-2 pi i / L_l),
// so that
//   Sbar = M0 o M1 o M2,  Tbar = K0 o M1 o M2 + M0 o K1 o M2 + M0 o M1 o K2,
//   Vbar = sum_r c_r C0_r o C1_r o C2_r,  Hbar = Tbar / 2 - Vbar   (all hatted, complex).
// Only 1D transforms are taken (sum_l L_l (R_tot + 2) m0^2 factor entries instead of the
// L0 L1 L2 m0^2 blocks), and no real-space block is formed.
//
// k_factor_dft: one CTA per (system, direction, factor slot, chunk of kKappaChunk k-points);
//   threads over the m0^2 entries, each summing the window blocks (direct sum over the window,
//   twiddles for a tile of window blocks in shared memory).  Mirrored window blocks are read
//   from their contracted partners (factor_entry).
// k_kspace_blocks: thread per (solved k-point, entry): the Hadamard products and the rank sum;
//   the conjugate k-point receives the complex conjugate (real lattice matrices).
#include "lhf_internal.cuh"

namespace lhf {
namespace {

constexpr int kKsThreads = 256;
constexpr int kKappaChunk = 8;
constexpr int kWinTile = 32;

__global__ void __launch_bounds__(kKsThreads) k_factor_dft(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box) return;
  int b = blockIdx.x, l = 0;
  for (; l < 3; ++l) {
    const int cnt = (s.Rt + 2) * ((s.d[l].L + kKappaChunk - 1) / kKappaChunk);
    if (b < cnt) break;
    b -= cnt;
  }
  if (l == 3) return;
  const DirDev &D = s.d[l];
  const int nch = (D.L + kKappaChunk - 1) / kKappaChunk;
  const int slot = b / nch, kap0 = (b - slot * nch) * kKappaChunk;
  const int m0 = s.m0, mm = m0 * m0, L = D.L, J = D.J;
  __shared__ double2 tw[kKappaChunk][kWinTile];
  double2 *F = reinterpret_cast<double2 *>(s.ws + D.offF);
  for (int e0 = 0; e0 < mm; e0 += kKsThreads) {
    const int e = e0 + threadIdx.x;
    const int mu = e / m0, nu = e - (e / m0) * m0;
    double2 acc[kKappaChunk];
#pragma unroll
    for (int k = 0; k < kKappaChunk; ++k) acc[k] = make_double2(0.0, 0.0);
    for (int w0 = 0; w0 < J; w0 += kWinTile) {
      __syncthreads();
      // twiddles omega^{kappa j} for kappa = kap0 .. kap0 + 7 and the window tile j = jlo + w
      for (int t = threadIdx.x; t < kKappaChunk * kWinTile; t += kKsThreads) {
        const int k = t / kWinTile, w = t - k * kWinTile;
        const long long j = (long long)D.jlo + w0 + w;
        long long ph = ((long long)(kap0 + k) * j) % L;
        if (ph < 0) ph += L;
        double sn, cs;
        sincospi(-2.0 * (double)ph / (double)L, &sn, &cs);
        tw[k][w] = make_double2(cs, sn);
      }
      __syncthreads();
      if (e < mm) {
        const int wn = min(kWinTile, J - w0);
        for (int w = 0; w < wn; ++w) {
          const double x = factor_entry(s, D, w0 + w, mu, nu)[(int64_t)slot * mm];
#pragma unroll
          for (int k = 0; k < kKappaChunk; ++k) {
            acc[k].x = fma(x, tw[k][w].x, acc[k].x);
            acc[k].y = fma(x, tw[k][w].y, acc[k].y);
          }
        }
      }
    }
    if (e < mm)
#pragma unroll
      for (int k = 0; k < kKappaChunk; ++k)
        if (kap0 + k < L) F[((int64_t)(kap0 + k) * (s.Rt + 2) + slot) * mm + e] = acc[k];
  }
}

__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__global__ void __launch_bounds__(kKsThreads) k_kspace_blocks(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box || !s.klist) return;
  const int m0 = s.m0, mm = m0 * m0, Rt = s.Rt;
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= (int64_t)s.nkhalf * mm) return;
  const int w = (int)(item / mm), e = (int)(item - (int64_t)w * mm);
  const int kap = s.klist[w];
  const int L0 = s.d[0].L, L1 = s.d[1].L, L2 = s.d[2].L;
  const int k0 = kap / (L1 * L2), k1 = (kap / L2) % L1, k2 = kap % L2;
  const int mk = (((L0 - k0) % L0) * L1 + (L1 - k1) % L1) * L2 + (L2 - k2) % L2;
  const int64_t slots = Rt + 2;
  const double2 *F0 = reinterpret_cast<const double2 *>(s.ws + s.d[0].offF) + (int64_t)k0 * slots * mm + e;
  const double2 *F1 = reinterpret_cast<const double2 *>(s.ws + s.d[1].offF) + (int64_t)k1 * slots * mm + e;
  const double2 *F2 = reinterpret_cast<const double2 *>(s.ws + s.d[2].offF) + (int64_t)k2 * slots * mm + e;
  double2 v = make_double2(0.0, 0.0);
#pragma unroll 4
  for (int r = 0; r < Rt; ++r) {
    const int64_t o = (int64_t)r * mm;
    const double2 p = cmul2(cmul2(F1[o], F2[o]), F0[o]);
    v.x = fma(s.c[r], p.x, v.x);
    v.y = fma(s.c[r], p.y, v.y);
  }
  const int64_t ok = (int64_t)Rt * mm, om = (int64_t)(Rt + 1) * mm;
  const double2 K0 = F0[ok], K1 = F1[ok], K2 = F2[ok], M0 = F0[om], M1 = F1[om], M2 = F2[om];
  const double2 M12 = cmul2(M1, M2);
  const double2 Sv = cmul2(M0, M12);
  const double2 t = cmul2(K0, M12);
  const double2 u = cmul2(M0, cadd2(cmul2(K1, M2), cmul2(M1, K2)));
  const double2 Hv = make_double2(0.5 * (t.x + u.x) - v.x, 0.5 * (t.y + u.y) - v.y);
  double2 *Hb = reinterpret_cast<double2 *>(s.Hbar), *Sb = reinterpret_cast<double2 *>(s.Sbar);
  Hb[(int64_t)kap * mm + e] = Hv;
  Sb[(int64_t)kap * mm + e] = Sv;
  if (mk != kap) {
    Hb[(int64_t)mk * mm + e] = make_double2(Hv.x, -Hv.y);
    Sb[(int64_t)mk * mm + e] = make_double2(Sv.x, -Sv.y);
  }
}

}  // namespace

int kspace_factor_ctas(const SysDev &s) {
  int n = 0;
  for (int l = 0; l < 3; ++l) n += (s.Rt + 2) * ((s.d[l].L + kKappaChunk - 1) / kKappaChunk);
  return n;
}

cudaError_t launch_kspace(const SysDev *sys, int nsys, int max_factor_ctas, long long max_items, cudaStream_t st) {
  if (nsys <= 0 || max_factor_ctas <= 0 || max_items <= 0) return cudaSuccess;
  kmark(LHF_K_FACTOR_DFT, 1, st);
  k_factor_dft<<<dim3(max_factor_ctas, nsys), kKsThreads, 0, st>>>(sys);
  kmark(LHF_K_FACTOR_DFT, 0, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  kmark(LHF_K_KSPACE_BLOCKS, 1, st);
  k_kspace_blocks<<<dim3((unsigned)((max_items + kKsThreads - 1) / kKsThreads), nsys), kKsThreads, 0, st>>>(sys);
  kmark(LHF_K_KSPACE_BLOCKS, 0, st);
  return cudaGetLastError();
}

}  // namespace lhf
