// k_ranksum.cu -- step a5: Hadamard products over the three directions and the rank sum, FP64.
//
// For every window block j = (j0, j1, j2) and entry (mu, nu) (eq. (3.10), Lemma 3.1 proof;
// Lemma 4.1 eqs. (4.2), (4.5), (4.6); eq. (3.4)):
//   S_j = M0 M1 M2                              (overlap, rank 1 in the directions)
//   T_j = K0 M1 M2 + M0 K1 M2 + M0 M1 K2        (P1 Laplacian, rank 3)
//   V_j = sum_r c_r C0_r C1_r C2_r              (nuclear attraction, rank R_tot)
//   H_j = T_j / 2 - V_j
// written to block (j0 mod L0, j1 mod L1, j2 mod L2) of the first block column.  Blocks
// outside the window are zero-filled by the host before the launch (step a6).
// Thread per (block, entry): consecutive threads read consecutive entries of each factor slot
// (coalesced); the loop over r streams the three directions' factors.
#include "lhf_internal.cuh"

namespace lhf {
namespace {

__global__ void __launch_bounds__(256) k_ranksum(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box) return;
  const int m0 = s.m0, mm = m0 * m0, Rt = s.Rt;
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= (int64_t)s.nwin * mm) return;
  const int w = (int)(item / mm);
  const int e = (int)(item - (int64_t)w * mm);
  const int J1 = s.d[1].J, J2 = s.d[2].J;
  const int jw0 = w / (J1 * J2);
  const int jw1 = (w / J2) % J1;
  const int jw2 = w % J2;
  const int jw[3] = {jw0, jw1, jw2};
  const double *F[3];
  int jj[3];
  for (int l = 0; l < 3; ++l) {
    const DirDev &D = s.d[l];
    F[l] = s.ws + D.offC + (int64_t)jw[l] * (Rt + 2) * mm + e;
    int j = (D.jlo + jw[l]) % D.L;
    jj[l] = j < 0 ? j + D.L : j;
  }
  double v = 0.0;
  for (int r = 0; r < Rt; ++r) {
    const int64_t o = (int64_t)r * mm;
    v += s.c[r] * F[0][o] * F[1][o] * F[2][o];
  }
  const int64_t ok = (int64_t)Rt * mm, om = (int64_t)(Rt + 1) * mm;
  const double K0 = F[0][ok], K1 = F[1][ok], K2 = F[2][ok];
  const double M0 = F[0][om], M1 = F[1][om], M2 = F[2][om];
  const double S = M0 * M1 * M2;
  const double T = K0 * M1 * M2 + M0 * K1 * M2 + M0 * M1 * K2;
  const int64_t blk = ((int64_t)jj[0] * s.d[1].L + jj[1]) * s.d[2].L + jj[2];
  s.H[blk * mm + e] = 0.5 * T - v;
  s.S[blk * mm + e] = S;
}

}  // namespace

cudaError_t launch_ranksum(const SysDev *sys, int nsys, int max_items, cudaStream_t st) {
  if (max_items <= 0 || nsys <= 0) return cudaSuccess;
  dim3 grid((max_items + 255) / 256, nsys);
  k_ranksum<<<grid, 256, 0, st>>>(sys);
  return cudaGetLastError();
}

}  // namespace lhf
