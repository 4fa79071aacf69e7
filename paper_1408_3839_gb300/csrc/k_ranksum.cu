// k_ranksum.cu -- step a5: Hadamard products over the three directions and the rank sum, FP64.
//
// For every window block j = (j0, j1, j2) and entry (mu, nu) (eq. (3.10), Lemma 3.1 proof;
// Lemma 4.1 eqs. (4.2), (4.5), (4.6); eq. (3.4)):
//   S_j = M0 M1 M2                              (overlap, rank 1 in the directions)
//   T_j = K0 M1 M2 + M0 K1 M2 + M0 M1 K2        (P1 Laplacian, rank 3)
//   V_j = sum_r c_r C0_r C1_r C2_r              (nuclear attraction, rank R_tot)
//   H_j = T_j / 2 - V_j
// written to block (j0 mod L0, j1 mod L1, j2 mod L2) of the first block column; blocks outside
// the window are written as exact zeros by the same kernel (step a6).
// Thread per (block of the first block column, entry): consecutive threads read consecutive
// entries of each factor slot (coalesced); the loop over r streams the three directions' factors.
#include "lhf_internal.cuh"

namespace lhf {
namespace {

__global__ void __launch_bounds__(256) k_ranksum(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box) return;
  const int m0 = s.m0, mm = m0 * m0, Rt = s.Rt;
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= (int64_t)s.nblocks * mm) return;
  const int64_t blk = item / mm;
  const int e = (int)(item - blk * mm);
  const int L1 = s.d[1].L, L2 = s.d[2].L;
  const int jj[3] = {(int)(blk / ((int64_t)L1 * L2)), (int)((blk / L2) % L1), (int)(blk % L2)};
  // window index of each direction's displacement; outside the window the block is zero (a6)
  const double *F[3];
  bool inside = true;
  for (int l = 0; l < 3; ++l) {
    const DirDev &D = s.d[l];
    int jw = (jj[l] - D.jlo) % D.L;
    if (jw < 0) jw += D.L;
    if (jw >= D.J) inside = false;
    F[l] = s.ws + D.offC + (int64_t)(inside ? jw : 0) * (Rt + 2) * mm + e;
  }
  if (!inside) {
    s.H[item] = 0.0;
    s.S[item] = 0.0;
    return;
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
  s.H[item] = 0.5 * T - v;
  s.S[item] = S;
}

}  // namespace

cudaError_t launch_ranksum(const SysDev *sys, int nsys, int max_items, cudaStream_t st) {
  if (max_items <= 0 || nsys <= 0) return cudaSuccess;
  dim3 grid((max_items + 255) / 256, nsys);
  k_ranksum<<<grid, 256, 0, st>>>(sys);
  return cudaGetLastError();
}

}  // namespace lhf
