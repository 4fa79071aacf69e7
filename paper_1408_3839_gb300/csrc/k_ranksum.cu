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
//
// A thread takes one entry (mu, nu) of GROUP consecutive direction-0 window blocks with the
// same (j1, j2): the weights w_r = c_r C1_r C2_r are formed once and each block costs one FMA
// per rank term.  The blocks outside the window get one CTA each (block decoded once per CTA).
// Factor blocks outside the contracted half of a window are read from their mirrors,
// C_r[-j][mu][nu] = C_r[j][nu][mu] (the transposed entry of the mirrored block).
// Consecutive threads take consecutive entries: the factor slots are read coalesced.  GROUP = 2
// when every system's windows in directions 1 and 2 are single blocks (tubes: more threads for a
// latency-bound loop), else 4 (fewer redundant weights where the (j1, j2) window is wide).
#include "lhf_internal.cuh"

namespace lhf {
namespace {


__device__ __forceinline__ int wrap_block(int j, int L) {
  j %= L;
  return j < 0 ? j + L : j;
}

template <int GROUP>
__global__ void __launch_bounds__(256) k_ranksum(const SysDev *__restrict__ sysv, int compute_ctas) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box) return;
  const int m0 = s.m0, mm = m0 * m0, Rt = s.Rt;
  const DirDev &D0 = s.d[0], &D1 = s.d[1], &D2 = s.d[2];
  if ((int)blockIdx.x >= compute_ctas) {
    // zeros outside the window (a6): CTA per block, thread per entry
    const int blk = (int)blockIdx.x - compute_ctas;
    if (blk >= s.nblocks) return;
    const int jj[3] = {blk / (D1.L * D2.L), (blk / D2.L) % D1.L, blk % D2.L};
    bool outside = false;
    for (int l = 0; l < 3; ++l) outside |= wrap_block(jj[l] - s.d[l].jlo, s.d[l].L) >= s.d[l].J;
    if (!outside) return;  // inside the window: written by the compute threads
    double *H = s.H + (int64_t)blk * mm, *S = s.S + (int64_t)blk * mm;
    for (int i = threadIdx.x; i < mm; i += blockDim.x) {
      H[i] = 0.0;
      S[i] = 0.0;
    }
    return;
  }
  const int groups = (D0.J + GROUP - 1) / GROUP;
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= (int64_t)D1.J * D2.J * groups * mm) return;
  const int e = (int)(item % mm);
  int64_t rest = item / mm;
  const int g = (int)(rest % groups);
  rest /= groups;
  const int jw2 = (int)(rest % D2.J), jw1 = (int)(rest / D2.J);
  const int mu = e / m0, nu = e - mu * m0;
  const double *F1 = factor_entry(s, D1, jw1, mu, nu);
  const double *F2 = factor_entry(s, D2, jw2, mu, nu);
  const double *F0[GROUP];
  const int jw0_0 = g * GROUP;
  const int nb = min(GROUP, D0.J - jw0_0);
#pragma unroll
  for (int b = 0; b < GROUP; ++b) F0[b] = factor_entry(s, D0, jw0_0 + (b < nb ? b : 0), mu, nu);
  double acc[GROUP];
#pragma unroll
  for (int b = 0; b < GROUP; ++b) acc[b] = 0.0;
  // unrolled: the loads of four rank terms are in flight together
#pragma unroll 4
  for (int r = 0; r < Rt; ++r) {
    const int64_t o = (int64_t)r * mm;
    const double w = s.c[r] * F1[o] * F2[o];
#pragma unroll
    for (int b = 0; b < GROUP; ++b) acc[b] = fma(w, F0[b][o], acc[b]);
  }
  const int64_t ok = (int64_t)Rt * mm, om = (int64_t)(Rt + 1) * mm;
  const double K1 = F1[ok], K2 = F2[ok], M1 = F1[om], M2 = F2[om];
  const double P = M1 * M2, Q = K1 * M2 + M1 * K2;
  const int64_t col = ((int64_t)wrap_block(D1.jlo + jw1, D1.L)) * D2.L + wrap_block(D2.jlo + jw2, D2.L);
#pragma unroll
  for (int b = 0; b < GROUP; ++b) {
    if (b >= nb) break;
    const double K0 = F0[b][ok], M0 = F0[b][om];
    const int64_t blk = (int64_t)wrap_block(D0.jlo + jw0_0 + b, D0.L) * D1.L * D2.L + col;
    s.H[blk * mm + e] = 0.5 * (K0 * P + M0 * Q) - acc[b];
    s.S[blk * mm + e] = M0 * P;
  }
}

}  // namespace

int ranksum_group(const SysDev &s) { return s.d[1].J * s.d[2].J == 1 ? 2 : 4; }

int ranksum_compute_items(const SysDev &s, int group) {
  const int groups = (s.d[0].J + group - 1) / group;
  return s.d[1].J * s.d[2].J * groups * s.m0 * s.m0;
}

cudaError_t launch_ranksum(const SysDev *sys, int nsys, int max_compute_items, int max_blocks, int group,
                           cudaStream_t st) {
  if (max_blocks <= 0 || nsys <= 0) return cudaSuccess;
  const int compute_ctas = (max_compute_items + 255) / 256;
  dim3 grid(compute_ctas + max_blocks, nsys);
  kmark(LHF_K_RANKSUM, 1, st);
  if (group == 2)
    k_ranksum<2><<<grid, 256, 0, st>>>(sys, compute_ctas);
  else
    k_ranksum<4><<<grid, 256, 0, st>>>(sys, compute_ctas);
  kmark(LHF_K_RANKSUM, 0, st);
  return cudaGetLastError();
}

}  // namespace lhf
