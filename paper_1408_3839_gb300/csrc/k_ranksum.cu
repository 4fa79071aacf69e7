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
// A CTA takes 32 consecutive entries (mu, nu) of one transverse block pair (j1, j2) and a group
// of kRsGroup direction-0 window blocks: its 8 warps first form the weights w_r = c_r C1_r C2_r
// of its entries in shared memory (two multiplications per term and entry), then each warp runs
// kRsNB blocks at one FMA per rank term and block, a lane per entry (the factor slots read
// coalesced).  Recomputing c_r C1_r C2_r for every block would double the FP64 work (issued at
// 1/64 of the FP32 rate here); small groups keep many CTAs resident for the loads of the factor
// slots, which bound the kernel (measured on tube_256: one block per warp, 48 warps per SM).  The
// blocks outside the window get one CTA each (block decoded once per CTA).  Factor blocks outside
// the contracted half of a window are read from their mirrors, C_r[-j][mu][nu] = C_r[j][nu][mu]
// (the transposed entry of the mirrored block).
#include "lhf_internal.cuh"

namespace lhf {
namespace {


__device__ __forceinline__ int wrap_block(int j, int L) {
  j %= L;
  return j < 0 ? j + L : j;
}

constexpr int kRsThreads = 256, kRsWarps = kRsThreads / 32, kRsNB = 1;
constexpr int kRsGroup = kRsWarps * kRsNB;  // direction-0 blocks per CTA

__global__ void __launch_bounds__(kRsThreads, 6) k_ranksum(const SysDev *__restrict__ sysv, int compute_ctas) {
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
    if (!outside) return;  // inside the window: written by the compute CTAs
    double *H = s.H + (int64_t)blk * mm, *S = s.S + (int64_t)blk * mm;
    for (int i = threadIdx.x; i < mm; i += blockDim.x) {
      H[i] = 0.0;
      S[i] = 0.0;
    }
    return;
  }
  const int echunks = (mm + 31) / 32, bgroups = (D0.J + kRsGroup - 1) / kRsGroup;
  const int cta = (int)blockIdx.x;
  if (cta >= D1.J * D2.J * echunks * bgroups) return;  // CTA-uniform
  const int bg = cta % bgroups, ec = (cta / bgroups) % echunks, pair = cta / (bgroups * echunks);
  const int jw2 = pair % D2.J, jw1 = pair / D2.J;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e = ec * 32 + lane;
  const bool act = e < mm;
  const int mu = act ? e / m0 : 0, nu = act ? e - (e / m0) * m0 : 0;
  const double *F1 = factor_entry(s, D1, jw1, mu, nu);
  const double *F2 = factor_entry(s, D2, jw2, mu, nu);
  extern __shared__ double wsh[];  // [Rt][32]
  for (int r = warp; r < Rt; r += kRsWarps)
    wsh[r * 32 + lane] = act ? s.c[r] * F1[(int64_t)r * mm] * F2[(int64_t)r * mm] : 0.0;
  __syncthreads();
  if (!act) return;
  const int64_t ok = (int64_t)Rt * mm, om = (int64_t)(Rt + 1) * mm;
  const double K1 = F1[ok], K2 = F2[ok], M1 = F1[om], M2 = F2[om];
  const double P = M1 * M2, Q = K1 * M2 + M1 * K2;
  const int64_t col = ((int64_t)wrap_block(D1.jlo + jw1, D1.L)) * D2.L + wrap_block(D2.jlo + jw2, D2.L);
  const int bend = min(D0.J, (bg + 1) * kRsGroup);
  for (int b0 = bg * kRsGroup + warp; b0 < bend; b0 += kRsGroup) {
    // the batch's factor entries as offsets from the direction-0 factors (fewer registers than
    // pointers; the region holds fewer than 2^31 values)
    const double *C0 = s.ws + D0.offC;
    int f0[kRsNB];
#pragma unroll
    for (int i = 0; i < kRsNB; ++i) {
      const int b = b0 + kRsWarps * i;
      f0[i] = (int)(factor_entry(s, D0, b < bend ? b : b0, mu, nu) - C0);
    }
    double acc[kRsNB];
#pragma unroll
    for (int i = 0; i < kRsNB; ++i) acc[i] = 0.0;
    // unrolled: the loads of several rank terms are in flight together
#pragma unroll 4
    for (int r = 0; r < Rt; ++r) {
      const double *Cr = C0 + (int64_t)r * mm;
      const double w = wsh[r * 32 + lane];
#pragma unroll
      for (int i = 0; i < kRsNB; ++i) acc[i] = fma(w, Cr[f0[i]], acc[i]);
    }
#pragma unroll
    for (int i = 0; i < kRsNB; ++i) {
      const int b = b0 + kRsWarps * i;
      if (b >= bend) break;
      const double K0 = C0[ok + f0[i]], M0 = C0[om + f0[i]];
      const int64_t blk = (int64_t)wrap_block(D0.jlo + b, D0.L) * D1.L * D2.L + col;
      s.H[blk * mm + e] = 0.5 * (K0 * P + M0 * Q) - acc[i];
      s.S[blk * mm + e] = M0 * P;
    }
  }
}

}  // namespace

int ranksum_ctas(const SysDev &s) {
  return s.d[1].J * s.d[2].J * ((s.m0 * s.m0 + 31) / 32) * ((s.d[0].J + kRsGroup - 1) / kRsGroup);
}

cudaError_t launch_ranksum(const SysDev *sys, int nsys, int max_compute_ctas, int max_blocks, int max_rt,
                           cudaStream_t st) {
  if (max_blocks <= 0 || nsys <= 0) return cudaSuccess;
  const size_t smem = (size_t)max_rt * 32 * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_ranksum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(max_compute_ctas + max_blocks, nsys);
  kmark(LHF_K_RANKSUM, 1, st);
  k_ranksum<<<grid, kRsThreads, smem, st>>>(sys, max_compute_ctas);
  kmark(LHF_K_RANKSUM, 0, st);
  return cudaGetLastError();
}

}  // namespace lhf
