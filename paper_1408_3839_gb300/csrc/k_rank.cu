// k_rank.cu -- rank reduction of the lattice-summed potential of a one-dimensional lattice
// (the rank optimisation of the canonical potential tensor, Sec. 3.2).
//
// The nuclear part of a block of an (L,1,1) lattice is a sum over the R_tot = M0 R rank terms
// (Lemma 3.1, eq. (4.1)):
//   V_j[mu][nu] = sum_r <Q_j,mu,nu, v_r> T_r[mu][nu],   T_r = c_r C1_r (.) C2_r,
// with v_r the direction-0 factor over one cell (the potential rows, n_v = n_cell nodes), Q the
// fold over the cells of the product row g_mu,j g_nu (the weighted Gram's left operand) and C1,
// C2 the single-cell transverse factors.  The R_tot rows v_r are far from independent: after the
// lattice sum the wide Gaussians are nearly constant over a cell.  With weights
// w_r = max_e |T_r[e]|, a rank-revealing Gram-Schmidt of the weighted rows a_r = v_r w_r (at each
// step the row with the largest residual is normalised into q_k and projected out of the others,
// twice) stops once every residual is at most eps times the first pivot's norm, leaving
// a_r = sum_k R[r][k] q_k + res_r, ||res_r|| <= rho.  Then
//   V_j[e] ~ sum_{k < r1} <Q, q_k> D_k[e],   D_k[e] = sum_r R[r][k] T_r[e] / w_r,
// a rank-r1 form with the same structure: new direction-0 factors q_k, a transverse factor D_k
// in place of C1 (and 1 in place of C2), coefficients 1; every entry moves by at most
// sum_r |<Q, res_r>| |T_r[e]| / w_r <= rho ||Q_j,mu,nu||_2 R_tot.  One CTA per system, r1
// sequential steps.
#include <math.h>

#include "lhf_internal.cuh"

namespace lhf {
namespace {

constexpr int kRankThreads = 1024;
constexpr int kRankMaxRt = kRankReduceMaxRt;

__global__ void __launch_bounds__(kRankThreads) k_rank_reduce(SysDev *__restrict__ sysv) {
  SysDev &s = sysv[blockIdx.x];
  if (!(s.rank_eps > 0.0) || s.box) return;
  const int R = s.Rt, m0 = s.m0, mm = m0 * m0;
  const DirDev &D0 = s.d[0];
  const int nv = D0.nv;
  extern __shared__ double sm[];
  double *A = sm;                      // [R][nv] weighted rows, turned into their residuals
  double *Qb = A + (size_t)R * nv;     // [R][nv] the orthonormal rows q_k
  double *Rc = Qb + (size_t)R * nv;    // [R][R] coefficients: a_r = sum_k Rc[r][k] q_k + residual_r
  __shared__ double w[kRankMaxRt], nrm[kRankMaxRt];
  __shared__ int done[kRankMaxRt];
  __shared__ int piv, r1_sh;
  __shared__ double rho0, rho;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int kWarps = kRankThreads / 32;
  double *scratch = s.ws + s.offRR;    // [header 8][D: R mm][P1 of dir 1: 2 mm][P1 of dir 2: 2 mm]
  const double *C1 = s.ws + s.d[1].offC, *C2 = s.ws + s.d[2].offC;
  const double *V0 = s.ws + D0.offV;
  // weights w_r = max_e |c_r C1_r[e] C2_r[e]|
  for (int r = warp; r < R; r += kWarps) {
    double m = 0.0;
    for (int e = lane; e < mm; e += 32) m = fmax(m, fabs(s.c[r] * C1[(int64_t)r * mm + e] * C2[(int64_t)r * mm + e]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) w[r] = m;
  }
  __syncthreads();
  for (int64_t t = tid; t < (int64_t)R * nv; t += kRankThreads) A[t] = V0[t] * w[(int)(t / nv)];
  for (int t = tid; t < R * R; t += kRankThreads) Rc[t] = 0.0;
  for (int r = tid; r < R; r += kRankThreads) done[r] = 0;
  __syncthreads();
  int k = 0;
  for (; k < R; ++k) {
    // residual norms, the pivot (largest), the stopping test against the first pivot's norm
    for (int r = warp; r < R; r += kWarps) {
      double n2 = 0.0;
      for (int i = lane; i < nv; i += 32) n2 = fma(A[(size_t)r * nv + i], A[(size_t)r * nv + i], n2);
      for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
      if (lane == 0) nrm[r] = done[r] ? -1.0 : n2;
    }
    __syncthreads();
    if (tid == 0) {
      int p = -1;
      double best = -1.0;
      for (int r = 0; r < R; ++r)
        if (nrm[r] > best) {
          best = nrm[r];
          p = r;
        }
      const double rn = best > 0.0 ? sqrt(best) : 0.0;
      if (k == 0) rho0 = rn;
      rho = rn;
      piv = (p >= 0 && rn > s.rank_eps * rho0 && rn > 0.0) ? p : -1;
    }
    __syncthreads();
    const int p = piv;
    if (p < 0) break;
    // q_k = residual_p / ||residual_p||; Rc[p][k] = ||residual_p||
    const double inv = 1.0 / rho;
    for (int i = tid; i < nv; i += kRankThreads) Qb[(size_t)k * nv + i] = A[(size_t)p * nv + i] * inv;
    if (tid == 0) {
      Rc[p * R + k] = rho;
      done[p] = 1;
    }
    __syncthreads();
    // every other row: a_r -= <a_r, q_k> q_k, twice (reorthogonalisation), coefficients summed
    for (int pass = 0; pass < 2; ++pass) {
      for (int r = warp; r < R; r += kWarps) {
        if (done[r]) continue;
        double d = 0.0;
        for (int i = lane; i < nv; i += 32) d = fma(A[(size_t)r * nv + i], Qb[(size_t)k * nv + i], d);
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        for (int i = lane; i < nv; i += 32) A[(size_t)r * nv + i] -= d * Qb[(size_t)k * nv + i];
        if (lane == 0) Rc[r * R + k] += d;
      }
      __syncthreads();
    }
    for (int i = tid; i < nv; i += kRankThreads) A[(size_t)p * nv + i] = 0.0;
    __syncthreads();
  }
  if (tid == 0) {
    r1_sh = k < 1 ? 1 : k;
    scratch[0] = (double)R;
    scratch[1] = (double)r1_sh;
    scratch[2] = k < R ? rho : 0.0;  // the largest residual row norm left out
    scratch[3] = rho0;
  }
  __syncthreads();
  const int r1 = r1_sh;
  if (r1 >= R) return;  // nothing to drop: the descriptor stays as it is
  double *Dsc = scratch + 8, *P1a = Dsc + (size_t)r1 * mm, *P1b = P1a + 2 * mm;
  // D_k[e] = sum_r Rc[r][k] T_r[e] / w_r; the P1 slots of C1, C2
  for (int t = tid; t < r1 * mm; t += kRankThreads) {
    const int kk = t / mm, e = t - (t / mm) * mm;
    double acc = 0.0;
    for (int r = 0; r < R; ++r)
      if (w[r] > 0.0) acc = fma(Rc[r * R + kk] / w[r], s.c[r] * C1[(int64_t)r * mm + e] * C2[(int64_t)r * mm + e], acc);
    Dsc[t] = acc;
  }
  for (int t = tid; t < 2 * mm; t += kRankThreads) {
    P1a[t] = C1[(int64_t)R * mm + t];
    P1b[t] = C2[(int64_t)R * mm + t];
  }
  __syncthreads();
  // the reduced system: direction-0 rows q_k, transverse factors D_k and 1, P1 slots after the
  // r1 rank slots, coefficients 1
  double *V0w = s.ws + D0.offV;
  double *C1w = s.ws + s.d[1].offC, *C2w = s.ws + s.d[2].offC;
  for (int64_t t = tid; t < (int64_t)r1 * nv; t += kRankThreads) V0w[t] = Qb[t];
  for (int t = tid; t < r1 * mm; t += kRankThreads) {
    C1w[t] = Dsc[t];
    C2w[t] = 1.0;
  }
  for (int t = tid; t < 2 * mm; t += kRankThreads) {
    C1w[(int64_t)r1 * mm + t] = P1a[t];
    C2w[(int64_t)r1 * mm + t] = P1b[t];
  }
  for (int kk = tid; kk < r1; kk += kRankThreads) s.c[kk] = 1.0;
  __syncthreads();
  if (tid == 0) s.Rt = r1;
}

}  // namespace

size_t rank_reduce_smem_bytes(int R, int nv) { return ((size_t)2 * R * nv + (size_t)R * R) * sizeof(double); }

cudaError_t launch_rank_reduce(SysDev *sys, int nsys, size_t smem, cudaStream_t st) {
  if (nsys <= 0 || smem == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_rank_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kmark(LHF_K_GRAM_FP64, 1, st);
  k_rank_reduce<<<nsys, kRankThreads, smem, st>>>(sys);
  kmark(LHF_K_GRAM_FP64, 0, st);
  return cudaGetLastError();
}

}  // namespace lhf
