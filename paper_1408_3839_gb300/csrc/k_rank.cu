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
// w_r = max_e |T_r[e]|, the truncated SVD of the weighted rows, v_r w_r = sum_a Y[r][a] s_a u_a,
// gives
//   V_j[e] ~ sum_{a < r1} <Q, u_a> D_a[e],   D_a[e] = s_a sum_r Y[r][a] T_r[e] / w_r,
// a rank-r1 form with the same structure: new direction-0 factors u_a, a transverse factor D_a
// in place of C1 (and 1 in place of C2), coefficients 1.  Keeping s_a > eps s_0, every entry
// moves by at most s_r1 ||Q_j,mu,nu||_2 ||(T_r[e] / w_r)_r||_2 <= s_r1 ||Q||_2 sqrt(R_tot).
// The SVD is a one-sided Jacobi on the rows (a warp per pair of rows, pairs in the round-robin
// order, rotations until every pair is orthogonal to 1e-15), in one CTA per system.
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
  double *A = sm;                      // [R][nv] weighted rows
  double *Y = A + (size_t)R * nv;      // [R][R] accumulated rotations (Y[r][a])
  __shared__ double w[kRankMaxRt], sg[kRankMaxRt];
  __shared__ int order[kRankMaxRt];
  __shared__ int r1_sh, busy;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  double *scratch = s.ws + s.offRR;    // [header 8][D: R mm][P1 of dir 1: 2 mm][P1 of dir 2: 2 mm]
  const double *C1 = s.ws + s.d[1].offC, *C2 = s.ws + s.d[2].offC;
  const double *V0 = s.ws + D0.offV;
  // weights w_r = max_e |c_r C1_r[e] C2_r[e]|
  for (int r = warp; r < R; r += kRankThreads / 32) {
    double m = 0.0;
    for (int e = lane; e < mm; e += 32) m = fmax(m, fabs(s.c[r] * C1[(int64_t)r * mm + e] * C2[(int64_t)r * mm + e]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) w[r] = m;
  }
  __syncthreads();
  for (int64_t t = tid; t < (int64_t)R * nv; t += kRankThreads) {
    const int r = (int)(t / nv);
    A[t] = V0[t] * w[r];
  }
  for (int t = tid; t < R * R; t += kRankThreads) Y[t] = (t / R == t % R) ? 1.0 : 0.0;
  __syncthreads();
  // one-sided Jacobi: rows p, q rotated until orthogonal
  const int np = (R + 1) / 2 * 2, half = np / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (tid == 0) busy = 0;
    __syncthreads();
    for (int step = 0; step < np - 1; ++step) {
      for (int k = warp; k < half; k += kRankThreads / 32) {
        int a, b;
        if (k == 0) {
          a = step;
          b = np - 1;
        } else {
          a = (step + k) % (np - 1);
          b = (step - k + (np - 1)) % (np - 1);
        }
        const int p = min(a, b), q = max(a, b);
        if (q >= R) continue;
        double *ap = A + (size_t)p * nv, *aq = A + (size_t)q * nv;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < nv; i += 32) {
          al = fma(ap[i], ap[i], al);
          be = fma(aq[i], aq[i], be);
          ga = fma(ap[i], aq[i], ga);
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (!(fabs(ga) > 1e-15 * sqrt(al * be))) continue;  // orthogonal (or a zero row)
        const double ze = (be - al) / (2.0 * ga);
        const double t = (ze >= 0.0 ? 1.0 : -1.0) / (fabs(ze) + sqrt(1.0 + ze * ze));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
        for (int i = lane; i < nv; i += 32) {
          const double x = ap[i], y = aq[i];
          ap[i] = c * x - sn * y;
          aq[i] = sn * x + c * y;
        }
        for (int r = lane; r < R; r += 32) {
          const double x = Y[r * R + p], y = Y[r * R + q];
          Y[r * R + p] = c * x - sn * y;
          Y[r * R + q] = sn * x + c * y;
        }
        if (lane == 0) busy = 1;
      }
      __syncthreads();
    }
    if (!busy) break;
    __syncthreads();
  }
  // singular values, descending order, rank
  for (int a = warp; a < R; a += kRankThreads / 32) {
    double n2 = 0.0;
    for (int i = lane; i < nv; i += 32) n2 = fma(A[(size_t)a * nv + i], A[(size_t)a * nv + i], n2);
    for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    if (lane == 0) sg[a] = sqrt(n2);
  }
  __syncthreads();
  for (int a = tid; a < R; a += kRankThreads) {
    int rank = 0;
    for (int b = 0; b < R; ++b)
      if (sg[b] > sg[a] || (sg[b] == sg[a] && b < a)) ++rank;
    order[rank] = a;
  }
  __syncthreads();
  if (tid == 0) {
    const double smax = sg[order[0]];
    int r1 = 0;
    while (r1 < R && sg[order[r1]] > s.rank_eps * smax) ++r1;
    if (r1 < 1) r1 = 1;
    r1_sh = r1;
    scratch[0] = (double)R;
    scratch[1] = (double)r1;
    scratch[2] = r1 < R ? sg[order[r1]] : 0.0;  // s_r1, the largest dropped singular value
    scratch[3] = smax;
  }
  __syncthreads();
  const int r1 = r1_sh;
  if (r1 >= R) return;  // nothing to drop: the descriptor stays as it is
  double *Dsc = scratch + 8, *P1a = Dsc + (size_t)r1 * mm, *P1b = P1a + 2 * mm;
  // D_k[e] = s_a sum_r Y[r][a] T_r[e] / w_r for the k-th largest a; the P1 slots of C1, C2
  for (int t = tid; t < r1 * mm; t += kRankThreads) {
    const int k = t / mm, e = t - (t / mm) * mm, a = order[k];
    double acc = 0.0;
    for (int r = 0; r < R; ++r)
      if (w[r] > 0.0) acc = fma(Y[r * R + a] / w[r], s.c[r] * C1[(int64_t)r * mm + e] * C2[(int64_t)r * mm + e], acc);
    Dsc[t] = sg[a] * acc;
  }
  for (int t = tid; t < 2 * mm; t += kRankThreads) {
    P1a[t] = C1[(int64_t)R * mm + t];
    P1b[t] = C2[(int64_t)R * mm + t];
  }
  __syncthreads();
  // the reduced system: direction-0 rows u_k = A_a / s_a, transverse factors D_k and 1, P1
  // slots after the r1 rank slots, coefficients 1
  double *V0w = s.ws + D0.offV;
  double *C1w = s.ws + s.d[1].offC, *C2w = s.ws + s.d[2].offC;
  for (int64_t t = tid; t < (int64_t)r1 * nv; t += kRankThreads) {
    const int k = (int)(t / nv), i = (int)(t - (int64_t)k * nv), a = order[k];
    V0w[t] = A[(size_t)a * nv + i] / sg[a];
  }
  for (int t = tid; t < r1 * mm; t += kRankThreads) {
    C1w[t] = Dsc[t];
    C2w[t] = 1.0;
  }
  for (int t = tid; t < 2 * mm; t += kRankThreads) {
    C1w[(int64_t)r1 * mm + t] = P1a[t];
    C2w[(int64_t)r1 * mm + t] = P1b[t];
  }
  for (int k = tid; k < r1; k += kRankThreads) s.c[k] = 1.0;
  __syncthreads();
  if (tid == 0) s.Rt = r1;
}

}  // namespace

size_t rank_reduce_smem_bytes(int R, int nv) { return ((size_t)R * nv + (size_t)R * R) * sizeof(double); }

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
