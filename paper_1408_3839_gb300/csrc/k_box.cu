// k_box.cu -- step a9, assembly: the open (L0,1,1) box, whose Hamiltonian is not block-circulant.
//
// In an open lattice direction the potential (summed over the actual nuclei of the L0 cells,
// eq. (3.8)-(3.9)) is not periodic, so the direction-0 factors of an entry depend on both
// cells, not only on their distance (Lemma 3.1 and its proof; the sparsity of Lemma 4.2 still
// limits the pairs to those whose supports overlap).  For the copy of mu in cell p and of nu in
// cell p + d (d in the overlap window):
//   C_r[p][d][mu][nu] = sum_i g_mu(i - p n_c) v_r(i) g_nu(i - (p + d) n_c)      r < R_tot
//   K[p][d][mu][nu]   = g_{mu,p}^T A g_{nu,p+d},  A = (1/h) tridiag(-1, 2, -1)  (Dirichlet)
//   M[p][d][mu][nu]   = g_{mu,p}^T S g_{nu,p+d},  S = (h/6) tridiag(1, 4, 1)
// with g_mu the cell-0 samples (stored on an index range extended by (L0 - 1) n_c nodes to the
// left so that every shifted copy is a plain offset).  Substituting i' = i - p n_c:
//   C_r[p][d] = sum_i' P_d(i') v_r(i' + p n_c),  P_d(i') = g_mu(i') g_nu(i' - d n_c),
// for i' + p n_c on the grid: one product row per (mu, nu, d), contracted with the potential
// rows at every cell offset p -- a GEMM-shaped sum with a Toeplitz right operand.  Directions 1
// and 2 (single open cells) use the ordinary per-direction factors.
//
// The dense matrices (eq. (3.10)) are then, for row (p, mu) and column (p + d, nu):
//   S = M0 M1 M2,  H = (K0 M1 M2 + M0 K1 M2 + M0 M1 K2) / 2 - sum_r c_r C0_r C1_r C2_r,
// and exact zeros outside the window.
#include "lhf_internal.cuh"

namespace lhf {
namespace {

constexpr int kBoxThreads = 256;

// One CTA per (system, dd, mu, nu): the product row P and the P1 cross terms X in shared memory,
// then every (p, slot) output of the row.  Deterministic (fixed-order sums).
__global__ void __launch_bounds__(kBoxThreads) k_box_gram(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  if (!s.box) return;
  const int m0 = s.m0, mm = m0 * m0;
  const int b = blockIdx.x;
  if (b >= s.bJ * mm) return;
  const int dd = b / mm, e = b - dd * mm, mu = e / m0, nu = e - mu * m0;
  const int d = s.bjlo + dd;
  const DirDev &D = s.d[0];
  const int n = D.n, nc = D.nc, gx = D.gext, nx = n + gx, L0 = D.L;
  const int Rt = s.Rt, slots = Rt + 2;
  const double *G = s.ws + D.offG;
  const double *f = G + (int64_t)mu * nx;  // f(i') = f[i' + gx]
  const double *g = G + (int64_t)nu * nx;
  // supports in i' coordinates (widened node ranges of the cell-0 copies)
  const int fa = s.node_lo[0][mu] - gx, fb = fa + s.node_span[0][mu];
  const int ga = s.node_lo[0][nu] - gx + d * nc, gb = ga + s.node_span[0][nu];
  const int ia = max(fa, ga), ib = min(fb, gb);
  const int W = ib - ia;  // may be <= 0: every output is zero
  extern __shared__ double sm[];
  double *P = sm;       // [W]
  double *X = sm + (W > 0 ? W : 0);  // [W]
  const int tid = threadIdx.x;
  for (int u = tid; u < W; u += kBoxThreads) {
    const int ip = ia + u;
    const int ef = ip + gx, eg = ip - d * nc + gx;  // extended indices of f(i'), g(i' - d n_c)
    const double fi = (ef >= 0 && ef < nx) ? f[ef] : 0.0;
    const double gi = (eg >= 0 && eg < nx) ? g[eg] : 0.0;
    const double f1 = (ef + 1 >= 0 && ef + 1 < nx) ? f[ef + 1] : 0.0;
    const double g1 = (eg + 1 >= 0 && eg + 1 < nx) ? g[eg + 1] : 0.0;
    P[u] = fi * gi;
    X[u] = fi * g1 + f1 * gi;
  }
  __syncthreads();
  const double *V = s.ws + D.offV;  // [Rt][n]
  double *Cb = s.ws + s.offCb;
  const int outs = L0 * slots;
  const int warp = tid >> 5, lane = tid & 31;
  // one warp per output (cell p, slot), lanes over the nodes (coalesced potential rows), a fixed
  // shuffle tree for the sum
  for (int o = warp; o < outs; o += kBoxThreads / 32) {
    const int p = o / slots, slot = o - p * slots;
    if (p + d < 0 || p + d >= L0) continue;  // column cell outside the box: never read
    // grid nodes i = i' + p n_c in [0, n): i' in [-p n_c, n - p n_c)
    const int lo = max(ia, -p * nc), hi = min(ib, n - p * nc);
    double acc = 0.0;
    if (slot < Rt) {
      const double *vr = V + (int64_t)slot * n + p * nc;
      for (int ip = lo + lane; ip < hi; ip += 32) acc += P[ip - ia] * __ldg(vr + ip);
    } else {
      // P1 forms node by node: diagonal terms over i in [0, n), cross terms over i in [0, n - 1)
      // (the stiffness sum cancels to O(h^2) of its terms, so each node's 2 f g - cross is formed
      // before summing rather than two large partial sums)
      const int hx = min(ib, n - 1 - p * nc);
      const double wd = (slot == Rt) ? 2.0 : 4.0, wx = (slot == Rt) ? -1.0 : 1.0;
      for (int ip = lo + lane; ip < hi; ip += 32) acc += wd * P[ip - ia] + (ip < hx ? wx * X[ip - ia] : 0.0);
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
      if (slot == Rt) acc /= D.h;
      else if (slot == Rt + 1) acc *= D.h / 6.0;
      Cb[(((int64_t)p * s.bJ + dd) * slots + slot) * mm + e] = acc;
    }
  }
}

// Dense H, S: thread per entry (row (p, mu), column (q, nu)), row-major [N_b][N_b].
__global__ void __launch_bounds__(256) k_box_assemble(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  if (!s.box) return;
  const int m0 = s.m0, mm = m0 * m0, Rt = s.Rt, slots = Rt + 2;
  const int L0 = s.d[0].L;
  const int64_t N = (int64_t)L0 * m0;
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (item >= N * N) return;
  const int row = (int)(item / N), col = (int)(item - (int64_t)row * N);
  const int p = row / m0, mu = row - p * m0, q = col / m0, nu = col - q * m0;
  const int dd = q - p - s.bjlo;
  double h = 0.0, sv = 0.0;
  if (dd >= 0 && dd < s.bJ) {
    const int e = mu * m0 + nu;
    const double *F0 = s.ws + s.offCb + ((int64_t)p * s.bJ + dd) * slots * mm + e;
    const double *F1 = s.ws + s.d[1].offC + e;
    const double *F2 = s.ws + s.d[2].offC + e;
    double v = 0.0;
    for (int r = 0; r < Rt; ++r) {
      const int64_t o = (int64_t)r * mm;
      v += s.c[r] * F0[o] * F1[o] * F2[o];
    }
    const int64_t ok = (int64_t)Rt * mm, om = (int64_t)(Rt + 1) * mm;
    const double K0 = F0[ok], K1 = F1[ok], K2 = F2[ok];
    const double M0 = F0[om], M1 = F1[om], M2 = F2[om];
    sv = M0 * M1 * M2;
    h = 0.5 * (K0 * M1 * M2 + M0 * K1 * M2 + M0 * M1 * K2) - v;
  }
  s.H[item] = h;
  s.S[item] = sv;
}

}  // namespace

size_t box_gram_smem_bytes(int max_width) { return (size_t)2 * (max_width > 0 ? max_width : 0) * sizeof(double); }

cudaError_t launch_box_gram(const SysDev *sys, int nsys, int max_items, int max_width, cudaStream_t st) {
  if (max_items <= 0 || nsys <= 0) return cudaSuccess;
  const size_t smem = box_gram_smem_bytes(max_width);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_box_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kmark(LHF_K_BOX_GRAM, 1, st);
  k_box_gram<<<dim3(max_items, nsys), kBoxThreads, smem, st>>>(sys);
  kmark(LHF_K_BOX_GRAM, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_box_assemble(const SysDev *sys, int nsys, long long max_entries, cudaStream_t st) {
  if (max_entries <= 0 || nsys <= 0) return cudaSuccess;
  dim3 grid((unsigned)((max_entries + 255) / 256), nsys);
  kmark(LHF_K_BOX_ASSEMBLE, 1, st);
  k_box_assemble<<<grid, 256, 0, st>>>(sys);
  kmark(LHF_K_BOX_ASSEMBLE, 0, st);
  return cudaGetLastError();
}

}  // namespace lhf
