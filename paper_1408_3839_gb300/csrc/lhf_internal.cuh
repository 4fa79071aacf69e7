// lhf_internal.cuh -- device-side system descriptors and kernel entry points of liblhf.
//
// Every kernel works on a batch of systems: blockIdx.y (or the decoded work item) selects the
// system, whose descriptor SysDev lives in device memory.  One system is a batch of one.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lhf.h"

namespace lhf {

constexpr int kMaxM0 = LHF_MAX_M0;
constexpr int kMaxNuc = LHF_MAX_NUCLEI;
constexpr int kMaxR = LHF_MAX_R;
constexpr int kMaxRt = kMaxNuc * kMaxR;
constexpr int kSlices = 7;  // base-2^7 digit slices per FP64 operand on the tensor-core route
// Digit planes are stored chunk-major, [plane][K / kPlaneChunk][row][kPlaneChunk]: the tile of 128
// (or 64) rows x kPlaneChunk columns that one tensor-core load takes is one contiguous block.
constexpr int kPlaneChunk = 32;
// A Bloch function is numerically absent at a k-point when Re Sbar_ii <= kDropTol * s0_i.
constexpr double kDropTol = LHF_DROP_TOL;
// Canonical orthogonalisation drops directions of the scaled overlap below kLindepTol.  The
// Cholesky route is taken only when every scaled pivot is at least kCholTol: the smallest
// overlap eigenvalue never exceeds the smallest pivot, and with no eigenvalue below kLindepTol
// both routes solve the same pencil.
constexpr double kLindepTol = LHF_LINDEP_TOL;
constexpr double kCholTol = 1e-5;

// One direction of one system.
struct DirDev {
  int L;          // cells
  int n;          // grid nodes
  int nc;         // nodes per lattice cell (n for a single-cell open direction)
  int nv;         // potential factor length: nc (periodic, replicated per cell) or n
  int periodic;   // block-circulant direction
  int lattice;    // L > 1 or periodic: basis copies shifted by k b
  int K;          // periodic image window
  int J;          // window blocks computed (<= L)
  int jlo;        // first displacement of the window (may be negative; blocks taken mod L)
  int gext;       // basis samples start gext nodes left of the grid (open box direction 0)
  double h, x0, cell0, b;
  double invP;     // 1 / (L b): supercell period of a periodic direction
  int64_t offG;   // basis samples [m0][gext + n]   (doubles, from SysDev::ws)
  int64_t offD;   // forward differences g_i - g_(i+1) [m0][n] (periodic wrap; open: g_n = 0), or -1
  int64_t offV;   // potential factors [Rt][nv]
  int64_t offC;   // Gram factors [J][Rt+2][m0][m0]
  // C[j][mu][nu] = C[-j][nu][mu] (Q_j and its mirror are the same sums): only the window blocks
  // jw = cw0 .. cw0 + Jc - 1 (displacements j >= 0) are contracted, the others are mirrored
  int cw0, Jc;
  // tensor-core route (LHF_MIXED): digit planes and scale exponents
  int Kpad;       // nv rounded up to a multiple of 64
  int pad2_;
  float p1h[6];   // 1 / h, h, h / 6 as FP32 pairs (hi, lo): the P1 factors of the mixed route
  int64_t offGD;  // float4 [m0][n] {sample, difference} as FP32 pairs h + l (written with offG and
                  // offD on the mixed route), or -1
  int64_t offA;   // BF16 [kSlices][Kpad / 32][Jc m0 m0][32] digit planes of the folded products
  int64_t offB;   // BF16 [kSlices][Kpad / 32][Rt][32] digit planes of the potential factors
  int64_t offRE;  // int [Jc m0 m0] row scale exponents
  int64_t offRM;  // int [2][Jc m0 m0] rows with overlap: full -> compact index (-1: none), compact -> full
  int rows_c;     // rows (window block, mu, nu) whose functions overlap: the tensor-core route's rows
  int pad3_;
  int64_t offCE;  // int [Rt] potential-row scale exponents
  int64_t offF;   // k-space route: complex [L][Rt+2][m0][m0] 1D DFTs of the factors (0 when unused)
};

struct SysDev {
  DirDev d[3];
  int m0, M0, R, Rt;
  int nblocks;     // L0 L1 L2
  int nwin;        // J0 J1 J2
  int box;         // open lattice direction 0 (dense matrices)
  int nkhalf;      // k-points solved (the rest are complex conjugates)
  int kind[kMaxM0];
  double alpha[kMaxM0];
  double centre[kMaxM0][3];
  double cut[kMaxM0];     // truncation radius sqrt(rho / alpha)
  double pnorm[kMaxM0];   // sqrt(2 alpha e)
  int cell_lo[3][kMaxM0]; // support cells of the cell-0 copy (unwrapped, dilated by one node)
  int cell_hi[3][kMaxM0];
  int node_lo[3][kMaxM0];   // grid nodes that may be inside the cut of the cell-0 copy: from
  int node_span[3][kMaxM0]; // node_lo, node_span nodes (mod n in periodic directions; widened)
  int node_wrap[3][kMaxM0]; // periodic, node_span < n: the unwrapped first node is node_lo + node_wrap n
  double Z[kMaxNuc];
  double a[kMaxNuc][3];
  double t[kMaxR];        // sinc nodes
  double c[kMaxRt];       // rank coefficients Z_nu w_q, r = nu R + q
  double *ws;             // workspace of this system
  double *H, *S;          // first block column [L0][L1][L2][m0][m0] (or dense [Nb][Nb])
  double *Hbar, *Sbar;    // complex [L0][L1][L2][m0][m0][2]
  double *eig;            // [nblocks][m0]
  int *kstat;             // [nblocks] or null
  double *s0;             // [m0] mean over k-points of Re Sbar_ii (cell-periodic norms)
  const int *klist;       // [nkhalf] k-points solved (one per conjugate pair), or null
  double *tri;            // [nkhalf][2 m0 + 1] tridiagonal of each solved k-point, or null (Jacobi)
  double *evs;            // complex [nblocks][m0][m0] scratch of the k-point solves, or null
  double *vecs;           // complex [nblocks][m0][m0] Bloch eigenvectors (rows), or null
  double *dftw;           // complex [2][L0][m0][m0] scratch of the four-step DFT (L0 > kDftTileMax), or null
  // rank reduction of the direction-0 potential factors (one-dimensional lattices, FP64 route):
  // singular values below rank_eps of the largest dropped (0: off); scratch at ws + offRR
  double rank_eps;
  int64_t offRR;
  // k-point reduction (Cholesky route, then Householder) in compensated FP32 pairs instead of
  // FP64: set for the mixed route (LHF_MIXED), whose eigenvalue target is 1e-6 Ha
  int eig_df;
  // open box (direction 0 an open lattice): factors between cells p and p + d, d = bjlo ..
  // bjlo + bJ - 1, at ws + offCb, layout [L0][bJ][Rt+2][m0][m0]
  int bJ, bjlo;
  int64_t offCb;
  int64_t offPC;          // potential row constants [3][R][kPotConst] (k_pot_rows, read by k_potential)
  const double *zcell;    // box charges [L0][M0] (device) or null
};

// Cells p where the copy of mu shifted by the window displacement j and nu overlap (the runs of
// the Gram's fold): [plo, phi] (nu's support, at most L cells) against the images of [mlo, mhi]
// modulo L; a single open cell overlaps itself.  The same integers on host and device.
__host__ __device__ inline int gram_row_cells(const SysDev &s, int l, int j, int mu, int nu) {
  const DirDev &D = s.d[l];
  if (!D.periodic) return 1;
  const int L = D.L;
  const int mlo = s.cell_lo[l][mu] + j, mhi = s.cell_hi[l][mu] + j;
  const int plo = s.cell_lo[l][nu];
  int phi = s.cell_hi[l][nu];
  if (phi > plo + L - 1) phi = plo + L - 1;
  if (mhi - mlo >= L - 1) return phi - plo + 1;
  const int a = plo - mhi + L - 1;
  const int k0 = a >= 0 ? a / L : -((-a + L - 1) / L);
  int cells = 0;
  for (int k = k0; k <= k0 + 1; ++k) {
    const int lo = plo > mlo + k * L ? plo : mlo + k * L;
    const int hi = phi < mhi + k * L ? phi : mhi + k * L;
    if (hi >= lo) cells += hi - lo + 1;
  }
  return cells;
}

// 2^e as a double from its exponent field (normal range), else by ldexp.
__device__ __forceinline__ double pow2(int e) {
  if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(1.0, e);
}

// 2^e for |e| <= 2046 as a double (0 or inf beyond the representable range).
__device__ __forceinline__ double pow2_scale(int e) { return ldexp(1.0, e); }

// x 2^e, exact whenever the result is a normal number (two power-of-two factors when 2^e itself
// is out of range).
__device__ __forceinline__ double scale_pow2(double x, int e) {
  if (e >= -1022 && e <= 1023) return x * pow2(e);
  const int h = e / 2;
  return (x * pow2(h)) * pow2(e - h);
}

// Window block jw of direction D, entry (mu, nu): pointer to slot 0 of that entry (slots are m0^2
// doubles apart).  Blocks outside the contracted half of the window are read from their
// mirrors, C_r[-j][mu][nu] = C_r[j][nu][mu] (the transposed entry of the mirrored block).
__device__ __forceinline__ const double *factor_entry(const SysDev &s, const DirDev &D, int jw, int mu, int nu) {
  const int m0 = s.m0, mm = m0 * m0, slots = s.Rt + 2;
  if (jw >= D.cw0 && jw < D.cw0 + D.Jc) return s.ws + D.offC + (int64_t)jw * slots * mm + mu * m0 + nu;
  int jm;  // mirror: j -> -j (mod L when the window is the whole lattice)
  if (D.J == D.L && D.jlo == 0)
    jm = jw == 0 ? 0 : D.L - jw;
  else
    jm = -2 * D.jlo - jw;
  return s.ws + D.offC + (int64_t)jm * slots * mm + nu * m0 + mu;
}

// Per-launch status word written by kernels (atomicOr of flag bits).
enum : unsigned { kFlagNotSpd = 1u, kFlagBadArg = 2u, kFlagTimeout = 4u };

// Samples written by k_basis for row (l, mu): in a periodic lattice direction the nodes of the
// support cells of the cell-0 copy (at most the whole row), elsewhere the whole (extended) row.
// The host sizes the basis launch with the same count.
constexpr int kBasisChunk = 512;  // samples per k_basis CTA
__host__ __device__ inline int basis_row_samples(const SysDev &s, int l, int mu) {
  const DirDev &D = s.d[l];
  const int nx = D.n + D.gext;
  if (!D.periodic) return nx;
  const int span = s.cell_hi[l][mu] - s.cell_lo[l][mu] + 1;
  const int cells = span < D.L ? span : D.L;
  return D.n < cells * D.nc ? D.n : cells * D.nc;
}
__host__ __device__ inline int basis_ctas(const SysDev &s) {
  int n = 0;
  for (int r = 0; r < 3 * s.m0; ++r) n += (basis_row_samples(s, r / s.m0, r % s.m0) + kBasisChunk - 1) / kBasisChunk;
  return n;
}

// Potential rows: one CTA per (direction, rank term, chunk of kPotChunk cells); the host sizes
// the launch with potential_ctas.
constexpr int kPotChunk = 512;
// Per (direction, sinc node) constants of a potential row: degree J of the cell series, its
// coefficients, the Euler-Maclaurin polynomial, the Poisson weights, the row's scalars and flags.
constexpr int kPotConst = 54;
__host__ __device__ inline int potential_ctas(const SysDev &s) {
  int n = 0;
  for (int l = 0; l < 3; ++l) n += s.Rt * ((s.d[l].nv + kPotChunk - 1) / kPotChunk);
  return n;
}

// Per-kernel timing hook: while a context with profiling enabled is launching, kclock.mark is
// set and every launcher brackets each of its kernel launches with kmark(kernel, 1 / 0, st)
// (kernel = LHF_K_*).  Unset (the default) the calls do nothing.
struct KernelClock {
  void *owner;
  void (*mark)(void *owner, int kernel, int begin, cudaStream_t st);
};
extern thread_local KernelClock kclock;
inline void kmark(int kernel, int begin, cudaStream_t st) {
  if (kclock.mark) kclock.mark(kclock.owner, kernel, begin, st);
}

// ---- kernel launchers (each returns the launch error) ------------------------------------
// One CTA per (direction, function, chunk of kBasisChunk samples): max_rows = basis_ctas over the
// batch.  Periodic lattice directions write only the support-cell window of each row (see
// k_basis).
cudaError_t launch_basis(const SysDev *sys, int nsys, int max_rows, cudaStream_t st);
// One CTA per (direction, rank term, chunk of kPotChunk cells): max_rows = potential_ctas over
// the batch.
cudaError_t launch_potential(const SysDev *sys, int nsys, int max_rows, cudaStream_t st);
// Weighted Grams (FP64 route) and the folded products' digit planes (tensor-core route): one CTA
// per (direction, contracted window block, mu); ldir >= 0 restricts a launch to direction ldir
// (max_blocks, max_nv then over that direction: the shared memory fits its rows), -1 takes all.
cudaError_t launch_gram_fp64(const SysDev *sys, int nsys, int max_blocks, int max_m0,
                             int max_nv, cudaStream_t st, int ldir = -1);
// With rowmap, the launch first maps the rows with overlap of every direction (k_gram_rowmap: the
// tensor-core route contracts only those); the first slicing launch of a step takes it.
cudaError_t launch_gram_slices(const SysDev *sys, int nsys, int max_blocks, int max_m0, int max_nv, cudaStream_t st,
                               int ldir, bool rowmap);
// Digit planes of the potential factors: one CTA per (direction, rank term), max_rt3 = 3 R_tot.
cudaError_t launch_vslices(const SysDev *sys, int nsys, int max_rt3, cudaStream_t st);
// Rank reduction (k_rank.cu), one CTA per system with rank_eps > 0, after the transverse Grams
// and before the direction-0 Gram: rewrites the direction-0 potential rows, the transverse
// factors, the rank coefficients and Rt of the device descriptor.  Its scratch header holds
// [R_tot, r1, rho (largest residual row norm left out), the first pivot's norm].
// R_tot <= kRankReduceMaxRt.
constexpr int kRankReduceMaxRt = 64;
size_t rank_reduce_smem_bytes(int R, int nv);
cudaError_t launch_rank_reduce(SysDev *sys, int nsys, size_t smem, cudaStream_t st);
// The window blocks outside cw0 .. cw0 + Jc - 1 from their mirrors (thread per element).
cudaError_t launch_gram_mirror(const SysDev *sys, int nsys, long long max_items, cudaStream_t st);
// Tensor-core contraction of the digit planes (tcgen05), one job per (system, direction, 128-row
// tile, 64-column tile).  host_sys: host copies of the descriptors (device workspace pointers).
// dev_buf (dev_bytes >= gram_tc_args_bytes) receives the tensor maps and the job list through the
// pinned host_buf, which must stay untouched until the copy has executed.  Returns
// cudaErrorNotSupported for shapes outside the kernel's limits (K padded above 448).
size_t gram_tc_args_bytes(const SysDev *host_sys, int nsys);
cudaError_t launch_gram_tc_impl(const SysDev *host_sys, int nsys, void *dev_buf, size_t dev_bytes,
                                void *host_buf, size_t host_bytes, unsigned *flags, cudaStream_t st);
// The same in two parts: tensor maps and jobs into host_buf (nothing launched; *jobs_off is the
// byte offset of the job list), then the launch on a device copy of that buffer.
cudaError_t gram_tc_prepare(const SysDev *host_sys, int nsys, void *host_buf, size_t host_bytes, int *njobs,
                            size_t *jobs_off);
cudaError_t gram_tc_launch(const void *dev_buf, int njobs, size_t jobs_off, unsigned *flags, cudaStream_t st);
// Rank sum over the window blocks (max_compute_ctas = ranksum_ctas over the batch) and zeros for
// the blocks outside it (max_blocks = nblocks over the batch); max_rt: the largest R_tot of the
// batch (shared memory of the rank weights).  Reads mirrored window blocks from their contracted
// partners (no mirror pass needed).
int ranksum_ctas(const SysDev &s);
cudaError_t launch_ranksum(const SysDev *sys, int nsys, int max_compute_ctas, int max_blocks, int max_rt,
                           cudaStream_t st);
// A lattice dimension of at most kDftTileMax positions is transformed in one shared-memory tile
// per pass; a one-dimensional lattice of up to kDftMaxL1 cells with L0 > kDftTileMax takes the
// four-step route (L0 = A B, A, B <= kDftTileMax) through the scratch SysDev::dftw.
constexpr int kDftTileMax = 4096;
constexpr int kDftMaxL1 = 32768;
bool dft_four_step_split(int L, int *A, int *B);  // a split with A, B <= kDftTileMax, A >= B
cudaError_t launch_dft(const SysDev *sys, int nsys, const int *host_L, int *passes,
                       cudaStream_t st);  // *passes += kernel launches (may be null)
// k-point eigensolves; tri: systems carry a tridiagonal scratch (SysDev::tri), and the
// tridiagonal eigenvalues are taken by a second kernel (else Jacobi inside k_eig).
// eig_warps: k-points (warps) per CTA of k_eig, 1 .. 8; tri_threads: threads per CTA of the
// tridiagonal kernel (a multiple of its 16 or 32 lanes per matrix, at most 256).  The two
// kernels alone (launch_eig_reduce, launch_tridiag) serve the launch-shape autotuner.
// full: a whole warp per matrix even up to order 16 (the mixed route's pair arithmetic).
// vglob: every system carries the per-k-point scratch SysDev::evs, which then holds each
// solve's third matrix instead of shared memory (more resident solves per SM).
cudaError_t launch_eig(const SysDev *sys, int nsys, int max_k, int max_m0, unsigned *flags,
                       unsigned long long *counters, cudaStream_t st, bool tri, int eig_warps = 4,
                       int tri_threads = 128, bool full = false, bool vglob = false);
cudaError_t launch_eig_reduce(const SysDev *sys, int nsys, int max_k, int max_m0, unsigned *flags,
                              unsigned long long *counters, cudaStream_t st, int warps, bool full = false,
                              bool vglob = false);
// most k_eig warps per CTA whose shared memory fits an SM
int eig_max_warps(int max_m0, bool full = false, bool vglob = false);
cudaError_t launch_tridiag(const SysDev *sys, int nsys, int max_k, int max_m0, unsigned *flags,
                           unsigned long long *counters, cudaStream_t st, int threads);
cudaError_t launch_overlap_norms(const SysDev *sys, int nsys, cudaStream_t st);
// Separable k-space route (Theorem 2.5): 1D DFTs of the factors (max_factor_ctas =
// kspace_factor_ctas over the batch) into D.offF, then Hbar / Sbar of every solved k-point and its
// conjugate (max_items = nkhalf m0^2 over the batch).  The factors' mirrored blocks are read
// from their partners.
int kspace_factor_ctas(const SysDev &s);
cudaError_t launch_kspace(const SysDev *sys, int nsys, int max_factor_ctas, long long max_items, cudaStream_t st);
// Bloch orbitals on a window of the grid: kappa, lo, cnt host [3]; coef device complex
// [norb][m0]; B device scratch of 6 m0 max(cnt) doubles; out device complex [norb][cnt0][cnt1]
// [cnt2].  The basis samples of the (single) system must be in its workspace, zero outside the
// support windows.  maxL: the largest L_l.
cudaError_t launch_orbitals(const SysDev *sys, const int *kappa, const int *lo, const int *cnt, int norb,
                            const double *coef, double *B, double *out, int m0, int maxL, cudaStream_t st);
// One spectrum of lhf_cell_energies: values eig[off .. off + cnt), the n_low smallest selected,
// their sum divided by cells.
struct SpectrumSeg {
  long long off;
  int cnt;
  int n_low;
  double cells;
};
// One CTA per spectrum: energy[s] = (sum of the n_low smallest) / cells, level[s] (may be null) =
// the n_low-th smallest value.  seg: device array [nseg].
cudaError_t launch_cell_energy(const double *eig, const SpectrumSeg *seg, int nseg, double *energy, double *level,
                               cudaStream_t st);
// Lattice-sum extrapolation: eig [nK][n] (device), K device [nK] (2 <= nK <= 8); A, B [n] (B may be null).
constexpr int kMaxExtrapolationWindows = 8;
cudaError_t launch_lattice_extrapolate(const double *eig, const double *K, int nK, long long n, double *A, double *B,
                                       cudaStream_t st);
// Open box: direction-0 factors (one CTA per (d, mu, nu), max_width = widest product row) and
// the dense matrices (thread per entry).
size_t box_gram_smem_bytes(int max_width);
cudaError_t launch_box_gram(const SysDev *sys, int nsys, int max_items, int max_width, cudaStream_t st);
cudaError_t launch_box_assemble(const SysDev *sys, int nsys, long long max_entries, cudaStream_t st);
// Dense generalized symmetric-definite eigenvalues (cooperative launch, one CTA per SM).
// work: dense_eig_workspace_doubles(N) doubles.  cudaErrorNotSupported without cooperative launch.
// wait_cycles: bound of each grid-barrier wait (<= 0: kDefaultWaitCycles); stall: the barriers
// expect one CTA more than launched, so that every wait runs out (failure-detection test).
constexpr long long kDefaultWaitCycles = 2000000000ll;  // about a second at 2 GHz
cudaError_t launch_dense_eig(const double *H, const double *S, int N, double *eig,
                             double *work, unsigned *flags, cudaStream_t st,
                             long long wait_cycles = kDefaultWaitCycles, int stall = 0);
size_t dense_eig_workspace_doubles(int N);
// Iterative solver of large open boxes (k_lobpcg.cu): band H, S [L][bJ][m0][m0] from the box
// factors (one system at sys[0]); banded products of kv vectors ([kv][N], N = L m0); the
// block-circulant preconditioner of M cells (power of two >= L + bJ): the band averaged over the
// rows [bJ][m0][m0] and its kappa blocks, their Cholesky factors at a shift (bad |= 1 when one is not positive definite), and
// its application Y = T X (Vk: kv M m0 complex scratch); Gram matrices G = Z^T Y of nz vectors;
// out = sum_{j0 <= j < j1} C[j][c] Z[j] for c < kv; residuals R = YH - theta YS and their norms;
// seeded start vectors; the Rayleigh-Ritz step on a pencil of order n <= rayleigh_ritz_max().
cudaError_t launch_box_band(const SysDev *sys, long long items, double *Hband, double *Sband, cudaStream_t st);
cudaError_t launch_band_mv(const double *Hb, const double *Sb, const double *X, double *YH, double *YS, int L,
                           int bJ, int bjlo, int m0, int kv, cudaStream_t st);
cudaError_t launch_band_average(const double *Hb, const double *Sb, int L, int bJ, int bjlo, int m0, double *Ha,
                                double *Sa, cudaStream_t st);
cudaError_t launch_prec_blocks(const double *Hb, const double *Sb, int mid, int bJ, int bjlo, int m0, int M,
                               double2 *Hk, double2 *Sk, cudaStream_t st);
cudaError_t launch_prec_factor(const double2 *Hk, const double2 *Sk, double sigma, int m0, int M, double2 *Lk,
                               unsigned *bad, cudaStream_t st);
cudaError_t launch_prec_apply(const double2 *Lk, const double *X, double *Y, double2 *Vk, int L, int m0, int M,
                              int kv, cudaStream_t st);
// Block-tridiagonal Cholesky of H - sigma S (super-cells of g cells, B = g m0, nb = ceil(L / g)
// blocks; D, E: nb B^2 doubles each; bad |= 1 when not positive definite) and its solve of kv
// right-hand sides in place in Y [kv][N] (scratch V: kv nb B doubles).
cudaError_t launch_tri_factor(const double *Hb, const double *Sb, double sigma, int L, int bJ, int bjlo, int m0,
                              int g, int nb, double *D, double *E, unsigned *bad, cudaStream_t st);
cudaError_t launch_tri_solve(const double *D, const double *E, int B, int nb, long long N, int kv, double *Y,
                             double *V, cudaStream_t st);
cudaError_t launch_gram_vec(const double *Z, const double *Y, int nz, long long N, double *G, cudaStream_t st);
cudaError_t launch_lincomb(const double *Z, const double *C, int ldc, int j0, int j1, int kv, long long N,
                           double *out, cudaStream_t st);
cudaError_t launch_residual(const double *YH, const double *YS, const double *theta, int kv, long long N,
                            double *R, double *rnorm, cudaStream_t st);
cudaError_t launch_start_vectors(double *X, int kv, long long N, unsigned long long seed, cudaStream_t st);
int rayleigh_ritz_max();
cudaError_t launch_rayleigh_ritz(const double *A, const double *B, int n, int kv, double cut, double *theta,
                                 double *C, int *info, cudaStream_t st);

}  // namespace lhf
