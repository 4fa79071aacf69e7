// k_gram.cu -- steps a3 + a4 in FP64: per-direction weighted 1D Grams and P1 forms.
//
// For direction l, window block j (displacement), row function mu and column function nu
// (eq. (3.10) and the proof of Lemma 3.1; Sec. 3.4 for the P1 matrices):
//   C_r[j][mu][nu] = sum_i g_{mu,j}(i) v_r(i) g_{nu,0}(i)            r < R_tot
//   K[j][mu][nu]   = g_{mu,j}^T A g_{nu,0},  A = (1/h) tridiag(-1, 2, -1)
//   M[j][mu][nu]   = g_{mu,j}^T S g_{nu,0},  S = (h/6) tridiag(1, 4, 1)
// with g_{mu,j}(i) = g_mu(i - j n_c) (the copy in cell j).  In a periodic direction v_r has the
// period n_c of one cell (the potential is replicated from cell 0, eq. (4.1)), so the sum over
// the grid folds onto the n_c nodes of one cell:
//   C_r[j][mu][nu] = sum_c v_r(c) Q_j[mu][nu](c),  Q_j[mu][nu](c) = sum_p g_{mu,j}(c + p n_c) g_nu(c + p n_c)
// -- the same sum regrouped, exact up to rounding.  The second step is a dense contraction over
// c of the R_tot potential rows with the m0^2 folded products (a GEMM with K = n_c).
//
// Substituting p -> p + j shows Q_{-j}[nu][mu](c) = Q_j[mu][nu](c), hence C_r[-j][nu][mu] =
// C_r[j][mu][nu] and the same for the P1 forms (A and S are symmetric circulants): only the
// blocks with j >= 0 (window indices cw0 .. cw0 + Jc - 1) are contracted; k_gram_mirror copies
// the others from their mirrors.
//
// One CTA per (system, direction, window block, mu): phase 1 forms Q[nu][c] for all nu in
// shared memory (only the cells where both supports can be nonzero are visited) together with
// the P1 sums; phase 2 contracts with the R_tot potential rows.  Deterministic (fixed-order
// reductions, no atomics).
#include "lhf_internal.cuh"

namespace lhf {
namespace {

constexpr int kGramThreads = 256;

struct GramItem {
  int l, jw, mu;
};

// CTA b of a system -> (direction, window block, mu) over the contracted blocks jw = cw0 ..
// cw0 + Jc - 1 of each direction (of direction ldir alone when ldir >= 0).
__device__ __forceinline__ bool decode_gram(const SysDev &s, int b, GramItem &it, int ldir) {
  for (int l = ldir < 0 ? 0 : ldir; l < (ldir < 0 ? 3 : ldir + 1); ++l) {
    const int cnt = s.d[l].Jc * s.m0;
    if (b < cnt) {
      it.l = l;
      const int jc = b / s.m0;
      it.jw = s.d[l].cw0 + jc;
      it.mu = b - jc * s.m0;
      return true;
    }
    b -= cnt;
  }
  return false;
}

// floor(a / b) for b > 0
__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Phase 1 for one CTA: Q[nu][c] and the difference products E[nu][c] = sum_p D_i(g_mu,j) D_i(g_nu)
// in shared memory, their row sums in red[2 nu], and the P1 stiffness/mass slots of C written
// out.  With D_i(f) = f_i - f_(i+1) (periodic wrap; open: f_(-1) = f_n = 0),
//   g^T A f = (1/h) sum_i D_i(f) D_i(g),   g^T S f = h sum_i f_i g_i - (h/6) sum_i D_i(f) D_i(g),
// the same sums as (1/h) sum (2 f_i g_i - f_i g_(i+1) - f_(i+1) g_i) and (h/6) sum (4 f_i g_i +
// cross terms) regrouped: no cancellation in the stiffness sum and two products per node.
__device__ void gram_phase1(const SysDev &s, const GramItem &it, double *Q, double *E, double *red) {
  const DirDev &D = s.d[it.l];
  const int m0 = s.m0, nv = D.nv, n = D.n, nc = D.nc, L = D.L;
  const int ld = nv + 1;
  const double *G = s.ws + D.offG;
  const double *Dg = s.ws + D.offD;
  const int mu = it.mu;
  const int j = D.jlo + it.jw;
  const double *f = G + (int64_t)mu * n;
  const double *df = Dg + (int64_t)mu * n;
  const int tid = threadIdx.x;
  // support of the shifted row function (cells), tested modulo L
  const int mlo = s.cell_lo[it.l][mu] + j, mhi = s.cell_hi[it.l][mu] + j;
  const int mspan = mhi - mlo;
  const bool periodic = D.periodic != 0;
  // per column function nu: the cells p of g_nu's support where the shifted row function is
  // present, as up to two runs of consecutive cells -- [plo, phi] meets the row support
  // [mlo, mhi] modulo L; unless the row support covers every residue its images [mlo + kL,
  // mhi + kL] are disjoint, and [plo, phi] (at most L cells) meets at most two of them, k0 (the
  // first that ends at or after plo) and k0 + 1 -- each run given by its length and the nodes of
  // its first cell (for c = 0) in g_nu and in the shifted row function; formed once per CTA
  __shared__ int seg[kMaxM0][2][3];  // [nu][run]: cells, first node of g_nu, first node of the row
  if (periodic && tid < m0) {
    const int nu = tid;
    const int plo = s.cell_lo[it.l][nu];
    int phi = s.cell_hi[it.l][nu];
    if (phi > plo + L - 1) phi = plo + L - 1;
    int seg_lo[2] = {plo, 1}, seg_hi[2] = {phi, 0};
    if (mspan < L - 1) {
      const int k0 = floor_div(plo - mhi + L - 1, L);
      seg_lo[0] = max(plo, mlo + k0 * L);
      seg_hi[0] = min(phi, mhi + k0 * L);
      seg_lo[1] = max(plo, mlo + (k0 + 1) * L);
      seg_hi[1] = min(phi, mhi + (k0 + 1) * L);
    }
    for (int sg = 0; sg < 2; ++sg) {
      seg[nu][sg][0] = seg_hi[sg] >= seg_lo[sg] ? seg_hi[sg] - seg_lo[sg] + 1 : 0;
      seg[nu][sg][1] = wrap(seg_lo[sg], L) * nc;      // node of g_nu in the run's first cell
      seg[nu][sg][2] = wrap(seg_lo[sg] - j, L) * nc;  // node of the row function shifted by j
    }
  }
  __syncthreads();
  const int items = m0 * nv;
  for (int p0 = tid; p0 < items; p0 += kGramThreads) {
    const int nu = p0 / nv;
    const int c = p0 - nu * nv;
    const double *g = G + (int64_t)nu * n;
    const double *dg = Dg + (int64_t)nu * n;
    double q = 0.0, e = 0.0;
    if (periodic) {
      // visited in increasing p; the indices advance by one cell per p (no division in the loop)
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        const int cnt = seg[nu][sg][0];
        int iv = seg[nu][sg][1] + c;
        int iu = seg[nu][sg][2] + c;
        for (int t = 0; t < cnt; ++t) {
          q += f[iu] * g[iv];
          e += df[iu] * dg[iv];
          iv += nc;
          if (iv >= n) iv -= n;
          iu += nc;
          if (iu >= n) iu -= n;
        }
      }
    } else {
      // single open cell: nodes c = 0..n-1, Dirichlet ends (the virtual node -1 adds f_0 g_0)
      q = f[c] * g[c];
      e = df[c] * dg[c];
      if (c == 0) e += f[0] * g[0];
    }
    Q[nu * ld + c] = q;
    E[nu * ld + c] = e;
  }
  __syncthreads();
  // P1 sums per nu: red[2 nu] = sum_c Q[nu][c], red[2 nu + 1] = sum_c E[nu][c], each by a group
  // of 8 lanes (strided partial sums, then a fixed 3-level shuffle tree)
  {
    const int sub = tid & 7, lane = tid & 31;
    const unsigned gmask = 0xffu << (lane & 24);
    for (int sidx = tid >> 3; sidx < 2 * m0; sidx += kGramThreads / 8) {
      const double *row = ((sidx & 1) ? E : Q) + (sidx >> 1) * ld;
      double acc = 0.0;
      for (int c = sub; c < nv; c += 8) acc += row[c];
      acc += __shfl_xor_sync(gmask, acc, 4);
      acc += __shfl_xor_sync(gmask, acc, 2);
      acc += __shfl_xor_sync(gmask, acc, 1);
      if (sub == 0) red[sidx] = acc;
    }
  }
  __syncthreads();
  const int Rt = s.Rt, mm = m0 * m0;
  double *Cout = s.ws + D.offC + (int64_t)it.jw * (Rt + 2) * mm + mu * m0;
  if (tid < m0) {
    const double dq = red[2 * tid], de = red[2 * tid + 1];
    Cout[(int64_t)Rt * mm + tid] = de / D.h;
    Cout[(int64_t)(Rt + 1) * mm + tid] = D.h * dq - de * D.h / 6.0;
  }
}

__global__ void __launch_bounds__(kGramThreads) k_gram_fp64(const SysDev *__restrict__ sysv, int ldir) {
  const SysDev &s = sysv[blockIdx.y];
  GramItem it;  // open boxes: directions 1, 2 only (direction 0 has no window here)
  if (!decode_gram(s, blockIdx.x, it, ldir)) return;
  const DirDev &D = s.d[it.l];
  const int m0 = s.m0, nv = D.nv;
  const int ld = nv + 1;  // padded row stride of Q (bank-conflict-free column reads)
  extern __shared__ double sm[];
  double *Q = sm;               // [m0][ld]
  double *E = Q + m0 * ld;      // [m0][ld]  difference products per node (P1 forms)
  double *red = E + m0 * ld;    // [m0][2]   Dsum, Esum per nu
  gram_phase1(s, it, Q, E, red);

  // ---- phase 2: C_r[nu] = sum_c V[r][c] Q[nu][c] ------------------------------------------
  const int Rt = s.Rt;
  const int mm = m0 * m0;
  const int mu = it.mu;
  double *Cout = s.ws + D.offC + (int64_t)it.jw * (Rt + 2) * mm + mu * m0;
  const double *V = s.ws + D.offV;
  const int outs = Rt * m0;
  for (int o = threadIdx.x; o < outs; o += kGramThreads) {
    const int r = o / m0;
    const int nu = o - r * m0;
    const double *vr = V + (int64_t)r * nv;
    const double *qn = Q + nu * ld;
    double acc0 = 0.0, acc1 = 0.0;
    int c = 0;
    for (; c + 1 < nv; c += 2) {
      acc0 += __ldg(vr + c) * qn[c];
      acc1 += __ldg(vr + c + 1) * qn[c + 1];
    }
    if (c < nv) acc0 += __ldg(vr + c) * qn[c];
    Cout[(int64_t)r * mm + nu] = acc0 + acc1;
  }
}

// ---- tensor-core route: exact digit slices of the FP64 operands -------------------------
//
// A row x[c] (c < nv) with max|x| = f 2^e, 1/2 <= f < 1, becomes the 62-bit fixed-point integers
// X[c] = rint(x[c] 2^(62-e)) and then 7 balanced base-2^7 digits
//   X = a_0 2^55 + a_1 2^48 + ... + a_6 2^13 + r,  a_0 in [-128, 128], a_k in [-64, 64], |r| <= 2^12,
// so x[c] = 2^e (sum_k a_k 2^(-7(k+1)) + O(2^-50)).  Every digit is an integer of at most 8
// significant bits, exact in BF16; products of two digits are exact in FP32 and sums of up to
// 2^24 / 2^14 of them accumulate exactly.  Digit plane k of a row block goes to
// planes + k * rows * Kpad + row * Kpad + c (BF16, Kpad >= nv, zero padded).
//
// X is formed from the bit fields of x with integer arithmetic only (the FP64 pipe of this GPU
// runs at a small fraction of the integer rate): |x| = M 2^(ex - 1075) with M the 53-bit
// significand, so X = M 2^(ex - 1013 - e), a left shift by at most 9 bits (|x| < 2^e) or a right
// shift rounded to nearest, ties to even.
__device__ __forceinline__ long long fixed62(double x, int e) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int bex = (int)((u >> 52) & 0x7ff);
  const unsigned long long M = (u & ((1ull << 52) - 1)) | (bex ? (1ull << 52) : 0ull);
  const int sh = (bex ? bex : 1) - 1013 - e;
  unsigned long long X;
  if (sh >= 0) {
    X = M << sh;
  } else if (sh > -64) {
    const int r = -sh;
    X = M >> r;
    const unsigned long long rem = M & ((1ull << r) - 1), half = 1ull << (r - 1);
    if (rem > half || (rem == half && (X & 1ull))) ++X;
  } else {
    X = 0;
  }
  return (u >> 63) ? -(long long)X : (long long)X;
}

__device__ __forceinline__ void digits7(double x, int e, int *a) {
  long long X = fixed62(x, e);  // |X| <= 2^62
#pragma unroll
  for (int k = 0; k < kSlices; ++k) {
    const int sh = 55 - 7 * k;
    const long long d = (X + (1ll << (sh - 1))) >> sh;
    X -= d << sh;
    a[k] = (int)d;
  }
}

__device__ __forceinline__ unsigned short bf16_of_int(int v) {  // exact for |v| <= 256
  return (unsigned short)(__float_as_uint((float)v) >> 16);
}

// Magnitude key of x: the high word without the sign.  Keys order like |x| up to the low word,
// and the largest key of a row carries the largest biased exponent.
__device__ __forceinline__ unsigned mag_key(double x) { return (unsigned)__double2hiint(x) & 0x7fffffffu; }

// e with max |x| < 2^e over a row from its largest magnitude key: frexp's exponent of the largest
// element (f 2^e, 1/2 <= f < 1) when it is normal, 0 when every element is below 2^-1022 (those
// round to zero digits).
__device__ __forceinline__ int scale_exponent_key(unsigned key) {
  const int bex = (int)(key >> 20);
  return bex ? bex - 1022 : 0;
}

__global__ void __launch_bounds__(kGramThreads, 5) k_gram_slice(const SysDev *__restrict__ sysv, int ldir) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box) return;
  GramItem it;
  if (!decode_gram(s, blockIdx.x, it, ldir)) return;
  const DirDev &D = s.d[it.l];
  const int m0 = s.m0, nv = D.nv, Kp = D.Kpad;
  const int ld = nv + 1;
  extern __shared__ double sm[];
  double *Q = sm;
  double *E = Q + m0 * ld;
  double *red = E + m0 * ld;
  __shared__ int rexp[kMaxM0];
  gram_phase1(s, it, Q, E, red);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int nu = warp; nu < m0; nu += kGramThreads / 32) {
    unsigned mx = 0;
    for (int c = lane; c < nv; c += 32) mx = max(mx, mag_key(Q[nu * ld + c]));
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) rexp[nu] = scale_exponent_key(mx);
  }
  __syncthreads();
  const int64_t rows = (int64_t)D.Jc * m0 * m0;
  const int64_t row0 = ((int64_t)(it.jw - D.cw0) * m0 + it.mu) * m0;
  unsigned short *planes = reinterpret_cast<unsigned short *>(s.ws + D.offA);
  int *rowexp = reinterpret_cast<int *>(s.ws + D.offRE);
  if (tid < m0) rowexp[row0 + tid] = rexp[tid];
  // two adjacent columns per thread (Kp is even): one 32-bit store per digit plane
  const int half = Kp >> 1;
  const int items = m0 * half;
  for (int p0 = tid; p0 < items; p0 += kGramThreads) {
    const int nu = p0 / half, c = 2 * (p0 - nu * half);
    int a[kSlices], b[kSlices];
#pragma unroll
    for (int k = 0; k < kSlices; ++k) a[k] = b[k] = 0;
    if (c < nv) digits7(Q[nu * ld + c], rexp[nu], a);
    if (c + 1 < nv) digits7(Q[nu * ld + c + 1], rexp[nu], b);
    const int64_t at = (row0 + nu) * Kp + c;
#pragma unroll
    for (int k = 0; k < kSlices; ++k)
      *reinterpret_cast<unsigned *>(planes + k * rows * Kp + at) =
          (unsigned)bf16_of_int(a[k]) | ((unsigned)bf16_of_int(b[k]) << 16);
  }
}

// Digit planes of the potential factors: one CTA per (system, direction, rank term r).
__global__ void __launch_bounds__(kGramThreads) k_vslice(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box) return;
  int b = blockIdx.x, l = 0;
  for (; l < 3; ++l) {
    if (b < s.Rt) break;
    b -= s.Rt;
  }
  if (l == 3) return;
  const DirDev &D = s.d[l];
  const int r = b, nv = D.nv, Kp = D.Kpad, Rt = s.Rt;
  const double *v = s.ws + D.offV + (int64_t)r * nv;
  __shared__ unsigned part[kGramThreads / 32];
  __shared__ int e_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned mx = 0;
  for (int c = tid; c < nv; c += kGramThreads) mx = max(mx, mag_key(v[c]));
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 0) part[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    unsigned m = 0;
    for (int w = 0; w < kGramThreads / 32; ++w) m = max(m, part[w]);
    e_sh = scale_exponent_key(m);
    reinterpret_cast<int *>(s.ws + D.offCE)[r] = e_sh;
  }
  __syncthreads();
  const int e = e_sh;
  unsigned short *planes = reinterpret_cast<unsigned short *>(s.ws + D.offB);
  for (int c = 2 * tid; c < Kp; c += 2 * kGramThreads) {
    int a[kSlices], b[kSlices];
#pragma unroll
    for (int k = 0; k < kSlices; ++k) a[k] = b[k] = 0;
    if (c < nv) digits7(v[c], e, a);
    if (c + 1 < nv) digits7(v[c + 1], e, b);
#pragma unroll
    for (int k = 0; k < kSlices; ++k)
      *reinterpret_cast<unsigned *>(planes + ((int64_t)k * Rt + r) * Kp + c) =
          (unsigned)bf16_of_int(a[k]) | ((unsigned)bf16_of_int(b[k]) << 16);
  }
}

// C[jw][slot][mu][nu] = C[mirror(jw)][slot][nu][mu] for the window blocks that were not
// contracted: thread per element, systems on blockIdx.y.
__global__ void __launch_bounds__(256) k_gram_mirror(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box) return;
  int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int m0 = s.m0, mm = m0 * m0, slots = s.Rt + 2;
  int l = 0;
  for (; l < 3; ++l) {
    const int64_t cnt = (int64_t)(s.d[l].J - s.d[l].Jc) * slots * mm;
    if (item < cnt) break;
    item -= cnt;
  }
  if (l == 3) return;
  const DirDev &D = s.d[l];
  const int64_t per_block = (int64_t)slots * mm;
  int k = (int)(item / per_block);  // k-th block outside cw0 .. cw0 + Jc - 1
  const int rem = (int)(item - (int64_t)k * per_block);
  const int jw = k < D.cw0 ? k : k + D.Jc;
  // mirror: j' = -j; in the window j = jlo + jw, taken mod L when the window is the whole lattice
  int jm;
  if (D.J == D.L && D.jlo == 0) {
    jm = jw == 0 ? 0 : D.L - jw;
  } else {
    jm = -2 * D.jlo - jw;
  }
  const int slot = rem / mm, e = rem - slot * mm, mu = e / m0, nu = e - mu * m0;
  const double *src = s.ws + D.offC + ((int64_t)jm * slots + slot) * mm + nu * m0 + mu;
  s.ws[D.offC + ((int64_t)jw * slots + slot) * mm + e] = *src;
}

}  // namespace

cudaError_t launch_gram_mirror(const SysDev *sys, int nsys, long long max_items, cudaStream_t st) {
  if (max_items <= 0 || nsys <= 0) return cudaSuccess;
  dim3 grid((unsigned)((max_items + 255) / 256), nsys);
  kmark(LHF_K_GRAM_MIRROR, 1, st);
  k_gram_mirror<<<grid, 256, 0, st>>>(sys);
  kmark(LHF_K_GRAM_MIRROR, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_gram_fp64(const SysDev *sys, int nsys, int max_blocks, int max_m0,
                             int max_nv, cudaStream_t st, int ldir) {
  if (max_blocks <= 0 || nsys <= 0) return cudaSuccess;
  const size_t smem = sizeof(double) * ((size_t)2 * max_m0 * (max_nv + 1) + 2 * max_m0);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(max_blocks, nsys);
  kmark(LHF_K_GRAM_FP64, 1, st);
  k_gram_fp64<<<grid, kGramThreads, smem, st>>>(sys, ldir);
  kmark(LHF_K_GRAM_FP64, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_gram_slices(const SysDev *sys, int nsys, int max_blocks, int max_m0, int max_nv, cudaStream_t st,
                               int ldir) {
  if (max_blocks <= 0 || nsys <= 0) return cudaSuccess;
  const size_t smem = sizeof(double) * ((size_t)2 * max_m0 * (max_nv + 1) + 2 * max_m0);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_slice, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  kmark(LHF_K_GRAM_SLICE, 1, st);
  k_gram_slice<<<dim3(max_blocks, nsys), kGramThreads, smem, st>>>(sys, ldir);
  kmark(LHF_K_GRAM_SLICE, 0, st);
  return cudaGetLastError();
}

cudaError_t launch_vslices(const SysDev *sys, int nsys, int max_rt3, cudaStream_t st) {
  if (max_rt3 <= 0 || nsys <= 0) return cudaSuccess;
  kmark(LHF_K_VSLICE, 1, st);
  k_vslice<<<dim3(max_rt3, nsys), kGramThreads, 0, st>>>(sys);
  kmark(LHF_K_VSLICE, 0, st);
  return cudaGetLastError();
}

}  // namespace lhf
