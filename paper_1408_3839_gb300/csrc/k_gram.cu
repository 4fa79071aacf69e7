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
// the P1 sums; phase 2 contracts with the R_tot potential rows.  Deterministic: fixed-order
// floating-point reductions, and exact integer sums (whose order does not matter).
#include "lhf_internal.cuh"
#include "lhf_pairs.cuh"

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

// ---- exact fixed-point forms of FP64 rows ----------------------------------------------
//
// A row x[c] (c < nv) with max|x| = f 2^e, 1/2 <= f < 1, becomes the 62-bit fixed-point integers
// X[c] = rint(x[c] 2^(62-e)).  X is formed from the bit fields of x with integer arithmetic only
// (the FP64 pipe of this GPU runs at a small fraction of the integer rate): |x| = M 2^(ex - 1075)
// with M the 53-bit significand, so X = M 2^(ex - 1013 - e), a left shift by at most 9 bits
// (|x| < 2^e) or a right shift rounded to nearest, ties to even.
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

// Magnitude key of x: the high word without the sign.  Keys order like |x| up to the low word,
// and the largest key of a row carries the largest biased exponent.
__device__ __forceinline__ unsigned mag_key(double x) { return (unsigned)__double2hiint(x) & 0x7fffffffu; }

// e with max |x| < 2^e over a row from its largest magnitude key: frexp's exponent of the largest
// element (f 2^e, 1/2 <= f < 1) when it is normal, 0 when every element is below 2^-1022 (those
// round to zero).
__device__ __forceinline__ int scale_exponent_key(unsigned key) {
  const int bex = (int)(key >> 20);
  return bex ? bex - 1022 : 0;
}

// Row sums of Q as exact integer sums: term(c) = round(X[c] / 2^qsh) (X the fixed-point form
// above), sum = 2^(e + qsh - 62) sum_c term(c) -- each term within 2^(e + qsh - 63) of Q[c], the
// integer sum exact whatever its order, one rounding on conversion.  qsh >= 10 with nv < 2^qsh
// keeps |sum_c term| < 2^62 + 2^qsh (no overflow); for nv < 1024 the terms resolve 2^-52 of the
// row's largest element, the resolution of an FP64 sum.
__device__ __forceinline__ int row_sum_shift(int nv) {
  int qsh = 10;
  while (nv >= (1 << qsh)) ++qsh;
  return qsh;
}

__device__ __forceinline__ long long row_sum_term(long long X, int qsh) {
  return (X + (1ll << (qsh - 1))) >> qsh;
}

__device__ __forceinline__ long long warp_sum_i64(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// rexp[nu]: the scale exponent of row nu of Q (warp per row).
__device__ __forceinline__ void q_row_exponents(const double *Q, int ld, int m0, int nv, int *rexp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int nu = warp; nu < m0; nu += kGramThreads / 32) {
    unsigned mx = 0;
    for (int c = lane; c < nv; c += 32) mx = max(mx, mag_key(Q[nu * ld + c]));
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) rexp[nu] = scale_exponent_key(mx);
  }
}

// The P1 slots of C for row function mu (thread nu < m0): stiffness (1/h) sum D D and mass
// h sum f g - (h/6) sum D D, from dq = sum_c Q[nu][c] and de = red[2 nu + 1].
__device__ __forceinline__ void write_p1_slots(const SysDev &s, const GramItem &it, int nu, double dq, double de) {
  const DirDev &D = s.d[it.l];
  const int m0 = s.m0, Rt = s.Rt, mm = m0 * m0;
  double *Cout = s.ws + D.offC + (int64_t)it.jw * (Rt + 2) * mm + it.mu * m0;
  Cout[(int64_t)Rt * mm + nu] = de / D.h;
  Cout[(int64_t)(Rt + 1) * mm + nu] = D.h * dq - de * D.h / 6.0;
}

// Per column function nu (thread nu < m0 of a periodic direction): the cells p of g_nu's support
// where the row function shifted by j is present, as up to two runs of consecutive cells --
// [plo, phi] meets the row support [mlo, mhi] modulo L; unless the row support covers every
// residue its images [mlo + kL, mhi + kL] are disjoint, and [plo, phi] (at most L cells) meets at
// most two of them, k0 (the first that ends at or after plo) and k0 + 1 -- each run given by its
// length and the nodes of its first cell (for c = 0) in g_nu and in the shifted row function.
__device__ __forceinline__ void gram_runs(const SysDev &s, const GramItem &it, int (*seg)[2][3]) {
  const DirDev &D = s.d[it.l];
  const int m0 = s.m0, nc = D.nc, L = D.L, mu = it.mu, j = D.jlo + it.jw;
  const int tid = threadIdx.x;
  if (!D.periodic || tid >= m0) return;
  const int mlo = s.cell_lo[it.l][mu] + j, mhi = s.cell_hi[it.l][mu] + j;
  const int nu = tid;
  const int plo = s.cell_lo[it.l][nu];
  int phi = s.cell_hi[it.l][nu];
  if (phi > plo + L - 1) phi = plo + L - 1;
  int seg_lo[2] = {plo, 1}, seg_hi[2] = {phi, 0};
  if (mhi - mlo < L - 1) {
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

// Phase 1 for one CTA: Q[nu][c] in shared memory and red[2 nu + 1] = the sum over all nodes of the
// difference products D_i(g_mu,j) D_i(g_nu), with D_i(f) = f_i - f_(i+1) (periodic wrap; open:
// f_(-1) = f_n = 0).  The P1 forms follow from these sums and the row sums of Q:
//   g^T A f = (1/h) sum_i D_i(f) D_i(g),   g^T S f = h sum_i f_i g_i - (h/6) sum_i D_i(f) D_i(g),
// the same sums as (1/h) sum (2 f_i g_i - f_i g_(i+1) - f_(i+1) g_i) and (h/6) sum (4 f_i g_i +
// cross terms) regrouped: no cancellation in the stiffness sum and two products per node.
// A warp takes one column function nu at a time, its lanes the nodes c = lane + 32 k: the
// difference products of every node a lane visits accumulate in one register, so only a warp
// reduction per function is left (two functions per butterfly).
__device__ __forceinline__ void gram_phase1(const SysDev &s, const GramItem &it, double *Q, double *red) {
  const DirDev &D = s.d[it.l];
  const int m0 = s.m0, nv = D.nv, n = D.n, nc = D.nc;
  const int ld = nv + 1;
  const double *G = s.ws + D.offG;
  const double *Dg = s.ws + D.offD;
  const int mu = it.mu;
  const double *f = G + (int64_t)mu * n;
  const double *df = Dg + (int64_t)mu * n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kWarps = kGramThreads / 32;
  const bool periodic = D.periodic != 0;
  __shared__ int seg[kMaxM0][2][3];  // [nu][run]: cells, first node of g_nu, first node of the row
  gram_runs(s, it, seg);
  __syncthreads();
  for (int nu0 = warp; nu0 < m0; nu0 += 2 * kWarps) {
    double es0 = 0.0, es1 = 0.0;
    for (int h = 0; h < 2; ++h) {
      const int nu = nu0 + h * kWarps;
      if (nu >= m0) break;  // warp-uniform
      const double *g = G + (int64_t)nu * n;
      const double *dg = Dg + (int64_t)nu * n;
      double e = 0.0;
      if (periodic) {
        for (int c = lane; c < nv; c += 32) {
          // visited in increasing p; the indices advance by one cell per p (no division in the loop)
          double q = 0.0;
#pragma unroll
          for (int sg = 0; sg < 2; ++sg) {
            const int cnt = seg[nu][sg][0];
            int iv = seg[nu][sg][1] + c;
            int iu = seg[nu][sg][2] + c;
            for (int t = 0; t < cnt; ++t) {
              q = fma(f[iu], g[iv], q);
              e = fma(df[iu], dg[iv], e);
              iv += nc;
              if (iv >= n) iv -= n;
              iu += nc;
              if (iu >= n) iu -= n;
            }
          }
          Q[nu * ld + c] = q;
        }
      } else {
        // single open cell: nodes c = 0..n-1, Dirichlet ends (the virtual node -1 adds f_0 g_0)
        if (lane == 0) e = f[0] * g[0];
        for (int c = lane; c < nv; c += 32) {
          Q[nu * ld + c] = f[c] * g[c];
          e = fma(df[c], dg[c], e);
        }
      }
      if (h == 0) es0 = e;
      else es1 = e;
    }
    // lanes 0-15 end with the warp's total for nu0, lanes 16-31 with that for nu0 + kWarps: one
    // exchanging step (each half keeps one function), then four steps within the halves
    const bool up = (lane & 16) != 0;
    double v = (up ? es1 : es0) + __shfl_xor_sync(0xffffffffu, up ? es0 : es1, 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[2 * nu0 + 1] = v;
    if (lane == 16 && nu0 + kWarps < m0) red[2 * (nu0 + kWarps) + 1] = v;
  }
  __syncthreads();
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
  double *red = Q + m0 * ld;    // [m0][2]   row sum of Q, sum of the difference products per nu
  __shared__ int rexp[kMaxM0];
  gram_phase1(s, it, Q, red);
  // P1 slots: the row sums of Q as exact fixed-point sums (the same numbers as the tensor-core
  // route, which forms them from its digit planes)
  q_row_exponents(Q, ld, m0, nv, rexp);
  __syncthreads();
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, qsh = row_sum_shift(nv);
    for (int nu = warp; nu < m0; nu += kGramThreads / 32) {
      long long acc = 0;
      for (int c = lane; c < nv; c += 32) acc += row_sum_term(fixed62(Q[nu * ld + c], rexp[nu]), qsh);
      acc = warp_sum_i64(acc);
      if (lane == 0) red[2 * nu] = scale_pow2((double)acc, rexp[nu] + qsh - 62);
    }
  }
  __syncthreads();
  if (threadIdx.x < m0) write_p1_slots(s, it, threadIdx.x, red[2 * threadIdx.x], red[2 * threadIdx.x + 1]);

  // ---- phase 2: C_r[nu] = sum_c V[r][c] Q[nu][c] ------------------------------------------
  // over the rows whose functions share a cell (listed first, so that every thread's dot product
  // is one that can be nonzero); the others' slots are exact zeros
  const int Rt = s.Rt;
  const int mm = m0 * m0;
  const int mu = it.mu;
  double *Cout = s.ws + D.offC + (int64_t)it.jw * (Rt + 2) * mm + mu * m0;
  const double *V = s.ws + D.offV;
  __shared__ int nzl[kMaxM0], nnz_sh;
  __shared__ unsigned zmask_sh;
  if (threadIdx.x == 0) {
    int k = 0;
    unsigned zm = 0u;
    for (int nu = 0; nu < m0; ++nu) {
      if (D.periodic && gram_row_cells(s, it.l, D.jlo + it.jw, mu, nu) == 0)
        zm |= 1u << nu;
      else
        nzl[k++] = nu;
    }
    nnz_sh = k;
    zmask_sh = zm;
  }
  __syncthreads();
  const int nnz = nnz_sh;
  const unsigned zmask = zmask_sh;
  if (zmask)
    for (int o = threadIdx.x; o < Rt * m0; o += kGramThreads)
      if ((zmask >> (o % m0)) & 1u) Cout[(int64_t)(o / m0) * mm + o % m0] = 0.0;
  const int outs = Rt * nnz;
  for (int o = threadIdx.x; o < outs; o += kGramThreads) {
    const int r = o / nnz;
    const int nu = nzl[o - r * nnz];
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
// The fixed-point integers X[c] of a row (fixed62 above) split into 7 balanced base-2^7 digits
//   X = a_0 2^55 + a_1 2^48 + ... + a_6 2^13 + r,  a_0 in [-128, 128], a_k in [-64, 63], -2^12 <= r < 2^12,
// so x[c] = 2^e (sum_k a_k 2^(-7(k+1)) + O(2^-50)).  Every digit is an integer of at most 8
// significant bits, exact in BF16; products of two digits are exact in FP32 and sums of up to
// 2^24 / 2^14 of them accumulate exactly.  Digit k of (row, c) goes to
// planes + ((k * Kpad / 32 + c / 32) * rows + row) * 32 + c % 32 (BF16, Kpad >= nv, zero padded):
// chunk-major, so that a 32-column tile of consecutive rows is contiguous.
// Digits from the least significant end: the 13 remainder bits round half up into digit 6 (a carry
// when bit 12 is set), then each 7-bit field plus the incoming carry becomes a digit in [-64, 63]
// and a carry; the top digit takes the bits from 55 up and the last carry.  The digits and the
// remainder (X mod 2^13, balanced) are those of rounding from the top down, up to the choice
// between +64 and -64 plus a carry, with one field extract and three integer steps per digit.
__device__ __forceinline__ void digits7(long long X, int *a) {  // |X| <= 2^62
  const unsigned long long U = (unsigned long long)X;
  int carry = (int)((U >> 12) & 1u);
#pragma unroll
  for (int k = kSlices - 1; k >= 1; --k) {
    const int sh = 55 - 7 * k;
    const int t = (int)((U >> sh) & 0x7fu) + carry;
    carry = (t + 64) >> 7;
    a[k] = t - (carry << 7);
  }
  a[0] = (int)(X >> 55) + carry;
}

__device__ __forceinline__ unsigned short bf16_of_int(int v) {  // exact for |v| <= 256
  return (unsigned short)(__float_as_uint((float)v) >> 16);
}

// The 7 digits of x = h + l (a pair, |x| < 1) as integer-valued floats, x = sum_k a_k 2^(-7(k+1))
// + O(2^-50): each digit the nearest integer to 128 times the remainder, decided by the
// remainder's leading word; TwoSum folds the trailing word in before digits 2, 4 and 6 (before
// it can reach 2^-11 of the remainder), so a_0 is in [-128, 128] and |a_k| <= 64 after it, the
// bounds of digits7.  A digit takes three exact steps: t = 128 h + 1.5 2^23 (rounds 128 h to an
// integer), d = t - 1.5 2^23, h <- 128 h - d (one FMA: the difference is representable); the
// trailing word is scaled only when folded in (by 2^14, for the two digits since the last fold).
__device__ __forceinline__ void digits7f(float h, float l, float *a) {
  const float m = 12582912.0f;
#pragma unroll
  for (int k = 0; k < kSlices; ++k) {
    if (k == 2 || k == 4 || k == 6) {
      float t, e;
      two_sum(h, __fmul_rn(l, 16384.0f), t, e);
      h = t;
      l = e;
    }
    const float d = __fadd_rn(__fmaf_rn(h, 128.0f, m), -m);
    a[k] = d;
    h = __fmaf_rn(h, 128.0f, -d);
  }
}

// The folded products in compensated FP32 pairs and their digit planes (tensor-core route), one
// CTA per (system, direction, window block, mu).  GB300 issues FP64 at 1/64 of the FP32 rate, so
// the fold runs on the pairs h + l of the samples and differences written by k_basis (one 16-byte
// load per node and function gives both): each
// product exact as a pair (an FMA gives its rounding error), the sums compensated (TwoSum), a
// relative error of a few units of 2^-48 of sum |g_mu,j g_nu| per folded value.  Per row nu:
//   * Q[nu][c] (pairs) in shared memory, a warp per nu, lanes over the nodes c;
//   * the row scale e with max_c |Q| < 2^e (frexp's exponent of the largest |h| + |l|);
//   * the P1 slots from the compensated sums over the nodes of Q and of the difference products:
//     stiffness (1/h) sum D D and mass h sum f g - (h/6) sum D D, in pairs (the factors 1/h, h,
//     h/6 as pairs from the host), converted to FP64 once;
//   * the 7 digit planes of Q 2^-e (digits7f), two adjacent nodes per thread and store, in the
//     chunk-major layout of digits7 (c >= n_v: zero).
__global__ void __launch_bounds__(kGramThreads, 4) k_gram_slice(const SysDev *__restrict__ sysv, int ldir) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box) return;
  GramItem it;
  if (!decode_gram(s, blockIdx.x, it, ldir)) return;
  const DirDev &D = s.d[it.l];
  const int m0 = s.m0, nv = D.nv, n = D.n, nc = D.nc, Kp = D.Kpad, Rt = s.Rt, mm = m0 * m0;
  const int ld = nv + 1;
  const bool periodic = D.periodic != 0;
  extern __shared__ float2 Qp[];  // [m0][ld] folded products as pairs
  __shared__ int seg[kMaxM0][2][3];
  __shared__ int rexp[kMaxM0];
  __shared__ float2 qsum[kMaxM0], esum[kMaxM0];
  gram_runs(s, it, seg);
  __syncthreads();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int kWarps = kGramThreads / 32;
  const float4 *GD = reinterpret_cast<const float4 *>(s.ws + D.offGD);  // {sample, difference} pairs
  const float4 *f = GD + (int64_t)it.mu * n;
  for (int nu = warp; nu < m0; nu += kWarps) {
    if (periodic && seg[nu][0][0] == 0 && seg[nu][1][0] == 0) {
      // no cell where both functions live: every folded value and sum is an exact zero
      for (int c = lane; c < nv; c += 32) Qp[nu * ld + c] = make_float2(0.0f, 0.0f);
      if (lane == 0) {
        rexp[nu] = 0;
        qsum[nu] = esum[nu] = make_float2(0.0f, 0.0f);
      }
      continue;  // warp-uniform
    }
    const float4 *g = GD + (int64_t)nu * n;
    float q0 = 0.0f, q1 = 0.0f, e0 = 0.0f, e1 = 0.0f, mx = 0.0f;
    if (!periodic && lane == 0) {
      // single open cell, Dirichlet ends: the virtual node -1 adds f_0 g_0 to the difference sum
      const float4 a = __ldg(&f[0]), b = __ldg(&g[0]);
      acc_prod(e0, e1, a.x, a.y, b.x, b.y);
    }
    for (int c = lane; c < nv; c += 32) {
      float qs = 0.0f, qc = 0.0f;
      if (periodic) {
        // visited in increasing p; the indices advance by one cell per p
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
          const int cnt = seg[nu][sg][0];
          int iv = seg[nu][sg][1] + c, iu = seg[nu][sg][2] + c;
#pragma unroll 2
          for (int t = 0; t < cnt; ++t) {
            const float4 a = __ldg(&f[iu]), b = __ldg(&g[iv]);
            acc_prod(qs, qc, a.x, a.y, b.x, b.y);
            acc_prod(e0, e1, a.z, a.w, b.z, b.w);
            iv += nc;
            if (iv >= n) iv -= n;
            iu += nc;
            if (iu >= n) iu -= n;
          }
        }
      } else {
        const float4 a = __ldg(&f[c]), b = __ldg(&g[c]);
        acc_prod(qs, qc, a.x, a.y, b.x, b.y);
        acc_prod(e0, e1, a.z, a.w, b.z, b.w);
      }
      float2 q;
      two_sum(qs, qc, q.x, q.y);
      Qp[nu * ld + c] = q;
      mx = fmaxf(mx, fabsf(q.x) + fabsf(q.y));
      acc_add(q0, q1, q.x, q.y);
    }
    const unsigned key = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));  // mx >= 0: bits order as values
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float a0 = __shfl_xor_sync(0xffffffffu, q0, o), a1 = __shfl_xor_sync(0xffffffffu, q1, o);
      const float b0 = __shfl_xor_sync(0xffffffffu, e0, o), b1 = __shfl_xor_sync(0xffffffffu, e1, o);
      acc_add(q0, q1, a0, a1);
      acc_add(e0, e1, b0, b1);
    }
    if (lane == 0) {
      // |Q| <= |h| + |l| < 2^e (frexp's exponent; the e of a denormal maximum is -126)
      const int be = (int)(key >> 23);
      rexp[nu] = key == 0u ? 0 : (be == 0 ? -126 : min(be - 126, 126));
      qsum[nu] = df_norm(q0, q1);
      esum[nu] = df_norm(e0, e1);
    }
  }
  __syncthreads();
  // rows with overlap only (compact index from k_gram_rowmap); the others' rank slots are zeros
  const int64_t rows = D.rows_c;
  const int64_t row0 = ((int64_t)(it.jw - D.cw0) * m0 + it.mu) * m0;
  const int *f2c = reinterpret_cast<const int *>(s.ws + D.offRM);
  __shared__ int crow[kMaxM0];
  if (tid < m0) crow[tid] = f2c[row0 + tid];
  {
    double *Cz = s.ws + D.offC + (int64_t)it.jw * (Rt + 2) * mm + it.mu * m0;
    for (int e = tid; e < Rt * m0; e += kGramThreads) {
      const int r = e / m0, nu = e - r * m0;
      if (f2c[row0 + nu] < 0) Cz[(int64_t)r * mm + nu] = 0.0;
    }
  }
  if (tid < m0) {
    if (crow[tid] >= 0) reinterpret_cast<int *>(s.ws + D.offRE)[crow[tid]] = rexp[tid];
    // P1 slots in pairs, converted once (m0 threads of one warp: one FP64 pass)
    const float2 invh = make_float2(D.p1h[0], D.p1h[1]), h1 = make_float2(D.p1h[2], D.p1h[3]);
    const float2 h6 = make_float2(D.p1h[4], D.p1h[5]);
    const float2 stiff = df_mul(esum[tid], invh);
    const float2 mass = df_add(df_mul(qsum[tid], h1), df_neg(df_mul(esum[tid], h6)));
    double *Cout = s.ws + D.offC + (int64_t)it.jw * (Rt + 2) * mm + it.mu * m0;
    Cout[(int64_t)Rt * mm + tid] = (double)stiff.x + (double)stiff.y;
    Cout[(int64_t)(Rt + 1) * mm + tid] = (double)mass.x + (double)mass.y;
  }
  // digit planes: two adjacent columns per thread (Kp is a multiple of 64, so c and c + 1 share a
  // 32-column chunk), one 32-bit store per plane
  unsigned short *planes = reinterpret_cast<unsigned short *>(s.ws + D.offA);
  const int half = Kp >> 1;
  const int64_t plane = (int64_t)(Kp / kPlaneChunk) * rows * kPlaneChunk;  // = rows * Kp
  __syncthreads();  // crow
  for (int p0 = tid; p0 < m0 * half; p0 += kGramThreads) {
    const int nu = p0 / half, c = 2 * (p0 - nu * half);
    if (crow[nu] < 0) continue;  // warp-uniform: a warp's 64 columns share nu
    const float sc = __int_as_float((127 - rexp[nu]) << 23);  // 2^-e, e in [-126, 126]
    float a[kSlices], b[kSlices];
#pragma unroll
    for (int k = 0; k < kSlices; ++k) a[k] = b[k] = 0.0f;
    if (c < nv) {
      const float2 q = Qp[nu * ld + c];
      digits7f(__fmul_rn(q.x, sc), __fmul_rn(q.y, sc), a);
    }
    if (c + 1 < nv) {
      const float2 q = Qp[nu * ld + c + 1];
      digits7f(__fmul_rn(q.x, sc), __fmul_rn(q.y, sc), b);
    }
    const int64_t at = ((int64_t)(c / kPlaneChunk) * rows + crow[nu]) * kPlaneChunk + c % kPlaneChunk;
    // BF16 of an integer-valued float of at most 8 significant bits: its upper half, exact
#pragma unroll
    for (int k = 0; k < kSlices; ++k)
      *reinterpret_cast<unsigned *>(planes + k * plane + at) =
          (__float_as_uint(a[k]) >> 16) | (__float_as_uint(b[k]) & 0xffff0000u);
  }
}

// The rows with overlap (gram_row_cells > 0) of one direction's contracted window, in row order:
// full -> compact index (-1 for a row whose folded products vanish identically), compact -> full.
// One CTA per (system, direction), rows in rounds of the block: a ballot per warp, the warps'
// counts prefixed through shared memory.
__global__ void __launch_bounds__(kGramThreads) k_gram_rowmap(const SysDev *__restrict__ sysv) {
  const SysDev &s = sysv[blockIdx.y];
  const int l = blockIdx.x;
  if (s.box || l > 2) return;
  const DirDev &D = s.d[l];
  if (D.Jc <= 0 || D.offRM < 0) return;
  const int m0 = s.m0, mm = m0 * m0, rows = D.Jc * mm;
  int *f2c = reinterpret_cast<int *>(s.ws + D.offRM), *c2f = f2c + rows;
  __shared__ int wcount[kGramThreads / 32];
  __shared__ int base_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) base_sh = 0;
  __syncthreads();
  for (int r0 = 0; r0 < rows; r0 += kGramThreads) {
    const int row = r0 + tid;
    bool nz = false;
    if (row < rows) {
      const int jc = row / mm, mu = (row / m0) % m0, nu = row % m0;
      nz = gram_row_cells(s, l, D.jlo + D.cw0 + jc, mu, nu) > 0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, nz);
    if (lane == 0) wcount[warp] = __popc(bal);
    __syncthreads();
    int before = base_sh;
    for (int w = 0; w < warp; ++w) before += wcount[w];
    const int k = before + __popc(bal & ((1u << lane) - 1u));
    if (row < rows) {
      f2c[row] = nz ? k : -1;
      if (nz) c2f[k] = row;
    }
    __syncthreads();
    if (tid == 0)
      for (int w = 0; w < kGramThreads / 32; ++w) base_sh += wcount[w];
    __syncthreads();
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
    if (c < nv) digits7(fixed62(v[c], e), a);
    if (c + 1 < nv) digits7(fixed62(v[c + 1], e), b);
#pragma unroll
    for (int k = 0; k < kSlices; ++k)
      *reinterpret_cast<unsigned *>(
          planes + (((int64_t)k * (Kp / kPlaneChunk) + c / kPlaneChunk) * Rt + r) * kPlaneChunk + c % kPlaneChunk) =
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
  const size_t smem = sizeof(double) * ((size_t)max_m0 * (max_nv + 1) + 2 * max_m0);
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
                               int ldir, bool rowmap) {
  if (max_blocks <= 0 || nsys <= 0) return cudaSuccess;
  const size_t smem = sizeof(float2) * (size_t)max_m0 * (max_nv + 1);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_slice, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  kmark(LHF_K_GRAM_SLICE, 1, st);
  // the row map, once, inside the first slicing launch's bracket (it precedes every slicing launch)
  if (rowmap) k_gram_rowmap<<<dim3(3, nsys), kGramThreads, 0, st>>>(sys);
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
