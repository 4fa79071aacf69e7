// k_dft.cu -- step a7: DFT of the first block column along the lattice indices, FP64 complex.
//
// Xbar_kappa = sum_j omega^{kappa . j} X_j, omega_l = exp(-2 pi i / L_l)  (Prop. 6.1 eq. (6.6);
// Lemma 2.2 eq. (2.1): the multilevel transform F_L = F_L0 x F_L1 x F_L2 applied to every entry
// (mu, nu) of the folded block column).  The three levels are separable, so the transform runs
// as one pass per lattice dimension with L_d > 1 (d = 2, 1, 0); the first pass of a system
// reads the real blocks, later passes work in place on the complex output.
//
// A CTA owns a tile of TW consecutive inner indices (entries (mu, nu) and the faster lattice
// dimensions) for all L_d positions of one outer index: global loads and stores are rows of TW
// contiguous values.  The blocks of a real lattice matrix satisfy H_-j = H_j^T, so every
// transformed block is Hermitian, Hbar_kappa[nu][mu] = conj(Hbar_kappa[mu][nu]) (the same holds
// for S): the last pass transforms only the entries mu <= nu and writes the others as their
// conjugates (earlier passes of a multi-dimensional lattice still relate entries of different
// outer indices and transform every entry).  The tile is transformed in shared memory: an
// iterative radix-4 FFT (fft_columns) when L_d is a power of two, Bluestein's chirp transform
// through such FFTs of length M >= 2 L_d - 1 otherwise (64 <= L_d <= 1024), the direct O(L_d^2)
// sum for the other lengths.  Twiddles come from a per-CTA table built with sincospi
// (correctly-rounded arguments).
#include "lhf_internal.cuh"

namespace lhf {
namespace {

constexpr int kDftThreads = 256;

__host__ __device__ inline int tile_width(int Ld) {
  int tw = 16;
  while (tw > 1 && (size_t)Ld * tw * 2 > 8192) tw >>= 1;  // <= 128 KB of complex data
  return tw;
}

__device__ inline unsigned bitrev(unsigned x, int bits) { return __brev(x) >> (32 - bits); }

// Bluestein's transform for a length L that is not a power of two: with w_n = exp(-pi i n^2 / L),
// omega^(j k) = w_j w_k conj(w_(k-j)) (since 2 j k = j^2 + k^2 - (k - j)^2), so
//   Xbar_k = w_k sum_j (x_j w_j) conj(w_(k-j)),
// a cyclic convolution of length M (the power of two >= 2 L - 1) taken by power-of-two FFTs:
// A = F_M(x w) (zero-padded), B = F_M(b) with b_n = conj(w_|n|) at n mod M for |n| < L (the
// same for every column: once per CTA), Xbar_k = w_k conj(F_M(conj(A B)))_k / M.  O(M log M) per
// column instead of the direct sum's L^2.  For kBluesteinMinL <= L <= kBluesteinMaxL (M <=
// 2048; shorter lengths keep the direct sum, as cheap there); the chirp arguments n^2 / L are
// reduced modulo 2 exactly in integers.
constexpr int kBluesteinMinL = 64, kBluesteinMaxL = 1024;

__host__ __device__ inline int bluestein_m(int Ld) {
  if ((Ld & (Ld - 1)) == 0 || Ld < kBluesteinMinL || Ld > kBluesteinMaxL) return 0;
  int M = 1;
  while (M < 2 * Ld - 1) M <<= 1;
  return M;
}

// Tile width of a transform pass: the columns of one CTA, so that the transformed length (Ld, or
// Bluestein's M) times the width fits 128 KB of complex values.
__host__ __device__ inline int pass_tile_width(int Ld) {
  const int M = bluestein_m(Ld);
  const int len = M ? M : Ld;
  int tw = 16;
  while (tw > 1 && (size_t)len * tw * 2 > 8192) tw >>= 1;
  return tw;
}

// Shared memory of a transform pass of length Ld (the tile, the twiddle table; Bluestein: the
// length-M table, the filter's transform and the chirp).
__host__ __device__ inline size_t pass_smem_bytes(int Ld) {
  const int M = bluestein_m(Ld), TW = pass_tile_width(Ld);
  return sizeof(double2) * (M ? (size_t)M * TW + 2 * (size_t)M + Ld : (size_t)Ld * TW + Ld);
}

// In-place FFT of M (a power of two) positions x TW columns stored bit-reversed (x[j * TW + t]),
// output in natural order; tab[m] = omega_M^m.  Decimation in time, two levels (spans hs and
// 2 hs) per pass (radix 4): with w2 = omega_(4 hs)^kk, the level-hs twiddle is w1 = w2^2 and the
// two level-2hs twiddles are w2 and -i w2, so the outputs at positions p + {0, 1, 2, 3} hs are
//   A + C, B - i D, A - C, B + i D,   A, B = x0 +- w1 x1,   C, D = w2 x2 +- w3 x3,   w3 = w2^3:
// three complex multiplications per four points where two radix-2 levels take four, and one
// shared-memory round trip and barrier per two levels.  An odd number of levels starts with one
// radix-2 level (twiddle 1); the first pass (hs = 1) needs no multiplication.
__device__ void fft_columns(double2 *x, int M, int TW, const double2 *tab) {
  const int bits = __ffs(M) - 1;
  int hs = 1;
  if (bits & 1) {
    for (int k = threadIdx.x; k < (M / 2) * TW; k += blockDim.x) {
      const int t = k % TW, top = 2 * (k / TW);
      const double2 u = x[top * TW + t], v = x[(top + 1) * TW + t];
      x[top * TW + t] = make_double2(u.x + v.x, u.y + v.y);
      x[(top + 1) * TW + t] = make_double2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
    hs = 2;
  }
  for (; hs < M; hs <<= 2) {
    const int s4 = M / (4 * hs);  // table stride of omega_(4 hs)
    for (int k = threadIdx.x; k < (M / 4) * TW; k += blockDim.x) {
      const int t = k % TW, gq = k / TW;
      const int kk = gq % hs, p0 = (gq / hs) * 4 * hs + kk;
      double2 x0 = x[p0 * TW + t], x1 = x[(p0 + hs) * TW + t];
      double2 x2 = x[(p0 + 2 * hs) * TW + t], x3 = x[(p0 + 3 * hs) * TW + t];
      if (kk != 0) {
        const double2 w1 = tab[2 * kk * s4], w2 = tab[kk * s4], w3 = tab[3 * kk * s4];
        x1 = make_double2(w1.x * x1.x - w1.y * x1.y, w1.x * x1.y + w1.y * x1.x);
        x2 = make_double2(w2.x * x2.x - w2.y * x2.y, w2.x * x2.y + w2.y * x2.x);
        x3 = make_double2(w3.x * x3.x - w3.y * x3.y, w3.x * x3.y + w3.y * x3.x);
      }
      const double2 A = make_double2(x0.x + x1.x, x0.y + x1.y), B = make_double2(x0.x - x1.x, x0.y - x1.y);
      const double2 C = make_double2(x2.x + x3.x, x2.y + x3.y), D = make_double2(x2.x - x3.x, x2.y - x3.y);
      x[p0 * TW + t] = make_double2(A.x + C.x, A.y + C.y);
      x[(p0 + hs) * TW + t] = make_double2(B.x + D.y, B.y - D.x);  // B - i D
      x[(p0 + 2 * hs) * TW + t] = make_double2(A.x - C.x, A.y - C.y);
      x[(p0 + 3 * hs) * TW + t] = make_double2(B.x - D.y, B.y + D.x);  // B + i D
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kDftThreads) k_dft_pass(const SysDev *__restrict__ sysv, int d) {
  const SysDev &s = sysv[blockIdx.y];
  if (s.box || s.d[0].L > kDftTileMax) return;  // long chains take the four-step route
  const int L0 = s.d[0].L, L1 = s.d[1].L, L2 = s.d[2].L;
  const int Ls[3] = {L0, L1, L2};
  const bool all_one = (L0 == 1 && L1 == 1 && L2 == 1);
  if (!(Ls[d] > 1 || (d == 0 && all_one))) return;
  // first pass of this system reads the real blocks
  int first = 0;
  for (int q = 2; q >= 0; --q)
    if (Ls[q] > 1) {
      first = q;
      break;
    }
  const bool real_in = (d == first);
  int last = 0;  // the final pass: the lowest dimension with L_d > 1 (0 for a single block)
  for (int q = 0; q < 3; ++q)
    if (Ls[q] > 1) {
      last = q;
      break;
    }
  const bool upper = (d == last);
  const int Ld = Ls[d];
  const int m0 = s.m0, mm = m0 * m0, nup = upper ? m0 * (m0 + 1) / 2 : mm;
  int64_t nlat = 1;  // faster lattice positions
  for (int q = d + 1; q < 3; ++q) nlat *= Ls[q];
  const int64_t inner = nlat * mm;       // stride of one position along dimension d
  const int64_t items = nlat * nup;      // inner items transformed
  int64_t outer = 1;
  for (int q = 0; q < d; ++q) outer *= Ls[q];
  const int TW = pass_tile_width(Ld);
  const int64_t tiles_inner = (items + TW - 1) / TW;
  const int64_t tile = blockIdx.x;
  if (tile >= outer * tiles_inner) return;
  const int64_t o = tile / tiles_inner;
  const int64_t i0 = (tile - o * tiles_inner) * TW;
  const int tw_valid = (int)((items - i0) < TW ? (items - i0) : TW);
  // inner offsets of this tile's items (and of their transposed entries), kept by thread t < TW
  __shared__ int64_t off_sh[16], offT_sh[16];
  if ((int)threadIdx.x < TW) {
    const int t = threadIdx.x;
    int64_t u = i0 + t < items ? i0 + t : 0;
    const int64_t lat = u / nup;
    int r = (int)(u - lat * nup), mu = 0, nu = 0;
    if (upper) {
      while (r >= m0 - mu) {  // row mu holds nu = mu .. m0 - 1
        r -= m0 - mu;
        ++mu;
      }
      nu = mu + r;
    } else {
      mu = r / m0;
      nu = r - mu * m0;
    }
    off_sh[t] = lat * mm + mu * m0 + nu;
    offT_sh[t] = (upper && mu != nu) ? lat * mm + nu * m0 + mu : -1;
  }
  __syncthreads();

  const int Mb = bluestein_m(Ld);
  if (Mb > 0) {
    // Bluestein (see bluestein_m): H and S in separate transforms (blockIdx.z)
    const double *Xr = blockIdx.z == 0 ? s.H : s.S;
    double *Xc = blockIdx.z == 0 ? s.Hbar : s.Sbar;
    extern __shared__ double smb[];
    double2 *x = reinterpret_cast<double2 *>(smb);  // [Mb][TW]
    double2 *tab = x + (size_t)Mb * TW;             // [Mb] omega_M^m
    double2 *Bf = tab + Mb;                         // [Mb] F_M(b)
    double2 *wch = Bf + Mb;                         // [Ld] w_n
    const int tid = threadIdx.x, bitsM = __ffs(Mb) - 1;
    for (int m = tid; m < Mb; m += kDftThreads) {
      double sn, cs;
      sincospi(2.0 * (double)m / (double)Mb, &sn, &cs);
      tab[m] = make_double2(cs, -sn);
    }
    for (int n = tid; n < Ld; n += kDftThreads) {
      const long long r = ((long long)n * n) % (2ll * Ld);  // n^2 mod 2L: exp(-pi i n^2 / L) exactly periodic
      double sn, cs;
      sincospi((double)r / (double)Ld, &sn, &cs);
      wch[n] = make_double2(cs, -sn);
    }
    __syncthreads();
    for (int p = tid; p < Mb; p += kDftThreads) {  // b, bit-reversed
      const int n = p < Ld ? p : (p > Mb - Ld ? Mb - p : -1);
      Bf[bitrev((unsigned)p, bitsM)] = n >= 0 ? make_double2(wch[n].x, -wch[n].y) : make_double2(0.0, 0.0);
    }
    for (int k = tid; k < Mb * TW; k += kDftThreads) {  // a = x w, zero-padded, bit-reversed
      const int j = k / TW, t = k - j * TW;
      double2 v = make_double2(0.0, 0.0);
      if (j < Ld && t < tw_valid) {
        const int64_t idx = (o * Ld + j) * inner + off_sh[t];
        const double2 xv = real_in ? make_double2(Xr[idx], 0.0) : reinterpret_cast<const double2 *>(Xc)[idx];
        const double2 w = wch[j];
        v = make_double2(xv.x * w.x - xv.y * w.y, xv.x * w.y + xv.y * w.x);
      }
      x[bitrev((unsigned)j, bitsM) * TW + t] = v;
    }
    __syncthreads();
    fft_columns(Bf, Mb, 1, tab);
    fft_columns(x, Mb, TW, tab);
    // conj(A B), moved to bit-reversed order for the second transform (pairs of swapped slots)
    for (int k = tid; k < Mb * TW; k += kDftThreads) {
      const int j = k / TW, t = k - j * TW;
      const int jr = (int)bitrev((unsigned)j, bitsM);
      if (jr < j) continue;
      const double2 a = x[j * TW + t], b = Bf[j], a2 = x[jr * TW + t], b2 = Bf[jr];
      const double2 u = make_double2(a.x * b.x - a.y * b.y, -(a.x * b.y + a.y * b.x));
      const double2 u2 = make_double2(a2.x * b2.x - a2.y * b2.y, -(a2.x * b2.y + a2.y * b2.x));
      x[jr * TW + t] = u;
      x[j * TW + t] = u2;
    }
    __syncthreads();
    fft_columns(x, Mb, TW, tab);
    const double invM = 1.0 / (double)Mb;  // a power of two: exact
    for (int k = tid; k < Ld * TW; k += kDftThreads) {
      const int kap = k / TW, t = k - kap * TW;
      if (t >= tw_valid) continue;
      const double2 z = x[kap * TW + t], w = wch[kap];  // Xbar = w conj(z) / M
      const double re = invM * (w.x * z.x + w.y * z.y), im = invM * (w.y * z.x - w.x * z.y);
      const int64_t base = (o * Ld + kap) * inner;
      reinterpret_cast<double2 *>(Xc)[base + off_sh[t]] = make_double2(re, im);
      if (offT_sh[t] >= 0) reinterpret_cast<double2 *>(Xc)[base + offT_sh[t]] = make_double2(re, -im);
    }
    return;
  }

  const bool pow2 = (Ld & (Ld - 1)) == 0;
  // real first pass of a power-of-two length: H and S in one complex transform of
  // z = H + i sigma S (sigma a power of two balancing the tile's magnitudes), unpacked as
  // Hbar_k = (Z_k + conj Z_-k) / 2, Sbar_k = (Z_k - conj Z_-k) / (2 i sigma); the z = 1 CTAs idle
  const bool packed = real_in && pow2;
  if (packed && blockIdx.z == 1) return;
  const double *Xr = blockIdx.z == 0 ? s.H : s.S;
  double *Xc = blockIdx.z == 0 ? s.Hbar : s.Sbar;

  extern __shared__ double sm[];
  double2 *x = reinterpret_cast<double2 *>(sm);  // [Ld][TW]
  double2 *tab = x + (size_t)Ld * TW;            // [Ld] omega^m
  const int tid = threadIdx.x;
  for (int m = tid; m < Ld; m += kDftThreads) {
    double sn, cs;
    sincospi(2.0 * (double)m / (double)Ld, &sn, &cs);
    tab[m] = make_double2(cs, -sn);
  }
  const int bits = pow2 ? __ffs(Ld) - 1 : 0;
  int sig_e = 0;  // sigma = 2^sig_e
  if (packed) {
    // the exponents of max |H| and max |S| over the tile, from the largest high words without the
    // sign (integer operations: they order like the magnitudes up to the low word, and carry the
    // largest biased exponent; frexp's exponent is that exponent - 1022 for a normal maximum)
    unsigned kh = 0u, ks = 0u;
    for (int k = tid; k < Ld * TW; k += kDftThreads) {
      const int j = k / TW, t = k - j * TW;
      if (t < tw_valid) {
        const int64_t idx = (o * Ld + j) * inner + off_sh[t];
        kh = max(kh, (unsigned)__double2hiint(s.H[idx]) & 0x7fffffffu);
        ks = max(ks, (unsigned)__double2hiint(s.S[idx]) & 0x7fffffffu);
      }
    }
    kh = __reduce_max_sync(0xffffffffu, kh);
    ks = __reduce_max_sync(0xffffffffu, ks);
    __shared__ unsigned redk[2 * (kDftThreads / 32)];
    if ((tid & 31) == 0) {
      redk[2 * (tid >> 5)] = kh;
      redk[2 * (tid >> 5) + 1] = ks;
    }
    __syncthreads();
    kh = redk[0];
    ks = redk[1];
    for (int w = 1; w < kDftThreads / 32; ++w) {
      kh = max(kh, redk[2 * w]);
      ks = max(ks, redk[2 * w + 1]);
    }
    // biased exponents (0: zero or subnormal; 2047: an inf or NaN entry, which must not set the
    // scale of the whole tile -- without balancing, only the transforms it enters go non-finite)
    const int bh = (int)(kh >> 20), bs = (int)(ks >> 20);
    if (bh > 0 && bs > 0 && bh < 2047 && bs < 2047) sig_e = bh - bs;
  }
  const double sig = pow2_scale(sig_e);
  for (int k = tid; k < Ld * TW; k += kDftThreads) {
    const int j = k / TW, t = k - j * TW;
    double2 v = make_double2(0.0, 0.0);
    if (t < tw_valid) {
      const int64_t idx = (o * Ld + j) * inner + off_sh[t];
      if (packed)
        v = make_double2(s.H[idx], sig * s.S[idx]);
      else if (real_in)
        v.x = Xr[idx];
      else
        v = reinterpret_cast<const double2 *>(Xc)[idx];
    }
    const int pos = (pow2 && bits > 0) ? (int)bitrev((unsigned)j, bits) : j;
    x[pos * TW + t] = v;
  }
  __syncthreads();
  if (pow2) {
    fft_columns(x, Ld, TW, tab);
    if (packed) {
      const double hs2 = 0.5 / sig;
      for (int k = tid; k < Ld * TW; k += kDftThreads) {
        const int kap = k / TW, t = k - kap * TW;
        if (t < tw_valid) {
          const int kn = kap == 0 ? 0 : Ld - kap;
          const double2 z = x[kap * TW + t], zc = x[kn * TW + t];  // Z_k, Z_-k
          const int64_t base = (o * Ld + kap) * inner;
          const double2 h = make_double2(0.5 * (z.x + zc.x), 0.5 * (z.y - zc.y));
          // (Z_k - conj Z_-k) / (2 i sigma)
          const double2 sv = make_double2(hs2 * (z.y + zc.y), -hs2 * (z.x - zc.x));
          reinterpret_cast<double2 *>(s.Hbar)[base + off_sh[t]] = h;
          reinterpret_cast<double2 *>(s.Sbar)[base + off_sh[t]] = sv;
          if (offT_sh[t] >= 0) {
            reinterpret_cast<double2 *>(s.Hbar)[base + offT_sh[t]] = make_double2(h.x, -h.y);
            reinterpret_cast<double2 *>(s.Sbar)[base + offT_sh[t]] = make_double2(sv.x, -sv.y);
          }
        }
      }
    } else {
      for (int k = tid; k < Ld * TW; k += kDftThreads) {
        const int kap = k / TW, t = k - kap * TW;
        if (t < tw_valid) {
          const int64_t base = (o * Ld + kap) * inner;
          const double2 v = x[kap * TW + t];
          reinterpret_cast<double2 *>(Xc)[base + off_sh[t]] = v;
          if (offT_sh[t] >= 0) reinterpret_cast<double2 *>(Xc)[base + offT_sh[t]] = make_double2(v.x, -v.y);
        }
      }
    }
  } else {
    for (int k = tid; k < Ld * TW; k += kDftThreads) {
      const int kap = k / TW, t = k - kap * TW;
      if (t >= tw_valid) continue;
      double re = 0.0, im = 0.0;
      int m = 0;  // (kap * j) mod Ld, advanced incrementally
      for (int j = 0; j < Ld; ++j) {
        const double2 w = tab[m], v = x[j * TW + t];
        re += w.x * v.x - w.y * v.y;
        im += w.x * v.y + w.y * v.x;
        m += kap;
        if (m >= Ld) m -= Ld;
      }
      const int64_t base = (o * Ld + kap) * inner;
      reinterpret_cast<double2 *>(Xc)[base + off_sh[t]] = make_double2(re, im);
      if (offT_sh[t] >= 0) reinterpret_cast<double2 *>(Xc)[base + offT_sh[t]] = make_double2(re, -im);
    }
  }
}

// ---- four-step DFT of long one-dimensional lattices ----------------------------------------
// For L = A B, j = B j1 + j2 and kappa = kappa1 + A kappa2 (j1, kappa1 < A; j2, kappa2 < B):
//   Xbar_kappa = sum_j2 omega_B^(j2 kappa2) [omega_L^(j2 kappa1) sum_j1 omega_A^(j1 kappa1) X_(B j1 + j2)]
// (the factorisation of F_L behind Lemma 2.2's fast transform): pass 1 transforms along j1 for
// every (j2, entry) and applies the twiddle omega_L^(j2 kappa1), writing Y[kappa1][j2]; pass 2
// transforms along j2 for every (kappa1, entry) and writes Xbar at kappa1 + A kappa2.  Every entry
// (mu, nu) of H and S is transformed (blockIdx.z: 0 H, 1 S).  A tile holds TW consecutive entries
// for all positions of one transform in shared memory: the radix-4 FFT (fft_columns) when the
// length is a power of two, the direct sum with a twiddle table otherwise.

// In-place transform of Ld positions x TW columns (x[j * TW + t]); tab[m] = omega^m.  For a power
// of two the input must have been stored bit-reversed.
__device__ void tile_transform(double2 *x, int Ld, int TW, int tw_valid, const double2 *tab, bool pow2,
                               double2 *tmp) {
  const int tid = threadIdx.x;
  if (pow2) {
    fft_columns(x, Ld, TW, tab);
    return;
  }
  // direct sum into tmp, then back
  for (int k = tid; k < Ld * TW; k += kDftThreads) {
    const int kap = k / TW, t = k - kap * TW;
    double re = 0.0, im = 0.0;
    if (t < tw_valid) {
      int m = 0;
      for (int j = 0; j < Ld; ++j) {
        const double2 w = tab[m], v = x[j * TW + t];
        re += w.x * v.x - w.y * v.y;
        im += w.x * v.y + w.y * v.x;
        m += kap;
        if (m >= Ld) m -= Ld;
      }
    }
    tmp[k] = make_double2(re, im);
  }
  __syncthreads();
  for (int k = tid; k < Ld * TW; k += kDftThreads) x[k] = tmp[k];
  __syncthreads();
}

__device__ void twiddle_table(double2 *tab, int Ld) {
  for (int m = threadIdx.x; m < Ld; m += kDftThreads) {
    double sn, cs;
    sincospi(2.0 * (double)m / (double)Ld, &sn, &cs);
    tab[m] = make_double2(cs, -sn);
  }
}

// pass: 1 (along j1, length A, then the twiddle) or 2 (along j2, length B).  Grid x: (pass 1: j2,
// pass 2: kappa1) x entry tiles; z: H / S.
__global__ void __launch_bounds__(kDftThreads) k_dft_four_step(const SysDev *__restrict__ sysv, int A, int B,
                                                               int pass) {
  const SysDev &s = *sysv;
  const int m0 = s.m0, mm = m0 * m0, L = A * B;
  const int Ld = pass == 1 ? A : B;
  const int TW = tile_width(Ld);
  const int tiles_e = (mm + TW - 1) / TW;
  const int line = blockIdx.x / tiles_e, e0 = (blockIdx.x % tiles_e) * TW;
  const int tw_valid = mm - e0 < TW ? mm - e0 : TW;
  const bool pow2 = (Ld & (Ld - 1)) == 0;
  const int bits = pow2 ? __ffs(Ld) - 1 : 0;
  extern __shared__ double sm[];
  double2 *x = reinterpret_cast<double2 *>(sm);  // [Ld][TW]
  double2 *tab = x + (size_t)Ld * TW;            // [Ld]
  double2 *tmp = tab + Ld;                       // [Ld][TW] (direct sums only)
  twiddle_table(tab, Ld);
  double2 *Y = reinterpret_cast<double2 *>(s.dftw) + (size_t)blockIdx.z * L * mm;
  for (int k = threadIdx.x; k < Ld * TW; k += kDftThreads) {
    const int j = k / TW, t = k - j * TW;
    double2 v = make_double2(0.0, 0.0);
    if (t < tw_valid) {
      if (pass == 1) {  // X_(B j + j2), real
        const double *X = blockIdx.z == 0 ? s.H : s.S;
        v.x = X[((int64_t)B * j + line) * mm + e0 + t];
      } else {  // Y[kappa1][j]
        v = Y[((int64_t)line * B + j) * mm + e0 + t];
      }
    }
    const int pos = (pow2 && bits > 0) ? (int)bitrev((unsigned)j, bits) : j;
    x[pos * TW + t] = v;
  }
  __syncthreads();
  tile_transform(x, Ld, TW, tw_valid, tab, pow2, tmp);
  for (int k = threadIdx.x; k < Ld * TW; k += kDftThreads) {
    const int kap = k / TW, t = k - kap * TW;
    if (t >= tw_valid) continue;
    double2 v = x[kap * TW + t];
    if (pass == 1) {
      // omega_L^(j2 kappa1), the phase reduced mod L in integers
      const long long ph = ((long long)line * kap) % L;
      double sn, cs;
      sincospi(2.0 * (double)ph / (double)L, &sn, &cs);
      v = make_double2(cs * v.x + sn * v.y, cs * v.y - sn * v.x);  // (cs - i sn) v
      Y[((int64_t)kap * B + line) * mm + e0 + t] = v;
    } else {
      double2 *Xc = reinterpret_cast<double2 *>(blockIdx.z == 0 ? s.Hbar : s.Sbar);
      Xc[((int64_t)line + (int64_t)A * kap) * mm + e0 + t] = v;
    }
  }
}

}  // namespace

bool dft_four_step_split(int L, int *A, int *B) {
  // the most balanced split L = A B with B <= A <= kDftTileMax
  int best = 0;
  for (int b = 1; (long long)b * b <= L; ++b)
    if (L % b == 0 && L / b <= kDftTileMax) best = b;
  if (!best) return false;
  *A = L / best;
  *B = best;
  return true;
}

// host_L: [nsys][3] lattice sizes (host copy) used to size the grid of each pass.
cudaError_t launch_dft(const SysDev *sys, int nsys, const int *host_L, int *passes,
                       cudaStream_t st) {
  if (nsys <= 0) return cudaSuccess;
  for (int s = 0; s < nsys; ++s) {
    const int *L = host_L + 4 * s;
    if (L[0] <= kDftTileMax) continue;
    int A = 0, B = 0;
    if (L[1] != 1 || L[2] != 1 || !dft_four_step_split(L[0], &A, &B)) return cudaErrorInvalidValue;
    const int m0 = L[3], mm = m0 * m0;
    for (int pass = 1; pass <= 2; ++pass) {
      const int Ld = pass == 1 ? A : B, lines = pass == 1 ? B : A;
      const int TW = tile_width(Ld);
      const bool pow2 = (Ld & (Ld - 1)) == 0;
      const size_t smem = sizeof(double2) * ((size_t)Ld * TW * (pow2 ? 1 : 2) + Ld);
      cudaError_t e = cudaFuncSetAttribute(k_dft_four_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      dim3 grid((unsigned)(lines * ((mm + TW - 1) / TW)), 1, 2);
      kmark(LHF_K_DFT, 1, st);
      k_dft_four_step<<<grid, kDftThreads, smem, st>>>(sys + s, A, B, pass);
      kmark(LHF_K_DFT, 0, st);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if (passes) ++*passes;
    }
  }
  for (int d = 2; d >= 0; --d) {
    int64_t max_tiles = 0;
    int max_Ld = 0;
    for (int s = 0; s < nsys; ++s) {
      const int *L = host_L + 4 * s;  // L0, L1, L2, m0
      if (L[0] > kDftTileMax) continue;  // four-step route above
      const bool all_one = (L[0] == 1 && L[1] == 1 && L[2] == 1);
      if (!(L[d] > 1 || (d == 0 && all_one))) continue;
      int last = 0;
      for (int q = 0; q < 3; ++q)
        if (L[q] > 1) {
          last = q;
          break;
        }
      int64_t items = (d == last) ? (int64_t)L[3] * (L[3] + 1) / 2 : (int64_t)L[3] * L[3];
      for (int q = d + 1; q < 3; ++q) items *= L[q];
      int64_t outer = 1;
      for (int q = 0; q < d; ++q) outer *= L[q];
      const int TW = pass_tile_width(L[d]);
      const int64_t tiles = outer * ((items + TW - 1) / TW);
      if (tiles > max_tiles) max_tiles = tiles;
      if (L[d] > max_Ld) max_Ld = L[d];
    }
    if (max_tiles == 0) continue;
    // shared memory: the largest Ld fixes both TW and the table
    size_t smem = 0;
    for (int s = 0; s < nsys; ++s) {
      const int *L = host_L + 4 * s;
      if (L[0] > kDftTileMax) continue;
      if (!(L[d] > 1 || (d == 0 && L[0] == 1 && L[1] == 1 && L[2] == 1))) continue;
      const size_t need = pass_smem_bytes(L[d]);
      if (need > smem) smem = need;
    }
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_dft_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)max_tiles, nsys, 2);
    kmark(LHF_K_DFT, 1, st);
    k_dft_pass<<<grid, kDftThreads, smem, st>>>(sys, d);
    kmark(LHF_K_DFT, 0, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (passes) ++*passes;
  }
  return cudaSuccess;
}

}  // namespace lhf
