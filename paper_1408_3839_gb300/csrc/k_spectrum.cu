// k_spectrum.cu -- energy per cell of the lowest states of a computed spectrum (Sec. 5: the
// relaxation of the average energy per unit cell of a (L,1,1) chain with L, open and periodic).
//
// The spectrum of the lattice matrix is the union of the k-point spectra (Prop. 6.1); that of an
// open box is its dense pencil's.  For each spectrum the kernel selects the n_low smallest values
// of that set and returns their sum divided by the number of cells, and the largest selected
// value.  Selection is an exact radix select on an order-preserving 64-bit key of each double:
// eight passes of one byte, each a histogram of the candidates that agree with the key prefix
// chosen so far; no sort of the spectrum, and the result does not depend on the order in which
// the k-points are stored.  The sum over the values below the selected key is taken in a fixed
// order (strided per-thread sums, then a fixed shuffle tree), so repeated calls agree bit for bit;
// the ties at the selected key enter as count x value.  One CTA per spectrum.
#include "lhf_internal.cuh"

namespace lhf {
namespace {

constexpr int kSelThreads = 512;
constexpr int kSelWarps = kSelThreads / 32;
constexpr unsigned long long kSign = 0x8000000000000000ull;

// x < y  <=>  order_key(x) < order_key(y) for non-NaN doubles (-0 sorts just below +0).
__device__ __forceinline__ unsigned long long order_key(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return (u & kSign) ? ~u : (u | kSign);
}

__device__ __forceinline__ double key_value(unsigned long long k) {
  return __longlong_as_double((long long)((k & kSign) ? (k ^ kSign) : ~k));
}

__global__ void __launch_bounds__(kSelThreads) k_cell_energy(const double *__restrict__ eig,
                                                             const SpectrumSeg *__restrict__ seg,
                                                             double *__restrict__ energy,
                                                             double *__restrict__ level) {
  __shared__ unsigned hist[kSelWarps][256];
  __shared__ unsigned long long s_prefix;
  __shared__ unsigned s_rank;
  __shared__ double red[kSelWarps];
  const SpectrumSeg g = seg[blockIdx.x];
  const double *e = eig + g.off;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long prefix = 0, mask = 0;
  unsigned rank = (unsigned)g.n_low;  // 1-based rank of the wanted value among the candidates
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < kSelWarps * 256; i += kSelThreads) (&hist[0][0])[i] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < g.cnt; i += kSelThreads) {
      const unsigned long long k = order_key(e[i]);
      if ((k & mask) == prefix) atomicAdd(&hist[warp][(unsigned)(k >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 256) {  // per-bin totals over the warps' histograms, kept in warp 0's row
      unsigned t = 0;
      for (int w = 0; w < kSelWarps; ++w) t += hist[w][threadIdx.x];
      hist[0][threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned below = 0;
      int b = 0;
      for (; b < 255; ++b) {
        if (below + hist[0][b] >= rank) break;
        below += hist[0][b];
      }
      s_prefix = prefix | ((unsigned long long)b << shift);
      s_rank = rank - below;
    }
    __syncthreads();
    prefix = s_prefix;
    rank = s_rank;
    mask |= 0xffull << shift;
  }
  // prefix: the key of the n_low-th smallest value; rank: how many of its copies are selected.
  double acc = 0.0;
  for (int i = threadIdx.x; i < g.cnt; i += kSelThreads) {
    const double x = e[i];
    if (order_key(x) < prefix) acc += x;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < kSelWarps; ++w) sum += red[w];
    const double top = key_value(prefix);
    energy[blockIdx.x] = (sum + (double)rank * top) / g.cells;
    if (level) level[blockIdx.x] = top;
  }
}

// Extrapolation of the lattice sum to the limit (the regularisation of Sec. 4.1): spectra of one
// lattice computed with nK image windows K_k, fitted per value to
//   lambda(K) = A + B ln K + C / K
// (least squares through the normal equations; two windows fit A + B ln K), thread per value.
// For a chain the far images add a potential that is constant over the cell, -(2 Z / b) sum 1/k,
// so B tends to -2 Z_cell / b and A is the finite part.  Non-finite inputs give non-finite output.
__global__ void k_lattice_extrapolate(const double *__restrict__ eig, const double *__restrict__ K, int nK, int64_t n,
                                      double *A, double *B) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double y[kMaxExtrapolationWindows];
  bool fin = true;
  for (int k = 0; k < nK; ++k) {
    y[k] = eig[(int64_t)k * n + i];
    if (!isfinite(y[k])) fin = false;
  }
  if (!fin) {
    A[i] = y[0] + y[nK - 1];  // inf or NaN, as the inputs
    if (B) B[i] = A[i];
    return;
  }
  const int nb = nK >= 3 ? 3 : 2;
  double M[3][3] = {{0.0}}, r[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < nK; ++k) {
    const double x[3] = {1.0, log(K[k]), 1.0 / K[k]};
    for (int a = 0; a < nb; ++a) {
      r[a] += x[a] * y[k];
      for (int b = 0; b < nb; ++b) M[a][b] += x[a] * x[b];
    }
  }
  double a0, b0;
  if (nb == 2) {
    const double det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
    a0 = (r[0] * M[1][1] - M[0][1] * r[1]) / det;
    b0 = (M[0][0] * r[1] - M[1][0] * r[0]) / det;
  } else {
    const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                       M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                       M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    a0 = (r[0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (r[1] * M[2][2] - M[1][2] * r[2]) +
          M[0][2] * (r[1] * M[2][1] - M[1][1] * r[2])) / det;
    b0 = (M[0][0] * (r[1] * M[2][2] - M[1][2] * r[2]) - r[0] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
          M[0][2] * (M[1][0] * r[2] - r[1] * M[2][0])) / det;
  }
  A[i] = a0;
  if (B) B[i] = b0;
}

}  // namespace

cudaError_t launch_lattice_extrapolate(const double *eig, const double *K, int nK, long long n, double *A, double *B,
                                       cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_lattice_extrapolate<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(eig, K, nK, n, A, B);
  return cudaGetLastError();
}

cudaError_t launch_cell_energy(const double *eig, const SpectrumSeg *seg, int nseg, double *energy, double *level,
                               cudaStream_t st) {
  k_cell_energy<<<nseg, kSelThreads, 0, st>>>(eig, seg, energy, level);
  return cudaGetLastError();
}

}  // namespace lhf
