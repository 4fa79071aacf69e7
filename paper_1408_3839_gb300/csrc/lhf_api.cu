// lhf_api.cu -- the C ABI of liblhf: descriptor validation, per-system layout (overlap window,
// workspace offsets), workspace management and the launch sequence of the path
//   a1 basis -> a2 potential -> a3/a4 Grams -> a5 rank sum (+ a6 zero fill) -> a7 DFT -> a8 eig.
// Host code only prepares descriptors and launches; every arithmetic step of the path runs in
// the kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <unordered_map>
#include <set>
#include <string>
#include <vector>

#include "lhf_internal.cuh"

using lhf::DirDev;
using lhf::SysDev;

namespace lhf {
thread_local KernelClock kclock = {nullptr, nullptr};
}

namespace {

struct HostSystem {
  int L[3] = {1, 1, 1};
  double b[3] = {1, 1, 1};
  int periodic[3] = {0, 0, 0};
  int K[3] = {1, 1, 1};
  int M0 = 0;
  std::vector<double> Z, a, zcell;
  int m0 = 0;
  std::vector<int> kind;
  std::vector<double> alpha, centre;
  double rho = 40.0;
  int n[3] = {1, 1, 1}, nc[3] = {1, 1, 1};
  double h[3] = {1, 1, 1}, x0[3] = {0, 0, 0}, cell0[3] = {0, 0, 0};
  int R = 0;
  double u0 = 0, du = 0;
};

// Sizes of the per-system workspace regions (doubles) and launch extents.
struct Plan {
  SysDev sd;
  size_t ws = 0;       // doubles of G, V, C and the overlap norms s0
  size_t s0_off = 0;   // offset of s0 [m0]
  bool mixed = false;  // digit planes for the tensor-core route allocated
  size_t blocks_doubles = 0;  // nblocks * m0^2
  int basis_items = 0 /* rows */, pot_rows = 0, gram_blocks = 0, rank_items = 0 /* blocks */, rank_ctas = 0;
  int nv_max = 0;
  // open box: direction-0 factor rows, widest product row, zcell and dense-solver regions
  int box_items = 0, box_width = 0;
  long long mirror_items = 0;  // window-block elements filled from their mirrors
  size_t zcell_off = 0, dense_off = 0;
  size_t tri_off = 0;  // tridiagonal scratch of the k-point solves (periodic)
  size_t evs_off = 0;  // per-k-point matrix scratch of the k-point solves (periodic)
  size_t dft_off = 0;  // four-step DFT scratch of a long chain (0: none)
  size_t rank_smem = 0;  // shared memory of the rank reduction (0: not reduced)
  std::vector<double> zcell;  // host copy of the per-cell charges (box)
};

constexpr size_t kAlign = 32;  // doubles (256 bytes)
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool finite(double x) { return isfinite(x) != 0; }

}  // namespace

struct lhf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  bool has_lat = false, has_basis = false, has_grid = false;
  HostSystem cur;
  double *ws = nullptr;
  size_t ws_cap = 0;  // doubles
  SysDev *d_sys = nullptr;
  size_t d_sys_cap = 0;
  SysDev *h_sys = nullptr;  // pinned staging
  size_t h_sys_cap = 0;
  cudaEvent_t upload_done = nullptr;
  // the mixed route's potential runs on a side stream, beside the basis samples and the fold
  // (they do not depend on it): forked after the upload, joined before its digit planes
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  bool join_pending = false;
  unsigned *d_flags = nullptr;
  unsigned long long *d_counters = nullptr;  // [0] Jacobi sweeps, [1] matrices, [2] canonical route
  double *d_zcell = nullptr;
  size_t zcell_cap = 0;
  double *d_out = nullptr;  // device staging of lhf_bloch_spectra_host
  size_t out_cap = 0;
  void *tc_buf = nullptr;   // tensor maps and job list of the tensor-core Gram (device)
  void *tc_host = nullptr;  // their pinned staging copy
  size_t tc_cap = 0;
  cudaEvent_t tc_copied = nullptr;  // the staging copy has been consumed
  // while a graph is captured: its prepared tensor-core argument buffer (device)
  const void *graph_tc = nullptr;
  int graph_tc_jobs = 0;
  size_t graph_tc_off = 0;
  std::vector<int> host_L;
  // graphs created from this context (detached, not freed, when the context is destroyed first)
  std::set<lhf_graph *> graphs;
  // failure detection: bound of the dense solver's grid-barrier waits, a one-shot injected
  // barrier stall (test), and a cap on the workspace bytes (0: none)
  double rank_eps = 0.0;  // rank reduction of one-dimensional lattices (FP64 route); 0: off
  long long wait_cycles = lhf::kDefaultWaitCycles;
  bool stall_next = false;
  size_t ws_limit = 0;
  // solved k-points (one per conjugate pair) per lattice shape, on the device
  std::map<std::array<int, 3>, std::pair<int *, int>> klists;
  // plans of the batched entry points by descriptor content (cached_plan)
  std::unordered_map<std::string, Plan> plan_cache;
  // launch-shape autotuner of the k-point eigensolver: per (m0, tridiagonal route, log2 of the
  // solved matrices) the fastest k_eig warps per CTA and tridiagonal threads per CTA, timed on
  // the first batch of that class (outside graph capture); results do not depend on the shape
  bool autotune = true;
  bool capturing = false;
  std::map<std::array<int, 3>, std::array<int, 2>> eig_tune;
  int last_eig_warps = 4, last_tri_threads = 128;
  // live stage timing
  bool prof = false;
  struct Mark {
    int stage;
    cudaEvent_t a, b;
    int kernels;  // kernel launches (or copies/fills) inside the bracket
  };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> pool;
  Mark open_mark{-1, nullptr, nullptr, 0};
  // per-kernel marks (Mark::stage holds the kernel id, Mark::kernels = 1)
  std::vector<Mark> kmarks;
  Mark open_kmark{-1, nullptr, nullptr, 0};

  static void kernel_mark(void *owner, int kernel, int begin, cudaStream_t st) {
    lhf_ctx *c = static_cast<lhf_ctx *>(owner);
    if (begin) {
      c->open_kmark = {kernel, c->take_event(), c->take_event(), 1};
      if (c->open_kmark.a) cudaEventRecord(c->open_kmark.a, st);
    } else if (c->open_kmark.stage == kernel) {
      if (c->open_kmark.b) cudaEventRecord(c->open_kmark.b, st);
      if (c->open_kmark.a && c->open_kmark.b) c->kmarks.push_back(c->open_kmark);
      c->open_kmark = {-1, nullptr, nullptr, 0};
    }
  }

  cudaEvent_t take_event() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }
  void begin(int stage, cudaStream_t st = nullptr) {
    if (!prof) return;
    open_mark = {stage, take_event(), take_event(), 0};
    if (open_mark.a) cudaEventRecord(open_mark.a, st ? st : stream);
    lhf::kclock = {this, &lhf_ctx::kernel_mark};
  }
  void end(int kernels = 1, cudaStream_t st = nullptr) {
    lhf::kclock = {nullptr, nullptr};
    if (!prof || open_mark.stage < 0) return;
    if (open_mark.b) cudaEventRecord(open_mark.b, st ? st : stream);
    open_mark.kernels = kernels;
    if (open_mark.a && open_mark.b) marks.push_back(open_mark);
    open_mark = {-1, nullptr, nullptr, 0};
  }

  lhf_status fail(lhf_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    err = buf;
    return st;
  }
  lhf_status cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return LHF_OK;
    return fail(LHF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  }
  // the main stream waits for the side stream's work (a no-op when nothing was forked)
  lhf_status join() {
    if (!join_pending) return LHF_OK;
    join_pending = false;
    return cuda(cudaStreamWaitEvent(stream, join_ev, 0), "cudaStreamWaitEvent");
  }
};

struct lhf_graph {
  lhf_ctx *ctx = nullptr;
  double *ws = nullptr;        // the graph's own workspace (factors and internal blocks)
  SysDev *d_sys = nullptr;     // its descriptors
  void *tc_dev = nullptr;      // tensor-core maps and jobs (LHF_MIXED)
  int tc_jobs = 0;
  size_t tc_off = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int nsys = 0;
};

namespace {

// ------------------------------------------------------------------------------------------
// validation

lhf_status check_lattice(lhf_ctx *c, const lhf_lattice_desc *d) {
  if (!d) return c->fail(LHF_ERR_ARG, "lattice descriptor is NULL");
  for (int l = 0; l < 3; ++l) {
    // up to kDftTileMax per direction; a one-dimensional lattice up to kDftMaxL1 cells
    const int lmax = (l == 0 && d->L[1] == 1 && d->L[2] == 1) ? lhf::kDftMaxL1 : lhf::kDftTileMax;
    if (d->L[l] < 1 || d->L[l] > lmax) return c->fail(LHF_ERR_ARG, "L[%d] = %d outside [1, %d]", l, d->L[l], lmax);
    if (!(d->b[l] > 0) || !finite(d->b[l])) return c->fail(LHF_ERR_ARG, "b[%d] must be positive", l);
    if (d->periodic[l] != 0 && d->periodic[l] != 1) return c->fail(LHF_ERR_ARG, "periodic[%d] must be 0 or 1", l);
    if (d->periodic[l] && (d->K_sum[l] < 1 || d->K_sum[l] > 1 << 20))
      return c->fail(LHF_ERR_ARG, "K_sum[%d] = %d must be >= 1", l, d->K_sum[l]);
  }
  if (d->M0 < 1 || d->M0 > LHF_MAX_NUCLEI) return c->fail(LHF_ERR_ARG, "M0 = %d outside [1, %d]", d->M0, LHF_MAX_NUCLEI);
  if (!d->Z || !d->a) return c->fail(LHF_ERR_ARG, "Z and a must be given");
  for (int nu = 0; nu < d->M0; ++nu) {
    if (!(d->Z[nu] > 0) || !finite(d->Z[nu])) return c->fail(LHF_ERR_ARG, "Z[%d] must be positive", nu);
    for (int l = 0; l < 3; ++l)
      if (!finite(d->a[3 * nu + l])) return c->fail(LHF_ERR_ARG, "a[%d][%d] not finite", nu, l);
  }
  if (d->Z_cell) {
    if (d->L[1] != 1 || d->L[2] != 1 || d->periodic[0])
      return c->fail(LHF_ERR_UNSUPPORTED, "per-cell charges need an open box with lattice direction 0 only");
    for (int k = 0; k < d->L[0] * d->M0; ++k)
      if (!(d->Z_cell[k] >= 0) || !finite(d->Z_cell[k])) return c->fail(LHF_ERR_ARG, "Z_cell[%d] must be >= 0", k);
  }
  return LHF_OK;
}

lhf_status check_basis(lhf_ctx *c, const lhf_basis_desc *d) {
  if (!d) return c->fail(LHF_ERR_ARG, "basis descriptor is NULL");
  if (d->m0 < 1 || d->m0 > LHF_MAX_M0) return c->fail(LHF_ERR_ARG, "m0 = %d outside [1, %d]", d->m0, LHF_MAX_M0);
  if (!d->kind || !d->alpha || !d->centre) return c->fail(LHF_ERR_ARG, "kind, alpha and centre must be given");
  if (!(d->rho > 0) || !finite(d->rho)) return c->fail(LHF_ERR_ARG, "rho must be positive");
  for (int mu = 0; mu < d->m0; ++mu) {
    if (d->kind[mu] < 0 || d->kind[mu] > 3) return c->fail(LHF_ERR_ARG, "kind[%d] = %d outside [0, 3]", mu, d->kind[mu]);
    if (!(d->alpha[mu] > 0) || !finite(d->alpha[mu])) return c->fail(LHF_ERR_ARG, "alpha[%d] must be positive", mu);
    for (int l = 0; l < 3; ++l)
      if (!finite(d->centre[3 * mu + l])) return c->fail(LHF_ERR_ARG, "centre[%d][%d] not finite", mu, l);
  }
  return LHF_OK;
}

lhf_status check_grid(lhf_ctx *c, const lhf_grid_desc *d) {
  if (!d) return c->fail(LHF_ERR_ARG, "grid descriptor is NULL");
  for (int l = 0; l < 3; ++l) {
    if (d->n[l] < 1 || d->n[l] > (1 << 24)) return c->fail(LHF_ERR_ARG, "n[%d] = %d invalid", l, d->n[l]);
    if (d->n_cell[l] < 1) return c->fail(LHF_ERR_ARG, "n_cell[%d] = %d invalid", l, d->n_cell[l]);
    if (!(d->h[l] > 0) || !finite(d->h[l])) return c->fail(LHF_ERR_ARG, "h[%d] must be positive", l);
    if (!finite(d->x0[l]) || !finite(d->cell0[l])) return c->fail(LHF_ERR_ARG, "x0/cell0[%d] not finite", l);
  }
  if (d->R < 1 || d->R > LHF_MAX_R) return c->fail(LHF_ERR_ARG, "R = %d outside [1, %d]", d->R, LHF_MAX_R);
  if (!(d->du > 0) || !finite(d->du) || !finite(d->u0)) return c->fail(LHF_ERR_ARG, "sinc parameters invalid");
  return LHF_OK;
}

void copy_lattice(HostSystem &s, const lhf_lattice_desc *d) {
  for (int l = 0; l < 3; ++l) {
    s.L[l] = d->L[l];
    s.b[l] = d->b[l];
    s.periodic[l] = d->periodic[l];
    s.K[l] = d->periodic[l] ? d->K_sum[l] : 1;
  }
  s.M0 = d->M0;
  s.Z.assign(d->Z, d->Z + d->M0);
  s.a.assign(d->a, d->a + 3 * d->M0);
  if (d->Z_cell)
    s.zcell.assign(d->Z_cell, d->Z_cell + (size_t)d->L[0] * d->M0);
  else
    s.zcell.clear();
}

void copy_basis(HostSystem &s, const lhf_basis_desc *d) {
  s.m0 = d->m0;
  s.kind.assign(d->kind, d->kind + d->m0);
  s.alpha.assign(d->alpha, d->alpha + d->m0);
  s.centre.assign(d->centre, d->centre + 3 * d->m0);
  s.rho = d->rho;
}

void copy_grid(HostSystem &s, const lhf_grid_desc *d) {
  for (int l = 0; l < 3; ++l) {
    s.n[l] = d->n[l];
    s.nc[l] = d->n_cell[l];
    s.h[l] = d->h[l];
    s.x0[l] = d->x0[l];
    s.cell0[l] = d->cell0[l];
  }
  s.R = d->R;
  s.u0 = d->u0;
  s.du = d->du;
}

// Consistency of the three parts; fills the plan (descriptor, window, workspace sizes).
lhf_status make_plan(lhf_ctx *c, const HostSystem &s, Plan &P, bool mixed = false, bool dense_box = true) {
  SysDev &sd = P.sd;
  memset(&sd, 0, sizeof sd);
  if (s.M0 * s.R > lhf::kMaxRt) return c->fail(LHF_ERR_ARG, "M0 R = %d exceeds %d", s.M0 * s.R, lhf::kMaxRt);
  int open_lattice = 0;
  for (int l = 0; l < 3; ++l) {
    const bool lat = s.L[l] > 1 || s.periodic[l];
    if (s.periodic[l]) {
      if ((long long)s.L[l] * s.nc[l] != s.n[l])
        return c->fail(LHF_ERR_ARG, "direction %d: n = %d must equal L n_cell = %d", l, s.n[l], s.L[l] * s.nc[l]);
      if (fabs(s.nc[l] * s.h[l] - s.b[l]) > 1e-9 * s.b[l])
        return c->fail(LHF_ERR_ARG, "direction %d: n_cell h = %.17g must equal b = %.17g", l, s.nc[l] * s.h[l], s.b[l]);
      if (fabs(s.x0[l] - s.cell0[l]) > 1e-12 * s.b[l])
        return c->fail(LHF_ERR_ARG, "direction %d: periodic grid must start at cell0", l);
    } else if (lat) {
      open_lattice |= 1 << l;
      if (fabs(s.nc[l] * s.h[l] - s.b[l]) > 1e-9 * s.b[l])
        return c->fail(LHF_ERR_ARG, "direction %d: n_cell h must equal b", l);
    }
  }
  // open lattice (Sec. 3.2 box): direction 0 only, single cells across
  const bool box = open_lattice != 0;
  if (box && (open_lattice != 1 || s.L[1] != 1 || s.L[2] != 1 || s.periodic[1] || s.periodic[2]))
    return c->fail(LHF_ERR_UNSUPPORTED, "open lattices are supported along direction 0 only, as an (L,1,1) box");
  if (!s.zcell.empty() && !box) return c->fail(LHF_ERR_UNSUPPORTED, "per-cell charges need an open box");

  const int m0 = s.m0, Rt = s.M0 * s.R, mm = m0 * m0;
  sd.m0 = m0;
  sd.M0 = s.M0;
  sd.R = s.R;
  sd.Rt = Rt;
  sd.box = box ? 1 : 0;
  for (int mu = 0; mu < m0; ++mu) {
    sd.kind[mu] = s.kind[mu];
    sd.alpha[mu] = s.alpha[mu];
    for (int l = 0; l < 3; ++l) sd.centre[mu][l] = s.centre[3 * mu + l];
    sd.cut[mu] = sqrt(s.rho / s.alpha[mu]);
    sd.pnorm[mu] = sqrt(2.0 * s.alpha[mu] * exp(1.0));
  }
  for (int nu = 0; nu < s.M0; ++nu) {
    sd.Z[nu] = s.Z[nu];
    for (int l = 0; l < 3; ++l) sd.a[nu][l] = s.a[3 * nu + l];
  }
  // sinc nodes and weights (eq. (3.6)): t_q = exp(u0 + q du), w_q = 2/sqrt(pi) du t_q, the
  // nodes below u0 folded into w_0 (geometric tail)
  double w[lhf::kMaxR];
  for (int q = 0; q < s.R; ++q) {
    sd.t[q] = exp(s.u0 + q * s.du);
    w[q] = 2.0 / sqrt(M_PI) * s.du * sd.t[q];
  }
  w[0] = w[0] / (1.0 - exp(-s.du));
  for (int nu = 0; nu < s.M0; ++nu)
    for (int q = 0; q < s.R; ++q) sd.c[nu * s.R + q] = s.Z[nu] * w[q];

  size_t off = 0;
  P.basis_items = P.pot_rows = P.gram_blocks = 0;
  P.nv_max = 0;
  sd.nwin = 1;
  sd.nblocks = 1;
  for (int l = 0; l < 3; ++l) {
    DirDev &D = sd.d[l];
    D.L = s.L[l];
    D.n = s.n[l];
    D.periodic = s.periodic[l];
    D.lattice = (s.L[l] > 1 || s.periodic[l]) ? 1 : 0;
    D.nc = D.lattice ? s.nc[l] : s.n[l];
    D.nv = D.periodic ? D.nc : D.n;
    D.K = s.K[l];
    D.h = s.h[l];
    {
      const double hv[3] = {1.0 / D.h, D.h, D.h / 6.0};
      for (int k = 0; k < 3; ++k) {
        const float hi = (float)hv[k];
        D.p1h[2 * k] = hi;
        D.p1h[2 * k + 1] = (float)(hv[k] - (double)hi);
      }
    }
    D.x0 = s.x0[l];
    D.cell0 = s.cell0[l];
    D.b = s.b[l];
    D.invP = 1.0 / (s.L[l] * s.b[l]);
    // open box direction 0: the cell-0 basis copies are sampled (L0 - 1) n_c nodes further to
    // the left, so that the copy in cell p is the plain offset p n_c
    D.gext = (box && l == 0) ? (s.L[0] - 1) * D.nc : 0;
    // support cells of each cell-0 basis copy, dilated by one node for the P1 cross terms
    for (int mu = 0; mu < m0; ++mu) {
      if (D.lattice) {
        const double A = s.centre[3 * mu + l], cut = sd.cut[mu];
        sd.cell_lo[l][mu] = (int)floor((A - cut - D.h - D.cell0) / D.b);
        sd.cell_hi[l][mu] = (int)floor((A + cut + D.h - D.cell0) / D.b);
      } else {
        sd.cell_lo[l][mu] = sd.cell_hi[l][mu] = 0;
      }
      // samples e (node i = e - gext, x = x0 + (i + 1/2) h) with |x - A| <= cut, widened by two
      // nodes per side
      const double A = s.centre[3 * mu + l], cut = sd.cut[mu];
      const double flo = floor((A - cut - D.x0) / D.h - 0.5) + D.gext - 2.0;
      const double fhi = ceil((A + cut - D.x0) / D.h - 0.5) + D.gext + 2.0;
      if (D.periodic) {
        if (fhi - flo + 1.0 >= (double)D.n) {
          sd.node_lo[l][mu] = 0;
          sd.node_span[l][mu] = D.n;
        } else {
          const long long lo = (long long)flo;
          sd.node_lo[l][mu] = (int)(((lo % D.n) + D.n) % D.n);
          sd.node_span[l][mu] = (int)(fhi - flo) + 1;
          sd.node_wrap[l][mu] = (int)((lo - sd.node_lo[l][mu]) / D.n);
        }
      } else {
        const double nx = (double)D.n + D.gext;
        const double lo = std::max(flo, 0.0), hi = std::min(fhi, nx - 1.0);
        sd.node_lo[l][mu] = (int)std::min(lo, nx);
        sd.node_span[l][mu] = hi >= lo ? (int)(hi - lo) + 1 : 0;
      }
    }
    // overlap window of displacements j: blocks outside are exact zeros
    if (D.periodic) {
      int jmin = 1 << 30, jmax = -(1 << 30);
      for (int mu = 0; mu < m0; ++mu)
        for (int nu = 0; nu < m0; ++nu) {
          jmin = std::min(jmin, sd.cell_lo[l][nu] - sd.cell_hi[l][mu]);
          jmax = std::max(jmax, sd.cell_hi[l][nu] - sd.cell_lo[l][mu]);
        }
      if ((long long)jmax - jmin + 1 >= D.L) {
        D.jlo = 0;
        D.J = D.L;
      } else {
        D.jlo = jmin;
        D.J = jmax - jmin + 1;
      }
    } else if (box && l == 0) {
      // cell pairs (p, p + d) whose supports can meet; the factors live in the box region
      int dmin = 1 << 30, dmax = -(1 << 30);
      for (int mu = 0; mu < m0; ++mu)
        for (int nu = 0; nu < m0; ++nu) {
          dmin = std::min(dmin, sd.cell_lo[l][mu] - sd.cell_hi[l][nu]);
          dmax = std::max(dmax, sd.cell_hi[l][mu] - sd.cell_lo[l][nu]);
        }
      dmin = std::max(dmin, 1 - D.L);
      dmax = std::min(dmax, D.L - 1);
      sd.bjlo = dmin;
      sd.bJ = dmax - dmin + 1;
      D.jlo = 0;
      D.J = 0;  // no translation-invariant window
    } else {
      D.jlo = 0;
      D.J = 1;
    }
    // blocks contracted: j >= 0 of the (symmetric) window; the rest are mirrors
    if (D.J == 0) {
      D.cw0 = 0;
      D.Jc = 0;
    } else if (D.J == D.L && D.jlo == 0) {
      D.cw0 = 0;
      D.Jc = D.L / 2 + 1;
    } else {
      D.cw0 = -D.jlo;
      D.Jc = D.J - D.cw0;
      if (D.jlo > 0 || D.J != 2 * D.cw0 + 1) return c->fail(LHF_ERR_ARG, "direction %d: asymmetric window", l);
    }
    P.mirror_items += (long long)(D.J - D.Jc) * (Rt + 2) * mm;
    if (!(box && l == 0)) sd.nwin *= D.J;
    sd.nblocks *= D.L;
    P.gram_blocks += D.Jc * m0;
    if (D.J > 0) P.nv_max = std::max(P.nv_max, D.nv);  // rows contracted by the Gram kernels
  }
  for (int l = 0; l < 3; ++l) {
    sd.d[l].offGD = sd.d[l].offRM = -1;
    sd.d[l].rows_c = 0;
    sd.d[l].offG = (int64_t)off;
    off = align_up(off + (size_t)m0 * (sd.d[l].n + sd.d[l].gext));
    if (sd.d[l].gext == 0 && sd.d[l].J > 0) {  // differences for the P1 forms of the Gram kernels
      sd.d[l].offD = (int64_t)off;
      off = align_up(off + (size_t)m0 * sd.d[l].n);
    } else {
      sd.d[l].offD = -1;
    }
  }
  for (int l = 0; l < 3; ++l) {
    sd.d[l].offV = (int64_t)off;
    off = align_up(off + (size_t)Rt * sd.d[l].nv);
  }
  sd.offPC = (int64_t)off;
  off = align_up(off + (size_t)3 * s.R * lhf::kPotConst);
  for (int l = 0; l < 3; ++l) {
    sd.d[l].offC = (int64_t)off;
    off = align_up(off + (size_t)sd.d[l].J * (Rt + 2) * mm);
  }
  P.s0_off = off;
  off = align_up(off + (size_t)m0);
  if (box) {
    sd.offCb = (int64_t)off;
    off = align_up(off + (size_t)s.L[0] * sd.bJ * (Rt + 2) * mm);
    P.box_items = sd.bJ * mm;
    for (int mu = 0; mu < m0; ++mu) P.box_width = std::max(P.box_width, sd.node_span[0][mu]);
    if (lhf::box_gram_smem_bytes(P.box_width) > 200 * 1024)
      return c->fail(LHF_ERR_UNSUPPORTED, "open box: a basis function spans %d nodes (limit 12800)", P.box_width);
    P.zcell = s.zcell;
    P.zcell_off = off;
    off = align_up(off + (size_t)s.L[0] * s.M0);
  }
  for (int l = 0; l < 3; ++l) {
    DirDev &D = sd.d[l];
    D.Kpad = (D.nv + 63) / 64 * 64;
    if (mixed && !box) {
      const size_t rows = (size_t)D.Jc * mm;
      if (D.J > 0 && D.offD >= 0) {
        // the samples and differences as FP32 pairs, interleaved (16 bytes a node: two doubles)
        D.offGD = (int64_t)off;
        off = align_up(off + (size_t)2 * m0 * D.n);
      }
      D.offA = (int64_t)off;
      off = align_up(off + (lhf::kSlices * rows * D.Kpad * 2 + 7) / 8);
      D.offB = (int64_t)off;
      off = align_up(off + (lhf::kSlices * (size_t)Rt * D.Kpad * 2 + 7) / 8);
      D.offRE = (int64_t)off;
      off = align_up(off + (rows * 4 + 7) / 8);
      D.offRM = (int64_t)off;
      off = align_up(off + (2 * rows * 4 + 7) / 8);
      D.rows_c = 0;
      for (int jc = 0; jc < D.Jc; ++jc)
        for (int mu = 0; mu < m0; ++mu)
          for (int nu = 0; nu < m0; ++nu) D.rows_c += lhf::gram_row_cells(sd, l, D.jlo + D.cw0 + jc, mu, nu) > 0;
      D.offCE = (int64_t)off;
      off = align_up(off + ((size_t)Rt * 4 + 7) / 8);
      if (D.Kpad > 448) return c->fail(LHF_ERR_UNSUPPORTED, "mixed precision: direction %d has %d nodes per contraction (limit 448)", l, D.nv);
    }
  }
  P.mixed = mixed && !box;  // the box's Grams run in FP64 in both modes
  sd.eig_df = P.mixed ? 1 : 0;
  if (box && !dense_box) {  // banded matrices and an iterative solver (lhf_box_lowest_eigenvalues)
    P.blocks_doubles = 0;
    P.rank_items = 0;
  } else if (box) {
    const size_t Nb = (size_t)m0 * s.L[0];
    if (Nb > 8192) return c->fail(LHF_ERR_UNSUPPORTED, "open box: N_b = %zu above 8192", Nb);
    P.dense_off = off;
    off = align_up(off + lhf::dense_eig_workspace_doubles((int)Nb));
    P.blocks_doubles = align_up(Nb * Nb);
    P.rank_items = 0;
  } else {
    P.tri_off = off;  // one slot per k-point bounds the solved ones
    off = align_up(off + (size_t)sd.nblocks * (2 * m0 + 1));
    P.evs_off = off;
    off = align_up(off + (size_t)sd.nblocks * 2 * mm);
    if (s.L[0] > lhf::kDftTileMax) {  // scratch of the four-step DFT
      int A = 0, B = 0;
      if (!lhf::dft_four_step_split(s.L[0], &A, &B))
        return c->fail(LHF_ERR_UNSUPPORTED, "L = %d has no split A B with A, B <= %d for the DFT", s.L[0], lhf::kDftTileMax);
      P.dft_off = off;
      off = align_up(off + (size_t)4 * s.L[0] * mm);
    }
    P.blocks_doubles = align_up((size_t)sd.nblocks * mm);
    P.rank_items = sd.nblocks;  // zeros outside the window: CTA per block
    P.rank_ctas = lhf::ranksum_ctas(sd);
    if ((size_t)sd.nblocks * mm > (size_t)1 << 31) return c->fail(LHF_ERR_UNSUPPORTED, "too many block entries");
  }
  // rank reduction: periodic (L,1,1) lattices with open single-cell transverse directions, FP64
  sd.rank_eps = 0.0;
  sd.offRR = 0;
  if (c->rank_eps > 0.0 && !box && !mixed && s.periodic[0] && !s.periodic[1] && !s.periodic[2] && s.L[1] == 1 &&
      s.L[2] == 1 && Rt <= lhf::kRankReduceMaxRt && lhf::rank_reduce_smem_bytes(Rt, sd.d[0].nv) <= 200 * 1024) {
    sd.rank_eps = c->rank_eps;
    sd.offRR = (int64_t)off;
    off = align_up(off + 8 + (size_t)(Rt + 4) * mm);
    P.rank_smem = lhf::rank_reduce_smem_bytes(Rt, sd.d[0].nv);
  }
  P.basis_items = lhf::basis_ctas(sd);  // one CTA per (direction, function, chunk of samples)
  P.pot_rows = lhf::potential_ctas(sd);  // one CTA per (direction, rank term, chunk of cells)
  P.ws = off;
  return LHF_OK;
}

// The batched entry points' plans, memoized by the validated descriptor's content with the
// precision and the context's rank-reduction setting (make_plan reads nothing else): building a
// plan (overlap windows, workspace layout, the count of overlapping Gram rows) costs ~13 us per
// tube_256 system, the largest host share of a 64-system call, and repeats identically for
// repeated lattices.  Bounded (a plan is ~10 KB): the cache is cleared when it reaches 1024 plans.
std::string plan_key(const HostSystem &s, bool mixed, double rank_eps) {
  std::string k;
  auto put = [&k](const void *p, size_t n) { k.append(static_cast<const char *>(p), n); };
  auto putv = [&put](const auto &v) {
    const size_t n = v.size();
    put(&n, sizeof n);
    if (n) put(v.data(), n * sizeof(v[0]));
  };
  put(s.L, sizeof s.L);
  put(s.b, sizeof s.b);
  put(s.periodic, sizeof s.periodic);
  put(s.K, sizeof s.K);
  put(&s.M0, sizeof s.M0);
  putv(s.Z);
  putv(s.a);
  putv(s.zcell);
  put(&s.m0, sizeof s.m0);
  putv(s.kind);
  putv(s.alpha);
  putv(s.centre);
  put(&s.rho, sizeof s.rho);
  put(s.n, sizeof s.n);
  put(s.nc, sizeof s.nc);
  put(s.h, sizeof s.h);
  put(s.x0, sizeof s.x0);
  put(s.cell0, sizeof s.cell0);
  put(&s.R, sizeof s.R);
  put(&s.u0, sizeof s.u0);
  put(&s.du, sizeof s.du);
  const char m = mixed ? 1 : 0;
  put(&m, 1);
  put(&rank_eps, sizeof rank_eps);
  return k;
}

lhf_status cached_plan(lhf_ctx *c, const HostSystem &hs, Plan &P, bool mixed) {
  std::string key = plan_key(hs, mixed, c->rank_eps);
  const auto it = c->plan_cache.find(key);
  if (it != c->plan_cache.end()) {
    P = it->second;
    return LHF_OK;
  }
  const lhf_status st = make_plan(c, hs, P, mixed);
  if (st != LHF_OK) return st;
  if (c->plan_cache.size() >= 1024) c->plan_cache.clear();
  c->plan_cache.emplace(std::move(key), P);
  return LHF_OK;
}

lhf_status current_plan(lhf_ctx *c, Plan &P, bool mixed = false) {
  if (!c->has_lat || !c->has_basis || !c->has_grid)
    return c->fail(LHF_ERR_STATE, "lattice, basis and grid setup must precede this call");
  return make_plan(c, c->cur, P, mixed);
}

lhf_status ensure_ws(lhf_ctx *c, size_t doubles) {
  if (doubles <= c->ws_cap) return LHF_OK;
  if (c->ws_limit && doubles * sizeof(double) > c->ws_limit)
    return c->fail(LHF_ERR_NOMEM, "workspace of %zu bytes exceeds the context's limit of %zu bytes",
                   doubles * sizeof(double), c->ws_limit);
  lhf_status st = c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (st != LHF_OK) return st;
  if (c->ws) cudaFree(c->ws);
  c->ws = nullptr;
  c->ws_cap = 0;
  size_t want = std::max(doubles, c->ws_cap + c->ws_cap / 4);
  if (c->ws_limit) want = std::min(want, std::max(doubles, c->ws_limit / sizeof(double)));
  cudaError_t e = cudaMalloc(&c->ws, want * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&c->ws, doubles * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return c->fail(LHF_ERR_NOMEM, "workspace of %zu bytes: %s", doubles * sizeof(double), cudaGetErrorString(e));
    }
    want = doubles;
  }
  c->ws_cap = want;
  return LHF_OK;
}

// Copy nsys descriptors to the device through the pinned staging buffer.
lhf_status upload(lhf_ctx *c, const std::vector<SysDev> &v) {
  const size_t n = v.size();
  lhf_status st;
  if (c->upload_done) {
    st = c->cuda(cudaEventSynchronize(c->upload_done), "cudaEventSynchronize");
    if (st != LHF_OK) return st;
  }
  if (n > c->h_sys_cap) {
    if (c->h_sys) cudaFreeHost(c->h_sys);
    c->h_sys = nullptr;
    st = c->cuda(cudaMallocHost(&c->h_sys, n * sizeof(SysDev)), "cudaMallocHost");
    if (st != LHF_OK) return st;
    c->h_sys_cap = n;
  }
  if (n > c->d_sys_cap) {
    st = c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (st != LHF_OK) return st;
    if (c->d_sys) cudaFree(c->d_sys);
    c->d_sys = nullptr;
    st = c->cuda(cudaMalloc(&c->d_sys, n * sizeof(SysDev)), "cudaMalloc");
    if (st != LHF_OK) return st;
    c->d_sys_cap = n;
  }
  memcpy(c->h_sys, v.data(), n * sizeof(SysDev));
  c->begin(7);
  st = c->cuda(cudaMemcpyAsync(c->d_sys, c->h_sys, n * sizeof(SysDev), cudaMemcpyHostToDevice, c->stream),
               "cudaMemcpyAsync");
  c->end();
  if (st != LHF_OK) return st;
  return c->cuda(cudaEventRecord(c->upload_done, c->stream), "cudaEventRecord");
}

int max_of(const std::vector<Plan> &ps, int Plan::*f) {
  int m = 0;
  for (const Plan &p : ps) m = std::max(m, p.*f);
  return m;
}

// a3 + a4 for the uploaded systems: FP64 contraction, or digit planes + tensor cores.  The
// window blocks with j < 0 are filled from their mirrors only with_mirror (the rank-sum kernel
// reads the mirrors itself).
lhf_status run_gram(lhf_ctx *c, const std::vector<Plan> &ps, bool with_mirror) {
  const int nsys = (int)ps.size();
  int max_m0 = 0, max_rt = 0;
  for (const Plan &p : ps) {
    max_m0 = std::max(max_m0, p.sd.m0);
    max_rt = std::max(max_rt, p.sd.Rt);
  }
  long long mirror = 0;
  if (with_mirror)
    for (const Plan &p : ps) mirror = std::max(mirror, p.mirror_items);
  // one launch per direction, each sized by that direction's rows (shared memory per CTA holds two
  // rows of n_v values for each of m0 functions: the short rows of a long periodic direction do
  // not inherit the transverse directions' footprint)
  int dir_blocks[3] = {0, 0, 0}, dir_nv[3] = {0, 0, 0};
  for (const Plan &p : ps)
    for (int l = 0; l < 3; ++l) {
      const DirDev &D = p.sd.d[l];
      if (D.Jc <= 0) continue;
      dir_blocks[l] = std::max(dir_blocks[l], D.Jc * p.sd.m0);
      dir_nv[l] = std::max(dir_nv[l], D.nv);
    }
  int gram_launches = 0;
  lhf_status st = LHF_OK;
  if (!ps[0].mixed) {
    // with a rank reduction, the transverse directions first, then the reduction (which rewrites
    // the direction-0 potential rows and the transverse factors), then direction 0
    size_t rsmem = 0;
    for (const Plan &p : ps) rsmem = std::max(rsmem, p.rank_smem);
    const int order[3] = {rsmem ? 1 : 0, rsmem ? 2 : 1, rsmem ? 0 : 2};
    c->begin(2);
    for (int o = 0; o < 3 && st == LHF_OK; ++o) {
      const int l = order[o];
      if (rsmem && l == 0) {
        st = c->cuda(lhf::launch_rank_reduce(c->d_sys, nsys, rsmem, c->stream), "rank-reduction kernel");
        ++gram_launches;
        if (st != LHF_OK) break;
      }
      if (dir_blocks[l] > 0) {
        st = c->cuda(lhf::launch_gram_fp64(c->d_sys, nsys, dir_blocks[l], max_m0, dir_nv[l], c->stream, l),
                     "Gram kernel");
        ++gram_launches;
      }
    }
    if (st == LHF_OK) st = c->cuda(lhf::launch_gram_mirror(c->d_sys, nsys, mirror, c->stream), "mirror kernel");
    c->end(gram_launches + (mirror > 0 ? 1 : 0));
    return st;
  }
  c->begin(2);
  for (int l = 0; l < 3 && st == LHF_OK; ++l)
    if (dir_blocks[l] > 0) {
      st = c->cuda(lhf::launch_gram_slices(c->d_sys, nsys, dir_blocks[l], max_m0, dir_nv[l], c->stream, l,
                                           gram_launches == 0),
                   "digit-plane kernel");
      ++gram_launches;
    }
  const lhf_status sj = c->join();  // the potential rows, for their digit planes
  if (st == LHF_OK) st = sj;
  if (st == LHF_OK) st = c->cuda(lhf::launch_vslices(c->d_sys, nsys, 3 * max_rt, c->stream), "digit-plane kernel");
  c->end(gram_launches + 1);
  if (st != LHF_OK) return st;
  if (c->graph_tc) {  // capture: the arguments were prepared and copied before the capture
    c->begin(8);
    st = c->cuda(lhf::gram_tc_launch(c->graph_tc, c->graph_tc_jobs, c->graph_tc_off, c->d_flags, c->stream),
                 "tensor-core Gram kernel");
    c->end();
    if (st != LHF_OK) return st;
    c->begin(2);
    st = c->cuda(lhf::launch_gram_mirror(c->d_sys, nsys, mirror, c->stream), "mirror kernel");
    c->end(mirror > 0 ? 1 : 0);
    return st;
  }
  std::vector<SysDev> host(nsys);
  for (int i = 0; i < nsys; ++i) host[i] = ps[i].sd;
  const size_t need = lhf::gram_tc_args_bytes(host.data(), nsys);
  // the pinned staging buffer of the previous launch must have been copied out
  st = c->cuda(cudaEventSynchronize(c->tc_copied), "cudaEventSynchronize");
  if (st != LHF_OK) return st;
  if (need > c->tc_cap) {
    st = c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (st != LHF_OK) return st;
    if (c->tc_buf) cudaFree(c->tc_buf);
    c->tc_buf = nullptr;
    if (c->tc_host) cudaFreeHost(c->tc_host);
    c->tc_host = nullptr;
    c->tc_cap = 0;
    st = c->cuda(cudaMalloc(&c->tc_buf, need), "cudaMalloc");
    if (st != LHF_OK) return st;
    st = c->cuda(cudaMallocHost(&c->tc_host, need), "cudaMallocHost");
    if (st != LHF_OK) return st;
    c->tc_cap = need;
  }
  c->begin(8);
  cudaError_t e = lhf::launch_gram_tc_impl(host.data(), nsys, c->tc_buf, c->tc_cap, c->tc_host, c->tc_cap,
                                           c->d_flags, c->stream);
  c->end();
  if (e == cudaErrorNotSupported) return c->fail(LHF_ERR_UNSUPPORTED, "shape outside the tensor-core kernel's limits");
  st = c->cuda(e, "tensor-core Gram kernel");
  if (st != LHF_OK) return st;
  c->begin(2);
  st = c->cuda(lhf::launch_gram_mirror(c->d_sys, nsys, mirror, c->stream), "mirror kernel");
  c->end(mirror > 0 ? 1 : 0);
  if (st != LHF_OK) return st;
  return c->cuda(cudaEventRecord(c->tc_copied, c->stream), "cudaEventRecord");
}

// Launch a1..a5 for the uploaded systems (H, S already set in the descriptors).
// a1, a2 and the Gram factors (with the rank reduction when planned), without the rank sum.
// a1, a2 and the Gram factors.  On the mixed route the potential rows (FP64-bound) run on the
// side stream beside the basis samples and the fold into digit planes (FP32- and ALU-bound),
// which do not read them; the main stream waits for them before their own digit planes.  A CUDA
// graph captured over this records the two as parallel branches.  With per-kernel timing on, the
// potential stays on the main stream, so that every bracketed kernel runs alone.
lhf_status run_factors_gram(lhf_ctx *c, const std::vector<Plan> &ps) {
  const int nsys = (int)ps.size();
  const bool fork = ps[0].mixed && c->side && !c->prof;
  lhf_status st = LHF_OK;
  if (fork) {
    st = c->cuda(cudaEventRecord(c->fork_ev, c->stream), "cudaEventRecord");
    if (st == LHF_OK) st = c->cuda(cudaStreamWaitEvent(c->side, c->fork_ev, 0), "cudaStreamWaitEvent");
    if (st != LHF_OK) return st;
    c->begin(1, c->side);
    st = c->cuda(lhf::launch_potential(c->d_sys, nsys, max_of(ps, &Plan::pot_rows), c->side), "potential kernel");
    c->end(1, c->side);
    // the join is recorded whatever the launch returned: the main stream never runs ahead of it
    const lhf_status sr = c->cuda(cudaEventRecord(c->join_ev, c->side), "cudaEventRecord");
    if (sr != LHF_OK) return sr;
    c->join_pending = true;
    if (st != LHF_OK) {
      c->join();
      return st;
    }
  }
  c->begin(0);
  st = c->cuda(lhf::launch_basis(c->d_sys, nsys, max_of(ps, &Plan::basis_items), c->stream), "basis kernel");
  c->end();
  if (st == LHF_OK && !fork) {
    c->begin(1);
    st = c->cuda(lhf::launch_potential(c->d_sys, nsys, max_of(ps, &Plan::pot_rows), c->stream), "potential kernel");
    c->end();
  }
  if (st == LHF_OK) st = run_gram(c, ps, false);
  const lhf_status sj = c->join();
  return st != LHF_OK ? st : sj;
}

lhf_status run_assembly_factors(lhf_ctx *c, const std::vector<Plan> &ps) { return run_factors_gram(c, ps); }

lhf_status run_assembly(lhf_ctx *c, const std::vector<Plan> &ps) {
  const int nsys = (int)ps.size();
  // (a6, the zero blocks outside the window, is written by the rank-sum kernel)
  lhf_status st = run_factors_gram(c, ps);
  if (st != LHF_OK) return st;
  c->begin(3);
  int max_rt = 0;
  for (const Plan &p : ps) max_rt = std::max(max_rt, p.sd.Rt);
  st = c->cuda(lhf::launch_ranksum(c->d_sys, nsys, max_of(ps, &Plan::rank_ctas), max_of(ps, &Plan::rank_items),
                                   max_rt, c->stream),
               "rank-sum kernel");
  c->end();
  return st;
}

// Per-cell charges of open boxes into their workspace regions (pageable source: the copy is
// staged before cudaMemcpyAsync returns).
lhf_status upload_zcell(lhf_ctx *c, const std::vector<Plan> &ps) {
  for (const Plan &p : ps)
    if (p.sd.zcell) {
      lhf_status st = c->cuda(cudaMemcpyAsync(const_cast<double *>(p.sd.zcell), p.zcell.data(),
                                              p.zcell.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                              "cudaMemcpyAsync");
      if (st != LHF_OK) return st;
    }
  return LHF_OK;
}

// a1, a2 and the factors of open boxes (uploaded, all plans boxes): FP64 Grams of the single-cell
// directions, then the direction-0 factors between cell pairs.
lhf_status run_box_factors(lhf_ctx *c, const std::vector<Plan> &ps) {
  const int nsys = (int)ps.size();
  lhf_status st = upload_zcell(c, ps);
  if (st != LHF_OK) return st;
  int max_m0 = 0, width = 0;
  for (const Plan &p : ps) {
    max_m0 = std::max(max_m0, p.sd.m0);
    width = std::max(width, p.box_width);
  }
  c->begin(0);
  st = c->cuda(lhf::launch_basis(c->d_sys, nsys, max_of(ps, &Plan::basis_items), c->stream), "basis kernel");
  c->end();
  if (st != LHF_OK) return st;
  c->begin(1);
  st = c->cuda(lhf::launch_potential(c->d_sys, nsys, max_of(ps, &Plan::pot_rows), c->stream), "potential kernel");
  c->end();
  if (st != LHF_OK) return st;
  c->begin(2);
  st = c->cuda(lhf::launch_gram_fp64(c->d_sys, nsys, max_of(ps, &Plan::gram_blocks), max_m0,
                                     max_of(ps, &Plan::nv_max), c->stream),
               "Gram kernel");
  if (st == LHF_OK)
    st = c->cuda(lhf::launch_box_gram(c->d_sys, nsys, max_of(ps, &Plan::box_items), width, c->stream),
                 "box Gram kernel");
  c->end(2);
  return st;
}

// Dense H, S of open boxes (after run_box_factors).
lhf_status run_box_assemble(lhf_ctx *c, const std::vector<Plan> &ps) {
  long long entries = 0;
  for (const Plan &p : ps) {
    const long long nb = (long long)p.sd.m0 * p.sd.d[0].L;
    entries = std::max(entries, nb * nb);
  }
  c->begin(3);
  lhf_status st = c->cuda(lhf::launch_box_assemble(c->d_sys, (int)ps.size(), entries, c->stream), "box assembly kernel");
  c->end();
  return st;
}

// Dense generalized eigensolve of one pencil with the context's flags word.
lhf_status run_dense_eig(lhf_ctx *c, const double *H, const double *S, int N, double *eig, double *work) {
  c->begin(5);
  const int stall = c->stall_next ? 1 : 0;
  c->stall_next = false;
  cudaError_t e = lhf::launch_dense_eig(H, S, N, eig, work, c->d_flags, c->stream, c->wait_cycles, stall);
  c->end();
  if (e == cudaErrorNotSupported) return c->fail(LHF_ERR_UNSUPPORTED, "cooperative launch not available");
  return c->cuda(e, "dense eigensolver");
}

lhf_status run_dft(lhf_ctx *c, const std::vector<Plan> &ps) {
  c->host_L.resize(4 * ps.size());
  for (size_t i = 0; i < ps.size(); ++i) {
    for (int l = 0; l < 3; ++l) c->host_L[4 * i + l] = ps[i].sd.d[l].L;
    c->host_L[4 * i + 3] = ps[i].sd.m0;
  }
  c->begin(4);
  int passes = 0;
  lhf_status st = c->cuda(lhf::launch_dft(c->d_sys, (int)ps.size(), c->host_L.data(), &passes, c->stream), "DFT kernel");
  c->end(passes);
  return st;
}

// List of the k-points kappa with kappa <= -kappa (row-major index of (k0, k1, k2) mod L):
// one per conjugate pair; built once per lattice shape and kept on the device.
lhf_status klist_for(lhf_ctx *c, const int *L, const int **out, int *count) {
  const std::array<int, 3> key{L[0], L[1], L[2]};
  auto it = c->klists.find(key);
  if (it == c->klists.end()) {
    std::vector<int> v;
    for (int a = 0; a < L[0]; ++a)
      for (int b = 0; b < L[1]; ++b)
        for (int d = 0; d < L[2]; ++d) {
          const int k = (a * L[1] + b) * L[2] + d;
          const int mk = (((L[0] - a) % L[0]) * L[1] + (L[1] - b) % L[1]) * L[2] + (L[2] - d) % L[2];
          if (k <= mk) v.push_back(k);
        }
    int *dptr = nullptr;
    lhf_status st = c->cuda(cudaMalloc(&dptr, v.size() * sizeof(int)), "cudaMalloc");
    if (st != LHF_OK) return st;
    st = c->cuda(cudaMemcpy(dptr, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice), "cudaMemcpy");
    if (st != LHF_OK) {
      cudaFree(dptr);
      return st;
    }
    it = c->klists.emplace(key, std::make_pair(dptr, (int)v.size())).first;
  }
  *out = it->second.first;
  *count = it->second.second;
  return LHF_OK;
}

lhf_status set_klist(lhf_ctx *c, SysDev &sd) {
  const int L[3] = {sd.d[0].L, sd.d[1].L, sd.d[2].L};
  return klist_for(c, L, &sd.klist, &sd.nkhalf);
}

// Times each candidate launch shape of k_eig (warps per CTA) and, on the tridiagonal route, of
// k_tridiag_eig (threads per CTA) once on the uploaded batch (the overlap norms already
// launched); both kernels rewrite the same outputs, so the trial runs leave no trace beyond
// the time they take.  Returns the fastest pair.
lhf_status tune_eig(lhf_ctx *c, int nsys, int max_k, int max_m0, bool tri, bool full, bool vglob,
                    std::array<int, 2> *best) {
  cudaEvent_t a = nullptr, b = nullptr;
  lhf_status st = c->cuda(cudaEventCreate(&a), "cudaEventCreate");
  if (st == LHF_OK) st = c->cuda(cudaEventCreate(&b), "cudaEventCreate");
  auto timed = [&](auto launch, float *ms) -> lhf_status {
    lhf_status s2 = c->cuda(cudaEventRecord(a, c->stream), "cudaEventRecord");
    if (s2 == LHF_OK) s2 = c->cuda(launch(), "eigen kernel (tuning)");
    if (s2 == LHF_OK) s2 = c->cuda(cudaEventRecord(b, c->stream), "cudaEventRecord");
    if (s2 == LHF_OK) s2 = c->cuda(cudaEventSynchronize(b), "cudaEventSynchronize");
    if (s2 == LHF_OK) s2 = c->cuda(cudaEventElapsedTime(ms, a, b), "cudaEventElapsedTime");
    return s2;
  };
  (*best)[0] = 4;
  (*best)[1] = 128;
  float tbest = 1e30f, t = 0.f;
  const int wmax = lhf::eig_max_warps(max_m0, full, vglob);
  // a first run at the default shape warms the caches (and its output feeds the tridiagonal trials)
  if (st == LHF_OK)
    st = timed([&] { return lhf::launch_eig_reduce(c->d_sys, nsys, max_k, max_m0, c->d_flags, nullptr, c->stream,
                                                   std::min(4, wmax), full, vglob); },
               &t);
  for (int w : {1, 2, 4, 8}) {
    if (st != LHF_OK || w > wmax) break;
    st = timed([&] { return lhf::launch_eig_reduce(c->d_sys, nsys, max_k, max_m0, c->d_flags, nullptr, c->stream, w,
                                                   full, vglob); },
               &t);
    if (st == LHF_OK && t < tbest) {
      tbest = t;
      (*best)[0] = w;
    }
  }
  if (tri) {
    tbest = 1e30f;
    const int G = max_m0 <= 16 ? 16 : 32;
    for (int th : {32, 64, 128, 256}) {
      if (st != LHF_OK) break;
      if (th < G) continue;
      st = timed([&] { return lhf::launch_tridiag(c->d_sys, nsys, max_k, max_m0, c->d_flags, nullptr, c->stream, th); },
                 &t);
      if (st == LHF_OK && t < tbest) {
        tbest = t;
        (*best)[1] = th;
      }
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return st;
}

lhf_status run_eig(lhf_ctx *c, const std::vector<Plan> &ps, bool tri = true) {
  int max_k = 0, max_m0 = 0;
  long long total = 0;
  bool full = tri;  // every system on the mixed route's pair arithmetic: a warp per matrix
  bool vglob = true;  // every system has the per-k-point matrix scratch
  for (const Plan &p : ps) {
    vglob = vglob && p.sd.evs != nullptr;
    const int k = p.sd.klist ? p.sd.nkhalf : p.sd.nblocks;
    max_k = std::max(max_k, k);
    max_m0 = std::max(max_m0, p.sd.m0);
    total += k;
    full = full && p.sd.eig_df != 0 && p.sd.vecs == nullptr;
  }
  int lg = 0;
  while ((1ll << (lg + 1)) <= total) ++lg;
  const std::array<int, 3> key{max_m0, (tri ? 1 : 0) | (full ? 2 : 0) | (vglob ? 4 : 0), lg};
  std::array<int, 2> shape{std::min(4, lhf::eig_max_warps(max_m0, full, vglob)), 128};
  c->begin(5);
  lhf_status st = c->cuda(lhf::launch_overlap_norms(c->d_sys, (int)ps.size(), c->stream), "overlap-norm kernel");
  auto it = c->eig_tune.find(key);
  if (it != c->eig_tune.end()) {
    shape = it->second;
  } else if (st == LHF_OK && c->autotune && !c->capturing) {
    st = tune_eig(c, (int)ps.size(), max_k, max_m0, tri, full, vglob, &shape);
    if (st == LHF_OK) c->eig_tune[key] = shape;
  }
  c->last_eig_warps = shape[0];
  c->last_tri_threads = shape[1];
  if (st == LHF_OK)
    st = c->cuda(lhf::launch_eig(c->d_sys, (int)ps.size(), max_k, max_m0, c->d_flags, c->d_counters, c->stream,
                                 tri, shape[0], shape[1], full, vglob),
                 "eigen kernel");
  c->end(tri ? 3 : 2);
  return st;
}

lhf_status system_from_desc(lhf_ctx *c, const lhf_system_desc *d, HostSystem &s) {
  lhf_status st = check_lattice(c, &d->lattice);
  if (st != LHF_OK) return st;
  st = check_basis(c, &d->basis);
  if (st != LHF_OK) return st;
  st = check_grid(c, &d->grid);
  if (st != LHF_OK) return st;
  copy_lattice(s, &d->lattice);
  copy_basis(s, &d->basis);
  copy_grid(s, &d->grid);
  return LHF_OK;
}

// Point the descriptor's workspace regions at base.
void bind_ws(Plan &p, double *base) {
  p.sd.ws = base;
  p.sd.s0 = base + p.s0_off;
  p.sd.zcell = (p.sd.box && !p.zcell.empty()) ? base + p.zcell_off : nullptr;
  p.sd.tri = p.sd.box ? nullptr : base + p.tri_off;
  p.sd.evs = p.sd.box ? nullptr : base + p.evs_off;
  p.sd.dftw = p.dft_off ? base + p.dft_off : nullptr;
}

// Plan one system with workspace at ws_base and internal H, S, Hbar, Sbar after its factors.
size_t internal_doubles(const Plan &p) { return p.ws + 6 * p.blocks_doubles; }

void place_internal(Plan &p, double *base) {
  bind_ws(p, base);
  double *blk = base + p.ws;
  p.sd.H = blk;
  p.sd.S = blk + p.blocks_doubles;
  p.sd.Hbar = blk + 2 * p.blocks_doubles;
  p.sd.Sbar = blk + 4 * p.blocks_doubles;
}

}  // namespace

// ==========================================================================================
// C ABI

extern "C" {

lhf_status lhf_create(lhf_ctx **out, int device, void *stream) {
  if (!out) return LHF_ERR_ARG;
  *out = nullptr;
  lhf_ctx *c = new (std::nothrow) lhf_ctx();
  if (!c) return LHF_ERR_NOMEM;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    delete c;
    return LHF_ERR_CUDA;
  }
  c->device = device;
  c->stream = (cudaStream_t)stream;
  if (cudaSetDevice(device) != cudaSuccess || cudaEventCreateWithFlags(&c->upload_done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->tc_copied, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&c->d_flags, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(c->d_flags, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&c->d_counters, 3 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(c->d_counters, 0, 3 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    if (c->upload_done) cudaEventDestroy(c->upload_done);
    if (c->tc_copied) cudaEventDestroy(c->tc_copied);
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->d_flags) cudaFree(c->d_flags);
    if (c->d_counters) cudaFree(c->d_counters);
    delete c;
    return LHF_ERR_CUDA;
  }
  *out = c;
  return LHF_OK;
}

void lhf_destroy(lhf_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (lhf_graph *g : c->graphs) g->ctx = nullptr;  // their owners still free them
  if (c->ws) cudaFree(c->ws);
  if (c->d_sys) cudaFree(c->d_sys);
  if (c->h_sys) cudaFreeHost(c->h_sys);
  if (c->d_flags) cudaFree(c->d_flags);
  if (c->d_counters) cudaFree(c->d_counters);
  if (c->d_zcell) cudaFree(c->d_zcell);
  if (c->d_out) cudaFree(c->d_out);
  if (c->tc_buf) cudaFree(c->tc_buf);
  if (c->tc_host) cudaFreeHost(c->tc_host);
  if (c->upload_done) cudaEventDestroy(c->upload_done);
  if (c->tc_copied) cudaEventDestroy(c->tc_copied);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  if (c->side) cudaStreamDestroy(c->side);
  for (auto &m : c->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (auto &m : c->kmarks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  for (auto &kv : c->klists) cudaFree(kv.second.first);
  delete c;
}

lhf_status lhf_eig_counters(lhf_ctx *c, unsigned long long *passes, unsigned long long *matrices) {
  if (!c || !passes || !matrices) return LHF_ERR_ARG;
  unsigned long long h[3] = {0, 0, 0};
  lhf_status st = c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (st != LHF_OK) return st;
  st = c->cuda(cudaMemcpy(h, c->d_counters, sizeof h, cudaMemcpyDeviceToHost), "cudaMemcpy");
  if (st != LHF_OK) return st;
  st = c->cuda(cudaMemset(c->d_counters, 0, sizeof h), "cudaMemset");
  *passes = h[0];
  *matrices = h[1];
  return st;
}

lhf_status lhf_set_autotune(lhf_ctx *c, int enable) {
  if (!c) return LHF_ERR_ARG;
  c->autotune = enable != 0;
  return LHF_OK;
}

lhf_status lhf_launch_shapes(lhf_ctx *c, int *eig_warps, int *tri_threads) {
  if (!c || !eig_warps || !tri_threads) return LHF_ERR_ARG;
  *eig_warps = c->last_eig_warps;
  *tri_threads = c->last_tri_threads;
  return LHF_OK;
}

lhf_status lhf_set_rank_reduction(lhf_ctx *c, double eps) {
  if (!c) return LHF_ERR_ARG;
  if (!(eps == 0.0 || (eps >= 1e-14 && eps < 1.0))) return c->fail(LHF_ERR_ARG, "eps = %g: 0 or in [1e-14, 1)", eps);
  c->rank_eps = eps;
  return LHF_OK;
}

lhf_status lhf_rank_reduction_info(lhf_ctx *c, int *rank_in, int *rank_out, double *dropped, double *largest) {
  if (!c) return LHF_ERR_ARG;
  if (!(c->rank_eps > 0.0)) return c->fail(LHF_ERR_STATE, "rank reduction is off");
  Plan P;
  lhf_status st = current_plan(c, P);
  if (st != LHF_OK) return st;
  if (!P.rank_smem) return c->fail(LHF_ERR_UNSUPPORTED, "the current system takes no rank reduction");
  st = ensure_ws(c, P.ws);
  if (st != LHF_OK) return st;
  bind_ws(P, c->ws);
  st = upload(c, {P.sd});
  if (st != LHF_OK) return st;
  std::vector<Plan> one(1, P);
  st = run_assembly_factors(c, one);
  if (st != LHF_OK) return st;
  double h[4] = {0, 0, 0, 0};
  st = c->cuda(cudaMemcpyAsync(h, P.sd.ws + P.sd.offRR, sizeof h, cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
  if (st == LHF_OK) st = c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (st != LHF_OK) return st;
  if (rank_in) *rank_in = (int)h[0];
  if (rank_out) *rank_out = (int)h[1];
  if (dropped) *dropped = h[2];
  if (largest) *largest = h[3];
  return LHF_OK;
}

lhf_status lhf_extrapolate_lattice_sum(lhf_ctx *c, int nK, const double *K, long long n, const double *eig,
                                       double *eig_limit, double *slope) {
  if (!c) return LHF_ERR_ARG;
  if (nK < 2 || nK > lhf::kMaxExtrapolationWindows || !K || !eig || !eig_limit || n < 0)
    return c->fail(LHF_ERR_ARG, "nK in [2, %d], K, eig and eig_limit are required", lhf::kMaxExtrapolationWindows);
  for (int k = 0; k < nK; ++k) {
    if (!(K[k] >= 1.0) || !std::isfinite(K[k])) return c->fail(LHF_ERR_ARG, "K[%d] = %g must be >= 1", k, K[k]);
    for (int q = 0; q < k; ++q)
      if (K[q] == K[k]) return c->fail(LHF_ERR_ARG, "K values must differ");
  }
  // the windows into the workspace (pinned staging is not needed for nK doubles: a pageable
  // source is staged before cudaMemcpyAsync returns)
  lhf_status st = ensure_ws(c, 32);
  if (st != LHF_OK) return st;
  st = c->cuda(cudaMemcpyAsync(c->ws, K, nK * sizeof(double), cudaMemcpyHostToDevice, c->stream), "cudaMemcpyAsync");
  if (st != LHF_OK) return st;
  return c->cuda(lhf::launch_lattice_extrapolate(eig, c->ws, nK, n, eig_limit, slope, c->stream), "extrapolation kernel");
}

lhf_status lhf_set_wait_limit(lhf_ctx *c, long long cycles) {
  if (!c) return LHF_ERR_ARG;
  c->wait_cycles = cycles > 0 ? cycles : lhf::kDefaultWaitCycles;
  return LHF_OK;
}

lhf_status lhf_inject_barrier_stall(lhf_ctx *c) {
  if (!c) return LHF_ERR_ARG;
  c->stall_next = true;
  return LHF_OK;
}

lhf_status lhf_set_workspace_limit(lhf_ctx *c, size_t bytes) {
  if (!c) return LHF_ERR_ARG;
  c->ws_limit = bytes;
  return LHF_OK;
}

lhf_status lhf_set_profiling(lhf_ctx *c, int enable) {
  if (!c) return LHF_ERR_ARG;
  c->prof = enable != 0;
  return LHF_OK;
}

lhf_status lhf_stage_times(lhf_ctx *c, double *ms, int *launches) {
  if (!c || !ms || !launches) return LHF_ERR_ARG;
  for (int i = 0; i < LHF_NUM_STAGES; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  lhf_status st = c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (st != LHF_OK) return st;
  for (auto &m : c->marks) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess && m.stage >= 0 && m.stage < LHF_NUM_STAGES) {
      ms[m.stage] += t;
      launches[m.stage] += m.kernels;
    } else {
      cudaGetLastError();
    }
    c->pool.push_back(m.a);
    c->pool.push_back(m.b);
  }
  c->marks.clear();
  return LHF_OK;
}

lhf_status lhf_kernel_times(lhf_ctx *c, double *ms, int *launches) {
  if (!c || !ms || !launches) return LHF_ERR_ARG;
  for (int i = 0; i < LHF_NUM_KERNELS; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  lhf_status st = c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (st != LHF_OK) return st;
  for (auto &m : c->kmarks) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess && m.stage >= 0 && m.stage < LHF_NUM_KERNELS) {
      ms[m.stage] += t;
      launches[m.stage] += 1;
    } else {
      cudaGetLastError();
    }
    c->pool.push_back(m.a);
    c->pool.push_back(m.b);
  }
  c->kmarks.clear();
  return LHF_OK;
}

const char *lhf_kernel_name(int kernel) {
  static const char *const names[LHF_NUM_KERNELS] = {
      "k_basis",   "k_potential",   "k_gram_fp64", "k_gram_slice",   "k_vslice",        "k_gram_tc",
      "k_gram_mirror", "k_ranksum", "k_dft_pass",  "k_overlap_norms", "k_eig",          "k_tridiag_eig",
      "k_box_gram", "k_box_assemble", "k_dense_eig", "k_factor_dft", "k_kspace_blocks", "k_box_solve"};
  return kernel >= 0 && kernel < LHF_NUM_KERNELS ? names[kernel] : nullptr;
}

const char *lhf_last_error(const lhf_ctx *c) { return c ? c->err.c_str() : "null context"; }

lhf_status lhf_set_stream(lhf_ctx *c, void *stream) {
  if (!c) return LHF_ERR_ARG;
  lhf_status st = c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (st != LHF_OK) return st;
  c->stream = (cudaStream_t)stream;
  return LHF_OK;
}

lhf_status lhf_sync(lhf_ctx *c) {
  if (!c) return LHF_ERR_ARG;
  lhf_status st = c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (st != LHF_OK) return st;
  unsigned flags = 0;
  st = c->cuda(cudaMemcpy(&flags, c->d_flags, sizeof flags, cudaMemcpyDeviceToHost), "cudaMemcpy");
  if (st != LHF_OK) return st;
  st = c->cuda(cudaMemset(c->d_flags, 0, sizeof(unsigned)), "cudaMemset");
  if (st != LHF_OK) return st;
  if (flags & lhf::kFlagTimeout) return c->fail(LHF_ERR_TIMEOUT, "a bounded device-side wait gave up (tensor-core Gram pipeline or dense-solver grid barrier)");
  if (flags & lhf::kFlagNotSpd) return c->fail(LHF_ERR_NOT_SPD, "an overlap block was not positive definite");
  return LHF_OK;
}

lhf_status lhf_lattice_setup(lhf_ctx *c, const lhf_lattice_desc *d) {
  if (!c) return LHF_ERR_ARG;
  lhf_status st = check_lattice(c, d);
  if (st != LHF_OK) return st;
  copy_lattice(c->cur, d);
  c->has_lat = true;
  return LHF_OK;
}

lhf_status lhf_basis_setup(lhf_ctx *c, const lhf_basis_desc *d) {
  if (!c) return LHF_ERR_ARG;
  lhf_status st = check_basis(c, d);
  if (st != LHF_OK) return st;
  copy_basis(c->cur, d);
  c->has_basis = true;
  return LHF_OK;
}

lhf_status lhf_grid_setup(lhf_ctx *c, const lhf_grid_desc *d) {
  if (!c) return LHF_ERR_ARG;
  lhf_status st = check_grid(c, d);
  if (st != LHF_OK) return st;
  copy_grid(c->cur, d);
  c->has_grid = true;
  return LHF_OK;
}

lhf_status lhf_query_sizes(lhf_ctx *c, lhf_sizes *out) {
  if (!c || !out) return LHF_ERR_ARG;
  Plan P;
  lhf_status st = current_plan(c, P);
  if (st != LHF_OK) return st;
  memset(out, 0, sizeof *out);
  out->m0 = P.sd.m0;
  out->n_blocks = P.sd.nblocks;
  out->n_kpoints = P.sd.nblocks;
  out->n_basis = P.sd.m0 * P.sd.nblocks;
  out->rank = P.sd.Rt;
  out->periodic = P.sd.box ? 0 : 1;
  out->desc_bytes = (int)sizeof(SysDev);
  for (int l = 0; l < 3; ++l) {
    out->window[l] = (P.sd.box && l == 0) ? P.sd.bJ : P.sd.d[l].J;
    out->n_potential[l] = P.sd.d[l].nv;
    const DirDev &D = P.sd.d[l];
    if (P.sd.box && l == 0) continue;  // the box's cell-pair factors (no window Gram)
    for (int jc = 0; jc < D.Jc; ++jc)
      for (int mu = 0; mu < P.sd.m0; ++mu)
        for (int nu = 0; nu < P.sd.m0; ++nu)
          out->overlap_rows[l] += lhf::gram_row_cells(P.sd, l, D.jlo + D.cw0 + jc, mu, nu) > 0;
  }
  return LHF_OK;
}

static lhf_status check_precision(lhf_ctx *c, lhf_precision p) {
  if (p == LHF_FP64 || p == LHF_MIXED) return LHF_OK;
  return c->fail(LHF_ERR_ARG, "unknown precision %d", (int)p);
}

lhf_status lhf_assemble_core_hamiltonian(lhf_ctx *c, lhf_precision prec, double *H, double *S) {
  if (!c) return LHF_ERR_ARG;
  if (!H || !S) return c->fail(LHF_ERR_ARG, "H and S must be device pointers");
  lhf_status st = check_precision(c, prec);
  if (st != LHF_OK) return st;
  std::vector<Plan> ps(1);
  st = current_plan(c, ps[0], prec == LHF_MIXED);
  if (st != LHF_OK) return st;
  st = ensure_ws(c, ps[0].ws);
  if (st != LHF_OK) return st;
  bind_ws(ps[0], c->ws);
  ps[0].sd.H = H;
  ps[0].sd.S = S;
  st = upload(c, {ps[0].sd});
  if (st != LHF_OK) return st;
  if (ps[0].sd.box) {
    st = run_box_factors(c, ps);
    if (st != LHF_OK) return st;
    return run_box_assemble(c, ps);
  }
  return run_assembly(c, ps);
}

lhf_status lhf_kspace_blocks(lhf_ctx *c, lhf_precision prec, double *Hbar, double *Sbar) {
  if (!c) return LHF_ERR_ARG;
  if (!Hbar || !Sbar) return c->fail(LHF_ERR_ARG, "Hbar and Sbar must be device pointers");
  lhf_status st = check_precision(c, prec);
  if (st != LHF_OK) return st;
  std::vector<Plan> ps(1);
  st = current_plan(c, ps[0], prec == LHF_MIXED);
  if (st != LHF_OK) return st;
  Plan &P = ps[0];
  if (P.sd.box) return c->fail(LHF_ERR_UNSUPPORTED, "the k-space route needs a periodic lattice");
  // the 1D factor transforms after the plan's regions
  const size_t mm = (size_t)P.sd.m0 * P.sd.m0;
  for (int l = 0; l < 3; ++l) {
    P.sd.d[l].offF = (int64_t)P.ws;
    P.ws = align_up(P.ws + 2 * (size_t)P.sd.d[l].L * (P.sd.Rt + 2) * mm);
  }
  st = ensure_ws(c, P.ws);
  if (st != LHF_OK) return st;
  bind_ws(P, c->ws);
  P.sd.Hbar = Hbar;
  P.sd.Sbar = Sbar;
  st = set_klist(c, P.sd);
  if (st != LHF_OK) return st;
  st = upload(c, {P.sd});
  if (st != LHF_OK) return st;
  c->begin(0);
  st = c->cuda(lhf::launch_basis(c->d_sys, 1, P.basis_items, c->stream), "basis kernel");
  c->end();
  if (st != LHF_OK) return st;
  c->begin(1);
  st = c->cuda(lhf::launch_potential(c->d_sys, 1, P.pot_rows, c->stream), "potential kernel");
  c->end();
  if (st != LHF_OK) return st;
  st = run_gram(c, ps, false);
  if (st != LHF_OK) return st;
  c->begin(4);
  st = c->cuda(lhf::launch_kspace(c->d_sys, 1, lhf::kspace_factor_ctas(P.sd), (long long)P.sd.nkhalf * mm, c->stream),
               "k-space kernels");
  c->end(2);
  return st;
}

lhf_status lhf_circulant_fft(lhf_ctx *c, const double *H, const double *S, double *Hbar, double *Sbar) {
  if (!c) return LHF_ERR_ARG;
  if (!H || !S || !Hbar || !Sbar) return c->fail(LHF_ERR_ARG, "all four pointers are required");
  std::vector<Plan> ps(1);
  lhf_status st = current_plan(c, ps[0]);
  if (st != LHF_OK) return st;
  if (ps[0].sd.box) return c->fail(LHF_ERR_UNSUPPORTED, "the block DFT needs a periodic lattice");
  st = ensure_ws(c, ps[0].ws);  // the four-step route of long chains uses the plan's scratch
  if (st != LHF_OK) return st;
  bind_ws(ps[0], c->ws);
  ps[0].sd.H = const_cast<double *>(H);
  ps[0].sd.S = const_cast<double *>(S);
  ps[0].sd.Hbar = Hbar;
  ps[0].sd.Sbar = Sbar;
  st = upload(c, {ps[0].sd});
  if (st != LHF_OK) return st;
  return run_dft(c, ps);
}

lhf_status lhf_k_point_eigensolve(lhf_ctx *c, const double *Hbar, const double *Sbar, double *eig, int *kstat) {
  if (!c) return LHF_ERR_ARG;
  if (!Hbar || !Sbar || !eig) return c->fail(LHF_ERR_ARG, "Hbar, Sbar and eig are required");
  std::vector<Plan> ps(1);
  lhf_status st = current_plan(c, ps[0]);
  if (st != LHF_OK) return st;
  if (ps[0].sd.box) return c->fail(LHF_ERR_UNSUPPORTED, "k-point eigensolves need a periodic lattice");
  st = ensure_ws(c, ps[0].ws);
  if (st != LHF_OK) return st;
  bind_ws(ps[0], c->ws);
  ps[0].sd.Hbar = const_cast<double *>(Hbar);
  ps[0].sd.Sbar = const_cast<double *>(Sbar);
  ps[0].sd.eig = eig;
  ps[0].sd.kstat = kstat;
  st = set_klist(c, ps[0].sd);
  if (st != LHF_OK) return st;
  st = upload(c, {ps[0].sd});
  if (st != LHF_OK) return st;
  return run_eig(c, ps);
}

lhf_status lhf_k_point_eigenvectors(lhf_ctx *c, const double *Hbar, const double *Sbar, double *eig, double *vecs,
                                    int *kstat) {
  if (!c) return LHF_ERR_ARG;
  if (!Hbar || !Sbar || !eig || !vecs) return c->fail(LHF_ERR_ARG, "Hbar, Sbar, eig and vecs are required");
  std::vector<Plan> ps(1);
  lhf_status st = current_plan(c, ps[0]);
  if (st != LHF_OK) return st;
  if (ps[0].sd.box) return c->fail(LHF_ERR_UNSUPPORTED, "k-point eigensolves need a periodic lattice");
  st = ensure_ws(c, ps[0].ws);
  if (st != LHF_OK) return st;
  bind_ws(ps[0], c->ws);
  ps[0].sd.Hbar = const_cast<double *>(Hbar);
  ps[0].sd.Sbar = const_cast<double *>(Sbar);
  ps[0].sd.eig = eig;
  ps[0].sd.kstat = kstat;
  ps[0].sd.vecs = vecs;
  ps[0].sd.tri = nullptr;  // Jacobi with accumulated rotations at every k-point
  st = set_klist(c, ps[0].sd);
  if (st != LHF_OK) return st;
  st = upload(c, {ps[0].sd});
  if (st != LHF_OK) return st;
  return run_eig(c, ps, false);
}

lhf_status lhf_dense_eigensolve(lhf_ctx *c, const double *H, const double *S, int N, double *eig) {
  if (!c) return LHF_ERR_ARG;
  if (!H || !S || !eig) return c->fail(LHF_ERR_ARG, "H, S and eig are required");
  if (N < 1 || N > 8192) return c->fail(LHF_ERR_ARG, "N = %d outside [1, 8192]", N);
  lhf_status st = ensure_ws(c, lhf::dense_eig_workspace_doubles(N));
  if (st != LHF_OK) return st;
  return run_dense_eig(c, H, S, N, eig, c->ws);
}

lhf_status lhf_box_lowest_eigenvalues(lhf_ctx *c, const lhf_system_desc *box, int n_ev, double tol, int max_iter,
                                      double *eig, int *iterations, double *residual) {
  if (!c) return LHF_ERR_ARG;
  if (!box || !eig) return c->fail(LHF_ERR_ARG, "box and eig are required");
  if (iterations) *iterations = 0;
  if (residual) *residual = 0.0;
  HostSystem hs;
  lhf_status st = system_from_desc(c, box, hs);
  if (st != LHF_OK) return st;
  Plan P;
  st = make_plan(c, hs, P, false, false);
  if (st != LHF_OK) return st;
  if (!P.sd.box) return c->fail(LHF_ERR_ARG, "lhf_box_lowest_eigenvalues needs an open (L,1,1) box");
  const int L = P.sd.d[0].L, m0 = P.sd.m0, bJ = P.sd.bJ, bjlo = P.sd.bjlo;
  const long long N = (long long)L * m0;
  const int kv = std::min(n_ev + std::max(4, n_ev / 4), (int)std::min<long long>(N, 24));
  if (n_ev < 1 || n_ev > 20 || n_ev > kv) return c->fail(LHF_ERR_ARG, "n_ev = %d outside [1, min(20, N)]", n_ev);
  if (!(tol > 0.0) || max_iter < 1) return c->fail(LHF_ERR_ARG, "tol > 0 and max_iter >= 1 are required");
  int M = 1;
  while (M < L + bJ) M <<= 1;
  if (M > 8192) return c->fail(LHF_ERR_UNSUPPORTED, "box of %d cells with a window of %d: circulant above 8192 cells", L, bJ);
  // workspace: factors | band H, S | Z, HZ, SZ [3kv][N] | Z' [2kv][N] | R [kv][N] |
  // Hk, Sk, Lk [M][m0][m0] complex | Vk [kv][M][m0] complex | GA, GB [72^2] | C [72][kv] |
  // theta, rnorm [kv] | flags (one double: bad word + info)
  const size_t band = align_up((size_t)L * bJ * m0 * m0);
  const size_t vec = (size_t)N;  // vector stride (doubles)
  const size_t kblk = align_up((size_t)M * m0 * m0 * 2);
  const int nrr = lhf::rayleigh_ritz_max();
  size_t off = P.ws;
  const size_t o_hb = off, o_sb = o_hb + band;
  off = o_sb + band;
  const size_t blk3 = align_up(3 * kv * vec), blk2 = align_up(2 * kv * vec);
  const size_t o_z = off, o_hz = o_z + blk3, o_sz = o_hz + blk3;
  off = o_sz + blk3;
  const size_t o_z2 = off;
  off = o_z2 + blk2;
  const size_t o_r = off;
  off += align_up(kv * vec);
  const size_t o_hk = off, o_sk = o_hk + kblk, o_lk = o_sk + kblk;
  off = o_lk + kblk;
  const size_t o_vk = off;
  off = align_up(off + (size_t)kv * M * m0 * 2);
  const size_t o_ha = off, o_sa = o_ha + align_up((size_t)bJ * m0 * m0);
  off = o_sa + align_up((size_t)bJ * m0 * m0);
  const size_t o_ga = off, o_gb = o_ga + align_up((size_t)nrr * nrr);
  off = o_gb + align_up((size_t)nrr * nrr);
  const size_t o_c = off;
  off = align_up(off + (size_t)nrr * kv);
  const size_t o_th = off, o_rn = o_th + align_up(kv);
  off = o_rn + align_up(kv);
  const size_t o_fl = off;
  off = align_up(off + 4);
  // block-tridiagonal factor of H - sigma S: super-cells of g cells (the band's reach)
  const int g = std::max(1, std::max(-bjlo, bjlo + bJ - 1));
  const int Bt = g * m0, nbt = (L + g - 1) / g;
  const size_t o_td = off, o_te = o_td + align_up((size_t)nbt * Bt * Bt);
  off = o_te + align_up((size_t)nbt * Bt * Bt);
  const size_t o_tv = off;
  off = align_up(off + (size_t)kv * nbt * Bt);
  st = ensure_ws(c, off);
  if (st != LHF_OK) return st;
  double *w = c->ws;
  bind_ws(P, w);
  double *Hb = w + o_hb, *Sb = w + o_sb, *Z = w + o_z, *HZ = w + o_hz, *SZ = w + o_sz;
  double *Z2 = w + o_z2, *R = w + o_r;
  double2 *Hk = reinterpret_cast<double2 *>(w + o_hk), *Sk = reinterpret_cast<double2 *>(w + o_sk);
  double2 *Lk = reinterpret_cast<double2 *>(w + o_lk), *Vk = reinterpret_cast<double2 *>(w + o_vk);
  double *Ha = w + o_ha, *Sa = w + o_sa;
  double *GA = w + o_ga, *GB = w + o_gb, *C = w + o_c, *theta = w + o_th, *rnorm = w + o_rn;
  double *TD = w + o_td, *TE = w + o_te, *TV = w + o_tv;
  unsigned *bad = reinterpret_cast<unsigned *>(w + o_fl);
  int *info = reinterpret_cast<int *>(w + o_fl + 1);
  std::vector<Plan> one(1, P);
  st = upload(c, {P.sd});
  if (st != LHF_OK) return st;
  st = run_box_factors(c, one);
  if (st != LHF_OK) return st;
  auto cu = [&](cudaError_t e, const char *what) { return c->cuda(e, what); };
  c->begin(5);
  st = cu(lhf::launch_box_band(c->d_sys, (long long)L * bJ * m0 * m0, Hb, Sb, c->stream), "band kernel");
  if (st == LHF_OK) st = cu(lhf::launch_band_average(Hb, Sb, L, bJ, bjlo, m0, Ha, Sa, c->stream), "band average");
  if (st == LHF_OK)
    st = cu(lhf::launch_prec_blocks(Ha, Sa, 0, bJ, bjlo, m0, M, Hk, Sk, c->stream), "preconditioner blocks");
  c->end();
  if (st != LHF_OK) return st;
  // the preconditioner's shift: Pbar_kappa(sigma) = Hbar_kappa - sigma Sbar_kappa is positive
  // definite for every kappa exactly when sigma lies below the spectrum of the bulk circulant
  // (Sylvester's law of inertia per kappa); bisection on that test, then a margin below
  auto pd = [&](double sigma, bool *ok) -> lhf_status {
    lhf_status s2 = cu(cudaMemsetAsync(bad, 0, sizeof(unsigned), c->stream), "cudaMemsetAsync");
    if (s2 == LHF_OK) s2 = cu(lhf::launch_prec_factor(Hk, Sk, sigma, m0, M, Lk, bad, c->stream), "preconditioner factor");
    unsigned h = 0;
    if (s2 == LHF_OK) s2 = cu(cudaMemcpyAsync(&h, bad, sizeof h, cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
    if (s2 == LHF_OK) s2 = cu(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    *ok = h == 0;
    return s2;
  };
  double lo = -1.0, hi = 0.0;
  bool ok = false;
  for (int t = 0; t < 64; ++t) {
    if ((st = pd(lo, &ok)) != LHF_OK) return st;
    if (ok) break;
    hi = lo;
    lo = 2.0 * lo - 1.0;
  }
  if (!ok) return c->fail(LHF_ERR_NOT_SPD, "no shift makes the bulk circulant positive definite");
  for (int t = 0; t < 64; ++t) {  // an upper end where the test fails
    if ((st = pd(hi, &ok)) != LHF_OK) return st;
    if (!ok) break;
    const double step = 2.0 * (hi - lo) + 1.0;
    lo = hi;
    hi += step;
  }
  for (int t = 0; t < 48 && hi - lo > 1e-12 * (1.0 + fabs(lo)); ++t) {
    const double mid = 0.5 * (lo + hi);
    if ((st = pd(mid, &ok)) != LHF_OK) return st;
    (ok ? lo : hi) = mid;
  }
  const double sigma = lo - 0.05 * (1.0 + fabs(lo));
  if ((st = pd(sigma, &ok)) != LHF_OK) return st;
  if (!ok) return c->fail(LHF_ERR_NOT_SPD, "preconditioner not positive definite at sigma = %g", sigma);
  const size_t vb = vec * sizeof(double);
  c->begin(5);
  // start: preconditioned seeded vectors, their products, Rayleigh-Ritz on X alone
  st = cu(lhf::launch_start_vectors(R, kv, (long long)vec, 0x5eedull, c->stream), "start vectors");
  if (st == LHF_OK) st = cu(lhf::launch_prec_apply(Lk, R, Z, Vk, L, m0, M, kv, c->stream), "preconditioner");
  if (st == LHF_OK) st = cu(lhf::launch_band_mv(Hb, Sb, Z, HZ, SZ, L, bJ, bjlo, m0, kv, c->stream), "band matvec");
  c->end();
  if (st != LHF_OK) return st;
  auto rr = [&](int n, int *kept) -> lhf_status {
    lhf_status s2 = cu(lhf::launch_gram_vec(Z, HZ, n, N, GA, c->stream), "Gram kernel");
    if (s2 == LHF_OK) s2 = cu(lhf::launch_gram_vec(Z, SZ, n, N, GB, c->stream), "Gram kernel");
    if (s2 == LHF_OK) s2 = cu(lhf::launch_rayleigh_ritz(GA, GB, n, kv, 1e-12, theta, C, info, c->stream), "Rayleigh-Ritz kernel");
    int h = 0;
    if (s2 == LHF_OK) s2 = cu(cudaMemcpyAsync(&h, info, sizeof h, cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
    if (s2 == LHF_OK) s2 = cu(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    *kept = h;
    return s2;
  };
  // X <- Z C (rows 0 .. n), P <- Z[kv..n] C[kv..n] (when with_p), then their products H X, S X,
  // H P, S P by banded matvecs: updating the products by the same combinations would carry the
  // rounding of coefficients of nearly dependent directions (up to 1 / sqrt(cut)) into them
  auto update = [&](int n, bool with_p) -> lhf_status {
    lhf_status s2 = cu(lhf::launch_lincomb(Z, C, kv, 0, n, kv, N, Z2, c->stream), "linear combination");
    if (s2 == LHF_OK && with_p)
      s2 = cu(lhf::launch_lincomb(Z, C, kv, kv, n, kv, N, Z2 + kv * vec, c->stream), "linear combination");
    if (s2 == LHF_OK) s2 = cu(cudaMemcpyAsync(Z, Z2, kv * vb, cudaMemcpyDeviceToDevice, c->stream), "cudaMemcpyAsync");
    if (s2 == LHF_OK && with_p)
      s2 = cu(cudaMemcpyAsync(Z + 2 * kv * vec, Z2 + kv * vec, kv * vb, cudaMemcpyDeviceToDevice, c->stream),
              "cudaMemcpyAsync");
    if (s2 == LHF_OK) s2 = cu(lhf::launch_band_mv(Hb, Sb, Z, HZ, SZ, L, bJ, bjlo, m0, kv, c->stream), "band matvec");
    if (s2 == LHF_OK && with_p)
      s2 = cu(lhf::launch_band_mv(Hb, Sb, Z + 2 * kv * vec, HZ + 2 * kv * vec, SZ + 2 * kv * vec, L, bJ, bjlo, m0,
                                  kv, c->stream),
              "band matvec");
    return s2;
  };
  int kept = 0;
  if ((st = rr(kv, &kept)) != LHF_OK) return st;
  if (kept < kv) return c->fail(LHF_ERR_NOT_SPD, "start block of rank %d < %d", kept, kv);
  if ((st = update(kv, false)) != LHF_OK) return st;
  std::vector<double> th(kv), rn(kv);
  // the shift of the exact preconditioner (H - sigma S)^{-1}: below the lowest Ritz value of the
  // start block by a quarter of its spread; lowered until the block Cholesky succeeds (positive
  // definite exactly when sigma lies below the box's lowest eigenvalue)
  st = cu(cudaMemcpyAsync(th.data(), theta, kv * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
  if (st == LHF_OK) st = cu(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
  if (st != LHF_OK) return st;
  const double spread = std::max(th[kv - 1] - th[0], 0.1);
  double shift = th[0] - 0.25 * spread;
  for (int t = 0;; ++t) {
    lhf_status s2 = cu(cudaMemsetAsync(bad, 0, sizeof(unsigned), c->stream), "cudaMemsetAsync");
    if (s2 == LHF_OK)
      s2 = cu(lhf::launch_tri_factor(Hb, Sb, shift, L, bJ, bjlo, m0, g, nbt, TD, TE, bad, c->stream), "band factor");
    unsigned h = 0;
    if (s2 == LHF_OK) s2 = cu(cudaMemcpyAsync(&h, bad, sizeof h, cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
    if (s2 == LHF_OK) s2 = cu(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (s2 != LHF_OK) return s2;
    if (h == 0) break;
    if (t == 30) return c->fail(LHF_ERR_NOT_SPD, "no shift below the box spectrum found (last %g)", shift);
    shift -= spread * (double)(1 << std::min(t, 20));
  }
  bool have_p = false;
  int it = 0;
  double worst = 0.0;
  bool converged = false;
  for (it = 0; it < max_iter; ++it) {
    st = cu(lhf::launch_residual(HZ, SZ, theta, kv, N, R, rnorm, c->stream), "residual kernel");
    if (st == LHF_OK) st = cu(cudaMemcpyAsync(th.data(), theta, kv * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
    if (st == LHF_OK) st = cu(cudaMemcpyAsync(rn.data(), rnorm, kv * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
    if (st == LHF_OK) st = cu(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (st != LHF_OK) return st;
    worst = 0.0;
    for (int i = 0; i < n_ev; ++i) worst = std::max(worst, rn[i] / std::max(1.0, fabs(th[i])));
    if (worst <= tol) {
      converged = true;
      break;
    }
    // W = (H - shift S)^{-1} R into Z[kv .. 2kv), its products
    st = cu(cudaMemcpyAsync(Z + kv * vec, R, kv * vb, cudaMemcpyDeviceToDevice, c->stream), "cudaMemcpyAsync");
    if (st == LHF_OK) st = cu(lhf::launch_tri_solve(TD, TE, Bt, nbt, N, kv, Z + kv * vec, TV, c->stream), "band solve");
    if (st == LHF_OK)
      st = cu(lhf::launch_band_mv(Hb, Sb, Z + kv * vec, HZ + kv * vec, SZ + kv * vec, L, bJ, bjlo, m0, kv, c->stream),
              "band matvec");
    if (st != LHF_OK) return st;
    int n = have_p ? 3 * kv : 2 * kv;
    if ((st = rr(n, &kept)) != LHF_OK) return st;
    if (kept < kv && have_p) {  // the previous directions made the basis degenerate: drop them
      n = 2 * kv;
      if ((st = rr(n, &kept)) != LHF_OK) return st;
    }
    if (kept < kv) return c->fail(LHF_ERR_NOT_SPD, "LOBPCG basis of rank %d < %d", kept, kv);
    if ((st = update(n, true)) != LHF_OK) return st;
    have_p = true;
  }
  if (iterations) *iterations = it;
  if (residual) *residual = worst;
  st = cu(cudaMemcpyAsync(eig, theta, n_ev * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "cudaMemcpyAsync");
  if (st != LHF_OK) return st;
  if (!converged) return c->fail(LHF_ERR_NOT_CONVERGED, "LOBPCG: residual %.3g above %.3g after %d iterations", worst, tol, it);
  return LHF_OK;
}

lhf_status lhf_bloch_spectra(lhf_ctx *c, int nsys, const lhf_system_desc *systems, lhf_precision prec,
                             double *eig, int *kstat) {
  if (!c) return LHF_ERR_ARG;
  if (nsys < 1 || !systems || !eig) return c->fail(LHF_ERR_ARG, "nsys >= 1, systems and eig are required");
  lhf_status st = check_precision(c, prec);
  if (st != LHF_OK) return st;
  std::vector<Plan> all(nsys);
  size_t total = 0;
  for (int i = 0; i < nsys; ++i) {
    HostSystem hs;
    st = system_from_desc(c, &systems[i], hs);
    if (st != LHF_OK) return c->fail(st, "system %d: %s", i, c->err.c_str());
    st = cached_plan(c, hs, all[i], prec == LHF_MIXED);
    if (st != LHF_OK) return c->fail(st, "system %d: %s", i, c->err.c_str());
    total += internal_doubles(all[i]);
  }
  st = ensure_ws(c, total);
  if (st != LHF_OK) return st;
  // periodic lattices go through one batched pass; open boxes (dense matrices) one at a time
  std::vector<Plan> ps, boxes;
  size_t base = 0, eoff = 0, koff = 0;
  for (int i = 0; i < nsys; ++i) {
    Plan &p = all[i];
    place_internal(p, c->ws + base);
    base += internal_doubles(p);
    p.sd.eig = eig + eoff;                        // [n_kpoints][m0] per system
    p.sd.kstat = kstat ? kstat + koff : nullptr;  // [n_kpoints] per system
    eoff += (size_t)p.sd.nblocks * p.sd.m0;
    koff += p.sd.nblocks;
    if (p.sd.box) {
      boxes.push_back(p);
    } else {
      st = set_klist(c, p.sd);
      if (st != LHF_OK) return st;
      ps.push_back(p);
    }
  }
  if (!ps.empty()) {
    std::vector<SysDev> sds(ps.size());
    for (size_t i = 0; i < ps.size(); ++i) sds[i] = ps[i].sd;
    st = upload(c, sds);
    if (st != LHF_OK) return st;
    st = run_assembly(c, ps);
    if (st != LHF_OK) return st;
    st = run_dft(c, ps);
    if (st != LHF_OK) return st;
    st = run_eig(c, ps);
    if (st != LHF_OK) return st;
  }
  for (Plan &p : boxes) {
    std::vector<Plan> one(1, p);
    st = upload(c, {p.sd});
    if (st != LHF_OK) return st;
    st = run_box_factors(c, one);
    if (st != LHF_OK) return st;
    st = run_box_assemble(c, one);
    if (st != LHF_OK) return st;
    const int N = p.sd.m0 * p.sd.d[0].L;
    st = run_dense_eig(c, p.sd.H, p.sd.S, N, p.sd.eig, p.sd.ws + p.dense_off);
    if (st != LHF_OK) return st;
    if (p.sd.kstat) {  // no functions are removed in the dense solve
      st = c->cuda(cudaMemsetAsync(p.sd.kstat, 0, sizeof(int) * (size_t)p.sd.nblocks, c->stream), "cudaMemsetAsync");
      if (st != LHF_OK) return st;
    }
  }
  return LHF_OK;
}

// ------------------------------------------------------------------------------------------
// CUDA graph of the batched path

lhf_status lhf_graph_create(lhf_ctx *c, int nsys, const lhf_system_desc *systems, lhf_precision prec,
                            double *eig, int *kstat, lhf_graph **out) {
  if (!c) return LHF_ERR_ARG;
  if (!out) return c->fail(LHF_ERR_ARG, "out is required");
  *out = nullptr;
  if (nsys < 1 || !systems || !eig) return c->fail(LHF_ERR_ARG, "nsys >= 1, systems and eig are required");
  lhf_status st = check_precision(c, prec);
  if (st != LHF_OK) return st;
  std::vector<Plan> ps(nsys);
  size_t total = 0;
  for (int i = 0; i < nsys; ++i) {
    HostSystem hs;
    st = system_from_desc(c, &systems[i], hs);
    if (st != LHF_OK) return c->fail(st, "system %d: %s", i, c->err.c_str());
    st = cached_plan(c, hs, ps[i], prec == LHF_MIXED);
    if (ps[i].rank_smem) {  // a replay would read the descriptor the reduction rewrote
      ps[i].sd.rank_eps = 0.0;
      ps[i].rank_smem = 0;
    }
    if (st != LHF_OK) return c->fail(st, "system %d: %s", i, c->err.c_str());
    if (ps[i].sd.box) return c->fail(LHF_ERR_UNSUPPORTED, "system %d: open boxes are not captured in graphs", i);
    total += internal_doubles(ps[i]);
  }
  lhf_graph *g = new (std::nothrow) lhf_graph();
  if (!g) return c->fail(LHF_ERR_NOMEM, "graph");
  g->ctx = c;
  c->graphs.insert(g);
  auto cleanup = [&](lhf_status s) {
    lhf_graph_destroy(g);
    return s;
  };
  if (c->ws_limit && total * sizeof(double) > c->ws_limit)
    return cleanup(c->fail(LHF_ERR_NOMEM, "graph workspace of %zu bytes exceeds the context's limit of %zu bytes",
                           total * sizeof(double), c->ws_limit));
  if (cudaMalloc(&g->ws, total * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return cleanup(c->fail(LHF_ERR_NOMEM, "graph workspace of %zu bytes", total * sizeof(double)));
  }
  size_t base = 0, eoff = 0, koff = 0;
  std::vector<SysDev> sds(nsys);
  for (int i = 0; i < nsys; ++i) {
    place_internal(ps[i], g->ws + base);
    base += internal_doubles(ps[i]);
    st = set_klist(c, ps[i].sd);
    if (st != LHF_OK) return cleanup(st);
    ps[i].sd.eig = eig + eoff;
    ps[i].sd.kstat = kstat ? kstat + koff : nullptr;
    eoff += (size_t)ps[i].sd.nblocks * ps[i].sd.m0;
    koff += ps[i].sd.nblocks;
    sds[i] = ps[i].sd;
  }
  st = c->cuda(cudaMalloc(&g->d_sys, nsys * sizeof(SysDev)), "cudaMalloc");
  if (st != LHF_OK) return cleanup(st);
  st = c->cuda(cudaMemcpy(g->d_sys, sds.data(), nsys * sizeof(SysDev), cudaMemcpyHostToDevice), "cudaMemcpy");
  if (st != LHF_OK) return cleanup(st);
  if (ps[0].mixed) {
    std::vector<unsigned char> hbuf(lhf::gram_tc_args_bytes(sds.data(), nsys));
    cudaError_t e = lhf::gram_tc_prepare(sds.data(), nsys, hbuf.data(), hbuf.size(), &g->tc_jobs, &g->tc_off);
    if (e == cudaErrorNotSupported) return cleanup(c->fail(LHF_ERR_UNSUPPORTED, "shape outside the tensor-core kernel's limits"));
    st = c->cuda(e, "tensor-core preparation");
    if (st != LHF_OK) return cleanup(st);
    st = c->cuda(cudaMalloc(&g->tc_dev, hbuf.size()), "cudaMalloc");
    if (st != LHF_OK) return cleanup(st);
    st = c->cuda(cudaMemcpy(g->tc_dev, hbuf.data(), hbuf.size(), cudaMemcpyHostToDevice), "cudaMemcpy");
    if (st != LHF_OK) return cleanup(st);
  }
  // capture on a private stream (the legacy default stream cannot be captured)
  cudaStream_t cs = nullptr;
  st = c->cuda(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
  if (st != LHF_OK) return cleanup(st);
  SysDev *saved_sys = c->d_sys;
  cudaStream_t saved_stream = c->stream;
  const bool saved_prof = c->prof;
  c->d_sys = g->d_sys;
  c->stream = cs;
  c->prof = false;
  c->graph_tc = g->tc_dev;
  c->graph_tc_jobs = g->tc_jobs;
  c->graph_tc_off = g->tc_off;
  c->capturing = true;  // no autotuning (it synchronises) inside the capture
  lhf_status run = c->cuda(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  if (run == LHF_OK) {
    run = run_assembly(c, ps);
    if (run == LHF_OK) run = run_dft(c, ps);
    if (run == LHF_OK) run = run_eig(c, ps);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (run == LHF_OK) run = c->cuda(e, "cudaStreamEndCapture");
    g->graph = graph;
  }
  c->d_sys = saved_sys;
  c->stream = saved_stream;
  c->prof = saved_prof;
  c->graph_tc = nullptr;
  c->graph_tc_jobs = 0;
  c->graph_tc_off = 0;
  c->capturing = false;
  cudaStreamDestroy(cs);
  if (run != LHF_OK) return cleanup(run);
  st = c->cuda(cudaGraphInstantiate(&g->exec, g->graph, 0), "cudaGraphInstantiate");
  if (st != LHF_OK) return cleanup(st);
  g->nsys = nsys;
  *out = g;
  return LHF_OK;
}

lhf_status lhf_graph_launch(lhf_graph *g) {
  if (!g || !g->exec) return LHF_ERR_ARG;
  if (!g->ctx) return LHF_ERR_STATE;  // its context was destroyed
  return g->ctx->cuda(cudaGraphLaunch(g->exec, g->ctx->stream), "cudaGraphLaunch");
}

void lhf_graph_destroy(lhf_graph *g) {
  if (!g) return;
  if (g->ctx) {
    cudaStreamSynchronize(g->ctx->stream);
    g->ctx->graphs.erase(g);
  } else {
    cudaDeviceSynchronize();  // detached: its context (and stream) are gone
  }
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->tc_dev) cudaFree(g->tc_dev);
  if (g->d_sys) cudaFree(g->d_sys);
  if (g->ws) cudaFree(g->ws);
  cudaGetLastError();
  delete g;
}

lhf_status lhf_bloch_spectra_host(lhf_ctx *c, int nsys, const lhf_system_desc *systems, lhf_precision prec,
                                  double *eig_host, int *kstat_host) {
  if (!c) return LHF_ERR_ARG;
  if (nsys < 1 || !systems || !eig_host) return c->fail(LHF_ERR_ARG, "nsys >= 1, systems and eig_host are required");
  // count outputs first (from the validated descriptors: L0 L1 L2 blocks or k-points and m0
  // values each, periodic or box; the plans are made once, by lhf_bloch_spectra)
  size_t neig = 0, nk = 0;
  for (int i = 0; i < nsys; ++i) {
    HostSystem hs;
    lhf_status st = system_from_desc(c, &systems[i], hs);
    if (st != LHF_OK) return st;
    const size_t nb = (size_t)hs.L[0] * hs.L[1] * hs.L[2];
    neig += nb * hs.m0;
    nk += nb;
  }
  const size_t need = align_up(neig) + (nk + 1) / 2 + 1;
  if (need > c->out_cap) {
    lhf_status st = c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (st != LHF_OK) return st;
    if (c->d_out) cudaFree(c->d_out);
    c->d_out = nullptr;
    c->out_cap = 0;
    st = c->cuda(cudaMalloc(&c->d_out, need * sizeof(double)), "cudaMalloc");
    if (st != LHF_OK) return st;
    c->out_cap = need;
  }
  double *d_out = c->d_out;
  int *d_k = reinterpret_cast<int *>(d_out + align_up(neig));
  lhf_status st = lhf_bloch_spectra(c, nsys, systems, prec, d_out, d_k);
  if (st != LHF_OK) return st;
  st = c->cuda(cudaMemcpyAsync(eig_host, d_out, neig * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
  if (st != LHF_OK) return st;
  if (kstat_host) {
    st = c->cuda(cudaMemcpyAsync(kstat_host, d_k, nk * sizeof(int), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
    if (st != LHF_OK) return st;
  }
  return c->cuda(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
}

lhf_status lhf_basis_factors(lhf_ctx *c, int l, double *G) {
  if (!c) return LHF_ERR_ARG;
  if (l < 0 || l > 2 || !G) return c->fail(LHF_ERR_ARG, "direction 0..2 and an output pointer are required");
  std::vector<Plan> ps(1);
  lhf_status st = current_plan(c, ps[0]);
  if (st != LHF_OK) return st;
  st = ensure_ws(c, ps[0].ws);
  if (st != LHF_OK) return st;
  bind_ws(ps[0], c->ws);
  st = upload(c, {ps[0].sd});
  if (st != LHF_OK) return st;
  const DirDev &D = ps[0].sd.d[l];
  // the basis kernel writes only the support windows of periodic rows: the rest are zeros
  st = c->cuda(cudaMemsetAsync(c->ws + D.offG, 0, sizeof(double) * (size_t)ps[0].sd.m0 * (D.n + D.gext), c->stream),
               "cudaMemsetAsync");
  if (st != LHF_OK) return st;
  st = c->cuda(lhf::launch_basis(c->d_sys, 1, ps[0].basis_items, c->stream), "basis kernel");
  if (st != LHF_OK) return st;
  // rows of n nodes out of rows of gext + n samples
  return c->cuda(cudaMemcpy2DAsync(G, sizeof(double) * (size_t)D.n, c->ws + D.offG + D.gext,
                                   sizeof(double) * (size_t)(D.n + D.gext), sizeof(double) * (size_t)D.n,
                                   (size_t)ps[0].sd.m0, cudaMemcpyDeviceToDevice, c->stream),
                 "cudaMemcpy2DAsync");
}

lhf_status lhf_bloch_orbitals(lhf_ctx *c, const int *kappa, int norb, const double *coef, const int *lo,
                              const int *cnt, double *out) {
  if (!c) return LHF_ERR_ARG;
  if (!kappa || !coef || !lo || !cnt || !out || norb < 1)
    return c->fail(LHF_ERR_ARG, "kappa, coef, lo, cnt, out and norb >= 1 are required");
  std::vector<Plan> ps(1);
  lhf_status st = current_plan(c, ps[0]);
  if (st != LHF_OK) return st;
  Plan &P = ps[0];
  if (P.sd.box) return c->fail(LHF_ERR_UNSUPPORTED, "Bloch orbitals need a periodic lattice");
  int maxcnt = 0, maxL = 1;
  long long npts = 1;
  for (int l = 0; l < 3; ++l) {
    const DirDev &D = P.sd.d[l];
    if (kappa[l] < 0 || kappa[l] >= D.L) return c->fail(LHF_ERR_ARG, "kappa[%d] = %d outside [0, %d)", l, kappa[l], D.L);
    if (lo[l] < 0 || cnt[l] < 1 || (long long)lo[l] + cnt[l] > D.n)
      return c->fail(LHF_ERR_ARG, "direction %d: nodes [%d, %d + %d) outside [0, %d)", l, lo[l], lo[l], cnt[l], D.n);
    maxcnt = std::max(maxcnt, cnt[l]);
    maxL = std::max(maxL, D.L);
    npts *= cnt[l];
  }
  if (npts * norb > (1ll << 31)) return c->fail(LHF_ERR_ARG, "too many output values");
  const size_t boff = P.ws;
  st = ensure_ws(c, boff + align_up((size_t)6 * P.sd.m0 * maxcnt));
  if (st != LHF_OK) return st;
  bind_ws(P, c->ws);
  st = upload(c, {P.sd});
  if (st != LHF_OK) return st;
  for (int l = 0; l < 3; ++l) {  // rows zero outside the support windows the basis kernel writes
    const DirDev &D = P.sd.d[l];
    st = c->cuda(cudaMemsetAsync(c->ws + D.offG, 0, sizeof(double) * (size_t)P.sd.m0 * (D.n + D.gext), c->stream),
                 "cudaMemsetAsync");
    if (st != LHF_OK) return st;
  }
  st = c->cuda(lhf::launch_basis(c->d_sys, 1, P.basis_items, c->stream), "basis kernel");
  if (st != LHF_OK) return st;
  return c->cuda(lhf::launch_orbitals(c->d_sys, kappa, lo, cnt, norb, coef, c->ws + boff, out, P.sd.m0, maxL,
                                      c->stream),
                 "orbital kernels");
}

lhf_status lhf_cell_energies(lhf_ctx *c, int nseg, const double *eig, const long long *off, const int *cnt,
                             const int *n_low, const double *cells, double *energy, double *level) {
  if (!c) return LHF_ERR_ARG;
  if (nseg < 1 || !eig || !off || !cnt || !n_low || !cells || !energy)
    return c->fail(LHF_ERR_ARG, "nseg >= 1, eig, off, cnt, n_low, cells and energy are required");
  if (nseg > (1 << 30)) return c->fail(LHF_ERR_ARG, "nseg = %d too large", nseg);
  std::vector<lhf::SpectrumSeg> seg((size_t)nseg);
  for (int s = 0; s < nseg; ++s) {
    if (off[s] < 0 || cnt[s] < 1 || n_low[s] < 1 || n_low[s] > cnt[s] || !(cells[s] > 0.0))
      return c->fail(LHF_ERR_ARG, "spectrum %d: off = %lld, cnt = %d, n_low = %d, cells = %g", s, off[s], cnt[s],
                     n_low[s], cells[s]);
    seg[s] = lhf::SpectrumSeg{off[s], cnt[s], n_low[s], cells[s]};
  }
  const size_t bytes = seg.size() * sizeof(lhf::SpectrumSeg);
  lhf_status st = ensure_ws(c, (bytes + sizeof(double) - 1) / sizeof(double));
  if (st != LHF_OK) return st;
  auto *d_seg = reinterpret_cast<lhf::SpectrumSeg *>(c->ws);
  st = c->cuda(cudaMemcpyAsync(d_seg, seg.data(), bytes, cudaMemcpyHostToDevice, c->stream), "cudaMemcpyAsync");
  if (st != LHF_OK) return st;
  // a pageable source is staged before the call returns; the stream orders the kernel after it
  return c->cuda(lhf::launch_cell_energy(eig, d_seg, nseg, energy, level, c->stream), "cell energy kernel");
}

lhf_status lhf_potential_factors(lhf_ctx *c, int l, double *V) {
  if (!c) return LHF_ERR_ARG;
  if (l < 0 || l > 2 || !V) return c->fail(LHF_ERR_ARG, "direction 0..2 and an output pointer are required");
  std::vector<Plan> ps(1);
  lhf_status st = current_plan(c, ps[0]);
  if (st != LHF_OK) return st;
  st = ensure_ws(c, ps[0].ws);
  if (st != LHF_OK) return st;
  bind_ws(ps[0], c->ws);
  st = upload(c, {ps[0].sd});
  if (st != LHF_OK) return st;
  st = upload_zcell(c, ps);
  if (st != LHF_OK) return st;
  st = c->cuda(lhf::launch_potential(c->d_sys, 1, ps[0].pot_rows, c->stream), "potential kernel");
  if (st != LHF_OK) return st;
  const DirDev &D = ps[0].sd.d[l];
  return c->cuda(cudaMemcpyAsync(V, c->ws + D.offV, sizeof(double) * (size_t)ps[0].sd.Rt * D.nv,
                                 cudaMemcpyDeviceToDevice, c->stream),
                 "cudaMemcpyAsync");
}

lhf_status lhf_gram_factors(lhf_ctx *c, lhf_precision prec, int l, double *C, int *jlo) {
  if (!c) return LHF_ERR_ARG;
  if (l < 0 || l > 2 || !C) return c->fail(LHF_ERR_ARG, "direction 0..2 and an output pointer are required");
  lhf_status st = check_precision(c, prec);
  if (st != LHF_OK) return st;
  std::vector<Plan> ps(1);
  st = current_plan(c, ps[0], prec == LHF_MIXED);
  if (st != LHF_OK) return st;
  st = ensure_ws(c, ps[0].ws);
  if (st != LHF_OK) return st;
  bind_ws(ps[0], c->ws);
  st = upload(c, {ps[0].sd});
  if (st != LHF_OK) return st;
  const size_t mm = (size_t)ps[0].sd.m0 * ps[0].sd.m0;
  if (ps[0].sd.box) {
    st = run_box_factors(c, ps);
    if (st != LHF_OK) return st;
    if (l == 0) {  // [L0][bJ][Rt+2][m0][m0]: cells p and p + bjlo + dd
      if (jlo) *jlo = ps[0].sd.bjlo;
      return c->cuda(cudaMemcpyAsync(C, c->ws + ps[0].sd.offCb,
                                     sizeof(double) * (size_t)ps[0].sd.d[0].L * ps[0].sd.bJ * (ps[0].sd.Rt + 2) * mm,
                                     cudaMemcpyDeviceToDevice, c->stream),
                     "cudaMemcpyAsync");
    }
  } else {
    st = c->cuda(lhf::launch_basis(c->d_sys, 1, ps[0].basis_items, c->stream), "basis kernel");
    if (st != LHF_OK) return st;
    st = c->cuda(lhf::launch_potential(c->d_sys, 1, ps[0].pot_rows, c->stream), "potential kernel");
    if (st != LHF_OK) return st;
    st = run_gram(c, ps, true);
    if (st != LHF_OK) return st;
  }
  const DirDev &D = ps[0].sd.d[l];
  if (jlo) *jlo = D.jlo;
  return c->cuda(cudaMemcpyAsync(C, c->ws + D.offC, sizeof(double) * (size_t)D.J * (ps[0].sd.Rt + 2) * mm,
                                 cudaMemcpyDeviceToDevice, c->stream),
                 "cudaMemcpyAsync");
}

}  // extern "C"
