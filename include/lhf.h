/*
 * lhf.h -- C ABI of the GB300 lattice core-Hamiltonian library (liblhf.so).
 *
 * Method: Khoromskaia & Khoromskij, "Tensor numerical approach to linearized Hartree-Fock
 * equation for lattice-type and periodic systems" (arXiv:1408.3839).  The library assembles the
 * Galerkin matrices of the core Hamiltonian h = -1/2 Laplacian - v_c (eqs. (3.1), (3.4)) and of
 * the overlap in a lattice-translated separable Gaussian basis, block-diagonalises the
 * block-circulant matrices of a periodic lattice by a DFT along the lattice indices (Lemma 2.2,
 * Prop. 6.1) and solves the small generalized Hermitian eigenproblems at every k-point
 * (eq. (4.7)).  Every step runs in this library's CUDA kernels on one GPU; there is no CPU path.
 *
 * Conventions common to all calls
 *   - Units are atomic (bohr, Hartree).  Directions l = 0, 1, 2.
 *   - Device pointers are caller-owned CUDA device memory; host pointers are plain host memory.
 *     The library never frees caller memory.  It owns only its context and internal workspace.
 *   - Calls are asynchronous on the context's CUDA stream (set at creation or by
 *     lhf_set_stream).  Arguments are validated on the host before any launch; an invalid
 *     argument returns LHF_ERR_ARG and launches nothing.  Conditions found on the device (a
 *     k-point overlap block that is not positive definite) are reported per k-point through
 *     k_status and summarised by the next lhf_sync.
 *   - No call throws; every call returns an lhf_status.  lhf_last_error gives a message for the
 *     last failing call on that context.
 *   - Matrices are row-major FP64.  Complex arrays are interleaved (re, im) FP64.
 *   - A context is not thread-safe: use one context per host thread.
 */
#ifndef LHF_H
#define LHF_H

#ifdef __cplusplus
extern "C" {
#endif

#define LHF_MAX_M0 32     /* basis functions per cell */
#define LHF_MAX_NUCLEI 8  /* nuclei per cell */
#define LHF_MAX_R 64      /* sinc-quadrature terms */

typedef enum {
    LHF_OK = 0,
    LHF_ERR_ARG = -1,         /* invalid argument or descriptor; nothing was launched */
    LHF_ERR_CUDA = -2,        /* a CUDA runtime call failed (message in lhf_last_error) */
    LHF_ERR_NOT_SPD = -3,     /* an overlap block was not positive definite (see k_status) */
    LHF_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
    LHF_ERR_UNSUPPORTED = -5, /* valid input outside what this build supports */
    LHF_ERR_STATE = -6,       /* call order violated (e.g. assemble before setup) */
    LHF_ERR_NOMEM = -7,       /* workspace allocation failed */
    LHF_ERR_NOT_CONVERGED = -8 /* an iterative solver stopped above its tolerance */
} lhf_status;

/* Arithmetic route.  Potential factors, rank sum and DFT are FP64 in both modes.
 *   LHF_FP64:   FP64 CUDA-core Gram contraction; FP64 k-point reduction.
 *   LHF_MIXED:  tensor-core Gram contraction (tcgen05) on BF16 slices of the FP64 operands with
 *               exact FP32 accumulation per slice pair, recombined in FP64; the k-point
 *               reduction of the Cholesky route (Cholesky, triangular solves, Householder) in
 *               compensated pairs of FP32 words (48 significant bits, compensated dot products),
 *               the canonical route, Jacobi and the tridiagonal eigenvalues in FP64.  Target:
 *               eigenvalues within 1e-6 Ha of the FP64 ones (measured: within the FP64 route's
 *               perturbation bound, 3.5e-11 Ha on the benchmark system). */
typedef enum { LHF_FP64 = 0, LHF_MIXED = 1 } lhf_precision;

typedef struct lhf_ctx lhf_ctx;

/* Lattice (Sec. 3.2, Sec. 4.1).  L[l] cells of side b[l] per direction; periodic[l] = 1 makes
 * direction l block-circulant (supercell of L[l] cells, basis periodised over L[l] b[l]).
 * M0 nuclei per cell with charges Z[nu] > 0 at positions a[3 nu + l] (coordinates of the copy in
 * lattice cell 0).  K_sum[l] = number of lattice images in the periodic potential sum of
 * direction l (images k = -floor(K/2) .. floor(K/2), weight 1/2 on |k| = K/2 for even K; the sum
 * is evaluated in cell 0 and replicated, eq. (4.1)).  Open directions ignore K_sum.  Z_cell
 * (optional, NULL otherwise) gives per-cell charges Z_cell[k M0 + nu] of an open box whose only
 * lattice direction is l = 0 (eq. (3.8)).  L[l] is 1 .. 4096, except that a one-dimensional
 * lattice (L[1] = L[2] = 1) may have up to 32768 cells along l = 0 when L[0] splits as A B with
 * A, B <= 4096 (its block DFT then runs as two passes of such lengths).  Host pointers; copied
 * during setup. */
typedef struct {
    int L[3];
    double b[3];
    int periodic[3];
    int K_sum[3];
    int M0;
    const double *Z;
    const double *a;
    const double *Z_cell;
} lhf_lattice_desc;

/* Separable Gaussian basis of one cell (eq. (3.14)): m0 functions; kind[mu] = 0 (s) or 1 + d
 * (p along direction d); exponent alpha[mu] > 0; centre[3 mu + l] (cell-0 coordinates).  1D
 * factors: exp(-alpha d^2), or sqrt(2 alpha e) d exp(-alpha d^2) along a p function's own
 * direction (unit peak); each factor is cut to zero where |d| > sqrt(rho / alpha).  The copy
 * in lattice cell k is shifted by k b.  Host pointers; copied during setup. */
typedef struct {
    int m0;
    const int *kind;
    const double *alpha;
    const double *centre;
    double rho;
} lhf_basis_desc;

/* Tensor grid and potential quadrature (Sec. 3.2, Sec. 3.4).  Nodes x_i = x0[l] + (i + 1/2) h[l],
 * i = 0 .. n[l]-1, serve both as P1 nodes (kinetic, overlap) and as centres of the cells of the
 * piecewise-constant potential.  In a lattice direction (periodic, or open with L > 1) lattice
 * cell k spans [cell0 + k b, cell0 + (k+1) b) and holds n_cell[l] = b / h nodes; a periodic
 * direction requires n[l] = L[l] n_cell[l] and x0[l] = cell0[l].  A single-cell open
 * direction uses n_cell[l] = n[l].  Newton kernel: R sinc terms, t_q = exp(u0 + q du),
 * w_q = 2/sqrt(pi) du t_q, with w_0 divided by (1 - exp(-du)) (the nodes below u0 folded into
 * the first one), eq. (3.6). */
typedef struct {
    int n[3];
    int n_cell[3];
    double h[3];
    double x0[3];
    double cell0[3];
    int R;
    double u0;
    double du;
} lhf_grid_desc;

typedef struct {
    lhf_lattice_desc lattice;
    lhf_basis_desc basis;
    lhf_grid_desc grid;
} lhf_system_desc;

/* Sizes of the current system (after the three setup calls). */
typedef struct {
    int m0;             /* basis functions per cell */
    int n_blocks;       /* L0 L1 L2: blocks of the first block column (periodic) */
    int n_kpoints;      /* = n_blocks; eigenvalue rows */
    int n_basis;        /* N_b = m0 L0 L1 L2 */
    int rank;           /* R_tot = M0 R rank terms of the potential */
    int window[3];      /* blocks computed per direction (overlap window, <= L) */
    int n_potential[3]; /* length of each direction's potential factor (n_cell periodic, else n) */
    int periodic;       /* 1 if every direction with L > 1 is periodic */
    int desc_bytes;     /* bytes of the device descriptor copied host -> device per system and call */
    int overlap_rows[3]; /* rows (contracted window block j >= 0, mu, nu) of each direction's weighted
                            Gram whose two functions share a cell; the other rows' factors are exact
                            zeros and are not contracted (0 where the direction has no such Gram) */
} lhf_sizes;

/* Context creation.  device: CUDA ordinal; stream: a cudaStream_t (NULL = default stream).
 * *out receives the context (NULL on failure). */
lhf_status lhf_create(lhf_ctx **out, int device, void *stream);
void lhf_destroy(lhf_ctx *ctx);
const char *lhf_last_error(const lhf_ctx *ctx);
lhf_status lhf_set_stream(lhf_ctx *ctx, void *stream);
/* Wait for the context stream; returns LHF_ERR_NOT_SPD if any k-point since the last sync
 * reported a non-positive-definite overlap, LHF_ERR_CUDA on a CUDA error. */
lhf_status lhf_sync(lhf_ctx *ctx);

/* Setup of the current system (Sec. 3.2-3.4 define its parts).  Each call validates its
 * descriptor and keeps a copy; the three together define the problem. */
lhf_status lhf_lattice_setup(lhf_ctx *ctx, const lhf_lattice_desc *lattice);
lhf_status lhf_basis_setup(lhf_ctx *ctx, const lhf_basis_desc *basis);
lhf_status lhf_grid_setup(lhf_ctx *ctx, const lhf_grid_desc *grid);
lhf_status lhf_query_sizes(lhf_ctx *ctx, lhf_sizes *out);

/* Core Hamiltonian and overlap (eqs. (3.4), (3.10); Lemma 4.1 eqs. (4.2), (4.5), (4.6)).
 * Periodic lattice: H, S receive the first block column A_j[mu][nu] = <g_{mu,j}, H g_{nu,0}>,
 * layout [L0][L1][L2][m0][m0] (j = (j0, j1, j2)); blocks outside the overlap window are exact
 * zeros.  Open box (periodic = 0 in a lattice direction): H, S receive the full [N_b][N_b]
 * matrices, index (cell, mu).  Device pointers of n_blocks m0^2 (periodic) or N_b^2 doubles. */
lhf_status lhf_assemble_core_hamiltonian(lhf_ctx *ctx, lhf_precision precision, double *H, double *S);

/* Block DFT along the lattice indices (Prop. 6.1 eq. (6.6), Lemma 2.2 eq. (2.1)):
 * Xbar_kappa = sum_j omega^{kappa . j} X_j, omega_l = exp(-2 pi i / L_l), for X = H, S given
 * as first block columns [L0][L1][L2][m0][m0] (device).  Hbar, Sbar: device, complex
 * interleaved [L0][L1][L2][m0][m0][2].  Periodic lattices only. */
lhf_status lhf_circulant_fft(lhf_ctx *ctx, const double *H, const double *S, double *Hbar,
                             double *Sbar);

/* The k-point blocks of a periodic lattice by the separable route (Theorem 2.5, Prop. 4.2): the
 * per-direction factors of steps a3-a4 (in the given precision) are transformed by 1D DFTs along
 * their own lattice index, Fl_r(kappa_l) = sum_{j_l} omega_l^{kappa_l j_l} Cl_r[j_l], and each
 * k-point block is assembled from their Hadamard products: Sbar = M0 M1 M2, Hbar = (K0 M1 M2 +
 * M0 K1 M2 + M0 M1 K2) / 2 - sum_r c_r C0_r C1_r C2_r (entry-wise, complex).  Same result as
 * lhf_assemble_core_hamiltonian followed by lhf_circulant_fft up to rounding, without forming
 * the real-space blocks; the workspace holds sum_l L_l (R_tot + 2) m0^2 complex factor entries.
 * Hbar, Sbar: device, complex interleaved [L0][L1][L2][m0][m0][2]. */
lhf_status lhf_kspace_blocks(lhf_ctx *ctx, lhf_precision precision, double *Hbar, double *Sbar);

/* Generalized Hermitian eigenproblems Hbar_kappa u = lambda Sbar_kappa u at every k-point
 * (eq. (4.7); spectrum = union over kappa, eq. (6.7)).  Inputs as produced by
 * lhf_circulant_fft (device): blocks of a real lattice matrix, so that Xbar at -kappa is the
 * complex conjugate of Xbar at kappa; one k-point of each conjugate pair is solved and its
 * eigenvalues are written to both.  eig: device [n_kpoints][m0], ascending per k-point.
 * FP64 data resolve a Bloch function whose overlap diagonal has cancelled to a fraction r of
 * its cell-periodic norm only to about eps / r relative: with s0_i = mean over kappa of
 * Re Sbar_ii, function i is removed at kappa when Re Sbar_ii(kappa) <= LHF_DROP_TOL s0_i (at
 * 1e-6 its scaled overlap row is still good to ~2e-10, far below LHF_LINDEP_TOL); the remaining
 * pencil is diagonally scaled, reduced (Cholesky), brought to real tridiagonal form by
 * Householder reflections, and each eigenvalue of the tridiagonal matrix is isolated by Sturm
 * bisection and refined by Newton's iteration on its characteristic polynomial; removed slots hold
 * +INFINITY (sorted last).  k_status: device [n_kpoints] (may be NULL): the number of removed
 * functions (>= 0), or LHF_ERR_NOT_SPD when the reduced overlap is not positive definite (the
 * eigenvalues of such a k-point are NaN). */
#define LHF_DROP_TOL 1e-6
/* The kept pencil is scaled to unit overlap diagonal; where the scaled overlap may be nearly
 * singular (a Cholesky pivot below 1e-5, or trace(S~^-1) above 1 / LHF_LINDEP_TOL) the k-point
 * is solved by canonical orthogonalisation,
 * dropping the overlap eigen-directions below LHF_LINDEP_TOL (their slots also hold +INFINITY
 * and are counted in k_status). */
#define LHF_LINDEP_TOL 1e-8
lhf_status lhf_k_point_eigensolve(lhf_ctx *ctx, const double *Hbar, const double *Sbar,
                                  double *eig, int *k_status);

/* Bloch eigenvectors (Prop. 6.1, eq. (6.8)): the eigenpairs Hbar_kappa u = lambda Sbar_kappa u at
 * every k-point, inputs and eig / k_status as for lhf_k_point_eigensolve (same removal,
 * scaling and Cholesky-or-canonical reduction; the reduced Hermitian matrix is diagonalised by
 * cyclic Jacobi with accumulated rotations at every k-point).  vecs: device, complex interleaved
 * [n_kpoints][m0][m0]: row r of k-point kappa is the eigenvector u of the r-th smallest
 * eigenvalue, components over the m0 cell functions, normalised to u^H Sbar_kappa u = 1 on the
 * kept functions (removed functions have component 0; dropped slots are zero rows, rows of a
 * k-point whose overlap is not positive definite are NaN).  Its phase is fixed: the first
 * component of largest magnitude is real and positive.  The vectors at -kappa are the complex
 * conjugates of those at kappa.  The eigenvector of the lattice matrix for (kappa, r) is
 * x_p = exp(2 pi i kappa . p / L) u / sqrt(L0 L1 L2) on cell p (eq. (6.8)). */
lhf_status lhf_k_point_eigenvectors(lhf_ctx *ctx, const double *Hbar, const double *Sbar, double *eig,
                                    double *vecs, int *k_status);

/* Bloch orbitals on the grid (eq. (6.8) expanded in the basis, eq. (3.14)): for k-point kappa
 * (host [3], 0 <= kappa_l < L_l) and Bloch vectors coef (device, complex [norb][m0], e.g. rows of
 * lhf_k_point_eigenvectors), the values on the grid window lo[l] .. lo[l] + cnt[l] - 1 (host [3])
 * of psi(x) = (L0 L1 L2)^{-1/2} sum_p exp(2 pi i kappa . p / L) sum_mu coef_mu phi_mu(x - p b),
 * summed over all lattice cells p, in the rank-m0 separable form
 * sum_mu coef_mu prod_l Bl_mu(i_l) with Bl_mu(i) = sum_p exp(2 pi i kappa_l p / L_l) g_mu^l(i - p n_c).
 * out: device, complex interleaved [norb][cnt0][cnt1][cnt2].  Periodic lattices only.  With
 * coef S-normalised the orbital has unit norm in the P1 mass inner product of the grid. */
lhf_status lhf_bloch_orbitals(lhf_ctx *ctx, const int *kappa, int norb, const double *coef, const int *lo,
                              const int *cnt, double *out);

/* Energy per cell of the lowest states (Sec. 5, the average energy per unit cell of a (L,1,1)
 * chain against L, open and periodic): for each of nseg spectra, held on the device in
 * eig[off[s] .. off[s] + cnt[s]) -- the eigenvalues of all k-points of one lattice (their union is
 * the lattice matrix's spectrum, Prop. 6.1) or of one open box -- energy[s] = (sum of the n_low[s]
 * smallest values) / cells[s], and level[s] = the n_low[s]-th smallest value (the highest
 * selected state).  Equal values are counted with multiplicity; the selected set and level do not
 * depend on the order of the values within a segment (the sum's rounding may), and repeated calls
 * agree bit for bit.  +inf (removed functions, see
 * lhf_k_point_eigensolve) sorts last: a segment with fewer than n_low[s] finite values gets
 * energy = level = +inf.  NaN values give an undefined result.
 * eig, energy, level: device (level may be NULL); off, cnt, n_low, cells: host arrays [nseg] with
 * off[s] >= 0, 1 <= n_low[s] <= cnt[s], cells[s] > 0 (else LHF_ERR_ARG).  Uses the context's
 * workspace (nseg records of 24 bytes). */
lhf_status lhf_cell_energies(lhf_ctx *ctx, int nseg, const double *eig, const long long *off, const int *cnt,
                             const int *n_low, const double *cells, double *energy, double *level);

/* Generalized symmetric-definite eigenvalues of dense N x N matrices (open box, Table 4.1's
 * full eigensolver): H x = lambda S x.  Device pointers; eig [N] ascending. */
lhf_status lhf_dense_eigensolve(lhf_ctx *ctx, const double *H, const double *S, int N, double *eig);

/* The n_ev lowest eigenvalues of an open (L,1,1) box (Sec. 3.3, eqs. (3.8)-(3.10); the box case of
 * Table 4.1) without the dense eigensolve, for boxes beyond it (N_b = m0 L up to 4096 cells).
 * The box's H and S are block-banded -- the block of cells (p, q) vanishes outside the overlap
 * window (Lemma 3.1) -- and their overlap and kinetic parts are block-Toeplitz; the solver is
 * block LOBPCG in FP64 on the banded matrices.  Its start block is a seeded block preconditioned
 * by the block-circulant matrix whose blocks are the band's diagonals averaged over the rows (the
 * Toeplitz-to-circulant embedding of Remark 2.4, padded to a power of two of at least L + window
 * cells), which the DFT along the cells block-diagonalises (Lemma 2.2): one m0 x m0 Cholesky
 * solve per k-point, shifted just below that circulant's spectrum.  The iterations are
 * preconditioned by (H - sigma S)^{-1} itself, factored exactly as a block-tridiagonal Cholesky
 * over super-cells that span the band, with sigma below the box's lowest eigenvalue (lowered
 * until the factorisation succeeds).
 *   box: one system, open along direction 0 (the lhf_bloch_spectra box layout); n_ev: 1 .. 20
 *   (at most N_b); tol: convergence when every one of the n_ev residuals ||H x - theta S x|| (x
 *   S-normalised) is at most tol max(1, |theta|) -- an eigenvalue is then accurate to about
 *   ||r||^2 / (its gap to the rest of the spectrum); max_iter >= 1.
 *   eig: device [n_ev], ascending (written also when not converged); iterations, residual: host,
 *   optional: iterations run and the largest scaled residual at exit.
 * Synchronising.  Returns LHF_OK, LHF_ERR_NOT_CONVERGED (eig holds the last Ritz values),
 * LHF_ERR_ARG, LHF_ERR_UNSUPPORTED (a circulant of more than 8192 cells would be needed),
 * LHF_ERR_NOT_SPD, LHF_ERR_NOMEM or LHF_ERR_CUDA. */
lhf_status lhf_box_lowest_eigenvalues(lhf_ctx *ctx, const lhf_system_desc *box, int n_ev, double tol, int max_iter,
                                      double *eig, int *iterations, double *residual);

/* Batched Bloch spectra: for every system s of an array of nsys periodic lattices, the whole
 * path (basis and potential factors, Grams, rank sum, block DFT, k-point eigensolves) in one
 * pass of batched launches.  eig: device, systems concatenated, system s at offset
 * sum_{t<s} n_kpoints(t) m0(t), conventions of lhf_k_point_eigensolve.  k_status: device (may
 * be NULL), concatenated likewise.
 * Scratch memory is the context's workspace (grown on demand).  The context keeps each system's
 * plan (its layout and launch extents, a pure function of the descriptor's content, the
 * precision and the rank-reduction setting) and reuses it when a later call passes the same
 * content; at most 1024 plans are kept. */
lhf_status lhf_bloch_spectra(lhf_ctx *ctx, int nsys, const lhf_system_desc *systems,
                             lhf_precision precision, double *eig, int *k_status);

/* The batched path of lhf_bloch_spectra captured once into a CUDA graph and replayed by
 * lhf_graph_launch on the context stream (one graph launch instead of a dozen kernel launches
 * and no host work per replay).  The graph owns its workspace and descriptors; every replay
 * recomputes the same systems into the same eig / k_status device buffers (which must outlive
 * the graph).  Periodic lattices only (LHF_ERR_UNSUPPORTED for open boxes).  Destroy the graph
 * before its context when possible (lhf_graph_destroy then waits for the context stream); a
 * context destroyed first detaches its graphs: lhf_graph_launch on them returns LHF_ERR_STATE and
 * lhf_graph_destroy still frees them (after a device-wide synchronisation). */
typedef struct lhf_graph lhf_graph;
lhf_status lhf_graph_create(lhf_ctx *ctx, int nsys, const lhf_system_desc *systems, lhf_precision precision,
                            double *eig, int *k_status, lhf_graph **out);
lhf_status lhf_graph_launch(lhf_graph *graph);
void lhf_graph_destroy(lhf_graph *graph);

/* Same as lhf_bloch_spectra with a HOST output buffer: the call copies the eigenvalues back
 * and returns after the stream has finished (synchronising). */
lhf_status lhf_bloch_spectra_host(lhf_ctx *ctx, int nsys, const lhf_system_desc *systems,
                                  lhf_precision precision, double *eig_host, int *k_status_host);

/* Stage outputs of the current system, for verification (same kernels as the full path).
 * lhf_basis_factors: 1D basis samples of direction l for the cell-0 copies, [m0][n_l]
 * (periodic directions periodised), eq. (3.14).
 * lhf_potential_factors: 1D potential factors of direction l, [R_tot][n_potential_l], rank
 * r = nu R + q, eqs. (3.5), (3.9), (4.1).
 * lhf_gram_factors: per-direction factors for the window blocks j = jlo .. jlo+J-1 (mod L),
 * [J][R_tot + 2][m0][m0]: slots r < R_tot hold the weighted Grams sum_i g_{mu,j} v_r g_{nu,0},
 * slot R_tot the P1 stiffness form, slot R_tot + 1 the P1 mass form (Lemma 3.1 proof, Sec. 3.4).
 * *jlo receives the first displacement of the window (host int, may be NULL). */
lhf_status lhf_basis_factors(lhf_ctx *ctx, int l, double *G);
lhf_status lhf_potential_factors(lhf_ctx *ctx, int l, double *V);
lhf_status lhf_gram_factors(lhf_ctx *ctx, lhf_precision precision, int l, double *C, int *jlo);

/* Launch-shape autotuner (enabled by default).  The first time a context solves the k-points of
 * a batch class -- (m0, route, log2 of the number of solved matrices) -- it times each candidate
 * launch shape of the eigensolver kernels (k-points per CTA of the reduction kernel: 1, 2, 4, 8;
 * threads per CTA of the tridiagonal kernel: 32 .. 256) once on that batch, synchronising the
 * stream, and keeps the fastest for the class.  The shape changes no result (every k-point is
 * solved by the same code in any shape).  Graph capture uses the shapes tuned before it (else
 * the defaults 4 and 128): tune a class with one direct call before capturing it.
 * lhf_launch_shapes reports the shapes of the last k-point solve (host outputs). */
lhf_status lhf_set_autotune(lhf_ctx *ctx, int enable);
lhf_status lhf_launch_shapes(lhf_ctx *ctx, int *eig_warps, int *tri_threads);

/* Live stage timing.  With profiling enabled, every launch of the path is bracketed by CUDA
 * events recorded on the context stream (no synchronisation is added).  lhf_stage_times waits
 * for the stream, adds the elapsed times of all launches recorded since the previous call into
 * ms[stage] and the number of kernels launched into launches[stage] (memory fills and copies
 * for stages 6 and 7) (arrays of LHF_NUM_STAGES, host), and clears
 * the record.  Stages: 0 basis samples (a1), 1 potential factors (a2), 2 Gram factors (a3-a4:
 * the FP64 contraction, or the folding and digit slicing of LHF_MIXED), 3 rank sum (a5; open
 * box: dense assembly; the zero blocks outside the overlap window, a6, are written by the same
 * kernel), 4 block DFT (a7), 5 eigensolve (a8; open box: dense), 6 unused, 7 descriptor upload,
 * 8 tensor-core contraction of LHF_MIXED. */
#define LHF_NUM_STAGES 9
lhf_status lhf_set_profiling(lhf_ctx *ctx, int enable);
lhf_status lhf_stage_times(lhf_ctx *ctx, double *ms, int *launches);

/* Live per-kernel timing (same switch as the stage timing): with profiling enabled every kernel
 * launch of the path is bracketed by its own pair of CUDA events on the context stream.
 * lhf_kernel_times waits for the stream, adds the elapsed time of every launch recorded since
 * the previous call into ms[kernel] and the launch count into launches[kernel] (host arrays of
 * LHF_NUM_KERNELS), and clears the record.  lhf_kernel_name gives the kernel's name (static
 * string; NULL outside 0 .. LHF_NUM_KERNELS - 1). */
enum {
    LHF_K_BASIS = 0,         /* a1 basis samples and differences */
    LHF_K_POTENTIAL = 1,     /* a2 potential factors (two launches: row constants, rows) */
    LHF_K_GRAM_FP64 = 2,     /* a3-a4 FP64 weighted Grams */
    LHF_K_GRAM_SLICE = 3,    /* a3-a4 folded products and their digit planes (LHF_MIXED) */
    LHF_K_VSLICE = 4,        /* digit planes of the potential factors (LHF_MIXED) */
    LHF_K_GRAM_TC = 5,       /* tensor-core contraction of the digit planes (LHF_MIXED) */
    LHF_K_GRAM_MIRROR = 6,   /* window blocks j < 0 from their mirrors */
    LHF_K_RANKSUM = 7,       /* a5 Hadamard products and rank sum, a6 zero blocks */
    LHF_K_DFT = 8,           /* a7 block DFT, one launch per lattice level */
    LHF_K_OVERLAP_NORMS = 9, /* a8 cell-periodic overlap norms s0 */
    LHF_K_EIG = 10,          /* a8 removal, scaling, reduction, Householder tridiagonalisation */
    LHF_K_TRIDIAG_EIG = 11,  /* a8 tridiagonal eigenvalues */
    LHF_K_BOX_GRAM = 12,     /* a9 direction-0 factors between cell pairs */
    LHF_K_BOX_ASSEMBLE = 13, /* a9 dense H, S */
    LHF_K_DENSE_EIG = 14,    /* a9 dense generalized eigensolve */
    LHF_K_FACTOR_DFT = 15,   /* k-space route: 1D DFTs of the per-direction factors */
    LHF_K_KSPACE_BLOCKS = 16, /* k-space route: Hadamard products and rank sum per k-point */
    LHF_K_BOX_SOLVE = 17,    /* large box: banded products, preconditioner, Rayleigh-Ritz */
    LHF_NUM_KERNELS = 18
};
lhf_status lhf_kernel_times(lhf_ctx *ctx, double *ms, int *launches);
const char *lhf_kernel_name(int kernel);

/* Work counters of the k-point eigensolver since the previous call (synchronising; host
 * outputs): total FP64 characteristic-polynomial passes of the tridiagonal eigenvalue stage (one
 * pass: the order-m recurrence for the leading minors and their derivatives at one point; k-points
 * solved by Jacobi instead add their sweeps) and number of matrices solved (one per conjugate pair
 * of k-points).  Reset by the call. */
lhf_status lhf_eig_counters(lhf_ctx *ctx, unsigned long long *passes, unsigned long long *matrices);

/* Rank reduction of the lattice-summed potential (the rank optimisation of Sec. 3.2) for periodic
 * (L,1,1) lattices on the FP64 route.  The nuclear part of a block is a sum over R_tot = M0 R rank
 * terms, V_j = sum_r <Q_j, v_r> T_r (v_r the direction-0 factor over one cell, Q_j the cell fold of
 * the product row, T_r = c_r C1_r (.) C2_r the single-cell transverse factors).  With weights
 * w_r = max |T_r|, a rank-revealing (pivoted, reorthogonalised) Gram-Schmidt of the weighted
 * factor rows a_r = v_r w_r stops once every residual row is at most eps times the first pivot,
 * a_r = sum_k R_rk q_k + res_r with ||res_r|| <= rho, and the sum becomes r1 terms,
 * V_j ~ sum_k <Q_j, q_k> D_k with D_k = sum_r R_rk T_r / w_r; every entry of V_j then moves by at
 * most rho ||Q_j,mu,nu||_2 R_tot.  The direction-0 Gram and the rank sum then run over r1 terms.
 * lhf_set_rank_reduction: eps in [1e-14, 1) turns it on for the context's later FP64 assemblies and
 * spectra of such lattices with R_tot <= 64 (other systems, the mixed route and graphs are
 * unaffected); 0 turns it off.  lhf_rank_reduction_info: for the current setup system (reduction
 * on), runs the factor stages and returns R_tot, r1, rho and the first pivot (host outputs, each optional;
 * synchronising): "dropped" is rho, "largest" the first pivot's norm. */
lhf_status lhf_set_rank_reduction(lhf_ctx *ctx, double eps);
lhf_status lhf_rank_reduction_info(lhf_ctx *ctx, int *rank_in, int *rank_out, double *dropped, double *largest);

/* Extrapolation of the lattice sum to the limit (the regularisation of Sec. 4.1: the nuclear lattice
 * sum converges only conditionally and is extrapolated over a sequence of lattice parameters).
 * eig: device [nK][n], the same n spectral values of one lattice computed with nK image windows
 * K[k] (host [nK], distinct, >= 1; e.g. lhf_bloch_spectra of copies of the system differing only
 * in K_sum[0]); each value is fitted to lambda(K) = A + B ln K + C / K (least squares; nK = 2
 * fits A + B ln K).  eig_limit: device [n] the finite parts A; slope: device [n] the coefficients
 * B (may be NULL).  For an (L,1,1) chain the far images shift every eigenvalue by
 * -(2 Z_cell / b) sum_k 1/k, so B tends to -2 Z_cell / b (Z_cell the charge per cell) and A is the
 * regularised eigenvalue.  Non-finite inputs (removed functions) stay non-finite.  2 <= nK <= 8.
 * Asynchronous on the context stream; uses the first nK doubles of the context workspace. */
lhf_status lhf_extrapolate_lattice_sum(lhf_ctx *ctx, int nK, const double *K, long long n, const double *eig,
                                       double *eig_limit, double *slope);

/* Failure detection (no counterpart in the paper: controls of this library's own error paths).
 * lhf_set_wait_limit: the bound, in SM clock cycles, of every wait at a grid barrier of the dense
 *   eigensolver (lhf_dense_eigensolve and the open-box path); cycles <= 0 restores the default
 *   2e9 (about a second).  A wait that runs out sets the context's device error word and makes
 *   every CTA of that launch return; the next lhf_sync returns LHF_ERR_TIMEOUT, and the context
 *   stays usable (the outputs of that solve are undefined).
 * lhf_inject_barrier_stall: the next dense eigensolve of this context runs with grid barriers
 *   that expect one CTA more than the launch holds, so that their waits run out as above (a test
 *   of the time-out path that faults nothing; consumed by that solve).
 * lhf_set_workspace_limit: the most bytes of device workspace the context (and each graph created
 *   from it) may allocate; a call needing more returns LHF_ERR_NOMEM before any kernel launch.
 *   0 = no limit (default).  Small fixed buffers (descriptors, status words) are not counted.
 * Each returns LHF_OK, or LHF_ERR_ARG for a null context. */
lhf_status lhf_set_wait_limit(lhf_ctx *ctx, long long cycles);
lhf_status lhf_inject_barrier_stall(lhf_ctx *ctx);
lhf_status lhf_set_workspace_limit(lhf_ctx *ctx, size_t bytes);

/* Allocation-free variant of lhf_k_point_eigensolve (the paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory -- services held to a fixed
 * device-memory budget set at start-up, and hosts whose allocator policy forbids raw CUDA
 * allocations because another framework owns the device memory).  It needs no context and
 * calls no cudaMalloc/cudaFree or allocating library routine: its scratch (the kernel's descriptor, a status word and the overlap norms s0) lives
 * in one file-scope device array of LHF_NOALLOC_SCRATCH_BYTES that every GPU loading the
 * library holds until the process exits.
 *   L[3]   host: lattice sizes (each 1..4096); m0: functions per cell, 1..LHF_MAX_M0 (larger m0
 *          returns LHF_ERR_ARG: s0 would not fit the scratch);
 *   Hbar, Sbar, eig, k_status: as for lhf_k_point_eigensolve (caller-owned device memory;
 *          k_status may be NULL); stream: cudaStream_t (NULL = default stream).
 * Asynchronous on the stream; the descriptor is written into the array by a kernel on the same
 * stream, so no host buffer of the call has to outlive it.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture is active on the calling thread.  All calls share the one
 * array, which keeps the last call's contents: calls whose work may overlap on the GPU
 * (different streams without ordering) race and must be serialised by the caller.  Returns LHF_OK, LHF_ERR_ARG or LHF_ERR_CUDA. */
#define LHF_NOALLOC_SCRATCH_BYTES 16384
lhf_status lhf_k_point_eigensolve_noalloc(const int *L, int m0, const double *Hbar, const double *Sbar,
                                          double *eig, int *k_status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LHF_H */
