/*
 * lhf_oracle.c -- plain, slow, FP64 CPU oracle for the lattice core-Hamiltonian path of
 * Khoromskaia & Khoromskij, "Tensor numerical approach to linearized Hartree-Fock equation for
 * lattice-type and periodic systems" (arXiv:1408.3839).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this library.  It shares no code, header, table or helper with the CUDA path
 * and must never be linked into it.
 *
 * Every quantity is computed from its definition in the paper's order and notation, with no
 * blocking, fusion or reordering of sums beyond skipping terms that are exactly zero:
 *   - sinc quadrature of the Newton kernel ........................ Sec. 3.2, eq. (3.6)
 *   - piecewise-constant cell integrals of the kernel ............ Sec. 3.2, eq. (3.5)
 *   - lattice sum of shifted kernels (box) ........................ eqs. (3.8), (3.9)
 *   - periodic lattice sum restricted to cell 0 and replicated .... Sec. 4.1, eq. (4.1)
 *   - separable basis sampled at grid nodes ....................... Sec. 3.4, eq. (3.14)
 *   - per-entry 1D weighted inner products, product over directions,
 *     sum over rank terms (nuclear part) ........................... eq. (3.10), Lemma 3.1 proof
 *   - P1 stiffness / mass quadratic forms (kinetic and overlap) ..... Sec. 3.4, Lemma 4.1 proof
 *   - core Hamiltonian entries h = 1/2 grad.grad - v_c ............. eqs. (3.1), (3.4)
 *   - block DFT of the first block column .......................... Prop. 6.1, Lemma 2.2
 *   - generalized eigenproblem per k-point ......................... eq. (4.7), eq. (6.7)
 * Eigenvalues use Cholesky plus the real 2m x 2m symmetric embedding of each Hermitian block and
 * a textbook cyclic Jacobi (Golub & Van Loan, Sec. 8.5), an algorithm different from the GPU's.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NOT_SPD (-3)
#define ORC_ERR_NOMEM (-7)

typedef struct {
    int L[3];
    double b[3];
    int periodic[3];
    int n[3];
    int n_cell[3];
    double h[3];
    double x0[3];
    double cell0[3];
    int K_sum[3];
    int M0;
    const double *Z;      /* [M0] */
    const double *Z_cell; /* [L0*L1*L2][M0] or NULL */
    const double *a;      /* [M0][3] */
    int m0;
    const int *kind;      /* [m0] 0 = s, 1 + d = p along d */
    const double *alpha;  /* [m0] */
    const double *centre; /* [m0][3] */
    int R;
    double u0, du;
    double rho;
} orc_system;

static const double ORC_PI = 3.14159265358979323846;

/* ---------------------------------------------------------------------------------------- */
/* Sinc quadrature for 1/r (Sec. 3.2, eq. (3.6)): 1/r = 2/sqrt(pi) int_0^inf exp(-r^2 t^2) dt,
 * substituted t = exp(u) and discretised by the trapezoid rule on u_q = u0 + q du, q = 0..R-1,
 * weight w_q = 2/sqrt(pi) du t_q.  The nodes below u0 (where exp(-t^2 r^2) ~ exp(-t_0^2 r^2)) form
 * a geometric series that is folded into the first weight: w_0 <- w_0 / (1 - exp(-du)).      */

void orc_sinc_nodes(int R, double u0, double du, double *t, double *w)
{
    for (int q = 0; q < R; ++q) {
        t[q] = exp(u0 + q * du);
        w[q] = 2.0 / sqrt(ORC_PI) * du * t[q];
    }
    w[0] = w[0] / (1.0 - exp(-du));
}

double orc_sinc_inverse_r(int R, double u0, double du, double r)
{
    double t[256], w[256];
    if (R > 256) return NAN;
    orc_sinc_nodes(R, u0, du, t, w);
    double s = 0.0;
    for (int q = 0; q < R; ++q) s += w[q] * exp(-t[q] * t[q] * r * r);
    return s;
}

/* ---------------------------------------------------------------------------------------- */
/* Gauss-Legendre nodes on [-1, 1] by Newton iteration on the Legendre polynomial.            */

#define ORC_GL_N 16
static double gl_x[ORC_GL_N], gl_w[ORC_GL_N];
static int gl_ready = 0;

static void gl_init(void)
{
    if (gl_ready) return;
    int n = ORC_GL_N;
    for (int i = 0; i < n; ++i) {
        double x = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (x * p1 - p0) / (x * x - 1.0);
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

/* Exact integral of exp(-t^2 (x - c)^2) over [lo, hi]: the 1D factor of the piecewise-constant
 * projection of one sinc term (Sec. 3.2, eq. (3.5) with the kernel of eq. (3.6)).
 * Narrow cells (t (hi - lo) <= 2): 16-point Gauss-Legendre, exact to rounding there.
 * Wide cells: erf differences, written so that the two terms never cancel badly.          */
double orc_gauss_cell_integral(double t, double lo, double hi, double c)
{
    gl_init();
    double A = t * (lo - c), B = t * (hi - c);
    if (B - A <= 2.0) {
        double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo), s = 0.0;
        for (int k = 0; k < ORC_GL_N; ++k) {
            double x = mid + half * gl_x[k];
            double d = t * (x - c);
            s += gl_w[k] * exp(-d * d);
        }
        return s * half;
    }
    double f = sqrt(ORC_PI) / (2.0 * t);
    if (A >= 0.0) return f * (erfc(A) - erfc(B));
    if (B <= 0.0) return f * (erfc(-B) - erfc(-A));
    return f * (erf(B) + erf(-A));
}

/* ---------------------------------------------------------------------------------------- */
/* Separable Gaussian basis (Sec. 3.4, eq. (3.14)): 1D factor of function mu in direction l.
 * s-type / transverse factor: exp(-alpha d^2); p-type along l: sqrt(2 alpha e) d exp(-alpha d^2)
 * (unit peak).  Cut to zero beyond |d| > sqrt(rho / alpha).                                 */

static double gto_factor(const orc_system *s, int mu, int l, double d)
{
    double al = s->alpha[mu];
    double cut = sqrt(s->rho / al);
    if (fabs(d) > cut) return 0.0;
    double g = exp(-al * d * d);
    if (s->kind[mu] == 1 + l) g *= sqrt(2.0 * al * exp(1.0)) * d;
    return g;
}

/* Sample of the basis function mu copied to lattice cell `cell` (direction l) at grid node i.
 * Periodic directions sum the images of period L b (the supercell); open directions do not.  */
double orc_basis_sample(const orc_system *s, int l, int mu, int cell, int i)
{
    double x = s->x0[l] + (i + 0.5) * s->h[l];
    double A = s->centre[3 * mu + l] + cell * s->b[l];
    if (!s->periodic[l]) return gto_factor(s, mu, l, x - A);
    double P = s->L[l] * s->b[l];
    double cut = sqrt(s->rho / s->alpha[mu]);
    double d0 = x - A;
    long mlo = (long)floor((d0 - cut) / P) - 1, mhi = (long)ceil((d0 + cut) / P) + 1;
    double g = 0.0;
    for (long m = mlo; m <= mhi; ++m) g += gto_factor(s, mu, l, d0 - m * P);
    return g;
}

/* ---------------------------------------------------------------------------------------- */
/* 1D factor of rank term r = (nu, q) of the lattice-summed potential in direction l at grid
 * cell i (eq. (3.9) for a box, eq. (4.1) restricted to cell 0 and replicated for periodic).
 * Periodic: images k = -floor(K/2) .. floor(K/2) (weight 1/2 on |k| = K/2 for even K), the cell
 * integral taken for the cell-0 node i mod n_cell.  Open lattice: all L cells k = 0 .. L-1,
 * weighted by Z_cell[k][nu] / Z[nu].  Single-cell open direction: k = 0 only.
 * Terms whose integrand underflows to exactly zero over the whole cell are skipped.        */
double orc_potential_factor(const orc_system *s, int l, int nu, int q, int i)
{
    double t = exp(s->u0 + q * s->du);
    double h = s->h[l];
    double c0 = s->a[3 * nu + l];
    if (s->periodic[l]) {
        int ic = i % s->n_cell[l];
        double lo = s->cell0[l] + ic * h, hi = lo + h;
        int K = s->K_sum[l];
        int kmax = K / 2;
        double v = 0.0;
        for (int k = -kmax; k <= kmax; ++k) {
            double wk = (K % 2 == 0 && (k == kmax || k == -kmax)) ? 0.5 : 1.0;
            double c = c0 + k * s->b[l];
            double dmin = (c < lo) ? lo - c : (c > hi ? c - hi : 0.0);
            if (t * dmin > 28.0) continue; /* exp(-784) underflows: exact zero */
            v += wk * orc_gauss_cell_integral(t, lo, hi, c);
        }
        return v;
    }
    double lo = s->x0[l] + i * h, hi = lo + h;
    if (s->L[l] > 1) {
        int ncells = s->L[0] * s->L[1] * s->L[2];
        (void)ncells;
        double v = 0.0;
        for (int k = 0; k < s->L[l]; ++k) {
            double wk = 1.0;
            if (s->Z_cell) {
                /* cells are counted along the single lattice direction of a box tube */
                wk = s->Z_cell[k * s->M0 + nu] / s->Z[nu];
            }
            double c = c0 + k * s->b[l];
            double dmin = (c < lo) ? lo - c : (c > hi ? c - hi : 0.0);
            if (t * dmin > 28.0) continue;
            v += wk * orc_gauss_cell_integral(t, lo, hi, c);
        }
        return v;
    }
    return orc_gauss_cell_integral(t, lo, hi, c0);
}

/* All potential factors of direction l: out[r][i], r = nu * R + q, i = 0 .. n[l]-1.        */
void orc_potential_factors(const orc_system *s, int l, double *out)
{
    int n = s->n[l];
    int nc = s->periodic[l] ? s->n_cell[l] : n;
    for (int nu = 0; nu < s->M0; ++nu)
        for (int q = 0; q < s->R; ++q) {
            double *row = out + ((size_t)(nu * s->R + q)) * n;
            for (int i = 0; i < nc; ++i) row[i] = orc_potential_factor(s, l, nu, q, i);
            for (int i = nc; i < n; ++i) row[i] = row[i % nc]; /* periodic replication */
        }
}

/* All basis samples of direction l for cell copy `cell`: out[mu][i].                        */
void orc_basis_samples(const orc_system *s, int l, int cell, double *out)
{
    int n = s->n[l];
    for (int mu = 0; mu < s->m0; ++mu)
        for (int i = 0; i < n; ++i) out[(size_t)mu * n + i] = orc_basis_sample(s, l, mu, cell, i);
}

/* ---------------------------------------------------------------------------------------- */
/* 1D factors of every matrix entry between the copy of mu in cell p and the copy of nu in cell
 * q along direction l (eq. (3.10) and Lemma 3.1, proof; Sec. 3.4 for A and S):
 *   C[r][mu][nu] = sum_i g_{mu,p}(x_i) v_r(i) g_{nu,q}(x_i)         (nuclear, rank term r)
 *   K[mu][nu]    = g_{mu,p}^T A g_{nu,q},  A = (1/h) tridiag(-1, 2, -1)   (P1 stiffness)
 *   M[mu][nu]    = g_{mu,p}^T S g_{nu,q},  S = (h/6) tridiag(1, 4, 1)     (P1 mass)
 * The tridiagonal matrices wrap around in periodic directions and are truncated (Dirichlet)
 * in open ones.  V holds the potential factors of direction l (orc_potential_factors).     */
int orc_gram_1d(const orc_system *s, int l, int p, int q, const double *V, double *C,
                double *K, double *M)
{
    int n = s->n[l], m0 = s->m0, Rt = s->M0 * s->R;
    double h = s->h[l];
    int per = s->periodic[l];
    double *gp = (double *)malloc(sizeof(double) * (size_t)m0 * n);
    double *gq = (double *)malloc(sizeof(double) * (size_t)m0 * n);
    int *idx = (int *)malloc(sizeof(int) * (size_t)n);
    if (!gp || !gq || !idx) {
        free(gp);
        free(gq);
        free(idx);
        return ORC_ERR_NOMEM;
    }
    orc_basis_samples(s, l, p, gp);
    orc_basis_samples(s, l, q, gq);
    for (int mu = 0; mu < m0; ++mu) {
        const double *f = gp + (size_t)mu * n;
        /* nodes i where f_i or f_{i+1} is nonzero: every other node contributes exact zeros */
        int cnt = 0;
        for (int i = 0; i < n; ++i) {
            int ip = i + 1 < n ? i + 1 : (per ? 0 : -1);
            if (f[i] != 0.0 || (ip >= 0 && f[ip] != 0.0)) idx[cnt++] = i;
        }
        for (int nu = 0; nu < m0; ++nu) {
            const double *g = gq + (size_t)nu * n;
            double kin = 0.0, mass = 0.0;
            for (int r = 0; r < Rt; ++r) C[((size_t)r * m0 + mu) * m0 + nu] = 0.0;
            for (int u = 0; u < cnt; ++u) {
                int i = idx[u];
                int ip = i + 1 < n ? i + 1 : (per ? 0 : -1);
                double fi = f[i], gi = g[i];
                double fg = fi * gi;
                double cross = 0.0;
                if (ip >= 0) cross = fi * g[ip] + f[ip] * gi;
                kin += 2.0 * fg - cross;
                mass += 4.0 * fg + cross;
                if (fg == 0.0) continue; /* exact zero term */
                for (int r = 0; r < Rt; ++r)
                    C[((size_t)r * m0 + mu) * m0 + nu] += fi * V[(size_t)r * n + i] * gi;
            }
            K[mu * m0 + nu] = kin / h;
            M[mu * m0 + nu] = mass * h / 6.0;
        }
    }
    free(gp);
    free(gq);
    free(idx);
    return ORC_OK;
}

/* Rank-term coefficients c_r = Z_nu w_q, r = nu * R + q (eq. (3.9) with eq. (3.6)).       */
static void rank_coefficients(const orc_system *s, double *c)
{
    double t[256], w[256];
    orc_sinc_nodes(s->R, s->u0, s->du, t, w);
    for (int nu = 0; nu < s->M0; ++nu)
        for (int q = 0; q < s->R; ++q) c[nu * s->R + q] = s->Z[nu] * w[q];
}

/* Combine the three directions' 1D factors into one m0 x m0 block (Lemma 3.1 proof and
 * Lemma 4.1):  S = M1 M2 M3,  T = K1 M2 M3 + M1 K2 M3 + M1 M2 K3 (the rank-3 Laplacian),
 * V = sum_r c_r C1_r C2_r C3_r,  H = T/2 - V  (eq. (3.4): h = 1/2 grad.grad - v_c).       */
static void combine_block(int m0, int Rt, const double *c, const double *C[3], const double *K[3],
                          const double *M[3], double *Hb, double *Sb)
{
    for (int mu = 0; mu < m0; ++mu)
        for (int nu = 0; nu < m0; ++nu) {
            int e = mu * m0 + nu;
            double s = M[0][e] * M[1][e] * M[2][e];
            double tk = K[0][e] * M[1][e] * M[2][e] + M[0][e] * K[1][e] * M[2][e] +
                        M[0][e] * M[1][e] * K[2][e];
            double v = 0.0;
            for (int r = 0; r < Rt; ++r) {
                size_t o = (size_t)r * m0 * m0 + e;
                v += c[r] * C[0][o] * C[1][o] * C[2][o];
            }
            Hb[e] = 0.5 * tk - v;
            Sb[e] = s;
        }
}

typedef struct {
    double *V[3];
    double *C[3];
    double *K[3];
    double *M[3];
    double *c;
} orc_work;

static void work_free(orc_work *w)
{
    for (int l = 0; l < 3; ++l) {
        free(w->V[l]);
        free(w->C[l]);
        free(w->K[l]);
        free(w->M[l]);
    }
    free(w->c);
}

static int work_alloc(const orc_system *s, orc_work *w, int ncells_max)
{
    memset(w, 0, sizeof(*w));
    int m0 = s->m0, Rt = s->M0 * s->R;
    size_t mm = (size_t)m0 * m0;
    for (int l = 0; l < 3; ++l) {
        w->V[l] = (double *)malloc(sizeof(double) * (size_t)Rt * s->n[l]);
        w->C[l] = (double *)malloc(sizeof(double) * (size_t)ncells_max * Rt * mm);
        w->K[l] = (double *)malloc(sizeof(double) * (size_t)ncells_max * mm);
        w->M[l] = (double *)malloc(sizeof(double) * (size_t)ncells_max * mm);
        if (!w->V[l] || !w->C[l] || !w->K[l] || !w->M[l]) {
            work_free(w);
            return ORC_ERR_NOMEM;
        }
    }
    w->c = (double *)malloc(sizeof(double) * Rt);
    if (!w->c) {
        work_free(w);
        return ORC_ERR_NOMEM;
    }
    rank_coefficients(s, w->c);
    return ORC_OK;
}

/* First block column of the periodic (block-circulant) core Hamiltonian and overlap
 * (Lemma 4.1, eqs. (4.2), (4.5), (4.6)): A_j[mu][nu] = <g_{mu,j}, H g_{nu,0}> for every
 * lattice displacement j = (j0, j1, j2), j_l = 0 .. L_l - 1.  Out: H, S [L0][L1][L2][m0][m0]. */
int orc_core_blocks(const orc_system *s, double *H, double *S)
{
    if (s->R > 256) return ORC_ERR_ARG;
    int m0 = s->m0, Rt = s->M0 * s->R;
    size_t mm = (size_t)m0 * m0;
    int Lmax = s->L[0];
    if (s->L[1] > Lmax) Lmax = s->L[1];
    if (s->L[2] > Lmax) Lmax = s->L[2];
    orc_work w;
    if (work_alloc(s, &w, Lmax) != ORC_OK) return ORC_ERR_NOMEM;
    for (int l = 0; l < 3; ++l) {
        orc_potential_factors(s, l, w.V[l]);
        for (int j = 0; j < s->L[l]; ++j) {
            int rc = orc_gram_1d(s, l, j, 0, w.V[l], w.C[l] + (size_t)j * Rt * mm,
                                 w.K[l] + (size_t)j * mm, w.M[l] + (size_t)j * mm);
            if (rc != ORC_OK) {
                work_free(&w);
                return rc;
            }
        }
    }
    for (int j0 = 0; j0 < s->L[0]; ++j0)
        for (int j1 = 0; j1 < s->L[1]; ++j1)
            for (int j2 = 0; j2 < s->L[2]; ++j2) {
                int jj[3] = {j0, j1, j2};
                const double *C[3], *K[3], *M[3];
                for (int l = 0; l < 3; ++l) {
                    C[l] = w.C[l] + (size_t)jj[l] * Rt * mm;
                    K[l] = w.K[l] + (size_t)jj[l] * mm;
                    M[l] = w.M[l] + (size_t)jj[l] * mm;
                }
                size_t blk = ((size_t)j0 * s->L[1] + j1) * s->L[2] + j2;
                combine_block(m0, Rt, w.c, C, K, M, H + blk * mm, S + blk * mm);
            }
    work_free(&w);
    return ORC_OK;
}

/* Full N_b x N_b matrices (N_b = m0 L0 L1 L2), row index (cell P, mu), column (cell Q, nu),
 * cell index (p0 L1 + p1) L2 + p2, every entry from its own per-direction factors between the
 * copies in cells P and Q (Lemma 3.1).  Used for open boxes and, for small periodic lattices,
 * to check the block-circulant structure directly.                                         */
int orc_core_dense(const orc_system *s, double *H, double *S)
{
    if (s->R > 256) return ORC_ERR_ARG;
    int m0 = s->m0, Rt = s->M0 * s->R;
    size_t mm = (size_t)m0 * m0;
    int ncell = s->L[0] * s->L[1] * s->L[2];
    size_t Nb = (size_t)m0 * ncell;
    int Lmax = s->L[0];
    if (s->L[1] > Lmax) Lmax = s->L[1];
    if (s->L[2] > Lmax) Lmax = s->L[2];
    orc_work w;
    if (work_alloc(s, &w, Lmax * Lmax) != ORC_OK) return ORC_ERR_NOMEM;
    for (int l = 0; l < 3; ++l) {
        orc_potential_factors(s, l, w.V[l]);
        for (int p = 0; p < s->L[l]; ++p)
            for (int q = 0; q < s->L[l]; ++q) {
                size_t pq = (size_t)p * s->L[l] + q;
                int rc = orc_gram_1d(s, l, p, q, w.V[l], w.C[l] + pq * Rt * mm, w.K[l] + pq * mm,
                                     w.M[l] + pq * mm);
                if (rc != ORC_OK) {
                    work_free(&w);
                    return rc;
                }
            }
    }
    double *Hb = (double *)malloc(sizeof(double) * mm), *Sb = (double *)malloc(sizeof(double) * mm);
    if (!Hb || !Sb) {
        free(Hb);
        free(Sb);
        work_free(&w);
        return ORC_ERR_NOMEM;
    }
    for (int P = 0; P < ncell; ++P)
        for (int Q = 0; Q < ncell; ++Q) {
            int pp[3] = {P / (s->L[1] * s->L[2]), (P / s->L[2]) % s->L[1], P % s->L[2]};
            int qq[3] = {Q / (s->L[1] * s->L[2]), (Q / s->L[2]) % s->L[1], Q % s->L[2]};
            const double *C[3], *K[3], *M[3];
            for (int l = 0; l < 3; ++l) {
                size_t pq = (size_t)pp[l] * s->L[l] + qq[l];
                C[l] = w.C[l] + pq * Rt * mm;
                K[l] = w.K[l] + pq * mm;
                M[l] = w.M[l] + pq * mm;
            }
            combine_block(m0, Rt, w.c, C, K, M, Hb, Sb);
            for (int mu = 0; mu < m0; ++mu)
                for (int nu = 0; nu < m0; ++nu) {
                    size_t row = (size_t)P * m0 + mu, col = (size_t)Q * m0 + nu;
                    H[row * Nb + col] = Hb[mu * m0 + nu];
                    S[row * Nb + col] = Sb[mu * m0 + nu];
                }
        }
    free(Hb);
    free(Sb);
    work_free(&w);
    return ORC_OK;
}

/* ---------------------------------------------------------------------------------------- */
/* Block DFT of the first block column along the lattice indices (Prop. 6.1, Lemma 2.2):
 *   Abar_kappa = sum_j omega^{kappa . j} A_j,  omega_l = exp(-2 pi i / L_l),
 * evaluated directly from the definition, O(|L|^2).  Abar is complex, interleaved (re, im). */
void orc_block_dft(const int *L, int m0, const double *A, double *Abar)
{
    size_t mm = (size_t)m0 * m0;
    int L0 = L[0], L1 = L[1], L2 = L[2];
    for (int k0 = 0; k0 < L0; ++k0)
        for (int k1 = 0; k1 < L1; ++k1)
            for (int k2 = 0; k2 < L2; ++k2) {
                size_t kb = ((size_t)k0 * L1 + k1) * L2 + k2;
                double *out = Abar + 2 * kb * mm;
                for (size_t e = 0; e < 2 * mm; ++e) out[e] = 0.0;
                for (int j0 = 0; j0 < L0; ++j0)
                    for (int j1 = 0; j1 < L1; ++j1)
                        for (int j2 = 0; j2 < L2; ++j2) {
                            double ph = -2.0 * ORC_PI *
                                        ((double)((long)k0 * j0 % L0) / L0 +
                                         (double)((long)k1 * j1 % L1) / L1 +
                                         (double)((long)k2 * j2 % L2) / L2);
                            double cr = cos(ph), ci = sin(ph);
                            size_t jb = ((size_t)j0 * L1 + j1) * L2 + j2;
                            const double *in = A + jb * mm;
                            for (size_t e = 0; e < mm; ++e) {
                                out[2 * e] += cr * in[e];
                                out[2 * e + 1] += ci * in[e];
                            }
                        }
            }
}

/* ---------------------------------------------------------------------------------------- */
/* Dense real symmetric linear algebra (textbook).                                          */

/* Cholesky A = G G^T (lower G), A overwritten by G.  Returns ORC_ERR_NOT_SPD on a non-positive
 * pivot.                                                                                    */
static int cholesky(int n, double *A)
{
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0.0)) return ORC_ERR_NOT_SPD;
        d = sqrt(d);
        A[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) v -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = v / d;
        }
        for (int k = j + 1; k < n; ++k) A[(size_t)j * n + k] = 0.0;
    }
    return ORC_OK;
}

/* C = G^{-1} H G^{-T} for lower-triangular G (forward substitution on both sides).        */
static void reduce_standard(int n, const double *G, double *H)
{
    /* H <- G^{-1} H: solve column by column */
    for (int c = 0; c < n; ++c)
        for (int i = 0; i < n; ++i) {
            double v = H[(size_t)i * n + c];
            for (int k = 0; k < i; ++k) v -= G[(size_t)i * n + k] * H[(size_t)k * n + c];
            H[(size_t)i * n + c] = v / G[(size_t)i * n + i];
        }
    /* H <- H G^{-T}: solve row by row, X G^T = H  <=>  G X^T = H^T */
    for (int r = 0; r < n; ++r)
        for (int i = 0; i < n; ++i) {
            double v = H[(size_t)r * n + i];
            for (int k = 0; k < i; ++k) v -= G[(size_t)i * n + k] * H[(size_t)r * n + k];
            H[(size_t)r * n + i] = v / G[(size_t)i * n + i];
        }
    /* symmetrise the rounding */
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double v = 0.5 * (H[(size_t)i * n + j] + H[(size_t)j * n + i]);
            H[(size_t)i * n + j] = v;
            H[(size_t)j * n + i] = v;
        }
}

static double off_norm2(int n, const double *A)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (i != j) s += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    return s;
}

static int cmp_double(const void *x, const void *y)
{
    double a = *(const double *)x, b = *(const double *)y;
    return (a > b) - (a < b);
}

/* Cyclic-by-row Jacobi for a real symmetric matrix (Golub & Van Loan, Alg. 8.5.3): sweeps of
 * 2x2 symmetric Schur rotations until off(A) <= tol ||A||_F.  Eigenvalues ascending.        */
int orc_jacobi_eigenvalues(int n, double *A, double *eig)
{
    double fro = 0.0;
    for (size_t e = 0; e < (size_t)n * n; ++e) fro += A[e] * A[e];
    double tol2 = 1e-30 * fro;
    int sweep;
    for (sweep = 0; sweep < 100 && off_norm2(n, A) > tol2; ++sweep) {
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                /* A <- J^T A J with J = [c s; -s c] in the (p, q) plane */
                for (int k = 0; k < n; ++k) {
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - sn * akq;
                    A[(size_t)k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + c * aqk;
                }
            }
    }
    for (int i = 0; i < n; ++i) eig[i] = A[(size_t)i * n + i];
    qsort(eig, n, sizeof(double), cmp_double);
    return sweep;
}

/* Cyclic-by-row Jacobi with accumulated rotations: on return A is (numerically) diagonal,
 * diag(A) holds the eigenvalues and the columns of V (n x n, initialised here) the eigenvectors,
 * in matching order.                                                                         */
static void jacobi_vectors(int n, double *A, double *V)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (size_t e = 0; e < (size_t)n * n; ++e) fro += A[e] * A[e];
    double tol2 = 1e-30 * fro;
    for (int sweep = 0; sweep < 100 && off_norm2(n, A) > tol2; ++sweep)
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - sn * akq;
                    A[(size_t)k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - sn * vkq;
                    V[(size_t)k * n + q] = sn * vkp + c * vkq;
                }
            }
}

/* Generalized symmetric-definite eigenvalues H x = lambda S x (dense real, ascending):
 * Cholesky S = G G^T, C = G^{-1} H G^{-T}, cyclic Jacobi on C.                            */
int orc_dense_gen_eigenvalues(int n, const double *H, const double *S, double *eig)
{
    size_t nn = (size_t)n * n;
    double *G = (double *)malloc(sizeof(double) * nn), *C = (double *)malloc(sizeof(double) * nn);
    if (!G || !C) {
        free(G);
        free(C);
        return ORC_ERR_NOMEM;
    }
    memcpy(G, S, sizeof(double) * nn);
    memcpy(C, H, sizeof(double) * nn);
    int rc = cholesky(n, G);
    if (rc == ORC_OK) {
        reduce_standard(n, G, C);
        orc_jacobi_eigenvalues(n, C, eig);
    }
    free(G);
    free(C);
    return rc;
}

/* Real symmetric embedding [[Re X, -Im X], [Im X, Re X]] (2m x 2m) of a Hermitian m x m
 * matrix X given as interleaved (re, im); every eigenvalue of X appears twice.             */
static void embed(int m, const double *X, double *Xe)
{
    int n = 2 * m;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            size_t e = (size_t)i * m + j;
            double xr = X[2 * e], xi = X[2 * e + 1];
            Xe[(size_t)i * n + j] = xr;
            Xe[(size_t)i * n + j + m] = -xi;
            Xe[(size_t)(i + m) * n + j] = xi;
            Xe[(size_t)(i + m) * n + j + m] = xr;
        }
}

/* Eigenvalues of one Hermitian generalized problem Hbar u = lambda Sbar u (eq. (4.7)) through
 * the real symmetric embedding [[Re X, -Im X], [Im X, Re X]] of both m x m blocks: each
 * eigenvalue of the 2m x 2m real pencil appears twice; every other one is returned.        */
int orc_herm_gen_eigenvalues(int m, const double *Hbar, const double *Sbar, double *eig)
{
    int n = 2 * m;
    size_t nn = (size_t)n * n;
    double *He = (double *)malloc(sizeof(double) * nn), *Se = (double *)malloc(sizeof(double) * nn);
    double *ev = (double *)malloc(sizeof(double) * n);
    if (!He || !Se || !ev) {
        free(He);
        free(Se);
        free(ev);
        return ORC_ERR_NOMEM;
    }
    embed(m, Hbar, He);
    embed(m, Sbar, Se);
    int rc = orc_dense_gen_eigenvalues(n, He, Se, ev);
    if (rc == ORC_OK)
        for (int i = 0; i < m; ++i) eig[i] = ev[2 * i];
    free(He);
    free(Se);
    free(ev);
    return rc;
}

/* Canonical orthogonalisation (Loewdin) of one Hermitian pencil given as m x m complex blocks:
 * eigen-decompose the real embedding of S, keep the directions with eigenvalue >= tau2,
 * X = V_kept diag(sigma)^{-1/2}, and solve the standard problem X^T H X.  Each complex
 * eigenvalue appears twice in the embedding, so the kept directions come in pairs.  eig[0..]
 * receives the kept eigenvalues (ascending); *removed the number of complex directions
 * dropped.                                                                                   */
static int canonical_eigenvalues(int m, const double *Hbar, const double *Sbar, double tau2,
                                 double *eig, int *removed)
{
    int n = 2 * m;
    size_t nn = (size_t)n * n;
    double *He = (double *)malloc(sizeof(double) * nn), *Se = (double *)malloc(sizeof(double) * nn);
    double *V = (double *)malloc(sizeof(double) * nn), *X = (double *)malloc(sizeof(double) * nn);
    double *W = (double *)malloc(sizeof(double) * nn), *ev = (double *)malloc(sizeof(double) * n);
    int *kept = (int *)malloc(sizeof(int) * n);
    if (!He || !Se || !V || !X || !W || !ev || !kept) {
        free(He);
        free(Se);
        free(V);
        free(X);
        free(W);
        free(ev);
        free(kept);
        return ORC_ERR_NOMEM;
    }
    embed(m, Hbar, He);
    embed(m, Sbar, Se);
    jacobi_vectors(n, Se, V);
    int nk = 0;
    for (int i = 0; i < n; ++i)
        if (Se[(size_t)i * n + i] >= tau2) kept[nk++] = i;
    if (nk & 1) { /* a pair split by rounding at the threshold: drop its kept member */
        int lo = 0;
        for (int a = 1; a < nk; ++a)
            if (Se[(size_t)kept[a] * n + kept[a]] < Se[(size_t)kept[lo] * n + kept[lo]]) lo = a;
        for (int a = lo; a < nk - 1; ++a) kept[a] = kept[a + 1];
        --nk;
    }
    /* X = V_kept diag(sigma)^{-1/2}  (n x nk) */
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < nk; ++a)
            X[(size_t)i * nk + a] = V[(size_t)i * n + kept[a]] / sqrt(Se[(size_t)kept[a] * n + kept[a]]);
    /* W = He X (n x nk); C = X^T W (nk x nk) stored in V */
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < nk; ++a) {
            double v = 0.0;
            for (int k = 0; k < n; ++k) v += He[(size_t)i * n + k] * X[(size_t)k * nk + a];
            W[(size_t)i * nk + a] = v;
        }
    for (int a = 0; a < nk; ++a)
        for (int b = 0; b < nk; ++b) {
            double v = 0.0;
            for (int k = 0; k < n; ++k) v += X[(size_t)k * nk + a] * W[(size_t)k * nk + b];
            V[(size_t)a * nk + b] = v;
        }
    for (int a = 0; a < nk; ++a)
        for (int b = a + 1; b < nk; ++b) {
            double v = 0.5 * (V[(size_t)a * nk + b] + V[(size_t)b * nk + a]);
            V[(size_t)a * nk + b] = v;
            V[(size_t)b * nk + a] = v;
        }
    if (nk > 0) orc_jacobi_eigenvalues(nk, V, ev);
    for (int i = 0; i < nk / 2; ++i) eig[i] = ev[2 * i];
    *removed = m - nk / 2;
    free(He);
    free(Se);
    free(V);
    free(X);
    free(W);
    free(ev);
    free(kept);
    return ORC_OK;
}

/* Per-k-point eigenvalues for K blocks (Prop. 6.1, eq. (6.7); eq. (4.7)).
 * Reading for FP64 data: a Bloch function whose overlap diagonal cancels to rounding level is
 * numerically absent.  With s0_i = mean over kappa of Re Sbar_ii (= S_0,ii, the cell-periodic
 * norm of basis function i), function i is removed at kappa when Re Sbar_ii(kappa) <= tau s0_i.
 * The remaining pencil is scaled by D = diag(Sbar)^{-1/2} on both sides (a congruence: same
 * eigenvalues) and solved by canonical orthogonalisation with threshold tau2 on the scaled
 * overlap (directions of near-linear dependence dropped); removed slots hold +INFINITY (sorted
 * last).  status[k] = number of removed directions (>= 0), or ORC_ERR_NOT_SPD when the input
 * has no positive norms.  Returns the number of k-points reported as not positive definite. */
int orc_k_point_eigenvalues(int K, int m, const double *Hbar, const double *Sbar, double tau,
                            double tau2, double *eig, int *status)
{
    int bad = 0;
    size_t mm2 = 2 * (size_t)m * m;
    double *s0 = (double *)calloc((size_t)m, sizeof(double));
    double *Hr = (double *)malloc(sizeof(double) * mm2), *Sr = (double *)malloc(sizeof(double) * mm2);
    double *ev = (double *)malloc(sizeof(double) * (size_t)m);
    int *keep = (int *)malloc(sizeof(int) * (size_t)m);
    if (!s0 || !Hr || !Sr || !ev || !keep) {
        free(s0);
        free(Hr);
        free(Sr);
        free(ev);
        free(keep);
        return -1;
    }
    for (int k = 0; k < K; ++k)
        for (int i = 0; i < m; ++i) s0[i] += Sbar[k * mm2 + 2 * ((size_t)i * m + i)];
    int valid = 1;
    for (int i = 0; i < m; ++i) {
        s0[i] /= K;
        if (!(s0[i] > 0.0)) valid = 0; /* not an overlap matrix: no positive norm */
    }
    for (int k = 0; k < K && !valid; ++k) {
        status[k] = ORC_ERR_NOT_SPD;
        for (int i = 0; i < m; ++i) eig[(size_t)k * m + i] = NAN;
    }
    if (!valid) bad = K;
    for (int k = 0; k < K && valid; ++k) {
        const double *Hk = Hbar + k * mm2, *Sk = Sbar + k * mm2;
        int mr = 0;
        for (int i = 0; i < m; ++i)
            if (Sk[2 * ((size_t)i * m + i)] > tau * s0[i]) keep[mr++] = i;
        for (int a = 0; a < mr; ++a)
            for (int b = 0; b < mr; ++b) {
                size_t e = (size_t)keep[a] * m + keep[b];
                double da = 1.0 / sqrt(Sk[2 * ((size_t)keep[a] * m + keep[a])]);
                double db = 1.0 / sqrt(Sk[2 * ((size_t)keep[b] * m + keep[b])]);
                size_t f = (size_t)a * mr + b;
                Hr[2 * f] = Hk[2 * e] * da * db;
                Hr[2 * f + 1] = Hk[2 * e + 1] * da * db;
                Sr[2 * f] = Sk[2 * e] * da * db;
                Sr[2 * f + 1] = Sk[2 * e + 1] * da * db;
            }
        /* the blocks are Hermitian (eq. (4.7)) up to the rounding of the transform: the pencil
         * solved is their Hermitian part (X + X^H) / 2 */
        for (int a = 0; a < mr; ++a)
            for (int b = a; b < mr; ++b) {
                size_t f = (size_t)a * mr + b, g = (size_t)b * mr + a;
                double hr = 0.5 * (Hr[2 * f] + Hr[2 * g]), hi = 0.5 * (Hr[2 * f + 1] - Hr[2 * g + 1]);
                double sr = 0.5 * (Sr[2 * f] + Sr[2 * g]), si = 0.5 * (Sr[2 * f + 1] - Sr[2 * g + 1]);
                if (a == b) hi = si = 0.0;
                Hr[2 * f] = hr;
                Hr[2 * f + 1] = hi;
                Hr[2 * g] = hr;
                Hr[2 * g + 1] = -hi;
                Sr[2 * f] = sr;
                Sr[2 * f + 1] = si;
                Sr[2 * g] = sr;
                Sr[2 * g + 1] = -si;
            }
        int removed2 = 0;
        int rc = mr > 0 ? canonical_eigenvalues(mr, Hr, Sr, tau2, ev, &removed2) : ORC_OK;
        if (rc != ORC_OK) {
            ++bad;
            status[k] = rc;
            for (int i = 0; i < m; ++i) eig[(size_t)k * m + i] = NAN;
            continue;
        }
        int nkept = mr - removed2;
        status[k] = m - nkept;
        for (int i = 0; i < nkept; ++i) eig[(size_t)k * m + i] = ev[i];
        for (int i = nkept; i < m; ++i) eig[(size_t)k * m + i] = INFINITY;
    }
    free(s0);
    free(Hr);
    free(Sr);
    free(ev);
    free(keep);
    return bad;
}
