/*
 * ep_oracle.c -- plain FP64 CPU oracle for the voxel bidomain/monodomain step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  Only tests, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Everything is written directly from the thesis' definitions, in FP64, with
 * no blocking, fusion or reordering beyond what the definitions state:
 *
 *  - Mitchell-Schaeffer ionic model, Eqs. ms1/ms2 (Sec. "Mitchell-Schaeffer
 *    Model"), integrated with one explicit Euler step (Sec. "Algorithm
 *    Details / Electrophysiology / Reaction").  Reading: the closing branch of
 *    Eq. ms2 is -w/tau_close (the printed (1-w)/tau_close can never
 *    repolarise), and the printed w-update "w = v + dt dw/dt" is read as
 *    w + dt dw/dt.
 *  - Conductivity tensor Sigma = sT I + (sL - sT) f f^T, Eq. sigma1; sT I
 *    where the fibre is zero (Sec. "Fibre Directions").
 *  - Self-dual Laplacian (Sec. "Operators / Laplacian", Eqs. refgrad2,
 *    refdiv2/3, refintp2): the gradient of the voxel field at every grid vertex
 *    is the average of the edge differences of the 2x2x2 voxel block around the
 *    vertex; the conductivity tensor at the vertex is the average over the
 *    block (non-tissue voxels contribute zero conductivity); the divergence
 *    at a voxel sums the face-averaged fluxes.  Written as L = G'^T S G'
 *    (matrix-free assembly of Sec. "Matrix-Free Assembly", Eq. ass3, with
 *    F = dx I so the scale is 1/dx^2).  No-flux at the tissue mask: a voxel pair
 *    contributes to a vertex gradient only if both voxels are tissue, and the
 *    average is over the contributing pairs.  L u approximates -div(Sigma grad u).
 *  - Operator splitting (Sec. "Algorithm Details / Electrophysiology"):
 *    reaction, then diffusion, then (bidomain) the elliptic equation of
 *    Eq. bidomain1 (second line).  Diffusion is explicit Euler:
 *      monodomain  v+ = v* - dt/K * lambda/(1+lambda) * L_i v*     (Eq. monodomain1)
 *      bidomain    v+ = v* - dt/K * L_i (v* + ve^n)                (Eq. bidomain1, line 1)
 *                  (L_i + L_e) ve^{n+1} = -L_i v+                   (Eq. bidomain1, line 2)
 *    or implicit Euler (Sec. "Implicit Euler", Sec. "Diffusion"), whose linear
 *    system (I - alpha A) u^{t+1} = u^t is solved by the Jacobi step of
 *    Eq. iejac1 with A = -L (L approximates -div Sigma grad):
 *      monodomain  (I + a L_i) v+ = v*,             a = dt/K lambda/(1+lambda)
 *      bidomain    (I + a L_i) v+ = v* - a L_i ve^n, a = dt/K   (ve lagged to step n)
 *  - Torso (Eq. bidomain1, lines 3-5): an optional set of conducting voxels
 *    around the tissue with isotropic conductivity sig_o.  The extracellular
 *    potential extends into it, and the elliptic operator on tissue + torso
 *    is the sum of two vertex operators: the tissue's (pairs of tissue
 *    voxels, Sigma_i + Sigma_e of the tissue voxels of the block) and the
 *    torso's (pairs of any two domain voxels, sig_o I times the fraction of
 *    torso voxels in the block).  The torso term carries the current across
 *    the heart surface and through the torso; no current leaves the torso's
 *    outer surface; both terms conserve charge.  Keeping the tissue term on
 *    tissue pairs makes the operator dominate the intracellular one, which
 *    the explicit split needs to stay stable (one vertex average over both
 *    media does not, and the step diverges).  The intracellular operator and
 *    the membrane state stay on the tissue.
 *  - Elliptic solve by damped Jacobi, Eq. dampjac1, from the previous ve,
 *    stopping when ||b - A x||_2 <= tol ||b||_2 (checked every m sweeps), then
 *    the reference potential is fixed by subtracting the mean over every
 *    face-connected tissue component (the pure-Neumann null space).  Two
 *    other solves of the same equation: the Chebyshev semi-iteration on the
 *    Jacobi step, and eight-colour Gauss-Seidel (the deterministic form of
 *    the thesis' in-place Jacobi), both to the same stop rule.
 *
 * Units: mm, ms, mS/mm; v dimensionless (0 rest, 1 peak).
 * Index: q = i + nx*(j + ny*k).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "ep_oracle.h"

/* ------------------------------------------------------------------------ */
/* grid helpers                                                              */
/* ------------------------------------------------------------------------ */

static long og_idx(const og_grid *g, int i, int j, int k)
{
    return (long)i + (long)g->nx * ((long)j + (long)g->ny * (long)k);
}

/* Voxel q belongs to the domain of the operator: tissue, or torso when the
 * grid carries one. */
static int og_in(const og_grid *g, long q)
{
    return g->mask[q] != 0 || (g->torso && g->torso[q] != 0);
}

static int og_tissue(const og_grid *g, int i, int j, int k)
{
    if (i < 0 || j < 0 || k < 0 || i >= g->nx || j >= g->ny || k >= g->nz)
        return 0;
    return og_in(g, og_idx(g, i, j, k));
}

/* The operator is a sum of vertex terms in two parts.  OG_TISSUE: pairs of
 * tissue voxels, tensor from the tissue voxels of the block (the operator of
 * the thesis).  OG_TORSO (grids with a torso): pairs of domain voxels, tensor
 * sig_o I from the torso voxels of the block. */
enum { OG_TISSUE = 0, OG_TORSO = 1 };

static int og_member(const og_grid *g, int part, int i, int j, int k)
{
    if (i < 0 || j < 0 || k < 0 || i >= g->nx || j >= g->ny || k >= g->nz)
        return 0;
    return part == OG_TISSUE ? g->mask[og_idx(g, i, j, k)] != 0 : og_in(g, og_idx(g, i, j, k));
}

/* Offsets of the two voxels of pair number p (0..3) along axis a, inside the
 * 2x2x2 block of vertex (I,J,K).  The block voxels are (I-1+s, J-1+t, K-1+u)
 * with s,t,u in {0,1}; along axis a the pair is (lo: offset 0, hi: offset 1)
 * and p enumerates the offsets of the two other axes. */
static void og_pair(int I, int J, int K, int a, int p, int lo[3], int hi[3])
{
    int o1 = p & 1, o2 = (p >> 1) & 1;
    int base[3] = {I - 1, J - 1, K - 1};
    int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
    lo[0] = base[0]; lo[1] = base[1]; lo[2] = base[2];
    lo[b1] += o1;
    lo[b2] += o2;
    hi[0] = lo[0]; hi[1] = lo[1]; hi[2] = lo[2];
    hi[a] += 1;
}

/* Block tensor of a part: OG_TISSUE S_p = (1/8) sum_{tissue j in block} Sigma_j;
 * OG_TORSO S_p = (1/8) (torso voxels in block) sig_o I. */
static void og_vertex_tensor(const og_grid *g, int part, int I, int J, int K, double sL, double sT,
                             double S[3][3])
{
    int a, b, s, t, u;
    for (a = 0; a < 3; a++)
        for (b = 0; b < 3; b++)
            S[a][b] = 0.0;
    for (u = 0; u < 2; u++)
        for (t = 0; t < 2; t++)
            for (s = 0; s < 2; s++) {
                int i = I - 1 + s, j = J - 1 + t, k = K - 1 + u;
                if (!og_member(g, part, i, j, k))
                    continue;
                long q = og_idx(g, i, j, k);
                if (part == OG_TORSO) {
                    if (!g->mask[q])
                        for (a = 0; a < 3; a++)
                            S[a][a] += g->sig_o;
                    continue;
                }
                const double *f = g->fib + 3 * q;
                for (a = 0; a < 3; a++)
                    for (b = 0; b < 3; b++)
                        S[a][b] += (a == b ? sT : 0.0) + (sL - sT) * f[a] * f[b];
            }
    for (a = 0; a < 3; a++)
        for (b = 0; b < 3; b++)
            S[a][b] *= 0.125;
}

static int og_count_pairs(const og_grid *g, int part, int I, int J, int K, int a)
{
    int p, n = 0, lo[3], hi[3];
    for (p = 0; p < 4; p++) {
        og_pair(I, J, K, a, p, lo, hi);
        if (og_member(g, part, lo[0], lo[1], lo[2]) && og_member(g, part, hi[0], hi[1], hi[2]))
            n++;
    }
    return n;
}

/* Contribution of one part of vertex (I,J,K) to out = L u:  g = G'_p u,
 * F = S_p g, out += G'_p^T F. */
static void og_vertex_apply(const og_grid *g, int part, int I, int J, int K, double sL, double sT,
                            const double *u, double *out)
{
    double S[3][3], grad[3], F[3];
    int np[3], a, b, p, lo[3], hi[3];
    for (a = 0; a < 3; a++) {
        double sum = 0.0;
        np[a] = 0;
        for (p = 0; p < 4; p++) {
            og_pair(I, J, K, a, p, lo, hi);
            if (og_member(g, part, lo[0], lo[1], lo[2]) && og_member(g, part, hi[0], hi[1], hi[2])) {
                sum += u[og_idx(g, hi[0], hi[1], hi[2])] - u[og_idx(g, lo[0], lo[1], lo[2])];
                np[a]++;
            }
        }
        grad[a] = np[a] ? sum / (np[a] * g->dx) : 0.0;
    }
    if (!np[0] && !np[1] && !np[2])
        return;
    og_vertex_tensor(g, part, I, J, K, sL, sT, S);
    for (a = 0; a < 3; a++) {
        F[a] = 0.0;
        for (b = 0; b < 3; b++)
            F[a] += S[a][b] * grad[b];
    }
    for (a = 0; a < 3; a++) {
        if (!np[a])
            continue;
        double wgt = F[a] / (np[a] * g->dx);
        for (p = 0; p < 4; p++) {
            og_pair(I, J, K, a, p, lo, hi);
            if (og_member(g, part, lo[0], lo[1], lo[2]) && og_member(g, part, hi[0], hi[1], hi[2])) {
                out[og_idx(g, hi[0], hi[1], hi[2])] += wgt;
                out[og_idx(g, lo[0], lo[1], lo[2])] -= wgt;
            }
        }
    }
}

/* Contribution of one part of vertex (I,J,K) to the diagonal of L: for every
 * member voxel q of the block, c = d g_p / d u_q and diag_q += c^T S_p c. */
static void og_vertex_diag(const og_grid *g, int part, int I, int J, int K, double sL, double sT,
                           double *diag)
{
    double S[3][3];
    int np[3], a, b, s, t, u;
    for (a = 0; a < 3; a++)
        np[a] = og_count_pairs(g, part, I, J, K, a);
    if (!np[0] && !np[1] && !np[2])
        return;
    og_vertex_tensor(g, part, I, J, K, sL, sT, S);
    for (u = 0; u < 2; u++)
        for (t = 0; t < 2; t++)
            for (s = 0; s < 2; s++) {
                int q[3] = {I - 1 + s, J - 1 + t, K - 1 + u};
                int off[3] = {s, t, u};
                double c[3], acc = 0.0;
                if (!og_member(g, part, q[0], q[1], q[2]))
                    continue;
                for (a = 0; a < 3; a++) {
                    /* partner of q along a inside the block */
                    int r[3] = {q[0], q[1], q[2]};
                    r[a] += off[a] ? -1 : 1;
                    c[a] = 0.0;
                    if (np[a] && og_member(g, part, r[0], r[1], r[2]))
                        c[a] = (off[a] ? 1.0 : -1.0) / (np[a] * g->dx);
                }
                for (a = 0; a < 3; a++)
                    for (b = 0; b < 3; b++)
                        acc += c[a] * S[a][b] * c[b];
                diag[og_idx(g, q[0], q[1], q[2])] += acc;
            }
}

/* Vertex planes K and K+2 touch disjoint voxel planes, so the scatter runs
 * over even planes, then odd planes; every voxel gets its two contributions
 * in the same order whatever the thread count. */
void og_apply_L(const og_grid *g, double sL, double sT, const double *u, double *out)
{
    long n = (long)g->nx * g->ny * g->nz;
    int color;
    memset(out, 0, sizeof(double) * (size_t)n);
    for (color = 0; color < 2; color++) {
        int K;
#pragma omp parallel for schedule(static)
        for (K = color; K <= g->nz; K += 2) {
            int I, J;
            for (J = 0; J <= g->ny; J++)
                for (I = 0; I <= g->nx; I++) {
                    og_vertex_apply(g, OG_TISSUE, I, J, K, sL, sT, u, out);
                    if (g->torso)
                        og_vertex_apply(g, OG_TORSO, I, J, K, sL, sT, u, out);
                }
        }
    }
}

void og_diag_L(const og_grid *g, double sL, double sT, double *diag)
{
    long n = (long)g->nx * g->ny * g->nz;
    int color;
    memset(diag, 0, sizeof(double) * (size_t)n);
    for (color = 0; color < 2; color++) {
        int K;
#pragma omp parallel for schedule(static)
        for (K = color; K <= g->nz; K += 2) {
            int I, J;
            for (J = 0; J <= g->ny; J++)
                for (I = 0; I <= g->nx; I++) {
                    og_vertex_diag(g, OG_TISSUE, I, J, K, sL, sT, diag);
                    if (g->torso)
                        og_vertex_diag(g, OG_TORSO, I, J, K, sL, sT, diag);
                }
        }
    }
}

/* Face-connected (6-neighbour) components of the domain (tissue, and torso if
 * present); comp[q] = -1 outside. */
int og_components(const og_grid *g, int *comp)
{
    long n = (long)g->nx * g->ny * g->nz, q, head, tail;
    long *queue = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    int ncomp = 0;
    for (q = 0; q < n; q++)
        comp[q] = -1;
    for (q = 0; q < n; q++) {
        if (!og_in(g, q) || comp[q] >= 0)
            continue;
        head = tail = 0;
        queue[tail++] = q;
        comp[q] = ncomp;
        while (head < tail) {
            long c = queue[head++];
            int i = (int)(c % g->nx), j = (int)((c / g->nx) % g->ny), k = (int)(c / ((long)g->nx * g->ny));
            int d;
            for (d = 0; d < 6; d++) {
                int ii = i + (d == 0) - (d == 1), jj = j + (d == 2) - (d == 3), kk = k + (d == 4) - (d == 5);
                if (og_tissue(g, ii, jj, kk)) {
                    long r = og_idx(g, ii, jj, kk);
                    if (comp[r] < 0) {
                        comp[r] = ncomp;
                        queue[tail++] = r;
                    }
                }
            }
        }
        ncomp++;
    }
    free(queue);
    return ncomp;
}

/* x <- x - mean_c(x) on every component c (FP64, plain loop order). */
static void og_project(long n, int ncomp, const int *comp, double *x)
{
    double *sum = (double *)calloc((size_t)(ncomp > 0 ? ncomp : 1), sizeof(double));
    long *cnt = (long *)calloc((size_t)(ncomp > 0 ? ncomp : 1), sizeof(long));
    long q;
    for (q = 0; q < n; q++)
        if (comp[q] >= 0) {
            sum[comp[q]] += x[q];
            cnt[comp[q]]++;
        }
    for (q = 0; q < n; q++)
        if (comp[q] >= 0)
            x[q] -= sum[comp[q]] / (double)cnt[comp[q]];
    free(sum);
    free(cnt);
}

/* Default damping when the caller passes omega <= 0.  The thesis requires
 * damping but gives no value.  For a constant tensor with eigenvalues
 * (sL, sT, sT) the Fourier symbol of L on the infinite grid gives
 * rho(D^-1 L) <= 4 lambda_max(S) / (tr(S) / 2) = 8 sL / (sL + 2 sT); omega is
 * chosen so that omega * rho = 1.8 (capped at 1). */
double og_default_omega(double sL, double sT)
{
    double w = 1.8 * (sL + 2.0 * sT) / (8.0 * sL);
    return w > 1.0 ? 1.0 : w;
}

/* Damped Jacobi (Eq. dampjac1) for A x = b on the domain, A = L_{sL,sT}:
 *   r^k = b - A x^k ;  x^{k+1} = x^k + omega D^{-1} r^k   (x_q kept where D_q = 0).
 * At k = 0, m, 2m, ... the relative residual ||r^k|| / ||b|| is formed; when it
 * is <= tol the sweep that used r^k is the last one.  Stops with status 1
 * after max_iter sweeps.  If ||b|| = 0, x is left unchanged (0 sweeps). */
int og_jacobi(const og_grid *g, double sL, double sT, const double *b, double *x,
              double omega, double tol, int m, int max_iter, int *iters, double *relres)
{
    long n = (long)g->nx * g->ny * g->nz, q;
    double *diag = (double *)malloc(sizeof(double) * (size_t)n);
    double *Ax = (double *)malloc(sizeof(double) * (size_t)n);
    double nb = 0.0, nr = 0.0;
    int k = 0, status = 1;
    for (q = 0; q < n; q++)
        if (og_in(g, q))
            nb += b[q] * b[q];
    nb = sqrt(nb);
    *relres = 0.0;
    if (nb == 0.0) {
        *iters = 0;
        free(diag);
        free(Ax);
        return 0;
    }
    if (m < 1)
        m = 1;
    if (omega <= 0.0)
        omega = og_default_omega(sL, sT);
    og_diag_L(g, sL, sT, diag);
    for (k = 0; k < max_iter; k++) {
        og_apply_L(g, sL, sT, x, Ax);
        int check = (k % m) == 0;
        if (check)
            nr = 0.0;
        for (q = 0; q < n; q++) {
            if (!og_in(g, q))
                continue;
            double r = b[q] - Ax[q];
            if (check)
                nr += r * r;
            if (diag[q] > 0.0)      /* an isolated voxel has an empty row */
                x[q] += omega * r / diag[q];
        }
        if (check) {
            *relres = sqrt(nr) / nb;
            if (*relres <= tol) {
                status = 0;
                k++;
                break;
            }
        }
    }
    *iters = k;
    free(diag);
    free(Ax);
    return status;
}

/* Implicit-Euler Jacobi, Eq. iejac1, for (I + alpha L) x = f on the tissue
 * (the thesis writes (I - alpha A) with A = D + L + U its operator; here
 * A = -L_{sL,sT}, so its diagonal is -D and its off-diagonal part -(L - D)):
 *   x^{k+1} = [I + alpha D]^{-1} [ f - alpha (L - D) x^k ].
 * The stop rule is the one of og_jacobi: at k = 0, m, 2m, ... the relative
 * residual ||f - (I + alpha L) x^k|| / ||f|| is formed, and when it is <= tol
 * the sweep that used it is the last one.  Status 1 after max_iter sweeps;
 * ||f|| = 0 gives x = 0 after 0 sweeps. */
int og_ie_jacobi(const og_grid *g, double sL, double sT, double alpha, const double *f, double *x,
                 double tol, int m, int max_iter, int *iters, double *relres)
{
    long n = (long)g->nx * g->ny * g->nz, q;
    double *diag = (double *)malloc(sizeof(double) * (size_t)n);
    double *Lx = (double *)malloc(sizeof(double) * (size_t)n);
    double *xn = (double *)malloc(sizeof(double) * (size_t)n);
    double nf = 0.0, nr = 0.0;
    int k = 0, status = 1;
    for (q = 0; q < n; q++)
        if (og_in(g, q))
            nf += f[q] * f[q];
    nf = sqrt(nf);
    *relres = 0.0;
    if (nf == 0.0) {
        for (q = 0; q < n; q++)
            if (og_in(g, q))
                x[q] = 0.0;
        *iters = 0;
        free(diag);
        free(Lx);
        free(xn);
        return 0;
    }
    if (m < 1)
        m = 1;
    og_diag_L(g, sL, sT, diag);
    for (k = 0; k < max_iter; k++) {
        og_apply_L(g, sL, sT, x, Lx);
        int check = (k % m) == 0;
        if (check)
            nr = 0.0;
        for (q = 0; q < n; q++) {
            if (!og_in(g, q))
                continue;
            if (check) {
                double r = f[q] - (x[q] + alpha * Lx[q]);
                nr += r * r;
            }
            /* off-diagonal part of L applied to x^k: (L x)_q - D_q x_q */
            xn[q] = (f[q] - alpha * (Lx[q] - diag[q] * x[q])) / (1.0 + alpha * diag[q]);
        }
        for (q = 0; q < n; q++)
            if (og_in(g, q))
                x[q] = xn[q];
        if (check) {
            *relres = sqrt(nr) / nf;
            if (*relres <= tol) {
                status = 0;
                k++;
                break;
            }
        }
    }
    *iters = k;
    free(diag);
    free(Lx);
    free(xn);
    return status;
}

/* Chebyshev semi-iterative acceleration of the Jacobi iteration (not in the
 * thesis: its faster-solver future work; the method is Golub and Varga's,
 * 1961, as stated in Varga, "Matrix Iterative Analysis", Ch. 5).  For
 * A x = b with A = L_{sL,sT}, D = diag(A) and the eigenvalues of D^-1 A that
 * matter in [lmin, lmax], the basic step y -> y + tau D^-1 (b - A y),
 * tau = 2 / (lmin + lmax), has spectral radius rho = (lmax - lmin) / (lmax +
 * lmin) on that interval, and the semi-iteration is
 *   y_{k+1} = w_{k+1} (y_k + tau D^-1 (b - A y_k) - y_{k-1}) + y_{k-1},
 *   w_1 = 1,  w_2 = 2 / (2 - rho^2),  w_{k+1} = 1 / (1 - rho^2 w_k / 4).
 * Eigenvalue 0 (constants per component) is left alone, as in Jacobi.  Stop
 * rule and cap as og_jacobi. */
int og_chebyshev(const og_grid *g, double sL, double sT, const double *b, double *x, double lmin, double lmax,
                 double tol, int m, int max_iter, int *iters, double *relres)
{
    long n = (long)g->nx * g->ny * g->nz, q;
    double *diag = (double *)malloc(sizeof(double) * (size_t)n);
    double *Ax = (double *)malloc(sizeof(double) * (size_t)n);
    double *prev = (double *)malloc(sizeof(double) * (size_t)n);
    double nb = 0.0, nr = 0.0, w = 1.0;
    const double tau = 2.0 / (lmin + lmax), rho = (lmax - lmin) / (lmax + lmin);
    int k = 0, status = 1;
    for (q = 0; q < n; q++) {
        prev[q] = x[q];
        if (og_in(g, q))
            nb += b[q] * b[q];
    }
    nb = sqrt(nb);
    *relres = 0.0;
    if (nb == 0.0) {
        *iters = 0;
        free(diag);
        free(Ax);
        free(prev);
        return 0;
    }
    if (m < 1)
        m = 1;
    og_diag_L(g, sL, sT, diag);
    for (k = 0; k < max_iter; k++) {
        /* weight of this step: w_1 = 1, w_2 = 2 / (2 - rho^2), then the recurrence */
        if (k == 0)
            w = 1.0;
        else if (k == 1)
            w = 2.0 / (2.0 - rho * rho);
        else
            w = 1.0 / (1.0 - rho * rho * w / 4.0);
        og_apply_L(g, sL, sT, x, Ax);
        int check = (k % m) == 0;
        if (check)
            nr = 0.0;
        for (q = 0; q < n; q++) {
            if (!og_in(g, q))
                continue;
            double r = b[q] - Ax[q];
            if (check)
                nr += r * r;
            double basic = diag[q] > 0.0 ? x[q] + tau * r / diag[q] : x[q];
            double next = k == 0 ? basic : w * (basic - prev[q]) + prev[q];   /* y_1 = G y_0 + g */
            prev[q] = x[q];
            x[q] = next;
        }
        if (check) {
            *relres = sqrt(nr) / nb;
            if (*relres <= tol) {
                status = 0;
                k++;
                break;
            }
        }
    }
    *iters = k;
    free(diag);
    free(Ax);
    free(prev);
    return status;
}

/* Gauss-Seidel over eight colour classes: the deterministic form of the
 * thesis' in-place Jacobi, whose races let a sweep read values that other
 * work-items have already updated (Sec. "Jacobi method").  Voxel (i, j, k)
 * has colour (i mod 2) + 2 (j mod 2) + 4 (k mod 2).  Two voxels of one colour
 * differ by an even amount in some index, so the 27-point operator, which
 * reaches one voxel in each index, never couples them: the order within a
 * colour does not matter.  A sweep visits colours 0, 1, ..., 7; at colour c,
 * with A x formed from the current iterate (colours < c of this sweep already
 * updated), every domain voxel q of colour c with D_q > 0 takes
 *   r_q = b_q - (A x)_q,   x_q <- x_q + omega r_q / D_q
 * (successive over-relaxation; omega = 1 is Gauss-Seidel, omega <= 0 selects
 * 1).  Stop rule: at sweeps k = 0, m, 2m, ... the residuals r_q as they are
 * formed at their colour's update, squared and summed over all eight
 * colours, are compared with tol^2 ||b||^2; the sweep that forms the sum is
 * completed and, if it passes, is the last.  Status 1 after max_iter sweeps;
 * ||b|| = 0 returns at once after 0 sweeps. */
int og_gauss_seidel(const og_grid *g, double sL, double sT, const double *b, double *x, double omega,
                    double tol, int m, int max_iter, int *iters, double *relres)
{
    long n = (long)g->nx * g->ny * g->nz, q;
    double *diag = (double *)malloc(sizeof(double) * (size_t)n);
    double *Ax = (double *)malloc(sizeof(double) * (size_t)n);
    double nb = 0.0, nr = 0.0;
    int k = 0, status = 1, c;
    for (q = 0; q < n; q++)
        if (og_in(g, q))
            nb += b[q] * b[q];
    nb = sqrt(nb);
    *relres = 0.0;
    if (nb == 0.0) {
        *iters = 0;
        free(diag);
        free(Ax);
        return 0;
    }
    if (m < 1)
        m = 1;
    if (omega <= 0.0)
        omega = 1.0;
    og_diag_L(g, sL, sT, diag);
    for (k = 0; k < max_iter; k++) {
        int check = (k % m) == 0;
        if (check)
            nr = 0.0;
        for (c = 0; c < 8; c++) {
            og_apply_L(g, sL, sT, x, Ax);
            for (q = 0; q < n; q++) {
                int i = (int)(q % g->nx), j = (int)((q / g->nx) % g->ny), kk = (int)(q / ((long)g->nx * g->ny));
                if (!og_in(g, q) || (i & 1) + 2 * (j & 1) + 4 * (kk & 1) != c)
                    continue;
                double r = b[q] - Ax[q];
                if (check)
                    nr += r * r;
                if (diag[q] > 0.0)
                    x[q] += omega * r / diag[q];
            }
        }
        if (check) {
            *relres = sqrt(nr) / nb;
            if (*relres <= tol) {
                status = 0;
                k++;
                break;
            }
        }
    }
    *iters = k;
    free(diag);
    free(Ax);
    return status;
}

/* ------------------------------------------------------------------------ */
/* time stepping                                                            */
/* ------------------------------------------------------------------------ */

struct og_sim {
    og_grid g;                  /* tissue: membrane state and the intracellular operator */
    og_grid ge;                 /* domain of the elliptic equation: tissue, plus the torso if set */
    unsigned char *torso;       /* NULL without a torso */
    unsigned char *mask;
    double *fib;
    og_params p;
    og_stim *stim;
    int nstim;
    long n;
    int ncomp;
    int *comp;
    double *v, *w, *ve, *tact;
    double *vs, *tmp, *b, *u;
    long step;
    long total_iters;
    long ie_total_iters;
};

og_sim *og_create(int nx, int ny, int nz, double dx, const unsigned char *mask,
                  const double *fib, const og_params *p, const og_stim *stim, int nstim)
{
    og_sim *s = (og_sim *)calloc(1, sizeof(og_sim));
    long n = (long)nx * ny * nz, q;
    s->n = n;
    s->mask = (unsigned char *)malloc((size_t)n);
    memcpy(s->mask, mask, (size_t)n);
    s->fib = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    memcpy(s->fib, fib, sizeof(double) * 3 * (size_t)n);
    s->g.nx = nx;
    s->g.ny = ny;
    s->g.nz = nz;
    s->g.dx = dx;
    s->g.mask = s->mask;
    s->g.fib = s->fib;
    s->g.torso = NULL;
    s->g.sig_o = 0.0;
    s->ge = s->g;
    s->p = *p;
    s->nstim = nstim;
    s->stim = (og_stim *)malloc(sizeof(og_stim) * (size_t)(nstim > 0 ? nstim : 1));
    if (nstim > 0)
        memcpy(s->stim, stim, sizeof(og_stim) * (size_t)nstim);
    s->comp = (int *)malloc(sizeof(int) * (size_t)n);
    s->ncomp = og_components(&s->g, s->comp);
    s->v = (double *)calloc((size_t)n, sizeof(double));
    s->w = (double *)malloc(sizeof(double) * (size_t)n);
    s->ve = (double *)calloc((size_t)n, sizeof(double));
    s->tact = (double *)malloc(sizeof(double) * (size_t)n);
    s->vs = (double *)calloc((size_t)n, sizeof(double));
    s->tmp = (double *)calloc((size_t)n, sizeof(double));
    s->b = (double *)calloc((size_t)n, sizeof(double));
    s->u = (double *)calloc((size_t)n, sizeof(double));
    for (q = 0; q < n; q++) {
        s->w[q] = 1.0;
        s->tact[q] = -1.0;
    }
    return s;
}

void og_destroy(og_sim *s)
{
    if (!s)
        return;
    free(s->mask);
    free(s->fib);
    free(s->torso);
    free(s->stim);
    free(s->comp);
    free(s->v);
    free(s->w);
    free(s->ve);
    free(s->tact);
    free(s->vs);
    free(s->tmp);
    free(s->b);
    free(s->u);
    free(s);
}

/* Conducting torso around the tissue (voxels with torso[q] != 0 that are not
 * tissue), conductivity p->sig_o.  The elliptic equation, its null space
 * and v_e then live on tissue + torso.  Returns the number of domain
 * components. */
int og_set_torso(og_sim *s, const unsigned char *torso)
{
    long q;
    if (!s->torso)
        s->torso = (unsigned char *)malloc((size_t)s->n);
    for (q = 0; q < s->n; q++)
        s->torso[q] = (torso[q] != 0 && !s->mask[q]) ? 1 : 0;
    s->ge = s->g;
    s->ge.torso = s->torso;
    s->ge.sig_o = s->p.sig_o;
    s->ncomp = og_components(&s->ge, s->comp);
    return s->ncomp;
}

/* v, w are taken on the tissue, ve on the domain of the elliptic equation. */
void og_set_state(og_sim *s, const double *v, const double *w, const double *ve, long step)
{
    long q;
    for (q = 0; q < s->n; q++) {
        if (ve && og_in(&s->ge, q))
            s->ve[q] = ve[q];
        if (!s->mask[q])
            continue;
        if (v)
            s->v[q] = v[q];
        if (w)
            s->w[q] = w[q];
    }
    s->step = step;
}

void og_get_state(const og_sim *s, double *v, double *w, double *ve, double *tact, long *step)
{
    size_t bytes = sizeof(double) * (size_t)s->n;
    if (v)
        memcpy(v, s->v, bytes);
    if (w)
        memcpy(w, s->w, bytes);
    if (ve)
        memcpy(ve, s->ve, bytes);
    if (tact)
        memcpy(tact, s->tact, bytes);
    if (step)
        *step = s->step;
}

int og_ncomp(const og_sim *s) { return s->ncomp; }
long og_total_iters(const og_sim *s) { return s->total_iters; }
long og_ie_total_iters(const og_sim *s) { return s->ie_total_iters; }

/* One step n -> n+1 (t_n = n dt).  Returns 0, or 1 if the elliptic solve hit
 * its sweep cap (the step is still completed with the last iterate). */
int og_step(og_sim *s, int *iters, double *relres)
{
    const og_params *p = &s->p;
    const og_grid *g = &s->g;
    long q, n = s->n;
    double tn = (double)s->step * p->dt;
    int status = 0, si;
    *iters = 0;
    *relres = 0.0;

    /* 1. reaction: explicit Euler on (v, w), both from the old state */
    for (q = 0; q < n; q++) {
        if (!s->mask[q]) {
            s->vs[q] = s->v[q];
            continue;
        }
        int i = (int)(q % g->nx), j = (int)((q / g->nx) % g->ny), k = (int)(q / ((long)g->nx * g->ny));
        double v = s->v[q], w = s->w[q], jst = 0.0;
        for (si = 0; si < s->nstim; si++) {
            const og_stim *st = &s->stim[si];
            if (tn >= st->t_start && tn < st->t_start + st->dur &&
                i >= st->lo[0] && i < st->hi[0] && j >= st->lo[1] && j < st->hi[1] &&
                k >= st->lo[2] && k < st->hi[2])
                jst += st->amp;
        }
        double jin = v * v * (1.0 - v) * w / p->tau_in;
        double jout = -v / p->tau_out;
        double dw = (v < p->v_gate) ? (1.0 - w) / p->tau_open : -w / p->tau_close;
        s->vs[q] = v + p->dt * (jin + jout + jst);
        s->w[q] = w + p->dt * dw;
    }

    /* 2. parabolic diffusion, implicit Euler (Eq. iejac1) or explicit Euler */
    if (p->diffusion == OG_IMPLICIT) {
        double a = p->model == OG_MONO ? p->dt / p->K * p->lam / (1.0 + p->lam) : p->dt / p->K;
        int ie_it = 0;
        double ie_rr = 0.0;
        if (p->model == OG_MONO) {
            for (q = 0; q < n; q++)
                s->b[q] = s->mask[q] ? s->vs[q] : 0.0;
        } else {
            og_apply_L(g, p->sig_iL, p->sig_iT, s->ve, s->u);
            for (q = 0; q < n; q++)
                s->b[q] = s->mask[q] ? s->vs[q] - a * s->u[q] : 0.0;
        }
        for (q = 0; q < n; q++)          /* first iterate: the reaction update */
            s->tmp[q] = s->mask[q] ? s->vs[q] : 0.0;
        status |= og_ie_jacobi(g, p->sig_iL, p->sig_iT, a, s->b, s->tmp, p->rel_tol, p->check_every,
                               p->max_iter, &ie_it, &ie_rr);
        s->ie_total_iters += ie_it;
    } else if (p->model == OG_MONO) {
        og_apply_L(g, p->sig_iL, p->sig_iT, s->vs, s->tmp);
        double c = p->dt / p->K * p->lam / (1.0 + p->lam);
        for (q = 0; q < n; q++)
            if (s->mask[q])
                s->tmp[q] = s->vs[q] - c * s->tmp[q];
    } else {
        for (q = 0; q < n; q++)
            s->u[q] = s->mask[q] ? s->vs[q] + s->ve[q] : 0.0;
        og_apply_L(g, p->sig_iL, p->sig_iT, s->u, s->tmp);
        double c = p->dt / p->K;
        for (q = 0; q < n; q++)
            if (s->mask[q])
                s->tmp[q] = s->vs[q] - c * s->tmp[q];
    }

    /* activation time: first upward crossing of v = 0.5, linear in t */
    for (q = 0; q < n; q++) {
        if (!s->mask[q])
            continue;
        double v0 = s->v[q], v1 = s->tmp[q];
        if (s->tact[q] < 0.0 && v0 < 0.5 && v1 >= 0.5)
            s->tact[q] = tn + p->dt * (0.5 - v0) / (v1 - v0);
        s->v[q] = v1;
    }

    /* 3. elliptic: (L_i + L_e) ve = -L_i v+ (plus sig_o on the torso, where the
     *    right-hand side is 0), zero mean per component of the domain */
    if (p->model == OG_BI) {
        const og_grid *ge = &s->ge;
        og_apply_L(g, p->sig_iL, p->sig_iT, s->v, s->b);
        for (q = 0; q < n; q++)
            s->b[q] = s->mask[q] ? -s->b[q] : 0.0;
        og_project(n, s->ncomp, s->comp, s->b);
        if (p->solver == OG_CHEBYSHEV)
            status = og_chebyshev(ge, p->sig_iL + p->sig_eL, p->sig_iT + p->sig_eT, s->b, s->ve, p->cheb_lmin,
                                  p->cheb_lmax, p->rel_tol, p->check_every, p->max_iter, iters, relres);
        else if (p->solver == OG_GAUSS_SEIDEL)
            status = og_gauss_seidel(ge, p->sig_iL + p->sig_eL, p->sig_iT + p->sig_eT, s->b, s->ve, p->omega,
                                     p->rel_tol, p->check_every, p->max_iter, iters, relres);
        else
            status = og_jacobi(ge, p->sig_iL + p->sig_eL, p->sig_iT + p->sig_eT, s->b, s->ve,
                               p->omega, p->rel_tol, p->check_every, p->max_iter, iters, relres);
        og_project(n, s->ncomp, s->comp, s->ve);
        s->total_iters += *iters;
    }
    s->step++;
    return status;
}

int og_run(og_sim *s, int nsteps, int *last_iters, double *last_relres)
{
    int st = 0, k, it = 0;
    double rr = 0.0;
    for (k = 0; k < nsteps; k++)
        st |= og_step(s, &it, &rr);
    if (last_iters)
        *last_iters = it;
    if (last_relres)
        *last_relres = rr;
    return st;
}

/* ------------------------------------------------------------------------ */
/* geometry: signed distance functions and their two-pass encoding          */
/* ------------------------------------------------------------------------ */

/* Sec. "Geometry", subsections "Primitives" and "Encoding".  All arithmetic
 * that decides an integer (inside or outside) is FP32, as in the thesis'
 * kernels, one rounded operation at a time (the file is built without
 * contraction): translate, rotate (row by row, left to right), then the
 * primitive's formula:
 *   cuboid     max_i(|p_i / r_i|) - 1             (a box in the max norm)
 *   ellipsoid  |p / r|_2 - 1
 *   cylinder   max(|p_xy| - r, |p_z| - h)
 *   cone       max(|p_xy| - slope p_z - r, |p_z| - h)
 * and the set algebra union = min, intersection = max, S1 minus S2 =
 * max(s1, -s2), hollow = |s| - t.  The smoothed minimum is read as the
 * quadratic blend min(a, b) - h^2 k / 4, h = max(k - |a - b|, 0) / k (the
 * thesis shows it for several k without a formula). */
static float og_sdf_prim(const og_sdf_node *nd, const float x[3])
{
    float d[3], p[3];
    int i;
    for (i = 0; i < 3; i++)
        d[i] = x[i] - nd->centre[i];
    for (i = 0; i < 3; i++) {
        float t0 = nd->rot[3 * i] * d[0];
        float t1 = nd->rot[3 * i + 1] * d[1];
        float t2 = nd->rot[3 * i + 2] * d[2];
        p[i] = (t0 + t1) + t2;
    }
    switch (nd->op) {
    case OG_SDF_CUBOID: {
        float q0 = fabsf(p[0] / nd->a), q1 = fabsf(p[1] / nd->b), q2 = fabsf(p[2] / nd->c);
        return fmaxf(q0 - 1.0f, fmaxf(q1 - 1.0f, q2 - 1.0f));
    }
    case OG_SDF_ELLIPSOID: {
        float q0 = p[0] / nd->a, q1 = p[1] / nd->b, q2 = p[2] / nd->c;
        float s0 = q0 * q0, s1 = q1 * q1, s2 = q2 * q2;
        return sqrtf((s0 + s1) + s2) - 1.0f;
    }
    case OG_SDF_CYLINDER: {
        float s0 = p[0] * p[0], s1 = p[1] * p[1];
        return fmaxf(sqrtf(s0 + s1) - nd->a, fabsf(p[2]) - nd->b);
    }
    default: { /* OG_SDF_CONE */
        float s0 = p[0] * p[0], s1 = p[1] * p[1];
        float lean = nd->c * p[2];
        return fmaxf((sqrtf(s0 + s1) - lean) - nd->a, fabsf(p[2]) - nd->b);
    }
    }
}

float og_sdf_eval(const og_sdf_node *nodes, int count, const float x[3])
{
    float st[32];
    int sp = 0, i;
    for (i = 0; i < count; i++) {
        const og_sdf_node *nd = &nodes[i];
        if (nd->op < OG_SDF_UNION) {
            st[sp++] = og_sdf_prim(nd, x);
        } else if (nd->op == OG_SDF_HOLLOW) {
            st[sp - 1] = fabsf(st[sp - 1]) - nd->a;
        } else {
            float b = st[--sp], a = st[--sp], r;
            if (nd->op == OG_SDF_UNION)
                r = fminf(a, b);
            else if (nd->op == OG_SDF_INTERSECT)
                r = fmaxf(a, b);
            else if (nd->op == OG_SDF_SUBTRACT)
                r = fmaxf(a, -b);
            else { /* OG_SDF_SMOOTH_UNION */
                float k = nd->a;
                float h = fmaxf(k - fabsf(a - b), 0.0f) / k;
                float hh = h * h;
                float hk = hh * k;
                r = fminf(a, b) - hk * 0.25f;
            }
            st[sp++] = r;
        }
    }
    return st[0];
}

/* Volume pass: every voxel takes the kind of the last region whose SDF is
 * negative at its centre (0 = none); tissue = myocardium or fast fibre.
 * Fibres (FP64): myocardium follows Sec. "Fibre Directions" -- the horizontal
 * unit vector orthogonal to the position vector p (from the scene origin),
 * h = (-p_y, p_x, 0) / |p_xy|, rotated by helix_rad about p:
 * f = cos(a) h + sin(a) (p / |p|) x h (h is orthogonal to p); zero where p is
 * vertical.  Fast fibre: scale * axis.  Vertex pass: a vertex is 1 (solid)
 * when every voxel incident to it is tissue, 0 (fluid) when none is, 2
 * (surface) otherwise; only voxels inside the grid count.  Returns the number
 * of tissue voxels. */
int og_sdf_encode(const og_sdf_node *nodes, const og_sdf_region *regions, int n_regions, int nx, int ny, int nz,
                  float dx, const float origin[3], double helix_rad, unsigned char *label, unsigned char *mask,
                  double *fib, unsigned char *vclass)
{
    long q, n = (long)nx * ny * nz;
    int count = 0;
    const double ca = cos(helix_rad), sa = sin(helix_rad);
    for (q = 0; q < n; q++) {
        int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((long)nx * ny)), r;
        float x[3];
        float ci[3] = {(float)i + 0.5f, (float)j + 0.5f, (float)k + 0.5f};
        int c;
        for (c = 0; c < 3; c++)
            x[c] = origin[c] + ci[c] * dx;
        int last = -1;
        for (r = 0; r < n_regions; r++)
            if (og_sdf_eval(nodes + regions[r].first, regions[r].count, x) < 0.0f)
                last = r;
        int kind = last >= 0 ? regions[last].kind : 0;
        label[q] = (unsigned char)kind;
        mask[q] = (kind == OG_REGION_MYOCARDIUM || kind == OG_REGION_FAST) ? 1 : 0;
        fib[3 * q] = fib[3 * q + 1] = fib[3 * q + 2] = 0.0;
        if (kind == OG_REGION_MYOCARDIUM) {
            double px = x[0], py = x[1], pz = x[2];
            double hl = sqrt(px * px + py * py), pl = sqrt(px * px + py * py + pz * pz);
            if (hl > 0.0) {
                double h[3] = {-py / hl, px / hl, 0.0};
                double u[3] = {px / pl, py / pl, pz / pl};
                double w[3] = {u[1] * h[2] - u[2] * h[1], u[2] * h[0] - u[0] * h[2], u[0] * h[1] - u[1] * h[0]};
                for (c = 0; c < 3; c++)
                    fib[3 * q + c] = ca * h[c] + sa * w[c];
            }
        } else if (kind == OG_REGION_FAST) {
            for (c = 0; c < 3; c++)
                fib[3 * q + c] = (double)regions[last].scale * (double)regions[last].axis[c];
        }
        count += mask[q];
    }
    if (vclass) {
        int I, J, K;
        for (K = 0; K <= nz; K++)
            for (J = 0; J <= ny; J++)
                for (I = 0; I <= nx; I++) {
                    int in = 0, tis = 0, s, t, u;
                    for (u = 0; u < 2; u++)
                        for (t = 0; t < 2; t++)
                            for (s = 0; s < 2; s++) {
                                int i = I - 1 + s, j = J - 1 + t, k = K - 1 + u;
                                if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz)
                                    continue;
                                in++;
                                tis += mask[(long)i + (long)nx * ((long)j + (long)ny * k)];
                            }
                    vclass[(long)I + (long)(nx + 1) * ((long)J + (long)(ny + 1) * K)] =
                        (unsigned char)(tis == 0 ? 0 : (tis == in ? 1 : 2));
                }
    }
    return count;
}

int og_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
