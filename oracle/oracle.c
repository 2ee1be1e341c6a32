/*
 * FP64 CPU oracle for the P1 finite-element optical-flow system with an
 * illumination unknown (Gilliocq-Hirtz & Belhachmi, arXiv 1508.02977).
 *
 * TEST INFRASTRUCTURE ONLY.  This file defines what the CUDA library must
 * compute; it is written from the paper, shares no code with the CUDA path
 * and is only linked by the tests, by the package's smoke check and by the
 * CPU-baseline leg of the benchmark.  Nothing in the product path calls it.
 *
 * Plain and slow on purpose: every operator is formed element by element
 * from the 3x3 element matrices, the global matrix is stored in CSR, and the
 * solvers are textbook (banded Cholesky, block-Jacobi PCG, exact-solve
 * Schwarz).  No blocking or fusion.
 *
 * Conventions (readings of the paper where it is silent):
 *  - one node per pixel centre, W x H nodes, unit spacing (Section 2.2,
 *    Fig. sch-mesh: "each square represents a pixel");
 *  - square (x,y), 0<=x<W-1, 0<=y<H-1, is cut along (x,y)->(x+1,y+1):
 *      t=0: a=(x,y)  b=(x+1,y)  c=(x+1,y+1)
 *      t=1: a=(x,y)  d=(x,y+1)  c=(x+1,y+1)
 *    |K| = 1/2, diameter h_K = sqrt(2);
 *  - element data (Section 1, Eq. OF2, with K_sigma = K_rho = identity):
 *      g_K = (d/dx f2_h, d/dy f2_h, -mean_K f1),  ft_K = mean_K (f2 - f1)
 *    where f2_h is the P1 interpolant of frame 2 on K and means are over the
 *    three vertices (P0 coefficients);
 *  - unknowns U = (u1, u2, m) per node, m = delta m = M - 1 (Eq. deltam);
 *  - vectors are component planes [3][H][W]; alpha is [H-1][W-1][2];
 *  - the element matrix is the exact integral of the weak form (Eq. weakform,
 *    Eq. discret-form) for P1 functions and P0 coefficients:
 *      (A_K)_{(i,c),(j,d)} = |K|/12 (1+delta_ij) g_c g_d
 *                            + delta_cd |K| Lambda_c grad(phi_i).grad(phi_j)
 *      (b_K)_{(i,c)}       = -|K|/3 ft g_c
 *    with Lambda = (alpha_K, alpha_K, lambda)  (Eq. eqpro1illu, F = -ft g).
 *
 * Every function is pinned by tests (closed forms, quadrature of the energy,
 * dense LAPACK solves, invariants, finite differences); see the tests for
 * the pins.  The Schwarz iteration function follows Eq. schwarz step by step.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KAREA 0.5
#define HK 1.4142135623730951

/* ------------------------------------------------------------ geometry -- */

/* Vertices of triangle t of square (x,y) (Section 2.2). */
static void tri_vertices(int x, int y, int t, int vx[3], int vy[3])
{
    vx[0] = x;     vy[0] = y;
    if (t == 0) { vx[1] = x + 1; vy[1] = y; }
    else        { vx[1] = x;     vy[1] = y + 1; }
    vx[2] = x + 1; vy[2] = y + 1;
}

/* Constant gradients of the three P1 basis functions on triangle t. */
static void tri_grads(int t, double gx[3], double gy[3])
{
    if (t == 0) {
        /* phi_a = 1 - X, phi_b = X - Y, phi_c = Y  (local X, Y in [0,1]) */
        gx[0] = -1.0; gy[0] = 0.0;
        gx[1] = 1.0;  gy[1] = -1.0;
        gx[2] = 0.0;  gy[2] = 1.0;
    } else {
        /* phi_a = 1 - Y, phi_d = Y - X, phi_c = X */
        gx[0] = 0.0;  gy[0] = -1.0;
        gx[1] = -1.0; gy[1] = 1.0;
        gx[2] = 1.0;  gy[2] = 0.0;
    }
}

static long elem_index(int W, int x, int y, int t) { return ((long)y * (W - 1) + x) * 2 + t; }

/* ------------------------------------------------- element coefficients -- */

/* g_K (3 per element) and ft_K (1 per element) from the two frames. */
int orc_coefficients(int W, int H, const double *f1, const double *f2, double *g, double *ft)
{
    if (W < 2 || H < 2) return 1;
    for (int y = 0; y < H - 1; y++)
        for (int x = 0; x < W - 1; x++)
            for (int t = 0; t < 2; t++) {
                int vx[3], vy[3];
                double gx[3], gy[3];
                tri_vertices(x, y, t, vx, vy);
                tri_grads(t, gx, gy);
                double dfx = 0, dfy = 0, m1 = 0, mt = 0;
                for (int i = 0; i < 3; i++) {
                    double a = f1[(long)vy[i] * W + vx[i]];
                    double b = f2[(long)vy[i] * W + vx[i]];
                    dfx += b * gx[i];
                    dfy += b * gy[i];
                    m1 += a / 3.0;
                    mt += (b - a) / 3.0;
                }
                long e = elem_index(W, x, y, t);
                g[3 * e + 0] = dfx;
                g[3 * e + 1] = dfy;
                g[3 * e + 2] = -m1;
                ft[e] = mt;
            }
    return 0;
}

/* 9x9 element matrix (row/col index 3*i + c: vertex i, component c) and 9
 * element load entries. */
static void element_matrix(int t, const double g[3], double ft, double alpha, double lambda,
                           double K[9][9], double bK[9])
{
    double gx[3], gy[3];
    tri_grads(t, gx, gy);
    double lam[3] = {alpha, alpha, lambda};
    for (int i = 0; i < 3; i++)
        for (int c = 0; c < 3; c++) {
            for (int j = 0; j < 3; j++)
                for (int d = 0; d < 3; d++) {
                    double v = KAREA / 12.0 * (i == j ? 2.0 : 1.0) * (g[c] * g[d]);
                    if (c == d) v += KAREA * lam[c] * (gx[i] * gx[j] + gy[i] * gy[j]);
                    K[3 * i + c][3 * j + d] = v;
                }
            bK[3 * i + c] = -KAREA / 3.0 * ft * g[c];
        }
}

/* Element matrix with a general symmetric data tensor (Section 1, the
 * matrix A_rho and vector F with K_rho applied): the data block is
 * |K|/12 (1+delta_ij) A_cd, the load |K|/3 F_c.  A6 = (A00, A01, A02, A11,
 * A12, A22).  With A = g g^T and F = -ft g this is element_matrix. */
static void element_matrix_el(int t, const double A6[6], const double F[3], double alpha, double lambda,
                              double K[9][9], double bK[9])
{
    double gx[3], gy[3];
    tri_grads(t, gx, gy);
    const double Am[3][3] = {{A6[0], A6[1], A6[2]}, {A6[1], A6[3], A6[4]}, {A6[2], A6[4], A6[5]}};
    double lam[3] = {alpha, alpha, lambda};
    for (int i = 0; i < 3; i++)
        for (int c = 0; c < 3; c++) {
            for (int j = 0; j < 3; j++)
                for (int d = 0; d < 3; d++) {
                    double v = KAREA / 12.0 * (i == j ? 2.0 : 1.0) * Am[c][d];
                    if (c == d) v += KAREA * lam[c] * (gx[i] * gx[j] + gy[i] * gy[j]);
                    K[3 * i + c][3 * j + d] = v;
                }
            bK[3 * i + c] = KAREA / 3.0 * F[c];
        }
}

/* ------------------------------------------------------------ assembly -- */

/* Neighbour offsets of the 7-point pattern, in increasing linear order for a
 * row-major node index (dy major, dx minor). */
static const int NB_DX[7] = {-1, 0, -1, 0, 1, 0, 1};
static const int NB_DY[7] = {-1, -1, 0, 0, 0, 1, 1};

/* Number of stored entries of the CSR matrix of a W x H grid. */
int64_t orc_csr_nnz(int W, int H)
{
    int64_t nnz = 0;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            for (int k = 0; k < 7; k++) {
                int xx = x + NB_DX[k], yy = y + NB_DY[k];
                if (xx >= 0 && xx < W && yy >= 0 && yy < H) nnz += 3;
            }
    return nnz * 3;
}

/* Sparsity pattern: row (c, node) holds columns (d, node') for d = 0..2 and
 * node' in the 7-point pattern; unknown index = c*W*H + y*W + x.  Columns in
 * increasing order. */
int orc_csr_pattern(int W, int H, int64_t *rowptr, int64_t *col)
{
    long N = (long)W * H;
    int64_t p = 0;
    for (int c = 0; c < 3; c++)
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++) {
                rowptr[c * N + (long)y * W + x] = p;
                for (int d = 0; d < 3; d++)
                    for (int k = 0; k < 7; k++) {
                        int xx = x + NB_DX[k], yy = y + NB_DY[k];
                        if (xx >= 0 && xx < W && yy >= 0 && yy < H)
                            col[p++] = d * N + (long)yy * W + xx;
                    }
            }
    rowptr[3 * N] = p;
    return 0;
}

static int csr_add(const int64_t *rowptr, const int64_t *col, double *val, int64_t r, int64_t cidx, double v)
{
    for (int64_t p = rowptr[r]; p < rowptr[r + 1]; p++)
        if (col[p] == cidx) { val[p] += v; return 0; }
    return 1; /* entry not in the pattern: a bug, reported to the caller */
}

/* lambda of element e: the per-element field when given (Section 1: Lambda
 * piecewise constant per element), else the constant */
#define LAMBDA_OF(lamel, lambda, e) ((lamel) ? (lamel)[e] : (lambda))

/* Element-by-element assembly of A (values on the pattern above) and b;
 * lamel (may be NULL) is a per-element lambda [H-1][W-1][2]. */
int orc_assemble(int W, int H, const double *g, const double *ft, const double *alpha, double lambda,
                 const double *lamel, const int64_t *rowptr, const int64_t *col, double *val, double *b)
{
    long N = (long)W * H;
    memset(val, 0, sizeof(double) * rowptr[3 * N]);
    memset(b, 0, sizeof(double) * 3 * N);
    int bad = 0;
    /* two passes over square rows (even, then odd) so that rows assembled at
     * the same time touch disjoint node rows */
    for (int parity = 0; parity < 2; parity++) {
#pragma omp parallel for schedule(static) reduction(+ : bad)
        for (int y = parity; y < H - 1; y += 2)
            for (int x = 0; x < W - 1; x++)
                for (int t = 0; t < 2; t++) {
                    long e = elem_index(W, x, y, t);
                    double K[9][9], bK[9];
                    element_matrix(t, &g[3 * e], ft[e], alpha[e], LAMBDA_OF(lamel, lambda, e), K, bK);
                    int vx[3], vy[3];
                    tri_vertices(x, y, t, vx, vy);
                    for (int i = 0; i < 3; i++)
                        for (int c = 0; c < 3; c++) {
                            int64_t r = c * N + (long)vy[i] * W + vx[i];
                            b[r] += bK[3 * i + c];
                            for (int j = 0; j < 3; j++)
                                for (int d = 0; d < 3; d++)
                                    bad += csr_add(rowptr, col, val, r, d * N + (long)vy[j] * W + vx[j],
                                                   K[3 * i + c][3 * j + d]);
                        }
                }
    }
    return bad ? 2 : 0;
}

/* Assembly with general element data (K_rho > 0): Ael [H-1][W-1][2][6],
 * Fel [H-1][W-1][2][3]; otherwise as orc_assemble. */
int orc_assemble_el(int W, int H, const double *Ael, const double *Fel, const double *alpha, double lambda,
                    const double *lamel, const int64_t *rowptr, const int64_t *col, double *val, double *b)
{
    long N = (long)W * H;
    memset(val, 0, sizeof(double) * rowptr[3 * N]);
    memset(b, 0, sizeof(double) * 3 * N);
    int bad = 0;
    for (int parity = 0; parity < 2; parity++) {
#pragma omp parallel for schedule(static) reduction(+ : bad)
        for (int y = parity; y < H - 1; y += 2)
            for (int x = 0; x < W - 1; x++)
                for (int t = 0; t < 2; t++) {
                    long e = elem_index(W, x, y, t);
                    double K[9][9], bK[9];
                    element_matrix_el(t, &Ael[6 * e], &Fel[3 * e], alpha[e], LAMBDA_OF(lamel, lambda, e), K, bK);
                    int vx[3], vy[3];
                    tri_vertices(x, y, t, vx, vy);
                    for (int i = 0; i < 3; i++)
                        for (int c = 0; c < 3; c++) {
                            int64_t r = c * N + (long)vy[i] * W + vx[i];
                            b[r] += bK[3 * i + c];
                            for (int j = 0; j < 3; j++)
                                for (int d = 0; d < 3; d++)
                                    bad += csr_add(rowptr, col, val, r, d * N + (long)vy[j] * W + vx[j],
                                                   K[3 * i + c][3 * j + d]);
                        }
                }
    }
    return bad ? 2 : 0;
}

void orc_csr_matvec(int64_t n, const int64_t *rowptr, const int64_t *col, const double *val,
                    const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; r++) {
        double s = 0.0;
        for (int64_t p = rowptr[r]; p < rowptr[r + 1]; p++) s += val[p] * x[col[p]];
        y[r] = s;
    }
}

/* y = A x and, if b != NULL, r = b - A x, formed element by element without
 * storing A (for grids too large for the CSR). */
int orc_apply_elementwise(int W, int H, const double *g, const double *ft, const double *alpha, double lambda,
                          const double *lamel, const double *x, double *y, double *b)
{
    long N = (long)W * H;
    memset(y, 0, sizeof(double) * 3 * N);
    if (b) memset(b, 0, sizeof(double) * 3 * N);
    for (int parity = 0; parity < 2; parity++) {
#pragma omp parallel for schedule(static)
        for (int yy = parity; yy < H - 1; yy += 2)
            for (int xx = 0; xx < W - 1; xx++)
                for (int t = 0; t < 2; t++) {
                    long e = elem_index(W, xx, yy, t);
                    double K[9][9], bK[9];
                    element_matrix(t, &g[3 * e], ft[e], alpha[e], LAMBDA_OF(lamel, lambda, e), K, bK);
                    int vx[3], vy[3];
                    tri_vertices(xx, yy, t, vx, vy);
                    double xl[9];
                    for (int j = 0; j < 3; j++)
                        for (int d = 0; d < 3; d++) xl[3 * j + d] = x[d * N + (long)vy[j] * W + vx[j]];
                    for (int i = 0; i < 3; i++)
                        for (int c = 0; c < 3; c++) {
                            double s = 0.0;
                            for (int k = 0; k < 9; k++) s += K[3 * i + c][k] * xl[k];
                            long r = c * N + (long)vy[i] * W + vx[i];
                            y[r] += s;
                            if (b) b[r] += bK[3 * i + c];
                        }
                }
    }
    return 0;
}

/* ---------------------------------------------------- banded Cholesky -- */

/* Banded Cholesky factor of the CSR matrix of a W x H grid.  Unknowns are
 * renumbered node-major with the shorter grid side as the fast index, giving
 * half-bandwidth bw = 3*(min(W,H)+1)+2; L is stored by rows, entry (i, j),
 * j <= i, at L[i*(bw+1) + (i-j)]. */
typedef struct {
    long n, bw;
    long *perm; /* perm[global] = banded index */
    double *L;
} band_t;

static void band_free(band_t *F)
{
    free(F->perm);
    free(F->L);
    F->perm = NULL;
    F->L = NULL;
}

/* Returns 0, 3 if A is not positive definite, 4 on allocation failure, 5 if
 * an entry lies outside the band. */
static int band_factor(int W, int H, const int64_t *rowptr, const int64_t *col, const double *val, band_t *F)
{
    long N = (long)W * H;
    long n = 3 * N;
    int fastW = (W <= H);
    long fast = fastW ? W : H;
    long bw = 3 * (fast + 1) + 2;
    F->n = n;
    F->bw = bw;
    F->perm = malloc(sizeof(long) * n);
    F->L = calloc((size_t)n * (bw + 1), sizeof(double));
    if (!F->perm || !F->L) { band_free(F); return 4; }
    long *perm = F->perm;
    double *L = F->L;
    for (int c = 0; c < 3; c++)
        for (int y = 0; y < H; y++)
            for (int xx = 0; xx < W; xx++) {
                long node = fastW ? ((long)y * W + xx) : ((long)xx * H + y);
                perm[c * N + (long)y * W + xx] = 3 * node + c;
            }
    /* scatter the lower triangle: L[i*(bw+1) + (i-j)] = A[i][j], j <= i */
    for (long r = 0; r < n; r++)
        for (int64_t p = rowptr[r]; p < rowptr[r + 1]; p++) {
            long i = perm[r], j = perm[col[p]];
            if (j <= i) {
                if (i - j > bw) { band_free(F); return 5; }
                L[i * (bw + 1) + (i - j)] = val[p];
            }
        }
    for (long j = 0; j < n; j++) {
        double d = L[j * (bw + 1)];
        long k0 = j - bw > 0 ? j - bw : 0;
        for (long k = k0; k < j; k++) { double v = L[j * (bw + 1) + (j - k)]; d -= v * v; }
        if (!(d > 0.0)) { band_free(F); return 3; }
        d = sqrt(d);
        L[j * (bw + 1)] = d;
        long i1 = j + bw < n - 1 ? j + bw : n - 1;
        for (long i = j + 1; i <= i1; i++) {
            double s = L[i * (bw + 1) + (i - j)];
            long kk0 = i - bw > 0 ? i - bw : 0;
            for (long k = kk0; k < j; k++) s -= L[i * (bw + 1) + (i - k)] * L[j * (bw + 1) + (j - k)];
            L[i * (bw + 1) + (i - j)] = s / d;
        }
    }
    return 0;
}

/* x = A^{-1} b from the factor: forward L z = P b, backward L^T w = z.  z is
 * work space of n doubles. */
static void band_solve(const band_t *F, const double *b, double *x, double *z)
{
    const long n = F->n, bw = F->bw;
    const long *perm = F->perm;
    const double *L = F->L;
    for (long r = 0; r < n; r++) z[perm[r]] = b[r];
    for (long i = 0; i < n; i++) {
        double s = z[i];
        long k0 = i - bw > 0 ? i - bw : 0;
        for (long k = k0; k < i; k++) s -= L[i * (bw + 1) + (i - k)] * z[k];
        z[i] = s / L[i * (bw + 1)];
    }
    for (long i = n - 1; i >= 0; i--) {
        double s = z[i];
        long k1 = i + bw < n - 1 ? i + bw : n - 1;
        for (long k = i + 1; k <= k1; k++) s -= L[k * (bw + 1) + (k - i)] * z[k];
        z[i] = s / L[i * (bw + 1)];
    }
    for (long r = 0; r < n; r++) x[r] = z[perm[r]];
}

/* Solves A x = b for the CSR matrix of a W x H grid by banded Cholesky.
 * Returns 3 if A is not positive definite, 4 on allocation failure. */
int orc_band_cholesky_solve(int W, int H, const int64_t *rowptr, const int64_t *col, const double *val,
                            const double *b, double *x)
{
    band_t F = {0, 0, NULL, NULL};
    int rc = band_factor(W, H, rowptr, col, val, &F);
    if (rc) return rc;
    double *z = malloc(sizeof(double) * F.n);
    if (!z) { band_free(&F); return 4; }
    band_solve(&F, b, x, z);
    free(z);
    band_free(&F);
    return 0;
}

/* ------------------------------------------------------------------ PCG -- */

static double dot(long n, const double *a, const double *b)
{
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (long i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* Inverse of the 3x3 node block of A (cofactors / determinant). */
static int inv3(const double a[9], double inv[9])
{
    double c00 = a[4] * a[8] - a[5] * a[7];
    double c01 = a[5] * a[6] - a[3] * a[8];
    double c02 = a[3] * a[7] - a[4] * a[6];
    double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    if (!(fabs(det) > 0.0)) return 1;
    inv[0] = c00 / det;
    inv[1] = (a[2] * a[7] - a[1] * a[8]) / det;
    inv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
    inv[3] = c01 / det;
    inv[4] = (a[0] * a[8] - a[2] * a[6]) / det;
    inv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
    inv[6] = c02 / det;
    inv[7] = (a[1] * a[6] - a[0] * a[7]) / det;
    inv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
    return 0;
}

/* Conjugate gradients with the node-block Jacobi preconditioner, FP64.
 * Starts from x (warm start), stops when ||b - A x||_2 <= tol ||b||_2.
 * Returns the iteration count, or -1 on breakdown / allocation failure;
 * *relres receives the final relative residual (recomputed as b - A x). */
int orc_pcg(int W, int H, const int64_t *rowptr, const int64_t *col, const double *val,
            const double *b, double *x, double tol, int maxit, double *relres)
{
    long N = (long)W * H, n = 3 * N;
    double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
    double *p = malloc(sizeof(double) * n), *q = malloc(sizeof(double) * n);
    double *Dinv = malloc(sizeof(double) * 9 * N);
    if (!r || !z || !p || !q || !Dinv) { free(r); free(z); free(p); free(q); free(Dinv); return -1; }
    int fail = 0;
    for (long node = 0; node < N; node++) {
        double blk[9] = {0};
        for (int c = 0; c < 3; c++)
            for (int64_t pp = rowptr[c * N + node]; pp < rowptr[c * N + node + 1]; pp++)
                if (col[pp] % N == node) blk[3 * c + col[pp] / N] = val[pp];
        fail |= inv3(blk, &Dinv[9 * node]);
    }
    if (fail) { free(r); free(z); free(p); free(q); free(Dinv); return -1; }
    orc_csr_matvec(n, rowptr, col, val, x, q);
    for (long i = 0; i < n; i++) r[i] = b[i] - q[i];
    double nb = sqrt(dot(n, b, b));
    if (nb == 0.0) nb = 1.0;
    int it = 0;
    double rz = 0.0;
    double rn = sqrt(dot(n, r, r));
    while (rn > tol * nb && it < maxit) {
        for (long node = 0; node < N; node++)
            for (int c = 0; c < 3; c++) {
                double s = 0;
                for (int d = 0; d < 3; d++) s += Dinv[9 * node + 3 * c + d] * r[d * N + node];
                z[c * N + node] = s;
            }
        double rz_new = dot(n, r, z);
        if (it == 0) memcpy(p, z, sizeof(double) * n);
        else {
            double beta = rz_new / rz;
            for (long i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        }
        rz = rz_new;
        orc_csr_matvec(n, rowptr, col, val, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) { it = -1; break; }
        double a = rz / pq;
        for (long i = 0; i < n; i++) { x[i] += a * p[i]; r[i] -= a * q[i]; }
        rn = sqrt(dot(n, r, r));
        it++;
    }
    orc_csr_matvec(n, rowptr, col, val, x, q);
    for (long i = 0; i < n; i++) r[i] = b[i] - q[i];
    if (relres) *relres = sqrt(dot(n, r, r)) / nb;
    free(r); free(z); free(p); free(q); free(Dinv);
    return it;
}

/* ------------------------------------------------- Schwarz (Eq. schwarz) -- */

/* Subdomain bounds of a px x py partition: owned [x0,x1) x [y0,y1), tiles of
 * near-equal size (boundary k at floor(k*W/px)); extended by `ov` node
 * layers on every side that is not on the image boundary. */
static void subdomain(int W, int H, int px, int py, int i, int ov, int own[4], int ext[4])
{
    int ix = i % px, iy = i / px;
    own[0] = (int)((long)ix * W / px);
    own[1] = (int)((long)(ix + 1) * W / px);
    own[2] = (int)((long)iy * H / py);
    own[3] = (int)((long)(iy + 1) * H / py);
    ext[0] = own[0] - ov < 0 ? 0 : own[0] - ov;
    ext[1] = own[1] + ov > W ? W : own[1] + ov;
    ext[2] = own[2] - ov < 0 ? 0 : own[2] - ov;
    ext[3] = own[3] + ov > H ? H : own[3] + ov;
}

/* The paper's Schwarz iteration (Eq. schwarz), algebraic form: at sweep k
 * every subdomain solves its extended problem exactly, with Dirichlet data
 * U^{k-1} taken from the previous global iterate at the nodes outside its
 * extended tile (Gamma_ij), natural (Neumann) conditions on the image
 * boundary; the new global iterate takes each node's value from the
 * subdomain that owns it.  Starts from U (in/out), runs `iters` sweeps and
 * records ||U^k - U^{k-1}||_2 per sweep in hist (may be NULL). */
int orc_schwarz(int W, int H, const int64_t *rowptr, const int64_t *col, const double *val,
                const double *b, int px, int py, int ov, int iters, double *U, double *hist)
{
    long N = (long)W * H, n = 3 * N;
    int nsub = px * py;
    double *Unew = malloc(sizeof(double) * n);
    if (!Unew) return 4;
    int rc = 0;
    for (int k = 0; k < iters && !rc; k++) {
        memcpy(Unew, U, sizeof(double) * n);
        for (int s = 0; s < nsub && !rc; s++) {
            int own[4], ext[4];
            subdomain(W, H, px, py, s, ov, own, ext);
            int w = ext[1] - ext[0], h = ext[3] - ext[2];
            long m = 3L * w * h;
            /* local numbering: c*w*h + (y-ext2)*w + (x-ext0) */
            long *loc = malloc(sizeof(long) * n);
            double *rhs = malloc(sizeof(double) * m), *sol = malloc(sizeof(double) * m);
            int64_t nnzl = orc_csr_nnz(w, h);
            int64_t *rp = malloc(sizeof(int64_t) * (m + 1)), *cl = malloc(sizeof(int64_t) * nnzl);
            double *vl = calloc(nnzl, sizeof(double));
            if (!loc || !rhs || !sol || !rp || !cl || !vl) rc = 4;
            if (!rc) {
                for (long i = 0; i < n; i++) loc[i] = -1;
                for (int c = 0; c < 3; c++)
                    for (int y = ext[2]; y < ext[3]; y++)
                        for (int x = ext[0]; x < ext[1]; x++)
                            loc[c * N + (long)y * W + x] = c * (long)w * h + (long)(y - ext[2]) * w + (x - ext[0]);
                orc_csr_pattern(w, h, rp, cl);
                /* local matrix = rows/cols of A inside the extended tile;
                 * RHS = b - (couplings to outside nodes) * U^{k-1} */
                for (long r = 0; r < n; r++) {
                    long lr = loc[r];
                    if (lr < 0) continue;
                    double s = b[r];
                    for (int64_t p = rowptr[r]; p < rowptr[r + 1]; p++) {
                        long lc = loc[col[p]];
                        if (lc < 0) s -= val[p] * U[col[p]];
                        else if (csr_add(rp, cl, vl, lr, lc, val[p])) rc = 2;
                    }
                    rhs[lr] = s;
                }
            }
            if (!rc) rc = orc_band_cholesky_solve(w, h, rp, cl, vl, rhs, sol);
            if (!rc)
                for (int c = 0; c < 3; c++)
                    for (int y = own[2]; y < own[3]; y++)
                        for (int x = own[0]; x < own[1]; x++) {
                            long gi = c * N + (long)y * W + x;
                            Unew[gi] = sol[loc[gi]];
                        }
            free(loc); free(rhs); free(sol); free(rp); free(cl); free(vl);
        }
        if (rc) break;
        double d = 0.0;
        for (long i = 0; i < n; i++) { double e = Unew[i] - U[i]; d += e * e; }
        if (hist) hist[k] = sqrt(d);
        memcpy(U, Unew, sizeof(double) * n);
    }
    free(Unew);
    return rc;
}

/* ------------------------------- PCG with additive Schwarz (large grids) -- */

/* The rows and columns of A inside the extended tile ext = [x0,x1) x [y0,y1),
 * stored as the CSR matrix of a w x h grid (local unknown c*w*h + (y-y0)*w +
 * (x-x0)): the local matrix A_i = R_i A R_i^T of a subdomain with zero
 * Dirichlet values outside it. */
static int local_matrix(int W, int H, const int64_t *rowptr, const int64_t *col, const double *val,
                        const int ext[4], int64_t *rp, int64_t *cl, double *vl)
{
    long N = (long)W * H;
    int w = ext[1] - ext[0], h = ext[3] - ext[2];
    long wh = (long)w * h;
    orc_csr_pattern(w, h, rp, cl);
    memset(vl, 0, sizeof(double) * rp[3 * wh]);
    for (int c = 0; c < 3; c++)
        for (int y = ext[2]; y < ext[3]; y++)
            for (int x = ext[0]; x < ext[1]; x++) {
                long r = c * N + (long)y * W + x;
                long lr = c * wh + (long)(y - ext[2]) * w + (x - ext[0]);
                for (int64_t p = rowptr[r]; p < rowptr[r + 1]; p++) {
                    long gc = col[p], nd = gc % N;
                    int d = (int)(gc / N), yy = (int)(nd / W), xx = (int)(nd % W);
                    if (xx < ext[0] || xx >= ext[1] || yy < ext[2] || yy >= ext[3]) continue;
                    long lc = d * wh + (long)(yy - ext[2]) * w + (xx - ext[0]);
                    if (csr_add(rp, cl, vl, lr, lc, val[p])) return 2;
                }
            }
    return 0;
}

/* Conjugate gradients with the one-level additive Schwarz preconditioner
 * with exact subdomain solves (the textbook ASM):
 *     z = sum_i R_i^T A_i^{-1} R_i r,
 * R_i the restriction to the extended tile i of a px x py partition (tiles
 * of near-equal size, extended by ov node layers where not on the image
 * boundary: the subdomains of orc_schwarz), A_i = R_i A R_i^T factored once
 * by banded Cholesky.  The sum is symmetric positive definite, so CG applies.
 * The local solves run in parallel into separate buffers and are added in
 * tile order (deterministic).  Starts from x, stops when ||b - A x||_2 <=
 * tol ||b||_2 (the recursive residual; *relres is recomputed as b - A x).
 * Returns the iteration count, -1 on breakdown or a failed factorisation,
 * -2 on allocation failure. */
int orc_asm_pcg(int W, int H, const int64_t *rowptr, const int64_t *col, const double *val,
                const double *b, double *x, int px, int py, int ov, double tol, int maxit, double *relres)
{
    long N = (long)W * H, n = 3 * N;
    int nsub = px * py;
    band_t *F = calloc(nsub, sizeof(band_t));
    long *off = malloc(sizeof(long) * (nsub + 1));
    int (*ext)[4] = malloc(sizeof(int[4]) * nsub);
    if (!F || !off || !ext) { free(F); free(off); free(ext); return -2; }
    long maxm = 0;
    off[0] = 0;
    for (int s = 0; s < nsub; s++) {
        int own[4];
        subdomain(W, H, px, py, s, ov, own, ext[s]);
        long m = 3L * (ext[s][1] - ext[s][0]) * (ext[s][3] - ext[s][2]);
        off[s + 1] = off[s] + m;
        if (m > maxm) maxm = m;
    }
    int fail = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : fail)
    for (int s = 0; s < nsub; s++) {
        int w = ext[s][1] - ext[s][0], h = ext[s][3] - ext[s][2];
        int64_t nnzl = orc_csr_nnz(w, h);
        long m = 3L * w * h;
        int64_t *rp = malloc(sizeof(int64_t) * (m + 1)), *cl = malloc(sizeof(int64_t) * nnzl);
        double *vl = malloc(sizeof(double) * nnzl);
        if (!rp || !cl || !vl) fail |= 4;
        else if (local_matrix(W, H, rowptr, col, val, ext[s], rp, cl, vl)) fail |= 2;
        else if (band_factor(w, h, rp, cl, vl, &F[s])) fail |= 1;
        free(rp); free(cl); free(vl);
    }
    double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n);
    double *p = malloc(sizeof(double) * n), *q = malloc(sizeof(double) * n);
    double *loc = malloc(sizeof(double) * (off[nsub] > 0 ? off[nsub] : 1));
    int it = 0;
    if (fail || !r || !z || !p || !q || !loc) {
        it = (fail & 4) || !r || !z || !p || !q || !loc ? -2 : -1;
        goto done;
    }
    orc_csr_matvec(n, rowptr, col, val, x, q);
    for (long i = 0; i < n; i++) r[i] = b[i] - q[i];
    double nb = sqrt(dot(n, b, b));
    if (nb == 0.0) nb = 1.0;
    double rz = 0.0;
    double rn = sqrt(dot(n, r, r));
    while (rn > tol * nb && it < maxit) {
        /* z = M r: local solves of R_i r, then the sum of R_i^T z_i */
        int afail = 0;
#pragma omp parallel reduction(| : afail)
        {
            double *rhs = malloc(sizeof(double) * maxm), *wk = malloc(sizeof(double) * maxm);
            if (!rhs || !wk) afail |= 1;
#pragma omp for schedule(dynamic)
            for (int s = 0; s < nsub; s++) {
                if (!rhs || !wk) continue;
                int w = ext[s][1] - ext[s][0], h = ext[s][3] - ext[s][2];
                long wh = (long)w * h;
                for (int c = 0; c < 3; c++)
                    for (int y = ext[s][2]; y < ext[s][3]; y++)
                        for (int xx = ext[s][0]; xx < ext[s][1]; xx++)
                            rhs[c * wh + (long)(y - ext[s][2]) * w + (xx - ext[s][0])] = r[c * N + (long)y * W + xx];
                band_solve(&F[s], rhs, loc + off[s], wk);
            }
            free(rhs); free(wk);
        }
        if (afail) { it = -2; goto done; }
        memset(z, 0, sizeof(double) * n);
        for (int s = 0; s < nsub; s++) {
            int w = ext[s][1] - ext[s][0], h = ext[s][3] - ext[s][2];
            long wh = (long)w * h;
            const double *zl = loc + off[s];
            for (int c = 0; c < 3; c++)
                for (int y = ext[s][2]; y < ext[s][3]; y++)
                    for (int xx = ext[s][0]; xx < ext[s][1]; xx++)
                        z[c * N + (long)y * W + xx] += zl[c * wh + (long)(y - ext[s][2]) * w + (xx - ext[s][0])];
        }
        double rz_new = dot(n, r, z);
        if (it == 0) memcpy(p, z, sizeof(double) * n);
        else {
            double beta = rz_new / rz;
            for (long i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        }
        rz = rz_new;
        orc_csr_matvec(n, rowptr, col, val, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) { it = -1; goto done; }
        double a = rz / pq;
        for (long i = 0; i < n; i++) { x[i] += a * p[i]; r[i] -= a * q[i]; }
        rn = sqrt(dot(n, r, r));
        it++;
    }
    orc_csr_matvec(n, rowptr, col, val, x, q);
    for (long i = 0; i < n; i++) r[i] = b[i] - q[i];
    if (relres) *relres = sqrt(dot(n, r, r)) / nb;
done:
    for (int s = 0; s < nsub; s++) band_free(&F[s]);
    free(F); free(off); free(ext); free(r); free(z); free(p); free(q); free(loc);
    return it;
}

/* --------------------------------------- error indicator (Eq. errind) -- */

/* eta_K for every element (Section 2.3, Eq. errind), read as
 *   eta_K = h_K || Lambda_K^{-1/2} R_K ||_{L2(K)}
 *         + 1/2 sum_{e in K} h_e^{1/2} || Lambda_e^{-1/2} J_e ||_{L2(e)}
 * with R_K = F + div(Lambda grad U) - A U = -g (g.U + ft) inside K (the
 * divergence of a P1 flux with constant Lambda vanishes), J_e the jump
 * (outside minus inside) of Lambda grad U . n_e across e, outside flux 0 on
 * the image boundary (Neumann), Lambda_e the componentwise max over the two
 * elements of e, Lambda^{-1/2} applied per component inside the Euclidean
 * norm.  L2(K) by the edge-midpoint rule (exact for the quadratic
 * integrand); the jump is constant on e. */
static int indicator_impl(int W, int H, const double *g, const double *ft, const double *Ael, const double *Fel,
                          const double *alpha, double lambda, const double *lamel, const double *U, double *eta)
{
    long N = (long)W * H;
    /* per-element flux gradients */
    long NE = 2L * (W - 1) * (H - 1);
    double *grad = malloc(sizeof(double) * 6 * NE); /* [e][c][2] */
    if (!grad) return 4;
    for (int y = 0; y < H - 1; y++)
        for (int x = 0; x < W - 1; x++)
            for (int t = 0; t < 2; t++) {
                int vx[3], vy[3];
                double gx[3], gy[3];
                tri_vertices(x, y, t, vx, vy);
                tri_grads(t, gx, gy);
                long e = elem_index(W, x, y, t);
                for (int c = 0; c < 3; c++) {
                    double sx = 0, sy = 0;
                    for (int i = 0; i < 3; i++) {
                        double u = U[c * N + (long)vy[i] * W + vx[i]];
                        sx += u * gx[i];
                        sy += u * gy[i];
                    }
                    grad[6 * e + 2 * c + 0] = sx;
                    grad[6 * e + 2 * c + 1] = sy;
                }
            }
    for (int y = 0; y < H - 1; y++)
        for (int x = 0; x < W - 1; x++)
            for (int t = 0; t < 2; t++) {
                long e = elem_index(W, x, y, t);
                const double *ge = g ? &g[3 * e] : NULL;
                double lamK[3] = {alpha[e], alpha[e], LAMBDA_OF(lamel, lambda, e)};
                int vx[3], vy[3];
                tri_vertices(x, y, t, vx, vy);
                /* interior term: integrate |Lambda^{-1/2} R|^2 over K by the
                 * edge-midpoint rule  int_K q = |K|/3 sum_{midpoints} q */
                double integ = 0.0;
                for (int a = 0; a < 3; a++) {
                    int bb = (a + 1) % 3;
                    double um[3];
                    for (int c = 0; c < 3; c++)
                        um[c] = 0.5 * (U[c * N + (long)vy[a] * W + vx[a]] + U[c * N + (long)vy[bb] * W + vx[bb]]);
                    double q = 0.0;
                    if (!Ael) {
                        /* R = F - A U = -g (g.U + ft) */
                        double s = ft[e];
                        for (int c = 0; c < 3; c++) s += ge[c] * um[c];
                        for (int c = 0; c < 3; c++) {
                            double R = -ge[c] * s;
                            q += R * R / lamK[c];
                        }
                    } else {
                        /* R = F - A U with the general element tensor */
                        const double *A6 = &Ael[6 * e];
                        const double Am[3][3] = {{A6[0], A6[1], A6[2]}, {A6[1], A6[3], A6[4]}, {A6[2], A6[4], A6[5]}};
                        for (int c = 0; c < 3; c++) {
                            double R = Fel[3 * e + c];
                            for (int d = 0; d < 3; d++) R -= Am[c][d] * um[d];
                            q += R * R / lamK[c];
                        }
                    }
                    integ += KAREA / 3.0 * q;
                }
                double val = HK * sqrt(integ);
                /* edges: (outward normal, neighbour element, length) */
                double nx[3], ny[3], he[3];
                long nbr[3];
                if (t == 0) {
                    nx[0] = 0;  ny[0] = -1; he[0] = 1.0; nbr[0] = y > 0 ? elem_index(W, x, y - 1, 1) : -1;      /* bottom */
                    nx[1] = 1;  ny[1] = 0;  he[1] = 1.0; nbr[1] = x < W - 2 ? elem_index(W, x + 1, y, 1) : -1;  /* right */
                    nx[2] = -M_SQRT1_2; ny[2] = M_SQRT1_2; he[2] = HK; nbr[2] = elem_index(W, x, y, 1);          /* diagonal */
                } else {
                    nx[0] = -1; ny[0] = 0;  he[0] = 1.0; nbr[0] = x > 0 ? elem_index(W, x - 1, y, 0) : -1;      /* left */
                    nx[1] = 0;  ny[1] = 1;  he[1] = 1.0; nbr[1] = y < H - 2 ? elem_index(W, x, y + 1, 0) : -1;  /* top */
                    nx[2] = M_SQRT1_2; ny[2] = -M_SQRT1_2; he[2] = HK; nbr[2] = elem_index(W, x, y, 0);          /* diagonal */
                }
                for (int k = 0; k < 3; k++) {
                    double q = 0.0;
                    for (int c = 0; c < 3; c++) {
                        double in = lamK[c] * (grad[6 * e + 2 * c] * nx[k] + grad[6 * e + 2 * c + 1] * ny[k]);
                        double out = 0.0, lamE = lamK[c];
                        if (nbr[k] >= 0) {
                            long o = nbr[k];
                            double lamO = c < 2 ? alpha[o] : LAMBDA_OF(lamel, lambda, o);
                            out = lamO * (grad[6 * o + 2 * c] * nx[k] + grad[6 * o + 2 * c + 1] * ny[k]);
                            lamE = lamO > lamE ? lamO : lamE;
                        }
                        double J = out - in;
                        q += J * J / lamE;
                    }
                    /* || . ||_{L2(e)} of a constant = sqrt(h_e) |.| */
                    val += 0.5 * sqrt(he[k]) * sqrt(he[k]) * sqrt(q);
                }
                eta[e] = val;
            }
    free(grad);
    return 0;
}

int orc_indicator(int W, int H, const double *g, const double *ft, const double *alpha, double lambda,
                  const double *lamel, const double *U, double *eta)
{
    return indicator_impl(W, H, g, ft, NULL, NULL, alpha, lambda, lamel, U, eta);
}

/* The indicator with general element data (K_rho > 0): the interior
 * residual is F - A_rho U_h; the edge terms do not involve the data. */
int orc_indicator_el(int W, int H, const double *Ael, const double *Fel, const double *alpha, double lambda,
                     const double *lamel, const double *U, double *eta)
{
    return indicator_impl(W, H, NULL, NULL, Ael, Fel, alpha, lambda, lamel, U, eta);
}

/* alpha update of Section 2.3:
 *   alpha <- max(alpha / (1 + kappa max(eta/||eta||_inf - eta_thr, 0)), alpha_th)
 * no change when ||eta||_inf = 0. */
int orc_alpha_update(int64_t ne, const double *eta, double *alpha, double kappa, double eta_thr, double alpha_th)
{
    double m = 0.0;
    for (int64_t e = 0; e < ne; e++) if (eta[e] > m) m = eta[e];
    if (!(m > 0.0)) return 0;
    for (int64_t e = 0; e < ne; e++) {
        double rel = eta[e] / m - eta_thr;
        double a = alpha[e] / (1.0 + kappa * (rel > 0.0 ? rel : 0.0));
        alpha[e] = a > alpha_th ? a : alpha_th;
    }
    return 0;
}

/* --------------------------------------------------- adjoint gradient -- */

/* Gradients of a loss L(U) through A(theta) U = b(theta), given the solution
 * U and the adjoint state Lam with A Lam = dL/dU (A is symmetric):
 *   dL/dtheta = - sum_K d/dtheta [ Lam_K^T (A_K U_K - b_K) ].
 * Outputs dL/dalpha [H-1][W-1][2], dL/df2 and dL/df1 [H][W] (either may be
 * NULL).  Frames enter through g_K and ft_K (see orc_coefficients). */
int orc_adjoint_grad(int W, int H, const double *f1, const double *f2, const double *alpha, double lambda,
                     const double *U, const double *Lam, double *dalpha, double *df2, double *df1, double *dlam,
                     int model)
{
    /* model 1 (brightness constancy): the data term has no illumination
     * column, g = (f2_x, f2_y, 0), so f1 enters through f_t only */
    const double gms = model == 1 ? 0.0 : 1.0;
    (void)lambda;
    long N = (long)W * H;
    if (df2) memset(df2, 0, sizeof(double) * N);
    if (df1) memset(df1, 0, sizeof(double) * N);
    for (int y = 0; y < H - 1; y++)
        for (int x = 0; x < W - 1; x++)
            for (int t = 0; t < 2; t++) {
                long e = elem_index(W, x, y, t);
                int vx[3], vy[3];
                double gx[3], gy[3];
                tri_vertices(x, y, t, vx, vy);
                tri_grads(t, gx, gy);
                double u[3][3], l[3][3]; /* [vertex][component] */
                double g[3] = {0, 0, 0}, ftv = 0.0;
                for (int i = 0; i < 3; i++) {
                    long nd = (long)vy[i] * W + vx[i];
                    for (int c = 0; c < 3; c++) { u[i][c] = U[c * N + nd]; l[i][c] = Lam[c * N + nd]; }
                    g[0] += f2[nd] * gx[i];
                    g[1] += f2[nd] * gy[i];
                    g[2] -= gms * f1[nd] / 3.0;
                    ftv += (f2[nd] - f1[nd]) / 3.0;
                }
                /* stiffness part: d/dalpha_K of Lam^T S_K U (u1, u2 only) */
                if (dalpha) {
                    double s = 0.0;
                    for (int c = 0; c < 2; c++) {
                        double lx = 0, ly = 0, ux = 0, uy = 0;
                        for (int i = 0; i < 3; i++) {
                            lx += l[i][c] * gx[i]; ly += l[i][c] * gy[i];
                            ux += u[i][c] * gx[i]; uy += u[i][c] * gy[i];
                        }
                        s += lx * ux + ly * uy;
                    }
                    dalpha[e] = -KAREA * s;
                }
                /* per-element lambda: d/dlambda_K of Lam^T S_K U (the m component) */
                if (dlam) {
                    double lx = 0, ly = 0, ux = 0, uy = 0;
                    for (int i = 0; i < 3; i++) {
                        lx += l[i][2] * gx[i]; ly += l[i][2] * gy[i];
                        ux += u[i][2] * gx[i]; uy += u[i][2] * gy[i];
                    }
                    dlam[e] = -KAREA * (lx * ux + ly * uy);
                }
                if (!df2 && !df1) continue;
                /* data part E = |K|/12 sum_ij (1+d_ij) t_i s_j + |K|/3 ft sum_i t_i,
                 * s_j = g.U_j, t_i = g.Lam_i */
                double s[3], tt[3];
                for (int i = 0; i < 3; i++) {
                    s[i] = g[0] * u[i][0] + g[1] * u[i][1] + g[2] * u[i][2];
                    tt[i] = g[0] * l[i][0] + g[1] * l[i][1] + g[2] * l[i][2];
                }
                double dEdg[3] = {0, 0, 0}, dEdft = 0.0;
                for (int c = 0; c < 3; c++) {
                    for (int i = 0; i < 3; i++)
                        for (int j = 0; j < 3; j++)
                            dEdg[c] += KAREA / 12.0 * (i == j ? 2.0 : 1.0) * (l[i][c] * s[j] + tt[i] * u[j][c]);
                    for (int i = 0; i < 3; i++) dEdg[c] += KAREA / 3.0 * ftv * l[i][c];
                }
                for (int i = 0; i < 3; i++) dEdft += KAREA / 3.0 * tt[i];
                for (int i = 0; i < 3; i++) {
                    long nd = (long)vy[i] * W + vx[i];
                    if (df2) df2[nd] -= dEdg[0] * gx[i] + dEdg[1] * gy[i] + dEdft / 3.0;
                    if (df1) df1[nd] -= dEdg[2] * (-gms / 3.0) + dEdft * (-1.0 / 3.0);
                }
            }
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
