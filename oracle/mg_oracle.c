/*
 * mg_oracle.c -- plain, slow FP64 CPU statement of the diagonally oriented
 * multigrid V-cycle for Poisson's equation (A.J. Roberts, "Fast and accurate
 * multigrid solution of Poisson's equation using diagonally oriented grids")
 * and of the conventional 2^-l V-cycle the paper compares it with.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Conventions (every function):
 *   - A grid of side n has n interior points per axis and is stored as a full
 *     (n+2)^dim array including the Dirichlet ring, x fastest:
 *     2D index (i,j) -> j*(n+2)+i,  3D (i,j,k) -> (k*(n+2)+j)*(n+2)+i.
 *   - Every level of one 2D pair (green, red) or one 3D triple (green, red,
 *     magenta) is stored on that pair's/triple's green grid and indexed with
 *     the green grid's subscripts, as the paper does in Sections 2 and 3.
 *     A level only owns the points of its lattice; the other entries are not
 *     read.  The coarser blue grid of side (n-1)/2 is the next green grid;
 *     its point (a,b[,c]) is the green point (2a,2b[,2c]).
 *   - Stage functions write exactly the interior points of their output
 *     level and leave every other entry (ring included) as the caller set it.
 *     Inputs are read on the ring where a stencil reaches it; the V-cycle
 *     keeps rings at zero (homogeneous Dirichlet data).
 *   - Floating-point expressions are written in the order of the paper's
 *     formulas; the library is built without FMA contraction.
 *   - Threads.  In an OpenMP build the loops over the points of a stage (each
 *     point computed from inputs the loop does not write) are split across
 *     threads; sums (norms) and the coarsest solve stay serial, so the
 *     results do not depend on the thread count.  One thread by default
 *     (orc_set_threads).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX2(n, i, j) ((size_t)(j) * (size_t)((n) + 2) + (size_t)(i))
#define IDX3(n, i, j, k) \
    (((size_t)(k) * (size_t)((n) + 2) + (size_t)(j)) * (size_t)((n) + 2) + (size_t)(i))

enum { ORC_DIAG = 0, ORC_USUAL = 1 };

#define ORC_PAR _Pragma("omp parallel for schedule(static)")

/* threads of the per-point loops (OpenMP builds; ignored otherwise); returns
 * the count in effect */
int orc_set_threads(int t)
{
#ifdef _OPENMP
    omp_set_num_threads(t > 0 ? t : 1);
    return omp_get_max_threads();
#else
    (void)t;
    return 1;
#endif
}

static size_t grid_len(int dim, int n)
{
    size_t s = (size_t)(n + 2);
    return dim == 2 ? s * s : s * s * s;
}

/* n = 2^m - 1 with m >= 1; returns m or -1 */
static int log2_side(int n)
{
    int m = 0;
    long v = (long)n + 1;
    if (n < 1) return -1;
    while ((v & 1) == 0) { v >>= 1; m++; }
    return v == 1 ? m : -1;
}

/* ------------------------------------------------------------------------ */
/* Residuals (Eq. Evpois with the 5/7-point Laplacian; Eq. Efos2, Eq. Efos4) */
/* ------------------------------------------------------------------------ */

/* 2D: order 2: r = f - (u_E + u_W + u_N + u_S - 4u)/h^2            (Eq. Evpois)
 *     order 4: r = (8f + sum4 f)/12
 *                  - [-20u + 4 sum4axis u + sum4diag u]/(6h^2)     (Eq. Efos2) */
void orc_residual2d(int n, double h, int order, const double *f, const double *u, double *r)
{
    ORC_PAR
    for (int j = 1; j <= n; j++)
        for (int i = 1; i <= n; i++) {
            double res;
            if (order == 2) {
                double lap = (u[IDX2(n, i + 1, j)] + u[IDX2(n, i - 1, j)] + u[IDX2(n, i, j + 1)] +
                              u[IDX2(n, i, j - 1)] - 4.0 * u[IDX2(n, i, j)]) / (h * h);
                res = f[IDX2(n, i, j)] - lap;
            } else {
                double ft = (8.0 * f[IDX2(n, i, j)] + f[IDX2(n, i + 1, j)] + f[IDX2(n, i, j + 1)] +
                             f[IDX2(n, i - 1, j)] + f[IDX2(n, i, j - 1)]) / 12.0;
                double axis = u[IDX2(n, i, j - 1)] + u[IDX2(n, i, j + 1)] + u[IDX2(n, i - 1, j)] +
                              u[IDX2(n, i + 1, j)];
                double diag = u[IDX2(n, i + 1, j + 1)] + u[IDX2(n, i - 1, j + 1)] +
                              u[IDX2(n, i - 1, j - 1)] + u[IDX2(n, i + 1, j - 1)];
                res = ft - (-20.0 * u[IDX2(n, i, j)] + 4.0 * axis + diag) / (6.0 * h * h);
            }
            r[IDX2(n, i, j)] = res;
        }
}

/* 3D: order 2: r = f - (sum6 u - 6u)/h^2
 *     order 4: r = (6f + sum6 f)/12 - [-24u + 2 sum6 u + sum12 u]/(6h^2)  (Eq. Efos4) */
void orc_residual3d(int n, double h, int order, const double *f, const double *u, double *r)
{
    ORC_PAR
    for (int k = 1; k <= n; k++)
        for (int j = 1; j <= n; j++)
            for (int i = 1; i <= n; i++) {
                double c = u[IDX3(n, i, j, k)];
                double axis = u[IDX3(n, i + 1, j, k)] + u[IDX3(n, i - 1, j, k)] +
                              u[IDX3(n, i, j + 1, k)] + u[IDX3(n, i, j - 1, k)] +
                              u[IDX3(n, i, j, k + 1)] + u[IDX3(n, i, j, k - 1)];
                double res;
                if (order == 2) {
                    res = f[IDX3(n, i, j, k)] - (axis - 6.0 * c) / (h * h);
                } else {
                    double ft = (6.0 * f[IDX3(n, i, j, k)] + f[IDX3(n, i + 1, j, k)] +
                                 f[IDX3(n, i, j + 1, k)] + f[IDX3(n, i - 1, j, k)] +
                                 f[IDX3(n, i, j - 1, k)] + f[IDX3(n, i, j, k + 1)] +
                                 f[IDX3(n, i, j, k - 1)]) / 12.0;
                    double edge = u[IDX3(n, i + 1, j + 1, k)] + u[IDX3(n, i - 1, j + 1, k)] +
                                  u[IDX3(n, i - 1, j - 1, k)] + u[IDX3(n, i + 1, j - 1, k)] +
                                  u[IDX3(n, i, j + 1, k + 1)] + u[IDX3(n, i, j + 1, k - 1)] +
                                  u[IDX3(n, i, j - 1, k - 1)] + u[IDX3(n, i, j - 1, k + 1)] +
                                  u[IDX3(n, i + 1, j, k + 1)] + u[IDX3(n, i - 1, j, k + 1)] +
                                  u[IDX3(n, i - 1, j, k - 1)] + u[IDX3(n, i + 1, j, k - 1)];
                    res = ft - (-24.0 * c + 2.0 * axis + edge) / (6.0 * h * h);
                }
                r[IDX3(n, i, j, k)] = res;
            }
}

void orc_residual(int dim, int n, double h, int order, const double *f, const double *u, double *r)
{
    if (dim == 2) orc_residual2d(n, h, order, f, u, r);
    else orc_residual3d(n, h, order, f, u, r);
}

/* ------------------------------------------------------------------------ */
/* 2D diagonal hierarchy (Section 2)                                         */
/* ------------------------------------------------------------------------ */

/* green -> red, Eq. Erest2r: at i+j even, r' = (4r + 4 axis neighbours)/8 */
void orc_restrict2d_g2r(int n, const double *rg, double *rr)
{
    ORC_PAR
    for (int j = 1; j <= n; j++)
        for (int i = 1; i <= n; i++) {
            if ((i + j) % 2 != 0) continue;
            rr[IDX2(n, i, j)] = (4.0 * rg[IDX2(n, i, j)] + rg[IDX2(n, i - 1, j)] +
                                 rg[IDX2(n, i, j - 1)] + rg[IDX2(n, i + 1, j)] +
                                 rg[IDX2(n, i, j + 1)]) / 8.0;
        }
}

/* red -> blue, Eq. Erest2b: at i,j even, r' = (4r + 4 diagonal neighbours)/8.
 * rb is the blue grid of side (n-1)/2. */
void orc_restrict2d_r2b(int n, const double *rr, double *rb)
{
    int nb = (n - 1) / 2;
    ORC_PAR
    for (int b = 1; b <= nb; b++)
        for (int a = 1; a <= nb; a++) {
            int i = 2 * a, j = 2 * b;
            rb[IDX2(nb, a, b)] = (4.0 * rr[IDX2(n, i, j)] + rr[IDX2(n, i - 1, j - 1)] +
                                  rr[IDX2(n, i + 1, j - 1)] + rr[IDX2(n, i + 1, j + 1)] +
                                  rr[IDX2(n, i - 1, j + 1)]) / 8.0;
        }
}

/* blue -> red Jacobi prolongation, Eq. Eajacr then Eq. Eajacb (p = 1 gives
 * Eq. Ejacr, Ejacb).  h is the green spacing of the pair, so the red spacing
 * is sqrt(2) h.  First the red points that are not blue (i,j odd) from the
 * four diagonal blue values, then the blue points (i,j even) from the four new
 * red values; the coarse values at the blue points are replaced. */
void orc_prolong2d_b2r(int n, double h, double p, const double *vb, const double *rr, double *vr)
{
    int nb = (n - 1) / 2;
    ORC_PAR
    for (int j = 1; j <= n; j += 2)
        for (int i = 1; i <= n; i += 2) {
            /* diagonal neighbours (i+-1, j+-1) are blue points ((i+-1)/2, (j+-1)/2) */
            double s = vb[IDX2(nb, (i - 1) / 2, (j - 1) / 2)] + vb[IDX2(nb, (i + 1) / 2, (j - 1) / 2)] +
                       vb[IDX2(nb, (i + 1) / 2, (j + 1) / 2)] + vb[IDX2(nb, (i - 1) / 2, (j + 1) / 2)];
            vr[IDX2(n, i, j)] = (-2.0 * p * h * h * rr[IDX2(n, i, j)] + s) / 4.0;
        }
    ORC_PAR
    for (int j = 2; j <= n; j += 2)
        for (int i = 2; i <= n; i += 2) {
            double s = vr[IDX2(n, i - 1, j - 1)] + vr[IDX2(n, i + 1, j - 1)] +
                       vr[IDX2(n, i + 1, j + 1)] + vr[IDX2(n, i - 1, j + 1)];
            vr[IDX2(n, i, j)] = (-2.0 * p * h * h * rr[IDX2(n, i, j)] + s) / 4.0;
        }
}

/* red -> green Jacobi prolongation ("similarly for a green grid", Section 2.3):
 * green-only points (i+j odd) from the four axis red values, then the red
 * points (i+j even) from the four new green values; spacing h. */
void orc_prolong2d_r2g(int n, double h, double p, const double *vr, const double *rg, double *vg)
{
    ORC_PAR
    for (int j = 1; j <= n; j++)
        for (int i = 1; i <= n; i++) {
            if ((i + j) % 2 == 0) continue;
            double s = vr[IDX2(n, i - 1, j)] + vr[IDX2(n, i + 1, j)] + vr[IDX2(n, i, j - 1)] +
                       vr[IDX2(n, i, j + 1)];
            vg[IDX2(n, i, j)] = (-p * h * h * rg[IDX2(n, i, j)] + s) / 4.0;
        }
    ORC_PAR
    for (int j = 1; j <= n; j++)
        for (int i = 1; i <= n; i++) {
            if ((i + j) % 2 != 0) continue;
            double s = vg[IDX2(n, i - 1, j)] + vg[IDX2(n, i + 1, j)] + vg[IDX2(n, i, j - 1)] +
                       vg[IDX2(n, i, j + 1)];
            vg[IDX2(n, i, j)] = (-p * h * h * rg[IDX2(n, i, j)] + s) / 4.0;
        }
}

/* Extra Jacobi sweeps at each level of the 2D diagonal hierarchy, the
 * extension Section 5 leaves open.  One extra sweep repeats the level's two
 * half-sweeps with the level's own current values in place of the coarse
 * ones: on a red level the points that are not blue (i,j odd) from their four
 * diagonal neighbours, then the blue points (i,j even) from theirs, both with
 * 2 p h^2; on a green level the green-only points (i+j odd) from their four
 * axis neighbours, then the red points (i+j even), both with p h^2. */
void orc_sweep2d_red(int n, double h, double p, const double *rr, double *vr)
{
    for (int par = 1; par >= 0; par--)
        ORC_PAR
        for (int j = 2 - par; j <= n; j += 2)
            for (int i = 2 - par; i <= n; i += 2) {
                double s = vr[IDX2(n, i - 1, j - 1)] + vr[IDX2(n, i + 1, j - 1)] +
                           vr[IDX2(n, i + 1, j + 1)] + vr[IDX2(n, i - 1, j + 1)];
                vr[IDX2(n, i, j)] = (-2.0 * p * h * h * rr[IDX2(n, i, j)] + s) / 4.0;
            }
}

void orc_sweep2d_green(int n, double h, double p, const double *rg, double *vg)
{
    for (int par = 1; par >= 0; par--)
        ORC_PAR
        for (int j = 1; j <= n; j++)
            for (int i = 1; i <= n; i++) {
                if ((i + j) % 2 != par) continue;
                double s = vg[IDX2(n, i - 1, j)] + vg[IDX2(n, i + 1, j)] + vg[IDX2(n, i, j - 1)] +
                           vg[IDX2(n, i, j + 1)];
                vg[IDX2(n, i, j)] = (-p * h * h * rg[IDX2(n, i, j)] + s) / 4.0;
            }
}

/* ------------------------------------------------------------------------ */
/* 3D diagonal hierarchy (Section 3): green (cubic) -> red (i+j+k even) ->   */
/* magenta (corners (e,e,e) and centres (o,o,o)) -> blue (e,e,e)             */
/* ------------------------------------------------------------------------ */

static int is_even(int x) { return (x % 2) == 0; }

/* green -> red, Eq. Erred: at i+j+k even, r' = (6r + 6 axis neighbours)/12 */
void orc_restrict3d_g2r(int n, const double *rg, double *rr)
{
    ORC_PAR
    for (int k = 1; k <= n; k++)
        for (int j = 1; j <= n; j++)
            for (int i = 1; i <= n; i++) {
                if ((i + j + k) % 2 != 0) continue;
                rr[IDX3(n, i, j, k)] =
                    (6.0 * rg[IDX3(n, i, j, k)] + rg[IDX3(n, i + 1, j, k)] + rg[IDX3(n, i - 1, j, k)] +
                     rg[IDX3(n, i, j + 1, k)] + rg[IDX3(n, i, j - 1, k)] + rg[IDX3(n, i, j, k + 1)] +
                     rg[IDX3(n, i, j, k - 1)]) / 12.0;
            }
}

/* red -> magenta: corners (e,e,e), Eq. Ermagc: (12r + 12 FCC neighbours)/24;
 * centres (o,o,o), Eq. Ermagm: mean of the 6 axis (face-centre) red values. */
void orc_restrict3d_r2m(int n, const double *rr, double *rm)
{
    ORC_PAR
    for (int k = 1; k <= n; k++)
        for (int j = 1; j <= n; j++)
            for (int i = 1; i <= n; i++) {
                if (is_even(i) && is_even(j) && is_even(k)) {
                    rm[IDX3(n, i, j, k)] =
                        (12.0 * rr[IDX3(n, i, j, k)] + rr[IDX3(n, i + 1, j + 1, k)] +
                         rr[IDX3(n, i + 1, j - 1, k)] + rr[IDX3(n, i - 1, j - 1, k)] +
                         rr[IDX3(n, i - 1, j + 1, k)] + rr[IDX3(n, i + 1, j, k + 1)] +
                         rr[IDX3(n, i + 1, j, k - 1)] + rr[IDX3(n, i - 1, j, k - 1)] +
                         rr[IDX3(n, i - 1, j, k + 1)] + rr[IDX3(n, i, j + 1, k + 1)] +
                         rr[IDX3(n, i, j + 1, k - 1)] + rr[IDX3(n, i, j - 1, k - 1)] +
                         rr[IDX3(n, i, j - 1, k + 1)]) / 24.0;
                } else if (!is_even(i) && !is_even(j) && !is_even(k)) {
                    rm[IDX3(n, i, j, k)] =
                        (rr[IDX3(n, i + 1, j, k)] + rr[IDX3(n, i - 1, j, k)] + rr[IDX3(n, i, j + 1, k)] +
                         rr[IDX3(n, i, j - 1, k)] + rr[IDX3(n, i, j, k + 1)] + rr[IDX3(n, i, j, k - 1)]) / 6.0;
                }
            }
}

/* magenta -> blue, Eq. Erblu: at (e,e,e), (8r + 8 centre neighbours)/16.
 * rb is the blue grid of side (n-1)/2. */
void orc_restrict3d_m2b(int n, const double *rm, double *rb)
{
    int nb = (n - 1) / 2;
    ORC_PAR
    for (int c = 1; c <= nb; c++)
        for (int b = 1; b <= nb; b++)
            for (int a = 1; a <= nb; a++) {
                int i = 2 * a, j = 2 * b, k = 2 * c;
                rb[IDX3(nb, a, b, c)] =
                    (8.0 * rm[IDX3(n, i, j, k)] + rm[IDX3(n, i + 1, j + 1, k + 1)] +
                     rm[IDX3(n, i + 1, j + 1, k - 1)] + rm[IDX3(n, i + 1, j - 1, k + 1)] +
                     rm[IDX3(n, i + 1, j - 1, k - 1)] + rm[IDX3(n, i - 1, j + 1, k + 1)] +
                     rm[IDX3(n, i - 1, j + 1, k - 1)] + rm[IDX3(n, i - 1, j - 1, k + 1)] +
                     rm[IDX3(n, i - 1, j - 1, k - 1)]) / 16.0;
            }
}

/* blue -> magenta Jacobi, Eq. Emprolm (centres (o,o,o) from the 8 blue
 * corners) then Eq. Emprolb (blue corners (e,e,e) from the 8 new centres). */
void orc_prolong3d_b2m(int n, double h, double pm, const double *vb, const double *rm, double *vm)
{
    int nb = (n - 1) / 2;
    ORC_PAR
    for (int k = 1; k <= n; k += 2)
        for (int j = 1; j <= n; j += 2)
            for (int i = 1; i <= n; i += 2) {
                int a0 = (i - 1) / 2, a1 = (i + 1) / 2;
                int b0 = (j - 1) / 2, b1 = (j + 1) / 2;
                int c0 = (k - 1) / 2, c1 = (k + 1) / 2;
                double s = vb[IDX3(nb, a1, b1, c1)] + vb[IDX3(nb, a1, b1, c0)] + vb[IDX3(nb, a1, b0, c1)] +
                           vb[IDX3(nb, a1, b0, c0)] + vb[IDX3(nb, a0, b1, c1)] + vb[IDX3(nb, a0, b1, c0)] +
                           vb[IDX3(nb, a0, b0, c1)] + vb[IDX3(nb, a0, b0, c0)];
                vm[IDX3(n, i, j, k)] = (-4.0 * pm * h * h * rm[IDX3(n, i, j, k)] + s) / 8.0;
            }
    ORC_PAR
    for (int k = 2; k <= n; k += 2)
        for (int j = 2; j <= n; j += 2)
            for (int i = 2; i <= n; i += 2) {
                double s = vm[IDX3(n, i + 1, j + 1, k + 1)] + vm[IDX3(n, i + 1, j + 1, k - 1)] +
                           vm[IDX3(n, i + 1, j - 1, k + 1)] + vm[IDX3(n, i + 1, j - 1, k - 1)] +
                           vm[IDX3(n, i - 1, j + 1, k + 1)] + vm[IDX3(n, i - 1, j + 1, k - 1)] +
                           vm[IDX3(n, i - 1, j - 1, k + 1)] + vm[IDX3(n, i - 1, j - 1, k - 1)];
                vm[IDX3(n, i, j, k)] = (-4.0 * pm * h * h * rm[IDX3(n, i, j, k)] + s) / 8.0;
            }
}

/* magenta -> red Jacobi.  Red face centres (exactly one even index, the face
 * normal), Eq. Erprolr with its cyclic permutations: the two magenta centres
 * along the normal carry weight 2, the four in-plane diagonal magenta corners
 * weight 1.  Then the magenta corners (e,e,e), Eq. Erprolm, from the 12 new
 * face-centre values.  Magenta centres are not red points and are not written. */
void orc_prolong3d_m2r(int n, double h, double pr1, double pr2, const double *vm, const double *rr,
                       double *vr)
{
    ORC_PAR
    for (int k = 1; k <= n; k++)
        for (int j = 1; j <= n; j++)
            for (int i = 1; i <= n; i++) {
                int ei = is_even(i), ej = is_even(j), ek = is_even(k);
                if (ei + ej + ek != 1) continue;
                double centres, corners;
                if (ek) { /* face normal to z: (o,o,e) */
                    centres = vm[IDX3(n, i, j, k + 1)] + vm[IDX3(n, i, j, k - 1)];
                    corners = vm[IDX3(n, i + 1, j + 1, k)] + vm[IDX3(n, i + 1, j - 1, k)] +
                              vm[IDX3(n, i - 1, j - 1, k)] + vm[IDX3(n, i - 1, j + 1, k)];
                } else if (ei) { /* face normal to x: (e,o,o) */
                    centres = vm[IDX3(n, i + 1, j, k)] + vm[IDX3(n, i - 1, j, k)];
                    corners = vm[IDX3(n, i, j + 1, k + 1)] + vm[IDX3(n, i, j + 1, k - 1)] +
                              vm[IDX3(n, i, j - 1, k - 1)] + vm[IDX3(n, i, j - 1, k + 1)];
                } else { /* face normal to y: (o,e,o) */
                    centres = vm[IDX3(n, i, j + 1, k)] + vm[IDX3(n, i, j - 1, k)];
                    corners = vm[IDX3(n, i + 1, j, k + 1)] + vm[IDX3(n, i - 1, j, k + 1)] +
                              vm[IDX3(n, i - 1, j, k - 1)] + vm[IDX3(n, i + 1, j, k - 1)];
                }
                vr[IDX3(n, i, j, k)] =
                    (-2.0 * pr1 * h * h * rr[IDX3(n, i, j, k)] + 2.0 * centres + corners) / 8.0;
            }
    ORC_PAR
    for (int k = 2; k <= n; k += 2)
        for (int j = 2; j <= n; j += 2)
            for (int i = 2; i <= n; i += 2) {
                double s = vr[IDX3(n, i + 1, j + 1, k)] + vr[IDX3(n, i + 1, j - 1, k)] +
                           vr[IDX3(n, i - 1, j - 1, k)] + vr[IDX3(n, i - 1, j + 1, k)] +
                           vr[IDX3(n, i + 1, j, k + 1)] + vr[IDX3(n, i + 1, j, k - 1)] +
                           vr[IDX3(n, i - 1, j, k - 1)] + vr[IDX3(n, i - 1, j, k + 1)] +
                           vr[IDX3(n, i, j + 1, k + 1)] + vr[IDX3(n, i, j + 1, k - 1)] +
                           vr[IDX3(n, i, j - 1, k - 1)] + vr[IDX3(n, i, j - 1, k + 1)];
                vr[IDX3(n, i, j, k)] = (-4.0 * pr2 * h * h * rr[IDX3(n, i, j, k)] + s) / 12.0;
            }
}

/* red -> green Jacobi, Eq. Egprolg (green-only points, i+j+k odd, from the six
 * axis red values) then Eq. Egprolr (red points from the six new green values). */
void orc_prolong3d_r2g(int n, double h, double pg, const double *vr, const double *rg, double *vg)
{
    for (int pass = 0; pass < 2; pass++) {
        const double *src = pass == 0 ? vr : vg;
        ORC_PAR
        for (int k = 1; k <= n; k++)
            for (int j = 1; j <= n; j++)
                for (int i = 1; i <= n; i++) {
                    if ((i + j + k) % 2 != (pass == 0 ? 1 : 0)) continue;
                    double s = src[IDX3(n, i + 1, j, k)] + src[IDX3(n, i - 1, j, k)] +
                               src[IDX3(n, i, j + 1, k)] + src[IDX3(n, i, j - 1, k)] +
                               src[IDX3(n, i, j, k + 1)] + src[IDX3(n, i, j, k - 1)];
                    vg[IDX3(n, i, j, k)] = (-pg * h * h * rg[IDX3(n, i, j, k)] + s) / 6.0;
                }
    }
}

/* ------------------------------------------------------------------------ */
/* Conventional 2^-l hierarchy (Sections 2.1, 2.2, 3.1, 3.2)                 */
/* ------------------------------------------------------------------------ */

/* full weighting: 2D (1/16)[1 2 1] x [1 2 1], 3D (1/64)[1 2 1]^3.
 * rf has side n, rc side (n-1)/2. */
void orc_restrict_fw(int dim, int n, const double *rf, double *rc)
{
    static const double w[3] = {1.0, 2.0, 1.0};
    int nc = (n - 1) / 2;
    if (dim == 2) {
        ORC_PAR
        for (int b = 1; b <= nc; b++)
            for (int a = 1; a <= nc; a++) {
                double s = 0.0;
                for (int dj = -1; dj <= 1; dj++)
                    for (int di = -1; di <= 1; di++)
                        s += w[di + 1] * w[dj + 1] * rf[IDX2(n, 2 * a + di, 2 * b + dj)];
                rc[IDX2(nc, a, b)] = s / 16.0;
            }
    } else {
        ORC_PAR
        for (int c = 1; c <= nc; c++)
            for (int b = 1; b <= nc; b++)
                for (int a = 1; a <= nc; a++) {
                    double s = 0.0;
                    for (int dk = -1; dk <= 1; dk++)
                        for (int dj = -1; dj <= 1; dj++)
                            for (int di = -1; di <= 1; di++)
                                s += w[di + 1] * w[dj + 1] * w[dk + 1] *
                                     rf[IDX3(n, 2 * a + di, 2 * b + dj, 2 * c + dk)];
                    rc[IDX3(nc, a, b, c)] = s / 64.0;
                }
    }
}

/* bilinear / trilinear interpolation of vc (side (n-1)/2, ring included) to
 * the fine grid of side n (interior points only) */
static void interp_usual(int dim, int n, const double *vc, double *vf)
{
    int nc = (n - 1) / 2;
    if (dim == 2) {
        ORC_PAR
        for (int j = 1; j <= n; j++)
            for (int i = 1; i <= n; i++) {
                int a0 = i / 2, a1 = (i + 1) / 2, b0 = j / 2, b1 = (j + 1) / 2;
                vf[IDX2(n, i, j)] = (vc[IDX2(nc, a0, b0)] + vc[IDX2(nc, a1, b0)] +
                                     vc[IDX2(nc, a0, b1)] + vc[IDX2(nc, a1, b1)]) / 4.0;
            }
    } else {
        ORC_PAR
        for (int k = 1; k <= n; k++)
            for (int j = 1; j <= n; j++)
                for (int i = 1; i <= n; i++) {
                    int a0 = i / 2, a1 = (i + 1) / 2, b0 = j / 2, b1 = (j + 1) / 2;
                    int c0 = k / 2, c1 = (k + 1) / 2;
                    vf[IDX3(n, i, j, k)] =
                        (vc[IDX3(nc, a0, b0, c0)] + vc[IDX3(nc, a1, b0, c0)] + vc[IDX3(nc, a0, b1, c0)] +
                         vc[IDX3(nc, a1, b1, c0)] + vc[IDX3(nc, a0, b0, c1)] + vc[IDX3(nc, a1, b0, c1)] +
                         vc[IDX3(nc, a0, b1, c1)] + vc[IDX3(nc, a1, b1, c1)]) / 8.0;
                }
    }
}

/* conventional prolongation: interpolate, then one Jacobi iteration of the
 * residual equation ordered red-black like the paper's own sweeps (nu1 = 0,
 * nu2 = 1, Section 2.2): first the points with odd index sum, then those with
 * even index sum from the new values, each v <- (sum of the 2d axis
 * neighbours - p h^2 r)/(2d).  A simultaneous (unordered) Jacobi sweep leaves
 * the checkerboard error mode undamped and cannot give the convergence
 * factors of Tables 1-3; the red-black order does.  vf: ring as set by the
 * caller (zero in the V-cycle). */
void orc_prolong_usual(int dim, int n, double h, double p, const double *vc, const double *rf, double *vf)
{
    interp_usual(dim, n, vc, vf);
    for (int parity = 1; parity >= 0; parity--) {
        if (dim == 2) {
            ORC_PAR
            for (int j = 1; j <= n; j++)
                for (int i = 1; i <= n; i++) {
                    if ((i + j) % 2 != parity) continue;
                    double s = vf[IDX2(n, i - 1, j)] + vf[IDX2(n, i + 1, j)] + vf[IDX2(n, i, j - 1)] +
                               vf[IDX2(n, i, j + 1)];
                    vf[IDX2(n, i, j)] = (-p * h * h * rf[IDX2(n, i, j)] + s) / 4.0;
                }
        } else {
            ORC_PAR
            for (int k = 1; k <= n; k++)
                for (int j = 1; j <= n; j++)
                    for (int i = 1; i <= n; i++) {
                        if ((i + j + k) % 2 != parity) continue;
                        double s = vf[IDX3(n, i + 1, j, k)] + vf[IDX3(n, i - 1, j, k)] +
                                   vf[IDX3(n, i, j + 1, k)] + vf[IDX3(n, i, j - 1, k)] +
                                   vf[IDX3(n, i, j, k + 1)] + vf[IDX3(n, i, j, k - 1)];
                        vf[IDX3(n, i, j, k)] = (-p * h * h * rf[IDX3(n, i, j, k)] + s) / 6.0;
                    }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Coarsest level: exact solve of the 5/7-point system L_H v = r             */
/* (the paper leaves the coarsest treatment open; this is the exact solve).  */
/* ------------------------------------------------------------------------ */

int orc_coarse_solve(int dim, int n, double H, const double *r, double *v)
{
    int nn = dim == 2 ? n * n : n * n * n;
    double *A = (double *)calloc((size_t)nn * nn, sizeof(double));
    double *b = (double *)malloc((size_t)nn * sizeof(double));
    if (!A || !b) { free(A); free(b); return -1; }
    /* unknown q <-> interior point (i,j[,k]) with q = ((k-1)*n + (j-1))*n + (i-1) */
    for (int q = 0; q < nn; q++) {
        int i = q % n + 1, j = (q / n) % n + 1, k = dim == 3 ? q / (n * n) + 1 : 0;
        int pos[3] = {i, j, k};
        A[(size_t)q * nn + q] = -2.0 * dim / (H * H);
        for (int ax = 0; ax < dim; ax++)
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                int nb[3] = {pos[0], pos[1], pos[2]};
                nb[ax] += sgn;
                if (nb[ax] < 1 || nb[ax] > n) continue; /* Dirichlet ring: v = 0 */
                int qn = (nb[0] - 1) + (nb[1] - 1) * n + (dim == 3 ? (nb[2] - 1) * n * n : 0);
                A[(size_t)q * nn + qn] = 1.0 / (H * H);
            }
        b[q] = dim == 2 ? r[IDX2(n, i, j)] : r[IDX3(n, i, j, k)];
    }
    /* Gaussian elimination with partial pivoting */
    for (int c = 0; c < nn; c++) {
        int piv = c;
        for (int q = c + 1; q < nn; q++)
            if (fabs(A[(size_t)q * nn + c]) > fabs(A[(size_t)piv * nn + c])) piv = q;
        if (piv != c) {
            for (int t = 0; t < nn; t++) {
                double tmp = A[(size_t)c * nn + t];
                A[(size_t)c * nn + t] = A[(size_t)piv * nn + t];
                A[(size_t)piv * nn + t] = tmp;
            }
            double tmp = b[c]; b[c] = b[piv]; b[piv] = tmp;
        }
        for (int q = c + 1; q < nn; q++) {
            double m = A[(size_t)q * nn + c] / A[(size_t)c * nn + c];
            if (m == 0.0) continue;
            for (int t = c; t < nn; t++) A[(size_t)q * nn + t] -= m * A[(size_t)c * nn + t];
            b[q] -= m * b[c];
        }
    }
    for (int c = nn - 1; c >= 0; c--) {
        double s = b[c];
        for (int t = c + 1; t < nn; t++) s -= A[(size_t)c * nn + t] * b[t];
        b[c] = s / A[(size_t)c * nn + c];
    }
    for (int q = 0; q < nn; q++) {
        int i = q % n + 1, j = (q / n) % n + 1, k = dim == 3 ? q / (n * n) + 1 : 0;
        if (dim == 2) v[IDX2(n, i, j)] = b[q];
        else v[IDX3(n, i, j, k)] = b[q];
    }
    free(A);
    free(b);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One V-cycle: u <- u + v with v the multigrid estimate of L^-1 r           */
/* ------------------------------------------------------------------------ */

/* omega: 2D diag {p}; 3D diag {p_m, p_r1, p_r2, p_g}; usual {p} (p_g in 3D).
 * coarsest: interior side of the coarsest axis grid (2^c - 1, <= n).
 * extra: extra Jacobi sweeps after each level's prolongation (2D diagonal
 * hierarchy only; 0 is the paper's cycle).
 * Returns 0, or -1 on invalid arguments / allocation failure. */
int orc_vcycle_sweeps(int dim, int n, int hier, int order, int coarsest, const double *omega, int extra,
                      const double *f, double *u)
{
    int m = log2_side(n), c = log2_side(coarsest);
    if ((dim != 2 && dim != 3) || m < 1 || c < 1 || c > m || (order != 2 && order != 4) ||
        (hier != ORC_DIAG && hier != ORC_USUAL) || extra < 0 || (extra > 0 && (dim != 2 || hier != ORC_DIAG)))
        return -1;
    int K = m - c; /* number of pairs (2D diag), triples (3D diag) or coarsenings (usual) */
    double h = 1.0 / (n + 1);
    int nk[64];
    double *rg[64], *vg[64], *rr[64], *vr[64], *rm[64], *vm[64];
    for (int k = 0; k <= K; k++) {
        nk[k] = (1 << (m - k)) - 1;
        size_t len = grid_len(dim, nk[k]);
        rg[k] = (double *)calloc(len, sizeof(double));
        vg[k] = (double *)calloc(len, sizeof(double));
        rr[k] = vr[k] = rm[k] = vm[k] = NULL;
        if (k < K && hier == ORC_DIAG) {
            rr[k] = (double *)calloc(len, sizeof(double));
            vr[k] = (double *)calloc(len, sizeof(double));
            if (dim == 3) {
                rm[k] = (double *)calloc(len, sizeof(double));
                vm[k] = (double *)calloc(len, sizeof(double));
            }
        }
    }
    orc_residual(dim, n, h, order, f, u, rg[0]);
    /* down: restriction of the residual */
    for (int k = 0; k < K; k++) {
        if (hier == ORC_USUAL) orc_restrict_fw(dim, nk[k], rg[k], rg[k + 1]);
        else if (dim == 2) {
            orc_restrict2d_g2r(nk[k], rg[k], rr[k]);
            orc_restrict2d_r2b(nk[k], rr[k], rg[k + 1]);
        } else {
            orc_restrict3d_g2r(nk[k], rg[k], rr[k]);
            orc_restrict3d_r2m(nk[k], rr[k], rm[k]);
            orc_restrict3d_m2b(nk[k], rm[k], rg[k + 1]);
        }
    }
    /* coarsest: exact solve with spacing H = 2^K h */
    int rc = orc_coarse_solve(dim, nk[K], h * (double)(1 << K), rg[K], vg[K]);
    /* up: prolongation by Jacobi sweeps (diag) or interpolation + Jacobi (usual) */
    for (int k = K - 1; k >= 0 && rc == 0; k--) {
        double hk = h * (double)(1 << k);
        if (hier == ORC_USUAL) orc_prolong_usual(dim, nk[k], hk, omega[0], vg[k + 1], rg[k], vg[k]);
        else if (dim == 2) {
            orc_prolong2d_b2r(nk[k], hk, omega[0], vg[k + 1], rr[k], vr[k]);
            for (int e = 0; e < extra; e++) orc_sweep2d_red(nk[k], hk, omega[0], rr[k], vr[k]);
            orc_prolong2d_r2g(nk[k], hk, omega[0], vr[k], rg[k], vg[k]);
            for (int e = 0; e < extra; e++) orc_sweep2d_green(nk[k], hk, omega[0], rg[k], vg[k]);
        } else {
            orc_prolong3d_b2m(nk[k], hk, omega[0], vg[k + 1], rm[k], vm[k]);
            orc_prolong3d_m2r(nk[k], hk, omega[1], omega[2], vm[k], rr[k], vr[k]);
            orc_prolong3d_r2g(nk[k], hk, omega[3], vr[k], rg[k], vg[k]);
        }
    }
    if (rc == 0) {
        if (dim == 2) {
            ORC_PAR
            for (int j = 1; j <= n; j++)
                for (int i = 1; i <= n; i++) u[IDX2(n, i, j)] += vg[0][IDX2(n, i, j)];
        } else {
            ORC_PAR
            for (int k = 1; k <= n; k++)
                for (int j = 1; j <= n; j++)
                    for (int i = 1; i <= n; i++) u[IDX3(n, i, j, k)] += vg[0][IDX3(n, i, j, k)];
        }
    }
    for (int k = 0; k <= K; k++) {
        free(rg[k]); free(vg[k]); free(rr[k]); free(vr[k]); free(rm[k]); free(vm[k]);
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Gamma-cycles (W-cycles for gamma = 2) of the diagonal hierarchy: the      */
/* extension the paper's conclusion (Section 5) leaves open.                 */
/* ------------------------------------------------------------------------ */

/* 5/7-point residual on an axis grid of side n and spacing h: out = r - L v */
static void green_residual(int dim, int n, double h, const double *r, const double *v, double *out)
{
    if (dim == 2) {
        ORC_PAR
        for (int j = 1; j <= n; j++)
            for (int i = 1; i <= n; i++) {
                double lap = (v[IDX2(n, i + 1, j)] + v[IDX2(n, i - 1, j)] + v[IDX2(n, i, j + 1)] +
                              v[IDX2(n, i, j - 1)] - 4.0 * v[IDX2(n, i, j)]) / (h * h);
                out[IDX2(n, i, j)] = r[IDX2(n, i, j)] - lap;
            }
    } else {
        ORC_PAR
        for (int k = 1; k <= n; k++)
            for (int j = 1; j <= n; j++)
                for (int i = 1; i <= n; i++) {
                    double lap = (v[IDX3(n, i + 1, j, k)] + v[IDX3(n, i - 1, j, k)] + v[IDX3(n, i, j + 1, k)] +
                                  v[IDX3(n, i, j - 1, k)] + v[IDX3(n, i, j, k + 1)] + v[IDX3(n, i, j, k - 1)] -
                                  6.0 * v[IDX3(n, i, j, k)]) / (h * h);
                    out[IDX3(n, i, j, k)] = r[IDX3(n, i, j, k)] - lap;
                }
    }
}

/* The correction of pair / triple k (green grid of side nk[k], spacing
 * h 2^k) for the green residual rg, into vg: restriction down to the blue
 * level (2D: Eq. Erest2r, Eq. Erest2b; 3D: Eq. Erred, Eq. Ermagc/Ermagm,
 * Eq. Erblu); on the blue grid -- the next green grid, an axis grid with the
 * 5/7-point Laplacian at spacing h 2^(k+1) -- gamma cycles of pair / triple
 * k+1 from a zero correction, each after the first on the residual of the
 * correction so far (the exact solve when it is the coarsest grid); then the
 * prolongation sweeps (2D: Eq. Eajacr, Eq. Eajacb, the green-red sweep; 3D:
 * Eq. Emprolm .. Eq. Egprolr).  gamma = 1 is the V-cycle of orc_vcycle. */
static int gamma_level(int dim, int k, int K, const int *nk, double h, const double *om, int gamma,
                       const double *rg, double *vg)
{
    const int n = nk[k], nb = nk[k + 1];
    const double hk = h * (double)(1 << k);
    const size_t len = grid_len(dim, n), lb = grid_len(dim, nb);
    double *rr = (double *)calloc(len, sizeof(double)), *vr = (double *)calloc(len, sizeof(double));
    double *rm = dim == 3 ? (double *)calloc(len, sizeof(double)) : NULL;
    double *vm = dim == 3 ? (double *)calloc(len, sizeof(double)) : NULL;
    double *rb = (double *)calloc(lb, sizeof(double)), *vb = (double *)calloc(lb, sizeof(double));
    double *res = (double *)calloc(lb, sizeof(double)), *w = (double *)calloc(lb, sizeof(double));
    int rc = (rr && vr && rb && vb && res && w && (dim == 2 || (rm && vm))) ? 0 : -1;
    if (rc == 0) {
        if (dim == 2) {
            orc_restrict2d_g2r(n, rg, rr);
            orc_restrict2d_r2b(n, rr, rb);
        } else {
            orc_restrict3d_g2r(n, rg, rr);
            orc_restrict3d_r2m(n, rr, rm);
            orc_restrict3d_m2b(n, rm, rb);
        }
        if (k + 1 == K) {
            rc = orc_coarse_solve(dim, nb, 2.0 * hk, rb, vb);
        } else {
            for (int it = 0; it < gamma && rc == 0; it++) {
                if (it == 0) memcpy(res, rb, lb * sizeof(double));
                else green_residual(dim, nb, 2.0 * hk, rb, vb, res);
                memset(w, 0, lb * sizeof(double));
                rc = gamma_level(dim, k + 1, K, nk, h, om, gamma, res, w);
                for (size_t q = 0; q < lb; q++) vb[q] += w[q];  /* w is zero on the ring */
            }
        }
    }
    if (rc == 0) {
        if (dim == 2) {
            orc_prolong2d_b2r(n, hk, om[0], vb, rr, vr);
            orc_prolong2d_r2g(n, hk, om[0], vr, rg, vg);
        } else {
            orc_prolong3d_b2m(n, hk, om[0], vb, rm, vm);
            orc_prolong3d_m2r(n, hk, om[1], om[2], vm, rr, vr);
            orc_prolong3d_r2g(n, hk, om[3], vr, rg, vg);
        }
    }
    free(rr); free(vr); free(rm); free(vm); free(rb); free(vb); free(res); free(w);
    return rc;
}

/* One gamma-cycle of the diagonal hierarchy in place on u (order 2 or 4
 * residual on the finest grid; omega as for orc_vcycle).  Returns 0, or -1
 * on invalid arguments. */
int orc_wcycle(int dim, int n, int order, int coarsest, const double *omega, int gamma, const double *f, double *u)
{
    int m = log2_side(n), c = log2_side(coarsest);
    if ((dim != 2 && dim != 3) || m < 1 || c < 1 || c > m || gamma < 1 || (order != 2 && order != 4)) return -1;
    const int K = m - c;
    const double h = 1.0 / (n + 1);
    int nk[64];
    for (int k = 0; k <= K; k++) nk[k] = (1 << (m - k)) - 1;
    const size_t len = grid_len(dim, n);
    double *r = (double *)calloc(len, sizeof(double)), *v = (double *)calloc(len, sizeof(double));
    int rc = (r && v) ? 0 : -1;
    if (rc == 0) {
        orc_residual(dim, n, h, order, f, u, r);
        if (K == 0) rc = orc_coarse_solve(dim, n, h, r, v);
        else rc = gamma_level(dim, 0, K, nk, h, omega, gamma, r, v);
    }
    if (rc == 0) {
        if (dim == 2) {
            ORC_PAR
            for (int j = 1; j <= n; j++)
                for (int i = 1; i <= n; i++) u[IDX2(n, i, j)] += v[IDX2(n, i, j)];
        } else {
            ORC_PAR
            for (int k = 1; k <= n; k++)
                for (int j = 1; j <= n; j++)
                    for (int i = 1; i <= n; i++) u[IDX3(n, i, j, k)] += v[IDX3(n, i, j, k)];
        }
    }
    free(r);
    free(v);
    return rc;
}

int orc_vcycle(int dim, int n, int hier, int order, int coarsest, const double *omega, const double *f,
               double *u)
{
    return orc_vcycle_sweeps(dim, n, hier, order, coarsest, omega, 0, f, u);
}

/* sum of squares of the interior points of a full grid */
double orc_norm2_interior(int dim, int n, const double *x)
{
    double s = 0.0;
    if (dim == 2) {
        for (int j = 1; j <= n; j++)
            for (int i = 1; i <= n; i++) s += x[IDX2(n, i, j)] * x[IDX2(n, i, j)];
    } else {
        for (int k = 1; k <= n; k++)
            for (int j = 1; j <= n; j++)
                for (int i = 1; i <= n; i++) s += x[IDX3(n, i, j, k)] * x[IDX3(n, i, j, k)];
    }
    return s;
}

/* Repeated V-cycles until ||r||_2 / ||r(u=0)||_2 <= rtol (r the residual of
 * the chosen order, so r(u=0) is f for order 2 and the Mehrstellen right-hand
 * side for order 4) or max_cycles cycles.  history (nullable) receives the
 * relative residual after each cycle.  Returns the number of cycles done, or
 * -1 on invalid arguments. */
int orc_solve_sweeps(int dim, int n, int hier, int order, int coarsest, const double *omega, int extra,
                     const double *f, double *u, double rtol, int max_cycles, double *history, double *relres_out)
{
    size_t len = grid_len(dim, n);
    double h = 1.0 / (n + 1);
    double *r = (double *)calloc(len, sizeof(double));
    double *zero = (double *)calloc(len, sizeof(double));
    if (!r || !zero) { free(r); free(zero); return -1; }
    orc_residual(dim, n, h, order, f, zero, r);
    double fnorm = sqrt(orc_norm2_interior(dim, n, r));
    orc_residual(dim, n, h, order, f, u, r);
    double rel = fnorm > 0.0 ? sqrt(orc_norm2_interior(dim, n, r)) / fnorm : 0.0;
    int it = 0;
    while (rel > rtol && it < max_cycles) {
        if (orc_vcycle_sweeps(dim, n, hier, order, coarsest, omega, extra, f, u) != 0) { it = -1; break; }
        orc_residual(dim, n, h, order, f, u, r);
        rel = fnorm > 0.0 ? sqrt(orc_norm2_interior(dim, n, r)) / fnorm : 0.0;
        if (history) history[it] = rel;
        it++;
    }
    if (relres_out) *relres_out = rel;
    free(r);
    free(zero);
    return it;
}

int orc_solve(int dim, int n, int hier, int order, int coarsest, const double *omega, const double *f,
              double *u, double rtol, int max_cycles, double *history, double *relres_out)
{
    return orc_solve_sweeps(dim, n, hier, order, coarsest, omega, 0, f, u, rtol, max_cycles, history,
                            relres_out);
}
