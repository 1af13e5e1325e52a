/*
 * rt_oracle.c -- plain, slow FP64 CPU oracle for the hot path of the 3D
 * radiative transfer framework of Hauschildt & Baron, "A 3D radiative
 * transfer framework XIII: OpenCL implementation" (2011):
 *
 *   - the characteristics formal solution on a Cartesian voxel slab that is
 *     periodic in x and y (Sect. 2.2, first paragraph), giving the
 *     intensities I, the mean intensity J and the nearest-neighbour Lambda*
 *     (Sect. 2.2; abstract);
 *   - the operator-splitting step for the new J, solved by Jordan (=Jacobi)
 *     iterations (Sect. 2.3);
 *   - the outer iteration "formal solution -> operator splitting" (Sect. 2,
 *     first paragraph) for coherent isotropic scattering,
 *     S = eps B + (1 - eps) J (Sect. 3.1, list item 5).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only users.  The GPU library never
 * links, loads or calls this file, and this file shares no code, header or
 * table with it.
 *
 * The paper states the problem but defers the discretisation to the
 * earlier papers of its series, which are not at hand.  This file therefore
 * DEFINES the discretisation, written straight from its mathematical
 * statement, with no blocking, fusion or reordering:
 *
 *  Grid.  Voxel (i,j,k), i<nx, j<ny, k<nz, centres on the integer lattice
 *   scaled by (dx,dy,dz).  k is the depth index: k=0 is the outer (top)
 *   boundary, k=nz-1 the inner (bottom) one.  Arrays are [nz][ny][nx].
 *   x and y are periodic (node i+nx == node i).
 *
 *  Directions.  d = (mu, phi, w); the propagation vector is
 *   (sin t cos phi, sin t sin phi, mu) with sin t = sqrt(1-mu^2); mu > 0
 *   propagates towards larger k.  J = sum_d w_d I_d.
 *
 *  Characteristic (long characteristic in gather form, one z-plane per
 *   step).  For voxel (i0,j0,k0) the upstream points are
 *     p_m = (i0 - m*ax, j0 - m*ay, k0 - m*s),   m = 0..M,
 *   with s = sign(mu), ax = (dz/dx) sin t cos phi / |mu|,
 *   ay = (dz/dy) sin t sin phi / |mu|, M = k0 for mu > 0 and nz-1-k0 for
 *   mu < 0.  Each step has path length ds = dz/|mu|.
 *
 *  Interpolation.  chi, S and B at p_m are bilinear in the plane k - m*s
 *   with periodic wrap of the four lattice nodes.
 *
 *  Optical depth.  dtau_m = ds (chi(p_m) + chi(p_{m+1})) / 2 (trapezoid).
 *
 *  Source integral.  S linear in tau on each segment.  With x = dtau and
 *   e = exp(-x), the segment from p_{m+1} to p_m contributes
 *     I(p_m) = I(p_{m+1}) e + w_cur S(p_m) + w_up S(p_{m+1}),
 *     w_cur = 1 - (1-e)/x,   w_up = (1-e)/x - e,
 *   i.e. the exact integral of S(t) e^{-t} over the segment for a linear
 *   S(t).  I(p_M) = I_bc: 0 (zero mode), B(p_M) (Planck mode), or at the
 *   inner boundary B(p_M) + |mu| G(p_M) (LTE diffusion mode, Sect. 3.1
 *   item 4: the diffusion approximation I = B + mu dB/dtau), where G is
 *   dB/dtau at each bottom node, (B[nz-1] - B[nz-2]) / (dz (chi[nz-1] +
 *   chi[nz-2]) / 2), interpolated bilinearly like B.
 *
 *  Parabolic source (second-order variant, src_order = 1; the paper names
 *   no order).  On segment m (from p_{m+1} to p_m, optical depth a = dtau_m)
 *   S is the quadratic in t (optical depth measured upstream from p_m)
 *   through (a, S(p_{m+1})), (0, S(p_m)) and (-b, S(p_{m-1})), b = dtau_{m-1}
 *   the optical depth of the next segment downstream.  With the moments
 *   E_n = int_0^a t^n e^{-t} dt and the Lagrange basis of those nodes, the
 *   segment adds  P_up S(p_{m+1}) + P_cur S(p_m) + P_down S(p_{m-1}):
 *     P_up   = (E2 + b E1) / (a (a + b)),
 *     P_cur  = (a b E0 - (b - a) E1 - E2) / (a b),
 *     P_down = (E2 - a E1) / (b (a + b)),
 *   exact for S quadratic in t.  For m = 0 the downstream point p_{-1} =
 *   (i0 + ax, j0 + ay, k0 + s) is used when plane k0 + s exists (b from the
 *   trapezoid rule like every dtau); otherwise segment 0 keeps the linear
 *   weights.  Lambda* then also has entries on plane k0 + s and may have
 *   negative entries.
 *
 *  Short characteristics (the O(1)-per-pair alternative; the paper's own
 *   boundary-started tracking is also O(1) per pair, Sect. 2.2).  Per
 *   direction the planes are taken in the order of propagation; on the plane
 *   where the direction enters, I = I_bc at each node (as above, evaluated at
 *   the node); on every other plane k each node takes the intensity from its
 *   upstream point p = (i - ax, j - ay) on the preceding plane k - s only:
 *     I(i,j,k) = I(p) e + w_cur S(i,j,k) + w_up S(p),
 *     dtau = ds (chi(p) + chi(i,j,k)) / 2,
 *   with I(p), chi(p), S(p) bilinear in that plane (whose intensities are
 *   complete).  Its Lambda* (same definition as below) has, per direction,
 *   the diagonal w_cur and, at the four nodes c of p, b_c (w_up + e w_cur(c)),
 *   w_cur(c) being the weight of c's own segment (0 where c lies on the
 *   entry plane): I(p) depends on S(c) only through c's own last segment.
 *
 *  Lambda*.  I is linear in S.  Lambda_{i,j} = sum_d w_d dI_{i,d}/dS_j with
 *   the boundary intensity excluded; Lambda*_{i,o} = Lambda_{i,wrap(i+o)}
 *   for the 27 offsets o in {-1,0,1}^3 (index o = (oz+1)*9+(oy+1)*3+(ox+1));
 *   entries whose plane k0+oz lies outside the grid are 0.  Stored
 *   [27][nz][ny][nx].
 *
 *  Operator splitting.  With D = diag(1 - eps), the new J solves
 *     (1 - Lambda* D) J_new = J_fs - Lambda* D J_old ,
 *   by Jacobi sweeps started from J_old, stopped when
 *   max_i |J^{n+1}_i - J^n_i| / |J^{n+1}_i| < tol_inner or after max_sweeps.
 *   Gauss-Seidel variant (the paper's host code offers it beside the
 *   Jordan method, Sect. 2.3) in red-black order: voxel (i,j,k) is red if
 *   i+j+k is even, black otherwise.  One sweep first updates every red voxel
 *   from the values at the start of the sweep, then every black voxel from
 *   the new red and the old black values.  Within one colour the updates
 *   are simultaneous (the 27-point stencil couples voxels of equal colour
 *   through its edge offsets and, for odd nx or ny, across the periodic
 *   seam), so the result does not depend on the visiting order.  The
 *   stopping test is the Jacobi one, over all voxels of the sweep.
 *
 *  Outer iteration.  J^0 = B unless given; S = eps B + (1-eps) J; formal
 *   solution -> J_fs (Lambda* on the first pass); operator splitting ->
 *   J_new; delta = max_i |J_new_i - J_i| / |J_new_i|; stop when delta < tol
 *   or after max_iter.
 *
 *  Ng acceleration (the paper leaves it, with the set-up, to host code,
 *   Sect. 2).  Second-order Ng extrapolation of the iterates: with the four
 *   latest iterates x0 (newest) .. x3 and d0 = x0 - x1, d1 = x1 - x2,
 *   d2 = x2 - x3, choose a, b minimising
 *     sum_i w_i (d0 - a (d0 - d1) - b (d0 - d2))_i^2,   w_i = 1 / x0_i^2,
 *   and replace x0 by (1 - a - b) x0 + a x1 + b x2.  In the outer loop it is
 *   applied after every `ng_period`-th iteration once four iterates exist
 *   since the last extrapolation, provided the previous iteration's delta
 *   was at least `ng_min_delta` (extrapolating iterates whose differences
 *   are down at rounding level only amplifies the rounding); delta is then
 *   measured against the extrapolated iterate.
 */

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    int top_bc, bottom_bc;      /* 0: I_bc = 0, 1: I_bc = B at the entry point,
                                   2 (bottom only): LTE diffusion, see below */
    int src_order;              /* 0: linear source, 1: parabolic (long characteristics) */
} orc_grid;

static long vidx(const orc_grid *g, long i, long j, long k)
{
    return (k * g->ny + j) * g->nx + i;
}

static long wrapi(long a, long n)       /* Euclidean modulo */
{
    long r = a % n;
    return r < 0 ? r + n : r;
}

/* Bilinear value of field f in plane k at the (real) lattice position (x,y),
 * with periodic wrap of the nodes. */
static double bilinear(const orc_grid *g, const double *f, long k, double x, double y)
{
    double fx0 = floor(x), fy0 = floor(y);
    double tx = x - fx0, ty = y - fy0;
    long i0 = wrapi((long)fx0, g->nx), i1 = wrapi((long)fx0 + 1, g->nx);
    long j0 = wrapi((long)fy0, g->ny), j1 = wrapi((long)fy0 + 1, g->ny);
    return (1.0 - tx) * (1.0 - ty) * f[vidx(g, i0, j0, k)]
         + tx * (1.0 - ty) * f[vidx(g, i1, j0, k)]
         + (1.0 - tx) * ty * f[vidx(g, i0, j1, k)]
         + tx * ty * f[vidx(g, i1, j1, k)];
}

/* Linear-source segment weights (see header).  For small x the closed form
 * cancels, so the Taylor series of e^{-x} is used:
 *   w_cur = sum_{n>=1} (-1)^{n+1} x^n / (n+1)!
 *   w_up  = sum_{n>=1} (-1)^{n+1} n x^n / (n+1)!
 * below x = 0.1, through x^10 (truncation < 1e-17 relative); above it the
 * closed form loses at most a factor ~20 to cancellation. */
void orc_weights(double x, double *w_cur, double *w_up)
{
    if (x < 0.1) {
        double wc = 0.0, wu = 0.0, xn = 1.0, fact = 1.0;
        for (int n = 1; n <= 10; ++n) {
            xn *= x;
            fact *= (double)(n + 1);
            double sgn = (n % 2) ? 1.0 : -1.0;
            wc += sgn * xn / fact;
            wu += sgn * (double)n * xn / fact;
        }
        *w_cur = wc;
        *w_up = wu;
    } else {
        double one_minus_e = -expm1(-x);
        double e = exp(-x);
        *w_cur = 1.0 - one_minus_e / x;
        *w_up = one_minus_e / x - e;
    }
}

/* Moments E_n = int_0^a t^n e^{-t} dt, n = 0, 1, 2: below a = 1 the
 * series E_n = sum_{k>=0} (-1)^k a^{n+k+1} / (k! (n+k+1)) (40 terms), above
 * it E_0 = 1 - e^{-a}, E_1 = 1 - e^{-a} (1 + a), E_2 = 2 - e^{-a} (a^2 + 2a + 2). */
static void exp_moments(double a, double E[3])
{
    if (a < 1.0) {
        for (int n = 0; n < 3; ++n) {
            double sum = 0.0, ak = 1.0, fact = 1.0;   /* a^k, k! */
            for (int k = 0; k < 40; ++k) {
                if (k > 0) { ak *= a; fact *= (double)k; }
                double sgn = (k % 2) ? -1.0 : 1.0;
                sum += sgn * ak * pow(a, n + 1) / (fact * (double)(n + k + 1));
            }
            E[n] = sum;
        }
    } else {
        double e = exp(-a);
        E[0] = -expm1(-a);
        E[1] = 1.0 - e * (1.0 + a);
        E[2] = 2.0 - e * (a * a + 2.0 * a + 2.0);
    }
}

/* Parabolic segment weights (see header): a the segment's optical depth, b
 * the next downstream segment's. */
void orc_weights_parabolic(double a, double b, double *p_up, double *p_cur, double *p_down)
{
    double E[3];
    exp_moments(a, E);
    *p_up = (E[2] + b * E[1]) / (a * (a + b));
    *p_cur = (a * b * E[0] - (b - a) * E[1] - E[2]) / (a * b);
    *p_down = (E[2] - a * E[1]) / (b * (a + b));
}

/* Geometry of one direction. */
typedef struct {
    int s;          /* +1: propagates to larger k (came from the top); -1 */
    double ax, ay;  /* upstream shift per step, in grid units */
    double ds;      /* path length per step */
} orc_dir;

static orc_dir dir_geometry(const orc_grid *g, double mu, double phi)
{
    orc_dir d;
    double amu = fabs(mu);
    double sint = sqrt(1.0 - mu * mu);
    d.s = mu > 0.0 ? 1 : -1;
    d.ax = (g->dz / g->dx) * sint * cos(phi) / amu;
    d.ay = (g->dz / g->dy) * sint * sin(phi) / amu;
    d.ds = g->dz / amu;
    return d;
}

/* dB/dtau at bottom node (i, j): vertical difference over the trapezoid
 * optical depth between the two deepest planes. */
static double diffusion_gradient(const orc_grid *g, const double *chi, const double *B,
                                 long i, long j)
{
    long a = vidx(g, i, j, g->nz - 1), b = vidx(g, i, j, g->nz - 2);
    return (B[a] - B[b]) / (g->dz * (chi[a] + chi[b]) / 2.0);
}

/* Bilinear value of the bottom-node gradient at (x, y). */
static double diffusion_gradient_at(const orc_grid *g, const double *chi, const double *B,
                                    double x, double y)
{
    double fx0 = floor(x), fy0 = floor(y);
    double tx = x - fx0, ty = y - fy0;
    long i0 = wrapi((long)fx0, g->nx), i1 = wrapi((long)fx0 + 1, g->nx);
    long j0 = wrapi((long)fy0, g->ny), j1 = wrapi((long)fy0 + 1, g->ny);
    return (1.0 - tx) * (1.0 - ty) * diffusion_gradient(g, chi, B, i0, j0)
         + tx * (1.0 - ty) * diffusion_gradient(g, chi, B, i1, j0)
         + (1.0 - tx) * ty * diffusion_gradient(g, chi, B, i0, j1)
         + tx * ty * diffusion_gradient(g, chi, B, i1, j1);
}

/* Incoming intensity at the entry point (xM, yM) of plane kM for boundary
 * mode bc (0: none, 1: B, 2: B + |mu| dB/dtau). */
static double boundary_intensity(const orc_grid *g, const double *chi, const double *B, int bc,
                                 double mu, long kM, double xM, double yM)
{
    double I = bc ? bilinear(g, B, kM, xM, yM) : 0.0;
    if (bc == 2) I += fabs(mu) * diffusion_gradient_at(g, chi, B, xM, yM);
    return I;
}

static int steps_to_boundary(const orc_grid *g, const orc_dir *d, long k0)
{
    return d->s > 0 ? (int)k0 : (int)(g->nz - 1 - k0);
}

/* Intensity at voxel (i0,j0,k0) in direction (mu,phi): textbook
 * back-to-front recursion along the characteristic. */
static double intensity_parabolic(const orc_grid *g, const double *chi, const double *S,
                                  const double *B, double mu, double phi,
                                  long i0, long j0, long k0);

double orc_intensity(const orc_grid *g, const double *chi, const double *S,
                     const double *B, double mu, double phi,
                     long i0, long j0, long k0)
{
    if (g->src_order == 1) return intensity_parabolic(g, chi, S, B, mu, phi, i0, j0, k0);
    orc_dir d = dir_geometry(g, mu, phi);
    int M = steps_to_boundary(g, &d, k0);
    int bc = d.s > 0 ? g->top_bc : g->bottom_bc;
    double xM = (double)i0 - M * d.ax, yM = (double)j0 - M * d.ay;
    long kM = k0 - (long)M * d.s;
    double I = boundary_intensity(g, chi, B, bc, mu, kM, xM, yM);
    for (int m = M - 1; m >= 0; --m) {
        double xa = (double)i0 - m * d.ax, ya = (double)j0 - m * d.ay;
        double xb = (double)i0 - (m + 1) * d.ax, yb = (double)j0 - (m + 1) * d.ay;
        long ka = k0 - (long)m * d.s, kb = k0 - (long)(m + 1) * d.s;
        double chi_a = bilinear(g, chi, ka, xa, ya), chi_b = bilinear(g, chi, kb, xb, yb);
        double S_a = bilinear(g, S, ka, xa, ya), S_b = bilinear(g, S, kb, xb, yb);
        double dtau = d.ds * (chi_a + chi_b) / 2.0;
        double wc, wu;
        orc_weights(dtau, &wc, &wu);
        I = I * exp(-dtau) + wc * S_a + wu * S_b;
    }
    return I;
}

/* Point p_m of the characteristic of voxel (i0, j0, k0) (m = -1 is the
 * downstream point): its plane and lattice position. */
static void char_point(const orc_dir *d, long i0, long j0, long k0, int m, long *k,
                       double *x, double *y)
{
    *x = (double)i0 - m * d->ax;
    *y = (double)j0 - m * d->ay;
    *k = k0 - (long)m * d->s;
}

/* Optical depths dtau_m, m = -1..M-1, of the segments of the characteristic
 * (dtau_{-1} only if plane k0 + s exists; has_down says whether it does). */
static void segment_depths(const orc_grid *g, const double *chi, const orc_dir *d, long i0,
                           long j0, long k0, int M, double *dtau /*[M+1], index m+1*/,
                           int *has_down)
{
    long kd = k0 + d->s;
    *has_down = kd >= 0 && kd < g->nz;
    for (int m = *has_down ? -1 : 0; m < M; ++m) {
        long ka, kb;
        double xa, ya, xb, yb;
        char_point(d, i0, j0, k0, m, &ka, &xa, &ya);
        char_point(d, i0, j0, k0, m + 1, &kb, &xb, &yb);
        dtau[m + 1] = d->ds * (bilinear(g, chi, ka, xa, ya) + bilinear(g, chi, kb, xb, yb)) / 2.0;
    }
}

/* Weights (on S(p_{m+1}), S(p_m), S(p_{m-1})) of segment m under the
 * parabolic source; segment 0 falls back to the linear weights when there
 * is no downstream plane. */
static void parabolic_segment(const double *dtau, int m, int has_down, double *wu, double *wc,
                              double *wd)
{
    if (m == 0 && !has_down) {
        orc_weights(dtau[1], wc, wu);
        *wd = 0.0;
    } else {
        orc_weights_parabolic(dtau[m + 1], dtau[m], wu, wc, wd);
    }
}

/* Intensity under the parabolic source: back-to-front recursion
 * I(p_m) = I(p_{m+1}) e^{-dtau_m} + P_up S(p_{m+1}) + P_cur S(p_m) + P_down S(p_{m-1}). */
static double intensity_parabolic(const orc_grid *g, const double *chi, const double *S,
                                  const double *B, double mu, double phi,
                                  long i0, long j0, long k0)
{
    orc_dir d = dir_geometry(g, mu, phi);
    int M = steps_to_boundary(g, &d, k0);
    int bc = d.s > 0 ? g->top_bc : g->bottom_bc;
    long kM;
    double xM, yM;
    char_point(&d, i0, j0, k0, M, &kM, &xM, &yM);
    double I = boundary_intensity(g, chi, B, bc, mu, kM, xM, yM);
    double *dtau = malloc(sizeof(double) * (M + 1));
    int has_down;
    segment_depths(g, chi, &d, i0, j0, k0, M, dtau, &has_down);
    for (int m = M - 1; m >= 0; --m) {
        double wu, wc, wd, Sm1 = 0.0;
        parabolic_segment(dtau, m, has_down, &wu, &wc, &wd);
        long ka, kb, kc;
        double xa, ya, xb, yb, xc, yc;
        char_point(&d, i0, j0, k0, m, &ka, &xa, &ya);
        char_point(&d, i0, j0, k0, m + 1, &kb, &xb, &yb);
        if (wd != 0.0) {
            char_point(&d, i0, j0, k0, m - 1, &kc, &xc, &yc);
            Sm1 = bilinear(g, S, kc, xc, yc);
        }
        I = I * exp(-dtau[m + 1]) + wu * bilinear(g, S, kb, xb, yb) + wc * bilinear(g, S, ka, xa, ya)
          + wd * Sm1;
    }
    free(dtau);
    return I;
}

/* Offset index of node (a,b,kk) relative to voxel (i0,j0,k0), or -1 if the
 * node is not one of the 27 periodic nearest neighbours. */
static int neighbour_offset(const orc_grid *g, long a, long b, long kk,
                            long i0, long j0, long k0)
{
    long rx = wrapi(a - i0, g->nx), ry = wrapi(b - j0, g->ny), dzv = kk - k0;
    int ox, oy;
    if (rx == 0) ox = 0; else if (rx == 1) ox = 1; else if (rx == g->nx - 1) ox = -1; else return -1;
    if (ry == 0) oy = 0; else if (ry == 1) oy = 1; else if (ry == g->ny - 1) oy = -1; else return -1;
    if (dzv < -1 || dzv > 1) return -1;
    return ((int)dzv + 1) * 9 + (oy + 1) * 3 + (ox + 1);
}

/* Contribution of one (voxel, direction) to Lambda*: the coefficient of
 * S(p_m) in I is c_m = T_m w_cur(m) [m < M] + T_{m-1} w_up(m-1) [m >= 1],
 * T_m = prod_{l<m} exp(-dtau_l); c_m is shared among the four bilinear
 * nodes of p_m and kept where the node is a nearest neighbour. */
static void lstar_one_parabolic(const orc_grid *g, const double *chi, double mu, double phi,
                                double wdir, long i0, long j0, long k0, double *lrow);

static void lstar_one(const orc_grid *g, const double *chi, double mu, double phi,
                      double wd, long i0, long j0, long k0, double *lrow /*[27]*/)
{
    if (g->src_order == 1) {
        lstar_one_parabolic(g, chi, mu, phi, wd, i0, j0, k0, lrow);
        return;
    }
    orc_dir d = dir_geometry(g, mu, phi);
    int M = steps_to_boundary(g, &d, k0);
    if (M == 0) return;
    double *T = malloc(sizeof(double) * (M + 1));
    double *wc = malloc(sizeof(double) * (M + 1));
    double *wu = malloc(sizeof(double) * (M + 1));
    T[0] = 1.0;
    for (int m = 0; m < M; ++m) {
        double xa = (double)i0 - m * d.ax, ya = (double)j0 - m * d.ay;
        double xb = (double)i0 - (m + 1) * d.ax, yb = (double)j0 - (m + 1) * d.ay;
        long ka = k0 - (long)m * d.s, kb = k0 - (long)(m + 1) * d.s;
        double dtau = d.ds * (bilinear(g, chi, ka, xa, ya) + bilinear(g, chi, kb, xb, yb)) / 2.0;
        orc_weights(dtau, &wc[m], &wu[m]);
        T[m + 1] = T[m] * exp(-dtau);
    }
    for (int m = 0; m <= M; ++m) {
        double c = 0.0;
        if (m < M) c += T[m] * wc[m];
        if (m >= 1) c += T[m - 1] * wu[m - 1];
        double x = (double)i0 - m * d.ax, y = (double)j0 - m * d.ay;
        long km = k0 - (long)m * d.s;
        double fx0 = floor(x), fy0 = floor(y);
        double tx = x - fx0, ty = y - fy0;
        long nodes_x[2] = {(long)fx0, (long)fx0 + 1}, nodes_y[2] = {(long)fy0, (long)fy0 + 1};
        double bx[2] = {1.0 - tx, tx}, by[2] = {1.0 - ty, ty};
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                int o = neighbour_offset(g, nodes_x[a], nodes_y[b], km, i0, j0, k0);
                if (o >= 0) lrow[o] += wd * c * bx[a] * by[b];
            }
    }
    free(T); free(wc); free(wu);
}

/* Lambda* under the parabolic source: the coefficient of S(p_j) in I(p_0)
 * is c_j = T_{j-1} P_up(j-1) + T_j P_cur(j) + T_{j+1} P_down(j+1) over the
 * segments that exist (T_m = prod_{l<m} e^{-dtau_l}); j runs from -1 (the
 * downstream point) to M; c_j is shared among the bilinear nodes of p_j and
 * kept where they are nearest neighbours. */
static void lstar_one_parabolic(const orc_grid *g, const double *chi, double mu, double phi,
                                double wdir, long i0, long j0, long k0, double *lrow)
{
    orc_dir d = dir_geometry(g, mu, phi);
    int M = steps_to_boundary(g, &d, k0);
    if (M == 0) return;
    double *dtau = malloc(sizeof(double) * (M + 1));
    double *T = malloc(sizeof(double) * (M + 1));
    double *wu = malloc(sizeof(double) * M), *wc = malloc(sizeof(double) * M);
    double *wdn = malloc(sizeof(double) * M);
    int has_down;
    segment_depths(g, chi, &d, i0, j0, k0, M, dtau, &has_down);
    T[0] = 1.0;
    for (int m = 0; m < M; ++m) {
        parabolic_segment(dtau, m, has_down, &wu[m], &wc[m], &wdn[m]);
        T[m + 1] = T[m] * exp(-dtau[m + 1]);
    }
    for (int j = -1; j <= M; ++j) {
        double c = 0.0;
        if (j >= 1) c += T[j - 1] * wu[j - 1];
        if (j >= 0 && j < M) c += T[j] * wc[j];
        if (j + 1 < M) c += T[j + 1] * wdn[j + 1];
        if (c == 0.0) continue;
        long km;
        double x, y;
        char_point(&d, i0, j0, k0, j, &km, &x, &y);
        double fx0 = floor(x), fy0 = floor(y);
        double tx = x - fx0, ty = y - fy0;
        long nodes_x[2] = {(long)fx0, (long)fx0 + 1}, nodes_y[2] = {(long)fy0, (long)fy0 + 1};
        double bx[2] = {1.0 - tx, tx}, by[2] = {1.0 - ty, ty};
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                int o = neighbour_offset(g, nodes_x[a], nodes_y[b], km, i0, j0, k0);
                if (o >= 0) lrow[o] += wdir * c * bx[a] * by[b];
            }
    }
    free(dtau); free(T); free(wu); free(wc); free(wdn);
}

static int check_grid(const orc_grid *g)
{
    if (!g || g->nx < 3 || g->ny < 3 || g->nz < 2) return ORC_EINVAL;
    if (g->top_bc < 0 || g->top_bc > 1 || g->bottom_bc < 0 || g->bottom_bc > 2) return ORC_EINVAL;
    if (g->src_order < 0 || g->src_order > 1) return ORC_EINVAL;
    if (!(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0)) return ORC_EINVAL;
    return ORC_OK;
}

static int check_dirs(int ndir, const double *mu)
{
    if (ndir < 1) return ORC_EINVAL;
    for (int d = 0; d < ndir; ++d)
        if (!(fabs(mu[d]) > 0.0) || !(fabs(mu[d]) <= 1.0)) return ORC_EINVAL;
    return ORC_OK;
}

/* Formal solution for a given source function S: J_out[N] and, if
 * lstar_out != NULL, Lambda* [27][N].  nthreads <= 0 uses the OpenMP
 * default. */
int orc_formal_solution(const orc_grid *g, const double *chi, const double *S,
                        const double *B, int ndir, const double *mu,
                        const double *phi, const double *w, double *J_out,
                        double *lstar_out, int nthreads)
{
    if (check_grid(g) || check_dirs(ndir, mu)) return ORC_EINVAL;
    long N = (long)g->nx * g->ny * g->nz;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (long v = 0; v < N; ++v) {
        long i0 = v % g->nx, j0 = (v / g->nx) % g->ny, k0 = v / ((long)g->nx * g->ny);
        double J = 0.0;
        for (int d = 0; d < ndir; ++d)
            J += w[d] * orc_intensity(g, chi, S, B, mu[d], phi[d], i0, j0, k0);
        J_out[v] = J;
        if (lstar_out) {
            double row[27] = {0};
            for (int d = 0; d < ndir; ++d)
                lstar_one(g, chi, mu[d], phi[d], w[d], i0, j0, k0, row);
            for (int o = 0; o < 27; ++o) lstar_out[(long)o * N + v] = row[o];
        }
    }
    return ORC_OK;
}

/* ---- Short characteristics (see header) ---------------------------------- */

/* Intensity on the entry plane of a direction, at node (i, j, k). */
static double sc_entry_intensity(const orc_grid *g, const double *chi, const double *B,
                                 int bc, double amu, long i, long j, long k)
{
    if (!bc) return 0.0;
    double I = B[vidx(g, i, j, k)];
    if (bc == 2) I += amu * diffusion_gradient(g, chi, B, i, j);
    return I;
}

/* w_cur and e of the last segment into node (i, j, k), whose upstream
 * point lies on plane k - s. */
static void sc_segment(const orc_grid *g, const double *chi, const orc_dir *d, long i, long j,
                       long k, double *wc, double *wu, double *e)
{
    double x = (double)i - d->ax, y = (double)j - d->ay;
    double dtau = d->ds * (bilinear(g, chi, k - d->s, x, y) + chi[vidx(g, i, j, k)]) / 2.0;
    orc_weights(dtau, wc, wu);
    *e = exp(-dtau);
}

/* Lambda* row of voxel (i0, j0, k0) for one direction (see header). */
static void sc_lstar_one(const orc_grid *g, const double *chi, double mu, double phi,
                         double wd, long i0, long j0, long k0, double *lrow /*[27]*/)
{
    orc_dir d = dir_geometry(g, mu, phi);
    long kin = d.s > 0 ? 0 : g->nz - 1;
    if (k0 == kin) return;                 /* I = I_bc there: no dependence on S */
    long ku = k0 - d.s;
    double wc, wu, e;
    sc_segment(g, chi, &d, i0, j0, k0, &wc, &wu, &e);
    lrow[13] += wd * wc;
    double x = (double)i0 - d.ax, y = (double)j0 - d.ay;
    double fx0 = floor(x), fy0 = floor(y);
    double tx = x - fx0, ty = y - fy0;
    long nodes_x[2] = {(long)fx0, (long)fx0 + 1}, nodes_y[2] = {(long)fy0, (long)fy0 + 1};
    double bx[2] = {1.0 - tx, tx}, by[2] = {1.0 - ty, ty};
    for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
            long ic = wrapi(nodes_x[a], g->nx), jc = wrapi(nodes_y[b], g->ny);
            double wcc = 0.0, wuc, ec;
            if (ku != kin) sc_segment(g, chi, &d, ic, jc, ku, &wcc, &wuc, &ec);
            int o = neighbour_offset(g, nodes_x[a], nodes_y[b], ku, i0, j0, k0);
            if (o >= 0) lrow[o] += wd * bx[a] * by[b] * (wu + e * wcc);
        }
}

/* Short-characteristics formal solution: J_out[N] and, if lstar_out !=
 * NULL, its Lambda* [27][N].  Directions are summed in index order. */
int orc_formal_solution_sc(const orc_grid *g, const double *chi, const double *S,
                           const double *B, int ndir, const double *mu,
                           const double *phi, const double *w, double *J_out,
                           double *lstar_out, int nthreads)
{
    if (check_grid(g) || check_dirs(ndir, mu) || g->src_order != 0) return ORC_EINVAL;
    long nxy = (long)g->nx * g->ny, N = nxy * g->nz;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    double *I = malloc(sizeof(double) * N);
    if (!I) return ORC_ENOMEM;
    for (long v = 0; v < N; ++v) J_out[v] = 0.0;
    for (int dd = 0; dd < ndir; ++dd) {
        orc_dir d = dir_geometry(g, mu[dd], phi[dd]);
        int bc = d.s > 0 ? g->top_bc : g->bottom_bc;
        long kin = d.s > 0 ? 0 : g->nz - 1;
        for (long n = 0; n < g->nz; ++n) {
            long k = d.s > 0 ? n : g->nz - 1 - n;
#pragma omp parallel for schedule(static)
            for (long t = 0; t < nxy; ++t) {
                long i = t % g->nx, j = t / g->nx, v = vidx(g, i, j, k);
                if (k == kin) {
                    I[v] = sc_entry_intensity(g, chi, B, bc, fabs(mu[dd]), i, j, k);
                    continue;
                }
                long ku = k - d.s;
                double x = (double)i - d.ax, y = (double)j - d.ay;
                double wc, wu, e;
                sc_segment(g, chi, &d, i, j, k, &wc, &wu, &e);
                I[v] = bilinear(g, I, ku, x, y) * e + wc * S[v] + wu * bilinear(g, S, ku, x, y);
            }
        }
        for (long v = 0; v < N; ++v) J_out[v] += w[dd] * I[v];
    }
    free(I);
    if (lstar_out) {
#pragma omp parallel for schedule(dynamic, 16)
        for (long v = 0; v < N; ++v) {
            long i0 = v % g->nx, j0 = (v / g->nx) % g->ny, k0 = v / nxy;
            double row[27] = {0};
            for (int dd = 0; dd < ndir; ++dd)
                sc_lstar_one(g, chi, mu[dd], phi[dd], w[dd], i0, j0, k0, row);
            for (int o = 0; o < 27; ++o) lstar_out[(long)o * N + v] = row[o];
        }
    }
    return ORC_OK;
}

/* Mean intensity at a sample of voxels only (full-size spot checks). */
int orc_mean_intensity_at(const orc_grid *g, const double *chi, const double *S,
                          const double *B, int ndir, const double *mu,
                          const double *phi, const double *w, long nsample,
                          const long *voxels, double *J_out, int nthreads)
{
    if (check_grid(g) || check_dirs(ndir, mu)) return ORC_EINVAL;
    long N = (long)g->nx * g->ny * g->nz;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (long q = 0; q < nsample; ++q) {
        long v = voxels[q];
        if (v < 0 || v >= N) { J_out[q] = NAN; continue; }
        long i0 = v % g->nx, j0 = (v / g->nx) % g->ny, k0 = v / ((long)g->nx * g->ny);
        double J = 0.0;
        for (int d = 0; d < ndir; ++d)
            J += w[d] * orc_intensity(g, chi, S, B, mu[d], phi[d], i0, j0, k0);
        J_out[q] = J;
    }
    return ORC_OK;
}

/* Lambda* rows [27] of a sample of voxels only (full-size spot checks):
 * the same per-characteristic contributions (lstar_one) as
 * orc_formal_solution, for the listed flat voxel indices; lstar_out is
 * [nsample][27], rows of indices outside the grid are NaN. */
int orc_lstar_at(const orc_grid *g, const double *chi, int ndir, const double *mu,
                 const double *phi, const double *w, long nsample, const long *voxels,
                 double *lstar_out, int nthreads)
{
    if (check_grid(g) || check_dirs(ndir, mu)) return ORC_EINVAL;
    long N = (long)g->nx * g->ny * g->nz;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (long q = 0; q < nsample; ++q) {
        long v = voxels[q];
        double *row = lstar_out + q * 27;
        if (v < 0 || v >= N) {
            for (int o = 0; o < 27; ++o) row[o] = NAN;
            continue;
        }
        long i0 = v % g->nx, j0 = (v / g->nx) % g->ny, k0 = v / ((long)g->nx * g->ny);
        for (int o = 0; o < 27; ++o) row[o] = 0.0;
        for (int d = 0; d < ndir; ++d)
            lstar_one(g, chi, mu[d], phi[d], w[d], i0, j0, k0, row);
    }
    return ORC_OK;
}

/* Index of the neighbour of voxel v at offset o, or -1 outside the grid. */
static long neighbour_index(const orc_grid *g, long v, int o)
{
    long i0 = v % g->nx, j0 = (v / g->nx) % g->ny, k0 = v / ((long)g->nx * g->ny);
    int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
    long kk = k0 + oz;
    if (kk < 0 || kk >= g->nz) return -1;
    return vidx(g, wrapi(i0 + ox, g->nx), wrapi(j0 + oy, g->ny), kk);
}

/* New value of voxel v from the current iterate X (all offsets but the
 * centre), given the right-hand side rhs[v]. */
static double os_update(const orc_grid *g, const double *lstar, const double *eps,
                        const double *rhs, const double *X, long v, long N)
{
    double acc = rhs[v];
    for (int o = 0; o < 27; ++o) {
        if (o == 13) continue;
        long j = neighbour_index(g, v, o);
        if (j >= 0) acc += lstar[(long)o * N + v] * (1.0 - eps[j]) * X[j];
    }
    return acc / (1.0 - lstar[13L * N + v] * (1.0 - eps[v]));
}

static int colour_of(const orc_grid *g, long v)
{
    long i = v % g->nx, j = (v / g->nx) % g->ny, k = v / ((long)g->nx * g->ny);
    return (int)((i + j + k) & 1);
}

/* Operator-splitting step from J_old: Jacobi ("Jordan") sweeps (method 0)
 * or red-black Gauss-Seidel sweeps (method 1). */
int orc_os_step_method(const orc_grid *g, const double *lstar, const double *eps,
                       const double *J_fs, const double *J_old, double *J_new,
                       double tol_inner, int max_sweeps, int *sweeps_out, int method)
{
    if (check_grid(g) || max_sweeps < 1 || method < 0 || method > 1) return ORC_EINVAL;
    long N = (long)g->nx * g->ny * g->nz;
    double *rhs = malloc(sizeof(double) * N);
    double *Jc = malloc(sizeof(double) * N);
    double *Jn = malloc(sizeof(double) * N);
    double *upd = malloc(sizeof(double) * N);
    if (!rhs || !Jc || !Jn || !upd) {
        free(rhs); free(Jc); free(Jn); free(upd);
        return ORC_ENOMEM;
    }
    for (long v = 0; v < N; ++v) {
        double r = J_fs[v];
        for (int o = 0; o < 27; ++o) {
            long j = neighbour_index(g, v, o);
            if (j >= 0) r -= lstar[(long)o * N + v] * (1.0 - eps[j]) * J_old[j];
        }
        rhs[v] = r;
        Jc[v] = J_old[v];
    }
    int sweeps = 0;
    for (int n = 0; n < max_sweeps; ++n) {
        if (method == 0) {
            for (long v = 0; v < N; ++v) Jn[v] = os_update(g, lstar, eps, rhs, Jc, v, N);
        } else {
            /* red from the old values; then black from new red + old black */
            memcpy(Jn, Jc, sizeof(double) * N);
            for (int colour = 0; colour < 2; ++colour) {
                for (long v = 0; v < N; ++v)
                    if (colour_of(g, v) == colour) upd[v] = os_update(g, lstar, eps, rhs, Jn, v, N);
                for (long v = 0; v < N; ++v)
                    if (colour_of(g, v) == colour) Jn[v] = upd[v];
            }
        }
        double delta = 0.0;
        for (long v = 0; v < N; ++v) {
            double rel = fabs(Jn[v] - Jc[v]) / fabs(Jn[v]);
            if (!(rel <= delta)) delta = rel;     /* NaN propagates */
        }
        memcpy(Jc, Jn, sizeof(double) * N);
        sweeps = n + 1;
        if (delta < tol_inner) break;
    }
    memcpy(J_new, Jc, sizeof(double) * N);
    if (sweeps_out) *sweeps_out = sweeps;
    free(rhs); free(Jc); free(Jn); free(upd);
    return ORC_OK;
}

/* Operator-splitting step, Jacobi ("Jordan") iterations from J_old. */
int orc_os_step(const orc_grid *g, const double *lstar, const double *eps,
                const double *J_fs, const double *J_old, double *J_new,
                double tol_inner, int max_sweeps, int *sweeps_out)
{
    return orc_os_step_method(g, lstar, eps, J_fs, J_old, J_new, tol_inner, max_sweeps,
                              sweeps_out, 0);
}

/* Second-order Ng extrapolation (see header).  Returns 0, or 1 if the 2x2
 * system is singular (x0 is then left unchanged). */
int orc_ng_step(long N, const double *x0, const double *x1, const double *x2,
                const double *x3, double *out, double *a_out, double *b_out)
{
    double a11 = 0, a12 = 0, a22 = 0, b1 = 0, b2 = 0;
    for (long i = 0; i < N; ++i) {
        double d0 = x0[i] - x1[i], d1 = x1[i] - x2[i], d2 = x2[i] - x3[i];
        double q1 = d0 - d1, q2 = d0 - d2;
        double w = 1.0 / (x0[i] * x0[i]);
        a11 += w * q1 * q1;
        a12 += w * q1 * q2;
        a22 += w * q2 * q2;
        b1 += w * d0 * q1;
        b2 += w * d0 * q2;
    }
    double det = a11 * a22 - a12 * a12;
    if (!(fabs(det) > 1e-300) || !(det == det)) {
        for (long i = 0; i < N; ++i) out[i] = x0[i];
        if (a_out) *a_out = 0.0;
        if (b_out) *b_out = 0.0;
        return 1;
    }
    double a = (b1 * a22 - b2 * a12) / det;
    double b = (b2 * a11 - b1 * a12) / det;
    for (long i = 0; i < N; ++i) out[i] = (1.0 - a - b) * x0[i] + a * x1[i] + b * x2[i];
    if (a_out) *a_out = a;
    if (b_out) *b_out = b;
    return 0;
}

/* Outer iteration.  J_inout holds J^0 on entry if use_initial != 0 (else
 * J^0 = B) and the last iterate on exit.  deltas/sweeps (may be NULL) get
 * one entry per outer iteration.  Returns 0 on convergence, 3 if max_iter
 * was reached first (both leave J_inout valid). */
int orc_solve_ng(const orc_grid *g, const double *chi, const double *eps,
                 const double *B, int ndir, const double *mu, const double *phi,
                 const double *w, double tol, int max_iter, double tol_inner,
                 int max_sweeps, int use_initial, double *J_inout,
                 double *lstar_out, int *iters_out, double *deltas, int *sweeps,
                 int nthreads, int ng_period, double ng_min_delta);

int orc_solve_ex(const orc_grid *g, const double *chi, const double *eps,
                 const double *B, int ndir, const double *mu, const double *phi,
                 const double *w, double tol, int max_iter, double tol_inner,
                 int max_sweeps, int use_initial, double *J_inout,
                 double *lstar_out, int *iters_out, double *deltas, int *sweeps,
                 int nthreads, int ng_period, double ng_min_delta, int os_method,
                 int fs_method);

int orc_solve(const orc_grid *g, const double *chi, const double *eps,
              const double *B, int ndir, const double *mu, const double *phi,
              const double *w, double tol, int max_iter, double tol_inner,
              int max_sweeps, int use_initial, double *J_inout,
              double *lstar_out, int *iters_out, double *deltas, int *sweeps,
              int nthreads)
{
    return orc_solve_ng(g, chi, eps, B, ndir, mu, phi, w, tol, max_iter, tol_inner, max_sweeps,
                        use_initial, J_inout, lstar_out, iters_out, deltas, sweeps, nthreads, 0,
                        0.0);
}

/* Outer iteration with Ng acceleration every ng_period >= 4 iterations
 * (0: none) while the previous delta >= ng_min_delta. */
int orc_solve_ng(const orc_grid *g, const double *chi, const double *eps,
                 const double *B, int ndir, const double *mu, const double *phi,
                 const double *w, double tol, int max_iter, double tol_inner,
                 int max_sweeps, int use_initial, double *J_inout,
                 double *lstar_out, int *iters_out, double *deltas, int *sweeps,
                 int nthreads, int ng_period, double ng_min_delta)
{
    return orc_solve_ex(g, chi, eps, B, ndir, mu, phi, w, tol, max_iter, tol_inner, max_sweeps,
                        use_initial, J_inout, lstar_out, iters_out, deltas, sweeps, nthreads,
                        ng_period, ng_min_delta, 0, 0);
}

/* The same with the operator-splitting method (0 Jacobi, 1 red-black
 * Gauss-Seidel) and the formal solution (0 long characteristics, 1 short
 * characteristics) chosen. */
int orc_solve_ex(const orc_grid *g, const double *chi, const double *eps,
                 const double *B, int ndir, const double *mu, const double *phi,
                 const double *w, double tol, int max_iter, double tol_inner,
                 int max_sweeps, int use_initial, double *J_inout,
                 double *lstar_out, int *iters_out, double *deltas, int *sweeps,
                 int nthreads, int ng_period, double ng_min_delta, int os_method,
                 int fs_method)
{
    if (ng_period != 0 && ng_period < 4) return ORC_EINVAL;
    if (os_method < 0 || os_method > 1 || fs_method < 0 || fs_method > 1) return ORC_EINVAL;
    if (check_grid(g) || check_dirs(ndir, mu) || max_iter < 1) return ORC_EINVAL;
    long N = (long)g->nx * g->ny * g->nz;
    double *J = malloc(sizeof(double) * N), *S = malloc(sizeof(double) * N);
    double *Jfs = malloc(sizeof(double) * N), *Jn = malloc(sizeof(double) * N);
    double *L = malloc(sizeof(double) * N * 27);
    double *hist = malloc(sizeof(double) * N * 4);   /* ring of the last four iterates */
    if (!J || !S || !Jfs || !Jn || !L || !hist) {
        free(J); free(S); free(Jfs); free(Jn); free(L); free(hist);
        return ORC_ENOMEM;
    }
    for (long v = 0; v < N; ++v) J[v] = use_initial ? J_inout[v] : B[v];
    int it, status = 3, nhist = 0;
    double prev_delta = 0.0;
    memcpy(hist, J, sizeof(double) * N);
    nhist = 1;
    for (it = 1; it <= max_iter; ++it) {
        for (long v = 0; v < N; ++v) S[v] = eps[v] * B[v] + (1.0 - eps[v]) * J[v];
        if (fs_method == 1)
            orc_formal_solution_sc(g, chi, S, B, ndir, mu, phi, w, Jfs, it == 1 ? L : NULL,
                                   nthreads);
        else
            orc_formal_solution(g, chi, S, B, ndir, mu, phi, w, Jfs, it == 1 ? L : NULL, nthreads);
        int ns = 0;
        orc_os_step_method(g, L, eps, Jfs, J, Jn, tol_inner, max_sweeps, &ns, os_method);
        if (ng_period) {
            /* history: hist[k] holds the iterate k steps back (k = 0 newest) */
            memmove(hist + N, hist, sizeof(double) * N * 3);
            memcpy(hist, Jn, sizeof(double) * N);
            if (nhist < 4) ++nhist;
            if (nhist == 4 && it % ng_period == 0 && (it == 1 || prev_delta >= ng_min_delta)) {
                orc_ng_step(N, hist, hist + N, hist + 2 * N, hist + 3 * N, Jn, NULL, NULL);
                memcpy(hist, Jn, sizeof(double) * N);
                nhist = 1;
            }
        }
        double delta = 0.0;
        for (long v = 0; v < N; ++v) {
            double rel = fabs(Jn[v] - J[v]) / fabs(Jn[v]);
            if (!(rel <= delta)) delta = rel;
        }
        memcpy(J, Jn, sizeof(double) * N);
        prev_delta = delta;
        if (deltas) deltas[it - 1] = delta;
        if (sweeps) sweeps[it - 1] = ns;
        if (delta < tol) { status = 0; break; }
    }
    if (iters_out) *iters_out = it > max_iter ? max_iter : it;
    memcpy(J_inout, J, sizeof(double) * N);
    if (lstar_out) memcpy(lstar_out, L, sizeof(double) * N * 27);
    free(J); free(S); free(Jfs); free(Jn); free(L); free(hist);
    return status;
}
