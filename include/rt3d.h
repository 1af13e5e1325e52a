/*
 * rt3d.h -- C ABI of the GB300 (sm_103a) hot path of the 3D radiative
 * transfer framework of Hauschildt & Baron, "A 3D radiative transfer
 * framework XIII: OpenCL implementation" (2011).
 *
 * The library solves, on one GPU, the problem the paper hands to its GPU
 * kernels (Sect. 2, first paragraph; abstract): the formal solution on a
 * Cartesian voxel slab with periodic boundary conditions in x and y, the
 * construction of the nearest-neighbour Lambda*, and the operator-splitting
 * step for the mean intensity J, iterated to convergence for coherent
 * isotropic scattering S = eps B + (1 - eps) J (Sect. 3.1, list item 5).
 *
 * Conventions shared by every call
 * --------------------------------
 *  Grid.  nx x ny x nz voxels, spacings dx, dy, dz.  Arrays are C-ordered
 *   [nz][ny][nx] (x fastest), N = nx*ny*nz.  k is the depth index: k = 0 is
 *   the outer (top) boundary, k = nz-1 the inner (bottom) one (Sect. 3.1:
 *   z_max outside, z_min inside).  x and y are periodic (Sect. 2.2).
 *  Directions.  d = (mu_d, phi_d, w_d); propagation vector
 *   (sqrt(1-mu^2) cos phi, sqrt(1-mu^2) sin phi, mu); mu > 0 propagates
 *   towards larger k.  J = sum_d w_d I_d.  1e-6 <= |mu| <= 1.
 *  Characteristic.  Each (voxel, direction) is integrated back along its
 *   characteristic one z-plane per step (path length dz/|mu| per step) to
 *   the boundary plane it entered through; chi, S and B are bilinear in
 *   each plane with periodic wrap; segment optical depths are trapezoidal;
 *   the source is linear in tau on each segment.
 *  Lambda*.  27 entries per voxel, Lambda*_{i,o} = dJ_i/dS_{wrap(i+o)},
 *   offset index o = (oz+1)*9 + (oy+1)*3 + (ox+1), stored [27][nz][ny][nx];
 *   entries whose plane lies outside the grid are 0.
 *  Operator splitting (Sect. 2.3).  (1 - Lambda* D) J_new = J_fs -
 *   Lambda* D J_old with D = diag(1 - eps), solved by Jacobi ("Jordan")
 *   sweeps started from J_old until max|dJ|/|J| < tol_inner or max_sweeps.
 *  Outer iteration (Sect. 2).  S = eps B + (1-eps) J -> formal solution ->
 *   operator splitting; delta = max_i |J_new - J_old| / |J_new|; stop when
 *   delta < tol or after max_iter.  J starts from B (set by rt_set_planck)
 *   unless rt_set_J gave another start.
 *
 *  Precision.  RT_FP64: every step in FP64.  RT_FP32_SWEEP: the march
 *   along the characteristics (interpolation, exp weights, transmission,
 *   intensity) runs in FP32 on FP32 copies of chi and S; J, Lambda*, the
 *   operator-splitting solve and the convergence test stay in FP64
 *   (Sect. 3.1: smaller eps needs double precision for the operator
 *   splitting equations).  RT_DF64: the march runs in double-float
 *   arithmetic (pairs of FP32 numbers, ~48 significant bits) on the FP32
 *   pipes, to FP64-level accuracy; J, Lambda*, the operator splitting and
 *   the convergence test are FP64.
 *
 *  Memory and ownership.  The caller owns every pointer it passes and
 *   every buffer it receives.  Host-pointer calls copy in and out and
 *   return when the result is in the caller's buffer.  *_dev calls take
 *   device pointers of the context's device, run on the context's stream
 *   (rt_set_stream; default: a stream the context creates) and return
 *   without synchronising unless the call itself needs a value on the host
 *   (solve and os_step read convergence flags).  The context allocates its
 *   own working storage on the device (opacities, Lambda*, tables, scratch)
 *   in the rt_set_* calls and frees it in rt_destroy; the paper keeps all
 *   of it on the GPU and moves only inputs and J across the bus (Sect. 2).
 *
 *  Errors.  Every call returns an rt_status.  On error the context is left
 *   usable, the outputs are unspecified and rt_last_error() describes the
 *   cause.  Invalid arguments (null pointers, nx or ny < 3, nz < 2, chi <= 0
 *   or not finite, eps outside (0,1], |mu| < 1e-6 or > 1, weights that do
 *   not sum to 1 within 1e-12) give RT_EINVAL; calls before the data they
 *   need was set give RT_ESTATE; CUDA failures give RT_ECUDA.
 *
 *  Threading.  A context may be used by one host thread at a time.
 */
#ifndef RT3D_H
#define RT3D_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RT_OK = 0,
    RT_EINVAL = 1,      /* invalid argument */
    RT_ENOMEM = 2,      /* device allocation failed */
    RT_ECUDA = 3,       /* a CUDA call failed */
    RT_ENOTCONV = 4,    /* max_iter reached before delta < tol (outputs valid) */
    RT_ETIMEOUT = 5,    /* a bounded device-side wait gave up */
    RT_ESTATE = 6,      /* the call needs data that was not set yet */
    RT_ESCRATCH = 7,    /* too large for rt_formal_solution_noalloc's fixed scratch */
    RT_EBOUNDS = 8      /* checked build: a kernel found an index outside its buffer */
} rt_status;

enum { RT_FP64 = 0, RT_FP32_SWEEP = 1, RT_DF64 = 2 };
enum { RT_BC_ZERO = 0, RT_BC_PLANCK = 1, RT_BC_DIFFUSION = 2 };
/* Operator-splitting methods (Sect. 2.3), see rt_set_os_method. */
enum { RT_OS_JACOBI = 0, RT_OS_GAUSS_SEIDEL = 1 };
/* Formal-solution methods, see rt_set_fs_method. */
enum { RT_FS_LONG = 0, RT_FS_SHORT = 1 };
/* Source interpolation along a characteristic, see rt_set_source_order. */
enum { RT_SRC_LINEAR = 0, RT_SRC_PARABOLIC = 1 };

typedef struct rt_ctx rt_ctx;

/* Library version string (static storage). */
const char *rt_version(void);

/* Create a context on CUDA device `device` for precision RT_FP64,
 * RT_FP32_SWEEP or RT_DF64.  *ctx receives the handle (NULL on failure). */
int rt_create(rt_ctx **ctx, int device, int precision);

/* Free the context and every device buffer it owns.  NULL is accepted. */
int rt_destroy(rt_ctx *ctx);

/* Text of the last error on this context ("" if none; static storage of
 * the context, valid until the next call on it). */
const char *rt_last_error(const rt_ctx *ctx);

/* Use `stream` (a cudaStream_t of the context's device, e.g. the current
 * PyTorch stream) for all later work; NULL restores the context's own. */
int rt_set_stream(rt_ctx *ctx, void *stream);

/* Grid of nx x ny x nz voxels with spacings dx, dy, dz (> 0).  nx, ny >= 3
 * (a smaller periodic grid would alias the 27-point neighbourhood),
 * 2 <= nz <= 65535 (the march launches give the planes a grid dimension of
 * at most 65535 blocks), nx * ny <= 2^30.  Invalidates every field set
 * before. */
int rt_set_grid(rt_ctx *ctx, int nx, int ny, int nz, double dx, double dy, double dz);

/* Incoming intensity at the top (entered by mu > 0) and bottom (mu < 0):
 * RT_BC_ZERO (I = 0, the outer boundary of Sect. 3.1), RT_BC_PLANCK
 * (I = B interpolated at the entry point) or, at the bottom only,
 * RT_BC_DIFFUSION (the inner boundary's LTE diffusion, Sect. 3.1 item 4:
 * I = B + |mu| dB/dtau, with dB/dtau taken at each bottom node as
 * (B[nz-1] - B[nz-2]) / (dz (chi[nz-1] + chi[nz-2]) / 2) and interpolated
 * like B).  Default: ZERO top, PLANCK bottom. */
int rt_set_boundary(rt_ctx *ctx, int top_mode, int bottom_mode);

/* Solid-angle quadrature: ndir directions, host arrays mu[ndir],
 * phi[ndir] (radians), w[ndir] (sum 1).  Builds the per-(direction, plane)
 * geometry tables on the device; needs the grid. */
int rt_set_quadrature(rt_ctx *ctx, int ndir, const double *mu, const double *phi,
                      const double *w);

/* Opacity chi[N] (> 0, host).  Invalidates Lambda*. */
int rt_set_opacity(rt_ctx *ctx, const double *chi);
/* Thermalisation parameter eps[N] in (0, 1] (host). */
int rt_set_epsilon(rt_ctx *ctx, const double *eps);
/* Planck function B[N] (host).  Also resets the iterate J to B. */
int rt_set_planck(rt_ctx *ctx, const double *B);

/* Device-pointer forms of the three setters above (copied on the stream). */
int rt_set_opacity_dev(rt_ctx *ctx, const double *chi);
int rt_set_epsilon_dev(rt_ctx *ctx, const double *eps);
int rt_set_planck_dev(rt_ctx *ctx, const double *B);

/* Formal solution (Sect. 2.2).  S[N]: the source function on the voxel
 * nodes, or NULL to use S = eps B + (1 - eps) J of the current iterate.
 * J_fs[N] receives J = sum_d w_d I_d; lstar[27*N] (or NULL) receives
 * Lambda*, which is built on the first call after the opacity changed.
 * Host pointers. */
int rt_formal_solution(rt_ctx *ctx, const double *S, double *J_fs, double *lstar);
/* Same with device pointers (S may be NULL; lstar may be NULL). */
int rt_formal_solution_dev(rt_ctx *ctx, const double *S, double *J_fs, double *lstar);

/* One operator-splitting solve (Sect. 2.3) with the context's Lambda* and
 * eps: J_new[N] from J_fs[N] and J_old[N].  *sweeps (or NULL) receives the
 * number of Jacobi sweeps.  Needs Lambda* (a formal solution since the
 * opacity was set).  Host pointers. */
int rt_os_step(rt_ctx *ctx, const double *J_fs, const double *J_old, double *J_new,
               double tol_inner, int max_sweeps, int *sweeps);
/* Same with device pointers. */
int rt_os_step_dev(rt_ctx *ctx, const double *J_fs, const double *J_old, double *J_new,
                   double tol_inner, int max_sweeps, int *sweeps);

/* Outer iteration from the context's current J until delta < tol or
 * max_iter iterations; tol = 0 runs exactly max_iter iterations.  J_out[N]
 * (host, or NULL) receives the final iterate, which also stays in the
 * context.  iters, last_delta (or NULL) receive the count and the final
 * delta; deltas[max_iter] and sweeps[max_iter] (host, or NULL) receive the
 * per-iteration delta and Jacobi sweep count.  Returns RT_ENOTCONV if
 * max_iter was reached with tol > 0 (outputs still valid). */
int rt_solve(rt_ctx *ctx, double tol, int max_iter, double tol_inner, int max_sweeps,
             double *J_out, int *iters, double *last_delta, double *deltas, int *sweeps);
/* Same, J_out a device pointer (or NULL). */
int rt_solve_dev(rt_ctx *ctx, double tol, int max_iter, double tol_inner, int max_sweeps,
                 double *J_out, int *iters, double *last_delta, double *deltas, int *sweeps);

/* Read or replace the current iterate J[N] (checkpoint / resume). */
int rt_get_J(rt_ctx *ctx, double *J);
int rt_set_J(rt_ctx *ctx, const double *J);

/* Number of march steps executed by the last formal solution (steps cut by
 * the transmission cutoff are not counted). */
int rt_last_step_count(rt_ctx *ctx, unsigned long long *steps);

/* Recorded formal solution (long characteristics: RT_FP64 with the linear
 * or the parabolic source, RT_FP32_SWEEP, RT_DF64).
 * The march is linear in the source S once the opacities, directions and
 * boundary values are fixed (Sect. 2.2: I is a sum of weighted S values
 * along the characteristic plus the transmitted boundary intensity).  The
 * first formal solution after any of them changes runs the march as usual
 * and also stores, per (voxel, direction, step), the coefficient of S at
 * that step's upstream point (the products of transmissions and segment
 * weights), cut at 1e-2 times the cutoff; every formal solution then
 * evaluates J from those coefficients and its S (FP64: five FP64
 * operations per step instead of the weights' exponential and division),
 * so J does not depend on which formal solution recorded.  The parabolic
 * source also keeps the coefficient of S at the downstream point per
 * (voxel, direction).  The FP32 sweep records FP32 coefficients of
 * S(p_m) - S_0 for its difference form and replays them with the
 * interpolated source differences of its march (its finishing stage
 * replays the same recording for the source change); the double-float
 * form records double-float coefficients of S(p_m) - S_0.  Memory, FP64
 * and double-float: 8 ndir nx ny nz (nz-1)/2 bytes of coefficients plus
 * 4 ndir nz ceil(nx ny/32) + 128 N bytes (65^3 x 1024 directions: 72 GB;
 * parabolic: + 8 ndir N); FP32 sweep: about 8 ndir nx ceil(ny/2) nz (nz+6)/2
 * bytes of coefficients (blocks of four steps) plus 4 ndir nz nx ny/64 +
 * 128 N + the source records (65^3 x 1024: 38.9 GB).  max_bytes: -1
 * (default) records when that fits in 60% of the device and leaves 2 GiB
 * free, 0 never records, > 0 records when it fits in max_bytes; otherwise
 * every formal solution marches.  J agrees with the march to rounding (the
 * terms are summed in another order).  Short characteristics ignore the
 * setting.  RT_EINVAL for max_bytes < -1. */
int rt_set_fs_record(rt_ctx *ctx, long long max_bytes);
/* Bytes held for the recorded march (0 if none) and whether a recording
 * valid for the current opacities, directions and boundary is held. */
int rt_fs_record_info(rt_ctx *ctx, long long *bytes, int *valid);

/* Diagnostics for the FP32-sweep long-characteristics march: march the
 * source S (host array [N], or NULL for S = eps B + (1 - eps) J from the
 * current iterate) once through a branch-counting copy of the march kernel
 * and return the steps executed (*steps, as rt_last_step_count) and how
 * many of them evaluated the linear-source segment weights (Sect. 2.2)
 * through the series branch, optical depth x < 2 (*series; the rest took
 * the closed form).
 * J is not returned and the iterate is unchanged.  RT_EINVAL for another
 * precision or method, or NULL outputs. */
int rt_fs32_branch_counts(rt_ctx *ctx, const double *S, unsigned long long *steps,
                          unsigned long long *series);

/* Ng acceleration of the outer iteration (the paper keeps it, with the
 * set-up, in host code, Sect. 2): after every `period`-th iteration, once
 * the four latest iterates x0 (newest) .. x3 are held, x0 is replaced by
 * (1 - a - b) x0 + a x1 + b x2 with a, b minimising
 * sum_i (d0 - a (d0 - d1) - b (d0 - d2))_i^2 / x0_i^2, d0 = x0 - x1,
 * d1 = x1 - x2, d2 = x2 - x3 (second-order Ng extrapolation); the history
 * then restarts.  The extrapolation is skipped while the previous
 * iteration's delta is below min_delta (>= 0): once the iterates differ only
 * by rounding noise (about 5e-8 relative for the FP32 sweep) the
 * extrapolation would amplify that noise.  delta is measured against the
 * extrapolated iterate.  The weighted sums and the 2x2 system are reduced
 * and solved on the GPU (the system in FP64 with products and differences
 * rounded as written; a singular system leaves x0 unchanged), so Ng adds
 * no host synchronisation.  period 0 (default) = off; otherwise >= 4. */
int rt_set_ng(rt_ctx *ctx, int period, double min_delta);

/* Formal-solution method.  RT_FS_LONG (default): the long characteristic
 * of every (voxel, direction), integrated back to the boundary plane it
 * entered through, O(nz) steps per pair.  RT_FS_SHORT: short
 * characteristics, O(1) per pair (the paper's own tracking of
 * characteristics started on the boundary planes is O(1) per pair too,
 * Sect. 2.2): per direction the planes are swept in the order of
 * propagation and each node takes the intensity from its upstream point on
 * the preceding plane only, I = I(p) e + w_cur S + w_up S(p) with I(p),
 * chi(p), S(p) bilinear in that plane; on the entry plane I = I_bc at the
 * node.  A different discretisation: J differs from the long
 * characteristics by the interpolation of I (it agrees exactly where every
 * upstream point is a lattice node, and on horizontally uniform slabs).
 * Lambda* is that of the chosen method (per direction the diagonal w_cur
 * and, at the nodes c of p, b_c (w_up + e w_cur(c))).  RT_FS_SHORT runs in
 * precision RT_FP64 or RT_DF64 (the latter in double-float arithmetic,
 * carrying D = I - S from plane to plane: D = e D(p) + (1 - w_cur)(S(p) - S));
 * RT_EINVAL for RT_FP32_SWEEP.  Its working memory is min(ndir, 1024) * N
 * doubles, allocated at the first formal solution.  Changing the method
 * invalidates Lambda*. */
int rt_set_fs_method(rt_ctx *ctx, int method);

/* Switch a context between RT_FP32_SWEEP and RT_DF64 (either direction;
 * RT_EINVAL for RT_FP64 on either side).  J and all settings are kept; the
 * Ng history restarts; Lambda* and the OS coefficients are rebuilt by the
 * new form at its first formal solution (the FP32-sweep form builds Lambda*
 * in FP64, the double-float form in double-float).  Typical use:
 * iterate with the FP32 sweep to its tolerance (about 5e-8; its iterate then
 * sits near its ~1e-8 rounding floor), then switch to RT_DF64 and continue
 * with Ng on to the final tolerance: the FP64-accurate iterates let Ng
 * remove the slowly converging error that small eps leaves behind.
 * Allocates the double-float tables on the first switch to RT_DF64. */
int rt_set_precision(rt_ctx *ctx, int precision);

/* Operator-splitting steps as CUDA graphs (default on): the right-hand side,
 * the sweep loop and the pick of the last sweep's iterate form one graph
 * whose WHILE node runs the sweeps and their convergence test on the
 * device, so the host launches it without waiting; an outer iteration of
 * rt_solve waits for the GPU once (for delta and the sweep count) instead
 * of once per chunk of sweeps.  Results are identical either way (same
 * kernels, same sweep count).  on = 0 selects the host-driven loop. */
int rt_set_graphs(rt_ctx *ctx, int on);

/* Automatic finishing stage for RT_FP32_SWEEP contexts: within rt_solve,
 * once an iteration's delta falls below delta_switch (and not yet below
 * tol), the next formal solution is a double-float (FP64-accurate) one,
 * J_ref = J_FS(S_ref) of the current source S_ref, and every later one is
 * J_FS(S) = J_ref + J_FS(S - S_ref) with the second term marched in FP32
 * with zero boundary intensities (the formal solution is linear in S and
 * in the boundary intensities): its FP32 rounding scales with |S - S_ref|,
 * ~1e-6 of S, so these formal solutions are accurate to ~1e-12 of J at
 * the FP32 march's cost (less: its transmission cutoff is relative to
 * |S - S_ref| against min |S_ref|).  Ng is applied every period from the
 * switch on, its history restarted.  When the solve returns (converged or
 * not) the context is back in the plain FP32 sweep with its Ng threshold.
 * The FP32 sweep's iterate stops improving near delta 1e-8 and its Ng must
 * stop near 1e-6; at small eps the remaining iterations converge slowly,
 * which the finishing stage with Ng avoids: where the error of a solve
 * stopped at delta is ~ delta / (1 - rho) for a contraction rho close to 1
 * (about 70 delta at eps = 1e-6), a 1e-6 accuracy target needs tol ~ 1e-8,
 * below the FP32 sweep's floor.  Default for RT_FP32_SWEEP contexts (and
 * batches): on, delta_switch = 1e-6; delta_switch = 0 turns it off (the
 * FP32 sweep alone, tol >= 5e-8).  The batch version applies it per
 * problem: the reference formal solution runs one double-float launch per
 * problem, the later ones share the fused FP32 launch. */
int rt_set_df_finish(rt_ctx *ctx, double delta_switch);

/* Source interpolation on each segment of a characteristic (the paper
 * names no order).  RT_SRC_LINEAR (default): S linear in optical depth
 * between the segment's end points.  RT_SRC_PARABOLIC: S quadratic through
 * the segment's two end points and the next point downstream, in optical
 * depth t measured upstream from the segment's downstream end (nodes at
 * t = a, 0, -b; a, b the optical depths of the segment and of the next one
 * downstream); with E_n = int_0^a t^n e^{-t} dt the segment adds
 * P_up S_up + P_cur S_cur + P_down S_down, P_up = (E2 + b E1)/(a(a+b)),
 * P_cur = (a b E0 - (b-a) E1 - E2)/(a b), P_down = (E2 - a E1)/(b(a+b)).
 * The last segment into a voxel uses the point one plane beyond the voxel
 * when that plane exists, else the linear weights.  Lambda* then also
 * couples to the downstream plane and may have negative entries.  Needs
 * precision RT_FP64 and RT_FS_LONG (RT_EINVAL otherwise); changing it
 * invalidates Lambda*. */
int rt_set_source_order(rt_ctx *ctx, int order);

/* Operator-splitting method (Sect. 2.3 names the Jordan method and
 * Gauss-Seidel iterations).  RT_OS_JACOBI (default): every sweep updates
 * all voxels from the previous iterate.  RT_OS_GAUSS_SEIDEL: red-black
 * order; voxel (i,j,k) is red if i+j+k is even; a sweep updates the red
 * voxels from the iterate at its start, then the black voxels from the new
 * red and the old black values (updates within a colour are simultaneous,
 * so the result does not depend on thread order).  Both stop on the same
 * test, max |J^{n+1} - J^n| / |J^{n+1}| < tol_inner, and solve the same
 * system; the sweep counts reported are sweeps (two launches each for
 * Gauss-Seidel).  Takes effect at the next operator-splitting step.
 * RT_EINVAL for another value. */
int rt_set_os_method(rt_ctx *ctx, int method);

/* Tuning: the directions are summed into J in 8 fixed slots (direction d in
 * slot d mod 8, each slot in increasing d, then the slots in order), so J
 * is bit-reproducible and independent of this knob.  `groups` (1..8) sets
 * how many thread blocks share the slots of one voxel tile; 0 = auto. */
int rt_set_direction_groups(rt_ctx *ctx, int groups);
/* Tuning: threads per block of the FP32-sweep march, 64, 128 or 256 (0 =
 * default, 128).  64 and 128 keep 896 resident threads per SM (72
 * registers per thread), 256 keeps 768 (80 registers); the fused batch
 * launch keeps 768 at every size.  J does not depend on it.  RT_EINVAL
 * otherwise. */
int rt_set_block_threads(rt_ctx *ctx, int threads);
/* Tuning: block order of the FP32-sweep march.  1: the tiles of a plane
 * are consecutive blocks, so the resident blocks share a few planes and
 * read every plane within their rays' reach; 2: the planes of a tile are
 * consecutive, so they share a few lateral tiles through every plane;
 * 0 (default): 2 once the padded source planes of the grid exceed 64 MiB
 * (no longer held in L2 together), else 1.  J does not depend on it.
 * RT_EINVAL for another value. */
int rt_set_block_order(rt_ctx *ctx, int order);

/* Tuning: relative transmission cutoff.  The march along a characteristic
 * stops once T * max(|S|, |I_bc|) <= cut * |I| (the rest can change I by
 * at most that much).  0 disables the cutoff.  Default 1e-17 (FP64) and
 * 1e-9 (FP32 sweep). */
int rt_set_cutoff(rt_ctx *ctx, double cut);

/* Diagnostic: evaluate, on the current device, the segment weights the
 * march uses for n optical depths x[n] (device pointers): w_cur (weight of
 * the downstream node), w_up (upstream node) and e = exp(-x) of the linear-
 * in-tau source integral over one segment, in the arithmetic of `precision`
 * (RT_FP64 or RT_FP32_SWEEP; FP32 results are widened to double).  Below
 * x = 2 the FP32 march itself forms T w_up from the next transmission
 * (T e = T_next) with the same polynomials instead of multiplying by e.
 * Enqueued on `stream`. */
int rt_segment_weights(int precision, long long n, const double *x, double *w_cur,
                       double *w_up, double *e, void *stream);

/* Measured arithmetic peaks of `device` (diagnostics; the paper has no
 * counterpart): dense FP64 and FP32 fused multiply-add throughput in
 * TFLOP/s (an FMA counts 2 flops), from register-resident FMA chains that
 * fill every SM, timed with CUDA events at the clocks the GPU runs at.
 * These are the denominators of the formal-solution marches' rooflines,
 * which are bound by arithmetic, not memory.  Allocates and frees a small
 * device buffer; synchronises the device. */
int rt_probe_peaks(int device, double *fp64_tflops, double *fp32_tflops);

/* Allocation-free formal solution.
 *
 * Some callers must not allocate device memory once they are running: a
 * plug-in inside a host application that owns every device allocation
 * through its own pool, a service that budgets its memory up front and may
 * not grow, or code that must not pay the implicit device-wide
 * synchronisation a cudaMalloc can cause.  For them this entry point does
 * the same work as rt_formal_solution_dev (the paper has no counterpart;
 * it only changes where the working memory comes from) without creating a
 * context and without any cudaMalloc, cudaFree or allocating library call:
 * its working memory (geometry tables, the per-direction-slot partial sums
 * of J, the source bound of the transmission cutoff) lives in one
 * statically sized device array of RT_NOALLOC_SCRATCH_BYTES bytes that the
 * library owns.  Every GPU that loads the library holds that array until
 * the process exits.
 *
 * Arguments: grid (nx, ny >= 3, 2 <= nz <= 65535, spacings > 0), boundary modes,
 * ndir and HOST arrays mu, phi, w of the quadrature (same rules as
 * rt_set_quadrature); DEVICE pointers chi[N] (> 0), S[N], B[N] (only read
 * where a boundary mode is RT_BC_PLANCK; may be NULL otherwise) and the
 * output J_fs[N]; `stream` is a cudaStream_t of the current device (NULL:
 * the legacy default stream).  The work runs in FP64 on the calling
 * thread's current device and is enqueued on `stream`; the call returns
 * without waiting for it (only the small quadrature copy from host memory
 * is synchronous).  Returns RT_ESCRATCH, before touching the GPU, when
 * 64*N + 88*ndir*nz + 88*ndir + 8 bytes (plus up to 2.5 KiB of alignment
 * padding) exceed the scratch: per voxel the eight direction-slot partial
 * sums of J, per (direction, plane) the lattice offset and three tables of
 * bilinear weights, per direction mu, phi, w and the direction record; the
 * 65^3 slab with 1024 directions takes 23.5 MB.  RT_EINVAL for invalid
 * arguments (device data is not inspected); RT_ECUDA if a CUDA call fails.
 *
 * Every call copies mu, phi and w from the caller's host arrays into the
 * scratch with cudaMemcpyAsync on `stream`.  The first call on a device
 * looks up the device address of the scratch array (once per device, with
 * that device current); make that first call before any stream capture.  All calls share the one array and it keeps
 * the last call's contents, so calls whose GPU work may overlap (several
 * streams, several host threads) race with each other: serialise them. */
#define RT_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int rt_formal_solution_noalloc(int nx, int ny, int nz, double dx, double dy, double dz,
                               int top_mode, int bottom_mode, int ndir, const double *mu,
                               const double *phi, const double *w, const double *chi,
                               const double *S, const double *B, double *J_fs, void *stream);

/* ---- Batched wavelengths ------------------------------------------------
 *
 * Many monochromatic problems (wavelength points), each its own 3DRT
 * problem with its own grid, chi, eps and B, share one quadrature and
 * boundary modes and are solved together: every outer iteration runs the
 * formal solutions of all unconverged problems in ONE launch (RT_FP32_SWEEP;
 * RT_FP64 launches per problem), then their Jacobi sweeps, then their
 * convergence tests; a problem leaves the iteration when its own delta
 * drops below tol.  The paper solves one wavelength at a time on the GPU
 * (Sect. 2); this is the batched form of the same per-wavelength solve, and
 * each problem's iterates are the ones rt_solve would produce for it. */
typedef struct {
    int nx, ny, nz;             /* grid of this problem (same rules as rt_set_grid) */
    double dx, dy, dz;
    const double *chi;          /* host [nz][ny][nx], > 0 */
    const double *eps;          /* host, in (0, 1] */
    const double *B;            /* host */
} rt_problem;

typedef struct rt_batch rt_batch;

/* Create a batch of nprob problems on `device` (precision RT_FP32_SWEEP or
 * RT_FP64), copying every problem's fields to the device and building its
 * tables.  *batch receives a handle whenever the arguments are usable, also
 * when creation then fails (read rt_batch_last_error, then destroy it). */
int rt_batch_create(rt_batch **batch, int device, int precision, int nprob,
                    const rt_problem *probs, int top_mode, int bottom_mode, int ndir,
                    const double *mu, const double *phi, const double *w);
int rt_batch_destroy(rt_batch *batch);
const char *rt_batch_last_error(const rt_batch *batch);
/* Run all work on `stream` (NULL: the batch's own stream). */
int rt_batch_set_stream(rt_batch *batch, void *stream);
/* Restart every problem from J = B; rebuild_lstar != 0 also rebuilds
 * Lambda* (and the OS coefficients) at the next iteration. */
int rt_batch_reset(rt_batch *batch, int rebuild_lstar);
/* Switch every problem between RT_FP32_SWEEP and RT_DF64 (rt_set_precision)
 * and start a new stage from the current iterates: iteration counts, deltas
 * and convergence flags restart, J and Lambda* are kept.  The FP32 stage runs
 * as one fused launch per iteration, the double-float stage as one launch per
 * problem. */
int rt_batch_set_precision(rt_batch *batch, int precision);
/* As rt_set_df_finish, for every problem of the batch. */
int rt_batch_set_df_finish(rt_batch *batch, double delta_switch);
/* Iterate until every problem has delta < tol or max_iter iterations.
 * iters[nprob], deltas[nprob] (host, may be NULL) receive each problem's
 * iteration count and last delta; *n_converged the number converged.
 * Returns RT_ENOTCONV if some problem did not converge (outputs valid). */
int rt_batch_solve(rt_batch *batch, double tol, int max_iter, double tol_inner, int max_sweeps,
                   int *iters, double *deltas, int *n_converged);
/* J of problem p into host (get_J) or device (get_J_dev) memory. */
int rt_batch_get_J(rt_batch *batch, int p, double *J);
int rt_batch_get_J_dev(rt_batch *batch, int p, double *J);
/* As rt_set_direction_groups, for the fused launch (0 = auto). */
int rt_batch_set_direction_groups(rt_batch *batch, int groups);
/* As rt_set_block_threads, for the fused FP32 launch. */
int rt_batch_set_block_threads(rt_batch *batch, int threads);
/* As rt_set_block_order, for every problem of the fused FP32 launch. */
int rt_batch_set_block_order(rt_batch *batch, int order);
/* Recorded formal solutions in a batch (see rt_set_fs_record): every
 * problem records its march in its first formal solution and replays it
 * afterwards (FP32 sweep: all replays in one fused launch), exactly as a
 * single solve does, so the batch's iterates stay bit-identical to single
 * solves.  A problem starts iterating once its recording fits in the
 * budget beside the recordings held (max_bytes: -1 (default) 60% of the
 * device, while what the unconverged problems still allocate at their
 * finishing stage and 4 GiB stay free; 0 no recordings; > 0 a byte
 * limit), and returns the memory when
 * it converges or reaches max_iter; problems run in waves when the budget
 * holds fewer than all (65^3 x 1024 directions, FP32 sweep: 39 GB each).
 * A problem whose recording could never fit marches from the start.
 * Releases the recordings held.  RT_EINVAL for max_bytes < -1. */
int rt_batch_set_fs_record(rt_batch *batch, long long max_bytes);
/* on != 0 (the default): every outer iteration runs the operator-splitting
 * solves of all active problems (Sect. 2.3) as ONE CUDA graph, one
 * independent branch per problem (right-hand side, a device-side loop of
 * sweeps to tol_inner or max_sweeps, the pick of the last sweep's iterate),
 * so the host launches once and waits once per iteration (Ng runs on the
 * device too); the graph is rebuilt when the set of active problems
 * changes.  on == 0: the sweeps are enqueued from the host in growing chunks
 * with one wait per chunk.  Results are identical. */
int rt_batch_set_graphs(rt_batch *batch, int on);
/* As rt_set_ng, for every problem of the batch. */
int rt_batch_set_ng(rt_batch *batch, int period, double min_delta);
/* As rt_set_os_method, for every problem of the batch. */
int rt_batch_set_os_method(rt_batch *batch, int method);

/* Checked build (librt3d_checked.so, compiled with RT_CHECKED): the gathers
 * of the formal-solution marches and of the operator-splitting stencils test
 * every index against its buffer; the first index found outside is recorded
 * on the device and the access skipped, and the call that launched the
 * kernel returns RT_EBOUNDS naming the index, the limit and the kernel site
 * (1 FP64 march, 2 its Lambda*, 3 FP32 sweep, 4 double-float march, 5 short
 * characteristics, 6 their Lambda*, 7 parabolic march, 8 its Lambda*,
 * 9 Jacobi stencil, 10 Gauss-Seidel stencil).  Results of such a call are
 * not valid.  rt_checked_build() says which library is loaded;
 * rt_bounds_selftest(ctx) runs one guard on an index never dereferenced
 * (site 99): RT_EBOUNDS in the checked build, RT_OK otherwise. */
int rt_checked_build(void);
int rt_bounds_selftest(rt_ctx *ctx);

/* Scheduling of the FP64 march launches (linear and parabolic source).
 * Their thread blocks are dispatched plane by plane over all direction
 * slots, heaviest plane first, so that the light planes fill the end of a
 * launch (the hardware hands out blocks in index order).  The FP32-sweep
 * and double-float marches keep the planes in index order: reading the
 * plane from the order table slowed the FP32 march by a third.  A
 * plane's work is estimated, whenever the opacity is set, by marching the
 * plane means of chi up and down to an optical depth of 40 or the boundary
 * at |mu| = 1, 1/2 and 1/5.  The order changes no result: every voxel and
 * direction slot is computed by the same thread code whatever the order.
 * rt_get_plane_order copies it (nz ints, order[r] = plane of rank r) to
 * host memory; RT_ESTATE before the opacity is set. */
int rt_get_plane_order(rt_ctx *ctx, int *order);

/* Counters of this context since the last rt_reset_stats: kernel launches,
 * formal-solution march launches and their device time, Jacobi sweeps and
 * their device time, march steps executed.  Device times are measured with
 * CUDA events recorded on the context's stream around those kernels, and
 * only while profiling is on (rt_set_profiling); the other counters are
 * always kept. */
typedef struct {
    unsigned long long launches;        /* all kernels of this library */
    unsigned long long fs_launches;     /* formal-solution march kernels */
    double fs_ms;                       /* their summed device time (profiling on) */
    unsigned long long jacobi_launches; /* Jacobi sweep kernels */
    double jacobi_ms;                   /* their summed device time (profiling on) */
    unsigned long long steps;           /* march steps executed */
    unsigned long long lstar_launches;  /* Lambda* builds */
    unsigned long long iterations;      /* outer iterations of rt_solve / rt_batch_solve */
    unsigned long long host_syncs;      /* host waits for the stream inside those solves */
} rt_stats;

int rt_set_profiling(rt_ctx *ctx, int on);
int rt_get_stats(rt_ctx *ctx, rt_stats *out);
int rt_reset_stats(rt_ctx *ctx);
/* The same counters for a batch (fs_ms: device time of the fused launches). */
int rt_batch_set_profiling(rt_batch *batch, int on);
int rt_batch_get_stats(rt_batch *batch, rt_stats *out);
int rt_batch_reset_stats(rt_batch *batch);

#ifdef __cplusplus
}
#endif
#endif /* RT3D_H */
