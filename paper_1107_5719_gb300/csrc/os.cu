// Operator splitting (Hauschildt & Baron 2011, Sect. 2.3), source update
// and the max-reductions of the convergence tests.
//
// The new J solves (1 - Lambda* D) J_new = J_fs - Lambda* D J_old with
// D = diag(1 - eps).  Jacobi ("Jordan") form, with the coefficients of the
// 27-band operator precomputed once per (chi, eps):
//   diag_v  = 1 - Lambda*_{v,13} (1 - eps_v)
//   c_{v,o} = Lambda*_{v,o} (1 - eps_{nb(v,o)}) / diag_v
//   r_v     = J_fs,v / diag_v - sum_o c_{v,o} J_old,nb(v,o)
//   J^{n+1}_v = r_v + sum_{o != 13} c_{v,o} J^n_{nb(v,o)}
// The coefficients are stored offset-major ([27][N]) so that a warp reads
// 32 consecutive voxels of one offset (coalesced).
//
// Red-black Gauss-Seidel (the other method of Sect. 2.3): voxel (i,j,k) is
// red if i+j+k is even.  A sweep is two launches: the red voxels from the
// iterate at the start of the sweep, then the black voxels from the new red
// and the old black values; within a colour the updates are simultaneous,
// so each launch reads only values no thread of it writes.  For this method
// c, 1/diag and r are stored colour-split, [colour][nz][ny][h] with
// h = ceil(nx/2) and the voxel at x = 2q + ((colour + j + k) & 1) at q, so
// that a warp of one colour still reads 32 consecutive coefficients.  Max-reductions of
// non-negative doubles use atomicMax on their bit patterns, which order
// like the values; max is independent of the order, so results are
// reproducible.
#include "internal.h"

namespace rt3d {

namespace {

__device__ __forceinline__ void block_max_to(double val, double* out)
{
    // val >= 0 or NaN; NaN must win so that a broken iterate never "converges".
    __shared__ unsigned long long sm[32];
    unsigned long long b = (unsigned long long)__double_as_longlong(val);
    for (int s = 16; s > 0; s >>= 1) {
        const unsigned long long o = __shfl_down_sync(0xffffffffu, b, s);
        b = o > b ? o : b;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = b;
    __syncthreads();
    if (wid == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        b = lane < nw ? sm[lane] : 0ull;
        for (int s = 16; s > 0; s >>= 1) {
            const unsigned long long o = __shfl_down_sync(0xffffffffu, b, s);
            b = o > b ? o : b;
        }
        if (lane == 0 && b) atomicMax((unsigned long long*)out, b);
    }
}

__device__ __forceinline__ double nonneg(double x)
{
    return fabs(x);  // clears the sign bit of NaN too
}

// |a - b| / |a| for the inner convergence test of the sweeps, as |a - b|
// times 1/|a| from the hardware reciprocal seed and two Newton steps
// instead of an IEEE division, which on GB300 (where the FP64 pipe bounds
// the sweep) took about a third of the sweep's FP64 instructions.  The
// product is within a few units in the last place of the quotient, so the
// stopping decision differs from an exact one only where the relative
// change lies within ~1e-15 of the tolerance.  NaN propagates; a zero a
// gives inf or NaN, never a false "converged".
__device__ __forceinline__ double rel_change(double a, double b)
{
    const double d = fabs(a);
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    return fabs(a - b) * r;
}

__global__ void k_source(long long N, const double* __restrict__ eps, const double* __restrict__ B,
                         const double* __restrict__ J, double* __restrict__ S,
                         float* __restrict__ S32, const double* __restrict__ Bbound,
                         double* __restrict__ smax)
{
    double m = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
        const double e = eps[v];
        const double s = fma(e, B[v], (1.0 - e) * J[v]);
        S[v] = s;
        if (S32) S32[v] = (float)s;
        double a = nonneg(s);
        if (Bbound) a = fmax(a, nonneg(Bbound[v]));
        if (!(a <= m)) m = a;
    }
    block_max_to(m, smax);
}

__global__ void k_absmax(long long N, const double* __restrict__ S, const double* __restrict__ B,
                         double* __restrict__ smax, float* __restrict__ S32)
{
    double m = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
        const double s = S[v];
        if (S32) S32[v] = (float)s;
        double a = nonneg(s);
        if (B) a = fmax(a, nonneg(B[v]));
        if (!(a <= m)) m = a;
    }
    block_max_to(m, smax);
}

__global__ void k_to_float(long long N, const double* __restrict__ x, float* __restrict__ y)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x)
        y[v] = (float)x[v];
}

// Neighbour (ox, oy, oz) of voxel (i, j, k) with periodic x, y.
__device__ __forceinline__ int wrap1(int a, int n)
{
    return a < 0 ? a + n : (a >= n ? a - n : a);
}

constexpr int kOsThreads = 128;

// Colour-split storage: h = ceil(nx/2) slots per row and colour.
__device__ __host__ __forceinline__ int split_h(int nx) { return (nx + 1) >> 1; }

__device__ __forceinline__ long long split_index(const Geometry& g, int i, int j, int k)
{
    const int col = (i + j + k) & 1;
    return (((long long)col * g.nz + k) * g.ny + j) * split_h(g.nx) + (i >> 1);
}

// Coefficient storage size per offset: N ([27][N]) or the colour-split size.
__device__ __host__ __forceinline__ long long coef_stride(const Geometry& g, bool split)
{
    return split ? 2LL * g.nz * g.ny * split_h(g.nx) : g.N;
}

template <bool SPLIT>
__global__ void __launch_bounds__(kOsThreads)
k_os_coef(Geometry g, const double* __restrict__ L, const double* __restrict__ eps,
          double* __restrict__ c, double* __restrict__ rdiag)
{
    const int nx = g.nx, ny = g.ny, nxy = nx * ny;
    const int t = blockIdx.x * kOsThreads + threadIdx.x;
    const int k = blockIdx.y;
    if (t >= nxy) return;
    const int j = t / nx, i = t - j * nx;
    const long long v = (long long)k * nxy + t;
    const long long ci = SPLIT ? split_index(g, i, j, k) : v;
    const long long cs = coef_stride(g, SPLIT);
    const double rd = 1.0 / (1.0 - L[13 * g.N + v] * (1.0 - eps[v]));
    rdiag[ci] = rd;
    for (int o = 0; o < 27; ++o) {
        const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
        const int kk = k + oz;
        double cv = 0.0;
        if (kk >= 0 && kk < g.nz) {
            const long long nb = (long long)kk * nxy + wrap1(j + oy, ny) * nx + wrap1(i + ox, nx);
            cv = L[o * g.N + v] * (1.0 - eps[nb]) * rd;
        }
        c[o * cs + ci] = cv;
    }
}

// sum_o c[o][v] * J[nb(v,o)] over the offsets, skipping the centre if
// SKIP_CENTRE and planes outside the grid.
template <bool SKIP_CENTRE>
__device__ __forceinline__ double stencil(const Geometry& g, const double* __restrict__ c,
                                          const double* __restrict__ J, int i, int j, int k,
                                          long long v, long long cs)
{
    const int nx = g.nx, ny = g.ny, nxy = nx * ny;
    const int xm = wrap1(i - 1, nx), xp = wrap1(i + 1, nx);
    const int ym = wrap1(j - 1, ny), yp = wrap1(j + 1, ny);
    const int xs[3] = {xm, i, xp};
    const int ys[3] = {ym, j, yp};
    double acc = 0.0;
#pragma unroll
    for (int oz = 0; oz < 3; ++oz) {
        const int kk = k + oz - 1;
        if (kk < 0 || kk >= g.nz) continue;
        const double* Jp = J + (long long)kk * nxy;
#pragma unroll
        for (int oy = 0; oy < 3; ++oy) {
            const double* Jr = Jp + ys[oy] * nx;
#pragma unroll
            for (int ox = 0; ox < 3; ++ox) {
                const int o = oz * 9 + oy * 3 + ox;
                if (SKIP_CENTRE && o == 13) continue;
                RT_GUARD(g, (Jr - J) + xs[ox], g.N, kSiteStencil) continue;
                RT_GUARD(g, o * cs + v, 27 * cs, kSiteStencil) continue;
                acc = fma(__ldg(c + o * cs + v), __ldg(Jr + xs[ox]), acc);
            }
        }
    }
    return acc;
}

template <bool SPLIT>
__global__ void __launch_bounds__(kOsThreads)
k_os_rhs(Geometry g, const double* __restrict__ c, const double* __restrict__ rdiag,
         const double* __restrict__ Jfs, const double* __restrict__ Jold, double* __restrict__ r)
{
    const int nx = g.nx, nxy = nx * g.ny;
    const int t = blockIdx.x * kOsThreads + threadIdx.x;
    const int k = blockIdx.y;
    if (t >= nxy) return;
    const int j = t / nx, i = t - j * nx;
    const long long v = (long long)k * nxy + t;
    const long long ci = SPLIT ? split_index(g, i, j, k) : v;
    r[ci] = Jfs[v] * rdiag[ci] - stencil<false>(g, c, Jold, i, j, k, ci, coef_stride(g, SPLIT));
}

// Sweep n of a Jacobi solve.  dlt[n] receives max |Jn - J| / |Jn|; if the
// previous sweep already met the tolerance (dlt[n-1] < tol) the sweep does
// nothing, so a host loop may enqueue several sweeps per check without
// changing the result.  dlt must be zeroed before sweep 0.
//
// With nsw != null the sweep index is *nsw + n (a device-side counter: the
// sweep loop of a CUDA graph), and sweeps at or past max_sweeps do nothing.
__global__ void __launch_bounds__(kOsThreads)
k_jacobi(Geometry g, const double* __restrict__ c, const double* __restrict__ r,
         const double* __restrict__ J, double* __restrict__ Jn, double* __restrict__ dlt, int n,
         double tol, const int* __restrict__ nsw, int max_sweeps)
{
    if (nsw) {
        n += *nsw;
        if (n >= max_sweeps) return;
    }
    if (n > 0 && dlt[n - 1] < tol) return;
    double* delta = dlt + n;
    const int nx = g.nx, nxy = nx * g.ny;
    const int t = blockIdx.x * kOsThreads + threadIdx.x;
    const int k = blockIdx.y;
    double rel = 0.0;
    if (t < nxy) {
        const int j = t / nx, i = t - j * nx;
        const long long v = (long long)k * nxy + t;
        const double jn = r[v] + stencil<true>(g, c, J, i, j, k, v, g.N);
        Jn[v] = jn;
        rel = rel_change(jn, J[v]);
    }
    block_max_to(rel, delta);
}

// Half of sweep n of a red-black Gauss-Seidel solve: the voxels of one
// colour, from `same` for neighbours of that colour (the iterate at the
// start of the sweep) and from `other` for the rest (the start iterate for
// the red half, the new red values for the black half), written to `dst`.
// dst == other in the black half: this launch reads only the other colour's
// entries of it and writes only its own.  Same no-op rule as k_jacobi.
__global__ void __launch_bounds__(kOsThreads)
k_gs_half(Geometry g, const double* __restrict__ c, const double* __restrict__ r,
          const double* __restrict__ same, const double* other, double* dst,
          double* __restrict__ dlt, int n, double tol, int colour,
          const int* __restrict__ nsw, int max_sweeps)
{
    if (nsw) {
        n += *nsw;
        if (n >= max_sweeps) return;
    }
    if (n > 0 && dlt[n - 1] < tol) return;
    const int nx = g.nx, ny = g.ny, nxy = nx * ny, h = split_h(nx);
    const int t = blockIdx.x * kOsThreads + threadIdx.x;
    const int k = blockIdx.y;
    const int j = t / h, q = t - j * h;
    const int i = 2 * q + ((colour + j + k) & 1);
    double rel = 0.0;
    if (j < ny && i < nx) {
        const long long cs = coef_stride(g, true);
        const long long ci = (((long long)colour * g.nz + k) * ny + j) * h + q;
        const long long v = (long long)k * nxy + (long long)j * nx + i;
        const int xm = wrap1(i - 1, nx), xp = wrap1(i + 1, nx);
        const int ym = wrap1(j - 1, ny), yp = wrap1(j + 1, ny);
        const int xs[3] = {xm, i, xp};
        const int ys[3] = {ym, j, yp};
        double acc = r[ci];
#pragma unroll
        for (int oz = 0; oz < 3; ++oz) {
            const int kk = k + oz - 1;
            if (kk < 0 || kk >= g.nz) continue;
#pragma unroll
            for (int oy = 0; oy < 3; ++oy) {
                const long long row = (long long)kk * nxy + (long long)ys[oy] * nx;
#pragma unroll
                for (int ox = 0; ox < 3; ++ox) {
                    const int o = oz * 9 + oy * 3 + ox;
                    if (o == 13) continue;
                    const int x = xs[ox];
                    RT_GUARD(g, row + x, g.N, kSiteGs) continue;
                    RT_GUARD(g, o * cs + ci, 27 * cs, kSiteGs) continue;
                    const double* src = ((x + ys[oy] + kk) & 1) == colour ? same : other;
                    acc = fma(__ldg(c + o * cs + ci), __ldg(src + row + x), acc);
                }
            }
        }
        dst[v] = acc;
        rel = rel_change(acc, same[v]);
    }
    block_max_to(rel, dlt + n);
}

// End of one pass of the graph's sweep loop (two sweeps): advance the
// counter and continue while sweeps remain and the last one had not met
// the tolerance.
__global__ void k_sweep_cond(cudaGraphConditionalHandle h, int* nsw, const double* __restrict__ dlt,
                             int max_sweeps, double tol)
{
    const int n = *nsw + 2;
    *nsw = n;
    const bool more = n < max_sweeps && !(dlt[n - 1] < tol);
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// End of a device-side sweep loop: the solve stopped at the first sweep n
// whose dlt[n] < tol (all sweeps when none did), and that sweep wrote Ja
// (n even) or Jb (n odd): copy it to Jn and record the sweep count.  Every
// block finds the count itself (the deltas are a few hundred doubles).
__global__ void k_os_select(long long N, const double* __restrict__ dlt, int max_sweeps,
                            double tol, const double* __restrict__ Ja,
                            const double* __restrict__ Jb, double* __restrict__ Jn,
                            int* __restrict__ sweeps_out)
{
    __shared__ int s_sweeps;
    if (threadIdx.x == 0) {
        int s = max_sweeps;
        for (int n = 0; n < max_sweeps; ++n)
            if (dlt[n] < tol) {
                s = n + 1;
                break;
            }
        s_sweeps = s;
        if (blockIdx.x == 0 && sweeps_out) *sweeps_out = s;
    }
    __syncthreads();
    const double* src = ((s_sweeps - 1) & 1) ? Jb : Ja;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x)
        Jn[v] = src[v];
}

__global__ void k_rel_change(long long N, const double* __restrict__ Jn,
                             const double* __restrict__ Jo, double* __restrict__ delta)
{
    double m = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
        const double a = nonneg((Jn[v] - Jo[v]) / Jn[v]);
        if (!(a <= m)) m = a;
    }
    block_max_to(m, delta);
}

// ---- Ng acceleration --------------------------------------------------------
// Second-order Ng extrapolation of the outer iterates x0 (newest) .. x3:
// the five weighted sums of the 2x2 least-squares system (weights 1/x0^2)
// are reduced in a fixed order (fixed grid, fixed per-thread strides, fixed
// tree), so the extrapolation is reproducible.
constexpr int kNgBlocks = 1024, kNgThreads = 256;

__global__ void __launch_bounds__(kNgThreads)
k_ng_dots(long long N, const double* __restrict__ x0, const double* __restrict__ x1,
          const double* __restrict__ x2, const double* __restrict__ x3, double* __restrict__ part)
{
    double s[5] = {0, 0, 0, 0, 0};
    for (long long i = blockIdx.x * (long long)kNgThreads + threadIdx.x; i < N;
         i += (long long)kNgBlocks * kNgThreads) {
        const double d0 = x0[i] - x1[i], d1 = x1[i] - x2[i], d2 = x2[i] - x3[i];
        const double q1 = d0 - d1, q2 = d0 - d2;
        const double w = 1.0 / (x0[i] * x0[i]);
        s[0] += w * q1 * q1;
        s[1] += w * q1 * q2;
        s[2] += w * q2 * q2;
        s[3] += w * d0 * q1;
        s[4] += w * d0 * q2;
    }
    __shared__ double sm[5][kNgThreads];
    for (int k = 0; k < 5; ++k) sm[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int h = kNgThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int k = 0; k < 5; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 5) part[blockIdx.x * 5 + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void __launch_bounds__(kNgThreads)
k_ng_sum(const double* __restrict__ part, double* __restrict__ out)
{
    double s[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < kNgBlocks; b += kNgThreads)
        for (int k = 0; k < 5; ++k) s[k] += part[b * 5 + k];
    __shared__ double sm[5][kNgThreads];
    for (int k = 0; k < 5; ++k) sm[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int h = kNgThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int k = 0; k < 5; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 5) out[threadIdx.x] = sm[threadIdx.x][0];
}

// The Ng extrapolation with its 2x2 least-squares system solved on the
// device from the five sums s5 = {a11, a12, a22, b1, b2} (every thread
// solves it; products and differences rounded separately, as written):
// x0 <- (1 - a - b) x0 + a x1 + b x2, left unchanged when the system is
// singular (|det| <= 1e-300) or not finite.
__global__ void k_ng_apply(long long N, const double* __restrict__ s5,
                           const double* __restrict__ x1, const double* __restrict__ x2,
                           double* __restrict__ x0)
{
    const double s0 = s5[0], s1 = s5[1], s2 = s5[2], s3 = s5[3], s4 = s5[4];
    const double det = __dsub_rn(__dmul_rn(s0, s2), __dmul_rn(s1, s1));
    if (!(fabs(det) > 1e-300) || det != det) return;
    const double a = __ddiv_rn(__dsub_rn(__dmul_rn(s3, s2), __dmul_rn(s4, s1)), det);
    const double b = __ddiv_rn(__dsub_rn(__dmul_rn(s4, s0), __dmul_rn(s3, s1)), det);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        x0[i] = (1.0 - a - b) * x0[i] + a * x1[i] + b * x2[i];
}

unsigned grid_1d(long long N, int threads)
{
    long long b = (N + threads - 1) / threads;
    if (b > 152LL * 32) b = 152LL * 32;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

cudaError_t launch_source(long long N, const double* eps, const double* B, const double* J,
                          double* S, float* S32, const double* Bbound, double* smax,
                          cudaStream_t st)
{
    k_source<<<grid_1d(N, 256), 256, 0, st>>>(N, eps, B, J, S, S32, Bbound, smax);
    return cudaGetLastError();
}

cudaError_t launch_absmax(long long N, const double* S, const double* B, double* smax,
                          float* S32, cudaStream_t st)
{
    k_absmax<<<grid_1d(N, 256), 256, 0, st>>>(N, S, B, smax, S32);
    return cudaGetLastError();
}

cudaError_t launch_to_float(long long N, const double* x, float* y, cudaStream_t st)
{
    k_to_float<<<grid_1d(N, 256), 256, 0, st>>>(N, x, y);
    return cudaGetLastError();
}

long long os_coef_stride(const Geometry& g, bool split) { return coef_stride(g, split); }

cudaError_t launch_os_coef(const Geometry& g, const double* lstar, const double* eps,
                           double* coef, double* rdiag, bool split, cudaStream_t st)
{
    dim3 grid((g.nx * g.ny + kOsThreads - 1) / kOsThreads, g.nz);
    if (split)
        k_os_coef<true><<<grid, kOsThreads, 0, st>>>(g, lstar, eps, coef, rdiag);
    else
        k_os_coef<false><<<grid, kOsThreads, 0, st>>>(g, lstar, eps, coef, rdiag);
    return cudaGetLastError();
}

cudaError_t launch_os_rhs(const Geometry& g, const double* coef, const double* rdiag,
                          const double* J_fs, const double* J_old, double* r, bool split,
                          cudaStream_t st)
{
    dim3 grid((g.nx * g.ny + kOsThreads - 1) / kOsThreads, g.nz);
    if (split)
        k_os_rhs<true><<<grid, kOsThreads, 0, st>>>(g, coef, rdiag, J_fs, J_old, r);
    else
        k_os_rhs<false><<<grid, kOsThreads, 0, st>>>(g, coef, rdiag, J_fs, J_old, r);
    return cudaGetLastError();
}

cudaError_t launch_gs_sweep(const Geometry& g, const double* coef, const double* r,
                            const double* J, double* Jn, double* dlt, int n, double tol,
                            cudaStream_t st)
{
    dim3 grid((g.ny * split_h(g.nx) + kOsThreads - 1) / kOsThreads, g.nz);
    k_gs_half<<<grid, kOsThreads, 0, st>>>(g, coef, r, J, J, Jn, dlt, n, tol, 0, nullptr, 0);
    k_gs_half<<<grid, kOsThreads, 0, st>>>(g, coef, r, J, Jn, Jn, dlt, n, tol, 1, nullptr, 0);
    return cudaGetLastError();
}

cudaError_t launch_sweep_pass(const Geometry& g, const double* coef, const double* r, double* b0,
                              double* b1, double* dlt, int* nsw, int max_sweeps, double tol,
                              bool gs, cudaGraphConditionalHandle h, cudaStream_t st)
{
    // sweep *nsw: b1 -> b0; sweep *nsw + 1: b0 -> b1
    if (gs) {
        dim3 grid((g.ny * split_h(g.nx) + kOsThreads - 1) / kOsThreads, g.nz);
        k_gs_half<<<grid, kOsThreads, 0, st>>>(g, coef, r, b1, b1, b0, dlt, 0, tol, 0, nsw, max_sweeps);
        k_gs_half<<<grid, kOsThreads, 0, st>>>(g, coef, r, b1, b0, b0, dlt, 0, tol, 1, nsw, max_sweeps);
        k_gs_half<<<grid, kOsThreads, 0, st>>>(g, coef, r, b0, b0, b1, dlt, 1, tol, 0, nsw, max_sweeps);
        k_gs_half<<<grid, kOsThreads, 0, st>>>(g, coef, r, b0, b1, b1, dlt, 1, tol, 1, nsw, max_sweeps);
    } else {
        dim3 grid((g.nx * g.ny + kOsThreads - 1) / kOsThreads, g.nz);
        k_jacobi<<<grid, kOsThreads, 0, st>>>(g, coef, r, b1, b0, dlt, 0, tol, nsw, max_sweeps);
        k_jacobi<<<grid, kOsThreads, 0, st>>>(g, coef, r, b0, b1, dlt, 1, tol, nsw, max_sweeps);
    }
    k_sweep_cond<<<1, 1, 0, st>>>(h, nsw, dlt, max_sweeps, tol);
    return cudaGetLastError();
}

cudaError_t launch_os_select(long long N, const double* dlt, int max_sweeps, double tol,
                             const double* Ja, const double* Jb, double* Jn, int* sweeps_out,
                             cudaStream_t st)
{
    long long blocks = (N + 255) / 256;
    if (blocks > 152LL * 8) blocks = 152LL * 8;
    k_os_select<<<(unsigned)blocks, 256, 0, st>>>(N, dlt, max_sweeps, tol, Ja, Jb, Jn, sweeps_out);
    return cudaGetLastError();
}

cudaError_t launch_jacobi(const Geometry& g, const double* coef, const double* r,
                          const double* J, double* Jn, double* dlt, int n, double tol,
                          cudaStream_t st)
{
    dim3 grid((g.nx * g.ny + kOsThreads - 1) / kOsThreads, g.nz);
    k_jacobi<<<grid, kOsThreads, 0, st>>>(g, coef, r, J, Jn, dlt, n, tol, nullptr, 0);
    return cudaGetLastError();
}

int ng_partial_size() { return kNgBlocks * 5; }

cudaError_t launch_ng_dots(long long N, const double* x0, const double* x1, const double* x2,
                           const double* x3, double* part, double* out5, cudaStream_t st)
{
    k_ng_dots<<<kNgBlocks, kNgThreads, 0, st>>>(N, x0, x1, x2, x3, part);
    k_ng_sum<<<1, kNgThreads, 0, st>>>(part, out5);
    return cudaGetLastError();
}

cudaError_t launch_ng_apply(long long N, const double* s5, const double* x1, const double* x2,
                            double* x0, cudaStream_t st)
{
    k_ng_apply<<<grid_1d(N, 256), 256, 0, st>>>(N, s5, x1, x2, x0);
    return cudaGetLastError();
}

cudaError_t launch_rel_change(long long N, const double* Jn, const double* Jo, double* delta,
                              cudaStream_t st)
{
    k_rel_change<<<grid_1d(N, 256), 256, 0, st>>>(N, Jn, Jo, delta);
    return cudaGetLastError();
}

}  // namespace rt3d
