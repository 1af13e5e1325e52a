// Formal solution kernels (Hauschildt & Baron 2011, Sect. 2.2): geometry
// tables, the gather-form march along the characteristics, its recording as
// a linear map of the source and the replay of that recording, the J
// reduction over directions and the nearest-neighbour Lambda*.
//
// Design (GB300).  The paper tracks every characteristic from the boundary
// planes in a 2D kernel and collects per-voxel results in a second pass
// with integer atomics, because OpenCL 1.x has no floating-point atomics
// (Sect. 2.2).  Here each thread owns one voxel and integrates I back
// along the characteristic of each of its directions, one z-plane per step.
// Because voxel centres are lattice points, the upstream point of step m
// has the same lattice offset and bilinear weights for every voxel of a
// direction; they are tabulated once per (direction, step) and read as
// warp-uniform broadcasts.  The 32 lanes of a warp are 32 consecutive
// voxels of one plane, so at every step they read 32 consecutive nodes of
// the same upstream plane (coalesced, mostly L1 hits) and run identical
// loop bounds.  Each thread sums its directions in fixed order; direction
// groups (grid z) are then summed in fixed order, so J is bit-reproducible
// without atomics on floating-point data.
#include "internal.h"
#include "weights.cuh"

#include <cmath>

namespace rt3d {

namespace {

constexpr int kThreads = 128;

__device__ __forceinline__ int wrap_mod(long long a, int n)
{
    long long r = a % n;
    return (int)(r < 0 ? r + n : r);
}

__global__ void k_dir_tables(Geometry g, double dx, double dy, double dz,
                             const double* __restrict__ mu, const double* __restrict__ phi,
                             const double* __restrict__ w, DirInfo* __restrict__ info,
                             StepGeo* __restrict__ off, Bw4d* __restrict__ bw,
                             Bw4d* __restrict__ bwh, float4* __restrict__ bw32)
{
    const int d = blockIdx.x;
    const double m_u = mu[d];
    const double amu = fabs(m_u);
    const double hs = dz / (2.0 * amu);
    const double sint = sqrt(1.0 - m_u * m_u);
    const double ax = (dz / dx) * sint * cos(phi[d]) / amu;
    const double ay = (dz / dy) * sint * sin(phi[d]) / amu;
    for (int m = threadIdx.x; m < g.nz; m += blockDim.x) {
        const double X = -(double)m * ax, Y = -(double)m * ay;
        const double fX = floor(X), fY = floor(Y);
        const double tx = X - fX, ty = Y - fY;
        StepGeo o;
        o.ox = wrap_mod((long long)fX, g.nx);
        o.oy = wrap_mod((long long)fY, g.ny);
        const long long e = (long long)d * g.nz + m;
        off[e] = o;
        const Bw4d b = Bw4d{(1.0 - tx) * (1.0 - ty), tx * (1.0 - ty), (1.0 - tx) * ty, tx * ty};
        bw[e] = b;
        bwh[e] = Bw4d{hs * b.x, hs * b.y, hs * b.z, hs * b.w};
        bw32[e] = make_float4((float)b.x, (float)b.y, (float)b.z, (float)b.w);
    }
    if (threadIdx.x == 0) {
        DirInfo di;
        di.hs = hs;
        di.hs32 = (float)di.hs;
        di.amu = amu;
        di.amu32 = (float)amu;
        di.hs32lo = (float)(di.hs - (double)di.hs32);
        di.amu32lo = (float)(amu - (double)di.amu32);
        di.w = w[d];
        di.w32 = (float)di.w;
        di.sgn = m_u > 0.0 ? 1 : -1;
        // Lambda* offsets of the four nodes of p_1 (plane k0 - sgn).
        const long long ix = (long long)floor(-ax), iy = (long long)floor(-ay);
        const int oz = -di.sgn;
        for (int q = 0; q < 4; ++q) {
            const int rx = wrap_mod(ix + (q & 1), g.nx), ry = wrap_mod(iy + (q >> 1), g.ny);
            const int ox = rx == 0 ? 0 : rx == 1 ? 1 : rx == g.nx - 1 ? -1 : 9;
            const int oy = ry == 0 ? 0 : ry == 1 ? 1 : ry == g.ny - 1 ? -1 : 9;
            di.lo[q] = (ox == 9 || oy == 9 || g.nz < 2) ? -1 : (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1);
        }
        info[d] = di;
    }
}

struct Nodes {
    int a00, a10, a01, a11;
};

__device__ __forceinline__ Nodes nodes_of(int i0, int j0, StepGeo o, int nx, int ny)
{
    int x0 = i0 + o.ox;
    x0 -= (x0 >= nx) ? nx : 0;
    int x1 = x0 + 1;
    x1 = (x1 == nx) ? 0 : x1;
    int y0 = j0 + o.oy;
    y0 -= (y0 >= ny) ? ny : 0;
    int y1 = y0 + 1;
    y1 = (y1 == ny) ? 0 : y1;
    return Nodes{y0 * nx + x0, y0 * nx + x1, y1 * nx + x0, y1 * nx + x1};
}

// Extremes of the four node indices (checked builds test both).
__device__ __forceinline__ int nodes_min(Nodes n) { return min(min(n.a00, n.a10), min(n.a01, n.a11)); }
__device__ __forceinline__ int nodes_max(Nodes n) { return max(max(n.a00, n.a10), max(n.a01, n.a11)); }

template <typename T, typename V4>
__device__ __forceinline__ T bilin(const T* __restrict__ p, Nodes n, V4 b)
{
    return b.x * __ldg(p + n.a00) + b.y * __ldg(p + n.a10) + b.z * __ldg(p + n.a01) +
           b.w * __ldg(p + n.a11);
}

__device__ __forceinline__ void add_steps(unsigned long long* steps, unsigned long long n)
{
    for (int s = 16; s > 0; s >>= 1) n += __shfl_down_sync(0xffffffffu, n, s);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(steps, n);
}

// One thread per voxel of plane plane_at(g, blockIdx.z).  Direction d
// belongs to slot d mod kSlots; each slot is summed in increasing d and
// written to partial[slot]; block y walks slots zb, zb + gridDim.y, ...
// The slot sums are then added in slot order, so J depends neither on
// gridDim.y nor on the plane dispatch order.
//
// REC: also record the march as a linear map of S (the recorded operator,
// FsRec): per (voxel, direction) the coefficient c_m of S(p_m), m >= 1,
//   c_m = T_{m-1} w_up,{m-1} + T_m w_cur,m   (the last point: T_{L-1} w_up),
// and per voxel and slot the coefficient of S at the voxel itself,
// sum_d w_d w_cur,0, and the boundary term sum_d w_d T_L I_bc (rays that
// reach the boundary plane); partial is not written (J comes from the
// replay).  The march runs to the stricter cutoff cut * kRecCutMargin, so
// that later sources, whose intensities may be smaller, still meet the
// cutoff with the recorded lengths.
template <bool REC>
__global__ void __launch_bounds__(kThreads)
k_fs64(Geometry g, const double* __restrict__ chi, const double* __restrict__ S,
       const double* __restrict__ B, const double* __restrict__ G,
       const DirInfo* __restrict__ info,
       const StepGeo* __restrict__ off, const Bw4d* __restrict__ bw,
       const Bw4d* __restrict__ bwh, const double* __restrict__ smax_p, double cut,
       double* __restrict__ partial, unsigned long long* __restrict__ steps, FsRec rec)
{
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const int t = blockIdx.x * kThreads + threadIdx.x;
    const int k0 = plane_at(g, blockIdx.z), zb = blockIdx.y, ZB = gridDim.y;
    const bool active = t < nxy;
    __shared__ double tab[kExpTable];
    fill_exp_table(tab);
    __syncthreads();
    // lanes of this warp holding a voxel (the recorded lengths are per warp)
    const unsigned amask = __ballot_sync(0xffffffffu, active);
    unsigned long long nsteps = 0;
    if (active) {
        const int j0 = t / nx, i0 = t - j0 * nx;
        const long long v = (long long)k0 * nxy + t;
        const int need = REC ? cut_need(*smax_p, cut * kRecCutMargin) : cut_need(*smax_p, cut);
        const double chi0 = chi[v], S0 = S[v];
        for (int slot = zb; slot < kSlots; slot += ZB) {
            double Jp = 0.0, C0 = 0.0, Bc = 0.0;
            for (int d = slot; d < g.ndir; d += kSlots) {
                const DirInfo di = info[d];
                const int s = di.sgn;
                const int M = s > 0 ? k0 : nz - 1 - k0;
                const StepGeo* od = off + (long long)d * nz;
                const Bw4d* bd = bw + (long long)d * nz;
                const Bw4d* bh = bwh + (long long)d * nz;
                double* rc = REC ? rec.coef + rec_base(g, d, k0, s) + t : nullptr;
                // ca, cb: chi times the half path length hs, so that a
                // segment's optical depth is their sum
                double I = 0.0, T = 1.0, ca = di.hs * chi0, sa = S0, cprev = 0.0;
                bool early = false;
                int m = 0;
                for (; m < M; ++m) {
                    const long long pb = (long long)(k0 - (m + 1) * s) * nxy;
                    const Nodes n = nodes_of(i0, j0, od[m + 1], nx, ny);
                    RT_GUARD(g, pb + nodes_min(n), g.N, kSiteFs64) { early = true; break; }
                    RT_GUARD(g, pb + nodes_max(n), g.N, kSiteFs64) { early = true; break; }
                    const double cb = bilin(chi + pb, n, bh[m + 1]);
                    const double sb = bilin(S + pb, n, bd[m + 1]);
                    double wc, wu, e;
                    seg_weights64(ca + cb, tab, wc, wu, e);
                    if (REC) {
                        if (m == 0) C0 = fma(di.w, wc, C0);
                        else rc[(long long)(m - 1) * nxy] = fma(T, wc, cprev);
                        cprev = T * wu;
                    }
                    I = fma(T, fma(wc, sa, wu * sb), I);
                    T *= e;
                    ca = cb;
                    sa = sb;
                    if (cut_now(T, I, need)) {
                        early = true;
                        ++m;
                        break;
                    }
                }
                const int bc = s > 0 ? g.top_bc : g.bottom_bc;
                bool bc_ok = true;
                if (!early && bc) {
                    const long long pb = (long long)(k0 - M * s) * nxy;
                    const Nodes n = nodes_of(i0, j0, od[M], nx, ny);
                    RT_GUARD(g, pb + nodes_max(n), g.N, kSiteFs64) bc_ok = false;
                    RT_GUARD(g, pb + nodes_min(n), g.N, kSiteFs64) bc_ok = false;
                }
                if (!early && bc && bc_ok) {
                    const long long pb = (long long)(k0 - M * s) * nxy;
                    const Nodes n = nodes_of(i0, j0, od[M], nx, ny);
                    double ibc = bilin(B + pb, n, bd[M]);
                    if (bc == 2) ibc = fma(di.amu, bilin(G, n, bd[M]), ibc);  // B + |mu| dB/dtau
                    I = fma(T, ibc, I);
                    if (REC) Bc = fma(di.w, T * ibc, Bc);
                }
                if (REC) {
                    // the last point's coefficient, then zeros up to the
                    // warp's longest ray (the replay runs that many steps)
                    if (m > 0) rc[(long long)(m - 1) * nxy] = cprev;
                    const int Lw = __reduce_max_sync(amask, m);
                    for (int q = m; q < Lw; ++q) rc[(long long)q * nxy] = 0.0;
                    if ((threadIdx.x & 31) == __ffs(amask) - 1)
                        rec.lmax[((long long)d * nz + k0) * rec.nwp + (t >> 5)] = Lw;
                }
                nsteps += (unsigned long long)m;
                Jp = fma(di.w, I, Jp);
            }
            if (REC) {
                rec.c0[(long long)slot * g.N + v] = C0;
                rec.bc[(long long)slot * g.N + v] = Bc;
            } else {
                partial[(long long)slot * g.N + v] = Jp;
            }
        }
    }
    if (steps) add_steps(steps, nsteps);
}

// Replay of the recorded march (FsRec) for a new source S: per (voxel,
// direction) I = sum_m c_m S(p_m) over the warp's recorded length (and,
// for the parabolic source, c_-1 S(p_-1) at the downstream point), plus
// per slot the voxel's own term and the boundary term.  Five FP64
// operations per step (the bilinear interpolation of S and one FMA)
// against ~32 for the march, and 8 coefficient bytes streamed from memory.
__global__ void __launch_bounds__(kThreads)
k_fs64rep(Geometry g, const double* __restrict__ S, const DirInfo* __restrict__ info,
          const StepGeo* __restrict__ off, const Bw4d* __restrict__ bw, FsRec rec,
          double* __restrict__ partial, unsigned long long* __restrict__ steps)
{
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const int t = blockIdx.x * kThreads + threadIdx.x;
    const int k0 = plane_at(g, blockIdx.z), zb = blockIdx.y, ZB = gridDim.y;
    unsigned long long nsteps = 0;
    if (t < nxy) {
        const int j0 = t / nx, i0 = t - j0 * nx;
        const long long v = (long long)k0 * nxy + t;
        const double S0 = S[v];
        const double* __restrict__ coef = rec.coef;
        for (int slot = zb; slot < kSlots; slot += ZB) {
            double Jp = fma(rec.c0[(long long)slot * g.N + v], S0, rec.bc[(long long)slot * g.N + v]);
            for (int d = slot; d < g.ndir; d += kSlots) {
                const DirInfo di = info[d];
                const int s = di.sgn;
                const StepGeo* od = off + (long long)d * nz;
                const Bw4d* bd = bw + (long long)d * nz;
                const double* rc = coef + rec_base(g, d, k0, s) + t;
                const int L = rec.lmax[((long long)d * nz + k0) * rec.nwp + (t >> 5)];
                double I = 0.0;
                if (rec.cdn) {   // parabolic source: the downstream point p_-1
                    const int kd = k0 + s;
                    if (kd >= 0 && kd < nz) {
                        const DownGeo q = rec.dn[d];
                        const Nodes n = nodes_of(i0, j0, StepGeo{q.ox, q.oy}, nx, ny);
                        RT_GUARD(g, nodes_max(n), nxy, kSiteFs64) continue;
                        I = rec.cdn[(long long)d * g.N + v] * bilin(S + (long long)kd * nxy, n, q.b);
                    }
                }
                for (int m = 0; m < L; ++m) {
                    const long long pb = (long long)(k0 - (m + 1) * s) * nxy;
                    const Nodes n = nodes_of(i0, j0, od[m + 1], nx, ny);
                    RT_GUARD(g, pb + nodes_min(n), g.N, kSiteFs64) break;
                    RT_GUARD(g, pb + nodes_max(n), g.N, kSiteFs64) break;
                    I = fma(__ldcs(rc + (long long)m * nxy), bilin(S + pb, n, bd[m + 1]), I);
                }
                nsteps += (unsigned long long)L;
                Jp = fma(di.w, I, Jp);
            }
            partial[(long long)slot * g.N + v] = Jp;
        }
    }
    if (steps) add_steps(steps, nsteps);
}

// Mean of chi over each plane (block k: plane k), fixed summation order.
__global__ void k_plane_mean(Geometry g, const double* __restrict__ chi, double* __restrict__ mean)
{
    __shared__ double red[256];
    const int nxy = g.nx * g.ny;
    const double* pk = chi + (long long)blockIdx.x * nxy;
    double s = 0.0;
    for (int t = threadIdx.x; t < nxy; t += 256) s += pk[t];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) mean[blockIdx.x] = red[0] / nxy;
}

// Estimated march work of every plane (w[k]) and the planes by decreasing
// work (order[rank] = plane).  One block.
__global__ void k_plane_rank(int nz, double dz, const double* __restrict__ mean,
                             double* __restrict__ w, int* __restrict__ order)
{
    constexpr double kTauEnd = 40.0;
    const double amu[3] = {1.0, 0.5, 0.2};
    for (int k0 = threadIdx.x; k0 < nz; k0 += blockDim.x) {
        double work = 0.0;
        for (int q = 0; q < 3; ++q) {
            const double hs = dz / (2.0 * amu[q]);
            for (int s = -1; s <= 1; s += 2) {
                double tau = 0.0;
                int n = 1;   // per-characteristic overhead, about one step
                for (int k = k0; k - s >= 0 && k - s < nz && tau <= kTauEnd; k -= s, ++n)
                    tau += hs * (mean[k] + mean[k - s]);
                work += n;
            }
        }
        w[k0] = work;
    }
    __syncthreads();
    for (int k0 = threadIdx.x; k0 < nz; k0 += blockDim.x) {
        int rank = 0;
        for (int j = 0; j < nz; ++j) rank += (w[j] > w[k0]) || (w[j] == w[k0] && j < k0);
        order[rank] = k0;
    }
}

__global__ void k_sum_groups(long long N, const double* __restrict__ partial,
                             double* __restrict__ J)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < kSlots; ++q) s += partial[q * N + v];
        J[v] = s;
    }
}

// Lambda*: the coefficient of S at p_0 is w_cur(0); at p_1 it is
// w_up(0) + e_0 w_cur(1) (just w_up(0) if p_1 is on the boundary).  p_m for
// m >= 2 lies two or more planes away, outside the 27-point neighbourhood.
// The p_1 coefficient is shared among its four bilinear nodes, whose
// neighbour offsets are tabulated per direction.
__global__ void __launch_bounds__(kThreads)
k_lstar64(Geometry g, const double* __restrict__ chi, const DirInfo* __restrict__ info,
          const StepGeo* __restrict__ off, const Bw4d* __restrict__ bw,
          double* __restrict__ lstar)
{
    __shared__ double lam[27][kThreads];
    __shared__ double tab[kExpTable];
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const int t = blockIdx.x * kThreads + threadIdx.x;
    const int k0 = blockIdx.y;
    for (int o = 0; o < 27; ++o) lam[o][threadIdx.x] = 0.0;
    fill_exp_table(tab);
    __syncthreads();
    if (t >= nxy) return;
    const int j0 = t / nx, i0 = t - j0 * nx;
    const long long v = (long long)k0 * nxy + t;
    const double chi0 = chi[v];
    for (int d = 0; d < g.ndir; ++d) {
        const DirInfo di = info[d];
        const int s = di.sgn;
        const int M = s > 0 ? k0 : nz - 1 - k0;
        if (M == 0) continue;
        const StepGeo* od = off + (long long)d * nz;
        const Bw4d* bd = bw + (long long)d * nz;
        const Bw4d b1 = bd[1];
        const Nodes n1 = nodes_of(i0, j0, od[1], nx, ny);
        RT_GUARD(g, (long long)(k0 - s) * nxy + nodes_max(n1), g.N, kSiteLstar64) continue;
        RT_GUARD(g, (long long)(k0 - s) * nxy + nodes_min(n1), g.N, kSiteLstar64) continue;
        const double chi1 = bilin(chi + (long long)(k0 - s) * nxy, n1, b1);
        double wc0, wu0, e0;
        seg_weights64(di.hs * (chi0 + chi1), tab, wc0, wu0, e0);
        double c1 = wu0;
        if (M >= 2) {
            const Nodes n2 = nodes_of(i0, j0, od[2], nx, ny);
            RT_GUARD(g, (long long)(k0 - 2 * s) * nxy + nodes_max(n2), g.N, kSiteLstar64) continue;
            RT_GUARD(g, (long long)(k0 - 2 * s) * nxy + nodes_min(n2), g.N, kSiteLstar64) continue;
            const double chi2 = bilin(chi + (long long)(k0 - 2 * s) * nxy, n2, bd[2]);
            double wc1, wu1, e1;
            seg_weights64(di.hs * (chi1 + chi2), tab, wc1, wu1, e1);
            c1 = fma(e0, wc1, wu0);
        }
        lam[13][threadIdx.x] += di.w * wc0;
        const double cw = di.w * c1;
        if (di.lo[0] >= 0) lam[di.lo[0]][threadIdx.x] += cw * b1.x;
        if (di.lo[1] >= 0) lam[di.lo[1]][threadIdx.x] += cw * b1.y;
        if (di.lo[2] >= 0) lam[di.lo[2]][threadIdx.x] += cw * b1.z;
        if (di.lo[3] >= 0) lam[di.lo[3]][threadIdx.x] += cw * b1.w;
    }
    for (int o = 0; o < 27; ++o) lstar[(long long)o * g.N + v] = lam[o][threadIdx.x];
}

// dB/dtau at the bottom nodes for the LTE-diffusion inner boundary
// (Sect. 3.1 item 4): vertical difference over the trapezoid optical depth
// between the two deepest planes; also the padded FP32 copy.
__global__ void k_diffusion_grad(Geometry g, double dz, const double* __restrict__ chi,
                                 const double* __restrict__ B, double* __restrict__ G,
                                 float* __restrict__ g2)
{
    const int nx = g.nx, ny = g.ny, nxy = nx * ny;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nxy; t += gridDim.x * blockDim.x) {
        const long long a = (long long)(g.nz - 1) * nxy + t, b = (long long)(g.nz - 2) * nxy + t;
        const double v = (B[a] - B[b]) / (dz * (chi[a] + chi[b]) / 2.0);
        G[t] = v;
        if (g2) {
            const int i = t % nx, j = t / nx;
            const long long W = 2LL * nx;
            float* p = g2 + (long long)j * W + i;
            const float f = (float)v;
            p[0] = f;
            p[nx] = f;
            p[(long long)ny * W] = f;
            p[(long long)ny * W + nx] = f;
        }
    }
}

// Diagnostic: the segment weights the marches use, at given optical depths.
__global__ void k_seg_eval(long long n, int fp32, const double* __restrict__ x,
                           double* __restrict__ wc, double* __restrict__ wu,
                           double* __restrict__ e)
{
    __shared__ double tab[kExpTable];
    fill_exp_table(tab);
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (fp32) {
            float a, b, c;
            seg_weights32((float)x[i], a, b, c);
            wc[i] = a; wu[i] = b; e[i] = c;
        } else {
            double a, b, c;
            seg_weights64(x[i], tab, a, b, c);
            wc[i] = a; wu[i] = b; e[i] = c;
        }
    }
}

}  // namespace

cudaError_t launch_dir_tables(const Geometry& g, double dx, double dy, double dz,
                              const double* mu, const double* phi, const double* w,
                              DirInfo* info, StepGeo* off, Bw4d* bw, Bw4d* bwh, float4* bw32,
                              cudaStream_t st)
{
    k_dir_tables<<<g.ndir, 128, 0, st>>>(g, dx, dy, dz, mu, phi, w, info, off, bw, bwh, bw32);
    return cudaGetLastError();
}

cudaError_t launch_plane_order(const Geometry& g, double dz, const double* chi, double* scratch,
                               int* order, cudaStream_t st)
{
    k_plane_mean<<<g.nz, 256, 0, st>>>(g, chi, scratch);
    k_plane_rank<<<1, 256, 0, st>>>(g.nz, dz, scratch, scratch + g.nz, order);
    return cudaGetLastError();
}

cudaError_t launch_fs64(const Geometry& g, const double* chi, const double* S, const double* B,
                        const double* G, const DirInfo* info, const StepGeo* off,
                        const Bw4d* bw, const Bw4d* bwh, const double* smax, double cut,
                        int groups, double* partial, unsigned long long* steps, cudaStream_t st,
                        const FsRec* rec)
{
    const int nxy = g.nx * g.ny;
    dim3 grid((nxy + kThreads - 1) / kThreads, groups, g.nz);
    if (rec)
        k_fs64<true><<<grid, kThreads, 0, st>>>(g, chi, S, B, G, info, off, bw, bwh, smax, cut,
                                                partial, steps, *rec);
    else
        k_fs64<false><<<grid, kThreads, 0, st>>>(g, chi, S, B, G, info, off, bw, bwh, smax, cut,
                                                 partial, steps, FsRec{});
    return cudaGetLastError();
}

cudaError_t launch_fs64rep(const Geometry& g, const double* S, const DirInfo* info,
                           const StepGeo* off, const Bw4d* bw, const FsRec& rec, int groups,
                           double* partial, unsigned long long* steps, cudaStream_t st)
{
    const int nxy = g.nx * g.ny;
    dim3 grid((nxy + kThreads - 1) / kThreads, groups, g.nz);
    k_fs64rep<<<grid, kThreads, 0, st>>>(g, S, info, off, bw, rec, partial, steps);
    return cudaGetLastError();
}

long long rec_bytes(const Geometry& g)
{
    const long long nxy = (long long)g.nx * g.ny;
    const long long nwp = (nxy + 31) / 32;
    return (long long)g.ndir * nxy * ((long long)g.nz * (g.nz - 1) / 2) * (long long)sizeof(double) +
           (long long)g.ndir * g.nz * nwp * (long long)sizeof(int) +
           2LL * kSlots * g.N * (long long)sizeof(double);
}

namespace {
__global__ void k_bounds_selftest(Geometry g)
{
    RT_GUARD(g, g.N, g.N, kSiteSelfTest) return;
}
}  // namespace

cudaError_t launch_bounds_selftest(const Geometry& g, cudaStream_t st)
{
    k_bounds_selftest<<<1, 1, 0, st>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_sum_groups(long long N, const double* partial, double* J,
                              cudaStream_t st)
{
    const int threads = 256;
    long long blocks = (N + threads - 1) / threads;
    if (blocks > 65535LL * 16) blocks = 65535LL * 16;
    k_sum_groups<<<(unsigned)blocks, threads, 0, st>>>(N, partial, J);
    return cudaGetLastError();
}

cudaError_t launch_diffusion_grad(const Geometry& g, double dz, const double* chi,
                                  const double* B, double* G, float* g2, cudaStream_t st)
{
    const int nxy = g.nx * g.ny;
    k_diffusion_grad<<<(nxy + 255) / 256, 256, 0, st>>>(g, dz, chi, B, G, g2);
    return cudaGetLastError();
}

cudaError_t launch_seg_eval(long long n, int fp32, const double* x, double* wc, double* wu,
                            double* e, cudaStream_t st)
{
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_seg_eval<<<(unsigned)blocks, 256, 0, st>>>(n, fp32, x, wc, wu, e);
    return cudaGetLastError();
}

cudaError_t launch_lstar64(const Geometry& g, const double* chi, const DirInfo* info,
                           const StepGeo* off, const Bw4d* bw, double* lstar,
                           cudaStream_t st)
{
    const int nxy = g.nx * g.ny;
    dim3 grid((nxy + kThreads - 1) / kThreads, g.nz, 1);
    k_lstar64<<<grid, kThreads, 0, st>>>(g, chi, info, off, bw, lstar);
    return cudaGetLastError();
}

}  // namespace rt3d
