// Parabolic (second-order) source variant of the FP64 long-characteristics
// march and its Lambda*.  On segment m (from p_{m+1} to p_m, optical depth
// a) S is the quadratic through S(p_{m+1}), S(p_m), S(p_{m-1}) in the
// optical depth t measured upstream from p_m, the last node at t = -b
// (b the optical depth of segment m-1).  With E_n = int_0^a t^n e^{-t} dt,
//   P_up   = (E2 + b E1) / (a (a + b)),
//   P_cur  = (a b E0 - (b - a) E1 - E2) / (a b),
//   P_down = (E2 - a E1) / (b (a + b)),
// and I += T (P_up S(p_{m+1}) + P_cur S(p_m) + P_down S(p_{m-1})).  For
// m = 0 the downstream point p_{-1} = (i0 + ax, j0 + ay, k0 + s) is used when
// plane k0 + s exists, else segment 0 keeps the linear weights.
//
// Moments: E_n = n! e^{-a} sum_{k>n} a^k / k!.  Below a = 1 the tail sums
// are formed by Horner from their positive series (no cancellation), above
// it from E0 = 1 - e, E1 = E0 - a e, E2 = 2 E1 - a^2 e.
#include "internal.h"
#include "weights.cuh"

namespace rt3d {

namespace {

constexpr int kThreadsP = 128;

__device__ __forceinline__ int wrap_mod_p(long long a, int n)
{
    long long r = a % n;
    return (int)(r < 0 ? r + n : r);
}

struct NodesP {
    int a00, a10, a01, a11;
};

__device__ __forceinline__ NodesP nodes_p(int i0, int j0, int ox, int oy, int nx, int ny)
{
    int x0 = i0 + ox;
    x0 -= x0 >= nx ? nx : 0;
    const int x1 = x0 + 1 == nx ? 0 : x0 + 1;
    int y0 = j0 + oy;
    y0 -= y0 >= ny ? ny : 0;
    const int y1 = y0 + 1 == ny ? 0 : y0 + 1;
    return NodesP{y0 * nx + x0, y0 * nx + x1, y1 * nx + x0, y1 * nx + x1};
}

__device__ __forceinline__ int nmin_p(NodesP n) { return min(min(n.a00, n.a10), min(n.a01, n.a11)); }
__device__ __forceinline__ int nmax_p(NodesP n) { return max(max(n.a00, n.a10), max(n.a01, n.a11)); }

__device__ __forceinline__ double bilin_p(const double* __restrict__ f, NodesP n, Bw4d b)
{
    return b.x * __ldg(f + n.a00) + b.y * __ldg(f + n.a10) + b.z * __ldg(f + n.a01) +
           b.w * __ldg(f + n.a11);
}

// Parabolic weights of a segment of optical depth a whose downstream
// neighbour segment has optical depth b; e = e^{-a}.
__device__ __forceinline__ void para_weights64(double a, double b, const double* __restrict__ tab,
                                               double& pu, double& pc, double& pd, double& e)
{
    e = a <= 700.0 ? exp_neg_tang(a, tab) : 0.0;
    double E0, E1, E2;
    if (a < 1.0) {
        // T2 = sum_{k>=3} a^k/k! (through k = 18: truncation < 1e-16 relative)
        double h = 1.0 / 6402373705728000.0;                      // 1/18!
        h = fma(h, a, 1.0 / 355687428096000.0);                    // 1/17!
        h = fma(h, a, 1.0 / 20922789888000.0);
        h = fma(h, a, 1.0 / 1307674368000.0);
        h = fma(h, a, 1.0 / 87178291200.0);
        h = fma(h, a, 1.0 / 6227020800.0);
        h = fma(h, a, 1.0 / 479001600.0);
        h = fma(h, a, 1.0 / 39916800.0);
        h = fma(h, a, 1.0 / 3628800.0);
        h = fma(h, a, 1.0 / 362880.0);
        h = fma(h, a, 1.0 / 40320.0);
        h = fma(h, a, 1.0 / 5040.0);
        h = fma(h, a, 1.0 / 720.0);
        h = fma(h, a, 1.0 / 120.0);
        h = fma(h, a, 1.0 / 24.0);
        h = fma(h, a, 1.0 / 6.0);                                  // 1/3!
        const double a2 = a * a;
        const double T2 = h * a2 * a;
        const double T1 = fma(0.5, a2, T2);
        const double T0 = a + T1;
        E0 = e * T0;
        E1 = e * T1;
        E2 = 2.0 * e * T2;
    } else {
        E0 = 1.0 - e;
        E1 = E0 - a * e;
        E2 = 2.0 * E1 - a * a * e;
    }
    const double r = recip_newton(a * b * (a + b));
    pu = (E2 + b * E1) * b * r;
    pc = (a * b * E0 - (b - a) * E1 - E2) * (a + b) * r;
    pd = (E2 - a * E1) * a * r;
}

__global__ void k_down_tables(Geometry g, double dx, double dy, double dz,
                              const double* __restrict__ mu, const double* __restrict__ phi,
                              DownGeo* __restrict__ dn)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= g.ndir) return;
    const double m_u = mu[d];
    const double amu = fabs(m_u);
    const double sint = sqrt(1.0 - m_u * m_u);
    const double X = (dz / dx) * sint * cos(phi[d]) / amu;   // downstream point: +ax, +ay
    const double Y = (dz / dy) * sint * sin(phi[d]) / amu;
    const double fX = floor(X), fY = floor(Y);
    const double tx = X - fX, ty = Y - fY;
    DownGeo q;
    q.b = Bw4d{(1.0 - tx) * (1.0 - ty), tx * (1.0 - ty), (1.0 - tx) * ty, tx * ty};
    q.ox = wrap_mod_p((long long)fX, g.nx);
    q.oy = wrap_mod_p((long long)fY, g.ny);
    const int oz = m_u > 0.0 ? 1 : -1;                        // plane k0 + s
    for (int c = 0; c < 4; ++c) {
        const int rx = wrap_mod_p((long long)fX + (c & 1), g.nx);
        const int ry = wrap_mod_p((long long)fY + (c >> 1), g.ny);
        const int ox = rx == 0 ? 0 : rx == 1 ? 1 : rx == g.nx - 1 ? -1 : 9;
        const int oy = ry == 0 ? 0 : ry == 1 ? 1 : ry == g.ny - 1 ? -1 : 9;
        q.ld[c] = (ox == 9 || oy == 9) ? -1 : (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1);
    }
    dn[d] = q;
}

__device__ __forceinline__ void add_steps_p(unsigned long long* steps, unsigned long long n)
{
    for (int s = 16; s > 0; s >>= 1) n += __shfl_down_sync(0xffffffffu, n, s);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(steps, n);
}

// Same decomposition as the linear march (one thread per voxel, 8 direction
// slots summed in fixed order into partial[slot]).
//
// REC: also record the march as a linear map of S (FsRec).  Segment m adds
// T_m P_up to the coefficient of S(p_{m+1}), T_m P_cur to p_m's and T_m
// P_down to p_{m-1}'s (the first segment without a downstream point: the
// linear weights), so p_{m-1}'s coefficient is complete after segment m:
// p_{-1}'s goes to cdn, p_0's to the per-voxel c0, p_m's (m >= 1) to coef.
template <bool REC>
__global__ void __launch_bounds__(kThreadsP)
k_fs64p(Geometry g, const double* __restrict__ chi, const double* __restrict__ S,
        const double* __restrict__ B, const double* __restrict__ G,
        const DirInfo* __restrict__ info, const StepGeo* __restrict__ off,
        const Bw4d* __restrict__ bw, const DownGeo* __restrict__ dn,
        const double* __restrict__ smax_p, double cut, double* __restrict__ partial,
        unsigned long long* __restrict__ steps, FsRec rec)
{
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const int t = blockIdx.x * kThreadsP + threadIdx.x;
    const int k0 = plane_at(g, blockIdx.z), zb = blockIdx.y, ZB = gridDim.y;
    const bool active = t < nxy;
    __shared__ double tab[kExpTable];
    fill_exp_table(tab);
    __syncthreads();
    const unsigned amask = __ballot_sync(0xffffffffu, active);
    unsigned long long nsteps = 0;
    if (active) {
        const int j0 = t / nx, i0 = t - j0 * nx;
        const long long v = (long long)k0 * nxy + t;
        // parabolic weights exceed the linear ones in magnitude by a small
        // factor: 4 more bits of margin in the transmission cutoff
        const int need = cut_need(*smax_p, REC ? cut * kRecCutMargin : cut) + 4;
        const double chi0 = chi[v], S0 = S[v];
        for (int slot = zb; slot < kSlots; slot += ZB) {
            double Jp = 0.0, C0 = 0.0, Bc = 0.0;
            for (int d = slot; d < g.ndir; d += kSlots) {
                const DirInfo di = info[d];
                const int s = di.sgn;
                const int M = s > 0 ? k0 : nz - 1 - k0;
                const StepGeo* od = off + (long long)d * nz;
                const Bw4d* bd = bw + (long long)d * nz;
                // downstream point p_{-1}
                const int kd = k0 + s;
                const bool down = kd >= 0 && kd < nz;
                double xprev = 0.0, sprev = 0.0;
                if (down) {
                    const DownGeo q = dn[d];
                    NodesP n = nodes_p(i0, j0, q.ox, q.oy, nx, ny);
                    RT_GUARD(g, nmax_p(n), nxy, kSiteFs64p) n = NodesP{0, 0, 0, 0};
                    RT_GUARD(g, nmin_p(n), nxy, kSiteFs64p) n = NodesP{0, 0, 0, 0};
                    const long long pd = (long long)kd * nxy;
                    xprev = di.hs * (chi0 + bilin_p(chi + pd, n, q.b));
                    sprev = bilin_p(S + pd, n, q.b);
                }
                double I = 0.0, T = 1.0, ca = chi0, sa = S0;
                // REC: pending coefficients of p_{m-1}, p_m and p_{m+1}
                double* rc = REC ? rec.coef + rec_base(g, d, k0, s) + t : nullptr;
                double pm1 = 0.0, p0 = 0.0, p1 = 0.0;
                bool early = false;
                int m = 0;
                for (; m < M; ++m) {
                    const long long pb = (long long)(k0 - (m + 1) * s) * nxy;
                    const StepGeo o = od[m + 1];
                    const NodesP n = nodes_p(i0, j0, o.ox, o.oy, nx, ny);
                    RT_GUARD(g, pb + nmax_p(n), g.N, kSiteFs64p) { early = true; break; }
                    RT_GUARD(g, pb + nmin_p(n), g.N, kSiteFs64p) { early = true; break; }
                    const Bw4d b = bd[m + 1];
                    const double cb = bilin_p(chi + pb, n, b);
                    const double sb = bilin_p(S + pb, n, b);
                    const double x = di.hs * (ca + cb);
                    double e;
                    if (m == 0 && !down) {
                        double wc, wu;
                        seg_weights64(x, tab, wc, wu, e);
                        I = fma(T, fma(wc, sa, wu * sb), I);
                        if (REC) {
                            p0 += wc;
                            p1 += wu;
                        }
                    } else {
                        double pu, pc, pdn;
                        para_weights64(x, xprev, tab, pu, pc, pdn, e);
                        I = fma(T, fma(pu, sb, fma(pc, sa, pdn * sprev)), I);
                        if (REC) {
                            p1 = fma(T, pu, p1);
                            p0 = fma(T, pc, p0);
                            pm1 = fma(T, pdn, pm1);
                        }
                    }
                    if (REC) {
                        // p_{m-1} is complete
                        if (m == 0) rec.cdn[(long long)d * g.N + v] = pm1;
                        else if (m == 1) C0 = fma(di.w, pm1, C0);
                        else rc[(long long)(m - 2) * nxy] = pm1;
                        pm1 = p0;
                        p0 = p1;
                        p1 = 0.0;
                    }
                    T *= e;
                    xprev = x;
                    sprev = sa;
                    ca = cb;
                    sa = sb;
                    if (cut_now(T, I, need)) {
                        early = true;
                        ++m;
                        break;
                    }
                }
                const int bc = s > 0 ? g.top_bc : g.bottom_bc;
                if (!early && bc) {
                    const long long pb = (long long)(k0 - M * s) * nxy;
                    const StepGeo o = od[M];
                    const NodesP n = nodes_p(i0, j0, o.ox, o.oy, nx, ny);
                    double ibc = bilin_p(B + pb, n, bd[M]);
                    if (bc == 2) ibc = fma(di.amu, bilin_p(G, n, bd[M]), ibc);
                    I = fma(T, ibc, I);
                    if (REC) Bc = fma(di.w, T * ibc, Bc);
                }
                if (REC) {
                    // the last two points (p_{m-1}, p_m); then zeros up to
                    // the warp's longest ray
                    if (m == 0) {
                        rec.cdn[(long long)d * g.N + v] = 0.0;
                    } else {
                        if (m == 1) C0 = fma(di.w, pm1, C0);
                        else rc[(long long)(m - 2) * nxy] = pm1;
                        rc[(long long)(m - 1) * nxy] = p0;
                    }
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
    if (steps) add_steps_p(steps, nsteps);
}

// Lambda* under the parabolic source.  With T_1 = e_0, T_2 = e_0 e_1 and
// segment weights (P_up, P_cur, P_down)_m, the coefficient of S at
//   p_{-1}: P_down(0)
//   p_0:    P_cur(0) + T_1 P_down(1)
//   p_1:    P_up(0) + T_1 P_cur(1) + T_2 P_down(2)
// (terms of segments that do not exist dropped); p_{-1} lies on plane
// k0 + s, p_1 on k0 - s, farther points outside the neighbourhood.
__global__ void __launch_bounds__(kThreadsP)
k_lstar64p(Geometry g, const double* __restrict__ chi, const DirInfo* __restrict__ info,
           const StepGeo* __restrict__ off, const Bw4d* __restrict__ bw,
           const DownGeo* __restrict__ dn, double* __restrict__ lstar)
{
    __shared__ double lam[27][kThreadsP];
    __shared__ double tab[kExpTable];
    for (int q = 0; q < 27; ++q) lam[q][threadIdx.x] = 0.0;
    fill_exp_table(tab);
    __syncthreads();
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const int t = blockIdx.x * kThreadsP + threadIdx.x;
    const int k0 = blockIdx.y;
    if (t >= nxy) return;
    const int j0 = t / nx, i0 = t - j0 * nx;
    const long long v = (long long)k0 * nxy + t;
    const double chi0 = chi[v];
    for (int d = 0; d < g.ndir; ++d) {
        const DirInfo di = info[d];
        const int s = di.sgn;
        const int M = s > 0 ? k0 : nz - 1 - k0;
        const int kd = k0 + s;
        const bool down = kd >= 0 && kd < nz;
        if (M == 0 && !down) continue;
        const StepGeo* od = off + (long long)d * nz;
        const Bw4d* bd = bw + (long long)d * nz;
        // optical depths of segments -1 .. 2 (those that exist)
        double xm1 = 0.0, x0 = 0.0, x1 = 0.0, x2 = 0.0;
        const DownGeo q = dn[d];
        if (down) {
            const NodesP n = nodes_p(i0, j0, q.ox, q.oy, nx, ny);
            xm1 = di.hs * (chi0 + bilin_p(chi + (long long)kd * nxy, n, q.b));
        }
        double chi1 = 0.0, chi2 = 0.0;
        if (M >= 1) {
            const NodesP n = nodes_p(i0, j0, od[1].ox, od[1].oy, nx, ny);
            chi1 = bilin_p(chi + (long long)(k0 - s) * nxy, n, bd[1]);
            x0 = di.hs * (chi0 + chi1);
        }
        if (M >= 2) {
            const NodesP n = nodes_p(i0, j0, od[2].ox, od[2].oy, nx, ny);
            chi2 = bilin_p(chi + (long long)(k0 - 2 * s) * nxy, n, bd[2]);
            x1 = di.hs * (chi1 + chi2);
        }
        if (M >= 3) {
            const NodesP n = nodes_p(i0, j0, od[3].ox, od[3].oy, nx, ny);
            x2 = di.hs * (chi2 + bilin_p(chi + (long long)(k0 - 3 * s) * nxy, n, bd[3]));
        }
        double cm1 = 0.0, c0 = 0.0, c1 = 0.0;
        if (M >= 1) {
            double u0, w0, d0, e0;
            if (down) {
                para_weights64(x0, xm1, tab, u0, w0, d0, e0);
            } else {
                seg_weights64(x0, tab, w0, u0, e0);
                d0 = 0.0;
            }
            cm1 = d0;
            c0 = w0;
            c1 = u0;
            if (M >= 2) {
                double u1, w1, d1, e1;
                para_weights64(x1, x0, tab, u1, w1, d1, e1);
                c0 = fma(e0, d1, c0);
                c1 = fma(e0, w1, c1);
                if (M >= 3) {
                    double u2, w2, d2, e2;
                    para_weights64(x2, x1, tab, u2, w2, d2, e2);
                    c1 = fma(e0 * e1, d2, c1);
                }
            }
        }
        lam[13][threadIdx.x] += di.w * c0;
        if (M >= 1) {
            const Bw4d b1 = bd[1];
            const double cw = di.w * c1;
            if (di.lo[0] >= 0) lam[di.lo[0]][threadIdx.x] += cw * b1.x;
            if (di.lo[1] >= 0) lam[di.lo[1]][threadIdx.x] += cw * b1.y;
            if (di.lo[2] >= 0) lam[di.lo[2]][threadIdx.x] += cw * b1.z;
            if (di.lo[3] >= 0) lam[di.lo[3]][threadIdx.x] += cw * b1.w;
        }
        if (down) {
            const double cw = di.w * cm1;
            if (q.ld[0] >= 0) lam[q.ld[0]][threadIdx.x] += cw * q.b.x;
            if (q.ld[1] >= 0) lam[q.ld[1]][threadIdx.x] += cw * q.b.y;
            if (q.ld[2] >= 0) lam[q.ld[2]][threadIdx.x] += cw * q.b.z;
            if (q.ld[3] >= 0) lam[q.ld[3]][threadIdx.x] += cw * q.b.w;
        }
    }
    for (int o = 0; o < 27; ++o) lstar[(long long)o * g.N + v] = lam[o][threadIdx.x];
}

}  // namespace

cudaError_t launch_down_tables(const Geometry& g, double dx, double dy, double dz,
                               const double* mu, const double* phi, DownGeo* dn, cudaStream_t st)
{
    k_down_tables<<<(g.ndir + 127) / 128, 128, 0, st>>>(g, dx, dy, dz, mu, phi, dn);
    return cudaGetLastError();
}

cudaError_t launch_fs64p(const Geometry& g, const double* chi, const double* S, const double* B,
                         const double* G, const DirInfo* info, const StepGeo* off,
                         const Bw4d* bw, const DownGeo* dn, const double* smax, double cut,
                         int groups, double* partial, unsigned long long* steps, cudaStream_t st,
                         const FsRec* rec)
{
    const int nxy = g.nx * g.ny;
    dim3 grid((nxy + kThreadsP - 1) / kThreadsP, groups, g.nz);
    if (rec)
        k_fs64p<true><<<grid, kThreadsP, 0, st>>>(g, chi, S, B, G, info, off, bw, dn, smax, cut,
                                                  partial, steps, *rec);
    else
        k_fs64p<false><<<grid, kThreadsP, 0, st>>>(g, chi, S, B, G, info, off, bw, dn, smax, cut,
                                                   partial, steps, FsRec{});
    return cudaGetLastError();
}

cudaError_t launch_lstar64p(const Geometry& g, const double* chi, const DirInfo* info,
                            const StepGeo* off, const Bw4d* bw, const DownGeo* dn, double* lstar,
                            cudaStream_t st)
{
    const int nxy = g.nx * g.ny;
    dim3 grid((nxy + kThreadsP - 1) / kThreadsP, g.nz, 1);
    k_lstar64p<<<grid, kThreadsP, 0, st>>>(g, chi, info, off, bw, dn, lstar);
    return cudaGetLastError();
}

}  // namespace rt3d
