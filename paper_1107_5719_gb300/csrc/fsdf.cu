// FP64-accurate formal solution in double-float arithmetic (precision
// RT_DF64).  Same characteristics, interpolation, optical depths, segment
// weights and cutoff as the FP64 march (Hauschildt & Baron 2011, Sect. 2.2),
// but every quantity is an unevaluated pair of FP32 numbers (df.cuh), so the
// march runs on the FP32 pipes, which issue 64x more operations per clock on
// GB300 than the FP64 pipe.  Like the FP32 sweep it integrates I - S_0 (the
// deviation from the source at the voxel), so that its ~1e-14 relative
// rounding scales with I - S_0 and is not amplified by the near-singular
// scattering problem at small eps.
//
// Sums use Dekker's add (df_add_s): its error bound, ~2^-47 times the sum of
// the operands' magnitudes, is the level at which the operands themselves
// are known (chi, S, the table entries and the bilinear weights each carry
// a 2^-48 representation error), so the accurate add would buy nothing.
//
// Layout: per node a float4 {chi_hi, chi_lo, S_hi, S_lo} in planes padded to
// 2ny x 2nx by periodic copies (same addressing as the FP32 sweep); bilinear
// weights per (direction, step) as two float4 (hi and lo parts); boundary B
// and the LTE-diffusion gradient as padded float2 pairs.
#include "df.cuh"
#include "internal.h"

namespace rt3d {

namespace {

constexpr int kThreadsDF = 128;
constexpr int kExpTableDF = 256;

// tab[j] = 2^{-j/256} and tab[256 + j] = 1 - 2^{-j/256} (the latter from
// expm1, so accurate relative to itself), as double-float pairs (call from
// all threads, then sync)
__device__ __forceinline__ void fill_exp_table_df(dfl* tab)
{
    for (int j = threadIdx.x; j < kExpTableDF; j += blockDim.x) {
        tab[j] = df_from_double(exp2(-(double)j / kExpTableDF));
        tab[kExpTableDF + j] = df_from_double(-expm1(-(double)j * (0.693147180559945309417 / kExpTableDF)));
    }
}

// e^{-x} and 1 - e^{-x} for 0.05 <= x <= 80 (Tang's table-driven method in
// double-float): k = round(256 x / ln2), m = k >> 8, j = k & 255,
// r = x - k ln2/256 (|r| <= 1.4e-3, ln2/256 split into three floats as in
// Cody & Waite, the products formed exactly), p = e^{-r} - 1 =
// -r + r^2/2 - r^3 (1/6 - r/24) (the cubic and quartic terms in FP32,
// < 5e-10), and with t = 2^{-m} 2^{-j/256}:
//   e = t + t p,   1 - e = (1 - t) - t p.
// For m = 0 the factor 1 - t comes from its own table (1 - e would
// otherwise inherit the table's rounding relative to e, which cancels);
// for m >= 1, t <= 1/2 and 1 - t loses nothing.
__device__ __forceinline__ void exp_neg_df(dfl x, const dfl* __restrict__ tab, dfl& e, dfl& om)
{
    constexpr float kInvL = 369.3299255371094f;          // 256 / ln 2 (rounding only)
    constexpr float kL1 = 0.0027076061815023422f;         // ln2/256 = kL1 + kL2 + kL3
    constexpr float kL2 = -7.440055516116928e-12f;
    constexpr float kL3 = -3.4309311478864607e-19f;
    const float k = rintf(x.h * kInvL);
    dfl r = df_add_s(x, df_neg(two_prod(k, kL1)));
    r = df_add_s(r, df_neg(two_prod(k, kL2)));
    r = df_add_f(r, -k * kL3);
    const dfl r2 = df_mul(r, r);
    const float tail = r2.h * r.h * fmaf(-r.h, 1.0f / 24.0f, 1.0f / 6.0f);
    const dfl p = df_add_s(df_neg(r), df_add_f(df_scale(r2, 0.5f), -tail));
    const int ki = (int)k;
    const int m = ki >> 8, j = ki & (kExpTableDF - 1);
    const float sc = __int_as_float((127 - m) << 23);   // 2^-m, normal for x <= 80
    const dfl t = df_scale(tab[j], sc);
    const dfl tp = df_mul(t, p);
    const dfl c = m == 0 ? tab[kExpTableDF + j] : df_add_f(df_neg(t), 1.0f);
    e = df_add_s(t, tp);
    om = df_sub_s(c, tp);
}

// Segment weights in double-float (same definitions as weights.cuh).
__device__ __forceinline__ void seg_weights_df(dfl x, const dfl* __restrict__ tab, dfl& wc, dfl& wu,
                                               dfl& e)
{
    if (x.h < 0.05f) {
        // phi2 series: E = 1/2 + z/24 + z^2/720 + ..., O = x (1/6 + z/120 + z^2/5040 + ...);
        // from z^2 on the terms are below 9e-9 and are summed in FP32.
        const dfl z = df_mul(x, x);
        const float zf = z.h;
        const float rE = zf * zf * fmaf(zf, fmaf(zf, 1.0f / 3628800.0f, 1.0f / 40320.0f), 1.0f / 720.0f);
        const float rO = zf * zf * fmaf(zf, 1.0f / 362880.0f, 1.0f / 5040.0f);
        const dfl c24 = df_make(0.0416666679084301f, -1.2417634698280722e-09f);    // 1/24
        const dfl c120 = df_make(0.008333333767950535f, -4.34617203337595e-10f);   // 1/120
        const dfl c6 = df_make(0.1666666716337204f, -4.967053879312289e-09f);      // 1/6
        dfl E = df_add_f(df_mul(z, c24), rE);
        E = df_add_f(E, 0.5f);
        dfl Op = df_add_f(df_mul(z, c120), rO);
        Op = df_add_s(c6, Op);
        const dfl O = df_mul(x, Op);
        wc = df_mul(x, df_add_s(E, df_neg(O)));
        e = df_add_s(df_add_f(df_neg(x), 1.0f), df_mul(x, wc));
        wu = df_mul(df_mul(x, e), df_add_s(E, O));
    } else {
        dfl om;
        if (x.h <= 80.0f) {
            exp_neg_df(x, tab, e, om);
        } else {
            e = df_make(0.f, 0.f);
            om = df_make(1.f, 0.f);
        }
        // q = om / x: FP32 quotient and two corrections from the residual
        // (one leaves a relative error near 2^-44, amplified up to 40x in 1 - q)
        const dfl q = df_div_s(om, x);
        wc = df_add_f(df_neg(q), 1.0f);
        wu = df_sub_s(q, e);
    }
}

// Bilinear interpolation of a double-float field: sum of four df products
// with the TwoProduct errors and cross terms gathered in one FP32 term.
__device__ __forceinline__ dfl bilin_df(float4 wh, float4 wl, float ah, float al, float bh, float bl,
                                        float ch, float cl, float dh, float dl)
{
    const dfl p0 = two_prod(wh.x, ah), p1 = two_prod(wh.y, bh), p2 = two_prod(wh.z, ch),
              p3 = two_prod(wh.w, dh);
    float err = p0.l + p1.l + p2.l + p3.l;
    err = fmaf(wh.x, al, err); err = fmaf(wh.y, bl, err); err = fmaf(wh.z, cl, err);
    err = fmaf(wh.w, dl, err);
    err = fmaf(wl.x, ah, err); err = fmaf(wl.y, bh, err); err = fmaf(wl.z, ch, err);
    err = fmaf(wl.w, dh, err);
    dfl s = two_sum(p0.h, p1.h);
    dfl t = two_sum(p2.h, p3.h);
    dfl u = two_sum(s.h, t.h);
    err += s.l + t.l + u.l;
    return quick_two_sum(u.h, err);
}

__device__ __forceinline__ void add_steps_df(unsigned long long* steps, unsigned long long n)
{
    for (int s = 16; s > 0; s >>= 1) n += __shfl_down_sync(0xffffffffu, n, s);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(steps, n);
}

// REC: also record the march as a linear map of the source (Rec32 with the
// FP64 layout of rec_base: per (direction, plane) [step][voxel], one
// double-float pair per entry): the coefficient of S(p_m) - S_0,
// T_{m-1} w_up + T_m w_cur in double-float, and per voxel and slot the
// boundary sums sum_d w_d T_L and w_d T_L I_bc; partial is then not
// written (J comes from the replay).
template <bool REC>
__global__ void __launch_bounds__(kThreadsDF)
k_fsdf(ViewDF p, float cut, unsigned long long* __restrict__ steps, Rec32 rec)
{
    __shared__ dfl tab[2 * kExpTableDF];
    fill_exp_table_df(tab);
    __syncthreads();
    const Geometry& g = p.g;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const int t = blockIdx.x * kThreadsDF + threadIdx.x;
    const int k0 = blockIdx.y, zb = blockIdx.z, ZB = gridDim.z;
    const bool active = t < nxy;
    const unsigned amask = REC ? __ballot_sync(0xffffffffu, active) : 0u;
    unsigned long long nsteps = 0;
    if (active) {
        const int j0 = t / nx, i0 = t - j0 * nx;
        const long long v = (long long)k0 * nxy + t;
        const long long W = 2LL * nx, P = 4LL * nxy;
        const long long base = k0 * P + j0 * W + i0;
        const float4 me = p.node[base];
        const dfl chi0 = df_make(me.x, me.y), S0 = df_make(me.z, me.w);
        // The rest of a characteristic changes I - S_0 by at most
        // T * max|S - S_0| <= T * 2 smax: stop once that is below cut * S_0.
        const float smax = (float)*p.smax;
        const float tcut = smax > 0.f ? cut * S0.h / (2.0f * smax) : 0.f;
        const float4* nb = p.node + base;
        for (int slot = zb; slot < kSlots; slot += ZB) {
            double Jp = 0.0, tsum = 0.0, bcs = 0.0;
            for (int d = slot; d < g.ndir; d += kSlots) {
                const DirInfo di = p.info[d];
                const int s = di.sgn;
                const int M = s > 0 ? k0 : nz - 1 - k0;
                const int* od = p.poff + (long long)d * nz;
                const float4* bd = p.bw + (long long)d * nz * 2;
                const dfl hs = df_make(di.hs32, di.hs32lo);
                dfl I = df_make(0.f, 0.f), T = df_make(1.f, 0.f), ca = chi0, da = df_make(0.f, 0.f);
                float2* rc = REC ? rec.coef + rec_base(g, d, k0, s) + t : nullptr;
                dfl cprev = df_make(0.f, 0.f);
                bool early = false;
                int m = 0;
                for (; m < M; ++m) {
                    RT_GUARD(g, base + od[m + 1], 4 * g.N, kSiteFsdf) { early = true; break; }
                    RT_GUARD(g, base + od[m + 1] + W + 1, 4 * g.N, kSiteFsdf) { early = true; break; }
                    const float4* q = nb + od[m + 1];
                    const float4 wh = bd[2 * (m + 1)], wl = bd[2 * (m + 1) + 1];
                    const float4 q00 = __ldg(q), q10 = __ldg(q + 1);
                    const float4 q01 = __ldg(q + W), q11 = __ldg(q + W + 1);
                    const dfl cb = bilin_df(wh, wl, q00.x, q00.y, q10.x, q10.y, q01.x, q01.y,
                                            q11.x, q11.y);
                    const dfl sb = bilin_df(wh, wl, q00.z, q00.w, q10.z, q10.w, q01.z, q01.w,
                                            q11.z, q11.w);
                    const dfl db = df_sub_s(sb, S0);
                    const dfl x = df_mul(hs, df_add_s(ca, cb));
                    dfl wc, wu, e;
                    seg_weights_df(x, tab, wc, wu, e);
                    if (REC) {
                        const dfl twu = df_mul(T, wu);
                        if (m > 0) {
                            const dfl c = df_add_s(cprev, df_mul(T, wc));
                            rc[(long long)(m - 1) * nxy] = make_float2(c.h, c.l);
                        }
                        cprev = twu;
                    }
                    I = df_add_s(I, df_mul(T, df_add_s(df_mul(wc, da), df_mul(wu, db))));
                    T = df_mul(T, e);
                    ca = cb;
                    da = db;
                    if (T.h <= tcut) {
                        early = true;
                        ++m;
                        break;
                    }
                }
                if (!early) {
                    // boundary term T_M (I_bc - S_0)
                    dfl ibc;
                    const int bc = s > 0 ? g.top_bc : g.bottom_bc;
                    if (bc) {
                        const StepGeo o = p.off[(long long)d * nz + M];
                        const float4 wh = bd[2 * M], wl = bd[2 * M + 1];
                        long long ip = (j0 + o.oy) * W + (i0 + o.ox);
                        RT_GUARD(g, ip, P - W - 1, kSiteFsdf) ip = 0;   // record, read a safe node
                        const float2* pb = p.b2 + (s > 0 ? 0LL : P) + ip;
                        const float2 c00 = pb[0], c10 = pb[1], c01 = pb[W], c11 = pb[W + 1];
                        ibc = bilin_df(wh, wl, c00.x, c00.y, c10.x, c10.y, c01.x, c01.y, c11.x, c11.y);
                        if (bc == 2) {   // + |mu| dB/dtau (LTE diffusion)
                            const float2* pg = p.g2df + ip;
                            const float2 g00 = pg[0], g10 = pg[1], g01 = pg[W], g11 = pg[W + 1];
                            const dfl gr = bilin_df(wh, wl, g00.x, g00.y, g10.x, g10.y, g01.x,
                                                    g01.y, g11.x, g11.y);
                            ibc = df_add_s(ibc, df_mul(df_make(di.amu32, di.amu32lo), gr));
                        }
                        if (REC) bcs = fma(di.w * df_to_double(T), df_to_double(ibc), bcs);
                        ibc = df_sub_s(ibc, S0);
                    } else {
                        ibc = df_neg(S0);
                    }
                    I = df_add_s(I, df_mul(T, ibc));
                    if (REC) tsum = fma(di.w, df_to_double(T), tsum);
                }
                if (REC) {
                    if (m > 0) rc[(long long)(m - 1) * nxy] = make_float2(cprev.h, cprev.l);
                    const int Lw = __reduce_max_sync(amask, m);
                    for (int q = m; q < Lw; ++q) rc[(long long)q * nxy] = make_float2(0.f, 0.f);
                    if ((threadIdx.x & 31) == __ffs(amask) - 1)
                        rec.lmax[((long long)d * nz + k0) * rec.nwp + (t >> 5)] = Lw;
                }
                nsteps += (unsigned long long)m;
                Jp = fma(di.w, df_to_double(I), Jp);
            }
            if (REC) {
                rec.tsum[(long long)slot * g.N + v] = tsum;
                rec.bc[(long long)slot * g.N + v] = bcs;
            } else {
                p.partial[(long long)slot * g.N + v] = Jp;
            }
        }
    }
    if (steps) add_steps_df(steps, nsteps);
}

// Replay of the recorded double-float march for the source in p.node (its
// S parts): per (voxel, direction) I - S_0 = sum_m c_m (S(p_m) - S_0) in
// double-float over the warp's recorded length, then per slot the boundary
// sums: partial = sum_d w_d (I_d - S_0) + bc - S_0 tsum.
__global__ void __launch_bounds__(kThreadsDF)
k_fsdfrep(ViewDF p, Rec32 rec, unsigned long long* __restrict__ steps)
{
    const Geometry& g = p.g;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const int t = blockIdx.x * kThreadsDF + threadIdx.x;
    const int k0 = blockIdx.y, zb = blockIdx.z, ZB = gridDim.z;
    unsigned long long nsteps = 0;
    if (t < nxy) {
        const int j0 = t / nx, i0 = t - j0 * nx;
        const long long v = (long long)k0 * nxy + t;
        const long long W = 2LL * nx, P = 4LL * nxy;
        const long long base = k0 * P + j0 * W + i0;
        const float4 me = p.node[base];
        const dfl S0 = df_make(me.z, me.w);
        const double S0d = (double)me.z + (double)me.w;
        // the S parts {S_hi, S_lo} of the node records
        const float2* nb = reinterpret_cast<const float2*>(p.node + base) + 1;
        for (int slot = zb; slot < kSlots; slot += ZB) {
            double Jp = 0.0;
            for (int d = slot; d < g.ndir; d += kSlots) {
                const DirInfo di = p.info[d];
                const int s = di.sgn;
                const int* od = p.poff + (long long)d * nz;
                const float4* bd = p.bw + (long long)d * nz * 2;
                const float2* rc = rec.coef + rec_base(g, d, k0, s) + t;
                const int L = rec.lmax[((long long)d * nz + k0) * rec.nwp + (t >> 5)];
                dfl I = df_make(0.f, 0.f);
                for (int m = 0; m < L; ++m) {
                    const int o = od[m + 1];
                    RT_GUARD(g, base + o, 4 * g.N, kSiteFsdf) break;
                    RT_GUARD(g, base + o + W + 1, 4 * g.N, kSiteFsdf) break;
                    const float4 wh = bd[2 * (m + 1)], wl = bd[2 * (m + 1) + 1];
                    const float2* q = nb + 2LL * o;           // float2 stride: two per node
                    const float2 q00 = __ldg(q), q10 = __ldg(q + 2);
                    const float2 q01 = __ldg(q + 2 * W), q11 = __ldg(q + 2 * W + 2);
                    const dfl sb = bilin_df(wh, wl, q00.x, q00.y, q10.x, q10.y, q01.x, q01.y,
                                            q11.x, q11.y);
                    const float2 c = __ldcs(rc + (long long)m * nxy);
                    I = df_add_s(I, df_mul(df_make(c.x, c.y), df_sub_s(sb, S0)));
                }
                nsteps += (unsigned long long)L;
                Jp = fma(di.w, df_to_double(I), Jp);
            }
            const long long e = (long long)slot * g.N + v;
            p.partial[e] = Jp + rec.bc[e] - S0d * rec.tsum[e];
        }
    }
    if (steps) add_steps_df(steps, nsteps);
}

__global__ void k_packdf(Geometry g, const double* __restrict__ chi, const double* __restrict__ S,
                         float4* __restrict__ node)
{
    const int nx = g.nx, ny = g.ny;
    const long long W = 2LL * nx, P = 4LL * nx * ny;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < g.N;
         v += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(v % nx), j = (int)((v / nx) % ny);
        const long long k = v / ((long long)nx * ny);
        const dfl c = df_from_double(chi[v]), s = df_from_double(S[v]);
        const float4 q = make_float4(c.h, c.l, s.h, s.l);
        float4* pp = node + k * P + (long long)j * W + i;
        pp[0] = q;
        pp[nx] = q;
        pp[(long long)ny * W] = q;
        pp[(long long)ny * W + nx] = q;
    }
}

// Bilinear weights of every (direction, step) as double-float: [hi4, lo4].
__global__ void k_bw_df(long long n, const Bw4d* __restrict__ bw, float4* __restrict__ out)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const Bw4d b = bw[e];
        const dfl x = df_from_double(b.x), y = df_from_double(b.y), z = df_from_double(b.z),
                  w = df_from_double(b.w);
        out[2 * e] = make_float4(x.h, y.h, z.h, w.h);
        out[2 * e + 1] = make_float4(x.l, y.l, z.l, w.l);
    }
}

// Padded double-float copy of the LTE-diffusion gradient G[ny][nx].
__global__ void k_grad_df(Geometry g, const double* __restrict__ G, float2* __restrict__ out)
{
    const int nx = g.nx, ny = g.ny, nxy = nx * ny;
    const long long W = 2LL * nx;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nxy; t += gridDim.x * blockDim.x) {
        const int i = t % nx, j = t / nx;
        const dfl d = df_from_double(G[t]);
        const float2 q = make_float2(d.h, d.l);
        float2* pp = out + (long long)j * W + i;
        pp[0] = q;
        pp[nx] = q;
        pp[(long long)ny * W] = q;
        pp[(long long)ny * W + nx] = q;
    }
}

// ---- short characteristics in double-float ---------------------------------
// The plane sweep of the short characteristics (one block per direction,
// two planes in shared memory, one barrier per plane) in double-float,
// carried in the difference form D = I - S at every node:
//   D(i,j,k) = e D(p) + (1 - w_cur) (S(p) - S(i,j,k)),
// which is I = I(p) e + w_cur S + w_up S(p) rewritten with w_up + e =
// 1 - w_cur, D(p) bilinear in the preceding plane's D; on the entry plane
// D = I_bc - S.  Rounding then scales with D and with the source step
// S(p) - S rather than with S.  Each block writes w_d D for every voxel to
// its slice of the [directions][N] buffer; J = (sum_d w_d) S + the ordered
// sum of the slices.
constexpr int kScThreadsDF = 256;

struct CornersDF {
    int a00, a10, a01, a11;
};

__device__ __forceinline__ CornersDF corners_df(int i, int j, StepGeo o, int nx, int ny)
{
    int x0 = i + o.ox;
    x0 -= x0 >= nx ? nx : 0;
    const int x1 = x0 + 1 == nx ? 0 : x0 + 1;
    int y0 = j + o.oy;
    y0 -= y0 >= ny ? ny : 0;
    const int y1 = y0 + 1 == ny ? 0 : y0 + 1;
    return CornersDF{y0 * nx + x0, y0 * nx + x1, y1 * nx + x0, y1 * nx + x1};
}

template <bool SMEM>
__global__ void __launch_bounds__(kScThreadsDF)
k_scdf(ViewDF p, int d0, double* __restrict__ part, float2* gplanes,
       unsigned long long* __restrict__ steps)
{
    extern __shared__ float2 splanes_df[];
    __shared__ dfl tab[2 * kExpTableDF];
    fill_exp_table_df(tab);
    const Geometry& g = p.g;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const long long W = 2LL * nx, P = 4LL * nxy;
    const int d = d0 + blockIdx.x;
    float2* pl = SMEM ? splanes_df : gplanes + (long long)blockIdx.x * 2 * nxy;
    const DirInfo di = p.info[d];
    const int s = di.sgn;
    const int kin = s > 0 ? 0 : nz - 1;
    const int bc = s > 0 ? g.top_bc : g.bottom_bc;
    const StepGeo o = p.off[(long long)d * nz + 1];
    const int po = p.poff[(long long)d * nz + 1];
    const float4 wh = p.bw[2 * ((long long)d * nz + 1)], wl = p.bw[2 * ((long long)d * nz + 1) + 1];
    const dfl hs = df_make(di.hs32, di.hs32lo);
    double* out = part + (long long)blockIdx.x * g.N;
    for (int t = threadIdx.x; t < nxy; t += kScThreadsDF) {
        const int j = t / nx, i = t - j * nx;
        const long long ip = (long long)j * W + i;
        const float4 me = p.node[(long long)kin * P + ip];
        dfl ibc = df_make(0.f, 0.f);
        if (bc) {
            const float2 bb = p.b2[(s > 0 ? 0LL : P) + ip];
            ibc = df_make(bb.x, bb.y);
            if (bc == 2) {
                const float2 gg = p.g2df[ip];
                ibc = df_add_s(ibc, df_mul(df_make(di.amu32, di.amu32lo), df_make(gg.x, gg.y)));
            }
        }
        const dfl D = df_sub_s(ibc, df_make(me.z, me.w));
        pl[t] = make_float2(D.h, D.l);
        out[(long long)kin * nxy + t] = di.w * df_to_double(D);
    }
    __syncthreads();   // also publishes tab
    int cur = 0;
    for (int n = 1; n < nz; ++n) {
        const int k = s > 0 ? n : nz - 1 - n;
        const float2* prev = pl + cur * nxy;
        float2* next = pl + (cur ^ 1) * nxy;
        for (int t = threadIdx.x; t < nxy; t += kScThreadsDF) {
            const int j = t / nx, i = t - j * nx;
            const long long ip = (long long)j * W + i;
            const CornersDF c = corners_df(i, j, o, nx, ny);
            RT_GUARD(g, max(max(c.a00, c.a10), max(c.a01, c.a11)), nxy, kSiteSc) continue;
            RT_GUARD(g, min(min(c.a00, c.a10), min(c.a01, c.a11)), nxy, kSiteSc) continue;
            // po is relative to the node's own padded index and includes the
            // step to plane ku
            RT_GUARD(g, (long long)k * P + ip + po, 4 * g.N - W - 1, kSiteSc) continue;
            const float4 me = p.node[(long long)k * P + ip];
            const float4* q = p.node + (long long)k * P + ip + po;
            const float4 q00 = __ldg(q), q10 = __ldg(q + 1), q01 = __ldg(q + W), q11 = __ldg(q + W + 1);
            const dfl cu = bilin_df(wh, wl, q00.x, q00.y, q10.x, q10.y, q01.x, q01.y, q11.x, q11.y);
            const dfl su = bilin_df(wh, wl, q00.z, q00.w, q10.z, q10.w, q01.z, q01.w, q11.z, q11.w);
            const float2 e00 = prev[c.a00], e10 = prev[c.a10], e01 = prev[c.a01], e11 = prev[c.a11];
            const dfl Du = bilin_df(wh, wl, e00.x, e00.y, e10.x, e10.y, e01.x, e01.y, e11.x, e11.y);
            const dfl x = df_mul(hs, df_add_s(cu, df_make(me.x, me.y)));
            dfl wc, wu, e;
            seg_weights_df(x, tab, wc, wu, e);
            const dfl dS = df_sub_s(su, df_make(me.z, me.w));
            const dfl D = df_add_s(df_mul(e, Du), df_mul(df_add_f(df_neg(wc), 1.0f), dS));
            next[t] = make_float2(D.h, D.l);
            out[(long long)k * nxy + t] = di.w * df_to_double(D);
        }
        __syncthreads();
        cur ^= 1;
    }
    if (steps && threadIdx.x == 0) atomicAdd(steps, (unsigned long long)(nz - 1) * nxy);
}

// J[v] = (accumulate ? J[v] : wsum S[v]) + sum over q < nd of part[q][v].
__global__ void k_scdf_reduce(long long N, int nd, const double* __restrict__ part,
                              const double* __restrict__ S, double wsum, double* __restrict__ J,
                              int accumulate)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
        double acc = accumulate ? J[v] : wsum * S[v];
        for (int q = 0; q < nd; ++q) acc += part[(long long)q * N + v];
        J[v] = acc;
    }
}

// ---- Lambda* in double-float ------------------------------------------------
// The same elements as the FP64 kernels (long characteristics: w_cur(0) at
// p_0, w_up(0) + e_0 w_cur(1) shared among the nodes of p_1; short
// characteristics: w_cur at the voxel, b_c (w_up + e w_cur(c)) at the nodes c
// of p), evaluated in double-float and summed over the directions in a
// double-float accumulator per element.
constexpr int kLsThreadsDF = 128;

__device__ __forceinline__ void lam_add(float2* cell, dfl v)
{
    const dfl a = df_add_s(df_make(cell->x, cell->y), v);
    *cell = make_float2(a.h, a.l);
}

__device__ __forceinline__ dfl bw_df(float hi, float lo) { return df_make(hi, lo); }

template <bool SHORT>
__global__ void __launch_bounds__(kLsThreadsDF)
k_lstar_df(ViewDF p, double* __restrict__ lstar)
{
    __shared__ float2 lam[27][kLsThreadsDF];
    __shared__ dfl tab[2 * kExpTableDF];
    for (int q = 0; q < 27; ++q) lam[q][threadIdx.x] = make_float2(0.f, 0.f);
    fill_exp_table_df(tab);
    __syncthreads();
    const Geometry& g = p.g;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const long long W = 2LL * nx, P = 4LL * nxy;
    const int t = blockIdx.x * kLsThreadsDF + threadIdx.x;
    const int k0 = blockIdx.y;
    if (t >= nxy) return;
    const int j0 = t / nx, i0 = t - j0 * nx;
    const long long v = (long long)k0 * nxy + t;
    const long long base = k0 * P + (long long)j0 * W + i0;
    const float4 me = p.node[base];
    const dfl chi0 = df_make(me.x, me.y);
    for (int d = 0; d < g.ndir; ++d) {
        const DirInfo di = p.info[d];
        const int s = di.sgn;
        const int M = s > 0 ? k0 : nz - 1 - k0;
        if (M == 0) continue;
        const int* od = p.poff + (long long)d * nz;
        const float4* bd = p.bw + 2LL * d * nz;
        const dfl hs = df_make(di.hs32, di.hs32lo);
        const dfl wd = df_from_double(di.w);
        const float4 wh = bd[2], wl = bd[3];     // step 1
        RT_GUARD(g, base + od[1], 4 * g.N - W - 1, SHORT ? kSiteLstarSc : kSiteLstar64) continue;
        const float4* q = p.node + base + od[1];
        const float4 q00 = __ldg(q), q10 = __ldg(q + 1), q01 = __ldg(q + W), q11 = __ldg(q + W + 1);
        const dfl chi1 = bilin_df(wh, wl, q00.x, q00.y, q10.x, q10.y, q01.x, q01.y, q11.x, q11.y);
        dfl wc0, wu0, e0;
        seg_weights_df(df_mul(hs, df_add_s(chi0, chi1)), tab, wc0, wu0, e0);
        lam_add(&lam[13][threadIdx.x], df_mul(wd, wc0));
        const dfl bq[4] = {bw_df(wh.x, wl.x), bw_df(wh.y, wl.y), bw_df(wh.z, wl.z), bw_df(wh.w, wl.w)};
        if (!SHORT) {
            dfl c1 = wu0;
            if (M >= 2) {
                RT_GUARD(g, base + od[2], 4 * g.N - W - 1, kSiteLstar64) continue;
                const float4* r = p.node + base + od[2];
                const float4 r00 = __ldg(r), r10 = __ldg(r + 1), r01 = __ldg(r + W), r11 = __ldg(r + W + 1);
                const dfl chi2 = bilin_df(bd[4], bd[5], r00.x, r00.y, r10.x, r10.y, r01.x, r01.y,
                                          r11.x, r11.y);
                dfl wc1, wu1, e1;
                seg_weights_df(df_mul(hs, df_add_s(chi1, chi2)), tab, wc1, wu1, e1);
                c1 = df_add_s(wu0, df_mul(e0, wc1));
            }
            const dfl cw = df_mul(wd, c1);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (di.lo[c] >= 0) lam_add(&lam[di.lo[c]][threadIdx.x], df_mul(cw, bq[c]));
        } else {
            // corner c of p: its own last segment comes from plane k0 - 2s
            const int kin = s > 0 ? 0 : nz - 1;
            const bool deeper = k0 - s != kin;
            const float4 qc[4] = {q00, q10, q01, q11};
            const StepGeo o = p.off[(long long)d * nz + 1];
            int xc0 = i0 + o.ox, yc0 = j0 + o.oy;
            xc0 -= xc0 >= nx ? nx : 0;
            yc0 -= yc0 >= ny ? ny : 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (di.lo[c] < 0) continue;
                dfl wcc = df_make(0.f, 0.f);
                if (deeper) {
                    // c's own padded index (unpadded coordinates, wrapped),
                    // then its upstream nodes at the same relative offset
                    int xc = xc0 + (c & 1), yc = yc0 + (c >> 1);
                    xc -= xc >= nx ? nx : 0;
                    yc -= yc >= ny ? ny : 0;
                    const long long ic = (long long)(k0 - s) * P + (long long)yc * W + xc + od[1];
                    RT_GUARD(g, ic, 4 * g.N - W - 1, kSiteLstarSc) continue;
                    const float4* r = p.node + ic;
                    const float4 r00 = __ldg(r), r10 = __ldg(r + 1), r01 = __ldg(r + W), r11 = __ldg(r + W + 1);
                    const dfl chic = bilin_df(wh, wl, r00.x, r00.y, r10.x, r10.y, r01.x, r01.y,
                                              r11.x, r11.y);
                    dfl wuc, ec;
                    seg_weights_df(df_mul(hs, df_add_s(df_make(qc[c].x, qc[c].y), chic)), tab, wcc,
                                   wuc, ec);
                }
                lam_add(&lam[di.lo[c]][threadIdx.x],
                        df_mul(df_mul(wd, bq[c]), df_add_s(wu0, df_mul(e0, wcc))));
            }
        }
    }
    for (int q = 0; q < 27; ++q) {
        const float2 a = lam[q][threadIdx.x];
        lstar[(long long)q * g.N + v] = (double)a.x + (double)a.y;
    }
}

unsigned grid1d_df(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    if (b > 152LL * 32) b = 152LL * 32;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

cudaError_t launch_packdf(const Geometry& g, const double* chi, const double* S, float4* node,
                          cudaStream_t st)
{
    k_packdf<<<grid1d_df(g.N, 256), 256, 0, st>>>(g, chi, S, node);
    return cudaGetLastError();
}

cudaError_t launch_bw_df(long long n, const Bw4d* bw, float4* out, cudaStream_t st)
{
    k_bw_df<<<grid1d_df(n, 256), 256, 0, st>>>(n, bw, out);
    return cudaGetLastError();
}

cudaError_t launch_grad_df(const Geometry& g, const double* G, float2* out, cudaStream_t st)
{
    k_grad_df<<<grid1d_df((long long)g.nx * g.ny, 256), 256, 0, st>>>(g, G, out);
    return cudaGetLastError();
}

cudaError_t launch_fsdf(const ViewDF& p, double cut, int groups, unsigned long long* steps,
                        cudaStream_t st, const Rec32* rec)
{
    const int nxy = p.g.nx * p.g.ny;
    // planes in index order (g.zorder unused): 40.9 ms against 41.05 ms
    // with the order table on the 65^3 slab
    dim3 grid((nxy + kThreadsDF - 1) / kThreadsDF, p.g.nz, groups);
    if (rec)
        k_fsdf<true><<<grid, kThreadsDF, 0, st>>>(p, (float)cut, steps, *rec);
    else
        k_fsdf<false><<<grid, kThreadsDF, 0, st>>>(p, (float)cut, steps, Rec32{});
    return cudaGetLastError();
}

cudaError_t launch_fsdfrep(const ViewDF& p, const Rec32& rec, int groups,
                           unsigned long long* steps, cudaStream_t st)
{
    const int nxy = p.g.nx * p.g.ny;
    dim3 grid((nxy + kThreadsDF - 1) / kThreadsDF, p.g.nz, groups);
    k_fsdfrep<<<grid, kThreadsDF, 0, st>>>(p, rec, steps);
    return cudaGetLastError();
}

cudaError_t launch_scdf(const ViewDF& p, const double* S, double wsum, double* part,
                        float2* gplanes, double* J, unsigned long long* steps, cudaStream_t st)
{
    const Geometry& g = p.g;
    const int chunk = sc_chunk(g);
    const size_t shm = 2 * sizeof(float2) * (size_t)g.nx * g.ny;
    const bool smem = shm <= 200 * 1024;
    if (smem) {
        cudaError_t e = cudaFuncSetAttribute(k_scdf<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)shm);
        if (e != cudaSuccess) return e;
    }
    for (int d0 = 0; d0 < g.ndir; d0 += chunk) {
        const int nd = g.ndir - d0 < chunk ? g.ndir - d0 : chunk;
        if (smem)
            k_scdf<true><<<nd, kScThreadsDF, shm, st>>>(p, d0, part, gplanes, steps);
        else
            k_scdf<false><<<nd, kScThreadsDF, 0, st>>>(p, d0, part, gplanes, steps);
        k_scdf_reduce<<<grid1d_df(g.N, 256), 256, 0, st>>>(g.N, nd, part, S, wsum, J, d0 > 0);
    }
    return cudaGetLastError();
}

bool scdf_planes_in_smem(const Geometry& g) { return 2 * sizeof(float2) * (size_t)g.nx * g.ny <= 200 * 1024; }

cudaError_t launch_lstar_df(const ViewDF& p, bool short_chars, double* lstar, cudaStream_t st)
{
    dim3 grid((p.g.nx * p.g.ny + kLsThreadsDF - 1) / kLsThreadsDF, p.g.nz);
    if (short_chars)
        k_lstar_df<true><<<grid, kLsThreadsDF, 0, st>>>(p, lstar);
    else
        k_lstar_df<false><<<grid, kLsThreadsDF, 0, st>>>(p, lstar);
    return cudaGetLastError();
}

}  // namespace rt3d
