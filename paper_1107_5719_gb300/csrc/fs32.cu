// FP32-sweep formal solution ("precision form", Hauschildt & Baron 2011,
// Sect. 3.1: single precision suffices for the march at eps ~ 1e-2, smaller
// eps needs double precision in the operator-splitting equations).
//
// At small eps the converged J inherits the error of the formal solution
// amplified by up to ~1/eps in the thermalised layers, because there J is
// close to S and the scattering problem is nearly singular.  A march that
// accumulates I itself in FP32 carries an error ~6e-8 S, i.e. ~6e-2 in J at
// eps = 1e-6.  So this march integrates the deviation I - S_0 of the
// intensity from the source at its own voxel:
//
//   I - S_0 = sum_m T_m [w_cur,m (S(p_m) - S_0) + w_up,m (S(p_m+1) - S_0)]
//             + T_M (I_bc - S_0),
//
// which is exact because sum_m T_m (w_cur,m + w_up,m) = 1 - T_M.  The
// differences are formed from S stored as an unevaluated FP32 pair
// (hi + lo, hi = fl32(S)), so they are accurate to FP32 relative to
// themselves, and every FP32 rounding in the march scales with I - S_0
// instead of S.  J = sum_d w_d S_0 + sum_d w_d (I_d - S_0), the sum over the
// directions of a slot as an FP32 pair, the slots in FP64.  Lambda*, the
// operator splitting and the convergence test are FP64.
//
// Recording.  For fixed opacities the march is linear in S: k_fs32rec
// records, per voxel pair and step, the FP32 coefficients of S(p_m) - S_0
// (and the boundary sums), and k_fs32rep / k_fs32rep_batch evaluate the
// formal solution of any later source from them, forming the interpolated
// source differences exactly as the march does.
//
// Layout.  chi and the S pair of two x-neighbouring nodes share one record:
// pair[k][y][x] = {chi(x), S_hi(x), chi(x+1), S_hi(x+1)} (float4) and
// lo[k][y][x] = {S_lo(x), S_lo(x+1)} (float2), in planes padded by periodic
// copies to 2ny+1 rows of 2nx records.  The upstream nodes of every
// voxel at every step are then plain offsets from the voxel's own record
// (one integer add per step, no wrap arithmetic), and one thread marches
// the two voxels (i, j) and (i, j+1): their bilinear stencils share the
// middle row, so a step reads three records and three lo pairs (72 bytes,
// exactly the twelve values each voxel needs, with the middle row read
// once for both) where one voxel per thread with one record per node read
// four 16-byte records per voxel.  B of the two boundary planes is kept as
// padded float2 {B_hi, B_lo} (planes 2ny x 2nx).
#include "internal.h"
#include "weights.cuh"

namespace rt3d {

namespace {

constexpr int kThreads32 = 128;     // default threads per block
// 72 registers (seven blocks of 128 threads per SM) and the step loop
// unrolled twice: measured on the 65^3 slab with 32x32 directions, 8.40 ms
// per formal solution against 8.70 ms at 80 registers (six blocks) and
// 8.89 ms at 64 (eight blocks, spilling in the loop); with the earlier
// step, 9.43 ms against 9.94 ms without unrolling, 9.88 ms at 96 registers
// and 10.1-11.1 ms for variants that load the next step's records before
// computing the current one (more registers, fewer warps).
#ifndef RT_FS32_MINB
#define RT_FS32_MINB 7
#endif
#ifndef RT_FS32B_MINB
#define RT_FS32B_MINB 6
#endif
constexpr int kMinBlocks32 = RT_FS32_MINB;
// Threads per block are a launch knob (64, 128 or 256, rt_set_block_threads);
// 64 and 128 keep the same resident threads per SM and registers, 256
// rounds down to three blocks (768 threads, 80 registers).
constexpr int kResident32 = kThreads32 * kMinBlocks32;
// The fused batch launch keeps six blocks (80 registers): at seven it
// spills in the loop, 171 against 157 ms per launch of 16 x 65^3 problems.
constexpr int kResidentB32 = kThreads32 * RT_FS32B_MINB;
#ifndef RT_FS32R_MINB
#define RT_FS32R_MINB 8
#endif
// The replay of the recorded march: eight blocks (64 registers), since its
// loads wait on memory more than its arithmetic; measured on the 65^3 slab,
// 6.14 ms per replay against 6.49 at seven blocks (72 registers); at ten
// blocks it spills 800 bytes per thread.
constexpr int kResidentR32 = kThreads32 * RT_FS32R_MINB;


// poff[d][m] = offset of the upstream node (x0, y0) of step m from the
// voxel's own node in planes of `rows` padded rows of 2nx entries.
__global__ void k_pad_offsets(Geometry g, const DirInfo* __restrict__ info,
                              const StepGeo* __restrict__ off, long long rows,
                              int* __restrict__ poff)
{
    const int d = blockIdx.x;
    const int s = info[d].sgn;
    const long long W = 2LL * g.nx;
    for (int m = threadIdx.x; m < g.nz; m += blockDim.x) {
        const StepGeo o = off[(long long)d * g.nz + m];
        poff[(long long)d * g.nz + m] = (int)((-(long long)m * s * rows + o.oy) * W + o.ox);
    }
}

// One thread per padded record (k, y, x): the nodes (x mod nx, y mod ny) and
// (x+1 mod nx, y mod ny) of plane k.
__global__ void k_pack_pairs(Geometry g, const double* __restrict__ chi,
                             const double* __restrict__ S, float4* __restrict__ pair,
                             float2* __restrict__ lo)
{
    const int nx = g.nx, ny = g.ny;
    const long long W = 2LL * nx, R = 2LL * ny + 1, P = R * W;
    const long long n = P * g.nz;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
         r += (long long)gridDim.x * blockDim.x) {
        const long long k = r / P, rem = r - k * P;
        const int y = (int)(rem / W), x = (int)(rem - (long long)y * W);
        int j = y, i0 = x, i1 = x + 1;
        while (j >= ny) j -= ny;
        while (i0 >= nx) i0 -= nx;
        while (i1 >= nx) i1 -= nx;
        const long long row = (k * ny + j) * (long long)nx;
        const double s0 = S[row + i0], s1 = S[row + i1];
        const float h0 = (float)s0, h1 = (float)s1;
        pair[r] = make_float4((float)chi[row + i0], h0, (float)chi[row + i1], h1);
        lo[r] = make_float2((float)(s0 - (double)h0), (float)(s1 - (double)h1));
    }
}

// The replay's source records: spair[k][y][x] = {S_hi, S_lo} of the nodes
// (x mod nx, y mod ny) and (x+1 mod nx, y mod ny), padded as k_pack_pairs.
__global__ void k_pack_spairs(Geometry g, const double* __restrict__ S, float4* __restrict__ sp)
{
    const int nx = g.nx, ny = g.ny;
    const long long W = 2LL * nx, R = 2LL * ny + 1, P = R * W;
    const long long n = P * g.nz;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
         r += (long long)gridDim.x * blockDim.x) {
        const long long k = r / P, rem = r - k * P;
        const int y = (int)(rem / W), x = (int)(rem - (long long)y * W);
        int j = y, i0 = x, i1 = x + 1;
        while (j >= ny) j -= ny;
        while (i0 >= nx) i0 -= nx;
        while (i1 >= nx) i1 -= nx;
        const long long row = (k * ny + j) * (long long)nx;
        const double s0 = S[row + i0], s1 = S[row + i1];
        const float h0 = (float)s0, h1 = (float)s1;
        sp[r] = make_float4(h0, (float)(s0 - (double)h0), h1, (float)(s1 - (double)h1));
    }
}

__global__ void k_pack_b2(Geometry g, const double* __restrict__ B, float2* __restrict__ b2)
{
    const int nx = g.nx, ny = g.ny, nxy = nx * ny;
    const long long W = 2LL * nx, P = 4LL * nxy;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * nxy; t += gridDim.x * blockDim.x) {
        const int plane = t / nxy, r = t - plane * nxy;
        const int i = r % nx, j = r / nx;
        const double b = B[(plane ? (long long)(g.nz - 1) * nxy : 0LL) + r];
        const float hi = (float)b;
        const float2 q = make_float2(hi, (float)(b - (double)hi));
        float2* p = b2 + plane * P + (long long)j * W + i;
        p[0] = q;
        p[nx] = q;
        p[(long long)ny * W] = q;
        p[(long long)ny * W + nx] = q;
    }
}

__device__ __forceinline__ void add_steps32(unsigned long long* steps, unsigned long long n)
{
    for (int s = 16; s > 0; s >>= 1) n += __shfl_down_sync(0xffffffffu, n, s);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(steps, n);
}

// Per-voxel state of one characteristic of the FP32 march.
struct Ray32 {
    float s0h, s0l, tcut;   // S_0 as an FP32 pair; transmission cutoff
    float I, Ilo;           // I - S_0 as an unevaluated sum I + Ilo
    float tau, T, ca, da;   // optical depth, transmission, hs chi and S - S_0 at p_m
};

// One step of a voxel's characteristic, from p_m to p_m+1: the upstream
// point's four nodes are u0 = {chi, S_hi} of (x0, y0) and (x1, y0), u1 the
// same of (x0, y1), (x1, y1); l0, l1 their S_lo; b the bilinear weights.
// Returns whether the segment took the series branch (x < 2); wc_T, wu_T:
// the segment's weights times the transmission T_m (the recording stores
// them as coefficients of S).
__device__ __forceinline__ bool step32(Ray32& r, float hs, float4 b, float4 u0, float4 u1,
                                       float2 l0, float2 l1, float& wc_T, float& wu_T)
{
    constexpr float kLog2e = 1.4426950408889634f;
    const float cb = b.x * u0.x + b.y * u0.z + b.z * u1.x + b.w * u1.z;
    // S(p) - S_0: hi differences are exact for nearby values
    const float dh = b.x * (u0.y - r.s0h) + b.y * (u0.w - r.s0h) + b.z * (u1.y - r.s0h) +
                     b.w * (u1.w - r.s0h);
    const float dl = b.x * l0.x + b.y * l0.y + b.z * l1.x + b.w * l1.y;
    const float db = dh + (dl - r.s0l);
    const float x = hs * (r.ca + cb);
    // I - S_0 += T_m w_cur D_m + T_m w_up D_m+1 (TwoSum), with
    // T_m w_up = T_m e x phi2(x) = T_{m+1} x phi2(x): below x = 2 the
    // upstream weight takes the next transmission (from the optical depth)
    // instead of e, which saves its exponential (measured on the 65^3 slab:
    // 9.49 against 9.73 ms; converged J at eps = 1e-6 within 2.1e-8 of FP64
    // against 3.3e-8)
    r.tau += x;
    const float Tn = ex2_approx(-r.tau * kLog2e);
    float wcT, wuT;
    if (x < 2.0f) {
        // x phi2(-+x) = x E -+ x^2 Q
        const float z = x * x;
        float E, Q;
        phi2_eq32(z, E, Q);
        const float xe = x * E, zq = z * Q;
        wcT = r.T * (xe - zq);
        wuT = Tn * (xe + zq);
    } else {
        const float e = ex2_approx(-x * kLog2e);
        const float q = (1.0f - e) * rcp_approx(x);
        wcT = r.T * (1.0f - q);
        wuT = r.T * (q - e);
    }
    // compensated (Kahan) accumulation of I - S_0 = I + Ilo: the carried
    // low part enters the increment's last FMA, and the rounding error of
    // the sum becomes the new low part
    const float y = fmaf(wcT, r.da, fmaf(wuT, db, r.Ilo));
    const float sI = r.I + y;
    r.Ilo = y - (sI - r.I);
    r.I = sI;
    r.T = Tn;
    r.ca = cb;
    r.da = db;
    wc_T = wcT;
    wu_T = wuT;
    return x < 2.0f;
}

// The boundary intensity at the ray's end point (B, or B + |mu| dB/dtau
// for the LTE-diffusion boundary) in FP64 from the FP32 pairs, for the
// recording; 0 for a zero boundary.
__device__ __forceinline__ double boundary_value32(const View32& p, const DirInfo& di, int d,
                                                   int M, int i0, int j0)
{
    const Geometry& g = p.g;
    const int s = di.sgn;
    const int bc = s > 0 ? g.top_bc : g.bottom_bc;
    if (!bc) return 0.0;
    const long long W = 2LL * g.nx, P = 4LL * g.nx * g.ny;
    const StepGeo o = p.off[(long long)d * g.nz + M];
    const float4 b = p.bw[(long long)d * g.nz + M];
    long long ip = (j0 + o.oy) * W + (i0 + o.ox);
    RT_GUARD(g, ip, P - W - 1, kSiteFs32) ip = 0;
    const float2* pb = p.b2 + (s > 0 ? 0LL : P) + ip;
    const float2 c00 = pb[0], c10 = pb[1], c01 = pb[W], c11 = pb[W + 1];
    double v = (double)b.x * ((double)c00.x + c00.y) + (double)b.y * ((double)c10.x + c10.y) +
               (double)b.z * ((double)c01.x + c01.y) + (double)b.w * ((double)c11.x + c11.y);
    if (bc == 2) {
        const float* pg = p.g2 + ip;
        v += (double)di.amu32 *
             ((double)b.x * pg[0] + (double)b.y * pg[1] + (double)b.z * pg[W] + (double)b.w * pg[W + 1]);
    }
    return v;
}

// s + lo += w (v + vlo): the product w v split exactly (TwoProduct by FMA)
// and added by TwoSum; the low parts are gathered in lo
__device__ __forceinline__ void pair_add(float& s, float& lo, float w, float v, float vlo)
{
    const float p = w * v;
    const float pe = fmaf(w, vlo, fmaf(w, v, -p));
    const float t = s + p, bb = t - s;
    lo += (s - (t - bb)) + (p - bb) + pe;
    s = t;
}

// Boundary term T_M (I_bc - S_0) of a characteristic that reached the
// boundary plane, added with its rounding error.  j0: the voxel's row.
__device__ __forceinline__ void boundary32(Ray32& r, const View32& p, const DirInfo& di,
                                           int d, int M, int i0, int j0)
{
    const Geometry& g = p.g;
    const int s = di.sgn;
    const int bc = s > 0 ? g.top_bc : g.bottom_bc;
    float inc, inc_lo;
    if (bc) {
        const long long W = 2LL * g.nx, P = 4LL * g.nx * g.ny;
        const StepGeo o = p.off[(long long)d * g.nz + M];
        const float4 b = p.bw[(long long)d * g.nz + M];
        long long ip = (j0 + o.oy) * W + (i0 + o.ox);
        RT_GUARD(g, ip, P - W - 1, kSiteFs32) ip = 0;   // record, read a safe node
        const float2* pb = p.b2 + (s > 0 ? 0LL : P) + ip;
        const float2 c00 = pb[0], c10 = pb[1], c01 = pb[W], c11 = pb[W + 1];
        const float h = b.x * (c00.x - r.s0h) + b.y * (c10.x - r.s0h) + b.z * (c01.x - r.s0h) +
                        b.w * (c11.x - r.s0h);
        const float l = b.x * c00.y + b.y * c10.y + b.z * c01.y + b.w * c11.y;
        float ibc = h + (l - r.s0l);
        if (bc == 2) {   // + |mu| dB/dtau (LTE diffusion)
            const float* pg = p.g2 + ip;
            ibc = fmaf(__ldg(&p.info[d].amu32),
                       b.x * pg[0] + b.y * pg[1] + b.z * pg[W] + b.w * pg[W + 1], ibc);
        }
        inc = r.T * ibc;
        inc_lo = fmaf(r.T, ibc, -inc);
    } else {
        inc = -r.T * r.s0h;
        inc_lo = fmaf(-r.T, r.s0h, -inc) - r.T * r.s0l;
    }
    const float sI = r.I + inc, bb = sI - r.I;
    r.Ilo += (r.I - (sI - bb)) + (inc - bb) + inc_lo;
    r.I = sI;
}

// One thread per pair of voxels (i0, j0) and (i0, j0 + 1) of plane k0,
// j0 even (the second one absent when j0 = ny - 1), tile `tile`
// (kThreads32 pairs); block z index zb of ZB walks the direction slots zb,
// zb + ZB, ... (d mod kSlots); partial[slot][v] = sum_{d in slot} w_d (I_d - S_0).
//
// Two details keep the FP32 rounding from reaching J at small eps:
//  - I - S_0 is accumulated as an unevaluated pair (Knuth's TwoSum), so the
//    sum does not lose the ~6e-8 |I - S_0| per step that a plain FP32 sum
//    loses where |I - S_0| ~ S (optically thin layers);
//  - the transmission is T = 2^(-tau log2 e) of the accumulated optical
//    depth tau, not the running product of the factors e ~ 1 - x, whose
//    roundings add up over the many thin segments near the surface.
// Measured on a 9x9x129 slab (32x8 directions): converged J within 2.5e-8
// of the FP64 solution at eps = 1e-6 (1.4e-6 with a plain FP32 sum and
// product).
//
// The two characteristics of a thread are marched together until both are
// cut off (or reach the boundary, where both take their boundary term); a
// voxel whose own cutoff came first keeps adding its (negligible) terms.
// The step count is that of each voxel's own cutoff.
// COUNT (diagnostics only): also count the steps that took the series
// branch of the segment weights into *series.  REC: also record the march
// into rec (Rec32): per step the coefficients of S(p_m) - S_0 of both
// voxels, T_{m-1} w_up + T_m w_cur while the voxel's ray is alive (zero
// after it is cut), and per voxel and slot the boundary sums; partial is
// then not written (J comes from the replay).
template <int TB, bool COUNT, bool REC>
__device__ __forceinline__ void march32(const View32& p, int tile, int k0, int zb, int ZB,
                                        float cut, unsigned long long* __restrict__ steps,
                                        unsigned long long* __restrict__ series, Rec32 rec)
{
    const Geometry& g = p.g;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const int nyp = (ny + 1) >> 1;
    const int t = tile * TB + threadIdx.x;
    const bool active = t < nx * nyp;
    const unsigned amask = REC ? __ballot_sync(0xffffffffu, active) : 0u;
    unsigned long long nsteps = 0, nseries = 0;
    if (active) {
        const int jp = t / nx, i0 = t - jp * nx, j0 = 2 * jp;
        const bool two = j0 + 1 < ny;
        const long long va = (long long)k0 * nxy + (long long)j0 * nx + i0;
        const long long W = 2LL * nx, P = (2LL * ny + 1) * W;
        const long long base = k0 * P + j0 * W + i0;
        const float4* pa = p.pair + base;
        const float2* pl = p.lo + base;
        const float4 ma = pa[0], mb = pa[W];
        const float2 la = pl[0], lb = pl[W];
        // The rest of a characteristic changes I - S_0 by at most
        // T * max|S - S_0| <= T * 2 smax: stop once that is below cut * S_0.
        // A march of a source change (p.sfloor set) stops once that is
        // below cut * sfloor, a lower bound of the source it changes.  An
        // absent second voxel counts as cut off from the start.
        const float smax = (float)*p.smax;
        float tca, tcb;
        if (p.sfloor) {
            const float t = smax > 0.f ? cut * (float)*p.sfloor / (2.0f * smax) : 2.0f;
            tca = t;
            tcb = two ? t : 2.0f;
        } else {
            const float ka = smax > 0.f ? cut / (2.0f * smax) : 0.f;
            tca = ka * (ma.y + la.x);
            tcb = two ? ka * (mb.y + lb.x) : 2.0f;
        }
        for (int slot = zb; slot < kSlots; slot += ZB) {
            // sum_d w_d (I_d - S_0) of the slot as an FP32 pair (the FP64
            // pipe of this GPU runs at 1/64 of the FP32 rate; measured on the
            // 65^3 slab: 8.7-9.0 ms against 9.13 with FP64 accumulation)
            float Ja = 0.f, Jalo = 0.f, Jb = 0.f, Jblo = 0.f;
            double tsa = 0.0, bca = 0.0, tsb = 0.0, bcb = 0.0;   // REC: boundary sums
            for (int d = slot; d < g.ndir; d += kSlots) {
                const DirInfo di = p.info[d];
                const int s = di.sgn;
                const int M = s > 0 ? k0 : nz - 1 - k0;
                const int* od = p.poff + (long long)d * nz;
                const float4* bd = p.bw + (long long)d * nz;
                Ray32 a{ma.y, la.x, tca, 0.f, 0.f, 0.f, 1.f, ma.x, 0.f};
                Ray32 b{mb.y, lb.x, tcb, 0.f, 0.f, 0.f, 1.f, mb.x, 0.f};
                bool alive_a = true, alive_b = two, early = false;
                int na = 0, nb = 0, sa = 0, sb = 0;
                // coefficient of p_m at rc[rec32_step(m)]
                float2* rc = REC ? rec.coef + rec32_at(g, d, k0, s, t) : nullptr;
                float cpa = 0.f, cpb = 0.f;   // REC: pending coefficient of the current point
                int m = 0;
#pragma unroll 2
                for (; m < M; ++m) {
                    const int o = od[m + 1];
                    RT_GUARD(g, base + o, P * nz, kSiteFs32) { early = true; break; }
                    RT_GUARD(g, base + o + 2 * W, P * nz, kSiteFs32) { early = true; break; }
                    const float4 bw = bd[m + 1];
                    const float4* q = pa + o;
                    const float2* ql = pl + o;
                    const float4 u0 = __ldg(q), u1 = __ldg(q + W), u2 = __ldg(q + 2 * W);
                    const float2 l0 = __ldg(ql), l1 = __ldg(ql + W), l2 = __ldg(ql + 2 * W);
                    float wca, wua, wcb, wub;
                    const bool ba = step32(a, di.hs32, bw, u0, u1, l0, l1, wca, wua);
                    const bool bb = step32(b, di.hs32, bw, u1, u2, l1, l2, wcb, wub);
                    if (COUNT) {
                        sa += alive_a && ba;
                        sb += alive_b && bb;
                    }
                    if (REC) {
                        // point p_m gets this segment's w_cur (if alive) after
                        // the previous segment's w_up
                        const float2 c = make_float2(alive_a ? cpa + wca : cpa,
                                                     alive_b ? cpb + wcb : cpb);
                        cpa = alive_a ? wua : 0.f;
                        cpb = alive_b ? wub : 0.f;
                        if (m > 0) rc[rec32_step(m)] = c;
                    }
                    na += alive_a;
                    nb += alive_b;
                    alive_a = alive_a && a.T > a.tcut;
                    alive_b = alive_b && b.T > b.tcut;
                    if (!alive_a && !alive_b) {
                        early = true;
                        ++m;
                        break;
                    }
                }
                if (REC) {
                    if (m > 0) rc[rec32_step(m)] = make_float2(cpa, cpb);
                    if (!early && alive_a) {
                        tsa = fma(di.w, (double)a.T, tsa);
                        bca = fma(di.w * (double)a.T, boundary_value32(p, di, d, M, i0, j0), bca);
                    }
                    if (!early && alive_b) {
                        tsb = fma(di.w, (double)b.T, tsb);
                        bcb = fma(di.w * (double)b.T, boundary_value32(p, di, d, M, i0, j0 + 1), bcb);
                    }
                    // zeros up to the warp's longest ray (the replay's length)
                    const int Lw = __reduce_max_sync(amask, m);
                    // (the replay reads whole blocks of four steps: zero them too,
                    // up to the ray's room M rounded to four)
                    const int Lz = min((Lw + 3) & ~3, (M + 3) & ~3);
                    for (int q = m + 1; q <= Lz; ++q) rc[rec32_step(q)] = make_float2(0.f, 0.f);
                    if ((threadIdx.x & 31) == __ffs(amask) - 1)
                        rec.lmax[((long long)d * nz + k0) * rec.nwp + (t >> 5)] = Lw;
                } else if (!early) {
                    boundary32(a, p, di, d, M, i0, j0);
                    if (two) boundary32(b, p, di, d, M, i0, j0 + 1);
                }
                nsteps += (unsigned long long)na + (two ? (unsigned long long)nb : 0ull);
                if (COUNT) nseries += (unsigned long long)sa + (two ? (unsigned long long)sb : 0ull);
                pair_add(Ja, Jalo, di.w32, a.I, a.Ilo);
                pair_add(Jb, Jblo, di.w32, b.I, b.Ilo);
            }
            if (REC) {
                rec.tsum[(long long)slot * g.N + va] = tsa;
                rec.bc[(long long)slot * g.N + va] = bca;
                if (two) {
                    rec.tsum[(long long)slot * g.N + va + nx] = tsb;
                    rec.bc[(long long)slot * g.N + va + nx] = bcb;
                }
            } else {
                p.partial[(long long)slot * g.N + va] = (double)Ja + (double)Jalo;
                if (two) p.partial[(long long)slot * g.N + va + nx] = (double)Jb + (double)Jblo;
            }
        }
    }
    if (steps) add_steps32(steps, nsteps);
    if (COUNT && series) add_steps32(series, nseries);
}

template <int TB, bool COUNT>
__global__ void __launch_bounds__(TB, kResident32 / TB)
k_fs32d(View32 p, float cut, unsigned long long* __restrict__ steps,
        unsigned long long* __restrict__ series)
{
    const int tile = p.pmajor ? blockIdx.y : blockIdx.x;
    const int k0 = p.pmajor ? blockIdx.x : blockIdx.y;
    march32<TB, COUNT, false>(p, tile, k0, blockIdx.z, gridDim.z, cut, steps, series, Rec32{});
}

// The recording march (128 threads per block, once per opacity).
__global__ void __launch_bounds__(kThreads32)
k_fs32rec(View32 p, float cut, unsigned long long* __restrict__ steps, Rec32 rec)
{
    const int tile = p.pmajor ? blockIdx.y : blockIdx.x;
    const int k0 = p.pmajor ? blockIdx.x : blockIdx.y;
    march32<kThreads32, false, true>(p, tile, k0, blockIdx.z, gridDim.z, cut, steps, nullptr, rec);
}

// Replay of the recorded FP32 march (Rec32) for the source packed in
// p.spair: per pair of voxels and direction, I - S_0 = sum_m c_m (S(p_m) -
// S_0) over the warp's recorded length (difference form, Kahan sum), then
// per voxel and slot the boundary sums: partial = sum_d w_d (I_d - S_0) +
// bc - S_0 tsum (bc omitted for zero boundary intensities).  The interpolated
// differences are formed as in the march (hi differences exact for nearby
// values, the lo parts added once).
template <int TB>
__device__ __forceinline__ void replay32(const Rep32& p, int tile, int k0, int zb, int ZB,
                                         unsigned long long* __restrict__ steps)
{
    const Geometry& g = p.g;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const int nyp = (ny + 1) >> 1;
    const int t = tile * TB + threadIdx.x;
    unsigned long long nsteps = 0;
    if (t < nx * nyp) {
        const int jp = t / nx, i0 = t - jp * nx, j0 = 2 * jp;
        const bool two = j0 + 1 < ny;
        const long long va = (long long)k0 * nxy + (long long)j0 * nx + i0;
        const long long W = 2LL * nx, P = (2LL * ny + 1) * W;
        const long long base = k0 * P + j0 * W + i0;
        const float4* pa = p.spair + base;
        const float4 ma = pa[0], mb = pa[W];     // {S_hi, S_lo} of the voxels (and x+1)
        const float sha = ma.x, sla = ma.y, shb = mb.x, slb = mb.y;
        const double S0a = (double)sha + (double)sla, S0b = (double)shb + (double)slb;
        for (int slot = zb; slot < kSlots; slot += ZB) {
            float Ja = 0.f, Jalo = 0.f, Jb = 0.f, Jblo = 0.f;
            for (int d = slot; d < g.ndir; d += kSlots) {
                const DirInfo di = p.info[d];
                const int s = di.sgn;
                const int* od = p.poff + (long long)d * nz;
                const float4* bd = p.bw + (long long)d * nz;
                const float2* rc = p.rec.coef + rec32_at(g, d, k0, s, t);
                const int L = p.rec.lmax[((long long)d * nz + k0) * p.rec.nwp + (t >> 5)];
                float Ia = 0.f, Ial = 0.f, Ib = 0.f, Ibl = 0.f;
                // one step: the upstream point of step m + 1, coefficients c
                auto step = [&](int m, float2 c) {
                    const int o = od[m + 1];
                    const float4 b = bd[m + 1];
                    const float4* q = pa + o;
                    const float4 u0 = __ldg(q), u1 = __ldg(q + W), u2 = __ldg(q + 2 * W);
                    const float dha = b.x * (u0.x - sha) + b.y * (u0.z - sha) + b.z * (u1.x - sha) +
                                      b.w * (u1.z - sha);
                    const float dla = b.x * u0.y + b.y * u0.w + b.z * u1.y + b.w * u1.w;
                    const float dhb = b.x * (u1.x - shb) + b.y * (u1.z - shb) + b.z * (u2.x - shb) +
                                      b.w * (u2.z - shb);
                    const float dlb = b.x * u1.y + b.y * u1.w + b.z * u2.y + b.w * u2.w;
                    const float ya = fmaf(c.x, dha + (dla - sla), Ial);
                    const float ta = Ia + ya;
                    Ial = ya - (ta - Ia);
                    Ia = ta;
                    const float yb = fmaf(c.y, dhb + (dlb - slb), Ibl);
                    const float tb = Ib + yb;
                    Ibl = yb - (tb - Ib);
                    Ib = tb;
                };
                int m = 0;
                // whole blocks of four steps without conditions, so that their
                // loads can be issued together; then the remaining steps
                for (; m + 4 <= L; m += 4) {
                    RT_GUARD(g, base + od[m + 4], P * nz, kSiteFs32) break;
                    RT_GUARD(g, base + od[m + 4] + 2 * W, P * nz, kSiteFs32) break;
                    // the coefficients are read once: streaming loads, so that
                    // they do not displace the source records from the caches
                    const float4* c4 = reinterpret_cast<const float4*>(rc + rec32_step(m + 1));
                    const float4 cA = __ldcs(c4), cB = __ldcs(c4 + 1);
                    step(m, make_float2(cA.x, cA.y));
                    step(m + 1, make_float2(cA.z, cA.w));
                    step(m + 2, make_float2(cB.x, cB.y));
                    step(m + 3, make_float2(cB.z, cB.w));
                }
                for (; m < L; ++m) {
                    RT_GUARD(g, base + od[m + 1], P * nz, kSiteFs32) break;
                    RT_GUARD(g, base + od[m + 1] + 2 * W, P * nz, kSiteFs32) break;
                    step(m, __ldcs(rc + rec32_step(m + 1)));
                }
                nsteps += (unsigned long long)L * (two ? 2ull : 1ull);
                pair_add(Ja, Jalo, di.w32, Ia, Ial);
                pair_add(Jb, Jblo, di.w32, Ib, Ibl);
            }
            const long long ea = (long long)slot * g.N + va;
            double ja = (double)Ja + (double)Jalo - S0a * p.rec.tsum[ea];
            if (!p.zero_bc) ja += p.rec.bc[ea];
            p.partial[ea] = ja;
            if (two) {
                const long long eb = ea + nx;
                double jb = (double)Jb + (double)Jblo - S0b * p.rec.tsum[eb];
                if (!p.zero_bc) jb += p.rec.bc[eb];
                p.partial[eb] = jb;
            }
        }
    }
    if (steps) add_steps32(steps, nsteps);
}

template <int TB>
__global__ void __launch_bounds__(TB, kResidentR32 / TB)
k_fs32rep(Rep32 p, unsigned long long* __restrict__ steps)
{
    // the view read from shared memory holds fewer registers
    __shared__ Rep32 sp;
    if (threadIdx.x == 0) sp = p;
    __syncthreads();
    const int tile = p.pmajor ? blockIdx.y : blockIdx.x;
    const int k0 = p.pmajor ? blockIdx.x : blockIdx.y;
    replay32<TB>(sp, tile, k0, blockIdx.z, gridDim.z, steps);
}

// The replays of many problems in one launch, blocks assigned to problems
// as in k_fs32_batch (the problem's view staged in shared memory).
template <int TB>
__global__ void __launch_bounds__(TB, kResidentR32 / TB)
k_fs32rep_batch(const Rep32* __restrict__ views, const int* __restrict__ ids,
                const long long* __restrict__ prefix, int nact, int ZB,
                unsigned long long* __restrict__ steps)
{
    __shared__ Rep32 p;
    __shared__ long long s_local;
    if (threadIdx.x == 0) {
        const long long b = blockIdx.x + (long long)blockIdx.y * gridDim.x;
        int lo = 0, hi = nact;  // prefix[lo] <= b < prefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (prefix[mid] <= b) lo = mid; else hi = mid;
        }
        s_local = b < prefix[nact] ? b - prefix[lo] : -1;
        if (s_local >= 0) p = views[ids[lo]];
    }
    __syncthreads();
    const long long local = s_local;
    if (local < 0) return;
    const int tiles = (p.g.nx * ((p.g.ny + 1) >> 1) + TB - 1) / TB;
    const long long tk = local % ((long long)tiles * p.g.nz);
    const int zb = (int)(local / ((long long)tiles * p.g.nz));
    const int tile = p.pmajor ? (int)(tk / p.g.nz) : (int)(tk % tiles);
    const int k0 = p.pmajor ? (int)(tk % p.g.nz) : (int)(tk / tiles);
    replay32<TB>(p, tile, k0, zb, ZB, steps);
}

int tiles32(const Geometry& g, int tb) { return (g.nx * ((g.ny + 1) / 2) + tb - 1) / tb; }

// Many problems in one launch: block b belongs to the active problem q with
// prefix[q] <= b < prefix[q+1]; within it, blocks run tile-fastest, then
// plane, then slot group.
template <int TB>
__global__ void __launch_bounds__(TB, kResidentB32 / TB)
k_fs32_batch(const View32* __restrict__ views, const int* __restrict__ ids,
             const long long* __restrict__ prefix, int nact, int ZB, float cut,
             unsigned long long* __restrict__ steps)
{
    // the block's problem view, staged once in shared memory by one
    // thread (measured: 157.1 against 158.0 ms per launch of 16 x 65^3
    // problems read from global memory by every thread)
    __shared__ View32 p;
    __shared__ long long s_local;
    if (threadIdx.x == 0) {
        const long long b = blockIdx.x + (long long)blockIdx.y * gridDim.x;
        int lo = 0, hi = nact;  // prefix[lo] <= b < prefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (prefix[mid] <= b) lo = mid; else hi = mid;
        }
        s_local = b < prefix[nact] ? b - prefix[lo] : -1;
        if (s_local >= 0) p = views[ids[lo]];
    }
    __syncthreads();
    const long long local = s_local;
    if (local < 0) return;
    const int tiles = (p.g.nx * ((p.g.ny + 1) >> 1) + TB - 1) / TB;
    const long long tk = local % ((long long)tiles * p.g.nz);
    const int zb = (int)(local / ((long long)tiles * p.g.nz));
    const int tile = p.pmajor ? (int)(tk / p.g.nz) : (int)(tk % tiles);
    const int k0 = p.pmajor ? (int)(tk % p.g.nz) : (int)(tk / tiles);
    march32<TB, false, false>(p, tile, k0, zb, ZB, cut, steps, nullptr, Rec32{});
}

// dS = S - Sref (the source change the finishing stage marches)
__global__ void k_delta_source(long long N, const double* __restrict__ S,
                               const double* __restrict__ Sref, double* __restrict__ dS)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x)
        dS[v] = S[v] - Sref[v];
}

// *out = min_v |x[v]| (one block, fixed reduction order)
__global__ void k_absmin(long long N, const double* __restrict__ x, double* __restrict__ out)
{
    __shared__ double sm[256];
    double m = __longlong_as_double(0x7FF0000000000000LL);   // +inf
    for (long long v = threadIdx.x; v < N; v += blockDim.x) m = fmin(m, fabs(x[v]));
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] = fmin(sm[threadIdx.x], sm[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

// J[v] = Jref[v] + wsum * dS[v] + sum_slot partial[slot][v]  (slot order fixed)
__global__ void k_sum_groups_ref(long long N, const double* __restrict__ partial,
                                 const double* __restrict__ dS, double wsum,
                                 const double* __restrict__ Jref, double* __restrict__ J)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < kSlots; ++q) s += partial[q * N + v];
        J[v] = Jref[v] + fma(wsum, dS[v], s);
    }
}

// J[v] = wsum * S[v] + sum_slot partial[slot][v]  (slot order fixed)
__global__ void k_sum_groups_src(long long N, const double* __restrict__ partial,
                                 const double* __restrict__ S, double wsum, double* __restrict__ J)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < kSlots; ++q) s += partial[q * N + v];
        J[v] = fma(wsum, S[v], s);
    }
}

unsigned grid1d(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    if (b > 152LL * 32) b = 152LL * 32;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

int plane_major32(const Geometry& g, int order)
{
    if (order == 1) return 0;
    const long long tiles = tiles32(g, 64);   // the most tiles of any block size
    if (tiles > 65535) return 0;              // grid y limit
    if (order == 2) return 1;
    const long long bytes = (2ll * g.ny + 1) * 2ll * g.nx * (long long)g.nz *
                            (long long)(sizeof(float4) + sizeof(float2));
    return bytes > kPlaneMajorBytes ? 1 : 0;
}

long long pair_records(const Geometry& g) { return (2LL * g.ny + 1) * 2LL * g.nx * g.nz; }

cudaError_t launch_pad_offsets(const Geometry& g, const DirInfo* info, const StepGeo* off,
                               long long rows, int* poff, cudaStream_t st)
{
    k_pad_offsets<<<g.ndir, 128, 0, st>>>(g, info, off, rows, poff);
    return cudaGetLastError();
}

cudaError_t launch_pack_pairs(const Geometry& g, const double* chi, const double* S, float4* pair,
                              float2* lo, cudaStream_t st)
{
    k_pack_pairs<<<grid1d(pair_records(g), 256), 256, 0, st>>>(g, chi, S, pair, lo);
    return cudaGetLastError();
}

cudaError_t launch_pack_spairs(const Geometry& g, const double* S, float4* spair, cudaStream_t st)
{
    k_pack_spairs<<<grid1d(pair_records(g), 256), 256, 0, st>>>(g, S, spair);
    return cudaGetLastError();
}

cudaError_t launch_fs32rec(const View32& p, double cut, int groups, const Rec32& rec,
                           unsigned long long* steps, cudaStream_t st)
{
    const int tiles = tiles32(p.g, kThreads32);
    if (p.pmajor && tiles32(p.g, 64) > 65535) return cudaErrorInvalidConfiguration;
    const dim3 grid = p.pmajor ? dim3(p.g.nz, tiles, groups) : dim3(tiles, p.g.nz, groups);
    k_fs32rec<<<grid, kThreads32, 0, st>>>(p, (float)cut, steps, rec);
    return cudaGetLastError();
}


cudaError_t launch_pack_b2(const Geometry& g, const double* B, float2* b2, cudaStream_t st)
{
    k_pack_b2<<<grid1d(2LL * g.nx * g.ny, 256), 256, 0, st>>>(g, B, b2);
    return cudaGetLastError();
}

int block_threads32(int threads) { return threads == 64 || threads == 256 ? threads : kThreads32; }

cudaError_t launch_fs32d(const View32& p, double cut, int groups, int threads,
                         unsigned long long* steps, cudaStream_t st, unsigned long long* series)
{
    // planes in index order (g.zorder unused): with the plane read from the
    // order table the march ran at 14.6 instead of 10.7 ms on the 65^3 slab
    const int tb = block_threads32(threads);
    auto shape = [&](int t) {
        const int tiles = tiles32(p.g, t);
        return p.pmajor ? dim3(p.g.nz, tiles, groups) : dim3(tiles, p.g.nz, groups);
    };
    if (p.pmajor && tiles32(p.g, 64) > 65535) return cudaErrorInvalidConfiguration;
    const dim3 grid = shape(tb);
    const float c = (float)cut;
    if (series)   // diagnostics: the branch-counting instantiation, 128 threads
        k_fs32d<kThreads32, true><<<shape(kThreads32), kThreads32, 0, st>>>(p, c, steps, series);
    else if (tb == 64)
        k_fs32d<64, false><<<grid, 64, 0, st>>>(p, c, steps, nullptr);
    else if (tb == 256)
        k_fs32d<256, false><<<grid, 256, 0, st>>>(p, c, steps, nullptr);
    else
        k_fs32d<kThreads32, false><<<grid, kThreads32, 0, st>>>(p, c, steps, nullptr);
    return cudaGetLastError();
}

long long fs32_blocks(const Geometry& g, int groups, int threads)
{
    return (long long)tiles32(g, block_threads32(threads)) * g.nz * groups;
}

cudaError_t launch_fs32_batch(const View32* views, const int* ids, const long long* prefix,
                              int nact, long long total_blocks, int groups, int threads, double cut,
                              unsigned long long* steps, cudaStream_t st)
{
    if (nact <= 0 || total_blocks <= 0) return cudaSuccess;
    dim3 grid((unsigned)total_blocks, 1, 1);
    if (total_blocks > 2147483647LL) {  // beyond grid.x: fold into y, surplus blocks return
        grid.x = 1u << 30;
        grid.y = (unsigned)((total_blocks + grid.x - 1) / grid.x);
    }
    const int tb = block_threads32(threads);
    const float c = (float)cut;
    if (tb == 64)
        k_fs32_batch<64><<<grid, 64, 0, st>>>(views, ids, prefix, nact, groups, c, steps);
    else if (tb == 256)
        k_fs32_batch<256><<<grid, 256, 0, st>>>(views, ids, prefix, nact, groups, c, steps);
    else
        k_fs32_batch<kThreads32><<<grid, kThreads32, 0, st>>>(views, ids, prefix, nact, groups, c,
                                                              steps);
    return cudaGetLastError();
}

cudaError_t launch_fs32rep_batch(const Rep32* views, const int* ids, const long long* prefix,
                                 int nact, long long total_blocks, int groups, int threads,
                                 unsigned long long* steps, cudaStream_t st)
{
    if (nact <= 0 || total_blocks <= 0) return cudaSuccess;
    dim3 grid((unsigned)total_blocks, 1, 1);
    if (total_blocks > 2147483647LL) {  // beyond grid.x: fold into y, surplus blocks return
        grid.x = 1u << 30;
        grid.y = (unsigned)((total_blocks + grid.x - 1) / grid.x);
    }
    const int tb = block_threads32(threads);
    if (tb == 64)
        k_fs32rep_batch<64><<<grid, 64, 0, st>>>(views, ids, prefix, nact, groups, steps);
    else if (tb == 256)
        k_fs32rep_batch<256><<<grid, 256, 0, st>>>(views, ids, prefix, nact, groups, steps);
    else
        k_fs32rep_batch<kThreads32><<<grid, kThreads32, 0, st>>>(views, ids, prefix, nact, groups,
                                                                 steps);
    return cudaGetLastError();
}

cudaError_t launch_delta_source(long long N, const double* S, const double* Sref, double* dS,
                                cudaStream_t st)
{
    k_delta_source<<<grid1d(N, 256), 256, 0, st>>>(N, S, Sref, dS);
    return cudaGetLastError();
}

cudaError_t launch_absmin(long long N, const double* x, double* out, cudaStream_t st)
{
    k_absmin<<<1, 256, 0, st>>>(N, x, out);
    return cudaGetLastError();
}

cudaError_t launch_sum_groups_ref(long long N, const double* partial, const double* dS,
                                  double wsum, const double* Jref, double* J, cudaStream_t st)
{
    k_sum_groups_ref<<<grid1d(N, 256), 256, 0, st>>>(N, partial, dS, wsum, Jref, J);
    return cudaGetLastError();
}

cudaError_t launch_sum_groups_src(long long N, const double* partial, const double* S,
                                  double wsum, double* J, cudaStream_t st)
{
    k_sum_groups_src<<<grid1d(N, 256), 256, 0, st>>>(N, partial, S, wsum, J);
    return cudaGetLastError();
}

cudaError_t launch_fs32rep(const Rep32& p, int groups, int threads, unsigned long long* steps,
                           cudaStream_t st)
{
    const int tb = block_threads32(threads);
    if (p.pmajor && tiles32(p.g, 64) > 65535) return cudaErrorInvalidConfiguration;
    const int tiles = tiles32(p.g, tb);
    const dim3 grid = p.pmajor ? dim3(p.g.nz, tiles, groups) : dim3(tiles, p.g.nz, groups);
    if (tb == 64)
        k_fs32rep<64><<<grid, 64, 0, st>>>(p, steps);
    else if (tb == 256)
        k_fs32rep<256><<<grid, 256, 0, st>>>(p, steps);
    else
        k_fs32rep<kThreads32><<<grid, kThreads32, 0, st>>>(p, steps);
    return cudaGetLastError();
}

}  // namespace rt3d
