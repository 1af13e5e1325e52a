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
// instead of S.  J = sum_d w_d S_0 + sum_d w_d (I_d - S_0) is accumulated in
// FP64.  Lambda*, the operator splitting and the convergence test are FP64.
//
// Layout: chi and the S pair are interleaved per node as float4
// {chi, S_hi, S_lo, 0} in planes padded to 2ny x 2nx by periodic copies, so
// that the four bilinear nodes of every upstream point are
// base(voxel) + off(direction, step) + {0, 1, 2nx, 2nx + 1}: one integer add
// per step and no wrap arithmetic.  B of the two boundary planes is kept as
// padded float2 {B_hi, B_lo}.
#include "internal.h"
#include "weights.cuh"

namespace rt3d {

namespace {

constexpr int kThreads32 = 128;

__global__ void k_pad_offsets(Geometry g, const DirInfo* __restrict__ info,
                              const StepGeo* __restrict__ off, int* __restrict__ poff)
{
    const int d = blockIdx.x;
    const int s = info[d].sgn;
    const long long W = 2LL * g.nx, H = 2LL * g.ny;
    for (int m = threadIdx.x; m < g.nz; m += blockDim.x) {
        const StepGeo o = off[(long long)d * g.nz + m];
        poff[(long long)d * g.nz + m] = (int)((-(long long)m * s * H + o.oy) * W + o.ox);
    }
}

__global__ void k_pack32(Geometry g, const double* __restrict__ chi, const double* __restrict__ S,
                         float4* __restrict__ node)
{
    const int nx = g.nx, ny = g.ny;
    const long long W = 2LL * nx, P = 4LL * nx * ny;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < g.N;
         v += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(v % nx), j = (int)((v / nx) % ny);
        const long long k = v / ((long long)nx * ny);
        const double s = S[v];
        const float hi = (float)s;
        const float4 q = make_float4((float)chi[v], hi, (float)(s - (double)hi), 0.f);
        float4* p = node + k * P + (long long)j * W + i;
        p[0] = q;
        p[nx] = q;
        p[(long long)ny * W] = q;
        p[(long long)ny * W + nx] = q;
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

// One thread per voxel of plane k0, tile `tile` (kThreads32 voxels); block z
// index zb of ZB walks the direction slots zb, zb + ZB, ... (d mod kSlots);
// partial[slot][v] = sum_{d in slot} w_d (I_d - S_0).
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
__device__ __forceinline__ void march32(const View32& p, int tile, int k0, int zb, int ZB,
                                        float cut, unsigned long long* __restrict__ steps)
{
    constexpr float kLog2e = 1.4426950408889634f;
    const Geometry& g = p.g;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const int t = tile * kThreads32 + threadIdx.x;
    const bool active = t < nxy;
    unsigned long long nsteps = 0;
    if (active) {
        const int j0 = t / nx, i0 = t - j0 * nx;
        const long long v = (long long)k0 * nxy + t;
        const long long W = 2LL * nx, P = 4LL * nxy;
        const long long base = k0 * P + j0 * W + i0;
        const float4 me = p.node[base];
        const float chi0 = me.x, s0h = me.y, s0l = me.z;
        const float s0 = s0h + s0l;
        // The rest of a characteristic changes I - S_0 by at most
        // T * max|S - S_0| <= T * 2 smax: stop once that is below cut * S_0.
        const float smax = (float)*p.smax;
        const float tcut = smax > 0.f ? cut * s0 / (2.0f * smax) : 0.f;
        const float4* nb = p.node + base;
        for (int slot = zb; slot < kSlots; slot += ZB) {
            double Jp = 0.0;
            for (int d = slot; d < g.ndir; d += kSlots) {
                const DirInfo di = p.info[d];
                const int s = di.sgn;
                const int M = s > 0 ? k0 : nz - 1 - k0;
                const int* od = p.poff + (long long)d * nz;
                const float4* bd = p.bw + (long long)d * nz;
                float I = 0.f, Ilo = 0.f, T = 1.f, tau = 0.f, ca = chi0, da = 0.f;
                bool early = false;
                int m = 0;
                for (; m < M; ++m) {
                    RT_GUARD(g, base + od[m + 1], 4 * g.N, kSiteFs32) { early = true; break; }
                    RT_GUARD(g, base + od[m + 1] + W + 1, 4 * g.N, kSiteFs32) { early = true; break; }
                    const float4* q = nb + od[m + 1];
                    const float4 b = bd[m + 1];
                    const float4 q00 = __ldg(q), q10 = __ldg(q + 1);
                    const float4 q01 = __ldg(q + W), q11 = __ldg(q + W + 1);
                    const float cb = b.x * q00.x + b.y * q10.x + b.z * q01.x + b.w * q11.x;
                    // S(p) - S_0: hi differences are exact for nearby values
                    const float dh = b.x * (q00.y - s0h) + b.y * (q10.y - s0h) +
                                     b.z * (q01.y - s0h) + b.w * (q11.y - s0h);
                    const float dl = b.x * q00.z + b.y * q10.z + b.z * q01.z + b.w * q11.z;
                    const float db = dh + (dl - s0l);
                    const float x = di.hs32 * (ca + cb);
                    float wc, wu, e;
                    seg_weights32(x, wc, wu, e);
                    // I - S_0 += T (w_cur D_m + w_up D_m+1), TwoSum
                    const float inc = T * fmaf(wc, da, wu * db);
                    const float sI = I + inc, bb = sI - I;
                    Ilo += (I - (sI - bb)) + (inc - bb);
                    I = sI;
                    tau += x;
                    T = ex2_approx(-tau * kLog2e);
                    ca = cb;
                    da = db;
                    if (T <= tcut) {
                        early = true;
                        ++m;
                        break;
                    }
                }
                if (!early) {
                    // boundary term T_M (I_bc - S_0), added with its rounding error
                    float inc, inc_lo;
                    const int bc = s > 0 ? g.top_bc : g.bottom_bc;
                    if (bc) {
                        const StepGeo o = p.off[(long long)d * nz + M];
                        const float4 b = bd[M];
                        long long ip = (j0 + o.oy) * W + (i0 + o.ox);
                        RT_GUARD(g, ip, P - W - 1, kSiteFs32) ip = 0;   // record, read a safe node
                        const float2* pb = p.b2 + (s > 0 ? 0LL : P) + ip;
                        const float2 c00 = pb[0], c10 = pb[1], c01 = pb[W], c11 = pb[W + 1];
                        const float h = b.x * (c00.x - s0h) + b.y * (c10.x - s0h) +
                                        b.z * (c01.x - s0h) + b.w * (c11.x - s0h);
                        const float l = b.x * c00.y + b.y * c10.y + b.z * c01.y + b.w * c11.y;
                        float ibc = h + (l - s0l);
                        if (bc == 2) {   // + |mu| dB/dtau (LTE diffusion)
                            // |mu| read here, not kept live through the march
                            // loop (that cost the loop 13%)
                            const float* pg = p.g2 + ip;
                            ibc = fmaf(__ldg(&p.info[d].amu32),
                                       b.x * pg[0] + b.y * pg[1] + b.z * pg[W] + b.w * pg[W + 1], ibc);
                        }
                        inc = T * ibc;
                        inc_lo = fmaf(T, ibc, -inc);
                    } else {
                        inc = -T * s0h;
                        inc_lo = fmaf(-T, s0h, -inc) - T * s0l;
                    }
                    const float sI = I + inc, bb = sI - I;
                    Ilo += (I - (sI - bb)) + (inc - bb) + inc_lo;
                    I = sI;
                }
                nsteps += (unsigned long long)m;
                Jp = fma(di.w, (double)I + (double)Ilo, Jp);
            }
            p.partial[(long long)slot * g.N + v] = Jp;
        }
    }
    if (steps) add_steps32(steps, nsteps);
}

__global__ void __launch_bounds__(kThreads32)
k_fs32d(View32 p, float cut, unsigned long long* __restrict__ steps)
{
    march32(p, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.z, cut, steps);
}

// Many problems in one launch: block b belongs to the active problem q with
// prefix[q] <= b < prefix[q+1]; within it, blocks run tile-fastest, then
// plane, then slot group.
__global__ void __launch_bounds__(kThreads32)
k_fs32_batch(const View32* __restrict__ views, const int* __restrict__ ids,
             const long long* __restrict__ prefix, int nact, int ZB, float cut,
             unsigned long long* __restrict__ steps)
{
    const long long b = blockIdx.x + (long long)blockIdx.y * gridDim.x;
    int lo = 0, hi = nact;  // prefix[lo] <= b < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= b) lo = mid; else hi = mid;
    }
    if (b >= prefix[nact]) return;
    const View32& p = views[ids[lo]];
    const long long local = b - prefix[lo];
    const int tiles = (p.g.nx * p.g.ny + kThreads32 - 1) / kThreads32;
    const int tile = (int)(local % tiles);
    const int k0 = (int)((local / tiles) % p.g.nz);
    const int zb = (int)(local / ((long long)tiles * p.g.nz));
    march32(p, tile, k0, zb, ZB, cut, steps);
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

cudaError_t launch_pad_offsets(const Geometry& g, const DirInfo* info, const StepGeo* off,
                               int* poff, cudaStream_t st)
{
    k_pad_offsets<<<g.ndir, 128, 0, st>>>(g, info, off, poff);
    return cudaGetLastError();
}

cudaError_t launch_pack32(const Geometry& g, const double* chi, const double* S, float4* node,
                          cudaStream_t st)
{
    k_pack32<<<grid1d(g.N, 256), 256, 0, st>>>(g, chi, S, node);
    return cudaGetLastError();
}

cudaError_t launch_pack_b2(const Geometry& g, const double* B, float2* b2, cudaStream_t st)
{
    k_pack_b2<<<grid1d(2LL * g.nx * g.ny, 256), 256, 0, st>>>(g, B, b2);
    return cudaGetLastError();
}

cudaError_t launch_fs32d(const View32& p, double cut, int groups, unsigned long long* steps,
                         cudaStream_t st)
{
    const int nxy = p.g.nx * p.g.ny;
    // planes in index order (g.zorder unused): with the plane read from the
    // order table the march ran at 14.6 instead of 10.7 ms on the 65^3 slab
    dim3 grid((nxy + kThreads32 - 1) / kThreads32, p.g.nz, groups);
    k_fs32d<<<grid, kThreads32, 0, st>>>(p, (float)cut, steps);
    return cudaGetLastError();
}

long long fs32_blocks(const Geometry& g, int groups)
{
    return (long long)((g.nx * g.ny + kThreads32 - 1) / kThreads32) * g.nz * groups;
}

cudaError_t launch_fs32_batch(const View32* views, const int* ids, const long long* prefix,
                              int nact, long long total_blocks, int groups, double cut,
                              unsigned long long* steps, cudaStream_t st)
{
    if (nact <= 0 || total_blocks <= 0) return cudaSuccess;
    dim3 grid((unsigned)total_blocks, 1, 1);
    if (total_blocks > 2147483647LL) {  // beyond grid.x: fold into y, surplus blocks return
        grid.x = 1u << 30;
        grid.y = (unsigned)((total_blocks + grid.x - 1) / grid.x);
    }
    k_fs32_batch<<<grid, kThreads32, 0, st>>>(views, ids, prefix, nact, groups, (float)cut, steps);
    return cudaGetLastError();
}

cudaError_t launch_sum_groups_src(long long N, const double* partial, const double* S,
                                  double wsum, double* J, cudaStream_t st)
{
    k_sum_groups_src<<<grid1d(N, 256), 256, 0, st>>>(N, partial, S, wsum, J);
    return cudaGetLastError();
}

}  // namespace rt3d
