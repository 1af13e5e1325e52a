// Short-characteristics formal solution (FP64): the O(1)-per-(voxel,
// direction) alternative to the long characteristics (Hauschildt & Baron
// 2011, Sect. 2.2, where the characteristics are tracked at O(1) cost per
// pair).  Per direction the z-planes are taken in the order of propagation;
// each node of a plane takes its intensity from the upstream point on the
// preceding plane only,
//   I(i,j,k) = I(p) e + w_cur S(i,j,k) + w_up S(p),  p = (i - ax, j - ay, k - s),
// I(p), chi(p), S(p) bilinear in that plane; on the entry plane I = I_bc at
// the node.  The upstream point of every node shares the lattice offset and
// bilinear weights of step 1 of the direction tables.
//
// Mapping: one thread block per direction walks the planes, holding the
// preceding and the current plane of I (in shared memory when two planes
// fit, else in a global scratch per block), with one barrier per plane.
// Each block writes w_d I_d for every voxel to its own slice of a
// [directions][N] buffer; a second kernel sums the slices in direction
// order, so J does not depend on the launch shape.  Directions are taken in
// chunks of at most kScChunk, each chunk's sum added to J in order.
#include "internal.h"
#include "weights.cuh"

namespace rt3d {

namespace {

constexpr int kScThreads = 256;
constexpr int kLsThreads = 128;                 // Lambda* kernel
constexpr int kScChunk = 1024;                  // directions per march launch
constexpr long long kScSmemMax = 200 * 1024;    // two planes of I in shared memory up to this

struct Corners {
    int a00, a10, a01, a11;
};

// Nodes of the upstream point of node (i, j): (i + ox, j + oy) and the next
// ones, periodic (ox in [0, nx), oy in [0, ny)).
__device__ __forceinline__ Corners corners_of(int i, int j, StepGeo o, int nx, int ny)
{
    int x0 = i + o.ox;
    x0 -= x0 >= nx ? nx : 0;
    const int x1 = x0 + 1 == nx ? 0 : x0 + 1;
    int y0 = j + o.oy;
    y0 -= y0 >= ny ? ny : 0;
    const int y1 = y0 + 1 == ny ? 0 : y0 + 1;
    return Corners{y0 * nx + x0, y0 * nx + x1, y1 * nx + x0, y1 * nx + x1};
}

__device__ __forceinline__ double bilin4(const double* f, Corners c, Bw4d b)
{
    return b.x * f[c.a00] + b.y * f[c.a10] + b.z * f[c.a01] + b.w * f[c.a11];
}

__device__ __forceinline__ double bilin4_ldg(const double* __restrict__ f, Corners c, Bw4d b)
{
    return b.x * __ldg(f + c.a00) + b.y * __ldg(f + c.a10) + b.z * __ldg(f + c.a01) +
           b.w * __ldg(f + c.a11);
}

template <bool SMEM>
__global__ void __launch_bounds__(kScThreads)
k_sc64(Geometry g, const double* __restrict__ chi, const double* __restrict__ S,
       const double* __restrict__ B, const double* __restrict__ G,
       const DirInfo* __restrict__ info, const StepGeo* __restrict__ off,
       const Bw4d* __restrict__ bw, int d0, double* __restrict__ part, double* gplanes,
       unsigned long long* __restrict__ steps)
{
    extern __shared__ double splanes[];
    __shared__ double tab[kExpTable];
    fill_exp_table(tab);
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const int d = d0 + blockIdx.x;
    double* pl = SMEM ? splanes : gplanes + (long long)blockIdx.x * 2 * nxy;
    const DirInfo di = info[d];
    const int s = di.sgn;
    const StepGeo o = off[(long long)d * nz + 1];
    const Bw4d b = bw[(long long)d * nz + 1];
    const int bc = s > 0 ? g.top_bc : g.bottom_bc;
    const int kin = s > 0 ? 0 : nz - 1;
    double* out = part + (long long)blockIdx.x * g.N;
    // entry plane: I = I_bc at the node
    for (int t = threadIdx.x; t < nxy; t += kScThreads) {
        double I = 0.0;
        if (bc) {
            I = B[(long long)kin * nxy + t];
            if (bc == 2) I = fma(di.amu, G[t], I);
        }
        pl[t] = I;
        out[(long long)kin * nxy + t] = di.w * I;
    }
    __syncthreads();   // also publishes tab
    int cur = 0;
    for (int n = 1; n < nz; ++n) {
        const int k = s > 0 ? n : nz - 1 - n;
        const int ku = k - s;
        const double* prev = pl + cur * nxy;
        double* next = pl + (cur ^ 1) * nxy;
        const double* chik = chi + (long long)k * nxy;
        const double* chiu = chi + (long long)ku * nxy;
        const double* Sk = S + (long long)k * nxy;
        const double* Su = S + (long long)ku * nxy;
        double* outk = out + (long long)k * nxy;
        for (int t = threadIdx.x; t < nxy; t += kScThreads) {
            const int j = t / nx, i = t - j * nx;
            const Corners c = corners_of(i, j, o, nx, ny);
            RT_GUARD(g, max(max(c.a00, c.a10), max(c.a01, c.a11)), nxy, kSiteSc) continue;
            RT_GUARD(g, min(min(c.a00, c.a10), min(c.a01, c.a11)), nxy, kSiteSc) continue;
            const double Iu = bilin4(prev, c, b);
            const double cu = bilin4_ldg(chiu, c, b);
            const double su = bilin4_ldg(Su, c, b);
            double wc, wu, e;
            seg_weights64(di.hs * (cu + __ldg(chik + t)), tab, wc, wu, e);
            const double I = fma(Iu, e, fma(wc, __ldg(Sk + t), wu * su));
            next[t] = I;
            outk[t] = di.w * I;
        }
        __syncthreads();
        cur ^= 1;
    }
    if (steps && threadIdx.x == 0) atomicAdd(steps, (unsigned long long)(nz - 1) * nxy);
}

// J[v] (=, or += if accumulate) sum over q < nd of part[q][v], in q order.
__global__ void k_sc_reduce(long long N, int nd, const double* __restrict__ part,
                            double* __restrict__ J, int accumulate)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
        double acc = accumulate ? J[v] : 0.0;
        for (int q = 0; q < nd; ++q) acc += part[(long long)q * N + v];
        J[v] = acc;
    }
}

// Lambda* of the short characteristics: per direction the diagonal w_cur
// of the voxel's segment and, at the four nodes c of its upstream point,
// b_c (w_up + e w_cur(c)), w_cur(c) the weight of c's own last segment (0
// on the entry plane).  One thread per voxel, directions in order.
__global__ void __launch_bounds__(kLsThreads)
k_lstar_sc64(Geometry g, const double* __restrict__ chi, const DirInfo* __restrict__ info,
             const StepGeo* __restrict__ off, const Bw4d* __restrict__ bw,
             double* __restrict__ lstar)
{
    __shared__ double lam[27][kLsThreads];
    __shared__ double tab[kExpTable];
    for (int q = 0; q < 27; ++q) lam[q][threadIdx.x] = 0.0;
    fill_exp_table(tab);
    __syncthreads();
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    const int t = blockIdx.x * kLsThreads + threadIdx.x;
    const int k0 = blockIdx.y;
    if (t >= nxy) return;
    const int j0 = t / nx, i0 = t - j0 * nx;
    const long long v = (long long)k0 * nxy + t;
    const double chi0 = chi[v];
    for (int d = 0; d < g.ndir; ++d) {
        const DirInfo di = info[d];
        const int s = di.sgn;
        const int kin = s > 0 ? 0 : nz - 1;
        if (k0 == kin) continue;
        const int ku = k0 - s;
        const StepGeo o = off[(long long)d * nz + 1];
        const Bw4d b = bw[(long long)d * nz + 1];
        const Corners c = corners_of(i0, j0, o, nx, ny);
        RT_GUARD(g, max(max(c.a00, c.a10), max(c.a01, c.a11)), nxy, kSiteLstarSc) continue;
        RT_GUARD(g, min(min(c.a00, c.a10), min(c.a01, c.a11)), nxy, kSiteLstarSc) continue;
        const double* chiu = chi + (long long)ku * nxy;
        double wc, wu, e;
        seg_weights64(di.hs * (bilin4_ldg(chiu, c, b) + chi0), tab, wc, wu, e);
        lam[13][threadIdx.x] += di.w * wc;
        const int cn[4] = {c.a00, c.a10, c.a01, c.a11};
        const double bq[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int lo = di.lo[q];
            if (lo < 0) continue;
            double wcc = 0.0;
            if (ku != kin) {   // then plane ku - s exists
                const int jc = cn[q] / nx, ic = cn[q] - jc * nx;
                const Corners cc = corners_of(ic, jc, o, nx, ny);
                double wuc, ec;
                seg_weights64(di.hs * (bilin4_ldg(chi + (long long)(ku - s) * nxy, cc, b) +
                                       __ldg(chiu + cn[q])),
                              tab, wcc, wuc, ec);
            }
            lam[lo][threadIdx.x] += di.w * bq[q] * (wu + e * wcc);
        }
    }
    for (int q = 0; q < 27; ++q) lstar[(long long)q * g.N + v] = lam[q][threadIdx.x];
}

bool sc_planes_in_smem(const Geometry& g) { return 16LL * g.nx * g.ny <= kScSmemMax; }

}  // namespace

int sc_chunk(const Geometry& g) { return g.ndir < kScChunk ? g.ndir : kScChunk; }

size_t sc_scratch_planes(const Geometry& g)
{
    return sc_planes_in_smem(g) ? 0 : (size_t)sc_chunk(g) * 2 * g.nx * g.ny;
}

cudaError_t launch_sc64(const Geometry& g, const double* chi, const double* S, const double* B,
                        const double* G, const DirInfo* info, const StepGeo* off,
                        const Bw4d* bw, double* part, double* gplanes, double* J,
                        unsigned long long* steps, cudaStream_t st)
{
    const int chunk = sc_chunk(g);
    const bool smem = sc_planes_in_smem(g);
    const size_t shm = smem ? 16 * (size_t)g.nx * g.ny : 0;
    if (smem) {
        cudaError_t e = cudaFuncSetAttribute(k_sc64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)shm);
        if (e != cudaSuccess) return e;
    }
    long long rb = (g.N + 255) / 256;
    if (rb > 152LL * 16) rb = 152LL * 16;
    for (int d0 = 0; d0 < g.ndir; d0 += chunk) {
        const int nd = g.ndir - d0 < chunk ? g.ndir - d0 : chunk;
        if (smem)
            k_sc64<true><<<nd, kScThreads, shm, st>>>(g, chi, S, B, G, info, off, bw, d0, part,
                                                      gplanes, steps);
        else
            k_sc64<false><<<nd, kScThreads, 0, st>>>(g, chi, S, B, G, info, off, bw, d0, part,
                                                     gplanes, steps);
        k_sc_reduce<<<(unsigned)rb, 256, 0, st>>>(g.N, nd, part, J, d0 > 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_lstar_sc64(const Geometry& g, const double* chi, const DirInfo* info,
                              const StepGeo* off, const Bw4d* bw, double* lstar, cudaStream_t st)
{
    dim3 grid((g.nx * g.ny + kLsThreads - 1) / kLsThreads, g.nz);
    k_lstar_sc64<<<grid, kLsThreads, 0, st>>>(g, chi, info, off, bw, lstar);
    return cudaGetLastError();
}

}  // namespace rt3d
