// Internal declarations shared by the translation units of librt3d.so.
// Not part of the public ABI (include/rt3d.h is).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace rt3d {

// Directions are summed into J in kSlots fixed slots (d mod kSlots), each in
// increasing d, then the slots in order: J is independent of the launch
// shape.  The formal solution writes kSlots partial sums per voxel.
constexpr int kSlots = 8;

// Per-direction constants of the march (one entry per direction).
struct DirInfo {
    double hs;      // half path length per z-plane step, dz / (2 |mu|)
    double w;       // quadrature weight
    int sgn;        // +1: propagates to larger k (entered at the top), -1: from the bottom
    int lo[4];      // Lambda* offset index of the four bilinear nodes of p_1, -1 if none
    float hs32;     // hs in FP32 (sweep form)
    float amu32;    // |mu| in FP32
    float w32;      // w in FP32 (sweep form)
    double amu;     // |mu| (LTE-diffusion boundary)
    float hs32lo;   // hs - hs32: hs as a double-float pair (RT_DF64 march)
    float amu32lo;  // |mu| - amu32
};

// Per-(direction, step m) lattice geometry.  The upstream point p_m of voxel
// (i0, j0) lies at (i0 - m ax, j0 - m ay); because voxel centres are lattice
// points its integer part and fraction do not depend on the voxel:
//   node x0 = (i0 + ox) mod nx, x1 = x0 + 1 (mod nx), likewise y, and the
//   bilinear weights of (x0,y0), (x1,y0), (x0,y1), (x1,y1).
struct StepGeo {
    int ox, oy;
};

// Bilinear weights of (x0,y0), (x1,y0), (x0,y1), (x1,y1) in FP64.
struct alignas(32) Bw4d {
    double x, y, z, w;
};

// Downstream point p_{-1} = (i0 + ax, j0 + ay) of a direction (parabolic
// source): lattice offset, bilinear weights, and the Lambda* offset index of
// its four nodes on plane k0 + s (-1 where not a nearest neighbour).
struct alignas(32) DownGeo {
    Bw4d b;
    int ox, oy;
    int ld[4];
};

struct Geometry {
    int nx, ny, nz, ndir;
    long long N;            // nx * ny * nz
    int top_bc, bottom_bc;  // 0 zero, 1 Planck, 2 (bottom) LTE diffusion
    // Checked builds only: device record {hit, site, index, limit} of the
    // first gathered index found outside its buffer (null: no record).
    unsigned long long* berr;
    // Dispatch order of the planes in the FP64 march launches: the blocks
    // of plane rank r work on plane zorder[r]; null means plane r.  A
    // permutation of 0..nz-1 whenever it is set.
    const int* zorder;
};

// Plane worked on by the blocks of dispatch rank r.
__host__ __device__ __forceinline__ int plane_at(const Geometry& g, int r)
{
    return g.zorder ? g.zorder[r] : r;
}

// Checked builds (compiled with -DRT_CHECKED into librt3d_checked.so): the
// gathers of the marches and of the operator-splitting stencils test each
// index against its buffer before the access.  The first index found
// outside is recorded in g.berr and the access is skipped (RT_GUARD runs
// its statement: leave the characteristic, skip the voxel), so the kernel
// runs to its end and the host reports RT_EBOUNDS instead of the GPU
// faulting.  In normal builds RT_GUARD compiles to nothing.
#ifdef RT_CHECKED
__device__ __forceinline__ bool rt_in_bounds(const Geometry& g, long long i, long long n, int site)
{
    if (i >= 0 && i < n) return true;
    if (g.berr && atomicCAS(g.berr, 0ull, 1ull) == 0ull) {
        g.berr[1] = (unsigned long long)site;
        g.berr[2] = (unsigned long long)i;
        g.berr[3] = (unsigned long long)n;
    }
    return false;
}
#define RT_GUARD(g, i, n, site) if (!rt_in_bounds((g), (long long)(i), (long long)(n), (site)))
#else
#define RT_GUARD(g, i, n, site) if (false)
#endif
// Sites named in the RT_EBOUNDS message.
enum {
    kSiteFs64 = 1, kSiteLstar64 = 2, kSiteFs32 = 3, kSiteFsdf = 4, kSiteSc = 5,
    kSiteLstarSc = 6, kSiteFs64p = 7, kSiteLstar64p = 8, kSiteStencil = 9, kSiteGs = 10,
    kSiteSelfTest = 99
};
// Launch one guard on an index that is never dereferenced (index = limit),
// so that a checked build records site kSiteSelfTest (a no-op otherwise).
cudaError_t launch_bounds_selftest(const Geometry& g, cudaStream_t st);

// ---- launchers (fs.cu) -----------------------------------------------------
// Per (direction d, step m) at index d * nz + m: off (lattice offset), bw
// (bilinear weights), bwh (the weights times hs = dz / (2 |mu|), so that
// interpolating chi with them gives hs chi) and bw32 (bw in FP32).
cudaError_t launch_dir_tables(const Geometry& g, double dx, double dy, double dz,
                              const double* mu, const double* phi, const double* w,
                              DirInfo* info, StepGeo* off, Bw4d* bw, Bw4d* bwh, float4* bw32,
                              cudaStream_t st);

// Plane dispatch order of the FP64 march launches, heaviest plane first: the
// march work of each plane is estimated from the plane means of chi (steps
// until an optical depth of 40 or the boundary, upward and downward, for
// |mu| = 1, 1/2, 1/5), and order[r] is the plane of rank r (ties by plane
// index).  scratch: 2 nz doubles.  Light planes dispatched last fill the end
// of the launch, where otherwise a partial wave of heavy blocks would run
// alone.
cudaError_t launch_plane_order(const Geometry& g, double dz, const double* chi, double* scratch,
                               int* order, cudaStream_t st);

// The FP64 march recorded as a linear map of the source S (the opacities,
// directions and boundary values fixed): J = sum_slots [c0 S_v + bc +
// sum_{d in slot} w_d sum_{m=1..L} c_m S(p_m)].
//   coef: c_m of voxel t of plane k0 and direction d at
//     rec_base(g, d, k0, sgn_d) + (m-1) nx ny + t, m = 1..M (M the steps to
//     the boundary plane), zero past the ray's own length;
//   lmax[(d nz + k0) nwp + t/32]: the longest ray of the warp, the length
//     the replay runs (nwp = warps per plane);
//   c0, bc [kSlots][N]: the voxel's own coefficient and the boundary term.
struct FsRec {
    double* coef;
    int* lmax;
    double* c0;
    double* bc;
    int nwp;
    // parabolic source: cdn[d N + v], the coefficient of S at the
    // downstream point p_-1 (DownGeo) of voxel v in direction d; null for
    // the linear source
    double* cdn;
    const DownGeo* dn;
};
// The recording march cuts the characteristics at cut * kRecCutMargin, so
// that the recorded lengths still meet the cutoff for sources whose
// intensities are up to 1/kRecCutMargin times smaller.
constexpr double kRecCutMargin = 1e-2;
__host__ __device__ __forceinline__ long long rec_base(const Geometry& g, int d, int k0, int sgn)
{
    const long long nxy = (long long)g.nx * g.ny;
    const long long k = k0;
    const long long before = sgn > 0 ? k * (k - 1) / 2 : k * (g.nz - 1) - k * (k - 1) / 2;
    return ((long long)d * ((long long)g.nz * (g.nz - 1) / 2) + before) * nxy;
}
// Device bytes of an FsRec for grid g (coefficients, lengths, c0 and bc).
long long rec_bytes(const Geometry& g);

// FP64 formal solution: partial[kSlots][N]; `groups` (1..kSlots) is the
// number of z-blocks walking the slots (a tuning knob, no effect on J).
// G[ny][nx]: dB/dtau at the bottom nodes (LTE-diffusion inner boundary),
// read only when bottom_bc == 2 (may be null otherwise).  rec != null:
// also record the march into *rec (FsRec), cut at cut * kRecCutMargin.
cudaError_t launch_fs64(const Geometry& g, const double* chi, const double* S, const double* B,
                        const double* G, const DirInfo* info, const StepGeo* off,
                        const Bw4d* bw, const Bw4d* bwh, const double* smax, double cut,
                        int groups, double* partial, unsigned long long* steps, cudaStream_t st,
                        const FsRec* rec = nullptr);
// The recorded march for source S: partial[kSlots][N] as launch_fs64.
cudaError_t launch_fs64rep(const Geometry& g, const double* S, const DirInfo* info,
                           const StepGeo* off, const Bw4d* bw, const FsRec& rec, int groups,
                           double* partial, unsigned long long* steps, cudaStream_t st);
// G[j][i] = (B[nz-1] - B[nz-2]) / (dz (chi[nz-1] + chi[nz-2]) / 2), and its
// padded FP32 copy g2[2ny][2nx] if g2 != null.
cudaError_t launch_diffusion_grad(const Geometry& g, double dz, const double* chi,
                                  const double* B, double* G, float* g2, cudaStream_t st);

// ---- parabolic source (para.cu) --------------------------------------------
cudaError_t launch_down_tables(const Geometry& g, double dx, double dy, double dz,
                               const double* mu, const double* phi, DownGeo* dn, cudaStream_t st);
// As launch_fs64 with the parabolic source (rec != null: also record it,
// with rec->cdn, cut at cut * kRecCutMargin).
cudaError_t launch_fs64p(const Geometry& g, const double* chi, const double* S, const double* B,
                         const double* G, const DirInfo* info, const StepGeo* off,
                         const Bw4d* bw, const DownGeo* dn, const double* smax, double cut,
                         int groups, double* partial, unsigned long long* steps, cudaStream_t st,
                         const FsRec* rec = nullptr);
cudaError_t launch_lstar64p(const Geometry& g, const double* chi, const DirInfo* info,
                            const StepGeo* off, const Bw4d* bw, const DownGeo* dn, double* lstar,
                            cudaStream_t st);

// ---- short characteristics (sc.cu) -----------------------------------------
// Directions per march launch (the [directions][N] partial buffer holds
// sc_chunk(g) slices) and the global plane scratch it needs (doubles; 0 when
// two planes of I fit in shared memory).
int sc_chunk(const Geometry& g);
size_t sc_scratch_planes(const Geometry& g);
// J[N] = sum_d w_d I_d of the short-characteristics march; part holds
// sc_chunk(g) * N doubles, gplanes sc_scratch_planes(g) doubles (or null).
cudaError_t launch_sc64(const Geometry& g, const double* chi, const double* S, const double* B,
                        const double* G, const DirInfo* info, const StepGeo* off,
                        const Bw4d* bw, double* part, double* gplanes, double* J,
                        unsigned long long* steps, cudaStream_t st);
// Lambda* [27][N] of the short characteristics.
cudaError_t launch_lstar_sc64(const Geometry& g, const double* chi, const DirInfo* info,
                              const StepGeo* off, const Bw4d* bw, double* lstar, cudaStream_t st);

// ---- FP32-sweep form (fs32.cu) ---------------------------------------------
// poff[d][m]: offset of the upstream node (x0, y0) of step m from the
// voxel's own entry in planes of `rows` padded rows of 2nx entries
// ([nz][rows][2nx]; rows = 2ny for the double-float nodes, 2ny + 1 for the
// FP32 pair records).
cudaError_t launch_pad_offsets(const Geometry& g, const DirInfo* info, const StepGeo* off,
                               long long rows, int* poff, cudaStream_t st);
// Entries of the padded FP32 pair planes: nz * (2ny + 1) * 2nx.
long long pair_records(const Geometry& g);
// pair[k][y][x] = {chi, S_hi} of the nodes (x mod nx, y mod ny) and
// (x+1 mod nx, y mod ny); lo[k][y][x] = their S_lo (planes (2ny+1) x 2nx).
cudaError_t launch_pack_pairs(const Geometry& g, const double* chi, const double* S, float4* pair,
                              float2* lo, cudaStream_t st);
// b2[plane][y][x] = {B_hi, B_lo} of the top (0) and bottom (1) planes, padded.
cudaError_t launch_pack_b2(const Geometry& g, const double* B, float2* b2, cudaStream_t st);
// Everything the FP32 march of one problem reads and writes.
struct View32 {
    Geometry g;
    const float4* pair;     // padded pair records {chi, S_hi, chi', S_hi'}
    const float2* lo;       // padded {S_lo, S_lo'}
    const float2* b2;       // padded boundary {B_hi, B_lo}
    const float* g2;        // padded dB/dtau of the bottom nodes (diffusion boundary)
    const DirInfo* info;
    const StepGeo* off;
    const int* poff;        // offsets in the pair planes (rows = 2ny + 1)
    const float4* bw;       // FP32 bilinear weights per (direction, step)
    const double* smax;     // source bound of the cutoff
    // Null: the march's source is S itself and the cutoff is relative to
    // each voxel's S.  Otherwise the source is a change dS of a source whose
    // magnitude is at least *sfloor, and the cutoff is relative to that.
    const double* sfloor;
    double* partial;        // [kSlots][N]
    // Block order of the launch: 0 = tiles of a plane consecutive (the
    // resident blocks share a few planes), 1 = planes consecutive (they
    // share a few lateral tiles through every plane).
    int pmajor;
};
// Block order of the FP32 march for grid g: order 1 = tile-major, 2 =
// plane-major, 0 = automatic (plane-major once the padded pair planes
// exceed kPlaneMajorBytes, i.e. no longer stay in L2 together).
constexpr long long kPlaneMajorBytes = 64ll << 20;
int plane_major32(const Geometry& g, int order);
// The FP32-sweep march recorded as a linear map of the source (difference
// form): thread t of plane k0 marches voxels (i0, j0) and (i0, j0 + 1),
// t = (j0/2) nx + i0 < npair = nx ceil(ny/2);
//   coef: {c_m of the first voxel, of the second} at rec32_at(g, d, k0,
//     sgn_d, t) + rec32_step(m), m = 1..M, c_m the coefficient of
//     S(p_m) - S_0 (zero past the ray's cutoff);
//   lmax[(d nz + k0) nwp + t/32]: the warp's longest ray (nwp = warps per
//     plane of pairs);
//   tsum, bc [kSlots][N]: sum_{d in slot} w_d T_L and w_d T_L I_bc over the
//     rays that reach the boundary plane.
struct Rec32 {
    float2* coef;
    int* lmax;
    double* tsum;
    double* bc;
    int nwp;
};
// F(K) = sum_{k<K} 4 ceil(k/4): the steps of planes 0..K-1 rounded up to
// blocks of four.
__host__ __device__ __forceinline__ long long rec32_steps4(long long K)
{
    const int part[4] = {0, 0, 3, 5};
    return K * (K - 1) / 2 + 6 * (K / 4) + part[K & 3];
}
// Offset of the coefficients of thread t (step 1) of plane k0, direction
// d: per (direction, plane) one block per warp, [step/4][lane][step%4], so
// that each lane reads four steps' pairs with two 16-byte loads and the
// warp streams 1 KB per four steps; step m (1-based) is at
// rec32_at(...) + rec32_step(m).
__host__ __device__ __forceinline__ long long rec32_at(const Geometry& g, int d, int k0, int sgn,
                                                        int t)
{
    const long long nw = ((long long)g.nx * ((g.ny + 1) / 2) + 31) / 32;   // warps per plane
    const long long k = k0, nz = g.nz;
    const long long before = sgn > 0 ? rec32_steps4(k) : rec32_steps4(nz) - rec32_steps4(nz - k);
    const long long M = sgn > 0 ? k : nz - 1 - k;
    const long long M4 = (M + 3) / 4 * 4;
    return ((long long)d * rec32_steps4(nz) + before) * nw * 32 + (t >> 5) * M4 * 32 + (t & 31) * 4;
}
__host__ __device__ __forceinline__ long long rec32_step(int m)
{
    return (long long)((m - 1) >> 2) * 128 + ((m - 1) & 3);
}
// The replay: the source in spair (k_pack_spairs records), the march's
// geometry tables and block order, the recording; zero_bc: the boundary
// intensities are zero (the finishing stage's source change).
struct Rep32 {
    Geometry g;
    const float4* spair;
    const DirInfo* info;
    const int* poff;
    const float4* bw;
    Rec32 rec;
    double* partial;
    int zero_bc;
    int pmajor;
};
cudaError_t launch_pack_spairs(const Geometry& g, const double* S, float4* spair, cudaStream_t st);
// Record the march of p (cut at `cut`, the caller's stricter cutoff) into rec.
cudaError_t launch_fs32rec(const View32& p, double cut, int groups, const Rec32& rec,
                           unsigned long long* steps, cudaStream_t st);
cudaError_t launch_fs32rep(const Rep32& p, int groups, int threads, unsigned long long* steps,
                           cudaStream_t st);
// The replays of the problems ids[0..nact) (views in device memory, blocks
// as launch_fs32_batch: prefix of fs32_blocks per problem).
cudaError_t launch_fs32rep_batch(const Rep32* views, const int* ids, const long long* prefix,
                                 int nact, long long total_blocks, int groups, int threads,
                                 unsigned long long* steps, cudaStream_t st);

// FP32 march of I - S_0: partial[kSlots][N] of sum_d w_d (I_d - S_0).
// threads: threads per block, 64, 128 or 256 (anything else: 128); J does
// not depend on it.  series != null (diagnostics): a kernel instantiation
// that also counts the steps whose segment took the series branch of the
// weights (x < 2) into *series (same J).
cudaError_t launch_fs32d(const View32& p, double cut, int groups, int threads,
                         unsigned long long* steps, cudaStream_t st,
                         unsigned long long* series = nullptr);
// Blocks one problem takes in a batched launch with `groups` slot groups.
long long fs32_blocks(const Geometry& g, int groups, int threads);
// One launch over the active problems ids[0..nact) of views (device arrays);
// prefix[q] = first block of active problem q, prefix[nact] = total_blocks.
cudaError_t launch_fs32_batch(const View32* views, const int* ids, const long long* prefix,
                              int nact, long long total_blocks, int groups, int threads, double cut,
                              unsigned long long* steps, cudaStream_t st);
// ---- double-float march (fsdf.cu) -------------------------------------------
struct ViewDF {
    Geometry g;
    const float4* node;     // padded {chi_hi, chi_lo, S_hi, S_lo}
    const float2* b2;       // padded boundary {B_hi, B_lo}
    const float2* g2df;     // padded LTE-diffusion gradient {hi, lo}
    const DirInfo* info;
    const StepGeo* off;
    const int* poff;
    const float4* bw;       // per (direction, step): hi4, lo4 of the bilinear weights
    const double* smax;
    double* partial;        // [kSlots][N] of sum_d w_d (I_d - S_0)
};
// Double-float short characteristics (context in RT_DF64): J[N] = wsum S +
// sum_d w_d (I_d - S); part as for launch_sc64, gplanes 2 * sc_chunk(g) *
// nx * ny float2 when scdf_planes_in_smem(g) is false (else null).
cudaError_t launch_scdf(const ViewDF& p, const double* S, double wsum, double* part,
                        float2* gplanes, double* J, unsigned long long* steps, cudaStream_t st);
bool scdf_planes_in_smem(const Geometry& g);
// Lambda* [27][N] in double-float from the packed nodes (long or short
// characteristics).
cudaError_t launch_lstar_df(const ViewDF& p, bool short_chars, double* lstar, cudaStream_t st);
cudaError_t launch_packdf(const Geometry& g, const double* chi, const double* S, float4* node,
                          cudaStream_t st);
cudaError_t launch_bw_df(long long n, const Bw4d* bw, float4* out, cudaStream_t st);
cudaError_t launch_grad_df(const Geometry& g, const double* G, float2* out, cudaStream_t st);
// rec != null: also record the march (Rec32 in the layout of rec_base, one
// double-float pair per entry; lmax, tsum, bc as for the FP32 sweep).
cudaError_t launch_fsdf(const ViewDF& p, double cut, int groups, unsigned long long* steps,
                        cudaStream_t st, const Rec32* rec = nullptr);
// The recorded double-float march for the source in p.node.
cudaError_t launch_fsdfrep(const ViewDF& p, const Rec32& rec, int groups,
                           unsigned long long* steps, cudaStream_t st);

// Finishing stage of the FP32 sweep (formal solution of a source change):
// dS = S - Sref; *out = min |x|; J = Jref + wsum dS + sum_slot partial.
cudaError_t launch_delta_source(long long N, const double* S, const double* Sref, double* dS,
                                cudaStream_t st);
cudaError_t launch_absmin(long long N, const double* x, double* out, cudaStream_t st);
cudaError_t launch_sum_groups_ref(long long N, const double* partial, const double* dS,
                                  double wsum, const double* Jref, double* J, cudaStream_t st);

// J[v] = wsum S[v] + sum_slot partial[slot][v].
cudaError_t launch_sum_groups_src(long long N, const double* partial, const double* S,
                                  double wsum, double* J, cudaStream_t st);

// J[v] = sum_slot partial[slot][v] in slot order.
cudaError_t launch_sum_groups(long long N, const double* partial, double* J,
                              cudaStream_t st);

// Lambda* [27][N] (FP64, exact elements, first two steps of each characteristic).
cudaError_t launch_lstar64(const Geometry& g, const double* chi, const DirInfo* info,
                           const StepGeo* off, const Bw4d* bw, double* lstar,
                           cudaStream_t st);

// Diagnostic evaluation of the segment weights (FP64 or FP32 form).
cudaError_t launch_seg_eval(long long n, int fp32, const double* x, double* wc, double* wu,
                            double* e, cudaStream_t st);

// ---- launchers (os.cu) -----------------------------------------------------
// S = eps B + (1 - eps) J; smax = max(|S|, |B| if any Planck boundary).
cudaError_t launch_source(long long N, const double* eps, const double* B, const double* J,
                          double* S, float* S32, const double* Bbound, double* smax,
                          cudaStream_t st);
// smax = max(|S|, |B| if B != nullptr), also the FP32 copy of S if S32 != nullptr.
cudaError_t launch_absmax(long long N, const double* S, const double* B, double* smax,
                          float* S32, cudaStream_t st);
cudaError_t launch_to_float(long long N, const double* x, float* y, cudaStream_t st);

// Operator-splitting coefficients: c[o][v] = Lambda*_{v,o} (1 - eps_j) / diag_v,
// rdiag[v] = 1 / diag_v, diag_v = 1 - Lambda*_{v,13} (1 - eps_v).
// split: colour-split storage for red-black Gauss-Seidel (coef holds 27 *
// os_coef_stride(g, split) doubles, rdiag and r os_coef_stride(g, split)).
long long os_coef_stride(const Geometry& g, bool split);
cudaError_t launch_os_coef(const Geometry& g, const double* lstar, const double* eps,
                           double* coef, double* rdiag, bool split, cudaStream_t st);
// r[v] = J_fs[v] / diag_v - sum_o c[o][v] J_old[nb(v,o)]
cudaError_t launch_os_rhs(const Geometry& g, const double* coef, const double* rdiag,
                          const double* J_fs, const double* J_old, double* r, bool split,
                          cudaStream_t st);
// One red-black Gauss-Seidel sweep n (two launches), J -> Jn, same no-op
// and dlt rules as launch_jacobi; coef, r colour-split.
cudaError_t launch_gs_sweep(const Geometry& g, const double* coef, const double* r,
                            const double* J, double* Jn, double* dlt, int n, double tol,
                            cudaStream_t st);
// One pass of the device-side sweep loop (body of a CUDA graph WHILE node):
// sweeps *nsw (b1 -> b0) and *nsw + 1 (b0 -> b1), Jacobi or Gauss-Seidel,
// then *nsw += 2 and the loop condition h = (*nsw < max_sweeps and the last
// sweep's dlt >= tol).  Same no-op rule and dlt layout as the host loop.
cudaError_t launch_sweep_pass(const Geometry& g, const double* coef, const double* r, double* b0,
                              double* b1, double* dlt, int* nsw, int max_sweeps, double tol,
                              bool gs, cudaGraphConditionalHandle h, cudaStream_t st);
// After a device-side sweep loop from the buffers Ja (even sweeps) and Jb
// (odd sweeps): Jn = the iterate of the last sweep that ran (the first n
// with dlt[n] < tol, else max_sweeps - 1) and *sweeps_out = n + 1 (may be
// null).  The host loop picks the same buffer from the same deltas.
cudaError_t launch_os_select(long long N, const double* dlt, int max_sweeps, double tol,
                             const double* Ja, const double* Jb, double* Jn, int* sweeps_out,
                             cudaStream_t st);
// Sweep n: Jn[v] = r[v] + sum_{o != 13} c[o][v] J[nb(v,o)];  dlt[n] = max |Jn - J| / |Jn|;
// no-op when n > 0 and dlt[n-1] < tol.
cudaError_t launch_jacobi(const Geometry& g, const double* coef, const double* r,
                          const double* J, double* Jn, double* dlt, int n, double tol,
                          cudaStream_t st);
// Ng acceleration: out5 = the five weighted sums (fixed reduction order) of
// iterates x0 (newest) .. x3; part is scratch of ng_partial_size() doubles.
int ng_partial_size();
cudaError_t launch_ng_dots(long long N, const double* x0, const double* x1, const double* x2,
                           const double* x3, double* part, double* out5, cudaStream_t st);
// x0 = (1 - a - b) x0 + a x1 + b x2 with (a, b) the solution of the 2x2
// system of the five sums s5 (device), computed on the device; no change
// when the system is singular.
cudaError_t launch_ng_apply(long long N, const double* s5, const double* x1, const double* x2,
                            double* x0, cudaStream_t st);
// *delta = max |Jn - Jo| / |Jn|
cudaError_t launch_rel_change(long long N, const double* Jn, const double* Jo, double* delta,
                              cudaStream_t st);

}  // namespace rt3d
