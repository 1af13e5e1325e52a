// C ABI of librt3d.so (declared in include/rt3d.h): the context, argument
// checks, device buffers and the host-side driver of the outer iteration
// (Hauschildt & Baron 2011, Sect. 2: formal solution -> operator splitting,
// everything resident on the GPU, only inputs and J cross the bus).
#include "../../include/rt3d.h"
#include "internal.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <vector>

using namespace rt3d;

struct rt_ctx {
    int device = 0;
    int precision = RT_FP64;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    int num_sms = 0;

    Geometry g{};
    double dx = 1, dy = 1, dz = 1;
    bool have_grid = false, have_quad = false, have_chi = false, have_eps = false, have_B = false;
    bool lstar_valid = false, coef_valid = false, b2_valid = false;
    int os_method = RT_OS_JACOBI;
    double df_switch = 0.0;   // FP32 sweep: finishing stage once delta < this
    // Finishing stage of an FP32-sweep solve: 0 off; 1 the next formal
    // solution is the double-float reference J_ref = J_FS(S_ref) of the
    // current source; 2 formal solutions march the source change
    // dS = S - S_ref in FP32 and add it: J_FS(S) = J_ref + J_FS(dS) with zero
    // boundary intensities (the formal solution is linear in S).
    int fin = 0;
    double *S_ref = nullptr, *J_ref = nullptr, *dS = nullptr;
    // operator-splitting step as a CUDA graph with the sweep loop in a WHILE
    // node (two cached instances: J_old alternates between two buffers)
    struct OsGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        const double* jold = nullptr;
        const double* jfs = nullptr;
        const double* jnew = nullptr;
        const double* dlt = nullptr;
        int max_sweeps = 0, method = -1;
        double tol = -1.0;
    } osg[2];
    int osg_next = 0;
    int* d_nsw = nullptr;     // the graph's sweep counter
    int* d_sw = nullptr;      // sweeps of the graph's last OS step (device), and a pinned copy
    int* h_sw = nullptr;
    bool use_graphs = true;
    unsigned long long* berr = nullptr;   // checked builds: out-of-bounds record
    int fs_method = RT_FS_LONG;
    int src_order = RT_SRC_LINEAR;
    DownGeo* dn = nullptr;   // downstream-point table (FP64 contexts)
    double *scpart = nullptr, *scplanes = nullptr;   // short characteristics
    size_t scpart_n = 0, scplanes_n = 0;
    int groups_req = 0;
    int threads32 = 0;       // threads per block of the FP32 march (0: 128)
    int order32 = 0;         // block order of the FP32 march (0 auto, 1 tile-, 2 plane-major)
    double cut = -1.0;
    // recorded FP64 march (FsRec): the first formal solution after the
    // opacities, directions or boundary change records it, later ones
    // replay it.  rec_mode: -1 automatic, 0 off, > 0 a byte limit.
    long long rec_mode = -1;
    FsRec rec{};
    Rec32 rec32{};              // the FP32-sweep recording (same memory block)
    float4* spair = nullptr;    // the replay's source records
    char* rec_mem = nullptr;
    long long rec_cap = 0;
    bool rec_valid = false;

    // device state, FP64
    double *chi = nullptr, *eps = nullptr, *B = nullptr, *J = nullptr, *S = nullptr;
    double *Jfs = nullptr, *Jn = nullptr, *Ja = nullptr, *Jb = nullptr, *r = nullptr;
    double *lstar = nullptr, *coef = nullptr, *rdiag = nullptr, *partial = nullptr;
    int partial_groups = 0;
    // plane dispatch order of the marches (c->g.zorder points here once set)
    int* zorder = nullptr;
    double* zscratch = nullptr;
    // FP32-sweep form: padded pair records {chi, S_hi} x 2 and their S_lo,
    // step offsets in those planes (poff32); double-float march: padded
    // {chi_hi, chi_lo, S_hi, S_lo} nodes and their step offsets (poff); both:
    // padded boundary B pairs; sum of the quadrature weights
    float4* pair = nullptr;
    float2* plo = nullptr;
    int* poff32 = nullptr;
    float4* node4 = nullptr;
    float2* b2 = nullptr;
    // LTE-diffusion inner boundary: dB/dtau of the bottom nodes (FP64, padded FP32)
    double* gdiff = nullptr;
    float* g2 = nullptr;
    bool gdiff_valid = false;
    // double-float march: df bilinear weights, df diffusion gradient
    float4* bwdf = nullptr;
    float2* g2df = nullptr;
    int* poff = nullptr;
    double wsum = 1.0;
    // direction tables
    DirInfo* info = nullptr;
    StepGeo* off = nullptr;
    Bw4d* bw = nullptr;
    Bw4d* bwh = nullptr;
    float4* bw32 = nullptr;
    double *d_mu = nullptr, *d_phi = nullptr, *d_w = nullptr;
    // scalars: [0] smax, [1] inner delta, [2] outer delta
    double* scal = nullptr;
    unsigned long long* d_steps = nullptr;
    double* h_scal = nullptr;               // pinned
    unsigned long long* h_steps = nullptr;  // pinned
    // per-sweep deltas of one Jacobi solve (device) and a pinned copy
    double* dlt = nullptr;
    double* h_dlt = nullptr;
    int dlt_cap = 0;
    unsigned long long last_steps = 0;

    // Ng acceleration: period (0 = off), older iterates, reduction scratch
    int ng_period = 0;
    double ng_min_delta = 0.0;          // extrapolate only while the last delta >= this
    double ng_last_delta = 0.0;         // delta of the previous iteration
    int ng_count = 1;                   // iterates held, newest included
    double* ng_old[3] = {nullptr, nullptr, nullptr};  // J_{n-1}, J_{n-2}, J_{n-3}
    double* ng_part = nullptr;
    double* ng_out = nullptr;           // device [5]
    int ng_applied = 0;

    // profiling
    rt_stats stats{};
    bool profiling = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // fs begin/end, jacobi begin/end
    bool fs_pending = false, jac_pending = false;

    std::string err;
};

namespace {

int fail(rt_ctx* c, int code, const char* fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(c, e_ == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA,      \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

template <typename T>
void dfree(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

template <typename T>
cudaError_t dalloc(T*& p, size_t count)
{
    dfree(p);
    if (count == 0) return cudaSuccess;
    return cudaMalloc((void**)&p, count * sizeof(T));
}

void free_ng(rt_ctx* c)
{
    for (auto& p : c->ng_old) dfree(p);
    dfree(c->ng_part);
    dfree(c->ng_out);
}

void free_os_graphs(rt_ctx* c)
{
    for (auto& e : c->osg) {
        if (e.exec) cudaGraphExecDestroy(e.exec);
        if (e.graph) cudaGraphDestroy(e.graph);
        e = rt_ctx::OsGraph{};
    }
}

void free_rec(rt_ctx* c)
{
    if (c->rec_mem) cudaFree(c->rec_mem);
    c->rec_mem = nullptr;
    c->rec = FsRec{};
    c->rec32 = Rec32{};
    c->spair = nullptr;
    c->rec_cap = 0;
    c->rec_valid = false;
}

void free_grid_buffers(rt_ctx* c)
{
    free_os_graphs(c);
    dfree(c->chi); dfree(c->eps); dfree(c->B); dfree(c->J); dfree(c->S);
    dfree(c->Jfs); dfree(c->Jn); dfree(c->Ja); dfree(c->Jb); dfree(c->r);
    dfree(c->lstar); dfree(c->coef); dfree(c->rdiag); dfree(c->partial);
    dfree(c->node4); dfree(c->pair); dfree(c->plo);
    dfree(c->S_ref); dfree(c->J_ref); dfree(c->dS);
    dfree(c->b2); dfree(c->gdiff); dfree(c->g2); dfree(c->g2df);
    dfree(c->scpart); dfree(c->scplanes);
    dfree(c->zorder); dfree(c->zscratch);
    c->g.zorder = nullptr;
    c->scpart_n = c->scplanes_n = 0;
    free_ng(c);
    c->partial_groups = 0;
    free_rec(c);
}

void free_tables(rt_ctx* c)
{
    dfree(c->info); dfree(c->off); dfree(c->bw); dfree(c->bwh); dfree(c->bw32);
    dfree(c->poff); dfree(c->poff32); dfree(c->bwdf);
    dfree(c->dn);
    dfree(c->d_mu); dfree(c->d_phi); dfree(c->d_w);
}

// Add the device time of the kernels bracketed since the last harvest;
// called right after a stream synchronisation.
void harvest(rt_ctx* c)
{
    float ms = 0.f;
    if (c->fs_pending && cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]) == cudaSuccess)
        c->stats.fs_ms += ms;
    if (c->jac_pending && cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]) == cudaSuccess)
        c->stats.jacobi_ms += ms;
    c->fs_pending = c->jac_pending = false;
}

int enter(rt_ctx* c)
{
    if (!c) return RT_EINVAL;
    c->err.clear();
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, RT_ECUDA, "cudaSetDevice(%d): %s", c->device, cudaGetErrorString(e));
    return RT_OK;
}

// Default delta below which an RT_FP32_SWEEP solve continues in double-float
// (rt_set_df_finish): where the FP32 sweep's Ng extrapolation has to stop.
constexpr double kDefaultDfSwitch = 1e-6;

double default_cut(int precision)
{
    // FP32 sweep and double-float march: the cut is relative to S at the
    // voxel (see fs32.cu); 2^-46 (2^-52) keeps the truncation far below what
    // 1/eps can amplify at eps = 1e-6 (far below double-float rounding).
    if (precision == RT_FP64) return 1e-17;
    return precision == RT_DF64 ? 2.220446049250313e-16 : 1.4210854715202004e-14;
}

// Number of z-blocks that walk the kSlots direction slots: enough blocks to
// give every SM many waves, fewer (longer) blocks on large grids.
int auto_groups(const rt_ctx* c)
{
    if (c->groups_req > 0) return c->groups_req < kSlots ? c->groups_req : kSlots;
    const long long blocks = (long long)((c->g.nx * c->g.ny + 127) / 128) * c->g.nz;
    const long long target = 64LL * (c->num_sms > 0 ? c->num_sms : 152);
    int G = 1;
    while (G < kSlots && blocks * G < target) G *= 2;
    return G;
}

// Device memory for a recording of `need` bytes within the context's
// budget (rec_mode): false when it does not fit or cannot be allocated.
bool rec_reserve(rt_ctx* c, long long need)
{
    if (need <= c->rec_cap) return true;
    long long limit = c->rec_mode;
    if (limit < 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        // at most 60% of the device, leaving 2 GiB free
        limit = (long long)(0.6 * (double)tot);
        const long long avail = (long long)fr + c->rec_cap - (2LL << 30);
        if (avail < limit) limit = avail;
    }
    if (need > limit) return false;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return false;
    free_rec(c);
    if (cudaMalloc((void**)&c->rec_mem, (size_t)need) != cudaSuccess) {
        cudaGetLastError();
        c->rec_mem = nullptr;
        return false;
    }
    c->rec_cap = need;
    return true;
}

long long up256(long long b) { return (b + 255) / 256 * 256; }

// The recorded march: whether this context records and replays it (FP64
// with long characteristics and the linear source, or the FP32 sweep; a
// byte budget that admits it), with its buffers carved from one block.
// When it does not fit, the march runs as it is every time.
// Bytes a recording of this context's march takes (0: its form does not record).
long long rec_need(const rt_ctx* c)
{
    if (c->fs_method != RT_FS_LONG || c->g.nz < 2 ||
        (c->src_order != RT_SRC_LINEAR && c->precision != RT_FP64))
        return 0;
    const long long tri = (long long)c->g.nz * (c->g.nz - 1) / 2;
    const long long b_slot = up256((long long)kSlots * c->g.N * (long long)sizeof(double));
    if (c->precision == RT_FP64 || c->precision == RT_DF64) {   // same bytes per entry
        const long long nxy = (long long)c->g.nx * c->g.ny, nwp = (nxy + 31) / 32;
        const long long b_cdn = c->src_order == RT_SRC_PARABOLIC
                                    ? up256((long long)c->g.ndir * c->g.N * (long long)sizeof(double))
                                    : 0;
        return up256((long long)c->g.ndir * nxy * tri * (long long)sizeof(double)) +
               up256((long long)c->g.ndir * c->g.nz * nwp * (long long)sizeof(int)) + 2 * b_slot +
               b_cdn;
    }
    const long long npair = (long long)c->g.nx * ((c->g.ny + 1) / 2), nwp = (npair + 31) / 32;
    return up256((long long)c->g.ndir * rec32_steps4(c->g.nz) * nwp * 32 * (long long)sizeof(float2)) +
           up256((long long)c->g.ndir * c->g.nz * nwp * (long long)sizeof(int)) + 2 * b_slot +
           up256(pair_records(c->g) * (long long)sizeof(float4));
}

int ensure_rec(rt_ctx* c, bool& use)
{
    use = false;
    const long long need = rec_need(c);
    if (c->rec_mode == 0 || need == 0) return RT_OK;
    const long long tri = (long long)c->g.nz * (c->g.nz - 1) / 2;
    const long long b_slot = up256((long long)kSlots * c->g.N * (long long)sizeof(double));
    if (c->precision == RT_DF64) {
        const long long nxy = (long long)c->g.nx * c->g.ny;
        const long long nwp = (nxy + 31) / 32;
        const long long b_coef = up256((long long)c->g.ndir * nxy * tri * (long long)sizeof(float2));
        const long long b_lmax = up256((long long)c->g.ndir * c->g.nz * nwp * (long long)sizeof(int));
        if (!rec_reserve(c, need)) return RT_OK;
        c->rec32.coef = reinterpret_cast<float2*>(c->rec_mem);
        c->rec32.lmax = reinterpret_cast<int*>(c->rec_mem + b_coef);
        c->rec32.tsum = reinterpret_cast<double*>(c->rec_mem + b_coef + b_lmax);
        c->rec32.bc = reinterpret_cast<double*>(c->rec_mem + b_coef + b_lmax + b_slot);
        c->rec32.nwp = (int)nwp;
    } else if (c->precision == RT_FP64) {
        const long long nxy = (long long)c->g.nx * c->g.ny;
        const long long nwp = (nxy + 31) / 32;
        const long long b_coef = up256((long long)c->g.ndir * nxy * tri * (long long)sizeof(double));
        const long long b_lmax = up256((long long)c->g.ndir * c->g.nz * nwp * (long long)sizeof(int));
        if (!rec_reserve(c, need)) return RT_OK;
        c->rec.coef = reinterpret_cast<double*>(c->rec_mem);
        c->rec.lmax = reinterpret_cast<int*>(c->rec_mem + b_coef);
        c->rec.c0 = reinterpret_cast<double*>(c->rec_mem + b_coef + b_lmax);
        c->rec.bc = reinterpret_cast<double*>(c->rec_mem + b_coef + b_lmax + b_slot);
        c->rec.nwp = (int)nwp;
        const bool para = c->src_order == RT_SRC_PARABOLIC;
        c->rec.cdn = para ? reinterpret_cast<double*>(c->rec_mem + b_coef + b_lmax + 2 * b_slot)
                          : nullptr;
        c->rec.dn = para ? c->dn : nullptr;
    } else {
        const long long npair = (long long)c->g.nx * ((c->g.ny + 1) / 2);
        const long long nwp = (npair + 31) / 32;
        const long long b_coef = up256((long long)c->g.ndir * rec32_steps4(c->g.nz) * nwp * 32 *
                                       (long long)sizeof(float2));
        const long long b_lmax = up256((long long)c->g.ndir * c->g.nz * nwp * (long long)sizeof(int));
        const long long b_sp = up256(pair_records(c->g) * (long long)sizeof(float4));
        if (!rec_reserve(c, b_coef + b_lmax + 2 * b_slot + b_sp)) return RT_OK;
        char* q = c->rec_mem;
        c->rec32.coef = reinterpret_cast<float2*>(q);
        c->rec32.lmax = reinterpret_cast<int*>(q + b_coef);
        c->rec32.tsum = reinterpret_cast<double*>(q + b_coef + b_lmax);
        c->rec32.bc = reinterpret_cast<double*>(q + b_coef + b_lmax + b_slot);
        c->rec32.nwp = (int)nwp;
        c->spair = reinterpret_cast<float4*>(q + b_coef + b_lmax + 2 * b_slot);
    }
    use = true;
    return RT_OK;
}

// Buffers of the short-characteristics march (sized by grid and directions).
int ensure_sc(rt_ctx* c)
{
    const size_t np = (size_t)sc_chunk(c->g) * (size_t)c->g.N;
    if (c->scpart_n < np) {
        dfree(c->scpart);
        c->scpart_n = 0;
        CK(dalloc(c->scpart, np));
        c->scpart_n = np;
    }
    const size_t ns = sc_scratch_planes(c->g);
    if (ns && c->scplanes_n < ns) {
        dfree(c->scplanes);
        c->scplanes_n = 0;
        CK(dalloc(c->scplanes, ns));
        c->scplanes_n = ns;
    }
    return RT_OK;
}

int ensure_partial(rt_ctx* c)
{
    if (c->partial_groups >= kSlots) return RT_OK;
    CK(dalloc(c->partial, (size_t)kSlots * c->g.N));
    c->partial_groups = kSlots;
    return RT_OK;
}

// Buffers the march of `precision` needs beyond the ones every form has:
// the FP32 pair planes, or the double-float nodes, gradient and weights
// (allocated once, also when a live context switches form).
int form_buffers(rt_ctx* c, int precision)
{
    if (c->have_grid && precision == RT_FP32_SWEEP && !c->pair) {
        CK(dalloc(c->pair, (size_t)pair_records(c->g)));
        CK(dalloc(c->plo, (size_t)pair_records(c->g)));
    }
    if (c->have_grid && precision == RT_DF64) {
        if (!c->node4) CK(dalloc(c->node4, (size_t)(4 * c->g.N)));
        if (!c->g2df) CK(dalloc(c->g2df, (size_t)4 * c->g.nx * c->g.ny));
    }
    if (c->have_quad && precision == RT_DF64 && !c->bwdf) {
        const long long T = (long long)c->g.ndir * c->g.nz;
        CK(dalloc(c->bwdf, (size_t)(2 * T)));
        CK(launch_bw_df(T, c->bw, c->bwdf, c->stream));
        c->stats.launches += 1;
    }
    return RT_OK;
}

int check_field(rt_ctx* c, const double* h, const char* what, bool positive, bool eps_range)
{
    for (long long v = 0; v < c->g.N; ++v) {
        const double x = h[v];
        if (!std::isfinite(x)) return fail(c, RT_EINVAL, "%s[%lld] is not finite", what, v);
        if (positive && !(x > 0)) return fail(c, RT_EINVAL, "%s[%lld] = %g must be > 0", what, v, x);
        if (eps_range && !(x > 0 && x <= 1))
            return fail(c, RT_EINVAL, "%s[%lld] = %g must lie in (0, 1]", what, v, x);
    }
    return RT_OK;
}

int need(rt_ctx* c, bool ok, const char* what)
{
    return ok ? RT_OK : fail(c, RT_ESTATE, "%s has not been set", what);
}

int need_all(rt_ctx* c)
{
    int rc;
    if ((rc = need(c, c->have_grid, "the grid"))) return rc;
    if ((rc = need(c, c->have_quad, "the quadrature"))) return rc;
    if ((rc = need(c, c->have_chi, "the opacity"))) return rc;
    if ((rc = need(c, c->have_eps, "epsilon"))) return rc;
    if ((rc = need(c, c->have_B, "the Planck function"))) return rc;
    return RT_OK;
}

cudaMemcpyKind kind(bool device) { return device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }

int set_field(rt_ctx* c, const double* src, double* dst, bool device, const char* what,
              bool positive, bool eps_range)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = need(c, c->have_grid, "the grid"))) return rc;
    if (!src) return fail(c, RT_EINVAL, "%s is NULL", what);
    if (!device && (rc = check_field(c, src, what, positive, eps_range))) return rc;
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * c->g.N, kind(device), c->stream));
    if (!device) CK(cudaStreamSynchronize(c->stream));
    return RT_OK;
}

View32 view32(rt_ctx* c)
{
    View32 v;
    v.g = c->g;
    v.pair = c->pair;
    v.lo = c->plo;
    v.b2 = c->b2;
    v.g2 = c->g2;
    v.info = c->info;
    v.off = c->off;
    v.poff = c->poff32;
    v.bw = c->bw32;
    v.smax = c->scal + 0;
    v.sfloor = nullptr;
    v.partial = c->partial;
    v.pmajor = plane_major32(c->g, c->order32);
    return v;
}

// The FP32 march of the finishing stage: source dS (packed in the pair
// planes), zero boundary intensities, cutoff relative to min |S_ref|.
View32 view32_fin(rt_ctx* c)
{
    View32 v = view32(c);
    v.g.top_bc = RT_BC_ZERO;
    v.g.bottom_bc = RT_BC_ZERO;
    v.sfloor = c->scal + 3;
    return v;
}

ViewDF viewdf(rt_ctx* c)
{
    ViewDF v;
    v.g = c->g;
    v.node = c->node4;
    v.b2 = c->b2;
    v.g2df = c->g2df;
    v.info = c->info;
    v.off = c->off;
    v.poff = c->poff;
    v.bw = c->bwdf;
    v.smax = c->scal + 0;
    v.partial = c->partial;
    return v;
}

// Formal solution: source in c->S (already set), result J into Jout (device).
// Pieces of one formal solution: per-problem preparation, the march itself,
// and the reduction over direction slots plus (once per opacity) Lambda*.
int fs_prepare(rt_ctx* c)
{
    int rc = ensure_partial(c);
    if (rc) return rc;
    if (c->g.bottom_bc == RT_BC_DIFFUSION && !c->gdiff_valid) {
        CK(launch_diffusion_grad(c->g, c->dz, c->chi, c->B, c->gdiff,
                                 c->precision == RT_FP32_SWEEP ? c->g2 : nullptr, c->stream));
        c->stats.launches += 1;
        if (c->precision == RT_DF64) {
            CK(launch_grad_df(c->g, c->gdiff, c->g2df, c->stream));
            c->stats.launches += 1;
        }
        c->gdiff_valid = true;
    }
    if (c->precision != RT_FP64 && !c->b2_valid) {
        CK(launch_pack_b2(c->g, c->B, c->b2, c->stream));
        c->b2_valid = true;
        c->stats.launches += 1;
    }
    return RT_OK;
}

double cut_of(const rt_ctx* c) { return c->cut >= 0 ? c->cut : default_cut(c->precision); }

int fs_finish(rt_ctx* c, double* Jout)
{
    if (c->precision == RT_FP64)
        CK(launch_sum_groups(c->g.N, c->partial, Jout, c->stream));
    else if (c->precision == RT_FP32_SWEEP && c->fin == 2)
        CK(launch_sum_groups_ref(c->g.N, c->partial, c->dS, c->wsum, c->J_ref, Jout, c->stream));
    else
        CK(launch_sum_groups_src(c->g.N, c->partial, c->S, c->wsum, Jout, c->stream));
    c->stats.launches += 1;
    if (!c->lstar_valid) {
        if (c->src_order == RT_SRC_PARABOLIC) {
            CK(launch_lstar64p(c->g, c->chi, c->info, c->off, c->bw, c->dn, c->lstar, c->stream));
        } else if (c->precision == RT_FP64) {
            CK(launch_lstar64(c->g, c->chi, c->info, c->off, c->bw, c->lstar, c->stream));
        } else {
            // FP32 sweep and double-float march: Lambda* in double-float
            // (FP64-accurate; 5.7 against 25 ms for the FP64 kernel on the
            // 65^3 slab with 1024 directions), from the double-float nodes
            if (c->precision == RT_FP32_SWEEP) {
                int rc = form_buffers(c, RT_DF64);
                if (rc) return rc;
                CK(launch_packdf(c->g, c->chi, c->S, c->node4, c->stream));
                c->stats.launches += 1;
            }
            CK(launch_lstar_df(viewdf(c), false, c->lstar, c->stream));
        }
        c->lstar_valid = true;
        c->coef_valid = false;
        c->stats.launches += 1;
        c->stats.lstar_launches += 1;
    }
    return RT_OK;
}

// The finishing stage's reference (c->fin == 1): a double-float formal
// solution of the current source S into c->partial (same sum convention as
// the FP32 march); fin_record() then keeps S and J as the reference.
int fin_reference_march(rt_ctx* c, int G, unsigned long long* steps, cudaStream_t st)
{
    int rc = form_buffers(c, RT_DF64);
    if (rc) return rc;
    if (!c->S_ref) {
        CK(dalloc(c->S_ref, (size_t)c->g.N));
        CK(dalloc(c->J_ref, (size_t)c->g.N));
        CK(dalloc(c->dS, (size_t)c->g.N));
    }
    if (c->g.bottom_bc == RT_BC_DIFFUSION) {
        CK(launch_grad_df(c->g, c->gdiff, c->g2df, st));
        c->stats.launches += 1;
    }
    CK(launch_packdf(c->g, c->chi, c->S, c->node4, st));
    CK(launch_fsdf(viewdf(c), c->cut >= 0 ? c->cut : default_cut(RT_DF64), G, steps, st));
    c->stats.launches += 2;
    return RT_OK;
}

int fin_record(rt_ctx* c, const double* Jfs, cudaStream_t st)
{
    CK(cudaMemcpyAsync(c->S_ref, c->S, sizeof(double) * c->g.N, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(c->J_ref, Jfs, sizeof(double) * c->g.N, cudaMemcpyDeviceToDevice, st));
    CK(launch_absmin(c->g.N, c->S, c->scal + 3, st));
    c->stats.launches += 1;
    c->fin = 2;
    return RT_OK;
}

// Short-characteristics formal solution (FP64 only): J straight from the
// march's ordered reduction, Lambda* from its own kernel once per opacity.
int run_fs_short(rt_ctx* c, double* Jout, bool count_steps)
{
    int rc = fs_prepare(c);
    if (rc) return rc;
    if ((rc = ensure_sc(c))) return rc;
    if (count_steps) CK(cudaMemsetAsync(c->d_steps, 0, sizeof(unsigned long long), c->stream));
    if (c->profiling) CK(cudaEventRecord(c->ev[0], c->stream));
    if (c->precision == RT_DF64)
        CK(launch_scdf(viewdf(c), c->S, c->wsum, c->scpart, (float2*)c->scplanes, Jout,
                       count_steps ? c->d_steps : nullptr, c->stream));
    else
        CK(launch_sc64(c->g, c->chi, c->S, c->B, c->gdiff, c->info, c->off, c->bw, c->scpart,
                       c->scplanes, Jout, count_steps ? c->d_steps : nullptr, c->stream));
    if (c->profiling) {
        CK(cudaEventRecord(c->ev[1], c->stream));
        c->fs_pending = true;
    }
    const int chunks = (c->g.ndir + sc_chunk(c->g) - 1) / sc_chunk(c->g);
    c->stats.fs_launches += 1;
    c->stats.launches += 2 * chunks;
    if (!c->lstar_valid) {
        if (c->precision == RT_DF64)
            CK(launch_lstar_df(viewdf(c), true, c->lstar, c->stream));
        else
            CK(launch_lstar_sc64(c->g, c->chi, c->info, c->off, c->bw, c->lstar, c->stream));
        c->lstar_valid = true;
        c->coef_valid = false;
        c->stats.launches += 1;
        c->stats.lstar_launches += 1;
    }
    if (count_steps) {
        CK(cudaMemcpyAsync(c->h_steps, c->d_steps, sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, c->stream));
    }
    return RT_OK;
}

// The double-float formal solution of a context: recorded in the first one
// after the opacities change and replayed, or marched when the recording
// does not fit.
int df_formal(rt_ctx* c, int G, unsigned long long* steps, cudaStream_t st)
{
    bool use = false;
    int rc = ensure_rec(c, use);
    if (rc) return rc;
    const double cut = cut_of(c);
    if (use && !c->rec_valid) {
        CK(launch_fsdf(viewdf(c), cut * kRecCutMargin, G, steps, st, &c->rec32));
        c->rec_valid = true;
        c->stats.launches += 1;
    }
    if (use)
        CK(launch_fsdfrep(viewdf(c), c->rec32, G, steps, st));
    else
        CK(launch_fsdf(viewdf(c), cut, G, steps, st));
    return RT_OK;
}

int run_fs(rt_ctx* c, double* Jout, bool count_steps)
{
    if (c->fs_method == RT_FS_SHORT) return run_fs_short(c, Jout, count_steps);
    const int G = auto_groups(c);
    int rc = fs_prepare(c);
    if (rc) return rc;
    if (count_steps) CK(cudaMemsetAsync(c->d_steps, 0, sizeof(unsigned long long), c->stream));
    const double cut = cut_of(c);
    if (c->profiling) CK(cudaEventRecord(c->ev[0], c->stream));
    if (c->precision == RT_FP64 && c->src_order == RT_SRC_PARABOLIC) {
        // recorded like the linear source (with the downstream point's
        // coefficients), else marched
        bool use = false;
        if ((rc = ensure_rec(c, use))) return rc;
        unsigned long long* sp = count_steps ? c->d_steps : nullptr;
        if (use && !c->rec_valid) {
            CK(launch_fs64p(c->g, c->chi, c->S, c->B, c->gdiff, c->info, c->off, c->bw, c->dn,
                            c->scal + 0, cut, G, c->partial, sp, c->stream, &c->rec));
            c->rec_valid = true;
            c->stats.launches += 1;
        }
        if (use)
            CK(launch_fs64rep(c->g, c->S, c->info, c->off, c->bw, c->rec, G, c->partial, sp,
                              c->stream));
        else
            CK(launch_fs64p(c->g, c->chi, c->S, c->B, c->gdiff, c->info, c->off, c->bw, c->dn,
                            c->scal + 0, cut, G, c->partial, sp, c->stream));
    } else if (c->precision == RT_FP64) {
        bool use = false;
        if ((rc = ensure_rec(c, use))) return rc;
        if (use && !c->rec_valid) {
            // record; J then comes from the replay like every later one, so
            // that it does not depend on which formal solution recorded
            CK(launch_fs64(c->g, c->chi, c->S, c->B, c->gdiff, c->info, c->off, c->bw, c->bwh,
                           c->scal + 0, cut, G, c->partial, count_steps ? c->d_steps : nullptr,
                           c->stream, &c->rec));
            c->rec_valid = true;
            c->stats.launches += 1;
        }
        if (use) {
            CK(launch_fs64rep(c->g, c->S, c->info, c->off, c->bw, c->rec, G, c->partial,
                              count_steps ? c->d_steps : nullptr, c->stream));
        } else {
            CK(launch_fs64(c->g, c->chi, c->S, c->B, c->gdiff, c->info, c->off, c->bw, c->bwh,
                           c->scal + 0, cut, G, c->partial, count_steps ? c->d_steps : nullptr,
                           c->stream));
        }
    } else if (c->precision == RT_DF64) {
        if ((rc = df_formal(c, G, count_steps ? c->d_steps : nullptr, c->stream))) return rc;
    } else if (c->fin == 1) {
        if ((rc = fin_reference_march(c, G, count_steps ? c->d_steps : nullptr, c->stream)))
            return rc;
    } else {
        // FP32 sweep (fin 0, or 2: the finishing stage's source change).  The
        // recording is made from the source itself (fin 0) and serves both.
        bool use = false;
        if ((rc = ensure_rec(c, use))) return rc;
        unsigned long long* sp = count_steps ? c->d_steps : nullptr;
        if (use && !c->rec_valid && c->fin == 0) {
            CK(launch_fs32rec(view32(c), cut * kRecCutMargin, G, c->rec32, sp, c->stream));
            c->rec_valid = true;
            c->stats.launches += 1;
        }
        if (use && c->rec_valid) {
            CK(launch_pack_spairs(c->g, c->fin == 2 ? c->dS : c->S, c->spair, c->stream));
            Rep32 rp{c->g, c->spair, c->info, c->poff32, c->bw32, c->rec32, c->partial,
                     c->fin == 2 ? 1 : 0, plane_major32(c->g, c->order32)};
            CK(launch_fs32rep(rp, G, c->threads32, sp, c->stream));
            c->stats.launches += 1;
        } else {
            CK(launch_fs32d(c->fin == 2 ? view32_fin(c) : view32(c), cut, G, c->threads32, sp,
                            c->stream));
        }
    }
    if (c->profiling) {
        CK(cudaEventRecord(c->ev[1], c->stream));
        c->fs_pending = true;
    }
    c->stats.fs_launches += 1;
    c->stats.launches += 1;
    if ((rc = fs_finish(c, Jout))) return rc;
    if (c->precision == RT_FP32_SWEEP && c->fin == 1 && (rc = fin_record(c, Jout, c->stream)))
        return rc;
    if (count_steps) {
        CK(cudaMemcpyAsync(c->h_steps, c->d_steps, sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, c->stream));
    }
    return RT_OK;
}

// S = eps B + (1 - eps) J (or the caller's S), then smax; FP32 copy if needed.
int prepare_source(rt_ctx* c, const double* S_in, bool device)
{
    const bool bnd = c->g.top_bc || c->g.bottom_bc;
    CK(cudaMemsetAsync(c->scal + 0, 0, sizeof(double), c->stream));
    if (S_in) {
        CK(cudaMemcpyAsync(c->S, S_in, sizeof(double) * c->g.N, kind(device), c->stream));
        CK(launch_absmax(c->g.N, c->S, bnd ? c->B : nullptr, c->scal + 0, nullptr, c->stream));
    } else {
        CK(launch_source(c->g.N, c->eps, c->B, c->J, c->S, nullptr, bnd ? c->B : nullptr,
                         c->scal + 0, c->stream));
    }
    c->stats.launches += 1;
    if (c->precision == RT_FP32_SWEEP && c->fin == 2) {
        // finishing stage: march dS = S - S_ref, cutoff bound max |dS|
        CK(launch_delta_source(c->g.N, c->S, c->S_ref, c->dS, c->stream));
        CK(cudaMemsetAsync(c->scal + 0, 0, sizeof(double), c->stream));
        CK(launch_absmax(c->g.N, c->dS, nullptr, c->scal + 0, nullptr, c->stream));
        if (!c->rec_valid) {   // the replay packs its own source records
            CK(launch_pack_pairs(c->g, c->chi, c->dS, c->pair, c->plo, c->stream));
            c->stats.launches += 1;
        }
        c->stats.launches += 2;
    } else if (c->precision == RT_FP32_SWEEP && c->fin == 1) {
        // the reference formal solution packs its own double-float nodes
    } else if (c->precision == RT_FP32_SWEEP && c->rec_valid) {
        // the replay packs its own source records
    } else if (c->precision == RT_FP32_SWEEP) {
        CK(launch_pack_pairs(c->g, c->chi, c->S, c->pair, c->plo, c->stream));
        c->stats.launches += 1;
    } else if (c->precision == RT_DF64) {
        CK(launch_packdf(c->g, c->chi, c->S, c->node4, c->stream));
        c->stats.launches += 1;
    }
    return RT_OK;
}

// Checked builds: report (and clear) the first out-of-bounds index the
// kernels recorded since the last check.  Normal builds: nothing to do.
int check_bounds(rt_ctx* c, int rc)
{
#ifdef RT_CHECKED
    unsigned long long h[4] = {0, 0, 0, 0};
    if (cudaMemcpy(h, c->berr, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(c, RT_ECUDA, "reading the bounds record failed");
    if (h[0]) {
        cudaMemset(c->berr, 0, sizeof(h));
        return fail(c, RT_EBOUNDS, "index %lld outside [0, %lld) at site %llu",
                    (long long)h[2], (long long)h[3], h[1]);
    }
#else
    (void)c;
#endif
    return rc;
}

int formal_solution(rt_ctx* c, const double* S, double* Jfs_out, double* lstar_out, bool device)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = need_all(c))) return rc;
    if (!Jfs_out) return fail(c, RT_EINVAL, "J_fs is NULL");
    if ((rc = prepare_source(c, S, device))) return rc;
    if ((rc = run_fs(c, c->Jfs, true))) return rc;
    const cudaMemcpyKind out = device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(Jfs_out, c->Jfs, sizeof(double) * c->g.N, out, c->stream));
    if (lstar_out)
        CK(cudaMemcpyAsync(lstar_out, c->lstar, sizeof(double) * 27 * c->g.N, out, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    harvest(c);
    c->last_steps = *c->h_steps;
    c->stats.steps += c->last_steps;
    return RT_OK;
}

int ensure_coef(rt_ctx* c)
{
    if (c->coef_valid) return RT_OK;
    CK(launch_os_coef(c->g, c->lstar, c->eps, c->coef, c->rdiag,
                      c->os_method == RT_OS_GAUSS_SEIDEL, c->stream));
    c->coef_valid = true;
    c->stats.launches += 1;
    return RT_OK;
}

int ensure_dlt(rt_ctx* c, int max_sweeps)
{
    if (c->dlt_cap >= max_sweeps) return RT_OK;
    int cap = max_sweeps < 1024 ? 1024 : max_sweeps;
    free_os_graphs(c);          // they hold the old dlt pointer
    CK(dalloc(c->dlt, (size_t)cap));
    if (c->h_dlt) cudaFreeHost(c->h_dlt);
    c->h_dlt = nullptr;
    CK(cudaMallocHost((void**)&c->h_dlt, sizeof(double) * cap));
    c->dlt_cap = cap;
    return RT_OK;
}

// Jacobi solve from J_old (device) into J_new (device); J_fs device.  Sweeps
// are enqueued in growing chunks; a sweep that follows a converged one is a
// no-op on the device, so checking once per chunk gives exactly the sweeps
// of a check after every sweep.
// The operator-splitting step as one CUDA graph: right-hand side, zeroed
// deltas, J_old copied to the sweep buffer read first, a zeroed sweep
// counter, then a WHILE node whose body runs two sweeps and the loop test on
// the device.  The host launches it once and reads the deltas once, instead
// of synchronising after every chunk of sweeps.  Results are those of the
// host loop: same kernels, same no-op rule after convergence.
int build_os_graph(rt_ctx* c, rt_ctx::OsGraph& e, const double* Jfs, const double* Jold,
                   double* Jnew, double tol, int max_sweeps)
{
    const bool gs = c->os_method == RT_OS_GAUSS_SEIDEL;
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t err = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    std::vector<cudaGraphNode_t> deps;
    if (err == cudaSuccess)
        err = cudaStreamBeginCaptureToGraph(c->stream, g, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
        // prologue; every call is attempted so that the capture is always ended
        cudaError_t e1 = launch_os_rhs(c->g, c->coef, c->rdiag, Jfs, Jold, c->r, gs, c->stream);
        cudaError_t e2 = cudaMemsetAsync(c->dlt, 0, sizeof(double) * (max_sweeps + 2), c->stream);
        cudaError_t e3 = cudaMemcpyAsync(c->Jb, Jold, sizeof(double) * c->g.N,
                                         cudaMemcpyDeviceToDevice, c->stream);
        cudaError_t e4 = cudaMemsetAsync(c->d_nsw, 0, sizeof(int), c->stream);
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* dp = nullptr;
        size_t nd = 0;
        cudaError_t e5 = cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, nullptr, &dp, nullptr, &nd);
        if (e5 == cudaSuccess) deps.assign(dp, dp + nd);
        cudaGraph_t out = nullptr;
        cudaError_t e6 = cudaStreamEndCapture(c->stream, &out);
        for (cudaError_t x : {e1, e2, e3, e4, e5, e6})
            if (err == cudaSuccess && x != cudaSuccess) err = x;
    }
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t cn;
    if (err == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        err = cudaGraphAddNode(&cn, g, deps.data(), nullptr, deps.size(), &cp);
    }
    if (err == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        err = cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal);
        if (err == cudaSuccess) {
            cudaError_t e1 = launch_sweep_pass(c->g, c->coef, c->r, c->Ja, c->Jb, c->dlt, c->d_nsw,
                                               max_sweeps, tol, gs, h, c->stream);
            cudaGraph_t out = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(c->stream, &out);
            err = e1 != cudaSuccess ? e1 : e2;
        }
    }
    if (err == cudaSuccess) {
        // epilogue after the loop: the last sweep's iterate into J_new and
        // the sweep count, on the device
        err = cudaStreamBeginCaptureToGraph(c->stream, g, &cn, nullptr, 1,
                                            cudaStreamCaptureModeThreadLocal);
        if (err == cudaSuccess) {
            cudaError_t e1 = launch_os_select(c->g.N, c->dlt, max_sweeps, tol, c->Ja, c->Jb, Jnew,
                                              c->d_sw, c->stream);
            cudaGraph_t out = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(c->stream, &out);
            err = e1 != cudaSuccess ? e1 : e2;
        }
    }
    cudaGraphExec_t exec = nullptr;
    if (err == cudaSuccess) err = cudaGraphInstantiate(&exec, g, 0);
    if (err != cudaSuccess) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(c, RT_ECUDA, "building the operator-splitting graph: %s", cudaGetErrorString(err));
    }
    e.graph = g;
    e.exec = exec;
    e.jold = Jold;
    e.jfs = Jfs;
    e.jnew = Jnew;
    e.dlt = c->dlt;
    e.max_sweeps = max_sweeps;
    e.method = c->os_method;
    e.tol = tol;
    return RT_OK;
}

// The operator-splitting step as one graph launch, without waiting for it:
// J_new and the sweep count (c->d_sw) are written on the device.  The
// caller copies d_sw to h_sw before its next synchronisation and then calls
// os_graph_done().
int run_os_graph(rt_ctx* c, const double* Jfs, const double* Jold, double* Jnew, double tol_inner,
                 int max_sweeps)
{
    int rc;
    if ((rc = ensure_dlt(c, max_sweeps + 2))) return rc;
    if (!c->d_nsw) CK(cudaMalloc((void**)&c->d_nsw, sizeof(int)));
    if (!c->d_sw) {
        CK(cudaMalloc((void**)&c->d_sw, sizeof(int)));
        CK(cudaMallocHost((void**)&c->h_sw, sizeof(int)));
    }
    rt_ctx::OsGraph* e = nullptr;
    for (auto& x : c->osg)
        if (x.exec && x.jold == Jold && x.jfs == Jfs && x.jnew == Jnew && x.dlt == c->dlt &&
            x.max_sweeps == max_sweeps && x.tol == tol_inner && x.method == c->os_method)
            e = &x;
    if (!e) {
        e = &c->osg[c->osg_next];
        c->osg_next ^= 1;
        if (e->exec) cudaGraphExecDestroy(e->exec);
        if (e->graph) cudaGraphDestroy(e->graph);
        *e = rt_ctx::OsGraph{};
        if ((rc = build_os_graph(c, *e, Jfs, Jold, Jnew, tol_inner, max_sweeps))) return rc;
    }
    if (c->profiling) CK(cudaEventRecord(c->ev[2], c->stream));
    CK(cudaGraphLaunch(e->exec, c->stream));
    if (c->profiling) {
        CK(cudaEventRecord(c->ev[3], c->stream));
        c->jac_pending = true;
    }
    CK(cudaMemcpyAsync(c->h_sw, c->d_sw, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    return RT_OK;
}

// After the synchronisation that follows run_os_graph: the sweep count and
// the launch counters of that step.
int os_graph_done(rt_ctx* c)
{
    const int sweeps = *c->h_sw;
    const int per = c->os_method == RT_OS_GAUSS_SEIDEL ? 2 : 1;
    const int passes = (sweeps + 1) / 2;
    c->stats.launches += 2 + passes * (2 * per + 1);
    c->stats.jacobi_launches += passes * 2 * per;
    return sweeps;
}

int run_os(rt_ctx* c, const double* Jfs, const double* Jold, double* Jnew, double tol_inner,
           int max_sweeps, int* sweeps_out)
{
    int rc = ensure_coef(c);
    if (rc) return rc;
    if (c->use_graphs) {
        // sweep count after the caller's synchronisation (os_graph_done)
        if (sweeps_out) *sweeps_out = -1;
        return run_os_graph(c, Jfs, Jold, Jnew, tol_inner, max_sweeps);
    }
    if ((rc = ensure_dlt(c, max_sweeps))) return rc;
    const bool gs = c->os_method == RT_OS_GAUSS_SEIDEL;
    CK(launch_os_rhs(c->g, c->coef, c->rdiag, Jfs, Jold, c->r, gs, c->stream));
    c->stats.launches += 1;
    CK(cudaMemsetAsync(c->dlt, 0, sizeof(double) * max_sweeps, c->stream));
    double* bufs[2] = {c->Ja, c->Jb};
    int launched = 0, done = -1, chunk = 2;
    while (launched < max_sweeps && done < 0) {
        const int n0 = launched;
        const int n1 = launched + chunk < max_sweeps ? launched + chunk : max_sweeps;
        if (c->profiling) CK(cudaEventRecord(c->ev[2], c->stream));
        for (int n = n0; n < n1; ++n) {
            const double* cur = n == 0 ? Jold : bufs[(n - 1) & 1];
            if (gs)
                CK(launch_gs_sweep(c->g, c->coef, c->r, cur, bufs[n & 1], c->dlt, n, tol_inner,
                                   c->stream));
            else
                CK(launch_jacobi(c->g, c->coef, c->r, cur, bufs[n & 1], c->dlt, n, tol_inner,
                                 c->stream));
        }
        if (c->profiling) {
            CK(cudaEventRecord(c->ev[3], c->stream));
            c->jac_pending = true;
        }
        c->stats.launches += (gs ? 2 : 1) * (n1 - n0);
        c->stats.jacobi_launches += (gs ? 2 : 1) * (n1 - n0);
        CK(cudaMemcpyAsync(c->h_dlt + n0, c->dlt + n0, sizeof(double) * (n1 - n0),
                           cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->stats.host_syncs += 1;
        harvest(c);
        for (int n = n0; n < n1; ++n)
            if (c->h_dlt[n] < tol_inner) {
                done = n;
                break;
            }
        launched = n1;
        if (chunk < 32) chunk *= 2;
    }
    const int sweeps = done >= 0 ? done + 1 : max_sweeps;
    CK(cudaMemcpyAsync(Jnew, bufs[(sweeps - 1) & 1], sizeof(double) * c->g.N,
                       cudaMemcpyDeviceToDevice, c->stream));
    if (sweeps_out) *sweeps_out = sweeps;
    return RT_OK;
}

int os_step(rt_ctx* c, const double* Jfs, const double* Jold, double* Jnew, double tol_inner,
            int max_sweeps, int* sweeps, bool device)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = need_all(c))) return rc;
    if (!c->lstar_valid) return fail(c, RT_ESTATE, "Lambda* is not built: run a formal solution first");
    if (!Jfs || !Jold || !Jnew) return fail(c, RT_EINVAL, "null J pointer");
    if (max_sweeps < 1) return fail(c, RT_EINVAL, "max_sweeps must be >= 1");
    const double* dfs = Jfs;
    const double* dold = Jold;
    if (!device) {
        CK(cudaMemcpyAsync(c->Jfs, Jfs, sizeof(double) * c->g.N, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->Jn, Jold, sizeof(double) * c->g.N, cudaMemcpyHostToDevice, c->stream));
        dfs = c->Jfs;
        dold = c->Jn;
    }
    double* dnew = device ? Jnew : c->S;  // S is free as scratch here
    int ns = 0;
    if ((rc = run_os(c, dfs, dold, dnew, tol_inner, max_sweeps, &ns))) return rc;
    if (!device)
        CK(cudaMemcpyAsync(Jnew, dnew, sizeof(double) * c->g.N, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    harvest(c);
    if (ns < 0) ns = os_graph_done(c);
    if (sweeps) *sweeps = ns;
    return RT_OK;
}

int ensure_ng(rt_ctx* c)
{
    if (c->ng_out) return RT_OK;
    for (auto& p : c->ng_old) CK(dalloc(p, (size_t)c->g.N));
    CK(dalloc(c->ng_part, (size_t)ng_partial_size()));
    CK(dalloc(c->ng_out, 5));
    return RT_OK;
}

// Ng bookkeeping after iteration `it` (1-based) produced J_new in c->Jn from
// the previous iterate c->J: remember c->J, and when four iterates are held
// and it is a multiple of the period, enqueue the weighted sums and the
// extrapolation of J_new, whose 2x2 system is solved on the device (no
// host synchronisation; the iterate is left unchanged if it is singular).
int ng_push(rt_ctx* c, int it)
{
    if (!c->ng_period) return RT_OK;
    int rc = ensure_ng(c);
    if (rc) return rc;
    double* t = c->ng_old[2];
    c->ng_old[2] = c->ng_old[1];
    c->ng_old[1] = c->ng_old[0];
    c->ng_old[0] = t;
    CK(cudaMemcpyAsync(c->ng_old[0], c->J, sizeof(double) * c->g.N, cudaMemcpyDeviceToDevice,
                       c->stream));
    if (c->ng_count < 4) ++c->ng_count;
    if (c->ng_count == 4 && it % c->ng_period == 0 &&
        (it == 1 || c->ng_last_delta >= c->ng_min_delta)) {
        CK(launch_ng_dots(c->g.N, c->Jn, c->ng_old[0], c->ng_old[1], c->ng_old[2], c->ng_part,
                          c->ng_out, c->stream));
        CK(launch_ng_apply(c->g.N, c->ng_out, c->ng_old[0], c->ng_old[1], c->Jn, c->stream));
        c->stats.launches += 3;
        c->ng_applied += 1;
        c->ng_count = 1;
    }
    return RT_OK;
}

// Switch between the FP32 sweep and the double-float march (see rt_set_precision).
int switch_precision(rt_ctx* c, int precision)
{
    if (precision == c->precision) return RT_OK;
    const bool ok = (precision == RT_FP32_SWEEP || precision == RT_DF64) &&
                    (c->precision == RT_FP32_SWEEP || c->precision == RT_DF64);
    if (!ok) return fail(c, RT_EINVAL, "precision switches only between RT_FP32_SWEEP and RT_DF64");
    if (precision == RT_FP32_SWEEP && c->fs_method == RT_FS_SHORT)
        return fail(c, RT_EINVAL, "short characteristics have no FP32-sweep form");
    int rc = form_buffers(c, precision);
    if (rc) return rc;
    c->precision = precision;
    c->rec_valid = false;
    c->gdiff_valid = false;    // the gradient's packed copy differs between the forms
    c->lstar_valid = c->coef_valid = false;   // Lambda* is rebuilt by the new form's kernel
    c->ng_count = 1;           // restart the Ng history with iterates of the new form
    return RT_OK;
}

int solve(rt_ctx* c, double tol, int max_iter, double tol_inner, int max_sweeps, double* J_out,
          int* iters, double* last_delta, double* deltas, int* sweeps, bool device)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = need_all(c))) return rc;
    if (max_iter < 1 || max_sweeps < 1 || !(tol >= 0) || !(tol_inner >= 0))
        return fail(c, RT_EINVAL, "bad iteration controls");
    // finishing stage: the context leaves it, and gets its Ng threshold
    // back, when the solve ends, whichever way it ends
    struct FinishGuard {
        rt_ctx* c;
        double ng_min;
        bool on;
        ~FinishGuard()
        {
            if (on) {
                c->fin = 0;
                c->ng_min_delta = ng_min;
            }
        }
    } guard{c, c->ng_min_delta, false};
    int it = 0;
    double delta = 0.0;
    bool converged = false;
    unsigned long long total_steps = 0;
    while (it < max_iter) {
        if ((rc = prepare_source(c, nullptr, true))) return rc;
        if ((rc = run_fs(c, c->Jfs, true))) return rc;
        int ns = 0;
        if ((rc = run_os(c, c->Jfs, c->J, c->Jn, tol_inner, max_sweeps, &ns))) return rc;
        if ((rc = ng_push(c, it + 1))) return rc;
        CK(cudaMemsetAsync(c->scal + 2, 0, sizeof(double), c->stream));
        CK(launch_rel_change(c->g.N, c->Jn, c->J, c->scal + 2, c->stream));
        c->stats.launches += 1;
        CK(cudaMemcpyAsync(c->h_scal + 2, c->scal + 2, sizeof(double), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->stats.host_syncs += 1;
        c->stats.iterations += 1;
        harvest(c);
        if (ns < 0) ns = os_graph_done(c);
        total_steps += *c->h_steps;
        delta = c->h_scal[2];
        c->ng_last_delta = delta;
        double* t = c->J;
        c->J = c->Jn;
        c->Jn = t;
        if (deltas) deltas[it] = delta;
        if (sweeps) sweeps[it] = ns;
        ++it;
        if (tol > 0 && delta < tol) {
            converged = true;
            break;
        }
        if (!guard.on && c->df_switch > 0 && c->precision == RT_FP32_SWEEP && delta < c->df_switch) {
            c->fin = 1;               // next formal solution: the double-float reference
            c->ng_min_delta = 0.0;    // Ng on every period from here
            c->ng_count = 1;          // its history restarts with FP64-accurate iterates
            guard.on = true;
        }
    }
    c->last_steps = total_steps;
    c->stats.steps += total_steps;
    if (J_out) {
        CK(cudaMemcpyAsync(J_out, c->J, sizeof(double) * c->g.N,
                           device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    if (iters) *iters = it;
    if (last_delta) *last_delta = delta;
    if (tol > 0 && !converged)
        return fail(c, RT_ENOTCONV, "not converged after %d iterations (delta %.3e >= tol %.3e)",
                    it, delta, tol);
    return RT_OK;
}

// ---- batched wavelengths ----------------------------------------------------

}  // namespace

struct rt_batch {
    int device = 0;
    int precision = RT_FP32_SWEEP;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    std::vector<rt_ctx*> ctx;       // one per wavelength, all on `stream`
    std::vector<int> order;         // problems by decreasing size (fused launch order)
    std::vector<int> iters;         // outer iterations done since the last reset
    std::vector<double> delta;      // last outer delta
    std::vector<char> converged;
    View32* d_views = nullptr;      // device copies of the per-problem FP32 views
    View32* h_views = nullptr;      // pinned host copies (uploaded when a view changes)
    std::vector<char> view_fin;     // problems whose device view is the finishing-stage one
    int* d_ids = nullptr;
    long long* d_prefix = nullptr;
    int* h_ids = nullptr;           // pinned
    long long* h_prefix = nullptr;  // pinned
    double* d_delta = nullptr;      // outer deltas [nprob]
    double* h_delta = nullptr;      // pinned
    unsigned long long* d_steps = nullptr;
    unsigned long long* h_steps = nullptr;
    int groups_req = 0;
    int threads32 = 0;              // threads per block of the fused FP32 launch (0: 128)
    bool profiling = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool jac_pending = false;
    // The operator-splitting step of all active problems as one CUDA graph:
    // per problem an independent branch (right-hand side, a device-side
    // WHILE loop of sweeps, the pick of the last sweep's buffer).  Keyed by
    // the active set and the buffers it touches; two cached instances,
    // because J and J_new alternate between two buffers.
    struct OsGraph {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        std::vector<const void*> key;
    } osg[2];
    int osg_next = 0;
    bool use_graphs = true;
    int* d_sweeps = nullptr;        // sweeps of each problem's last OS step
    int* h_sweeps = nullptr;        // pinned
    // Recorded marches: a problem starts iterating once its recording fits
    // in the batch's budget (rec_mode: -1 automatic, 0 off, > 0 bytes), so
    // that every problem records in its first formal solution as a single
    // solve does; its memory returns when it converges.
    long long rec_mode = -1;
    std::vector<char> admitted;
    // recording blocks returned by converged problems, handed to the next
    // admitted ones (a large cudaMalloc/cudaFree per problem costs tens of
    // milliseconds); freed when a solve ends
    std::vector<std::pair<char*, long long>> rec_pool;
    Rep32* d_rviews = nullptr;      // replay views (device) and pinned host copies
    Rep32* h_rviews = nullptr;
    int* d_rids = nullptr;
    long long* d_rprefix = nullptr;
    int* h_rids = nullptr;          // pinned
    long long* h_rprefix = nullptr; // pinned
    rt_stats stats{};
    std::string err;
};

namespace {

int bfail(rt_batch* b, int code, const char* fmt, ...)
{
    if (b) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        b->err = buf;
    }
    return code;
}

#define BCK(call)                                                                       \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA,     \
                         "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// Propagate a per-problem failure with the problem's message.
int bpass(rt_batch* b, int p, int rc)
{
    if (rc == RT_OK) return RT_OK;
    return bfail(b, rc, "problem %d: %s", p, b->ctx[p]->err.c_str());
}

int batch_groups(const rt_batch* b, const std::vector<int>& act)
{
    if (b->groups_req > 0) return b->groups_req < kSlots ? b->groups_req : kSlots;
    long long blocks = 0;
    for (int p : act) blocks += fs32_blocks(b->ctx[p]->g, 1, b->threads32);
    int G = 1;
    while (G < kSlots && blocks * G < 64LL * (b->num_sms > 0 ? b->num_sms : 152)) G *= 2;
    return G;
}

// Admit waiting problems (in launch order) whose recorded march fits in the
// batch's budget beside the recordings held; a problem whose form does not
// record, or whose recording could never fit, starts at once and marches.
// When nothing runs and a problem cannot get its memory, it starts marching
// too, so that the solve always progresses.
int batch_admit(rt_batch* b, int max_iter)
{
    long long limit = b->rec_mode, reserve = 0, free_now = 0;
    if (limit < 0) {
        // automatic: recordings up to 60% of the device, each admitted only
        // while what the unconverged problems still allocate (Ng's iterates;
        // at their finishing stage the reference's double-float node planes
        // and tables, S_ref, J_ref and the source change) stays free beside
        // it, with 4 GiB to spare
        size_t fr = 0, tot = 0;
        BCK(cudaMemGetInfo(&fr, &tot));
        limit = (long long)(0.6 * (double)tot);
        reserve = 4LL << 30;
        for (size_t p = 0; p < b->ctx.size(); ++p) {
            const rt_ctx* c = b->ctx[p];
            if (b->converged[p] || c->S_ref) continue;
            reserve += 24 * c->g.N + (c->node4 ? 0 : 64 * c->g.N) +
                       (c->ng_old[0] ? 0 : 24 * c->g.N) +     // Ng's older iterates
                       36LL * c->g.ndir * c->g.nz + (1LL << 20);
        }
        free_now = (long long)fr;
    }
    long long used = 0;
    bool running = false;
    for (size_t p = 0; p < b->ctx.size(); ++p) {
        used += b->ctx[p]->rec_cap;
        if (b->admitted[p] && !b->converged[p] && b->iters[p] < max_iter) running = true;
    }
    for (auto& blk : b->rec_pool) used += blk.second;
    for (int p : b->order) {
        rt_ctx* c = b->ctx[p];
        if (b->admitted[p] || b->converged[p] || b->iters[p] >= max_iter) continue;
        const long long need = rec_need(c);
        // a pooled block that holds the recording
        int pick = -1;
        for (size_t i = 0; i < b->rec_pool.size(); ++i)
            if (b->rec_pool[i].second >= need &&
                (pick < 0 || b->rec_pool[i].second < b->rec_pool[pick].second))
                pick = (int)i;
        if (b->rec_mode != 0 && need > 0 && pick >= 0) {
            c->rec_mem = b->rec_pool[pick].first;
            c->rec_cap = b->rec_pool[pick].second;
            b->rec_pool.erase(b->rec_pool.begin() + pick);
            c->rec_mode = c->rec_cap;
            bool use = false;
            const int rc = ensure_rec(c, use);
            if (rc) return bfail(b, rc, "problem %d: %s", p, rt_last_error(c));
        } else if (b->rec_mode == 0 || need == 0 || need > limit) {
            c->rec_mode = 0;                      // marches
        } else if (used + need <= limit && (reserve == 0 || need + reserve <= free_now)) {
            c->rec_mode = need;
            bool use = false;
            const int rc = ensure_rec(c, use);
            if (rc) return bfail(b, rc, "problem %d: %s", p, rt_last_error(c));
            if (use) {
                used += c->rec_cap;
                free_now -= c->rec_cap;
            } else if (running) {
                continue;                         // wait for memory
            } else {
                c->rec_mode = 0;
            }
        } else if (running) {
            continue;                             // wait for memory
        } else {
            c->rec_mode = 0;
        }
        b->admitted[p] = 1;
        running = true;
    }
    return RT_OK;
}

// A problem that stops iterating returns its recording's memory to the
// batch's pool.
void batch_release(rt_batch* b, int p)
{
    rt_ctx* c = b->ctx[p];
    if (c->rec_cap) {
        cudaStreamSynchronize(b->stream);
        b->rec_pool.emplace_back(c->rec_mem, c->rec_cap);
        c->rec_mem = nullptr;
        c->rec_cap = 0;
        c->rec = FsRec{};
        c->rec32 = Rec32{};
        c->spair = nullptr;
        c->rec_valid = false;
    }
}

void batch_free_pool(rt_batch* b)
{
    if (b->rec_pool.empty()) return;
    cudaStreamSynchronize(b->stream);
    for (auto& blk : b->rec_pool) cudaFree(blk.first);
    b->rec_pool.clear();
}

void bharvest(rt_batch* b)
{
    float ms = 0.f;
    if (b->profiling && cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]) == cudaSuccess)
        b->stats.fs_ms += ms;
    if (b->jac_pending && cudaEventElapsedTime(&ms, b->ev[2], b->ev[3]) == cudaSuccess)
        b->stats.jacobi_ms += ms;
    b->jac_pending = false;
}

void free_batch_graphs(rt_batch* b)
{
    for (auto& e : b->osg) {
        if (e.exec) cudaGraphExecDestroy(e.exec);
        if (e.graph) cudaGraphDestroy(e.graph);
        e = rt_batch::OsGraph{};
    }
}

std::vector<const void*> batch_graph_key(const rt_batch* b, const std::vector<int>& act,
                                         double tol, int max_sweeps)
{
    std::vector<const void*> k;
    k.push_back(reinterpret_cast<const void*>((intptr_t)max_sweeps));
    long long tb;
    std::memcpy(&tb, &tol, sizeof tb);
    k.push_back(reinterpret_cast<const void*>((intptr_t)tb));
    for (int p : act) {
        const rt_ctx* c = b->ctx[p];
        k.push_back(reinterpret_cast<const void*>((intptr_t)p));
        k.push_back(reinterpret_cast<const void*>((intptr_t)c->os_method));
        for (const void* q : {(const void*)c->J, (const void*)c->Jn, (const void*)c->Jfs,
                              (const void*)c->coef, (const void*)c->rdiag, (const void*)c->r,
                              (const void*)c->Ja, (const void*)c->Jb, (const void*)c->dlt,
                              (const void*)c->d_nsw})
            k.push_back(q);
    }
    return k;
}

// Capture the per-problem branches of the batch operator-splitting graph.
// Every capture that begins is ended, also after an error.
cudaError_t build_batch_os_graph(rt_batch* b, const std::vector<int>& act, double tol,
                                 int max_sweeps, cudaGraph_t* out)
{
    cudaGraph_t g = nullptr;
    cudaError_t err = cudaGraphCreate(&g, 0);
    if (err != cudaSuccess) return err;
    const cudaStream_t st = b->stream;
    for (int p : act) {
        rt_ctx* c = b->ctx[p];
        const bool gs = c->os_method == RT_OS_GAUSS_SEIDEL;
        cudaGraphConditionalHandle h;
        err = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
        if (err != cudaSuccess) break;
        // prologue, a branch of its own (no dependencies)
        err = cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal);
        if (err != cudaSuccess) break;
        std::vector<cudaGraphNode_t> deps;
        {
            cudaError_t e1 = launch_os_rhs(c->g, c->coef, c->rdiag, c->Jfs, c->J, c->r, gs, st);
            cudaError_t e2 = cudaMemsetAsync(c->dlt, 0, sizeof(double) * (max_sweeps + 2), st);
            cudaError_t e3 = cudaMemcpyAsync(c->Jb, c->J, sizeof(double) * c->g.N,
                                             cudaMemcpyDeviceToDevice, st);
            cudaError_t e4 = cudaMemsetAsync(c->d_nsw, 0, sizeof(int), st);
            cudaStreamCaptureStatus cs;
            const cudaGraphNode_t* dp = nullptr;
            size_t nd = 0;
            cudaError_t e5 = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &dp, nullptr, &nd);
            if (e5 == cudaSuccess) deps.assign(dp, dp + nd);
            cudaGraph_t o = nullptr;
            cudaError_t e6 = cudaStreamEndCapture(st, &o);
            for (cudaError_t x : {e1, e2, e3, e4, e5, e6})
                if (err == cudaSuccess && x != cudaSuccess) err = x;
        }
        if (err != cudaSuccess) break;
        // the sweep loop
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cn;
        err = cudaGraphAddNode(&cn, g, deps.data(), nullptr, deps.size(), &cp);
        if (err != cudaSuccess) break;
        err = cudaStreamBeginCaptureToGraph(st, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal);
        if (err != cudaSuccess) break;
        {
            cudaError_t e1 = launch_sweep_pass(c->g, c->coef, c->r, c->Ja, c->Jb, c->dlt, c->d_nsw,
                                               max_sweeps, tol, gs, h, st);
            cudaGraph_t o = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(st, &o);
            err = e1 != cudaSuccess ? e1 : e2;
        }
        if (err != cudaSuccess) break;
        // epilogue: the last sweep's iterate into J_new, after the loop
        err = cudaStreamBeginCaptureToGraph(st, g, &cn, nullptr, 1, cudaStreamCaptureModeThreadLocal);
        if (err != cudaSuccess) break;
        {
            cudaError_t e1 = launch_os_select(c->g.N, c->dlt, max_sweeps, tol, c->Ja, c->Jb, c->Jn,
                                              b->d_sweeps + p, st);
            cudaGraph_t o = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(st, &o);
            err = e1 != cudaSuccess ? e1 : e2;
        }
        if (err != cudaSuccess) break;
    }
    if (err != cudaSuccess) {
        cudaGraphDestroy(g);
        return err;
    }
    *out = g;
    return cudaSuccess;
}

// Formal solutions of the active problems: FP32 sweep in one fused launch,
// FP64 one launch per problem.
int batch_fs(rt_batch* b, const std::vector<int>& act)
{
    int rc;
    for (int p : act) {
        rt_ctx* c = b->ctx[p];
        if ((rc = bpass(b, p, prepare_source(c, nullptr, true)))) return rc;
        if ((rc = bpass(b, p, fs_prepare(c)))) return rc;
    }
    const int G = batch_groups(b, act);
    BCK(cudaMemsetAsync(b->d_steps, 0, sizeof(unsigned long long), b->stream));
    if (b->profiling) BCK(cudaEventRecord(b->ev[0], b->stream));
    if (b->precision == RT_FP32_SWEEP) {
        // problems holding a recording: record it in their first formal
        // solution, then one fused replay over all of them (their source, or
        // in the finishing stage its change, packed for the replay)
        long long rtotal = 0;
        int rq = 0;
        std::vector<char> replays(b->ctx.size(), 0);
        for (int p : act) {
            rt_ctx* c = b->ctx[p];
            if (c->precision != RT_FP32_SWEEP || c->fin == 1) continue;
            bool use = false;
            if ((rc = bpass(b, p, ensure_rec(c, use)))) return rc;
            if (!use) continue;
            if (!c->rec_valid) {
                if (c->fin != 0) continue;
                BCK(launch_fs32rec(view32(c), cut_of(c) * kRecCutMargin, G, c->rec32, b->d_steps,
                                   b->stream));
                c->rec_valid = true;
                b->stats.launches += 1;
            }
            BCK(launch_pack_spairs(c->g, c->fin == 2 ? c->dS : c->S, c->spair, b->stream));
            b->stats.launches += 1;
            b->h_rviews[p] = Rep32{c->g, c->spair, c->info, c->poff32, c->bw32, c->rec32,
                                   c->partial, c->fin == 2 ? 1 : 0, plane_major32(c->g, c->order32)};
            b->h_rids[rq] = p;
            b->h_rprefix[rq] = rtotal;
            rtotal += fs32_blocks(c->g, G, b->threads32);
            ++rq;
            replays[p] = 1;
        }
        b->h_rprefix[rq] = rtotal;
        if (rq > 0) {
            BCK(cudaMemcpyAsync(b->d_rviews, b->h_rviews, sizeof(Rep32) * b->ctx.size(),
                                cudaMemcpyHostToDevice, b->stream));
            BCK(cudaMemcpyAsync(b->d_rids, b->h_rids, sizeof(int) * rq, cudaMemcpyHostToDevice,
                                b->stream));
            BCK(cudaMemcpyAsync(b->d_rprefix, b->h_rprefix, sizeof(long long) * (rq + 1),
                                cudaMemcpyHostToDevice, b->stream));
            BCK(launch_fs32rep_batch(b->d_rviews, b->d_rids, b->d_rprefix, rq, rtotal, G,
                                     b->threads32, b->d_steps, b->stream));
            b->stats.fs_launches += 1;
            b->stats.launches += 1;
        }
        // one fused launch over the other problems in the FP32 sweep, including
        // those marching their source change in the finishing stage (act is
        // in launch order); a finishing-stage reference and problems switched
        // to the double-float march by hand run one launch each
        long long total = 0;
        int q = 0;
        for (int p : act) {
            rt_ctx* c = b->ctx[p];
            if (c->precision != RT_FP32_SWEEP || c->fin == 1 || replays[p]) continue;
            const char want = c->fin == 2;
            if (b->view_fin[p] != want) {     // this problem's view changed form
                b->h_views[p] = want ? view32_fin(c) : view32(c);
                BCK(cudaMemcpyAsync(b->d_views + p, b->h_views + p, sizeof(View32),
                                    cudaMemcpyHostToDevice, b->stream));
                b->view_fin[p] = want;
            }
            b->h_ids[q] = p;
            b->h_prefix[q] = total;
            total += fs32_blocks(c->g, G, b->threads32);
            ++q;
        }
        b->h_prefix[q] = total;
        if (q > 0) {
            BCK(cudaMemcpyAsync(b->d_ids, b->h_ids, sizeof(int) * q, cudaMemcpyHostToDevice,
                                b->stream));
            BCK(cudaMemcpyAsync(b->d_prefix, b->h_prefix, sizeof(long long) * (q + 1),
                                cudaMemcpyHostToDevice, b->stream));
            BCK(launch_fs32_batch(b->d_views, b->d_ids, b->d_prefix, q, total, G, b->threads32,
                                  cut_of(b->ctx[0]), b->d_steps, b->stream));
            b->stats.fs_launches += 1;
            b->stats.launches += 1;
        }
        for (int p : act) {
            rt_ctx* c = b->ctx[p];
            if (c->precision == RT_DF64) {
                if ((rc = bpass(b, p, df_formal(c, G, b->d_steps, b->stream)))) return rc;
            } else if (c->fin == 1) {
                if ((rc = bpass(b, p, fin_reference_march(c, G, b->d_steps, b->stream)))) return rc;
            } else {
                continue;
            }
            b->stats.fs_launches += 1;
            b->stats.launches += 1;
        }
    } else {
        for (int p : act) {
            rt_ctx* c = b->ctx[p];
            bool use = false;
            if (b->precision == RT_FP64 && (rc = bpass(b, p, ensure_rec(c, use)))) return rc;
            if (b->precision == RT_DF64) {
                if ((rc = bpass(b, p, df_formal(c, G, b->d_steps, b->stream)))) return rc;
            } else if (use) {
                if (!c->rec_valid) {
                    BCK(launch_fs64(c->g, c->chi, c->S, c->B, c->gdiff, c->info, c->off, c->bw,
                                    c->bwh, c->scal + 0, cut_of(c), G, c->partial, b->d_steps,
                                    b->stream, &c->rec));
                    c->rec_valid = true;
                    b->stats.launches += 1;
                }
                BCK(launch_fs64rep(c->g, c->S, c->info, c->off, c->bw, c->rec, G, c->partial,
                                   b->d_steps, b->stream));
            } else {
                BCK(launch_fs64(c->g, c->chi, c->S, c->B, c->gdiff, c->info, c->off, c->bw,
                                c->bwh, c->scal + 0, cut_of(c), G, c->partial, b->d_steps,
                                b->stream));
            }
            b->stats.fs_launches += 1;
            b->stats.launches += 1;
        }
    }
    if (b->profiling) BCK(cudaEventRecord(b->ev[1], b->stream));
    for (int p : act) {
        rt_ctx* c = b->ctx[p];
        if ((rc = bpass(b, p, fs_finish(c, c->Jfs)))) return rc;
        if (c->precision == RT_FP32_SWEEP && c->fin == 1 &&
            (rc = bpass(b, p, fin_record(c, c->Jfs, b->stream))))
            return rc;
    }
    BCK(cudaMemcpyAsync(b->h_steps, b->d_steps, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        b->stream));
    return RT_OK;
}

// Operator-splitting solves of the active problems as one graph launch (no
// host synchronisation); the sweep counts reach b->d_sweeps.
int batch_os_graph(rt_batch* b, const std::vector<int>& act, double tol_inner, int max_sweeps)
{
    int rc;
    for (int p : act) {
        rt_ctx* c = b->ctx[p];
        if ((rc = bpass(b, p, ensure_coef(c)))) return rc;
        if ((rc = bpass(b, p, ensure_dlt(c, max_sweeps + 2)))) return rc;
        if (!c->d_nsw) BCK(cudaMalloc((void**)&c->d_nsw, sizeof(int)));
    }
    std::vector<const void*> key = batch_graph_key(b, act, tol_inner, max_sweeps);
    rt_batch::OsGraph* e = nullptr;
    for (auto& x : b->osg)
        if (x.exec && x.key == key) e = &x;
    if (!e) {
        e = &b->osg[b->osg_next];
        b->osg_next ^= 1;
        if (e->exec) cudaGraphExecDestroy(e->exec);
        if (e->graph) cudaGraphDestroy(e->graph);
        *e = rt_batch::OsGraph{};
        cudaGraph_t g = nullptr;
        cudaError_t err = build_batch_os_graph(b, act, tol_inner, max_sweeps, &g);
        cudaGraphExec_t exec = nullptr;
        if (err == cudaSuccess) {
            err = cudaGraphInstantiate(&exec, g, 0);
            if (err != cudaSuccess) cudaGraphDestroy(g);
        }
        if (err != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, RT_ECUDA, "building the batch operator-splitting graph: %s",
                         cudaGetErrorString(err));
        }
        e->graph = g;
        e->exec = exec;
        e->key.swap(key);
        b->stats.launches += 0;
    }
    if (b->profiling) BCK(cudaEventRecord(b->ev[2], b->stream));
    BCK(cudaGraphLaunch(e->exec, b->stream));
    if (b->profiling) {
        BCK(cudaEventRecord(b->ev[3], b->stream));
        b->jac_pending = true;
    }
    return RT_OK;
}

// Launch counts of the graph-driven operator splitting of `act`, from the
// sweep counts the graph wrote (read after the iteration's synchronisation).
void batch_os_graph_counts(rt_batch* b, const std::vector<int>& act)
{
    for (int p : act) {
        const int per = b->ctx[p]->os_method == RT_OS_GAUSS_SEIDEL ? 2 : 1;
        const int passes = (b->h_sweeps[p] + 1) / 2;
        b->stats.launches += 2 + passes * (2 * per + 1);
        b->stats.jacobi_launches += passes * 2 * per;
    }
}

// Operator-splitting solves of the active problems without graphs; sweeps
// are enqueued in chunks for every problem still iterating and checked with
// one host sync per chunk (a sweep after a converged one is a device-side
// no-op).
int batch_os(rt_batch* b, const std::vector<int>& act, double tol_inner, int max_sweeps)
{
    int rc;
    std::vector<int> inner;
    for (int p : act) {
        rt_ctx* c = b->ctx[p];
        if ((rc = bpass(b, p, ensure_coef(c)))) return rc;
        if ((rc = bpass(b, p, ensure_dlt(c, max_sweeps)))) return rc;
        BCK(launch_os_rhs(c->g, c->coef, c->rdiag, c->Jfs, c->J, c->r,
                          c->os_method == RT_OS_GAUSS_SEIDEL, b->stream));
        BCK(cudaMemsetAsync(c->dlt, 0, sizeof(double) * max_sweeps, b->stream));
        b->stats.launches += 1;
        inner.push_back(p);
    }
    std::vector<int> sweeps(b->ctx.size(), max_sweeps);
    int launched = 0, chunk = 2;
    while (!inner.empty() && launched < max_sweeps) {
        const int n0 = launched;
        const int n1 = launched + chunk < max_sweeps ? launched + chunk : max_sweeps;
        for (int p : inner) {
            rt_ctx* c = b->ctx[p];
            for (int n = n0; n < n1; ++n) {
                const double* cur = n == 0 ? c->J : (n & 1 ? c->Ja : c->Jb);
                double* nxt = n & 1 ? c->Jb : c->Ja;
                if (c->os_method == RT_OS_GAUSS_SEIDEL)
                    BCK(launch_gs_sweep(c->g, c->coef, c->r, cur, nxt, c->dlt, n, tol_inner,
                                        b->stream));
                else
                    BCK(launch_jacobi(c->g, c->coef, c->r, cur, nxt, c->dlt, n, tol_inner,
                                      b->stream));
            }
            BCK(cudaMemcpyAsync(c->h_dlt + n0, c->dlt + n0, sizeof(double) * (n1 - n0),
                                cudaMemcpyDeviceToHost, b->stream));
            const int per = c->os_method == RT_OS_GAUSS_SEIDEL ? 2 : 1;
            b->stats.launches += per * (n1 - n0);
            b->stats.jacobi_launches += per * (n1 - n0);
        }
        BCK(cudaStreamSynchronize(b->stream));
        b->stats.host_syncs += 1;
        std::vector<int> still;
        for (int p : inner) {
            rt_ctx* c = b->ctx[p];
            int done = -1;
            for (int n = n0; n < n1; ++n)
                if (c->h_dlt[n] < tol_inner) {
                    done = n;
                    break;
                }
            if (done >= 0) sweeps[p] = done + 1; else still.push_back(p);
        }
        inner.swap(still);
        launched = n1;
        if (chunk < 32) chunk *= 2;
    }
    for (int p : act) {
        rt_ctx* c = b->ctx[p];
        BCK(cudaMemcpyAsync(c->Jn, (sweeps[p] - 1) & 1 ? c->Jb : c->Ja, sizeof(double) * c->g.N,
                            cudaMemcpyDeviceToDevice, b->stream));
    }
    return RT_OK;
}

}  // namespace

extern "C" {

const char* rt_version(void) { return "rt3d 0.1 (sm_103a)"; }

int rt_create(rt_ctx** out, int device, int precision)
{
    if (!out) return RT_EINVAL;
    *out = nullptr;
    if (precision != RT_FP64 && precision != RT_FP32_SWEEP && precision != RT_DF64) return RT_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return RT_ECUDA;
    rt_ctx* c = new rt_ctx();
    c->device = device;
    c->precision = precision;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc((void**)&c->scal, 4 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&c->d_steps, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_scal, 4 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_steps, sizeof(unsigned long long)) != cudaSuccess ||
        cudaEventCreate(&c->ev[0]) != cudaSuccess || cudaEventCreate(&c->ev[1]) != cudaSuccess ||
        cudaEventCreate(&c->ev[2]) != cudaSuccess || cudaEventCreate(&c->ev[3]) != cudaSuccess) {
        rt_destroy(c);
        return RT_ECUDA;
    }
    *c->h_steps = 0;
    c->stream = c->own_stream;
    // the FP32 sweep finishes in double-float by default (rt_set_df_finish)
    c->df_switch = precision == RT_FP32_SWEEP ? kDefaultDfSwitch : 0.0;
    c->g.top_bc = RT_BC_ZERO;
    c->g.bottom_bc = RT_BC_PLANCK;
#ifdef RT_CHECKED
    if (cudaMalloc((void**)&c->berr, 4 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(c->berr, 0, 4 * sizeof(unsigned long long)) != cudaSuccess) {
        rt_destroy(c);
        return RT_ECUDA;
    }
#endif
    c->g.berr = c->berr;
    *out = c;
    return RT_OK;
}

int rt_destroy(rt_ctx* c)
{
    if (!c) return RT_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_grid_buffers(c);
    free_tables(c);
    dfree(c->scal);
    dfree(c->d_steps);
    dfree(c->berr);
    if (c->d_nsw) cudaFree(c->d_nsw);
    c->d_nsw = nullptr;
    if (c->d_sw) cudaFree(c->d_sw);
    c->d_sw = nullptr;
    if (c->h_sw) cudaFreeHost(c->h_sw);
    c->h_sw = nullptr;
    if (c->h_scal) cudaFreeHost(c->h_scal);
    if (c->h_steps) cudaFreeHost(c->h_steps);
    if (c->h_dlt) cudaFreeHost(c->h_dlt);
    dfree(c->dlt);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
    return RT_OK;
}

const char* rt_last_error(const rt_ctx* c) { return c ? c->err.c_str() : "null context"; }

int rt_set_stream(rt_ctx* c, void* stream)
{
    int rc = enter(c);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    c->stream = stream ? (cudaStream_t)stream : c->own_stream;
    return RT_OK;
}

int rt_set_grid(rt_ctx* c, int nx, int ny, int nz, double dx, double dy, double dz)
{
    int rc = enter(c);
    if (rc) return rc;
    if (nx < 3 || ny < 3 || nz < 2 || nz > 65535)
        return fail(c, RT_EINVAL, "grid %dx%dx%d: need nx, ny >= 3 and 2 <= nz <= 65535", nx, ny,
                    nz);
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !std::isfinite(dx) || !std::isfinite(dy) ||
        !std::isfinite(dz))
        return fail(c, RT_EINVAL, "spacings must be finite and > 0");
    if ((long long)nx * ny > (1LL << 30) || (long long)nx * ny * nz > (1LL << 40))
        return fail(c, RT_EINVAL, "grid too large");
    if (c->precision != RT_FP64 && (2LL * ny + 1) * 2LL * nx * nz >= (1LL << 31))
        return fail(c, RT_EINVAL,
                    "grid too large for the FP32-sweep and double-float forms "
                    "((2ny+1)*2nx*nz >= 2^31)");
    CK(cudaStreamSynchronize(c->stream));
    free_grid_buffers(c);
    free_tables(c);
    c->have_grid = c->have_quad = c->have_chi = c->have_eps = c->have_B = false;
    c->lstar_valid = c->coef_valid = c->b2_valid = c->rec_valid = false;
    c->g.nx = nx; c->g.ny = ny; c->g.nz = nz;
    c->g.N = (long long)nx * ny * nz;
    c->g.ndir = 0;
    c->dx = dx; c->dy = dy; c->dz = dz;
    const size_t N = (size_t)c->g.N;
    CK(dalloc(c->chi, N)); CK(dalloc(c->eps, N)); CK(dalloc(c->B, N)); CK(dalloc(c->J, N));
    CK(dalloc(c->S, N)); CK(dalloc(c->Jfs, N)); CK(dalloc(c->Jn, N)); CK(dalloc(c->Ja, N));
    // r, 1/diag and c sized for either storage (colour-split >= N)
    const size_t Ns = (size_t)os_coef_stride(c->g, true);
    CK(dalloc(c->Jb, N)); CK(dalloc(c->r, Ns)); CK(dalloc(c->rdiag, Ns));
    CK(dalloc(c->lstar, 27 * N)); CK(dalloc(c->coef, 27 * Ns));
    CK(dalloc(c->gdiff, (size_t)nx * ny));
    CK(dalloc(c->zorder, (size_t)nz)); CK(dalloc(c->zscratch, 2 * (size_t)nz));
    if (c->precision != RT_FP64) {
        CK(dalloc(c->b2, (size_t)8 * nx * ny));
        CK(dalloc(c->g2, (size_t)4 * nx * ny));
    }
    c->have_grid = true;
    return form_buffers(c, c->precision);
}

int rt_set_boundary(rt_ctx* c, int top_mode, int bottom_mode)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((top_mode != RT_BC_ZERO && top_mode != RT_BC_PLANCK) ||
        (bottom_mode != RT_BC_ZERO && bottom_mode != RT_BC_PLANCK && bottom_mode != RT_BC_DIFFUSION))
        return fail(c, RT_EINVAL, "boundary modes: top ZERO or PLANCK, bottom ZERO, PLANCK or DIFFUSION");
    c->g.top_bc = top_mode;
    c->g.bottom_bc = bottom_mode;
    c->gdiff_valid = c->rec_valid = false;
    return RT_OK;
}

int rt_set_quadrature(rt_ctx* c, int ndir, const double* mu, const double* phi, const double* w)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = need(c, c->have_grid, "the grid"))) return rc;
    if (ndir < 1 || !mu || !phi || !w) return fail(c, RT_EINVAL, "bad quadrature arrays");
    double sw = 0.0;
    for (int d = 0; d < ndir; ++d) {
        if (!std::isfinite(mu[d]) || !std::isfinite(phi[d]) || !std::isfinite(w[d]))
            return fail(c, RT_EINVAL, "direction %d is not finite", d);
        if (!(std::fabs(mu[d]) >= 1e-6) || !(std::fabs(mu[d]) <= 1.0))
            return fail(c, RT_EINVAL, "mu[%d] = %g: need 1e-6 <= |mu| <= 1", d, mu[d]);
        if (!(w[d] >= 0)) return fail(c, RT_EINVAL, "w[%d] = %g < 0", d, w[d]);
        sw += w[d];
    }
    if (std::fabs(sw - 1.0) > 1e-12) return fail(c, RT_EINVAL, "weights sum to %.17g, not 1", sw);
    CK(cudaStreamSynchronize(c->stream));
    free_tables(c);
    c->have_quad = false;
    c->g.ndir = ndir;
    const size_t T = (size_t)ndir * c->g.nz;
    CK(dalloc(c->d_mu, ndir)); CK(dalloc(c->d_phi, ndir)); CK(dalloc(c->d_w, ndir));
    CK(dalloc(c->info, ndir)); CK(dalloc(c->off, T)); CK(dalloc(c->bw, T));
    CK(dalloc(c->bwh, T)); CK(dalloc(c->bw32, T));
    CK(cudaMemcpyAsync(c->d_mu, mu, sizeof(double) * ndir, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_phi, phi, sizeof(double) * ndir, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_w, w, sizeof(double) * ndir, cudaMemcpyHostToDevice, c->stream));
    CK(launch_dir_tables(c->g, c->dx, c->dy, c->dz, c->d_mu, c->d_phi, c->d_w, c->info, c->off,
                         c->bw, c->bwh, c->bw32, c->stream));
    c->stats.launches += 1;
    if (c->precision != RT_FP64) {
        CK(dalloc(c->poff, T));
        CK(dalloc(c->poff32, T));
        CK(launch_pad_offsets(c->g, c->info, c->off, 2LL * c->g.ny, c->poff, c->stream));
        CK(launch_pad_offsets(c->g, c->info, c->off, 2LL * c->g.ny + 1, c->poff32, c->stream));
        c->stats.launches += 2;
    } else {
        CK(dalloc(c->dn, (size_t)ndir));
        CK(launch_down_tables(c->g, c->dx, c->dy, c->dz, c->d_mu, c->d_phi, c->dn, c->stream));
        c->stats.launches += 1;
    }
    c->wsum = sw;
    c->have_quad = true;
    if ((rc = form_buffers(c, c->precision))) {
        c->have_quad = false;
        return rc;
    }
    CK(cudaStreamSynchronize(c->stream));
    c->lstar_valid = c->coef_valid = c->rec_valid = false;
    return RT_OK;
}

static int set_chi(rt_ctx* c, const double* chi, bool device)
{
    int rc = set_field(c, chi, c ? c->chi : nullptr, device, "chi", true, false);
    if (rc) return rc;
    // the planes' dispatch order follows the new opacities (stream-ordered
    // before any march that reads it)
    CK(launch_plane_order(c->g, c->dz, c->chi, c->zscratch, c->zorder, c->stream));
    c->g.zorder = c->zorder;
    c->stats.launches += 2;
    c->have_chi = true;
    c->lstar_valid = c->coef_valid = c->gdiff_valid = c->rec_valid = false;
    return RT_OK;
}

static int set_eps(rt_ctx* c, const double* eps, bool device)
{
    int rc = set_field(c, eps, c ? c->eps : nullptr, device, "eps", false, true);
    if (rc) return rc;
    c->have_eps = true;
    c->coef_valid = false;
    return RT_OK;
}

static int set_B(rt_ctx* c, const double* B, bool device)
{
    int rc = set_field(c, B, c ? c->B : nullptr, device, "B", false, false);
    if (rc) return rc;
    CK(cudaMemcpyAsync(c->J, c->B, sizeof(double) * c->g.N, cudaMemcpyDeviceToDevice, c->stream));
    c->ng_count = 1;
    c->ng_last_delta = 0.0;
    c->have_B = true;
    c->b2_valid = c->gdiff_valid = c->rec_valid = false;
    return RT_OK;
}

int rt_set_opacity(rt_ctx* c, const double* chi) { return set_chi(c, chi, false); }
int rt_set_epsilon(rt_ctx* c, const double* eps) { return set_eps(c, eps, false); }
int rt_set_planck(rt_ctx* c, const double* B) { return set_B(c, B, false); }
int rt_set_opacity_dev(rt_ctx* c, const double* chi) { return set_chi(c, chi, true); }
int rt_set_epsilon_dev(rt_ctx* c, const double* eps) { return set_eps(c, eps, true); }
int rt_set_planck_dev(rt_ctx* c, const double* B) { return set_B(c, B, true); }

int rt_formal_solution(rt_ctx* c, const double* S, double* J_fs, double* lstar)
{
    return check_bounds(c, formal_solution(c, S, J_fs, lstar, false));
}

int rt_formal_solution_dev(rt_ctx* c, const double* S, double* J_fs, double* lstar)
{
    return check_bounds(c, formal_solution(c, S, J_fs, lstar, true));
}

int rt_os_step(rt_ctx* c, const double* J_fs, const double* J_old, double* J_new, double tol_inner,
               int max_sweeps, int* sweeps)
{
    return check_bounds(c, os_step(c, J_fs, J_old, J_new, tol_inner, max_sweeps, sweeps, false));
}

int rt_os_step_dev(rt_ctx* c, const double* J_fs, const double* J_old, double* J_new,
                   double tol_inner, int max_sweeps, int* sweeps)
{
    return check_bounds(c, os_step(c, J_fs, J_old, J_new, tol_inner, max_sweeps, sweeps, true));
}

int rt_solve(rt_ctx* c, double tol, int max_iter, double tol_inner, int max_sweeps, double* J_out,
             int* iters, double* last_delta, double* deltas, int* sweeps)
{
    return check_bounds(c, solve(c, tol, max_iter, tol_inner, max_sweeps, J_out, iters, last_delta,
                                 deltas, sweeps, false));
}

int rt_solve_dev(rt_ctx* c, double tol, int max_iter, double tol_inner, int max_sweeps,
                 double* J_out, int* iters, double* last_delta, double* deltas, int* sweeps)
{
    return check_bounds(c, solve(c, tol, max_iter, tol_inner, max_sweeps, J_out, iters, last_delta,
                                 deltas, sweeps, true));
}

int rt_get_J(rt_ctx* c, double* J)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = need(c, c->have_B, "the Planck function (initial J)"))) return rc;
    if (!J) return fail(c, RT_EINVAL, "J is NULL");
    CK(cudaMemcpyAsync(J, c->J, sizeof(double) * c->g.N, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return RT_OK;
}

int rt_set_J(rt_ctx* c, const double* J)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = need(c, c->have_B, "the Planck function"))) return rc;
    if (!J) return fail(c, RT_EINVAL, "J is NULL");
    if ((rc = check_field(c, J, "J", false, false))) return rc;
    CK(cudaMemcpyAsync(c->J, J, sizeof(double) * c->g.N, cudaMemcpyHostToDevice, c->stream));
    c->ng_count = 1;
    CK(cudaStreamSynchronize(c->stream));
    return RT_OK;
}

// Diagnostics: one FP32 march of the source S (host, or NULL for
// eps B + (1 - eps) J) through the branch-counting kernel instantiation.
static int fs32_branch_counts(rt_ctx* c, const double* S, unsigned long long* steps,
                              unsigned long long* series)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = need_all(c))) return rc;
    if (!steps || !series) return fail(c, RT_EINVAL, "steps or series is NULL");
    if (c->precision != RT_FP32_SWEEP || c->fs_method != RT_FS_LONG)
        return fail(c, RT_EINVAL, "branch counts need the FP32-sweep long-characteristics march");
    if ((rc = prepare_source(c, S, false))) return rc;
    if ((rc = fs_prepare(c))) return rc;
    CK(launch_pack_pairs(c->g, c->chi, c->S, c->pair, c->plo, c->stream));
    unsigned long long* d = nullptr;
    CK(cudaMalloc((void**)&d, 2 * sizeof(unsigned long long)));
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(d, 0, 2 * sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess)
        e = launch_fs32d(view32(c), cut_of(c), auto_groups(c), c->threads32, d, c->stream, d + 1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(c, RT_ECUDA, "CUDA error %s", cudaGetErrorString(e));
    c->stats.launches += 1;
    *steps = h[0];
    *series = h[1];
    return RT_OK;
}

int rt_fs32_branch_counts(rt_ctx* c, const double* S, unsigned long long* steps,
                          unsigned long long* series)
{
    return check_bounds(c, fs32_branch_counts(c, S, steps, series));
}

int rt_last_step_count(rt_ctx* c, unsigned long long* steps)
{
    if (!c || !steps) return RT_EINVAL;
    *steps = c->last_steps;
    return RT_OK;
}

int rt_set_direction_groups(rt_ctx* c, int groups)
{
    if (!c) return RT_EINVAL;
    if (groups < 0 || groups > kSlots) return fail(c, RT_EINVAL, "groups must be in [0, %d]", kSlots);
    c->groups_req = groups;
    return RT_OK;
}

int rt_set_block_threads(rt_ctx* c, int threads)
{
    int rc = enter(c);
    if (rc) return rc;
    if (threads != 0 && threads != 64 && threads != 128 && threads != 256)
        return fail(c, RT_EINVAL, "threads per block must be 0 (default), 64, 128 or 256");
    c->threads32 = threads;
    return RT_OK;
}

int rt_set_block_order(rt_ctx* c, int order)
{
    int rc = enter(c);
    if (rc) return rc;
    if (order < 0 || order > 2)
        return fail(c, RT_EINVAL, "block order must be 0 (automatic), 1 (tile-major) or 2 (plane-major)");
    c->order32 = order;
    return RT_OK;
}

int rt_set_cutoff(rt_ctx* c, double cut)
{
    if (!c) return RT_EINVAL;
    if (!(cut >= 0) || !(cut < 1)) return fail(c, RT_EINVAL, "cutoff must lie in [0, 1)");
    c->cut = cut;
    c->rec_valid = false;
    return RT_OK;
}

int rt_set_fs_record(rt_ctx* c, long long max_bytes)
{
    int rc = enter(c);
    if (rc) return rc;
    if (max_bytes < -1) return fail(c, RT_EINVAL, "max_bytes must be -1 (automatic), 0 (off) or a byte limit");
    CK(cudaStreamSynchronize(c->stream));
    c->rec_mode = max_bytes;
    if (max_bytes >= 0 && c->rec_cap > max_bytes) free_rec(c);
    c->rec_valid = false;
    return RT_OK;
}

int rt_fs_record_info(rt_ctx* c, long long* bytes, int* valid)
{
    if (!c || !bytes || !valid) return RT_EINVAL;
    *bytes = c->rec_cap;
    *valid = c->rec_valid ? 1 : 0;
    return RT_OK;
}

int rt_segment_weights(int precision, long long n, const double* x, double* w_cur, double* w_up,
                       double* e, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !w_cur || !w_up || !e))) return RT_EINVAL;
    if (precision != RT_FP64 && precision != RT_FP32_SWEEP) return RT_EINVAL;
    if (n == 0) return RT_OK;
    if (launch_seg_eval(n, precision == RT_FP32_SWEEP, x, w_cur, w_up, e, (cudaStream_t)stream) !=
        cudaSuccess)
        return RT_ECUDA;
    return RT_OK;
}

int rt_set_ng(rt_ctx* c, int period, double min_delta)
{
    if (!c) return RT_EINVAL;
    if (period != 0 && period < 4) return fail(c, RT_EINVAL, "Ng period must be 0 (off) or >= 4");
    if (!(min_delta >= 0)) return fail(c, RT_EINVAL, "Ng min_delta must be >= 0");
    c->ng_period = period;
    c->ng_min_delta = min_delta;
    c->ng_count = 1;
    return RT_OK;
}

int rt_set_fs_method(rt_ctx* c, int method)
{
    if (!c) return RT_EINVAL;
    if (method != RT_FS_LONG && method != RT_FS_SHORT)
        return fail(c, RT_EINVAL, "unknown formal-solution method");
    if (method == RT_FS_SHORT && c->precision != RT_FP64 && c->precision != RT_DF64)
        return fail(c, RT_EINVAL, "short characteristics need precision RT_FP64 or RT_DF64");
    if (method == RT_FS_SHORT && c->src_order != RT_SRC_LINEAR)
        return fail(c, RT_EINVAL, "short characteristics take the linear source only");
    if (method != c->fs_method) {
        c->fs_method = method;
        c->lstar_valid = c->coef_valid = c->rec_valid = false;   // Lambda* differs between methods
    }
    return RT_OK;
}

int rt_set_precision(rt_ctx* c, int precision)
{
    int rc = enter(c);
    if (rc) return rc;
    return switch_precision(c, precision);
}


int rt_set_graphs(rt_ctx* c, int on)
{
    if (!c) return RT_EINVAL;
    c->use_graphs = on != 0;
    return RT_OK;
}

int rt_set_df_finish(rt_ctx* c, double delta_switch)
{
    if (!c) return RT_EINVAL;
    if (!(delta_switch >= 0)) return fail(c, RT_EINVAL, "delta_switch must be >= 0");
    c->df_switch = delta_switch;
    return RT_OK;
}

int rt_batch_set_df_finish(rt_batch* b, double delta_switch)
{
    if (!b) return RT_EINVAL;
    if (!(delta_switch >= 0)) return bfail(b, RT_EINVAL, "delta_switch must be >= 0");
    for (rt_ctx* c : b->ctx) c->df_switch = delta_switch;
    return RT_OK;
}

int rt_set_source_order(rt_ctx* c, int order)
{
    if (!c) return RT_EINVAL;
    if (order != RT_SRC_LINEAR && order != RT_SRC_PARABOLIC)
        return fail(c, RT_EINVAL, "unknown source order");
    if (order == RT_SRC_PARABOLIC && (c->precision != RT_FP64 || c->fs_method != RT_FS_LONG))
        return fail(c, RT_EINVAL, "the parabolic source needs RT_FP64 and long characteristics");
    if (order != c->src_order) {
        c->src_order = order;
        c->lstar_valid = c->coef_valid = c->rec_valid = false;
    }
    return RT_OK;
}

int rt_set_os_method(rt_ctx* c, int method)
{
    if (!c) return RT_EINVAL;
    if (method != RT_OS_JACOBI && method != RT_OS_GAUSS_SEIDEL)
        return fail(c, RT_EINVAL, "unknown operator-splitting method");
    if (method != c->os_method) {
        c->os_method = method;
        c->coef_valid = false;   // the storage of c, 1/diag, r differs
    }
    return RT_OK;
}

int rt_batch_set_os_method(rt_batch* b, int method)
{
    if (!b) return RT_EINVAL;
    if (method != RT_OS_JACOBI && method != RT_OS_GAUSS_SEIDEL)
        return bfail(b, RT_EINVAL, "unknown operator-splitting method");
    for (rt_ctx* c : b->ctx) rt_set_os_method(c, method);
    return RT_OK;
}

int rt_batch_set_ng(rt_batch* b, int period, double min_delta)
{
    if (!b) return RT_EINVAL;
    if (period != 0 && period < 4) return bfail(b, RT_EINVAL, "Ng period must be 0 (off) or >= 4");
    if (!(min_delta >= 0)) return bfail(b, RT_EINVAL, "Ng min_delta must be >= 0");
    for (rt_ctx* c : b->ctx) rt_set_ng(c, period, min_delta);
    return RT_OK;
}

int rt_set_profiling(rt_ctx* c, int on)
{
    if (!c) return RT_EINVAL;
    c->profiling = on != 0;
    return RT_OK;
}

int rt_get_stats(rt_ctx* c, rt_stats* out)
{
    if (!c || !out) return RT_EINVAL;
    *out = c->stats;
    return RT_OK;
}

int rt_reset_stats(rt_ctx* c)
{
    if (!c) return RT_EINVAL;
    c->stats = rt_stats{};
    return RT_OK;
}

// ---- batched wavelengths (C ABI) --------------------------------------------

int rt_batch_create(rt_batch** out, int device, int precision, int nprob, const rt_problem* probs,
                    int top_mode, int bottom_mode, int ndir, const double* mu, const double* phi,
                    const double* w)
{
    if (!out) return RT_EINVAL;
    *out = nullptr;
    if (nprob < 1 || !probs ||
        (precision != RT_FP64 && precision != RT_FP32_SWEEP && precision != RT_DF64))
        return RT_EINVAL;
    rt_batch* b = new rt_batch();
    b->device = device;
    b->precision = precision;
    *out = b;  // also on failure, for rt_batch_last_error; the caller destroys it
    int rc = RT_OK;
    auto bail = [&](int code) { return code; };
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return bail(bfail(b, RT_ECUDA, "device %d unavailable", device));
    b->stream = b->own_stream;
    for (int e = 0; e < 4; ++e) BCK(cudaEventCreate(&b->ev[e]));
    b->ctx.assign(nprob, nullptr);
    for (int p = 0; p < nprob; ++p) {
        const rt_problem& q = probs[p];
        rt_ctx* c = nullptr;
        if ((rc = rt_create(&c, device, precision))) return bail(bfail(b, rc, "problem %d: context", p));
        b->ctx[p] = c;
        if ((rc = rt_set_stream(c, b->stream)) || (rc = rt_set_grid(c, q.nx, q.ny, q.nz, q.dx, q.dy, q.dz)) ||
            (rc = rt_set_boundary(c, top_mode, bottom_mode)) ||
            (rc = rt_set_quadrature(c, ndir, mu, phi, w)) || (rc = rt_set_opacity(c, q.chi)) ||
            (rc = rt_set_epsilon(c, q.eps)) || (rc = rt_set_planck(c, q.B)) ||
            (rc = ensure_partial(c)))
            return bail(bpass(b, p, rc));
    }
    b->order.resize(nprob);
    for (int p = 0; p < nprob; ++p) b->order[p] = p;
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](int x, int y) { return b->ctx[x]->g.N > b->ctx[y]->g.N; });
    b->iters.assign(nprob, 0);
    b->delta.assign(nprob, 0.0);
    b->converged.assign(nprob, 0);
    b->admitted.assign(nprob, 0);
    BCK(cudaMallocHost((void**)&b->h_views, sizeof(View32) * nprob));
    for (int p = 0; p < nprob; ++p) b->h_views[p] = view32(b->ctx[p]);
    b->view_fin.assign(nprob, 0);
    BCK(cudaMalloc((void**)&b->d_views, sizeof(View32) * nprob));
    BCK(cudaMemcpy(b->d_views, b->h_views, sizeof(View32) * nprob, cudaMemcpyHostToDevice));
    BCK(cudaMalloc((void**)&b->d_ids, sizeof(int) * nprob));
    BCK(cudaMalloc((void**)&b->d_prefix, sizeof(long long) * (nprob + 1)));
    BCK(cudaMalloc((void**)&b->d_delta, sizeof(double) * nprob));
    BCK(cudaMalloc((void**)&b->d_steps, sizeof(unsigned long long)));
    BCK(cudaMallocHost((void**)&b->h_ids, sizeof(int) * nprob));
    BCK(cudaMalloc((void**)&b->d_rviews, sizeof(Rep32) * nprob));
    BCK(cudaMallocHost((void**)&b->h_rviews, sizeof(Rep32) * nprob));
    memset(b->h_rviews, 0, sizeof(Rep32) * nprob);
    BCK(cudaMalloc((void**)&b->d_rids, sizeof(int) * nprob));
    BCK(cudaMalloc((void**)&b->d_rprefix, sizeof(long long) * (nprob + 1)));
    BCK(cudaMallocHost((void**)&b->h_rids, sizeof(int) * nprob));
    BCK(cudaMallocHost((void**)&b->h_rprefix, sizeof(long long) * (nprob + 1)));
    BCK(cudaMallocHost((void**)&b->h_prefix, sizeof(long long) * (nprob + 1)));
    BCK(cudaMallocHost((void**)&b->h_delta, sizeof(double) * nprob));
    BCK(cudaMallocHost((void**)&b->h_steps, sizeof(unsigned long long)));
    BCK(cudaMalloc((void**)&b->d_sweeps, sizeof(int) * nprob));
    BCK(cudaMemset(b->d_sweeps, 0, sizeof(int) * nprob));
    BCK(cudaMallocHost((void**)&b->h_sweeps, sizeof(int) * nprob));
    *out = b;
    return RT_OK;
}

int rt_batch_destroy(rt_batch* b)
{
    if (!b) return RT_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    free_batch_graphs(b);
    batch_free_pool(b);
    for (rt_ctx* c : b->ctx) rt_destroy(c);
    if (b->d_sweeps) cudaFree(b->d_sweeps);
    if (b->h_sweeps) cudaFreeHost(b->h_sweeps);
    if (b->d_views) cudaFree(b->d_views);
    if (b->h_views) cudaFreeHost(b->h_views);
    if (b->d_rviews) cudaFree(b->d_rviews);
    if (b->h_rviews) cudaFreeHost(b->h_rviews);
    if (b->d_rids) cudaFree(b->d_rids);
    if (b->d_rprefix) cudaFree(b->d_rprefix);
    if (b->h_rids) cudaFreeHost(b->h_rids);
    if (b->h_rprefix) cudaFreeHost(b->h_rprefix);
    if (b->d_ids) cudaFree(b->d_ids);
    if (b->d_prefix) cudaFree(b->d_prefix);
    if (b->d_delta) cudaFree(b->d_delta);
    if (b->d_steps) cudaFree(b->d_steps);
    if (b->h_ids) cudaFreeHost(b->h_ids);
    if (b->h_prefix) cudaFreeHost(b->h_prefix);
    if (b->h_delta) cudaFreeHost(b->h_delta);
    if (b->h_steps) cudaFreeHost(b->h_steps);
    for (auto& e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    delete b;
    return RT_OK;
}

const char* rt_batch_last_error(const rt_batch* b) { return b ? b->err.c_str() : "null batch"; }

int rt_batch_set_stream(rt_batch* b, void* stream)
{
    if (!b) return RT_EINVAL;
    b->err.clear();
    BCK(cudaSetDevice(b->device));
    BCK(cudaStreamSynchronize(b->stream));
    b->stream = stream ? (cudaStream_t)stream : b->own_stream;
    free_batch_graphs(b);
    for (size_t p = 0; p < b->ctx.size(); ++p) {
        int rc = rt_set_stream(b->ctx[p], b->stream);
        if (rc) return bpass(b, (int)p, rc);
    }
    return RT_OK;
}

int rt_batch_reset(rt_batch* b, int rebuild_lstar)
{
    if (!b) return RT_EINVAL;
    b->err.clear();
    BCK(cudaSetDevice(b->device));
    for (size_t p = 0; p < b->ctx.size(); ++p) {
        rt_ctx* c = b->ctx[p];
        BCK(cudaMemcpyAsync(c->J, c->B, sizeof(double) * c->g.N, cudaMemcpyDeviceToDevice,
                            b->stream));
        c->ng_count = 1;
        c->ng_last_delta = 0.0;
        if (rebuild_lstar) c->lstar_valid = c->coef_valid = false;
        b->iters[p] = 0;
        b->delta[p] = 0.0;
        b->converged[p] = 0;
        b->admitted[p] = c->rec_cap > 0;   // a held recording keeps its place
    }
    return RT_OK;
}

int rt_batch_set_fs_record(rt_batch* b, long long max_bytes)
{
    if (!b) return RT_EINVAL;
    b->err.clear();
    if (max_bytes < -1) return bfail(b, RT_EINVAL, "max_bytes must be -1 (automatic), 0 (off) or a byte limit");
    BCK(cudaSetDevice(b->device));
    for (size_t p = 0; p < b->ctx.size(); ++p) batch_release(b, (int)p);
    batch_free_pool(b);
    std::fill(b->admitted.begin(), b->admitted.end(), 0);
    b->rec_mode = max_bytes;
    return RT_OK;
}

int rt_batch_set_precision(rt_batch* b, int precision)
{
    if (!b) return RT_EINVAL;
    b->err.clear();
    BCK(cudaSetDevice(b->device));
    if (precision == b->precision) return RT_OK;
    if (!((precision == RT_FP32_SWEEP || precision == RT_DF64) &&
          (b->precision == RT_FP32_SWEEP || b->precision == RT_DF64)))
        return bfail(b, RT_EINVAL, "precision switches only between RT_FP32_SWEEP and RT_DF64");
    for (size_t p = 0; p < b->ctx.size(); ++p) {
        const int rc = rt_set_precision(b->ctx[p], precision);
        if (rc) return bfail(b, rc, "problem %zu: %s", p, rt_last_error(b->ctx[p]));
        b->iters[p] = 0;        // a new stage: counts, deltas and convergence restart
        b->delta[p] = 0.0;
        b->converged[p] = 0;
        batch_release(b, (int)p);
        b->admitted[p] = 0;
    }
    batch_free_pool(b);
    b->precision = precision;
    return RT_OK;
}

static int batch_solve(rt_batch* b, double tol, int max_iter, double tol_inner, int max_sweeps,
                       int* iters, double* deltas, int* n_converged);

int rt_batch_solve(rt_batch* b, double tol, int max_iter, double tol_inner, int max_sweeps,
                   int* iters, double* deltas, int* n_converged)
{
    int rc = batch_solve(b, tol, max_iter, tol_inner, max_sweeps, iters, deltas, n_converged);
    if (!b) return rc;
    for (size_t p = 0; p < b->ctx.size(); ++p) {
        const int r2 = check_bounds(b->ctx[p], RT_OK);
        if (r2) return bfail(b, r2, "problem %zu: %s", p, rt_last_error(b->ctx[p]));
    }
    return rc;
}

int rt_checked_build(void)
{
#ifdef RT_CHECKED
    return 1;
#else
    return 0;
#endif
}

int rt_bounds_selftest(rt_ctx* c)
{
    int rc = enter(c);
    if (rc) return rc;
    CK(launch_bounds_selftest(c->g, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return check_bounds(c, RT_OK);
}

int rt_get_plane_order(rt_ctx* c, int* order)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((rc = need(c, c->have_chi, "the opacity"))) return rc;
    if (!order) return fail(c, RT_EINVAL, "order is NULL");
    CK(cudaMemcpyAsync(order, c->zorder, sizeof(int) * c->g.nz, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return RT_OK;
}

static int batch_solve(rt_batch* b, double tol, int max_iter, double tol_inner, int max_sweeps,
                       int* iters, double* deltas, int* n_converged)
{
    if (!b) return RT_EINVAL;
    b->err.clear();
    BCK(cudaSetDevice(b->device));
    if (max_iter < 1 || max_sweeps < 1 || !(tol >= 0) || !(tol_inner >= 0))
        return bfail(b, RT_EINVAL, "bad iteration controls");
    const int P = (int)b->ctx.size();
    int rc;
    // problems in their finishing stage leave it (and get their Ng threshold
    // back) when the solve ends, whichever way it ends
    struct FinishGuard {
        rt_batch* b;
        std::vector<char> switched;
        std::vector<double> ng_min0;
        ~FinishGuard()
        {
            for (size_t p = 0; p < switched.size(); ++p)
                if (switched[p]) {
                    b->ctx[p]->fin = 0;
                    b->ctx[p]->ng_min_delta = ng_min0[p];
                }
        }
    } guard{b, std::vector<char>(P, 0), std::vector<double>(P, 0.0)};
    std::vector<char>& switched = guard.switched;
    std::vector<double>& ng_min0 = guard.ng_min0;
    // (problems admitted in waves: the loop runs until none is left)
    for (long long it = 0; it < (long long)max_iter * P + 1; ++it) {
        if ((rc = batch_admit(b, max_iter))) return rc;
        std::vector<int> act;
        for (int p : b->order)
            if (b->admitted[p] && !b->converged[p] && b->iters[p] < max_iter) act.push_back(p);
        if (act.empty()) break;
        if ((rc = batch_fs(b, act))) return rc;
        if (b->use_graphs)
            rc = batch_os_graph(b, act, tol_inner, max_sweeps);
        else
            rc = batch_os(b, act, tol_inner, max_sweeps);
        if (rc) return rc;
        for (int p : act)
            if ((rc = bpass(b, p, ng_push(b->ctx[p], b->iters[p] + 1)))) return rc;
        BCK(cudaMemsetAsync(b->d_delta, 0, sizeof(double) * P, b->stream));
        for (int p : act) {
            rt_ctx* c = b->ctx[p];
            BCK(launch_rel_change(c->g.N, c->Jn, c->J, b->d_delta + p, b->stream));
            b->stats.launches += 1;
        }
        BCK(cudaMemcpyAsync(b->h_delta, b->d_delta, sizeof(double) * P, cudaMemcpyDeviceToHost,
                            b->stream));
        if (b->use_graphs)
            BCK(cudaMemcpyAsync(b->h_sweeps, b->d_sweeps, sizeof(int) * P, cudaMemcpyDeviceToHost,
                                b->stream));
        BCK(cudaStreamSynchronize(b->stream));
        b->stats.host_syncs += 1;
        b->stats.iterations += 1;
        if (b->use_graphs) batch_os_graph_counts(b, act);
        bharvest(b);
        b->stats.steps += *b->h_steps;
        for (int p : act) {
            rt_ctx* c = b->ctx[p];
            std::swap(c->J, c->Jn);
            b->iters[p] += 1;
            b->delta[p] = b->h_delta[p];
            c->ng_last_delta = b->h_delta[p];
            if (tol > 0 && b->h_delta[p] < tol) {
                b->converged[p] = 1;
            } else if (c->df_switch > 0 && c->precision == RT_FP32_SWEEP &&
                       b->precision == RT_FP32_SWEEP && c->fin == 0 &&
                       b->h_delta[p] < c->df_switch) {
                // finishing stage for this problem (see solve())
                c->fin = 1;
                switched[p] = 1;
                ng_min0[p] = c->ng_min_delta;
                c->ng_min_delta = 0.0;
                c->ng_count = 1;
            }
            if (b->converged[p] || b->iters[p] >= max_iter) batch_release(b, p);
        }
    }
    batch_free_pool(b);
    int nconv = 0;
    for (int p = 0; p < P; ++p) {
        if (iters) iters[p] = b->iters[p];
        if (deltas) deltas[p] = b->delta[p];
        nconv += b->converged[p];
    }
    if (n_converged) *n_converged = nconv;
    if (tol > 0 && nconv < P)
        return bfail(b, RT_ENOTCONV, "%d of %d problems not converged", P - nconv, P);
    return RT_OK;
}

int rt_batch_get_J(rt_batch* b, int p, double* J)
{
    if (!b || !J || p < 0 || p >= (int)b->ctx.size()) return RT_EINVAL;
    b->err.clear();
    BCK(cudaSetDevice(b->device));
    BCK(cudaStreamSynchronize(b->stream));
    int rc = rt_get_J(b->ctx[p], J);
    return bpass(b, p, rc);
}

int rt_batch_get_J_dev(rt_batch* b, int p, double* J)
{
    if (!b || !J || p < 0 || p >= (int)b->ctx.size()) return RT_EINVAL;
    b->err.clear();
    BCK(cudaSetDevice(b->device));
    rt_ctx* c = b->ctx[p];
    BCK(cudaMemcpyAsync(J, c->J, sizeof(double) * c->g.N, cudaMemcpyDeviceToDevice, b->stream));
    return RT_OK;
}

int rt_batch_set_block_threads(rt_batch* b, int threads)
{
    if (!b) return RT_EINVAL;
    if (threads != 0 && threads != 64 && threads != 128 && threads != 256)
        return bfail(b, RT_EINVAL, "threads per block must be 0 (default), 64, 128 or 256");
    b->threads32 = threads;
    return RT_OK;
}

int rt_batch_set_block_order(rt_batch* b, int order)
{
    if (!b) return RT_EINVAL;
    b->err.clear();
    if (order < 0 || order > 2)
        return bfail(b, RT_EINVAL, "block order must be 0 (automatic), 1 (tile-major) or 2 (plane-major)");
    for (rt_ctx* c : b->ctx) c->order32 = order;
    const int n = (int)b->ctx.size();
    for (int p = 0; p < n; ++p)
        b->h_views[p] = b->view_fin[p] ? view32_fin(b->ctx[p]) : view32(b->ctx[p]);
    BCK(cudaMemcpyAsync(b->d_views, b->h_views, sizeof(View32) * n, cudaMemcpyHostToDevice,
                        b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return RT_OK;
}

int rt_batch_set_graphs(rt_batch* b, int on)
{
    if (!b) return RT_EINVAL;
    b->err.clear();
    BCK(cudaSetDevice(b->device));
    BCK(cudaStreamSynchronize(b->stream));
    free_batch_graphs(b);
    b->use_graphs = on != 0;
    return RT_OK;
}

int rt_batch_set_direction_groups(rt_batch* b, int groups)
{
    if (!b) return RT_EINVAL;
    if (groups < 0 || groups > kSlots) return bfail(b, RT_EINVAL, "groups must be in [0, %d]", kSlots);
    b->groups_req = groups;
    return RT_OK;
}

int rt_batch_set_profiling(rt_batch* b, int on)
{
    if (!b) return RT_EINVAL;
    b->profiling = on != 0;
    return RT_OK;
}

int rt_batch_get_stats(rt_batch* b, rt_stats* out)
{
    if (!b || !out) return RT_EINVAL;
    rt_stats s = b->stats;
    for (rt_ctx* c : b->ctx) {   // per-problem kernels (source, sums, Lambda*, OS set-up)
        s.launches += c->stats.launches;
        s.lstar_launches += c->stats.lstar_launches;
    }
    *out = s;
    return RT_OK;
}

int rt_batch_reset_stats(rt_batch* b)
{
    if (!b) return RT_EINVAL;
    b->stats = rt_stats{};
    for (rt_ctx* c : b->ctx) c->stats = rt_stats{};
    return RT_OK;
}

}  // extern "C"
