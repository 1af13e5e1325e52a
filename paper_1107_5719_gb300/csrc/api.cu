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
    bool lstar_valid = false, coef_valid = false, chi32_valid = false;
    int groups_req = 0;
    double cut = -1.0;

    // device state, FP64
    double *chi = nullptr, *eps = nullptr, *B = nullptr, *J = nullptr, *S = nullptr;
    double *Jfs = nullptr, *Jn = nullptr, *Ja = nullptr, *Jb = nullptr, *r = nullptr;
    double *lstar = nullptr, *coef = nullptr, *rdiag = nullptr, *partial = nullptr;
    int partial_groups = 0;
    // FP32 copies for the sweep form
    float *chi32 = nullptr, *S32 = nullptr, *B32 = nullptr;
    // direction tables
    DirInfo* info = nullptr;
    StepGeo* off = nullptr;
    Bw4d* bw = nullptr;
    float4* bw32 = nullptr;
    double *d_mu = nullptr, *d_phi = nullptr, *d_w = nullptr;
    // scalars: [0] smax, [1] inner delta, [2] outer delta
    double* scal = nullptr;
    unsigned long long* d_steps = nullptr;
    double* h_scal = nullptr;               // pinned
    unsigned long long* h_steps = nullptr;  // pinned
    unsigned long long last_steps = 0;

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

void free_grid_buffers(rt_ctx* c)
{
    dfree(c->chi); dfree(c->eps); dfree(c->B); dfree(c->J); dfree(c->S);
    dfree(c->Jfs); dfree(c->Jn); dfree(c->Ja); dfree(c->Jb); dfree(c->r);
    dfree(c->lstar); dfree(c->coef); dfree(c->rdiag); dfree(c->partial);
    dfree(c->chi32); dfree(c->S32); dfree(c->B32);
    c->partial_groups = 0;
}

void free_tables(rt_ctx* c)
{
    dfree(c->info); dfree(c->off); dfree(c->bw); dfree(c->bw32);
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

double default_cut(int precision)
{
    return precision == RT_FP64 ? 1e-17 : 1e-9;
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

int ensure_partial(rt_ctx* c)
{
    if (c->partial_groups >= kSlots) return RT_OK;
    CK(dalloc(c->partial, (size_t)kSlots * c->g.N));
    c->partial_groups = kSlots;
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

// Formal solution: source in c->S (already set), result J into Jout (device).
int run_fs(rt_ctx* c, double* Jout, bool count_steps)
{
    const bool bnd = c->g.top_bc || c->g.bottom_bc;
    const int G = auto_groups(c);
    int rc = ensure_partial(c);
    if (rc) return rc;
    if (count_steps) CK(cudaMemsetAsync(c->d_steps, 0, sizeof(unsigned long long), c->stream));
    const double cut = c->cut >= 0 ? c->cut : default_cut(c->precision);
    if (c->profiling) CK(cudaEventRecord(c->ev[0], c->stream));
    if (c->precision == RT_FP64) {
        CK(launch_fs64(c->g, c->chi, c->S, c->B, c->info, c->off, c->bw, c->scal + 0, cut, G,
                       c->partial, count_steps ? c->d_steps : nullptr, c->stream));
    } else {
        if (!c->chi32_valid) {
            CK(launch_to_float(c->g.N, c->chi, c->chi32, c->stream));
            CK(launch_to_float(c->g.N, c->B, c->B32, c->stream));
            c->chi32_valid = true;
            c->stats.launches += 2;
        }
        CK(launch_fs32(c->g, c->chi32, c->S32, c->B32, c->info, c->off, c->bw32, c->scal + 0, cut,
                       G, c->partial, count_steps ? c->d_steps : nullptr, c->stream));
    }
    if (c->profiling) {
        CK(cudaEventRecord(c->ev[1], c->stream));
        c->fs_pending = true;
    }
    c->stats.fs_launches += 1;
    c->stats.launches += 2;
    (void)bnd;
    CK(launch_sum_groups(c->g.N, c->partial, Jout, c->stream));
    if (!c->lstar_valid) {
        CK(launch_lstar64(c->g, c->chi, c->info, c->off, c->bw, c->lstar, c->stream));
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

// S = eps B + (1 - eps) J (or the caller's S), then smax; FP32 copy if needed.
int prepare_source(rt_ctx* c, const double* S_in, bool device)
{
    const bool bnd = c->g.top_bc || c->g.bottom_bc;
    float* s32 = c->precision == RT_FP64 ? nullptr : c->S32;
    CK(cudaMemsetAsync(c->scal + 0, 0, sizeof(double), c->stream));
    if (S_in) {
        CK(cudaMemcpyAsync(c->S, S_in, sizeof(double) * c->g.N, kind(device), c->stream));
        CK(launch_absmax(c->g.N, c->S, bnd ? c->B : nullptr, c->scal + 0, s32, c->stream));
    } else {
        CK(launch_source(c->g.N, c->eps, c->B, c->J, c->S, s32, bnd ? c->B : nullptr, c->scal + 0,
                         c->stream));
    }
    c->stats.launches += 1;
    return RT_OK;
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
    CK(launch_os_coef(c->g, c->lstar, c->eps, c->coef, c->rdiag, c->stream));
    c->coef_valid = true;
    c->stats.launches += 1;
    return RT_OK;
}

// Jacobi solve from J_old (device) into J_new (device); J_fs device.
int run_os(rt_ctx* c, const double* Jfs, const double* Jold, double* Jnew, double tol_inner,
           int max_sweeps, int* sweeps_out)
{
    int rc = ensure_coef(c);
    if (rc) return rc;
    CK(launch_os_rhs(c->g, c->coef, c->rdiag, Jfs, Jold, c->r, c->stream));
    c->stats.launches += 1;
    const double* cur = Jold;
    double* bufs[2] = {c->Ja, c->Jb};
    int n = 0;
    for (; n < max_sweeps;) {
        double* nxt = bufs[n & 1];
        CK(cudaMemsetAsync(c->scal + 1, 0, sizeof(double), c->stream));
        if (c->profiling) CK(cudaEventRecord(c->ev[2], c->stream));
        CK(launch_jacobi(c->g, c->coef, c->r, cur, nxt, c->scal + 1, c->stream));
        if (c->profiling) {
            CK(cudaEventRecord(c->ev[3], c->stream));
            c->jac_pending = true;
        }
        c->stats.launches += 1;
        c->stats.jacobi_launches += 1;
        CK(cudaMemcpyAsync(c->h_scal + 1, c->scal + 1, sizeof(double), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
        harvest(c);
        cur = nxt;
        ++n;
        if (*(c->h_scal + 1) < tol_inner) break;
    }
    CK(cudaMemcpyAsync(Jnew, cur, sizeof(double) * c->g.N, cudaMemcpyDeviceToDevice, c->stream));
    if (sweeps_out) *sweeps_out = n;
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
    if ((rc = run_os(c, dfs, dold, dnew, tol_inner, max_sweeps, sweeps))) return rc;
    if (!device)
        CK(cudaMemcpyAsync(Jnew, dnew, sizeof(double) * c->g.N, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
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
    int it = 0;
    double delta = 0.0;
    bool converged = false;
    unsigned long long total_steps = 0;
    while (it < max_iter) {
        if ((rc = prepare_source(c, nullptr, true))) return rc;
        if ((rc = run_fs(c, c->Jfs, true))) return rc;
        int ns = 0;
        if ((rc = run_os(c, c->Jfs, c->J, c->Jn, tol_inner, max_sweeps, &ns))) return rc;
        CK(cudaMemsetAsync(c->scal + 2, 0, sizeof(double), c->stream));
        CK(launch_rel_change(c->g.N, c->Jn, c->J, c->scal + 2, c->stream));
        c->stats.launches += 1;
        CK(cudaMemcpyAsync(c->h_scal + 2, c->scal + 2, sizeof(double), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
        harvest(c);
        total_steps += *c->h_steps;
        delta = c->h_scal[2];
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

}  // namespace

extern "C" {

const char* rt_version(void) { return "rt3d 0.1 (sm_103a)"; }

int rt_create(rt_ctx** out, int device, int precision)
{
    if (!out) return RT_EINVAL;
    *out = nullptr;
    if (precision != RT_FP64 && precision != RT_FP32_SWEEP) return RT_EINVAL;
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
    c->g.top_bc = RT_BC_ZERO;
    c->g.bottom_bc = RT_BC_PLANCK;
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
    if (c->h_scal) cudaFreeHost(c->h_scal);
    if (c->h_steps) cudaFreeHost(c->h_steps);
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
    if (nx < 3 || ny < 3 || nz < 2)
        return fail(c, RT_EINVAL, "grid %dx%dx%d: need nx, ny >= 3 and nz >= 2", nx, ny, nz);
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !std::isfinite(dx) || !std::isfinite(dy) ||
        !std::isfinite(dz))
        return fail(c, RT_EINVAL, "spacings must be finite and > 0");
    if ((long long)nx * ny > (1LL << 30) || (long long)nx * ny * nz > (1LL << 40))
        return fail(c, RT_EINVAL, "grid too large");
    CK(cudaStreamSynchronize(c->stream));
    free_grid_buffers(c);
    free_tables(c);
    c->have_grid = c->have_quad = c->have_chi = c->have_eps = c->have_B = false;
    c->lstar_valid = c->coef_valid = c->chi32_valid = false;
    c->g.nx = nx; c->g.ny = ny; c->g.nz = nz;
    c->g.N = (long long)nx * ny * nz;
    c->g.ndir = 0;
    c->dx = dx; c->dy = dy; c->dz = dz;
    const size_t N = (size_t)c->g.N;
    CK(dalloc(c->chi, N)); CK(dalloc(c->eps, N)); CK(dalloc(c->B, N)); CK(dalloc(c->J, N));
    CK(dalloc(c->S, N)); CK(dalloc(c->Jfs, N)); CK(dalloc(c->Jn, N)); CK(dalloc(c->Ja, N));
    CK(dalloc(c->Jb, N)); CK(dalloc(c->r, N)); CK(dalloc(c->rdiag, N));
    CK(dalloc(c->lstar, 27 * N)); CK(dalloc(c->coef, 27 * N));
    if (c->precision != RT_FP64) {
        CK(dalloc(c->chi32, N)); CK(dalloc(c->S32, N)); CK(dalloc(c->B32, N));
    }
    c->have_grid = true;
    return RT_OK;
}

int rt_set_boundary(rt_ctx* c, int top_mode, int bottom_mode)
{
    int rc = enter(c);
    if (rc) return rc;
    if ((top_mode != RT_BC_ZERO && top_mode != RT_BC_PLANCK) ||
        (bottom_mode != RT_BC_ZERO && bottom_mode != RT_BC_PLANCK))
        return fail(c, RT_EINVAL, "boundary modes must be RT_BC_ZERO or RT_BC_PLANCK");
    c->g.top_bc = top_mode;
    c->g.bottom_bc = bottom_mode;
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
    CK(dalloc(c->info, ndir)); CK(dalloc(c->off, T)); CK(dalloc(c->bw, T)); CK(dalloc(c->bw32, T));
    CK(cudaMemcpyAsync(c->d_mu, mu, sizeof(double) * ndir, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_phi, phi, sizeof(double) * ndir, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_w, w, sizeof(double) * ndir, cudaMemcpyHostToDevice, c->stream));
    CK(launch_dir_tables(c->g, c->dx, c->dy, c->dz, c->d_mu, c->d_phi, c->d_w, c->info, c->off,
                         c->bw, c->bw32, c->stream));
    c->stats.launches += 1;
    CK(cudaStreamSynchronize(c->stream));
    c->have_quad = true;
    c->lstar_valid = c->coef_valid = false;
    return RT_OK;
}

static int set_chi(rt_ctx* c, const double* chi, bool device)
{
    int rc = set_field(c, chi, c ? c->chi : nullptr, device, "chi", true, false);
    if (rc) return rc;
    c->have_chi = true;
    c->lstar_valid = c->coef_valid = c->chi32_valid = false;
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
    c->have_B = true;
    c->chi32_valid = false;
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
    return formal_solution(c, S, J_fs, lstar, false);
}

int rt_formal_solution_dev(rt_ctx* c, const double* S, double* J_fs, double* lstar)
{
    return formal_solution(c, S, J_fs, lstar, true);
}

int rt_os_step(rt_ctx* c, const double* J_fs, const double* J_old, double* J_new, double tol_inner,
               int max_sweeps, int* sweeps)
{
    return os_step(c, J_fs, J_old, J_new, tol_inner, max_sweeps, sweeps, false);
}

int rt_os_step_dev(rt_ctx* c, const double* J_fs, const double* J_old, double* J_new,
                   double tol_inner, int max_sweeps, int* sweeps)
{
    return os_step(c, J_fs, J_old, J_new, tol_inner, max_sweeps, sweeps, true);
}

int rt_solve(rt_ctx* c, double tol, int max_iter, double tol_inner, int max_sweeps, double* J_out,
             int* iters, double* last_delta, double* deltas, int* sweeps)
{
    return solve(c, tol, max_iter, tol_inner, max_sweeps, J_out, iters, last_delta, deltas, sweeps,
                 false);
}

int rt_solve_dev(rt_ctx* c, double tol, int max_iter, double tol_inner, int max_sweeps,
                 double* J_out, int* iters, double* last_delta, double* deltas, int* sweeps)
{
    return solve(c, tol, max_iter, tol_inner, max_sweeps, J_out, iters, last_delta, deltas, sweeps,
                 true);
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
    CK(cudaStreamSynchronize(c->stream));
    return RT_OK;
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

int rt_set_cutoff(rt_ctx* c, double cut)
{
    if (!c) return RT_EINVAL;
    if (!(cut >= 0) || !(cut < 1)) return fail(c, RT_EINVAL, "cutoff must lie in [0, 1)");
    c->cut = cut;
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

}  // extern "C"
