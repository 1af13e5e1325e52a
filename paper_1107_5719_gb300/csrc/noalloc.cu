// Allocation-free formal solution (declared in include/rt3d.h).
//
// For callers that may not allocate device memory while they run (their
// host application owns all device memory through its own pool, their
// memory budget is fixed up front, or they cannot afford the implicit
// synchronisation of cudaMalloc).  The work is the same as
// rt_formal_solution_dev's FP64 path; only the working memory differs: it
// is carved out of one file-scope device array of fixed size instead of
// context buffers.  The paper has no counterpart of this entry point.
#include "../../include/rt3d.h"
#include "internal.h"

#include <cmath>
#include <mutex>

using namespace rt3d;

namespace {

// The scratch every call of rt_formal_solution_noalloc works in.  Host code
// must not use this name as an address (on the host it names a stand-in
// object, not device memory): it passes the address cudaGetSymbolAddress
// returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[RT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current).
cudaError_t scratch_address(int dev, unsigned char** out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// The scratch size stated in include/rt3d.h (64*N + 88*ndir*nz + 88*ndir + 8
// bytes plus alignment) counts these record sizes.
static_assert(sizeof(DirInfo) == 64, "direction record size changed: update the stated scratch size");
static_assert(sizeof(StepGeo) + 2 * sizeof(Bw4d) + sizeof(float4) == 88,
              "per-(direction, plane) tables changed: update the stated scratch size");
static_assert(kSlots * sizeof(double) == 64, "partial sums per voxel changed: update the stated scratch size");

struct Layout {
    size_t smax, mu, phi, w, info, off, bw, bwh, bw32, partial, total;
};

Layout layout(long long N, int ndir, int nz)
{
    Layout L{};
    size_t o = 0;
    L.smax = o;    o = align256(o + sizeof(double));
    L.mu = o;      o = align256(o + sizeof(double) * ndir);
    L.phi = o;     o = align256(o + sizeof(double) * ndir);
    L.w = o;       o = align256(o + sizeof(double) * ndir);
    L.info = o;    o = align256(o + sizeof(DirInfo) * ndir);
    L.off = o;     o = align256(o + sizeof(StepGeo) * (size_t)ndir * nz);
    L.bw = o;      o = align256(o + sizeof(Bw4d) * (size_t)ndir * nz);
    L.bwh = o;     o = align256(o + sizeof(Bw4d) * (size_t)ndir * nz);
    L.bw32 = o;    o = align256(o + sizeof(float4) * (size_t)ndir * nz);
    L.partial = o; o = align256(o + sizeof(double) * (size_t)kSlots * (size_t)N);
    L.total = o;
    return L;
}

}  // namespace

extern "C" int rt_formal_solution_noalloc(int nx, int ny, int nz, double dx, double dy, double dz,
                                          int top_mode, int bottom_mode, int ndir,
                                          const double* mu, const double* phi, const double* w,
                                          const double* chi, const double* S, const double* B,
                                          double* J_fs, void* stream)
{
    // Host-side checks first: nothing below touches the GPU if they fail.
    if (nx < 3 || ny < 3 || nz < 2 || nz > 65535 || ndir < 1) return RT_EINVAL;
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !std::isfinite(dx) || !std::isfinite(dy) ||
        !std::isfinite(dz))
        return RT_EINVAL;
    if ((top_mode != RT_BC_ZERO && top_mode != RT_BC_PLANCK) ||
        (bottom_mode != RT_BC_ZERO && bottom_mode != RT_BC_PLANCK))
        return RT_EINVAL;
    const bool planck = top_mode == RT_BC_PLANCK || bottom_mode == RT_BC_PLANCK;
    if (!mu || !phi || !w || !chi || !S || !J_fs || (planck && !B)) return RT_EINVAL;
    double sw = 0.0;
    for (int d = 0; d < ndir; ++d) {
        if (!std::isfinite(mu[d]) || !std::isfinite(phi[d]) || !std::isfinite(w[d])) return RT_EINVAL;
        if (!(std::fabs(mu[d]) >= 1e-6) || !(std::fabs(mu[d]) <= 1.0) || !(w[d] >= 0)) return RT_EINVAL;
        sw += w[d];
    }
    if (std::fabs(sw - 1.0) > 1e-12) return RT_EINVAL;
    if ((long long)nx * ny > (1LL << 30)) return RT_ESCRATCH;
    const long long N = (long long)nx * ny * nz;
    const Layout L = layout(N, ndir, nz);
    if (L.total > (size_t)RT_NOALLOC_SCRATCH_BYTES) return RT_ESCRATCH;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RT_ECUDA;
    unsigned char* base = nullptr;
    if (scratch_address(dev, &base) != cudaSuccess) return RT_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RT_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;

    Geometry g{};
    g.nx = nx; g.ny = ny; g.nz = nz; g.ndir = ndir; g.N = N;
    g.top_bc = top_mode; g.bottom_bc = bottom_mode;
    double* smax = reinterpret_cast<double*>(base + L.smax);
    double* d_mu = reinterpret_cast<double*>(base + L.mu);
    double* d_phi = reinterpret_cast<double*>(base + L.phi);
    double* d_w = reinterpret_cast<double*>(base + L.w);
    DirInfo* info = reinterpret_cast<DirInfo*>(base + L.info);
    StepGeo* off = reinterpret_cast<StepGeo*>(base + L.off);
    Bw4d* bw = reinterpret_cast<Bw4d*>(base + L.bw);
    Bw4d* bwh = reinterpret_cast<Bw4d*>(base + L.bwh);
    float4* bw32 = reinterpret_cast<float4*>(base + L.bw32);
    double* partial = reinterpret_cast<double*>(base + L.partial);

    // As many z-blocks over the direction slots as keep every SM busy; J
    // does not depend on this choice.
    const long long blocks = (long long)((nx * ny + 127) / 128) * nz;
    int G = 1;
    while (G < kSlots && blocks * G < 64LL * sms) G *= 2;

    if (cudaMemcpyAsync(d_mu, mu, sizeof(double) * ndir, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(d_phi, phi, sizeof(double) * ndir, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(d_w, w, sizeof(double) * ndir, cudaMemcpyHostToDevice, st))
        return RT_ECUDA;
    if (launch_dir_tables(g, dx, dy, dz, d_mu, d_phi, d_w, info, off, bw, bwh, bw32, st)) return RT_ECUDA;
    // The cutoff bound is a max-reduction: it must start from zero on every call.
    if (cudaMemsetAsync(smax, 0, sizeof(double), st)) return RT_ECUDA;
    if (launch_absmax(N, S, planck ? B : nullptr, smax, nullptr, st)) return RT_ECUDA;
    if (launch_fs64(g, chi, S, B, nullptr, info, off, bw, bwh, smax, 1e-17, G, partial, nullptr, st))
        return RT_ECUDA;
    if (launch_sum_groups(N, partial, J_fs, st)) return RT_ECUDA;
    return RT_OK;
}
