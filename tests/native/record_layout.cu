// Host-side check of the recordings' index maps (internal.h): every
// coefficient index a recording kernel writes for a grid lies inside the
// block the context allocates for it and no two coincide.  Prints one line
// per grid: "nx ny nz ndir fp64_ok fp32_ok".
#include "../../paper_1107_5719_gb300/csrc/internal.h"

#include <cstdio>
#include <vector>

using namespace rt3d;

static bool check_fp64(Geometry g)
{
    const long long nxy = (long long)g.nx * g.ny;
    const long long size = (long long)g.ndir * nxy * ((long long)g.nz * (g.nz - 1) / 2);
    std::vector<char> seen((size_t)size, 0);
    for (int d = 0; d < g.ndir; ++d) {
        const int s = d % 2 ? 1 : -1;
        for (int k0 = 0; k0 < g.nz; ++k0) {
            const int M = s > 0 ? k0 : g.nz - 1 - k0;
            for (long long t = 0; t < nxy; ++t)
                for (int m = 1; m <= M; ++m) {
                    const long long i = rec_base(g, d, k0, s) + (long long)(m - 1) * nxy + t;
                    if (i < 0 || i >= size || seen[(size_t)i]) return false;
                    seen[(size_t)i] = 1;
                }
        }
    }
    return true;
}

static bool check_fp32(Geometry g)
{
    const long long npair = (long long)g.nx * ((g.ny + 1) / 2), nwp = (npair + 31) / 32;
    const long long size = (long long)g.ndir * rec32_steps4(g.nz) * nwp * 32;
    std::vector<char> seen((size_t)size, 0);
    for (int d = 0; d < g.ndir; ++d) {
        const int s = d % 2 ? 1 : -1;
        for (int k0 = 0; k0 < g.nz; ++k0) {
            const int M = s > 0 ? k0 : g.nz - 1 - k0;
            const int M4 = (M + 3) / 4 * 4;             // the replay reads whole blocks of four
            for (int t = 0; t < npair; ++t)
                for (int m = 1; m <= M4; ++m) {
                    const long long i = rec32_at(g, d, k0, s, t) + rec32_step(m);
                    if (i < 0 || i >= size || seen[(size_t)i]) return false;
                    seen[(size_t)i] = 1;
                    // four steps' pairs of a lane start 16-byte aligned
                    if (m % 4 == 1 && (i * 8) % 32 != 0) return false;
                }
        }
    }
    return true;
}

int main()
{
    const int grids[][4] = {{5, 5, 5, 4}, {17, 9, 6, 6}, {3, 3, 4, 2}, {4, 3, 2, 2},
                            {13, 11, 7, 4}, {21, 13, 9, 3}, {33, 33, 11, 2}};
    for (auto& q : grids) {
        Geometry g{};
        g.nx = q[0];
        g.ny = q[1];
        g.nz = q[2];
        g.ndir = q[3];
        g.N = (long long)g.nx * g.ny * g.nz;
        std::printf("%d %d %d %d %d %d\n", g.nx, g.ny, g.nz, g.ndir, check_fp64(g) ? 1 : 0,
                    check_fp32(g) ? 1 : 0);
    }
    return 0;
}
