// Runs the HOME-LBM step kernel's own device functions (halo load, Hermite
// rebuild into the ring, pull and collide) on the host, block by block and
// thread by thread in the kernel's phase order, so that the tiling, the
// ring's lifetimes and the boundary handling can be checked on a machine
// without a GPU. Stale ring entries are poisoned, so a read of one shows.
//
//   home_tile_emulator rebuild-check
//   home_tile_emulator nx ny nz tau uin_x uin_y uin_z F_x F_y F_z bc_x steps
//                      in.bin out.bin [solid.bin [planes_per_block]]
#include <cstdio>
#include <cstdlib>
#include <random>
#include <string>
#include <vector>

#include "../paper_2603_09668_gb300/csrc/lbm.cu"

using namespace dw;

// home_rebuild_all against the per-direction home_rebuild, in units of w_i
static int rebuild_check() {
    std::mt19937 gen(1);
    std::normal_distribution<float> nd(0.0f, 1.0f);
    double worst = 0.0;
    for (int t = 0; t < 1000; ++t) {
        float a[10];
        a[0] = 0.01f * nd(gen);
        for (int k = 1; k < 4; ++k) a[k] = 0.05f * nd(gen);
        for (int k = 4; k < 10; ++k) a[k] = 3e-3f * nd(gen);
        float g[19];
        home_rebuild_all(a, g);
        for (int i = 0; i < 19; ++i) {
            const double d = fabs((double)g[i] - (double)home_rebuild(i, a)) / D3Q19::w(i);
            worst = d > worst ? d : worst;
        }
    }
    printf("%.3e\n", worst);
    return 0;
}

int main(int argc, char **argv) {
    if (argc == 2 && std::string(argv[1]) == "rebuild-check") return rebuild_check();
    if (argc < 15) return 2;
    dw_lbm_desc d{};
    d.nx = atoi(argv[1]);
    d.ny = atoi(argv[2]);
    d.nz = atoi(argv[3]);
    d.tau = (float)atof(argv[4]);
    for (int a = 0; a < 3; ++a) {
        d.u_inlet[a] = (float)atof(argv[5 + a]);
        d.force[a] = (float)atof(argv[8 + a]);
    }
    d.bc_x = atoi(argv[11]);
    d.max_tape = 1;
    const int steps = atoi(argv[12]);
    LbmHandle h;
    h.desc = d;
    fill_lbm_params(&h);
    const LbmParams &L = h.L;
    const HomeParams H = home_params(d);
    const int nc = L.ncell;
    std::vector<float> a(10 * (size_t)nc), b(10 * (size_t)nc);
    FILE *f = fopen(argv[13], "rb");
    if (!f || fread(a.data(), 4, a.size(), f) != a.size()) return 3;
    fclose(f);
    std::vector<uint8_t> solid(nc, 0);
    const bool has_solid = argc > 15;
    if (has_solid) {
        f = fopen(argv[15], "rb");
        if (!f || fread(solid.data(), 1, nc, f) != (size_t)nc) return 4;
        fclose(f);
    }
    // link words as the link-mask kernel builds them
    std::vector<uint32_t> links(nc, 0);
    for (int cell = 0; cell < nc; ++cell) {
        const int x = cell % L.nx, y = (cell / L.nx) % L.ny, z = cell / (L.nx * L.ny);
        uint32_t m = solid[cell] ? 1u : 0u;
        for (int i = 1; i < 19; ++i) {
            const int tx = x + D3Q19::cx(i);
            if (L.bc_x == 1 && (tx < 0 || tx > L.nx - 1)) continue;
            const int t = (wrap_full(z + D3Q19::cz(i), L.nz) * L.ny +
                           wrap_full(y + D3Q19::cy(i), L.ny)) * L.nx + wrap_full(tx, L.nx);
            if (solid[t]) m |= 1u << i;
        }
        links[cell] = m;
    }
    const uint8_t *sp = has_solid ? solid.data() : nullptr;
    const uint32_t *lp = has_solid ? links.data() : nullptr;
    const int tz = argc > 16 ? atoi(argv[16]) : 5;
    const int gx = (L.nx + HOME_TX - 1) / HOME_TX, gy = (L.ny + HOME_TY - 1) / HOME_TY;
    const int gz = (L.nz + tz - 1) / tz;
    std::vector<float> sm(HOME_SMEM / sizeof(float));
    for (int s = 0; s < steps; ++s) {
        for (int bz = 0; bz < gz; ++bz)
            for (int by = 0; by < gy; ++by)
                for (int bx = 0; bx < gx; ++bx) {
                    std::fill(sm.begin(), sm.end(), 1e30f);
                    const int x0 = bx * HOME_TX, y0 = by * HOME_TY, z0 = bz * tz;
                    const int z1 = std::min(z0 + tz, L.nz);
                    const int plane = L.nx * L.ny;
                    HomeHalo hh;
                    for (int c = 0; c < HOME_PLANE; ++c) {
                        const int xy = home_halo_xy(L, x0, y0, c);
                        home_halo_load(L, a.data(), sp, xy, home_wrap_z(L, z0 - 1), hh);
                        home_halo_store(hh, sm.data(), 0, c);
                        home_halo_load(L, a.data(), sp, xy, z0, hh);
                        home_halo_store(hh, sm.data(), 1, c);
                    }
                    for (int z = z0; z < z1; ++z) {
                        const int q = z - z0 + 1;
                        for (int c = 0; c < HOME_PLANE; ++c) {
                            home_halo_load(L, a.data(), sp, home_halo_xy(L, x0, y0, c),
                                           home_wrap_z(L, z + 1), hh);
                            home_halo_store(hh, sm.data(), q + 1, c);
                        }
                        for (int tid = 0; tid < 256; ++tid) {
                            int ix, iy;
                            if (!home_interior(tid, ix, iy)) continue;
                            const bool inside = x0 + ix < L.nx && y0 + iy < L.ny;
                            const uint32_t lk =
                                (lp && inside) ? lp[z * plane + (y0 + iy) * L.nx + x0 + ix] : 0u;
                            home_tile_cell(L, H, a.data(), b.data(), lk, sm.data(), q, x0, y0, z,
                                           ix, iy);
                        }
                    }
                }
        std::swap(a, b);
    }
    f = fopen(argv[14], "wb");
    if (!f) return 5;
    fwrite(a.data(), 4, a.size(), f);
    fclose(f);
    return 0;
}
