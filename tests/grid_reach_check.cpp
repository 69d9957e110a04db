// Brute-force check of the library's culling lists (compiled against pack.cpp by
// tests/test_grid_reach.py; host code only).  For seeded points around the pocket it takes
// the list prefix a ligand atom at that point uses -- the reach level chosen with the same
// float arithmetic as the kernels -- and checks that it holds
//   candidate lists: every pocket atom within the cutoff,
//   near lists:      every pocket atom within the near cutoff,
//   residue lists:   every residue with an atom within 5 A,
// plus the table invariants (levels non-decreasing, the last level = the whole list).
// Input (binary, argv[1]): int32 M, float32 xyz[M][3], int32 residue[M].
// argv[2..4]: cutoff, near cutoff, cell edge; argv[5]: number of points.
// Prints "ok <points> <mean candidate entries used> <mean of the whole lists>" or the first
// failures, and exits non-zero on a failure.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "trids_internal.h"

using namespace trids;

namespace {

// The level of a point at fractional cell coordinates (fx, fy, fz), exactly as the kernels
// compute it: floor(|u| / (sqrt(3) / 2) * kReachLevels), capped at the last level.
int reach_level(float fx, float fy, float fz, int cx, int cy, int cz) {
    const float ux = fx - ((float)cx + 0.5f), uy = fy - ((float)cy + 0.5f), uz = fz - ((float)cz + 0.5f);
    const float scale = (float)kReachLevels * 1.1547005383792515f;
    return std::min(kReachLevels - 1, (int)(sqrtf(fmaf(uz, uz, fmaf(uy, uy, ux * ux))) * scale));
}

bool monotone(const std::vector<uint16_t>& lev, size_t cell, uint32_t whole, uint32_t unit) {
    for (int k = 1; k < kReachLevels; ++k)
        if (lev[cell * kReachLevels + k] < lev[cell * kReachLevels + k - 1]) return false;
    return (uint32_t)lev[cell * kReachLevels + kReachLevels - 1] * unit == whole;
}

}  // namespace

int main(int argc, char** argv) {
    if (argc < 6) return 2;
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    int M = 0;
    if (std::fread(&M, 4, 1, f) != 1 || M < 1) return 2;
    std::vector<float> xyz(3 * (size_t)M);
    std::vector<int32_t> res(M);
    if (std::fread(xyz.data(), 4, 3 * (size_t)M, f) != 3 * (size_t)M ||
        std::fread(res.data(), 4, M, f) != (size_t)M)
        return 2;
    std::fclose(f);
    const float cutoff = std::strtof(argv[2], nullptr), near_cut = std::strtof(argv[3], nullptr),
                h = std::strtof(argv[4], nullptr);
    const int n_pts = std::atoi(argv[5]);
    int n_res = 0;
    for (int r : res) n_res = std::max(n_res, r + 1);

    CandidateGrid g;
    build_grid(M, xyz.data(), cutoff, h, &g);
    std::vector<uint32_t> ns;
    std::vector<uint16_t> nl, nlev;
    build_near_lists(M, xyz.data(), near_cut, g, &ns, &nl, &nlev);
    ResidueGrid rg;
    build_residue_grid(M, xyz.data(), res.data(), n_res, g, &rg);

    const int nx = g.dims[0], ny = g.dims[1], nz = g.dims[2];
    const float inv_h = 1.f / h;
    std::mt19937 rng(12345);
    std::uniform_real_distribution<float> U(-0.5f, 0.5f);
    long pts = 0, fails = 0, used = 0, whole = 0;
    std::vector<char> in_c(M + 1), in_n(M), in_r(n_res);
    std::vector<float> rmin(n_res);
    for (int t = 0; t < n_pts && fails < 10; ++t) {
        // around a random pocket atom, out to past the cutoff; every fourth point on a cell
        // corner or face, where the level is the last one or the arithmetic is tight
        const int j0 = (int)(rng() % (uint32_t)M);
        float x = xyz[3 * j0] + U(rng) * 2.4f * cutoff, y = xyz[3 * j0 + 1] + U(rng) * 2.4f * cutoff,
              z = xyz[3 * j0 + 2] + U(rng) * 2.4f * cutoff;
        if (t % 4 == 0) {
            x = g.lo[0] + std::round((x - g.lo[0]) * inv_h) * h;
            if (t % 8 == 0) y = g.lo[1] + std::round((y - g.lo[1]) * inv_h) * h;
        }
        const float fx = (x - g.lo[0]) * inv_h, fy = (y - g.lo[1]) * inv_h, fz = (z - g.lo[2]) * inv_h;
        if (!(fx >= 0.f && fy >= 0.f && fz >= 0.f && fx < (float)nx && fy < (float)ny && fz < (float)nz)) continue;
        const int cx = std::min((int)fx, nx - 1), cy = std::min((int)fy, ny - 1), cz = std::min((int)fz, nz - 1);
        const size_t cell = ((size_t)cz * ny + cy) * nx + cx;
        const int k = reach_level(fx, fy, fz, cx, cy, cz);
        ++pts;
        if (!monotone(g.levels, cell, g.start[cell + 1] - g.start[cell], 8) ||
            !monotone(nlev, cell, ns[cell + 1] - ns[cell], 1) ||
            !monotone(rg.levels, cell, rg.cell_start[cell + 1] - rg.cell_start[cell], 1)) {
            std::printf("level table of cell %zu is not monotone or does not end at the whole list\n", cell);
            ++fails;
            continue;
        }
        std::fill(in_c.begin(), in_c.end(), 0);
        std::fill(in_n.begin(), in_n.end(), 0);
        std::fill(in_r.begin(), in_r.end(), 0);
        std::fill(rmin.begin(), rmin.end(), 3.0e38f);
        const uint32_t nc = 8u * g.levels[cell * kReachLevels + k];
        for (uint32_t q = 0; q < nc; ++q) in_c[g.cand[g.start[cell] + q]] = 1;
        for (int q = 0; q < nlev[cell * kReachLevels + k]; ++q) in_n[nl[ns[cell] + q]] = 1;
        for (int q = 0; q < rg.levels[cell * kReachLevels + k]; ++q)
            in_r[rg.list[rg.cell_start[cell] + q] & 0x1fffu] = 1;
        used += nc;
        whole += g.start[cell + 1] - g.start[cell];
        for (int j = 0; j < M; ++j) {
            const float dx = x - xyz[3 * j], dy = y - xyz[3 * j + 1], dz = z - xyz[3 * j + 2];
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (r2 < cutoff * cutoff && !in_c[j]) {
                std::printf("candidate list misses atom %d at r = %.5f (level %d)\n", j, std::sqrt(r2), k);
                ++fails;
            }
            if (r2 < near_cut * near_cut && !in_n[j]) {
                std::printf("near list misses atom %d at r = %.5f (level %d)\n", j, std::sqrt(r2), k);
                ++fails;
            }
            rmin[res[j]] = std::min(rmin[res[j]], r2);
        }
        for (int r = 0; r < n_res; ++r)
            if (rmin[r] < kMdnCut * kMdnCut && !in_r[r]) {
                std::printf("residue list misses residue %d at d = %.5f (level %d)\n", r, std::sqrt(rmin[r]), k);
                ++fails;
            }
    }
    if (fails) return 1;
    std::printf("ok %ld %.2f %.2f\n", pts, pts ? (double)used / pts : 0.0, pts ? (double)whole / pts : 0.0);
    return 0;
}
