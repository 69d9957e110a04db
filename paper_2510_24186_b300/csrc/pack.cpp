// Host-side ligand packing: torsion tree, packed atom order, intra-ligand pair list.
//
// The paper fixes the degrees of freedom (Sec. 2 "Conformation sampling":
// translation, rotation, torsion angles of rotatable bonds) and counts N_tor
// (Eq. E_screen) but not the tree layout.  Rules used (also stated in trids.h):
// fragments are the components left after cutting rotatable bonds; the root is
// the fragment of minimum height in the fragment tree (ties: smallest input atom
// index); torsions are numbered in BFS order from the root with children ordered
// by their smallest input atom index; atoms are laid out in DFS pre-order of
// fragments (same child order, ascending input index inside a fragment) so each
// torsion's moving subtree is one contiguous index range; intra-ligand pairs are
// atoms in different fragments at least 4 bonds apart.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "trids_internal.h"

namespace trids {

namespace {

std::string fmt(const char* f, int a, int b = 0) {
    char buf[160];
    std::snprintf(buf, sizeof buf, f, a, b);
    return buf;
}

}  // namespace

namespace {

constexpr int kFmax = kTmax + 1;   // a connected ligand with <= kTmax rotatable bonds has <= kTmax + 1 fragments

// The fragment tree's working arrays (fixed size: no heap traffic per ligand, so that many
// ligands pack in parallel without contending for the allocator).
struct FragTree {
    int nf = 0;
    int n_nbr[kFmax];
    int nbr_f[kFmax][kFmax];   // neighbour fragments, ascending
    int nbr_a[kFmax][kFmax];   // ... and this fragment's atom of the joining bond
    int other_atom[kFmax][kFmax];
    int parent[kFmax], tor_of[kFmax], first[kFmax], sub[kFmax], count[kFmax];
};

// Eccentricity of fragment s in the fragment tree.
int frag_height(const FragTree& F, int s) {
    int d[kFmax], q[kFmax];
    for (int f = 0; f < F.nf; ++f) d[f] = -1;
    int head = 0, tail = 0, h = 0;
    d[s] = 0;
    q[tail++] = s;
    while (head < tail) {
        const int u = q[head++];
        h = std::max(h, d[u]);
        for (int k = 0; k < F.n_nbr[u]; ++k) {
            const int v = F.nbr_f[u][k];
            if (d[v] < 0) { d[v] = d[u] + 1; q[tail++] = v; }
        }
    }
    return h;
}

// DFS pre-order layout from fragment u: its atoms (ascending input index), then its
// children in ascending fragment number.
void frag_dfs(FragTree& F, int u, int n, const int* fragof, std::vector<int>* perm) {
    F.first[u] = (int)perm->size();
    for (int i = 0; i < n; ++i)
        if (fragof[i] == u) perm->push_back(i);
    F.sub[u] = F.count[u];
    for (int k = 0; k < F.n_nbr[u]; ++k) {
        const int v = F.nbr_f[u][k];
        if (F.parent[v] == u) {
            frag_dfs(F, v, n, fragof, perm);
            F.sub[u] += F.sub[v];
        }
    }
}

}  // namespace

std::string pack_ligand(int n, const float* xyz, const int32_t* type, int n_types, int nb,
                        const int32_t* bonds, const uint8_t* rot, PackedLigand* out) {
    if (n < 1 || n > kLmax) return fmt("ligand has %d atoms (allowed 1..%d)", n, kLmax);
    if (nb < 0) return "negative bond count";
    for (int i = 0; i < n; ++i) {
        if (type[i] < 0 || type[i] >= n_types) return fmt("atom %d has type %d out of range", i, type[i]);
        if (!std::isfinite(xyz[3 * i]) || !std::isfinite(xyz[3 * i + 1]) || !std::isfinite(xyz[3 * i + 2]))
            return fmt("atom %d has a non-finite coordinate", i);
    }
    // bond matrix: 0 none, 1 rigid, 2 rotatable
    uint8_t bm[kLmax * kLmax];
    std::memset(bm, 0, (size_t)n * n);
    int n_rot = 0;
    for (int b = 0; b < nb; ++b) {
        int a0 = bonds[2 * b], a1 = bonds[2 * b + 1];
        if (a0 < 0 || a1 < 0 || a0 >= n || a1 >= n) return fmt("bond %d has an atom index out of range", b);
        if (a0 == a1) return fmt("bond %d joins atom %d to itself", b, a0);
        if (bm[a0 * n + a1]) return fmt("bond %d duplicates an earlier bond", b);
        uint8_t kind = rot[b] ? 2 : 1;
        bm[a0 * n + a1] = bm[a1 * n + a0] = kind;
        n_rot += rot[b] ? 1 : 0;
    }
    if (n_rot > kTmax) return fmt("%d rotatable bonds (at most %d)", n_rot, kTmax);

    // adjacency as bit sets; atoms within three bonds of each other (walks of up to three
    // bonds reach exactly the atoms at bond distance <= 3)
    constexpr int kW = (kLmax + 63) / 64;
    uint64_t adj[kLmax][kW], near2[kLmax][kW], near3[kLmax][kW];
    std::memset(adj, 0, sizeof adj);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (bm[i * n + j]) adj[i][j >> 6] |= 1ull << (j & 63);
    auto spread = [&](const uint64_t (*from)[kW], uint64_t (*to)[kW]) {
        for (int i = 0; i < n; ++i) {
            for (int w = 0; w < kW; ++w) to[i][w] = from[i][w];
            for (int w = 0; w < kW; ++w)
                for (uint64_t m = adj[i][w]; m; m &= m - 1) {
                    const int j = 64 * w + __builtin_ctzll(m);
                    for (int x = 0; x < kW; ++x) to[i][x] |= from[j][x];
                }
        }
    };
    spread(adj, near2);     // within two bonds (and the atom itself through its neighbours)
    spread(near2, near3);   // within three bonds
    // connectivity: the atoms reachable from atom 0
    {
        uint64_t seen[kW] = {0}, front[kW] = {0};
        seen[0] = front[0] = 1ull;
        for (bool grew = true; grew;) {
            uint64_t next[kW] = {0};
            for (int w = 0; w < kW; ++w)
                for (uint64_t m = front[w]; m; m &= m - 1) {
                    const int j = 64 * w + __builtin_ctzll(m);
                    for (int x = 0; x < kW; ++x) next[x] |= adj[j][x];
                }
            grew = false;
            for (int w = 0; w < kW; ++w) {
                front[w] = next[w] & ~seen[w];
                seen[w] |= front[w];
                grew |= front[w] != 0;
            }
        }
        for (int i = 1; i < n; ++i)
            if (!((seen[i >> 6] >> (i & 63)) & 1ull)) return fmt("atom %d is not connected to atom 0", i);
    }

    // fragments: union over rigid bonds, numbered by their smallest atom index
    int up[kLmax];
    for (int i = 0; i < n; ++i) up[i] = i;
    auto find = [&](int a) {
        while (up[a] != a) a = up[a] = up[up[a]];
        return a;
    };
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (bm[i * n + j] == 1) up[find(i)] = find(j);
    int rep_to_frag[kLmax], fragof[kLmax];
    for (int i = 0; i < n; ++i) rep_to_frag[i] = -1;
    int nf = 0;
    for (int i = 0; i < n; ++i) {   // ascending i: first atom seen is the fragment minimum
        int r = find(i);
        if (rep_to_frag[r] < 0) rep_to_frag[r] = nf++;
        fragof[i] = rep_to_frag[r];
    }
    if (n_rot != nf - 1) return "a rotatable bond lies in a ring (the fragments do not form a tree)";
    // fragment tree edges with the bond atoms on each side
    FragTree F;
    F.nf = nf;
    for (int f = 0; f < nf; ++f) {
        F.n_nbr[f] = 0;
        F.count[f] = 0;
        for (int g = 0; g < nf; ++g) F.other_atom[f][g] = -1;
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (bm[i * n + j] == 2) {
                int fi = fragof[i], fj = fragof[j];
                if (fi == fj) return "a rotatable bond lies inside a rigid fragment (ring)";
                if (F.other_atom[fi][fj] >= 0 && F.other_atom[fi][fj] != i)
                    return "two rotatable bonds join the same pair of fragments (ring)";
                if (F.other_atom[fi][fj] < 0) {
                    F.nbr_f[fi][F.n_nbr[fi]] = fj;
                    F.nbr_a[fi][F.n_nbr[fi]++] = i;
                }
                F.other_atom[fi][fj] = i;
            }
    for (int f = 0; f < nf; ++f) {   // neighbours by ascending fragment (each appears once)
        for (int x = 1; x < F.n_nbr[f]; ++x)
            for (int y = x; y > 0 && F.nbr_f[f][y - 1] > F.nbr_f[f][y]; --y) {
                std::swap(F.nbr_f[f][y - 1], F.nbr_f[f][y]);
                std::swap(F.nbr_a[f][y - 1], F.nbr_a[f][y]);
            }
    }

    // root: smallest height (eccentricity in the fragment tree), ties by fragment number
    int root = 0, best = 1 << 20;
    for (int f = 0; f < nf; ++f) {
        int h = frag_height(F, f);
        if (h < best) { best = h; root = f; }
    }
    // BFS: torsion numbers and parents
    int bfs[kFmax], nbfs = 0;
    for (int f = 0; f < nf; ++f) { F.parent[f] = -2; F.tor_of[f] = -1; }
    F.parent[root] = -1;
    bfs[nbfs++] = root;
    for (int h = 0; h < nbfs; ++h) {
        int u = bfs[h];
        for (int k = 0; k < F.n_nbr[u]; ++k) {
            const int v = F.nbr_f[u][k];
            if (F.parent[v] == -2) {
                F.parent[v] = u;
                F.tor_of[v] = nbfs - 1;
                bfs[nbfs++] = v;
            }
        }
    }
    // DFS pre-order layout and subtree atom counts
    for (int i = 0; i < n; ++i) F.count[fragof[i]]++;
    out->perm.clear();
    out->perm.reserve(n);
    frag_dfs(F, root, n, fragof, &out->perm);
    int packed_of[kLmax];
    for (int k = 0; k < n; ++k) packed_of[out->perm[k]] = k;

    int T = nf - 1;
    out->n_atoms = n;
    out->n_tor = T;
    out->frag.assign(n, 0);
    for (int k = 0; k < n; ++k) {
        int f = fragof[out->perm[k]];
        out->frag[k] = (f == root) ? 0 : F.tor_of[f] + 1;
    }
    out->tp.assign(T, 0); out->th.assign(T, 0); out->tpar.assign(T, -1);
    out->sb.assign(T, 0); out->se.assign(T, 0);
    for (int f = 0; f < nf; ++f) {
        if (f == root) continue;
        int k = F.tor_of[f], p = F.parent[f];
        out->tp[k] = packed_of[F.other_atom[p][f]];
        out->th[k] = packed_of[F.other_atom[f][p]];
        out->tpar[k] = (p == root) ? -1 : F.tor_of[p];
        out->sb[k] = F.first[f];
        out->se[k] = F.first[f] + F.sub[f];
    }
    double s[3] = {0, 0, 0};
    int cnt = 0;
    for (int i = 0; i < n; ++i)
        if (fragof[i] == root) {
            for (int d = 0; d < 3; ++d) s[d] += (double)xyz[3 * i + d];
            ++cnt;
        }
    for (int d = 0; d < 3; ++d) out->c[d] = s[d] / cnt;
    // intra pairs: different fragments, at least four bonds apart
    out->pairs.clear();
    for (int a = 0; a < n; ++a) {
        const int ia = out->perm[a];
        for (int b = a + 1; b < n; ++b) {
            const int ib = out->perm[b];
            if (out->frag[a] != out->frag[b] && !((near3[ia][ib >> 6] >> (ib & 63)) & 1ull))
                out->pairs.push_back({a, b});
        }
    }
    return "";
}

void topology_ints(const PackedLigand& lg, std::vector<int32_t>* o) {
    o->clear();
    o->push_back(lg.n_atoms);
    o->push_back(lg.n_tor);
    o->push_back((int)lg.pairs.size());
    o->insert(o->end(), lg.perm.begin(), lg.perm.end());
    o->insert(o->end(), lg.frag.begin(), lg.frag.end());
    for (int k = 0; k < lg.n_tor; ++k) {
        o->push_back(lg.tp[k]); o->push_back(lg.th[k]); o->push_back(lg.tpar[k]);
        o->push_back(lg.sb[k]); o->push_back(lg.se[k]);
    }
    for (auto& p : lg.pairs) { o->push_back(p.first); o->push_back(p.second); }
}

// ---------------------------------------------------------------- candidate grid
void build_grid(int M, const float* xyz, float cutoff, float h, CandidateGrid* g) {
    double lo[3] = {1e30, 1e30, 1e30}, hi[3] = {-1e30, -1e30, -1e30};
    for (int j = 0; j < M; ++j)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], (double)xyz[3 * j + d]);
            hi[d] = std::max(hi[d], (double)xyz[3 * j + d]);
        }
    for (int d = 0; d < 3; ++d) {
        double a = lo[d] - cutoff - h, b = hi[d] + cutoff + h;
        g->lo[d] = (float)a;
        g->dims[d] = (int)std::ceil((b - (double)g->lo[d]) / h);
    }
    g->h = h;
    const int nx = g->dims[0], ny = g->dims[1], nz = g->dims[2];
    const size_t ncell = (size_t)nx * ny * nz;
    // a point in a cell is within h*sqrt(3)/2 of its centre; the margin covers float rounding
    const double reach = cutoff + 0.5 * std::sqrt(3.0) * h + 1e-3 * h + 1e-4;
    const double reach2 = reach * reach;
    const int span = (int)std::ceil(reach / h) + 1;
    // two passes over (atom, nearby cell): count, then fill in ascending atom order
    auto visit = [&](int j, auto&& fn) {
        const double p[3] = {xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2]};
        int c[3];
        for (int d = 0; d < 3; ++d) c[d] = (int)std::floor((p[d] - g->lo[d]) / h);
        for (int iz = std::max(0, c[2] - span); iz <= std::min(nz - 1, c[2] + span); ++iz) {
            const double cz = g->lo[2] + (iz + 0.5) * h - p[2];
            for (int iy = std::max(0, c[1] - span); iy <= std::min(ny - 1, c[1] + span); ++iy) {
                const double cy = g->lo[1] + (iy + 0.5) * h - p[1];
                const double r2yz = cy * cy + cz * cz;
                if (r2yz > reach2) continue;
                for (int ix = std::max(0, c[0] - span); ix <= std::min(nx - 1, c[0] + span); ++ix) {
                    const double cx = g->lo[0] + (ix + 0.5) * h - p[0];
                    if (cx * cx + r2yz <= reach2) fn(((size_t)iz * ny + iy) * nx + ix);
                }
            }
        }
    };
    std::vector<uint32_t> count(ncell, 0);
    for (int j = 0; j < M; ++j) visit(j, [&](size_t cell) { ++count[cell]; });
    g->start.assign(ncell + 1, 0);
    size_t total = 0;
    for (size_t cidx = 0; cidx < ncell; ++cidx) {
        g->start[cidx] = (uint32_t)total;
        total += (count[cidx] + 7) / 8 * 8;
    }
    g->start[ncell] = (uint32_t)total;
    g->cand.assign(total, (uint16_t)M);
    std::vector<uint32_t> fill(g->start.begin(), g->start.end() - 1);
    for (int j = 0; j < M; ++j) visit(j, [&](size_t cell) { g->cand[fill[cell]++] = (uint16_t)j; });
    // Reach levels: a point at distance delta from its cell centre only needs the entries
    // within cutoff + delta of the centre.  Level k covers delta <= (k + 1) / kReachLevels of
    // the half diagonal; each cell's entries are ordered by level (ascending atom index
    // inside a level) and level k's block count is stored.
    g->levels.assign(ncell * kReachLevels, 0);
    const double half = 0.5 * std::sqrt(3.0) * h, margin = 1e-3 * h + 1e-4;
    double thr2[kReachLevels];
    for (int k = 0; k < kReachLevels; ++k) {
        const double t = cutoff + half * (k + 1) / kReachLevels + margin;
        thr2[k] = t * t;
    }
    std::vector<uint16_t> tmp;
    std::vector<int> lvl;
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                const size_t cell = ((size_t)iz * ny + iy) * nx + ix;
                const uint32_t b = g->start[cell], n = count[cell];
                if (n == 0) continue;
                const double c[3] = {g->lo[0] + (ix + 0.5) * h, g->lo[1] + (iy + 0.5) * h, g->lo[2] + (iz + 0.5) * h};
                int cnt[kReachLevels] = {0};
                lvl.resize(n);
                for (uint32_t q = 0; q < n; ++q) {
                    const int j = g->cand[b + q];
                    double r2 = 0;
                    for (int d = 0; d < 3; ++d) {
                        const double u = (double)xyz[3 * j + d] - c[d];
                        r2 += u * u;
                    }
                    int k = 0;
                    while (k < kReachLevels - 1 && r2 > thr2[k]) ++k;
                    lvl[q] = k;
                    ++cnt[k];
                }
                int at[kReachLevels];
                for (int k = 0, acc = 0; k < kReachLevels; ++k) {
                    at[k] = acc;
                    acc += cnt[k];
                    g->levels[cell * kReachLevels + k] = (uint16_t)((acc + 7) / 8);
                }
                tmp.assign(g->cand.begin() + b, g->cand.begin() + b + n);
                for (uint32_t q = 0; q < n; ++q) g->cand[b + at[lvl[q]]++] = tmp[q];
            }
}

// Orders each cell's list [start[c], start[c+1]) by reach level and fills levels[c][k] with
// the number of entries of levels 0..k (level k: distance from the cell centre within
// base + (k + 1) / kReachLevels of the half diagonal, plus the rounding margin; the last level
// takes the rest).  dist2(entry, centre) is an entry's squared distance from a cell centre.
template <class E, class D>
static void order_by_reach(const CandidateGrid& g, double base, const std::vector<uint32_t>& start, std::vector<E>* list,
                           std::vector<uint16_t>* levels, D&& dist2) {
    const int nx = g.dims[0], ny = g.dims[1], nz = g.dims[2];
    const double h = g.h, half = 0.5 * std::sqrt(3.0) * h, margin = 1e-3 * h + 1e-4;
    double thr2[kReachLevels];
    for (int k = 0; k < kReachLevels; ++k) {
        const double t = base + half * (k + 1) / kReachLevels + margin;
        thr2[k] = t * t;
    }
    levels->assign((size_t)nx * ny * nz * kReachLevels, 0);
    std::vector<E> tmp;
    std::vector<int> lvl;
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                const size_t cell = ((size_t)iz * ny + iy) * nx + ix;
                const uint32_t b = start[cell], n = start[cell + 1] - b;
                if (n == 0) continue;
                const double c[3] = {g.lo[0] + (ix + 0.5) * h, g.lo[1] + (iy + 0.5) * h, g.lo[2] + (iz + 0.5) * h};
                int cnt[kReachLevels] = {0};
                lvl.resize(n);
                for (uint32_t q = 0; q < n; ++q) {
                    const double r2 = dist2((*list)[b + q], c);
                    int k = 0;
                    while (k < kReachLevels - 1 && r2 > thr2[k]) ++k;
                    lvl[q] = k;
                    ++cnt[k];
                }
                int at[kReachLevels];
                for (int k = 0, acc = 0; k < kReachLevels; ++k) {
                    at[k] = acc;
                    acc += cnt[k];
                    (*levels)[cell * kReachLevels + k] = (uint16_t)acc;
                }
                tmp.assign(list->begin() + b, list->begin() + b + n);
                for (uint32_t q = 0; q < n; ++q) (*list)[b + at[lvl[q]]++] = tmp[q];
            }
}

void build_residue_grid(int M, const float* xyz, const int32_t* res, int n_res, const CandidateGrid& g,
                        ResidueGrid* out) {
    out->n_res = n_res;
    out->start.assign(n_res + 1, 0);
    for (int j = 0; j < M; ++j) ++out->start[res[j] + 1];
    for (int r = 0; r < n_res; ++r) out->start[r + 1] += out->start[r];
    out->atoms.assign(M, 0);
    {
        std::vector<int32_t> fill(out->start.begin(), out->start.end() - 1);
        for (int j = 0; j < M; ++j) out->atoms[fill[res[j]]++] = (uint16_t)j;   // ascending j per residue
    }
    const int nx = g.dims[0], ny = g.dims[1], nz = g.dims[2];
    const double h = g.h;
    const size_t ncell = (size_t)nx * ny * nz;
    const double reach = kMdnCut + 0.5 * std::sqrt(3.0) * h + 1e-3 * h + 1e-4;
    const double reach2 = reach * reach;
    const int span = (int)std::ceil(reach / h) + 1;
    // cells within reach of any atom of residue r, each once (mark = last residue seen)
    std::vector<int32_t> mark(ncell, -1);
    auto visit_residue = [&](int r, auto&& fn) {
        for (int a = out->start[r]; a < out->start[r + 1]; ++a) {
            const int j = out->atoms[a];
            const double p[3] = {xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2]};
            int c[3];
            for (int d = 0; d < 3; ++d) c[d] = (int)std::floor((p[d] - g.lo[d]) / h);
            for (int iz = std::max(0, c[2] - span); iz <= std::min(nz - 1, c[2] + span); ++iz) {
                const double cz = g.lo[2] + (iz + 0.5) * h - p[2];
                for (int iy = std::max(0, c[1] - span); iy <= std::min(ny - 1, c[1] + span); ++iy) {
                    const double cy = g.lo[1] + (iy + 0.5) * h - p[1];
                    const double r2yz = cy * cy + cz * cz;
                    if (r2yz > reach2) continue;
                    for (int ix = std::max(0, c[0] - span); ix <= std::min(nx - 1, c[0] + span); ++ix) {
                        const double cx = g.lo[0] + (ix + 0.5) * h - p[0];
                        if (cx * cx + r2yz > reach2) continue;
                        const size_t cell = ((size_t)iz * ny + iy) * nx + ix;
                        if (mark[cell] == r) continue;
                        mark[cell] = r;
                        fn(cell);
                    }
                }
            }
        }
    };
    std::vector<uint32_t> count(ncell, 0);
    for (int r = 0; r < n_res; ++r) visit_residue(r, [&](size_t cell) { ++count[cell]; });
    out->cell_start.assign(ncell + 1, 0);
    size_t total = 0;
    for (size_t c = 0; c < ncell; ++c) {
        out->cell_start[c] = (uint32_t)total;
        total += count[c];
    }
    out->cell_start[ncell] = (uint32_t)total;
    out->list.assign(total, 0);
    std::fill(mark.begin(), mark.end(), -1);
    std::vector<uint32_t> fill(out->cell_start.begin(), out->cell_start.end() - 1);
    for (int r = 0; r < n_res; ++r) {
        const uint32_t ent = (uint32_t)r | ((uint32_t)out->start[r] << 13) |
                             ((uint32_t)(out->start[r + 1] - out->start[r]) << 26);
        visit_residue(r, [&](size_t cell) { out->list[fill[cell]++] = ent; });
    }
    // reach levels by the residue's nearest atom to the cell centre
    order_by_reach(g, kMdnCut, out->cell_start, &out->list, &out->levels, [&](uint32_t ent, const double* c) {
        const int a0 = (int)((ent >> 13) & 0x1fffu), a1 = a0 + (int)(ent >> 26);
        double best = 1e300;
        for (int a = a0; a < a1; ++a) {
            const int j = out->atoms[a];
            double r2 = 0;
            for (int d = 0; d < 3; ++d) {
                const double u = (double)xyz[3 * j + d] - c[d];
                r2 += u * u;
            }
            best = std::min(best, r2);
        }
        return best;
    });
}

void build_near_lists(int M, const float* xyz, float cutoff, const CandidateGrid& g, std::vector<uint32_t>* start,
                      std::vector<uint16_t>* list, std::vector<uint16_t>* levels) {
    const int nx = g.dims[0], ny = g.dims[1], nz = g.dims[2];
    const double h = g.h;
    const size_t ncell = (size_t)nx * ny * nz;
    const double reach = cutoff + 0.5 * std::sqrt(3.0) * h + 1e-3 * h + 1e-4;
    const double reach2 = reach * reach;
    const int span = (int)std::ceil(reach / h) + 1;
    auto visit = [&](int j, auto&& fn) {
        const double p[3] = {xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2]};
        int c[3];
        for (int d = 0; d < 3; ++d) c[d] = (int)std::floor((p[d] - g.lo[d]) / h);
        for (int iz = std::max(0, c[2] - span); iz <= std::min(nz - 1, c[2] + span); ++iz) {
            const double cz = g.lo[2] + (iz + 0.5) * h - p[2];
            for (int iy = std::max(0, c[1] - span); iy <= std::min(ny - 1, c[1] + span); ++iy) {
                const double cy = g.lo[1] + (iy + 0.5) * h - p[1];
                const double r2yz = cy * cy + cz * cz;
                if (r2yz > reach2) continue;
                for (int ix = std::max(0, c[0] - span); ix <= std::min(nx - 1, c[0] + span); ++ix) {
                    const double cx = g.lo[0] + (ix + 0.5) * h - p[0];
                    if (cx * cx + r2yz <= reach2) fn(((size_t)iz * ny + iy) * nx + ix);
                }
            }
        }
    };
    std::vector<uint32_t> count(ncell, 0);
    for (int j = 0; j < M; ++j) visit(j, [&](size_t cell) { ++count[cell]; });
    start->assign(ncell + 1, 0);
    size_t total = 0;
    for (size_t c = 0; c < ncell; ++c) {
        (*start)[c] = (uint32_t)total;
        total += count[c];
    }
    (*start)[ncell] = (uint32_t)total;
    list->assign(total, 0);
    std::vector<uint32_t> fill(start->begin(), start->end() - 1);
    for (int j = 0; j < M; ++j) visit(j, [&](size_t cell) { (*list)[fill[cell]++] = (uint16_t)j; });
    order_by_reach(g, (double)cutoff, *start, list, levels, [&](uint16_t j, const double* c) {
        double r2 = 0;
        for (int d = 0; d < 3; ++d) {
            const double u = (double)xyz[3 * j + d] - c[d];
            r2 += u * u;
        }
        return r2;
    });
}

}  // namespace trids
