// libtrids: device code and C-ABI entry points for gradient-guided pose sampling
// (TRIDS, arXiv 2510.24186, Sec. 2 "Scoring functions" and "Conformation sampling",
// Sec. 4 items 1-4) on sm_103a.
//
// Mapping: one warp per pose.  The pose's coordinates, forces and sampler state live in
// the warp's shared-memory region; every block stages the scoring tables and the pocket
// (float4 per atom) into shared memory with bulk asynchronous copies.  Ligand-pocket pairs
// come from a precomputed candidate grid (each cell lists the pocket atoms that can lie
// within the cutoff of any point of the cell); a pose's candidate blocks and intra-ligand
// partner blocks are split into 32 equal contiguous lane segments, and per-atom partial
// forces are added in lane order.  Every sum runs in a fixed order, so results are
// bit-reproducible and the persistent and per-launch forms agree bit for bit.
//
// The device code is split over device_core.cuh, device_passes.cuh and device_kernels.cuh,
// the host objects over host_objects.cuh; this file holds the C-ABI and includes them all,
// so the whole library is one translation unit.
#include <cuda.h>   // driver types (CUcontext); the entry points are fetched at run time
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "trids_internal.h"

using namespace trids;

// =============================================================== error handling
namespace {
thread_local std::string g_err;

int fail(int code, const char* f, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, f);
    std::vsnprintf(buf, sizeof buf, f, ap);
    va_end(ap);
    g_err = buf;
    return code;
}
}  // namespace

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(TRIDS_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

#include "device_core.cuh"
#include "device_passes.cuh"
#include "device_kernels.cuh"
#include "host_objects.cuh"

// =============================================================== C-ABI
extern "C" {

const char* trids_last_error(void) { return g_err.c_str(); }

int trids_version(void) { return 100; }

int trids_make_pocket(const float* xyz, const int32_t* type, int32_t n_atoms, const float box_center[3],
                      const float box_size[3], float cell, const trids_params* prm, trids_pocket** out) {
    g_err.clear();
    if (!out) return fail(TRIDS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!xyz || !type || !box_center || !box_size) return fail(TRIDS_EINVAL, "NULL input array");
    if (n_atoms < 1 || n_atoms > 8191) return fail(TRIDS_EINVAL, "pocket has %d atoms (allowed 1..8191)", n_atoms);
    int rc = check_params(prm);
    if (rc) return rc;
    for (int j = 0; j < n_atoms; ++j) {
        if (type[j] < 0 || type[j] >= prm->n_types) return fail(TRIDS_EINVAL, "pocket atom %d type out of range", j);
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(xyz[3 * j + d])) return fail(TRIDS_EINVAL, "pocket atom %d non-finite", j);
    }
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(box_center[d]) || !(box_size[d] >= 0.f) || !std::isfinite(box_size[d]))
            return fail(TRIDS_EINVAL, "box must be finite with size >= 0");
    if (cell < 0.f || !std::isfinite(cell) || (cell > 0.f && cell < 0.25f))
        return fail(TRIDS_EINVAL, "cell must be 0 (default) or >= 0.25 A");
    std::unique_ptr<trids_pocket> pk(new trids_pocket());
    CK(cudaGetDevice(&pk->device));
    pk->M = n_atoms;
    pk->prm = *prm;
    pk->cutoff_built = prm->cutoff;
    pk->cell = cell > 0.f ? cell : 0.5f;
    pk->xyz.assign(xyz, xyz + 3 * (size_t)n_atoms);
    pk->type.assign(type, type + n_atoms);
    pk->orig.resize(n_atoms);
    for (int j = 0; j < n_atoms; ++j) pk->orig[j] = j;
    for (int d = 0; d < 3; ++d) {
        for (int b = 0; b < kMaxBoxes; ++b) {
            pk->box_lo[b][d] = box_center[d] - 0.5f * box_size[d];
            pk->box_hi[b][d] = box_center[d] + 0.5f * box_size[d];
        }
    }
    build_grid(n_atoms, xyz, prm->cutoff, pk->cell, &pk->grid);
    if (pk->grid.cand.size() >= (1ull << 32)) return fail(TRIDS_ENOMEM, "candidate grid too large");
    std::vector<float4> atoms(n_atoms + 1);
    std::vector<uint8_t> ptype(align_up((size_t)n_atoms + 1, 16), 0);
    for (int j = 0; j < n_atoms; ++j) ptype[j] = (uint8_t)type[j];
    fill_dev_params(prm, &pk->hp);
    std::vector<DevParams> hp(1, pk->hp);
    if ((rc = upload(&pk->d_atoms, atoms)) || (rc = upload(&pk->d_ptype, ptype)) ||
        (rc = upload(&pk->d_cell, pk->grid.start)) || (rc = upload(&pk->d_cand, pk->grid.cand)) ||
        (rc = upload(&pk->d_levels, pk->grid.levels)) ||
        (rc = upload(&pk->d_params, hp)) || (rc = upload_pocket_arrays(pk.get(), nullptr)) ||
        (rc = upload_near_lists(pk.get()))) {
        trids_free_pocket(pk.release());
        return rc;
    }
    *out = pk.release();
    return TRIDS_OK;
}

int trids_set_params(trids_pocket* pk, const trids_params* prm, void* stream) {
    g_err.clear();
    if (!pk) return fail(TRIDS_EINVAL, "pocket is NULL");
    int rc = check_params(prm);
    if (rc) return rc;
    if (prm->cutoff > pk->cutoff_built)
        return fail(TRIDS_EINVAL, "cutoff %.3f exceeds the %.3f the pocket grid was built for", prm->cutoff,
                    pk->cutoff_built);
    if ((rc = device_guard(pk->device))) return rc;
    const bool flags_changed = std::memcmp(pk->prm.flags, prm->flags, sizeof prm->flags) != 0;
    pk->prm = *prm;
    if (pk->d_maps) pk->maps_stale = true;
    if ((rc = upload_pocket_arrays(pk, (cudaStream_t)stream))) return rc;
    if (flags_changed)
        for (trids_batch* b : pk->batches)
            if ((rc = encode_intra(pk, b))) return rc;
    return TRIDS_OK;
}

int trids_set_boxes(trids_pocket* pk, int32_t n_boxes, const float* centers, const float* sizes) {
    g_err.clear();
    if (!pk || !centers || !sizes) return fail(TRIDS_EINVAL, "NULL argument");
    if (n_boxes < 1 || n_boxes > kMaxBoxes) return fail(TRIDS_EINVAL, "n_boxes must be in 1..%d", kMaxBoxes);
    for (int b = 0; b < n_boxes; ++b)
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(centers[3 * b + d]) || !(sizes[3 * b + d] >= 0.f) || !std::isfinite(sizes[3 * b + d]))
                return fail(TRIDS_EINVAL, "box %d must be finite with size >= 0", b);
    pk->n_boxes = n_boxes;
    for (int b = 0; b < kMaxBoxes; ++b) {
        const int s = b < n_boxes ? b : 0;
        for (int d = 0; d < 3; ++d) {
            pk->box_lo[b][d] = centers[3 * s + d] - 0.5f * sizes[3 * s + d];
            pk->box_hi[b][d] = centers[3 * s + d] + 0.5f * sizes[3 * s + d];
        }
    }
    return TRIDS_OK;
}

int trids_free_pocket(trids_pocket* pk) {
    if (!pk) return TRIDS_OK;
    for (trids_batch* b : pk->batches) b->owner = nullptr;
    pk->graph.clear();
    cudaFree(pk->d_atoms);
    cudaFree(pk->d_ptype);
    cudaFree(pk->d_cell);
    cudaFree(pk->d_cand);
    cudaFree(pk->d_levels);
    cudaFree(pk->d_params);
    cudaFree(pk->d_maps);
    cudaFree(pk->d_ncell);
    cudaFree(pk->d_nlist);
    cudaFree(pk->d_res_start);
    cudaFree(pk->d_rcell);
    cudaFree(pk->d_rlist);
    cudaFree(pk->d_rlevels);
    cudaFree(pk->d_nlevels);
    delete pk;
    return TRIDS_OK;
}

int trids_set_residues(trids_pocket* pk, int32_t n_res, const int32_t* residue) {
    g_err.clear();
    if (!pk || !residue) return fail(TRIDS_EINVAL, "NULL argument");
    if (n_res < 1 || n_res > TRIDS_MAX_RESIDUES)
        return fail(TRIDS_EINVAL, "n_res %d outside 1..%d", n_res, TRIDS_MAX_RESIDUES);
    if (pk->cutoff_built < kMdnCut)
        return fail(TRIDS_EINVAL, "the pocket grid was built for cutoff %.3f; residue terms need >= 5",
                    pk->cutoff_built);
    {
        std::vector<int> count(n_res, 0);
        for (int j = 0; j < pk->M; ++j) {
            if (residue[j] < 0 || residue[j] >= n_res) return fail(TRIDS_EINVAL, "atom %d: residue out of range", j);
            if (++count[residue[j]] > kMaxResidueAtoms)
                return fail(TRIDS_EINVAL, "residue %d has more than %d atoms", residue[j], kMaxResidueAtoms);
        }
    }
    int rc = device_guard(pk->device);
    if (rc) return rc;
    // Store the pocket atoms grouped by residue (ascending input index inside a residue), so
    // that a residue is one contiguous range of the staged pocket.  residue[] is indexed by
    // input atom; pk->orig maps the current storage order to input indices.
    const int M = pk->M;
    std::vector<int> order(M);
    for (int c = 0; c < M; ++c) order[c] = c;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        const int ra = residue[pk->orig[a]], rb = residue[pk->orig[b]];
        return ra != rb ? ra < rb : pk->orig[a] < pk->orig[b];
    });
    std::vector<float> xyz(3 * (size_t)M);
    std::vector<int> type(M), orig(M), res_sorted(M);
    for (int c = 0; c < M; ++c) {
        for (int d = 0; d < 3; ++d) xyz[3 * c + d] = pk->xyz[3 * order[c] + d];
        type[c] = pk->type[order[c]];
        orig[c] = pk->orig[order[c]];
        res_sorted[c] = residue[orig[c]];
    }
    CandidateGrid grid;
    build_grid(M, xyz.data(), pk->cutoff_built, pk->cell, &grid);
    if (grid.cand.size() != pk->grid.cand.size() || grid.start.size() != pk->grid.start.size())
        return fail(TRIDS_ECUDA, "internal: the reordered candidate grid changed size");
    ResidueGrid rg;
    build_residue_grid(M, xyz.data(), res_sorted.data(), n_res, grid, &rg);
    int32_t* d_start = nullptr;
    uint32_t* d_list = nullptr;
    uint32_t* d_cell = nullptr;
    uint16_t* d_rlev = nullptr;
    if ((rc = upload(&d_start, rg.start)) || (rc = upload(&d_cell, rg.cell_start)) || (rc = upload(&d_list, rg.list)) ||
        (rc = upload(&d_rlev, rg.levels))) {
        cudaFree(d_start); cudaFree(d_cell); cudaFree(d_list); cudaFree(d_rlev);
        return rc;
    }
    CK(cudaDeviceSynchronize());   // no launch may still read the arrays being replaced
    std::vector<uint8_t> ptype(align_up((size_t)M + 1, 16), 0);
    for (int j = 0; j < M; ++j) ptype[j] = (uint8_t)type[j];
    CK(cudaMemcpy(pk->d_ptype, ptype.data(), ptype.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(pk->d_cell, grid.start.data(), grid.start.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(pk->d_levels, grid.levels.data(), grid.levels.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    pk->xyz.swap(xyz);
    pk->type.swap(type);
    pk->orig.swap(orig);
    pk->grid = std::move(grid);
    if ((rc = upload_pocket_arrays(pk, nullptr))) return rc;   // atoms + candidate entries with flags
    if ((rc = upload_near_lists(pk))) return rc;
    cudaFree(pk->d_res_start); cudaFree(pk->d_rcell); cudaFree(pk->d_rlist); cudaFree(pk->d_rlevels);
    pk->d_res_start = d_start; pk->d_rcell = d_cell; pk->d_rlist = d_list; pk->d_rlevels = d_rlev;
    pk->rgrid = std::move(rg);
    return TRIDS_OK;
}

int trids_build_maps(trids_pocket* pk, float spacing, float margin, void* stream) {
    g_err.clear();
    if (!pk) return fail(TRIDS_EINVAL, "pocket is NULL");
    int rc = device_guard(pk->device);
    if (rc) return rc;
    if (spacing == 0.f) {
        if (pk->d_maps) {
            CK(cudaDeviceSynchronize());   // no launch may still read the maps
            cudaFree(pk->d_maps);
        }
        pk->d_maps = nullptr;
        pk->mdims[0] = pk->mdims[1] = pk->mdims[2] = 0;
        pk->maps_stale = false;
        return TRIDS_OK;
    }
    if (!(spacing >= 0.05f && spacing <= 4.f)) return fail(TRIDS_EINVAL, "spacing must be 0 or in [0.05, 4] A");
    if (!(margin >= 0.f && margin <= 64.f)) return fail(TRIDS_EINVAL, "margin must be in [0, 64] A");
    float lo[3], hi[3];
    int n[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = pk->box_lo[0][d];
        hi[d] = pk->box_hi[0][d];
        for (int b = 1; b < pk->n_boxes; ++b) {
            lo[d] = std::min(lo[d], pk->box_lo[b][d]);
            hi[d] = std::max(hi[d], pk->box_hi[b][d]);
        }
        lo[d] -= margin;
        hi[d] += margin;
        n[d] = (int)std::ceil((double)(hi[d] - lo[d]) / spacing) + 1;
        if (n[d] < 2) n[d] = 2;
    }
    const size_t pts = (size_t)n[0] * n[1] * n[2];
    const size_t bytes = pts * pk->prm.n_types * sizeof(float);
    if (pts > (size_t)1 << 31) return fail(TRIDS_EINVAL, "map grid of %zu points is too large", pts);
    float* d = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) return fail(TRIDS_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
    DevPocket v = pk->view();
    v.mx = n[0]; v.my = n[1]; v.mz = n[2];
    for (int k = 0; k < 3; ++k) v.mlo[k] = lo[k];
    v.mh = spacing;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (int)std::min<size_t>((pts + 255) / 256, (size_t)n_sms(pk->device) * 16);
    switch (pk->prm.term_set) {
    case TRIDS_TERMS_TRIDS: k_build_maps<TRIDS_TERMS_TRIDS><<<blocks, 256, 0, st>>>(v, pk->d_params, d); break;
    case TRIDS_TERMS_TRIDS_RES: k_build_maps<TRIDS_TERMS_TRIDS_RES><<<blocks, 256, 0, st>>>(v, pk->d_params, d); break;
    default: k_build_maps<TRIDS_TERMS_VINA5><<<blocks, 256, 0, st>>>(v, pk->d_params, d); break;
    }
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
        cudaFree(d);
        return fail(TRIDS_ECUDA, "map build launch: %s", cudaGetErrorString(le));
    }
    if (pk->d_maps) {
        CK(cudaDeviceSynchronize());
        cudaFree(pk->d_maps);
    }
    pk->d_maps = d;
    for (int k = 0; k < 3; ++k) { pk->mdims[k] = n[k]; pk->mlo[k] = lo[k]; }
    pk->mh = spacing;
    pk->maps_stale = false;
    return TRIDS_OK;
}

int trids_maps_info(const trids_pocket* pk, float lo[3], float* spacing, int32_t dims[3]) {
    g_err.clear();
    if (!pk || !lo || !spacing || !dims) return fail(TRIDS_EINVAL, "NULL argument");
    for (int d = 0; d < 3; ++d) { lo[d] = pk->mlo[d]; dims[d] = pk->mdims[d]; }
    *spacing = pk->mh;
    return TRIDS_OK;
}

int trids_pack_topology(int32_t n_atoms, const float* xyz, const int32_t* type, int32_t n_types, int32_t n_bonds,
                        const int32_t* bonds, const uint8_t* rotatable, int32_t* topo, int32_t topo_cap,
                        int32_t* topo_len) {
    g_err.clear();
    if (!xyz || !type || (n_bonds > 0 && (!bonds || !rotatable)) || !topo)
        return fail(TRIDS_EINVAL, "NULL input array");
    if (n_types < 1 || n_types > kNT) return fail(TRIDS_EINVAL, "n_types outside 1..%d", kNT);
    PackedLigand lg;
    std::string m = pack_ligand(n_atoms, xyz, type, n_types, n_bonds, bonds, rotatable, &lg);
    if (!m.empty()) return fail(TRIDS_EINVAL, "%s", m.c_str());
    std::vector<int32_t> v;
    topology_ints(lg, &v);
    if ((int)v.size() > topo_cap) return fail(TRIDS_EINVAL, "topology needs %zu ints", v.size());
    std::copy(v.begin(), v.end(), topo);
    if (topo_len) *topo_len = (int32_t)v.size();
    return TRIDS_OK;
}

// Packs every ligand on host threads (torsion tree, intra pairs and partner lists), lays
// the batch's device arrays out in one host staging buffer (each ligand fills its own
// slices, again on host threads) and uploads it with one allocation and one copy.
int trids_pack_ligands(const trids_pocket* pk, int32_t n_lig, const int32_t* n_atoms, const float* xyz,
                       const int32_t* type, const int32_t* n_bonds, const int32_t* bonds,
                       const uint8_t* rotatable, trids_batch** out) {
    g_err.clear();
    if (!out) return fail(TRIDS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!pk) return fail(TRIDS_EINVAL, "pocket is NULL");
    if (n_lig < 1) return fail(TRIDS_EINVAL, "n_lig must be >= 1");
    if (!n_atoms || !xyz || !type || !n_bonds) return fail(TRIDS_EINVAL, "NULL input array");
    int rc = device_guard(pk->device);
    if (rc) return rc;
    std::unique_ptr<trids_batch> b(new trids_batch());
    b->device = pk->device;
    b->n_types = pk->prm.n_types;
    b->ligs.resize(n_lig);
    std::vector<size_t> aoff(n_lig + 1, 0), boff(n_lig + 1, 0);
    int Lmax = 1;
    for (int l = 0; l < n_lig; ++l) {
        if (n_bonds[l] < 0) return fail(TRIDS_EINVAL, "ligand %d: negative bond count", l);
        if (n_bonds[l] > 0 && (!bonds || !rotatable)) return fail(TRIDS_EINVAL, "bonds is NULL");
        if (n_atoms[l] < 0) return fail(TRIDS_EINVAL, "ligand %d: negative atom count", l);
        aoff[l + 1] = aoff[l] + (size_t)n_atoms[l];
        boff[l + 1] = boff[l] + (size_t)n_bonds[l];
        Lmax = std::max(Lmax, (int)n_atoms[l]);
    }
    // 1. torsion trees and partner lists (the first failing ligand in index order is reported)
    std::vector<std::string> msg(n_lig);
    std::vector<std::vector<int>> lpre(n_lig);
    std::vector<std::vector<uint16_t>> lent(n_lig);
    for_ligands(n_lig, [&](int l) {
        msg[l] = pack_ligand(n_atoms[l], xyz + 3 * aoff[l], type + aoff[l], pk->prm.n_types, n_bonds[l],
                             bonds ? bonds + 2 * boff[l] : nullptr, rotatable ? rotatable + boff[l] : nullptr,
                             &b->ligs[l]);
        if (msg[l].empty()) partner_lists(b->ligs[l], Lmax, &lpre[l], &lent[l]);
    });
    int Tmax = 0;
    int64_t npairs = 0;
    std::vector<int64_t> toff(n_lig + 1, 0), poff(n_lig + 1, 0), eoff(n_lig + 1, 0);
    for (int l = 0; l < n_lig; ++l) {
        if (!msg[l].empty()) return fail(TRIDS_EINVAL, "ligand %d: %s", l, msg[l].c_str());
        Tmax = std::max(Tmax, b->ligs[l].n_tor);
        npairs += (int64_t)b->ligs[l].pairs.size();
        toff[l + 1] = toff[l] + b->ligs[l].n_tor;
        poff[l + 1] = poff[l] + n_atoms[l] + 1;
        eoff[l + 1] = eoff[l] + (int64_t)lent[l].size();
    }
    if ((int64_t)aoff[n_lig] > INT32_MAX || poff[n_lig] > INT32_MAX || eoff[n_lig] > INT32_MAX)
        return fail(TRIDS_EINVAL, "batch too large: split it (more than 2^31 atoms or partner entries)");
    b->dims.n_lig = n_lig;
    b->dims.max_atoms = Lmax;
    b->dims.max_tor = Tmax;
    b->dims.dof_stride = 7 + Tmax;
    b->dims.state_fields = state_fields(Tmax);
    b->dims.n_intra = npairs;
    // 2. device layout: one buffer of 256-byte aligned sections
    const size_t A = aoff[n_lig], T = (size_t)toff[n_lig], P = (size_t)poff[n_lig], E = (size_t)eoff[n_lig];
    size_t total = 0;
    auto section = [&](size_t bytes) {
        const size_t o = total;
        total = align_up(o + bytes, 256);
        return o;
    };
    const size_t o_hdr = section(sizeof(LigHdr) * n_lig), o_ay = section(sizeof(float4) * A),
                 o_orig = section(sizeof(int) * A), o_tidx = section(sizeof(int4) * T),
                 o_tu = section(sizeof(float4) * T), o_tp = section(sizeof(float4) * T), o_ipre = section(sizeof(int) * P),
                 o_ient = section(sizeof(uint16_t) * E), o_mask = section(sizeof(uint32_t) * A),
                 o_order = section(sizeof(int) * n_lig), o_cnt = section(4 * sizeof(unsigned int)),
                 o_err = section(2 * sizeof(int));
    std::vector<unsigned char> stage(total, 0);
    unsigned char* hs = stage.data();
    b->hdr.resize(n_lig);
    b->ient_j.resize(E);
    b->ient_type.resize(E);
    // 3. each ligand's slices (atoms about the root centroid, torsions, partner lists)
    for_ligands(n_lig, [&](int l) {
        const PackedLigand& lg = b->ligs[l];
        LigHdr h{};
        h.n_atoms = lg.n_atoms;
        h.n_tor = lg.n_tor;
        h.atom_off = (int)aoff[l];
        h.tor_off = (int)toff[l];
        h.ipre_off = (int)poff[l];
        h.ient_off = (int)eoff[l];
        h.n_pairs = (int)lg.pairs.size();
        h.sid = l;
        b->hdr[l] = h;
        const float* X = xyz + 3 * aoff[l];
        const int32_t* Ty = type + aoff[l];
        float4* ay = reinterpret_cast<float4*>(hs + o_ay) + aoff[l];
        int* orig = reinterpret_cast<int*>(hs + o_orig) + aoff[l];
        uint32_t* amask = reinterpret_cast<uint32_t*>(hs + o_mask) + aoff[l];
        for (int i = 0; i < lg.n_atoms; ++i) {
            const int a = lg.perm[i];
            float tb;
            const int t = Ty[a];
            std::memcpy(&tb, &t, 4);
            ay[i] = make_float4((float)((double)X[3 * a] - lg.c[0]), (float)((double)X[3 * a + 1] - lg.c[1]),
                                (float)((double)X[3 * a + 2] - lg.c[2]), tb);
            orig[i] = a;
            uint32_t m = 0;
            for (int k = lg.frag[i] - 1; k >= 0; k = lg.tpar[k]) m |= 1u << k;
            amask[i] = m;
        }
        int4* tidx = reinterpret_cast<int4*>(hs + o_tidx) + toff[l];
        float4* tu = reinterpret_cast<float4*>(hs + o_tu) + toff[l];
        float4* tp = reinterpret_cast<float4*>(hs + o_tp) + toff[l];
        for (int k = 0; k < lg.n_tor; ++k) {
            const int pa = lg.perm[lg.tp[k]], ha = lg.perm[lg.th[k]];
            double u[3], nn = 0;
            for (int d = 0; d < 3; ++d) {
                u[d] = (double)X[3 * ha + d] - (double)X[3 * pa + d];
                nn += u[d] * u[d];
            }
            nn = std::sqrt(nn);
            if (!(nn > 1e-6)) {
                char buf[96];
                std::snprintf(buf, sizeof buf, "rotatable bond %d has zero length", k);
                msg[l] = buf;
                return;
            }
            tidx[k] = make_int4(lg.tp[k], lg.th[k], lg.sb[k], lg.se[k]);
            tu[k] = make_float4((float)(u[0] / nn), (float)(u[1] / nn), (float)(u[2] / nn), 0.f);
            tp[k] = make_float4((float)((double)X[3 * pa] - lg.c[0]), (float)((double)X[3 * pa + 1] - lg.c[1]),
                                (float)((double)X[3 * pa + 2] - lg.c[2]), 0.f);
        }
        std::memcpy(reinterpret_cast<int*>(hs + o_ipre) + poff[l], lpre[l].data(), sizeof(int) * lpre[l].size());
        uint16_t* ient = reinterpret_cast<uint16_t*>(hs + o_ient) + eoff[l];
        for (size_t k = 0; k < lent[l].size(); ++k) {
            const int j = lent[l][k];
            const uint8_t ty = j == Lmax ? (uint8_t)0xff : (uint8_t)Ty[lg.perm[j]];
            const uint32_t f = ty == 0xff ? 0u : (uint32_t)(pk->prm.flags[ty] & 7);
            b->ient_j[eoff[l] + k] = (uint16_t)j;
            b->ient_type[eoff[l] + k] = ty;
            ient[k] = (uint16_t)((uint32_t)j | (f << 13));
        }
    });
    for (int l = 0; l < n_lig; ++l)
        if (!msg[l].empty()) return fail(TRIDS_EINVAL, "ligand %d: %s", l, msg[l].c_str());
    std::memcpy(hs + o_hdr, b->hdr.data(), sizeof(LigHdr) * n_lig);
    b->lig_order_h = lig_cost_order(b->hdr);
    std::memcpy(hs + o_order, b->lig_order_h.data(), sizeof(int) * n_lig);
    // 4. one allocation (a pooled block of a freed batch if one fits), one copy (a private
    // non-blocking stream: the copy neither waits for nor stalls kernels on other streams)
    b->d_block = pool_take(pk->device, total, &b->block_bytes);
    if (!b->d_block) {
        if (cudaMalloc(&b->d_block, total) != cudaSuccess) {
            b->d_block = nullptr;
            trids_free_batch(b.release());
            return fail(TRIDS_ENOMEM, "cudaMalloc of %zu bytes failed", total);
        }
        b->block_bytes = total;
    }
    {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            trids_free_batch(b.release());
            return fail(TRIDS_ECUDA, "cudaStreamCreateWithFlags failed");
        }
        cudaError_t e = cudaMemcpyAsync(b->d_block, hs, total, cudaMemcpyHostToDevice, s);
        cudaError_t e2 = cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            trids_free_batch(b.release());
            return fail(TRIDS_ECUDA, "upload failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
    }
    unsigned char* d = b->d_block;
    b->d_lig = reinterpret_cast<LigHdr*>(d + o_hdr);
    b->d_atom_y = reinterpret_cast<float4*>(d + o_ay);
    b->d_atom_orig = reinterpret_cast<int*>(d + o_orig);
    b->d_tor_idx = reinterpret_cast<int4*>(d + o_tidx);
    b->d_tor_u = reinterpret_cast<float4*>(d + o_tu);
    b->d_tor_p = reinterpret_cast<float4*>(d + o_tp);
    b->d_ipre = reinterpret_cast<int*>(d + o_ipre);
    b->d_ient = reinterpret_cast<uint16_t*>(d + o_ient);
    b->d_atom_mask = reinterpret_cast<uint32_t*>(d + o_mask);
    b->d_lig_order = reinterpret_cast<int*>(d + o_order);
    if (cudaEventCreateWithFlags(&b->ev_use, cudaEventDisableTiming) != cudaSuccess) {
        b->ev_use = nullptr;
        trids_free_batch(b.release());
        return fail(TRIDS_ECUDA, "cudaEventCreateWithFlags failed");
    }
    b->d_counter = reinterpret_cast<unsigned int*>(d + o_cnt);
    b->d_err = reinterpret_cast<int*>(d + o_err);
    b->dims.upload_bytes = (int64_t)total;
    b->owner = const_cast<trids_pocket*>(pk);
    b->owner->batches.push_back(b.get());
    *out = b.release();
    return TRIDS_OK;
}

int trids_free_batch(trids_batch* b) {
    if (!b) return TRIDS_OK;
    if (b->owner) {
        auto& v = b->owner->batches;
        v.erase(std::remove(v.begin(), v.end(), b), v.end());
    }
    if (b->side) cudaStreamDestroy(b->side);
    if (b->ev_a) cudaEventDestroy(b->ev_a);
    if (b->ev_b) cudaEventDestroy(b->ev_b);
    if (b->d_block) {   // every packed array, the ligand order, the pop counter and the error words
        int cur = -1;
        if (cudaGetDevice(&cur) == cudaSuccess && cur != b->device) cudaSetDevice(b->device);
        // the batch's last recorded work must be done before a new batch may take its block
        const cudaError_t e = b->ev_use ? cudaEventSynchronize(b->ev_use) : cudaSuccess;
        if (e == cudaSuccess) pool_give(b->device, b->d_block, b->block_bytes);
        else cudaFree(b->d_block);
    }
    if (b->ev_use) cudaEventDestroy(b->ev_use);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_partials) cudaFree(b->d_partials);
    if (b->d_mdn) cudaFree(b->d_mdn);
    delete b;
    return TRIDS_OK;
}

int trids_set_mdn(trids_batch* b, int32_t n_res, int32_t K, const float* mdn, void* stream) {
    g_err.clear();
    UseMark use_mark(b, stream);   // the batch's last work, for trids_free_batch
    if (!b) return fail(TRIDS_EINVAL, "batch is NULL");
    if (n_res < 1 || n_res > TRIDS_MAX_RESIDUES) return fail(TRIDS_EINVAL, "n_res %d outside 1..%d", n_res, TRIDS_MAX_RESIDUES);
    if (K < 1 || K > TRIDS_MAX_MDN_K) return fail(TRIDS_EINVAL, "K %d outside 1..%d", K, TRIDS_MAX_MDN_K);
    int rc = device_guard(b->device);
    if (rc) return rc;
    if ((rc = check_device_ptr(mdn, "mdn", false))) return rc;
    std::vector<int> in_row;
    for (int l = 0; l < b->dims.n_lig; ++l)
        for (int i = 0; i < b->ligs[l].n_atoms; ++i) in_row.push_back(b->hdr[l].atom_off + b->ligs[l].perm[i]);
    const int64_t rows = (int64_t)in_row.size(), RK = (int64_t)n_res * K;
    float4* d_out = nullptr;
    int* d_row = nullptr;
    int* d_bad = nullptr;
    const size_t bytes = (size_t)(rows * RK) * sizeof(float4);
    if (cudaMalloc(&d_out, bytes) != cudaSuccess) return fail(TRIDS_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
    std::vector<int> zero(1, 0);
    if ((rc = upload(&d_row, in_row)) || (rc = upload(&d_bad, zero))) {
        cudaFree(d_out); cudaFree(d_row); cudaFree(d_bad);
        return rc;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = rows * RK;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 32);
    k_mdn_pack<<<blocks, 256, 0, st>>>(mdn, d_row, rows, (int)RK, d_out, d_bad);
    cudaError_t le = cudaGetLastError();
    int bad = 0;
    cudaError_t ce = le == cudaSuccess ? cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st) : le;
    cudaError_t se = cudaStreamSynchronize(st);
    cudaFree(d_row);
    cudaFree(d_bad);
    if (ce != cudaSuccess || se != cudaSuccess) {
        cudaFree(d_out);
        return fail(TRIDS_ECUDA, "kernel conversion failed: %s", cudaGetErrorString(ce != cudaSuccess ? ce : se));
    }
    if (bad) {
        cudaFree(d_out);
        return fail(TRIDS_EINVAL, "mdn holds non-finite values or sigma <= 0");
    }
    cudaFree(b->d_mdn);
    b->d_mdn = d_out;
    b->mdn_res = n_res;
    b->mdn_k = K;
    return TRIDS_OK;
}

int trids_set_stream_ids(trids_batch* b, const int32_t* ids) {
    g_err.clear();
    if (!b || !ids) return fail(TRIDS_EINVAL, "NULL argument");
    for (int l = 0; l < b->dims.n_lig; ++l)
        if (ids[l] < 0) return fail(TRIDS_EINVAL, "stream id of ligand %d is negative", l);
    int rc = device_guard(b->device);
    if (rc) return rc;
    std::vector<LigHdr> hdr = b->hdr;
    for (int l = 0; l < b->dims.n_lig; ++l) hdr[l].sid = ids[l];
    CK(cudaMemcpy(b->d_lig, hdr.data(), hdr.size() * sizeof(LigHdr), cudaMemcpyHostToDevice));
    b->hdr = hdr;
    return TRIDS_OK;
}

int trids_batch_info(const trids_batch* b, trids_batch_dims* dims) {
    if (!b || !dims) return fail(TRIDS_EINVAL, "NULL argument");
    *dims = b->dims;
    return TRIDS_OK;
}

int trids_batch_query(const trids_batch* b, int32_t* n_tor, int32_t* n_atoms, int32_t lig, int32_t* topo,
                      int32_t topo_cap) {
    g_err.clear();
    if (!b) return fail(TRIDS_EINVAL, "batch is NULL");
    for (int l = 0; l < b->dims.n_lig; ++l) {
        if (n_tor) n_tor[l] = b->ligs[l].n_tor;
        if (n_atoms) n_atoms[l] = b->ligs[l].n_atoms;
    }
    if (topo) {
        if (lig < 0 || lig >= b->dims.n_lig) return fail(TRIDS_EINVAL, "ligand %d out of range", lig);
        std::vector<int32_t> v;
        topology_ints(b->ligs[lig], &v);
        if ((int)v.size() > topo_cap) return fail(TRIDS_EINVAL, "topology needs %zu ints", v.size());
        std::copy(v.begin(), v.end(), topo);
    }
    return TRIDS_OK;
}

int64_t trids_state_floats(const trids_batch* b, int32_t poses) {
    if (!b || poses < 1) return 0;
    return (int64_t)b->dims.n_lig * poses * b->dims.state_fields;
}

int trids_score_grad(const trids_pocket* pk, const trids_batch* bc, int32_t poses, const float* dof, float* energy,
                     float* e_inter, float* g_dof, float* g_xyz, const float* e_bar, float* g_w, float* g_radius,
                     void* stream) {
    g_err.clear();
    UseMark use_mark(bc, stream);   // the batch's last work, for trids_free_batch
    trids_batch* b = const_cast<trids_batch*>(bc);
    if (!pk || !b) return fail(TRIDS_EINVAL, "pocket or batch is NULL");
    if (pk->device != b->device) return fail(TRIDS_EINVAL, "pocket and batch live on different devices");
    if (poses < 1) return fail(TRIDS_EINVAL, "poses must be >= 1");
    int rc = device_guard(pk->device);
    if (rc) return rc;
    if ((rc = check_device_ptr(dof, "dof", false)) || (rc = check_device_ptr(energy, "energy", false)) ||
        (rc = check_device_ptr(e_inter, "e_inter", true)) || (rc = check_device_ptr(g_dof, "g_dof", true)) ||
        (rc = check_device_ptr(g_xyz, "g_xyz", true)) || (rc = check_device_ptr(e_bar, "e_bar", true)) ||
        (rc = check_device_ptr(g_w, "g_w", true)) || (rc = check_device_ptr(g_radius, "g_radius", true)) ||
        (rc = check_terms(pk, b)))
        return rc;
    if ((rc = ensure_items(b, poses))) return rc;
    const bool params = g_w || g_radius;
    if (params && pk->d_maps)
        return fail(TRIDS_EINVAL, "parameter gradients need direct scoring: free the grid maps first");
    if (params) {
        const size_t need = (size_t)b->n_items * (5 + kNT);
        if (need > b->partials_cap) {
            cudaFree(b->d_partials);
            b->d_partials = nullptr;
            if (cudaMalloc(&b->d_partials, need * sizeof(float)) != cudaSuccess)
                return fail(TRIDS_ENOMEM, "cudaMalloc of parameter partials failed");
            b->partials_cap = need;
        }
    }
    Layout L;
    const int warps = pick_warps(8, pk, b, params, &L);
    if (!warps) return fail(TRIDS_EINVAL, "pocket of %d atoms does not fit in shared memory", pk->M);
    ScoreArgs A;
    std::memset(&A, 0, sizeof A);
    A.pk = pk->view(); A.B = b->view(); A.P = poses; A.dof = dof; A.energy = energy; A.e_inter = e_inter;
    A.g_dof = g_dof; A.g_xyz = g_xyz; A.e_bar = e_bar; A.partials = b->d_partials; A.items = b->d_items;
    A.n_items = b->n_items; A.counter = b->d_counter + 1; A.err = b->d_err;
    A.params_bytes = L.params_bytes; A.pocket_off = L.pocket_off; A.ptype_off = L.ptype_off;
    A.mbar_off = L.mbar_off;
    A.warp_off = L.warp_off; A.warp_bytes = L.warp_bytes;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemsetAsync(A.counter, 0, sizeof(unsigned int), st));
    int grid = 0;
    {
        const ScoreKernel kern = score_kernel(pk->prm.term_set, params);
        if ((rc = grid_for(kern, warps, L.total, pk->device, b->n_items, &grid))) return rc;
        kern<<<grid, 32 * warps, L.total, st>>>(A);
    }
    CK(cudaGetLastError());
    if (params) {
        k_reduce_params<<<1, 32, 0, st>>>(b->d_partials, b->n_items, g_w, g_radius, b->n_types);
        CK(cudaGetLastError());
    }
    return TRIDS_OK;
}

int trids_sample(const trids_pocket* pk, const trids_batch* bc, const trids_sample_cfg* cfg, float* dof, float* state,
                 float* energy, void* stream) {
    g_err.clear();
    UseMark use_mark(bc, stream);   // the batch's last work, for trids_free_batch
    trids_batch* b = const_cast<trids_batch*>(bc);
    if (!pk || !b || !cfg) return fail(TRIDS_EINVAL, "pocket, batch or cfg is NULL");
    if (pk->device != b->device) return fail(TRIDS_EINVAL, "pocket and batch live on different devices");
    const trids_sample_cfg& c = *cfg;
    if (c.poses < 1) return fail(TRIDS_EINVAL, "poses must be >= 1");
    if (c.steps < 1 || c.mc_loops < 1) return fail(TRIDS_EINVAL, "steps and mc_loops must be >= 1");
    if (c.step_begin < 0 || c.step_end > c.steps || c.step_begin >= c.step_end)
        return fail(TRIDS_EINVAL, "need 0 <= step_begin < step_end <= steps");
    if (!(c.lr > 0.f) || !std::isfinite(c.lr) || !(c.beta1 >= 0.f && c.beta1 < 1.f) ||
        !(c.beta2 >= 0.f && c.beta2 < 1.f) || !(c.eps > 0.f) || !std::isfinite(c.beta))
        return fail(TRIDS_EINVAL, "invalid Adam or Metropolis parameters");
    if (c.optimizer < TRIDS_OPT_ADAM || c.optimizer > TRIDS_OPT_SGD)
        return fail(TRIDS_EINVAL, "unknown optimizer %d", c.optimizer);
    if (!(c.weight_decay >= 0.f) || !std::isfinite(c.weight_decay) || !(c.momentum >= 0.f && c.momentum < 1.f) ||
        !(c.alpha >= 0.f && c.alpha < 1.f))
        return fail(TRIDS_EINVAL, "need weight_decay >= 0, 0 <= momentum < 1, 0 <= alpha < 1");
    if (c.mode != TRIDS_MODE_PERSISTENT && c.mode != TRIDS_MODE_PER_LIGAND)
        return fail(TRIDS_EINVAL, "unknown mode %d", c.mode);
    if (c.trace && (!c.trace_slot || c.n_trace < 1))
        return fail(TRIDS_EINVAL, "trace needs trace_slot and n_trace >= 1");
    int rc = device_guard(pk->device);
    if (rc) return rc;
    if ((rc = check_device_ptr(dof, "dof", false)) || (rc = check_device_ptr(state, "state", false)) ||
        (rc = check_device_ptr(energy, "energy", false)) || (rc = check_device_ptr(c.trace, "trace", true)) ||
        (rc = check_device_ptr(c.trace_slot, "trace_slot", true)) ||
        (rc = check_device_ptr(c.pair_count, "pair_count", true)) ||
        (rc = check_device_ptr(c.phase_cycles, "phase_cycles", true)) ||
        (rc = check_device_ptr(c.work_count, "work_count", true)) || (rc = check_terms(pk, b)))
        return rc;
    Layout L;
    const int ts = pk->prm.term_set;
    const bool cnt = c.pair_count != nullptr || c.phase_cycles != nullptr || c.work_count != nullptr;
    // the general kernels carry the other update rules, the grid maps and the two-term
    // flag evaluation; the plain ones (Adam, direct pair sums, no type both hydrophobic and
    // donor/acceptor: the paper's configuration) leave that code out
    bool dual = false;
    for (int t = 0; t < pk->prm.n_types; ++t)
        dual |= (pk->prm.flags[t] & 1) && (pk->prm.flags[t] & 6);
    const bool gen = c.optimizer != TRIDS_OPT_ADAM || pk->d_maps != nullptr || dual;
    const int wmax = sample_warps_max(ts, gen);
    const int warps = pick_warps(c.warps_per_block > 0 ? c.warps_per_block : wmax, pk, b, false, &L, wmax);
    if (!warps) return fail(TRIDS_EINVAL, "pocket of %d atoms does not fit in shared memory", pk->M);
    SampleArgs A;
    std::memset(&A, 0, sizeof A);  // padding too: the bytes are compared with the graph's last arguments
    A.pk = pk->view(); A.B = b->view(); A.P = c.poses; A.S = c.steps; A.step_begin = c.step_begin;
    A.step_end = c.step_end; A.Lmc = c.mc_loops; A.lr = c.lr; A.b1 = c.beta1; A.b2 = c.beta2; A.eps = c.eps;
    A.beta = c.beta; A.opt = c.optimizer; A.wd = c.weight_decay; A.momentum = c.momentum; A.alpha = c.alpha;
    A.seed = c.seed; A.lig_base = c.lig_base; A.dof = dof; A.state = state; A.energy = energy;
    A.trace = c.trace; A.trace_slot = c.trace_slot; A.n_trace = c.n_trace; A.pair_count = c.pair_count;
    A.phase_cycles = c.phase_cycles;
    A.work_count = c.work_count;
    A.lig_order = b->d_lig_order; A.n_items = b->dims.n_lig * c.poses; A.counter = b->d_counter; A.err = b->d_err;
    A.params_bytes = L.params_bytes; A.pocket_off = L.pocket_off; A.ptype_off = L.ptype_off;
    A.mbar_off = L.mbar_off;
    A.warp_off = L.warp_off; A.warp_bytes = L.warp_bytes;
    cudaStream_t st = (cudaStream_t)stream;
    if (c.mode == TRIDS_MODE_PER_LIGAND) {
        const StepKernel kern = step_kernel(ts, cnt, gen);
        CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total));
        const int blocks = (c.poses + warps - 1) / warps;
        for (int s = c.step_begin; s < c.step_end; ++s)
            for (int l = 0; l < b->dims.n_lig; ++l) kern<<<blocks, 32 * warps, L.total, st>>>(A, l, s);
        CK(cudaGetLastError());
        return TRIDS_OK;
    }
    const PersistentKernel kern = persistent_kernel(ts, cnt, gen);
    int grid = 0;
    if ((rc = grid_for(kern, warps, L.total, pk->device, A.n_items, &grid))) return rc;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cap));
    if (!c.use_graph || cap != cudaStreamCaptureStatusNone) {
        CK(cudaMemsetAsync(A.counter, 0, sizeof(unsigned int), st));
        kern<<<grid, 32 * warps, L.total, st>>>(A);
        CK(cudaGetLastError());
        return TRIDS_OK;
    }
    // CUDA graph (Sec. 4 item 2), kept on the pocket: built once per launch shape and
    // replayed; other arguments update its nodes.  The legacy default stream cannot carry
    // graph work ordered like a capture-free launch, so for it the graph runs on a side
    // stream ordered against the caller's by events.
    const bool legacy = st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread;
    if (legacy && !b->side) {
        CK(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&b->ev_a, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&b->ev_b, cudaEventDisableTiming));
    }
    cudaStream_t run = legacy ? b->side : st;
    GraphCache& G = const_cast<trids_pocket*>(pk)->graph;
    std::lock_guard<std::mutex> lock(G.mu);
    void* kargs[] = {&A};
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.func = reinterpret_cast<void*>(kern);
    kp.gridDim = dim3((unsigned)grid);
    kp.blockDim = dim3(32u * (unsigned)warps);
    kp.sharedMemBytes = (unsigned)L.total;
    kp.kernelParams = kargs;
    cudaMemsetParams mp;
    std::memset(&mp, 0, sizeof mp);
    mp.dst = A.counter;
    mp.value = 0;
    mp.elementSize = sizeof(unsigned int);
    mp.width = 1;
    mp.height = 1;
    const unsigned char* ab = reinterpret_cast<const unsigned char*>(&A);
    const bool same_shape = G.exec && G.func == kp.func && G.grid == grid && G.block == 32 * warps &&
                            G.smem == L.total;
    if (!same_shape) {
        G.clear();
        CK(cudaGraphCreate(&G.graph, 0));
        CK(cudaGraphAddMemsetNode(&G.reset, G.graph, nullptr, 0, &mp));
        CK(cudaGraphAddKernelNode(&G.launch, G.graph, &G.reset, 1, &kp));
        cudaError_t ie = cudaGraphInstantiate(&G.exec, G.graph, 0);
        if (ie != cudaSuccess) {
            G.clear();
            return fail(TRIDS_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
        }
        G.func = kp.func; G.grid = grid; G.block = 32 * warps; G.smem = L.total;
        G.counter = A.counter;
        G.args.assign(ab, ab + sizeof(SampleArgs));
        ++G.instantiations;
    } else if (G.counter != A.counter || G.args.size() != sizeof(SampleArgs) ||
               std::memcmp(G.args.data(), ab, sizeof(SampleArgs)) != 0) {
        if (G.counter != A.counter) CK(cudaGraphExecMemsetNodeSetParams(G.exec, G.reset, &mp));
        CK(cudaGraphExecKernelNodeSetParams(G.exec, G.launch, &kp));
        G.counter = A.counter;
        G.args.assign(ab, ab + sizeof(SampleArgs));
        ++G.updates;
    }
    if (!legacy) {
        CK(cudaGraphLaunch(G.exec, run));
        ++G.launches;
        return TRIDS_OK;
    }
    CK(cudaEventRecord(b->ev_a, st));
    CK(cudaStreamWaitEvent(run, b->ev_a, 0));
    CK(cudaGraphLaunch(G.exec, run));
    ++G.launches;
    CK(cudaEventRecord(b->ev_b, run));
    CK(cudaStreamWaitEvent(st, b->ev_b, 0));
    return TRIDS_OK;
}

int trids_graph_stats(const trids_pocket* pk, int64_t* instantiations, int64_t* updates, int64_t* launches) {
    g_err.clear();
    if (!pk) return fail(TRIDS_EINVAL, "pocket is NULL");
    GraphCache& G = const_cast<trids_pocket*>(pk)->graph;
    std::lock_guard<std::mutex> lock(G.mu);
    if (instantiations) *instantiations = G.instantiations;
    if (updates) *updates = G.updates;
    if (launches) *launches = G.launches;
    return TRIDS_OK;
}

int trids_topk(const trids_batch* b, int32_t poses, const float* energy, const float* dof, int32_t k, float rmsd,
               int32_t* idx, float* e_out, void* stream) {
    g_err.clear();
    UseMark use_mark(b, stream);   // the batch's last work, for trids_free_batch
    if (!b) return fail(TRIDS_EINVAL, "batch is NULL");
    if (poses < 1 || k < 1 || k > 64) return fail(TRIDS_EINVAL, "need poses >= 1 and 1 <= k <= 64");
    if (!(rmsd >= 0.f) || !std::isfinite(rmsd)) return fail(TRIDS_EINVAL, "rmsd must be finite and >= 0");
    int rc = device_guard(b->device);
    if (rc) return rc;
    if ((rc = check_device_ptr(energy, "energy", false)) || (rc = check_device_ptr(dof, "dof", false)) ||
        (rc = check_device_ptr(idx, "idx", false)) || (rc = check_device_ptr(e_out, "e_out", true)))
        return rc;
    const size_t smem = align_up((size_t)poses, 4) * sizeof(int) +
                        (size_t)(3 * kLmax + (size_t)k * 3 * kLmax + 8) * sizeof(float);
    if (smem > max_smem(b->device)) return fail(TRIDS_EINVAL, "too many poses for top-k");
    CK(cudaFuncSetAttribute(k_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_topk<<<b->dims.n_lig, 128, smem, (cudaStream_t)stream>>>(b->view(), poses, energy, dof, k, rmsd, idx, e_out);
    CK(cudaGetLastError());
    return TRIDS_OK;
}

int trids_screen_energy(const trids_pocket* pk, const trids_batch* b, int32_t poses, int32_t k,
                        const int32_t* idx, const float* e_inter, float* e_screen, void* stream) {
    g_err.clear();
    UseMark use_mark(b, stream);   // the batch's last work, for trids_free_batch
    if (!pk || !b) return fail(TRIDS_EINVAL, "pocket or batch is NULL");
    if (pk->device != b->device) return fail(TRIDS_EINVAL, "pocket and batch live on different devices");
    if (poses < 1 || k < 1) return fail(TRIDS_EINVAL, "need poses >= 1 and k >= 1");
    int rc = device_guard(b->device);
    if (rc) return rc;
    if ((rc = check_device_ptr(idx, "idx", false)) || (rc = check_device_ptr(e_inter, "e_inter", false)) ||
        (rc = check_device_ptr(e_screen, "e_screen", false)))
        return rc;
    const long long n = (long long)b->dims.n_lig * k;
    if (n > (long long)INT32_MAX * 256) return fail(TRIDS_EINVAL, "n_lig x k too large");
    if (n == 0) return TRIDS_OK;
    k_screen<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(b->view(), poses, k, idx, e_inter,
                                                                            pk->prm.w_tor, e_screen);
    CK(cudaGetLastError());
    return TRIDS_OK;
}

int trids_sync(const trids_batch* b, int32_t poses, const float* state, void* stream, double timeout_ms) {
    g_err.clear();
    UseMark use_mark(b, stream);   // the batch's last work, for trids_free_batch
    if (!b) return fail(TRIDS_EINVAL, "batch is NULL");
    int rc = device_guard(b->device);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (state) {
        CK(cudaMemsetAsync(b->d_err + 1, 0, sizeof(int), st));
        k_status<<<64, 256, 0, st>>>(state, b->dims.n_lig, poses, b->dims.state_fields, b->d_err + 1);
        CK(cudaGetLastError());
    }
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaStreamQuery(st);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return fail(TRIDS_ECUDA, "stream failed: %s", cudaGetErrorString(q));
        double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (timeout_ms > 0 && ms > timeout_ms) return fail(TRIDS_ETIMEOUT, "stream not done after %.1f ms", ms);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    int flags[2] = {0, 0};
    CK(cudaMemcpy(flags, b->d_err, sizeof flags, cudaMemcpyDeviceToHost));
    if (flags[0]) return fail(TRIDS_ECUDA, "shared-memory staging did not complete");
    if (state && flags[1]) return fail(TRIDS_ENONFINITE, "a pose produced a non-finite energy (status %d)", flags[1]);
    return TRIDS_OK;
}

// Id of the calling thread's current CUDA context (the device's primary context after
// device_guard), through driver entry points fetched at run time; 0 when they are not
// available.  A context gets a new id when it is created again (after cudaDeviceReset, say).
static unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

// Device address of g_noalloc_scratch for `dev` (current): looked up once per device and
// context with that device current (host code cannot use the symbol itself as a device
// address), and looked up again when the device's context has changed since, as after a
// cudaDeviceReset, when the old address would be stale.  Where the driver gives no
// context id, every call looks it up.
static int noalloc_scratch(int dev, unsigned char** out) {
    static std::mutex mu;
    static void* addr[256] = {};
    static unsigned long long ctx_of[256] = {};
    if (dev < 0 || dev >= 256) return fail(TRIDS_EINVAL, "device %d out of range", dev);
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev] || ctx_of[dev] != ctx || ctx == 0) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(TRIDS_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
        addr[dev] = p;
        ctx_of[dev] = ctx;
    }
    *out = static_cast<unsigned char*>(addr[dev]);
    return TRIDS_OK;
}

int trids_score_grad_noalloc(const trids_pocket* pk, const trids_batch* b, int32_t poses, const float* dof,
                             float* energy, float* e_inter, float* g_dof, float* g_xyz, const float* e_bar,
                             float* g_w, float* g_radius, void* stream) {
    g_err.clear();
    UseMark use_mark(b, stream);   // the batch's last work, for trids_free_batch
    if (!pk || !b) return fail(TRIDS_EINVAL, "pocket or batch is NULL");
    if (pk->device != b->device) return fail(TRIDS_EINVAL, "pocket and batch live on different devices");
    if (poses < 1) return fail(TRIDS_EINVAL, "poses must be >= 1");
    int rc = device_guard(pk->device);
    if (rc) return rc;
    if ((rc = check_device_ptr(dof, "dof", false)) || (rc = check_device_ptr(energy, "energy", false)) ||
        (rc = check_device_ptr(e_inter, "e_inter", true)) || (rc = check_device_ptr(g_dof, "g_dof", true)) ||
        (rc = check_device_ptr(g_xyz, "g_xyz", true)) || (rc = check_device_ptr(e_bar, "e_bar", true)) ||
        (rc = check_device_ptr(g_w, "g_w", true)) || (rc = check_device_ptr(g_radius, "g_radius", true)) ||
        (rc = check_terms(pk, b)))
        return rc;
    const bool params = g_w || g_radius;
    if (params && pk->d_maps)
        return fail(TRIDS_EINVAL, "parameter gradients need direct scoring: free the grid maps first");
    const int tiles = (poses + 31) / 32;
    const size_t n_items = (size_t)b->dims.n_lig * tiles;
    const size_t items_off = 256;
    const size_t partials_off = align_up(items_off + n_items * sizeof(int2), 256);
    const size_t need = params ? partials_off + n_items * (5 + kNT) * sizeof(float) : items_off + n_items * sizeof(int2);
    if (n_items > (size_t)INT32_MAX || need > kNoAllocScratchBytes)
        return fail(TRIDS_EINVAL,
                    "trids_score_grad_noalloc needs %zu bytes of static scratch for %d ligands x %d poses%s; "
                    "the limit is %zu bytes: split the batch or call trids_score_grad",
                    need, b->dims.n_lig, poses, params ? " with parameter gradients" : "", kNoAllocScratchBytes);
    unsigned char* scratch = nullptr;
    if ((rc = noalloc_scratch(pk->device, &scratch))) return rc;
    Layout L;
    const int warps = pick_warps(8, pk, b, params, &L);
    if (!warps) return fail(TRIDS_EINVAL, "pocket of %d atoms does not fit in shared memory", pk->M);
    ScoreArgs A;
    std::memset(&A, 0, sizeof A);
    A.pk = pk->view(); A.B = b->view(); A.P = poses; A.dof = dof; A.energy = energy; A.e_inter = e_inter;
    A.g_dof = g_dof; A.g_xyz = g_xyz; A.e_bar = e_bar;
    A.partials = reinterpret_cast<float*>(scratch + partials_off);
    A.items = reinterpret_cast<const int2*>(scratch + items_off);
    A.n_items = (int)n_items; A.counter = reinterpret_cast<unsigned int*>(scratch); A.err = b->d_err;
    A.params_bytes = L.params_bytes; A.pocket_off = L.pocket_off; A.ptype_off = L.ptype_off;
    A.mbar_off = L.mbar_off;
    A.warp_off = L.warp_off; A.warp_bytes = L.warp_bytes;
    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's contents: reset the counter, rewrite the items
    CK(cudaMemsetAsync(A.counter, 0, sizeof(unsigned int), st));
    k_items_natural<<<(int)((n_items + 255) / 256), 256, 0, st>>>(reinterpret_cast<int2*>(scratch + items_off),
                                                                  b->dims.n_lig, tiles);
    CK(cudaGetLastError());
    int grid = 0;
    {
        const ScoreKernel kern = score_kernel(pk->prm.term_set, params);
        if ((rc = grid_for(kern, warps, L.total, pk->device, (int)n_items, &grid))) return rc;
        kern<<<grid, 32 * warps, L.total, st>>>(A);
    }
    CK(cudaGetLastError());
    if (params) {
        k_reduce_params<<<1, 32, 0, st>>>(A.partials, (int)n_items, g_w, g_radius, b->n_types);
        CK(cudaGetLastError());
    }
    return TRIDS_OK;
}

}  // extern "C"
