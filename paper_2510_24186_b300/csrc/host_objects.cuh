// libtrids host side: the allocation-free scratch, the pocket and batch objects, uploads,
// parameter encoding, launch-shape helpers and kernel selection.  Included by trids.cu only.
#pragma once

// =============================================================== allocation-free scoring
// Scratch of trids_score_grad_noalloc: one statically sized device array per device
// that loads the library (kept until the process exits).  Layout: work counter at
// offset 0, item list at 256, parameter partials after it (256-aligned).
constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// =============================================================== host objects
// CUDA graph of the persistent sampler (Sec. 4 item 2: the repeated operators are kept
// on the GPU as a graph): a counter-reset node and one persistent-kernel node, built once
// per launch shape (kernel, grid, block, shared memory) and replayed.  A call with other
// arguments (seed, ligand ids, step range, buffers, another batch of the same shape)
// updates the two nodes of the executable graph in place instead of building a new one.
struct GraphCache {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t reset = nullptr, launch = nullptr;
    const void* func = nullptr;
    int grid = 0, block = 0;
    size_t smem = 0;
    std::vector<unsigned char> args;   // kernel arguments of the last launch
    const void* counter = nullptr;     // the reset node's target
    int64_t instantiations = 0, updates = 0, launches = 0;
    std::mutex mu;
    void clear() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        reset = launch = nullptr;
        func = nullptr;
        args.clear();
        counter = nullptr;
    }
};

struct trids_pocket {
    int device = 0;
    int M = 0;
    std::vector<float> xyz;            // storage order (grouped by residue after trids_set_residues)
    std::vector<int> type;
    std::vector<int> orig;             // storage index -> input index
    uint8_t* d_ptype = nullptr;
    std::vector<trids_batch*> batches;   // batches whose intra entries carry this pocket's flags
    float cutoff_built = 0.f;
    float cell = 1.f;
    int n_boxes = 1;
    float box_lo[kMaxBoxes][3], box_hi[kMaxBoxes][3];
    trids_params prm;
    DevParams hp;
    CandidateGrid grid;
    float4* d_atoms = nullptr;
    uint32_t* d_cell = nullptr;
    uint16_t* d_cand = nullptr;
    uint16_t* d_levels = nullptr;        // candidate-grid reach levels [ncell][kReachLevels]
    DevParams* d_params = nullptr;
    uint32_t* d_ncell = nullptr;         // near lists of the atom-pair E_MDN (term set 1)
    uint16_t* d_nlist = nullptr;
    uint16_t* d_nlevels = nullptr;
    float* d_maps = nullptr;             // grid maps [type][z][y][x]
    int mdims[3] = {0, 0, 0};
    float mlo[3] = {0.f, 0.f, 0.f}, mh = 0.f;
    bool maps_stale = false;             // parameters changed since the maps were built
    ResidueGrid rgrid;                   // residue-level E_MDN (term set 2)
    int32_t* d_res_start = nullptr;
    uint32_t* d_rcell = nullptr;
    uint32_t* d_rlist = nullptr;
    uint16_t* d_rlevels = nullptr;
    GraphCache graph;                    // the persistent sampler's CUDA graph
    DevPocket view() const {
        DevPocket v;
        v.atoms = d_atoms; v.ptype = d_ptype; v.cell_start = d_cell; v.cand = d_cand; v.params = d_params; v.M = M;
        v.cell_levels = d_levels;
        v.n_res = rgrid.n_res; v.res_start = d_res_start; v.rcell_start = d_rcell;
        v.rlist = d_rlist; v.rlevels = d_rlevels;
        v.ncell_start = d_ncell; v.nlist = d_nlist; v.nlevels = d_nlevels;
        {
            const float nc = std::min(kMdnCut, prm.cutoff);
            v.near_cut2 = nc * nc;
        }
        v.use_maps = d_maps != nullptr;
        v.mx = mdims[0]; v.my = mdims[1]; v.mz = mdims[2];
        for (int d = 0; d < 3; ++d) v.mlo[d] = mlo[d];
        v.mh = mh; v.inv_mh = mh > 0.f ? 1.f / mh : 0.f;
        v.maps = d_maps;
        v.nx = grid.dims[0]; v.ny = grid.dims[1]; v.nz = grid.dims[2];
        v.gx = grid.lo[0]; v.gy = grid.lo[1]; v.gz = grid.lo[2]; v.inv_h = 1.f / grid.h;
        v.n_boxes = n_boxes;
        for (int b = 0; b < kMaxBoxes; ++b)
            for (int d = 0; d < 3; ++d) { v.box_lo[b][d] = box_lo[b][d]; v.box_hi[b][d] = box_hi[b][d]; }
        return v;
    }
};

struct trids_batch {
    int device = 0;
    int n_types = 0;
    trids_batch_dims dims{};
    std::vector<PackedLigand> ligs;
    std::vector<LigHdr> hdr;
    unsigned char* d_block = nullptr;   // one allocation holding the arrays below up to d_err
    size_t block_bytes = 0;             // its capacity (a reused block may be larger than needed)
    std::vector<int> lig_order_h;       // ligands by decreasing cost (host copy of d_lig_order)
    LigHdr* d_lig = nullptr;
    float4* d_atom_y = nullptr;
    int* d_atom_orig = nullptr;
    int4* d_tor_idx = nullptr;
    float4* d_tor_u = nullptr;
    float4* d_tor_p = nullptr;
    int* d_ipre = nullptr;
    uint16_t* d_ient = nullptr;
    uint32_t* d_atom_mask = nullptr;
    std::vector<uint16_t> ient_j;     // intra partner lists: target index (pad = max_atoms)
    std::vector<uint8_t> ient_type;   // target type (for re-encoding flags)
    trids_pocket* owner = nullptr;    // pocket whose flags are encoded in d_ient
    // per-pose-count caches
    int items_P = -1;
    int2* d_items = nullptr;        // (ligand, first pose of a 32-pose tile), by decreasing cost
    int n_items = 0;
    int* d_lig_order = nullptr;     // ligands by decreasing cost (a section of d_block)
    unsigned int* d_counter = nullptr;   // [4]
    int* d_err = nullptr;                // [2]: staging timeout, status OR
    float* d_partials = nullptr;
    size_t partials_cap = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    cudaEvent_t ev_use = nullptr;   // recorded after each call's work on the batch (UseMark)
    float4* d_mdn = nullptr;        // residue-level E_MDN kernels, packed rows
    int mdn_res = 0, mdn_k = 0;
    DevBatch view() const {
        DevBatch v;
        v.n_lig = dims.n_lig; v.max_atoms = dims.max_atoms; v.max_tor = dims.max_tor;
        v.dof_stride = dims.dof_stride; v.n_fields = dims.state_fields;
        v.lig = d_lig; v.atom_y = d_atom_y; v.atom_orig = d_atom_orig; v.tor_idx = d_tor_idx;
        v.tor_u = d_tor_u; v.tor_p = d_tor_p; v.ipre = d_ipre; v.ient = d_ient;
        v.atom_mask = d_atom_mask;
        v.mdn = d_mdn; v.mdn_res = mdn_res; v.mdn_k = mdn_k;
        return v;
    }
};

namespace {

// Device copy of a host vector.  The copy goes through a private non-blocking stream so it
// does not wait for (or stall) kernels running on other streams, e.g. while the next
// batch of a screening stream is packed during sampling.
template <class T>
int upload(T** dst, const std::vector<T>& src) {
    size_t n = std::max<size_t>(src.size(), 1) * sizeof(T);
    if (cudaMalloc(dst, n) != cudaSuccess) return fail(TRIDS_ENOMEM, "cudaMalloc of %zu bytes failed", n);
    if (!src.empty()) {
        cudaStream_t s;
        CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        cudaError_t e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
        cudaError_t e2 = cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
        if (e != cudaSuccess || e2 != cudaSuccess)
            return fail(TRIDS_ECUDA, "upload failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    return TRIDS_OK;
}

int check_params(const trids_params* p) {
    if (!p) return fail(TRIDS_EINVAL, "params is NULL");
    if (p->term_set != TRIDS_TERMS_VINA5 && p->term_set != TRIDS_TERMS_TRIDS && p->term_set != TRIDS_TERMS_TRIDS_RES)
        return fail(TRIDS_EINVAL, "term_set %d unknown", p->term_set);
    if (p->n_types < 1 || p->n_types > kNT) return fail(TRIDS_EINVAL, "n_types %d outside 1..%d", p->n_types, kNT);
    if (!(p->cutoff > 0.f) || !std::isfinite(p->cutoff) || p->cutoff > 64.f)
        return fail(TRIDS_EINVAL, "cutoff must be in (0, 64]");
    for (int t = 0; t < 5; ++t)
        if (!std::isfinite(p->w[t])) return fail(TRIDS_EINVAL, "weight %d is not finite", t);
    for (int a = 0; a < p->n_types; ++a)
        if (!std::isfinite(p->radius[a]) || p->radius[a] < 0.f) return fail(TRIDS_EINVAL, "radius %d invalid", a);
    if (p->gmm_k < 0 || p->gmm_k > kK) return fail(TRIDS_EINVAL, "gmm_k %d outside 0..%d", p->gmm_k, kK);
    for (int a = 0; a < p->n_types; ++a)
        for (int b = 0; b < p->n_types; ++b)
            for (int k = 0; k < p->gmm_k; ++k) {
                const float* g = p->gmm[a][b][k];
                if (!std::isfinite(g[0]) || !std::isfinite(g[1]) || !(g[2] > 0.f) || !std::isfinite(g[2]))
                    return fail(TRIDS_EINVAL, "gmm[%d][%d][%d] invalid (sigma must be > 0)", a, b, k);
            }
    return TRIDS_OK;
}

void fill_dev_params(const trids_params* p, DevParams* d) {
    std::memset(d, 0, sizeof *d);
    d->term_set = p->term_set;
    d->n_types = p->n_types;
    d->gmm_k = p->gmm_k;
    for (int t = 0; t < 5; ++t) d->w[t] = p->w[t];
    d->cutoff = p->cutoff;
    d->cut2 = p->cutoff * p->cutoff;
    d->w_tor = p->w_tor;
    for (int a = 0; a < kNT; ++a) d->radius[a] = a < p->n_types ? p->radius[a] : 0.f;
    for (int a = 0; a < kNT; ++a) d->tflags[a] = a < p->n_types ? (uint32_t)(p->flags[a] & 7) : 0u;
    for (int a = 0; a < kNT; ++a) {
        // a hydrophobic type meets w3 sat(1.5 - d) with hydrophobic candidates; a donor and/or
        // acceptor type w4 sat(-d / 0.7) with candidates of the complementary flag
        const uint32_t f = d->tflags[a];
        const bool hyd = (f & 1u) != 0u;
        const uint32_t m = hyd ? (1u << 13) : ((((f & 2u) << 1) | ((f & 4u) >> 1)) << 13);
        float mb;
        std::memcpy(&mb, &m, 4);
        d->ftab[a] = make_float4(mb, hyd ? -1.f : -1.f / 0.7f, hyd ? 1.5f : 0.f, hyd ? p->w[3] : p->w[4]);
    }
    for (int a = 0; a < kNT; ++a)
        for (int b = 0; b < kNT; ++b) {
            const bool in = a < p->n_types && b < p->n_types;
            const int fa = in ? p->flags[a] : 0, fb = in ? p->flags[b] : 0;
            const int hyd = (fa & 1) && (fb & 1);
            const int hb = ((fa & 2) && (fb & 4)) || ((fa & 4) && (fb & 2));
            int bits = (hyd ? 1 : 0) | (hb ? 2 : 0);
            float rs = in ? p->radius[a] + p->radius[b] : 0.f;
            float fb_bits;
            std::memcpy(&fb_bits, &bits, 4);
            d->pairtab[a][b] = make_float2(rs, fb_bits);
            for (int k = 0; k < kK; ++k) {
                if (in && k < p->gmm_k) {
                    const float* g = p->gmm[a][b][k];
                    d->gmm[a][b][k] = make_float4(g[0], g[1], -kLog2e / (2.f * g[2] * g[2]), 1.f / (g[2] * g[2]));
                } else {
                    d->gmm[a][b][k] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
}

// Pocket arrays that depend on the parameters: atoms as (x, y, z, radius of the type)
// and candidate entries carrying each atom's flags.  Stream-ordered, then synchronised
// (the host staging vectors are temporaries).
int upload_pocket_arrays(trids_pocket* pk, cudaStream_t st) {
    const int M = pk->M;
    std::vector<float4> atoms(M + 1);
    for (int j = 0; j < M; ++j)
        atoms[j] = make_float4(pk->xyz[3 * j], pk->xyz[3 * j + 1], pk->xyz[3 * j + 2], pk->prm.radius[pk->type[j]]);
    atoms[M] = make_float4(1e6f, 1e6f, 1e6f, 0.f);  // sentinel: never within the cutoff
    std::vector<uint16_t> cand(pk->grid.cand.size());
    for (size_t k = 0; k < cand.size(); ++k) {
        const int j = pk->grid.cand[k];
        const uint32_t f = j < M ? (uint32_t)(pk->prm.flags[pk->type[j]] & 7) : 0u;
        cand[k] = (uint16_t)((uint32_t)j | (f << 13));
    }
    fill_dev_params(&pk->prm, &pk->hp);
    CK(cudaMemcpyAsync(pk->d_atoms, atoms.data(), atoms.size() * sizeof(float4), cudaMemcpyHostToDevice, st));
    if (!cand.empty())
        CK(cudaMemcpyAsync(pk->d_cand, cand.data(), cand.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(pk->d_params, &pk->hp, sizeof(DevParams), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    return TRIDS_OK;
}

// Runs fn(l) for every ligand l in [0, n) on up to 32 host threads (ligands are independent).
template <class F>
void for_ligands(int n, F&& fn) {
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int nt = std::max(1, std::min({hw, 32, n / 16}));
    auto work = [&](int t) {
        for (int l = t; l < n; l += nt) fn(l);
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(work, t);
    work(0);
    for (auto& x : th) x.join();
}

// Intra partner lists of one packed ligand: per atom, every partner (both directions,
// ascending) in blocks of 8 padded with the far sentinel index pad; pre[i] is atom i's
// first block (n_atoms + 1 entries).
void partner_lists(const PackedLigand& lg, int pad, std::vector<int>* pre, std::vector<uint16_t>* ent) {
    const int n = lg.n_atoms;
    std::vector<int> deg(n + 1, 0);
    for (const auto& pr : lg.pairs) {
        ++deg[pr.first + 1];
        ++deg[pr.second + 1];
    }
    for (int i = 0; i < n; ++i) deg[i + 1] += deg[i];
    std::vector<int> adj(deg[n]), fill(deg.begin(), deg.end() - 1);
    for (const auto& pr : lg.pairs) {
        adj[fill[pr.first]++] = pr.second;
        adj[fill[pr.second]++] = pr.first;
    }
    pre->assign(n + 1, 0);
    for (int i = 0; i < n; ++i) (*pre)[i + 1] = (*pre)[i] + (deg[i + 1] - deg[i] + 7) / 8;
    ent->assign(8 * (size_t)(*pre)[n], (uint16_t)pad);
    for (int i = 0; i < n; ++i) {
        std::sort(adj.begin() + deg[i], adj.begin() + deg[i + 1]);
        for (int k = deg[i]; k < deg[i + 1]; ++k) (*ent)[8 * (size_t)(*pre)[i] + (k - deg[i])] = (uint16_t)adj[k];
    }
}

// (Re-)encode a batch's intra partner entries with the pocket's current type flags.
int encode_intra(const trids_pocket* pk, trids_batch* b) {
    std::vector<uint16_t> ent(b->ient_j.size());
    for (size_t k = 0; k < ent.size(); ++k) {
        const uint32_t f = b->ient_type[k] == 0xff ? 0u : (uint32_t)(pk->prm.flags[b->ient_type[k]] & 7);
        ent[k] = (uint16_t)((uint32_t)b->ient_j[k] | (f << 13));
    }
    if (!ent.empty()) CK(cudaMemcpy(b->d_ient, ent.data(), ent.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    return TRIDS_OK;
}

int device_guard(int dev) {
    int cur = -1;
    CK(cudaGetDevice(&cur));
    if (cur != dev) CK(cudaSetDevice(dev));
    return TRIDS_OK;
}

// Ligands by decreasing estimated cost (atoms, intra pairs, torsions; ties by index): the
// order in which the persistent sampler pops them and the scorer's items run.
std::vector<int> lig_cost_order(const std::vector<LigHdr>& hdr) {
    std::vector<std::pair<double, int>> lc(hdr.size());
    for (size_t l = 0; l < hdr.size(); ++l) {
        const LigHdr& h = hdr[l];
        lc[l] = {60.0 * h.n_atoms + 2.0 * h.n_pairs + 20.0 * h.n_tor + 10.0, (int)l};
    }
    std::stable_sort(lc.begin(), lc.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& c) {
        return a.first > c.first;
    });
    std::vector<int> order(lc.size());
    for (size_t i = 0; i < lc.size(); ++i) order[i] = lc[i].second;
    return order;
}

// The scorer's (ligand, 32-pose tile) items for P poses, ligands by decreasing cost.
int ensure_items(trids_batch* b, int P) {
    if (b->items_P == P) return TRIDS_OK;
    const int tiles = (P + 31) / 32;
    std::vector<int2> items;
    items.reserve((size_t)b->dims.n_lig * tiles);
    for (int l : b->lig_order_h)
        for (int t = 0; t < tiles; ++t) items.push_back(make_int2(l, t * 32));
    cudaFree(b->d_items);
    b->d_items = nullptr;
    int rc = upload(&b->d_items, items);
    if (rc) return rc;
    b->n_items = (int)items.size();
    b->items_P = P;
    return TRIDS_OK;
}

// Records the batch's use event on the call's stream when the entry point returns (whatever
// it launched), so that trids_free_batch waits for the batch's last work before it pools the
// batch's memory.
struct UseMark {
    const trids_batch* b;
    cudaStream_t st;
    UseMark(const trids_batch* b_, void* stream) : b(b_), st((cudaStream_t)stream) {}
    ~UseMark() {
        if (b && b->ev_use) cudaEventRecord(b->ev_use, st);
    }
};

// Device blocks of freed batches, kept for the next batches of the same device: a stream of
// batches then allocates and frees its device memory once instead of once per batch.
// trids_free_batch waits for the batch's last recorded work before it pools a block, so no
// launch still reads a block that a new batch takes.  At most kPoolBlocks blocks stay
// pooled (the smallest goes first); they are released when the process exits.
constexpr size_t kPoolBlocks = 2;
struct BlockPool {
    struct Entry {
        int device;
        unsigned char* p;
        size_t bytes;
    };
    std::mutex mu;
    std::vector<Entry> free;
};
inline BlockPool& block_pool() {
    static BlockPool pool;
    return pool;
}

// A pooled block of the device with at least `bytes` (and at most 4 x bytes + 1 MiB, so a
// small batch does not pin a large block), or nullptr; *cap gets its size.
unsigned char* pool_take(int device, size_t bytes, size_t* cap) {
    BlockPool& P = block_pool();
    std::lock_guard<std::mutex> lock(P.mu);
    int at = -1;
    for (size_t k = 0; k < P.free.size(); ++k) {
        const BlockPool::Entry& e = P.free[k];
        if (e.device == device && e.bytes >= bytes && e.bytes <= 4 * bytes + (1u << 20) &&
            (at < 0 || e.bytes < P.free[at].bytes))
            at = (int)k;
    }
    if (at < 0) return nullptr;
    unsigned char* p = P.free[at].p;
    *cap = P.free[at].bytes;
    P.free.erase(P.free.begin() + at);
    return p;
}

// Pool a block of the current device (the caller has synchronized it).
void pool_give(int device, unsigned char* p, size_t bytes) {
    BlockPool& P = block_pool();
    std::lock_guard<std::mutex> lock(P.mu);
    P.free.push_back({device, p, bytes});
    size_t n_dev = 0;
    for (const BlockPool::Entry& e : P.free) n_dev += e.device == device;
    if (n_dev > kPoolBlocks) {   // drop this device's smallest block
        int at = -1;
        for (size_t k = 0; k < P.free.size(); ++k)
            if (P.free[k].device == device && (at < 0 || P.free[k].bytes < P.free[at].bytes)) at = (int)k;
        cudaFree(P.free[at].p);
        P.free.erase(P.free.begin() + at);
    }
}

int n_sms(int dev) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

size_t max_smem(int dev) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (size_t)v;
}

// Pick warps per block: the requested count (at most max_warps), capped so the block fits
// in shared memory.
int pick_warps(int requested, const trids_pocket* pk, const trids_batch* b, bool params, Layout* L,
               int max_warps = 20) {
    const size_t cap = max_smem(pk->device);
    int w = requested > 0 ? std::min(requested, max_warps) : 8;
    for (; w >= 1; --w) {
        *L = make_layout(pk->prm.term_set, pk->M, b->dims.max_atoms, b->dims.max_tor, w, params);
        if (L->total <= cap) return w;
    }
    return 0;
}

template <class K>
int grid_for(K kernel, int warps, size_t smem, int dev, int n_items, int* grid) {
    CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * warps, smem));
    if (per_sm < 1) return fail(TRIDS_EINVAL, "kernel does not fit on an SM (shared memory %zu bytes)", smem);
    const int need = (n_items + warps - 1) / warps;
    *grid = std::max(1, std::min(need, per_sm * n_sms(dev)));
    return TRIDS_OK;
}

int check_device_ptr(const void* p, const char* name, bool nullable) {
    if (!p) return nullable ? TRIDS_OK : fail(TRIDS_EINVAL, "%s is NULL", name);
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return fail(TRIDS_EINVAL, "%s is not a CUDA pointer", name);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(TRIDS_EINVAL, "%s must be device memory", name);
    return TRIDS_OK;
}

// Near lists of the atom-pair E_MDN on the pocket's current grid (storage order).
int upload_near_lists(trids_pocket* pk) {
    std::vector<uint32_t> start;
    std::vector<uint16_t> list, levels;
    build_near_lists(pk->M, pk->xyz.data(), std::min(kMdnCut, pk->cutoff_built), pk->grid, &start, &list, &levels);
    uint32_t* d_start = nullptr;
    uint16_t* d_list = nullptr;
    uint16_t* d_levels = nullptr;
    int rc;
    if ((rc = upload(&d_start, start)) || (rc = upload(&d_list, list)) || (rc = upload(&d_levels, levels))) {
        cudaFree(d_start);
        cudaFree(d_list);
        cudaFree(d_levels);
        return rc;
    }
    cudaFree(pk->d_ncell);
    cudaFree(pk->d_nlist);
    cudaFree(pk->d_nlevels);
    pk->d_ncell = d_start;
    pk->d_nlist = d_list;
    pk->d_nlevels = d_levels;
    return TRIDS_OK;
}

// Inputs a term set needs beyond the pocket and the batch.
int check_terms(const trids_pocket* pk, const trids_batch* b) {
    if (pk->d_maps && pk->maps_stale)
        return fail(TRIDS_EINVAL, "the grid maps predate trids_set_params: call trids_build_maps again");
    if (pk->prm.term_set != TRIDS_TERMS_TRIDS_RES) return TRIDS_OK;
    if (pk->rgrid.n_res < 1) return fail(TRIDS_EINVAL, "term set 2 needs trids_set_residues on the pocket");
    if (!b->d_mdn) return fail(TRIDS_EINVAL, "term set 2 needs trids_set_mdn on the batch");
    if (b->mdn_res != pk->rgrid.n_res)
        return fail(TRIDS_EINVAL, "batch kernels are for %d residues, the pocket has %d", b->mdn_res, pk->rgrid.n_res);
    return TRIDS_OK;
}

using PersistentKernel = void (*)(SampleArgs);
using StepKernel = void (*)(SampleArgs, int, int);
using ScoreKernel = void (*)(ScoreArgs);

template <int TS>
PersistentKernel persistent_for(bool cnt, bool gen) {
    return gen ? (cnt ? k_sample_persistent<TS, true, true> : k_sample_persistent<TS, false, true>)
                : (cnt ? k_sample_persistent<TS, true, false> : k_sample_persistent<TS, false, false>);
}
template <int TS>
StepKernel step_for(bool cnt, bool gen) {
    return gen ? (cnt ? k_sample_step<TS, true, true> : k_sample_step<TS, false, true>)
                : (cnt ? k_sample_step<TS, true, false> : k_sample_step<TS, false, false>);
}
template <int TS>
ScoreKernel score_for(bool params) { return params ? k_score<TS, true> : k_score<TS, false>; }

PersistentKernel persistent_kernel(int ts, bool cnt, bool gen) {
    return ts == TRIDS_TERMS_TRIDS ? persistent_for<TRIDS_TERMS_TRIDS>(cnt, gen)
         : ts == TRIDS_TERMS_TRIDS_RES ? persistent_for<TRIDS_TERMS_TRIDS_RES>(cnt, gen)
                                       : persistent_for<TRIDS_TERMS_VINA5>(cnt, gen);
}
StepKernel step_kernel(int ts, bool cnt, bool gen) {
    return ts == TRIDS_TERMS_TRIDS ? step_for<TRIDS_TERMS_TRIDS>(cnt, gen)
         : ts == TRIDS_TERMS_TRIDS_RES ? step_for<TRIDS_TERMS_TRIDS_RES>(cnt, gen)
                                       : step_for<TRIDS_TERMS_VINA5>(cnt, gen);
}
ScoreKernel score_kernel(int ts, bool params) {
    return ts == TRIDS_TERMS_TRIDS ? score_for<TRIDS_TERMS_TRIDS>(params)
         : ts == TRIDS_TERMS_TRIDS_RES ? score_for<TRIDS_TERMS_TRIDS_RES>(params)
                                       : score_for<TRIDS_TERMS_VINA5>(params);
}

// Residue-level E_MDN kernels: input rows (input atom order) -> packed rows as
// (pi, mu, -log2(e)/(2 sigma^2), 1/sigma^2), the exponent scaled for ex2; flags entries with
// non-finite values or sigma <= 0.
__global__ void k_mdn_pack(const float* __restrict__ in, const int* __restrict__ in_row, int64_t rows, int RK,
                           float4* __restrict__ out, int* bad) {
    const int64_t n = rows * RK;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / RK, rk = e - s * RK;
        const float* g = in + ((int64_t)in_row[s] * RK + rk) * 3;
        const float pi = g[0], mu = g[1], sg = g[2];
        if (!isfinite(pi) || !isfinite(mu) || !isfinite(sg) || !(sg > 0.f)) atomicOr(bad, 1);
        const float is2 = 1.f / (sg * sg);
        out[e] = make_float4(pi, mu, -0.5f * kLog2e * is2, is2);
    }
}

}  // namespace

