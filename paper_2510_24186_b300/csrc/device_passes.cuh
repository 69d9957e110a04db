// libtrids device code, part 2: the per-pose passes of one evaluation -- the balanced pair
// loop, the grid-map, atom-pair E_MDN and residue E_MDN passes, the score and the adjoint.
// Included by trids.cu only.
#pragma once

namespace {

// ------------------------------------------------------------------ balanced item loops
// The pair loop and the E_MDN passes number a pose's work items atom by atom and give
// lane k the k-th of 32 equal contiguous segments.  A lane accumulates its current atom's
// force in registers and leaves a partial in slot (atom + lane) of W.rec: slots are unique
// because atoms never decrease along the lanes.  The partials of an atom are then added in
// lane order, so the result does not depend on timing.

// Per-atom item counts -> exclusive prefix W.meta[0..L].w, 32 atoms per call: atom i =
// base + lane has n items (0 for i >= L); carry runs over the calls.  seg_finish then sets
// W.meta[0].w, clears W.rec and returns the total.
__device__ __forceinline__ void seg_scan(const PW& W, int L, int i, int n, int& carry) {
    const int lane = W.lane;
    int v = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    if (i < L) W.meta[i + 1].w = carry + v;
    carry += __shfl_sync(kFull, v, 31);
}

__device__ __forceinline__ int seg_finish(const PW& W, int L, int carry) {
    if (W.lane == 0) W.meta[0].w = 0;
    for (int r = W.lane; r < L + 32; r += 32) W.rec[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
    return carry;
}

// The lane's item range [lo, hi) of N items and the atom holding item lo (when lo < hi).
__device__ __forceinline__ int seg_range(const PW& W, int L, int N, int& lo, int& hi) {
    lo = (int)(((long long)N * W.lane) >> 5);
    hi = (int)(((long long)N * (W.lane + 1)) >> 5);
    int a = 0, b = L - 1;
    while (a < b) {
        const int m = (a + b + 1) >> 1;
        if (W.meta[m].w <= lo) a = m; else b = m - 1;
    }
    return a;
}

// Each atom's partials in lane order: W.gs[i] = sum (ADD: W.gs[i] += sum).
template <bool ADD>
__device__ __forceinline__ void seg_combine(const PW& W, int L, int N) {
    __syncwarp();
    for (int i = W.lane; i < L; i += 32) {
        float gx = 0.f, gy = 0.f, gz = 0.f;
        const int b0 = W.meta[i].w, b1 = W.meta[i + 1].w;
        if (b0 < b1) {
            const int l0 = min(31, (32 * (b0 + 1) - 1) / N), l1 = min(31, (32 * b1 - 1) / N);
            for (int l = l0; l <= l1; ++l) {
                const float4 r = W.rec[i + l];
                gx += r.x; gy += r.y; gz += r.z;
            }
        }
        if (ADD) {
            if (b0 < b1) {
                float4 g = W.gs[i];
                g.x += gx; g.y += gy; g.z += gz;
                W.gs[i] = g;
            }
        } else {
            W.gs[i] = make_float4(gx, gy, gz, 0.f);
        }
    }
    __syncwarp();
}

// All pairs of the warp's pose.  Atom i's work list is its cell's candidate pocket atoms
// followed by its intra-ligand partners (every intra pair appears once from each side),
// both in blocks of 8 uint16 entries (target index, 13 bits | target's flags << 13;
// padding points at a far sentinel).  Pocket targets are read from the block's staged
// pocket, ligand targets from the pose's own coordinates (W.xs); both float4 carry
// (x, y, z, radius).  The pose's blocks are numbered atom by atom (prefix in W.meta[].w) and
// split into 32 equal contiguous segments, one per lane, so the lanes stay balanced
// whatever the atoms' list lengths.  A lane accumulates the force on its current atom
// in registers and leaves a partial in slot (atom + lane) of W.rec; the partials of an
// atom are added in lane order (bit-reproducible).  The Vina-form block is branch-free:
// all candidates are evaluated and masked by r^2 < cutoff^2.  While the loop runs, W.gs
// holds each atom's negated (x, y, z, R), the packed evaluation's atom operands, so that a
// lane changing atom loads them ready-made.  Writes the forces to W.gs; returns the lane's
// ligand-pocket energy and, in *e_in2, twice its intra energy.
template <int TS, bool PARAMS, bool COUNT, bool MAPS>
__device__ float pairs_warp(const DevBatch& B, const DevPocket& pk, const Smem& S, const LigHdr& h, const PW& W,
                           const float w[5], float ebar, ParamAcc& acc, WorkCount& wc, float* e_in2) {
    const DevParams& P = *S.P;
    const float cut2 = P.cut2;
    const VinaX2 K = make_vina_x2(w);
    const int L = h.n_atoms, lane = W.lane;
    const uint16_t* __restrict__ cand = pk.cand;
    const uint16_t* __restrict__ ient = B.ient + h.ient_off;
    // 1. per-atom work: candidate blocks of the cell + intra-partner blocks; prefix
    int carry = 0;
    for (int base = 0; base < L; base += 32) {
        const int i = base + lane;
        int nblk = 0;
        if (i < L) {
            const float4 x = W.xs[i];
            W.gs[i] = make_float4(-x.x, -x.y, -x.z, -x.w);   // the packed pair's atom operands
            uint32_t beg;
            int nb;
            cell_levels(pk, pk.cell_start, pk.cell_levels, x.x, x.y, x.z, beg, nb);
            const int i0 = __ldg(&B.ipre[h.ipre_off + i]), i1 = __ldg(&B.ipre[h.ipre_off + i + 1]);
            const int cbk = (MAPS && map_cell(pk, x.x, x.y, x.z, nullptr)) ? 0 : nb;
            const int ty = __float_as_int(__ldg(&B.atom_y[h.atom_off + i]).w);
            W.meta[i].x = beg;
            W.meta[i].y = cbk | (int)((P.tflags[ty] & 7u) << 24) | (ty << 27);   // blocks | flags | type
            W.meta[i].z = i0;
            nblk = cbk + (i1 - i0);
        }
        seg_scan(W, L, i, nblk, carry);
    }
    const int N = seg_finish(W, L, carry);
    int lo, hi;
    int i = seg_range(W, L, N, lo, hi);
    float e_lp = 0.f, e_in = 0.f;
    if (lo < hi) {
        int first = W.meta[i].w, nxt = W.meta[i + 1].w, cbw = W.meta[i].y, ipb = W.meta[i].z;
        int cbk = cbw & 0xffffff, ti = cbw >> 27;
        uint32_t fi = (uint32_t)(cbw >> 24) & 7u;
        uint32_t csb = W.meta[i].x;
        float4 xa = W.xs[i];
        float ri = xa.w;
        // per-atom operands of the packed evaluation, set when the lane changes atom
        float2 nxy = make_float2(-xa.x, -xa.y), nzr = make_float2(-xa.z, -ri);
        // the plain Vina-form kernels take the single flag term from the type table; the two-term
        // form and the TRIDS terms (donor-acceptor bits) build the operands from the flags
        FlagTerm F = (MAPS || TS != TRIDS_TERMS_VINA5) ? make_flag_term(fi, P.w[3], P.w[4]) : flag_term_of(P.ftab[ti]);
        float ax = 0.f, ay = 0.f, az = 0.f;
        auto block_ptr = [&](int blk) -> const uint4* {
            const int loc = blk - first;
            return loc < cbk ? reinterpret_cast<const uint4*>(cand + csb + 8u * (uint32_t)loc)
                             : reinterpret_cast<const uint4*>(ient + 8 * (ipb + loc - cbk));
        };
        const uint4* pb = block_ptr(lo);          // address of the block held in v
        uint4 v = __ldg(pb);
        int icut = first + cbk;                   // the atom's first intra block
        const uint4* ib = reinterpret_cast<const uint4*>(ient + 8 * ipb);
        for (int blk = lo; blk < hi; ++blk) {
            if (blk == nxt) {                      // move to the atom owning block blk
                // the new atom's records are read before the old atom's partial is stored, so
                // that the search's last prefix read is the new nxt (no reload after the store)
                const int io = i;
                int nx;
                do { ++i; nx = W.meta[i + 1].w; } while (nx == blk);
                first = blk;                       // a lane enters an atom at its first block
                nxt = nx;
                const int4 mt = W.meta[i];             // (cell list, blocks | flags | type, intra list, prefix)
                W.rec[io + lane] = make_float4(ax, ay, az, 0.f);
                ax = ay = az = 0.f;
                cbw = mt.y;
                cbk = cbw & 0xffffff;
                ti = cbw >> 27;
                fi = (uint32_t)(cbw >> 24) & 7u;
                ipb = mt.z;
                csb = (uint32_t)mt.x;
                if constexpr (PARAMS) {
                    xa = W.xs[i];
                    ri = xa.w;
                }
                {
                    const float4 ng = W.gs[i];
                    nxy = make_float2(ng.x, ng.y);
                    nzr = make_float2(ng.z, ng.w);
                }
                F = (MAPS || TS != TRIDS_TERMS_VINA5) ? make_flag_term(fi, P.w[3], P.w[4]) : flag_term_of(P.ftab[ti]);
                icut = first + cbk;
                ib = reinterpret_cast<const uint4*>(ient + 8 * ipb);
                pb = cbk ? reinterpret_cast<const uint4*>(cand + csb) : ib;
                v = __ldg(pb);
            }
            const uint4 vc = v;
            const bool intra = blk >= icut;
            if (blk + 1 < hi && blk + 1 < nxt) {   // the atom's lists are contiguous blocks
                pb = blk + 1 == icut ? ib : pb + 1;
                v = __ldg(pb);
            }
            const float4* __restrict__ src = intra ? W.xs : S.pocket;
            // pair-flag selectors: hydrophobic needs both bit0; donor-acceptor needs
            // (donor_i & acceptor_j) | (acceptor_i & donor_j)
            const uint32_t f_hyd = fi & 1u;
            const uint32_t f_hb = ((fi & 2u) << 1) | ((fi & 4u) >> 1);
            float eb = 0.f;
            float2 eb2 = make_float2(0.f, 0.f);
            // two halves of four candidates: unrolled in the plain Vina-form and atom-pair TRIDS
            // kernels; the residue-level TRIDS kernel and the general kernels (other update
            // rules, grid maps) keep one half per iteration (unrolled they run slower)
            constexpr int kHalves = (TS != TRIDS_TERMS_TRIDS_RES && !PARAMS && !MAPS) ? 2 : 1;
#pragma unroll kHalves
            for (int hv = 0; hv < 2; ++hv) {
                const uint32_t wv[2] = {hv ? vc.z : vc.x, hv ? vc.w : vc.y};
                if constexpr (TS == TRIDS_TERMS_VINA5 && !PARAMS) {
#pragma unroll
                    for (int u = 0; u < 2; ++u)
                        vina_x2<COUNT, !MAPS>(wv[u], src, nxy, nzr, cut2, K, F, eb2, ax, ay, az, wc.pairs,
                                              intra ? 1u : 2u);   // doubled: intra pairs come twice
                } else if constexpr (!PARAMS) {
                    const float4* gm = nullptr;   // term set 1: the atom-pair E_MDN runs in gmm_warp
#pragma unroll
                    for (int u = 0; u < 2; ++u)
                        trids_x2<COUNT>(wv[u], src, nxy, nzr, cut2, w, F.mb, gm, S.ptype, P.gmm_k, eb2, ax, ay, az,
                                        wc, intra ? 1u : 2u);
                } else {
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        const uint32_t ent = (s & 1) ? (wv[s >> 1] >> 16) : (wv[s >> 1] & 0xffffu);
                        const int j = (int)(ent & 0x1fffu);
                        const uint32_t fj = ent >> 13;
                        const float4 a = src[j];
                        const float dx = xa.x - a.x, dy = xa.y - a.y, dz = xa.z - a.z;
                        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        const bool in = r2 < cut2;
                        if (TS == TRIDS_TERMS_VINA5) {
                            float dd, rinv, et[5];
                            const float e = vina_eval<PARAMS>(r2, ri + a.w, (f_hyd & fj) ? 1.f : 0.f,
                                                              (f_hb & fj) ? 1.f : 0.f, w, dd, rinv, et);
                            const float fr = in ? dd * rinv : 0.f;
                            eb += in ? e : 0.f;
                            ax = fmaf(fr, dx, ax); ay = fmaf(fr, dy, ay); az = fmaf(fr, dz, az);
                            if (PARAMS && in) {
                                const float sc = intra ? 0.5f * ebar : ebar;
#pragma unroll
                                for (int t = 0; t < 5; ++t) acc.gw[t] = fmaf(sc, et[t], acc.gw[t]);
                                W.grs[ti * 32 + lane] -= ebar * dd;
                                if (!intra) W.grs[S.ptype[j] * 32 + lane] -= ebar * dd;
                            }
                        } else if (in) {
                            const int tj = intra ? 0 : S.ptype[j];
                            const bool mdn = TS == TRIDS_TERMS_TRIDS && !intra;   // atom-pair E_MDN
                            float fr, dRs;
                            float et[5];
                            const float e = pair_trids<PARAMS>(fmaxf(r2, 1e-12f), ri + a.w, (f_hb & fj) ? 2 : 0,
                                                               mdn ? &P.gmm[ti][tj][0] : nullptr, P.gmm_k, mdn, w, fr,
                                                               et, dRs);
                            eb += e;
                            ax = fmaf(fr, dx, ax); ay = fmaf(fr, dy, ay); az = fmaf(fr, dz, az);
                            if (PARAMS) {
                                const float sc = intra ? 0.5f * ebar : ebar;
#pragma unroll
                                for (int t = 0; t < 5; ++t) acc.gw[t] = fmaf(sc, et[t], acc.gw[t]);
                                W.grs[ti * 32 + lane] += ebar * dRs;
                                if (!intra) W.grs[tj * 32 + lane] += ebar * dRs;
                            }
                        }
                        if (COUNT) wc.pairs += in ? (intra ? 1u : 2u) : 0u;   // doubled: intra pairs come twice
                    }
                }
            }
            if (!PARAMS) eb = eb2.x + eb2.y;
            if (intra) e_in += eb; else e_lp += eb;
        }
        W.rec[i + lane] = make_float4(ax, ay, az, 0.f);
    }
    // 2. add each atom's partials in lane order
    seg_combine<false>(W, L, N);
    *e_in2 = e_in;
    return e_lp;
}

// Grid-map energy of the warp's pose: each lane takes its atoms whose cell lies inside
// the map domain (the pair loop skipped their pocket candidates): trilinear interpolation
// of the atom type's map at the 8 corners and its analytic gradient, added to W.gs.
// Out of line: the direct-sum sampler keeps its instruction footprint.
__device__ __noinline__ float map_warp(const DevBatch& B, const DevPocket& pk, const LigHdr& h, const PW& W) {
    float e = 0.f;
    for (int i = W.lane; i < h.n_atoms; i += 32) {
        const float4 x = W.xs[i];
        float4 u;
        if (!map_cell(pk, x.x, x.y, x.z, &u)) continue;
        const int cx = (int)u.x, cy = (int)u.y, cz = (int)u.z;
        const float fx = u.x - (float)cx, fy = u.y - (float)cy, fz = u.z - (float)cz;
        const int t = __float_as_int(__ldg(&B.atom_y[h.atom_off + i]).w);
        const size_t sx = 1, sy = (size_t)pk.mx, sz = (size_t)pk.mx * pk.my;
        const float* __restrict__ m = pk.maps + (size_t)t * sz * pk.mz + cz * sz + cy * sy + cx;
        const float v000 = __ldg(m), v100 = __ldg(m + sx), v010 = __ldg(m + sy), v110 = __ldg(m + sy + sx);
        const float v001 = __ldg(m + sz), v101 = __ldg(m + sz + sx), v011 = __ldg(m + sz + sy),
                    v111 = __ldg(m + sz + sy + sx);
        // along x, then y, then z
        const float a00 = fmaf(fx, v100 - v000, v000), a10 = fmaf(fx, v110 - v010, v010);
        const float a01 = fmaf(fx, v101 - v001, v001), a11 = fmaf(fx, v111 - v011, v011);
        const float b0 = fmaf(fy, a10 - a00, a00), b1 = fmaf(fy, a11 - a01, a01);
        e += fmaf(fz, b1 - b0, b0);
        const float dz = b1 - b0;
        const float dy = fmaf(fz, (a11 - a01) - (a10 - a00), a10 - a00);
        const float d00 = v100 - v000, d10 = v110 - v010, d01 = v101 - v001, d11 = v111 - v011;
        const float c0 = fmaf(fy, d10 - d00, d00), c1 = fmaf(fy, d11 - d01, d01);
        const float dx = fmaf(fz, c1 - c0, c0);
        float4 g = W.gs[i];
        g.x = fmaf(dx, pk.inv_mh, g.x);
        g.y = fmaf(dy, pk.inv_mh, g.y);
        g.z = fmaf(dz, pk.inv_mh, g.z);
        W.gs[i] = g;
    }
    __syncwarp();
    return e;
}

// Atom-pair E_MDN of the warp's pose (term set 1; Sec. 2, Eqs. P(d) and E_MDN on atom
// pairs): each ligand atom against the pocket atoms of its cell's near list (within 5 A
// plus half the cell diagonal); a pair with r < min(5 A, cutoff) adds
// -w0 sum_k pi_k exp(-(r - mu_k)^2 / (2 sigma_k^2)) with (pi, mu, sigma) by the atom-type
// pair.  A separate pass over these short lists keeps the K Gaussians off the 10 A pair
// loop (about 1 in 8 of its candidates is within 5 A).  Items (atom, near-list entry) are
// split into 32 equal contiguous lane segments; per-atom partials go to slot (atom + lane)
// of W.rec and are added to W.gs in lane order.  Atoms that the grid maps cover are
// skipped (their maps hold this term).  Returns the lane's energy.
template <bool MAPS, bool COUNT>
__device__ float gmm_warp(const DevBatch& B, const DevPocket& pk, const Smem& S, const LigHdr& h, const PW& W,
                          float w0, WorkCount& wc) {
    const DevParams& P = *S.P;
    const int K = P.gmm_k, L = h.n_atoms, lane = W.lane;
    const float nc2 = pk.near_cut2;
    int carry = 0;
    for (int base = 0; base < L; base += 32) {
        const int i = base + lane;
        int n = 0;
        if (i < L) {
            const float4 x = W.xs[i];
            uint32_t beg = 0;
            if (!(MAPS && map_cell(pk, x.x, x.y, x.z, nullptr)))
                cell_levels(pk, pk.ncell_start, pk.nlevels, x.x, x.y, x.z, beg, n);
            W.meta[i].x = beg;
            W.meta[i].y = __float_as_int(__ldg(&B.atom_y[h.atom_off + i]).w);   // the atom's type
        }
        seg_scan(W, L, i, n, carry);
    }
    const int N = seg_finish(W, L, carry);
    int lo, hi;
    int i = seg_range(W, L, N, lo, hi);
    float e = 0.f;
    if (lo < hi) {
        int first = W.meta[i].w, nxt = W.meta[i + 1].w;
        uint32_t cs = W.meta[i].x;
        float4 x = W.xs[i];
        const float4* g = &P.gmm[W.meta[i].y][0][0];
        float gx = 0.f, gy = 0.f, gz = 0.f, ei = 0.f;
        int jn = __ldg(&pk.nlist[cs + (uint32_t)(lo - first)]);
        for (int it = lo; it < hi; ++it) {
            if (it == nxt) {
                W.rec[i + lane] = make_float4(gx, gy, gz, 0.f);
                e = fmaf(w0, ei, e);
                gx = gy = gz = ei = 0.f;
                do { ++i; } while (W.meta[i + 1].w == it);
                first = W.meta[i].w;
                nxt = W.meta[i + 1].w;
                cs = W.meta[i].x;
                x = W.xs[i];
                g = &P.gmm[W.meta[i].y][0][0];
                jn = __ldg(&pk.nlist[cs + (uint32_t)(it - first)]);
            }
            const int j = jn;
            if (it + 1 < hi && it + 1 < nxt) jn = __ldg(&pk.nlist[cs + (uint32_t)(it + 1 - first)]);   // prefetch
            const float4 p = S.pocket[j];
            const float dx = x.x - p.x, dy = x.y - p.y, dz = x.z - p.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float in = r2 < nc2 ? 1.f : 0.f;
            const float rinv = rsqrt_normal(fmaxf(r2, 1e-12f));
            const float r = r2 * rinv;
            const float4* gk = g + S.ptype[j] * kKP;
            float e0 = 0.f, d0 = 0.f;
            for (int k = 0; k < K; ++k) {
                const float4 u = gk[k];                          // (pi, mu, -log2(e)/(2 sigma^2), 1/sigma^2)
                const float z = r - u.y;
                const float ex = u.x * ex2_approx(u.z * z * z);
                e0 += ex;
                d0 = fmaf(ex * z, u.w, d0);
            }
            ei = fmaf(-in, e0, ei);
            if (COUNT) wc.mdn += r2 < nc2;
            const float f = in * w0 * d0 * rinv;                 // (dE/dr) / r
            gx = fmaf(f, dx, gx); gy = fmaf(f, dy, gy); gz = fmaf(f, dz, gz);
        }
        W.rec[i + lane] = make_float4(gx, gy, gz, 0.f);
        e = fmaf(w0, ei, e);
    }
    seg_combine<true>(W, L, N);
    return e;
}

// Residue-level E_MDN of the warp's pose (term set 2; Sec. 2, Eqs. P(d) and E_MDN): for
// each ligand atom and each residue listed for its cell, the minimum distance d over the
// residue's atoms (one contiguous range of the staged pocket, ascending input index, so a
// strict < keeps the lowest index on ties); d < 5 A adds
// -w0 sum_k pi_k exp(-(d - mu_k)^2 / (2 sigma_k^2)) with the force along the nearest atom.
// The (atom, residue) items are numbered atom by atom and split into 32 equal contiguous
// segments, one per lane, as in the pair loop; per-atom partial forces go to slot
// (atom + lane) of W.rec and are added to W.gs in lane order.  Returns the lane's energy.
template <bool PARAMS, bool COUNT>
__device__ float residue_warp(const DevBatch& B, const DevPocket& pk, const Smem& S, const LigHdr& h, const PW& W,
                              float w0, float ebar, ParamAcc& acc, WorkCount& wc) {
    constexpr float kCut2 = kMdnCut * kMdnCut;
    const int K = B.mdn_k, R = B.mdn_res, L = h.n_atoms, lane = W.lane;
    int carry = 0;
    for (int base = 0; base < L; base += 32) {
        const int i = base + lane;
        int n = 0;
        if (i < L) {
            const float4 x = W.xs[i];
            uint32_t beg;
            cell_levels(pk, pk.rcell_start, pk.rlevels, x.x, x.y, x.z, beg, n);
            W.meta[i].x = beg;
        }
        seg_scan(W, L, i, n, carry);
    }
    const int N = seg_finish(W, L, carry);
    int lo, hi;
    int i = seg_range(W, L, N, lo, hi);
    float e = 0.f;
    if (lo < hi) {
        int first = W.meta[i].w, nxt = W.meta[i + 1].w;
        uint32_t cs = W.meta[i].x;
        float4 x = W.xs[i];
        const float4* __restrict__ kern = B.mdn + (size_t)(h.atom_off + i) * R * K;
        float gx = 0.f, gy = 0.f, gz = 0.f, ei = 0.f;
        uint32_t ent = __ldg(&pk.rlist[cs + (uint32_t)(lo - first)]);
        for (int it = lo; it < hi; ++it) {
            if (it == nxt) {                       // move to the atom owning item it
                W.rec[i + lane] = make_float4(gx, gy, gz, 0.f);
                e = fmaf(w0, ei, e);
                if (PARAMS) acc.gw[0] = fmaf(ebar, ei, acc.gw[0]);
                gx = gy = gz = ei = 0.f;
                do { ++i; } while (W.meta[i + 1].w == it);
                first = W.meta[i].w;
                nxt = W.meta[i + 1].w;
                cs = W.meta[i].x;
                x = W.xs[i];
                kern = B.mdn + (size_t)(h.atom_off + i) * R * K;
                ent = __ldg(&pk.rlist[cs + (uint32_t)(it - first)]);
            }
            const uint32_t cur = ent;
            if (it + 1 < hi && it + 1 < nxt) ent = __ldg(&pk.rlist[cs + (uint32_t)(it + 1 - first)]);   // prefetch
            const int r = (int)(cur & 0x1fffu);
            const int a0 = (int)((cur >> 13) & 0x1fffu), a1 = a0 + (int)(cur >> 26);
            // two interleaved streams (even / odd offsets), each keeping its first minimum;
            // the merge takes the smaller distance, on a tie the lower atom index: the same
            // atom a single ascending scan with a strict < would keep
            float b0 = 3.0e38f, b1 = 3.0e38f;
            int i0 = a0, i1 = a0;
            int a = a0;
            for (; a + 1 < a1; a += 2) {
                const float4 p = S.pocket[a], q = S.pocket[a + 1];
                const float px = x.x - p.x, py = x.y - p.y, pz = x.z - p.z;
                const float qx = x.x - q.x, qy = x.y - q.y, qz = x.z - q.z;
                const float rp = fmaf(pz, pz, fmaf(py, py, px * px)), rq = fmaf(qz, qz, fmaf(qy, qy, qx * qx));
                if (rp < b0) { b0 = rp; i0 = a; }
                if (rq < b1) { b1 = rq; i1 = a + 1; }
            }
            if (a < a1) {
                const float4 p = S.pocket[a];
                const float px = x.x - p.x, py = x.y - p.y, pz = x.z - p.z;
                const float rp = fmaf(pz, pz, fmaf(py, py, px * px));
                if (rp < b0) { b0 = rp; i0 = a; }
            }
            if (COUNT) wc.scan += (uint32_t)(a1 - a0);
            const bool take1 = b1 < b0 || (b1 == b0 && i1 < i0);
            const float best = take1 ? b1 : b0;
            const float4 pb = S.pocket[take1 ? i1 : i0];
            const float bx = x.x - pb.x, by = x.y - pb.y, bz = x.z - pb.z;
            if (best < kCut2) {
                if (COUNT) ++wc.res;
                const float rinv = rsqrt_normal(fmaxf(best, 1e-12f));
                const float d = best * rinv;
                float P = 0.f, dP = 0.f;
#pragma unroll 4   // the kernel-row loads of four kernels in flight together
                for (int k = 0; k < K; ++k) {
                    const float4 g = __ldg(&kern[r * K + k]);   // (pi, mu, -log2(e)/(2 sigma^2), 1/sigma^2)
                    const float z = d - g.y;
                    const float ex = g.x * ex2_approx(g.z * z * z);
                    P += ex;
                    dP = fmaf(-ex * z, g.w, dP);                // dP/dd
                }
                ei -= P;
                const float f = -w0 * dP * rinv;                // (dE/dd) / d
                gx = fmaf(f, bx, gx); gy = fmaf(f, by, gy); gz = fmaf(f, bz, gz);
            }
        }
        W.rec[i + lane] = make_float4(gx, gy, gz, 0.f);
        e = fmaf(w0, ei, e);
        if (PARAMS) acc.gw[0] = fmaf(ebar, ei, acc.gw[0]);
    }
    seg_combine<true>(W, L, N);
    return e;
}

// Per-phase SM clock cycles of a warp (the counting form of the sampler only), kept in
// the warp's shared-memory clock slots so that the timed code keeps its registers: lap(k)
// charges the cycles since the previous lap to phase k (TRIDS_PHASE_*); lane 0 keeps the
// books.
struct PhaseClock {
    unsigned long long* c;   // W.clk: [TRIDS_PHASES] sums, then the time of the last lap
    __device__ __forceinline__ explicit PhaseClock(const PW& W) : c(W.clk) {}
    __device__ __forceinline__ void start() {
        if ((threadIdx.x & 31) == 0) {
#pragma unroll
            for (int k = 0; k < TRIDS_PHASES; ++k) c[k] = 0ull;
            c[TRIDS_PHASES] = (unsigned long long)clock64();
        }
    }
    __device__ __forceinline__ void lap(int k) {
        if ((threadIdx.x & 31) == 0) {
            const unsigned long long n = (unsigned long long)clock64();
            c[k] += n - c[TRIDS_PHASES];
            c[TRIDS_PHASES] = n;
        }
    }
    __device__ __forceinline__ void flush(unsigned long long* out) const {
        if (out && (threadIdx.x & 31) == 0)
#pragma unroll
            for (int k = 0; k < TRIDS_PHASES; ++k) atomicAdd(out + k, c[k]);
    }
};

// E_total of the warp's pose (same value on every lane); forces in W.gs.  COUNT kernels
// time the pair loop and the other passes on pc.
template <int TS, bool PARAMS, bool COUNT, bool MAPS>
__device__ float score_warp(const DevBatch& B, const DevPocket& pk, const Smem& S, const LigHdr& h, const PW& W,
                            float ebar, ParamAcc& acc, float* e_inter, WorkCount& wc, PhaseClock* pc = nullptr) {
    float w[5];
#pragma unroll
    for (int t = 0; t < 5; ++t) w[t] = S.P->w[t];
    float ein2;
    float el = pairs_warp<TS, PARAMS, COUNT, MAPS>(B, pk, S, h, W, w, ebar, acc, wc, &ein2);
    if (COUNT && pc) pc->lap(TRIDS_PHASE_PAIRS);
    if (MAPS && pk.use_maps) el += map_warp(B, pk, h, W);
    if constexpr (TS == TRIDS_TERMS_TRIDS && !PARAMS) el += gmm_warp<MAPS, COUNT>(B, pk, S, h, W, w[0], wc);
    if constexpr (TS == TRIDS_TERMS_TRIDS_RES) el += residue_warp<PARAMS, COUNT>(B, pk, S, h, W, w[0], ebar, acc, wc);
    if (COUNT && pc) pc->lap(TRIDS_PHASE_PASSES);
    const float e_lp = warp_sum(el);
    *e_inter = e_lp;
    return e_lp + 0.5f * warp_sum(ein2);
}

// dE/dt = sum g_i and world torque tau = sum (x_i - t) x g_i (every lane), and
// dE/dtheta_k = a_k . sum over the moving subtree of (x_i - p_k) x g_i with a_k the world
// axis (parent atom -> child atom) and p_k the world parent atom.  A torsion's moving
// subtree is one contiguous atom range [z_k, w_k), so one warp scan gives inclusive
// prefixes G(i) = sum_{i' <= i} g_i' and U(i) = sum_{i' <= i} (x_i' - t) x g_i' (kept in
// W.rec and the per-atom list arrays, free at this point); lane k then takes
// sum_[z,w) (x_i - p_k) x g_i = dU - (p_k - t) x dG with dU, dG the range differences.
__device__ float adjoint_warp(const DevBatch& B, const LigHdr& h, const PW& W, const float t[3], float gt[3],
                              float tau[3]) {
    const int L = h.n_atoms, T = h.n_tor, lane = W.lane;
    float4* __restrict__ pu = W.rec;                                  // U prefix, [L]
    float4* __restrict__ pg = reinterpret_cast<float4*>(W.meta);       // G prefix, [L]
    float c[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};                      // totals of the rounds so far
    for (int base = 0; base < L; base += 32) {
        const int i = base + lane;
        float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (i < L) {
            const float4 g = W.gs[i], x = W.xs[i];
            const float rx = x.x - t[0], ry = x.y - t[1], rz = x.z - t[2];
            v[0] = g.x; v[1] = g.y; v[2] = g.z;
            v[3] = ry * g.z - rz * g.y;
            v[4] = rz * g.x - rx * g.z;
            v[5] = rx * g.y - ry * g.x;
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float u = __shfl_up_sync(kFull, v[k], o);
                if (lane >= o) v[k] += u;
            }
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] += c[k];
        if (i < L) {
            pg[i] = make_float4(v[0], v[1], v[2], 0.f);
            pu[i] = make_float4(v[3], v[4], v[5], 0.f);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) c[k] = __shfl_sync(kFull, v[k], 31);
    }
    gt[0] = c[0]; gt[1] = c[1]; gt[2] = c[2];
    tau[0] = c[3]; tau[1] = c[4]; tau[2] = c[5];
    __syncwarp();
    // torsion k on lane k: its moving subtree is the contiguous atom range [ti.z, ti.w)
    float mine = 0.f;
    if (lane < T) {
        const int4 ti = __ldg(&B.tor_idx[h.tor_off + lane]);
        const float4 p = W.xs[ti.x], cc = W.xs[ti.y];
        const float4 gw = pg[ti.w - 1], uw = pu[ti.w - 1];
        const float4 gz = ti.z > 0 ? pg[ti.z - 1] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 uz = ti.z > 0 ? pu[ti.z - 1] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float dgx = gw.x - gz.x, dgy = gw.y - gz.y, dgz = gw.z - gz.z;
        const float px = p.x - t[0], py = p.y - t[1], pz = p.z - t[2];
        const float sx = (uw.x - uz.x) - (py * dgz - pz * dgy);
        const float sy = (uw.y - uz.y) - (pz * dgx - px * dgz);
        const float sz = (uw.z - uz.z) - (px * dgy - py * dgx);
        const float ax = cc.x - p.x, ay = cc.y - p.y, az = cc.z - p.z;
        const float n = rsqrt_normal(ax * ax + ay * ay + az * az);
        mine = (ax * sx + ay * sy + az * sz) * n;
    }
    return mine;
}


}  // namespace
