// libtrids device code, part 3: sampler state and update rules, the sampler, scorer,
// parameter-reduction, top-k, map-build and status kernels.  Included by trids.cu only.
#pragma once

namespace {

// ------------------------------------------------------------------ sampler state
// The rigid state is the same on every lane (every lane computes it); lane k < T holds
// torsion k's angle, Adam moments and saved angle.  PoseState is a handle on the warp's
// shared-memory copy.
struct RigidState {
    float t[3], q[4], m[6], v[6], st[3], sq[4];
    float ecur, esaved;
    int status;
    int sid;          // the ligand's random-stream id (lig_base + stream id)
    float pad[2];
};
struct TorState {
    float th, mth, vth, sth;
};
static_assert(sizeof(RigidState) == kRigidStateBytes && sizeof(TorState) == kTorStateBytes, "pose state size");

struct PoseState {
    float (&t)[3];
    float (&q)[4];
    float (&m)[6];
    float (&v)[6];
    float (&st)[3];
    float (&sq)[4];
    float& ecur;
    float& esaved;
    int& status;
    int& sid;
    float& th;
    float& mth;
    float& vth;
    float& sth;
    __device__ PoseState(RigidState& r, TorState& k)
        : t(r.t), q(r.q), m(r.m), v(r.v), st(r.st), sq(r.sq), ecur(r.ecur), esaved(r.esaved), status(r.status), sid(r.sid),
          th(k.th), mth(k.mth), vth(k.vth), sth(k.sth) {}
};

struct SampleArgs {
    DevPocket pk;
    DevBatch B;
    int P, S, step_begin, step_end, Lmc;
    float lr, b1, b2, eps, beta;
    int opt;
    float wd, momentum, alpha;
    uint64_t seed;
    int lig_base;
    float* dof;
    float* state;
    float* energy;
    float* trace;
    const int* trace_slot;
    int n_trace;
    unsigned long long* pair_count;
    unsigned long long* phase_cycles;
    unsigned long long* work_count;
    const int* lig_order;      // ligands by decreasing cost; item it = (lig_order[it / P], it % P)
    int n_items;
    unsigned int* counter;
    int* err;
    size_t params_bytes, pocket_off, ptype_off, mbar_off, warp_off, warp_bytes;
};

struct Sched {
    int loop, j, n;
};

__device__ __forceinline__ Sched schedule(int S, int Lmc, int s) {
    const int base = S / Lmc, rem = S % Lmc;
    Sched r;
    const int head = rem * (base + 1);
    if (s < head) {
        r.loop = s / (base + 1); r.j = s % (base + 1); r.n = base + 1;
    } else {
        const int s2 = s - head;
        r.loop = rem + s2 / base; r.j = s2 % base; r.n = base;
    }
    return r;
}

__device__ __forceinline__ float* fld(const SampleArgs& A, int l, int f, int p) {
    return A.state + ((size_t)l * A.B.n_fields + f) * A.P + p;
}

__device__ void init_pose(const SampleArgs& A, const LigHdr& h, int lane, int l, int p, PoseState& st) {
    const uint32_t lig = (uint32_t)(A.lig_base + h.sid);
    st.sid = (int)lig;
    const uint4 r0 = rand_block(A.seed, lig, (uint32_t)p, 0u, 0u, 0u);
    const uint4 r1 = rand_block(A.seed, lig, (uint32_t)p, 0u, 0u, 1u);
    const float u[6] = {u01(r0.x), u01(r0.y), u01(r0.z), u01(r0.w), u01(r1.x), u01(r1.y)};
    const int bx = A.pk.n_boxes > 1 ? p % A.pk.n_boxes : 0;
    for (int d = 0; d < 3; ++d)
        st.t[d] = fmaf(u[d], A.pk.box_hi[bx][d] - A.pk.box_lo[bx][d], A.pk.box_lo[bx][d]);
    const float a = sqrtf(1.f - u[3]), b = sqrtf(u[3]);
    float s1, c1, s2, c2;
    sincospif(2.f * u[4], &s1, &c1);
    sincospif(2.f * u[5], &s2, &c2);
    st.q[0] = a * s1; st.q[1] = a * c1; st.q[2] = b * s2; st.q[3] = b * c2;
    st.th = 0.f;
    if (lane < h.n_tor) {
        const int n = 6 + lane;
        const uint4 r = rand_block(A.seed, lig, (uint32_t)p, 0u, 0u, (uint32_t)(n >> 2));
        st.th = fmaf(u01(pick(r, n & 3)), kTwoPi, -kPi);
    }
    for (int d = 0; d < 6; ++d) { st.m[d] = 0.f; st.v[d] = 0.f; }
    for (int d = 0; d < 3; ++d) st.st[d] = st.t[d];
    for (int d = 0; d < 4; ++d) st.sq[d] = st.q[d];
    st.ecur = __int_as_float(0x7fc00000);
    st.esaved = st.ecur;
    st.status = 0;
    st.mth = st.vth = 0.f;
    st.sth = st.th;
}

__device__ void load_pose(const SampleArgs& A, const LigHdr& h, int lane, int l, int p, PoseState& st) {
    const float* row = A.dof + ((size_t)l * A.P + p) * A.B.dof_stride;
    for (int d = 0; d < 3; ++d) st.t[d] = row[d];
    for (int d = 0; d < 4; ++d) st.q[d] = row[3 + d];
    for (int d = 0; d < 6; ++d) { st.m[d] = *fld(A, l, kFieldM + d, p); st.v[d] = *fld(A, l, kFieldV + d, p); }
    for (int d = 0; d < 3; ++d) st.st[d] = *fld(A, l, kFieldSaved + d, p);
    for (int d = 0; d < 4; ++d) st.sq[d] = *fld(A, l, kFieldSaved + 3 + d, p);
    st.sid = A.lig_base + h.sid;
    st.ecur = *fld(A, l, kFieldEcur, p);
    st.esaved = *fld(A, l, kFieldEsaved, p);
    st.status = __float_as_int(*fld(A, l, kFieldStatus, p));
    st.th = st.mth = st.vth = st.sth = 0.f;
    if (lane < h.n_tor) {
        const int M = A.B.max_tor;
        st.th = row[7 + lane];
        st.mth = *fld(A, l, kFieldTheta + lane, p);
        st.vth = *fld(A, l, kFieldTheta + M + lane, p);
        st.sth = *fld(A, l, kFieldTheta + 2 * M + lane, p);
    }
}

__device__ void store_pose(const SampleArgs& A, const LigHdr& h, int lane, int l, int p, const PoseState& st) {
    float* row = A.dof + ((size_t)l * A.P + p) * A.B.dof_stride;
    const int M = A.B.max_tor;
    if (lane == 0) {
        for (int d = 0; d < 3; ++d) row[d] = st.t[d];
        for (int d = 0; d < 4; ++d) row[3 + d] = st.q[d];
        for (int d = 0; d < 6; ++d) { *fld(A, l, kFieldM + d, p) = st.m[d]; *fld(A, l, kFieldV + d, p) = st.v[d]; }
        for (int d = 0; d < 3; ++d) *fld(A, l, kFieldSaved + d, p) = st.st[d];
        for (int d = 0; d < 4; ++d) *fld(A, l, kFieldSaved + 3 + d, p) = st.sq[d];
        *fld(A, l, kFieldEcur, p) = st.ecur;
        *fld(A, l, kFieldEsaved, p) = st.esaved;
        *fld(A, l, kFieldStatus, p) = __int_as_float(st.status);
        A.energy[(size_t)l * A.P + p] = st.ecur;
    }
    if (lane < M) {
        const bool own = lane < h.n_tor;
        row[7 + lane] = own ? st.th : 0.f;
        *fld(A, l, kFieldTheta + lane, p) = own ? st.mth : 0.f;
        *fld(A, l, kFieldTheta + M + lane, p) = own ? st.vth : 0.f;
        *fld(A, l, kFieldTheta + 2 * M + lane, p) = own ? st.sth : 0.f;
    }
}

// b^n, n >= 0, by repeated squaring: the same float operations in every form of the sampler.
__device__ __forceinline__ float ipowf(float b, int n) {
    float r = 1.f;
    while (n) {
        if (n & 1) r *= b;
        b *= b;
        n >>= 1;
    }
    return r;
}

// Step of one variable under the configured update rule (trids.h, TRIDS_OPT_*); pv is
// the value a weight decay acts on.  For Adam(W) lr_bc1 = lr / (1 - b1^k) and
// rsbc2 = 1 / sqrt(1 - b2^k), k = the step within the Monte-Carlo loop.
// GEN = false compiles Adam alone: the other rules' code would otherwise enlarge the
// sampler kernel, which costs the pair loop instruction-cache hits.
template <bool GEN>
__device__ __forceinline__ float opt_delta(const SampleArgs& A, float g, float pv, float& m, float& v, float lr_bc1,
                                           float rsbc2) {
    if (GEN) {
        switch (A.opt) {
        case TRIDS_OPT_RMSPROP:
            v = fmaf(A.alpha, v, (1.f - A.alpha) * g * g);
            return -A.lr * g / (sqrt_fast(v) + A.eps);
        case TRIDS_OPT_ADAGRAD:
            v = fmaf(g, g, v);
            return -A.lr * g / (sqrt_fast(v) + A.eps);
        case TRIDS_OPT_SGD:
            m = fmaf(A.momentum, m, g);
            return -A.lr * m;
        default:
            break;
        }
    }
    m = fmaf(A.b1, m, (1.f - A.b1) * g);
    v = fmaf(A.b2, v, (1.f - A.b2) * g * g);
    const float denom = fmaf(sqrt_fast(v), rsbc2, A.eps);
    const float d = -lr_bc1 * __fdividef(m, denom);
    return GEN && A.opt == TRIDS_OPT_ADAMW ? fmaf(-A.lr * A.wd, pv, d) : d;
}

// One evaluation (and its update or acceptance test) of the warp's pose; s is the
// global evaluation index of the schedule.  Every branch below is uniform across the
// warp except the per-torsion lanes.
template <int TS, bool COUNT, bool GEN>
__device__ void sample_step(const SampleArgs& A, const Smem& S, const LigHdr& h, const PW& W, int l, int p, int s,
                            const Sched& sc, PoseState& st, WorkCount& wc, PhaseClock& pc) {
    __syncwarp();               // the rigid state is one shared copy written by every lane
    if (st.status & 1) return;  // frozen after a non-finite energy
    const int T = h.n_tor, lane = W.lane;
    const int bx = A.pk.n_boxes > 1 ? p % A.pk.n_boxes : 0;   // the pose's docking box
    const bool own = lane < T;
    const uint32_t lig = (uint32_t)st.sid;
    if (sc.j == 0) {
        if (sc.loop > 0) {
            // save the state, then resample one of the 6+T variables in its range
            for (int d = 0; d < 3; ++d) st.st[d] = st.t[d];
            for (int d = 0; d < 4; ++d) st.sq[d] = st.q[d];
            st.sth = st.th;
            st.esaved = st.ecur;
            const uint4 r = rand_block(A.seed, lig, (uint32_t)p, (uint32_t)sc.loop, 1u, 0u);
            const int c = (int)(((unsigned long long)(r.x >> 8) * (unsigned long long)(6 + T)) >> 24);
            const float u1 = u01(r.y);
            if (c < 3) {
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    if (d == c) st.t[d] = fmaf(u1, A.pk.box_hi[bx][d] - A.pk.box_lo[bx][d], A.pk.box_lo[bx][d]);
            } else if (c < 6) {
                const float ang = fmaf(u1, kTwoPi, -kPi);
                float sh, ch;
                __sincosf(0.5f * ang, &sh, &ch);   // half angles in [-pi/2, pi/2]: hardware sin/cos
                const float rq[4] = {ch, c == 3 ? sh : 0.f, c == 4 ? sh : 0.f, c == 5 ? sh : 0.f};
                quat_premul(rq, st.q);
            } else if (lane == c - 6) {
                st.th = fmaf(u1, kTwoPi, -kPi);
            }
        }
        for (int d = 0; d < 6; ++d) { st.m[d] = 0.f; st.v[d] = 0.f; }
        st.mth = st.vth = 0.f;
    }
    // evaluate
    if (COUNT) pc.lap(TRIDS_PHASE_UPDATE);
    fk_warp(A.B, h, W, st.t, st.q, st.th, S.P->radius);
    if (COUNT) pc.lap(TRIDS_PHASE_FK);
    ParamAcc acc;
    float e_inter;
    const float E = score_warp<TS, false, COUNT, GEN>(A.B, A.pk, S, h, W, 1.f, acc, &e_inter, wc, &pc);
    float gt[3], tau[3];
    const float gth = adjoint_warp(A.B, h, W, st.t, gt, tau);
    if (COUNT) pc.lap(TRIDS_PHASE_ADJOINT);
    if (A.trace) {
        const int slot = A.trace_slot[(size_t)l * A.P + p];
        if (slot >= 0) {
            float* rec = A.trace + ((size_t)(s - A.step_begin) * A.n_trace + slot) * trace_record(A.B.max_tor);
            const int o = A.B.dof_stride;
            if (lane == 0) {
                for (int d = 0; d < 3; ++d) rec[d] = st.t[d];
                for (int d = 0; d < 4; ++d) rec[3 + d] = st.q[d];
                rec[o] = E;
                for (int d = 0; d < 3; ++d) { rec[o + 1 + d] = gt[d]; rec[o + 4 + d] = tau[d]; }
            }
            if (lane < A.B.max_tor) {
                rec[7 + lane] = own ? st.th : 0.f;
                rec[o + 7 + lane] = own ? gth : 0.f;
            }
        }
    }
    if (!isfinite(E)) {
        st.status |= 1;
        st.ecur = E;
        return;
    }
    if (sc.j < sc.n - 1) {
        const int ta = sc.j + 1;
        const float lr_bc1 = __fdividef(A.lr, 1.f - ipowf(A.b1, ta));
        const float rsbc2 = rsqrt_normal(1.f - ipowf(A.b2, ta));
        if (own) st.th = wrap_pi(st.th + opt_delta<GEN>(A, gth, st.th, st.mth, st.vth, lr_bc1, rsbc2));
        for (int d = 0; d < 3; ++d) {
            const float lo = A.pk.box_lo[bx][d], hi = A.pk.box_hi[bx][d];
            const float dlt = opt_delta<GEN>(A, gt[d], st.t[d] - 0.5f * (lo + hi), st.m[d], st.v[d], lr_bc1, rsbc2);
            st.t[d] = fminf(fmaxf(st.t[d] + dlt, lo), hi);
        }
        float dw[3];
        for (int d = 0; d < 3; ++d) dw[d] = opt_delta<GEN>(A, tau[d], 0.f, st.m[3 + d], st.v[3 + d], lr_bc1, rsbc2);
        const float phi = sqrt_fast(dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2]);
        if (phi > 0.f) {
            float sh, ch;
            __sincosf(0.5f * phi, &sh, &ch);   // absolute error about 4e-7, far below a step's own size
            const float sc2 = __fdividef(sh, phi);
            const float rq[4] = {ch, sc2 * dw[0], sc2 * dw[1], sc2 * dw[2]};
            quat_premul(rq, st.q);
        }
    } else {
        st.ecur = E;
        if (sc.loop > 0) {
            const uint4 r = rand_block(A.seed, lig, (uint32_t)p, (uint32_t)sc.loop, 2u, 0u);
            const float u = u01(r.x);
            if (!(u < expf(-A.beta * (E - st.esaved)))) {
                for (int d = 0; d < 3; ++d) st.t[d] = st.st[d];
                for (int d = 0; d < 4; ++d) st.q[d] = st.sq[d];
                st.th = st.sth;
                st.ecur = st.esaved;
            }
        }
    }
}

// Warp totals of the lanes' work counts.  Pair counts are kept doubled per lane (an intra
// pair is seen from both of its atoms, possibly by different lanes) and halved here.
__device__ __forceinline__ unsigned long long warp_total(uint32_t n) {
    unsigned long long v = n;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ void flush_count(unsigned long long* cnt, unsigned long long* work, const WorkCount& wc) {
    const unsigned long long v[TRIDS_WORK_COUNTS + 1] = {warp_total(wc.pairs) >> 1, warp_total(wc.clash) >> 1,
                                                        warp_total(wc.hb) >> 1, warp_total(wc.mdn),
                                                        warp_total(wc.scan), warp_total(wc.res)};
    if ((threadIdx.x & 31) != 0) return;
    if (cnt && v[0]) atomicAdd(cnt, v[0]);
    if (work)
        for (int k = 0; k < TRIDS_WORK_COUNTS; ++k)
            if (v[k + 1]) atomicAdd(work + k, v[k + 1]);
}

// Warps per block the sampler kernels are compiled for (their register budget): 28 for the
// plain Vina-form kernels (72 registers per thread), 24 for the others (80), the counts that
// ran fastest on a B300; fewer warps per block are allowed.
__host__ __device__ constexpr int sample_warps_max(int ts, bool gen) {
    return ts == TRIDS_TERMS_VINA5 && !gen ? 28 : 24;
}

// Persistent fused sampler: each warp pops poses from a global counter (ligands in
// decreasing-cost order) and runs every evaluation of the pose with its state on chip.
template <int TS, bool COUNT, bool GEN>
__global__ void __launch_bounds__(32 * sample_warps_max(TS, GEN), 1) k_sample_persistent(SampleArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (!stage_block(smem, A.pk, A.params_bytes, A.pocket_off, A.ptype_off, A.mbar_off, A.err)) return;
    Smem S{reinterpret_cast<const DevParams*>(smem), reinterpret_cast<const float4*>(smem + A.pocket_off),
           reinterpret_cast<const uint8_t*>(smem + A.ptype_off)};
    const PW W = make_pw(smem, A.warp_off, A.warp_bytes, A.B.max_atoms, A.B.max_tor);
    WorkCount wc;
    PhaseClock pc(W);
    if (COUNT) pc.start();
    for (;;) {
        int it = 0;
        if (W.lane == 0) it = (int)atomicAdd(A.counter, 1u);
        it = __shfl_sync(kFull, it, 0);
        if (it >= A.n_items) break;
        const int l = A.lig_order[it / A.P];
        const int p = it % A.P;
        if (W.lane == 0) *W.hdr = A.B.lig[l];
        __syncwarp();
        const LigHdr& h = *W.hdr;              // in shared memory, like the pose state
        PoseState st(*W.rig, W.tor[W.lane]);   // in shared memory: no registers across the pair loop
        if (A.step_begin == 0) init_pose(A, h, W.lane, l, p, st);
        else load_pose(A, h, W.lane, l, p, st);
        __syncwarp();
        if (COUNT) pc.lap(TRIDS_PHASE_OTHER);
        Sched sc = schedule(A.S, A.Lmc, A.step_begin);
        for (int s = A.step_begin; s < A.step_end; ++s) {
            sample_step<TS, COUNT, GEN>(A, S, h, W, l, p, s, sc, st, wc, pc);
            if (COUNT) pc.lap(TRIDS_PHASE_UPDATE);
            if (++sc.j == sc.n) {   // next Monte-Carlo loop: the schedule of evaluation s + 1
                ++sc.loop;
                sc.j = 0;
                sc.n = A.S / A.Lmc + (sc.loop < A.S % A.Lmc ? 1 : 0);
            }
        }
        __syncwarp();
        store_pose(A, h, W.lane, l, p, st);
        __syncwarp();
        if (COUNT) pc.lap(TRIDS_PHASE_OTHER);
    }
    if (COUNT) {
        flush_count(A.pair_count, A.work_count, wc);
        pc.flush(A.phase_cycles);
    }
}

// Plain form: one launch per (ligand, evaluation), one warp per pose, the state in
// global memory between launches; the same device code as the persistent sampler.
template <int TS, bool COUNT, bool GEN>
__global__ void __launch_bounds__(32 * sample_warps_max(TS, GEN), 1) k_sample_step(SampleArgs A, int l, int s) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (!stage_block(smem, A.pk, A.params_bytes, A.pocket_off, A.ptype_off, A.mbar_off, A.err)) return;
    Smem S{reinterpret_cast<const DevParams*>(smem), reinterpret_cast<const float4*>(smem + A.pocket_off),
           reinterpret_cast<const uint8_t*>(smem + A.ptype_off)};
    const PW W = make_pw(smem, A.warp_off, A.warp_bytes, A.B.max_atoms, A.B.max_tor);
    const int p = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    if (p >= A.P) return;
    const LigHdr h = A.B.lig[l];
    WorkCount wc;
    PhaseClock pc(W);
    if (COUNT) pc.start();
    PoseState st(*W.rig, W.tor[W.lane]);
    if (s == 0) init_pose(A, h, W.lane, l, p, st);
    else load_pose(A, h, W.lane, l, p, st);
    __syncwarp();
    if (COUNT) pc.lap(TRIDS_PHASE_OTHER);
    sample_step<TS, COUNT, GEN>(A, S, h, W, l, p, s, schedule(A.S, A.Lmc, s), st, wc, pc);
    if (COUNT) pc.lap(TRIDS_PHASE_UPDATE);
    __syncwarp();
    store_pose(A, h, W.lane, l, p, st);
    if (COUNT) {
        pc.lap(TRIDS_PHASE_OTHER);
        flush_count(A.pair_count, A.work_count, wc);
        pc.flush(A.phase_cycles);
    }
}

// ------------------------------------------------------------------ score + gradient
struct ScoreArgs {
    DevPocket pk;
    DevBatch B;
    int P;
    const float* dof;
    float* energy;
    float* e_inter;
    float* g_dof;
    float* g_xyz;
    const float* e_bar;
    float* partials;   // [n_items][5 + kNT]
    const int2* items; // (ligand, first pose of a 32-pose tile)
    int n_items;
    unsigned int* counter;
    int* err;
    size_t params_bytes, pocket_off, ptype_off, mbar_off, warp_off, warp_bytes;
};

// Each warp takes a (ligand, 32-pose tile) item and scores its poses one after another;
// parameter-gradient sums of the tile are reduced in a fixed order into one row.
template <int TS, bool PARAMS>
__global__ void __launch_bounds__(512, 1) k_score(ScoreArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (!stage_block(smem, A.pk, A.params_bytes, A.pocket_off, A.ptype_off, A.mbar_off, A.err)) return;
    Smem S{reinterpret_cast<const DevParams*>(smem), reinterpret_cast<const float4*>(smem + A.pocket_off),
           reinterpret_cast<const uint8_t*>(smem + A.ptype_off)};
    const PW W = make_pw(smem, A.warp_off, A.warp_bytes, A.B.max_atoms, A.B.max_tor);
    const int D = A.B.dof_stride, lane = W.lane;
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(A.counter, 1u);
        it = __shfl_sync(kFull, it, 0);
        if (it >= A.n_items) break;
        const int2 item = A.items[it];
        const int l = item.x;
        const LigHdr h = A.B.lig[l];
        ParamAcc acc;
        for (int t5 = 0; t5 < 5; ++t5) acc.gw[t5] = 0.f;
        if (PARAMS)
            for (int a = 0; a < kNT; ++a) W.grs[a * 32 + lane] = 0.f;
        const int p_end = min(item.y + 32, A.P);
        for (int p = item.y; p < p_end; ++p) {
            const size_t gp = (size_t)l * A.P + p;
            const float* row = A.dof + gp * D;
            const float t[3] = {row[0], row[1], row[2]};
            const float q[4] = {row[3], row[4], row[5], row[6]};
            const float th = lane < h.n_tor ? row[7 + lane] : 0.f;
            const float ebar = A.e_bar ? A.e_bar[gp] : 1.f;
            fk_warp(A.B, h, W, t, q, th, S.P->radius);
            float e_inter;
            WorkCount wc;
            const float E = score_warp<TS, PARAMS, false, !PARAMS>(A.B, A.pk, S, h, W, ebar, acc, &e_inter, wc);
            if (lane == 0) {
                A.energy[gp] = E;
                if (A.e_inter) A.e_inter[gp] = e_inter;
            }
            if (A.g_dof) {
                float gt[3], tau[3];
                const float gth = adjoint_warp(A.B, h, W, t, gt, tau);
                float* o = A.g_dof + gp * D;
                const float sc = A.e_bar ? ebar : 1.f;
                if (lane == 0) {
                    for (int d = 0; d < 3; ++d) o[d] = sc * gt[d];
                    // dE/dq of E(q/|q|) = 4 M(qhat) tau / |q|, M(q) = 1/2 [-v^T ; w I - [v]x]
                    const float n = rsqrt_normal(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
                    const float w = q[0] * n, vx = q[1] * n, vy = q[2] * n, vz = q[3] * n;
                    const float c0 = vy * tau[2] - vz * tau[1], c1 = vz * tau[0] - vx * tau[2],
                                c2 = vx * tau[1] - vy * tau[0];
                    o[3] = sc * 2.f * n * (-(vx * tau[0] + vy * tau[1] + vz * tau[2]));
                    o[4] = sc * 2.f * n * (w * tau[0] - c0);
                    o[5] = sc * 2.f * n * (w * tau[1] - c1);
                    o[6] = sc * 2.f * n * (w * tau[2] - c2);
                }
                if (lane < A.B.max_tor) o[7 + lane] = lane < h.n_tor ? sc * gth : 0.f;
            }
            if (A.g_xyz) {
                const float sc = A.e_bar ? ebar : 1.f;
                float* o = A.g_xyz + gp * A.B.max_atoms * 3;
                for (int i = lane; i < A.B.max_atoms; i += 32) {
                    if (i < h.n_atoms) {
                        const int oi = __ldg(&A.B.atom_orig[h.atom_off + i]);
                        const float4 g = W.gs[i];
                        o[3 * oi] = sc * g.x; o[3 * oi + 1] = sc * g.y; o[3 * oi + 2] = sc * g.z;
                    } else {
                        o[3 * i] = 0.f; o[3 * i + 1] = 0.f; o[3 * i + 2] = 0.f;
                    }
                }
            }
            __syncwarp();
        }
        if (PARAMS) {
            float* prow = A.partials + (size_t)it * (5 + kNT);
            for (int t5 = 0; t5 < 5; ++t5) {
                const float v = warp_sum(acc.gw[t5]);
                if (lane == 0) prow[t5] = v;
            }
            for (int a = 0; a < kNT; ++a) {
                const float v = warp_sum(W.grs[a * 32 + lane]);
                if (lane == 0) prow[5 + a] = v;
            }
        }
        __syncwarp();
    }
}

// Sum item partials in item order: out_w[5], out_r[n_types].
__global__ void k_reduce_params(const float* partials, int n_items, float* g_w, float* g_r, int n_types) {
    const int c = threadIdx.x;
    if (c >= 5 + n_types) return;
    float s = 0.f;
    for (int i = 0; i < n_items; ++i) s += partials[(size_t)i * (5 + kNT) + c];
    if (c < 5) { if (g_w) g_w[c] = s; }
    else if (g_r) g_r[c - 5] = s;
}

// E_screen of the kept poses: e_inter of pose idx / (1 + w_tor * N_tor), one thread per
// (ligand, slot); empty or out-of-range slots get NaN.
__global__ void __launch_bounds__(256) k_screen(DevBatch B, int P, int k, const int* __restrict__ idx,
                                               const float* __restrict__ e_inter, float w_tor, float* e_screen) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)B.n_lig * k) return;
    const int l = (int)(t / k);
    const int j = idx[t];
    const float den = fmaf(w_tor, (float)B.lig[l].n_tor, 1.f);
    e_screen[t] = (j >= 0 && j < P) ? __fdiv_rn(e_inter[(size_t)l * P + j], den) : __int_as_float(0x7fc00000);
}

// ------------------------------------------------------------------ top-k
// One block per ligand: rank by (E, index) with non-finite energies last, then walk
// the ranking and keep a pose unless its RMSD to a kept pose is below rho.
__global__ void __launch_bounds__(128) k_topk(DevBatch B, int P, const float* energy, const float* dof, int k,
                                              float rho, int* idx, float* e_out) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int l = blockIdx.x;
    const LigHdr h = B.lig[l];
    const int L = h.n_atoms;
    int* order = reinterpret_cast<int*>(smem);
    float* cand = reinterpret_cast<float*>(order + align_up(P, 4));
    float* kept = cand + 3 * kLmax;
    float* red = kept + (size_t)k * 3 * kLmax;
    __shared__ int s_flag;
    const float* E = energy + (size_t)l * P;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const float ep = E[p];
        const bool fp = isfinite(ep);
        int rank = 0;
        for (int q = 0; q < P; ++q) {
            const float eq = E[q];
            const bool fq = isfinite(eq);
            bool before;
            if (fq != fp) before = fq;
            else if (fq && eq != ep) before = eq < ep;
            else before = q < p;
            rank += before ? 1 : 0;
        }
        order[rank] = p;
    }
    __syncthreads();
    int nk = 0;
    for (int n = 0; n < P && nk < k; ++n) {
        const int p = order[n];
        if (!isfinite(E[p])) break;
        // coordinates of pose p: torsions deepest first, then the rigid placement
        const float* row = dof + ((size_t)l * P + p) * B.dof_stride;
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            const float4 y = B.atom_y[h.atom_off + i];
            float x0 = y.x, x1 = y.y, x2 = y.z;
            for (int kk = h.n_tor - 1; kk >= 0; --kk) {
                const int4 ti = B.tor_idx[h.tor_off + kk];
                if (i < ti.z || i >= ti.w) continue;
                const float4 u = B.tor_u[h.tor_off + kk];
                const float4 pp = B.tor_p[h.tor_off + kk];
                float s, c;
                sincosf(row[7 + kk], &s, &c);
                const float kc = 1.f - c;
                const float vx = x0 - pp.x, vy = x1 - pp.y, vz = x2 - pp.z;
                x0 = pp.x + ((c + kc * u.x * u.x) * vx + (kc * u.x * u.y - s * u.z) * vy + (kc * u.x * u.z + s * u.y) * vz);
                x1 = pp.y + ((kc * u.y * u.x + s * u.z) * vx + (c + kc * u.y * u.y) * vy + (kc * u.y * u.z - s * u.x) * vz);
                x2 = pp.z + ((kc * u.z * u.x - s * u.y) * vx + (kc * u.z * u.y + s * u.x) * vy + (c + kc * u.z * u.z) * vz);
            }
            float q[4] = {row[3], row[4], row[5], row[6]}, R[9];
            quat_to_mat(q, R);
            cand[i] = row[0] + (R[0] * x0 + R[1] * x1 + R[2] * x2);
            cand[kLmax + i] = row[1] + (R[3] * x0 + R[4] * x1 + R[5] * x2);
            cand[2 * kLmax + i] = row[2] + (R[6] * x0 + R[7] * x1 + R[8] * x2);
        }
        if (threadIdx.x == 0) s_flag = 0;
        __syncthreads();
        for (int m = 0; m < nk; ++m) {
            float acc = 0.f;
            for (int i = threadIdx.x; i < L; i += blockDim.x)
                for (int c = 0; c < 3; ++c) {
                    const float d = cand[c * kLmax + i] - kept[((size_t)m * 3 + c) * kLmax + i];
                    acc = fmaf(d, d, acc);
                }
            for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                float s = 0.f;
                for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += red[wv];
                if (s < rho * rho * (float)L) s_flag = 1;
            }
            __syncthreads();
        }
        if (!s_flag) {
            for (int i = threadIdx.x; i < L; i += blockDim.x)
                for (int c = 0; c < 3; ++c) kept[((size_t)nk * 3 + c) * kLmax + i] = cand[c * kLmax + i];
            if (threadIdx.x == 0) {
                idx[(size_t)l * k + nk] = p;
                if (e_out) e_out[(size_t)l * k + nk] = E[p];
            }
            ++nk;
        }
        __syncthreads();
    }
    for (int m = nk + threadIdx.x; m < k; m += blockDim.x) {
        idx[(size_t)l * k + m] = -1;
        if (e_out) e_out[(size_t)l * k + m] = __int_as_float(0x7fc00000);
    }
}

// Grid maps: one thread per map point; the ligand-pocket atom-pair energy an atom of each
// ligand type would have there, summed over the pocket atoms of the point's candidate-grid
// cell within the cutoff (residue-level E_MDN is not mapped).
template <int TS>
__global__ void __launch_bounds__(256) k_build_maps(DevPocket pk, const DevParams* __restrict__ prm, float* maps) {
    __shared__ DevParams P;
    for (int k = threadIdx.x; k < (int)(sizeof(DevParams) / 4); k += blockDim.x)
        reinterpret_cast<uint32_t*>(&P)[k] = reinterpret_cast<const uint32_t*>(prm)[k];
    __syncthreads();
    const int nt = P.n_types;
    const int64_t npts = (int64_t)pk.mx * pk.my * pk.mz;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < npts;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(idx % pk.mx), iy = (int)((idx / pk.mx) % pk.my), iz = (int)(idx / ((int64_t)pk.mx * pk.my));
        const float gx = fmaf(pk.mh, (float)ix, pk.mlo[0]), gy = fmaf(pk.mh, (float)iy, pk.mlo[1]),
                    gz = fmaf(pk.mh, (float)iz, pk.mlo[2]);
        uint32_t beg, end;
        cell_range(pk, pk.cell_start, gx, gy, gz, beg, end);
        float acc[kNT];
#pragma unroll
        for (int t = 0; t < kNT; ++t) acc[t] = 0.f;
        for (uint32_t q = beg; q < end; ++q) {
            const int j = __ldg(&pk.cand[q]) & 0x1fff;
            const float4 a = __ldg(&pk.atoms[j]);
            const float dx = gx - a.x, dy = gy - a.y, dz = gz - a.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (!(r2 < P.cut2)) continue;
            const int tj = pk.ptype[j];
            const uint32_t fj = P.tflags[tj];
#pragma unroll
            for (int t = 0; t < kNT; ++t) {
                if (t >= nt) break;
                const uint32_t fi = P.tflags[t];
                const bool hb = ((fi & 2u) && (fj & 4u)) || ((fi & 4u) && (fj & 2u));
                float e;
                if (TS == TRIDS_TERMS_VINA5) {
                    float dd, rinv;
                    e = vina_eval<false>(r2, P.radius[t] + a.w, (fi & fj & 1u) ? 1.f : 0.f, hb ? 1.f : 0.f, P.w, dd,
                                         rinv, nullptr);
                } else {
                    float fr, dRs;
                    const bool mdn = TS == TRIDS_TERMS_TRIDS;
                    e = pair_trids<false>(fmaxf(r2, 1e-12f), P.radius[t] + a.w, hb ? 2 : 0,
                                          mdn ? &P.gmm[t][tj][0] : nullptr, P.gmm_k, mdn, P.w, fr, nullptr, dRs);
                }
                acc[t] += e;
            }
        }
#pragma unroll
        for (int t = 0; t < kNT; ++t)
            if (t < nt) maps[t * npts + idx] = acc[t];
    }
}

__global__ void k_status(const float* state, int n_lig, int P, int n_fields, int* out) {
    const size_t n = (size_t)n_lig * P;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t l = i / P, p = i % P;
        const int s = __float_as_int(state[(l * n_fields + kFieldStatus) * P + p]);
        if (s) atomicOr(out, s);
    }
}

// Item list in plain (ligand, tile) order, written into caller-independent scratch.
__global__ void k_items_natural(int2* items, int n_lig, int tiles) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_lig * tiles) items[i] = make_int2(i / tiles, (i % tiles) * 32);
}


}  // namespace
