// libtrids device code, part 1: constants, Philox, rotations, pair terms, shared-memory
// layout and staging, per-warp scratch, forward kinematics, the packed pair evaluations.
// Included by trids.cu only (one translation unit: the kernels inline everything).
#pragma once

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoPi = 6.28318530717958647692f;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    // Salmon et al., SC'11: ten rounds of two 32x32->64 products, key bumped by the
    // Weyl constants between rounds.
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Block `blk` of the random stream (seed, ligand, pose, loop, purpose).
__device__ __forceinline__ uint4 rand_block(uint64_t seed, uint32_t lig, uint32_t pose, uint32_t loop,
                                            uint32_t purpose, uint32_t blk) {
    return philox4x32_10(make_uint4(pose, lig, (loop << 16) | (purpose << 8) | blk, 0u),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

__device__ __forceinline__ float u01(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }

__device__ __forceinline__ uint32_t pick(uint4 v, int i) {
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/sqrt(x) for normal x > 0 (the callers' arguments: squared distances guarded to
// >= 1e-12, quaternion norms near 1, Adam's bias correction 1 - b2^k): the hardware
// approximation without the subnormal-input handling of rsqrtf, the same value for such x.
__device__ __forceinline__ float rsqrt_normal(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sqrt(x), x >= 0, by the hardware approximation (relative error about 2^-22; subnormal x
// gives 0).  Used by the pose update only (Adam's sqrt(v), the rotation-step length), where
// that error is far below the update's own rounding budget.
__device__ __forceinline__ float sqrt_fast(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// quaternion (w,x,y,z) -> rotation matrix of q/|q|
__device__ __forceinline__ void quat_to_mat(const float q[4], float R[9]) {
    float n = rsqrt_normal(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    float w = q[0] * n, x = q[1] * n, y = q[2] * n, z = q[3] * n;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

// q <- normalize(r (x) q)
__device__ __forceinline__ void quat_premul(const float r[4], float q[4]) {
    float o0 = r[0] * q[0] - r[1] * q[1] - r[2] * q[2] - r[3] * q[3];
    float o1 = r[0] * q[1] + q[0] * r[1] + r[2] * q[3] - r[3] * q[2];
    float o2 = r[0] * q[2] + q[0] * r[2] + r[3] * q[1] - r[1] * q[3];
    float o3 = r[0] * q[3] + q[0] * r[3] + r[1] * q[2] - r[2] * q[1];
    float n = rsqrt_normal(o0 * o0 + o1 * o1 + o2 * o2 + o3 * o3);
    q[0] = o0 * n; q[1] = o1 * n; q[2] = o2 * n; q[3] = o3 * n;
}

__device__ __forceinline__ float wrap_pi(float a) { return a - kTwoPi * floorf((a + kPi) * (1.0f / kTwoPi)); }

// ------------------------------------------------------------------ pair terms
// TRIDS E_dock terms on r (see trids.h).
template <bool TERMS>
__device__ __forceinline__ float pair_trids(float r2, float rsum, int pf, const float4* __restrict__ gmm,
                                            int K, bool inter, const float* __restrict__ w, float& fr,
                                            float* et, float& dRs) {
    const float rinv = rsqrt_normal(r2);
    const float r = r2 * rinv;
    float e0 = 0.f, d0 = 0.f, e1 = 0.f, d1 = 0.f, e2 = 0.f, d2 = 0.f, r2d = 0.f, e3 = 0.f, d3 = 0.f;
    if (inter && r < 5.f) {
        for (int k = 0; k < K; ++k) {
            const float4 g = gmm[k];                           // (pi, mu, -log2(e)/(2 sigma^2), 1/sigma^2)
            const float z = r - g.y;
            const float ex = g.x * ex2_approx(g.z * z * z);
            e0 -= ex;
            d0 = fmaf(ex * z, g.w, d0);
        }
    }
    if (r < 10.f) {
        const float z = r - rsum - 3.f;
        const float gl = __expf(-0.25f * z * z);
        e1 = -gl;
        d1 = 0.5f * gl * z;
    }
    const float dcl = (pf & 2) ? 2.6f : rsum;
    if (r < dcl) {
        const float rr = r < 0.5f ? 0.5f : r;
        e2 = -logf(rr / dcl);
        d2 = r < 0.5f ? 0.f : -rinv;
        r2d = (pf & 2) ? 0.f : 1.f / dcl;
    }
    if ((pf & 2) && r < 3.4f) {
        const float z = r - 2.88f;
        const float gh = __expf(z * z * (-1.f / 0.18f));
        e3 = -gh;
        d3 = gh * z * (1.f / 0.09f);
    }
    const float e = w[0] * e0 + w[1] * e1 + w[2] * e2 + w[3] * e3;
    fr = (w[0] * d0 + w[1] * d1 + w[2] * d2 + w[3] * d3) * rinv;
    if (TERMS) {
        et[0] = e0; et[1] = e1; et[2] = e2; et[3] = e3; et[4] = 0.f;
        dRs = w[1] * (-d1) + w[2] * r2d;
    }
    return e;
}

// ------------------------------------------------------------------ shared layout
struct Smem {
    const DevParams* P;
    const float4* pocket;      // (x, y, z, radius), [M + 1]
    const uint8_t* ptype;      // pocket atom types, [M + 1]
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
    size_t params_bytes, pocket_off, pocket_bytes, ptype_off, ptype_bytes, mbar_off, warp_off, warp_bytes, total;
};

__host__ __device__ inline size_t pose_warp_core_bytes(int Lm, int Tm) {
    return 16 * (size_t)(Lm + 1) + 16 * (size_t)Lm + 48 * (size_t)(Tm > 0 ? Tm : 1) + 16 * (size_t)(Lm + 32) +
           16 * (size_t)(Lm + 1);
}

constexpr size_t kRigidStateBytes = 128;   // sizeof(RigidState), checked below
constexpr size_t kTorStateBytes = 16;      // sizeof(TorState)
constexpr size_t kClockBytes = 8 * (TRIDS_PHASES + 1);   // phase clock of the counting sampler
// per-warp region: [core][rigid pose state][torsion state, 32 lanes][phase clock][per-lane
// dE/dR (parameter-gradient kernels)]
__host__ __device__ inline size_t pose_state_off(int Lm, int Tm) { return align_up(pose_warp_core_bytes(Lm, Tm), 16); }
__host__ __device__ inline size_t pose_hdr_off(int Lm, int Tm) {
    return align_up(pose_state_off(Lm, Tm) + kRigidStateBytes + 32 * kTorStateBytes, 16);
}
__host__ __device__ inline size_t pose_clk_off(int Lm, int Tm) { return pose_hdr_off(Lm, Tm) + sizeof(LigHdr); }
__host__ __device__ inline size_t pose_grs_off(int Lm, int Tm) {
    return align_up(pose_clk_off(Lm, Tm) + kClockBytes, 16);
}
__host__ __device__ inline size_t pose_warp_bytes(int Lm, int Tm, bool params) {
    size_t b = pose_grs_off(Lm, Tm);
    if (params) b += 4 * (size_t)kNT * 32;
    return align_up(b, 128);
}

inline Layout make_layout(int term_set, int M, int Lmax, int Tmax, int warps, bool params) {
    Layout L;
    L.params_bytes = term_set == TRIDS_TERMS_TRIDS ? sizeof(DevParams) : offsetof(DevParams, gmm);
    L.pocket_off = align_up(L.params_bytes, 128);
    L.pocket_bytes = (size_t)(M + 1) * sizeof(float4);
    L.ptype_off = L.pocket_off + L.pocket_bytes;
    L.ptype_bytes = align_up((size_t)(M + 1), 16);
    L.mbar_off = align_up(L.ptype_off + L.ptype_bytes, 16);
    L.warp_off = align_up(L.mbar_off + 16, 128);
    L.warp_bytes = pose_warp_bytes(Lmax, Tmax, params);
    L.total = L.warp_off + L.warp_bytes * warps;
    return L;
}

// Stage the scoring tables and the pocket into shared memory with bulk async copies
// completing on one mbarrier.  Returns false (and sets *err) if the copy did not
// complete within a bounded wait.
__device__ bool stage_block(unsigned char* smem, const DevPocket& pk, size_t params_bytes, size_t pocket_off,
                            size_t ptype_off, size_t mbar_off, int* err) {
    const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(smem + mbar_off);
    const uint32_t bytes_p = (uint32_t)params_bytes;
    const uint32_t bytes_k = (uint32_t)((size_t)(pk.M + 1) * sizeof(float4));
    const uint32_t bytes_t = (uint32_t)align_up((size_t)(pk.M + 1), 16);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar),
                     "r"(bytes_p + bytes_k + bytes_t)
                     : "memory");
        const uint32_t dp = (uint32_t)__cvta_generic_to_shared(smem);
        const uint32_t dk = (uint32_t)__cvta_generic_to_shared(smem + pocket_off);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dp),
            "l"(pk.params), "r"(bytes_p), "r"(mbar)
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dk),
            "l"(pk.atoms), "r"(bytes_k), "r"(mbar)
            : "memory");
        const uint32_t dt = (uint32_t)__cvta_generic_to_shared(smem + ptype_off);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dt),
            "l"(pk.ptype), "r"(bytes_t), "r"(mbar)
            : "memory");
    }
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar)
            : "memory");
    }
    const int ok = __syncthreads_and(done ? 1 : 0);
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    return ok != 0;
}

// ------------------------------------------------------------------ per-warp pose work
// One warp owns one pose.  Per-warp shared memory (pose_warp_bytes):
//   xs  float4[Lm]      world coordinates of the pose's atoms
//   gs  float4[Lm]      dE/dx_i
//   rk  float4[3 Tm]    rows of each torsion's rotation matrix; .w of the three rows holds
//                       the torsion's pivot (parent axis atom, local coordinates)
//   rec float4[Lm + 32] partial ligand-pocket forces, slot (atom + lane)
//   meta int4[Lm + 1]   per atom, one 16-byte record: candidate-list offset of its cell,
//                       candidate blocks | flags | type, first intra block, and the exclusive
//                       prefix of the atoms' work items (.w, Lm + 1 entries)
//   rig RigidState      the pose's rigid sampler state (t, q, Adam moments, saved state,
//                       loop energies, status), one copy per warp: every lane computes the
//                       same values
//   tor TorState[32]    lane k's torsion angle, moments and saved angle
//                       (kept in shared memory, the state holds no registers across the pair
//                       loop, so the plain Vina-form sampler runs 28 warps per SM at 72
//                       registers per thread)
//   hdr LigHdr          the pose's ligand header (sampler kernels)
//   clk u64[7]          per-phase cycle sums and the last lap's time (counting sampler)
//   grs float[kNT][32]  per-lane dE/dR_a (parameter-gradient kernels only)
struct RigidState;
struct TorState;
struct PW {
    RigidState* rig;  // the pose's rigid sampler state (sampler kernels)
    TorState* tor;    // [32] per-lane torsion state (sampler kernels)
    float4* xs;     // [Lm + 1] (x, y, z, radius); xs[Lm] is a far sentinel
    float4* gs;
    float4* rk;
    float4* rec;
    int4* meta;     // per atom: (.x candidate-list offset of its cell; .y candidate blocks of its
                    // cell | type flags << 24 | type << 27 in the pair loop, the atom type in the
                    // atom-pair E_MDN pass; .z first intra-partner block; .w exclusive prefix of
                    // the atom's work items, [Lm + 1])
    float* grs;
    unsigned long long* clk;   // phase clock (counting sampler)
    LigHdr* hdr;               // the pose's ligand header (sampler kernels)
    int lane;
};

__device__ __forceinline__ PW make_pw(unsigned char* smem, size_t warp_off, size_t warp_bytes, int Lm, int Tm) {
    PW W;
    unsigned char* base = smem + warp_off + warp_bytes * (threadIdx.x >> 5);
    W.xs = reinterpret_cast<float4*>(base);
    W.gs = W.xs + Lm + 1;
    W.rk = W.gs + Lm;
    W.rec = W.rk + 3 * (Tm > 0 ? Tm : 1);
    W.meta = reinterpret_cast<int4*>(W.rec + Lm + 32);
    W.rig = reinterpret_cast<RigidState*>(base + pose_state_off(Lm, Tm));
    W.tor = reinterpret_cast<TorState*>(base + pose_state_off(Lm, Tm) + kRigidStateBytes);
    W.grs = reinterpret_cast<float*>(base + pose_grs_off(Lm, Tm));
    W.clk = reinterpret_cast<unsigned long long*>(base + pose_clk_off(Lm, Tm));
    W.hdr = reinterpret_cast<LigHdr*>(base + pose_hdr_off(Lm, Tm));
    W.lane = threadIdx.x & 31;
    return W;
}

__device__ __forceinline__ float warp_sum(float v) {
    // butterfly: every lane ends with the same, fixed-order sum
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

struct ParamAcc {
    float gw[5];
};

// Branch-free Vina-form pair on surface distance d = r - rsum.  hyd / hb are 1 for a
// hydrophobic / donor-acceptor pair, else 0.  Returns the weighted energy and its
// derivative dd = dE/dd (= dE/dr); rinv = 1/r.  With TERMS, et[] gets the unweighted
// terms.  Piecewise pieces use saturate(): the kinks sit where the clamp engages.
template <bool TERMS>
__device__ __forceinline__ float vina_eval(float r2, float rsum, float hyd, float hb, const float w[5], float& dd,
                                           float& rinv, float* et) {
    constexpr float kC1 = -5.770780163555854f;   // -4 log2(e): exp(-(d/0.5)^2) = 2^(kC1 d^2)
    constexpr float kC2 = -1.4426950408889634f;  // -log2(e)
    const float rr = fmaxf(r2, 1e-12f);
    rinv = rsqrt_normal(rr);
    const float d = rr * rinv - rsum;
    const float g1 = ex2_approx(d * d * kC1);
    const float b = fmaf(0.5f, d, -1.5f);
    const float g2 = ex2_approx(b * b * kC2);
    const float dn = fminf(d, 0.f);
    const float w3h = w[3] * hyd, w4h = w[4] * hb;
    const float hraw = 1.5f - d;
    const float hy = __saturatef(hraw);
    const float hbraw = d * (-1.f / 0.7f);
    const float hbv = __saturatef(hbraw);
    float e = w[0] * g1;
    e = fmaf(w[1], g2, e);
    e = fmaf(w[2], dn * dn, e);
    e = fmaf(w3h, hy, e);
    e = fmaf(w4h, hbv, e);
    float g = w[0] * (-8.f * d * g1);
    g = fmaf(w[1], -b * g2, g);
    g = fmaf(w[2], 2.f * dn, g);
    g -= (hy == hraw) ? w3h : 0.f;
    g -= (hbv == hbraw) ? w4h * (1.f / 0.7f) : 0.f;
    dd = g;
    if (TERMS) {
        et[0] = g1; et[1] = g2; et[2] = dn * dn; et[3] = hyd * hy; et[4] = hb * hbv;
    }
    return e;
}

// Constants of the paired Vina-form evaluation; both halves of each float2 are equal.
struct VinaX2 {
    float2 w0, w1, w2, n0, n2, c1, c2, half, m15, m1, p15, m07, k07, tiny;
    float w3, w4;
};

// Work counts of the counting sampler, per lane: in-cutoff pairs and, for the TRIDS terms,
// the pairs inside the E_clash and E_Hbond ranges (all three doubled: an intra pair is seen
// from both of its atoms), atom-pair E_MDN pairs inside 5 A, residue atoms scanned for the
// residue minima and (atom, residue) pairs inside 5 A.
struct WorkCount {
    uint32_t pairs = 0, clash = 0, hb = 0, mdn = 0, scan = 0, res = 0;
};

// The ligand atom's flag-dependent piece of the Vina-form pair.  A type that is
// hydrophobic but neither donor nor acceptor meets only the hydrophobic term
// w3 sat(1.5 - d) (with hydrophobic candidates); a donor and/or acceptor type that is not
// hydrophobic meets only the H-bond term w4 sat(-d / 0.7) (with candidates of the
// complementary flag).  Either is one masked term w sat(a - b d) with per-atom (a, b, w)
// and candidate-flag mask m, evaluated once instead of twice; a type with no flags gets
// m = 0.  The full two-term evaluation serves parameter sets with a type that is both.
struct FlagTerm {
    uint32_t m;     // candidate flag bits (low entry; shifted by 16 for the high entry)
    float nb, a;    // -b, a
    float w;        // weight
    float b;        // b
    uint32_t mh, mb;   // two-term form: hydrophobic / donor-acceptor candidate bits
};

// The single flag term of a ligand type from its table row (DevParams::ftab).
__device__ __forceinline__ FlagTerm flag_term_of(float4 t) {
    FlagTerm F;
    F.m = __float_as_uint(t.x);
    F.nb = t.y;
    F.a = t.z;
    F.w = t.w;
    F.b = -t.y;
    F.mh = F.mb = 0u;
    return F;
}

// fi = the ligand atom's type flags (bit0 hydrophobic, bit1 donor, bit2 acceptor); w3, w4
// the hydrophobic and H-bond weights.
__device__ __forceinline__ FlagTerm make_flag_term(uint32_t fi, float w3, float w4) {
    FlagTerm F;
    F.mh = (fi & 1u) << 13;
    F.mb = (((fi & 2u) << 1) | ((fi & 4u) >> 1)) << 13;   // donor_i -> acceptor_j, acceptor_i -> donor_j
    const bool hyd = (fi & 1u) != 0u;
    F.m = hyd ? F.mh : F.mb;
    const float nb = hyd ? -1.f : -1.f / 0.7f, a = hyd ? 1.5f : 0.f, b = hyd ? 1.f : 1.f / 0.7f;
    F.nb = nb;
    F.a = a;
    F.b = b;
    F.w = hyd ? w3 : w4;
    return F;
}

__device__ __forceinline__ VinaX2 make_vina_x2(const float w[5]) {
    VinaX2 K;
    K.w0 = make_float2(w[0], w[0]);
    K.w1 = make_float2(w[1], w[1]);
    K.w2 = make_float2(w[2], w[2]);
    K.n0 = make_float2(8.f * w[0], 8.f * w[0]);
    K.n2 = make_float2(-2.f * w[2], -2.f * w[2]);
    K.c1 = make_float2(-5.770780163555854f, -5.770780163555854f);
    K.c2 = make_float2(-1.4426950408889634f, -1.4426950408889634f);
    K.half = make_float2(0.5f, 0.5f);
    K.m15 = make_float2(-1.5f, -1.5f);
    K.m1 = make_float2(-1.f, -1.f);
    K.p15 = make_float2(1.5f, 1.5f);
    K.m07 = make_float2(-1.f / 0.7f, -1.f / 0.7f);
    K.k07 = make_float2(1.f / 0.7f, 1.f / 0.7f);
    K.tiny = make_float2(1e-12f, 1e-12f);
    K.w3 = w[3];
    K.w4 = w[4];
    return K;
}

// The same Vina-form pair as vina_eval, for the two candidates packed in one 32-bit
// candidate-list word, on the packed FP32 pipe (f32x2).  The gradient's sign is folded
// into the constants so that no operand needs negating: with p = x_j - x_i and
// ng = -dE/dd, the force on atom i gains ng / r * p.  nxy = -(x_i, y_i) and
// nzr = -(z_i, R_i); F holds the ligand atom's flag-term operands (ONE: the single masked
// term of FlagTerm; else both terms with F.mh / F.mb selecting the candidate's
// hydrophobic / donor-acceptor bits).  in-cutoff pairs are masked by multiplying with
// 0/1, which is exact for the finite values every candidate (the far sentinel included)
// produces.  Both forms give the same bits: the term the single form leaves out is
// exactly zero for such a type.
template <bool COUNT, bool ONE>
__device__ __forceinline__ void vina_x2(uint32_t wd, const float4* __restrict__ src, float2 nxy, float2 nzr,
                                        float cut2, const VinaX2& K, const FlagTerm& F, float2& eb,
                                        float& ax, float& ay, float& az, uint32_t& cnt, uint32_t cw) {
    const float4 a = src[wd & 0x1fffu], c = src[(wd >> 16) & 0x1fffu];
    const float2 pm = make_float2(1.f, -1.f);
    const float2 pa = __fadd2_rn(make_float2(a.x, a.y), nxy);
    const float2 qa = __ffma2_rn(make_float2(a.z, a.w), pm, nzr);     // (z_j - z_i, -(R_i + R_j))
    const float2 pc = __fadd2_rn(make_float2(c.x, c.y), nxy);
    const float2 qc = __ffma2_rn(make_float2(c.z, c.w), pm, nzr);
    // r^2 + 2e-12 (1e-12 added to each of two squares): keeps 1/r finite at r = 0
    const float2 sa = __ffma2_rn(pa, pa, K.tiny), sc = __ffma2_rn(pc, pc, K.tiny);
    const float2 rr = make_float2(fmaf(qa.x, qa.x, sa.x) + sa.y, fmaf(qc.x, qc.x, sc.x) + sc.y);
    const float2 in = make_float2(rr.x < cut2 ? 1.f : 0.f, rr.y < cut2 ? 1.f : 0.f);
    const float2 ri = make_float2(rsqrt_normal(rr.x), rsqrt_normal(rr.y));
    const float2 d = make_float2(fmaf(rr.x, ri.x, qa.y), fmaf(rr.y, ri.y, qc.y));
    const float2 q1 = __fmul2_rn(__fmul2_rn(d, d), K.c1);
    const float2 g1 = make_float2(ex2_approx(q1.x), ex2_approx(q1.y));
    const float2 b = __ffma2_rn(d, K.half, K.m15);
    const float2 q2 = __fmul2_rn(__fmul2_rn(b, b), K.c2);
    const float2 g2 = make_float2(ex2_approx(q2.x), ex2_approx(q2.y));
    const float2 dn = make_float2(fminf(d.x, 0.f), fminf(d.y, 0.f));
    float2 e = __fmul2_rn(K.w0, g1);
    e = __ffma2_rn(K.w1, g2, e);
    e = __ffma2_rn(K.w2, __fmul2_rn(dn, dn), e);
    float2 ng = __fmul2_rn(__fmul2_rn(d, K.n0), g1);                    // 8 w0 d g1
    ng = __ffma2_rn(__fmul2_rn(b, K.w1), g2, ng);                       // + w1 b g2
    ng = __ffma2_rn(K.n2, dn, ng);                                      // - 2 w2 dn
    if constexpr (ONE) {
        const float2 hr = __ffma2_rn(d, make_float2(F.nb, F.nb), make_float2(F.a, F.a));   // a - b d
        const float2 hy = make_float2(__saturatef(hr.x), __saturatef(hr.y));
        const float2 ih = make_float2(hy.x == hr.x ? 1.f : 0.f, hy.y == hr.y ? 1.f : 0.f);
        const float2 wf = make_float2((wd & F.m) ? F.w : 0.f, (wd & (F.m << 16)) ? F.w : 0.f);
        e = __ffma2_rn(wf, hy, e);
        ng = __ffma2_rn(ih, __fmul2_rn(wf, make_float2(F.b, F.b)), ng);  // + w b inside the ramp
    } else {
        const float2 hr = __ffma2_rn(d, K.m1, K.p15);                  // 1.5 - d
        const float2 hy = make_float2(__saturatef(hr.x), __saturatef(hr.y));
        const float2 ih = make_float2(hy.x == hr.x ? 1.f : 0.f, hy.y == hr.y ? 1.f : 0.f);
        const float2 br = __fmul2_rn(d, K.m07);                        // -d / 0.7
        const float2 hb = make_float2(__saturatef(br.x), __saturatef(br.y));
        const float2 ib = make_float2(hb.x == br.x ? 1.f : 0.f, hb.y == br.y ? 1.f : 0.f);
        const float2 w3h = make_float2((wd & F.mh) ? K.w3 : 0.f, (wd & (F.mh << 16)) ? K.w3 : 0.f);
        const float2 w4h = make_float2((wd & F.mb) ? K.w4 : 0.f, (wd & (F.mb << 16)) ? K.w4 : 0.f);
        e = __ffma2_rn(w3h, hy, e);
        e = __ffma2_rn(w4h, hb, e);
        ng = __ffma2_rn(ih, w3h, ng);
        ng = __ffma2_rn(ib, __fmul2_rn(w4h, K.k07), ng);
    }
    eb = __ffma2_rn(e, in, eb);
    const float2 f = __fmul2_rn(__fmul2_rn(ng, in), ri);
    float2 axy = make_float2(ax, ay);
    axy = __ffma2_rn(make_float2(f.x, f.x), pa, axy); az = fmaf(f.x, qa.x, az);
    axy = __ffma2_rn(make_float2(f.y, f.y), pc, axy); az = fmaf(f.y, qc.x, az);
    ax = axy.x; ay = axy.y;
    if (COUNT) cnt += ((rr.x < cut2) + (rr.y < cut2)) * cw;
}

__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The TRIDS atom-pair terms (pair_trids) for the two candidates of one candidate-list
// word, branch-free on the packed FP32 pipe: every term is evaluated and masked (r^2 <
// min(cutoff^2, 100), which also ends E_long at 10 A; r < d_clash; donor-acceptor pair with
// r < 3.4; r < 5 for the atom-pair E_MDN) by multiplying with 0/1, exact for the finite
// values every candidate gives.  r^2 carries 1e-12 per square term (keeps 1/r finite at r =
// 0).  exp and log
// go through ex2 / lg2.  mb selects the candidate's donor/acceptor flag bits (low entry;
// shifted by 16 for the high entry).  gmm (term set 1, ligand-pocket pairs only; else
// null): the ligand atom type's row of (pi, mu, -1/(2 sigma^2), 1/sigma^2) by pocket type.
template <bool COUNT>
__device__ __forceinline__ void trids_x2(uint32_t wd, const float4* __restrict__ src, float2 nxy, float2 nzr,
                                         float cut2, const float w[5], uint32_t mb, const float4* __restrict__ gmm,
                                         const uint8_t* __restrict__ ptype, int K, float2& eb, float& ax, float& ay,
                                         float& az, WorkCount& wc, uint32_t cw) {
    constexpr float kL2e = 1.4426950408889634f, kLn2 = 0.6931471805599453f;
    const uint32_t ja = wd & 0x1fffu, jb = (wd >> 16) & 0x1fffu;
    const float4 a = src[ja], c = src[jb];
    const float2 pm = make_float2(1.f, -1.f);
    const float2 pa = __fadd2_rn(make_float2(a.x, a.y), nxy);
    const float2 qa = __ffma2_rn(make_float2(a.z, a.w), pm, nzr);      // (z_j - z_i, -(R_i + R_j))
    const float2 pc = __fadd2_rn(make_float2(c.x, c.y), nxy);
    const float2 qc = __ffma2_rn(make_float2(c.z, c.w), pm, nzr);
    const float2 tiny = make_float2(1e-12f, 1e-12f);
    const float2 sa = __ffma2_rn(pa, pa, tiny), sc = __ffma2_rn(pc, pc, tiny);
    const float2 rr = make_float2(fmaf(qa.x, qa.x, sa.x) + sa.y, fmaf(qc.x, qc.x, sc.x) + sc.y);
    // one mask for every term: E_long ends at 10 A, E_clash and E_Hbond far inside it
    const float c2 = fminf(cut2, 100.f);
    const float2 in = make_float2(rr.x < c2 ? 1.f : 0.f, rr.y < c2 ? 1.f : 0.f);
    const float2 ri = make_float2(rsqrt_normal(rr.x), rsqrt_normal(rr.y));
    const float2 r = __fmul2_rn(rr, ri);
    const float2 rs = make_float2(-qa.y, -qc.y);                            // R_i + R_j
    const float2 hb = make_float2((wd & mb) ? 1.f : 0.f, (wd & (mb << 16)) ? 1.f : 0.f);
    // E_long: -exp(-(r - R_i - R_j - 3)^2 / 4); dE/dr = 0.5 gl z
    const float2 z = __fadd2_rn(r, make_float2(qa.y - 3.f, qc.y - 3.f));
    const float2 al = __fmul2_rn(__fmul2_rn(z, z), make_float2(-0.25f * kL2e, -0.25f * kL2e));
    const float2 gl = make_float2(ex2_approx(al.x), ex2_approx(al.y));
    float2 e = __fmul2_rn(make_float2(-w[1], -w[1]), gl);
    float2 d = __fmul2_rn(__fmul2_rn(make_float2(0.5f * w[1], 0.5f * w[1]), gl), z);
    // E_clash: -ln(max(r, 0.5) / d_clash) for r < d_clash (2.6 for a donor-acceptor pair,
    // else R_i + R_j); dE/dr = -1/r above 0.5
    const float2 dcl = make_float2(hb.x != 0.f ? 2.6f : rs.x, hb.y != 0.f ? 2.6f : rs.y);
    const float2 mcl = make_float2(r.x < dcl.x ? 1.f : 0.f, r.y < dcl.y ? 1.f : 0.f);
    const float2 lr = make_float2(lg2_approx(fmaxf(r.x, 0.5f)) - lg2_approx(dcl.x),
                                  lg2_approx(fmaxf(r.y, 0.5f)) - lg2_approx(dcl.y));
    e = __ffma2_rn(__fmul2_rn(mcl, make_float2(-w[2] * kLn2, -w[2] * kLn2)), lr, e);
    const float2 m05 = make_float2(r.x < 0.5f ? 0.f : mcl.x, r.y < 0.5f ? 0.f : mcl.y);
    d = __ffma2_rn(__fmul2_rn(m05, make_float2(-w[2], -w[2])), ri, d);
    // E_Hbond: -exp(-(r - 2.88)^2 / (2 0.3^2)) for donor-acceptor pairs with r < 3.4
    const float2 mh = make_float2(r.x < 3.4f ? hb.x : 0.f, r.y < 3.4f ? hb.y : 0.f);
    const float2 zh = __fadd2_rn(r, make_float2(-2.88f, -2.88f));
    const float2 ah = __fmul2_rn(__fmul2_rn(zh, zh), make_float2(-kL2e / 0.18f, -kL2e / 0.18f));
    const float2 gh = __fmul2_rn(mh, make_float2(ex2_approx(ah.x), ex2_approx(ah.y)));
    e = __ffma2_rn(make_float2(-w[3], -w[3]), gh, e);
    d = __ffma2_rn(__fmul2_rn(make_float2(w[3] / 0.09f, w[3] / 0.09f), gh), zh, d);
    // E_MDN over atom pairs (term set 1, ligand-pocket): -sum_k pi_k exp(-(r - mu_k)^2 / (2 sigma_k^2))
    if (gmm) {
        const float2 m5 = make_float2(r.x < 5.f ? 1.f : 0.f, r.y < 5.f ? 1.f : 0.f);
        const float4* __restrict__ ga = gmm + ptype[ja] * kKP;
        const float4* __restrict__ gc = gmm + ptype[jb] * kKP;
        float2 e0 = make_float2(0.f, 0.f), d0 = make_float2(0.f, 0.f);
        for (int k = 0; k < K; ++k) {
            const float4 u = ga[k], v = gc[k];
            const float2 zz = __fadd2_rn(r, make_float2(-u.y, -v.y));
            const float2 ar = __fmul2_rn(__fmul2_rn(zz, zz), make_float2(u.z, v.z));
            const float2 ex = __fmul2_rn(make_float2(u.x, v.x), make_float2(ex2_approx(ar.x), ex2_approx(ar.y)));
            e0 = __fadd2_rn(e0, ex);
            d0 = __ffma2_rn(__fmul2_rn(ex, zz), make_float2(u.w, v.w), d0);
        }
        e = __ffma2_rn(__fmul2_rn(m5, make_float2(-w[0], -w[0])), e0, e);
        d = __ffma2_rn(__fmul2_rn(m5, make_float2(w[0], w[0])), d0, d);
    }
    eb = __ffma2_rn(e, in, eb);
    // force on i: dE/dr / r * (x_i - x_j) = -dE/dr / r * p
    const float2 f = __fmul2_rn(__fmul2_rn(d, in), make_float2(-ri.x, -ri.y));
    float2 axy = make_float2(ax, ay);
    axy = __ffma2_rn(make_float2(f.x, f.x), pa, axy); az = fmaf(f.x, qa.x, az);
    axy = __ffma2_rn(make_float2(f.y, f.y), pc, axy); az = fmaf(f.y, qc.x, az);
    ax = axy.x; ay = axy.y;
    if (COUNT) {
        const bool ia = rr.x < cut2, ic = rr.y < cut2;
        wc.pairs += (ia + ic) * cw;
        wc.clash += ((ia && mcl.x != 0.f) + (ic && mcl.y != 0.f)) * cw;
        wc.hb += ((ia && mh.x != 0.f) + (ic && mh.y != 0.f)) * cw;
    }
}

// Candidate-grid cell range (entries [beg, end) of pk.cand) of a point; empty outside
// the grid, where no pocket atom lies within the cutoff.
__device__ __forceinline__ void cell_range(const DevPocket& pk, const uint32_t* __restrict__ starts, float x, float y,
                                           float z, uint32_t& beg, uint32_t& end) {
    const float fx = (x - pk.gx) * pk.inv_h, fy = (y - pk.gy) * pk.inv_h, fz = (z - pk.gz) * pk.inv_h;
    beg = end = 0;
    if (fx >= 0.f && fy >= 0.f && fz >= 0.f && fx < (float)pk.nx && fy < (float)pk.ny && fz < (float)pk.nz) {
        const int cx = min((int)fx, pk.nx - 1), cy = min((int)fy, pk.ny - 1), cz = min((int)fz, pk.nz - 1);
        const size_t cell = ((size_t)cz * pk.ny + cy) * pk.nx + cx;
        beg = __ldg(&starts[cell]);
        end = __ldg(&starts[cell + 1]);
    }
}

// The part of a point's cell list the point needs: the list's first entry in beg and, in
// n, the count levels[cell][k] of the reach level that covers the point's distance from the
// cell centre (delta <= (k + 1) / kReachLevels of the half diagonal, k =
// floor(delta / half diagonal * kReachLevels)); n = 0 outside the grid.  For the candidate
// lists the counts are 8-entry blocks, for the near and residue lists entries.
__device__ __forceinline__ void cell_levels(const DevPocket& pk, const uint32_t* __restrict__ starts,
                                            const uint16_t* __restrict__ levels, float x, float y, float z,
                                            uint32_t& beg, int& n) {
    const float fx = (x - pk.gx) * pk.inv_h, fy = (y - pk.gy) * pk.inv_h, fz = (z - pk.gz) * pk.inv_h;
    beg = 0;
    n = 0;
    if (fx >= 0.f && fy >= 0.f && fz >= 0.f && fx < (float)pk.nx && fy < (float)pk.ny && fz < (float)pk.nz) {
        const int cx = min((int)fx, pk.nx - 1), cy = min((int)fy, pk.ny - 1), cz = min((int)fz, pk.nz - 1);
        const size_t cell = ((size_t)cz * pk.ny + cy) * pk.nx + cx;
        const float ux = fx - ((float)cx + 0.5f), uy = fy - ((float)cy + 0.5f), uz = fz - ((float)cz + 0.5f);
        // delta / half diagonal = |u| / (sqrt(3) / 2), in cell units
        constexpr float kScale = (float)kReachLevels * 1.1547005383792515f;
        const int k = min(kReachLevels - 1, (int)(sqrtf(fmaf(uz, uz, fmaf(uy, uy, ux * ux))) * kScale));
        beg = __ldg(&starts[cell]);
        n = __ldg(&levels[cell * kReachLevels + k]);
    }
}

// Grid-map cell of a point: true (and the cell + fractions in c / f) when maps are in use
// and all 8 corners of the point's cell lie inside the map domain.
__device__ __forceinline__ bool map_cell(const DevPocket& pk, float x, float y, float z, float4* cf) {
    if (!pk.use_maps) return false;
    const float ux = (x - pk.mlo[0]) * pk.inv_mh, uy = (y - pk.mlo[1]) * pk.inv_mh, uz = (z - pk.mlo[2]) * pk.inv_mh;
    if (!(ux >= 0.f && uy >= 0.f && uz >= 0.f && ux < (float)(pk.mx - 1) && uy < (float)(pk.my - 1) &&
          uz < (float)(pk.mz - 1)))
        return false;
    if (cf) *cf = make_float4(ux, uy, uz, 0.f);
    return true;
}

// Forward kinematics of the warp's pose.  Lane k < T builds torsion k's rotation
// (Rodrigues, angle th held by lane k) and pivot into W.rk; then each lane places its
// atoms: the torsions that move an atom (its fragment's torsion and that torsion's
// ancestors, the set bits of its mask), deepest first, about their input-geometry axes --
// the axis atoms of a torsion are never moved by the torsions below it -- then
// x = t + R(q) z.  Torsions are numbered breadth-first from the root, so a parent's
// number is below its children's and deepest first is descending bit order.
__device__ void fk_warp(const DevBatch& B, const LigHdr& h, const PW& W, const float t[3], const float q[4], float th,
                        const float* __restrict__ rad) {
    const int T = h.n_tor, L = h.n_atoms;
    if (W.lane < T) {
        const float4 u = __ldg(&B.tor_u[h.tor_off + W.lane]);
        float s, c;
        sincosf(th, &s, &c);
        const float kc = 1.f - c;
        const float4 pv = __ldg(&B.tor_p[h.tor_off + W.lane]);
        W.rk[3 * W.lane + 0] = make_float4(c + kc * u.x * u.x, kc * u.x * u.y - s * u.z, kc * u.x * u.z + s * u.y, pv.x);
        W.rk[3 * W.lane + 1] = make_float4(kc * u.y * u.x + s * u.z, c + kc * u.y * u.y, kc * u.y * u.z - s * u.x, pv.y);
        W.rk[3 * W.lane + 2] = make_float4(kc * u.z * u.x - s * u.y, kc * u.z * u.y + s * u.x, c + kc * u.z * u.z, pv.z);
    }
    __syncwarp();
    float R[9];
    quat_to_mat(q, R);
    for (int i = W.lane; i < L; i += 32) {
        const float4 y = __ldg(&B.atom_y[h.atom_off + i]);
        float x0 = y.x, x1 = y.y, x2 = y.z;
        // the torsions that move atom i, deepest (highest number) first
        for (uint32_t m = __ldg(&B.atom_mask[h.atom_off + i]); m;) {
            const int k = 31 - __clz(m);
            m ^= 1u << k;
            const float4 r0 = W.rk[3 * k], r1 = W.rk[3 * k + 1], r2 = W.rk[3 * k + 2];
            const float vx = x0 - r0.w, vy = x1 - r1.w, vz = x2 - r2.w;
            x0 = r0.w + (r0.x * vx + r0.y * vy + r0.z * vz);
            x1 = r1.w + (r1.x * vx + r1.y * vy + r1.z * vz);
            x2 = r2.w + (r2.x * vx + r2.y * vy + r2.z * vz);
        }
        W.xs[i] = make_float4(t[0] + (R[0] * x0 + R[1] * x1 + R[2] * x2), t[1] + (R[3] * x0 + R[4] * x1 + R[5] * x2),
                              t[2] + (R[6] * x0 + R[7] * x1 + R[8] * x2), rad[__float_as_int(y.w)]);
    }
    if (W.lane == 0) W.xs[B.max_atoms] = make_float4(1e6f, 1e6f, 1e6f, 0.f);   // padding target
    __syncwarp();
}


}  // namespace
