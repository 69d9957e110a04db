// libtrids: device code and C-ABI entry points for gradient-guided pose sampling
// (TRIDS, arXiv 2510.24186, Sec. 2 "Scoring functions" and "Conformation sampling",
// Sec. 4 items 1-4) on sm_103a.
//
// Thread mapping: one thread per pose.  A warp owns 32 poses of ONE ligand, so all
// lanes run the same topology (forward kinematics, intra-ligand pair list, adjoint
// and update loops are uniform across the warp) and only the ligand-pocket pair loop
// diverges.  Per-warp shared memory holds the poses' coordinates and forces as
// [component][atom][lane] (conflict-free); every block stages the scoring tables and
// the pocket (float4 per atom) into shared memory with one bulk asynchronous copy.
// Ligand-pocket pairs are culled by a precomputed candidate grid (each cell lists the
// pocket atoms that can lie within the cutoff of any point of the cell).  Every sum
// runs in a fixed order inside one thread, so results are bit-reproducible and the
// persistent and per-launch forms agree bit for bit.
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

// =============================================================== device helpers
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

// quaternion (w,x,y,z) -> rotation matrix of q/|q|
__device__ __forceinline__ void quat_to_mat(const float q[4], float R[9]) {
    float n = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
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
    float n = rsqrtf(o0 * o0 + o1 * o1 + o2 * o2 + o3 * o3);
    q[0] = o0 * n; q[1] = o1 * n; q[2] = o2 * n; q[3] = o3 * n;
}

__device__ __forceinline__ float wrap_pi(float a) { return a - kTwoPi * floorf((a + kPi) * (1.0f / kTwoPi)); }

// ------------------------------------------------------------------ pair terms
// TRIDS E_dock terms on r (see trids.h).
template <bool TERMS>
__device__ __forceinline__ float pair_trids(float r2, float rsum, int pf, const float4* __restrict__ gmm,
                                            int K, bool inter, const float* __restrict__ w, float& fr,
                                            float* et, float& dRs) {
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    float e0 = 0.f, d0 = 0.f, e1 = 0.f, d1 = 0.f, e2 = 0.f, d2 = 0.f, r2d = 0.f, e3 = 0.f, d3 = 0.f;
    if (inter && r < 5.f) {
        for (int k = 0; k < K; ++k) {
            const float4 g = gmm[k];
            const float z = r - g.y;
            const float ex = g.x * __expf(g.z * z * z);
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
           12 * (size_t)Lm + 4 * (size_t)(Lm + 1);
}

constexpr size_t kRigidStateBytes = 128;   // sizeof(RigidState), checked below
constexpr size_t kTorStateBytes = 16;      // sizeof(TorState)
// per-warp region: [core][rigid pose state][torsion state, 32 lanes][per-lane dE/dR
// (parameter-gradient kernels)]
__host__ __device__ inline size_t pose_state_off(int Lm, int Tm) { return align_up(pose_warp_core_bytes(Lm, Tm), 16); }
__host__ __device__ inline size_t pose_grs_off(int Lm, int Tm) {
    return align_up(pose_state_off(Lm, Tm) + kRigidStateBytes + 32 * kTorStateBytes, 16);
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
//   rk  float4[3 Tm]    rows of each torsion's rotation matrix
//   rec float4[Lm + 32] partial ligand-pocket forces, slot (atom + lane)
//   cs  uint32[Lm]      candidate-list offset of each atom's cell
//   pre int[Lm + 1]     exclusive prefix of each atom's candidate blocks
//   rig RigidState      the pose's rigid sampler state (t, q, Adam moments, saved state,
//                       loop energies, status), one copy per warp: every lane computes the
//                       same values
//   tor TorState[32]    lane k's torsion angle, moments and saved angle
//                       (kept in shared memory, the state holds no registers across the pair
//                       loop: the sampler fits 96 registers per thread, 20 warps per SM)
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
    uint32_t* cs;   // per atom: candidate-list offset of its cell
    int* cb;        // per atom: candidate blocks of its cell
    int* ip;        // per atom: first intra-partner block
    int* pre;
    float* grs;
    int lane;
};

__device__ __forceinline__ PW make_pw(unsigned char* smem, size_t warp_off, size_t warp_bytes, int Lm, int Tm) {
    PW W;
    unsigned char* base = smem + warp_off + warp_bytes * (threadIdx.x >> 5);
    W.xs = reinterpret_cast<float4*>(base);
    W.gs = W.xs + Lm + 1;
    W.rk = W.gs + Lm;
    W.rec = W.rk + 3 * (Tm > 0 ? Tm : 1);
    W.cs = reinterpret_cast<uint32_t*>(W.rec + Lm + 32);
    W.cb = reinterpret_cast<int*>(W.cs + Lm);
    W.ip = W.cb + Lm;
    W.pre = W.ip + Lm;
    W.rig = reinterpret_cast<RigidState*>(base + pose_state_off(Lm, Tm));
    W.tor = reinterpret_cast<TorState*>(base + pose_state_off(Lm, Tm) + kRigidStateBytes);
    W.grs = reinterpret_cast<float*>(base + pose_grs_off(Lm, Tm));
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

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

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
    rinv = rsqrtf(rr);
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
// nzr = -(z_i, R_i); mh / mb select the candidate's hydrophobic / donor-acceptor flag
// bits (low entry; shifted by 16 for the high entry).  in-cutoff pairs are masked by
// multiplying with 0/1, which is exact for the finite values every candidate (the far
// sentinel included) produces.
template <bool COUNT>
__device__ __forceinline__ void vina_x2(uint32_t wd, const float4* __restrict__ src, float2 nxy, float2 nzr,
                                        float cut2, const VinaX2& K, uint32_t mh, uint32_t mb, float2& eb,
                                        float& ax, float& ay, float& az, uint32_t& cnt, uint32_t cw) {
    const float4 a = src[wd & 0x1fffu], c = src[(wd >> 16) & 0x1fffu];
    const float2 pm = make_float2(1.f, -1.f);
    const float2 pa = __fadd2_rn(make_float2(a.x, a.y), nxy);
    const float2 qa = __ffma2_rn(make_float2(a.z, a.w), pm, nzr);     // (z_j - z_i, -(R_i + R_j))
    const float2 pc = __fadd2_rn(make_float2(c.x, c.y), nxy);
    const float2 qc = __ffma2_rn(make_float2(c.z, c.w), pm, nzr);
    const float2 sa = __fmul2_rn(pa, pa), sc = __fmul2_rn(pc, pc);
    const float2 r2 = make_float2(fmaf(qa.x, qa.x, sa.x) + sa.y, fmaf(qc.x, qc.x, sc.x) + sc.y);
    const float2 in = make_float2(r2.x < cut2 ? 1.f : 0.f, r2.y < cut2 ? 1.f : 0.f);
    const float2 rr = __fadd2_rn(r2, K.tiny);
    const float2 ri = make_float2(rsqrtf(rr.x), rsqrtf(rr.y));
    const float2 d = make_float2(fmaf(rr.x, ri.x, qa.y), fmaf(rr.y, ri.y, qc.y));
    const float2 q1 = __fmul2_rn(__fmul2_rn(d, d), K.c1);
    const float2 g1 = make_float2(ex2_approx(q1.x), ex2_approx(q1.y));
    const float2 b = __ffma2_rn(d, K.half, K.m15);
    const float2 q2 = __fmul2_rn(__fmul2_rn(b, b), K.c2);
    const float2 g2 = make_float2(ex2_approx(q2.x), ex2_approx(q2.y));
    const float2 dn = make_float2(fminf(d.x, 0.f), fminf(d.y, 0.f));
    const float2 hr = __ffma2_rn(d, K.m1, K.p15);                      // 1.5 - d
    const float2 hy = make_float2(__saturatef(hr.x), __saturatef(hr.y));
    const float2 ih = make_float2(hy.x == hr.x ? 1.f : 0.f, hy.y == hr.y ? 1.f : 0.f);
    const float2 br = __fmul2_rn(d, K.m07);                            // -d / 0.7
    const float2 hb = make_float2(__saturatef(br.x), __saturatef(br.y));
    const float2 ib = make_float2(hb.x == br.x ? 1.f : 0.f, hb.y == br.y ? 1.f : 0.f);
    const float2 w3h = make_float2((wd & mh) ? K.w3 : 0.f, (wd & (mh << 16)) ? K.w3 : 0.f);
    const float2 w4h = make_float2((wd & mb) ? K.w4 : 0.f, (wd & (mb << 16)) ? K.w4 : 0.f);
    float2 e = __fmul2_rn(K.w0, g1);
    e = __ffma2_rn(K.w1, g2, e);
    e = __ffma2_rn(K.w2, __fmul2_rn(dn, dn), e);
    e = __ffma2_rn(w3h, hy, e);
    e = __ffma2_rn(w4h, hb, e);
    float2 ng = __fmul2_rn(__fmul2_rn(d, K.n0), g1);                    // 8 w0 d g1
    ng = __ffma2_rn(__fmul2_rn(b, K.w1), g2, ng);                       // + w1 b g2
    ng = __ffma2_rn(K.n2, dn, ng);                                      // - 2 w2 dn
    ng = __ffma2_rn(ih, w3h, ng);
    ng = __ffma2_rn(ib, __fmul2_rn(w4h, K.k07), ng);
    eb = __ffma2_rn(e, in, eb);
    const float2 f = __fmul2_rn(__fmul2_rn(ng, in), ri);
    float2 axy = make_float2(ax, ay);
    axy = __ffma2_rn(make_float2(f.x, f.x), pa, axy); az = fmaf(f.x, qa.x, az);
    axy = __ffma2_rn(make_float2(f.y, f.y), pc, axy); az = fmaf(f.y, qc.x, az);
    ax = axy.x; ay = axy.y;
    if (COUNT) cnt += ((r2.x < cut2) + (r2.y < cut2)) * cw;
}

__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The TRIDS atom-pair terms (pair_trids) for the two candidates of one candidate-list
// word, branch-free on the packed FP32 pipe: every term is evaluated and masked (cutoff,
// r < 10 for E_long, r < d_clash, donor-acceptor pair with r < 3.4, r < 5 for the
// atom-pair E_MDN) by
// multiplying with 0/1, exact for the finite values every candidate gives.  exp and log
// go through ex2 / lg2.  mb selects the candidate's donor/acceptor flag bits (low entry;
// shifted by 16 for the high entry).  gmm (term set 1, ligand-pocket pairs only; else
// null): the ligand atom type's row of (pi, mu, -1/(2 sigma^2), 1/sigma^2) by pocket type.
template <bool COUNT>
__device__ __forceinline__ void trids_x2(uint32_t wd, const float4* __restrict__ src, float2 nxy, float2 nzr,
                                         float cut2, const float w[5], uint32_t mb, const float4* __restrict__ gmm,
                                         const uint8_t* __restrict__ ptype, int K, float2& eb, float& ax, float& ay,
                                         float& az, uint32_t& cnt, uint32_t cw) {
    constexpr float kL2e = 1.4426950408889634f, kLn2 = 0.6931471805599453f;
    const uint32_t ja = wd & 0x1fffu, jb = (wd >> 16) & 0x1fffu;
    const float4 a = src[ja], c = src[jb];
    const float2 pm = make_float2(1.f, -1.f);
    const float2 pa = __fadd2_rn(make_float2(a.x, a.y), nxy);
    const float2 qa = __ffma2_rn(make_float2(a.z, a.w), pm, nzr);      // (z_j - z_i, -(R_i + R_j))
    const float2 pc = __fadd2_rn(make_float2(c.x, c.y), nxy);
    const float2 qc = __ffma2_rn(make_float2(c.z, c.w), pm, nzr);
    const float2 sa = __fmul2_rn(pa, pa), sc = __fmul2_rn(pc, pc);
    const float2 r2 = make_float2(fmaf(qa.x, qa.x, sa.x) + sa.y, fmaf(qc.x, qc.x, sc.x) + sc.y);
    const float2 in = make_float2(r2.x < cut2 ? 1.f : 0.f, r2.y < cut2 ? 1.f : 0.f);
    const float2 rr = __fadd2_rn(r2, make_float2(1e-12f, 1e-12f));
    const float2 ri = make_float2(rsqrtf(rr.x), rsqrtf(rr.y));
    const float2 r = __fmul2_rn(rr, ri);
    const float2 rs = make_float2(-qa.y, -qc.y);                            // R_i + R_j
    const float2 hb = make_float2((wd & mb) ? 1.f : 0.f, (wd & (mb << 16)) ? 1.f : 0.f);
    // E_long: -exp(-(r - R_i - R_j - 3)^2 / 4); dE/dr = 0.5 gl z
    const float2 z = __fadd2_rn(r, make_float2(qa.y - 3.f, qc.y - 3.f));
    const float2 al = __fmul2_rn(__fmul2_rn(z, z), make_float2(-0.25f * kL2e, -0.25f * kL2e));
    const float2 gl = make_float2(r.x < 10.f ? ex2_approx(al.x) : 0.f, r.y < 10.f ? ex2_approx(al.y) : 0.f);
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
        const float4* __restrict__ ga = gmm + ptype[ja] * kK;
        const float4* __restrict__ gc = gmm + ptype[jb] * kK;
        float2 e0 = make_float2(0.f, 0.f), d0 = make_float2(0.f, 0.f);
        for (int k = 0; k < K; ++k) {
            const float4 u = ga[k], v = gc[k];
            const float2 zz = __fadd2_rn(r, make_float2(-u.y, -v.y));
            const float2 ar = __fmul2_rn(__fmul2_rn(zz, zz), make_float2(u.z * kL2e, v.z * kL2e));
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
    if (COUNT) cnt += ((r2.x < cut2) + (r2.y < cut2)) * cw;
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
// (Rodrigues, angle th held by lane k) into W.rk; then each lane places its atoms:
// the torsions that move an atom (its fragment's torsion and that torsion's ancestors),
// deepest first, about their input-geometry axes -- the axis atoms of a torsion are never
// moved by the torsions below it -- then x = t + R(q) z.
__device__ void fk_warp(const DevBatch& B, const LigHdr& h, const PW& W, const float t[3], const float q[4], float th,
                        const float* __restrict__ rad) {
    const int T = h.n_tor, L = h.n_atoms;
    if (W.lane < T) {
        const float4 u = __ldg(&B.tor_u[h.tor_off + W.lane]);
        float s, c;
        sincosf(th, &s, &c);
        const float kc = 1.f - c;
        W.rk[3 * W.lane + 0] = make_float4(c + kc * u.x * u.x, kc * u.x * u.y - s * u.z, kc * u.x * u.z + s * u.y, 0.f);
        W.rk[3 * W.lane + 1] = make_float4(kc * u.y * u.x + s * u.z, c + kc * u.y * u.y, kc * u.y * u.z - s * u.x, 0.f);
        W.rk[3 * W.lane + 2] = make_float4(kc * u.z * u.x - s * u.y, kc * u.z * u.y + s * u.x, c + kc * u.z * u.z, 0.f);
    }
    __syncwarp();
    float R[9];
    quat_to_mat(q, R);
    const int8_t* __restrict__ tpar = B.tor_par + h.tor_off;
    for (int i = W.lane; i < L; i += 32) {
        const float4 y = __ldg(&B.atom_y[h.atom_off + i]);
        float x0 = y.x, x1 = y.y, x2 = y.z;
        // the torsions that move atom i are its fragment's torsion and that torsion's
        // ancestors; walking up the tree visits them deepest first
        for (int k = __ldg(&B.atom_tor[h.atom_off + i]); k >= 0; k = __ldg(&tpar[k])) {
            const float4 p = __ldg(&B.tor_p[h.tor_off + k]);
            const float4 r0 = W.rk[3 * k], r1 = W.rk[3 * k + 1], r2 = W.rk[3 * k + 2];
            const float vx = x0 - p.x, vy = x1 - p.y, vz = x2 - p.z;
            x0 = p.x + (r0.x * vx + r0.y * vy + r0.z * vz);
            x1 = p.y + (r1.x * vx + r1.y * vy + r1.z * vz);
            x2 = p.z + (r2.x * vx + r2.y * vy + r2.z * vz);
        }
        W.xs[i] = make_float4(t[0] + (R[0] * x0 + R[1] * x1 + R[2] * x2), t[1] + (R[3] * x0 + R[4] * x1 + R[5] * x2),
                              t[2] + (R[6] * x0 + R[7] * x1 + R[8] * x2), rad[__float_as_int(y.w)]);
    }
    if (W.lane == 0) W.xs[B.max_atoms] = make_float4(1e6f, 1e6f, 1e6f, 0.f);   // padding target
    __syncwarp();
}

// ------------------------------------------------------------------ balanced item loops
// The pair loop and the E_MDN passes number a pose's work items atom by atom and give
// lane k the k-th of 32 equal contiguous segments.  A lane accumulates its current atom's
// force in registers and leaves a partial in slot (atom + lane) of W.rec: slots are unique
// because atoms never decrease along the lanes.  The partials of an atom are then added in
// lane order, so the result does not depend on timing.

// Per-atom item counts -> exclusive prefix W.pre[0..L], 32 atoms per call: atom i =
// base + lane has n items (0 for i >= L); carry runs over the calls.  seg_finish then sets
// W.pre[0], clears W.rec and returns the total.
__device__ __forceinline__ void seg_scan(const PW& W, int L, int i, int n, int& carry) {
    const int lane = W.lane;
    int v = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    if (i < L) W.pre[i + 1] = carry + v;
    carry += __shfl_sync(kFull, v, 31);
}

__device__ __forceinline__ int seg_finish(const PW& W, int L, int carry) {
    if (W.lane == 0) W.pre[0] = 0;
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
        if (W.pre[m] <= lo) a = m; else b = m - 1;
    }
    return a;
}

// Each atom's partials in lane order: W.gs[i] = sum (ADD: W.gs[i] += sum).
template <bool ADD>
__device__ __forceinline__ void seg_combine(const PW& W, int L, int N) {
    __syncwarp();
    for (int i = W.lane; i < L; i += 32) {
        float gx = 0.f, gy = 0.f, gz = 0.f;
        const int b0 = W.pre[i], b1 = W.pre[i + 1];
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
// (x, y, z, radius).  The pose's blocks are numbered atom by atom (prefix in W.pre) and
// split into 32 equal contiguous segments, one per lane, so the lanes stay balanced
// whatever the atoms' list lengths.  A lane accumulates the force on its current atom
// in registers and leaves a partial in slot (atom + lane) of W.rec; the partials of an
// atom are added in lane order (bit-reproducible).  The Vina-form block is branch-free:
// all candidates are evaluated and masked by r^2 < cutoff^2.  Writes the forces to W.gs;
// returns the lane's ligand-pocket energy and, in *e_in2, twice its intra energy.
template <int TS, bool PARAMS, bool COUNT, bool MAPS>
__device__ float pairs_warp(const DevBatch& B, const DevPocket& pk, const Smem& S, const LigHdr& h, const PW& W,
                           const float w[5], float ebar, ParamAcc& acc, uint32_t& npairs, float* e_in2) {
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
            uint32_t beg, end;
            cell_range(pk, pk.cell_start, x.x, x.y, x.z, beg, end);
            const int i0 = __ldg(&B.ipre[h.ipre_off + i]), i1 = __ldg(&B.ipre[h.ipre_off + i + 1]);
            const int cbk = (MAPS && map_cell(pk, x.x, x.y, x.z, nullptr)) ? 0 : (int)((end - beg) >> 3);
            W.cs[i] = beg;
            W.cb[i] = cbk;
            W.ip[i] = i0;
            nblk = cbk + (i1 - i0);
        }
        seg_scan(W, L, i, nblk, carry);
    }
    const int N = seg_finish(W, L, carry);
    int lo, hi;
    int i = seg_range(W, L, N, lo, hi);
    float e_lp = 0.f, e_in = 0.f;
    if (lo < hi) {
        int first = W.pre[i], nxt = W.pre[i + 1], cbk = W.cb[i], ipb = W.ip[i];
        uint32_t csb = W.cs[i];
        float4 xa = W.xs[i];
        int ti = __float_as_int(__ldg(&B.atom_y[h.atom_off + i]).w);
        float ri = xa.w;
        uint32_t fi = P.tflags[ti];
        float ax = 0.f, ay = 0.f, az = 0.f;
        auto block_ptr = [&](int blk) -> const uint4* {
            const int loc = blk - first;
            return loc < cbk ? reinterpret_cast<const uint4*>(cand + csb + 8u * (uint32_t)loc)
                             : reinterpret_cast<const uint4*>(ient + 8 * (ipb + loc - cbk));
        };
        uint4 v = __ldg(block_ptr(lo));
        for (int blk = lo; blk < hi; ++blk) {
            if (blk == nxt) {                      // move to the atom owning block blk
                W.rec[i + lane] = make_float4(ax, ay, az, 0.f);
                ax = ay = az = 0.f;
                do { ++i; } while (W.pre[i + 1] == blk);
                first = W.pre[i];
                nxt = W.pre[i + 1];
                cbk = W.cb[i];
                ipb = W.ip[i];
                csb = W.cs[i];
                xa = W.xs[i];
                ti = __float_as_int(__ldg(&B.atom_y[h.atom_off + i]).w);
                ri = xa.w;
                fi = P.tflags[ti];
                v = __ldg(block_ptr(blk));
            }
            const uint4 vc = v;
            const bool intra = blk - first >= cbk;
            if (blk + 1 < hi && blk + 1 < nxt) v = __ldg(block_ptr(blk + 1));
            const float4* __restrict__ src = intra ? W.xs : S.pocket;
            // pair-flag selectors: hydrophobic needs both bit0; donor-acceptor needs
            // (donor_i & acceptor_j) | (acceptor_i & donor_j)
            const uint32_t f_hyd = fi & 1u;
            const uint32_t f_hb = ((fi & 2u) << 1) | ((fi & 4u) >> 1);
            float eb = 0.f;
            float2 eb2 = make_float2(0.f, 0.f);
            const float2 nxy = make_float2(-xa.x, -xa.y), nzr = make_float2(-xa.z, -ri);
            const uint32_t mh = f_hyd << 13, mb = f_hb << 13;
            // two halves of four candidates: the loop body stays small for the
            // instruction cache, which the 16 resident warps share across all phases
#pragma unroll 1
            for (int hv = 0; hv < 2; ++hv) {
                const uint32_t wv[2] = {hv ? vc.z : vc.x, hv ? vc.w : vc.y};
                if constexpr (TS == TRIDS_TERMS_VINA5 && !PARAMS) {
#pragma unroll
                    for (int u = 0; u < 2; ++u)
                        vina_x2<COUNT>(wv[u], src, nxy, nzr, cut2, K, mh, mb, eb2, ax, ay, az, npairs,
                                       intra ? 1u : 2u);   // doubled: intra pairs come twice
                } else if constexpr (!PARAMS) {
                    const float4* gm = nullptr;   // term set 1: the atom-pair E_MDN runs in gmm_warp
#pragma unroll
                    for (int u = 0; u < 2; ++u)
                        trids_x2<COUNT>(wv[u], src, nxy, nzr, cut2, w, mb, gm, S.ptype, P.gmm_k, eb2, ax, ay, az,
                                        npairs, intra ? 1u : 2u);
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
                        if (COUNT) npairs += in ? (intra ? 1u : 2u) : 0u;   // doubled: intra pairs come twice
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
template <bool MAPS>
__device__ float gmm_warp(const DevBatch& B, const DevPocket& pk, const Smem& S, const LigHdr& h, const PW& W,
                          float w0) {
    constexpr float kL2e = 1.4426950408889634f;
    const DevParams& P = *S.P;
    const int K = P.gmm_k, L = h.n_atoms, lane = W.lane;
    const float nc2 = pk.near_cut2;
    int carry = 0;
    for (int base = 0; base < L; base += 32) {
        const int i = base + lane;
        int n = 0;
        if (i < L) {
            const float4 x = W.xs[i];
            uint32_t beg = 0, end = 0;
            if (!(MAPS && map_cell(pk, x.x, x.y, x.z, nullptr))) cell_range(pk, pk.ncell_start, x.x, x.y, x.z, beg, end);
            W.cs[i] = beg;
            n = (int)(end - beg);
        }
        seg_scan(W, L, i, n, carry);
    }
    const int N = seg_finish(W, L, carry);
    int lo, hi;
    int i = seg_range(W, L, N, lo, hi);
    float e = 0.f;
    if (lo < hi) {
        int first = W.pre[i], nxt = W.pre[i + 1];
        uint32_t cs = W.cs[i];
        float4 x = W.xs[i];
        const float4* g = &P.gmm[__float_as_int(__ldg(&B.atom_y[h.atom_off + i]).w)][0][0];
        float gx = 0.f, gy = 0.f, gz = 0.f, ei = 0.f;
        for (int it = lo; it < hi; ++it) {
            if (it == nxt) {
                W.rec[i + lane] = make_float4(gx, gy, gz, 0.f);
                e = fmaf(w0, ei, e);
                gx = gy = gz = ei = 0.f;
                do { ++i; } while (W.pre[i + 1] == it);
                first = W.pre[i];
                nxt = W.pre[i + 1];
                cs = W.cs[i];
                x = W.xs[i];
                g = &P.gmm[__float_as_int(__ldg(&B.atom_y[h.atom_off + i]).w)][0][0];
            }
            const int j = __ldg(&pk.nlist[cs + (uint32_t)(it - first)]);
            const float4 p = S.pocket[j];
            const float dx = x.x - p.x, dy = x.y - p.y, dz = x.z - p.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float in = r2 < nc2 ? 1.f : 0.f;
            const float rinv = rsqrtf(fmaxf(r2, 1e-12f));
            const float r = r2 * rinv;
            const float4* gk = g + S.ptype[j] * kK;
            float e0 = 0.f, d0 = 0.f;
            for (int k = 0; k < K; ++k) {
                const float4 u = gk[k];                          // (pi, mu, -1/(2 sigma^2), 1/sigma^2)
                const float z = r - u.y;
                const float ex = u.x * ex2_approx(u.z * kL2e * z * z);
                e0 += ex;
                d0 = fmaf(ex * z, u.w, d0);
            }
            ei = fmaf(-in, e0, ei);
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
template <bool PARAMS>
__device__ float residue_warp(const DevBatch& B, const DevPocket& pk, const Smem& S, const LigHdr& h, const PW& W,
                              float w0, float ebar, ParamAcc& acc) {
    constexpr float kCut2 = kMdnCut * kMdnCut;
    constexpr float kL2e = 1.4426950408889634f;
    const int K = B.mdn_k, R = B.mdn_res, L = h.n_atoms, lane = W.lane;
    int carry = 0;
    for (int base = 0; base < L; base += 32) {
        const int i = base + lane;
        int n = 0;
        if (i < L) {
            const float4 x = W.xs[i];
            uint32_t beg, end;
            cell_range(pk, pk.rcell_start, x.x, x.y, x.z, beg, end);
            W.cs[i] = beg;
            n = (int)(end - beg);
        }
        seg_scan(W, L, i, n, carry);
    }
    const int N = seg_finish(W, L, carry);
    int lo, hi;
    int i = seg_range(W, L, N, lo, hi);
    float e = 0.f;
    if (lo < hi) {
        int first = W.pre[i], nxt = W.pre[i + 1];
        uint32_t cs = W.cs[i];
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
                do { ++i; } while (W.pre[i + 1] == it);
                first = W.pre[i];
                nxt = W.pre[i + 1];
                cs = W.cs[i];
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
            const bool take1 = b1 < b0 || (b1 == b0 && i1 < i0);
            const float best = take1 ? b1 : b0;
            const float4 pb = S.pocket[take1 ? i1 : i0];
            const float bx = x.x - pb.x, by = x.y - pb.y, bz = x.z - pb.z;
            if (best < kCut2) {
                const float rinv = rsqrtf(fmaxf(best, 1e-12f));
                const float d = best * rinv;
                float P = 0.f, dP = 0.f;
                for (int k = 0; k < K; ++k) {
                    const float4 g = __ldg(&kern[r * K + k]);   // (pi, mu, -1/(2 sigma^2), 1/sigma^2)
                    const float z = d - g.y;
                    const float ex = g.x * ex2_approx(g.z * kL2e * z * z);
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

// E_total of the warp's pose (same value on every lane); forces in W.gs.
template <int TS, bool PARAMS, bool COUNT, bool MAPS>
__device__ float score_warp(const DevBatch& B, const DevPocket& pk, const Smem& S, const LigHdr& h, const PW& W,
                            float ebar, ParamAcc& acc, float* e_inter, uint32_t& npairs) {
    float w[5];
#pragma unroll
    for (int t = 0; t < 5; ++t) w[t] = S.P->w[t];
    float ein2;
    float el = pairs_warp<TS, PARAMS, COUNT, MAPS>(B, pk, S, h, W, w, ebar, acc, npairs, &ein2);
    if (MAPS && pk.use_maps) el += map_warp(B, pk, h, W);
    if constexpr (TS == TRIDS_TERMS_TRIDS && !PARAMS) el += gmm_warp<MAPS>(B, pk, S, h, W, w[0]);
    if constexpr (TS == TRIDS_TERMS_TRIDS_RES) el += residue_warp<PARAMS>(B, pk, S, h, W, w[0], ebar, acc);
    const float e_lp = warp_sum(el);
    *e_inter = e_lp;
    return e_lp + 0.5f * warp_sum(ein2);
}

// dE/dt = sum g_i and world torque tau = sum (x_i - t) x g_i (every lane), and
// dE/dtheta_k = a_k . sum over the moving subtree of (x_i - p_k) x g_i with a_k the world
// axis (parent atom -> child atom) and p_k the world parent atom (lane k, which sums its
// subtree serially: no shuffles, and the subtree is one contiguous range).
__device__ float adjoint_warp(const DevBatch& B, const LigHdr& h, const PW& W, const float t[3], float gt[3],
                              float tau[3]) {
    const int L = h.n_atoms, T = h.n_tor;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f, a5 = 0.f;
    for (int i = W.lane; i < L; i += 32) {
        const float4 g = W.gs[i], x = W.xs[i];
        const float rx = x.x - t[0], ry = x.y - t[1], rz = x.z - t[2];
        a0 += g.x; a1 += g.y; a2 += g.z;
        a3 += ry * g.z - rz * g.y;
        a4 += rz * g.x - rx * g.z;
        a5 += rx * g.y - ry * g.x;
    }
    gt[0] = warp_sum(a0); gt[1] = warp_sum(a1); gt[2] = warp_sum(a2);
    tau[0] = warp_sum(a3); tau[1] = warp_sum(a4); tau[2] = warp_sum(a5);
    // torsion k on lane k: its moving subtree is the contiguous atom range [ti.z, ti.w)
    float mine = 0.f;
    if (W.lane < T) {
        const int4 ti = __ldg(&B.tor_idx[h.tor_off + W.lane]);
        const float4 p = W.xs[ti.x], c = W.xs[ti.y];
        float sx = 0.f, sy = 0.f, sz = 0.f;
        for (int i = ti.z; i < ti.w; ++i) {
            const float4 x = W.xs[i], g = W.gs[i];
            const float rx = x.x - p.x, ry = x.y - p.y, rz = x.z - p.z;
            sx += ry * g.z - rz * g.y;
            sy += rz * g.x - rx * g.z;
            sz += rx * g.y - ry * g.x;
        }
        const float ax = c.x - p.x, ay = c.y - p.y, az = c.z - p.z;
        const float n = rsqrtf(ax * ax + ay * ay + az * az);
        mine = (ax * sx + ay * sy + az * sz) * n;
    }
    return mine;
}

// ------------------------------------------------------------------ sampler state
// The rigid state is the same on every lane (every lane computes it); lane k < T holds
// torsion k's angle, Adam moments and saved angle.  PoseState is a handle on the warp's
// shared-memory copy.
struct RigidState {
    float t[3], q[4], m[6], v[6], st[3], sq[4];
    float ecur, esaved;
    int status;
    float pad[3];
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
    float& th;
    float& mth;
    float& vth;
    float& sth;
    __device__ PoseState(RigidState& r, TorState& k)
        : t(r.t), q(r.q), m(r.m), v(r.v), st(r.st), sq(r.sq), ecur(r.ecur), esaved(r.esaved), status(r.status),
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
    const uint32_t lig = (uint32_t)(A.lig_base + l);
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
            return -A.lr * g / (sqrtf(v) + A.eps);
        case TRIDS_OPT_ADAGRAD:
            v = fmaf(g, g, v);
            return -A.lr * g / (sqrtf(v) + A.eps);
        case TRIDS_OPT_SGD:
            m = fmaf(A.momentum, m, g);
            return -A.lr * m;
        default:
            break;
        }
    }
    m = fmaf(A.b1, m, (1.f - A.b1) * g);
    v = fmaf(A.b2, v, (1.f - A.b2) * g * g);
    const float denom = fmaf(sqrtf(v), rsbc2, A.eps);
    const float d = -lr_bc1 * __fdividef(m, denom);
    return GEN && A.opt == TRIDS_OPT_ADAMW ? fmaf(-A.lr * A.wd, pv, d) : d;
}

// One evaluation (and its update or acceptance test) of the warp's pose; s is the
// global evaluation index of the schedule.  Every branch below is uniform across the
// warp except the per-torsion lanes.
template <int TS, bool COUNT, bool GEN>
__device__ void sample_step(const SampleArgs& A, const Smem& S, const LigHdr& h, const PW& W, int l, int p, int s,
                            const Sched& sc, PoseState& st, uint32_t& npairs) {
    __syncwarp();               // the rigid state is one shared copy written by every lane
    if (st.status & 1) return;  // frozen after a non-finite energy
    const int T = h.n_tor, lane = W.lane;
    const int bx = A.pk.n_boxes > 1 ? p % A.pk.n_boxes : 0;   // the pose's docking box
    const bool own = lane < T;
    const uint32_t lig = (uint32_t)(A.lig_base + l);
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
                sincosf(0.5f * ang, &sh, &ch);
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
    fk_warp(A.B, h, W, st.t, st.q, st.th, S.P->radius);
    ParamAcc acc;
    float e_inter;
    const float E = score_warp<TS, false, COUNT, GEN>(A.B, A.pk, S, h, W, 1.f, acc, &e_inter, npairs);
    float gt[3], tau[3];
    const float gth = adjoint_warp(A.B, h, W, st.t, gt, tau);
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
        const float rsbc2 = rsqrtf(1.f - ipowf(A.b2, ta));
        if (own) st.th = wrap_pi(st.th + opt_delta<GEN>(A, gth, st.th, st.mth, st.vth, lr_bc1, rsbc2));
        for (int d = 0; d < 3; ++d) {
            const float lo = A.pk.box_lo[bx][d], hi = A.pk.box_hi[bx][d];
            const float dlt = opt_delta<GEN>(A, gt[d], st.t[d] - 0.5f * (lo + hi), st.m[d], st.v[d], lr_bc1, rsbc2);
            st.t[d] = fminf(fmaxf(st.t[d] + dlt, lo), hi);
        }
        float dw[3];
        for (int d = 0; d < 3; ++d) dw[d] = opt_delta<GEN>(A, tau[d], 0.f, st.m[3 + d], st.v[3 + d], lr_bc1, rsbc2);
        const float phi = sqrtf(dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2]);
        if (phi > 0.f) {
            float sh, ch;
            sincosf(0.5f * phi, &sh, &ch);
            const float sc2 = sh / phi;
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

// Pair counts are kept doubled per lane (an intra pair is seen from both of its atoms,
// possibly by different lanes); the warp total is halved here.
__device__ __forceinline__ void flush_count(unsigned long long* cnt, uint32_t n) {
    unsigned long long v = n;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(cnt, v >> 1);
}

// Persistent fused sampler: each warp pops poses from a global counter (ligands in
// decreasing-cost order) and runs every evaluation of the pose with its state on chip.
template <int TS, bool COUNT, bool GEN>
__global__ void __launch_bounds__(640, 1) k_sample_persistent(SampleArgs A) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (!stage_block(smem, A.pk, A.params_bytes, A.pocket_off, A.ptype_off, A.mbar_off, A.err)) return;
    Smem S{reinterpret_cast<const DevParams*>(smem), reinterpret_cast<const float4*>(smem + A.pocket_off),
           reinterpret_cast<const uint8_t*>(smem + A.ptype_off)};
    const PW W = make_pw(smem, A.warp_off, A.warp_bytes, A.B.max_atoms, A.B.max_tor);
    uint32_t npairs = 0;
    for (;;) {
        int it = 0;
        if (W.lane == 0) it = (int)atomicAdd(A.counter, 1u);
        it = __shfl_sync(kFull, it, 0);
        if (it >= A.n_items) break;
        const int l = A.lig_order[it / A.P];
        const int p = it % A.P;
        const LigHdr h = A.B.lig[l];
        PoseState st(*W.rig, W.tor[W.lane]);   // in shared memory: no registers across the pair loop
        if (A.step_begin == 0) init_pose(A, h, W.lane, l, p, st);
        else load_pose(A, h, W.lane, l, p, st);
        __syncwarp();
        Sched sc = schedule(A.S, A.Lmc, A.step_begin);
        for (int s = A.step_begin; s < A.step_end; ++s) {
            sample_step<TS, COUNT, GEN>(A, S, h, W, l, p, s, sc, st, npairs);
            if (++sc.j == sc.n) {   // next Monte-Carlo loop: the schedule of evaluation s + 1
                ++sc.loop;
                sc.j = 0;
                sc.n = A.S / A.Lmc + (sc.loop < A.S % A.Lmc ? 1 : 0);
            }
        }
        __syncwarp();
        store_pose(A, h, W.lane, l, p, st);
        __syncwarp();
    }
    if (COUNT) flush_count(A.pair_count, npairs);
}

// Plain form: one launch per (ligand, evaluation), one warp per pose, the state in
// global memory between launches; the same device code as the persistent sampler.
template <int TS, bool COUNT, bool GEN>
__global__ void __launch_bounds__(640, 1) k_sample_step(SampleArgs A, int l, int s) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (!stage_block(smem, A.pk, A.params_bytes, A.pocket_off, A.ptype_off, A.mbar_off, A.err)) return;
    Smem S{reinterpret_cast<const DevParams*>(smem), reinterpret_cast<const float4*>(smem + A.pocket_off),
           reinterpret_cast<const uint8_t*>(smem + A.ptype_off)};
    const PW W = make_pw(smem, A.warp_off, A.warp_bytes, A.B.max_atoms, A.B.max_tor);
    const int p = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    if (p >= A.P) return;
    const LigHdr h = A.B.lig[l];
    uint32_t npairs = 0;
    PoseState st(*W.rig, W.tor[W.lane]);
    if (s == 0) init_pose(A, h, W.lane, l, p, st);
    else load_pose(A, h, W.lane, l, p, st);
    __syncwarp();
    sample_step<TS, COUNT, GEN>(A, S, h, W, l, p, s, schedule(A.S, A.Lmc, s), st, npairs);
    __syncwarp();
    store_pose(A, h, W.lane, l, p, st);
    if (COUNT) flush_count(A.pair_count, npairs);
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
            uint32_t np = 0;
            const float E = score_warp<TS, PARAMS, false, !PARAMS>(A.B, A.pk, S, h, W, ebar, acc, &e_inter, np);
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
                    const float n = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
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

// =============================================================== allocation-free scoring
// Scratch of trids_score_grad_noalloc: one statically sized device array per device
// that loads the library (kept until the process exits).  Layout: work counter at
// offset 0, item list at 256, parameter partials after it (256-aligned).
constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// =============================================================== host objects
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
    DevParams* d_params = nullptr;
    uint32_t* d_ncell = nullptr;         // near lists of the atom-pair E_MDN (term set 1)
    uint16_t* d_nlist = nullptr;
    float* d_maps = nullptr;             // grid maps [type][z][y][x]
    int mdims[3] = {0, 0, 0};
    float mlo[3] = {0.f, 0.f, 0.f}, mh = 0.f;
    bool maps_stale = false;             // parameters changed since the maps were built
    ResidueGrid rgrid;                   // residue-level E_MDN (term set 2)
    int32_t* d_res_start = nullptr;
    uint32_t* d_rcell = nullptr;
    uint32_t* d_rlist = nullptr;
    DevPocket view() const {
        DevPocket v;
        v.atoms = d_atoms; v.ptype = d_ptype; v.cell_start = d_cell; v.cand = d_cand; v.params = d_params; v.M = M;
        v.n_res = rgrid.n_res; v.res_start = d_res_start; v.rcell_start = d_rcell;
        v.rlist = d_rlist;
        v.ncell_start = d_ncell; v.nlist = d_nlist;
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

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;
};

struct trids_batch {
    int device = 0;
    int n_types = 0;
    trids_batch_dims dims{};
    std::vector<PackedLigand> ligs;
    std::vector<LigHdr> hdr;
    LigHdr* d_lig = nullptr;
    float4* d_atom_y = nullptr;
    int* d_atom_orig = nullptr;
    int4* d_tor_idx = nullptr;
    float4* d_tor_u = nullptr;
    float4* d_tor_p = nullptr;
    int* d_ipre = nullptr;
    uint16_t* d_ient = nullptr;
    int8_t* d_atom_tor = nullptr;
    int8_t* d_tor_par = nullptr;
    std::vector<uint16_t> ient_j;     // intra partner lists: target index (pad = max_atoms)
    std::vector<uint8_t> ient_type;   // target type (for re-encoding flags)
    trids_pocket* owner = nullptr;    // pocket whose flags are encoded in d_ient
    // per-pose-count caches
    int items_P = -1;
    int2* d_items = nullptr;        // (ligand, first pose of a 32-pose tile), by decreasing cost
    int n_items = 0;
    int* d_lig_order = nullptr;     // ligands by decreasing cost
    unsigned int* d_counter = nullptr;   // [4]
    int* d_err = nullptr;                // [2]: staging timeout, status OR
    float* d_partials = nullptr;
    size_t partials_cap = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    GraphCache graph;
    float4* d_mdn = nullptr;        // residue-level E_MDN kernels, packed rows
    int mdn_res = 0, mdn_k = 0;
    DevBatch view() const {
        DevBatch v;
        v.n_lig = dims.n_lig; v.max_atoms = dims.max_atoms; v.max_tor = dims.max_tor;
        v.dof_stride = dims.dof_stride; v.n_fields = dims.state_fields;
        v.lig = d_lig; v.atom_y = d_atom_y; v.atom_orig = d_atom_orig; v.tor_idx = d_tor_idx;
        v.tor_u = d_tor_u; v.tor_p = d_tor_p; v.ipre = d_ipre; v.ient = d_ient;
        v.atom_tor = d_atom_tor; v.tor_par = d_tor_par;
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
                    d->gmm[a][b][k] = make_float4(g[0], g[1], -1.f / (2.f * g[2] * g[2]), 1.f / (g[2] * g[2]));
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

// (Re-)encode a batch's intra partner entries with the pocket's current type flags.
int encode_intra(const trids_pocket* pk, trids_batch* b, bool allocate) {
    std::vector<uint16_t> ent(b->ient_j.size());
    for (size_t k = 0; k < ent.size(); ++k) {
        const uint32_t f = b->ient_type[k] == 0xff ? 0u : (uint32_t)(pk->prm.flags[b->ient_type[k]] & 7);
        ent[k] = (uint16_t)((uint32_t)b->ient_j[k] | (f << 13));
    }
    if (allocate) return upload(&b->d_ient, ent);
    if (!ent.empty()) CK(cudaMemcpy(b->d_ient, ent.data(), ent.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    return TRIDS_OK;
}

int device_guard(int dev) {
    int cur = -1;
    CK(cudaGetDevice(&cur));
    if (cur != dev) CK(cudaSetDevice(dev));
    return TRIDS_OK;
}

int ensure_items(trids_batch* b, int P) {
    if (b->items_P == P) return TRIDS_OK;
    const int tiles = (P + 31) / 32;
    std::vector<std::pair<double, int>> lc(b->dims.n_lig);
    for (int l = 0; l < b->dims.n_lig; ++l) {
        const LigHdr& h = b->hdr[l];
        lc[l] = {60.0 * h.n_atoms + 2.0 * h.n_pairs + 20.0 * h.n_tor + 10.0, l};
    }
    std::stable_sort(lc.begin(), lc.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& c) {
        return a.first > c.first;
    });
    std::vector<int> order(lc.size());
    std::vector<int2> items;
    items.reserve((size_t)b->dims.n_lig * tiles);
    for (size_t i = 0; i < lc.size(); ++i) {
        order[i] = lc[i].second;
        for (int t = 0; t < tiles; ++t) items.push_back(make_int2(lc[i].second, t * 32));
    }
    cudaFree(b->d_items);
    cudaFree(b->d_lig_order);
    b->d_items = nullptr;
    b->d_lig_order = nullptr;
    int rc = upload(&b->d_items, items);
    if (rc) return rc;
    if ((rc = upload(&b->d_lig_order, order))) return rc;
    b->n_items = (int)items.size();
    b->items_P = P;
    return TRIDS_OK;
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

// Pick warps per block: the requested count, capped so the block fits in shared memory.
int pick_warps(int requested, const trids_pocket* pk, const trids_batch* b, bool params, Layout* L) {
    const size_t cap = max_smem(pk->device);
    int w = requested > 0 ? std::min(requested, 20) : 8;
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
    std::vector<uint16_t> list;
    build_near_lists(pk->M, pk->xyz.data(), std::min(kMdnCut, pk->cutoff_built), pk->grid, &start, &list);
    uint32_t* d_start = nullptr;
    uint16_t* d_list = nullptr;
    int rc;
    if ((rc = upload(&d_start, start)) || (rc = upload(&d_list, list))) {
        cudaFree(d_start);
        cudaFree(d_list);
        return rc;
    }
    cudaFree(pk->d_ncell);
    cudaFree(pk->d_nlist);
    pk->d_ncell = d_start;
    pk->d_nlist = d_list;
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
// (pi, mu, -1/(2 sigma^2), 1/sigma^2); flags entries with non-finite values or sigma <= 0.
__global__ void k_mdn_pack(const float* __restrict__ in, const int* __restrict__ in_row, int64_t rows, int RK,
                           float4* __restrict__ out, int* bad) {
    const int64_t n = rows * RK;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / RK, rk = e - s * RK;
        const float* g = in + ((int64_t)in_row[s] * RK + rk) * 3;
        const float pi = g[0], mu = g[1], sg = g[2];
        if (!isfinite(pi) || !isfinite(mu) || !isfinite(sg) || !(sg > 0.f)) atomicOr(bad, 1);
        const float is2 = 1.f / (sg * sg);
        out[e] = make_float4(pi, mu, -0.5f * is2, is2);
    }
}

}  // namespace

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
            if ((rc = encode_intra(pk, b, false))) return rc;
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
    cudaFree(pk->d_atoms);
    cudaFree(pk->d_ptype);
    cudaFree(pk->d_cell);
    cudaFree(pk->d_cand);
    cudaFree(pk->d_params);
    cudaFree(pk->d_maps);
    cudaFree(pk->d_ncell);
    cudaFree(pk->d_nlist);
    cudaFree(pk->d_res_start);
    cudaFree(pk->d_rcell);
    cudaFree(pk->d_rlist);
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
    if ((rc = upload(&d_start, rg.start)) || (rc = upload(&d_cell, rg.cell_start)) || (rc = upload(&d_list, rg.list))) {
        cudaFree(d_start); cudaFree(d_cell); cudaFree(d_list);
        return rc;
    }
    CK(cudaDeviceSynchronize());   // no launch may still read the arrays being replaced
    std::vector<uint8_t> ptype(align_up((size_t)M + 1, 16), 0);
    for (int j = 0; j < M; ++j) ptype[j] = (uint8_t)type[j];
    CK(cudaMemcpy(pk->d_ptype, ptype.data(), ptype.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(pk->d_cell, grid.start.data(), grid.start.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    pk->xyz.swap(xyz);
    pk->type.swap(type);
    pk->orig.swap(orig);
    pk->grid = std::move(grid);
    if ((rc = upload_pocket_arrays(pk, nullptr))) return rc;   // atoms + candidate entries with flags
    if ((rc = upload_near_lists(pk))) return rc;
    cudaFree(pk->d_res_start); cudaFree(pk->d_rcell); cudaFree(pk->d_rlist);
    pk->d_res_start = d_start; pk->d_rcell = d_cell; pk->d_rlist = d_list;
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
    // per-ligand input offsets, then the ligands packed on host threads (each ligand is
    // independent; the first failing ligand in index order is reported)
    std::vector<size_t> aoff(n_lig + 1, 0), boff(n_lig + 1, 0);
    for (int l = 0; l < n_lig; ++l) {
        if (n_bonds[l] < 0) return fail(TRIDS_EINVAL, "ligand %d: negative bond count", l);
        if (n_bonds[l] > 0 && (!bonds || !rotatable)) return fail(TRIDS_EINVAL, "bonds is NULL");
        if (n_atoms[l] < 0) return fail(TRIDS_EINVAL, "ligand %d: negative atom count", l);
        aoff[l + 1] = aoff[l] + (size_t)n_atoms[l];
        boff[l + 1] = boff[l] + (size_t)n_bonds[l];
    }
    std::vector<std::string> msg(n_lig);
    {
        const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
        const int nt = std::max(1, std::min({hw, 32, n_lig / 16}));
        auto work = [&](int t) {
            for (int l = t; l < n_lig; l += nt)
                msg[l] = pack_ligand(n_atoms[l], xyz + 3 * aoff[l], type + aoff[l], pk->prm.n_types, n_bonds[l],
                                     bonds ? bonds + 2 * boff[l] : nullptr, rotatable ? rotatable + boff[l] : nullptr,
                                     &b->ligs[l]);
        };
        std::vector<std::thread> th;
        for (int t = 1; t < nt; ++t) th.emplace_back(work, t);
        work(0);
        for (auto& x : th) x.join();
    }
    int Lmax = 1, Tmax = 0;
    int64_t npairs = 0;
    for (int l = 0; l < n_lig; ++l) {
        if (!msg[l].empty()) return fail(TRIDS_EINVAL, "ligand %d: %s", l, msg[l].c_str());
        Lmax = std::max(Lmax, n_atoms[l]);
        Tmax = std::max(Tmax, b->ligs[l].n_tor);
        npairs += (int64_t)b->ligs[l].pairs.size();
    }
    size_t ao = 0;
    b->dims.n_lig = n_lig;
    b->dims.max_atoms = Lmax;
    b->dims.max_tor = Tmax;
    b->dims.dof_stride = 7 + Tmax;
    b->dims.state_fields = state_fields(Tmax);
    b->dims.n_intra = npairs;
    std::vector<float4> ay;
    std::vector<int> aorig;
    std::vector<int4> tidx;
    std::vector<float4> tu, tp;
    std::vector<int> ipre;
    std::vector<int8_t> atom_tor, tor_par;
    ao = 0;
    for (int l = 0; l < n_lig; ++l) {
        const PackedLigand& lg = b->ligs[l];
        LigHdr h{};
        h.n_atoms = lg.n_atoms;
        h.n_tor = lg.n_tor;
        h.atom_off = (int)ay.size();
        h.tor_off = (int)tidx.size();
        h.ipre_off = (int)ipre.size();
        h.ient_off = (int)b->ient_j.size();
        h.n_pairs = (int)lg.pairs.size();
        const float* X = xyz + 3 * ao;
        const int32_t* Ty = type + ao;
        for (int i = 0; i < lg.n_atoms; ++i) {
            const int a = lg.perm[i];
            float tb;
            int t = Ty[a];
            std::memcpy(&tb, &t, 4);
            ay.push_back(make_float4((float)((double)X[3 * a] - lg.c[0]), (float)((double)X[3 * a + 1] - lg.c[1]),
                                     (float)((double)X[3 * a + 2] - lg.c[2]), tb));
            aorig.push_back(a);
            atom_tor.push_back((int8_t)(lg.frag[i] - 1));
        }
        for (int k = 0; k < lg.n_tor; ++k) {
            const int pa = lg.perm[lg.tp[k]], ha = lg.perm[lg.th[k]];
            double u[3], nn = 0;
            for (int d = 0; d < 3; ++d) {
                u[d] = (double)X[3 * ha + d] - (double)X[3 * pa + d];
                nn += u[d] * u[d];
            }
            nn = std::sqrt(nn);
            if (!(nn > 1e-6)) return fail(TRIDS_EINVAL, "ligand %d: rotatable bond %d has zero length", l, k);
            tidx.push_back(make_int4(lg.tp[k], lg.th[k], lg.sb[k], lg.se[k]));
            tor_par.push_back((int8_t)lg.tpar[k]);
            tu.push_back(make_float4((float)(u[0] / nn), (float)(u[1] / nn), (float)(u[2] / nn), 0.f));
            tp.push_back(make_float4((float)((double)X[3 * pa] - lg.c[0]), (float)((double)X[3 * pa + 1] - lg.c[1]),
                                     (float)((double)X[3 * pa + 2] - lg.c[2]), 0.f));
        }
        // intra partner lists: per atom, every partner (both directions, ascending) in
        // blocks of 8, padded with the far sentinel index max_atoms
        {
            std::vector<std::vector<int>> part(lg.n_atoms);
            for (auto& pr : lg.pairs) {
                part[pr.first].push_back(pr.second);
                part[pr.second].push_back(pr.first);
            }
            int blocks = 0;
            for (int i = 0; i < lg.n_atoms; ++i) {
                std::sort(part[i].begin(), part[i].end());
                ipre.push_back(blocks);
                for (int j : part[i]) {
                    b->ient_j.push_back((uint16_t)j);
                    b->ient_type.push_back((uint8_t)Ty[lg.perm[j]]);
                }
                const size_t pad = (8 - part[i].size() % 8) % 8;
                for (size_t k = 0; k < pad; ++k) {
                    b->ient_j.push_back((uint16_t)Lmax);
                    b->ient_type.push_back(0xff);
                }
                blocks += (int)((part[i].size() + 7) / 8);
            }
            ipre.push_back(blocks);
        }
        b->hdr.push_back(h);
        ao += n_atoms[l];
    }
    if ((rc = upload(&b->d_lig, b->hdr)) || (rc = upload(&b->d_atom_y, ay)) || (rc = upload(&b->d_atom_orig, aorig)) ||
        (rc = upload(&b->d_tor_idx, tidx)) || (rc = upload(&b->d_tor_u, tu)) || (rc = upload(&b->d_tor_p, tp)) ||
        (rc = upload(&b->d_ipre, ipre)) || (rc = upload(&b->d_atom_tor, atom_tor)) ||
        (rc = upload(&b->d_tor_par, tor_par)) || (rc = encode_intra(pk, b.get(), true))) {
        trids_free_batch(b.release());
        return rc;
    }
    std::vector<unsigned int> zeros(4, 0u);
    std::vector<int> zi(2, 0);
    if ((rc = upload(&b->d_counter, zeros)) || (rc = upload(&b->d_err, zi))) {
        trids_free_batch(b.release());
        return rc;
    }
    b->dims.upload_bytes = (int64_t)(b->hdr.size() * sizeof(LigHdr) + ay.size() * sizeof(float4) +
                                     aorig.size() * sizeof(int) + atom_tor.size() + tor_par.size() +
                                     tidx.size() * sizeof(int4) + (tu.size() + tp.size()) * sizeof(float4) +
                                     ipre.size() * sizeof(int) + b->ient_j.size() * sizeof(uint16_t) +
                                     zeros.size() * sizeof(unsigned int) + zi.size() * sizeof(int));
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
    if (b->graph.exec) cudaGraphExecDestroy(b->graph.exec);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->ev_a) cudaEventDestroy(b->ev_a);
    if (b->ev_b) cudaEventDestroy(b->ev_b);
    cudaFree(b->d_lig); cudaFree(b->d_atom_y); cudaFree(b->d_atom_orig); cudaFree(b->d_tor_idx);
    cudaFree(b->d_tor_u); cudaFree(b->d_tor_p); cudaFree(b->d_ipre); cudaFree(b->d_ient); cudaFree(b->d_items); cudaFree(b->d_lig_order);
    cudaFree(b->d_counter); cudaFree(b->d_err); cudaFree(b->d_partials); cudaFree(b->d_mdn);
    cudaFree(b->d_atom_tor); cudaFree(b->d_tor_par);
    delete b;
    return TRIDS_OK;
}

int trids_set_mdn(trids_batch* b, int32_t n_res, int32_t K, const float* mdn, void* stream) {
    g_err.clear();
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
        (rc = check_device_ptr(c.pair_count, "pair_count", true)) || (rc = check_terms(pk, b)))
        return rc;
    if ((rc = ensure_items(b, c.poses))) return rc;
    Layout L;
    const int warps = pick_warps(c.warps_per_block > 0 ? c.warps_per_block : 20, pk, b, false, &L);
    if (!warps) return fail(TRIDS_EINVAL, "pocket of %d atoms does not fit in shared memory", pk->M);
    SampleArgs A;
    std::memset(&A, 0, sizeof A);  // the bytes form the graph-cache key
    A.pk = pk->view(); A.B = b->view(); A.P = c.poses; A.S = c.steps; A.step_begin = c.step_begin;
    A.step_end = c.step_end; A.Lmc = c.mc_loops; A.lr = c.lr; A.b1 = c.beta1; A.b2 = c.beta2; A.eps = c.eps;
    A.beta = c.beta; A.opt = c.optimizer; A.wd = c.weight_decay; A.momentum = c.momentum; A.alpha = c.alpha;
    A.seed = c.seed; A.lig_base = c.lig_base; A.dof = dof; A.state = state; A.energy = energy;
    A.trace = c.trace; A.trace_slot = c.trace_slot; A.n_trace = c.n_trace; A.pair_count = c.pair_count;
    A.lig_order = b->d_lig_order; A.n_items = b->dims.n_lig * c.poses; A.counter = b->d_counter; A.err = b->d_err;
    A.params_bytes = L.params_bytes; A.pocket_off = L.pocket_off; A.ptype_off = L.ptype_off;
    A.mbar_off = L.mbar_off;
    A.warp_off = L.warp_off; A.warp_bytes = L.warp_bytes;
    cudaStream_t st = (cudaStream_t)stream;
    const int ts = pk->prm.term_set;
    const bool cnt = c.pair_count != nullptr;
    // the general kernels carry the other update rules and the grid maps; the plain ones
    // (Adam, direct pair sums: the paper's configuration) leave that code out
    const bool gen = c.optimizer != TRIDS_OPT_ADAM || pk->d_maps != nullptr;
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
    // CUDA graph (Sec. 4 item 2): counter reset + persistent launch, captured once per
    // argument set and replayed on the caller's stream.  The legacy default stream
    // cannot be captured; for it capture and replay run on a side stream ordered
    // against the caller's by events.
    std::vector<unsigned char> key(sizeof(SampleArgs) + 4 * sizeof(int));
    std::memcpy(key.data(), &A, sizeof(SampleArgs));
    const int extra[4] = {grid, warps, ts, (cnt ? 1 : 0) | (gen ? 2 : 0)};
    std::memcpy(key.data() + sizeof(SampleArgs), extra, sizeof extra);
    const bool legacy = st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread;
    if (legacy && !b->side) {
        CK(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&b->ev_a, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&b->ev_b, cudaEventDisableTiming));
    }
    cudaStream_t run = legacy ? b->side : st;
    if (!b->graph.exec || b->graph.key != key) {
        if (b->graph.exec) { cudaGraphExecDestroy(b->graph.exec); b->graph.exec = nullptr; }
        if (!b->side) CK(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
        cudaStream_t cs = b->side;
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaMemsetAsync(A.counter, 0, sizeof(unsigned int), cs);
        kern<<<grid, 32 * warps, L.total, cs>>>(A);
        cudaError_t le = cudaGetLastError();
        CK(cudaStreamEndCapture(cs, &g));
        if (le != cudaSuccess) { cudaGraphDestroy(g); return fail(TRIDS_ECUDA, "launch during capture: %s", cudaGetErrorString(le)); }
        cudaError_t ie = cudaGraphInstantiate(&b->graph.exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return fail(TRIDS_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
        b->graph.key = key;
    }
    if (!legacy) {
        CK(cudaGraphLaunch(b->graph.exec, run));
        return TRIDS_OK;
    }
    CK(cudaEventRecord(b->ev_a, st));
    CK(cudaStreamWaitEvent(run, b->ev_a, 0));
    CK(cudaGraphLaunch(b->graph.exec, run));
    CK(cudaEventRecord(b->ev_b, run));
    CK(cudaStreamWaitEvent(st, b->ev_b, 0));
    return TRIDS_OK;
}

int trids_topk(const trids_batch* b, int32_t poses, const float* energy, const float* dof, int32_t k, float rmsd,
               int32_t* idx, float* e_out, void* stream) {
    g_err.clear();
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

int trids_sync(const trids_batch* b, int32_t poses, const float* state, void* stream, double timeout_ms) {
    g_err.clear();
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

// Device address of g_noalloc_scratch for `dev`, looked up once per device with that
// device current (host code cannot use the symbol itself as a device address).
static int noalloc_scratch(int dev, unsigned char** out) {
    static std::mutex mu;
    static void* addr[256] = {};
    if (dev < 0 || dev >= 256) return fail(TRIDS_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(TRIDS_ECUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
        addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(addr[dev]);
    return TRIDS_OK;
}

int trids_score_grad_noalloc(const trids_pocket* pk, const trids_batch* b, int32_t poses, const float* dof,
                             float* energy, float* e_inter, float* g_dof, float* g_xyz, const float* e_bar,
                             float* g_w, float* g_radius, void* stream) {
    g_err.clear();
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
