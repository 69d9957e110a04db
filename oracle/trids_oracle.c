/*
 * FP64 CPU oracle for gradient-guided pose sampling (TRIDS, arXiv 2510.24186).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header, table or constant generator with the CUDA
 * library; both sides are written separately from the same written rules.
 *
 * It is deliberately plain: every pair of atoms is visited by a direct double
 * loop (no cell list), every quantity is double precision, and each step follows
 * the method in the order the paper states it.  Functions cite the passage they
 * follow.  Where the paper is silent or garbled the reading taken is stated at
 * the function.
 *
 * Parity status per function (what pins it, see tests/):
 *   or_philox              pinned: cuRAND's host Philox4x32-10 generator
 *   or_rot, or_quat_mat    pinned: scipy.spatial.transform.Rotation
 *   or_pack                pinned: networkx components / eccentricity / BFS / shortest paths
 *   or_pair                pinned: hand-computed closed forms (tests/golden/terms.txt)
 *   or_fk                  pinned: or_fk_brute (independent algorithm) + invariants
 *   or_score               pinned: rigid-motion invariance, FD of energy, 1+1 atom closed form
 *   grid maps              pinned: trilinear reproduces linear fields exactly, grid-point values
 *                          equal the direct one-atom energy, FD of the interpolated energy,
 *                          convergence to the direct sum as the spacing shrinks
 *   residue E_MDN          pinned: closed forms (tests/golden/residue_mdn.txt), a numpy brute force of
 *                          the residue minimum, FD, rigid-motion invariance, argmin tie rule
 *   or_opt_step            pinned: torch.optim.Adam / AdamW / RMSprop / Adagrad / SGD
 *   or_init/perturb/metro  pinned: Philox pin + Shoemake uniformity + beta property
 *   or_sample              pinned: the Monte-Carlo loop (save, perturb, moment reset, accept
 *                          or restore) by a two-loop one-atom trajectory worked without the
 *                          oracle (numpy terms, torch.optim.Adam, raw Philox words) and by a
 *                          replay from the pinned parts, bit for bit, on 1-atom and T = 3-5
 *                          ligands; end-to-end trajectories are chaotic, so a whole sampled
 *                          trajectory is "parity unpinned" beyond the per-step checks
 *   or_topk                pinned: brute-force enumeration on tiny inputs
 *   or_screen_energy       pinned: hand-computed values (w_tor = 0.01), the w_tor = 0 and
 *                          N_tor = 0 identities, the sign of the torsion penalty
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_LMAX 70
#define OR_TMAX 20
#define OR_NT 16
#define OR_KMAX 4
#define OR_PMAX (OR_LMAX * (OR_LMAX - 1) / 2)

#define OR_OK 0
#define OR_EINVAL (-1)

typedef struct {
    int32_t term_set;            /* 0: Vina-form 5 terms, 1: TRIDS E_dock terms */
    int32_t n_types;
    double w[5];
    double radius[OR_NT];
    int32_t flags[OR_NT];        /* bit0 hydrophobic, bit1 donor, bit2 acceptor */
    double cutoff;               /* pair cutoff on the centre distance r */
    double w_tor;
    int32_t gmm_k;
    double gmm[OR_NT * OR_NT * OR_KMAX * 3]; /* [ti][tj][k] = (pi, mu, sigma) */
} or_params;

typedef struct {
    int32_t n_atoms, n_tor, n_pairs;
    int32_t perm[OR_LMAX];       /* packed index -> input index */
    int32_t frag[OR_LMAX];       /* 0 = root fragment, k+1 = moving fragment of torsion k */
    int32_t type[OR_LMAX];
    double y[OR_LMAX][3];        /* input geometry, packed order */
    double c[3];                 /* centroid of the root fragment */
    int32_t tp[OR_TMAX], th[OR_TMAX], tpar[OR_TMAX], sb[OR_TMAX], se[OR_TMAX];
    int32_t pi[OR_PMAX], pj[OR_PMAX];
} or_ligand;

typedef struct {
    double e_total, e_inter, e_intra;
    double g_dof[7 + OR_TMAX];   /* dE/dt, dE/dq (gradient of E(q/|q|)), dE/dtheta */
    double tau[3];               /* world torque = gradient w.r.t. the rotation tangent */
    double g_x[OR_LMAX][3];      /* dE/dx_i, packed order */
    double x[OR_LMAX][3];        /* world coordinates, packed order */
    double g_w[5];               /* dE/dw_t */
    double g_R[OR_NT];           /* dE/dR_a */
    int64_t n_inter, n_intra;    /* pairs inside the cutoff */
    int32_t n_straddle;          /* pairs within OR_STRADDLE of a cutoff or a kink */
    double e_slack, g_slack;     /* summed |value jump| and |dE/dr jump| of those pairs */
    /* condition magnitudes for a rounding bound: sum |pair energy|, and for each DOF the
     * sum over atoms of |lever arm| * (sum of |dE/dr| of the atom's pairs) (t: lever 1;
     * q: the lever about t; theta: the lever about the torsion's parent atom) */
    double e_mag;
    double g_mag[7 + OR_TMAX];
    int64_t n_res_pairs;         /* (ligand atom, residue) pairs inside the E_MDN cutoff */
    int64_t n_map_atoms;         /* ligand atoms scored from the grid maps */
} or_eval;

/* Residue-level E_MDN inputs (term_set 2).  res[j] = residue of pocket atom j;
 * prm[((i * n_res) + r) * K + k] = (pi, mu, sigma) of ligand atom i (input order),
 * residue r, kernel k: the parameters the paper's network predicts per pair. */
typedef struct {
    int32_t n_res, K;
    const int32_t* res;
    const double* prm;
} or_mdn;

/* Grid-map domain (the map form of the ligand-pocket terms): points lo + h (a, b, c),
 * 0 <= a < n[0], 0 <= b < n[1], 0 <= c < n[2]. */
typedef struct {
    double lo[3];
    double h;
    int32_t n[3];
} or_maps;

#define OR_MAX_BOXES 8
typedef struct {
    int32_t steps, mc_loops;
    double lr, b1, b2, eps, beta;
    uint64_t seed;
    int32_t n_boxes;                          /* pose p uses box p mod n_boxes */
    double box_lo[OR_MAX_BOXES][3], box_hi[OR_MAX_BOXES][3];
    int32_t optimizer;                        /* OR_OPT_*; the paper samples with Adam */
    double weight_decay, momentum, alpha;     /* AdamW decay, SGD momentum, RMSprop smoothing */
} or_sample_cfg;

#define OR_OPT_ADAM 0
#define OR_OPT_ADAMW 1
#define OR_OPT_RMSPROP 2
#define OR_OPT_ADAGRAD 3
#define OR_OPT_SGD 4

#define OR_STRADDLE 1e-4

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).  */
/* Round: two 32x32->64 products of counter words 0 and 2 with fixed          */
/* multipliers; the high halves are xored with counter words 1/3 and the key; */
/* the key is bumped by the two Weyl constants between rounds.                 */
/* ------------------------------------------------------------------------- */
void or_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Random stream of one (seed, ligand, pose, loop, purpose): 32-bit word n of the
 * stream is word n%4 of the Philox block with counter
 * (pose, ligand, loop<<16 | purpose<<8 | n/4, 0) and key (seed low, seed high). */
uint32_t or_rand_word(uint64_t seed, uint32_t lig, uint32_t pose, uint32_t loop,
                      uint32_t purpose, uint32_t n)
{
    uint32_t ctr[4] = {pose, lig, (loop << 16) | (purpose << 8) | (n >> 2), 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    or_philox(ctr, key, o);
    return o[n & 3u];
}

/* uniform in [0,1): the top 24 bits times 2^-24 (exact in float and double) */
static double u01(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------------- */
/* Small rotation helpers                                                     */
/* ------------------------------------------------------------------------- */
/* Rodrigues: rotation by angle th about unit axis u (right-hand rule). */
void or_rot(const double u[3], double th, double R[9])
{
    double c = cos(th), s = sin(th), k = 1.0 - c;
    R[0] = c + k * u[0] * u[0];        R[1] = k * u[0] * u[1] - s * u[2]; R[2] = k * u[0] * u[2] + s * u[1];
    R[3] = k * u[1] * u[0] + s * u[2]; R[4] = c + k * u[1] * u[1];        R[5] = k * u[1] * u[2] - s * u[0];
    R[6] = k * u[2] * u[0] - s * u[1]; R[7] = k * u[2] * u[1] + s * u[0]; R[8] = c + k * u[2] * u[2];
}

/* Rotation matrix of the unit quaternion q/|q|, q = (w, x, y, z). */
void or_quat_mat(const double qi[4], double R[9])
{
    double n = sqrt(qi[0] * qi[0] + qi[1] * qi[1] + qi[2] * qi[2] + qi[3] * qi[3]);
    double w = qi[0] / n, x = qi[1] / n, y = qi[2] / n, z = qi[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void mv(const double R[9], const double v[3], double o[3])
{
    o[0] = R[0] * v[0] + R[1] * v[1] + R[2] * v[2];
    o[1] = R[3] * v[0] + R[4] * v[1] + R[5] * v[2];
    o[2] = R[6] * v[0] + R[7] * v[1] + R[8] * v[2];
}

static void mm(const double A[9], const double B[9], double C[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

static void cross(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* a (x) b, quaternions (w, x, y, z) */
static void qmul(const double a[4], const double b[4], double o[4])
{
    double r[4];
    r[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    r[1] = a[0] * b[1] + b[0] * a[1] + a[2] * b[3] - a[3] * b[2];
    r[2] = a[0] * b[2] + b[0] * a[2] + a[3] * b[1] - a[1] * b[3];
    r[3] = a[0] * b[3] + b[0] * a[3] + a[1] * b[2] - a[2] * b[1];
    memcpy(o, r, sizeof r);
}

static void qnormalize(double q[4])
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) q[i] /= n;
}

/* ------------------------------------------------------------------------- */
/* Ligand packing (torsion tree).  The paper fixes only the degrees of freedom */
/* (Sec. 2 "Conformation sampling": translation, rotation, torsion angles of   */
/* rotatable bonds) and N_tor (Eq. E_screen).  Reading taken for the tree:     */
/*  - fragments = connected components after cutting the rotatable bonds;     */
/*  - root = fragment of minimum height in the fragment tree, ties -> the      */
/*    fragment holding the smallest input atom index;                          */
/*  - torsions numbered in BFS order from the root, children ordered by the    */
/*    smallest input atom index of their fragment;                             */
/*  - atoms renumbered in DFS pre-order of fragments (same child order),       */
/*    ascending input index inside a fragment, so each moving subtree is one   */
/*    contiguous range;                                                       */
/*  - intra pairs: atoms in different fragments that are >= 4 bonds apart.    */
/* ------------------------------------------------------------------------- */
int or_pack(int n, const double* xyz, const int32_t* type, int n_types, int nb,
            const int32_t* bonds, const uint8_t* rot, or_ligand* out)
{
    if (n < 1 || n > OR_LMAX || nb < 0 || n_types < 1 || n_types > OR_NT) return OR_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (type[i] < 0 || type[i] >= n_types) return OR_EINVAL;
        for (int d = 0; d < 3; ++d)
            if (!isfinite(xyz[3 * i + d])) return OR_EINVAL;
    }
    static __thread int adj[OR_LMAX][OR_LMAX];
    memset(adj, 0, sizeof adj);
    int n_rot = 0;
    for (int b = 0; b < nb; ++b) {
        int a0 = bonds[2 * b], a1 = bonds[2 * b + 1];
        if (a0 < 0 || a0 >= n || a1 < 0 || a1 >= n || a0 == a1) return OR_EINVAL;
        if (adj[a0][a1]) return OR_EINVAL; /* duplicate bond */
        adj[a0][a1] = adj[a1][a0] = rot[b] ? 2 : 1;
        n_rot += rot[b] ? 1 : 0;
    }
    if (n_rot > OR_TMAX) return OR_EINVAL;
    /* bond-graph distances (BFS from every atom) */
    static __thread int dist[OR_LMAX][OR_LMAX];
    for (int s = 0; s < n; ++s) {
        int q[OR_LMAX], h = 0, t = 0;
        for (int i = 0; i < n; ++i) dist[s][i] = -1;
        dist[s][s] = 0; q[t++] = s;
        while (h < t) {
            int u = q[h++];
            for (int v = 0; v < n; ++v)
                if (adj[u][v] && dist[s][v] < 0) { dist[s][v] = dist[s][u] + 1; q[t++] = v; }
        }
    }
    for (int i = 0; i < n; ++i)
        if (dist[0][i] < 0) return OR_EINVAL; /* disconnected */
    /* fragments: scan atoms in input order, flood over non-rotatable bonds; the
     * provisional fragment id is then ordered by the fragment's smallest atom */
    int lab[OR_LMAX], nf = 0;
    for (int i = 0; i < n; ++i) lab[i] = -1;
    for (int s = 0; s < n; ++s) {
        if (lab[s] >= 0) continue;
        int q[OR_LMAX], h = 0, t = 0;
        lab[s] = nf; q[t++] = s;
        while (h < t) {
            int u = q[h++];
            for (int v = 0; v < n; ++v)
                if (adj[u][v] == 1 && lab[v] < 0) { lab[v] = nf; q[t++] = v; }
        }
        ++nf;
    }
    if (n_rot != nf - 1) return OR_EINVAL; /* a rotatable bond closes a ring */
    int fadj[OR_TMAX + 1][OR_TMAX + 1];
    int fa[OR_TMAX + 1][OR_TMAX + 1]; /* atom of the row fragment on the bond */
    memset(fadj, 0, sizeof fadj);
    for (int b = 0; b < nb; ++b) {
        if (!rot[b]) continue;
        int a0 = bonds[2 * b], a1 = bonds[2 * b + 1];
        int f0 = lab[a0], f1 = lab[a1];
        if (f0 == f1 || fadj[f0][f1]) return OR_EINVAL;
        fadj[f0][f1] = fadj[f1][f0] = 1;
        fa[f0][f1] = a0; fa[f1][f0] = a1;
    }
    /* root = minimum eccentricity in the fragment tree, ties -> lowest id */
    int root = 0, best = 1 << 30;
    for (int s = 0; s < nf; ++s) {
        int d[OR_TMAX + 1], q[OR_TMAX + 1], h = 0, t = 0, ecc = 0;
        for (int f = 0; f < nf; ++f) d[f] = -1;
        d[s] = 0; q[t++] = s;
        while (h < t) {
            int u = q[h++];
            if (d[u] > ecc) ecc = d[u];
            for (int v = 0; v < nf; ++v)
                if (fadj[u][v] && d[v] < 0) { d[v] = d[u] + 1; q[t++] = v; }
        }
        if (ecc < best) { best = ecc; root = s; }
    }
    /* BFS from the root: torsion k = k-th discovered non-root fragment */
    int fpar[OR_TMAX + 1], ftor[OR_TMAX + 1], order[OR_TMAX + 1];
    for (int f = 0; f < nf; ++f) { fpar[f] = -2; ftor[f] = -1; }
    {
        int h = 0, t = 0, k = 0;
        fpar[root] = -1; order[t++] = root;
        while (h < t) {
            int u = order[h++];
            for (int v = 0; v < nf; ++v)          /* ascending id = ascending min atom */
                if (fadj[u][v] && fpar[v] == -2) { fpar[v] = u; ftor[v] = k++; order[t++] = v; }
        }
    }
    /* DFS pre-order of fragments -> packed atom order */
    int newidx[OR_LMAX], np = 0, fstart[OR_TMAX + 1], fend[OR_TMAX + 1];
    {
        int stack[OR_TMAX + 1], sp = 0;
        stack[sp++] = root;
        int visit[OR_TMAX + 1], nv = 0;
        while (sp) {
            int u = stack[--sp];
            visit[nv++] = u;
            for (int v = nf - 1; v >= 0; --v)       /* push in reverse: pop ascending */
                if (fadj[u][v] && fpar[v] == u) stack[sp++] = v;
        }
        for (int i = 0; i < nv; ++i) {
            int f = visit[i];
            fstart[f] = np;
            for (int a = 0; a < n; ++a)
                if (lab[a] == f) { out->perm[np] = a; newidx[a] = np; ++np; }
        }
        /* subtree end: walk the pre-order, a subtree ends where the next
         * fragment that is not a descendant starts */
        for (int i = 0; i < nv; ++i) {
            int f = visit[i], j = i + 1;
            while (j < nv) {
                int g = visit[j], anc = 0;
                while (g >= 0) { if (g == f) { anc = 1; break; } g = fpar[g]; }
                if (!anc) break;
                ++j;
            }
            fend[f] = (j < nv) ? fstart[visit[j]] : n;
        }
    }
    out->n_atoms = n;
    out->n_tor = nf - 1;
    for (int i = 0; i < n; ++i) {
        int a = out->perm[i];
        out->type[i] = type[a];
        for (int d = 0; d < 3; ++d) out->y[i][d] = xyz[3 * a + d];
        out->frag[i] = (lab[a] == root) ? 0 : ftor[lab[a]] + 1;
    }
    for (int f = 0; f < nf; ++f) {
        if (f == root) continue;
        int k = ftor[f], p = fpar[f];
        out->tp[k] = newidx[fa[p][f]];
        out->th[k] = newidx[fa[f][p]];
        out->tpar[k] = (p == root) ? -1 : ftor[p];
        out->sb[k] = fstart[f];
        out->se[k] = fend[f];
    }
    double cn = 0;
    out->c[0] = out->c[1] = out->c[2] = 0;
    for (int i = 0; i < n; ++i)
        if (out->frag[i] == 0) { for (int d = 0; d < 3; ++d) out->c[d] += out->y[i][d]; cn += 1; }
    for (int d = 0; d < 3; ++d) out->c[d] /= cn;
    int npair = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            int ai = out->perm[i], aj = out->perm[j];
            if (out->frag[i] != out->frag[j] && dist[ai][aj] >= 4) {
                out->pi[npair] = i; out->pj[npair] = j; ++npair;
            }
        }
    out->n_pairs = npair;
    return OR_OK;
}

/* Flat topology: [L, T, n_pairs, perm[L], frag[L], T x (tp, th, tpar, sb, se), n_pairs x (i, j)] */
int or_topology(const or_ligand* lg, int32_t* o, int cap)
{
    int L = lg->n_atoms, T = lg->n_tor, P = lg->n_pairs;
    int need = 3 + 2 * L + 5 * T + 2 * P;
    if (cap < need) return -need;
    int k = 0;
    o[k++] = L; o[k++] = T; o[k++] = P;
    for (int i = 0; i < L; ++i) o[k++] = lg->perm[i];
    for (int i = 0; i < L; ++i) o[k++] = lg->frag[i];
    for (int t = 0; t < T; ++t) {
        o[k++] = lg->tp[t]; o[k++] = lg->th[t]; o[k++] = lg->tpar[t]; o[k++] = lg->sb[t]; o[k++] = lg->se[t];
    }
    for (int p = 0; p < P; ++p) { o[k++] = lg->pi[p]; o[k++] = lg->pj[p]; }
    return need;
}

/* ------------------------------------------------------------------------- */
/* Forward kinematics (Sec. 2 "Conformation sampling"; Sec. 4 item 3).        */
/* x_i = t + R(q/|q|) z_i, z = local coordinates about the root centroid c     */
/* after the torsions.  Torsion k turns its moving subtree by theta_k about    */
/* the bond from parent atom p_k to child atom h_k (right-hand rule, theta = 0 */
/* is the input geometry).                                                     */
/* ------------------------------------------------------------------------- */

/* Frame composition, root to leaves: fragment f maps y to R_f (y - c) + o_f. */
static void fk_frames(const or_ligand* lg, const double* dof, double Rf[][9], double of[][3])
{
    int T = lg->n_tor;
    for (int d = 0; d < 9; ++d) Rf[0][d] = (d % 4 == 0) ? 1.0 : 0.0;
    of[0][0] = of[0][1] = of[0][2] = 0;
    for (int k = 0; k < T; ++k) {            /* BFS order: parent frame is ready */
        int P = (lg->tpar[k] < 0) ? 0 : lg->tpar[k] + 1, C = k + 1;
        const double* yp = lg->y[lg->tp[k]];
        const double* yh = lg->y[lg->th[k]];
        double u[3] = {yh[0] - yp[0], yh[1] - yp[1], yh[2] - yp[2]};
        double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int d = 0; d < 3; ++d) u[d] /= un;
        double Rk[9], pc[3] = {yp[0] - lg->c[0], yp[1] - lg->c[1], yp[2] - lg->c[2]}, zp[3], t1[3];
        or_rot(u, dof[7 + k], Rk);
        mm(Rf[P], Rk, Rf[C]);
        mv(Rf[P], pc, zp);
        for (int d = 0; d < 3; ++d) zp[d] += of[P][d];
        mv(Rf[C], pc, t1);
        for (int d = 0; d < 3; ++d) of[C][d] = zp[d] - t1[d];
    }
}

void or_fk(const or_ligand* lg, const double* dof, double* x)
{
    double Rf[OR_TMAX + 1][9], of[OR_TMAX + 1][3], Rq[9];
    fk_frames(lg, dof, Rf, of);
    or_quat_mat(dof + 3, Rq);
    for (int i = 0; i < lg->n_atoms; ++i) {
        int f = lg->frag[i];
        double yc[3] = {lg->y[i][0] - lg->c[0], lg->y[i][1] - lg->c[1], lg->y[i][2] - lg->c[2]};
        double z[3], w[3];
        mv(Rf[f], yc, z);
        for (int d = 0; d < 3; ++d) z[d] += of[f][d];
        mv(Rq, z, w);
        for (int d = 0; d < 3; ++d) x[3 * i + d] = dof[d] + w[d];
    }
}

/* Independent check: rotate the full coordinate array by explicit Rodrigues
 * matrices, deepest torsion first, about the input-geometry axes (the axis atoms
 * of a torsion are never moved by the torsions below it), then place rigidly. */
void or_fk_brute(const or_ligand* lg, const double* dof, double* x)
{
    double y[OR_LMAX][3], Rq[9];
    int L = lg->n_atoms;
    memcpy(y, lg->y, sizeof(double) * 3 * L);
    for (int k = lg->n_tor - 1; k >= 0; --k) {
        const double* p = lg->y[lg->tp[k]];
        const double* h = lg->y[lg->th[k]];
        double u[3] = {h[0] - p[0], h[1] - p[1], h[2] - p[2]};
        double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int d = 0; d < 3; ++d) u[d] /= un;
        double R[9];
        or_rot(u, dof[7 + k], R);
        for (int i = 0; i < L; ++i) {
            int inside = 0, f = lg->frag[i];
            while (f > 0) { if (f - 1 == k) { inside = 1; break; } f = lg->tpar[f - 1] + 1; }
            if (!inside) continue;
            double v[3] = {y[i][0] - p[0], y[i][1] - p[1], y[i][2] - p[2]}, r[3];
            mv(R, v, r);
            for (int d = 0; d < 3; ++d) y[i][d] = p[d] + r[d];
        }
    }
    or_quat_mat(dof + 3, Rq);
    for (int i = 0; i < L; ++i) {
        double v[3] = {y[i][0] - lg->c[0], y[i][1] - lg->c[1], y[i][2] - lg->c[2]}, w[3];
        mv(Rq, v, w);
        for (int d = 0; d < 3; ++d) x[3 * i + d] = dof[d] + w[d];
    }
}

/* ------------------------------------------------------------------------- */
/* Pair terms.  Values are unweighted per term; dr = d/dr, dR = d/d(R_a+R_b).  */
/* ------------------------------------------------------------------------- */
static int hyd_pair(const or_params* p, int a, int b) { return (p->flags[a] & 1) && (p->flags[b] & 1); }
static int hb_pair(const or_params* p, int a, int b)
{
    return ((p->flags[a] & 2) && (p->flags[b] & 4)) || ((p->flags[a] & 4) && (p->flags[b] & 2));
}

/*
 * term_set 0, Vina form (the analytic terms the DSDP line samples with; Sec. 1
 * and Sec. 2 name Vina's second Gaussian).  Surface distance d = r - R_a - R_b:
 *   gauss1 = exp(-(d/0.5)^2), gauss2 = exp(-((d-3)/2)^2), repulsion = d^2 (d<0),
 *   hydrophobic (both hydrophobic) = 1 (d<0.5), 1.5-d (d<1.5), else 0,
 *   hbond (donor-acceptor) = 1 (d<-0.7), -d/0.7 (d<0), else 0.
 * term_set 2: as term_set 1 without the atom-pair e0; E_MDN is then the
 *   residue-level sum of residue_mdn below.
 * term_set 1, the TRIDS E_dock terms (Sec. 2 "Scoring functions"), on r:
 *   e0 = E_MDN pair = -sum_k pi_k exp(-(r-mu_k)^2 / (2 sigma_k^2)) for r < 5 (inter only);
 *        exponent sign read as negative (Gaussian), no normalisation, as printed;
 *   e1 = E_long pair = -exp(-(r - d_vdw - 3)^2 / 4) for r < 10 (Vina gauss2 form);
 *   e2 = E_clash pair = -log(max(r,0.5)/d_clash) for r < d_clash, d_clash = 2.6 for a
 *        donor-acceptor pair else d_vdw (indicator read as r < d_clash);
 *   e3 = E_Hbond pair = -exp(-(r-2.88)^2/(2*0.3^2)) for donor-acceptor pairs, r < 3.4.
 */
void or_pair(const or_params* p, int ti, int tj, double r, int inter,
             double e[5], double dr[5], double dR[5], double* vjump, double* gjump)
{
    for (int t = 0; t < 5; ++t) e[t] = dr[t] = dR[t] = 0;
    double Rs = p->radius[ti] + p->radius[tj];
    int hyd = hyd_pair(p, ti, tj), hb = hb_pair(p, ti, tj);
    double vj = 0, gj = 0;
#define NEAR(a, b) (fabs((a) - (b)) < OR_STRADDLE)
    if (p->term_set == 0) {
        double d = r - Rs;
        double a = d / 0.5, g1 = exp(-a * a);
        e[0] = g1; dr[0] = -2.0 * a * g1 / 0.5;
        double b = (d - 3.0) / 2.0, g2 = exp(-b * b);
        e[1] = g2; dr[1] = -2.0 * b * g2 / 2.0;
        if (d < 0) { e[2] = d * d; dr[2] = 2.0 * d; }
        if (hyd) {
            if (d < 0.5) { e[3] = 1.0; }
            else if (d < 1.5) { e[3] = 1.5 - d; dr[3] = -1.0; }
            if (NEAR(d, 0.5) || NEAR(d, 1.5)) gj += fabs(p->w[3]);
        }
        if (hb) {
            if (d < -0.7) { e[4] = 1.0; }
            else if (d < 0) { e[4] = -d / 0.7; dr[4] = -1.0 / 0.7; }
            if (NEAR(d, -0.7) || NEAR(d, 0.0)) gj += fabs(p->w[4]) / 0.7;
        }
        for (int t = 0; t < 5; ++t) dR[t] = -dr[t];
    } else {
        const int atom_mdn = inter && p->term_set == 1;
        if (atom_mdn && r < 5.0) {
            const double* g = p->gmm + ((size_t)(ti * OR_NT + tj) * OR_KMAX) * 3;
            double P = 0, dP = 0;
            for (int k = 0; k < p->gmm_k; ++k) {
                double pk = g[3 * k], mu = g[3 * k + 1], sg = g[3 * k + 2];
                double z = r - mu, ex = pk * exp(-z * z / (2.0 * sg * sg));
                P += ex; dP += -ex * z / (sg * sg);
            }
            e[0] = -P; dr[0] = -dP;
        }
        if (atom_mdn && NEAR(r, 5.0)) {
            const double* g = p->gmm + ((size_t)(ti * OR_NT + tj) * OR_KMAX) * 3;
            for (int k = 0; k < p->gmm_k; ++k) {
                double z = 5.0 - g[3 * k + 1];
                double ex = g[3 * k] * exp(-z * z / (2.0 * g[3 * k + 2] * g[3 * k + 2]));
                vj += fabs(p->w[0] * ex);
                gj += fabs(p->w[0] * ex * z / (g[3 * k + 2] * g[3 * k + 2]));
            }
        }
        double zl = r - Rs - 3.0, gl = exp(-zl * zl / 4.0);
        if (r < 10.0) { e[1] = -gl; dr[1] = gl * zl / 2.0; dR[1] = -dr[1]; }
        if (NEAR(r, 10.0)) { vj += fabs(p->w[1] * gl); gj += fabs(p->w[1] * gl * zl / 2.0); }
        double dcl = hb ? 2.6 : Rs;
        if (r < dcl) {
            double rr = (r < 0.5) ? 0.5 : r;
            e[2] = -log(rr / dcl);
            dr[2] = (r < 0.5) ? 0.0 : -1.0 / r;
            dR[2] = hb ? 0.0 : 1.0 / dcl;
        }
        if (NEAR(r, dcl)) gj += fabs(p->w[2] / dcl);
        if (NEAR(r, 0.5)) gj += fabs(p->w[2] / 0.5);
        if (hb) {
            double zh = r - 2.88, gh = exp(-zh * zh / (2.0 * 0.3 * 0.3));
            if (r < 3.4) { e[3] = -gh; dr[3] = gh * zh / (0.3 * 0.3); }
            if (NEAR(r, 3.4)) { vj += fabs(p->w[3] * gh); gj += fabs(p->w[3] * gh * zh / 0.09); }
        }
    }
    if (NEAR(r, p->cutoff)) {
        double ev = 0, gv = 0;
        for (int t = 0; t < 5; ++t) { ev += p->w[t] * e[t]; gv += p->w[t] * dr[t]; }
        vj += fabs(ev); gj += fabs(gv);
    }
#undef NEAR
    *vjump = vj; *gjump = gj;
}

/* ------------------------------------------------------------------------- */
/* Score and gradient (Sec. 2: E_dock is a weighted sum of pairwise-distance   */
/* terms, so its gradient passes to the atom coordinates; Sec. 4 item 3:      */
/* analytic gradients of the Gaussian terms and of the DOF-to-coordinate map). */
/* E_total = inter (ligand-pocket) + intra (ligand-ligand pair list).          */
/* ------------------------------------------------------------------------- */
static void accumulate_pair(const or_params* p, int ti, int tj, const double* xi, const double* xj,
                            int inter, double* E, double* gi, double* gj, or_eval* ev, double scale,
                            double* mi, double* mj)
{
    double dx = xi[0] - xj[0], dy = xi[1] - xj[1], dz = xi[2] - xj[2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (!(r < p->cutoff)) {
        if (fabs(r - p->cutoff) < OR_STRADDLE) {
            double e[5], dr[5], dR[5], vj, gj2;
            or_pair(p, ti, tj, r, inter, e, dr, dR, &vj, &gj2);
            ev->n_straddle++; ev->e_slack += vj; ev->g_slack += gj2;
        }
        return;
    }
    double e[5], dr[5], dR[5], vj, gjump;
    or_pair(p, ti, tj, r, inter, e, dr, dR, &vj, &gjump);
    if (vj > 0 || gjump > 0) { ev->n_straddle++; ev->e_slack += vj; ev->g_slack += gjump; }
    double es = 0, dEdr = 0, dEdR = 0;
    for (int t = 0; t < 5; ++t) {
        es += p->w[t] * e[t];
        dEdr += p->w[t] * dr[t];
        dEdR += p->w[t] * dR[t];
        ev->g_w[t] += scale * e[t];
    }
    ev->g_R[ti] += scale * dEdR;
    ev->g_R[tj] += scale * dEdR;
    *E += es;
    ev->e_mag += fabs(es);
    *mi += fabs(dEdr);
    if (mj) *mj += fabs(dEdr);
    if (r > 0) {
        double f = dEdr / r;
        gi[0] += f * dx; gi[1] += f * dy; gi[2] += f * dz;
        if (gj) { gj[0] -= f * dx; gj[1] -= f * dy; gj[2] -= f * dz; }
    }
    if (inter) ev->n_inter++; else ev->n_intra++;
}

/*
 * Residue-level E_MDN (Sec. 2, Eqs. P(d) and E_MDN): d_ir = the minimum distance
 * between ligand atom i and the atoms of pocket residue r; each (i, r) with d_ir < 5 A
 * adds w0 * (-sum_k pi_k exp(-(d_ir - mu_k)^2 / (2 sigma_k^2))).  Readings: the exponent
 * is negative (a Gaussian) and P is unnormalised, as for the atom-pair form.  The force
 * acts along the nearest atom (the subgradient of the minimum; equal distances -> the
 * lowest atom index).  A pair within OR_STRADDLE of the cutoff, or whose two nearest
 * atoms are within OR_STRADDLE of each other, is a counted straddle.
 */
int or_score_mdn(const or_params* p, int M, const double* pxyz, const int32_t* ptype, const or_mdn* md,
                 const or_ligand* lg, const double* dof, or_eval* ev);

static void residue_mdn(const or_params* p, int M, const double* pxyz, const or_mdn* md, const or_ligand* lg,
                        or_eval* ev, double* gm)
{
    const int R = md->n_res, K = md->K;
    double* best = (double*)malloc(sizeof(double) * 2 * R);
    int* arg = (int*)malloc(sizeof(int) * R);
    double* second = best + R;
    for (int i = 0; i < lg->n_atoms; ++i) {
        const double* x = ev->x[i];
        for (int r = 0; r < R; ++r) { best[r] = second[r] = INFINITY; arg[r] = -1; }
        for (int a = 0; a < M; ++a) {
            const int r = md->res[a];
            double dx = x[0] - pxyz[3 * a], dy = x[1] - pxyz[3 * a + 1], dz = x[2] - pxyz[3 * a + 2];
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            if (d < best[r]) { second[r] = best[r]; best[r] = d; arg[r] = a; }
            else if (d < second[r]) second[r] = d;
        }
        const double* pi_row = md->prm + (size_t)lg->perm[i] * R * K * 3;
        for (int r = 0; r < R; ++r) {
            if (arg[r] < 0) continue;
            const double d = best[r];
            const double* g = pi_row + (size_t)r * K * 3;
            double P = 0, dP = 0;
            for (int k = 0; k < K; ++k) {
                double z = d - g[3 * k + 1], s2 = g[3 * k + 2] * g[3 * k + 2];
                double ex = g[3 * k] * exp(-z * z / (2.0 * s2));
                P += ex;
                dP -= ex * z / s2;
            }
            const double e = -P, dEdd = -dP;   /* unweighted term and its d-derivative */
            if (fabs(d - 5.0) < OR_STRADDLE) {
                ev->n_straddle++;
                ev->e_slack += fabs(p->w[0] * e);
                ev->g_slack += fabs(p->w[0] * dEdd);
            }
            if (!(d < 5.0)) continue;
            if (second[r] - d < OR_STRADDLE) { ev->n_straddle++; ev->g_slack += 2.0 * fabs(p->w[0] * dEdd); }
            ev->e_inter += p->w[0] * e;
            ev->g_w[0] += e;
            ev->e_mag += fabs(p->w[0] * e);
            gm[i] += fabs(p->w[0] * dEdd);
            ev->n_res_pairs++;
            if (d > 0) {
                const double* xa = pxyz + 3 * arg[r];
                double f = p->w[0] * dEdd / d;
                for (int c = 0; c < 3; ++c) ev->g_x[i][c] += f * (x[c] - xa[c]);
            }
        }
    }
    free(best);
    free(arg);
}

/*
 * Grid-map form of the ligand-pocket atom-pair terms (the DSDP / Vina practice; the paper
 * itself scores pairs directly, Sec. 4 item 4).  The map of ligand type ti holds at each
 * grid point g the ligand-pocket energy an atom of that type would have there: the sum of
 * the weighted pair terms over pocket atoms with |g - p_j| < cutoff.  An atom whose cell
 * (all 8 corners) lies inside the domain takes the trilinear interpolation of its cell's
 * corner values and the analytic derivative of that interpolation; any other atom keeps
 * the direct sum.  The residue-level E_MDN (term set 2) is never mapped.
 * Slack (counted as straddles): corner pairs on the cutoff or a value jump; an atom within
 * OR_STRADDLE (A) of a cell face (the gradient differs between the two cells) or of the
 * domain boundary (interpolated vs direct).
 */
static double map_value(const or_params* p, int M, const double* pxyz, const int32_t* ptype, int ti,
                        const double g[3], double* jump)
{
    double E = 0;
    for (int j = 0; j < M; ++j) {
        double dx = g[0] - pxyz[3 * j], dy = g[1] - pxyz[3 * j + 1], dz = g[2] - pxyz[3 * j + 2];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        double e[5], dr[5], dR[5], vj, gj;
        if (!(r < p->cutoff) && !(fabs(r - p->cutoff) < OR_STRADDLE)) continue;
        or_pair(p, ti, ptype[j], r, 1, e, dr, dR, &vj, &gj);
        double es = 0;
        for (int t = 0; t < 5; ++t) es += p->w[t] * e[t];
        *jump += vj;
        if (r < p->cutoff) E += es;
    }
    return E;
}

/* Interpolated energy and gradient in cell c (corner values V[a][b][k] at c + (a, b, k)). */
static void trilinear(const double V[2][2][2], const double f[3], double h, double* E, double g[3])
{
    double e = 0, gx = 0, gy = 0, gz = 0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int k = 0; k < 2; ++k) {
                double wx = a ? f[0] : 1 - f[0], wy = b ? f[1] : 1 - f[1], wz = k ? f[2] : 1 - f[2];
                double sx = a ? 1 : -1, sy = b ? 1 : -1, sz = k ? 1 : -1;
                e += wx * wy * wz * V[a][b][k];
                gx += sx * wy * wz * V[a][b][k];
                gy += wx * sy * wz * V[a][b][k];
                gz += wx * wy * sz * V[a][b][k];
            }
    *E = e;
    g[0] = gx / h; g[1] = gy / h; g[2] = gz / h;
}

static void cell_corners(const or_params* p, int M, const double* pxyz, const int32_t* ptype, const or_maps* mp,
                         int ti, const int c[3], double V[2][2][2], double* jump)
{
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int k = 0; k < 2; ++k) {
                double g[3] = {mp->lo[0] + mp->h * (c[0] + a), mp->lo[1] + mp->h * (c[1] + b),
                               mp->lo[2] + mp->h * (c[2] + k)};
                V[a][b][k] = map_value(p, M, pxyz, ptype, ti, g, jump);
            }
}

static int cell_inside(const or_maps* mp, const int c[3])
{
    for (int d = 0; d < 3; ++d)
        if (c[d] < 0 || c[d] + 1 >= mp->n[d]) return 0;
    return 1;
}

/* Map energy of atom i (returns 0 when the atom is left to the direct sum). */
static int map_atom(const or_params* p, int M, const double* pxyz, const int32_t* ptype, const or_maps* mp,
                    int ti, const double* x, double* E, double g[3], or_eval* ev, double* mag)
{
    double u[3], f[3];
    int c[3];
    for (int d = 0; d < 3; ++d) {
        u[d] = (x[d] - mp->lo[d]) / mp->h;
        c[d] = (int)floor(u[d]);
        f[d] = u[d] - c[d];
    }
    const double tol = OR_STRADDLE / mp->h;
    int inside = cell_inside(mp, c);
    int near_edge = 0;
    for (int d = 0; d < 3; ++d)
        if (fabs(u[d]) < tol || fabs(u[d] - (mp->n[d] - 1)) < tol) near_edge = 1;
    if (!inside && !near_edge) return 0;
    double V[2][2][2], jump = 0, Em = 0, gm3[3] = {0, 0, 0};
    if (inside) {
        cell_corners(p, M, pxyz, ptype, mp, ti, c, V, &jump);
        trilinear(V, f, mp->h, &Em, gm3);
        double sv = 0;
        for (int a = 0; a < 8; ++a) sv += fabs(((double*)V)[a]);
        *mag += 2.0 * sv / mp->h;
        ev->e_mag += sv;
        ev->e_slack += jump;
        if (jump > 0) ev->n_straddle++;
        /* near a face: the neighbouring cell's gradient */
        for (int d = 0; d < 3; ++d) {
            int side = f[d] < tol ? -1 : (f[d] > 1 - tol ? 1 : 0);
            if (!side) continue;
            int c2[3] = {c[0], c[1], c[2]};
            c2[d] += side;
            if (!cell_inside(mp, c2)) continue;   /* the domain-boundary case below covers it */
            double V2[2][2][2], j2 = 0, E2, g2[3], f2[3] = {f[0], f[1], f[2]};
            f2[d] = side < 0 ? f[d] + 1.0 : f[d] - 1.0;
            cell_corners(p, M, pxyz, ptype, mp, ti, c2, V2, &j2);
            trilinear(V2, f2, mp->h, &E2, g2);
            ev->n_straddle++;
            ev->g_slack += sqrt((g2[0] - gm3[0]) * (g2[0] - gm3[0]) + (g2[1] - gm3[1]) * (g2[1] - gm3[1]) +
                                (g2[2] - gm3[2]) * (g2[2] - gm3[2]));
        }
    }
    if (near_edge) {
        /* the GPU may take the other side of the domain boundary: interpolated vs direct */
        double Ed = 0, gd[3] = {0, 0, 0};
        for (int j = 0; j < M; ++j) {
            double dx = x[0] - pxyz[3 * j], dy = x[1] - pxyz[3 * j + 1], dz = x[2] - pxyz[3 * j + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (!(r < p->cutoff)) continue;
            double e[5], dr[5], dR[5], vj, gj;
            or_pair(p, ti, ptype[j], r, 1, e, dr, dR, &vj, &gj);
            double es = 0, de = 0;
            for (int t = 0; t < 5; ++t) { es += p->w[t] * e[t]; de += p->w[t] * dr[t]; }
            Ed += es;
            if (r > 0) { gd[0] += de * dx / r; gd[1] += de * dy / r; gd[2] += de * dz / r; }
        }
        ev->n_straddle++;
        if (inside) {
            ev->e_slack += fabs(Em - Ed);
            ev->g_slack += sqrt((gd[0] - gm3[0]) * (gd[0] - gm3[0]) + (gd[1] - gm3[1]) * (gd[1] - gm3[1]) +
                                (gd[2] - gm3[2]) * (gd[2] - gm3[2]));
        } else {
            /* outside by a hair: the direct sum stays, with the map's cell as the alternative */
            int c2[3];
            double f2[3];
            for (int d = 0; d < 3; ++d) {
                c2[d] = c[d] < 0 ? 0 : (c[d] > mp->n[d] - 2 ? mp->n[d] - 2 : c[d]);
                f2[d] = u[d] - c2[d];
            }
            double V2[2][2][2], j2 = 0, E2, g2[3];
            cell_corners(p, M, pxyz, ptype, mp, ti, c2, V2, &j2);
            trilinear(V2, f2, mp->h, &E2, g2);
            ev->e_slack += fabs(E2 - Ed);
            ev->g_slack += sqrt((gd[0] - g2[0]) * (gd[0] - g2[0]) + (gd[1] - g2[1]) * (gd[1] - g2[1]) +
                                (gd[2] - g2[2]) * (gd[2] - g2[2]));
            return 0;
        }
    }
    *E = Em;
    g[0] = gm3[0]; g[1] = gm3[1]; g[2] = gm3[2];
    return 1;
}

int or_score_full(const or_params* p, int M, const double* pxyz, const int32_t* ptype, const or_mdn* md,
                  const or_maps* mp, const or_ligand* lg, const double* dof, or_eval* ev);

int or_score(const or_params* p, int M, const double* pxyz, const int32_t* ptype,
             const or_ligand* lg, const double* dof, or_eval* ev)
{
    return or_score_full(p, M, pxyz, ptype, NULL, NULL, lg, dof, ev);
}

int or_score_mdn(const or_params* p, int M, const double* pxyz, const int32_t* ptype, const or_mdn* md,
                 const or_ligand* lg, const double* dof, or_eval* ev)
{
    return or_score_full(p, M, pxyz, ptype, md, NULL, lg, dof, ev);
}

/* term_set 2 needs md (residues and per-pair kernels); other term sets ignore it.
 * mp (nullable): grid-map form of the ligand-pocket atom-pair terms. */
int or_score_full(const or_params* p, int M, const double* pxyz, const int32_t* ptype, const or_mdn* md,
                  const or_maps* mp, const or_ligand* lg, const double* dof, or_eval* ev)
{
    memset(ev, 0, sizeof *ev);
    if (p->term_set == 2 && !md) return OR_EINVAL;
    int L = lg->n_atoms, T = lg->n_tor;
    double Rf[OR_TMAX + 1][9], of[OR_TMAX + 1][3], Rq[9];
    fk_frames(lg, dof, Rf, of);
    or_quat_mat(dof + 3, Rq);
    or_fk(lg, dof, &ev->x[0][0]);
    double gm[OR_LMAX];
    for (int i = 0; i < L; ++i) gm[i] = 0;
    for (int i = 0; i < L; ++i) {
        double Em, gmap[3];
        if (mp && map_atom(p, M, pxyz, ptype, mp, lg->type[i], ev->x[i], &Em, gmap, ev, &gm[i])) {
            ev->e_inter += Em;
            for (int d = 0; d < 3; ++d) ev->g_x[i][d] += gmap[d];
            ev->n_map_atoms++;
            continue;
        }
        for (int j = 0; j < M; ++j)
            accumulate_pair(p, lg->type[i], ptype[j], ev->x[i], pxyz + 3 * j, 1,
                            &ev->e_inter, ev->g_x[i], NULL, ev, 1.0, &gm[i], NULL);
    }
    for (int k = 0; k < lg->n_pairs; ++k) {
        int i = lg->pi[k], j = lg->pj[k];
        accumulate_pair(p, lg->type[i], lg->type[j], ev->x[i], ev->x[j], 0,
                        &ev->e_intra, ev->g_x[i], ev->g_x[j], ev, 1.0, &gm[i], &gm[j]);
    }
    if (p->term_set == 2) residue_mdn(p, M, pxyz, md, lg, ev, gm);
    for (int i = 0; i < L; ++i) {
        double lt = sqrt((ev->x[i][0] - dof[0]) * (ev->x[i][0] - dof[0]) + (ev->x[i][1] - dof[1]) * (ev->x[i][1] - dof[1]) +
                         (ev->x[i][2] - dof[2]) * (ev->x[i][2] - dof[2]));
        for (int d = 0; d < 3; ++d) ev->g_mag[d] += gm[i];
        for (int d = 0; d < 4; ++d) ev->g_mag[3 + d] += 2.0 * lt * gm[i];
    }
    for (int k = 0; k < T; ++k) {
        const double* pk0 = ev->x[lg->tp[k]];
        for (int i = lg->sb[k]; i < lg->se[k]; ++i) {
            double lv = sqrt((ev->x[i][0] - pk0[0]) * (ev->x[i][0] - pk0[0]) + (ev->x[i][1] - pk0[1]) * (ev->x[i][1] - pk0[1]) +
                             (ev->x[i][2] - pk0[2]) * (ev->x[i][2] - pk0[2]));
            ev->g_mag[7 + k] += lv * gm[i];
        }
    }
    ev->e_total = ev->e_inter + ev->e_intra;
    /* adjoint: translation, rotation tangent, torsions */
    for (int i = 0; i < L; ++i) {
        double rel[3] = {ev->x[i][0] - dof[0], ev->x[i][1] - dof[1], ev->x[i][2] - dof[2]}, c[3];
        cross(rel, ev->g_x[i], c);
        for (int d = 0; d < 3; ++d) { ev->g_dof[d] += ev->g_x[i][d]; ev->tau[d] += c[d]; }
    }
    /* dE/dq for E(q/|q|): 4 M(qhat) tau / |q|, M(q) = 1/2 [-v^T ; w I - [v]x] */
    {
        const double* q = dof + 3;
        double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double w = q[0] / n, v[3] = {q[1] / n, q[2] / n, q[3] / n}, vt[3];
        cross(v, ev->tau, vt);
        ev->g_dof[3] = 2.0 * (-(v[0] * ev->tau[0] + v[1] * ev->tau[1] + v[2] * ev->tau[2])) / n;
        for (int d = 0; d < 3; ++d) ev->g_dof[4 + d] = 2.0 * (w * ev->tau[d] - vt[d]) / n;
    }
    for (int k = 0; k < T; ++k) {
        int P = (lg->tpar[k] < 0) ? 0 : lg->tpar[k] + 1;
        const double* yp = lg->y[lg->tp[k]];
        const double* yh = lg->y[lg->th[k]];
        double u[3] = {yh[0] - yp[0], yh[1] - yp[1], yh[2] - yp[2]};
        double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int d = 0; d < 3; ++d) u[d] /= un;
        double a1[3], a[3];
        mv(Rf[P], u, a1);
        mv(Rq, a1, a);                       /* world axis */
        const double* pk = ev->x[lg->tp[k]];  /* world point on the axis */
        double s = 0;
        for (int i = lg->sb[k]; i < lg->se[k]; ++i) {
            double rel[3] = {ev->x[i][0] - pk[0], ev->x[i][1] - pk[1], ev->x[i][2] - pk[2]}, c[3];
            cross(rel, ev->g_x[i], c);
            s += a[0] * c[0] + a[1] * c[1] + a[2] * c[2];
        }
        ev->g_dof[7 + k] = s;
    }
    return isfinite(ev->e_total) ? OR_OK : -5;
}

/* ------------------------------------------------------------------------- */
/* Sampling (Sec. 2 "Conformation sampling", Fig. 2): random initial copies,   */
/* then loops of {perturb one variable, Adam refinement (lr 0.1), Metropolis   */
/* acceptance rand(0,1) < exp(-beta dE), beta = 0.069}.                         */
/* Readings where the paper is silent: loop l gets floor(S/Lmc) evaluations,   */
/* +1 for the first S mod Lmc loops; inside a loop every evaluation but the   */
/* last is followed by an Adam update and the last one gives the loop-end     */
/* energy; Adam moments reset at each loop start; a rejected loop restores    */
/* the state saved before its perturbation.  Rotation: unit quaternion with   */
/* Adam on a world rotation vector, q <- exp(dw/2) (x) q.                      */
/* ------------------------------------------------------------------------- */
int or_loop_steps(int S, int Lmc, int l) { return S / Lmc + ((l < S % Lmc) ? 1 : 0); }

static double wrap_pi(double a) { return a - 2.0 * M_PI * floor((a + M_PI) / (2.0 * M_PI)); }

/* Translation range of a pose (Sec. 2: t in [box_min, box_max]); with several docking
 * boxes (one per candidate cavity) pose p samples in box p mod n_boxes. */
static const double* box_lo(const or_sample_cfg* cfg, uint32_t pose)
{
    return cfg->box_lo[cfg->n_boxes > 1 ? pose % (uint32_t)cfg->n_boxes : 0];
}
static const double* box_hi(const or_sample_cfg* cfg, uint32_t pose)
{
    return cfg->box_hi[cfg->n_boxes > 1 ? pose % (uint32_t)cfg->n_boxes : 0];
}

void or_init_pose(const or_sample_cfg* cfg, int T, uint32_t lig, uint32_t pose, double* dof)
{
    double u[3 + 3 + OR_TMAX];
    const double *lo = box_lo(cfg, pose), *hi = box_hi(cfg, pose);
    for (int n = 0; n < 6 + T; ++n) u[n] = u01(or_rand_word(cfg->seed, lig, pose, 0, 0, (uint32_t)n));
    for (int d = 0; d < 3; ++d) dof[d] = lo[d] + u[d] * (hi[d] - lo[d]);
    /* Shoemake's subgroup method for a uniform unit quaternion */
    double a = sqrt(1.0 - u[3]), b = sqrt(u[3]);
    dof[3] = a * sin(2.0 * M_PI * u[4]);
    dof[4] = a * cos(2.0 * M_PI * u[4]);
    dof[5] = b * sin(2.0 * M_PI * u[5]);
    dof[6] = b * cos(2.0 * M_PI * u[5]);
    for (int k = 0; k < T; ++k) dof[7 + k] = -M_PI + 2.0 * M_PI * u[6 + k];
}

/* one scalar of the 6+T variables, drawn uniformly, is resampled in its range */
int or_perturb(const or_sample_cfg* cfg, int T, uint32_t lig, uint32_t pose, uint32_t loop, double* dof)
{
    uint32_t w0 = or_rand_word(cfg->seed, lig, pose, loop, 1, 0);
    double u1 = u01(or_rand_word(cfg->seed, lig, pose, loop, 1, 1));
    int c = (int)(((uint64_t)(w0 >> 8) * (uint64_t)(6 + T)) >> 24);
    if (c < 3) {
        dof[c] = box_lo(cfg, pose)[c] + u1 * (box_hi(cfg, pose)[c] - box_lo(cfg, pose)[c]);
    } else if (c < 6) {
        double ang = -M_PI + 2.0 * M_PI * u1;
        double r[4] = {cos(0.5 * ang), 0, 0, 0};
        r[1 + (c - 3)] = sin(0.5 * ang);
        qmul(r, dof + 3, dof + 3);
        qnormalize(dof + 3);
    } else {
        dof[7 + (c - 6)] = -M_PI + 2.0 * M_PI * u1;
    }
    return c;
}

double or_metropolis_u(uint64_t seed, uint32_t lig, uint32_t pose, uint32_t loop)
{
    return u01(or_rand_word(seed, lig, pose, loop, 2, 0));
}

int or_metropolis_accept(double e_new, double e_old, double beta, double u)
{
    return u < exp(-beta * (e_new - e_old));
}

/*
 * One update of the variables from g = (dE/dt, tau, dE/dtheta), step count ta >= 1 inside
 * the MC loop (the moments m, v restart with every loop).  Sec. 2 samples with Adam
 * (lr 0.1); Table S5 compares other optimisers.  Each rule is PyTorch's definition:
 *   Adam     m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 *            step = -(lr / (1 - b1^ta)) m / (sqrt(v) / sqrt(1 - b2^ta) + eps)
 *   AdamW    the Adam step plus the decoupled decay -lr wd p
 *   RMSprop  v = a v + (1-a) g^2; step = -lr g / (sqrt(v) + eps)
 *   Adagrad  v = v + g^2;         step = -lr g / (sqrt(v) + eps)
 *   SGD      m = mu m + g;        step = -lr m   (m = g on a loop's first step)
 * Reading for the values p a decay acts on: t - (centre of the pose's box), 0 for the
 * rotation vector (the tangent is re-centred at the current orientation every step),
 * and theta.  t is then clamped into the pose's box and theta wrapped to [-pi, pi).
 */
void or_opt_step(const or_sample_cfg* cfg, int T, int ta, uint32_t pose, const double* g, double* m, double* v,
                 double* dof)
{
    const double *lo = box_lo(cfg, pose), *hi = box_hi(cfg, pose);
    double bc1 = 1.0 - pow(cfg->b1, ta), bc2 = 1.0 - pow(cfg->b2, ta);
    double step[6 + OR_TMAX];
    for (int j = 0; j < 6 + T; ++j) {
        double pval = j < 3 ? dof[j] - 0.5 * (lo[j] + hi[j]) : (j < 6 ? 0.0 : dof[7 + (j - 6)]);
        switch (cfg->optimizer) {
        case OR_OPT_RMSPROP:
            v[j] = cfg->alpha * v[j] + (1.0 - cfg->alpha) * g[j] * g[j];
            step[j] = -cfg->lr * g[j] / (sqrt(v[j]) + cfg->eps);
            break;
        case OR_OPT_ADAGRAD:
            v[j] = v[j] + g[j] * g[j];
            step[j] = -cfg->lr * g[j] / (sqrt(v[j]) + cfg->eps);
            break;
        case OR_OPT_SGD:
            m[j] = cfg->momentum * m[j] + g[j];
            step[j] = -cfg->lr * m[j];
            break;
        default: {  /* Adam, AdamW */
            m[j] = cfg->b1 * m[j] + (1.0 - cfg->b1) * g[j];
            v[j] = cfg->b2 * v[j] + (1.0 - cfg->b2) * g[j] * g[j];
            double denom = sqrt(v[j]) / sqrt(bc2) + cfg->eps;
            step[j] = -(cfg->lr / bc1) * m[j] / denom;
            if (cfg->optimizer == OR_OPT_ADAMW) step[j] -= cfg->lr * cfg->weight_decay * pval;
        }
        }
    }
    for (int d = 0; d < 3; ++d) {
        double t = dof[d] + step[d];
        if (t < lo[d]) t = lo[d];
        if (t > hi[d]) t = hi[d];
        dof[d] = t;
    }
    double phi = sqrt(step[3] * step[3] + step[4] * step[4] + step[5] * step[5]);
    double r[4];
    if (phi > 0) {
        double s = sin(0.5 * phi) / phi;
        r[0] = cos(0.5 * phi); r[1] = s * step[3]; r[2] = s * step[4]; r[3] = s * step[5];
    } else {
        r[0] = 1; r[1] = r[2] = r[3] = 0;
    }
    qmul(r, dof + 3, dof + 3);
    qnormalize(dof + 3);
    for (int k = 0; k < T; ++k) dof[7 + k] = wrap_pi(dof[7 + k] + step[6 + k]);
}

/* Full FP64 trajectory of one pose; returns the final energy (NaN if a
 * non-finite energy froze the pose).  pairs (nullable) accumulates the number
 * of pairs inside the cutoff over all evaluations. */
double or_sample_pose(const or_sample_cfg* cfg, const or_params* p, int M, const double* pxyz,
                      const int32_t* ptype, const or_mdn* md, const or_maps* mp, const or_ligand* lg, uint32_t lig,
                      uint32_t pose, double* dof, int64_t* pairs)
{
    int T = lg->n_tor;
    double m[6 + OR_TMAX], v[6 + OR_TMAX], saved[7 + OR_TMAX], g[6 + OR_TMAX];
    double e_cur = NAN, e_saved = NAN;
    or_eval* ev = (or_eval*)malloc(sizeof(or_eval));
    or_init_pose(cfg, T, lig, pose, dof);
    for (int l = 0; l < cfg->mc_loops; ++l) {
        int n = or_loop_steps(cfg->steps, cfg->mc_loops, l);
        if (n == 0) continue;
        if (l > 0) {
            memcpy(saved, dof, sizeof(double) * (7 + T));
            e_saved = e_cur;
            or_perturb(cfg, T, lig, pose, (uint32_t)l, dof);
        }
        memset(m, 0, sizeof m);
        memset(v, 0, sizeof v);
        for (int j = 0; j < n; ++j) {
            int st = or_score_full(p, M, pxyz, ptype, md, mp, lg, dof, ev);
            if (pairs) *pairs += ev->n_inter + ev->n_intra;
            if (st != OR_OK) { free(ev); return NAN; }
            if (j < n - 1) {
                for (int d = 0; d < 3; ++d) { g[d] = ev->g_dof[d]; g[3 + d] = ev->tau[d]; }
                for (int k = 0; k < T; ++k) g[6 + k] = ev->g_dof[7 + k];
                or_opt_step(cfg, T, j + 1, pose, g, m, v, dof);
            } else {
                e_cur = ev->e_total;
            }
        }
        if (l > 0) {
            double u = or_metropolis_u(cfg->seed, lig, pose, (uint32_t)l);
            if (!or_metropolis_accept(e_cur, e_saved, cfg->beta, u)) {
                memcpy(dof, saved, sizeof(double) * (7 + T));
                e_cur = e_saved;
            }
        }
    }
    free(ev);
    return e_cur;
}

typedef struct {
    const or_sample_cfg* cfg; const or_params* p; int M; const double* pxyz; const int32_t* ptype;
    const or_mdn* md; const or_maps* mp; const or_ligand* lg; uint32_t lig; int pose0, pose1, dstride; double* dof; double* e; int64_t pairs;
} or_job;

static void* or_worker(void* arg)
{
    or_job* j = (or_job*)arg;
    for (int ps = j->pose0; ps < j->pose1; ++ps)
        j->e[ps] = or_sample_pose(j->cfg, j->p, j->M, j->pxyz, j->ptype, j->md, j->mp, j->lg, j->lig, (uint32_t)ps,
                                  j->dof + (size_t)ps * j->dstride, &j->pairs);
    return NULL;
}

/* Poses [0, P) of one ligand on n_threads POSIX threads (contiguous chunks).
 * dof: [P][dstride], e: [P].  Returns the number of in-cutoff pairs evaluated. */
int64_t or_sample_ligand(const or_sample_cfg* cfg, const or_params* p, int M, const double* pxyz,
                         const int32_t* ptype, const or_mdn* md, const or_maps* mp, const or_ligand* lg, uint32_t lig,
                         int P, int dstride,
                         double* dof, double* e, int n_threads)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > P) n_threads = P;
    or_job jobs[256];
    pthread_t th[256];
    if (n_threads > 256) n_threads = 256;
    for (int t = 0; t < n_threads; ++t) {
        or_job j = {cfg, p, M, pxyz, ptype, md, mp, lg, lig, (int)((int64_t)P * t / n_threads),
                    (int)((int64_t)P * (t + 1) / n_threads), dstride, dof, e, 0};
        jobs[t] = j;
        pthread_create(&th[t], NULL, or_worker, &jobs[t]);
    }
    int64_t pairs = 0;
    for (int t = 0; t < n_threads; ++t) { pthread_join(th[t], NULL); pairs += jobs[t].pairs; }
    return pairs;
}

/* ------------------------------------------------------------------------- */
/* Rank + cluster -> top N (Sec. 2, end of "Conformation sampling").  Reading: */
/* order by (energy ascending, pose index ascending); greedy dedupe skips a    */
/* pose whose heavy-atom RMSD (no symmetry) to a kept pose is below rho,       */
/* tested as sum d^2 < rho^2 L; non-finite energies are never kept; pad -1.    */
/* near counts decisions within 1e-4 A of rho.                                  */
/* ------------------------------------------------------------------------- */
static const double* g_sort_e;
static int cmp_pose(const void* a, const void* b)
{
    int i = *(const int*)a, j = *(const int*)b;
    double ei = g_sort_e[i], ej = g_sort_e[j];
    int fi = isfinite(ei), fj = isfinite(ej);
    if (fi != fj) return fi ? -1 : 1;
    if (fi && ei != ej) return ei < ej ? -1 : 1;
    return i < j ? -1 : (i > j);
}

void or_topk(int P, const double* E, const double* X, int L, int k, double rho,
             int32_t* idx, int32_t* near)
{
    int* ord = (int*)malloc(sizeof(int) * (size_t)P);
    for (int i = 0; i < P; ++i) ord[i] = i;
    g_sort_e = E;
    qsort(ord, (size_t)P, sizeof(int), cmp_pose);
    int nk = 0;
    *near = 0;
    for (int n = 0; n < P && nk < k; ++n) {
        int p = ord[n];
        if (!isfinite(E[p])) break;
        int dup = 0;
        for (int m = 0; m < nk && !dup; ++m) {
            const double* a = X + (size_t)p * L * 3;
            const double* b = X + (size_t)idx[m] * L * 3;
            double s = 0;
            for (int i = 0; i < 3 * L; ++i) s += (a[i] - b[i]) * (a[i] - b[i]);
            double rmsd = sqrt(s / L);
            if (fabs(rmsd - rho) < 1e-4) (*near)++;
            if (s < rho * rho * L) dup = 1;
        }
        if (!dup) idx[nk++] = p;
    }
    for (int m = nk; m < k; ++m) idx[m] = -1;
    free(ord);
}

/* E_screen (Sec. 2, virtual screening): the docking score divided by the torsion factor
 * 1 + w_tor N_tor, N_tor = the ligand's number of rotatable bonds in the sampling.
 * Reading: the docking score is the ligand-pocket energy E_inter (the paper's score has
 * no intra-ligand part; the intra energy the sampler adds is left out), as in Vina's
 * final rescaling of the intermolecular energy. */
double or_screen_energy(double e_inter, double w_tor, int n_tor)
{
    return e_inter / (1.0 + w_tor * (double)n_tor);
}

size_t or_sizeof_ligand(void) { return sizeof(or_ligand); }
size_t or_sizeof_eval(void) { return sizeof(or_eval); }
size_t or_sizeof_params(void) { return sizeof(or_params); }
