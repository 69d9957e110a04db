/*
 * trids.h -- C-ABI of libtrids: gradient-guided ligand pose sampling on one GPU
 * (the sampling hot path of TRIDS, arXiv 2510.24186), written for sm_103a.
 *
 * The problem, as the paper states it (Sec. 2 "Conformation sampling",
 * "Scoring functions", Fig. 2): a pocket of receptor atoms and a translation box;
 * ligands whose degrees of freedom are a translation in [box_min, box_max], a
 * rotation and the torsion angles of their rotatable bonds; a score that is a
 * weighted sum of pairwise-distance terms (E_dock, and E_screen = E_dock /
 * (1 + w_tor N_tor)); many copies per ligand refined by Adam on the score's
 * gradient inside Metropolis Monte-Carlo loops; the copies then ranked,
 * clustered and cut to the top N.
 *
 * Conventions
 *  - Every function returns an int status: TRIDS_OK (0) or a negative code.
 *    trids_last_error() returns a message for the calling thread's last failure.
 *  - Handles (trids_pocket, trids_batch) are owned by the library and freed with
 *    trids_free_pocket / trids_free_batch.  Array arguments are owned by the caller.
 *  - Host pointers are used only by pocket/batch construction and topology
 *    queries.  The hot calls (trids_score_grad, trids_sample, trids_topk) take
 *    DEVICE pointers (contiguous float32/int32, on the device that was current
 *    when the pocket was made) and a cudaStream_t passed as void* (NULL = the
 *    legacy default stream).  They are asynchronous on that stream: argument
 *    errors are reported synchronously; per-pose numerical failures are recorded
 *    in the per-pose status words and returned by trids_sync as TRIDS_ENONFINITE.
 *  - A batch and a pocket must not be used from two host threads at once.
 *  - All device arithmetic is float32; counts and indices are int32.
 */
#ifndef TRIDS_H
#define TRIDS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TRIDS_OK 0
#define TRIDS_EINVAL (-1)     /* bad argument or invalid molecule */
#define TRIDS_ENOMEM (-2)     /* host or device allocation failed */
#define TRIDS_ECUDA (-3)      /* a CUDA runtime call failed */
#define TRIDS_ETIMEOUT (-4)   /* trids_sync gave up waiting */
#define TRIDS_ENONFINITE (-5) /* a pose produced a non-finite energy */

#define TRIDS_MAX_TYPES 16
#define TRIDS_MAX_GMM 4
#define TRIDS_MAX_ATOMS 70    /* heavy atoms per ligand */
#define TRIDS_MAX_TOR 20      /* rotatable bonds per ligand */
#define TRIDS_MAX_BOXES 8     /* docking boxes per pocket */

#define TRIDS_TERMS_VINA5 0
#define TRIDS_TERMS_TRIDS 1
#define TRIDS_TERMS_TRIDS_RES 2

#define TRIDS_MAX_MDN_K 16    /* Gaussian kernels per (ligand atom, residue) pair */
#define TRIDS_MAX_RESIDUES 8191

/* Update rules of the refinement steps (Sec. 2 samples with Adam; Table S5 compares
 * the others).  Each is PyTorch's definition on g = (dE/dt, torque, dE/dtheta):
 *   ADAM     m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 *            step = -(lr / (1 - b1^k)) m / (sqrt(v) / sqrt(1 - b2^k) + eps), k = step in loop
 *   ADAMW    the Adam step - lr weight_decay p
 *   RMSPROP  v = alpha v + (1-alpha) g^2; step = -lr g / (sqrt(v) + eps)
 *   ADAGRAD  v = v + g^2; step = -lr g / (sqrt(v) + eps)
 *   SGD      m = momentum m + g; step = -lr m
 * m and v restart at every Monte-Carlo loop.  The values p a decay acts on: t minus the
 * centre of the pose's box, 0 for the rotation vector (the tangent is re-centred at the
 * current orientation every step), theta. */
#define TRIDS_OPT_ADAM 0
#define TRIDS_OPT_ADAMW 1
#define TRIDS_OPT_RMSPROP 2
#define TRIDS_OPT_ADAGRAD 3
#define TRIDS_OPT_SGD 4

/* Phases of one evaluation timed by trids_sample_cfg.phase_cycles (counting runs only). */
#define TRIDS_PHASE_FK 0        /* forward kinematics */
#define TRIDS_PHASE_PAIRS 1     /* pair loop: per-atom candidate set-up, pair sums, lane-order combine */
#define TRIDS_PHASE_PASSES 2    /* grid-map, atom-pair E_MDN and residue E_MDN passes */
#define TRIDS_PHASE_ADJOINT 3   /* forces -> dE/dt, torque, dE/dtheta */
#define TRIDS_PHASE_UPDATE 4    /* update rule, Monte-Carlo save/perturb/accept, trace records */
#define TRIDS_PHASE_OTHER 5     /* taking a pose, initial or resumed state, storing it */
#define TRIDS_PHASES 6

/* Work counted by trids_sample_cfg.work_count (counting runs only), beyond the in-cutoff
 * pairs of pair_count; the algorithmic FLOPs of an evaluation follow from them. */
#define TRIDS_WORK_CLASH 0      /* in-cutoff pairs inside the E_clash range (TRIDS terms) */
#define TRIDS_WORK_HBOND 1      /* donor-acceptor pairs inside the E_Hbond range (TRIDS terms) */
#define TRIDS_WORK_MDN_PAIRS 2  /* atom-pair E_MDN pairs inside 5 A (term set 1) */
#define TRIDS_WORK_RES_SCAN 3   /* residue atoms scanned for the residue minima (term set 2) */
#define TRIDS_WORK_RES_PAIRS 4  /* (ligand atom, residue) pairs inside 5 A (term set 2) */
#define TRIDS_WORK_COUNTS 5

#define TRIDS_MODE_PERSISTENT 0 /* one persistent fused launch (optionally a CUDA graph) */
#define TRIDS_MODE_PER_LIGAND 1 /* plain form: one launch per (ligand, step) */

/*
 * Scoring parameters.  Every term depends only on pair distances (Sec. 2
 * "Scoring functions": "all of these terms are calculated based on pairwise
 * distances"), so they are the same for ligand-pocket and intra-ligand pairs
 * except E_MDN, which is ligand-pocket only.  A pair contributes only if its
 * centre distance r < cutoff.
 *
 * term_set TRIDS_TERMS_VINA5 (the analytic terms the DSDP line samples with; the
 *   paper's E_long is "the second Gaussian term in VINA"): with surface distance
 *   d = r - R_a - R_b and weights w[0..4]:
 *     w0 exp(-(d/0.5)^2) + w1 exp(-((d-3)/2)^2) + w2 [d<0] d^2
 *     + w3 [both hydrophobic] (1 if d<0.5; 1.5-d if d<1.5; else 0)
 *     + w4 [donor-acceptor] (1 if d<-0.7; -d/0.7 if d<0; else 0).
 * term_set TRIDS_TERMS_TRIDS (Sec. 2 Eqs. P(d), E_MDN, E_long, E_clash, E_Hbond,
 *   E_dock; default w = 1.0, 0.2, 10.0, 0.6):
 *     w0 E_MDN:  -sum_k pi_k exp(-(r-mu_k)^2/(2 sigma_k^2)), r < 5, ligand-pocket only,
 *                (pi, mu, sigma) = gmm[type_lig][type_pocket][k] (the paper's network
 *                predicts them; here they are inputs);
 *     w1 E_long: -exp(-(r - R_a - R_b - 3)^2 / 4), r < 10;
 *     w2 E_clash: -ln(max(r,0.5)/d_clash), r < d_clash, d_clash = 2.6 for a donor-acceptor
 *                pair, else R_a + R_b;
 *     w3 E_Hbond: -exp(-(r-2.88)^2/(2*0.3^2)), donor-acceptor pairs, r < 3.4.
 * term_set TRIDS_TERMS_TRIDS_RES: E_MDN at residue level, the form Sec. 2 defines
 *   (d_ij in Eq. P(d) is the minimum distance between residue i's atoms and ligand
 *   atom j):
 *     w0 E_MDN:  -sum_r sum_j [d_rj < 5] sum_k pi_k exp(-(d_rj - mu_k)^2/(2 sigma_k^2)),
 *                d_rj = min over the atoms a of residue r of |x_j - x_a|; the force acts
 *                along the nearest atom (equal distances: the lowest pocket-atom index);
 *                (pi, mu, sigma) per (ligand atom, residue, k) from trids_set_mdn; the
 *                5 A cutoff is the paper's and does not depend on `cutoff`;
 *     w1..w3:    E_long, E_clash, E_Hbond over atom pairs, as for TRIDS_TERMS_TRIDS
 *                (gmm unused).
 *   Needs trids_set_residues on the pocket (built with cutoff >= 5) and trids_set_mdn
 *   on the batch; score and sample calls fail with TRIDS_EINVAL without them.
 * flags[type]: bit0 hydrophobic, bit1 donor, bit2 acceptor.  A donor-acceptor pair
 * is donor on one side and acceptor on the other, either way round.
 */
typedef struct trids_params {
    int32_t term_set;
    int32_t n_types;                 /* 1..TRIDS_MAX_TYPES */
    float w[5];
    float radius[TRIDS_MAX_TYPES];   /* van der Waals radius per type (A) */
    uint8_t flags[TRIDS_MAX_TYPES];
    float cutoff;                    /* pair cutoff on r (A), > 0 */
    float w_tor;                     /* E_screen weight (0.01 in the paper) */
    int32_t gmm_k;                   /* kernels per type pair, 0..TRIDS_MAX_GMM */
    float gmm[TRIDS_MAX_TYPES][TRIDS_MAX_TYPES][TRIDS_MAX_GMM][3]; /* (pi, mu, sigma) */
} trids_params;

typedef struct trids_pocket trids_pocket;
typedef struct trids_batch trids_batch;

typedef struct trids_batch_dims {
    int32_t n_lig;
    int32_t max_atoms;    /* L_max over the batch */
    int32_t max_tor;      /* T_max over the batch */
    int32_t dof_stride;   /* 7 + max_tor: floats per pose row of a DOF array */
    int32_t state_fields; /* floats per pose of the sampler state buffer */
    int64_t n_intra;      /* intra-ligand pairs over the batch */
    int64_t upload_bytes; /* host-to-device bytes trids_pack_ligands copied for the batch */
} trids_batch_dims;

/* Sampler configuration (Sec. 2 "Conformation sampling", Fig. 2). */
typedef struct trids_sample_cfg {
    int32_t poses;           /* copies per ligand (1,024 in the paper) */
    int32_t steps;           /* S: score+gradient evaluations of the whole schedule */
    int32_t step_begin;      /* run evaluations [step_begin, step_end) of the schedule; */
    int32_t step_end;        /*   step_begin > 0 resumes from dof + state */
    int32_t mc_loops;        /* Monte-Carlo loops (8 in the paper) */
    float lr, beta1, beta2, eps; /* update rule (Adam: lr 0.1 in the paper; torch defaults otherwise) */
    float beta;              /* Metropolis beta (0.069 in the paper) */
    uint64_t seed;           /* Philox4x32-10 key */
    int32_t lig_base;        /* random-stream id of ligand 0 of this batch */
    int32_t mode;            /* TRIDS_MODE_* */
    int32_t warps_per_block; /* poses (warps) per block: 1..28 for the plain Vina-form sampler (Adam,
                              * direct pair sums), 1..24 otherwise (larger values are capped); 0 = the
                              * maximum; fewer if the pocket needs the shared memory */
    int32_t use_graph;       /* persistent mode: launch through the pocket's CUDA graph (counter reset +
                              * persistent kernel), built once per launch shape and replayed; other
                              * arguments update its nodes (see trids_graph_stats) */
    float* trace;            /* nullable device buffer, see trids_sample */
    const int32_t* trace_slot; /* device [n_lig*poses]: trace slot of each pose or -1 */
    int32_t n_trace;         /* number of trace slots */
    unsigned long long* pair_count; /* nullable device counter: adds in-cutoff pairs evaluated */
    int32_t optimizer;       /* TRIDS_OPT_*; 0 = Adam, the paper's */
    float weight_decay;      /* AdamW decay (torch default 0.01), >= 0 */
    float momentum;          /* SGD momentum in [0, 1) (torch default 0) */
    float alpha;             /* RMSprop smoothing in [0, 1) (torch default 0.99) */
    unsigned long long* phase_cycles; /* nullable device [TRIDS_PHASES]: adds the SM clock cycles each
                                       * warp spent in each phase (TRIDS_PHASE_*).  Like pair_count it
                                       * selects the counting form of the sampler, which follows the
                                       * same trajectories; the sums give each phase's share of the
                                       * warps' time */
    unsigned long long* work_count;   /* nullable device [TRIDS_WORK_COUNTS]: adds the work counts
                                       * TRIDS_WORK_* (selects the counting form, like pair_count) */
} trids_sample_cfg;

/* Message of the calling thread's last failure ("" if none). */
const char* trids_last_error(void);

/* Library version (major*10000 + minor*100 + patch). */
int trids_version(void);

/*
 * trids_make_pocket -- build the pocket and translation box (Sec. 2: pocket of
 * receptor atoms near the reference ligand; translation range [box_min, box_max]
 * with box_min = center - size/2 and box_max = center + size/2).
 *   xyz   host [n_atoms][3] float32 coordinates (A), type host [n_atoms] int32 in
 *         [0, prm->n_types); n_atoms in [1, 8191].
 *   cell  edge (A) of the candidate grid used to cull ligand-pocket pairs; 0 selects
 *         0.5 A.  The grid changes which pairs outside the cutoff are tested (they add
 *         exact zeros) and the order of the pair sums, so only the last bits of a result.
 *   prm   scoring parameters, copied.
 * The pocket's device arrays live on the current CUDA device.  Errors: TRIDS_EINVAL
 * (bad sizes, non-finite values, types out of range), TRIDS_ENOMEM, TRIDS_ECUDA.
 */
int trids_make_pocket(const float* xyz, const int32_t* type, int32_t n_atoms,
                      const float box_center[3], const float box_size[3], float cell,
                      const trids_params* prm, trids_pocket** out);

/* Replace the scoring parameters (weights, radii, flags, GMM).  The cutoff may not
 * exceed the one the pocket was built with.  Stream-ordered on `stream`. */
int trids_set_params(trids_pocket* pk, const trids_params* prm, void* stream);

/*
 * Several docking boxes, e.g. one per candidate cavity of a receptor region (the paper
 * defines one box per task, Sec. 2 "Conformation sampling"; several boxes let one call
 * sample several cavities).  Pose p samples, is perturbed and is clamped in box
 * p mod n_boxes.  centers, sizes: host [n_boxes][3]; 1 <= n_boxes <= TRIDS_MAX_BOXES.
 * Takes effect for launches issued after the call.
 */
int trids_set_boxes(trids_pocket* pk, int32_t n_boxes, const float* centers, const float* sizes);

/* Free a pocket, its device arrays (maps, residue lists included) and its sampler CUDA
 * graph.  NULL is a no-op;
 * the caller must not free a pocket while work that uses it is in flight. */
int trids_free_pocket(trids_pocket* pk);

/*
 * Residues of the pocket for the residue-level E_MDN (term set TRIDS_TERMS_TRIDS_RES;
 * Sec. 2: the MDN scores atom-residue pairs by their minimum distance).
 *   residue  host [n_atoms] int32, residue index of each pocket atom in [0, n_res);
 *            a residue may hold any atoms, in any order, or none.
 *   n_res    1..TRIDS_MAX_RESIDUES.
 * Builds, per cell of the pocket's candidate grid, the list of residues with an atom
 * within 5 A of the cell (plus half its diagonal).  Replaces earlier residues.  The
 * pocket must have been built with cutoff >= 5.  Errors: TRIDS_EINVAL, TRIDS_ENOMEM,
 * TRIDS_ECUDA.  Synchronous.
 */
int trids_set_residues(trids_pocket* pk, int32_t n_res, const int32_t* residue);

/*
 * Grid maps of the ligand-pocket atom-pair terms (the DSDP / Vina practice; the paper
 * itself sums pairs directly, Sec. 4 item 4): for every ligand type, the energy an atom
 * of that type would have at each point lo + spacing * (x, y, z) of a regular grid,
 * summed over the pocket atoms within the cutoff.  While maps are present, a ligand atom
 * whose cell (all 8 corners) lies inside the grid takes the trilinear interpolation of
 * its type's map and the analytic gradient of that interpolation; any other atom keeps
 * the direct pair sum.  Intra-ligand pairs and the residue-level E_MDN stay direct.
 *   spacing  grid spacing (A) in [0.05, 4] (Vina uses 0.375); 0 frees the maps.
 *   margin   the grid spans the union of the docking boxes grown by margin (A) per side,
 *            in [0, 64].
 * Memory: n_types * (points per axis)^3 floats.  The maps hold the parameters of the
 * build: after trids_set_params, scoring and sampling fail with TRIDS_EINVAL until the
 * maps are rebuilt; parameter gradients (g_w, g_radius) are refused while maps are
 * present.  Launches on `stream`; later launches on that stream see the maps.
 */
int trids_build_maps(trids_pocket* pk, float spacing, float margin, void* stream);

/* Map grid in use: origin lo (A), spacing (A) and points per axis (all 0 without maps). */
int trids_maps_info(const trids_pocket* pk, float lo[3], float* spacing, int32_t dims[3]);

/*
 * trids_pack_ligands -- validate ligands, build their torsion trees and upload them.
 * Inputs are host arrays, concatenated over ligands: n_atoms[n_lig]; xyz[sum L][3]
 * float32 input geometry (theta = 0); type[sum L]; n_bonds[n_lig];
 * bonds[sum nb][2] ligand-local atom indices; rotatable[sum nb] (0/1).
 * Degrees of freedom (Sec. 2): translation t, rotation quaternion q = (w,x,y,z),
 * one torsion angle per rotatable bond.  World coordinates are
 * x_i = t + R(q/|q|) z_i, z = input geometry about the root-fragment centroid after
 * the torsions; torsion k turns the subtree on its child side by theta_k about the
 * bond from its parent atom toward its child atom (right-hand rule).
 * Tree rules (the paper is silent): fragments = components after cutting rotatable
 * bonds; root = fragment of minimum tree height (ties: smallest input atom index);
 * torsions in BFS order from the root, children by smallest input atom index; atoms
 * renumbered in DFS pre-order of fragments so each moving subtree is contiguous;
 * intra-ligand pairs = atoms in different fragments and >= 4 bonds apart.
 * Errors: TRIDS_EINVAL for L outside [1, 70], more than 20 rotatable bonds, a
 * disconnected ligand, a rotatable bond inside a ring, duplicate or self bonds,
 * non-finite coordinates or types out of range (the message names the ligand).
 */
int trids_pack_ligands(const trids_pocket* pk, int32_t n_lig, const int32_t* n_atoms,
                       const float* xyz, const int32_t* type, const int32_t* n_bonds,
                       const int32_t* bonds, const uint8_t* rotatable, trids_batch** out);

/* Free a batch, its device arrays and work lists.  NULL is a no-op; the caller must not
 * free a batch while work that uses it is in flight.  The call waits for the work of the
 * last library call that used the batch (on that call's stream) and keeps the batch's main
 * device block for the next trids_pack_ligands on that device (at most two blocks per
 * device stay pooled, until the process exits), so a stream of batches allocates its device
 * memory once instead of once per batch. */
int trids_free_batch(trids_batch* b);

/*
 * Per-pair Gaussian kernels of the residue-level E_MDN (the quantities the paper's
 * network predicts for each ligand atom / residue pair, Sec. 2 Eq. P(d)).
 *   mdn    DEVICE float32 [n_atoms_total][n_res][K][3] of (pi, mu, sigma), rows in the
 *          input atom order of trids_pack_ligands (ligand 0's atoms first); sigma > 0.
 *   n_res  must equal the pocket's residue count when scoring; K in 1..TRIDS_MAX_MDN_K.
 * The library keeps its own copy (rows reordered to the packed atom order), so `mdn`
 * may be freed after the call.  Runs on `stream` and synchronises it.  Errors:
 * TRIDS_EINVAL (sizes, host pointer, non-finite values or sigma <= 0), TRIDS_ENOMEM,
 * TRIDS_ECUDA.
 */
int trids_set_mdn(trids_batch* b, int32_t n_res, int32_t K, const float* mdn, void* stream);

/*
 * Random-stream ids of the batch's ligands (host int32 [n_lig], each >= 0): ligand l then
 * draws its random numbers as ligand lig_base + ids[l] (trids_sample), instead of
 * lig_base + l.  A ligand's samples depend only on its stream id, the seed and the
 * pocket, not on which batch holds it, so a ligand set split into shards (one per GPU,
 * say) and sampled with each ligand's global index as its id gives the same results as
 * the whole set in one batch.  Synchronous.  Errors: TRIDS_EINVAL (NULL, negative id),
 * TRIDS_ECUDA.
 */
int trids_set_stream_ids(trids_batch* b, const int32_t* ids);

/* Sizes of a packed batch (trids_batch_dims above), written to the host struct `dims`.
 * TRIDS_EINVAL for NULL arguments. */
int trids_batch_info(const trids_batch* b, trids_batch_dims* dims);

/*
 * Per-ligand sizes (host arrays, nullable): n_tor[n_lig], n_atoms[n_lig].  If topo is
 * non-null, the packed topology of ligand `lig` is written as int32
 * [L, T, n_pairs, perm[L] (packed -> input index), frag[L] (0 root, k+1 = moving
 * fragment of torsion k), T x (parent atom, child atom, parent torsion or -1,
 * subtree begin, subtree end), n_pairs x (i, j)] in packed indices; returns
 * TRIDS_EINVAL if topo_cap is too small.
 */
int trids_batch_query(const trids_batch* b, int32_t* n_tor, int32_t* n_atoms,
                      int32_t lig, int32_t* topo, int32_t topo_cap);

/* Host-only packing of one ligand (same rules and layout as trids_batch_query);
 * needs no GPU.  *topo_len receives the number of int32 written. */
int trids_pack_topology(int32_t n_atoms, const float* xyz, const int32_t* type, int32_t n_types,
                        int32_t n_bonds, const int32_t* bonds, const uint8_t* rotatable,
                        int32_t* topo, int32_t topo_cap, int32_t* topo_len);

/*
 * trids_score_grad -- score and analytic gradient of given poses (Sec. 2: the score
 * is differentiable in the ligand coordinates; Sec. 4 item 3: manual differentiation
 * of the Gaussian terms and of the DOF-to-coordinate map).  Kinematics are
 * recomputed, nothing per atom is stored between calls.
 *   dof      device [n_lig][poses][dof_stride]: t(3), q(4), theta(T), padding ignored.
 *   energy   device [n_lig][poses] out: E_total = ligand-pocket + intra-ligand.
 *   e_inter  nullable device [n_lig][poses] out: the ligand-pocket part.
 *   g_dof    nullable device, layout of dof, out: dE/dt, dE/dq (gradient of E(q/|q|)),
 *            dE/dtheta; padding written 0.
 *   g_xyz    nullable device [n_lig][poses][max_atoms][3] out: dE/dx_i of world
 *            coordinates in INPUT atom order, rows past L zero.
 *   e_bar    nullable device [n_lig][poses]: upstream weights; when given, g_dof and
 *            g_xyz are multiplied by e_bar and g_w, g_radius are sum e_bar dE/d(.)
 *            (the backward of a sum-reduced autograd node).
 *   g_w      nullable device [5] out: dE/dw_t summed over all poses.
 *   g_radius nullable device [n_types] out: dE/dR_a summed over all poses.
 * Parameter sums are reduced in a fixed order (bit-reproducible run to run).
 */
int trids_score_grad(const trids_pocket* pk, const trids_batch* b, int32_t poses,
                     const float* dof, float* energy, float* e_inter, float* g_dof,
                     float* g_xyz, const float* e_bar, float* g_w, float* g_radius,
                     void* stream);

/*
 * trids_score_grad_noalloc -- the same energies and gradients as trids_score_grad, but
 * the call allocates nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 * The paper has no counterpart; this entry point exists for callers that cannot let a
 * library allocate device memory in the middle of their work: programs that hand out
 * all device memory from their own pool or a fixed arena reserved at start-up (a
 * library allocation would escape their accounting or fail once the arena holds the
 * whole device), and latency-sensitive loops that cannot afford the device-wide
 * synchronisation an allocation can cause.  (trids_score_grad allocates its work list and
 * its parameter-gradient partials on first use of a pose count.)
 *   Arguments, layouts and results are those of trids_score_grad; the caller still owns
 *   and passes every input and output buffer.  Parameter sums are reduced in a fixed
 *   order, which differs from trids_score_grad's, so g_w and g_radius agree with it to
 *   rounding, not bit for bit.
 *   Scratch: a 1 MiB array compiled into the library, one per device that loads it, held
 *   until the process exits.  It holds 256 bytes of work counter, 8 bytes per work item
 *   (one item = one ligand x 32 poses) and, when g_w or g_radius is requested, 84 more
 *   bytes per item.  Larger requests fail with TRIDS_EINVAL and a message giving the
 *   bytes needed; split the batch or use trids_score_grad.
 *   The first call on a device looks up the array's device address (set-up done once per
 *   device, with that device current, and again after the device's context has been
 *   reset); make that first call before any stream capture begins.  Every call reuses the same
 *   array (it keeps the previous call's contents; each call resets what must start at
 *   zero), so calls that can overlap on the GPU -- on two streams, or from two host
 *   threads -- race with each other and must be serialised by the caller.
 */
int trids_score_grad_noalloc(const trids_pocket* pk, const trids_batch* b, int32_t poses,
                             const float* dof, float* energy, float* e_inter, float* g_dof,
                             float* g_xyz, const float* e_bar, float* g_w, float* g_radius,
                             void* stream);

/* Floats of sampler state per batch: n_lig * poses * dims.state_fields. */
int64_t trids_state_floats(const trids_batch* b, int32_t poses);

/*
 * trids_sample -- Metropolis Monte Carlo with Adam refinement (Sec. 2, Fig. 2).
 *   Each pose starts from random DOFs (t uniform in the box, q uniform on SO(3) by
 *   Shoemake's method, theta uniform in [-pi, pi)).  Loop l (of mc_loops) gets
 *   floor(S/mc_loops) evaluations, one more for the first S mod mc_loops loops.  At
 *   the start of every loop after the first, one of the 6+T scalar variables, drawn
 *   uniformly, is resampled in its range (t_c in the box; a rotation by U[-pi,pi)
 *   about world axis c; theta_k in [-pi,pi)) and the Adam moments are reset.  Every
 *   evaluation but the last of a loop is followed by an Adam step (lr, beta1, beta2,
 *   eps; PyTorch form) on t, the world rotation vector (q <- exp(dw/2) (x) q) and
 *   theta; t is clamped to the box and theta wrapped to [-pi, pi).  The last
 *   evaluation of a loop gives its energy; the loop is accepted if
 *   u < exp(-beta (E_new - E_old)), else the state from before its perturbation is
 *   restored.  Random numbers: Philox4x32-10, key = seed, counter = (pose, lig_base +
 *   ligand, loop<<16 | purpose<<8 | block, 0), purpose 0 init, 1 perturbation,
 *   2 acceptance; uniform = (word >> 8) * 2^-24.  (lig_base + ligand is lig_base + the
 *   ligand's stream id when trids_set_stream_ids set one.)
 *   dof     device [n_lig][poses][dof_stride], out (in as well when step_begin > 0).
 *   state   device [trids_state_floats] scratch: Adam moments, saved state, loop
 *           energies, per-pose status.  Keep it between calls to resume.
 *   energy  device [n_lig][poses] out: energy of the returned state (valid once
 *           step_end reaches a loop end).
 *   trace   if non-null, each traced pose writes one record per evaluation at
 *           trace[((s - step_begin) * n_trace + slot) * (2*max_tor + 14)]:
 *           state before the evaluation (dof_stride floats), E, dE/dt (3), world
 *           torque (3), dE/dtheta (max_tor).
 * A pose whose energy is not finite is frozen and flagged; trids_sync reports it.
 */
int trids_sample(const trids_pocket* pk, const trids_batch* b, const trids_sample_cfg* cfg,
                 float* dof, float* state, float* energy, void* stream);

/*
 * Counters of the pocket's CUDA graph of the persistent sampler (Sec. 4 item 2: the
 * repeated operators are compiled once as a graph and kept on the GPU): how many times
 * it was built (once per launch shape: kernel, grid, block, shared memory), how many
 * calls updated its nodes in place (a new seed, ligand ids, step range, buffers or a
 * batch of the same shape), and how many times it was launched.  Host pointers,
 * nullable.  TRIDS_EINVAL for a NULL pocket.
 */
int trids_graph_stats(const trids_pocket* pk, int64_t* instantiations, int64_t* updates, int64_t* launches);

/*
 * trids_topk -- rank and cluster (Sec. 2, end of "Conformation sampling"): per ligand,
 * poses ordered by (energy ascending, pose index ascending); a pose is skipped when
 * its heavy-atom RMSD (no symmetry) to an already kept pose is below rmsd (0 disables);
 * the first k kept are written.  Non-finite energies are never kept.
 *   idx device [n_lig][k] int32 out (pose index or -1), e_out nullable [n_lig][k].
 */
int trids_topk(const trids_batch* b, int32_t poses, const float* energy, const float* dof,
               int32_t k, float rmsd, int32_t* idx, float* e_out, void* stream);

/*
 * trids_screen_energy -- the virtual-screening score of the kept poses (Sec. 2, the
 * E_screen equation): E_screen = E_dock / (1 + w_tor * N_tor), with N_tor the ligand's
 * realised number of torsions and w_tor the pocket's parameter (0.01 in the paper).
 * Reading: E_dock is the ligand-pocket energy E_inter (the paper's score has no
 * intra-ligand part), i.e. trids_score_grad's e_inter.  E_screen only rescales each
 * ligand's energies, so it does not change the top-k order.
 *   idx      device [n_lig][k] int32 in: pose indices as written by trids_topk (-1 = empty).
 *   e_inter  device [n_lig][poses] float in.
 *   e_screen device [n_lig][k] float out: one correctly rounded FP32 division per slot;
 *            NaN where idx is -1 (or any index outside [0, poses)).
 * Errors: TRIDS_EINVAL for NULL handles or pointers, poses < 1, k < 1, or a pocket and
 * batch on different devices; asynchronous on `stream`.
 */
int trids_screen_energy(const trids_pocket* pk, const trids_batch* b, int32_t poses, int32_t k,
                        const int32_t* idx, const float* e_inter, float* e_screen, void* stream);

/*
 * Wait for `stream` (polling, at most timeout_ms; <= 0 waits without limit), then
 * check the per-pose status words of `state` (nullable): TRIDS_OK, TRIDS_ETIMEOUT,
 * TRIDS_ECUDA or TRIDS_ENONFINITE.
 */
int trids_sync(const trids_batch* b, int32_t poses, const float* state, void* stream,
               double timeout_ms);

#ifdef __cplusplus
}
#endif
#endif /* TRIDS_H */
