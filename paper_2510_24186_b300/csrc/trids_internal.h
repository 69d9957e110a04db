// Internal structures of libtrids shared by its host and device translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <vector_types.h>

#include "trids.h"

#ifdef __CUDACC__
#define TRIDS_HD __host__ __device__
#else
#define TRIDS_HD
#endif

namespace trids {

constexpr int kLmax = TRIDS_MAX_ATOMS;
constexpr int kTmax = TRIDS_MAX_TOR;
constexpr int kNT = TRIDS_MAX_TYPES;
constexpr float kLog2e = 1.4426950408889634f;   // log2(e): exp(x) = 2^(x log2 e)
constexpr int kK = TRIDS_MAX_GMM;
// Row stride of the staged GMM table (float4 per (ligand type, pocket type) row) and the row
// count per ligand type, both padded by one: the 16-byte shared-memory bank group of kernel k
// of row (a, b) is then (5 (a + b) + k) mod 8 instead of (4 b + k) mod 8, so lanes reading
// rows of different types rarely collide in a bank group.
constexpr int kKP = kK + 1;
constexpr int kNTP = kNT + 1;
constexpr int kMaxBoxes = TRIDS_MAX_BOXES;
static_assert(kTmax <= 32, "per-atom torsion masks are 32-bit");

// ---------------------------------------------------------------- host-side pack
// Packed torsion tree of one ligand (rules in trids.h, trids_pack_ligands).
struct PackedLigand {
    int n_atoms = 0, n_tor = 0;
    std::vector<int> perm;          // packed -> input index
    std::vector<int> frag;          // packed atom -> 0 (root) or k+1
    std::vector<int> tp, th, tpar, sb, se;
    std::vector<std::pair<int, int>> pairs;  // intra pairs, packed indices, i < j
    double c[3] = {0, 0, 0};        // root-fragment centroid (input frame)
};

// Returns "" on success, else a message.  xyz: [n][3].
std::string pack_ligand(int n, const float* xyz, const int32_t* type, int n_types, int nb,
                        const int32_t* bonds, const uint8_t* rot, PackedLigand* out);
void topology_ints(const PackedLigand& lg, std::vector<int32_t>* out);

// ---------------------------------------------------------------- candidate grid
// Uniform grid over the pocket's bounding box grown by the cutoff.  Each cell lists
// every pocket atom within cutoff + half the cell diagonal (+ a small margin) of the
// cell centre, padded to a multiple of 8 with the sentinel index M.  A ligand atom
// outside the grid has no pocket atom within the cutoff.  The entries of a cell are
// ordered by reach level: level k holds the atoms within cutoff + (k + 1) / kReachLevels
// of the half diagonal (+ the margin) of the centre and not in a lower level (ascending
// atom index inside a level); levels[cell][k] is the number of 8-entry blocks that
// covers levels 0..k, so a point at distance delta <= (k + 1) / kReachLevels of the half
// diagonal from its cell centre needs only those blocks.  The device copy carries each
// atom's flags in the top 3 bits of its entry (so M < 8192).
constexpr int kReachLevels = 8;
struct CandidateGrid {
    float lo[3];
    float h;
    int dims[3];
    std::vector<uint32_t> start;    // [ncell + 1], offsets in entries (multiples of 8)
    std::vector<uint16_t> cand;
    std::vector<uint16_t> levels;   // [ncell][kReachLevels] block counts
};
void build_grid(int M, const float* xyz, float cutoff, float h, CandidateGrid* g);

// Residue lists of the residue-level E_MDN.  Atoms are grouped by residue (ascending
// atom index inside a residue, so the first minimum met is the lowest index; the library
// stores the pocket in that order once residues are set).  On the candidate grid's cells,
// each cell lists every residue with an atom within kMdnCut + half the cell diagonal (+ a
// small margin) of the cell centre, ordered by the reach level of the residue's nearest
// atom (as for the candidate lists; ascending residue inside a level); levels[cell][k]
// counts the residues of levels 0..k.
constexpr float kMdnCut = 5.0f;   // Sec. 2: node pairs closer than d_cutoff = 5 A
constexpr int kMaxResidueAtoms = 63;
struct ResidueGrid {
    int n_res = 0;
    std::vector<int32_t> start;        // [n_res + 1] offsets into atoms
    std::vector<uint16_t> atoms;       // pocket atom indices grouped by residue
    std::vector<uint32_t> cell_start;  // [ncell + 1]
    std::vector<uint32_t> list;        // residue r | first atom << 13 | atom count << 26
    std::vector<uint16_t> levels;      // [ncell][kReachLevels]
};
void build_residue_grid(int M, const float* xyz, const int32_t* res, int n_res, const CandidateGrid& g,
                        ResidueGrid* out);

// Near lists of the atom-pair E_MDN (term set 1, r < 5 A): on the candidate grid's cells,
// each cell lists the pocket atoms within `cutoff` + half the cell diagonal (+ a small
// margin) of the cell centre, ordered by reach level (ascending atom index inside a level);
// levels[cell][k] counts the atoms of levels 0..k.  No padding.
void build_near_lists(int M, const float* xyz, float cutoff, const CandidateGrid& g, std::vector<uint32_t>* start,
                      std::vector<uint16_t>* list, std::vector<uint16_t>* levels);

// ---------------------------------------------------------------- device views
// Staged into shared memory by every block: the Vina-form path copies the prefix up
// to `gmm`, the TRIDS path the whole struct.
struct alignas(16) DevParams {
    int term_set, n_types, gmm_k, pad0;
    float w[5];
    float cutoff, cut2, w_tor;
    float radius[kNT];
    uint32_t tflags[kNT];          // per type: bit0 hydrophobic, bit1 donor, bit2 acceptor
    float2 pairtab[kNT][kNT];      // (R_a + R_b, pair flags as int bits: 1 hydrophobic, 2 donor-acceptor)
    float4 ftab[kNT];              // per ligand type, its Vina-form flag term w sat(a - b d) against
                                   // candidates with mask bits m: (m as bits << 13, -b, a, w)
    float4 gmm[kNT][kNTP][kKP];    // (pi, mu, -log2(e)/(2 sigma^2), 1/sigma^2): exp(-z^2/(2 sigma^2))
                                   // = ex2(z^2 * .z); [a][b][k] for b < kNT, k < kK (the rest is padding)
};

struct DevPocket {
    const float4* atoms;           // [M + 1]: (x, y, z, radius); atoms[M] = far sentinel
    const uint8_t* ptype;          // [M + 1] (padded to 16 bytes): atom types
    const uint32_t* cell_start;
    const uint16_t* cand;          // pocket index (13 bits) | flags of that atom << 13
    const uint16_t* cell_levels;   // [ncell][kReachLevels]: blocks needed per reach level
    const DevParams* params;
    int M;
    int nx, ny, nz;
    float gx, gy, gz, inv_h;
    int n_boxes;                   // pose p samples in box p mod n_boxes
    float box_lo[kMaxBoxes][3], box_hi[kMaxBoxes][3];
    // grid maps of the ligand-pocket atom-pair terms: maps[type][z][y][x] at points
    // mlo + mh * (x, y, z); an atom whose cell lies inside takes the trilinear value
    int use_maps;
    int mx, my, mz;
    float mlo[3], mh, inv_mh;
    const float* maps;
    // near lists of the atom-pair E_MDN (term set 1), same cells as cell_start
    const uint32_t* ncell_start;
    const uint16_t* nlist;
    const uint16_t* nlevels;       // [ncell][kReachLevels]: near-list entries per reach level
    float near_cut2;               // min(5 A, cutoff)^2
    // residue-level E_MDN (term set 2)
    int n_res;
    const int32_t* res_start;      // [n_res + 1]: residue r = staged pocket atoms [start[r], start[r+1])
    const uint32_t* rcell_start;   // [ncell + 1], same cells as cell_start
    const uint32_t* rlist;         // residues near each cell: r | first atom << 13 | atom count << 26
    const uint16_t* rlevels;       // [ncell][kReachLevels]: residue-list entries per reach level
};

struct LigHdr {
    int n_atoms, n_tor, atom_off, tor_off;
    int ipre_off, ient_off, n_pairs;   // intra partner lists: per-atom block prefix at ipre_off
                                       // (L + 1 ints), entries at ient_off (8 per block)
    int sid;                           // random-stream id of the ligand (before lig_base is added):
                                       // its batch index unless trids_set_stream_ids gave another
};

struct DevBatch {
    int n_lig, max_atoms, max_tor, dof_stride, n_fields;
    const LigHdr* lig;
    const float4* atom_y;          // local coords about the root centroid, w = type bits
    const int* atom_orig;          // input index of each packed atom
    const int4* tor_idx;           // (parent atom, child atom, subtree begin, subtree end)
    const float4* tor_u;           // unit axis, input geometry
    const float4* tor_p;           // parent atom, local coords
    const uint32_t* atom_mask;     // per packed atom: bit k set when torsion k moves it (its fragment's
                                   // torsion and that torsion's ancestors; 0 for the root fragment)
    const int* ipre;               // per atom: first block of its intra partner list
    const uint16_t* ient;          // partner index | partner flags << 13; each intra pair appears
                                   // once from each side; padding = max_atoms (far sentinel)
    // residue-level E_MDN kernels per packed atom row: [row][n_res][K] of
    // (pi, mu, -1/(2 sigma^2), 1/sigma^2)
    const float4* mdn;
    int mdn_res, mdn_k;
};

// Sampler state fields per pose (SoA over poses inside each ligand):
//   [0,6) Adam m of (t, w); [6,12) Adam v; [12,19) saved (t, q); 19 E_cur; 20 E_saved;
//   21 status bits; then T_max each of m_theta, v_theta, saved theta.
constexpr int kFieldM = 0, kFieldV = 6, kFieldSaved = 12, kFieldEcur = 19, kFieldEsaved = 20,
              kFieldStatus = 21, kFieldTheta = 22;
TRIDS_HD inline int state_fields(int max_tor) { return kFieldTheta + 3 * max_tor; }
TRIDS_HD inline int trace_record(int max_tor) { return 2 * max_tor + 14; }

}  // namespace trids
