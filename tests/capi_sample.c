/* End-to-end use of the C-ABI from C on the GPU: reads a pocket, scoring parameters and
 * ligands from a binary input file, builds the pocket and the batch, allocates the device
 * buffers with the CUDA runtime, samples, ranks, and writes energies, DOFs and top-k
 * indices to an output file.  Built and run by tests/test_gpu_capi_c.py, which compares
 * the output with the Python path bit for bit.
 *
 * Input (little-endian): int32 M, n_lig, total_atoms, total_bonds, poses, steps, mc_loops,
 * k; uint64 seed; float box_center[3], box_size[3]; float pocket_xyz[M*3]; int32
 * pocket_type[M]; int32 n_types; float radius[n_types]; uint8 flags[n_types]; float w[5],
 * cutoff; int32 n_atoms[n_lig]; float xyz[total_atoms*3]; int32 type[total_atoms]; int32
 * n_bonds[n_lig]; int32 bonds[total_bonds*2]; uint8 rotatable[total_bonds].
 * Output: int32 dof_stride; float energy[n_lig*poses]; float dof[n_lig*poses*dof_stride];
 * int32 idx[n_lig*k]. */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "trids.h"

#define RD(ptr, n)                                                                   \
    do {                                                                             \
        if (fread((ptr), sizeof(*(ptr)), (size_t)(n), f) != (size_t)(n)) {          \
            fprintf(stderr, "short read: %s\n", #ptr);                               \
            return 2;                                                                \
        }                                                                            \
    } while (0)
#define CK(call)                                                                     \
    do {                                                                             \
        int rc_ = (int)(call);                                                       \
        if (rc_ != 0) {                                                              \
            fprintf(stderr, "%s failed: %d %s\n", #call, rc_, trids_last_error());   \
            return 3;                                                                \
        }                                                                            \
    } while (0)
#define CU(call)                                                                     \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            fprintf(stderr, "%s failed: %s\n", #call, cudaGetErrorString(e_));       \
            return 4;                                                                \
        }                                                                            \
    } while (0)

int main(int argc, char** argv) {
    if (argc != 3) { fprintf(stderr, "usage: capi_sample in.bin out.bin\n"); return 1; }
    FILE* f = fopen(argv[1], "rb");
    if (!f) { perror("input"); return 1; }
    int32_t hdr[8];
    uint64_t seed;
    float center[3], size[3];
    RD(hdr, 8);
    RD(&seed, 1);
    RD(center, 3);
    RD(size, 3);
    const int32_t M = hdr[0], n_lig = hdr[1], n_at = hdr[2], n_bd = hdr[3], P = hdr[4], S = hdr[5], Lmc = hdr[6],
                  k = hdr[7];
    float* pxyz = malloc(sizeof(float) * 3 * M);
    int32_t* ptype = malloc(sizeof(int32_t) * M);
    RD(pxyz, 3 * M);
    RD(ptype, M);
    trids_params prm;
    memset(&prm, 0, sizeof prm);
    RD(&prm.n_types, 1);
    RD(prm.radius, prm.n_types);
    RD(prm.flags, prm.n_types);
    RD(prm.w, 5);
    RD(&prm.cutoff, 1);
    prm.term_set = TRIDS_TERMS_VINA5;
    prm.w_tor = 0.01f;
    int32_t* na = malloc(sizeof(int32_t) * n_lig);
    float* xyz = malloc(sizeof(float) * 3 * n_at);
    int32_t* ty = malloc(sizeof(int32_t) * n_at);
    int32_t* nb = malloc(sizeof(int32_t) * n_lig);
    int32_t* bonds = malloc(sizeof(int32_t) * 2 * (n_bd > 0 ? n_bd : 1));
    uint8_t* rot = malloc(n_bd > 0 ? n_bd : 1);
    RD(na, n_lig);
    RD(xyz, 3 * n_at);
    RD(ty, n_at);
    RD(nb, n_lig);
    RD(bonds, 2 * n_bd);
    RD(rot, n_bd);
    fclose(f);

    trids_pocket* pk = NULL;
    trids_batch* b = NULL;
    trids_batch_dims dims;
    CK(trids_make_pocket(pxyz, ptype, M, center, size, 0.f, &prm, &pk));
    CK(trids_pack_ligands(pk, n_lig, na, xyz, ty, nb, bonds, rot, &b));
    CK(trids_batch_info(b, &dims));
    const size_t n_dof = (size_t)n_lig * P * dims.dof_stride;
    const int64_t n_state = trids_state_floats(b, P);
    float *d_dof, *d_state, *d_energy, *d_etop;
    int32_t* d_idx;
    CU(cudaMalloc((void**)&d_dof, sizeof(float) * n_dof));
    CU(cudaMalloc((void**)&d_state, sizeof(float) * (size_t)n_state));
    CU(cudaMalloc((void**)&d_energy, sizeof(float) * (size_t)n_lig * P));
    CU(cudaMalloc((void**)&d_idx, sizeof(int32_t) * (size_t)n_lig * k));
    CU(cudaMalloc((void**)&d_etop, sizeof(float) * (size_t)n_lig * k));
    trids_sample_cfg cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.poses = P;
    cfg.steps = S;
    cfg.step_begin = 0;
    cfg.step_end = S;
    cfg.mc_loops = Lmc;
    cfg.lr = 0.1f;
    cfg.beta1 = 0.9f;
    cfg.beta2 = 0.999f;
    cfg.eps = 1e-8f;
    cfg.beta = 0.069f;
    cfg.seed = seed;
    cfg.mode = TRIDS_MODE_PERSISTENT;
    cfg.use_graph = 1;
    cfg.optimizer = TRIDS_OPT_ADAM;
    CK(trids_sample(pk, b, &cfg, d_dof, d_state, d_energy, NULL));
    CK(trids_topk(b, P, d_energy, d_dof, k, 1.0f, d_idx, d_etop, NULL));
    CK(trids_sync(b, P, d_state, NULL, 120000.0));

    float* energy = malloc(sizeof(float) * (size_t)n_lig * P);
    float* dof = malloc(sizeof(float) * n_dof);
    int32_t* idx = malloc(sizeof(int32_t) * (size_t)n_lig * k);
    CU(cudaMemcpy(energy, d_energy, sizeof(float) * (size_t)n_lig * P, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(dof, d_dof, sizeof(float) * n_dof, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(idx, d_idx, sizeof(int32_t) * (size_t)n_lig * k, cudaMemcpyDeviceToHost));
    FILE* o = fopen(argv[2], "wb");
    if (!o) { perror("output"); return 1; }
    fwrite(&dims.dof_stride, sizeof(int32_t), 1, o);
    fwrite(energy, sizeof(float), (size_t)n_lig * P, o);
    fwrite(dof, sizeof(float), n_dof, o);
    fwrite(idx, sizeof(int32_t), (size_t)n_lig * k, o);
    fclose(o);
    CU(cudaFree(d_dof));
    CU(cudaFree(d_state));
    CU(cudaFree(d_energy));
    CU(cudaFree(d_idx));
    CU(cudaFree(d_etop));
    CK(trids_free_batch(b));
    CK(trids_free_pocket(pk));
    printf("OK %d ligands x %d poses x %d evaluations\n", n_lig, P, S);
    return 0;
}
