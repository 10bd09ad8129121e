/*
 * c_abi_driver.c -- a plain C program that runs one DFT+U pass through the library's C ABI
 * (include/dftu.h) with device buffers and a stream of its own, for tests/test_gpu_c_abi.py.
 *
 * Usage: c_abi_driver IN OUT.  IN holds, in host byte order:
 *   int32  n[3], periodic, nk, spin (dftu_spin), nb, natoms, nspecies
 *   f64    h[3], origin[3], kvec[nk][3], wk[nk]
 *   f64    pos[natoms][3], radius[natoms];  int32 species[natoms], l[natoms]
 *   per species: int32 nr; f64 dr, R[nr], V[M^4] (the Coulomb integrals to use, M of the species)
 *   f64    psi [nk][nspin][nb][npts] interleaved complex; f [nk][nspin][nb]
 * OUT receives: int32 status[8]; f64 U[natoms], J[natoms], EU_atom[natoms], EU_total,
 *   n [sum over atoms of nspin M M] complex, p [nk][nspin][nb][sum M] complex,
 *   psi after psi += V_U psi, and the integrals dftu_coulomb_integrals computed per species.
 * The pass is project (Eq. 4 projections) -> occupations (Eqs. 4, 8, 9) -> ACBN0 U, J (Eqs. 10-11)
 * -> apply (Eq. 6).  Exit status 0 when every call returned; the statuses are written for the test.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "dftu.h"

static FILE* fin;

static void rd(void* dst, size_t size, size_t n) {
    if (n && fread(dst, size, n, fin) != n) {
        fprintf(stderr, "short input\n");
        exit(2);
    }
}

static void* xmalloc(size_t bytes) {
    void* p = malloc(bytes ? bytes : 1);
    if (!p) {
        fprintf(stderr, "out of host memory\n");
        exit(2);
    }
    return p;
}

#define CUDA_OR_EXIT(call)                                                       \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));          \
            exit(3);                                                             \
        }                                                                        \
    } while (0)

int main(int argc, char** argv) {
    if (argc != 3) {
        fprintf(stderr, "usage: %s IN OUT\n", argv[0]);
        return 2;
    }
    fin = fopen(argv[1], "rb");
    if (!fin) return 2;
    int32_t hdr[9];
    rd(hdr, 4, 9);
    dftu_grid g;
    for (int a = 0; a < 3; ++a) g.n[a] = hdr[a];
    g.periodic = hdr[3];
    const int nk = hdr[4], spin = hdr[5], nb = hdr[6], natoms = hdr[7], nspecies = hdr[8];
    const int nspin = spin == DFTU_COLLINEAR ? 2 : 1;
    const int64_t npts = (int64_t)g.n[0] * g.n[1] * g.n[2];
    rd(g.h, 8, 3);
    rd(g.origin, 8, 3);
    double* kvec = xmalloc(sizeof(double) * 3 * nk);
    double* wk = xmalloc(sizeof(double) * nk);
    rd(kvec, 8, 3 * (size_t)nk);
    rd(wk, 8, (size_t)nk);

    dftu_atom* atoms = xmalloc(sizeof(dftu_atom) * natoms);
    double* pos = xmalloc(sizeof(double) * 3 * natoms);
    double* radius = xmalloc(sizeof(double) * natoms);
    int32_t* species = xmalloc(sizeof(int32_t) * natoms);
    int32_t* l = xmalloc(sizeof(int32_t) * natoms);
    rd(pos, 8, 3 * (size_t)natoms);
    rd(radius, 8, (size_t)natoms);
    rd(species, 4, (size_t)natoms);
    rd(l, 4, (size_t)natoms);
    int MT = 0, nsum = 0;
    for (int I = 0; I < natoms; ++I) {
        memcpy(atoms[I].pos, pos + 3 * I, sizeof(double) * 3);
        atoms[I].species = species[I];
        atoms[I].l = l[I];
        atoms[I].radius = radius[I];
        MT += 2 * l[I] + 1;
        nsum += nspin * (2 * l[I] + 1) * (2 * l[I] + 1);
    }

    dftu_radial* rad = xmalloc(sizeof(dftu_radial) * nspecies);
    double** V = xmalloc(sizeof(double*) * nspecies);
    int* Msp = xmalloc(sizeof(int) * nspecies);
    for (int s = 0; s < nspecies; ++s) {
        Msp[s] = 0;
        for (int I = 0; I < natoms; ++I)
            if (species[I] == s) {
                Msp[s] = 2 * l[I] + 1;
                break;
            }
        int32_t nr;
        rd(&nr, 4, 1);
        double* R = xmalloc(sizeof(double) * (nr + 1));
        rd(&rad[s].dr, 8, 1);
        rd(R, 8, (size_t)nr);
        rad[s].nr = nr;
        rad[s].R = R;
        const size_t m4 = (size_t)Msp[s] * Msp[s] * Msp[s] * Msp[s];
        V[s] = xmalloc(sizeof(double) * m4);
        rd(V[s], 8, m4);
    }
    const size_t psi_doubles = (size_t)2 * nk * nspin * nb * npts;
    const size_t f_doubles = (size_t)nk * nspin * nb;
    double* psi_h = xmalloc(sizeof(double) * psi_doubles);
    double* f_h = xmalloc(sizeof(double) * f_doubles);
    rd(psi_h, 8, psi_doubles);
    rd(f_h, 8, f_doubles);
    if (fgetc(fin) != EOF) {
        fprintf(stderr, "trailing input\n");
        return 2;
    }
    fclose(fin);

    CUDA_OR_EXIT(cudaSetDevice(0));
    cudaStream_t stream;
    CUDA_OR_EXIT(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    void* psi_d;
    double* f_d;
    CUDA_OR_EXIT(cudaMalloc(&psi_d, sizeof(double) * psi_doubles));
    CUDA_OR_EXIT(cudaMalloc((void**)&f_d, sizeof(double) * f_doubles));
    CUDA_OR_EXIT(cudaMemcpyAsync(psi_d, psi_h, sizeof(double) * psi_doubles, cudaMemcpyHostToDevice, stream));
    CUDA_OR_EXIT(cudaMemcpyAsync(f_d, f_h, sizeof(double) * f_doubles, cudaMemcpyHostToDevice, stream));

    int32_t st[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    double* U = xmalloc(sizeof(double) * natoms);
    double* J = xmalloc(sizeof(double) * natoms);
    double* EUa = xmalloc(sizeof(double) * natoms);
    double EU = 0.0;
    double* n_out = xmalloc(sizeof(double) * 2 * nsum);
    double* p_out = xmalloc(sizeof(double) * 2 * (size_t)nk * nspin * nb * MT);
    double** Vg = xmalloc(sizeof(double*) * nspecies);
    for (int s = 0; s < nspecies; ++s) {
        Vg[s] = xmalloc(sizeof(double) * Msp[s] * Msp[s] * Msp[s] * Msp[s]);
        memset(Vg[s], 0, sizeof(double) * Msp[s] * Msp[s] * Msp[s] * Msp[s]);
    }

    dftu_handle h = NULL;
    st[0] = dftu_create(&h, &g, nk, kvec, wk, (dftu_spin)spin, nb, 0);
    if (st[0] == DFTU_OK) {
        st[1] = dftu_setup_atoms(h, natoms, atoms, nspecies, rad, NULL);
        st[2] = DFTU_OK;
        for (int s = 0; s < nspecies && st[1] == DFTU_OK && st[2] == DFTU_OK; ++s) {
            st[2] = dftu_coulomb_integrals(h, s, Vg[s]);
            if (st[2] == DFTU_OK) st[2] = dftu_set_coulomb(h, s, V[s]);
        }
        if (st[1] == DFTU_OK && st[2] == DFTU_OK) {
            st[3] = dftu_project(h, psi_d, DFTU_C128, nb, npts, stream);
            st[4] = dftu_occupations(h, f_d, stream);
            st[5] = dftu_acbn0_uj(h, stream);
            st[6] = dftu_apply(h, psi_d, DFTU_C128, nb, npts, NULL, 1, stream);
            if (dftu_get_results(h, n_out, U, J, EUa, &EU, stream) != DFTU_OK ||
                dftu_get_projections(h, p_out, stream) != DFTU_OK)
                st[7] = DFTU_ERR_CUDA;
            else
                st[7] = dftu_sync_status(h);
        }
        if (st[1] != DFTU_OK || st[2] != DFTU_OK) fprintf(stderr, "%s\n", dftu_last_error(h));
        dftu_destroy(h);
    }
    CUDA_OR_EXIT(cudaMemcpyAsync(psi_h, psi_d, sizeof(double) * psi_doubles, cudaMemcpyDeviceToHost, stream));
    CUDA_OR_EXIT(cudaStreamSynchronize(stream));

    FILE* fo = fopen(argv[2], "wb");
    if (!fo) return 2;
    fwrite(st, 4, 8, fo);
    fwrite(U, 8, (size_t)natoms, fo);
    fwrite(J, 8, (size_t)natoms, fo);
    fwrite(EUa, 8, (size_t)natoms, fo);
    fwrite(&EU, 8, 1, fo);
    fwrite(n_out, 8, 2 * (size_t)nsum, fo);
    fwrite(p_out, 8, 2 * (size_t)nk * nspin * nb * MT, fo);
    fwrite(psi_h, 8, psi_doubles, fo);
    for (int s = 0; s < nspecies; ++s) fwrite(Vg[s], 8, (size_t)Msp[s] * Msp[s] * Msp[s] * Msp[s], fo);
    fclose(fo);
    CUDA_OR_EXIT(cudaFree(psi_d));
    CUDA_OR_EXIT(cudaFree(f_d));
    CUDA_OR_EXIT(cudaStreamDestroy(stream));
    return 0;
}
