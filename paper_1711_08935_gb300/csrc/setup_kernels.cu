// Setup kernels: sphere membership, Bloch phases of the image segments, orbital sampling and the
// per-atom Loewdin orthonormalisation (Sec. II, Fig. 1; Sec. III).
#include "dftu_internal.cuh"

namespace dftu {

__device__ __forceinline__ int floor_div(int a, int n) {
    int q = a / n;
    return (a % n != 0 && ((a < 0) != (n < 0))) ? q - 1 : q;
}

// One thread per point of an atom's bounding box (z outer, y, x inner).  flag = image id (0..124)
// when the unfolded point lies in the sphere, else -1.  The distance test is the membership rule
// of the sub-grid: d2 = (dx*dx + dy*dy) + dz*dz <= R*R, each operation rounded to nearest, no FMA.
__global__ void k_sphere_flags(View v, const double* __restrict__ pos, const double* __restrict__ rad,
                               const int* __restrict__ box_lo, const int* __restrict__ box_dim,
                               const int64_t* __restrict__ box_off, int natoms, int64_t nbox,
                               signed char* __restrict__ flags) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nbox) return;
    int a = 0;
    while (a + 1 < natoms && box_off[a + 1] <= g) ++a;
    int64_t b = g - box_off[a];
    int bx = box_dim[3 * a], by = box_dim[3 * a + 1];
    int ix = box_lo[3 * a] + (int)(b % bx);
    int jy = box_lo[3 * a + 1] + (int)((b / bx) % by);
    int kz = box_lo[3 * a + 2] + (int)(b / ((int64_t)bx * by));
    double dx = __dsub_rn(__dadd_rn(__dmul_rn((double)ix, v.h0), v.o0), pos[3 * a]);
    double dy = __dsub_rn(__dadd_rn(__dmul_rn((double)jy, v.h1), v.o1), pos[3 * a + 1]);
    double dz = __dsub_rn(__dadd_rn(__dmul_rn((double)kz, v.h2), v.o2), pos[3 * a + 2]);
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    double R = rad[a];
    bool in = d2 <= __dmul_rn(R, R);
    int img = 62;  // (0,0,0)
    if (v.periodic) {
        int tx = floor_div(ix, v.n0), ty = floor_div(jy, v.n1), tz = floor_div(kz, v.n2);
        img = (tx + IMG_RANGE) + 5 * ((ty + IMG_RANGE) + 5 * (tz + IMG_RANGE));
    } else {
        in = in && ix >= 0 && ix < v.n0 && jy >= 0 && jy < v.n1 && kz >= 0 && kz < v.n2;
    }
    flags[g] = in ? (signed char)img : (signed char)-1;
}

cudaError_t launch_sphere_flags(const View& v, const double* pos, const double* rad, const int* box_lo,
                                const int* box_dim, const int64_t* box_off, int natoms, int64_t nbox,
                                signed char* flags, cudaStream_t st) {
    int64_t blocks = (nbox + 255) / 256;
    k_sphere_flags<<<(unsigned)blocks, 256, 0, st>>>(v, pos, rad, box_lo, box_dim, box_off, natoms, nbox, flags);
    return cudaGetLastError();
}

// exp(+i k.T) for each image segment and k-point; T in cells times the cell edge.
__global__ void k_seg_phases(View v) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= v.nseg * v.nk) return;
    int s = g / v.nk, k = g % v.nk;
    double Tx = v.seg_T[3 * s] * (v.n0 * v.h0), Ty = v.seg_T[3 * s + 1] * (v.n1 * v.h1),
           Tz = v.seg_T[3 * s + 2] * (v.n2 * v.h2);
    double arg = v.kvec[3 * k] * Tx + v.kvec[3 * k + 1] * Ty + v.kvec[3 * k + 2] * Tz;
    double sn, cs;
    sincos(arg, &sn, &cs);
    v.seg_phase[g] = make_double2(cs, sn);
}

cudaError_t launch_seg_phases(const View& v, cudaStream_t st) {
    int n = v.nseg * v.nk;
    k_seg_phases<<<(n + 127) / 128, 128, 0, st>>>(v);
    return cudaGetLastError();
}

// Real spherical harmonics, m = -l..l (s: 1 | p: y,z,x | d: xy,yz,3z^2-r^2,xz,x^2-y^2 | f: ...).
__device__ void real_ylm(int l, double x, double y, double z, double r, double* Y) {
    const double pi = 3.14159265358979323846;
    if (l == 0) { Y[0] = 0.5 / sqrt(pi); return; }
    if (r == 0.0) { for (int m = 0; m < 2 * l + 1; ++m) Y[m] = 0.0; return; }
    if (l == 1) {
        double c = sqrt(3.0 / (4 * pi)) / r;
        Y[0] = c * y; Y[1] = c * z; Y[2] = c * x;
    } else if (l == 2) {
        double r2 = r * r;
        double c1 = sqrt(15.0 / (4 * pi)) / r2, c2 = sqrt(5.0 / (16 * pi)) / r2, c3 = sqrt(15.0 / (16 * pi)) / r2;
        Y[0] = c1 * x * y; Y[1] = c1 * y * z; Y[2] = c2 * (3 * z * z - r2); Y[3] = c1 * x * z;
        Y[4] = c3 * (x * x - y * y);
    } else {
        double r2 = r * r, r3 = r2 * r;
        Y[0] = sqrt(35.0 / (32 * pi)) * y * (3 * x * x - y * y) / r3;
        Y[1] = sqrt(105.0 / (4 * pi)) * x * y * z / r3;
        Y[2] = sqrt(21.0 / (32 * pi)) * y * (5 * z * z - r2) / r3;
        Y[3] = sqrt(7.0 / (16 * pi)) * z * (5 * z * z - 3 * r2) / r3;
        Y[4] = sqrt(21.0 / (32 * pi)) * x * (5 * z * z - r2) / r3;
        Y[5] = sqrt(105.0 / (16 * pi)) * z * (x * x - y * y) / r3;
        Y[6] = sqrt(35.0 / (32 * pi)) * x * (x * x - 3 * y * y) / r3;
    }
}

// Four-point Lagrange interpolation of R on r_i = i*dr (nodes a..a+3, a = clamp(floor(r/dr)-1, 0, nr-4)),
// zero at and beyond the last node.
__device__ double radial_interp(const double* __restrict__ tab, int nr, double dr, double r) {
    double t = r / dr;
    double fi = floor(t);
    if (fi >= (double)(nr - 1)) return 0.0;
    int i = (int)fi;
    int a = min(max(i - 1, 0), nr - 4);
    double x = t - (double)a;
    double w0 = -(x - 1.0) * (x - 2.0) * (x - 3.0) / 6.0;
    double w1 = x * (x - 2.0) * (x - 3.0) / 2.0;
    double w2 = -x * (x - 1.0) * (x - 3.0) / 2.0;
    double w3 = x * (x - 1.0) * (x - 2.0) / 6.0;
    return w0 * tab[a] + w1 * tab[a + 1] + w2 * tab[a + 2] + w3 * tab[a + 3];
}

// One CTA per tile, one thread per point: raw orbitals phi_m = R(|d|) Y_lm(d).
__global__ void k_orbitals(View v, const double* __restrict__ rtab, const int* __restrict__ roff,
                           const int* __restrict__ rnr, const double* __restrict__ rdr) {
    const Tile t = v.tiles[blockIdx.x];
    int i = threadIdx.x;
    if (i >= t.np) return;
    int64_t j = t.p0 + i;
    int a = t.atom;
    int sp = v.atom_species[a];
    int ix = v.pt_u[3 * j], jy = v.pt_u[3 * j + 1], kz = v.pt_u[3 * j + 2];
    double dx = __dsub_rn(__dadd_rn(__dmul_rn((double)ix, v.h0), v.o0), v.atom_pos[3 * a]);
    double dy = __dsub_rn(__dadd_rn(__dmul_rn((double)jy, v.h1), v.o1), v.atom_pos[3 * a + 1]);
    double dz = __dsub_rn(__dadd_rn(__dmul_rn((double)kz, v.h2), v.o2), v.atom_pos[3 * a + 2]);
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    double r = sqrt(d2);
    double Rv = radial_interp(rtab + roff[sp], rnr[sp], rdr[sp], r);
    double Y[MAXM];
    int l = (t.M - 1) / 2;
    real_ylm(l, dx, dy, dz, r, Y);
    double* out = v.phi64 + t.phi0 + (int64_t)i * t.M;
    for (int m = 0; m < t.M; ++m) out[m] = Rv * Y[m];
}

cudaError_t launch_orbitals(const View& v, const double* radial_tab, const int* radial_off,
                            const int* radial_nr, const double* radial_dr, cudaStream_t st) {
    k_orbitals<<<v.ntiles, TILE, 0, st>>>(v, radial_tab, radial_off, radial_nr, radial_dr);
    return cudaGetLastError();
}

// S_{mm'} = dV sum_j phi_m phi_m' over the atom's points; one CTA per atom, fixed-order tree reduction.
__global__ void k_overlap(View v, double* __restrict__ S) {
    int a = blockIdx.x;
    int M = v.atom_M[a];
    int P = M * M;
    __shared__ double red[CTA];
    for (int pq = 0; pq < P; ++pq) {
        int pm = pq / M, qm = pq % M;
        double acc = 0.0;
        for (int t = v.atom_tile_beg[a]; t < v.atom_tile_end[a]; ++t) {
            const Tile tl = v.tiles[t];
            const double* ph = v.phi64 + tl.phi0;
            for (int i = threadIdx.x; i < tl.np; i += blockDim.x) acc += ph[i * M + pm] * ph[i * M + qm];
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) S[a * MAXM * MAXM + pq] = red[0] * v.dV;
        __syncthreads();
    }
}

// Cyclic Jacobi diagonalisation of the symmetric S (one thread per atom), then T = S^{-1/2} = U L^{-1/2} U^T
// stored over S.
// cond[a] receives lambda_min / lambda_max of the atom's overlap matrix, or -1 when that ratio is not
// defined (no positive or a non-finite eigenvalue); the host refuses atoms whose orbitals are linearly
// dependent on the sphere, for which S^(-1/2) does not exist.
__global__ void k_inv_sqrt(View v, double* __restrict__ S, double* __restrict__ cond) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= v.natoms) return;
    int M = v.atom_M[a];
    double A[MAXM][MAXM], U[MAXM][MAXM];
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < M; ++q) {
            A[p][q] = 0.5 * (S[a * MAXM * MAXM + p * M + q] + S[a * MAXM * MAXM + q * M + p]);
            U[p][q] = (p == q) ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int p = 0; p < M; ++p) {
            dia += A[p][p] * A[p][p];
            for (int q = p + 1; q < M; ++q) off += A[p][q] * A[p][q];
        }
        if (off <= 1e-34 * dia) break;
        for (int p = 0; p < M; ++p)
            for (int q = p + 1; q < M; ++q) {
                if (A[p][q] == 0.0) continue;
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < M; ++k) {
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < M; ++k) {
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < M; ++k) {
                    double ukp = U[k][p], ukq = U[k][q];
                    U[k][p] = c * ukp - s * ukq;
                    U[k][q] = s * ukp + c * ukq;
                }
            }
    }
    double lmin = A[0][0], lmax = A[0][0];
    for (int p = 1; p < M; ++p) { lmin = fmin(lmin, A[p][p]); lmax = fmax(lmax, A[p][p]); }
    cond[a] = (isfinite(lmin) && isfinite(lmax) && lmax > 0.0) ? lmin / lmax : -1.0;
    double il[MAXM];
    for (int p = 0; p < M; ++p) il[p] = 1.0 / sqrt(A[p][p]);
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < M; ++q) {
            double s = 0.0;
            for (int k = 0; k < M; ++k) s += U[p][k] * il[k] * U[q][k];
            S[a * MAXM * MAXM + p * M + q] = s;
        }
}

// phi'_m = sum_m' phi_m' T_{m'm}; also the FP32 split phi = hi + lo used by the reduced-precision paths.
__global__ void k_lowdin_apply(View v, const double* __restrict__ T) {
    const Tile t = v.tiles[blockIdx.x];
    int i = threadIdx.x;
    if (i >= t.np) return;
    int M = t.M;
    const double* Ta = T + t.atom * MAXM * MAXM;
    double* ph = v.phi64 + t.phi0 + (int64_t)i * M;
    double x[MAXM], y[MAXM];
    for (int m = 0; m < M; ++m) x[m] = ph[m];
    for (int m = 0; m < M; ++m) {
        double s = 0.0;
        for (int q = 0; q < M; ++q) s += x[q] * Ta[q * M + m];
        y[m] = s;
    }
    for (int m = 0; m < M; ++m) {
        ph[m] = y[m];
        float hi = __double2float_rn(y[m]);
        v.phi_hi[t.phi0 + (int64_t)i * M + m] = hi;
        v.phi_lo[t.phi0 + (int64_t)i * M + m] = __double2float_rn(y[m] - (double)hi);
    }
}

cudaError_t launch_lowdin(const View& v, double* work_S, double* cond, cudaStream_t st) {
    k_overlap<<<v.natoms, CTA, 0, st>>>(v, work_S);
    k_inv_sqrt<<<(v.natoms + 63) / 64, 64, 0, st>>>(v, work_S, cond);
    k_lowdin_apply<<<v.ntiles, TILE, 0, st>>>(v, work_S);
    return cudaGetLastError();
}

}  // namespace dftu
