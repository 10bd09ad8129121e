// Gauge-invariant Hubbard operator and Hubbard current under a uniform vector potential A (Sec. V).
//
// Eq. (16) attaches the phase exp(-i A.r) to every localised orbital.  Measured from the atom the
// orbital belongs to (d = r - R_I, the atom-relative reading of Eq. 16), the projector becomes
//   p^A_m = <phi_m exp(-i A.d)|psi> = dV sum_j phi_m(j) exp(+i A.d_j) exp(+i k.T_j) psi(idx_j),
// and the operator scatters with exp(-i A.d_j).  The per-point phases are tabulated here once per A;
// the streaming kernels rotate each loaded state value (projection) or each update (apply) by them.
//
// Eq. (17), the Hubbard contribution to the current, is taken as J = sum w f <psi| -i [r, V_U^A] |psi>
// (the factor i of the velocity operator restored, since <[r, V]> + c.c. of a Hermitian V vanishes).
// With q^{(a)}_m = <phi_m d_a exp(-i A.d)|psi>, the projections onto orbitals weighted by the a-th
// displacement component,
//   J_a = -i sum w f sum_{mm'} V_{mm'} [conj(q_m) p_m' - conj(p_m) q_m'],
// a real number; it equals dE_U/dA at fixed states.
#include "dftu_internal.cuh"

namespace dftu {

__device__ __forceinline__ void displacement(const View& v, int64_t j, int atom, double& dx, double& dy, double& dz) {
    const int ix = v.pt_u[3 * j], jy = v.pt_u[3 * j + 1], kz = v.pt_u[3 * j + 2];
    dx = __dsub_rn(__dadd_rn(__dmul_rn((double)ix, v.h0), v.o0), v.atom_pos[3 * atom]);
    dy = __dsub_rn(__dadd_rn(__dmul_rn((double)jy, v.h1), v.o1), v.atom_pos[3 * atom + 1]);
    dz = __dsub_rn(__dadd_rn(__dmul_rn((double)kz, v.h2), v.o2), v.atom_pos[3 * atom + 2]);
}

// exp(+i A.d_j) for every sphere point: FP64 (cos, sin) and the FP32 pair split (hi, hi, lo, lo).
__global__ void k_gauge_phases(View v, const double* __restrict__ A) {
    if (blockIdx.x == 0 && threadIdx.x < 3) v.gaugeA[threadIdx.x] = A[threadIdx.x];   // for the real-time step
    const Tile t = v.tiles[blockIdx.x];
    const int i = threadIdx.x;
    if (i >= t.np) return;
    const int64_t j = t.p0 + i;
    double dx, dy, dz;
    displacement(v, j, t.atom, dx, dy, dz);
    const double th = fma(A[2], dz, fma(A[1], dy, A[0] * dx));
    double s, c;
    sincos(th, &s, &c);
    v.gauge_d[j] = make_double2(c, s);
    const float ch = __double2float_rn(c), sh = __double2float_rn(s);
    v.gauge_f[j] = make_float4(ch, sh, __double2float_rn(c - (double)ch), __double2float_rn(s - (double)sh));
}

cudaError_t launch_gauge_phases(const View& v, const double* A, cudaStream_t st) {
    k_gauge_phases<<<v.ntiles, TILE, 0, st>>>(v, A);
    return cudaGetLastError();
}

// phid[a][point][m] = phi_m(point) * d_a(point), with its FP32 split, for a = x, y, z.
__global__ void k_displaced_orbitals(View v, int64_t phi_total) {
    const Tile t = v.tiles[blockIdx.x];
    const int i = threadIdx.x;
    if (i >= t.np) return;
    double d[3];
    displacement(v, t.p0 + i, t.atom, d[0], d[1], d[2]);
    const int64_t e0 = t.phi0 + (int64_t)i * t.M;
    for (int a = 0; a < 3; ++a)
        for (int m = 0; m < t.M; ++m) {
            const double y = v.phi64[e0 + m] * d[a];
            const float hi = __double2float_rn(y);
            v.phid64[a * phi_total + e0 + m] = y;
            v.phid_hi[a * phi_total + e0 + m] = hi;
            v.phid_lo[a * phi_total + e0 + m] = __double2float_rn(y - (double)hi);
        }
}

cudaError_t launch_displaced_orbitals(const View& v, int64_t phi_total, cudaStream_t st) {
    k_displaced_orbitals<<<v.ntiles, TILE, 0, st>>>(v, phi_total);
    return cudaGetLastError();
}

// One CTA per (atom, direction a): Jat[atom][a] = mult Im( sum w f sum_{xy} V_xy [conj(q_x) p_y - conj(p_x) q_y] ),
// q = pgrad[a] (projections onto the displaced orbitals).  Collinear or unpolarised states.
__global__ void __launch_bounds__(CTA) k_current(View v, const double* __restrict__ f, int nbands, double* __restrict__ Jat) {
    const int atom = blockIdx.x, dir = blockIdx.y;
    const int M = v.atom_M[atom], mo = v.atom_moff[atom];
    const int64_t vo = v.atom_mat_off[atom];
    const double2* g = v.pgrad + dir * (int64_t)v.nk * v.ns * v.max_bands * v.MT;
    const int total = v.nk * v.ns * nbands;
    double acc = 0.0;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int ks = e / nbands, band = e % nbands, k = ks / v.ns, s = ks % v.ns;
        const double w = v.wk[k] * f[(int64_t)ks * nbands + band];
        const double2* pr = v.p + ((int64_t)ks * v.max_bands + band) * v.MT + mo;
        const double2* qr = g + ((int64_t)ks * v.max_bands + band) * v.MT + mo;
        const double2* Vm = v.V + vo + (int64_t)s * M * M;
        double part = 0.0;
        for (int x = 0; x < M; ++x)
            for (int y = 0; y < M; ++y) {
                const double2 px = pr[x], py = pr[y], qx = qr[x], qy = qr[y], V = Vm[x * M + y];
                // z = conj(q_x) p_y - conj(p_x) q_y ;  Im(V z)
                const double zr = qx.x * py.x + qx.y * py.y - px.x * qy.x - px.y * qy.y;
                const double zi = qx.x * py.y - qx.y * py.x - px.x * qy.y + px.y * qy.x;
                part += V.x * zi + V.y * zr;
            }
        acc += w * part;
    }
    __shared__ double red[CTA];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) Jat[atom * 3 + dir] = ((v.ns == 1) ? 2.0 : 1.0) * red[0];
}

cudaError_t launch_current(const View& v, const double* f, int nbands, double* Jat, cudaStream_t st) {
    k_current<<<dim3(v.natoms, 3), CTA, 0, st>>>(v, f, nbands, Jat);
    return cudaGetLastError();
}

}  // namespace dftu
