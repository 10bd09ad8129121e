// Real-time step with the Hubbard term (Sec. V, Eq. 15) carried out in the span of the orbitals.
//
// V_U maps every state into the span of the scattered orbitals: V_U x = scatter(V p(x)), where p(x) are
// the projections (gather) and scatter(a) = sum_{I,m} a_Im exp(-i k.T) phi_Im on the sphere points.  A
// Taylor term term_j = c_j V_U term_{j-1} (c_j = -i dt / j) is therefore scatter(a_j), and its
// projections are p(term_j) = O a_j with O the overlap of the gathered with the scattered orbitals:
//   O_{Im,Jm'} = dV sum over point pairs (a of atom I, b of atom J) on the same grid point of
//                phi_Im(a) phi_Jm'(b) exp(+i k.(T_a - T_b) L)      [times exp(+i A.(d_a - d_b)), Eq. 16]
// (the identity on each atom's own points after the Loewdin step of Sec. III, plus the blocks of
// overlapping spheres and of spheres overlapping their own images).  So with p_0 = p(psi):
//   a_j = c_j V p_{j-1},  p_j = O a_j,  psi <- psi + scatter(sum_j a_j),
// the same polynomial in V_U as the grid form, applied with one gather and one scatter of the states.
#include "dftu_internal.cuh"

namespace dftu {

// exp(+i k.D_b), times exp(+i A.Dg_b) when the gauge phases are on, for every (k, block).
__global__ void k_block_phases(View v, int gauge) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= v.nk * v.nblk) return;
    const int k = g / v.nblk, b = g - k * v.nblk;
    const double* kv = v.kvec + 3 * k;
    const double* D = v.blk_D + 3 * b;
    double th = fma(kv[2], D[2], fma(kv[1], D[1], kv[0] * D[0]));
    if (gauge) {
        const double* Dg = v.blk_Dg + 3 * b;
        th += fma(v.gaugeA[2], Dg[2], fma(v.gaugeA[1], Dg[1], v.gaugeA[0] * Dg[0]));
    }
    double s, c;
    sincos(th, &s, &c);
    v.blk_phase[g] = make_double2(c, s);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// One CTA per state (k, spin, band; non-collinear: k, band with both components).  Vectors live in
// global memory: X = p_{j-1} (scratch), W = V p_{j-1} (scratch), cv = sum_j a_j.
__global__ void __launch_bounds__(128) k_taylor_cv(View v, int nbands, int order, const double2* __restrict__ coefs,
                                                  double2* __restrict__ X, double2* __restrict__ W) {
    const int ncomp = v.noncollinear ? 2 : 1;
    const int row = blockIdx.x;
    int k, s0, band;
    if (v.noncollinear) {
        k = row / nbands; band = row - k * nbands; s0 = 0;
    } else {
        const int ks = row / nbands;
        band = row - ks * nbands; k = ks / v.ns; s0 = ks - k * v.ns;
    }
    const int nel = ncomp * v.MT;
    // row of vector component c (spin channel of a collinear state, spinor component otherwise)
    auto vrow = [&](int c) -> int64_t {
        const int r = v.noncollinear ? k * 2 + c : k * v.ns + s0;
        return ((int64_t)r * v.max_bands + band) * v.MT;
    };
    for (int jt = 1; jt <= order; ++jt) {
        const double2 cj = coefs[jt - 1];
        const double2* xin = (jt == 1) ? v.p : X;
        // W = V x; cv (+)= c_j W
        for (int e = threadIdx.x; e < nel; e += blockDim.x) {
            const int c = e / v.MT, j = e - c * v.MT;
            const int a = v.orb_atom[j];
            const int M = v.atom_M[a], mo = v.atom_moff[a], m = j - mo;
            const int64_t vo = v.atom_mat_off[a];
            double re = 0.0, im = 0.0;
            if (!v.noncollinear) {
                const double2* Vm = v.V + vo + (int64_t)s0 * M * M + m * M;
                const double2* pr = xin + vrow(0) + mo;
                for (int qq = 0; qq < M; ++qq) {   // four fused multiply-adds per complex product
                    const double2 A = Vm[qq], B = pr[qq];
                    re = fma(A.x, B.x, fma(-A.y, B.y, re));
                    im = fma(A.x, B.y, fma(A.y, B.x, im));
                }
            } else {
                const double2* Vm = v.V + vo + (int64_t)(c * M + m) * (2 * M);
                for (int c2 = 0; c2 < 2; ++c2) {
                    const double2* pr = xin + vrow(c2) + mo;
                    for (int qq = 0; qq < M; ++qq) {
                        const double2 A = Vm[c2 * M + qq], B = pr[qq];
                        re = fma(A.x, B.x, fma(-A.y, B.y, re));
                        im = fma(A.x, B.y, fma(A.y, B.x, im));
                    }
                }
            }
            const int64_t o = vrow(c) + j;
            const double2 w = make_double2(re, im);
            W[o] = w;
            const double2 t = cmul(cj, w);
            v.cv[o] = (jt == 1) ? t : make_double2(v.cv[o].x + t.x, v.cv[o].y + t.y);
        }
        __syncthreads();
        if (jt < order) {
            // X = c_j O W
            for (int e = threadIdx.x; e < nel; e += blockDim.x) {
                const int c = e / v.MT, j = e - c * v.MT;
                const int I = v.orb_atom[j];
                const int m = j - v.atom_moff[I];
                const double2* wr = W + vrow(c);
                double re = 0.0, im = 0.0;
                for (int b = v.blk_rowptr[I]; b < v.blk_rowptr[I + 1]; ++b) {
                    const int J = v.blk_J[b];
                    const int MJ = v.atom_M[J], moJ = v.atom_moff[J];
                    const double* B = v.blk_data + v.blk_off[b] + (int64_t)m * MJ;
                    double tr = 0.0, ti = 0.0;
                    for (int q = 0; q < MJ; ++q) {
                        const double2 x = wr[moJ + q];
                        tr = fma(B[q], x.x, tr);
                        ti = fma(B[q], x.y, ti);
                    }
                    const double2 ph = v.blk_phase[k * v.nblk + b];
                    re = fma(ph.x, tr, fma(-ph.y, ti, re));
                    im = fma(ph.x, ti, fma(ph.y, tr, im));
                }
                X[vrow(c) + j] = cmul(cj, make_double2(re, im));
            }
            __syncthreads();
        }
    }
}

cudaError_t launch_taylor_cv(const View& v, int nbands, int order, const double* coefs, bool gauge, cudaStream_t st) {
    if (v.nblk > 0) {
        const int n = v.nk * v.nblk;
        k_block_phases<<<(n + 127) / 128, 128, 0, st>>>(v, gauge ? 1 : 0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int rows = (v.noncollinear ? v.nk : v.nk * v.ns) * nbands;
    const int64_t slice = (int64_t)v.nk * v.ns * v.max_bands * v.MT;   // one slice of the gradient-projection buffer
    k_taylor_cv<<<rows, 128, 0, st>>>(v, nbands, order, reinterpret_cast<const double2*>(coefs), v.pgrad, v.pgrad + slice);
    return cudaGetLastError();
}

}  // namespace dftu
