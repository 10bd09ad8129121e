// Occupations (Eq. 4), renormalised occupations (Eqs. 8-9), ACBN0 U and J (Eqs. 10-11, B5-B6),
// Dudarev energy (Eqs. 3, A5) and the Hubbard potential (Eq. 6).  All FP64, fixed summation order.
//
// Storage: rho = n^T, i.e. rho_{ab} = sum w f p_a conj(p_b) (a, b = m, or c*M+m for spinors).
// The paper's n_{ab} is rho_{ba}; the formulas below read it that way.
#include "dftu_internal.cuh"

namespace dftu {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }  // a conj(b)

// Eq. (9): Nbar per state = sum over atoms of the state's species-mates and m (and spinor components) of |p|^2.
// One warp per (state, species): the lanes stride over the state's row of projections (coalesced), keep
// the orbitals of that species, and the lane sums are added by a fixed butterfly.
__device__ __forceinline__ void nbar_warp(const View& v, int nbands, int64_t w) {
    const int rows = v.noncollinear ? v.nk : v.nk * v.ns;
    if (w >= (int64_t)rows * nbands * v.nspecies) return;   // uniform over the warp
    const int lane = threadIdx.x & 31;
    const int sp = (int)(w % v.nspecies);
    w /= v.nspecies;
    const int row = (int)(w / nbands), band = (int)(w % nbands);
    const int ncomp = v.noncollinear ? 2 : 1;
    double acc = 0.0;
    for (int c = 0; c < ncomp; ++c) {
        const int ks = v.noncollinear ? row * 2 + c : row;
        const double2* pr = v.p + ((int64_t)ks * v.max_bands + band) * v.MT;
        for (int j = lane; j < v.MT; j += 32)
            if (v.atom_species[v.orb_atom[j]] == sp) acc += pr[j].x * pr[j].x + pr[j].y * pr[j].y;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) v.nbar[((int64_t)row * v.max_bands + band) * v.nspecies + sp] = acc;
}

__global__ void k_nbar(View v, int nbands) { nbar_warp(v, nbands, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); }

__global__ void k_nbar_batch(const View* __restrict__ views, const ProjArgs* __restrict__ args) {
    nbar_warp(views[blockIdx.y], args[blockIdx.y].nbands, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
}

// Eqs. (4), (8), (A2), (B3).  The (k, band) sum of every (atom, spin channel) [collinear] or atom
// [non-collinear] is split over OCC_SPLIT CTAs.  In a CTA, thread (pair, slice) takes matrix element
// (a, b) over a strided subset of the CTA's (k, band) range; slices are added in order and the CTA
// stores its partial.  The CTA that finishes last (a counter per matrix, reset by that CTA) adds the
// OCC_SPLIT partials in order and writes rho and Pbar, so the result does not depend on scheduling.
__device__ __forceinline__ void occupations_block(const View& v, const double* __restrict__ f, int nbands, int a, int s,
                                                  int z) {
    const int M = v.atom_M[a], mo = v.atom_moff[a], sp = v.atom_species[a];
    const int D = v.noncollinear ? 2 * M : M;
    const int P = D * D;
    const int SL = max(1, (int)blockDim.x / P);
    const int pair = threadIdx.x % P, slice = threadIdx.x / P;
    const int ia = pair / D, ib = pair % D;
    __shared__ double2 red_r[CTA], red_p[CTA];
    __shared__ int s_last;
    const int total = v.nk * nbands;
    const int chunk = (total + OCC_SPLIT - 1) / OCC_SPLIT;
    const int kb0 = z * chunk, kb1 = min(total, kb0 + chunk);
    double2 r = make_double2(0.0, 0.0), pb = make_double2(0.0, 0.0);
    if (slice < SL) {
        for (int kb = kb0 + slice; kb < kb1; kb += SL) {
            int k = kb / nbands, band = kb % nbands;
            double2 pa, pbv;
            double w, nb;
            if (v.noncollinear) {
                int ca = ia / M, ma = ia % M, cb = ib / M, mb = ib % M;
                pa = v.p[((int64_t)(k * 2 + ca) * v.max_bands + band) * v.MT + mo + ma];
                pbv = v.p[((int64_t)(k * 2 + cb) * v.max_bands + band) * v.MT + mo + mb];
                w = v.wk[k] * f[(int64_t)k * nbands + band];
                nb = v.nbar[((int64_t)k * v.max_bands + band) * v.nspecies + sp];
            } else {
                int ks = k * v.ns + s;
                const double2* pr = v.p + ((int64_t)ks * v.max_bands + band) * v.MT + mo;
                pa = pr[ia];
                pbv = pr[ib];
                w = v.wk[k] * f[((int64_t)k * v.ns + s) * nbands + band];
                nb = v.nbar[((int64_t)ks * v.max_bands + band) * v.nspecies + sp];
            }
            double2 c = cmulc(pa, pbv);
            r.x += w * c.x; r.y += w * c.y;
            pb.x += w * nb * c.x; pb.y += w * nb * c.y;
        }
    }
    red_r[threadIdx.x] = r;
    red_p[threadIdx.x] = pb;
    __syncthreads();
    const int mat = a * 2 + s;
    double2* part = v.occ_part + ((int64_t)mat * OCC_SPLIT + z) * 2 * OCC_MAXP;
    if (slice == 0 && threadIdx.x < P) {
        for (int q = 1; q < SL; ++q) {
            double2 x = red_r[q * P + pair], y = red_p[q * P + pair];
            r.x += x.x; r.y += x.y; pb.x += y.x; pb.y += y.y;
        }
        part[pair] = r;
        part[OCC_MAXP + pair] = pb;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&v.occ_count[mat], 1) == OCC_SPLIT - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < P) {
        double2 rr = make_double2(0.0, 0.0), pp = make_double2(0.0, 0.0);
        for (int q = 0; q < OCC_SPLIT; ++q) {
            const double2* pq = v.occ_part + ((int64_t)mat * OCC_SPLIT + q) * 2 * OCC_MAXP;
            double2 x = __ldcg(pq + pair), y = __ldcg(pq + OCC_MAXP + pair);
            rr.x += x.x; rr.y += x.y; pp.x += y.x; pp.y += y.y;
        }
        int64_t o = v.atom_mat_off[a] + (int64_t)s * P + pair;
        v.rho[o] = rr;
        v.pbar[o] = pp;
    }
    if (threadIdx.x == 0) v.occ_count[mat] = 0;
}

__global__ void k_occupations(View v, const double* __restrict__ f, int nbands) {
    occupations_block(v, f, nbands, blockIdx.x, blockIdx.y, blockIdx.z);
}

__global__ void k_occupations_batch(const View* __restrict__ views, const ProjArgs* __restrict__ args, const double* const* f) {
    const View& v = views[blockIdx.z];
    const int s = blockIdx.y / OCC_SPLIT, z = blockIdx.y % OCC_SPLIT;
    if ((int)blockIdx.x >= v.natoms || s >= (v.noncollinear ? 1 : v.ns)) return;
    occupations_block(v, f[blockIdx.z], args[blockIdx.z].nbands, blockIdx.x, s, z);
}

__device__ __forceinline__ double warp_sum(double x) {
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

// Eqs. (10)-(11) [collinear/unpolarised] or (B5)-(B6) [non-collinear], then Eq. (3)/(A5) and Eq. (6).
// One warp per atom (atoms warp0, warp0 + nw, ...); sums are lane-strided then tree-reduced (fixed order).
__device__ __forceinline__ void acbn0_atoms(const View& v, int warp0, int nw) {
    const int lane = threadIdx.x & 31;
    for (int a = warp0; a < v.natoms; a += nw) {
        const int M = v.atom_M[a], sp = v.atom_species[a];
        const int64_t mo = v.atom_mat_off[a];
        const double* Vc = v.coul + v.species_coul_off[sp];
        const int M2 = M * M, M4 = M2 * M2;
        double U, J, num_u = 0.0, num_j = 0.0, den_u = 0.0, den_j = 0.0;
        const bool fixed = !isnan(v.fixU[a]);
        if (!v.noncollinear) {
            const int nchan = v.ns;   // stored channels; alpha = 0,1 maps to channel alpha % nchan
            // paper's Pbar^alpha_{xy} = stored pbar[alpha][y][x]
            if (!fixed) {
                for (int e = lane; e < M4; e += 32) {
                    int x = e / (M2 * M), y = (e / M2) % M, z = (e / M) % M, w = e % M;
                    double vxyzw = Vc[((x * M + y) * M + z) * M + w];
                    double vxwzy = Vc[((x * M + w) * M + z) * M + y];
                    double2 Pt1 = make_double2(0, 0), Pt2 = make_double2(0, 0);
                    for (int al = 0; al < 2; ++al) {
                        int c = al % nchan;
                        double2 p1 = v.pbar[mo + c * M2 + y * M + x], p2 = v.pbar[mo + c * M2 + w * M + z];
                        Pt1.x += p1.x; Pt1.y += p1.y; Pt2.x += p2.x; Pt2.y += p2.y;
                        num_j += (p1.x * p2.x - p1.y * p2.y) * vxwzy;
                    }
                    num_u += (Pt1.x * Pt2.x - Pt1.y * Pt2.y) * vxyzw;
                }
                num_u = warp_sum(num_u);
                num_j = warp_sum(num_j);
                double Nt[2] = {0, 0}, N2[2] = {0, 0};
                for (int al = 0; al < 2; ++al) {
                    int c = al % nchan;
                    for (int m = 0; m < M; ++m) {
                        double N = v.rho[mo + c * M2 + m * M + m].x;
                        Nt[al] += N;
                        N2[al] += N * N;
                    }
                }
                double same = (Nt[0] * Nt[0] - N2[0]) + (Nt[1] * Nt[1] - N2[1]);
                double opp = Nt[0] * Nt[1] + Nt[1] * Nt[0];
                den_u = same + opp;
                den_j = same;
            }
        } else {
            const int D = 2 * M;
            // paper's n^{st}_{xy} = stored rho[(t*M+y)][(s*M+x)]
            auto PB = [&](int s, int t, int x, int y) { return v.pbar[mo + (t * M + y) * D + (s * M + x)]; };
            auto NN = [&](int s, int t, int x) { return v.rho[mo + (t * M + x) * D + (s * M + x)]; };
            if (!fixed) {
                for (int e = lane; e < M4; e += 32) {
                    int x = e / (M2 * M), y = (e / M2) % M, z = (e / M) % M, w = e % M;
                    double vxyzw = Vc[((x * M + y) * M + z) * M + w];
                    double vxwzy = Vc[((x * M + w) * M + z) * M + y];
                    double2 d1 = make_double2(0, 0), d2 = make_double2(0, 0);
                    for (int s = 0; s < 2; ++s) {
                        double2 q1 = PB(s, s, x, y), q2 = PB(s, s, z, w);
                        d1.x += q1.x; d1.y += q1.y; d2.x += q2.x; d2.y += q2.y;
                        for (int t = 0; t < 2; ++t) {
                            double2 r1 = PB(s, t, x, y), r2 = PB(t, s, z, w);
                            num_j += (r1.x * r2.x - r1.y * r2.y) * vxwzy;
                        }
                    }
                    num_u += (d1.x * d2.x - d1.y * d2.y) * vxyzw;
                }
                num_u = warp_sum(num_u);
                num_j = warp_sum(num_j);
                for (int s = 0; s < 2; ++s) {
                    int o = 1 - s;
                    for (int x = 0; x < M; ++x)
                        for (int y = 0; y < M; ++y) {
                            double2 ss_x = NN(s, s, x), ss_y = NN(s, s, y), oo_y = NN(o, o, y);
                            double2 so_x = NN(s, o, x), os_y = NN(o, s, y);
                            den_u += ss_x.x * oo_y.x - ss_x.y * oo_y.y;
                            if (x != y) {
                                double nss = ss_x.x * ss_y.x - ss_x.y * ss_y.y;
                                den_u += nss;
                                den_j += nss + (so_x.x * os_y.x - so_x.y * os_y.y);
                            }
                        }
                    for (int x = 0; x < M; ++x) {
                        double2 so = NN(s, o, x), os = NN(o, s, x);
                        den_u -= so.x * os.x - so.y * os.y;
                    }
                }
            }
        }
        bool zero = false;
        if (fixed) {
            U = v.fixU[a];
            J = v.fixJ[a];
        } else if (fabs(den_u) < 1e-14 || fabs(den_j) < 1e-14) {
            U = 0.0; J = 0.0; zero = true;
        } else {
            U = num_u / den_u;
            J = num_j / den_j;
        }
        const double Ue = U - J;
        // Energy (Eq. 3 / A5): U_eff/2 sum_blocks (Tr n - Tr n^2); potential (Eq. 6): U_eff (1/2 - rho)
        const int D = v.noncollinear ? 2 * M : M;
        const int nblk = v.noncollinear ? 1 : v.ns;
        double tr = 0.0;
        for (int b = 0; b < nblk; ++b) {
            const double2* R = v.rho + mo + (int64_t)b * D * D;
            double part = 0.0;
            for (int e = lane; e < D * D; e += 32) {
                int x = e / D, y = e % D;
                double2 rxy = R[x * D + y], ryx = R[y * D + x];
                part -= rxy.x * ryx.x - rxy.y * ryx.y;
                if (x == y) part += rxy.x;
                double2 Vv = make_double2(Ue * ((x == y ? 0.5 : 0.0) - rxy.x), -Ue * rxy.y);
                v.V[mo + (int64_t)b * D * D + e] = Vv;
            }
            tr += warp_sum(part);
        }
        if (!v.noncollinear && v.ns == 1) tr *= 2.0;
        if (lane == 0) {
            v.U[a] = U;
            v.J[a] = J;
            v.E[a] = 0.5 * Ue * tr;
            if (zero) atomicOr(v.status, ST_ZERO_DENOM);
        }
    }
}

// E_U summed over atoms in atom order.
__device__ __forceinline__ void energy_total(const View& v) {
    double s = 0.0;
    for (int a = 0; a < v.natoms; ++a) s += v.E[a];
    v.Etot[0] = s;
}

constexpr int ACBN0_WARPS = 4;   // atoms per CTA of k_acbn0 (one warp each)

__global__ void __launch_bounds__(32 * ACBN0_WARPS) k_acbn0(View v) {
    acbn0_atoms(v, blockIdx.x * ACBN0_WARPS + (threadIdx.x >> 5), gridDim.x * ACBN0_WARPS);
}

__global__ void k_energy_total(View v) {
    if (threadIdx.x == 0) energy_total(v);
}

__global__ void __launch_bounds__(256) k_acbn0_batch(const View* __restrict__ views) {
    const View& v = views[blockIdx.x];
    acbn0_atoms(v, threadIdx.x >> 5, blockDim.x >> 5);
    __syncthreads();
    if (threadIdx.x == 0) energy_total(v);
}

// Hubbard forces (Sec. IV, state-gradient form, U_eff fixed): one CTA per (atom, direction),
// F = -sum_{blocks} sum_{ab} V_ab sum_{k,n} w f [conj(g_a) p_b + conj(p_a) g_b], g = <phi|d_i psi>.
__global__ void __launch_bounds__(CTA) k_forces(View v, const double* __restrict__ f, int nbands, double* __restrict__ F) {
    const int a = blockIdx.x, dir = blockIdx.y;
    const int M = v.atom_M[a], mo = v.atom_moff[a];
    const int64_t vo = v.atom_mat_off[a];
    const int64_t gstride = (int64_t)v.nk * v.ns * v.max_bands * v.MT;
    const double2* g = v.pgrad + dir * gstride;
    double acc = 0.0;
    if (!v.noncollinear) {
        const int total = v.nk * v.ns * nbands;
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            const int ks = e / nbands, band = e % nbands, k = ks / v.ns, s = ks % v.ns;
            const double w = v.wk[k] * f[(int64_t)ks * nbands + band];
            const double2* pr = v.p + ((int64_t)ks * v.max_bands + band) * v.MT + mo;
            const double2* gr = g + ((int64_t)ks * v.max_bands + band) * v.MT + mo;
            const double2* Vm = v.V + vo + (int64_t)s * M * M;
            double part = 0.0;
            for (int x = 0; x < M; ++x)
                for (int y = 0; y < M; ++y) {
                    double2 px = pr[x], py = pr[y], gx = gr[x], gy = gr[y], V = Vm[x * M + y];
                    // conj(g_x) p_y + conj(p_x) g_y
                    double re = gx.x * py.x + gx.y * py.y + px.x * gy.x + px.y * gy.y;
                    double im = gx.x * py.y - gx.y * py.x + px.x * gy.y - px.y * gy.x;
                    part += V.x * re - V.y * im;
                }
            acc += w * part;
        }
    } else {
        const int D = 2 * M;
        const int total = v.nk * nbands;
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            const int k = e / nbands, band = e % nbands;
            const double w = v.wk[k] * f[(int64_t)k * nbands + band];
            double part = 0.0;
            for (int x = 0; x < D; ++x)
                for (int y = 0; y < D; ++y) {
                    const int cx = x / M, mx = x % M, cy = y / M, my = y % M;
                    double2 px = v.p[((int64_t)(k * 2 + cx) * v.max_bands + band) * v.MT + mo + mx];
                    double2 py = v.p[((int64_t)(k * 2 + cy) * v.max_bands + band) * v.MT + mo + my];
                    double2 gx = g[((int64_t)(k * 2 + cx) * v.max_bands + band) * v.MT + mo + mx];
                    double2 gy = g[((int64_t)(k * 2 + cy) * v.max_bands + band) * v.MT + mo + my];
                    double2 V = v.V[vo + x * D + y];
                    double re = gx.x * py.x + gx.y * py.y + px.x * gy.x + px.y * gy.y;
                    double im = gx.x * py.y - gx.y * py.x + px.x * gy.y - px.y * gy.x;
                    part += V.x * re - V.y * im;
                }
            acc += w * part;
        }
    }
    __shared__ double red[CTA];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) F[a * 3 + dir] = -((!v.noncollinear && v.ns == 1) ? 2.0 : 1.0) * red[0];
}

cudaError_t launch_forces(const View& v, const double* f, int nbands, double* F, cudaStream_t st) {
    k_forces<<<dim3(v.natoms, 3), CTA, 0, st>>>(v, f, nbands, F);
    return cudaGetLastError();
}

// Fully-localised-limit decomposition of App. A for each atom: E_ee of Eq. (A1), evaluated on the
// orbital-diagonal entries n^{st}_mm (the form the paper prints), and the double counting E_DC of
// Eq. (A3) with N = Tr n and the moment m_i = Tr_s(sigma_i Tr_l n).  One thread per atom, FP64.
// out[atom] = (E_ee, E_DC).
__global__ void k_fll(View v, double2* __restrict__ out) {
    const int a = blockIdx.x;
    if (threadIdx.x != 0) return;
    const int M = v.atom_M[a];
    const double2* r = v.rho + v.atom_mat_off[a];
    const double2 zero = make_double2(0.0, 0.0);
    double2 d[2][2][MAXM];
    for (int s = 0; s < 2; ++s)
        for (int t = 0; t < 2; ++t)
            for (int m = 0; m < M; ++m) {
                if (v.noncollinear) d[s][t][m] = r[(t * M + m) * (2 * M) + s * M + m];   // rho = n^T
                else d[s][t][m] = (s == t) ? r[(v.ns == 2 ? s : 0) * M * M + m * M + m] : zero;
            }
    double2 tr[2][2];
    for (int s = 0; s < 2; ++s)
        for (int t = 0; t < 2; ++t) {
            double2 x = zero;
            for (int m = 0; m < M; ++m) { x.x += d[s][t][m].x; x.y += d[s][t][m].y; }
            tr[s][t] = x;
        }
    auto re_mul = [](double2 x, double2 y) { return x.x * y.x - x.y * y.y; };
    const double U = v.U[a], J = v.J[a];
    double ee = 0.0;
    for (int s = 0; s < 2; ++s) {
        const int o = 1 - s;
        double flip = 0.0, same = 0.0;
        for (int m = 0; m < M; ++m) {
            flip += re_mul(d[s][o][m], d[o][s][m]);
            same += re_mul(d[s][s][m], d[s][s][m]);
        }
        ee += 0.5 * U * re_mul(tr[s][s], tr[o][o]);
        ee -= 0.5 * U * flip;
        ee -= 0.5 * J * (re_mul(tr[s][o], tr[o][s]) - flip);
        ee += 0.5 * (U - J) * (re_mul(tr[s][s], tr[s][s]) - same);
    }
    // m_x = rho_10 + rho_01, m_y = i (rho_01 - rho_10), m_z = rho_00 - rho_11 (rho = Tr_l n, [s][s'])
    const double2 mx = make_double2(tr[1][0].x + tr[0][1].x, tr[1][0].y + tr[0][1].y);
    const double2 my = make_double2(-(tr[0][1].y - tr[1][0].y), tr[0][1].x - tr[1][0].x);
    const double2 mz = make_double2(tr[0][0].x - tr[1][1].x, tr[0][0].y - tr[1][1].y);
    const double mm = re_mul(mx, mx) + re_mul(my, my) + re_mul(mz, mz);
    const double N = tr[0][0].x + tr[1][1].x;
    const double dc = 0.5 * U * N * (N - 1.0) - 0.5 * J * N * (0.5 * N - 1.0) - 0.25 * J * mm;
    out[a] = make_double2(ee, dc);
}

cudaError_t launch_fll(const View& v, double* out, cudaStream_t st) {
    k_fll<<<v.natoms, 32, 0, st>>>(v, reinterpret_cast<double2*>(out));
    return cudaGetLastError();
}

cudaError_t launch_nbar(const View& v, int nbands, cudaStream_t st) {
    int rows = v.noncollinear ? v.nk : v.nk * v.ns;
    int64_t n = (int64_t)rows * nbands * v.nspecies;   // warps, 8 per CTA
    k_nbar<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(v, nbands);
    return cudaGetLastError();
}

cudaError_t launch_occupations(const View& v, const double* f, int nbands, cudaStream_t st) {
    dim3 grid(v.natoms, v.noncollinear ? 1 : v.ns, OCC_SPLIT);
    k_occupations<<<grid, CTA, 0, st>>>(v, f, nbands);
    return cudaGetLastError();
}

cudaError_t launch_acbn0(const View& v, cudaStream_t st) {
    k_acbn0<<<(v.natoms + ACBN0_WARPS - 1) / ACBN0_WARPS, 32 * ACBN0_WARPS, 0, st>>>(v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_energy_total<<<1, 32, 0, st>>>(v);
    return cudaGetLastError();
}

cudaError_t launch_occupations_batch(const BatchLaunch& b, cudaStream_t st) {
    dim3 g1((unsigned)((b.max_rows_nbar + 7) / 8), b.nsys);   // one warp per (state, species), 8 per CTA
    k_nbar_batch<<<g1, 256, 0, st>>>(b.views, b.args);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g2(b.max_atoms, b.max_ns * OCC_SPLIT, b.nsys);
    k_occupations_batch<<<g2, CTA, 0, st>>>(b.views, b.args, b.f);
    return cudaGetLastError();
}

cudaError_t launch_acbn0_batch(const BatchLaunch& b, cudaStream_t st) {
    k_acbn0_batch<<<b.nsys, 256, 0, st>>>(b.views);
    return cudaGetLastError();
}

}  // namespace dftu
