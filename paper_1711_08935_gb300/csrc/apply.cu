// Hubbard operator applied back onto the states (Eq. 6):
//   psi(idx_j) += c * exp(-i k.T_j) * sum_m phi_m(j) (V p)_m
// One CTA per (tile, band chunk, k*spin-or-component).  The CTA first forms the coefficients
// c_{band,m} = c * conj(phase_tile) * (V p)_m for its bands (FP64), then every lane group of Q
// lanes read-modify-writes its band's points.  Tiles are launched colour by colour: tiles of one
// colour touch disjoint grid points, so a point shared by several spheres (or by periodic images
// of one sphere) is updated by successive launches in a fixed order, without atomics.
#include "dftu_internal.cuh"

namespace dftu {

struct ApplyArgs {
    void* psi;
    int64_t sk, ss, sn;
    int nbands;
    const double* coef;   // device complex, never null (the handle supplies 1)
    const int* tile_list;  // tiles of this colour
};

enum APol { A_F64 = 0, A_PAIR = 1, A_F32 = 2 };

// (hi, lo) float split of a double (round-to-nearest hi, exact-ish remainder) -- used only for the
// per-CTA coefficients, so the FP64 conversion cost is negligible.
__device__ __forceinline__ void dsplit(double x, float& h, float& l) {
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
}

// Exact float -> double by bit manipulation (the FP32->FP64 conversion instruction runs on the slow
// FP64 path of this GPU).  Zeros and FP32 denormals give 0.
__device__ __forceinline__ double f2d_bits(float f) {
    unsigned u = __float_as_uint(f);
    unsigned e = (u >> 23) & 0xFFu;
    unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    unsigned lo = u << 29;
    return e == 0 ? 0.0 : __hiloint2double((int)hi, (int)lo);
}

template <int POL, int Q, int M>
__device__ __forceinline__ void apply_body(const Tile& t, const ApplyArgs& a, int64_t off, int q, int bl, const int* s_idx,
                                           const unsigned char* after_idx, const unsigned char* after_c) {
    if (POL == A_F64) {
        double2* row = reinterpret_cast<double2*>(a.psi) + off;
        const double* s_phi = reinterpret_cast<const double*>(after_c);
        const double2* s_c = reinterpret_cast<const double2*>(after_idx);
        double2 cc[M];
#pragma unroll
        for (int m = 0; m < M; ++m) cc[m] = s_c[bl * MAXM + m];
        for (int i = q; i < t.np; i += Q) {
            int idx = s_idx[i];
            double2 x = row[idx];
            const double* ph = s_phi + i * M;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                x.x = fma(ph[m], cc[m].x, x.x);
                x.y = fma(ph[m], cc[m].y, x.y);
            }
            row[idx] = x;
        }
    } else if (POL == A_PAIR) {
        // delta = sum_m phi_m c_m as a float pair (TwoProd of the leading products, TwoSum of the
        // running sum, FP32 corrections), then psi + delta with two FP64 additions per component.
        double2* row = reinterpret_cast<double2*>(a.psi) + off;
        const float2* s_phi = reinterpret_cast<const float2*>(after_c);
        const float4* s_c = reinterpret_cast<const float4*>(after_idx);
        float2 ch[M], cl[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            float4 c4 = s_c[bl * MAXM + m];
            ch[m] = make_float2(c4.x, c4.y);
            cl[m] = make_float2(c4.z, c4.w);
        }
        for (int i = q; i < t.np; i += Q) {
            int idx = s_idx[i];
            double2 x = row[idx];
            const float2* ph = s_phi + i * M;
            float2 sh = make_float2(0.f, 0.f), sl = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                float2 f = ph[m];
                float2 fh = make_float2(f.x, f.x), fl = make_float2(f.y, f.y);
                float2 pr = __fmul2_rn(fh, ch[m]);
                float2 pe = __ffma2_rn(fh, ch[m], make_float2(-pr.x, -pr.y));   // exact product error
                float2 s2 = __fadd2_rn(sh, pr);                                   // TwoSum(sh, pr)
                float2 bb = __fadd2_rn(s2, make_float2(-sh.x, -sh.y));
                float2 e = __fadd2_rn(__fadd2_rn(sh, make_float2(-(s2.x - bb.x), -(s2.y - bb.y))),
                                      __fadd2_rn(pr, make_float2(-bb.x, -bb.y)));
                sh = s2;
                sl = __fadd2_rn(sl, __fadd2_rn(e, pe));
                sl = __ffma2_rn(fh, cl[m], sl);
                sl = __ffma2_rn(fl, ch[m], sl);
            }
            x.x = (x.x + f2d_bits(sh.x)) + f2d_bits(sl.x);
            x.y = (x.y + f2d_bits(sh.y)) + f2d_bits(sl.y);
            row[idx] = x;
        }
    } else {
        float2* row = reinterpret_cast<float2*>(a.psi) + off;
        const float2* s_phi = reinterpret_cast<const float2*>(after_c);
        const float2* s_c = reinterpret_cast<const float2*>(after_idx);
        float2 cc[M];
#pragma unroll
        for (int m = 0; m < M; ++m) cc[m] = s_c[bl * MAXM + m];
        for (int i = q; i < t.np; i += Q) {
            int idx = s_idx[i];
            float2 x = row[idx];
            const float2* ph = s_phi + i * M;
#pragma unroll
            for (int m = 0; m < M; ++m) x = __ffma2_rn(make_float2(ph[m].x, ph[m].x), cc[m], x);
            row[idx] = x;
        }
    }
}

template <int POL, int Q>
__global__ void __launch_bounds__(CTA) k_apply(View v, ApplyArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    int* s_idx = reinterpret_cast<int*>(smem);
    constexpr int BPW = 32 / Q;
    constexpr int BPC = (CTA / 32) * BPW;
    const Tile t = v.tiles[a.tile_list[blockIdx.x]];
    const int ks = blockIdx.z;
    const int k = ks / v.ns, s = ks % v.ns;
    const int band0 = blockIdx.y * BPC;
    const int M = t.M;
    unsigned char* after_idx = smem + TILE * sizeof(int);
    // coefficient table [BPC][M] complex: FP64 (F64), (hi.re,hi.im,lo.re,lo.im) (PAIR), float2 (F32)
    double2* s_c64 = reinterpret_cast<double2*>(after_idx);
    float4* s_c4 = reinterpret_cast<float4*>(after_idx);
    float2* s_c32 = reinterpret_cast<float2*>(after_idx);
    unsigned char* after_c = after_idx + BPC * MAXM * sizeof(double2);

    for (int i = threadIdx.x; i < TILE; i += CTA) s_idx[i] = (i < t.np) ? v.pt_idx[t.p0 + i] : 0;
    if (threadIdx.x < BPC * M) {
        int bl = threadIdx.x / M, m = threadIdx.x % M;
        int band = band0 + bl;
        double2 c = make_double2(0.0, 0.0);
        if (band < a.nbands) {
            const int mo = v.atom_moff[t.atom];
            const int64_t vo = v.atom_mat_off[t.atom];
            double re = 0.0, im = 0.0;
            if (!v.noncollinear) {
                const double2* Vm = v.V + vo + (int64_t)s * M * M + m * M;
                const double2* pr = v.p + ((int64_t)ks * v.max_bands + band) * v.MT + mo;
                for (int q = 0; q < M; ++q) {
                    double2 A = Vm[q], B = pr[q];
                    re += A.x * B.x - A.y * B.y;
                    im += A.x * B.y + A.y * B.x;
                }
            } else {
                const int D = 2 * M;
                const double2* Vm = v.V + vo + (int64_t)(s * M + m) * D;
                for (int c2 = 0; c2 < 2; ++c2) {
                    const double2* pr = v.p + ((int64_t)(k * 2 + c2) * v.max_bands + band) * v.MT + mo;
                    for (int q = 0; q < M; ++q) {
                        double2 A = Vm[c2 * M + q], B = pr[q];
                        re += A.x * B.x - A.y * B.y;
                        im += A.x * B.y + A.y * B.x;
                    }
                }
            }
            double2 ph = v.seg_phase[t.seg * v.nk + k];   // exp(+ikT); the scatter uses its conjugate
            double2 cf = *reinterpret_cast<const double2*>(a.coef);
            double2 pc = make_double2(cf.x * ph.x + cf.y * ph.y, cf.y * ph.x - cf.x * ph.y);   // cf * conj(ph)
            c = make_double2(pc.x * re - pc.y * im, pc.x * im + pc.y * re);
        }
        if (POL == A_F64) s_c64[bl * MAXM + m] = c;
        else if (POL == A_PAIR) {
            float hr, lr, hi, li;
            dsplit(c.x, hr, lr);
            dsplit(c.y, hi, li);
            s_c4[bl * MAXM + m] = make_float4(hr, hi, lr, li);
        } else s_c32[bl * MAXM + m] = make_float2((float)c.x, (float)c.y);
    }
    if (POL == A_F64) {
        double* s_phi = reinterpret_cast<double*>(after_c);
        for (int e = threadIdx.x; e < TILE * M; e += CTA) s_phi[e] = (e < t.np * M) ? v.phi64[t.phi0 + e] : 0.0;
    } else {
        float2* s_phi = reinterpret_cast<float2*>(after_c);
        for (int e = threadIdx.x; e < TILE * M; e += CTA)
            s_phi[e] = (e < t.np * M) ? make_float2(v.phi_hi[t.phi0 + e], v.phi_lo[t.phi0 + e]) : make_float2(0.f, 0.f);
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int bl = (threadIdx.x >> 5) * BPW + lane / Q;
    const int q = lane & (Q - 1);
    const int band = band0 + bl;
    if (band >= a.nbands) return;
    const int64_t off = (int64_t)k * a.sk + (int64_t)s * a.ss + (int64_t)band * a.sn;
    switch (M) {
        case 1: apply_body<POL, Q, 1>(t, a, off, q, bl, s_idx, after_idx, after_c); break;
        case 3: apply_body<POL, Q, 3>(t, a, off, q, bl, s_idx, after_idx, after_c); break;
        case 5: apply_body<POL, Q, 5>(t, a, off, q, bl, s_idx, after_idx, after_c); break;
        default: apply_body<POL, Q, 7>(t, a, off, q, bl, s_idx, after_idx, after_c); break;
    }
}

template <int POL, int Q>
static cudaError_t run_apply(const View& v, ApplyArgs a, const int* color_order, const std::vector<int>& color_beg,
                             cudaStream_t st) {
    constexpr int BPC = (CTA / 32) * (32 / Q);
    size_t smem = TILE * sizeof(int) + BPC * MAXM * sizeof(double2) +
                  (size_t)TILE * MAXM * (POL == A_F64 ? sizeof(double) : sizeof(float2));
    cudaError_t e = cudaFuncSetAttribute(k_apply<POL, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (size_t c = 0; c + 1 < color_beg.size(); ++c) {
        int n = color_beg[c + 1] - color_beg[c];
        if (n == 0) continue;
        a.tile_list = color_order + color_beg[c];
        dim3 grid(n, (a.nbands + BPC - 1) / BPC, v.nk * v.ns);
        k_apply<POL, Q><<<grid, CTA, smem, st>>>(v, a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_apply(const View& v, void* psi, dftu_prec prec, dftu_f64_mode mode, int nbands,
                         int64_t sk, int64_t ss, int64_t sn, const double* coef, const int* color_order,
                         const std::vector<int>& color_beg, cudaStream_t st) {
    ApplyArgs a{psi, sk, ss, sn, nbands, coef, nullptr};
    if (prec == DFTU_C64) return run_apply<A_F32, 16>(v, a, color_order, color_beg, st);
    if (mode == DFTU_F64_NATIVE) return run_apply<A_F64, 8>(v, a, color_order, color_beg, st);
    return run_apply<A_PAIR, 8>(v, a, color_order, color_beg, st);
}

}  // namespace dftu
