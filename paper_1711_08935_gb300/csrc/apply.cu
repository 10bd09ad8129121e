// Hubbard operator applied back onto the states (Eq. 6):
//   psi(idx_j) += c * exp(-i k.T_j) * sum_m phi_m(j) (V p)_m
// One CTA per (tile, band chunk, k*spin-or-component).  The CTA first forms the coefficients
// c_{band,m} = c * conj(phase_tile) * (V p)_m for its bands (FP64), then every lane group of Q
// lanes read-modify-writes its band's points.  Tiles are launched colour by colour: tiles of one
// colour touch disjoint grid points, so a point shared by several spheres (or by periodic images
// of one sphere) is updated by successive launches in a fixed order, without atomics.
#include <algorithm>

#include "dftu_internal.cuh"

namespace dftu {

struct ApplyArgs {
    void* psi;
    int64_t sk, ss, sn;
    int nbands;
    const double* coef;   // device complex, never null (the handle supplies 1)
    const int* tile_list;  // tiles of this colour
    int accumulate;        // 1: psi += c V_U psi_proj ; 0: psi = c V_U psi_proj on the sphere points
};

// A_F32P: complex64, paired orbital rows.  A_F32PJ: the same apply, which also projects the updated values
// of a final tile (Tile_final) onto its orbitals: the gather of the next real-time step fused into this
// step's scatter (dftu_taylor_steps).
enum APol { A_F64 = 0, A_PAIR = 1, A_F32 = 2, A_F32P = 3, A_F32PJ = 4 };

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

__device__ __forceinline__ float pow2f(int e) { return e < -126 ? 0.0f : __int_as_float((e + 127) << 23); }

__device__ __forceinline__ int exp_field_d(double x) { return (__double2hiint(x) >> 20) & 0x7FF; }

// Nearest double to (h + l) * 2^sc for a normalised float pair (|l| <= ulp(h)/2), assembled with
// integer operations: the bit pattern of h as a double plus l counted in units of that double's ulp
// (half-ulps when h is a power of two and l points toward zero).
__device__ __forceinline__ double pair_to_double(float h, float l, int sc) {
    unsigned u = __float_as_uint(h);
    int e = (u >> 23) & 0xFF;
    if (e == 0) return 0.0;
    unsigned hi = (u & 0x80000000u) | ((unsigned)(e + 896 + sc) << 20) | ((u & 0x7FFFFFu) >> 3);
    unsigned lo = u << 29;
    unsigned lu = __float_as_uint(l);
    int el = (lu >> 23) & 0xFF;
    // t = l * 2^(179 - e): exponent-field add (|t| <= 2^28, no overflow); sign flipped to magnitude direction
    unsigned tb = (lu + ((unsigned)(179 - e) << 23)) ^ (u & 0x80000000u);
    float tm = (el == 0) ? 0.0f : __uint_as_float(tb);
    if ((u & 0x7FFFFFu) == 0 && tm < 0.0f) tm *= 2.0f;
    long long K = (long long)__float2int_rn(tm);
    unsigned long long D = (((unsigned long long)hi << 32) | lo) + (unsigned long long)K;
    return __longlong_as_double((long long)D);
}

// (bh + bl) * (g.x + g.z + i (g.y + g.w)) componentwise as a new float pair (exact hi products, TwoSum,
// cross terms with the low parts in the low word), renormalised with TwoSum so that |lo| <= ulp(hi)/2.
__device__ __forceinline__ void rot_pair_norm(float2& bh, float2& bl, float4 g) {
    const float2 uh = make_float2(g.x, g.y), wh = make_float2(-g.y, g.x);
    const float2 ul = make_float2(g.z, g.w), wl = make_float2(-g.w, g.z);
    const float2 xr = make_float2(bh.x, bh.x), xi = make_float2(bh.y, bh.y);
    const float2 P = __fmul2_rn(uh, xr), R = __fmul2_rn(wh, xi);
    const float2 eP = __ffma2_rn(uh, xr, make_float2(-P.x, -P.y));
    const float2 eR = __ffma2_rn(wh, xi, make_float2(-R.x, -R.y));
    float2 s = __fadd2_rn(P, R);
    float2 bb = __fadd2_rn(s, make_float2(-P.x, -P.y));
    float2 t = __fadd2_rn(__fadd2_rn(P, make_float2(bb.x - s.x, bb.y - s.y)), __fadd2_rn(R, make_float2(-bb.x, -bb.y)));
    float2 lo = __fadd2_rn(__fadd2_rn(eP, eR), t);
    lo = __ffma2_rn(uh, make_float2(bl.x, bl.x), lo);
    lo = __ffma2_rn(ul, xr, lo);
    lo = __ffma2_rn(wh, make_float2(bl.y, bl.y), lo);
    lo = __ffma2_rn(wl, xi, lo);
    const float2 h = __fadd2_rn(s, lo);   // TwoSum(s, lo)
    bb = __fadd2_rn(h, make_float2(-s.x, -s.y));
    bl = __fadd2_rn(__fadd2_rn(s, make_float2(bb.x - h.x, bb.y - h.y)), __fadd2_rn(lo, make_float2(-bb.x, -bb.y)));
    bh = h;
}

// Each lane handles U points of its band at a time: U loads in flight, then the arithmetic, then U
// stores (the points of one tile are distinct grid points, so the batch never aliases).  Orbital rows
// up to Q*U past the tile are staged as zeros, so the arithmetic needs no bounds test.
// With G, the update of point j is multiplied by exp(-i A.d_j) (the gauge phase table in s_gauge).
template <int POL, int Q, int M, int U, int PF, int G>
__device__ __forceinline__ void apply_body(const Tile& t, const ApplyArgs& a, int64_t off, int q, int bl, const int* s_idx,
                                           const unsigned char* s_first, const unsigned char* after_idx,
                                           const unsigned char* after_c, int pe, const unsigned char* s_gauge) {
    if (POL == A_F64) {
        double2* row = reinterpret_cast<double2*>(a.psi) + off;
        const double* s_phi = reinterpret_cast<const double*>(after_c);
        const double2* s_c = reinterpret_cast<const double2*>(after_idx);
        double2 cc[M];
#pragma unroll
        for (int m = 0; m < M; ++m) cc[m] = s_c[bl * MAXM + m];
        for (int i0 = q; i0 < t.np; i0 += Q * U) {
            double2 x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int i = i0 + u * Q;
                x[u] = (i < t.np && (a.accumulate || !s_first[i])) ? row[s_idx[i]] : make_double2(0.0, 0.0);
            }
            if (PF) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    int i = i0 + Q * U + u * Q;
                    if (i < t.np) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + s_idx[i]));
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const double* ph = s_phi + (i0 + u * Q) * M;
                if (G) {
                    double2 d = make_double2(0.0, 0.0);
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        d.x = fma(ph[m], cc[m].x, d.x);
                        d.y = fma(ph[m], cc[m].y, d.y);
                    }
                    const double2 g = reinterpret_cast<const double2*>(s_gauge)[i0 + u * Q];   // x += conj(g) d
                    x[u].x += fma(g.x, d.x, g.y * d.y);
                    x[u].y += fma(g.x, d.y, -g.y * d.x);
                } else {
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        x[u].x = fma(ph[m], cc[m].x, x[u].x);
                        x[u].y = fma(ph[m], cc[m].y, x[u].y);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int i = i0 + u * Q;
                if (i < t.np) row[s_idx[i]] = x[u];
            }
        }
    } else if (POL == A_PAIR) {
        // delta = sum_m phi_m c_m with the offset accumulator (C >= 4 sum|phi c|: every partial sum stays in
        // C's binade, so acc - s is exact and the rounding residual is caught in a second float), then the
        // pair is renormalised, assembled into the nearest double with integer operations, and added to psi
        // with one FP64 addition per component.
        double2* row = reinterpret_cast<double2*>(a.psi) + off;
        const float4* s_phi = reinterpret_cast<const float4*>(after_c);
        const float4* s_c = reinterpret_cast<const float4*>(after_idx);
        float2 ch[M], cl[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            float4 c4 = s_c[bl * MAXM + m];
            ch[m] = make_float2(c4.x, c4.y);
            cl[m] = make_float2(c4.z, c4.w);
        }
        int ce = -126;                                               // |c_hi| < 2^ce
#pragma unroll
        for (int m = 0; m < M; ++m)
            ce = max(ce, max((__float_as_int(ch[m].x) >> 23) & 0xFF, (__float_as_int(ch[m].y) >> 23) & 0xFF) - 126);
        const int ebound = min(max(pe + ce, -120), 120);          // |phi_hi c_hi| < 2^ebound
        // (the gauge rotation acts on the finished sum, so the accumulator bound is unchanged)
        const float Cv = pow2f(ebound + 5);
        const float2 C2 = make_float2(Cv, Cv), mone = make_float2(-1.f, -1.f);
        for (int i0 = q; i0 < t.np; i0 += Q * U) {
            double2 x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int i = i0 + u * Q;
                x[u] = (i < t.np && (a.accumulate || !s_first[i])) ? row[s_idx[i]] : make_double2(0.0, 0.0);
            }
            if (PF) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    int i = i0 + Q * U + u * Q;
                    if (i < t.np) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + s_idx[i]));
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float4* ph = s_phi + (i0 + u * Q) * M;
                float2 acc = C2, lo = make_float2(0.f, 0.f);
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    float4 f = ph[m];                                      // (hi, hi, lo, lo)
                    float2 fh = make_float2(f.x, f.y), fl = make_float2(f.z, f.w);
                    float2 sacc = __ffma2_rn(fh, ch[m], acc);
                    float2 tneg = __ffma2_rn(sacc, mone, acc);             // acc - sacc, exact
                    float2 r = __ffma2_rn(fh, ch[m], tneg);
                    lo = __fadd2_rn(lo, r);
                    lo = __ffma2_rn(fh, cl[m], lo);
                    lo = __ffma2_rn(fl, ch[m], lo);
                    acc = sacc;
                }
                float2 dh = __fadd2_rn(acc, make_float2(-Cv, -Cv));          // exact
                float2 hh = __fadd2_rn(dh, lo);                               // Fast2Sum: |lo| << |dh| or dh = 0
                float2 ll = __fadd2_rn(lo, make_float2(-(hh.x - dh.x), -(hh.y - dh.y)));
                if (G) {
                    const float4 g = reinterpret_cast<const float4*>(s_gauge)[i0 + u * Q];
                    rot_pair_norm(hh, ll, make_float4(g.x, -g.y, g.z, -g.w));   // times conj(g)
                }
                x[u].x += pair_to_double(hh.x, ll.x, 0);
                x[u].y += pair_to_double(hh.y, ll.y, 0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int i = i0 + u * Q;
                if (i < t.np) row[s_idx[i]] = x[u];
            }
        }
    } else if (POL == A_F32P) {
        // Orbital rows [hi_0 .. hi_{MP-1}] per point (MP = M rounded up to even, zero padded): one 8-byte
        // shared load feeds two orbitals, whose real and imaginary coefficients sit in float pairs.
        constexpr int MP = (M + 1) & ~1, NP = MP / 2;
        float2* row = reinterpret_cast<float2*>(a.psi) + off;
        const float* s_phf = reinterpret_cast<const float*>(after_c);
        const float2* s_c = reinterpret_cast<const float2*>(after_idx);
        float2 cre[NP], cim[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            const float2 c0 = s_c[bl * MAXM + 2 * j];
            const float2 c1 = (2 * j + 1 < M) ? s_c[bl * MAXM + 2 * j + 1] : make_float2(0.f, 0.f);
            cre[j] = make_float2(c0.x, c1.x);
            cim[j] = make_float2(c0.y, c1.y);
        }
        for (int i0 = q; i0 < t.np; i0 += Q * U) {
            float2 x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int i = i0 + u * Q;
                x[u] = (i < t.np && (a.accumulate || !s_first[i])) ? row[s_idx[i]] : make_float2(0.f, 0.f);
            }
            if (PF) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    int i = i0 + Q * U + u * Q;
                    if (i < t.np) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + s_idx[i]));
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float* ph = s_phf + (i0 + u * Q) * MP;
                float2 ar = make_float2(0.f, 0.f), ai = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    const float2 f2 = *reinterpret_cast<const float2*>(ph + 2 * j);
                    ar = __ffma2_rn(f2, cre[j], ar);
                    ai = __ffma2_rn(f2, cim[j], ai);
                }
                x[u] = __fadd2_rn(x[u], make_float2(ar.x + ar.y, ai.x + ai.y));
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int i = i0 + u * Q;
                if (i < t.np) row[s_idx[i]] = x[u];
            }
        }
    } else {
        float2* row = reinterpret_cast<float2*>(a.psi) + off;
        const float4* s_phi = reinterpret_cast<const float4*>(after_c);
        const float2* s_c = reinterpret_cast<const float2*>(after_idx);
        float2 cc[M];
#pragma unroll
        for (int m = 0; m < M; ++m) cc[m] = s_c[bl * MAXM + m];
        for (int i0 = q; i0 < t.np; i0 += Q * U) {
            float2 x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int i = i0 + u * Q;
                x[u] = (i < t.np && (a.accumulate || !s_first[i])) ? row[s_idx[i]] : make_float2(0.f, 0.f);
            }
            if (PF) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    int i = i0 + Q * U + u * Q;
                    if (i < t.np) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + s_idx[i]));
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float4* ph = s_phi + (i0 + u * Q) * M;
                if (G) {
                    float2 d = make_float2(0.f, 0.f);
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        float4 f = ph[m];
                        d = __ffma2_rn(make_float2(f.x, f.y), cc[m], d);
                    }
                    const float4 g = reinterpret_cast<const float4*>(s_gauge)[i0 + u * Q];   // x += conj(g) d
                    x[u] = __ffma2_rn(make_float2(g.x, -g.y), make_float2(d.x, d.x), x[u]);
                    x[u] = __ffma2_rn(make_float2(g.y, g.x), make_float2(d.y, d.y), x[u]);
                } else {
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        float4 f = ph[m];
                        x[u] = __ffma2_rn(make_float2(f.x, f.y), cc[m], x[u]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int i = i0 + u * Q;
                if (i < t.np) row[s_idx[i]] = x[u];
            }
        }
    }
}

// A_F32PJ: the A_F32P read-modify-write with orbital rows [hi pairs | lo pairs] per point; with PROJ the
// updated value x of every point is also projected, p_m += (phi_hi + phi_lo)_m x, both halves folded into
// one FP32 sum per orbital by two fused multiply-adds (the compensated products of the complex64
// projection).  The sums run over the lane's points, then over the Q lanes of the band; the tile's
// partial sums are written in FP64 without the Bloch phase, in the layout k_tile_reduce reads.
// Every lane of the warp calls it (the lane sums are combined with shuffles); lanes whose band is past
// nbands (active = false) touch no memory.
template <int Q, int M, int U, int PF, int PROJ>
__device__ __forceinline__ void apply_project_body(const View& v, const Tile& t, const ApplyArgs& a, int64_t off, int q,
                                                   int bl, int ks, int band, bool active, const int* s_idx,
                                                   const unsigned char* s_first, const unsigned char* after_idx,
                                                   const unsigned char* after_c) {
    constexpr int MP = (M + 1) & ~1, NP = MP / 2;
    float2* row = reinterpret_cast<float2*>(a.psi) + off;
    const float* s_phf = reinterpret_cast<const float*>(after_c);
    const float2* s_c = reinterpret_cast<const float2*>(after_idx);
    float2 cre[NP], cim[NP], Sr[NP], Si[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const float2 c0 = s_c[bl * MAXM + 2 * j];
        const float2 c1 = (2 * j + 1 < M) ? s_c[bl * MAXM + 2 * j + 1] : make_float2(0.f, 0.f);
        cre[j] = make_float2(c0.x, c1.x);
        cim[j] = make_float2(c0.y, c1.y);
        Sr[j] = make_float2(0.f, 0.f);
        Si[j] = make_float2(0.f, 0.f);
    }
    const int np = active ? t.np : 0;
    for (int i0 = q; i0 < np; i0 += Q * U) {
        float2 x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int i = i0 + u * Q;
            x[u] = (i < np && (a.accumulate || !s_first[i])) ? row[s_idx[i]] : make_float2(0.f, 0.f);
        }
        if (PF) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int i = i0 + Q * U + u * Q;
                if (i < np) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + s_idx[i]));
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float* ph = s_phf + (i0 + u * Q) * (2 * MP);
            float2 ar = make_float2(0.f, 0.f), ai = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                const float2 f2 = *reinterpret_cast<const float2*>(ph + 2 * j);
                ar = __ffma2_rn(f2, cre[j], ar);
                ai = __ffma2_rn(f2, cim[j], ai);
            }
            x[u] = __fadd2_rn(x[u], make_float2(ar.x + ar.y, ai.x + ai.y));
            if (PROJ) {   // rows past the tile are zeros, so the padded points add nothing
                const float2 r = make_float2(x[u].x, x[u].x), m = make_float2(x[u].y, x[u].y);
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    const float2 h2 = *reinterpret_cast<const float2*>(ph + 2 * j);
                    const float2 l2 = *reinterpret_cast<const float2*>(ph + MP + 2 * j);
                    Sr[j] = __ffma2_rn(l2, r, __ffma2_rn(h2, r, Sr[j]));
                    Si[j] = __ffma2_rn(l2, m, __ffma2_rn(h2, m, Si[j]));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int i = i0 + u * Q;
            if (i < np) row[s_idx[i]] = x[u];
        }
    }
    if (PROJ) {
#pragma unroll
        for (int o = Q / 2; o > 0; o >>= 1)
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                Sr[j] = __fadd2_rn(Sr[j], make_float2(__shfl_xor_sync(0xffffffffu, Sr[j].x, o), __shfl_xor_sync(0xffffffffu, Sr[j].y, o)));
                Si[j] = __fadd2_rn(Si[j], make_float2(__shfl_xor_sync(0xffffffffu, Si[j].x, o), __shfl_xor_sync(0xffffffffu, Si[j].y, o)));
            }
        // every lane of the band's group holds the sums; lane q writes orbital q (and q + Q, ...)
#pragma unroll
        for (int m0 = 0; m0 < M; m0 += Q) {
            const int mq = m0 + q;
            if (active && mq < M) {
                float re = Sr[0].x, im = Si[0].x;
#pragma unroll
                for (int mm = 1; mm < M; ++mm)
                    if (mm == mq) {
                        re = (mm & 1) ? Sr[mm / 2].y : Sr[mm / 2].x;
                        im = (mm & 1) ? Si[mm / 2].y : Si[mm / 2].x;
                    }
                v.part[((int64_t)ks * v.TM + t.moff + mq) * v.max_bands + band] = make_double2(f2d_bits(re), f2d_bits(im));
            }
        }
    }
}

// One work item: tile `tile_id` (a tile of the current colour) of the system (v, a), component ks, band chunk `chunk`.
template <int POL, int Q, int NBG, int U, int PF, int G>
__device__ __forceinline__ void apply_item(const View& v, const ApplyArgs& a, int tile_id, int ks, int chunk,
                                           unsigned char* smem, int& s_pe, unsigned char* s_first) {
    static_assert(Q * U <= TILE_PAD - TILE, "batched loops read up to Q*U rows past the tile");
    int* s_idx = reinterpret_cast<int*>(smem);
    constexpr int BPW = 32 / Q;
    constexpr int BPC = (CTA / 32) * BPW;
    const Tile t = v.tiles[tile_id];
    const int k = ks / v.ns, s = ks % v.ns;
    const int M = t.M;
    unsigned char* after_idx = smem + TILE * sizeof(int);
    // coefficient table [BPC][MAXM] in 16-byte slots: double2 (F64), (hi.re, hi.im, lo.re, lo.im) (PAIR), float2 (F32)
    unsigned char* after_c = after_idx + BPC * MAXM * 16;

    // ---- stage the tile once: grid indices and orbital rows (+ the orbitals' exponent bound)
    if (threadIdx.x == 0) s_pe = -200;
    for (int i = threadIdx.x; i < TILE; i += CTA) {
        s_idx[i] = (i < t.np) ? v.pt_idx[t.p0 + i] : 0;
        s_first[i] = (i < t.np) ? v.pt_first[t.p0 + i] : 0;
    }
    __syncthreads();
    if (POL == A_F64) {
        double* s_phi = reinterpret_cast<double*>(after_c);
        for (int e = threadIdx.x; e < TILE_PAD * M; e += CTA) s_phi[e] = (e < t.np * M) ? v.phi64[t.phi0 + e] : 0.0;
    } else if (POL == A_F32P) {
        float* s_phf = reinterpret_cast<float*>(after_c);
        const int MP = (M + 1) & ~1;
        for (int e = threadIdx.x; e < TILE_PAD * MP; e += CTA) {
            const int i = e / MP, m = e - i * MP;
            s_phf[e] = (i < t.np && m < M) ? v.phi_hi[t.phi0 + (int64_t)i * M + m] : 0.f;
        }
    } else if (POL == A_F32PJ) {
        float* s_phf = reinterpret_cast<float*>(after_c);
        const int MP = (M + 1) & ~1;
        for (int e = threadIdx.x; e < TILE_PAD * MP; e += CTA) {
            const int i = e / MP, m = e - i * MP;
            const bool in = i < t.np && m < M;
            s_phf[i * 2 * MP + m] = in ? v.phi_hi[t.phi0 + (int64_t)i * M + m] : 0.f;
            s_phf[i * 2 * MP + MP + m] = in ? v.phi_lo[t.phi0 + (int64_t)i * M + m] : 0.f;
        }
    } else {
        float4* s_phi = reinterpret_cast<float4*>(after_c);
        int pe = -200;
        for (int e = threadIdx.x; e < TILE_PAD * M; e += CTA) {
            float hi = 0.f, lo = 0.f;
            if (e < t.np * M) { hi = v.phi_hi[t.phi0 + e]; lo = v.phi_lo[t.phi0 + e]; }
            s_phi[e] = make_float4(hi, hi, lo, lo);
            if (hi != 0.f) pe = max(pe, ((__float_as_int(hi) >> 23) & 0xFF) - 126);
        }
        if (POL == A_PAIR) atomicMax(&s_pe, pe);
    }
    // gauge phases of the tile's points (zeros past the tile), after the orbital rows of the largest shell
    unsigned char* s_gauge = after_c + (size_t)TILE_PAD * v.maxM * (POL == A_F64 ? sizeof(double) : sizeof(float4));
    if (G) {
        if (POL == A_F64)
            for (int i = threadIdx.x; i < TILE_PAD; i += CTA)
                reinterpret_cast<double2*>(s_gauge)[i] = (i < t.np) ? v.gauge_d[t.p0 + i] : make_double2(0.0, 0.0);
        else
            for (int i = threadIdx.x; i < TILE_PAD; i += CTA)
                reinterpret_cast<float4*>(s_gauge)[i] = (i < t.np) ? v.gauge_f[t.p0 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int lane = threadIdx.x & 31;
    const int bl = (threadIdx.x >> 5) * BPW + lane / Q;
    const int q = lane & (Q - 1);
    const int mo = v.atom_moff[t.atom];
    for (int g = 0; g < NBG; ++g) {
        const int band0 = (chunk * NBG + g) * BPC;
        if (band0 >= a.nbands) break;
        __syncthreads();   // staging done / previous group's readers done with the coefficient table
        for (int e = threadIdx.x; e < BPC * M; e += CTA) {   // BPC * M exceeds CTA when Q = 4 and M >= 5
            int cb = e / M, m = e % M;
            int band = band0 + cb;
            double2 c = make_double2(0.0, 0.0);
            if (band < a.nbands) {
                const double2 w = v.cv[((int64_t)ks * v.max_bands + band) * v.MT + mo + m];   // (V p)_m
                const double re = w.x, im = w.y;
                double2 ph = v.seg_phase[t.seg * v.nk + k];   // exp(+ikT); the scatter uses its conjugate
                double2 cf = *reinterpret_cast<const double2*>(a.coef);
                double2 pc = make_double2(cf.x * ph.x + cf.y * ph.y, cf.y * ph.x - cf.x * ph.y);   // cf * conj(ph)
                c = make_double2(pc.x * re - pc.y * im, pc.x * im + pc.y * re);
            }
            if (POL == A_F64) reinterpret_cast<double2*>(after_idx)[cb * MAXM + m] = c;
            else if (POL == A_PAIR) {
                float hr, lr, hi, li;
                dsplit(c.x, hr, lr);
                dsplit(c.y, hi, li);
                reinterpret_cast<float4*>(after_idx)[cb * MAXM + m] = make_float4(hr, hi, lr, li);
            } else reinterpret_cast<float2*>(after_idx)[cb * MAXM + m] = make_float2((float)c.x, (float)c.y);
        }
        __syncthreads();
        const int band = band0 + bl;
        if constexpr (POL == A_F32PJ) {
            const bool active = band < a.nbands;
            const int64_t off = active ? (int64_t)k * a.sk + (int64_t)s * a.ss + (int64_t)band * a.sn : 0;
            const int qq = lane & (Q - 1);
#define DFTU_PJ(MM, PR) apply_project_body<Q, MM, U, PF, PR>(v, t, a, off, qq, bl, ks, band, active, s_idx, s_first, after_idx, after_c)
            if (v.tile_final[tile_id]) {
                switch (M) {
                    case 1: DFTU_PJ(1, 1); break;
                    case 3: DFTU_PJ(3, 1); break;
                    case 5: DFTU_PJ(5, 1); break;
                    default: DFTU_PJ(7, 1); break;
                }
            } else {
                switch (M) {
                    case 1: DFTU_PJ(1, 0); break;
                    case 3: DFTU_PJ(3, 0); break;
                    case 5: DFTU_PJ(5, 0); break;
                    default: DFTU_PJ(7, 0); break;
                }
            }
#undef DFTU_PJ
        } else if (band < a.nbands) {
            const int64_t off = (int64_t)k * a.sk + (int64_t)s * a.ss + (int64_t)band * a.sn;
            const int pe = s_pe;
            switch (M) {
                case 1: apply_body<POL, Q, 1, U, PF, G>(t, a, off, q, bl, s_idx, s_first, after_idx, after_c, pe, s_gauge); break;
                case 3: apply_body<POL, Q, 3, U, PF, G>(t, a, off, q, bl, s_idx, s_first, after_idx, after_c, pe, s_gauge); break;
                case 5: apply_body<POL, Q, 5, U, PF, G>(t, a, off, q, bl, s_idx, s_first, after_idx, after_c, pe, s_gauge); break;
                default: apply_body<POL, Q, 7, U, PF, G>(t, a, off, q, bl, s_idx, s_first, after_idx, after_c, pe, s_gauge); break;
            }
        }
    }
}

template <int POL, int Q, int NBG, int U, int PF, int G>
__global__ void __launch_bounds__(CTA, 3) k_apply(View v, ApplyArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_pe;
    __shared__ unsigned char s_first[TILE];
    apply_item<POL, Q, NBG, U, PF, G>(v, a, a.tile_list[blockIdx.x], blockIdx.z, blockIdx.y, smem, s_pe, s_first);
}

// Persistent form over many systems: (system, tile, k*spin) items of one colour from a counter.
template <int POL, int Q, int NBG, int U, int PF>
__global__ void __launch_bounds__(CTA, 3) k_apply_batch(const View* __restrict__ views, const ProjArgs* __restrict__ args,
                                                        const int4* __restrict__ items, int nitems, int* counter,
                                                        const double* coef, int accumulate) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_pe, s_item;
    __shared__ unsigned char s_first[TILE];
    constexpr int BPC = (CTA / 32) * (32 / Q);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int4 w = items[it];
        const View& v = views[w.x];
        const ProjArgs& pa = args[w.x];
        ApplyArgs a{const_cast<void*>(pa.psi), pa.sk, pa.ss, pa.sn, pa.nbands, coef, nullptr, accumulate};
        const int nchunks = (pa.nbands + BPC * NBG - 1) / (BPC * NBG);
        for (int c = 0; c < nchunks; ++c) {
            apply_item<POL, Q, NBG, U, PF, 0>(v, a, w.y, w.z, c, smem, s_pe, s_first);
            __syncthreads();
        }
    }
}

template <int POL, int Q, int NBG, int U, int PF, int G = 0>
static cudaError_t run_apply(const View& v, ApplyArgs a, const int* color_order, const std::vector<int>& color_beg,
                             cudaStream_t st) {
    constexpr int BPC = (CTA / 32) * (32 / Q);
    size_t smem = TILE * sizeof(int) + BPC * MAXM * 16 + (size_t)TILE_PAD * v.maxM * (POL == A_F64 ? sizeof(double) : sizeof(float4)) +
                  (G ? (size_t)TILE_PAD * 16 : 0);
    auto fn = k_apply<POL, Q, NBG, U, PF, G>;
    cudaError_t e = cudaSuccess;
    if (!smem_configured((const void*)fn, (int)smem)) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    for (size_t c = 0; c + 1 < color_beg.size(); ++c) {
        int n = color_beg[c + 1] - color_beg[c];
        if (n == 0) continue;
        a.tile_list = color_order + color_beg[c];
        dim3 grid(n, (a.nbands + BPC * NBG - 1) / (BPC * NBG), v.nk * v.ns);
        fn<<<grid, CTA, smem, st>>>(v, a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The shapes selectable with dftu_set_kernel_variant, listed once for the single-system and the batched
// launches: X(variant, lanes per band Q, band groups per CTA, points in flight per lane, L2 prefetch).
// Variant 0 takes the default case of each switch.
#define DFTU_APPLY_SHAPES_F32(X) X(1, A_F32, 8, 4, 8, 1) X(2, A_F32, 16, 4, 8, 1) X(3, A_F32P, 8, 4, 8, 1) \
    X(4, A_F32P, 8, 4, 16, 1) X(5, A_F32P, 16, 4, 4, 1) X(6, A_F32P, 16, 8, 4, 1) X(7, A_F32P, 8, 8, 8, 1)
#define DFTU_APPLY_DEFAULT_F32 A_F32P, 16, 4, 8, 1
#define DFTU_APPLY_SHAPES_PAIR(X) X(1, 8, 4, 4, 1) X(2, 16, 4, 2, 1) X(3, 8, 4, 8, 1) X(4, 16, 2, 4, 1) X(5, 16, 4, 4, 0) \
    X(6, 16, 8, 2, 1) X(7, 8, 8, 4, 1)
#define DFTU_APPLY_DEFAULT_PAIR 16, 4, 4, 1

cudaError_t launch_apply(const View& v, void* psi, dftu_prec prec, dftu_f64_mode mode, int nbands,
                         int64_t sk, int64_t ss, int64_t sn, const double* coef, const int* color_order,
                         const std::vector<int>& color_beg, int variant, int accumulate, cudaStream_t st, bool gauge) {
    ApplyArgs a{psi, sk, ss, sn, nbands, coef, nullptr, accumulate};
    if (gauge) {   // one shape per arithmetic policy with the gauge phases (Sec. V)
        if (prec == DFTU_C64) return run_apply<A_F32, 8, 4, 8, 1, 1>(v, a, color_order, color_beg, st);
        if (mode == DFTU_F64_NATIVE) return run_apply<A_F64, 8, 4, 4, 0, 1>(v, a, color_order, color_beg, st);
        return run_apply<A_PAIR, 8, 4, 4, 1, 1>(v, a, color_order, color_beg, st);
    }
#define DFTU_CASE_F32(i, POL, Q, NBG, U, PF) case i: return run_apply<POL, Q, NBG, U, PF>(v, a, color_order, color_beg, st);
#define DFTU_CASE_PAIR(i, Q, NBG, U, PF) case i: return run_apply<A_PAIR, Q, NBG, U, PF>(v, a, color_order, color_beg, st);
    if (prec == DFTU_C64) {
        switch (variant) {
            DFTU_APPLY_SHAPES_F32(DFTU_CASE_F32)
            default: return run_apply<DFTU_APPLY_DEFAULT_F32>(v, a, color_order, color_beg, st);
        }
    }
    if (mode == DFTU_F64_NATIVE) return run_apply<A_F64, 8, 4, 4, 0>(v, a, color_order, color_beg, st);
    switch (variant) {
        DFTU_APPLY_SHAPES_PAIR(DFTU_CASE_PAIR)
        default: return run_apply<A_PAIR, DFTU_APPLY_DEFAULT_PAIR>(v, a, color_order, color_beg, st);
    }
#undef DFTU_CASE_F32
#undef DFTU_CASE_PAIR
}

// The complex64 scatter of dftu_taylor_steps, fused with the next step's gather on the final tiles: the
// default complex64 apply shape (16 lanes per band, 8 points in flight, L2 prefetch).
cudaError_t launch_apply_project_c64(const View& v, void* psi, int nbands, int64_t sk, int64_t ss, int64_t sn,
                                     const double* coef, const int* color_order, const std::vector<int>& color_beg,
                                     cudaStream_t st) {
    ApplyArgs a{psi, sk, ss, sn, nbands, coef, nullptr, 1};
    return run_apply<A_F32PJ, 16, 4, 8, 1>(v, a, color_order, color_beg, st);
}

// cv[ks][band][moff_I + m] = sum_m' V^I_mm' p_m' (collinear: the spin block of ks; non-collinear: the
// 2M x 2M matrix over both spinor components of the band).  The apply multiplies it by each segment's
// conjugate Bloch phase and the caller's coefficient.
__device__ __forceinline__ void coefvec_elem(const View& v, int nbands, int64_t g) {
    const int64_t rows = (int64_t)v.nk * v.ns * nbands;
    if (g >= rows * v.MT) return;
    const int64_t rowi = g / v.MT;
    const int j = (int)(g % v.MT);
    const int ks = (int)(rowi / nbands), band = (int)(rowi % nbands);
    const int a = v.orb_atom[j];
    const int M = v.atom_M[a], mo = v.atom_moff[a], m = j - mo;
    const int64_t vo = v.atom_mat_off[a];
    const int k = ks / v.ns, s = ks % v.ns;
    double re = 0.0, im = 0.0;
    if (!v.noncollinear) {
        const double2* Vm = v.V + vo + (int64_t)s * M * M + m * M;
        const double2* pr = v.p + ((int64_t)ks * v.max_bands + band) * v.MT + mo;
        for (int qq = 0; qq < M; ++qq) {
            const double2 A = Vm[qq], B = pr[qq];
            re += A.x * B.x - A.y * B.y;
            im += A.x * B.y + A.y * B.x;
        }
    } else {
        const int D = 2 * M;
        const double2* Vm = v.V + vo + (int64_t)(s * M + m) * D;
        for (int c2 = 0; c2 < 2; ++c2) {
            const double2* pr = v.p + ((int64_t)(k * 2 + c2) * v.max_bands + band) * v.MT + mo;
            for (int qq = 0; qq < M; ++qq) {
                const double2 A = Vm[c2 * M + qq], B = pr[qq];
                re += A.x * B.x - A.y * B.y;
                im += A.x * B.y + A.y * B.x;
            }
        }
    }
    v.cv[((int64_t)ks * v.max_bands + band) * v.MT + j] = make_double2(re, im);
}

__global__ void k_coefvec(View v, int nbands) { coefvec_elem(v, nbands, (int64_t)blockIdx.x * blockDim.x + threadIdx.x); }

__global__ void k_coefvec_batch(const View* __restrict__ views, const ProjArgs* __restrict__ args) {
    coefvec_elem(views[blockIdx.y], args[blockIdx.y].nbands, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

cudaError_t launch_coefvec(const View& v, int nbands, cudaStream_t st) {
    const int64_t n = (int64_t)v.nk * v.ns * nbands * v.MT;
    k_coefvec<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v, nbands);
    return cudaGetLastError();
}

cudaError_t launch_coefvec_batch(const BatchLaunch& b, cudaStream_t st) {
    dim3 grid((unsigned)((b.max_reduce + 255) / 256), b.nsys);
    k_coefvec_batch<<<grid, 256, 0, st>>>(b.views, b.args);
    return cudaGetLastError();
}

// Taylor coefficients of exp(-i dt H): term j = (-i dt / j) H term_{j-1}.
__global__ void k_taylor_coefs(double dt, int order, double2* c) {
    int j = threadIdx.x + 1;
    if (j <= order) c[j - 1] = make_double2(0.0, -dt / (double)j);
}

cudaError_t launch_taylor_coefs(double dt, int order, double* coefs, cudaStream_t st) {
    k_taylor_coefs<<<1, MAX_TAYLOR, 0, st>>>(dt, order, reinterpret_cast<double2*>(coefs));
    return cudaGetLastError();
}

template <int POL, int Q, int NBG, int U, int PF>
static cudaError_t run_apply_batch(const BatchLaunch& b, const double* coef, int accumulate, cudaStream_t st) {
    constexpr int BPC = (CTA / 32) * (32 / Q);
    size_t smem = TILE * sizeof(int) + BPC * MAXM * 16 + (size_t)TILE_PAD * b.maxM * (POL == A_F64 ? sizeof(double) : sizeof(float4));
    auto fn = k_apply_batch<POL, Q, NBG, U, PF>;
    cudaError_t e = cudaSuccess;
    if (!smem_configured((const void*)fn, (int)smem)) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, CTA, smem);
    if (e != cudaSuccess) return e;
    for (size_t c = 0; c + 1 < b.color_beg.size(); ++c) {
        int n = b.color_beg[c + 1] - b.color_beg[c];
        if (n == 0) continue;
        e = cudaMemsetAsync(b.counter, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
        int grid = std::max(1, std::min(per_sm * nsm, n));
        fn<<<grid, CTA, smem, st>>>(b.views, b.args, b.color_items + b.color_beg[c], n, b.counter, coef, accumulate);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_apply_batch(const BatchLaunch& b, dftu_prec prec, dftu_f64_mode mode, int variant, const double* coef,
                               int accumulate, cudaStream_t st) {
#define DFTU_CASE_F32(i, POL, Q, NBG, U, PF) case i: return run_apply_batch<POL, Q, NBG, U, PF>(b, coef, accumulate, st);
#define DFTU_CASE_PAIR(i, Q, NBG, U, PF) case i: return run_apply_batch<A_PAIR, Q, NBG, U, PF>(b, coef, accumulate, st);
    if (prec == DFTU_C64) {
        switch (variant) {
            DFTU_APPLY_SHAPES_F32(DFTU_CASE_F32)
            default: return run_apply_batch<DFTU_APPLY_DEFAULT_F32>(b, coef, accumulate, st);
        }
    }
    if (mode == DFTU_F64_NATIVE) return run_apply_batch<A_F64, 8, 4, 4, 0>(b, coef, accumulate, st);
    switch (variant) {
        DFTU_APPLY_SHAPES_PAIR(DFTU_CASE_PAIR)
        default: return run_apply_batch<A_PAIR, DFTU_APPLY_DEFAULT_PAIR>(b, coef, accumulate, st);
    }
#undef DFTU_CASE_F32
#undef DFTU_CASE_PAIR
}

}  // namespace dftu
