// Sphere gather + projection p = dV sum_j phi_m(j) exp(+i k.T_j) psi(idx_j)   (inside Eqs. 4 and 6).
//
// Work decomposition: one CTA per (tile, band chunk, k*spin).  A tile holds up to TILE points of one
// (atom, lattice image) segment, so its Bloch phase is a single number.  The CTA stages the tile's
// grid indices and orbital values in shared memory once and streams the bands of its chunk: Q
// adjacent lanes walk the points of one band (Q*16 or Q*8 contiguous bytes per band row when the
// points run along x), 32/Q bands per warp.  Partial sums per tile are written in FP64 without the
// phase; k_tile_reduce sums the tiles of each atom in a fixed order, applies each image segment's
// phase once and scales by dV, so results are deterministic.
//
// Arithmetic policies
//   F64  : complex128 states, FP64 FMAs (the FP64 pipe of this GPU runs at ~1/70 of FP32).
//   PAIR : complex128 states carried as pairs of FP32 numbers.  Each double is split (integer ops,
//          47 significant bits) into hi + lo floats scaled by 2^-Emax of its chain; products accumulate
//          into an accumulator offset by a power of two C >= 4*sum|terms| so that the running sum
//          moves in one binade: t = s - acc is exact and the rounding residual a*b - t is caught
//          in a second float.  Chains are merged with TwoSum.  Accuracy ~2^-44 of the chain scale.
//   F32  : complex64 states, FP32 orbitals hi + lo paired two orbitals at a time, FP32 chunk sums
//          merged with TwoSum per lane, FP64 across tiles.
#include <algorithm>
#include <mutex>
#include <utility>

#include "dftu_internal.cuh"

namespace dftu {

// ------------------------------------------------------------------------------------------------
// small helpers
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }

struct DF2 { float2 h, l; };

// Ask L2 to start fetching a line a later chain will read (no register is held for it).
__device__ __forceinline__ void prefetch_l2(const void* ptr) { asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr)); }   // (re, im) pair of double-float numbers

// TwoSum(a.h, b.h) with the low parts added: a <- a + b.
__device__ __forceinline__ void df_add(DF2& a, const DF2& b) {
    float2 s = fadd2(a.h, b.h);
    float2 bb = fadd2(s, make_float2(-a.h.x, -a.h.y));
    float2 e1 = fadd2(a.h, make_float2(-(s.x - bb.x), -(s.y - bb.y)));
    float2 e2 = fadd2(b.h, make_float2(-bb.x, -bb.y));
    float2 e = fadd2(e1, e2);
    float2 l = fadd2(fadd2(a.l, b.l), e);
    a.h = s;
    a.l = l;
}

__device__ __forceinline__ float shfl_x(float x, int off) { return __shfl_xor_sync(0xffffffffu, x, off); }
__device__ __forceinline__ double shfl_x(double x, int off) { return __shfl_xor_sync(0xffffffffu, x, off); }

__device__ __forceinline__ float pow2f(int e) {   // 2^e as float for e in [-126, 127], 0 below
    return e < -126 ? 0.0f : __int_as_float((e + 127) << 23);
}

// Tile partial sum, before the Bloch phase and dV (k_tile_reduce applies both once per image segment).
// Layout [k*spin][tile slot (moff + m)][band], band fastest, so the reduce reads 32 bands of one slot in
// one coalesced access.  poff: offset of the direction's slice (three-table projections), 0 otherwise.
__device__ __forceinline__ void write_partial(const View& v, const Tile& t, int ks, int band, int m, double re, double im,
                                              int64_t poff) {
    v.part[poff + ((int64_t)ks * v.TM + t.moff + m) * v.max_bands + band] = make_double2(re, im);
}

// Exact float -> double times 2^s with integer operations (the conversion instruction runs on the
// FP64 pipe).  Zeros and FP32 denormals give 0; s must keep the result normal.
__device__ __forceinline__ double f2d_scaled(float f, int s) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned hi = (u & 0x80000000u) | ((e + 896u + (unsigned)s) << 20) | ((u & 0x7FFFFFu) >> 3);
    return e == 0 ? 0.0 : __hiloint2double((int)hi, (int)(u << 29));
}

// After the butterfly reductions every lane of a band's group holds the same sums, so the FP64
// epilogue (conversion, Bloch phase, dV) is spread over the lanes, one orbital each: it then issues
// once per warp instead of once per orbital on this GPU's narrow FP64 pipe.
template <int M, int Q, typename F>
__device__ __forceinline__ void per_lane_orbital(int q, F&& body) {
#pragma unroll
    for (int m0 = 0; m0 < M; m0 += Q)
        if (m0 + q < M) body(m0 + q);
}

// ------------------------------------------------------------------------------------------------
// F64 policy
// ------------------------------------------------------------------------------------------------
// x * (g.x + i g.y)
__device__ __forceinline__ double2 crot(double2 x, double2 g) {
    return make_double2(fma(g.x, x.x, -g.y * x.y), fma(g.y, x.x, g.x * x.y));
}

template <int M, int Q, int G>
__device__ __forceinline__ void proj_body_f64(const View& v, const Tile& t, int ks, int band, const double2* __restrict__ row,
                                              const int* s_idx, const double* s_phi, const double2* s_g, int64_t poff) {
    const int q = threadIdx.x & (Q - 1);
    double2 acc[M];
#pragma unroll
    for (int m = 0; m < M; ++m) acc[m] = make_double2(0.0, 0.0);
    if (row) {
        int i = q;
        for (; i + 3 * Q < t.np; i += 4 * Q) {
            double2 x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = __ldg(row + s_idx[i + u * Q]);
            if (G)
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = crot(x[u], s_g[i + u * Q]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double* ph = s_phi + (i + u * Q) * M;
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    acc[m].x = fma(ph[m], x[u].x, acc[m].x);
                    acc[m].y = fma(ph[m], x[u].y, acc[m].y);
                }
            }
        }
        for (; i < t.np; i += Q) {
            double2 x = __ldg(row + s_idx[i]);
            if (G) x = crot(x, s_g[i]);
            const double* ph = s_phi + i * M;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                acc[m].x = fma(ph[m], x.x, acc[m].x);
                acc[m].y = fma(ph[m], x.y, acc[m].y);
            }
        }
    }
#pragma unroll
    for (int off = Q / 2; off > 0; off >>= 1)
#pragma unroll
        for (int m = 0; m < M; ++m) {
            acc[m].x += shfl_x(acc[m].x, off);
            acc[m].y += shfl_x(acc[m].y, off);
        }
    if (row)
        per_lane_orbital<M, Q>(q, [&](int mq) {
            double2 a = acc[0];
#pragma unroll
            for (int m = 1; m < M; ++m)
                if (m == mq) a = acc[m];
            write_partial(v, t, ks, band, mq, a.x, a.y, poff);
        });
}

// ------------------------------------------------------------------------------------------------
// F32 policy (complex64 states)
// ------------------------------------------------------------------------------------------------
// Orbital rows of a tile for this policy: per point 2*MP floats, [hi_0 .. hi_{MP-1}, lo_0 .. lo_{MP-1}]
// with MP = M rounded up to even (zero padding).  Products pair two orbitals against one broadcast
// state component, (phi_m, phi_m+1) x (x_re, x_re), so one 8-byte shared load feeds two orbitals:
// half the shared-memory wavefronts of a per-orbital (hi, hi, lo, lo) row, which bound this kernel.
template <int M, int Q, int CH, int PF, int G>
__device__ __forceinline__ void proj_body_f32(const View& v, const Tile& t, int ks, int band, const float2* __restrict__ row,
                                              const int* s_idx, const float* s_phf, const float4* s_g, int64_t poff) {
    constexpr int MP = (M + 1) & ~1, NP = MP / 2;
    const int q = threadIdx.x & (Q - 1);
    DF2 Rr[NP], Ri[NP];   // running sums of the real and imaginary parts of orbitals (2j, 2j+1)
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        Rr[j] = DF2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        Ri[j] = Rr[j];
    }
    if (row) {
        for (int i0 = q; i0 < t.np; i0 += Q * CH) {
            float2 x[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                int i = i0 + c * Q;
                x[c] = (i < t.np) ? __ldg(row + s_idx[i]) : make_float2(0.f, 0.f);
            }
            if (G)
#pragma unroll
                for (int c = 0; c < CH; ++c) {   // x * (cos + i sin) in FP32 (rows past the tile hold zeros)
                    const float4 g = s_g[i0 + c * Q];
                    x[c] = ffma2(make_float2(-g.y, g.x), make_float2(x[c].y, x[c].y),
                                 __fmul2_rn(make_float2(g.x, g.y), make_float2(x[c].x, x[c].x)));
                }
            if (PF) {
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    int i = i0 + Q * CH + c * Q;
                    if (i < t.np) prefetch_l2(row + s_idx[i]);
                }
            }
            DF2 cr[NP], ci[NP];
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                cr[j] = DF2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                ci[j] = cr[j];
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const float* ph = s_phf + (i0 + c * Q) * (2 * MP);
                const float2 xr = make_float2(x[c].x, x[c].x), xi = make_float2(x[c].y, x[c].y);
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    const float2 h2 = *reinterpret_cast<const float2*>(ph + 2 * j);
                    const float2 l2 = *reinterpret_cast<const float2*>(ph + MP + 2 * j);
                    cr[j].h = ffma2(h2, xr, cr[j].h);
                    ci[j].h = ffma2(h2, xi, ci[j].h);
                    cr[j].l = ffma2(l2, xr, cr[j].l);
                    ci[j].l = ffma2(l2, xi, ci[j].l);
                }
            }
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                df_add(Rr[j], cr[j]);
                df_add(Ri[j], ci[j]);
            }
        }
    }
#pragma unroll
    for (int off = Q / 2; off > 0; off >>= 1)
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            DF2 o{make_float2(shfl_x(Rr[j].h.x, off), shfl_x(Rr[j].h.y, off)),
                  make_float2(shfl_x(Rr[j].l.x, off), shfl_x(Rr[j].l.y, off))};
            df_add(Rr[j], o);
            DF2 u{make_float2(shfl_x(Ri[j].h.x, off), shfl_x(Ri[j].h.y, off)),
                  make_float2(shfl_x(Ri[j].l.x, off), shfl_x(Ri[j].l.y, off))};
            df_add(Ri[j], u);
        }
    if (row)
        per_lane_orbital<M, Q>(q, [&](int mq) {
            float rh = Rr[0].h.x, rl = Rr[0].l.x, ih = Ri[0].h.x, il = Ri[0].l.x;
#pragma unroll
            for (int m = 1; m < M; ++m)
                if (m == mq) {
                    const DF2& a = Rr[m / 2];
                    const DF2& b = Ri[m / 2];
                    rh = (m & 1) ? a.h.y : a.h.x;
                    rl = (m & 1) ? a.l.y : a.l.x;
                    ih = (m & 1) ? b.h.y : b.h.x;
                    il = (m & 1) ? b.l.y : b.l.x;
                }
            write_partial(v, t, ks, band, mq, f2d_scaled(rh, 0) + f2d_scaled(rl, 0), f2d_scaled(ih, 0) + f2d_scaled(il, 0), poff);
        });
}

// ------------------------------------------------------------------------------------------------
// PAIR policy (complex128 states, FP32-pair arithmetic)
// ------------------------------------------------------------------------------------------------
// Split a double x with biased exponent field E <= Em (Em >= 127, the chain's largest) into floats
// hi + lo of x * 2^(1023-Em) by assembling their bit patterns with integer operations: hi takes the
// sign, the exponent E - Em + 127 and the top 23 fraction bits (a funnel shift of the two words after
// the exponent is rebased in place); lo the next 23 fraction bits under the exponent of hi less 23,
// minus the implicit one of that pattern (an exact subtraction).  47 significant bits, error below
// 2^-46 of 2^(E-Em).  bias = (Em - 127) << 20.  Magnitudes more than 2^103 below 2^(Em-1023), zeros
// included, are raised to that floor (an absolute change below 2^-102 of the chain scale), so both
// exponents stay normal without a branch.
__device__ __forceinline__ void split_bits(double x, int bias, float& hi, float& lo) {
    const unsigned whi = (unsigned)__double2hiint(x), wlo = (unsigned)__double2loint(x);
    const int a = max((int)(whi & 0x7FFFFFFFu) - bias, 24 << 20);                 // exponent field E' >= 24
    const unsigned hb = __funnelshift_l(wlo, (unsigned)a, 3) | (whi & 0x80000000u);
    const unsigned one = (hb - (23u << 23)) & 0xFF800000u;                         // +-2^(E' - 150)
    hi = __uint_as_float(hb);
    lo = __uint_as_float(one | ((wlo >> 6) & 0x007FFFFFu)) - __uint_as_float(one);
}

// the exponent field of x in place (a mask other than the split's, so the compiler does not keep one
// shared masked word per point alive across the chain)
__device__ __forceinline__ unsigned exp_bits(double x) { return (unsigned)__double2hiint(x) & 0x7FF00000u; }

// (bh + bl) * (g.x + g.z + i (g.y + g.w)) as a new float pair, componentwise for (re, im): the hi
// products are formed exactly (product + FMA residual) and added with TwoSum, the cross terms with
// the low parts go into the low word.  Error ~2^-47 of |b|; the modulus grows by at most sqrt(2) per
// component.
__device__ __forceinline__ void rot_pair(float2& bh, float2& bl, float4 g) {
    const float2 uh = make_float2(g.x, g.y), wh = make_float2(-g.y, g.x);
    const float2 ul = make_float2(g.z, g.w), wl = make_float2(-g.w, g.z);
    const float2 xr = make_float2(bh.x, bh.x), xi = make_float2(bh.y, bh.y);
    const float2 P = __fmul2_rn(uh, xr), R = __fmul2_rn(wh, xi);
    const float2 eP = ffma2(uh, xr, make_float2(-P.x, -P.y));
    const float2 eR = ffma2(wh, xi, make_float2(-R.x, -R.y));
    const float2 s = fadd2(P, R);
    const float2 bb = fadd2(s, make_float2(-P.x, -P.y));
    const float2 t = fadd2(fadd2(P, make_float2(bb.x - s.x, bb.y - s.y)), fadd2(R, make_float2(-bb.x, -bb.y)));
    float2 lo = fadd2(fadd2(eP, eR), t);
    lo = ffma2(uh, make_float2(bl.x, bl.x), lo);
    lo = ffma2(ul, xr, lo);
    lo = ffma2(wh, make_float2(bl.y, bl.y), lo);
    lo = ffma2(wl, xi, lo);
    bh = s;
    bl = lo;
}

// The Q*CH-point chain starting at i0 (lane points i0 + c*Q) into registers, zeros past the tile.
template <int Q, int CH>
__device__ __forceinline__ void pair_load(double2 (&x)[CH], int i0, const double2* __restrict__ row, const int* s_idx, int np) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        int i = i0 + c * Q;
        x[c] = (i < np) ? __ldg(row + s_idx[i]) : make_double2(0.0, 0.0);
    }
}

// One chain of the FP32-pair projection: the chain's scale (Em_run rises to its largest exponent and R
// is rescaled), the split states, the offset-accumulated products, merged into R.
template <int M, int Q, int CH, int G>
__device__ __forceinline__ void pair_chain(const double2 (&x)[CH], int i0, DF2 (&R)[M], int& Em_run, bool& bad, float Cv,
                                           const float4* s_phi, const float4* s_g) {
    const float2 C2 = make_float2(Cv, Cv);
    const float2 mone = make_float2(-1.f, -1.f);
    unsigned am = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) am = max(am, max(exp_bits(x[c].x), exp_bits(x[c].y)));
    int Ec = (int)(am >> 20);
    if (Ec == 0x7FF) bad = true;
    if (Ec == 0) return;
    Ec = max(Ec, 127);   // the split needs Em >= 127 (zeros then scale to 0)
    if (Ec > Em_run) {
        if (Em_run != 0) {
            float s = pow2f(Em_run - Ec);
            float2 s2 = make_float2(s, s);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                R[m].h = __fmul2_rn(R[m].h, s2);
                R[m].l = __fmul2_rn(R[m].l, s2);
            }
        }
        Em_run = Ec;
    }
    float2 acc[M], lo[M];
#pragma unroll
    for (int m = 0; m < M; ++m) { acc[m] = C2; lo[m] = make_float2(0.f, 0.f); }
    const int bias = (Em_run - 127) << 20;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        float2 bh, bl;
        split_bits(x[c].x, bias, bh.x, bl.x);
        split_bits(x[c].y, bias, bh.y, bl.y);
        if (G) rot_pair(bh, bl, s_g[i0 + c * Q]);
        const float4* ph = s_phi + (i0 + c * Q) * M;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            float4 f = ph[m];                                  // (hi, hi, lo, lo)
            float2 ah = make_float2(f.x, f.y), al = make_float2(f.z, f.w);
            float2 s = ffma2(ah, bh, acc[m]);                  // acc + a*b, rounded
            float2 tneg = ffma2(s, mone, acc[m]);              // acc - s  (exact: same binade)
            float2 r = ffma2(ah, bh, tneg);                    // rounding residual a*b - (s - acc)
            lo[m] = fadd2(lo[m], r);
            lo[m] = ffma2(ah, bl, lo[m]);
            lo[m] = ffma2(al, bh, lo[m]);
            acc[m] = s;
        }
    }
#pragma unroll
    for (int m = 0; m < M; ++m) {
        DF2 chn{fadd2(acc[m], make_float2(-Cv, -Cv)), lo[m]};  // exact removal of the offset
        df_add(R[m], chn);
    }
}

// Each lane takes chains of CH points (i0 + c*Q), one after another, and merges each into R.
// PF = 1: every chain asks L2 for the next one; PF = 5: in addition the last chain of the tile asks for
// the first chain of the band the lane takes next (row_next, null if none), so only the first band
// group of a CTA starts cold.
template <int M, int Q, int CH, int PF, int G>
__device__ __forceinline__ void proj_body_pair(const View& v, const Tile& t, int ks, int band, const double2* __restrict__ row,
                                               const double2* __restrict__ row_next, const int* s_idx, const float4* s_phi,
                                               int pe, const float4* s_g, int64_t poff) {
    const int q = threadIdx.x & (Q - 1);
    DF2 R[M];
#pragma unroll
    for (int m = 0; m < M; ++m) R[m] = DF2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    int Em_run = 0;
    bool bad = false;
    // chain offset C = 2^(pe + 1 + log2 CH + 2) >= 4 * CH * max|phi x'|, |x'| < 2, |phi| < 2^pe
    // (one more power of two when x' is rotated by a gauge phase: |x'| < 2 sqrt 2)
    constexpr int LOG2CH = (CH >= 16) ? 4 : (CH >= 8) ? 3 : (CH >= 4) ? 2 : (CH >= 2) ? 1 : 0;
    const float Cv = pow2f(min(max(pe + 3 + G + LOG2CH, -100), 100));
#define DFTU_PAIR_CHAIN(x, i0) pair_chain<M, Q, CH, G>(x, i0, R, Em_run, bad, Cv, s_phi, s_g)
#define DFTU_PAIR_LOAD(x, i0) pair_load<Q, CH>(x, i0, row, s_idx, t.np)
    // L2 prefetch of the chain starting at i0; past the tile (PF == 5) the first chain of the next band
    auto prefetch = [&](int i0) {
        if (PF == 1 || PF == 5 || (PF == 2 && (q == 0 || q == Q - 1))) {   // PF == 2: the group's edge lanes only
            if (PF == 5 && i0 >= t.np) {
                if (row_next)
#pragma unroll
                    for (int c = 0; c < CH; ++c) {
                        int i = q + c * Q;
                        if (i < t.np) prefetch_l2(row_next + s_idx[i]);
                    }
            } else {
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    int i = i0 + c * Q;
                    if (i < t.np) prefetch_l2(row + s_idx[i]);
                }
            }
        }
    };
    if (row)
        for (int i0 = q; i0 < t.np; i0 += Q * CH) {
            double2 x[CH];
            DFTU_PAIR_LOAD(x, i0);
            prefetch(i0 + Q * CH);
            DFTU_PAIR_CHAIN(x, i0);
        }
#undef DFTU_PAIR_CHAIN
#undef DFTU_PAIR_LOAD
    // bring the Q lanes of this band to a common scale, then add in pairs
    int Em_max = Em_run;
#pragma unroll
    for (int off = Q / 2; off > 0; off >>= 1) Em_max = max(Em_max, __shfl_xor_sync(0xffffffffu, Em_max, off));
    if (Em_run != Em_max) {
        float s = (Em_run == 0) ? 0.0f : pow2f(Em_run - Em_max);
        float2 s2 = make_float2(s, s);
#pragma unroll
        for (int m = 0; m < M; ++m) {
            R[m].h = __fmul2_rn(R[m].h, s2);
            R[m].l = __fmul2_rn(R[m].l, s2);
        }
    }
#pragma unroll
    for (int off = Q / 2; off > 0; off >>= 1)
#pragma unroll
        for (int m = 0; m < M; ++m) {
            DF2 o{make_float2(shfl_x(R[m].h.x, off), shfl_x(R[m].h.y, off)),
                  make_float2(shfl_x(R[m].l.x, off), shfl_x(R[m].l.y, off))};
            df_add(R[m], o);
        }
    int anybad = bad ? 1 : 0;   // any non-finite value among this band's lanes
#pragma unroll
    for (int off = Q / 2; off > 0; off >>= 1) anybad |= __shfl_xor_sync(0xffffffffu, anybad, off);
    if (row) {
        const int sc = Em_max - 1023;   // the sums are in units of 2^(Em_max - 1023), Em_max >= 127 or sums zero
        per_lane_orbital<M, Q>(q, [&](int mq) {
            DF2 a = R[0];
#pragma unroll
            for (int m = 1; m < M; ++m)
                if (m == mq) a = R[m];
            double re = f2d_scaled(a.h.x, sc) + f2d_scaled(a.l.x, sc);
            double im = f2d_scaled(a.h.y, sc) + f2d_scaled(a.l.y, sc);
            if (anybad) { re = __longlong_as_double(0x7FF8000000000000LL); im = re; }
            write_partial(v, t, ks, band, mq, re, im, poff);
        });
    }
}

// ------------------------------------------------------------------------------------------------
// F32 policy, two bands per lane (complex64 states)
// ------------------------------------------------------------------------------------------------
// Every lane walks its points for two bands at once, so each grid index and each paired orbital load
// from shared memory serves both.  Products are compensated as in proj_body_f32 (phi = hi + lo, both
// halves multiplied by the FP32 state value); the sums are plain FP32 over the lane's points of the
// tile, then over the Q lanes, and FP64 from there on (across tiles).
// FOLD: each product phi x is formed from both halves of phi by two fused multiply-adds into one FP32 sum
// (hi then lo), instead of separate sums of the hi and lo products: half the accumulator registers, the
// same products; the lo half then enters at the sum's rounding, which plain FP32 accumulation over a
// lane's points already sets.
template <int M, int Q, int CH, int PF, int FOLD = 0>
__device__ __forceinline__ void proj_body_f32x2(const View& v, const Tile& t, int ks, int band, int nbands,
                                                const float2* __restrict__ row0, const float2* __restrict__ row1,
                                                const int* s_idx, const float* s_phf, int64_t poff) {
    constexpr int MP = (M + 1) & ~1, NP = MP / 2;
    constexpr int NS = FOLD ? 2 : 4;
    const int q = threadIdx.x & (Q - 1);
    // [band][part]: real hi, imaginary hi (real lo, imaginary lo unless folded) of orbitals (2j, 2j+1)
    float2 S0[NS][NP], S1[NS][NP];
#pragma unroll
    for (int a = 0; a < NS; ++a)
#pragma unroll
        for (int j = 0; j < NP; ++j) { S0[a][j] = make_float2(0.f, 0.f); S1[a][j] = S0[a][j]; }
    if (row0) {
        for (int i0 = q; i0 < t.np; i0 += Q * CH) {
            float2 x0[CH], x1[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int i = i0 + c * Q;
                const bool in = i < t.np;
                const int g = in ? s_idx[i] : 0;
                x0[c] = in ? __ldg(row0 + g) : make_float2(0.f, 0.f);
                x1[c] = (in && row1) ? __ldg(row1 + g) : make_float2(0.f, 0.f);
            }
            if (PF) {
                // PF == 2: only the first and last lane of a band's group, whose points bound the Q
                // consecutive points the group reads next (at most two 128-byte lines per row)
                if (PF == 1 || q == 0 || q == Q - 1) {
#pragma unroll
                    for (int c = 0; c < CH; ++c) {
                        const int i = i0 + Q * CH + c * Q;
                        if (i < t.np) {
                            prefetch_l2(row0 + s_idx[i]);
                            if (row1) prefetch_l2(row1 + s_idx[i]);
                        }
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const float* ph = s_phf + (i0 + c * Q) * (2 * MP);
                const float2 r0 = make_float2(x0[c].x, x0[c].x), m0 = make_float2(x0[c].y, x0[c].y);
                const float2 r1 = make_float2(x1[c].x, x1[c].x), m1 = make_float2(x1[c].y, x1[c].y);
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    const float2 h2 = *reinterpret_cast<const float2*>(ph + 2 * j);
                    const float2 l2 = *reinterpret_cast<const float2*>(ph + MP + 2 * j);
                    if (FOLD) {
                        S0[0][j] = ffma2(l2, r0, ffma2(h2, r0, S0[0][j]));
                        S0[1][j] = ffma2(l2, m0, ffma2(h2, m0, S0[1][j]));
                        S1[0][j] = ffma2(l2, r1, ffma2(h2, r1, S1[0][j]));
                        S1[1][j] = ffma2(l2, m1, ffma2(h2, m1, S1[1][j]));
                    } else {
                        S0[0][j] = ffma2(h2, r0, S0[0][j]); S0[1][j] = ffma2(h2, m0, S0[1][j]);
                        S0[NS - 2][j] = ffma2(l2, r0, S0[NS - 2][j]); S0[NS - 1][j] = ffma2(l2, m0, S0[NS - 1][j]);
                        S1[0][j] = ffma2(h2, r1, S1[0][j]); S1[1][j] = ffma2(h2, m1, S1[1][j]);
                        S1[NS - 2][j] = ffma2(l2, r1, S1[NS - 2][j]); S1[NS - 1][j] = ffma2(l2, m1, S1[NS - 1][j]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int off = Q / 2; off > 0; off >>= 1)
#pragma unroll
        for (int a = 0; a < NS; ++a)
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                S0[a][j] = fadd2(S0[a][j], make_float2(shfl_x(S0[a][j].x, off), shfl_x(S0[a][j].y, off)));
                S1[a][j] = fadd2(S1[a][j], make_float2(shfl_x(S1[a][j].x, off), shfl_x(S1[a][j].y, off)));
            }
    if (row0) {
        per_lane_orbital<M, Q>(q, [&](int mq) {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                if (b == 1 && !row1) break;
                float v4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int a = 0; a < NS; ++a) {
                    const float2 w = (b == 0) ? S0[a][0] : S1[a][0];
                    v4[a] = w.x;
                }
#pragma unroll
                for (int m = 1; m < M; ++m)
                    if (m == mq)
#pragma unroll
                        for (int a = 0; a < NS; ++a) {
                            const float2 w = (b == 0) ? S0[a][m / 2] : S1[a][m / 2];
                            v4[a] = (m & 1) ? w.y : w.x;
                        }
                write_partial(v, t, ks, band + b, mq, f2d_scaled(v4[0], 0) + f2d_scaled(v4[2], 0),
                              f2d_scaled(v4[1], 0) + f2d_scaled(v4[3], 0), poff);
            }
        });
    }
    (void)nbands;
}

// ------------------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------------------
enum Pol { P_F64 = 0, P_PAIR = 1, P_F32 = 2, P_F32B2 = 4, P_F32B2F = 5 };

// bands a lane carries at once
template <int POL> struct LaneBands { static constexpr int value = (POL == P_F32B2 || POL == P_F32B2F) ? 2 : 1; };

// Bytes of one staged orbital row (one point) for the largest shell maxM: FP64 values, (hi, hi, lo, lo)
// per orbital for the FP32-pair policy, [hi pairs | lo pairs] for the complex64 policies.
__host__ __device__ constexpr size_t phi_row_bytes(int pol, int maxM) {
    return pol == P_F64 ? 8 * (size_t)maxM : pol == P_PAIR ? 16 * (size_t)maxM : 8 * (size_t)((maxM + 1) & ~1);
}

// One work item: tile `tile_id` of the system described by (v, a), spin/component index ks, every band of
// band chunk `chunk` (NBG groups of BPC bands), against orbital table `dir` (0 unless the launch projects
// onto several tables).  The tile is staged in shared memory once.  TP: the tiling's largest tile (TILE,
// or PTILE when the launch's View carries the projection's own tiling); shared memory holds TP grid
// indices, then TP + 128 orbital rows (zeros past the tile), then the gauge phases.
template <int POL, int Q, int CH, int NBG, int PF, int G, int NT = CTA, int TP = TILE>
__device__ __forceinline__ void project_item(const View& v, const ProjArgs& a, int tile_id, int ks, int chunk,
                                             unsigned char* smem, int* s_pe, int dir = 0) {
    int* s_idx = reinterpret_cast<int*>(smem);
    const Tile t = v.tiles[tile_id];
    const int64_t ph0 = t.phi0 + dir * v.phi_dir_stride;   // this table's rows of the tile
    const int64_t poff = dir * v.part_dir_stride;
    const int k = ks / v.ns, s = ks % v.ns;
    constexpr int NBL = LaneBands<POL>::value;   // bands per lane
    constexpr int BPW = (32 / Q) * NBL;
    constexpr int BPC = (NT / 32) * BPW;

    // ---- stage the tile once (grid indices, orbital rows, orbital exponent bound)
    if (threadIdx.x == 0) *s_pe = -200;
    constexpr int TPAD = TP + (TILE_PAD - TILE);
    for (int i = threadIdx.x; i < TP; i += NT) s_idx[i] = (i < t.np) ? v.pt_idx[t.p0 + i] : 0;
    __syncthreads();
    if (POL == P_F64) {
        double* s_phi = reinterpret_cast<double*>(smem + TP * sizeof(int));
        for (int e = threadIdx.x; e < TP * t.M; e += NT)
            s_phi[e] = (e < t.np * t.M) ? v.phi64[ph0 + e] : 0.0;
    } else if (POL == P_F32 || POL == P_F32B2 || POL == P_F32B2F) {
        float* s_phf = reinterpret_cast<float*>(smem + TP * sizeof(int));
        const int MP = (t.M + 1) & ~1;
        int pe = -200;
        for (int e = threadIdx.x; e < TPAD * MP; e += NT) {
            const int i = e / MP, m = e - i * MP;
            float hi = 0.f, lo = 0.f;
            if (i < t.np && m < t.M) { hi = v.phi_hi[ph0 + (int64_t)i * t.M + m]; lo = v.phi_lo[ph0 + (int64_t)i * t.M + m]; }
            s_phf[i * 2 * MP + m] = hi;
            s_phf[i * 2 * MP + MP + m] = lo;
            if (hi != 0.f) pe = max(pe, ((__float_as_int(hi) >> 23) & 0xFF) - 127 + 1);   // |hi| < 2^pe
        }
    } else {
        float4* s_phi = reinterpret_cast<float4*>(smem + TP * sizeof(int));
        int pe = -200;
        for (int e = threadIdx.x; e < TPAD * t.M; e += NT) {
            float hi = 0.f, lo = 0.f;
            if (e < t.np * t.M) { hi = v.phi_hi[ph0 + e]; lo = v.phi_lo[ph0 + e]; }
            s_phi[e] = make_float4(hi, hi, lo, lo);
            if (hi != 0.f) pe = max(pe, ((__float_as_int(hi) >> 23) & 0xFF) - 127 + 1);   // |hi| < 2^pe
        }
        if (POL == P_PAIR) atomicMax(s_pe, pe);
    }
    // gauge phases of the tile's points (zeros past the tile), after the orbital rows of the largest shell
    unsigned char* s_gauge = smem + TP * sizeof(int) + (size_t)TPAD * phi_row_bytes(POL, v.maxM);
    if (G) {
        if (POL == P_F64)
            for (int i = threadIdx.x; i < TPAD; i += NT)
                reinterpret_cast<double2*>(s_gauge)[i] = (i < t.np) ? v.gauge_d[t.p0 + i] : make_double2(0.0, 0.0);
        else
            for (int i = threadIdx.x; i < TPAD; i += NT)
                reinterpret_cast<float4*>(s_gauge)[i] = (i < t.np) ? v.gauge_f[t.p0 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();

    // ---- stream NBG groups of BPC bands over the staged tile
    for (int g = 0; g < NBG; ++g) {
        const int band0 = (chunk * NBG + g) * BPC;
        if (band0 >= a.nbands) break;
        const int band = band0 + (threadIdx.x >> 5) * BPW + ((threadIdx.x & 31) / Q) * NBL;
        const bool active = band < a.nbands;
        const int64_t off = (int64_t)k * a.sk + (int64_t)s * a.ss + (int64_t)band * a.sn;
        if (POL == P_F32B2 || POL == P_F32B2F) {
            constexpr int FOLD = (POL == P_F32B2F) ? 1 : 0;
            const float* s_phf = reinterpret_cast<const float*>(smem + TP * sizeof(int));
            const float2* row0 = active ? reinterpret_cast<const float2*>(a.psi) + off : nullptr;
            const float2* row1 = (band + 1 < a.nbands) ? row0 + a.sn : nullptr;
            switch (t.M) {
                case 1: proj_body_f32x2<1, Q, CH, PF, FOLD>(v, t, ks, band, a.nbands, row0, row1, s_idx, s_phf, poff); break;
                case 3: proj_body_f32x2<3, Q, CH, PF, FOLD>(v, t, ks, band, a.nbands, row0, row1, s_idx, s_phf, poff); break;
                case 5: proj_body_f32x2<5, Q, CH, PF, FOLD>(v, t, ks, band, a.nbands, row0, row1, s_idx, s_phf, poff); break;
                default: proj_body_f32x2<7, Q, CH, PF, FOLD>(v, t, ks, band, a.nbands, row0, row1, s_idx, s_phf, poff); break;
            }
        } else if (POL == P_F64) {
            const double* s_phi = reinterpret_cast<const double*>(smem + TP * sizeof(int));
            const double2* row = active ? reinterpret_cast<const double2*>(a.psi) + off : nullptr;
            const double2* s_g = reinterpret_cast<const double2*>(s_gauge);
            switch (t.M) {
                case 1: proj_body_f64<1, Q, G>(v, t, ks, band, row, s_idx, s_phi, s_g, poff); break;
                case 3: proj_body_f64<3, Q, G>(v, t, ks, band, row, s_idx, s_phi, s_g, poff); break;
                case 5: proj_body_f64<5, Q, G>(v, t, ks, band, row, s_idx, s_phi, s_g, poff); break;
                default: proj_body_f64<7, Q, G>(v, t, ks, band, row, s_idx, s_phi, s_g, poff); break;
            }
        } else if (POL == P_PAIR) {
            const float4* s_phi = reinterpret_cast<const float4*>(smem + TP * sizeof(int));
            const double2* row = active ? reinterpret_cast<const double2*>(a.psi) + off : nullptr;
            const double2* row_next = (active && g + 1 < NBG && band + BPC < a.nbands) ? row + (int64_t)BPC * a.sn : nullptr;
            const int pe = *s_pe;
            const float4* s_g = reinterpret_cast<const float4*>(s_gauge);
            switch (t.M) {
                case 1: proj_body_pair<1, Q, CH, PF, G>(v, t, ks, band, row, row_next, s_idx, s_phi, pe, s_g, poff); break;
                case 3: proj_body_pair<3, Q, CH, PF, G>(v, t, ks, band, row, row_next, s_idx, s_phi, pe, s_g, poff); break;
                case 5: proj_body_pair<5, Q, CH, PF, G>(v, t, ks, band, row, row_next, s_idx, s_phi, pe, s_g, poff); break;
                default: proj_body_pair<7, Q, CH, PF, G>(v, t, ks, band, row, row_next, s_idx, s_phi, pe, s_g, poff); break;
            }
        } else {
            const float* s_phf = reinterpret_cast<const float*>(smem + TP * sizeof(int));
            const float2* row = active ? reinterpret_cast<const float2*>(a.psi) + off : nullptr;
            const float4* s_g = reinterpret_cast<const float4*>(s_gauge);
            switch (t.M) {
                case 1: proj_body_f32<1, Q, CH, PF, G>(v, t, ks, band, row, s_idx, s_phf, s_g, poff); break;
                case 3: proj_body_f32<3, Q, CH, PF, G>(v, t, ks, band, row, s_idx, s_phf, s_g, poff); break;
                case 5: proj_body_f32<5, Q, CH, PF, G>(v, t, ks, band, row, s_idx, s_phf, s_g, poff); break;
                default: proj_body_f32<7, Q, CH, PF, G>(v, t, ks, band, row, s_idx, s_phf, s_g, poff); break;
            }
        }
    }
}

// NDIR > 1: blockIdx.x = tile * NDIR + direction, so the CTAs of one tile and band chunk for the
// NDIR orbital tables are neighbours in the launch and read the same states while they sit in L2.
template <int POL, int Q, int CH, int NBG, int PF, int MINB, int G, int NDIR = 1, int NT = CTA, int TP = TILE>
__global__ void __launch_bounds__(NT, MINB) k_project(View v, ProjArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_pe;
    const int tile = (NDIR == 1) ? (int)blockIdx.x : (int)blockIdx.x / NDIR;
    const int dir = (NDIR == 1) ? 0 : (int)blockIdx.x % NDIR;
    project_item<POL, Q, CH, NBG, PF, G, NT, TP>(v, a, tile, blockIdx.z, blockIdx.y, smem, &s_pe, dir);
}

// Persistent form over many systems: every CTA takes (system, tile, k*spin) items from a counter until
// the list is exhausted and processes all band chunks of the item's system.
template <int POL, int Q, int CH, int NBG, int PF, int MINB, int NT = CTA>
__global__ void __launch_bounds__(NT, MINB) k_project_batch(const View* __restrict__ views, const ProjArgs* __restrict__ args,
                                                          const int4* __restrict__ items, int nitems, int* counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_pe, s_item;
    constexpr int BPC = (NT / 32) * (32 / Q) * LaneBands<POL>::value;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int4 w = items[it];   // (system, tile, k*spin, unused)
        const View& v = views[w.x];
        const ProjArgs& a = args[w.x];
        const int nchunks = (a.nbands + BPC * NBG - 1) / (BPC * NBG);
        for (int c = 0; c < nchunks; ++c) {
            project_item<POL, Q, CH, NBG, PF, 0, NT>(v, a, w.y, w.z, c, smem, &s_pe);
            __syncthreads();   // the next chunk or item restages shared memory
        }
    }
}

// One record per (kernel, device): the largest dynamic shared memory size already allowed.
bool smem_configured(const void* fn, int bytes) {
    static std::mutex mu;
    static std::vector<std::pair<std::pair<const void*, int>, int>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    for (auto& d : done)
        if (d.first.first == fn && d.first.second == dev) {
            if (d.second >= bytes) return true;
            d.second = bytes;
            return false;
        }
    done.push_back({{fn, dev}, bytes});
    return false;
}

// p[ks][band][moff_I + m] = sum over the atom's tiles (fixed order) of the tile partials; one thread per
// (k*spin, orbital slot, band), band fastest.
__device__ __forceinline__ void tile_reduce_elem(const View& v, int nbands, int64_t g) {
    if (g >= (int64_t)v.nk * v.ns * v.MT * nbands) return;
    const int band = (int)(g % nbands);
    const int64_t r = g / nbands;
    const int j = (int)(r % v.MT);
    const int ks = (int)(r / v.MT);
    const int a = v.orb_atom[j];
    const int m = j - v.atom_moff[a];
    const double2* pks = v.part + (int64_t)ks * v.TM * v.max_bands + band;
    auto prow_at = [&](int slot) { return pks[(int64_t)slot * v.max_bands]; };
    const int k = ks / v.ns;
    // tiles of one image segment are consecutive: sum them, then apply that segment's Bloch phase
    double re = 0.0, im = 0.0, sr = 0.0, si = 0.0;
    int seg = -1;
    for (int t = v.atom_tile_beg[a]; t < v.atom_tile_end[a]; ++t) {
        const Tile& tl = v.tiles[t];
        if (tl.seg != seg) {
            if (seg >= 0) {
                const double2 ph = v.seg_phase[seg * v.nk + k];
                re += ph.x * sr - ph.y * si;
                im += ph.x * si + ph.y * sr;
            }
            seg = tl.seg;
            sr = si = 0.0;
        }
        const double2 x = prow_at(tl.moff + m);
        sr += x.x;
        si += x.y;
    }
    if (seg >= 0) {
        const double2 ph = v.seg_phase[seg * v.nk + k];
        re += ph.x * sr - ph.y * si;
        im += ph.x * si + ph.y * sr;
    }
    re *= v.dV;
    im *= v.dV;
    if (!isfinite(re) || !isfinite(im)) atomicOr(v.status, ST_NONFINITE);
    v.p[((int64_t)ks * v.max_bands + band) * v.MT + j] = make_double2(re, im);
}

__global__ void k_tile_reduce(View v, int nbands) {
    tile_reduce_elem(v, nbands, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_tile_reduce_batch(const View* __restrict__ views, const ProjArgs* __restrict__ args) {
    tile_reduce_elem(views[blockIdx.y], args[blockIdx.y].nbands, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// Whether MINB CTAs of fn with smem bytes of dynamic shared memory fit on one SM (cached per kernel and size).
static bool fits_per_sm(const void* fn, int nt, size_t smem, int minb) {
    static std::mutex mu;
    static std::vector<std::pair<std::pair<const void*, size_t>, bool>> seen;
    std::lock_guard<std::mutex> lock(mu);
    for (auto& s : seen)
        if (s.first.first == fn && s.first.second == smem) return s.second;
    int n = 0;
    // the attribute only ever grows (smem_configured keeps the largest size set), so a smaller system
    // asked about later cannot leave it below what an earlier launch configured
    cudaError_t e = cudaSuccess;
    if (!smem_configured(fn, (int)smem)) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, nt, smem) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    seen.push_back({{fn, smem}, n >= minb});
    return n >= minb;
}

// One projection launch.  TP = PTILE runs over the projection's own tiling (View::ptiles) when MINB CTAs
// with that shared memory still fit on an SM, and over the TILE tiling otherwise; *used receives the View
// the launch ran with, whose tiling the tile reduce must follow.
template <int POL, int Q, int CH, int NBG, int PF, int MINB = 2, int G = 0, int NDIR = 1, int NT = CTA, int TP = TILE>
static cudaError_t run_project(const View& v, const ProjArgs& a, cudaStream_t st, View* used = nullptr) {
    static_assert(Q * CH <= TILE_PAD - TILE, "chained loops read up to Q*CH rows past the tile");
    static_assert(TP == TILE || TP == PTILE, "a tiling the View carries");
    constexpr int TPAD = TP + (TILE_PAD - TILE);
    size_t smem = TP * sizeof(int) + (size_t)TPAD * phi_row_bytes(POL, v.maxM) + (G ? (size_t)TPAD * 16 : 0);
    auto fn = k_project<POL, Q, CH, NBG, PF, MINB, G, NDIR, NT, TP>;
    View vl = v;
    if (TP != TILE) {
        if (!fits_per_sm((const void*)fn, NT, smem, MINB)) return run_project<POL, Q, CH, NBG, PF, MINB, G, NDIR, NT, TILE>(v, a, st, used);
        vl.tiles = v.ptiles; vl.ntiles = v.nptiles; vl.TM = v.pTM;
        vl.atom_tile_beg = v.patom_tile_beg; vl.atom_tile_end = v.patom_tile_end;
    }
    if (used) *used = vl;
    cudaError_t e = cudaSuccess;
    if (!smem_configured((const void*)fn, (int)smem)) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    constexpr int BPC = (NT / 32) * (32 / Q) * LaneBands<POL>::value;
    dim3 grid(vl.ntiles * NDIR, (a.nbands + BPC * NBG - 1) / (BPC * NBG), vl.nk * vl.ns);
    fn<<<grid, NT, smem, st>>>(vl, a);
    return cudaGetLastError();
}

// The default shape of a table row (variant 0): run_project with its thread count and tiling in the last
// places.
template <int POL, int Q, int CH, int NBG, int PF, int MINB, int NT, int TP>
static cudaError_t run_project_default(const View& v, const ProjArgs& a, cudaStream_t st, View* used) {
    return run_project<POL, Q, CH, NBG, PF, MINB, 0, 1, NT, TP>(v, a, st, used);
}

// The shapes selectable with dftu_set_kernel_variant, listed once for the single-system and the batched
// launches: X(variant, policy, lanes per band Q, points per chain, band groups per CTA, L2 prefetch,
// minimum blocks per SM, threads per CTA, tile size).  Variant 0 is the default case of each switch.
// P_F32B2 is the complex64 form with two bands per lane, P_F32B2F the same with each product's hi and lo
// halves folded into one sum, P_F32 one band per lane.  PAIR L2 prefetch: 1 = the next chain, 5 = also
// the next band's first chain.  Tile size PTILE selects the projection's own tiling (single-system
// launches; batched launches use TILE, on which PAIR variant 1 is the default shape).
#define DFTU_PROJECT_SHAPES_F32(X) \
    X(1, P_F32B2F, 16, 8, 4, 0, 3, 256, PTILE) X(2, P_F32B2F, 8, 8, 4, 0, 3, 256, TILE) X(3, P_F32B2, 8, 8, 4, 0, 2, 256, TILE) \
    X(4, P_F32B2F, 16, 8, 4, 0, 2, 256, TILE) X(5, P_F32B2F, 16, 8, 8, 0, 3, 256, TILE) \
    X(6, P_F32B2F, 16, 6, 4, 0, 3, 256, TILE) X(7, P_F32, 8, 16, 8, 0, 2, 256, TILE)
#define DFTU_PROJECT_DEFAULT_F32 P_F32B2F, 16, 8, 4, 0, 3, 256, TILE
#define DFTU_PROJECT_SHAPES_PAIR(X) \
    X(1, P_PAIR, 8, 8, 8, 5, 2, 256, TILE) X(2, P_PAIR, 8, 8, 4, 5, 2, 256, PTILE) X(3, P_PAIR, 8, 8, 16, 5, 2, 256, PTILE) \
    X(4, P_PAIR, 16, 8, 16, 5, 2, 256, PTILE) X(5, P_PAIR, 8, 8, 8, 1, 2, 256, PTILE) X(6, P_PAIR, 8, 8, 4, 5, 2, 256, TILE) \
    X(7, P_PAIR, 8, 6, 8, 5, 2, 256, PTILE)
#define DFTU_PROJECT_DEFAULT_PAIR P_PAIR, 8, 8, 8, 5, 2, 256, PTILE

cudaError_t launch_project(const View& v, const void* psi, dftu_prec prec, dftu_f64_mode mode, int nbands,
                           int64_t sk, int64_t ss, int64_t sn, int variant, cudaStream_t st, bool gauge) {
    ProjArgs a{psi, sk, ss, sn, nbands};
    cudaError_t e;
    View vp = v;   // the View the projection ran with: its tiling feeds the tile reduce
#define DFTU_CASE_F32(i, POL, Q, CH, NBG, PF, MB, NT, TP) case i: e = run_project<POL, Q, CH, NBG, PF, MB, 0, 1, NT, TP>(v, a, st, &vp); break;
#define DFTU_CASE_PAIR(i, POL, Q, CH, NBG, PF, MB, NT, TP) case i: e = run_project<POL, Q, CH, NBG, PF, MB, 0, 1, NT, TP>(v, a, st, &vp); break;
    if (gauge) {   // one shape per arithmetic policy with the gauge phases (Sec. V)
        if (prec == DFTU_C64) e = run_project<P_F32, 8, 16, 8, 0, 2, 1>(v, a, st);
        else if (mode == DFTU_F64_NATIVE) e = run_project<P_F64, 8, 1, 4, 0, 2, 1>(v, a, st);
        else e = run_project<P_PAIR, 8, 8, 8, 5, 2, 1>(v, a, st);
    } else if (prec == DFTU_C64) {
        switch (variant) {
            DFTU_PROJECT_SHAPES_F32(DFTU_CASE_F32)
            default: e = run_project_default<DFTU_PROJECT_DEFAULT_F32>(v, a, st, &vp); break;
        }
    } else if (mode == DFTU_F64_NATIVE) {
        e = run_project<P_F64, 8, 1, 4, 0>(v, a, st);
    } else {
        switch (variant) {
            DFTU_PROJECT_SHAPES_PAIR(DFTU_CASE_PAIR)
            default: e = run_project_default<DFTU_PROJECT_DEFAULT_PAIR>(v, a, st, &vp); break;
        }
    }
#undef DFTU_CASE_F32
#undef DFTU_CASE_PAIR
    if (e != cudaSuccess) return e;
    int64_t n = (int64_t)v.nk * v.ns * nbands * v.MT;
    k_tile_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(vp, nbands);
    return cudaGetLastError();
}

cudaError_t launch_project_c64_tiles(const View& sub, const void* psi, int nbands, int64_t sk, int64_t ss, int64_t sn,
                                     cudaStream_t st) {
    ProjArgs a{psi, sk, ss, sn, nbands};
    return run_project<P_F32B2F, 16, 8, 4, 0, 3, 0, 1, 256, TILE>(sub, a, st);
}

cudaError_t launch_tile_reduce(const View& v, int nbands, cudaStream_t st) {
    int64_t n = (int64_t)v.nk * v.ns * nbands * v.MT;
    k_tile_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v, nbands);
    return cudaGetLastError();
}

cudaError_t launch_project_dirs(const View& v, const void* psi, dftu_prec prec, dftu_f64_mode mode, int nbands,
                                int64_t sk, int64_t ss, int64_t sn, bool gauge, double2* p_out, int64_t p_stride,
                                cudaStream_t st) {
    ProjArgs a{psi, sk, ss, sn, nbands};
    cudaError_t e;
    // the fixed shapes of the gauge path, with and without the phases
    if (prec == DFTU_C64) e = gauge ? run_project<P_F32, 8, 16, 8, 0, 2, 1, 3>(v, a, st) : run_project<P_F32, 8, 16, 8, 0, 2, 0, 3>(v, a, st);
    else if (mode == DFTU_F64_NATIVE) e = gauge ? run_project<P_F64, 8, 1, 4, 0, 2, 1, 3>(v, a, st) : run_project<P_F64, 8, 1, 4, 0, 2, 0, 3>(v, a, st);
    else e = gauge ? run_project<P_PAIR, 8, 8, 8, 5, 2, 1, 3>(v, a, st) : run_project<P_PAIR, 8, 8, 8, 5, 2, 0, 3>(v, a, st);
    if (e != cudaSuccess) return e;
    int64_t n = (int64_t)v.nk * v.ns * nbands * v.MT;
    for (int d = 0; d < 3; ++d) {
        View vd = v;
        vd.part = v.part + d * v.part_dir_stride;
        vd.p = p_out + d * p_stride;
        k_tile_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(vd, nbands);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int POL, int Q, int CH, int NBG, int PF, int MINB = 2, int NT = CTA>
static cudaError_t run_project_batch(const BatchLaunch& b, cudaStream_t st) {
    size_t smem = TILE * sizeof(int) + (size_t)TILE_PAD * phi_row_bytes(POL, b.maxM);
    cudaError_t e = cudaSuccess;
    auto fn = k_project_batch<POL, Q, CH, NBG, PF, MINB, NT>;
    if (!smem_configured((const void*)fn, (int)smem)) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b.counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    int grid = std::max(1, std::min(per_sm * nsm, b.nitems));
    fn<<<grid, NT, smem, st>>>(b.views, b.args, b.items, b.nitems, b.counter);
    return cudaGetLastError();
}

// The default shape of a table row for the batched launch (always the TILE tiling).
template <int POL, int Q, int CH, int NBG, int PF, int MINB, int NT, int TP>
static cudaError_t run_project_batch_default(const BatchLaunch& b, cudaStream_t st) {
    return run_project_batch<POL, Q, CH, NBG, PF, MINB, NT>(b, st);
}

cudaError_t launch_project_batch(const BatchLaunch& b, dftu_prec prec, dftu_f64_mode mode, int variant, cudaStream_t st) {
    cudaError_t e;
#define DFTU_CASE_F32(i, POL, Q, CH, NBG, PF, MB, NT, TP) case i: e = run_project_batch<POL, Q, CH, NBG, PF, MB, NT>(b, st); break;
#define DFTU_CASE_PAIR(i, POL, Q, CH, NBG, PF, MB, NT, TP) case i: e = run_project_batch<POL, Q, CH, NBG, PF, MB, NT>(b, st); break;
    if (prec == DFTU_C64) {
        switch (variant) {
            DFTU_PROJECT_SHAPES_F32(DFTU_CASE_F32)
            default: e = run_project_batch_default<DFTU_PROJECT_DEFAULT_F32>(b, st); break;
        }
    } else if (mode == DFTU_F64_NATIVE) {
        e = run_project_batch<P_F64, 8, 1, 4, 0>(b, st);
    } else {
        switch (variant) {
            DFTU_PROJECT_SHAPES_PAIR(DFTU_CASE_PAIR)
            default: e = run_project_batch_default<DFTU_PROJECT_DEFAULT_PAIR>(b, st); break;
        }
    }
#undef DFTU_CASE_F32
#undef DFTU_CASE_PAIR
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((b.max_reduce + 255) / 256), b.nsys);
    k_tile_reduce_batch<<<grid, 256, 0, st>>>(b.views, b.args);
    return cudaGetLastError();
}

}  // namespace dftu
