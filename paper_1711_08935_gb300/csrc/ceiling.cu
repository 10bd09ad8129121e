// The memory-system ceiling of the projector's access pattern: every sphere point of every state read
// once (the projection's gather), or read and written back unchanged (the apply's read-modify-write),
// with no arithmetic.  The tiles, grid order and lanes per band are those of the streaming kernels, so
// the time of one pass bounds what the projection and the apply can reach on this GPU; roofline
// fractions are quoted against it beside the copy bandwidth.
#include "dftu_internal.cuh"

namespace dftu {

template <int B, int Q, int CH, int RMW>
__global__ void __launch_bounds__(CTA) k_access_ceiling(View v, ProjArgs a, int* __restrict__ sink) {
    __shared__ int s_idx[TILE];
    const Tile t = v.tiles[blockIdx.x];
    for (int i = threadIdx.x; i < TILE; i += CTA) s_idx[i] = (i < t.np) ? v.pt_idx[t.p0 + i] : 0;
    __syncthreads();
    constexpr int BPC = CTA / Q;
    const int band = blockIdx.y * BPC + threadIdx.x / Q;
    const int q = threadIdx.x % Q;
    if (band >= a.nbands) return;
    const int k = blockIdx.z / v.ns, s = blockIdx.z % v.ns;
    const int64_t off = (int64_t)k * a.sk + (int64_t)s * a.ss + (int64_t)band * a.sn;
    unsigned acc = 0;
    if (B == 16) {
        int4* row = reinterpret_cast<int4*>(const_cast<void*>(a.psi)) + off;
        for (int i0 = q; i0 < t.np; i0 += Q * CH) {
            int4 x[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int i = i0 + c * Q;
                x[c] = (i < t.np) ? row[s_idx[i]] : make_int4(0, 0, 0, 0);
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int i = i0 + c * Q;
                if (RMW) {
                    if (i < t.np) row[s_idx[i]] = x[c];
                } else {
                    acc ^= (unsigned)(x[c].x ^ x[c].y ^ x[c].z ^ x[c].w);
                }
            }
        }
    } else {
        int2* row = reinterpret_cast<int2*>(const_cast<void*>(a.psi)) + off;
        for (int i0 = q; i0 < t.np; i0 += Q * CH) {
            int2 x[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int i = i0 + c * Q;
                x[c] = (i < t.np) ? row[s_idx[i]] : make_int2(0, 0);
            }
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int i = i0 + c * Q;
                if (RMW) {
                    if (i < t.np) row[s_idx[i]] = x[c];
                } else {
                    acc ^= (unsigned)(x[c].x ^ x[c].y);
                }
            }
        }
    }
    if (!RMW && acc == 0x5bd1e995u) sink[0] = (int)acc;   // keeps the loads; almost never taken
}

template <int B, int Q, int CH, int RMW>
static cudaError_t run_ceiling(const View& v, const ProjArgs& a, int* sink, cudaStream_t st) {
    dim3 grid(v.ntiles, (a.nbands + CTA / Q - 1) / (CTA / Q), v.nk * v.ns);
    k_access_ceiling<B, Q, CH, RMW><<<grid, CTA, 0, st>>>(v, a, sink);
    return cudaGetLastError();
}

cudaError_t launch_access_ceiling(const View& v, void* psi, dftu_prec prec, int nbands, int64_t sk, int64_t ss, int64_t sn,
                                  int rmw, int* sink, cudaStream_t st) {
    ProjArgs a{psi, sk, ss, sn, nbands};
    // the fastest layouts of this pattern: 128 contiguous bytes per band and instruction
    if (prec == DFTU_C128) return rmw ? run_ceiling<16, 16, 4, 1>(v, a, sink, st) : run_ceiling<16, 8, 8, 0>(v, a, sink, st);
    return rmw ? run_ceiling<8, 16, 8, 1>(v, a, sink, st) : run_ceiling<8, 16, 8, 0>(v, a, sink, st);
}

}  // namespace dftu
