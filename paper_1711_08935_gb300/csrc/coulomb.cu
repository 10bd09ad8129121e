// Coulomb integrals (mm'|m''m''') on the real-space grid (Sec. III; definition Eq. B2).
// The pair densities phi_c phi_d (c <= d) of one atom are placed on a zero-padded box around its sphere,
// all M(M+1)/2 of them at once; the Hartree potentials come from a 3-D discrete Fourier transform with the
// truncated Coulomb kernel 4 pi (1 - cos(G Rc)) / G^2 (2 pi Rc^2 at G = 0); (ab|cd) = dV sum_j phi_a(j)
// phi_b(j) v_cd(j).  Box edge >= 2R + Rc per axis rounded up to a 2,3,5-smooth size, Rc = 2R + 2 max(h):
// the potential inside the sphere is then free of periodic-image contributions.
//
// The transforms are the library's own: mixed-radix (5, 4, 3, 2) self-sorting Stockham passes along one
// axis at a time, every line of every pair density in one launch per axis, in shared memory, FP64, with
// the roots of unity tabulated once per transform length.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dftu_internal.cuh"

namespace dftu {

static int smooth235(int n) {
    for (int m = std::max(n, 1);; ++m) {
        int k = m;
        for (int p : {2, 3, 5})
            while (k % p == 0) k /= p;
        if (k == 1) return m;
    }
}

constexpr int FFT_MAXN = 512;     // longest transform (box edge) handled
constexpr int FFT_MAXSTAGES = 12;
constexpr int FFT_LINES = 8;      // lines per CTA (adjacent in memory for the strided axes)

struct FftPlan {
    int n;
    int nst;
    int radix[FFT_MAXSTAGES];
};

static bool make_plan(int n, FftPlan& p) {
    p.n = n;
    p.nst = 0;
    int m = n;
    for (int r : {5, 4, 3, 2})
        while (m % r == 0) {
            if (p.nst == FFT_MAXSTAGES) return false;
            p.radix[p.nst++] = r;
            m /= r;
        }
    return m == 1 && n <= FFT_MAXN;
}

// w[k] = exp(-2 pi i k / n), k < n
__global__ void k_fft_roots(double2* w, int n) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)n, &s, &c);
    w[k] = make_double2(c, s);
}

// One pass of FFT_LINES transforms of length n along an axis.  Line L starts at
// (L / inner) * (inner * n) + L % inner and has stride `inner`; lines L .. L + FFT_LINES - 1 of one CTA are
// adjacent in memory when inner > 1.  sign = -1 forward, +1 inverse (unnormalised).
__global__ void __launch_bounds__(256) k_fft_axis(double2* __restrict__ data, int64_t nlines, int64_t inner, FftPlan plan,
                                                  const double2* __restrict__ w, int sign) {
    extern __shared__ double2 fft_smem[];   // two buffers of [FFT_LINES][n]
    const int n = plan.n;
    auto buf = [&](int b, int l, int pos) -> double2& { return fft_smem[((size_t)b * FFT_LINES + l) * n + pos]; };
    const int64_t L0 = (int64_t)blockIdx.x * FFT_LINES;
    auto addr = [&](int64_t L, int pos) -> int64_t { return (L / inner) * (inner * n) + (L % inner) + (int64_t)pos * inner; };
    for (int e = threadIdx.x; e < n * FFT_LINES; e += blockDim.x) {
        const int l = e % FFT_LINES, pos = e / FFT_LINES;
        const int64_t L = L0 + l;
        buf(0, l, pos) = (L < nlines) ? data[addr(L, pos)] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    int src = 0, p = 1;
    for (int s = 0; s < plan.nst; ++s) {
        const int R = plan.radix[s];
        const int T = n / R;
        for (int e = threadIdx.x; e < T * FFT_LINES; e += blockDim.x) {
            const int l = e % FFT_LINES, i = e / FFT_LINES;
            const int k = i % p;
            double2 u[5];
            for (int r = 0; r < R; ++r) {
                double2 x = buf(src, l, i + r * T);
                // twiddle exp(sign 2 pi i k r / (p R)) = w[k r n / (p R)] (conjugated for sign = +1)
                const int idx = (int)(((int64_t)k * r * (n / (p * R))) % n);
                double2 t = w[idx];
                if (sign > 0) t.y = -t.y;
                u[r] = make_double2(x.x * t.x - x.y * t.y, x.x * t.y + x.y * t.x);
            }
            const int j = (i / p) * p * R + k;
            for (int q = 0; q < R; ++q) {
                double re = 0.0, im = 0.0;
                for (int r = 0; r < R; ++r) {
                    const int idx = (int)(((int64_t)q * r % R) * (n / R));
                    double2 t = w[idx];
                    if (sign > 0) t.y = -t.y;
                    re += u[r].x * t.x - u[r].y * t.y;
                    im += u[r].x * t.y + u[r].y * t.x;
                }
                buf(1 - src, l, j + q * p) = make_double2(re, im);
            }
        }
        __syncthreads();
        src = 1 - src;
        p *= R;
    }
    for (int e = threadIdx.x; e < n * FFT_LINES; e += blockDim.x) {
        const int l = e % FFT_LINES, pos = e / FFT_LINES;
        const int64_t L = L0 + l;
        if (L < nlines) data[addr(L, pos)] = buf(src, l, pos);
    }
}

// box[pair][point] = phi_c phi_d for every pair c <= d (pair index in the order of the (c, d) loop).
__global__ void k_scatter_pairs(const double* __restrict__ phi, const int* __restrict__ u, int64_t p0, int np, int M, int P,
                                int ux, int uy, int uz, int nb0, int nb1, int64_t N, double2* __restrict__ box) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (int64_t)np * P) return;
    const int pcd = (int)(g / np), j = (int)(g % np);
    int c = 0, rem = pcd;
    while (rem >= M - c) { rem -= M - c; ++c; }
    const int d = c + rem;
    const int64_t q = p0 + j;
    const int x = u[3 * q] - ux, y = u[3 * q + 1] - uy, z = u[3 * q + 2] - uz;
    const double* ph = phi + (int64_t)j * M;
    box[(int64_t)pcd * N + x + (int64_t)nb0 * (y + (int64_t)nb1 * z)] = make_double2(ph[c] * ph[d], 0.0);
}

// Multiply every pair density's transform by the truncated Coulomb kernel; frequencies in transform
// order (0..n/2-1, -n/2..-1).
__global__ void k_kernel_mul(double2* __restrict__ box, int P, int nb0, int nb1, int nb2, double h0, double h1, double h2, double Rc) {
    const int64_t N = (int64_t)nb0 * nb1 * nb2;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * P) return;
    const int64_t g = e % N;
    const int x = (int)(g % nb0), y = (int)((g / nb0) % nb1), z = (int)(g / ((int64_t)nb0 * nb1));
    const double tpi = 6.283185307179586476925286766559;
    const int fx = (x <= (nb0 - 1) / 2) ? x : x - nb0;
    const int fy = (y <= (nb1 - 1) / 2) ? y : y - nb1;
    const int fz = (z <= (nb2 - 1) / 2) ? z : z - nb2;
    const double gx = tpi * fx / (nb0 * h0), gy = tpi * fy / (nb1 * h1), gz = tpi * fz / (nb2 * h2);
    const double G2 = gx * gx + gy * gy + gz * gz;
    const double K = (g == 0) ? tpi * Rc * Rc : 2.0 * tpi * (1.0 - cos(sqrt(G2) * Rc)) / G2;   // 2 pi Rc^2 ; 4 pi (1-cos)/G^2
    const double2 b = box[e];
    box[e] = make_double2(b.x * K, b.y * K);
}

// W[ab][cd] = scale * sum_j phi_a(j) phi_b(j) Re v_cd(u_j); one CTA per (ab, cd), fixed-order reduction.
__global__ void k_pair_dot(const double* __restrict__ phi, const int* __restrict__ u, int64_t p0, int np, int M, int P,
                           const double2* __restrict__ box, int ux, int uy, int uz, int nb0, int nb1, int64_t N, double scale,
                           double* __restrict__ W) {
    const int pab = blockIdx.x, pcd = blockIdx.y;
    int a = 0, rem = pab;
    while (rem >= M - a) { rem -= M - a; ++a; }
    const int b = a + rem;
    const double2* v = box + (int64_t)pcd * N;
    __shared__ double red[CTA];
    double acc = 0.0;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const int64_t q = p0 + j;
        const int x = u[3 * q] - ux, y = u[3 * q + 1] - uy, z = u[3 * q + 2] - uz;
        const double* ph = phi + (int64_t)j * M;
        acc += ph[a] * ph[b] * v[x + (int64_t)nb0 * (y + (int64_t)nb1 * z)].x;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) W[pab * P + pcd] = red[0] * scale;
}

__global__ void k_expand(const double* __restrict__ W, int M, int P, double* __restrict__ V) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * M * M * M) return;
    int a = e / (M * M * M), b = (e / (M * M)) % M, c = (e / M) % M, d = e % M;
    auto pidx = [M](int x, int y) {
        int lo = x < y ? x : y, hi = x < y ? y : x;
        return lo * M - lo * (lo - 1) / 2 + (hi - lo);
    };
    V[e] = W[pidx(a, b) * P + pidx(c, d)];
}

// 3-D transform of P boxes [P][nb2][nb1][nb0] in place: one pass per axis.
static cudaError_t fft3d(double2* box, int P, const int nb[3], const FftPlan plans[3], double2* const roots[3], int sign,
                         cudaStream_t st) {
    int64_t inner = 1;
    for (int a = 0; a < 3; ++a) {
        const int64_t N = (int64_t)nb[0] * nb[1] * nb[2];
        const int64_t nlines = (int64_t)P * N / nb[a];
        const unsigned blocks = (unsigned)((nlines + FFT_LINES - 1) / FFT_LINES);
        const int smem = 2 * FFT_LINES * nb[a] * (int)sizeof(double2);
        cudaError_t e = cudaSuccess;
        if (smem > 48 * 1024 && !smem_configured((const void*)k_fft_axis, smem))
            e = cudaFuncSetAttribute(k_fft_axis, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        k_fft_axis<<<blocks, 256, smem, st>>>(box, nlines, inner, plans[a], roots[a], sign);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        inner *= nb[a];
    }
    return cudaSuccess;
}

int coulomb_atom(const View& v, const Ctx& c, int atom, double* V_dev, std::string& err) {
    const dftu_atom& at = c.atoms[atom];
    const int M = c.M[atom];
    const int P = M * (M + 1) / 2;
    const double R = at.radius;
    const double hmax = std::max(c.grid.h[0], std::max(c.grid.h[1], c.grid.h[2]));
    const double Rc = 2.0 * R + 2.0 * hmax;
    int nb[3];
    FftPlan plans[3];
    for (int a = 0; a < 3; ++a) {
        nb[a] = smooth235((int)std::ceil((2.0 * R + Rc) / c.grid.h[a]));
        if (!make_plan(nb[a], plans[a])) {
            err = "coulomb: Poisson box edge " + std::to_string(nb[a]) + " exceeds " + std::to_string(FFT_MAXN) + " points";
            return DFTU_ERR_INVALID_ARG;
        }
    }
    const int64_t N = (int64_t)nb[0] * nb[1] * nb[2];
    const int np = c.npts[atom];
    const int64_t p0 = c.atom_p0[atom];
    const double* phi = v.phi64 + c.atom_phi0[atom];
    const int ux = c.atom_umin[atom][0], uy = c.atom_umin[atom][1], uz = c.atom_umin[atom][2];
    // Everything runs on a private stream with stream-ordered scratch: no device-wide synchronisation,
    // only this stream is waited for before the result is returned.
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) { cudaGetLastError(); err = std::string("coulomb: ") + cudaGetErrorString(e); return DFTU_ERR_CUDA; }
    double2* box = nullptr;
    double* W = nullptr;
    double2* roots[3] = {nullptr, nullptr, nullptr};
    size_t nroot = (size_t)nb[0] + nb[1] + nb[2];
    e = cudaMallocAsync(reinterpret_cast<void**>(&box), (size_t)P * N * sizeof(double2), st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&W), (size_t)P * P * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&roots[0]), nroot * sizeof(double2), st);
    if (e == cudaSuccess) {
        roots[1] = roots[0] + nb[0];
        roots[2] = roots[1] + nb[1];
        for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
            k_fft_roots<<<(nb[a] + 127) / 128, 128, 0, st>>>(roots[a], nb[a]);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(box, 0, (size_t)P * N * sizeof(double2), st);
    if (e == cudaSuccess) {
        const int64_t work = (int64_t)np * P;
        k_scatter_pairs<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(phi, v.pt_u, p0, np, M, P, ux, uy, uz, nb[0], nb[1], N, box);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = fft3d(box, P, nb, plans, roots, -1, st);
    if (e == cudaSuccess) {
        k_kernel_mul<<<(unsigned)((N * P + 255) / 256), 256, 0, st>>>(box, P, nb[0], nb[1], nb[2], c.grid.h[0], c.grid.h[1],
                                                                      c.grid.h[2], Rc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = fft3d(box, P, nb, plans, roots, +1, st);
    if (e == cudaSuccess) {
        k_pair_dot<<<dim3(P, P), CTA, 0, st>>>(phi, v.pt_u, p0, np, M, P, box, ux, uy, uz, nb[0], nb[1], N, v.dV / (double)N, W);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_expand<<<(M * M * M * M + 255) / 256, 256, 0, st>>>(W, M, P, V_dev);
        e = cudaGetLastError();
    }
    if (box) cudaFreeAsync(box, st);
    if (W) cudaFreeAsync(W, st);
    if (roots[0]) cudaFreeAsync(roots[0], st);
    cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        err = std::string("coulomb: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DFTU_ERR_ALLOC : DFTU_ERR_CUDA;
    }
    return DFTU_OK;
}

}  // namespace dftu
