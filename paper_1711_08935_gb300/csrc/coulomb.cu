// Coulomb integrals (mm'|m''m''') on the real-space grid (Sec. III; definition Eq. B2).
// Pair densities phi_c phi_d of one atom are placed on a zero-padded box around its sphere, the
// Hartree potential is solved with FFTs and the truncated Coulomb kernel 4 pi (1 - cos(G Rc)) / G^2
// (2 pi Rc^2 at G = 0), and (ab|cd) = dV sum_j phi_a(j) phi_b(j) v_cd(j).  Box edge >= 2R + Rc per
// axis rounded up to a 2,3,5-smooth size, Rc = 2R + 2 max(h): the potential inside the sphere is
// then free of periodic-image contributions.
#include <cufft.h>

#include <algorithm>
#include <cmath>

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

__global__ void k_scatter_pair(const double* __restrict__ phi, const int* __restrict__ u, int64_t p0, int np, int M, int c,
                               int d, int ux, int uy, int uz, int nb0, int nb1, double2* __restrict__ box) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    int64_t g = p0 + j;
    int x = u[3 * g] - ux, y = u[3 * g + 1] - uy, z = u[3 * g + 2] - uz;
    const double* ph = phi + (int64_t)j * M;
    box[x + (int64_t)nb0 * (y + (int64_t)nb1 * z)] = make_double2(ph[c] * ph[d], 0.0);
}

// Multiply by the truncated Coulomb kernel; frequencies follow the FFT ordering (0..n/2-1, -n/2..-1).
__global__ void k_kernel_mul(double2* __restrict__ box, int nb0, int nb1, int nb2, double h0, double h1, double h2, double Rc) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t n = (int64_t)nb0 * nb1 * nb2;
    if (g >= n) return;
    int x = (int)(g % nb0), y = (int)((g / nb0) % nb1), z = (int)(g / ((int64_t)nb0 * nb1));
    const double tpi = 6.283185307179586476925286766559;
    int fx = (x <= (nb0 - 1) / 2) ? x : x - nb0;
    int fy = (y <= (nb1 - 1) / 2) ? y : y - nb1;
    int fz = (z <= (nb2 - 1) / 2) ? z : z - nb2;
    double gx = tpi * fx / (nb0 * h0), gy = tpi * fy / (nb1 * h1), gz = tpi * fz / (nb2 * h2);
    double G2 = gx * gx + gy * gy + gz * gz;
    double K = (g == 0) ? tpi * Rc * Rc : 2.0 * tpi * (1.0 - cos(sqrt(G2) * Rc)) / G2;   // 2 pi Rc^2 ; 4 pi (1-cos)/G^2
    double2 b = box[g];
    box[g] = make_double2(b.x * K, b.y * K);
}

// W[ab] = scale * sum_j phi_a(j) phi_b(j) Re v(u_j); one CTA per pair (a <= b), fixed-order reduction.
__global__ void k_pair_dot(const double* __restrict__ phi, const int* __restrict__ u, int64_t p0, int np, int M,
                           const double2* __restrict__ box, int ux, int uy, int uz, int nb0, int nb1, double scale,
                           double* __restrict__ Wcol, int P) {
    int pab = blockIdx.x;
    int a = 0, rem = pab;
    while (rem >= M - a) { rem -= M - a; ++a; }
    int b = a + rem;
    __shared__ double red[CTA];
    double acc = 0.0;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        int64_t g = p0 + j;
        int x = u[3 * g] - ux, y = u[3 * g + 1] - uy, z = u[3 * g + 2] - uz;
        const double* ph = phi + (int64_t)j * M;
        acc += ph[a] * ph[b] * box[x + (int64_t)nb0 * (y + (int64_t)nb1 * z)].x;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) Wcol[pab * P] = red[0] * scale;
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

int coulomb_atom(const View& v, const Ctx& c, int atom, double* V_dev, std::string& err) {
    const dftu_atom& at = c.atoms[atom];
    const int M = c.M[atom];
    const int P = M * (M + 1) / 2;
    const double R = at.radius;
    const double hmax = std::max(c.grid.h[0], std::max(c.grid.h[1], c.grid.h[2]));
    const double Rc = 2.0 * R + 2.0 * hmax;
    int nb[3];
    for (int a = 0; a < 3; ++a) nb[a] = smooth235((int)std::ceil((2.0 * R + Rc) / c.grid.h[a]));
    const int64_t N = (int64_t)nb[0] * nb[1] * nb[2];
    const int np = c.npts[atom];
    const int64_t p0 = c.atom_p0[atom];
    const double* phi = v.phi64 + c.atom_phi0[atom];
    const int ux = c.atom_umin[atom][0], uy = c.atom_umin[atom][1], uz = c.atom_umin[atom][2];
    double2* box = nullptr;
    double* W = nullptr;
    cufftHandle plan = 0;
    int rc = DFTU_OK;
    auto fail = [&](int code, const char* msg) { err = msg; rc = code; };
    if (cudaMalloc(&box, N * sizeof(double2)) != cudaSuccess || cudaMalloc(&W, (size_t)P * P * sizeof(double)) != cudaSuccess) {
        fail(DFTU_ERR_ALLOC, "coulomb: device allocation failed");
    } else if (cufftPlan3d(&plan, nb[2], nb[1], nb[0], CUFFT_Z2Z) != CUFFT_SUCCESS) {
        fail(DFTU_ERR_CUDA, "coulomb: cufftPlan3d failed");
        plan = 0;
    } else {
        int pcd = 0;
        for (int cc = 0; cc < M && rc == DFTU_OK; ++cc)
            for (int dd = cc; dd < M && rc == DFTU_OK; ++dd, ++pcd) {
                cudaMemset(box, 0, N * sizeof(double2));
                k_scatter_pair<<<(np + 255) / 256, 256>>>(phi, v.pt_u, p0, np, M, cc, dd, ux, uy, uz, nb[0], nb[1], box);
                if (cufftExecZ2Z(plan, reinterpret_cast<cufftDoubleComplex*>(box), reinterpret_cast<cufftDoubleComplex*>(box),
                                 CUFFT_FORWARD) != CUFFT_SUCCESS) { fail(DFTU_ERR_CUDA, "coulomb: forward FFT failed"); break; }
                k_kernel_mul<<<(unsigned)((N + 255) / 256), 256>>>(box, nb[0], nb[1], nb[2], c.grid.h[0], c.grid.h[1],
                                                                   c.grid.h[2], Rc);
                if (cufftExecZ2Z(plan, reinterpret_cast<cufftDoubleComplex*>(box), reinterpret_cast<cufftDoubleComplex*>(box),
                                 CUFFT_INVERSE) != CUFFT_SUCCESS) { fail(DFTU_ERR_CUDA, "coulomb: inverse FFT failed"); break; }
                k_pair_dot<<<P, CTA>>>(phi, v.pt_u, p0, np, M, box, ux, uy, uz, nb[0], nb[1], v.dV / (double)N, W + pcd, P);
            }
        if (rc == DFTU_OK) {
            k_expand<<<(M * M * M * M + 255) / 256, 256>>>(W, M, P, V_dev);
            cudaError_t e = cudaDeviceSynchronize();
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) fail(DFTU_ERR_CUDA, cudaGetErrorString(e));
        }
    }
    if (plan) cufftDestroy(plan);
    if (box) cudaFree(box);
    if (W) cudaFree(W);
    return rc;
}

}  // namespace dftu
