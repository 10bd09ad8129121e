// Projection onto one atom's orbitals without any GPU memory allocation.
//
// Some callers cannot allocate device memory at all: code that runs while another component owns
// the whole device memory pool, real-time loops where an allocation (and the device-wide
// synchronisation cudaMalloc/cudaFree may imply) is not allowed, or plug-in code that only receives
// pointers from its host application.  This entry point takes every input and the output as caller
// pointers and keeps its scratch (per-tile partial sums) in a fixed array that is part of the
// library's device image, so nothing is allocated when it runs.
#include <mutex>

#include "dftu_internal.cuh"

namespace {

constexpr int NA_TILE = 512;                          // sphere points per CTA
constexpr int64_t NA_SCRATCH_ELEMS = 524288;          // complex FP64 partial sums: 8 MiB
constexpr int NA_CTA = 256;
constexpr int NA_MAXDEV = 64;

// Scratch shared by every call on a device; it keeps the previous call's contents.  Every slot a
// call reads is written by the same call first, so nothing needs clearing.
static __device__ __align__(256) double2 g_na_scratch[NA_SCRATCH_ELEMS];

std::mutex g_na_mutex;
double2* g_na_ptr[NA_MAXDEV] = {nullptr};

// partial[tile][band][m] = dV sum_{j in tile} phi[j][m] phase[j] psi[band][idx[j]]   (FP64).
// A grid index outside [0, ld) is never read: the tile then writes NaN partial sums for every band,
// so the projections of the call come out NaN.
template <typename T>
__global__ void __launch_bounds__(NA_CTA) k_na_tiles(const T* __restrict__ psi, int nbands, int64_t ld,
                                                     const int* __restrict__ idx, const double2* __restrict__ phase,
                                                     const double* __restrict__ phi, int npts, int M, double dV,
                                                     double2* __restrict__ part) {
    __shared__ int s_idx[NA_TILE];
    __shared__ double2 s_ph[NA_TILE];
    __shared__ double s_phi[NA_TILE * dftu::MAXM];
    __shared__ int s_bad;
    const int tile = blockIdx.x;
    const int p0 = tile * NA_TILE;
    const int np = min(NA_TILE, npts - p0);
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < np; i += NA_CTA) {
        const int g = idx[p0 + i];
        const bool ok = g >= 0 && (int64_t)g < ld;
        if (!ok) s_bad = 1;
        s_idx[i] = ok ? g : 0;
        s_ph[i] = phase ? phase[p0 + i] : make_double2(1.0, 0.0);
    }
    for (int e = threadIdx.x; e < np * M; e += NA_CTA) s_phi[e] = phi[(int64_t)p0 * M + e];
    __syncthreads();
    const bool bad = s_bad != 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int band = warp; band < nbands; band += NA_CTA / 32) {
        const T* row = psi + (int64_t)band * ld;
        double re[dftu::MAXM], im[dftu::MAXM];
        for (int m = 0; m < M; ++m) { re[m] = 0.0; im[m] = 0.0; }
        for (int i = lane; i < np; i += 32) {
            T x = row[s_idx[i]];
            double xr = (double)x.x, xi = (double)x.y;
            double2 ph = s_ph[i];
            double yr = ph.x * xr - ph.y * xi, yi = ph.x * xi + ph.y * xr;
            for (int m = 0; m < M; ++m) {
                double f = s_phi[i * M + m];
                re[m] += f * yr;
                im[m] += f * yi;
            }
        }
        for (int m = 0; m < M; ++m) {
            for (int off = 16; off > 0; off >>= 1) {
                re[m] += __shfl_xor_sync(0xffffffffu, re[m], off);
                im[m] += __shfl_xor_sync(0xffffffffu, im[m], off);
            }
        }
        if (lane == 0) {
            const double nan = __longlong_as_double(0x7FF8000000000000LL);
            for (int m = 0; m < M; ++m)
                part[((int64_t)tile * nbands + band) * M + m] =
                    bad ? make_double2(nan, nan) : make_double2(dV * re[m], dV * im[m]);
        }
    }
}

// p[band][m] = sum over tiles in order of the partial sums.
__global__ void k_na_reduce(const double2* __restrict__ part, int ntiles, int nbands, int M, double2* __restrict__ p) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nbands * M) return;
    double re = 0.0, im = 0.0;
    for (int t = 0; t < ntiles; ++t) {
        double2 x = part[(int64_t)t * nbands * M + g];
        re += x.x;
        im += x.y;
    }
    p[g] = make_double2(re, im);
}

// Device address of the scratch array on the current device, looked up once per device.
double2* scratch_for_current_device(int& dev) {
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAXDEV) return nullptr;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_na_scratch) != cudaSuccess) return nullptr;
        g_na_ptr[dev] = static_cast<double2*>(ptr);
    }
    return g_na_ptr[dev];
}

}  // namespace

extern "C" dftu_status dftu_project_sphere_noalloc(const void* psi, dftu_prec prec, int nbands, int64_t ld_band,
                                                   const int32_t* idx, const double* phase, const double* phi, int npts,
                                                   int M, double dV, double* p_out, dftu_stream stream) {
    if (!psi || !idx || !phi || !p_out || nbands < 1 || npts < 1 || M < 1 || M > dftu::MAXM || !(dV > 0.0) || ld_band < 1 ||
        (prec != DFTU_C128 && prec != DFTU_C64))
        return DFTU_ERR_INVALID_ARG;
    const int ntiles = (npts + NA_TILE - 1) / NA_TILE;
    if ((int64_t)ntiles * nbands * M > NA_SCRATCH_ELEMS) return DFTU_ERR_INVALID_ARG;   // beyond the fixed scratch
    int dev = -1;
    double2* part = scratch_for_current_device(dev);
    if (!part) return DFTU_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // every operand must be memory this GPU can address (a pageable host array would fault the kernel)
    if (!dftu::gpu_addressable(dev, psi, st) || !dftu::gpu_addressable(dev, idx, st) || !dftu::gpu_addressable(dev, phi, st) ||
        !dftu::gpu_addressable(dev, p_out, st) || (phase && !dftu::gpu_addressable(dev, phase, st)))
        return DFTU_ERR_INVALID_ARG;
    // Launch errors are taken from the launch calls themselves, so an unrelated error the caller left
    // pending is neither reported as ours nor cleared.
    const double2* ph = reinterpret_cast<const double2*>(phase);
    int nt = ntiles;
    void* tile_args[] = {(void*)&psi, (void*)&nbands, (void*)&ld_band, (void*)&idx, (void*)&ph,
                         (void*)&phi, (void*)&npts, (void*)&M, (void*)&dV, (void*)&part};
    const void* fn = (prec == DFTU_C128) ? reinterpret_cast<const void*>(&k_na_tiles<double2>)
                                         : reinterpret_cast<const void*>(&k_na_tiles<float2>);
    cudaError_t e = cudaLaunchKernel(fn, dim3(ntiles), dim3(NA_CTA), tile_args, 0, st);
    if (e == cudaSuccess) {
        double2* p = reinterpret_cast<double2*>(p_out);
        void* red_args[] = {(void*)&part, (void*)&nt, (void*)&nbands, (void*)&M, (void*)&p};
        const int n = nbands * M;
        e = cudaLaunchKernel(reinterpret_cast<const void*>(&k_na_reduce), dim3((n + 255) / 256), dim3(256), red_args, 0, st);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();   // the failed launch is reported here, not left for the caller's next check
        return DFTU_ERR_CUDA;
    }
    return DFTU_OK;
}
