// Internal definitions shared by the translation units of libdftu.so.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "dftu.h"

#include <nvtx3/nvToolsExt.h>

namespace dftu {

// Names an entry point on profiler timelines (NVTX range for the lifetime of the object; a no-op when no
// profiler is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int TILE = 512;      // sphere points per tile (one CTA stages a tile in shared memory)
constexpr int PTILE = 1024;    // sphere points per tile of the projection's own tiling (View::ptiles)
constexpr int TILE_PAD = TILE + 128;   // staged orbital rows incl. zero padding read by chained loops (Q*CH <= 128)
constexpr int MAXM = 7;        // orbitals per shell, l <= 3
constexpr int IMG_RANGE = 2;   // lattice images |T| <= 2 cells per axis
constexpr int NIMG = 125;      // (2*IMG_RANGE+1)^3 image ids
constexpr int CTA = 256;       // threads per CTA of the streaming kernels
constexpr int MAX_TAYLOR = 8;  // highest Taylor order of dftu_taylor_step
constexpr int OCC_SPLIT = 8;   // CTAs sharing the (k, band) sum of one occupation matrix
constexpr int OCC_MAXP = (2 * MAXM) * (2 * MAXM);   // largest matrix (non-collinear f shell), elements
constexpr double LOWDIN_MIN_RATIO = 1e-10;   // smallest accepted lambda_min / lambda_max of an atom's orbital
                                            // overlap; below it S^(-1/2) is refused (orbitals dependent)

enum StatusBits : int { ST_NONFINITE = 1, ST_ZERO_DENOM = 2, ST_TIMEOUT = 4 };

// A tile: up to TILE consecutive points of one (atom, image) segment in GPU point order.
struct Tile {
    int atom;
    int M;          // orbitals of the atom
    int seg;        // image segment (row of the phase table)
    int np;         // points in the tile
    int64_t p0;     // first point, GPU order
    int64_t phi0;   // element offset of the first point's orbital values ([point][M] layout)
    int moff;       // slot of this tile's M partial sums in a row of the per-tile partial buffer
    int color;      // apply colour: tiles of one colour touch disjoint grid points
};

// Everything a kernel may need, passed by value.
struct View {
    int n0, n1, n2;
    double h0, h1, h2, o0, o1, o2;
    int periodic;
    double dV;
    int nk;
    int ns;           // stored spin channels (collinear 2, unpolarised 1) or spinor components (2)
    int noncollinear;
    int natoms, nspecies;
    int MT;           // sum over atoms of M
    int TM;           // sum over tiles of M
    int ntiles, nseg;
    int max_bands;
    int maxM;         // largest shell present (sizes the staged orbital rows)

    const double* kvec;      // [nk][3]
    const double* wk;        // [nk]
    const double* atom_pos;  // [natoms][3]
    const double* atom_rad;  // [natoms]
    const int* atom_M;
    const int* atom_species;
    const int* atom_moff;     // offset of the atom's orbitals in [MT]
    const int* atom_mat_off;  // offset of the atom's matrices (complex elements) in rho/pbar/V
    const int* atom_tile_beg; // tiles of atom I are [beg, end) in tile order
    const int* atom_tile_end;
    const int* species_coul_off;  // offset of (mm'|m''m''') of each species in coul
    const int* species_M;

    const Tile* tiles;
    const unsigned char* tile_final;   // [ntiles] 1 if no tile of a later apply colour covers any of its points
    // The projection's own tiling: the same image segments cut into tiles of up to PTILE points (half
    // the tile epilogues and partial sums of TILE-point tiles).  A projection launch that uses it swaps
    // these into its copy of the View for tiles, ntiles, TM and atom_tile_beg/end, so k_tile_reduce
    // follows unchanged; the partial buffer, sized for TM >= pTM, serves both.
    const Tile* ptiles;
    int nptiles, pTM;
    const int* patom_tile_beg;
    const int* patom_tile_end;
    const int* pt_idx;     // [S] wrapped linear index, GPU order
    const int* pt_u;       // [S][3] unfolded integer coordinates, GPU order
    const unsigned char* pt_first;   // [S] 1 if no tile of an earlier apply colour covers this grid point
    double2* gauge_d;      // [S] (cos, sin) of A.d_j, d_j = point minus atom centre (Sec. V, Eq. 16)
    float4* gauge_f;       // [S] the same as FP32 pairs (cos_hi, sin_hi, cos_lo, sin_lo)
    double* phid64;        // [3][sum S_I M_I] orbitals times the displacement component d_a (Eq. 17)
    float* phid_hi;        // [3][sum S_I M_I] FP32 split of phid64
    float* phid_lo;
    double* phi64;         // [sum S_I M_I]
    float* phi_hi;
    float* phi_lo;
    const int* seg_T;      // [nseg][3] lattice image of each segment, in cells
    double2* seg_phase;    // [nseg][nk] exp(+i k.T)

    double2* p;            // [nk*ns][max_bands][MT]
    double2* pgrad;        // [3][nk*ns][max_bands][MT] projections of the state gradients (forces)
    double2* part;         // [3][nk*ns][max_bands][TM]: one slice per direction of a three-table projection
    int64_t phi_dir_stride;    // elements between the orbital tables of successive directions (0: one table)
    int64_t part_dir_stride;   // elements between the partial-sum slices of successive directions
    double* nbar;          // collinear [nk*ns][max_bands][nspecies]; non-collinear [nk][max_bands][nspecies]
    double2* rho;          // per atom: collinear [ns][M][M]; non-collinear [2M][2M]   (rho = n^T)
    double2* pbar;         // same layout, renormalised (Eq. 8), transposed like rho
    double2* occ_part;     // [natoms][2][OCC_SPLIT][2][OCC_MAXP] partial rho / Pbar sums of the split CTAs
    int* occ_count;        // [natoms][2] CTAs done per matrix; zero between launches
    double2* V;            // same layout, U_eff (1/2 - rho)
    const double* coul;
    const int* coul_set;   // [nspecies] 1 if set
    double2* cv;           // [nk*ns][max_bands][MT] coefficient vectors the apply scatters: V p, or the sum
                           // of the Taylor terms' coefficients (dftu_taylor_step)
    const int* orb_atom;   // [MT] atom of each orbital slot
    // Overlap of the scattered orbitals with the gathered ones, by blocks of atom pairs (I, J) that share
    // grid points, per lattice-image difference: B[m][m'] = dV sum phi_Im(a) phi_Jm'(b) over point pairs
    // (a of I, b of J) on the same grid point.  Rows of the block list are grouped by I.
    int nblk;
    const int* blk_rowptr;    // [natoms + 1]
    const int* blk_J;         // [nblk]
    const int64_t* blk_off;   // [nblk] offset of the block's M_I x M_J values in blk_data
    const double* blk_data;
    const double* blk_D;      // [nblk][3] image difference (T_a - T_b) L, bohr
    const double* blk_Dg;     // [nblk][3] the same minus (R_I - R_J): d_a - d_b of the gauge phases
    double2* blk_phase;       // [nk][nblk] exp(+i k.D) (times exp(+i A.Dg) with a vector potential)
    double* gaugeA;           // [3] the vector potential of the last dftu_set_vector_potential
    double* U;
    double* J;
    double* E;             // [natoms]
    double* Etot;          // [1]
    const double* fixU;    // [natoms] NaN = ACBN0
    const double* fixJ;
    int* status;
};

// Host-side context behind dftu_handle.
struct Ctx {
    int device = 0;
    dftu_grid grid{};
    dftu_spin spin = DFTU_COLLINEAR;
    int nk = 0, ns = 1, max_bands = 0;
    dftu_f64_mode f64_mode = DFTU_F64_PAIR;
    std::vector<double> kvec, wk;
    bool atoms_ready = false, proj_ready = false, occ_ready = false, pot_ready = false;
    int proj_nbands = 0;
    int variant[4] = {0, 0, 0, 0};   // project c128, project c64, apply c128, apply c64
    bool gauge_on = false;           // dftu_set_vector_potential with a non-null A
    cudaStream_t last_stream = nullptr;
    std::string err;

    // atoms
    std::vector<dftu_atom> atoms;
    std::vector<int> M, moff, mat_off, npts, species_M, coul_off;
    std::vector<std::vector<int>> canon_to_gpu;   // per atom: canonical point -> GPU-order point
    std::vector<int64_t> atom_p0, atom_phi0;       // first GPU-order point / phi element of each atom
    std::vector<Tile> tiles;
    std::vector<int> color_order;                  // tile indices grouped by colour
    std::vector<int> color_beg;                    // colour c is color_order[color_beg[c] .. color_beg[c+1])
    std::vector<std::vector<int>> atom_umin;        // per atom minimum unfolded coordinate
    int nspecies = 0, MT = 0, TM = 0, mat_total = 0;
    int64_t S = 0, phi_total = 0;

    View v{};
    std::vector<void*> allocs;   // every device allocation, freed by dftu_destroy
    int* d_color_order = nullptr;
    Tile* d_nonfinal_tiles = nullptr;   // copies of the tiles that are not final (tile_final == 0), colour order
    int n_nonfinal = 0;
    double* d_coef_one = nullptr;
    double* d_taylor = nullptr;      // [MAX_TAYLOR] complex Taylor coefficients -i dt / j
    double* d_forces = nullptr;      // [natoms][3]
    double* d_current = nullptr;     // [natoms][3] per-atom Hubbard current
    double* d_fll = nullptr;         // [natoms][2] E_ee, E_DC of App. A
    int* d_sink = nullptr;           // [1] output of the access-ceiling pass
    std::vector<int> h_coul_set;     // host copies, so hot-path calls never read the device
    std::vector<double> h_fixU;
};

// Arguments of a streaming kernel for one system's states: base pointer, element strides of k, spin (or
// spinor component) and band, and the number of bands.
struct ProjArgs {
    const void* psi;
    int64_t sk, ss, sn;
    int nbands;
};

// Device tables of a batch of systems for the persistent kernels.
struct BatchLaunch {
    const View* views;        // [nsys]
    const ProjArgs* args;     // [nsys]
    const double* const* f;   // [nsys] occupations, device pointers
    const int4* items;        // (system, tile, k*spin, 0) work items, all tiles
    int nitems;
    const int4* color_items;  // work items of the apply, grouped by colour
    std::vector<int> color_beg;
    int* counter;             // work-queue counter (reset before each persistent launch)
    int nsys;
    int maxM;
    int64_t max_reduce;       // max over systems of (k*spin rows) * nbands * sum M
    int max_rows_nbar;        // max over systems of rows * nbands * species (the Nbar threads)
    int max_atoms, max_ns;
};

// ---- launchers implemented in the .cu files (all asynchronous on `st`) -------------------------
cudaError_t launch_sphere_flags(const View& v, const double* pos, const double* rad, const int* box_lo,
                                const int* box_dim, const int64_t* box_off, int natoms, int64_t nbox,
                                signed char* flags, cudaStream_t st);
cudaError_t launch_seg_phases(const View& v, cudaStream_t st);
cudaError_t launch_orbitals(const View& v, const double* radial_tab, const int* radial_off,
                            const int* radial_nr, const double* radial_dr, cudaStream_t st);
cudaError_t launch_lowdin(const View& v, double* work_S, double* cond, cudaStream_t st);

constexpr int NVARIANTS = 8;   // shapes per streaming kernel (see dftu_set_kernel_variant)
cudaError_t launch_project(const View& v, const void* psi, dftu_prec prec, dftu_f64_mode mode, int nbands,
                           int64_t sk, int64_t ss, int64_t sn, int variant, cudaStream_t st, bool gauge = false);
cudaError_t launch_nbar(const View& v, int nbands, cudaStream_t st);
cudaError_t launch_occupations(const View& v, const double* f, int nbands, cudaStream_t st);
cudaError_t launch_acbn0(const View& v, cudaStream_t st);
cudaError_t launch_apply(const View& v, void* psi, dftu_prec prec, dftu_f64_mode mode, int nbands,
                         int64_t sk, int64_t ss, int64_t sn, const double* coef, const int* color_order,
                         const std::vector<int>& color_beg, int variant, int accumulate, cudaStream_t st,
                         bool gauge = false);
// The complex64 scatter (accumulate, coefficient coef) fused with the gather of the updated states on the
// final tiles (View::tile_final): their partial sums land in v.part (TILE tiling) as a projection writes them.
cudaError_t launch_apply_project_c64(const View& v, void* psi, int nbands, int64_t sk, int64_t ss, int64_t sn,
                                     const double* coef, const int* color_order, const std::vector<int>& color_beg,
                                     cudaStream_t st);
// Complex64 projection partial sums of the tiles of `sub` only (a View whose tiles are a subset of the TILE
// tiling, with that tiling's TM), without the tile reduce.
cudaError_t launch_project_c64_tiles(const View& sub, const void* psi, int nbands, int64_t sk, int64_t ss, int64_t sn,
                                     cudaStream_t st);
// p from the partial sums of v's tiling (Bloch phase per segment, dV).
cudaError_t launch_tile_reduce(const View& v, int nbands, cudaStream_t st);
cudaError_t launch_gauge_phases(const View& v, const double* A, cudaStream_t st);
// cv = V p for the first nbands bands (the coefficients the apply scatters).
cudaError_t launch_coefvec(const View& v, int nbands, cudaStream_t st);
// One pass of the access pattern alone: read (rmw = 0) or read and write back unchanged (rmw = 1) every
// sphere point of the states, no arithmetic; sink: one device int the read pass may write.
cudaError_t launch_access_ceiling(const View& v, void* psi, dftu_prec prec, int nbands, int64_t sk, int64_t ss, int64_t sn,
                                  int rmw, int* sink, cudaStream_t st);
cudaError_t launch_coefvec_batch(const BatchLaunch& b, cudaStream_t st);
// Taylor step in the span of the orbitals: cv = sum_{j=1}^{order} c_j V p_{j-1}, p_0 = p, p_j = c_j O V p_{j-1}
// (O: the block overlap above), coefs = the order complex c_j on the device.
cudaError_t launch_taylor_cv(const View& v, int nbands, int order, const double* coefs, bool gauge, cudaStream_t st);
// Projections onto three orbital tables (v.phi* + a * v.phi_dir_stride, a = 0..2) in one launch, the
// directions interleaved per tile so that the three reads of a tile's states share L2; results go to
// p_out + a * p_stride.
cudaError_t launch_project_dirs(const View& v, const void* psi, dftu_prec prec, dftu_f64_mode mode, int nbands,
                                int64_t sk, int64_t ss, int64_t sn, bool gauge, double2* p_out, int64_t p_stride,
                                cudaStream_t st);
cudaError_t launch_displaced_orbitals(const View& v, int64_t phi_total, cudaStream_t st);
cudaError_t launch_current(const View& v, const double* f, int nbands, double* Jat, cudaStream_t st);
cudaError_t launch_taylor_coefs(double dt, int order, double* coefs, cudaStream_t st);
cudaError_t launch_forces(const View& v, const double* f, int nbands, double* F, cudaStream_t st);
cudaError_t launch_fll(const View& v, double* out, cudaStream_t st);
// True when GPU `device` can address p: its own or managed memory, page-locked host memory mapped at
// the same address (cudaHostAlloc / cudaHostRegister), or any host memory when the device reads
// pageable memory (address translation over the host link).  While `st` is capturing a graph the
// check is skipped (pointers are checked when the work is set up eagerly).
bool gpu_addressable(int device, const void* p, cudaStream_t st);
cudaError_t launch_project_batch(const BatchLaunch& b, dftu_prec prec, dftu_f64_mode mode, int variant, cudaStream_t st);
cudaError_t launch_occupations_batch(const BatchLaunch& b, cudaStream_t st);
cudaError_t launch_acbn0_batch(const BatchLaunch& b, cudaStream_t st);
cudaError_t launch_apply_batch(const BatchLaunch& b, dftu_prec prec, dftu_f64_mode mode, int variant, const double* coef,
                               int accumulate, cudaStream_t st);

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per kernel and device, never inside a capture.
bool smem_configured(const void* fn, int bytes);

// Coulomb integrals of one atom's orbitals (blocking); W_out [P][P] with P = M(M+1)/2 pair index.
int coulomb_atom(const View& v, const Ctx& c, int atom, double* V_dev, std::string& err);

}  // namespace dftu
