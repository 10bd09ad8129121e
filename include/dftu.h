/*
 * dftu.h -- C ABI of the GB300 Hubbard-projector library (libdftu.so).
 *
 * The library implements the data-parallel hot path of self-consistent DFT+U (ACBN0) on a
 * real-space grid, after Tancogne-Dejean, Oliveira and Rubio, "Self-consistent DFT+U method for
 * real-space time-dependent density functional theory calculations":
 *
 *   dftu_setup_atoms   spherical sub-grids and localised orbitals           Sec. II, Fig. 1
 *   dftu_project       p = <phi_{I,m,k} | psi_{n,k}>                         inside Eqs. (4), (6)
 *   dftu_occupations   n^{I,sigma}_{mm'}, Nbar, Pbar                         Eqs. (4), (8), (9), (A2), (B3)
 *   dftu_acbn0_uj      Ubar, Jbar, U_eff, E_U and the potential V            Eqs. (3), (6), (10), (11), (A5), (B5), (B6)
 *   dftu_apply         psi += c * sum_{mm'} V_{mm'} |phi_m><phi_m'|psi>      Eq. (6)
 *
 * Conventions shared by every entry point
 *   - Units are Hartree atomic units (bohr, Hartree).  U, J and E_U are returned in Hartree.
 *   - Grid point (i,j,k) has linear index i + n0*(j + n1*k) and position (i*h0+o0, j*h1+o1, k*h2+o2).
 *   - States are caller-owned DEVICE arrays of interleaved complex numbers (complex128 for
 *     DFTU_C128, complex64 for DFTU_C64).  Layout, with ld_band >= npts elements between bands:
 *       collinear / unpolarised: psi[k][spin][band][ld_band]  (spin extent 2 or 1)
 *       non-collinear:           psi[k][band][component][ld_band] (component extent 2)
 *   - State arrays (psi, work, gradients) may live in this GPU's memory, in managed memory, or in
 *     page-locked host memory (cudaHostAlloc / cudaHostRegister, mapped at the same address), or in
 *     any host memory when the GPU reads pageable memory.  Host-resident states are read and
 *     written by the kernels directly over the host link: only the sphere points move.  Other
 *     pointers are refused with DFTU_ERR_INVALID_ARG; the check is skipped while the stream is
 *     capturing a graph.  The small device inputs (occupations f, the apply coefficient, the vector
 *     potential A) are checked the same way and may also sit in page-locked host memory.
 *   - psi is the full Bloch function on the cell.  A sphere point at unfolded position r_u folds
 *     to r_w = r_u - T; the gather multiplies psi(r_w) by exp(+i k.T), the scatter by exp(-i k.T).
 *   - Occupation matrices are reported as the paper's n_{mm'} = sum w f <psi|phi_m><phi_m'|psi>.
 *     Internally the library holds rho = n^T and applies V = U_eff (1/2 - rho): with complex
 *     projections this is the gradient of E_U (the printed V = U_eff (1/2 - n) is its transpose).
 *   - Spin-unpolarised runs hold one channel whose occupations are per spin; spin sums count it twice.
 *   - Every compute call is asynchronous on the given stream (a cudaStream_t passed as void*;
 *     NULL = legacy default stream) and allocates nothing: all device memory is allocated by
 *     dftu_create and dftu_setup_atoms.  The calls of one handle share its buffers (projections,
 *     tile partials, occupation counters), so they must be ordered: one stream, or streams the
 *     caller orders with events.  Different handles are independent.  Errors detected on the device (non-finite projections,
 *     zero ACBN0 denominators) set bits of a device status word read by dftu_sync_status.
 *   - Return value: DFTU_OK, or an error code; dftu_last_error() gives a message.  On an argument
 *     error nothing is launched and the handle is unchanged.
 */
#ifndef DFTU_H
#define DFTU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dftu_ctx* dftu_handle;
typedef void* dftu_stream; /* a cudaStream_t */

typedef enum {
    DFTU_OK = 0,
    DFTU_ERR_INVALID_ARG = 1,  /* bad argument; nothing was launched */
    DFTU_ERR_NOT_READY = 2,    /* a prerequisite call is missing (setup, Coulomb, project, ...) */
    DFTU_ERR_ALLOC = 3,        /* device or host allocation failed */
    DFTU_ERR_CUDA = 4,         /* a CUDA runtime call or a kernel launch failed */
    DFTU_ERR_NONFINITE = 5,    /* a projection was NaN or infinite (device status) */
    DFTU_ERR_ZERO_DENOM = 6,   /* an ACBN0 denominator was < 1e-14: U = J = 0 for that atom (warning) */
    DFTU_ERR_TIMEOUT = 7       /* a bounded device-side wait gave up (device status) */
} dftu_status;

/* Orthorhombic grid. periodic = 1: the cell repeats; 0: isolated box (sphere points outside it are dropped). */
typedef struct { int n[3]; double h[3]; double origin[3]; int periodic; } dftu_grid;

/* A correlated atom: one shell of angular momentum l (0..3, M = 2l+1 orbitals) on a sphere of the
 * given radius (bohr).  species indexes the radial table and the Coulomb integrals; Nbar (Eq. 9)
 * sums over all atoms of the same species. */
typedef struct { double pos[3]; int species; int l; double radius; } dftu_atom;

/* Radial function R(r) of a species' localised orbital on the uniform grid r_i = i*dr, i < nr (nr >= 4).
 * Host pointer, copied during dftu_setup_atoms.  The library interpolates it with 4-point Lagrange
 * polynomials (nodes a..a+3, a = clamp(floor(r/dr)-1, 0, nr-4)) and takes R = 0 at and beyond r_{nr-1}. */
typedef struct { int nr; double dr; const double* R; } dftu_radial;

typedef enum { DFTU_C128 = 0, DFTU_C64 = 1 } dftu_prec;
typedef enum { DFTU_COLLINEAR = 0, DFTU_UNPOLARIZED = 1, DFTU_NONCOLLINEAR = 2 } dftu_spin;

/* Arithmetic used for DFTU_C128 states.
 *   DFTU_F64_PAIR   (default) products and sums carried as pairs of FP32 numbers on the FP32 pipes,
 *                   about 2^-44 relative; needed because this GPU's FP64 pipe is ~1/70 of its FP32 rate.
 *   DFTU_F64_NATIVE plain FP64 fused multiply-adds. */
typedef enum { DFTU_F64_PAIR = 0, DFTU_F64_NATIVE = 1 } dftu_f64_mode;

/* Create a context on CUDA device `device`.
 *   kvec  host [nk][3] Cartesian k-points, 1/bohr (copied).
 *   wk    host [nk] k-point weights (copied; they should sum to 1).
 *   max_bands  upper bound on the nbands of later calls; sizes the internal buffers.
 * Ownership: the handle owns everything it allocates; release with dftu_destroy. */
dftu_status dftu_create(dftu_handle* out, const dftu_grid* grid, int nk, const double* kvec,
                        const double* wk, dftu_spin spin, int max_bands, int device);

/* Build the spherical sub-grid of every atom (Sec. II, Fig. 1): grid points with
 * (dx*dx + dy*dy) + dz*dz <= R*R in FP64 round-to-nearest without fused multiply-add,
 * dx = (i*h + origin) - X over unfolded integer coordinates, folded into the cell with their
 * lattice image T (|T| <= 2 cells per axis).  Sample phi = R(|d|) Y_lm(d) (real harmonics,
 * m = -l..l: p = y,z,x; d = xy,yz,3z^2-r^2,xz,x^2-y^2) and orthonormalise each atom's orbitals
 * with S^{-1/2}, S = dV phi^T phi (Sec. III assumes an orthogonal basis on each atom).
 * atoms, radials: host arrays (copied).  npts_out: host [natoms] sphere point counts, or NULL.
 * S^{-1/2} exists only for orbitals that are linearly independent on the sphere: an atom whose
 * overlap has lambda_min <= 1e-10 lambda_max (fewer useful points than orbitals, or a radial
 * function that vanishes on the sphere) is refused with DFTU_ERR_INVALID_ARG, as is an atom with
 * no grid point in its sphere; the handle then has no atoms and should be destroyed.
 * Blocking (synchronises the device).  May be called once per handle. */
dftu_status dftu_setup_atoms(dftu_handle h, int natoms, const dftu_atom* atoms, int nspecies,
                             const dftu_radial* radials, int* npts_out);

/* Sphere radii by the second and third methods of Sec. II (the first, the pseudopotential's non-local
 * cut-off, needs a pseudopotential the library does not read).  Host functions; no device work.
 *   dftu_radius_cell:      the smallest edge n_a h_a of the cell.
 *   dftu_radius_threshold: the radius beyond which the tabulated radial function stays below the
 *                          threshold in magnitude: (i + 1) dr for the last node i with |R_i| >= threshold
 *                          (0 when no node reaches it; -1 for an invalid table). */
double dftu_radius_cell(const dftu_grid* grid);
double dftu_radius_threshold(const dftu_radial* radial, double threshold);

/* Copy atom `atom`'s sphere map to host arrays in canonical order (z outer, y, x inner, ascending
 * unfolded coordinates): idx_out [npts] wrapped linear index, image_out [npts][3] lattice image in
 * cells, phi_out [npts][M] orthonormal orbitals (any of the three may be NULL).  Blocking. */
dftu_status dftu_get_sphere(dftu_handle h, int atom, int32_t* idx_out, int32_t* image_out, double* phi_out);

/* Coulomb integrals (mm'|m''m''') of a species (Sec. III; definition Eq. B2), computed on the GPU
 * from the orbitals of the species' first atom: pair densities on a zero-padded box of edge
 * >= 2R + Rc (2,3,5-smooth sizes), Rc = 2R + 2 max(h), FFT Poisson solve with the truncated kernel
 * 4 pi (1 - cos(G Rc)) / G^2 (2 pi Rc^2 at G = 0), then dV sum phi_m phi_m' v_{m''m'''}.
 * The result is stored in the handle for dftu_acbn0_uj; V_out: host [M^4] Hartree, or NULL.  Blocking. */
dftu_status dftu_coulomb_integrals(dftu_handle h, int species, double* V_out);

/* Set a species' Coulomb integrals from host memory instead: V [M][M][M][M] Hartree (copied). */
dftu_status dftu_set_coulomb(dftu_handle h, int species, const double* V);

/* Fixed-U DFT+U for one atom (Sec. II): dftu_acbn0_uj then uses these U, J (Hartree) for it
 * instead of evaluating ACBN0.  U = J = NaN returns the atom to ACBN0. */
dftu_status dftu_set_u(dftu_handle h, int atom, double U, double J);

/* Choose the arithmetic for DFTU_C128 states (see dftu_f64_mode). */
dftu_status dftu_set_f64_mode(dftu_handle h, dftu_f64_mode mode);

/* Kernel variant for one of the streaming kernels (the library's autotuner in the Python binding picks
 * them by timing): which = 0 projection of complex128 states, 1 projection of complex64 states,
 * 2 apply of complex128 states, 3 apply of complex64 states; variant indexes a fixed table of
 * (lanes per band, points per chain, band groups per CTA, prefetch, tile size) shapes, 0 = default.
 * Results do not depend on the variant beyond floating-point summation order.  Batched calls
 * (dftu_batch_*) run every projection shape on 512-point tiles. */
dftu_status dftu_set_kernel_variant(dftu_handle h, int which, int variant);

/* Number of kernel variants available for `which` (see dftu_set_kernel_variant); 0 for a bad `which`. */
int dftu_kernel_variants(int which);

/* Projections p^{k,s}_{I,m,n} = dV sum_j phi_{I,m}(j) exp(+i k.T_j) psi_{k,s,n}(idx_j) of the first
 * nbands bands (nbands <= max_bands) of psi (layout and memory above) onto every atom's orbitals.
 * DFTU_C64 states are multiplied by FP32 orbitals with an FP32 low-part correction, summed in FP32
 * within a point tile and in FP64 across tiles; DFTU_C128 follows dftu_set_f64_mode.
 * The result stays on the device for the calls below. */
dftu_status dftu_project(dftu_handle h, const void* psi, dftu_prec prec, int nbands, int64_t ld_band,
                         dftu_stream stream);

/* Occupations from the last projections, Eq. (4), with Nbar (Eq. 9: sum over the atoms of the same
 * species and all m of |p|^2; non-collinear: also over both spinor components) and Pbar (Eq. 8).
 * f: device FP64 occupations, [nk][spin][nbands] (non-collinear [nk][nbands]), per spin. */
dftu_status dftu_occupations(dftu_handle h, const double* f, dftu_stream stream);

/* Per atom: ACBN0 Ubar and Jbar (Eqs. 10-11 collinear, B5-B6 non-collinear; numerators with
 * Pbar_{mm'} Pbar_{m''m'''} as in Eq. 7, denominators with N_m = n_mm), or the fixed U, J of
 * dftu_set_u; then U_eff = U - J, E_U (Eq. 3 / A5) and V = U_eff (1/2 - n^T) (Eq. 6).
 * A denominator < 1e-14 gives U = J = 0 and sets DFTU_ERR_ZERO_DENOM in the device status. */
dftu_status dftu_acbn0_uj(dftu_handle h, dftu_stream stream);

/* psi_out(idx_j) += c exp(-i k.T_j) sum_m phi_m(j) (V p)_m for every atom and sphere point (Eq. 6),
 * with p from the last dftu_project (which may have read a different array) and V from the last
 * dftu_acbn0_uj.  coef: device pointer to one complex FP64 number c, or NULL for c = 1.
 * accumulate = 0 writes psi_out = c V_U psi_projected on the sphere points instead (other grid points
 * are not touched), so a term vector needs no clearing.  Points shared by several spheres receive
 * every contribution, in a fixed order. */
dftu_status dftu_apply(dftu_handle h, void* psi_out, dftu_prec prec, int nbands, int64_t ld_band,
                       const double* coef, int accumulate, dftu_stream stream);

/* One real-time step with the adiabatic Hubbard potential (Sec. V, Eq. 15): occupations, U and J and
 * V_U are rebuilt from the incoming psi (f: device occupations as for dftu_occupations) and held fixed,
 * then psi <- sum_{j=0}^{order} (-i dt V_U)^j / j! psi.  order <= 8.  Only the Hubbard term of the
 * Hamiltonian is propagated (the paper does not name its propagator; 4th-order Taylor with dt = 0.01 a.u.
 * is the workload's choice).
 * Every term lies in the span of the scattered orbitals, term_j = scatter(a_j), so the step is computed
 * there: a_1 = c_1 V p(psi), a_j = c_j V O a_{j-1} with c_j = -i dt / j and O the overlap of the gathered
 * with the scattered orbitals (the identity on each atom's own points after the Loewdin step, plus the
 * blocks of overlapping spheres and self-overlapping images, built by dftu_setup_atoms), then
 * psi += scatter(sum_j a_j): one projection and one apply of the states per step, the same polynomial in
 * V_U as term-by-term on the grid.  work is not used (it may be NULL; if given it must differ from psi).
 * Afterwards the handle's projections, occupations, U, J and V are those of the incoming psi.
 * Launches only, no host synchronisation and no allocation: a CUDA graph can capture it. */
dftu_status dftu_taylor_step(dftu_handle h, void* psi, void* work, dftu_prec prec, int nbands, int64_t ld_band,
                             const double* f, double dt, int order, dftu_stream stream);

/* nsteps successive real-time steps of dftu_taylor_step (Sec. V, Eq. 15) on psi, each with occupations,
 * U, J and V_U rebuilt from that step's incoming states.  Between two steps nothing but the Hubbard term
 * changes psi, so the gather of step s+1 reads the values the scatter of step s writes: for complex64
 * collinear or unpolarised states without a vector potential, the scatter kernel projects the values it
 * has just written on every tile that no later apply colour touches (the projection of the remaining
 * tiles, where spheres overlap, runs after the last colour), and each step reads and writes every sphere
 * point once.  Other states run the steps one projection and one apply at a time.  The projections use
 * the complex64 projection's arithmetic (compensated FP32 products, FP32 sums within a tile, FP64 across
 * tiles).  Afterwards the handle's projections are those of the outgoing psi, and its occupations, U, J
 * and V those of the last step's incoming psi.  order <= 8, nsteps >= 1.  Launches only, no host
 * synchronisation and no allocation: a CUDA graph can capture it. */
dftu_status dftu_taylor_steps(dftu_handle h, void* psi, dftu_prec prec, int nbands, int64_t ld_band, const double* f,
                              double dt, int order, int nsteps, dftu_stream stream);

/* Gauge-invariant Hubbard operator under a uniform vector potential A (Sec. V, Eq. 16).  Every
 * localised orbital carries the phase exp(-i A.d), d = r - R_I measured from its own atom (the
 * atom-relative reading of Eq. 16), so after this call
 *   dftu_project gives p^A_m = dV sum_j phi_m(j) exp(+i A.d_j) exp(+i k.T_j) psi(idx_j), and
 *   dftu_apply / dftu_taylor_step scatter with exp(-i A.d_j) exp(-i k.T_j),
 * while dftu_occupations and dftu_acbn0_uj are unchanged (they read p^A).  A: device pointer to three
 * FP64 numbers (atomic units, the phase is A.d with d in bohr), read by a kernel on `stream` when it
 * runs, so a graph may capture this call and replay it after A changes.  A = NULL switches the phases
 * off.  Setting A, or clearing one that was set, marks the handle's projections, occupations and
 * potential stale (the next dftu_apply then needs a new dftu_project / occupations / acbn0).
 * Collinear and unpolarised states only (INVALID_ARG for a non-collinear handle with A != NULL);
 * dftu_forces returns INVALID_ARG while A is set.  Launches only, no synchronisation. */
dftu_status dftu_set_vector_potential(dftu_handle h, const double* A, dftu_stream stream);

/* Hubbard contribution to the current (Sec. V, Eq. 17), read as J = sum_{k,n} w_k f <psi| -i [r, V_U^A] |psi>
 * (the printed commutator expectation plus its conjugate vanishes for a Hermitian V_U; the velocity
 * operator's factor i is restored).  With q^(a)_m = <phi_m d_a exp(-i A.d)|psi>,
 *   J_a = mult Im sum_{k,s,n} w_k f sum_{mm'} V_{mm'} [conj(q_m) p_m' - conj(p_m) q_m'],
 * mult = 2 for unpolarised states, and J = dE_U/dA at fixed states.  p and V are those of the last
 * dftu_project (which must have read psi itself, with the same nbands and the current vector potential)
 * and dftu_acbn0_uj.  f: device occupations as for dftu_occupations.  J_out: host [3] (sum over atoms)
 * and/or J_atom_out: host [natoms][3]; either may be NULL, not both.  Collinear and unpolarised states
 * only.  Blocking on stream. */
dftu_status dftu_hubbard_current(dftu_handle h, const void* psi, dftu_prec prec, int nbands, int64_t ld_band,
                                 const double* f, double* J_out, double* J_atom_out, dftu_stream stream);

/* Fully-localised-limit decomposition of the shell energy (App. A) for every atom, with the U and J of
 * the last dftu_acbn0_uj (ACBN0, or the values fixed by dftu_set_u):
 *   E_ee = U/2 sum_s sum_{mm'} n^{ss}_mm n^{-s-s}_m'm' - U/2 sum_s sum_m n^{s-s}_mm n^{-ss}_mm
 *          - J/2 sum_s sum_{m!=m'} n^{s-s}_mm n^{-ss}_m'm' + (U-J)/2 sum_s sum_{m!=m'} n^{ss}_mm n^{ss}_m'm'   (Eq. A1)
 *   E_DC = U/2 N(N-1) - J/2 N(N/2-1) - J/4 m.m,  N = Tr n,  m_i = Tr_s(sigma_i Tr_l n)                (Eq. A3)
 * E_ee is evaluated on the orbital-diagonal entries n^{ss'}_mm, the form the paper prints (it assumes
 * diagonal occupation matrices); E_ee - E_DC equals the Dudarev E_U of Eq. (3) / (A5) when n is
 * orbital-diagonal and collinear.  Collinear handles use the spin-diagonal blocks (an unpolarised
 * channel stands for both spins).  Eee_out, Edc_out: host [natoms] in Hartree, either may be NULL
 * (not both).  Blocking on stream.  The reported E_U and the potential are not changed by this call. */
dftu_status dftu_fll_energy(dftu_handle h, double* Eee_out, double* Edc_out, dftu_stream stream);

/* Hubbard forces (Sec. IV) on every atom, in the form that differentiates the states: with
 * g_a = <phi_a|d_i psi> and p_a = <phi_a|psi>,
 *   F_{I,i} = -sum_{spin blocks} sum_{ab} V_ab sum_{k,n} w_k f [conj(g_a) p_b + conj(p_a) g_b]
 * where V = U_eff (1/2 - n^T) is the potential of the last dftu_acbn0_uj (U_eff held fixed, as in the
 * paper).  dpsi: host array of three device pointers to d psi/dx, d psi/dy, d psi/dz in the layout of
 * psi (the caller computes the gradients, e.g. with its finite-difference stencil).  Requires that the
 * last dftu_project read psi itself, with the same nbands, and dftu_occupations/dftu_acbn0_uj after it.
 * F_out: host [natoms][3], Hartree/bohr.  Blocking on stream. */
dftu_status dftu_forces(dftu_handle h, const void* const* dpsi, dftu_prec prec, int nbands, int64_t ld_band,
                        const double* f, double* F_out, dftu_stream stream);

/* Projection onto ONE atom's orbitals that allocates nothing, for callers that cannot allocate GPU
 * memory (an application or framework that owns the whole device memory pool, a real-time loop where
 * allocation is not allowed, plug-in code that only receives pointers).  It needs no handle: the caller
 * passes every input and the output as device pointers, and the scratch (per-tile partial sums) lives
 * in a fixed 8 MiB array that is part of the library's device image (every GPU that loads the library
 * holds it until the process exits).  The paper has no counterpart; this is a packaging of the
 * projection for such callers.
 *   psi    nbands rows of ld_band complex numbers (complex128 or complex64 per prec), device.
 *   idx    [npts] grid index of each sphere point in a row (0 <= idx < ld_band), device int32.
 *   phase  [npts] complex128 factor of each point (e.g. exp(+i k.T) of its lattice image), device, or NULL for 1.
 *   phi    [npts][M] orbital values (FP64), device.
 *   p_out  [nbands][M] complex128 result, device:  p[n][m] = dV sum_j phi[j][m] phase[j] psi[n][idx[j]], in FP64.
 * Errors: DFTU_ERR_INVALID_ARG for null pointers, a pointer this GPU cannot address (checked as for the
 * states of the handle calls), M outside 1..7, or ceil(npts/512)*nbands*M above 524288 (the scratch
 * size); DFTU_ERR_CUDA if a launch fails (an error the caller left pending is neither reported nor
 * cleared).  A grid index outside [0, ld_band) is never read: the projections of that call then come
 * out NaN.  The first call on a device looks up the
 * scratch array's device address (once per device), so make that first call before any stream
 * capture.  Every call uses the same scratch: calls that overlap on the GPU (other streams, other
 * threads) race and give wrong results; calls ordered on one stream are safe. */
dftu_status dftu_project_sphere_noalloc(const void* psi, dftu_prec prec, int nbands, int64_t ld_band,
                                        const int32_t* idx, const double* phase, const double* phi, int npts,
                                        int M, double dV, double* p_out, dftu_stream stream);

/* The memory-system ceiling of the access pattern, for roofline comparisons: one pass that reads every
 * sphere point of the first nbands states once (rmw = 0, the gather of dftu_project) or reads and writes
 * each back unchanged (rmw = 1, the read-modify-write of dftu_apply), with the same tiles and no
 * arithmetic.  The states' values are not changed.  Not part of the method (the paper has no counterpart);
 * the time of one pass bounds the projection and the apply on this GPU.  Asynchronous on stream. */
dftu_status dftu_access_ceiling(dftu_handle h, void* psi, dftu_prec prec, int nbands, int64_t ld_band, int rmw,
                                dftu_stream stream);

/* ---- Several GPUs: occupation sums over disjoint parts of the (k, band) set -----------------------
 * Eq. (4) and Eq. (8) are sums over k-points and bands of w_k f |p><p| (Pbar with the per-band factor Nbar
 * of Eq. 9, which needs only the projections of that band), so ranks that each hold a disjoint part of the
 * (k, band) set -- every rank a handle with its own k-points (keeping their weights in the whole set) and
 * its own bands and occupations -- form partial sums with dftu_project + dftu_occupations, add them over
 * the ranks (one allreduce of dftu_occupation_elems doubles), and write the totals back before
 * dftu_acbn0_uj, which then gives every rank the U, J, E_U and potential of the whole set; each rank's
 * dftu_apply works on its own states.  The paper's code is single-process; this is the exchange step of
 * the sums it defines.
 *
 * dftu_occupation_elems: the number of doubles of the sums (rho = n^T then Pbar, interleaved complex, in
 *   the library's internal order; the caller only adds them elementwise).  0 before dftu_setup_atoms.
 * dftu_export_occupations: copy this handle's sums of the last dftu_occupations to out (device or page-
 *   locked host memory, dftu_occupation_elems doubles), asynchronously on stream.
 * dftu_import_occupations: overwrite the handle's sums with in (same layout, e.g. the allreduced totals);
 *   dftu_acbn0_uj may follow.  Asynchronous on stream. */
int64_t dftu_occupation_elems(dftu_handle h);
dftu_status dftu_export_occupations(dftu_handle h, double* out, dftu_stream stream);
dftu_status dftu_import_occupations(dftu_handle h, const double* in, dftu_stream stream);

/* ---- Batches of independent systems -------------------------------------------------------------
 * Many small systems (e.g. molecules with their own isolated grids) in one context: every member is an
 * ordinary handle that went through dftu_create/dftu_setup_atoms (and Coulomb integrals or fixed U), all
 * on one device.  The batch launches ONE persistent projection kernel and ONE persistent apply kernel
 * per apply colour over the tiles of all members: every CTA takes (system, tile, k*spin) work items from
 * an atomic counter until the list is exhausted, so uneven systems balance themselves.  The small
 * per-system steps (Nbar, occupations, U/J, potential) run as single batched launches.  Results are
 * read per member with the handle calls above (dftu_get_results etc.); the arithmetic is that of the
 * single-system calls, in the same order per member.  The paper has no counterpart for the batching;
 * it packages Eqs. (4)-(11) for many systems at once.  All members must use the same FP64 mode and
 * have no vector potential set (dftu_set_vector_potential); otherwise dftu_batch_project and
 * dftu_batch_apply return DFTU_ERR_INVALID_ARG. */
typedef struct dftu_batch_ctx* dftu_batch;

/* systems: host array of nsys set-up handles (not owned; they must outlive the batch). */
dftu_status dftu_batch_create(dftu_batch* out, int nsys, const dftu_handle* systems);

/* Bind the members' states and occupations (host arrays of nsys entries): psi[s] device states in the
 * member's layout with nbands[s] bands and ld_band[s] elements per band, f[s] device occupations as for
 * dftu_occupations.  One precision for the whole batch.  Copies a small pointer table to the device. */
dftu_status dftu_batch_bind(dftu_batch b, const void* const* psi, dftu_prec prec, const int* nbands,
                            const int64_t* ld_band, const double* const* f);

dftu_status dftu_batch_project(dftu_batch b, dftu_stream stream);
dftu_status dftu_batch_occupations(dftu_batch b, dftu_stream stream);
dftu_status dftu_batch_acbn0_uj(dftu_batch b, dftu_stream stream);
/* coef: device complex FP64 or NULL for 1; accumulate as for dftu_apply.  Writes the bound states. */
dftu_status dftu_batch_apply(dftu_batch b, const double* coef, int accumulate, dftu_stream stream);
const char* dftu_batch_last_error(dftu_batch b);
void dftu_batch_destroy(dftu_batch b);

/* Results to host memory (blocking on stream).  Any pointer may be NULL.
 *   n_out     [atom][spin][M][M] interleaved complex (paper's n, Eq. 4); non-collinear [atom][2M][2M]
 *             with index (component*M + m); atoms packed one after another with their own M.
 *   U, J, EU_atom  [natoms] Hartree;  EU_total: sum over atoms (Hartree). */
dftu_status dftu_get_results(dftu_handle h, double* n_out, double* U, double* J, double* EU_atom,
                             double* EU_total, dftu_stream stream);

/* Pbar (Eq. 8) in the same layout as n_out, and Nbar [nk][spin][nbands][nspecies] (non-collinear
 * [nk][nbands][nspecies]) to host memory (blocking). */
dftu_status dftu_get_renormalized(dftu_handle h, double* Pbar_out, double* Nbar_out, dftu_stream stream);

/* Last projections to host: [nk][spin or component][nbands][sum_I M_I] interleaved complex (blocking). */
dftu_status dftu_get_projections(dftu_handle h, double* p_out, dftu_stream stream);

/* Number of orbitals summed over atoms (sum_I M_I), and the number of sphere points of an atom. */
int dftu_total_orbitals(dftu_handle h);
int dftu_atom_points(dftu_handle h, int atom);

/* Synchronise the stream of the last compute call and return the device status word as a
 * dftu_status (first set of: NONFINITE, TIMEOUT, ZERO_DENOM), clearing it. */
dftu_status dftu_sync_status(dftu_handle h);

/* Message of the last error on this handle (never NULL; valid until the next call). */
const char* dftu_last_error(dftu_handle h);

/* Release everything the handle owns.  NULL is ignored. */
void dftu_destroy(dftu_handle h);

#ifdef __cplusplus
}
#endif
#endif /* DFTU_H */
