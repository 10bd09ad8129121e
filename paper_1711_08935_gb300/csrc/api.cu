// C ABI entry points of libdftu.so (declared in include/dftu.h): argument checks, the one-off
// geometry set-up (sphere membership on the device, point ordering, tiling and apply colouring on the
// host), buffer ownership, and the asynchronous launches of the hot path.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <cstdio>
#include <cstring>
#include <new>

#include "dftu_internal.cuh"

using namespace dftu;

namespace {

struct Guard {   // sets the context's device for the duration of an entry point
    int prev = -1;
    explicit Guard(int dev) { cudaGetDevice(&prev); cudaSetDevice(dev); }
    ~Guard() { if (prev >= 0) cudaSetDevice(prev); }
};

dftu_status fail(Ctx* c, dftu_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

dftu_status cuda_fail(Ctx* c, cudaError_t e, const char* where) {
    cudaGetLastError();   // a failed allocation or launch must not leak into the caller's next CUDA check
    return fail(c, e == cudaErrorMemoryAllocation ? DFTU_ERR_ALLOC : DFTU_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

template <class T>
cudaError_t dalloc(Ctx* c, T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
    if (e == cudaSuccess) c->allocs.push_back(*p);
    return e;
}

template <class T>
cudaError_t upload(Ctx* c, T** p, const std::vector<T>& h) {
    cudaError_t e = dalloc(c, p, h.size());
    if (e != cudaSuccess) return e;
    if (!h.empty()) e = cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

int64_t floor_div64(int64_t a, int64_t n) {
    int64_t q = a / n;
    return (a % n != 0 && ((a < 0) != (n < 0))) ? q - 1 : q;
}

bool valid_stride_args(Ctx* c, int nbands, int64_t ld) {
    return nbands >= 1 && nbands <= c->max_bands && ld >= (int64_t)c->grid.n[0] * c->grid.n[1] * c->grid.n[2];
}

}  // namespace

bool dftu::gpu_addressable(int device, const void* p, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    if (cs != cudaStreamCaptureStatusNone) return true;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    if (a.type == cudaMemoryTypeDevice) return a.device == device;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer == p;
    int pageable = 0;
    cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device);
    return pageable != 0;
}

namespace {

void strides(const Ctx* c, int nbands, int64_t ld, int64_t& sk, int64_t& ss, int64_t& sn) {
    if (c->spin == DFTU_NONCOLLINEAR) {
        ss = ld;
        sn = 2 * ld;
        sk = (int64_t)nbands * 2 * ld;
    } else {
        sn = ld;
        ss = (int64_t)nbands * ld;
        sk = (int64_t)c->ns * nbands * ld;
    }
}

}  // namespace

extern "C" {

dftu_status dftu_create(dftu_handle* out, const dftu_grid* grid, int nk, const double* kvec, const double* wk,
                        dftu_spin spin, int max_bands, int device) {
    if (!out) return DFTU_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grid || nk < 1 || !kvec || !wk || max_bands < 1 ||
        (spin != DFTU_COLLINEAR && spin != DFTU_UNPOLARIZED && spin != DFTU_NONCOLLINEAR))
        return DFTU_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (grid->n[a] < 1 || !(grid->h[a] > 0.0) || !std::isfinite(grid->origin[a])) return DFTU_ERR_INVALID_ARG;
    if ((int64_t)grid->n[0] * grid->n[1] * grid->n[2] >= (int64_t)1 << 31) return DFTU_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return DFTU_ERR_INVALID_ARG;
    Ctx* c = new (std::nothrow) Ctx();
    if (!c) return DFTU_ERR_ALLOC;
    c->device = device;
    c->grid = *grid;
    c->nk = nk;
    c->spin = spin;
    c->ns = (spin == DFTU_UNPOLARIZED) ? 1 : 2;
    c->max_bands = max_bands;
    c->kvec.assign(kvec, kvec + 3 * nk);
    c->wk.assign(wk, wk + nk);
    Guard g(device);
    View& v = c->v;
    v.n0 = grid->n[0]; v.n1 = grid->n[1]; v.n2 = grid->n[2];
    v.h0 = grid->h[0]; v.h1 = grid->h[1]; v.h2 = grid->h[2];
    v.o0 = grid->origin[0]; v.o1 = grid->origin[1]; v.o2 = grid->origin[2];
    v.periodic = grid->periodic ? 1 : 0;
    v.dV = grid->h[0] * grid->h[1] * grid->h[2];
    v.nk = nk;
    v.ns = c->ns;
    v.noncollinear = spin == DFTU_NONCOLLINEAR;
    v.max_bands = max_bands;
    int* st = nullptr;
    double* one = nullptr;
    cudaError_t e = upload(c, const_cast<double**>(&v.kvec), c->kvec);
    if (e == cudaSuccess) e = upload(c, const_cast<double**>(&v.wk), c->wk);
    if (e == cudaSuccess) e = dalloc(c, &st, 1);
    if (e == cudaSuccess) e = cudaMemset(st, 0, sizeof(int));
    if (e == cudaSuccess) e = upload(c, &one, std::vector<double>{1.0, 0.0});
    if (e == cudaSuccess) e = dalloc(c, &c->d_taylor, 2 * MAX_TAYLOR);
    if (e == cudaSuccess) e = dalloc(c, &c->d_sink, 1);
    if (e != cudaSuccess) {
        for (void* p : c->allocs) cudaFree(p);
        delete c;
        return e == cudaErrorMemoryAllocation ? DFTU_ERR_ALLOC : DFTU_ERR_CUDA;
    }
    v.status = st;
    c->d_coef_one = one;
    *out = reinterpret_cast<dftu_handle>(c);
    return DFTU_OK;
}

dftu_status dftu_setup_atoms(dftu_handle h, int natoms, const dftu_atom* atoms, int nspecies, const dftu_radial* radials,
                             int* npts_out) {
    NvtxRange nvtx_range("dftu_setup_atoms");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (c->atoms_ready) return fail(c, DFTU_ERR_INVALID_ARG, "setup_atoms: already called on this handle");
    if (natoms < 1 || !atoms || nspecies < 1 || !radials) return fail(c, DFTU_ERR_INVALID_ARG, "setup_atoms: bad counts or null arrays");
    std::vector<int> spM(nspecies, -1);
    for (int s = 0; s < nspecies; ++s)
        if (radials[s].nr < 4 || !(radials[s].dr > 0.0) || !radials[s].R)
            return fail(c, DFTU_ERR_INVALID_ARG, "setup_atoms: radial table needs nr >= 4, dr > 0 and data");
    const dftu_grid& G = c->grid;
    for (int a = 0; a < natoms; ++a) {
        const dftu_atom& at = atoms[a];
        if (at.species < 0 || at.species >= nspecies || at.l < 0 || at.l > 3 || !(at.radius > 0.0) ||
            !std::isfinite(at.pos[0]) || !std::isfinite(at.pos[1]) || !std::isfinite(at.pos[2]))
            return fail(c, DFTU_ERR_INVALID_ARG, "setup_atoms: atom " + std::to_string(a) + " has a bad species, l, radius or position");
        int M = 2 * at.l + 1;
        if (spM[at.species] >= 0 && spM[at.species] != M)
            return fail(c, DFTU_ERR_INVALID_ARG, "setup_atoms: atoms of one species must share l");
        spM[at.species] = M;
    }
    for (int s = 0; s < nspecies; ++s)
        if (spM[s] < 0) spM[s] = 1;
    Guard g(c->device);
    View& v = c->v;
    // ---- bounding boxes and device membership flags ----
    std::vector<int> box_lo(3 * natoms), box_dim(3 * natoms);
    std::vector<int64_t> box_off(natoms + 1, 0);
    std::vector<double> pos(3 * natoms), rad(natoms);
    for (int a = 0; a < natoms; ++a) {
        const dftu_atom& at = atoms[a];
        rad[a] = at.radius;
        for (int d = 0; d < 3; ++d) {
            pos[3 * a + d] = at.pos[d];
            double lo = std::floor((at.pos[d] - at.radius - G.origin[d]) / G.h[d]) - 1;
            double hi = std::ceil((at.pos[d] + at.radius - G.origin[d]) / G.h[d]) + 1;
            if (std::fabs(lo) > 1e8 || std::fabs(hi) > 1e8)
                return fail(c, DFTU_ERR_INVALID_ARG, "setup_atoms: sphere too far from the grid");
            box_lo[3 * a + d] = (int)lo;
            box_dim[3 * a + d] = (int)(hi - lo) + 1;
            if (G.periodic) {
                int64_t tlo = floor_div64((int64_t)lo, G.n[d]), thi = floor_div64((int64_t)hi, G.n[d]);
                if (tlo < -IMG_RANGE || thi > IMG_RANGE)
                    return fail(c, DFTU_ERR_INVALID_ARG, "setup_atoms: a sphere reaches beyond two periodic images");
            }
        }
        box_off[a + 1] = box_off[a] + (int64_t)box_dim[3 * a] * box_dim[3 * a + 1] * box_dim[3 * a + 2];
    }
    const int64_t nbox = box_off[natoms];
    std::vector<signed char> flags(nbox);
    {
        double *dpos, *drad;
        int *dlo, *ddim;
        int64_t* doff;
        signed char* dflags;
        cudaError_t e = cudaMalloc(&dpos, pos.size() * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&drad, rad.size() * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&dlo, box_lo.size() * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&ddim, box_dim.size() * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&doff, box_off.size() * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMalloc(&dflags, (size_t)nbox);
        if (e != cudaSuccess) return cuda_fail(c, e, "setup_atoms: temporary allocation");
        cudaMemcpy(dpos, pos.data(), pos.size() * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(drad, rad.data(), rad.size() * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(dlo, box_lo.data(), box_lo.size() * sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy(ddim, box_dim.data(), box_dim.size() * sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy(doff, box_off.data(), box_off.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
        e = launch_sphere_flags(v, dpos, drad, dlo, ddim, doff, natoms, nbox, dflags, 0);
        if (e == cudaSuccess) e = cudaMemcpy(flags.data(), dflags, (size_t)nbox, cudaMemcpyDeviceToHost);
        cudaFree(dpos); cudaFree(drad); cudaFree(dlo); cudaFree(ddim); cudaFree(doff); cudaFree(dflags);
        if (e != cudaSuccess) return cuda_fail(c, e, "setup_atoms: sphere membership");
    }
    // ---- point order: atom-major, then image segment, then canonical (z, y, x) ----
    c->atoms.assign(atoms, atoms + natoms);
    c->nspecies = nspecies;
    c->species_M = spM;
    c->M.resize(natoms); c->moff.resize(natoms); c->mat_off.resize(natoms); c->npts.resize(natoms);
    c->canon_to_gpu.assign(natoms, {});
    c->atom_p0.resize(natoms); c->atom_phi0.resize(natoms);
    c->atom_umin.assign(natoms, std::vector<int>(3, 0));
    std::vector<int> pt_idx, pt_u, seg_T;
    std::vector<int> seg_atom;
    c->tiles.clear();
    std::vector<Tile> ptiles;   // the projection's tiling of the same segments (up to PTILE points)
    int MT = 0, TM = 0, pTM = 0, mat = 0;
    int64_t phi_off = 0;
    const int64_t n0 = G.n[0], n1 = G.n[1], n2 = G.n[2];
    for (int a = 0; a < natoms; ++a) {
        const int M = 2 * atoms[a].l + 1;
        c->M[a] = M;
        c->moff[a] = MT;
        MT += M;
        c->mat_off[a] = mat;
        mat += (c->spin == DFTU_NONCOLLINEAR) ? 4 * M * M : c->ns * M * M;
        int bx = box_dim[3 * a], by = box_dim[3 * a + 1];
        std::vector<std::vector<int64_t>> by_img(NIMG);
        int64_t nin = 0;
        for (int64_t b = 0; b < box_off[a + 1] - box_off[a]; ++b) {
            signed char f = flags[box_off[a] + b];
            if (f < 0) continue;
            by_img[f].push_back(b);
            ++nin;
        }
        if (nin == 0) return fail(c, DFTU_ERR_INVALID_ARG, "setup_atoms: atom " + std::to_string(a) + " has no grid point in its sphere");
        if (nin > (int64_t)1 << 30) return fail(c, DFTU_ERR_INVALID_ARG, "setup_atoms: sphere too large");
        c->npts[a] = (int)nin;
        c->atom_p0[a] = (int64_t)pt_idx.size();
        c->atom_phi0[a] = phi_off;
        // canonical rank of every box point inside the sphere
        std::vector<int64_t> canon_rank(box_off[a + 1] - box_off[a], -1);
        {
            int64_t r = 0;
            for (int64_t b = 0; b < box_off[a + 1] - box_off[a]; ++b)
                if (flags[box_off[a] + b] >= 0) canon_rank[b] = r++;
        }
        c->canon_to_gpu[a].assign(nin, 0);
        int umin[3] = {1 << 30, 1 << 30, 1 << 30};
        int local = 0;
        for (int img = 0; img < NIMG; ++img) {
            const auto& L = by_img[img];
            if (L.empty()) continue;
            int segid = (int)seg_atom.size();
            seg_atom.push_back(a);
            int tx = img % 5 - IMG_RANGE, ty = (img / 5) % 5 - IMG_RANGE, tz = img / 25 - IMG_RANGE;
            if (!G.periodic) tx = ty = tz = 0;
            seg_T.push_back(tx); seg_T.push_back(ty); seg_T.push_back(tz);
            int64_t first = (int64_t)pt_idx.size();
            for (int64_t b : L) {
                int ix = box_lo[3 * a] + (int)(b % bx);
                int jy = box_lo[3 * a + 1] + (int)((b / bx) % by);
                int kz = box_lo[3 * a + 2] + (int)(b / ((int64_t)bx * by));
                int64_t wx = ix - (int64_t)tx * n0, wy = jy - (int64_t)ty * n1, wz = kz - (int64_t)tz * n2;
                int idx = (int)(wx + n0 * (wy + n1 * wz));
                pt_idx.push_back(idx);
                pt_u.push_back(ix); pt_u.push_back(jy); pt_u.push_back(kz);
                umin[0] = std::min(umin[0], ix); umin[1] = std::min(umin[1], jy); umin[2] = std::min(umin[2], kz);
                c->canon_to_gpu[a][canon_rank[b]] = local++;
            }
            int64_t len = (int64_t)pt_idx.size() - first;
            int64_t nt = (len + TILE - 1) / TILE;
            int64_t base = len / nt, rem = len % nt, at = first;
            for (int64_t q = 0; q < nt; ++q) {
                int np = (int)(base + (q < rem ? 1 : 0));
                Tile t{};
                t.atom = a; t.M = M; t.seg = segid; t.np = np; t.p0 = at;
                t.phi0 = phi_off + (at - c->atom_p0[a]) * M;
                t.moff = TM;
                t.color = 0;
                TM += M;
                c->tiles.push_back(t);
                at += np;
            }
            const int64_t npt = (len + PTILE - 1) / PTILE;
            const int64_t pbase = len / npt, prem = len % npt;
            at = first;
            for (int64_t q = 0; q < npt; ++q) {
                int np = (int)(pbase + (q < prem ? 1 : 0));
                Tile t{};
                t.atom = a; t.M = M; t.seg = segid; t.np = np; t.p0 = at;
                t.phi0 = phi_off + (at - c->atom_p0[a]) * M;
                t.moff = pTM;
                t.color = 0;
                pTM += M;
                ptiles.push_back(t);
                at += np;
            }
        }
        for (int d = 0; d < 3; ++d) c->atom_umin[a][d] = umin[d];
        phi_off += nin * M;
    }
    c->MT = MT;
    c->TM = TM;
    c->mat_total = mat;
    c->S = (int64_t)pt_idx.size();
    c->phi_total = phi_off;
    // ---- apply colouring: greedy over tiles, tiles sharing a grid point get different colours ----
    // Colouring tiles rather than whole segments keeps every tile away from an overlap in colour 0, so
    // the later colours hold only the few tiles that reach a shared point.
    const int nseg = (int)seg_atom.size();
    {
        const int64_t npts = n0 * n1 * n2;
        std::vector<std::vector<unsigned char>> used;
        std::vector<int> tile_color(c->tiles.size(), 0);
        for (size_t t = 0; t < c->tiles.size(); ++t) {
            const Tile& tt = c->tiles[t];
            int col = 0;
            for (;; ++col) {
                if (col == (int)used.size()) used.emplace_back(npts, 0);
                bool clash = false;
                for (int i = 0; i < tt.np; ++i)
                    if (used[col][pt_idx[tt.p0 + i]]) { clash = true; break; }
                if (!clash) break;
                if (col >= 255) return fail(c, DFTU_ERR_INVALID_ARG, "setup_atoms: too many overlapping spheres");
            }
            tile_color[t] = col;
            for (int i = 0; i < tt.np; ++i) used[col][pt_idx[tt.p0 + i]] = 1;
        }
        int ncol = used.size();
        c->color_beg.assign(ncol + 1, 0);
        c->color_order.clear();
        for (int col = 0; col < ncol; ++col) {
            c->color_beg[col] = (int)c->color_order.size();
            for (size_t t = 0; t < c->tiles.size(); ++t)
                if (tile_color[t] == col) {
                    c->tiles[t].color = col;
                    c->color_order.push_back((int)t);
                }
        }
        c->color_beg[ncol] = (int)c->color_order.size();
    }
    // ---- first-cover flags: in colour order, the first tile that reaches a grid point owns it ----
    std::vector<unsigned char> pt_first(pt_idx.size(), 0);
    {
        std::vector<unsigned char> written((size_t)(n0 * n1 * n2), 0);
        for (int ti : c->color_order) {
            const Tile& t = c->tiles[ti];
            for (int i = 0; i < t.np; ++i) {
                int idx = pt_idx[t.p0 + i];
                pt_first[t.p0 + i] = written[idx] ? 0 : 1;
                written[idx] = 1;
            }
        }
    }
    // ---- final tiles: no tile of a later apply colour covers any of their points, so the values an apply
    // of their colour leaves are the values after the whole apply (the fused scatter-gather projects them)
    std::vector<unsigned char> tile_final(c->tiles.size(), 1);
    std::vector<Tile> nonfinal;
    {
        std::vector<int> last((size_t)(n0 * n1 * n2), -1);
        for (int ti : c->color_order) {
            const Tile& t = c->tiles[ti];
            for (int i = 0; i < t.np; ++i) last[pt_idx[t.p0 + i]] = ti;
        }
        for (int ti : c->color_order) {
            const Tile& t = c->tiles[ti];
            for (int i = 0; i < t.np; ++i)
                if (last[pt_idx[t.p0 + i]] != ti) { tile_final[ti] = 0; break; }
            if (!tile_final[ti]) nonfinal.push_back(t);
        }
    }
    // ---- per-atom tile ranges, species data, radial tables ----
    std::vector<int> tbeg(natoms, 0), tend(natoms, 0), ptbeg(natoms, 0), ptend(natoms, 0);
    for (size_t t = 0; t < c->tiles.size(); ++t) {
        int a = c->tiles[t].atom;
        if (t == 0 || c->tiles[t - 1].atom != a) tbeg[a] = (int)t;
        tend[a] = (int)t + 1;
    }
    for (size_t t = 0; t < ptiles.size(); ++t) {
        int a = ptiles[t].atom;
        if (t == 0 || ptiles[t - 1].atom != a) ptbeg[a] = (int)t;
        ptend[a] = (int)t + 1;
    }
    std::vector<int> aM(c->M), asp(natoms), amoff(c->moff), amat(c->mat_off);
    for (int a = 0; a < natoms; ++a) asp[a] = atoms[a].species;
    c->coul_off.assign(nspecies, 0);
    int coul_total = 0;
    for (int s = 0; s < nspecies; ++s) { c->coul_off[s] = coul_total; coul_total += spM[s] * spM[s] * spM[s] * spM[s]; }
    std::vector<double> rtab;
    std::vector<int> roff(nspecies), rnr(nspecies);
    std::vector<double> rdr(nspecies);
    for (int s = 0; s < nspecies; ++s) {
        roff[s] = (int)rtab.size();
        rnr[s] = radials[s].nr;
        rdr[s] = radials[s].dr;
        rtab.insert(rtab.end(), radials[s].R, radials[s].R + radials[s].nr);
    }
    std::vector<double> nanv(natoms, std::nan(""));
    cudaError_t e = cudaSuccess;
    Tile* dt = nullptr;
    int *d_idx, *d_u, *d_segT, *d_aM, *d_asp, *d_amoff, *d_amat, *d_tb, *d_te, *d_coff, *d_spM, *d_cset;
    double *d_pos, *d_rad, *d_rtab, *d_rdr, *d_fu, *d_fj, *d_coul;
    int *d_roff, *d_rnr;
    double2* d_segph;
    Tile* dpt = nullptr;
    int *d_ptb = nullptr, *d_pte = nullptr;
    e = upload(c, &dt, c->tiles);
    if (e == cudaSuccess) e = upload(c, &dpt, ptiles);
    if (e == cudaSuccess) e = upload(c, &d_ptb, ptbeg);
    if (e == cudaSuccess) e = upload(c, &d_pte, ptend);
    if (e == cudaSuccess) e = upload(c, &d_idx, pt_idx);
    if (e == cudaSuccess) e = upload(c, &d_u, pt_u);
    unsigned char* d_first = nullptr;
    if (e == cudaSuccess) e = upload(c, &d_first, pt_first);
    unsigned char* d_tfinal = nullptr;
    if (e == cudaSuccess) e = upload(c, &d_tfinal, tile_final);
    c->n_nonfinal = (int)nonfinal.size();
    if (e == cudaSuccess && !nonfinal.empty()) e = upload(c, &c->d_nonfinal_tiles, nonfinal);
    if (e == cudaSuccess) e = upload(c, &d_segT, seg_T);
    if (e == cudaSuccess) e = dalloc(c, &d_segph, (size_t)nseg * c->nk);
    if (e == cudaSuccess) e = upload(c, &d_aM, aM);
    if (e == cudaSuccess) e = upload(c, &d_asp, asp);
    if (e == cudaSuccess) e = upload(c, &d_amoff, amoff);
    if (e == cudaSuccess) e = upload(c, &d_amat, amat);
    if (e == cudaSuccess) e = upload(c, &d_tb, tbeg);
    if (e == cudaSuccess) e = upload(c, &d_te, tend);
    if (e == cudaSuccess) e = upload(c, &d_coff, c->coul_off);
    if (e == cudaSuccess) e = upload(c, &d_spM, spM);
    if (e == cudaSuccess) e = upload(c, &d_pos, pos);
    if (e == cudaSuccess) e = upload(c, &d_rad, rad);
    if (e == cudaSuccess) e = upload(c, &d_rtab, rtab);
    if (e == cudaSuccess) e = upload(c, &d_roff, roff);
    if (e == cudaSuccess) e = upload(c, &d_rnr, rnr);
    if (e == cudaSuccess) e = upload(c, &d_rdr, rdr);
    if (e == cudaSuccess) e = upload(c, &d_fu, nanv);
    if (e == cudaSuccess) e = upload(c, &d_fj, nanv);
    if (e == cudaSuccess) e = upload(c, &d_cset, std::vector<int>(nspecies, 0));
    if (e == cudaSuccess) e = dalloc(c, &d_coul, (size_t)coul_total);
    if (e == cudaSuccess) e = upload(c, &c->d_color_order, c->color_order);
    if (e != cudaSuccess) return cuda_fail(c, e, "setup_atoms: upload");
    v.natoms = natoms; v.nspecies = nspecies; v.MT = MT; v.TM = TM; v.ntiles = (int)c->tiles.size(); v.nseg = nseg;
    v.maxM = *std::max_element(c->M.begin(), c->M.end());
    v.atom_pos = d_pos; v.atom_rad = d_rad; v.atom_M = d_aM; v.atom_species = d_asp; v.atom_moff = d_amoff;
    v.atom_mat_off = d_amat; v.atom_tile_beg = d_tb; v.atom_tile_end = d_te; v.species_coul_off = d_coff; v.species_M = d_spM;
    v.ptiles = dpt; v.nptiles = (int)ptiles.size(); v.pTM = pTM; v.patom_tile_beg = d_ptb; v.patom_tile_end = d_pte;
    v.tiles = dt; v.tile_final = d_tfinal; v.pt_idx = d_idx; v.pt_u = d_u; v.pt_first = d_first; v.seg_T = d_segT; v.seg_phase = d_segph;
    c->h_coul_set.assign(nspecies, 0);
    c->h_fixU.assign(natoms, std::nan(""));
    v.coul = d_coul; v.coul_set = d_cset; v.fixU = d_fu; v.fixJ = d_fj;
    // ---- work buffers ----
    const int rowsP = c->nk * c->ns;
    const int rowsN = (c->spin == DFTU_NONCOLLINEAR) ? c->nk : c->nk * c->ns;
    e = dalloc(c, &v.phi64, (size_t)phi_off);
    if (e == cudaSuccess) e = dalloc(c, &v.phi_hi, (size_t)phi_off);
    if (e == cudaSuccess) e = dalloc(c, &v.phi_lo, (size_t)phi_off);
    if (e == cudaSuccess) e = dalloc(c, &v.p, (size_t)rowsP * c->max_bands * MT);
    v.part_dir_stride = (int64_t)rowsP * c->max_bands * TM;   // three slices: the current's three directions
    if (e == cudaSuccess) e = dalloc(c, &v.part, (size_t)3 * v.part_dir_stride);
    if (e == cudaSuccess) e = dalloc(c, &v.pgrad, (size_t)3 * rowsP * c->max_bands * MT);
    if (e == cudaSuccess) e = dalloc(c, &c->d_forces, (size_t)3 * natoms);
    if (e == cudaSuccess) e = dalloc(c, &c->d_current, (size_t)3 * natoms);
    if (e == cudaSuccess) e = dalloc(c, &c->d_fll, (size_t)2 * natoms);
    if (e == cudaSuccess) e = dalloc(c, &v.gauge_d, (size_t)c->S);
    if (e == cudaSuccess) e = dalloc(c, &v.gauge_f, (size_t)c->S);
    if (e == cudaSuccess) e = dalloc(c, &v.phid64, (size_t)3 * phi_off);
    if (e == cudaSuccess) e = dalloc(c, &v.phid_hi, (size_t)3 * phi_off);
    if (e == cudaSuccess) e = dalloc(c, &v.phid_lo, (size_t)3 * phi_off);
    if (e == cudaSuccess) e = dalloc(c, &v.nbar, (size_t)rowsN * c->max_bands * nspecies);
    if (e == cudaSuccess) e = dalloc(c, &v.rho, (size_t)2 * mat);   // rho, then Pbar: one block for the sharded sums
    if (e == cudaSuccess) v.pbar = v.rho + mat;
    if (e == cudaSuccess) e = dalloc(c, &v.occ_part, (size_t)natoms * 2 * OCC_SPLIT * 2 * OCC_MAXP);
    if (e == cudaSuccess) e = dalloc(c, &v.occ_count, (size_t)natoms * 2);
    if (e == cudaSuccess) e = cudaMemset(v.occ_count, 0, (size_t)natoms * 2 * sizeof(int));
    if (e == cudaSuccess) e = dalloc(c, &v.V, (size_t)mat);
    if (e == cudaSuccess) e = dalloc(c, &v.U, (size_t)natoms);
    if (e == cudaSuccess) e = dalloc(c, &v.J, (size_t)natoms);
    if (e == cudaSuccess) e = dalloc(c, &v.E, (size_t)natoms);
    if (e == cudaSuccess) e = dalloc(c, &v.Etot, 1);
    double* work = nullptr;
    if (e == cudaSuccess) e = dalloc(c, &work, (size_t)natoms * MAXM * MAXM + natoms);   // overlaps, then conditions
    if (e != cudaSuccess) return cuda_fail(c, e, "setup_atoms: work buffers");
    // ---- phases, orbitals, Loewdin ----
    e = launch_seg_phases(v, 0);
    if (e == cudaSuccess) e = launch_orbitals(v, d_rtab, d_roff, d_rnr, d_rdr, 0);
    double* cond = work + (size_t)natoms * MAXM * MAXM;
    if (e == cudaSuccess) e = launch_lowdin(v, work, cond, 0);
    if (e == cudaSuccess) e = launch_displaced_orbitals(v, phi_off, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "setup_atoms: orbitals");
    // S^(-1/2) exists only for orbitals that are linearly independent on the sphere (Sec. III)
    std::vector<double> hcond(natoms);
    e = cudaMemcpy(hcond.data(), cond, sizeof(double) * natoms, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "setup_atoms: overlap conditions");
    for (int a = 0; a < natoms; ++a)
        if (!(hcond[a] > LOWDIN_MIN_RATIO))
            return fail(c, DFTU_ERR_INVALID_ARG, "setup_atoms: the orbitals of atom " + std::to_string(a) +
                                                 " are linearly dependent on its sphere (overlap eigenvalue ratio " +
                                                 std::to_string(hcond[a]) + ")");
    // ---- overlap blocks of the scattered and gathered orbitals (used by the real-time step) ----
    {
        std::vector<double> phi_h((size_t)phi_off);
        e = cudaMemcpy(phi_h.data(), v.phi64, (size_t)phi_off * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "setup_atoms: orbitals to host");
        const int64_t S = c->S;
        std::vector<int> pt_atom((size_t)S), pt_seg((size_t)S);
        for (const Tile& t : c->tiles)
            for (int i = 0; i < t.np; ++i) { pt_atom[t.p0 + i] = t.atom; pt_seg[t.p0 + i] = t.seg; }
        std::vector<std::pair<int, int64_t>> by_idx((size_t)S);
        for (int64_t p = 0; p < S; ++p) by_idx[p] = {pt_idx[p], p};
        std::sort(by_idx.begin(), by_idx.end());
        // key: (I, J, dTx, dTy, dTz) -> M_I x M_J values
        std::map<std::array<int, 5>, std::vector<double>> blocks;
        const double dV = v.dV;
        auto orb = [&](int64_t p) { const int a = pt_atom[p]; return phi_h.data() + c->atom_phi0[a] + (p - c->atom_p0[a]) * c->M[a]; };
        for (size_t g0 = 0; g0 < by_idx.size();) {
            size_t g1 = g0 + 1;
            while (g1 < by_idx.size() && by_idx[g1].first == by_idx[g0].first) ++g1;
            for (size_t x = g0; x < g1; ++x)
                for (size_t y = g0; y < g1; ++y) {
                    const int64_t pa = by_idx[x].second, pb = by_idx[y].second;
                    const int I = pt_atom[pa], J = pt_atom[pb];
                    const int* Ta = &seg_T[3 * pt_seg[pa]];
                    const int* Tb = &seg_T[3 * pt_seg[pb]];
                    std::vector<double>& B = blocks[{I, J, Ta[0] - Tb[0], Ta[1] - Tb[1], Ta[2] - Tb[2]}];
                    const int MI = c->M[I], MJ = c->M[J];
                    if (B.empty()) B.assign((size_t)MI * MJ, 0.0);
                    const double* fa = orb(pa);
                    const double* fb = orb(pb);
                    for (int m = 0; m < MI; ++m)
                        for (int q = 0; q < MJ; ++q) B[(size_t)m * MJ + q] += dV * fa[m] * fb[q];
                }
            g0 = g1;
        }
        std::vector<int> rowptr(natoms + 1, 0), bJ;
        std::vector<int64_t> boff;
        std::vector<double> bdata, bD, bDg;
        for (const auto& kv : blocks) {
            const auto& key = kv.first;
            ++rowptr[key[0] + 1];
            bJ.push_back(key[1]);
            boff.push_back((int64_t)bdata.size());
            bdata.insert(bdata.end(), kv.second.begin(), kv.second.end());
            for (int d = 0; d < 3; ++d) {
                const double Ld = G.periodic ? G.n[d] * G.h[d] : 0.0;
                const double Dd = key[2 + d] * Ld;
                bD.push_back(Dd);
                bDg.push_back(Dd - (atoms[key[0]].pos[d] - atoms[key[1]].pos[d]));
            }
        }
        for (int a = 0; a < natoms; ++a) rowptr[a + 1] += rowptr[a];
        std::vector<int> orb_atom(MT);
        for (int a = 0; a < natoms; ++a)
            for (int m = 0; m < c->M[a]; ++m) orb_atom[c->moff[a] + m] = a;
        int *d_rp = nullptr, *d_bJ = nullptr, *d_oa = nullptr;
        int64_t* d_boff = nullptr;
        double *d_bdata = nullptr, *d_bD = nullptr, *d_bDg = nullptr;
        e = upload(c, &d_rp, rowptr);
        if (e == cudaSuccess) e = upload(c, &d_bJ, bJ);
        if (e == cudaSuccess) e = upload(c, &d_boff, boff);
        if (e == cudaSuccess) e = upload(c, &d_bdata, bdata);
        if (e == cudaSuccess) e = upload(c, &d_bD, bD);
        if (e == cudaSuccess) e = upload(c, &d_bDg, bDg);
        if (e == cudaSuccess) e = upload(c, &d_oa, orb_atom);
        if (e == cudaSuccess) e = dalloc(c, &v.blk_phase, (size_t)c->nk * std::max<size_t>(1, bJ.size()));
        if (e == cudaSuccess) e = dalloc(c, &v.cv, (size_t)rowsP * c->max_bands * MT);
        if (e == cudaSuccess) e = dalloc(c, &v.gaugeA, 3);
        if (e == cudaSuccess) e = cudaMemset(v.gaugeA, 0, 3 * sizeof(double));
        if (e != cudaSuccess) return cuda_fail(c, e, "setup_atoms: overlap blocks");
        v.nblk = (int)bJ.size();
        v.blk_rowptr = d_rp; v.blk_J = d_bJ; v.blk_off = d_boff; v.blk_data = d_bdata; v.blk_D = d_bD; v.blk_Dg = d_bDg;
        v.orb_atom = d_oa;
    }
    if (npts_out)
        for (int a = 0; a < natoms; ++a) npts_out[a] = c->npts[a];
    c->atoms_ready = true;
    return DFTU_OK;
}

double dftu_radius_cell(const dftu_grid* grid) {
    if (!grid) return -1.0;
    double r = grid->n[0] * grid->h[0];
    for (int d = 1; d < 3; ++d) r = std::min(r, grid->n[d] * grid->h[d]);
    return r;
}

double dftu_radius_threshold(const dftu_radial* radial, double threshold) {
    if (!radial || !radial->R || radial->nr < 1 || !(radial->dr > 0.0) || !(threshold > 0.0)) return -1.0;
    for (int i = radial->nr - 1; i >= 0; --i)
        if (std::fabs(radial->R[i]) >= threshold) return (i + 1) * radial->dr;
    return 0.0;
}

dftu_status dftu_get_sphere(dftu_handle h, int atom, int32_t* idx_out, int32_t* image_out, double* phi_out) {
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->atoms_ready) return fail(c, DFTU_ERR_NOT_READY, "get_sphere: call dftu_setup_atoms first");
    if (atom < 0 || atom >= (int)c->atoms.size()) return fail(c, DFTU_ERR_INVALID_ARG, "get_sphere: bad atom");
    Guard g(c->device);
    const int n = c->npts[atom], M = c->M[atom];
    std::vector<int> idx(n), u(3 * (size_t)n);
    std::vector<double> phi((size_t)n * M);
    cudaError_t e = cudaMemcpy(idx.data(), c->v.pt_idx + c->atom_p0[atom], n * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(u.data(), c->v.pt_u + 3 * c->atom_p0[atom], 3 * (size_t)n * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(phi.data(), c->v.phi64 + c->atom_phi0[atom], (size_t)n * M * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_sphere");
    const int* nn = c->grid.n;
    for (int r = 0; r < n; ++r) {
        int gpos = c->canon_to_gpu[atom][r];
        if (idx_out) idx_out[r] = idx[gpos];
        if (image_out) {
            int wx = idx[gpos] % nn[0], wy = (idx[gpos] / nn[0]) % nn[1], wz = idx[gpos] / (nn[0] * nn[1]);
            image_out[3 * r] = (int)floor_div64(u[3 * gpos] - wx, nn[0]);
            image_out[3 * r + 1] = (int)floor_div64(u[3 * gpos + 1] - wy, nn[1]);
            image_out[3 * r + 2] = (int)floor_div64(u[3 * gpos + 2] - wz, nn[2]);
        }
        if (phi_out)
            for (int m = 0; m < M; ++m) phi_out[(size_t)r * M + m] = phi[(size_t)gpos * M + m];
    }
    return DFTU_OK;
}

dftu_status dftu_coulomb_integrals(dftu_handle h, int species, double* V_out) {
    NvtxRange nvtx_range("dftu_coulomb_integrals");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->atoms_ready) return fail(c, DFTU_ERR_NOT_READY, "coulomb_integrals: call dftu_setup_atoms first");
    if (species < 0 || species >= c->nspecies) return fail(c, DFTU_ERR_INVALID_ARG, "coulomb_integrals: bad species");
    int atom = -1;
    for (size_t a = 0; a < c->atoms.size(); ++a)
        if (c->atoms[a].species == species) { atom = (int)a; break; }
    if (atom < 0) return fail(c, DFTU_ERR_INVALID_ARG, "coulomb_integrals: no atom of this species");
    Guard g(c->device);
    double* dst = const_cast<double*>(c->v.coul) + c->coul_off[species];
    int rc = coulomb_atom(c->v, *c, atom, dst, c->err);
    if (rc != DFTU_OK) return (dftu_status)rc;
    int one = 1;
    cudaError_t e = cudaMemcpy(const_cast<int*>(c->v.coul_set) + species, &one, sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) c->h_coul_set[species] = 1;
    const int M = c->M[atom];
    if (e == cudaSuccess && V_out) e = cudaMemcpy(V_out, dst, (size_t)M * M * M * M * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "coulomb_integrals");
    return DFTU_OK;
}

dftu_status dftu_set_coulomb(dftu_handle h, int species, const double* V) {
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->atoms_ready) return fail(c, DFTU_ERR_NOT_READY, "set_coulomb: call dftu_setup_atoms first");
    if (species < 0 || species >= c->nspecies || !V) return fail(c, DFTU_ERR_INVALID_ARG, "set_coulomb: bad species or null V");
    Guard g(c->device);
    const int M = c->species_M[species];
    for (int e = 0; e < M * M * M * M; ++e)
        if (!std::isfinite(V[e])) return fail(c, DFTU_ERR_INVALID_ARG, "set_coulomb: non-finite entry");
    cudaError_t e = cudaMemcpy(const_cast<double*>(c->v.coul) + c->coul_off[species], V, (size_t)M * M * M * M * sizeof(double),
                               cudaMemcpyHostToDevice);
    int one = 1;
    if (e == cudaSuccess) e = cudaMemcpy(const_cast<int*>(c->v.coul_set) + species, &one, sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_coulomb");
    c->h_coul_set[species] = 1;
    return DFTU_OK;
}

dftu_status dftu_set_u(dftu_handle h, int atom, double U, double J) {
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->atoms_ready) return fail(c, DFTU_ERR_NOT_READY, "set_u: call dftu_setup_atoms first");
    if (atom < 0 || atom >= (int)c->atoms.size()) return fail(c, DFTU_ERR_INVALID_ARG, "set_u: bad atom");
    if (std::isnan(U) != std::isnan(J) || std::isinf(U) || std::isinf(J))
        return fail(c, DFTU_ERR_INVALID_ARG, "set_u: U and J must both be finite, or both NaN");
    Guard g(c->device);
    cudaError_t e = cudaMemcpy(const_cast<double*>(c->v.fixU) + atom, &U, sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(const_cast<double*>(c->v.fixJ) + atom, &J, sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_u");
    c->h_fixU[atom] = U;
    return DFTU_OK;
}

dftu_status dftu_set_f64_mode(dftu_handle h, dftu_f64_mode mode) {
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (mode != DFTU_F64_PAIR && mode != DFTU_F64_NATIVE) return fail(c, DFTU_ERR_INVALID_ARG, "set_f64_mode: bad mode");
    c->f64_mode = mode;
    return DFTU_OK;
}

dftu_status dftu_set_kernel_variant(dftu_handle h, int which, int variant) {
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (which < 0 || which > 3 || variant < 0 || variant >= NVARIANTS)
        return fail(c, DFTU_ERR_INVALID_ARG, "set_kernel_variant: which must be 0..3 and variant 0.." + std::to_string(NVARIANTS - 1));
    c->variant[which] = variant;
    return DFTU_OK;
}

int dftu_kernel_variants(int which) { return (which >= 0 && which <= 3) ? NVARIANTS : 0; }

dftu_status dftu_project(dftu_handle h, const void* psi, dftu_prec prec, int nbands, int64_t ld_band, dftu_stream stream) {
    NvtxRange nvtx_range("dftu_project");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->atoms_ready) return fail(c, DFTU_ERR_NOT_READY, "project: call dftu_setup_atoms first");
    if (!psi || (prec != DFTU_C128 && prec != DFTU_C64) || !valid_stride_args(c, nbands, ld_band))
        return fail(c, DFTU_ERR_INVALID_ARG, "project: null psi, bad precision, nbands outside [1, max_bands] or ld_band < npts");
    Guard g(c->device);
    int64_t sk, ss, sn;
    strides(c, nbands, ld_band, sk, ss, sn);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!gpu_addressable(c->device, psi, st)) return fail(c, DFTU_ERR_INVALID_ARG, "project: the states are not addressable by this GPU (device memory of another GPU, or pageable host memory on a device without pageable access)");
    cudaError_t e = launch_project(c->v, psi, prec, c->f64_mode, nbands, sk, ss, sn, c->variant[prec == DFTU_C64 ? 1 : 0], st,
                                   c->gauge_on);
    if (e != cudaSuccess) return cuda_fail(c, e, "project");
    c->last_stream = st;
    c->proj_ready = true;
    c->proj_nbands = nbands;
    return DFTU_OK;
}

dftu_status dftu_occupations(dftu_handle h, const double* f, dftu_stream stream) {
    NvtxRange nvtx_range("dftu_occupations");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->proj_ready) return fail(c, DFTU_ERR_NOT_READY, "occupations: call dftu_project first");
    if (!f) return fail(c, DFTU_ERR_INVALID_ARG, "occupations: null f");
    Guard g(c->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!gpu_addressable(c->device, f, st)) return fail(c, DFTU_ERR_INVALID_ARG, "occupations: f is not addressable by this GPU");
    cudaError_t e = launch_nbar(c->v, c->proj_nbands, st);
    if (e == cudaSuccess) e = launch_occupations(c->v, f, c->proj_nbands, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "occupations");
    c->last_stream = st;
    c->occ_ready = true;
    return DFTU_OK;
}

dftu_status dftu_acbn0_uj(dftu_handle h, dftu_stream stream) {
    NvtxRange nvtx_range("dftu_acbn0_uj");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->occ_ready) return fail(c, DFTU_ERR_NOT_READY, "acbn0_uj: call dftu_occupations first");
    Guard g(c->device);
    for (size_t a = 0; a < c->atoms.size(); ++a)
        if (std::isnan(c->h_fixU[a]) && !c->h_coul_set[c->atoms[a].species])
            return fail(c, DFTU_ERR_NOT_READY, "acbn0_uj: Coulomb integrals of species " + std::to_string(c->atoms[a].species) +
                                                   " not set (dftu_coulomb_integrals or dftu_set_coulomb), and no fixed U");
    cudaError_t e;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    e = launch_acbn0(c->v, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "acbn0_uj");
    c->last_stream = st;
    c->pot_ready = true;
    return DFTU_OK;
}

dftu_status dftu_apply(dftu_handle h, void* psi_out, dftu_prec prec, int nbands, int64_t ld_band, const double* coef,
                       int accumulate, dftu_stream stream) {
    NvtxRange nvtx_range("dftu_apply");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->pot_ready || !c->proj_ready) return fail(c, DFTU_ERR_NOT_READY, "apply: call dftu_project and dftu_acbn0_uj first");
    if (!psi_out || (prec != DFTU_C128 && prec != DFTU_C64) || !valid_stride_args(c, nbands, ld_band) || nbands > c->proj_nbands)
        return fail(c, DFTU_ERR_INVALID_ARG, "apply: null psi, bad precision, ld_band < npts or nbands outside [1, projected bands]");
    Guard g(c->device);
    int64_t sk, ss, sn;
    strides(c, nbands, ld_band, sk, ss, sn);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!gpu_addressable(c->device, psi_out, st)) return fail(c, DFTU_ERR_INVALID_ARG, "apply: the states are not addressable by this GPU (device memory of another GPU, or pageable host memory on a device without pageable access)");
    if (coef && !gpu_addressable(c->device, coef, st)) return fail(c, DFTU_ERR_INVALID_ARG, "apply: coef is not addressable by this GPU");
    cudaError_t e = launch_coefvec(c->v, nbands, st);
    if (e == cudaSuccess)
        e = launch_apply(c->v, psi_out, prec, c->f64_mode, nbands, sk, ss, sn, coef ? coef : c->d_coef_one, c->d_color_order,
                         c->color_beg, c->variant[prec == DFTU_C64 ? 3 : 2], accumulate ? 1 : 0, st, c->gauge_on);
    if (e != cudaSuccess) return cuda_fail(c, e, "apply");
    c->last_stream = st;
    return DFTU_OK;
}

dftu_status dftu_taylor_step(dftu_handle h, void* psi, void* work, dftu_prec prec, int nbands, int64_t ld_band,
                             const double* f, double dt, int order, dftu_stream stream) {
    NvtxRange nvtx_range("dftu_taylor_step");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->atoms_ready) return fail(c, DFTU_ERR_NOT_READY, "taylor_step: call dftu_setup_atoms first");
    if (!psi || psi == work || !f || (prec != DFTU_C128 && prec != DFTU_C64) || !valid_stride_args(c, nbands, ld_band) ||
        order < 1 || order > MAX_TAYLOR || !std::isfinite(dt))
        return fail(c, DFTU_ERR_INVALID_ARG, "taylor_step: null or aliased buffers, bad precision, band count, order or dt");
    for (size_t a = 0; a < c->atoms.size(); ++a)
        if (std::isnan(c->h_fixU[a]) && !c->h_coul_set[c->atoms[a].species])
            return fail(c, DFTU_ERR_NOT_READY, "taylor_step: Coulomb integrals missing for an ACBN0 atom");
    Guard g(c->device);
    int64_t sk, ss, sn;
    strides(c, nbands, ld_band, sk, ss, sn);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!gpu_addressable(c->device, psi, st)) return fail(c, DFTU_ERR_INVALID_ARG, "taylor_step: the states are not addressable by this GPU (device memory of another GPU, or pageable host memory on a device without pageable access)");
    if (!gpu_addressable(c->device, f, st)) return fail(c, DFTU_ERR_INVALID_ARG, "taylor_step: f is not addressable by this GPU");
    const int vp = c->variant[prec == DFTU_C64 ? 1 : 0], va = c->variant[prec == DFTU_C64 ? 3 : 2];
    const bool G = c->gauge_on;
    cudaError_t e = launch_project(c->v, psi, prec, c->f64_mode, nbands, sk, ss, sn, vp, st, G);
    if (e == cudaSuccess) e = launch_nbar(c->v, nbands, st);
    if (e == cudaSuccess) e = launch_occupations(c->v, f, nbands, st);
    if (e == cudaSuccess) e = launch_acbn0(c->v, st);
    if (e == cudaSuccess) e = launch_taylor_coefs(dt, order, c->d_taylor, st);
    // the terms' coefficients in the span of the orbitals, then one scatter of their sum onto psi
    if (e == cudaSuccess) e = launch_taylor_cv(c->v, nbands, order, c->d_taylor, G, st);
    if (e == cudaSuccess)
        e = launch_apply(c->v, psi, prec, c->f64_mode, nbands, sk, ss, sn, c->d_coef_one, c->d_color_order, c->color_beg, va, 1, st, G);
    if (e != cudaSuccess) return cuda_fail(c, e, "taylor_step");
    c->last_stream = st;
    c->proj_ready = c->occ_ready = c->pot_ready = true;
    c->proj_nbands = nbands;
    return DFTU_OK;
}

dftu_status dftu_taylor_steps(dftu_handle h, void* psi, dftu_prec prec, int nbands, int64_t ld_band, const double* f,
                              double dt, int order, int nsteps, dftu_stream stream) {
    NvtxRange nvtx_range("dftu_taylor_steps");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->atoms_ready) return fail(c, DFTU_ERR_NOT_READY, "taylor_steps: call dftu_setup_atoms first");
    if (!psi || !f || (prec != DFTU_C128 && prec != DFTU_C64) || !valid_stride_args(c, nbands, ld_band) ||
        order < 1 || order > MAX_TAYLOR || !std::isfinite(dt) || nsteps < 1)
        return fail(c, DFTU_ERR_INVALID_ARG, "taylor_steps: null buffers, bad precision, band count, order, dt or step count");
    for (size_t a = 0; a < c->atoms.size(); ++a)
        if (std::isnan(c->h_fixU[a]) && !c->h_coul_set[c->atoms[a].species])
            return fail(c, DFTU_ERR_NOT_READY, "taylor_steps: Coulomb integrals missing for an ACBN0 atom");
    Guard g(c->device);
    int64_t sk, ss, sn;
    strides(c, nbands, ld_band, sk, ss, sn);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!gpu_addressable(c->device, psi, st)) return fail(c, DFTU_ERR_INVALID_ARG, "taylor_steps: the states are not addressable by this GPU (device memory of another GPU, or pageable host memory on a device without pageable access)");
    if (!gpu_addressable(c->device, f, st)) return fail(c, DFTU_ERR_INVALID_ARG, "taylor_steps: f is not addressable by this GPU");
    const int vp = c->variant[prec == DFTU_C64 ? 1 : 0], va = c->variant[prec == DFTU_C64 ? 3 : 2];
    const bool G = c->gauge_on;
    // complex64 collinear states without a vector potential: the scatter of each step also gathers the
    // updated states on the final tiles, and a projection of the remaining tiles completes the gather
    const bool fused = prec == DFTU_C64 && c->spin != DFTU_NONCOLLINEAR && !G;
    View sub = c->v;
    sub.tiles = c->d_nonfinal_tiles;
    sub.ntiles = c->n_nonfinal;
    cudaError_t e = launch_project(c->v, psi, prec, c->f64_mode, nbands, sk, ss, sn, vp, st, G);
    if (e == cudaSuccess) e = launch_taylor_coefs(dt, order, c->d_taylor, st);
    for (int step = 0; step < nsteps && e == cudaSuccess; ++step) {
        e = launch_nbar(c->v, nbands, st);
        if (e == cudaSuccess) e = launch_occupations(c->v, f, nbands, st);
        if (e == cudaSuccess) e = launch_acbn0(c->v, st);
        if (e == cudaSuccess) e = launch_taylor_cv(c->v, nbands, order, c->d_taylor, G, st);
        if (e != cudaSuccess) break;
        if (fused) {
            e = launch_apply_project_c64(c->v, psi, nbands, sk, ss, sn, c->d_coef_one, c->d_color_order, c->color_beg, st);
            if (e == cudaSuccess && sub.ntiles > 0) e = launch_project_c64_tiles(sub, psi, nbands, sk, ss, sn, st);
            if (e == cudaSuccess) e = launch_tile_reduce(c->v, nbands, st);
        } else {
            e = launch_apply(c->v, psi, prec, c->f64_mode, nbands, sk, ss, sn, c->d_coef_one, c->d_color_order, c->color_beg, va, 1, st, G);
            if (e == cudaSuccess) e = launch_project(c->v, psi, prec, c->f64_mode, nbands, sk, ss, sn, vp, st, G);
        }
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "taylor_steps");
    c->last_stream = st;
    c->proj_ready = c->occ_ready = c->pot_ready = true;
    c->proj_nbands = nbands;
    return DFTU_OK;
}

dftu_status dftu_forces(dftu_handle h, const void* const* dpsi, dftu_prec prec, int nbands, int64_t ld_band, const double* f,
                        double* F_out, dftu_stream stream) {
    NvtxRange nvtx_range("dftu_forces");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->pot_ready || !c->proj_ready) return fail(c, DFTU_ERR_NOT_READY, "forces: call dftu_project, dftu_occupations and dftu_acbn0_uj first");
    if (c->gauge_on) return fail(c, DFTU_ERR_INVALID_ARG, "forces: not defined with a vector potential set (dftu_set_vector_potential with NULL clears it)");
    if (!dpsi || !dpsi[0] || !dpsi[1] || !dpsi[2] || !f || !F_out || (prec != DFTU_C128 && prec != DFTU_C64) ||
        !valid_stride_args(c, nbands, ld_band) || nbands != c->proj_nbands)
        return fail(c, DFTU_ERR_INVALID_ARG, "forces: null pointers, bad precision, ld_band < npts or nbands differs from the projected states");
    Guard g(c->device);
    int64_t sk, ss, sn;
    strides(c, nbands, ld_band, sk, ss, sn);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int i = 0; i < 3; ++i)
        if (!gpu_addressable(c->device, dpsi[i], st)) return fail(c, DFTU_ERR_INVALID_ARG, "forces: the states are not addressable by this GPU (device memory of another GPU, or pageable host memory on a device without pageable access)");
    if (!gpu_addressable(c->device, f, st)) return fail(c, DFTU_ERR_INVALID_ARG, "forces: f is not addressable by this GPU");
    const int64_t gstride = (int64_t)c->nk * c->ns * c->max_bands * c->MT;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
        View vg = c->v;
        vg.p = c->v.pgrad + i * gstride;   // the gradient projections land in their own buffer
        e = launch_project(vg, dpsi[i], prec, c->f64_mode, nbands, sk, ss, sn, c->variant[prec == DFTU_C64 ? 1 : 0], st);
    }
    if (e == cudaSuccess) e = launch_forces(c->v, f, nbands, c->d_forces, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(F_out, c->d_forces, 3 * c->atoms.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "forces");
    c->last_stream = st;
    return DFTU_OK;
}

dftu_status dftu_set_vector_potential(dftu_handle h, const double* A, dftu_stream stream) {
    NvtxRange nvtx_range("dftu_set_vector_potential");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->atoms_ready) return fail(c, DFTU_ERR_NOT_READY, "set_vector_potential: call dftu_setup_atoms first");
    if (c->spin == DFTU_NONCOLLINEAR && A)
        return fail(c, DFTU_ERR_INVALID_ARG, "set_vector_potential: the gauge-invariant operator is built for collinear and unpolarised states");
    if (!A) {
        if (c->gauge_on) c->proj_ready = c->occ_ready = c->pot_ready = false;   // made with the phases
        c->gauge_on = false;
        return DFTU_OK;
    }
    Guard g(c->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!gpu_addressable(c->device, A, st)) return fail(c, DFTU_ERR_INVALID_ARG, "set_vector_potential: A is not addressable by this GPU");
    cudaError_t e = launch_gauge_phases(c->v, A, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_vector_potential");
    c->gauge_on = true;
    c->proj_ready = c->occ_ready = c->pot_ready = false;   // earlier projections used the previous phases
    c->last_stream = st;
    return DFTU_OK;
}

dftu_status dftu_hubbard_current(dftu_handle h, const void* psi, dftu_prec prec, int nbands, int64_t ld_band, const double* f,
                                 double* J_out, double* J_atom_out, dftu_stream stream) {
    NvtxRange nvtx_range("dftu_hubbard_current");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->pot_ready || !c->proj_ready)
        return fail(c, DFTU_ERR_NOT_READY, "hubbard_current: call dftu_project, dftu_occupations and dftu_acbn0_uj first");
    if (c->spin == DFTU_NONCOLLINEAR) return fail(c, DFTU_ERR_INVALID_ARG, "hubbard_current: collinear and unpolarised states only");
    if (!psi || !f || (!J_out && !J_atom_out) || (prec != DFTU_C128 && prec != DFTU_C64) || !valid_stride_args(c, nbands, ld_band) ||
        nbands != c->proj_nbands)
        return fail(c, DFTU_ERR_INVALID_ARG, "hubbard_current: null pointers, bad precision, ld_band < npts or nbands differs from the projected states");
    Guard g(c->device);
    int64_t sk, ss, sn;
    strides(c, nbands, ld_band, sk, ss, sn);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!gpu_addressable(c->device, psi, st)) return fail(c, DFTU_ERR_INVALID_ARG, "hubbard_current: the states are not addressable by this GPU (device memory of another GPU, or pageable host memory on a device without pageable access)");
    if (!gpu_addressable(c->device, f, st)) return fail(c, DFTU_ERR_INVALID_ARG, "hubbard_current: f is not addressable by this GPU");
    const int64_t gstride = (int64_t)c->nk * c->ns * c->max_bands * c->MT;
    View vq = c->v;   // the same states projected onto phi_m d_a (a = x, y, z) in one launch, into the gradient buffer
    vq.phi64 = c->v.phid64;
    vq.phi_hi = c->v.phid_hi;
    vq.phi_lo = c->v.phid_lo;
    vq.phi_dir_stride = c->phi_total;
    cudaError_t e = launch_project_dirs(vq, psi, prec, c->f64_mode, nbands, sk, ss, sn, c->gauge_on, c->v.pgrad, gstride, st);
    if (e == cudaSuccess) e = launch_current(c->v, f, nbands, c->d_current, st);
    const int na = (int)c->atoms.size();
    std::vector<double> Jat(3 * (size_t)na);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Jat.data(), c->d_current, Jat.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "hubbard_current");
    if (J_atom_out) std::copy(Jat.begin(), Jat.end(), J_atom_out);
    if (J_out) {
        J_out[0] = J_out[1] = J_out[2] = 0.0;
        for (int a = 0; a < na; ++a)
            for (int d = 0; d < 3; ++d) J_out[d] += Jat[3 * a + d];
    }
    c->last_stream = st;
    return DFTU_OK;
}

dftu_status dftu_fll_energy(dftu_handle h, double* Eee_out, double* Edc_out, dftu_stream stream) {
    NvtxRange nvtx_range("dftu_fll_energy");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->pot_ready) return fail(c, DFTU_ERR_NOT_READY, "fll_energy: call dftu_occupations and dftu_acbn0_uj first");
    if (!Eee_out && !Edc_out) return fail(c, DFTU_ERR_INVALID_ARG, "fll_energy: both outputs are NULL");
    Guard g(c->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int na = (int)c->atoms.size();
    std::vector<double> out(2 * (size_t)na);
    cudaError_t e = launch_fll(c->v, c->d_fll, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out.data(), c->d_fll, out.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "fll_energy");
    for (int a = 0; a < na; ++a) {
        if (Eee_out) Eee_out[a] = out[2 * a];
        if (Edc_out) Edc_out[a] = out[2 * a + 1];
    }
    c->last_stream = st;
    return DFTU_OK;
}

dftu_status dftu_get_results(dftu_handle h, double* n_out, double* U, double* J, double* EU_atom, double* EU_total,
                             dftu_stream stream) {
    NvtxRange nvtx_range("dftu_get_results");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if ((n_out && !c->occ_ready) || ((U || J || EU_atom || EU_total) && !c->pot_ready))
        return fail(c, DFTU_ERR_NOT_READY, "get_results: the requested quantities have not been computed");
    Guard g(c->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    const int na = (int)c->atoms.size();
    if (e == cudaSuccess && n_out) {
        std::vector<double2> rho(c->mat_total);
        e = cudaMemcpy(rho.data(), c->v.rho, rho.size() * sizeof(double2), cudaMemcpyDeviceToHost);
        size_t o = 0;
        for (int a = 0; a < na && e == cudaSuccess; ++a) {
            const int M = c->M[a];
            const int D = (c->spin == DFTU_NONCOLLINEAR) ? 2 * M : M;
            const int nb = (c->spin == DFTU_NONCOLLINEAR) ? 1 : c->ns;
            for (int b = 0; b < nb; ++b)
                for (int x = 0; x < D; ++x)
                    for (int y = 0; y < D; ++y) {   // paper's n_{xy} = rho_{yx}
                        double2 r = rho[c->mat_off[a] + (size_t)b * D * D + y * D + x];
                        n_out[2 * o] = r.x;
                        n_out[2 * o + 1] = r.y;
                        ++o;
                    }
        }
    }
    if (e == cudaSuccess && U) e = cudaMemcpy(U, c->v.U, na * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && J) e = cudaMemcpy(J, c->v.J, na * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && EU_atom) e = cudaMemcpy(EU_atom, c->v.E, na * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && EU_total) e = cudaMemcpy(EU_total, c->v.Etot, sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_results");
    return DFTU_OK;
}

dftu_status dftu_access_ceiling(dftu_handle h, void* psi, dftu_prec prec, int nbands, int64_t ld_band, int rmw,
                                dftu_stream stream) {
    NvtxRange nvtx_range("dftu_access_ceiling");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->atoms_ready) return fail(c, DFTU_ERR_NOT_READY, "access_ceiling: call dftu_setup_atoms first");
    if (!psi || (prec != DFTU_C128 && prec != DFTU_C64) || !valid_stride_args(c, nbands, ld_band) || (rmw != 0 && rmw != 1))
        return fail(c, DFTU_ERR_INVALID_ARG, "access_ceiling: null psi, bad precision, band count, ld_band or mode");
    Guard g(c->device);
    int64_t sk, ss, sn;
    strides(c, nbands, ld_band, sk, ss, sn);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!gpu_addressable(c->device, psi, st)) return fail(c, DFTU_ERR_INVALID_ARG, "access_ceiling: the states are not addressable by this GPU");
    cudaError_t e = launch_access_ceiling(c->v, psi, prec, nbands, sk, ss, sn, rmw, c->d_sink, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "access_ceiling");
    c->last_stream = st;
    return DFTU_OK;
}

int64_t dftu_occupation_elems(dftu_handle h) {
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c || !c->atoms_ready) return 0;
    return (int64_t)4 * c->mat_total;
}

dftu_status dftu_export_occupations(dftu_handle h, double* out, dftu_stream stream) {
    NvtxRange nvtx_range("dftu_export_occupations");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->occ_ready) return fail(c, DFTU_ERR_NOT_READY, "export_occupations: call dftu_occupations first");
    if (!out) return fail(c, DFTU_ERR_INVALID_ARG, "export_occupations: null output");
    Guard g(c->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!gpu_addressable(c->device, out, st)) return fail(c, DFTU_ERR_INVALID_ARG, "export_occupations: the output is not addressable by this GPU");
    cudaError_t e = cudaMemcpyAsync(out, c->v.rho, (size_t)2 * c->mat_total * sizeof(double2), cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "export_occupations");
    c->last_stream = st;
    return DFTU_OK;
}

dftu_status dftu_import_occupations(dftu_handle h, const double* in, dftu_stream stream) {
    NvtxRange nvtx_range("dftu_import_occupations");
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->atoms_ready) return fail(c, DFTU_ERR_NOT_READY, "import_occupations: call dftu_setup_atoms first");
    if (!in) return fail(c, DFTU_ERR_INVALID_ARG, "import_occupations: null input");
    Guard g(c->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!gpu_addressable(c->device, in, st)) return fail(c, DFTU_ERR_INVALID_ARG, "import_occupations: the input is not addressable by this GPU");
    cudaError_t e = cudaMemcpyAsync(c->v.rho, in, (size_t)2 * c->mat_total * sizeof(double2), cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "import_occupations");
    c->last_stream = st;
    c->occ_ready = true;
    return DFTU_OK;
}

dftu_status dftu_get_renormalized(dftu_handle h, double* Pbar_out, double* Nbar_out, dftu_stream stream) {
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->occ_ready) return fail(c, DFTU_ERR_NOT_READY, "get_renormalized: call dftu_occupations first");
    Guard g(c->device);
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    const int na = (int)c->atoms.size();
    if (e == cudaSuccess && Pbar_out) {
        std::vector<double2> pb(c->mat_total);
        e = cudaMemcpy(pb.data(), c->v.pbar, pb.size() * sizeof(double2), cudaMemcpyDeviceToHost);
        size_t o = 0;
        for (int a = 0; a < na && e == cudaSuccess; ++a) {
            const int M = c->M[a];
            const int D = (c->spin == DFTU_NONCOLLINEAR) ? 2 * M : M;
            const int nb = (c->spin == DFTU_NONCOLLINEAR) ? 1 : c->ns;
            for (int b = 0; b < nb; ++b)
                for (int x = 0; x < D; ++x)
                    for (int y = 0; y < D; ++y) {
                        double2 r = pb[c->mat_off[a] + (size_t)b * D * D + y * D + x];
                        Pbar_out[2 * o] = r.x;
                        Pbar_out[2 * o + 1] = r.y;
                        ++o;
                    }
        }
    }
    if (e == cudaSuccess && Nbar_out) {
        const int rows = (c->spin == DFTU_NONCOLLINEAR) ? c->nk : c->nk * c->ns;
        const int nb = c->proj_nbands;
        for (int r = 0; r < rows && e == cudaSuccess; ++r)
            e = cudaMemcpy(Nbar_out + (size_t)r * nb * c->nspecies, c->v.nbar + (size_t)r * c->max_bands * c->nspecies,
                           (size_t)nb * c->nspecies * sizeof(double), cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "get_renormalized");
    return DFTU_OK;
}

dftu_status dftu_get_projections(dftu_handle h, double* p_out, dftu_stream stream) {
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    if (!c->proj_ready) return fail(c, DFTU_ERR_NOT_READY, "get_projections: call dftu_project first");
    if (!p_out) return fail(c, DFTU_ERR_INVALID_ARG, "get_projections: null output");
    Guard g(c->device);
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    const int rows = c->nk * c->ns, nb = c->proj_nbands;
    for (int r = 0; r < rows && e == cudaSuccess; ++r)
        e = cudaMemcpy(p_out + 2 * (size_t)r * nb * c->MT, c->v.p + (size_t)r * c->max_bands * c->MT,
                       (size_t)nb * c->MT * sizeof(double2), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_projections");
    return DFTU_OK;
}

int dftu_total_orbitals(dftu_handle h) {
    Ctx* c = reinterpret_cast<Ctx*>(h);
    return (c && c->atoms_ready) ? c->MT : 0;
}

int dftu_atom_points(dftu_handle h, int atom) {
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c || !c->atoms_ready || atom < 0 || atom >= (int)c->atoms.size()) return 0;
    return c->npts[atom];
}

dftu_status dftu_sync_status(dftu_handle h) {
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return DFTU_ERR_INVALID_ARG;
    Guard g(c->device);
    cudaError_t e = cudaStreamSynchronize(c->last_stream);
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, c->v.status, sizeof(int), cudaMemcpyDeviceToHost);
    int zero = 0;
    if (e == cudaSuccess) e = cudaMemcpy(c->v.status, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "sync_status");
    if (st & ST_NONFINITE) return fail(c, DFTU_ERR_NONFINITE, "a projection was not finite");
    if (st & ST_TIMEOUT) return fail(c, DFTU_ERR_TIMEOUT, "a bounded device wait gave up");
    if (st & ST_ZERO_DENOM) return fail(c, DFTU_ERR_ZERO_DENOM, "an ACBN0 denominator was below 1e-14; U = J = 0 there");
    return DFTU_OK;
}

const char* dftu_last_error(dftu_handle h) {
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return "null handle";
    return c->err.c_str();
}

void dftu_destroy(dftu_handle h) {
    Ctx* c = reinterpret_cast<Ctx*>(h);
    if (!c) return;
    {
        Guard g(c->device);
        for (void* p : c->allocs) cudaFree(p);
    }
    delete c;
}

}  // extern "C"
