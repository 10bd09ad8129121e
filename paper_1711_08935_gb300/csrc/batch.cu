// Batches of independent systems: one persistent launch per streaming kernel over the tiles of every
// member system, plus batched launches of the small per-system kernels.  Each member is an ordinary
// handle (its own grid, atoms, k-points, spin and buffers); the batch only adds device tables of the
// members' views, state pointers and work items.
#include <algorithm>
#include <cmath>
#include <new>

#include "dftu_internal.cuh"

using namespace dftu;

struct dftu_batch_ctx {
    int device = 0;
    std::vector<Ctx*> members;
    std::string err;
    bool bound = false;
    dftu_prec prec = DFTU_C128;
    BatchLaunch L{};
    View* d_views = nullptr;
    ProjArgs* d_args = nullptr;
    const double** d_f = nullptr;
    int4* d_items = nullptr;
    int4* d_color_items = nullptr;
    int* d_counter = nullptr;
    std::vector<int> nbands;
};

namespace {

dftu_status bfail(dftu_batch_ctx* b, dftu_status s, const std::string& m) {
    b->err = m;
    return s;
}

void free_tables(dftu_batch_ctx* b) {
    cudaFree(b->d_args);
    cudaFree(b->d_f);
    b->d_args = nullptr;
    b->d_f = nullptr;
}

}  // namespace

extern "C" {

dftu_status dftu_batch_create(dftu_batch* out, int nsys, const dftu_handle* systems) {
    if (!out) return DFTU_ERR_INVALID_ARG;
    *out = nullptr;
    if (nsys < 1 || !systems) return DFTU_ERR_INVALID_ARG;
    auto* b = new (std::nothrow) dftu_batch_ctx();
    if (!b) return DFTU_ERR_ALLOC;
    for (int i = 0; i < nsys; ++i) {
        Ctx* c = reinterpret_cast<Ctx*>(systems[i]);
        if (!c || !c->atoms_ready || (i > 0 && c->device != b->members[0]->device)) {
            delete b;
            return DFTU_ERR_INVALID_ARG;
        }
        b->members.push_back(c);
    }
    b->device = b->members[0]->device;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    std::vector<View> views;
    std::vector<int4> items;
    int ncol = 0;
    for (auto* c : b->members) ncol = std::max(ncol, (int)c->color_beg.size() - 1);
    std::vector<std::vector<int4>> by_color(ncol);
    BatchLaunch& L = b->L;
    L.nsys = nsys;
    L.maxM = 1;
    L.max_atoms = 1;
    L.max_ns = 1;
    for (int s = 0; s < nsys; ++s) {
        Ctx* c = b->members[s];
        views.push_back(c->v);
        L.maxM = std::max(L.maxM, c->v.maxM);
        L.max_atoms = std::max(L.max_atoms, (int)c->atoms.size());
        L.max_ns = std::max(L.max_ns, c->spin == DFTU_NONCOLLINEAR ? 1 : c->ns);
        const int rows = c->nk * c->ns;
        for (int t = 0; t < (int)c->tiles.size(); ++t)
            for (int ks = 0; ks < rows; ++ks) items.push_back(make_int4(s, t, ks, 0));
        for (int col = 0; col + 1 < (int)c->color_beg.size(); ++col)
            for (int q = c->color_beg[col]; q < c->color_beg[col + 1]; ++q)
                for (int ks = 0; ks < rows; ++ks) by_color[col].push_back(make_int4(s, c->color_order[q], ks, 0));
    }
    std::vector<int4> citems;
    L.color_beg.assign(1, 0);
    for (auto& v : by_color) {
        citems.insert(citems.end(), v.begin(), v.end());
        L.color_beg.push_back((int)citems.size());
    }
    cudaError_t e = cudaMalloc(&b->d_views, views.size() * sizeof(View));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_views, views.data(), views.size() * sizeof(View), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, items.size() * sizeof(int4));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_color_items, std::max<size_t>(1, citems.size()) * sizeof(int4));
    if (e == cudaSuccess && !citems.empty())
        e = cudaMemcpy(b->d_color_items, citems.data(), citems.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int));
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaFree(b->d_views); cudaFree(b->d_items); cudaFree(b->d_color_items); cudaFree(b->d_counter);
        delete b;
        return e == cudaErrorMemoryAllocation ? DFTU_ERR_ALLOC : DFTU_ERR_CUDA;
    }
    L.views = b->d_views;
    L.items = b->d_items;
    L.nitems = (int)items.size();
    L.color_items = b->d_color_items;
    L.counter = b->d_counter;
    *out = b;
    return DFTU_OK;
}

dftu_status dftu_batch_bind(dftu_batch b, const void* const* psi, dftu_prec prec, const int* nbands, const int64_t* ld_band,
                            const double* const* f) {
    if (!b) return DFTU_ERR_INVALID_ARG;
    if (!psi || !nbands || !ld_band || !f || (prec != DFTU_C128 && prec != DFTU_C64))
        return bfail(b, DFTU_ERR_INVALID_ARG, "batch_bind: null arrays or bad precision");
    const int n = (int)b->members.size();
    std::vector<ProjArgs> args(n);
    int64_t max_reduce = 1;
    int max_rows = 1;
    for (int s = 0; s < n; ++s) {
        Ctx* c = b->members[s];
        const int64_t npts = (int64_t)c->grid.n[0] * c->grid.n[1] * c->grid.n[2];
        if (!psi[s] || !f[s] || nbands[s] < 1 || nbands[s] > c->max_bands || ld_band[s] < npts)
            return bfail(b, DFTU_ERR_INVALID_ARG, "batch_bind: system " + std::to_string(s) + " has a null pointer, bad band count or ld_band");
        if (!gpu_addressable(b->device, psi[s], nullptr) || !gpu_addressable(b->device, f[s], nullptr))
            return bfail(b, DFTU_ERR_INVALID_ARG, "batch_bind: the states or occupations of system " + std::to_string(s) + " are not addressable by this GPU");
        ProjArgs a{};
        a.psi = psi[s];
        a.nbands = nbands[s];
        if (c->spin == DFTU_NONCOLLINEAR) {
            a.ss = ld_band[s]; a.sn = 2 * ld_band[s]; a.sk = (int64_t)nbands[s] * 2 * ld_band[s];
        } else {
            a.sn = ld_band[s]; a.ss = (int64_t)nbands[s] * ld_band[s]; a.sk = (int64_t)c->ns * nbands[s] * ld_band[s];
        }
        args[s] = a;
        max_reduce = std::max<int64_t>(max_reduce, (int64_t)c->nk * c->ns * nbands[s] * c->MT);
        max_rows = std::max(max_rows, (c->spin == DFTU_NONCOLLINEAR ? c->nk : c->nk * c->ns) * nbands[s] * c->nspecies);
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    free_tables(b);
    cudaError_t e = cudaMalloc(&b->d_args, n * sizeof(ProjArgs));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_args, args.data(), n * sizeof(ProjArgs), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_f, n * sizeof(double*));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_f, f, n * sizeof(double*), cudaMemcpyHostToDevice);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return bfail(b, DFTU_ERR_CUDA, std::string("batch_bind: ") + cudaGetErrorString(e));
    b->L.args = b->d_args;
    b->L.f = b->d_f;
    b->L.max_reduce = max_reduce;
    b->L.max_rows_nbar = max_rows;
    b->prec = prec;
    b->nbands.assign(nbands, nbands + n);
    b->bound = true;
    return DFTU_OK;
}

// The batched kernels run one arithmetic for all members and no gauge phases: members must agree.
static dftu_status members_uniform(dftu_batch b, const char* what) {
    const Ctx* c0 = b->members[0];
    for (size_t s = 0; s < b->members.size(); ++s) {
        const Ctx* c = b->members[s];
        if (c->gauge_on)
            return bfail(b, DFTU_ERR_INVALID_ARG, std::string(what) + ": member " + std::to_string(s) +
                                                      " has a vector potential set; batches run the plain operator");
        if (c->f64_mode != c0->f64_mode)
            return bfail(b, DFTU_ERR_INVALID_ARG, std::string(what) + ": member " + std::to_string(s) +
                                                      " uses another FP64 mode than member 0");
    }
    return DFTU_OK;
}

dftu_status dftu_batch_project(dftu_batch b, dftu_stream stream) {
    dftu::NvtxRange nvtx_range("dftu_batch_project");
    if (!b) return DFTU_ERR_INVALID_ARG;
    if (!b->bound) return bfail(b, DFTU_ERR_NOT_READY, "batch_project: call dftu_batch_bind first");
    if (dftu_status u = members_uniform(b, "batch_project")) return u;
    Ctx* c0 = b->members[0];
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_project_batch(b->L, b->prec, c0->f64_mode, c0->variant[b->prec == DFTU_C64 ? 1 : 0], st);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return bfail(b, DFTU_ERR_CUDA, std::string("batch_project: ") + cudaGetErrorString(e));
    for (size_t s = 0; s < b->members.size(); ++s) {
        Ctx* c = b->members[s];
        c->proj_ready = true;
        c->proj_nbands = b->nbands[s];
        c->last_stream = st;
    }
    return DFTU_OK;
}

dftu_status dftu_batch_occupations(dftu_batch b, dftu_stream stream) {
    dftu::NvtxRange nvtx_range("dftu_batch_occupations");
    if (!b) return DFTU_ERR_INVALID_ARG;
    for (auto* c : b->members)
        if (!c->proj_ready) return bfail(b, DFTU_ERR_NOT_READY, "batch_occupations: call dftu_batch_project first");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaError_t e = launch_occupations_batch(b->L, reinterpret_cast<cudaStream_t>(stream));
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return bfail(b, DFTU_ERR_CUDA, std::string("batch_occupations: ") + cudaGetErrorString(e));
    for (auto* c : b->members) c->occ_ready = true;
    return DFTU_OK;
}

dftu_status dftu_batch_acbn0_uj(dftu_batch b, dftu_stream stream) {
    dftu::NvtxRange nvtx_range("dftu_batch_acbn0_uj");
    if (!b) return DFTU_ERR_INVALID_ARG;
    for (auto* c : b->members) {
        if (!c->occ_ready) return bfail(b, DFTU_ERR_NOT_READY, "batch_acbn0_uj: call dftu_batch_occupations first");
        for (size_t a = 0; a < c->atoms.size(); ++a)
            if (std::isnan(c->h_fixU[a]) && !c->h_coul_set[c->atoms[a].species])
                return bfail(b, DFTU_ERR_NOT_READY, "batch_acbn0_uj: a member lacks Coulomb integrals for an ACBN0 atom");
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaError_t e = launch_acbn0_batch(b->L, reinterpret_cast<cudaStream_t>(stream));
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return bfail(b, DFTU_ERR_CUDA, std::string("batch_acbn0_uj: ") + cudaGetErrorString(e));
    for (auto* c : b->members) c->pot_ready = true;
    return DFTU_OK;
}

dftu_status dftu_batch_apply(dftu_batch b, const double* coef, int accumulate, dftu_stream stream) {
    dftu::NvtxRange nvtx_range("dftu_batch_apply");
    if (!b) return DFTU_ERR_INVALID_ARG;
    if (!b->bound) return bfail(b, DFTU_ERR_NOT_READY, "batch_apply: call dftu_batch_bind first");
    if (dftu_status u = members_uniform(b, "batch_apply")) return u;
    for (auto* c : b->members)
        if (!c->pot_ready) return bfail(b, DFTU_ERR_NOT_READY, "batch_apply: call dftu_batch_acbn0_uj first");
    Ctx* c0 = b->members[0];
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaError_t e = launch_coefvec_batch(b->L, reinterpret_cast<cudaStream_t>(stream));
    if (e == cudaSuccess)
        e = launch_apply_batch(b->L, b->prec, c0->f64_mode, c0->variant[b->prec == DFTU_C64 ? 3 : 2], coef ? coef : c0->d_coef_one,
                               accumulate ? 1 : 0, reinterpret_cast<cudaStream_t>(stream));
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return bfail(b, DFTU_ERR_CUDA, std::string("batch_apply: ") + cudaGetErrorString(e));
    return DFTU_OK;
}

const char* dftu_batch_last_error(dftu_batch b) { return b ? b->err.c_str() : "null batch"; }

void dftu_batch_destroy(dftu_batch b) {
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    free_tables(b);
    cudaFree(b->d_views);
    cudaFree(b->d_items);
    cudaFree(b->d_color_items);
    cudaFree(b->d_counter);
    if (prev >= 0) cudaSetDevice(prev);
    delete b;
}

}  // extern "C"
