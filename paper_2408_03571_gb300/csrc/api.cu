// C ABI (include/hzs.h): handles, validation, set-up and the GMRES driver.
//
// The driver is host-issued: each Arnoldi step enqueues the preconditioner,
// the matrix-vector product and the CGS2 / Givens kernels on the handle's
// stream.  The host keeps one step in flight ahead of the convergence flag it
// reads back (pinned memory, one event per step), and every kernel of a step
// that is enqueued after convergence returns immediately.  With HZS_SOLVE_GRAPH
// the same launches are captured 8 steps at a time into a CUDA graph that is
// replayed on the handle's stream (one chunk in flight ahead of the flag).
// Set-up can time the launch shapes of the subdomain solve and keep the fastest
// (the autotuner below).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <algorithm>
#include <tuple>
#include <vector>

#include "kernels.cuh"

using namespace hzs;

namespace {

thread_local std::string g_global_err;

struct AxisBlock {
    int own_lo, own_hi, ext_lo, ext_hi;
};

}  // namespace

struct hzs_grid {
    hzs_grid_desc desc{};
    cudaStream_t stream = nullptr;
    double* kappa = nullptr;          // owned copy of the field (or null)
    OpDesc op{};
    int num_sms = 0;
    int lo = 0, hi = 0;               // unknown index range per axis
    int nsx = 0, nsy = 0;             // subdomains along x and y
    std::vector<AxisBlock> xblocks, yblocks;
    std::vector<Tile> tiles;          // nsx * nsy, tile = by * nsx + bx
    std::vector<int4> cover_x, cover_y;   // per grid index: (block, offset, block, offset) along x, y
    int max_mx = 0, max_my = 0;
    std::string err;
};

struct hzs_precond {
    hzs_grid* g = nullptr;
    hzs_precond_desc desc{};
    Ctx cx{};
    HostCoarseTab hct;
    int use_coarse = 0;
    int Nc = 0;
    // device coarse tables
    int *c0 = nullptr, *lo = nullptr, *hi = nullptr, *off = nullptr;
    double *w = nullptr, *wt = nullptr;
    float *wf = nullptr, *wtf = nullptr;
    double2* Ainv = nullptr;
    int coarse_block = 0;             // coarse solve by block-tridiagonal LU instead of Ainv
    CoarseBlockLU cblk;
    int coarse_ml = 0;                // coarse solve by SHS2 on G_H (multilevel) instead of Ainv
    CoarseML cml;
    float2* c2f = nullptr;            // complex64 copy of the coarse solution
    int* err = nullptr;               // device error word (HZS_ERR_TIMEOUT from bounded waits)
    int* groups_d = nullptr;          // tiles grouped by shared factor
    int ngroups = 0, group_T = 1;
    int* groups1_d = nullptr;         // one tile per group (kept when group_T == 2, for the autotuner)
    int ngroups1 = 0;
    // launch shape of the subdomain solve: tiles per block, copy-ring depth, threads per
    // block row (0 = chosen per launch); set by the autotuner when asked for
    int tile_T = 1, tile_nst = 0, tile_tpr = 0;
    int autotuned = 0;
    double apply_us_default = 0.0, apply_us_tuned = 0.0;
    double coarse_minpiv = 0.0;
    // local factors
    int nfactors = 0;
    double2* W64 = nullptr;
    float2* W32 = nullptr;
    std::vector<FactorStat> fstats;
    Tile* tiles_d = nullptr;
    int4* cover_d = nullptr;          // per grid index along x (cover_yd: along y), see hzs_grid::cover_x
    int4* cover_yd = nullptr;
    long long ytiles_elems = 0;
    // apply work space
    void* t_buf = nullptr;            // n * nc1 working complex
    double2* c_buf = nullptr;         // Nc
    double2* c2_buf = nullptr;        // Nc
    void* w_buf = nullptr;            // n*n working complex
    void* ytiles = nullptr;           // sum of tile sizes, working complex
    float2* zc64 = nullptr;           // n*n (mixed public apply)
    int wcap = 0;                     // batch capacity of the apply work space above
    // solve work space
    KrylovBufs kb{};
    int kb_maxit = 0;
    int lo_pad = -1;                  // remainder width (kb.lo16) whose padding is zero; -1: none yet
    float2* Z = nullptr;              // nb x maxit x ld (mixed)
    double2* ztmp = nullptr;          // nb x ld (FP64 z / x)
    double2* rtmp = nullptr;          // nb x ld
    double* dres = nullptr;           // nb
    int* h_done = nullptr;            // pinned, 2 slots
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    std::vector<cudaEvent_t> prof_ev;  // 4 per step when phase timing is on
    // HZS_SOLVE_GRAPH: Arnoldi steps captured in chunks on a private stream and replayed
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t gexec_first = nullptr;          // the chunk that starts at step 0
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // later chunks, alternating
};

// The tile groups and launch shape the subdomain solve of this handle uses.
static TileGroups tile_groups(const hzs_precond* p) {
    if (p->tile_T == 1 && p->group_T == 2) return TileGroups{p->groups1_d, p->ngroups1, 1, p->tile_nst, p->tile_tpr};
    return TileGroups{p->groups_d, p->ngroups, p->group_T, p->tile_nst, p->tile_tpr};
}

// ------------------------------------------------------------------ helpers
static hzs_status fail(hzs_grid* g, hzs_status s, const std::string& msg) {
    if (g) g->err = msg; else g_global_err = msg;
    return s;
}

static hzs_status cuda_fail(hzs_grid* g, cudaError_t e, const char* where) {
    return fail(g, e == cudaErrorMemoryAllocation ? HZS_ERR_OOM : HZS_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

#define HZS_CUDA(g, call)                                             \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail((g), e_, #call);      \
    } while (0)

template <typename T>
static cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, count * sizeof(T));
}

static size_t cplx_size(hzs_precision prec) { return prec == HZS_MIXED ? sizeof(float2) : sizeof(double2); }

static hzs_status ensure_work(hzs_precond* p, int nb);

// largest coarse space solved through an explicit inverse when the solver is AUTO
constexpr int kDenseCoarseMax = 4096;
// Smallest tolerance at which the delayed-CGS2 basis keeps bf16 remainders: the
// 32-bit basis lets the true residual drift from the GMRES estimate by a few
// times 1e-10 relative (at most about 1e-9 on the test problems), well below tol.
constexpr double kNarrowBasisTol = 1e-7;

// ------------------------------------------------------------------ grid
extern "C" hzs_status hzs_grid_create(const hzs_grid_desc* d, void* cuda_stream, hzs_grid** out) {
    if (!out) return fail(nullptr, HZS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!d) return fail(nullptr, HZS_ERR_INVALID_ARG, "desc is NULL");
    if (d->n < 5 || d->n % 2 != 1) return fail(nullptr, HZS_ERR_INVALID_ARG, "n must be odd and >= 5");
    if (d->bc != HZS_DIRICHLET && d->bc != HZS_SOMMERFELD) return fail(nullptr, HZS_ERR_INVALID_ARG, "bad bc");
    const int nsx = d->nsub, nsy = d->nsub_y > 0 ? d->nsub_y : d->nsub;
    if (nsx < 1 || (d->n - 1) % nsx != 0) return fail(nullptr, HZS_ERR_INVALID_ARG, "nsub must divide n-1");
    if (d->nsub_y < 0 || (d->n - 1) % nsy != 0) return fail(nullptr, HZS_ERR_INVALID_ARG, "nsub_y must divide n-1");
    const int wx = (d->n - 1) / nsx, wy = (d->n - 1) / nsy;
    if (d->overlap < 0) return fail(nullptr, HZS_ERR_INVALID_ARG, "overlap must be >= 0");
    if (2 * d->overlap > std::min(wx, wy))
        return fail(nullptr, HZS_ERR_INVALID_ARG, "overlap must be at most half the subdomain width");
    if (d->bc == HZS_DIRICHLET && std::min(wx, wy) < 2)
        return fail(nullptr, HZS_ERR_INVALID_ARG, "subdomain width must be >= 2");
    if (!d->kappa_dev && !(d->k > 0.0 && std::isfinite(d->k)))
        return fail(nullptr, HZS_ERR_INVALID_ARG, "k must be positive and finite");

    hzs_grid* g = new hzs_grid();
    g->desc = *d;
    g->stream = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete g;
        return fail(nullptr, HZS_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    const int n = d->n;
    if (d->kappa_dev) {
        e = dalloc(&g->kappa, (size_t)n * n);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->kappa, d->kappa_dev, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice,
                                g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) {
            cudaFree(g->kappa);
            delete g;
            return fail(nullptr, HZS_ERR_CUDA, std::string("kappa copy: ") + cudaGetErrorString(e));
        }
    }
    const double h = 1.0 / (n - 1);
    g->op.n = n;
    g->op.bc = d->bc;
    g->op.inv_h2 = 1.0 / (h * h);
    g->op.inv_h = 1.0 / h;
    g->op.kappa0 = d->kappa_dev ? 0.0 : d->k * d->k;
    g->op.kappa = g->kappa;
    g->lo = d->bc == HZS_DIRICHLET ? 1 : 0;
    g->hi = d->bc == HZS_DIRICHLET ? n - 2 : n - 1;
    g->nsx = nsx;
    g->nsy = nsy;
    // per axis: owned blocks [a w, (a+1) w) (last one closed at n-1) within the unknowns,
    // extended by overlap, and for every grid index the (at most two) blocks containing it
    auto axis = [&](int ns, int w, std::vector<AxisBlock>& blocks, std::vector<int4>& cover) {
        for (int a = 0; a < ns; ++a) {
            AxisBlock b;
            b.own_lo = std::max(a * w, g->lo);
            b.own_hi = std::min(a < ns - 1 ? (a + 1) * w - 1 : n - 1, g->hi);
            b.ext_lo = std::max(b.own_lo - d->overlap, g->lo);
            b.ext_hi = std::min(b.own_hi + d->overlap, g->hi);
            blocks.push_back(b);
        }
        cover.assign(n, make_int4(-1, 0, -1, 0));
        for (int i = 0; i < n; ++i) {
            int cnt = 0;
            int4 c = make_int4(-1, 0, -1, 0);
            for (int a = 0; a < ns; ++a) {
                const AxisBlock& b = blocks[a];
                if (i >= b.ext_lo && i <= b.ext_hi) {
                    if (cnt == 0) { c.x = a; c.y = i - b.ext_lo; }
                    else if (cnt == 1) { c.z = a; c.w = i - b.ext_lo; }
                    ++cnt;
                }
            }
            if (cnt > 2) return false;
            cover[i] = c;
        }
        return true;
    };
    if (!axis(nsx, wx, g->xblocks, g->cover_x) || !axis(nsy, wy, g->yblocks, g->cover_y)) {
        cudaFree(g->kappa);
        delete g;
        return fail(nullptr, HZS_ERR_INVALID_ARG, "a node lies in more than two subdomains per axis");
    }
    long long yoff = 0;
    for (int by = 0; by < nsy; ++by)
        for (int bx = 0; bx < nsx; ++bx) {
            const AxisBlock &X = g->xblocks[bx], &Y = g->yblocks[by];
            Tile t{};
            t.x0 = X.ext_lo; t.y0 = Y.ext_lo;
            t.mx = X.ext_hi - X.ext_lo + 1; t.my = Y.ext_hi - Y.ext_lo + 1;
            t.ox0 = X.own_lo; t.ox1 = X.own_hi; t.oy0 = Y.own_lo; t.oy1 = Y.own_hi;
            t.factor = -1; t.woff = 0; t.yoff = yoff;
            yoff += (long long)t.mx * t.my;
            g->max_mx = std::max(g->max_mx, t.mx);
            g->max_my = std::max(g->max_my, t.my);
            g->tiles.push_back(t);
        }
    *out = g;
    return HZS_OK;
}

extern "C" void hzs_grid_destroy(hzs_grid* g) {
    if (!g) return;
    cudaFree(g->kappa);
    delete g;
}

// ------------------------------------------------------------------ preconditioner
static void free_krylov(hzs_precond* p) {
    KrylovBufs& kb = p->kb;
    cudaFree(kb.V); cudaFree(kb.V32); cudaFree(kb.V32lo); cudaFree(kb.sigma); cudaFree(kb.H); cudaFree(kb.cs); cudaFree(kb.sn); cudaFree(kb.g);
    cudaFree(kb.y); cudaFree(kb.h1); cudaFree(kb.h2); cudaFree(kb.hn); cudaFree(kb.sigt); cudaFree(kb.part); cudaFree(kb.npart); cudaFree(kb.st);
    cudaFree(kb.active);
    if (kb.side) cudaStreamDestroy(kb.side);
    if (kb.ev_c) cudaEventDestroy(kb.ev_c);
    if (kb.ev_g) cudaEventDestroy(kb.ev_g);
    cudaFree(p->Z); cudaFree(p->ztmp); cudaFree(p->rtmp); cudaFree(p->dres);
    kb = KrylovBufs{};
    p->Z = nullptr;
    p->ztmp = p->rtmp = nullptr;
    p->dres = nullptr;
    p->kb_maxit = 0;
}

extern "C" void hzs_precond_destroy(hzs_precond* p) {
    if (!p) return;
    free_krylov(p);
    cudaFree(p->c0); cudaFree(p->lo); cudaFree(p->hi); cudaFree(p->off); cudaFree(p->w); cudaFree(p->wt);
    cudaFree(p->wf); cudaFree(p->wtf); cudaFree(p->c2f); cudaFree(p->err); cudaFree(p->groups_d);
    coarse_block_free(p->cblk);
    coarse_ml_free(p->cml);
    cudaFree(p->Ainv); cudaFree(p->W64); cudaFree(p->W32); cudaFree(p->tiles_d);
    cudaFree(p->cover_d); cudaFree(p->cover_yd);
    cudaFree(p->t_buf); cudaFree(p->c_buf); cudaFree(p->c2_buf); cudaFree(p->w_buf); cudaFree(p->ytiles);
    cudaFree(p->zc64);
    if (p->h_done) cudaFreeHost(p->h_done);
    for (auto& e : p->ev) if (e) cudaEventDestroy(e);
    if (p->t0) cudaEventDestroy(p->t0);
    if (p->t1) cudaEventDestroy(p->t1);
    for (auto e : p->prof_ev) cudaEventDestroy(e);
    cudaFree(p->groups1_d);
    if (p->gexec_first) cudaGraphExecDestroy(p->gexec_first);
    for (auto& x : p->gexec) if (x) cudaGraphExecDestroy(x);
    if (p->gstream) cudaStreamDestroy(p->gstream);
    delete p;
}

template <typename T>
static cudaError_t upload(T** dst, const std::vector<T>& src, cudaStream_t s) {
    cudaError_t e = dalloc(dst, src.size());
    if (e != cudaSuccess || src.empty()) return e;
    return cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

static hzs_status setup_impl(hzs_grid* g, const hzs_precond_desc* d, hzs_precond* p) {
    if (d->scaling_mode != HZS_SCALING_OWNER && d->scaling_mode != HZS_SCALING_MULTIPLICITY)
        return fail(g, HZS_ERR_INVALID_ARG, "scaling_mode must be HZS_SCALING_OWNER or HZS_SCALING_MULTIPLICITY");
    const int n = g->desc.n;
    cudaStream_t s = g->stream;
    p->cx.op = g->op;
    p->cx.stream = s;
    p->cx.num_sms = g->num_sms;
    p->use_coarse = d->kind != HZS_AS1;
    // ---- coarse level
    if (p->use_coarse) {
        if (d->coarse != HZS_COARSE_P1 && d->coarse != HZS_COARSE_B2)
            return fail(g, HZS_ERR_INVALID_ARG, "two-level preconditioners need coarse = P1 or B2");
        const int pr = d->coarse_ratio;
        if (pr < 2 || (n - 1) % pr != 0) return fail(g, HZS_ERR_INVALID_ARG, "coarse_ratio must be >= 2 and divide n-1");
        build_coarse_tables(n, g->desc.bc, d->coarse, pr, p->hct);
        if (p->hct.nc1 < 1) return fail(g, HZS_ERR_INVALID_ARG, "coarse mesh has no interior nodes");
        if (p->hct.bad) return fail(g, HZS_ERR_INVALID_ARG, "coarse basis wider than three coarse cells");
        p->Nc = p->hct.nc1 * p->hct.nc1;
        if (d->coarse_solver < HZS_COARSE_SOLVER_AUTO || d->coarse_solver > HZS_COARSE_SOLVER_MULTILEVEL)
            return fail(g, HZS_ERR_INVALID_ARG, "coarse_solver must be AUTO, DENSE, BLOCK or MULTILEVEL");
        p->coarse_ml = d->coarse_solver == HZS_COARSE_SOLVER_MULTILEVEL;
        p->coarse_block = !p->coarse_ml && (d->coarse_solver == HZS_COARSE_SOLVER_BLOCK ||
                                            (d->coarse_solver == HZS_COARSE_SOLVER_AUTO && p->Nc > kDenseCoarseMax));
        if (!p->coarse_block && !p->coarse_ml && p->Nc > 8192)
            return fail(g, HZS_ERR_INVALID_ARG, "coarse space larger than 8192 for the dense coarse inverse");
        if ((p->coarse_block || p->coarse_ml) && p->hct.nc1 > 512)
            return fail(g, HZS_ERR_INVALID_ARG, "more than 512 coarse nodes per axis for the block coarse solve");
        HZS_CUDA(g, upload(&p->c0, p->hct.c0, s));
        HZS_CUDA(g, upload(&p->w, p->hct.w, s));
        HZS_CUDA(g, upload(&p->lo, p->hct.lo, s));
        HZS_CUDA(g, upload(&p->hi, p->hct.hi, s));
        HZS_CUDA(g, upload(&p->off, p->hct.off, s));
        HZS_CUDA(g, upload(&p->wt, p->hct.wt, s));
        const std::vector<float> wf(p->hct.w.begin(), p->hct.w.end());
        const std::vector<float> wtf(p->hct.wt.begin(), p->hct.wt.end());
        HZS_CUDA(g, upload(&p->wf, wf, s));
        HZS_CUDA(g, upload(&p->wtf, wtf, s));
        HZS_CUDA(g, cudaStreamSynchronize(s));   // the host vectors above go out of scope
        p->cx.ct.nc1 = p->hct.nc1;
        p->cx.ct.max_sup = 1;
        for (int I = 0; I < p->hct.nc1; ++I) p->cx.ct.max_sup = std::max(p->cx.ct.max_sup, p->hct.hi[I] - p->hct.lo[I] + 1);
        p->cx.ct.c0 = p->c0; p->cx.ct.w = p->w; p->cx.ct.lo = p->lo; p->cx.ct.hi = p->hi;
        p->cx.ct.off = p->off; p->cx.ct.wt = p->wt;
        p->cx.ct.wf = p->wf; p->cx.ct.wtf = p->wtf;
        if (p->coarse_ml) {
            double2* A0b = nullptr;
            HZS_CUDA(g, dalloc(&A0b, (size_t)p->Nc * 25));
            launch_galerkin_banded(p->cx, A0b);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) { cudaFree(A0b); return cuda_fail(g, e, "coarse assembly"); }
            double minpiv = 0.0;
            std::string why;
            // the multilevel solver keeps A0b (its level-2 residual and local blocks) and frees it
            const int rc = coarse_ml_setup(p->cx, p->hct.nc1, g->desc.bc, A0b, d->ml_nsub, d->ml_overlap,
                                           d->ml_ratio, p->cml, &minpiv, &why);
            if (rc == -2) return fail(g, HZS_ERR_INVALID_ARG, why);
            if (rc < 0) return fail(g, HZS_ERR_CUDA, "multilevel coarse set-up failed");
            p->coarse_minpiv = minpiv;
            if (rc > 0) return fail(g, HZS_ERR_SINGULAR_COARSE, "a block of the coarse matrix A_0 has a zero pivot");
        } else if (p->coarse_block) {
            double2* A0b = nullptr;
            HZS_CUDA(g, dalloc(&A0b, (size_t)p->Nc * 25));
            launch_galerkin_banded(p->cx, A0b);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) { cudaFree(A0b); return cuda_fail(g, e, "coarse assembly"); }
            double minpiv = 0.0;
            // the factorisation keeps A0b (the couplings of its solve) and frees it
            const int rc = coarse_block_setup(p->cx, p->hct.nc1, d->coarse == HZS_COARSE_B2 ? 2 : 1, 2, A0b,
                                              p->cblk, &minpiv);
            if (rc < 0) return fail(g, HZS_ERR_CUDA, "coarse block factorisation failed");
            p->coarse_minpiv = minpiv;
            if (rc > 0) return fail(g, HZS_ERR_SINGULAR_COARSE, "coarse matrix A_0 has a zero pivot");
            // the dense products of the sweeps with more than two right-hand sides on the
            // tensor cores (digit slices of the W_i); HZS_COARSE_TC=0 keeps them on the FP64 pipe
            const char* tc = std::getenv("HZS_COARSE_TC");
            if (!(tc && std::atoi(tc) == 0) && coarse_oz_setup(p->cx, p->cblk) < 0)
                return fail(g, HZS_ERR_CUDA, "tensor-core form of the coarse block solve failed");
        } else {
        HZS_CUDA(g, dalloc(&p->Ainv, (size_t)p->Nc * p->Nc));
        launch_galerkin(p->cx, p->Ainv);
        HZS_CUDA(g, cudaGetLastError());
        double minpiv = 0.0;
        const int rc = gj_invert(p->cx, p->Ainv, p->Nc, &minpiv);
        if (rc < 0) return fail(g, HZS_ERR_CUDA, "coarse factorisation failed");
        p->coarse_minpiv = minpiv;
        if (rc > 0) return fail(g, HZS_ERR_SINGULAR_COARSE, "coarse matrix A_0 has a zero pivot");
        }
    }
    HZS_CUDA(g, dalloc(&p->err, 1));
    HZS_CUDA(g, cudaMemsetAsync(p->err, 0, sizeof(int), s));
    p->cx.err = p->err;
    // diagnostic knob: HZS_STAGE_WAIT_POLLS bounds the polls of the subdomain solve's factor-copy
    // waits (default 2^24); a block whose wait runs out records HZS_ERR_TIMEOUT, waits (with the
    // full bound) for its copies still in flight and returns
    if (const char* ev = std::getenv("HZS_STAGE_WAIT_POLLS")) {
        char* end = nullptr;
        const long long v = std::strtoll(ev, &end, 10);
        if (end != ev && v >= 0) p->cx.spin_limit = v;
    }
    if (g->max_mx > max_tile_extent() || g->max_my > max_tile_extent())
        return fail(g, HZS_ERR_INVALID_ARG,
                    "subdomain tile larger than " + std::to_string(max_tile_extent()) + " nodes per axis");
    p->group_T = tile_group_width(g->max_mx, g->max_my, (int)cplx_size(d->precision));
    if (p->group_T == 0)
        return fail(g, HZS_ERR_INVALID_ARG, "subdomain tiles too large for the shared-memory solver");
    // ---- local factors (dedup identical tiles when kappa is constant)
    std::vector<Tile> tiles = g->tiles;
    std::vector<FactorDesc> fds;
    std::map<std::tuple<int, int, int, int, int, int>, int> keys;
    long long woff = 0;
    const bool dedup = d->dedup_tiles && g->kappa == nullptr;
    for (size_t t = 0; t < tiles.size(); ++t) {
        Tile& T = tiles[t];
        const bool sf = g->desc.bc == HZS_SOMMERFELD;
        auto key = std::make_tuple(T.mx, T.my, sf && T.x0 == 0, sf && T.x0 + T.mx - 1 == n - 1, sf && T.y0 == 0,
                                   sf && T.y0 + T.my - 1 == n - 1);
        auto it = dedup ? keys.find(key) : keys.end();
        if (it != keys.end()) {
            T.factor = it->second;
            T.woff = fds[it->second].woff;
            continue;
        }
        FactorDesc fd{T.x0, T.y0, T.mx, T.my, woff};
        T.factor = (int)fds.size();
        T.woff = woff;
        if (dedup) keys[key] = T.factor;
        fds.push_back(fd);
        woff += (long long)T.my * block_stride(T.mx);
    }
    // group tiles that share a factor, group_T at a time
    {
        std::vector<std::vector<int>> by_factor(fds.size());
        for (size_t t = 0; t < tiles.size(); ++t) by_factor[tiles[t].factor].push_back((int)t);
        size_t share = 0;
        for (auto& lst : by_factor) share = std::max(share, lst.size());
        if (share < 2) p->group_T = 1;    // no factor is shared: one tile per block
        std::vector<int> groups;
        for (auto& lst : by_factor)
            for (size_t k = 0; k < lst.size(); k += p->group_T)
                for (int u = 0; u < p->group_T; ++u)
                    groups.push_back(k + u < lst.size() ? lst[k + u] : -1);
        p->ngroups = (int)(groups.size() / p->group_T);
        HZS_CUDA(g, upload(&p->groups_d, groups, s));
        if (p->group_T == 2) {
            std::vector<int> g1;
            for (auto& lst : by_factor) g1.insert(g1.end(), lst.begin(), lst.end());
            p->ngroups1 = (int)g1.size();
            HZS_CUDA(g, upload(&p->groups1_d, g1, s));
        }
        HZS_CUDA(g, cudaStreamSynchronize(s));
        p->tile_T = p->group_T;
    }
    p->nfactors = (int)fds.size();
    HZS_CUDA(g, dalloc(&p->W64, (size_t)woff));
    if (d->precision == HZS_MIXED) HZS_CUDA(g, dalloc(&p->W32, (size_t)woff));
    FactorDesc* fds_d = nullptr;
    FactorStat* st_d = nullptr;
    HZS_CUDA(g, upload(&fds_d, fds, s));
    HZS_CUDA(g, dalloc(&st_d, fds.size()));
    int max_m = 0;
    for (auto& f : fds) max_m = std::max(max_m, f.mx);
    if (launch_tile_factor(p->cx, fds_d, p->nfactors, max_m, p->W64, p->W32, st_d) != 0) {
        cudaFree(fds_d); cudaFree(st_d);
        return fail(g, HZS_ERR_CUDA, "subdomain factorisation launch failed");
    }
    p->fstats.resize(fds.size());
    cudaError_t e = cudaMemcpyAsync(p->fstats.data(), st_d, fds.size() * sizeof(FactorStat), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(fds_d); cudaFree(st_d);
    if (e != cudaSuccess) return cuda_fail(g, e, "subdomain factorisation");
    for (auto& fs : p->fstats)
        if (fs.singular) return fail(g, HZS_ERR_SINGULAR_LOCAL, "a subdomain matrix has a zero pivot");
    HZS_CUDA(g, upload(&p->tiles_d, tiles, s));
    HZS_CUDA(g, upload(&p->cover_d, g->cover_x, s));
    HZS_CUDA(g, upload(&p->cover_yd, g->cover_y, s));
    // ---- apply work space (one right-hand side; batched calls grow it)
    for (auto& T : tiles) p->ytiles_elems += (long long)T.mx * T.my;
    {
        hzs_status st = ensure_work(p, 1);
        if (st != HZS_OK) return st;
    }
    HZS_CUDA(g, cudaHostAlloc((void**)&p->h_done, 2 * sizeof(int), cudaHostAllocDefault));
    for (auto& ev : p->ev) HZS_CUDA(g, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    HZS_CUDA(g, cudaEventCreate(&p->t0));
    HZS_CUDA(g, cudaEventCreate(&p->t1));
    HZS_CUDA(g, cudaStreamSynchronize(s));
    return HZS_OK;
}

static hzs_status autotune_tile_shape(hzs_precond* p);

extern "C" hzs_status hzs_precond_setup(hzs_grid* g, const hzs_precond_desc* d, hzs_precond** out) {
    if (!out) return fail(g, HZS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!g || !d) return fail(g, HZS_ERR_INVALID_ARG, "grid or desc is NULL");
    if (d->kind < HZS_AS1 || d->kind > HZS_SHS2) return fail(g, HZS_ERR_INVALID_ARG, "bad preconditioner kind");
    if (d->precision != HZS_FP64 && d->precision != HZS_MIXED) return fail(g, HZS_ERR_INVALID_ARG, "bad precision");
    if (d->coarse_solver < HZS_COARSE_SOLVER_AUTO || d->coarse_solver > HZS_COARSE_SOLVER_MULTILEVEL)
        return fail(g, HZS_ERR_INVALID_ARG, "bad coarse_solver");
    if (d->autotune < 0 || d->autotune > 2) return fail(g, HZS_ERR_INVALID_ARG, "bad autotune");
    hzs_precond* p = new hzs_precond();
    p->g = g;
    p->desc = *d;
    hzs_status st = setup_impl(g, d, p);
    if (st == HZS_OK && d->autotune) st = autotune_tile_shape(p);
    if (st != HZS_OK) {
        hzs_precond_destroy(p);
        return st;
    }
    *out = p;
    return HZS_OK;
}

// ------------------------------------------------------------------ preconditioner apply
// Per-call work buffers of the preconditioner, for batches of up to nb right-hand sides.
static hzs_status ensure_work(hzs_precond* p, int nb) {
    if (p->wcap >= nb) return HZS_OK;
    hzs_grid* g = p->g;
    cudaFree(p->t_buf); cudaFree(p->c_buf); cudaFree(p->c2_buf); cudaFree(p->c2f);
    cudaFree(p->w_buf); cudaFree(p->ytiles); cudaFree(p->zc64);
    p->t_buf = p->w_buf = p->ytiles = nullptr;
    p->c_buf = p->c2_buf = nullptr;
    p->c2f = p->zc64 = nullptr;
    p->wcap = 0;
    const size_t n = g->desc.n, cs = cplx_size(p->desc.precision);
    if (p->use_coarse) {
        HZS_CUDA(g, cudaMalloc(&p->t_buf, n * p->hct.nc1 * cs * nb));
        HZS_CUDA(g, dalloc(&p->c_buf, (size_t)p->Nc * nb));
        HZS_CUDA(g, dalloc(&p->c2_buf, (size_t)p->Nc * nb));
        HZS_CUDA(g, dalloc(&p->c2f, (size_t)p->Nc * nb));
        if (p->coarse_ml && coarse_ml_reserve(p->cml, nb) != 0)
            return fail(g, HZS_ERR_CUDA, "multilevel coarse work space");
        if (p->coarse_block && nb > 2 && coarse_oz_reserve(p->cblk, nb) != 0)
            return fail(g, HZS_ERR_CUDA, "coarse block work space");
    }
    HZS_CUDA(g, cudaMalloc(&p->w_buf, n * n * cs * nb));
    if (p->desc.kind == HZS_AS1 || p->desc.kind == HZS_AS2 || p->desc.scaling_mode == HZS_SCALING_MULTIPLICITY)
        HZS_CUDA(g, cudaMalloc(&p->ytiles, (size_t)p->ytiles_elems * cs * nb));
    if (p->desc.precision == HZS_MIXED) HZS_CUDA(g, dalloc(&p->zc64, n * n * nb));
    p->wcap = nb;
    return HZS_OK;
}

// z_r = M^{-1} (s_r v_r) for nb batch entries (v_r = v + r vs, s_r = vscale[r vss] or 1,
// z_r = z + r zs).  R: arithmetic of the stencil, transfers and subdomain solves;
// the coarse solve is FP64 either way.  Needs ensure_work(p, nb).
template <typename R, typename Cv>
static hzs_status precond_apply(hzs_precond* p, int nb, const Cv* v, long long vs, const double* vscale,
                                long long vss, cplx_t<R>* z, long long zs, BatchSkip sk) {
    using C = cplx_t<R>;
    constexpr bool f32 = sizeof(R) == sizeof(float);
    const Ctx& cx = p->cx;
    hzs_grid* g = p->g;
    const long long nn = (long long)g->desc.n * g->desc.n;
    const long long Nc = p->Nc;
    const C* W = nullptr;
    const C* cc = nullptr;            // coarse solution in the kernels' precision
    if constexpr (f32) { W = p->W32; cc = p->c2f; } else { W = p->W64; cc = p->c2_buf; }
    const TileGroups grp = tile_groups(p);
    const int kind = p->desc.kind;
    if (p->use_coarse) {
        launch_restrict<Cv, R>(cx, nb, v, vs, vscale, vss, (C*)p->t_buf, p->c_buf, sk);
        if (p->coarse_ml)
            launch_coarse_ml_solve(cx, nb, p->cml, p->c_buf, p->c2_buf, f32 ? p->c2f : nullptr, sk);
        else if (p->coarse_block)
            launch_coarse_block_solve(cx, nb, p->cblk, p->c_buf, p->c2_buf, f32 ? p->c2f : nullptr, sk);
        else
            launch_coarse_matvec(cx, nb, p->Ainv, p->Nc, p->c_buf, p->c2_buf, f32 ? p->c2f : nullptr, sk);
    }
    int rc = 0;
    if (p->desc.scaling_mode == HZS_SCALING_MULTIPLICITY && (kind == HZS_SHS2 || kind == HZS_SAS2)) {
        // D_i = 1/multiplicity: every tile's solution is kept and the combination weights each
        // node's contributions by the number of subdomains that contain it
        const C* src = nullptr;
        if (kind == HZS_SHS2) {
            launch_deflate<Cv, C, R>(cx, nb, cc, Nc, v, vs, vscale, vss, (C*)p->w_buf, nn, sk);
            src = (const C*)p->w_buf;
            rc = launch_tile_solve<C, C, R>(cx, nb, p->tiles_d, grp, g->max_mx, g->max_my, W, src, nn, nullptr, 0, 1,
                                            cc, Nc, 0, (C*)nullptr, 0, (C*)p->ytiles, p->ytiles_elems, sk);
        } else {
            rc = launch_tile_solve<Cv, C, R>(cx, nb, p->tiles_d, grp, g->max_mx, g->max_my, W, v, vs, vscale, vss, 1,
                                             cc, Nc, 0, (C*)nullptr, 0, (C*)p->ytiles, p->ytiles_elems, sk);
        }
        launch_combine_additive<C, C, R>(cx, nb, cc, Nc, p->use_coarse, p->cover_d, p->cover_yd, p->tiles_d, g->nsx,
                                         (const C*)p->ytiles, p->ytiles_elems, z, zs, sk, 1);
    } else if (kind == HZS_SHS2) {
        launch_deflate<Cv, C, R>(cx, nb, cc, Nc, v, vs, vscale, vss, (C*)p->w_buf, nn, sk);
        rc = launch_tile_solve<C, C, R>(cx, nb, p->tiles_d, grp, g->max_mx, g->max_my, W, (const C*)p->w_buf, nn,
                                        nullptr, 0, 0, cc, Nc, 1, z, zs, nullptr, 0, sk);
    } else if (kind == HZS_SAS2) {
        rc = launch_tile_solve<Cv, C, R>(cx, nb, p->tiles_d, grp, g->max_mx, g->max_my, W, v, vs, vscale, vss, 0, cc,
                                         Nc, 1, z, zs, nullptr, 0, sk);
    } else {
        rc = launch_tile_solve<Cv, C, R>(cx, nb, p->tiles_d, grp, g->max_mx, g->max_my, W, v, vs, vscale, vss, 1, cc,
                                         Nc, 0, (C*)nullptr, 0, (C*)p->ytiles, p->ytiles_elems, sk);
        launch_combine_additive<C, C, R>(cx, nb, cc, Nc, p->use_coarse, p->cover_d, p->cover_yd, p->tiles_d, g->nsx,
                                         (const C*)p->ytiles, p->ytiles_elems, z, zs, sk, 0);
    }
    if (rc != 0) return fail(g, HZS_ERR_CUDA, "subdomain solve launch failed");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(g, e, "preconditioner launch");
    return HZS_OK;
}

static const BatchSkip kNoSkip{nullptr, 0};
constexpr int kApplyChunk = 16;       // right-hand sides per batched preconditioner apply

extern "C" hzs_status hzs_apply_operator(hzs_precond* p, const void* x_dev, void* y_dev, int nrhs) {
    if (!p) return fail(nullptr, HZS_ERR_INVALID_ARG, "precond is NULL");
    if (!x_dev || !y_dev || nrhs < 0) return fail(p->g, HZS_ERR_INVALID_ARG, "bad buffers or nrhs");
    if (nrhs == 0) return HZS_OK;
    const long long nn = (long long)p->g->desc.n * p->g->desc.n;
    launch_apply_A<double2, double2, double>(p->cx, nrhs, (const double2*)x_dev, nn, (double2*)y_dev, nn, nullptr, 0,
                                             kNoSkip);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(p->g, e, "apply_operator");
    return HZS_OK;
}

__global__ void k_c64_to_c128(long long N, const float2* __restrict__ a, double2* __restrict__ b) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x)
        b[e] = to_d(a[e]);
}

extern "C" hzs_status hzs_apply_precond(hzs_precond* p, const void* v_dev, void* z_dev, int nrhs) {
    if (!p) return fail(nullptr, HZS_ERR_INVALID_ARG, "precond is NULL");
    if (!v_dev || !z_dev || nrhs < 0) return fail(p->g, HZS_ERR_INVALID_ARG, "bad buffers or nrhs");
    const long long nn = (long long)p->g->desc.n * p->g->desc.n;
    for (int r0 = 0; r0 < nrhs; r0 += kApplyChunk) {
        const int nb = std::min(kApplyChunk, nrhs - r0);
        hzs_status st = ensure_work(p, nb);
        if (st != HZS_OK) return st;
        const double2* v = (const double2*)v_dev + r0 * nn;
        double2* z = (double2*)z_dev + r0 * nn;
        if (p->desc.precision == HZS_MIXED) {
            st = precond_apply<float, double2>(p, nb, v, nn, nullptr, 0, p->zc64, nn, kNoSkip);
            if (st == HZS_OK)
                k_c64_to_c128<<<4 * p->cx.num_sms, 256, 0, p->cx.stream>>>(nn * nb, p->zc64, z);
        } else {
            st = precond_apply<double, double2>(p, nb, v, nn, nullptr, 0, z, nn, kNoSkip);
        }
        if (st != HZS_OK) return st;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(p->g, e, "apply_precond");
    return HZS_OK;
}

// ------------------------------------------------------------------ subdomain-solve autotuner
// Picks the launch shape of the subdomain solve - tiles per block (pairs that share a
// factor, or single tiles), depth of the factor-block copy ring, threads per block row -
// by timing whole preconditioner applies of this handle (one right-hand side, CUDA
// events on its stream).  Every shape computes the same tile solves; only the order of
// the partial sums of a block row changes with the threads per row.  A shape replaces
// the default only when it is more than 2 % faster.  Choices are kept per process for
// problems of the same size and decomposition (autotune = 1); autotune = 2 re-times.
namespace {
struct TileChoice {
    int T, nst, tpr;
    double us_default, us_best;
};
std::mutex g_tune_mu;
std::map<std::string, TileChoice> g_tune_cache;
constexpr int kTuneReps = 10;
}  // namespace

static hzs_status autotune_tile_shape(hzs_precond* p) {
    hzs_grid* g = p->g;
    const hzs_grid_desc& gd = g->desc;
    const hzs_precond_desc& d = p->desc;
    const cudaStream_t s = p->cx.stream;
    int dev = 0;
    HZS_CUDA(g, cudaGetDevice(&dev));
    char kb[256];
    snprintf(kb, sizeof kb, "%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d", dev, gd.n, (int)gd.bc, g->nsx, g->nsy,
             gd.overlap, (int)d.kind, (int)d.coarse, d.coarse_ratio, (int)d.precision, p->coarse_block, p->nfactors,
             p->group_T, g->max_mx, g->max_my, d.scaling_mode);
    const std::string key(kb);
    if (d.autotune == 1) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            p->tile_T = it->second.T; p->tile_nst = it->second.nst; p->tile_tpr = it->second.tpr;
            p->apply_us_default = it->second.us_default; p->apply_us_tuned = it->second.us_best;
            p->autotuned = 1;
            return HZS_OK;
        }
    }
    const int eb = (int)cplx_size(d.precision);
    struct Cand { int T, nst, tpr; };
    std::vector<Cand> cands;
    // the shape the launch picks by itself, first
    int dT = 0, dN = 0, dP = 0;
    if (!tile_shape_resolve(TileGroups{nullptr, 0, p->group_T, 0, 0}, g->max_mx, g->max_my, eb, &dT, &dN, &dP))
        return fail(g, HZS_ERR_INVALID_ARG, "no launch shape of the subdomain solve fits these tiles");
    cands.push_back({dT, dN, dP});
    const int Ts[2] = {p->group_T, 1};
    for (int ti = 0; ti < (p->group_T == 2 ? 2 : 1); ++ti)
        for (int nst : {4, 2, 1})
            for (int tpr : {8, 4}) {
                int a = 0, b = 0, c = 0;
                if (!tile_shape_resolve(TileGroups{nullptr, 0, Ts[ti], nst, tpr}, g->max_mx, g->max_my, eb, &a, &b, &c))
                    continue;
                // a one-stage ring only where no deeper one fits
                if (nst == 1 && tile_shape_resolve(TileGroups{nullptr, 0, Ts[ti], 2, tpr}, g->max_mx, g->max_my, eb,
                                                   &a, &b, &c))
                    continue;
                if (Ts[ti] == dT && nst == dN && tpr == dP) continue;
                cands.push_back({Ts[ti], nst, tpr});
            }
    const long long nn = (long long)gd.n * gd.n;
    double2* v = nullptr;
    void* z = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        cudaFree(v); cudaFree(z);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = dalloc(&v, (size_t)nn);
    if (e == cudaSuccess) e = cudaMalloc(&z, (size_t)nn * eb);
    if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, (size_t)nn * sizeof(double2), s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(g, e, "autotune set-up"); }
    auto run = [&]() -> bool {
        const hzs_status st =
            d.precision == HZS_MIXED
                ? precond_apply<float, double2>(p, 1, v, nn, nullptr, 0, static_cast<float2*>(z), nn, kNoSkip)
                : precond_apply<double, double2>(p, 1, v, nn, nullptr, 0, static_cast<double2*>(z), nn, kNoSkip);
        return st == HZS_OK;
    };
    double best = 0.0, us_def = 0.0;
    int bi = -1;
    for (size_t i = 0; i < cands.size(); ++i) {
        p->tile_T = cands[i].T; p->tile_nst = cands[i].nst; p->tile_tpr = cands[i].tpr;
        bool ok = run() && run();
        if (ok) e = cudaEventRecord(e0, s);
        for (int r = 0; r < kTuneReps && ok && e == cudaSuccess; ++r) ok = run();
        if (ok && e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { cleanup(); return cuda_fail(g, e, "autotune"); }
        if (!ok) {                 // a shape that cannot launch here is skipped
            cudaGetLastError();
            continue;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double us = 1e3 * ms / kTuneReps;
        if (i == 0) us_def = us;
        if (bi < 0 || us < best) { best = us; bi = (int)i; }
    }
    int kerr = 0;
    e = cudaMemcpyAsync(&kerr, p->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(g, e, "autotune");
    g->err.clear();
    if (kerr != 0) {
        cudaMemsetAsync(p->err, 0, sizeof(int), s);
        return fail(g, HZS_ERR_TIMEOUT, "a subdomain-solve block gave up waiting for its factor copies");
    }
    if (bi < 0 || us_def <= 0.0) return fail(g, HZS_ERR_CUDA, "autotune: the default subdomain-solve shape failed");
    if (best > 0.98 * us_def) { bi = 0; best = us_def; }   // keep the default unless clearly faster
    TileChoice tc{cands[bi].T, cands[bi].nst, cands[bi].tpr, us_def, best};
    p->tile_T = tc.T; p->tile_nst = tc.nst; p->tile_tpr = tc.tpr;
    p->apply_us_default = us_def; p->apply_us_tuned = best;
    p->autotuned = 1;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = tc;
    return HZS_OK;
}

extern "C" hzs_status hzs_precond_get_info(const hzs_precond* p, hzs_precond_info* out) {
    if (!p || !out) return fail(nullptr, HZS_ERR_INVALID_ARG, "precond or out is NULL");
    hzs_precond_info in{};
    in.nfactors = p->nfactors;
    in.coarse_unknowns = p->use_coarse ? p->Nc : 0;
    in.coarse_solver = !p->use_coarse ? 0
                       : p->coarse_ml  ? HZS_COARSE_SOLVER_MULTILEVEL
                       : (p->coarse_block ? HZS_COARSE_SOLVER_BLOCK : HZS_COARSE_SOLVER_DENSE);
    in.coarse_min_pivot = p->coarse_minpiv;
    int T = 0, nst = 0, tpr = 0;
    if (tile_shape_resolve(tile_groups(p), p->g->max_mx, p->g->max_my, (int)cplx_size(p->desc.precision), &T, &nst,
                           &tpr)) {
        in.tile_group = T; in.tile_stages = nst; in.tile_threads_per_row = tpr;
    }
    in.autotuned = p->autotuned;
    in.apply_us_default = p->apply_us_default;
    in.apply_us_tuned = p->apply_us_tuned;
    in.coarse_tensor_cores = p->coarse_block && p->cblk.Aoz ? 1 : 0;
    *out = in;
    return HZS_OK;
}

// ------------------------------------------------------------------ solve
// Device bytes one batch entry of the Krylov work space takes.
static size_t krylov_entry_bytes(const hzs_precond* p, int maxit, long long ld, bool full_v) {
    const bool mixed = p->desc.precision == HZS_MIXED;
    size_t b = (size_t)(full_v ? maxit + 1 : 1) * ld * sizeof(double2);   // V
    if (mixed && !full_v) b += 2 * (size_t)(maxit + 1) * ld * sizeof(float2);   // V32, V32lo
    if (mixed) b += (size_t)maxit * ld * sizeof(float2);                   // Z
    b += 2 * (size_t)ld * sizeof(double2);                                 // ztmp, rtmp
    b += (size_t)(maxit + 1) * maxit * sizeof(double2);                    // H
    return b;
}

// Krylov work space for batches of up to nb right-hand sides with maxit steps.
// full_v: keep the whole complex128 basis (FP64 CGS2, FP64 delayed CGS2); otherwise
// only its slot 0 and the double-float basis V32 + V32lo.
static hzs_status ensure_krylov(hzs_precond* p, int maxit, int nb, bool full_v) {
    hzs_grid* g = p->g;
    if (p->kb.V && p->kb.maxit >= maxit && p->kb.nb >= nb && p->kb.vfull == (full_v ? 1 : 0)) return HZS_OK;
    free_krylov(p);
    const long long N = (long long)g->desc.n * g->desc.n;
    const long long ld = (N + 63) / 64 * 64;
    KrylovBufs& kb = p->kb;
    kb.maxit = maxit;
    kb.nb = nb;
    kb.N = N;
    kb.ld = ld;
    // basis sweeps: 3 blocks of 256 threads per SM (80 registers a thread); the
    // delayed-CGS2 dot pass, 64 registers a thread, runs 4 per SM
    kb.nblk = 3 * g->num_sms;
    kb.nblk_dot = 4 * g->num_sms;
    // tuning knobs of the f53 passes (the defaults in KrylovBufs are the fastest measured at
    // the headline size), read when the work space is made:
    //   HZS_F53_MASK="dot,update"  two 8-bit masks of the vectors (index mod 8) summed with
    //                              FP64 FMAs; the others take the FP32 path
    //   HZS_F53_OCC=2|3            blocks per SM of both passes; HZS_F53_DOT_OCC=2..4 the dot pass
    //   HZS_F53_WS=0|1             dot pass with warp tasks on one path each, or mixed tasks
    //   HZS_F53_GROUP=1|2|4        vectors per FP32 (or mixed) warp task of the dot pass (4:
    //                              specialised warps only)
    //   HZS_F53_RING=0|3|4         stages of the dot pass's copy ring (mixed tasks; 0: none)
    //   HZS_F53_UPD_E=1|2          entries per thread and sweep of the update pass
    //   HZS_F53_G64=4|8            vectors per FP64 task of the dot pass (specialised warps)
    //   HZS_F53_RING64=0|1         FP64 tasks of the dot pass through the copy ring as well
    //   HZS_F53_DOT_WAVES=1|2      dot pass at 2 blocks/SM in one or two waves of blocks
    if (const char* ev = std::getenv("HZS_F53_OCC")) {
        const int v = std::atoi(ev);
        if (v == 2 || v == 3) kb.s53_minb = kb.s53_dot_minb = v;
    }
    if (const char* ev = std::getenv("HZS_F53_DOT_OCC")) {
        const int v = std::atoi(ev);
        if (v >= 2 && v <= 4) kb.s53_dot_minb = v;
    }
    if (const char* ev = std::getenv("HZS_F53_RING")) {
        const int v = std::atoi(ev);
        if (v == 0 || v == 3 || v == 4) kb.s53_ring = v;
    }
    if (const char* ev = std::getenv("HZS_F53_WS")) kb.s53_ws = std::atoi(ev) ? 1 : 0;
    if (const char* ev = std::getenv("HZS_F53_UPD_E")) kb.s53_upd_e = std::atoi(ev) == 2 ? 2 : 1;
    if (const char* ev = std::getenv("HZS_F53_G64")) kb.s53_g64 = std::atoi(ev) == 8 ? 8 : 4;
    if (const char* ev = std::getenv("HZS_F53_RING64")) kb.s53_ring64 = std::atoi(ev) ? 1 : 0;
    if (const char* ev = std::getenv("HZS_F53_DOT_WAVES")) kb.s53_dot_waves = std::atoi(ev) == 1 ? 1 : 2;
    if (const char* ev = std::getenv("HZS_F53_GROUP")) {
        const int v = std::atoi(ev);
        if (v == 1 || v == 2 || v == 4) kb.s53_group = v;
    }
    if (const char* ev = std::getenv("HZS_F53_MASK")) {
        unsigned a = 0, b = 0;
        if (std::sscanf(ev, "%i,%i", (int*)&a, (int*)&b) == 2 && a <= 255u && b <= 255u) {
            kb.dmask_dot = a;
            kb.dmask_upd = b;
        }
    }
    const size_t S = (size_t)(maxit + 1);
    kb.vfull = full_v ? 1 : 0;
    HZS_CUDA(g, dalloc(&kb.V, (size_t)nb * kb.sVd()));
    HZS_CUDA(g, dalloc(&kb.sigma, nb * S));
    HZS_CUDA(g, dalloc(&kb.H, (size_t)nb * kb.sH()));
    HZS_CUDA(g, dalloc(&kb.cs, nb * S));
    HZS_CUDA(g, dalloc(&kb.sn, nb * S));
    HZS_CUDA(g, dalloc(&kb.g, nb * S));
    HZS_CUDA(g, dalloc(&kb.y, nb * S));
    HZS_CUDA(g, dalloc(&kb.h1, nb * S));
    HZS_CUDA(g, dalloc(&kb.h2, nb * S));
    HZS_CUDA(g, dalloc(&kb.hn, (size_t)nb * kb.sN()));
    HZS_CUDA(g, dalloc(&kb.sigt, nb * S));
    HZS_CUDA(g, dalloc(&kb.part, (size_t)nb * kb.sP()));
    HZS_CUDA(g, dalloc(&kb.npart, (size_t)nb * kb.nblk));
    HZS_CUDA(g, dalloc(&kb.st, (size_t)nb));
    HZS_CUDA(g, dalloc(&kb.active, 1));
    // side stream for the Givens rotation of a delayed-CGS2 step (without it, the
    // rotation runs on the solve stream)
    if (cudaStreamCreateWithFlags(&kb.side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&kb.ev_c, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&kb.ev_g, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (kb.side) cudaStreamDestroy(kb.side);
        if (kb.ev_c) cudaEventDestroy(kb.ev_c);
        if (kb.ev_g) cudaEventDestroy(kb.ev_g);
        kb.side = nullptr; kb.ev_c = kb.ev_g = nullptr;
    }
    if (p->desc.precision == HZS_MIXED && !full_v) {
        HZS_CUDA(g, dalloc(&kb.V32, (size_t)nb * kb.sV()));
        float2* lo = nullptr;
        HZS_CUDA(g, dalloc(&lo, (size_t)nb * kb.sV()));
        kb.V32lo = lo;
        kb.lo16 = 0;
        p->lo_pad = -1;
        // the vectorised basis kernels read entries N .. ld-1 of each basis vector
        // (pairs of entries); they must hold zero and nothing else writes them
        // (the remainders' padding depends on their width: see set_basis_width)
        if (ld > N)
            HZS_CUDA(g, cudaMemset2DAsync(kb.V32 + N, ld * sizeof(float2), 0, (ld - N) * sizeof(float2),
                                          (size_t)nb * (maxit + 1), g->stream));
    }
    if (p->desc.precision == HZS_MIXED) HZS_CUDA(g, dalloc(&p->Z, (size_t)nb * maxit * ld));
    HZS_CUDA(g, dalloc(&p->ztmp, (size_t)nb * ld));
    HZS_CUDA(g, dalloc(&p->rtmp, (size_t)nb * ld));
    HZS_CUDA(g, dalloc(&p->dres, (size_t)nb));
    return ensure_work(p, nb);
}

// Selects the remainder width of the double-float basis for a solve and zeroes
// the padding entries N .. ld-1 of every basis slot in that layout (the wide and
// narrow layouts put the padding at different bytes of the buffer).
static hzs_status set_basis_width(hzs_precond* p, int lo16) {
    KrylovBufs& kb = p->kb;
    kb.lo16 = lo16;
    if (p->lo_pad != lo16 && kb.ld > kb.N) {
        const size_t es = lo16 ? sizeof(__nv_bfloat162) : sizeof(float2);
        char* base = static_cast<char*>(kb.V32lo) + kb.N * es;
        HZS_CUDA(p->g, cudaMemset2DAsync(base, kb.ld * es, 0, (kb.ld - kb.N) * es, (size_t)kb.nb * (kb.maxit + 1),
                                         p->cx.stream));
    }
    p->lo_pad = lo16;
    return HZS_OK;
}

// Arnoldi orthogonalisation of a solve (Section 5; the paper fixes no variant):
// FP64 CGS2 on a complex128 basis (four passes per step) for HZS_FP64 or with
// HZS_SOLVE_ORTH_FP64; for HZS_MIXED by default the delayed CGS2 on the complex128
// basis (two passes per step, FP64 reorthogonalisation); with HZS_SOLVE_BASIS_DF the
// delayed CGS2 on the narrower double-float basis.
constexpr int kOrthCGS2 = 0, kOrthS53 = 1, kOrthDF = 2, kOrthD64 = 3;   // values of hzs_solve_info.orth_kind
static int orth_mode(const hzs_precond* p, const hzs_solve_desc* sd) {
    if (p->desc.precision != HZS_MIXED || (sd->flags & HZS_SOLVE_ORTH_FP64)) return kOrthCGS2;
    if (sd->flags & HZS_SOLVE_BASIS_DF) return kOrthDF;
    if (sd->flags & HZS_SOLVE_ORTH_DFMA) return kOrthD64;
    // the f53 update pass keeps 96 bytes of coefficients per basis vector in shared
    // memory; longer runs use the all-FMA variant (32 bytes per vector)
    return s53_update_smem(sd->maxit) + 8192 <= (size_t)227 * 1024 ? kOrthS53 : kOrthD64;
}

// Kernel launches of one preconditioner apply.
static int precond_launches(const hzs_precond* p) {
    int n = p->use_coarse ? 3 : 0;   // restriction (2) + coarse solve
    if (p->desc.kind == HZS_SHS2) n += 2;       // deflated residual + subdomain solves
    else if (p->desc.kind == HZS_SAS2) n += 1;  // subdomain solves
    else n += 2;                                 // subdomain solves + additive combination
    return n;
}

static hzs_status ensure_prof_events(hzs_precond* p, int maxit) {
    const size_t need = (size_t)8 * (maxit + 1);
    while (p->prof_ev.size() < need) {
        cudaEvent_t e;
        HZS_CUDA(p->g, cudaEventCreate(&e));
        p->prof_ev.push_back(e);
    }
    return HZS_OK;
}

// Arnoldi steps per captured graph (HZS_SOLVE_GRAPH)
constexpr int kGraphChunk = 8;

// Launches graph gr on stream s through the executable graph *ex: updated in place when
// its topology matches gr (only kernel arguments and launch sizes differ between chunks),
// else (re-)instantiated.  The caller guarantees that no launch of *ex is still running.
static cudaError_t graph_replay(cudaGraphExec_t* ex, cudaGraph_t gr, cudaStream_t s) {
    if (*ex) {
        cudaGraphExecUpdateResultInfo ri{};
        if (cudaGraphExecUpdate(*ex, gr, &ri) != cudaSuccess) {
            cudaGetLastError();   // a topology mismatch is not an error here: instantiate anew
            cudaGraphExecDestroy(*ex);
            *ex = nullptr;
        }
    }
    cudaError_t e = cudaSuccess;
    if (!*ex) e = cudaGraphInstantiate(ex, gr, 0ULL);
    if (e != cudaSuccess) { *ex = nullptr; return e; }
    return cudaGraphLaunch(*ex, s);
}

// nb right-hand sides in lockstep: A u_r = f_r (conj_io: solve A mu = conj(f), return
// conj(mu)).  f_r = f + r nn, u_r = u + r nn.  Every Arnoldi step advances all entries
// that have not finished; finished entries skip their work.  info gets nb entries.
static hzs_status solve_batch(hzs_precond* p, const hzs_solve_desc* sd, const double2* f, double2* u, int nb,
                              int conj_io, hzs_solve_info* info) {
    hzs_grid* g = p->g;
    const Ctx& cx = p->cx;
    KrylovBufs& kb = p->kb;
    cudaStream_t s = cx.stream;
    const long long nn = (long long)g->desc.n * g->desc.n;
    const long long sV = kb.sV(), sS = kb.sS(), ld = kb.ld;
    const long long sZ = (long long)kb.maxit * ld;
    const bool mixed = p->desc.precision == HZS_MIXED;
    const bool prof = (sd->flags & HZS_SOLVE_PROFILE) != 0;
    const int orth = orth_mode(p, sd);
    // delayed CGS2 on the double-float basis, or on the FP64 basis
    const bool orth32 = orth == kOrthDF;
    const bool d64 = orth == kOrthD64;
    const bool s53 = orth == kOrthS53;
    // bf16 remainders (a basis of about 32 significant bits) for loose tolerances
    const bool lo16 = orth32 && !(sd->flags & HZS_SOLVE_BASIS_WIDE) && sd->tol >= kNarrowBasisTol;
    const BatchSkip sk = kb.skip();
    const int pl = precond_launches(p);
    long long launches = 0;
    const bool graph = (sd->flags & HZS_SOLVE_GRAPH) && !prof;
    if (graph && !p->gstream) HZS_CUDA(g, cudaStreamCreateWithFlags(&p->gstream, cudaStreamNonBlocking));
    if (prof) {
        hzs_status st = ensure_prof_events(p, sd->maxit);
        if (st != HZS_OK) return st;
    }
    if (orth32) {
        hzs_status st = set_basis_width(p, lo16 ? 1 : 0);
        if (st != HZS_OK) return st;
    }
    HZS_CUDA(g, cudaEventRecord(p->t0, s));
    // V_0 = f (masked; it is never rescaled in place), plus its double-float copy for orth32
    launch_mask_copy_c128(cx, nb, f, nn, kb.V, kb.sVd(), conj_io, orth32 ? kb.V32 : nullptr, sV,
                          orth32 ? kb.lo_at(0) : LoDst{nullptr, nullptr});
    launch_norm_init(cx, kb, nb, sd->tol);
    launches += 3;
    uint2* Vt = static_cast<uint2*>(kb.V32lo);
    if ((s53 || orth32) && (!kb.V32 || !kb.V32lo))
        return fail(g, HZS_ERR_CUDA, "Krylov work space lacks the head/remainder arrays of this orthogonalisation");
    if ((d64 || orth == kOrthCGS2) && !kb.vfull)
        return fail(g, HZS_ERR_CUDA, "Krylov work space lacks the complex128 basis of this orthogonalisation");
    if (s53) {
        // the f53 copy of V_0, scaled by a power of two to unit size (sigma_0 takes the factor)
        launch_f53_scale0(cx, nb, kb.sigma, kb.sigt, sS, p->dres);
        launch_f53_encode(cx, nb, kb.N, kb.V, kb.sVd(), kb.V32, Vt, sV, p->dres, nullptr);
        launches += 2;
    }
    int steps = 0;
    // enqueues Arnoldi step j of every entry on cx.stream
    auto issue_step = [&](int j) -> hzs_status {
        cudaEvent_t* pe = prof ? &p->prof_ev[(size_t)8 * j] : nullptr;
        if (prof) HZS_CUDA(g, cudaEventRecord(pe[0], cx.stream));
        hzs_status st;
        if (s53) {
            // the complex64 preconditioner reads the heads of u~_j scaled by 1/|u~_j|; A z_j in
            // FP64, stored as f53 in slot j+1
            float2* Zj = p->Z + (size_t)j * ld;
            st = precond_apply<float, float2>(p, nb, kb.V32 + (size_t)j * ld, sV, kb.sigt + j, sS, Zj, sZ, sk);
            if (prof) HZS_CUDA(g, cudaEventRecord(pe[1], cx.stream));
            launch_apply_A_f53(cx, nb, Zj, sZ, kb.V32 + (size_t)(j + 1) * ld, Vt + (size_t)(j + 1) * ld, sV, sk);
        } else if (d64) {
            // the complex64 preconditioner reads u~_j (the once-projected vector of the previous
            // step, see launch_dcgs2_step64) scaled by 1/|u~_j|; A z_j in FP64 into slot j+1
            float2* Zj = p->Z + (size_t)j * ld;
            st = precond_apply<float, double2>(p, nb, kb.V + (size_t)j * ld, sV, kb.sigt + j, sS, Zj, sZ, sk);
            if (prof) HZS_CUDA(g, cudaEventRecord(pe[1], cx.stream));
            launch_apply_A<float2, double2, double>(cx, nb, Zj, sZ, kb.V + (size_t)(j + 1) * ld, sV, nullptr, 0, sk);
        } else if (orth32) {
            // the complex64 preconditioner reads the leading words of u~_j (the once-projected
            // vector of the previous step, see launch_dcgs2_step) scaled by 1/|u~_j|
            float2* Zj = p->Z + (size_t)j * ld;
            st = precond_apply<float, float2>(p, nb, kb.V32 + (size_t)j * ld, sV, kb.sigt + j, sS, Zj, sZ, sk);
            if (prof) HZS_CUDA(g, cudaEventRecord(pe[1], cx.stream));
            // A z_j as a double-float pair (the FP64 copy of the basis is not used on this path)
            if (!launch_apply_A_df(cx, nb, Zj, sZ, kb.V32 + (size_t)(j + 1) * ld, kb.lo_at(j + 1), sV, sk))
                launch_apply_A<float2, double2, double>(cx, nb, Zj, sZ, (double2*)nullptr, 0,
                                                        kb.V32 + (size_t)(j + 1) * ld, sV, sk, kb.lo_at(j + 1));
        } else if (mixed) {
            float2* Zj = p->Z + (size_t)j * ld;
            st = precond_apply<float, double2>(p, nb, kb.V + (size_t)j * ld, sV, kb.sigma + j, sS, Zj, sZ, sk);
            if (prof) HZS_CUDA(g, cudaEventRecord(pe[1], cx.stream));
            launch_apply_A<float2, double2, double>(cx, nb, Zj, sZ, kb.V + (size_t)(j + 1) * ld, sV, nullptr, 0, sk);
        } else {
            st = precond_apply<double, double2>(p, nb, kb.V + (size_t)j * ld, sV, kb.sigma + j, sS, p->ztmp, ld, sk);
            if (prof) HZS_CUDA(g, cudaEventRecord(pe[1], cx.stream));
            launch_apply_A<double2, double2, double>(cx, nb, p->ztmp, ld, kb.V + (size_t)(j + 1) * ld, sV, nullptr, 0,
                                                     sk);
        }
        if (st != HZS_OK) return st;
        if (prof) HZS_CUDA(g, cudaEventRecord(pe[2], cx.stream));
        if (s53) {
            if (!launch_dcgs2_step53(cx, kb, nb, j, 0, prof ? pe + 4 : nullptr))
                return fail(g, HZS_ERR_CUDA, "Arnoldi step on the f53 basis could not be launched");
        } else if (d64) {
            launch_dcgs2_step64(cx, kb, nb, j, 0, prof ? pe + 4 : nullptr);
        } else if (orth32) {
            launch_dcgs2_step(cx, kb, nb, j, 0, prof ? pe + 4 : nullptr);
        } else {
            launch_arnoldi_step(cx, kb, nb, j);
        }
        if (prof) HZS_CUDA(g, cudaEventRecord(pe[3], cx.stream));
        launches += pl + 1 + (orth32 || d64 || s53 ? (j > 0 ? 6 : 5) : 7);
        steps = j + 1;
        // a launch that could not start (e.g. its resources) must not pass silently
        HZS_CUDA(g, cudaGetLastError());
        return HZS_OK;
    };
    if (!graph) {
        for (int j = 0; j < sd->maxit; ++j) {
            const hzs_status st = issue_step(j);
            if (st != HZS_OK) return st;
            // the host runs one step ahead of the count of running entries it reads back
            HZS_CUDA(g, cudaMemcpyAsync(&p->h_done[j & 1], kb.active, sizeof(int), cudaMemcpyDeviceToHost, s));
            HZS_CUDA(g, cudaEventRecord(p->ev[j & 1], s));
            if (j >= 1) {
                HZS_CUDA(g, cudaEventSynchronize(p->ev[(j - 1) & 1]));
                if (p->h_done[(j - 1) & 1] == 0) break;
            }
        }
    } else {
        // chunks of kGraphChunk steps: captured on the private stream (the grid's stream may
        // be the legacy default stream, which cannot be captured), replayed on s
        for (int j0 = 0, c = 0; j0 < sd->maxit; j0 += kGraphChunk, ++c) {
            const int j1 = std::min(sd->maxit, j0 + kGraphChunk);
            cudaGraph_t gr = nullptr;
            p->cx.stream = p->gstream;
            cudaError_t e = cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeRelaxed);
            hzs_status st = HZS_OK;
            if (e == cudaSuccess) {
                for (int j = j0; j < j1 && st == HZS_OK; ++j) st = issue_step(j);
                const cudaError_t e2 = cudaStreamEndCapture(p->gstream, &gr);
                e = e2;
            }
            p->cx.stream = s;
            if (st == HZS_OK && e != cudaSuccess) st = cuda_fail(g, e, "capture of the Arnoldi steps");
            if (st == HZS_OK) {
                e = graph_replay(j0 == 0 ? &p->gexec_first : &p->gexec[c & 1], gr, s);
                if (e != cudaSuccess) st = cuda_fail(g, e, "replay of the Arnoldi steps");
            }
            if (gr) cudaGraphDestroy(gr);
            if (st != HZS_OK) return st;
            // the host runs one chunk ahead of the count of running entries it reads back; the
            // executable graph of chunk c + 1 is updated only after chunk c - 1 has finished
            HZS_CUDA(g, cudaMemcpyAsync(&p->h_done[c & 1], kb.active, sizeof(int), cudaMemcpyDeviceToHost, s));
            HZS_CUDA(g, cudaEventRecord(p->ev[c & 1], s));
            if (c >= 1) {
                HZS_CUDA(g, cudaEventSynchronize(p->ev[(c - 1) & 1]));
                if (p->h_done[(c - 1) & 1] == 0) break;
            }
        }
    }
    // delayed CGS2: the last column is completed by one more dot pass over the basis
    if ((orth32 || d64 || s53) && steps == sd->maxit) {
        if (s53) launch_dcgs2_step53(cx, kb, nb, sd->maxit, 1);
        else if (d64) launch_dcgs2_step64(cx, kb, nb, sd->maxit, 1);
        else launch_dcgs2_step(cx, kb, nb, sd->maxit, 1);
        launches += 4;
    }
    launch_lsq_solve(cx, kb, nb);
    launches += 1;
    if (mixed) {
        launch_combine_Z(cx, kb, nb, p->Z, ld, sZ, u, nn);
        launches += 1;
    } else {
        launch_combine_basis(cx, kb, nb, p->ztmp, ld);
        hzs_status st = precond_apply<double, double2>(p, nb, p->ztmp, ld, nullptr, 0, u, nn, kNoSkip);
        if (st != HZS_OK) return st;
        launches += 1 + pl;
    }
    // true residual ||f - A u|| against the masked right-hand side in V_0
    launch_apply_A<double2, double2, double>(cx, nb, u, nn, p->rtmp, ld, nullptr, 0, kNoSkip);
    launch_residual_norm(cx, kb, nb, kb.V, kb.sVd(), p->rtmp, ld, p->dres);
    launches += 3;
    if (conj_io) { launch_mask_copy_c128(cx, nb, u, nn, u, nn, 1, nullptr, 0); launches += 1; }
    HZS_CUDA(g, cudaGetLastError());
    HZS_CUDA(g, cudaEventRecord(p->t1, s));
    std::vector<KState> hs(nb);
    std::vector<double> rnorm(nb);
    int kerr = 0;
    HZS_CUDA(g, cudaMemcpyAsync(hs.data(), kb.st, nb * sizeof(KState), cudaMemcpyDeviceToHost, s));
    HZS_CUDA(g, cudaMemcpyAsync(rnorm.data(), p->dres, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    HZS_CUDA(g, cudaMemcpyAsync(&kerr, p->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    HZS_CUDA(g, cudaStreamSynchronize(s));
    if (kerr != 0) {
        cudaMemsetAsync(p->err, 0, sizeof(int), s);
        return fail(g, HZS_ERR_TIMEOUT, "a subdomain-solve block gave up waiting for its factor copies");
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p->t0, p->t1);
    double tp = 0, tm = 0, to = 0, tdot = 0, tupd = 0;
    if (prof) {
        for (int k = 0; k < steps; ++k) {
            cudaEvent_t* pe = &p->prof_ev[(size_t)8 * k];
            float a = 0, b = 0, c = 0;
            cudaEventElapsedTime(&a, pe[0], pe[1]);
            cudaEventElapsedTime(&b, pe[1], pe[2]);
            cudaEventElapsedTime(&c, pe[2], pe[3]);
            tp += a; tm += b; to += c;
            if (orth32 || d64 || s53) {
                float d = 0, u = 0;
                cudaEventElapsedTime(&d, pe[4], pe[5]);
                cudaEventElapsedTime(&u, pe[6], pe[7]);
                tdot += d; tupd += u;
            }
        }
    }
    hzs_status worst = HZS_OK;
    for (int r = 0; r < nb; ++r) {
        hzs_solve_info inf{};
        inf.t_precond_ms = tp; inf.t_matvec_ms = tm; inf.t_orth_ms = to;
        inf.t_orth_dot_ms = tdot; inf.t_orth_update_ms = tupd;
        inf.iterations = hs[r].iters;
        inf.converged = hs[r].conv;
        inf.relres_est = hs[r].beta0 > 0 ? hs[r].resid / hs[r].beta0 : 0.0;
        inf.relres_true = hs[r].beta0 > 0 ? rnorm[r] / hs[r].beta0 : 0.0;
        inf.t_solve_ms = ms;
        inf.launches = launches;
        inf.basis_bits = !orth32 ? 53 : (lo16 ? 32 : 48);
        inf.orth_kind = orth;
        inf.status = hs[r].nonfinite ? HZS_ERR_NONFINITE : (hs[r].conv ? HZS_OK : HZS_NOT_CONVERGED);
        if (info) info[r] = inf;
        if (inf.status == HZS_ERR_NONFINITE) worst = HZS_ERR_NONFINITE;
        else if (inf.status == HZS_NOT_CONVERGED && worst == HZS_OK) worst = HZS_NOT_CONVERGED;
    }
    if (worst == HZS_ERR_NONFINITE)
        return fail(g, HZS_ERR_NONFINITE, "non-finite value in a right-hand side or in the iteration");
    return worst;
}

// All right-hand sides of one call, in lockstep batches as large as the free
// device memory allows (the Krylov space of every entry is resident).
// budget: device bytes this call may take for Krylov space (0: 80 % of the free memory).
static hzs_status solve_many(hzs_precond* p, const hzs_solve_desc* sd, const void* f_dev, void* u_dev, int nrhs,
                             hzs_solve_info* info, int conj_io, size_t budget = 0) {
    if (!p) return fail(nullptr, HZS_ERR_INVALID_ARG, "precond is NULL");
    hzs_grid* g = p->g;
    if (!sd || !f_dev || !u_dev || nrhs < 0) return fail(g, HZS_ERR_INVALID_ARG, "bad arguments");
    if (!(sd->tol > 0.0) || sd->maxit < 1) return fail(g, HZS_ERR_INVALID_ARG, "tol must be > 0 and maxit >= 1");
    if (nrhs == 0) return HZS_OK;
    int nb = nrhs;
    // the complex128 basis for the FP64 CGS2 and the all-FMA delayed CGS2; the double-float
    // and f53 paths keep only its slot 0 (the right-hand side) and the head/remainder arrays
    const int om = orth_mode(p, sd);
    const bool full_v = om == kOrthCGS2 || om == kOrthD64;
    if (!(p->kb.V && p->kb.maxit >= sd->maxit && p->kb.nb >= nrhs && p->kb.vfull == (full_v ? 1 : 0))) {
        free_krylov(p);
        size_t fr = 0, tot = 0;
        HZS_CUDA(g, cudaMemGetInfo(&fr, &tot));
        const long long N = (long long)g->desc.n * g->desc.n;
        const size_t per = krylov_entry_bytes(p, sd->maxit, (N + 63) / 64 * 64, full_v);
        const double avail = budget ? std::min((double)budget, 0.9 * (double)fr) : 0.8 * (double)fr;
        const long long fit = (long long)avail / (long long)per;
        if (fit < 1) return fail(g, HZS_ERR_OOM, "not enough device memory for one Krylov space of maxit steps");
        nb = (int)std::min<long long>(nrhs, fit);
        hzs_status st = ensure_krylov(p, sd->maxit, nb, full_v);
        if (st != HZS_OK) return st;
    }
    nb = std::min(nrhs, p->kb.nb);
    const long long nn = (long long)g->desc.n * g->desc.n;
    hzs_status worst = HZS_OK;
    for (int r0 = 0; r0 < nrhs; r0 += nb) {
        const int cnt = std::min(nb, nrhs - r0);
        hzs_status st = solve_batch(p, sd, (const double2*)f_dev + r0 * nn, (double2*)u_dev + r0 * nn, cnt, conj_io,
                                    info ? info + r0 : nullptr);
        if (st < 0) return st;
        if (st == HZS_NOT_CONVERGED) worst = HZS_NOT_CONVERGED;
    }
    return worst;
}

extern "C" hzs_status hzs_solve(hzs_precond* p, const hzs_solve_desc* sd, const void* f_dev, void* u_dev, int nrhs,
                                hzs_solve_info* info) {
    return solve_many(p, sd, f_dev, u_dev, nrhs, info, 0);
}

extern "C" hzs_status hzs_adjoint_solve(hzs_precond* p, const hzs_solve_desc* sd, const void* g_dev, void* lam_dev,
                                        int nrhs, hzs_solve_info* info) {
    return solve_many(p, sd, g_dev, lam_dev, nrhs, info, 1);
}

extern "C" hzs_status hzs_solve_batched(int nprob, hzs_precond* const* probs, const hzs_solve_desc* sd,
                                        const void* const* f_dev, void* const* u_dev, const int* nrhs,
                                        hzs_solve_info* info) {
    if (nprob < 0 || (nprob > 0 && (!probs || !f_dev || !u_dev || !nrhs)))
        return fail(nullptr, HZS_ERR_INVALID_ARG, "bad batched-solve arguments");
    for (int k = 0; k < nprob; ++k) {
        if (!probs[k]) return fail(nullptr, HZS_ERR_INVALID_ARG, "NULL preconditioner in batch");
        for (int l = 0; l < k; ++l)
            if (probs[l] == probs[k]) return fail(nullptr, HZS_ERR_INVALID_ARG, "a preconditioner appears twice");
    }
    std::vector<long long> off(nprob + 1, 0);
    for (int k = 0; k < nprob; ++k) off[k + 1] = off[k] + nrhs[k];
    std::vector<hzs_status> st(nprob, HZS_OK);
    int dev = 0;
    cudaGetDevice(&dev);
    // the problems allocate their Krylov spaces at the same time: split 80 % of the free
    // memory by water-filling, each problem at most what all its right-hand sides need
    // (so that the small problems leave the rest to the large ones, which then solve
    // their right-hand sides in fewer, larger lockstep batches)
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    std::vector<double> need(nprob), share(nprob, 0.0);
    for (int k = 0; k < nprob; ++k) {
        const long long N = (long long)probs[k]->g->desc.n * probs[k]->g->desc.n;
        const int om = orth_mode(probs[k], sd);
        need[k] = (double)krylov_entry_bytes(probs[k], sd->maxit, (N + 63) / 64 * 64,
                                             om == kOrthCGS2 || om == kOrthD64) * std::max(nrhs[k], 1);
    }
    {
        double left = 0.8 * (double)fr;
        std::vector<int> open;
        for (int k = 0; k < nprob; ++k) open.push_back(k);
        while (!open.empty()) {
            const double each = left / (double)open.size();
            std::vector<int> rest;
            for (int k : open) {
                if (need[k] <= each) { share[k] = need[k]; left -= need[k]; }
                else rest.push_back(k);
            }
            if (rest.size() == open.size()) {
                for (int k : rest) share[k] = each;
                break;
            }
            open.swap(rest);
        }
    }
    std::vector<std::thread> th;
    for (int k = 0; k < nprob; ++k) {
        th.emplace_back([&, k]() {
            cudaSetDevice(dev);
            st[k] = solve_many(probs[k], sd, f_dev[k], u_dev[k], nrhs[k], info ? info + off[k] : nullptr, 0,
                               share[k] >= 1.0 ? (size_t)share[k] : 1);
        });
    }
    for (auto& t : th) t.join();
    hzs_status worst = HZS_OK;
    for (int k = 0; k < nprob; ++k) {
        if (st[k] < 0) {
            g_global_err = std::string("problem ") + std::to_string(k) + ": " + probs[k]->g->err;
            return st[k];
        }
        if (st[k] == HZS_NOT_CONVERGED) worst = HZS_NOT_CONVERGED;
    }
    return worst;
}

extern "C" hzs_status hzs_kappa_gradient(hzs_precond* p, const void* u_dev, const void* lam_dev, double* grad_dev) {
    if (!p) return fail(nullptr, HZS_ERR_INVALID_ARG, "precond is NULL");
    if (!u_dev || !lam_dev || !grad_dev) return fail(p->g, HZS_ERR_INVALID_ARG, "NULL buffer");
    launch_kappa_gradient(p->cx, (const double2*)u_dev, (const double2*)lam_dev, grad_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(p->g, e, "kappa_gradient");
    return HZS_OK;
}

extern "C" const char* hzs_status_string(hzs_status s) {
    switch (s) {
        case HZS_OK: return "ok";
        case HZS_NOT_CONVERGED: return "not converged";
        case HZS_ERR_INVALID_ARG: return "invalid argument";
        case HZS_ERR_CUDA: return "CUDA error";
        case HZS_ERR_OOM: return "out of device memory";
        case HZS_ERR_SINGULAR_LOCAL: return "singular subdomain matrix";
        case HZS_ERR_SINGULAR_COARSE: return "singular coarse matrix";
        case HZS_ERR_NONFINITE: return "non-finite value";
        case HZS_ERR_TIMEOUT: return "timeout";
        case HZS_ERR_BREAKDOWN: return "breakdown";
    }
    return "unknown status";
}

extern "C" const char* hzs_last_error(const hzs_grid* g) { return g ? g->err.c_str() : g_global_err.c_str(); }

extern "C" const char* hzs_version(void) { return "hzs 0.1 (sm_103a)"; }

// ------------------------------------------------------------------ internal accessors (noalloc.cu)
hzs_status hzs_internal_set_error(hzs_precond* p, hzs_status s, const std::string& msg) {
    return fail(p ? p->g : nullptr, s, msg);
}

hzs_status hzs_internal_noalloc_view(hzs_precond* p, NoAllocView* v, std::string* err) {
    if (!p) return fail(nullptr, HZS_ERR_INVALID_ARG, "precond is NULL");
    if (p->coarse_block || p->coarse_ml)
        return fail(p->g, HZS_ERR_INVALID_ARG,
                    "the allocation-free apply supports the dense coarse inverse only (coarse_solver DENSE/AUTO "
                    "with at most 4096 coarse unknowns)");
    v->cx = p->cx;
    v->kind = p->desc.kind;
    v->precision = p->desc.precision;
    v->nc1 = p->hct.nc1;
    v->Nc = p->Nc;
    v->groups = tile_groups(p);
    v->max_mx = p->g->max_mx;
    v->max_my = p->g->max_my;
    v->Ainv = p->Ainv;
    v->W64 = p->W64;
    v->W32 = p->W32;
    v->tiles = p->tiles_d;
    (void)err;
    return HZS_OK;
}
