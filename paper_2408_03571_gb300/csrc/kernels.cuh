// Internal declarations shared by the kernel files and the C ABI layer.
//
// Batches: every per-iteration launcher takes the number of right-hand sides
// nb it works on; batch entry r addresses its vectors at r times the stride
// given for each buffer (element counts), and is skipped when its "done" flag
// (BatchSkip) is set.
#pragma once

#include <string>

#include <vector>

#include "common.cuh"

namespace hzs {

// Lets fn launch with `bytes` of dynamic shared memory.  Without an opt-in a
// block may use 48 KB of static and dynamic shared memory together, so the
// check counts the function's static shared memory too.  The function's cap is
// process-wide state shared by every host thread, so it is always raised to the
// same value (the device's opt-in maximum less the function's static shared
// memory) rather than to this launch's size: a concurrent caller that needs less
// can then never lower the cap under a launch that needs more.
inline cudaError_t allow_dynamic_smem(const void* fn, size_t bytes) {
    constexpr size_t kDefault = 48 * 1024;
    if (bytes <= kDefault / 2) return cudaSuccess;      // no kernel here has 24 KB of static shared memory
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if (bytes + fa.sharedSizeBytes <= kDefault) return cudaSuccess;
    int dev = 0, optin = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t cap = (size_t)optin - fa.sharedSizeBytes;
    if (bytes > cap) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
}

// Host copy of the 1-D coarse tables (see CoarseTab).
struct HostCoarseTab {
    int nc1 = 0;
    int bad = 0;                 // a fine node touches coarse indices outside its 3-wide window
    std::vector<int> c0;
    std::vector<double> w;
    std::vector<int> lo, hi, off;
    std::vector<double> wt;
};
void build_coarse_tables(int n, int bc, int kind, int p, HostCoarseTab& t);

// Everything a launch needs about the problem.
struct Ctx {
    OpDesc op;
    CoarseTab ct;
    cudaStream_t stream;
    int num_sms;
    int* err;          // device error word: kernels that time out set it (HZS_ERR_TIMEOUT); may be null
    long long spin_limit = 1LL << 24;   // polls of a subdomain-solve stage wait before it is declared timed out
};

// Per-batch-entry skip flag: entry r is skipped when flag[r * stride] != 0 (flag may be null).
struct BatchSkip {
    const int* flag;
    int stride;
};

// Subdomain tiles grouped by shared factor: group g solves tiles idx[g*T .. g*T+T-1]
// (entries -1 are empty); all tiles of a group have the same factor.  nst (depth of
// the factor-block copy ring: 1, 2 or 4) and tpr (threads per block row: 4 or 8)
// fix the launch shape of the subdomain solve; 0 lets the launch pick (deepest
// ring that fits, 8 threads per row while a block stays within 1024 threads).
struct TileGroups {
    const int* idx;
    int count;
    int T;
    int nst;
    int tpr;
};

// Per distinct subdomain factor: representative tile geometry.
struct FactorDesc {
    int x0, y0, mx, my;
    long long woff;
};

struct FactorStat {
    double minpiv;     // smallest |pivot| over the factor's block inversions
    double maxabs;     // largest |entry| of the stored inverse blocks
    int singular;
    int pad;
};

// ---- operator.cu
template <typename Cin, typename Cout, typename R>
void launch_apply_A(const Ctx& cx, int nb, const Cin* x, long long xs, Cout* y, long long ys, float2* y32,
                    long long y32s, BatchSkip sk, LoDst y32lo = LoDst{nullptr, nullptr});
// y = A x in double-float arithmetic, y as the pair yh + yl (see LoDst); false (nothing
// launched) when the couplings are not exact in FP32 (n > 4097).
// y = A x (complex64 x, FP64 arithmetic) stored as f53 heads yh and tails yt
void launch_apply_A_f53(const Ctx& cx, int nb, const float2* x, long long xs, float2* yh, uint2* yt, long long ys,
                        BatchSkip sk);
bool launch_apply_A_df(const Ctx& cx, int nb, const float2* x, long long xs, float2* yh, LoDst yl, long long ys,
                       BatchSkip sk);
template <typename Cv, typename Cw, typename R>
void launch_deflate(const Ctx& cx, int nb, const cplx_t<R>* c, long long cs, const Cv* v, long long vs,
                    const double* vscale, long long vss, Cw* w, long long ws, BatchSkip sk);
template <typename Cz, typename Cy, typename R>
void launch_combine_additive(const Ctx& cx, int nb, const cplx_t<R>* c, long long cs, int use_coarse,
                             const int4* cover_x, const int4* cover_y, const Tile* tiles, int nsx, const Cy* ytiles,
                             long long yts, Cz* z, long long zs, BatchSkip sk, int weighted);
void launch_mask_copy_c128(const Ctx& cx, int nb, const double2* src, long long ss, double2* dst, long long ds,
                           int conj, float2* dst32, long long d32s, LoDst dst32lo = LoDst{nullptr, nullptr});
void launch_kappa_gradient(const Ctx& cx, const double2* u, const double2* lam, double* grad);

// ---- coarse.cu
// t = x-pass of R_0 (s v) (stride ts per entry), c = R_0 (s v) in FP64 (stride Nc)
template <typename Cv, typename R>
void launch_restrict(const Ctx& cx, int nb, const Cv* v, long long vs, const double* vscale, long long vss,
                     cplx_t<R>* t, double2* c, BatchSkip sk);
// out = Ainv c in FP64 (stride Nc); outf (if given) receives a complex64 copy
void launch_coarse_matvec(const Ctx& cx, int nb, const double2* Ainv, int Nc, const double2* c, double2* out,
                          float2* outf, BatchSkip sk);
void launch_galerkin(const Ctx& cx, double2* A0);
// banded A_0: 25 entries per coarse row, offset (dI, dJ) at (dJ + 2) * 5 + (dI + 2)
void launch_galerkin_banded(const Ctx& cx, double2* A0b);

// ---- coarse_block.cu: block-tridiagonal LU of A_0 over groups of s coarse rows
struct CoarseBlockLU {
    int nc1 = 0, s = 0, m = 0;            // m block rows of s coarse rows (the last may be shorter)
    int rad = 2;                          // band radius of the matrix (its couplings reach rad rows)
    std::vector<int> b, r0;               // block sizes and first unknowns
    std::vector<long long> wo, po, qo;    // offsets of W_i, P_i, Q_i
    double2* W = nullptr;                 // W_i = S_i^{-1}        (b_i x b_i)
    double2* P = nullptr;                 // P_i = W_i L_i         (b_i x b_{i-1})
    double2* Q = nullptr;                 // Q_i = W_i U_i         (b_i x b_{i+1})
    double2* A0b = nullptr;               // A_0 in band form (Nc x 25), owned: the couplings L_i, U_i
    // tensor-core form of the many-right-hand-side products W_i X (coarse_oz.cu); Aoz is
    // null when it is not built
    unsigned char* Aoz = nullptr;         // bf16 digit slices of [Re W_i | Im W_i], block i at aoz[i]
    std::vector<long long> aoz;
    std::vector<int> oz_mt, oz_kch;       // per block: 128-row tiles, 64-wide K chunks
    int* eoz = nullptr;                   // per coarse unknown: scale exponent of its row of W_i
    int oz_cap = 0;                       // right-hand sides the work space below holds
    unsigned char* Boz = nullptr;         // digit slices of one block step's right-hand sides
    float* Poz = nullptr;                 // per-CTA partial sums (three-word expansions)
    int* foz = nullptr;                   // per right-hand side: scale exponent
};
// 0 on success, 1 if a pivot was zero, -1 on a CUDA error; *minpiv = smallest |pivot|.
// Takes ownership of A0b (freed by coarse_block_free, or here on failure).
int coarse_block_setup(const Ctx& cx, int nc1, int s, int rad, double2* A0b, CoarseBlockLU& lu, double* minpiv);
void coarse_block_free(CoarseBlockLU& lu);
// out = A_0^{-1} c (FP64, stride nc1^2 per batch entry); outf (if given) its complex64 rounding.
// c is overwritten (it holds the intermediate vectors of the sweeps).
void launch_coarse_block_solve(const Ctx& cx, int nb, const CoarseBlockLU& lu, double2* c, double2* out,
                               float2* outf, BatchSkip sk);
// Tensor-core products of the many-right-hand-side sweeps (coarse_oz.cu).  setup: 0 built,
// 1 not applicable (a block wider than 520), -1 CUDA error; reserve: work space for nb
// right-hand sides (0 / -1).  One step: out = W_i x (or out - W_i x when subtract), FP64-
// accurate, for the nb vectors x + c stride.
int coarse_oz_setup(const Ctx& cx, CoarseBlockLU& lu);
int coarse_oz_reserve(CoarseBlockLU& lu, int nb);
void coarse_oz_free(CoarseBlockLU& lu);
void launch_coarse_oz_step(const Ctx& cx, int nb, const CoarseBlockLU& lu, int i, const double2* x, double2* out,
                           bool subtract, long long stride, BatchSkip sk);

// Multilevel coarse solve (coarse_ml.cu): SHS2 on the coarse grid G_H in place of A_0^{-1}.
struct CoarseML {
    int nc1 = 0, Nc = 0;        // G_H unknowns per axis, in all
    int lo0 = 0;                // pseudo-grid index of G_H unknown 0 (1 for MP-1, 0 for MP-2)
    int nc00 = 0, Nc00 = 0;     // coarse-of-coarse unknowns per axis, in all
    int *lo2 = nullptr, *hi2 = nullptr, *off2 = nullptr, *c02 = nullptr;   // level-2 B_2 tables
    double *wt2 = nullptr, *w2 = nullptr;
    double2* A00inv = nullptr;  // Nc00 x Nc00
    int nsub = 0, max_own = 0, max_m = 0;
    int4* sub = nullptr;        // per coarse subdomain: extended rectangle x0, y0, mx, my (G_H indices)
    int4* own = nullptr;        // per coarse subdomain: owned x0, x1, y0, y1 (inclusive)
    long long* aoff = nullptr;  // per coarse subdomain: offset of its dense inverse in Ainv
    double2* Ainv = nullptr;
    double2* A0b = nullptr;     // A_0 in band form (Nc x 25), owned
    double2 *c00 = nullptr, *c00p = nullptr, *q = nullptr, *wv = nullptr;   // work, nb_cap right-hand sides
    int nb_cap = 0;
    int blk00 = 0;              // coarse-of-coarse solve by block LU (above 4096 unknowns) instead of A00inv
    CoarseBlockLU cblk00;
};
// 0 on success, 1 if a pivot was zero, -1 on a CUDA error, -2 on a bad parameter (*why);
// takes ownership of A0b.
int coarse_ml_setup(const Ctx& cx, int nc1, int bc, double2* A0b, int ns0, int ov0, int p0, CoarseML& ml,
                    double* minpiv, std::string* why);
void coarse_ml_free(CoarseML& ml);
int coarse_ml_reserve(CoarseML& ml, int nb);
// out = M_0^{-1} c (FP64, stride nc1^2 per batch entry); outf (if given) its complex64 rounding
void launch_coarse_ml_solve(const Ctx& cx, int nb, const CoarseML& ml, const double2* c, double2* out, float2* outf,
                            BatchSkip sk);

int gj_invert(const Ctx& cx, double2* a, int N, double* minpiv);

// ---- local.cu
int max_tile_extent();
int launch_tile_factor(const Ctx& cx, const FactorDesc* fdesc_dev, int nfactors, int max_m, double2* W64,
                       float2* W32, FactorStat* stat_dev);
// mode 0: restricted (D_i) write z = [q] + y on owned nodes; mode 1: write tile y to ytiles
template <typename Cw, typename Cz, typename R>
int launch_tile_solve(const Ctx& cx, int nb, const Tile* tiles, TileGroups grp, int max_mx, int max_my,
                      const cplx_t<R>* W, const Cw* w, long long ws, const double* vscale, long long vss, int mode,
                      const cplx_t<R>* c, long long cs, int use_coarse, Cz* z, long long zs, cplx_t<R>* ytiles,
                      long long yts, BatchSkip sk);
// Largest number of tiles per group (1 or 2) whose shared-memory footprint fits for
// tiles of at most max_mx x max_my in arithmetic of size elem_bytes; 0 if none fits.
int tile_group_width(int max_mx, int max_my, int elem_bytes);
// The launch shape (T, nst, tpr) that launch_tile_solve uses for grp (resolving zeros
// as it does); false if that shape does not fit (shared memory, threads per block).
bool tile_shape_resolve(const TileGroups& grp, int max_mx, int max_my, int elem_bytes, int* T, int* nst, int* tpr);

// ---- krylov.cu
struct alignas(16) KState {
    double beta0;      // ||f||
    double tolabs;     // tol * ||f||
    double resid;      // current GMRES residual estimate |g_{j+1}|
    double hnext;      // ||w|| of the last step
    int done;          // iteration finished (converged, breakdown or non-finite)
    int conv;
    int iters;         // completed Arnoldi steps
    int nonfinite;
    int breakdown;
    int pad[3];
};
constexpr int kStateInts = (int)(sizeof(KState) / sizeof(int));   // stride of KState::done in ints

// Krylov work space for a batch of nb right-hand sides.  Every array holds nb
// entries; entry r starts at r times the per-entry stride.
struct KrylovBufs {
    int maxit;
    int nb;            // batch capacity
    long long N;       // vector length (n*n)
    long long ld;      // leading dimension between basis vectors (elements)
    int nblk;          // blocks of the reduction kernels
    int nblk_dot;      // blocks of the delayed-CGS2 dot pass (rows of part; >= nblk)
    double2* V;        // complex128 basis: (maxit+1) x ld per entry, or only slot 0 (the masked
                       // right-hand side) when vfull == 0 (the double-float path keeps no FP64 basis)
    int vfull;
    float2* V32;       // (maxit+1) x ld complex64 roundings of the basis (delayed CGS2 path), or null
    void* V32lo;       // (maxit+1) x ld remainders: V32 + V32lo is the basis as double-float pairs,
                       // complex64 words or, with lo16, bf16 pairs (LoDst); sized for complex64
    int lo16;          // remainders stored as bf16 pairs (set per solve)
    // f53 basis: vectors i with bit i % 8 set are summed with FP64 FMAs in the dot pass / the
    // update pass, the others in FP32 error-free arithmetic.  Defaults: the fastest of the
    // splits, occupancies, task sizes and copy rings measured at the headline size
    unsigned dmask_dot = 0x6Du;    // 5 of 8 vectors on the FP64 path
    unsigned dmask_upd = 0x6Du;    // 5 of 8
    int s53_minb = 2;      // update pass: blocks per SM it is compiled for (2 or 3)
    int s53_ring = 4;      // dot pass: stages of its per-thread shared-memory copy ring (0: none)
    int s53_group = 4;     // dot pass: basis vectors per warp task on the FP32 path (1, 2; 4 with
                           // specialised warps)
    int s53_dot_minb = 2;  // dot pass: blocks per SM it is compiled for (2, 3 or 4)
    int s53_ws = 1;        // dot pass: each warp task on one of the two paths (k_s53_dot_ws)
    int s53_upd_e = 2;     // update pass: entries per thread and sweep (1 or 2)
    int s53_g64 = 4;       // dot pass, specialised warps: vectors per FP64 task (4 or 8)
    int s53_ring64 = 1;    // dot pass, specialised warps: FP64 tasks also through the copy ring
    int s53_dot_waves = 1; // dot pass at 2 blocks/SM: launched as one or two waves of blocks
    double* sigma;     // (maxit+1): basis vector i = sigma[i] * V_i
    double2* H;        // (maxit+1) x maxit, column j at H[j*(maxit+1)]
    double* cs;        // maxit+1
    double2* sn;       // maxit+1
    double2* g;        // maxit+1
    double2* y;        // maxit+1
    double2* h1;       // maxit+1
    double2* h2;       // maxit+1
    double2* hn;       // maxit+2: reduced dots of the delayed CGS2 step (new column, then c and d)
    double* sigt;      // maxit+1: 1 / |u~_j|, the preconditioner's input scale on the delayed CGS2 path
    double2* part;     // nblk x pstride()
    double* npart;     // nblk
    KState* st;        // 1
    int* active;       // one counter per batch: entries not yet done
    cudaStream_t side; // runs the Givens rotation of a delayed-CGS2 step beside its update pass (or null)
    cudaEvent_t ev_c;  // coefficients of the step ready (recorded on the solve stream)
    cudaEvent_t ev_g;  // Givens rotation of the step done (recorded on side)
    long long sV() const { return (long long)(maxit + 1) * ld; }
    long long sVd() const { return vfull ? sV() : ld; }   // per-entry stride of V
    long long sH() const { return (long long)(maxit + 1) * maxit; }
    long long sS() const { return maxit + 1; }
    long long sN() const { return maxit + 2; }
    int pstride() const { return 2 * (maxit + 1) + 2; }
    long long sP() const { return (long long)nblk_dot * pstride(); }
    BatchSkip skip() const { return BatchSkip{&st->done, kStateInts}; }
    // remainders of basis slot i of batch entry 0 (entry r at r * sV() further)
    LoDst lo_at(long long i) const {
        const long long off = i * ld;
        return lo16 ? LoDst{nullptr, static_cast<__nv_bfloat162*>(V32lo) + off}
                    : LoDst{static_cast<float2*>(V32lo) + off, nullptr};
    }
};
void launch_norm_init(const Ctx& cx, const KrylovBufs& kb, int nb, double tol);
void launch_arnoldi_step(const Ctx& cx, const KrylovBufs& kb, int nb, int j);
// Step j of the delayed CGS2 Arnoldi on the double-float basis (V32 + V32lo, lo16 selects
// the remainder width; the rotation of column j-1 runs on kb.side beside the update pass,
// and the solve stream waits for it before the step ends);
// last_only (j == maxit) completes the last Hessenberg column only.  ev (optional,
// 4 events) is recorded before and after the dot pass and the update pass.
void launch_dcgs2_step(const Ctx& cx, const KrylovBufs& kb, int nb, int j, int last_only, cudaEvent_t* ev = nullptr);
// Step j of the delayed CGS2 Arnoldi on the FP64 basis kb.V (FP64 reorthogonalisation
// dots and first-projection update, complex64 first-projection dots; same arguments).
void launch_dcgs2_step64(const Ctx& cx, const KrylovBufs& kb, int nb, int j, int last_only,
                         cudaEvent_t* ev = nullptr);
// Step j of the delayed CGS2 on the f53 basis (heads V32, 29-bit tails V32lo), the
// FP64-accurate work split between the FP64 and the FP32 pipes; false if the update
// pass could not be launched (its coefficients exceed shared memory).
bool launch_dcgs2_step53(const Ctx& cx, const KrylovBufs& kb, int nb, int j, int last_only,
                         cudaEvent_t* ev = nullptr);
// ---- orth53.cu
void launch_f53_encode(const Ctx& cx, int nb, long long N, const double2* src, long long ss, float2* dh, uint2* dt,
                       long long ds, const double* scale, const KState* st);
void launch_f53_scale0(const Ctx& cx, int nb, double* sigma, double* sigt, long long sS, double* scale);
size_t s53_update_smem(int j);
int launch_s53_dot(const Ctx& cx, const KrylovBufs& kb, int nb, int j, int has_w, unsigned dmask);
int launch_s53_update(const Ctx& cx, const KrylovBufs& kb, int nb, int j, unsigned dmask);
void launch_lsq_solve(const Ctx& cx, const KrylovBufs& kb, int nb);
void launch_combine_basis(const Ctx& cx, const KrylovBufs& kb, int nb, double2* x, long long xs);
void launch_combine_Z(const Ctx& cx, const KrylovBufs& kb, int nb, const float2* Z, long long ldz, long long zs,
                      double2* x, long long xs);
void launch_residual_norm(const Ctx& cx, const KrylovBufs& kb, int nb, const double2* f, long long fs,
                          const double2* Ax, long long axs, double* out);

// What the allocation-free apply (noalloc.cu) needs from a preconditioner handle.
struct NoAllocView {
    Ctx cx;
    int kind, precision, nc1, Nc, max_mx, max_my;
    TileGroups groups;
    const double2* Ainv;
    const double2* W64;
    const float2* W32;
    const Tile* tiles;
};

}  // namespace hzs
