// GMRES kernels (Section 5): Arnoldi with classical Gram-Schmidt and one
// reorthogonalisation (CGS2), Givens rotations on the Hessenberg matrix,
// the triangular solve and the solution update.
//
// Basis vectors are stored unnormalised: the i-th orthonormal vector is
// sigma[i] * V_i.  The scale is folded into the dot products and the update
// coefficients, so no separate normalisation pass over the vector is needed.
//
// Every per-iteration kernel returns at once when the iteration has already
// finished (st->done), so the host may enqueue an iteration before it knows
// whether the previous one converged.
//
// Reductions are deterministic: fixed chunks per block, fixed lane order in
// the warp trees, and the cross-block sums in a fixed order.
#include "kernels.cuh"

namespace hzs {

constexpr int kRedThreads = 256;
constexpr int kDotGroup64 = 4;     // basis vectors per warp pass (FP64 multi-dot)
constexpr int kDotGroup32 = 8;     // basis vectors per warp pass (complex64 multi-dot)

__device__ __forceinline__ void chunk_of(long long N, long long& e0, long long& e1) {
    const long long per = (N + gridDim.x - 1) / gridDim.x;
    e0 = (long long)blockIdx.x * per;
    e1 = e0 + per < N ? e0 + per : N;
}

// part[b][i] = sum_{e in chunk b} conj(V_i[e]) w[e], i = 0..j, with products and
// sums in the precision of C.  Each warp takes groups of G basis vectors and
// sweeps the whole chunk of its block for them (w is re-read from L1), so no
// block-wide barrier is needed; lane 0 of the warp writes the group's partials.
template <typename C, int G>
__global__ void __launch_bounds__(kRedThreads) k_multidot(int j, long long N, long long ld, int stride,
                                                          const C* __restrict__ V, const C* __restrict__ w,
                                                          double2* __restrict__ part,
                                                          const KState* __restrict__ st) {
    if (st->done) return;
    long long e0, e1;
    chunk_of(N, e0, e1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ngroups = (j + G) / G;
    for (int gi = warp; gi < ngroups; gi += nw) {
        const int i0 = gi * G;
        C acc[G];
#pragma unroll
        for (int t = 0; t < G; ++t) { acc[t].x = 0; acc[t].y = 0; }
        for (long long e = e0 + lane; e < e1; e += 32) {
            const C we = w[e];
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (i0 + t <= j) acc[t] = cfma_conj(V[(size_t)(i0 + t) * ld + e], we, acc[t]);
        }
#pragma unroll
        for (int t = 0; t < G; ++t) acc[t] = warp_sum(acc[t]);
        if (lane == 0) {
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (i0 + t <= j) part[(size_t)blockIdx.x * stride + i0 + t] = to_d(acc[t]);
        }
    }
}

// h[i] = sigma[i] * sum_b part[b][i]   (one warp per i, fixed order)
__global__ void k_reduce_dots(int j, int nblk, int stride, const double2* __restrict__ part,
                              const double* __restrict__ sigma, double2* __restrict__ h,
                              const KState* __restrict__ st) {
    if (st->done) return;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i > j) return;
    double2 s = make_double2(0.0, 0.0);
    for (int b = lane; b < nblk; b += 32) s = cadd(s, part[(size_t)b * stride + i]);
    s = warp_sum(s);
    if (lane == 0) h[i] = cscale(s, sigma[i]);
}

__device__ __forceinline__ void block_norm_part(double nrm, double* __restrict__ npart) {
    __shared__ double nred[kRedThreads / 32];
    nrm = warp_sum_d(nrm);
    if ((threadIdx.x & 31) == 0) nred[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += nred[k];
        npart[blockIdx.x] = s;
    }
}

// w[e] -= sum_i (h[i] sigma[i]) V_i[e] in FP64; optionally npart[b] = sum_e |w[e]|^2.
// Four independent partial sums per element keep several loads in flight.
__global__ void __launch_bounds__(kRedThreads) k_axpy_multi(int j, long long N, long long ld,
                                                            const double2* __restrict__ V,
                                                            const double* __restrict__ sigma,
                                                            const double2* __restrict__ h, double2* __restrict__ w,
                                                            double* __restrict__ npart, const KState* __restrict__ st) {
    if (st->done) return;
    extern __shared__ double2 coef[];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) coef[i] = cscale(h[i], sigma[i]);
    __syncthreads();
    long long e0, e1;
    chunk_of(N, e0, e1);
    double nrm = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        double2 a0 = w[e];
        double2 a1 = make_double2(0.0, 0.0), a2 = a1, a3 = a1;
        int i = 0;
        for (; i + 3 <= j; i += 4) {
            a0 = cfms(coef[i], V[(size_t)i * ld + e], a0);
            a1 = cfms(coef[i + 1], V[(size_t)(i + 1) * ld + e], a1);
            a2 = cfms(coef[i + 2], V[(size_t)(i + 2) * ld + e], a2);
            a3 = cfms(coef[i + 3], V[(size_t)(i + 3) * ld + e], a3);
        }
        for (; i <= j; ++i) a0 = cfms(coef[i], V[(size_t)i * ld + e], a0);
        double2 we;
        we.x = (a0.x + a1.x) + (a2.x + a3.x);
        we.y = (a0.y + a1.y) + (a2.y + a3.y);
        w[e] = we;
        nrm = fma(we.x, we.x, fma(we.y, we.y, nrm));
    }
    if (npart) block_norm_part(nrm, npart);
}

// w[e] -= sum_i (h[i] sigma[i]) V32_i[e], the sum in complex64 and the
// subtraction in FP64 (h is the small reorthogonalisation coefficient, so a
// single-precision sum is accurate to FP64 level relative to w); also writes
// w32 = complex64(w) and npart[b] = sum_e |w[e]|^2.
__global__ void __launch_bounds__(kRedThreads) k_correct32(int j, long long N, long long ld,
                                                           const float2* __restrict__ V32,
                                                           const double* __restrict__ sigma,
                                                           const double2* __restrict__ h, double2* __restrict__ w,
                                                           float2* __restrict__ w32, double* __restrict__ npart,
                                                           const KState* __restrict__ st) {
    if (st->done) return;
    extern __shared__ float2 coef32[];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) coef32[i] = to_f(cscale(h[i], sigma[i]));
    __syncthreads();
    long long e0, e1;
    chunk_of(N, e0, e1);
    double nrm = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        float2 c0 = make_float2(0.f, 0.f), c1 = c0, c2 = c0, c3 = c0;
        int i = 0;
        for (; i + 3 <= j; i += 4) {
            c0 = cfma(coef32[i], V32[(size_t)i * ld + e], c0);
            c1 = cfma(coef32[i + 1], V32[(size_t)(i + 1) * ld + e], c1);
            c2 = cfma(coef32[i + 2], V32[(size_t)(i + 2) * ld + e], c2);
            c3 = cfma(coef32[i + 3], V32[(size_t)(i + 3) * ld + e], c3);
        }
        for (; i <= j; ++i) c0 = cfma(coef32[i], V32[(size_t)i * ld + e], c0);
        double2 we = w[e];
        we.x -= (double)((c0.x + c1.x) + (c2.x + c3.x));
        we.y -= (double)((c0.y + c1.y) + (c2.y + c3.y));
        w[e] = we;
        w32[e] = to_f(we);
        nrm = fma(we.x, we.x, fma(we.y, we.y, nrm));
    }
    block_norm_part(nrm, npart);
}

// Completes step j: h_{j+1,j} = ||w||, column j of H = h1 + h2, Givens
// rotations, residual estimate, convergence / breakdown flags.  One warp: the
// block norm partials are summed in a fixed lane order, the column and the
// rotations are staged in shared memory, and lane 0 applies the rotation chain.
__global__ void k_arnoldi_finish(int j, int maxit, int nblk, const double* __restrict__ npart,
                                 const double2* __restrict__ h1, const double2* __restrict__ h2,
                                 double2* __restrict__ H, double* __restrict__ cs, double2* __restrict__ sn,
                                 double2* __restrict__ g, double* __restrict__ sigma, KState* __restrict__ st) {
    if (st->done) return;
    extern __shared__ double2 fsm[];
    double2* col = fsm;                                   // j + 2
    double2* ssn = col + (j + 2);                         // j
    double* scs = reinterpret_cast<double*>(ssn + j);     // j
    const int lane = threadIdx.x;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += npart[b];
    s = warp_sum_d(s);
    const double beta = __shfl_sync(0xffffffffu, sqrt(s), 0);
    for (int i = lane; i <= j; i += 32) col[i] = cadd(h1[i], h2[i]);
    for (int i = lane; i < j; i += 32) { ssn[i] = sn[i]; scs[i] = cs[i]; }
    if (lane == 0) col[j + 1] = make_double2(beta, 0.0);
    __syncwarp();
    const int ldh = maxit + 1;
    if (lane == 0) {
        // previous rotations
        double2 a = col[0];
        for (int i = 0; i < j; ++i) {
            const double c = scs[i];
            const double2 sv = ssn[i];
            const double2 b = col[i + 1];
            // t = c a + s b ; b' = -conj(s) a + c b
            double2 t = cscale(a, c);
            t = cfma(sv, b, t);
            double2 nb = cscale(b, c);
            const double2 csn = make_double2(sv.x, -sv.y);
            nb = cfms(csn, a, nb);
            col[i] = t;
            a = nb;
        }
        // new rotation zeroing the subdiagonal entry
        const double2 b = col[j + 1];
        const double aa = hypot(a.x, a.y), bb = hypot(b.x, b.y);
        double c; double2 sv;
        if (bb == 0.0) { c = 1.0; sv = make_double2(0.0, 0.0); }
        else if (aa == 0.0) { c = 0.0; sv = make_double2(b.x / bb, -b.y / bb); }
        else {
            const double rho = hypot(aa, bb);
            c = aa / rho;
            const double2 ph = make_double2(a.x / aa, a.y / aa);          // a / |a|
            const double2 cb = make_double2(b.x / rho, -b.y / rho);       // conj(b) / rho
            sv = cmul(ph, cb);
        }
        cs[j] = c; sn[j] = sv;
        col[j] = cfma(sv, b, cscale(a, c));
        col[j + 1] = make_double2(0.0, 0.0);
        const double2 gj = g[j];
        const double2 csn = make_double2(sv.x, -sv.y);
        const double2 gn = cscale(cmul(csn, gj), -1.0);
        g[j + 1] = gn;
        g[j] = cscale(gj, c);
        const double resid = hypot(gn.x, gn.y);
        st->resid = resid;
        st->hnext = beta;
        st->iters = j + 1;
        sigma[j + 1] = beta > 0.0 ? 1.0 / beta : 0.0;
        if (!isfinite(resid) || !isfinite(beta)) { st->nonfinite = 1; st->done = 1; }
        else if (resid <= st->tolabs) { st->conv = 1; st->done = 1; }
        else if (beta == 0.0) { st->breakdown = 1; st->conv = 1; st->done = 1; }
        else if (j + 1 >= maxit) st->done = 1;
    }
    __syncwarp();
    double2* out = H + (size_t)j * ldh;
    for (int i = lane; i <= j + 1; i += 32) out[i] = col[i];
}

// ||f||: V_0 holds f; sets sigma[0], g[0], tolerance and flags.
__global__ void __launch_bounds__(kRedThreads) k_norm_part(long long N, const double2* __restrict__ x,
                                                           double* __restrict__ npart) {
    __shared__ double nred[kRedThreads / 32];
    long long e0, e1;
    chunk_of(N, e0, e1);
    double nrm = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const double2 v = x[e];
        nrm = fma(v.x, v.x, fma(v.y, v.y, nrm));
    }
    nrm = warp_sum_d(nrm);
    if ((threadIdx.x & 31) == 0) nred[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += nred[k];
        npart[blockIdx.x] = s;
    }
}

__global__ void k_init_state(int nblk, double tol, const double* __restrict__ npart, double* __restrict__ sigma,
                             double2* __restrict__ g, KState* __restrict__ st) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += npart[b];
    const double beta = sqrt(s);
    st->beta0 = beta;
    st->tolabs = tol * beta;
    st->resid = beta;
    st->hnext = 0.0;
    st->conv = 0; st->iters = 0; st->nonfinite = 0; st->breakdown = 0;
    st->done = 0;
    g[0] = make_double2(beta, 0.0);
    sigma[0] = beta > 0.0 ? 1.0 / beta : 0.0;
    if (!isfinite(beta)) { st->nonfinite = 1; st->done = 1; }
    else if (beta == 0.0) { st->conv = 1; st->done = 1; }
}

// y = R^{-1} g (m x m upper triangular in H after the rotations), column oriented.
__global__ void k_lsq_solve(int maxit, const double2* __restrict__ H, double2* __restrict__ g,
                            double2* __restrict__ y, const KState* __restrict__ st) {
    const int m = st->iters;
    const int ldh = maxit + 1;
    __shared__ double2 yi;
    for (int i = m - 1; i >= 0; --i) {
        if (threadIdx.x == 0) {
            const double2 d = H[(size_t)i * ldh + i];
            const double den = d.x * d.x + d.y * d.y;
            const double2 inv = den > 0.0 ? make_double2(d.x / den, -d.y / den) : make_double2(0.0, 0.0);
            yi = cmul(g[i], inv);
            y[i] = yi;
        }
        __syncthreads();
        const double2 v = yi;
        for (int r = threadIdx.x; r < i; r += blockDim.x) g[r] = cfms(H[(size_t)i * ldh + r], v, g[r]);
        __syncthreads();
    }
}

// x[e] = sum_{i < m} y_i sigma_i V_i[e]
__global__ void k_combine_basis(long long N, long long ld, int maxit, const double2* __restrict__ V,
                                const double* __restrict__ sigma, const double2* __restrict__ y,
                                double2* __restrict__ x, const KState* __restrict__ st) {
    extern __shared__ double2 coef[];
    const int m = st->iters;
    for (int i = threadIdx.x; i < m; i += blockDim.x) coef[i] = cscale(y[i], sigma[i]);
    __syncthreads();
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int i = 0; i < m; ++i) acc = cfma(coef[i], V[(size_t)i * ld + e], acc);
        x[e] = acc;
    }
}

// x[e] = sum_{i < m} y_i Z_i[e]
template <typename CZ>
__global__ void k_combine_Z(long long N, long long ldz, const CZ* __restrict__ Z, const double2* __restrict__ y,
                            double2* __restrict__ x, const KState* __restrict__ st) {
    extern __shared__ double2 coef[];
    const int m = st->iters;
    for (int i = threadIdx.x; i < m; i += blockDim.x) coef[i] = y[i];
    __syncthreads();
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int i = 0; i < m; ++i) acc = cfma(coef[i], to_d(Z[(size_t)i * ldz + e]), acc);
        x[e] = acc;
    }
}

// out[0] = ||f - Ax|| (two kernels: parts then a one-thread finish)
__global__ void __launch_bounds__(kRedThreads) k_resid_part(long long N, const double2* __restrict__ f,
                                                            const double2* __restrict__ ax,
                                                            double* __restrict__ npart) {
    __shared__ double nred[kRedThreads / 32];
    long long e0, e1;
    chunk_of(N, e0, e1);
    double nrm = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const double2 a = f[e], b = ax[e];
        const double rx = a.x - b.x, ry = a.y - b.y;
        nrm = fma(rx, rx, fma(ry, ry, nrm));
    }
    nrm = warp_sum_d(nrm);
    if ((threadIdx.x & 31) == 0) nred[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += nred[k];
        npart[blockIdx.x] = s;
    }
}
__global__ void k_sum_sqrt(int nblk, const double* __restrict__ npart, double* __restrict__ out) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += npart[b];
    out[0] = sqrt(s);
}

// ------------------------------------------------------------------ launchers
static size_t coef_smem(int count) { return (size_t)(count > 0 ? count : 1) * sizeof(double2); }

static size_t finish_smem(int j) {
    const size_t b = (size_t)(j + 2) * sizeof(double2) + (size_t)j * (sizeof(double2) + sizeof(double));
    if (b > 48 * 1024) cudaFuncSetAttribute(k_arnoldi_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b);
    return b;
}

static void set_coef_smem_limit(const void* fn, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void launch_norm_init(const Ctx& cx, const KrylovBufs& kb, double tol) {
    k_norm_part<<<kb.nblk, kRedThreads, 0, cx.stream>>>(kb.N, kb.V, kb.npart);
    k_init_state<<<1, 32, 0, cx.stream>>>(kb.nblk, tol, kb.npart, kb.sigma, kb.g, kb.st);
}

// After the preconditioner and the matrix-vector product have written
// w = A z_j into V_{j+1}: CGS2 against V_0..V_j, then the Givens update.
void launch_arnoldi_step(const Ctx& cx, const KrylovBufs& kb, int j) {
    const int stride = kb.maxit + 1;
    double2* w = kb.V + (size_t)(j + 1) * kb.ld;
    const int rblocks = ((j + 1) * 32 + 255) / 256;
    const size_t cs = coef_smem(j + 1);
    set_coef_smem_limit((const void*)k_axpy_multi, cs);
    // pass 1: h1 = V^H w ; w -= V h1
    k_multidot<double2, kDotGroup64><<<kb.nblk, kRedThreads, 0, cx.stream>>>(j, kb.N, kb.ld, stride, kb.V, w, kb.part, kb.st);
    k_reduce_dots<<<rblocks, 256, 0, cx.stream>>>(j, kb.nblk, stride, kb.part, kb.sigma, kb.h1, kb.st);
    k_axpy_multi<<<kb.nblk, kRedThreads, cs, cx.stream>>>(j, kb.N, kb.ld, kb.V, kb.sigma, kb.h1, w, nullptr, kb.st);
    // pass 2 (reorthogonalisation): h2 = V^H w ; w -= V h2 ; ||w||
    k_multidot<double2, kDotGroup64><<<kb.nblk, kRedThreads, 0, cx.stream>>>(j, kb.N, kb.ld, stride, kb.V, w, kb.part, kb.st);
    k_reduce_dots<<<rblocks, 256, 0, cx.stream>>>(j, kb.nblk, stride, kb.part, kb.sigma, kb.h2, kb.st);
    k_axpy_multi<<<kb.nblk, kRedThreads, cs, cx.stream>>>(j, kb.N, kb.ld, kb.V, kb.sigma, kb.h2, w, kb.npart, kb.st);
    k_arnoldi_finish<<<1, 32, finish_smem(j), cx.stream>>>(j, kb.maxit, kb.nblk, kb.npart, kb.h1, kb.h2, kb.H, kb.cs, kb.sn, kb.g,
                                              kb.sigma, kb.st);
}

// Mixed-precision CGS2 (used with the complex64 preconditioner): the first
// projection h1 = V^H w is computed in complex64 from complex64 copies of the
// basis and of w; the update w -= V h1, the reorthogonalisation h2 = V^H w and
// the Hessenberg column stay FP64; the second update w -= V h2 sums in
// complex64 (h2 is of the size of the first pass's rounding, so its complex64
// product is exact to FP64 level) and subtracts in FP64.  Orthogonality and the
// Arnoldi relation therefore hold to FP64 level, with half the FP64 work of
// the all-FP64 CGS2.  kb.V32 must hold complex64 copies of V_0 .. V_{j+1}
// (V_{j+1} = A z_j written by the matrix-vector product).
void launch_arnoldi_step_mixed(const Ctx& cx, const KrylovBufs& kb, int j) {
    const int stride = kb.maxit + 1;
    double2* w = kb.V + (size_t)(j + 1) * kb.ld;
    float2* w32 = kb.V32 + (size_t)(j + 1) * kb.ld;
    const int rblocks = ((j + 1) * 32 + 255) / 256;
    const size_t cs = coef_smem(j + 1);
    set_coef_smem_limit((const void*)k_axpy_multi, cs);
    k_multidot<float2, kDotGroup32><<<kb.nblk, kRedThreads, 0, cx.stream>>>(j, kb.N, kb.ld, stride, kb.V32, w32, kb.part, kb.st);
    k_reduce_dots<<<rblocks, 256, 0, cx.stream>>>(j, kb.nblk, stride, kb.part, kb.sigma, kb.h1, kb.st);
    k_axpy_multi<<<kb.nblk, kRedThreads, cs, cx.stream>>>(j, kb.N, kb.ld, kb.V, kb.sigma, kb.h1, w, nullptr, kb.st);
    k_multidot<double2, kDotGroup64><<<kb.nblk, kRedThreads, 0, cx.stream>>>(j, kb.N, kb.ld, stride, kb.V, w, kb.part, kb.st);
    k_reduce_dots<<<rblocks, 256, 0, cx.stream>>>(j, kb.nblk, stride, kb.part, kb.sigma, kb.h2, kb.st);
    k_correct32<<<kb.nblk, kRedThreads, (size_t)(j + 1) * sizeof(float2), cx.stream>>>(
        j, kb.N, kb.ld, kb.V32, kb.sigma, kb.h2, w, w32, kb.npart, kb.st);
    k_arnoldi_finish<<<1, 32, finish_smem(j), cx.stream>>>(j, kb.maxit, kb.nblk, kb.npart, kb.h1, kb.h2, kb.H, kb.cs, kb.sn, kb.g,
                                              kb.sigma, kb.st);
}

void launch_lsq_solve(const Ctx& cx, const KrylovBufs& kb) {
    k_lsq_solve<<<1, 1024, 0, cx.stream>>>(kb.maxit, kb.H, kb.g, kb.y, kb.st);
}

void launch_combine_basis(const Ctx& cx, const KrylovBufs& kb, double2* x) {
    const size_t cs = coef_smem(kb.maxit);
    set_coef_smem_limit((const void*)k_combine_basis, cs);
    k_combine_basis<<<kb.nblk, 256, cs, cx.stream>>>(kb.N, kb.ld, kb.maxit, kb.V, kb.sigma, kb.y, x, kb.st);
}

void launch_combine_Z(const Ctx& cx, const KrylovBufs& kb, const float2* Z, long long ldz, double2* x) {
    const size_t cs = coef_smem(kb.maxit);
    set_coef_smem_limit((const void*)k_combine_Z<float2>, cs);
    k_combine_Z<float2><<<kb.nblk, 256, cs, cx.stream>>>(kb.N, ldz, Z, kb.y, x, kb.st);
}

void launch_combine_Z64(const Ctx& cx, const KrylovBufs& kb, const double2* Z, long long ldz, double2* x) {
    const size_t cs = coef_smem(kb.maxit);
    set_coef_smem_limit((const void*)k_combine_Z<double2>, cs);
    k_combine_Z<double2><<<kb.nblk, 256, cs, cx.stream>>>(kb.N, ldz, Z, kb.y, x, kb.st);
}

void launch_residual_norm(const Ctx& cx, const KrylovBufs& kb, const double2* f, const double2* Ax, double* out) {
    k_resid_part<<<kb.nblk, kRedThreads, 0, cx.stream>>>(kb.N, f, Ax, kb.npart);
    k_sum_sqrt<<<1, 32, 0, cx.stream>>>(kb.nblk, kb.npart, out);
}

}  // namespace hzs
