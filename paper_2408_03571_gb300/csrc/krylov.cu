// GMRES kernels (Section 5): Arnoldi with classical Gram-Schmidt and one
// reorthogonalisation (CGS2), Givens rotations on the Hessenberg matrix,
// the triangular solve and the solution update, all in FP64 complex.
//
// Basis vectors are stored unnormalised: the i-th orthonormal vector is
// sigma[i] * V_i.  The scale is folded into the dot products and the update
// coefficients, so no separate normalisation pass over the vector is needed.
//
// Every per-iteration kernel returns at once when the iteration has already
// finished (st->done), so the host may enqueue an iteration before it knows
// whether the previous one converged.
#include "kernels.cuh"

namespace hzs {

constexpr int kRedThreads = 256;
constexpr int kDotGroup = 4;

// Block-wide sum of G complex values per thread; result valid in thread 0's out[].
template <int G>
__device__ __forceinline__ void block_sum(double2 (&acc)[G], double2 (*red)[G], double2 (&out)[G]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = warp_sum(acc[g]);
    if (lane == 0) {
#pragma unroll
        for (int g = 0; g < G; ++g) red[wid][g] = acc[g];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
            double2 s = make_double2(0.0, 0.0);
            for (int w = 0; w < nw; ++w) s = cadd(s, red[w][g]);
            out[g] = s;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void chunk_of(long long N, long long& e0, long long& e1) {
    const long long per = (N + gridDim.x - 1) / gridDim.x;
    e0 = (long long)blockIdx.x * per;
    e1 = e0 + per < N ? e0 + per : N;
}

// part[b][i] = sum_{e in chunk b} conj(V_i[e]) w[e],  i = 0..j
__global__ void __launch_bounds__(kRedThreads) k_multidot(int j, long long N, long long ld, int stride,
                                                          const double2* __restrict__ V,
                                                          const double2* __restrict__ w, double2* __restrict__ part,
                                                          const KState* __restrict__ st) {
    if (st->done) return;
    __shared__ double2 red[kRedThreads / 32][kDotGroup];
    long long e0, e1;
    chunk_of(N, e0, e1);
    for (int i0 = 0; i0 <= j; i0 += kDotGroup) {
        double2 acc[kDotGroup];
#pragma unroll
        for (int g = 0; g < kDotGroup; ++g) acc[g] = make_double2(0.0, 0.0);
        for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const double2 we = w[e];
#pragma unroll
            for (int g = 0; g < kDotGroup; ++g)
                if (i0 + g <= j) acc[g] = cfma_conj(V[(size_t)(i0 + g) * ld + e], we, acc[g]);
        }
        double2 out[kDotGroup];
        block_sum<kDotGroup>(acc, red, out);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int g = 0; g < kDotGroup; ++g)
                if (i0 + g <= j) part[(size_t)blockIdx.x * stride + i0 + g] = out[g];
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

// w[e] -= sum_i (h[i] sigma[i]) V_i[e]; optionally npart[b] = sum_e |w[e]|^2
__global__ void __launch_bounds__(kRedThreads) k_axpy_multi(int j, long long N, long long ld,
                                                            const double2* __restrict__ V,
                                                            const double* __restrict__ sigma,
                                                            const double2* __restrict__ h, double2* __restrict__ w,
                                                            double* __restrict__ npart, const KState* __restrict__ st) {
    if (st->done) return;
    extern __shared__ double2 coef[];
    __shared__ double nred[kRedThreads / 32];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) coef[i] = cscale(h[i], sigma[i]);
    __syncthreads();
    long long e0, e1;
    chunk_of(N, e0, e1);
    double nrm = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        double2 we = w[e];
        for (int i = 0; i <= j; ++i) we = cfms(coef[i], V[(size_t)i * ld + e], we);
        w[e] = we;
        nrm = fma(we.x, we.x, fma(we.y, we.y, nrm));
    }
    if (npart) {
        nrm = warp_sum_d(nrm);
        if ((threadIdx.x & 31) == 0) nred[threadIdx.x >> 5] = nrm;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += nred[k];
            npart[blockIdx.x] = s;
        }
    }
}

// Completes step j: h_{j+1,j} = ||w||, column j of H = h1 + h2, Givens
// rotations, residual estimate, convergence / breakdown flags.
__global__ void k_arnoldi_finish(int j, int maxit, int nblk, const double* __restrict__ npart,
                                 const double2* __restrict__ h1, const double2* __restrict__ h2,
                                 double2* __restrict__ H, double* __restrict__ cs, double2* __restrict__ sn,
                                 double2* __restrict__ g, double* __restrict__ sigma, KState* __restrict__ st) {
    if (threadIdx.x != 0 || st->done) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += npart[b];
    const double beta = sqrt(s);
    const int ldh = maxit + 1;
    double2* col = H + (size_t)j * ldh;
    for (int i = 0; i <= j; ++i) col[i] = cadd(h1[i], h2[i]);
    col[j + 1] = make_double2(beta, 0.0);
    // previous rotations
    for (int i = 0; i < j; ++i) {
        const double c = cs[i];
        const double2 sv = sn[i];
        const double2 a = col[i], b = col[i + 1];
        // t = c a + s b ; b' = -conj(s) a + c b
        double2 t = cscale(a, c);
        t = cfma(sv, b, t);
        double2 nb = cscale(b, c);
        const double2 csn = make_double2(sv.x, -sv.y);
        nb = cfms(csn, a, nb);
        col[i] = t; col[i + 1] = nb;
    }
    // new rotation zeroing col[j+1]
    const double2 a = col[j], b = col[j + 1];
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
    g[j + 1] = cscale(cmul(csn, gj), -1.0);
    g[j] = cscale(gj, c);
    const double resid = hypot(g[j + 1].x, g[j + 1].y);
    st->resid = resid;
    st->hnext = beta;
    st->iters = j + 1;
    sigma[j + 1] = beta > 0.0 ? 1.0 / beta : 0.0;
    if (!isfinite(resid) || !isfinite(beta)) { st->nonfinite = 1; st->done = 1; return; }
    if (resid <= st->tolabs) { st->conv = 1; st->done = 1; return; }
    if (beta == 0.0) { st->breakdown = 1; st->conv = 1; st->done = 1; return; }
    if (j + 1 >= maxit) st->done = 1;
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
    k_multidot<<<kb.nblk, kRedThreads, 0, cx.stream>>>(j, kb.N, kb.ld, stride, kb.V, w, kb.part, kb.st);
    k_reduce_dots<<<rblocks, 256, 0, cx.stream>>>(j, kb.nblk, stride, kb.part, kb.sigma, kb.h1, kb.st);
    k_axpy_multi<<<kb.nblk, kRedThreads, cs, cx.stream>>>(j, kb.N, kb.ld, kb.V, kb.sigma, kb.h1, w, nullptr, kb.st);
    // pass 2 (reorthogonalisation): h2 = V^H w ; w -= V h2 ; ||w||
    k_multidot<<<kb.nblk, kRedThreads, 0, cx.stream>>>(j, kb.N, kb.ld, stride, kb.V, w, kb.part, kb.st);
    k_reduce_dots<<<rblocks, 256, 0, cx.stream>>>(j, kb.nblk, stride, kb.part, kb.sigma, kb.h2, kb.st);
    k_axpy_multi<<<kb.nblk, kRedThreads, cs, cx.stream>>>(j, kb.N, kb.ld, kb.V, kb.sigma, kb.h2, w, kb.npart, kb.st);
    k_arnoldi_finish<<<1, 32, 0, cx.stream>>>(j, kb.maxit, kb.nblk, kb.npart, kb.h1, kb.h2, kb.H, kb.cs, kb.sn, kb.g,
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
