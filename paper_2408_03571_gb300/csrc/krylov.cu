// GMRES kernels (Section 5): Arnoldi with classical Gram-Schmidt and one
// reorthogonalisation (CGS2), Givens rotations on the Hessenberg matrix,
// the triangular solve and the solution update.
//
// Basis vectors are stored unnormalised: the i-th orthonormal vector is
// sigma[i] * V_i.  The scale is folded into the dot products and the update
// coefficients, so no separate normalisation pass over the vector is needed.
//
// All kernels work on a batch of right-hand sides (batch entry r =
// blockIdx.y, or blockIdx.x for the one-block-per-entry kernels); entry r's
// arrays start at r times the per-entry strides of KrylovBufs.  Every
// per-iteration kernel returns at once when its entry has already finished
// (st[r].done), so the host may enqueue an iteration before it knows whether
// the previous one converged, and converged entries of a batch cost nothing.
//
// Reductions are deterministic: fixed chunks per block, fixed lane order in
// the warp trees, and the cross-block sums in a fixed order.
#include "kernels.cuh"

namespace hzs {

constexpr int kRedThreads = 256;
constexpr int kDotGroup64 = 4;     // basis vectors per warp pass (FP64 multi-dot)
constexpr int kDotGroup32 = 8;     // basis vectors per warp pass (complex64 multi-dot)
constexpr int kDotGroupDF = 4;     // basis vectors per warp pass (double-float multi-dot)

__device__ __forceinline__ void chunk_of(long long N, long long& e0, long long& e1) {
    const long long per = (N + gridDim.x - 1) / gridDim.x;
    e0 = (long long)blockIdx.x * per;
    e1 = e0 + per < N ? e0 + per : N;
}

// part[b][i] = sum_{e in chunk b} conj(V_i[e]) w[e], i = 0..j, with products and
// sums in the precision of C (w = V + wofs).  Each warp takes groups of G basis
// vectors and sweeps the whole chunk of its block for them (w is re-read from
// L1), so no block-wide barrier is needed; lane 0 writes the group's partials.
template <typename C, int G>
__global__ void __launch_bounds__(kRedThreads) k_multidot(int j, long long N, long long ld, int stride,
                                                          const C* __restrict__ V, long long sV,
                                                          long long wofs, double2* __restrict__ part,
                                                          long long sP, const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (st[r].done) return;
    V += r * sV;
    const C* w = V + wofs;
    part += r * sP;
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
__global__ void k_reduce_dots(int j, int nblk, int stride, const double2* __restrict__ part, long long sP,
                              const double* __restrict__ sigma, double2* __restrict__ h, long long sS,
                              const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (st[r].done) return;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i > j) return;
    part += r * sP; sigma += r * sS; h += r * sS;
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

// w[e] -= sum_i (h[i] sigma[i]) V_i[e] in FP64 (w = V + wofs); optionally
// npart[b] = sum_e |w[e]|^2.  Four independent partial sums per element keep
// several loads in flight.
__global__ void __launch_bounds__(kRedThreads) k_axpy_multi(int j, long long N, long long ld,
                                                            double2* __restrict__ V, long long sV,
                                                            const double* __restrict__ sigma,
                                                            const double2* __restrict__ h, long long sS,
                                                            long long wofs, double* __restrict__ npart,
                                                            int nblk, const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (st[r].done) return;
    V += r * sV; sigma += r * sS; h += r * sS;
    double2* w = V + wofs;
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
    if (npart) block_norm_part(nrm, npart + (size_t)r * nblk);
}

// ---- double-float passes of the mixed-precision CGS2 (see launch_arnoldi_step_mixed)
// The basis is held as double-float pairs V32 + V32lo (complex64 rounding and
// remainder), w = V32[j+1] + V32lo[j+1].

// w -= sum_i c_i v_i with c_i = h[i] sigma[i], all in double-float arithmetic
// (two interleaved accumulators per component); also writes nothing else.
__global__ void __launch_bounds__(kRedThreads) k_axpy_df(int j, long long N, long long ld,
                                                         float2* __restrict__ V32, float2* __restrict__ V32lo,
                                                         long long sV, const double* __restrict__ sigma,
                                                         const double2* __restrict__ h, long long sS, long long wofs,
                                                         const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (st[r].done) return;
    V32 += r * sV; V32lo += r * sV; sigma += r * sS; h += r * sS;
    float2* wh = V32 + wofs;
    float2* wl = V32lo + wofs;
    extern __shared__ float4 coefdf[];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const double2 c = cscale(h[i], sigma[i]);
        float4 q;
        split_d(c.x, q.x, q.y);
        split_d(c.y, q.z, q.w);
        coefdf[i] = q;
    }
    __syncthreads();
    long long e0, e1;
    chunk_of(N, e0, e1);
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;      // real part, two accumulators
        float ch = 0.f, cl = 0.f, dh = 0.f, dl = 0.f;      // imaginary part
        int i = 0;
        for (; i + 1 <= j; i += 2) {
            {
                const float4 q = coefdf[i];
                const float2 vh = V32[(size_t)i * ld + e], vl = V32lo[(size_t)i * ld + e];
                df_fma(ah, al, q.x, q.y, vh.x, vl.x);
                df_fma(ah, al, -q.z, -q.w, vh.y, vl.y);
                df_fma(ch, cl, q.x, q.y, vh.y, vl.y);
                df_fma(ch, cl, q.z, q.w, vh.x, vl.x);
            }
            {
                const float4 q = coefdf[i + 1];
                const float2 vh = V32[(size_t)(i + 1) * ld + e], vl = V32lo[(size_t)(i + 1) * ld + e];
                df_fma(bh, bl, q.x, q.y, vh.x, vl.x);
                df_fma(bh, bl, -q.z, -q.w, vh.y, vl.y);
                df_fma(dh, dl, q.x, q.y, vh.y, vl.y);
                df_fma(dh, dl, q.z, q.w, vh.x, vl.x);
            }
            if ((i & 15) == 14) { df_norm(ah, al); df_norm(bh, bl); df_norm(ch, cl); df_norm(dh, dl); }
        }
        for (; i <= j; ++i) {
            const float4 q = coefdf[i];
            const float2 vh = V32[(size_t)i * ld + e], vl = V32lo[(size_t)i * ld + e];
            df_fma(ah, al, q.x, q.y, vh.x, vl.x);
            df_fma(ah, al, -q.z, -q.w, vh.y, vl.y);
            df_fma(ch, cl, q.x, q.y, vh.y, vl.y);
            df_fma(ch, cl, q.z, q.w, vh.x, vl.x);
        }
        df_add(ah, al, bh, bl);
        df_add(ch, cl, dh, dl);
        // w - s
        float2 xh = wh[e], xl = wl[e];
        df_add(xh.x, xl.x, -ah, -al);
        df_add(xh.y, xl.y, -ch, -cl);
        df_norm(xh.x, xl.x);
        df_norm(xh.y, xl.y);
        wh[e] = xh;
        wl[e] = xl;
    }
}

// part[b][i] = sum_{e in chunk b} conj(v_i[e]) w[e] in double-float arithmetic,
// warp-parallel over groups of G basis vectors as k_multidot.
template <int G>
__global__ void __launch_bounds__(kRedThreads) k_multidot_df(int j, long long N, long long ld, int stride,
                                                             const float2* __restrict__ V32,
                                                             const float2* __restrict__ V32lo, long long sV,
                                                             long long wofs, double2* __restrict__ part, long long sP,
                                                             const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (st[r].done) return;
    V32 += r * sV; V32lo += r * sV;
    const float2* wh = V32 + wofs;
    const float2* wl = V32lo + wofs;
    part += r * sP;
    long long e0, e1;
    chunk_of(N, e0, e1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ngroups = (j + G) / G;
    for (int gi = warp; gi < ngroups; gi += nw) {
        const int i0 = gi * G;
        float rh[G], rl[G], ih[G], il[G];
#pragma unroll
        for (int t = 0; t < G; ++t) { rh[t] = rl[t] = ih[t] = il[t] = 0.f; }
        int cnt = 0;
        for (long long e = e0 + lane; e < e1; e += 32) {
            const float2 xh = wh[e], xl = wl[e];
#pragma unroll
            for (int t = 0; t < G; ++t) {
                if (i0 + t > j) continue;
                const float2 vh = V32[(size_t)(i0 + t) * ld + e], vl = V32lo[(size_t)(i0 + t) * ld + e];
                // conj(v) w: re = vr wr + vi wi, im = vr wi - vi wr
                df_fma(rh[t], rl[t], vh.x, vl.x, xh.x, xl.x);
                df_fma(rh[t], rl[t], vh.y, vl.y, xh.y, xl.y);
                df_fma(ih[t], il[t], vh.x, vl.x, xh.y, xl.y);
                df_fma(ih[t], il[t], -vh.y, -vl.y, xh.x, xl.x);
            }
            if ((++cnt & 15) == 0) {
#pragma unroll
                for (int t = 0; t < G; ++t) { df_norm(rh[t], rl[t]); df_norm(ih[t], il[t]); }
            }
        }
#pragma unroll
        for (int t = 0; t < G; ++t) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float orh = __shfl_down_sync(0xffffffffu, rh[t], o);
                const float orl = __shfl_down_sync(0xffffffffu, rl[t], o);
                const float oih = __shfl_down_sync(0xffffffffu, ih[t], o);
                const float oil = __shfl_down_sync(0xffffffffu, il[t], o);
                df_add(rh[t], rl[t], orh, orl);
                df_add(ih[t], il[t], oih, oil);
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (i0 + t <= j)
                    part[(size_t)blockIdx.x * stride + i0 + t] =
                        make_double2((double)rh[t] + (double)rl[t], (double)ih[t] + (double)il[t]);
        }
    }
}

// w -= sum_i (h[i] sigma[i]) V32_i, the sum in complex64 (h is the small
// reorthogonalisation coefficient, so a single-precision sum is accurate to
// the working precision relative to w) and the subtraction in double-float;
// npart[b] = sum_e |w[e]|^2.
__global__ void __launch_bounds__(kRedThreads) k_correct_df(int j, long long N, long long ld,
                                                            float2* __restrict__ V32, float2* __restrict__ V32lo,
                                                            long long sV, const double* __restrict__ sigma,
                                                            const double2* __restrict__ h, long long sS,
                                                            long long wofs, double* __restrict__ npart, int nblk,
                                                            const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (st[r].done) return;
    V32 += r * sV; V32lo += r * sV; sigma += r * sS; h += r * sS;
    float2* wh = V32 + wofs;
    float2* wl = V32lo + wofs;
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
        float2 xh = wh[e], xl = wl[e];
        df_add(xh.x, xl.x, -((c0.x + c1.x) + (c2.x + c3.x)), 0.f);
        df_add(xh.y, xl.y, -((c0.y + c1.y) + (c2.y + c3.y)), 0.f);
        df_norm(xh.x, xl.x);
        df_norm(xh.y, xl.y);
        wh[e] = xh;
        wl[e] = xl;
        const double vx = (double)xh.x + (double)xl.x, vy = (double)xh.y + (double)xl.y;
        nrm = fma(vx, vx, fma(vy, vy, nrm));
    }
    block_norm_part(nrm, npart + (size_t)r * nblk);
}

// Completes step j of entry r = blockIdx.x: h_{j+1,j} = ||w||, column j of
// H = h1 + h2, Givens rotations, residual estimate, convergence / breakdown
// flags.  One warp per entry: the block norm partials are summed in a fixed
// lane order, the column and the rotations are staged in shared memory, and
// lane 0 applies the rotation chain.  An entry that finishes decrements the
// batch's active counter.
__global__ void k_arnoldi_finish(int j, int maxit, int nblk, const double* __restrict__ npart,
                                 const double2* __restrict__ h1, const double2* __restrict__ h2,
                                 double2* __restrict__ H, long long sH, double* __restrict__ cs,
                                 double2* __restrict__ sn, double2* __restrict__ g, double* __restrict__ sigma,
                                 long long sS, KState* __restrict__ st, int* __restrict__ active) {
    const int r = blockIdx.x;
    if (st[r].done) return;
    npart += (size_t)r * nblk;
    h1 += r * sS; h2 += r * sS; H += r * sH; cs += r * sS; sn += r * sS; g += r * sS; sigma += r * sS;
    KState* s0 = st + r;
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
        s0->resid = resid;
        s0->hnext = beta;
        s0->iters = j + 1;
        sigma[j + 1] = beta > 0.0 ? 1.0 / beta : 0.0;
        int fin = 1;
        if (!isfinite(resid) || !isfinite(beta)) s0->nonfinite = 1;
        else if (resid <= s0->tolabs) s0->conv = 1;
        else if (beta == 0.0) { s0->breakdown = 1; s0->conv = 1; }
        else if (!(j + 1 >= maxit)) fin = 0;
        if (fin) { s0->done = 1; atomicSub(active, 1); }
    }
    __syncwarp();
    double2* out = H + (size_t)j * ldh;
    for (int i = lane; i <= j + 1; i += 32) out[i] = col[i];
}

// ||f||: V_0 holds f; sets sigma[0], g[0], tolerance and flags.
__global__ void __launch_bounds__(kRedThreads) k_norm_part(long long N, const double2* __restrict__ x, long long xs,
                                                           double* __restrict__ npart, int nblk) {
    const int r = blockIdx.y;
    x += r * xs;
    long long e0, e1;
    chunk_of(N, e0, e1);
    double nrm = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const double2 v = x[e];
        nrm = fma(v.x, v.x, fma(v.y, v.y, nrm));
    }
    block_norm_part(nrm, npart + (size_t)r * nblk);
}

// One block; thread r initialises entry r; active = entries still running.
__global__ void k_init_state(int nb, int nblk, double tol, const double* __restrict__ npart,
                             double* __restrict__ sigma, double2* __restrict__ g, long long sS,
                             KState* __restrict__ st, int* __restrict__ active) {
    __shared__ int run;
    if (threadIdx.x == 0) run = 0;
    __syncthreads();
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += npart[(size_t)r * nblk + b];
        const double beta = sqrt(s);
        KState* s0 = st + r;
        s0->beta0 = beta;
        s0->tolabs = tol * beta;
        s0->resid = beta;
        s0->hnext = 0.0;
        s0->conv = 0; s0->iters = 0; s0->nonfinite = 0; s0->breakdown = 0;
        s0->done = 0;
        g[r * sS] = make_double2(beta, 0.0);
        sigma[r * sS] = beta > 0.0 ? 1.0 / beta : 0.0;
        if (!isfinite(beta)) { s0->nonfinite = 1; s0->done = 1; }
        else if (beta == 0.0) { s0->conv = 1; s0->done = 1; }
        else atomicAdd(&run, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *active = run;
}

// y = R^{-1} g (m x m upper triangular in H after the rotations), column oriented; one block per entry.
__global__ void k_lsq_solve(int maxit, const double2* __restrict__ H, long long sH, double2* __restrict__ g,
                            double2* __restrict__ y, long long sS, const KState* __restrict__ st) {
    const int r = blockIdx.x;
    H += r * sH; g += r * sS; y += r * sS;
    const int m = st[r].iters;
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
        for (int rr = threadIdx.x; rr < i; rr += blockDim.x) g[rr] = cfms(H[(size_t)i * ldh + rr], v, g[rr]);
        __syncthreads();
    }
}

// x[e] = sum_{i < m} y_i sigma_i V_i[e]
__global__ void k_combine_basis(long long N, long long ld, const double2* __restrict__ V, long long sV,
                                const double* __restrict__ sigma, const double2* __restrict__ y, long long sS,
                                double2* __restrict__ x, long long xs, const KState* __restrict__ st) {
    const int r = blockIdx.y;
    V += r * sV; sigma += r * sS; y += r * sS; x += r * xs;
    extern __shared__ double2 coef[];
    const int m = st[r].iters;
    for (int i = threadIdx.x; i < m; i += blockDim.x) coef[i] = cscale(y[i], sigma[i]);
    __syncthreads();
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int i = 0; i < m; ++i) acc = cfma(coef[i], V[(size_t)i * ld + e], acc);
        x[e] = acc;
    }
}

// x[e] = sum_{i < m} y_i Z_i[e]
__global__ void k_combine_Z(long long N, long long ldz, const float2* __restrict__ Z, long long zs,
                            const double2* __restrict__ y, long long sS, double2* __restrict__ x, long long xs,
                            const KState* __restrict__ st) {
    const int r = blockIdx.y;
    Z += r * zs; y += r * sS; x += r * xs;
    extern __shared__ double2 coef[];
    const int m = st[r].iters;
    for (int i = threadIdx.x; i < m; i += blockDim.x) coef[i] = y[i];
    __syncthreads();
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int i = 0; i < m; ++i) acc = cfma(coef[i], to_d(Z[(size_t)i * ldz + e]), acc);
        x[e] = acc;
    }
}

// out[r] = ||f_r - Ax_r|| (parts, then one thread per entry)
__global__ void __launch_bounds__(kRedThreads) k_resid_part(long long N, const double2* __restrict__ f, long long fs,
                                                            const double2* __restrict__ ax, long long axs,
                                                            double* __restrict__ npart, int nblk) {
    const int r = blockIdx.y;
    f += r * fs; ax += r * axs;
    long long e0, e1;
    chunk_of(N, e0, e1);
    double nrm = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const double2 a = f[e], b = ax[e];
        const double rx = a.x - b.x, ry = a.y - b.y;
        nrm = fma(rx, rx, fma(ry, ry, nrm));
    }
    block_norm_part(nrm, npart + (size_t)r * nblk);
}
__global__ void k_sum_sqrt(int nb, int nblk, const double* __restrict__ npart, double* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nb) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += npart[(size_t)r * nblk + b];
    out[r] = sqrt(s);
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

void launch_norm_init(const Ctx& cx, const KrylovBufs& kb, int nb, double tol) {
    k_norm_part<<<dim3(kb.nblk, nb), kRedThreads, 0, cx.stream>>>(kb.N, kb.V, kb.sV(), kb.npart, kb.nblk);
    k_init_state<<<1, 256, 0, cx.stream>>>(nb, kb.nblk, tol, kb.npart, kb.sigma, kb.g, kb.sS(), kb.st, kb.active);
}

// After the preconditioner and the matrix-vector product have written
// w = A z_j into V_{j+1} of every entry: CGS2 against V_0..V_j, then the Givens update.
void launch_arnoldi_step(const Ctx& cx, const KrylovBufs& kb, int nb, int j) {
    const int stride = kb.maxit + 1;
    const long long wofs = (long long)(j + 1) * kb.ld;
    const dim3 gr(kb.nblk, nb);
    const dim3 rg(((j + 1) * 32 + 255) / 256, nb);
    const size_t cs = coef_smem(j + 1);
    set_coef_smem_limit((const void*)k_axpy_multi, cs);
    // pass 1: h1 = V^H w ; w -= V h1
    k_multidot<double2, kDotGroup64><<<gr, kRedThreads, 0, cx.stream>>>(j, kb.N, kb.ld, stride, kb.V, kb.sV(), wofs,
                                                                        kb.part, kb.sP(), kb.st);
    k_reduce_dots<<<rg, 256, 0, cx.stream>>>(j, kb.nblk, stride, kb.part, kb.sP(), kb.sigma, kb.h1, kb.sS(), kb.st);
    k_axpy_multi<<<gr, kRedThreads, cs, cx.stream>>>(j, kb.N, kb.ld, kb.V, kb.sV(), kb.sigma, kb.h1, kb.sS(), wofs,
                                                     nullptr, kb.nblk, kb.st);
    // pass 2 (reorthogonalisation): h2 = V^H w ; w -= V h2 ; ||w||
    k_multidot<double2, kDotGroup64><<<gr, kRedThreads, 0, cx.stream>>>(j, kb.N, kb.ld, stride, kb.V, kb.sV(), wofs,
                                                                        kb.part, kb.sP(), kb.st);
    k_reduce_dots<<<rg, 256, 0, cx.stream>>>(j, kb.nblk, stride, kb.part, kb.sP(), kb.sigma, kb.h2, kb.sS(), kb.st);
    k_axpy_multi<<<gr, kRedThreads, cs, cx.stream>>>(j, kb.N, kb.ld, kb.V, kb.sV(), kb.sigma, kb.h2, kb.sS(), wofs,
                                                     kb.npart, kb.nblk, kb.st);
    k_arnoldi_finish<<<nb, 32, finish_smem(j), cx.stream>>>(j, kb.maxit, kb.nblk, kb.npart, kb.h1, kb.h2, kb.H,
                                                            kb.sH(), kb.cs, kb.sn, kb.g, kb.sigma, kb.sS(), kb.st,
                                                            kb.active);
}

// Mixed-precision CGS2 (used with the complex64 preconditioner).  The basis
// is held as double-float pairs V32 + V32lo (complex64 rounding and remainder,
// about 48 significand bits), written by the matrix-vector product and the
// last pass.  The first projection h1 = V^H w is computed in complex64 from
// V32 alone; the update w -= V h1 and the reorthogonalisation h2 = V^H w run
// in double-float arithmetic (error-free FMA products and TwoSum accumulation
// on the FP32 pipes); the second update w -= V h2 sums in complex64 (h2 is of
// the size of the first pass's rounding) and subtracts in double-float.  The
// FP64 Hessenberg column, norms and Givens update are unchanged.
// Orthogonality and the Arnoldi relation hold to about 1e-12 relative (the
// double-float accumulation), far below any GMRES tolerance used here, while
// no basis pass executes an FP64 instruction per basis entry.
void launch_arnoldi_step_mixed(const Ctx& cx, const KrylovBufs& kb, int nb, int j) {
    const int stride = kb.maxit + 1;
    const long long wofs = (long long)(j + 1) * kb.ld;
    const dim3 gr(kb.nblk, nb);
    const dim3 rg(((j + 1) * 32 + 255) / 256, nb);
    const size_t cdf = (size_t)(j + 1) * sizeof(float4);
    set_coef_smem_limit((const void*)k_axpy_df, cdf);
    k_multidot<float2, kDotGroup32><<<gr, kRedThreads, 0, cx.stream>>>(j, kb.N, kb.ld, stride, kb.V32, kb.sV(), wofs,
                                                                       kb.part, kb.sP(), kb.st);
    k_reduce_dots<<<rg, 256, 0, cx.stream>>>(j, kb.nblk, stride, kb.part, kb.sP(), kb.sigma, kb.h1, kb.sS(), kb.st);
    k_axpy_df<<<gr, kRedThreads, cdf, cx.stream>>>(j, kb.N, kb.ld, kb.V32, kb.V32lo, kb.sV(), kb.sigma, kb.h1,
                                                   kb.sS(), wofs, kb.st);
    k_multidot_df<kDotGroupDF><<<gr, kRedThreads, 0, cx.stream>>>(j, kb.N, kb.ld, stride, kb.V32, kb.V32lo, kb.sV(),
                                                                  wofs, kb.part, kb.sP(), kb.st);
    k_reduce_dots<<<rg, 256, 0, cx.stream>>>(j, kb.nblk, stride, kb.part, kb.sP(), kb.sigma, kb.h2, kb.sS(), kb.st);
    k_correct_df<<<gr, kRedThreads, (size_t)(j + 1) * sizeof(float2), cx.stream>>>(
        j, kb.N, kb.ld, kb.V32, kb.V32lo, kb.sV(), kb.sigma, kb.h2, kb.sS(), wofs, kb.npart, kb.nblk, kb.st);
    k_arnoldi_finish<<<nb, 32, finish_smem(j), cx.stream>>>(j, kb.maxit, kb.nblk, kb.npart, kb.h1, kb.h2, kb.H,
                                                            kb.sH(), kb.cs, kb.sn, kb.g, kb.sigma, kb.sS(), kb.st,
                                                            kb.active);
}

void launch_lsq_solve(const Ctx& cx, const KrylovBufs& kb, int nb) {
    k_lsq_solve<<<nb, 1024, 0, cx.stream>>>(kb.maxit, kb.H, kb.sH(), kb.g, kb.y, kb.sS(), kb.st);
}

void launch_combine_basis(const Ctx& cx, const KrylovBufs& kb, int nb, double2* x, long long xs) {
    const size_t cs = coef_smem(kb.maxit);
    set_coef_smem_limit((const void*)k_combine_basis, cs);
    k_combine_basis<<<dim3(kb.nblk, nb), 256, cs, cx.stream>>>(kb.N, kb.ld, kb.V, kb.sV(), kb.sigma, kb.y, kb.sS(), x,
                                                               xs, kb.st);
}

void launch_combine_Z(const Ctx& cx, const KrylovBufs& kb, int nb, const float2* Z, long long ldz, long long zs,
                      double2* x, long long xs) {
    const size_t cs = coef_smem(kb.maxit);
    set_coef_smem_limit((const void*)k_combine_Z, cs);
    k_combine_Z<<<dim3(kb.nblk, nb), 256, cs, cx.stream>>>(kb.N, ldz, Z, zs, kb.y, kb.sS(), x, xs, kb.st);
}

void launch_residual_norm(const Ctx& cx, const KrylovBufs& kb, int nb, const double2* f, long long fs,
                          const double2* Ax, long long axs, double* out) {
    k_resid_part<<<dim3(kb.nblk, nb), kRedThreads, 0, cx.stream>>>(kb.N, f, fs, Ax, axs, kb.npart, kb.nblk);
    k_sum_sqrt<<<(nb + 255) / 256, 256, 0, cx.stream>>>(nb, kb.nblk, kb.npart, out);
}

}  // namespace hzs
