// GMRES kernels (Section 5): Arnoldi with classical Gram-Schmidt and one
// reorthogonalisation (CGS2; on the mixed-precision path the delayed variant
// over a double-float basis), Givens rotations on the Hessenberg matrix, the
// triangular solve and the solution update.
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
#include "f32x2.cuh"
#include "kernels.cuh"

namespace hzs {

constexpr int kRedThreads = 256;
constexpr int kDotGroup64 = 4;     // basis vectors per warp pass (FP64 multi-dot)
constexpr int kDotGroupDC = 4;     // basis vectors per warp pass (delayed CGS2 multi-dot)
constexpr int kUpdUnroll = 4;      // basis vectors per group of the delayed CGS2 update
constexpr int kUpdBlocksPerSM = 2; // resident blocks of the delayed CGS2 update (up to 128 registers a thread)
constexpr int kSmemPerSM = 228 * 1024;   // shared memory of one SM (GB300)

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

// ---- double-float basis (mixed-precision path)
// The basis is held as double-float pairs V32 + V32lo (complex64 rounding and
// remainder).  The kernels on it move two consecutive entries per lane per load
// (16-byte accesses); vectors are padded to an even length whose padding stays
// zero (the buffers are cleared when allocated and no kernel writes the padding
// with anything but zero).  Indices count entry pairs: Np pairs per vector, ldp
// between vectors.

__device__ __forceinline__ float2 lo2(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(float4 a) { return make_float2(a.z, a.w); }

// Remainders of an entry pair, stored as L: float4 (complex64 words, wide) or
// uint2 (bf16 pairs, narrow: word k holds entry k's real part in its low half and
// its imaginary part in its high half, the layout of LoDst's narrow array).
// Unpacked to (re0, im0, re1, im1); a bf16 widens to FP32 exactly by a shift.
__device__ __forceinline__ float4 lo_unpack(float4 v) { return v; }
__device__ __forceinline__ float4 lo_unpack(uint2 v) {
    return make_float4(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u), __uint_as_float(v.y << 16),
                       __uint_as_float(v.y & 0xffff0000u));
}
__device__ __forceinline__ void lo_store(float4* p, float4 v) { *p = v; }
__device__ __forceinline__ void lo_store(uint2* p, float4 v) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    memcpy(&u.x, &a, 4);
    memcpy(&u.y, &b, 4);
    *p = u;
}

// (sh, sl) += c * v for one complex component pair, double-float:
// re += cr vr - ci vi ; im += cr vi + ci vr
__device__ __forceinline__ void df_cmac(float& rh, float& rl, float& ih, float& il, const float4& c, float vrh,
                                        float vrl, float vih, float vil) {
    df_fma(rh, rl, c.x, c.y, vrh, vrl);
    df_fma(rh, rl, -c.z, -c.w, vih, vil);
    df_fma(ih, il, c.x, c.y, vih, vil);
    df_fma(ih, il, c.z, c.w, vrh, vrl);
}

constexpr int kFinWarps = 4;                   // warps per right-hand side in the Givens kernels
constexpr int kFinThreads = 32 * kFinWarps;

__device__ __forceinline__ double2 shfl_up_c(double2 v, int off) {
    return make_double2(__shfl_up_sync(0xffffffffu, v.x, off), __shfl_up_sync(0xffffffffu, v.y, off));
}

// Block-wide sums for the Givens kernels (kFinThreads threads, every thread gets the result).
__device__ __forceinline__ double fin_sum(double v, double* red) {
    v = warp_sum_d(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < kFinWarps; ++k) s += red[k];
    return s;
}
__device__ __forceinline__ double2 fin_sum2(double2 v, double* red) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { red[2 * (threadIdx.x >> 5)] = v.x; red[2 * (threadIdx.x >> 5) + 1] = v.y; }
    __syncthreads();
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < kFinWarps; ++k) { s.x += red[2 * k]; s.y += red[2 * k + 1]; }
    return s;
}

// Brings Hessenberg column jc (col[0..jc+1], in shared memory) to triangular
// form: applies the stored rotations 0..jc-1 (scs, ssn: shared copies of cs, sn),
// computes rotation jc that zeroes col[jc+1] (stored in cs[jc], sn[jc]), applies
// it to the right-hand side g and returns the new residual estimate |g[jc+1]|.
// Called by all kFinThreads threads of the block.
//
// Applying the old rotations is a linear recurrence in the running entry a:
//   col'[i] = c_i a_i + s_i col[i+1],   a_{i+1} = -conj(s_i) a_i + c_i col[i+1],
// i.e. a_{i+1} = M_i(a_i) with the affine map M_i(a) = alpha_i a + beta_i.  Affine
// maps compose associatively, so each thread composes the maps of its own segment
// of consecutive rotations, a scan (Kogge-Stone within each warp, then the warp
// totals in order) combines the segments, and each thread replays its segment
// from the a it receives.  |alpha_i| <= 1, so the composed maps stay bounded.
// The FP64 pipe executes one warp instruction per 16 cycles per SM, so the work
// is spread over one warp per SM sub-partition.
__device__ double givens_column(int jc, double2* col, const double* scs, const double2* ssn, double* cs,
                                double2* sn, double2* g) {
    __shared__ double2 wA[kFinWarps], wB[kFinWarps], s_a;
    __shared__ double s_res;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = (jc + kFinThreads - 1) / kFinThreads;
    const int s0 = min(tid * L, jc), s1 = min(s0 + L, jc);
    const double2 a0 = col[0];
    const double2 bnd = col[s1];     // col[i+1] for the segment's last i; the next thread overwrites it
    double2 A = make_double2(1.0, 0.0), B = make_double2(0.0, 0.0);
    for (int i = s0; i < s1; ++i) {
        const double2 al = make_double2(-ssn[i].x, ssn[i].y);      // -conj(s_i)
        const double2 be = cscale(col[i + 1], scs[i]);
        B = cfma(al, B, be);
        A = cmul(al, A);
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double2 A1 = shfl_up_c(A, off), B1 = shfl_up_c(B, off);
        if (lane >= off) {            // (A, B) <- (A, B) o (A1, B1): the earlier segments first
            B = cfma(A, B1, B);
            A = cmul(A, A1);
        }
    }
    if (lane == 31) { wA[warp] = A; wB[warp] = B; }
    __syncthreads();                  // also orders every read of col above before the writes below
    double2 aw = a0;                  // value entering this warp: earlier warps' totals applied in order
    for (int k = 0; k < warp; ++k) aw = cfma(wA[k], aw, wB[k]);
    const double2 Ap = shfl_up_c(A, 1), Bp = shfl_up_c(B, 1);
    double2 a = lane == 0 ? aw : cfma(Ap, aw, Bp);
    for (int i = s0; i < s1; ++i) {
        const double c = scs[i];
        const double2 sv = ssn[i];
        const double2 b = i + 1 == s1 ? bnd : col[i + 1];
        // t = c a + s b ; a' = -conj(s) a + c b
        const double2 t = cfma(sv, b, cscale(a, c));
        const double2 csn = make_double2(sv.x, -sv.y);
        a = cfms(csn, a, cscale(b, c));
        col[i] = t;
    }
    // the last thread ends with a_jc (a thread with an empty segment passes its incoming value on)
    if (tid == kFinThreads - 1) s_a = a;
    __syncthreads();
    if (tid == 0) {
        a = s_a;
        const double2 b = col[jc + 1];
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
        cs[jc] = c; sn[jc] = sv;
        col[jc] = cfma(sv, b, cscale(a, c));
        col[jc + 1] = make_double2(0.0, 0.0);
        const double2 gj = g[jc];
        const double2 csn = make_double2(sv.x, -sv.y);
        const double2 gn = cscale(cmul(csn, gj), -1.0);
        g[jc + 1] = gn;
        g[jc] = cscale(gj, c);
        s_res = hypot(gn.x, gn.y);
    }
    __syncthreads();
    return s_res;
}

// ---- delayed CGS2 (mixed-precision path, see launch_dcgs2_step)
// Classical Gram-Schmidt with the reorthogonalisation of basis vector j
// postponed to step j, where it shares one read of the basis with the first
// projection of the new vector w = A z_j (Bielich, Langou, Thomas, Swirydowicz,
// Yamazaki and Boman, "Low-synch Gram-Schmidt with delayed reorthogonalization
// for Krylov solvers", Parallel Computing 112, 2022).  Per Arnoldi step the
// basis is read twice (one multi-dot, one update) instead of four times.
// At the start of step j, slot j holds u~_j, the once-projected w of step j-1
// (not yet reorthogonalised or normalised), and slot j+1 holds w.  With Q the
// orthonormal vectors 0..j-1 (vector i = sigma[i] V_i):
//   dot pass:  alpha = Q^H u~_j, b = Q^H w, c = |u~_j|^2, d = u~_j^H w, all in
//              complex64 on the leading words of the basis;
//   finish:    beta_j^2 = c - |alpha|^2, column j-1 of H is completed as
//              h1_{j-1} + alpha with subdiagonal beta_j, the first-pass
//              coefficients of column j are b and (d - alpha^H b) / beta_j;
//   update:    V_j = u~_j - Q alpha (sigma_j = 1/beta_j),
//              w  <- w - Q b - h_jj q_j  (double-float), |w|^2.
// The preconditioner of step j is applied to u~_j / |u~_j|: the flexible
// Arnoldi relation A Z = Q H holds for any z_j, and span{u~_0..u~_j} equals
// span{q_0..q_j}, so the iterates are those of FGMRES with z_j = M q_j.
// Precision: the update pass applies the coefficients it is given exactly (to
// the basis's double-float width), so the Arnoldi relation holds to that width
// whatever their accuracy; the coefficients' complex64 rounding only sets how
// orthogonal the basis stays (CGS2 in a precision keeps it orthogonal to a
// small multiple of that precision, about 1e-6 here), which changes neither the
// Krylov space nor, by more than that factor, the residual estimate.  c enters
// beta_j, which therefore carries complex64 relative accuracy: q_j = V_j / beta_j
// by definition, so the relation is unaffected.
// Row layout of the dot partials per block (16 B slots): alpha at [0, S) and b at
// [S, 2S) as complex64 in the first 8 bytes of a slot, c at 2S and d at 2S+1 as
// complex128 (S = maxit+1).

template <int G>
__global__ void __launch_bounds__(kRedThreads, 4) k_dcgs_dot(int j, long long Np, long long ldp, int ps, int S,
                                                          const float4* __restrict__ V32, long long sVp, int has_w,
                                                          double2* __restrict__ part, long long sP,
                                                          const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (st[r].done) return;
    V32 += r * sVp;
    const float4* uh = V32 + (size_t)j * ldp;
    const float4* wh = has_w ? V32 + (size_t)(j + 1) * ldp : uh;     // slot j+1 exists only with w
    part += r * sP + (size_t)blockIdx.x * ps;
    long long e0, e1;
    chunk_of(Np, e0, e1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ngroups = (j + G - 1) / G;
    for (int gi = warp; gi <= ngroups; gi += nw) {
        if (gi == ngroups) {
            // c = |u~|^2 and d = u~^H w
            float c = 0.f;
            float2 d = make_float2(0.f, 0.f);
            for (long long e = e0 + lane; e < e1; e += 32) {
                const float4 xh = uh[e];
                c = fmaf(xh.x, xh.x, fmaf(xh.y, xh.y, fmaf(xh.z, xh.z, fmaf(xh.w, xh.w, c))));
                if (has_w) {
                    const float4 yh = wh[e];
                    d = cfma_conj(lo2(xh), lo2(yh), d);
                    d = cfma_conj(hi2(xh), hi2(yh), d);
                }
            }
            const double cs = warp_sum_d((double)c);
            const double2 ds = warp_sum(make_double2((double)d.x, (double)d.y));
            if (lane == 0) {
                part[2 * S] = make_double2(cs, 0.0);
                part[2 * S + 1] = ds;
            }
            continue;
        }
        const int i0 = gi * G;
        float2 aa[G], bb[G];
#pragma unroll
        for (int t = 0; t < G; ++t) aa[t] = bb[t] = make_float2(0.f, 0.f);
        for (long long e = e0 + lane; e < e1; e += 32) {
            // u~ and w are re-read by every warp of the block: read-only cache path;
            // the basis is read once: streaming (evict-first) loads
            const float4 xh = __ldg(uh + e);
            const float4 yh = has_w ? __ldg(wh + e) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 vh[G];
#pragma unroll
            for (int t = 0; t < G; ++t)
                vh[t] = i0 + t < j ? __ldcs(V32 + (size_t)(i0 + t) * ldp + e) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int t = 0; t < G; ++t) {
                aa[t] = cfma_conj(lo2(vh[t]), lo2(xh), aa[t]);      // alpha: conj(v) u~
                aa[t] = cfma_conj(hi2(vh[t]), hi2(xh), aa[t]);
                bb[t] = cfma_conj(lo2(vh[t]), lo2(yh), bb[t]);      // b: conj(v) w
                bb[t] = cfma_conj(hi2(vh[t]), hi2(yh), bb[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < G; ++t) {
            aa[t] = warp_sum(aa[t]);
            bb[t] = warp_sum(bb[t]);
        }
        if (lane == 0) {
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (i0 + t < j) {
                    // raw FP32 words; the reduction converts (FP64 instructions stay out of this loop)
                    reinterpret_cast<float4*>(part)[i0 + t] = make_float4(aa[t].x, aa[t].y, 0.f, 0.f);
                    reinterpret_cast<float4*>(part)[S + i0 + t] = make_float4(bb[t].x, bb[t].y, 0.f, 0.f);
                }
        }
    }
}

// Cross-block sums of the dot pass, one warp per value (fixed order):
// h2[i] = sigma_i alpha_i, hn[i] = sigma_i b_i (i < j), hn[j] = c, hn[j+1] = d.
// The b partials arrive as FP32 words (see k_dcgs_dot), c and d as FP64; alpha as
// FP32 words on the double-float path (A64 false) and as FP64 on the FP64 basis.
template <bool A64>
__global__ void k_dcgs_reduce(int j, int nblk, int ps, int S, const double2* __restrict__ part, long long sP,
                              const double* __restrict__ sigma, double2* __restrict__ h2, double2* __restrict__ hn,
                              long long sS, long long sN, const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (st[r].done) return;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= 2 * j + 2) return;
    part += r * sP; sigma += r * sS; h2 += r * sS; hn += r * sN;
    const int col = k < j ? k : (k < 2 * j ? S + (k - j) : 2 * S + (k - 2 * j));
    double2 s = make_double2(0.0, 0.0);
    if (A64 && k < j) {
        for (int b = lane; b < nblk; b += 32) s = cadd(s, part[(size_t)b * ps + col]);
    } else if (k < 2 * j) {
        // alpha and b: complex64 in the first 8 bytes of the slot
        const float4* pf = reinterpret_cast<const float4*>(part);
        for (int b = lane; b < nblk; b += 32) {
            const float4 v = pf[(size_t)b * ps + col];
            s.x += (double)v.x;
            s.y += (double)v.y;
        }
    } else {
        for (int b = lane; b < nblk; b += 32) s = cadd(s, part[(size_t)b * ps + col]);
    }
    s = warp_sum(s);
    if (lane == 0) {
        if (k < j) h2[k] = cscale(s, sigma[k]);
        else if (k < 2 * j) hn[k - j] = cscale(s, sigma[k - j]);
        else hn[j + (k - 2 * j)] = s;
    }
}

// Step j's coefficients for entry r = blockIdx.x (kFinThreads threads): beta_j,
// column j-1 of H before rotation (h1 + alpha over beta_j; NaN in place of beta_j
// when beta_j^2 is not finite), and the first-pass coefficients of column j (h1,
// for the update pass and the next completion) with sigma_j = 1 / beta_j.
// j == maxit (last_only) writes the last column only.  The rotation of the column
// and the stop test (k_dcgs_givens) are left off the path to the update pass.
__global__ void __launch_bounds__(kFinThreads) k_dcgs_coef(int j, int maxit, int last_only,
                                                          const double2* __restrict__ hn, long long sN,
                                                          double2* __restrict__ h1, const double2* __restrict__ h2,
                                                          double2* __restrict__ H, long long sH,
                                                          double* __restrict__ sigma, long long sS,
                                                          KState* __restrict__ st, int* __restrict__ active) {
    const int r = blockIdx.x;
    if (st[r].done) return;
    hn += r * sN; h1 += r * sS; h2 += r * sS; H += r * sH; sigma += r * sS;
    KState* s0 = st + r;
    __shared__ double red[2 * kFinWarps];
    const int tid = threadIdx.x;
    // |alpha|^2 and alpha^H b
    double aa = 0.0;
    double2 ab = make_double2(0.0, 0.0);
    for (int i = tid; i < j; i += kFinThreads) {
        const double2 a = h2[i], b = hn[i];
        aa = fma(a.x, a.x, fma(a.y, a.y, aa));
        ab = cfma_conj(a, b, ab);
    }
    aa = fin_sum(aa, red);
    ab = fin_sum2(ab, red);
    const double c = hn[j].x;
    const double2 d = hn[j + 1];
    const double b2 = c - aa;
    const double beta = b2 > 0.0 ? sqrt(b2) : 0.0;
    if (j > 0) {
        double2* out = H + (size_t)(j - 1) * (maxit + 1);
        for (int i = tid; i < j; i += kFinThreads) out[i] = cadd(h1[i], h2[i]);
        if (tid == 0) out[j] = make_double2(isfinite(b2) ? beta : nan(""), 0.0);
        __syncthreads();                     // the old h1 is read before it is overwritten below
    }
    if (last_only) return;
    // column j, first pass (alpha is complete for the old vectors; q_j = (u~ - Q alpha) / beta).
    // The update pass applies sigma_i h1_i to V_i as an FP32 number (the coefficient comes
    // from complex64 dot products, so rounding it loses nothing): h1_i is recorded as that
    // rounded product over sigma_i, the value the Arnoldi relation then holds for.
    const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
    for (int i = tid; i < j; i += kFinThreads) {
        const double si = sigma[i];
        const double2 c = cscale(hn[i], si);
        const double2 cr = make_double2((double)(float)c.x, (double)(float)c.y);
        h1[i] = si > 0.0 ? cscale(cr, 1.0 / si) : hn[i];
    }
    if (tid == 0) {
        h1[j] = cscale(csub(d, ab), ib);
        sigma[j] = ib;
        if (j == 0 && !(beta > 0.0)) { s0->done = 1; s0->conv = 1; s0->breakdown = 1; atomicSub(active, 1); }
    }
}

// Step j >= 1, entry r = blockIdx.x (kFinThreads threads): rotation of column j-1
// of H (from k_dcgs_coef), residual estimate with j columns and the stop test.
// Runs beside the update pass of the same step; the next step waits for it.
__global__ void __launch_bounds__(kFinThreads) k_dcgs_givens(int j, int maxit, int last_only,
                                                            double2* __restrict__ H, long long sH,
                                                            double* __restrict__ cs, double2* __restrict__ sn,
                                                            double2* __restrict__ g, long long sS,
                                                            KState* __restrict__ st, int* __restrict__ active) {
    const int r = blockIdx.x;
    if (st[r].done) return;
    H += r * sH; cs += r * sS; sn += r * sS; g += r * sS;
    KState* s0 = st + r;
    extern __shared__ double2 fsm[];
    double2* col = fsm;                                   // j + 1
    double2* ssn = col + (j + 1);                         // j - 1
    double* scs = reinterpret_cast<double*>(ssn + (j > 0 ? j - 1 : 0));
    const int tid = threadIdx.x;
    double2* out = H + (size_t)(j - 1) * (maxit + 1);
    for (int i = tid; i <= j; i += kFinThreads) col[i] = out[i];
    for (int i = tid; i < j - 1; i += kFinThreads) { ssn[i] = sn[i]; scs[i] = cs[i]; }
    __syncthreads();
    const double beta = col[j].x;
    const double resid = givens_column(j - 1, col, scs, ssn, cs, sn, g);
    if (tid == 0) {
        s0->resid = resid;
        s0->hnext = beta;
        s0->iters = j;
        int fin = 1;
        if (!isfinite(resid) || !isfinite(beta)) s0->nonfinite = 1;
        else if (resid <= s0->tolabs) s0->conv = 1;
        else if (beta == 0.0) { s0->breakdown = 1; s0->conv = 1; }
        else if (!last_only && j < maxit) fin = 0;
        if (fin) { s0->done = 1; atomicSub(active, 1); }
    }
    for (int i = tid; i <= j; i += kFinThreads) out[i] = col[i];
}

// Remainder pairs of one entry pair as two packed (re, im) lanes.
__device__ __forceinline__ void lo_pairs(float4 v, f2x& l0, f2x& l1) {
    const ulonglong2 u = *reinterpret_cast<const ulonglong2*>(&v);
    l0 = u.x; l1 = u.y;
}
__device__ __forceinline__ void lo_pairs(uint2 v, f2x& l0, f2x& l1) {
    l0 = f2_pack(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u));
    l1 = f2_pack(__uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
}

// Per-thread asynchronous copies global -> shared (each thread later reads back only
// what it copied itself, after cp.async.wait_group: no block barrier is involved).
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_lo(float4* smem, const float4* gmem) { cp_async_16(smem, gmem); }
__device__ __forceinline__ void cp_async_lo(uint2* smem, const uint2* gmem) { cp_async_8(smem, gmem); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Coefficients of basis vector i for the update pass, as broadcast packed pairs
// (see df_fma2): c = h1_i sigma_i in double-float, a = h2_i sigma_i in complex64.
struct alignas(16) UpdCoef {
    f2x Pr, Nr, Pi, Ni;                 // c.re and c.im
    f2x ar, ai;                         // a.re and a.im
};

// Update pass of step j (two entries per lane): V_j = u~_j - sum_i (sigma_i alpha_i) V_i
// (the small reorthogonalisation sum in complex64, its subtraction in double-float),
// w = w - sum_i (sigma_i b_i) V_i - (h_jj sigma_j) V_j in double-float;
// npart[b] = sum_e |w[e]|^2 (FP32 on the leading words: it only sets a scale).
// The sums over the basis run on packed FP32 pairs, one entry's (re, im) per
// register: sum_i c_i v_i = sum_i Re(c_i) v_i + i sum_i Im(c_i) v_i, so each entry
// keeps the two real-coefficient sums A = sum Re(c) v and B = sum Im(c) v (and the
// same for the reorthogonalisation) and forms A + i B once at the end.
template <typename L, int NS>
__global__ void __launch_bounds__(kRedThreads, kUpdBlocksPerSM) k_dcgs_update(int j, long long Np, long long ldp,
                                                             float4* __restrict__ V32, L* __restrict__ V32lo,
                                                             long long sVp, const double* __restrict__ sigma,
                                                             const double2* __restrict__ h1,
                                                             const double2* __restrict__ h2, long long sS,
                                                             double* __restrict__ npart, int nblk,
                                                             const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (st[r].done) return;
    V32 += r * sVp; V32lo += r * sVp; sigma += r * sS; h1 += r * sS; h2 += r * sS;
    float4* uh = V32 + (size_t)j * ldp;
    L* ul = V32lo + (size_t)j * ldp;
    float4* wh = V32 + (size_t)(j + 1) * ldp;
    L* wl = V32lo + (size_t)(j + 1) * ldp;
    // dynamic shared memory: j coefficient sets, then (NS > 0) the per-thread copy ring
    // of NS groups of kUpdUnroll basis vectors (leading words, then remainders); NS == 0
    // keeps two groups in registers instead
    extern __shared__ UpdCoef ucs[];
    __shared__ float4 s_cj;                                 // h_jj sigma_j (double-float)
    ulonglong2* ring_h = reinterpret_cast<ulonglong2*>(ucs + (j > 0 ? j : 1));
    L* ring_l = reinterpret_cast<L*>(ring_h + NS * kUpdUnroll * blockDim.x);
    (void)ring_h; (void)ring_l;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const double2 c = cscale(h1[i], sigma[i]);
        float crh, crl, cih, cil;
        split_d(c.x, crh, crl);
        split_d(c.y, cih, cil);
        if (i == j) { s_cj = make_float4(crh, crl, cih, cil); continue; }
        const float2 a = to_f(cscale(h2[i], sigma[i]));
        UpdCoef u;
        // c is an FP32 value for i < j (k_dcgs_coef records the rounded coefficient): crl and
        // cil are below 2^-50 of it and are dropped
        u.Pr = f2_pack(crh, crh); u.Nr = f2_pack(-crh, -crh);
        u.Pi = f2_pack(cih, cih); u.Ni = f2_pack(-cih, -cih);
        u.ar = f2_pack(a.x, a.x); u.ai = f2_pack(a.y, a.y);
        ucs[i] = u;
    }
    __syncthreads();
    const float4 cj = s_cj;
    long long e0, e1;
    chunk_of(Np, e0, e1);
    float nrmf = 0.f;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        // per entry k of the pair: A_k, B_k (double-float) and S_k, T_k (reorthogonalisation)
        f2x A0h = 0, A0l = 0, B0h = 0, B0l = 0, A1h = 0, A1l = 0, B1h = 0, B1l = 0;
        f2x S0 = 0, T0 = 0, S1 = 0, T1 = 0;
        const ulonglong2* ph = reinterpret_cast<const ulonglong2*>(V32 + e);
        const L* pl = V32lo + e;
        // basis vectors in the order j-1 .. 0: the dot pass read 0 .. j-1, so the vectors
        // still in L2 come first, and this pass leaves vectors 0, 1, .. in L2 for the next
        // dot pass
        auto vi = [&](int k) { return j - 1 - k; };
        auto step = [&](const UpdCoef& u, ulonglong2 vh, L vlr) {
            f2x l0, l1;
            lo_pairs(vlr, l0, l1);
            df_fma2(A0h, A0l, u.Pr, u.Nr, vh.x, l0);
            df_fma2(B0h, B0l, u.Pi, u.Ni, vh.x, l0);
            df_fma2(A1h, A1l, u.Pr, u.Nr, vh.y, l1);
            df_fma2(B1h, B1l, u.Pi, u.Ni, vh.y, l1);
            S0 = fma2(u.ar, vh.x, S0); T0 = fma2(u.ai, vh.x, T0);
            S1 = fma2(u.ar, vh.y, S1); T1 = fma2(u.ai, vh.y, T1);
        };
        if constexpr (NS > 0) {
            // groups of kUpdUnroll vectors stream through a per-thread ring of NS stages in
            // shared memory (cp.async): NS - 1 groups are in flight while one is consumed,
            // and no registers are held for them
            const int ngrp = j / kUpdUnroll;
            auto slot = [&](int stage, int t) { return (stage * kUpdUnroll + t) * (int)blockDim.x + (int)threadIdx.x; };
            auto issue = [&](int g, int stage) {
    #pragma unroll
                for (int t = 0; t < kUpdUnroll; ++t) {
                    const size_t off = (size_t)vi(g * kUpdUnroll + t) * ldp;
                    cp_async_16(ring_h + slot(stage, t), ph + off);
                    cp_async_lo(ring_l + slot(stage, t), pl + off);
                }
            };
    #pragma unroll
            for (int g = 0; g < NS - 1; ++g) {
                if (g < ngrp) issue(g, g);
                cp_async_commit();
            }
            int cs = 0;                                         // stage of group g
            for (int g = 0; g < ngrp; ++g) {
                const int is = cs == 0 ? NS - 1 : cs - 1;       // stage of group g + NS - 1 (consumed at g - 1)
                if (g + NS - 1 < ngrp) issue(g + NS - 1, is);
                cp_async_commit();
                cp_async_wait<NS - 1>();                        // group g has landed
    #pragma unroll
                for (int t = 0; t < kUpdUnroll; ++t) step(ucs[vi(g * kUpdUnroll + t)], ring_h[slot(cs, t)], ring_l[slot(cs, t)]);
                df_norm2(A0h, A0l); df_norm2(B0h, B0l); df_norm2(A1h, A1l); df_norm2(B1h, B1l);
                cs = cs + 1 == NS ? 0 : cs + 1;
            }
            for (int i = ngrp * kUpdUnroll; i < j; ++i) step(ucs[vi(i)], ph[(size_t)vi(i) * ldp], pl[(size_t)vi(i) * ldp]);
        } else {
            // two groups of kUpdUnroll vectors in registers: the loads of the next group are
            // issued before the current group is consumed (the work on one group covers less
            // time than a DRAM round trip)
            ulonglong2 ha[kUpdUnroll], hb[kUpdUnroll];
            L la[kUpdUnroll], lb[kUpdUnroll];
            int i = 0;
            if (kUpdUnroll <= j) {
    #pragma unroll
                for (int t = 0; t < kUpdUnroll; ++t) {
                    ha[t] = ph[(size_t)vi(t) * ldp];
                    la[t] = pl[(size_t)vi(t) * ldp];
                }
            }
            // invariant: ha, la hold group i whenever i + kUpdUnroll <= j
            for (; i + 2 * kUpdUnroll <= j; i += 2 * kUpdUnroll) {
    #pragma unroll
                for (int t = 0; t < kUpdUnroll; ++t) {
                    hb[t] = ph[(size_t)vi(i + kUpdUnroll + t) * ldp];
                    lb[t] = pl[(size_t)vi(i + kUpdUnroll + t) * ldp];
                }
    #pragma unroll
                for (int t = 0; t < kUpdUnroll; ++t) step(ucs[vi(i + t)], ha[t], la[t]);
                df_norm2(A0h, A0l); df_norm2(B0h, B0l); df_norm2(A1h, A1l); df_norm2(B1h, B1l);
                if (i + 3 * kUpdUnroll <= j) {
    #pragma unroll
                    for (int t = 0; t < kUpdUnroll; ++t) {
                        ha[t] = ph[(size_t)vi(i + 2 * kUpdUnroll + t) * ldp];
                        la[t] = pl[(size_t)vi(i + 2 * kUpdUnroll + t) * ldp];
                    }
                }
    #pragma unroll
                for (int t = 0; t < kUpdUnroll; ++t) step(ucs[vi(i + kUpdUnroll + t)], hb[t], lb[t]);
                df_norm2(A0h, A0l); df_norm2(B0h, B0l); df_norm2(A1h, A1l); df_norm2(B1h, B1l);
            }
            if (i + kUpdUnroll <= j) {
    #pragma unroll
                for (int t = 0; t < kUpdUnroll; ++t) step(ucs[vi(i + t)], ha[t], la[t]);
                df_norm2(A0h, A0l); df_norm2(B0h, B0l); df_norm2(A1h, A1l); df_norm2(B1h, B1l);
                i += kUpdUnroll;
            }
            for (; i < j; ++i) step(ucs[vi(i)], ph[(size_t)vi(i) * ldp], pl[(size_t)vi(i) * ldp]);
        }
        // sum_i c_i v_i = A + i B per entry: re = A.re - B.im, im = A.im + B.re
        float a0h, a0l, b0h, b0l, a1h, a1l, b1h, b1l;
        {
            const float2 ah = f2_unpack(A0h), al = f2_unpack(A0l), bh = f2_unpack(B0h), bl = f2_unpack(B0l);
            a0h = ah.x; a0l = al.x; df_add(a0h, a0l, -bh.y, -bl.y);
            b0h = ah.y; b0l = al.y; df_add(b0h, b0l, bh.x, bl.x);
        }
        {
            const float2 ah = f2_unpack(A1h), al = f2_unpack(A1l), bh = f2_unpack(B1h), bl = f2_unpack(B1l);
            a1h = ah.x; a1l = al.x; df_add(a1h, a1l, -bh.y, -bl.y);
            b1h = ah.y; b1l = al.y; df_add(b1h, b1l, bh.x, bl.x);
        }
        const float2 sa0 = f2_unpack(S0), ta0 = f2_unpack(T0), sa1 = f2_unpack(S1), ta1 = f2_unpack(T1);
        const float2 s0 = make_float2(sa0.x - ta0.y, sa0.y + ta0.x);
        const float2 s1 = make_float2(sa1.x - ta1.y, sa1.y + ta1.x);
        // V_j = u~ - s
        float4 xh = uh[e], xl = lo_unpack(ul[e]);
        df_add(xh.x, xl.x, -s0.x, 0.f); df_norm(xh.x, xl.x);
        df_add(xh.y, xl.y, -s0.y, 0.f); df_norm(xh.y, xl.y);
        df_add(xh.z, xl.z, -s1.x, 0.f); df_norm(xh.z, xl.z);
        df_add(xh.w, xl.w, -s1.y, 0.f); df_norm(xh.w, xl.w);
        uh[e] = xh;
        lo_store(ul + e, xl);
        // + (h_jj sigma_j) V_j
        df_cmac(a0h, a0l, b0h, b0l, cj, xh.x, xl.x, xh.y, xl.y);
        df_cmac(a1h, a1l, b1h, b1l, cj, xh.z, xl.z, xh.w, xl.w);
        float4 yh = wh[e], yl = lo_unpack(wl[e]);
        df_add(yh.x, yl.x, -a0h, -a0l); df_norm(yh.x, yl.x);
        df_add(yh.y, yl.y, -b0h, -b0l); df_norm(yh.y, yl.y);
        df_add(yh.z, yl.z, -a1h, -a1l); df_norm(yh.z, yl.z);
        df_add(yh.w, yl.w, -b1h, -b1l); df_norm(yh.w, yl.w);
        wh[e] = yh;
        lo_store(wl + e, yl);
        // |u~_{j+1}| only scales the next preconditioner input: FP32 on the leading words
        nrmf = fmaf(yh.x, yh.x, fmaf(yh.y, yh.y, fmaf(yh.z, yh.z, fmaf(yh.w, yh.w, nrmf))));
    }
    const double nrm = nrmf;
    block_norm_part(nrm, npart + (size_t)r * nblk);
}

// ---- delayed CGS2 on an FP64 basis (mixed-precision path, see launch_dcgs2_step64)
// The same step as above with the basis, u~_j and w held as complex128.  The
// quantities that set the Arnoldi process - the reorthogonalisation coefficients
// alpha = Q^H u~_j, c = |u~_j|^2, d = u~_j^H w and the first-projection update
// w - Q b - h_jj q_j - are computed with FP64 fused multiply-adds.  The
// first-projection coefficients b = Q^H w are complex64 dot products on the
// leading 24 bits of each entry: they are recorded in H exactly as the update
// applies them, so the Arnoldi relation holds to FP64 whatever their accuracy,
// and the projection they leave behind (about 2^-24 |w| along Q) is what alpha
// removes one step later, in FP64.  The reorthogonalisation update u~_j - Q alpha
// is a sum of small terms (|alpha_i| of that order relative to |u~_j|), so it
// runs in double-float arithmetic on the FP32 pipes: its error is about 2^-46
// of terms that are themselves 2^-20 of |u~_j| or less, below the FP64 rounding
// of the result (the part's FP64 pipe runs at 1/64 of the FP32 rate).

// Leading 24 significant bits of x (the fraction truncated) as an FP32 value,
// from integer operations on the FP64 word: the exponent is rebiased from 1023
// to 127.  |x| < 2^-126 gives 0; |x| must be below 2^128.
__device__ __forceinline__ float dhead(double x) {
    const unsigned H = (unsigned)__double2hiint(x), L = (unsigned)__double2loint(x);
    const unsigned a = H & 0x7fffffffu;
    const unsigned h = __funnelshift_l(L, a - (896u << 20), 3);
    return __uint_as_float((a >= (897u << 20) ? h : 0u) | (H & 0x80000000u));
}
// x = hd + md + r with hd = dhead(x), md the next 23 fraction bits (exact FP32
// values) and |r| < 2^-46 |x|: md = rb * 2^(e-1069) with rb = fraction bits 28..6
// and e the biased FP64 exponent, built as as_float(E | rb) - as_float(E) for the
// FP32 exponent field E = e - 919.  |x| < 2^-97 gives two zeros.
__device__ __forceinline__ void dsplit(double x, float& hd, float& md) {
    const unsigned H = (unsigned)__double2hiint(x), L = (unsigned)__double2loint(x);
    const unsigned a = H & 0x7fffffffu, sg = H & 0x80000000u;
    const bool ok = a >= (926u << 20);
    const unsigned h = __funnelshift_l(L, a - (896u << 20), 3);
    const unsigned E = sg | (((a - (919u << 20)) << 3) & 0x7f800000u);
    const float m = __uint_as_float(E | ((L >> 6) & 0x7fffffu)) - __uint_as_float(E);
    hd = ok ? __uint_as_float(sg | h) : 0.f;
    md = ok ? m : 0.f;
}

// Dot pass of step j on the FP64 basis V (entry r = blockIdx.y): per block chunk,
// alpha_i = conj(V_i) . u~ (FP64), b_i = conj(head V_i) . head w (complex64),
// c = |u~|^2 and d = conj(u~) . w (FP64).  Partials: alpha at [0, S) as FP64,
// b at [S, 2S) as FP32 words in the first 8 bytes, c at 2S and d at 2S+1 as FP64.
template <int G>
__global__ void __launch_bounds__(kRedThreads, 3) k_d64_dot(int j, long long N, long long ld, int ps, int S,
                                                           const double2* __restrict__ V, long long sV, int has_w,
                                                           double2* __restrict__ part, long long sP,
                                                           const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (st[r].done) return;
    V += r * sV;
    const double2* u = V + (size_t)j * ld;
    const double2* w = has_w ? V + (size_t)(j + 1) * ld : u;
    part += r * sP + (size_t)blockIdx.x * ps;
    long long e0, e1;
    chunk_of(N, e0, e1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ngroups = (j + G - 1) / G;
    for (int gi = warp; gi <= ngroups; gi += nw) {
        if (gi == ngroups) {
            double c = 0.0;
            double2 d = make_double2(0.0, 0.0);
            for (long long e = e0 + lane; e < e1; e += 32) {
                const double2 x = __ldg(u + e);
                c = fma(x.x, x.x, fma(x.y, x.y, c));
                if (has_w) d = cfma_conj(x, __ldg(w + e), d);
            }
            c = warp_sum_d(c);
            d = warp_sum(d);
            if (lane == 0) {
                part[2 * S] = make_double2(c, 0.0);
                part[2 * S + 1] = d;
            }
            continue;
        }
        const int i0 = gi * G;
        double2 aa[G];
        float2 bb[G];
#pragma unroll
        for (int t = 0; t < G; ++t) { aa[t] = make_double2(0.0, 0.0); bb[t] = make_float2(0.f, 0.f); }
        for (long long e = e0 + lane; e < e1; e += 32) {
            const double2 x = __ldg(u + e);
            float2 yh = make_float2(0.f, 0.f);
            if (has_w) {
                const double2 y = __ldg(w + e);
                yh = make_float2(dhead(y.x), dhead(y.y));
            }
            double2 v[G];
#pragma unroll
            for (int t = 0; t < G; ++t)
                v[t] = i0 + t < j ? __ldcs(V + (size_t)(i0 + t) * ld + e) : make_double2(0.0, 0.0);
#pragma unroll
            for (int t = 0; t < G; ++t) {
                aa[t] = cfma_conj(v[t], x, aa[t]);
                bb[t] = cfma_conj(make_float2(dhead(v[t].x), dhead(v[t].y)), yh, bb[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < G; ++t) {
            aa[t] = warp_sum(aa[t]);
            bb[t] = warp_sum(bb[t]);
        }
        if (lane == 0) {
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (i0 + t < j) {
                    part[i0 + t] = aa[t];
                    reinterpret_cast<float4*>(part)[S + i0 + t] = make_float4(bb[t].x, bb[t].y, 0.f, 0.f);
                }
        }
    }
}

// Coefficients of basis vector i for the FP64-basis update pass: c = sigma_i h1_i
// (an FP32 value, see k_dcgs_coef) and the reorthogonalisation coefficient
// a = sigma_i alpha_i as double-float pairs (re and im).
struct alignas(16) Upd64Coef {
    double2 c;
    float arh, arl, aih, ail;
};

// Update pass of step j on the FP64 basis (one entry per thread and sweep):
// V_j = u~_j - sum_i a_i V_i (double-float sum, FP64 subtraction),
// w <- w - sum_i c_i V_i - (h_jj sigma_j) V_j (FP64), npart[b] = sum_e |w[e]|^2.
__global__ void __launch_bounds__(kRedThreads, 3) k_d64_update(int j, long long N, long long ld,
                                                              double2* __restrict__ V, long long sV,
                                                              const double* __restrict__ sigma,
                                                              const double2* __restrict__ h1,
                                                              const double2* __restrict__ h2, long long sS,
                                                              double* __restrict__ npart, int nblk,
                                                              const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (st[r].done) return;
    V += r * sV; sigma += r * sS; h1 += r * sS; h2 += r * sS;
    double2* u = V + (size_t)j * ld;
    double2* w = V + (size_t)(j + 1) * ld;
    extern __shared__ Upd64Coef u64c[];
    __shared__ double2 s_cj;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const double2 c = cscale(h1[i], sigma[i]);
        if (i == j) { s_cj = c; continue; }
        const double2 a = cscale(h2[i], sigma[i]);
        Upd64Coef k;
        k.c = c;
        k.arh = (float)a.x; k.arl = (float)(a.x - (double)k.arh);
        k.aih = (float)a.y; k.ail = (float)(a.y - (double)k.aih);
        u64c[i] = k;
    }
    __syncthreads();
    const double2 cj = s_cj;
    long long e0, e1;
    chunk_of(N, e0, e1);
    double nrm = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0), acc2 = acc;
        float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;      // sum a_i V_i (double-float, re and im)
        auto step = [&](const Upd64Coef& k, double2 v, double2& ac) {
            ac = cfma(k.c, v, ac);
            float xh, xm, yh, ym;
            dsplit(v.x, xh, xm);
            dsplit(v.y, yh, ym);
            // re += ar vr - ai vi ; im += ar vi + ai vr
            df_fma(rh, rl, k.arh, k.arl, xh, xm);
            df_fma(rh, rl, -k.aih, -k.ail, yh, ym);
            df_fma(ih, il, k.arh, k.arl, yh, ym);
            df_fma(ih, il, k.aih, k.ail, xh, xm);
        };
        // basis vectors j-1 .. 0: the dot pass read 0 .. j-1, so those still in L2 come first
        int i = j - 1;
        for (; i >= 3; i -= 4) {
            const double2 v0 = __ldcs(V + (size_t)i * ld + e), v1 = __ldcs(V + (size_t)(i - 1) * ld + e);
            const double2 v2 = __ldcs(V + (size_t)(i - 2) * ld + e), v3 = __ldcs(V + (size_t)(i - 3) * ld + e);
            step(u64c[i], v0, acc);
            step(u64c[i - 1], v1, acc2);
            step(u64c[i - 2], v2, acc);
            step(u64c[i - 3], v3, acc2);
            df_norm(rh, rl);
            df_norm(ih, il);
        }
        for (; i >= 0; --i) step(u64c[i], __ldcs(V + (size_t)i * ld + e), acc);
        acc = cadd(acc, acc2);
        // V_j = u~ - (sum a_i V_i)
        double2 x = u[e];
        x.x = (x.x - (double)rh) - (double)rl;
        x.y = (x.y - (double)ih) - (double)il;
        u[e] = x;
        // w - sum c_i V_i - c_j V_j
        double2 y = csub(w[e], acc);
        y = cfms(cj, x, y);
        w[e] = y;
        nrm = fma(y.x, y.x, fma(y.y, y.y, nrm));
    }
    block_norm_part(nrm, npart + (size_t)r * nblk);
}

// sigt[j+1] = 1 / |u~_{j+1}| from the update pass's partial norms (one warp per entry;
// count partials per entry, stride apart).
__global__ void k_dcgs_scale(int j, int count, int stride, const double* __restrict__ npart,
                             double* __restrict__ sigt, long long sS, const KState* __restrict__ st) {
    const int r = blockIdx.x;
    if (st[r].done) return;
    npart += (size_t)r * stride;
    double s = 0.0;
    for (int b = threadIdx.x; b < count; b += 32) s += npart[b];
    s = warp_sum_d(s);
    if (threadIdx.x == 0) sigt[r * sS + j + 1] = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
}

// Completes step j of entry r = blockIdx.x (kFinThreads threads): h_{j+1,j} =
// ||w||, column j of H = h1 + h2, Givens rotations, residual estimate,
// convergence / breakdown flags.  The block norm partials are summed in a fixed
// order; an entry that finishes decrements the batch's active counter.
__global__ void __launch_bounds__(kFinThreads) k_arnoldi_finish(int j, int maxit, int nblk,
                                                               const double* __restrict__ npart,
                                                               const double2* __restrict__ h1,
                                                               const double2* __restrict__ h2,
                                                               double2* __restrict__ H, long long sH,
                                                               double* __restrict__ cs, double2* __restrict__ sn,
                                                               double2* __restrict__ g, double* __restrict__ sigma,
                                                               long long sS, KState* __restrict__ st,
                                                               int* __restrict__ active) {
    const int r = blockIdx.x;
    if (st[r].done) return;
    npart += (size_t)r * nblk;
    h1 += r * sS; h2 += r * sS; H += r * sH; cs += r * sS; sn += r * sS; g += r * sS; sigma += r * sS;
    KState* s0 = st + r;
    extern __shared__ double2 fsm[];
    __shared__ double red[2 * kFinWarps];
    double2* col = fsm;                                   // j + 2
    double2* ssn = col + (j + 2);                         // j
    double* scs = reinterpret_cast<double*>(ssn + j);     // j
    const int tid = threadIdx.x;
    double s = 0.0;
    for (int b = tid; b < nblk; b += kFinThreads) s += npart[b];
    s = fin_sum(s, red);
    const double beta = sqrt(s);
    for (int i = tid; i <= j; i += kFinThreads) col[i] = cadd(h1[i], h2[i]);
    for (int i = tid; i < j; i += kFinThreads) { ssn[i] = sn[i]; scs[i] = cs[i]; }
    if (tid == 0) col[j + 1] = make_double2(beta, 0.0);
    __syncthreads();
    const int ldh = maxit + 1;
    const double resid = givens_column(j, col, scs, ssn, cs, sn, g);
    if (tid == 0) {
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
    double2* out = H + (size_t)j * ldh;
    for (int i = tid; i <= j + 1; i += kFinThreads) out[i] = col[i];
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
                             double* __restrict__ sigma, double* __restrict__ sigt, double2* __restrict__ g, long long sS,
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
        if (sigt) sigt[r * sS] = sigma[r * sS];
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
    allow_dynamic_smem((const void*)k_arnoldi_finish, b);
    return b;
}

static void set_coef_smem_limit(const void* fn, size_t bytes) {
    allow_dynamic_smem(fn, bytes);
}

void launch_norm_init(const Ctx& cx, const KrylovBufs& kb, int nb, double tol) {
    k_norm_part<<<dim3(kb.nblk, nb), kRedThreads, 0, cx.stream>>>(kb.N, kb.V, kb.sVd(), kb.npart, kb.nblk);
    k_init_state<<<1, 256, 0, cx.stream>>>(nb, kb.nblk, tol, kb.npart, kb.sigma, kb.sigt, kb.g, kb.sS(), kb.st,
                                           kb.active);
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
    k_arnoldi_finish<<<nb, kFinThreads, finish_smem(j), cx.stream>>>(j, kb.maxit, kb.nblk, kb.npart, kb.h1, kb.h2,
                                                                     kb.H, kb.sH(), kb.cs, kb.sn, kb.g, kb.sigma,
                                                                     kb.sS(), kb.st, kb.active);
}

// Delayed CGS2 on the double-float basis (used with the complex64
// preconditioner, see k_dcgs_dot): the basis passes run on the FP32 pipes in
// double-float arithmetic (error-free FMA products, TwoSum accumulation); the
// Hessenberg column, norms and Givens update stay in FP64.  Wide remainders give
// the basis about 48 significant bits, so orthogonality and the Arnoldi relation
// hold far below any GMRES tolerance used here; narrow (bf16) remainders give it
// about 32 bits and move 12 instead of 16 bytes an entry, the caller's choice
// for loose tolerances.
static size_t dcgs_givens_smem(int j) {
    const size_t b = (size_t)(j + 1) * sizeof(double2) + (size_t)(j > 0 ? j - 1 : 0) * (sizeof(double2) + sizeof(double));
    allow_dynamic_smem((const void*)k_dcgs_givens, b);
    return b;
}

void launch_dcgs2_step(const Ctx& cx, const KrylovBufs& kb, int nb, int j, int last_only, cudaEvent_t* ev) {
    const int S = kb.maxit + 1, ps = kb.pstride();
    // entry pairs: the padded vector length and all strides are even
    const long long Np = (kb.N + 1) / 2, ldp = kb.ld / 2, sVp = kb.sV() / 2;
    float4* V32 = reinterpret_cast<float4*>(kb.V32);
    if (ev) cudaEventRecord(ev[0], cx.stream);
    k_dcgs_dot<kDotGroupDC><<<dim3(kb.nblk_dot, nb), kRedThreads, 0, cx.stream>>>(j, Np, ldp, ps, S, V32, sVp,
                                                                                 !last_only, kb.part, kb.sP(),
                                                                                 kb.st);
    if (ev) cudaEventRecord(ev[1], cx.stream);
    const dim3 rg(((2 * j + 2) * 32 + 255) / 256, nb);
    k_dcgs_reduce<false><<<rg, 256, 0, cx.stream>>>(j, kb.nblk_dot, ps, S, kb.part, kb.sP(), kb.sigma, kb.h2, kb.hn,
                                             kb.sS(), kb.sN(), kb.st);
    k_dcgs_coef<<<nb, kFinThreads, 0, cx.stream>>>(j, kb.maxit, last_only, kb.hn, kb.sN(), kb.h1, kb.h2, kb.H,
                                                   kb.sH(), kb.sigma, kb.sS(), kb.st, kb.active);
    // rotation and stop test of column j-1 beside the update pass (on the side stream when
    // there is one); the step's end waits for them
    const bool side = j > 0 && kb.side && kb.ev_c && kb.ev_g;
    if (j > 0) {
        cudaStream_t gs = cx.stream;
        if (side) {
            cudaEventRecord(kb.ev_c, cx.stream);
            cudaStreamWaitEvent(kb.side, kb.ev_c, 0);
            gs = kb.side;
        }
        k_dcgs_givens<<<nb, kFinThreads, dcgs_givens_smem(j), gs>>>(j, kb.maxit, last_only, kb.H, kb.sH(), kb.cs,
                                                                     kb.sn, kb.g, kb.sS(), kb.st, kb.active);
        if (side) cudaEventRecord(kb.ev_g, kb.side);
    }
    if (!last_only) {
        // narrow remainders: a copy ring of 3 stages (24 B per vector slot); wide remainders
        // (32 B per slot, where 3 stages would leave one block per SM): two groups in registers
        const int ns = kb.lo16 ? 3 : 0;
        const size_t slot_bytes = sizeof(ulonglong2) + sizeof(uint2);
        const size_t us = (size_t)(j > 0 ? j : 1) * sizeof(UpdCoef) + (size_t)ns * kUpdUnroll * kRedThreads * slot_bytes;
        // two blocks per SM when their shared memory fits (long runs fall back to one)
        const int bps = 2 * (us + 1024) <= (size_t)kSmemPerSM ? kUpdBlocksPerSM : 1;
        const int nupd = bps * cx.num_sms;                       // <= kb.nblk, the partials' stride
        const dim3 gu(nupd, nb);
        if (ev) cudaEventRecord(ev[2], cx.stream);
        if (kb.lo16) {
            set_coef_smem_limit((const void*)k_dcgs_update<uint2, 3>, us);
            k_dcgs_update<uint2, 3><<<gu, kRedThreads, us, cx.stream>>>(j, Np, ldp, V32,
                                                                        static_cast<uint2*>(kb.V32lo), sVp, kb.sigma,
                                                                        kb.h1, kb.h2, kb.sS(), kb.npart, kb.nblk,
                                                                        kb.st);
        } else {
            set_coef_smem_limit((const void*)k_dcgs_update<float4, 0>, us);
            k_dcgs_update<float4, 0><<<gu, kRedThreads, us, cx.stream>>>(j, Np, ldp, V32,
                                                                         static_cast<float4*>(kb.V32lo), sVp,
                                                                         kb.sigma, kb.h1, kb.h2, kb.sS(), kb.npart,
                                                                         kb.nblk, kb.st);
        }
        if (ev) cudaEventRecord(ev[3], cx.stream);
        k_dcgs_scale<<<nb, 32, 0, cx.stream>>>(j, nupd, kb.nblk, kb.npart, kb.sigt, kb.sS(), kb.st);
    }
    if (side) cudaStreamWaitEvent(cx.stream, kb.ev_g, 0);
}

// Delayed CGS2 on the FP64 basis kb.V (see k_d64_dot): the same step structure as
// launch_dcgs2_step (dot pass, reduction, coefficients, Givens rotation of column
// j-1 on the side stream beside the update pass, scale of the next preconditioner
// input); ev as there.
void launch_dcgs2_step64(const Ctx& cx, const KrylovBufs& kb, int nb, int j, int last_only, cudaEvent_t* ev) {
    const int S = kb.maxit + 1, ps = kb.pstride();
    if (ev) cudaEventRecord(ev[0], cx.stream);
    k_d64_dot<kDotGroup64><<<dim3(kb.nblk_dot, nb), kRedThreads, 0, cx.stream>>>(j, kb.N, kb.ld, ps, S, kb.V, kb.sV(),
                                                                                !last_only, kb.part, kb.sP(), kb.st);
    if (ev) cudaEventRecord(ev[1], cx.stream);
    const dim3 rg(((2 * j + 2) * 32 + 255) / 256, nb);
    k_dcgs_reduce<true><<<rg, 256, 0, cx.stream>>>(j, kb.nblk_dot, ps, S, kb.part, kb.sP(), kb.sigma, kb.h2, kb.hn,
                                                   kb.sS(), kb.sN(), kb.st);
    k_dcgs_coef<<<nb, kFinThreads, 0, cx.stream>>>(j, kb.maxit, last_only, kb.hn, kb.sN(), kb.h1, kb.h2, kb.H,
                                                   kb.sH(), kb.sigma, kb.sS(), kb.st, kb.active);
    const bool side = j > 0 && kb.side && kb.ev_c && kb.ev_g;
    if (j > 0) {
        cudaStream_t gs = cx.stream;
        if (side) {
            cudaEventRecord(kb.ev_c, cx.stream);
            cudaStreamWaitEvent(kb.side, kb.ev_c, 0);
            gs = kb.side;
        }
        k_dcgs_givens<<<nb, kFinThreads, dcgs_givens_smem(j), gs>>>(j, kb.maxit, last_only, kb.H, kb.sH(), kb.cs,
                                                                     kb.sn, kb.g, kb.sS(), kb.st, kb.active);
        if (side) cudaEventRecord(kb.ev_g, kb.side);
    }
    if (!last_only) {
        const size_t us = (size_t)(j > 0 ? j : 1) * sizeof(Upd64Coef);
        set_coef_smem_limit((const void*)k_d64_update, us);
        const dim3 gu(kb.nblk, nb);
        if (ev) cudaEventRecord(ev[2], cx.stream);
        k_d64_update<<<gu, kRedThreads, us, cx.stream>>>(j, kb.N, kb.ld, kb.V, kb.sV(), kb.sigma, kb.h1, kb.h2,
                                                         kb.sS(), kb.npart, kb.nblk, kb.st);
        if (ev) cudaEventRecord(ev[3], cx.stream);
        k_dcgs_scale<<<nb, 32, 0, cx.stream>>>(j, kb.nblk, kb.nblk, kb.npart, kb.sigt, kb.sS(), kb.st);
    }
    if (side) cudaStreamWaitEvent(cx.stream, kb.ev_g, 0);
}

// Delayed CGS2 on the f53 basis (heads kb.V32, tails kb.V32lo; see orth53.cu): the
// step structure of launch_dcgs2_step64 with the passes split between the FP64 and
// FP32 pipes (kb.dmask_dot, kb.dmask_upd: the vectors on the FP64 path).
// False (nothing launched after the failed pass) when the dot pass could not be
// launched or the update pass's coefficients do not fit in shared memory.
bool launch_dcgs2_step53(const Ctx& cx, const KrylovBufs& kb, int nb, int j, int last_only, cudaEvent_t* ev) {
    const int S = kb.maxit + 1, ps = kb.pstride();
    if (ev) cudaEventRecord(ev[0], cx.stream);
    const int ndot = launch_s53_dot(cx, kb, nb, j, !last_only, kb.dmask_dot);
    if (ev) cudaEventRecord(ev[1], cx.stream);
    if (ndot == 0) return false;
    const dim3 rg(((2 * j + 2) * 32 + 255) / 256, nb);
    k_dcgs_reduce<true><<<rg, 256, 0, cx.stream>>>(j, ndot, ps, S, kb.part, kb.sP(), kb.sigma, kb.h2, kb.hn,
                                                   kb.sS(), kb.sN(), kb.st);
    k_dcgs_coef<<<nb, kFinThreads, 0, cx.stream>>>(j, kb.maxit, last_only, kb.hn, kb.sN(), kb.h1, kb.h2, kb.H,
                                                   kb.sH(), kb.sigma, kb.sS(), kb.st, kb.active);
    const bool side = j > 0 && kb.side && kb.ev_c && kb.ev_g;
    if (j > 0) {
        cudaStream_t gs = cx.stream;
        if (side) {
            cudaEventRecord(kb.ev_c, cx.stream);
            cudaStreamWaitEvent(kb.side, kb.ev_c, 0);
            gs = kb.side;
        }
        k_dcgs_givens<<<nb, kFinThreads, dcgs_givens_smem(j), gs>>>(j, kb.maxit, last_only, kb.H, kb.sH(), kb.cs,
                                                                     kb.sn, kb.g, kb.sS(), kb.st, kb.active);
        if (side) cudaEventRecord(kb.ev_g, kb.side);
    }
    bool ok = true;
    if (!last_only) {
        if (ev) cudaEventRecord(ev[2], cx.stream);
        const int nupd = launch_s53_update(cx, kb, nb, j, kb.dmask_upd);
        if (ev) cudaEventRecord(ev[3], cx.stream);
        if (nupd > 0) k_dcgs_scale<<<nb, 32, 0, cx.stream>>>(j, nupd, kb.nblk, kb.npart, kb.sigt, kb.sS(), kb.st);
        ok = nupd > 0;
    }
    if (side) cudaStreamWaitEvent(cx.stream, kb.ev_g, 0);
    return ok;
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
