// Delayed CGS2 (Section 5's GMRES, Arnoldi step) on an FP64 Krylov basis whose
// arithmetic is spread over the FP64 and the FP32 pipes.
//
// The basis vectors, u~_j and w are FP64 vectors stored exactly as an FP32 head
// (the value with its fraction truncated to 23 bits) and a 29-bit integer tail
// (f53, see f32x2.cuh): 16 bytes a complex entry, as complex128.  The heads are a
// complex64 array of their own, so the complex64 preconditioner and the
// complex64 first-projection dot products read 8 bytes an entry, and the FP64
// value or its three FP32 pieces are rebuilt with a few integer operations.
//
// The step is the delayed CGS2 of launch_dcgs2_step64 (krylov.cu): the
// reorthogonalisation coefficients alpha = Q^H u~_j, the norm c = |u~_j|^2,
// d = u~_j^H w and the first-projection update w - Q b - h_jj q_j are computed
// to FP64 accuracy or better; the first-projection dot products b are complex64
// on the heads.  The part's FP64 pipe runs at 1/64 of its FP32 rate, so each
// pass splits the basis vectors between two arithmetic paths that run
// concurrently:
//   - FP64 fused multiply-adds on the rebuilt FP64 values (the vectors i whose bit
//     i % 8 is set in a mask), interleaved in every warp with
//   - FP32 error-free arithmetic on the three FP32 pieces of each value
//     (head + 23 + 6 bits): products split exactly by FMAs (TwoProd) and summed
//     in three-word expansions (TwoSum at the two upper levels), every rounding
//     that is not carried below 2^-69 of the partial sums, so the error bound is
//     tighter than that of the FP64 operations it replaces.
// The reorthogonalisation update u~_j - Q alpha sums terms of order 2^-24 |u~_j|
// (what the complex64 first projection left) and runs in double-float on the
// FP32 pipes for every vector; its error is about 2^-46 of those terms.
#include <algorithm>

#include "f32x2.cuh"
#include "kernels.cuh"

namespace hzs {

constexpr int kS53Threads = 256;
constexpr int kS53Group = 2;            // basis vectors per warp task (dot pass) and per group (update)

// per-thread asynchronous 8-byte copies global -> shared (read back by the same thread
// after cp.async.wait_group, so no block barrier is involved)
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void chunk_of53(long long N, long long& e0, long long& e1) {
    const long long per = (N + gridDim.x - 1) / gridDim.x;
    e0 = (long long)blockIdx.x * per;
    e1 = e0 + per < N ? e0 + per : N;
}

__device__ __forceinline__ double2 f53_load(const float2* __restrict__ h, const uint2* __restrict__ t, long long e) {
    const float2 a = h[e];
    const uint2 b = t[e];
    return make_double2(f53_double(a.x, b.x), f53_double(a.y, b.y));
}
__device__ __forceinline__ void f53_store(float2* __restrict__ h, uint2* __restrict__ t, long long e, double2 v) {
    float2 a;
    uint2 b;
    f53_encode(v.x, a.x, b.x);
    f53_encode(v.y, a.y, b.y);
    h[e] = a;
    t[e] = b;
}

// dst_r = scale_r * src_r (scale a power of two, or 1 without scale) stored as f53,
// entries 0 .. N-1 of batch entry r = blockIdx.y.
__global__ void k_f53_encode(long long N, const double2* __restrict__ src, long long ss, float2* __restrict__ dh,
                             uint2* __restrict__ dt, long long ds, const double* __restrict__ scale,
                             const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (st && st[r].done) return;
    src += r * ss; dh += r * ds; dt += r * ds;
    const double s = scale ? scale[r] : 1.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x)
        f53_store(dh, dt, e, cscale(src[e], s));
}

// The stored right-hand side V_0 is scaled by the power of two nearest to 1/|f|,
// so that its entries lie in the range of the f53 form whatever the scale of f;
// sigma_0 and the preconditioner's input scale absorb the factor: scale[r] = 2^k,
// sigma_0 <- sigma_0 / 2^k.
__global__ void k_f53_scale0(int nb, double* __restrict__ sigma, double* __restrict__ sigt, long long sS,
                             double* __restrict__ scale) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nb) return;
    const double s0 = sigma[r * sS];
    double sc = 1.0;
    if (s0 > 0.0 && isfinite(s0)) {
        int ex;
        frexp(s0, &ex);
        sc = ldexp(1.0, ex - 1);
    }
    scale[r] = sc;
    sigma[r * sS] = s0 / sc;
    sigt[r * sS] = s0 / sc;
}

// Dot pass of step j (entry r = blockIdx.y; slot j holds u~_j, slot j+1 w; heads Vh,
// tails Vt).  Warp tasks of kS53Group basis vectors, each vector i summed with FP64 FMAs
// when bit i % 8 of dmask is set, else in FP32 three-word expansions; the last task
// computes c and d.
// Partials per block as in k_d64_dot: alpha at [0, S) (FP64), b at [S, 2S) (FP32 words),
// c at 2S, d at 2S+1 (FP64).
// NS > 0: the basis vectors' and u~'s entries and w's heads stream through a per-thread
// ring of NS stages in shared memory (cp.async; each thread reads back only what it
// copied itself), NS - 1 entries ahead of the one being summed; NS == 0 loads them
// into registers where they are used.
template <int MINB, int NS, int G>
__global__ void __launch_bounds__(kS53Threads, MINB) k_s53_dot(int j, long long N, long long ld, int ps, int S,
                                                           const float2* __restrict__ Vh, const uint2* __restrict__ Vt,
                                                           long long sV, int has_w, unsigned dmask,
                                                           double2* __restrict__ part, long long sP,
                                                           const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (st[r].done) return;
    Vh += r * sV; Vt += r * sV;
    const float2* uh = Vh + (size_t)j * ld;
    const uint2* ut = Vt + (size_t)j * ld;
    const float2* wh = Vh + (size_t)(has_w ? j + 1 : j) * ld;
    const uint2* wt = Vt + (size_t)(has_w ? j + 1 : j) * ld;
    part += r * sP + (size_t)blockIdx.x * ps;
    extern __shared__ uint2 s53ring[];              // NS x (2G + 3) x kS53Threads 8-byte slots
    long long e0, e1;
    chunk_of53(N, e0, e1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ngroups = (j + G - 1) / G;
    for (int gi = warp; gi <= ngroups; gi += nw) {
        const int i0 = gi * G;
        double2 al[G];
        f2x B1[G], B2[G];                       // b = conj(head v) . head w as (wr x V0, wi x V0) sums
#pragma unroll
        for (int t = 0; t < G; ++t) { al[t] = make_double2(0.0, 0.0); B1[t] = B2[t] = 0ull; }
        if (gi == ngroups) {
            // c = |u~|^2 and d = u~^H w in FP64
            double c = 0.0;
            double2 d = make_double2(0.0, 0.0);
            for (long long e = e0 + lane; e < e1; e += 32) {
                const double2 x = f53_load(uh, ut, e);
                c = fma(x.x, x.x, fma(x.y, x.y, c));
                if (has_w) d = cfma_conj(x, f53_load(wh, wt, e), d);
            }
            c = warp_sum_d(c);
            d = warp_sum(d);
            if (lane == 0) {
                part[2 * S] = make_double2(c, 0.0);
                part[2 * S + 1] = d;
            }
            continue;
        }
        // vector i0 + t on the FP64 path when bit (i0 + t) % 8 of dmask is set, else in FP32
        // three-word expansions: alpha = sum_e conj(v) u~ = (P.x + R.y, R.x - P.y) with
        // P = sum_e ur (vr, vi), R = sum_e ui (vr, vi); the two paths interleave in every
        // warp, so that the FP64 and FP32 pipes work at once
        bool d64[G];
        TF2 P[G], R[G];
#pragma unroll
        for (int t = 0; t < G; ++t) {
            d64[t] = (dmask >> ((i0 + t) & 7)) & 1;
            tf_zero(P[t]);
            tf_zero(R[t]);
        }
        int cnt = 0;
        // ring slots: items 0 .. G-1 heads and G .. 2G-1 tails of the vectors, 2G and 2G+1
        // head and tail of u~, 2G+2 head of w
        constexpr int IT = 2 * G + 3;
        auto slot = [&](int stage, int item) { return s53ring + ((stage * IT + item) * kS53Threads + threadIdx.x); };
        const long long K = e1 - e0 - lane > 0 ? (e1 - e0 - lane + 31) / 32 : 0;
        auto issue = [&](long long k, int stage) {
            const long long e = e0 + lane + 32 * k;
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (i0 + t < j) {
                    cp_async_8(slot(stage, t), Vh + (size_t)(i0 + t) * ld + e);
                    cp_async_8(slot(stage, G + t), Vt + (size_t)(i0 + t) * ld + e);
                }
            cp_async_8(slot(stage, 2 * G), uh + e);
            cp_async_8(slot(stage, 2 * G + 1), ut + e);
            if (has_w) cp_async_8(slot(stage, 2 * G + 2), wh + e);
        };
        if constexpr (NS > 0) {
#pragma unroll
            for (int s0 = 0; s0 < NS - 1; ++s0) {
                if (s0 < K) issue(s0, s0);
                cp_async_commit();
            }
        }
        int cs = 0;                                     // stage of entry k
        for (long long k = 0; k < K; ++k) {
            const long long e = e0 + lane + 32 * k;
            float2 xh, yh;
            uint2 xt;
            float2 vh[G];
            uint2 vt[G];
            if constexpr (NS > 0) {
                const int is = cs == 0 ? NS - 1 : cs - 1;   // stage of entry k + NS - 1 (read at k - 1)
                if (k + NS - 1 < K) issue(k + NS - 1, is);
                cp_async_commit();
                cp_async_wait<NS - 1>();                    // entry k has landed
                const uint2 a = *slot(cs, 2 * G), c = *slot(cs, 2 * G + 2);
                xh = make_float2(__uint_as_float(a.x), __uint_as_float(a.y));
                xt = *slot(cs, 2 * G + 1);
                yh = has_w ? make_float2(__uint_as_float(c.x), __uint_as_float(c.y)) : make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < G; ++t) {
                    const bool in = i0 + t < j;
                    const uint2 h = *slot(cs, t);
                    vh[t] = in ? make_float2(__uint_as_float(h.x), __uint_as_float(h.y)) : make_float2(0.f, 0.f);
                    vt[t] = in ? *slot(cs, G + t) : make_uint2(0u, 0u);
                }
                cs = cs + 1 == NS ? 0 : cs + 1;
            } else {
                xh = __ldg(uh + e);
                xt = __ldg(ut + e);
                yh = has_w ? __ldg(wh + e) : make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < G; ++t) {
                    const bool in = i0 + t < j;
                    vh[t] = in ? __ldcs(Vh + (size_t)(i0 + t) * ld + e) : make_float2(0.f, 0.f);
                    vt[t] = in ? __ldcs(Vt + (size_t)(i0 + t) * ld + e) : make_uint2(0u, 0u);
                }
            }
            const double2 x = make_double2(f53_double(xh.x, xt.x), f53_double(xh.y, xt.y));
            float ur1, ur2, ui1, ui2;
            f53_low(xh.x, xt.x, ur1, ur2);
            f53_low(xh.y, xt.y, ui1, ui2);
            const f2x Ur0 = f2_bcast(xh.x), NUr0 = f2_bcast(-xh.x), Ur1 = f2_bcast(ur1), NUr1 = f2_bcast(-ur1),
                      Ur2 = f2_bcast(ur2);
            const f2x Ui0 = f2_bcast(xh.y), NUi0 = f2_bcast(-xh.y), Ui1 = f2_bcast(ui1), NUi1 = f2_bcast(-ui1),
                      Ui2 = f2_bcast(ui2);
            const f2x Wr = f2_bcast(yh.x), Wi = f2_bcast(yh.y);
#pragma unroll
            for (int t = 0; t < G; ++t) {
                const f2x V0 = f2_of(vh[t]);
                if (d64[t]) {
                    const double2 v = make_double2(f53_double(vh[t].x, vt[t].x), f53_double(vh[t].y, vt[t].y));
                    al[t] = cfma_conj(v, x, al[t]);
                } else {
                    f2x V1, V2;
                    f53_low2(vh[t], vt[t], V1, V2);
                    tf_mac53(P[t], Ur0, Ur1, Ur2, NUr0, NUr1, V0, V1, V2);
                    tf_mac53(R[t], Ui0, Ui1, Ui2, NUi0, NUi1, V0, V1, V2);
                }
                B1[t] = fma2(Wr, V0, B1[t]);
                B2[t] = fma2(Wi, V0, B2[t]);
            }
            if ((++cnt & 3) == 0) {
#pragma unroll
                for (int t = 0; t < G; ++t)
                    if (!d64[t]) { tf_renorm(P[t]); tf_renorm(R[t]); }
            }
        }
        if constexpr (NS > 0) cp_async_wait<0>();      // (only empty groups remain) the slots are free
#pragma unroll
        for (int t = 0; t < G; ++t)
            if (!d64[t])
                al[t] = make_double2(tf_lane(P[t], 0) + tf_lane(R[t], 1), tf_lane(R[t], 0) - tf_lane(P[t], 1));
#pragma unroll
        for (int t = 0; t < G; ++t) {
            al[t] = warp_sum(al[t]);
            const float2 b1 = f2_unpack(B1[t]), b2 = f2_unpack(B2[t]);
            float2 b = make_float2(b1.x + b2.y, b2.x - b1.y);
            b = warp_sum(b);
            if (lane == 0 && i0 + t < j) {
                part[i0 + t] = al[t];
                reinterpret_cast<float4*>(part)[S + i0 + t] = make_float4(b.x, b.y, 0.f, 0.f);
            }
        }
    }
}

// The i-th of the basis vectors 0 .. j-1 whose index mod 8 is a set bit of mask
// (pos: the set bits in increasing order, pop of them).
__device__ __forceinline__ int s53_vec(int m, const int* pos, int pop) { return (m / pop) * 8 + pos[m % pop]; }
__device__ __forceinline__ int s53_count(int j, unsigned mask) {
    return (j >> 3) * __popc(mask) + __popc(mask & ((1u << (j & 7)) - 1u));
}

// Dot pass of step j with specialised warps: the same sums as k_s53_dot, but a warp task
// holds either G64 vectors of the FP64 path or G32 vectors of the FP32 path, so that a
// warp on the FP32 path never waits on an FP64 result (the two paths of k_s53_dot share
// each warp's iterations).  Tasks are ordered so that the two kinds alternate in
// proportion and are taken by the warps of a block from a shared counter, so the FP64
// pipe and the FP32 pipes are fed by different warps at the same time.  The FP32 path's
// entries stream through a per-thread shared-memory ring of NS stages (cp.async).
template <int MINB, int G64, int G32, int NS, bool R64>
__global__ void __launch_bounds__(kS53Threads, MINB) k_s53_dot_ws(int j, long long N, long long ld, int ps, int S,
                                                              const float2* __restrict__ Vh,
                                                              const uint2* __restrict__ Vt, long long sV, int has_w,
                                                              unsigned dmask, double2* __restrict__ part,
                                                              long long sP, const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (st[r].done) return;
    Vh += r * sV; Vt += r * sV;
    const float2* uh = Vh + (size_t)j * ld;
    const uint2* ut = Vt + (size_t)j * ld;
    const float2* wh = Vh + (size_t)(has_w ? j + 1 : j) * ld;
    part += r * sP + (size_t)blockIdx.x * ps;
    // NS x IT x kS53Threads 8-byte slots, IT = 2 G + 3 for the larger task that uses the ring
    extern __shared__ uint2 s53ring[];
    constexpr int IT = 2 * (R64 && G64 > G32 ? G64 : G32) + 3;
    auto slot = [&](int stage, int item) { return s53ring + ((stage * IT + item) * kS53Threads + threadIdx.x); };
    __shared__ int s_next;
    long long e0, e1;
    chunk_of53(N, e0, e1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned m64 = dmask & 0xffu, m32 = ~dmask & 0xffu;
    int pos64[8], pos32[8], pop64 = 0, pop32 = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if ((m64 >> b) & 1u) pos64[pop64++] = b;
        else pos32[pop32++] = b;
    }
    const int n64 = s53_count(j, m64), n32 = j - n64;
    const int T64 = (n64 + G64 - 1) / G64, T32 = (n32 + G32 - 1) / G32, T = T64 + T32;
    if (threadIdx.x == 0) s_next = nw;
    __syncthreads();
    const long long K = e1 - e0 - lane > 0 ? (e1 - e0 - lane + 31) / 32 : 0;
    int gi = warp;
    while (gi <= T) {
        if (gi == T) {
            // c = |u~|^2 and d = u~^H w in FP64
            double c = 0.0;
            double2 d = make_double2(0.0, 0.0);
            for (long long e = e0 + lane; e < e1; e += 32) {
                const double2 x = f53_load(uh, ut, e);
                c = fma(x.x, x.x, fma(x.y, x.y, c));
                if (has_w) d = cfma_conj(x, f53_load(wh, Vt + (size_t)(j + 1) * ld, e), d);
            }
            c = warp_sum_d(c);
            d = warp_sum(d);
            if (lane == 0) {
                part[2 * S] = make_double2(c, 0.0);
                part[2 * S + 1] = d;
            }
        } else {
            // task gi is FP64 task a when the interleave steps at gi, else FP32 task gi - a
            const int a = (int)((long long)gi * T64 / T), a1 = (int)((long long)(gi + 1) * T64 / T);
            if (a1 > a) {
                int vi[G64];
                double2 al[G64];
                f2x B1[G64], B2[G64];
#pragma unroll
                for (int t = 0; t < G64; ++t) {
                    const int m = a * G64 + t;
                    vi[t] = m < n64 ? s53_vec(m, pos64, pop64) : -1;
                    al[t] = make_double2(0.0, 0.0);
                    B1[t] = B2[t] = 0ull;
                }
                auto issue64 = [&](long long k, int stage) {
                    const long long e = e0 + lane + 32 * k;
#pragma unroll
                    for (int t = 0; t < G64; ++t)
                        if (vi[t] >= 0) {
                            cp_async_8(slot(stage, t), Vh + (size_t)vi[t] * ld + e);
                            cp_async_8(slot(stage, G64 + t), Vt + (size_t)vi[t] * ld + e);
                        }
                    cp_async_8(slot(stage, 2 * G64), uh + e);
                    cp_async_8(slot(stage, 2 * G64 + 1), ut + e);
                    if (has_w) cp_async_8(slot(stage, 2 * G64 + 2), wh + e);
                };
                if constexpr (R64) {
#pragma unroll
                    for (int s0 = 0; s0 < NS - 1; ++s0) {
                        if (s0 < K) issue64(s0, s0);
                        cp_async_commit();
                    }
                }
                int cs = 0;
                for (long long k = 0; k < K; ++k) {
                    const long long e = e0 + lane + 32 * k;
                    float2 xh, yh;
                    uint2 xt;
                    float2 vh[G64];
                    uint2 vt[G64];
                    if constexpr (R64) {
                        const int is = cs == 0 ? NS - 1 : cs - 1;   // stage of entry k + NS - 1 (read at k - 1)
                        if (k + NS - 1 < K) issue64(k + NS - 1, is);
                        cp_async_commit();
                        cp_async_wait<NS - 1>();                    // entry k has landed
                        const uint2 xa = *slot(cs, 2 * G64), ya = *slot(cs, 2 * G64 + 2);
                        xh = make_float2(__uint_as_float(xa.x), __uint_as_float(xa.y));
                        xt = *slot(cs, 2 * G64 + 1);
                        yh = has_w ? make_float2(__uint_as_float(ya.x), __uint_as_float(ya.y)) : make_float2(0.f, 0.f);
#pragma unroll
                        for (int t = 0; t < G64; ++t) {
                            const uint2 h = *slot(cs, t);
                            vh[t] = vi[t] >= 0 ? make_float2(__uint_as_float(h.x), __uint_as_float(h.y))
                                               : make_float2(0.f, 0.f);
                            vt[t] = vi[t] >= 0 ? *slot(cs, G64 + t) : make_uint2(0u, 0u);
                        }
                        cs = cs + 1 == NS ? 0 : cs + 1;
                    } else {
                        xh = __ldg(uh + e);
                        xt = __ldg(ut + e);
                        yh = has_w ? __ldg(wh + e) : make_float2(0.f, 0.f);
#pragma unroll
                        for (int t = 0; t < G64; ++t) {
                            vh[t] = vi[t] >= 0 ? __ldcs(Vh + (size_t)vi[t] * ld + e) : make_float2(0.f, 0.f);
                            vt[t] = vi[t] >= 0 ? __ldcs(Vt + (size_t)vi[t] * ld + e) : make_uint2(0u, 0u);
                        }
                    }
                    const double2 x = make_double2(f53_double(xh.x, xt.x), f53_double(xh.y, xt.y));
                    const f2x Wr = f2_bcast(yh.x), Wi = f2_bcast(yh.y);
#pragma unroll
                    for (int t = 0; t < G64; ++t) {
                        const double2 v = make_double2(f53_double(vh[t].x, vt[t].x), f53_double(vh[t].y, vt[t].y));
                        al[t] = cfma_conj(v, x, al[t]);
                        const f2x V0 = f2_of(vh[t]);
                        B1[t] = fma2(Wr, V0, B1[t]);
                        B2[t] = fma2(Wi, V0, B2[t]);
                    }
                }
                if constexpr (R64) cp_async_wait<0>();          // (only empty groups remain) the slots are free
#pragma unroll
                for (int t = 0; t < G64; ++t) {
                    const double2 sa = warp_sum(al[t]);
                    const float2 b1 = f2_unpack(B1[t]), b2 = f2_unpack(B2[t]);
                    const float2 b = warp_sum(make_float2(b1.x + b2.y, b2.x - b1.y));
                    if (lane == 0 && vi[t] >= 0) {
                        part[vi[t]] = sa;
                        reinterpret_cast<float4*>(part)[S + vi[t]] = make_float4(b.x, b.y, 0.f, 0.f);
                    }
                }
            } else {
                const int q = gi - a;
                int vi[G32];
                TF2 P[G32], R[G32];
                f2x B1[G32], B2[G32];
#pragma unroll
                for (int t = 0; t < G32; ++t) {
                    const int m = q * G32 + t;
                    vi[t] = m < n32 ? s53_vec(m, pos32, pop32) : -1;
                    tf_zero(P[t]);
                    tf_zero(R[t]);
                    B1[t] = B2[t] = 0ull;
                }
                auto issue = [&](long long k, int stage) {
                    const long long e = e0 + lane + 32 * k;
#pragma unroll
                    for (int t = 0; t < G32; ++t)
                        if (vi[t] >= 0) {
                            cp_async_8(slot(stage, t), Vh + (size_t)vi[t] * ld + e);
                            cp_async_8(slot(stage, G32 + t), Vt + (size_t)vi[t] * ld + e);
                        }
                    cp_async_8(slot(stage, 2 * G32), uh + e);
                    cp_async_8(slot(stage, 2 * G32 + 1), ut + e);
                    if (has_w) cp_async_8(slot(stage, 2 * G32 + 2), wh + e);
                };
#pragma unroll
                for (int s0 = 0; s0 < NS - 1; ++s0) {
                    if (s0 < K) issue(s0, s0);
                    cp_async_commit();
                }
                int cs = 0, cnt = 0;
                for (long long k = 0; k < K; ++k) {
                    const int is = cs == 0 ? NS - 1 : cs - 1;   // stage of entry k + NS - 1 (read at k - 1)
                    if (k + NS - 1 < K) issue(k + NS - 1, is);
                    cp_async_commit();
                    cp_async_wait<NS - 1>();                    // entry k has landed
                    const uint2 xa = *slot(cs, 2 * G32), ya = *slot(cs, 2 * G32 + 2);
                    const float2 xh = make_float2(__uint_as_float(xa.x), __uint_as_float(xa.y));
                    const uint2 xt = *slot(cs, 2 * G32 + 1);
                    const float2 yh = has_w ? make_float2(__uint_as_float(ya.x), __uint_as_float(ya.y))
                                            : make_float2(0.f, 0.f);
                    float ur1, ur2, ui1, ui2;
                    f53_low(xh.x, xt.x, ur1, ur2);
                    f53_low(xh.y, xt.y, ui1, ui2);
                    const f2x Ur0 = f2_bcast(xh.x), NUr0 = f2_bcast(-xh.x), Ur1 = f2_bcast(ur1), NUr1 = f2_bcast(-ur1),
                              Ur2 = f2_bcast(ur2);
                    const f2x Ui0 = f2_bcast(xh.y), NUi0 = f2_bcast(-xh.y), Ui1 = f2_bcast(ui1), NUi1 = f2_bcast(-ui1),
                              Ui2 = f2_bcast(ui2);
                    const f2x Wr = f2_bcast(yh.x), Wi = f2_bcast(yh.y);
#pragma unroll
                    for (int t = 0; t < G32; ++t) {
                        const uint2 h = *slot(cs, t);
                        const float2 vh = vi[t] >= 0 ? make_float2(__uint_as_float(h.x), __uint_as_float(h.y))
                                                     : make_float2(0.f, 0.f);
                        const uint2 vt = vi[t] >= 0 ? *slot(cs, G32 + t) : make_uint2(0u, 0u);
                        const f2x V0 = f2_of(vh);
                        f2x V1, V2;
                        f53_low2(vh, vt, V1, V2);
                        tf_mac53(P[t], Ur0, Ur1, Ur2, NUr0, NUr1, V0, V1, V2);
                        tf_mac53(R[t], Ui0, Ui1, Ui2, NUi0, NUi1, V0, V1, V2);
                        B1[t] = fma2(Wr, V0, B1[t]);
                        B2[t] = fma2(Wi, V0, B2[t]);
                    }
                    if ((++cnt & 3) == 0) {
#pragma unroll
                        for (int t = 0; t < G32; ++t) { tf_renorm(P[t]); tf_renorm(R[t]); }
                    }
                    cs = cs + 1 == NS ? 0 : cs + 1;
                }
                cp_async_wait<0>();                             // (only empty groups remain) the slots are free
#pragma unroll
                for (int t = 0; t < G32; ++t) {
                    double2 al = make_double2(tf_lane(P[t], 0) + tf_lane(R[t], 1), tf_lane(R[t], 0) - tf_lane(P[t], 1));
                    al = warp_sum(al);
                    const float2 b1 = f2_unpack(B1[t]), b2 = f2_unpack(B2[t]);
                    const float2 b = warp_sum(make_float2(b1.x + b2.y, b2.x - b1.y));
                    if (lane == 0 && vi[t] >= 0) {
                        part[vi[t]] = al;
                        reinterpret_cast<float4*>(part)[S + vi[t]] = make_float4(b.x, b.y, 0.f, 0.f);
                    }
                }
            }
        }
        int nx = 0;
        if (lane == 0) nx = atomicAdd(&s_next, 1);
        gi = __shfl_sync(0xffffffffu, nx, 0);
    }
}

// Coefficients of basis vector i for the update pass: c = sigma_i h1_i (an FP32
// value, see k_dcgs_coef) as broadcast pairs and as FP64, and the
// reorthogonalisation coefficient a = sigma_i alpha_i as double-float broadcast pairs.
struct alignas(16) S53Coef {
    f2x Pcr, Ncr, Pci, Nci;
    f2x Parh, Narh, Narl, Paih, Naih, Nail;
    double2 c;
};

// Update pass of step j (one entry per thread and sweep): V_j = u~_j - sum_i a_i V_i,
// w <- w - sum_i c_i V_i - (h_jj sigma_j) V_j, npart[b] = sum_e |w[e]|^2 (FP64).
// sum_i c_i V_i: vector i with FP64 FMAs when bit i % 8 of dmask is set, else in
// three-word expansions A = sum cr (vr, vi),
// B = sum ci (vr, vi) (c V = (A.x - B.y, A.y + B.x)); sum_i a_i V_i in double-float
// for every vector.  The final sums and both results are FP64.
template <int MINB>
__global__ void __launch_bounds__(kS53Threads, MINB) k_s53_update(int j, long long N, long long ld,
                                                              float2* __restrict__ Vh, uint2* __restrict__ Vt,
                                                              long long sV, const double* __restrict__ sigma,
                                                              const double2* __restrict__ h1,
                                                              const double2* __restrict__ h2, long long sS,
                                                              unsigned dmask,
                                                              double* __restrict__ npart, int nblk,
                                                              const KState* __restrict__ st) {
    constexpr int G = kS53Group;
    const int r = blockIdx.y;
    if (st[r].done) return;
    Vh += r * sV; Vt += r * sV; sigma += r * sS; h1 += r * sS; h2 += r * sS;
    float2* uh = Vh + (size_t)j * ld;
    uint2* ut = Vt + (size_t)j * ld;
    float2* wh = Vh + (size_t)(j + 1) * ld;
    uint2* wt = Vt + (size_t)(j + 1) * ld;
    extern __shared__ S53Coef s53c[];
    __shared__ double2 s_cj;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const double2 c = cscale(h1[i], sigma[i]);
        if (i == j) { s_cj = c; continue; }
        const double2 a = cscale(h2[i], sigma[i]);
        const float cr = (float)c.x, ci = (float)c.y;          // exact: c is an FP32 value
        const float arh = (float)a.x, arl = (float)(a.x - (double)arh);
        const float aih = (float)a.y, ail = (float)(a.y - (double)aih);
        S53Coef k;
        k.Pcr = f2_bcast(cr); k.Ncr = f2_bcast(-cr); k.Pci = f2_bcast(ci); k.Nci = f2_bcast(-ci);
        k.Parh = f2_bcast(arh); k.Narh = f2_bcast(-arh); k.Narl = f2_bcast(-arl);
        k.Paih = f2_bcast(aih); k.Naih = f2_bcast(-aih); k.Nail = f2_bcast(-ail);
        k.c = make_double2((double)cr, (double)ci);
        s53c[i] = k;
    }
    __syncthreads();
    const double2 cj = s_cj;
    long long e0, e1;
    chunk_of53(N, e0, e1);
    double nrm = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        TF2 A, B;
        tf_zero(A);
        tf_zero(B);
        double2 acc = make_double2(0.0, 0.0);
        f2x rah = 0ull, ral = 0ull, rbh = 0ull, rbl = 0ull;   // sum a (vr, vi): re part ar, im part ai
        // one basis vector, index i, on the FP64 (d64) or the FP32 path
        auto vec = [&](int i, float2 vh, uint2 vt, bool d64) {
            const S53Coef& k = s53c[i];
            f2x V1, V2;
            f53_low2(vh, vt, V1, V2);
            const f2x V0 = f2_of(vh);
            if (d64) {
                const double2 v = make_double2(f53_double(vh.x, vt.x), f53_double(vh.y, vt.y));
                acc = cfma(k.c, v, acc);
            } else {
                tf_mac24(A, k.Pcr, k.Ncr, V0, V1, V2);
                tf_mac24(B, k.Pci, k.Nci, V0, V1, V2);
            }
            df_mac2(rah, ral, k.Parh, k.Narh, k.Narl, V0, V1);
            df_mac2(rbh, rbl, k.Paih, k.Naih, k.Nail, V0, V1);
        };
        // vectors j-1 .. 0 in groups of G (the dot pass read 0 .. j-1, so those still in
        // L2 come first); the loads of the next group are issued before this one is used
        int i = j - 1, g = 0;
        float2 ch[G], nh[G];
        uint2 ct[G], nt[G];
        auto load = [&](int i0, float2* hh, uint2* tt) {
#pragma unroll
            for (int t = 0; t < G; ++t) {
                const bool in = i0 - t >= 0;
                hh[t] = in ? __ldcs(Vh + (size_t)(i0 - t) * ld + e) : make_float2(0.f, 0.f);
                tt[t] = in ? __ldcs(Vt + (size_t)(i0 - t) * ld + e) : make_uint2(0u, 0u);
            }
        };
        if (i >= 0) load(i, ch, ct);
        for (; i >= 0; i -= G, ++g) {
            if (i - G >= 0) load(i - G, nh, nt);
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (i - t >= 0) vec(i - t, ch[t], ct[t], (dmask >> ((i - t) & 7)) & 1);
            if ((g & 1) == 1) {
                tf_renorm(A);
                tf_renorm(B);
                df_norm2(rah, ral);
                df_norm2(rbh, rbl);
            }
#pragma unroll
            for (int t = 0; t < G; ++t) { ch[t] = nh[t]; ct[t] = nt[t]; }
        }
        // sum c_i V_i and sum a_i V_i in FP64
        const double2 s = make_double2(acc.x + (tf_lane(A, 0) - tf_lane(B, 1)), acc.y + (tf_lane(A, 1) + tf_lane(B, 0)));
        const float2 pah = f2_unpack(rah), pal = f2_unpack(ral), pbh = f2_unpack(rbh), pbl = f2_unpack(rbl);
        const double rre = (f53_double(pah.x, 0u) + f53_double(pal.x, 0u)) - (f53_double(pbh.y, 0u) + f53_double(pbl.y, 0u));
        const double rim = (f53_double(pah.y, 0u) + f53_double(pal.y, 0u)) + (f53_double(pbh.x, 0u) + f53_double(pbl.x, 0u));
        // V_j = u~ - sum a_i V_i
        double2 x = f53_load(uh, ut, e);
        x.x -= rre;
        x.y -= rim;
        f53_store(uh, ut, e, x);
        // w - sum c_i V_i - c_j V_j
        double2 y = csub(f53_load(wh, wt, e), s);
        y = cfms(cj, x, y);
        f53_store(wh, wt, e, y);
        nrm = fma(y.x, y.x, fma(y.y, y.y, nrm));
    }
    __shared__ double nred[kS53Threads / 32];
    nrm = warp_sum_d(nrm);
    if ((threadIdx.x & 31) == 0) nred[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += nred[k];
        npart[(size_t)r * nblk + blockIdx.x] = t;
    }
}

// The update pass with two entries per thread and sweep (e and e + blockDim.x): each
// vector's coefficients are read from shared memory once for both entries, and the
// two entries' sums are independent chains of arithmetic.
template <int MINB>
__global__ void __launch_bounds__(kS53Threads, MINB) k_s53_update2(int j, long long N, long long ld,
                                                               float2* __restrict__ Vh, uint2* __restrict__ Vt,
                                                               long long sV, const double* __restrict__ sigma,
                                                               const double2* __restrict__ h1,
                                                               const double2* __restrict__ h2, long long sS,
                                                               unsigned dmask, double* __restrict__ npart, int nblk,
                                                               const KState* __restrict__ st) {
    constexpr int G = kS53Group;
    const int r = blockIdx.y;
    if (st[r].done) return;
    Vh += r * sV; Vt += r * sV; sigma += r * sS; h1 += r * sS; h2 += r * sS;
    float2* uh = Vh + (size_t)j * ld;
    uint2* ut = Vt + (size_t)j * ld;
    float2* wh = Vh + (size_t)(j + 1) * ld;
    uint2* wt = Vt + (size_t)(j + 1) * ld;
    extern __shared__ S53Coef s53c[];
    __shared__ double2 s_cj;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const double2 c = cscale(h1[i], sigma[i]);
        if (i == j) { s_cj = c; continue; }
        const double2 a = cscale(h2[i], sigma[i]);
        const float cr = (float)c.x, ci = (float)c.y;          // exact: c is an FP32 value
        const float arh = (float)a.x, arl = (float)(a.x - (double)arh);
        const float aih = (float)a.y, ail = (float)(a.y - (double)aih);
        S53Coef k;
        k.Pcr = f2_bcast(cr); k.Ncr = f2_bcast(-cr); k.Pci = f2_bcast(ci); k.Nci = f2_bcast(-ci);
        k.Parh = f2_bcast(arh); k.Narh = f2_bcast(-arh); k.Narl = f2_bcast(-arl);
        k.Paih = f2_bcast(aih); k.Naih = f2_bcast(-aih); k.Nail = f2_bcast(-ail);
        k.c = make_double2((double)cr, (double)ci);
        s53c[i] = k;
    }
    __syncthreads();
    const double2 cj = s_cj;
    long long e0, e1;
    chunk_of53(N, e0, e1);
    const long long bd = blockDim.x;
    double nrm = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += 2 * bd) {
        const long long ee[2] = {e, e + bd};
        const bool in1 = e + bd < e1;
        TF2 A[2], B[2];
        double2 acc[2];
        f2x rah[2], ral[2], rbh[2], rbl[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            tf_zero(A[q]);
            tf_zero(B[q]);
            acc[q] = make_double2(0.0, 0.0);
            rah[q] = ral[q] = rbh[q] = rbl[q] = 0ull;
        }
        auto vec = [&](int i, const float2* vh, const uint2* vt, bool d64) {
            const S53Coef& k = s53c[i];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                f2x V1, V2;
                f53_low2(vh[q], vt[q], V1, V2);
                const f2x V0 = f2_of(vh[q]);
                if (d64) {
                    const double2 v = make_double2(f53_double(vh[q].x, vt[q].x), f53_double(vh[q].y, vt[q].y));
                    acc[q] = cfma(k.c, v, acc[q]);
                } else {
                    tf_mac24(A[q], k.Pcr, k.Ncr, V0, V1, V2);
                    tf_mac24(B[q], k.Pci, k.Nci, V0, V1, V2);
                }
                df_mac2(rah[q], ral[q], k.Parh, k.Narh, k.Narl, V0, V1);
                df_mac2(rbh[q], rbl[q], k.Paih, k.Naih, k.Nail, V0, V1);
            }
        };
        int i = j - 1, g = 0;
        float2 ch[G][2], nh[G][2];
        uint2 ct[G][2], nt[G][2];
        auto load = [&](int i0, float2 (*hh)[2], uint2 (*tt)[2]) {
#pragma unroll
            for (int t = 0; t < G; ++t)
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const bool in = i0 - t >= 0 && (q == 0 || in1);
                    hh[t][q] = in ? __ldcs(Vh + (size_t)(i0 - t) * ld + ee[q]) : make_float2(0.f, 0.f);
                    tt[t][q] = in ? __ldcs(Vt + (size_t)(i0 - t) * ld + ee[q]) : make_uint2(0u, 0u);
                }
        };
        if (i >= 0) load(i, ch, ct);
        for (; i >= 0; i -= G, ++g) {
            if (i - G >= 0) load(i - G, nh, nt);
#pragma unroll
            for (int t = 0; t < G; ++t)
                if (i - t >= 0) vec(i - t, ch[t], ct[t], (dmask >> ((i - t) & 7)) & 1);
            if ((g & 1) == 1) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    tf_renorm(A[q]);
                    tf_renorm(B[q]);
                    df_norm2(rah[q], ral[q]);
                    df_norm2(rbh[q], rbl[q]);
                }
            }
#pragma unroll
            for (int t = 0; t < G; ++t)
#pragma unroll
                for (int q = 0; q < 2; ++q) { ch[t][q] = nh[t][q]; ct[t][q] = nt[t][q]; }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (q == 1 && !in1) break;
            const long long eq = ee[q];
            const double2 s = make_double2(acc[q].x + (tf_lane(A[q], 0) - tf_lane(B[q], 1)),
                                           acc[q].y + (tf_lane(A[q], 1) + tf_lane(B[q], 0)));
            const float2 pah = f2_unpack(rah[q]), pal = f2_unpack(ral[q]), pbh = f2_unpack(rbh[q]),
                         pbl = f2_unpack(rbl[q]);
            const double rre = (f53_double(pah.x, 0u) + f53_double(pal.x, 0u)) -
                               (f53_double(pbh.y, 0u) + f53_double(pbl.y, 0u));
            const double rim = (f53_double(pah.y, 0u) + f53_double(pal.y, 0u)) +
                               (f53_double(pbh.x, 0u) + f53_double(pbl.x, 0u));
            double2 x = f53_load(uh, ut, eq);
            x.x -= rre;
            x.y -= rim;
            f53_store(uh, ut, eq, x);
            double2 y = csub(f53_load(wh, wt, eq), s);
            y = cfms(cj, x, y);
            f53_store(wh, wt, eq, y);
            nrm = fma(y.x, y.x, fma(y.y, y.y, nrm));
        }
    }
    __shared__ double nred[kS53Threads / 32];
    nrm = warp_sum_d(nrm);
    if ((threadIdx.x & 31) == 0) nred[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += nred[k];
        npart[(size_t)r * nblk + blockIdx.x] = t;
    }
}

// ------------------------------------------------------------------ launchers
void launch_f53_encode(const Ctx& cx, int nb, long long N, const double2* src, long long ss, float2* dh, uint2* dt,
                       long long ds, const double* scale, const KState* st) {
    k_f53_encode<<<dim3(4 * cx.num_sms, nb), 256, 0, cx.stream>>>(N, src, ss, dh, dt, ds, scale, st);
}

void launch_f53_scale0(const Ctx& cx, int nb, double* sigma, double* sigt, long long sS, double* scale) {
    k_f53_scale0<<<(nb + 127) / 128, 128, 0, cx.stream>>>(nb, sigma, sigt, sS, scale);
}

size_t s53_update_smem(int j) { return (size_t)(j > 0 ? j : 1) * sizeof(S53Coef); }

// returns the number of blocks (rows of partials the reduction sums): whole waves of
// resident blocks, at most kb.nblk_dot
template <int MINB, int NS>
static const void* s53_dot_fn(int g) {
    return g == 1 ? (const void*)k_s53_dot<MINB, NS, 1> : (const void*)k_s53_dot<MINB, NS, 2>;
}
template <int MINB>
static const void* s53_dot_fn(int ns, int g) {
    return ns == 4 ? s53_dot_fn<MINB, 4>(g) : ns == 3 ? s53_dot_fn<MINB, 3>(g) : s53_dot_fn<MINB, 0>(g);
}

int launch_s53_dot(const Ctx& cx, const KrylovBufs& kb, int nb, int j, int has_w, unsigned dmask) {
    const float2* Vh = kb.V32;
    const uint2* Vt = static_cast<const uint2*>(kb.V32lo);
    const int minb = kb.s53_dot_minb;
    const int ns = kb.s53_ring == 4 ? 4 : (kb.s53_ring == 3 ? 3 : 0);
    const int gsz = kb.s53_group == 1 ? 1 : (kb.s53_group == 4 && kb.s53_ws ? 4 : 2);
    const size_t smem = (size_t)ns * (2 * gsz + 3) * kS53Threads * sizeof(uint2);
    const void* fn = minb == 4 ? s53_dot_fn<4>(ns, gsz) : minb == 3 ? s53_dot_fn<3>(ns, gsz) : s53_dot_fn<2>(ns, gsz);
    // (s53_dot_fn maps a group of 4 to 2: only the specialised kernel takes 4)
    size_t smem_l = smem;
    if (kb.s53_ws) {
        // specialised warps: FP64 tasks of s53_g64 vectors, FP32 tasks of s53_group vectors, 4-stage
        // ring; compiled for 3 blocks per SM with FP32 tasks of 1 or 2 vectors and FP64 tasks of 4,
        // else for 2 blocks per SM
        const int g32 = minb == 3 && gsz == 4 ? 2 : gsz;
        const bool g8 = kb.s53_g64 == 8 && minb != 3;
        // FP64 tasks through the ring too (FP64 tasks of 4 and FP32 tasks of 4 only)
        const bool r64 = kb.s53_ring64 && minb != 3 && !g8 && g32 == 4;
        smem_l = (size_t)4 * (2 * g32 + 3) * kS53Threads * sizeof(uint2);
        fn = minb == 3 ? (g32 == 1 ? (const void*)k_s53_dot_ws<3, 4, 1, 4, false>
                                   : (const void*)k_s53_dot_ws<3, 4, 2, 4, false>)
             : g32 == 1 ? (const void*)k_s53_dot_ws<2, 4, 1, 4, false>
             : g32 == 4 ? (g8  ? (const void*)k_s53_dot_ws<2, 8, 4, 4, false>
                           : r64 ? (const void*)k_s53_dot_ws<2, 4, 4, 4, true>
                                 : (const void*)k_s53_dot_ws<2, 4, 4, 4, false>)
                        : (g8 ? (const void*)k_s53_dot_ws<2, 8, 2, 4, false>
                              : (const void*)k_s53_dot_ws<2, 4, 2, 4, false>);
    }
    if (smem_l > 0 && allow_dynamic_smem(fn, smem_l) != cudaSuccess) return 0;
    const int per_sm = minb == 3 ? 3 : (kb.s53_dot_waves == 1 ? 2 : 4);   // 2 blocks/SM: one or two waves
    const int blocks = std::min(kb.nblk_dot, per_sm * cx.num_sms);
    int S = kb.maxit + 1;
    long long N = kb.N, ld = kb.ld, sV = kb.sV(), sP = kb.sP();
    int ps = kb.pstride();
    double2* part = kb.part;
    const KState* st = kb.st;
    void* args[] = {&j, &N, &ld, &ps, &S, (void*)&Vh, (void*)&Vt, &sV, &has_w, &dmask, &part, &sP, (void*)&st};
    if (cudaLaunchKernel(fn, dim3(blocks, nb), dim3(kS53Threads), args, smem_l, cx.stream) != cudaSuccess) return 0;
    return blocks;
}

// returns the number of blocks (the count of norm partials per entry), 0 if the
// coefficients do not fit in shared memory
int launch_s53_update(const Ctx& cx, const KrylovBufs& kb, int nb, int j, unsigned dmask) {
    const size_t us = s53_update_smem(j);
    const bool three = kb.s53_minb == 3;
    const void* fn = kb.s53_upd_e == 2 ? (three ? (const void*)k_s53_update2<3> : (const void*)k_s53_update2<2>)
                                       : (three ? (const void*)k_s53_update<3> : (const void*)k_s53_update<2>);
    if (allow_dynamic_smem(fn, us) != cudaSuccess) return 0;
    // blocks per SM: as the registers allow while their shared memory fits (<= kb.nblk / SMs,
    // the partials' stride)
    int bps = three ? 3 : 2;
    while (bps > 1 && (size_t)bps * (us + 8192) > (size_t)(228 * 1024)) --bps;
    const int blocks = bps * cx.num_sms;
    float2* Vh = kb.V32;
    uint2* Vt = static_cast<uint2*>(kb.V32lo);
    long long N = kb.N, ld = kb.ld, sV = kb.sV(), sS = kb.sS();
    const double* sigma = kb.sigma;
    const double2 *h1 = kb.h1, *h2 = kb.h2;
    double* npart = kb.npart;
    int nblk = kb.nblk;
    const KState* st = kb.st;
    void* args[] = {&j, &N, &ld, (void*)&Vh, (void*)&Vt, &sV, (void*)&sigma, (void*)&h1, (void*)&h2, &sS, &dmask,
                    (void*)&npart, &nblk, (void*)&st};
    if (cudaLaunchKernel(fn, dim3(blocks, nb), dim3(kS53Threads), args, us, cx.stream) != cudaSuccess) return 0;
    return blocks;
}

}  // namespace hzs
