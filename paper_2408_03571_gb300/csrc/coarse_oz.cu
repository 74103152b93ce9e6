// FP64-accurate block products of the block-tridiagonal coarse solve (Eq. 4, Section 4)
// on the tensor cores, for many right-hand sides at once.
//
// Each block step of the many-right-hand-side sweeps is y = W_i x for the nb vectors x of
// one block row (W_i = S_i^{-1}, b_i x b_i complex FP64).  In real form
//     [Re y | Im y] = [Re W_i | Im W_i] [[Re x, Im x], [-Im x, Re x]]  =  A B,
// with A of b_i x 2 b_i and B of 2 b_i x 2 nb.  The product is formed by splitting
// (Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012): every row of A and every
// column of B is scaled by a power of two that bounds it, and the scaled values are cut
// into 8 signed digits of 7 bits (56 bits, truncated toward zero):
//     A = 2^{e_r} sum_s 2^{-7s} A_s,   B = 2^{f_c} sum_t 2^{-7t} B_t,   |digits| <= 127.
// A digit is exact in bf16, a product of two digits in FP32, and a sum of K <= 1040 of
// them stays below 2^24, so every slice product A_s B_t of the tensor cores (bf16 inputs,
// FP32 accumulation) is exact.  The pairs with s + t <= 9 are kept (36 products); with
// the digits cut off after 56 bits, the result differs from the exact product by less
// than about 2^-50.5 K max|A_r| max|B_c|, a few units of the rounding bound of an FP64 dot
// product of length K.  Each kept product is scaled by 2^{-7(s+t)} (exact) and summed in
// three-word FP32 expansions, and the sum is rounded once to FP64: no step runs on the
// FP64 pipe except that final conversion and the scaling.
//
// Layout: a slice of A (or B) is stored in chunks of 128 (32) rows by 64 K, each chunk the
// canonical no-swizzle K-major arrangement of the tensor cores (core matrices of 8 rows by
// 8 K, 128 contiguous bytes; consecutive core matrices along K, then along rows).  The
// chunks one CTA reads for one K range sit side by side (A: the two slices s and 9 - s of
// a row tile; B: slices 1..8 of a column tile), so two bulk copies fill a pipeline stage.
//
// One CTA computes a 128 x 32 output tile for the slice pairs (s, t) with s in
// {sp + 1, 8 - sp} (sp = 0..3) and s + t <= 9: 9 pairs for every sp, so the four CTAs of a
// tile carry equal work.  K streams through a 3-stage ring (bulk copies on full barriers,
// MMA completion on empty barriers; one thread copies, another issues the MMAs); the 9
// accumulators (128 x 32 FP32 each) live in
// tensor memory.  A combine kernel adds the four CTAs' expansions, converts to FP64 and
// applies the scales.
#include <vector>

#include "async.cuh"
#include "kernels.cuh"

namespace hzs {

namespace {
constexpr int kOzS = 8;                                        // digit slices per operand
constexpr int kOzMT = 128;                                     // rows of an output tile (MMA M)
constexpr int kOzNC = 32;                                      // columns of an output tile (MMA N)
constexpr int kOzKC = 64;                                      // K of one pipeline chunk
constexpr int kOzStages = 3;
constexpr int kOzAChunk = kOzMT * kOzKC * 2;                   // bytes of an A chunk (bf16)
constexpr int kOzBChunk = kOzNC * kOzKC * 2;                   // bytes of a B chunk
constexpr int kOzStageBytes = 2 * kOzAChunk + kOzS * kOzBChunk;
constexpr int kOzSmem = kOzStages * kOzStageBytes;             // 192 KB
constexpr int kOzKMax = 1040;                                  // K 127^2 < 2^24
constexpr int kOzNonFinite = 1 << 20;                          // exponent marking a non-finite column
}  // namespace

// byte offset of element (r, k) inside a chunk (core matrices of 8 rows x 8 K)
__host__ __device__ __forceinline__ int oz_off(int r, int k) {
    return ((((r >> 3) << 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1);
}

__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}
// exponent e with |v| < 2^e for the largest |v| (given as its bit pattern); 0 for zero
// or subnormal maxima (all digits are then zero), kOzNonFinite for inf / NaN
__device__ __forceinline__ int oz_exponent(unsigned long long maxbits) {
    const int ex = (int)(maxbits >> 52);
    if (ex == 0x7FF) return kOzNonFinite;
    return ex == 0 ? 0 : ex - 1022;
}
// trunc(|v| 2^(56 - e)) (< 2^56) and the sign of v, by integer operations on the bit
// pattern; subnormal v count as zero
__device__ __forceinline__ unsigned long long oz_fixed(double v, int e, bool& neg) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    neg = (bits >> 63) != 0;
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex == 0 || ex == 0x7FF || e == kOzNonFinite) return 0;
    const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = ex - 1075 + 56 - e;                          // |v| = mant 2^(ex - 1075)
    if (sh >= 0) return sh < 4 ? mant << sh : 0;
    return sh > -64 ? mant >> (-sh) : 0;
}
// bf16 bit pattern of the signed digit s (1..8) of a
__device__ __forceinline__ unsigned short oz_digit(unsigned long long a, bool neg, int s) {
    const float d = (float)(int)((a >> (56 - 7 * s)) & 127ull);
    return (unsigned short)(__float_as_uint(neg ? -d : d) >> 16);
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long m, unsigned long long* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long x = __shfl_xor_sync(0xffffffffu, m, o);
        m = x > m ? x : m;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = m;
    __syncthreads();
    m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
    return m;
}

// Chunk of A slice s (1..8) for row tile mt and K chunk kc: slices s and 9 - s are paired
// (sp = min(s, 9 - s) - 1, the smaller first) and stored side by side.
__host__ __device__ __forceinline__ size_t oz_achunk(int s, int mt, int kc, int MT, int KCH) {
    const int sp = (s <= 4 ? s : 9 - s) - 1, h = s <= 4 ? 0 : 1;
    return (((size_t)sp * MT + mt) * KCH + kc) * 2 + h;
}
// Chunk of B slice t (1..8) for column tile nq and K chunk kc: slices 1..8 side by side.
__host__ __device__ __forceinline__ size_t oz_bchunk(int t, int nq, int kc, int KCH) {
    return ((size_t)nq * KCH + kc) * kOzS + (t - 1);
}

// Set-up: digit slices of A = [Re W | Im W] (b x b complex, row-major), one block per row;
// As (zeroed beforehand) receives slice s at chunk oz_achunk; erow[r] = e_r.
__global__ void k_oz_split_a(const double2* __restrict__ W, int b, int MT, int KCH, unsigned short* __restrict__ As,
                             int* __restrict__ erow) {
    __shared__ unsigned long long red[32];
    const int row = blockIdx.x;
    const double2* w = W + (size_t)row * b;
    unsigned long long m = 0;
    for (int k = threadIdx.x; k < b; k += blockDim.x) {
        const double2 v = w[k];
        const unsigned long long a = abs_bits(v.x), c = abs_bits(v.y);
        m = a > m ? a : m;
        m = c > m ? c : m;
    }
    m = block_max_u64(m, red);
    const int e = oz_exponent(m);
    if (threadIdx.x == 0) erow[row] = e;
    const int mt = row / kOzMT, rl = row % kOzMT;
    for (int k2 = threadIdx.x; k2 < 2 * b; k2 += blockDim.x) {
        const double v = k2 < b ? w[k2].x : w[k2 - b].y;
        bool neg;
        const unsigned long long a = oz_fixed(v, e, neg);
        const int kc = k2 / kOzKC, kl = k2 % kOzKC;
        const size_t in_chunk = (size_t)oz_off(rl, kl) / 2;
#pragma unroll
        for (int s = 1; s <= kOzS; ++s)
            As[oz_achunk(s, mt, kc, MT, KCH) * (kOzAChunk / 2) + in_chunk] = oz_digit(a, neg, s);
    }
}

// Per block step: digit slices of B for the nb right-hand sides x_c (b entries each, x_c =
// x + c stride); slot c (one block each, NQ * 16 slots) fills columns 2c ([Re x; -Im x])
// and 2c + 1 ([Im x; Re x]) over the whole padded K, zeros for empty or skipped slots;
// fcol[c] = f_c.
__global__ void k_oz_split_b(const double2* __restrict__ x, long long stride, int b, int nb, int NQ, int KCH,
                             unsigned short* __restrict__ Bs, int* __restrict__ fcol, BatchSkip sk) {
    __shared__ unsigned long long red[32];
    const int c = blockIdx.x;
    const bool real = c < nb && !(sk.flag && sk.flag[(size_t)c * sk.stride]);
    const double2* xc = x + (size_t)c * stride;
    unsigned long long m = 0;
    if (real)
        for (int k = threadIdx.x; k < b; k += blockDim.x) {
            const double2 v = xc[k];
            const unsigned long long a = abs_bits(v.x), d = abs_bits(v.y);
            m = a > m ? a : m;
            m = d > m ? d : m;
        }
    m = block_max_u64(m, red);
    const int e = oz_exponent(m);
    if (threadIdx.x == 0) fcol[c] = real ? e : 0;
    const int n0 = 2 * c, nq = n0 / kOzNC, nl = n0 % kOzNC;   // both columns in the same chunk
    // one thread per 8 consecutive K: the 16-byte row of a core matrix, written whole for
    // each slice and column
    for (int ko = threadIdx.x; ko < KCH * kOzKC / 8; ko += blockDim.x) {
        const int k0 = ko * 8;
        uint32_t w0[kOzS][4], w1[kOzS][4];
#pragma unroll
        for (int s = 0; s < kOzS; ++s)
#pragma unroll
            for (int q = 0; q < 4; ++q) w0[s][q] = w1[s][q] = 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k2 = k0 + j;
            double v0 = 0.0, v1 = 0.0;
            if (real && k2 < 2 * b) {
                const double2 z = xc[k2 < b ? k2 : k2 - b];
                v0 = k2 < b ? z.x : -z.y;
                v1 = k2 < b ? z.y : z.x;
            }
            bool g0, g1;
            const unsigned long long a0 = oz_fixed(v0, e, g0), a1 = oz_fixed(v1, e, g1);
#pragma unroll
            for (int s = 0; s < kOzS; ++s) {
                w0[s][j >> 1] |= (uint32_t)oz_digit(a0, g0, s + 1) << ((j & 1) * 16);
                w1[s][j >> 1] |= (uint32_t)oz_digit(a1, g1, s + 1) << ((j & 1) * 16);
            }
        }
        const int kc = k0 / kOzKC, kl = k0 % kOzKC;             // kl a multiple of 8
        const size_t o0 = (size_t)oz_off(nl, kl) / 2, o1 = (size_t)oz_off(nl + 1, kl) / 2;
#pragma unroll
        for (int s = 0; s < kOzS; ++s) {
            unsigned short* chunk = Bs + oz_bchunk(s + 1, nq, kc, KCH) * (kOzBChunk / 2);
            *reinterpret_cast<uint4*>(chunk + o0) = make_uint4(w0[s][0], w0[s][1], w0[s][2], w0[s][3]);
            *reinterpret_cast<uint4*>(chunk + o1) = make_uint4(w1[s][0], w1[s][1], w1[s][2], w1[s][3]);
        }
    }
}

// Three-word FP32 expansion (s0, s1, s2) += x: error-free at the two upper levels.
__device__ __forceinline__ void acc3_add(float& s0, float& s1, float& s2, float x) {
    float e0, e1;
    two_sum(s0, x, s0, e0);
    two_sum(s1, e0, s1, e1);
    s2 += e1;
}

// The slice products of one 128 x 32 output tile (blockIdx.x: row tile, .y: sp, .z: column
// tile); writes the three words of its sum to part[((sp 3 + w) Mrows + row) Ncols + col].
// Every wait is bounded (2^24 polls): on expiry the CTA records HZS_ERR_TIMEOUT, waits
// (bounded) for its copies and MMAs, frees its tensor memory and returns.
__global__ void __launch_bounds__(128, 1) k_oz_gemm(const unsigned char* __restrict__ As,
                                                    const unsigned char* __restrict__ Bs, int MT, int KCH, int NQ,
                                                    float* __restrict__ part, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char oz_smem[];
    __shared__ __align__(8) uint64_t full[kOzStages], empty[kOzStages], done;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    const int mt = blockIdx.x, sp = blockIdx.y, nq = blockIdx.z;
    const int sa = sp + 1, sb = kOzS - sp;                    // sa + sb = 9
    const int tmax = 9 - sa;                                  // B slices read: 1 .. tmax (>= 9 - sb)
    const uint32_t stage_bytes = (uint32_t)(2 * kOzAChunk + tmax * kOzBChunk);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int q = 0; q < kOzStages; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        mbar_init(&done, 1);
        mbar_init_fence();
        s_fail = 0;
    }
    if (warp == 0) tmem_alloc(&tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    auto load = [&](int kc, int st) {
        unsigned char* S = oz_smem + (size_t)st * kOzStageBytes;
        mbar_expect_tx(&full[st], stage_bytes);
        bulk_g2s(S, As + oz_achunk(sa, mt, kc, MT, KCH) * kOzAChunk, 2 * kOzAChunk, &full[st]);
        bulk_g2s(S + 2 * kOzAChunk, Bs + oz_bchunk(1, nq, kc, KCH) * kOzBChunk, (uint32_t)(tmax * kOzBChunk),
                 &full[st]);
    };
    // warp 0 copies, warp 1 issues the MMAs: neither waits on the other's barriers
    __shared__ int s_loaded, s_consumed;
    if (tid == 0) {
        // a stage is refilled once the MMAs of the chunk kOzStages back have read it
        int kc = 0;
        for (; kc < KCH; ++kc) {
            const int st = kc % kOzStages;
            if (kc >= kOzStages &&
                !mbar_wait_bounded(&empty[st], (uint32_t)(((kc - kOzStages) / kOzStages) & 1))) {
                s_fail = 1;
                break;
            }
            load(kc, st);
        }
        s_loaded = kc;
    } else if (tid == 32) {
        const uint32_t idesc = idesc_bf16_f32(kOzMT, kOzNC);
        // the 9 pairs' A and B slots in a stage, in the 16-byte units of a descriptor's start
        // address: each MMA's descriptors are then one 64-bit add to the stage's (shared
        // addresses stay below 2^14 units, so the field never carries)
        // (pairs 0 .. na - 1 are (sa, t = p + 1), the rest (sb, t = p - na + 1))
        const int na = 9 - sa;
        uint32_t aoff[9], boff[9];
#pragma unroll
        for (int p = 0; p < 9; ++p) {
            const int h = p >= na, t = h ? p - na + 1 : p + 1;
            aoff[p] = (uint32_t)(h * kOzAChunk) >> 4;
            boff[p] = (uint32_t)(2 * kOzAChunk + (t - 1) * kOzBChunk) >> 4;
        }
        const uint64_t dbase = smem_desc(smem_u32(oz_smem), 128, 1024);
        int kc = 0;
        for (; kc < KCH; ++kc) {
            const int st = kc % kOzStages;
            if (!mbar_wait_bounded(&full[st], (uint32_t)((kc / kOzStages) & 1))) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            const uint64_t dst = dbase + (uint64_t)((uint32_t)(st * kOzStageBytes) >> 4);
            const uint32_t first = kc != 0;
#pragma unroll
            for (int p = 0; p < 9; ++p)
#pragma unroll
                for (int ks = 0; ks < kOzKC / 16; ++ks)
                    mma_bf16(tmem + (uint32_t)(p * kOzNC), dst + aoff[p] + (uint32_t)(ks * 16),
                             dst + boff[p] + (uint32_t)(ks * 16), idesc, ks == 0 ? first : 1u);
            mma_commit(&empty[st]);
        }
        mma_commit(&done);
        s_consumed = kc;
    }
    __syncthreads();
    if (tid == 0 && s_fail) {
        if (err) atomicExch(err, (int)HZS_ERR_TIMEOUT);
        for (int c = s_consumed; c < s_loaded; ++c)           // copies possibly in flight
            mbar_wait_bounded(&full[c % kOzStages], (uint32_t)((c / kOzStages) & 1));
    }
    __syncthreads();
    bool ok = mbar_wait_bounded(&done, 0);
    if (!ok) ok = mbar_wait_bounded(&done, 0);                // again before the memory is freed
    const bool fail = __syncthreads_or(!ok || s_fail) != 0;
    tc_fence_after();
    if (!fail) {
        float a0[kOzNC], a1[kOzNC], a2[kOzNC];
#pragma unroll
        for (int j = 0; j < kOzNC; ++j) a0[j] = a1[j] = a2[j] = 0.f;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        int p = 0;
        for (int h = 0; h < 2; ++h) {
            const int s = h ? sb : sa;
            for (int t = 1; t <= 9 - s; ++t, ++p) {
                uint32_t v[kOzNC];
                tmem_ld32(lane_base + (uint32_t)(p * kOzNC), v);
                const float sc = __int_as_float((127 - 7 * (s + t)) << 23);   // 2^{-7(s+t)}
#pragma unroll
                for (int j = 0; j < kOzNC; ++j) acc3_add(a0[j], a1[j], a2[j], __uint_as_float(v[j]) * sc);
            }
        }
        const int Mrows = MT * kOzMT, Ncols = NQ * kOzNC;
        const size_t row = (size_t)mt * kOzMT + warp * 32 + lane;
        float* p0 = part + (((size_t)sp * 3 + 0) * Mrows + row) * Ncols + (size_t)nq * kOzNC;
        float* p1 = part + (((size_t)sp * 3 + 1) * Mrows + row) * Ncols + (size_t)nq * kOzNC;
        float* p2 = part + (((size_t)sp * 3 + 2) * Mrows + row) * Ncols + (size_t)nq * kOzNC;
#pragma unroll
        for (int j = 0; j < kOzNC; j += 4) {
            *reinterpret_cast<float4*>(p0 + j) = make_float4(a0[j], a0[j + 1], a0[j + 2], a0[j + 3]);
            *reinterpret_cast<float4*>(p1 + j) = make_float4(a1[j], a1[j + 1], a1[j + 2], a1[j + 3]);
            *reinterpret_cast<float4*>(p2 + j) = make_float4(a2[j], a2[j + 1], a2[j + 2], a2[j + 3]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// out[c stride + r] = 2^{e_r + f_c} (y_r + i y_i), the FP64 rounding of the four CTAs'
// expansions for (row r, column 2c) and (r, 2c + 1); base - that when base is given.
__global__ void k_oz_combine(const float* __restrict__ part, int Mrows, int Ncols, int b, int nb,
                             const int* __restrict__ erow, const int* __restrict__ fcol, const double2* base,
                             double2* out, long long stride, BatchSkip sk) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)b * nb) return;
    const int c = (int)(t % nb), r = (int)(t / nb);
    if (sk.flag && sk.flag[(size_t)c * sk.stride]) return;
    const int f = fcol[c];
    double y[2];
#pragma unroll
    for (int comp = 0; comp < 2; ++comp) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int w = 0; w < 3; ++w)
                acc3_add(s0, s1, s2, part[(((size_t)sp * 3 + w) * Mrows + r) * Ncols + 2 * c + comp]);
        y[comp] = ((double)s2 + (double)s1) + (double)s0;
    }
    double2 v;
    if (f == kOzNonFinite) {
        v = make_double2(__longlong_as_double(0x7FF8000000000000ll), __longlong_as_double(0x7FF8000000000000ll));
    } else {
        const double sc = ldexp(1.0, erow[r] + f);
        v = make_double2(y[0] * sc, y[1] * sc);
    }
    const size_t o = (size_t)c * stride + r;
    if (base) {
        const double2 bv = base[o];
        v = make_double2(bv.x - v.x, bv.y - v.y);
    }
    out[o] = v;
}

// ------------------------------------------------------------------ host
int coarse_oz_setup(const Ctx& cx, CoarseBlockLU& lu) {
    const int m = lu.m;
    for (int i = 0; i < m; ++i)
        if (2 * lu.b[i] > kOzKMax) return 1;                  // a slice product would not be exact
    lu.oz_mt.assign(m, 0);
    lu.oz_kch.assign(m, 0);
    lu.aoz.assign(m, 0);
    long long total = 0;
    for (int i = 0; i < m; ++i) {
        lu.oz_mt[i] = (lu.b[i] + kOzMT - 1) / kOzMT;
        lu.oz_kch[i] = (2 * lu.b[i] + kOzKC - 1) / kOzKC;
        lu.aoz[i] = total;
        total += (long long)kOzS * lu.oz_mt[i] * lu.oz_kch[i] * kOzAChunk;
    }
    const int Nc = lu.nc1 * lu.nc1;
    if (cudaMalloc(&lu.Aoz, (size_t)total) != cudaSuccess) return -1;
    if (cudaMalloc(&lu.eoz, (size_t)Nc * sizeof(int)) != cudaSuccess) return -1;
    if (cudaMemsetAsync(lu.Aoz, 0, (size_t)total, cx.stream) != cudaSuccess) return -1;
    for (int i = 0; i < m; ++i)
        k_oz_split_a<<<lu.b[i], 128, 0, cx.stream>>>(lu.W + lu.wo[i], lu.b[i], lu.oz_mt[i], lu.oz_kch[i],
                                                     reinterpret_cast<unsigned short*>(lu.Aoz + lu.aoz[i]),
                                                     lu.eoz + lu.r0[i]);
    if (allow_dynamic_smem((const void*)k_oz_gemm, kOzSmem) != cudaSuccess) return -1;
    return cudaStreamSynchronize(cx.stream) == cudaSuccess ? 0 : -1;
}

int coarse_oz_reserve(CoarseBlockLU& lu, int nb) {
    if (!lu.Aoz || nb <= lu.oz_cap) return 0;
    cudaFree(lu.Boz); cudaFree(lu.Poz); cudaFree(lu.foz);
    lu.Boz = nullptr; lu.Poz = nullptr; lu.foz = nullptr;
    lu.oz_cap = 0;
    int mtmax = 0, kchmax = 0;
    for (int i = 0; i < lu.m; ++i) {
        mtmax = std::max(mtmax, lu.oz_mt[i]);
        kchmax = std::max(kchmax, lu.oz_kch[i]);
    }
    const int NQ = (2 * nb + kOzNC - 1) / kOzNC;
    if (cudaMalloc(&lu.Boz, (size_t)kOzS * NQ * kchmax * kOzBChunk) != cudaSuccess) return -1;
    if (cudaMalloc(&lu.Poz, (size_t)4 * 3 * mtmax * kOzMT * NQ * kOzNC * sizeof(float)) != cudaSuccess) return -1;
    if (cudaMalloc(&lu.foz, (size_t)NQ * (kOzNC / 2) * sizeof(int)) != cudaSuccess) return -1;
    lu.oz_cap = nb;
    return 0;
}

void coarse_oz_free(CoarseBlockLU& lu) {
    cudaFree(lu.Aoz); cudaFree(lu.eoz); cudaFree(lu.Boz); cudaFree(lu.Poz); cudaFree(lu.foz);
    lu.Aoz = nullptr; lu.eoz = nullptr; lu.Boz = nullptr; lu.Poz = nullptr; lu.foz = nullptr;
    lu.oz_cap = 0;
}

void launch_coarse_oz_step(const Ctx& cx, int nb, const CoarseBlockLU& lu, int i, const double2* x, double2* out,
                           bool subtract, long long stride, BatchSkip sk) {
    const int b = lu.b[i], MT = lu.oz_mt[i], KCH = lu.oz_kch[i];
    const int NQ = (2 * nb + kOzNC - 1) / kOzNC;
    k_oz_split_b<<<NQ * (kOzNC / 2), 128, 0, cx.stream>>>(x, stride, b, nb, NQ, KCH,
                                                           reinterpret_cast<unsigned short*>(lu.Boz), lu.foz, sk);
    k_oz_gemm<<<dim3(MT, 4, NQ), 128, kOzSmem, cx.stream>>>(lu.Aoz + lu.aoz[i], lu.Boz, MT, KCH, NQ, lu.Poz, cx.err);
    const long long n = (long long)b * nb;
    k_oz_combine<<<(unsigned)((n + 255) / 256), 256, 0, cx.stream>>>(lu.Poz, MT * kOzMT, NQ * kOzNC, b, nb,
                                                                     lu.eoz + lu.r0[i], lu.foz,
                                                                     subtract ? out : nullptr, out, stride, sk);
}

}  // namespace hzs
