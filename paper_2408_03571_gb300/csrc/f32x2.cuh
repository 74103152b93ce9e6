// Packed FP32 pairs and the error-free FP32 arithmetic built on them, shared by
// the Krylov kernels.
#pragma once

#include <cuda_runtime.h>

namespace hzs {

// Packed FP32 pairs (two lanes in one 64-bit register: add/sub/mul/fma .f32x2,
// one issue slot for two FP32 operations).  The low half is the first lane: a
// complex64 entry loaded as 8 bytes is the pair (re, im).
typedef unsigned long long f2x;
__device__ __forceinline__ f2x f2_pack(float a, float b) {
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(f2x r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
    f2x d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
    f2x d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b) {
    f2x d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c) {
    f2x d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// Lane-wise double-float multiply-add (sh, sl) += c * (vh + vl) for an FP32 c given
// as the broadcast pairs P = (c, c), N = (-c, -c) (no negation modifier exists for the
// packed forms): the product c vh is split exactly by an FMA, c vl is added to its
// error, and the accumulation is a TwoSum.
__device__ __forceinline__ void df_fma2(f2x& sh, f2x& sl, f2x P, f2x N, f2x vh, f2x vl) {
    const f2x p = mul2(P, vh);
    f2x en = fma2(N, vh, p);            // -(c vh - p), exact
    en = fma2(N, vl, en);               // en = -(error + c vl)
    const f2x s = add2(sh, p);          // TwoSum(sh, p)
    const f2x bb = sub2(s, sh);
    const f2x t = add2(sub2(sh, sub2(s, bb)), sub2(p, bb));
    sh = s;
    sl = add2(sl, sub2(t, en));
}
__device__ __forceinline__ void df_norm2(f2x& sh, f2x& sl) {
    const f2x s = add2(sh, sl);
    sl = sub2(sl, sub2(s, sh));
    sh = s;
}

// ---- three-word FP32 expansion accumulators (packed pairs)
// An accumulator is the unevaluated sum s0 + s1 + s2 per lane.  Terms enter at the
// level of their magnitude: additions at levels 0 and 1 are error-free (TwoSum, the
// rounding error carried one level down), level 2 is a plain FP32 sum.  With a
// renormalisation (tf_renorm) every few terms, |s1| <= 2^-24 |s0| + (new level-1
// terms) and |s2| <= 2^-24 |s1| + ..., so every rounding that is not carried costs
// at most about 2^-69 of the magnitude of the partial sums and terms - far below the
// 2^-53 of an FP64 addition.
struct TF2 {
    f2x s0, s1, s2;
};
__device__ __forceinline__ void two_sum2(f2x a, f2x b, f2x& s, f2x& e) {
    s = add2(a, b);
    const f2x bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// s - e = a - b exactly (TwoSum of a and -b): e is the negated rounding error
__device__ __forceinline__ void two_diff2(f2x a, f2x b, f2x& s, f2x& en) {
    s = sub2(a, b);
    const f2x bb = sub2(s, a);                  // = -b rounded
    en = add2(sub2(sub2(s, bb), a), add2(b, bb));
}
__device__ __forceinline__ void tf_zero(TF2& A) { A.s0 = A.s1 = A.s2 = 0ull; }
__device__ __forceinline__ void tf_add0(TF2& A, f2x x) {
    f2x t, t2;
    two_sum2(A.s0, x, A.s0, t);
    two_sum2(A.s1, t, A.s1, t2);
    A.s2 = add2(A.s2, t2);
}
__device__ __forceinline__ void tf_add1(TF2& A, f2x x) {
    f2x t;
    two_sum2(A.s1, x, A.s1, t);
    A.s2 = add2(A.s2, t);
}
__device__ __forceinline__ void tf_sub1(TF2& A, f2x x) {
    f2x en;
    two_diff2(A.s1, x, A.s1, en);
    A.s2 = sub2(A.s2, en);
}
__device__ __forceinline__ void tf_renorm(TF2& A) {
    f2x t;
    two_sum2(A.s0, A.s1, A.s0, t);
    two_sum2(t, A.s2, A.s1, A.s2);
}
// A += s * V for a scalar s = s0 + s1 + s2 (broadcast pairs S0, S1, S2 and the negated
// NS0, NS1) and a pair V = V0 + V1 + V2 (|s1| <= 2^-23 |s0|, |s2| <= 2^-46 |s0|, the
// same for V): the products s0 V0, s0 V1 and s1 V0 are split exactly by FMAs, the
// terms of order 2^-46 enter level 2 as FP32 products, those below 2^-69 are dropped.
__device__ __forceinline__ void tf_mac53(TF2& A, f2x S0, f2x S1, f2x S2, f2x NS0, f2x NS1, f2x V0, f2x V1,
                                         f2x V2) {
    const f2x p0 = mul2(S0, V0), e0n = fma2(NS0, V0, p0);       // s0 V0 = p0 - e0n
    const f2x p1 = mul2(S0, V1), e1n = fma2(NS0, V1, p1);       // s0 V1 = p1 - e1n
    const f2x p2 = mul2(S1, V0), e2n = fma2(NS1, V0, p2);       // s1 V0 = p2 - e2n
    tf_add0(A, p0);
    tf_add1(A, p1);
    tf_add1(A, p2);
    tf_sub1(A, e0n);
    f2x l2 = fma2(S0, V2, A.s2);
    l2 = fma2(S1, V1, l2);
    l2 = fma2(S2, V0, l2);
    A.s2 = sub2(sub2(l2, e1n), e2n);
}
// A += c * V for an FP32 scalar c (broadcast C, negated NC) and V as above.
__device__ __forceinline__ void tf_mac24(TF2& A, f2x C, f2x NC, f2x V0, f2x V1, f2x V2) {
    const f2x p0 = mul2(C, V0), e0n = fma2(NC, V0, p0);
    const f2x p1 = mul2(C, V1), e1n = fma2(NC, V1, p1);
    tf_add0(A, p0);
    tf_add1(A, p1);
    tf_sub1(A, e0n);
    A.s2 = sub2(fma2(C, V2, A.s2), e1n);
}
// (rh, rl) += a * (V0 + V1) for a double-float scalar a = ah + al (broadcast AH and the
// negated NAH, NAL): error-free head product, the cross terms added to its error.
__device__ __forceinline__ void df_mac2(f2x& rh, f2x& rl, f2x AH, f2x NAH, f2x NAL, f2x V0, f2x V1) {
    const f2x p = mul2(AH, V0);
    f2x en = fma2(NAH, V0, p);
    en = fma2(NAH, V1, en);
    en = fma2(NAL, V0, en);
    f2x s, t;
    two_sum2(rh, p, s, t);
    rh = s;
    rl = add2(rl, sub2(t, en));
}

// ---- FP64 values stored as an FP32 head and a 29-bit integer tail ("f53")
// x = head + tail * 2^(E - 179) exactly, where head is x with its fraction truncated
// to 23 bits, as FP32 (biased exponent E), and tail holds the low 29 fraction bits
// of x.  Only integer operations convert between the forms (the FP64 pipe and its
// conversions run at 1/64 of the FP32 rate on this part).  Range: |x| below 2^-97 is
// stored as a signed zero (so that the tail's FP32 pieces stay normal); |x| >= 2^128
// and non-finite values as NaN.
__device__ __forceinline__ void f53_encode(double x, float& head, unsigned& tail) {
    const unsigned H = (unsigned)__double2hiint(x), L = (unsigned)__double2loint(x);
    const unsigned a = H & 0x7fffffffu, sg = H & 0x80000000u;
    unsigned hb = __funnelshift_l(L, a - (896u << 20), 3) | sg;
    unsigned t = L & 0x1fffffffu;
    if (a < (926u << 20)) { hb = sg; t = 0u; }
    if (a >= (1151u << 20)) { hb = 0x7fc00000u; t = 0u; }
    head = __uint_as_float(hb);
    tail = t;
}
__device__ __forceinline__ double f53_double(float head, unsigned tail) {
    const unsigned hb = __float_as_uint(head), a = hb & 0x7fffffffu;
    unsigned H = (hb & 0x80000000u) | ((a >> 3) + (896u << 20));
    if (a < 0x00800000u) H = hb & 0x80000000u;          // zero (subnormal heads: below 2^-126, read as tiny)
    if (a >= 0x7f800000u) H = 0x7ff80000u;
    return __hiloint2double((int)H, (int)((hb << 29) | tail));
}
// the two FP32 pieces below the head: x = head + v1 + v2, v1 = (tail >> 6) 2^(E-173),
// v2 = (tail & 63) 2^(E-179), each built as as_float(F | m) - as_float(F) for the
// FP32 exponent field F of its unit
__device__ __forceinline__ void f53_low(float head, unsigned tail, float& v1, float& v2) {
    const unsigned F1 = (__float_as_uint(head) & 0xff800000u) - (23u << 23);
    const unsigned F2 = F1 - (6u << 23);
    v1 = __uint_as_float(F1 | (tail >> 6)) - __uint_as_float(F1);
    v2 = __uint_as_float(F2 | (tail & 63u)) - __uint_as_float(F2);
}
// the same for a complex entry (head pair, tail pair) as packed (re, im) pairs
__device__ __forceinline__ void f53_low2(float2 h, uint2 t, f2x& V1, f2x& V2) {
    const unsigned F1r = (__float_as_uint(h.x) & 0xff800000u) - (23u << 23);
    const unsigned F1i = (__float_as_uint(h.y) & 0xff800000u) - (23u << 23);
    const unsigned F2r = F1r - (6u << 23), F2i = F1i - (6u << 23);
    V1 = sub2(f2_pack(__uint_as_float(F1r | (t.x >> 6)), __uint_as_float(F1i | (t.y >> 6))),
              f2_pack(__uint_as_float(F1r), __uint_as_float(F1i)));
    V2 = sub2(f2_pack(__uint_as_float(F2r | (t.x & 63u)), __uint_as_float(F2i | (t.y & 63u))),
              f2_pack(__uint_as_float(F2r), __uint_as_float(F2i)));
}
__device__ __forceinline__ f2x f2_of(float2 v) { return f2_pack(v.x, v.y); }
__device__ __forceinline__ f2x f2_bcast(float a) { return f2_pack(a, a); }
// FP64 sum of the three words of lane k (0: re, 1: im) of an accumulator
__device__ __forceinline__ double tf_lane(const TF2& A, int k) {
    const float2 a = f2_unpack(A.s0), b = f2_unpack(A.s1), c = f2_unpack(A.s2);
    return k == 0 ? (f53_double(a.x, 0u) + f53_double(b.x, 0u)) + f53_double(c.x, 0u)
                  : (f53_double(a.y, 0u) + f53_double(b.y, 0u)) + f53_double(c.y, 0u);
}

}  // namespace hzs
