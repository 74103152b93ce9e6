// Shared device helpers for the Helmholtz / Schwarz kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hzs.h"

namespace hzs {

// ---------------------------------------------------------------- complex
template <typename R> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float> { using type = float2; };
template <typename R> using cplx_t = typename cplx<R>::type;

template <typename C> __host__ __device__ __forceinline__ C mk(double re, double im);
template <> __host__ __device__ __forceinline__ double2 mk<double2>(double re, double im) { return make_double2(re, im); }
template <> __host__ __device__ __forceinline__ float2 mk<float2>(double re, double im) {
    return make_float2((float)re, (float)im);
}

__host__ __device__ __forceinline__ double2 to_d(double2 a) { return a; }
__host__ __device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
__host__ __device__ __forceinline__ float2 to_f(double2 a) { return make_float2((float)a.x, (float)a.y); }
__host__ __device__ __forceinline__ float2 to_f(float2 a) { return a; }
template <typename C> __host__ __device__ __forceinline__ C cvt(double2 a);
template <> __host__ __device__ __forceinline__ double2 cvt<double2>(double2 a) { return a; }
template <> __host__ __device__ __forceinline__ float2 cvt<float2>(double2 a) { return to_f(a); }
template <typename C> __host__ __device__ __forceinline__ C cvtf(float2 a);
template <> __host__ __device__ __forceinline__ double2 cvtf<double2>(float2 a) { return to_d(a); }
template <> __host__ __device__ __forceinline__ float2 cvtf<float2>(float2 a) { return a; }

// Precision conversion that is the identity when the types agree (so that a
// complex64 kernel never routes a value through double).
template <typename C> __host__ __device__ __forceinline__ C conv(double2 a);
template <typename C> __host__ __device__ __forceinline__ C conv(float2 a);
template <> __host__ __device__ __forceinline__ double2 conv<double2>(double2 a) { return a; }
template <> __host__ __device__ __forceinline__ float2 conv<float2>(double2 a) { return to_f(a); }
template <> __host__ __device__ __forceinline__ double2 conv<double2>(float2 a) { return to_d(a); }
template <> __host__ __device__ __forceinline__ float2 conv<float2>(float2 a) { return a; }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }
// a * b
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// acc + a * b
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
// acc + conj(a) * b
template <typename C> __device__ __forceinline__ C cfma_conj(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}
// acc - a * b
template <typename C> __device__ __forceinline__ C cfms(C a, C b, C acc) {
    acc.x = fma(-a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}

// ---------------------------------------------------------------- double-float
// A value is carried as an unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2
// after normalisation): about 48 significand bits from FP32 instructions only.
// Error-free transformations: Knuth's TwoSum and the FMA form of Dekker's product.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {   // |a| >= |b|
    s = a + b;
    e = b - (s - a);
}
// (sh, sl) += (xh + xl) * (yh + yl), dropping the xl*yl term (2^-48 relative)
__device__ __forceinline__ void df_fma(float& sh, float& sl, float xh, float xl, float yh, float yl) {
    const float p = xh * yh;
    float e = fmaf(xh, yh, -p);
    e = fmaf(xh, yl, e);
    e = fmaf(xl, yh, e);
    float s, t;
    two_sum(sh, p, s, t);
    sh = s;
    sl += t + e;
}
// (sh, sl) += (oh, ol)
__device__ __forceinline__ void df_add(float& sh, float& sl, float oh, float ol) {
    float s, t;
    two_sum(sh, oh, s, t);
    sh = s;
    sl += t + ol;
}
__device__ __forceinline__ void df_norm(float& sh, float& sl) {
    float s, t;
    fast_two_sum(sh, sl, s, t);
    sh = s; sl = t;
}
// split a double into hi = fl32(x) and lo = fl32(x - hi)
__device__ __forceinline__ void split_d(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// Remainder words of a double-float complex vector whose leading words are a
// separate complex64 array: complex64 (wide: 8 bytes an entry, about 48
// significant bits in all) or a bf16 pair (narrow: 4 bytes an entry, about 32
// bits, the bf16 keeping the top 8 of the remainder's 24).  At most one
// pointer is set; with neither, nothing is written.
struct LoDst {
    float2* wide;
    __nv_bfloat162* narrow;
    __host__ __device__ __forceinline__ LoDst at(long long off) const {
        return LoDst{wide ? wide + off : nullptr, narrow ? narrow + off : nullptr};
    }
    __host__ __device__ __forceinline__ bool any() const { return wide != nullptr || narrow != nullptr; }
    __device__ __forceinline__ void put(long long i, float2 v) const {
        if (wide) wide[i] = v;
        else if (narrow) narrow[i] = __floats2bfloat162_rn(v.x, v.y);
    }
};

template <typename C> __device__ __forceinline__ C shfl_down(C v, int off) {
    v.x = __shfl_down_sync(0xffffffffu, v.x, off);
    v.y = __shfl_down_sync(0xffffffffu, v.y, off);
    return v;
}
template <typename C> __device__ __forceinline__ C warp_sum(C v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = cadd(v, shfl_down(v, o));
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- operator
// Coefficients of one row of the scaled symmetric system (Section 2).  With
// ``vx`` = node on a vertical boundary line (i = 0 or n-1) and ``hy`` = node
// on a horizontal one (j = 0 or n-1):
//   coupling to x-neighbours  cx = -(1/h^2) * (hy ? 1/2 : 1)
//   coupling to y-neighbours  cy = -(1/h^2) * (vx ? 1/2 : 1)
//   diagonal = -(sum of couplings to neighbours inside the grid)
//              - kappa * (vx ? 1/2 : 1) * (hy ? 1/2 : 1)
//              - i sqrt(kappa)/h * (vx || hy)
// which for MP-2 is the ghost-node Sommerfeld row halved on edges and
// quartered at corners.  MP-1 uses the interior row everywhere (its boundary
// values are zero and are not unknowns).
struct OpDesc {
    int n;
    int bc;              // HZS_DIRICHLET / HZS_SOMMERFELD
    double inv_h2;       // 1/h^2
    double inv_h;        // 1/h
    double kappa0;       // constant kappa when kappa == nullptr
    const double* kappa; // n*n field or nullptr
};

__host__ __device__ __forceinline__ double op_kappa(const OpDesc& op, int i, int j) {
    return op.kappa ? op.kappa[(size_t)j * op.n + i] : op.kappa0;
}
__host__ __device__ __forceinline__ bool op_is_unknown(const OpDesc& op, int i, int j) {
    if (op.bc == HZS_SOMMERFELD) return true;
    return i > 0 && j > 0 && i < op.n - 1 && j < op.n - 1;
}
// coupling weights of node (i,j) in x and y directions
__host__ __device__ __forceinline__ double op_cx(const OpDesc& op, int j) {
    bool hy = op.bc == HZS_SOMMERFELD && (j == 0 || j == op.n - 1);
    return -op.inv_h2 * (hy ? 0.5 : 1.0);
}
__host__ __device__ __forceinline__ double op_cy(const OpDesc& op, int i) {
    bool vx = op.bc == HZS_SOMMERFELD && (i == 0 || i == op.n - 1);
    return -op.inv_h2 * (vx ? 0.5 : 1.0);
}
// diagonal entry for a given kappa at node (i, j)
__host__ __device__ __forceinline__ double2 op_diag_k(const OpDesc& op, int i, int j, double kap) {
    const int n = op.n;
    if (op.bc != HZS_SOMMERFELD) return make_double2(4.0 * op.inv_h2 - kap, 0.0);
    const bool vx = (i == 0 || i == n - 1), hy = (j == 0 || j == n - 1);
    const double cx = op_cx(op, j), cy = op_cy(op, i);
    double lap = 0.0;
    lap -= (i > 0 ? cx : 0.0) + (i < n - 1 ? cx : 0.0);
    lap -= (j > 0 ? cy : 0.0) + (j < n - 1 ? cy : 0.0);
    const double mass = (vx ? 0.5 : 1.0) * (hy ? 0.5 : 1.0);
    const double im = (vx || hy) ? -sqrt(kap) * op.inv_h : 0.0;
    return make_double2(lap - kap * mass, im);
}
__host__ __device__ __forceinline__ double2 op_diag(const OpDesc& op, int i, int j) {
    return op_diag_k(op, i, j, op_kappa(op, i, j));
}
// d A_PP / d kappa_P
__host__ __device__ __forceinline__ double2 op_ddiag_dkappa(const OpDesc& op, int i, int j) {
    const int n = op.n;
    if (op.bc != HZS_SOMMERFELD) return make_double2(-1.0, 0.0);
    const bool vx = (i == 0 || i == n - 1), hy = (j == 0 || j == n - 1);
    const double mass = (vx ? 0.5 : 1.0) * (hy ? 0.5 : 1.0);
    const double kap = op_kappa(op, i, j);
    const double im = (vx || hy) ? -0.5 / sqrt(kap) * op.inv_h : 0.0;
    return make_double2(-mass, im);
}

// ---------------------------------------------------------------- coarse tables
// 1-D coarse basis sampled at the fine nodes.  Fine node i touches coarse
// indices c0[i] .. c0[i]+2 (weights w[3*i + 0..2], zero where absent).
// Coarse index I has support fine nodes lo[I] .. hi[I] with weights
// wt[off[I] + (i - lo[I])].
struct CoarseTab {
    int nc1;            // coarse nodes per axis (kept)
    int max_sup;        // longest support hi - lo + 1 (sets the lanes per restricted value)
    int* c0;            // [n]
    double* w;          // [3n]
    float* wf;          // [3n]
    int* lo;            // [nc1]
    int* hi;            // [nc1]
    int* off;           // [nc1]
    double* wt;         // [sum support]
    float* wtf;         // the same weights in single precision (complex64 kernels use these,
                        // so that no FP64 instruction runs inside them)
};

// Coarse weights in the arithmetic precision R of a kernel.
template <typename R> struct CoarseW;
template <> struct CoarseW<double> {
    static __device__ __forceinline__ double w3(const CoarseTab& ct, int k) { return ct.w[k]; }
    static __device__ __forceinline__ double wt(const CoarseTab& ct, int k) { return ct.wt[k]; }
};
template <> struct CoarseW<float> {
    static __device__ __forceinline__ float w3(const CoarseTab& ct, int k) { return ct.wf[k]; }
    static __device__ __forceinline__ float wt(const CoarseTab& ct, int k) { return ct.wtf[k]; }
};

// ---------------------------------------------------------------- subdomain tiles
// A dense block W_j of a factor is stored row by row with the row length padded to
// an even count (the pad column holds zeros): every row, and every block, then
// starts on a 16-byte boundary in complex64 as well as complex128, as the bulk
// copies that stage the blocks and the paired 16-byte loads of the solve require.
__host__ __device__ __forceinline__ int block_ld(int mx) { return mx + (mx & 1); }
__host__ __device__ __forceinline__ long long block_stride(int mx) { return (long long)mx * block_ld(mx); }

struct Tile {
    int x0, y0;          // first grid node of the extended tile
    int mx, my;          // tile extent (unknowns)
    int ox0, ox1, oy0, oy1;  // owned node range (inclusive), grid indices
    int factor;          // index into the factor table
    int pad;
    long long woff;      // element offset of the factor's first block
    long long yoff;      // element offset of this tile's slot in tile-sized scratch
};

}  // namespace hzs
