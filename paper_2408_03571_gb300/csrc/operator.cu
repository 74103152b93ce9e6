// Operator kernels: y = A x (Eq. 3), the SHS2 deflated residual
// w = s v - A R_0^T c (Eq. 6, with the coarse solution c = A_0^{-1} R_0 s v
// already computed), the additive (D_i = I) combination of subdomain
// solutions, and the element-wise helpers of the solve driver.
//
// Kernels instantiated with R = float do all arithmetic in single precision
// (coarse weights and the coarse solution are read as float copies).
// Every kernel handles a batch of right-hand sides: batch entry r = blockIdx.z
// reads and writes its vectors at r times the stride given for each buffer,
// and is skipped when skip[r * skip_stride] is set.
#include "f32x2.cuh"
#include "kernels.cuh"

namespace hzs {

__device__ __forceinline__ bool skipped(const BatchSkip& sk, int r) {
    return sk.flag && sk.flag[(size_t)r * sk.stride];
}

// y = A x over the n x n grid.  Arithmetic in R; x read as Cin; y (if given)
// written as Cout; y32 (if given) receives the complex64 rounding of the
// result and y32lo (if set, see LoDst) the remainder, so that y32 + y32lo
// carries the result as a double-float pair.  MP-1 boundary nodes:
// y = 0, and their x values are never read.
template <typename Cin, typename Cout, typename R>
__global__ void k_apply_A(OpDesc op, const Cin* __restrict__ x, long long xs, Cout* __restrict__ y, long long ys,
                          float2* __restrict__ y32, long long y32s, LoDst y32lo, BatchSkip sk) {
    using C = cplx_t<R>;
    const int r = blockIdx.z;
    if (skipped(sk, r)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int n = op.n;
    if (i >= n || j >= n) return;
    x += r * xs;
    if (y) y += r * ys;
    if (y32) y32 += r * y32s;
    y32lo = y32lo.at(r * y32s);
    const size_t p = (size_t)j * n + i;
    if (!op_is_unknown(op, i, j)) {
        if (y) y[p] = mk<Cout>(0.0, 0.0);
        if (y32) y32[p] = make_float2(0.f, 0.f);
        y32lo.put(p, make_float2(0.f, 0.f));
        return;
    }
    const double2 d = op_diag(op, i, j);
    const R cx = (R)op_cx(op, j), cy = (R)op_cy(op, i);
    const C xp = conv<C>(x[p]);
    C acc;
    acc.x = (R)d.x * xp.x - (R)d.y * xp.y;
    acc.y = (R)d.x * xp.y + (R)d.y * xp.x;
    C sx; sx.x = 0; sx.y = 0;
    C sy; sy.x = 0; sy.y = 0;
    if (i > 0 && op_is_unknown(op, i - 1, j)) sx = cadd(sx, conv<C>(x[p - 1]));
    if (i < n - 1 && op_is_unknown(op, i + 1, j)) sx = cadd(sx, conv<C>(x[p + 1]));
    if (j > 0 && op_is_unknown(op, i, j - 1)) sy = cadd(sy, conv<C>(x[p - n]));
    if (j < n - 1 && op_is_unknown(op, i, j + 1)) sy = cadd(sy, conv<C>(x[p + n]));
    acc.x += cx * sx.x + cy * sy.x;
    acc.y += cx * sx.y + cy * sy.y;
    if (y) y[p] = conv<Cout>(acc);
    if (y32lo.any()) {
        const double2 a = to_d(acc);
        float2 hi, lo;
        split_d(a.x, hi.x, lo.x);
        split_d(a.y, hi.y, lo.y);
        y32[p] = hi;
        y32lo.put(p, lo);
    } else if (y32) {
        y32[p] = conv<float2>(acc);
    }
}

// y = A x for a complex64 x, in double-float arithmetic on the FP32 pipes (the
// FP64 rate is 1/62 of FP32 on GB300): y is written as the pair yh + yl
// (remainders wide or narrow, see LoDst).
// The couplings -1/h^2 (halved on Sommerfeld edges) are exact in FP32 for
// n <= 4097 (checked by the launcher); the diagonal is the double-float pair
// (dh, dl) for interior nodes of a constant-kappa grid and is otherwise formed
// in FP64 and split.  The neighbour sums are exact (TwoSum), every product is
// error-free (FMA form of Dekker's product), so y carries about 47 significant
// bits relative to the largest term of the stencil sum before the remainder is
// stored.
// FP32 -> FP64 by integer operations (exact, as the conversion instruction, which runs
// on the part's FP64 pipe): subnormal FP32 inputs take the conversion instruction.
__device__ __forceinline__ double f2d_exact(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu, sg = u & 0x80000000u;
    if (e == 0u) return m ? (double)x : __hiloint2double((int)sg, 0);
    const unsigned hi = sg | ((e == 0xffu ? 0x7ffu : e + 896u) << 20) | (m >> 3);
    return __hiloint2double((int)hi, (int)(m << 29));
}
__device__ __forceinline__ double2 f2d_exact2(float2 v) { return make_double2(f2d_exact(v.x), f2d_exact(v.y)); }

// y = A x for a complex64 x with the FP64 arithmetic of k_apply_A<float2, double2, double>
// (the same operations in the same order, so the same FP64 values), stored as f53 (an
// FP32 head and a 29-bit tail, see f32x2.cuh): the outer product of the mixed solve
// written straight into the Krylov slot it fills.
__global__ void k_apply_A_f53(OpDesc op, const float2* __restrict__ x, long long xs, float2* __restrict__ yh,
                              uint2* __restrict__ yt, long long ys, BatchSkip sk) {
    const int r = blockIdx.z;
    if (skipped(sk, r)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int n = op.n;
    if (i >= n || j >= n) return;
    x += r * xs;
    yh += r * ys;
    yt += r * ys;
    const size_t p = (size_t)j * n + i;
    if (!op_is_unknown(op, i, j)) {
        yh[p] = make_float2(0.f, 0.f);
        yt[p] = make_uint2(0u, 0u);
        return;
    }
    const double2 d = op_diag(op, i, j);
    const double cx = op_cx(op, j), cy = op_cy(op, i);
    const double2 xp = f2d_exact2(x[p]);
    double2 acc;
    acc.x = d.x * xp.x - d.y * xp.y;
    acc.y = d.x * xp.y + d.y * xp.x;
    double2 sx = make_double2(0.0, 0.0), sy = make_double2(0.0, 0.0);
    if (i > 0 && op_is_unknown(op, i - 1, j)) sx = cadd(sx, f2d_exact2(x[p - 1]));
    if (i < n - 1 && op_is_unknown(op, i + 1, j)) sx = cadd(sx, f2d_exact2(x[p + 1]));
    if (j > 0 && op_is_unknown(op, i, j - 1)) sy = cadd(sy, f2d_exact2(x[p - n]));
    if (j < n - 1 && op_is_unknown(op, i, j + 1)) sy = cadd(sy, f2d_exact2(x[p + n]));
    acc.x += cx * sx.x + cy * sy.x;
    acc.y += cx * sx.y + cy * sy.y;
    float2 h;
    uint2 t;
    f53_encode(acc.x, h.x, t.x);
    f53_encode(acc.y, h.y, t.y);
    yh[p] = h;
    yt[p] = t;
}

__global__ void k_apply_A_df(OpDesc op, float ch, float dh, float dl, const float2* __restrict__ x, long long xs,
                             float2* __restrict__ yh, LoDst yl, long long ys, BatchSkip sk) {
    const int r = blockIdx.z;
    if (skipped(sk, r)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int n = op.n;
    if (i >= n || j >= n) return;
    x += r * xs; yh += r * ys; yl = yl.at(r * ys);
    const size_t p = (size_t)j * n + i;
    if (!op_is_unknown(op, i, j)) {
        yh[p] = make_float2(0.f, 0.f);
        yl.put(p, make_float2(0.f, 0.f));
        return;
    }
    const bool edge_x = i == 0 || i == n - 1, edge_y = j == 0 || j == n - 1;
    float drh = dh, drl = dl, dih = 0.f, dil = 0.f;
    float cx = ch, cy = ch;
    if (op.bc == HZS_SOMMERFELD) {
        if (edge_y) cx *= 0.5f;
        if (edge_x) cy *= 0.5f;
    }
    if (op.kappa || edge_x || edge_y) {
        const double2 d = op_diag(op, i, j);
        split_d(d.x, drh, drl);
        split_d(d.y, dih, dil);
    }
    const float2 xp = x[p];
    const float2 z = make_float2(0.f, 0.f);
    const float2 a = (i > 0 && op_is_unknown(op, i - 1, j)) ? x[p - 1] : z;
    const float2 b = (i < n - 1 && op_is_unknown(op, i + 1, j)) ? x[p + 1] : z;
    const float2 c = (j > 0 && op_is_unknown(op, i, j - 1)) ? x[p - n] : z;
    const float2 e = (j < n - 1 && op_is_unknown(op, i, j + 1)) ? x[p + n] : z;
    float sxr, sxrl, sxi, sxil, syr, syrl, syi, syil;
    two_sum(a.x, b.x, sxr, sxrl);
    two_sum(a.y, b.y, sxi, sxil);
    two_sum(c.x, e.x, syr, syrl);
    two_sum(c.y, e.y, syi, syil);
    float reh = 0.f, rel = 0.f, imh = 0.f, iml = 0.f;
    df_fma(reh, rel, drh, drl, xp.x, 0.f);
    df_fma(reh, rel, -dih, -dil, xp.y, 0.f);
    df_fma(reh, rel, cx, 0.f, sxr, sxrl);
    df_fma(reh, rel, cy, 0.f, syr, syrl);
    df_fma(imh, iml, drh, drl, xp.y, 0.f);
    df_fma(imh, iml, dih, dil, xp.x, 0.f);
    df_fma(imh, iml, cx, 0.f, sxi, sxil);
    df_fma(imh, iml, cy, 0.f, syi, syil);
    df_norm(reh, rel);
    df_norm(imh, iml);
    yh[p] = make_float2(reh, imh);
    yl.put(p, make_float2(rel, iml));
}

// q(i, j) = sum_{a,b} wx(i,a) wy(j,b) c[(c0[j]+b) nc1 + c0[i]+a]   (prolongation R_0^T c)
template <typename R>
__device__ __forceinline__ cplx_t<R> prolong_at(const CoarseTab& ct, const cplx_t<R>* __restrict__ c, int i, int j) {
    using C = cplx_t<R>;
    C q; q.x = 0; q.y = 0;
    const int ci = ct.c0[i], cj = ct.c0[j];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const R wyb = CoarseW<R>::w3(ct, 3 * j + b);
        if (wyb == (R)0) continue;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const R wxa = CoarseW<R>::w3(ct, 3 * i + a);
            if (wxa == (R)0) continue;
            const C cv = c[(size_t)(cj + b) * ct.nc1 + (ci + a)];
            const R wgt = wxa * wyb;
            q.x += wgt * cv.x;
            q.y += wgt * cv.y;
        }
    }
    return q;
}

// w = s v - A q with q = R_0^T c evaluated on the fly; s = vscale[r * vss] (or 1).
// Block tile TX x TY nodes; q for the tile plus a one-node halo is staged in
// shared memory.
template <typename Cv, typename Cw, typename R, int TX, int TY>
__global__ void k_deflate(OpDesc op, CoarseTab ct, const cplx_t<R>* __restrict__ c, long long cs,
                          const Cv* __restrict__ v, long long vs, const double* __restrict__ vscale, long long vss,
                          Cw* __restrict__ w, long long ws, BatchSkip sk, R ch, R dint) {
    using C = cplx_t<R>;
    const int r = blockIdx.z;
    if (skipped(sk, r)) return;
    c += r * cs; v += r * vs; w += r * ws;
    __shared__ C qs[TY + 2][TX + 2];
    const int n = op.n;
    const int bx = blockIdx.x * TX, by = blockIdx.y * TY;
    for (int t = threadIdx.y * TX + threadIdx.x; t < (TX + 2) * (TY + 2); t += TX * TY) {
        const int li = t % (TX + 2), lj = t / (TX + 2);
        const int gi = bx + li - 1, gj = by + lj - 1;
        C q; q.x = 0; q.y = 0;
        if (gi >= 0 && gj >= 0 && gi < n && gj < n && op_is_unknown(op, gi, gj)) q = prolong_at<R>(ct, c, gi, gj);
        qs[lj][li] = q;
    }
    __syncthreads();
    const int i = bx + threadIdx.x, j = by + threadIdx.y;
    if (i >= n || j >= n) return;
    const size_t p = (size_t)j * n + i;
    if (!op_is_unknown(op, i, j)) { w[p] = mk<Cw>(0.0, 0.0); return; }
    const R s = vscale ? (R)vscale[r * vss] : (R)1;
    C d;
    R cx, cy;
    if (sizeof(R) == sizeof(float)) {
        // single precision: coefficients from the FP32 constants, FP64 only where the
        // diagonal varies (kappa field, Sommerfeld edges)
        const bool ex = i == 0 || i == n - 1, ey = j == 0 || j == n - 1;
        cx = ch; cy = ch;
        if (op.bc == HZS_SOMMERFELD) {
            if (ey) cx *= (R)0.5;
            if (ex) cy *= (R)0.5;
        }
        if (op.kappa || ex || ey) {
            const double2 dd = op_diag(op, i, j);
            d.x = (R)dd.x; d.y = (R)dd.y;
        } else {
            d.x = dint; d.y = 0;
        }
    } else {
        const double2 dd = op_diag(op, i, j);
        d.x = (R)dd.x; d.y = (R)dd.y;
        cx = (R)op_cx(op, j); cy = (R)op_cy(op, i);
    }
    const int li = threadIdx.x + 1, lj = threadIdx.y + 1;
    const C qp = qs[lj][li];
    C aq;
    aq.x = (R)d.x * qp.x - (R)d.y * qp.y;
    aq.y = (R)d.x * qp.y + (R)d.y * qp.x;
    // neighbours outside the grid or not unknowns hold q = 0 in the halo
    const C sx = cadd(qs[lj][li - 1], qs[lj][li + 1]);
    const C sy = cadd(qs[lj - 1][li], qs[lj + 1][li]);
    aq.x += cx * sx.x + cy * sy.x;
    aq.y += cx * sx.y + cy * sy.y;
    const C vp = conv<C>(v[p]);
    C out;
    out.x = s * vp.x - aq.x;
    out.y = s * vp.y - aq.y;
    w[p] = conv<Cw>(out);
}

// z = [q] + sum over the subdomains covering the node of y_tile (D_i = I:
// AS1 and AS2).  Per axis a node lies in at most two extended blocks;
// cover[i] = (block a, offset of i in a, block b, offset in b), -1 if absent.
template <typename Cz, typename Cy, typename R>
__global__ void k_combine_additive(OpDesc op, CoarseTab ct, const cplx_t<R>* __restrict__ c, long long cs,
                                   int use_coarse, const int4* __restrict__ cover_x,
                                   const int4* __restrict__ cover_y, const Tile* __restrict__ tiles, int nsx,
                                   const Cy* __restrict__ ytiles, long long yts, Cz* __restrict__ z, long long zs,
                                   BatchSkip sk, int weighted) {
    using C = cplx_t<R>;
    const int r = blockIdx.z;
    if (skipped(sk, r)) return;
    c += r * cs; ytiles += r * yts; z += r * zs;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int n = op.n;
    if (i >= n || j >= n) return;
    const size_t p = (size_t)j * n + i;
    if (!op_is_unknown(op, i, j)) { z[p] = mk<Cz>(0.0, 0.0); return; }
    C acc; acc.x = 0; acc.y = 0;
    const int4 cxv = cover_x[i], cyv = cover_y[j];
    const int ta[2] = {cxv.x, cxv.z}, la[2] = {cxv.y, cxv.w};
    const int tb[2] = {cyv.x, cyv.z}, lb[2] = {cyv.y, cyv.w};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        if (tb[u] < 0) continue;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (ta[s] < 0) continue;
            const Tile& T = tiles[tb[u] * nsx + ta[s]];
            acc = cadd(acc, conv<C>(ytiles[T.yoff + (size_t)lb[u] * T.mx + la[s]]));
        }
    }
    if (weighted) {
        // D_i = 1 / (number of subdomains containing the node)
        const int m = ((ta[0] >= 0) + (ta[1] >= 0)) * ((tb[0] >= 0) + (tb[1] >= 0));
        const R inv = (R)1 / (R)m;
        acc.x *= inv; acc.y *= inv;
    }
    if (use_coarse) acc = cadd(acc, prolong_at<R>(ct, c, i, j));
    z[p] = conv<Cz>(acc);
}

// dst = src (or conj(src)) on unknowns, 0 on MP-1 boundary nodes; dst32 (if
// given) receives the same values in complex64 and dst32lo (if set, see
// LoDst) the remainders of the double-float pairs.
__global__ void k_mask_copy(OpDesc op, const double2* __restrict__ src, long long ss, double2* __restrict__ dst,
                            long long ds, int conj, float2* __restrict__ dst32, long long d32s, LoDst dst32lo) {
    const int r = blockIdx.z;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int n = op.n;
    if (i >= n || j >= n) return;
    src += r * ss; dst += r * ds;
    const size_t p = (size_t)j * n + i;
    double2 v = op_is_unknown(op, i, j) ? src[p] : make_double2(0.0, 0.0);
    if (conj) v.y = -v.y;
    dst[p] = v;
    if (dst32lo.any()) {
        float2 hi, lo;
        split_d(v.x, hi.x, lo.x);
        split_d(v.y, hi.y, lo.y);
        dst32[r * d32s + p] = hi;
        dst32lo.put(r * d32s + p, lo);
    } else if (dst32) {
        dst32[r * d32s + p] = to_f(v);
    }
}

// grad = -Re(conj(lam) * dA_PP/dkappa_P * u) on unknowns, 0 elsewhere.
__global__ void k_kappa_gradient(OpDesc op, const double2* __restrict__ u, const double2* __restrict__ lam,
                                 double* __restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int n = op.n;
    if (i >= n || j >= n) return;
    const size_t p = (size_t)j * n + i;
    if (!op_is_unknown(op, i, j)) { grad[p] = 0.0; return; }
    const double2 d = op_ddiag_dkappa(op, i, j);
    const double2 du = cmul(d, u[p]);
    const double2 l = lam[p];
    // Re(conj(l) * du) = l.x du.x + l.y du.y
    grad[p] = -(l.x * du.x + l.y * du.y);
}

// ------------------------------------------------------------------ launchers
static inline dim3 grid2d(int n, dim3 b, int nb) {
    return dim3((n + b.x - 1) / b.x, (n + b.y - 1) / b.y, nb);
}

template <typename Cin, typename Cout, typename R>
void launch_apply_A(const Ctx& cx, int nb, const Cin* x, long long xs, Cout* y, long long ys, float2* y32,
                    long long y32s, BatchSkip sk, LoDst y32lo) {
    const dim3 b(32, 8);
    k_apply_A<Cin, Cout, R><<<grid2d(cx.op.n, b, nb), b, 0, cx.stream>>>(cx.op, x, xs, y, ys, y32, y32s, y32lo, sk);
}
template void launch_apply_A<double2, double2, double>(const Ctx&, int, const double2*, long long, double2*,
                                                       long long, float2*, long long, BatchSkip, LoDst);
template void launch_apply_A<float2, double2, double>(const Ctx&, int, const float2*, long long, double2*, long long,
                                                      float2*, long long, BatchSkip, LoDst);

void launch_apply_A_f53(const Ctx& cx, int nb, const float2* x, long long xs, float2* yh, uint2* yt, long long ys,
                        BatchSkip sk) {
    const dim3 b(32, 8);
    k_apply_A_f53<<<grid2d(cx.op.n, b, nb), b, 0, cx.stream>>>(cx.op, x, xs, yh, yt, ys, sk);
}

bool launch_apply_A_df(const Ctx& cx, int nb, const float2* x, long long xs, float2* yh, LoDst yl, long long ys,
                       BatchSkip sk) {
    const double ch = -cx.op.inv_h2;
    if ((double)(float)ch != ch) return false;                  // coupling not exact in FP32
    float dh = 0.f, dl = 0.f;
    if (!cx.op.kappa) {
        const double d = 4.0 * cx.op.inv_h2 - cx.op.kappa0;     // interior diagonal, constant kappa
        dh = (float)d;
        dl = (float)(d - (double)dh);
    }
    const dim3 b(32, 8);
    k_apply_A_df<<<grid2d(cx.op.n, b, nb), b, 0, cx.stream>>>(cx.op, (float)ch, dh, dl, x, xs, yh, yl, ys, sk);
    return true;
}

template <typename Cv, typename Cw, typename R>
void launch_deflate(const Ctx& cx, int nb, const cplx_t<R>* c, long long cs, const Cv* v, long long vs,
                    const double* vscale, long long vss, Cw* w, long long ws, BatchSkip sk) {
    constexpr int TX = 32, TY = 8;
    const dim3 b(TX, TY);
    // -1/h^2 and the constant-kappa interior diagonal 4/h^2 - kappa, rounded once
    const R ch = (R)(-cx.op.inv_h2), dint = (R)(4.0 * cx.op.inv_h2 - cx.op.kappa0);
    k_deflate<Cv, Cw, R, TX, TY><<<grid2d(cx.op.n, b, nb), b, 0, cx.stream>>>(cx.op, cx.ct, c, cs, v, vs, vscale, vss,
                                                                              w, ws, sk, ch, dint);
}
#define HZS_DEF(Cv, Cw, R)                                                                                     \
    template void launch_deflate<Cv, Cw, R>(const Ctx&, int, const cplx_t<R>*, long long, const Cv*, long long, \
                                            const double*, long long, Cw*, long long, BatchSkip);
HZS_DEF(double2, double2, double)
HZS_DEF(double2, float2, float)
HZS_DEF(float2, float2, float)
#undef HZS_DEF

template <typename Cz, typename Cy, typename R>
void launch_combine_additive(const Ctx& cx, int nb, const cplx_t<R>* c, long long cs, int use_coarse,
                             const int4* cover_x, const int4* cover_y, const Tile* tiles, int nsx, const Cy* ytiles,
                             long long yts, Cz* z, long long zs, BatchSkip sk, int weighted) {
    const dim3 b(32, 8);
    k_combine_additive<Cz, Cy, R><<<grid2d(cx.op.n, b, nb), b, 0, cx.stream>>>(
        cx.op, cx.ct, c, cs, use_coarse, cover_x, cover_y, tiles, nsx, ytiles, yts, z, zs, sk, weighted);
}
#define HZS_CMB(Cz, Cy, R)                                                                                     \
    template void launch_combine_additive<Cz, Cy, R>(const Ctx&, int, const cplx_t<R>*, long long, int,       \
                                                     const int4*, const int4*, const Tile*, int, const Cy*,     \
                                                     long long, Cz*, long long, BatchSkip, int);
HZS_CMB(double2, double2, double)
HZS_CMB(float2, float2, float)
#undef HZS_CMB

void launch_mask_copy_c128(const Ctx& cx, int nb, const double2* src, long long ss, double2* dst, long long ds,
                           int conj, float2* dst32, long long d32s, LoDst dst32lo) {
    const dim3 b(32, 8);
    k_mask_copy<<<grid2d(cx.op.n, b, nb), b, 0, cx.stream>>>(cx.op, src, ss, dst, ds, conj, dst32, d32s, dst32lo);
}

void launch_kappa_gradient(const Ctx& cx, const double2* u, const double2* lam, double* grad) {
    const dim3 b(32, 8);
    k_kappa_gradient<<<grid2d(cx.op.n, b, 1), b, 0, cx.stream>>>(cx.op, u, lam, grad);
}

}  // namespace hzs
