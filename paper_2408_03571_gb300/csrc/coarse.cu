// Coarse level (Section 4, Eq. 4): the 1-D P_1 / B_2 tables, restriction
// c = R_0 v (separable, two passes), the Galerkin matrix A_0 = R_0 A R_0^T,
// its FP64 Gauss-Jordan inverse and the coarse solve c' = A_0^{-1} c.
#include <cmath>
#include <vector>

#include "kernels.cuh"

namespace hzs {

// ------------------------------------------------------------------ 1-D tables
// Cardinal quadratic B-spline on [0, 3].
static double bspline2(double t) {
    if (t < 0.0 || t > 3.0) return 0.0;
    if (t < 1.0) return 0.5 * t * t;
    if (t < 2.0) return 0.5 * (-2.0 * t * t + 6.0 * t - 3.0);
    const double u = 3.0 - t;
    return 0.5 * u * u;
}

// phi_I at fine node i for coarse ratio p.  B_2: B-spline of knot spacing
// H = p h centred on X_I (for p = 2 the weights (1,4,6,4,1)/8 of Eq. 7);
// P_1: hat of half-width H.
static double basis_value(int kind, int I_node, int i, int p) {
    const double s = (double)(i - I_node * p) / (double)p;   // (x_i - X_I) / H
    if (kind == HZS_COARSE_B2) return bspline2(s + 1.5);
    const double a = std::fabs(s);
    return a < 1.0 ? 1.0 - a : 0.0;
}

void build_coarse_tables(int n, int bc, int kind, int p, HostCoarseTab& t) {
    const int ncoarse_all = (n - 1) / p + 1;
    const int first = (bc == HZS_DIRICHLET) ? 1 : 0;          // MP-1 drops the coarse boundary nodes
    const int nc1 = (bc == HZS_DIRICHLET) ? ncoarse_all - 2 : ncoarse_all;
    const int flo = (bc == HZS_DIRICHLET) ? 1 : 0, fhi = (bc == HZS_DIRICHLET) ? n - 2 : n - 1;
    t.nc1 = nc1;
    t.c0.assign(n, 0);
    t.w.assign(3 * n, 0.0);
    t.lo.assign(nc1, 0); t.hi.assign(nc1, -1); t.off.assign(nc1, 0);
    t.wt.clear();
    for (int I = 0; I < nc1; ++I) {
        const int node = I + first;
        int lo = -1, hi = -2;
        for (int i = flo; i <= fhi; ++i) {
            if (basis_value(kind, node, i, p) != 0.0) { if (lo < 0) lo = i; hi = i; }
        }
        t.off[I] = (int)t.wt.size();
        t.lo[I] = lo; t.hi[I] = hi;
        for (int i = lo; lo >= 0 && i <= hi; ++i) t.wt.push_back(basis_value(kind, node, i, p));
    }
    // per fine node: first touching coarse index (clamped so c0+2 < nc1 where possible)
    for (int i = 0; i < n; ++i) {
        if (i < flo || i > fhi) { t.c0[i] = 0; continue; }
        int first_I = -1;
        for (int I = 0; I < nc1; ++I)
            if (basis_value(kind, I + first, i, p) != 0.0) { first_I = I; break; }
        if (first_I < 0) { t.c0[i] = 0; continue; }
        int c0 = first_I;
        if (c0 + 2 >= nc1) c0 = nc1 - 3 < 0 ? 0 : nc1 - 3;
        if (c0 > first_I) c0 = first_I;
        t.c0[i] = c0;
        for (int a = 0; a < 3; ++a) {
            const int I = c0 + a;
            t.w[3 * i + a] = (I < nc1) ? basis_value(kind, I + first, i, p) : 0.0;
        }
        // every touching coarse index must be inside the 3-wide window
        for (int I = 0; I < nc1; ++I)
            if (basis_value(kind, I + first, i, p) != 0.0 && (I < c0 || I > c0 + 2)) t.bad = 1;
    }
}

// ------------------------------------------------------------------ restriction
// t[j * nc1 + I] = s * sum_{i in supp I} phi_I(x_i) v[j n + i]   (x pass)
// G lanes per restricted value (G divides 32; G is about a quarter of the support, so
// the lanes stay busy for the short supports of H = 4h and the wide ones of H = 32h);
// consecutive groups take consecutive I of the same fine row, whose supports overlap.
template <typename Cv, typename R, int G>
__global__ void k_restrict_x(int n, CoarseTab ct, const Cv* __restrict__ v, long long vs,
                             const double* __restrict__ vscale, long long vss, cplx_t<R>* __restrict__ t,
                             BatchSkip sk) {
    using C = cplx_t<R>;
    const int r = blockIdx.y;
    if (sk.flag && sk.flag[(size_t)r * sk.stride]) return;
    const int nc1 = ct.nc1;
    const long long o = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int sub = threadIdx.x % G;
    const bool ok = o < (long long)n * nc1;
    v += r * vs;
    t += (size_t)r * n * nc1;
    C acc; acc.x = 0; acc.y = 0;
    if (ok) {
        const int j = (int)(o / nc1), I = (int)(o % nc1);
        const int lo = ct.lo[I], hi = ct.hi[I];
        const int off = ct.off[I];
        const Cv* row = v + (size_t)j * n;
        for (int i = lo + sub; i <= hi; i += G) {
            const R wgt = CoarseW<R>::wt(ct, off + i - lo);
            const C x = conv<C>(row[i]);
            acc.x += wgt * x.x; acc.y += wgt * x.y;
        }
    }
#pragma unroll
    for (int m = G / 2; m > 0; m >>= 1) {        // every lane of the warp takes part
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, m);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, m);
    }
    if (ok && sub == 0) {
        const R s = vscale ? (R)vscale[r * vss] : (R)1;
        acc.x *= s; acc.y *= s;
        t[o] = acc;
    }
}

// c[J * nc1 + I] = sum_{j in supp J} phi_J(y_j) t[j * nc1 + I]   (y pass, FP64 result);
// G lanes per value as in the x pass: lane sub of consecutive groups reads consecutive I
// of the same row j, so the loads coalesce across the groups of a warp.
template <typename R, int G>
__global__ void k_restrict_y(int n, CoarseTab ct, const cplx_t<R>* __restrict__ t, double2* __restrict__ c,
                             BatchSkip sk) {
    const int r = blockIdx.y;
    if (sk.flag && sk.flag[(size_t)r * sk.stride]) return;
    const int nc1 = ct.nc1;
    const long long o = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int sub = threadIdx.x % G;
    const bool ok = o < (long long)nc1 * nc1;
    t += (size_t)r * n * nc1;
    c += (size_t)r * nc1 * nc1;
    double2 acc = make_double2(0.0, 0.0);
    if (ok) {
        const int J = (int)(o / nc1), I = (int)(o % nc1);
        const int lo = ct.lo[J], hi = ct.hi[J];
        const int off = ct.off[J];
        for (int j = lo + sub; j <= hi; j += G) {
            const double wgt = ct.wt[off + j - lo];
            const double2 x = to_d(t[(size_t)j * nc1 + I]);
            acc.x += wgt * x.x; acc.y += wgt * x.y;
        }
    }
#pragma unroll
    for (int m = G / 2; m > 0; m >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, m);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, m);
    }
    if (ok && sub == 0) c[o] = acc;
}

// ------------------------------------------------------------------ coarse solve
// out = Ainv * c (dense, FP64; outf, if given, gets its complex64 rounding).
// kCmvWarpsPerRow warps share a row (the matrix, 16 B per entry, is re-read from
// DRAM every apply: the basis passes evict it from L2, so each lane keeps kCmvLoads
// loads in flight); c staged in shared memory.
constexpr int kCmvWarpsPerRow = 4;
constexpr int kCmvLoads = 8;
constexpr int kCmvThreads = 512;
__global__ void __launch_bounds__(kCmvThreads) k_coarse_matvec(int Nc, const double2* __restrict__ Ainv,
                                                               const double2* __restrict__ c,
                                                               double2* __restrict__ out, float2* __restrict__ outf,
                                                               BatchSkip sk) {
    const int r = blockIdx.y;
    if (sk.flag && sk.flag[(size_t)r * sk.stride]) return;
    c += (size_t)r * Nc;
    out += (size_t)r * Nc;
    if (outf) outf += (size_t)r * Nc;
    extern __shared__ double2 cs[];
    __shared__ double2 part[kCmvThreads / 32];
    for (int k = threadIdx.x; k < Nc; k += blockDim.x) cs[k] = c[k];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = warp % kCmvWarpsPerRow;                 // this warp's share of the row
    const int rows_per_block = (kCmvThreads / 32) / kCmvWarpsPerRow;
    const int row = blockIdx.x * rows_per_block + warp / kCmvWarpsPerRow;
    double2 acc = make_double2(0.0, 0.0), acc2 = acc;
    if (row < Nc) {
        const double2* arow = Ainv + (size_t)row * Nc;
        constexpr int span = 32 * kCmvWarpsPerRow * kCmvLoads;   // columns per round of the row's warps
        for (int k0 = 0; k0 < Nc; k0 += span) {
            double2 a[kCmvLoads];
#pragma unroll
            for (int q = 0; q < kCmvLoads; ++q) {
                const int k = k0 + 32 * (sub + kCmvWarpsPerRow * q) + lane;
                a[q] = k < Nc ? arow[k] : make_double2(0.0, 0.0);
            }
#pragma unroll
            for (int q = 0; q < kCmvLoads; q += 2) {
                const int k = k0 + 32 * (sub + kCmvWarpsPerRow * q) + lane;
                const int k2 = k + 32 * kCmvWarpsPerRow;
                acc = cfma(a[q], k < Nc ? cs[k] : make_double2(0.0, 0.0), acc);
                acc2 = cfma(a[q + 1], k2 < Nc ? cs[k2] : make_double2(0.0, 0.0), acc2);
            }
        }
    }
    acc = warp_sum(cadd(acc, acc2));
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (sub == 0 && lane == 0 && row < Nc) {
        double2 s = part[warp];
        for (int q = 1; q < kCmvWarpsPerRow; ++q) s = cadd(s, part[warp + q]);
        out[row] = s;
        if (outf) outf[row] = to_f(s);
    }
}

// ------------------------------------------------------------------ Galerkin A_0
// A0[(J,I), (J+dJ, I+dI)] = sum_{fine (i,j)} phi_I(i) phi_J(j) (A phi_{I+dI, J+dJ})(i, j)
// One block per (row, offset) pair; offsets |dI|, |dJ| <= 2 cover B_2 (P_1 uses <= 1).
__global__ void k_galerkin(OpDesc op, CoarseTab ct, double2* __restrict__ A0, int banded) {
    const int nc1 = ct.nc1;
    const int row = blockIdx.x;
    const int o = blockIdx.y;              // 0..24
    const int dI = o % 5 - 2, dJ = o / 5 - 2;
    const int I = row % nc1, J = row / nc1;
    const int I2 = I + dI, J2 = J + dJ;
    if (I2 < 0 || J2 < 0 || I2 >= nc1 || J2 >= nc1) return;
    const int ilo = ct.lo[I], ihi = ct.hi[I], jlo = ct.lo[J], jhi = ct.hi[J];
    if (ilo < 0 || jlo < 0) return;
    const int w = ihi - ilo + 1, hgt = jhi - jlo + 1;
    // phi_{I2}(i) with support check
    auto phi = [&](int K, int i) -> double {
        if (i < ct.lo[K] || i > ct.hi[K]) return 0.0;
        return ct.wt[ct.off[K] + i - ct.lo[K]];
    };
    double2 acc = make_double2(0.0, 0.0);
    for (int t = threadIdx.x; t < w * hgt; t += blockDim.x) {
        const int i = ilo + t % w, j = jlo + t / w;
        if (!op_is_unknown(op, i, j)) continue;
        const double a = ct.wt[ct.off[I] + i - ilo] * ct.wt[ct.off[J] + j - jlo];
        if (a == 0.0) continue;
        // (A phi2)(i, j)
        const double2 d = op_diag(op, i, j);
        const double p0 = phi(I2, i) * phi(J2, j);
        double re = d.x * p0, im = d.y * p0;
        const double cx = op_cx(op, j), cy = op_cy(op, i);
        double nb = 0.0;
        if (i > 0 && op_is_unknown(op, i - 1, j)) nb += cx * phi(I2, i - 1) * phi(J2, j);
        if (i < op.n - 1 && op_is_unknown(op, i + 1, j)) nb += cx * phi(I2, i + 1) * phi(J2, j);
        if (j > 0 && op_is_unknown(op, i, j - 1)) nb += cy * phi(I2, i) * phi(J2, j - 1);
        if (j < op.n - 1 && op_is_unknown(op, i, j + 1)) nb += cy * phi(I2, i) * phi(J2, j + 1);
        re += nb;
        acc.x += a * re; acc.y += a * im;
    }
    __shared__ double2 red[32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double2 v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : make_double2(0.0, 0.0);
        v = warp_sum(v);
        if (threadIdx.x == 0) {
            if (banded) A0[(size_t)row * 25 + o] = v;
            else A0[(size_t)row * (nc1 * nc1) + (size_t)J2 * nc1 + I2] = v;
        }
    }
}

// ------------------------------------------------------------------ Gauss-Jordan inverse
// In-place inversion with partial pivoting of a dense N x N complex matrix in
// global memory, one pivot column per step.
struct GJState {
    int piv;          // pivot row of the current step
    int singular;     // set if a pivot was zero or not finite
    double minpiv;    // smallest |pivot| seen
    double2 pivval;   // pivot value of the current step
};

__global__ void k_gj_pivot(int N, int k, const double2* __restrict__ a, int* __restrict__ perm, GJState* st) {
    // one block: argmax_{r >= k} |a[r][k]|
    __shared__ double bv[32];
    __shared__ int bi[32];
    double best = -1.0; int bidx = k;
    for (int r = k + threadIdx.x; r < N; r += blockDim.x) {
        const double2 v = a[(size_t)r * N + k];
        const double m = hypot(v.x, v.y);
        if (m > best) { best = m; bidx = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bidx, o);
        if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = bidx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (bv[w] > bv[0] || (bv[w] == bv[0] && bi[w] < bi[0])) { bv[0] = bv[w]; bi[0] = bi[w]; }
        st->piv = bi[0];
        st->pivval = a[(size_t)bi[0] * N + k];
        perm[k] = bi[0];
        if (!(bv[0] > 0.0) || !isfinite(bv[0])) st->singular = 1;
        if (bv[0] < st->minpiv) st->minpiv = bv[0];
    }
}

// swap rows k and piv, scale row k, save column k
__global__ void k_gj_swap_scale(int N, int k, double2* __restrict__ a, double2* __restrict__ colk, const GJState* st) {
    const int p = st->piv;
    const double2 pv = st->pivval;
    const double den = pv.x * pv.x + pv.y * pv.y;
    const double2 inv = den > 0.0 ? make_double2(pv.x / den, -pv.y / den) : make_double2(0.0, 0.0);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        double2 rk = a[(size_t)k * N + c], rp = a[(size_t)p * N + c];
        if (p != k) { const double2 tmp = rk; rk = rp; rp = tmp; a[(size_t)p * N + c] = rp; }
        // row k scaled; column k of row k becomes 1/pivot
        a[(size_t)k * N + c] = (c == k) ? inv : cmul(rk, inv);
    }
}

__global__ void k_gj_savecol(int N, int k, const double2* __restrict__ a, double2* __restrict__ colk) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < N; r += gridDim.x * blockDim.x)
        colk[r] = a[(size_t)r * N + k];
}

// a[r][c] -= colk[r] * a[k][c] for r != k; column k: a[r][k] = -colk[r] * a[k][k]
__global__ void k_gj_eliminate(int N, int k, double2* __restrict__ a, const double2* __restrict__ colk) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (c >= N || r == k) return;
    const double2 f = colk[r];
    const double2 akc = a[(size_t)k * N + c];
    double2 v = (c == k) ? make_double2(0.0, 0.0) : a[(size_t)r * N + c];
    v = cfms(f, akc, v);
    a[(size_t)r * N + c] = v;
}

// undo the row interchanges: swap columns k and perm[k] for k = N-1 .. 0
__global__ void k_gj_colswap(int N, int k, double2* __restrict__ a, const int* __restrict__ perm) {
    const int p = perm[k];
    if (p == k) return;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < N; r += gridDim.x * blockDim.x) {
        const double2 t = a[(size_t)r * N + k];
        a[(size_t)r * N + k] = a[(size_t)r * N + p];
        a[(size_t)r * N + p] = t;
    }
}

// ------------------------------------------------------------------ launchers
template <typename Cv, typename R, int G>
static void launch_restrict_g(const Ctx& cx, int nb, const Cv* v, long long vs, const double* vscale, long long vss,
                              cplx_t<R>* t, double2* c, BatchSkip sk) {
    const int n = cx.op.n, nc1 = cx.ct.nc1;
    const int threads = 256;
    {
        const long long lanes = (long long)n * nc1 * G;
        const dim3 grid((unsigned)((lanes + threads - 1) / threads), nb);
        k_restrict_x<Cv, R, G><<<grid, threads, 0, cx.stream>>>(n, cx.ct, v, vs, vscale, vss, t, sk);
    }
    {
        const long long lanes = (long long)nc1 * nc1 * G;
        const dim3 grid((unsigned)((lanes + threads - 1) / threads), nb);
        k_restrict_y<R, G><<<grid, threads, 0, cx.stream>>>(n, cx.ct, t, c, sk);
    }
}

template <typename Cv, typename R>
void launch_restrict(const Ctx& cx, int nb, const Cv* v, long long vs, const double* vscale, long long vss,
                     cplx_t<R>* t, double2* c, BatchSkip sk) {
    // lanes per restricted value: about a quarter of the longest support (3p - 1 fine
    // nodes for B_2 and 2p - 1 for P_1 at H = p h), at least 4
    if (cx.ct.max_sup <= 16)
        launch_restrict_g<Cv, R, 4>(cx, nb, v, vs, vscale, vss, t, c, sk);
    else if (cx.ct.max_sup <= 32)
        launch_restrict_g<Cv, R, 8>(cx, nb, v, vs, vscale, vss, t, c, sk);
    else
        launch_restrict_g<Cv, R, 32>(cx, nb, v, vs, vscale, vss, t, c, sk);
}
#define HZS_RS(Cv, R)                                                                                          \
    template void launch_restrict<Cv, R>(const Ctx&, int, const Cv*, long long, const double*, long long,     \
                                         cplx_t<R>*, double2*, BatchSkip);
HZS_RS(double2, double)
HZS_RS(double2, float)
HZS_RS(float2, float)
#undef HZS_RS

void launch_coarse_matvec(const Ctx& cx, int nb, const double2* Ainv, int Nc, const double2* c, double2* out,
                          float2* outf, BatchSkip sk) {
    const int rows_per_block = (kCmvThreads / 32) / kCmvWarpsPerRow;
    const int blocks = (Nc + rows_per_block - 1) / rows_per_block;   // one row per warp group, no grid stride
    const size_t smem = (size_t)Nc * sizeof(double2);
    allow_dynamic_smem((const void*)k_coarse_matvec, smem);
    k_coarse_matvec<<<dim3(blocks, nb), kCmvThreads, smem, cx.stream>>>(Nc, Ainv, c, out, outf, sk);
}

void launch_galerkin(const Ctx& cx, double2* A0) {
    const int nc1 = cx.ct.nc1;
    const int Nc = nc1 * nc1;
    cudaMemsetAsync(A0, 0, (size_t)Nc * Nc * sizeof(double2), cx.stream);
    dim3 grid(Nc, 25);
    k_galerkin<<<grid, 256, 0, cx.stream>>>(cx.op, cx.ct, A0, 0);
}

void launch_galerkin_banded(const Ctx& cx, double2* A0b) {
    const int nc1 = cx.ct.nc1;
    const int Nc = nc1 * nc1;
    cudaMemsetAsync(A0b, 0, (size_t)Nc * 25 * sizeof(double2), cx.stream);
    dim3 grid(Nc, 25);
    k_galerkin<<<grid, 256, 0, cx.stream>>>(cx.op, cx.ct, A0b, 1);
}

// Returns 0 on success, 1 if a pivot was zero; *minpiv receives min |pivot|.
int gj_invert(const Ctx& cx, double2* a, int N, double* minpiv) {
    double2* colk = nullptr; int* perm = nullptr; GJState* st = nullptr;
    if (cudaMalloc(&colk, N * sizeof(double2)) != cudaSuccess) return -1;
    if (cudaMalloc(&perm, N * sizeof(int)) != cudaSuccess) { cudaFree(colk); return -1; }
    if (cudaMalloc(&st, sizeof(GJState)) != cudaSuccess) { cudaFree(colk); cudaFree(perm); return -1; }
    GJState h0{0, 0, 1e300, make_double2(0.0, 0.0)};
    cudaMemcpyAsync(st, &h0, sizeof(GJState), cudaMemcpyHostToDevice, cx.stream);
    const int t = 256;
    const int cb = (N + t - 1) / t;
    for (int k = 0; k < N; ++k) {
        k_gj_pivot<<<1, 512, 0, cx.stream>>>(N, k, a, perm, st);
        k_gj_swap_scale<<<cb, t, 0, cx.stream>>>(N, k, a, colk, st);
        k_gj_savecol<<<cb, t, 0, cx.stream>>>(N, k, a, colk);
        k_gj_eliminate<<<dim3(cb, N), t, 0, cx.stream>>>(N, k, a, colk);
    }
    for (int k = N - 1; k >= 0; --k) k_gj_colswap<<<cb, t, 0, cx.stream>>>(N, k, a, perm);
    GJState h;
    cudaMemcpyAsync(&h, st, sizeof(GJState), cudaMemcpyDeviceToHost, cx.stream);
    cudaError_t e = cudaStreamSynchronize(cx.stream);
    cudaFree(colk); cudaFree(perm); cudaFree(st);
    if (e != cudaSuccess) return -1;
    *minpiv = h.minpiv;
    return h.singular ? 1 : 0;
}

}  // namespace hzs
