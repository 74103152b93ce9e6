// Exact subdomain solves A_i^{-1} (Section 3: "local problems ... solved using
// a sparse direct solver").  A subdomain tile of mx x my unknowns in
// lexicographic order is block tridiagonal: diagonal blocks T_j (tridiagonal,
// one grid row each) and diagonal couplings C between consecutive rows.
// Block LU (block Thomas) gives
//   S_0 = T_0,  S_j = T_j - C S_{j-1}^{-1} C,   W_j = S_j^{-1}
//   forward:  g_0 = W_0 b_0,  g_j = W_j (b_j - C g_{j-1})
//   backward: x_last = g_last,  x_j = g_j - W_j (C x_{j+1})
// The dense blocks W_j are inverted once in FP64 (Gauss-Jordan with partial
// pivoting inside each block) and stored; the solve is then 2 my dense
// mx x mx matrix-vector products per tile.
#include "kernels.cuh"

namespace hzs {

constexpr int kMaxTile = 112;   // largest tile extent per axis (an FP64 block fits in shared memory)
int max_tile_extent() { return kMaxTile; }

// ------------------------------------------------------------------ set-up
// One block per distinct factor; S (mx x mx complex double) lives in shared memory.
__global__ void __launch_bounds__(512) k_tile_factor(OpDesc op, const FactorDesc* __restrict__ fds,
                                                     double2* __restrict__ W64, float2* __restrict__ W32,
                                                     FactorStat* __restrict__ stats) {
    extern __shared__ double2 smem[];
    const FactorDesc fd = fds[blockIdx.x];
    const int m = fd.mx;
    double2* S = smem;                       // m*m
    double2* colk = S + m * m;               // m
    int* perm = reinterpret_cast<int*>(colk + m);
    __shared__ int s_piv_row;
    __shared__ double2 s_piv_val;
    __shared__ double s_minpiv, s_maxabs;
    __shared__ int s_singular;
    __shared__ double red_v[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    if (tid == 0) { s_minpiv = 1e300; s_maxabs = 0.0; s_singular = 0; }

    for (int j = 0; j < fd.my; ++j) {
        const int gy = fd.y0 + j;
        const double cxj = op_cx(op, gy);
        // S_j = T_j - C W_{j-1} C   (W_{j-1} is the current content of S)
        for (int t = tid; t < m * m; t += nt) {
            const int a = t / m, b = t % m;
            double2 v = make_double2(0.0, 0.0);
            if (j > 0) {
                const double s = op_cy(op, fd.x0 + a) * op_cy(op, fd.x0 + b);
                v = S[t];
                v.x = -s * v.x; v.y = -s * v.y;
            }
            if (a == b) {
                const double2 d = op_diag(op, fd.x0 + a, gy);
                v.x += d.x; v.y += d.y;
            } else if (a - b == 1 || b - a == 1) {
                v.x += cxj;
            }
            S[t] = v;
        }
        __syncthreads();
        // in-place Gauss-Jordan inversion with partial pivoting
        for (int k = 0; k < m; ++k) {
            if (wid == 0) {
                double best = -1.0; int bi = k;
                for (int r = k + lane; r < m; r += 32) {
                    const double2 v = S[r * m + k];
                    const double av = hypot(v.x, v.y);
                    if (av > best) { best = av; bi = r; }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const double ob = __shfl_down_sync(0xffffffffu, best, o);
                    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                }
                if (lane == 0) {
                    s_piv_row = bi; s_piv_val = S[bi * m + k];
                    perm[k] = bi;
                    if (!(best > 0.0) || !isfinite(best)) s_singular = 1;
                    if (best < s_minpiv) s_minpiv = best;
                }
            }
            __syncthreads();
            const int p = s_piv_row;
            const double2 pv = s_piv_val;
            const double den = pv.x * pv.x + pv.y * pv.y;
            const double2 inv = den > 0.0 ? make_double2(pv.x / den, -pv.y / den) : make_double2(0.0, 0.0);
            for (int c = tid; c < m; c += nt) {
                double2 rk = S[k * m + c];
                if (p != k) { const double2 rp = S[p * m + c]; S[p * m + c] = rk; rk = rp; }
                S[k * m + c] = (c == k) ? inv : cmul(rk, inv);
            }
            __syncthreads();
            for (int r = tid; r < m; r += nt) colk[r] = S[r * m + k];
            __syncthreads();
            for (int t = tid; t < m * m; t += nt) {
                const int r = t / m, c = t % m;
                if (r == k) continue;
                const double2 f = colk[r];
                double2 v = (c == k) ? make_double2(0.0, 0.0) : S[t];
                S[t] = cfms(f, S[k * m + c], v);
            }
            __syncthreads();
        }
        for (int k = m - 1; k >= 0; --k) {
            const int p = perm[k];
            if (p != k) {
                for (int r = tid; r < m; r += nt) {
                    const double2 t0 = S[r * m + k];
                    S[r * m + k] = S[r * m + p];
                    S[r * m + p] = t0;
                }
            }
            __syncthreads();
        }
        // store W_j
        double mx_abs = 0.0;
        double2* dst64 = W64 + fd.woff + (long long)j * m * m;
        float2* dst32 = W32 ? W32 + fd.woff + (long long)j * m * m : nullptr;
        for (int t = tid; t < m * m; t += nt) {
            const double2 v = S[t];
            dst64[t] = v;
            if (dst32) dst32[t] = to_f(v);
            mx_abs = fmax(mx_abs, hypot(v.x, v.y));
        }
        for (int o = 16; o > 0; o >>= 1) mx_abs = fmax(mx_abs, __shfl_down_sync(0xffffffffu, mx_abs, o));
        if (lane == 0) red_v[wid] = mx_abs;
        __syncthreads();
        if (tid == 0) {
            for (int w = 0; w < nw; ++w) s_maxabs = fmax(s_maxabs, red_v[w]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        stats[blockIdx.x].minpiv = s_minpiv;
        stats[blockIdx.x].maxabs = s_maxabs;
        stats[blockIdx.x].singular = s_singular;
    }
}

int launch_tile_factor(const Ctx& cx, const FactorDesc* fdesc_dev, int nfactors, int max_m, double2* W64,
                       float2* W32, FactorStat* stat_dev) {
    const size_t smem = (size_t)max_m * max_m * sizeof(double2) + (size_t)max_m * sizeof(double2) +
                        (size_t)max_m * sizeof(int) + 16;
    if (cudaFuncSetAttribute(k_tile_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    k_tile_factor<<<nfactors, 512, smem, cx.stream>>>(cx.op, fdesc_dev, W64, W32, stat_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ------------------------------------------------------------------ solve
// One block per tile.  The tile right-hand side b = R_i w is gathered into
// shared memory (g), swept forward and backward in place, and written out:
// mode 0 (restricted, D_i = owner indicator): z = [R_0^T c] + x on owned nodes;
// mode 1 (additive, D_i = I): the whole tile x into ytiles.
template <typename Cw, typename Cz, typename R>
__global__ void __launch_bounds__(256) k_tile_solve(OpDesc op, CoarseTab ct, const Tile* __restrict__ tiles,
                                                    const cplx_t<R>* __restrict__ W, const Cw* __restrict__ w,
                                                    const double* __restrict__ vscale, int mode, const double2* __restrict__ c, int use_coarse,
                                                    Cz* __restrict__ z, cplx_t<R>* __restrict__ ytiles,
                                                    const int* __restrict__ skip) {
    using C = cplx_t<R>;
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    const Tile T = tiles[blockIdx.x];
    const int mx = T.mx, my = T.my, n = op.n;
    C* g = reinterpret_cast<C*>(smem_raw);          // mx*my
    C* r = g + mx * my;                              // mx
    R* cy = reinterpret_cast<R*>(r + mx);            // mx
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    const double sc = vscale ? vscale[0] : 1.0;
    for (int t = tid; t < mx * my; t += nt) {
        const int a = t % mx, b = t / mx;
        double2 v = to_d(w[(size_t)(T.y0 + b) * n + (T.x0 + a)]);
        v.x *= sc; v.y *= sc;
        g[t] = cvt<C>(v);
    }
    for (int a = tid; a < mx; a += nt) cy[a] = (R)op_cy(op, T.x0 + a);
    __syncthreads();
    const C* Wt = W + T.woff;
    const size_t bs = (size_t)mx * mx;
    // forward sweep
    for (int j = 0; j < my; ++j) {
        C* gj = g + j * mx;
        for (int a = tid; a < mx; a += nt) {
            C v = gj[a];
            if (j > 0) { const C gp = gj[a - mx]; v.x -= cy[a] * gp.x; v.y -= cy[a] * gp.y; }
            r[a] = v;
        }
        __syncthreads();
        const C* Wj = Wt + j * bs;
        for (int row = wid; row < mx; row += nw) {
            C acc; acc.x = 0; acc.y = 0;
            const C* wr = Wj + (size_t)row * mx;
            for (int col = lane; col < mx; col += 32) acc = cfma(wr[col], r[col], acc);
            acc = warp_sum(acc);
            if (lane == 0) gj[row] = acc;
        }
        __syncthreads();
    }
    // backward sweep
    for (int j = my - 2; j >= 0; --j) {
        C* gj = g + j * mx;
        for (int a = tid; a < mx; a += nt) {
            const C xn = gj[a + mx];
            C v; v.x = cy[a] * xn.x; v.y = cy[a] * xn.y;
            r[a] = v;
        }
        __syncthreads();
        const C* Wj = Wt + j * bs;
        for (int row = wid; row < mx; row += nw) {
            C acc; acc.x = 0; acc.y = 0;
            const C* wr = Wj + (size_t)row * mx;
            for (int col = lane; col < mx; col += 32) acc = cfma(wr[col], r[col], acc);
            acc = warp_sum(acc);
            if (lane == 0) { C v = gj[row]; v.x -= acc.x; v.y -= acc.y; gj[row] = v; }
        }
        __syncthreads();
    }
    if (mode == 1) {
        C* dst = ytiles + T.yoff;
        for (int t = tid; t < mx * my; t += nt) dst[t] = g[t];
        return;
    }
    // owned nodes; for MP-1 a tile at the edge of the unknowns also writes the
    // adjacent (eliminated) boundary nodes, as zeros, so that z is defined everywhere
    const bool dir = op.bc == HZS_DIRICHLET;
    const int wx0 = (dir && T.ox0 == 1) ? 0 : T.ox0, wx1 = (dir && T.ox1 == n - 2) ? n - 1 : T.ox1;
    const int wy0 = (dir && T.oy0 == 1) ? 0 : T.oy0, wy1 = (dir && T.oy1 == n - 2) ? n - 1 : T.oy1;
    const int ow = wx1 - wx0 + 1, oh = wy1 - wy0 + 1;
    for (int t = tid; t < ow * oh; t += nt) {
        const int gi = wx0 + t % ow, gj = wy0 + t / ow;
        if (!op_is_unknown(op, gi, gj)) { z[(size_t)gj * n + gi] = mk<Cz>(0.0, 0.0); continue; }
        C v = g[(gj - T.y0) * mx + (gi - T.x0)];
        if (use_coarse) {
            // q = R_0^T c at this node
            const int ci = ct.c0[gi], cjj = ct.c0[gj];
            for (int b = 0; b < 3; ++b) {
                const double wyb = ct.w[3 * gj + b];
                if (wyb == 0.0) continue;
                for (int a = 0; a < 3; ++a) {
                    const double wxa = ct.w[3 * gi + a];
                    if (wxa == 0.0) continue;
                    const double2 cv = c[(size_t)(cjj + b) * ct.nc1 + (ci + a)];
                    const R wgt = (R)(wxa * wyb);
                    v.x += wgt * (R)cv.x; v.y += wgt * (R)cv.y;
                }
            }
        }
        z[(size_t)gj * n + gi] = cvt<Cz>(to_d(v));
    }
}

template <typename Cw, typename Cz, typename R>
int launch_tile_solve(const Ctx& cx, const Tile* tiles, int ntiles, int max_mx, int max_my, const cplx_t<R>* W,
                      const Cw* w, const double* vscale, int mode, const double2* c, int use_coarse, Cz* z,
                      cplx_t<R>* ytiles, const int* skip) {
    using C = cplx_t<R>;
    const size_t smem = (size_t)max_mx * max_my * sizeof(C) + (size_t)max_mx * sizeof(C) + (size_t)max_mx * sizeof(R);
    auto kern = k_tile_solve<Cw, Cz, R>;
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return -1;
    }
    kern<<<ntiles, 256, smem, cx.stream>>>(cx.op, cx.ct, tiles, W, w, vscale, mode, c, use_coarse, z, ytiles, skip);
    return 0;
}
template int launch_tile_solve<double2, double2, double>(const Ctx&, const Tile*, int, int, int, const double2*,
                                                         const double2*, const double*, int, const double2*, int,
                                                         double2*, double2*, const int*);
template int launch_tile_solve<float2, float2, float>(const Ctx&, const Tile*, int, int, int, const float2*,
                                                      const float2*, const double*, int, const double2*, int,
                                                      float2*, float2*, const int*);
template int launch_tile_solve<double2, float2, float>(const Ctx&, const Tile*, int, int, int, const float2*,
                                                       const double2*, const double*, int, const double2*, int,
                                                       float2*, float2*, const int*);

}  // namespace hzs
// complex64 arithmetic written straight to a complex128 output (allocation-free apply)
template int hzs::launch_tile_solve<double2, double2, float>(const Ctx&, const Tile*, int, int, int, const float2*,
                                                             const double2*, const double*, int, const double2*, int,
                                                             double2*, float2*, const int*);
