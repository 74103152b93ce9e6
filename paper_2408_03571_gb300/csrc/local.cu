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
#include "async.cuh"
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
        double2* dst64 = W64 + fd.woff + (long long)j * block_stride(m);
        float2* dst32 = W32 ? W32 + fd.woff + (long long)j * block_stride(m) : nullptr;
        const int ms = block_ld(m);
        for (int t = tid; t < m * ms; t += nt) {
            const int a = t / ms, b = t % ms;
            const double2 v = b < m ? S[a * m + b] : make_double2(0.0, 0.0);   // pad column: zero
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
    if (allow_dynamic_smem((const void*)k_tile_factor, smem) != cudaSuccess) return -1;
    k_tile_factor<<<nfactors, 512, smem, cx.stream>>>(cx.op, fdesc_dev, W64, W32, stat_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ------------------------------------------------------------------ solve
// One block per group of T tiles that share a factor.  The tile right-hand
// sides b = R_i w are gathered into shared memory (g), swept forward and
// backward in place, and written out: mode 0 (restricted, D_i = owner
// indicator): z = [R_0^T c] + x on owned nodes; mode 1 (additive, D_i = I):
// the whole tile x into ytiles.
//
// The dense blocks W_j stream from global memory (L2-resident when factors are
// shared) into an NST-deep ring of shared-memory stages by bulk asynchronous
// copies (cp.async.bulk, completion counted on an mbarrier per stage) issued
// by thread 0, NST-1 block steps ahead of their use.  The 2 my - 1 block steps
// use blocks 0, 1, .., my-1 (forward) then my-2, .., 0 (backward).  TPR threads
// (8 when the tile allows, else 4) share one output row of a block product; each
// step ends with one barrier.
// Every mbarrier wait is bounded: on expiry the block records HZS_ERR_TIMEOUT in
// the error word, drains its outstanding copies (again bounded) and returns.

template <typename R, int T, int NST>
__host__ __device__ constexpr size_t tile_smem_bytes(int mx, int my) {
    // W stages | g (T tiles) | r (2 x T x block_ld(mx), 16-byte aligned) | cy (mx) | mbarriers
    return ((size_t)NST * block_stride(mx) * sizeof(cplx_t<R>) + 127) / 128 * 128 +
           ((size_t)T * mx * my * sizeof(cplx_t<R>) + 15) / 16 * 16 +
           (size_t)2 * T * block_ld(mx) * sizeof(cplx_t<R>) + (size_t)mx * sizeof(R) + 16 + (size_t)NST * 8 + 16;
}

// ---- stages of the tile solve

// Gathers b = R_i (s w) for the group's T tiles into g (T x mx*my), the row
// couplings cy (mx) and the first right-hand side r = b_0 (T x block_ld(mx), the
// second buffer zeroed); ends with a block barrier.
template <typename Cw, typename R, int T>
__device__ __forceinline__ void tile_gather(const OpDesc& op, const Tile* __restrict__ tiles, const int* tix,
                                            const Tile& T0, const Cw* __restrict__ w, R sc, cplx_t<R>* g,
                                            cplx_t<R>* r, R* cy) {
    using C = cplx_t<R>;
    const int mx = T0.mx, my = T0.my, n = op.n;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = 0; t < T; ++t) {
        C* gt = g + (size_t)t * mx * my;
        if (tix[t] < 0) {
            for (int e = tid; e < mx * my; e += nt) gt[e] = mk<C>(0.0, 0.0);
            continue;
        }
        const Tile Ti = tiles[tix[t]];
        for (int e = tid; e < mx * my; e += nt) {
            const int a = e % mx, b = e / mx;
            C v = conv<C>(w[(size_t)(Ti.y0 + b) * n + (Ti.x0 + a)]);
            v.x *= sc; v.y *= sc;
            gt[e] = v;
        }
    }
    for (int a = tid; a < mx; a += nt) cy[a] = (R)op_cy(op, T0.x0 + a);
    __syncthreads();
    // both right-hand-side buffers (2 x T x block_ld(mx)); the pad entries stay zero
    const int ms = block_ld(mx);
    for (int e = tid; e < 2 * T * ms; e += nt) {
        const int t = (e / ms) % T, a = e % ms;
        r[e] = (e < T * ms && a < mx) ? g[(size_t)t * mx * my + a] : mk<C>(0.0, 0.0);
    }
    __syncthreads();
}

// Completes block step j for row `row` of each tile from the row products acc
// (thread sub == 0 of the row): forward g_j = W_j (b_j - C g_{j-1}), backward
// x_j = g_j - W_j (C x_{j+1}); writes the next step's right-hand side into rn.
template <typename R, int T>
__device__ __forceinline__ void tile_step_finish(bool fwd, int j, int my, int mx, int row, const cplx_t<R>* acc,
                                                 cplx_t<R>* g, cplx_t<R>* rn, const R* cy) {
    using C = cplx_t<R>;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        C* gt = g + (size_t)t * mx * my;
        C x;
        if (fwd) {
            x = acc[t];
        } else {
            x = gt[(size_t)j * mx + row];
            x.x -= acc[t].x; x.y -= acc[t].y;
        }
        gt[(size_t)j * mx + row] = x;
        C nr;
        if (fwd && j + 1 < my) {
            const C b = gt[(size_t)(j + 1) * mx + row];
            nr.x = b.x - cy[row] * x.x; nr.y = b.y - cy[row] * x.y;
        } else {
            nr.x = cy[row] * x.x; nr.y = cy[row] * x.y;   // C x_j for the backward step j-1
        }
        rn[t * mx + row] = nr;
    }
}

// Writes the solved tiles: mode 0 (restricted, D_i = owner indicator): z =
// [R_0^T c] + x on owned nodes; mode 1 (additive): the whole tile into ytiles.
template <typename Cz, typename R, int T>
__device__ __forceinline__ void tile_output(const OpDesc& op, const CoarseTab& ct, const Tile* __restrict__ tiles,
                                            const int* tix, const Tile& T0, const cplx_t<R>* g, int mode,
                                            const cplx_t<R>* __restrict__ c, int use_coarse, Cz* __restrict__ z,
                                            cplx_t<R>* __restrict__ ytiles) {
    using C = cplx_t<R>;
    const int mx = T0.mx, my = T0.my, n = op.n;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = 0; t < T; ++t) {
        if (tix[t] < 0) continue;
        const Tile Ti = tiles[tix[t]];
        const C* gt = g + (size_t)t * mx * my;
        if (mode == 1) {
            C* dst = ytiles + Ti.yoff;
            for (int e = tid; e < mx * my; e += nt) dst[e] = gt[e];
            continue;
        }
        // owned nodes; for MP-1 a tile at the edge of the unknowns also writes the
        // adjacent (eliminated) boundary nodes, as zeros, so that z is defined everywhere
        const bool dir = op.bc == HZS_DIRICHLET;
        const int wx0 = (dir && Ti.ox0 == 1) ? 0 : Ti.ox0, wx1 = (dir && Ti.ox1 == n - 2) ? n - 1 : Ti.ox1;
        const int wy0 = (dir && Ti.oy0 == 1) ? 0 : Ti.oy0, wy1 = (dir && Ti.oy1 == n - 2) ? n - 1 : Ti.oy1;
        const int ow = wx1 - wx0 + 1, oh = wy1 - wy0 + 1;
        for (int e = tid; e < ow * oh; e += nt) {
            const int gi = wx0 + e % ow, gj = wy0 + e / ow;
            if (!op_is_unknown(op, gi, gj)) { z[(size_t)gj * n + gi] = mk<Cz>(0.0, 0.0); continue; }
            C v = gt[(gj - Ti.y0) * mx + (gi - Ti.x0)];
            if (use_coarse) {
                // q = R_0^T c at this node
                const int ci = ct.c0[gi], cjj = ct.c0[gj];
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const R wyb = CoarseW<R>::w3(ct, 3 * gj + b);
                    if (wyb == (R)0) continue;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const R wxa = CoarseW<R>::w3(ct, 3 * gi + a);
                        if (wxa == (R)0) continue;
                        const C cv = c[(size_t)(cjj + b) * ct.nc1 + (ci + a)];
                        const R wgt = wxa * wyb;
                        v.x += wgt * cv.x; v.y += wgt * cv.y;
                    }
                }
            }
            z[(size_t)gj * n + gi] = conv<Cz>(v);
        }
    }
}

template <typename Cw, typename Cz, typename R, int T, int NST, int TPR, int MAXT>
__global__ void __launch_bounds__(MAXT) k_tile_solve(OpDesc op, CoarseTab ct, const Tile* __restrict__ tiles,
                                                    const int* __restrict__ groups, const cplx_t<R>* __restrict__ W,
                                                    const Cw* __restrict__ w, long long ws,
                                                    const double* __restrict__ vscale, long long vss, int mode,
                                                    const cplx_t<R>* __restrict__ c, long long cs, int use_coarse,
                                                    Cz* __restrict__ z, long long zs, cplx_t<R>* __restrict__ ytiles,
                                                    long long yts, BatchSkip sk, int* __restrict__ err,
                                                    long long spin) {
    using C = cplx_t<R>;
    const int rb = blockIdx.y;                      // batch entry
    if (sk.flag && sk.flag[(size_t)rb * sk.stride]) return;
    w += rb * ws;
    c += rb * cs;
    if (z) z += rb * zs;
    if (ytiles) ytiles += rb * yts;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    int tix[T];
#pragma unroll
    for (int t = 0; t < T; ++t) tix[t] = groups[blockIdx.x * T + t];
    const Tile T0 = tiles[tix[0]];
    const int mx = T0.mx, my = T0.my;
    const long long bs = block_stride(mx);
    const uint32_t bbytes = (uint32_t)(bs * sizeof(C));
    C* wst = reinterpret_cast<C*>(smem_raw);                                        // NST stages
    const int ms = block_ld(mx);                                                    // padded row length
    C* g = reinterpret_cast<C*>(smem_raw + ((size_t)NST * bs * sizeof(C) + 127) / 128 * 128);   // T x mx*my
    C* r = reinterpret_cast<C*>((reinterpret_cast<uintptr_t>(g + (size_t)T * mx * my) + 15) & ~uintptr_t(15));
    R* cy = reinterpret_cast<R*>(r + 2 * T * ms);                                   // mx
    uint64_t* bar = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(cy + mx) + 15) & ~uintptr_t(15));
    const int tid = threadIdx.x;
    const C* Wt = W + T0.woff;
    const int nsteps = 2 * my - 1;
    auto blk = [&](int q) { return q < my ? q : 2 * my - 2 - q; };

    if (tid == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        for (int q = 0; q < NST && q < nsteps; ++q) {
            mbar_expect_tx(&bar[q], bbytes);
            bulk_g2s(wst + (size_t)q * bs, Wt + (size_t)blk(q) * bs, bbytes, &bar[q]);
        }
    }
    tile_gather<Cw, R, T>(op, tiles, tix, T0, w, vscale ? (R)vscale[rb * vss] : (R)1, g, r, cy);

    const int row = tid / TPR, sub = tid % TPR;
    const bool active = row < mx;
    int q_fail = -1;
    __shared__ int s_fail;
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int q = 0; q < nsteps; ++q) {
        const int st = q % NST;
        const uint32_t parity = (uint32_t)((q / NST) & 1);
        // a thread whose wait expires flags it and finishes the step on whatever the
        // stage holds; the step's closing barrier then ends the sweep for every thread
        if (!mbar_wait_bounded(&bar[st], parity, spin)) s_fail = 1;
        const C* Wq = wst + (size_t)st * bs;
        const C* rc = r + (size_t)(q & 1) * T * ms;
        C* rn = r + (size_t)((q + 1) & 1) * T * ms;
        // every thread of the block runs the shuffles below (inactive rows add zeros)
        C acc[T];
#pragma unroll
        for (int t = 0; t < T; ++t) { acc[t].x = 0; acc[t].y = 0; }
        if (active) {
            const C* wr = Wq + (size_t)row * ms;
            if constexpr (sizeof(R) == sizeof(float)) {
                // complex64: two entries per 16-byte load (rows and buffers are 16-byte
                // aligned; the zero pad column makes ms/2 pairs exact)
                const float4* w4 = reinterpret_cast<const float4*>(wr);
                // tiles of at most 72 (launch bound 576): at most KP pairs per thread, and
                // the loop below is fully unrolled
                constexpr int KP = MAXT <= 576 ? (36 + TPR - 1) / TPR : 1024;
#pragma unroll 8
                for (int m = 0; m < KP; ++m) {
                    const int k2 = sub + TPR * m;
                    if (k2 >= ms / 2) break;
                    const float4 wv = w4[k2];
#pragma unroll
                    for (int t = 0; t < T; ++t) {
                        const float4 rv = reinterpret_cast<const float4*>(rc + t * ms)[k2];
                        acc[t] = cfma(make_float2(wv.x, wv.y), make_float2(rv.x, rv.y), acc[t]);
                        acc[t] = cfma(make_float2(wv.z, wv.w), make_float2(rv.z, rv.w), acc[t]);
                    }
                }
            } else {
                for (int k = sub; k < mx; k += TPR) {
                    const C wv = wr[k];
#pragma unroll
                    for (int t = 0; t < T; ++t) acc[t] = cfma(wv, rc[t * ms + k], acc[t]);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
#pragma unroll
            for (int o = 1; o < TPR; o <<= 1) {
                acc[t].x += __shfl_xor_sync(0xffffffffu, acc[t].x, o);
                acc[t].y += __shfl_xor_sync(0xffffffffu, acc[t].y, o);
            }
        }
        // lane sub == t of the row completes tile t (all lanes hold the row sums)
        if (active && sub < T) {
            C a = acc[0];
#pragma unroll
            for (int t = 1; t < T; ++t)
                if (sub == t) a = acc[t];
            tile_step_finish<R, 1>(q < my, blk(q), my, mx, row, &a, g + (size_t)sub * mx * my, rn + (size_t)sub * ms,
                                   cy);
        }
        __syncthreads();   // stage st fully read; next r complete
        if (s_fail) { q_fail = q; break; }
        if (tid == 0 && q + NST < nsteps) {
            mbar_expect_tx(&bar[st], bbytes);
            bulk_g2s(wst + (size_t)st * bs, Wt + (size_t)blk(q + NST) * bs, bbytes, &bar[st]);
        }
    }
    if (q_fail >= 0) {
        if (tid == 0) {
            if (err) atomicExch(err, (int)HZS_ERR_TIMEOUT);
            // copies in flight: steps q_fail .. q_fail + NST - 1; wait for each (bounded)
            for (int qq = q_fail; qq < q_fail + NST && qq < nsteps; ++qq)
                mbar_wait_bounded(&bar[qq % NST], (uint32_t)((qq / NST) & 1));
        }
        __syncthreads();
        return;
    }
    tile_output<Cz, R, T>(op, ct, tiles, tix, T0, g, mode, c, use_coarse, z, ytiles);
}

constexpr size_t kSmemLimit = 227 * 1024;

int tile_group_width(int max_mx, int max_my, int elem_bytes) {
    if (elem_bytes == (int)sizeof(float2)) {
        if (tile_smem_bytes<float, 2, 2>(max_mx, max_my) <= kSmemLimit) return 2;
        if (tile_smem_bytes<float, 1, 1>(max_mx, max_my) <= kSmemLimit) return 1;
        return 0;
    }
    return tile_smem_bytes<double, 1, 1>(max_mx, max_my) <= kSmemLimit ? 1 : 0;
}

// Threads per block row: tpr 8 or 4 as asked, 0 = 8 while the block stays within 1024
// threads, else 4; 0 if the asked value does not fit.
static int resolve_tpr(int tpr, int max_mx) {
    if (tpr == 0) return max_mx * 8 <= 1024 ? 8 : 4;
    if (tpr == 8) return max_mx * 8 <= 1024 ? 8 : 0;
    if (tpr == 4) return max_mx * 4 <= 1024 ? 4 : 0;
    return 0;
}

template <typename Cw, typename Cz, typename R, int T, int NST>
static int launch_tile_solve_t(const Ctx& cx, int nb, const Tile* tiles, TileGroups grp, int max_mx, int max_my,
                               const cplx_t<R>* W, const Cw* w, long long ws, const double* vscale, long long vss,
                               int mode, const cplx_t<R>* c, long long cs, int use_coarse, Cz* z, long long zs,
                               cplx_t<R>* ytiles, long long yts, BatchSkip sk) {
    const size_t smem = tile_smem_bytes<R, T, NST>(max_mx, max_my);
    const int tpr = resolve_tpr(grp.tpr, max_mx);
    if (tpr == 0) return -1;
    // eight threads per block row while the block stays within 1024 threads: more warps
    // to hide the per-step latency and half the dependent multiply-adds per thread
    if (tpr == 8 && max_mx <= 72) {   // the common tile sizes: a tighter launch bound leaves more registers
        auto kern = k_tile_solve<Cw, Cz, R, T, NST, 8, 576>;
        if (allow_dynamic_smem((const void*)kern, smem) != cudaSuccess) return -1;
        const int threads = (max_mx * 8 + 31) / 32 * 32;
        kern<<<dim3(grp.count, nb), threads, smem, cx.stream>>>(cx.op, cx.ct, tiles, grp.idx, W, w, ws, vscale, vss,
                                                                mode, c, cs, use_coarse, z, zs, ytiles, yts, sk,
                                                                cx.err, cx.spin_limit);
        return 0;
    }
    if (tpr == 8) {
        auto kern = k_tile_solve<Cw, Cz, R, T, NST, 8, 1024>;
        if (allow_dynamic_smem((const void*)kern, smem) != cudaSuccess) return -1;
        const int threads = (max_mx * 8 + 31) / 32 * 32;
        kern<<<dim3(grp.count, nb), threads, smem, cx.stream>>>(cx.op, cx.ct, tiles, grp.idx, W, w, ws, vscale, vss,
                                                                mode, c, cs, use_coarse, z, zs, ytiles, yts, sk,
                                                                cx.err, cx.spin_limit);
        return 0;
    }
    auto kern = k_tile_solve<Cw, Cz, R, T, NST, 4, 1024>;
    if (allow_dynamic_smem((const void*)kern, smem) != cudaSuccess) return -1;
    const int threads = (max_mx * 4 + 31) / 32 * 32;
    kern<<<dim3(grp.count, nb), threads, smem, cx.stream>>>(cx.op, cx.ct, tiles, grp.idx, W, w, ws, vscale, vss, mode,
                                                            c, cs, use_coarse, z, zs, ytiles, yts, sk, cx.err,
                                                            cx.spin_limit);
    return 0;
}

// Ring depth used for T tiles per group: nst as asked (if it fits), 0 = the deepest of
// 4, 2 (and 1 for single tiles) that fits; 0 if none fits.
template <typename R>
static int resolve_nst(int T, int nst, int max_mx, int max_my) {
    auto fits = [&](int ns) -> bool {
        if (T == 2) {
            if (ns == 4) return tile_smem_bytes<R, 2, 4>(max_mx, max_my) <= kSmemLimit;
            if (ns == 2) return tile_smem_bytes<R, 2, 2>(max_mx, max_my) <= kSmemLimit;
            return false;   // pairs of tiles keep at least two stages
        }
        if (T != 1) return false;
        if (ns == 4) return tile_smem_bytes<R, 1, 4>(max_mx, max_my) <= kSmemLimit;
        if (ns == 2) return tile_smem_bytes<R, 1, 2>(max_mx, max_my) <= kSmemLimit;
        if (ns == 1) return tile_smem_bytes<R, 1, 1>(max_mx, max_my) <= kSmemLimit;
        return false;
    };
    if (nst != 0) return fits(nst) ? nst : 0;
    for (int ns : {4, 2, 1})
        if (fits(ns)) return ns;
    return 0;
}

bool tile_shape_resolve(const TileGroups& grp, int max_mx, int max_my, int elem_bytes, int* T, int* nst, int* tpr) {
    if (max_mx * 4 > 512) return false;
    const int ns = elem_bytes == (int)sizeof(float2) ? resolve_nst<float>(grp.T, grp.nst, max_mx, max_my)
                                                     : resolve_nst<double>(grp.T, grp.nst, max_mx, max_my);
    const int tp = resolve_tpr(grp.tpr, max_mx);
    if (ns == 0 || tp == 0) return false;
    *T = grp.T; *nst = ns; *tpr = tp;
    return true;
}

template <typename Cw, typename Cz, typename R>
int launch_tile_solve(const Ctx& cx, int nb, const Tile* tiles, TileGroups grp, int max_mx, int max_my,
                      const cplx_t<R>* W, const Cw* w, long long ws, const double* vscale, long long vss, int mode,
                      const cplx_t<R>* c, long long cs, int use_coarse, Cz* z, long long zs, cplx_t<R>* ytiles,
                      long long yts, BatchSkip sk) {
    if (max_mx * 4 > 512) return -1;
    // deepest ring of factor-block stages that fits (more stages hide the L2 latency of
    // the copies), unless the group fixes the depth
    const int nst = resolve_nst<R>(grp.T, grp.nst, max_mx, max_my);
#define HZS_TRY(TT, NS)                                                                                        \
    if (grp.T == TT && nst == NS)                                                                             \
        return launch_tile_solve_t<Cw, Cz, R, TT, NS>(cx, nb, tiles, grp, max_mx, max_my, W, w, ws, vscale, vss, \
                                                      mode, c, cs, use_coarse, z, zs, ytiles, yts, sk);
    HZS_TRY(2, 4)
    HZS_TRY(2, 2)
    HZS_TRY(1, 4)
    HZS_TRY(1, 2)
    HZS_TRY(1, 1)
#undef HZS_TRY
    return -1;
}

#define HZS_TS(Cw, Cz, R)                                                                                      \
    template int launch_tile_solve<Cw, Cz, R>(const Ctx&, int, const Tile*, TileGroups, int, int,               \
                                              const cplx_t<R>*, const Cw*, long long, const double*, long long,  \
                                              int, const cplx_t<R>*, long long, int, Cz*, long long, cplx_t<R>*, \
                                              long long, BatchSkip);
HZS_TS(double2, double2, double)
HZS_TS(float2, float2, float)
HZS_TS(double2, float2, float)
HZS_TS(double2, double2, float)
#undef HZS_TS

}  // namespace hzs
