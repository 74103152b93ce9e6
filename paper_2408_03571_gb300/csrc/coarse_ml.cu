// Multilevel coarse solve: the exact coarse solve c' = A_0^{-1} c (Eq. 4) replaced by
// one application of the two-level Schwarz method SHS2 (Eq. 6) on the coarse grid G_H
// itself, the cost the paper names as the bottleneck for large coarse spaces
// (Section 5).  G_H is treated as a grid of its own: MP-1 keeps only its interior
// coarse nodes, so it is the interior of a Dirichlet grid of nc1 + 2 nodes per axis;
// MP-2 keeps all nc1.  On that grid:
//   - coarse subdomains: ns0 x ns0 owned blocks [a w0, (a+1) w0) (the last one closed at
//     the grid's end) within its unknowns, extended by ov0 layers (the rule of the fine
//     level), each with an exact solve of its block of A_0 (an explicit FP64 inverse);
//   - a coarse-of-coarse space of B_2 functions of ratio p0 on that grid with its own
//     exact Galerkin solve A_00 = R_00 A_0 R_00^T (explicit FP64 inverse up to 4096
//     unknowns, block-tridiagonal LU above, as on the level above);
//   - c' = q + sum_i R_i^T D_i A_0i^{-1} R_i (c - A_0 q),  q = R_00^T A_00^{-1} R_00 c,
//     D_i the owner indicator.
// Everything is FP64 (the coarse solve is FP64 on both precisions of the library).
#include <algorithm>
#include <cstdlib>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace hzs {

// weight of the level-2 basis function K (one axis) at pseudo-grid node i, from the
// tables of build_coarse_tables (support [lo, hi], weights wt[off + i - lo])
__device__ __forceinline__ double ml_w1(const int* __restrict__ lo, const int* __restrict__ hi,
                                        const int* __restrict__ off, const double* __restrict__ wt, int K, int i) {
    const int a = lo[K], b = hi[K];
    return (i >= a && i <= b) ? wt[off[K] + i - a] : 0.0;
}

// ------------------------------------------------------------------ set-up
// A_00[I, J] = sum_{a in supp I} R_00[I, a] sum_{o} A_0[a, a + o] R_00[J, a + o] for the
// 7 x 7 level-2 neighbours J of I (supports of width 3 p0 - 1 and A_0's band of 2 leave
// no other nonzeros); one block per (I, window entry), threads over a, fixed-order sum.
// A_00 is written dense (band == 0: row I, column J of an Nc00 x Nc00 array) or in band
// form (band == 1: 49 offsets a row, offset index = the window entry (dJy + 3) 7 + dJx + 3).
__global__ void k_ml_galerkin(int nc1, int lo0, int nc00, const double2* __restrict__ A0b, const int* __restrict__ lo,
                              const int* __restrict__ hi, const int* __restrict__ off,
                              const double* __restrict__ wt, double2* __restrict__ A00, int band) {
    __shared__ double2 red[128];
    const int I = blockIdx.y, win = blockIdx.x;
    const int Ix = I % nc00, Iy = I / nc00;
    const int Jx = Ix + win % 7 - 3, Jy = Iy + win / 7 - 3;
    const bool inJ = Jx >= 0 && Jx < nc00 && Jy >= 0 && Jy < nc00;
    double2 acc = make_double2(0.0, 0.0);
    if (inJ) {
        const int ax0 = lo[Ix], ax1 = hi[Ix], ay0 = lo[Iy], ay1 = hi[Iy];   // pseudo-grid nodes
        const int wx = ax1 - ax0 + 1, cnt = wx * (ay1 - ay0 + 1);
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int px = ax0 + t % wx, py = ay0 + t / wx;
            const double wi = ml_w1(lo, hi, off, wt, Ix, px) * ml_w1(lo, hi, off, wt, Iy, py);
            if (wi == 0.0) continue;
            const int gx = px - lo0, gy = py - lo0;                          // G_H unknown (gx, gy)
            double2 s = make_double2(0.0, 0.0);
            for (int dJ = -2; dJ <= 2; ++dJ) {
                const int gy2 = gy + dJ;
                if (gy2 < 0 || gy2 >= nc1) continue;
                const double wy = ml_w1(lo, hi, off, wt, Jy, gy2 + lo0);
                if (wy == 0.0) continue;
                for (int dI = -2; dI <= 2; ++dI) {
                    const int gx2 = gx + dI;
                    if (gx2 < 0 || gx2 >= nc1) continue;
                    const double wj = wy * ml_w1(lo, hi, off, wt, Jx, gx2 + lo0);
                    if (wj == 0.0) continue;
                    const double2 a = A0b[((size_t)gy * nc1 + gx) * 25 + (dJ + 2) * 5 + (dI + 2)];
                    s.x += a.x * wj;
                    s.y += a.y * wj;
                }
            }
            acc.x += wi * s.x;
            acc.y += wi * s.y;
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0 && inJ) {
        if (band) A00[(size_t)I * 49 + win] = red[0];
        else A00[(size_t)I * (nc00 * nc00) + (size_t)Jy * nc00 + Jx] = red[0];
    }
}

// Dense block of A_0 of coarse subdomain s = blockIdx.y (its extended rectangle of G_H,
// row-major, x fastest) from the band.
__global__ void k_ml_extract(int nc1, const double2* __restrict__ A0b, const int4* __restrict__ sub,
                             const long long* __restrict__ aoff, double2* __restrict__ Aloc) {
    const int s = blockIdx.y;
    const int4 R = sub[s];                       // x0, y0, mx, my
    const int m = R.z * R.w;
    const long long total = (long long)m * m;
    double2* dst = Aloc + aoff[s];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int pl = (int)(t / m), ql = (int)(t % m);
        const int px = R.x + pl % R.z, py = R.y + pl / R.z;
        const int qx = R.x + ql % R.z, qy = R.y + ql / R.z;
        const int dI = qx - px, dJ = qy - py;
        double2 v = make_double2(0.0, 0.0);
        if (dI >= -2 && dI <= 2 && dJ >= -2 && dJ <= 2)
            v = A0b[((size_t)py * nc1 + px) * 25 + (dJ + 2) * 5 + (dI + 2)];
        dst[t] = v;
    }
}

// ------------------------------------------------------------------ apply (batch entry r = blockIdx.y)
// c00 = R_00 c
__global__ void k_ml_restrict(int nc1, int lo0, int nc00, const int* __restrict__ lo, const int* __restrict__ hi,
                              const int* __restrict__ off, const double* __restrict__ wt,
                              const double2* __restrict__ c, double2* __restrict__ c00, BatchSkip sk) {
    const int r = blockIdx.y;
    if (sk.flag && sk.flag[(size_t)r * sk.stride]) return;
    const int J = blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= nc00 * nc00) return;
    const int Jx = J % nc00, Jy = J / nc00;
    c += (size_t)r * nc1 * nc1;
    double2 acc = make_double2(0.0, 0.0);
    for (int py = lo[Jy]; py <= hi[Jy]; ++py) {
        const double wy = wt[off[Jy] + py - lo[Jy]];
        double2 row = make_double2(0.0, 0.0);
        for (int px = lo[Jx]; px <= hi[Jx]; ++px) {
            const double wx = wt[off[Jx] + px - lo[Jx]];
            const double2 v = c[(size_t)(py - lo0) * nc1 + (px - lo0)];
            row.x += wx * v.x;
            row.y += wx * v.y;
        }
        acc.x += wy * row.x;
        acc.y += wy * row.y;
    }
    c00[(size_t)r * nc00 * nc00 + J] = acc;
}

// q = R_00^T c00p  (per G_H node: the at most 3 x 3 level-2 functions touching it)
__global__ void k_ml_prolong(int nc1, int lo0, int nc00, const int* __restrict__ c0, const double* __restrict__ w3,
                             const double2* __restrict__ c00p, double2* __restrict__ q, BatchSkip sk) {
    const int r = blockIdx.y;
    if (sk.flag && sk.flag[(size_t)r * sk.stride]) return;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nc1 * nc1) return;
    const int px = a % nc1 + lo0, py = a / nc1 + lo0;
    const double2* cc = c00p + (size_t)r * nc00 * nc00;
    double2 v = make_double2(0.0, 0.0);
    for (int b = 0; b < 3; ++b) {
        const double wy = w3[3 * py + b];
        if (wy == 0.0) continue;
        for (int d = 0; d < 3; ++d) {
            const double wx = w3[3 * px + d];
            if (wx == 0.0) continue;
            const double2 x = cc[(size_t)(c0[py] + b) * nc00 + (c0[px] + d)];
            v.x += wy * wx * x.x;
            v.y += wy * wx * x.y;
        }
    }
    q[(size_t)r * nc1 * nc1 + a] = v;
}

// wv = c - A_0 q
__global__ void k_ml_resid(int nc1, const double2* __restrict__ A0b, const double2* __restrict__ c,
                           const double2* __restrict__ q, double2* __restrict__ wv, BatchSkip sk) {
    const int r = blockIdx.y;
    if (sk.flag && sk.flag[(size_t)r * sk.stride]) return;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int Nc = nc1 * nc1;
    if (a >= Nc) return;
    const long long o = (long long)r * Nc;
    const int gx = a % nc1, gy = a / nc1;
    double2 acc = make_double2(0.0, 0.0);
    for (int dJ = -2; dJ <= 2; ++dJ) {
        const int y2 = gy + dJ;
        if (y2 < 0 || y2 >= nc1) continue;
        for (int dI = -2; dI <= 2; ++dI) {
            const int x2 = gx + dI;
            if (x2 < 0 || x2 >= nc1) continue;
            acc = cfma(A0b[(size_t)a * 25 + (dJ + 2) * 5 + (dI + 2)], q[o + (size_t)y2 * nc1 + x2], acc);
        }
    }
    wv[o + a] = csub(c[o + a], acc);
}

// out = q + (A_0s^{-1} R_s wv) on the nodes subdomain s = blockIdx.y owns (one warp per
// owned node; every G_H node is owned by exactly one coarse subdomain); batch entry
// r = blockIdx.z
__global__ void k_ml_local(int nc1, const int4* __restrict__ sub, const int4* __restrict__ own,
                           const long long* __restrict__ aoff, const double2* __restrict__ Ainv,
                           const double2* __restrict__ q, const double2* __restrict__ wv, double2* __restrict__ out,
                           BatchSkip sk) {
    const int r = blockIdx.z;
    if (sk.flag && sk.flag[(size_t)r * sk.stride]) return;
    const int s = blockIdx.y;
    const int4 R = sub[s], O = own[s];             // R: x0, y0, mx, my; O: x0, x1, y0, y1
    const int ow = O.y - O.x + 1, oh = O.w - O.z + 1;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (t >= ow * oh) return;
    const int gx = O.x + t % ow, gy = O.z + t / ow;
    const int m = R.z * R.w;
    const int pl = (gy - R.y) * R.z + (gx - R.x);
    const double2* row = Ainv + aoff[s] + (size_t)pl * m;
    const long long o = (long long)r * nc1 * nc1;
    double2 acc = make_double2(0.0, 0.0);
    for (int kb = 0; kb < R.w; ++kb) {
        const double2* rw = row + (size_t)kb * R.z;
        const double2* xv = wv + o + (size_t)(R.y + kb) * nc1 + R.x;
        for (int ka = lane; ka < R.z; ka += 32) acc = cfma(rw[ka], xv[ka], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) {
        const size_t g = (size_t)gy * nc1 + gx;
        out[o + g] = cadd(q[o + g], acc);
    }
}

__global__ void k_ml_to_c64(int Nc, const double2* __restrict__ a, float2* __restrict__ b, BatchSkip sk) {
    const int r = blockIdx.y;
    if (sk.flag && sk.flag[(size_t)r * sk.stride]) return;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Nc; e += gridDim.x * blockDim.x)
        b[(size_t)r * Nc + e] = to_f(a[(size_t)r * Nc + e]);
}

// ------------------------------------------------------------------ host
template <typename T>
static cudaError_t ml_upload(T** dst, const std::vector<T>& src, cudaStream_t s) {
    if (cudaMalloc(dst, std::max<size_t>(1, src.size()) * sizeof(T)) != cudaSuccess) return cudaErrorMemoryAllocation;
    if (src.empty()) return cudaSuccess;
    return cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

void coarse_ml_free(CoarseML& ml) {
    cudaFree(ml.lo2); cudaFree(ml.hi2); cudaFree(ml.off2); cudaFree(ml.c02); cudaFree(ml.wt2); cudaFree(ml.w2);
    cudaFree(ml.A00inv); cudaFree(ml.sub); cudaFree(ml.own); cudaFree(ml.aoff); cudaFree(ml.Ainv); cudaFree(ml.A0b);
    cudaFree(ml.c00); cudaFree(ml.c00p); cudaFree(ml.q); cudaFree(ml.wv);
    coarse_block_free(ml.cblk00);
    ml = CoarseML{};
}

int coarse_ml_setup(const Ctx& cx, int nc1, int bc, double2* A0b, int ns0, int ov0, int p0, CoarseML& ml,
                    double* minpiv, std::string* why) {
    ml = CoarseML{};
    ml.A0b = A0b;
    auto bad = [&](const char* msg) {
        *why = msg;
        coarse_ml_free(ml);
        return -2;
    };
    const bool dir = bc == HZS_DIRICHLET;
    const int n0 = dir ? nc1 + 2 : nc1, lo0 = dir ? 1 : 0, hi0 = dir ? n0 - 2 : n0 - 1;
    if (n0 < 3 || ns0 < 1 || (n0 - 1) % ns0 != 0) return bad("ml_nsub must divide the coarse grid's n0 - 1");
    const int w0 = (n0 - 1) / ns0;
    if (ov0 < 0 || 2 * ov0 > w0) return bad("ml_overlap must be >= 0 and at most half the coarse subdomain width");
    if (p0 < 2 || (n0 - 1) % p0 != 0) return bad("ml_ratio must be >= 2 and divide the coarse grid's n0 - 1");
    HostCoarseTab t2;
    build_coarse_tables(n0, bc, HZS_COARSE_B2, p0, t2);
    if (t2.nc1 < 1 || t2.bad) return bad("the coarse-of-coarse space is empty");
    ml.nc1 = nc1; ml.Nc = nc1 * nc1; ml.lo0 = lo0;
    ml.nc00 = t2.nc1; ml.Nc00 = t2.nc1 * t2.nc1;
    // the coarse-of-coarse solve as the level above: dense inverse up to 4096 unknowns,
    // block-tridiagonal LU (groups of 3 rows: A_00 couples rows up to 3 apart) above
    ml.blk00 = ml.Nc00 > 4096;
    // test knob: HZS_ML_BLOCK00=1 takes the block LU at any size (to compare it with the dense inverse)
    if (const char* ev = std::getenv("HZS_ML_BLOCK00")) ml.blk00 = ml.blk00 || std::atoi(ev) != 0;
    if (ml.nc00 > 512) return bad("more than 512 coarse-of-coarse nodes per axis");
    // coarse subdomains (pseudo-grid rule of the fine level, then G_H indices)
    std::vector<int2> own_ax, ext_ax;
    for (int a = 0; a < ns0; ++a) {
        const int olo = std::max(a * w0, lo0), ohi = std::min(a < ns0 - 1 ? (a + 1) * w0 - 1 : n0 - 1, hi0);
        if (olo > ohi) return bad("a coarse subdomain owns no coarse unknown");
        own_ax.push_back(make_int2(olo - lo0, ohi - lo0));
        ext_ax.push_back(make_int2(std::max(olo - ov0, lo0) - lo0, std::min(ohi + ov0, hi0) - lo0));
    }
    std::vector<int4> sub, own;
    std::vector<long long> aoff;
    long long tot = 0;
    for (int by = 0; by < ns0; ++by)
        for (int bx = 0; bx < ns0; ++bx) {
            const int mx = ext_ax[bx].y - ext_ax[bx].x + 1, my = ext_ax[by].y - ext_ax[by].x + 1;
            sub.push_back(make_int4(ext_ax[bx].x, ext_ax[by].x, mx, my));
            own.push_back(make_int4(own_ax[bx].x, own_ax[bx].y, own_ax[by].x, own_ax[by].y));
            aoff.push_back(tot);
            tot += (long long)mx * my * mx * my;
            ml.max_own = std::max(ml.max_own, (own_ax[bx].y - own_ax[bx].x + 1) * (own_ax[by].y - own_ax[by].x + 1));
            ml.max_m = std::max(ml.max_m, mx * my);
        }
    if ((double)tot * sizeof(double2) > 64.0 * (1ull << 30)) return bad("coarse subdomain inverses above 64 GB");
    ml.nsub = ns0 * ns0;
    cudaStream_t st = cx.stream;
    if (ml_upload(&ml.lo2, t2.lo, st) || ml_upload(&ml.hi2, t2.hi, st) || ml_upload(&ml.off2, t2.off, st) ||
        ml_upload(&ml.c02, t2.c0, st) || ml_upload(&ml.wt2, t2.wt, st) || ml_upload(&ml.w2, t2.w, st) ||
        ml_upload(&ml.sub, sub, st) || ml_upload(&ml.own, own, st) || ml_upload(&ml.aoff, aoff, st)) {
        coarse_ml_free(ml);
        return -1;
    }
    if (cudaMalloc(&ml.Ainv, (size_t)tot * sizeof(double2)) != cudaSuccess) {
        coarse_ml_free(ml);
        return -1;
    }
    double mp = 1e300, piv = 0.0;
    int singular = 0, rc = 0;
    if (!ml.blk00) {
        // A_00 dense (banded by construction) and its inverse
        if (cudaMalloc(&ml.A00inv, (size_t)ml.Nc00 * ml.Nc00 * sizeof(double2)) != cudaSuccess) {
            coarse_ml_free(ml);
            return -1;
        }
        cudaMemsetAsync(ml.A00inv, 0, (size_t)ml.Nc00 * ml.Nc00 * sizeof(double2), st);
        k_ml_galerkin<<<dim3(49, ml.Nc00), 128, 0, st>>>(nc1, lo0, ml.nc00, A0b, ml.lo2, ml.hi2, ml.off2, ml.wt2,
                                                         ml.A00inv, 0);
        rc = gj_invert(cx, ml.A00inv, ml.Nc00, &piv);
    } else {
        // A_00 in band form (radius 3) and its block-tridiagonal LU (which owns the band)
        double2* A00b = nullptr;
        if (cudaMalloc(&A00b, (size_t)ml.Nc00 * 49 * sizeof(double2)) != cudaSuccess) {
            coarse_ml_free(ml);
            return -1;
        }
        cudaMemsetAsync(A00b, 0, (size_t)ml.Nc00 * 49 * sizeof(double2), st);
        k_ml_galerkin<<<dim3(49, ml.Nc00), 128, 0, st>>>(nc1, lo0, ml.nc00, A0b, ml.lo2, ml.hi2, ml.off2, ml.wt2,
                                                         A00b, 1);
        rc = coarse_block_setup(cx, ml.nc00, 3, 3, A00b, ml.cblk00, &piv);
    }
    if (rc < 0) { coarse_ml_free(ml); return -1; }
    singular |= rc > 0;
    mp = std::min(mp, piv);
    // the coarse subdomains' blocks of A_0 and their inverses
    k_ml_extract<<<dim3(4 * cx.num_sms, ml.nsub), 256, 0, st>>>(nc1, A0b, ml.sub, ml.aoff, ml.Ainv);
    for (int s = 0; s < ml.nsub; ++s) {
        rc = gj_invert(cx, ml.Ainv + aoff[s], sub[s].z * sub[s].w, &piv);
        if (rc < 0) { coarse_ml_free(ml); return -1; }
        singular |= rc > 0;
        mp = std::min(mp, piv);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) { coarse_ml_free(ml); return -1; }
    *minpiv = mp;
    return singular ? 1 : 0;
}

int coarse_ml_reserve(CoarseML& ml, int nb) {
    if (ml.nb_cap >= nb) return 0;
    cudaFree(ml.c00); cudaFree(ml.c00p); cudaFree(ml.q); cudaFree(ml.wv);
    ml.c00 = ml.c00p = ml.q = ml.wv = nullptr;
    ml.nb_cap = 0;
    if (cudaMalloc(&ml.c00, (size_t)nb * ml.Nc00 * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&ml.c00p, (size_t)nb * ml.Nc00 * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&ml.q, (size_t)nb * ml.Nc * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&ml.wv, (size_t)nb * ml.Nc * sizeof(double2)) != cudaSuccess)
        return -1;
    ml.nb_cap = nb;
    return 0;
}

void launch_coarse_ml_solve(const Ctx& cx, int nb, const CoarseML& ml, const double2* c, double2* out, float2* outf,
                            BatchSkip sk) {
    // (the level-2 solve may overwrite ml.c00, a scratch array)
    const int t = 256;
    k_ml_restrict<<<dim3((ml.Nc00 + t - 1) / t, nb), t, 0, cx.stream>>>(ml.nc1, ml.lo0, ml.nc00, ml.lo2, ml.hi2,
                                                                       ml.off2, ml.wt2, c, ml.c00, sk);
    if (ml.blk00) launch_coarse_block_solve(cx, nb, ml.cblk00, ml.c00, ml.c00p, nullptr, sk);   // (c00 overwritten)
    else launch_coarse_matvec(cx, nb, ml.A00inv, ml.Nc00, ml.c00, ml.c00p, nullptr, sk);
    k_ml_prolong<<<dim3((ml.Nc + t - 1) / t, nb), t, 0, cx.stream>>>(ml.nc1, ml.lo0, ml.nc00, ml.c02, ml.w2, ml.c00p,
                                                                    ml.q, sk);
    k_ml_resid<<<dim3((ml.Nc + t - 1) / t, nb), t, 0, cx.stream>>>(ml.nc1, ml.A0b, c, ml.q, ml.wv, sk);
    k_ml_local<<<dim3((ml.max_own + 7) / 8, ml.nsub, nb), t, 0, cx.stream>>>(ml.nc1, ml.sub, ml.own, ml.aoff, ml.Ainv,
                                                                            ml.q, ml.wv, out, sk);
    if (outf) k_ml_to_c64<<<dim3((ml.Nc + t - 1) / t, nb), t, 0, cx.stream>>>(ml.Nc, out, outf, sk);
}

}  // namespace hzs
