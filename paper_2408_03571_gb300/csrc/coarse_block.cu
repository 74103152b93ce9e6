// Exact coarse solve A_0 c' = c (Eq. 4, Section 4) by block-tridiagonal LU, for
// coarse spaces too large for the dense inverse (|G_H| up to 40 401 in the
// H = 4h experiments of Section 5).
//
// Coarse unknown (J, I) has index J nc1 + I.  A coarse basis function couples
// coarse rows J and J + dJ only for |dJ| <= s (s = 2 for B_2, 1 for P_1), so
// grouping s consecutive coarse rows into one block row gives a block-
// tridiagonal matrix with blocks of size b_i = (rows in group i) * nc1:
//   D_i (b_i x b_i), L_i (b_i x b_{i-1}), U_i (b_i x b_{i+1}).
// Set-up (FP64): S_0 = D_0, S_i = D_i - L_i Q_{i-1};  W_i = S_i^{-1} (Gauss-Jordan
// with partial pivoting), P_i = W_i L_i, Q_i = W_i U_i; A_0's band form is kept too
// (L_i and U_i have at most 10 entries a row there).
// Solve, two forms of the same block substitution:
//  - many right-hand sides (FP64-bound): y_0 = W_0 c_0, y_i = W_i (c_i - L_i y_{i-1});
//    x_{m-1} = y_{m-1}, x_i = y_i - W_i (U_i x_{i+1}): 2m - 1 dense products with the
//    W_i (one warp per row and right-hand side), each after a banded product;
//  - one or two right-hand sides (latency-bound): y_i = W_i c_i - P_i y_{i-1},
//    x_i = y_i - Q_i x_{i+1}: one launch per block step, 3m - 2 dense products.
#include <vector>

#include "kernels.cuh"

namespace hzs {

// dst (rows x cols, row-major) = the block of the banded matrix with row range
// [r0, r0+rows) and column range [c0, c0+cols); the band of radius rad holds
// (2 rad + 1)^2 offsets (dI, dJ) in [-rad, rad]^2 per row, offset index
// o = (dJ + rad) (2 rad + 1) + (dI + rad) (rad = 2: A_0; rad = 3: the Galerkin matrix
// of a coarse space on G_H).
__global__ void k_band_to_block(int nc1, int rad, const double2* __restrict__ A0b, int r0, int rows, int c0, int cols,
                                double2* __restrict__ dst) {
    const int bw = 2 * rad + 1;
    const long long total = (long long)rows * cols;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int rr = (int)(t / cols), cc = (int)(t % cols);
        const int row = r0 + rr, col = c0 + cc;
        const int I = row % nc1, J = row / nc1, I2 = col % nc1, J2 = col / nc1;
        const int dI = I2 - I, dJ = J2 - J;
        double2 v = make_double2(0.0, 0.0);
        if (dI >= -rad && dI <= rad && dJ >= -rad && dJ <= rad)
            v = A0b[(size_t)row * bw * bw + (dJ + rad) * bw + (dI + rad)];
        dst[t] = v;
    }
}

// C (M x N) = beta C + alpha A (M x K) B (K x N), complex FP64, row-major.
// 16 x 16 output tile per block, K in steps of 16 through shared memory.
__global__ void k_zgemm(int M, int N, int K, double alpha, const double2* __restrict__ A, int lda,
                        const double2* __restrict__ B, int ldb, double beta, double2* __restrict__ C, int ldc) {
    __shared__ double2 As[16][17], Bs[16][17];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    double2 acc = make_double2(0.0, 0.0);
    for (int k0 = 0; k0 < K; k0 += 16) {
        As[ty][tx] = (row < M && k0 + tx < K) ? A[(size_t)row * lda + k0 + tx] : make_double2(0.0, 0.0);
        Bs[ty][tx] = (k0 + ty < K && col < N) ? B[(size_t)(k0 + ty) * ldb + col] : make_double2(0.0, 0.0);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = cfma(As[ty][k], Bs[k][tx], acc);
        __syncthreads();
    }
    if (row < M && col < N) {
        double2 c = beta != 0.0 ? cscale(C[(size_t)row * ldc + col], beta) : make_double2(0.0, 0.0);
        c.x += alpha * acc.x; c.y += alpha * acc.y;
        C[(size_t)row * ldc + col] = c;
    }
}

static void zgemm(const Ctx& cx, int M, int N, int K, double alpha, const double2* A, int lda, const double2* B,
                  int ldb, double beta, double2* C, int ldc) {
    const dim3 blk(16, 16), grd((N + 15) / 16, (M + 15) / 16);
    k_zgemm<<<grd, blk, 0, cx.stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

// One block step of the solve, batch entry r = blockIdx.y, one warp per row:
//   out[row] = sign_a * (Ma x_a)[row] + sign_b * (Mb x_b)[row] + (base ? base[row] : 0)
// (Ma: rows x na, Mb: rows x nb, either may be absent).
__global__ void k_cb_step(int rows, const double2* __restrict__ Ma, const double2* __restrict__ xa, int na,
                          const double2* __restrict__ Mb, const double2* __restrict__ xb, int nbc,
                          const double2* __restrict__ base, double2* __restrict__ out, long long stride,
                          BatchSkip sk) {
    const int r = blockIdx.y;
    if (sk.flag && sk.flag[(size_t)r * sk.stride]) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= rows) return;
    const long long off = (long long)r * stride;
    double2 acc = make_double2(0.0, 0.0);
    if (Ma) {
        const double2* m = Ma + (size_t)warp * na;
        const double2* x = xa + off;
        for (int k = lane; k < na; k += 32) acc = cfma(m[k], x[k], acc);
    }
    if (Mb) {
        const double2* m = Mb + (size_t)warp * nbc;
        const double2* x = xb + off;
        for (int k = lane; k < nbc; k += 32) acc = cfms(m[k], x[k], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) {
        if (base) acc = cadd(acc, base[off + warp]);
        out[off + warp] = acc;
    }
}

// The same step with each row split over kCbWarpsPerRow warps (few right-hand sides:
// the step's latency, not the FP64 pipe, bounds it): every warp sums a strided quarter
// of the row, the quarters are added in a fixed order through shared memory.
constexpr int kCbWarpsPerRow = 4;
__global__ void __launch_bounds__(256) k_cb_step_split(int rows, const double2* __restrict__ Ma,
                                                       const double2* __restrict__ xa, int na,
                                                       const double2* __restrict__ Mb,
                                                       const double2* __restrict__ xb, int nbc,
                                                       const double2* __restrict__ base,
                                                       double2* __restrict__ out, long long stride, BatchSkip sk) {
    constexpr int W = kCbWarpsPerRow, RPB = 256 / 32 / W;     // rows per block
    __shared__ double2 part[RPB][W];
    const int r = blockIdx.y;
    if (sk.flag && sk.flag[(size_t)r * sk.stride]) return;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rib = wib / W, q = wib % W;
    const int row = blockIdx.x * RPB + rib;
    const long long off = (long long)r * stride;
    double2 acc = make_double2(0.0, 0.0);
    if (row < rows) {
        if (Ma) {
            const double2* m = Ma + (size_t)row * na;
            const double2* x = xa + off;
            for (int k = q * 32 + lane; k < na; k += 32 * W) acc = cfma(m[k], x[k], acc);
        }
        if (Mb) {
            const double2* m = Mb + (size_t)row * nbc;
            const double2* x = xb + off;
            for (int k = q * 32 + lane; k < nbc; k += 32 * W) acc = cfms(m[k], x[k], acc);
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) part[rib][q] = acc;
    __syncthreads();
    if (q == 0 && lane == 0 && row < rows) {
        double2 t = part[rib][0];
#pragma unroll
        for (int u = 1; u < W; ++u) t = cadd(t, part[rib][u]);
        if (base) t = cadd(t, base[off + row]);
        out[off + row] = t;
    }
}

// Banded coupling of block row i (rows [r0, r0 + rows)) with the unknowns
// [cr0, cr0 + crows) of a neighbouring block row, batch entry r = blockIdx.y, one
// thread per row: acc = sum over A_0's band entries of the row whose column lies in
// that range of A0b[row, o] x[col];  v[row] = v[row] - acc (subtract) or acc.
__global__ void k_cb_band(int nc1, int rad, const double2* __restrict__ A0b, int r0, int rows, int cr0, int crows,
                          const double2* __restrict__ x, double2* __restrict__ v, long long stride, int subtract,
                          BatchSkip sk) {
    const int bw = 2 * rad + 1;
    const int r = blockIdx.y;
    if (sk.flag && sk.flag[(size_t)r * sk.stride]) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows) return;
    const long long off = (long long)r * stride;
    const int row = r0 + t, I = row % nc1, J = row / nc1;
    double2 acc = make_double2(0.0, 0.0);
    for (int dJ = -rad; dJ <= rad; ++dJ) {
        const int J2 = J + dJ;
        if (J2 < 0 || J2 >= nc1) continue;
        for (int dI = -rad; dI <= rad; ++dI) {
            const int I2 = I + dI;
            if (I2 < 0 || I2 >= nc1) continue;
            const int col = J2 * nc1 + I2;
            if (col < cr0 || col >= cr0 + crows) continue;
            acc = cfma(A0b[(size_t)row * bw * bw + (dJ + rad) * bw + (dI + rad)], x[off + col], acc);
        }
    }
    v[off + row] = subtract ? csub(v[off + row], acc) : acc;
}

__global__ void k_c128_to_c64_batched(int Nc, const double2* __restrict__ a, float2* __restrict__ b, BatchSkip sk) {
    const int r = blockIdx.y;
    if (sk.flag && sk.flag[(size_t)r * sk.stride]) return;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Nc; e += gridDim.x * blockDim.x)
        b[(size_t)r * Nc + e] = to_f(a[(size_t)r * Nc + e]);
}

int coarse_block_setup(const Ctx& cx, int nc1, int s, int rad, double2* A0b, CoarseBlockLU& lu, double* minpiv) {
    lu = CoarseBlockLU{};
    lu.nc1 = nc1;
    lu.s = s;
    lu.rad = rad;
    lu.m = (nc1 + s - 1) / s;
    lu.A0b = A0b;
    const int m = lu.m;
    std::vector<int> b(m), r0(m);
    for (int i = 0; i < m; ++i) {
        r0[i] = i * s * nc1;
        b[i] = (std::min(nc1, (i + 1) * s) - i * s) * nc1;
    }
    long long wsz = 0, psz = 0, qsz = 0;
    std::vector<long long> wo(m), po(m), qo(m);
    for (int i = 0; i < m; ++i) {
        wo[i] = wsz; wsz += (long long)b[i] * b[i];
        po[i] = psz; if (i > 0) psz += (long long)b[i] * b[i - 1];
        qo[i] = qsz; if (i + 1 < m) qsz += (long long)b[i] * b[i + 1];
    }
    const int bmax = s * nc1;
    double2 *D = nullptr, *Lb = nullptr, *Ub = nullptr;
    auto fail = [&]() {
        cudaFree(D); cudaFree(Lb); cudaFree(Ub);
        cudaFree(lu.W); cudaFree(lu.P); cudaFree(lu.Q); cudaFree(lu.A0b);
        lu = CoarseBlockLU{};
        return -1;
    };
    if (cudaMalloc(&lu.W, (size_t)wsz * sizeof(double2)) != cudaSuccess) return fail();
    if (cudaMalloc(&lu.P, (size_t)(psz > 0 ? psz : 1) * sizeof(double2)) != cudaSuccess) return fail();
    if (cudaMalloc(&lu.Q, (size_t)(qsz > 0 ? qsz : 1) * sizeof(double2)) != cudaSuccess) return fail();
    if (cudaMalloc(&D, (size_t)bmax * bmax * sizeof(double2)) != cudaSuccess) return fail();
    if (cudaMalloc(&Lb, (size_t)bmax * bmax * sizeof(double2)) != cudaSuccess) return fail();
    if (cudaMalloc(&Ub, (size_t)bmax * bmax * sizeof(double2)) != cudaSuccess) return fail();
    double mp = 1e300;
    int singular = 0;
    const int cb = 4 * cx.num_sms;
    for (int i = 0; i < m; ++i) {
        const int bi = b[i];
        k_band_to_block<<<cb, 256, 0, cx.stream>>>(nc1, rad, A0b, r0[i], bi, r0[i], bi, D);
        if (i > 0) {
            // S_i = D_i - L_i Q_{i-1}
            k_band_to_block<<<cb, 256, 0, cx.stream>>>(nc1, rad, A0b, r0[i], bi, r0[i - 1], b[i - 1], Lb);
            zgemm(cx, bi, bi, b[i - 1], -1.0, Lb, b[i - 1], lu.Q + qo[i - 1], bi, 1.0, D, bi);
        }
        double piv = 0.0;
        const int rc = gj_invert(cx, D, bi, &piv);      // D <- S_i^{-1}
        if (rc < 0) return fail();
        if (rc > 0) singular = 1;
        mp = std::min(mp, piv);
        if (cudaMemcpyAsync(lu.W + wo[i], D, (size_t)bi * bi * sizeof(double2), cudaMemcpyDeviceToDevice,
                            cx.stream) != cudaSuccess)
            return fail();
        if (i > 0) zgemm(cx, bi, b[i - 1], bi, 1.0, lu.W + wo[i], bi, Lb, b[i - 1], 0.0, lu.P + po[i], b[i - 1]);
        if (i + 1 < m) {
            k_band_to_block<<<cb, 256, 0, cx.stream>>>(nc1, rad, A0b, r0[i], bi, r0[i + 1], b[i + 1], Ub);
            zgemm(cx, bi, b[i + 1], bi, 1.0, lu.W + wo[i], bi, Ub, b[i + 1], 0.0, lu.Q + qo[i], b[i + 1]);
        }
    }
    const cudaError_t e = cudaStreamSynchronize(cx.stream);
    cudaFree(D); cudaFree(Lb); cudaFree(Ub);
    if (e != cudaSuccess) {
        cudaFree(lu.W); cudaFree(lu.P); cudaFree(lu.Q); cudaFree(lu.A0b);
        lu = CoarseBlockLU{};
        return -1;
    }
    lu.b = b; lu.r0 = r0; lu.wo = wo; lu.po = po; lu.qo = qo;
    *minpiv = mp;
    return singular ? 1 : 0;
}

void coarse_block_free(CoarseBlockLU& lu) {
    coarse_oz_free(lu);
    cudaFree(lu.W); cudaFree(lu.P); cudaFree(lu.Q); cudaFree(lu.A0b);
    lu = CoarseBlockLU{};
}

void launch_coarse_block_solve(const Ctx& cx, int nb, const CoarseBlockLU& lu, double2* c, double2* out,
                               float2* outf, BatchSkip sk) {
    const int m = lu.m, Nc = lu.nc1 * lu.nc1;
    const int threads = 256, wpb = threads / 32;
    if (nb <= 2) {
        // few right-hand sides: one launch per block step, W_i c_i - P_i y_{i-1} and
        // y_i - Q_i x_{i+1}, each row split over kCbWarpsPerRow warps
        constexpr int rpb = 256 / 32 / kCbWarpsPerRow;
        for (int i = 0; i < m; ++i) {
            const int bi = lu.b[i];
            const dim3 grd((bi + rpb - 1) / rpb, nb);
            k_cb_step_split<<<grd, threads, 0, cx.stream>>>(bi, lu.W + lu.wo[i], c + lu.r0[i], bi,
                                                            i > 0 ? lu.P + lu.po[i] : nullptr,
                                                            i > 0 ? out + lu.r0[i - 1] : nullptr,
                                                            i > 0 ? lu.b[i - 1] : 0, nullptr, out + lu.r0[i], Nc, sk);
        }
        for (int i = m - 2; i >= 0; --i) {
            const int bi = lu.b[i];
            const dim3 grd((bi + rpb - 1) / rpb, nb);
            k_cb_step_split<<<grd, threads, 0, cx.stream>>>(bi, nullptr, nullptr, 0, lu.Q + lu.qo[i],
                                                            out + lu.r0[i + 1], lu.b[i + 1], out + lu.r0[i],
                                                            out + lu.r0[i], Nc, sk);
        }
        if (outf) k_c128_to_c64_batched<<<dim3((Nc + 255) / 256, nb), 256, 0, cx.stream>>>(Nc, out, outf, sk);
        return;
    }
    // the dense products on the tensor cores (FP64-accurate digit-slice products) when
    // they are built and the work space holds nb right-hand sides, else on the FP64 pipe
    const bool oz = lu.Aoz && nb <= lu.oz_cap;
    // forward: c_i <- c_i - L_i y_{i-1}, y_i = W_i c_i
    for (int i = 0; i < m; ++i) {
        const int bi = lu.b[i];
        if (i > 0)
            k_cb_band<<<dim3((bi + 127) / 128, nb), 128, 0, cx.stream>>>(lu.nc1, lu.rad, lu.A0b, lu.r0[i], bi, lu.r0[i - 1],
                                                                         lu.b[i - 1], out, c, Nc, 1, sk);
        if (oz) {
            launch_coarse_oz_step(cx, nb, lu, i, c + lu.r0[i], out + lu.r0[i], false, Nc, sk);
            continue;
        }
        const dim3 grd((bi + wpb - 1) / wpb, nb);
        k_cb_step<<<grd, threads, 0, cx.stream>>>(bi, lu.W + lu.wo[i], c + lu.r0[i], bi, nullptr, nullptr, 0, nullptr,
                                                  out + lu.r0[i], Nc, sk);
    }
    // backward: c_i <- U_i x_{i+1}, x_i = y_i - W_i c_i
    for (int i = m - 2; i >= 0; --i) {
        const int bi = lu.b[i];
        k_cb_band<<<dim3((bi + 127) / 128, nb), 128, 0, cx.stream>>>(lu.nc1, lu.rad, lu.A0b, lu.r0[i], bi, lu.r0[i + 1],
                                                                     lu.b[i + 1], out, c, Nc, 0, sk);
        if (oz) {
            launch_coarse_oz_step(cx, nb, lu, i, c + lu.r0[i], out + lu.r0[i], true, Nc, sk);
            continue;
        }
        const dim3 grd((bi + wpb - 1) / wpb, nb);
        k_cb_step<<<grd, threads, 0, cx.stream>>>(bi, nullptr, nullptr, 0, lu.W + lu.wo[i], c + lu.r0[i], bi,
                                                  out + lu.r0[i], out + lu.r0[i], Nc, sk);
    }
    if (outf) k_c128_to_c64_batched<<<dim3((Nc + 255) / 256, nb), 256, 0, cx.stream>>>(Nc, out, outf, sk);
}

}  // namespace hzs
