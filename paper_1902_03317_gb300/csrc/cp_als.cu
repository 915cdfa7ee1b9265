// One sweep of CP alternating least squares (the CPD method of Sec. 2.2,
// whose bottleneck is MTTKRP; steps as in the Kolda-Bader survey the paper
// cites).  Per mode n: M = MTTKRP_n (the streaming kernel), V = Hadamard
// product of the other factors' Gram matrices, U_n = M V^{-1}, column
// 2-norms lam, U_n /= lam; then the fit from the norm expansion.
//
// Everything but MTTKRP is small or a single pass over a factor:
//   k_gram        U^T U of an I x R factor: rows staged in shared memory 32
//                 at a time, FP32 sums over 128 rows folded into FP64, one
//                 R x R FP64 partial per block, summed in fixed order
//   k_als_solve   V^{-1} by in-place Gauss-Jordan in FP64 (V is symmetric
//                 positive definite when the factors have full column rank,
//                 so no pivoting), one block
//   k_als_rows    U_n = M W, a warp per four rows, W in shared memory
//   k_als_norm    lam and the normalised Gram matrix of U_n from the raw one
//   k_als_scale   U_n(:, r) *= 1 / lam_r, and on the last mode the column
//                 sums of M .* U_n for <X, model>
//   k_als_fit     ||model||^2 = lam^T (Hadamard of all Grams) lam and the fit
// All of these are HBM- or latency-bound and take a few percent of a sweep.
#include <algorithm>

#include "pasta_internal.cuh"

namespace pasta {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int kGramThreads = 512;
constexpr int kGramRows = 32;     // rows staged per batch
constexpr int kGramFold = 4;      // batches summed in FP32 before the FP64 fold
constexpr int kSolveThreads = 1024;

// Per-block partial Gram matrix of rows [b * chunk, (b + 1) * chunk).  Thread
// t owns the pairs p = t + kGramThreads * q (q < PPT) of the R x R matrix.
template <int PPT>
__global__ void __launch_bounds__(kGramThreads) k_gram(const float *U, uint64_t I, int R,
                                                       uint64_t chunk, double *part) {
    __shared__ float sU[kGramRows * PASTA_ALS_MAX_RANK];
    const int t = threadIdx.x;
    const int RR = R * R;
    uint32_t prs[PPT];  // (r << 16) | s of each owned pair
    float a32[PPT];
    double a64[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int p = t + kGramThreads * q;
        prs[q] = p < RR ? ((uint32_t)(p / R) << 16) | (uint32_t)(p % R) : 0u;
        a32[q] = 0.f;
        a64[q] = 0.0;
    }
    const uint64_t r0 = (uint64_t)blockIdx.x * chunk;
    const uint64_t r1 = min(I, r0 + chunk);
    int fold = 0;
    for (uint64_t b = r0; b < r1; b += kGramRows) {
        const int nrows = (int)min((uint64_t)kGramRows, r1 - b);
        const float *src = U + b * (uint64_t)R;
        for (int e = t; e < kGramRows * R; e += kGramThreads)
            sU[e] = e < nrows * R ? src[e] : 0.f;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            float s = 0.f;
#pragma unroll 8
            for (int j = 0; j < kGramRows; ++j)
                s = fmaf(sU[j * R + (prs[q] >> 16)], sU[j * R + (prs[q] & 0xFFFFu)], s);
            a32[q] += s;
        }
        if (++fold == kGramFold) {
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                a64[q] += (double)a32[q];
                a32[q] = 0.f;
            }
            fold = 0;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int p = t + kGramThreads * q;
        if (p < RR) part[(uint64_t)blockIdx.x * RR + p] = a64[q] + (double)a32[q];
    }
}

// out[p] = sum over blocks b of part[b * n + p], in block order.
__global__ void k_sum_parts(const double *part, int nblk, int n, double *out) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[(uint64_t)b * n + p];
        out[p] = s;
    }
}

// W = V^{-1} with V = prod_{k != n} G_k (element-wise).  In-place
// Gauss-Jordan: for each k the pivot row is divided by the pivot and every
// other row loses its multiple of it.  A pivot that is not positive relative
// to its original diagonal marks V singular: status = n + 1.
__global__ void __launch_bounds__(kSolveThreads) k_als_solve(const double *grams, int N, int n,
                                                             int R, float *W, int *status) {
    extern __shared__ double sA[];  // R * R, then R column factors, then R diagonals
    double *f = sA + R * R;
    double *d0 = f + R;
    const int t = threadIdx.x;
    const int RR = R * R;
    for (int p = t; p < RR; p += kSolveThreads) {
        double v = 1.0;
        for (int k = 0; k < N; ++k)
            if (k != n) v *= grams[(uint64_t)k * RR + p];
        sA[p] = v;
    }
    __syncthreads();
    for (int i = t; i < R; i += kSolveThreads) d0[i] = sA[i * R + i];
    __syncthreads();
    for (int k = 0; k < R; ++k) {
        const double piv = sA[k * R + k];
        if (!(piv > 1e-14 * d0[k]) || !isfinite(piv)) {  // uniform across the block
            if (t == 0) atomicCAS(status, 0, n + 1);
            for (int p = t; p < RR; p += kSolveThreads) W[p] = 0.f;
            return;
        }
        for (int i = t; i < R; i += kSolveThreads) f[i] = sA[i * R + k];
        __syncthreads();
        for (int j = t; j < R; j += kSolveThreads) sA[k * R + j] = (j == k ? 1.0 : sA[k * R + j]) / piv;
        __syncthreads();
        for (int p = t; p < RR; p += kSolveThreads) {
            const int i = p / R, j = p - (p / R) * R;
            if (i != k) sA[p] = (j == k ? 0.0 : sA[p]) - f[i] * sA[k * R + j];
        }
        __syncthreads();
    }
    for (int p = t; p < RR; p += kSolveThreads) W[p] = (float)sA[p];
}

// U(i, :) = M(i, :) W for four rows per warp iteration; lane owns columns
// lane + 32 c (c < CPL); W (R x R) sits in shared memory.
template <int CPL>
__global__ void __launch_bounds__(256) k_als_rows(const float *M, uint64_t I, int R, const float *W,
                                                  float *U) {
    extern __shared__ float sW[];
    for (int p = threadIdx.x; p < R * R; p += blockDim.x) sW[p] = W[p];
    __syncthreads();
    constexpr int ROWS = 4;
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t i0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * ROWS; i0 < I;
         i0 += warps * ROWS) {
        float mv[ROWS][CPL], acc[ROWS][CPL];
#pragma unroll
        for (int q = 0; q < ROWS; ++q)
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int col = lane + 32 * c;
                mv[q][c] = (i0 + q < I && col < R) ? M[(i0 + q) * R + col] : 0.f;
                acc[q][c] = 0.f;
            }
        for (int r = 0; r < R; ++r) {
            float w[CPL];
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int col = lane + 32 * c;
                w[c] = col < R ? sW[r * R + col] : 0.f;
            }
            const int src_c = r >> 5;  // register slot holding column r
#pragma unroll
            for (int q = 0; q < ROWS; ++q) {
                float held = mv[q][0];
#pragma unroll
                for (int c = 1; c < CPL; ++c)
                    if (src_c == c) held = mv[q][c];
                const float m = __shfl_sync(FULL, held, r & 31);
#pragma unroll
                for (int c = 0; c < CPL; ++c) acc[q][c] = fmaf(m, w[c], acc[q][c]);
            }
        }
#pragma unroll
        for (int q = 0; q < ROWS; ++q)
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int col = lane + 32 * c;
                if (i0 + q < I && col < R) U[(i0 + q) * R + col] = acc[q][c];
            }
    }
}

// lam_r = sqrt(Graw(r, r)); inv_r = 1 / lam_r (0 for a zero column);
// Gn(r, s) = Graw(r, s) inv_r inv_s, the Gram matrix of the scaled factor.
__global__ void k_als_norm(const double *graw, int R, double *lam, double *inv, double *gn) {
    __shared__ double sinv[PASTA_ALS_MAX_RANK];
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const double l = sqrt(max(graw[r * R + r], 0.0));
        lam[r] = l;
        sinv[r] = l > 0.0 ? 1.0 / l : 0.0;
        inv[r] = sinv[r];
    }
    __syncthreads();
    for (int p = threadIdx.x; p < R * R; p += blockDim.x) gn[p] = graw[p] * sinv[p / R] * sinv[p % R];
}

// U(:, r) *= inv_r.  With M given, also per-block column sums of M .* U
// (the scaled U): thread t works on column t % R of rows t / R, t / R + rpb,
// ... (rpb = 256 / R rows per block step).
__global__ void __launch_bounds__(256) k_als_scale(float *U, const float *M, uint64_t I, int R,
                                                   const double *inv, double *part) {
    __shared__ double col[PASTA_ALS_MAX_RANK];
    const int t = threadIdx.x;
    const int rpb = 256 / R;
    const int c = t % R;
    const bool active = t < rpb * R;
    for (int r = t; r < R; r += 256) col[r] = 0.0;
    __syncthreads();
    const float s = (float)inv[c];
    double acc64 = 0.0;
    float acc = 0.f;
    int n = 0;
    if (active) {
        for (uint64_t i = (uint64_t)blockIdx.x * rpb + t / R; i < I; i += (uint64_t)gridDim.x * rpb) {
            const uint64_t e = i * R + c;
            const float u = U[e] * s;
            U[e] = u;
            if (M) {
                acc = fmaf(M[e], u, acc);
                if (++n == 64) {
                    acc64 += (double)acc;
                    acc = 0.f;
                    n = 0;
                }
            }
        }
    }
    if (!M) return;
    acc64 += (double)acc;
    if (active) atomicAdd(&col[c], acc64);
    __syncthreads();
    for (int r = t; r < R; r += 256) part[(uint64_t)blockIdx.x * R + r] = col[r];
}

// Fit from ||X||^2, lam, the Gram matrices of the final factors and the
// column sums of M_{N-1} .* U_{N-1}; fixed-order reductions.
__global__ void __launch_bounds__(256) k_als_fit(const double *grams, int N, int R, const double *lam,
                                                 const double *inner, const double *normx2,
                                                 double *fit) {
    __shared__ double ws[8];
    const int t = threadIdx.x;
    const int RR = R * R;
    double acc = 0.0;
    for (int p = t; p < RR; p += 256) {
        double h = lam[p / R] * lam[p % R];
        for (int k = 0; k < N; ++k) h *= grams[(uint64_t)k * RR + p];
        acc += h;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if ((t & 31) == 0) ws[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
        double model2 = 0.0;
        for (int w = 0; w < 8; ++w) model2 += ws[w];
        double in = 0.0;
        for (int r = 0; r < R; ++r) in += lam[r] * inner[r];
        const double x2 = *normx2;
        const double res2 = max(x2 + model2 - 2.0 * in, 0.0);
        *fit = x2 > 0.0 ? 1.0 - sqrt(res2) / sqrt(x2) : 0.0;
    }
}

// Per-block sums of squared values: FP32 over 64 values, FP64 beyond.
__global__ void __launch_bounds__(256) k_sumsq(const float *val, uint64_t n, double *part) {
    __shared__ double ws[8];
    double acc64 = 0.0;
    float acc = 0.f;
    int c = 0;
    for (uint64_t m = (uint64_t)blockIdx.x * 256 + threadIdx.x; m < n; m += (uint64_t)gridDim.x * 256) {
        acc = fmaf(val[m], val[m], acc);
        if (++c == 64) {
            acc64 += (double)acc;
            acc = 0.f;
            c = 0;
        }
    }
    acc64 += (double)acc;
    for (int o = 16; o > 0; o >>= 1) acc64 += __shfl_xor_sync(FULL, acc64, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc64;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += ws[w];
        part[blockIdx.x] = s;
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Launch k_gram for an I x R factor into G (R x R), using `part` (room for
// gram_blocks() * R * R doubles).
pasta_status gram(const float *U, uint64_t I, int R, int nblk_max, double *part, double *G,
                  cudaStream_t s) {
    const uint64_t batches = (I + kGramRows - 1) / kGramRows;
    const int nblk = (int)std::max<uint64_t>(1, std::min<uint64_t>(batches, (uint64_t)nblk_max));
    const uint64_t chunk = ((batches + nblk - 1) / nblk) * kGramRows;
    const int RR = R * R;
    if (RR <= kGramThreads)
        k_gram<1><<<nblk, kGramThreads, 0, s>>>(U, I, R, chunk, part);
    else if (RR <= 2 * kGramThreads)
        k_gram<2><<<nblk, kGramThreads, 0, s>>>(U, I, R, chunk, part);
    else if (RR <= 8 * kGramThreads)
        k_gram<8><<<nblk, kGramThreads, 0, s>>>(U, I, R, chunk, part);
    else
        k_gram<32><<<nblk, kGramThreads, 0, s>>>(U, I, R, chunk, part);
    k_sum_parts<<<(RR + 255) / 256, 256, 0, s>>>(part, nblk, RR, G);
    return PASTA_OK;
}

pasta_status rows(const float *M, uint64_t I, int R, const float *W, float *U, int num_sms,
                  cudaStream_t s) {
    const size_t smem = (size_t)R * R * sizeof(float);
    const uint64_t need = (I + 31) / 32;  // blocks of 8 warps x 4 rows
    const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)num_sms * 4));
    if (R <= 32) {
        PASTA_CUDA(cudaFuncSetAttribute(k_als_rows<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_als_rows<1><<<blocks, 256, smem, s>>>(M, I, R, W, U);
    } else if (R <= 64) {
        PASTA_CUDA(cudaFuncSetAttribute(k_als_rows<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_als_rows<2><<<blocks, 256, smem, s>>>(M, I, R, W, U);
    } else {
        PASTA_CUDA(cudaFuncSetAttribute(k_als_rows<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_als_rows<4><<<blocks, 256, smem, s>>>(M, I, R, W, U);
    }
    return PASTA_OK;
}

}  // namespace

pasta_status run_cp_als_sweep(pasta_coo_s *X, float *const *U, int R, double *lambda, double *fit,
                              cudaStream_t s) {
    const int N = X->order;
    const int RR = R * R;
    uint64_t imax = 0;
    for (int k = 0; k < N; ++k) imax = std::max(imax, X->dims[k]);
    const int nblk = 2 * X->num_sms;  // k_gram / k_als_scale grid cap

    // one scratch allocation, 256-byte aligned pieces
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t oM = take(imax * (size_t)R * sizeof(float));
    const size_t oG = take((size_t)N * RR * sizeof(double));
    const size_t oGraw = take((size_t)RR * sizeof(double));
    const size_t oW = take((size_t)RR * sizeof(float));
    const size_t oInv = take((size_t)R * sizeof(double));
    const size_t oPart = take((size_t)nblk * RR * sizeof(double));
    const size_t oInner = take((size_t)R * sizeof(double));
    const size_t oStatus = take(sizeof(int));
    char *base = nullptr;
    PASTA_CUDA(scratch_alloc((void **)&base, off, s));
    float *M = reinterpret_cast<float *>(base + oM);
    double *G = reinterpret_cast<double *>(base + oG);
    double *graw = reinterpret_cast<double *>(base + oGraw);
    float *W = reinterpret_cast<float *>(base + oW);
    double *inv = reinterpret_cast<double *>(base + oInv);
    double *part = reinterpret_cast<double *>(base + oPart);
    double *inner = reinterpret_cast<double *>(base + oInner);
    int *status = reinterpret_cast<int *>(base + oStatus);

    pasta_status st = PASTA_OK;
    auto fail = [&](pasta_status e) {
        cudaFreeAsync(base, s);
        return e;
    };
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "cudaMemsetAsync(status)"));

    // ||X||^2 once per handle (the values never change after create)
    if (!X->als_normsq) {
        cudaError_t e = cudaMalloc(&X->als_normsq, sizeof(double));
        if (e != cudaSuccess) {
            X->als_normsq = nullptr;
            return fail(cuda_fail(e, "cudaMalloc(normsq)"));
        }
        const int b = (int)std::max<uint64_t>(1, std::min<uint64_t>((X->nnz + 255) / 256, (uint64_t)nblk));
        k_sumsq<<<b, 256, 0, s>>>(X->orig.val, X->nnz, part);
        k_sum_parts<<<1, 32, 0, s>>>(part, b, 1, X->als_normsq);
    }

    for (int k = 0; k < N; ++k) gram(U[k], X->dims[k], R, nblk, part, G + (size_t)k * RR, s);

    const size_t solve_smem = ((size_t)RR + 2 * R) * sizeof(double);
    if (cudaFuncSetAttribute(k_als_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)solve_smem) != cudaSuccess)
        return fail(cuda_fail(cudaGetLastError(), "cudaFuncSetAttribute(k_als_solve)"));
    for (int n = 0; n < N; ++n) {
        const uint64_t I = X->dims[n];
        st = launch_mttkrp(X, X->sorted[n], reinterpret_cast<const void *const *>(U), PASTA_F32, n, R,
                           M, s);
        if (st != PASTA_OK) return fail(st);
        k_als_solve<<<1, kSolveThreads, solve_smem, s>>>(G, N, n, R, W, status);
        st = rows(M, I, R, W, U[n], X->num_sms, s);
        if (st != PASTA_OK) return fail(st);
        gram(U[n], I, R, nblk, part, graw, s);
        k_als_norm<<<1, 256, 0, s>>>(graw, R, lambda, inv, G + (size_t)n * RR);
        const bool last = (n == N - 1);
        const int rpb = 256 / R;
        const int b = (int)std::max<uint64_t>(1, std::min<uint64_t>((I + rpb - 1) / rpb, (uint64_t)nblk));
        k_als_scale<<<b, 256, 0, s>>>(U[n], last ? M : nullptr, I, R, inv, part);
        if (last) k_sum_parts<<<1, 128, 0, s>>>(part, b, R, inner);
    }
    if (fit) k_als_fit<<<1, 256, 0, s>>>(G, N, R, lambda, inner, X->als_normsq, fit);
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return fail(cuda_fail(le, "CP-ALS kernels"));

    int h_status = 0;
    cudaError_t e = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(base, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "CP-ALS status read");
    if (h_status != 0) {
        set_error("CP-ALS: V of mode %d is singular (non-positive pivot)", h_status - 1);
        return PASTA_ERR_SINGULAR;
    }
    return PASTA_OK;
}

}  // namespace pasta
