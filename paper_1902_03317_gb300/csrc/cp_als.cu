// One sweep of CP alternating least squares (the CPD method of Sec. 2.2,
// whose bottleneck is MTTKRP; steps as in the Kolda-Bader survey the paper
// cites).  Per mode n: M = MTTKRP_n (the streaming kernel), V = Hadamard
// product of the other factors' Gram matrices, U_n = M V^{-1}, column 2-norms
// lam, U_n /= lam; then the fit from the norm expansion.
//
// Besides MTTKRP, two passes over I_n x R data remain per mode: U_n = M W
// (W = V^{-1}), which also sums each column's squares and its products with
// M; and one pass that divides the columns by lam and forms the Gram matrix
// of the factor as stored, which the next modes' V uses.  (Forming lam from
// W G_M W instead, to fold the normalisation into the first pass, lost
// accuracy: that quadratic form cancels when V is ill-conditioned.)
//   k_gram        U^T U (optionally scaling U in place first): 4 x 4 register
//                 tiles per thread over rows staged in shared memory, FP32
//                 per batch, FP64 across batches; per-block partials summed
//                 in fixed order (k_sum_parts)
//   k_als_solve   V^{-1} by in-place Gauss-Jordan in FP64 (V is symmetric
//                 positive definite when the factors have full column rank,
//                 so no pivoting), one block
//   k_als_rows    U_n = M W, a warp per four rows, plus column statistics
//   k_als_lambda  lam, 1 / lam and <M, U_n> per column
//   k_als_fit     ||model||^2 = lam^T (Hadamard of all Grams) lam and the fit
#include <algorithm>

#include "pasta_internal.cuh"

namespace pasta {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int kGramFloats = 4096;  // floats staged per batch (16 KB)
constexpr int kGramFold = 4;       // batches summed in FP32 before the FP64 fold
constexpr int kSolveThreads = 1024;

// Per-block partial Gram matrix U^T U of rows [b * chunk, (b + 1) * chunk);
// with SCALE, each row is first multiplied column-wise by inv and written
// back, and the Gram matrix is that of the scaled rows.
// The R x R result (R padded to R4, a multiple of 4) is cut into 4 x 4 tiles,
// one per thread; THREADS / tiles row groups share a staged batch (group g
// takes rows g, g + groups, ...), so each row costs a thread two 16-byte
// shared loads for 16 FMAs.  FP32 within a batch, FP64 across batches and
// groups (at most 4 x 4096 / R4 / groups rows per FP32 sum).  The next batch
// is loaded into registers while this one is used.
template <int THREADS, bool SCALE>
__global__ void __launch_bounds__(THREADS) k_gram(float *U, uint64_t I, int R, uint64_t chunk,
                                                  const float *inv, double *part) {
    __shared__ __align__(16) float sU[kGramFloats];
    __shared__ __align__(16) float sinv[PASTA_ALS_MAX_RANK];
    constexpr int kPre = kGramFloats / 4 / THREADS;  // float4 per thread per batch
    const int t = threadIdx.x;
    const int R4 = (R + 3) & ~3;
    const int nt = R4 / 4;
    const int T = nt * nt;
    const int groups = THREADS >= 1024 ? 1 : THREADS / T;  // see the combine below
    const int g = t / T, q = t % T;
    const bool active = g < groups;
    const int r0 = 4 * (q / nt), s0 = 4 * (q % nt);
    const int B = kGramFloats / R4;  // rows per batch
    const bool vec = (R == R4) && ((reinterpret_cast<uintptr_t>(U) & 15u) == 0);
    if (SCALE) {
        for (int c = t; c < R4; c += THREADS) sinv[c] = c < R ? inv[c] : 0.f;
        __syncthreads();
    }

    const uint64_t rbeg = (uint64_t)blockIdx.x * chunk;
    const uint64_t rend = min(I, rbeg + chunk);
    float4 pre[kPre];
    auto load = [&](uint64_t b) {
#pragma unroll
        for (int u = 0; u < kPre; ++u) {
            const int e4 = t + THREADS * u;  // float4 slot of the batch
            const int row = e4 / nt, c = 4 * (e4 % nt);
            const uint64_t i = b + (uint64_t)row;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row < B && i < rend) {
                float *src = U + i * (uint64_t)R + c;
                if (vec) {
                    v = *reinterpret_cast<const float4 *>(src);
                } else {
                    v.x = c < R ? src[0] : 0.f;
                    v.y = c + 1 < R ? src[1] : 0.f;
                    v.z = c + 2 < R ? src[2] : 0.f;
                    v.w = c + 3 < R ? src[3] : 0.f;
                }
                if (SCALE) {  // U(i, c..c+3) *= inv, written back in place
                    v.x *= sinv[c];
                    v.y *= sinv[c + 1];
                    v.z *= sinv[c + 2];
                    v.w *= sinv[c + 3];
                    if (vec) {
                        *reinterpret_cast<float4 *>(src) = v;
                    } else {
                        if (c < R) src[0] = v.x;
                        if (c + 1 < R) src[1] = v.y;
                        if (c + 2 < R) src[2] = v.z;
                        if (c + 3 < R) src[3] = v.w;
                    }
                }
            }
            pre[u] = v;
        }
    };
    double a64[16];
    float a32[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        a64[e] = 0.0;
        a32[e] = 0.f;
    }
    int fold = 0;
    if (rbeg < rend) load(rbeg);
    for (uint64_t b = rbeg; b < rend; b += B) {
#pragma unroll
        for (int u = 0; u < kPre; ++u) reinterpret_cast<float4 *>(sU)[t + THREADS * u] = pre[u];
        __syncthreads();
        if (b + B < rend) load(b + B);
        if (active) {
            for (int j = g; j < B; j += groups) {
                const float4 x = *reinterpret_cast<const float4 *>(&sU[j * R4 + r0]);
                const float4 y = *reinterpret_cast<const float4 *>(&sU[j * R4 + s0]);
                const float xa[4] = {x.x, x.y, x.z, x.w};
                const float ya[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int k = 0; k < 4; ++k) a32[4 * i + k] = fmaf(xa[i], ya[k], a32[4 * i + k]);
            }
        }
        // GB300's FP64 pipe is narrow: fold into FP64 every kGramFold batches
        if (++fold == kGramFold) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                a64[e] += (double)a32[e];
                a32[e] = 0.f;
            }
            fold = 0;
        }
        __syncthreads();
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) a64[e] += (double)a32[e];
    // combine the row groups in group order (the staging buffer holds the
    // R4 x R4 doubles: groups > 1 only with 256 threads and R4 <= 44)
    const int RR = R * R;
    if (groups > 1) {
        double *acc = reinterpret_cast<double *>(sU);
        for (int gg = 0; gg < groups; ++gg) {
            if (active && g == gg) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int idx = (r0 + i) * R4 + s0 + k;
                        acc[idx] = (gg == 0 ? 0.0 : acc[idx]) + a64[4 * i + k];
                    }
            }
            __syncthreads();
        }
        for (int p = t; p < RR; p += THREADS)
            part[(uint64_t)blockIdx.x * RR + p] = acc[(p / R) * R4 + p % R];
    } else if (active) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (r0 + i < R && s0 + k < R)
                    part[(uint64_t)blockIdx.x * RR + (r0 + i) * R + s0 + k] = a64[4 * i + k];
    }
}

// out[p] = sum over blocks b of part[b * n + p]: block x takes 32 consecutive
// p, its 8 warps stride over the blocks, and the warp sums are added in warp
// order (deterministic).
__global__ void __launch_bounds__(256) k_sum_parts(const double *part, int nblk, int n, double *out) {
    __shared__ double ws[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (p < n)
        for (int b = warp; b < nblk; b += 8) s += part[(uint64_t)b * n + p];
    ws[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && p < n) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += ws[w][lane];
        out[p] = tot;
    }
}

// W = V^{-1} (computed in FP64, stored FP32) with V = prod_{k != n} G_k
// (element-wise).  In-place
// Gauss-Jordan: for each k the pivot row is scaled by the reciprocal pivot and
// every other row loses its multiple of it.  A pivot that is not positive
// relative to its original diagonal marks V singular: status = n + 1.
__global__ void __launch_bounds__(kSolveThreads) k_als_solve(const double *grams, int N, int n,
                                                             int R, float *W, int *status) {
    extern __shared__ double sA[];  // R * R, R column factors, R diagonals, 1/pivot
    const int RR = R * R;
    double *f = sA + RR;
    double *d0 = f + R;
    double *sip = d0 + R;
    const int t = threadIdx.x;
    for (int p = t; p < RR; p += kSolveThreads) {
        double v = 1.0;
        for (int k = 0; k < N; ++k)
            if (k != n) v *= grams[(uint64_t)k * RR + p];
        sA[p] = v;
    }
    __syncthreads();
    for (int i = t; i < R; i += kSolveThreads) d0[i] = sA[i * R + i];
    // thread t eliminates column jc of rows ic, ic + rpp, ... (rpp = rows per pass)
    const int rpp = kSolveThreads / R;
    const int jc = t % R, ic = t / R;
    for (int k = 0; k < R; ++k) {
        for (int i = t; i < R; i += kSolveThreads) f[i] = sA[i * R + k];
        if (t == 0) *sip = 1.0 / sA[k * R + k];
        __syncthreads();
        const double piv = f[k];
        if (!(piv > 1e-14 * d0[k]) || !isfinite(piv)) {  // the same for every thread
            if (t == 0) atomicCAS(status, 0, n + 1);
            for (int p = t; p < RR; p += kSolveThreads) W[p] = 0.f;
            return;
        }
        const double ip = *sip;
        for (int j = t; j < R; j += kSolveThreads) sA[k * R + j] = (j == k ? 1.0 : sA[k * R + j]) * ip;
        __syncthreads();
        if (ic < rpp) {
            const double akj = sA[k * R + jc];
            for (int i = ic; i < R; i += rpp)
                if (i != k) sA[i * R + jc] = (jc == k ? 0.0 : sA[i * R + jc]) - f[i] * akj;
        }
        __syncthreads();
    }
    for (int p = t; p < RR; p += kSolveThreads) W[p] = (float)sA[p];
}

// U(i, :) = M(i, :) W for four rows per warp iteration; lane owns columns
// lane + 32 c (c < CPL); W (R x R) sits in shared memory.  Also per-block
// column statistics of the rows written: part[b][r] = sum_i U(i, r)^2 and
// part[b][R + r] = sum_i M(i, r) U(i, r) (FP32 per 64 rows, FP64 beyond,
// warps added in order).
template <int CPL>
__global__ void __launch_bounds__(256) k_als_rows(const float *M, uint64_t I, int R, const float *W,
                                                  float *U, double *part) {
    extern __shared__ float sW[];  // R * R
    __shared__ double wst[8][2 * PASTA_ALS_MAX_RANK];
    for (int p = threadIdx.x; p < R * R; p += blockDim.x) sW[p] = W[p];
    __syncthreads();
    constexpr int ROWS = 4;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float sq32[CPL], cr32[CPL];
    double sq64[CPL], cr64[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        sq32[c] = cr32[c] = 0.f;
        sq64[c] = cr64[c] = 0.0;
    }
    int fold = 0;
    const uint64_t step = (uint64_t)gridDim.x * (blockDim.x >> 5) * ROWS;
    float nxt[ROWS][CPL];  // the next iteration's rows, loaded during this one
    auto load = [&](uint64_t i0) {
#pragma unroll
        for (int q = 0; q < ROWS; ++q)
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int col = lane + 32 * c;
                nxt[q][c] = (i0 + q < I && col < R) ? M[(i0 + q) * R + col] : 0.f;
            }
    };
    const uint64_t first = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + warp) * ROWS;
    if (first < I) load(first);
    for (uint64_t i0 = first; i0 < I; i0 += step) {
        float mv[ROWS][CPL], acc[ROWS][CPL];
#pragma unroll
        for (int q = 0; q < ROWS; ++q)
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                mv[q][c] = nxt[q][c];
                acc[q][c] = 0.f;
            }
        if (i0 + step < I) load(i0 + step);
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
                // rows past I and columns past R hold zeros in mv and acc
                sq32[c] = fmaf(acc[q][c], acc[q][c], sq32[c]);
                cr32[c] = fmaf(mv[q][c], acc[q][c], cr32[c]);
            }
        if (++fold == 16) {
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                sq64[c] += (double)sq32[c];
                cr64[c] += (double)cr32[c];
                sq32[c] = cr32[c] = 0.f;
            }
            fold = 0;
        }
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int col = lane + 32 * c;
        if (col < R) {
            wst[warp][col] = sq64[c] + (double)sq32[c];
            wst[warp][R + col] = cr64[c] + (double)cr32[c];
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < 2 * R; p += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += wst[w][p];
        part[(uint64_t)blockIdx.x * 2 * R + p] = t;
    }
}

// From the column statistics st = [sum U_raw^2 (R), sum M .* U_raw (R)]:
// lam_r = sqrt(st_r), inv_r = 1 / lam_r (0 for a zero column), and
// inner_r = sum_i M(i, r) U_n(i, r) = st_{R+r} inv_r for the normalised U_n.
__global__ void k_als_lambda(const double *st, int R, double *lam, float *inv, double *inner) {
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const double l = sqrt(max(st[r], 0.0));
        const double iv = l > 0.0 ? 1.0 / l : 0.0;
        lam[r] = l;
        inv[r] = (float)iv;
        inner[r] = st[R + r] * iv;
    }
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

// G = U^T U of an I x R FP32 matrix (FP64), through per-block partials in
// `part` (room for nblk_max * R * R doubles).  With inv, U(:, r) *= inv_r in
// place first and G is the Gram matrix of the result.
void gram(float *U, uint64_t I, int R, int nblk_max, double *part, double *G, cudaStream_t s,
          const float *inv = nullptr) {
    const int R4 = (R + 3) & ~3;
    const uint64_t B = kGramFloats / R4;
    const uint64_t batches = (I + B - 1) / B;
    const int nblk = (int)std::max<uint64_t>(1, std::min<uint64_t>(batches, (uint64_t)nblk_max));
    const uint64_t chunk = ((batches + nblk - 1) / nblk) * B;
    if (R4 <= 64) {
        if (inv)
            k_gram<256, true><<<nblk, 256, 0, s>>>(U, I, R, chunk, inv, part);
        else
            k_gram<256, false><<<nblk, 256, 0, s>>>(U, I, R, chunk, nullptr, part);
    } else {
        if (inv)
            k_gram<1024, true><<<nblk, 1024, 0, s>>>(U, I, R, chunk, inv, part);
        else
            k_gram<1024, false><<<nblk, 1024, 0, s>>>(U, I, R, chunk, nullptr, part);
    }
    const int RR = R * R;
    k_sum_parts<<<(RR + 31) / 32, 256, 0, s>>>(part, nblk, RR, G);
}

// Blocks of k_als_rows for I rows (also the number of column-statistics
// partials it writes).
int rows_blocks(uint64_t I, int num_sms) {
    const uint64_t need = (I + 31) / 32;  // blocks of 8 warps x 4 rows
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)num_sms * 4));
}

pasta_status rows(const float *M, uint64_t I, int R, const float *W, float *U, double *part,
                  int num_sms, cudaStream_t s) {
    const size_t smem = (size_t)R * R * sizeof(float);
    const int blocks = rows_blocks(I, num_sms);
    if (R <= 32) {
        PASTA_CUDA(cudaFuncSetAttribute(k_als_rows<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_als_rows<1><<<blocks, 256, smem, s>>>(M, I, R, W, U, part);
    } else if (R <= 64) {
        PASTA_CUDA(cudaFuncSetAttribute(k_als_rows<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_als_rows<2><<<blocks, 256, smem, s>>>(M, I, R, W, U, part);
    } else {
        PASTA_CUDA(cudaFuncSetAttribute(k_als_rows<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_als_rows<4><<<blocks, 256, smem, s>>>(M, I, R, W, U, part);
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
    const int nblk = 2 * X->num_sms;  // k_gram grid cap

    // the handle's scratch, cut into 256-byte aligned pieces
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t oM = take(imax * (size_t)R * sizeof(float));
    const size_t oG = take((size_t)N * RR * sizeof(double));
    const size_t oW = take((size_t)RR * sizeof(float));
    const size_t oSt = take((size_t)2 * R * sizeof(double));
    const size_t oInv = take((size_t)R * sizeof(float));
    const size_t oInner = take((size_t)R * sizeof(double));
    const size_t oPart = take(std::max((size_t)nblk * RR, (size_t)rows_blocks(imax, X->num_sms) * 2 * R) *
                              sizeof(double));
    const size_t oStatus = take(sizeof(int));
    char *base = nullptr;
    {
        void *p = nullptr;
        const pasta_status hs = handle_scratch(X, off, &p);
        if (hs != PASTA_OK) return hs;
        base = static_cast<char *>(p);
    }
    float *M = reinterpret_cast<float *>(base + oM);
    double *G = reinterpret_cast<double *>(base + oG);
    float *W = reinterpret_cast<float *>(base + oW);
    double *st2 = reinterpret_cast<double *>(base + oSt);
    float *inv = reinterpret_cast<float *>(base + oInv);
    double *inner = reinterpret_cast<double *>(base + oInner);
    double *part = reinterpret_cast<double *>(base + oPart);
    int *status = reinterpret_cast<int *>(base + oStatus);

    auto fail = [&](pasta_status e) { return e; };
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemsetAsync(status)"));

    // ||X||^2 once per handle (the values never change after create)
    if (!X->als_normsq) {
        e = dev_malloc(reinterpret_cast<void **>(&X->als_normsq), sizeof(double), s);
        if (e != cudaSuccess) {
            X->als_normsq = nullptr;
            return fail(cuda_fail(e, "allocation of normsq"));
        }
        const int b = (int)std::max<uint64_t>(1, std::min<uint64_t>((X->nnz + 255) / 256, (uint64_t)nblk));
        k_sumsq<<<b, 256, 0, s>>>(X->orig.val, X->nnz, part);
        k_sum_parts<<<1, 256, 0, s>>>(part, b, 1, X->als_normsq);
    }

    for (int k = 0; k < N; ++k) gram(U[k], X->dims[k], R, nblk, part, G + (size_t)k * RR, s);

    const size_t solve_smem = ((size_t)RR + 2 * R + 1) * sizeof(double);
    e = cudaFuncSetAttribute(k_als_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)solve_smem);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaFuncSetAttribute(k_als_solve)"));
    for (int n = 0; n < N; ++n) {
        const uint64_t I = X->dims[n];
        pasta_status st = launch_mttkrp(X, X->sorted[n], reinterpret_cast<const void *const *>(U),
                                        PASTA_F32, n, R, M, s);
        if (st != PASTA_OK) return fail(st);
        k_als_solve<<<1, kSolveThreads, solve_smem, s>>>(G, N, n, R, W, status);
        st = rows(M, I, R, W, U[n], part, X->num_sms, s);  // U_n = M W and its column statistics
        if (st != PASTA_OK) return fail(st);
        k_sum_parts<<<(2 * R + 31) / 32, 256, 0, s>>>(part, rows_blocks(I, X->num_sms), 2 * R, st2);
        k_als_lambda<<<1, 128, 0, s>>>(st2, R, lambda, inv, inner);
        gram(U[n], I, R, nblk, part, G + (size_t)n * RR, s, inv);  // normalise in place + Gram
    }
    if (fit) k_als_fit<<<1, 256, 0, s>>>(G, N, R, lambda, inner, X->als_normsq, fit);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(cuda_fail(e, "CP-ALS kernels"));

    int h_status = 0;
    e = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "CP-ALS status read");
    if (h_status != 0) {
        set_error("CP-ALS: V of mode %d is singular (non-positive pivot)", h_status - 1);
        return PASTA_ERR_SINGULAR;
    }
    return PASTA_OK;
}

}  // namespace pasta
