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
//                 tiles on or above the diagonal, one per thread, over rows
//                 staged in shared memory; FP32 per batch and over batch
//                 sums, FP64 beyond; per-block partials summed in fixed
//                 order (k_sum_parts)
//   k_als_solve   V^{-1} by in-place Gauss-Jordan in FP64 (V is symmetric
//                 positive definite when the factors have full column rank,
//                 so no pivoting), one block, one barrier per step
//   k_als_rows    U_n = M W plus column statistics: for R <= 32 (R a
//                 multiple of 4) W's columns in registers and M's rows read
//                 back from shared memory as broadcasts (k_als_rows32), else
//                 a warp per four rows with shuffles
//   k_als_lambda  lam, 1 / lam and <M, U_n> per column
//   k_als_fit     ||model||^2 = lam^T (Hadamard of all Grams) lam and the fit
#include <algorithm>
#include <cmath>

#include "pasta_internal.cuh"

namespace pasta {
namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int kGramFloats = 4096;  // floats staged per batch (16 KB)
constexpr int kGramStages = 4;     // batches in the cp.async ring
constexpr int kGramFold = 32;      // batch sums added in FP32 before the FP64 fold
constexpr int kSolveThreads = 256;

// 16-byte asynchronous copy global -> shared (L1 bypassed); src_bytes = 0
// fills the 16 bytes with zeros and reads nothing.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;"); }
template <int K> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K)); }

// Per-block partial Gram matrix U^T U of rows [b * chunk, (b + 1) * chunk);
// with SCALE, each row is first multiplied column-wise by inv and written
// back, and the Gram matrix is that of the scaled rows.
// G is symmetric: its extent (R padded to R4, a multiple of 4) is cut into
// 4 x 4 tiles and only the nt (nt + 1) / 2 tiles on or above the diagonal
// are formed (nt = R4 / 4), one per thread; the partial written out is the
// full R x R matrix, mirrored.  THREADS / tiles row groups share a staged
// batch (group g takes rows g, g + groups, ...), so a row costs a thread two
// 16-byte shared loads for 16 FMAs.  Batches of kGramFloats floats reach
// shared memory through a kGramStages-deep cp.async ring (rows with R a
// multiple of 4 and a 16-byte aligned U; otherwise by plain loads); with
// SCALE each thread scales the slots it copied, in shared memory and in U.
// Sums: FP32 within a batch, FP32 over up to kGramFold batch sums, FP64
// beyond (GB300's FP64 pipe is narrow, so FP64 adds stay rare).
template <int THREADS, bool SCALE>
__global__ void __launch_bounds__(THREADS) k_gram(float *U, uint64_t I, int R, uint64_t chunk,
                                                  const float *inv, double *part) {
    extern __shared__ __align__(16) float ring[];  // kGramStages x kGramFloats
    __shared__ __align__(16) float sinv[PASTA_ALS_MAX_RANK];
    constexpr int kSlots = kGramFloats / 4 / THREADS;  // float4 per thread per batch
    const int t = threadIdx.x;
    const int R4 = (R + 3) & ~3;
    const int nt = R4 / 4;
    const int T = nt * (nt + 1) / 2;
    // groups > 1 needs the T x 16 doubles of the combine below to fit in a stage
    const int groups = THREADS >= 1024 ? 1 : max(1, THREADS / T);
    const int g = t / T, q = t % T;
    const bool active = g < groups;
    int ti = 0, rem = q;  // tile q -> (ti, tj), ti <= tj, row-major over the upper triangle
    while (rem >= nt - ti) {
        rem -= nt - ti;
        ++ti;
    }
    const int tj = ti + rem;
    const int r0 = 4 * ti, s0 = 4 * tj;
    const int B = kGramFloats / R4;  // rows per batch
    const bool vec = (R == R4) && ((reinterpret_cast<uintptr_t>(U) & 15u) == 0);
    if (SCALE) {
        for (int c = t; c < R4; c += THREADS) sinv[c] = c < R ? inv[c] : 0.f;
        __syncthreads();
    }

    const uint64_t rbeg = (uint64_t)blockIdx.x * chunk;
    const uint64_t rend = min(I, rbeg + chunk);
    const int nb = rbeg < rend ? (int)((rend - rbeg + B - 1) / B) : 0;
    // copy batch j into its stage (or commit an empty group past the end)
    auto issue = [&](int j) {
        if (j < nb) {
            float *st = ring + (size_t)(j % kGramStages) * kGramFloats;
            const uint64_t b = rbeg + (uint64_t)j * B;
#pragma unroll
            for (int u = 0; u < kSlots; ++u) {
                const int e4 = t + THREADS * u;  // float4 slot of the batch
                const int row = e4 / nt, c = 4 * (e4 % nt);
                const uint64_t i = b + (uint64_t)row;
                const bool ok = row < B && i < rend;
                if (vec) {
                    cp_async16(st + 4 * e4, ok ? U + i * (uint64_t)R + c : U, ok ? 16 : 0);
                } else {
                    const float *src = U + i * (uint64_t)R + c;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (ok) {
                        v.x = c < R ? src[0] : 0.f;
                        v.y = c + 1 < R ? src[1] : 0.f;
                        v.z = c + 2 < R ? src[2] : 0.f;
                        v.w = c + 3 < R ? src[3] : 0.f;
                    }
                    *reinterpret_cast<float4 *>(st + 4 * e4) = v;
                }
            }
        }
        cp_commit();
    };
    double a64[16];
    float a32[16], b32[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        a64[e] = 0.0;
        a32[e] = b32[e] = 0.f;
    }
    int fold = 0;
#pragma unroll
    for (int j = 0; j < kGramStages - 1; ++j) issue(j);
    for (int j = 0; j < nb; ++j) {
        issue(j + kGramStages - 1);
        cp_wait<kGramStages - 1>();  // this thread's copies of batch j have landed
        float *st = ring + (size_t)(j % kGramStages) * kGramFloats;
        if (SCALE) {  // U(i, c..c+3) *= inv for this thread's slots, in place
            const uint64_t b = rbeg + (uint64_t)j * B;
#pragma unroll
            for (int u = 0; u < kSlots; ++u) {
                const int e4 = t + THREADS * u;
                const int row = e4 / nt, c = 4 * (e4 % nt);
                const uint64_t i = b + (uint64_t)row;
                if (row < B && i < rend) {
                    float4 v = *reinterpret_cast<float4 *>(st + 4 * e4);
                    v.x *= sinv[c];
                    v.y *= sinv[c + 1];
                    v.z *= sinv[c + 2];
                    v.w *= sinv[c + 3];
                    *reinterpret_cast<float4 *>(st + 4 * e4) = v;
                    float *dst = U + i * (uint64_t)R + c;
                    if (vec) {
                        *reinterpret_cast<float4 *>(dst) = v;
                    } else {
                        if (c < R) dst[0] = v.x;
                        if (c + 1 < R) dst[1] = v.y;
                        if (c + 2 < R) dst[2] = v.z;
                        if (c + 3 < R) dst[3] = v.w;
                    }
                }
            }
        }
        __syncthreads();
        if (active) {
            for (int r = g; r < B; r += groups) {
                const float4 x = *reinterpret_cast<const float4 *>(&st[r * R4 + r0]);
                const float4 y = *reinterpret_cast<const float4 *>(&st[r * R4 + s0]);
                const float xa[4] = {x.x, x.y, x.z, x.w};
                const float ya[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int k = 0; k < 4; ++k) a32[4 * i + k] = fmaf(xa[i], ya[k], a32[4 * i + k]);
            }
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            b32[e] += a32[e];
            a32[e] = 0.f;
        }
        if (++fold == kGramFold) {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                a64[e] += (double)b32[e];
                b32[e] = 0.f;
            }
            fold = 0;
        }
        __syncthreads();  // the stage is refilled kGramStages - 1 batches later
    }
    cp_wait<0>();  // only empty groups remain
#pragma unroll
    for (int e = 0; e < 16; ++e) a64[e] += (double)b32[e];
    const int RR = R * R;
    if (groups > 1) {
        // combine the row groups in group order, per tile
        double *acc = reinterpret_cast<double *>(ring);
        for (int gg = 0; gg < groups; ++gg) {
            if (active && g == gg) {
#pragma unroll
                for (int e = 0; e < 16; ++e) acc[q * 16 + e] = (gg == 0 ? 0.0 : acc[q * 16 + e]) + a64[e];
            }
            __syncthreads();
        }
        for (int p = t; p < RR; p += THREADS) {
            int r = p / R, c = p % R;
            if (r / 4 > c / 4) {  // below the diagonal tiles: mirrored
                const int x = r;
                r = c;
                c = x;
            }
            const int a = r / 4, bb = c / 4;
            const int qq = a * nt - a * (a - 1) / 2 + (bb - a);
            part[(uint64_t)blockIdx.x * RR + p] = acc[qq * 16 + 4 * (r % 4) + c % 4];
        }
    } else if (active) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int r = r0 + i, c = s0 + k;
                if (r < R && c < R) {
                    part[(uint64_t)blockIdx.x * RR + (uint64_t)r * R + c] = a64[4 * i + k];
                    if (ti != tj) part[(uint64_t)blockIdx.x * RR + (uint64_t)c * R + r] = a64[4 * i + k];
                }
            }
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

// 1 / x for finite x > 0 in FP64 without a division: x = m 2^e with m in
// [0.5, 1), an FP32 reciprocal of m (about 2^-23 relative error) refined by
// two Newton-Raphson steps r <- r (2 - m r), each of which squares the
// relative error, then scaled by 2^-e.
__device__ __forceinline__ double recip_pos(double x) {
    int e;
    const double m = frexp(x, &e);
    double r = (double)__frcp_rn((float)m);
    r = fma(r, fma(-m, r, 1.0), r);
    r = fma(r, fma(-m, r, 1.0), r);
    return ldexp(r, -e);
}

// W = V^{-1} (computed in FP64, stored FP32) with V = prod_{k != n} G_k
// (element-wise), by in-place Gauss-Jordan: step k scales the pivot row by
// 1 / V_kk and removes its multiples from every other row.  Thread t owns
// column jc = t % R of rows ic, ic + rpp, ... (rpp = threads / R); the
// column and row of step k, read by every thread, come from two ping-pong
// buffers that the owners of step k + 1's column and row fill as they
// update, and the owner of the next pivot stores its reciprocal (or marks it
// bad), so each step needs one barrier.  A pivot that is not positive
// relative to its original diagonal marks V singular: status = n + 1.
__global__ void __launch_bounds__(kSolveThreads) k_als_solve(const double *grams, int N, int n,
                                                             int R, float *W, int *status) {
    extern __shared__ double sA[];  // R * R, column [2][R], row [2][R], thresholds [R], 1/pivot [2]
    const int RR = R * R;
    double *col = sA + RR;
    double *row = col + 2 * R;
    double *thr = row + 2 * R;
    double *sip = thr + R;  // NaN marks a bad pivot
    const int t = threadIdx.x;
    for (int p = t; p < RR; p += kSolveThreads) {
        double v = 1.0;
        for (int k = 0; k < N; ++k)
            if (k != n) v *= grams[(uint64_t)k * RR + p];
        sA[p] = v;
    }
    __syncthreads();
    for (int i = t; i < R; i += kSolveThreads) {
        thr[i] = 1e-14 * sA[i * R + i];
        col[i] = sA[i * R];  // step 0 reads buffer 0
        row[i] = sA[i];
    }
    if (t == 0) {
        const double p0 = sA[0];
        sip[0] = (p0 > 1e-14 * p0 && isfinite(p0)) ? recip_pos(p0) : __longlong_as_double(-1ll);
    }
    __syncthreads();
    const int rpp = kSolveThreads / R;  // R <= PASTA_ALS_MAX_RANK <= kSolveThreads
    const int jc = t % R, ic = t / R;
    const bool worker = ic < rpp;
    for (int k = 0; k < R; ++k) {
        const int b = k & 1, nb = b ^ 1;
        const double ip = sip[b];
        if (isnan(ip)) {  // the same for every thread
            if (t == 0) atomicCAS(status, 0, n + 1);
            for (int p = t; p < RR; p += kSolveThreads) W[p] = 0.f;
            return;
        }
        if (worker) {
            const double rk = (jc == k ? 1.0 : row[b * R + jc]) * ip;  // new pivot-row entry
            for (int i = ic; i < R; i += rpp) {
                const double v = i == k ? rk : (jc == k ? 0.0 : sA[i * R + jc]) - col[b * R + i] * rk;
                sA[i * R + jc] = v;
                if (k + 1 < R) {
                    if (jc == k + 1) col[nb * R + i] = v;
                    if (i == k + 1) row[nb * R + jc] = v;
                    if (i == k + 1 && jc == k + 1)
                        sip[nb] = (v > thr[k + 1] && isfinite(v)) ? recip_pos(v) : __longlong_as_double(-1ll);
                }
            }
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

// The same product for R <= 32 with R a multiple of 4, without shuffles: lane
// c < R owns column c and holds W(:, c) in registers; each warp streams its
// blocks of kRowsW rows of M (kRowsW * R contiguous floats) into a
// kRowsStages-deep cp.async ring in shared memory and reads them back four
// columns at a time as broadcast float4 loads, so a row costs R / 4
// broadcast loads and R FMAs per lane.  Column statistics as in k_als_rows
// (FP32 over 64 rows, FP64 beyond, warps added in order).
constexpr int kRowsW = 8;       // rows per warp iteration
constexpr int kRowsStages = 4;  // blocks of rows in flight per warp
__global__ void __launch_bounds__(256) k_als_rows32(const float *M, uint64_t I, int R, const float *W,
                                                    float *U, double *part) {
    __shared__ __align__(16) float sM[8][kRowsStages][kRowsW * 32];
    __shared__ double wst[8][64];
    constexpr int kSlots = kRowsW * 32 / 4 / 32;  // float4 per lane per block (at R = 32)
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const bool own = lane < R;
    float w[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) w[r] = (own && r < R) ? W[r * R + lane] : 0.f;
    const int nf4 = kRowsW * R / 4;  // float4 per block of kRowsW rows
    const uint64_t step = (uint64_t)gridDim.x * 8 * kRowsW;
    const uint64_t first = ((uint64_t)blockIdx.x * 8 + warp) * kRowsW;
    const int nblk = first < I ? (int)((I - first + step - 1) / step) : 0;  // this warp's row blocks
    auto issue = [&](int j) {
        if (j < nblk) {
            const uint64_t i0 = first + (uint64_t)j * step;
            float *st = sM[warp][j % kRowsStages];
#pragma unroll
            for (int u = 0; u < kSlots; ++u) {
                const int f = lane + 32 * u;
                if (f < nf4) {
                    const bool ok = i0 + (uint64_t)(4 * f / R) < I;
                    cp_async16(st + 4 * f, ok ? M + i0 * (uint64_t)R + 4 * f : M, ok ? 16 : 0);
                }
            }
        }
        cp_commit();
    };
    float sq32 = 0.f, cr32 = 0.f;
    double sq64 = 0.0, cr64 = 0.0;
    int fold = 0;
#pragma unroll
    for (int j = 0; j < kRowsStages - 1; ++j) issue(j);
    for (int j = 0; j < nblk; ++j) {
        issue(j + kRowsStages - 1);
        cp_wait<kRowsStages - 1>();
        __syncwarp();  // every lane's copies of block j have landed
        const uint64_t i0 = first + (uint64_t)j * step;
        const float *st = sM[warp][j % kRowsStages];
        const float4 *st4 = reinterpret_cast<const float4 *>(st);
        float acc[kRowsW];
#pragma unroll
        for (int q = 0; q < kRowsW; ++q) acc[q] = 0.f;
#pragma unroll
        for (int r4 = 0; r4 < 8; ++r4) {
            if (4 * r4 < R) {
#pragma unroll
                for (int q = 0; q < kRowsW; ++q) {
                    const float4 m = st4[q * R / 4 + r4];  // the same address in every lane
                    acc[q] = fmaf(m.x, w[4 * r4], acc[q]);
                    acc[q] = fmaf(m.y, w[4 * r4 + 1], acc[q]);
                    acc[q] = fmaf(m.z, w[4 * r4 + 2], acc[q]);
                    acc[q] = fmaf(m.w, w[4 * r4 + 3], acc[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kRowsW; ++q) {
            if (own && i0 + q < I) {
                const float mq = st[q * R + lane];
                U[(i0 + q) * R + lane] = acc[q];
                sq32 = fmaf(acc[q], acc[q], sq32);
                cr32 = fmaf(mq, acc[q], cr32);
            }
        }
        if (++fold == 64 / kRowsW) {
            sq64 += (double)sq32;
            cr64 += (double)cr32;
            sq32 = cr32 = 0.f;
            fold = 0;
        }
        __syncwarp();  // the stage is refilled kRowsStages - 1 blocks later
    }
    cp_wait<0>();
    if (own) {
        wst[warp][lane] = sq64 + (double)sq32;
        wst[warp][R + lane] = cr64 + (double)cr32;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < 2 * R; p += blockDim.x) {
        double t = 0.0;
        for (int v = 0; v < 8; ++v) t += wst[v][p];
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

// Allows k_gram<THREADS, SCALE> its dynamic shared memory and returns the
// blocks resident per SM in *per_sm.
template <int THREADS, bool SCALE>
cudaError_t gram_config(int *per_sm) {
    const int smem = kGramStages * kGramFloats * (int)sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_gram<THREADS, SCALE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_gram<THREADS, SCALE>, THREADS, smem);
    return e;
}

template <int THREADS, bool SCALE>
pasta_status gram_launch(float *U, uint64_t I, int R, int num_sms, int nblk_max, const float *inv,
                         double *part, int *nblk_out, cudaStream_t s) {
    int per_sm = 0;
    const cudaError_t e = gram_config<THREADS, SCALE>(&per_sm);
    if (e != cudaSuccess) return cuda_fail(e, "k_gram configuration");
    per_sm = std::max(per_sm, 1);
    const int R4 = (R + 3) & ~3;
    const uint64_t B = kGramFloats / R4;
    const uint64_t batches = (I + B - 1) / B;
    const uint64_t cap = std::min<uint64_t>((uint64_t)nblk_max, (uint64_t)num_sms * per_sm);
    const int nblk = (int)std::max<uint64_t>(1, std::min<uint64_t>(batches, cap));
    const uint64_t chunk = ((batches + nblk - 1) / nblk) * B;
    k_gram<THREADS, SCALE><<<nblk, THREADS, kGramStages * kGramFloats * sizeof(float), s>>>(U, I, R, chunk, inv,
                                                                                         part);
    *nblk_out = nblk;
    return PASTA_OK;
}

// G = U^T U of an I x R FP32 matrix (FP64), through per-block partials in
// `part` (room for nblk_max * R * R doubles).  With inv, U(:, r) *= inv_r in
// place first and G is the Gram matrix of the result.
pasta_status gram(float *U, uint64_t I, int R, int num_sms, int nblk_max, double *part, double *G,
                  cudaStream_t s, const float *inv = nullptr) {
    const int R4 = (R + 3) & ~3;
    int nblk = 0;
    pasta_status st;
    if (R4 <= 64)
        st = inv ? gram_launch<256, true>(U, I, R, num_sms, nblk_max, inv, part, &nblk, s)
                 : gram_launch<256, false>(U, I, R, num_sms, nblk_max, nullptr, part, &nblk, s);
    else
        st = inv ? gram_launch<1024, true>(U, I, R, num_sms, nblk_max, inv, part, &nblk, s)
                 : gram_launch<1024, false>(U, I, R, num_sms, nblk_max, nullptr, part, &nblk, s);
    if (st != PASTA_OK) return st;
    const int RR = R * R;
    k_sum_parts<<<(RR + 31) / 32, 256, 0, s>>>(part, nblk, RR, G);
    return PASTA_OK;
}

bool rows32(int R) { return R <= 32 && R % 4 == 0; }

// Allows the row kernel for R its dynamic shared memory (W, R x R floats,
// for k_als_rows) and returns its resident blocks per SM (1 if unknown).
template <typename K>
int rows_config(K kernel, int smem) {
    int per_sm = 0;
    if (smem > 0 && cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem) != cudaSuccess) return 1;
    return std::max(per_sm, 1);
}
int rows_per_sm(int R) {
    const int smem = R * R * (int)sizeof(float);
    if (rows32(R)) return rows_config(k_als_rows32, 0);
    if (R <= 32) return rows_config(k_als_rows<1>, smem);
    if (R <= 64) return rows_config(k_als_rows<2>, smem);
    return rows_config(k_als_rows<4>, smem);
}

// Blocks of k_als_rows / k_als_rows32 for I rows (also the number of
// column-statistics partials they write): one wave of resident blocks at
// most.
int rows_blocks(uint64_t I, int R, int num_sms) {
    const uint64_t per = rows32(R) ? 8 * kRowsW : 32;  // rows per block iteration
    const uint64_t need = (I + per - 1) / per;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)num_sms * rows_per_sm(R)));
}

pasta_status rows(const float *M, uint64_t I, int R, const float *W, float *U, double *part,
                  int num_sms, cudaStream_t s) {
    const size_t smem = (size_t)R * R * sizeof(float);
    const int blocks = rows_blocks(I, R, num_sms);  // also allows the dynamic shared memory
    if (rows32(R))
        k_als_rows32<<<blocks, 256, 0, s>>>(M, I, R, W, U, part);
    else if (R <= 32)
        k_als_rows<1><<<blocks, 256, smem, s>>>(M, I, R, W, U, part);
    else if (R <= 64)
        k_als_rows<2><<<blocks, 256, smem, s>>>(M, I, R, W, U, part);
    else
        k_als_rows<4><<<blocks, 256, smem, s>>>(M, I, R, W, U, part);
    return PASTA_OK;
}

}  // namespace

pasta_status run_cp_als(pasta_coo_s *X, float *const *U, int R, int max_sweeps, double tol, double *lambda,
                        double *fit, double *h_fits, int *h_sweeps, cudaStream_t s) {
    const int N = X->order;
    const int RR = R * R;
    uint64_t imax = 0;
    for (int k = 0; k < N; ++k) imax = std::max(imax, X->dims[k]);
    const int nblk = 2 * X->num_sms;  // k_gram grid cap
    if (h_sweeps) *h_sweeps = 0;

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
    const size_t oPart = take(std::max((size_t)nblk * RR, (size_t)rows_blocks(imax, R, X->num_sms) * 2 * R) *
                              sizeof(double));
    const size_t oStatus = take(sizeof(int));
    const size_t oFit = take(sizeof(double));
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
    double *fitp = fit ? fit : (h_fits ? reinterpret_cast<double *>(base + oFit) : nullptr);

    cudaError_t e;
    // ||X||^2 once per handle (the values never change after create)
    if (!X->als_normsq) {
        e = dev_malloc(reinterpret_cast<void **>(&X->als_normsq), sizeof(double), s);
        if (e != cudaSuccess) {
            X->als_normsq = nullptr;
            return cuda_fail(e, "allocation of normsq");
        }
        const int b = (int)std::max<uint64_t>(1, std::min<uint64_t>((X->nnz + 255) / 256, (uint64_t)nblk));
        k_sumsq<<<b, 256, 0, s>>>(X->orig.val, X->nnz, part);
        k_sum_parts<<<1, 256, 0, s>>>(part, b, 1, X->als_normsq);
    }
    const size_t solve_smem = ((size_t)RR + 5 * R + 2) * sizeof(double);
    e = cudaFuncSetAttribute(k_als_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)solve_smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_als_solve)");

    double prev_fit = 0.0;
    for (int it = 0; it < max_sweeps; ++it) {
        e = cudaMemsetAsync(status, 0, sizeof(int), s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(status)");
        // The Gram matrices of the factors as given; later sweeps keep those
        // formed when each factor was last normalised.
        if (it == 0)
            for (int k = 0; k < N; ++k) {
                const pasta_status gs = gram(U[k], X->dims[k], R, X->num_sms, nblk, part, G + (size_t)k * RR, s);
                if (gs != PASTA_OK) return gs;
            }
        for (int n = 0; n < N; ++n) {
            const uint64_t I = X->dims[n];
            pasta_status st = launch_mttkrp(X, X->sorted[n], reinterpret_cast<const void *const *>(U),
                                            PASTA_F32, n, R, M, s);
            if (st != PASTA_OK) return st;
            k_als_solve<<<1, kSolveThreads, solve_smem, s>>>(G, N, n, R, W, status);
            st = rows(M, I, R, W, U[n], part, X->num_sms, s);  // U_n = M W and its column statistics
            if (st != PASTA_OK) return st;
            k_sum_parts<<<(2 * R + 31) / 32, 256, 0, s>>>(part, rows_blocks(I, R, X->num_sms), 2 * R, st2);
            k_als_lambda<<<1, 128, 0, s>>>(st2, R, lambda, inv, inner);
            st = gram(U[n], I, R, X->num_sms, nblk, part, G + (size_t)n * RR, s, inv);  // normalise + Gram
            if (st != PASTA_OK) return st;
        }
        if (fitp) k_als_fit<<<1, 256, 0, s>>>(G, N, R, lambda, inner, X->als_normsq, fitp);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "CP-ALS kernels");

        int h_status = 0;
        double h_fit = 0.0;
        e = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && h_fits) e = cudaMemcpyAsync(&h_fit, fitp, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "CP-ALS status read");
        if (h_status != 0) {
            set_error("CP-ALS: V of mode %d is singular (non-positive pivot)", h_status - 1);
            return PASTA_ERR_SINGULAR;
        }
        if (h_fits) h_fits[it] = h_fit;
        if (h_sweeps) *h_sweeps = it + 1;
        if (h_fits && tol >= 0.0 && it > 0 && std::fabs(h_fit - prev_fit) < tol) break;
        prev_fit = h_fit;
    }
    return PASTA_OK;
}

}  // namespace pasta
