/*
 * pasta_cpu_parallel.c -- multicore CPU MTTKRP, the timed CPU baseline.
 *
 * BENCHMARK INFRASTRUCTURE, NOT PART OF THE PRODUCT and not a correctness
 * reference (the FP64 oracle in pasta_oracle.c is).  Only tests/ and the CPU
 * legs of bench.py load it.  It shares no code with the CUDA library.
 *
 * What it computes: the mode-n MTTKRP of Eq. (mttkrp-init) / Algorithm 6,
 *     M(i, r) = sum_{m : i_n(m) = i} val(m) * prod_{k != n} U_k(i_k(m), r),
 * in FP32 (32-bit values and factors as in Table 2's caption), on all host
 * cores, with the race on M resolved the way Sec. 5.3 describes and Sec. 7
 * measures: privatization.  The stored entries are split into one contiguous
 * range per thread (the parallel loop over nonzeros); each thread adds its
 * entries into its own zero-initialised copy of M; a second parallel loop,
 * over the rows of M, sums the private copies into M.  The private copies
 * cost threads x dims[mode] x R floats, the buffer size Sec. 7 blames for the
 * slow darpa case.
 *
 * Built with gcc -O3 -fopenmp (a tuned baseline, unlike the oracle).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

/* Number of threads an OpenMP parallel region would use. */
int cpu_threads(void) { return omp_get_max_threads(); }

/*
 * order, dims[order], nnz; idx: order pointers to uint32 indices; val: FP32
 * values; U: order pointers to row-major dims[k] x R FP32 factors (U[mode]
 * unused); M: dims[mode] x R FP32 output (overwritten); threads <= 0 uses
 * every available thread.  Returns 0, or -1 on bad arguments / allocation
 * failure.
 */
int cpu_mttkrp_privatized(int order, const uint64_t *dims, uint64_t nnz, const uint32_t *const *idx,
                          const float *val, const float *const *U, int mode, int R, float *M,
                          int threads) {
    if (order < 2 || order > 8 || mode < 0 || mode >= order || R < 1 || R > 256 || !dims || !M) return -1;
    if (threads <= 0) threads = omp_get_max_threads();
    const uint64_t I = dims[mode];
    const size_t rowsz = (size_t)I * (size_t)R;
    float *priv = (float *)malloc(sizeof(float) * rowsz * (size_t)threads);
    if (!priv) return -1;
    int other[8];
    int no = 0;
    for (int k = 0; k < order; ++k)
        if (k != mode) other[no++] = k;

#pragma omp parallel num_threads(threads)
    {
        const int t = omp_get_thread_num();
        const int nt = omp_get_num_threads();
        float *mine = priv + (size_t)t * rowsz;
        memset(mine, 0, sizeof(float) * rowsz);
        const uint64_t lo = nnz * (uint64_t)t / (uint64_t)nt;
        const uint64_t hi = nnz * (uint64_t)(t + 1) / (uint64_t)nt;
        float prod[256];
        for (uint64_t m = lo; m < hi; ++m) {
            const float v = val[m];
            const float *u0 = U[other[0]] + (size_t)idx[other[0]][m] * (size_t)R;
            for (int r = 0; r < R; ++r) prod[r] = v * u0[r];
            for (int j = 1; j < no; ++j) {
                const float *uj = U[other[j]] + (size_t)idx[other[j]][m] * (size_t)R;
                for (int r = 0; r < R; ++r) prod[r] *= uj[r];
            }
            float *out = mine + (size_t)idx[mode][m] * (size_t)R;
            for (int r = 0; r < R; ++r) out[r] += prod[r];
        }
#pragma omp barrier
        /* global reduction of the private copies, rows split over threads */
#pragma omp for schedule(static)
        for (uint64_t i = 0; i < I; ++i) {
            float *dst = M + i * (size_t)R;
            const float *src0 = priv + i * (size_t)R;
            for (int r = 0; r < R; ++r) dst[r] = src0[r];
            for (int s = 1; s < nt; ++s) {
                const float *src = priv + (size_t)s * rowsz + i * (size_t)R;
                for (int r = 0; r < R; ++r) dst[r] += src[r];
            }
        }
    }
    free(priv);
    return 0;
}
