/*
 * FP64 CPU oracle for COO MTTKRP and the sparse CP least-squares loss.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only tests/, the smoke()
 * entry of __graft_entry__.py and the cpu_baseline leg of bench.py may build,
 * load or call this file.  It shares no code, header or constant with the
 * CUDA library: it is a plain, slow, single-threaded restatement of the
 * definitions, written so that a reader can check it against the paper by eye.
 *
 * Conventions (readings of the paper):
 *   - COO storage (Sec. 5.1): one index array per mode ("inds") and one value
 *     array ("val"), both of length nnz; indices are 0-based (the Sec. 5.1
 *     example names entries (1,0,0) and (1,0,2) of a 4x4x3 tensor).
 *   - Factor matrices are row-major I_k x R, element (i, r) at i*R + r
 *     (footnote to Eq. (ttm) in Sec. 3.4; Algorithm 6 indexes A(i*R + r)).
 *   - The output is zero-filled and then accumulated into (Sec. 5.2.6 has
 *     the output set up beforehand, the kernel only adding to it).
 *   - Duplicate coordinates are separate stored entries; MTTKRP is linear,
 *     so they add.
 *
 * All arithmetic is in double precision, in storage order, with no blocking,
 * fusion or reordering.
 */
#include <stdint.h>
#include <string.h>

/*
 * Mode-n MTTKRP, Eq. (mttkrp-init):  M = X_(n) (U_N o ... o U_{n+1} o U_{n-1} o ... o U_1).
 * Written element-wise as in Algorithm 6 (the third-order listing), taken to
 * order N: for every stored entry m and every column r,
 *     M(i_n(m), r) += val(m) * prod_{k != n} U_k(i_k(m), r).
 *
 *   order  number of modes N (>= 1)
 *   dims   N mode sizes
 *   nnz    number of stored entries
 *   idx    N pointers, idx[k][m] = index of entry m in mode k
 *   val    nnz values
 *   U      N pointers to row-major dims[k] x R factors; U[mode] is not read
 *   mode   0-based output mode n
 *   R      rank (columns)
 *   M      output, dims[mode] x R row-major, overwritten
 * Returns 0, or -1 on an argument error (nothing written).
 */
int oracle_mttkrp(int order, const uint64_t *dims, uint64_t nnz,
                  const uint32_t *const *idx, const double *val,
                  const double *const *U, int mode, int R, double *M)
{
    if (order < 1 || mode < 0 || mode >= order || R < 1)
        return -1;
    memset(M, 0, (size_t)dims[mode] * (size_t)R * sizeof(double));
    for (uint64_t m = 0; m < nnz; ++m) {
        double *out_row = M + (uint64_t)idx[mode][m] * (uint64_t)R;
        for (int r = 0; r < R; ++r) {
            double t = val[m];
            for (int k = 0; k < order; ++k) {
                if (k == mode)
                    continue;
                t *= U[k][(uint64_t)idx[k][m] * (uint64_t)R + (uint64_t)r];
            }
            out_row[r] += t;
        }
    }
    return 0;
}

/*
 * CP model value at one stored coordinate (the rank-R CP model of Sec. 2.2,
 * a sum of R rank-one terms without weights):
 *     model(m) = sum_r prod_k U_k(i_k(m), r).
 */
static double cp_model_at(int order, const uint32_t *const *idx, uint64_t m,
                          const double *const *U, int R)
{
    double s = 0.0;
    for (int r = 0; r < R; ++r) {
        double p = 1.0;
        for (int k = 0; k < order; ++k)
            p *= U[k][(uint64_t)idx[k][m] * (uint64_t)R + (uint64_t)r];
        s += p;
    }
    return s;
}

/*
 * CP model values at every stored coordinate, out[m] = model(m) (Sec. 2.2).
 * Also makes the values of the planted-model test workload (the model's
 * values plus noise); the generator that draws the coordinates does not
 * evaluate the model itself.
 */
int oracle_cp_model(int order, uint64_t nnz, const uint32_t *const *idx,
                    const double *const *U, int R, double *out)
{
    if (order < 1 || R < 1)
        return -1;
    for (uint64_t m = 0; m < nnz; ++m)
        out[m] = cp_model_at(order, idx, m, U, R);
    return 0;
}

/*
 * Sparse CP least-squares loss over the stored entries only:
 *     e(m) = val(m) - model(m),   L = 1/2 * sum_m e(m)^2.
 * The paper names gradient-descent CPD (Sec. 2.2) but prints no loss; this is
 * the least-squares objective of that method restricted to the nonzeros.
 *
 *   resid  optional (may be NULL): nnz residuals e(m) in storage order
 *   loss   output scalar
 */
int oracle_cp_loss(int order, const uint64_t *dims, uint64_t nnz,
                   const uint32_t *const *idx, const double *val,
                   const double *const *U, int R, double *resid, double *loss)
{
    (void)dims;
    if (order < 1 || R < 1)
        return -1;
    double acc = 0.0;
    for (uint64_t m = 0; m < nnz; ++m) {
        double e = val[m] - cp_model_at(order, idx, m, U, R);
        if (resid)
            resid[m] = e;
        acc += e * e;
    }
    *loss = 0.5 * acc;
    return 0;
}

/*
 * Gradient of the loss above with respect to every factor, scaled by g
 * (the incoming gradient of the scalar loss).  Differentiating
 * 1/2 * (val - sum_r prod_k U_k)^2 in U_n(i_n(m), r) gives
 *     -e(m) * prod_{k != n} U_k(i_k(m), r),
 * so
 *     G_n(i, r) = -g * sum_{m : i_n(m) = i} e(m) * prod_{k != n} U_k(i_k(m), r),
 * i.e. -g times the mode-n MTTKRP of the residual tensor.  Written here as its
 * own loop, not through oracle_mttkrp.
 *
 *   G  N pointers to row-major dims[k] x R outputs, all overwritten
 */
int oracle_cp_grad(int order, const uint64_t *dims, uint64_t nnz,
                   const uint32_t *const *idx, const double *val,
                   const double *const *U, int R, double g, double *const *G)
{
    if (order < 1 || R < 1)
        return -1;
    for (int n = 0; n < order; ++n)
        memset(G[n], 0, (size_t)dims[n] * (size_t)R * sizeof(double));
    for (uint64_t m = 0; m < nnz; ++m) {
        double e = val[m] - cp_model_at(order, idx, m, U, R);
        for (int n = 0; n < order; ++n) {
            double *g_row = G[n] + (uint64_t)idx[n][m] * (uint64_t)R;
            for (int r = 0; r < R; ++r) {
                double p = 1.0;
                for (int k = 0; k < order; ++k) {
                    if (k == n)
                        continue;
                    p *= U[k][(uint64_t)idx[k][m] * (uint64_t)R + (uint64_t)r];
                }
                g_row[r] -= g * e * p;
            }
        }
    }
    return 0;
}
