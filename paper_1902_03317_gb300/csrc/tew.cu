// Element-wise operations on the stored values: TEW-eq (Sec. 3.1,
// Algorithm 1: two tensors with the same coordinates) and TS (Sec. 3.2,
// Algorithm 3: a tensor and a scalar).  Both are pure streams over the
// creation-order copy, so they are HBM-bound: 16-byte vector loads and
// stores over the padded arrays (the padding is zero and allocated), a grid
// of a few blocks per SM, several vectors in flight per thread.
#include <algorithm>

#include "pasta_internal.cuh"

namespace pasta {
namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;  // float4 per thread per iteration

__device__ __forceinline__ float apply(int op, float a, float b) {
    switch (op) {
        case PASTA_OP_ADD: return __fadd_rn(a, b);
        case PASTA_OP_SUB: return __fsub_rn(a, b);
        case PASTA_OP_MUL: return __fmul_rn(a, b);
        default: return __fdiv_rn(a, b);
    }
}

__device__ __forceinline__ float4 apply4(int op, float4 a, float4 b) {
    return make_float4(apply(op, a.x, b.x), apply(op, a.y, b.y), apply(op, a.z, b.z),
                       apply(op, a.w, b.w));
}

// z = x op y (y == nullptr: z = x op s), n4 float4 vectors.
template <bool SCALAR>
__global__ void __launch_bounds__(kThreads) k_elementwise(const float4 *x, const float4 *y, float s,
                                                           float4 *z, uint64_t n4, int op) {
    const uint64_t step = (uint64_t)gridDim.x * kThreads;
    for (uint64_t i0 = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i0 < n4; i0 += step * kUnroll) {
        float4 a[kUnroll], b[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint64_t i = i0 + (uint64_t)u * step;
            a[u] = i < n4 ? x[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            b[u] = SCALAR ? make_float4(s, s, s, s) : (i < n4 ? y[i] : make_float4(1.f, 1.f, 1.f, 1.f));
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint64_t i = i0 + (uint64_t)u * step;
            if (i < n4) z[i] = apply4(op, a[u], b[u]);
        }
    }
}

// *diff |= 1 if any of the n4 uint4 words of a and b differ.
__global__ void __launch_bounds__(kThreads) k_same_words(const uint4 *a, const uint4 *b, uint64_t n4,
                                                          unsigned *diff) {
    const uint64_t step = (uint64_t)gridDim.x * kThreads;
    bool d = false;
    for (uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i < n4; i += step) {
        const uint4 p = a[i], q = b[i];
        d |= (p.x != q.x) | (p.y != q.y) | (p.z != q.z) | (p.w != q.w);
    }
    if (__any_sync(0xFFFFFFFFu, d) && (threadIdx.x & 31) == 0) atomicOr(diff, 1u);
}

int grid_for(uint64_t n4, int num_sms) {
    const uint64_t want = (n4 + kThreads - 1) / kThreads;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)num_sms * 8));
}

}  // namespace

pasta_status same_coordinates(const pasta_coo_s *X, const pasta_coo_s *Y, cudaStream_t s, bool *same) {
    unsigned *d_diff = nullptr;
    PASTA_CUDA(cudaMallocAsync((void **)&d_diff, sizeof(unsigned), s));
    cudaError_t e = cudaMemsetAsync(d_diff, 0, sizeof(unsigned), s);
    // both copies are padded to nnz_pad (a multiple of 4) with zeros
    const uint64_t n4 = X->nnz_pad / 4;
    for (int k = 0; k < X->order && e == cudaSuccess; ++k) {
        k_same_words<<<grid_for(n4, X->num_sms), kThreads, 0, s>>>(
            reinterpret_cast<const uint4 *>(X->orig.idx[k]), reinterpret_cast<const uint4 *>(Y->orig.idx[k]),
            n4, d_diff);
        e = cudaGetLastError();
    }
    unsigned h = 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_diff, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d_diff, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "coordinate comparison");
    *same = (h == 0);
    return PASTA_OK;
}

pasta_status launch_elementwise(const float *x, const float *y, double s, float *z, uint64_t n_pad,
                                int op, int num_sms, cudaStream_t st) {
    const uint64_t n4 = n_pad / 4;
    const int grid = grid_for((n4 + kUnroll - 1) / kUnroll, num_sms);
    if (y)
        k_elementwise<false><<<grid, kThreads, 0, st>>>(reinterpret_cast<const float4 *>(x),
                                                        reinterpret_cast<const float4 *>(y), 0.f,
                                                        reinterpret_cast<float4 *>(z), n4, op);
    else
        k_elementwise<true><<<grid, kThreads, 0, st>>>(reinterpret_cast<const float4 *>(x), nullptr,
                                                       (float)s, reinterpret_cast<float4 *>(z), n4, op);
    PASTA_CUDA(cudaGetLastError());
    return PASTA_OK;
}

}  // namespace pasta
