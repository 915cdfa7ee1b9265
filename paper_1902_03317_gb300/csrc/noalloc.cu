// pasta_cp_loss_fwd_noalloc: the sparse CP loss forward for callers that
// cannot allocate device memory.
//
// Some callers must not call cudaMalloc at the point they need the loss: code
// running inside a stream capture owned by another framework, a real-time
// or callback context, or a process whose device memory is entirely owned by
// a different allocator.  The handle path cannot serve them:
// pasta_coo_create copies the tensor into library memory and keeps the
// per-handle scratch array that pasta_cp_loss_fwd uses.  This entry point
// takes the caller's own device arrays and keeps its scratch (the FP64
// per-block partial sums of the loss) in a fixed file-scope device array
// instead, so it allocates nothing.
//
// The scratch array is part of the library image: every GPU that loads the
// library holds it (kNoallocPartials doubles, 32 KB) until the process exits.
// Calls share it, so calls whose work overlaps on the GPU race; successive
// calls on one stream are fine.  Nothing in it needs clearing: every block of
// a launch writes its own partial and the final sum reads only those.

#include "pasta_internal.cuh"

namespace pasta {
namespace {

constexpr int kNoallocPartials = PASTA_NOALLOC_MAX_PARTIALS;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoallocPartials];

// Device address of g_noalloc_partials on the current device, looked up on
// every call (in host code the symbol's name is only a host-side stand-in and
// must not be passed to a kernel).  Not cached: after cudaDeviceReset the
// module is loaded again and the array may sit elsewhere.  The lookup itself
// allocates nothing once the module is loaded (the first call on a device,
// and the first after a reset, may load it).
pasta_status partials_address(int device, double **out) {
    if (device < 0 || device >= kMaxDevices) {
        set_error("device ordinal %d beyond the %d devices this entry point supports", device,
                  kMaxDevices);
        return PASTA_ERR_UNSUPPORTED;
    }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_partials)");
    *out = static_cast<double *>(p);
    return PASTA_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace
}  // namespace pasta

using namespace pasta;

extern "C" pasta_status pasta_cp_loss_fwd_noalloc(int order, const uint64_t *dims, uint64_t nnz,
                                                  const uint32_t *const *d_idx,
                                                  const float *d_val, const void *const *d_U,
                                                  pasta_dtype u_dtype, int R, double *d_loss,
                                                  void *d_resid, void *stream) {
    if (order < 2 || order > PASTA_MAX_ORDER || !dims) {
        set_error("order must be in [2, %d] and dims non-NULL", PASTA_MAX_ORDER);
        return PASTA_ERR_INVALID_ARG;
    }
    for (int k = 0; k < order; ++k)
        if (dims[k] < 1 || dims[k] > 0xFFFFFFFFull) {
            set_error("dims[%d] out of [1, 2^32)", k);
            return PASTA_ERR_INVALID_ARG;
        }
    if (nnz >= 0xFFFF0000ull) {
        set_error("nnz must be < 2^32 - 2^16");
        return PASTA_ERR_INVALID_ARG;
    }
    if (u_dtype < PASTA_F32 || u_dtype > PASTA_F64 || R < 1 || R > PASTA_MAX_RANK || !d_U ||
        !d_loss) {
        set_error("bad dtype, R out of [1, %d], or NULL d_U/d_loss", PASTA_MAX_RANK);
        return PASTA_ERR_INVALID_ARG;
    }
    for (int k = 0; k < order; ++k)
        if (!d_U[k]) {
            set_error("d_U[%d] is NULL", k);
            return PASTA_ERR_INVALID_ARG;
        }
    if (nnz > 0) {
        if (!d_idx || !d_val) {
            set_error("d_idx/d_val is NULL");
            return PASTA_ERR_INVALID_ARG;
        }
        // The kernel reads each array 16 bytes (4 entries) at a time.
        for (int k = 0; k < order; ++k)
            if (!d_idx[k] || !aligned16(d_idx[k])) {
                set_error("d_idx[%d] is NULL or not 16-byte aligned", k);
                return PASTA_ERR_ALIGNMENT;
            }
        if (!aligned16(d_val)) {
            set_error("d_val is not 16-byte aligned");
            return PASTA_ERR_ALIGNMENT;
        }
    }
    int device = 0, num_sms = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    double *partials = nullptr;
    pasta_status st = partials_address(device, &partials);
    if (st != PASTA_OK) return st;

    CooView v{};
    for (int k = 0; k < order; ++k) v.idx[k] = d_idx ? d_idx[k] : nullptr;
    v.val = d_val;
    v.nnz = nnz;
    v.order = order;
    // The launch never uses more blocks than the scratch holds (the grid is
    // capped at kNoallocPartials; the kernel's grid-stride loop covers any nnz).
    return launch_cp_loss_fwd(v, 0, num_sms, d_U, u_dtype, R, d_loss, d_resid, partials,
                              kNoallocPartials, static_cast<cudaStream_t>(stream));
}
