// Copies between host and device memory shared by the handle code (api.cu)
// and the pipelined create-and-sort (sort.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pasta.h"

namespace pasta {

// Copy of `bytes` from src to dst on stream s.  Where one side is pinned host
// memory (16-byte aligned, whole 32-bit words) a kernel moves the data with
// the SMs; otherwise cudaMemcpyAsync.  Defined in api.cu.
cudaError_t copy_bytes(void *dst, const void *src, uint64_t bytes, int num_sms, cudaStream_t s);

// Device-side address of p if it is pinned host memory the device can reach,
// else NULL.  Defined in api.cu.
const void *pinned_device_address(const void *p);

// True when the mode's sort key holds every index whole (sort.cu).
bool sort_key_holds_all(const ::pasta_coo_s *X, int mode);

// The creation-order copy filled from pinned host arrays and the mode's sorted
// copy built, overlapped: the entries are cut into K parts (4 from 2^24
// entries on, else 2); each part is sorted as soon as it has been copied
// while the later parts are still being copied (on a high-priority stream of
// their own), and the sorted parts are merged into the sorted copy (stable,
// earlier parts first on ties: the same order as one sort).  Needs a key that
// holds every index and at least 1024 entries per part; the sorted copy must
// be allocated.  Defined in sort.cu.
pasta_status copy_in_and_sort(::pasta_coo_s *X, int mode, const void *const *h_idx, const void *h_val,
                              cudaStream_t s);

}  // namespace pasta
