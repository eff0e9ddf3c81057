// Tensor-core form of the grouped code scan.
#include "rq_scan.cuh"

namespace rq {

bool mma_supported(const rq_index*) { return false; }

rq_status launch_scan_mma(rq_index*, const SearchShape&, Workspace&, cudaStream_t, int) {
  return fail(RQ_ERR_NOT_IMPLEMENTED, "tensor-core scan not built");
}

}  // namespace rq
