// lloyd_tc.cu -- PQ Lloyd pass on the tcgen05 tensor cores (BF16 operands,
// FP32 accumulation in tensor memory).  Not built yet: reports unsupported.
#include "common.cuh"
#include "internal.h"

namespace pqgb {

bool tc_pass_supported(int, int, int) { return false; }

int launch_pq_pass_tc(PqPass &, cudaStream_t) { return fail(PQ_ENOTSUP, "BF16 tensor-core pass not available"); }

}  // namespace pqgb
