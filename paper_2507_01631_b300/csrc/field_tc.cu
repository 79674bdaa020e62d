// Mixed-precision field path (FP16 tables, BF16 MLP on the tensor cores).
#include "kernels.cuh"

namespace snk {

cudaError_t launch_field_tc(const FieldArgs &, int, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace snk
