// Mixed-precision tracing kernels with 3 transfer slots (see trace_mixed.cuh).
#include "trace_mixed.cuh"

namespace odx {
template cudaError_t launch_mixed_nf<3>(const TraceArgs &, const odx_launch &, dim3, cudaStream_t);
}  // namespace odx
