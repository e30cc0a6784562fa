// Mixed-precision tracer (FP32 stages in bulk): not built yet.
#include <cuda_runtime.h>

#include "odx_internal.h"

namespace odx {

cudaError_t launch_trace_mixed(const TraceArgs &, int32_t, const odx_launch &, int32_t,
                               cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace odx
