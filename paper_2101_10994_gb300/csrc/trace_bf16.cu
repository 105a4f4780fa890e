// BF16 decode on the fifth-generation tensor cores (tcgen05): filled in by
// the tensor-core sphere tracer.
#include "nglod_internal.cuh"
#include "trace_common.cuh"

namespace nglod {

int launch_trace_bf16(const nglod_svo*, const nglod_decoder*, const Tables&, const TraceArgs&, bool,
                      cudaStream_t) {
    return fail(NGLOD_ERR_NOT_SUPPORTED, "sphere_trace: BF16 decode not built");
}

int launch_query_bf16(const nglod_svo*, const Tables&, const nglod_decoder*, const float*, long long, int,
                      float*, int8_t*, bool, cudaStream_t) {
    return fail(NGLOD_ERR_NOT_SUPPORTED, "sdf_query: BF16 decode not built");
}

}  // namespace nglod
