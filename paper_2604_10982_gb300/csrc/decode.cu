// a6: query decode (placeholder until the tensor-core kernel lands).
#include "common.cuh"

namespace psi {

cudaError_t launch_decode(const void *, int64_t, int, const void *, int, const float *, int32_t *, void *, DevStatus *,
                          cudaStream_t, const char **)
{
    return cudaErrorNotSupported;
}

} // namespace psi
