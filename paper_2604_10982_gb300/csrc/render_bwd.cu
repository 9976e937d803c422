// a5: adjoint of the per-tile compositing (placeholder until the kernel lands).
#include "raster.cuh"

namespace psi {

size_t render_bwd_workspace_bytes(int64_t n_records)
{
    return align_up(static_cast<size_t>(std::max<int64_t>(n_records, 1)) * 32, 256);
}

cudaError_t launch_render_bwd(const FrameParams &, const psi_surfels &, const FeatView &, const float4 *,
                              const uint32_t *, const uint32_t *, const float *, const float *, const float *,
                              const psi_grads &, void *, DevStatus *, cudaStream_t)
{
    return cudaErrorNotSupported;
}

} // namespace psi
