// Launchers of the per-surfel depth/normal table and its adjoint (geometry.cu).
#pragma once

#include "common.cuh"

namespace psi {

cudaError_t launch_geometry(const psi_surfels &s, const psi_camera &cam, float *table, int ld, cudaStream_t st);
cudaError_t launch_geometry_bwd(const psi_surfels &s, const psi_camera &cam, const float *g_table, int ld,
                                const psi_grads &g, cudaStream_t st);

} // namespace psi
