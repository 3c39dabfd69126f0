// rti_launch.h -- launchers of the kernels, one set per state precision.
#pragma once

#include <cuda_runtime.h>

#include "rti_layout.h"

namespace rti {

// Enqueue one chunk of kp.nsteps steps with the given schedule, followed by the
// scenario advance. grid = CTAs of the persistent / grid-stride kernels.
template <class T>
cudaError_t launch_chunk(const KParams<T>& kp, int schedule, int grid, const int* nscen,
                         cudaStream_t st);
// sum(eta) per tile at the current level
template <class T>
cudaError_t launch_snapshot(const KParams<T>& kp, int grid, cudaStream_t st);
// child edge fluxes of parity p materialised into the flux arrays
template <class T>
cudaError_t launch_fill_edges(const KParams<T>& kp, int grid, int parity, cudaStream_t st);
// largest co-resident grid of the persistent kernel variant `mode` (kStep*) on the
// current device, with at most `cap` CTAs per SM when cap > 0
template <class T>
cudaError_t persistent_grid(int* grid, int tx, int ty, int mode, int cap);

}  // namespace rti
