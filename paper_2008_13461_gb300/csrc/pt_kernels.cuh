// Host-side launchers of the stage kernels (one per translation unit).
#pragma once

#include "pt_common.cuh"

namespace ptk {

void launch_scan(int32_t *a, int64_t n, int32_t *part, cudaStream_t s);
void launch_binning(const Params &p, int grid, cudaStream_t s);
void launch_doublets(const Params &p, int lanes, int grid, cudaStream_t s);
void launch_fishbone(const Params &p, float unit_thr, float du, int grid, cudaStream_t s);
void launch_connect(const Params &p, int grid, cudaStream_t s);
void launch_ntuplets(const Params &p, int grid, cudaStream_t s);
void launch_select(const Params &p, int grid, cudaStream_t s);
void launch_fit(const Params &p, int grid, cudaStream_t s);

}  // namespace ptk
