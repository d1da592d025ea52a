// Host-side launchers of the stage kernels (one per translation unit).
#pragma once

#include "pt_common.cuh"

namespace ptk {

// Brackets the kernel launches of its scope with two CUDA events on the
// stream while kernel timing is enabled (pt_kernel_timing); does nothing
// otherwise or while the stream is being captured.
class KernelTimer {
  public:
    KernelTimer(const char *name, cudaStream_t s);
    ~KernelTimer();
    KernelTimer(const KernelTimer &) = delete;
    KernelTimer &operator=(const KernelTimer &) = delete;

  private:
    const char *name_;
    cudaStream_t s_;
    cudaEvent_t a_;
};

void launch_scan(int32_t *a, int64_t n, int32_t *part, cudaStream_t s);
void launch_binning(const Params &p, int grid, cudaStream_t s);
void launch_doublets(const Params &p, int lanes, int grid, cudaStream_t s);
void launch_fishbone(const Params &p, float unit_thr, float du, int grid, cudaStream_t s);
void launch_connect(const Params &p, int grid, cudaStream_t s);
void launch_ntuplets(const Params &p, int grid, cudaStream_t s);
void launch_select(const Params &p, int grid, cudaStream_t s);
void launch_fit(const Params &p, int grid, cudaStream_t s);
void launch_fit_grad(const Params &p, const float *gpar, const float *gchi, float *gx, float *gy, float *gz, int grid,
                     cudaStream_t s);
void launch_ambiguities(const int32_t *hits, const int32_t *cells, const uint8_t *n, const int32_t *track_tuple,
                        int32_t n_tracks, const float *chi2, const float *tip, int32_t tip_stride, int32_t n_cells,
                        int32_t n_hits, uint32_t *scratch, uint8_t *keep, int grid, cudaStream_t s);
void launch_align(int n, const float *x, const float *y, const float *z, const int32_t *module, const float *centre,
                  const float *shift, const float *rot, float *xo, float *yo, float *zo, int grid, cudaStream_t s);
void launch_align_grad(int n, const float *x, const float *y, const float *z, const int32_t *module,
                       const float *centre, const float *rot, const float *gxa, const float *gya, const float *gza,
                       float *gx, float *gy, float *gz, float *gshift, float *grot, int grid, cudaStream_t s);
size_t vertex_scratch_bytes(int32_t n_tracks, int32_t n_events);
pt_status launch_vertices(const pt_vertex_tracks &in, int32_t n_tracks, int32_t n_events,
                          const pt_vertex_cuts &cuts, int32_t max_vertices, void *scratch, const pt_vertices &out,
                          int grid, cudaStream_t s);
void launch_track_summary(int32_t n_tracks, const int32_t *hits, const uint8_t *tn, const float *params,
                          const float *cov, const int32_t *tuple, const int32_t *ev_off, int32_t n_events, float bz,
                          int32_t *ev, float *z0, float *ez0, float *pt, uint8_t *nhits, int grid, cudaStream_t s);

}  // namespace ptk
