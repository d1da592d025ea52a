// Post-fit steps (Sec. 3.5-3.6).
//
// Ambiguity resolution (Sec. 3.5): tracks sharing a hit-doublet (a cell)
// keep only the best chi2; then triplets sharing a hit keep only the
// smallest |transverse impact parameter|.  Each rule is a minimum per cell
// (per hit) taken with 32-bit atomicMin on the float's bits (order-preserving
// for non-negative floats; NaN counts as +inf), and a track survives when it
// attains the minimum at every cell (hit) it has: equal values all survive,
// and the result does not depend on the order of the tracks.
#include "pt_common.cuh"
#include "pt_kernels.cuh"

namespace ptk {
namespace {

__device__ __forceinline__ uint32_t key_of(float v) {
    return v >= 0.f ? __float_as_uint(v) : 0x7f800000u;    // NaN and negatives -> +inf
}

struct AmbArgs {
    const int32_t *hits, *cells, *track_tuple;
    const uint8_t *n;
    const float *chi2, *tip;
    int32_t tip_stride, n_tracks, n_cells, n_hits;
    uint32_t *best_cell, *best_hit;
    uint8_t *keep;
};

__global__ void __launch_bounds__(kThreads) k_amb_cells(AmbArgs a) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n_tracks; k += gridDim.x * blockDim.x) {
        const int t = a.track_tuple[k];
        const int n = a.n[t];
        const uint32_t key = key_of(a.chi2[k]);
        for (int j = 0; j + 1 < n; j++) {
            const int c = a.cells[(int64_t)t * PT_NMAX + j];
            if (c >= 0 && c < a.n_cells) atomicMin(a.best_cell + c, key);
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_amb_hits(AmbArgs a) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n_tracks; k += gridDim.x * blockDim.x) {
        const int t = a.track_tuple[k];
        const int n = a.n[t];
        const uint32_t key = key_of(a.chi2[k]);
        bool keep = true;
        for (int j = 0; j + 1 < n; j++) {
            const int c = a.cells[(int64_t)t * PT_NMAX + j];
            if (c >= 0 && c < a.n_cells) keep &= a.best_cell[c] == key;
        }
        a.keep[k] = keep;
        if (keep && n == 3) {
            const uint32_t k2 = key_of(fabsf(a.tip[(int64_t)k * a.tip_stride]));
            for (int j = 0; j < 3; j++) {
                const int h = a.hits[(int64_t)t * PT_NMAX + j];
                if (h >= 0 && h < a.n_hits) atomicMin(a.best_hit + h, k2);
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_amb_final(AmbArgs a) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n_tracks; k += gridDim.x * blockDim.x) {
        const int t = a.track_tuple[k];
        if (!a.keep[k] || a.n[t] != 3) continue;
        const uint32_t k2 = key_of(fabsf(a.tip[(int64_t)k * a.tip_stride]));
        bool keep = true;
        for (int j = 0; j < 3; j++) {
            const int h = a.hits[(int64_t)t * PT_NMAX + j];
            if (h >= 0 && h < a.n_hits) keep &= a.best_hit[h] == k2;
        }
        a.keep[k] = keep;
    }
}

}  // namespace

void launch_ambiguities(const int32_t *hits, const int32_t *cells, const uint8_t *n, const int32_t *track_tuple,
                        int32_t n_tracks, const float *chi2, const float *tip, int32_t tip_stride, int32_t n_cells,
                        int32_t n_hits, uint32_t *scratch, uint8_t *keep, int grid, cudaStream_t s) {
    AmbArgs a{hits, cells, track_tuple, n, chi2, tip, tip_stride, n_tracks, n_cells, n_hits,
              scratch, scratch + n_cells, keep};
    {
        KernelTimer t("k_amb_cells", s);
        k_amb_cells<<<grid, kThreads, 0, s>>>(a);
    }
    {
        KernelTimer t("k_amb_hits", s);
        k_amb_hits<<<grid, kThreads, 0, s>>>(a);
    }
    KernelTimer t("k_amb_final", s);
    k_amb_final<<<grid, kThreads, 0, s>>>(a);
}

}  // namespace ptk
