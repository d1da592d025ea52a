// Hit binning without any allocation: the same kernels as the binning step
// of pt_build_doublets, with their scratch (per-hit tile and rank, event and
// layer of each binned hit, scan partial sums, device flags) in a
// file-scope device array instead of a caller-provided workspace.  For
// callers that cannot allocate device memory (see pt.h).
#include <string.h>

#include <atomic>

#include "pt_common.cuh"
#include "pt_kernels.cuh"

using namespace ptk;

namespace {

// Maximum problem accepted: 2^20 hits and 2^22 tiles (events x layers x
// phi tiles x t tiles).  Scratch: 13 bytes per hit, 4 bytes per 4096 tiles,
// plus the counters.
constexpr int64_t kMaxHits = int64_t(1) << 20;
constexpr int64_t kMaxTiles = int64_t(1) << 22;
constexpr size_t kCountersBytes = 256;
constexpr size_t kPartBytes = 4 * (size_t)(kMaxTiles / kScanItems + 256);
constexpr size_t kScratchBytes = kCountersBytes + kPartBytes + 13 * (size_t)kMaxHits + 8 * 256;

// Lives on every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch for the current device, looked up once per
// device (the name of a __device__ array is only a host-side stand-in).
// Host threads may race on the first lookup; each stores the same address.
std::atomic<void *> g_scratch_ptr[64];

pt_status scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PT_ERR_CUDA;
    void *ptr = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!ptr) {
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return PT_ERR_CUDA;
        g_scratch_ptr[dev].store(ptr, std::memory_order_release);
    }
    *out = ptr;
    return PT_OK;
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" pt_status pt_bin_hits_noalloc(const pt_hits *hits, const pt_geometry *geometry, int32_t n_phi_bins,
                                         int32_t n_t_bins, float *binned, int32_t *hit_order, int32_t *tile_off,
                                         int32_t *flags, void *stream) {
    if (!hits || !geometry || !binned || !hit_order || !tile_off || !flags || !hits->ev_off) return PT_ERR_INVALID_ARG;
    if (hits->n_hits < 0 || hits->n_events < 1) return PT_ERR_INVALID_ARG;
    if (hits->n_hits > 0 && (!hits->x || !hits->y || !hits->z || !hits->r || !hits->module))
        return PT_ERR_INVALID_ARG;
    if (n_phi_bins < 16 || n_phi_bins > 1024 || n_t_bins < 1 || n_t_bins > 64) return PT_ERR_INVALID_ARG;
    if (((uintptr_t)binned & 15) != 0) return PT_ERR_INVALID_ARG;
    if (!geometry->module_layer || geometry->n_modules <= 0) return PT_ERR_INVALID_ARG;
    for (int i = 0; i < PT_N_LAYERS; i++) {
        const pt_layer &l = geometry->layer[i];
        if ((l.kind != PT_LAYER_BARREL && l.kind != PT_LAYER_DISK) || !(l.rmin < l.rmax) || !(l.zmin < l.zmax))
            return PT_ERR_INVALID_ARG;
    }
    const int64_t n_tiles = (int64_t)hits->n_events * PT_N_LAYERS * n_phi_bins * n_t_bins;
    if ((int64_t)hits->n_hits > kMaxHits || n_tiles > kMaxTiles) return PT_ERR_TOO_LARGE;

    void *base = nullptr;
    pt_status st = scratch_address(&base);
    if (st != PT_OK) return st;
    char *w = (char *)base;
    const size_t nh = (size_t)(hits->n_hits > 0 ? hits->n_hits : 1);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = up256(o + bytes);
        return w + at;
    };

    Params p;
    memset(&p, 0, sizeof p);
    p.x = hits->x;
    p.y = hits->y;
    p.z = hits->z;
    p.r = hits->r;
    p.module = hits->module;
    p.ev_off = hits->ev_off;
    p.module_layer = geometry->module_layer;
    p.n_hits = hits->n_hits;
    p.n_events = hits->n_events;
    p.n_modules = geometry->n_modules;
    p.counters = (int32_t *)take(kCountersBytes);
    p.scan_part = (int32_t *)take(kPartBytes);
    p.hit_bin = (int32_t *)take(4 * nh);
    p.hit_rank = (int32_t *)take(4 * nh);
    p.bev = (int32_t *)take(4 * nh);
    p.blayer = (int8_t *)take(nh);
    p.bin_cnt = tile_off;
    p.bh = (float4 *)binned;
    p.perm = hit_order;
    p.n_phi = n_phi_bins;
    p.n_t = n_t_bins;
    p.n_bins = n_tiles;
    p.n_scan_blocks = (int32_t)((n_tiles + kScanItems - 1) / kScanItems);
    for (int i = 0; i < PT_N_LAYERS; i++) p.layer[i] = geometry->layer[i];

    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's contents: clear what must start at zero
    if (cudaMemsetAsync(p.counters, 0, kCountersBytes, s) != cudaSuccess) return PT_ERR_CUDA;
    if (cudaMemsetAsync(tile_off, 0, sizeof(int32_t) * (size_t)(n_tiles + 1), s) != cudaSuccess) return PT_ERR_CUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PT_ERR_CUDA;
    launch_binning(p, sms * 8, s);
    if (cudaMemcpyAsync(flags, p.counters + C_FLAGS, sizeof(int32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return PT_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA;
}
