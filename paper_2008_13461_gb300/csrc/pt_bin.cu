// Step a0: tile the hits of every (event, layer) in phi x t (t = z on barrel
// layers, r on disks) -- the paper's phi-tiled hit structure of Sec. 3.2,
// here two-dimensional.  Counting sort: per-hit tile + rank by
// warp-aggregated atomics, exclusive scan of the tile counts (block prefix
// scans), scatter into a binned structure of arrays.  Tiles only accelerate the doublet search; results do not depend
// on them.
#include "pt_common.cuh"
#include "pt_kernels.cuh"

namespace ptk {

__device__ __forceinline__ bool on_grid(float v) {
    float s = v * 16384.0f;
    return fabsf(v) < 64.0f && s == rintf(s);
}

// Tile and rank of every hit.  The warp takes 32 consecutive hits; lanes
// whose hits fall in the same tile reserve their ranks with one atomic
// (warp-aggregated: __match_any_sync groups them, the lowest lane adds the
// group's size and shares the old count).
__global__ void __launch_bounds__(kThreads) k_bin_count(Params p) {
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    for (int h0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); h0 < p.n_hits; h0 += stride) {
        const int h = h0 + lane;
        int bin = -1;
        if (h < p.n_hits) {
            float x = p.x[h], y = p.y[h], z = p.z[h], r = p.r[h];
            int m = p.module[h];
            bool bad = m < 0 || m >= p.n_modules;
            int L = bad ? 0 : p.module_layer[m];
            bad = bad || L < 0 || L >= PT_N_LAYERS;
            bad = bad || !on_grid(x) || !on_grid(y) || !on_grid(z) || !on_grid(r);
            float tmin = 0.f, tmax = 1.f, t = 0.f;
            if (!bad) {
                const pt_layer ly = p.layer[L];
                bad = r < ly.rmin || r > ly.rmax || z < ly.zmin || z > ly.zmax;
                if (ly.kind == PT_LAYER_BARREL) {
                    t = z; tmin = ly.zmin; tmax = ly.zmax;
                } else {
                    t = r; tmin = ly.rmin; tmax = ly.rmax;
                }
            }
            if (bad) {
                set_flag(p.counters, PT_FLAG_INPUT);
            } else {
                // event of hit h: ev_off[e] <= h < ev_off[e+1]
                int lo = 0, hi = p.n_events - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (__ldg(p.ev_off + mid) <= h) lo = mid; else hi = mid - 1;
                }
                int pb = phi_tile(atan2f(y, x), p.n_phi);
                int tb = t_tile(t, tmin, tmax, p.n_t);
                bin = ((lo * PT_N_LAYERS + L) * p.n_phi + pb) * p.n_t + tb;
            }
            p.hit_bin[h] = bin;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, bin);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader && bin >= 0) base = atomicAdd(p.bin_cnt + bin, __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (bin >= 0) p.hit_rank[h] = base + __popc(peers & ((1u << lane) - 1u));
    }
}

// exclusive scan of bin_cnt[0 .. n_bins) in place; bin_cnt[n_bins] = total
__device__ __forceinline__ int block_exclusive_scan(int v, int *smem_warp, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int s = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, s, d);
        if (lane >= d) s += t;
    }
    if (lane == 31) smem_warp[warp] = s;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (kThreads / 32) ? smem_warp[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += t;
        }
        if (lane < (kThreads / 32)) smem_warp[lane] = w;
    }
    __syncthreads();
    int excl = s - v + (warp > 0 ? smem_warp[warp - 1] : 0);
    total = smem_warp[kThreads / 32 - 1];
    __syncthreads();
    return excl;
}

constexpr int kPerThread = kScanItems / kThreads;   // 16

// Exclusive scan of a[0 .. n) in place, a[n] = total, in three kernels:
// per-block sums, a one-block scan of those, per-block scans plus offset.
__global__ void __launch_bounds__(kThreads) k_scan_reduce(const int32_t *a, int64_t n, int32_t *part) {
    __shared__ int sw[kThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanItems + (int64_t)threadIdx.x * kPerThread;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kPerThread; k++) {
        int64_t i = base + k;
        if (i < n) s += a[i];
    }
    int total;
    block_exclusive_scan(s, sw, total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kThreads) k_scan_partials(int32_t *part, int nblocks, int32_t *total_out) {
    __shared__ int sw[kThreads / 32];
    int carry = 0;
    for (int b0 = 0; b0 < nblocks; b0 += kThreads) {
        int i = b0 + threadIdx.x;
        int v = i < nblocks ? part[i] : 0;
        int total;
        int e = block_exclusive_scan(v, sw, total);
        if (i < nblocks) part[i] = carry + e;
        carry += total;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void __launch_bounds__(kThreads) k_scan_apply(int32_t *a, int64_t n, const int32_t *part) {
    __shared__ int sw[kThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanItems + (int64_t)threadIdx.x * kPerThread;
    int v[kPerThread];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kPerThread; k++) {
        int64_t i = base + k;
        v[k] = i < n ? a[i] : 0;
        s += v[k];
    }
    int total;
    int e = block_exclusive_scan(s, sw, total) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kPerThread; k++) {
        int64_t i = base + k;
        if (i < n) a[i] = e;
        e += v[k];
    }
}

void launch_scan(int32_t *a, int64_t n, int32_t *part, cudaStream_t s) {
    const int nb = (int)((n + kScanItems - 1) / kScanItems);
    if (nb > 0) {
        KernelTimer t("k_scan_reduce", s);
        k_scan_reduce<<<nb, kThreads, 0, s>>>(a, n, part);
    }
    {
        KernelTimer t("k_scan_partials", s);
        k_scan_partials<<<1, kThreads, 0, s>>>(part, nb, a + n);
    }
    if (nb > 0) {
        KernelTimer t("k_scan_apply", s);
        k_scan_apply<<<nb, kThreads, 0, s>>>(a, n, part);
    }
}

__global__ void __launch_bounds__(kThreads) k_bin_fill(Params p) {
    const int stride = gridDim.x * blockDim.x;
    const int per_event = PT_N_LAYERS * p.n_phi * p.n_t;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < p.n_hits; h += stride) {
        int bin = p.hit_bin[h];
        if (bin < 0) continue;
        int pos = p.bin_cnt[bin] + p.hit_rank[h];
        p.bh[pos] = make_float4(p.x[h], p.y[h], p.z[h], p.r[h]);
        p.perm[pos] = h;
        p.bev[pos] = bin / per_event;
        p.blayer[pos] = (int8_t)((bin / (p.n_phi * p.n_t)) % PT_N_LAYERS);
    }
}

void launch_binning(const Params &p, int grid, cudaStream_t s) {
    {
        KernelTimer t("k_bin_count", s);
        k_bin_count<<<grid, kThreads, 0, s>>>(p);
    }
    launch_scan(p.bin_cnt, p.n_bins, p.scan_part, s);
    KernelTimer t("k_bin_fill", s);
    k_bin_fill<<<grid, kThreads, 0, s>>>(p);
}

}  // namespace ptk
