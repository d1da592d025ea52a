// Steps a4 + a5: roots, depth-first search and shared-doublet cleaning
// (Sec. 3.2, 3.3).
//
// The paper runs one DFS per root along outgoing edges.  Here every maximal
// path is enumerated from its other end: one thread per edge into a leaf cell
// (live, no outer neighbour) walks incoming edges -- stored contiguously per
// cell by the connection kernel -- back to cells with no inner neighbour,
// and emits the path when that cell is a root (inner hit on BPix1, or on
// BPix2 / FPix1+- which, having no inner neighbour, qualifies) and the path
// has at least three hits.  Root-to-leaf paths are the same set either way, and no
// outgoing-edge lists need to be built.  Path length is bounded on the host
// (the layer-pair graph admits no path longer than PT_NMAX hits).
#include "pt_common.cuh"
#include "pt_kernels.cuh"

namespace ptk {

__device__ __forceinline__ bool root_layer(int L) { return L == 0 || L == 1 || L == 4 || L == 7; }

// One record per edge with what the search needs of its source cell, so that
// each step back along a path is one dependent load: the source, its own
// incoming-edge range, and its inner hit (input index) with the root flag.
__global__ void __launch_bounds__(kThreads) k_edge_records(Params p) {
    if (upstream_overflow(p, PT_FLAG_CELLS)) return;
    const int64_t ne = min((int64_t)p.counters[C_EDGES], p.cap_edges);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
        const int src = p.edge_src[e];
        // a cell starting on a layer no cell ends on has no incoming edges
        // (and the connection wrote no range for it)
        const int2 r = p.pair_inner_is_outer[p.cell_pair[src]] ? p.edge_rng[src] : make_int2(0, 0);
        const int bi = p.cell_inner[src];
        p.erec[e] = make_int4(src, r.x, r.y, p.perm[bi] * 2 + (root_layer(p.blayer[bi]) ? 1 : 0));
    }
}

// A path being searched: per depth d (0 = the leaf), the cell and its inner
// hit's input index * 2 + root flag.  Indexed with compile-time depths only,
// so it lives in registers.
struct DfsPath {
    int32_t cell[PT_NMAX - 1];
    int32_t hit[PT_NMAX - 1];
};

// the path of cells cell[D] (a root) .. cell[0] (the leaf) as an n-tuplet
template <int D>
__device__ __forceinline__ void dfs_emit(const Params &p, const DfsPath &pa, int leaf_outer) {
    // one atomic for the lanes that emit together
    const unsigned am = __activemask();
    const int leader = __ffs(am) - 1, lane = threadIdx.x & 31;
    int t = 0;
    if (lane == leader) t = atomicAdd(p.counters + C_TUPLES, __popc(am));
    t = __shfl_sync(am, t, leader) + __popc(am & ((1u << lane) - 1u));
    if (t >= p.cap_tuples) {
        set_flag(p.counters, PT_FLAG_TUPLES);
        return;
    }
    int32_t *hits = p.tup_hits + (int64_t)t * PT_NMAX;
    int32_t *cells = p.tup_cells + (int64_t)t * PT_NMAX;
    hits[0] = pa.hit[D] >> 1;
#pragma unroll
    for (int q = 0; q <= D; q++) {
        // the outer hit of a cell is the inner hit of the next one
        cells[q] = pa.cell[D - q];
        hits[q + 1] = D - q >= 1 ? pa.hit[D - q - 1] >> 1 : leaf_outer;
    }
    p.tup_n[t] = (uint8_t)(D + 2);
    p.tup_alive[t] = 1;
}

// Depth D of the search: cell[D] has cnt incoming edges from position first.
// No incoming edge: a path starts here, emitted if cell[D] is a root and the
// path has at least three hits.  Paths longer than PT_NMAX hits are cut.
template <int D>
__device__ __forceinline__ void dfs_level(const Params &p, DfsPath &pa, int first, int cnt, int leaf_outer) {
    if (cnt == 0) {
        if (D >= 1 && (pa.hit[D] & 1)) dfs_emit<D>(p, pa, leaf_outer);
        return;
    }
    if constexpr (D + 1 < PT_NMAX - 1) {
        for (int it = 0; it < cnt; it++) {
            const int64_t e = (int64_t)first + it;
            if (e >= p.cap_edges) continue;
            const int4 r = p.erec[e];
            pa.cell[D + 1] = r.x;
            pa.hit[D + 1] = r.w;
            dfs_level<D + 1>(p, pa, r.y, r.z, leaf_outer);
        }
    }
}

// One thread per edge; an edge into a leaf (a live cell with no outer
// neighbour) starts the search: the leaf and the edge's source are the
// path's first two cells, searched back from there.
__global__ void __launch_bounds__(kThreads) k_dfs(Params p) {
    if (upstream_overflow(p, PT_FLAG_CELLS)) return;
    const int64_t ne = min((int64_t)p.counters[C_EDGES], p.cap_edges);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride) {
        const int c = p.edge_dst[e];
        if (p.has_out[c]) continue;
        const int4 r = p.erec[e];
        DfsPath pa;
        pa.cell[0] = c;
        pa.hit[0] = p.perm[p.cell_inner[c]] * 2;
        pa.cell[1] = r.x;
        pa.hit[1] = r.w;
        dfs_level<1>(p, pa, r.y, r.z, p.perm[p.cell_outer[c]]);
    }
}

// L(c) = longest n-tuplet containing cell c
__global__ void __launch_bounds__(kThreads) k_clean_max(Params p) {
    const int64_t nt = min((int64_t)p.counters[C_TUPLES], p.cap_tuples);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
        const int n = p.tup_n[t];
        const int32_t *cells = p.tup_cells + t * PT_NMAX;
        for (int k = 0; k < n - 1; k++) atomicMax(p.maxlen + cells[k], n);
    }
}

// keep an n-tuplet unless one of its cells belongs to a longer one
__global__ void __launch_bounds__(kThreads) k_clean_keep(Params p) {
    const int64_t nt = min((int64_t)p.counters[C_TUPLES], p.cap_tuples);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int kept = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
        const int n = p.tup_n[t];
        const int32_t *cells = p.tup_cells + t * PT_NMAX;
        bool keep = true;
#pragma unroll
        for (int k = 0; k < PT_NMAX - 1; k++)     // independent loads
            if (k < n - 1) keep &= n >= p.maxlen[cells[k]];
        p.tup_alive[t] = keep;
        kept += keep;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, d);
    if ((threadIdx.x & 31) == 0 && kept) atomicAdd(p.counters + C_ALIVE_TUPLES, kept);
}

// queue the surviving n-tuplets with >= min_hits hits for the fit
// Tracks are the surviving n-tuplets with at least min_hits hits.  Their
// indices are grouped by hit count (3, 4, 5, 6..8) so that each fit kernel,
// compiled for one count, works on a dense range, and within a class follow
// the n-tuplet order, so a fit repeated on moved hits lists the same tracks
// in the same order.  Block b of kSelBlocks owns a contiguous slice of the
// n-tuplets: the first kernel counts each slice's classes, the second turns
// the counts into offsets and ranks each slice's tracks in order.
__device__ __forceinline__ int track_class_of(const Params &p, int64_t t) {
    const int n = p.tup_n[t];
    return p.tup_alive[t] && n >= p.min_hits ? track_class(n) : -1;
}

__global__ void __launch_bounds__(kThreads) k_count_tracks(Params p) {
    __shared__ int s_cnt[4];
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t nt = min((int64_t)p.counters[C_TUPLES], p.cap_tuples);
    const int64_t per = (nt + kSelBlocks - 1) / kSelBlocks;
    const int64_t t0 = blockIdx.x * per, t1 = min(t0 + per, nt);
    for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        const int c = track_class_of(p, t);
        if (c >= 0) atomicAdd(&s_cnt[c], 1);
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        p.trk_blk[blockIdx.x * 4 + threadIdx.x] = s_cnt[threadIdx.x];
        if (s_cnt[threadIdx.x]) atomicAdd(p.counters + C_TRK_CNT + threadIdx.x, s_cnt[threadIdx.x]);
    }
}

__global__ void __launch_bounds__(kThreads) k_select_tracks(Params p) {
    __shared__ int s_base[4];
    __shared__ int s_wcnt[kThreads / 32][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int off[4], total = 0;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        off[c] = total;
        total += p.counters[C_TRK_CNT + c];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        p.counters[C_TRACKS] = total;
        if (total > p.cap_tracks) set_flag(p.counters, PT_FLAG_TRACKS);
    }
    // this slice's start in each class: the counts of the slices before it
    if (threadIdx.x < 4) {
        int b = 0;
        for (int q = 0; q < (int)blockIdx.x; q++) b += p.trk_blk[q * 4 + threadIdx.x];
        s_base[threadIdx.x] = off[threadIdx.x] + b;
    }
    __syncthreads();
    const int64_t nt = min((int64_t)p.counters[C_TUPLES], p.cap_tuples);
    const int64_t per = (nt + kSelBlocks - 1) / kSelBlocks;
    const int64_t t0 = blockIdx.x * per, t1 = min(t0 + per, nt);
    for (int64_t tb = t0; tb < t1; tb += blockDim.x) {
        const int64_t t = tb + threadIdx.x;
        const int c = t < t1 ? track_class_of(p, t) : -1;
        // rank in n-tuplet order: within the warp by ballot, across warps
        // by the warps' counts
        int rank = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const unsigned m = __ballot_sync(0xffffffffu, c == q);
            if (lane == 0) s_wcnt[w][q] = __popc(m);
            if (c == q) rank = __popc(m & ((1u << lane) - 1u));
        }
        __syncthreads();
        if (c >= 0) {
            int before = 0;
            for (int q = 0; q < w; q++) before += s_wcnt[q][c];
            const int k = s_base[c] + before + rank;
            if (k < p.cap_tracks) p.trk_tuple[k] = (int32_t)t;
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            int add = 0;
            for (int q = 0; q < kThreads / 32; q++) add += s_wcnt[q][threadIdx.x];
            s_base[threadIdx.x] += add;
        }
        __syncthreads();
    }
}

void launch_select(const Params &p, int grid, cudaStream_t s) {
    (void)grid;
    {
        KernelTimer t("k_count_tracks", s);
        k_count_tracks<<<kSelBlocks, kThreads, 0, s>>>(p);
    }
    KernelTimer t("k_select_tracks", s);
    k_select_tracks<<<kSelBlocks, kThreads, 0, s>>>(p);
}

void launch_ntuplets(const Params &p, int grid, cudaStream_t s) {
    {
        KernelTimer t("k_edge_records", s);
        k_edge_records<<<grid, kThreads, 0, s>>>(p);
    }
    {
        KernelTimer t("k_dfs", s);
        k_dfs<<<grid, kThreads, 0, s>>>(p);
    }
    {
        KernelTimer t("k_clean_max", s);
        k_clean_max<<<grid, kThreads, 0, s>>>(p);
    }
    KernelTimer t("k_clean_keep", s);
    k_clean_keep<<<grid, kThreads, 0, s>>>(p);
}

}  // namespace ptk
