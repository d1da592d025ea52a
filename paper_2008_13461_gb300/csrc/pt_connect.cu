// Step a3: Cellular-Automaton connection (Sec. 3.2).  Every live cell
// (b,c) is tested against every live cell (a,b) ending on its inner hit --
// those form one contiguous range thanks to the doublet kernel -- with the
// dz, R-z alignment, curvature and beamspot predicates of the region of b
// (barrel or endcap, Sec. 4.2).  A group of G lanes owns one outer cell; each
// lane records its verdicts for up to 32 candidates in a bit mask, so the
// accepted incoming edges of a cell are reserved with one atomic and written
// contiguously (the depth-first search walks them backwards).  Cells with
// more than 32 G candidates take a count-then-write path.
#include "pt_common.cuh"
#include "pt_kernels.cuh"

namespace ptk {

__device__ __forceinline__ bool ca_ok(const Params &p, int64_t ci, const FHit &B, const FHit &Cc,
                                      const pt_ca_cuts &rg) {
    if (!p.cell_alive[ci]) return false;
    const int a = p.cell_inner[ci];
    const FHit A = {p.bx[a], p.by[a], p.bz[a], p.br[a]};
    return pred_dz(A, Cc, rg.zmax, p.counters) && pred_rz(A, B, Cc, rg.tol_rz2, p.counters) &&
           pred_curv(A, B, Cc, rg.k_curv, p.counters) && pred_beamspot(A, B, Cc, rg.rmax2, p.counters);
}

template <int G>
__global__ void __launch_bounds__(kThreads) k_connect(Params p) {
    constexpr int kGroups = kThreads / G;
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int gshift = (threadIdx.x & 31) & ~(G - 1);
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << gshift);
    __shared__ int s_alive;
    if (threadIdx.x == 0) s_alive = 0;
    __syncthreads();
    int my_alive = 0;
    const int64_t n_cells = min((int64_t)p.counters[C_CELLS], p.cap_cells);
    for (int64_t co = (int64_t)blockIdx.x * kGroups + grp; co < n_cells; co += (int64_t)gridDim.x * kGroups) {
        if (lane == 0) {
            p.maxlen[co] = 0;
            my_alive += p.cell_alive[co];
        }
        int nin = 0;
        int64_t b0 = 0;
        FHit B, Cc;
        pt_ca_cuts rg = p.region[0];
        if (p.cell_alive[co]) {
            const int b = p.cell_inner[co], c = p.cell_outer[co];
            nin = p.in_cnt[b];
            b0 = p.in_off[b];
            if (b0 + nin > p.cap_cells) nin = 0;
            B = {p.bx[b], p.by[b], p.bz[b], p.br[b]};
            Cc = {p.bx[c], p.by[c], p.bz[c], p.br[c]};
            rg = p.region[p.layer[p.blayer[b]].kind == PT_LAYER_DISK ? 1 : 0];
        }
        const int iters = (nin + G - 1) / G;
        unsigned mask = 0;
        int mine = 0;
        if (iters <= 32) {
            for (int it = 0; it < iters; it++) {
                const int q = it * G + lane;
                if (q < nin && ca_ok(p, b0 + q, B, Cc, rg)) mask |= 1u << it;
            }
            mine = __popc(mask);
        } else {
            for (int q = lane; q < nin; q += G) mine += ca_ok(p, b0 + q, B, Cc, rg);
        }
        // exclusive prefix of per-lane counts within the group
        int incl = mine;
#pragma unroll
        for (int d = 1; d < G; d <<= 1) {
            int t = __shfl_up_sync(gmask, incl, d, G);
            if (lane >= d) incl += t;
        }
        const int total = __shfl_sync(gmask, incl, gshift + G - 1);
        int64_t base = 0;
        if (lane == 0 && total > 0) base = atomicAdd(p.counters + C_EDGES, total);
        base = __shfl_sync(gmask, base, gshift);
        int64_t e = base + incl - mine;
        if (iters <= 32) {
            while (mask) {
                const int it = __ffs(mask) - 1;
                mask &= mask - 1;
                const int64_t ci = b0 + it * G + lane;
                if (e < p.cap_edges) {
                    p.edge_src[e] = (int32_t)ci;
                    p.edge_dst[e] = (int32_t)co;
                }
                p.has_out[ci] = 1;
                e++;
            }
        } else {
            for (int q = lane; q < nin; q += G) {
                if (ca_ok(p, b0 + q, B, Cc, rg)) {
                    if (e < p.cap_edges) {
                        p.edge_src[e] = (int32_t)(b0 + q);
                        p.edge_dst[e] = (int32_t)co;
                    }
                    p.has_out[b0 + q] = 1;
                    e++;
                }
            }
        }
        if (lane == 0) {
            p.edge_off[co] = (int32_t)base;
            p.edge_cnt[co] = total;
            if (base + total > p.cap_edges) set_flag(p.counters, PT_FLAG_EDGES);
        }
    }
    if (my_alive) atomicAdd(&s_alive, my_alive);
    __syncthreads();
    if (threadIdx.x == 0 && s_alive) atomicAdd(p.counters + C_ALIVE_CELLS, s_alive);
}

void launch_connect(const Params &p, int lanes, int grid, cudaStream_t s) {
    switch (lanes) {
    case 4: k_connect<4><<<grid, kThreads, 0, s>>>(p); break;
    case 8: k_connect<8><<<grid, kThreads, 0, s>>>(p); break;
    case 16: k_connect<16><<<grid, kThreads, 0, s>>>(p); break;
    default: k_connect<32><<<grid, kThreads, 0, s>>>(p); break;
    }
}

}  // namespace ptk
