// Step a3: Cellular-Automaton connection (Sec. 3.2).  Cells (a,b) and (b,c)
// sharing hit b are linked when the dz, R-z alignment, curvature and
// beamspot predicates of b's region (barrel or endcap, Sec. 4.2) pass.
//
// One warp owns one middle hit b.  It stages the live cells ending on b
// (their inner hits a) in shared memory once, then each lane takes one live
// cell (b,c) starting on b -- from the out-lists built after the Fishbone --
// and tests it against every staged cell.  All lanes do the same number of
// tests and read the staged hits as shared-memory broadcasts; the per-pair
// data are reused by every outer cell of b instead of being gathered again.
// Each lane keeps its verdicts in a register bit mask, so the incoming edges
// of a cell are reserved together and written contiguously (the depth-first
// search walks them backwards).  Cells with incoming edges are appended to a
// list the search starts from.  Hits with more than kCaMax live incoming
// cells use a count-then-write path over global memory.
#include "pt_common.cuh"
#include "pt_kernels.cuh"

namespace ptk {

constexpr int kCaWarps = 4;
constexpr int kCaWords = 8;
constexpr int kCaMax = 32 * kCaWords;    // staged incoming cells per hit

__device__ __forceinline__ bool ca_test(const FHit &A, const FHit &B, const FHit &C, const pt_ca_cuts &rg,
                                        int32_t *cnt) {
    return pred_rz(A, B, C, rg.tol_rz2, cnt) && pred_dz(A, C, rg.zmax, cnt) && pred_curv(A, B, C, rg.k_curv, cnt) &&
           pred_beamspot(A, B, C, rg.rmax2, cnt);
}

// exclusive prefix of v over the warp, and the warp total
__device__ __forceinline__ int warp_excl(int v, int lane, int &total) {
    int incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - v;
}

__device__ __forceinline__ void finish_cell(const Params &p, int co, int64_t base, int total) {
    p.edge_off[co] = (int32_t)base;
    p.edge_cnt[co] = total;
    p.maxlen[co] = 0;
    if (base + total > p.cap_edges) set_flag(p.counters, PT_FLAG_EDGES);
    if (total > 0) {
        const int k = atomicAdd(p.counters + C_LEAVES, 1);
        if (k < p.cap_cells) p.leaf_list[k] = co;
    }
}

__global__ void __launch_bounds__(32 * kCaWarps) k_connect(Params p) {
    __shared__ float4 s_a[kCaWarps][kCaMax];
    __shared__ int32_t s_c[kCaWarps][kCaMax];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n_binned = p.bin_cnt[p.n_bins];
    for (int b = blockIdx.x * kCaWarps + w; b < n_binned; b += gridDim.x * kCaWarps) {
        const int o0 = p.out_off[b], nout = p.out_off[b + 1] - o0;
        if (nout == 0) continue;
        int nin = p.in_cnt[b];
        const int64_t b0 = p.in_off[b];
        if (b0 + nin > p.cap_cells) nin = 0;
        const FHit B = load_hit(p.bh, b);
        const pt_ca_cuts rg = p.region[p.layer[p.blayer[b]].kind == PT_LAYER_DISK ? 1 : 0];
        // stage the live incoming cells of b
        int ns = 0;
        for (int j0 = 0; j0 < nin; j0 += 32) {
            const int j = j0 + lane;
            const bool live = j < nin && p.cell_alive[b0 + j];
            const unsigned m = __ballot_sync(0xffffffffu, live);
            if (live) {
                const int slot = ns + __popc(m & ((1u << lane) - 1u));
                if (slot < kCaMax) {
                    s_c[w][slot] = (int32_t)(b0 + j);
                    s_a[w][slot] = __ldg(p.bh + p.cell_inner[b0 + j]);
                }
            }
            ns += __popc(m);
        }
        __syncwarp();
        for (int q0 = 0; q0 < nout; q0 += 32) {
            const int q = q0 + lane;
            const bool act = q < nout;
            int co = 0;
            FHit C = B;
            if (act) {
                co = p.out_idx[o0 + q];
                C = load_hit(p.bh, p.cell_outer[co]);
            }
            if (ns <= kCaMax) {
                unsigned mask[kCaWords];
                int mine = 0;
#pragma unroll
                for (int wd = 0; wd < kCaWords; wd++) {
                    unsigned m = 0;
                    if (act && wd * 32 < ns) {
                        const int kend = min(32, ns - wd * 32);
                        for (int kk = 0; kk < kend; kk++) {
                            const float4 a4 = s_a[w][wd * 32 + kk];
                            const FHit A = {a4.x, a4.y, a4.z, a4.w};
                            if (ca_test(A, B, C, rg, p.counters)) m |= 1u << kk;
                        }
                    }
                    mask[wd] = m;
                    mine += __popc(m);
                }
                int total;
                const int excl = warp_excl(mine, lane, total);
                int64_t base = 0;
                if (lane == 0 && total > 0) base = atomicAdd(p.counters + C_EDGES, total);
                base = __shfl_sync(0xffffffffu, base, 0) + excl;
                int64_t e = base;
#pragma unroll
                for (int wd = 0; wd < kCaWords; wd++) {
                    unsigned m = mask[wd];
                    while (m) {
                        const int kk = __ffs(m) - 1;
                        m &= m - 1;
                        const int ci = s_c[w][wd * 32 + kk];
                        if (e < p.cap_edges) {
                            p.edge_src[e] = ci;
                            p.edge_dst[e] = co;
                        }
                        p.has_out[ci] = 1;
                        e++;
                    }
                }
                if (act) finish_cell(p, co, base, mine);
            } else {
                // many incoming cells: count, reserve, then write
                int mine = 0;
                if (act)
                    for (int j = 0; j < nin; j++)
                        if (p.cell_alive[b0 + j] &&
                            ca_test(load_hit(p.bh, p.cell_inner[b0 + j]), B, C, rg, p.counters))
                            mine++;
                int total;
                const int excl = warp_excl(mine, lane, total);
                int64_t base = 0;
                if (lane == 0 && total > 0) base = atomicAdd(p.counters + C_EDGES, total);
                base = __shfl_sync(0xffffffffu, base, 0) + excl;
                int64_t e = base;
                if (act)
                    for (int j = 0; j < nin; j++)
                        if (p.cell_alive[b0 + j] &&
                            ca_test(load_hit(p.bh, p.cell_inner[b0 + j]), B, C, rg, p.counters)) {
                            if (e < p.cap_edges) {
                                p.edge_src[e] = (int32_t)(b0 + j);
                                p.edge_dst[e] = co;
                            }
                            p.has_out[b0 + j] = 1;
                            e++;
                        }
                if (act) finish_cell(p, co, base, mine);
            }
        }
        __syncwarp();
    }
}

void launch_connect(const Params &p, int grid, cudaStream_t s) {
    k_connect<<<grid * (kThreads / (32 * kCaWarps)), 32 * kCaWarps, 0, s>>>(p);
}

}  // namespace ptk
