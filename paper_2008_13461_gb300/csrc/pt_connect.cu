// Step a3: Cellular-Automaton connection (Sec. 3.2).  Cells (a,b) and (b,c)
// sharing hit b are linked when the R-z alignment, dz, curvature and
// beamspot predicates of b's region (barrel or endcap, Sec. 4.2) pass.
//
// One warp owns one middle hit b.  It stages the live cells ending on b in
// shared memory once -- inner hit a, cell index and slope key -- and each
// lane takes one live cell (b,c) starting on b (from the out-lists built
// after the Fishbone) and scans the staged cells; the staged data are
// shared-memory broadcasts reused by every outer cell of b.
//
// The R-z cut is very tight, so it is first used as a window on the slope
// key.  For a barrel b, with key = dz/dr of a segment,
//     X = (r_b-r_a)(z_c-z_b) - (z_b-z_a)(r_c-r_b) = dr_ab dr_bc (key_c - key_a)
// and |X| <= tol |ac| <= tol (|ab| + |bc|) give
//     |key_c - key_a| <= tol (sqrt(1+key_a^2)/dr_bc + sqrt(1+key_c^2)/dr_ab);
// for a disk b the same holds with r and z exchanged.  With sqrt(1+key_a^2)
// and 1/dr_ab bounded by their maximum over the cells ending on b (both
// computed with the keys in the Fishbone kernel), every aligned candidate
// falls in the window; the
// few inside it take a float32 R-z test with an error bound and then the
// exact predicate chain.
//
// Each lane counts its accepted candidates and remembers the first few in a
// small shared-memory queue, so the incoming edges of a cell are reserved
// together and written contiguously (the depth-first search walks them
// backwards); the edge range of a cell is stored at its out-list position.
// Cells with incoming edges join the list the search starts from.  Hits with
// more than kCaMax live incoming cells scan them in global memory.
#include "pt_common.cuh"
#include "pt_kernels.cuh"

namespace ptk {

constexpr int kCaWarps = 4;
constexpr int kCaWords = 8;
constexpr int kCaMax = 32 * kCaWords;    // staged incoming cells per hit

// The full chain runs for the few candidates that pass the window and the
// float R-z test; out of line so that the scan loop stays small.
static __device__ __noinline__ bool ca_test(const FHit A, const FHit B, const FHit C, const pt_ca_cuts rg,
                                            int32_t *cnt) {
    return pred_rz(A, B, C, rg.tol_rz2, cnt) && pred_dz(A, C, rg.zmax, cnt) && pred_curv(A, B, C, rg.k_curv, cnt) &&
           pred_beamspot(A, B, C, rg.rmax2, cnt);
}

// Branch-free part of the R-z test: false only when the float32 evaluation
// with its error bound proves the alignment cut fails.
__device__ __forceinline__ bool rz_maybe(const float4 &a, const FHit &b, const FHit &c, float tol2) {
    const float d1 = b.r - a.w, d2 = c.z - b.z, d3 = b.z - a.z, d4 = c.r - b.r;
    const float p = d1 * d2, q = d3 * d4;
    const float X = p - q, Xb = fabsf(p) + fabsf(q);
    const float e1 = c.r - a.w, e2 = c.z - a.z;
    const float T = tol2 * (e1 * e1 + e2 * e2);
    return T - X * X >= -ferr(4, T + Xb * Xb);
}

__device__ __forceinline__ bool connects(const Params &p, const float4 &a, const FHit &B, const FHit &C,
                                         const pt_ca_cuts &rg) {
    if (!rz_maybe(a, B, C, rg.tol_rz2)) return false;
    const FHit A = {a.x, a.y, a.z, a.w};
    return ca_test(A, B, C, rg, p.counters);
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

constexpr int kCaQueue = 8;     // accepted candidates remembered per lane

__global__ void __launch_bounds__(32 * kCaWarps) k_connect(Params p) {
    __shared__ float4 s_a[kCaWarps][kCaMax];
    __shared__ float s_k[kCaWarps][kCaMax];
    __shared__ int32_t s_c[kCaWarps][kCaMax];
    __shared__ int16_t s_q[kCaWarps][kCaQueue][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n_binned = p.bin_cnt[p.n_bins];
    for (int b = blockIdx.x * kCaWarps + w; b < n_binned; b += gridDim.x * kCaWarps) {
        const int o0 = p.out_off[b], nout = p.out_off[b + 1] - o0;
        if (nout == 0) continue;
        int nin = p.in_cnt[b];
        const int64_t b0 = p.in_off[b];
        if (b0 + nin > p.cap_cells) nin = 0;
        const FHit B = load_hit(p.bh, b);
        const bool disk = p.layer[p.blayer[b]].kind == PT_LAYER_DISK;
        const pt_ca_cuts rg = p.region[disk ? 1 : 0];
        const float tol = p.region_tol[disk ? 1 : 0];
        const float2 hk = p.hk[b];
        // stage the live incoming cells of b (dead cells carry a NaN key)
        int ns = 0;
        for (int j0 = 0; j0 < nin; j0 += 32) {
            const int j = j0 + lane;
            const float key = j < nin ? p.ck[b0 + j] : 0.f;
            const bool live = j < nin && key == key;
            const unsigned m = __ballot_sync(0xffffffffu, live);
            if (live) {
                const int slot = ns + __popc(m & ((1u << lane) - 1u));
                if (slot < kCaMax) {
                    s_c[w][slot] = (int32_t)(b0 + j);
                    s_k[w][slot] = key;
                    s_a[w][slot] = __ldg(p.bh + p.cell_inner[b0 + j]);
                }
            }
            ns += __popc(m);
        }
        __syncwarp();
        const bool staged = ns <= kCaMax;
        for (int q0 = 0; q0 < nout; q0 += 32) {
            const int q = q0 + lane;
            const bool act = q < nout;
            int co = 0;
            FHit C = B;
            float key_c = 0.f, wdt = -1.f;
            if (act) {
                co = p.out_idx[o0 + q];
                C = load_hit(p.bh, p.cell_outer[co]);
                const float dr = C.r - B.r, dz = C.z - B.z;
                const float num = disk ? dr : dz, den = disk ? dz : dr;
                key_c = den != 0.f ? num / den : __int_as_float(0x7f800000);
                // window half-width, widened for float32 rounding of the keys
                wdt = tol * (hk.x / fabsf(den) + sqrtf(1.0f + key_c * key_c) / hk.y);
                wdt = wdt * (1.0f + 1e-5f) + 1e-5f * (1.0f + fabsf(key_c) + hk.x);
                if (!(wdt == wdt) || den == 0.f) wdt = __int_as_float(0x7f800000);
            }
            // count accepted candidates; remember the first kCaQueue
            int mine = 0;
            const int nc = act ? (staged ? ns : nin) : 0;
            for (int k = 0; k < nc; k++) {
                const float key = staged ? s_k[w][k] : p.ck[b0 + k];
                if (!(fabsf(key - key_c) <= wdt)) continue;
                const float4 a = staged ? s_a[w][k] : __ldg(p.bh + p.cell_inner[b0 + k]);
                if (connects(p, a, B, C, rg)) {
                    if (mine < kCaQueue) s_q[w][mine][lane] = (int16_t)k;
                    mine++;
                }
            }
            int total;
            const int excl = warp_excl(mine, lane, total);
            int64_t base = 0;
            if (lane == 0 && total > 0) base = atomicAdd(p.counters + C_EDGES, total);
            base = __shfl_sync(0xffffffffu, base, 0) + excl;
            if (mine > 0 && mine <= kCaQueue) {
                for (int t = 0; t < mine; t++) {
                    const int k = s_q[w][t][lane];
                    const int ci = staged ? s_c[w][k] : (int32_t)(b0 + k);
                    if (base + t < p.cap_edges) {
                        p.edge_src[base + t] = ci;
                        p.edge_dst[base + t] = co;
                    }
                    p.has_out[ci] = 1;
                }
            } else if (mine > kCaQueue) {   // rare: scan again to write all
                int64_t e = base;
                for (int k = 0; k < nc; k++) {
                    const float key = staged ? s_k[w][k] : p.ck[b0 + k];
                    if (!(fabsf(key - key_c) <= wdt)) continue;
                    const float4 a = staged ? s_a[w][k] : __ldg(p.bh + p.cell_inner[b0 + k]);
                    if (connects(p, a, B, C, rg)) {
                        const int ci = staged ? s_c[w][k] : (int32_t)(b0 + k);
                        if (e < p.cap_edges) {
                            p.edge_src[e] = ci;
                            p.edge_dst[e] = co;
                        }
                        p.has_out[ci] = 1;
                        e++;
                    }
                }
            }
            // list of cells with incoming edges (one atomic per warp)
            const unsigned lm = __ballot_sync(0xffffffffu, mine > 0);
            int lb = 0;
            if (lane == 0 && lm) lb = atomicAdd(p.counters + C_LEAVES, __popc(lm));
            lb = __shfl_sync(0xffffffffu, lb, 0) + __popc(lm & ((1u << lane) - 1u));
            if (act) {
                // incoming-edge range, stored at the cell's out-list position
                // (coalesced); the search finds it through the cell's rank
                p.edge_rng[o0 + q] = make_int2((int32_t)base, mine);
                if (base + mine > p.cap_edges) set_flag(p.counters, PT_FLAG_EDGES);
                if (mine > 0 && lb < p.cap_cells) p.leaf_list[lb] = co;
            }
            __syncwarp();
        }
        __syncwarp();
    }
}

void launch_connect(const Params &p, int grid, cudaStream_t s) {
    k_connect<<<grid * (kThreads / (32 * kCaWarps)), 32 * kCaWarps, 0, s>>>(p);
}

}  // namespace ptk
