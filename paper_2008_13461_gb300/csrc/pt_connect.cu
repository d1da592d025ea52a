// Step a3: Cellular-Automaton connection (Sec. 3.2).  Cells (a,b) and (b,c)
// sharing hit b are linked when the R-z alignment, dz, curvature and
// beamspot predicates of b's region (barrel or endcap, Sec. 4.2) pass.
//
// Cells (b,c) are taken in cell order (cells are grouped by their outer hit
// c, so neighbouring threads work on neighbouring middle hits).
// The live cells ending on b were written by the Fishbone kernel ordered by
// a bucket of their R-z slope key relative to b (monotone in the key, about
// one cell per bucket), with their inner hits, so the candidates (a,b) of a
// cell lie in a contiguous run of that array (the buckets of its key
// window), found by binary search over the buckets.
//
// The R-z cut is very tight, so it is first used as a window on the slope
// key.  For a barrel b, with key = dz/dr of a segment,
//     X = (r_b-r_a)(z_c-z_b) - (z_b-z_a)(r_c-r_b) = dr_ab dr_bc (key_c - key_a)
// and |X| <= tol |ac| <= tol (|ab| + |bc|) give
//     |key_c - key_a| <= tol (sqrt(1+key_a^2)/dr_bc + sqrt(1+key_c^2)/dr_ab);
// for a disk b the same holds with r and z exchanged.  With sqrt(1+key_a^2)
// and 1/dr_ab bounded by their maximum over the cells ending on b, every
// aligned candidate falls in the window; the run searched is the window
// widened far beyond the rounding of the key differences, and inside it the
// window test itself, a float32 R-z test with an error bound and then the
// exact predicate chain decide.
//
// The kernel waits on dependent L2 loads, so it is compiled for 10
// resident blocks of 4 warps per SM (48 registers), which hides more of that
// latency than 8 blocks did, and spills less than 12.
//
// A warp takes 128 consecutive cells at a time, in order from a queue.
// Only cells whose inner hit has live cells ending on it have candidates at
// all (about a quarter), so the warp first lists those and then runs their
// searches on full lanes.
// The incoming edges of a cell are written contiguously (the depth-first
// search walks them backwards from the cell's edge range); the warp
// reserves the edges of its 128 cells with one atomic, each cell remembers
// its first few accepted candidates in shared memory, and a cell with more
// (rare) scans again to write them all.
//
// The predicates run as float32 filters only; a cell with a candidate they
// cannot decide (about one in 10^5) is left to a second pass that has the
// exact forms, which keeps the big-integer code and its registers out of
// the main kernel.
#include "pt_common.cuh"
#include "pt_kernels.cuh"

namespace ptk {

constexpr int kCaWarps = 4;
constexpr int kCaQueue = 4;         // accepted candidates remembered per cell
constexpr int kCaChunk = 4;         // rounds of 32 cells per edge reservation

// The predicate chain: 1 connects, 0 does not; with kExact = false, 2 when
// a float32 filter cannot decide and none fails.
template <bool kExact>
__device__ __forceinline__ int ca_chain(const FHit &A, const FHit &B, const FHit &C, const pt_ca_cuts &rg,
                                        int32_t *cnt) {
    const int r1 = pred_rz<kExact>(A, B, C, rg.tol_rz2, cnt);
    if (!r1) return 0;
    const int r2 = pred_dz<kExact>(A, C, rg.zmax, cnt);
    if (!r2) return 0;
    const int r3 = pred_curv<kExact>(A, B, C, rg.k_curv, cnt);
    if (!r3) return 0;
    const int r4 = pred_beamspot<kExact>(A, B, C, rg.rmax2, cnt);
    if (!r4) return 0;
    return (r1 | r2 | r3 | r4) == 1 ? 1 : 2;
}

// the exact chain, out of line (only the pass over undecided cells uses it)
static __device__ __noinline__ int ca_test(const FHit A, const FHit B, const FHit C, const pt_ca_cuts rg,
                                           int32_t *cnt) {
    return ca_chain<true>(A, B, C, rg, cnt);
}

// Branch-free part of the R-z test: false only when the float32 evaluation
// with its error bound proves the alignment cut fails.
__device__ __forceinline__ bool rz_maybe(const float4 &a, const FHit &b, const FHit &c, float tol2) {
    const float X = det2(b.r - a.w, c.z - b.z, b.z - a.z, c.r - b.r);
    const float e1 = c.r - a.w, e2 = c.z - a.z;
    const float T = tol2 * (e1 * e1 + e2 * e2);
    return T - X * X >= -ferr(4, T + X * X);
}

template <bool kExact>
__device__ __forceinline__ int connects(const Params &p, const float4 &a, const FHit &B, const FHit &C,
                                        const pt_ca_cuts &rg) {
    if (!rz_maybe(a, B, C, rg.tol_rz2)) return 0;
    const FHit A = {a.x, a.y, a.z, a.w};
    if (kExact) return ca_test(A, B, C, rg, p.counters);
    return ca_chain<false>(A, B, C, rg, p.counters);
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

// first position of s[0, n) whose key's bucket is >= bk (buckets ascending)
__device__ __forceinline__ int lower_bucket(const float2 *s, int n, int bk, float k0, float iw) {
    const float fb = (float)bk;
    int l = 0, h = bk > 0 ? n : 0;
    while (l < h) {
        const int m = (l + h) >> 1;
        if (sk_coord(__ldg(s + m).x, k0, iw) < fb) l = m + 1;
        else h = m;
    }
    return l;
}

// Every inner cell (a,b) connecting to the live cell x = (b,c), in the
// order of b's bucket-ordered arrays: emit(t, i) for the t-th one, i its
// index there.
// Returns their number, or -2 (kExact = false) when a candidate is
// undecided.
template <bool kExact, class Emit>
__device__ __forceinline__ int scan_cell(const Params &p, int x, Emit &&emit) {
    const int b = p.cell_inner[x], c = p.cell_outer[x];
    const int64_t b0 = p.in_off[b];
    int ns = p.in_live[b];
    if (b0 + ns > p.cap_cells) ns = 0;
    if (ns == 0) return 0;
    const FHit B = load_hit(p.bh, b), C = load_hit(p.bh, c);
    const bool disk = p.layer[p.blayer[b]].kind == PT_LAYER_DISK;
    const pt_ca_cuts rg = p.region[disk ? 1 : 0];
    const float tol = p.region_tol[disk ? 1 : 0];
    const float4 hk = p.hk[b];
    const float dr = C.r - B.r, dz = C.z - B.z;
    const float num = disk ? dr : dz, den = disk ? dz : dr;
    const float key_c = den != 0.f ? num / den : __int_as_float(0x7f800000);
    // window half-width, widened for float32 rounding of the keys
    float wdt = tol * (hk.x / fabsf(den) + sqrtf(1.0f + key_c * key_c) / hk.y);
    wdt = wdt * (1.0f + 1e-5f) + 1e-5f * (1.0f + fabsf(key_c) + hk.x);
    if (!(wdt == wdt) || den == 0.f) wdt = __int_as_float(0x7f800000);
    // keys passing the window test lie in [lo, hi]
    const float sl = (fabsf(key_c) + wdt) * 9.5367431640625e-7f;
    const float lo = key_c - wdt - sl;
    float hi = key_c + wdt + sl;
    if (!(hi == hi)) hi = __int_as_float(0x7f800000);
    // the cells are ordered by a bucket of their key, monotone in the key:
    // the run searched is that of the buckets of [lo, hi]
    const float2 *S = p.sk + b0;
    const int nb = sk_buckets(ns);
    const int bhi = sk_bucket(hi, hk.z, hk.w, nb);
    const float fend = bhi < nb - 1 ? (float)(bhi + 1) : __int_as_float(0x7f800000);
    int n = 0;
    for (int r = lower_bucket(S, ns, sk_bucket(lo, hk.z, hk.w, nb), hk.z, hk.w); r < ns; r++) {
        const float2 e = __ldg(S + r);
        if (sk_coord(e.x, hk.z, hk.w) >= fend) break;     // a bucket above hi's
        if (!(fabsf(e.x - key_c) <= wdt)) continue;
        const int v = connects<kExact>(p, __ldg(p.bh + __float_as_int(e.y)), B, C, rg);
        if (v == 2) return -2;
        if (v) emit(n++, b0 + r);
    }
    return n;
}

__global__ void __launch_bounds__(32 * kCaWarps, 10) k_connect(Params p) {
    constexpr int kPer = 32 * kCaChunk;
    __shared__ int32_t s_q[kCaWarps][kCaQueue][kPer];   // accepted inner cells per chunk position
    __shared__ int32_t s_m[kCaWarps][kPer];             // edges per chunk position (-1: no live cell,
                                                        //   -2: a cell that can have no incoming edge)
    __shared__ int16_t s_list[kCaWarps][kPer];          // positions whose inner hit has live cells
    if (upstream_overflow(p, PT_FLAG_CELLS)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    const int64_t n_cells = min((int64_t)p.counters[C_CELLS], p.cap_cells);
    const int n_chunks = (int)((n_cells + kPer - 1) / kPer);
    // the warps take the chunks in order from a queue: the chunks in flight
    // are neighbours, and so are the middle hits whose sorted cells they read
    for (;;) {
        int ch = 0;
        if (lane == 0) ch = atomicAdd(p.counters + C_CA_NEXT, 1);
        ch = __shfl_sync(0xffffffffu, ch, 0);
        if (ch >= n_chunks) break;
        const int64_t x0 = (int64_t)ch * kPer;
        // 1) live cells, and a list of those with candidates at all (the
        //    inner hit has live cells ending on it), so that the searches
        //    run on full warps
        int nlist = 0;
        unsigned ranged = 0;     // lanes with a cell whose edge range is written
#pragma unroll
        for (int it = 0; it < kCaChunk; it++) {
            const int pos = it * 32 + lane;
            const int64_t x = x0 + pos;
            int st = -1;
            bool need = false;
            if (x < n_cells && p.cell_alive[x]) {
                // no cell ends on an inner hit on a layer that is the outer
                // layer of no pair (most cells start on BPix1): such a cell
                // has no incoming edges, and no edge range is written for
                // it (-2; the search records read none)
                st = -2;
                if (p.pair_inner_is_outer[p.cell_pair[x]]) {
                    st = 0;
                    need = p.in_live[p.cell_inner[x]] > 0;
                }
            }
            s_m[w][pos] = st;
            ranged |= __ballot_sync(0xffffffffu, st >= 0);
            const unsigned m = __ballot_sync(0xffffffffu, need);
            if (need) s_list[w][nlist + __popc(m & below)] = (int16_t)pos;
            nlist += __popc(m);
        }
        // a chunk of cells that can have no incoming edge (the cells of
        // outer hits on BPix2 all start on BPix1) has nothing more to do
        if (!ranged) continue;
        __syncwarp();
        // 2) the searches
        for (int i = lane; i < nlist; i += 32) {
            const int pos = s_list[w][i];
            int m = scan_cell<false>(p, (int)(x0 + pos), [&](int t, int64_t k) {
                if (t < kCaQueue) s_q[w][t][pos] = p.sci[k];
            });
            if (m == -2) {   // undecided: left to the exact pass
                const int k = atomicAdd(p.counters + C_CA_PENDING, 1);
                if (k < p.cap_cells) reinterpret_cast<int32_t *>(p.ck)[k] = (int32_t)(x0 + pos);
                else set_flag(p.counters, PT_FLAG_CELLS);
                m = -1;
            }
            s_m[w][pos] = m;
        }
        __syncwarp();
        // 3) edges of the chunk: one reservation, then each cell's edges
        //    contiguously and its edge range
        int tot = 0;
#pragma unroll
        for (int it = 0; it < kCaChunk; it++) tot += max(s_m[w][it * 32 + lane], 0);
        int total;
        const int excl = warp_excl(tot, lane, total);
        int64_t base = 0;
        if (lane == 0 && total > 0) base = atomicAdd(p.counters + C_EDGES, total);
        base = __shfl_sync(0xffffffffu, base, 0) + excl;
#pragma unroll 1
        for (int it = 0; it < kCaChunk; it++) {
            const int pos = it * 32 + lane;
            const int64_t x = x0 + pos;
            const int m = s_m[w][pos];
            if (m < 0) continue;
            if (m > 0) {
                if (m <= kCaQueue) {
                    for (int t = 0; t < m; t++) {
                        const int ci = s_q[w][t][pos];
                        if (base + t < p.cap_edges) {
                            p.edge_src[base + t] = ci;
                            p.edge_dst[base + t] = (int32_t)x;
                        }
                        p.has_out[ci] = 1;
                    }
                } else {   // rare: scan again to write them all
                    const int64_t e0 = base;
                    scan_cell<false>(p, (int)x, [&](int t, int64_t k) {
                        const int ci = p.sci[k];
                        if (e0 + t < p.cap_edges) {
                            p.edge_src[e0 + t] = ci;
                            p.edge_dst[e0 + t] = (int32_t)x;
                        }
                        p.has_out[ci] = 1;
                    });
                }
                if (base + m > p.cap_edges) set_flag(p.counters, PT_FLAG_EDGES);
            }
            p.edge_rng[x] = make_int2((int32_t)base, m);
            base += m;
        }
        __syncwarp();
    }
}

// The cells with an undecided candidate (a few hundred), one thread each,
// with the exact predicates; each reserves its own edges.
__global__ void __launch_bounds__(128) k_connect_exact(Params p) {
    if (upstream_overflow(p, PT_FLAG_CELLS)) return;
    const int n = (int)min((int64_t)p.counters[C_CA_PENDING], p.cap_cells);
    const int32_t *list = reinterpret_cast<const int32_t *>(p.ck);
    // cells dealt round the blocks first: they spread over the SMs, and a
    // warp seldom holds two cells whose exact fallbacks would run in turn
    for (int k = threadIdx.x * gridDim.x + blockIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int x = list[k];
        const int m = scan_cell<true>(p, x, [](int, int64_t) {});
        const int64_t base = m > 0 ? atomicAdd(p.counters + C_EDGES, m) : 0;
        scan_cell<true>(p, x, [&](int t, int64_t i) {
            const int ci = p.sci[i];
            if (base + t < p.cap_edges) {
                p.edge_src[base + t] = ci;
                p.edge_dst[base + t] = x;
            }
            p.has_out[ci] = 1;
        });
        if (base + m > p.cap_edges) set_flag(p.counters, PT_FLAG_EDGES);
        p.edge_rng[x] = make_int2((int32_t)base, m);
    }
}

void launch_connect(const Params &p, int grid, cudaStream_t s) {
    {
        KernelTimer t("k_connect", s);
        k_connect<<<grid * (kThreads / (32 * kCaWarps)), 32 * kCaWarps, 0, s>>>(p);
    }
    KernelTimer t("k_connect_exact", s);
    k_connect_exact<<<grid / 8 + 1, 128, 0, s>>>(p);
}

}  // namespace ptk
