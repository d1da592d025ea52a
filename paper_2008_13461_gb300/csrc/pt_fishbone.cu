// Step a2: the Fishbone (Sec. 3.3), and the per-cell data the CA connection
// needs from it.
//
// Cells sharing an outer hit o whose inner hits lie on one layer and are
// aligned as seen from o form a fishbone; every cell of it dies except the
// shortest (equal lengths: the smaller input index of the inner hit wins).
//
// One warp per outer hit.  The warp keeps, per cell, the difference vector
// u = h_inner - h_o in shared memory; hits are multiples of 2^-14 below 64 in
// magnitude, so u is exact in float32 and the alignment test and the squared
// length (an integer in grid units) are evaluated from it with no further
// memory traffic.  Alignment within eps implies that the unit directions of
// two siblings differ by at most du = eps pi/2 (plus float32 slack), hence
// so does any 1-Lipschitz key of them (u^_z for a barrel o, the radial
// component for a disk o).  The siblings are counting-sorted into about
// one key bucket each, and each cell is compared only with the later cells
// of its own bucket and of the next K buckets, K covering a key difference
// of du: a superset of its aligned siblings, so the result is exact at
// ~O(k) work per outer hit.
//
// Shared memory per warp bounds the siblings it can hold, and the warps an
// SM can keep resident bound how well the gathers of the inner hits are
// hidden.  Most outer hits have fewer than ~200 cells, so three launches
// share the work: many small warps take chunks of 32 outer hits from a queue
// and list the outer hits with more cells, which medium (up to 320 cells)
// and large warps (up to 512) then take one at a time; an exact pass takes
// the rest (undecided tests, more cells) with a pairwise loop over global
// memory beyond 512.
//
// The same pass prepares the CA connection: it writes the live cells of o
// ordered by a bucket of their R-z slope key relative to o (with the inner
// hit and the cell index; the bucket is monotone in the key, about one cell
// per bucket, free order inside), the bucket parameters, and per hit the
// bounds the slope window needs (taken over all cells of o, a superset of
// the live ones, so the window only widens).
#include "pt_common.cuh"
#include "pt_kernels.cuh"

namespace ptk {

constexpr int kFbDirect = 12;        // up to this many siblings: compare all pairs

// Per warp and cell: u = h_inner - h_o (exact) and 1/|u| in w; the cell's
// position (bits 0-9), its inner layer (10-14) and key bucket (16-25).
// C: the cell's R-z slope key and inner hit are kept for the second pass
// (else written to and read back from global memory).
template <int W, int M, int NB, bool C>
struct FbSmem {
    float4 rec[W][M];
    int meta[W][M];
    int16_t idx[W][M];               // cell positions sorted by bucket
    uint8_t dead[W][M];
    int pos[W][NB];
    float ck[W][C ? M : 1];
    int32_t inner[W][C ? M : 1];
};

__device__ __forceinline__ int rec_cell(int m) { return m & 1023; }
constexpr int kRecLayerMask = 31 << 10;

// Bucket key of a record: u^_z (barrel o) or the radial component of u^
// (disk o; (rx, ry) is o's radial direction).  Explicit roundings, so every
// evaluation gives the same bits.
__device__ __forceinline__ float fb_key(const float4 &r, bool disk, float rx, float ry) {
    const float k = disk ? __fmul_rn(__fmaf_rn(r.x, rx, __fmul_rn(r.y, ry)), r.w) : __fmul_rn(r.z, r.w);
    return k == k ? k : 0.f;
}

// squared length of a difference vector, in grid units (exact)
__device__ __forceinline__ long long len2u(float ux, float uy, float uz) {
    const int x = __float2int_rn(ux * 16384.0f), y = __float2int_rn(uy * 16384.0f), z = __float2int_rn(uz * 16384.0f);
    return (long long)x * x + (long long)y * y + (long long)z * z;     // |x| < 2^21: 32x32 -> 64-bit products
}

__device__ __forceinline__ int cell_layer(const Params &p, int64_t c) { return p.pair[p.cell_pair[c]].inner; }

// Does sibling d (record r2, meta m2) kill cell j (record r1, unit vector
// v1, meta m1)?  Same inner layer, unit directions close (a necessary
// condition of alignment), aligned, and strictly shorter or as long with a
// smaller input index of the inner hit.  kExact = false: an undecided
// alignment sets und.
template <bool kExact>
__device__ __forceinline__ bool fb_kills(const Params &p, int64_t b, int j, const float4 &r1, const float3 &v1,
                                         int m1, int d, int m2, const float4 &r2, float unit_thr, bool &und) {
    if (d == j || ((m1 ^ m2) & kRecLayerMask)) return false;
    const float dx = v1.x - r2.x * r2.w, dy = v1.y - r2.y * r2.w, dz = v1.z - r2.z * r2.w;
    if (dx * dx + dy * dy + dz * dz > unit_thr) return false;
    const int v = pred_fb_d<kExact>(r1.x, r1.y, r1.z, r2.x, r2.y, r2.z, p.fishbone_eps2, p.counters);
    if (v == 2) und = true;
    if (v != 1) return false;
    const long long l1 = len2u(r1.x, r1.y, r1.z), l2 = len2u(r2.x, r2.y, r2.z);
    return l2 < l1 || (l2 == l1 && p.perm[p.cell_inner[b + d]] < p.perm[p.cell_inner[b + j]]);
}

// Warp-wide minimum, maximum and sum with one redux instruction each.  The
// float map keeps their order (non-negative floats keep their bits,
// negative ones have the magnitude bits flipped; no NaN reaches it), and a
// minimum or maximum is one of the inputs, so nothing is rounded.
__device__ __forceinline__ int ford(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float fval(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }
__device__ __forceinline__ float warp_min(float f) { return fval(__reduce_min_sync(0xffffffffu, ford(f))); }
__device__ __forceinline__ float warp_max(float f) { return fval(__reduce_max_sync(0xffffffffu, ford(f))); }
__device__ __forceinline__ int warp_sum(int v) { return __reduce_add_sync(0xffffffffu, v); }

// exclusive prefix sum of a[0, nb) in place (nb a power of two >= 32;
// one warp, nb / 32 entries per lane)
__device__ __forceinline__ void warp_exclusive_scan(int *a, int nb, int lane) {
    const int per = nb >> 5;
    int sum = 0;
    for (int q = 0; q < per; q++) sum += a[lane * per + q];
    int incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    int run = incl - sum;
    for (int q = 0; q < per; q++) {
        const int v = a[lane * per + q];
        a[lane * per + q] = run;
        run += v;
    }
}

// Verdicts of the n cells of outer hit o (one warp); returns the lane's
// count of live cells.  kGlobal: n may exceed M (pairwise loop compiled in).
// kExact = false (float32 filters only): returns -1, having written no
// verdict, when n > M or an alignment test is undecided.
template <int W, int M, int NB, bool kGlobal, bool kExact, bool C>
__device__ __forceinline__ int fishbone_hit(const Params &p, int o, int n, int64_t b, int lane, int w,
                                            float unit_thr, float du, FbSmem<W, M, NB, C> &sm) {
    // NB: at least the buckets of M cells (sk_buckets), and of the direction sort
    static_assert(NB >= 32 && NB >= M && (NB & (NB - 1)) == 0, "bucket array too small");
    if (!kExact && n > M) return -1;
    const float4 ho = __ldg(p.bh + o);
    const bool disk = p.layer[p.blayer[o]].kind == PT_LAYER_DISK;
    const bool in_smem = !kGlobal || n <= M;
    const float irr = rsqrtf(ho.x * ho.x + ho.y * ho.y);
    const float rx = ho.x * irr, ry = ho.y * irr;
    // a hit on a layer that is the inner layer of no pair starts no cell:
    // the connection never reads the slope keys of the cells ending on it
    const bool starts = p.layer_is_inner[p.blayer[o]] != 0;
    // pass 1: R-z slope keys (barrel o: (z_o - z_a)/(r_o - r_a); disk o:
    // (r_o - r_a)/(z_o - z_a)) with the per-hit bounds; records and the
    // range of the bucket keys
    float k2max = 0.f, gmin = 3.0e38f, bmin = 3.0f, bmax = -3.0f;
    for (int j = lane; j < n; j += 32) {
        const int i = p.cell_inner[b + j];
        const int L = cell_layer(p, b + j);
        const float4 a = __ldg(p.bh + i);
        if (starts) {
            const float dr = ho.w - a.w, dz = ho.z - a.z;
            const float num = disk ? dr : dz, den = disk ? dz : dr;
            // the key only places the cell in the connection's search window,
            // whose margins (1e-5 relative) are far above the 2 ulp of this quotient
            const float ck = den != 0.f ? __fdividef(num, den) : __int_as_float(0x7f800000);
            k2max = fmaxf(k2max, ck * ck);
            gmin = fminf(gmin, fabsf(den));
            if (C && in_smem) {
                sm.ck[w][j] = ck;
                sm.inner[w][j] = i;
            } else {
                p.ck[b + j] = ck;
            }
        }
        if (in_smem) {
            const float ux = a.x - ho.x, uy = a.y - ho.y, uz = a.z - ho.z;
            const float4 r = make_float4(ux, uy, uz, rsqrtf(ux * ux + uy * uy + uz * uz));
            sm.rec[w][j] = r;
            sm.meta[w][j] = j | (L << 10) | (p.pair_slot[p.cell_pair[b + j]] << 26);
            sm.dead[w][j] = 0;
            const float key = fb_key(r, disk, rx, ry);
            bmin = fminf(bmin, key);
            bmax = fmaxf(bmax, key);
        }
    }
    k2max = warp_max(k2max);
    gmin = warp_min(gmin);
    const float kmax = sqrtf(1.0f + k2max);        // max of sqrt(1 + key^2)
    if (lane == 0 && starts) reinterpret_cast<float2 *>(p.hk + o)[0] = make_float2(kmax, gmin);
    __syncwarp();

    bool und = false;
    if (kGlobal && !in_smem) {
        // more siblings than the warp holds: plain pairwise loop
        const GHit gh = ghit(ho.x, ho.y, ho.z, ho.w);
        const FHit h = {ho.x, ho.y, ho.z, ho.w};
        for (int j = lane; j < n; j += 32) {
            const int i1 = p.cell_inner[b + j];
            const int L1 = cell_layer(p, b + j);
            const FHit h1 = load_hit(p.bh, i1);
            const GHit g1 = ghit(h1.x, h1.y, h1.z, h1.r);
            const long long l1 = (g1.x - gh.x) * (g1.x - gh.x) + (g1.y - gh.y) * (g1.y - gh.y) +
                                 (g1.z - gh.z) * (g1.z - gh.z);
            bool dead = false;
            for (int d = 0; d < n && !dead; d++) {
                if (d == j || cell_layer(p, b + d) != L1) continue;
                const int i2 = p.cell_inner[b + d];
                const FHit h2 = load_hit(p.bh, i2);
                if (!pred_fb(h1, h2, h, p.fishbone_eps2, p.counters)) continue;
                const GHit g2 = ghit(h2.x, h2.y, h2.z, h2.r);
                const long long l2 = (g2.x - gh.x) * (g2.x - gh.x) + (g2.y - gh.y) * (g2.y - gh.y) +
                                     (g2.z - gh.z) * (g2.z - gh.z);
                dead = l2 < l1 || (l2 == l1 && p.perm[i2] < p.perm[i1]);
            }
            if (dead) p.cell_alive[b + j] = 0;
        }
    } else if (n <= kFbDirect) {
        for (int j = lane; j < n; j += 32) {
            const float4 r1 = sm.rec[w][j];
            const float3 v1 = make_float3(r1.x * r1.w, r1.y * r1.w, r1.z * r1.w);
            const int m1 = sm.meta[w][j];
            bool dead = false;
            for (int d = 0; d < n && !dead; d++)
                dead = fb_kills<kExact>(p, b, j, r1, v1, m1, d, sm.meta[w][d], sm.rec[w][d], unit_thr, und);
            if (dead) sm.dead[w][j] = 1;
        }
    } else {
        bmin = warp_min(bmin);
        bmax = warp_max(bmax);
        // counting sort of the cells into buckets of (inner layer, direction
        // key): each inner layer of o has its own aligned range of nbr
        // buckets (about one bucket per cell), so a cell meets only siblings
        // on its own layer.  Two keys within du lie at most K buckets apart
        // (K bounds du / width plus the rounding of the bucket coordinates,
        // below 3e-4 for up to 1024 buckets).
        const int nb = min(NB, max(32, 1 << (32 - __clz(n - 1))));
        const int ssh = p.fb_slot_shift[p.blayer[o]];
        const int nbr = nb >> ssh;
        const float span = fmaxf(bmax - bmin, fmaxf(fabsf(bmin), fabsf(bmax)) * 1e-6f);
        const float iw = span > 0.f ? (float)nbr / span : 0.f;
        const int K = (int)fminf(du * iw + 3e-4f, (float)nbr) + 1;
        for (int q = lane; q < nb; q += 32) sm.pos[w][q] = 0;
        __syncwarp();
        for (int j = lane; j < n; j += 32) {
            const float key = fb_key(sm.rec[w][j], disk, rx, ry);
            const int m = sm.meta[w][j];
            const int bk = (m >> 26) * nbr + min(max((int)((key - bmin) * iw), 0), nbr - 1);
            sm.meta[w][j] = (m & 0xffff) | (bk << 16);
            atomicAdd(&sm.pos[w][bk], 1);
        }
        __syncwarp();
        warp_exclusive_scan(sm.pos[w], nb, lane);
        __syncwarp();
        for (int j = lane; j < n; j += 32) sm.idx[w][atomicAdd(&sm.pos[w][sm.meta[w][j] >> 16], 1)] = (int16_t)j;
        __syncwarp();
        // sm.pos[bk] is now the end of bucket bk.  Each pair once: every cell
        // against the cells after it in its own bucket and the next K
        // buckets of its layer (a superset of its siblings within du of its
        // key); of an aligned pair the longer cell dies (equal lengths: the
        // larger input index of the inner hit).
        for (int q0 = lane; q0 < n; q0 += 32) {
            const int j = sm.idx[w][q0];
            const float4 r1 = sm.rec[w][j];
            const float3 v1 = make_float3(r1.x * r1.w, r1.y * r1.w, r1.z * r1.w);
            const int bk1 = sm.meta[w][j] >> 16;
            const int qend = sm.pos[w][min(bk1 + K, bk1 | (nbr - 1))];
            for (int q = q0 + 1; q < qend; q++) {
                const int d = sm.idx[w][q];
                const float4 r2 = sm.rec[w][d];
                const float dx = v1.x - r2.x * r2.w, dy = v1.y - r2.y * r2.w, dz = v1.z - r2.z * r2.w;
                if (dx * dx + dy * dy + dz * dz > unit_thr) continue;
                const int v = pred_fb_d<kExact>(r1.x, r1.y, r1.z, r2.x, r2.y, r2.z, p.fishbone_eps2, p.counters);
                if (v == 2) und = true;
                if (v != 1) continue;
                const long long l1 = len2u(r1.x, r1.y, r1.z), l2 = len2u(r2.x, r2.y, r2.z);
                const bool j_wins = l1 < l2 || (l1 == l2 && p.perm[p.cell_inner[b + j]] < p.perm[p.cell_inner[b + d]]);
                sm.dead[w][j_wins ? d : j] = 1;
            }
        }
    }
    __syncwarp();
    if (!kExact && __any_sync(0xffffffffu, und)) return -1;

    // pass 2: the live cells, grouped by slope-key bucket for the CA
    // connection.  A hit on a layer that is the inner layer of no pair
    // starts no cell, so the connection never searches the cells ending on
    // it: only their Fishbone verdicts are written.
    int alive = 0;
    if (!starts) {
        int nl = 0;
        for (int j = lane; j < n; j += 32) {
            const bool dead = in_smem ? sm.dead[w][j] != 0 : p.cell_alive[b + j] == 0;
            if (dead && in_smem) p.cell_alive[b + j] = 0;
            alive += !dead;
        }
        nl = warp_sum(alive);
        if (lane == 0) p.in_live[o] = nl;
    } else if (in_smem) {
        // slope key and inner hit of each live cell (the records are free)
        float smin = __int_as_float(0x7f800000), smax = -smin;
        for (int j = lane; j < n; j += 32) {
            if (sm.dead[w][j]) {
                p.cell_alive[b + j] = 0;
                continue;
            }
            const float key = C ? sm.ck[w][j] : p.ck[b + j];
            const int ii = C ? sm.inner[w][j] : p.cell_inner[b + j];
            sm.rec[w][j] = make_float4(key, __int_as_float(ii), 0.f, 0.f);
            if (fabsf(key) <= 3.4e38f) {
                smin = fminf(smin, key);
                smax = fmaxf(smax, key);
            }
            alive++;
        }
        const int nl = warp_sum(alive);
        smin = warp_min(smin);
        smax = warp_max(smax);
        // counting sort into about one bucket per cell; the connection
        // searches by bucket, so the order inside a bucket is free
        const int nb = sk_buckets(nl);
        const float span = fmaxf(smax - smin, fmaxf(fabsf(smin), fabsf(smax)) * 1e-6f);
        const float iw = span > 0.f && span <= 3.4e38f ? (float)nb / span : 0.f;
        for (int q = lane; q < nb; q += 32) sm.pos[w][q] = 0;
        __syncwarp();
        for (int j = lane; j < n; j += 32) {
            if (sm.dead[w][j]) continue;
            const int bk = sk_bucket(sm.rec[w][j].x, smin, iw, nb);
            sm.meta[w][j] = bk;
            atomicAdd(&sm.pos[w][bk], 1);
        }
        __syncwarp();
        warp_exclusive_scan(sm.pos[w], nb, lane);
        __syncwarp();
        for (int j = lane; j < n; j += 32) {
            if (sm.dead[w][j]) continue;
            const float4 r = sm.rec[w][j];
            const int q = atomicAdd(&sm.pos[w][sm.meta[w][j]], 1);
            p.sk[b + q] = make_float2(r.x, r.y);
            p.sci[b + q] = (int32_t)(b + j);
        }
        if (lane == 0) {
            p.in_live[o] = nl;
            reinterpret_cast<float2 *>(p.hk + o)[1] = make_float2(smin, iw);
        }
    } else {
        // (only outer hits with very many cells) rank by direct comparison:
        // sorted keys, so sorted buckets too
        float smin = __int_as_float(0x7f800000), smax = -smin;
        for (int j = lane; j < n; j += 32) {
            if (!p.cell_alive[b + j]) continue;
            const float key = p.ck[b + j];
            const int ii = p.cell_inner[b + j];
            int rank = 0;
            for (int i = 0; i < n; i++) {
                if (!p.cell_alive[b + i]) continue;
                const float ki = p.ck[b + i];
                rank += ki < key || (ki == key && i < j);
            }
            p.sk[b + rank] = make_float2(key, __int_as_float(ii));
            p.sci[b + rank] = (int32_t)(b + j);
            if (fabsf(key) <= 3.4e38f) {
                smin = fminf(smin, key);
                smax = fmaxf(smax, key);
            }
            alive++;
        }
        const int nl = warp_sum(alive);
        smin = warp_min(smin);
        smax = warp_max(smax);
        const float span = fmaxf(smax - smin, fmaxf(fabsf(smin), fabsf(smax)) * 1e-6f);
        const float iw = span > 0.f && span <= 3.4e38f ? (float)sk_buckets(nl) / span : 0.f;
        if (lane == 0) {
            p.in_live[o] = nl;
            reinterpret_cast<float2 *>(p.hk + o)[1] = make_float2(smin, iw);
        }
    }
    __syncwarp();
    return alive;
}

// an outer hit left to the exact pass (listed in hit_bin, free once the
// hits are binned and the doublets' exact pass has run)
__device__ __forceinline__ void list_pending(const Params &p, int o, int lane) {
    if (lane == 0) p.hit_bin[atomicAdd(p.counters + C_FB_PENDING, 1)] = o;
}

__device__ __forceinline__ void add_alive(const Params &p, int v) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(p.counters + C_ALIVE_CELLS, v);
}

// Small warps: take chunks of 32 consecutive binned hits from a queue, load
// their cell counts together, work through those with 1..M cells and list
// the ones with more: up to kFbMidMax cells from the front of the list
// array, more from its back.
constexpr int kFbSmallMax = 192;
constexpr int kFbMidMax = 320;

template <int W, int M, int NB, int kMinBlocks>
__global__ void __launch_bounds__(32 * W, kMinBlocks) k_fishbone_small(Params p, float unit_thr, float du) {
    __shared__ FbSmem<W, M, NB, true> sm;
    if (upstream_overflow(p, PT_FLAG_CELLS)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    int my_alive = 0;
    const int n_binned = p.bin_cnt[p.n_bins];
    const int n_chunks = (n_binned + 31) >> 5;
    for (;;) {
        int ch = 0;
        if (lane == 0) ch = atomicAdd(p.counters + C_FB_NEXT, 1);
        ch = __shfl_sync(0xffffffffu, ch, 0);
        if (ch >= n_chunks) break;
        const int ol = (ch << 5) + lane;
        int nl = 0, bl = 0;
        if (ol < n_binned) {
            nl = p.in_cnt[ol];
            bl = p.in_off[ol];
        }
        const bool ok = nl >= 1 && (int64_t)bl + nl <= p.cap_cells;
        const unsigned mid = __ballot_sync(0xffffffffu, ok && nl > M && nl <= kFbMidMax);
        const unsigned huge = __ballot_sync(0xffffffffu, ok && nl > kFbMidMax);
        if (mid | huge) {
            int bm = 0, bh = 0;
            if (lane == 0) {
                if (mid) bm = atomicAdd(p.counters + C_FB_BIG, __popc(mid));
                if (huge) bh = atomicAdd(p.counters + C_FB_HUGE, __popc(huge));
            }
            bm = __shfl_sync(0xffffffffu, bm, 0);
            bh = __shfl_sync(0xffffffffu, bh, 0);
            if ((mid >> lane) & 1) p.fb_big[bm + __popc(mid & below)] = ol;
            if ((huge >> lane) & 1) p.fb_big[p.n_hits - 1 - (bh + __popc(huge & below))] = ol;
        }
        unsigned todo = __ballot_sync(0xffffffffu, ok && nl <= M);
        while (todo) {
            const int t = __ffs(todo) - 1;
            todo &= todo - 1;
            const int n = __shfl_sync(0xffffffffu, nl, t);
            const int b = __shfl_sync(0xffffffffu, bl, t);
            const int a = fishbone_hit<W, M, NB, false, false, true>(p, (ch << 5) + t, n, b, lane, w, unit_thr, du,
                                                                     sm);
            if (a >= 0) my_alive += a;
            else list_pending(p, (ch << 5) + t, lane);
        }
    }
    add_alive(p, my_alive);
}

// Larger warps: the listed outer hits, one at a time from a queue (kFromBack:
// the list at the back of the array).
template <int W, int M, int NB, bool kFromBack, bool C>
__global__ void __launch_bounds__(32 * W) k_fishbone_large(Params p, float unit_thr, float du) {
    __shared__ FbSmem<W, M, NB, C> sm;
    if (upstream_overflow(p, PT_FLAG_CELLS)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int my_alive = 0;
    const int n_list = p.counters[kFromBack ? C_FB_HUGE : C_FB_BIG];
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(p.counters + (kFromBack ? C_FB_HUGE_NEXT : C_FB_BIG_NEXT), 1);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= n_list) break;
        const int o = p.fb_big[kFromBack ? p.n_hits - 1 - k : k];
        const int a = fishbone_hit<W, M, NB, false, false, C>(p, o, p.in_cnt[o], p.in_off[o], lane, w, unit_thr, du,
                                                              sm);
        if (a >= 0) my_alive += a;
        else list_pending(p, o, lane);
    }
    add_alive(p, my_alive);
}

// Exact pass: the outer hits listed by the kernels above (an undecided
// alignment test, or more cells than a large warp holds), with the exact
// predicate and the pairwise loop for any number of cells.
template <int W, int M, int NB>
__global__ void __launch_bounds__(32 * W) k_fishbone_exact(Params p, float unit_thr, float du) {
    __shared__ FbSmem<W, M, NB, true> sm;
    if (upstream_overflow(p, PT_FLAG_CELLS)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int my_alive = 0;
    const int n_list = p.counters[C_FB_PENDING];
    for (int k = blockIdx.x * W + w; k < n_list; k += gridDim.x * W) {
        const int o = p.hit_bin[k];
        my_alive += fishbone_hit<W, M, NB, true, true, true>(p, o, p.in_cnt[o], p.in_off[o], lane, w, unit_thr, du, sm);
    }
    add_alive(p, my_alive);
}

void launch_fishbone(const Params &p, float unit_thr, float du, int grid, cudaStream_t s) {
    {
        KernelTimer t("k_fishbone_small", s);
        k_fishbone_small<8, kFbSmallMax, 256, 4><<<grid, 256, 0, s>>>(p, unit_thr, du);
    }
    {
        KernelTimer t("k_fishbone_medium", s);
        k_fishbone_large<4, kFbMidMax, 512, false, false><<<grid, 128, 0, s>>>(p, unit_thr, du);
    }
    {
        KernelTimer t("k_fishbone_large", s);
        k_fishbone_large<2, 512, 1024, true, true><<<grid / 4 + 1, 64, 0, s>>>(p, unit_thr, du);
    }
    KernelTimer t("k_fishbone_exact", s);
    k_fishbone_exact<2, 512, 1024><<<grid / 8 + 1, 64, 0, s>>>(p, unit_thr, du);
}

}  // namespace ptk
