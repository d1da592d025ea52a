// Steps a1 + a2: doublets on layer pairs (Sec. 3.2, cuts of Table 1) and the
// Fishbone (Sec. 3.3).
//
// Doublets: a group of G lanes owns one outer hit (persistent grid-stride
// over the binned hits).  For every layer pair ending on the outer hit's
// layer it derives the phi window (PhiW) and a conservative window along z
// (barrel) or r (disk) from ZIP and ZW, widened by one tile on each side, and
// sweeps the inner tiles row by row: consecutive lanes load consecutive
// binned hits (coalesced), evaluate ZW, ZIP, PhiW, PT exactly, and compact
// the accepted ones with a ballot into a shared-memory buffer.  The cells of
// one outer hit are written contiguously, so the cells sharing an outer hit
// (needed by the Fishbone and the CA connection) form one range.
#include "pt_common.cuh"
#include "pt_kernels.cuh"

namespace ptk {

constexpr float kTwoPiInv = 0.159154943f;
constexpr float kPi = 3.14159265f;

// Conservative window of the inner hit's t coordinate for a pair, from ZIP
// (z-intercept within +-zmax) and ZW, over the inner layer's envelope.
__device__ __forceinline__ void t_window(const Params &p, const pt_pair_cuts &pc, float ro, float zo,
                                         float &tlo, float &thi) {
    const pt_layer li = p.layer[pc.inner];
    const float zm = pc.zmax;
    if (li.kind == PT_LAYER_BARREL) {
        float f0 = li.rmin / ro, f1 = li.rmax / ro;
        float c0 = -zm + (zo + zm) * f0, c1 = -zm + (zo + zm) * f1;
        float c2 = zm + (zo - zm) * f0, c3 = zm + (zo - zm) * f1;
        tlo = fmaxf(fminf(fminf(c0, c1), fminf(c2, c3)), pc.zlo);
        thi = fminf(fmaxf(fmaxf(c0, c1), fmaxf(c2, c3)), pc.zhi);
        if (tlo > thi) tlo = thi = 0.5f * (tlo + thi);
    } else {
        float za = fmaxf(li.zmin, pc.zlo), zb = fminf(li.zmax, pc.zhi);
        if (fabsf(zo) > zm * 1.001f + 0.01f && za <= zb) {
            float d0 = zo + zm, d1 = zo - zm;   // same sign
            float c0 = ro * (za + zm) / d0, c1 = ro * (zb + zm) / d0;
            float c2 = ro * (za - zm) / d1, c3 = ro * (zb - zm) / d1;
            tlo = fminf(fminf(c0, c1), fminf(c2, c3));
            thi = fminf(fmaxf(fmaxf(c0, c1), fmaxf(c2, c3)), ro);
            if (tlo > thi) tlo = thi = 0.5f * (tlo + thi);
        } else {
            tlo = li.rmin;
            thi = li.rmax;
        }
    }
}

// Sweep all candidate inner hits of outer hit o.  kWrite = false: fill the
// group's shared buffer (up to cap entries) and count; kWrite = true: write
// cells directly at global index base + slot.
template <int G, bool kWrite>
__device__ int sweep_outer(const Params &p, int o, int lane, unsigned gmask, int gshift, int32_t *s_inner,
                           uint8_t *s_pair, int cap, int64_t base) {
    const float4 ho = __ldg(p.bh + o);
    const float xo = ho.x, yo = ho.y, zo = ho.z, ro = ho.w;
    const int Lo = p.blayer[o], ev = p.bev[o];
    const float phio = atan2f(yo, xo);
    const unsigned lanes = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
    const unsigned below = (1u << lane) - 1u;
    int count = 0;
    const int npo = p.n_pairs_by_outer[Lo];
    for (int k = 0; k < npo; k++) {
        const int pi = p.pairs_by_outer[Lo][k];
        const pt_pair_cuts pc = p.pair[pi];
        float tlo, thi;
        t_window(p, pc, ro, zo, tlo, thi);
        const pt_layer li = p.layer[pc.inner];
        const float tmin = li.kind == PT_LAYER_BARREL ? li.zmin : li.rmin;
        const float tmax = li.kind == PT_LAYER_BARREL ? li.zmax : li.rmax;
        const int tb0 = max(t_tile(tlo, tmin, tmax, p.n_t) - 1, 0);
        const int tb1 = min(t_tile(thi, tmin, tmax, p.n_t) + 1, p.n_t - 1);
        const float dphi = p.pair_dphi[pi];
        int f0 = __float2int_rd((phio - dphi + kPi) * (p.n_phi * kTwoPiInv)) - 1;
        int f1 = __float2int_rd((phio + dphi + kPi) * (p.n_phi * kTwoPiInv)) + 1;
        if (f1 - f0 + 1 >= p.n_phi) {
            f0 = 0;
            f1 = p.n_phi - 1;
        }
        const int row0 = (ev * PT_N_LAYERS + pc.inner) * p.n_phi;
        for (int f = f0; f <= f1; f++) {
            const int fb = ((f % p.n_phi) + p.n_phi) % p.n_phi;
            const int tile = (row0 + fb) * p.n_t;
            const int beg = p.bin_cnt[tile + tb0], end = p.bin_cnt[tile + tb1 + 1];
            for (int i0 = beg; i0 < end; i0 += G) {
                const int i = i0 + lane;
                bool acc = false;
                if (i < end) {
                    const float4 hi = __ldg(p.bh + i);
                    const float xi = hi.x, yi = hi.y, zi = hi.z, ri = hi.w;
                    acc = zi >= pc.zlo && zi <= pc.zhi &&
                          pred_zip(xi, yi, zi, ri, xo, yo, zo, ro, pc.zmax, p.counters) &&
                          pred_phiw(xi, yi, xo, yo, pc.tan2_dphi, p.counters, zi, ri, zo, ro) &&
                          pred_pt(xi, yi, zi, ri, xo, yo, zo, ro, pc.k_pt, p.counters);
                }
                const unsigned m = (__ballot_sync(gmask, acc) >> gshift) & lanes;
                if (acc) {
                    const int slot = count + __popc(m & below);
                    if (kWrite) {
                        const int64_t c = base + slot;
                        if (c < p.cap_cells) {
                            p.cell_inner[c] = i;
                            p.cell_outer[c] = o;
                            p.cell_pair[c] = (uint8_t)pi;
                            p.cell_alive[c] = 1;
                            p.has_out[c] = 0;
                        }
                    } else if (slot < cap) {
                        s_inner[slot] = i;
                        s_pair[slot] = (uint8_t)pi;
                    }
                }
                count += __popc(m);
            }
        }
    }
    return count;
}

template <int G>
__global__ void __launch_bounds__(kThreads) k_doublets(Params p) {
    constexpr int kGroups = kThreads / G;
    constexpr int kBuf = 32 * G;   // 40 KB of shared memory per block for every G
    __shared__ int32_t s_inner[kGroups][kBuf];
    __shared__ uint8_t s_pair[kGroups][kBuf];
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int gshift = (threadIdx.x & 31) & ~(G - 1);
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << gshift);
    const int n_binned = p.bin_cnt[p.n_bins];
    for (int o = blockIdx.x * kGroups + grp; o < n_binned; o += gridDim.x * kGroups) {
        const int n = sweep_outer<G, false>(p, o, lane, gmask, gshift, s_inner[grp], s_pair[grp], kBuf, 0);
        int64_t base = 0;
        if (lane == 0 && n > 0) base = atomicAdd(p.counters + C_CELLS, n);
        base = __shfl_sync(gmask, base, gshift);
        if (n <= kBuf) {
            __syncwarp(gmask);
            for (int k = lane; k < n; k += G) {
                const int64_t c = base + k;
                if (c < p.cap_cells) {
                    p.cell_inner[c] = s_inner[grp][k];
                    p.cell_outer[c] = o;
                    p.cell_pair[c] = s_pair[grp][k];
                    p.cell_alive[c] = 1;
                    p.has_out[c] = 0;
                }
            }
        } else {
            sweep_outer<G, true>(p, o, lane, gmask, gshift, nullptr, nullptr, 0, base);
        }
        if (lane == 0) {
            p.in_off[o] = (int32_t)base;
            p.in_cnt[o] = n;
            if (base + n > p.cap_cells) set_flag(p.counters, PT_FLAG_CELLS);
        }
        __syncwarp(gmask);
    }
}

// Fishbone: cells sharing the outer hit o whose inner hits lie on one layer
// and are aligned; a cell dies when an aligned sibling is strictly shorter,
// or as long with a smaller input index.
//
// One warp per outer hit.  Alignment within eps implies that the unit
// directions u^ = (h_i - h_o)/|h_i - h_o| of two siblings differ by at most
// du = eps pi/2 (plus float32 slack), hence so does any 1-Lipschitz key of
// them (u^_z for a barrel outer hit, the radial component for a disk).  The
// siblings are counting-sorted into key buckets of width >= du in shared
// memory and each cell is compared only with the cells of its own and the two
// neighbouring buckets -- a superset of its aligned siblings -- so the result
// is exact while the work drops from O(k^2) to ~O(k).  Outer hits with more
// than kFbMax cells use the plain pairwise loop.
constexpr int kFbWarps = 4;
constexpr int kFbMax = 512;
constexpr int kFbBuckets = 512;
constexpr int kFbDirect = 12;      // below this many siblings compare all pairs

__device__ __forceinline__ bool fb_shorter_sibling(const Params &p, int i1, int i2, const FHit &h, const GHit &gh,
                                                   long long l1) {
    const FHit h1 = load_hit(p.bh, i1);
    const FHit h2 = load_hit(p.bh, i2);
    if (!pred_fb(h1, h2, h, p.fishbone_eps2, p.counters)) return false;
    const GHit g2 = ghit(h2.x, h2.y, h2.z, h2.r);
    const long long l2 =
        (g2.x - gh.x) * (g2.x - gh.x) + (g2.y - gh.y) * (g2.y - gh.y) + (g2.z - gh.z) * (g2.z - gh.z);
    return l2 < l1 || (l2 == l1 && p.perm[i2] < p.perm[i1]);
}

__device__ __forceinline__ long long len2_to(const Params &p, int i, const GHit &gh) {
    const FHit f = load_hit(p.bh, i);
    const GHit g = ghit(f.x, f.y, f.z, f.r);
    return (g.x - gh.x) * (g.x - gh.x) + (g.y - gh.y) * (g.y - gh.y) + (g.z - gh.z) * (g.z - gh.z);
}

// Fishbone verdicts for the n >= 2 cells of outer hit o (one warp).
__device__ __forceinline__ void fishbone_hit(const Params &p, int o, int n, int64_t b, int lane, int w,
                                          float unit_thr, float du, float (*s_ux)[kFbMax],
                                          float (*s_uy)[kFbMax], float (*s_uz)[kFbMax],
                                          int8_t (*s_lay)[kFbMax], int16_t (*s_sorted)[kFbMax],
                                          int (*s_pos)[kFbBuckets]) {
    {
        const FHit h = load_hit(p.bh, o);
        const GHit gh = ghit(h.x, h.y, h.z, h.r);
        if (n > kFbMax) {
            for (int j = lane; j < n; j += 32) {
                const int i1 = p.cell_inner[b + j];
                const int L1 = p.blayer[i1];
                const long long l1 = len2_to(p, i1, gh);
                bool dead = false;
                for (int d = 0; d < n && !dead; d++) {
                    if (d == j) continue;
                    const int i2 = p.cell_inner[b + d];
                    if (p.blayer[i2] != L1) continue;
                    dead = fb_shorter_sibling(p, i1, i2, h, gh, l1);
                }
                if (dead) p.cell_alive[b + j] = 0;
            }
            return;
        }
        const bool radial = p.layer[p.blayer[o]].kind == PT_LAYER_DISK;
        const float irr = rsqrtf(h.x * h.x + h.y * h.y);
        const float rx = h.x * irr, ry = h.y * irr;
        float kmin = 3.0f, kmax = -3.0f;
        for (int j = lane; j < n; j += 32) {
            const int i = p.cell_inner[b + j];
            const FHit hi = load_hit(p.bh, i);
            const float ux = hi.x - h.x, uy = hi.y - h.y, uz = hi.z - h.z;
            const float iu = rsqrtf(ux * ux + uy * uy + uz * uz);
            const float ax = ux * iu, ay = uy * iu, az = uz * iu;
            s_ux[w][j] = ax;
            s_uy[w][j] = ay;
            s_uz[w][j] = az;
            s_lay[w][j] = p.blayer[i];
            const float key = radial ? ax * rx + ay * ry : az;
            kmin = fminf(kmin, key);
            kmax = fmaxf(kmax, key);
        }
        __syncwarp();
        if (n <= kFbDirect) {
            // few siblings: compare every pair directly
            for (int j = lane; j < n; j += 32) {
                const float ax = s_ux[w][j], ay = s_uy[w][j], az = s_uz[w][j];
                const int L1 = s_lay[w][j];
                const int i1 = p.cell_inner[b + j];
                long long l1 = -1;
                bool dead = false;
                for (int d = 0; d < n && !dead; d++) {
                    if (d == j || s_lay[w][d] != L1) continue;
                    const float dx = ax - s_ux[w][d], dy = ay - s_uy[w][d], dz = az - s_uz[w][d];
                    if (dx * dx + dy * dy + dz * dz > unit_thr) continue;
                    if (l1 < 0) l1 = len2_to(p, i1, gh);
                    dead = fb_shorter_sibling(p, i1, p.cell_inner[b + d], h, gh, l1);
                }
                if (dead) p.cell_alive[b + j] = 0;
            }
            __syncwarp();
            return;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            kmin = fminf(kmin, __shfl_xor_sync(0xffffffffu, kmin, d));
            kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, d));
        }
        // as many buckets as about twice the cells (a power of two, 32 .. max)
        const int nb = min(kFbBuckets, max(32, 1 << (32 - __clz(2 * n - 1))));
        const float width = fmaxf(du, (kmax - kmin) / (float)(nb - 2));
        const float iw = 1.0f / width;
        for (int q = lane; q < nb; q += 32) s_pos[w][q] = 0;
        __syncwarp();
        for (int j = lane; j < n; j += 32) {
            const float key = radial ? s_ux[w][j] * rx + s_uy[w][j] * ry : s_uz[w][j];
            const int bk = min(__float2int_rd((key - kmin) * iw), nb - 1);
            atomicAdd(&s_pos[w][bk], 1);
        }
        __syncwarp();
        {   // exclusive scan of the bucket counts, nb / 32 buckets per lane
            const int per = nb >> 5;
            int sum = 0;
            for (int q = 0; q < per; q++) sum += s_pos[w][lane * per + q];
            int incl = sum;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += t;
            }
            int run = incl - sum;
            for (int q = 0; q < per; q++) {
                const int v = s_pos[w][lane * per + q];
                s_pos[w][lane * per + q] = run;
                run += v;
            }
        }
        __syncwarp();
        for (int j = lane; j < n; j += 32) {
            const float key = radial ? s_ux[w][j] * rx + s_uy[w][j] * ry : s_uz[w][j];
            const int bk = min(__float2int_rd((key - kmin) * iw), nb - 1);
            s_sorted[w][atomicAdd(&s_pos[w][bk], 1)] = (int16_t)j;
        }
        __syncwarp();
        // s_pos[bk] is now the end of bucket bk
        for (int j = lane; j < n; j += 32) {
            const float ax = s_ux[w][j], ay = s_uy[w][j], az = s_uz[w][j];
            const float key = radial ? ax * rx + ay * ry : az;
            const int bk = min(__float2int_rd((key - kmin) * iw), nb - 1);
            const int start = bk >= 2 ? s_pos[w][bk - 2] : 0;
            const int end = s_pos[w][min(bk + 1, nb - 1)];
            const int L1 = s_lay[w][j];
            const int i1 = p.cell_inner[b + j];
            long long l1 = -1;
            bool dead = false;
            for (int q = start; q < end && !dead; q++) {
                const int d = s_sorted[w][q];
                if (d == j || s_lay[w][d] != L1) continue;
                const float dx = ax - s_ux[w][d], dy = ay - s_uy[w][d], dz = az - s_uz[w][d];
                if (dx * dx + dy * dy + dz * dz > unit_thr) continue;
                if (l1 < 0) l1 = len2_to(p, i1, gh);
                dead = fb_shorter_sibling(p, i1, p.cell_inner[b + d], h, gh, l1);
            }
            if (dead) p.cell_alive[b + j] = 0;
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(32 * kFbWarps) k_fishbone(Params p, float unit_thr, float du) {
    __shared__ float s_ux[kFbWarps][kFbMax], s_uy[kFbWarps][kFbMax], s_uz[kFbWarps][kFbMax];
    __shared__ int8_t s_lay[kFbWarps][kFbMax];
    __shared__ int16_t s_sorted[kFbWarps][kFbMax];
    __shared__ int s_pos[kFbWarps][kFbBuckets];
    __shared__ int s_alive;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_alive = 0;
    __syncthreads();
    int my_alive = 0;
    const int n_binned = p.bin_cnt[p.n_bins];
    for (int o = blockIdx.x * kFbWarps + w; o < n_binned; o += gridDim.x * kFbWarps) {
        const int n = p.in_cnt[o];
        const int64_t b = p.in_off[o];
        if (n < 1 || b + n > p.cap_cells) continue;
        if (n >= 2) fishbone_hit(p, o, n, b, lane, w, unit_thr, du, s_ux, s_uy, s_uz, s_lay, s_sorted, s_pos);
        // R-z slope keys of the cells ending on o, for the CA connection:
        // barrel o: (z_o - z_a)/(r_o - r_a); disk o: (r_o - r_a)/(z_o - z_a);
        // NaN for dead cells.  Per hit: max sqrt(1 + key^2) and min gap.
        const float4 ho = __ldg(p.bh + o);
        const bool disk = p.layer[p.blayer[o]].kind == PT_LAYER_DISK;
        float kmax = 0.f, gmin = 3.0e38f;
        for (int j = lane; j < n; j += 32) {
            float key = __int_as_float(0x7fc00000);
            if (p.cell_alive[b + j]) {
                const float4 ha = __ldg(p.bh + p.cell_inner[b + j]);
                const float dr = ho.w - ha.w, dz = ho.z - ha.z;
                const float num = disk ? dr : dz, den = disk ? dz : dr;
                key = den != 0.f ? num / den : __int_as_float(0x7f800000);
                kmax = fmaxf(kmax, sqrtf(1.0f + key * key));
                gmin = fminf(gmin, fabsf(den));
                my_alive++;
                // join the out-list of the inner hit (rank by atomics)
                p.cell_rank[b + j] = atomicAdd(p.out_off + p.cell_inner[b + j], 1);
            }
            p.ck[b + j] = key;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            kmax = fmaxf(kmax, __shfl_xor_sync(0xffffffffu, kmax, d));
            gmin = fminf(gmin, __shfl_xor_sync(0xffffffffu, gmin, d));
        }
        if (lane == 0) p.hk[o] = make_float2(kmax, gmin);
    }
    if (my_alive) atomicAdd(&s_alive, my_alive);
    __syncthreads();
    if (threadIdx.x == 0 && s_alive) atomicAdd(p.counters + C_ALIVE_CELLS, s_alive);
}

// Out-lists: live cells grouped by their inner hit (CSR), from the ranks
// taken in the Fishbone kernel and the scanned per-hit counts.
__global__ void __launch_bounds__(kThreads) k_out_fill(Params p) {
    const int64_t n_cells = min((int64_t)p.counters[C_CELLS], p.cap_cells);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += stride) {
        if (!p.cell_alive[c]) continue;
        const int i = p.cell_inner[c];
        p.out_idx[p.out_off[i] + p.cell_rank[c]] = (int32_t)c;
    }
}

void launch_out_lists(const Params &p, int grid, cudaStream_t s) {
    launch_scan(p.out_off, p.n_hits, p.scan_part, s);
    k_out_fill<<<grid, kThreads, 0, s>>>(p);
}

void launch_doublets(const Params &p, int lanes, int grid, cudaStream_t s) {
    switch (lanes) {
    case 4: k_doublets<4><<<grid, kThreads, 0, s>>>(p); break;
    case 8: k_doublets<8><<<grid, kThreads, 0, s>>>(p); break;
    case 16: k_doublets<16><<<grid, kThreads, 0, s>>>(p); break;
    default: k_doublets<32><<<grid, kThreads, 0, s>>>(p); break;
    }
}

void launch_fishbone(const Params &p, float unit_thr, float du, int grid, cudaStream_t s) {
    k_fishbone<<<grid * (kThreads / (32 * kFbWarps)), 32 * kFbWarps, 0, s>>>(p, unit_thr, du);
}

}  // namespace ptk
