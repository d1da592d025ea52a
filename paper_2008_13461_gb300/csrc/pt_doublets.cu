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
    const float xo = p.bx[o], yo = p.by[o], zo = p.bz[o], ro = p.br[o];
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
                    const float xi = p.bx[i], yi = p.by[i], zi = p.bz[i], ri = p.br[i];
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
// or as long with a smaller input index.  A cheap conservative test on unit
// direction vectors (|u^ - v^|^2 <= fb_unit_thr, implied by alignment) skips
// most sibling pairs before the exact predicate.
template <int G>
__global__ void __launch_bounds__(kThreads) k_fishbone(Params p, float unit_thr) {
    constexpr int kGroups = kThreads / G;
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int n_binned = p.bin_cnt[p.n_bins];
    for (int o = blockIdx.x * kGroups + grp; o < n_binned; o += gridDim.x * kGroups) {
        const int n = p.in_cnt[o];
        const int64_t b = p.in_off[o];
        if (n < 2 || b + n > p.cap_cells) continue;
        const FHit h = {p.bx[o], p.by[o], p.bz[o], p.br[o]};
        const GHit gh = ghit(h.x, h.y, h.z, h.r);
        for (int64_t c = b + lane; c < b + n; c += G) {
            const int i1 = p.cell_inner[c];
            const int L1 = p.blayer[i1];
            const FHit h1 = {p.bx[i1], p.by[i1], p.bz[i1], p.br[i1]};
            const float ux = h1.x - h.x, uy = h1.y - h.y, uz = h1.z - h.z;
            const float iu = rsqrtf(ux * ux + uy * uy + uz * uz);
            const float ax = ux * iu, ay = uy * iu, az = uz * iu;
            const GHit g1 = ghit(h1.x, h1.y, h1.z, h1.r);
            const long long l1 = (g1.x - gh.x) * (g1.x - gh.x) + (g1.y - gh.y) * (g1.y - gh.y) +
                                 (g1.z - gh.z) * (g1.z - gh.z);
            bool dead = false;
            for (int64_t d = b; d < b + n && !dead; d++) {
                if (d == c) continue;
                const int i2 = p.cell_inner[d];
                if (p.blayer[i2] != L1) continue;
                const FHit h2 = {p.bx[i2], p.by[i2], p.bz[i2], p.br[i2]};
                const float vx = h2.x - h.x, vy = h2.y - h.y, vz = h2.z - h.z;
                const float iv = rsqrtf(vx * vx + vy * vy + vz * vz);
                const float dx = ax - vx * iv, dy = ay - vy * iv, dz = az - vz * iv;
                if (dx * dx + dy * dy + dz * dz > unit_thr) continue;
                if (!pred_fb(h1, h2, h, p.fishbone_eps2, p.counters)) continue;
                const GHit g2 = ghit(h2.x, h2.y, h2.z, h2.r);
                const long long l2 = (g2.x - gh.x) * (g2.x - gh.x) + (g2.y - gh.y) * (g2.y - gh.y) +
                                     (g2.z - gh.z) * (g2.z - gh.z);
                if (l2 < l1 || (l2 == l1 && p.perm[i2] < p.perm[i1])) dead = true;
            }
            if (dead) p.cell_alive[c] = 0;
        }
    }
}

void launch_doublets(const Params &p, int lanes, int grid, cudaStream_t s) {
    switch (lanes) {
    case 4: k_doublets<4><<<grid, kThreads, 0, s>>>(p); break;
    case 8: k_doublets<8><<<grid, kThreads, 0, s>>>(p); break;
    case 16: k_doublets<16><<<grid, kThreads, 0, s>>>(p); break;
    default: k_doublets<32><<<grid, kThreads, 0, s>>>(p); break;
    }
}

void launch_fishbone(const Params &p, float unit_thr, int grid, cudaStream_t s) {
    k_fishbone<8><<<grid, kThreads, 0, s>>>(p, unit_thr);
}

}  // namespace ptk
