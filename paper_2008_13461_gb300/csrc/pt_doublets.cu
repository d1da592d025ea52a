// Step a1: doublets on layer pairs (Sec. 3.2, cuts of Table 1).
//
// Doublets: a group of G lanes owns one outer hit (the warps take the binned
// hits from a queue, in order).  For every layer pair ending on the outer
// hit's layer it derives the phi window (PhiW) and a conservative window
// along z (barrel) or r (disk) from ZIP and ZW, with margins above float32
// rounding, and sweeps the inner tiles' rows of that window laid end to end:
// consecutive lanes load consecutive binned hits (coalesced), evaluate ZW,
// ZIP, PhiW, PT exactly, and compact the accepted ones with a ballot into a
// shared-memory buffer.  The cells of one outer hit are written
// contiguously, so the cells sharing an outer hit (needed by the Fishbone
// and the CA connection) form one range.
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
// cells directly at global index base + slot.  kExact = false: the
// predicates are float32 filters only, and *undecided is set on the lanes
// that met a candidate they cannot decide.  s_cand (or null): per-pair
// counts of the candidate inner hits tested, summed in shared memory.
template <int G, bool kWrite, bool kExact>
__device__ int sweep_outer(const Params &p, int o, int lane, unsigned gmask, int gshift, int32_t *s_inner,
                           uint8_t *s_pair, int32_t *s_row, int cap, int64_t base, bool *undecided,
                           unsigned long long *s_cand = nullptr) {
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
        // Tile ranges: the t window's float32 bounds are within ~1e-5 cm of
        // the exact ones, so a margin of 1e-4 cm keeps every accepted hit
        // inside; the half-width in phi already carries a 1e-4 rad margin
        // over PhiW's exact bound, far above the rounding of the angles.
        // Tile indices are monotone in t and phi (the binning uses the
        // same functions), so the tiles cover a superset of the accepted
        // hits whatever the tile counts.
        const float mt = 1e-4f + 1e-6f * fmaxf(fabsf(tlo), fabsf(thi));
        const int tb0 = t_tile(tlo - mt, tmin, tmax, p.n_t);
        const int tb1 = t_tile(thi + mt, tmin, tmax, p.n_t);
        // The PT cut (circumradius of beam line, inner and outer hit >= R)
        // accepts an azimuth difference up to |asin(r_o / 2R) - asin(r_i / 2R)|
        // or from pi - asin(r_o / 2R) - asin(r_i / 2R) on (both radii below
        // 2R: on a circle through the beam line a chord of length r makes
        // the angle asin(r / 2R) with the tangent there).  While the second
        // range lies beyond the pair's PhiW window, the first, taken over the
        // inner layer's radii with a margin far above the rounding of the
        // float32 arcsines, narrows the window to this outer hit.
        float dphi = p.pair_dphi[pi];
        const float pa = p.pair_pt_a[pi];
        if (pa > 0.f && ro * pa < 1.f && li.rmax * pa < 1.f) {
            const float so = asinf(ro * pa), si = asinf(li.rmin * pa), sx = asinf(li.rmax * pa);
            if (kPi - so - sx > dphi + 1e-3f) dphi = fminf(dphi, fmaxf(so - si, sx - so) + 1e-4f);
        }
        int f0 = __float2int_rd((phio - dphi + kPi) * (p.n_phi * kTwoPiInv));
        int f1 = __float2int_rd((phio + dphi + kPi) * (p.n_phi * kTwoPiInv));
        if (f1 - f0 + 1 >= p.n_phi) {
            f0 = 0;
            f1 = p.n_phi - 1;
        }
        const int row0 = (ev * PT_N_LAYERS + pc.inner) * p.n_phi;
        const int nrows = f1 - f0 + 1;
        unsigned cand = 0;
        // The rows of the window are separate ranges of the binned hits,
        // about as long as a group is wide: G of them at a time are laid
        // end to end in one range of slots, so the lanes stay busy across
        // row ends.  s_row holds, per row, the offset from slot to binned
        // index and the row's end in slot space.
        for (int r0 = 0; r0 < nrows; r0 += G) {
            int beg = 0, len = 0;
            if (r0 + lane < nrows) {
                const int f = f0 + r0 + lane;
                const int fb = ((f % p.n_phi) + p.n_phi) % p.n_phi;
                const int tile = (row0 + fb) * p.n_t;
                beg = p.bin_cnt[tile + tb0];
                len = p.bin_cnt[tile + tb1 + 1] - beg;
            }
            int incl = len;
#pragma unroll
            for (int d = 1; d < G; d <<= 1) {
                const int t = __shfl_up_sync(gmask, incl, d, G);
                if (lane >= d) incl += t;
            }
            const int total = __shfl_sync(gmask, incl, G - 1, G);
            cand += (unsigned)total;
            if (total == 0) continue;
            __syncwarp(gmask);       // the previous rows' table is no longer read
            s_row[lane] = beg - (incl - len);
            s_row[G + lane] = incl;
            __syncwarp(gmask);
            for (int s0 = 0; s0 < total; s0 += G) {
                const int sl = s0 + lane;
                int v = 0;     // 1 accepted, 0 rejected, 2|3 undecided (kExact = false)
                int i = 0;
                if (sl < total) {
                    // the slot's row: the first whose end lies beyond it
                    int j = 0;
#pragma unroll
                    for (int h = G / 2; h > 0; h >>= 1)
                        if (s_row[G + j + h - 1] <= sl) j += h;
                    i = sl + s_row[j];
                    const float4 hi = __ldg(p.bh + i);
                    const float xi = hi.x, yi = hi.y, zi = hi.z, ri = hi.w;
                    if (zi >= pc.zlo && zi <= pc.zhi) {
                        v = pred_zip<kExact>(xi, yi, zi, ri, xo, yo, zo, ro, pc.zmax, p.counters);
                        if (v) {
                            const int v2 = pred_phiw<kExact>(xi, yi, xo, yo, pc.tan2_dphi, p.counters, zi, ri, zo, ro);
                            v = v2 ? (v | v2) : 0;
                        }
                        if (v) {
                            const int v3 = pred_pt<kExact>(xi, yi, zi, ri, xo, yo, zo, ro, pc.k_pt, p.counters);
                            v = v3 ? (v | v3) : 0;
                        }
                    }
                }
                const bool acc = v == 1;
                if (!kExact && v > 1) *undecided = true;
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
        if (s_cand && lane == 0 && cand) atomicAdd(s_cand + pi, (unsigned long long)cand);
    }
    return count;
}

// Cells of outer hit o (one group of G lanes).  kExact = false: returns
// false without writing anything when a candidate is undecided.
template <int G, bool kExact>
__device__ __forceinline__ bool doublets_hit(const Params &p, int o, int lane, unsigned gmask, int gshift,
                                             int32_t *s_inner, uint8_t *s_pair, int32_t *s_row, int cap,
                                             unsigned long long *s_cand = nullptr) {
    bool und = false;
    const int n = sweep_outer<G, false, kExact>(p, o, lane, gmask, gshift, s_inner, s_pair, s_row, cap, 0, &und,
                                                 s_cand);
    if (!kExact && __ballot_sync(gmask, und)) return false;
    int64_t base = 0;
    if (lane == 0 && n > 0) base = atomicAdd(p.counters + C_CELLS, n);
    base = __shfl_sync(gmask, base, gshift);
    if (n <= cap) {
        __syncwarp(gmask);
        for (int k = lane; k < n; k += G) {
            const int64_t c = base + k;
            if (c < p.cap_cells) {
                p.cell_inner[c] = s_inner[k];
                p.cell_outer[c] = o;
                p.cell_pair[c] = s_pair[k];
                p.cell_alive[c] = 1;
                p.has_out[c] = 0;
            }
        }
    } else {
        sweep_outer<G, true, kExact>(p, o, lane, gmask, gshift, nullptr, nullptr, s_row, 0, base, &und);
    }
    if (lane == 0) {
        p.in_off[o] = (int32_t)base;
        p.in_cnt[o] = n;
        if (base + n > p.cap_cells) set_flag(p.counters, PT_FLAG_CELLS);
    }
    __syncwarp(gmask);
    return true;
}

// Main pass: float32 filters only (no big-integer code, so far fewer
// registers); an outer hit with an undecided candidate (about one in 10^3)
// is listed for the exact pass.  It also counts the candidates tested per
// layer pair (the exact pass repeats a few of them and does not count).
template <int G>
__global__ void __launch_bounds__(kThreads, 5) k_doublets(Params p) {
    constexpr int kGroups = kThreads / G;
    constexpr int kBuf = 32 * G;   // 40 KB of shared memory per block for every G
    __shared__ int32_t s_inner[kGroups][kBuf];
    __shared__ uint8_t s_pair[kGroups][kBuf];
    __shared__ int32_t s_row[kGroups][2 * G];
    __shared__ unsigned long long s_cand[PT_MAX_PAIRS];
    if (threadIdx.x < PT_MAX_PAIRS) s_cand[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x % G, grp = threadIdx.x / G, wl = threadIdx.x & 31;
    const int gshift = wl & ~(G - 1);
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << gshift);
    const int n_binned = p.bin_cnt[p.n_bins];
    // the warps take the binned outer hits in order, 32 / G at a time: the
    // cells are laid out nearly in the order of their outer hits
    for (;;) {
        int o0 = 0;
        if (wl == 0) o0 = atomicAdd(p.counters + C_DB_NEXT, 32 / G);
        o0 = __shfl_sync(0xffffffffu, o0, 0);
        if (o0 >= n_binned) break;
        const int o = o0 + wl / G;
        if (o < n_binned &&
            !doublets_hit<G, false>(p, o, lane, gmask, gshift, s_inner[grp], s_pair[grp], s_row[grp], kBuf, s_cand) &&
            lane == 0) {
            // listed in hit_bin, free once the hits are binned (one slot per hit)
            p.hit_bin[atomicAdd(p.counters + C_DB_PENDING, 1)] = o;
        }
    }
    __syncthreads();
    if (threadIdx.x < p.n_pairs && s_cand[threadIdx.x])
        atomicAdd(reinterpret_cast<unsigned long long *>(p.counters + C_PAIR_CAND) + threadIdx.x, s_cand[threadIdx.x]);
}

// Exact pass over the listed outer hits (a few hundred): a warp per hit,
// the hits dealt round the blocks first, so that they spread over the SMs
// and no warp runs two hits' exact fallbacks one after the other.
__global__ void __launch_bounds__(kThreads) k_doublets_exact(Params p) {
    constexpr int G = 32, kGroups = kThreads / G, kBuf = 32 * G;
    __shared__ int32_t s_inner[kGroups][kBuf];
    __shared__ uint8_t s_pair[kGroups][kBuf];
    __shared__ int32_t s_row[kGroups][2 * G];
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int n = p.counters[C_DB_PENDING];
    for (int k = grp * gridDim.x + blockIdx.x; k < n; k += gridDim.x * kGroups)
        doublets_hit<G, true>(p, p.hit_bin[k], lane, 0xffffffffu, 0, s_inner[grp], s_pair[grp], s_row[grp], kBuf);
}

void launch_doublets(const Params &p, int lanes, int grid, cudaStream_t s) {
    {
        KernelTimer t("k_doublets", s);
        switch (lanes) {
        case 4: k_doublets<4><<<grid, kThreads, 0, s>>>(p); break;
        case 8: k_doublets<8><<<grid, kThreads, 0, s>>>(p); break;
        case 16: k_doublets<16><<<grid, kThreads, 0, s>>>(p); break;
        default: k_doublets<32><<<grid, kThreads, 0, s>>>(p); break;
        }
    }
    KernelTimer t("k_doublets_exact", s);
    k_doublets_exact<<<grid / 4 + 1, kThreads, 0, s>>>(p);
}

}  // namespace ptk
