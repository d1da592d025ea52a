// Pixel vertices (Sec. 3.6): clusters of tracks in z0, the z of each
// track's point of closest approach to the beam line.
//
// Tracks are eligible when kept by the ambiguity resolution, with at least
// min_hits hits, pT > pt_min, 0 < ez0 < ez0_max and a finite z0.  Two tracks
// i, j of an event are compatible when dz = z0_i - z0_j satisfies
// |dz| < dz_cut and dz^2 < chi2_max (ez0_i^2 + ez0_j^2).  A track's density
// rho is 1 + the number of tracks compatible with it; each track links to the
// nearest compatible track (smallest |dz|, then smaller z0, then smaller
// index) of higher rank (larger rho, or equal rho and smaller z0, or equal
// rho and z0 and smaller index: ties go by z0 first, so the result does not
// depend on the order of the tracks unless two share a z0); the links end at roots
// (ranks grow along them, so there are no cycles), and a root with rho > 1
// seeds a candidate made of every track whose links lead to it.  Candidates
// with at least min_tracks tracks become vertices: z the mean of z0 weighted
// by 1/ez0^2, ez = 1/sqrt(sum of weights), chi2 = sum w (z0 - z)^2, ndf =
// n - 1.  A vertex with chi2/ndf > split_chi2 is split by 2-means in z
// (centres from the tracks below / at-or-above z, each track to the nearer
// centre, ties to the lower one, until no assignment changes, at most 20
// rounds) when both parts keep min_tracks tracks.  The vertices of an event
// are ordered by the sum of pT^2 of their tracks, largest first.
//
// Cuts compare float32 values rounded as written (no contraction); sums and
// the vertex quantities are float64, converted to float32 on output.
//
// GPU form: a counting sort groups the eligible tracks by event; one block of
// 1024 threads per event then sorts its tracks by (z0, index) in shared
// memory (bitonic), so that every track's compatible tracks lie in a window
// around it; densities and links come from window scans (one thread per
// track), roots from pointer jumping, candidates from a second sort of
// (root, position) keys.  The candidates' fits and 2-means splits, the
// float64 part, then run one warp per candidate over the candidates of all
// events at once (shuffle reductions), so that every SM takes part; a last
// block per event orders its vertices and labels their tracks.
#include "pt_common.cuh"
#include "pt_kernels.cuh"

namespace ptk {
namespace {

constexpr int kVtxMax = PT_VTX_MAX_TRACKS;   // eligible tracks per event (sorted in shared memory)
constexpr int kPosBits = 14;                 // bits of a sorted position
constexpr int kPosMask = kVtxMax - 1;
constexpr int kSideBit = 30;                 // 2-means side of a member, kept in its key
constexpr int kVtxCap = PT_VTX_MAX_VERTICES; // vertex candidates / vertices per event
constexpr int kVtxThreads = 1024;
constexpr size_t kVtxDynSmem = 3 * sizeof(int32_t) * kVtxMax;
constexpr int kKmeansRounds = 20;
constexpr unsigned kFull = 0xffffffffu;

static_assert((1 << kPosBits) == kVtxMax, "sorted positions must fit their key field");

struct VtxArgs {
    int32_t n_tracks, n_events, max_vertices;
    pt_vertex_tracks in;
    pt_vertex_cuts cuts;
    // scratch; arrays "by sorted position" hold each event's tracks at its ev_off
    int32_t *ev_off, *ev_cur, *order, *rho, *root;
    double2 *wz;                     // (1 / ez0^2, z0) in float64 by sorted position
    int32_t *key;                    // (root, position) keys, grouped by root; the members of the candidates
    int32_t *sid;                    // track index by sorted position
    int32_t *nc, *nv;                // per event: candidates, provisional vertices
    int32_t *cq, *cn, *cv0, *cv1;    // per event and candidate (kVtxCap each): first key, members, its vertices
    double *vz, *vsp;                // per event and provisional vertex (kVtxCap each): z, sum of pT^2
    float *vez, *vc2;                //   its error and chi2
    int32_t *vnt, *vkey;             //   its tracks and (2 * first key + part)
    pt_vertices out;
};

__device__ __forceinline__ bool eligible(const VtxArgs &a, int i) {
    const float e = a.in.ez0[i], z = a.in.z0[i];
    const int ev = a.in.ev[i];
    return (!a.in.keep || a.in.keep[i]) && (int)a.in.nhits[i] >= a.cuts.min_hits && a.in.pt[i] > a.cuts.pt_min &&
           e > 0.f && e < a.cuts.ez0_max && fabsf(z) <= 3.402823466e38f && ev >= 0 && ev < a.n_events;
}

__device__ __forceinline__ void set_status(const VtxArgs &a, int bit) { atomicOr(a.out.status, bit); }

// Tracks of one event are mostly consecutive, so the per-event atomics are
// aggregated over the lanes of a warp that share an event.
__global__ void __launch_bounds__(kThreads) k_vtx_count(VtxArgs a) {
    const int lane = threadIdx.x & 31;
    for (int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < a.n_tracks; i0 += gridDim.x * blockDim.x) {
        const int i = i0 + lane;
        const bool ok = i < a.n_tracks && eligible(a, i);
        if (i < a.n_tracks) a.out.track_vertex[i] = -1;
        const int e = ok ? a.in.ev[i] : -1;
        const unsigned grp = __match_any_sync(kFull, e);
        if (ok && lane == __ffs(grp) - 1) atomicAdd(a.ev_off + e, __popc(grp));
    }
}

__global__ void __launch_bounds__(kThreads) k_vtx_fill(VtxArgs a) {
    const int lane = threadIdx.x & 31;
    for (int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < a.n_tracks; i0 += gridDim.x * blockDim.x) {
        const int i = i0 + lane;
        const bool ok = i < a.n_tracks && eligible(a, i);
        const int e = ok ? a.in.ev[i] : -1;
        const unsigned grp = __match_any_sync(kFull, e);
        const int leader = __ffs(grp) - 1;
        int slot = 0;
        if (ok && lane == leader) slot = atomicAdd(a.ev_cur + e, __popc(grp));
        slot = __shfl_sync(kFull, slot, leader) + __popc(grp & ((1u << lane) - 1u));
        if (ok) a.order[a.ev_off[e] + slot] = i;
    }
}

// the chi2 half of the compatibility of a track (squared error ep2) with a
// track of error eq at distance dz: dz^2 < chi2_max (ep2 + eq^2)
__device__ __forceinline__ bool chi2_ok(float dz, float ep2, float eq, float c2m) {
    return __fmul_rn(dz, dz) < __fmul_rn(c2m, __fadd_rn(ep2, __fmul_rn(eq, eq)));
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);    // every lane ends with the same bits
    return v;
}

__device__ __forceinline__ int warp_sum(int v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

struct WSums {
    double sw, swz;
    int n;
};

// Weighted sums over the members mk[0, n) of a candidate (one warp); sel < 0:
// every member, else those whose side bit equals sel.  wz: each track's
// weight 1/ez0^2 and z0 in float64 by sorted position, computed once per
// track (the float64 pipe is the slow one on this GPU, and a division, or a
// conversion to float64, costs many of its cycles).
__device__ __forceinline__ WSums member_sums(const int32_t *mk, int n, int sel, const double2 *wz) {
    double sw = 0.0, swz = 0.0;
    int c = 0;
    for (int k = threadIdx.x & 31; k < n; k += 32) {
        const int32_t kk = mk[k];
        if (sel >= 0 && ((kk >> kSideBit) & 1) != sel) continue;
        const double2 v = wz[kk & kPosMask];
        sw += v.x;
        swz += v.x * v.y;
        c++;
    }
    return WSums{warp_sum(sw), warp_sum(swz), warp_sum(c)};
}

__device__ __forceinline__ double member_chi2(const int32_t *mk, int n, int sel, double z, const double2 *wz) {
    double c = 0.0;
    for (int k = threadIdx.x & 31; k < n; k += 32) {
        const int32_t kk = mk[k];
        if (sel >= 0 && ((kk >> kSideBit) & 1) != sel) continue;
        const double2 v = wz[kk & kPosMask];
        const double d = v.y - z;
        c += v.x * d * d;
    }
    return warp_sum(c);
}

__device__ __forceinline__ double member_sumpt2(const VtxArgs &a, const int32_t *mk, int n, int sel,
                                                const int32_t *sid) {
    // (sid: the event's track index by sorted position)
    double s = 0.0;
    for (int k = threadIdx.x & 31; k < n; k += 32) {
        const int32_t kk = mk[k];
        if (sel >= 0 && ((kk >> kSideBit) & 1) != sel) continue;
        const double t = a.in.pt[sid[kk & kPosMask]];
        s += t * t;
    }
    return warp_sum(s);
}

// sort elements: (z0, track index) in order of both, or plain int keys
struct ZId {
    float z;
    int id;
};
__device__ __forceinline__ bool elem_gt(const ZId &a, const ZId &b) { return a.z > b.z || (a.z == b.z && a.id > b.id); }
__device__ __forceinline__ bool elem_gt(int a, int b) { return a > b; }
__device__ __forceinline__ ZId elem_shfl_xor(const ZId &e, int j) {
    return {__shfl_xor_sync(0xffffffffu, e.z, j), __shfl_xor_sync(0xffffffffu, e.id, j)};
}
__device__ __forceinline__ int elem_shfl_xor(int e, int j) { return __shfl_xor_sync(0xffffffffu, e, j); }

// Ascending bitonic sort of P entries (P a power of two, at least 32; the
// block a multiple of 32 threads).  Position p is handled by thread p mod
// blockDim, so the partners of the stages at distance 16 or less are lanes
// of one warp: those stages of each merge run in registers with shuffles,
// one barrier per merge instead of one per stage.
template <class E, class Load, class Store>
__device__ __forceinline__ void bitonic(int P, Load load, Store store) {
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j >= 32; j >>= 1) {
            for (int p = threadIdx.x; p < P; p += blockDim.x) {
                const int q = p ^ j;
                if (q > p) {
                    const E a = load(p), b = load(q);
                    if (elem_gt(a, b) == ((p & k) == 0)) {
                        store(p, b);
                        store(q, a);
                    }
                }
            }
            __syncthreads();
        }
        // whole warps take part: P and blockDim are multiples of 32
        for (int p = threadIdx.x; p < P; p += blockDim.x) {
            E e = load(p);
            const bool up = (p & k) == 0;
            for (int j = min(k >> 1, 16); j > 0; j >>= 1) {
                const E o = elem_shfl_xor(e, j);
                // the lower of a pair keeps the smaller entry in an ascending
                // run and the larger in a descending one
                if (((p & j) == 0) == up ? elem_gt(e, o) : elem_gt(o, e)) e = o;
            }
            store(p, e);
        }
        __syncthreads();
    }
}

// Per event: sort, densities, links, roots, candidates (one block).
__global__ void __launch_bounds__(kVtxThreads, 1) k_vtx_group(VtxArgs a) {
    extern __shared__ __align__(16) unsigned char vsm[];
    float *sz = reinterpret_cast<float *>(vsm);                   // z0 by sorted position
    int32_t *sid = reinterpret_cast<int32_t *>(sz + kVtxMax);     // track index by sorted position
    int32_t *key = sid + kVtxMax;                                 // root << kPosBits | position
    __shared__ int s_nc;

    const int e = blockIdx.x, tid = threadIdx.x;
    const int base = a.ev_off[e], cnt = a.ev_off[e + 1] - base;
    if (tid == 0) {
        a.nc[e] = 0;
        a.nv[e] = 0;
    }
    if (cnt > kVtxMax) {                                          // uniform over the block
        if (tid == 0) set_status(a, PT_VTX_EVENT_TOO_LARGE);
        return;
    }
    if (tid == 0) s_nc = 0;
    int P = 32;
    while (P < cnt) P <<= 1;
    for (int p = tid; p < P; p += blockDim.x) {
        if (p < cnt) {
            const int i = a.order[base + p];
            sz[p] = a.in.z0[i];
            sid[p] = i;
        } else {
            sz[p] = __int_as_float(0x7f800000);
            sid[p] = 0x7fffffff;
        }
    }
    __syncthreads();
    bitonic<ZId>(
        P, [&](int p) { return ZId{sz[p], sid[p]}; },
        [&](int p, const ZId &e) {
            sz[p] = e.z;
            sid[p] = e.id;
        });

    const float dzc = a.cuts.dz_cut, c2m = a.cuts.chi2_max;
    int32_t *rho = a.rho + base, *root = a.root + base;
    // the z0 errors by sorted position, in the key array until the keys are
    // built, and the weights 1/ez0^2 of the vertex fits
    float *sez = reinterpret_cast<float *>(key);
    double2 *wz = a.wz + base;
    for (int p = tid; p < cnt; p += blockDim.x) {
        const float ez = a.in.ez0[sid[p]];
        sez[p] = ez;
        const double e = ez;
        wz[p] = make_double2(1.0 / (e * e), (double)sz[p]);
        a.sid[base + p] = sid[p];
    }
    __syncthreads();
    // densities: the compatible tracks lie in the window |z0 - z0_p| < dz_cut
    // (rounded differences are monotonic along the sorted order)
    for (int p = tid; p < cnt; p += blockDim.x) {
        const float zp = sz[p], ep = sez[p], ep2 = __fmul_rn(ep, ep);
        int r = 1;
        for (int q = p - 1; q >= 0; q--) {
            const float dz = __fsub_rn(zp, sz[q]);
            if (!(fabsf(dz) < dzc)) break;
            r += chi2_ok(dz, ep2, sez[q], c2m);
        }
        for (int q = p + 1; q < cnt; q++) {
            const float dz = __fsub_rn(zp, sz[q]);
            if (!(fabsf(dz) < dzc)) break;
            r += chi2_ok(dz, ep2, sez[q], c2m);
        }
        rho[p] = r;
    }
    __syncthreads();
    // links to the nearest compatible track of higher rank; the sorted
    // position orders equal densities and equal distances by (z0, index)
    for (int p = tid; p < cnt; p += blockDim.x) {
        const float zp = sz[p];
        const int rp = rho[p];
        const float ep = sez[p], ep2 = __fmul_rn(ep, ep);
        int best = -1;
        float bd = 0.f;
        for (int dir = -1; dir <= 1; dir += 2)
            for (int q = p + dir; q >= 0 && q < cnt; q += dir) {
                const float dz = __fsub_rn(zp, sz[q]), ad = fabsf(dz);
                if (!(ad < dzc)) break;
                const int rq = rho[q];
                if (!(rq > rp || (rq == rp && q < p))) continue;
                if (!chi2_ok(dz, ep2, sez[q], c2m)) continue;
                if (best < 0 || ad < bd || (ad == bd && q < best)) {
                    best = q;
                    bd = ad;
                }
            }
        root[p] = best < 0 ? p : best;
    }
    __syncthreads();
    // roots by pointer jumping; a racing read sees an old or a new value, both
    // ancestors, so the iteration still converges (path lengths halve)
    bool done = false;
    for (int it = 0; it < 2 * kPosBits + 4 && !done; it++) {
        bool ch = false;
        for (int p = tid; p < cnt; p += blockDim.x) {
            const int r = root[p], rr = root[r];
            if (rr != r) {
                root[p] = rr;
                ch = true;
            }
        }
        done = !__syncthreads_or(ch);
    }
    if (!done) {                                                  // uniform over the block
        if (tid == 0) set_status(a, PT_VTX_INTERNAL);
        return;
    }
    // group the tracks by root: sort the (root, position) keys
    for (int p = tid; p < P; p += blockDim.x) key[p] = p < cnt ? (root[p] << kPosBits | p) : 0x7fffffff;
    __syncthreads();
    bitonic<int>(
        P, [&](int p) { return key[p]; }, [&](int p, int e) { key[p] = e; });
    // candidates: groups whose root has rho > 1 and at least min_tracks tracks
    for (int q = tid; q < cnt; q += blockDim.x) {
        const int r = key[q] >> kPosBits;
        if (q > 0 && (key[q - 1] >> kPosBits) == r) continue;
        int n = 1;
        while (q + n < cnt && (key[q + n] >> kPosBits) == r) n++;
        if (rho[r] > 1 && n >= a.cuts.min_tracks) {
            const int c = atomicAdd(&s_nc, 1);
            if (c < kVtxCap) {
                a.cq[e * kVtxCap + c] = q;
                a.cn[e * kVtxCap + c] = n;
            } else {
                set_status(a, PT_VTX_TOO_MANY);
            }
        }
    }
    for (int q = tid; q < cnt; q += blockDim.x) a.key[base + q] = key[q];
    __syncthreads();
    if (tid == 0) a.nc[e] = min(s_nc, kVtxCap);
}

// The candidates of all events, one warp each: fit, 2-means split,
// provisional vertices (grid: candidates / warps per block x events).
constexpr int kFitWarps = 8;

__global__ void __launch_bounds__(32 * kFitWarps) k_vtx_fit(VtxArgs a) {
    const int e = blockIdx.y, c = blockIdx.x * kFitWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= a.nc[e]) return;                                     // uniform over the warp
    const int base = a.ev_off[e];
    int32_t *key = a.key + base;
    const int32_t *sid = a.sid + base;
    const double2 *wz = a.wz + base;
    {
        const int q = a.cq[e * kVtxCap + c], n = a.cn[e * kVtxCap + c];
        int32_t *mk = key + q;
        const WSums all = member_sums(mk, n, -1, wz);
        const double z = all.swz / all.sw;
        const double chi2 = member_chi2(mk, n, -1, z, wz);
        bool split = false;
        if (n > 1 && chi2 / (double)(n - 1) > (double)a.cuts.split_chi2) {
            int hi = 0;
            for (int k = lane; k < n; k += 32) {
                const int32_t kk = mk[k];
                const int s = wz[kk & kPosMask].y >= z;
                mk[k] = (kk & ~(1 << kSideBit)) | (s << kSideBit);
                hi += s;
            }
            hi = warp_sum(hi);
            __syncwarp();
            if (hi > 0 && hi < n) {
                WSums s0 = member_sums(mk, n, 0, wz), s1 = member_sums(mk, n, 1, wz);
                double c0 = s0.swz / s0.sw, c1 = s1.swz / s1.sw;
                int up = 0;
                bool have = false;
                for (int round = 0; round < kKmeansRounds; round++) {
                    bool diff = false;
                    up = 0;
                    for (int k = lane; k < n; k += 32) {
                        const int32_t kk = mk[k];
                        const double zz = wz[kk & kPosMask].y;
                        const int u = fabs(zz - c1) < fabs(zz - c0);      // ties: the lower centre
                        diff |= u != ((kk >> kSideBit) & 1);
                        mk[k] = (kk & ~(1 << kSideBit)) | (u << kSideBit);
                        up += u;
                    }
                    up = warp_sum(up);
                    diff = __any_sync(kFull, diff);
                    __syncwarp();
                    if (have && !diff) break;
                    have = true;
                    if (up == 0 || up == n) break;
                    s0 = member_sums(mk, n, 0, wz);
                    s1 = member_sums(mk, n, 1, wz);
                    c0 = s0.swz / s0.sw;
                    c1 = s1.swz / s1.sw;
                }
                split = up >= a.cuts.min_tracks && n - up >= a.cuts.min_tracks;
            }
        }
        for (int part = 0; part < (split ? 2 : 1); part++) {
            const int sel = split ? part : -1;
            const WSums s = member_sums(mk, n, sel, wz);
            const double zv = s.swz / s.sw;
            const double c2v = member_chi2(mk, n, sel, zv, wz);
            const double sp = member_sumpt2(a, mk, n, sel, sid);
            int v = 0;
            if (lane == 0) {
                v = atomicAdd(a.nv + e, 1);
                if (v < kVtxCap) {
                    const int o = e * kVtxCap + v;
                    a.vz[o] = zv;
                    a.vez[o] = (float)(1.0 / sqrt(s.sw));
                    a.vc2[o] = (float)c2v;
                    a.vnt[o] = s.n;
                    a.vsp[o] = sp;
                    a.vkey[o] = 2 * q + part;
                } else {
                    set_status(a, PT_VTX_TOO_MANY);
                }
                if (part == 0) a.cv0[e * kVtxCap + c] = v;
                else a.cv1[e * kVtxCap + c] = v;
                if (!split) a.cv1[e * kVtxCap + c] = -1;
            }
        }
    }
}

// Per event: the vertices by sum of pT^2 (then z, then the key), their
// outputs and the vertex of every member track (one block).
constexpr int kOrderThreads = 256;

__global__ void __launch_bounds__(kOrderThreads) k_vtx_order(VtxArgs a) {
    __shared__ double s_z[kVtxCap], s_sp[kVtxCap];
    __shared__ int s_vkey[kVtxCap], s_rank[kVtxCap];
    const int e = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int base = a.ev_off[e];
    const int nv = min(a.nv[e], kVtxCap), nc = a.nc[e];
    const int32_t *key = a.key + base, *sid = a.sid + base;
    for (int v = tid; v < nv; v += blockDim.x) {
        s_z[v] = a.vz[e * kVtxCap + v];
        s_sp[v] = a.vsp[e * kVtxCap + v];
        s_vkey[v] = a.vkey[e * kVtxCap + v];
    }
    __syncthreads();
    for (int v = tid; v < nv; v += blockDim.x) {
        const double sv = s_sp[v], zv = s_z[v];
        const int kv = s_vkey[v];
        int r = 0;
        for (int u = 0; u < nv; u++)
            r += s_sp[u] > sv || (s_sp[u] == sv && (s_z[u] < zv || (s_z[u] == zv && s_vkey[u] < kv)));
        s_rank[v] = r;
        if (r < a.max_vertices) {
            const int64_t o = (int64_t)e * a.max_vertices + r;
            a.out.z[o] = (float)zv;
            a.out.ez[o] = a.vez[e * kVtxCap + v];
            a.out.chi2[o] = a.vc2[e * kVtxCap + v];
            a.out.ndf[o] = a.vnt[e * kVtxCap + v] - 1;
            a.out.ntracks[o] = a.vnt[e * kVtxCap + v];
            a.out.sumpt2[o] = (float)sv;
        }
    }
    if (tid == 0) {
        a.out.n[e] = min(nv, a.max_vertices);
        if (nv > a.max_vertices) set_status(a, PT_VTX_TOO_MANY);
    }
    __syncthreads();
    for (int c = wid; c < nc; c += nw) {
        const int q = a.cq[e * kVtxCap + c], n = a.cn[e * kVtxCap + c];
        const int v0 = a.cv0[e * kVtxCap + c], v1 = a.cv1[e * kVtxCap + c];
        for (int k = lane; k < n; k += 32) {
            const int32_t kk = key[q + k];
            const int v = (v1 >= 0 && ((kk >> kSideBit) & 1)) ? v1 : v0;
            if (v < nv && s_rank[v] < a.max_vertices) a.out.track_vertex[sid[kk & kPosMask]] = s_rank[v];
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_track_summary(int32_t n_tracks, const int32_t *hits, const uint8_t *tn,
                                                            const float *params, const float *cov,
                                                            const int32_t *tuple, const int32_t *ev_off,
                                                            int32_t n_events, float pt_of_kappa, int32_t *ev,
                                                            float *z0, float *ez0, float *pt, uint8_t *nh) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_tracks; k += gridDim.x * blockDim.x) {
        const int t = tuple[k];
        const int h = hits[(int64_t)t * PT_NMAX];
        int lo = 0, hi = n_events;                       // the last e with ev_off[e] <= h
        while (hi - lo > 1) {
            const int m = (lo + hi) >> 1;
            if (ev_off[m] <= h) lo = m;
            else hi = m;
        }
        ev[k] = lo;
        z0[k] = params[(int64_t)k * 5 + 4];
        ez0[k] = sqrtf(cov[(int64_t)k * 15 + 14]);
        pt[k] = pt_of_kappa / fabsf(params[(int64_t)k * 5]);
        nh[k] = tn[t];
    }
}

}  // namespace

// Scratch layout (byte offsets, each array 16-byte aligned).
struct VtxLayout {
    size_t ev_off, ev_cur, part, order, rho, root, wz, key, sid, nc, nv, cq, cn, cv0, cv1, vz, vsp, vez, vc2, vnt,
        vkey, total;
};

VtxLayout vertex_layout(int32_t n_tracks, int32_t n_events) {
    VtxLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 15) & ~(size_t)15;
        return at;
    };
    const size_t nt = (size_t)n_tracks + 1, ne = (size_t)n_events + 1, ncap = (size_t)n_events * kVtxCap + 1;
    L.ev_off = take(4 * ne);
    L.ev_cur = take(4 * ne);
    L.part = take(4 * ((size_t)n_events / kScanItems + 2));
    L.order = take(4 * nt);
    L.rho = take(4 * nt);
    L.root = take(4 * nt);
    L.wz = take(16 * nt);
    L.key = take(4 * nt);
    L.sid = take(4 * nt);
    L.nc = take(4 * ne);
    L.nv = take(4 * ne);
    L.cq = take(4 * ncap);
    L.cn = take(4 * ncap);
    L.cv0 = take(4 * ncap);
    L.cv1 = take(4 * ncap);
    L.vz = take(8 * ncap);
    L.vsp = take(8 * ncap);
    L.vez = take(4 * ncap);
    L.vc2 = take(4 * ncap);
    L.vnt = take(4 * ncap);
    L.vkey = take(4 * ncap);
    L.total = o;
    return L;
}

size_t vertex_scratch_bytes(int32_t n_tracks, int32_t n_events) { return vertex_layout(n_tracks, n_events).total; }

pt_status launch_vertices(const pt_vertex_tracks &in, int32_t n_tracks, int32_t n_events,
                          const pt_vertex_cuts &cuts, int32_t max_vertices, void *scratch, const pt_vertices &out,
                          int grid, cudaStream_t s) {
    VtxArgs a;
    a.n_tracks = n_tracks;
    a.n_events = n_events;
    a.max_vertices = max_vertices;
    a.in = in;
    a.cuts = cuts;
    const VtxLayout L = vertex_layout(n_tracks, n_events);
    char *w = (char *)scratch;
    a.ev_off = (int32_t *)(w + L.ev_off);
    a.ev_cur = (int32_t *)(w + L.ev_cur);
    int32_t *part = (int32_t *)(w + L.part);
    a.order = (int32_t *)(w + L.order);
    a.rho = (int32_t *)(w + L.rho);
    a.root = (int32_t *)(w + L.root);
    a.wz = (double2 *)(w + L.wz);
    a.key = (int32_t *)(w + L.key);
    a.sid = (int32_t *)(w + L.sid);
    a.nc = (int32_t *)(w + L.nc);
    a.nv = (int32_t *)(w + L.nv);
    a.cq = (int32_t *)(w + L.cq);
    a.cn = (int32_t *)(w + L.cn);
    a.cv0 = (int32_t *)(w + L.cv0);
    a.cv1 = (int32_t *)(w + L.cv1);
    a.vz = (double *)(w + L.vz);
    a.vsp = (double *)(w + L.vsp);
    a.vez = (float *)(w + L.vez);
    a.vc2 = (float *)(w + L.vc2);
    a.vnt = (int32_t *)(w + L.vnt);
    a.vkey = (int32_t *)(w + L.vkey);
    a.out = out;
    // per device and call (cheap; no shared state between threads or devices)
    if (cudaFuncSetAttribute(k_vtx_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kVtxDynSmem) !=
        cudaSuccess)
        return PT_ERR_CUDA;
    if (cudaMemsetAsync(a.ev_off, 0, sizeof(int32_t) * ((size_t)n_events + 1), s) != cudaSuccess ||
        cudaMemsetAsync(a.ev_cur, 0, sizeof(int32_t) * ((size_t)n_events + 1), s) != cudaSuccess ||
        cudaMemsetAsync(out.status, 0, sizeof(int32_t), s) != cudaSuccess)
        return PT_ERR_CUDA;
    {
        KernelTimer t("k_vtx_count", s);
        k_vtx_count<<<grid, kThreads, 0, s>>>(a);
    }
    launch_scan(a.ev_off, n_events, part, s);
    {
        KernelTimer t("k_vtx_fill", s);
        k_vtx_fill<<<grid, kThreads, 0, s>>>(a);
    }
    {
        KernelTimer t("k_vtx_group", s);
        k_vtx_group<<<n_events, kVtxThreads, kVtxDynSmem, s>>>(a);
    }
    {
        KernelTimer t("k_vtx_fit", s);
        k_vtx_fit<<<dim3(kVtxCap / kFitWarps, n_events), 32 * kFitWarps, 0, s>>>(a);
    }
    KernelTimer t("k_vtx_order", s);
    k_vtx_order<<<n_events, kOrderThreads, 0, s>>>(a);
    return PT_OK;
}

void launch_track_summary(int32_t n_tracks, const int32_t *hits, const uint8_t *tn, const float *params,
                          const float *cov, const int32_t *tuple, const int32_t *ev_off, int32_t n_events, float bz,
                          int32_t *ev, float *z0, float *ez0, float *pt, uint8_t *nhits, int grid, cudaStream_t s) {
    // pT [GeV] = 0.299792458 B[T] R[m], R = 1 / (100 |kappa|) with kappa in 1/cm
    const float pt_of_kappa = 0.299792458e-2f * bz;
    KernelTimer t("k_track_summary", s);
    k_track_summary<<<grid, kThreads, 0, s>>>(n_tracks, hits, tn, params, cov, tuple, ev_off, n_events, pt_of_kappa,
                                             ev, z0, ez0, pt, nhits);
}

}  // namespace ptk
