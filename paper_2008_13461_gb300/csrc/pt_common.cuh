// Shared device-side definitions of the GB300 seeding + fitting kernels:
// workspace layout, launch configuration and the exact geometric predicates
// (float32 evaluation with a proven error bound, exact integer fallback).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pt.h"

namespace ptk {

constexpr int kThreads = 256;            // threads per block of every kernel
constexpr int kMaxPairsPerLayer = 8;
constexpr int kCounters = 32 + 2 * PT_MAX_PAIRS;

// workspace counters (int32 slots at the start of ws)
enum Counter {
    C_CELLS = 0, C_EDGES = 1, C_TUPLES = 2, C_TRACKS = 3, C_FLAGS = 4, C_FALLBACK = 5,
    C_ALIVE_CELLS = 6, C_ALIVE_TUPLES = 7,
    C_FB_NEXT = 9,        // Fishbone: next chunk of outer hits to take
    C_FB_BIG = 10,        // Fishbone: outer hits listed for the large warps
    C_FB_BIG_NEXT = 11,   // Fishbone: next listed outer hit to take
    C_CA_PENDING = 12,    // CA connection: cells left to the exact pass
    C_DB_PENDING = 13,    // doublets: outer hits left to the exact pass
    C_FB_PENDING = 14,    // Fishbone: outer hits left to the exact pass
    C_DB_NEXT = 15,       // doublets: next outer hits to take
    C_TRK_CNT = 16,       // tracks with 3, 4, 5, 6..8 hits (4 slots)
    C_TRK_CUR = 20,       // next track index of each of those classes (4 slots)
    C_FB_HUGE = 24,       // Fishbone: outer hits listed for the largest warps
    C_FB_HUGE_NEXT = 25,  // Fishbone: next of those to take
    C_CA_NEXT = 26,       // CA connection: next chunk of cells to take
    C_PAIR_CAND = 32      // doublet candidates per layer pair (64-bit, PT_MAX_PAIRS of them)
};

// Slope-key bucket of a live incoming cell of a hit with n of them (lowest
// key k0, inverse bucket width iw): the Fishbone orders the cells by it and
// the connection searches by it, so both evaluate these same roundings.
// For an integer b in [1, nb - 1], sk_bucket(key) < b exactly when
// sk_coord(key) < b (truncation of a coordinate below b is below b, of one
// at or above b is at or above b), which compares without a conversion.
__device__ __forceinline__ int sk_buckets(int n) { return max(32, 1 << (32 - __clz(max(n, 1) - 1))); }
__device__ __forceinline__ float sk_coord(float key, float k0, float iw) { return __fmul_rn(__fsub_rn(key, k0), iw); }
__device__ __forceinline__ int sk_bucket(float key, float k0, float iw, int nb) {
    return min(max(__float2int_rz(sk_coord(key, k0, iw)), 0), nb - 1);
}

// class of a track by its hit count: 3, 4, 5, 6..8 -> 0..3
__device__ __forceinline__ int track_class(int n) { return min(n, 6) - 3; }

// Byte offsets of every workspace array (all 256-byte aligned).
struct WsLayout {
    size_t counters, bin_cnt, scan_part, hit_bin, hit_rank;
    size_t bh, blayer, bev, perm, in_off, in_cnt, in_live, hk, ck, sk, sci, trk_blk;
    size_t edge_rng, has_out, maxlen, erec;
    size_t total;
    int64_t n_bins;        // events * layers * phi bins * t bins
    int32_t n_scan_blocks;
};

constexpr int kScanItems = 4096;         // bins per scan block (256 threads x 16)
constexpr int kSelBlocks = 1024;         // blocks of the track selection

// Everything a kernel needs, passed by value.
struct Params {
    // inputs
    const float *x, *y, *z, *r;
    const int32_t *module, *ev_off, *module_layer;
    int32_t n_hits, n_events, n_modules;
    // workspace
    int32_t *counters, *bin_cnt, *scan_part, *hit_bin, *hit_rank;
    float4 *bh;                          // binned hits (x, y, z, r)
    int8_t *blayer;
    int32_t *bev, *perm, *in_off, *in_cnt;
    int32_t *fb_big;                     // outer hits with many cells (reuses hit_rank after binning)
    int2 *edge_rng;                      // per cell: (first incoming edge, count)
    int4 *erec;                          // per edge: its source cell, that cell's (first, count) of
                                         //   incoming edges, input index of its inner hit * 2 + root
    float *ck;                           // R-z slope key of each cell w.r.t. its outer hit (scratch)
    float4 *hk;                          // per hit: max sqrt(1+key^2) and min gap of its incoming
                                         //   cells; lowest key and inverse bucket width of the live ones
    int32_t *in_live;                    // per hit: live incoming cells
    float2 *sk;                          // live incoming cells of each hit by slope-key bucket:
    int32_t *sci;                        //   (key, inner hit as int bits) and the cell index
    uint8_t *has_out;
    int32_t *maxlen;
    int32_t *trk_blk;                    // track selection: per block and class, counts then offsets
    // outputs
    int32_t *cell_inner, *cell_outer;
    uint8_t *cell_pair, *cell_alive;
    int32_t *edge_src, *edge_dst;
    int32_t *tup_hits, *tup_cells;
    uint8_t *tup_n, *tup_alive;
    float *trk_params, *trk_cov, *trk_chi2;
    int8_t *trk_ndf;
    int32_t *trk_tuple;
    // capacities
    int64_t cap_cells, cap_edges, cap_tuples, cap_tracks;
    // binning
    int32_t n_phi, n_t;
    int64_t n_bins;
    int32_t n_scan_blocks;
    // cuts
    pt_layer layer[PT_N_LAYERS];
    pt_pair_cuts pair[PT_MAX_PAIRS];
    float pair_dphi[PT_MAX_PAIRS];       // azimuthal half window of PhiW (rad)
    float pair_pt_a[PT_MAX_PAIRS];       // 1 / (2 R) of the PT cut's minimum circumradius R (0: no cut)
    int32_t n_pairs;
    int8_t pairs_by_outer[PT_N_LAYERS][kMaxPairsPerLayer];
    int32_t n_pairs_by_outer[PT_N_LAYERS];
    int8_t layer_is_inner[PT_N_LAYERS];  // 1 if the layer is the inner layer of some pair
    int8_t pair_inner_is_outer[PT_MAX_PAIRS];  // 1 if cells can end on the pair's inner layer
    int8_t pair_slot[PT_MAX_PAIRS];      // rank of the pair's inner layer among those of its outer layer
    int8_t fb_slot_shift[PT_N_LAYERS];   // log2 of a power of two >= the inner layers of the layer
    pt_ca_cuts region[2];
    float region_tol[2];                 // sqrt(tol_rz2) rounded up
    float fishbone_eps2;
    int32_t min_hits;
    pt_fit_params fit;
};

// ---------------------------------------------------------------- utilities
__device__ __forceinline__ void set_flag(int32_t *counters, uint32_t f) {
    atomicOr(reinterpret_cast<unsigned int *>(counters + C_FLAGS), f);
}

// True when an earlier stage ran out of capacity in one of the mask's
// outputs: this stage's inputs are incomplete, and it does nothing (the
// caller reads the flags and reruns with larger buffers).
__device__ __forceinline__ bool upstream_overflow(const Params &p, uint32_t mask) {
    return (p.counters[C_FLAGS] & mask) != 0;
}

__device__ __forceinline__ long long grid_int(float v) {
    // exact: v is a multiple of 2^-14 below 2^17 in magnitude (hits below 64
    // and their differences), so v * 2^14 is an integer that fits 32 bits;
    // the 32-bit conversion avoids the 64-bit one, which is slow here
    return (long long)__float2int_rn(v * 16384.0f);
}

// Azimuthal tile of angle phi in [-pi, pi]: monotone in phi, clamped.
__device__ __forceinline__ int phi_tile(float phi, int n_phi) {
    int b = __float2int_rd((phi + 3.14159265f) * (n_phi * 0.159154943f));
    return min(max(b, 0), n_phi - 1);
}

__device__ __forceinline__ int t_tile(float t, float tmin, float tmax, int n_t) {
    int b = __float2int_rd((t - tmin) * (n_t / (tmax - tmin)));
    return min(max(b, 0), n_t - 1);
}

// ------------------------------------------------ exact integer arithmetic
// 320-bit two's-complement integer used only when a float32 filter cannot
// decide the sign of a predicate polynomial.
struct Big {
    unsigned long long w[5];
};

__device__ __forceinline__ Big big_from(long long v) {
    Big r;
    unsigned long long s = v < 0 ? ~0ull : 0ull;
    r.w[0] = (unsigned long long)v;
#pragma unroll
    for (int i = 1; i < 5; i++) r.w[i] = s;
    return r;
}

__device__ __forceinline__ Big big_add(const Big &a, const Big &b) {
    Big r;
    unsigned long long c = 0;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        unsigned long long s = a.w[i] + c;
        unsigned long long c1 = s < c;
        unsigned long long t = s + b.w[i];
        c = c1 + (t < s);
        r.w[i] = t;
    }
    return r;
}

__device__ __forceinline__ Big big_neg(const Big &a) {
    Big r;
#pragma unroll
    for (int i = 0; i < 5; i++) r.w[i] = ~a.w[i];
    return big_add(r, big_from(1));
}

__device__ __forceinline__ Big big_sub(const Big &a, const Big &b) { return big_add(a, big_neg(b)); }

__device__ __forceinline__ bool big_isneg(const Big &a) { return (a.w[4] >> 63) != 0; }

__device__ __forceinline__ int big_sign(const Big &a) {
    if (big_isneg(a)) return -1;
    unsigned long long o = 0;
#pragma unroll
    for (int i = 0; i < 5; i++) o |= a.w[i];
    return o ? 1 : 0;
}

// product modulo 2^320 (callers keep |a*b| < 2^319)
__device__ __forceinline__ Big big_mul(const Big &a, const Big &b) {
    bool na = big_isneg(a), nb = big_isneg(b);
    Big ma = na ? big_neg(a) : a, mb = nb ? big_neg(b) : b;
    Big r;
#pragma unroll
    for (int i = 0; i < 5; i++) r.w[i] = 0;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        unsigned long long carry = 0;
#pragma unroll
        for (int j = 0; j < 5 - i; j++) {
            unsigned long long lo = ma.w[i] * mb.w[j];
            unsigned long long hi = __umul64hi(ma.w[i], mb.w[j]);
            unsigned long long s = r.w[i + j] + lo;
            hi += (s < lo);
            unsigned long long s2 = s + carry;
            hi += (s2 < s);
            r.w[i + j] = s2;
            carry = hi;
        }
    }
    return (na != nb) ? big_neg(r) : r;
}

__device__ __forceinline__ Big big_shl(const Big &a, int k) {
    Big r;
    int ls = k >> 6, bs = k & 63;
#pragma unroll
    for (int i = 4; i >= 0; i--) {
        int src = i - ls;
        unsigned long long v = 0;
        if (src >= 0) {
            v = a.w[src] << bs;
            if (bs && src >= 1) v |= a.w[src - 1] >> (64 - bs);
        }
        r.w[i] = v;
    }
    return r;
}

// sign of (B - K * 2^s * A) for a float32 constant K (its exact binary value)
static __device__ __noinline__ int big_cmp_scaled(const Big &B, float K, int s, const Big &A) {
    int ex;
    float fr = frexpf(K, &ex);
    long long m = (long long)ldexpf(fr, 24);
    int E = ex - 24 + s;
    Big MA = big_mul(big_from(m), A);
    Big d = (E >= 0) ? big_sub(B, big_shl(MA, E)) : big_sub(big_shl(B, -E), MA);
    return big_sign(d);
}

// ------------------------------------------------------- float32 filters
// A polynomial evaluated in float32 by a fixed tree of + - x on exact inputs
// differs from its exact value by at most gamma_d * Pbar, Pbar being the same
// tree evaluated on absolute values (d = depth, gamma_d = d u / (1 - d u),
// u = 2^-24; Higham, Accuracy and Stability of Numerical Algorithms, Sec. 3).
// The bound below is that with a factor-two margin, plus an absolute term
// that covers gradual underflow.  Values within it go to the exact path.
constexpr float kU = 5.9604645e-8f;
__device__ __forceinline__ float ferr(int depth, float pbar) {
    return (2.0f * depth + 2.0f) * kU * pbar + 1e-27f;
}

struct GHit {
    long long x, y, z, r;
};

__device__ __forceinline__ GHit ghit(float x, float y, float z, float r) {
    GHit h = {grid_int(x), grid_int(y), grid_int(z), grid_int(r)};
    return h;
}

// ---- exact forms (integer polynomials; see pt.h for the predicates)
static __device__ __noinline__ int exact_phiw(GHit i, GHit o, float T, int32_t *counters) {
    atomicAdd(counters + C_FALLBACK, 1);
    long long Dt = i.x * o.x + i.y * o.y;
    if (Dt <= 0) return 0;
    long long C = i.x * o.y - i.y * o.x;
    Big c = big_from(C), d = big_from(Dt);
    return big_cmp_scaled(big_mul(c, c), T, 0, big_mul(d, d)) <= 0;
}

static __device__ __noinline__ int exact_zip(GHit i, GHit o, float zmax, int32_t *counters) {
    atomicAdd(counters + C_FALLBACK, 1);
    if (!(o.r > i.r)) return 0;
    long long L = i.z * o.r - o.z * i.r;
    if (L < 0) L = -L;
    return big_cmp_scaled(big_from(L), zmax, 14, big_from(o.r - i.r)) <= 0;
}

static __device__ __noinline__ int exact_pt(GHit i, GHit o, float K, int32_t *counters) {
    atomicAdd(counters + C_FALLBACK, 1);
    long long C = i.x * o.y - i.y * o.x;
    long long dx = o.x - i.x, dy = o.y - i.y;
    Big P = big_mul(big_mul(big_from(dx * dx + dy * dy), big_from(i.x * i.x + i.y * i.y)),
                    big_from(o.x * o.x + o.y * o.y));
    Big c = big_from(C);
    return big_cmp_scaled(P, K, 28, big_mul(c, c)) >= 0;
}

static __device__ __noinline__ int exact_rz(GHit a, GHit b, GHit c, float tol2, int32_t *counters) {
    atomicAdd(counters + C_FALLBACK, 1);
    Big X = big_sub(big_mul(big_from(b.r - a.r), big_from(c.z - b.z)),
                    big_mul(big_from(b.z - a.z), big_from(c.r - b.r)));
    long long dr = c.r - a.r, dz = c.z - a.z;
    Big L2 = big_add(big_mul(big_from(dr), big_from(dr)), big_mul(big_from(dz), big_from(dz)));
    return big_cmp_scaled(big_mul(X, X), tol2, 28, L2) <= 0;
}

__device__ __forceinline__ long long sq2(long long dx, long long dy) { return dx * dx + dy * dy; }

static __device__ __noinline__ int exact_curv(GHit a, GHit b, GHit c, float K, int32_t *counters) {
    atomicAdd(counters + C_FALLBACK, 1);
    long long O = (b.x - a.x) * (c.y - a.y) - (b.y - a.y) * (c.x - a.x);
    Big P = big_mul(big_mul(big_from(sq2(b.x - a.x, b.y - a.y)), big_from(sq2(c.x - b.x, c.y - b.y))),
                    big_from(sq2(a.x - c.x, a.y - c.y)));
    Big o = big_from(O);
    return big_cmp_scaled(P, K, 28, big_mul(o, o)) >= 0;
}

static __device__ __noinline__ int exact_beamspot(GHit a, GHit b, GHit c, float rmax2, int32_t *counters) {
    atomicAdd(counters + C_FALLBACK, 1);
    Big a2 = big_from(sq2(a.x, a.y)), b2 = big_from(sq2(b.x, b.y)), c2 = big_from(sq2(c.x, c.y));
    Big m1 = big_sub(big_mul(big_from(b.y), c2), big_mul(b2, big_from(c.y)));
    Big m2 = big_sub(big_mul(big_from(b.x), c2), big_mul(b2, big_from(c.x)));
    Big m3 = big_from(b.x * c.y - b.y * c.x);
    Big I = big_add(big_sub(big_mul(big_from(a.x), m1), big_mul(big_from(a.y), m2)), big_mul(a2, m3));
    Big P = big_mul(big_mul(big_from(sq2(b.x - a.x, b.y - a.y)), big_from(sq2(c.x - b.x, c.y - b.y))),
                    big_from(sq2(a.x - c.x, a.y - c.y)));
    return big_cmp_scaled(big_mul(I, I), rmax2, 28, P) <= 0;
}

static __device__ __noinline__ int exact_fb(GHit h1, GHit h2, GHit h, float eps2, int32_t *counters) {
    atomicAdd(counters + C_FALLBACK, 1);
    long long ux = h1.x - h.x, uy = h1.y - h.y, uz = h1.z - h.z;
    long long vx = h2.x - h.x, vy = h2.y - h.y, vz = h2.z - h.z;
    if (ux * vx + uy * vy + uz * vz <= 0) return 0;
    Big cx = big_from(uy * vz - uz * vy), cy = big_from(uz * vx - ux * vz), cz = big_from(ux * vy - uy * vx);
    Big cr = big_add(big_add(big_mul(cx, cx), big_mul(cy, cy)), big_mul(cz, cz));
    Big uv = big_mul(big_from(ux * ux + uy * uy + uz * uz), big_from(vx * vx + vy * vy + vz * vz));
    return big_cmp_scaled(cr, eps2, 0, uv) <= 0;
}

// a*b - c*d with one rounding: Kahan's algorithm with FMA, relative error
// at most 2u (Jeannerod, Louvet, Muller, Math. Comp. 82 (2013) 2245).
__device__ __forceinline__ float det2(float a, float b, float c, float d) {
    const float w = __fmul_rn(c, d);
    const float e = __fmaf_rn(-c, d, w);
    const float f = __fmaf_rn(a, b, -w);
    return __fadd_rn(f, e);
}

// ---- filtered predicates (float32 with proven bound; exact when undecided)
// Each returns 1 (holds) or 0 (fails).  With kExact = false an undecided
// float32 evaluation returns 2 instead of calling the exact form, so that
// hot kernels carry no big-integer code and can defer the rare undecided
// unit to a kernel that has it.
// Cross-product-like differences a*b - c*d that cancel for the accepted
// configurations are taken with det2 (relative error <= 2u), so the bounds
// scale with the result rather than with the products.
// i = inner, o = outer.

// PhiW: Dt > 0 and C^2 <= T Dt^2
template <bool kExact = true>
__device__ __forceinline__ int pred_phiw(float xi, float yi, float xo, float yo, float T, int32_t *cnt,
                                         float zi, float ri, float zo, float ro) {
    float p1 = xi * xo, p2 = yi * yo;
    float Dt = p1 + p2, Dtb = fabsf(p1) + fabsf(p2);
    float eD = ferr(2, Dtb);
    if (Dt < -eD) return 0;
    const float C = det2(xi, yo, yi, xo);
    if (Dt > eD) {
        float F = T * (Dt * Dt) - C * C;
        float e = ferr(5, T * (Dtb * Dtb) + C * C);
        if (F > e) return 1;
        if (F < -e) return 0;
    }
    if (!kExact) return 2;
    return exact_phiw(ghit(xi, yi, zi, ri), ghit(xo, yo, zo, ro), T, cnt);
}

// ZIP: r_o > r_i and |z_i r_o - z_o r_i| <= zmax (r_o - r_i)
template <bool kExact = true>
__device__ __forceinline__ int pred_zip(float xi, float yi, float zi, float ri, float xo, float yo, float zo,
                                        float ro, float zmax, int32_t *cnt) {
    if (!(ro > ri)) return 0;
    float a = zi * ro, b = zo * ri;
    float L = a - b, Lb = fabsf(a) + fabsf(b);
    float R = zmax * (ro - ri);
    float F = R - fabsf(L);
    float e = ferr(3, R + Lb);
    if (F > e) return 1;
    if (F < -e) return 0;
    if (!kExact) return 2;
    return exact_zip(ghit(xi, yi, zi, ri), ghit(xo, yo, zo, ro), zmax, cnt);
}

// PT: K C^2 <= |o-i|^2 |i|^2 |o|^2
template <bool kExact = true>
__device__ __forceinline__ int pred_pt(float xi, float yi, float zi, float ri, float xo, float yo, float zo,
                                       float ro, float K, int32_t *cnt) {
    float dx = xo - xi, dy = yo - yi;
    float P = ((dx * dx + dy * dy) * (xi * xi + yi * yi)) * (xo * xo + yo * yo);
    const float C = det2(xi, yo, yi, xo);
    float F = P - K * (C * C);
    float e = ferr(5, P + K * (C * C));
    if (F > e) return 1;
    if (F < -e) return 0;
    if (!kExact) return 2;
    return exact_pt(ghit(xi, yi, zi, ri), ghit(xo, yo, zo, ro), K, cnt);
}

struct FHit {
    float x, y, z, r;
};

__device__ __forceinline__ FHit load_hit(const float4 *bh, int i) {
    const float4 v = __ldg(bh + i);
    FHit h = {v.x, v.y, v.z, v.w};
    return h;
}

// CA dz: |z_a r_c - z_c r_a| <= zmax (r_c - r_a)
template <bool kExact = true>
__device__ __forceinline__ int pred_dz(const FHit &a, const FHit &c, float zmax, int32_t *cnt) {
    return pred_zip<kExact>(a.x, a.y, a.z, a.r, c.x, c.y, c.z, c.r, zmax, cnt);
}

// CA R-z: X^2 <= tol2 ((r_c-r_a)^2 + (z_c-z_a)^2)
template <bool kExact = true>
__device__ __forceinline__ int pred_rz(const FHit &a, const FHit &b, const FHit &c, float tol2, int32_t *cnt) {
    const float X = det2(b.r - a.r, c.z - b.z, b.z - a.z, c.r - b.r);
    float e1 = c.r - a.r, e2 = c.z - a.z;
    float T = tol2 * (e1 * e1 + e2 * e2);
    float F = T - X * X;
    float e = ferr(4, T + X * X);
    if (F > e) return 1;
    if (F < -e) return 0;
    if (!kExact) return 2;
    return exact_rz(ghit(a.x, a.y, a.z, a.r), ghit(b.x, b.y, b.z, b.r), ghit(c.x, c.y, c.z, c.r), tol2, cnt);
}

// CA curvature: |ab|^2 |bc|^2 |ca|^2 >= K O^2
template <bool kExact = true>
__device__ __forceinline__ int pred_curv(const FHit &a, const FHit &b, const FHit &c, float K, int32_t *cnt) {
    float abx = b.x - a.x, aby = b.y - a.y, acx = c.x - a.x, acy = c.y - a.y;
    float bcx = c.x - b.x, bcy = c.y - b.y;
    const float O = det2(abx, acy, aby, acx);
    float P = ((abx * abx + aby * aby) * (bcx * bcx + bcy * bcy)) * (acx * acx + acy * acy);
    float F = P - K * (O * O);
    float e = ferr(5, P + K * (O * O));
    if (F > e) return 1;
    if (F < -e) return 0;
    if (!kExact) return 2;
    return exact_curv(ghit(a.x, a.y, a.z, a.r), ghit(b.x, b.y, b.z, b.r), ghit(c.x, c.y, c.z, c.r), K, cnt);
}

// CA beamspot: I^2 <= rmax2 |ab|^2 |bc|^2 |ca|^2.  The lifted 4x4 in-circle
// determinant is invariant under translation, so I is evaluated about hit a
// (B = b-a, C = c-a, D = origin-a), where its terms are small; I is then
// bounded as an interval (its own error bound) before squaring.
template <bool kExact = true>
__device__ __forceinline__ int pred_beamspot(const FHit &a, const FHit &b, const FHit &c, float rmax2,
                                             int32_t *cnt) {
    const float Bx = b.x - a.x, By = b.y - a.y, Cx = c.x - a.x, Cy = c.y - a.y, Dx = -a.x, Dy = -a.y;
    const float B2 = Bx * Bx + By * By, C2 = Cx * Cx + Cy * Cy, D2 = Dx * Dx + Dy * Dy;
    const float t1 = Cy * D2, t2 = C2 * Dy, t3 = Cx * D2, t4 = C2 * Dx, t5 = Cx * Dy, t6 = Cy * Dx;
    const float m1 = t1 - t2, m2 = t3 - t4, m3 = t5 - t6;
    const float s1 = Bx * m1, s2 = By * m2, s3 = B2 * m3;
    const float I = (s1 - s2) + s3;
    const float Ib = fabsf(Bx) * (fabsf(t1) + fabsf(t2)) + fabsf(By) * (fabsf(t3) + fabsf(t4)) +
                     B2 * (fabsf(t5) + fabsf(t6));
    const float eI = ferr(7, Ib);
    const float bcx = c.x - b.x, bcy = c.y - b.y;
    const float T = rmax2 * ((B2 * (bcx * bcx + bcy * bcy)) * C2);
    const float eT = ferr(5, T);
    const float aI = fabsf(I);
    const float hi = aI + eI, lo = aI - eI;
    if (hi * hi * (1.0f + 8.0f * kU) < T - eT) return 1;
    if (lo > 0.0f && lo * lo * (1.0f - 8.0f * kU) > T + eT) return 0;
    if (!kExact) return 2;
    return exact_beamspot(ghit(a.x, a.y, a.z, a.r), ghit(b.x, b.y, b.z, b.r), ghit(c.x, c.y, c.z, c.r), rmax2,
                          cnt);
}


// Fishbone alignment: u.v > 0 and |u x v|^2 <= eps2 |u|^2 |v|^2 (3-D), for
// u = h1 - h and v = h2 - h.  Hits are multiples of 2^-14 below 64 in
// magnitude, so these differences are exact in float32 and the test can be
// given them directly.  The cross product of nearly parallel u, v cancels,
// so its components are taken with det2 (relative error <= 2u each); the
// squared norms and products of positive terms then carry relative errors
// below 8u, which bounds F.
template <bool kExact = true>
__device__ __forceinline__ int pred_fb_d(float ux, float uy, float uz, float vx, float vy, float vz, float eps2,
                                         int32_t *cnt) {
    const float d1 = ux * vx, d2 = uy * vy, d3 = uz * vz;
    const float dot = (d1 + d2) + d3, dotb = (fabsf(d1) + fabsf(d2)) + fabsf(d3);
    const float eD = ferr(3, dotb);
    if (dot < -eD) return 0;
    if (dot > eD) {
        const float cx = det2(uy, vz, uz, vy), cy = det2(uz, vx, ux, vz), cz = det2(ux, vy, uy, vx);
        const float cr = (cx * cx + cy * cy) + cz * cz;
        const float E = eps2 * ((ux * ux + uy * uy + uz * uz) * (vx * vx + vy * vy + vz * vz));
        const float F = E - cr;
        const float e = 12.0f * kU * (E + cr) + 1e-27f;
        if (F > e) return 1;
        if (F < -e) return 0;
    }
    if (!kExact) return 2;
    const GHit o = {0, 0, 0, 0};
    return exact_fb(ghit(ux, uy, uz, 0.f), ghit(vx, vy, vz, 0.f), o, eps2, cnt);
}

__device__ __forceinline__ int pred_fb(const FHit &h1, const FHit &h2, const FHit &h, float eps2, int32_t *cnt) {
    return pred_fb_d(h1.x - h.x, h1.y - h.y, h1.z - h.z, h2.x - h.x, h2.y - h.y, h2.z - h.z, eps2, cnt);
}

}  // namespace ptk
