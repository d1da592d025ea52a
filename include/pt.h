/*
 * pt.h - C ABI of the GB300 pixel seeding + broken-line fitting library.
 *
 * Implements the data-parallel hot path of Bocci, Kortelainen, Innocente,
 * Pantaleo, Rovere, "Heterogeneous reconstruction of tracks and primary
 * vertices with the CMS pixel tracker" (arXiv 2008.13461): from reconstructed
 * pixel hits to fitted tracks, in four calls issued in order on one CUDA
 * stream:
 *
 *   pt_build_doublets  Sec. 3.2 (doublets on layer pairs under the Table 1
 *                      cuts PhiW, ZW, ZIP, PT, hits tiled in phi) and the
 *                      Fishbone of Sec. 3.3;
 *   pt_connect_cells   Sec. 3.2 (Cellular-Automaton connection: R-z
 *                      alignment, curvature, beamspot and dz compatibility);
 *   pt_find_ntuplets   Sec. 3.2 (root doublets, depth-first search) and the
 *                      shared-doublet cleaning of Sec. 3.3;
 *   pt_fit_tracks      Sec. 3.4 (broken-line fit: transverse pre-fit, s-z
 *                      line fit, transverse circle fit, combined parameters
 *                      and covariance);
 *   pt_fit_tracks_grad its adjoint (gradient with respect to the hits),
 *   pt_align_hits[_grad] per-module alignment of the hits and its adjoint;
 *   pt_resolve_ambiguities  Sec. 3.5 (post-fit ambiguity resolution);
 *   pt_track_summary, pt_find_vertices  Sec. 3.6 (pixel vertices);
 *   pt_bin_hits_noalloc the binning step without a caller workspace;
 *   pt_fma_probe, pt_doublet_candidates, pt_kernel_timing[_read]
 *                      measurement aids (arithmetic peaks, search work,
 *                      per-kernel times), not part of the method.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All array pointers are DEVICE pointers owned by the caller (the library
 *    allocates nothing).  Structs passed by pointer are read on the host
 *    during the call and may be reused afterwards.
 *  - `ws` is a caller-allocated device workspace of at least
 *    pt_workspace_size() bytes, 256-byte aligned.  It carries state from one
 *    call to the next: the four calls must receive the same ws, hits and
 *    config, in order.  Each output array's pointer is checked (non-NULL
 *    while its capacity is positive) by the call that writes it; later calls
 *    that read it (cells in pt_connect_cells and pt_find_ntuplets, edges in
 *    pt_find_ntuplets, tuples in pt_fit_tracks) take the structs as the
 *    earlier calls received them and do not check them again.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream) and never synchronise, so a sequence of calls can be
 *    captured in a CUDA graph.  Argument errors are returned synchronously;
 *    errors found on the device (capacity overflow, malformed input) are
 *    recorded in the workspace and returned by pt_read_counts(), the only
 *    call that synchronises the stream.
 *  - Capacities are upper bounds on outputs.  On overflow the counters keep
 *    counting, so pt_read_counts() reports the sizes needed; the outputs of
 *    that run are then incomplete and must be discarded.
 *  - Inputs must satisfy the exactness contract: every hit coordinate
 *    (x, y, z, r) is a float32 multiple of 2^-14 cm with magnitude below
 *    64 cm, and each hit lies inside the envelope of its layer.  Violations
 *    set PT_FLAG_INPUT.  Under the contract every doublet / cell / n-tuplet
 *    decision is the sign of an integer polynomial in the hit coordinates and
 *    the exact binary values of the float32 cut constants, and is decided
 *    exactly (a float32 evaluation with a proven error bound, falling back to
 *    exact integer arithmetic when the bound cannot decide).
 *  - Output order is unspecified (atomics); sets are deterministic.
 */
#ifndef PT_H
#define PT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PT_N_LAYERS 10      /* 4 barrel + 3 + 3 disks */
#define PT_MAX_PAIRS 32
#define PT_NMAX 8           /* maximum hits per n-tuplet */

typedef enum {
    PT_OK = 0,
    PT_ERR_INVALID_ARG = 1, /* NULL pointer, bad size, bad tuning, small ws */
    PT_ERR_CAPACITY = 2,    /* a device buffer overflowed (pt_read_counts) */
    PT_ERR_INPUT = 3,       /* input violates the contract (pt_read_counts) */
    PT_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    PT_ERR_TOO_LARGE = 5    /* beyond the fixed scratch of pt_bin_hits_noalloc */
} pt_status;

/* bits of pt_counts.flags */
#define PT_FLAG_CELLS 1u    /* cell capacity exceeded */
#define PT_FLAG_EDGES 2u    /* edge capacity exceeded */
#define PT_FLAG_TUPLES 4u   /* n-tuplet capacity exceeded */
#define PT_FLAG_TRACKS 8u   /* track capacity exceeded */
#define PT_FLAG_INPUT 16u   /* module id out of range, coordinate off the grid
                               or outside its layer envelope */

#define PT_LAYER_BARREL 0
#define PT_LAYER_DISK 1

/* One detector layer: its kind and the envelope that contains every hit on
 * it (used to bound search windows; hits outside set PT_FLAG_INPUT). */
typedef struct {
    int32_t kind;           /* PT_LAYER_BARREL or PT_LAYER_DISK */
    float rmin, rmax, zmin, zmax;
} pt_layer;

/* Geometry: layers plus the module -> layer table (device, n_modules). */
typedef struct {
    pt_layer layer[PT_N_LAYERS];
    const int32_t *module_layer;
    int32_t n_modules;
} pt_geometry;

/* Doublet cuts of one layer pair (Table 1), each stored in the form its
 * predicate uses (i = inner hit, o = outer hit; C = i x o, Dt = i . o in the
 * transverse plane):
 *   PhiW  Dt > 0 and C^2 <= tan2_dphi * Dt^2
 *   ZW    zlo <= z_i <= zhi
 *   ZIP   r_o > r_i and |z_i r_o - z_o r_i| <= zmax (r_o - r_i)
 *   PT    k_pt C^2 <= |o-i|^2 |i|^2 |o|^2      (k_pt = 4 rho_min^2)   */
typedef struct {
    int32_t inner, outer;   /* layer indices, inner closer to the beam */
    float tan2_dphi, zlo, zhi, zmax, k_pt;
} pt_pair_cuts;

/* Cellular-Automaton cuts for cells (a,b),(b,c) (Sec. 3.2), chosen by the
 * kind of the shared hit b's layer (barrel / endcap, Sec. 4.2):
 *   dz    |z_a r_c - z_c r_a| <= zmax (r_c - r_a)
 *   R-z   X^2 <= tol_rz2 ((r_c-r_a)^2 + (z_c-z_a)^2),
 *         X = (r_b-r_a)(z_c-z_b) - (z_b-z_a)(r_c-r_b)
 *   curv  |ab|^2 |bc|^2 |ca|^2 >= k_curv O^2, O = (b-a) x (c-a)
 *   R_max I^2 <= rmax2 |ab|^2 |bc|^2 |ca|^2, I = in-circle determinant of
 *         (a, b, c, origin)                                               */
typedef struct {
    float tol_rz2, k_curv, rmax2, zmax;
} pt_ca_cuts;

/* All cut constants.  Every float constant must lie in [2^-30, 2^40].
 * Fishbone (Sec. 3.3): cells (h1,h) and (h2,h) sharing the outer hit h, with
 * inner hits on one layer, are aligned when u = h1-h, v = h2-h satisfy
 * u.v > 0 and |u x v|^2 <= fishbone_eps2 |u|^2 |v|^2; an aligned cell dies if
 * its sibling is strictly shorter (3-D), or equally long with a smaller
 * input index.  min_hits: n-tuplets shorter than this are not fitted. */
typedef struct {
    int32_t n_pairs;
    pt_pair_cuts pair[PT_MAX_PAIRS];
    pt_ca_cuts region[2];   /* [0] barrel, [1] endcap */
    float fishbone_eps2;
    int32_t min_hits;
} pt_cuts;

/* Broken-line fit constants (Sec. 3.4): field (T), hit resolutions (cm),
 * material per module crossing (radiation lengths).  solve_fp32 = 0: the
 * normal equations, their Cholesky factors, solutions and chi2 in float64
 * (default); 1: everything in float32 (the precision variant; its deviation
 * from the float64 solve is characterised by the tests, not bounded). */
typedef struct {
    float bz, sigma_rphi, sigma_z, sigma_r, x0_barrel, x0_disk;
    int32_t solve_fp32;
} pt_fit_params;

/* Speed knobs; results do not depend on them. */
typedef struct {
    int32_t n_phi_bins;     /* azimuthal tiles per layer, 16..1024 */
    int32_t n_t_bins;       /* tiles along z (barrel) or r (disks), 1..64 */
    int32_t doublet_lanes;  /* lanes per outer hit: 4, 8, 16 or 32 */
    int32_t connect_lanes;  /* reserved (4, 8, 16 or 32 accepted); the CA
                               connection runs one warp per middle hit */
    int32_t blocks_per_sm;  /* persistent grid size factor, 1..32 */
} pt_tuning;

typedef struct {
    int64_t cells, edges, tuples, tracks;
} pt_capacity;

typedef struct {
    pt_geometry geometry;
    pt_cuts cuts;
    pt_fit_params fit;
    pt_tuning tuning;
    pt_capacity capacity;
} pt_config;

/* Hits of a batch of events (structure of arrays, device).  Event e owns
 * hits [ev_off[e], ev_off[e+1]); ev_off[0] = 0, ev_off[n_events] = n_hits;
 * n_hits at most 2^30. */
typedef struct {
    const float *x, *y, *z, *r;
    const int32_t *module;
    const int32_t *ev_off;
    int32_t n_hits, n_events;
} pt_hits;

/* Cells (doublets).  inner/outer are indices into the BINNED hit order
 * (pt_hit_order() maps them to input indices); pair indexes cuts.pair;
 * alive is 0 for cells removed by the Fishbone.  capacity.cells entries. */
typedef struct {
    int32_t *inner, *outer;
    uint8_t *pair, *alive;
} pt_cells;

/* CA edges: cell src (a,b) -> cell dst (b,c).  capacity.edges entries. */
typedef struct {
    int32_t *src, *dst;
} pt_edges;

/* n-tuplets: hits[t*PT_NMAX + k] input hit indices inner to outer,
 * cells[t*PT_NMAX + k] cell indices (k < n-1), n[t] hit count, alive[t] 0 if
 * removed by the shared-doublet cleaning.  capacity.tuples entries. */
typedef struct {
    int32_t *hits, *cells;
    uint8_t *n, *alive;
} pt_tuples;

/* Fitted tracks: params[k*5 + j] = (kappa [1/cm, q/rho, positive bends
 * clockwise for B along +z], phi0, tan(lambda), d0 [cm, PCA = d0 (sin phi0,
 * -cos phi0)], z0 [cm]); cov[k*15 + ...] lower triangle of the 5x5 covariance
 * in that order, row major; chi2; ndf = 2n-5; tuple = n-tuplet index.
 * capacity.tracks entries. */
typedef struct {
    float *params, *cov, *chi2;
    int8_t *ndf;
    int32_t *tuple;
} pt_tracks;

typedef struct {
    int64_t n_cells, n_edges, n_tuples, n_tracks; /* counts produced (or needed) */
    int64_t n_alive_cells, n_alive_tuples;
    int64_t n_exact_fallbacks;                    /* predicates decided exactly */
    int64_t n_doublet_candidates;                 /* inner hits the doublet search tested
                                                     (all layer pairs; see pt_doublet_candidates) */
    uint32_t flags;                               /* PT_FLAG_* */
} pt_counts;

/* Bytes of workspace needed for `hits` and `cfg` (reads only n_hits,
 * n_events of hits and tuning + capacity of cfg).  Returns 0 if invalid. */
size_t pt_workspace_size(const pt_hits *hits, const pt_config *cfg);

/* Sec. 3.2 + 3.3: tile hits per (event, layer, phi, z|r), build doublets of
 * all layer pairs, apply the Fishbone.  Resets the workspace counters. */
pt_status pt_build_doublets(void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg,
                            pt_cells *cells, void *stream);

/* Sec. 3.2: connect live cells sharing a hit into the CA graph. */
pt_status pt_connect_cells(void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg,
                           const pt_cells *cells, pt_edges *edges, void *stream);

/* Sec. 3.2 + 3.3: roots, depth-first search for maximal paths of >= 3 hits,
 * shared-doublet cleaning. */
pt_status pt_find_ntuplets(void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg,
                           const pt_cells *cells, const pt_edges *edges, pt_tuples *tuples,
                           void *stream);

/* Sec. 3.4: broken-line fit of every live n-tuplet with >= min_hits hits.
 * It may be called again on the same workspace with moved hit coordinates
 * (same n-tuplets; e.g. after an alignment update): it selects and fits the
 * tracks afresh. */
pt_status pt_fit_tracks(void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg,
                        const pt_tuples *tuples, pt_tracks *tracks, void *stream);

/* Adjoint of pt_fit_tracks (Sec. 3.4 differentiated): for the tracks of
 * the last pt_fit_tracks call on this workspace (same hits, config,
 * tuples, tracks), given the gradient of a scalar loss with respect to each
 * track's parameters, grad_params[K*5] in the order of pt_tracks.params
 * (kappa, phi0, tan lambda, d0, z0), and with respect to its chi2,
 * grad_chi2[K] (may be NULL: zero), ADDS the gradient with respect to the
 * input hit coordinates to grad_x, grad_y, grad_z[n_hits] (device,
 * caller-zeroed; hits on no track get nothing).  The fit is recomputed in
 * float64 for each track (nothing is stored by the forward call); the
 * covariance is not differentiated; clamps of the fit (minimum segment
 * length, curvature and |tan lambda|, maximum scattering weight) have zero
 * derivative where active.  K = pt_counts.n_tracks. */
pt_status pt_fit_tracks_grad(void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg,
                             const pt_tuples *tuples, const pt_tracks *tracks, const float *grad_params,
                             const float *grad_chi2, float *grad_x, float *grad_y, float *grad_z,
                             void *stream);

/* Sec. 3.5: ambiguity resolution of fitted tracks.  Tracks that share a
 * hit-doublet (a cell) are ambiguous and only the smallest chi2 is kept;
 * then triplets (3 hits) that share a hit are ambiguous and only the
 * smallest |transverse impact parameter| is kept.  Equal values are all
 * kept; the result does not depend on the order of the tracks.
 *
 * Track k is n-tuplet track_tuple[k] of `tuples` (its hits, cells and
 * length), with chi2[k] and impact parameter tip[k * tip_stride] (for
 * pt_tracks: tip = params + 3, tip_stride = 5).  Cell ids must lie in
 * [0, n_cells) and hit ids in [0, n_hits) to take part (others are
 * ignored); NaN chi2 or tip ranks last.  scratch: uint32[n_cells + n_hits]
 * device work space; keep: uint8[n_tracks] output (1 = kept).  All device
 * arrays; asynchronous on `stream`. */
pt_status pt_resolve_ambiguities(const pt_tuples *tuples, const int32_t *track_tuple, int32_t n_tracks,
                                 const float *chi2, const float *tip, int32_t tip_stride, int32_t n_cells,
                                 int32_t n_hits, uint32_t *scratch, uint8_t *keep, void *stream);

/* Sec. 3.6, pixel vertices.  Per-track inputs of the vertex finder (device
 * arrays of n_tracks): event index, z0 and its error ez0 [cm], pT [GeV], hit
 * count, and the ambiguity-resolution flag (keep may be NULL: all kept). */
typedef struct {
    const int32_t *ev;
    const float *z0, *ez0, *pt;
    const uint8_t *nhits, *keep;
} pt_vertex_tracks;

/* Vertex-finder cuts.  Track i is eligible when kept, nhits >= min_hits,
 * pt > pt_min, 0 < ez0 < ez0_max, z0 finite and 0 <= ev < n_events.  Tracks
 * i, j of one event are compatible when dz = z0_i - z0_j (float32) has
 * |dz| < dz_cut and dz*dz < chi2_max * (ez0_i*ez0_i + ez0_j*ez0_j) (float32,
 * rounded in that order).  A vertex with chi2/ndf > split_chi2 is split by
 * 2-means; vertices (and each part of a split) need min_tracks >= 1 tracks. */
typedef struct {
    float pt_min, ez0_max, dz_cut, chi2_max, split_chi2;
    int32_t min_hits, min_tracks;
} pt_vertex_cuts;

/* Vertices found, per event e at [e * max_vertices, ...) in decreasing sum of
 * pT^2 (the first is the primary vertex): z, its error ez, chi2, ndf = n-1,
 * ntracks n, sumpt2; n[e] vertices of event e (at most max_vertices).
 * track_vertex[n_tracks]: the track's vertex index within its event, -1 for
 * none.  status[1]: PT_VTX_* bits (0 = complete). */
typedef struct {
    int32_t *n;
    float *z, *ez, *chi2, *sumpt2;
    int32_t *ndf, *ntracks;
    int32_t *track_vertex;
    int32_t *status;
} pt_vertices;

#define PT_VTX_MAX_TRACKS 16384   /* eligible tracks per event */
#define PT_VTX_MAX_VERTICES 512   /* vertex candidates per event */
#define PT_VTX_EVENT_TOO_LARGE 1  /* an event had > PT_VTX_MAX_TRACKS eligible tracks: it got no vertices */
#define PT_VTX_TOO_MANY 2         /* more than PT_VTX_MAX_VERTICES candidates or max_vertices vertices in an
                                     event: the extra ones were dropped */
#define PT_VTX_INTERNAL 4         /* link chains did not resolve (not expected) */

/* Per-track summary of fitted tracks for pt_find_vertices: for track k of
 * `tracks` (n-tuplet tracks->tuple[k] of `tuples`), ev[k] = the event of its
 * first hit (by hits->ev_off), z0[k] = params z0, ez0[k] = sqrt(cov z0,z0),
 * pt[k] = 0.299792458e-2 bz / |kappa| (GeV, bz in T, kappa in 1/cm),
 * nhits[k] = the n-tuplet length.  Device outputs of n_tracks each. */
pt_status pt_track_summary(const pt_hits *hits, const pt_tuples *tuples, const pt_tracks *tracks, int32_t n_tracks,
                           float bz, int32_t *ev, float *z0, float *ez0, float *pt, uint8_t *nhits, void *stream);

/* Bytes of device scratch pt_find_vertices needs. */
size_t pt_vertex_scratch_size(int32_t n_tracks, int32_t n_events);

/* Sec. 3.6: vertices as clusters of tracks in z0.  Each eligible track gets a
 * density rho = 1 + the number of compatible tracks; it links to the nearest
 * compatible track (smallest |dz|, then smaller z0, then smaller index) of
 * higher rank (larger rho, or equal rho and smaller z0, or equal rho and z0
 * and smaller index); every track whose links lead
 * to a root with rho > 1 joins that root's candidate, and candidates of at
 * least min_tracks tracks are vertices: z the mean of z0 weighted by
 * 1/ez0^2, ez = 1/sqrt(sum of weights), chi2 = sum w (z0 - z)^2 (float64).
 * A vertex with chi2/ndf > split_chi2 is split in two by 2-means in z when
 * both parts keep min_tracks tracks; vertices are sorted by sum of pT^2.
 * scratch: device, >= pt_vertex_scratch_size() bytes, 16-byte aligned.
 * Asynchronous on `stream`; capacity problems are reported in out->status. */
pt_status pt_find_vertices(const pt_vertex_tracks *tracks, int32_t n_tracks, int32_t n_events,
                           const pt_vertex_cuts *cuts, int32_t max_vertices, void *scratch, size_t scratch_bytes,
                           pt_vertices *out, void *stream);

/* Alignment of the hits (per-module rigid corrections, the quantity whose
 * gradient a track-based alignment needs): a hit on module m moves to
 *     x' = c_m + (I + [w_m]x) (x - c_m) + d_m
 * with the module centre c_m, shift d_m and small rotation w_m (first order
 * in w; [w]x the cross-product matrix).  centre, shift, rot: float[n_modules
 * * 3] device arrays (x, y, z per module).  x, y, z, module: the hits
 * (n_hits); x_out, y_out, z_out: the moved hits (may not alias the inputs).
 * The result is not snapped to the exactness grid: use it for fitting, not
 * for pt_build_doublets. */
pt_status pt_align_hits(int32_t n_hits, const float *x, const float *y, const float *z, const int32_t *module,
                        int32_t n_modules, const float *centre, const float *shift, const float *rot,
                        float *x_out, float *y_out, float *z_out, void *stream);

/* Adjoint of pt_align_hits: given the gradient at the moved hits (gx_out,
 * gy_out, gz_out[n_hits]), ADDS the gradient with respect to the original
 * hits to gx, gy, gz (each may be NULL together: skipped) and, summed over
 * the hits of each module, with respect to the shifts (grad_shift) and the
 * rotations (grad_rot, float[n_modules * 3]; each may be NULL). */
pt_status pt_align_hits_grad(int32_t n_hits, const float *x, const float *y, const float *z,
                             const int32_t *module, int32_t n_modules, const float *centre, const float *rot,
                             const float *gx_out, const float *gy_out, const float *gz_out, float *gx, float *gy,
                             float *gz, float *grad_shift, float *grad_rot, void *stream);

/* Measurement helper, not part of the method: launches n_threads threads (a
 * positive multiple of 256) that each run 8 independent chains of `iters`
 * fused multiply-adds in float64 (fp64 = 1) or float32 (fp64 = 0) and write
 * one value each to out (device, n_threads elements of that type): 16 *
 * iters * n_threads flops, to be timed on `stream` for the device's
 * arithmetic peak. */
pt_status pt_fma_probe(int32_t fp64, int32_t iters, int32_t n_threads, void *out, void *stream);

/* Synchronises `stream`, then reports counts and device flags.  Returns
 * PT_ERR_CAPACITY or PT_ERR_INPUT when the corresponding flags are set. */
pt_status pt_read_counts(const void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg,
                         pt_counts *out, void *stream);

/* Measurement aid, not part of the method: synchronises `stream`, then
 * writes to per_pair[PT_MAX_PAIRS] (host) how many candidate inner hits the
 * doublet search of the last pt_build_doublets on ws tested for each layer
 * pair (cfg->cuts.pair order; the rest 0): the hits of the tiles its search
 * window covered, every one of which the Table 1 cuts were evaluated on.
 * Their sum is pt_counts.n_doublet_candidates. */
pt_status pt_doublet_candidates(const void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg,
                                int64_t *per_pair, void *stream);

/* Kernel timing (measurement aid, not part of the method).  While enabled,
 * every kernel this library launches on a stream that is not being captured
 * is bracketed by two CUDA events on that stream; pt_kernel_timing_read
 * waits for them and accumulates, per kernel name, the launches and their
 * total duration (ms).  pt_kernel_timing(1) clears the totals and starts
 * recording, pt_kernel_timing(0) stops it.  Host-side cost: two event
 * records per launch.  Not for use while another host thread launches
 * kernels of this library and reads the totals at the same time. */
typedef struct {
    char name[48];          /* kernel name, NUL-terminated */
    int64_t launches;
    double total_ms;
} pt_kernel_time;

pt_status pt_kernel_timing(int32_t enable);

/* Waits for the recorded launches and returns how many kernels have
 * totals; writes up to max_entries of them to out (host). */
int32_t pt_kernel_timing_read(pt_kernel_time *out, int32_t max_entries);

/* Device pointer (inside ws) to int32[n_hits]: binned position -> input hit
 * index, valid after pt_build_doublets. */
const int32_t *pt_hit_order(const void *ws, size_t ws_bytes, const pt_hits *hits,
                            const pt_config *cfg);

const char *pt_status_string(pt_status s);

/* Allocation-free hit binning, for callers that cannot allocate device
 * memory -- for instance code running where cudaMalloc is not allowed, or a
 * host program whose device memory is fully budgeted up front.  The paper
 * has no counterpart: this is the binning step of pt_build_doublets (hits
 * tiled per event, layer, phi tile and z|r tile) with its scratch kept in a
 * fixed array inside the library (about 14 MB held on every GPU that loads
 * the library, until the process exits) instead of a workspace.
 *
 * Inputs: hits and geometry as for pt_build_doublets (device arrays), tile
 * counts n_phi_bins in 16..1024 and n_t_bins in 1..64.  Outputs (device,
 * caller-allocated): binned[n_hits*4] float x, y, z, r in binned order,
 * 16-byte aligned; hit_order[n_hits] binned position -> input index;
 * tile_off[T+1] exclusive offsets of the T = n_events*10*n_phi_bins*n_t_bins
 * tiles (tile_off[T] = number of binned hits); flags[1] receives
 * PT_FLAG_INPUT when a hit violates the input contract (such hits are left
 * out).  The tile order and the offsets equal those of pt_build_doublets for
 * the same tuning; the order of hits inside a tile is unspecified.
 *
 * Limits: at most 2^20 hits and 2^22 tiles, else PT_ERR_TOO_LARGE.  The
 * library allocates nothing (no cudaMalloc / cudaFree); it only enqueues
 * memsets, kernels and one 4-byte device copy on `stream`.  The first call on
 * each device looks up the address of the fixed array with
 * cudaGetSymbolAddress, so make that first call before any stream capture.
 * The address is kept for the life of the process: after cudaDeviceReset()
 * (or anything else that destroys the device's primary context) it is
 * stale, so do not call this function again in that process.
 * All calls share the one array: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller. */
pt_status pt_bin_hits_noalloc(const pt_hits *hits, const pt_geometry *geometry, int32_t n_phi_bins,
                              int32_t n_t_bins, float *binned, int32_t *hit_order, int32_t *tile_off,
                              int32_t *flags, void *stream);

#ifdef __cplusplus
}
#endif
#endif
