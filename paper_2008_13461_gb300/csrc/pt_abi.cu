// C ABI of the seeding + fitting library (declarations and contracts in
// include/pt.h): argument validation, workspace layout, kernel launches.
#include <math.h>
#include <string.h>

#include "pt_common.cuh"
#include "pt_kernels.cuh"

using namespace ptk;

namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

bool tuning_ok(const pt_tuning &t) {
    auto lanes_ok = [](int g) { return g == 4 || g == 8 || g == 16 || g == 32; };
    return t.n_phi_bins >= 16 && t.n_phi_bins <= 1024 && t.n_t_bins >= 1 && t.n_t_bins <= 64 &&
           lanes_ok(t.doublet_lanes) && lanes_ok(t.connect_lanes) && t.blocks_per_sm >= 1 &&
           t.blocks_per_sm <= 32;
}

bool capacity_ok(const pt_capacity &c) {
    const int64_t lim = 0x7fffffff;
    return c.cells >= 0 && c.cells <= lim && c.edges >= 0 && c.edges <= lim && c.tuples >= 0 &&
           c.tuples <= lim && c.tracks >= 0 && c.tracks <= lim;
}

bool layout(const pt_hits *h, const pt_config *cfg, WsLayout &L) {
    if (!h || !cfg || h->n_hits < 0 || h->n_events < 1) return false;
    if (!tuning_ok(cfg->tuning) || !capacity_ok(cfg->capacity)) return false;
    const int64_t n_bins =
        (int64_t)h->n_events * PT_N_LAYERS * cfg->tuning.n_phi_bins * cfg->tuning.n_t_bins;
    if (n_bins >= 0x7fffffff) return false;
    const size_t nh = (size_t)(h->n_hits > 0 ? h->n_hits : 1);
    const size_t nc = (size_t)(cfg->capacity.cells > 0 ? cfg->capacity.cells : 1);
    L.n_bins = n_bins;
    L.n_scan_blocks = (int32_t)((n_bins + kScanItems - 1) / kScanItems);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    L.counters = take(sizeof(int32_t) * kCounters);
    L.bin_cnt = take(sizeof(int32_t) * (size_t)(n_bins + 1));
    const int64_t hit_blocks = (int64_t)(nh + kScanItems - 1) / kScanItems;
    L.scan_part = take(sizeof(int32_t) * (size_t)((L.n_scan_blocks > hit_blocks ? L.n_scan_blocks : hit_blocks) + 1));
    L.hit_bin = take(4 * nh);
    L.hit_rank = take(4 * nh);
    L.bh = take(16 * nh);
    L.blayer = take(nh);
    L.bev = take(4 * nh);
    L.perm = take(4 * nh);
    L.in_off = take(4 * nh);
    L.in_cnt = take(4 * nh);
    L.in_live = take(4 * nh);
    L.hk = take(16 * nh);
    L.ck = take(4 * nc);
    L.sk = take(8 * nc);
    L.sci = take(4 * nc);
    L.edge_rng = take(8 * nc);
    L.has_out = take(nc);
    L.maxlen = take(4 * nc);
    L.erec = take(16 * (size_t)(cfg->capacity.edges > 0 ? cfg->capacity.edges : 1));
    L.trk_blk = take(sizeof(int32_t) * 4 * kSelBlocks);
    L.total = o;
    return true;
}

// Longest path (in hits) of the layer-pair graph, or -1 if it has a cycle.
int longest_layer_path(const pt_cuts &c) {
    int best[PT_N_LAYERS];
    for (int i = 0; i < PT_N_LAYERS; i++) best[i] = 1;
    for (int round = 0; round <= PT_N_LAYERS; round++) {
        bool changed = false;
        for (int k = 0; k < c.n_pairs; k++) {
            int a = c.pair[k].inner, b = c.pair[k].outer;
            if (best[a] + 1 > best[b]) {
                best[b] = best[a] + 1;
                changed = true;
            }
        }
        if (!changed) {
            int m = 1;
            for (int i = 0; i < PT_N_LAYERS; i++) m = best[i] > m ? best[i] : m;
            return m;
        }
    }
    return -1;
}

bool const_ok(float v) { return isfinite(v) && v >= ldexpf(1.0f, -30) && v <= ldexpf(1.0f, 40); }

bool config_ok(const pt_config *cfg) {
    const pt_cuts &c = cfg->cuts;
    const pt_geometry &g = cfg->geometry;
    if (!g.module_layer || g.n_modules <= 0) return false;
    for (int i = 0; i < PT_N_LAYERS; i++) {
        const pt_layer &l = g.layer[i];
        if ((l.kind != PT_LAYER_BARREL && l.kind != PT_LAYER_DISK) || !(l.rmin < l.rmax) || !(l.zmin < l.zmax) ||
            !isfinite(l.rmin) || !isfinite(l.rmax) || !isfinite(l.zmin) || !isfinite(l.zmax))
            return false;
    }
    if (c.n_pairs < 1 || c.n_pairs > PT_MAX_PAIRS) return false;
    int per_outer[PT_N_LAYERS] = {0};
    for (int k = 0; k < c.n_pairs; k++) {
        const pt_pair_cuts &p = c.pair[k];
        if (p.inner < 0 || p.inner >= PT_N_LAYERS || p.outer < 0 || p.outer >= PT_N_LAYERS || p.inner == p.outer)
            return false;
        for (int j = 0; j < k; j++)
            if (c.pair[j].inner == p.inner && c.pair[j].outer == p.outer) return false;
        if (++per_outer[p.outer] > kMaxPairsPerLayer) return false;
        if (!const_ok(p.tan2_dphi) || !const_ok(p.zmax) || !const_ok(p.k_pt)) return false;
        if (!isfinite(p.zlo) || !isfinite(p.zhi) || p.zlo > p.zhi) return false;
    }
    for (int r = 0; r < 2; r++) {
        const pt_ca_cuts &q = c.region[r];
        if (!const_ok(q.tol_rz2) || !const_ok(q.k_curv) || !const_ok(q.rmax2) || !const_ok(q.zmax)) return false;
    }
    if (!const_ok(c.fishbone_eps2) || c.fishbone_eps2 >= 1.0f) return false;
    if (c.min_hits < 3 || c.min_hits > PT_NMAX) return false;
    const int lp = longest_layer_path(c);
    if (lp < 0 || lp > PT_NMAX) return false;
    const pt_fit_params &f = cfg->fit;
    if (!(f.bz > 0) || !(f.sigma_rphi > 0) || !(f.sigma_z > 0) || !(f.sigma_r > 0) || !(f.x0_barrel > 0) ||
        !(f.x0_disk > 0) || (f.solve_fp32 != 0 && f.solve_fp32 != 1))
        return false;
    return true;
}

bool hits_ok(const pt_hits *h) {
    if (!h || h->n_hits < 0 || h->n_hits > (1 << 30) || h->n_events < 1 || !h->ev_off) return false;
    if (h->n_hits > 0 && (!h->x || !h->y || !h->z || !h->r || !h->module)) return false;
    return true;
}

int num_sms() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cache[dev] = n;
    }
    return cache[dev];
}

// Fill kernel parameters; outputs not yet produced may be null.
Params make_params(void *ws, const WsLayout &L, const pt_hits *h, const pt_config *cfg) {
    Params p;
    memset(&p, 0, sizeof p);
    char *w = (char *)ws;
    p.x = h->x; p.y = h->y; p.z = h->z; p.r = h->r;
    p.module = h->module;
    p.ev_off = h->ev_off;
    p.module_layer = cfg->geometry.module_layer;
    p.n_hits = h->n_hits;
    p.n_events = h->n_events;
    p.n_modules = cfg->geometry.n_modules;
    p.counters = (int32_t *)(w + L.counters);
    p.bin_cnt = (int32_t *)(w + L.bin_cnt);
    p.scan_part = (int32_t *)(w + L.scan_part);
    p.hit_bin = (int32_t *)(w + L.hit_bin);
    p.hit_rank = (int32_t *)(w + L.hit_rank);
    p.fb_big = p.hit_rank;     // free once the hits are binned
    p.bh = (float4 *)(w + L.bh);
    p.blayer = (int8_t *)(w + L.blayer);
    p.bev = (int32_t *)(w + L.bev);
    p.perm = (int32_t *)(w + L.perm);
    p.in_off = (int32_t *)(w + L.in_off);
    p.in_cnt = (int32_t *)(w + L.in_cnt);
    p.hk = (float4 *)(w + L.hk);
    p.ck = (float *)(w + L.ck);
    p.sk = (float2 *)(w + L.sk);
    p.sci = (int32_t *)(w + L.sci);
    p.in_live = (int32_t *)(w + L.in_live);
    p.edge_rng = (int2 *)(w + L.edge_rng);
    p.has_out = (uint8_t *)(w + L.has_out);
    p.maxlen = (int32_t *)(w + L.maxlen);
    p.erec = (int4 *)(w + L.erec);
    p.trk_blk = (int32_t *)(w + L.trk_blk);
    p.cap_cells = cfg->capacity.cells;
    p.cap_edges = cfg->capacity.edges;
    p.cap_tuples = cfg->capacity.tuples;
    p.cap_tracks = cfg->capacity.tracks;
    p.n_phi = cfg->tuning.n_phi_bins;
    p.n_t = cfg->tuning.n_t_bins;
    p.n_bins = L.n_bins;
    p.n_scan_blocks = L.n_scan_blocks;
    const pt_cuts &c = cfg->cuts;
    for (int i = 0; i < PT_N_LAYERS; i++) p.layer[i] = cfg->geometry.layer[i];
    p.n_pairs = c.n_pairs;
    for (int k = 0; k < c.n_pairs; k++) {
        p.pair[k] = c.pair[k];
        // PhiW accepts |dphi| <= atan(sqrt(tan2)); the window adds a margin
        // far above float32 rounding of the angles involved
        p.pair_dphi[k] = (float)(atan(sqrt((double)c.pair[k].tan2_dphi)) + 1e-4);
        p.pair_pt_a[k] = c.pair[k].k_pt > 0.f ? (float)(1.0 / sqrt((double)c.pair[k].k_pt)) : 0.f;
        const int lo = c.pair[k].outer;
        p.pairs_by_outer[lo][p.n_pairs_by_outer[lo]++] = (int8_t)k;
        p.layer_is_inner[c.pair[k].inner] = 1;
    }
    for (int k = 0; k < c.n_pairs; k++) p.pair_inner_is_outer[k] = p.n_pairs_by_outer[c.pair[k].inner] > 0;
    // Fishbone slots: the distinct inner layers of each outer layer, ranked
    for (int lo = 0; lo < PT_N_LAYERS; lo++) {
        int inner_of_slot[kMaxPairsPerLayer], n_slots = 0;
        for (int q = 0; q < p.n_pairs_by_outer[lo]; q++) {
            const int k = p.pairs_by_outer[lo][q];
            int sl = 0;
            while (sl < n_slots && inner_of_slot[sl] != c.pair[k].inner) sl++;
            if (sl == n_slots) inner_of_slot[n_slots++] = c.pair[k].inner;
            p.pair_slot[k] = (int8_t)sl;
        }
        int sh = 0;
        while ((1 << sh) < n_slots) sh++;
        p.fb_slot_shift[lo] = (int8_t)sh;
    }
    p.region[0] = c.region[0];
    p.region[1] = c.region[1];
    for (int r = 0; r < 2; r++)   // tolerance as a distance, rounded up
        p.region_tol[r] = (float)(sqrt((double)c.region[r].tol_rz2) * (1.0 + 1e-6));
    p.fishbone_eps2 = c.fishbone_eps2;
    p.min_hits = c.min_hits;
    p.fit = cfg->fit;
    return p;
}

pt_status check_common(void *ws, size_t ws_bytes, const pt_hits *h, const pt_config *cfg, WsLayout &L) {
    if (!ws || ((uintptr_t)ws & 255) || !hits_ok(h) || !cfg || !config_ok(cfg)) return PT_ERR_INVALID_ARG;
    if (!layout(h, cfg, L) || ws_bytes < L.total) return PT_ERR_INVALID_ARG;
    return PT_OK;
}

int grid_for(const pt_config *cfg) {
    int sms = num_sms();
    return (sms > 0 ? sms : 1) * cfg->tuning.blocks_per_sm;
}

pt_status launched() { return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ERR_CUDA; }

// the 64-bit candidate counter of layer pair k in a host copy of the counters
int64_t pair_candidates(const int32_t *c, int k) {
    uint64_t v;
    memcpy(&v, c + C_PAIR_CAND + 2 * k, sizeof v);
    return (int64_t)v;
}

}  // namespace

extern "C" {

size_t pt_workspace_size(const pt_hits *hits, const pt_config *cfg) {
    WsLayout L;
    if (!layout(hits, cfg, L)) return 0;
    return L.total;
}

pt_status pt_build_doublets(void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg, pt_cells *cells,
                            void *stream) {
    WsLayout L;
    pt_status st = check_common(ws, ws_bytes, hits, cfg, L);
    if (st != PT_OK) return st;
    if (!cells || (cfg->capacity.cells > 0 && (!cells->inner || !cells->outer || !cells->pair || !cells->alive)))
        return PT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Params p = make_params(ws, L, hits, cfg);
    p.cell_inner = cells->inner;
    p.cell_outer = cells->outer;
    p.cell_pair = cells->pair;
    p.cell_alive = cells->alive;
    if (cudaMemsetAsync(p.counters, 0, sizeof(int32_t) * kCounters, s) != cudaSuccess) return PT_ERR_CUDA;
    if (cudaMemsetAsync(p.bin_cnt, 0, sizeof(int32_t) * (size_t)(L.n_bins + 1), s) != cudaSuccess)
        return PT_ERR_CUDA;
    if (cudaMemsetAsync(p.in_live, 0, sizeof(int32_t) * (size_t)hits->n_hits, s) != cudaSuccess) return PT_ERR_CUDA;
    const int grid = grid_for(cfg);
    launch_binning(p, grid, s);
    launch_doublets(p, cfg->tuning.doublet_lanes, grid, s);
    // alignment within eps (sin) implies |u^ - v^| <= 2 sin(asin(eps)/2) <= eps pi/2;
    // 4e-6 covers the float32 rounding of the unit vectors.  Key buckets are
    // at least that wide, with room for the rounding of the bucket index.
    const double dmax = sqrt((double)cfg->cuts.fishbone_eps2) * 1.5707963267948966 + 4e-6;
    launch_fishbone(p, (float)(dmax * dmax), (float)(dmax * 1.01 + 1e-5), grid, s);
    return launched();
}

pt_status pt_connect_cells(void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg,
                           const pt_cells *cells, pt_edges *edges, void *stream) {
    WsLayout L;
    pt_status st = check_common(ws, ws_bytes, hits, cfg, L);
    if (st != PT_OK) return st;
    if (!cells || !edges || (cfg->capacity.edges > 0 && (!edges->src || !edges->dst))) return PT_ERR_INVALID_ARG;
    Params p = make_params(ws, L, hits, cfg);
    p.cell_inner = cells->inner;
    p.cell_outer = cells->outer;
    p.cell_pair = cells->pair;
    p.cell_alive = cells->alive;
    p.edge_src = edges->src;
    p.edge_dst = edges->dst;
    launch_connect(p, grid_for(cfg), (cudaStream_t)stream);
    return launched();
}

pt_status pt_find_ntuplets(void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg,
                           const pt_cells *cells, const pt_edges *edges, pt_tuples *tuples, void *stream) {
    WsLayout L;
    pt_status st = check_common(ws, ws_bytes, hits, cfg, L);
    if (st != PT_OK) return st;
    if (!cells || !edges || !tuples ||
        (cfg->capacity.tuples > 0 && (!tuples->hits || !tuples->cells || !tuples->n || !tuples->alive)))
        return PT_ERR_INVALID_ARG;
    Params p = make_params(ws, L, hits, cfg);
    p.cell_inner = cells->inner;
    p.cell_outer = cells->outer;
    p.cell_pair = cells->pair;
    p.cell_alive = cells->alive;
    p.edge_src = edges->src;
    p.edge_dst = edges->dst;
    p.tup_hits = tuples->hits;
    p.tup_cells = tuples->cells;
    p.tup_n = tuples->n;
    p.tup_alive = tuples->alive;
    if (cfg->capacity.cells > 0 &&
        cudaMemsetAsync(p.maxlen, 0, sizeof(int32_t) * (size_t)cfg->capacity.cells, (cudaStream_t)stream) !=
            cudaSuccess)
        return PT_ERR_CUDA;
    launch_ntuplets(p, grid_for(cfg), (cudaStream_t)stream);
    return launched();
}

pt_status pt_fit_tracks(void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg,
                        const pt_tuples *tuples, pt_tracks *tracks, void *stream) {
    WsLayout L;
    pt_status st = check_common(ws, ws_bytes, hits, cfg, L);
    if (st != PT_OK) return st;
    if (!tuples || !tracks ||
        (cfg->capacity.tracks > 0 &&
         (!tracks->params || !tracks->cov || !tracks->chi2 || !tracks->ndf || !tracks->tuple)))
        return PT_ERR_INVALID_ARG;
    Params p = make_params(ws, L, hits, cfg);
    p.tup_hits = tuples->hits;
    p.tup_cells = tuples->cells;
    p.tup_n = tuples->n;
    p.tup_alive = tuples->alive;
    p.trk_params = tracks->params;
    p.trk_cov = tracks->cov;
    p.trk_chi2 = tracks->chi2;
    p.trk_ndf = tracks->ndf;
    p.trk_tuple = tracks->tuple;
    const int grid = grid_for(cfg);
    cudaStream_t s = (cudaStream_t)stream;
    // the selection counts afresh on every call
    if (cudaMemsetAsync(p.counters + C_TRACKS, 0, sizeof(int32_t), s) != cudaSuccess ||
        cudaMemsetAsync(p.counters + C_TRK_CNT, 0, sizeof(int32_t) * 8, s) != cudaSuccess)
        return PT_ERR_CUDA;
    launch_select(p, grid, s);
    launch_fit(p, grid, s);
    return launched();
}

pt_status pt_fit_tracks_grad(void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg,
                             const pt_tuples *tuples, const pt_tracks *tracks, const float *grad_params,
                             const float *grad_chi2, float *grad_x, float *grad_y, float *grad_z, void *stream) {
    WsLayout L;
    pt_status st = check_common(ws, ws_bytes, hits, cfg, L);
    if (st != PT_OK) return st;
    if (!tuples || !tracks || !tuples->hits || !tuples->n || !tracks->tuple || !grad_params || !grad_x ||
        !grad_y || !grad_z)
        return PT_ERR_INVALID_ARG;
    Params p = make_params(ws, L, hits, cfg);
    p.tup_hits = tuples->hits;
    p.tup_n = tuples->n;
    p.trk_tuple = tracks->tuple;
    launch_fit_grad(p, grad_params, grad_chi2, grad_x, grad_y, grad_z, grid_for(cfg), (cudaStream_t)stream);
    return launched();
}

static int align_grid(int32_t n);

pt_status pt_resolve_ambiguities(const pt_tuples *tuples, const int32_t *track_tuple, int32_t n_tracks,
                                 const float *chi2, const float *tip, int32_t tip_stride, int32_t n_cells,
                                 int32_t n_hits, uint32_t *scratch, uint8_t *keep, void *stream) {
    if (n_tracks < 0 || n_cells < 0 || n_hits < 0 || tip_stride < 1) return PT_ERR_INVALID_ARG;
    if (n_tracks == 0) return PT_OK;
    const int64_t n_scratch = (int64_t)n_cells + n_hits;      // both up to 2^31 - 1: sum in 64 bits
    if (!tuples || !tuples->hits || !tuples->cells || !tuples->n || !track_tuple || !chi2 || !tip || !keep ||
        (!scratch && n_scratch > 0))
        return PT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_scratch > 0 && cudaMemsetAsync(scratch, 0xff, sizeof(uint32_t) * (size_t)n_scratch, s) != cudaSuccess)
        return PT_ERR_CUDA;
    launch_ambiguities(tuples->hits, tuples->cells, tuples->n, track_tuple, n_tracks, chi2, tip, tip_stride, n_cells,
                       n_hits, scratch, keep, align_grid(n_tracks), s);
    return launched();
}

static int align_grid(int32_t n) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int need = (n + kThreads - 1) / kThreads;
    return need < 1 ? 1 : (need < sms * 8 ? need : sms * 8);
}

pt_status pt_align_hits(int32_t n_hits, const float *x, const float *y, const float *z, const int32_t *module,
                        int32_t n_modules, const float *centre, const float *shift, const float *rot,
                        float *x_out, float *y_out, float *z_out, void *stream) {
    if (n_hits < 0 || n_modules <= 0) return PT_ERR_INVALID_ARG;
    if (n_hits == 0) return PT_OK;
    if (!x || !y || !z || !module || !centre || !shift || !rot || !x_out || !y_out || !z_out)
        return PT_ERR_INVALID_ARG;
    launch_align(n_hits, x, y, z, module, centre, shift, rot, x_out, y_out, z_out, align_grid(n_hits),
                 (cudaStream_t)stream);
    return launched();
}

pt_status pt_align_hits_grad(int32_t n_hits, const float *x, const float *y, const float *z,
                             const int32_t *module, int32_t n_modules, const float *centre, const float *rot,
                             const float *gx_out, const float *gy_out, const float *gz_out, float *gx, float *gy,
                             float *gz, float *grad_shift, float *grad_rot, void *stream) {
    if (n_hits < 0 || n_modules <= 0) return PT_ERR_INVALID_ARG;
    if (n_hits == 0) return PT_OK;
    if (!x || !y || !z || !module || !centre || !rot || !gx_out || !gy_out || !gz_out) return PT_ERR_INVALID_ARG;
    if ((gx != nullptr) != (gy != nullptr) || (gx != nullptr) != (gz != nullptr)) return PT_ERR_INVALID_ARG;
    launch_align_grad(n_hits, x, y, z, module, centre, rot, gx_out, gy_out, gz_out, gx, gy, gz, grad_shift, grad_rot,
                      align_grid(n_hits), (cudaStream_t)stream);
    return launched();
}

pt_status pt_track_summary(const pt_hits *hits, const pt_tuples *tuples, const pt_tracks *tracks, int32_t n_tracks,
                           float bz, int32_t *ev, float *z0, float *ez0, float *pt, uint8_t *nhits, void *stream) {
    if (!hits || !tuples || !tracks || n_tracks < 0 || hits->n_events < 1 || !hits->ev_off) return PT_ERR_INVALID_ARG;
    if (n_tracks == 0) return PT_OK;
    if (!tuples->hits || !tuples->n || !tracks->params || !tracks->cov || !tracks->tuple || !ev || !z0 || !ez0 ||
        !pt || !nhits)
        return PT_ERR_INVALID_ARG;
    launch_track_summary(n_tracks, tuples->hits, tuples->n, tracks->params, tracks->cov, tracks->tuple, hits->ev_off,
                         hits->n_events, bz, ev, z0, ez0, pt, nhits, align_grid(n_tracks), (cudaStream_t)stream);
    return launched();
}

size_t pt_vertex_scratch_size(int32_t n_tracks, int32_t n_events) {
    if (n_tracks < 0 || n_events < 0) return 0;
    return vertex_scratch_bytes(n_tracks, n_events);
}

pt_status pt_find_vertices(const pt_vertex_tracks *tracks, int32_t n_tracks, int32_t n_events,
                           const pt_vertex_cuts *cuts, int32_t max_vertices, void *scratch, size_t scratch_bytes,
                           pt_vertices *out, void *stream) {
    if (!tracks || !cuts || !out || n_tracks < 0 || n_events < 0 || max_vertices < 1 || cuts->min_tracks < 1)
        return PT_ERR_INVALID_ARG;
    if (!out->status) return PT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n_events == 0) return cudaMemsetAsync(out->status, 0, sizeof(int32_t), s) == cudaSuccess ? PT_OK : PT_ERR_CUDA;
    if (!out->n || !out->z || !out->ez || !out->chi2 || !out->sumpt2 || !out->ndf || !out->ntracks ||
        (n_tracks > 0 && (!out->track_vertex || !tracks->ev || !tracks->z0 || !tracks->ez0 || !tracks->pt ||
                          !tracks->nhits)))
        return PT_ERR_INVALID_ARG;
    if (!scratch || ((uintptr_t)scratch & 15) || scratch_bytes < vertex_scratch_bytes(n_tracks, n_events))
        return PT_ERR_INVALID_ARG;
    if ((int64_t)n_events * max_vertices > INT32_MAX) return PT_ERR_INVALID_ARG;
    const pt_status st = launch_vertices(*tracks, n_tracks, n_events, *cuts, max_vertices, scratch, *out,
                                         align_grid(n_tracks > 0 ? n_tracks : 1), s);
    return st != PT_OK ? st : launched();
}

pt_status pt_read_counts(const void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg,
                         pt_counts *out, void *stream) {
    WsLayout L;
    if (!ws || !out || !layout(hits, cfg, L) || ws_bytes < L.total) return PT_ERR_INVALID_ARG;
    int32_t c[kCounters];
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(c, (const char *)ws + L.counters, sizeof c, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PT_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PT_ERR_CUDA;
    out->n_cells = (uint32_t)c[C_CELLS];
    out->n_edges = (uint32_t)c[C_EDGES];
    out->n_tuples = (uint32_t)c[C_TUPLES];
    out->n_tracks = (uint32_t)c[C_TRACKS];
    out->n_alive_cells = (uint32_t)c[C_ALIVE_CELLS];
    out->n_alive_tuples = (uint32_t)c[C_ALIVE_TUPLES];
    out->n_exact_fallbacks = (uint32_t)c[C_FALLBACK];
    int64_t cand = 0;
    for (int k = 0; k < PT_MAX_PAIRS; k++) cand += pair_candidates(c, k);
    out->n_doublet_candidates = cand;
    out->flags = (uint32_t)c[C_FLAGS];
    if (out->flags & PT_FLAG_INPUT) return PT_ERR_INPUT;
    if (out->flags & (PT_FLAG_CELLS | PT_FLAG_EDGES | PT_FLAG_TUPLES | PT_FLAG_TRACKS)) return PT_ERR_CAPACITY;
    return PT_OK;
}

pt_status pt_doublet_candidates(const void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg,
                                int64_t *per_pair, void *stream) {
    WsLayout L;
    if (!ws || !per_pair || !layout(hits, cfg, L) || ws_bytes < L.total) return PT_ERR_INVALID_ARG;
    int32_t c[kCounters];
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(c, (const char *)ws + L.counters, sizeof c, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PT_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PT_ERR_CUDA;
    for (int k = 0; k < PT_MAX_PAIRS; k++) per_pair[k] = pair_candidates(c, k);
    return PT_OK;
}

const int32_t *pt_hit_order(const void *ws, size_t ws_bytes, const pt_hits *hits, const pt_config *cfg) {
    WsLayout L;
    if (!ws || !layout(hits, cfg, L) || ws_bytes < L.total) return nullptr;
    return (const int32_t *)((const char *)ws + L.perm);
}

const char *pt_status_string(pt_status s) {
    switch (s) {
    case PT_OK: return "ok";
    case PT_ERR_INVALID_ARG: return "invalid argument";
    case PT_ERR_CAPACITY: return "output capacity exceeded";
    case PT_ERR_INPUT: return "input violates the contract";
    case PT_ERR_CUDA: return "CUDA error";
    case PT_ERR_TOO_LARGE: return "problem larger than the fixed scratch of the allocation-free entry point";
    }
    return "unknown status";
}

}  // extern "C"
