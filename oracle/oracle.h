/*
 * CPU oracle for the pixel seeding + broken-line fitting path
 * (arXiv 2008.13461, Sec. 3.2-3.4).  TEST INFRASTRUCTURE ONLY: it is called
 * by the tests, the smoke check and the CPU-baseline leg of the benchmark,
 * never by the library.  It shares no header or helper with the CUDA code.
 */
#ifndef PT_ORACLE_H
#define PT_ORACLE_H
#include <stdint.h>

#define OR_NMAX 8          /* maximum hits of an n-tuplet */
#define OR_NLAYERS 10
#define OR_MAX_PAIRS 32

enum {
    OR_PRED_PHIW = 0, OR_PRED_ZIP = 1, OR_PRED_PT = 2, OR_PRED_RZ = 3,
    OR_PRED_CURV = 4, OR_PRED_BEAMSPOT = 5, OR_PRED_DZ = 6, OR_PRED_FB = 7
};

typedef struct {
    int32_t inner, outer;       /* layer indices */
    float tan2_dphi, zlo, zhi, zmax, k_pt;
} or_pair;

typedef struct { float tol_rz2, k_curv, rmax2, zmax; } or_region;

typedef struct {
    int32_t n_pairs;
    or_pair pair[OR_MAX_PAIRS];
    or_region region[2];        /* 0 barrel, 1 endcap (layer of the shared hit) */
    float fishbone_eps2;
    int32_t min_hits;
} or_cuts;

typedef struct {
    double bz, sigma_rphi, sigma_z, sigma_r, x0_barrel, x0_disk;
    double ms_scale;            /* multiplies the scattering variance (1 = physical) */
} or_fitpar;

typedef struct {
    const float *x, *y, *z, *r;
    const int32_t *module;
    int32_t n_hits;
    const int32_t *ev_off;
    int32_t n_events;
    const int32_t *module_layer;
    int32_t n_modules;
    int32_t layer_is_disk[OR_NLAYERS];
    const or_cuts *cuts;
    const or_fitpar *fitpar;
} or_input;

typedef struct {
    int32_t n;                  /* hits */
    int32_t hits[OR_NMAX];      /* input hit indices, inner to outer */
    int32_t cells[OR_NMAX - 1]; /* cell indices (into or_result.cells) */
} or_tuple;

typedef struct {
    int64_t n_cells;
    int32_t *cells;             /* [n_cells][3]: inner hit, outer hit, pair */
    uint8_t *cell_alive;        /* after Fishbone */
    int64_t n_edges;
    int64_t *edges;             /* [n_edges][2]: inner cell, outer cell */
    int64_t n_tuples;
    or_tuple *tuples;
    uint8_t *tuple_alive;       /* after shared-doublet cleaning */
    int64_t n_tracks;
    int64_t *track_tuple;
    double *params;             /* [n_tracks][5]: kappa, phi0, tan(lambda), d0, z0 */
    double *cov;                /* [n_tracks][15]: lower triangle, row major */
    double *chi2;
    int32_t *ndf;
} or_result;

int oracle_pred(int which, const float *hits /* [k][4] x,y,z,r */, int nh, float k);
/* 2-norm condition number of a symmetric n x n matrix (row-major), cyclic
 * Jacobi eigenvalues; -1 for a bad size. */
double oracle_sym_condition(int n, const double *M);

int oracle_fit(int n, const double *hx, const double *hy, const double *hz, const int *is_disk,
               const or_fitpar *fp, double *params, double *cov, double *chi2, int *ndf,
               double *extra);
int oracle_run(const or_input *in, int max_stage, or_result *res);
void oracle_free(or_result *res);

#endif
