/*
 * Plain, slow CPU oracle for the pixel seeding + fitting path of
 * Bocci et al., "Heterogeneous reconstruction of tracks and primary vertices
 * with the CMS pixel tracker" (arXiv 2008.13461).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may call this code.  It shares nothing with
 * the CUDA implementation (no headers, no helpers, no tables).
 *
 * What it computes, stage by stage, in the paper's order (Sec. 3.2-3.4):
 *   1. doublets on the layer pairs of the cut table, every inner hit against
 *      every outer hit of the same event (no binning), kept when the PhiW, ZW,
 *      ZIP and PT cuts of Table 1 pass;
 *   2. Fishbone (Sec. 3.3): among aligned cells sharing the outer hit whose
 *      inner hits lie on the same layer, only the shortest survives;
 *   3. Cellular-Automaton connection (Sec. 3.2): cells (a,b) and (b,c) are
 *      linked when the three hits are aligned in R-z, the circle through them
 *      has a radius above the pT_min radius and passes within R_max of the
 *      beamspot, and the a-c line points within z_max of the origin along z;
 *   4. roots (inner hit on BPix1, or on BPix2 / FPix1+- with no inner
 *      neighbour) and a depth-first search emitting every maximal path of at
 *      least three hits (Sec. 3.2);
 *   5. shared-doublet cleaning (Sec. 3.3): among tuples sharing a cell only
 *      those with the largest number of hits survive;
 *   6. the broken-line fit of every surviving tuple with at least min_hits
 *      hits (Sec. 3.4, method of Blobel 2006), in double precision.
 *
 * Exactness.  Hits are float32 multiples of g = 2^-14 cm with |coord| < 64
 * cm, so X = x / g is an integer below 2^20.  Every graph decision is the sign
 * of an integer polynomial in these integers and in the exact binary values
 * of float32 cut constants; the oracle evaluates it with a signed big integer
 * (below), so it is decided exactly.
 *
 * The paper names each cut but gives no formula; the forms used (one per
 * cut) are written next to each predicate.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* ------------------------------------------------------------------ bigint
 * Sign-magnitude integer, little-endian 64-bit limbs. */
#define BIG_LIMBS 12
typedef struct {
    int neg;          /* 1 if negative (never set for zero) */
    int n;            /* limbs in use; 0 means the value zero */
    uint64_t w[BIG_LIMBS];
} big;

static void big_fail(const char *what) {
    fprintf(stderr, "oracle bigint overflow in %s\n", what);
    abort();
}

static void big_norm(big *a) {
    while (a->n > 0 && a->w[a->n - 1] == 0) a->n--;
    if (a->n == 0) a->neg = 0;
}

static big big_i64(int64_t v) {
    big r;
    memset(&r, 0, sizeof r);
    if (v < 0) {
        r.neg = 1;
        r.w[0] = (uint64_t)(-(v + 1)) + 1u;
    } else {
        r.w[0] = (uint64_t)v;
    }
    r.n = 1;
    big_norm(&r);
    return r;
}

static int mag_cmp(const big *a, const big *b) {
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    for (int i = a->n - 1; i >= 0; i--)
        if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
    return 0;
}

static big mag_add(const big *a, const big *b) {
    big r;
    memset(&r, 0, sizeof r);
    int n = a->n > b->n ? a->n : b->n;
    unsigned __int128 carry = 0;
    for (int i = 0; i < n; i++) {
        unsigned __int128 s = carry;
        if (i < a->n) s += a->w[i];
        if (i < b->n) s += b->w[i];
        r.w[i] = (uint64_t)s;
        carry = s >> 64;
    }
    r.n = n;
    if (carry) {
        if (n == BIG_LIMBS) big_fail("add");
        r.w[n] = (uint64_t)carry;
        r.n = n + 1;
    }
    return r;
}

/* |a| - |b| assuming |a| >= |b| */
static big mag_sub(const big *a, const big *b) {
    big r;
    memset(&r, 0, sizeof r);
    uint64_t borrow = 0;
    for (int i = 0; i < a->n; i++) {
        uint64_t bi = i < b->n ? b->w[i] : 0;
        uint64_t d = a->w[i] - bi - borrow;
        borrow = (a->w[i] < bi) || (a->w[i] - bi < borrow);
        r.w[i] = d;
    }
    r.n = a->n;
    big_norm(&r);
    return r;
}

static big big_add(const big *a, const big *b) {
    big r;
    if (a->neg == b->neg) {
        r = mag_add(a, b);
        r.neg = a->neg;
    } else if (mag_cmp(a, b) >= 0) {
        r = mag_sub(a, b);
        r.neg = a->neg;
    } else {
        r = mag_sub(b, a);
        r.neg = b->neg;
    }
    big_norm(&r);
    return r;
}

static big big_neg(const big *a) {
    big r = *a;
    if (r.n) r.neg = !r.neg;
    return r;
}

static big big_sub(const big *a, const big *b) {
    big nb = big_neg(b);
    return big_add(a, &nb);
}

static big big_mul(const big *a, const big *b) {
    big r;
    memset(&r, 0, sizeof r);
    if (a->n == 0 || b->n == 0) return r;
    if (a->n + b->n > BIG_LIMBS) big_fail("mul");
    for (int i = 0; i < a->n; i++) {
        unsigned __int128 carry = 0;
        for (int j = 0; j < b->n; j++) {
            unsigned __int128 t = (unsigned __int128)a->w[i] * b->w[j] + r.w[i + j] + carry;
            r.w[i + j] = (uint64_t)t;
            carry = t >> 64;
        }
        r.w[i + b->n] = (uint64_t)carry;
    }
    r.n = a->n + b->n;
    r.neg = a->neg ^ b->neg;
    big_norm(&r);
    return r;
}

static big big_shl(const big *a, int k) {
    big r;
    memset(&r, 0, sizeof r);
    if (a->n == 0) return r;
    int ls = k / 64, bs = k % 64;
    if (a->n + ls + 1 > BIG_LIMBS) big_fail("shl");
    for (int i = 0; i < a->n; i++) {
        r.w[i + ls] |= a->w[i] << bs;
        if (bs) r.w[i + ls + 1] |= a->w[i] >> (64 - bs);
    }
    r.n = a->n + ls + 1;
    r.neg = a->neg;
    big_norm(&r);
    return r;
}

static int big_sign(const big *a) { return a->n == 0 ? 0 : (a->neg ? -1 : 1); }

static big big_mul3(big a, big b, big c) {
    big t = big_mul(&a, &b);
    return big_mul(&t, &c);
}

/* sign of (B - K * 2^s * A) for a float32 constant K (exact binary value). */
static int big_cmp_scaled(const big *B, float K, int s, const big *A) {
    int ex;
    float fr = frexpf(K, &ex);                 /* K = fr * 2^ex, 0.5 <= |fr| < 1 */
    int64_t m = (int64_t)ldexpf(fr, 24);      /* exact: float32 has 24 bits */
    int E = ex - 24 + s;                       /* K * 2^s = m * 2^E */
    big M = big_i64(m);
    big MA = big_mul(&M, A);
    big d;
    if (E >= 0) {
        big rhs = big_shl(&MA, E);
        d = big_sub(B, &rhs);
    } else {
        big lhs = big_shl(B, -E);
        d = big_sub(&lhs, &MA);
    }
    return big_sign(&d);
}

/* ---------------------------------------------------------------- grid hits */
typedef struct { int64_t x, y, z, r; } ghit;

static int64_t to_grid(float v) {
    /* exact for multiples of 2^-14 below 64 in magnitude */
    return (int64_t)llrint((double)v * 16384.0);
}

static ghit mk_ghit(float x, float y, float z, float r) {
    ghit h = {to_grid(x), to_grid(y), to_grid(z), to_grid(r)};
    return h;
}

/* ------------------------------------------------------------- predicates
 * i = inner hit, o = outer hit. */

/* PhiW (Table 1): azimuthal window |phi_o - phi_i| <= dphi_max, written
 * without angles: Dt = i.o > 0 and C^2 <= tan^2(dphi_max) Dt^2 with
 * C = i x o (transverse). */
static int pred_phiw(const ghit *i, const ghit *o, float tan2) {
    int64_t C = i->x * o->y - i->y * o->x;
    int64_t Dt = i->x * o->x + i->y * o->y;
    if (Dt <= 0) return 0;
    big c = big_i64(C), d = big_i64(Dt);
    big c2 = big_mul(&c, &c), d2 = big_mul(&d, &d);
    return big_cmp_scaled(&c2, tan2, 0, &d2) <= 0;
}

/* ZW (Table 1): window on the z of the inner hit. */
static int pred_zw(float zi, float zlo, float zhi) { return zi >= zlo && zi <= zhi; }

/* ZIP (Table 1): the r-z line through the two hits meets r = 0 within
 * |z| <= zmax:  r_o > r_i and |z_i r_o - z_o r_i| <= zmax (r_o - r_i). */
static int pred_zip(const ghit *i, const ghit *o, float zmax) {
    if (!(o->r > i->r)) return 0;
    int64_t L = i->z * o->r - o->z * i->r;
    if (L < 0) L = -L;
    big b = big_i64(L), a = big_i64(o->r - i->r);
    return big_cmp_scaled(&b, zmax, 14, &a) <= 0;
}

/* PT (Table 1): curvature assuming zero transverse impact parameter, i.e. the
 * circle through the origin, i and o has radius >= rho_min:
 *   4 rho_min^2 (i x o)^2 <= |o - i|^2 |i|^2 |o|^2. */
static int pred_pt(const ghit *i, const ghit *o, float k_pt) {
    int64_t C = i->x * o->y - i->y * o->x;
    int64_t dx = o->x - i->x, dy = o->y - i->y;
    big d2 = big_i64(dx * dx + dy * dy);
    big i2 = big_i64(i->x * i->x + i->y * i->y);
    big o2 = big_i64(o->x * o->x + o->y * o->y);
    big P = big_mul3(d2, i2, o2);
    big c = big_i64(C);
    big c2 = big_mul(&c, &c);
    return big_cmp_scaled(&P, k_pt, 28, &c2) >= 0;
}

/* CA R-z alignment (Sec. 3.2): distance of b from the line a-c in the (r,z)
 * plane at most tol:  X^2 <= tol^2 ((r_c-r_a)^2 + (z_c-z_a)^2),
 * X = (r_b-r_a)(z_c-z_b) - (z_b-z_a)(r_c-r_b). */
static int pred_rz(const ghit *a, const ghit *b, const ghit *c, float tol2) {
    big t1 = big_i64(b->r - a->r), t2 = big_i64(c->z - b->z);
    big t3 = big_i64(b->z - a->z), t4 = big_i64(c->r - b->r);
    big p1 = big_mul(&t1, &t2), p2 = big_mul(&t3, &t4);
    big X = big_sub(&p1, &p2);
    big X2 = big_mul(&X, &X);
    int64_t dr = c->r - a->r, dz = c->z - a->z;
    big dr_ = big_i64(dr), dz_ = big_i64(dz);
    big dr2 = big_mul(&dr_, &dr_), dz2 = big_mul(&dz_, &dz_);
    big L2 = big_add(&dr2, &dz2);
    return big_cmp_scaled(&X2, tol2, 28, &L2) <= 0;
}

/* CA curvature (pT_min, Sec. 3.2): circumradius of a, b, c at least rho_min:
 *   |ab|^2 |bc|^2 |ca|^2 >= 4 rho_min^2 O^2, O = (b-a) x (c-a). */
static int pred_curv(const ghit *a, const ghit *b, const ghit *c, float k_curv) {
    int64_t O = (b->x - a->x) * (c->y - a->y) - (b->y - a->y) * (c->x - a->x);
    int64_t ab = (b->x - a->x) * (b->x - a->x) + (b->y - a->y) * (b->y - a->y);
    int64_t bc = (c->x - b->x) * (c->x - b->x) + (c->y - b->y) * (c->y - b->y);
    int64_t ca = (a->x - c->x) * (a->x - c->x) + (a->y - c->y) * (a->y - c->y);
    big P = big_mul3(big_i64(ab), big_i64(bc), big_i64(ca));
    big o = big_i64(O);
    big o2 = big_mul(&o, &o);
    return big_cmp_scaled(&P, k_curv, 28, &o2) >= 0;
}

/* CA beamspot compatibility (R_max, Sec. 3.2): the circle through a, b, c
 * passes within R_max of the beam line.  With I the in-circle determinant of
 * (a, b, c, origin) one has |I| = |O| |pow| (pow = power of the origin) and
 * |pow| / (2 rho) = |I| / (|ab||bc||ca|) approximates the distance of closest
 * approach; the cut is  I^2 <= R_max^2 |ab|^2 |bc|^2 |ca|^2. */
static int pred_beamspot(const ghit *a, const ghit *b, const ghit *c, float rmax2) {
    big ax = big_i64(a->x), ay = big_i64(a->y), a2 = big_i64(a->x * a->x + a->y * a->y);
    big bx = big_i64(b->x), by = big_i64(b->y), b2 = big_i64(b->x * b->x + b->y * b->y);
    big cx = big_i64(c->x), cy = big_i64(c->y), c2 = big_i64(c->x * c->x + c->y * c->y);
    /* I = ax (by c2 - b2 cy) - ay (bx c2 - b2 cx) + a2 (bx cy - by cx) */
    big t1 = big_mul(&by, &c2), t2 = big_mul(&b2, &cy);
    big m1 = big_sub(&t1, &t2);
    big t3 = big_mul(&bx, &c2), t4 = big_mul(&b2, &cx);
    big m2 = big_sub(&t3, &t4);
    big t5 = big_mul(&bx, &cy), t6 = big_mul(&by, &cx);
    big m3 = big_sub(&t5, &t6);
    big s1 = big_mul(&ax, &m1), s2 = big_mul(&ay, &m2), s3 = big_mul(&a2, &m3);
    big I = big_sub(&s1, &s2);
    I = big_add(&I, &s3);
    big I2 = big_mul(&I, &I);
    int64_t ab = (b->x - a->x) * (b->x - a->x) + (b->y - a->y) * (b->y - a->y);
    int64_t bc = (c->x - b->x) * (c->x - b->x) + (c->y - b->y) * (c->y - b->y);
    int64_t ca = (a->x - c->x) * (a->x - c->x) + (a->y - c->y) * (a->y - c->y);
    big P = big_mul3(big_i64(ab), big_i64(bc), big_i64(ca));
    return big_cmp_scaled(&I2, rmax2, 28, &P) <= 0;
}

/* CA dz compatibility: the a-c line meets r = 0 within |z| <= zmax:
 *   |z_a r_c - z_c r_a| <= zmax (r_c - r_a). */
static int pred_dz(const ghit *a, const ghit *c, float zmax) {
    int64_t L = a->z * c->r - c->z * a->r;
    if (L < 0) L = -L;
    big b = big_i64(L), d = big_i64(c->r - a->r);
    return big_cmp_scaled(&b, zmax, 14, &d) <= 0;
}

/* Fishbone alignment (Sec. 3.3): cells (h1 -> h) and (h2 -> h) are aligned
 * when u = h1 - h and v = h2 - h point the same way within eps:
 *   u.v > 0 and |u x v|^2 <= eps^2 |u|^2 |v|^2 (3-D). */
static int pred_fb_aligned(const ghit *h1, const ghit *h2, const ghit *h, float eps2) {
    int64_t ux = h1->x - h->x, uy = h1->y - h->y, uz = h1->z - h->z;
    int64_t vx = h2->x - h->x, vy = h2->y - h->y, vz = h2->z - h->z;
    int64_t dot = ux * vx + uy * vy + uz * vz;
    if (dot <= 0) return 0;
    big cx = big_i64(uy * vz - uz * vy), cy = big_i64(uz * vx - ux * vz), cz = big_i64(ux * vy - uy * vx);
    big x2 = big_mul(&cx, &cx), y2 = big_mul(&cy, &cy), z2 = big_mul(&cz, &cz);
    big cr = big_add(&x2, &y2);
    cr = big_add(&cr, &z2);
    big u2 = big_i64(ux * ux + uy * uy + uz * uz), v2 = big_i64(vx * vx + vy * vy + vz * vz);
    big uv = big_mul(&u2, &v2);
    return big_cmp_scaled(&cr, eps2, 0, &uv) <= 0;
}

static int64_t len2_3d(const ghit *a, const ghit *b) {
    int64_t dx = a->x - b->x, dy = a->y - b->y, dz = a->z - b->z;
    return dx * dx + dy * dy + dz * dz;
}

/* exported single-predicate entry points (for the tests) */
int oracle_pred(int which, const float *h, int nh, float k) {
    ghit g[3];
    for (int i = 0; i < nh && i < 3; i++) g[i] = mk_ghit(h[4 * i], h[4 * i + 1], h[4 * i + 2], h[4 * i + 3]);
    switch (which) {
    case OR_PRED_PHIW: return pred_phiw(&g[0], &g[1], k);
    case OR_PRED_ZIP: return pred_zip(&g[0], &g[1], k);
    case OR_PRED_PT: return pred_pt(&g[0], &g[1], k);
    case OR_PRED_RZ: return pred_rz(&g[0], &g[1], &g[2], k);
    case OR_PRED_CURV: return pred_curv(&g[0], &g[1], &g[2], k);
    case OR_PRED_BEAMSPOT: return pred_beamspot(&g[0], &g[1], &g[2], k);
    case OR_PRED_DZ: return pred_dz(&g[0], &g[2], k);
    case OR_PRED_FB: return pred_fb_aligned(&g[0], &g[1], &g[2], k);
    default: return -1;
    }
}

/* ------------------------------------------------------------ growable arrays */
typedef struct { void *p; int64_t n, cap; size_t el; } vec;

static void vec_init(vec *v, size_t el) { v->p = NULL; v->n = 0; v->cap = 0; v->el = el; }
static void *vec_push(vec *v) {
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 1024;
        v->p = realloc(v->p, (size_t)v->cap * v->el);
        if (!v->p) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
    }
    return (char *)v->p + (size_t)(v->n++) * v->el;
}

/* ------------------------------------------------------------- broken line */
static void cholesky_solve(int n, double *A /* n*n, overwritten by L */, double *b /* n, overwritten */) {
    for (int j = 0; j < n; j++) {
        double s = A[j * n + j];
        for (int k = 0; k < j; k++) s -= A[j * n + k] * A[j * n + k];
        double d = sqrt(s > 0 ? s : 1e-300);
        A[j * n + j] = d;
        for (int i = j + 1; i < n; i++) {
            double t = A[i * n + j];
            for (int k = 0; k < j; k++) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / d;
        }
    }
    if (!b) return;
    for (int i = 0; i < n; i++) {
        double t = b[i];
        for (int k = 0; k < i; k++) t -= A[i * n + k] * b[k];
        b[i] = t / A[i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
        double t = b[i];
        for (int k = i + 1; k < n; k++) t -= A[k * n + i] * b[k];
        b[i] = t / A[i * n + i];
    }
}

static void chol_apply(int n, const double *L, double *b) {
    for (int i = 0; i < n; i++) {
        double t = b[i];
        for (int k = 0; k < i; k++) t -= L[i * n + k] * b[k];
        b[i] = t / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {
        double t = b[i];
        for (int k = i + 1; k < n; k++) t -= L[k * n + i] * b[k];
        b[i] = t / L[i * n + i];
    }
}

static double asinc(double x) {
    if (x > 1) x = 1;
    if (x < -1) x = -1;
    return x == 0 ? 1.0 : asin(x) / x;
}

/* Perigee of the circle through P with direction psi and signed curvature k
 * (left turning positive) with respect to the origin.  Outputs phi0 (not
 * wrapped), d0 (PCA = d0 (sin phi0, -cos phi0)) and the signed transverse arc
 * length from P to the PCA. */
static void perigee(double px, double py, double psi, double k, double *phi0, double *d0, double *arc) {
    double c = cos(psi), s = sin(psi);
    double Xo = -(px * c + py * s);
    double Yo = -(-px * s + py * c);
    double U = k * (Xo * Xo + Yo * Yo) - 2.0 * Yo;
    double q = 1.0 + k * U;
    *d0 = -U / (1.0 + sqrt(q > 0 ? q : 0));
    double dpsi = atan2(k * Xo, 1.0 - k * Yo);
    *phi0 = psi + dpsi;
    *arc = k != 0 ? dpsi / k : Xo;
}

static double wrap_pi(double a) {
    while (a > M_PI) a -= 2 * M_PI;
    while (a <= -M_PI) a += 2 * M_PI;
    return a;
}

/* circle parameters (kappa, phi0, d0) as a function of the circle-fit
 * unknowns (u0, u1, dk) around the reference (h0, psi0, k0). */
static void circ_map(double h0x, double h0y, double psi0, double k0, double ds1,
                     double u0, double u1, double dk, double out[3]) {
    double nx = -sin(psi0), ny = cos(psi0);
    double px = h0x + u0 * nx, py = h0y + u0 * ny;
    double psi = psi0 + (u1 - u0) / ds1 - dk * ds1 / 2;
    double k = k0 + dk;
    double phi0, d0, arc;
    perigee(px, py, psi, k, &phi0, &d0, &arc);
    out[0] = -k;
    out[1] = phi0;
    out[2] = d0;
}

/* 2-norm condition number max|l| / min|l| of a symmetric n x n matrix
 * (row-major, n <= OR_NMAX + 1) from its eigenvalues l, found by the cyclic
 * Jacobi method: plane rotations that zero the off-diagonal entries in turn
 * until their squared sum is negligible against the diagonal's. */
double oracle_sym_condition(int n, const double *M) {
    double a[(OR_NMAX + 1) * (OR_NMAX + 1)];
    if (n < 1 || n > OR_NMAX + 1) return -1;
    memcpy(a, M, sizeof(double) * n * n);
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0, diag = 0;
        for (int p = 0; p < n; p++)
            for (int q = 0; q < n; q++) {
                if (p == q) diag += a[p * n + q] * a[p * n + q];
                else off += a[p * n + q] * a[p * n + q];
            }
        if (off <= 1e-32 * diag) break;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                const double apq = a[p * n + q];
                if (apq == 0) continue;
                /* rotation angle with tan = t zeroing a[p][q]: t solves
                 * t^2 + 2 theta t - 1 = 0, theta = (a_qq - a_pp) / (2 a_pq) */
                const double theta = (a[q * n + q] - a[p * n + p]) / (2 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1));
                const double c = 1 / sqrt(t * t + 1), sn = t * c;
                for (int k = 0; k < n; k++) {          /* columns p, q */
                    const double akp = a[k * n + p], akq = a[k * n + q];
                    a[k * n + p] = c * akp - sn * akq;
                    a[k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {          /* rows p, q */
                    const double apk = a[p * n + k], aqk = a[q * n + k];
                    a[p * n + k] = c * apk - sn * aqk;
                    a[q * n + k] = sn * apk + c * aqk;
                }
            }
    }
    double lo = INFINITY, hi = 0;
    for (int i = 0; i < n; i++) {
        const double l = fabs(a[i * n + i]);
        if (l < lo) lo = l;
        if (l > hi) hi = l;
    }
    return lo > 0 ? hi / lo : INFINITY;
}

int oracle_fit(int n, const double *hx, const double *hy, const double *hz, const int *is_disk,
               const or_fitpar *fp, double *params, double *cov, double *chi2, int *ndf,
               double *extra /* optional [10]: chi2_line, chi2_circle, k0, psi0, tanl0, dk, arc, 0,
                                cond(line normal matrix), cond(circle normal matrix) */) {
    if (n < 3 || n > OR_NMAX) return -1;
    /* 1) pre-fit: circle through hits 0, n/2, n-1 */
    int ia = 0, ib = n / 2, ic = n - 1;
    double ax = hx[ia], ay = hy[ia], bx = hx[ib], by = hy[ib], cx = hx[ic], cy = hy[ic];
    double orient = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
    double dab = hypot(bx - ax, by - ay), dbc = hypot(cx - bx, cy - by), dca = hypot(ax - cx, ay - cy);
    double den = dab * dbc * dca;
    double k0 = den > 0 ? 2.0 * orient / den : 0.0;
    double alpha = atan2(by - ay, bx - ax);
    double hx_ = k0 * dab / 2;
    if (hx_ > 1) hx_ = 1;
    if (hx_ < -1) hx_ = -1;
    double psi0 = alpha - asin(hx_);
    double tx = cos(psi0), ty = sin(psi0), nx = -ty, ny = tx;
    double s[OR_NMAX], m[OR_NMAX], ds[OR_NMAX];
    for (int i = 0; i < n; i++) {
        double dx = hx[i] - hx[0], dy = hy[i] - hy[0];
        double dist = hypot(dx, dy);
        s[i] = dist * asinc(k0 * dist / 2);
        double X = dx * tx + dy * ty, Y = dx * nx + dy * ny;
        double U = k0 * (X * X + Y * Y) - 2 * Y;
        double q = 1 + k0 * U;
        m[i] = -U / (1 + sqrt(q > 0 ? q : 0));
    }
    ds[0] = 0;
    for (int i = 1; i < n; i++) {
        ds[i] = s[i] - s[i - 1];
        if (ds[i] < 1e-4) ds[i] = 1e-4;
    }
    double sl = s[n - 1] > 1e-4 ? s[n - 1] : 1e-4;
    double tanl0 = (hz[n - 1] - hz[0]) / sl;
    double sec2 = 1 + tanl0 * tanl0;
    double ak0 = fabs(k0) > 1e-7 ? fabs(k0) : 1e-7;
    double pt0 = 0.00299792458 * fp->bz / ak0;
    double p = pt0 * sqrt(sec2);
    double atl = fabs(tanl0) > 1e-3 ? fabs(tanl0) : 1e-3;
    /* 2) multiple-scattering variances at the inner hits (Highland) */
    double vb[OR_NMAX], vg[OR_NMAX];
    for (int i = 1; i < n - 1; i++) {
        double xx0 = is_disk[i] ? fp->x0_disk * sqrt(sec2) / atl : fp->x0_barrel * sqrt(sec2);
        double th = 0.0136 / p * sqrt(xx0) * (1 + 0.038 * log(xx0));
        double th2 = th * th * fp->ms_scale;
        vb[i] = th2 * sec2;
        vg[i] = th2 * sec2 * sec2;
        if (vb[i] < 1e-20) vb[i] = 1e-20;
        if (vg[i] < 1e-20) vg[i] = 1e-20;
    }
    /* 3) line fit in s-z */
    double A[(OR_NMAX + 1) * (OR_NMAX + 1)], rhs[OR_NMAX + 1], wz[OR_NMAX];
    memset(A, 0, sizeof A);
    for (int i = 0; i < n; i++) {
        double sz = is_disk[i] ? fp->sigma_r * atl : fp->sigma_z;
        wz[i] = 1 / (sz * sz);
        A[i * n + i] = wz[i];
        rhs[i] = wz[i] * hz[i];
    }
    for (int i = 1; i < n - 1; i++) {
        double g[3] = {1 / ds[i], -(1 / ds[i] + 1 / ds[i + 1]), 1 / ds[i + 1]};
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) A[(i - 1 + a) * n + (i - 1 + b)] += g[a] * g[b] / vg[i];
    }
    const double cond_line = extra ? oracle_sym_condition(n, A) : 0;
    double v[OR_NMAX];
    memcpy(v, rhs, sizeof(double) * n);
    cholesky_solve(n, A, v);
    double chi2l = 0;
    for (int i = 0; i < n; i++) chi2l += wz[i] * (v[i] - hz[i]) * (v[i] - hz[i]);
    for (int i = 1; i < n - 1; i++) {
        double gam = (v[i + 1] - v[i]) / ds[i + 1] - (v[i] - v[i - 1]) / ds[i];
        chi2l += gam * gam / vg[i];
    }
    double Cv[2][2];
    for (int c = 0; c < 2; c++) {
        double e[OR_NMAX];
        memset(e, 0, sizeof e);
        e[c] = 1;
        chol_apply(n, A, e);
        Cv[0][c] = e[0];
        Cv[1][c] = e[1];
    }
    /* 4) circle fit in the transverse plane: unknowns u_0..u_{n-1}, dk */
    int N = n + 1;
    double B[(OR_NMAX + 1) * (OR_NMAX + 1)], x[OR_NMAX + 1];
    memset(B, 0, sizeof B);
    double wu = 1 / (fp->sigma_rphi * fp->sigma_rphi);
    for (int i = 0; i < n; i++) {
        B[i * N + i] = wu;
        x[i] = wu * m[i];
    }
    x[n] = 0;
    for (int i = 1; i < n - 1; i++) {
        double h[4] = {1 / ds[i], -(1 / ds[i] + 1 / ds[i + 1]), 1 / ds[i + 1], -(ds[i] + ds[i + 1]) / 2};
        int idx[4] = {i - 1, i, i + 1, n};
        for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++) B[idx[a] * N + idx[b]] += h[a] * h[b] / vb[i];
    }
    const double cond_circle = extra ? oracle_sym_condition(N, B) : 0;
    cholesky_solve(N, B, x);
    double dk = x[n];
    double chi2c = 0;
    for (int i = 0; i < n; i++) chi2c += wu * (x[i] - m[i]) * (x[i] - m[i]);
    for (int i = 1; i < n - 1; i++) {
        double be = (x[i + 1] - x[i]) / ds[i + 1] - (x[i] - x[i - 1]) / ds[i] - dk * (ds[i] + ds[i + 1]) / 2;
        chi2c += be * be / vb[i];
    }
    double Cc[3][3];
    int sel[3] = {0, 1, n};
    for (int c = 0; c < 3; c++) {
        double e[OR_NMAX + 1];
        memset(e, 0, sizeof e);
        e[sel[c]] = 1;
        chol_apply(N, B, e);
        for (int r = 0; r < 3; r++) Cc[r][c] = e[sel[r]];
    }
    /* 5) final circle and perigee parameters */
    double k = k0 + dk;
    double px = hx[0] + x[0] * nx, py = hy[0] + x[0] * ny;
    double psi = psi0 + (x[1] - x[0]) / ds[1] - dk * ds[1] / 2;
    double phi0, d0, arc;
    perigee(px, py, psi, k, &phi0, &d0, &arc);
    double tanl = (v[1] - v[0]) / ds[1];
    double z0 = v[0] + tanl * arc;
    params[0] = -k;
    params[1] = wrap_pi(phi0);
    params[2] = tanl;
    params[3] = d0;
    params[4] = z0;
    /* 6) covariance: line block by its linear Jacobian, circle block by
     *    central differences of the circle map */
    double Jl[2][2] = {{-1 / ds[1], 1 / ds[1]}, {1 - arc / ds[1], arc / ds[1]}};
    double Cl[2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
            double t = 0;
            for (int c = 0; c < 2; c++)
                for (int d = 0; d < 2; d++) t += Jl[a][c] * Cv[c][d] * Jl[b][d];
            Cl[a][b] = t;
        }
    double Jc[3][3];
    double hstep[3] = {1e-5, 1e-5, 1e-7};
    double base[3] = {x[0], x[1], dk};
    for (int c = 0; c < 3; c++) {
        double up[3], dn[3], qp[3], qm[3];
        memcpy(up, base, sizeof up);
        memcpy(dn, base, sizeof dn);
        up[c] += hstep[c];
        dn[c] -= hstep[c];
        circ_map(hx[0], hy[0], psi0, k0, ds[1], up[0], up[1], up[2], qp);
        circ_map(hx[0], hy[0], psi0, k0, ds[1], dn[0], dn[1], dn[2], qm);
        for (int r = 0; r < 3; r++) Jc[r][c] = (qp[r] - qm[r]) / (2 * hstep[c]);
    }
    double Ccirc[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double t = 0;
            for (int c = 0; c < 3; c++)
                for (int d = 0; d < 3; d++) t += Jc[a][c] * Cc[c][d] * Jc[b][d];
            Ccirc[a][b] = t;
        }
    /* full 5x5 in the order (kappa, phi0, tanl, d0, z0) */
    double F[5][5];
    memset(F, 0, sizeof F);
    int ci[3] = {0, 1, 3}, li[2] = {2, 4};
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) F[ci[a]][ci[b]] = Ccirc[a][b];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) F[li[a]][li[b]] = Cl[a][b];
    int t = 0;
    for (int a = 0; a < 5; a++)
        for (int b = 0; b <= a; b++) cov[t++] = F[a][b];
    *chi2 = chi2l + chi2c;
    *ndf = 2 * n - 5;
    if (extra) {
        extra[0] = chi2l;
        extra[1] = chi2c;
        extra[2] = k0;
        extra[3] = psi0;
        extra[4] = tanl0;
        extra[5] = dk;
        extra[6] = arc;
        extra[7] = 0;
        extra[8] = cond_line;
        extra[9] = cond_circle;
    }
    return 0;
}

/* ------------------------------------------------------------- full chain */
typedef struct { int32_t inner, outer; int32_t pair; } cellrec;

static void emit(int ncells, const int32_t *path, const cellrec *cells, vec *tup) {
    or_tuple *t = (or_tuple *)vec_push(tup);
    memset(t, 0, sizeof *t);
    t->n = ncells + 1;
    t->hits[0] = cells[path[0]].inner;
    for (int i = 0; i < ncells; i++) {
        t->hits[i + 1] = cells[path[i]].outer;
        t->cells[i] = path[i];
    }
}

/* Depth-first search from a root cell: every path that cannot be extended
 * (its last cell has no outer neighbour) is emitted when it has >= 3 hits;
 * a path that reaches the hit limit nmax is emitted there. */
static void dfs(int32_t c, int depth, int32_t *path, const int64_t *out_off, const int64_t *out_idx,
                const cellrec *cells, vec *tup, const int nmax) {
    path[depth] = c;
    int ncells = depth + 1;
    int64_t b = out_off[c], e = out_off[c + 1];
    if (b == e) {
        if (ncells + 1 >= 3) emit(ncells, path, cells, tup);
        return;
    }
    if (ncells + 1 == nmax) {
        emit(ncells, path, cells, tup);
        return;
    }
    for (int64_t q = b; q < e; q++) dfs((int32_t)out_idx[q], depth + 1, path, out_off, out_idx, cells, tup, nmax);
}

int oracle_run(const or_input *in, int max_stage, or_result *res) {
    memset(res, 0, sizeof *res);
    const or_cuts *cu = in->cuts;
    vec cells, alive, edges, tups;
    vec_init(&cells, sizeof(cellrec));
    vec_init(&alive, 1);
    vec_init(&edges, sizeof(int64_t) * 2);
    vec_init(&tups, sizeof(or_tuple));
    int32_t nh = in->n_hits;
    int32_t *layer = (int32_t *)malloc(sizeof(int32_t) * (nh > 0 ? nh : 1));
    ghit *g = (ghit *)malloc(sizeof(ghit) * (nh > 0 ? nh : 1));
    for (int32_t i = 0; i < nh; i++) {
        int32_t mod = in->module[i];
        if (mod < 0 || mod >= in->n_modules) { free(layer); free(g); return -2; }
        layer[i] = in->module_layer[mod];
        g[i] = mk_ghit(in->x[i], in->y[i], in->z[i], in->r[i]);
    }
    for (int32_t ev = 0; ev < in->n_events; ev++) {
        int32_t h0 = in->ev_off[ev], h1 = in->ev_off[ev + 1];
        int64_t cell_base = cells.n;
        /* hits of this event on each layer */
        int32_t nev = h1 - h0;
        int32_t *lay_off = (int32_t *)calloc(OR_NLAYERS + 1, sizeof(int32_t));
        int32_t *lay_hit = (int32_t *)malloc(sizeof(int32_t) * (nev > 0 ? nev : 1));
        for (int32_t i = h0; i < h1; i++) lay_off[layer[i] + 1]++;
        for (int L = 0; L < OR_NLAYERS; L++) lay_off[L + 1] += lay_off[L];
        {
            int32_t fillp[OR_NLAYERS];
            for (int L = 0; L < OR_NLAYERS; L++) fillp[L] = lay_off[L];
            for (int32_t i = h0; i < h1; i++) lay_hit[fillp[layer[i]]++] = i;
        }
        /* --- stage 1: doublets (every inner hit against every outer hit of
         * the pair's two layers) */
        for (int p = 0; p < cu->n_pairs; p++) {
            const or_pair *pp = &cu->pair[p];
            for (int32_t qo = lay_off[pp->outer]; qo < lay_off[pp->outer + 1]; qo++) {
                int32_t o = lay_hit[qo];
                for (int32_t qi = lay_off[pp->inner]; qi < lay_off[pp->inner + 1]; qi++) {
                    int32_t i = lay_hit[qi];
                    if (!pred_zw(in->z[i], pp->zlo, pp->zhi)) continue;
                    if (!pred_zip(&g[i], &g[o], pp->zmax)) continue;
                    if (!pred_phiw(&g[i], &g[o], pp->tan2_dphi)) continue;
                    if (!pred_pt(&g[i], &g[o], pp->k_pt)) continue;
                    cellrec *c = (cellrec *)vec_push(&cells);
                    c->inner = i;
                    c->outer = o;
                    c->pair = p;
                    *(uint8_t *)vec_push(&alive) = 1;
                }
            }
        }
        free(lay_off);
        free(lay_hit);
        int64_t nc = cells.n - cell_base;
        cellrec *C = (cellrec *)cells.p + cell_base;
        uint8_t *A = (uint8_t *)alive.p + cell_base;
        /* cells of this event listed by their outer hit */
        int64_t *by_out_off = (int64_t *)calloc((size_t)nev + 1, sizeof(int64_t));
        int64_t *by_out = (int64_t *)malloc(sizeof(int64_t) * (nc > 0 ? nc : 1));
        for (int64_t c = 0; c < nc; c++) by_out_off[C[c].outer - h0 + 1]++;
        for (int32_t i = 0; i < nev; i++) by_out_off[i + 1] += by_out_off[i];
        {
            int64_t *fp2 = (int64_t *)malloc(sizeof(int64_t) * ((size_t)nev + 1));
            for (int32_t i = 0; i <= nev; i++) fp2[i] = by_out_off[i];
            for (int64_t c = 0; c < nc; c++) by_out[fp2[C[c].outer - h0]++] = c;
            free(fp2);
        }
        /* --- Fishbone: a cell dies when an aligned sibling (same outer hit,
         * inner hit on the same layer) is strictly shorter, or equally long
         * with a smaller inner hit index. */
        uint8_t *kill = (uint8_t *)calloc(nc > 0 ? nc : 1, 1);
        for (int64_t c = 0; c < nc; c++) {
            int32_t ho = C[c].outer - h0;
            for (int64_t q = by_out_off[ho]; q < by_out_off[ho + 1]; q++) {
                int64_t d = by_out[q];
                if (d == c) continue;
                if (layer[C[d].inner] != layer[C[c].inner]) continue;
                if (!pred_fb_aligned(&g[C[c].inner], &g[C[d].inner], &g[C[c].outer], cu->fishbone_eps2)) continue;
                int64_t lc = len2_3d(&g[C[c].inner], &g[C[c].outer]);
                int64_t ld = len2_3d(&g[C[d].inner], &g[C[d].outer]);
                if (ld < lc || (ld == lc && C[d].inner < C[c].inner)) { kill[c] = 1; break; }
            }
        }
        for (int64_t c = 0; c < nc; c++) A[c] = !kill[c];
        free(kill);
        if (max_stage < 2) { free(by_out_off); free(by_out); continue; }
        /* --- stage 2: CA connection of live cells (a,b) -> (b,c) */
        int64_t edge_base = edges.n;
        for (int64_t co = 0; co < nc; co++) {
            if (!A[co]) continue;
            int32_t b = C[co].inner, c = C[co].outer;
            int reg = in->layer_is_disk[layer[b]] ? 1 : 0;
            const or_region *rg = &cu->region[reg];
            int32_t hb = b - h0;
            for (int64_t q = by_out_off[hb]; q < by_out_off[hb + 1]; q++) {
                int64_t ci = by_out[q];
                if (!A[ci]) continue;
                int32_t a = C[ci].inner;
                if (!pred_dz(&g[a], &g[c], rg->zmax)) continue;
                if (!pred_rz(&g[a], &g[b], &g[c], rg->tol_rz2)) continue;
                if (!pred_curv(&g[a], &g[b], &g[c], rg->k_curv)) continue;
                if (!pred_beamspot(&g[a], &g[b], &g[c], rg->rmax2)) continue;
                int64_t *e = (int64_t *)vec_push(&edges);
                e[0] = cell_base + ci;
                e[1] = cell_base + co;
            }
        }
        free(by_out_off);
        free(by_out);
        if (max_stage < 3) continue;
        /* --- stage 3: roots and depth-first search over the cell DAG */
        int64_t ne = edges.n - edge_base;
        int64_t *E = (int64_t *)edges.p + 2 * edge_base;
        int64_t *out_off = (int64_t *)calloc(nc + 1, sizeof(int64_t));
        int64_t *out_idx = (int64_t *)malloc(sizeof(int64_t) * (ne > 0 ? ne : 1));
        uint8_t *has_in = (uint8_t *)calloc(nc > 0 ? nc : 1, 1);
        for (int64_t q = 0; q < ne; q++) {
            out_off[E[2 * q] - cell_base + 1]++;
            has_in[E[2 * q + 1] - cell_base] = 1;
        }
        for (int64_t c = 0; c < nc; c++) out_off[c + 1] += out_off[c];
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (nc > 0 ? nc : 1));
        for (int64_t c = 0; c < nc; c++) fill[c] = out_off[c];
        for (int64_t q = 0; q < ne; q++) out_idx[fill[E[2 * q] - cell_base]++] = E[2 * q + 1] - cell_base;
        free(fill);
        int64_t tup_base = tups.n;
        int32_t path[OR_NMAX];
        for (int64_t c = 0; c < nc; c++) {
            if (!A[c]) continue;
            int li = layer[C[c].inner];
            int root = (li == 0) || ((li == 1 || li == 4 || li == 7) && !has_in[c]);
            if (!root) continue;
            dfs((int32_t)c, 0, path, out_off, out_idx, C, &tups, OR_NMAX);
        }
        /* translate event-local cell ids into batch-wide ones */
        for (int64_t t = tup_base; t < tups.n; t++) {
            or_tuple *tp = (or_tuple *)tups.p + t;
            for (int i = 0; i < tp->n - 1; i++) tp->cells[i] += (int32_t)cell_base;
        }
        free(out_off);
        free(out_idx);
        free(has_in);
    }
    int64_t nt = tups.n;
    or_tuple *T = (or_tuple *)tups.p;
    uint8_t *tal = (uint8_t *)malloc(nt > 0 ? nt : 1);
    if (max_stage >= 3) {
        /* --- shared-doublet cleaning: L(c) = max hits of tuples using c */
        uint8_t *L = (uint8_t *)calloc(cells.n > 0 ? cells.n : 1, 1);
        for (int64_t t = 0; t < nt; t++)
            for (int i = 0; i < T[t].n - 1; i++)
                if (L[T[t].cells[i]] < T[t].n) L[T[t].cells[i]] = (uint8_t)T[t].n;
        for (int64_t t = 0; t < nt; t++) {
            int ok = 1;
            for (int i = 0; i < T[t].n - 1; i++)
                if (T[t].n < L[T[t].cells[i]]) ok = 0;
            tal[t] = (uint8_t)ok;
        }
        free(L);
    }
    /* --- stage 4: broken-line fit of surviving tuples with >= min_hits */
    vec trk, par, cv, ch, nd;
    vec_init(&trk, sizeof(int64_t));
    vec_init(&par, sizeof(double) * 5);
    vec_init(&cv, sizeof(double) * 15);
    vec_init(&ch, sizeof(double));
    vec_init(&nd, sizeof(int32_t));
    if (max_stage >= 4) {
        for (int64_t t = 0; t < nt; t++) {
            if (!tal[t] || T[t].n < cu->min_hits) continue;
            double hx[OR_NMAX], hy[OR_NMAX], hz[OR_NMAX];
            int dk[OR_NMAX];
            for (int i = 0; i < T[t].n; i++) {
                int32_t h = T[t].hits[i];
                hx[i] = in->x[h];
                hy[i] = in->y[h];
                hz[i] = in->z[h];
                dk[i] = in->layer_is_disk[layer[h]];
            }
            double *pp = (double *)vec_push(&par);
            double *cc = (double *)vec_push(&cv);
            double *c2 = (double *)vec_push(&ch);
            int32_t *nn = (int32_t *)vec_push(&nd);
            int ndf;
            oracle_fit(T[t].n, hx, hy, hz, dk, in->fitpar, pp, cc, c2, &ndf, NULL);
            *nn = ndf;
            *(int64_t *)vec_push(&trk) = t;
        }
    }
    res->n_cells = cells.n;
    res->cells = (int32_t *)malloc(sizeof(int32_t) * 3 * (cells.n > 0 ? cells.n : 1));
    for (int64_t c = 0; c < cells.n; c++) {
        cellrec *cr = (cellrec *)cells.p + c;
        res->cells[3 * c] = cr->inner;
        res->cells[3 * c + 1] = cr->outer;
        res->cells[3 * c + 2] = cr->pair;
    }
    free(cells.p);
    res->cell_alive = (uint8_t *)alive.p;
    res->n_edges = edges.n;
    res->edges = (int64_t *)edges.p;
    res->n_tuples = nt;
    res->tuples = T;
    res->tuple_alive = tal;
    res->n_tracks = trk.n;
    res->track_tuple = (int64_t *)trk.p;
    res->params = (double *)par.p;
    res->cov = (double *)cv.p;
    res->chi2 = (double *)ch.p;
    res->ndf = (int32_t *)nd.p;
    free(layer);
    free(g);
    return 0;
}

void oracle_free(or_result *res) {
    free(res->cells);
    free(res->cell_alive);
    free(res->edges);
    free(res->tuples);
    free(res->tuple_alive);
    free(res->track_tuple);
    free(res->params);
    free(res->cov);
    free(res->chi2);
    free(res->ndf);
    memset(res, 0, sizeof *res);
}
