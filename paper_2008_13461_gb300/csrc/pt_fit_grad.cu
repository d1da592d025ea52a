// Adjoint of the broken-line fit (Sec. 3.4): the gradient of a scalar loss
// with respect to the hit coordinates, given the loss's gradient with
// respect to each track's parameters (kappa, phi0, tan lambda, d0, z0) and
// chi2.  One thread per track recomputes the fit in float64 (nothing of the
// forward pass is stored) and runs it backwards:
//
//  * the solutions of the normal equations A v = b (line) and B x = b
//    (circle): with xbar the adjoint of the solution, bbar = A^-1 xbar (one
//    more solve with the same Cholesky factor) and Abar = -bbar x^T, pushed
//    through the assembly of A and b to the weights, the kink coefficients
//    and the measurements;
//  * chi2 at the minimum: by the envelope theorem its derivative with
//    respect to any input is the partial derivative of the objective at the
//    fixed solution, so it needs no solve;
//  * every scalar step (pre-fit circle, arc lengths, offsets from the
//    pre-fit circle, scattering weights, perigee) by its chain rule.
//
// Clamps of the forward pass (segment length, curvature, scattering
// variance, |tan lambda|, asin arguments) have zero derivative where active.
// The gradients are added into per-hit arrays with atomics (a hit can belong
// to several tracks).  The alignment transform of the hits and its adjoint
// are here too.
#include "pt_common.cuh"
#include "pt_kernels.cuh"

namespace ptk {
namespace {

template <int M>
__device__ __forceinline__ int pk(int r, int c) { return r >= c ? r * (r + 1) / 2 + c : c * (c + 1) / 2 + r; }

// Reciprocal, reciprocal square root and square root from a float32 seed and
// one Newton step (relative error about 1e-14): a few FP64 multiply-adds
// instead of the full IEEE sequences on the slow FP64 pipe.  Used where the
// argument is nonzero and well inside the float32 range (lengths, weights,
// variances); sqrt_d(0) = 0.
__device__ __forceinline__ double rcp_d(double x) {
    const double r = (double)__frcp_rn((float)x);
    return r * (2.0 - x * r);
}
__device__ __forceinline__ double rsqrt_d(double x) {
    const double y = (double)rsqrtf((float)x);
    return y * (1.5 - 0.5 * x * y * y);
}
__device__ __forceinline__ double sqrt_d(double x) { return x > 0.0 ? x * rsqrt_d(x) : 0.0; }

// Cholesky in place (packed lower triangle), inverse diagonal stored
template <int M>
__device__ __forceinline__ void chol_d(double *A) {
#pragma unroll
    for (int j = 0; j < M; j++) {
        double s = A[pk<M>(j, j)];
#pragma unroll
        for (int k = 0; k < j; k++) s -= A[pk<M>(j, k)] * A[pk<M>(j, k)];
        const double id = rsqrt_d(s > 1e-30 ? s : 1e-30);
        A[pk<M>(j, j)] = id;
#pragma unroll
        for (int i = j + 1; i < M; i++) {
            double t = A[pk<M>(i, j)];
#pragma unroll
            for (int k = 0; k < j; k++) t -= A[pk<M>(i, k)] * A[pk<M>(j, k)];
            A[pk<M>(i, j)] = t * id;
        }
    }
}

// b := (L L^T)^-1 b
template <int M>
__device__ __forceinline__ void solve_d(const double *L, double *b) {
#pragma unroll
    for (int i = 0; i < M; i++) {
        double t = b[i];
#pragma unroll
        for (int k = 0; k < i; k++) t -= L[pk<M>(i, k)] * b[k];
        b[i] = t * L[pk<M>(i, i)];
    }
#pragma unroll
    for (int i = M - 1; i >= 0; i--) {
        double t = b[i];
#pragma unroll
        for (int k = i + 1; k < M; k++) t -= L[pk<M>(k, i)] * b[k];
        b[i] = t * L[pk<M>(i, i)];
    }
}

// asin(q)/q, keeping asin(q) in `as` for the derivative (q clamped to
// [-1, 1] by the caller; below 1e-4 the series, and `as` is not needed)
__device__ __forceinline__ double asinc_d(double q, double &as) {
    if (fabs(q) < 1e-4) {
        as = q;
        return 1.0 + q * q * (1.0 / 6.0);
    }
    as = asin(q);
    return as * rcp_d(q);
}
// d/dq of asin(q)/q, given as = asin(q)
__device__ __forceinline__ double dasinc_d(double q, double as) {
    if (fabs(q) < 1e-4) return q * (1.0 / 3.0);
    if (fabs(q) >= 1.0) return 0.0;
    return (q * rsqrt_d(1.0 - q * q) - as) * rcp_d(q * q);
}

template <int N>
__device__ void grad_track(const Params &p, int32_t t, const float *gp, float gc, float *gx, float *gy, float *gz) {
    constexpr int M = N + 1;
    const int32_t *hid = p.tup_hits + (int64_t)t * PT_NMAX;
    double x[N], y[N], z[N];
    bool disk[N];
#pragma unroll
    for (int i = 0; i < N; i++) {
        const int h = hid[i];
        x[i] = p.x[h];
        y[i] = p.y[h];
        z[i] = p.z[h];
        disk[i] = p.layer[p.module_layer[p.module[h]]].kind == PT_LAYER_DISK;
    }
    const double bz = p.fit.bz;
    // ---------------- forward, float64 ----------------
    // 1) pre-fit circle through hits 0, n/2, n-1
    constexpr int ib = N / 2, ic = N - 1;
    const double abx = x[ib] - x[0], aby = y[ib] - y[0];
    const double acx = x[ic] - x[0], acy = y[ic] - y[0];
    const double bcx = x[ic] - x[ib], bcy = y[ic] - y[ib];
    const double orient = abx * acy - aby * acx;
    const double dab = sqrt_d(abx * abx + aby * aby), dbc = sqrt_d(bcx * bcx + bcy * bcy);
    const double dca = sqrt_d(acx * acx + acy * acy);
    const double den = dab * dbc * dca;
    const double iden = den > 0.0 ? rcp_d(den) : 0.0;
    const double k0 = 2.0 * orient * iden;
    const double ta = 0.5 * k0 * dab;
    const bool ta_in = fabs(ta) < 1.0;
    const double tac = fmin(fmax(ta, -1.0), 1.0);
    // sin and cos of psi0 = atan2(aby, abx) - asin(ta) by the angle
    // difference formula: (ex, ey) = (cos, sin) of the first, (ct, ta) of
    // the second (nothing needs the angle itself)
    const double idab0 = dab > 0.0 ? rcp_d(dab) : 0.0;
    const double ex = dab > 0.0 ? abx * idab0 : 1.0, ey = aby * idab0;
    const double ct = sqrt_d(1.0 - tac * tac);
    const double cs = ex * ct + ey * tac, sn = ey * ct - ex * tac;
    // arc lengths and offsets from the pre-fit circle
    double s[N], m[N], dxs[N], dys[N], dist[N], qs[N], Xs[N], Ys[N], Us[N], Sq[N], i1Sq[N], asc[N], asq[N];
#pragma unroll
    for (int i = 0; i < N; i++) {
        dxs[i] = x[i] - x[0];
        dys[i] = y[i] - y[0];
        dist[i] = sqrt_d(dxs[i] * dxs[i] + dys[i] * dys[i]);
        qs[i] = fmin(fmax(0.5 * k0 * dist[i], -1.0), 1.0);
        asc[i] = asinc_d(qs[i], asq[i]);
        s[i] = dist[i] * asc[i];
        // the pre-fit circle passes through hits 0, n/2 and n-1: their
        // offsets are zero for any position of the hits
        if (i == 0 || i == ib || i == ic) {
            m[i] = 0.0;
        } else {
            Xs[i] = dxs[i] * cs + dys[i] * sn;
            Ys[i] = dys[i] * cs - dxs[i] * sn;
            Us[i] = k0 * (Xs[i] * Xs[i] + Ys[i] * Ys[i]) - 2.0 * Ys[i];
            Sq[i] = sqrt_d(fmax(1.0 + k0 * Us[i], 0.0));
            i1Sq[i] = rcp_d(1.0 + Sq[i]);
            m[i] = -Us[i] * i1Sq[i];
        }
    }
    double ds[N], ids[N];
    ds[0] = 0.0;
    ids[0] = 0.0;
#pragma unroll
    for (int i = 1; i < N; i++) {
        ds[i] = fmax(s[i] - s[i - 1], 1e-4);
        ids[i] = rcp_d(ds[i]);
    }
    const double Sl = fmax(s[N - 1], 1e-4);
    const double iSl = rcp_d(Sl);
    const double tanl0 = (z[N - 1] - z[0]) * iSl;
    const double sec2 = 1.0 + tanl0 * tanl0, rsec = sqrt_d(sec2);
    const double ak = fmax(fabs(k0), 1e-7), iak = rcp_d(ak);
    const double pt0 = 0.00299792458 * bz * iak;
    const double pmom = pt0 * rsec, ipmom = rcp_d(pmom);
    const double atl = fmax(fabs(tanl0), 1e-3), iatl = rcp_d(atl);
    // 2) scattering weights of the kinks at hits 1 .. n-2
    double vb[N], vg[N], th[N], xx0[N], lx0[N];
#pragma unroll
    for (int i = 0; i < N; i++) vb[i] = vg[i] = th[i] = xx0[i] = lx0[i] = 0.0;
#pragma unroll
    for (int i = 1; i < N - 1; i++) {
        xx0[i] = disk[i] ? p.fit.x0_disk * rsec * iatl : p.fit.x0_barrel * rsec;
        lx0[i] = log(xx0[i]);
        th[i] = 0.0136 * ipmom * sqrt_d(xx0[i]) * (1.0 + 0.038 * lx0[i]);
        vb[i] = rcp_d(fmax(th[i] * th[i] * sec2, 1e-20));
        vg[i] = rcp_d(fmax(th[i] * th[i] * sec2 * sec2, 1e-20));
    }
    // 3) line fit: A v = b
    double wz[N], vz[N], A[N * (N + 1) / 2], v[N];
#pragma unroll
    for (int i = 0; i < N * (N + 1) / 2; i++) A[i] = 0.0;
#pragma unroll
    for (int i = 0; i < N; i++) {
        const double sz = disk[i] ? (double)p.fit.sigma_r * atl : (double)p.fit.sigma_z;
        vz[i] = sz * sz;
        wz[i] = rcp_d(vz[i]);
        A[pk<N>(i, i)] = wz[i];
        v[i] = wz[i] * z[i];
    }
#pragma unroll
    for (int i = 1; i < N - 1; i++) {
        const double g[3] = {ids[i], -(ids[i] + ids[i + 1]), ids[i + 1]};
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int c = 0; c <= a; c++) A[pk<N>(i - 1 + a, i - 1 + c)] += vg[i] * g[a] * g[c];
    }
    // Three hits: one kink per plane.  A = diag(wz) + vg_1 g g^T is
    // inverted by Sherman-Morrison; B = wu diag(1, 1, 1, 0) + vb_1 h h^T has
    // the explicit inverse [[I, a], [a^T, |a|^2 + var_1 wu / h3^2]] / wu with
    // a = -(h0, h1, h2) / h3.  Four hits: two kinks per plane; A^-1 by
    // Woodbury (a 2 x 2 system), B^-1 through the Schur complement of its
    // curvature entry, a rank-one update of wu I (the forward fit's closed
    // forms).  Otherwise Cholesky.
    auto solve_line = [&](double *yv) {
        if constexpr (N == 3) {
            const double g0 = ids[1], g2 = ids[2], g1 = -(g0 + g2);
            const double r0 = vz[0], r1 = vz[1], r2 = vz[2];
            const double kz = fmax(th[1] * th[1] * sec2 * sec2, 1e-20);
            const double w0 = r0 * yv[0], w1 = r1 * yv[1], w2 = r2 * yv[2];
            const double f = (g0 * w0 + g1 * w1 + g2 * w2) * rcp_d(kz + g0 * g0 * r0 + g1 * g1 * r1 + g2 * g2 * r2);
            yv[0] = w0 - r0 * g0 * f;
            yv[1] = w1 - r1 * g1 * f;
            yv[2] = w2 - r2 * g2 * f;
        } else if constexpr (N == 4) {
            // A^-1 y = w - D^-1 G^T S^-1 G w, w = D^-1 y, S = diag(var_k) + G D^-1 G^T
            const double a0 = ids[1], a2 = ids[2], a1 = -(a0 + a2);      // kink 1 on 0, 1, 2
            const double b0 = ids[2], b2 = ids[3], b1 = -(b0 + b2);      // kink 2 on 1, 2, 3
            const double kz1 = fmax(th[1] * th[1] * sec2 * sec2, 1e-20), kz2 = fmax(th[2] * th[2] * sec2 * sec2, 1e-20);
            const double w0 = vz[0] * yv[0], w1 = vz[1] * yv[1], w2 = vz[2] * yv[2], w3 = vz[3] * yv[3];
            const double S11 = kz1 + a0 * a0 * vz[0] + a1 * a1 * vz[1] + a2 * a2 * vz[2];
            const double S22 = kz2 + b0 * b0 * vz[1] + b1 * b1 * vz[2] + b2 * b2 * vz[3];
            const double S12 = a1 * b0 * vz[1] + a2 * b1 * vz[2];
            const double q1 = a0 * w0 + a1 * w1 + a2 * w2, q2 = b0 * w1 + b1 * w2 + b2 * w3;
            const double idet = rcp_d(S11 * S22 - S12 * S12);
            const double r1 = (S22 * q1 - S12 * q2) * idet, r2 = (S11 * q2 - S12 * q1) * idet;
            yv[0] = w0 - vz[0] * a0 * r1;
            yv[1] = w1 - vz[1] * (a1 * r1 + b0 * r2);
            yv[2] = w2 - vz[2] * (a2 * r1 + b1 * r2);
            yv[3] = w3 - vz[3] * b2 * r2;
        } else {
            solve_d<N>(A, yv);
        }
    };
    if constexpr (N > 4) chol_d<N>(A);
    solve_line(v);
    // 4) circle fit: B x = b, x = (u_0 .. u_{n-1}, dk).  Three hits: the
    // pre-fit circle passes through all of them, so the offsets m are zero
    // for any position of the hits, the fit returns u = 0, dk = 0 (its kink
    // and chi2 vanish) and the track is that circle: nothing of the circle
    // fit depends on the hits, and its backward pass is skipped below.
    const double wu = rcp_d((double)p.fit.sigma_rphi * p.fit.sigma_rphi);
    double B[M * (M + 1) / 2], xs[M];
#pragma unroll
    for (int i = 0; i < M * (M + 1) / 2; i++) B[i] = 0.0;
#pragma unroll
    for (int i = 0; i < N; i++) {
        B[pk<M>(i, i)] = wu;
        xs[i] = wu * m[i];
    }
    xs[N] = 0.0;
#pragma unroll
    for (int i = 1; i < N - 1; i++) {
        const double h[4] = {ids[i], -(ids[i] + ids[i + 1]), ids[i + 1], -0.5 * (ds[i] + ds[i + 1])};
        const int at[4] = {i - 1, i, i + 1, N};
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int c = 0; c <= a; c++) B[pk<M>(at[a], at[c])] += vb[i] * h[a] * h[c];
    }
    auto solve_circle = [&](double *yv) {
        if constexpr (N == 3) {
            const double h0 = ids[1], h2 = ids[2], h1 = -(h0 + h2), ih3 = rcp_d(-0.5 * (ds[1] + ds[2]));
            const double a0 = -h0 * ih3, a1 = -h1 * ih3, a2 = -h2 * ih3;
            const double s2 = (double)p.fit.sigma_rphi * p.fit.sigma_rphi, kv = fmax(th[1] * th[1] * sec2, 1e-20);
            const double ay = a0 * yv[0] + a1 * yv[1] + a2 * yv[2], y3 = yv[3];
            yv[0] = s2 * (yv[0] + a0 * y3);
            yv[1] = s2 * (yv[1] + a1 * y3);
            yv[2] = s2 * (yv[2] + a2 * y3);
            yv[3] = s2 * ay + (s2 * (a0 * a0 + a1 * a1 + a2 * a2) + kv * ih3 * ih3) * y3;
        } else if constexpr (N == 4) {
            // B = [[S0, A12], [A12^T, C]] over (u, dk); with t = -A12 / C the
            // Schur complement S = S0 - A12 A12^T / C = wu I + w' c c^T (c =
            // H^T (h3_2, -h3_1), w' = 1 / (h3_1^2 var_2 + h3_2^2 var_1)), so
            // B^-1 (y, yd) = (S^-1 (y + t yd), t . S^-1 (y + t yd) + yd / C).
            const double h0 = ids[1], h2 = ids[2], h1 = -(h0 + h2);      // kink 1 on u0, u1, u2
            const double k0 = ids[2], k2 = ids[3], k1 = -(k0 + k2);      // kink 2 on u1, u2, u3
            const double g1 = -0.5 * (ds[1] + ds[2]), g2 = -0.5 * (ds[2] + ds[3]);
            const double kv1 = fmax(th[1] * th[1] * sec2, 1e-20), kv2 = fmax(th[2] * th[2] * sec2, 1e-20);
            const double wp = rcp_d(g1 * g1 * kv2 + g2 * g2 * kv1);
            const double c0 = g2 * h0, c1 = g2 * h1 - g1 * k0, c2 = g2 * h2 - g1 * k1, c3 = -g1 * k2;
            const double p1 = g1 * kv2 * wp, p2 = g2 * kv1 * wp;
            const double t0 = -p1 * h0, t1 = -(p1 * h1 + p2 * k0), t2 = -(p1 * h2 + p2 * k1), t3 = -p2 * k2;
            const double yd = yv[4];
            const double e0 = yv[0] + t0 * yd, e1 = yv[1] + t1 * yd, e2 = yv[2] + t2 * yd, e3 = yv[3] + t3 * yd;
            const double iwu = rcp_d(wu);
            const double f = wp * (c0 * e0 + c1 * e1 + c2 * e2 + c3 * e3) *
                             rcp_d(wu + wp * (c0 * c0 + c1 * c1 + c2 * c2 + c3 * c3));
            yv[0] = (e0 - f * c0) * iwu;
            yv[1] = (e1 - f * c1) * iwu;
            yv[2] = (e2 - f * c2) * iwu;
            yv[3] = (e3 - f * c3) * iwu;
            yv[4] = t0 * yv[0] + t1 * yv[1] + t2 * yv[2] + t3 * yv[3] + yd * kv1 * kv2 * wp;
        } else {
            solve_d<M>(B, yv);
        }
    };
    if constexpr (N != 3) {
        if constexpr (N > 4) chol_d<M>(B);
        solve_circle(xs);
    } else {
#pragma unroll
        for (int i = 0; i < M; i++) xs[i] = 0.0;
    }
    const double dk = xs[N];
    // 5) perigee
    const double kf = k0 + dk;
    const double px = x[0] - xs[0] * sn, py = y[0] + xs[0] * cs;
    // psi = psi0 + dl, dl = (u1 - u0) ids1 - dk ds1 / 2 (for triplets
    // dl = 0): its sin and cos from those of psi0 and of dl (Maclaurin
    // series while |dl| < 1e-2, where their next terms are below 1e-21)
    double sp = sn, cp = cs;
    if constexpr (N != 3) {
        const double dl = (xs[1] - xs[0]) * ids[1] - dk * 0.5 * ds[1];
        double sd, cd;
        if (fabs(dl) < 1e-2) {
            const double d2 = dl * dl;
            sd = dl * (1.0 - d2 * (1.0 / 6.0) * (1.0 - d2 * (1.0 / 20.0) * (1.0 - d2 * (1.0 / 42.0))));
            cd = 1.0 - d2 * 0.5 * (1.0 - d2 * (1.0 / 12.0) * (1.0 - d2 * (1.0 / 30.0) * (1.0 - d2 * (1.0 / 56.0))));
        } else {
            sincos(dl, &sd, &cd);
        }
        sp = sn * cd + cs * sd;
        cp = cs * cd - sn * sd;
    }
    const double Xo = -(px * cp + py * sp), Yo = px * sp - py * cp;
    const double U = kf * (Xo * Xo + Yo * Yo) - 2.0 * Yo;
    const double q1 = 1.0 + kf * U;
    const double S = sqrt_d(fmax(q1, 0.0)), i1S = rcp_d(1.0 + S);
    const double Aa = kf * Xo, Bb = 1.0 - kf * Yo;
    const double dpsi = atan2(Aa, Bb);
    const double tanl = (v[1] - v[0]) * ids[1];

    // ---------------- backward ----------------
    double xb[N], yb[N], zb[N];
#pragma unroll
    for (int i = 0; i < N; i++) xb[i] = yb[i] = zb[i] = 0.0;
    double k0b = 0.0, psi0b = 0.0, snb = 0.0, csb = 0.0;
    double dsb[N], idsb[N], vbb[N], vgb[N], wzb[N], mb[N], sb[N];
#pragma unroll
    for (int i = 0; i < N; i++) dsb[i] = idsb[i] = vbb[i] = vgb[i] = wzb[i] = mb[i] = sb[i] = 0.0;
    const double gk = gp[0], gphi = gp[1], gtan = gp[2], gd0 = gp[3], gz0 = gp[4], gch = gc;

    // 5) perigee
    double kfb = -gk;
    double arcb, tanlb = gtan, v0b = 0.0, v1b = 0.0;
    {
        const double arc = kf != 0.0 ? dpsi / kf : Xo;
        v0b += gz0;
        tanlb += gz0 * arc;
        arcb = gz0 * tanl;
    }
    v1b += tanlb * ids[1];
    v0b -= tanlb * ids[1];
    idsb[1] += tanlb * (v[1] - v[0]);
    double dpsib = gphi, Xob = 0.0, Yob = 0.0, Ub = 0.0, psib = gphi;
    if (kf != 0.0) {
        dpsib += arcb / kf;
        kfb -= arcb * dpsi / (kf * kf);
    } else {
        Xob += arcb;
    }
    {
        const double ir2 = rcp_d(Aa * Aa + Bb * Bb);
        const double Aab = dpsib * Bb * ir2, Bbb = -dpsib * Aa * ir2;
        kfb += Aab * Xo;
        Xob += Aab * kf;
        kfb -= Bbb * Yo;
        Yob -= Bbb * kf;
    }
    {
        // d0 = -U / (1 + S), S = sqrt(1 + kf U)
        Ub += -gd0 * i1S;
        const double Sb = gd0 * U * i1S * i1S;
        if (q1 > 0.0 && S > 0.0) {
            const double qb = 0.5 * Sb * rcp_d(S);
            kfb += qb * U;
            Ub += qb * kf;
        }
    }
    kfb += Ub * (Xo * Xo + Yo * Yo);
    Xob += Ub * 2.0 * kf * Xo;
    Yob += Ub * (2.0 * kf * Yo - 2.0);
    double pxb = -Xob * cp + Yob * sp, pyb = -Xob * sp - Yob * cp;
    const double cpb = -Xob * px - Yob * py, spb = -Xob * py + Yob * px;
    psib += spb * cp - cpb * sp;
    // psi = psi0 + (u1 - u0) ids1 - dk ds1 / 2
    double xsb[M];
#pragma unroll
    for (int i = 0; i < M; i++) xsb[i] = 0.0;
    psi0b += psib;
    xsb[1] += psib * ids[1];
    xsb[0] -= psib * ids[1];
    idsb[1] += psib * (xs[1] - xs[0]);
    xsb[N] -= psib * 0.5 * ds[1];
    dsb[1] -= psib * 0.5 * dk;
    // px = x0 - u0 sn, py = y0 + u0 cs
    xb[0] += pxb;
    xsb[0] -= pxb * sn;
    snb -= pxb * xs[0];
    yb[0] += pyb;
    xsb[0] += pyb * cs;
    csb += pyb * xs[0];
    // kf = k0 + dk
    k0b += kfb;
    xsb[N] += kfb;

    // 4) circle: parameters through the solve, chi2 by the envelope theorem
    if constexpr (N != 3) {
        double bb[M];
#pragma unroll
        for (int i = 0; i < M; i++) bb[i] = xsb[i];
        solve_circle(bb);                      // bbar = B^-1 xbar
#pragma unroll
        for (int i = 0; i < N; i++) {
            // b_i = wu m_i; diagonal wu constant
            mb[i] += wu * bb[i];
            mb[i] += gch * (-2.0 * wu * (xs[i] - m[i]));
        }
#pragma unroll
        for (int i = 1; i < N - 1; i++) {
            const double h[4] = {ids[i], -(ids[i] + ids[i + 1]), ids[i + 1], -0.5 * (ds[i] + ds[i + 1])};
            const int at[4] = {i - 1, i, i + 1, N};
            double hx = 0.0, hb = 0.0;
#pragma unroll
            for (int a = 0; a < 4; a++) {
                hx += h[a] * xs[at[a]];
                hb += h[a] * bb[at[a]];
            }
            vbb[i] += -hb * hx + gch * hx * hx;     // hx is the kink residual be_i
            double hbar[4];
#pragma unroll
            for (int a = 0; a < 4; a++) hbar[a] = -vb[i] * (bb[at[a]] * hx + xs[at[a]] * hb) + gch * 2.0 * vb[i] * hx * xs[at[a]];
            idsb[i] += hbar[0] - hbar[1];
            idsb[i + 1] += hbar[2] - hbar[1];
            dsb[i] += -0.5 * hbar[3];
            dsb[i + 1] += -0.5 * hbar[3];
        }
    }
    // 3) line
    {
        double bb[N];
#pragma unroll
        for (int i = 0; i < N; i++) bb[i] = 0.0;
        bb[0] = v0b;
        bb[1] = v1b;
        solve_line(bb);
#pragma unroll
        for (int i = 0; i < N; i++) {
            // b_i = wz_i z_i, A_ii += wz_i
            zb[i] += wz[i] * bb[i] + gch * (-2.0 * wz[i] * (v[i] - z[i]));
            wzb[i] += z[i] * bb[i] - bb[i] * v[i] + gch * (v[i] - z[i]) * (v[i] - z[i]);
        }
#pragma unroll
        for (int i = 1; i < N - 1; i++) {
            const double g[3] = {ids[i], -(ids[i] + ids[i + 1]), ids[i + 1]};
            double gv = 0.0, gb = 0.0;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                gv += g[a] * v[i - 1 + a];
                gb += g[a] * bb[i - 1 + a];
            }
            vgb[i] += -gb * gv + gch * gv * gv;      // gv is the kink residual gam_i
            double gbar[3];
#pragma unroll
            for (int a = 0; a < 3; a++) gbar[a] = -vg[i] * (bb[i - 1 + a] * gv + v[i - 1 + a] * gb) + gch * 2.0 * vg[i] * gv * v[i - 1 + a];
            idsb[i] += gbar[0] - gbar[1];
            idsb[i + 1] += gbar[2] - gbar[1];
        }
    }
    // 2) weights: wz (disk hits depend on |tan lambda0|), vb, vg
    double atlb = 0.0, sec2b = 0.0, pmomb = 0.0;
#pragma unroll
    for (int i = 0; i < N; i++)
        if (disk[i]) {
            // wz = 1 / (sigma_r atl)^2
            atlb += wzb[i] * (-2.0 * wz[i] * iatl);
        }
#pragma unroll
    for (int i = 1; i < N - 1; i++) {
        const double th2 = th[i] * th[i];
        double th2b = 0.0;
        if (th2 * sec2 > 1e-20) {
            th2b += -vbb[i] * vb[i] * vb[i] * sec2;
            sec2b += -vbb[i] * vb[i] * vb[i] * th2;
        }
        if (th2 * sec2 * sec2 > 1e-20) {
            th2b += -vgb[i] * vg[i] * vg[i] * sec2 * sec2;
            sec2b += -vgb[i] * vg[i] * vg[i] * th2 * 2.0 * sec2;
        }
        const double thb = 2.0 * th[i] * th2b;
        // th = 0.0136 / pmom * sqrt(xx0) * (1 + 0.038 ln xx0)
        pmomb += -thb * th[i] * ipmom;
        const double sx = sqrt_d(xx0[i]);
        const double xx0b =
            thb * 0.0136 * ipmom * ((1.0 + 0.038 * lx0[i]) * 0.5 * rcp_d(sx) + sx * 0.038 * rcp_d(xx0[i]));
        // xx0 = x0 sqrt(sec2) [/ atl]
        sec2b += 0.5 * xx0b * xx0[i] * rcp_d(sec2);
        if (disk[i]) atlb += -xx0b * xx0[i] * iatl;
    }
    double tanl0b = 0.0;
    if (fabs(tanl0) > 1e-3) tanl0b += atlb * (tanl0 > 0.0 ? 1.0 : -1.0);
    // pmom = pt0 sqrt(sec2), pt0 = c bz / max(|k0|, 1e-7)
    sec2b += 0.5 * pmomb * pt0 * rcp_d(rsec);
    const double pt0b = pmomb * rsec;
    if (fabs(k0) > 1e-7) k0b += pt0b * (-pt0 * iak) * (k0 > 0.0 ? 1.0 : -1.0);
    tanl0b += 2.0 * tanl0 * sec2b;
    // tanl0 = (z_{n-1} - z_0) / max(s_{n-1}, 1e-4)
    zb[N - 1] += tanl0b * iSl;
    zb[0] -= tanl0b * iSl;
    if (s[N - 1] > 1e-4) sb[N - 1] -= tanl0b * tanl0 * iSl;
    // ids = 1/ds, ds = max(s_i - s_{i-1}, 1e-4)
#pragma unroll
    for (int i = 1; i < N; i++) {
        dsb[i] += -idsb[i] * ids[i] * ids[i];
        if (s[i] - s[i - 1] > 1e-4) {
            sb[i] += dsb[i];
            sb[i - 1] -= dsb[i];
        }
    }
    // 1b) arc lengths and offsets, per hit
#pragma unroll
    for (int i = 1; i < N; i++) {
        double dxb = 0.0, dyb = 0.0;
        if (i != ib && i != ic) {         // (offsets identically zero on the pre-fit circle)
            // m = -U / (1 + Sq), Sq = sqrt(max(1 + k0 U, 0))
            double Ubi = -mb[i] * i1Sq[i];
            if (1.0 + k0 * Us[i] > 0.0 && Sq[i] > 0.0) {
                const double Sqb = mb[i] * Us[i] * i1Sq[i] * i1Sq[i];
                const double qb = 0.5 * Sqb * rcp_d(Sq[i]);
                k0b += qb * Us[i];
                Ubi += qb * k0;
            }
            // U = k0 (X^2 + Y^2) - 2 Y
            k0b += Ubi * (Xs[i] * Xs[i] + Ys[i] * Ys[i]);
            const double Xb = Ubi * 2.0 * k0 * Xs[i], Yb = Ubi * (2.0 * k0 * Ys[i] - 2.0);
            // X = dx cs + dy sn, Y = dy cs - dx sn
            dxb += Xb * cs - Yb * sn;
            dyb += Xb * sn + Yb * cs;
            csb += Xb * dxs[i] + Yb * dys[i];
            snb += Xb * dys[i] - Yb * dxs[i];
        }
        // s = dist asinc(q), q = 0.5 k0 dist (clamped)
        if (dist[i] > 0.0) {
            const bool qin = fabs(0.5 * k0 * dist[i]) < 1.0;
            const double da = qin ? dasinc_d(qs[i], asq[i]) : 0.0;
            const double distb = sb[i] * (asc[i] + dist[i] * da * 0.5 * k0);
            k0b += sb[i] * dist[i] * da * 0.5 * dist[i];
            const double idist = rcp_d(dist[i]);
            dxb += distb * dxs[i] * idist;
            dyb += distb * dys[i] * idist;
        }
        xb[i] += dxb;
        xb[0] -= dxb;
        yb[i] += dyb;
        yb[0] -= dyb;
    }
    // hit 0 has s = 0 and m = 0 identically (dx = dy = 0)
    // 1a) pre-fit: sn, cs from psi0
    psi0b += snb * cs - csb * sn;
    double abxb = 0.0, abyb = 0.0, acxb = 0.0, acyb = 0.0, bcxb = 0.0, bcyb = 0.0, dabb = 0.0;
    {
        // psi0 = atan2(aby, abx) - asin(ta), ta = k0 dab / 2
        const double ir2 = rcp_d(abx * abx + aby * aby);
        abyb += psi0b * abx * ir2;
        abxb += -psi0b * aby * ir2;
        if (ta_in) {
            const double tb = -psi0b * rsqrt_d(1.0 - ta * ta);
            k0b += tb * 0.5 * dab;
            dabb += tb * 0.5 * k0;
        }
    }
    if (den > 0.0) {
        // k0 = 2 orient / (dab dbc dca)
        const double orb = k0b * 2.0 * iden;
        const double denb = -k0b * k0 * iden;
        dabb += denb * dbc * dca;
        const double dbcb = denb * dab * dca, dcab = denb * dab * dbc;
        abxb += orb * acy;
        acyb += orb * abx;
        abyb -= orb * acx;
        acxb -= orb * aby;
        const double idab = rcp_d(dab), idbc = rcp_d(dbc), idca = rcp_d(dca);
        abxb += dabb * abx * idab;
        abyb += dabb * aby * idab;
        bcxb += dbcb * bcx * idbc;
        bcyb += dbcb * bcy * idbc;
        acxb += dcab * acx * idca;
        acyb += dcab * acy * idca;
    } else {
        const double r2 = abx * abx + aby * aby;
        (void)r2;
    }
    xb[ib] += abxb;
    xb[0] -= abxb;
    yb[ib] += abyb;
    yb[0] -= abyb;
    xb[ic] += acxb;
    xb[0] -= acxb;
    yb[ic] += acyb;
    yb[0] -= acyb;
    xb[ic] += bcxb;
    xb[ib] -= bcxb;
    yb[ic] += bcyb;
    yb[ib] -= bcyb;
#pragma unroll
    for (int i = 0; i < N; i++) {
        const int h = hid[i];
        atomicAdd(gx + h, (float)xb[i]);
        atomicAdd(gy + h, (float)yb[i]);
        atomicAdd(gz + h, (float)zb[i]);
    }
}

// One kernel per hit count, over the track range of that count.
template <int N>
__global__ void __launch_bounds__(128) k_fit_grad(Params p, const float *gpar, const float *gchi, float *gx, float *gy,
                                                  float *gz) {
    if (upstream_overflow(p, PT_FLAG_CELLS | PT_FLAG_TUPLES | PT_FLAG_TRACKS)) return;
    constexpr int c = N - 3;
    int64_t k0 = 0;
#pragma unroll
    for (int q = 0; q < c; q++) k0 += p.counters[C_TRK_CNT + q];
    const int64_t k1 = min(k0 + p.counters[C_TRK_CNT + c], p.cap_tracks);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = k0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < k1; k += stride) {
        const int32_t t = p.trk_tuple[k];
        const float *g = gpar + k * 5;
        const float gc = gchi ? gchi[k] : 0.f;
        if (N < 6) {
            grad_track<N>(p, t, g, gc, gx, gy, gz);
        } else {
            const int n = p.tup_n[t];
            if (n == 6) grad_track<6>(p, t, g, gc, gx, gy, gz);
            else if (n == 7) grad_track<7>(p, t, g, gc, gx, gy, gz);
            else grad_track<8>(p, t, g, gc, gx, gy, gz);
        }
    }
}

// Alignment of module m: x' = c_m + (I + [w_m]x)(x - c_m) + d_m for the
// hits on it (shift d and small rotation w about the module centre c).
__global__ void __launch_bounds__(kThreads) k_align(int n, const float *x, const float *y, const float *z,
                                                    const int32_t *module, const float *centre, const float *shift,
                                                    const float *rot, float *xo, float *yo, float *zo) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int mm = module[i];
        const float rx = x[i] - centre[3 * mm], ry = y[i] - centre[3 * mm + 1], rz = z[i] - centre[3 * mm + 2];
        const float wx = rot[3 * mm], wy = rot[3 * mm + 1], wz = rot[3 * mm + 2];
        xo[i] = x[i] + (wy * rz - wz * ry) + shift[3 * mm];
        yo[i] = y[i] + (wz * rx - wx * rz) + shift[3 * mm + 1];
        zo[i] = z[i] + (wx * ry - wy * rx) + shift[3 * mm + 2];
    }
}

// Its adjoint: given the gradient g' at the aligned hits, the gradients at
// the original hits (g' + g' x w) and, summed over the hits of each module,
// at the shift (g') and at the rotation ((x - c) x g').
__global__ void __launch_bounds__(kThreads) k_align_grad(int n, const float *x, const float *y, const float *z,
                                                         const int32_t *module, const float *centre, const float *rot,
                                                         const float *gxa, const float *gya, const float *gza,
                                                         float *gx, float *gy, float *gz, float *gshift,
                                                         float *grot) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int mm = module[i];
        const float ax = gxa[i], ay = gya[i], az = gza[i];
        if (gx) {
            const float wx = rot[3 * mm], wy = rot[3 * mm + 1], wz = rot[3 * mm + 2];
            gx[i] += ax + (ay * wz - az * wy);
            gy[i] += ay + (az * wx - ax * wz);
            gz[i] += az + (ax * wy - ay * wx);
        }
        if (ax == 0.f && ay == 0.f && az == 0.f) continue;
        const float rx = x[i] - centre[3 * mm], ry = y[i] - centre[3 * mm + 1], rz = z[i] - centre[3 * mm + 2];
        if (gshift) {
            atomicAdd(gshift + 3 * mm, ax);
            atomicAdd(gshift + 3 * mm + 1, ay);
            atomicAdd(gshift + 3 * mm + 2, az);
        }
        if (grot) {
            atomicAdd(grot + 3 * mm, ry * az - rz * ay);
            atomicAdd(grot + 3 * mm + 1, rz * ax - rx * az);
            atomicAdd(grot + 3 * mm + 2, rx * ay - ry * ax);
        }
    }
}

}  // namespace

void launch_fit_grad(const Params &p, const float *gpar, const float *gchi, float *gx, float *gy, float *gz, int grid,
                     cudaStream_t s) {
    {
        KernelTimer t("k_fit_grad<3>", s);
        k_fit_grad<3><<<grid, 128, 0, s>>>(p, gpar, gchi, gx, gy, gz);
    }
    {
        KernelTimer t("k_fit_grad<4>", s);
        k_fit_grad<4><<<grid, 128, 0, s>>>(p, gpar, gchi, gx, gy, gz);
    }
    {
        KernelTimer t("k_fit_grad<5>", s);
        k_fit_grad<5><<<grid, 128, 0, s>>>(p, gpar, gchi, gx, gy, gz);
    }
    KernelTimer t("k_fit_grad<6..8>", s);
    k_fit_grad<6><<<grid, 128, 0, s>>>(p, gpar, gchi, gx, gy, gz);
}

void launch_align(int n, const float *x, const float *y, const float *z, const int32_t *module, const float *centre,
                  const float *shift, const float *rot, float *xo, float *yo, float *zo, int grid, cudaStream_t s) {
    KernelTimer t("k_align", s);
    k_align<<<grid, kThreads, 0, s>>>(n, x, y, z, module, centre, shift, rot, xo, yo, zo);
}

void launch_align_grad(int n, const float *x, const float *y, const float *z, const int32_t *module,
                       const float *centre, const float *rot, const float *gxa, const float *gya, const float *gza,
                       float *gx, float *gy, float *gz, float *gshift, float *grot, int grid, cudaStream_t s) {
    KernelTimer t("k_align_grad", s);
    k_align_grad<<<grid, kThreads, 0, s>>>(n, x, y, z, module, centre, rot, gxa, gya, gza, gx, gy, gz, gshift, grot);
}

}  // namespace ptk
