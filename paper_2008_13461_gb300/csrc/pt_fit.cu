// Step a6: broken-line fit (Sec. 3.4; method of Blobel 2006), one thread per
// track, specialised at compile time for the number of hits so that every
// array lives in registers.
//
//  1. pre-fit: circle through hits 0, n/2, n-1 gives the curvature k0 and the
//     direction psi0 at hit 0; arc lengths s_i (chord formula) and signed
//     offsets m_i of the hits from that circle (left of the motion positive);
//  2. multiple-scattering variances of the kinks at the inner hits (Highland,
//     momentum from k0 and the pre-fit dip);
//  3. s-z line fit: unknowns v_i, measurement z_i (sigma_z; disks sigma_r
//     |tan lambda0|), kinks of the slope (three hits: one kink, solved in
//     closed form);
//  4. transverse circle fit: unknowns u_i and dk, measurement m_i
//     (sigma_rphi), kinks of the offset slope minus dk times the mean step
//     (three hits: solved in closed form, the offsets are fitted exactly);
//  5. perigee parameters w.r.t. the beam line and their covariance (line block
//     by its linear Jacobian, circle block by the analytic Jacobian).
//
// Precision: geometry in float32 -- coordinate differences are exact on the
// 2^-14 cm grid, and the near-cancelling 2x2 products (pre-fit orientation,
// projections on the pre-fit frame) use FMA-compensated evaluation -- and
// the normal equations, their Cholesky factorisation, solutions and chi2 in
// float64, where the kink weights (up to ~1e10) and measurement weights
// (~1e6) make the matrices too ill-conditioned for float32.
//
// The float64 pipe is the bound, so the unknowns are ordered with the ones
// the track parameters need (v0, v1; u0, u1, dk) last: with A = L L^T, their
// covariance is the inverse of the trailing block of L times its transpose
// (the Schur complement), with no unit-vector solves.  chi2 is taken from
// the residuals of the full solution: the shortcut c - |L^-1 b|^2 cancels
// catastrophically for ill-conditioned tracks with large |z|.
#include "pt_common.cuh"
#include "pt_kernels.cuh"

namespace ptk {

__device__ __forceinline__ float asinc(float x) {
    x = fminf(fmaxf(x, -1.0f), 1.0f);
    return fabsf(x) < 1e-4f ? 1.0f + x * x * (1.0f / 6.0f) : asinf(x) / x;
}

template <int M>
__device__ __forceinline__ int pidx(int r, int c) { return r * (r + 1) / 2 + c; }

// 1/sqrt(s) and 1/d in the solve's precision R.  Double: from a float32
// seed and one Newton step (relative error 1e-7 -> ~1e-14), to keep the slow
// FP64 pipe to a few multiply-adds; float: IEEE square root and division.
__device__ __forceinline__ double rsqrt_r(double s) {
    const double y = (double)rsqrtf((float)s);
    return y * (1.5 - 0.5 * s * y * y);
}
__device__ __forceinline__ float rsqrt_r(float s) { return 1.0f / sqrtf(s); }

__device__ __forceinline__ double recip_r(double d) {
    const double r = (double)(1.0f / (float)d);
    return r * (2.0 - d * r);
}
__device__ __forceinline__ float recip_r(float d) { return 1.0f / d; }

// in-place Cholesky of a packed lower-triangular SPD matrix; the diagonal
// holds the reciprocals of L's diagonal (so solves need no division)
template <int M, typename R>
__device__ __forceinline__ void chol(R *A) {
#pragma unroll
    for (int j = 0; j < M; j++) {
        R s = A[pidx<M>(j, j)];
#pragma unroll
        for (int k = 0; k < j; k++) s -= A[pidx<M>(j, k)] * A[pidx<M>(j, k)];
        const R id = rsqrt_r(s > R(1e-30) ? s : R(1e-30));
        A[pidx<M>(j, j)] = id;
#pragma unroll
        for (int i = j + 1; i < M; i++) {
            R t = A[pidx<M>(i, j)];
#pragma unroll
            for (int k = 0; k < j; k++) t -= A[pidx<M>(i, k)] * A[pidx<M>(j, k)];
            A[pidx<M>(i, j)] = t * id;
        }
    }
}

// Given the factor of chol(), b := the solution of A x = b (forward and
// back substitution), and C := the covariance of its last K unknowns, the
// inverse of L22 L22^T (L22 the trailing K x K block of L).
template <int M, int K, typename R>
__device__ __forceinline__ void solve_tail(const R *L, R *b, R (*C)[K]) {
#pragma unroll
    for (int i = 0; i < M; i++) {
        R t = b[i];
#pragma unroll
        for (int k = 0; k < i; k++) t -= L[pidx<M>(i, k)] * b[k];
        b[i] = t * L[pidx<M>(i, i)];
    }
#pragma unroll
    for (int i = M - 1; i >= 0; i--) {
        R t = b[i];
#pragma unroll
        for (int k = i + 1; k < M; k++) t -= L[pidx<M>(k, i)] * b[k];
        b[i] = t * L[pidx<M>(i, i)];
    }
    // T = L22^-1 (lower triangular), C = T^T T
    constexpr int o = M - K;
    R T[K][K];
#pragma unroll
    for (int j = 0; j < K; j++) {
#pragma unroll
        for (int i = 0; i < K; i++) {
            if (i < j) {
                T[i][j] = R(0);
            } else if (i == j) {
                T[i][j] = L[pidx<M>(o + i, o + i)];
            } else {
                R t = R(0);
#pragma unroll
                for (int k = j; k < i; k++) t -= L[pidx<M>(o + i, o + k)] * T[k][j];
                T[i][j] = t * L[pidx<M>(o + i, o + i)];
            }
        }
    }
#pragma unroll
    for (int a = 0; a < K; a++)
#pragma unroll
        for (int c = 0; c <= a; c++) {
            R t = R(0);
#pragma unroll
            for (int k = a; k < K; k++) t += T[k][a] * T[k][c];
            C[a][c] = t;
            C[c][a] = t;
        }
}

// packed index of the symmetric entry (i, j), either order
template <int M>
__device__ __forceinline__ int sidx(int i, int j) { return i >= j ? pidx<M>(i, j) : pidx<M>(j, i); }

template <int N, typename R>
__device__ void fit_track(const Params &p, int64_t k, int32_t t) {
    const int32_t *hid = p.tup_hits + (int64_t)t * PT_NMAX;
    float hx[N], hy[N], hz[N];
    bool disk[N];
#pragma unroll
    for (int i = 0; i < N; i++) {
        const int h = hid[i];
        hx[i] = p.x[h];
        hy[i] = p.y[h];
        hz[i] = p.z[h];
        disk[i] = p.layer[p.module_layer[p.module[h]]].kind == PT_LAYER_DISK;
    }
    // 1) pre-fit circle through hits 0, n/2, n-1
    constexpr int ib = N / 2, ic = N - 1;
    const float abx = hx[ib] - hx[0], aby = hy[ib] - hy[0];
    const float acx = hx[ic] - hx[0], acy = hy[ic] - hy[0];
    const float bcx = hx[ic] - hx[ib], bcy = hy[ic] - hy[ib];
    const float orient = det2(abx, acy, aby, acx);
    const float dab = sqrtf(abx * abx + aby * aby), dbc = sqrtf(bcx * bcx + bcy * bcy);
    const float dca = sqrtf(acx * acx + acy * acy);
    const float den = dab * dbc * dca;
    const float k0 = den > 0.f ? 2.0f * orient / den : 0.f;
    const float psi0 = atan2f(aby, abx) - asinf(fminf(fmaxf(0.5f * k0 * dab, -1.f), 1.f));
    float sn, cs;
    sincosf(psi0, &sn, &cs);
    float s[N], m[N], ds[N];
#pragma unroll
    for (int i = 0; i < N; i++) {
        const float dx = hx[i] - hx[0], dy = hy[i] - hy[0];
        const float dist = sqrtf(dx * dx + dy * dy);
        s[i] = dist * asinc(0.5f * k0 * dist);
        const float X = det2(dx, cs, -dy, sn);     // dx cs + dy sn
        const float Y = det2(dy, cs, dx, sn);      // -dx sn + dy cs
        const float U = k0 * (X * X + Y * Y) - 2.0f * Y;
        const float q = 1.0f + k0 * U;
        m[i] = -U / (1.0f + sqrtf(fmaxf(q, 0.f)));
    }
    ds[0] = 0.f;
    R ids[N];
    ids[0] = R(0);
#pragma unroll
    for (int i = 1; i < N; i++) {
        ds[i] = fmaxf(s[i] - s[i - 1], 1e-4f);
        ids[i] = recip_r((R)ds[i]);
    }
    const float tanl0 = (hz[N - 1] - hz[0]) / fmaxf(s[N - 1], 1e-4f);
    const float sec2 = 1.0f + tanl0 * tanl0;
    const float pt0 = 0.00299792458f * p.fit.bz / fmaxf(fabsf(k0), 1e-7f);
    const float pmom = pt0 * sqrtf(sec2);
    const float atl = fmaxf(fabsf(tanl0), 1e-3f);
    // 2) scattering variances of the kinks at hits 1 .. n-2
    R vb[N], vg[N], kv[N], kz[N];
#pragma unroll
    for (int i = 1; i < N - 1; i++) {
        const float xx0 = disk[i] ? p.fit.x0_disk * sqrtf(sec2) / atl : p.fit.x0_barrel * sqrtf(sec2);
        const float th = 0.0136f / pmom * sqrtf(xx0) * (1.0f + 0.038f * logf(xx0));
        const R th2 = (R)th * th;
        kv[i] = fmax(th2 * sec2, R(1e-20));                   // kink variances: transverse,
        kz[i] = fmax(th2 * sec2 * sec2, R(1e-20));            //   s-z slope
        if (N > 4) {
            vb[i] = recip_r(kv[i]);                           // weights 1/variance
            vg[i] = recip_r(kz[i]);
        }
    }
    // 3) line fit in s-z; unknown v_i at position ln(i): v2 .. v_{n-1}, v0, v1
    auto ln = [](int i) { return i >= 2 ? i - 2 : N - 2 + i; };
    R v[2], Cv[2][2], chi2;
    if constexpr (N == 3) {
        // One kink: the normal matrix is diag(1/var_i) + g g^T / var_k, and
        // its inverse follows from Sherman-Morrison: with q = g . z and
        // D = var_k + sum g_i^2 var_i, v_i = z_i - var_i g_i q / D, chi2 =
        // q^2 / D, cov(v_i, v_j) = var_i delta_ij - var_i g_i var_j g_j / D
        // (the diagonal as var_i (D - g_i^2 var_i) / D, a sum of positive
        // terms).
        R var[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const R sz = disk[i] ? (R)p.fit.sigma_r * atl : (R)p.fit.sigma_z;
            var[i] = sz * sz;
        }
        const R g0 = ids[1], g2 = ids[2], g1 = -(g0 + g2);
        const R t0 = g0 * g0 * var[0], t1 = g1 * g1 * var[1], t2 = g2 * g2 * var[2];
        const R iD = recip_r(kz[1] + t0 + t1 + t2);
        const R q = g0 * hz[0] + g1 * hz[1] + g2 * hz[2];
        const R f = q * iD;
        v[0] = hz[0] - var[0] * g0 * f;
        v[1] = hz[1] - var[1] * g1 * f;
        chi2 = q * f;
        Cv[0][0] = var[0] * (kz[1] + t1 + t2) * iD;
        Cv[1][1] = var[1] * (kz[1] + t0 + t2) * iD;
        Cv[0][1] = Cv[1][0] = -(var[0] * g0) * (var[1] * g1) * iD;
    } else if constexpr (N == 4) {
        // Two kinks (hits 1, 2): the normal matrix is D + G^T W G, D =
        // diag(1/var_i), W = diag(1/var_k), G the kinks' 2 x 4 slope
        // operator.  By Woodbury, with S = W^-1 + G D^-1 G^T (2 x 2) and r =
        // S^-1 G z: v = z - D^-1 G^T r, cov(v) = D^-1 - D^-1 G^T S^-1 G D^-1,
        // and chi2 from the residuals, v - z = -D^-1 G^T r and G v = W^-1 r:
        // sum_i var_i (G^T r)_i^2 + sum_k var_k r_k^2, every term positive.
        R var[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const R sz = disk[i] ? (R)p.fit.sigma_r * atl : (R)p.fit.sigma_z;
            var[i] = sz * sz;
        }
        const R a0 = ids[1], a2 = ids[2], a1 = -(a0 + a2);      // kink 1 on v0, v1, v2
        const R b0 = ids[2], b2 = ids[3], b1 = -(b0 + b2);      // kink 2 on v1, v2, v3
        const R S11 = kz[1] + a0 * a0 * var[0] + a1 * a1 * var[1] + a2 * a2 * var[2];
        const R S22 = kz[2] + b0 * b0 * var[1] + b1 * b1 * var[2] + b2 * b2 * var[3];
        const R S12 = a1 * b0 * var[1] + a2 * b1 * var[2];
        const R q1 = a0 * hz[0] + a1 * hz[1] + a2 * hz[2];
        const R q2 = b0 * hz[1] + b1 * hz[2] + b2 * hz[3];
        const R idet = recip_r(S11 * S22 - S12 * S12);
        const R i11 = S22 * idet, i22 = S11 * idet, i12 = -S12 * idet;
        const R r1 = i11 * q1 + i12 * q2, r2 = i12 * q1 + i22 * q2;
        const R e0 = a0 * r1, e1 = a1 * r1 + b0 * r2, e2 = a2 * r1 + b1 * r2, e3 = b2 * r2;     // G^T r
        v[0] = hz[0] - var[0] * e0;
        v[1] = hz[1] - var[1] * e1;
        chi2 = var[0] * e0 * e0 + var[1] * e1 * e1 + var[2] * e2 * e2 + var[3] * e3 * e3 + kz[1] * r1 * r1 +
               kz[2] * r2 * r2;
        // (G^T S^-1 G) on v0 (column (a0, 0)) and v1 (column (a1, b0))
        const R m00 = a0 * a0 * i11, m01 = a0 * (a1 * i11 + b0 * i12);
        const R m11 = a1 * a1 * i11 + 2 * a1 * b0 * i12 + b0 * b0 * i22;
        Cv[0][0] = var[0] - var[0] * var[0] * m00;
        Cv[1][1] = var[1] - var[1] * var[1] * m11;
        Cv[0][1] = Cv[1][0] = -var[0] * var[1] * m01;
    } else {
        R A[N * (N + 1) / 2], bv[N], wz[N];
#pragma unroll
        for (int i = 0; i < N * (N + 1) / 2; i++) A[i] = R(0);
#pragma unroll
        for (int i = 0; i < N; i++) {
            const R sz = disk[i] ? (R)p.fit.sigma_r * atl : (R)p.fit.sigma_z;
            wz[i] = recip_r(sz * sz);
            A[pidx<N>(ln(i), ln(i))] = wz[i];
            bv[ln(i)] = wz[i] * hz[i];
        }
#pragma unroll
        for (int i = 1; i < N - 1; i++) {
            const R g0 = ids[i], g2 = ids[i + 1], g1 = -(g0 + g2), w = vg[i];
            const R wg0 = g0 * w, wg1 = g1 * w, wg2 = g2 * w;
            A[sidx<N>(ln(i - 1), ln(i - 1))] += g0 * wg0;
            A[sidx<N>(ln(i), ln(i - 1))] += g1 * wg0;
            A[sidx<N>(ln(i), ln(i))] += g1 * wg1;
            A[sidx<N>(ln(i + 1), ln(i - 1))] += g2 * wg0;
            A[sidx<N>(ln(i + 1), ln(i))] += g2 * wg1;
            A[sidx<N>(ln(i + 1), ln(i + 1))] += g2 * wg2;
        }
        chol<N, R>(A);
        solve_tail<N, 2, R>(A, bv, Cv);      // bv[ln(i)] = v_i
        chi2 = R(0);
#pragma unroll
        for (int i = 0; i < N; i++) chi2 += wz[i] * (bv[ln(i)] - hz[i]) * (bv[ln(i)] - hz[i]);
#pragma unroll
        for (int i = 1; i < N - 1; i++) {
            const R gam = (bv[ln(i + 1)] - bv[ln(i)]) * ids[i + 1] - (bv[ln(i)] - bv[ln(i - 1)]) * ids[i];
            chi2 += gam * gam * vg[i];
        }
        v[0] = bv[ln(0)];
        v[1] = bv[ln(1)];
    }
    // 4) circle fit: unknowns u_0 .. u_{n-1}, dk; u_i at position ln(i), dk last
    R xu[3], Cc[3][3];
    if constexpr (N == 3) {
        // Three offsets and one kink: the minimum has u_i = m_i and the kink
        // at hit 1 zero, so dk = a . m with a_i = -h_i / h3; the inverse of
        // the normal matrix gives cov(u) = sigma^2 I, cov(u, dk) = sigma^2 a
        // and var(dk) = sigma^2 |a|^2 + var(kink) / h3^2; the circle chi2 is 0.
        const R h0 = ids[1], h2 = ids[2], h1 = -(h0 + h2);
        const R ih3 = recip_r(R(-0.5) * ((R)ds[1] + ds[2]));
        const R a0 = -h0 * ih3, a1 = -h1 * ih3, a2 = -h2 * ih3;
        const R s2 = (R)p.fit.sigma_rphi * p.fit.sigma_rphi;
        xu[0] = m[0];
        xu[1] = m[1];
        xu[2] = a0 * m[0] + a1 * m[1] + a2 * m[2];
        Cc[0][0] = s2;
        Cc[0][1] = Cc[1][0] = R(0);
        Cc[1][1] = s2;
        Cc[0][2] = Cc[2][0] = s2 * a0;
        Cc[1][2] = Cc[2][1] = s2 * a1;
        Cc[2][2] = s2 * (a0 * a0 + a1 * a1 + a2 * a2) + kv[1] * ih3 * ih3;
    } else if constexpr (N == 4) {
        // Two kinks, residuals beta_k = (H u)_k + h3_k dk (variances var_k).
        // Minimising over dk leaves the rank-one penalty w' (c . u)^2 with c
        // = H^T (h3_2, -h3_1) and w' = 1 / (h3_1^2 var_2 + h3_2^2 var_1); by
        // Sherman-Morrison, with alpha = w' / (wu + w' |c|^2): u = m - alpha
        // (c . m) c, cov(u) = (I - alpha c c^T) / wu, dk = t . u with t =
        // -w' (h3_1 var_2 H_1 + h3_2 var_1 H_2) (H_k the rows of H), cov(u,
        // dk) = cov(u) t, var(dk) = var_1 var_2 w' + t^T cov(u) t, and chi2 =
        // wu w' (c . m)^2 / (wu + w' |c|^2).
        const R s2 = (R)p.fit.sigma_rphi * p.fit.sigma_rphi;
        const R wu = recip_r(s2);
        const R h0 = ids[1], h2 = ids[2], h1 = -(h0 + h2);      // kink 1 on u0, u1, u2
        const R k0 = ids[2], k2 = ids[3], k1 = -(k0 + k2);      // kink 2 on u1, u2, u3
        const R g1 = R(-0.5) * ((R)ds[1] + ds[2]), g2 = R(-0.5) * ((R)ds[2] + ds[3]);
        const R wp = recip_r(g1 * g1 * kv[2] + g2 * g2 * kv[1]);
        const R c0 = g2 * h0, c1 = g2 * h1 - g1 * k0, c2 = g2 * h2 - g1 * k1, c3 = -g1 * k2;
        const R cc0 = c1 * c1 + c2 * c2 + c3 * c3, cc1 = c0 * c0 + c2 * c2 + c3 * c3;
        const R cc = c0 * c0 + cc0;
        const R iden = recip_r(wu + wp * cc), alpha = wp * iden;
        const R cm = c0 * m[0] + c1 * m[1] + c2 * m[2] + c3 * m[3];
        const R u0 = m[0] - alpha * cm * c0, u1 = m[1] - alpha * cm * c1;
        const R u2 = m[2] - alpha * cm * c2, u3 = m[3] - alpha * cm * c3;
        const R p1 = g1 * kv[2] * wp, p2 = g2 * kv[1] * wp;
        const R t0 = -p1 * h0, t1 = -(p1 * h1 + p2 * k0), t2 = -(p1 * h2 + p2 * k1), t3 = -p2 * k2;
        xu[0] = u0;
        xu[1] = u1;
        xu[2] = t0 * u0 + t1 * u1 + t2 * u2 + t3 * u3;
        const R ct = c0 * t0 + c1 * t1 + c2 * t2 + c3 * t3;
        Cc[0][0] = s2 * (wu + wp * cc0) * iden;
        Cc[1][1] = s2 * (wu + wp * cc1) * iden;
        Cc[0][1] = Cc[1][0] = -s2 * alpha * c0 * c1;
        Cc[0][2] = Cc[2][0] = s2 * (t0 - alpha * c0 * ct);
        Cc[1][2] = Cc[2][1] = s2 * (t1 - alpha * c1 * ct);
        Cc[2][2] = kv[1] * kv[2] * wp + s2 * (t0 * t0 + t1 * t1 + t2 * t2 + t3 * t3 - alpha * ct * ct);
        chi2 += wu * wp * cm * cm * iden;
    } else {
        constexpr int M = N + 1;
        R B[M * (M + 1) / 2], bu[M];
#pragma unroll
        for (int i = 0; i < M * (M + 1) / 2; i++) B[i] = R(0);
        const R wu = recip_r((R)p.fit.sigma_rphi * p.fit.sigma_rphi);
#pragma unroll
        for (int i = 0; i < N; i++) {
            B[pidx<M>(ln(i), ln(i))] = wu;
            bu[ln(i)] = wu * m[i];
        }
        bu[N] = R(0);
#pragma unroll
        for (int i = 1; i < N - 1; i++) {
            const R h0 = ids[i], h2 = ids[i + 1], h1 = -(h0 + h2);
            const R h3 = R(-0.5) * ((R)ds[i] + ds[i + 1]), w = vb[i];
            const R wh0 = h0 * w, wh1 = h1 * w, wh2 = h2 * w;
            B[sidx<M>(ln(i - 1), ln(i - 1))] += h0 * wh0;
            B[sidx<M>(ln(i), ln(i - 1))] += h1 * wh0;
            B[sidx<M>(ln(i), ln(i))] += h1 * wh1;
            B[sidx<M>(ln(i + 1), ln(i - 1))] += h2 * wh0;
            B[sidx<M>(ln(i + 1), ln(i))] += h2 * wh1;
            B[sidx<M>(ln(i + 1), ln(i + 1))] += h2 * wh2;
            B[pidx<M>(N, ln(i - 1))] += h3 * wh0;
            B[pidx<M>(N, ln(i))] += h3 * wh1;
            B[pidx<M>(N, ln(i + 1))] += h3 * wh2;
            B[pidx<M>(N, N)] += h3 * h3 * w;
        }
        chol<M, R>(B);
        solve_tail<M, 3, R>(B, bu, Cc);      // bu[ln(i)] = u_i, bu[N] = dk
        const R dkk = bu[N];
#pragma unroll
        for (int i = 0; i < N; i++) chi2 += wu * (bu[ln(i)] - m[i]) * (bu[ln(i)] - m[i]);
#pragma unroll
        for (int i = 1; i < N - 1; i++) {
            const R be = (bu[ln(i + 1)] - bu[ln(i)]) * ids[i + 1] - (bu[ln(i)] - bu[ln(i - 1)]) * ids[i] -
                         dkk * R(0.5) * ((R)ds[i] + ds[i + 1]);
            chi2 += be * be * vb[i];
        }
        xu[0] = bu[ln(0)];
        xu[1] = bu[ln(1)];
        xu[2] = dkk;
    }
    const R dk = xu[2];
    // 5) perigee of the fitted circle through P with direction psi
    const float kf = (float)((R)k0 + dk);
    const float u0 = (float)xu[0];
    const float px = hx[0] - u0 * sn, py = hy[0] + u0 * cs;
    const float ds1 = ds[1];
    const float psi = psi0 + (float)((xu[1] - xu[0]) * ids[1] - dk * R(0.5) * ds1);
    float sp, cp;
    sincosf(psi, &sp, &cp);
    const float Xo = -det2(px, cp, -py, sp);       // -(P . t)
    const float Yo = det2(px, sp, py, cp);         // -(P . n)
    const float U = kf * (Xo * Xo + Yo * Yo) - 2.0f * Yo;
    const float S = sqrtf(fmaxf(1.0f + kf * U, 0.f));
    const float d0 = -U / (1.0f + S);
    const float Aa = kf * Xo, Bb = 1.0f - kf * Yo;
    const float dpsi = atan2f(Aa, Bb);
    float phi0 = psi + dpsi;
    phi0 = phi0 - 6.28318531f * rintf(phi0 * 0.159154943f);
    const float arc = kf != 0.f ? dpsi / kf : Xo;
    const R tanl = (v[1] - v[0]) * ids[1];
    const R z0 = v[0] + tanl * arc;
    // circle-block Jacobian d(kappa, phi0, d0) / d(u0, u1, dk)
    float J[3][3];
    {
        const float dPx[3] = {-sn, 0.f, 0.f}, dPy[3] = {cs, 0.f, 0.f};
        const float dps[3] = {-1.0f / ds1, 1.0f / ds1, -0.5f * ds1};
        const float dkk[3] = {0.f, 0.f, 1.f};
        const float iS = S > 0.f ? 1.0f / S : 0.f;
        const float ab2 = Aa * Aa + Bb * Bb;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float dX = -(dPx[j] * cp + dPy[j] * sp) + Yo * dps[j];
            const float dY = (dPx[j] * sp - dPy[j] * cp) - Xo * dps[j];
            const float dU = (Xo * Xo + Yo * Yo) * dkk[j] + 2.0f * kf * Xo * dX + (2.0f * kf * Yo - 2.0f) * dY;
            const float dS = 0.5f * iS * (U * dkk[j] + kf * dU);
            const float dd0 = -dU / (1.0f + S) + U / ((1.0f + S) * (1.0f + S)) * dS;
            const float dA = Xo * dkk[j] + kf * dX, dB = -Yo * dkk[j] - kf * dY;
            const float ddpsi = (Bb * dA - Aa * dB) / ab2;
            J[0][j] = -dkk[j];
            J[1][j] = dps[j] + ddpsi;
            J[2][j] = dd0;
        }
    }
    // F = J C J^T as (J C) J^T; the first row of J is (0, 0, -1).  The
    // transform runs in float32, like J itself (the solve's covariance C is
    // float64): its rounding, ~1e-7 of the terms, stays far below the 1e-3
    // relative tolerance of the covariance (the diagonal departs from the
    // float64 oracle by under 2e-6 on whole events).
    float C3[3][3];
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int d = 0; d < 3; d++) C3[c][d] = (float)Cc[c][d];
    float JC[3][3];
#pragma unroll
    for (int a = 1; a < 3; a++)
#pragma unroll
        for (int d = 0; d < 3; d++) {
            float acc = 0.f;
#pragma unroll
            for (int c = 0; c < 3; c++) acc += J[a][c] * C3[c][d];
            JC[a][d] = acc;
        }
    float Fc[3][3];
    Fc[0][0] = C3[2][2];
#pragma unroll
    for (int a = 1; a < 3; a++) {
        Fc[a][0] = Fc[0][a] = -JC[a][2];
#pragma unroll
        for (int b = 1; b <= a; b++) {
            float acc = 0.f;
#pragma unroll
            for (int d = 0; d < 3; d++) acc += JC[a][d] * J[b][d];
            Fc[a][b] = acc;
            Fc[b][a] = Fc[a][b];
        }
    }
    // line block: tanl = (v1 - v0)/ds1, z0 = v0 + tanl arc (float32 as well)
    const float i1 = (float)ids[1];
    const float t0 = -i1, t1 = i1, z0a = 1.0f - arc * i1, z1a = arc * i1;
    const float c00 = (float)Cv[0][0], c01 = (float)Cv[0][1], c11 = (float)Cv[1][1];
    float Fl[2][2];
    Fl[0][0] = t0 * (t0 * c00 + t1 * c01) + t1 * (t0 * c01 + t1 * c11);
    Fl[1][0] = z0a * (t0 * c00 + t1 * c01) + z1a * (t0 * c01 + t1 * c11);
    Fl[1][1] = z0a * (z0a * c00 + z1a * c01) + z1a * (z0a * c01 + z1a * c11);
    Fl[0][1] = Fl[1][0];
    float *par = p.trk_params + k * 5;
    par[0] = -kf;
    par[1] = phi0;
    par[2] = (float)tanl;
    par[3] = d0;
    par[4] = (float)z0;
    // order (kappa, phi0, tanl, d0, z0): circle block on {0,1,3}, line on {2,4}
    float *cv = p.trk_cov + k * 15;
    cv[0] = Fc[0][0];
    cv[1] = Fc[1][0]; cv[2] = Fc[1][1];
    cv[3] = 0.f; cv[4] = 0.f; cv[5] = Fl[0][0];
    cv[6] = Fc[2][0]; cv[7] = Fc[2][1]; cv[8] = 0.f; cv[9] = Fc[2][2];
    cv[10] = 0.f; cv[11] = 0.f; cv[12] = Fl[1][0]; cv[13] = 0.f; cv[14] = Fl[1][1];
    p.trk_chi2[k] = (float)chi2;
    p.trk_ndf[k] = (int8_t)(2 * N - 5);
}

// One kernel per hit count (3, 4, 5, and 6..8), so each is compiled for its
// own register footprint; the tracks of each count occupy a contiguous range
// of track indices (see k_select_tracks), which each kernel walks.  R: the
// precision of the normal equations (double, or float for the all-float32
// variant).
template <int N, typename R>
__global__ void __launch_bounds__(kThreads) k_fit(Params p) {
    constexpr int c = N - 3;
    int64_t k0 = 0;
#pragma unroll
    for (int q = 0; q < c; q++) k0 += p.counters[C_TRK_CNT + q];
    const int64_t k1 = min(k0 + p.counters[C_TRK_CNT + c], p.cap_tracks);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = k0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < k1; k += stride) {
        const int32_t t = p.trk_tuple[k];
        if (N < 6) {
            fit_track<N, R>(p, k, t);
        } else {
            const int n = p.tup_n[t];
            if (n == 6) fit_track<6, R>(p, k, t);
            else if (n == 7) fit_track<7, R>(p, k, t);
            else fit_track<8, R>(p, k, t);
        }
    }
}

template <typename R>
void launch_fit_r(const Params &p, int grid, cudaStream_t s) {
    {
        KernelTimer t("k_fit<3>", s);
        k_fit<3, R><<<grid, kThreads, 0, s>>>(p);
    }
    {
        KernelTimer t("k_fit<4>", s);
        k_fit<4, R><<<grid, kThreads, 0, s>>>(p);
    }
    {
        KernelTimer t("k_fit<5>", s);
        k_fit<5, R><<<grid, kThreads, 0, s>>>(p);
    }
    KernelTimer t("k_fit<6..8>", s);
    k_fit<6, R><<<grid, kThreads, 0, s>>>(p);
}

void launch_fit(const Params &p, int grid, cudaStream_t s) {
    if (p.fit.solve_fp32) launch_fit_r<float>(p, grid, s);
    else launch_fit_r<double>(p, grid, s);
}

}  // namespace ptk
