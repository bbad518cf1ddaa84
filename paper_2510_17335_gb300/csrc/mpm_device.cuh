// Device-side physics of the MLS-MPM sand substep (DDBot, arXiv 2510.17335,
// Sec. III-A, Algorithm 1, Eqs. (3)-(7)) and of its adjoint (Sec. III-D,
// Appendix B), for sm_103a. FP32 state; the SVD + return mapping is redone in
// FP64 for the rare ill-conditioned deformation gradient.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm_types.h"
#include "mpm_reg.h"

#if defined(__CUDACC__)
#define MPM_HD __host__ __device__
#else
#define MPM_HD
#endif

namespace mpm {

// ---------------------------------------------------------------------------
// small helpers (host and device: the math below is also compiled for the
// host by a CPU test of the kernels' arithmetic)
// ---------------------------------------------------------------------------
template <typename T> MPM_HD __forceinline__ T dsqrt(T x);
template <> MPM_HD __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }
template <> MPM_HD __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }
template <typename T> MPM_HD __forceinline__ T dlog(T x);
template <> MPM_HD __forceinline__ float dlog<float>(float x) { return logf(x); }
template <> MPM_HD __forceinline__ double dlog<double>(double x) { return log(x); }
template <typename T> MPM_HD __forceinline__ T dexp(T x);
template <> MPM_HD __forceinline__ float dexp<float>(float x) { return expf(x); }
template <> MPM_HD __forceinline__ double dexp<double>(double x) { return exp(x); }
template <typename T> MPM_HD __forceinline__ T dlog1p(T x);
template <> MPM_HD __forceinline__ float dlog1p<float>(float x) { return log1pf(x); }
template <> MPM_HD __forceinline__ double dlog1p<double>(double x) { return log1p(x); }
template <typename T> MPM_HD __forceinline__ T dfma(T a, T b, T c);
template <> MPM_HD __forceinline__ float dfma<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <> MPM_HD __forceinline__ double dfma<double>(double a, double b, double c) { return fma(a, b, c); }
template <typename T> MPM_HD __forceinline__ T dexpm1(T x);
template <> MPM_HD __forceinline__ float dexpm1<float>(float x) { return expm1f(x); }
template <> MPM_HD __forceinline__ double dexpm1<double>(double x) { return expm1(x); }

// Jacobi rotations are skipped only for an (almost) exactly zero off-diagonal:
// H's entries are small, so any threshold tied to 1 would cap their accuracy.
template <typename T> MPM_HD __forceinline__ T jacobi_tiny();
template <> MPM_HD __forceinline__ float jacobi_tiny<float>() { return 1e-35f; }
template <> MPM_HD __forceinline__ double jacobi_tiny<double>() { return 1e-300; }
template <typename T> struct Sweeps;
#ifndef MPM_SVD_SWEEPS
#define MPM_SVD_SWEEPS 4
#endif
template <> struct Sweeps<float> { static constexpr int n = MPM_SVD_SWEEPS; };

// 1/sqrt(x) and 1/x for FP32 without the branches of the IEEE operations:
// the hardware approximation (device) refined by one Newton step, which
// brings it to about an ulp. The host, which compiles this code for the CPU
// test of the kernels' arithmetic, uses the exact operations.
MPM_HD __forceinline__ float rsqrt_nr(float x) {
#if defined(__CUDA_ARCH__)
    const float y = rsqrtf(x);
    return y * fmaf(-0.5f * x, y * y, 1.5f);
#else
    return 1.0f / sqrtf(x);
#endif
}
// for |x| in [2^-126, 2^126]
MPM_HD __forceinline__ float rcp_nr(float x) {
#if defined(__CUDA_ARCH__)
    const float y = __fdividef(1.0f, x);
    return fmaf(y, fmaf(-x, y, 1.0f), y);
#else
    return 1.0f / x;
#endif
}
template <> struct Sweeps<double> { static constexpr int n = 10; };

// ---------------------------------------------------------------------------
// 3x3 SVD: cyclic Jacobi eigen-decomposition of H = F^T F - I (gives V and
// sigma^2 - 1), then U from the columns of F V. U and V are proper rotations;
// the smallest singular value carries the sign of det F.
//
// H is formed with error-free products and sums (fma / TwoSum), so that its
// eigenvalues keep full relative accuracy when F is close to a rotation: the
// log strains 0.5 log1p(sigma^2 - 1) of a nearly unstrained particle are then
// exact to a few ulps of themselves instead of to a few ulps of 1, which is
// what the apex and yield decisions of the return mapping need in FP32.
// ---------------------------------------------------------------------------
template <typename T>
MPM_HD __forceinline__ void two_sum(T a, T b, T& s, T& e) {
    s = a + b;
    const T bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// sum_k x_k y_k - shift, compensated
template <typename T>
MPM_HD __forceinline__ T dot3_minus(T x0, T y0, T x1, T y1, T x2, T y2, T shift) {
    const T p0 = x0 * y0, p1 = x1 * y1, p2 = x2 * y2;
    const T e0 = dfma<T>(x0, y0, -p0), e1 = dfma<T>(x1, y1, -p1), e2 = dfma<T>(x2, y2, -p2);
    T s, c1, c2, c3;
    two_sum<T>(p0, p1, s, c1);
    two_sum<T>(s, p2, s, c2);
    two_sum<T>(s, -shift, s, c3);
    return s + (((c1 + c2) + c3) + ((e0 + e1) + e2));
}

// FP32 rotation: tan(theta) = sgn(d) e / (|d| + sqrt(d^2 + e^2)) with
// d = g_qq - g_pp, e = 2 g_pq, both first scaled by 1/max(|d|, |e|) (the
// quotient does not depend on that scale, so the reciprocal need not be
// exact) so that nothing under- or overflows; then no division, square root
// or branch remains. The diagonal update is Rutishauser's g -/+ t g_pq.
template <int p, int q, int r>
MPM_HD __forceinline__ void jacobi_rotate_f32(float (&G)[3][3], float (&V)[3][3]) {
    const float gpq = G[p][q], gpp = G[p][p], gqq = G[q][q];
    const bool on = fabsf(gpq) > jacobi_tiny<float>();
    const float d = gqq - gpp, e = 2.0f * gpq;
    const float inv = rcp_nr(on ? fmaxf(fabsf(d), fabsf(e)) : 1.0f);
    const float dn = d * inv, en = e * inv;
    const float r2 = fmaf(dn, dn, en * en);   // in [1, 2]
    const float root = r2 * rsqrt_nr(r2);
    float t = (d >= 0.0f ? en : -en) * rcp_nr(fabsf(dn) + root);
    t = on ? t : 0.0f;
    const float c = rsqrt_nr(fmaf(t, t, 1.0f)), s = c * t;
    G[p][p] = fmaf(-t, gpq, gpp);
    G[q][q] = fmaf(t, gpq, gqq);
    G[p][q] = G[q][p] = on ? 0.0f : gpq;
    const float grp = G[r][p], grq = G[r][q];
    G[r][p] = G[p][r] = c * grp - s * grq;
    G[r][q] = G[q][r] = s * grp + c * grq;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float a = V[k][p], b = V[k][q];
        V[k][p] = c * a - s * b;
        V[k][q] = s * a + c * b;
    }
}

template <typename T, int p, int q, int r>
MPM_HD __forceinline__ void jacobi_rotate(T (&G)[3][3], T (&V)[3][3]) {
    if constexpr (sizeof(T) == sizeof(float)) {
        jacobi_rotate_f32<p, q, r>(G, V);
    } else {
    const T gpq = G[p][q], gpp = G[p][p], gqq = G[q][q];
    if (!(fabs(gpq) > jacobi_tiny<T>())) return;
    const T zeta = (gqq - gpp) / (T(2) * gpq);
    T t;
    if (fabs(zeta) > T(1e15))
        t = T(0.5) / zeta;
    else
        t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + dsqrt<T>(T(1) + zeta * zeta));
    const T c = T(1) / dsqrt<T>(T(1) + t * t), s = c * t;
    G[p][p] = gpp - t * gpq;
    G[q][q] = gqq + t * gpq;
    G[p][q] = G[q][p] = T(0);
    const T grp = G[r][p], grq = G[r][q];
    G[r][p] = G[p][r] = c * grp - s * grq;
    G[r][q] = G[q][r] = s * grp + c * grq;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const T a = V[k][p], b = V[k][q];
        V[k][p] = c * a - s * b;
        V[k][q] = s * a + c * b;
    }
    }
}

// 1/sqrt(x) and 1/x: FP32 through rsqrt_nr / rcp_nr, FP64 exact
template <typename T> MPM_HD __forceinline__ T rsqrt_t(T x) { return T(1) / dsqrt<T>(x); }
template <> MPM_HD __forceinline__ float rsqrt_t<float>(float x) { return rsqrt_nr(x); }
template <typename T> MPM_HD __forceinline__ T rcp_t(T x) { return T(1) / x; }
template <> MPM_HD __forceinline__ float rcp_t<float>(float x) { return rcp_nr(x); }

// h[k] = sigma_k^2 - 1 to full relative accuracy
template <typename T>
MPM_HD __forceinline__ void svd3(const T (&F)[3][3], T (&U)[3][3], T (&s)[3], T (&V)[3][3], T (&h)[3]) {
    T G[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            if (j >= i)
                G[i][j] = dot3_minus<T>(F[0][i], F[0][j], F[1][i], F[1][j], F[2][i], F[2][j], i == j ? T(1) : T(0));
            else
                G[i][j] = G[j][i];
            V[i][j] = (i == j) ? T(1) : T(0);
        }
#pragma unroll
    for (int sw = 0; sw < Sweeps<T>::n; sw++) {
        jacobi_rotate<T, 0, 1, 2>(G, V);
        jacobi_rotate<T, 0, 2, 1>(G, V);
        jacobi_rotate<T, 1, 2, 0>(G, V);
    }
    // order: i = largest, m = smallest, j = the middle one
    const T l0 = G[0][0], l1 = G[1][1], l2 = G[2][2];
    int m = 0;
    if (l1 < l0) m = 1;
    if (l2 < (m == 0 ? l0 : l1)) m = 2;
    int i = (m == 0) ? 1 : 0;
    int j = 3 - m - i;
    const T li = (i == 0) ? l0 : l1;
    const T lj = (j == 1) ? l1 : l2;
    if (lj > li) { int tmp = i; i = j; j = tmp; }
    // B = F V, column k
    T b[3][3];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int k = 0; k < 3; k++) b[r][k] = F[r][0] * V[0][k] + F[r][1] * V[1][k] + F[r][2] * V[2][k];
    T bi[3], bj[3], bm[3];
#pragma unroll
    for (int r = 0; r < 3; r++) {
        bi[r] = (i == 0) ? b[r][0] : ((i == 1) ? b[r][1] : b[r][2]);
        bj[r] = (j == 0) ? b[r][0] : ((j == 1) ? b[r][1] : b[r][2]);
        bm[r] = (m == 0) ? b[r][0] : ((m == 1) ? b[r][1] : b[r][2]);
    }
    T ui[3], uj[3], um[3];
    const T ni = bi[0] * bi[0] + bi[1] * bi[1] + bi[2] * bi[2];
    const T inv_si = rsqrt_t<T>(ni);
    const T si = ni * inv_si;
    if (!(si > T(1e-30))) {
        // F == 0: any rotations will do
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int k = 0; k < 3; k++) U[r][k] = (r == k) ? T(1) : T(0);
        s[0] = s[1] = s[2] = T(0);
        h[0] = h[1] = h[2] = T(-1);
        return;
    }
#pragma unroll
    for (int r = 0; r < 3; r++) ui[r] = bi[r] * inv_si;
    const T dij = ui[0] * bj[0] + ui[1] * bj[1] + ui[2] * bj[2];
#pragma unroll
    for (int r = 0; r < 3; r++) uj[r] = bj[r] - dij * ui[r];
    const T nj = uj[0] * uj[0] + uj[1] * uj[1] + uj[2] * uj[2];
    const T inv_sj = rsqrt_t<T>(nj);
    T sj = nj * inv_sj;
    if (!(sj > T(1e-30) * si)) {
        // rank one: any unit vector orthogonal to u_i
        // (static indices only: a runtime index would put the caller's arrays in local memory)
        int a = 0;
        if (fabs(ui[1]) < fabs(ui[0])) a = 1;
        if (fabs(ui[2]) < fabs(a == 0 ? ui[0] : ui[1])) a = 2;
        const T d = a == 0 ? ui[0] : (a == 1 ? ui[1] : ui[2]);
#pragma unroll
        for (int r = 0; r < 3; r++) uj[r] = (r == a ? T(1) : T(0)) - d * ui[r];
        const T ne = dsqrt<T>(uj[0] * uj[0] + uj[1] * uj[1] + uj[2] * uj[2]);
#pragma unroll
        for (int r = 0; r < 3; r++) uj[r] /= ne;
        sj = uj[0] * bj[0] + uj[1] * bj[1] + uj[2] * bj[2];
    } else {
#pragma unroll
        for (int r = 0; r < 3; r++) uj[r] *= inv_sj;
        sj = uj[0] * bj[0] + uj[1] * bj[1] + uj[2] * bj[2];
    }
    // u_m completes a right-handed frame: (i, j, m) cyclic -> u_i x u_j
    const T par = (((j - i + 3) % 3) == 1) ? T(1) : T(-1);
    um[0] = par * (ui[1] * uj[2] - ui[2] * uj[1]);
    um[1] = par * (ui[2] * uj[0] - ui[0] * uj[2]);
    um[2] = par * (ui[0] * uj[1] - ui[1] * uj[0]);
    const T sm = um[0] * bm[0] + um[1] * bm[1] + um[2] * bm[2];
#pragma unroll
    for (int r = 0; r < 3; r++) {
        const T c0 = (i == 0) ? ui[r] : ((j == 0) ? uj[r] : um[r]);
        const T c1 = (i == 1) ? ui[r] : ((j == 1) ? uj[r] : um[r]);
        const T c2 = (i == 2) ? ui[r] : ((j == 2) ? uj[r] : um[r]);
        U[r][0] = c0;
        U[r][1] = c1;
        U[r][2] = c2;
    }
#pragma unroll
    for (int k = 0; k < 3; k++) s[k] = (k == i) ? si : ((k == j) ? sj : sm);
    h[0] = l0;
    h[1] = l1;
    h[2] = l2;
}

// ---------------------------------------------------------------------------
// Drucker-Prager return on the singular values and the SVK log-strain
// stress eigenvalues (Eqs. (3)-(7)).
// ---------------------------------------------------------------------------
template <typename T>
struct Spectral {
    T U[3][3], V[3][3], s[3];
    T h[3];               // s^2 - 1, accurate for small strains
    T eps[3], deps[3];    // ln max(s, s_min) and its derivative in s
    T ehat[3], nh, tr, kappa;
    T shat[3], e[3], t[3];
    int kase;             // 0: tr > 0 (apex, S^ = I); 1: inside the cone; 2: onto the cone
};

template <typename T>
MPM_HD __forceinline__ void return_map(Spectral<T>& S, T mu, T lam, T beta, T smin) {
    S.tr = T(0);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const bool ok = S.s[k] > smin;
        // ln s = 0.5 log1p(s^2 - 1), exact for s near 1
        S.eps[k] = ok ? T(0.5) * dlog1p<T>(S.h[k]) : dlog<T>(smin);
        S.deps[k] = ok ? rcp_t<T>(S.s[k]) : T(0);
        S.tr += S.eps[k];
    }
    T n2 = T(0);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        S.ehat[k] = S.eps[k] - S.tr * T(1.0 / 3.0);
        n2 += S.ehat[k] * S.ehat[k];
    }
    S.nh = dsqrt<T>(n2);
    const T dg = S.nh + beta * S.tr;
    S.kappa = T(0);
    if (S.tr > T(0)) {
        S.kase = 0;
#pragma unroll
        for (int k = 0; k < 3; k++) { S.shat[k] = T(1); S.e[k] = T(0); }
    } else if (dg <= T(0) || S.nh <= T(1e-12)) {
        S.kase = 1;
#pragma unroll
        for (int k = 0; k < 3; k++) { S.shat[k] = S.s[k]; S.e[k] = S.eps[k]; }
    } else {
        S.kase = 2;
        const T inv_nh = rcp_t<T>(S.nh);
        const T r = dg * inv_nh;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            S.e[k] = S.eps[k] - r * S.ehat[k];
            S.shat[k] = dexp<T>(S.e[k]);
        }
        S.kappa = -beta * S.tr * inv_nh;
    }
    const T se = S.e[0] + S.e[1] + S.e[2];
#pragma unroll
    for (int k = 0; k < 3; k++) S.t[k] = T(2) * mu * S.e[k] + lam * se;
}

// trial F -> spectral data (SVD + return mapping)
template <typename T>
MPM_HD __forceinline__ void constitutive_spectral(const T (&Ft)[3][3], T mu, T lam, T beta, T smin,
                                                      Spectral<T>& S) {
    svd3<T>(Ft, S.U, S.s, S.V, S.h);
    return_map<T>(S, mu, lam, beta, smin);
}

// F' = U diag(shat) V^T and tau = U diag(t) U^T
template <typename T, typename O>
MPM_HD __forceinline__ void spectral_outputs(const Spectral<T>& S, O (&Fn)[3][3], O (&tau)[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            T f = T(0), g = T(0);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                f += S.U[a][k] * S.shat[k] * S.V[b][k];
                g += S.U[a][k] * S.t[k] * S.U[b][k];
            }
            Fn[a][b] = O(f);
            tau[a][b] = O(g);
        }
}

// ill-conditioned or non-finite FP32 results are redone in FP64
MPM_HD __forceinline__ bool needs_fp64(const Spectral<float>& S) {
    const float amax = fmaxf(fabsf(S.s[0]), fmaxf(fabsf(S.s[1]), fabsf(S.s[2])));
    const float amin = fminf(fabsf(S.s[0]), fminf(fabsf(S.s[1]), fabsf(S.s[2])));
    return !(amin >= 1e-3f * amax) || !isfinite(amax);
}

// forward constitutive step with the FP64 fallback kept out of line
MPM_HD __noinline__ void constitutive_fp64(const float (&Ft)[3][3], float mu, float lam, float beta, float smin,
                                               float (&Fn)[3][3], float (&tau)[3][3]) {
    double Fd[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) Fd[a][b] = Ft[a][b];
    Spectral<double> S;
    constitutive_spectral<double>(Fd, mu, lam, beta, smin, S);
    spectral_outputs<double, float>(S, Fn, tau);
}

MPM_HD __forceinline__ bool constitutive(const float (&Ft)[3][3], float mu, float lam, float beta, float smin,
                                             float (&Fn)[3][3], float (&tau)[3][3]) {
    Spectral<float> S;
    constitutive_spectral<float>(Ft, mu, lam, beta, smin, S);
    if (needs_fp64(S)) {
        constitutive_fp64(Ft, mu, lam, beta, smin, Fn, tau);
        return true;
    }
    spectral_outputs<float, float>(S, Fn, tau);
    return false;
}

// ---------------------------------------------------------------------------
// Adjoint of the constitutive step. In the frame K = U^T dFt V the diagonal
// carries d(sigma); each pair (i, j) of the off-diagonal mixes through the
// divided differences (f_i - f_j)/(s_i - s_j) and (f_i + f_j)/(s_i + s_j) of
// the isotropic maps s -> shat and s -> t. The first quotient is evaluated
// through expm1 so that it stays exact at s_i = s_j.
// ---------------------------------------------------------------------------
// x / expm1(x) and expm1(k x) / expm1(x), given em = expm1(x); below
// |x| = 1e-30 they equal their limits 1 and k to working precision
template <typename T>
MPM_HD __forceinline__ T xm1(T x, T em) { return fabs(x) < T(1e-30) ? T(1) : x * rcp_t<T>(em); }
template <typename T>
MPM_HD __forceinline__ T em1ratio(T k, T x, T em) {
    return fabs(x) < T(1e-30) ? k : dexpm1<T>(k * x) * rcp_t<T>(em);
}

template <typename T>
MPM_HD __forceinline__ void constitutive_adjoint_spectral(const Spectral<T>& S, T mu, T lam, T alpha, T beta,
                                                              T smin, const T (&gFn)[3][3], const T (&gtau)[3][3],
                                                              T (&gFt)[3][3], T& gmu, T& glam, T& galpha) {
    // output adjoints in the singular frames: G = U^T gFn V, Th = U^T gtau U
    T G[3][3], Th[3][3];
    {
        T a1[3][3], a2[3][3];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                a1[a][b] = S.U[0][a] * gFn[0][b] + S.U[1][a] * gFn[1][b] + S.U[2][a] * gFn[2][b];
                a2[a][b] = S.U[0][a] * gtau[0][b] + S.U[1][a] * gtau[1][b] + S.U[2][a] * gtau[2][b];
            }
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                G[a][b] = a1[a][0] * S.V[0][b] + a1[a][1] * S.V[1][b] + a1[a][2] * S.V[2][b];
                Th[a][b] = a2[a][0] * S.U[0][b] + a2[a][1] * S.U[1][b] + a2[a][2] * S.U[2][b];
            }
    }
    // singular-value adjoints as vector-Jacobian products of
    // t = 2 mu e + lam (sum e) 1, shat = exp(e) (case 2) or s (case 1)
    const T tb[3] = {Th[0][0], Th[1][1], Th[2][2]};
    const T stb = tb[0] + tb[1] + tb[2];
    const T se = S.e[0] + S.e[1] + S.e[2];
    gmu += T(2) * (tb[0] * S.e[0] + tb[1] * S.e[1] + tb[2] * S.e[2]);
    glam += stb * se;
    T sb[3] = {T(0), T(0), T(0)};
    if (S.kase == 1) {
#pragma unroll
        for (int i = 0; i < 3; i++) sb[i] = G[i][i] + (T(2) * mu * tb[i] + lam * stb) * S.deps[i];
    } else if (S.kase == 2) {
        const T inv_nh = rcp_t<T>(S.nh);
        T eb[3], eh[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            eb[i] = T(2) * mu * tb[i] + lam * stb + S.shat[i] * G[i][i];
            eh[i] = S.ehat[i] * inv_nh;
        }
        const T sE = eb[0] + eb[1] + eb[2];
        const T eE = eb[0] * eh[0] + eb[1] * eh[1] + eb[2] * eh[2];
        const T third = sE * T(1.0 / 3.0);
        // e = (tr/3) 1 - beta tr ehat: eps_bar = (sum eb)/3 1 - beta [(eb.eh) 1 + tr/nh (P eb - (eb.eh) eh)]
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const T epsb = third - beta * (eE + S.tr * inv_nh * ((eb[i] - third) - eE * eh[i]));
            sb[i] = epsb * S.deps[i];
        }
        // beta = (3 lam + 2 mu)/(2 mu) alpha and de/dbeta = -tr ehat
        const T gb = -S.tr * eE;
        gmu += gb * alpha * (T(-1.5) * lam / (mu * mu));
        glam += gb * alpha * (T(1.5) / mu);
        galpha += gb * (T(1) + T(1.5) * lam / mu);
    }
    T K[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) K[a][b] = (a == b) ? sb[a] : T(0);
    // off-diagonal pairs: divided differences of shat and t
#pragma unroll
    for (int pr = 0; pr < 3; pr++) {
        const int i = (pr == 2) ? 1 : 0;
        const int j = (pr == 0) ? 1 : 2;
        const T si = S.s[i], sj = S.s[j];
        const bool smooth = (si > smin) && (sj > smin);
        const T dsig = si - sj;
        T sum = si + sj;
        if (fabs(sum) < T(1e-30)) sum = T(1e-30);
        const T inv_sum = rcp_t<T>(sum);
        // 1/s_j where smooth (s_j > smin)
        const T inv_sj = S.deps[j];
        // clamped singular values (below smin) only: plain quotients, 0 when equal
        const bool sep = fabs(dsig) > T(1e-30);
        T ds, dd, q1;
        if (S.kase == 0) {
            ds = T(0);
            dd = T(2) * inv_sum;
            q1 = T(0);
        } else if (S.kase == 1) {
            ds = T(1);
            dd = T(1);
            if (smooth) {
                const T D = S.eps[i] - S.eps[j];
                q1 = T(2) * mu * xm1<T>(D, dexpm1<T>(D)) * inv_sj;
            } else {
                q1 = sep ? (S.t[i] - S.t[j]) / dsig : T(0);
            }
        } else {
            if (smooth) {
                const T D = S.eps[i] - S.eps[j];
                const T em = dexpm1<T>(D);
                ds = S.shat[j] * inv_sj * em1ratio<T>(S.kappa, D, em);
                q1 = T(2) * mu * S.kappa * xm1<T>(D, em) * inv_sj;
            } else {
                ds = sep ? (S.shat[i] - S.shat[j]) / dsig : T(0);
                q1 = sep ? (S.t[i] - S.t[j]) / dsig : T(0);
            }
            dd = (S.shat[i] + S.shat[j]) * inv_sum;
        }
        const T q2 = (S.t[i] - S.t[j]) * inv_sum;
        const T a = T(0.5) * (ds + dd), b = T(0.5) * (ds - dd);
        const T Gij = G[i][j], Gji = G[j][i];
        const T St = Th[i][j] + Th[j][i];
        K[i][j] = a * Gij + b * Gji + T(0.5) * St * (q1 - q2);
        K[j][i] = b * Gij + a * Gji + T(0.5) * St * (q1 + q2);
    }
    // gFt = U K V^T
#pragma unroll
    for (int a = 0; a < 3; a++) {
        T r0 = S.U[a][0] * K[0][0] + S.U[a][1] * K[1][0] + S.U[a][2] * K[2][0];
        T r1 = S.U[a][0] * K[0][1] + S.U[a][1] * K[1][1] + S.U[a][2] * K[2][1];
        T r2 = S.U[a][0] * K[0][2] + S.U[a][1] * K[1][2] + S.U[a][2] * K[2][2];
#pragma unroll
        for (int b = 0; b < 3; b++) gFt[a][b] = r0 * S.V[b][0] + r1 * S.V[b][1] + r2 * S.V[b][2];
    }
}

MPM_HD __noinline__ void constitutive_adjoint_fp64(const float (&Ft)[3][3], float mu, float lam, float alpha,
                                                       float beta, float smin, const float (&gFn)[3][3],
                                                       const float (&gtau)[3][3], float (&tau)[3][3],
                                                       float (&gFt)[3][3], float& gmu, float& glam, float& galpha) {
    double Fd[3][3], gF[3][3], gT[3][3], out[3][3], Fn[3][3], td[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) { Fd[a][b] = Ft[a][b]; gF[a][b] = gFn[a][b]; gT[a][b] = gtau[a][b]; }
    Spectral<double> S;
    constitutive_spectral<double>(Fd, mu, lam, beta, smin, S);
    spectral_outputs<double, double>(S, Fn, td);
    double m = 0, l = 0, al = 0;
    constitutive_adjoint_spectral<double>(S, mu, lam, alpha, beta, smin, gF, gT, out, m, l, al);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) { gFt[a][b] = float(out[a][b]); tau[a][b] = float(td[a][b]); }
    gmu += float(m);
    glam += float(l);
    galpha += float(al);
}

// ---------------------------------------------------------------------------
// Quadratic B-spline stencil (MLS-MPM, Hu et al. 2018)
// ---------------------------------------------------------------------------
struct Stencil {
    int base[3];
    float fx[3];
    float w[3][3];
    float dw[3][3];   // derivative in x (already times inv_dx)
};

// Returns false if x is outside [dx, (res-2) dx) or not finite; base is then
// clamped so that every access stays inside the grid.
__device__ __forceinline__ bool make_stencil(const InstDev& I, const float (&x)[3], Stencil& st) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float X = x[a] * I.inv_dx;
        ok = ok && (X >= 1.0f) && (X < float(I.res[a] - 2));
        int b = __float2int_rd(X - 0.5f);
        const int bc = min(max(b, 0), I.res[a] - 3);
        ok = ok && (b == bc);
        b = bc;
        st.base[a] = b;
        const float f = X - float(b);
        st.fx[a] = f;
        const float t0 = 1.5f - f, t1 = f - 1.0f, t2 = f - 0.5f;
        st.w[a][0] = 0.5f * t0 * t0;
        st.w[a][1] = 0.75f - t1 * t1;
        st.w[a][2] = 0.5f * t2 * t2;
        st.dw[a][0] = -t0 * I.inv_dx;
        st.dw[a][1] = -2.0f * t1 * I.inv_dx;
        st.dw[a][2] = t2 * I.inv_dx;
    }
    return ok;
}

// blocked grid layout: 4x4x4 nodes per block, blocks in (x, y, z) row-major
__device__ __forceinline__ void node_offsets(const InstDev& I, const Stencil& st, int (&ox)[3], int (&oy)[3],
                                             int (&oz)[3]) {
    const int sx = I.nb[1] * I.nb[2] * 64, sy = I.nb[2] * 64;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int ix = st.base[0] + a, iy = st.base[1] + a, iz = st.base[2] + a;
        ox[a] = (ix >> 2) * sx + (ix & 3) * 16;
        oy[a] = (iy >> 2) * sy + (iy & 3) * 4;
        oz[a] = (iz >> 2) * 64 + (iz & 3);
    }
}

// ---------------------------------------------------------------------------
// Shovel: box SDF contact with Coulomb friction (Sec. III-A, collision)
// ---------------------------------------------------------------------------
struct Pose {
    float c[3], psi, cd[3], psid;
};

__device__ __forceinline__ Pose load_pose(const InstDev& I, int substep) {
    Pose P;
    if (I.n_poses <= 0) {
        P.c[0] = P.c[1] = P.c[2] = -1e6f;
        P.psi = 0.0f;
        P.cd[0] = P.cd[1] = P.cd[2] = 0.0f;
        P.psid = 0.0f;
        return P;
    }
    const bool past = substep >= I.n_poses;
    const int s = past ? I.n_poses - 1 : substep;
    const float* p = I.poses + 8 * s;
    P.c[0] = p[0]; P.c[1] = p[1]; P.c[2] = p[2]; P.psi = p[3];
    P.cd[0] = past ? 0.0f : p[4];
    P.cd[1] = past ? 0.0f : p[5];
    P.cd[2] = past ? 0.0f : p[6];
    P.psid = past ? 0.0f : p[7];
    return P;
}

// inside test; on success n (world) and nl (local) face normals
MPM_HD __forceinline__ bool shovel_inside(const InstDev& I, const Pose& P, float cs, float sn, const float (&q)[3],
                                              float (&n)[3], float (&nl)[3]) {
    const float r0 = q[0] - P.c[0], r1 = q[1] - P.c[1], r2 = q[2] - P.c[2];
    const float l0 = cs * r0 - sn * r1;
    const float l1 = sn * r0 + cs * r1 - I.sh[1];
    const float l2 = r2;
    const float d0 = fabsf(l0) - I.sh[0], d1 = fabsf(l1) - I.sh[1], d2 = fabsf(l2) - I.sh[2];
    if (!(d0 < 0.0f && d1 < 0.0f && d2 < 0.0f)) return false;
    // nearest face; faces whose distances are within 1e-7 m of each other
    // (an edge or corner) resolve to the lowest axis index
    int a = 0;
    float dm = d0;
    if (d1 > dm + 1e-7f) { a = 1; dm = d1; }
    if (d2 > dm + 1e-7f) { a = 2; }
    nl[0] = nl[1] = nl[2] = 0.0f;
    const float lv = (a == 0) ? l0 : ((a == 1) ? l1 : l2);
    nl[a] = lv > -1e-7f ? 1.0f : -1.0f;   // within 1e-7 m of the mid-plane: the + face
    n[0] = cs * nl[0] + sn * nl[1];
    n[1] = -sn * nl[0] + cs * nl[1];
    n[2] = nl[2];
    return true;
}

MPM_HD __forceinline__ void shovel_project(const InstDev& I, const Pose& P, float cs, float sn, const float (&q)[3],
                                               float (&v)[3]) {
    float n[3], nl[3];
    if (!shovel_inside(I, P, cs, sn, q, n, nl)) return;
    const float r0 = q[0] - P.c[0], r1 = q[1] - P.c[1];
    const float vs0 = P.cd[0] + P.psid * r1, vs1 = P.cd[1] - P.psid * r0, vs2 = P.cd[2];
    const float u0 = v[0] - vs0, u1 = v[1] - vs1, u2 = v[2] - vs2;
    const float un = u0 * n[0] + u1 * n[1] + u2 * n[2];
    if (un >= 0.0f) return;
    const float t0 = u0 - un * n[0], t1 = u1 - un * n[1], t2 = u2 - un * n[2];
    const float L = sqrtf(t0 * t0 + t1 * t1 + t2 * t2);
    float f = 0.0f;
    if (L > 0.0f) f = fmaxf(0.0f, 1.0f + I.friction * un / L);
    v[0] = vs0 + f * t0;
    v[1] = vs1 + f * t1;
    v[2] = vs2 + f * t2;
}

// reverse of shovel_project: g (adjoint of the output) -> adds to gv, gq, gp[8]
MPM_HD __forceinline__ void shovel_project_adj(const InstDev& I, const Pose& P, float cs, float sn,
                                                   const float (&q)[3], const float (&v)[3], const float (&g)[3],
                                                   float (&gv)[3], float (&gq)[3], float (&gp)[8]) {
    float n[3], nl[3];
    if (!shovel_inside(I, P, cs, sn, q, n, nl)) {
        gv[0] += g[0]; gv[1] += g[1]; gv[2] += g[2];
        return;
    }
    const float r0 = q[0] - P.c[0], r1 = q[1] - P.c[1];
    const float vs0 = P.cd[0] + P.psid * r1, vs1 = P.cd[1] - P.psid * r0, vs2 = P.cd[2];
    const float u[3] = {v[0] - vs0, v[1] - vs1, v[2] - vs2};
    const float un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    if (un >= 0.0f) {
        gv[0] += g[0]; gv[1] += g[1]; gv[2] += g[2];
        return;
    }
    const float ut[3] = {u[0] - un * n[0], u[1] - un * n[1], u[2] - un * n[2]};
    const float L = sqrtf(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
    float gvs[3] = {g[0], g[1], g[2]};
    float gu[3] = {0.0f, 0.0f, 0.0f}, gn[3] = {0.0f, 0.0f, 0.0f};
    const float f = L > 0.0f ? 1.0f + I.friction * un / L : 0.0f;
    if (L > 0.0f && f > 0.0f) {
        const float gdot = g[0] * ut[0] + g[1] * ut[1] + g[2] * ut[2];
        const float k = gdot * I.friction * un / (L * L * L);
        float gut[3];
#pragma unroll
        for (int a = 0; a < 3; a++) gut[a] = f * g[a] - k * ut[a];
        float gun = gdot * I.friction / L;
        const float gutn = gut[0] * n[0] + gut[1] * n[1] + gut[2] * n[2];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            gu[a] += gut[a];
            gn[a] -= un * gut[a];
        }
        gun -= gutn;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            gu[a] += gun * n[a];
            gn[a] += gun * u[a];
        }
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        gv[a] += gu[a];
        gvs[a] -= gu[a];
    }
    gp[4] += gvs[0];
    gp[5] += gvs[1];
    gp[6] += gvs[2];
    gp[7] += gvs[0] * r1 - gvs[1] * r0;
    const float gr0 = -P.psid * gvs[1], gr1 = P.psid * gvs[0];
    const float dn0 = -sn * nl[0] + cs * nl[1], dn1 = -cs * nl[0] - sn * nl[1];
    gp[3] += gn[0] * dn0 + gn[1] * dn1;
    gq[0] += gr0;
    gq[1] += gr1;
    gp[0] -= gr0;
    gp[1] -= gr1;
}

MPM_HD __forceinline__ float clipf(float g, float c) { return fminf(fmaxf(g, -c), c); }

// ---------------------------------------------------------------------------
// Block reduction of NV values per thread into dst (FP64 atomicAdd): each
// warp sums its 32 lanes in FP32 (a 32-term sum stays accurate to ~1e-6
// relative), the warp sums are then added in FP64 across the block and the
// blocks meet in FP64 atomics. FP64 shuffles would cost ~20 FP64 adds per
// thread at the FP64 pipe's 1/64 rate.
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_reduce_add(float (&v)[NV], double* dst, double* sred /* [NV*32] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; k++) sred[k * 32 + warp] = (double)v[k];
    __syncthreads();
    if (threadIdx.x < NV) {
        double x = 0.0;
        for (int w = 0; w < nw; w++) x += sred[threadIdx.x * 32 + w];
        if (x != 0.0) atomicAdd(dst + threadIdx.x, x);
    }
}

// one value per statistic: max (mode 1) or sum (mode 2) over the warp, then
// FP64 atomics into dst[0..NV) by lane 0 (largest magnitude via the integer
// order of non-negative doubles). All 32 lanes call it.
template <int NV>
__device__ __forceinline__ void warp_stat(int mode, float (&v)[NV], double* dst) {
#pragma unroll
    for (int k = 0; k < NV; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float w = __shfl_xor_sync(0xffffffffu, v[k], o);
            v[k] = mode == 1 ? fmaxf(v[k], w) : v[k] + w;
        }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < NV; k++) {
            if (!(v[k] > 0.0f)) continue;
            if (mode == 1)
                atomicMax(reinterpret_cast<unsigned long long*>(dst + k),
                          (unsigned long long)__double_as_longlong((double)v[k]));
            else
                atomicAdd(dst + k, (double)v[k]);
        }
}

// a value's contribution to a statistic
__device__ __forceinline__ float stat_of(int mode, float g) { return mode == 1 ? fabsf(g) : g * g; }

// block version of warp_stat: one atomic per statistic and CTA. All threads
// of the CTA call it; sred holds NV * 32 floats.
template <int NV>
__device__ __forceinline__ void block_stat(int mode, float (&v)[NV], double* dst, float* sred) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float w = __shfl_xor_sync(0xffffffffu, v[k], o);
            v[k] = mode == 1 ? fmaxf(v[k], w) : v[k] + w;
        }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; k++) sred[k * 32 + warp] = v[k];
    __syncthreads();
    if (threadIdx.x < NV) {
        double x = 0.0;
        for (int w = 0; w < nw; w++) {
            const double y = sred[threadIdx.x * 32 + w];
            x = mode == 1 ? fmax(x, y) : x + y;
        }
        if (x > 0.0) {
            if (mode == 1)
                atomicMax(reinterpret_cast<unsigned long long*>(dst + threadIdx.x),
                          (unsigned long long)__double_as_longlong(x));
            else
                atomicAdd(dst + threadIdx.x, x);
        }
    }
}

// Sum v over the warp and add it to dst (FP64 atomics, lane 0) when any lane
// has any: all 32 lanes must call it.
template <int NV>
__device__ __forceinline__ void warp_reduce_add(float (&v)[NV], double* dst, bool any) {
    if (!__any_sync(0xffffffffu, any)) return;
#pragma unroll
    for (int k = 0; k < NV; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < NV; k++)
            if (v[k] != 0.0f) atomicAdd(dst + k, (double)v[k]);
}

// ---------------------------------------------------------------------------
// Shared-memory tile for the 27-node scatters (P2G and the G2P adjoint).
// A CTA takes the bounding box of its particles' stencils; if it holds at
// most kTileNodes nodes, contributions are summed in shared memory and the
// CTA then adds every touched node to the global grid with one float4
// atomic. Otherwise (particles of the chunk far apart) the CTA scatters
// straight into the global grid. The decision is uniform per CTA.
// ---------------------------------------------------------------------------
constexpr int kTileNodes = 512;

struct TileSmem {
    float c[4][kTileNodes];   // the four accumulated components, SoA
    int lo[3], dim[3];
    int tiled;
};

// bounding box of the stencils of the active threads' particles: lo and
// dim (nodes per axis; 0 when no thread is active) are written by thread 0
// and visible to all after the call; all threads of the CTA must call it
__device__ __forceinline__ void stencil_bbox(bool active, const Stencil& st, int nthreads, int* lo_out,
                                             int* dim_out) {
    int lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        lo[a] = active ? st.base[a] : 0x3fffffff;
        hi[a] = active ? st.base[a] : -0x3fffffff;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    __shared__ int s_lo[3][32], s_hi[3][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (nthreads + 31) >> 5;
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < 3; a++) { s_lo[a][warp] = lo[a]; s_hi[a][warp] = hi[a]; }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            int l = s_lo[a][0], h = s_hi[a][0];
            for (int w = 1; w < nw; w++) { l = min(l, s_lo[a][w]); h = max(h, s_hi[a][w]); }
            lo_out[a] = l;
            dim_out[a] = (h >= l) ? h - l + 3 : 0;
        }
    }
    __syncthreads();
}

// the CTA's scatter tile: bounding box, tiled flag, zeroed sums; all threads
// of the CTA must call it
__device__ __forceinline__ void tile_begin(TileSmem& T, bool active, const Stencil& st, int nthreads) {
    stencil_bbox(active, st, nthreads, T.lo, T.dim);
    if (threadIdx.x == 0) {
        const int n = T.dim[0] * T.dim[1] * T.dim[2];
        T.tiled = (n > 0 && n <= kTileNodes) ? 1 : 0;
    }
    __syncthreads();
    if (T.tiled) {
        const int n = T.dim[0] * T.dim[1] * T.dim[2];
        for (int i = threadIdx.x; i < n; i += nthreads) {
            T.c[0][i] = 0.f; T.c[1][i] = 0.f; T.c[2][i] = 0.f; T.c[3][i] = 0.f;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void red_shared(float* p, float v) {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)), "f"(v) : "memory");
}

// add val to node base + (i, j, k): into the tile, or to the global grid
__device__ __forceinline__ void tile_add(TileSmem& T, float4* grid, int gofs, const Stencil& st, int i, int j, int k,
                                         float4 val, int ncomp) {
    if (T.tiled) {
        const int t = ((st.base[0] + i - T.lo[0]) * T.dim[1] + (st.base[1] + j - T.lo[1])) * T.dim[2] +
                      (st.base[2] + k - T.lo[2]);
        red_shared(&T.c[0][t], val.x);
        red_shared(&T.c[1][t], val.y);
        red_shared(&T.c[2][t], val.z);
        if (ncomp == 4) red_shared(&T.c[3][t], val.w);
    } else {
        atomicAdd(grid + gofs, val);
    }
}

// Programmatic dependent launch: the kernels of the substep path may be
// scheduled while the previous kernel in the stream is finishing; each of
// them calls this first, which returns once that grid has completed and its
// memory writes are visible (a no-op for a kernel launched normally).
__device__ __forceinline__ void wait_previous_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Touched grid blocks of one substep, kept in the int array `flags`:
//   flags[b] (b < n_blocks)     1 once block b received a P2G contribution
//   flags[n_blocks]             number of listed blocks
//   flags[n_blocks + 1 + i]     the i-th listed block, in no particular order
// The grid kernels walk the list instead of testing every block's flag.
// The kernel after the one that zeroes the flags (or a memset) empties it.
__device__ __forceinline__ void mark_block(int* flags, int n_blocks, int b) {
    // test first: the load mostly hits L1; the thread whose exchange sets the
    // flag lists the block
    if (flags[b] == 0 && atomicExch(flags + b, 1) == 0) flags[n_blocks + 1 + atomicAdd(flags + n_blocks, 1)] = b;
}

// flush a tile to the global grid (blocked layout of instance I); marks the
// grid blocks that received mass when flags != nullptr
__device__ __forceinline__ void tile_flush(TileSmem& T, const InstDev& I, float4* grid, int* flags, int n_blocks,
                                           int nthreads) {
    __syncthreads();
    if (!T.tiled) return;
    const int n = T.dim[0] * T.dim[1] * T.dim[2];
    const int sx = I.nb[1] * I.nb[2] * 64, sy = I.nb[2] * 64;
    for (int t = threadIdx.x; t < n; t += nthreads) {
        const float4 v = make_float4(T.c[0][t], T.c[1][t], T.c[2][t], T.c[3][t]);
        if (v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f) continue;
        const int iz = T.lo[2] + t % T.dim[2];
        const int iy = T.lo[1] + (t / T.dim[2]) % T.dim[1];
        const int ix = T.lo[0] + t / (T.dim[1] * T.dim[2]);
        const int ofs = (ix >> 2) * sx + (ix & 3) * 16 + (iy >> 2) * sy + (iy & 3) * 4 + (iz >> 2) * 64 + (iz & 3);
        atomicAdd(grid + I.node_off + ofs, v);
        if (flags) mark_block(flags, n_blocks, I.blk_off + ((ix >> 2) * I.nb[1] + (iy >> 2)) * I.nb[2] + (iz >> 2));
    }
}

}  // namespace mpm
