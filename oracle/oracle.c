/*
 * FP64 CPU oracle: MLS-MPM substep for sand/soil (DDBot, arXiv 2510.17335,
 * Sec. III-A, Algorithm 1, Eqs. (3)-(7)) and its reverse-mode adjoint
 * (Sec. III-D, Appendix B), plus the skill-to-action mapping (Sec. III-B,
 * Algorithm 2) and its Jacobian (Appendix A, rounded phase lengths), and
 * the surface observation and height-map distance of Sec. III-A (Eq. (2)).
 *
 * TEST INFRASTRUCTURE ONLY: plain, slow, written for a reader to check it
 * against the paper. Only tests, the smoke check and the benchmark's CPU
 * baseline use it. Every loop runs in the order the paper states; grid and
 * particle work is done one particle / one node at a time.
 *
 * Readings where the paper is silent (each one is also listed in the
 * design notes of the repository):
 *   - MLS-MPM (Hu et al. 2018, cited in Sec. III-A) with quadratic
 *     B-splines; the P2G stress term uses the Kirchhoff stress
 *     tau = P' F'^T because Sec. III-A imposes det F' = 1.
 *   - eps = ln max(sigma, sigma_min); the singular values are those of the
 *     trial F (Algorithm 1, SVD step).
 *   - contact: box SDF, contact where the SDF is negative, Coulomb
 *     projection of the relative velocity.
 *   - walls: a velocity component pointing out of the domain is zeroed on
 *     nodes within `bound` of a face.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_EDOMAIN (-4)

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------ */
/* 3x3 matrix helpers, row-major                                       */
/* ------------------------------------------------------------------ */
static void mm(const double* A, const double* B, double* C) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * k + j];
            T[3 * i + j] = s;
        }
    memcpy(C, T, sizeof T);
}
/* C = A^T B */
static void mtm(const double* A, const double* B, double* C) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += A[3 * k + i] * B[3 * k + j];
            T[3 * i + j] = s;
        }
    memcpy(C, T, sizeof T);
}
/* C = A B^T */
static void mmt(const double* A, const double* B, double* C) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * j + k];
            T[3 * i + j] = s;
        }
    memcpy(C, T, sizeof T);
}
/* U diag(d) V^T */
static void udvt(const double* U, const double* d, const double* V, double* out) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += U[3 * i + k] * d[k] * V[3 * j + k];
            out[3 * i + j] = s;
        }
}

/* ------------------------------------------------------------------ */
/* SVD: one-sided (Hestenes) Jacobi on the columns of F, run to         */
/* convergence in FP64. Columns of A = F V are orthogonalised; their    */
/* norms are the singular values.                                       */
/* ------------------------------------------------------------------ */
void orc_svd3(const double F[9], double U[9], double S[3], double V[9]) {
    double A[9], W[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    memcpy(A, F, sizeof A);
    static const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int sweep = 0; sweep < 60; sweep++) {
        int rotated = 0;
        for (int r = 0; r < 3; r++) {
            int p = P[r][0], q = P[r][1];
            double al = 0, be = 0, ga = 0;
            for (int k = 0; k < 3; k++) {
                al += A[3 * k + p] * A[3 * k + p];
                be += A[3 * k + q] * A[3 * k + q];
                ga += A[3 * k + p] * A[3 * k + q];
            }
            if (ga == 0.0 || fabs(ga) <= 1e-17 * sqrt(al * be)) continue;
            double zeta = (be - al) / (2.0 * ga);
            double t;
            if (fabs(zeta) > 1e150)
                t = 1.0 / (2.0 * zeta);
            else
                t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
            for (int k = 0; k < 3; k++) {
                double ap = A[3 * k + p], aq = A[3 * k + q];
                A[3 * k + p] = c * ap - s * aq;
                A[3 * k + q] = s * ap + c * aq;
                double wp = W[3 * k + p], wq = W[3 * k + q];
                W[3 * k + p] = c * wp - s * wq;
                W[3 * k + q] = s * wp + c * wq;
            }
            rotated = 1;
        }
        if (!rotated) break;
    }
    /* column norms, then sort descending; every swap also negates one
     * column (of A and W together) so that det W stays +1. */
    double nrm[3];
    for (int j = 0; j < 3; j++)
        nrm[j] = sqrt(A[j] * A[j] + A[3 + j] * A[3 + j] + A[6 + j] * A[6 + j]);
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2 - a; b++)
            if (nrm[b] < nrm[b + 1]) {
                double tn = nrm[b];
                nrm[b] = nrm[b + 1];
                nrm[b + 1] = tn;
                for (int k = 0; k < 3; k++) {
                    double ta = A[3 * k + b];
                    A[3 * k + b] = A[3 * k + b + 1];
                    A[3 * k + b + 1] = -ta;
                    double tw = W[3 * k + b];
                    W[3 * k + b] = W[3 * k + b + 1];
                    W[3 * k + b + 1] = -tw;
                }
            }
    memcpy(V, W, sizeof W);
    /* u1, u2 by normalisation (with fallbacks for rank deficiency); u3 is
     * u1 x u2 so that U is a proper rotation; S[2] = u3 . a3 is signed. */
    double u[3][3];
    for (int j = 0; j < 2; j++) {
        if (nrm[j] > 0) {
            for (int k = 0; k < 3; k++) u[j][k] = A[3 * k + j] / nrm[j];
        } else if (j == 0) {
            u[0][0] = 1; u[0][1] = 0; u[0][2] = 0;
        } else {
            /* any unit vector orthogonal to u1 */
            double e[3] = {0, 0, 0};
            int m = 0;
            for (int k = 1; k < 3; k++)
                if (fabs(u[0][k]) < fabs(u[0][m])) m = k;
            e[m] = 1;
            double d = e[0] * u[0][0] + e[1] * u[0][1] + e[2] * u[0][2];
            for (int k = 0; k < 3; k++) e[k] -= d * u[0][k];
            double ne = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
            for (int k = 0; k < 3; k++) u[1][k] = e[k] / ne;
        }
    }
    u[2][0] = u[0][1] * u[1][2] - u[0][2] * u[1][1];
    u[2][1] = u[0][2] * u[1][0] - u[0][0] * u[1][2];
    u[2][2] = u[0][0] * u[1][1] - u[0][1] * u[1][0];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) U[3 * i + j] = u[j][i];
    S[0] = nrm[0];
    S[1] = nrm[1];
    S[2] = u[2][0] * A[2] + u[2][1] * A[5] + u[2][2] * A[8];
}

/* ------------------------------------------------------------------ */
/* Material: Lame constants (Sec. III-A, Eq. (5)) and alpha_f           */
/* (Sec. III-A, Eq. (6)).                                               */
/* ------------------------------------------------------------------ */
void orc_material(double E, double nu, double phi_deg, double* mu, double* lam, double* alpha) {
    *mu = E / (2.0 * (1.0 + nu));
    *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    double sp = sin(phi_deg * ORC_PI / 180.0);
    *alpha = sqrt(2.0 / 3.0) * 2.0 * sp / (3.0 - sp);
}

/* ------------------------------------------------------------------ */
/* Constitutive model: SVK energy in log strain (Eq. (3)), its Piola     */
/* stress (Eq. (4)), Drucker-Prager return (Eqs. (6)-(7)), F' = U S^ V^T */
/* and the Kirchhoff stress P' F'^T (det F' := 1).                       */
/* ------------------------------------------------------------------ */
typedef struct {
    double U[9], V[9], sig[3];
    int kase; /* 0: tr(eps) > 0 -> S^ = I;  1: no projection;  2: cone projection */
    double eps[3], deps[3];
    double tr, ehat[3], nh, dg, beta, kappa;
    double shat[3], e[3], t[3];
} cons_state;

static void cons_eval(const double Ft[9], double mu, double lam, double alpha, double smin, cons_state* s) {
    orc_svd3(Ft, s->U, s->sig, s->V);
    s->tr = 0;
    for (int i = 0; i < 3; i++) {
        double sg = s->sig[i] > smin ? s->sig[i] : smin;
        s->eps[i] = log(sg);
        s->deps[i] = s->sig[i] > smin ? 1.0 / s->sig[i] : 0.0;
        s->tr += s->eps[i];
    }
    double n2 = 0;
    for (int i = 0; i < 3; i++) {
        s->ehat[i] = s->eps[i] - s->tr / 3.0;
        n2 += s->ehat[i] * s->ehat[i];
    }
    s->nh = sqrt(n2);
    s->beta = (3.0 * lam + 2.0 * mu) / (2.0 * mu) * alpha;
    s->dg = s->nh + s->beta * s->tr;
    s->kappa = 0;
    if (s->tr > 0) {
        s->kase = 0;
        for (int i = 0; i < 3; i++) { s->shat[i] = 1.0; s->e[i] = 0.0; }
    } else if (s->dg <= 0 || s->nh <= 1e-12) {
        s->kase = 1;
        for (int i = 0; i < 3; i++) { s->shat[i] = s->sig[i]; s->e[i] = s->eps[i]; }
    } else {
        s->kase = 2;
        for (int i = 0; i < 3; i++) {
            s->e[i] = s->eps[i] - s->dg * s->ehat[i] / s->nh;
            s->shat[i] = exp(s->e[i]);
        }
        s->kappa = -s->beta * s->tr / s->nh;
    }
    double se = s->e[0] + s->e[1] + s->e[2];
    for (int i = 0; i < 3; i++) s->t[i] = 2.0 * mu * s->e[i] + lam * se;
}

void orc_constitutive(const double Ft[9], double mu, double lam, double alpha, double sigma_min,
                      double Fn[9], double tau[9], double info[4]) {
    cons_state s;
    cons_eval(Ft, mu, lam, alpha, sigma_min, &s);
    udvt(s.U, s.shat, s.V, Fn);
    udvt(s.U, s.t, s.U, tau);
    if (info) {
        info[0] = s.kase;
        info[1] = s.tr;
        info[2] = s.dg;
        info[3] = s.nh;
    }
}

/* x / expm1(x), -> 1 at 0 */
static double x_over_expm1(double x) { return x == 0.0 ? 1.0 : x / expm1(x); }
/* expm1(k x) / expm1(x), -> k at 0 */
static double expm1_ratio(double k, double x) { return x == 0.0 ? k : expm1(k * x) / expm1(x); }

/* Reverse of the constitutive step. The trial F enters through its SVD;
 * F' = U diag(shat(sig)) V^T and tau = U diag(t(sig)) U^T are isotropic
 * functions of it, so in the frame K = U^T dF V the diagonal carries the
 * singular-value derivatives and each off-diagonal pair (i, j) mixes through
 * the divided differences (f_i - f_j)/(sig_i - sig_j) and
 * (f_i + f_j)/(sig_i + sig_j). Divided differences are evaluated in forms
 * that stay exact when sig_i = sig_j (the derivative limit). */
void orc_constitutive_adjoint(const double Ft[9], double mu, double lam, double alpha, double sigma_min,
                              const double gFn[9], const double gtau[9],
                              double gFt[9], double* gmu, double* glam, double* galpha) {
    cons_state s;
    cons_eval(Ft, mu, lam, alpha, sigma_min, &s);
    double G[9], T[9], tmp[9];
    mtm(s.U, gFn, tmp);
    mm(tmp, s.V, G);      /* U^T gFn V */
    mtm(s.U, gtau, tmp);
    mm(tmp, s.U, T);      /* U^T gtau U */

    /* Jacobians with respect to sig: J1 = d shat/d sig, Je = d e/d sig */
    double J1[9] = {0}, Je[9] = {0}, dsh_db[3] = {0}, de_db[3] = {0};
    if (s.kase == 1) {
        for (int i = 0; i < 3; i++) {
            J1[4 * i] = 1.0;
            Je[4 * i] = s.deps[i];
        }
    } else if (s.kase == 2) {
        double eh[3];
        for (int i = 0; i < 3; i++) eh[i] = s.ehat[i] / s.nh;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double Pij = (i == j ? 1.0 : 0.0) - 1.0 / 3.0;
                double de_deps = 1.0 / 3.0 - s.beta * (eh[i] + s.tr * (Pij - eh[i] * eh[j]) / s.nh);
                Je[3 * i + j] = de_deps * s.deps[j];
            }
        for (int i = 0; i < 3; i++) {
            for (int j = 0; j < 3; j++) J1[3 * i + j] = s.shat[i] * Je[3 * i + j];
            de_db[i] = -s.tr * eh[i];
            dsh_db[i] = s.shat[i] * de_db[i];
        }
    }
    /* t = 2 mu e + lam (sum e) 1 */
    double Jt[9], dt_db[3];
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++) {
            double colsum = Je[j] + Je[3 + j] + Je[6 + j];
            Jt[3 * i + j] = 2.0 * mu * Je[3 * i + j] + lam * colsum;
        }
        dt_db[i] = 2.0 * mu * de_db[i] + lam * (de_db[0] + de_db[1] + de_db[2]);
    }
    double K[9] = {0};
    for (int k = 0; k < 3; k++) {
        double g = 0;
        for (int i = 0; i < 3; i++) g += G[4 * i] * J1[3 * i + k] + T[4 * i] * Jt[3 * i + k];
        K[4 * k] = g;
    }
    double gbeta = 0, se = s.e[0] + s.e[1] + s.e[2];
    for (int i = 0; i < 3; i++) {
        gbeta += G[4 * i] * dsh_db[i] + T[4 * i] * dt_db[i];
        *gmu += T[4 * i] * 2.0 * s.e[i];
        *glam += T[4 * i] * se;
    }
    if (s.kase == 2) {
        double c = (3.0 * lam + 2.0 * mu) / (2.0 * mu);
        *gmu += gbeta * alpha * (-3.0 * lam / (2.0 * mu * mu));
        *glam += gbeta * alpha * 3.0 / (2.0 * mu);
        *galpha += gbeta * c;
    }
    static const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int r = 0; r < 3; r++) {
        int i = P[r][0], j = P[r][1];
        double si = s.sig[i], sj = s.sig[j];
        int smooth = si > sigma_min && sj > sigma_min;
        double dsig = si - sj;
        double sum = si + sj;
        if (fabs(sum) < 1e-300) sum = 1e-300;
        double ds, dd, q1, q2;
        /* generic divided difference with derivative limit */
        int close = fabs(dsig) <= 1e-12 * fmax(fabs(si), fabs(sj));
        if (s.kase == 0) {
            ds = 0.0;
            dd = 2.0 / sum;
            q1 = 0.0;
        } else if (s.kase == 1) {
            ds = 1.0;
            dd = 1.0;
            if (smooth)
                q1 = 2.0 * mu * x_over_expm1(s.eps[i] - s.eps[j]) / sj;
            else
                q1 = close ? (Jt[3 * i + i] - Jt[3 * i + j]) : (s.t[i] - s.t[j]) / dsig;
        } else {
            if (smooth) {
                double D = s.eps[i] - s.eps[j];
                ds = s.shat[j] / sj * expm1_ratio(s.kappa, D);
                q1 = 2.0 * mu * s.kappa * x_over_expm1(D) / sj;
            } else {
                ds = close ? (J1[3 * i + i] - J1[3 * i + j]) : (s.shat[i] - s.shat[j]) / dsig;
                q1 = close ? (Jt[3 * i + i] - Jt[3 * i + j]) : (s.t[i] - s.t[j]) / dsig;
            }
            dd = (s.shat[i] + s.shat[j]) / sum;
        }
        q2 = (s.t[i] - s.t[j]) / sum;
        double a = 0.5 * (ds + dd), b = 0.5 * (ds - dd);
        double Gij = G[3 * i + j], Gji = G[3 * j + i];
        K[3 * i + j] += a * Gij + b * Gji;
        K[3 * j + i] += b * Gij + a * Gji;
        double Sij = T[3 * i + j] + T[3 * j + i];
        K[3 * i + j] += 0.5 * Sij * (q1 - q2);
        K[3 * j + i] += 0.5 * Sij * (q1 + q2);
    }
    /* gFt = U K V^T */
    mm(s.U, K, tmp);
    mmt(tmp, s.V, gFt);
}

/* ------------------------------------------------------------------ */
/* Shovel: box SDF and Coulomb contact (Sec. III-A, collision).         */
/* ------------------------------------------------------------------ */
/* Returns 1 if q lies strictly inside the box; then n is the world normal of
 * the nearest face and n_local its local counterpart. */
static int shovel_inside(const orc_params* p, const double q[3], const double pose[8],
                         double n[3], double nloc[3]) {
    double cs = cos(pose[3]), sn = sin(pose[3]);
    double r[3] = {q[0] - pose[0], q[1] - pose[1], q[2] - pose[2]};
    /* local = R^T r - (0, hy, 0), R = [[cs, sn, 0], [-sn, cs, 0], [0, 0, 1]] */
    double l[3];
    l[0] = cs * r[0] - sn * r[1];
    l[1] = sn * r[0] + cs * r[1] - p->shovel_half[1];
    l[2] = r[2];
    double d[3];
    for (int k = 0; k < 3; k++) d[k] = fabs(l[k]) - p->shovel_half[k];
    if (!(d[0] < 0 && d[1] < 0 && d[2] < 0)) return 0;
    /* nearest face; at an edge or corner (face distances within 1e-7 m of
     * each other) the face of the lowest axis index is taken */
    int a = 0;
    for (int k = 1; k < 3; k++)
        if (d[k] > d[a] + 1e-7) a = k;
    nloc[0] = nloc[1] = nloc[2] = 0;
    /* a point within 1e-7 m of the mid-plane takes the + face */
    nloc[a] = l[a] > -1e-7 ? 1.0 : -1.0;
    n[0] = cs * nloc[0] + sn * nloc[1];
    n[1] = -sn * nloc[0] + cs * nloc[1];
    n[2] = nloc[2];
    return 1;
}

void orc_shovel_project(const orc_params* p, const double vel[3], const double q[3],
                        const double pose[8], double out[3]) {
    double n[3], nl[3];
    out[0] = vel[0]; out[1] = vel[1]; out[2] = vel[2];
    if (!p->shovel_on || !shovel_inside(p, q, pose, n, nl)) return;
    double r[3] = {q[0] - pose[0], q[1] - pose[1], q[2] - pose[2]};
    double vs[3] = {pose[4] + pose[7] * r[1], pose[5] - pose[7] * r[0], pose[6]};
    double u[3] = {vel[0] - vs[0], vel[1] - vs[1], vel[2] - vs[2]};
    double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    if (un >= 0) return;
    double ut[3] = {u[0] - un * n[0], u[1] - un * n[1], u[2] - un * n[2]};
    double L = sqrt(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
    double f = 0.0;
    if (L > 0) {
        f = 1.0 + p->friction * un / L;
        if (f < 0) f = 0.0;
    }
    for (int k = 0; k < 3; k++) out[k] = vs[k] + f * ut[k];
}

/* Reverse of orc_shovel_project: adds to gvel, gq, gpose. */
static void shovel_project_adjoint(const orc_params* p, const double vel[3], const double q[3],
                                   const double pose[8], const double gout[3],
                                   double gvel[3], double gq[3], double gpose[8]) {
    double n[3], nl[3];
    if (!p->shovel_on || !shovel_inside(p, q, pose, n, nl)) {
        for (int k = 0; k < 3; k++) gvel[k] += gout[k];
        return;
    }
    double cs = cos(pose[3]), sn = sin(pose[3]);
    double r[3] = {q[0] - pose[0], q[1] - pose[1], q[2] - pose[2]};
    double vs[3] = {pose[4] + pose[7] * r[1], pose[5] - pose[7] * r[0], pose[6]};
    double u[3] = {vel[0] - vs[0], vel[1] - vs[1], vel[2] - vs[2]};
    double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    if (un >= 0) {
        for (int k = 0; k < 3; k++) gvel[k] += gout[k];
        return;
    }
    double ut[3] = {u[0] - un * n[0], u[1] - un * n[1], u[2] - un * n[2]};
    double L = sqrt(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
    double gvs[3] = {gout[0], gout[1], gout[2]};
    double gu[3] = {0, 0, 0}, gn[3] = {0, 0, 0};
    double f = L > 0 ? 1.0 + p->friction * un / L : 0.0;
    if (L > 0 && f > 0) {
        /* out = vs + f ut, f = 1 + mu un / L */
        double gdot = gout[0] * ut[0] + gout[1] * ut[1] + gout[2] * ut[2];
        double gut[3], gun;
        for (int k = 0; k < 3; k++) gut[k] = f * gout[k] - gdot * p->friction * un / (L * L * L) * ut[k];
        gun = gdot * p->friction / L;
        /* ut = u - un n */
        double gutn = gut[0] * n[0] + gut[1] * n[1] + gut[2] * n[2];
        for (int k = 0; k < 3; k++) {
            gu[k] += gut[k];
            gn[k] -= un * gut[k];
        }
        gun -= gutn;
        /* un = u . n */
        for (int k = 0; k < 3; k++) {
            gu[k] += gun * n[k];
            gn[k] += gun * u[k];
        }
    }
    /* u = vel - vs */
    for (int k = 0; k < 3; k++) {
        gvel[k] += gu[k];
        gvs[k] -= gu[k];
    }
    /* vs = cdot + psidot * (r1, -r0, 0) */
    gpose[4] += gvs[0];
    gpose[5] += gvs[1];
    gpose[6] += gvs[2];
    gpose[7] += gvs[0] * r[1] - gvs[1] * r[0];
    double gr[3] = {-pose[7] * gvs[1], pose[7] * gvs[0], 0.0};
    /* n = R(psi) nloc */
    double dn[3] = {-sn * nl[0] + cs * nl[1], -cs * nl[0] - sn * nl[1], 0.0};
    gpose[3] += gn[0] * dn[0] + gn[1] * dn[1] + gn[2] * dn[2];
    /* r = q - c */
    for (int k = 0; k < 3; k++) {
        gq[k] += gr[k];
        gpose[k] -= gr[k];
    }
}

/* ------------------------------------------------------------------ */
/* Quadratic B-spline weights of MLS-MPM (Hu et al. 2018).              */
/* ------------------------------------------------------------------ */
typedef struct {
    int base[3];
    double fx[3], w[3][3], dw[3][3];
} stencil;

static int make_stencil(const orc_params* p, const double* xp, stencil* s) {
    double inv_dx = 1.0 / p->dx;
    int ok = 1;
    for (int a = 0; a < 3; a++) {
        double X = xp[a] * inv_dx;
        int b = (int)floor(X - 0.5);
        if (!(b >= 0 && b <= p->res[a] - 3)) ok = 0;
        s->base[a] = b;
        double f = X - b;
        s->fx[a] = f;
        s->w[a][0] = 0.5 * (1.5 - f) * (1.5 - f);
        s->w[a][1] = 0.75 - (f - 1.0) * (f - 1.0);
        s->w[a][2] = 0.5 * (f - 0.5) * (f - 0.5);
        s->dw[a][0] = -(1.5 - f) * inv_dx;
        s->dw[a][1] = -2.0 * (f - 1.0) * inv_dx;
        s->dw[a][2] = (f - 0.5) * inv_dx;
    }
    return ok;
}

static int64_t node_index(const orc_params* p, int i, int j, int k) {
    return ((int64_t)i * p->res[1] + j) * p->res[2] + k;
}

/* A box of grid nodes [o, o + d) per axis, stored row-major (x, y, z). The
 * whole grid is the box with o = 0 and d = res, whose index is node_index. */
typedef struct {
    int o[3], d[3];
} gview;

static gview whole_grid(const orc_params* p) {
    gview g = {{0, 0, 0}, {p->res[0], p->res[1], p->res[2]}};
    return g;
}

static int64_t view_index(const gview* g, int i, int j, int k) {
    return ((int64_t)(i - g->o[0]) * g->d[1] + (j - g->o[1])) * g->d[2] + (k - g->o[2]);
}

static int64_t view_size(const gview* g) { return (int64_t)g->d[0] * g->d[1] * g->d[2]; }

static int in_domain(const orc_params* p, const double* xp) {
    for (int a = 0; a < 3; a++)
        if (!(xp[a] >= p->dx && xp[a] < (p->res[a] - 2) * p->dx)) return 0;
    return 1;
}

/* Particle part of Algorithm 1 for particle q: F trial, SVD, constitutive,
 * P2G. Writes F' into Fout (if given) and scatters into m, mv (laid out as
 * the box g). */
static void p2g_one(const orc_params* p, double mu, double lam, double alpha, int64_t q, const double* x,
                    const double* v, const double* C, const double* F, double* Fout, const gview* g, double* m,
                    double* mv) {
    double mp = p->rho * p->vol;
    double inv_dx = 1.0 / p->dx;
    const double* Cp = C + 9 * q;
    double Ft[9], IC[9];
    for (int i = 0; i < 9; i++) IC[i] = p->dt * Cp[i] + (i % 4 == 0 ? 1.0 : 0.0);
    mm(IC, F + 9 * q, Ft);
    double Fn[9], tau[9];
    orc_constitutive(Ft, mu, lam, alpha, p->sigma_min, Fn, tau, NULL);
    if (Fout) memcpy(Fout + 9 * q, Fn, sizeof Fn);
    double A[9];
    for (int i = 0; i < 9; i++) A[i] = -p->dt * p->vol * 4.0 * inv_dx * inv_dx * tau[i] + mp * Cp[i];
    stencil s;
    make_stencil(p, x + 3 * q, &s);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            for (int c = 0; c < 3; c++) {
                double W = s.w[0][a] * s.w[1][b] * s.w[2][c];
                double d[3] = {(a - s.fx[0]) * p->dx, (b - s.fx[1]) * p->dx, (c - s.fx[2]) * p->dx};
                int64_t id = view_index(g, s.base[0] + a, s.base[1] + b, s.base[2] + c);
                m[id] += W * mp;
                for (int k = 0; k < 3; k++) {
                    double Ad = A[3 * k] * d[0] + A[3 * k + 1] * d[1] + A[3 * k + 2] * d[2];
                    mv[3 * id + k] += W * (mp * v[3 * q + k] + Ad);
                }
            }
}

/* Threads of the OpenMP paths: 1 runs the plain loops, one particle or node
 * at a time in index order. With more, particle loops are split across
 * threads; scatters go into per-thread grids over the box of the particles'
 * stencils, which are then added node by node in thread order, and scalar
 * sums are per-thread partials added in thread order: the same arithmetic
 * as one thread up to the order of the sums. */
static int orc_threads = 1;

void orc_set_threads(int n) { orc_threads = n < 1 ? 1 : n; }

int orc_get_threads(void) { return orc_threads; }

/* the box of nodes that the stencils of particles x[0..n) touch */
static gview stencil_box(const orc_params* p, int64_t n, const double* x) {
    int lo[3] = {p->res[0], p->res[1], p->res[2]}, hi[3] = {-1, -1, -1};
    for (int64_t q = 0; q < n; q++) {
        stencil s;
        make_stencil(p, x + 3 * q, &s);
        for (int a = 0; a < 3; a++) {
            if (s.base[a] < lo[a]) lo[a] = s.base[a];
            if (s.base[a] + 2 > hi[a]) hi[a] = s.base[a] + 2;
        }
    }
    gview g;
    for (int a = 0; a < 3; a++) {
        g.o[a] = n > 0 ? lo[a] : 0;
        g.d[a] = n > 0 ? hi[a] - lo[a] + 1 : 0;
    }
    return g;
}

/* adds the per-thread box grids part[t] (ncomp values per node) into the
 * whole grid dst, in thread order per node */
static void add_box_partials(const orc_params* p, const gview* g, int T, const double* part, int ncomp, double* dst) {
    const int64_t nb = view_size(g);
#ifdef _OPENMP
#pragma omp parallel for num_threads(orc_threads) schedule(static)
#endif
    for (int64_t b = 0; b < nb; b++) {
        const int iz = g->o[2] + (int)(b % g->d[2]);
        const int iy = g->o[1] + (int)((b / g->d[2]) % g->d[1]);
        const int ix = g->o[0] + (int)(b / ((int64_t)g->d[1] * g->d[2]));
        const int64_t id = node_index(p, ix, iy, iz);
        for (int t = 0; t < T; t++)
            for (int c = 0; c < ncomp; c++) dst[ncomp * id + c] += part[((int64_t)t * nb + b) * ncomp + c];
    }
}

/* Particle part of Algorithm 1 before the grid, for every particle: F
 * trial, SVD, constitutive, P2G. Writes F' into Fout and scatters into m,
 * mv (the whole grid, which the caller has zeroed). */
static void particle_to_grid(const orc_params* p, int64_t n, const double* x, const double* v,
                             const double* C, const double* F, double* Fout, double* m, double* mv) {
    double mu, lam, alpha;
    orc_material(p->E, p->nu, p->phi_deg, &mu, &lam, &alpha);
    if (orc_threads <= 1) {
        const gview g = whole_grid(p);
        for (int64_t q = 0; q < n; q++) p2g_one(p, mu, lam, alpha, q, x, v, C, F, Fout, &g, m, mv);
        return;
    }
    const gview g = stencil_box(p, n, x);
    const int T = orc_threads;
    const int64_t nb = view_size(&g);
    double* pm = calloc((size_t)T * nb, sizeof(double));
    double* pmv = calloc((size_t)T * nb * 3, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(T)
#endif
    {
#ifdef _OPENMP
        const int t = omp_get_thread_num();
#pragma omp for schedule(static)
#else
        const int t = 0;
#endif
        for (int64_t q = 0; q < n; q++) p2g_one(p, mu, lam, alpha, q, x, v, C, F, Fout, &g, pm + t * nb, pmv + 3 * t * nb);
    }
    add_box_partials(p, &g, T, pm, 1, m);
    add_box_partials(p, &g, T, pmv, 3, mv);
    free(pm);
    free(pmv);
}

/* Grid part of Algorithm 1: gravity, walls, shovel contact at one node. */
static void grid_node_update(const orc_params* p, int i, int j, int k, double m, const double* mv,
                             const double pose[8], double* vout) {
    int idx[3] = {i, j, k};
    double vg[3];
    for (int a = 0; a < 3; a++) vg[a] = mv[a] / m + p->dt * p->gravity[a];
    for (int a = 0; a < 3; a++) {
        if (idx[a] < p->bound && vg[a] < 0) vg[a] = 0;
        if (idx[a] > p->res[a] - p->bound && vg[a] > 0) vg[a] = 0;
    }
    double q[3] = {i * p->dx, j * p->dx, k * p->dx};
    orc_shovel_project(p, vg, q, pose, vout);
}

static void grid_update(const orc_params* p, const double* m, const double* mv, const double pose[8],
                        double* vout) {
    /* nodes are independent: threads give the same values */
#ifdef _OPENMP
#pragma omp parallel for num_threads(orc_threads) schedule(static) if (orc_threads > 1)
#endif
    for (int i = 0; i < p->res[0]; i++)
        for (int j = 0; j < p->res[1]; j++)
            for (int k = 0; k < p->res[2]; k++) {
                int64_t id = node_index(p, i, j, k);
                if (m[id] > 0)
                    grid_node_update(p, i, j, k, m[id], mv + 3 * id, pose, vout + 3 * id);
                else
                    vout[3 * id] = vout[3 * id + 1] = vout[3 * id + 2] = 0;
            }
}

/* G2P for one particle: APIC velocity and affine matrix from the grid. */
static void g2p_one(const orc_params* p, const double* xp, const double* vgrid, double vnew[3], double Cnew[9]) {
    stencil s;
    make_stencil(p, xp, &s);
    double inv_dx = 1.0 / p->dx;
    for (int k = 0; k < 3; k++) vnew[k] = 0;
    for (int k = 0; k < 9; k++) Cnew[k] = 0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            for (int c = 0; c < 3; c++) {
                double W = s.w[0][a] * s.w[1][b] * s.w[2][c];
                double d[3] = {(a - s.fx[0]) * p->dx, (b - s.fx[1]) * p->dx, (c - s.fx[2]) * p->dx};
                const double* vi = vgrid + 3 * node_index(p, s.base[0] + a, s.base[1] + b, s.base[2] + c);
                for (int r = 0; r < 3; r++) {
                    vnew[r] += W * vi[r];
                    for (int q = 0; q < 3; q++) Cnew[3 * r + q] += 4.0 * inv_dx * inv_dx * W * vi[r] * d[q];
                }
            }
}

static int64_t grid_size(const orc_params* p) { return (int64_t)p->res[0] * p->res[1] * p->res[2]; }

static int check_params(const orc_params* p) {
    if (p->res[0] < 4 || p->res[1] < 4 || p->res[2] < 4) return 0;
    if (!(p->dx > 0) || !(p->dt > 0) || !(p->vol > 0) || !(p->rho > 0) || !(p->E > 0)) return 0;
    if (!(p->nu > 0 && p->nu < 0.5)) return 0;
    return 1;
}

int orc_grid_of_substep(const orc_params* p, int64_t n, const double* x, const double* v,
                        const double* C, const double* F, const double pose[8],
                        double* m_out, double* mv_out, double* vout_out) {
    if (!check_params(p)) return ORC_EINVAL;
    for (int64_t q = 0; q < n; q++)
        if (!in_domain(p, x + 3 * q)) return ORC_EDOMAIN;
    int64_t G = grid_size(p);
    double* m = calloc(G, sizeof(double));
    double* mv = calloc(3 * G, sizeof(double));
    double* vo = calloc(3 * G, sizeof(double));
    particle_to_grid(p, n, x, v, C, F, NULL, m, mv);
    grid_update(p, m, mv, pose, vo);
    if (m_out) memcpy(m_out, m, G * sizeof(double));
    if (mv_out) memcpy(mv_out, mv, 3 * G * sizeof(double));
    if (vout_out) memcpy(vout_out, vo, 3 * G * sizeof(double));
    free(m); free(mv); free(vo);
    return ORC_OK;
}

/* One substep of Algorithm 1 in place. */
int orc_substep(const orc_params* p, int64_t n, double* x, double* v, double* C, double* F,
                const double pose[8]) {
    if (!check_params(p)) return ORC_EINVAL;
    for (int64_t q = 0; q < n; q++)
        if (!in_domain(p, x + 3 * q)) return ORC_EDOMAIN;
    int64_t G = grid_size(p);
    double* m = calloc(G, sizeof(double));
    double* mv = calloc(3 * G, sizeof(double));
    double* vo = calloc(3 * G, sizeof(double));
    /* particle loop: F trial, SVD, constitutive, P2G */
    particle_to_grid(p, n, x, v, C, F, F, m, mv);
    /* move agent: the pose of this substep is given; grid update */
    grid_update(p, m, mv, pose, vo);
    /* particle loop: G2P, particle collision, advection (particles are
     * independent: threads give the same values) */
    int status = ORC_OK;
#ifdef _OPENMP
#pragma omp parallel for num_threads(orc_threads) schedule(static) if (orc_threads > 1) reduction(min : status)
#endif
    for (int64_t q = 0; q < n; q++) {
        double vnew[3], Cnew[9], vpost[3];
        g2p_one(p, x + 3 * q, vo, vnew, Cnew);
        if (p->particle_collision)
            orc_shovel_project(p, vnew, x + 3 * q, pose, vpost);
        else
            memcpy(vpost, vnew, sizeof vpost);
        for (int k = 0; k < 3; k++) {
            v[3 * q + k] = vpost[k];
            x[3 * q + k] += p->dt * vpost[k];
        }
        memcpy(C + 9 * q, Cnew, sizeof Cnew);
        if (!in_domain(p, x + 3 * q)) status = ORC_EDOMAIN;
    }
    free(m); free(mv); free(vo);
    return status;
}

int orc_rollout(const orc_params* p, int64_t n, double* x, double* v, double* C, double* F,
                int nsub, const double* poses) {
    for (int s = 0; s < nsub; s++) {
        int st = orc_substep(p, n, x, v, C, F, poses + 8 * s);
        if (st != ORC_OK) return st;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Reverse-mode adjoint of a rollout (Sec. III-D; Appendix B for the    */
/* constitutive part). The whole trajectory is kept; each substep is    */
/* recomputed from its stored input state and then reversed.            */
/* ------------------------------------------------------------------ */
static double clipv(double g, const orc_params* p) {
    if (!p->clip_grads) return g;
    if (g > p->clip_value) return p->clip_value;
    if (g < -p->clip_value) return -p->clip_value;
    return g;
}

/* Clipping, dynamic scaling or normalisation of one whole adjoint vector
 * (Sec. III-E): the key variables are the particles' x, v, F and the grid's
 * m and velocities before and after the contact, each as one vector. */
void orc_grad_op(const orc_params* p, double* g, int64_t n) {
    if (p->clip_grads) {
        for (int64_t i = 0; i < n; i++) g[i] = clipv(g[i], p);
        return;
    }
    if (p->grad_scale == 1) {
        double mx = 0.0;
        for (int64_t i = 0; i < n; i++) mx = fabs(g[i]) > mx ? fabs(g[i]) : mx;
        if (!(mx > 0.0)) return;
        const double doom = round(log10(mx)) - p->oom_star;
        if (doom > 0.0) {
            const double div = pow(10.0, doom) + p->grad_delta;
            for (int64_t i = 0; i < n; i++) g[i] /= div;
        }
    } else if (p->grad_scale == 2) {
        double ss = 0.0;
        for (int64_t i = 0; i < n; i++) ss += g[i] * g[i];
        const double div = sqrt(ss) + p->grad_delta;
        for (int64_t i = 0; i < n; i++) g[i] /= div;
    }
}

/* Reverse of advection, particle collision and G2P for particle q of the
 * state x: reads its adjoints ax, av (already regularised) and aC, scatters
 * the grid-velocity adjoint into avo (laid out as the box g), adds to the
 * pose adjoint gpose and leaves the partial adjoint of x in ax. */
static void g2p_adjoint_one(const orc_params* p, int64_t q, const double* x, const double* vo, const double pose[8],
                            const gview* g, double* ax, const double* av, const double* aC, double* avo,
                            double gpose[8]) {
    double inv_dx = 1.0 / p->dx, kap = 4.0 * inv_dx * inv_dx;
    const double* xp = x + 3 * q;
    double gxp[3] = {ax[3 * q], ax[3 * q + 1], ax[3 * q + 2]};
    double gvpost[3];
    for (int k = 0; k < 3; k++) gvpost[k] = av[3 * q + k] + p->dt * ax[3 * q + k];
    double vnew[3], Cnew[9];
    g2p_one(p, xp, vo, vnew, Cnew);
    double gvnew[3] = {0, 0, 0};
    if (p->particle_collision)
        shovel_project_adjoint(p, vnew, xp, pose, gvpost, gvnew, gxp, gpose);
    else
        for (int k = 0; k < 3; k++) gvnew[k] = gvpost[k];
    const double* gCn = aC + 9 * q;
    stencil st;
    make_stencil(p, xp, &st);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            for (int c = 0; c < 3; c++) {
                int o[3] = {a, b, c};
                double wv[3] = {st.w[0][a], st.w[1][b], st.w[2][c]};
                double dwv[3] = {st.dw[0][a], st.dw[1][b], st.dw[2][c]};
                double W = wv[0] * wv[1] * wv[2];
                double gradW[3] = {dwv[0] * wv[1] * wv[2], wv[0] * dwv[1] * wv[2], wv[0] * wv[1] * dwv[2]};
                double d[3];
                for (int k = 0; k < 3; k++) d[k] = (o[k] - st.fx[k]) * p->dx;
                const double* vi = vo + 3 * node_index(p, st.base[0] + a, st.base[1] + b, st.base[2] + c);
                int64_t id = view_index(g, st.base[0] + a, st.base[1] + b, st.base[2] + c);
                double Wbar = 0, dbar[3] = {0, 0, 0};
                for (int r = 0; r < 3; r++) {
                    double Cd = gCn[3 * r] * d[0] + gCn[3 * r + 1] * d[1] + gCn[3 * r + 2] * d[2];
                    avo[3 * id + r] += W * gvnew[r] + kap * W * Cd;
                    Wbar += vi[r] * gvnew[r] + kap * vi[r] * Cd;
                    for (int k = 0; k < 3; k++) dbar[k] += kap * W * gCn[3 * r + k] * vi[r];
                }
                for (int k = 0; k < 3; k++) gxp[k] += Wbar * gradW[k] - dbar[k];
            }
    for (int k = 0; k < 3; k++) ax[3 * q + k] = gxp[k];
}

/* Reverse of the grid update for the nodes of slab x = i: from the
 * adjoint of the velocity after the contact (avo) to that of the momentum
 * before the division by the mass (amv, walls applied); adds to gpose. */
static void grid_adjoint_slab(const orc_params* p, int i, const double* m, const double* mv, const double pose[8],
                              const double* avo, double* amv, double gpose[8]) {
    for (int j = 0; j < p->res[1]; j++)
        for (int k = 0; k < p->res[2]; k++) {
            int64_t id = node_index(p, i, j, k);
            if (!(m[id] > 0)) continue;
            int idx[3] = {i, j, k};
            double vg[3], mask[3] = {1, 1, 1};
            for (int a = 0; a < 3; a++) vg[a] = mv[3 * id + a] / m[id] + p->dt * p->gravity[a];
            for (int a = 0; a < 3; a++) {
                if (idx[a] < p->bound && vg[a] < 0) { vg[a] = 0; mask[a] = 0; }
                if (idx[a] > p->res[a] - p->bound && vg[a] > 0) { vg[a] = 0; mask[a] = 0; }
            }
            double q[3] = {i * p->dx, j * p->dx, k * p->dx}, gq[3] = {0, 0, 0};
            double gvg[3] = {0, 0, 0};
            shovel_project_adjoint(p, vg, q, pose, avo + 3 * id, gvg, gq, gpose);
            for (int a = 0; a < 3; a++) amv[3 * id + a] = gvg[a] * mask[a];   /* v-bar before the contact */
        }
}

/* Reverse of P2G and of the constitutive step for particle q of the
 * state (x, v, C, F) with Kirchhoff stress tau: gathers the grid adjoints
 * am, amv; turns the adjoints of particle q (ax partial, aF) into those of
 * the state before the substep (ax, av, aC, aF) and adds to the sums of
 * dL/dmu, dL/dlambda, dL/dalpha and dL/dm_p. */
static void p2g_adjoint_one(const orc_params* p, double mu, double lam, double alpha, int64_t q, const double* x,
                            const double* v, const double* C, const double* F, const double* tau, const double* am,
                            const double* amv, double* ax, double* av, double* aC, double* aF, double* gmu_acc,
                            double* glam_acc, double* galpha_acc, double* gmp_acc) {
    double mp = p->rho * p->vol;
    double inv_dx = 1.0 / p->dx, kap = 4.0 * inv_dx * inv_dx;
    const double* xp = x + 3 * q;
    const double* Cp = C + 9 * q;
    const double* vp = v + 3 * q;
    double A[9];
    for (int i = 0; i < 9; i++) A[i] = -p->dt * p->vol * kap * tau[9 * q + i] + mp * Cp[i];
    double gxp[3] = {ax[3 * q], ax[3 * q + 1], ax[3 * q + 2]};
    double gvp[3] = {0, 0, 0}, gA[9] = {0}, gmpp = 0;
    stencil st;
    make_stencil(p, xp, &st);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            for (int c = 0; c < 3; c++) {
                int o[3] = {a, b, c};
                double wv[3] = {st.w[0][a], st.w[1][b], st.w[2][c]};
                double dwv[3] = {st.dw[0][a], st.dw[1][b], st.dw[2][c]};
                double W = wv[0] * wv[1] * wv[2];
                double gradW[3] = {dwv[0] * wv[1] * wv[2], wv[0] * dwv[1] * wv[2], wv[0] * wv[1] * dwv[2]};
                double d[3];
                for (int k = 0; k < 3; k++) d[k] = (o[k] - st.fx[k]) * p->dx;
                int64_t id = node_index(p, st.base[0] + a, st.base[1] + b, st.base[2] + c);
                const double* gmv = amv + 3 * id;
                double Wbar = am[id] * mp;
                double dbar[3] = {0, 0, 0};
                for (int r = 0; r < 3; r++) {
                    double Ad = A[3 * r] * d[0] + A[3 * r + 1] * d[1] + A[3 * r + 2] * d[2];
                    Wbar += gmv[r] * (mp * vp[r] + Ad);
                    gvp[r] += W * mp * gmv[r];
                    gmpp += W * gmv[r] * vp[r];
                    for (int k = 0; k < 3; k++) {
                        gA[3 * r + k] += W * gmv[r] * d[k];
                        dbar[k] += W * A[3 * r + k] * gmv[r];
                    }
                }
                gmpp += W * am[id];
                for (int k = 0; k < 3; k++) gxp[k] += Wbar * gradW[k] - dbar[k];
            }
    double gtau[9], gCp[9];
    for (int i = 0; i < 9; i++) {
        gtau[i] = -p->dt * p->vol * kap * gA[i];
        gCp[i] = mp * gA[i];
        gmpp += gA[i] * Cp[i];
    }
    double Ft[9], IC[9], gFt[9];
    for (int i = 0; i < 9; i++) IC[i] = p->dt * Cp[i] + (i % 4 == 0 ? 1.0 : 0.0);
    mm(IC, F + 9 * q, Ft);
    orc_constitutive_adjoint(Ft, mu, lam, alpha, p->sigma_min, aF + 9 * q, gtau, gFt, gmu_acc, glam_acc, galpha_acc);
    /* Ft = (I + dt C) F */
    double gFp[9], t2[9];
    mtm(IC, gFt, gFp);
    mmt(gFt, F + 9 * q, t2);
    for (int i = 0; i < 9; i++) gCp[i] += p->dt * t2[i];
    memcpy(ax + 3 * q, gxp, sizeof gxp);
    memcpy(av + 3 * q, gvp, sizeof gvp);
    memcpy(aC + 9 * q, gCp, sizeof gCp);
    memcpy(aF + 9 * q, gFp, sizeof gFp);
    *gmp_acc += gmpp;
}

int orc_rollout_adjoint(const orc_params* p, int64_t n, const double* x0, const double* v0,
                        const double* C0, const double* F0, int nsub, const double* poses,
                        const double* gx, const double* gv, const double* gC, const double* gF,
                        double* ax0, double* av0, double* aC0, double* aF0,
                        double gmat[4], double* gposes) {
    if (!check_params(p) || nsub < 0) return ORC_EINVAL;
    double mu, lam, alpha;
    orc_material(p->E, p->nu, p->phi_deg, &mu, &lam, &alpha);
    int64_t G = grid_size(p);
    /* tape of the states at the start of every substep */
    double* tx = malloc((size_t)(nsub + 1) * n * 3 * sizeof(double));
    double* tv = malloc((size_t)(nsub + 1) * n * 3 * sizeof(double));
    double* tC = malloc((size_t)(nsub + 1) * n * 9 * sizeof(double));
    double* tF = malloc((size_t)(nsub + 1) * n * 9 * sizeof(double));
    memcpy(tx, x0, n * 3 * sizeof(double));
    memcpy(tv, v0, n * 3 * sizeof(double));
    memcpy(tC, C0, n * 9 * sizeof(double));
    memcpy(tF, F0, n * 9 * sizeof(double));
    int status = ORC_OK;
    for (int s = 0; s < nsub && status == ORC_OK; s++) {
        memcpy(tx + (s + 1) * n * 3, tx + s * n * 3, n * 3 * sizeof(double));
        memcpy(tv + (s + 1) * n * 3, tv + s * n * 3, n * 3 * sizeof(double));
        memcpy(tC + (s + 1) * n * 9, tC + s * n * 9, n * 9 * sizeof(double));
        memcpy(tF + (s + 1) * n * 9, tF + s * n * 9, n * 9 * sizeof(double));
        status = orc_substep(p, n, tx + (s + 1) * n * 3, tv + (s + 1) * n * 3, tC + (s + 1) * n * 9,
                             tF + (s + 1) * n * 9, poses + 8 * s);
    }
    if (status != ORC_OK) {
        free(tx); free(tv); free(tC); free(tF);
        return status;
    }
    double* ax = calloc(n * 3, sizeof(double));
    double* av = calloc(n * 3, sizeof(double));
    double* aC = calloc(n * 9, sizeof(double));
    double* aF = calloc(n * 9, sizeof(double));
    if (gx) memcpy(ax, gx, n * 3 * sizeof(double));
    if (gv) memcpy(av, gv, n * 3 * sizeof(double));
    if (gC) memcpy(aC, gC, n * 9 * sizeof(double));
    if (gF) memcpy(aF, gF, n * 9 * sizeof(double));
    double* m = malloc(G * sizeof(double));
    double* mv = malloc(3 * G * sizeof(double));
    double* vo = malloc(3 * G * sizeof(double));
    double* am = malloc(G * sizeof(double));
    double* amv = malloc(3 * G * sizeof(double));
    double* avo = malloc(3 * G * sizeof(double));
    double* tau = malloc(n * 9 * sizeof(double));
    double gmu = 0, glam = 0, galpha = 0, gmp = 0;
    if (gposes) memset(gposes, 0, (size_t)nsub * 8 * sizeof(double));

    for (int s = nsub - 1; s >= 0; s--) {
        const double* x = tx + s * n * 3;
        const double* v = tv + s * n * 3;
        const double* C = tC + s * n * 9;
        const double* F = tF + s * n * 9;
        const double* pose = poses + 8 * s;
        double gpose[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        /* recompute the forward of this substep */
        memset(m, 0, G * sizeof(double));
        memset(mv, 0, 3 * G * sizeof(double));
        particle_to_grid(p, n, x, v, C, F, NULL, m, mv);
        grid_update(p, m, mv, pose, vo);
#ifdef _OPENMP
#pragma omp parallel for num_threads(orc_threads) schedule(static) if (orc_threads > 1)
#endif
        for (int64_t q = 0; q < n; q++) {
            double Ft[9], IC[9], Fn[9];
            for (int i = 0; i < 9; i++) IC[i] = p->dt * C[9 * q + i] + (i % 4 == 0 ? 1.0 : 0.0);
            mm(IC, F + 9 * q, Ft);
            orc_constitutive(Ft, mu, lam, alpha, p->sigma_min, Fn, tau + 9 * q, NULL);
        }
        /* regularised particle adjoints (Sec. III-E) */
        orc_grad_op(p, ax, n * 3);
        orc_grad_op(p, av, n * 3);
        orc_grad_op(p, aF, n * 9);

        /* reverse of advection, particle collision and G2P; the partial
         * adjoint of x is kept in ax, the grid velocity adjoint goes to avo */
        memset(avo, 0, 3 * G * sizeof(double));
        if (orc_threads <= 1) {
            const gview g = whole_grid(p);
            for (int64_t q = 0; q < n; q++) g2p_adjoint_one(p, q, x, vo, pose, &g, ax, av, aC, avo, gpose);
        } else {
            const gview g = stencil_box(p, n, x);
            const int T = orc_threads;
            const int64_t nb = view_size(&g);
            double* pavo = calloc((size_t)T * nb * 3, sizeof(double));
            double* pgp = calloc((size_t)T * 8, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(T)
#endif
            {
#ifdef _OPENMP
                const int t = omp_get_thread_num();
#pragma omp for schedule(static)
#else
                const int t = 0;
#endif
                for (int64_t q = 0; q < n; q++)
                    g2p_adjoint_one(p, q, x, vo, pose, &g, ax, av, aC, pavo + 3 * t * nb, pgp + 8 * t);
            }
            add_box_partials(p, &g, T, pavo, 3, avo);
            for (int t = 0; t < T; t++)
                for (int k = 0; k < 8; k++) gpose[k] += pgp[8 * t + k];
            free(pavo);
            free(pgp);
        }
        /* reverse of the grid update: the adjoint of the velocity after the
         * contact (regularised), then of the velocity before it (for every
         * node, then regularised), then of the mass (regularised) */
        orc_grad_op(p, avo, 3 * G);
        memset(am, 0, G * sizeof(double));
        memset(amv, 0, 3 * G * sizeof(double));
        if (orc_threads <= 1) {
            for (int i = 0; i < p->res[0]; i++) grid_adjoint_slab(p, i, m, mv, pose, avo, amv, gpose);
        } else {
            const int T = orc_threads;
            double* pgp = calloc((size_t)T * 8, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(T)
#endif
            {
#ifdef _OPENMP
                const int t = omp_get_thread_num();
#pragma omp for schedule(static)
#else
                const int t = 0;
#endif
                for (int i = 0; i < p->res[0]; i++) grid_adjoint_slab(p, i, m, mv, pose, avo, amv, pgp + 8 * t);
            }
            for (int t = 0; t < T; t++)
                for (int k = 0; k < 8; k++) gpose[k] += pgp[8 * t + k];
            free(pgp);
        }
        orc_grad_op(p, amv, 3 * G);
#ifdef _OPENMP
#pragma omp parallel for num_threads(orc_threads) schedule(static) if (orc_threads > 1)
#endif
        for (int64_t id = 0; id < G; id++) {
            if (!(m[id] > 0)) continue;
            double dot = 0;
            for (int a = 0; a < 3; a++) {
                dot += amv[3 * id + a] * mv[3 * id + a];
                amv[3 * id + a] /= m[id];
            }
            am[id] = -dot / (m[id] * m[id]);
        }
        orc_grad_op(p, am, G);
        /* reverse of P2G and the constitutive step */
        if (orc_threads <= 1) {
            for (int64_t q = 0; q < n; q++)
                p2g_adjoint_one(p, mu, lam, alpha, q, x, v, C, F, tau, am, amv, ax, av, aC, aF, &gmu, &glam, &galpha,
                                &gmp);
        } else {
            const int T = orc_threads;
            double* part = calloc((size_t)T * 4, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(T)
#endif
            {
#ifdef _OPENMP
                const int t = omp_get_thread_num();
#pragma omp for schedule(static)
#else
                const int t = 0;
#endif
                for (int64_t q = 0; q < n; q++)
                    p2g_adjoint_one(p, mu, lam, alpha, q, x, v, C, F, tau, am, amv, ax, av, aC, aF, part + 4 * t,
                                    part + 4 * t + 1, part + 4 * t + 2, part + 4 * t + 3);
            }
            for (int t = 0; t < T; t++) {
                gmu += part[4 * t];
                glam += part[4 * t + 1];
                galpha += part[4 * t + 2];
                gmp += part[4 * t + 3];
            }
            free(part);
        }
        if (gposes) memcpy(gposes + 8 * s, gpose, sizeof gpose);
    }
    /* material chain: mu(E, nu), lambda(E, nu), m_p = rho V_p, alpha(phi) */
    if (gmat) {
        double E = p->E, nu = p->nu;
        double dmu_dE = 1.0 / (2.0 * (1.0 + nu));
        double dmu_dnu = -E / (2.0 * (1.0 + nu) * (1.0 + nu));
        double dl_dE = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
        double dl_dnu = E * (1.0 + 2.0 * nu * nu) / ((1.0 + nu) * (1.0 + nu) * (1.0 - 2.0 * nu) * (1.0 - 2.0 * nu));
        double phi = p->phi_deg * ORC_PI / 180.0;
        double da_dphi = sqrt(2.0 / 3.0) * 6.0 * cos(phi) / ((3.0 - sin(phi)) * (3.0 - sin(phi)));
        gmat[0] = gmu * dmu_dE + glam * dl_dE;
        gmat[1] = gmu * dmu_dnu + glam * dl_dnu;
        gmat[2] = gmp * p->vol;
        gmat[3] = galpha * da_dphi * ORC_PI / 180.0;
    }
    if (ax0) memcpy(ax0, ax, n * 3 * sizeof(double));
    if (av0) memcpy(av0, av, n * 3 * sizeof(double));
    if (aC0) memcpy(aC0, aC, n * 9 * sizeof(double));
    if (aF0) memcpy(aF0, aF, n * 9 * sizeof(double));
    free(tx); free(tv); free(tC); free(tF);
    free(ax); free(av); free(aC); free(aF);
    free(m); free(mv); free(vo); free(am); free(amv); free(avo); free(tau);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Skill-to-action mapping, Sec. III-B and Algorithm 2, rounded phase   */
/* lengths. Paper frame (x forward, z up) -> simulator frame (x, y up). */
/* The sixth parameter sets the lift distance d4 = (theta_lift+1)*0.005 */
/* (theta_lift = 1 gives the paper's constant 0.01 m).                  */
/* ------------------------------------------------------------------ */
int orc_skill_actions(const double theta[6], double v_lin, double v_ang, double dt_step,
                      int max_actions, int unrounded, double* actions, int T[4], double* jac) {
    const double pi = ORC_PI;
    double th_disp = theta[0], th_rot = theta[1], th_ins = theta[2], th_pa = theta[3], th_pd = theta[4],
           th_lift = theta[5];
    /* phase 1 */
    double d1 = th_disp * 0.12, ph1 = th_rot * pi / 3.0;
    double Tfd1 = fabs(d1 / (v_lin * dt_step)), Tfp1 = fabs(ph1 / (v_ang * dt_step));
    double Tf1 = Tfd1 > Tfp1 ? Tfd1 : Tfp1;
    int T1 = (int)round(Tf1);
    /* phase 2 */
    double d2 = (th_ins + 1.0) * 0.03, ph2 = ph1 + pi / 2.0;
    int T2 = (int)round(d2 / (v_lin * dt_step));
    /* phase 3 */
    double d3 = (th_pd + 1.0) * 0.1 + 0.04, ph3 = (th_pa + 3.0) * pi / 3.0;
    int T3 = (int)round(fabs(d3 / (v_lin * dt_step)));
    /* phase 4 */
    double d4 = (th_lift + 1.0) * 0.005;
    double Tfd4 = d4 / (v_lin * dt_step);
    int T4 = (int)round(Tfp1 > Tfd4 ? Tfp1 : Tfd4);
    int Ttot = T1 + T2 + T3 + T4;
    if (T) { T[0] = T1; T[1] = T2; T[2] = T3; T[3] = T4; }
    if (Ttot > max_actions) return -1;
    /* phases 1 and 4 divide by the real-valued step counts in the unrounded
     * variant (Sec. III-B, the alternative mapping; phases 2 and 3 keep T_2,
     * T_3); the number of steps stays T_1, T_4 */
    double Tf4 = Tfp1 >= Tfd4 ? Tfp1 : Tfd4;
    double div1 = unrounded ? Tf1 : (double)T1, div4 = unrounded ? Tf4 : (double)T4;
    double dx1 = T1 > 0 ? d1 / div1 : 0, drx1 = T1 > 0 ? ph1 / div1 : 0;
    double dx2 = T2 > 0 ? d2 * cos(ph2) / T2 : 0, dz2 = T2 > 0 ? -d2 * sin(ph2) / T2 : 0;
    double dx3 = T3 > 0 ? d3 * cos(ph3) / T3 : 0, dz3 = T3 > 0 ? d3 * sin(ph3) / T3 : 0;
    double drx4 = T4 > 0 ? -ph1 / div4 : 0, dz4 = T4 > 0 ? d4 / div4 : 0;
    /* derivatives of the step divisors in the unrounded variant: the active
     * term of each max (the d term on ties in phase 1, the rotation term on
     * ties in phase 4, as the paper's case split reads) */
    const double sd1 = d1 > 0 ? 1.0 : (d1 < 0 ? -1.0 : 0.0), sp1 = ph1 > 0 ? 1.0 : (ph1 < 0 ? -1.0 : 0.0);
    double dTf1_ddisp = 0, dTf1_drot = 0, dTf4_drot = 0, dTf4_dlift = 0;
    if (Tfd1 >= Tfp1) dTf1_ddisp = sd1 * 0.12 / (v_lin * dt_step);
    else dTf1_drot = sp1 * (pi / 3.0) / (v_ang * dt_step);
    if (Tfp1 >= Tfd4) dTf4_drot = sp1 * (pi / 3.0) / (v_ang * dt_step);
    else dTf4_dlift = 0.005 / (v_lin * dt_step);
    memset(actions, 0, (size_t)Ttot * 6 * sizeof(double));
    if (jac) memset(jac, 0, (size_t)Ttot * 36 * sizeof(double));
    /* jac index: t*36 + k*6 + j  (k: action component, j: parameter) */
    for (int t = 0; t < Ttot; t++) {
        double* a = actions + 6 * t;
        double* J = jac ? jac + 36 * t : NULL;
        if (t < T1) {
            a[0] = dx1;
            a[3] = drx1;
            if (J && !unrounded) {
                J[0 * 6 + 0] = 0.12 / T1;
                J[3 * 6 + 1] = (pi / 3.0) / T1;
            } else if (J) {
                /* d(d1 / Tf1), d(ph1 / Tf1) */
                J[0 * 6 + 0] = 0.12 / Tf1 - d1 * dTf1_ddisp / (Tf1 * Tf1);
                J[0 * 6 + 1] = -d1 * dTf1_drot / (Tf1 * Tf1);
                J[3 * 6 + 0] = -ph1 * dTf1_ddisp / (Tf1 * Tf1);
                J[3 * 6 + 1] = (pi / 3.0) / Tf1 - ph1 * dTf1_drot / (Tf1 * Tf1);
            }
        } else if (t < T1 + T2) {
            a[0] = dx2;
            a[1] = dz2;
            if (J) {
                J[0 * 6 + 2] = 0.03 * cos(ph2) / T2;
                J[0 * 6 + 1] = -d2 * sin(ph2) * (pi / 3.0) / T2;
                J[1 * 6 + 2] = -0.03 * sin(ph2) / T2;
                J[1 * 6 + 1] = -d2 * cos(ph2) * (pi / 3.0) / T2;
            }
        } else if (t < T1 + T2 + T3) {
            a[0] = dx3;
            a[1] = dz3;
            if (J) {
                J[0 * 6 + 4] = 0.1 * cos(ph3) / T3;
                J[0 * 6 + 3] = -d3 * sin(ph3) * (pi / 3.0) / T3;
                J[1 * 6 + 4] = 0.1 * sin(ph3) / T3;
                J[1 * 6 + 3] = d3 * cos(ph3) * (pi / 3.0) / T3;
            }
        } else {
            a[3] = drx4;
            a[1] = dz4;
            if (J && !unrounded) {
                J[3 * 6 + 1] = -(pi / 3.0) / T4;
                J[1 * 6 + 5] = 0.005 / T4;
            } else if (J) {
                /* d(-ph1 / Tf4), d(d4 / Tf4) */
                J[3 * 6 + 1] = -(pi / 3.0) / Tf4 + ph1 * dTf4_drot / (Tf4 * Tf4);
                J[3 * 6 + 5] = ph1 * dTf4_dlift / (Tf4 * Tf4);
                J[1 * 6 + 1] = -d4 * dTf4_drot / (Tf4 * Tf4);
                J[1 * 6 + 5] = 0.005 / Tf4 - d4 * dTf4_dlift / (Tf4 * Tf4);
            }
        }
    }
    return Ttot;
}

/* Move agent (Sec. III-A, actions): the displacement of each global step is
 * split evenly over its substeps and added to the pose; the shovel velocity
 * of a substep is that increment over dt. */
void orc_pose_table(const double start[4], int n_actions, const double* actions, int substeps_per_action,
                    double dt_sub, int nsub, double* poses) {
    double cur[4] = {start[0], start[1], start[2], start[3]};
    for (int s = 0; s < nsub; s++) {
        int t = s / substeps_per_action;
        double inc[4] = {0, 0, 0, 0};
        if (t < n_actions)
            for (int k = 0; k < 4; k++) inc[k] = actions[6 * t + k] / substeps_per_action;
        for (int k = 0; k < 4; k++) {
            cur[k] += inc[k];
            poses[8 * s + k] = cur[k];
            poses[8 * s + 4 + k] = inc[k] / dt_sub;
        }
    }
}

void orc_pose_table_adjoint(int n_actions, int substeps_per_action, double dt_sub, int nsub,
                            const double* gposes, double* gactions) {
    memset(gactions, 0, (size_t)n_actions * 6 * sizeof(double));
    double suffix[4] = {0, 0, 0, 0};
    for (int s = nsub - 1; s >= 0; s--) {
        for (int k = 0; k < 4; k++) suffix[k] += gposes[8 * s + k];
        int t = s / substeps_per_action;
        if (t >= n_actions) continue;
        for (int k = 0; k < 4; k++)
            gactions[6 * t + k] += (suffix[k] + gposes[8 * s + 4 + k] / dt_sub) / substeps_per_action;
    }
}

/* ---------------------------------------------------------------------
 * Surface observation, height map and HMD (Sec. III-A; Eq. (2))
 * ------------------------------------------------------------------- */

/* the pixel of an FP32 point (x, z) or -1 outside the square */
static int64_t obs_pixel(const orc_obs_grid* g, float xf, float zf) {
    const float x0 = (float)(g->cx - 0.5 * g->size), z0 = (float)(g->cz - 0.5 * g->size);
    const float h = (float)(g->size / g->res);
    const float fi = floorf((xf - x0) / h), fj = floorf((zf - z0) / h);
    if (!(fi >= 0.0f && fi < (float)g->res && fj >= 0.0f && fj < (float)g->res)) return -1;
    return (int64_t)fi * g->res + (int64_t)fj;
}

int orc_surface_observation(const orc_obs_grid* g, int64_t n, const float* x, int64_t* idx) {
    const int64_t np = (int64_t)g->res * g->res;
    for (int64_t p = 0; p < np; p++) idx[p] = -1;
    for (int64_t q = 0; q < n; q++) {
        const int64_t p = obs_pixel(g, x[3 * q], x[3 * q + 2]);
        if (p < 0) continue;
        /* strictly higher replaces: the lowest index keeps a tie */
        if (idx[p] < 0 || x[3 * q + 1] > x[3 * idx[p] + 1]) idx[p] = q;
    }
    int count = 0;
    for (int64_t p = 0; p < np; p++) count += idx[p] >= 0;
    return count;
}

void orc_height_map(const orc_obs_grid* g, int64_t n, const float* x, double* I, int64_t* winner) {
    const int64_t np = (int64_t)g->res * g->res;
    for (int64_t p = 0; p < np; p++) {
        I[p] = 0.0;
        winner[p] = -1;
    }
    const float r = (float)g->tap;
    for (int64_t q = 0; q < n; q++) {
        const float xf = x[3 * q], yf = x[3 * q + 1], zf = x[3 * q + 2];
        const float tx[5] = {xf, xf + r, xf - r, xf, xf};
        const float tz[5] = {zf, zf, zf, zf + r, zf - r};
        for (int t = 0; t < 5; t++) {
            const int64_t p = obs_pixel(g, tx[t], tz[t]);
            if (p < 0) continue;
            if ((double)yf > I[p]) {
                I[p] = (double)yf;
                winner[p] = q;
            }
        }
    }
}

double orc_hmd(const orc_obs_grid* g, int64_t n, const float* x, const double* Ihat, double* dL_dx) {
    const int64_t np = (int64_t)g->res * g->res;
    double* I = (double*)malloc((size_t)np * sizeof(double));
    int64_t* w = (int64_t*)malloc((size_t)np * sizeof(int64_t));
    orc_height_map(g, n, x, I, w);
    if (dL_dx) memset(dL_dx, 0, (size_t)n * 3 * sizeof(double));
    double L = 0.0;
    for (int64_t p = 0; p < np; p++) {
        const double d = I[p] - Ihat[p];
        L += fabs(d);
        if (dL_dx && w[p] >= 0) dL_dx[3 * w[p] + 1] += (d > 0.0) - (d < 0.0);
    }
    free(I);
    free(w);
    return L;
}
