/*
 * FP64 CPU oracle for the 3D MLS-MPM sand/soil substep of DDBot
 * (arXiv 2510.17335) and its hand-written reverse-mode adjoint.
 *
 * TEST INFRASTRUCTURE ONLY. This library exists to check the GPU path.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it. It shares no code, header, table or helper with the CUDA library.
 *
 * Conventions (the same readings the GPU library documents in its header):
 *   - y is up; the domain is [0, res_k*dx) per axis; node (i,j,k) sits at
 *     (i,j,k)*dx; grid arrays are dense, index ((i*res1)+j)*res2+k.
 *   - particle state is x[3], v[3], C[9], F[9] per particle, 3x3 matrices
 *     row-major.
 *   - a shovel pose is 8 doubles: tip position c[3], tilt psi, tip velocity
 *     cdot[3], tilt rate psidot. The box spans local x in [-hx,hx],
 *     y in [0, 2hy], z in [-hz,hz] above the tip; local-to-world is
 *     R(psi) = [[cos, sin, 0], [-sin, cos, 0], [0, 0, 1]].
 *   - return codes: 0 ok, -1 invalid argument, -4 a particle left the
 *     valid domain [dx, (res-2)dx).
 */
#ifndef MPM_ORACLE_H
#define MPM_ORACLE_H
#include <stdint.h>

typedef struct {
    int res[3];
    double dx, dt;
    double gravity[3];
    int bound;                 /* wall thickness in nodes */
    double E, nu, rho, phi_deg;/* material, Sec. III-A */
    double vol;                /* particle volume V_p */
    double friction;           /* Coulomb coefficient of the shovel contact */
    int particle_collision;    /* apply the shovel contact to particles too */
    double sigma_min;          /* singular values are clamped here before ln */
    double shovel_half[3];     /* box half extents (x thickness, y length, z width) */
    int shovel_on;             /* 0: no shovel */
    int clip_grads;            /* clip adjoints of key variables (Sec. III-E) */
    double clip_value;
    int grad_scale;            /* 0 none, 1 dynamic scaling, 2 normalisation of the same
                                * adjoint vectors (Sec. III-E); not with clip_grads */
    double oom_star;           /* maximal order of magnitude (dynamic scaling) */
    double grad_delta;         /* the small constant delta of both operations */
} orc_params;

/* The gradient regularisers of Sec. III-E on one adjoint vector g[n]:
 * grad_scale 1: g /= 10^doom + delta with doom = round(log10 max|g_i|) -
 * oom_star, only when doom > 0; 2: g /= ||g||_2 + delta. clip_grads clips
 * each entry to [-clip_value, clip_value] instead. */
void orc_grad_op(const orc_params* p, double* g, int64_t n);

/* Threads of the particle and node loops (default 1: the plain loops, one
 * particle or node at a time in index order). With n > 1 (OpenMP) scatters
 * go into per-thread grids over the box of the particles' stencils, added
 * node by node in thread order, and parameter sums are per-thread partials
 * added in thread order: the same arithmetic up to the order of the sums. */
void orc_set_threads(int n);
int orc_get_threads(void);

/* 3x3 SVD with proper rotations U, V (det +1) and S sorted by magnitude,
 * S[2] carrying the sign of det(F). */
void orc_svd3(const double F[9], double U[9], double S[3], double V[9]);

/* Lame constants and the Drucker-Prager friction coefficient alpha_f. */
void orc_material(double E, double nu, double phi_deg, double* mu, double* lam, double* alpha);

/* The constitutive step: trial F -> projected F' and Kirchhoff stress.
 * info (optional, 4 doubles): case (0 tension/apex, 1 elastic, 2 cone
 * projection), tr(eps), delta_gamma, ||eps_hat||. */
void orc_constitutive(const double Ft[9], double mu, double lam, double alpha, double sigma_min,
                      double Fn[9], double tau[9], double info[4]);

/* Reverse of orc_constitutive: given adjoints of F' and tau, returns the
 * adjoint of the trial F and adds to the adjoints of mu, lambda, alpha. */
void orc_constitutive_adjoint(const double Ft[9], double mu, double lam, double alpha, double sigma_min,
                              const double gFn[9], const double gtau[9],
                              double gFt[9], double* gmu, double* glam, double* galpha);

/* Shovel SDF contact with Coulomb friction applied to one velocity. */
void orc_shovel_project(const orc_params* p, const double vel[3], const double q[3],
                        const double pose[8], double out[3]);

/* One substep in place. */
int orc_substep(const orc_params* p, int64_t n, double* x, double* v, double* C, double* F,
                const double pose[8]);

/* nsub substeps in place; poses holds nsub*8 doubles. */
int orc_rollout(const orc_params* p, int64_t n, double* x, double* v, double* C, double* F,
                int nsub, const double* poses);

/* Grid after P2G + grid update of one substep from a given state (for the
 * invariant tests): m[G], mv[3G] (P2G momentum), vout[3G] (after walls and
 * shovel). Any output pointer may be NULL. */
int orc_grid_of_substep(const orc_params* p, int64_t n, const double* x, const double* v,
                        const double* C, const double* F, const double pose[8],
                        double* m, double* mv, double* vout);

/* Reverse-mode adjoint of an nsub-substep rollout. Inputs: initial state and
 * the adjoints of the final state (gx, gv, gC, gF; any may be NULL = zero).
 * Outputs: adjoints of the initial state (any may be NULL), the material
 * gradient gmat = dL/d{E, nu, rho, phi_deg}, and gposes[nsub*8] =
 * dL/d(pose of each substep). */
int orc_rollout_adjoint(const orc_params* p, int64_t n, const double* x0, const double* v0,
                        const double* C0, const double* F0, int nsub, const double* poses,
                        const double* gx, const double* gv, const double* gC, const double* gF,
                        double* ax0, double* av0, double* aC0, double* aF0,
                        double gmat[4], double* gposes);

/* Algorithm 2 (skill-to-action mapping), rounded phase lengths by default.
 * theta = (displace, rotate, insert_dist, push_angle, push_dist, lift).
 * dt_step is the global step. Writes up to max_actions actions of 6 doubles
 * in the simulator frame [dx, dy(up), dz, dpsi, 0, 0], the phase lengths
 * T[4], and (if jac != NULL) jac[t*36 + k*6 + j] = d a_t[k] / d theta_j.
 * unrounded = 1: phases 1 and 4 divide their displacements by the
 * real-valued step counts T1f, T4f instead of T1, T4 (the alternative
 * mapping of Sec. III-B, whose gradients Appendix A prints).
 * Returns the number of actions T, or -1 if max_actions is too small. */
int orc_skill_actions(const double theta[6], double v_lin, double v_ang, double dt_step,
                      int max_actions, int unrounded, double* actions, int T[4], double* jac);

/* Per-substep pose table from a start pose (tip[3], psi) and an action list. */
void orc_pose_table(const double start[4], int n_actions, const double* actions, int substeps_per_action,
                    double dt_sub, int nsub, double* poses);

/* Chain rule through orc_pose_table: dL/d(action) from dL/d(pose table). */
void orc_pose_table_adjoint(int n_actions, int substeps_per_action, double dt_sub, int nsub,
                            const double* gposes, double* gactions);

/* ---------------------------------------------------------------------
 * Surface observation and height-map distance (Sec. III-A, "States and
 * observations" and Eq. (2) of "Goal and reward/loss").
 *
 * A res x res square of pixels of side `size` lies in the horizontal (x, z)
 * plane (y is up), centred at (cx, cz). Pixel (i, j) of a point holds
 *   i = floorf((xf - x0f) / hf),  j = floorf((zf - z0f) / hf)
 * in FP32 arithmetic, with x0f = (float)(cx - size/2), z0f = (float)(cz -
 * size/2), hf = (float)(size/res); points outside [0, res)^2 are skipped.
 * Pixel p = i * res + j. Particle positions are FP32 (the simulator's
 * state); every selection compares FP32 heights, so the GPU can be checked
 * index for index.
 * ------------------------------------------------------------------- */
typedef struct {
    double cx, cz;      /* centre of the square (x, z) */
    double size;        /* side (0.24 m in the paper) */
    int res;            /* pixels per side (40) */
    double tap;         /* height-map splat offset r_p (m) */
} orc_obs_grid;

/* Surface observation: per pixel the highest particle (largest y; equal
 * heights: the lowest particle index). idx[p] = that particle or -1.
 * Returns the number of non-empty pixels. */
int orc_surface_observation(const orc_obs_grid* g, int64_t n, const float* x, int64_t* idx);

/* Height map: each particle covers the pixels of (x, z), (x + r, z),
 * (x - r, z), (x, z + r), (x, z - r), r = (float)tap, FP32 sums. I starts at
 * zero and a pixel takes a covering particle's y when it is higher than the
 * current value, particles in index order (so equal heights keep the lowest
 * index). winner[p] = the particle whose y the pixel holds, or -1. */
void orc_height_map(const orc_obs_grid* g, int64_t n, const float* x, double* I, int64_t* winner);

/* d_HMD = sum_p |I_p - Ihat_p| and, if dL_dx != NULL, its gradient w.r.t.
 * the particle positions: dL/dy of a particle = the sum of sign(I_p - Ihat_p)
 * over the pixels it wins (0 for x and z, and sign(0) = 0). */
double orc_hmd(const orc_obs_grid* g, int64_t n, const float* x, const double* Ihat, double* dL_dx);

#endif
