/*
 * mpm.h -- C ABI of the GB300 (sm_103a) MLS-MPM sand/soil substep and its
 * reverse-mode adjoint, after DDBot (arXiv 2510.17335).
 *
 * What one substep computes (Sec. III-A, Algorithm 1; Eqs. (3)-(7)):
 *   per particle: trial F = (I + dt C) F; SVD; Drucker-Prager return of the
 *   singular values (Eqs. (6)-(7)); F' = U S^ V^T; Kirchhoff stress
 *   tau = P' F'^T of the SVK log-strain energy (Eqs. (3)-(4), det F' := 1);
 *   APIC/MLS-MPM scatter of mass and momentum with quadratic B-splines;
 *   per grid node: v = mv/m + dt g, slip walls, box-shovel SDF contact with
 *   Coulomb friction; per particle: APIC gather of v and C, the same shovel
 *   contact on the particle velocity, x += dt v.
 * The adjoint (Sec. III-D; Appendix B) is the exact reverse of that substep,
 * chained over a rollout with checkpointing, and yields dL/d{E, nu, rho,
 * phi} and dL/d(the six skill parameters) through the skill-to-action map
 * (Sec. III-B, Algorithm 2, rounded phase lengths).
 *
 * Conventions
 *   - y is up. Instance domains are [0, res_k * dx) per axis; node (i,j,k)
 *     sits at (i,j,k) * dx. A particle must stay in [dx, (res_k - 2) dx);
 *     leaving it is reported as MPM_ERR_OUT_OF_DOMAIN.
 *   - Particle arrays crossing this boundary are FP32, in "external order":
 *     the instances one after another, each in its own creation order, with
 *     no padding. Positions/velocities are 3 floats per particle, C and F 9
 *     floats per particle (row-major 3x3), interleaved per particle
 *     (x[3*p + k]).
 *   - A shovel pose is (tip x, y, z, tilt psi). The box spans local
 *     x in [-hx, hx], y in [0, 2 hy], z in [-hz, hz] above the tip, rotated
 *     by R(psi) = [[cos, sin, 0], [-sin, cos, 0], [0, 0, 1]] about the tip;
 *     psi tilts the pointing direction to (-sin psi, -cos psi, 0).
 *   - Actions are per global step, 6 doubles in the simulator frame
 *     [dx, dy, dz, dpsi, 0, 0]; each step's displacement is split evenly
 *     over its substeps (Sec. III-A, actions). Components 4 and 5 must be 0.
 *   - `device_ptrs` = 1 means the float pointers are CUDA device pointers
 *     (read/written on the handle's stream); 0 means host pointers (the call
 *     copies and synchronises).
 *   - Ownership: the library allocates and owns all of its device memory;
 *     inputs are copied in; outputs are written into caller buffers. A
 *     handle must not be used from two threads at once.
 *   - Errors: every int-returning call returns MPM_OK (0) or a negative
 *     code; no exception crosses the boundary. Device-side errors (domain,
 *     non-finite values) are collected in a status word and reported by the
 *     call that ran the kernels.
 */
#ifndef MPM_GB300_H
#define MPM_GB300_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPM_OK 0
#define MPM_ERR_INVALID_ARG (-1)  /* bad size, parameter out of range, NULL where required */
#define MPM_ERR_OOM (-2)          /* device allocation failed */
#define MPM_ERR_CUDA (-3)         /* a CUDA call failed */
#define MPM_ERR_OUT_OF_DOMAIN (-4)/* a particle left [dx, (res-2) dx) */
#define MPM_ERR_NON_FINITE (-5)   /* NaN/Inf in the state or an adjoint */
#define MPM_ERR_NO_RECORD (-6)    /* backward without a recorded forward */
#define MPM_ERR_TIMEOUT (-7)      /* a bounded device wait gave up */
#define MPM_ERR_NO_DEVICE (-8)    /* no usable sm_103 device */

typedef struct mpm_handle mpm_handle;

/* Material of one instance, Theta in Sec. III-A; E in Pa (the paper's table
 * prints a kPa header over Pa values), nu in (0, 0.5), rho in kg/m^3,
 * phi_deg (friction angle) in (0, 90). */
typedef struct {
    double E, nu, rho, phi_deg;
} mpm_material;

/* Grid and contact setup of one instance. */
typedef struct {
    int res[3];               /* grid nodes per axis, each in [8, 1024] */
    double dx;                /* node spacing (> 0) */
    double dt;                /* substep (> 0) */
    double gravity[3];        /* m/s^2 */
    int bound;                /* wall layer thickness in nodes (>= 0) */
    double particle_volume;   /* V_p; the particle mass is rho * V_p */
    double friction;          /* Coulomb coefficient of the shovel contact */
    int particle_collision;   /* 1: apply the shovel contact to particles too */
    double shovel_half[3];    /* box half extents (x thickness, y length, z width) */
    int shovel_on;            /* 0: no shovel */
} mpm_config;

/* Handle-wide options; pass NULL for the defaults in brackets. */
typedef struct {
    int checkpoint_every;     /* [50] substeps per checkpoint segment */
    int clip_grads;           /* [0] clip adjoints of x, v, F and of grid m, v, v' (Sec. III-E) */
    double clip_value;        /* [1e4] */
    double sigma_min;         /* [1e-4] singular values are clamped here before the log */
    int sort_every;           /* [0] reorder particles every n substeps (0: never): by grid block
                               * and, inside a 4x4x4-cell block, rank-major (the first particle of
                               * each occupied cell, then the second of each, ...), so that the
                               * lanes of a warp fall in different cells; mpm_autotune may set it */
    int tile_scatter;         /* [0] sum the 27-node scatters in shared-memory tiles per CTA
                               * (measured slower than the direct L2 reductions on GB300) */
    int cuda_graphs;          /* [1] replay repeated identical mpm_forward / mpm_backward calls
                               * from CUDA graphs (see below) */
    int grad_scale;           /* [0] regularise the adjoints of the particles' x, v, F and of the
                               * grid's velocities (after, before the contact) and mass, each as
                               * one vector per substep and instance (Sec. III-E): 1 dynamic
                               * scaling, g /= 10^doom + delta, doom = round(log10 max|g|) -
                               * oom_star when positive; 2 normalisation, g /= ||g|| + delta.
                               * Not together with clip_grads. */
    double oom_star;          /* [4] */
    double grad_delta;        /* [1e-6] */
    int fuse_adjoint;         /* [1] run the P2G adjoint of a substep and the G2P adjoint of the one
                               * before it in one pass over the particles where both lie in the same
                               * recorded segment (not with grad_scale or tile_scatter) */
} mpm_options;

/* Digging skill (Sec. III-B): theta = (displace, rotate, insert_dist,
 * push_angle, push_dist, lift) in [-1, 1]; lift sets d4 = (lift + 1) 0.005 m
 * (lift = 1 is the paper's 0.01 m). The global step is
 * substeps_per_action * dt. */
typedef struct {
    double theta[6];
    double v_lin, v_ang;      /* end-effector speeds (m/s, rad/s), > 0 */
    int substeps_per_action;  /* N >= 1 */
    double start_pose[4];     /* tip x, y, z, psi */
    int unrounded_T;          /* 1: phases 1 and 4 divide their displacements by the real-valued
                               * step counts (the alternative mapping of Sec. III-B, gradients
                               * of Appendix A); 0: by the rounded ones (Algorithm 2) */
} mpm_skill;

typedef struct {
    int n_inst;
    int64_t n_particles;      /* total over instances */
    int64_t substep;          /* substeps run since create/reset */
    int64_t recorded;         /* substeps recorded for backward (0 if none) */
    int64_t device_bytes;     /* device memory held */
    int64_t kernel_launches;  /* kernels launched by the library so far */
    int64_t fp64_fallbacks;   /* constitutive evaluations redone in FP64 */
    int64_t graph_launches;   /* forward / backward calls replayed from CUDA graphs */
} mpm_info_t;

/* Create a batch of n_inst independent instances. cfgs/mats have n_inst
 * entries; counts[i] particles of instance i (>= 0); x0 holds the initial
 * positions in external order (host pointer, sum(counts) * 3 floats). The
 * initial state is v = 0, C = 0, F = I. Runs on the current CUDA device. */
int mpm_create(int n_inst, const mpm_config* cfgs, const mpm_material* mats, const int64_t* counts,
               const float* x0, const mpm_options* opts, mpm_handle** out);

/* Replace the material of one instance (takes effect at the next call). */
int mpm_set_material(mpm_handle* h, int inst, const mpm_material* mat);

/* Scripted shovel motion: start pose and n_actions actions (host,
 * n_actions * 6 doubles). After the last action the shovel rests. */
int mpm_set_shovel_actions(mpm_handle* h, int inst, const double start_pose[4], int n_actions,
                           const double* actions, int substeps_per_action);

/* Skill-driven shovel motion: Algorithm 2 maps theta to actions; backward
 * then also returns dL/dtheta through the Jacobian with frozen T_i. */
int mpm_set_shovel_trajectory(mpm_handle* h, int inst, const mpm_skill* skill);

/* Number of actions of an instance's current trajectory (>= 0), or < 0. */
int mpm_num_actions(mpm_handle* h, int inst);

/* Back to the creation state (x0, v = 0, C = 0, F = I), substep 0, no record. */
int mpm_reset(mpm_handle* h);

/* Overwrite the current state (all instances, external order). NULL v/C/F
 * mean 0, 0 and I. Drops any record. */
int mpm_set_state(mpm_handle* h, const float* x, const float* v, const float* C, const float* F,
                  int device_ptrs);

/* Read the current state (any output may be NULL). */
int mpm_get_state(mpm_handle* h, float* x, float* v, float* C, float* F, int device_ptrs);

/* Advance all instances by n_substeps (>= 0). record = 1 keeps what the
 * backward needs: one state checkpoint every checkpoint_every substeps, and
 * every state and grid of the current segment (the backward reverses the
 * last segment directly and recomputes the earlier ones from their
 * checkpoints). A recording forward continues an existing record only if
 * the previous call recorded too. */
int mpm_forward(mpm_handle* h, int n_substeps, int record);

/* Surface observation and height map (Sec. III-A, "States and
 * observations"; Eq. (2)). Per instance a res x res square of pixels of
 * side `size` in the horizontal (x, z) plane (y is up) centred at center;
 * pixel (i, j) of a point is i = floorf((x - x0) / h), j = floorf((z - z0) /
 * h) in FP32 with IEEE division, x0 = (float)(center[0] - size/2),
 * z0 = (float)(center[1] - size/2), h = (float)(size/res); points outside the
 * square are ignored; pixel index i * res + j. All instances use the same res
 * (1..4096). The paper's observation is a 40 x 40 square of 0.24 m. */
typedef struct {
    double center[2];         /* (x, z) of the square's centre, m */
    double size;              /* side, m (> 0) */
    int res;                  /* pixels per side */
    double tap;               /* height-map splat offset r_p, m (>= 0) */
} mpm_obs_grid;

/* The observation: per pixel the highest particle of the current state
 * (largest y; equal heights: the lowest particle index of the instance).
 * points: n_inst * res^2 * 3 floats, the winners' positions, NaN where a
 * pixel is empty (may be NULL). counts: n_inst non-empty pixel counts (host,
 * may be NULL). grids: n_inst entries. */
int mpm_surface_observation(mpm_handle* h, const mpm_obs_grid* grids, float* points, int* counts, int device_ptrs);

/* The height map: every particle covers the pixels of (x, z), (x +- tap, z)
 * and (x, z +- tap) (FP32 sums); a pixel starts at 0 and holds the largest y
 * above 0 of the particles that cover it. maps: n_inst * res^2 floats. */
int mpm_height_map(mpm_handle* h, const mpm_obs_grid* grids, float* maps, int device_ptrs);

/* The height-map distance of Eq. (2) per instance, loss[i] = sum_pixels
 * |I - Ihat| (FP64, host), against target_maps (n_inst * res^2 floats), and,
 * if dL_dx != NULL, its gradient w.r.t. the positions (n_particles * 3,
 * external order): at each pixel the particle whose height it holds gets
 * sign(I - Ihat) in y; x and z get 0 (the map is piecewise constant in
 * them). Equal heights: the lowest particle index holds the pixel. */
int mpm_loss_hmd(mpm_handle* h, const mpm_obs_grid* grids, const float* target_maps, double* loss, float* dL_dx,
                 int device_ptrs);

/* The unnormalised Earth Mover's distance of Eq. (1) per instance between
 * the observation of mpm_surface_observation (grids; its non-empty pixels)
 * and a target cloud: loss[i] = min over one-to-one maps phi of
 * sum |x - phi(x)| (FP64, host). targets: n_inst * res^2 * 3 floats, the
 * first n_targets[i] rows (host ints) of instance i are its points; the map
 * needs n_targets[i] >= the observed points (else MPM_ERR_INVALID_ARG).
 * Found by an auction with epsilon scaling (Bertsekas); the result is within
 * (observed points) * 1e-6 * size of the optimum. dL_dx (may be NULL):
 * n_particles * 3, (x - phi(x)) / |x - phi(x)| on each observed particle,
 * 0 elsewhere. MPM_ERR_TIMEOUT if the auction does not finish within its
 * round limit. */
int mpm_loss_emd(mpm_handle* h, const mpm_obs_grid* grids, const float* targets, const int* n_targets,
                 double* loss, float* dL_dx, int device_ptrs);

/* The line search of Sec. III-F, batched: instances 0..n_cand-1 of h are the
 * candidates (the caller has set their start state); each gets mats[k]
 * and/or skills[k] (either may be NULL), all advance n_substeps in one
 * forward, and the candidate with the least height-map distance to its
 * target map wins (ties: the lowest k). losses: n_cand doubles (may be
 * NULL); *best: the winner. Instances past n_cand advance too. */
int mpm_line_search(mpm_handle* h, int n_cand, const mpm_material* mats, const mpm_skill* skills, int n_substeps,
                    const mpm_obs_grid* grids, const float* target_maps, int device_ptrs, double* losses,
                    int* best);

/* CUDA graphs (option cuda_graphs, on by default). An optimisation loop runs
 * the same rollout again and again: set the state (and material or skill),
 * mpm_forward(n, 1), a loss, mpm_backward. Such a call issues exactly the
 * launches of the previous identical call: same n, record flag, substep and
 * record position, and the same segment bookkeeping. The second time a call
 * is seen the library captures its launches into a CUDA graph; from the
 * third time on it replays that graph with one cudaGraphLaunch. Material,
 * skill, state and loss seeds live in device buffers the graph reads, so
 * they may change between replays. Replay gives results identical to eager
 * launches. No graph is used while profiling or sorting, and a capture
 * that fails (for example because it would allocate) falls back to eager
 * launches. Up to 16 graphs are kept per handle. */

/* L_i = (1/N_i) sum_p |x_p - xhat_p|^2 per instance (FP64 accumulation) and,
 * if dL_dx != NULL, dL/dx = 2 (x - xhat) / N_i (external order). */
int mpm_loss_mse(mpm_handle* h, const float* x_target, double* loss, float* dL_dx, int device_ptrs);

/* Reverse the recorded rollout. dL_dx / dL_dv: adjoints of the final
 * positions / velocities (external order; either may be NULL = 0).
 * dL_dmaterial: n_inst * 4 doubles (E, nu, rho, phi_deg). dL_dtheta:
 * n_inst * 6 doubles (zero for scripted trajectories), may be NULL.
 * The record is consumed. */
int mpm_backward(mpm_handle* h, const float* dL_dx, const float* dL_dv, int device_ptrs,
                 double* dL_dmaterial, double* dL_dtheta);

/* After mpm_backward: dL/d(initial state of the recorded rollout). */
int mpm_get_state_grad(mpm_handle* h, float* gx, float* gv, float* gC, float* gF, int device_ptrs);

/* After mpm_backward: dL/d(actions) of one instance (n_actions * 6 doubles)
 * and dL/d(start pose) (4 doubles, may be NULL). */
int mpm_get_action_grad(mpm_handle* h, int inst, double* dL_dactions, double* dL_dstart);

/* Diagnostic: total grid mass per instance (n_inst doubles) after the last
 * forward substep's P2G (summed in FP64 by its grid update; a backward's
 * recomputation of substeps leaves it alone); by the partition of unity of
 * the B-spline weights (Sec. III-A, MLS-MPM transfer) it equals
 * sum_p rho V_p up to rounding. */
int mpm_grid_mass(mpm_handle* h, double* mass);

/* Device memory of a recorded forward, for choosing checkpoint_every: one
 * state slot (x, v, C, F of every particle) and, per recorded substep, the
 * substep slot (the SVD record of the trial F per particle, the grid
 * accumulators, velocities and touched-block flags per node), for
 * n_particles particles on n_nodes grid nodes (all instances; nodes counted
 * in 4x4x4 blocks). A segment of K substeps holds K + 1 state slots and K
 * substep slots. Host only; no handle or device needed. */
int mpm_record_bytes(int64_t n_particles, int64_t n_nodes, int64_t* state_slot, int64_t* substep_slot);

/* Launch shape of the particle kernels: the register cap each is compiled
 * for, as the minimum number of resident CTAs per SM, shape[0] k_p2g (3 or
 * 4), shape[1] k_g2p (3 or 4), shape[2] the fused adjoint k_p2g_g2p_bwd (2,
 * 3 or 4); defaults 4, 4, 3 (the fastest of measured sweeps on the
 * 1M-particle bed). Other values: MPM_ERR_INVALID_ARG. A change drops the
 * handle's CUDA graphs. */
int mpm_set_launch_shape(mpm_handle* h, const int shape[3]);
int mpm_get_launch_shape(mpm_handle* h, int shape[3]);

/* Autotuner: from the current state, times a recorded forward of
 * trial_substeps plus its backward for each candidate and keeps the fastest:
 * first the register caps of mpm_set_launch_shape (every kernel's
 * candidates in the same trials, each kernel timed per launch with CUDA
 * events, each keeping its fastest cap), then, with those caps, no sort
 * against a sort by cell once per checkpoint segment (sort_every). Writes
 * chosen[0] = tile_scatter (not tuned), chosen[1] = sort_every (may be
 * NULL); mpm_get_launch_shape gives the caps. The choice is cached for the
 * process per device and workload (instance count, particle counts, grids):
 * a later call for the same workload with trial_substeps no larger than the
 * cached trial applies it without timing. The state, its particle order,
 * the substep counter and the options not tuned are restored on every
 * return, errors included; any record is dropped and the kernel-timing
 * counters are reset. */
int mpm_autotune(mpm_handle* h, int trial_substeps, int* chosen);

/* Set the substep counter (the index into the shovel pose tables) of the
 * next forward substep; drops any record. */
int mpm_set_substep(mpm_handle* h, int64_t substep);

/* Kernel timing: enable != 0 records a CUDA event pair around every kernel
 * launch on the handle's stream (counters reset on every call). Kernel ids:
 * 0 k_p2g, 1 k_grid, 2 k_g2p, 3 k_g2p_bwd, 4 k_grid_bwd, 5 k_p2g_bwd,
 * 6 k_grid_clear, 7 k_slot_clear, 8 k_p2g_fp64, 9 k_p2g_bwd_fp64,
 * 10 k_p2g_g2p_bwd, 11 k_p2g_g2p_bwd_fp64 (ids below MPM_PROFILE_KERNELS).
 * The _fp64 kernels redo, in FP64, the particles whose deformation gradient
 * is too ill-conditioned for the FP32 SVD; they launch every substep and
 * return at once when there are none. k_p2g_g2p_bwd is the fused adjoint
 * (option fuse_adjoint).
 * mpm_profile_read waits for the recorded events and gives the summed device
 * time (ms) and the launch count of one kernel. */
#define MPM_PROFILE_KERNELS 12
int mpm_profile(mpm_handle* h, int enable);
int mpm_profile_read(mpm_handle* h, int kernel, double* total_ms, int64_t* launches);
const char* mpm_kernel_name(int kernel);

/* The MSE loss of mpm_loss_mse for one point set given as plain device
 * arrays, for callers that cannot allocate device memory. (The paper has no
 * counterpart of this entry point.)
 *
 * Who needs it: a caller whose device memory is all owned by another
 * allocator (for example a framework's caching allocator that reserved the
 * GPU up front), or a control loop that must not take the implicit device
 * synchronisation of cudaMalloc. The call allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine. Its scratch is a file-scope device
 * array of 128 KiB (plus a result and a counter) that every GPU which loads
 * this library holds until the process exits.
 *
 * x, x_target: device pointers, n points of 3 floats (x[3*p + k]);
 * dL_dx: device pointer for 2 (x - xhat) / n, or NULL; loss: host pointer,
 * receives (1/n) sum_p |x_p - xhat_p|^2 accumulated in FP64. stream: a
 * cudaStream_t (NULL = legacy default); the call waits for it before it
 * returns. n must be in [0, MPM_NOALLOC_MAX_POINTS]; a larger n is rejected
 * with MPM_ERR_INVALID_ARG before anything runs.
 *
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for that
 * device's CUDA context; make that first call before any stream capture.
 * After a device reset (cudaDeviceReset) the next call finds a new context
 * and looks the address up again, so that call too should come before any
 * capture. All calls share the one scratch array, which
 * keeps the last call's contents (the call clears the part that must start
 * at zero), so calls that overlap on the GPU race with each other: issue
 * them on one stream or one after another. */
#define MPM_NOALLOC_MAX_POINTS 4194304
int mpm_loss_mse_noalloc(const float* x, const float* x_target, int64_t n, float* dL_dx, double* loss,
                         void* stream);

/* Run on this CUDA stream (a cudaStream_t; NULL = the legacy default). */
int mpm_set_stream(mpm_handle* h, void* stream);

int mpm_synchronize(mpm_handle* h);
int mpm_get_info(mpm_handle* h, mpm_info_t* out);
void mpm_destroy(mpm_handle* h);
const char* mpm_error_string(int code);
int mpm_version(void);

#ifdef __cplusplus
}
#endif
#endif
