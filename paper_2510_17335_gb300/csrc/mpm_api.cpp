// C ABI of the GB300 MLS-MPM sand substep library (see include/mpm.h).
//
// Host side: handle and device memory, the skill-to-action mapping of
// DDBot's Algorithm 2 (Sec. III-B) with its Jacobian, the per-substep shovel
// pose tables (Sec. III-A, actions), the checkpointed rollout driver and the
// chain from per-substep adjoints to dL/d{E, nu, rho, phi} and dL/dtheta.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/mpm.h"
#include "mpm_launch.h"
#include "mpm_reg.h"
#include "mpm_types.h"

using namespace mpm;

namespace {

constexpr double kPi = 3.14159265358979323846;

// touched-block set of one substep (the layout StepArgs::flags describes):
// n_blocks flags, list length, n_blocks list entries; the flags and the
// length start at zero, the list needs no initial value
size_t flag_ints(int n_blocks) { return 2 * (size_t)n_blocks + 1; }
size_t flag_bytes_zeroed(int n_blocks) { return ((size_t)n_blocks + 1) * sizeof(int); }

struct Instance {
    mpm_config cfg;
    mpm_material mat;
    int64_t n = 0;
    int64_t ext_off = 0;
    long long pbeg = 0;
    int n_chunks = 0;
    int nb[3] = {0, 0, 0};
    long long node_off = 0;
    int blk_off = 0;
    int n_blocks = 0;
    // trajectory
    bool has_traj = false;
    bool has_skill = false;
    mpm_skill skill;
    double start[4] = {0, 0, 0, 0};
    int spa = 1;                      // substeps per action
    std::vector<double> actions;      // n_actions * 6
    std::vector<double> jac;          // n_actions * 36 (skill only)
    long long pose_off = 0;           // offset (floats) into the pose buffer
    int n_poses = 0;
    // results of the last backward
    std::vector<double> gactions;
    double gstart[4] = {0, 0, 0, 0};
};

template <typename T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    int ensure(size_t count, int64_t& total) {
        if (count <= n) return MPM_OK;
        release();
        if (count == 0) return MPM_OK;
        if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return MPM_ERR_OOM;
        }
        total += (int64_t)((count - n) * sizeof(T));
        n = count;
        return MPM_OK;
    }
};

// CUDA-event timing of every kernel launch (on the launching stream),
// switched on by mpm_profile()
struct Profiler {
    bool on = false;
    struct Pending {
        int id;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    double total_ms[(int)KernelId::Count] = {0};
    int64_t count[(int)KernelId::Count] = {0};
    cudaEvent_t get() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void flush() {
        for (auto& p : pending) {
            cudaEventSynchronize(p.b);
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                total_ms[p.id] += ms;
                count[p.id] += 1;
            }
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
        cudaGetLastError();
    }
    void reset() {
        flush();
        for (int i = 0; i < (int)KernelId::Count; i++) {
            total_ms[i] = 0.0;
            count[i] = 0;
        }
    }
    void release() {
        flush();
        for (auto e : pool) cudaEventDestroy(e);
        pool.clear();
    }
};

}  // namespace

struct mpm_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    mpm_options opt;
    std::vector<Instance> inst;
    int64_t n_ext = 0;
    long long ncap = 0;
    int n_chunks = 0;
    int n_blocks = 0;
    long long n_nodes = 0;
    int64_t device_bytes = 0;
    int64_t launches = 0;

    DevBuf<InstDev> d_inst;
    DevBuf<int> d_chunk_inst, d_block_inst, d_ext_of_slot;
    DevBuf<float> d_state, d_x0, d_stage, d_poses, d_target;
    DevBuf<float4> d_acc, d_vout;
    DevBuf<int> d_flags;            // touched-block flags, list length, list (flag_ints)
    DevBuf<double> d_mass;          // grid mass per instance: running sums, last update's totals
    DevBuf<int> d_status;
    DevBuf<unsigned long long> d_fp64;
    DevBuf<int> d_fb_list, d_fb_count;   // particles deferred to the FP64 kernels
    DevBuf<double> d_loss;
    // surface observation / height map
    DevBuf<ObsDev> d_obs;
    DevBuf<unsigned long long> d_keys;
    DevBuf<float> d_obs_out, d_obs_target;
    DevBuf<double> d_obs_loss;
    DevBuf<int> d_obs_count;
    // Earth Mover's distance (auction)
    DevBuf<float> d_emd_price;
    DevBuf<int> d_emd_owner, d_emd_assign, d_emd_ntg, d_emd_cnt;
    DevBuf<unsigned long long> d_emd_bids;

    // record / backward
    int64_t substep = 0;
    bool recording = false;
    int64_t rec_start = 0, rec_len = 0;
    std::vector<DevBuf<float>> ckpt;
    // segment slots: state k of the segment in seg_state[k] (k = 0..K), the
    // grids of substep k in seg_acc/seg_vout/seg_flags[k] (k = 0..K-1)
    std::vector<DevBuf<float>> seg_state;
    std::vector<DevBuf<float4>> seg_acc, seg_vout;
    std::vector<DevBuf<int>> seg_flags;
    std::vector<DevBuf<float>> seg_spec;   // SVD of the trial F of substep k (k = 0..K-1)
    std::vector<char> seg_dirty;      // grid slot k holds accumulators/flags to clear
    int64_t seg_valid = -1;           // segment whose states/grids the slots hold
    int seg_valid_len = 0;
    DevBuf<float4> d_gacc, d_gacc2;   // grid adjoint; the second for the fused adjoint
    bool gacc_dirty = true;
    DevBuf<float> d_adj;
    DevBuf<double> d_gmat, d_gpose;
    DevBuf<double> d_pstat, d_gstat, d_gpose_raw;   // Sec. III-E regulariser statistics
    bool have_grad = false;
    int tile_scatter = 1;
    // particle sort by grid block
    DevBuf<float> d_state2, d_adj2;
    DevBuf<int> d_ext2, d_key, d_rank, d_bcount, d_bscan, d_part, d_remap, d_perm, d_ext_rec;
    std::vector<DevBuf<int>> seg_perm;
    std::vector<char> seg_sorted;
    int64_t since_sort = 1LL << 40;
    Profiler prof;
    LaunchShape shape;                // register caps of the particle kernels
    // CUDA graphs of repeated identical forward / backward calls
    std::vector<struct GraphEntry*> graphs;
    int64_t graph_tick = 0;
    int64_t graph_launches = 0;
};

// The host bookkeeping a forward or backward call reads and changes: two
// calls that start from equal snapshots (with the same arguments) issue the
// same launches and end in equal snapshots.
struct HostSnap {
    int64_t substep = 0, rec_start = 0, rec_len = 0, seg_valid = -1, since_sort = 0;
    int seg_valid_len = 0, tile = 0;
    bool recording = false, gacc_dirty = false;
    std::vector<char> seg_dirty, seg_sorted;
    // equal as far as the launches go: flags compare as if padded with
    // zeros, and the record position does not matter while not recording
    // (a recording forward starts a new record then)
    static bool same_flags(const std::vector<char>& a, const std::vector<char>& b) {
        const size_t n = std::max(a.size(), b.size());
        for (size_t i = 0; i < n; i++)
            if ((i < a.size() ? a[i] : 0) != (i < b.size() ? b[i] : 0)) return false;
        return true;
    }
    bool operator==(const HostSnap& o) const {
        if (recording != o.recording) return false;
        if (recording && (rec_start != o.rec_start || rec_len != o.rec_len)) return false;
        return substep == o.substep && seg_valid == o.seg_valid && since_sort == o.since_sort &&
               seg_valid_len == o.seg_valid_len && tile == o.tile && gacc_dirty == o.gacc_dirty &&
               same_flags(seg_dirty, o.seg_dirty) && same_flags(seg_sorted, o.seg_sorted);
    }
};

namespace {
void drop_graphs(mpm_handle* h);
}

struct GraphEntry {
    int kind = 0;            // 0 forward, 1 backward
    int64_t n = 0;           // substeps (forward)
    int flags = 0;           // record (forward) / seeds present (backward)
    HostSnap start, end;
    int64_t launches = 0;    // kernels in the graph
    int64_t used = 0;        // last use (eviction)
    bool capturable = true;
    int64_t alloc_bytes = 0; // device memory held at capture: any reallocation since voids the graph
    cudaGraphExec_t exec = nullptr;
};

namespace {

int cuda_err(cudaError_t e) {
    if (e == cudaSuccess) return MPM_OK;
    if (e == cudaErrorMemoryAllocation) return MPM_ERR_OOM;
    return MPM_ERR_CUDA;
}

#define CK(x)                                 \
    do {                                      \
        cudaError_t e__ = (x);                \
        if (e__ != cudaSuccess) {             \
            cudaGetLastError();               \
            return cuda_err(e__);             \
        }                                     \
    } while (0)

#define RK(x)                          \
    do {                               \
        int r__ = (x);                 \
        if (r__ != MPM_OK) return r__; \
    } while (0)

bool finite_pos(double x) { return std::isfinite(x) && x > 0; }

int validate_config(const mpm_config& c) {
    for (int k = 0; k < 3; k++)
        if (c.res[k] < 8 || c.res[k] > 1024) return MPM_ERR_INVALID_ARG;
    if (!finite_pos(c.dx) || !finite_pos(c.dt) || !finite_pos(c.particle_volume)) return MPM_ERR_INVALID_ARG;
    if (c.bound < 0 || c.bound > 16) return MPM_ERR_INVALID_ARG;
    if (!std::isfinite(c.friction) || c.friction < 0) return MPM_ERR_INVALID_ARG;
    for (int k = 0; k < 3; k++) {
        if (!std::isfinite(c.gravity[k])) return MPM_ERR_INVALID_ARG;
        if (c.shovel_on && !finite_pos(c.shovel_half[k])) return MPM_ERR_INVALID_ARG;
    }
    return MPM_OK;
}

int validate_material(const mpm_material& m) {
    if (!finite_pos(m.E) || !finite_pos(m.rho)) return MPM_ERR_INVALID_ARG;
    if (!(m.nu > 0 && m.nu < 0.5)) return MPM_ERR_INVALID_ARG;
    if (!(m.phi_deg > 0 && m.phi_deg < 90)) return MPM_ERR_INVALID_ARG;
    return MPM_OK;
}

// Lame constants (Sec. III-A, Eq. (5)) and the Drucker-Prager coefficient
// alpha_f (Eq. (6)); beta = (3 lambda + 2 mu) / (2 mu) alpha_f.
struct Lame {
    double mu, lam, alpha, beta;
};
Lame lame_of(const mpm_material& m) {
    Lame L;
    L.mu = m.E / (2.0 * (1.0 + m.nu));
    L.lam = m.E * m.nu / ((1.0 + m.nu) * (1.0 - 2.0 * m.nu));
    const double s = std::sin(m.phi_deg * kPi / 180.0);
    L.alpha = std::sqrt(2.0 / 3.0) * 2.0 * s / (3.0 - s);
    L.beta = (3.0 * L.lam + 2.0 * L.mu) / (2.0 * L.mu) * L.alpha;
    return L;
}

InstDev make_instdev(const mpm_handle* h, const Instance& I) {
    InstDev d;
    std::memset(&d, 0, sizeof d);
    for (int k = 0; k < 3; k++) {
        d.res[k] = I.cfg.res[k];
        d.nb[k] = I.nb[k];
        d.g[k] = (float)I.cfg.gravity[k];
        d.sh[k] = (float)I.cfg.shovel_half[k];
    }
    d.bound = I.cfg.bound;
    d.shovel_on = I.cfg.shovel_on;
    d.pcoll = I.cfg.particle_collision;
    d.n_poses = I.n_poses;
    d.n = (int)I.n;
    d.blk_off = I.blk_off;
    d.pbeg = I.pbeg;
    d.node_off = I.node_off;
    d.ext_off = I.ext_off;
    d.dx = (float)I.cfg.dx;
    d.inv_dx = (float)(1.0 / I.cfg.dx);
    d.dt = (float)I.cfg.dt;
    const Lame L = lame_of(I.mat);
    d.mu = (float)L.mu;
    d.lam = (float)L.lam;
    d.alpha = (float)L.alpha;
    d.beta = (float)L.beta;
    d.mp = (float)(I.mat.rho * I.cfg.particle_volume);
    d.vol = (float)I.cfg.particle_volume;
    d.stress_scale = (float)(-I.cfg.dt * I.cfg.particle_volume * 4.0 / (I.cfg.dx * I.cfg.dx));
    d.friction = (float)I.cfg.friction;
    d.smin = (float)h->opt.sigma_min;
    d.poses = I.n_poses > 0 ? h->d_poses.p + I.pose_off : nullptr;
    return d;
}

int upload_instances(mpm_handle* h) {
    std::vector<InstDev> v;
    for (auto& I : h->inst) v.push_back(make_instdev(h, I));
    CK(cudaMemcpyAsync(h->d_inst.p, v.data(), v.size() * sizeof(InstDev), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MPM_OK;
}

// Algorithm 2 (Sec. III-B) with rounded phase lengths, in the simulator
// frame: the paper's x stays x, its vertical z becomes y, its rx is the tilt
// psi. jac[t*36 + k*6 + j] = d a_t[k] / d theta_j with T_i frozen.
int skill_to_actions(const mpm_skill& s, double dt_step, std::vector<double>& act, std::vector<double>& jac) {
    const double* th = s.theta;
    const double vl = s.v_lin * dt_step, vw = s.v_ang * dt_step;
    // phase 1: displace along x and tilt
    const double d1 = 0.12 * th[0], phi1 = th[1] * kPi / 3.0;
    const double tp1 = std::fabs(phi1 / vw);
    const long T1 = std::lround(std::max(std::fabs(d1 / vl), tp1));
    // phase 2: insert along the tilted pointing direction
    const double d2 = 0.03 * (th[2] + 1.0), phi2 = phi1 + kPi / 2.0;
    const long T2 = std::lround(d2 / vl);
    // phase 3: push along the push angle
    const double d3 = 0.1 * (th[4] + 1.0) + 0.04, phi3 = (th[3] + 3.0) * kPi / 3.0;
    const long T3 = std::lround(std::fabs(d3 / vl));
    // phase 4: untilt and lift
    const double d4 = 0.005 * (th[5] + 1.0);
    const long T4 = std::lround(std::max(tp1, d4 / vl));
    const long T = T1 + T2 + T3 + T4;
    if (T < 0 || T > 10000000) return MPM_ERR_INVALID_ARG;
    act.assign((size_t)T * 6, 0.0);
    jac.assign((size_t)T * 36, 0.0);
    const double c2 = std::cos(phi2), s2 = std::sin(phi2), c3 = std::cos(phi3), s3 = std::sin(phi3);
    // Divisors of phases 1 and 4 and their gradients in (theta_displace,
    // theta_rotate, theta_lift): the integer step counts, or (unrounded_T)
    // the real-valued ones, max(|d1| / vl, |phi1| / vw) and max(|phi1| / vw,
    // d4 / vl), differentiated through their active term (the distance term
    // of phase 1 and the angle term of phase 4 on ties).
    double q1 = (double)T1, q4 = (double)T4, gq1[2] = {0.0, 0.0}, gq4[2] = {0.0, 0.0};  // [disp|rot], [rot|lift]
    if (s.unrounded_T) {
        const double td1 = std::fabs(d1 / vl), td4 = d4 / vl;
        const double sd1 = (d1 > 0) - (d1 < 0), sp1 = (phi1 > 0) - (phi1 < 0);
        if (td1 >= tp1) { q1 = td1; gq1[0] = sd1 * 0.12 / vl; }
        else { q1 = tp1; gq1[1] = sp1 * (kPi / 3.0) / vw; }
        if (tp1 >= td4) { q4 = tp1; gq4[0] = sp1 * (kPi / 3.0) / vw; }
        else { q4 = td4; gq4[1] = 0.005 / vl; }
    }
    for (long t = 0; t < T; t++) {
        double* a = &act[(size_t)t * 6];
        double* J = &jac[(size_t)t * 36];
        if (t < T1) {
            a[0] = d1 / q1;
            a[3] = phi1 / q1;
            // d(d1 / q1), d(phi1 / q1) by the quotient rule
            J[0 * 6 + 0] = 0.12 / q1 - a[0] * gq1[0] / q1;
            J[0 * 6 + 1] = -a[0] * gq1[1] / q1;
            J[3 * 6 + 0] = -a[3] * gq1[0] / q1;
            J[3 * 6 + 1] = (kPi / 3.0) / q1 - a[3] * gq1[1] / q1;
        } else if (t < T1 + T2) {
            a[0] = d2 * c2 / T2;
            a[1] = -d2 * s2 / T2;
            J[0 * 6 + 2] = 0.03 * c2 / T2;
            J[1 * 6 + 2] = -0.03 * s2 / T2;
            J[0 * 6 + 1] = -d2 * s2 * (kPi / 3.0) / T2;
            J[1 * 6 + 1] = -d2 * c2 * (kPi / 3.0) / T2;
        } else if (t < T1 + T2 + T3) {
            a[0] = d3 * c3 / T3;
            a[1] = d3 * s3 / T3;
            J[0 * 6 + 4] = 0.1 * c3 / T3;
            J[1 * 6 + 4] = 0.1 * s3 / T3;
            J[0 * 6 + 3] = -d3 * s3 * (kPi / 3.0) / T3;
            J[1 * 6 + 3] = d3 * c3 * (kPi / 3.0) / T3;
        } else {
            a[1] = d4 / q4;
            a[3] = -phi1 / q4;
            J[1 * 6 + 5] = 0.005 / q4 - a[1] * gq4[1] / q4;
            J[1 * 6 + 1] = -a[1] * gq4[0] / q4;
            J[3 * 6 + 1] = -(kPi / 3.0) / q4 - a[3] * gq4[0] / q4;
            J[3 * 6 + 5] = -a[3] * gq4[1] / q4;
        }
    }
    return MPM_OK;
}

// Per-substep pose table: each global step's action is spread evenly over
// its substeps and added to the pose; the velocity is that increment / dt.
void pose_table(const Instance& I, std::vector<float>& out) {
    const int na = (int)(I.actions.size() / 6);
    const int n = std::max(1, na * I.spa);
    out.assign((size_t)n * 8, 0.0f);
    double cur[4] = {I.start[0], I.start[1], I.start[2], I.start[3]};
    for (int s = 0; s < n; s++) {
        const int t = s / I.spa;
        double inc[4] = {0, 0, 0, 0};
        if (t < na)
            for (int k = 0; k < 4; k++) inc[k] = I.actions[(size_t)t * 6 + k] / I.spa;
        for (int k = 0; k < 4; k++) {
            cur[k] += inc[k];
            out[(size_t)s * 8 + k] = (float)cur[k];
            out[(size_t)s * 8 + 4 + k] = (float)(inc[k] / I.cfg.dt);
        }
    }
}

int upload_poses(mpm_handle* h) {
    std::vector<std::vector<float>> tabs(h->inst.size());
    long long total = 0;
    for (size_t i = 0; i < h->inst.size(); i++) {
        Instance& I = h->inst[i];
        if (I.has_traj) pose_table(I, tabs[i]);
        I.pose_off = total;
        I.n_poses = (int)(tabs[i].size() / 8);
        total += (long long)tabs[i].size();
    }
    RK(h->d_poses.ensure((size_t)std::max(total, 8LL), h->device_bytes));
    for (size_t i = 0; i < h->inst.size(); i++)
        if (!tabs[i].empty())
            CK(cudaMemcpyAsync(h->d_poses.p + h->inst[i].pose_off, tabs[i].data(), tabs[i].size() * sizeof(float),
                               cudaMemcpyHostToDevice, h->stream));
    return upload_instances(h);
}

StepArgs base_args(mpm_handle* h) {
    StepArgs a;
    std::memset(&a, 0, sizeof a);
    a.inst = h->d_inst.p;
    a.chunk_inst = h->d_chunk_inst.p;
    a.block_inst = h->d_block_inst.p;
    a.ncap = h->ncap;
    a.n_chunks = h->n_chunks;
    a.n_blocks = h->n_blocks;
    a.n_inst = (int)h->inst.size();
    a.mass = h->d_mass.p;
    a.status = h->d_status.p;
    a.fp64_count = h->d_fp64.p;
    a.fb_list = h->d_fb_list.p;
    a.fb_count = h->d_fb_count.p;
    a.clip = h->opt.clip_grads ? (float)h->opt.clip_value : 0.0f;
    a.tile = h->tile_scatter;
    return a;
}

int read_status(mpm_handle* h) {
    int st = 0;
    CK(cudaMemcpyAsync(&st, h->d_status.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (h->prof.on) h->prof.flush();
    if (st) {
        CK(cudaMemsetAsync(h->d_status.p, 0, sizeof(int), h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    if (st & kStatusNonFinite) return MPM_ERR_NON_FINITE;
    if (st & kStatusDomain) return MPM_ERR_OUT_OF_DOMAIN;
    return MPM_OK;
}

int check_inst(mpm_handle* h, int inst) {
    if (!h || inst < 0 || inst >= (int)h->inst.size()) return MPM_ERR_INVALID_ARG;
    return MPM_OK;
}

int set_device(mpm_handle* h) {
    CK(cudaSetDevice(h->device));
    return MPM_OK;
}

int ensure_stage(mpm_handle* h) { return h->d_stage.ensure((size_t)std::max<int64_t>(h->n_ext, 1) * 24, h->device_bytes); }

int run_kernel(mpm_handle* h, KernelId id, const AdjArgs& A) {
    if (h->prof.on) {
        Profiler::Pending p{(int)id, h->prof.get(), h->prof.get()};
        CK(cudaEventRecord(p.a, h->stream));
        CK(launch_kernel(id, A, h->shape, h->stream));
        CK(cudaEventRecord(p.b, h->stream));
        h->prof.pending.push_back(p);
        if (h->prof.pending.size() > 65536) h->prof.flush();
    } else {
        CK(launch_kernel(id, A, h->shape, h->stream));
    }
    h->launches++;
    return MPM_OK;
}

int run_fused(mpm_handle* h, KernelId id, const AdjArgs& A, const AdjArgs& G) {
    if (h->prof.on) {
        Profiler::Pending p{(int)id, h->prof.get(), h->prof.get()};
        CK(cudaEventRecord(p.a, h->stream));
        CK(launch_fused(id, A, G, h->shape, h->stream));
        CK(cudaEventRecord(p.b, h->stream));
        h->prof.pending.push_back(p);
        if (h->prof.pending.size() > 65536) h->prof.flush();
    } else {
        CK(launch_fused(id, A, G, h->shape, h->stream));
    }
    h->launches++;
    return MPM_OK;
}


int run_substep(mpm_handle* h, const StepArgs& a) {
    AdjArgs A;
    std::memset(&A, 0, sizeof A);
    A.f = a;
    RK(run_kernel(h, KernelId::P2G, A));
    RK(run_kernel(h, KernelId::P2GFp64, A));
    RK(run_kernel(h, KernelId::Grid, A));
    RK(run_kernel(h, KernelId::G2P, A));
    return MPM_OK;
}

// make segment slot k usable: state k+1 (and 0) and grid k, zeroed when new
int ensure_slot(mpm_handle* h, int k) {
    const size_t state_floats = (size_t)h->ncap * kStateComps;
    const size_t need = (size_t)k + 2;
    if (h->seg_state.size() < need) h->seg_state.resize(need);
    if (h->seg_acc.size() < need - 1) {
        h->seg_acc.resize(need - 1);
        h->seg_vout.resize(need - 1);
        h->seg_flags.resize(need - 1);
        h->seg_spec.resize(need - 1);
        h->seg_dirty.resize(need - 1, 0);
    }
    for (size_t i = 0; i < need; i++) RK(h->seg_state[i].ensure(state_floats, h->device_bytes));
    if (h->seg_acc[k].p == nullptr) {
        RK(h->seg_acc[k].ensure((size_t)h->n_nodes, h->device_bytes));
        RK(h->seg_vout[k].ensure((size_t)h->n_nodes, h->device_bytes));
        RK(h->seg_flags[k].ensure(flag_ints(h->n_blocks), h->device_bytes));
        RK(h->seg_spec[k].ensure((size_t)h->ncap * kSpecComps, h->device_bytes));
        CK(cudaMemsetAsync(h->seg_acc[k].p, 0, (size_t)h->n_nodes * sizeof(float4), h->stream));
        CK(cudaMemsetAsync(h->seg_flags[k].p, 0, flag_bytes_zeroed(h->n_blocks), h->stream));
        h->seg_dirty[k] = 0;
    }
    return MPM_OK;
}

// forward arguments for substep k of a segment (states k -> k+1, grid slot k, kept)
StepArgs slot_args(mpm_handle* h, int k, int64_t substep) {
    StepArgs a = base_args(h);
    a.sin = h->seg_state[k].p;
    a.sout = h->seg_state[k + 1].p;
    a.acc = h->seg_acc[k].p;
    a.vout = h->seg_vout[k].p;
    a.flags = h->seg_flags[k].p;
    a.spec = h->seg_spec[k].p;
    a.keep_grid = 1;
    a.substep = (int)substep;
    return a;
}


// Recorded substeps k0 .. k0+cnt-1 of the current segment (global substep
// s0 for k0), each into its slot (cleared first if it holds old sums); a
// backward's recomputation leaves the grid-mass totals alone (recompute).
int run_slot_range(mpm_handle* h, int k0, int cnt, int64_t s0, bool recompute) {
    for (int t = 0; t < cnt; t++) {
        const int k = k0 + t;
        RK(ensure_slot(h, k));
        StepArgs a = slot_args(h, k, s0 + t);
        if (recompute) a.mass = nullptr;
        if (h->seg_dirty[k]) {
            AdjArgs C;
            std::memset(&C, 0, sizeof C);
            C.f = a;
            RK(run_kernel(h, KernelId::SlotClear, C));
        }
        h->seg_dirty[k] = 1;
        RK(run_substep(h, a));
    }
    return MPM_OK;
}

int copy_state(mpm_handle* h, float* dst, const float* src) {
    if (dst == src) return MPM_OK;
    CK(cudaMemcpyAsync(dst, src, (size_t)h->ncap * kStateComps * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    return MPM_OK;
}

// reorder every instance's particles by cell (d_state and the external
// map in place); perm[new slot] = old slot
int sort_particles(mpm_handle* h, int* perm) {
    const size_t nc = (size_t)h->ncap;
    RK(h->d_state2.ensure(nc * kStateComps, h->device_bytes));
    RK(h->d_ext2.ensure(nc, h->device_bytes));
    RK(h->d_key.ensure(nc, h->device_bytes));
    RK(h->d_rank.ensure(nc, h->device_bytes));
    const int n_keys = (int)h->n_nodes;   // one key per cell (cells and nodes share the blocked layout)
    RK(h->d_bcount.ensure((size_t)n_keys, h->device_bytes));
    RK(h->d_bscan.ensure((size_t)n_keys, h->device_bytes));
    RK(h->d_part.ensure((size_t)(n_keys + 1023) / 1024, h->device_bytes));
    RK(h->d_remap.ensure((size_t)std::max<int64_t>(h->n_ext, 1), h->device_bytes));
    CK(launch_sort(h->d_inst.p, h->d_chunk_inst.p, h->n_chunks, h->ncap, n_keys, h->d_state.p, h->d_state2.p,
                   h->d_ext_of_slot.p, h->d_ext2.p, h->d_key.p, h->d_rank.p, h->d_bcount.p, h->d_bscan.p, h->d_part.p,
                   h->d_remap.p, perm, h->stream));
    h->launches += kSortLaunches;
    std::swap(h->d_state, h->d_state2);
    std::swap(h->d_ext_of_slot, h->d_ext2);
    h->since_sort = 0;
    return MPM_OK;
}

}  // namespace

extern "C" {

int mpm_version(void) { return 1; }

const char* mpm_error_string(int code) {
    switch (code) {
        case MPM_OK: return "ok";
        case MPM_ERR_INVALID_ARG: return "invalid argument";
        case MPM_ERR_OOM: return "out of device memory";
        case MPM_ERR_CUDA: return "CUDA error";
        case MPM_ERR_OUT_OF_DOMAIN: return "a particle left the valid domain [dx, (res-2) dx)";
        case MPM_ERR_NON_FINITE: return "non-finite value in the state or an adjoint";
        case MPM_ERR_NO_RECORD: return "backward without a recorded forward";
        case MPM_ERR_TIMEOUT: return "bounded device wait timed out";
        case MPM_ERR_NO_DEVICE: return "no usable CUDA device";
        default: return "unknown error";
    }
}

int mpm_create(int n_inst, const mpm_config* cfgs, const mpm_material* mats, const int64_t* counts,
               const float* x0, const mpm_options* opts, mpm_handle** out) {
    if (!out) return MPM_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_inst < 1 || n_inst > 65536 || !cfgs || !mats || !counts) return MPM_ERR_INVALID_ARG;
    int64_t n_ext = 0;
    for (int i = 0; i < n_inst; i++) {
        RK(validate_config(cfgs[i]));
        RK(validate_material(mats[i]));
        if (counts[i] < 0 || counts[i] > (1LL << 30)) return MPM_ERR_INVALID_ARG;
        n_ext += counts[i];
    }
    if (n_ext > 0 && !x0) return MPM_ERR_INVALID_ARG;
    for (int64_t e = 0; e < 3 * n_ext; e++)
        if (!std::isfinite(x0[e])) return MPM_ERR_INVALID_ARG;
    // every particle must start inside the valid domain [dx, (res-2) dx)
    {
        int64_t e = 0;
        for (int i = 0; i < n_inst; i++)
            for (int64_t p = 0; p < counts[i]; p++, e++)
                for (int k = 0; k < 3; k++) {
                    const double X = x0[3 * e + k] / cfgs[i].dx;
                    if (!(X >= 1.0 && X < cfgs[i].res[k] - 2)) return MPM_ERR_OUT_OF_DOMAIN;
                }
    }
    if (opts && (opts->checkpoint_every < 1 || !(opts->clip_value > 0) || !(opts->sigma_min > 0) ||
                 opts->sort_every < 0 || opts->grad_scale < 0 || opts->grad_scale > 2 ||
                 (opts->grad_scale && opts->clip_grads) || !std::isfinite(opts->oom_star) ||
                 !(opts->grad_delta > 0) || !std::isfinite(opts->grad_delta)))
        return MPM_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return MPM_ERR_NO_DEVICE;
    }
    mpm_handle* h = new (std::nothrow) mpm_handle();
    if (!h) return MPM_ERR_OOM;
    cudaGetDevice(&h->device);
    h->opt.checkpoint_every = 50;
    h->opt.clip_grads = 0;
    h->opt.clip_value = 1e4;
    h->opt.sigma_min = 1e-4;
    h->opt.sort_every = 0;
    h->opt.tile_scatter = 0;
    h->opt.cuda_graphs = 1;
    h->opt.grad_scale = 0;
    h->opt.oom_star = 4.0;
    h->opt.grad_delta = 1e-6;
    h->opt.fuse_adjoint = 1;
    if (opts) h->opt = *opts;
    h->tile_scatter = h->opt.tile_scatter ? 1 : 0;
    h->n_ext = n_ext;
    long long pbeg = 0, node = 0;
    int blk = 0, chunks = 0;
    int64_t ext = 0;
    h->inst.resize(n_inst);
    for (int i = 0; i < n_inst; i++) {
        Instance& I = h->inst[i];
        I.cfg = cfgs[i];
        I.mat = mats[i];
        I.n = counts[i];
        I.ext_off = ext;
        ext += I.n;
        I.pbeg = pbeg;
        I.n_chunks = (int)((I.n + kChunk - 1) / kChunk);
        pbeg += (long long)I.n_chunks * kChunk;
        chunks += I.n_chunks;
        for (int k = 0; k < 3; k++) I.nb[k] = (I.cfg.res[k] + 3) / 4;
        I.n_blocks = I.nb[0] * I.nb[1] * I.nb[2];
        I.blk_off = blk;
        I.node_off = node;
        blk += I.n_blocks;
        node += (long long)I.n_blocks * 64;
    }
    h->ncap = std::max(pbeg, (long long)kChunk);
    h->n_chunks = chunks;
    h->n_blocks = blk;
    h->n_nodes = node;
    int rc = MPM_OK;
    auto fail = [&](int r) {
        mpm_destroy(h);
        return r;
    };
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return MPM_ERR_CUDA;
    }
    h->own_stream = true;
    if ((rc = h->d_inst.ensure(n_inst, h->device_bytes)) || (rc = h->d_chunk_inst.ensure(std::max(chunks, 1), h->device_bytes)) ||
        (rc = h->d_block_inst.ensure(blk, h->device_bytes)) || (rc = h->d_ext_of_slot.ensure(h->ncap, h->device_bytes)) ||
        (rc = h->d_state.ensure((size_t)h->ncap * kStateComps, h->device_bytes)) ||
        (rc = h->d_x0.ensure((size_t)std::max<int64_t>(n_ext, 1) * 3, h->device_bytes)) ||
        (rc = h->d_acc.ensure(node, h->device_bytes)) || (rc = h->d_vout.ensure(node, h->device_bytes)) ||
        (rc = h->d_flags.ensure(flag_ints(blk), h->device_bytes)) || (rc = h->d_status.ensure(1, h->device_bytes)) ||
        (rc = h->d_mass.ensure((size_t)n_inst * 2, h->device_bytes)) ||
        (rc = h->d_fp64.ensure(1, h->device_bytes)) || (rc = h->d_loss.ensure(n_inst, h->device_bytes)) ||
        (rc = h->d_fb_list.ensure(std::max<int64_t>(h->ncap, 1), h->device_bytes)) ||
        (rc = h->d_fb_count.ensure(2, h->device_bytes)))
        return fail(rc);
    std::vector<int> ci(std::max(chunks, 1), 0), bi(blk), eos(h->ncap, -1);
    for (int i = 0; i < n_inst; i++) {
        const Instance& I = h->inst[i];
        for (int c = 0; c < I.n_chunks; c++) ci[(I.pbeg / kChunk) + c] = i;
        for (int b = 0; b < I.n_blocks; b++) bi[I.blk_off + b] = i;
        for (int64_t p = 0; p < I.n; p++) eos[I.pbeg + p] = (int)(I.ext_off + p);
    }
    cudaStream_t s = h->stream;
    if (cudaMemcpyAsync(h->d_chunk_inst.p, ci.data(), ci.size() * sizeof(int), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(h->d_block_inst.p, bi.data(), bi.size() * sizeof(int), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(h->d_ext_of_slot.p, eos.data(), eos.size() * sizeof(int), cudaMemcpyHostToDevice, s) ||
        (n_ext > 0 && cudaMemcpyAsync(h->d_x0.p, x0, (size_t)n_ext * 3 * sizeof(float), cudaMemcpyHostToDevice, s)) ||
        cudaMemsetAsync(h->d_acc.p, 0, node * sizeof(float4), s) ||
        cudaMemsetAsync(h->d_vout.p, 0, node * sizeof(float4), s) || cudaMemsetAsync(h->d_flags.p, 0, flag_bytes_zeroed(blk), s) ||
        cudaMemsetAsync(h->d_mass.p, 0, (size_t)n_inst * 2 * sizeof(double), s) ||
        cudaMemsetAsync(h->d_status.p, 0, sizeof(int), s) ||
        cudaMemsetAsync(h->d_fp64.p, 0, sizeof(unsigned long long), s) ||
        cudaMemsetAsync(h->d_fb_count.p, 0, 2 * sizeof(int), s) || cudaStreamSynchronize(s)) {
        cudaGetLastError();
        return fail(MPM_ERR_CUDA);
    }
    if ((rc = upload_poses(h))) return fail(rc);
    if ((rc = mpm_reset(h))) return fail(rc);
    *out = h;
    return MPM_OK;
}

void mpm_destroy(mpm_handle* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    h->d_inst.release(); h->d_chunk_inst.release(); h->d_block_inst.release(); h->d_ext_of_slot.release();
    h->d_state.release(); h->d_x0.release(); h->d_stage.release(); h->d_poses.release(); h->d_target.release();
    h->d_acc.release(); h->d_vout.release(); h->d_flags.release(); h->d_mass.release(); h->d_status.release(); h->d_fp64.release();
    h->d_loss.release(); h->d_fb_list.release(); h->d_fb_count.release();
    h->d_obs.release(); h->d_keys.release(); h->d_obs_out.release(); h->d_obs_target.release();
    h->d_obs_loss.release(); h->d_obs_count.release();
    h->d_emd_price.release(); h->d_emd_owner.release(); h->d_emd_assign.release(); h->d_emd_ntg.release();
    h->d_emd_cnt.release(); h->d_emd_bids.release();
    for (auto& c : h->ckpt) c.release();
    for (auto& b : h->seg_state) b.release();
    for (auto& b : h->seg_acc) b.release();
    for (auto& b : h->seg_vout) b.release();
    for (auto& b : h->seg_flags) b.release();
    for (auto& b : h->seg_spec) b.release();
    h->d_gacc.release(); h->d_gacc2.release();
    h->d_adj.release(); h->d_gmat.release(); h->d_gpose.release();
    h->d_pstat.release(); h->d_gstat.release(); h->d_gpose_raw.release();
    h->d_state2.release(); h->d_adj2.release(); h->d_ext2.release(); h->d_key.release(); h->d_rank.release();
    h->d_bcount.release(); h->d_bscan.release(); h->d_part.release(); h->d_remap.release(); h->d_perm.release();
    h->d_ext_rec.release();
    for (auto& b : h->seg_perm) b.release();
    h->prof.release();
    if (h->stream && h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

int mpm_set_stream(mpm_handle* h, void* stream) {
    if (!h) return MPM_ERR_INVALID_ARG;
    RK(set_device(h));
    CK(cudaStreamSynchronize(h->stream));
    // all later work is issued on the caller's stream (ordered with the
    // caller's own work); the library's private stream is released
    if (h->stream && h->own_stream) cudaStreamDestroy(h->stream);
    h->stream = (cudaStream_t)stream;
    h->own_stream = false;
    return MPM_OK;
}

int mpm_synchronize(mpm_handle* h) {
    if (!h) return MPM_ERR_INVALID_ARG;
    RK(set_device(h));
    CK(cudaStreamSynchronize(h->stream));
    return MPM_OK;
}

int mpm_set_material(mpm_handle* h, int inst, const mpm_material* mat) {
    RK(check_inst(h, inst));
    if (!mat) return MPM_ERR_INVALID_ARG;
    RK(validate_material(*mat));
    RK(set_device(h));
    h->inst[inst].mat = *mat;
    h->recording = false;
    h->seg_valid = -1;
    return upload_instances(h);
}

int mpm_set_shovel_actions(mpm_handle* h, int inst, const double start_pose[4], int n_actions, const double* actions,
                           int substeps_per_action) {
    RK(check_inst(h, inst));
    if (!start_pose || n_actions < 0 || (n_actions > 0 && !actions) || substeps_per_action < 1)
        return MPM_ERR_INVALID_ARG;
    if ((long long)n_actions * substeps_per_action > 100000000LL) return MPM_ERR_INVALID_ARG;
    for (int k = 0; k < 4; k++)
        if (!std::isfinite(start_pose[k])) return MPM_ERR_INVALID_ARG;
    for (long long t = 0; t < n_actions; t++) {
        for (int k = 0; k < 6; k++)
            if (!std::isfinite(actions[t * 6 + k])) return MPM_ERR_INVALID_ARG;
        if (actions[t * 6 + 4] != 0.0 || actions[t * 6 + 5] != 0.0) return MPM_ERR_INVALID_ARG;
    }
    RK(set_device(h));
    Instance& I = h->inst[inst];
    I.has_traj = true;
    I.has_skill = false;
    std::memcpy(I.start, start_pose, sizeof I.start);
    I.spa = substeps_per_action;
    I.actions.assign(actions, actions + (size_t)n_actions * 6);
    I.jac.clear();
    h->recording = false;
    h->seg_valid = -1;
    return upload_poses(h);
}

int mpm_set_shovel_trajectory(mpm_handle* h, int inst, const mpm_skill* skill) {
    RK(check_inst(h, inst));
    if (!skill || skill->substeps_per_action < 1 || !finite_pos(skill->v_lin) || !finite_pos(skill->v_ang))
        return MPM_ERR_INVALID_ARG;
    for (int k = 0; k < 6; k++)
        if (!std::isfinite(skill->theta[k]) || std::fabs(skill->theta[k]) > 1.0 + 1e-12) return MPM_ERR_INVALID_ARG;
    std::vector<double> act, jac;
    const double dt_step = skill->substeps_per_action * h->inst[inst].cfg.dt;
    RK(skill_to_actions(*skill, dt_step, act, jac));
    RK(mpm_set_shovel_actions(h, inst, skill->start_pose, (int)(act.size() / 6), act.data(),
                              skill->substeps_per_action));
    Instance& I = h->inst[inst];
    I.has_skill = true;
    I.skill = *skill;
    I.jac.swap(jac);
    return MPM_OK;
}

int mpm_num_actions(mpm_handle* h, int inst) {
    RK(check_inst(h, inst));
    return (int)(h->inst[inst].actions.size() / 6);
}

int mpm_reset(mpm_handle* h) {
    if (!h) return MPM_ERR_INVALID_ARG;
    RK(set_device(h));
    CK(launch_state_from_ext(h->ncap, h->ncap, h->d_ext_of_slot.p, h->d_x0.p, nullptr, nullptr, nullptr, h->d_state.p,
                             h->stream));
    h->launches++;
    CK(cudaStreamSynchronize(h->stream));
    h->substep = 0;
    h->recording = false;
    h->seg_valid = -1;
    h->rec_len = 0;
    return MPM_OK;
}

int mpm_set_state(mpm_handle* h, const float* x, const float* v, const float* C, const float* F, int device_ptrs) {
    if (!h || !x) return MPM_ERR_INVALID_ARG;
    RK(set_device(h));
    const float *dx = x, *dv = v, *dC = C, *dF = F;
    if (!device_ptrs) {
        RK(ensure_stage(h));
        float* st = h->d_stage.p;
        const size_t n = (size_t)h->n_ext;
        CK(cudaMemcpyAsync(st, x, n * 3 * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        dx = st;
        if (v) { CK(cudaMemcpyAsync(st + 3 * n, v, n * 3 * sizeof(float), cudaMemcpyHostToDevice, h->stream)); dv = st + 3 * n; }
        if (C) { CK(cudaMemcpyAsync(st + 6 * n, C, n * 9 * sizeof(float), cudaMemcpyHostToDevice, h->stream)); dC = st + 6 * n; }
        if (F) { CK(cudaMemcpyAsync(st + 15 * n, F, n * 9 * sizeof(float), cudaMemcpyHostToDevice, h->stream)); dF = st + 15 * n; }
    }
    CK(launch_state_from_ext(h->ncap, h->ncap, h->d_ext_of_slot.p, dx, dv, dC, dF, h->d_state.p, h->stream));
    h->launches++;
    h->recording = false;
    h->seg_valid = -1;
    h->rec_len = 0;
    if (!device_ptrs) CK(cudaStreamSynchronize(h->stream));
    return MPM_OK;
}

int mpm_get_state(mpm_handle* h, float* x, float* v, float* C, float* F, int device_ptrs) {
    if (!h) return MPM_ERR_INVALID_ARG;
    RK(set_device(h));
    if (device_ptrs) {
        CK(launch_state_to_ext(h->ncap, h->ncap, h->d_ext_of_slot.p, h->d_state.p, x, v, C, F, h->stream));
        h->launches++;
        return MPM_OK;
    }
    RK(ensure_stage(h));
    float* st = h->d_stage.p;
    const size_t n = (size_t)h->n_ext;
    CK(launch_state_to_ext(h->ncap, h->ncap, h->d_ext_of_slot.p, h->d_state.p, st, st + 3 * n, st + 6 * n, st + 15 * n,
                           h->stream));
    h->launches++;
    if (x) CK(cudaMemcpyAsync(x, st, n * 3 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (v) CK(cudaMemcpyAsync(v, st + 3 * n, n * 3 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (C) CK(cudaMemcpyAsync(C, st + 6 * n, n * 9 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (F) CK(cudaMemcpyAsync(F, st + 15 * n, n * 9 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MPM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// CUDA graphs of repeated identical calls
// ---------------------------------------------------------------------------
namespace {

HostSnap snap(const mpm_handle* h) {
    HostSnap s;
    s.substep = h->substep;
    s.rec_start = h->rec_start;
    s.rec_len = h->rec_len;
    s.seg_valid = h->seg_valid;
    s.since_sort = h->since_sort;
    s.seg_valid_len = h->seg_valid_len;
    s.tile = h->tile_scatter;
    s.recording = h->recording;
    s.gacc_dirty = h->gacc_dirty;
    s.seg_dirty = h->seg_dirty;
    s.seg_sorted = h->seg_sorted;
    return s;
}

void restore(mpm_handle* h, const HostSnap& s) {
    h->substep = s.substep;
    h->rec_start = s.rec_start;
    h->rec_len = s.rec_len;
    h->seg_valid = s.seg_valid;
    h->since_sort = s.since_sort;
    h->seg_valid_len = s.seg_valid_len;
    h->tile_scatter = s.tile;
    h->recording = s.recording;
    h->gacc_dirty = s.gacc_dirty;
    h->seg_dirty = s.seg_dirty;
    h->seg_sorted = s.seg_sorted;
}

void drop_graphs(mpm_handle* h) {
    for (GraphEntry* e : h->graphs) {
        if (e->exec) cudaGraphExecDestroy(e->exec);
        delete e;
    }
    h->graphs.clear();
}

constexpr size_t kMaxGraphs = 16;

// Run `launch` (kernel launches and host bookkeeping only: no allocation, no
// synchronisation) eagerly, or capture it, or replay its graph.
template <class F>
int run_graphed(mpm_handle* h, int kind, int64_t n, int flags, F&& launch) {
    if (!h->opt.cuda_graphs || h->prof.on || h->opt.sort_every > 0) return launch();
    const HostSnap start = snap(h);
    GraphEntry* e = nullptr;
    for (GraphEntry* g : h->graphs)
        if (g->kind == kind && g->n == n && g->flags == flags && g->start == start) e = g;
    if (e && e->alloc_bytes != h->device_bytes) {
        // a buffer was reallocated since: the graph may hold stale pointers
        if (e->exec) cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
        e->capturable = true;
        e->alloc_bytes = -1;
    }
    if (!e || e->alloc_bytes < 0) {
        // first time (with this memory): run eagerly, it may allocate
        if (!e) {
            if (h->graphs.size() >= kMaxGraphs) {
                auto old = std::min_element(h->graphs.begin(), h->graphs.end(), [](const GraphEntry* a,
                                                                                   const GraphEntry* b) {
                    return a->used < b->used;
                });
                if ((*old)->exec) cudaGraphExecDestroy((*old)->exec);
                delete *old;
                h->graphs.erase(old);
            }
            e = new GraphEntry();
            e->kind = kind;
            e->n = n;
            e->flags = flags;
            e->start = start;
            h->graphs.push_back(e);
        }
        e->used = ++h->graph_tick;
        e->alloc_bytes = -1;
        const int rc = launch();
        if (rc == MPM_OK) e->alloc_bytes = h->device_bytes;
        return rc;
    }
    e->used = ++h->graph_tick;
    if (e->exec) {
        CK(cudaGraphLaunch(e->exec, h->stream));
        h->graph_launches++;
        restore(h, e->end);
        h->launches += e->launches;
        return MPM_OK;
    }
    if (!e->capturable) return launch();
    // second time: capture the launches, then launch the graph
    const int64_t l0 = h->launches;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        e->capturable = false;
        return launch();
    }
    const int rc = launch();
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
    cudaGraphExec_t x = nullptr;
    bool ok = rc == MPM_OK && ce == cudaSuccess && g != nullptr && h->device_bytes == e->alloc_bytes;
    if (ok && cudaGraphInstantiate(&x, g, 0) != cudaSuccess) ok = false;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        // nothing of the captured work ran: undo the bookkeeping, run eagerly
        cudaGetLastError();
        if (x) cudaGraphExecDestroy(x);
        restore(h, start);
        h->launches = l0;
        e->capturable = false;
        return launch();
    }
    e->end = snap(h);
    e->launches = h->launches - l0;
    e->exec = x;
    CK(cudaGraphLaunch(x, h->stream));
    h->graph_launches++;
    return MPM_OK;
}

}  // namespace

// The launches of mpm_forward and their bookkeeping (no synchronisation).
static int forward_launch(mpm_handle* h, int n_substeps, int record) {
    const int K = h->opt.checkpoint_every;
    if (record) {
        if (!h->recording) {
            h->recording = true;
            h->rec_start = h->substep;
            h->rec_len = 0;
        }
    } else {
        h->recording = false;
        h->rec_len = 0;
        h->seg_valid = -1;
    }
    const size_t state_floats = (size_t)h->ncap * kStateComps;
    if (!record) {
        StepArgs a = base_args(h);
        a.sin = a.sout = h->d_state.p;
        a.acc = h->d_acc.p;
        a.vout = h->d_vout.p;
        a.flags = h->d_flags.p;
        a.keep_grid = 0;
        for (int i = 0; i < n_substeps; i++) {
            if (h->opt.sort_every > 0 && h->since_sort >= h->opt.sort_every) {
                RK(h->d_perm.ensure((size_t)h->ncap, h->device_bytes));
                RK(sort_particles(h, h->d_perm.p));
                a.sin = a.sout = h->d_state.p;
            }
            a.substep = (int)h->substep;
            RK(run_substep(h, a));
            h->substep++;
            h->since_sort++;
        }
    } else if (n_substeps > 0) {
        // Recorded substeps run in the segment slots, keeping every state
        // and grid of the current segment: the backward then reverses the
        // last segment without recomputing it. Earlier segments are
        // recomputed from their checkpoints.
        const float* cur = h->d_state.p;
        for (int i = 0; i < n_substeps;) {
            const int64_t j = h->rec_len / K;
            const int k = (int)(h->rec_len % K);
            if (k == 0) {
                if (h->rec_len == 0) {
                    // external order of the state the record starts from
                    RK(h->d_ext_rec.ensure((size_t)h->ncap, h->device_bytes));
                    CK(cudaMemcpyAsync(h->d_ext_rec.p, h->d_ext_of_slot.p, (size_t)h->ncap * sizeof(int),
                                       cudaMemcpyDeviceToDevice, h->stream));
                }
                if (h->seg_sorted.size() <= (size_t)j) {
                    h->seg_sorted.resize(j + 1, 0);
                    h->seg_perm.resize(j + 1);
                }
                h->seg_sorted[j] = 0;
                if (h->opt.sort_every > 0) {
                    // segments start sorted; the backward undoes the permutation
                    RK(copy_state(h, h->d_state.p, cur));
                    RK(h->seg_perm[j].ensure((size_t)h->ncap, h->device_bytes));
                    RK(sort_particles(h, h->seg_perm[j].p));
                    h->seg_sorted[j] = 1;
                    cur = h->d_state.p;
                }
                if (h->ckpt.size() <= (size_t)j) h->ckpt.resize(j + 1);
                RK(h->ckpt[j].ensure(state_floats, h->device_bytes));
                RK(copy_state(h, h->ckpt[j].p, cur));
                RK(ensure_slot(h, 0));
                RK(copy_state(h, h->seg_state[0].p, cur));
                h->seg_valid = j;
                h->seg_valid_len = 0;
            }
            // the rest of this call within the segment
            const int cnt = (int)std::min<int64_t>(K - k, n_substeps - i);
            RK(run_slot_range(h, k, cnt, h->substep, false));
            cur = h->seg_state[k + cnt].p;
            h->seg_valid_len = k + cnt;
            h->substep += cnt;
            h->rec_len += cnt;
            i += cnt;
        }
        RK(copy_state(h, h->d_state.p, cur));
    }
    return MPM_OK;
}

// The launches of mpm_backward and their bookkeeping (no synchronisation):
// seeds gx, gv (device, external order, may be NULL) -> adjoints, parameter
// and pose sums on the device.
static int backward_launch(mpm_handle* h, const float* gx, const float* gv, bool fresh_gacc) {
    const int K = h->opt.checkpoint_every;
    const int n_inst = (int)h->inst.size();
    const size_t state_floats = (size_t)h->ncap * kStateComps;
    cudaStream_t s = h->stream;
    const bool fuse = h->opt.fuse_adjoint && !h->opt.grad_scale && !h->tile_scatter;
    if (fresh_gacc || h->gacc_dirty) {
        CK(cudaMemsetAsync(h->d_gacc.p, 0, h->d_gacc.n * sizeof(float4), s));
        if (h->d_gacc2.p) CK(cudaMemsetAsync(h->d_gacc2.p, 0, h->d_gacc2.n * sizeof(float4), s));
    }
    h->gacc_dirty = true;   // until every reversed substep has cleared its blocks
    CK(launch_adj_from_ext(h->ncap, h->ncap, h->d_ext_of_slot.p, gx, gv, h->d_adj.p, s));
    h->launches++;
    CK(cudaMemsetAsync(h->d_gmat.p, 0, (size_t)n_inst * 4 * sizeof(double), s));
    CK(cudaMemsetAsync(h->d_gpose.p, 0, (size_t)h->rec_len * n_inst * 8 * sizeof(double), s));
    const int gscale = h->opt.grad_scale;
    if (gscale) {
        // statistics of every state's particle adjoints and every substep's
        // grid adjoints (Sec. III-E); the seed's first
        CK(cudaMemsetAsync(h->d_pstat.p, 0, (size_t)(h->rec_len + 1) * n_inst * 3 * sizeof(double), s));
        CK(cudaMemsetAsync(h->d_gstat.p, 0, (size_t)h->rec_len * n_inst * 3 * sizeof(double), s));
        CK(cudaMemsetAsync(h->d_gpose_raw.p, 0, (size_t)h->rec_len * n_inst * 8 * sizeof(double), s));
        CK(launch_adj_stats(h->d_inst.p, h->d_chunk_inst.p, h->n_chunks, h->ncap, h->d_adj.p, gscale,
                            h->d_pstat.p + (size_t)h->rec_len * n_inst * 3, s));
        h->launches++;
    }
    const int64_t n_seg = (h->rec_len + K - 1) / K;
    for (int64_t j = n_seg - 1; j >= 0; j--) {
        const int64_t seg_begin = j * K;
        const int seg_len = (int)std::min<int64_t>(K, h->rec_len - seg_begin);
        if (!(h->seg_valid == j && h->seg_valid_len == seg_len)) {
            // recompute the segment from its checkpoint, keeping every state and grid
            RK(ensure_slot(h, 0));
            RK(copy_state(h, h->seg_state[0].p, h->ckpt[j].p));
            RK(run_slot_range(h, 0, seg_len, h->rec_start + seg_begin, true));
            h->seg_valid = j;
            h->seg_valid_len = seg_len;
        }
        // reverse it; with fusion, the P2G adjoint of substep i and the G2P
        // adjoint of substep i-1 run as one kernel (grid adjoints ping-pong
        // between two buffers), so only the segment's last substep runs its
        // G2P adjoint alone and its first its P2G adjoint alone
        auto args = [&](int i, float4* gacc) {
            AdjArgs A;
            std::memset(&A, 0, sizeof A);
            A.f = slot_args(h, i, h->rec_start + seg_begin + i);
            A.f.sout = h->seg_state[i].p;
            A.adj = h->d_adj.p;
            A.gacc = gacc;
            A.gmat = h->d_gmat.p;
            A.gpose = h->d_gpose.p + (size_t)(seg_begin + i) * n_inst * 8;
            if (gscale) {
                const size_t r = (size_t)(seg_begin + i);
                A.gscale = gscale;
                A.oom = (float)h->opt.oom_star;
                A.gdelta = (float)h->opt.grad_delta;
                A.pstat_in = h->d_pstat.p + (r + 1) * n_inst * 3;
                A.pstat_out = h->d_pstat.p + r * n_inst * 3;
                A.gstat = h->d_gstat.p + r * n_inst * 3;
                A.gpose_raw = h->d_gpose_raw.p + r * n_inst * 8;
            }
            return A;
        };
        // With fusion the clearing of substep i+1 (its accumulators, flags
        // and the grid-adjoint buffer it used) is deferred into the grid
        // adjoint kernel of substep i, and the particle adjoint kernel after
        // it empties substep i+1's block list: one launch and one memset
        // less per substep. Only substep 0 keeps its own clearing launch.
        float4* gcur = h->d_gacc.p;
        float4* goth = h->d_gacc2.p;
        for (int i = seg_len - 1; i >= 0; i--) {
            AdjArgs A = args(i, gcur);
            const bool defer = fuse && i + 1 < seg_len;   // substep i+1 still to clear
            if (defer) {
                A.clr_flags = h->seg_flags[i + 1].p;
                A.clr_acc = h->seg_acc[i + 1].p;
                A.clr_gacc = goth;
                A.reset_list = h->seg_flags[i + 1].p + h->n_blocks;
            }
            if (!fuse || i == seg_len - 1) RK(run_kernel(h, KernelId::G2PBwd, A));
            RK(run_kernel(h, KernelId::GridBwd, A));
            if (fuse && i > 0) {
                const AdjArgs G = args(i - 1, goth);
                RK(run_fused(h, KernelId::P2GG2PBwd, A, G));
                RK(run_fused(h, KernelId::P2GG2PBwdFp64, A, G));
                std::swap(gcur, goth);
            } else {
                RK(run_kernel(h, KernelId::P2GBwd, A));
                RK(run_kernel(h, KernelId::P2GBwdFp64, A));
                AdjArgs C = A;
                C.clr_flags = nullptr;
                C.clr_acc = C.clr_gacc = nullptr;
                C.reset_list = nullptr;
                RK(run_kernel(h, KernelId::GridClear, C));
                h->seg_dirty[i] = 0;
            }
            if (defer) h->seg_dirty[i + 1] = 0;
        }
        h->seg_valid = -1;
        if ((size_t)j < h->seg_sorted.size() && h->seg_sorted[j]) {
            // adjoint w.r.t. the sorted segment start -> w.r.t. the state before the sort
            RK(h->d_adj2.ensure(state_floats, h->device_bytes));
            CK(launch_unpermute(h->d_inst.p, h->d_chunk_inst.p, h->n_chunks, h->ncap, h->seg_perm[j].p, h->d_adj.p,
                                h->d_adj2.p, s));
            h->launches++;
            std::swap(h->d_adj, h->d_adj2);
        }
    }
    h->gacc_dirty = false;
    return MPM_OK;
}

extern "C" {

int mpm_forward(mpm_handle* h, int n_substeps, int record) {
    if (!h || n_substeps < 0) return MPM_ERR_INVALID_ARG;
    RK(set_device(h));
    RK(run_graphed(h, 0, n_substeps, record ? 1 : 0, [&] { return forward_launch(h, n_substeps, record); }));
    const int st = read_status(h);
    if (st != MPM_OK) {
        h->recording = false;
        h->seg_valid = -1;
    }
    return st;
}

int mpm_loss_mse(mpm_handle* h, const float* x_target, double* loss, float* dL_dx, int device_ptrs) {
    if (!h || !x_target || !loss) return MPM_ERR_INVALID_ARG;
    RK(set_device(h));
    const size_t n = (size_t)h->n_ext;
    const float* tgt = x_target;
    float* out = dL_dx;
    if (!device_ptrs) {
        RK(h->d_target.ensure(std::max<size_t>(n, 1) * 6, h->device_bytes));
        CK(cudaMemcpyAsync(h->d_target.p, x_target, n * 3 * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        tgt = h->d_target.p;
        out = dL_dx ? h->d_target.p + 3 * n : nullptr;
    }
    CK(cudaMemsetAsync(h->d_loss.p, 0, h->inst.size() * sizeof(double), h->stream));
    CK(launch_loss_mse(h->d_inst.p, h->d_chunk_inst.p, h->n_chunks, h->ncap, h->d_ext_of_slot.p, h->d_state.p, tgt, out,
                       h->d_loss.p, h->stream));
    h->launches++;
    CK(cudaMemcpyAsync(loss, h->d_loss.p, h->inst.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (!device_ptrs && dL_dx)
        CK(cudaMemcpyAsync(dL_dx, out, n * 3 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MPM_OK;
}

int mpm_backward(mpm_handle* h, const float* dL_dx, const float* dL_dv, int device_ptrs, double* dL_dmaterial,
                 double* dL_dtheta) {
    if (!h) return MPM_ERR_INVALID_ARG;
    if (!h->recording || h->rec_len == 0) return MPM_ERR_NO_RECORD;
    RK(set_device(h));
    const int n_inst = (int)h->inst.size();
    const size_t state_floats = (size_t)h->ncap * kStateComps;
    const bool fresh_gacc = h->d_gacc.n < (size_t)h->n_nodes ||
                            (h->opt.fuse_adjoint && h->d_gacc2.n < (size_t)h->n_nodes);
    RK(h->d_gacc.ensure((size_t)h->n_nodes, h->device_bytes));
    if (h->opt.fuse_adjoint) RK(h->d_gacc2.ensure((size_t)h->n_nodes, h->device_bytes));
    RK(h->d_adj.ensure(state_floats, h->device_bytes));
    RK(h->d_gmat.ensure((size_t)n_inst * 4, h->device_bytes));
    RK(h->d_gpose.ensure((size_t)h->rec_len * n_inst * 8, h->device_bytes));
    if (h->opt.grad_scale) {
        RK(h->d_pstat.ensure((size_t)(h->rec_len + 1) * n_inst * 3, h->device_bytes));
        RK(h->d_gstat.ensure((size_t)h->rec_len * n_inst * 3, h->device_bytes));
        RK(h->d_gpose_raw.ensure((size_t)h->rec_len * n_inst * 8, h->device_bytes));
    }
    cudaStream_t s = h->stream;
    // seed the adjoint of the final state from library-owned copies, so
    // that a replayed graph never holds a caller's pointer
    const float *gx = nullptr, *gv = nullptr;
    if (dL_dx || dL_dv) {
        RK(ensure_stage(h));
        const size_t n = (size_t)h->n_ext;
        const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (dL_dx && n) { CK(cudaMemcpyAsync(h->d_stage.p, dL_dx, n * 3 * sizeof(float), kind, s)); gx = h->d_stage.p; }
        if (dL_dv && n) { CK(cudaMemcpyAsync(h->d_stage.p + 3 * n, dL_dv, n * 3 * sizeof(float), kind, s)); gv = h->d_stage.p + 3 * n; }
    }
    const int flags = (gx ? 1 : 0) | (gv ? 2 : 0);
    RK(run_graphed(h, 1, 0, flags, [&] { return backward_launch(h, gx, gv, fresh_gacc); }));
    std::vector<double> gm((size_t)n_inst * 4), gp((size_t)h->rec_len * n_inst * 8);
    CK(cudaMemcpyAsync(gm.data(), h->d_gmat.p, gm.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(gp.data(), h->d_gpose.p, gp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    std::vector<double> gst, gpr;
    if (h->opt.grad_scale) {
        gst.resize((size_t)h->rec_len * n_inst * 3);
        gpr.resize(gp.size());
        CK(cudaMemcpyAsync(gst.data(), h->d_gstat.p, gst.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(gpr.data(), h->d_gpose_raw.p, gpr.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    if (h->opt.grad_scale) {
        // the grid kernel's pose adjoint is linear in the post-contact
        // velocity adjoint: scale it by that vector's factor
        for (size_t r = 0; r < (size_t)h->rec_len * n_inst; r++) {
            const double s0 = reg_factor(h->opt.grad_scale, gst[3 * r], h->opt.oom_star, h->opt.grad_delta);
            for (int k = 0; k < 8; k++) gp[8 * r + k] += s0 * gpr[8 * r + k];
        }
    }
    const int st = read_status(h);
    // material chain: mu(E, nu), lambda(E, nu), alpha(phi), m_p = rho V_p
    for (int i = 0; i < n_inst; i++) {
        const Instance& I = h->inst[i];
        const double E = I.mat.E, nu = I.mat.nu;
        const double gmu = gm[4 * i], glam = gm[4 * i + 1], galpha = gm[4 * i + 2], gmp = gm[4 * i + 3];
        const double dmu_dE = 1.0 / (2.0 * (1.0 + nu)), dmu_dnu = -E / (2.0 * (1.0 + nu) * (1.0 + nu));
        const double dl_dE = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
        const double dl_dnu = E * (1.0 + 2.0 * nu * nu) / ((1.0 + nu) * (1.0 + nu) * (1.0 - 2.0 * nu) * (1.0 - 2.0 * nu));
        const double phi = I.mat.phi_deg * kPi / 180.0, sp = std::sin(phi);
        const double da_dphi = std::sqrt(2.0 / 3.0) * 6.0 * std::cos(phi) / ((3.0 - sp) * (3.0 - sp));
        if (dL_dmaterial) {
            dL_dmaterial[4 * i + 0] = gmu * dmu_dE + glam * dl_dE;
            dL_dmaterial[4 * i + 1] = gmu * dmu_dnu + glam * dl_dnu;
            dL_dmaterial[4 * i + 2] = gmp * I.cfg.particle_volume;
            dL_dmaterial[4 * i + 3] = galpha * da_dphi * kPi / 180.0;
        }
    }
    // pose adjoints -> action adjoints -> skill parameters
    for (int i = 0; i < n_inst; i++) {
        Instance& I = h->inst[i];
        const int na = (int)(I.actions.size() / 6);
        I.gactions.assign((size_t)na * 6, 0.0);
        for (int k = 0; k < 4; k++) I.gstart[k] = 0.0;
        if (!I.has_traj || I.n_poses == 0) {
            if (dL_dtheta)
                for (int k = 0; k < 6; k++) dL_dtheta[6 * i + k] = 0.0;
            continue;
        }
        // gradient per table entry; substeps past the table use its last pose
        std::vector<double> tab((size_t)I.n_poses * 8, 0.0);
        for (int64_t r = 0; r < h->rec_len; r++) {
            const int64_t sidx = h->rec_start + r;
            const double* g = &gp[((size_t)r * n_inst + i) * 8];
            if (sidx < I.n_poses) {
                for (int k = 0; k < 8; k++) tab[(size_t)sidx * 8 + k] += g[k];
            } else {
                for (int k = 0; k < 4; k++) tab[(size_t)(I.n_poses - 1) * 8 + k] += g[k];
            }
        }
        double suffix[4] = {0, 0, 0, 0};
        for (int64_t sidx = I.n_poses - 1; sidx >= 0; sidx--) {
            for (int k = 0; k < 4; k++) suffix[k] += tab[(size_t)sidx * 8 + k];
            const int64_t t = sidx / I.spa;
            if (t >= na) continue;
            for (int k = 0; k < 4; k++)
                I.gactions[(size_t)t * 6 + k] += (suffix[k] + tab[(size_t)sidx * 8 + 4 + k] / I.cfg.dt) / I.spa;
        }
        for (int k = 0; k < 4; k++) I.gstart[k] = suffix[k];
        if (dL_dtheta) {
            for (int j = 0; j < 6; j++) {
                double g = 0.0;
                if (I.has_skill)
                    for (int t = 0; t < na; t++)
                        for (int k = 0; k < 6; k++) g += I.gactions[(size_t)t * 6 + k] * I.jac[(size_t)t * 36 + k * 6 + j];
                dL_dtheta[6 * i + j] = g;
            }
        }
    }
    h->recording = false;
    h->seg_valid = -1;
    h->have_grad = true;
    return st;
}

int mpm_get_state_grad(mpm_handle* h, float* gx, float* gv, float* gC, float* gF, int device_ptrs) {
    if (!h) return MPM_ERR_INVALID_ARG;
    if (!h->have_grad) return MPM_ERR_NO_RECORD;
    RK(set_device(h));
    const int* ext = h->d_ext_rec.p ? h->d_ext_rec.p : h->d_ext_of_slot.p;
    if (device_ptrs) {
        CK(launch_state_to_ext(h->ncap, h->ncap, ext, h->d_adj.p, gx, gv, gC, gF, h->stream));
        h->launches++;
        return MPM_OK;
    }
    RK(ensure_stage(h));
    float* st = h->d_stage.p;
    const size_t n = (size_t)h->n_ext;
    CK(launch_state_to_ext(h->ncap, h->ncap, ext, h->d_adj.p, st, st + 3 * n, st + 6 * n, st + 15 * n, h->stream));
    h->launches++;
    if (gx) CK(cudaMemcpyAsync(gx, st, n * 3 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (gv) CK(cudaMemcpyAsync(gv, st + 3 * n, n * 3 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (gC) CK(cudaMemcpyAsync(gC, st + 6 * n, n * 9 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (gF) CK(cudaMemcpyAsync(gF, st + 15 * n, n * 9 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MPM_OK;
}

int mpm_get_action_grad(mpm_handle* h, int inst, double* dL_dactions, double* dL_dstart) {
    RK(check_inst(h, inst));
    if (!h->have_grad) return MPM_ERR_NO_RECORD;
    const Instance& I = h->inst[inst];
    if (dL_dactions && !I.gactions.empty())
        std::memcpy(dL_dactions, I.gactions.data(), I.gactions.size() * sizeof(double));
    if (dL_dstart) std::memcpy(dL_dstart, I.gstart, sizeof I.gstart);
    return MPM_OK;
}

int mpm_record_bytes(int64_t n_particles, int64_t n_nodes, int64_t* state_slot, int64_t* substep_slot) {
    if (n_particles < 0 || n_nodes < 0 || !state_slot || !substep_slot) return MPM_ERR_INVALID_ARG;
    *state_slot = n_particles * kStateComps * (int64_t)sizeof(float);
    *substep_slot = n_particles * kSpecComps * (int64_t)sizeof(float) + n_nodes * 2 * (int64_t)sizeof(float4) +
                    (int64_t)flag_ints((int)std::min<int64_t>(n_nodes / 64 + 1, 1LL << 30)) * (int64_t)sizeof(int);
    return MPM_OK;
}

int mpm_set_launch_shape(mpm_handle* h, const int shape[3]) {
    if (!h || !shape) return MPM_ERR_INVALID_ARG;
    if (shape[0] < 3 || shape[0] > 4 || shape[1] < 3 || shape[1] > 4 || shape[2] < 2 || shape[2] > 4)
        return MPM_ERR_INVALID_ARG;
    if (h->shape.p2g != shape[0] || h->shape.g2p != shape[1] || h->shape.fused != shape[2]) {
        h->shape.p2g = shape[0];
        h->shape.g2p = shape[1];
        h->shape.fused = shape[2];
        drop_graphs(h);   // the captured launches name the old instantiations
    }
    return MPM_OK;
}

int mpm_get_launch_shape(mpm_handle* h, int shape[3]) {
    if (!h || !shape) return MPM_ERR_INVALID_ARG;
    shape[0] = h->shape.p2g;
    shape[1] = h->shape.g2p;
    shape[2] = h->shape.fused;
    return MPM_OK;
}

}  // extern "C"

namespace {

// Choices of the autotuner per workload (device, instances, their particle
// counts and grids), kept for the life of the process.
struct TuneChoice {
    int trial = 0;
    int shape[3] = {4, 4, 3};
    int sort_every = 0;   // 0: no sort, else sort once per checkpoint segment
};
std::mutex g_tune_mu;
std::map<std::vector<int64_t>, TuneChoice> g_tune_cache;

std::vector<int64_t> tune_key(const mpm_handle* h) {
    std::vector<int64_t> k = {h->device, (int64_t)h->inst.size()};
    for (const Instance& I : h->inst) {
        k.push_back(I.n);
        for (int a = 0; a < 3; a++) k.push_back(I.cfg.res[a]);
    }
    return k;
}

// Everything mpm_autotune changes while it times candidates, put back on
// every way out: the state and its particle order, the substep counter, the
// options, the launch shape, the profiler switch; the CUDA events and the
// saved copies are released. Any record is dropped.
struct TuneGuard {
    mpm_handle* h;
    DevBuf<float> save;
    DevBuf<int> save_ext;
    int64_t substep0 = 0;
    mpm_options opt0;
    LaunchShape shape0;
    int tile0 = 0;
    bool prof0 = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bool saved = false;
    explicit TuneGuard(mpm_handle* hh) : h(hh) {
        substep0 = h->substep;
        opt0 = h->opt;
        shape0 = h->shape;
        tile0 = h->tile_scatter;
        prof0 = h->prof.on;
    }
    int save_state() {
        const size_t state_floats = (size_t)h->ncap * kStateComps;
        RK(save.ensure(state_floats, h->device_bytes));
        RK(save_ext.ensure((size_t)h->ncap, h->device_bytes));
        CK(cudaMemcpyAsync(save.p, h->d_state.p, state_floats * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(save_ext.p, h->d_ext_of_slot.p, (size_t)h->ncap * sizeof(int), cudaMemcpyDeviceToDevice,
                           h->stream));
        saved = true;
        return MPM_OK;
    }
    // the saved state again, as the start of a trial
    int restore_state() {
        const size_t state_floats = (size_t)h->ncap * kStateComps;
        CK(cudaMemcpyAsync(h->d_state.p, save.p, state_floats * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(h->d_ext_of_slot.p, save_ext.p, (size_t)h->ncap * sizeof(int), cudaMemcpyDeviceToDevice,
                           h->stream));
        h->substep = substep0;
        h->recording = false;
        h->seg_valid = -1;
        h->since_sort = 1LL << 40;
        return MPM_OK;
    }
    ~TuneGuard() {
        if (saved) restore_state();
        cudaStreamSynchronize(h->stream);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        h->device_bytes -= (int64_t)(save.n * sizeof(float) + save_ext.n * sizeof(int));
        save.release();
        save_ext.release();
        h->prof.reset();
        h->prof.on = prof0;
        h->have_grad = false;
        cudaGetLastError();
    }
    // put the options and the shape back (on failure: everything as found)
    void revert() {
        h->opt = opt0;
        h->tile_scatter = tile0;
        if (h->shape.p2g != shape0.p2g || h->shape.g2p != shape0.g2p || h->shape.fused != shape0.fused) {
            h->shape = shape0;
            drop_graphs(h);
        }
    }
};

// one trial from the saved state: a recorded forward and its backward;
// the elapsed device time in ms
int tune_trial(mpm_handle* h, TuneGuard& g, int trial_substeps, float* ms) {
    RK(g.restore_state());
    CK(cudaEventRecord(g.e0, h->stream));
    RK(mpm_forward(h, trial_substeps, 1));
    RK(mpm_backward(h, nullptr, nullptr, 1, nullptr, nullptr));
    CK(cudaEventRecord(g.e1, h->stream));
    CK(cudaEventSynchronize(g.e1));
    CK(cudaEventElapsedTime(ms, g.e0, g.e1));
    return MPM_OK;
}

}  // namespace

extern "C" {

int mpm_autotune(mpm_handle* h, int trial_substeps, int* chosen) {
    if (!h || trial_substeps < 1 || trial_substeps > 100000) return MPM_ERR_INVALID_ARG;
    RK(set_device(h));
    const std::vector<int64_t> key = tune_key(h);
    TuneChoice best;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end() && it->second.trial >= trial_substeps) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached) {
        TuneGuard g(h);
        RK(g.save_state());
        CK(cudaEventCreate(&g.e0));
        CK(cudaEventCreate(&g.e1));
        // every trial eager: a repeated call would otherwise be the one that
        // captures a CUDA graph, and its timing would include the capture
        h->opt.cuda_graphs = 0;
        int rc = MPM_OK;
        // 1. register caps: every kernel's candidates in the same trials
        // (timed per launch by the profiler), each kernel keeps its fastest
        const int shapes[3][3] = {{3, 3, 2}, {4, 4, 3}, {4, 4, 4}};
        double kbest[3] = {1e300, 1e300, 1e300};
        const KernelId kid[3] = {KernelId::P2G, KernelId::G2P, KernelId::P2GG2PBwd};
        h->opt.sort_every = 0;
        for (int c = 0; c < 3 && rc == MPM_OK; c++) {
            rc = mpm_set_launch_shape(h, shapes[c]);
            for (int rep = 0; rep < 2 && rc == MPM_OK; rep++) {   // the first run allocates
                h->prof.reset();
                h->prof.on = true;
                float ms = 0.f;
                rc = tune_trial(h, g, trial_substeps, &ms);
                h->prof.flush();
                h->prof.on = false;
                if (rc != MPM_OK || rep == 0) continue;
                for (int k = 0; k < 3; k++) {
                    const int id = (int)kid[k];
                    if (h->prof.count[id] == 0) continue;
                    const double avg = h->prof.total_ms[id] / (double)h->prof.count[id];
                    // candidates that repeat an earlier cap are not new
                    bool seen = false;
                    for (int e = 0; e < c; e++) seen = seen || shapes[e][k] == shapes[c][k];
                    if (!seen && avg < kbest[k]) {
                        kbest[k] = avg;
                        best.shape[k] = shapes[c][k];
                    }
                }
            }
        }
        // 2. sorting by cell (once per checkpoint segment) or not, with those caps
        float tbest = 1e30f;
        for (int srt = 0; srt < 2 && rc == MPM_OK; srt++) {
            rc = mpm_set_launch_shape(h, best.shape);
            h->opt.sort_every = srt ? std::max(h->opt.checkpoint_every, 1) : 0;
            for (int rep = 0; rep < 2 && rc == MPM_OK; rep++) {
                float ms = 0.f;
                rc = tune_trial(h, g, trial_substeps, &ms);
                if (rc == MPM_OK && rep == 1 && ms < tbest) {
                    tbest = ms;
                    best.sort_every = h->opt.sort_every;
                }
            }
        }
        g.revert();
        if (rc != MPM_OK) return rc;
        best.trial = trial_substeps;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = best;
    }
    RK(mpm_set_launch_shape(h, best.shape));
    h->opt.sort_every = best.sort_every;
    h->since_sort = 1LL << 40;
    if (chosen) {
        chosen[0] = h->opt.tile_scatter;
        chosen[1] = h->opt.sort_every;
    }
    return MPM_OK;
}

int mpm_set_substep(mpm_handle* h, int64_t substep) {
    if (!h || substep < 0 || substep > (1LL << 30)) return MPM_ERR_INVALID_ARG;
    h->substep = substep;
    h->recording = false;
    h->seg_valid = -1;
    h->rec_len = 0;
    return MPM_OK;
}

int mpm_profile(mpm_handle* h, int enable) {
    if (!h) return MPM_ERR_INVALID_ARG;
    RK(set_device(h));
    h->prof.reset();
    h->prof.on = enable != 0;
    return MPM_OK;
}

int mpm_profile_read(mpm_handle* h, int kernel, double* total_ms, int64_t* launches) {
    if (!h || kernel < 0 || kernel >= (int)KernelId::Count) return MPM_ERR_INVALID_ARG;
    RK(set_device(h));
    h->prof.flush();
    if (total_ms) *total_ms = h->prof.total_ms[kernel];
    if (launches) *launches = h->prof.count[kernel];
    return MPM_OK;
}

const char* mpm_kernel_name(int kernel) {
    static const char* names[] = {"k_p2g",     "k_grid",       "k_g2p",       "k_g2p_bwd",
                                  "k_grid_bwd", "k_p2g_bwd", "k_grid_clear", "k_slot_clear",
                                  "k_p2g_fp64", "k_p2g_bwd_fp64", "k_p2g_g2p_bwd", "k_p2g_g2p_bwd_fp64"};
    if (kernel < 0 || kernel >= (int)KernelId::Count) return "";
    return names[kernel];
}

int mpm_grid_mass(mpm_handle* h, double* mass) {
    if (!h || !mass) return MPM_ERR_INVALID_ARG;
    RK(set_device(h));
    const size_t n_inst = h->inst.size();
    CK(cudaMemcpyAsync(mass, h->d_mass.p + n_inst, n_inst * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return MPM_OK;
}

int mpm_get_info(mpm_handle* h, mpm_info_t* out) {
    if (!h || !out) return MPM_ERR_INVALID_ARG;
    RK(set_device(h));
    unsigned long long fb = 0;
    CK(cudaMemcpyAsync(&fb, h->d_fp64.p, sizeof fb, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    out->n_inst = (int)h->inst.size();
    out->n_particles = h->n_ext;
    out->substep = h->substep;
    out->recorded = h->recording ? h->rec_len : 0;
    out->device_bytes = h->device_bytes;
    out->kernel_launches = h->launches;
    out->fp64_fallbacks = (int64_t)fb;
    out->graph_launches = h->graph_launches;
    return MPM_OK;
}

// ---------------------------------------------------------------------------
// surface observation, height map, HMD and the line search (Sec. III-A,
// Eq. (2), Sec. III-F)
// ---------------------------------------------------------------------------
static int obs_keys(mpm_handle* h, const mpm_obs_grid* grids, int taps, int* npix_out) {
    if (!grids) return MPM_ERR_INVALID_ARG;
    const int n_inst = (int)h->inst.size();
    const int res = grids[0].res;
    std::vector<ObsDev> od(n_inst);
    for (int i = 0; i < n_inst; i++) {
        const mpm_obs_grid& g = grids[i];
        if (g.res != res || res < 1 || res > 4096 || !std::isfinite(g.center[0]) || !std::isfinite(g.center[1]) ||
            !(g.size > 0.0) || !std::isfinite(g.size) || !(g.tap >= 0.0) || !std::isfinite(g.tap))
            return MPM_ERR_INVALID_ARG;
        od[i].x0 = (float)(g.center[0] - 0.5 * g.size);
        od[i].z0 = (float)(g.center[1] - 0.5 * g.size);
        od[i].h = (float)(g.size / res);
        od[i].tap = (float)g.tap;
        od[i].res = res;
    }
    const int npix = res * res;
    RK(set_device(h));
    RK(h->d_obs.ensure((size_t)n_inst, h->device_bytes));
    RK(h->d_keys.ensure((size_t)n_inst * npix, h->device_bytes));
    cudaStream_t s = h->stream;
    CK(cudaMemcpyAsync(h->d_obs.p, od.data(), od.size() * sizeof(ObsDev), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(h->d_keys.p, 0, (size_t)n_inst * npix * sizeof(unsigned long long), s));
    CK(launch_obs_keys(h->d_inst.p, h->d_chunk_inst.p, h->n_chunks, h->ncap, h->d_ext_of_slot.p, h->d_state.p,
                       h->d_obs.p, npix, taps, h->d_keys.p, s));
    h->launches++;
    *npix_out = npix;
    return MPM_OK;
}

int mpm_surface_observation(mpm_handle* h, const mpm_obs_grid* grids, float* points, int* counts, int device_ptrs) {
    if (!h || (!points && !counts)) return MPM_ERR_INVALID_ARG;
    int npix = 0;
    RK(obs_keys(h, grids, 0, &npix));
    const int n_inst = (int)h->inst.size();
    const size_t nf = (size_t)n_inst * npix * 3;
    cudaStream_t s = h->stream;
    float* out = points;
    if (points && !device_ptrs) {
        RK(h->d_obs_out.ensure(nf, h->device_bytes));
        out = h->d_obs_out.p;
    }
    if (out) {
        CK(cudaMemsetAsync(out, 0xff, nf * sizeof(float), s));   // all-ones bits: NaN for empty pixels
        CK(launch_obs_points(h->d_inst.p, h->d_chunk_inst.p, h->n_chunks, h->ncap, h->d_ext_of_slot.p,
                             h->d_state.p, h->d_obs.p, npix, h->d_keys.p, out, s));
        h->launches++;
    }
    if (counts) {
        RK(h->d_obs_count.ensure((size_t)n_inst, h->device_bytes));
        CK(launch_obs_maps(h->d_inst.p, n_inst, npix, h->d_keys.p, nullptr, nullptr, nullptr, nullptr,
                           h->d_obs_count.p, s));
        h->launches++;
        CK(cudaMemcpyAsync(counts, h->d_obs_count.p, (size_t)n_inst * sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    if (points && !device_ptrs) CK(cudaMemcpyAsync(points, out, nf * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return MPM_OK;
}

int mpm_height_map(mpm_handle* h, const mpm_obs_grid* grids, float* maps, int device_ptrs) {
    if (!h || !maps) return MPM_ERR_INVALID_ARG;
    int npix = 0;
    RK(obs_keys(h, grids, 1, &npix));
    const int n_inst = (int)h->inst.size();
    const size_t nf = (size_t)n_inst * npix;
    cudaStream_t s = h->stream;
    float* out = maps;
    if (!device_ptrs) {
        RK(h->d_obs_out.ensure(nf, h->device_bytes));
        out = h->d_obs_out.p;
    }
    CK(launch_obs_maps(h->d_inst.p, n_inst, npix, h->d_keys.p, out, nullptr, nullptr, nullptr, nullptr, s));
    h->launches++;
    if (!device_ptrs) CK(cudaMemcpyAsync(maps, out, nf * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return MPM_OK;
}

int mpm_loss_hmd(mpm_handle* h, const mpm_obs_grid* grids, const float* target_maps, double* loss, float* dL_dx,
                 int device_ptrs) {
    if (!h || !target_maps || !loss) return MPM_ERR_INVALID_ARG;
    int npix = 0;
    RK(obs_keys(h, grids, 1, &npix));
    const int n_inst = (int)h->inst.size();
    const size_t nf = (size_t)n_inst * npix, n = (size_t)h->n_ext;
    cudaStream_t s = h->stream;
    const float* tgt = target_maps;
    float* g = dL_dx;
    if (!device_ptrs) {
        RK(h->d_obs_target.ensure(nf, h->device_bytes));
        CK(cudaMemcpyAsync(h->d_obs_target.p, target_maps, nf * sizeof(float), cudaMemcpyHostToDevice, s));
        tgt = h->d_obs_target.p;
        if (dL_dx) {
            RK(h->d_obs_out.ensure(std::max<size_t>(n * 3, 1), h->device_bytes));
            g = h->d_obs_out.p;
        }
    }
    if (g && n) CK(cudaMemsetAsync(g, 0, n * 3 * sizeof(float), s));
    RK(h->d_obs_loss.ensure((size_t)n_inst, h->device_bytes));
    CK(launch_obs_maps(h->d_inst.p, n_inst, npix, h->d_keys.p, nullptr, tgt, h->d_obs_loss.p, g, nullptr, s));
    h->launches++;
    CK(cudaMemcpyAsync(loss, h->d_obs_loss.p, (size_t)n_inst * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (dL_dx && !device_ptrs && n) CK(cudaMemcpyAsync(dL_dx, g, n * 3 * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return MPM_OK;
}

int mpm_loss_emd(mpm_handle* h, const mpm_obs_grid* grids, const float* targets, const int* n_targets,
                 double* loss, float* dL_dx, int device_ptrs) {
    if (!h || !targets || !n_targets || !loss) return MPM_ERR_INVALID_ARG;
    int npix = 0;
    RK(obs_keys(h, grids, 0, &npix));
    const int n_inst = (int)h->inst.size();
    if (2LL * n_inst * npix >= 0x7fffffffLL) return MPM_ERR_INVALID_ARG;   // bidder indices are 32-bit
    const int n = n_inst * npix;
    const size_t n_ext = (size_t)h->n_ext;
    cudaStream_t s = h->stream;
    // the observed points (NaN where a pixel is empty) and their counts
    RK(h->d_obs_out.ensure((size_t)n * 3, h->device_bytes));
    RK(h->d_obs_count.ensure((size_t)n_inst, h->device_bytes));
    CK(cudaMemsetAsync(h->d_obs_out.p, 0xff, (size_t)n * 3 * sizeof(float), s));
    CK(launch_obs_points(h->d_inst.p, h->d_chunk_inst.p, h->n_chunks, h->ncap, h->d_ext_of_slot.p, h->d_state.p,
                         h->d_obs.p, npix, h->d_keys.p, h->d_obs_out.p, s));
    CK(launch_obs_maps(h->d_inst.p, n_inst, npix, h->d_keys.p, nullptr, nullptr, nullptr, nullptr,
                       h->d_obs_count.p, s));
    h->launches += 2;
    std::vector<int> cnt(n_inst);
    CK(cudaMemcpyAsync(cnt.data(), h->d_obs_count.p, n_inst * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // a one-to-one map needs at least as many targets as observed points
    for (int i = 0; i < n_inst; i++)
        if (n_targets[i] < cnt[i] || n_targets[i] > npix) return MPM_ERR_INVALID_ARG;
    // targets, zero prices, the auction's arrays
    RK(h->d_obs_target.ensure((size_t)n * 3, h->device_bytes));
    RK(h->d_emd_price.ensure((size_t)n, h->device_bytes));
    RK(h->d_emd_owner.ensure((size_t)n, h->device_bytes));
    RK(h->d_emd_assign.ensure((size_t)2 * n, h->device_bytes));
    RK(h->d_emd_bids.ensure((size_t)n, h->device_bytes));
    RK(h->d_emd_ntg.ensure((size_t)n_inst, h->device_bytes));
    RK(h->d_emd_cnt.ensure(1, h->device_bytes));
    RK(h->d_obs_loss.ensure((size_t)n_inst, h->device_bytes));
    CK(cudaMemcpyAsync(h->d_obs_target.p, targets, (size_t)n * 3 * sizeof(float),
                       device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->d_emd_ntg.p, n_targets, n_inst * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(h->d_emd_price.p, 0, (size_t)n * sizeof(float), s));
    CK(cudaMemsetAsync(h->d_emd_bids.p, 0, (size_t)n * sizeof(unsigned long long), s));
    // epsilon scaling: from a quarter of the largest square side down to 1e-6
    // of it (a bid must stay several FP32 ulps above prices of that order)
    double side = 0.0;
    for (int i = 0; i < n_inst; i++) side = std::max(side, grids[i].size);
    const double eps_final = 1e-6 * side;
    constexpr int kRoundsPerCheck = 8;
    constexpr int64_t kMaxRounds = 2000000;   // per phase: an unfinished auction is an error, not a hang
    for (double eps = 0.25 * side;; eps = std::max(eps / 5.0, eps_final)) {
        CK(launch_emd_reset(n, h->d_emd_owner.p, h->d_emd_assign.p, s));
        h->launches++;
        int64_t rounds = 0;
        for (;;) {
            int bidders = 0;
            for (int r = 0; r < kRoundsPerCheck; r++) {
                CK(cudaMemsetAsync(h->d_emd_cnt.p, 0, sizeof(int), s));
                CK(launch_emd_round(n_inst, npix, h->d_obs_out.p, h->d_obs_target.p, h->d_emd_ntg.p,
                                    h->d_obs_count.p, h->d_emd_owner.p, h->d_emd_assign.p, h->d_emd_price.p,
                                    h->d_emd_bids.p, (float)eps, h->d_emd_cnt.p, s));
                h->launches += 2;
            }
            rounds += kRoundsPerCheck;
            CK(cudaMemcpyAsync(&bidders, h->d_emd_cnt.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (bidders == 0) break;
            if (rounds >= kMaxRounds) return MPM_ERR_TIMEOUT;
        }
        if (eps <= eps_final) break;
    }
    // the distance and its gradient w.r.t. the observed particles
    float* g = dL_dx;
    if (dL_dx && !device_ptrs) {
        RK(ensure_stage(h));
        g = h->d_stage.p;
    }
    if (g && n_ext) CK(cudaMemsetAsync(g, 0, n_ext * 3 * sizeof(float), s));
    CK(launch_emd_loss(h->d_inst.p, n_inst, npix, h->d_obs_out.p, h->d_obs_target.p, h->d_emd_assign.p,
                       h->d_keys.p, h->d_obs_loss.p, g, s));
    h->launches++;
    CK(cudaMemcpyAsync(loss, h->d_obs_loss.p, n_inst * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (dL_dx && !device_ptrs && n_ext) CK(cudaMemcpyAsync(dL_dx, g, n_ext * 3 * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return MPM_OK;
}

int mpm_line_search(mpm_handle* h, int n_cand, const mpm_material* mats, const mpm_skill* skills, int n_substeps,
                    const mpm_obs_grid* grids, const float* target_maps, int device_ptrs, double* losses,
                    int* best) {
    if (!h || n_cand < 1 || n_cand > (int)h->inst.size() || n_substeps < 0 || !grids || !target_maps || !best)
        return MPM_ERR_INVALID_ARG;
    for (int k = 0; k < n_cand; k++) {
        if (mats) RK(mpm_set_material(h, k, &mats[k]));
        if (skills) RK(mpm_set_shovel_trajectory(h, k, &skills[k]));
    }
    RK(mpm_forward(h, n_substeps, 0));
    std::vector<double> L(h->inst.size());
    RK(mpm_loss_hmd(h, grids, target_maps, L.data(), nullptr, device_ptrs));
    int b = 0;
    for (int k = 1; k < n_cand; k++)
        if (L[k] < L[b]) b = k;
    *best = b;
    if (losses)
        for (int k = 0; k < n_cand; k++) losses[k] = L[k];
    return MPM_OK;
}

}  // extern "C"
