// Types shared by the host side of the library and its kernels.
#pragma once
#include <stdint.h>

namespace mpm {

constexpr int kChunk = 256;        // particles per CTA in particle kernels; instances are padded to it
constexpr int kStateComps = 24;    // x 3, v 3, C 9, F 9 (structure of arrays)
constexpr int kX = 0, kV = 3, kC = 6, kF = 15;
constexpr int kSpecComps = 14;     // recorded SVD of the trial F: U and V as unit quaternions, sigma, sigma^2 - 1

// status bits written by kernels
constexpr int kStatusDomain = 1;
constexpr int kStatusNonFinite = 2;

// One instance, as the kernels see it (device memory, read-only in kernels).
struct InstDev {
    int res[3];
    int nb[3];              // 4x4x4 blocks per axis
    int bound;
    int shovel_on;
    int pcoll;
    int n_poses;
    int n;                  // particles
    int blk_off;            // first grid block of this instance
    long long pbeg;         // first particle slot
    long long node_off;     // first node (blocked layout)
    long long ext_off;      // first particle in external order
    float dx, inv_dx, dt;
    float g[3];
    float mu, lam, alpha, beta;   // beta = (3 lam + 2 mu) / (2 mu) * alpha
    float mp, vol;
    float stress_scale;     // -dt * vol * 4 / dx^2
    float friction;
    float sh[3];
    float smin;
    const float* poses;     // n_poses * 8: tip xyz, psi, tip velocity, psi rate
};

// Observation / height-map square of one instance (Sec. III-A), FP32 as the
// pixel index is computed: x0 = cx - size/2, z0 = cz - size/2, h = size/res.
struct ObsDev {
    float x0, z0, h, tap;
    int res;
};

// Arguments of one substep's kernels (passed by value).
struct StepArgs {
    const InstDev* inst;
    const int* chunk_inst;  // particle chunk -> instance
    const int* block_inst;  // grid block -> instance
    long long ncap;         // stride of a state component
    int n_chunks;
    int n_blocks;
    int substep;            // index into the pose tables
    const float* sin;       // state at the start of the substep [24][ncap]
    float* sout;            // state at the end (may equal sin)
    float4* acc;            // P2G accumulators (m, mv) of this substep
    float4* vout;           // grid velocity after the update (xyz), mass (w)
    int* flags;             // grid blocks touched this substep: [n_blocks] flags (0/1), then the
                            // list length, then [n_blocks] the listed blocks
    int keep_grid;          // 1: the grid kernel leaves acc/flags for the backward
    int n_inst;
    double* mass;           // n_inst running sums, then n_inst totals of the last grid update; may be null
    int* status;
    unsigned long long* fp64_count;
    float clip;             // > 0: clip adjoints to [-clip, clip]
    int tile;               // 1: sum scatters in a shared-memory tile per CTA
    float* spec;            // record mode: SVD of the trial F per particle [kSpecComps][ncap]
                            // (U row-major, V row-major, sigma, sigma^2 - 1), else null
    int* fb_list;           // particles deferred to the FP64 constitutive kernels [ncap]
    int* fb_count;          // [0] entries of fb_list, [1] CTA ticket; both zero between launches
};

// Arguments of one substep's adjoint kernels.
struct AdjArgs {
    StepArgs f;             // the forward substep being reversed (sin = state_k)
    float* adj;             // adjoint of the state [24][ncap], in place: k+1 -> k
    float4* gacc;           // grid adjoint buffer (zero on entry for touched blocks)
    double* gmat;           // n_inst * 4: d/d(mu, lambda, alpha, m_p)
    double* gpose;          // n_inst * 8: adjoint of this substep's pose
    // Sec. III-E regularisers of whole adjoint vectors (gscale 1: dynamic
    // scaling, 2: normalisation; 0: off). Statistics per instance are the
    // largest magnitude (1) or the sum of squares (2) of a vector.
    int gscale;
    float oom, gdelta;
    const double* pstat_in; // n_inst * 3: x, v, F adjoints of state k+1
    double* pstat_out;      // n_inst * 3: the same of state k (zeroed by the host)
    double* gstat;          // n_inst * 3: grid v-bar after / before the contact, m-bar of substep k,
                            // unregularised (zeroed by the host)
    double* gpose_raw;      // n_inst * 8: the grid kernel's pose adjoint, unregularised
    // Deferred clearing of the substep reversed just before (fused adjoint):
    // the grid adjoint kernel also zeroes the accumulators, grid adjoints and
    // flags of the blocks listed in clr_flags; the particle adjoint kernel
    // after it empties that list (*reset_list = 0). Null: nothing deferred.
    int* clr_flags;
    float4* clr_acc;
    float4* clr_gacc;
    int* reset_list;
};

}  // namespace mpm
