// Host-side launchers of the library's kernels.
#pragma once
#include <cuda_runtime.h>

#include "mpm_types.h"

namespace mpm {

enum class KernelId : int {
    P2G = 0, Grid, G2P, G2PBwd, GridBwd, P2GBwd, GridClear, SlotClear, P2GFp64, P2GBwdFp64, P2GG2PBwd,
    P2GG2PBwdFp64, Count
};
constexpr int kFp64Ctas = 152;   // CTAs of the FP64 fix-up kernels (grid-stride over the deferred list)
constexpr int kFp64Threads = 128;
constexpr int kListCtas = 152 * 8;   // CTAs of the grid kernels that walk the touched-block list

// Register caps of the particle kernels, as the minimum number of resident
// CTAs per SM each is compiled for: k_p2g and k_g2p 3 or 4, the fused
// adjoint 2, 3 or 4. The defaults are the fastest of measured sweeps on the
// 1M-particle bed; mpm_autotune times the alternatives for a handle.
struct LaunchShape {
    int p2g = 4, g2p = 4, fused = 3;
};

// one substep kernel; forward kernels read only A.f
cudaError_t launch_kernel(KernelId id, const AdjArgs& A, const LaunchShape& ls, cudaStream_t s);
// the fused adjoint (P2GG2PBwd, P2GG2PBwdFp64): the P2G adjoint of substep k
// (A) with the G2P adjoint of substep k-1 (G, whose gacc is the other grid
// adjoint buffer); not with the regularisers or the scatter tile
cudaError_t launch_fused(KernelId id, const AdjArgs& A, const AdjArgs& G, const LaunchShape& ls, cudaStream_t s);
cudaError_t launch_state_from_ext(long long ncap, long long nslots, const int* ext_of_slot, const float* x,
                                  const float* v, const float* C, const float* F, float* s, cudaStream_t st);
// statistics of the x, v, F adjoints of a state for the regularisers of
// Sec. III-E (mode 1: largest magnitude, 2: sum of squares) into
// pstat[3 * instance + {0, 1, 2}] (zeroed by the caller)
cudaError_t launch_adj_stats(const InstDev* inst, const int* chunk_inst, int n_chunks, long long ncap,
                             const float* adj, int mode, double* pstat, cudaStream_t st);
cudaError_t launch_adj_from_ext(long long ncap, long long nslots, const int* ext_of_slot, const float* gx,
                                const float* gv, float* adj, cudaStream_t st);
cudaError_t launch_state_to_ext(long long ncap, long long nslots, const int* ext_of_slot, const float* s, float* x,
                                float* v, float* C, float* F, cudaStream_t st);
// reorder the particles of every instance by grid block, rank-major inside
// a block (n_keys = cells of all instances, 64 per block): state ->
// state_out, ext_old -> ext_new, perm[new] = old; remap holds one int per
// particle (scratch); 7 kernels
cudaError_t launch_sort(const InstDev* inst, const int* chunk_inst, int n_chunks, long long ncap, int n_keys,
                        const float* state, float* state_out, const int* ext_old, int* ext_new, int* key, int* rank,
                        int* bcount, int* bscan, int* part, int* remap, int* perm, cudaStream_t st);
constexpr int kSortLaunches = 7;
// dst[perm[q]] = src[q] for all 24 components
cudaError_t launch_unpermute(const InstDev* inst, const int* chunk_inst, int n_chunks, long long ncap, const int* perm,
                             const float* src, float* dst, cudaStream_t st);
cudaError_t launch_loss_mse(const InstDev* inst, const int* chunk_inst, int n_chunks, long long ncap,
                            const int* ext_of_slot, const float* s, const float* target, float* dldx, double* loss,
                            cudaStream_t st);

// surface observation / height map (Sec. III-A): per-pixel winner keys of all
// instances (keys zeroed by the caller; taps 0: own pixel, 1: 5-tap cross)
cudaError_t launch_obs_keys(const InstDev* inst, const int* chunk_inst, int n_chunks, long long ncap,
                            const int* ext_of_slot, const float* s, const ObsDev* obs, int npix, int taps,
                            unsigned long long* keys, cudaStream_t st);
// positions of the winners (points prefilled by the caller)
cudaError_t launch_obs_points(const InstDev* inst, const int* chunk_inst, int n_chunks, long long ncap,
                              const int* ext_of_slot, const float* s, const ObsDev* obs, int npix,
                              const unsigned long long* keys, float* points, cudaStream_t st);
// heights, distance to a target map and its gradient, non-empty pixel counts
// (each output may be null)
cudaError_t launch_obs_maps(const InstDev* inst, int n_inst, int npix, const unsigned long long* keys, float* maps,
                            const float* target, double* loss, float* dL_dx, int* counts, cudaStream_t st);

// Earth Mover's distance (Eq. (1)) by an auction over all instances: bidders
// are observation pixels (points, NaN = empty) and n_targets[i] - counts[i]
// zero-cost dummies per instance (flat indices n + instance * npix + d),
// objects the first n_targets[i] target rows of instance i; assign (2n) /
// owner (n) hold flat indices. A round is one bid and one resolve kernel;
// *unassigned counts the bidders that bid (zero: the phase is over).
cudaError_t launch_emd_reset(int n, int* owner, int* assign, cudaStream_t st);
cudaError_t launch_emd_round(int n_inst, int npix, const float* points, const float* targets, const int* n_targets,
                             const int* counts, int* owner, int* assign, float* price, unsigned long long* bids,
                             float eps, int* unassigned, cudaStream_t st);
// the distance per instance (FP64) and the gradient of the observed particles
cudaError_t launch_emd_loss(const InstDev* inst, int n_inst, int npix, const float* points, const float* targets,
                            const int* assign, const unsigned long long* keys, double* loss, float* dL_dx,
                            cudaStream_t st);

}  // namespace mpm
