// Surface observation, height map and height-map distance (DDBot, arXiv
// 2510.17335, Sec. III-A "States and observations", Eq. (2)), for sm_103a.
//
// A pixel's winner is found with one 64-bit atomicMax per particle and
// pixel on the key (ordered FP32 height << 32) | (~local particle index):
// the highest particle wins, equal heights go to the lowest index, in any
// launch order. Pixel indices are computed in FP32 with IEEE division,
// floorf((x - x0) / h), so that they match a CPU evaluation bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm_launch.h"
#include "mpm_types.h"

namespace mpm {
namespace {

__device__ __forceinline__ int obs_pixel(const ObsDev& g, float x, float z) {
    const float fi = floorf(__fdiv_rn(x - g.x0, g.h)), fj = floorf(__fdiv_rn(z - g.z0, g.h));
    if (!(fi >= 0.0f && fi < (float)g.res && fj >= 0.0f && fj < (float)g.res)) return -1;
    return (int)fi * g.res + (int)fj;
}

// monotone map of a float to an unsigned int (total order of the reals)
__device__ __forceinline__ unsigned ordered(float y) {
    const unsigned u = __float_as_uint(y);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float unordered(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

__device__ __forceinline__ unsigned long long obs_key(float y, unsigned local) {
    return ((unsigned long long)ordered(y) << 32) | (unsigned long long)(0xffffffffu - local);
}

// keys of every instance's pixels; taps = 0: the particle's own pixel
// (observation), 1: the 5-tap cross and heights above 0 (height map)
__global__ void __launch_bounds__(kChunk) k_obs_keys(const InstDev* inst, const int* chunk_inst, long long ncap,
                                                     const int* ext_of_slot, const float* s, const ObsDev* obs,
                                                     int npix, int taps, unsigned long long* keys) {
    const int i = chunk_inst[blockIdx.x];
    const InstDev& I = inst[i];
    const long long p = (long long)blockIdx.x * kChunk + threadIdx.x;
    if (p - I.pbeg >= I.n) return;
    const float x = s[(kX + 0) * ncap + p], y = s[(kX + 1) * ncap + p], z = s[(kX + 2) * ncap + p];
    const unsigned local = (unsigned)((long long)ext_of_slot[p] - I.ext_off);
    const ObsDev g = obs[i];
    unsigned long long* kk = keys + (long long)i * npix;
    const unsigned long long key = obs_key(y, local);
    if (!taps) {
        const int q = obs_pixel(g, x, z);
        if (q >= 0) atomicMax(kk + q, key);
        return;
    }
    if (!(y > 0.0f)) return;   // the map starts at 0 and takes only higher values
    const float tx[5] = {x, x + g.tap, x - g.tap, x, x};
    const float tz[5] = {z, z, z, z + g.tap, z - g.tap};
#pragma unroll
    for (int t = 0; t < 5; t++) {
        const int q = obs_pixel(g, tx[t], tz[t]);
        if (q >= 0) atomicMax(kk + q, key);
    }
}

// observation points: each winner writes its position into its pixel
__global__ void __launch_bounds__(kChunk) k_obs_points(const InstDev* inst, const int* chunk_inst, long long ncap,
                                                       const int* ext_of_slot, const float* s, const ObsDev* obs,
                                                       int npix, const unsigned long long* keys, float* points) {
    const int i = chunk_inst[blockIdx.x];
    const InstDev& I = inst[i];
    const long long p = (long long)blockIdx.x * kChunk + threadIdx.x;
    if (p - I.pbeg >= I.n) return;
    const float x = s[(kX + 0) * ncap + p], y = s[(kX + 1) * ncap + p], z = s[(kX + 2) * ncap + p];
    const unsigned local = (unsigned)((long long)ext_of_slot[p] - I.ext_off);
    const int q = obs_pixel(obs[i], x, z);
    if (q < 0) return;
    const long long at = (long long)i * npix + q;
    if (keys[at] == obs_key(y, local)) {
        points[3 * at + 0] = x;
        points[3 * at + 1] = y;
        points[3 * at + 2] = z;
    }
}

// one CTA per instance: pixel heights (0 where empty), optional distance to a
// target map (FP64, fixed order: deterministic) and the gradient +-1 at each
// pixel's winner (dL_dx in external order, zeroed by the caller)
__global__ void __launch_bounds__(256) k_obs_maps(const InstDev* inst, int npix, const unsigned long long* keys,
                                                  float* maps, const float* target, double* loss, float* dL_dx,
                                                  int* counts) {
    const int i = blockIdx.x;
    const unsigned long long* kk = keys + (long long)i * npix;
    double acc = 0.0;
    int cnt = 0;
    for (int q = threadIdx.x; q < npix; q += blockDim.x) {
        const unsigned long long k = kk[q];
        const bool hit = k != 0ull;
        const float hgt = hit ? unordered((unsigned)(k >> 32)) : 0.0f;
        cnt += hit;
        if (maps) maps[(long long)i * npix + q] = hgt;
        if (target) {
            const double d = (double)hgt - (double)target[(long long)i * npix + q];
            acc += fabs(d);
            if (dL_dx && hit && d != 0.0) {
                const long long e = inst[i].ext_off + (long long)(0xffffffffu - (unsigned)(k & 0xffffffffull));
                atomicAdd(dL_dx + 3 * e + 1, d > 0.0 ? 1.0f : -1.0f);
            }
        }
    }
    __shared__ double sacc[256];
    __shared__ int scnt[256];
    sacc[threadIdx.x] = acc;
    scnt[threadIdx.x] = cnt;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sacc[threadIdx.x] += sacc[threadIdx.x + o];
            scnt[threadIdx.x] += scnt[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (loss) loss[i] = sacc[0];
        if (counts) counts[i] = scnt[0];
    }
}

}  // namespace

cudaError_t launch_obs_keys(const InstDev* inst, const int* chunk_inst, int n_chunks, long long ncap,
                            const int* ext_of_slot, const float* s, const ObsDev* obs, int npix, int taps,
                            unsigned long long* keys, cudaStream_t st) {
    if (n_chunks <= 0) return cudaSuccess;
    k_obs_keys<<<n_chunks, kChunk, 0, st>>>(inst, chunk_inst, ncap, ext_of_slot, s, obs, npix, taps, keys);
    return cudaGetLastError();
}

cudaError_t launch_obs_points(const InstDev* inst, const int* chunk_inst, int n_chunks, long long ncap,
                              const int* ext_of_slot, const float* s, const ObsDev* obs, int npix,
                              const unsigned long long* keys, float* points, cudaStream_t st) {
    if (n_chunks <= 0) return cudaSuccess;
    k_obs_points<<<n_chunks, kChunk, 0, st>>>(inst, chunk_inst, ncap, ext_of_slot, s, obs, npix, keys, points);
    return cudaGetLastError();
}

cudaError_t launch_obs_maps(const InstDev* inst, int n_inst, int npix, const unsigned long long* keys, float* maps,
                            const float* target, double* loss, float* dL_dx, int* counts, cudaStream_t st) {
    if (n_inst <= 0) return cudaSuccess;
    k_obs_maps<<<n_inst, 256, 0, st>>>(inst, npix, keys, maps, target, loss, dL_dx, counts);
    return cudaGetLastError();
}

}  // namespace mpm

// ---------------------------------------------------------------------------
// Earth Mover's distance of Eq. (1) (Sec. III-A): the least total Euclidean
// distance over one-to-one maps of an instance's observed points (the
// non-empty pixels of its observation) into its target points, by an
// auction (Bertsekas) with epsilon scaling. Bidders are pixels, objects are
// target rows; a bidder's value of object j is -|x - y_j| - price_j. One
// warp per unassigned bidder finds its best and second-best objects and bids
// price + (best - second) + eps with a 64-bit atomicMax on (ordered bid,
// bidder): the highest bid wins (ties: the higher bidder index), in any
// launch order. Each phase ends with every bidder assigned; the final
// assignment costs at most n * eps more than the optimum.
// ---------------------------------------------------------------------------
namespace mpm {
namespace {

// Bidders 0 .. n-1 are the pixels of all instances; bidders n .. 2n-1 are
// dummies, n_targets[i] - counts[i] of them per instance, that value every
// target at distance 0: they square the problem (as many bidders as
// targets), which the forward auction with epsilon scaling needs to end at
// the optimum when there are more targets than observed points.
__global__ void __launch_bounds__(256) k_emd_bid(int npix, const float* points, const float* targets,
                                                 const int* n_targets, const int* counts, const int* assign,
                                                 const float* price, unsigned long long* bids, float eps, int n,
                                                 int* unassigned) {
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= 2 * n) return;
    const bool dummy = b >= n;
    const int inst = (dummy ? b - n : b) / npix;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;
    if (dummy) {
        if ((b - n) % npix >= n_targets[inst] - counts[inst]) return;   // not one of this instance's dummies
    } else {
        const float* xp = points + 3 * (long long)b;
        x0 = xp[0]; x1 = xp[1]; x2 = xp[2];
        if (x0 != x0) return;   // empty pixel (NaN)
    }
    if (assign[b] >= 0) return;
    const int m = n_targets[inst];
    const float* tg = targets + 3 * (long long)inst * npix;
    const float* pr = price + (long long)inst * npix;
    float v1 = -3.0e38f, v2 = -3.0e38f;
    int j1 = -1;
    for (int j = lane; j < m; j += 32) {
        float dist = 0.0f;
        if (!dummy) {
            const float d0 = x0 - tg[3 * j], d1 = x1 - tg[3 * j + 1], d2 = x2 - tg[3 * j + 2];
            dist = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
        }
        const float v = -dist - pr[j];
        if (v > v1) { v2 = v1; v1 = v; j1 = j; }
        else if (v > v2) v2 = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov1 = __shfl_xor_sync(0xffffffffu, v1, o), ov2 = __shfl_xor_sync(0xffffffffu, v2, o);
        const int oj1 = __shfl_xor_sync(0xffffffffu, j1, o);
        // merge the two (best, second) pairs; equal values: the lower object
        const bool take = ov1 > v1 || (ov1 == v1 && oj1 >= 0 && (j1 < 0 || oj1 < j1));
        const float nv2 = take ? fmaxf(v1, ov2) : fmaxf(v2, ov1);
        if (take) { v1 = ov1; j1 = oj1; }
        v2 = nv2;
    }
    if (lane == 0 && j1 >= 0) {
        // with a single object the second best is minus infinity: bid its price + eps
        const float inc = (v2 > -3.0e38f ? v1 - v2 : 0.0f) + eps;
        const float bid = pr[j1] + inc;
        const unsigned u = __float_as_uint(bid);
        const unsigned ob = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
        atomicMax(bids + (long long)inst * npix + j1, ((unsigned long long)ob << 32) | (unsigned)b);
        atomicAdd(unassigned, 1);
    }
}

__global__ void __launch_bounds__(256) k_emd_resolve(int n_objects, int* owner, int* assign, float* price,
                                                     unsigned long long* bids) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_objects) return;
    const unsigned long long k = bids[j];
    if (k == 0ull) return;
    bids[j] = 0ull;
    const int winner = (int)(k & 0xffffffffull);
    const unsigned ob = (unsigned)(k >> 32);
    price[j] = __uint_as_float((ob & 0x80000000u) ? (ob & 0x7fffffffu) : ~ob);
    const int prev = owner[j];
    // only unassigned bidders bid, so the previous owner did not win elsewhere this round
    if (prev >= 0) assign[prev] = -1;
    owner[j] = winner;
    assign[winner] = j;   // flat object index: instance * npix + target row
}

// a new phase: nobody assigned (n objects, 2n bidders), prices kept
__global__ void __launch_bounds__(256) k_emd_reset(int n, int* owner, int* assign) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) owner[j] = -1;
    if (j < 2 * n) assign[j] = -1;
}

// one CTA per instance: d_EMD (FP64, fixed order) and the gradient of each
// observed particle, (x - y) / |x - y|, into dL_dx (external order) through
// the observation's winner keys
__global__ void __launch_bounds__(256) k_emd_loss(const InstDev* inst, int npix, const float* points,
                                                  const float* targets, const int* assign,
                                                  const unsigned long long* keys, double* loss, float* dL_dx) {
    const int i = blockIdx.x;
    double acc = 0.0;
    for (int q = threadIdx.x; q < npix; q += blockDim.x) {
        const long long b = (long long)i * npix + q;
        const int a = assign[b];
        if (a < 0) continue;
        const float* x = points + 3 * b;
        const float* y = targets + 3 * (long long)a;
        const float d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
        const double dist = sqrt((double)d0 * d0 + (double)d1 * d1 + (double)d2 * d2);
        acc += dist;
        if (dL_dx && dist > 0.0) {
            const long long e = inst[i].ext_off + (long long)(0xffffffffu - (unsigned)(keys[b] & 0xffffffffull));
            dL_dx[3 * e + 0] = (float)(d0 / dist);
            dL_dx[3 * e + 1] = (float)(d1 / dist);
            dL_dx[3 * e + 2] = (float)(d2 / dist);
        }
    }
    __shared__ double sacc[256];
    sacc[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sacc[threadIdx.x] += sacc[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[i] = sacc[0];
}

}  // namespace

cudaError_t launch_emd_reset(int n, int* owner, int* assign, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_emd_reset<<<(2 * n + 255) / 256, 256, 0, st>>>(n, owner, assign);
    return cudaGetLastError();
}

cudaError_t launch_emd_round(int n_inst, int npix, const float* points, const float* targets, const int* n_targets,
                             const int* counts, int* owner, int* assign, float* price, unsigned long long* bids,
                             float eps, int* unassigned, cudaStream_t st) {
    const int n = n_inst * npix;
    if (n <= 0) return cudaSuccess;
    k_emd_bid<<<(2 * n * 32 + 255) / 256, 256, 0, st>>>(npix, points, targets, n_targets, counts, assign, price,
                                                        bids, eps, n, unassigned);
    k_emd_resolve<<<(n + 255) / 256, 256, 0, st>>>(n, owner, assign, price, bids);
    return cudaGetLastError();
}

cudaError_t launch_emd_loss(const InstDev* inst, int n_inst, int npix, const float* points, const float* targets,
                            const int* assign, const unsigned long long* keys, double* loss, float* dL_dx,
                            cudaStream_t st) {
    if (n_inst <= 0) return cudaSuccess;
    k_emd_loss<<<n_inst, 256, 0, st>>>(inst, npix, points, targets, assign, keys, loss, dL_dx);
    return cudaGetLastError();
}

}  // namespace mpm
