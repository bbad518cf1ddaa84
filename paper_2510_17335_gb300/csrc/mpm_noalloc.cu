// mpm_loss_mse_noalloc: the MSE loss of a point set against a target without
// any device allocation.
//
// Some callers cannot call cudaMalloc: a process whose device memory is all
// owned by another allocator (for instance a framework's caching allocator
// that reserved the GPU up front), or a control loop that must not take the
// implicit device synchronisation of an allocation. This entry point serves
// them. Its only scratch is the file-scope device array below, of a fixed
// size that every GPU loading the library holds until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mpm.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = MPM_NOALLOC_MAX_POINTS / kThreads;

struct LossScratch {
    double partial[kMaxBlocks];  // one FP64 partial sum per CTA
    double result;               // the reduced loss of the last call
    unsigned int ticket;         // CTAs finished; must be 0 when a call starts
};

// 128 KiB of partial sums plus the result and the ticket
static __device__ __align__(256) LossScratch g_loss_scratch;

// Each CTA sums its points' squared distances in FP64 and stores the sum in
// its slot; the CTA that finishes last adds the slots in index order (so the
// result does not depend on CTA scheduling), stores it and resets the ticket.
__global__ void __launch_bounds__(kThreads) k_loss_mse_noalloc(const float* __restrict__ x,
                                                               const float* __restrict__ target, long long n,
                                                               float* __restrict__ dldx, LossScratch* sc) {
    __shared__ double warp_sum[kThreads / 32];
    __shared__ bool last;
    const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
    double l = 0.0;
    if (p < n) {
        const float inv_n = 1.0f / float(n);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float d = x[3 * p + k] - target[3 * p + k];
            l += double(d) * double(d);
            if (dldx) dldx[3 * p + k] = 2.0f * d * inv_n;
        }
        l /= double(n);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; w++) s += warp_sum[w];
        sc->partial[blockIdx.x] = s;
        __threadfence();
        const unsigned int done = atomicAdd(&sc->ticket, 1u);
        last = (done == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (unsigned int b = 0; b < gridDim.x; b++) s += ((volatile double*)sc->partial)[b];
        sc->result = s;
        sc->ticket = 0u;
    }
}

// Device address of g_loss_scratch per device, looked up once per CUDA
// context: a device reset (cudaDeviceReset) destroys the context and the
// module with it, and the array of the next context may sit elsewhere, so
// the cache is keyed by the context's process-unique ID (cuCtxGetId, reached
// through the runtime's driver entry points: no link to the driver library).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

struct ScratchCache {
    bool valid = false;
    unsigned long long ctx_id = 0;
    LossScratch* addr = nullptr;
};

std::mutex g_mu;
ScratchCache g_cache[64];
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_entry_points_tried = false;

// ID of the current context (the primary context of the current device);
// called with g_mu held
int current_context_id(unsigned long long* id) {
    if (!g_entry_points_tried) {
        g_entry_points_tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return MPM_ERR_CUDA;
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return MPM_ERR_NO_DEVICE;
    if (g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return MPM_ERR_CUDA;
    return MPM_OK;
}

int scratch_address(LossScratch** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return MPM_ERR_NO_DEVICE;
    }
    // makes the device's primary context current if nothing has yet (since
    // CUDA 12 cudaSetDevice initialises the primary context)
    if (cudaSetDevice(dev) != cudaSuccess) {
        cudaGetLastError();
        return MPM_ERR_NO_DEVICE;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long id = 0;
    const int rc = current_context_id(&id);
    if (rc != MPM_OK) return rc;
    ScratchCache& c = g_cache[dev];
    if (!c.valid || c.ctx_id != id) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_loss_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return MPM_ERR_CUDA;
        }
        c.addr = static_cast<LossScratch*>(p);
        c.ctx_id = id;
        c.valid = true;
    }
    *out = c.addr;
    return MPM_OK;
}

}  // namespace

extern "C" int mpm_loss_mse_noalloc(const float* x, const float* x_target, int64_t n, float* dL_dx, double* loss,
                                    void* stream) {
    if (!x || !x_target || !loss || n < 0) return MPM_ERR_INVALID_ARG;
    if (n > MPM_NOALLOC_MAX_POINTS) return MPM_ERR_INVALID_ARG;
    if (n == 0) {
        *loss = 0.0;
        return MPM_OK;
    }
    LossScratch* sc = nullptr;
    const int rc = scratch_address(&sc);
    if (rc != MPM_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // a call that failed part-way could have left the ticket non-zero
    if (cudaMemsetAsync(&sc->ticket, 0, sizeof(unsigned int), s) != cudaSuccess) {
        cudaGetLastError();
        return MPM_ERR_CUDA;
    }
    const unsigned int blocks = (unsigned int)((n + kThreads - 1) / kThreads);
    k_loss_mse_noalloc<<<blocks, kThreads, 0, s>>>(x, x_target, (long long)n, dL_dx, sc);
    if (cudaGetLastError() != cudaSuccess) return MPM_ERR_CUDA;
    if (cudaMemcpyAsync(loss, &sc->result, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return MPM_ERR_CUDA;
    }
    return MPM_OK;
}
