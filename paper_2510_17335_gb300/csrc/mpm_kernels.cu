// Kernels of the MLS-MPM sand substep (Algorithm 1 of DDBot, arXiv
// 2510.17335) and of its adjoint, for sm_103a.
//
// Forward substep (4 launches, all instances of a batch in each):
//   k_p2g       particle: trial F, SVD, Drucker-Prager return, Kirchhoff
//               stress, APIC scatter of (m, mv) into the blocked grid; marks
//               grid blocks. Particles whose F is ill-conditioned for FP32
//               go to a list instead.
//   k_p2g_fp64  the listed particles with the constitutive step in FP64
//   k_grid      touched grid block (one warp): v = mv/m + dt g, walls,
//               shovel contact
//   k_g2p       particle: APIC gather of v and C, particle contact, advection
// Adjoint substep: k_g2p_bwd (scatter into the grid adjoint), k_grid_bwd,
// k_p2g_bwd (gather, constitutive adjoint, parameter sums; the same
// deferral), k_p2g_bwd_fp64, k_grid_clear. Inside a recorded segment the
// P2G adjoint of substep k and the G2P adjoint of substep k-1 run as one
// kernel (k_p2g_g2p_bwd + its FP64 fix-up), and k_grid_bwd clears the blocks
// of the substep reversed before it, so a substep takes 4 launches.
// The substep kernels use programmatic dependent launch (launch_pdl).
//
// The FP64 code lives only in the fix-up kernels, so that the register
// budget of the main particle kernels is set by the FP32 path.
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "mpm_device.cuh"
#include "mpm_launch.h"

// 1: the substep kernels use programmatic dependent launch (launch_pdl)
#ifndef MPM_PDL
#define MPM_PDL 1
#endif
// minimum resident CTAs per SM (register caps) of the adjoint kernels that
// run once per checkpoint segment; those of k_p2g, k_g2p and the fused
// adjoint are template parameters chosen per handle (LaunchShape)
#ifndef MPM_MINB_G2P_BWD
#define MPM_MINB_G2P_BWD 3
#endif
#ifndef MPM_MINB_P2G_BWD
#define MPM_MINB_P2G_BWD 3
#endif

namespace mpm {

__device__ __forceinline__ float ld(const float* s, long long ncap, int comp, long long p) {
    return __ldcs(s + comp * ncap + p);
}

// a[i] through selects: where a stencil loop over i stays rolled (the P2G
// scatter and the P2G adjoint's gather; unrolled they spill more and run
// slower), a runtime index would move the whole stencil into local memory
template <typename T>
__device__ __forceinline__ T sel3(const T (&a)[3], int i) {
    return i == 0 ? a[0] : (i == 1 ? a[1] : a[2]);
}

// The x-axis weights, weight derivatives and node offsets of a stencil as a
// small array that a rolled loop over i indexes at run time (it lives in
// local memory; the rest of the stencil stays in registers). Fully unrolled
// loops index it at compile time and keep it in registers.
struct AxisX {
    float w[3], dw[3];
    int o[3];
};

__device__ __forceinline__ AxisX axis_x(const Stencil& st, const int (&ox)[3]) {
    AxisX l;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        l.w[i] = st.w[0][i];
        l.dw[i] = st.dw[0][i];
        l.o[i] = ox[i];
    }
    return l;
}

// Copy the CTA's instance record into shared memory (all threads call it).
// Reads of its fields are then shared-memory loads; from global memory the
// compiler would have to reload them after every store of the kernel.
__device__ __forceinline__ const InstDev& stage_instance(InstDev& sI, const InstDev* inst, int i) {
    static_assert(sizeof(InstDev) % 4 == 0, "InstDev is copied as 32-bit words");
    constexpr int W = sizeof(InstDev) / 4;
    const int* src = reinterpret_cast<const int*>(inst + i);
    int* dst = reinterpret_cast<int*>(&sI);
    for (int k = threadIdx.x; k < W; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    return sI;
}

// mark the (up to 8) grid blocks a stencil touches
__device__ __forceinline__ void mark_blocks(const InstDev& I, const Stencil& st, int* flags, int n_blocks) {
    const int b0x = st.base[0] >> 2, b1x = (st.base[0] + 2) >> 2;
    const int b0y = st.base[1] >> 2, b1y = (st.base[1] + 2) >> 2;
    const int b0z = st.base[2] >> 2, b1z = (st.base[2] + 2) >> 2;
    for (int bx = b0x; bx <= b1x; bx++)
        for (int by = b0y; by <= b1y; by++)
            for (int bz = b0z; bz <= b1z; bz++)
                mark_block(flags, n_blocks, I.blk_off + (bx * I.nb[1] + by) * I.nb[2] + bz);
}

// f(gw) for every block of the touched-block list, one warp per entry. A
// warp's first entry is loaded together with the list length (both written
// by the kernels before), so that the two loads overlap; entries at or past
// the length are loaded only within the list's capacity and never used.
template <class Fn>
__device__ __forceinline__ void for_listed_blocks(const int* flags, int n_blocks, Fn&& f) {
    const int* list = flags + n_blocks + 1;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int gw = i < n_blocks ? list[i] : 0;
    const int n = flags[n_blocks];
    for (; i < n; i += nw) {
        f(gw);
        gw = i + nw < n ? list[i + nw] : 0;
    }
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_trial(const InstDev& I, const StepArgs& a, long long p, float (&C)[3][3],
                                           float (&Ft)[3][3]) {
    const long long N = a.ncap;
    float F[3][3];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            C[r][c] = ld(a.sin, N, kC + 3 * r + c, p);
            F[r][c] = ld(a.sin, N, kF + 3 * r + c, p);
        }
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++)
            Ft[r][c] = F[r][c] + I.dt * (C[r][0] * F[0][c] + C[r][1] * F[1][c] + C[r][2] * F[2][c]);
}

// The recorded SVD of a particle's trial F (record mode): the adjoint
// rebuilds the return mapping from it instead of redoing the SVD. U and V are
// proper rotations and are kept as unit quaternions (w, x, y, z).
// Rotation -> quaternion: the largest of 4w^2 = 1 + tr R, 4x^2 = 1 + R00 -
// R11 - R22, ... is taken by its square root, the other three from the sums
// and differences of symmetric off-diagonal pairs divided by it.
__device__ __forceinline__ void rot_to_quat(const float (&R)[3][3], float (&q)[4]) {
    const float tw = 1.0f + R[0][0] + R[1][1] + R[2][2];
    const float tx = 1.0f + R[0][0] - R[1][1] - R[2][2];
    const float ty = 1.0f - R[0][0] + R[1][1] - R[2][2];
    const float tz = 1.0f - R[0][0] - R[1][1] + R[2][2];
    const float a21 = R[2][1] - R[1][2], a02 = R[0][2] - R[2][0], a10 = R[1][0] - R[0][1];
    const float s01 = R[0][1] + R[1][0], s02 = R[0][2] + R[2][0], s12 = R[1][2] + R[2][1];
    const bool bw = tw >= tx && tw >= ty && tw >= tz;
    const bool bx = !bw && tx >= ty && tx >= tz;
    const bool by = !bw && !bx && ty >= tz;
    const float t = bw ? tw : (bx ? tx : (by ? ty : tz));
    const float r = 0.5f * rsqrtf(t);   // 1 / (2 sqrt t) = 1 / (4 q_big)
    const float big = t * r;            // sqrt(t) / 2 = q_big
    if (bw) { q[0] = big; q[1] = a21 * r; q[2] = a02 * r; q[3] = a10 * r; }
    else if (bx) { q[0] = a21 * r; q[1] = big; q[2] = s01 * r; q[3] = s02 * r; }
    else if (by) { q[0] = a02 * r; q[1] = s01 * r; q[2] = big; q[3] = s12 * r; }
    else { q[0] = a10 * r; q[1] = s02 * r; q[2] = s12 * r; q[3] = big; }
}

__device__ __forceinline__ void quat_to_rot(const float (&q)[4], float (&R)[3][3]) {
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    // normalise away the rounding of the stored quaternion
    const float n = rsqrtf(w * w + x * x + y * y + z * z);
    const float s = 2.0f * n * n;
    const float xx = s * x * x, yy = s * y * y, zz = s * z * z;
    const float xy = s * x * y, xz = s * x * z, yz = s * y * z;
    const float wx = s * w * x, wy = s * w * y, wz = s * w * z;
    R[0][0] = 1.0f - yy - zz; R[0][1] = xy - wz; R[0][2] = xz + wy;
    R[1][0] = xy + wz; R[1][1] = 1.0f - xx - zz; R[1][2] = yz - wx;
    R[2][0] = xz - wy; R[2][1] = yz + wx; R[2][2] = 1.0f - xx - yy;
}

__device__ __forceinline__ void store_svd(float* spec, long long N, long long p, const Spectral<float>& S) {
    float qu[4], qv[4];
    rot_to_quat(S.U, qu);
    rot_to_quat(S.V, qv);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        __stcs(spec + k * N + p, qu[k]);
        __stcs(spec + (4 + k) * N + p, qv[k]);
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        __stcs(spec + (8 + k) * N + p, S.s[k]);
        __stcs(spec + (11 + k) * N + p, S.h[k]);
    }
}

// the record's quaternions of U and V (qu, qv), the rotations and sigma,
// sigma^2 - 1
__device__ __forceinline__ void load_svd(const float* spec, long long N, long long p, Spectral<float>& S,
                                         float (&qu)[4], float (&qv)[4]) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
        qu[k] = __ldcs(spec + k * N + p);
        qv[k] = __ldcs(spec + (4 + k) * N + p);
    }
    quat_to_rot(qu, S.U);
    quat_to_rot(qv, S.V);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        S.s[k] = __ldcs(spec + (8 + k) * N + p);
        S.h[k] = __ldcs(spec + (11 + k) * N + p);
    }
}

// APIC + MLS stress transfer of one particle to its 27 nodes: mass m_p W and
// momentum W (m_p v + A d), A = stress_scale tau + m_p C. Sums in the shared
// tile when T is given and tiled, else with global atomics.
__device__ __forceinline__ void p2g_scatter(TileSmem* T, const InstDev& I, float4* grid, const Stencil& st,
                                            const float (&v)[3], const float (&A)[3][3]) {
    int ox[3], oy[3], oz[3];
    node_offsets(I, st, ox, oy, oz);
    float4* acc = grid + I.node_off;
#pragma unroll 1
    for (int i = 0; i < 3; i++) {
        const float dxi = (float(i) - st.fx[0]) * I.dx;
        float ai[3];   // m_p v + A d, hoisted over the loops
#pragma unroll
        for (int r = 0; r < 3; r++) ai[r] = fmaf(A[r][0], dxi, I.mp * v[r]);
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float dyj = (float(j) - st.fx[1]) * I.dx;
            const float wij = sel3(st.w[0], i) * st.w[1][j];
            float aij[3];
#pragma unroll
            for (int r = 0; r < 3; r++) aij[r] = fmaf(A[r][1], dyj, ai[r]);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float dzk = (float(k) - st.fx[2]) * I.dx;
                const float W = wij * st.w[2][k];
                float4 val;
                val.x = W * I.mp;
                val.y = W * fmaf(A[0][2], dzk, aij[0]);
                val.z = W * fmaf(A[1][2], dzk, aij[1]);
                val.w = W * fmaf(A[2][2], dzk, aij[2]);
                if (T) tile_add(*T, acc, sel3(ox, i) + oy[j] + oz[k], st, i, j, k, val, 4);
                else atomicAdd(acc + sel3(ox, i) + oy[j] + oz[k], val);
            }
        }
    }
}

// stores F' = Fn and the affine matrix of the transfer
__device__ __forceinline__ void p2g_store_affine(const InstDev& I, const StepArgs& a, long long p,
                                                 const float (&Fn)[3][3], const float (&tau)[3][3],
                                                 const float (&C)[3][3], float (&A)[3][3]) {
    const long long N = a.ncap;
    bool finite = true;
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            __stcs(a.sout + (kF + 3 * r + c) * N + p, Fn[r][c]);
            finite = finite && isfinite(Fn[r][c]);
            A[r][c] = I.stress_scale * tau[r][c] + I.mp * C[r][c];
        }
    if (!finite) atomicOr(a.status, kStatusNonFinite);
}

// P2G with the constitutive step, FP32. A particle whose deformation is
// ill-conditioned for FP32 (see needs_fp64) is listed for k_p2g_fp64, which
// does its constitutive step and transfer.
template <int MINB>
__global__ void __launch_bounds__(kChunk, MINB) k_p2g(StepArgs a) {
    wait_previous_grid();
    __shared__ TileSmem T;
    __shared__ InstDev sI;
    const int inst = a.chunk_inst[blockIdx.x];
    const InstDev& I = stage_instance(sI, a.inst, inst);
    const long long p = (long long)blockIdx.x * kChunk + threadIdx.x;
    const bool active = p - I.pbeg < I.n;
    const long long N = a.ncap;
    float x[3] = {0.5f, 0.5f, 0.5f};
    if (active) {
#pragma unroll
        for (int k = 0; k < 3; k++) x[k] = ld(a.sin, N, kX + k, p);
    }
    Stencil st;
    const bool inside = make_stencil(I, x, st);
    if (active && !inside) atomicOr(a.status, kStatusDomain);
    if (a.tile) tile_begin(T, active, st, kChunk);
    else if (threadIdx.x == 0) T.tiled = 0;
    if (!a.tile) __syncthreads();
    if (active) {
        float v[3], C[3][3], Ft[3][3];
#pragma unroll
        for (int k = 0; k < 3; k++) v[k] = ld(a.sin, N, kV + k, p);
        load_trial(I, a, p, C, Ft);
        Spectral<float> S;
        constitutive_spectral<float>(Ft, I.mu, I.lam, I.beta, I.smin, S);
        if (a.spec) store_svd(a.spec, N, p, S);
        if (needs_fp64(S)) {
            a.fb_list[atomicAdd(a.fb_count, 1)] = (int)p;
        } else {
            float Fn[3][3], tau[3][3], A[3][3];
            spectral_outputs<float, float>(S, Fn, tau);
            p2g_store_affine(I, a, p, Fn, tau, C, A);
            p2g_scatter(&T, I, a.acc, st, v, A);
            if (!T.tiled) mark_blocks(I, st, a.flags, a.n_blocks);
        }
    }
    tile_flush(T, I, a.acc, a.flags, a.n_blocks, kChunk);
}

// Deferred-list bookkeeping of the FP64 fix-up kernels: every CTA reads the
// count, and the last CTA to finish zeroes the count and the ticket for the
// next launch (stream order keeps the next producer behind it). With an
// empty list (the usual case) no CTA takes a ticket: all read the same zero.
__device__ __forceinline__ int fb_begin(const int* fb_count, int* scount) {
    if (threadIdx.x == 0) *scount = *(volatile const int*)fb_count;
    __syncthreads();
    return *scount;
}

__device__ __forceinline__ void fb_end(int* fb_count, int count) {
    if (count == 0) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(fb_count + 1, 1) == (int)gridDim.x - 1) {
            fb_count[0] = 0;
            fb_count[1] = 0;
        }
    }
}

// The particles k_p2g listed: constitutive step in FP64, transfer with
// global atomics.
__global__ void __launch_bounds__(kFp64Threads) k_p2g_fp64(StepArgs a) {
    wait_previous_grid();
    __shared__ int scount;
    const int count = fb_begin(a.fb_count, &scount);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const long long p = a.fb_list[i];
        const InstDev& I = a.inst[a.chunk_inst[p / kChunk]];
        const long long N = a.ncap;
        float x[3], v[3], C[3][3], Ft[3][3], Fn[3][3], tau[3][3], A[3][3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            x[k] = ld(a.sin, N, kX + k, p);
            v[k] = ld(a.sin, N, kV + k, p);
        }
        Stencil st;
        make_stencil(I, x, st);
        load_trial(I, a, p, C, Ft);
        constitutive_fp64(Ft, I.mu, I.lam, I.beta, I.smin, Fn, tau);
        p2g_store_affine(I, a, p, Fn, tau, C, A);
        p2g_scatter(nullptr, I, a.acc, st, v, A);
        mark_blocks(I, st, a.flags, a.n_blocks);
        atomicAdd(a.fp64_count, 1ull);
    }
    fb_end(a.fb_count, count);
}

// velocity update of one node (gravity, walls); returns false for empty nodes
__device__ __forceinline__ void grid_node(const InstDev& I, const Pose& P, float cs, float sn, int ix, int iy, int iz,
                                          float4 acc, float (&vg)[3], float (&mask)[3]) {
    const float inv_m = 1.0f / acc.x;
    vg[0] = acc.y * inv_m + I.dt * I.g[0];
    vg[1] = acc.z * inv_m + I.dt * I.g[1];
    vg[2] = acc.w * inv_m + I.dt * I.g[2];
    const int idx[3] = {ix, iy, iz};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        mask[d] = 1.0f;
        if (idx[d] < I.bound && vg[d] < 0.0f) { vg[d] = 0.0f; mask[d] = 0.0f; }
        if (idx[d] > I.res[d] - I.bound && vg[d] > 0.0f) { vg[d] = 0.0f; mask[d] = 0.0f; }
    }
}

// grid update of one touched block gw (one warp, two nodes a lane)
__device__ __forceinline__ void grid_block(const StepArgs& a, int gw, int lane) {
    const int inst = a.block_inst[gw];
    const InstDev& I = a.inst[inst];
    const int lb = gw - I.blk_off;
    const int bz = lb % I.nb[2], by = (lb / I.nb[2]) % I.nb[1], bx = lb / (I.nb[1] * I.nb[2]);
    const Pose P = load_pose(I, a.substep);
    float sn, cs;
    sincosf(P.psi, &sn, &cs);
    const long long base = I.node_off + (long long)lb * 64;
    float m = 0.0f;   // the block's mass (FP32 within the block, FP64 across blocks)
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int nd = lane + 32 * h;
        const int ix = bx * 4 + (nd >> 4), iy = by * 4 + ((nd >> 2) & 3), iz = bz * 4 + (nd & 3);
        const float4 acc = a.acc[base + nd];
        float4 out = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (acc.x > 0.0f) {
            float vg[3], mask[3];
            grid_node(I, P, cs, sn, ix, iy, iz, acc, vg, mask);
            if (I.shovel_on) {
                const float q[3] = {ix * I.dx, iy * I.dx, iz * I.dx};
                shovel_project(I, P, cs, sn, q, vg);
            }
            out = make_float4(vg[0], vg[1], vg[2], acc.x);
        }
        a.vout[base + nd] = out;
        if (!a.keep_grid) a.acc[base + nd] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        m += acc.x;
    }
    if (a.mass) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m += __shfl_down_sync(0xffffffffu, m, o);
        if (lane == 0) atomicAdd(a.mass + inst, (double)m);
    }
    if (!a.keep_grid && lane == 0) a.flags[gw] = 0;
}

__global__ void __launch_bounds__(256) k_grid(StepArgs a) {
    wait_previous_grid();
    const int lane = threadIdx.x & 31;
    for_listed_blocks(a.flags, a.n_blocks, [&](int gw) { grid_block(a, gw, lane); });
}

// Run by the G2P of the same substep, which follows the grid update in stream
// order: the grid update's mass sums become the totals, and without kept
// grids the block list is emptied for the next substep (the grid update has
// zeroed every listed flag).
__device__ __forceinline__ void grid_epilogue(const StepArgs& a) {
    if (blockIdx.x != 0) return;
    if (a.mass)
        for (int i = threadIdx.x; i < a.n_inst; i += blockDim.x) {
            a.mass[a.n_inst + i] = a.mass[i];
            a.mass[i] = 0.0;
        }
    if (!a.keep_grid && threadIdx.x == 0) a.flags[a.n_blocks] = 0;
}

// The 27 nodes of a particle's stencil in the global grid.
struct GlobalNodes {
    const float4* g;      // the instance's grid
    int ox[3], oy[3], oz[3];
    __device__ __forceinline__ GlobalNodes(const InstDev& I, const Stencil& st, const float4* grid)
        : g(grid + I.node_off) {
        node_offsets(I, st, ox, oy, oz);
    }
    __device__ __forceinline__ float4 node(int i, int j, int k) const {
        return __ldg(g + sel3(ox, i) + oy[j] + oz[k]);
    }
};

// v = sum W v_node and B = sum W v_node (o - f)^T, summed over k first:
// T0 = sum_k wz v_node, T1 = sum_k wz (k - fz) v_node per (i, j)
template <class Nodes>
__device__ __forceinline__ void g2p_gather(const Stencil& st, const Nodes& src, float (&v)[3], float (&B)[3][3]) {
#pragma unroll
    for (int r = 0; r < 3; r++) {
        v[r] = 0.f;
        B[r][0] = B[r][1] = B[r][2] = 0.f;
    }
    float wzd[3];
#pragma unroll
    for (int k = 0; k < 3; k++) wzd[k] = st.w[2][k] * (float(k) - st.fx[2]);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float di = float(i) - st.fx[0];
        const float wx = sel3(st.w[0], i);
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float dj = float(j) - st.fx[1];
            float T0[3] = {0.f, 0.f, 0.f}, T1[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float4 g = src.node(i, j, k);
                const float gg[3] = {g.x, g.y, g.z};
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    T0[r] = fmaf(st.w[2][k], gg[r], T0[r]);
                    T1[r] = fmaf(wzd[k], gg[r], T1[r]);
                }
            }
            const float wxy = wx * st.w[1][j], wxyi = wxy * di, wxyj = wxy * dj;
#pragma unroll
            for (int r = 0; r < 3; r++) {
                v[r] = fmaf(wxy, T0[r], v[r]);
                B[r][0] = fmaf(wxyi, T0[r], B[r][0]);
                B[r][1] = fmaf(wxyj, T0[r], B[r][1]);
                B[r][2] = fmaf(wxy, T1[r], B[r][2]);
            }
        }
    }
}

// G2P of one particle (Algorithm 1: gather of v and C, particle contact,
// advection) into x, v, C of a.sout; returns them in xn, v, C as well.
__device__ __forceinline__ void g2p_particle(const InstDev& I, const StepArgs& a, long long p, float (&xn)[3],
                                             float (&v)[3], float (&C)[3][3]) {
    const long long N = a.ncap;
    float x[3];
#pragma unroll
    for (int k = 0; k < 3; k++) x[k] = ld(a.sin, N, kX + k, p);
    Stencil st;
    make_stencil(I, x, st);
    float B[3][3];
    g2p_gather(st, GlobalNodes(I, st, a.vout), v, B);
    if (I.pcoll && I.shovel_on) {
        const Pose P = load_pose(I, a.substep);
        float sn, cs;
        sincosf(P.psi, &sn, &cs);
        shovel_project(I, P, cs, sn, x, v);
    }
    bool finite = true;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        xn[k] = x[k] + I.dt * v[k];
        finite = finite && isfinite(xn[k]);
    }
    bool inside = true;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float X = xn[k] * I.inv_dx;
        inside = inside && (X >= 1.0f) && (X < float(I.res[k] - 2));
    }
    if (!finite) atomicOr(a.status, kStatusNonFinite);
    if (!inside) atomicOr(a.status, kStatusDomain);
    // C = 4/dx^2 sum W v d^T with d = (o - f) dx
    const float cscale = 4.0f * I.inv_dx;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        __stcs(a.sout + (kX + k) * N + p, xn[k]);
        __stcs(a.sout + (kV + k) * N + p, v[k]);
    }
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            C[r][c] = cscale * B[r][c];
            __stcs(a.sout + (kC + 3 * r + c) * N + p, C[r][c]);
        }
}

template <int MINB>
__global__ void __launch_bounds__(kChunk, MINB) k_g2p(StepArgs a) {
    wait_previous_grid();
    __shared__ InstDev sI;
    const int inst = a.chunk_inst[blockIdx.x];
    grid_epilogue(a);
    const InstDev& I = stage_instance(sI, a.inst, inst);
    const long long p = (long long)blockIdx.x * kChunk + threadIdx.x;
    if (p - I.pbeg >= I.n) return;
    float xn[3], v[3], C[3][3];
    g2p_particle(I, a, p, xn, v, C);
}


// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
// Adjoint of the APIC gather for one particle: scatter W b into the grid
// velocity adjoint with b = gvn + kap gC d (hoisted over the loops), and
// gx += sum Wbar grad W (Wbar = v_node . b); the terms of gx through d sum
// to -kap gC^T Sv with Sv = sum W v_node (velocities of the grid vg). The
// sums of Wbar run over k first (per (i, j): Pw = sum_k wz Wbar, Pd =
// sum_k wz' Wbar). KnownSv: the caller passes Sv, the particle's gathered
// velocity, which the forward stored as the next state's v wherever the
// particle contact left it alone; else Sv is summed here.
template <bool KnownSv>
__device__ __forceinline__ void g2p_bwd_scatter(const InstDev& I, const AdjArgs& A, const Stencil& st,
                                                const int (&ox)[3], const int (&oy)[3], const int (&oz)[3],
                                                const float4* vg, TileSmem* T, const float (&gvn)[3],
                                                const float (&gC)[3][3], float (&gx)[3], const float (&Sv_in)[3]) {
    const float kap = 4.0f * I.inv_dx * I.inv_dx;
    float kgC[3][3];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) kgC[r][c] = kap * gC[r][c];
    float Sv[3] = {0.f, 0.f, 0.f};
    float4* ga = A.gacc + I.node_off;
    const AxisX lx = axis_x(st, ox);
    float dz[3];
#pragma unroll
    for (int k = 0; k < 3; k++) dz[k] = (float(k) - st.fx[2]) * I.dx;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float wx = lx.w[i], dwx = lx.dw[i], dxi = (float(i) - st.fx[0]) * I.dx;
        float bi[3];
#pragma unroll
        for (int r = 0; r < 3; r++) bi[r] = fmaf(kgC[r][0], dxi, gvn[r]);
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float wy = st.w[1][j], dyj = (float(j) - st.fx[1]) * I.dx;
            const float wxy = wx * wy;
            float bij[3];
#pragma unroll
            for (int r = 0; r < 3; r++) bij[r] = fmaf(kgC[r][1], dyj, bi[r]);
            float Pw = 0.f, Pd = 0.f, Tv[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float wz = st.w[2][k];
                const float W = wxy * wz;
                const float4 g = __ldg(vg + lx.o[i] + oy[j] + oz[k]);
                float b[3];
#pragma unroll
                for (int r = 0; r < 3; r++) b[r] = fmaf(kgC[r][2], dz[k], bij[r]);
                const float4 contrib = make_float4(W * b[0], W * b[1], W * b[2], 0.f);
                if (T) tile_add(*T, ga, lx.o[i] + oy[j] + oz[k], st, i, j, k, contrib, 3);
                else atomicAdd(ga + lx.o[i] + oy[j] + oz[k], contrib);
                const float Wbar = g.x * b[0] + g.y * b[1] + g.z * b[2];
                Pw = fmaf(wz, Wbar, Pw);
                Pd = fmaf(st.dw[2][k], Wbar, Pd);
                if (!KnownSv) {
                    Tv[0] = fmaf(wz, g.x, Tv[0]);
                    Tv[1] = fmaf(wz, g.y, Tv[1]);
                    Tv[2] = fmaf(wz, g.z, Tv[2]);
                }
            }
            gx[0] = fmaf(dwx * wy, Pw, gx[0]);
            gx[1] = fmaf(wx * st.dw[1][j], Pw, gx[1]);
            gx[2] = fmaf(wxy, Pd, gx[2]);
            if (!KnownSv) {
#pragma unroll
                for (int r = 0; r < 3; r++) Sv[r] = fmaf(wxy, Tv[r], Sv[r]);
            }
        }
    }
    if (KnownSv) {
#pragma unroll
        for (int r = 0; r < 3; r++) Sv[r] = Sv_in[r];
    }
#pragma unroll
    for (int c = 0; c < 3; c++) gx[c] -= kgC[0][c] * Sv[0] + kgC[1][c] * Sv[1] + kgC[2][c] * Sv[2];
}

// Tiled: with the shared-memory scatter tile (option tile_scatter, launched
// with sizeof(TileSmem) bytes of dynamic shared memory); the plain
// instantiation carries neither its code nor its memory.
template <bool Tiled>
__global__ void __launch_bounds__(kChunk, MPM_MINB_G2P_BWD) k_g2p_bwd(AdjArgs A) {
    wait_previous_grid();
    extern __shared__ __align__(16) unsigned char s_tile[];
    __shared__ InstDev sI;
    __shared__ float sfac[2];
    const StepArgs& a = A.f;
    TileSmem* T = Tiled ? reinterpret_cast<TileSmem*>(s_tile) : nullptr;
    const int inst = a.chunk_inst[blockIdx.x];
    if (A.gscale && threadIdx.x == 0) {
        // regularisers of the x and v adjoints of state k+1 (Sec. III-E)
        sfac[0] = (float)reg_factor(A.gscale, A.pstat_in[3 * inst + 0], A.oom, A.gdelta);
        sfac[1] = (float)reg_factor(A.gscale, A.pstat_in[3 * inst + 1], A.oom, A.gdelta);
    }
    const InstDev& I = stage_instance(sI, a.inst, inst);
    const long long p = (long long)blockIdx.x * kChunk + threadIdx.x;
    const bool active = p - I.pbeg < I.n;
    const long long N = a.ncap;
    float x[3] = {0.5f, 0.5f, 0.5f};
    if (active) {
#pragma unroll
        for (int k = 0; k < 3; k++) x[k] = ld(a.sin, N, kX + k, p);
    }
    Stencil st;
    make_stencil(I, x, st);
    if (Tiled) tile_begin(*T, active, st, kChunk);
    int ox[3], oy[3], oz[3];
    node_offsets(I, st, ox, oy, oz);
    const float4* vg = a.vout + I.node_off;
    float gx[3] = {0.f, 0.f, 0.f}, gvn[3] = {0.f, 0.f, 0.f};
    if (active) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            gx[k] = A.adj[(kX + k) * N + p];
            float gv = A.adj[(kV + k) * N + p];
            if (a.clip > 0.f) { gx[k] = clipf(gx[k], a.clip); gv = clipf(gv, a.clip); }
            if (A.gscale) { gx[k] *= sfac[0]; gv *= sfac[1]; }
            // adjoint of the advection x' = x + dt v'
            gvn[k] = gv + I.dt * gx[k];
        }
    }
    if (I.pcoll && I.shovel_on) {   // uniform over the CTA
        // Particle-level shovel contact. Outside the shovel it is the
        // identity; inside, its adjoint needs the pre-contact G2P velocity,
        // gathered again here for those particles only.
        float gp[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bool contact = false;
        if (active) {
            const Pose P = load_pose(I, a.substep);
            float sn, cs, n[3], nl[3];
            sincosf(P.psi, &sn, &cs);
            if (shovel_inside(I, P, cs, sn, x, n, nl)) {
                contact = true;
                float v[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int j = 0; j < 3; j++)
#pragma unroll
                        for (int k = 0; k < 3; k++) {
                            const float W = st.w[0][i] * st.w[1][j] * st.w[2][k];
                            const float4 g = __ldg(vg + ox[i] + oy[j] + oz[k]);
                            v[0] += W * g.x; v[1] += W * g.y; v[2] += W * g.z;
                        }
                float g0[3] = {gvn[0], gvn[1], gvn[2]}, gq[3] = {0.f, 0.f, 0.f};
                gvn[0] = gvn[1] = gvn[2] = 0.f;
                shovel_project_adj(I, P, cs, sn, x, v, g0, gvn, gq, gp);
                gx[0] += gq[0]; gx[1] += gq[1]; gx[2] += gq[2];
            }
        }
        warp_reduce_add<8>(gp, A.gpose + 8 * inst, contact);
    }
    if (active) {
        float gC[3][3];
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int c = 0; c < 3; c++) gC[r][c] = A.adj[(kC + 3 * r + c) * N + p];
        const float none[3] = {0.f, 0.f, 0.f};
        g2p_bwd_scatter<false>(I, A, st, ox, oy, oz, vg, T, gvn, gC, gx, none);
#pragma unroll
        for (int k = 0; k < 3; k++) A.adj[(kX + k) * N + p] = gx[k];
    }
    if (Tiled) tile_flush(*T, I, A.gacc, nullptr, 0, kChunk);
}

// adjoint of the grid update of one touched block gw (one warp)
__device__ __forceinline__ void grid_bwd_block(const AdjArgs& A, int gw, int lane) {
    const StepArgs& a = A.f;
    const int inst = a.block_inst[gw];
    const InstDev& I = a.inst[inst];
    const int lb = gw - I.blk_off;
    const int bz = lb % I.nb[2], by = (lb / I.nb[2]) % I.nb[1], bx = lb / (I.nb[1] * I.nb[2]);
    const Pose P = load_pose(I, a.substep);
    float sn, cs;
    sincosf(P.psi, &sn, &cs);
    const long long base = I.node_off + (long long)lb * 64;
    float gp[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float st[3] = {0.f, 0.f, 0.f};   // statistics of v-bar after / before the contact and of m-bar
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int nd = lane + 32 * h;
        const int ix = bx * 4 + (nd >> 4), iy = by * 4 + ((nd >> 2) & 3), iz = bz * 4 + (nd & 3);
        const float4 acc = a.acc[base + nd];
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (acc.x > 0.f) {
            const float4 gin = A.gacc[base + nd];
            float g[3] = {gin.x, gin.y, gin.z};
            if (a.clip > 0.f) {
#pragma unroll
                for (int d = 0; d < 3; d++) g[d] = clipf(g[d], a.clip);
            }
            float vg[3], mask[3];
            grid_node(I, P, cs, sn, ix, iy, iz, acc, vg, mask);
            float gv[3] = {0.f, 0.f, 0.f};
            if (I.shovel_on) {
                const float q[3] = {ix * I.dx, iy * I.dx, iz * I.dx};
                float gq[3] = {0.f, 0.f, 0.f};
                shovel_project_adj(I, P, cs, sn, q, vg, g, gv, gq, gp);
            } else {
                gv[0] = g[0]; gv[1] = g[1]; gv[2] = g[2];
            }
            const float inv_m = 1.0f / acc.x;
            float dot = 0.f;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                gv[d] *= mask[d];
                if (a.clip > 0.f) gv[d] = clipf(gv[d], a.clip);
            }
            dot = gv[0] * acc.y + gv[1] * acc.z + gv[2] * acc.w;
            float gm = -dot * inv_m * inv_m;
            if (a.clip > 0.f) gm = clipf(gm, a.clip);
            if (A.gscale) {
                // unregularised values; the P2G adjoint applies the factors
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const float s0 = stat_of(A.gscale, g[d]), s1 = stat_of(A.gscale, gv[d]);
                    st[0] = A.gscale == 1 ? fmaxf(st[0], s0) : st[0] + s0;
                    st[1] = A.gscale == 1 ? fmaxf(st[1], s1) : st[1] + s1;
                }
                const float s2 = stat_of(A.gscale, gm);
                st[2] = A.gscale == 1 ? fmaxf(st[2], s2) : st[2] + s2;
            }
            out = make_float4(gm, gv[0] * inv_m, gv[1] * inv_m, gv[2] * inv_m);
        }
        A.gacc[base + nd] = out;
    }
    if (A.gscale) warp_stat<3>(A.gscale, st, A.gstat + 3 * inst);
    if (I.shovel_on) {
        // warp sum of the pose adjoint in FP64, one atomic per value and warp
        // (unregularised into gpose_raw when regularising: the host scales it)
        double* dst = A.gscale ? A.gpose_raw : A.gpose;
        bool any = false;
#pragma unroll
        for (int k = 0; k < 8; k++) any = any || (gp[k] != 0.f);
        if (__any_sync(0xffffffffu, any)) {
#pragma unroll
            for (int k = 0; k < 8; k++) {
                float x = gp[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
                if (lane == 0 && x != 0.f) atomicAdd(dst + 8 * inst + k, (double)x);
            }
        }
    }
}

// zero one touched block's accumulators (and grid adjoints) and its flag
__device__ __forceinline__ void clear_block(const StepArgs& a, int* flags, float4* acc, float4* gacc, int gw,
                                            int lane) {
    const InstDev& I = a.inst[a.block_inst[gw]];
    const long long base = I.node_off + (long long)(gw - I.blk_off) * 64;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gacc) {
        gacc[base + lane] = z;
        gacc[base + lane + 32] = z;
    }
    acc[base + lane] = z;
    acc[base + lane + 32] = z;
    if (lane == 0) flags[gw] = 0;
}

__global__ void __launch_bounds__(256) k_grid_bwd(AdjArgs A) {
    wait_previous_grid();
    const StepArgs& a = A.f;
    const int lane = threadIdx.x & 31;
    for_listed_blocks(a.flags, a.n_blocks, [&](int gw) { grid_bwd_block(A, gw, lane); });
    if (A.clr_flags)
        for_listed_blocks(A.clr_flags, a.n_blocks,
                          [&](int gw) { clear_block(a, A.clr_flags, A.clr_acc, A.clr_gacc, gw, lane); });
}

// Spectral data parked in shared memory across the gather (14 words a
// thread): the record as loaded (U and V as quaternions, sigma, sigma^2 - 1);
// unpark rebuilds U and V and redoes the return mapping from the same
// values (cheaper than parking its 23 results, whose shared memory the
// unified L1 keeps).
constexpr int kParked = 14;

__device__ __forceinline__ void park(volatile float* sS, const float (&qu)[4], const float (&qv)[4],
                                     const Spectral<float>& S) {
    const int t = threadIdx.x;
    int w = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        sS[(w++) * kChunk + t] = qu[k];
        sS[(w++) * kChunk + t] = qv[k];
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        sS[(w++) * kChunk + t] = S.s[k];
        sS[(w++) * kChunk + t] = S.h[k];
    }
}

__device__ __forceinline__ void unpark(const volatile float* sS, Spectral<float>& S, const InstDev& I) {
    const int t = threadIdx.x;
    int w = 0;
    float qu[4], qv[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        qu[k] = sS[(w++) * kChunk + t];
        qv[k] = sS[(w++) * kChunk + t];
    }
    quat_to_rot(qu, S.U);
    quat_to_rot(qv, S.V);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        S.s[k] = sS[(w++) * kChunk + t];
        S.h[k] = sS[(w++) * kChunk + t];
    }
    return_map<float>(S, I.mu, I.lam, I.beta, I.smin);
}

// a load the compiler may not merge with an earlier one (re-reading is
// cheaper than keeping the value live across the gather)
__device__ __forceinline__ float ld_again(const float* p) {
    float v;
    asm volatile("ld.global.cs.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// The gather half of the P2G adjoint for one particle: from the grid
// adjoint (m-bar, mv-bar) at the 27 nodes to gx (added), gv, the adjoint gA of
// the affine matrix A = stress_scale tau + m_p C, and gmp (added).
__device__ __forceinline__ void p2g_bwd_gather(const InstDev& I, const AdjArgs& A, const float (&x)[3],
                                               const float (&v)[3], const float (&Am)[3][3], float fm, float fv,
                                               float (&gx)[3], float (&gv)[3], float (&gA)[3][3], float& gmp) {
    Stencil st;
    make_stencil(I, x, st);
    int ox[3], oy[3], oz[3];
    node_offsets(I, st, ox, oy, oz);
    const float4* ga = A.gacc + I.node_off;
    const AxisX lx = axis_x(st, ox);
    // Per node: a = m_p v + Am d (hoisted over the loops), Wbar = m-bar m_p +
    // mv-bar . a, gx += Wbar grad W, gA += W mv-bar d^T. The terms of gx
    // through d = x_node - x_p sum to -Am^T S1 with S1 = sum W mv-bar, and
    // gv, gmp follow from S1 and S0 = sum W m-bar after the loop. The grid
    // holds m-bar / fm and mv-bar / fv (fm = fv = 1 unless regularising).
    // W and grad W factor per axis, so every sum runs over k first: per
    // (i, j) Pw = sum_k wz Wbar, Pd = sum_k wz' Wbar, Tm = sum_k wz m-bar,
    // T0 = sum_k wz mv-bar, T1 = sum_k wz dz mv-bar, then weighted by the
    // x and y factors.
    float S0 = 0.f, S1[3] = {0.f, 0.f, 0.f};
    const float mpf = I.mp * fm;
    float dz[3], wzd[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        dz[k] = (float(k) - st.fx[2]) * I.dx;
        wzd[k] = st.w[2][k] * dz[k];
    }
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) gA[r][c] = 0.f;
#pragma unroll 1
    for (int i = 0; i < 3; i++) {
        const float wx = lx.w[i], dwx = lx.dw[i], dxi = (float(i) - st.fx[0]) * I.dx;
        float ai[3];
#pragma unroll
        for (int r = 0; r < 3; r++) ai[r] = fmaf(Am[r][0], dxi, I.mp * v[r]);
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float dyj = (float(j) - st.fx[1]) * I.dx;
            float aij[3];
#pragma unroll
            for (int r = 0; r < 3; r++) aij[r] = fmaf(Am[r][1], dyj, ai[r]);
            float Pw = 0.f, Pd = 0.f, Tm = 0.f, T0[3] = {0.f, 0.f, 0.f}, T1[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float4 g = ga[lx.o[i] + oy[j] + oz[k]];
                const float gmv[3] = {g.y, g.z, g.w};
                float ma = 0.f;
#pragma unroll
                for (int r = 0; r < 3; r++) ma = fmaf(gmv[r], fmaf(Am[r][2], dz[k], aij[r]), ma);
                const float Wbar = fmaf(mpf, g.x, fv * ma);
                Pw = fmaf(st.w[2][k], Wbar, Pw);
                Pd = fmaf(st.dw[2][k], Wbar, Pd);
                Tm = fmaf(st.w[2][k], g.x, Tm);
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    T0[r] = fmaf(st.w[2][k], gmv[r], T0[r]);
                    T1[r] = fmaf(wzd[k], gmv[r], T1[r]);
                }
            }
            const float wy = st.w[1][j], wxy = wx * wy, wxyi = wxy * dxi, wxyj = wxy * dyj;
            gx[0] = fmaf(dwx * wy, Pw, gx[0]);
            gx[1] = fmaf(wx * st.dw[1][j], Pw, gx[1]);
            gx[2] = fmaf(wxy, Pd, gx[2]);
            S0 = fmaf(wxy, Tm, S0);
#pragma unroll
            for (int r = 0; r < 3; r++) {
                S1[r] = fmaf(wxy, T0[r], S1[r]);
                gA[r][0] = fmaf(wxyi, T0[r], gA[r][0]);
                gA[r][1] = fmaf(wxyj, T0[r], gA[r][1]);
                gA[r][2] = fmaf(wxy, T1[r], gA[r][2]);
            }
        }
    }
    S0 *= fm;
#pragma unroll
    for (int r = 0; r < 3; r++) {
        S1[r] *= fv;
#pragma unroll
        for (int c = 0; c < 3; c++) gA[r][c] *= fv;
    }
    gmp += S0 + S1[0] * v[0] + S1[1] * v[1] + S1[2] * v[2];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        gv[c] = I.mp * S1[c];
        gx[c] -= Am[0][c] * S1[0] + Am[1][c] * S1[1] + Am[2][c] * S1[2];
    }
}

// The chain through the trial F = (I + dt C) F and the stores of the
// adjoint of state k (in place of the adjoint of state k+1).
// (Store: every component of the adjoint of state k, or, when the caller
// goes on with the G2P adjoint of the substep before, F-bar only; gC leaves
// with the chain term added.)
template <bool Store = true>
__device__ __forceinline__ void p2g_bwd_finish(const InstDev& I, const AdjArgs& A, long long p, const float (&gx)[3],
                                               const float (&gv)[3], float (&gC)[3][3], const float (&gFt)[3][3],
                                               int mode, float (&st)[3]) {
    const StepArgs& a = A.f;
    const long long N = a.ncap;
    float C[3][3], F[3][3];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            C[r][c] = ld_again(a.sin + (kC + 3 * r + c) * N + p);
            F[r][c] = ld_again(a.sin + (kF + 3 * r + c) * N + p);
        }
    float gF[3][3];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            gF[r][c] = gFt[r][c] + I.dt * (C[0][r] * gFt[0][c] + C[1][r] * gFt[1][c] + C[2][r] * gFt[2][c]);
            gC[r][c] += I.dt * (gFt[r][0] * F[c][0] + gFt[r][1] * F[c][1] + gFt[r][2] * F[c][2]);
        }
    bool finite = true;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (Store) {
            A.adj[(kX + k) * N + p] = gx[k];
            A.adj[(kV + k) * N + p] = gv[k];
        }
        finite = finite && isfinite(gx[k]) && isfinite(gv[k]);
        if (mode) {
            const float sx = stat_of(mode, gx[k]), sv = stat_of(mode, gv[k]);
            st[0] = mode == 1 ? fmaxf(st[0], sx) : st[0] + sx;
            st[1] = mode == 1 ? fmaxf(st[1], sv) : st[1] + sv;
        }
    }
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            if (Store) A.adj[(kC + 3 * r + c) * N + p] = gC[r][c];
            A.adj[(kF + 3 * r + c) * N + p] = gF[r][c];
            finite = finite && isfinite(gF[r][c]) && isfinite(gC[r][c]);
            if (mode) {
                const float sF = stat_of(mode, gF[r][c]);
                st[2] = mode == 1 ? fmaxf(st[2], sF) : st[2] + sF;
            }
        }
    if (!finite) atomicOr(a.status, kStatusNonFinite);
}

// gtau, gC (the affine part), gmp (the A : C part) and the clipped adjoint of F'
__device__ __forceinline__ void p2g_bwd_affine(const InstDev& I, const AdjArgs& A, long long p, const float (&gA)[3][3],
                                               float fF, float (&gFn)[3][3], float (&gtau)[3][3], float (&gC)[3][3],
                                               float& gmp) {
    const StepArgs& a = A.f;
    const long long N = a.ncap;
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float g = ld_again(A.adj + (kF + 3 * r + c) * N + p);
            gFn[r][c] = (a.clip > 0.f ? clipf(g, a.clip) : g) * fF;
            gtau[r][c] = I.stress_scale * gA[r][c];
            gC[r][c] = I.mp * gA[r][c];
            gmp += gA[r][c] * ld_again(a.sin + (kC + 3 * r + c) * N + p);
        }
}


// Adjoint of P2G and of the constitutive step, FP32. A particle whose
// deformation is ill-conditioned for FP32 (see needs_fp64) is left untouched
// and listed for k_p2g_bwd_fp64.
// regulariser factors of a P2G-adjoint CTA (Sec. III-E): F-bar of state
// k+1, and m-bar / mv-bar of the grid; ones when not regularising
__device__ __forceinline__ void p2g_bwd_factors(const AdjArgs& A, int inst, float* f) {
    if (!A.gscale) {
        f[0] = f[1] = f[2] = 1.0f;
        return;
    }
    float s0;
    f[0] = (float)reg_factor(A.gscale, A.pstat_in[3 * inst + 2], A.oom, A.gdelta);
    reg_grid_factors(A.gscale, A.gstat + 3 * inst, A.oom, A.gdelta, s0, f[1], f[2]);
}

// The G2P adjoint of one particle for the substep of G, given the adjoints
// of the particle's x, v, C after that substep in registers (the second half
// of the fused adjoint): advection, particle contact (pose sums per warp when
// warp_uniform, all lanes calling; else per thread), scatter into G.gacc with
// global atomics, and the partial x-bar of the state before it into G.adj.
// sk: the state after G's substep, whose v is the particle's gathered
// velocity wherever the particle contact left it alone.
__device__ __forceinline__ void g2p_bwd_particle(const InstDev& I, const AdjArgs& G, int inst, long long p,
                                                 bool active, bool warp_uniform, const float (&gx_in)[3],
                                                 const float (&gv_in)[3], const float (&gC)[3][3],
                                                 const float* sk) {
    const StepArgs& a = G.f;
    const long long N = a.ncap;
    float x[3] = {0.5f, 0.5f, 0.5f};
    if (active) {
#pragma unroll
        for (int k = 0; k < 3; k++) x[k] = ld(a.sin, N, kX + k, p);
    }
    Stencil st;
    make_stencil(I, x, st);
    int ox[3], oy[3], oz[3];
    node_offsets(I, st, ox, oy, oz);
    const float4* vg = a.vout + I.node_off;
    float gx[3], gvn[3], Sv[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (active) Sv[k] = ld_again(sk + (kV + k) * N + p);
        gx[k] = a.clip > 0.f ? clipf(gx_in[k], a.clip) : gx_in[k];
        const float gv = a.clip > 0.f ? clipf(gv_in[k], a.clip) : gv_in[k];
        gvn[k] = gv + I.dt * gx[k];   // adjoint of the advection x' = x + dt v'
    }
    if (I.pcoll && I.shovel_on) {
        float gp[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bool contact = false;
        if (active) {
            const Pose P = load_pose(I, a.substep);
            float sn, cs, n[3], nl[3];
            sincosf(P.psi, &sn, &cs);
            if (shovel_inside(I, P, cs, sn, x, n, nl)) {
                contact = true;
                float v[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int j = 0; j < 3; j++)
#pragma unroll
                        for (int k = 0; k < 3; k++) {
                            const float W = st.w[0][i] * st.w[1][j] * st.w[2][k];
                            const float4 g = __ldg(vg + ox[i] + oy[j] + oz[k]);
                            v[0] += W * g.x; v[1] += W * g.y; v[2] += W * g.z;
                        }
                float g0[3] = {gvn[0], gvn[1], gvn[2]}, gq[3] = {0.f, 0.f, 0.f};
                gvn[0] = gvn[1] = gvn[2] = 0.f;
                shovel_project_adj(I, P, cs, sn, x, v, g0, gvn, gq, gp);
                gx[0] += gq[0]; gx[1] += gq[1]; gx[2] += gq[2];
                Sv[0] = v[0]; Sv[1] = v[1]; Sv[2] = v[2];
            }
        }
        if (warp_uniform) {
            warp_reduce_add<8>(gp, G.gpose + 8 * inst, contact);
        } else if (contact) {
#pragma unroll
            for (int k = 0; k < 8; k++)
                if (gp[k] != 0.f) atomicAdd(G.gpose + 8 * inst + k, (double)gp[k]);
        }
    }
    if (active) {
        g2p_bwd_scatter<true>(I, G, st, ox, oy, oz, vg, nullptr, gvn, gC, gx, Sv);
#pragma unroll
        for (int k = 0; k < 3; k++) G.adj[(kX + k) * N + p] = gx[k];
    }
}

// The P2G adjoint of one CTA; Reg: with the regularisers of Sec. III-E (a
// separate instantiation, so that the plain path carries none of their code).
// Fused: G is the G2P adjoint of the substep before, which this CTA runs
// for its particles right after (g2p_bwd_particle), instead of storing their
// x, v, C adjoints.
template <bool Reg, bool Fused>
__device__ __forceinline__ void p2g_bwd_cta(const AdjArgs& A, const AdjArgs* G) {
    __shared__ double sred[4 * 32];
    __shared__ InstDev sI;
    __shared__ float sS[kParked * kChunk];
    __shared__ float sfac[3];   // F-bar, m-bar, mv-bar factors
    const StepArgs& a = A.f;
    const int inst = a.chunk_inst[blockIdx.x];
    if (threadIdx.x == 0) {
        if (Reg) p2g_bwd_factors(A, inst, sfac);
        else sfac[0] = sfac[1] = sfac[2] = 1.0f;
        // the grid adjoint kernel before this one has cleared these blocks
        if (A.reset_list && blockIdx.x == 0) *A.reset_list = 0;
    }
    const InstDev& I = stage_instance(sI, a.inst, inst);
    const long long p = (long long)blockIdx.x * kChunk + threadIdx.x;
    const bool active = p - I.pbeg < I.n;
    const long long N = a.ncap;
    float gmu = 0.f, glam = 0.f, galpha = 0.f, gmp = 0.f;
    float st[3] = {0.f, 0.f, 0.f};   // statistics of the x, v, F adjoints of state k
    // fused: the x, v, C adjoints of state k for the G2P adjoint of substep k-1
    float gxk[3] = {0.f, 0.f, 0.f}, gvk[3] = {0.f, 0.f, 0.f}, gCk[3][3] = {{0.f}};
    bool go_on = false;
    if (active) {
        float x[3], v[3], gx[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            x[k] = ld(a.sin, N, kX + k, p);
            v[k] = ld(a.sin, N, kV + k, p);
            gx[k] = A.adj[(kX + k) * N + p];
        }
        // the forward's SVD of the trial F (recorded) and its return mapping
        // again: the stress for the gather, the spectral data for the adjoint
        // (parked in shared memory meanwhile)
        bool fb;
        float Am[3][3];
        {
            Spectral<float> S;
            float qu[4], qv[4];
            load_svd(a.spec, N, p, S, qu, qv);
            return_map<float>(S, I.mu, I.lam, I.beta, I.smin);
            fb = needs_fp64(S);
            float Fn[3][3], tau[3][3];
            spectral_outputs<float, float>(S, Fn, tau);
            park(sS, qu, qv, S);
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int c = 0; c < 3; c++) Am[r][c] = I.stress_scale * tau[r][c] + I.mp * ld(a.sin, N, kC + 3 * r + c, p);
        }
        if (fb) {
            a.fb_list[atomicAdd(a.fb_count, 1)] = (int)p;
        } else {
            float gv[3], gA[3][3];
            p2g_bwd_gather(I, A, x, v, Am, Reg ? sfac[1] : 1.0f, Reg ? sfac[2] : 1.0f, gx, gv, gA, gmp);
            float gFn[3][3], gtau[3][3], gC[3][3], gFt[3][3];
            p2g_bwd_affine(I, A, p, gA, Reg ? sfac[0] : 1.0f, gFn, gtau, gC, gmp);
            Spectral<float> S;
            unpark(sS, S, I);
            constitutive_adjoint_spectral<float>(S, I.mu, I.lam, I.alpha, I.beta, I.smin, gFn, gtau, gFt, gmu, glam,
                                                 galpha);
            p2g_bwd_finish<!Fused>(I, A, p, gx, gv, gC, gFt, Reg ? A.gscale : 0, st);
            if (Fused) {
#pragma unroll
                for (int k = 0; k < 3; k++) { gxk[k] = gx[k]; gvk[k] = gv[k]; }
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int c = 0; c < 3; c++) gCk[r][c] = gC[r][c];
                go_on = true;
            }
        }
    }
    // parameter sums first: their registers are free for the G2P adjoint
    float gd[4] = {gmu, glam, galpha, gmp};
    block_reduce_add<4>(gd, A.gmat + 4 * inst, sred);
    if (Fused) g2p_bwd_particle(I, *G, inst, p, go_on, true, gxk, gvk, gCk, a.sin);
    if (Reg) {
        __syncthreads();   // sred is reused
        block_stat<3>(A.gscale, st, A.pstat_out + 3 * inst, reinterpret_cast<float*>(sred));
    }
}

__global__ void __launch_bounds__(kChunk, MPM_MINB_P2G_BWD) k_p2g_bwd(AdjArgs A) {
    wait_previous_grid();
    p2g_bwd_cta<false, false>(A, nullptr);
}

__global__ void __launch_bounds__(kChunk, MPM_MINB_P2G_BWD) k_p2g_bwd_reg(AdjArgs A) {
    wait_previous_grid();
    p2g_bwd_cta<true, false>(A, nullptr);
}

// the P2G adjoint of substep k (A) and the G2P adjoint of substep k-1 (G) in
// one pass over the particles: the x, v, C adjoints of state k stay in
// registers. G.gacc is the other grid-adjoint buffer (zero on entry).
template <int MINB>
__global__ void __launch_bounds__(kChunk, MINB) k_p2g_g2p_bwd(AdjArgs A, AdjArgs G) {
    wait_previous_grid();
    p2g_bwd_cta<false, true>(A, &G);
}

// The particles k_p2g_bwd listed: the same adjoint with the SVD, the return
// mapping and their adjoint in FP64; Fused: then the G2P adjoint of the
// substep before (G) for them, as k_p2g_g2p_bwd does for the others.
template <bool Fused>
__device__ __forceinline__ void p2g_bwd_fp64_all(const AdjArgs& A, const AdjArgs* G) {
    __shared__ int scount;
    const StepArgs& a = A.f;
    const int count = fb_begin(a.fb_count, &scount);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const long long p = a.fb_list[i];
        const int inst = a.chunk_inst[p / kChunk];
        const InstDev& I = a.inst[inst];
        const long long N = a.ncap;
        float x[3], v[3], gx[3], C[3][3], Ft[3][3], Fn[3][3], tau[3][3], Am[3][3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            x[k] = ld(a.sin, N, kX + k, p);
            v[k] = ld(a.sin, N, kV + k, p);
            gx[k] = A.adj[(kX + k) * N + p];
        }
        load_trial(I, a, p, C, Ft);
        constitutive_fp64(Ft, I.mu, I.lam, I.beta, I.smin, Fn, tau);
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int c = 0; c < 3; c++) Am[r][c] = I.stress_scale * tau[r][c] + I.mp * C[r][c];
        float fac[3], st[3] = {0.f, 0.f, 0.f};
        p2g_bwd_factors(A, inst, fac);
        float gv[3], gA[3][3], gmp = 0.f, gmu = 0.f, glam = 0.f, galpha = 0.f;
        p2g_bwd_gather(I, A, x, v, Am, fac[1], fac[2], gx, gv, gA, gmp);
        float gFn[3][3], gtau[3][3], gC[3][3], gFt[3][3];
        p2g_bwd_affine(I, A, p, gA, fac[0], gFn, gtau, gC, gmp);
        constitutive_adjoint_fp64(Ft, I.mu, I.lam, I.alpha, I.beta, I.smin, gFn, gtau, tau, gFt, gmu, glam, galpha);
        p2g_bwd_finish<!Fused>(I, A, p, gx, gv, gC, gFt, A.gscale, st);
        if (Fused) g2p_bwd_particle(I, *G, inst, p, true, false, gx, gv, gC, a.sin);
        if (A.gscale)
            for (int k = 0; k < 3; k++) {
                if (!(st[k] > 0.0f)) continue;
                if (A.gscale == 1)
                    atomicMax(reinterpret_cast<unsigned long long*>(A.pstat_out + 3 * inst + k),
                              (unsigned long long)__double_as_longlong((double)st[k]));
                else
                    atomicAdd(A.pstat_out + 3 * inst + k, (double)st[k]);
            }
        atomicAdd(A.gmat + 4 * inst + 0, (double)gmu);
        atomicAdd(A.gmat + 4 * inst + 1, (double)glam);
        atomicAdd(A.gmat + 4 * inst + 2, (double)galpha);
        atomicAdd(A.gmat + 4 * inst + 3, (double)gmp);
        atomicAdd(a.fp64_count, 1ull);
    }
    fb_end(a.fb_count, count);
}

__global__ void __launch_bounds__(kFp64Threads) k_p2g_bwd_fp64(AdjArgs A) {
    wait_previous_grid();
    p2g_bwd_fp64_all<false>(A, nullptr);
}

__global__ void __launch_bounds__(kFp64Threads) k_p2g_g2p_bwd_fp64(AdjArgs A, AdjArgs G) {
    wait_previous_grid();
    p2g_bwd_fp64_all<true>(A, &G);
}

// zero the accumulators (and grid adjoints) and the flags of the listed
// blocks (the launcher then empties the list)
__global__ void __launch_bounds__(256) k_grid_clear(AdjArgs A) {
    wait_previous_grid();
    const StepArgs& a = A.f;
    const int lane = threadIdx.x & 31;
    for_listed_blocks(a.flags, a.n_blocks, [&](int gw) { clear_block(a, a.flags, a.acc, A.gacc, gw, lane); });
}

// ---------------------------------------------------------------------------
// layout conversion, loss, seeding
// ---------------------------------------------------------------------------
// external interleaved arrays (x[3e+k], M[9e+k]) <-> internal SoA slots
__global__ void k_state_from_ext(long long ncap, long long nslots, const int* ext_of_slot, const float* x,
                                 const float* v, const float* C, const float* F, float* s) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nslots) return;
    const int e = ext_of_slot[p];
    const bool on = e >= 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        s[(kX + k) * ncap + p] = (on && x) ? x[3LL * e + k] : 0.5f;
        s[(kV + k) * ncap + p] = (on && v) ? v[3LL * e + k] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 9; k++) {
        s[(kC + k) * ncap + p] = (on && C) ? C[9LL * e + k] : 0.f;
        s[(kF + k) * ncap + p] = (on && F) ? F[9LL * e + k] : ((k % 4 == 0) ? 1.f : 0.f);
    }
}

// adjoint seed: x and v adjoints from external arrays (or 0), C and F 0
__global__ void k_adj_from_ext(long long ncap, long long nslots, const int* ext_of_slot, const float* gx,
                               const float* gv, float* adj) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nslots) return;
    const int e = ext_of_slot[p];
    const bool on = e >= 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        adj[(kX + k) * ncap + p] = (on && gx) ? gx[3LL * e + k] : 0.f;
        adj[(kV + k) * ncap + p] = (on && gv) ? gv[3LL * e + k] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 18; k++) adj[(kC + k) * ncap + p] = 0.f;
}

__global__ void k_state_to_ext(long long ncap, long long nslots, const int* ext_of_slot, const float* s, float* x,
                               float* v, float* C, float* F) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nslots) return;
    const int e = ext_of_slot[p];
    if (e < 0) return;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (x) x[3LL * e + k] = s[(kX + k) * ncap + p];
        if (v) v[3LL * e + k] = s[(kV + k) * ncap + p];
    }
#pragma unroll
    for (int k = 0; k < 9; k++) {
        if (C) C[9LL * e + k] = s[(kC + k) * ncap + p];
        if (F) F[9LL * e + k] = s[(kF + k) * ncap + p];
    }
}

__global__ void __launch_bounds__(kChunk) k_loss_mse(const InstDev* inst, const int* chunk_inst, long long ncap,
                                                    const int* ext_of_slot, const float* s, const float* target,
                                                    float* dldx, double* loss) {
    __shared__ double sred[32];
    const int ii = chunk_inst[blockIdx.x];
    const InstDev& I = inst[ii];
    const long long p = (long long)blockIdx.x * kChunk + threadIdx.x;
    double l = 0.0;
    if (p - I.pbeg < I.n) {
        const int e = ext_of_slot[p];
        const float inv_n = 1.0f / float(I.n);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float d = s[(kX + k) * ncap + p] - target[3LL * e + k];
            l += double(d) * double(d);
            if (dldx) dldx[3LL * e + k] = 2.0f * d * inv_n;
        }
        l /= double(I.n);
    }
    // per-particle terms in FP64, one FP64 warp sum (the loss is reported in FP64)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0;
        for (int w = 0; w < kChunk / 32; w++) x += sred[w];
        if (x != 0.0) atomicAdd(loss + ii, x);
    }
}

// ---------------------------------------------------------------------------
// particle sort by cell (counting sort over the cells of every instance;
// the order inside a cell is the order in which the atomics hand out ranks)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kChunk) k_sort_keys(const InstDev* inst, const int* chunk_inst, long long ncap,
                                                     const float* s, int* key, int* rank, int* bcount) {
    const InstDev& I = inst[chunk_inst[blockIdx.x]];
    const long long p = (long long)blockIdx.x * kChunk + threadIdx.x;
    if (p - I.pbeg >= I.n) return;
    float x[3];
#pragma unroll
    for (int k = 0; k < 3; k++) x[k] = s[(kX + k) * ncap + p];
    Stencil st;
    make_stencil(I, x, st);
    // key: the particle's base cell, blocks in order and cells inside a block
    // in (x, y, z) order, so that a warp's particles share stencil nodes
    const int blk = I.blk_off + ((st.base[0] >> 2) * I.nb[1] + (st.base[1] >> 2)) * I.nb[2] + (st.base[2] >> 2);
    const int b = blk * 64 + ((st.base[0] & 3) * 4 + (st.base[1] & 3)) * 4 + (st.base[2] & 3);
    key[p] = b;
    rank[p] = atomicAdd(bcount + b, 1);
}

// exclusive scan of n ints: per-CTA scans of 1024, a scan of the CTA sums, an add
__global__ void __launch_bounds__(1024) k_scan_local(const int* in, int* out, int* part, int n) {
    __shared__ int warp_tot[32];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int v = i < n ? in[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    const int excl = x - v + (w > 0 ? warp_tot[w - 1] : 0);
    if (i < n) out[i] = excl;
    if (threadIdx.x == 1023) part[blockIdx.x] = warp_tot[31];
}

__global__ void __launch_bounds__(1024) k_scan_parts(int* part, int nparts) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < nparts; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < nparts ? part[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[w] = x;
        __syncthreads();
        if (w == 0) {
            int t = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const int excl = x - v + (w > 0 ? warp_tot[w - 1] : 0) + carry;
        if (i < nparts) part[i] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[31];
        __syncthreads();
    }
}

__global__ void k_scan_add(int* out, const int* part, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += part[i / 1024];
}

// Order inside a grid block: the cell-major order of the counting sort
// (cell_start + rank) is rearranged rank-major: first the rank-0 particle of
// every occupied cell of the block (cells in block order), then the rank-1
// particles, and so on. A warp then holds particles of up to 32 different
// cells, so the 32 lanes of a scatter instruction never add to one node, and
// a CTA's 256 particles still lie in one or two neighbouring blocks.
// remap[cell_start + rank] = the particle's position in that order (in the
// same numbering as cell_start). One 64-thread CTA (a thread per cell) per
// grid block.
__global__ void __launch_bounds__(64) k_sort_interleave(const int* bcount, const int* bscan, int* remap) {
    __shared__ int wtot[2], wmax[2];
    const int b = blockIdx.x, c = threadIdx.x, lane = c & 31, w = c >> 5;
    const int cnt = bcount[b * 64 + c];
    int m = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) wmax[w] = m;
    __syncthreads();
    const int rmax = max(wmax[0], wmax[1]);
    if (rmax == 0) return;   // empty block (uniform)
    const int start = bscan[b * 64 + c];
    const int bstart = bscan[b * 64];
    int base = 0;
    for (int r = 0; r < rmax; r++) {
        const bool has = cnt > r;
        const unsigned bal = __ballot_sync(0xffffffffu, has);
        __syncthreads();   // wtot of the previous round has been read
        if (lane == 0) wtot[w] = __popc(bal);
        __syncthreads();
        const int off = __popc(bal & ((1u << lane) - 1u)) + (w == 1 ? wtot[0] : 0);
        if (has) remap[start + r] = bstart + base + off;
        base += wtot[0] + wtot[1];
    }
}

// new slot of every particle; perm[new] = old, ext carried along
__global__ void __launch_bounds__(kChunk) k_sort_perm(const InstDev* inst, const int* chunk_inst, const int* key,
                                                     const int* rank, const int* bscan, const int* remap,
                                                     const int* ext_old, int* perm, int* ext_new) {
    const InstDev& I = inst[chunk_inst[blockIdx.x]];
    const long long p = (long long)blockIdx.x * kChunk + threadIdx.x;
    if (p - I.pbeg >= I.n) return;
    const long long q = I.pbeg + (remap[bscan[key[p]] + rank[p]] - I.ext_off);
    perm[q] = (int)p;
    ext_new[q] = ext_old[p];
}

// dst[q] = src[perm[q]] (gather into the sorted order), all 24 components
__global__ void __launch_bounds__(kChunk) k_permute(const InstDev* inst, const int* chunk_inst, long long ncap,
                                                   const int* perm, const float* src, float* dst) {
    const InstDev& I = inst[chunk_inst[blockIdx.x]];
    const long long q = (long long)blockIdx.x * kChunk + threadIdx.x;
    if (q - I.pbeg >= I.n) return;
    const long long p = perm[q];
#pragma unroll 8
    for (int c = 0; c < kStateComps; c++) dst[c * ncap + q] = src[c * ncap + p];
}

// dst[perm[q]] = src[q] (back to the order before the sort), all 24 components
__global__ void __launch_bounds__(kChunk) k_unpermute(const InstDev* inst, const int* chunk_inst, long long ncap,
                                                     const int* perm, const float* src, float* dst) {
    const InstDev& I = inst[chunk_inst[blockIdx.x]];
    const long long q = (long long)blockIdx.x * kChunk + threadIdx.x;
    if (q - I.pbeg >= I.n) return;
    const long long p = perm[q];
#pragma unroll 8
    for (int c = 0; c < kStateComps; c++) dst[c * ncap + p] = src[c * ncap + q];
}

// statistics (Sec. III-E) of the x, v and F adjoints of a state (the loss
// seed of a backward): largest magnitude (mode 1) or sum of squares (2)
__global__ void __launch_bounds__(kChunk) k_adj_stats(const InstDev* inst, const int* chunk_inst, long long ncap,
                                                      const float* adj, int mode, double* pstat) {
    __shared__ float sred[3 * 32];
    const int i = chunk_inst[blockIdx.x];
    const InstDev& I = inst[i];
    const long long p = (long long)blockIdx.x * kChunk + threadIdx.x;
    float st[3] = {0.f, 0.f, 0.f};
    if (p - I.pbeg < I.n) {
        for (int c = 0; c < kStateComps; c++) {
            const int which = c < kV ? 0 : (c < kC ? 1 : (c < kF ? -1 : 2));
            if (which < 0) continue;
            const float s = stat_of(mode, adj[c * ncap + p]);
            st[which] = mode == 1 ? fmaxf(st[which], s) : st[which] + s;
        }
    }
    block_stat<3>(mode, st, pstat + 3 * i, sred);
}

}  // namespace mpm

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
namespace mpm {

static inline int grid_ctas(int n_blocks) { return (n_blocks * 32 + 255) / 256; }

// Launch of a kernel of the substep path with programmatic stream
// serialization: its CTAs may be scheduled as the previous kernel's last
// CTAs retire (hiding the launch gap); every such kernel waits at its start
// (wait_previous_grid) until the previous grid has completed and its writes
// are visible, so the stream order of the results is unchanged.
template <typename... P, typename... A>
static cudaError_t launch_pdl_smem(void (*k)(P...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                                   A&&... args) {
#if MPM_PDL
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
#else
    k<<<grid, block, smem, s>>>(std::forward<A>(args)...);
    return cudaGetLastError();
#endif
}

template <typename... P, typename... A>
static cudaError_t launch_pdl(void (*k)(P...), unsigned grid, unsigned block, cudaStream_t s, A&&... args) {
    return launch_pdl_smem(k, grid, block, 0, s, std::forward<A>(args)...);
}

// CTAs of the kernels that walk a block list: a warp per block up to one
// full wave of 256-thread CTAs (8 per SM), grid-stride beyond
static inline int list_ctas(int n_blocks) { return std::min(grid_ctas(n_blocks), kListCtas); }

// the instantiation of a particle kernel for a register cap (minimum
// resident CTAs per SM); caps outside the instantiated set take the nearest
static unsigned p2g_minb(int m) { return m <= 3 ? 3 : 4; }

cudaError_t launch_kernel(KernelId id, const AdjArgs& A, const LaunchShape& ls, cudaStream_t s) {
    const StepArgs& a = A.f;
    const bool particle_kernel = id == KernelId::P2G || id == KernelId::G2P || id == KernelId::G2PBwd ||
                                 id == KernelId::P2GBwd || id == KernelId::P2GFp64 ||
                                 id == KernelId::P2GBwdFp64;
    if ((particle_kernel && a.n_chunks <= 0) || (!particle_kernel && a.n_blocks <= 0)) return cudaSuccess;
    switch (id) {
        case KernelId::P2G:
            return p2g_minb(ls.p2g) == 3 ? launch_pdl(k_p2g<3>, a.n_chunks, kChunk, s, a)
                                         : launch_pdl(k_p2g<4>, a.n_chunks, kChunk, s, a);
        case KernelId::Grid: return launch_pdl(k_grid, list_ctas(a.n_blocks), 256, s, a);
        case KernelId::G2P:
            return p2g_minb(ls.g2p) == 3 ? launch_pdl(k_g2p<3>, a.n_chunks, kChunk, s, a)
                                         : launch_pdl(k_g2p<4>, a.n_chunks, kChunk, s, a);
        case KernelId::G2PBwd:
            return a.tile ? launch_pdl_smem(k_g2p_bwd<true>, a.n_chunks, kChunk, sizeof(TileSmem), s, A)
                          : launch_pdl(k_g2p_bwd<false>, a.n_chunks, kChunk, s, A);
        case KernelId::GridBwd: return launch_pdl(k_grid_bwd, list_ctas(a.n_blocks), 256, s, A);
        case KernelId::P2GBwd:
            if (!a.spec) return cudaErrorInvalidValue;   // needs the recorded SVD
            return launch_pdl(A.gscale ? k_p2g_bwd_reg : k_p2g_bwd, a.n_chunks, kChunk, s, A);
        case KernelId::GridClear:
            if (const cudaError_t e = launch_pdl(k_grid_clear, list_ctas(a.n_blocks), 256, s, A)) return e;
            return cudaMemsetAsync(a.flags + a.n_blocks, 0, sizeof(int), s);   // empty list
        case KernelId::P2GFp64: return launch_pdl(k_p2g_fp64, kFp64Ctas, kFp64Threads, s, a);
        case KernelId::P2GBwdFp64: return launch_pdl(k_p2g_bwd_fp64, kFp64Ctas, kFp64Threads, s, A);
        case KernelId::P2GG2PBwd:
        case KernelId::P2GG2PBwdFp64: return cudaErrorInvalidValue;   // two argument sets: launch_fused
        case KernelId::SlotClear: {
            AdjArgs C = A;
            C.gacc = nullptr;
            if (const cudaError_t e = launch_pdl(k_grid_clear, list_ctas(a.n_blocks), 256, s, C)) return e;
            return cudaMemsetAsync(a.flags + a.n_blocks, 0, sizeof(int), s);   // empty list
        }
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_fused(KernelId id, const AdjArgs& A, const AdjArgs& G, const LaunchShape& ls, cudaStream_t s) {
    const StepArgs& a = A.f;
    if (a.n_chunks <= 0) return cudaSuccess;
    if (!a.spec || A.gscale || a.tile) return cudaErrorInvalidValue;
    switch (id) {
        case KernelId::P2GG2PBwd:
            if (ls.fused <= 2) return launch_pdl(k_p2g_g2p_bwd<2>, a.n_chunks, kChunk, s, A, G);
            if (ls.fused == 3) return launch_pdl(k_p2g_g2p_bwd<3>, a.n_chunks, kChunk, s, A, G);
            return launch_pdl(k_p2g_g2p_bwd<4>, a.n_chunks, kChunk, s, A, G);
        case KernelId::P2GG2PBwdFp64: return launch_pdl(k_p2g_g2p_bwd_fp64, kFp64Ctas, kFp64Threads, s, A, G);
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_stats(const InstDev* inst, const int* chunk_inst, int n_chunks, long long ncap,
                             const float* adj, int mode, double* pstat, cudaStream_t st) {
    if (n_chunks <= 0 || !mode) return cudaSuccess;
    k_adj_stats<<<n_chunks, kChunk, 0, st>>>(inst, chunk_inst, ncap, adj, mode, pstat);
    return cudaGetLastError();
}

cudaError_t launch_state_from_ext(long long ncap, long long nslots, const int* ext_of_slot, const float* x,
                                  const float* v, const float* C, const float* F, float* s, cudaStream_t st) {
    if (nslots == 0) return cudaSuccess;
    k_state_from_ext<<<(unsigned)((nslots + 255) / 256), 256, 0, st>>>(ncap, nslots, ext_of_slot, x, v, C, F, s);
    return cudaGetLastError();
}

cudaError_t launch_adj_from_ext(long long ncap, long long nslots, const int* ext_of_slot, const float* gx,
                                const float* gv, float* adj, cudaStream_t st) {
    if (nslots == 0) return cudaSuccess;
    k_adj_from_ext<<<(unsigned)((nslots + 255) / 256), 256, 0, st>>>(ncap, nslots, ext_of_slot, gx, gv, adj);
    return cudaGetLastError();
}

cudaError_t launch_state_to_ext(long long ncap, long long nslots, const int* ext_of_slot, const float* s, float* x,
                                float* v, float* C, float* F, cudaStream_t st) {
    if (nslots == 0) return cudaSuccess;
    k_state_to_ext<<<(unsigned)((nslots + 255) / 256), 256, 0, st>>>(ncap, nslots, ext_of_slot, s, x, v, C, F);
    return cudaGetLastError();
}

cudaError_t launch_sort(const InstDev* inst, const int* chunk_inst, int n_chunks, long long ncap, int n_keys,
                        const float* state, float* state_out, const int* ext_old, int* ext_new, int* key, int* rank,
                        int* bcount, int* bscan, int* part, int* remap, int* perm, cudaStream_t st) {
    if (n_chunks == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(bcount, 0, (size_t)n_keys * sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_sort_keys<<<n_chunks, kChunk, 0, st>>>(inst, chunk_inst, ncap, state, key, rank, bcount);
    const int nparts = (n_keys + 1023) / 1024;
    k_scan_local<<<nparts, 1024, 0, st>>>(bcount, bscan, part, n_keys);
    k_scan_parts<<<1, 1024, 0, st>>>(part, nparts);
    k_scan_add<<<(n_keys + 255) / 256, 256, 0, st>>>(bscan, part, n_keys);
    e = cudaMemcpyAsync(ext_new, ext_old, (size_t)ncap * sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    k_sort_interleave<<<n_keys / 64, 64, 0, st>>>(bcount, bscan, remap);
    k_sort_perm<<<n_chunks, kChunk, 0, st>>>(inst, chunk_inst, key, rank, bscan, remap, ext_old, perm, ext_new);
    k_permute<<<n_chunks, kChunk, 0, st>>>(inst, chunk_inst, ncap, perm, state, state_out);
    return cudaGetLastError();
}

cudaError_t launch_unpermute(const InstDev* inst, const int* chunk_inst, int n_chunks, long long ncap, const int* perm,
                             const float* src, float* dst, cudaStream_t st) {
    if (n_chunks == 0) return cudaSuccess;
    k_unpermute<<<n_chunks, kChunk, 0, st>>>(inst, chunk_inst, ncap, perm, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_loss_mse(const InstDev* inst, const int* chunk_inst, int n_chunks, long long ncap,
                            const int* ext_of_slot, const float* s, const float* target, float* dldx, double* loss,
                            cudaStream_t st) {
    if (n_chunks == 0) return cudaSuccess;
    k_loss_mse<<<n_chunks, kChunk, 0, st>>>(inst, chunk_inst, ncap, ext_of_slot, s, target, dldx, loss);
    return cudaGetLastError();
}

}  // namespace mpm
