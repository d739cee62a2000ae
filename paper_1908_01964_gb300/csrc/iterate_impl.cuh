// Kernels of the accelerated rule and their launcher for one (BLOCK, SPT) shape;
// included by iterate_inst.cu, which is compiled once per shape so that the
// shapes' large unrolled bodies build in parallel.  The kernels are described in
// iterate.cu.
#pragma once

#include <float.h>

#include <algorithm>

#include "accel_common.cuh"

namespace rcscm {
namespace {

// Resident CTAs per SM requested for the fused kernel: at 128 threads x 8 slots its
// projection and Wiener code would take it to 105 registers (4 CTAs per SM); 5 CTAs,
// as for the plain kernel, need at most 96.
constexpr int solve_min_blocks(int block, int spt) { return (block == 128 && spt == 8) ? 5 : 0; }

// Shared memory of the fused row body: the row's projection and steering vector.
struct FusedSmem {
    float2 phi[kMaxM * kMaxM];
    float2 a[kMaxM];
};

// One row, all n_iter passes with the row held in registers (RowState).
// FUSED: invariants from x first, Wiener output h last (h != nullptr).
template <int BLOCK, int NP, bool FUSED>
__device__ __forceinline__ void accel_row(const DevState& d, int r, int J, int64_t off, const RowConst& c,
                                          int n_iter, const IterParams& p,
                                          float (*red)[BLOCK / 32 > 0 ? BLOCK / 32 : 1], float2* __restrict__ h,
                                          FusedSmem* fs) {
    RowState<BLOCK, NP> st;
    const RowDesc* rd = d.rows + r;
    if constexpr (FUSED) {
        const int M = rd->M;
        for (int e = threadIdx.x; e < M * M; e += BLOCK) fs->phi[e] = d.phi[(size_t)r * 64 + e];
        if (threadIdx.x < M) fs->a[threadIdx.x] = d.a32[(size_t)r * kMaxM + threadIdx.x];
        __syncthreads();
        const float2* x = rd->x;
        st.load_inv_with(J, c, p, [&](int j, float4& t, float& kap) {
            project_slot_m(M, fs->phi, x + (int64_t)j * M, t, kap);
            d.inv4[off + j] = t;
            d.kap[off + j] = kap;
        });
        st.load_state(rd->rh0, rd->ru0, (float)d.lam0[r]);     // the initial state, whatever ran before
    } else {
        st.load_inv(d, off, J, c, p);
        st.load_state(d.rh + off, d.ru + off, d.lam[r]);
    }
    for (int it = 0; it < n_iter; ++it) {
        if (!FUSED && d.ckpt_stride > 0) {                   // checkpoint: state entering pass u
            const int u = p.ckpt_first + it;
            if (u % d.ckpt_stride == 0) {
                const size_t k = (size_t)(u / d.ckpt_stride);
                st.store_state(d.ckpt_rh + k * d.n_slots + off, d.ckpt_ru + k * d.n_slots + off);
                if (threadIdx.x == 0) d.ckpt_lam[k * d.n_rows + r] = st.lam;
            }
        }
        st.pass(c, p, red, it & 1);
    }
    st.store_state(d.rh + off, d.ru + off);
    if (n_iter > 0 && st.any_clamp(p.ru_floor)) atomicOr(d.status, kFlagClamp);
    if (threadIdx.x == 0) {
        d.lam[r] = st.lam;
        if (!(st.lam > 0.f) || !(st.lam <= FLT_MAX)) atomicOr(d.status, kFlagNonfinite);
    }
    if constexpr (FUSED) {                           // h = w a with the final state
        const int M = rd->M;
        const float2 sab = make_float2(c.sab_re, c.sab_im);
        float2* hrow = h + rd->out_off;
#pragma unroll
        for (int k = 0; k < 2 * NP; ++k) {
            const int j = k * BLOCK + threadIdx.x;
            if (j < J) {
                const float4 t = make_float4(k & 1 ? hi_of(st.tr[k >> 1]) : lo_of(st.tr[k >> 1]),
                                             k & 1 ? hi_of(st.ti[k >> 1]) : lo_of(st.ti[k >> 1]),
                                             k & 1 ? hi_of(st.sr[k >> 1]) : lo_of(st.sr[k >> 1]),
                                             k & 1 ? hi_of(st.si[k >> 1]) : lo_of(st.si[k >> 1]));
                const float2 w = wiener_weight(c.taa, c.sab2, sab, st.lam, t, st.rh_of(k), st.ru_of(k));
                float2* hj = hrow + (int64_t)j * M;
                for (int m = 0; m < M; ++m) hj[m] = cmul_exact(w, fs->a[m]);
            }
        }
    }
}

template <int BLOCK, int SPT, bool FUSED>
__device__ __forceinline__ void accel_one_row(const DevState& d, int r, int n_iter, const IterParams& p,
                                              float (*red)[BLOCK / 32 > 0 ? BLOCK / 32 : 1], float2* h,
                                              FusedSmem* fs) {
    const RowDesc* rd = d.rows + r;
    const int J = rd->J;
    const int64_t off = rd->slot_off;
    const RowConst c = d.rc[r];
    const int np = (J + 2 * BLOCK - 1) / (2 * BLOCK);     // chunk pairs, 1..SPT/2 (checked by the host)
    // The row's exact pair count selects the unrolled body (block-uniform branch).
#define RCSCM_ROW(N) \
    case N:          \
        if constexpr (2 * N <= SPT) accel_row<BLOCK, N, FUSED>(d, r, J, off, c, n_iter, p, red, h, fs); \
        break;
    switch (np) {
        RCSCM_ROW(1) RCSCM_ROW(2) RCSCM_ROW(3) RCSCM_ROW(4) RCSCM_ROW(5) RCSCM_ROW(6) RCSCM_ROW(7) RCSCM_ROW(8)
        default: break;
    }
#undef RCSCM_ROW
}

// One CTA per row, rows in the order table (longest first).
template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK) accel_kernel(DevState d, int n_iter, IterParams p) {
    __shared__ float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    RCSCM_CTA_CHECK(row_ok(d, d.order[blockIdx.x], BLOCK * SPT), d.status);
    accel_one_row<BLOCK, SPT, false>(d, d.order[blockIdx.x], n_iter, p, red, nullptr, nullptr);
}

// Launched as a programmatic dependent of the per-frequency setup: a CTA may start while
// the setup still runs.  Before griddepcontrol.wait it touches only the caller's inputs,
// and only to ask L2 for them (prefetch: no value is read, so a preceding kernel that
// writes them is still seen); every setup output is read after the wait.
template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK, solve_min_blocks(BLOCK, SPT)) solve_kernel(DevState d, int n_iter, IterParams p, float2* h) {
    __shared__ float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    __shared__ FusedSmem fs;
    const int r = d.order[blockIdx.x];
    RCSCM_CTA_CHECK(row_ok(d, r, BLOCK * SPT), d.status);
    {
        const RowDesc* rd = d.rows + r;
        const char* xb = reinterpret_cast<const char*>(rd->x);
        const int64_t xbytes = (int64_t)rd->J * rd->M * (int64_t)sizeof(float2);
        for (int64_t o = (int64_t)threadIdx.x * 128; o < xbytes; o += (int64_t)BLOCK * 128)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(xb + o));
        const int64_t sbytes = (int64_t)rd->J * (int64_t)sizeof(float);
        for (int64_t o = (int64_t)threadIdx.x * 128; o < sbytes; o += (int64_t)BLOCK * 128) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(rd->rh0) + o));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(rd->ru0) + o));
        }
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    accel_one_row<BLOCK, SPT, true>(d, r, n_iter, p, red, h, &fs);
}

#include "stream_kernel.cuh"

// Persistent variants: a fixed grid of resident CTAs takes rows from the order
// table through an atomic counter (dynamic longest-first scheduling).
template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK) accel_persistent_kernel(DevState d, int n_iter, IterParams p, int n_rows) {
    __shared__ float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    __shared__ int s_next;
    for (;;) {
        __syncthreads();                    // every thread is done with s_next and the previous row
        if (threadIdx.x == 0) s_next = atomicAdd(d.counter, 1);
        __syncthreads();
        const int k = s_next;
        if (k >= n_rows) break;
        RCSCM_CTA_CHECK(row_ok(d, d.order[k], BLOCK * SPT), d.status);
        accel_one_row<BLOCK, SPT, false>(d, d.order[k], n_iter, p, red, nullptr, nullptr);
    }
}

template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK, solve_min_blocks(BLOCK, SPT)) solve_persistent_kernel(DevState d, int n_iter, IterParams p, int n_rows,
                                                                 float2* h) {
    __shared__ float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    __shared__ FusedSmem fs;
    __shared__ int s_next;
    for (;;) {
        __syncthreads();                    // every thread is done with s_next, fs and the previous row
        if (threadIdx.x == 0) s_next = atomicAdd(d.counter, 1);
        __syncthreads();
        const int k = s_next;
        if (k >= n_rows) break;
        RCSCM_CTA_CHECK(row_ok(d, d.order[k], BLOCK * SPT), d.status);
        accel_one_row<BLOCK, SPT, true>(d, d.order[k], n_iter, p, red, h, &fs);
    }
}

template <class Kernel>
int resident_per_sm(Kernel k, int block) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, 0) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

}  // namespace

template <int BLOCK, int SPT>
cudaError_t launch_accel_t(const DevState& d, int n_rows, int n_iter, const IterParams& p, bool persistent,
                           float2* h, cudaStream_t s) {
    if (!persistent) {
        if (h) {                  // a programmatic dependent of the kernel before it (the setup)
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(n_rows);
            cfg.blockDim = dim3(BLOCK);
            cfg.dynamicSmemBytes = 0;
            cfg.stream = s;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            return cudaLaunchKernelEx(&cfg, solve_kernel<BLOCK, SPT>, d, n_iter, p, h);
        } else if (n_iter == 1)
            accel_stream_kernel<BLOCK, SPT><<<n_rows, BLOCK, 0, s>>>(d, p);
        else
            accel_kernel<BLOCK, SPT><<<n_rows, BLOCK, 0, s>>>(d, n_iter, p);
        return cudaGetLastError();
    }
    static const int per_sm = resident_per_sm(accel_persistent_kernel<BLOCK, SPT>, BLOCK);
    static const int per_sm_fused = resident_per_sm(solve_persistent_kernel<BLOCK, SPT>, BLOCK);
    const int grid = std::min(n_rows, (h ? per_sm_fused : per_sm) * d.n_sm);
    cudaError_t e = cudaMemsetAsync(d.counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (h)
        solve_persistent_kernel<BLOCK, SPT><<<grid, BLOCK, 0, s>>>(d, n_iter, p, n_rows, h);
    else
        accel_persistent_kernel<BLOCK, SPT><<<grid, BLOCK, 0, s>>>(d, n_iter, p, n_rows);
    return cudaGetLastError();
}

}  // namespace rcscm
