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
    accel_one_row<BLOCK, SPT, false>(d, d.order[blockIdx.x], n_iter, p, red, nullptr, nullptr);
}

template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK, solve_min_blocks(BLOCK, SPT)) solve_kernel(DevState d, int n_iter, IterParams p, float2* h) {
    __shared__ float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    __shared__ FusedSmem fs;
    accel_one_row<BLOCK, SPT, true>(d, d.order[blockIdx.x], n_iter, p, red, h, &fs);
}

// Streaming form of a launch that runs exactly one pass: the row's pairs are
// loaded, updated and stored one at a time, with A/M and B of pass A kept in
// shared memory for pass B, so few registers are live and several rows stream
// through each SM.  Same operations in the same order and the same reduction as
// the register-resident form, so the results are bitwise equal.
template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK) accel_stream_kernel(DevState d, IterParams p) {
    __shared__ float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    __shared__ f32x2 s_am[SPT / 2][BLOCK], s_b[SPT / 2][BLOCK];
    const int r = d.order[blockIdx.x];
    const RowDesc* rd = d.rows + r;
    const int J = rd->J;
    const int64_t off = rd->slot_off;
    const RowConst c = d.rc[r];
    const int tid = threadIdx.x;
    const int np = (J + 2 * BLOCK - 1) / (2 * BLOCK);     // 1..SPT/2 (checked by the host)
    const float lam0 = d.lam[r];
    const bool ckpt = d.ckpt_stride > 0 && p.ckpt_first % d.ckpt_stride == 0;
    const size_t kc = ckpt ? (size_t)(p.ckpt_first / d.ckpt_stride) : 0;
    const PassConsts k = pass_consts(c, p, lam0);
    f32x2 part = dup(0.f);
    for (int q = 0; q < np; ++q) {
        const int j0 = 2 * q * BLOCK + tid, j1 = j0 + BLOCK;
        const bool v0 = j0 < J, v1 = j1 < J;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 t0 = v0 ? d.inv4[off + j0] : z, t1 = v1 ? d.inv4[off + j1] : z;
        const float km0 = v0 ? fmaf(d.kap[off + j0], c.invM, p.ru_floor) : 1.f;
        const float km1 = v1 ? fmaf(d.kap[off + j1], c.invM, p.ru_floor) : 1.f;
        const float rh0 = v0 ? d.rh[off + j0] : 0.f, rh1 = v1 ? d.rh[off + j1] : 0.f;
        const float ru0 = v0 ? d.ru[off + j0] : 1.f, ru1 = v1 ? d.ru[off + j1] : 1.f;
        if (ckpt) {                                      // the state entering this pass
            float* crh = d.ckpt_rh + kc * d.n_slots + off;
            float* cru = d.ckpt_ru + kc * d.n_slots + off;
            if (v0) { crh[j0] = rh0; cru[j0] = ru0; }
            if (v1) { crh[j1] = rh1; cru[j1] = ru1; }
        }
        f32x2 rh = pk(rh0, rh1), ru = pk(ru0, ru1), B;
        const f32x2 cb = q == np - 1 ? pk(v0 ? p.c_b : 0.f, v1 ? p.c_b : 0.f) : k.CB;
        pass_a_pair(k, pk(t0.x, t1.x), pk(t0.y, t1.y), pk(t0.z, t1.z), pk(t0.w, t1.w), pk(km0, km1), cb, rh, ru, B,
                    part);
        if (v0) d.rh[off + j0] = lo_of(rh);
        if (v1) d.rh[off + j1] = hi_of(rh);
        s_am[q][tid] = ru;
        s_b[q][tid] = B;
    }
    if (ckpt && tid == 0) d.ckpt_lam[kc * d.n_rows + r] = lam0;
    const float lam = block_sum<BLOCK>(lo_of(part) + hi_of(part), red, 0) * (1.0f / (float)J);
    const f32x2 ILM = dup(rcp_refined(lam) * c.invM);
    bool clamp = false;
    for (int q = 0; q < np; ++q) {
        const f32x2 ru = fma2(s_b[q][tid], ILM, s_am[q][tid]);
        const int j0 = 2 * q * BLOCK + tid, j1 = j0 + BLOCK;
        if (j0 < J) {
            d.ru[off + j0] = lo_of(ru);
            clamp |= lo_of(ru) <= p.ru_floor;
        }
        if (j1 < J) {
            d.ru[off + j1] = hi_of(ru);
            clamp |= hi_of(ru) <= p.ru_floor;
        }
    }
    if (clamp) atomicOr(d.status, kFlagClamp);
    if (tid == 0) {
        d.lam[r] = lam;
        if (!(lam > 0.f) || !(lam <= FLT_MAX)) atomicOr(d.status, kFlagNonfinite);
    }
}

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
        if (h)
            solve_kernel<BLOCK, SPT><<<n_rows, BLOCK, 0, s>>>(d, n_iter, p, h);
        else if (n_iter == 1)
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
