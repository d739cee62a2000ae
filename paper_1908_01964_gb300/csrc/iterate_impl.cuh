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

// Shared memory of the fused row body: the row's projection and steering vector, and
// the Wiener weights of its SLOTS slots.
template <int SLOTS>
struct FusedSmem {
    float2 phi[kMaxM * kMaxM];
    float2 a[kMaxM];
    float2 w[SLOTS];
};

// The fused prologue: invariants of the row's slots j = threadIdx.x + k BLOCK, projected
// with Phi (shared memory) and stored to the context's arrays.  The prologue and the
// epilogue run once per row, so their code is fetched cold: a short loop with M fixed for
// the row (loads of G slots issued together) instead of a body unrolled over the slots
// with a dispatch on M in each, which took longer to fetch than to run.
template <int BLOCK, int M>
__device__ __forceinline__ void project_row(const float2* phi, const float2* x, int J, float4* inv, float* kap) {
    constexpr int G = M <= 4 ? 4 : 2;
#pragma unroll 1
    for (int j0 = threadIdx.x; j0 < J; j0 += G * BLOCK) {
        float2 xv[G][M];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int j = j0 + g * BLOCK;
#pragma unroll
            for (int n = 0; n < M; ++n) xv[g][n] = j < J ? x[(int64_t)j * M + n] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int j = j0 + g * BLOCK;
            if (j < J) {
                float4 t;
                float k;
                project_vals<M>(phi, xv[g], t, k);
                inv[j] = t;
                kap[j] = k;
            }
        }
    }
}

template <int BLOCK>
__device__ __forceinline__ void project_row_m(int M, const float2* phi, const float2* x, int J, float4* inv,
                                              float* kap) {
    switch (M) {
        case 2: project_row<BLOCK, 2>(phi, x, J, inv, kap); break;
        case 3: project_row<BLOCK, 3>(phi, x, J, inv, kap); break;
        case 4: project_row<BLOCK, 4>(phi, x, J, inv, kap); break;
        case 5: project_row<BLOCK, 5>(phi, x, J, inv, kap); break;
        case 6: project_row<BLOCK, 6>(phi, x, J, inv, kap); break;
        case 7: project_row<BLOCK, 7>(phi, x, J, inv, kap); break;
        default: project_row<BLOCK, 8>(phi, x, J, inv, kap); break;
    }
}

// One row, all n_iter passes with the row held in registers (RowState).
// FUSED: invariants from x first, Wiener output h last (h != nullptr).
template <int BLOCK, int NP, bool FUSED, class FS>
__device__ __forceinline__ void accel_row(const DevState& d, int r, int J, int64_t off, const RowConst& c,
                                          int n_iter, const IterParams& p,
                                          float (*red)[BLOCK / 32 > 0 ? BLOCK / 32 : 1], float2* __restrict__ h,
                                          FS* fs) {
    RowState<BLOCK, NP> st;
    const RowDesc* rd = d.rows + r;
    if constexpr (FUSED) {
        const int M = rd->M;
        for (int e = threadIdx.x; e < M * M; e += BLOCK) fs->phi[e] = d.phi[(size_t)r * 64 + e];
        if (threadIdx.x < M) fs->a[threadIdx.x] = d.a32[(size_t)r * kMaxM + threadIdx.x];
        __syncthreads();
        project_row_m<BLOCK>(M, fs->phi, rd->x, J, d.inv4 + off, d.kap + off);
        st.load_inv(d, off, J, c, p);                          // this thread's own slots, as just stored
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
#pragma unroll
        for (int k = 0; k < 2 * NP; ++k) {           // the weights of this thread's slots
            const int j = k * BLOCK + threadIdx.x;
            if (j < J) {
                const float4 t = make_float4(k & 1 ? hi_of(st.tr[k >> 1]) : lo_of(st.tr[k >> 1]),
                                             k & 1 ? hi_of(st.ti[k >> 1]) : lo_of(st.ti[k >> 1]),
                                             k & 1 ? hi_of(st.sr[k >> 1]) : lo_of(st.sr[k >> 1]),
                                             k & 1 ? hi_of(st.si[k >> 1]) : lo_of(st.si[k >> 1]));
                fs->w[j] = wiener_weight(c.taa, c.sab2, sab, st.lam, t, st.rh_of(k), st.ru_of(k));
            }
        }
        __syncthreads();
        // the row's J x M outputs are contiguous: entry e = j M + m, consecutive threads on
        // consecutive entries (coalesced stores)
        float2* hrow = h + rd->out_off;
        const int n_out = J * M, dj = BLOCK / M, dm = BLOCK - (BLOCK / M) * M;
        int j = threadIdx.x / M, m = threadIdx.x - (threadIdx.x / M) * M;
#pragma unroll 4
        for (int e = threadIdx.x; e < n_out; e += BLOCK) {
            hrow[e] = cmul_exact(fs->w[j], fs->a[m]);
            j += dj;
            m += dm;
            if (m >= M) {
                m -= M;
                ++j;
            }
        }
    }
}

template <int BLOCK, int SPT, bool FUSED, class FS>
__device__ __forceinline__ void accel_one_row(const DevState& d, int r, int n_iter, const IterParams& p,
                                              float (*red)[BLOCK / 32 > 0 ? BLOCK / 32 : 1], float2* h,
                                              FS* fs) {
    const RowDesc* rd = d.rows + r;
    const int J = rd->J;
    const int64_t off = rd->slot_off;
    const RowConst c = d.rc[r];
    const int np = (J + 2 * BLOCK - 1) / (2 * BLOCK);     // chunk pairs, 1..SPT/2 (checked by the host)
    // The row's exact pair count selects the unrolled body (block-uniform branch).
#define RCSCM_ROW(N) \
    case N:          \
        if constexpr (2 * N <= SPT) accel_row<BLOCK, N, FUSED, FS>(d, r, J, off, c, n_iter, p, red, h, fs); \
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
    __shared__ __align__(16) float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    RCSCM_CTA_CHECK(row_ok(d, d.order[blockIdx.x], BLOCK * SPT), d.status);
    accel_one_row<BLOCK, SPT, false>(d, d.order[blockIdx.x], n_iter, p, red, nullptr,
                                     static_cast<FusedSmem<1>*>(nullptr));
}

// Launched as a programmatic dependent of the per-frequency setup: a CTA may start while
// the setup still runs.  Before griddepcontrol.wait it touches only the caller's inputs,
// and only to ask L2 for them (prefetch: no value is read, so a preceding kernel that
// writes them is still seen); every setup output is read after the wait.
template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK, solve_min_blocks(BLOCK, SPT)) solve_kernel(DevState d, int n_iter, IterParams p, float2* h) {
    __shared__ __align__(16) float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    __shared__ FusedSmem<BLOCK * SPT> fs;
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
    __shared__ __align__(16) float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    __shared__ int s_next;
    for (;;) {
        __syncthreads();                    // every thread is done with s_next and the previous row
        if (threadIdx.x == 0) s_next = atomicAdd(d.counter, 1);
        __syncthreads();
        const int k = s_next;
        if (k >= n_rows) break;
        RCSCM_CTA_CHECK(row_ok(d, d.order[k], BLOCK * SPT), d.status);
        accel_one_row<BLOCK, SPT, false>(d, d.order[k], n_iter, p, red, nullptr, static_cast<FusedSmem<1>*>(nullptr));
    }
}

template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK, solve_min_blocks(BLOCK, SPT)) solve_persistent_kernel(DevState d, int n_iter, IterParams p, int n_rows,
                                                                 float2* h) {
    __shared__ __align__(16) float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    __shared__ FusedSmem<BLOCK * SPT> fs;
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
