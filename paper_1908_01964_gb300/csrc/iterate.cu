// Accelerated EM iteration kernel of the rank-constrained SCM estimator, sm_103a.
//
// accel_kernel<BLOCK, SPT>: second-stage accelerated rule (Algorithm 2,
//   Sec. III-C-2).  One CTA owns one row (utterance, frequency i) and keeps
//   the row's per-slot invariants and state in registers (SPT slots per
//   thread, slot j = k * BLOCK + threadIdx.x) for all n_iter passes, so the
//   only HBM traffic is one load and one store of the row per launch.  A pass:
//     pass A (per slot, old r~_h, r~_u, lambda~):
//       rho~_ax = tau_ax + sigma_ab sigma_bx / lambda~            (Sec. III-C-2)
//       gamma~  = r~_h / (r~_u + r~_h rho~_aa)                    Eq. (eq:tal)
//       c = gamma~ rho~_ax,  Q = gamma~ r~_u
//       r_h    <- (Q + |c|^2 + beta) / (alpha + 2)                Eq. (eq:1st_rh)
//       d = sigma_bx - c conj(sigma_ab)
//       B = Q |sigma_ab|^2 + |d|^2,  ell = B / r~_u               Eq. (eq:1st_li) summand
//       A = Q tau_aa + kappa + tau_aa |c - tau_ax / tau_aa|^2
//     lambda <- (1/J) sum_j ell_j  (fixed-order block reduction)  Eq. (eq:1st_li)
//     pass B: r_u <- (A + B / lambda) / M                         Eq. (eq:1st_ru)
//   Each CTA dispatches on its row's exact count of chunk pairs, and the slot
//   update runs on packed f32x2 instructions, one instruction for two slots.
//   Per-pass scalars use the hardware reciprocal with one Newton step instead of
//   IEEE division, and the r_u floor is part of kappa/M (all terms of r_u are
//   non-negative), so r_u >= ru_floor needs no extra operation.
//   The pass-B form is Eq. (eq:1st_ru) with R^u written as
//   gamma~ r~_u a a^H + (x - c a)(x - c a)^H and R_i^{-1} = R'^+ + b b^H / lambda
//   (Eq. (eq:riinv)): a sum of non-negative terms, so FP32 keeps r_u > 0 without
//   the cancellation of the printed difference form.
//
// solve_kernel / solve_persistent_kernel (FUSED): the same row body preceded by
// the per-slot invariants computed from x with the row's projection Phi (and
// stored, as the invariant kernel does) and followed by the Wiener filter
// h = w a with the final state, so setup's output, the passes and the target
// image need one launch and x is read once.  Results equal the separate
// kernels bit for bit (same device functions, same block).
//
// The naive rule (per-slot M x M inverse) is in naive.cu.
#include <float.h>

#include <algorithm>

#include "accel_common.cuh"

namespace rcscm {
namespace {

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
                                          FusedSmem* fs, void* row_smem) {
    RowState<BLOCK, NP> st(static_cast<RowSmem<BLOCK, NP>*>(row_smem));
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
    for (int it = 0; it < n_iter; ++it) st.pass(c, p, red, it & 1);
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
                                              FusedSmem* fs, void* row_smem) {
    const RowDesc* rd = d.rows + r;
    const int J = rd->J;
    const int64_t off = rd->slot_off;
    const RowConst c = d.rc[r];
    const int np = (J + 2 * BLOCK - 1) / (2 * BLOCK);     // chunk pairs, 1..SPT/2 (checked by the host)
    // The row's exact pair count selects the unrolled body (block-uniform branch).
#define RCSCM_ROW(N) \
    case N:          \
        if constexpr (2 * N <= SPT) accel_row<BLOCK, N, FUSED>(d, r, J, off, c, n_iter, p, red, h, fs, row_smem); \
        break;
    switch (np) {
        RCSCM_ROW(1) RCSCM_ROW(2) RCSCM_ROW(3) RCSCM_ROW(4) RCSCM_ROW(5) RCSCM_ROW(6) RCSCM_ROW(7) RCSCM_ROW(8)
        default: break;
    }
#undef RCSCM_ROW
}

// One CTA per row, rows in the order table (longest first).
template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK, accel_min_blocks(BLOCK, SPT)) accel_kernel(DevState d, int n_iter, IterParams p) {
    __shared__ float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    __shared__ RowSmem<BLOCK, SPT / 2> rs;
    accel_one_row<BLOCK, SPT, false>(d, d.order[blockIdx.x], n_iter, p, red, nullptr, nullptr, &rs);
}

template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK, accel_min_blocks(BLOCK, SPT)) solve_kernel(DevState d, int n_iter, IterParams p, float2* h) {
    __shared__ float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    __shared__ FusedSmem fs;
    __shared__ RowSmem<BLOCK, SPT / 2> rs;
    accel_one_row<BLOCK, SPT, true>(d, d.order[blockIdx.x], n_iter, p, red, h, &fs, &rs);
}

// Persistent variants: a fixed grid of resident CTAs takes rows from the order
// table through an atomic counter (dynamic longest-first scheduling).
template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK, accel_min_blocks(BLOCK, SPT)) accel_persistent_kernel(DevState d, int n_iter, IterParams p, int n_rows) {
    __shared__ float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    __shared__ RowSmem<BLOCK, SPT / 2> rs;
    __shared__ int s_next;
    for (;;) {
        __syncthreads();                    // every thread is done with s_next and the previous row
        if (threadIdx.x == 0) s_next = atomicAdd(d.counter, 1);
        __syncthreads();
        const int k = s_next;
        if (k >= n_rows) break;
        accel_one_row<BLOCK, SPT, false>(d, d.order[k], n_iter, p, red, nullptr, nullptr, &rs);
    }
}

template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK, accel_min_blocks(BLOCK, SPT)) solve_persistent_kernel(DevState d, int n_iter, IterParams p, int n_rows,
                                                                 float2* h) {
    __shared__ float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    __shared__ FusedSmem fs;
    __shared__ RowSmem<BLOCK, SPT / 2> rs;
    __shared__ int s_next;
    for (;;) {
        __syncthreads();                    // every thread is done with s_next, fs and the previous row
        if (threadIdx.x == 0) s_next = atomicAdd(d.counter, 1);
        __syncthreads();
        const int k = s_next;
        if (k >= n_rows) break;
        accel_one_row<BLOCK, SPT, true>(d, d.order[k], n_iter, p, red, h, &fs, &rs);
    }
}

template <class Kernel>
int resident_per_sm(Kernel k, int block) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, 0) != cudaSuccess) n = 1;
    return n > 0 ? n : 1;
}

template <int BLOCK, int SPT>
cudaError_t launch_accel_t(const DevState& d, int n_rows, int n_iter, const IterParams& p, bool persistent,
                           float2* h, cudaStream_t s) {
    if (!persistent) {
        if (h)
            solve_kernel<BLOCK, SPT><<<n_rows, BLOCK, 0, s>>>(d, n_iter, p, h);
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

template <int BLOCK>
cudaError_t launch_accel_b(const DevState& d, int n_rows, int spt, int n_iter, const IterParams& p, bool persistent,
                           float2* h, cudaStream_t s) {
    if (spt <= 4) return launch_accel_t<BLOCK, 4>(d, n_rows, n_iter, p, persistent, h, s);
    if constexpr (accel_max_spt(BLOCK) >= 8)
        if (spt <= 8) return launch_accel_t<BLOCK, 8>(d, n_rows, n_iter, p, persistent, h, s);
    if constexpr (accel_max_spt(BLOCK) >= 16)
        if (spt <= 16) return launch_accel_t<BLOCK, 16>(d, n_rows, n_iter, p, persistent, h, s);
    return cudaErrorInvalidValue;
}

}  // namespace

// The kernel keeps SPT = the smallest of {4, 8, 16} slots per thread that
// covers the longest row, so its register budget matches the work list.
cudaError_t launch_accel(const DevState& d, int n_rows, int max_j, int block, int n_iter,
                         const IterParams& p, bool persistent, cudaStream_t s, float2* h) {
    if (n_rows <= 0) return cudaSuccess;
    if (block == 0) block = accel_default_block(max_j);
    const int need = (max_j + block - 1) / block;
    if (need > accel_max_spt(block)) return cudaErrorInvalidValue;
    switch (block) {
        case 32: return launch_accel_b<32>(d, n_rows, need, n_iter, p, persistent, h, s);
        case 64: return launch_accel_b<64>(d, n_rows, need, n_iter, p, persistent, h, s);
        case 128: return launch_accel_b<128>(d, n_rows, need, n_iter, p, persistent, h, s);
        case 256: return launch_accel_b<256>(d, n_rows, need, n_iter, p, persistent, h, s);
        case 512: return launch_accel_b<512>(d, n_rows, need, n_iter, p, persistent, h, s);
        case 1024: return launch_accel_b<1024>(d, n_rows, need, n_iter, p, persistent, h, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rcscm
