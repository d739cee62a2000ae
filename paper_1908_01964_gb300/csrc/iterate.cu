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
// The naive rule (per-slot M x M inverse) is in naive.cu.
#include <float.h>

#include <algorithm>

#include "accel_common.cuh"

namespace rcscm {
namespace {

// One row, all n_iter passes with the row held in registers (RowState).
template <int BLOCK, int NP>
__device__ __forceinline__ void accel_row(const DevState& d, int r, int J, int64_t off, const RowConst& c,
                                          int n_iter, const IterParams& p,
                                          float (*red)[BLOCK / 32 > 0 ? BLOCK / 32 : 1]) {
    RowState<BLOCK, NP> st;
    st.load_inv(d, off, J, c, p);
    st.load_state(d.rh + off, d.ru + off, d.lam[r]);
    for (int it = 0; it < n_iter; ++it) st.pass(c, p, red, it & 1);
    st.store_state(d.rh + off, d.ru + off);
    if (n_iter > 0 && st.any_clamp(p.ru_floor)) atomicOr(d.status, kFlagClamp);
    if (threadIdx.x == 0) {
        d.lam[r] = st.lam;
        if (!(st.lam > 0.f) || !(st.lam <= FLT_MAX)) atomicOr(d.status, kFlagNonfinite);
    }
}

template <int BLOCK, int SPT>
__device__ __forceinline__ void accel_one_row(const DevState& d, int r, int n_iter, const IterParams& p,
                                              float (*red)[BLOCK / 32 > 0 ? BLOCK / 32 : 1]) {
    const RowDesc* rd = d.rows + r;
    const int J = rd->J;
    const int64_t off = rd->slot_off;
    const RowConst c = d.rc[r];
    const int np = (J + 2 * BLOCK - 1) / (2 * BLOCK);     // chunk pairs, 1..SPT/2 (checked by the host)
    // The row's exact pair count selects the unrolled body (block-uniform branch).
#define RCSCM_ROW(N) \
    case N:          \
        if constexpr (2 * N <= SPT) accel_row<BLOCK, N>(d, r, J, off, c, n_iter, p, red); \
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
    accel_one_row<BLOCK, SPT>(d, d.order[blockIdx.x], n_iter, p, red);
}

// Persistent variant: a fixed grid of resident CTAs takes rows from the order
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
        accel_one_row<BLOCK, SPT>(d, d.order[k], n_iter, p, red);
    }
}

template <int BLOCK, int SPT>
cudaError_t launch_accel_t(const DevState& d, int n_rows, int n_iter, const IterParams& p, bool persistent,
                           cudaStream_t s) {
    if (!persistent) {
        accel_kernel<BLOCK, SPT><<<n_rows, BLOCK, 0, s>>>(d, n_iter, p);
        return cudaGetLastError();
    }
    static const int per_sm = [] {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, accel_persistent_kernel<BLOCK, SPT>, BLOCK, 0) !=
            cudaSuccess)
            n = 1;
        return n > 0 ? n : 1;
    }();
    const int grid = std::min(n_rows, per_sm * d.n_sm);
    cudaError_t e = cudaMemsetAsync(d.counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    accel_persistent_kernel<BLOCK, SPT><<<grid, BLOCK, 0, s>>>(d, n_iter, p, n_rows);
    return cudaGetLastError();
}

template <int BLOCK>
cudaError_t launch_accel_b(const DevState& d, int n_rows, int spt, int n_iter, const IterParams& p, bool persistent,
                           cudaStream_t s) {
    if (spt <= 4) return launch_accel_t<BLOCK, 4>(d, n_rows, n_iter, p, persistent, s);
    if constexpr (accel_max_spt(BLOCK) >= 8)
        if (spt <= 8) return launch_accel_t<BLOCK, 8>(d, n_rows, n_iter, p, persistent, s);
    if constexpr (accel_max_spt(BLOCK) >= 16)
        if (spt <= 16) return launch_accel_t<BLOCK, 16>(d, n_rows, n_iter, p, persistent, s);
    return cudaErrorInvalidValue;
}

}  // namespace

// The kernel keeps SPT = the smallest of {4, 8, 16} slots per thread that
// covers the longest row, so its register budget matches the work list.
cudaError_t launch_accel(const DevState& d, int n_rows, int max_j, int block, int n_iter,
                         const IterParams& p, bool persistent, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    if (block == 0) block = accel_default_block(max_j);
    const int need = (max_j + block - 1) / block;
    if (need > accel_max_spt(block)) return cudaErrorInvalidValue;
    switch (block) {
        case 32: return launch_accel_b<32>(d, n_rows, need, n_iter, p, persistent, s);
        case 64: return launch_accel_b<64>(d, n_rows, need, n_iter, p, persistent, s);
        case 128: return launch_accel_b<128>(d, n_rows, need, n_iter, p, persistent, s);
        case 256: return launch_accel_b<256>(d, n_rows, need, n_iter, p, persistent, s);
        case 512: return launch_accel_b<512>(d, n_rows, need, n_iter, p, persistent, s);
        case 1024: return launch_accel_b<1024>(d, n_rows, need, n_iter, p, persistent, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rcscm
