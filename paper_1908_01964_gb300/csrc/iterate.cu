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
#include "rcscm_internal.cuh"

namespace rcscm {

// Defined in iterate_impl.cuh, instantiated once per shape by iterate_inst.cu.
template <int BLOCK, int SPT>
cudaError_t launch_accel_t(const DevState& d, int n_rows, int n_iter, const IterParams& p, bool persistent,
                           float2* h, cudaStream_t s);

namespace {

template <int BLOCK>
cudaError_t launch_accel_b(const DevState& d, int n_rows, int spt, int n_iter, const IterParams& p, bool persistent,
                           float2* h, cudaStream_t s) {
    if (spt <= 4) return launch_accel_t<BLOCK, 4>(d, n_rows, n_iter, p, persistent, h, s);
    if constexpr (accel_max_spt(BLOCK) >= 8)
        if (spt <= 8) return launch_accel_t<BLOCK, 8>(d, n_rows, n_iter, p, persistent, h, s);
    return cudaErrorInvalidValue;
}

}  // namespace

// The kernel keeps SPT = the smallest of {4, 8} slots per thread that
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
