// First-stage accelerated rule (Algorithm 1, Sec. III-C-1), sm_103a.
//
// The first stage keeps the per-frequency inverses R~_i^{-1}, R_i^{-1} and
// evaluates the per-slot quadratic forms of Eqs. (eq:traa)-(eq:rxx) from x_ij
// at every pass: O(M^2) work per slot and pass (Table I), against O(1) for the
// second stage, which computes tau_ax, sigma_bx and kappa once.  Here the
// inverses are applied through Eq. (eq:riinv), R_i^{-1} = (R'_i)^+ +
// b b^H / lambda_i, with (R'_i)^+ in the whitened form of the per-frequency
// projection Phi_i, so that every pass re-projects x (rho~_ax = tau_ax +
// sigma_ab sigma_bx / lambda~ with tau_ax = Phi_0 x, and the r_u numerator
// (x - c a)^H R_i^{-1} (x - c a) = kappa + tau_aa |c - tau_ax / tau_aa|^2 +
// |sigma_bx - c conj(sigma_ab)|^2 / lambda as a sum of squares) and then runs
// the scalar updates of the pass.  The results equal the second-stage kernel's
// bit for bit at the same block size, which is the paper's statement that the
// two stages are the same algorithm, made exact; the cost is the first stage's.
#include <float.h>

#include "accel_common.cuh"

namespace rcscm {
namespace {

template <int BLOCK, int NP>
__device__ __forceinline__ void accel1_row(const DevState& d, int r, int n_iter, const IterParams& p,
                                           float (*red)[BLOCK / 32], float2* sphi) {
    const RowDesc* rd = d.rows + r;
    const int J = rd->J;
    const int M = rd->M;
    const int64_t off = rd->slot_off;
    const RowConst c = d.rc[r];
    for (int e = threadIdx.x; e < M * M; e += BLOCK) sphi[e] = d.phi[(size_t)r * 64 + e];
    __syncthreads();
    const float2* x = rd->x;
    auto project = [&](int j, float4& t, float& kap) { project_slot_m(M, sphi, x + (int64_t)j * M, t, kap); };
    RowState<BLOCK, NP> st;
    st.load_inv_with(J, c, p, project);
    st.load_state(d.rh + off, d.ru + off, d.lam[r]);
    for (int it = 0; it < n_iter; ++it) {
        if (it > 0) st.load_inv_with(J, c, p, project);    // the quadratic forms, again from x
        st.pass(c, p, red, it & 1);
    }
    st.store_state(d.rh + off, d.ru + off);
    if (n_iter > 0 && st.any_clamp(p.ru_floor)) atomicOr(d.status, kFlagClamp);
    if (threadIdx.x == 0) {
        d.lam[r] = st.lam;
        if (!(st.lam > 0.f) || !(st.lam <= FLT_MAX)) atomicOr(d.status, kFlagNonfinite);
    }
}

// One CTA per row; the row's exact count of chunk pairs selects the body.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) accel1_kernel(DevState d, int n_iter, IterParams p) {
    __shared__ float red[2][BLOCK / 32];
    __shared__ float2 sphi[kMaxM * kMaxM];
    const int r = d.order[blockIdx.x];
    RCSCM_CTA_CHECK(row_ok(d, r, 8 * BLOCK), d.status);
    const int np = (d.rows[r].J + 2 * BLOCK - 1) / (2 * BLOCK);
    switch (np) {
        case 1: accel1_row<BLOCK, 1>(d, r, n_iter, p, red, sphi); break;
        case 2: accel1_row<BLOCK, 2>(d, r, n_iter, p, red, sphi); break;
        case 3: accel1_row<BLOCK, 3>(d, r, n_iter, p, red, sphi); break;
        case 4: accel1_row<BLOCK, 4>(d, r, n_iter, p, red, sphi); break;
        default: break;
    }
}

}  // namespace

// Rows of up to 2048 frames run with 256 threads, up to 4096 with 512 (8 slots
// per thread at most).
int accel1_block(int max_j) { return max_j <= 2048 ? 256 : (max_j <= 4096 ? 512 : 0); }

cudaError_t launch_accel1(const DevState& d, int n_rows, int max_j, int n_iter, const IterParams& p,
                          cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    switch (accel1_block(max_j)) {
        case 256: accel1_kernel<256><<<n_rows, 256, 0, s>>>(d, n_iter, p); break;
        case 512: accel1_kernel<512><<<n_rows, 512, 0, s>>>(d, n_iter, p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace rcscm
