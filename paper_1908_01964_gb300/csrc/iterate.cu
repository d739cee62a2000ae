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
//   Each CTA dispatches on its row's exact chunk count NK = ceil(J / BLOCK), so
//   only the last chunk carries a validity mask, and per-pass scalars use the
//   hardware reciprocal with one Newton step instead of IEEE division.
//   The pass-B form is Eq. (eq:1st_ru) with R^u written as
//   gamma~ r~_u a a^H + (x - c a)(x - c a)^H and R_i^{-1} = R'^+ + b b^H / lambda
//   (Eq. (eq:riinv)): a sum of non-negative terms, so FP32 keeps r_u > 0 without
//   the cancellation of the printed difference form.
//
// The naive rule (per-slot M x M inverse) is in naive.cu.
#include <float.h>

#include "rcscm_internal.cuh"

namespace rcscm {
namespace {

// Sum over the block with one __syncthreads; `red` is double-buffered by the
// pass parity so consecutive passes never race on it.  Every thread returns
// the same, order-fixed value.  A single-warp block needs no shared memory.
template <int BLOCK>
__device__ __forceinline__ float block_sum(float v, float (*red)[BLOCK / 32 > 0 ? BLOCK / 32 : 1], int parity) {
    constexpr int NW = BLOCK / 32;
    v = warp_sum(v);
    if constexpr (NW == 1) {
        return v;
    } else {
        const int lane = threadIdx.x & 31;
        if (lane == 0) red[parity][threadIdx.x >> 5] = v;
        __syncthreads();
        float t = red[parity][lane & (NW - 1)];
#pragma unroll
        for (int o = NW / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        return t;
    }
}

// 1/x for positive normal x: hardware approximation refined by one Newton step.
__device__ __forceinline__ float rcp_refined(float x) {
    const float r = rcp_approx(x);
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}

// One row, NK chunks of BLOCK slots (slot j = k * BLOCK + threadIdx.x), kept in
// registers for all n_iter passes.  Chunks 0..NK-2 are full; the last may be partial.
template <int BLOCK, int NK>
__device__ __forceinline__ void accel_row(const DevState& d, int r, int J, int64_t off, const RowConst& c,
                                          int n_iter, const IterParams& p,
                                          float (*red)[BLOCK / 32 > 0 ? BLOCK / 32 : 1]) {
    const int tid = threadIdx.x;
    const bool last_ok = (NK - 1) * BLOCK + tid < J;
    float4 t[NK];
    float kapM[NK], rh[NK], ru[NK], B[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int j = k * BLOCK + tid;
        if (k < NK - 1 || last_ok) {
            t[k] = d.inv4[off + j];
            kapM[k] = d.kap[off + j] * c.invM;
            rh[k] = d.rh[off + j];
            ru[k] = d.ru[off + j];
        } else {
            t[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            kapM[k] = 0.f;
            rh[k] = 0.f;
            ru[k] = 1.f;
        }
        B[k] = 0.f;
    }

    float lam = d.lam[r];
    const float invJ = 1.0f / (float)J;
    for (int it = 0; it < n_iter; ++it) {
        const float il = rcp_refined(lam);
        const float rtaa = fmaf(c.sab2, il, c.taa);          // rho~_aa, Eq. (eq:traa_accel)
        const float slr = c.sab_re * il, sli = c.sab_im * il;
        float part = 0.f;
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const float pr = fmaf(slr, t[k].z, fmaf(-sli, t[k].w, t[k].x));
            const float pi = fmaf(slr, t[k].w, fmaf(sli, t[k].z, t[k].y));
            const float g = rh[k] * rcp_approx(fmaf(rh[k], rtaa, ru[k]));
            const float cr = g * pr, ci = g * pi;
            const float Q = g * ru[k];
            const float rhat = fmaf(ci, ci, fmaf(cr, cr, Q));
            const float dr = fmaf(-cr, c.sab_re, fmaf(-ci, c.sab_im, t[k].z));
            const float di = fmaf(-ci, c.sab_re, fmaf(cr, c.sab_im, t[k].w));
            const float Bk = fmaf(dr, dr, fmaf(di, di, Q * c.sab2));
            if (k < NK - 1 || last_ok) part = fmaf(Bk, rcp_approx(ru[k]), part);
            const float er = fmaf(-t[k].x, c.inv_taa, cr);
            const float ei = fmaf(-t[k].y, c.inv_taa, ci);
            ru[k] = fmaf(c.taaM, fmaf(er, er, fmaf(ei, ei, Q)), kapM[k]);    // A / M
            B[k] = Bk;
            rh[k] = fmaf(rhat, p.c_a2, p.c_b);
        }
        lam = block_sum<BLOCK>(part, red, it & 1) * invJ;
        const float ilM = rcp_refined(lam) * c.invM;
#pragma unroll
        for (int k = 0; k < NK; ++k) ru[k] = fmaxf(fmaf(B[k], ilM, ru[k]), p.ru_floor);
    }

    bool clamp = false;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        if (k < NK - 1 || last_ok) {
            const int j = k * BLOCK + tid;
            d.rh[off + j] = rh[k];
            d.ru[off + j] = ru[k];
            clamp |= (n_iter > 0) && (ru[k] <= p.ru_floor);
        }
    }
    if (clamp) atomicOr(d.status, kFlagClamp);
    if (tid == 0) {
        d.lam[r] = lam;
        if (!(lam > 0.f) || !(lam <= FLT_MAX)) atomicOr(d.status, kFlagNonfinite);
    }
}

template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK) accel_kernel(DevState d, int n_iter, IterParams p) {
    __shared__ float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    const int r = d.order[blockIdx.x];
    const RowDesc* rd = d.rows + r;
    const int J = rd->J;
    const int64_t off = rd->slot_off;
    const RowConst c = d.rc[r];
    const int nk = (J + BLOCK - 1) / BLOCK;     // 1..SPT, checked by the host
    // The row's exact chunk count selects the unrolled body (block-uniform branch).
#define RCSCM_ROW(N) \
    case N:          \
        if constexpr (N <= SPT) accel_row<BLOCK, N>(d, r, J, off, c, n_iter, p, red); \
        break;
    switch (nk) {
        RCSCM_ROW(1) RCSCM_ROW(2) RCSCM_ROW(3) RCSCM_ROW(4) RCSCM_ROW(5) RCSCM_ROW(6) RCSCM_ROW(7) RCSCM_ROW(8)
        RCSCM_ROW(9) RCSCM_ROW(10) RCSCM_ROW(11) RCSCM_ROW(12) RCSCM_ROW(13) RCSCM_ROW(14) RCSCM_ROW(15)
        RCSCM_ROW(16)
        default: break;
    }
#undef RCSCM_ROW
}

template <int BLOCK, int SPT>
cudaError_t launch_accel_t(const DevState& d, int n_rows, int n_iter, const IterParams& p, cudaStream_t s) {
    accel_kernel<BLOCK, SPT><<<n_rows, BLOCK, 0, s>>>(d, n_iter, p);
    return cudaGetLastError();
}

template <int BLOCK>
cudaError_t launch_accel_b(const DevState& d, int n_rows, int spt, int n_iter, const IterParams& p, cudaStream_t s) {
    if (spt <= 4) return launch_accel_t<BLOCK, 4>(d, n_rows, n_iter, p, s);
    if constexpr (accel_max_spt(BLOCK) >= 8)
        if (spt <= 8) return launch_accel_t<BLOCK, 8>(d, n_rows, n_iter, p, s);
    if constexpr (accel_max_spt(BLOCK) >= 16)
        if (spt <= 16) return launch_accel_t<BLOCK, 16>(d, n_rows, n_iter, p, s);
    return cudaErrorInvalidValue;
}

}  // namespace

// The kernel keeps SPT = the smallest of {4, 8, 16} slots per thread that
// covers the longest row, so its register budget matches the work list.
cudaError_t launch_accel(const DevState& d, int n_rows, int max_j, int block, int n_iter,
                         const IterParams& p, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    if (block == 0) block = accel_default_block(max_j);
    const int need = (max_j + block - 1) / block;
    if (need > accel_max_spt(block)) return cudaErrorInvalidValue;
    switch (block) {
        case 32: return launch_accel_b<32>(d, n_rows, need, n_iter, p, s);
        case 64: return launch_accel_b<64>(d, n_rows, need, n_iter, p, s);
        case 128: return launch_accel_b<128>(d, n_rows, need, n_iter, p, s);
        case 256: return launch_accel_b<256>(d, n_rows, need, n_iter, p, s);
        case 512: return launch_accel_b<512>(d, n_rows, need, n_iter, p, s);
        case 1024: return launch_accel_b<1024>(d, n_rows, need, n_iter, p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rcscm
