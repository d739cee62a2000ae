// Objective of the rank-constrained SCM model, sm_103a: the observed-data log
// posterior of the generative model of Sec. II-B-1 with the current state,
// constants dropped,
//   L = sum_ij [ -log det R^(x)_ij - x^H (R^(x)_ij)^{-1} x - (alpha+1) log r_h - beta / r_h ],
//   R^(x) = r_h a a^H + r_u R,  R = R' + lambda b b^H,
// which every EM pass leaves non-decreasing.  Closed forms through the
// per-slot invariants (Eq. (eq:riinv) and Sherman-Morrison, Eq. (eq:rijxinv)):
//   log det R^(x) = M log r_u + log lambda + log pdet R' + log(1 + r_h rho_aa / r_u),
//   x^H (R^(x))^{-1} x = (1/r_u) [ rho_xx - |rho_ax|^2 / rho_aa
//                                 + |rho_ax|^2 r_u / (rho_aa (r_u + r_h rho_aa)) ],
//   rho_xx - |rho_ax|^2 / rho_aa = kappa + |tau_aa sigma_bx - conj(sigma_ab) tau_ax|^2 / (lambda tau_aa rho_aa),
// the last identity being Lagrange's identity in the R^{-1} inner product; every
// term is non-negative, so FP32 evaluation has no cancellation.  Per-slot terms
// in FP32, sums in FP64 in a fixed order (deterministic).
#include <float.h>

#include "rcscm_internal.cuh"

namespace rcscm {
namespace {

__global__ void __launch_bounds__(kSlotBlock) objective_kernel(DevState d, float alpha1, float beta) {
    __shared__ double red[kSlotBlock / 32];
    const BlockMap bm = d.bmap[blockIdx.x];
    RCSCM_CTA_CHECK(block_ok(d, bm), d.status);
    const RowDesc* rd = d.rows + bm.row;
    const int M = rd->M;
    const int J = rd->J;
    const int n = min(kSlotBlock, J - bm.j0);
    const int t = threadIdx.x;
    const RowConst c = d.rc[bm.row];
    const float lam = d.lam[bm.row];
    double v = 0.0;
    if (t < n) {
        const int64_t s = rd->slot_off + bm.j0 + t;
        const float4 tv = d.inv4[s];
        const float kap = d.kap[s];
        const float rh = d.rh[s], ru = d.ru[s];
        const float il = 1.0f / lam;
        const float2 tax = make_float2(tv.x, tv.y), sbx = make_float2(tv.z, tv.w);
        const float2 sab = make_float2(c.sab_re, c.sab_im);
        const float raa = fmaf(c.sab2, il, c.taa);
        const float2 rax = cadd(tax, cscale(cmul(sab, sbx), il));
        const float den = fmaf(rh, raa, ru);
        const float2 det = csub(cscale(sbx, c.taa), cmul(cconj(sab), tax));
        const float perp = kap + cabs2(det) * il / (c.taa * raa);
        const float quad = (perp + cabs2(rax) * ru / (raa * den)) / ru;
        const float logdet = (float)M * logf(ru) + log1pf(rh * raa / ru);
        v = (double)(-logdet - quad - alpha1 * logf(rh) - beta / rh);
    }
    if (t == 0 && bm.j0 == 0) {           // row constants: -J (log lambda + log pdet R')
        double lpd = 0.0;
        for (int k = 1; k < M; ++k) lpd += log(d.mu[(size_t)bm.row * kMaxM + k]);
        v -= (double)J * (log((double)lam) + lpd);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) red[t >> 5] = v;
    __syncthreads();
    if (t == 0) {
        double tot = 0.0;
        for (int w = 0; w < kSlotBlock / 32; ++w) tot += red[w];
        d.obj_part[blockIdx.x] = tot;
    }
}

// One CTA per utterance: thread t sums partials t, t + 256, ... in order, then a
// fixed tree over the threads (deterministic for a given block count).
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads) objective_sum_kernel(const double* __restrict__ part,
                                                                   const int* __restrict__ first_block,
                                                                   double* __restrict__ out) {
    __shared__ double red[kSumThreads];
    const int p = blockIdx.x;
    double s = 0.0;
    for (int b = first_block[p] + threadIdx.x; b < first_block[p + 1]; b += kSumThreads) s += part[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = kSumThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[p] = red[0];
}

}  // namespace

cudaError_t launch_objective(const DevState& d, int n_blocks, const IterParams& p, double alpha, double beta,
                             const int* first_block, int n_probs, double* out, cudaStream_t s) {
    (void)p;
    if (n_blocks <= 0) return cudaSuccess;
    objective_kernel<<<n_blocks, kSlotBlock, 0, s>>>(d, (float)(alpha + 1.0), (float)beta);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    objective_sum_kernel<<<n_probs, kSumThreads, 0, s>>>(d.obj_part, first_block, out);
    return cudaGetLastError();
}

}  // namespace rcscm
