// Multichannel Wiener extraction of the target image, sm_103a.
//
// With the final parameters, the posterior mean of h_ij = a_i s_ij given x_ij
// (Sec. II-B-1 model; the filter is named in Sec. II-A and Sec. IV-B) is
//   h_ij = r_h a a^H (R^(x)_ij)^{-1} x_ij = w_ij a_i,
//   w_ij = r_h rho^(ax)_ij / (r_u + r_h rho^(aa)_i),
// where (R^(x))^{-1} a is expanded by Sherman-Morrison (Eq. (eq:rijxinv)) and
// rho^(ax) = tau^(ax) + sigma^(ab) sigma^(bx) / lambda, rho^(aa) = tau^(aa) +
// |sigma^(ab)|^2 / lambda (Sec. III-C-2).  One thread per slot; x is not read.
#include "rcscm_internal.cuh"

namespace rcscm {
namespace {

__global__ void __launch_bounds__(kSlotBlock) extract_kernel(DevState d, float2* __restrict__ h) {
    __shared__ float2 sa[kMaxM];
    __shared__ __align__(16) float2 sh[kSlotBlock * kMaxM];
    const BlockMap bm = d.bmap[blockIdx.x];
    RCSCM_CTA_CHECK(block_ok(d, bm), d.status);
    const RowDesc* rd = d.rows + bm.row;
    const int M = rd->M;
    const int J = rd->J;
    const int n = min(kSlotBlock, J - bm.j0);            // slots of this block
    const int t = threadIdx.x;
    // the slot's state and the row constants, in flight while a_i is staged
    const RowConst c = d.rc[bm.row];
    const float lam = d.lam[bm.row];
    float4 tv = make_float4(0.f, 0.f, 0.f, 0.f);
    float rh = 0.f, ru = 0.f;
    if (t < n) {
        const int64_t s = rd->slot_off + bm.j0 + t;
        tv = d.inv4[s];
        rh = d.rh[s];
        ru = d.ru[s];
    }
    if (threadIdx.x < M) sa[threadIdx.x] = d.a32[(size_t)bm.row * kMaxM + threadIdx.x];
    __syncthreads();
    if (t < n) {
        const float2 w = wiener_weight(c.taa, c.sab2, make_float2(c.sab_re, c.sab_im), lam, tv, rh, ru);
        for (int m = 0; m < M; ++m) sh[t * M + m] = cmul_exact(w, sa[m]);
    }
    __syncthreads();
    // write the block's n * M outputs (contiguous) with coalesced 16-byte stores when aligned
    float2* dst = h + rd->out_off + (int64_t)bm.j0 * M;
    const int nc = n * M;
    if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
        float4* d4 = reinterpret_cast<float4*>(dst);
        const float4* s4 = reinterpret_cast<const float4*>(sh);
        for (int e = t; e < nc / 2; e += blockDim.x) d4[e] = s4[e];
        if ((nc & 1) && t == 0) dst[nc - 1] = sh[nc - 1];
    } else {
        for (int e = t; e < nc; e += blockDim.x) dst[e] = sh[e];
    }
}

}  // namespace

cudaError_t launch_extract(const DevState& d, int n_blocks, float2* h_out, cudaStream_t s) {
    if (n_blocks <= 0) return cudaSuccess;
    extract_kernel<<<n_blocks, kSlotBlock, 0, s>>>(d, h_out);
    return cudaGetLastError();
}

}  // namespace rcscm
