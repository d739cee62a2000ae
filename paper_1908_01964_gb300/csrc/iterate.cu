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

// ---- packed pairs of FP32 values (sm_100+ f32x2 instructions) ---------------------
// Two slots are updated by one packed instruction: each half is an ordinary
// IEEE FP32 operation, so results equal the scalar code bit for bit.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float lo_of(f32x2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a;
}
__device__ __forceinline__ float hi_of(f32x2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return b;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 rcp2(f32x2 v) { return pk(rcp_approx(lo_of(v)), rcp_approx(hi_of(v))); }
__device__ __forceinline__ f32x2 dup(float v) { return pk(v, v); }

// One row with NP pairs of chunks (chunk k = slots k * BLOCK + threadIdx.x;
// pair q = chunks 2q and 2q + 1), kept in registers for all n_iter passes.
// Slots past the end of the row are padding that contributes exactly zero:
// r_h = 0 and r_u = 1 throughout (their r_h offset beta/(alpha+2) is replaced by 0).
template <int BLOCK, int NP>
__device__ __forceinline__ void accel_row(const DevState& d, int r, int J, int64_t off, const RowConst& c,
                                          int n_iter, const IterParams& p,
                                          float (*red)[BLOCK / 32 > 0 ? BLOCK / 32 : 1]) {
    const int tid = threadIdx.x;
    f32x2 tr[NP], ti[NP], sr[NP], si[NP], kapM[NP], rh[NP], ru[NP], B[NP];
    float cb_lo = p.c_b, cb_hi = p.c_b;                       // r_h offset of the last pair
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        float v[2][6];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = (2 * q + h) * BLOCK + tid;
            if (j < J) {
                const float4 t = d.inv4[off + j];
                v[h][0] = t.x; v[h][1] = t.y; v[h][2] = t.z; v[h][3] = t.w;
                v[h][4] = fmaf(d.kap[off + j], c.invM, p.ru_floor);   // r_u >= ru_floor by construction
                v[h][5] = d.rh[off + j];
            } else {
                v[h][0] = v[h][1] = v[h][2] = v[h][3] = 0.f;
                v[h][4] = 1.f;                                       // padding keeps r_u = 1
                v[h][5] = 0.f;
                if (q == NP - 1) { if (h == 0) cb_lo = 0.f; else cb_hi = 0.f; }
            }
        }
        tr[q] = pk(v[0][0], v[1][0]);
        ti[q] = pk(v[0][1], v[1][1]);
        sr[q] = pk(v[0][2], v[1][2]);
        si[q] = pk(v[0][3], v[1][3]);
        kapM[q] = pk(v[0][4], v[1][4]);
        rh[q] = pk(v[0][5], v[1][5]);
        const int j0 = 2 * q * BLOCK + tid, j1 = j0 + BLOCK;
        ru[q] = pk(j0 < J ? d.ru[off + j0] : 1.f, j1 < J ? d.ru[off + j1] : 1.f);
        B[q] = 0;
    }

    const f32x2 NSR = dup(-c.sab_re), NSI = dup(-c.sab_im), SI = dup(c.sab_im), SAB2 = dup(c.sab2);
    const f32x2 NITAA = dup(-c.inv_taa), TAAM = dup(c.taaM), CA2 = dup(p.c_a2);
    const f32x2 CB = dup(p.c_b), CB_LAST = pk(cb_lo, cb_hi);
    float lam = d.lam[r];
    const float invJ = 1.0f / (float)J;
    for (int it = 0; it < n_iter; ++it) {
        const float il = rcp_refined(lam);
        const f32x2 RTAA = dup(fmaf(c.sab2, il, c.taa));          // rho~_aa, Eq. (eq:traa_accel)
        const float slr = c.sab_re * il, sli = c.sab_im * il;
        const f32x2 SLR = dup(slr), SLI = dup(sli), NSLI = dup(-sli);
        f32x2 part = dup(0.f);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const f32x2 pr = fma2(SLR, sr[q], fma2(NSLI, si[q], tr[q]));
            const f32x2 pi = fma2(SLR, si[q], fma2(SLI, sr[q], ti[q]));
            const f32x2 g = mul2(rh[q], rcp2(fma2(rh[q], RTAA, ru[q])));
            const f32x2 cr = mul2(g, pr), ci = mul2(g, pi);
            const f32x2 Q = mul2(g, ru[q]);
            const f32x2 rhat = fma2(ci, ci, fma2(cr, cr, Q));
            const f32x2 dr = fma2(cr, NSR, fma2(ci, NSI, sr[q]));
            const f32x2 di = fma2(ci, NSR, fma2(cr, SI, si[q]));
            const f32x2 Bk = fma2(dr, dr, fma2(di, di, mul2(Q, SAB2)));
            part = fma2(Bk, rcp2(ru[q]), part);
            const f32x2 er = fma2(tr[q], NITAA, cr);
            const f32x2 ei = fma2(ti[q], NITAA, ci);
            ru[q] = fma2(TAAM, fma2(er, er, fma2(ei, ei, Q)), kapM[q]);    // A / M
            B[q] = Bk;
            rh[q] = fma2(rhat, CA2, q == NP - 1 ? CB_LAST : CB);
        }
        lam = block_sum<BLOCK>(lo_of(part) + hi_of(part), red, it & 1) * invJ;
        const f32x2 ILM = dup(rcp_refined(lam) * c.invM);
#pragma unroll
        for (int q = 0; q < NP; ++q) ru[q] = fma2(B[q], ILM, ru[q]);
    }

    bool clamp = false;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = (2 * q + h) * BLOCK + tid;
            if (j < J) {
                const float rhv = h ? hi_of(rh[q]) : lo_of(rh[q]);
                const float ruv = h ? hi_of(ru[q]) : lo_of(ru[q]);
                d.rh[off + j] = rhv;
                d.ru[off + j] = ruv;
                clamp |= (n_iter > 0) && (ruv <= p.ru_floor);
            }
        }
    }
    if (clamp) atomicOr(d.status, kFlagClamp);
    if (tid == 0) {
        d.lam[r] = lam;
        if (!(lam > 0.f) || !(lam <= FLT_MAX)) atomicOr(d.status, kFlagNonfinite);
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
