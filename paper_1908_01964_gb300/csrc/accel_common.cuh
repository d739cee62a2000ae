// Shared device code of the accelerated rule (forward kernel in iterate.cu,
// adjoint kernel in adjoint.cu): packed f32x2 helpers, the block reduction and
// the register-resident state of one row with one EM pass of Algorithm 2
// (Sec. III-C-2).  Both kernels run the pass through this code, so the
// adjoint's recomputation from checkpoints reproduces the forward states bit
// for bit (for the same block size).
#pragma once

#include <float.h>

#include "rcscm_internal.cuh"

namespace rcscm {

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

// Shared memory a RowState needs: per thread and pair, kappa/M and B (read
// every pass, B also written), kept out of registers so that more rows are
// resident at once.  Each thread touches only its own entries.
template <int BLOCK, int NP>
struct RowSmem {
    f32x2 kapM[NP][BLOCK];
    f32x2 B[NP][BLOCK];
};

// One row with NP pairs of chunks (chunk k = slots k * BLOCK + threadIdx.x;
// pair q = chunks 2q and 2q + 1): invariants tau_ax, sigma_bx and the state in
// registers, kappa/M and B in the thread's own shared-memory entries.  Slots
// past the end of the row are padding that contributes exactly zero: r_h = 0
// and r_u = 1 throughout (their r_h offset beta/(alpha+2) is replaced by 0).
template <int BLOCK, int NP>
struct RowState {
    f32x2 tr[NP], ti[NP], sr[NP], si[NP], rh[NP], ru[NP];
    f32x2 CB_LAST;
    float lam;
    int J;
    RowSmem<BLOCK, NP>* sm;

    __device__ __forceinline__ explicit RowState(RowSmem<BLOCK, NP>* s) : sm(s) {}

    // Invariants tau_ax, sigma_bx and kappa/M (+ r_u floor) of the row's slots, from
    // fetch(j, float4& {tau_ax, sigma_bx}, float& kappa) for each slot j < J_.
    template <class Fetch>
    __device__ __forceinline__ void load_inv_with(int J_, const RowConst& c, const IterParams& p, Fetch fetch) {
        J = J_;
        const int tid = threadIdx.x;
        float cb_lo = p.c_b, cb_hi = p.c_b;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            float v[2][5];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = (2 * q + h) * BLOCK + tid;
                if (j < J) {
                    float4 t;
                    float kap;
                    fetch(j, t, kap);
                    v[h][0] = t.x; v[h][1] = t.y; v[h][2] = t.z; v[h][3] = t.w;
                    v[h][4] = fmaf(kap, c.invM, p.ru_floor);             // r_u >= ru_floor by construction
                } else {
                    v[h][0] = v[h][1] = v[h][2] = v[h][3] = 0.f;
                    v[h][4] = 1.f;                                       // padding keeps r_u = 1
                    if (q == NP - 1) { if (h == 0) cb_lo = 0.f; else cb_hi = 0.f; }
                }
            }
            tr[q] = pk(v[0][0], v[1][0]);
            ti[q] = pk(v[0][1], v[1][1]);
            sr[q] = pk(v[0][2], v[1][2]);
            si[q] = pk(v[0][3], v[1][3]);
            sm->kapM[q][tid] = pk(v[0][4], v[1][4]);
        }
        CB_LAST = pk(cb_lo, cb_hi);
    }

    // invariants of the row starting at slot `off`, from the context's arrays
    __device__ __forceinline__ void load_inv(const DevState& d, int64_t off, int J_, const RowConst& c,
                                             const IterParams& p) {
        load_inv_with(J_, c, p, [&](int j, float4& t, float& kap) {
            t = d.inv4[off + j];
            kap = d.kap[off + j];
        });
    }

    // state from arrays indexed by slot within the row (rh_src[j], ru_src[j]); padding: r_h = 0, r_u = 1
    __device__ __forceinline__ void load_state(const float* rh_src, const float* ru_src, float lam_) {
        const int tid = threadIdx.x;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const int j0 = 2 * q * BLOCK + tid, j1 = j0 + BLOCK;
            rh[q] = pk(j0 < J ? rh_src[j0] : 0.f, j1 < J ? rh_src[j1] : 0.f);
            ru[q] = pk(j0 < J ? ru_src[j0] : 1.f, j1 < J ? ru_src[j1] : 1.f);
        }
        lam = lam_;
    }

    __device__ __forceinline__ void store_state(float* rh_dst, float* ru_dst) const {
        const int tid = threadIdx.x;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = (2 * q + h) * BLOCK + tid;
                if (j < J) {
                    rh_dst[j] = h ? hi_of(rh[q]) : lo_of(rh[q]);
                    ru_dst[j] = h ? hi_of(ru[q]) : lo_of(ru[q]);
                }
            }
        }
    }

    // r_h, r_u of slot k (chunk index) of this thread
    __device__ __forceinline__ float rh_of(int k) const { return (k & 1) ? hi_of(rh[k >> 1]) : lo_of(rh[k >> 1]); }
    __device__ __forceinline__ float ru_of(int k) const { return (k & 1) ? hi_of(ru[k >> 1]) : lo_of(ru[k >> 1]); }

    __device__ __forceinline__ bool any_clamp(float ru_floor) const {
        bool clamp = false;
        const int tid = threadIdx.x;
#pragma unroll
        for (int q = 0; q < NP; ++q)
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if ((2 * q + h) * BLOCK + tid < J) clamp |= (h ? hi_of(ru[q]) : lo_of(ru[q])) <= ru_floor;
        return clamp;
    }

    // One EM pass (the repeat loop of Algorithm 2): pass A per slot, lambda by a
    // fixed-order block reduction, pass B per slot.  `parity` selects the half of `red`.
    __device__ __forceinline__ void pass(const RowConst& c, const IterParams& p,
                                         float (*red)[BLOCK / 32 > 0 ? BLOCK / 32 : 1], int parity) {
        const f32x2 NSR = dup(-c.sab_re), NSI = dup(-c.sab_im), SI = dup(c.sab_im), SAB2 = dup(c.sab2);
        const f32x2 NITAA = dup(-c.inv_taa), TAAM = dup(c.taaM), CA2 = dup(p.c_a2), CB = dup(p.c_b);
        const float invJ = 1.0f / (float)J;
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
            ru[q] = fma2(TAAM, fma2(er, er, fma2(ei, ei, Q)), sm->kapM[q][threadIdx.x]);    // A / M
            sm->B[q][threadIdx.x] = Bk;
            rh[q] = fma2(rhat, CA2, q == NP - 1 ? CB_LAST : CB);
        }
        lam = block_sum<BLOCK>(lo_of(part) + hi_of(part), red, parity) * invJ;
        const f32x2 ILM = dup(rcp_refined(lam) * c.invM);
#pragma unroll
        for (int q = 0; q < NP; ++q) ru[q] = fma2(sm->B[q][threadIdx.x], ILM, ru[q]);
    }
};

}  // namespace rcscm
