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

// Sum over the block with one __syncthreads; `red` (16-byte aligned) is double-buffered
// by the pass parity so consecutive passes never race on it.  Every thread returns the
// same, order-fixed value: the warp sums w_k combined as a butterfly over k, which for 4
// and 8 warps is read back as one or two 16-byte words and added in the butterfly's order
// (the same value, with a shorter dependency chain than two or three more shuffles).  A
// single-warp block needs no shared memory.
template <int BLOCK>
__device__ __forceinline__ float block_sum(float v, float (*red)[BLOCK / 32 > 0 ? BLOCK / 32 : 1], int parity) {
    constexpr int NW = BLOCK / 32;
    v = warp_sum(v);
    if constexpr (NW == 1) {
        return v;
    } else if constexpr (NW == 4) {
        if ((threadIdx.x & 31) == 0) red[parity][threadIdx.x >> 5] = v;
        __syncthreads();
        const float4 w = *reinterpret_cast<const float4*>(&red[parity][0]);
        return (w.x + w.z) + (w.y + w.w);
    } else if constexpr (NW == 8) {
        if ((threadIdx.x & 31) == 0) red[parity][threadIdx.x >> 5] = v;
        __syncthreads();
        const float4 a = *reinterpret_cast<const float4*>(&red[parity][0]);
        const float4 b = *reinterpret_cast<const float4*>(&red[parity][4]);
        return ((a.x + b.x) + (a.z + b.z)) + ((a.y + b.y) + (a.w + b.w));
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
    (void)b;
    return a;
}
__device__ __forceinline__ float hi_of(f32x2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    (void)a;
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

// Per-pass row scalars of Algorithm 2, duplicated into both halves of a pair.
struct PassConsts {
    f32x2 NSR, NSI, SI, SAB2, NITAA, TAAM, CA2, CB, RTAA, SLR, SLI, NSLI;
};
// il = rcp_refined(lambda) of the pass.
__device__ __forceinline__ PassConsts pass_consts(const RowConst& c, const IterParams& p, float il) {
    PassConsts k;
    k.NSR = dup(-c.sab_re);
    k.NSI = dup(-c.sab_im);
    k.SI = dup(c.sab_im);
    k.SAB2 = dup(c.sab2);
    k.NITAA = dup(-c.inv_taa);
    k.TAAM = dup(c.taaM);
    k.CA2 = dup(p.c_a2);
    k.CB = dup(p.c_b);
    k.RTAA = dup(fmaf(c.sab2, il, c.taa));                       // rho~_aa, Eq. (eq:traa_accel)
    const float slr = c.sab_re * il, sli = c.sab_im * il;
    k.SLR = dup(slr);
    k.SLI = dup(sli);
    k.NSLI = dup(-sli);
    return k;
}

// Pass A of one pair of slots (Algorithm 2 before the lambda update): r_h is
// replaced by its new value, r_u by A/M (the part of the new r_u that needs no
// lambda), B is returned, and B / r~_u is added to the lambda partial sum.
// `cb` is the r_h offset beta/(alpha+2), 0 in padding slots.
__device__ __forceinline__ void pass_a_pair(const PassConsts& k, f32x2 tr, f32x2 ti, f32x2 sr, f32x2 si, f32x2 kapM,
                                            f32x2 cb, f32x2& rh, f32x2& ru, f32x2& Bout, f32x2& part) {
    const f32x2 pr = fma2(k.SLR, sr, fma2(k.NSLI, si, tr));
    const f32x2 pi = fma2(k.SLR, si, fma2(k.SLI, sr, ti));
    const f32x2 g = mul2(rh, rcp2(fma2(rh, k.RTAA, ru)));
    const f32x2 cr = mul2(g, pr), ci = mul2(g, pi);
    const f32x2 Q = mul2(g, ru);
    const f32x2 rhat = fma2(ci, ci, fma2(cr, cr, Q));
    const f32x2 dr = fma2(cr, k.NSR, fma2(ci, k.NSI, sr));
    const f32x2 di = fma2(ci, k.NSR, fma2(cr, k.SI, si));
    const f32x2 Bk = fma2(dr, dr, fma2(di, di, mul2(Q, k.SAB2)));
    part = fma2(Bk, rcp2(ru), part);
    const f32x2 er = fma2(tr, k.NITAA, cr);
    const f32x2 ei = fma2(ti, k.NITAA, ci);
    ru = fma2(k.TAAM, fma2(er, er, fma2(ei, ei, Q)), kapM);              // A / M
    Bout = Bk;
    rh = fma2(rhat, k.CA2, cb);
}

// One row with NP pairs of chunks (chunk k = slots k * BLOCK + threadIdx.x;
// pair q = chunks 2q and 2q + 1), kept in registers.  Slots past the end of
// the row are padding that contributes exactly zero: r_h = 0 and r_u = 1
// throughout (their r_h offset beta/(alpha+2) is replaced by 0).  (Keeping
// kappa/M and B in shared memory instead, with launch bounds for more resident
// rows, measured slower: the extra loads and spills cost more than the wave
// tail they remove.)
template <int BLOCK, int NP>
struct RowState {
    f32x2 tr[NP], ti[NP], sr[NP], si[NP], kapM[NP], rh[NP], ru[NP], B[NP];
    f32x2 CB_LAST;
    float lam;
    float il;    // rcp_refined(lam), formed once per pass and used by this pass and the next
    int J;

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
            kapM[q] = pk(v[0][4], v[1][4]);
            B[q] = 0;
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
        il = rcp_refined(lam_);
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
        const PassConsts k = pass_consts(c, p, il);
        f32x2 part = dup(0.f);
#pragma unroll
        for (int q = 0; q < NP; ++q)
            pass_a_pair(k, tr[q], ti[q], sr[q], si[q], kapM[q], q == NP - 1 ? CB_LAST : k.CB, rh[q], ru[q], B[q],
                        part);
        lam = block_sum<BLOCK>(lo_of(part) + hi_of(part), red, parity) * (1.0f / (float)J);
        il = rcp_refined(lam);
        const f32x2 ILM = dup(il * c.invM);
#pragma unroll
        for (int q = 0; q < NP; ++q) ru[q] = fma2(B[q], ILM, ru[q]);
    }
};

}  // namespace rcscm
