// Adjoint of the accelerated estimator, sm_103a: gradients of a real loss of
// the extracted target image with respect to x_ij, a_i and R'_i, through K
// passes of Algorithm 2 (Sec. III-C-2), the multichannel Wiener filter
// (posterior mean) and the per-frequency setup.  The paper defines no
// gradient; this is reverse-mode differentiation of the forward computation.
//
// Convention (that of PyTorch for a real loss L of complex z): the gradient of z
// is dL/dRe z + i dL/dIm z, so dL = Re(conj(g_z) dz).
//
// adjoint_kernel<BLOCK, NP>: one CTA per row, NP pairs of chunks per thread
// (the forward kernel's RowState).  Steps:
//   1. Wiener filter h = w a, w = r_h rho_ax / (r_u + r_h rho_aa), at the final state.
//   2. Passes t = K-1 .. 0 by checkpoint segments: each segment is recomputed
//      once from its checkpoint with the forward pass code (bit-exact states,
//      kept in a scratch), then its passes are run backwards (two fixed-order
//      block reductions per pass).
//   3. Invariants: kappa = tau_xx - |tau_ax|^2 / tau_aa, tau_ax = a^H P x,
//      tau_xx = x^H P x, sigma_bx = b^H x with P = (R')^+ (Eq. (eq:riinv)):
//      g_x = P a g_tau + 2 g_txx P x + b g_sigma per slot, and the row sums
//      v_a = sum_j x_j conj(g_tau_j), v_b = sum_j x_j conj(g_sigma_j),
//      C = sum_j g_txx_j x_j x_j^H, staged through shared memory and added with
//      compensated FP32 sums (four interleaved per thread, joined as error-free pairs).
//   4. Setup (FP64, adjoint_setup_kernel: a group of 16 or 32 lanes per row, entry-
//      parallel, from a per-row record of the row kernel's sums), in the eigenbasis E of R' (mu_1 <
//      mu_2 <= ...; b = e_1; P = sum_{i>=2} e_i e_i^H / mu_i).  With G the
//      Hermitian gradient of P and g_b that of b (every use: tau_aa = a^H P a,
//      sigma_ab = a^H b and step 3), first-order perturbation of the
//      eigenpairs gives the gradient of R' as E F E^H with, for i, k >= 2,
//        F_ik = -G'_ik / (mu_i mu_k),
//        F_i1 = conj(F_1i) = G'_i1 / (mu_i (mu_i - mu_1)) - g'_i / (2 (mu_i - mu_1)),
//      F_11 = 0, G' = E^H G E and g' = E^H g_b.  This is the exact derivative
//      for any mu_1 (at mu_1 = 0 it reads -P G P + P^2 G B + B G P^2 minus the
//      Hermitian part of P g_b b^H, B = b b^H), and it does not depend on the
//      phase of b.
#include <float.h>

#include "accel_common.cuh"

namespace rcscm {
namespace {

// Sum of N values over the block with one __syncthreads (buffer half `parity`).
template <int BLOCK, int N>
__device__ __forceinline__ void block_sum_n(float (&v)[N], float (*red)[BLOCK / 32][N], int parity) {
    constexpr int NW = BLOCK / 32;
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = warp_sum(v[i]);
    const int lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) red[parity][threadIdx.x >> 5][i] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float t = 0.f;
        for (int w = 0; w < NW; ++w) t += red[parity][w][i];
        v[i] = t;
    }
}

// s += v with Kahan compensation c (s + (-c) tracks the exact running sum).  The
// compiler does not reassociate these operations (no fast-math).
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Unevaluated FP32 pairs hi + lo: the sum of two pairs with Knuth's error-free
// TwoSum and Dekker's renormalisation (additions only, no contraction).
__device__ __forceinline__ void pair_add(float& hi, float& lo, float hi2, float lo2) {
    const float s = hi + hi2;
    const float bb = s - hi;
    float e = (hi - (s - bb)) + (hi2 - bb);
    e += lo + lo2;
    hi = s + e;
    lo = e - (hi - s);
}

// staged slot record: x (2 kMaxM), g_tau (2), g_sigma (2), g_txx, 1
constexpr int kGtau = 2 * kMaxM, kGsig = 2 * kMaxM + 2, kGtxx = 2 * kMaxM + 4, kOne = 2 * kMaxM + 5;
constexpr int kStage = 2 * kMaxM + 6;

template <int BLOCK, int SPT>
struct AdjShared {
    float ga_w[2 * kMaxM];   // gradient of a from the Wiener filter (block-uniform)
    __align__(16) float red[2][BLOCK / 32];
    float redn[2][BLOCK / 32][8];
    float2 s_a[kMaxM], s_b[kMaxM], s_Pa[kMaxM], s_P[kMaxM * kMaxM];
    float stage[BLOCK * kStage];
    double2 dP[kMaxM][kMaxM], dE[kMaxM][kMaxM];
    double dmu[kMaxM], dimu[kMaxM];
};

template <int BLOCK, int NP, int SPT>
__device__ __forceinline__ void adjoint_row(const DevState& d, const AdjointArgs& g, const IterParams& p, int r,
                                            AdjShared<BLOCK, SPT>& sh, float* segsm) {
    constexpr int NK = 2 * NP;
    float (*red)[BLOCK / 32] = sh.red;
    float (*redn)[BLOCK / 32][8] = sh.redn;
    float2* s_a = sh.s_a;
    float2* s_b = sh.s_b;
    float2* s_Pa = sh.s_Pa;
    float2* s_P = sh.s_P;
    float* stage = sh.stage;
    double2(*dP)[kMaxM] = sh.dP;
    double2(*dE)[kMaxM] = sh.dE;
    double* dmu = sh.dmu;
    double* dimu = sh.dimu;

    const RowDesc* rd = d.rows + r;
    const int J = rd->J;
    const int M = rd->M;
    const int64_t off = rd->slot_off;
    const RowConst c = d.rc[r];
    const int tid = threadIdx.x;
    const int MM = M * M;
    {   // the row's upstream gradient (read by step 1) and x (step 3), asked of L2 now
        const int64_t bytes = (int64_t)J * M * (int64_t)sizeof(float2);
        const char* ghb = reinterpret_cast<const char*>(g.grad_h + rd->out_off);
        const char* xb = reinterpret_cast<const char*>(rd->x);
        for (int64_t o = (int64_t)tid * 128; o < bytes; o += (int64_t)BLOCK * 128) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ghb + o));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(xb + o));
        }
    }
    if (tid < M) {
        s_a[tid] = d.a32[(size_t)r * kMaxM + tid];
        s_b[tid] = d.b32[(size_t)r * kMaxM + tid];
        const double mu = d.mu[(size_t)r * kMaxM + tid];
        dmu[tid] = mu;
        dimu[tid] = tid >= 1 ? 1.0 / mu : 0.0;     // 1/mu_i of the nonzero eigenpairs
    }
    for (int e = tid; e < MM; e += BLOCK) dE[e / M][e % M] = d.evec64[(size_t)r * 64 + e];
    __syncthreads();
    for (int e = tid; e < MM; e += BLOCK) {          // P = sum_{i>=2} e_i e_i^H / mu_i (Eq. (eq:riinv))
        const int m = e / M, n = e % M;
        double2 v = make_double2(0.0, 0.0);
        for (int i = 1; i < M; ++i) v = zadd(v, zscale(zmulc(dE[n][i], dE[m][i]), dimu[i]));
        dP[m][n] = v;
        s_P[e] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    if (tid < M) {
        float2 v = make_float2(0.f, 0.f);
        for (int n = 0; n < M; ++n) v = cfma(s_P[tid * M + n], s_a[n], v);
        s_Pa[tid] = v;
    }

    RowState<BLOCK, NP> st;
    st.load_inv(d, off, J, c, p);
    float tr[NK], ti[NK], sr[NK], si[NK];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        tr[2 * q] = lo_of(st.tr[q]); tr[2 * q + 1] = hi_of(st.tr[q]);
        ti[2 * q] = lo_of(st.ti[q]); ti[2 * q + 1] = hi_of(st.ti[q]);
        sr[2 * q] = lo_of(st.sr[q]); sr[2 * q + 1] = hi_of(st.sr[q]);
        si[2 * q] = lo_of(st.si[q]); si[2 * q + 1] = hi_of(st.si[q]);
    }
    bool valid[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) valid[k] = k * BLOCK + tid < J;

    float g_rh[NK], g_ru[NK], g_tr[NK], g_ti[NK], g_sr[NK], g_si[NK], g_k[NK];
    // row-constant adjoints, accumulated per thread (reduced at the end)
    float p_taa = 0.f, p_taaM = 0.f, p_invtaa = 0.f, p_sab2 = 0.f, p_sre = 0.f, p_sim = 0.f;
    // uniform row adjoints (every thread holds the same value)
    float u_taa = 0.f, u_sab2 = 0.f, u_sre = 0.f, u_sim = 0.f;
    float g_lam = 0.f;

    // ---- 1. Wiener filter at the final state --------------------------------------------
    {
        st.load_state(d.rh + off, d.ru + off, d.lam[r]);
        const float lam = st.lam;
        const float il = 1.0f / lam;
        const float raa = c.taa + c.sab2 / lam;
        float pw[2 + 2 + 2 * kMaxM];                      // g_raa, g_il, g_sab (2), g_a (2M)
#pragma unroll
        for (int i = 0; i < 4 + 2 * kMaxM; ++i) pw[i] = 0.f;
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            g_rh[k] = g_ru[k] = g_tr[k] = g_ti[k] = g_sr[k] = g_si[k] = g_k[k] = 0.f;
            if (!valid[k]) continue;
            const int q = k >> 1;
            const float rh = (k & 1) ? hi_of(st.rh[q]) : lo_of(st.rh[q]);
            const float ru = (k & 1) ? hi_of(st.ru[q]) : lo_of(st.ru[q]);
            const int j = k * BLOCK + tid;
            const float2 u = cmul(make_float2(c.sab_re, c.sab_im), make_float2(sr[k], si[k]));
            const float2 rax = make_float2(tr[k] + u.x * il, ti[k] + u.y * il);
            const float E = ru + rh * raa;
            const float kk = rh / E;
            const float2 w = cscale(rax, kk);
            const float2* gh = g.grad_h + rd->out_off + (int64_t)j * M;
            float2 gw = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < kMaxM; ++m) {
                if (m < M) {
                    const float2 ghm = gh[m];
                    gw = cfma(ghm, cconj(s_a[m]), gw);               // g_w = sum_m g_h conj(a)
                    const float2 t = cmul(ghm, cconj(w));             // g_a += g_h conj(w)
                    pw[4 + 2 * m] += t.x;
                    pw[5 + 2 * m] += t.y;
                }
            }
            const float gk = gw.x * rax.x + gw.y * rax.y;          // Re(conj(g_w) rax)
            const float2 grax = cscale(gw, kk);
            float grh = gk / E;
            const float gE = -gk * rh / (E * E);
            g_ru[k] = gE;
            grh += gE * raa;
            g_rh[k] = grh;
            pw[0] += gE * rh;                                       // g_raa
            g_tr[k] = grax.x;
            g_ti[k] = grax.y;
            const float2 gu = cscale(grax, il);
            pw[1] += grax.x * u.x + grax.y * u.y;                   // g_il += Re(conj(g_rax) u)
            const float2 gs = cmul(gu, make_float2(c.sab_re, -c.sab_im));   // g_sigma += g_u conj(sab)
            g_sr[k] = gs.x;
            g_si[k] = gs.y;
            const float2 gsab = cmul(gu, make_float2(sr[k], -si[k]));       // g_sab += g_u conj(sigma)
            pw[2] += gsab.x;
            pw[3] += gsab.y;
        }
        // fixed-order block reductions (8 values at a time)
        float v0[8], v1[8], v2[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            v0[i] = pw[i];
            v1[i] = pw[8 + i];
            v2[i] = (i < 4) ? pw[16 + i] : 0.f;
        }
        block_sum_n<BLOCK, 8>(v0, redn, 0);                      // consecutive calls alternate halves
        block_sum_n<BLOCK, 8>(v1, redn, 1);
        block_sum_n<BLOCK, 8>(v2, redn, 0);
        const float graa = v0[0];
        float gil = v0[1];
        u_sre += v0[2];
        u_sim += v0[3];
        if (tid == 0) {                                             // block-uniform values
#pragma unroll
            for (int i = 0; i < 4; ++i) sh.ga_w[i] = v0[4 + i];
#pragma unroll
            for (int i = 0; i < 8; ++i) sh.ga_w[4 + i] = v1[i];
#pragma unroll
            for (int i = 0; i < 4; ++i) sh.ga_w[12 + i] = v2[i];
        }
        u_taa += graa;                                              // raa = taa + sab2 / lam
        u_sab2 += graa * il;
        gil += graa * c.sab2;
        g_lam = -gil * il * il;                                     // adjoint of lambda after the last pass
    }

    // ---- 2. passes t = K-1 .. 0, one checkpoint segment at a time ----------------------------
    // Each segment is recomputed once from its checkpoint with the forward pass code; the
    // state entering each of its passes goes to the segment buffer (each thread its own
    // slots, lambda by thread 0, read after the passes' barriers), then the passes are
    // reversed from the buffer.  The buffer is the CTA's shared memory when the launch gave
    // it room (segsm != nullptr: [stride][SPT * BLOCK] r_h, then r_u, then [stride] lambda),
    // else the context's scratch in global memory.
    constexpr int kPitch = SPT * BLOCK;
    auto seg_rh_at = [&](int tt) -> float* {
        return segsm ? segsm + (size_t)tt * kPitch : g.seg_rh + (size_t)tt * g.S + off;
    };
    auto seg_ru_at = [&](int tt) -> float* {
        return segsm ? segsm + (size_t)(g.stride + tt) * kPitch : g.seg_ru + (size_t)tt * g.S + off;
    };
    auto seg_lam_at = [&](int tt) -> float* {
        return segsm ? segsm + (size_t)2 * g.stride * kPitch + tt : g.seg_lam + (size_t)tt * g.R + r;
    };
    int parity = 1;                                                 // the next reduction uses half 1
    const int n_seg = (g.K + g.stride - 1) / g.stride;
    for (int seg = n_seg - 1; seg >= 0; --seg) {
        const int t0 = seg * g.stride, t1 = min(g.K, t0 + g.stride);
        st.load_state(g.ckpt_rh + (size_t)seg * g.S + off, g.ckpt_ru + (size_t)seg * g.S + off,
                      g.ckpt_lam[(size_t)seg * g.R + r]);
        for (int t = t0; t < t1; ++t) {
            st.store_state(seg_rh_at(t - t0), seg_ru_at(t - t0));
            if (tid == 0) *seg_lam_at(t - t0) = st.lam;
            st.pass(c, p, red, (parity++) & 1);
        }
        const float lam_end = st.lam;                               // lambda after pass t1 - 1
        for (int t = t1 - 1; t >= t0; --t) {
            // state entering pass t, and lambda after it
            float rh_t[NK], ru_t[NK];
            {
                const float* srh = seg_rh_at(t - t0);
                const float* sru = seg_ru_at(t - t0);
#pragma unroll
                for (int k = 0; k < NK; ++k) {
                    rh_t[k] = valid[k] ? srh[k * BLOCK + tid] : 0.f;
                    ru_t[k] = valid[k] ? sru[k * BLOCK + tid] : 1.f;
                }
            }
            const float lam_t = *seg_lam_at(t - t0);
            const float lam1 = t == t1 - 1 ? lam_end : *seg_lam_at(t + 1 - t0);
            const float il = rcp_refined(lam_t);
            const float rtaa = fmaf(c.sab2, il, c.taa);
            const float slr = c.sab_re * il, sli = c.sab_im * il;
            const float ilM = rcp_refined(lam1) * c.invM;
            // S1 = sum_j g_ru'_j B_j  (B needs the forward intermediates)
            float Bk[NK], rru[NK];
            float s1 = 0.f;
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const float rh = rh_t[k], ru = ru_t[k];
                const float pr = fmaf(slr, sr[k], fmaf(-sli, si[k], tr[k]));
                const float pi = fmaf(slr, si[k], fmaf(sli, sr[k], ti[k]));
                const float g_ = rh * rcp_approx(fmaf(rh, rtaa, ru));
                const float cr = g_ * pr, ci = g_ * pi;
                const float Q = g_ * ru;
                const float dr = fmaf(-cr, c.sab_re, fmaf(-ci, c.sab_im, sr[k]));
                const float di = fmaf(-ci, c.sab_re, fmaf(cr, c.sab_im, si[k]));
                Bk[k] = fmaf(dr, dr, fmaf(di, di, Q * c.sab2));
                rru[k] = rcp_approx(ru);
                if (valid[k]) s1 = fmaf(g_ru[k], Bk[k], s1);
            }
            s1 = block_sum<BLOCK>(s1, red, (parity++) & 1);
            const float glam1 = g_lam - s1 * ilM / lam1;             // ilM = invM / lambda'
            const float gell = glam1 / (float)J;
            float pr_rtaa = 0.f, pr_slr = 0.f, pr_sli = 0.f;
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                if (!valid[k]) {
                    g_rh[k] = g_ru[k] = 0.f;
                    continue;
                }
                const float rh = rh_t[k], ru = ru_t[k];
                const float pr = fmaf(slr, sr[k], fmaf(-sli, si[k], tr[k]));
                const float pi = fmaf(slr, si[k], fmaf(sli, sr[k], ti[k]));
                const float rD = rcp_approx(fmaf(rh, rtaa, ru));
                const float g_ = rh * rD;
                const float cr = g_ * pr, ci = g_ * pi;
                const float Q = g_ * ru;
                const float dr = fmaf(-cr, c.sab_re, fmaf(-ci, c.sab_im, sr[k]));
                const float di = fmaf(-ci, c.sab_re, fmaf(cr, c.sab_im, si[k]));
                const float er = fmaf(-tr[k], c.inv_taa, cr);
                const float ei = fmaf(-ti[k], c.inv_taa, ci);
                const float X = fmaf(er, er, fmaf(ei, ei, Q));
                const float gAk = g_ru[k];
                const float gBk = g_ru[k] * ilM + gell * rru[k];
                float gru = -gell * Bk[k] * rru[k] * rru[k];
                const float gX = gAk * c.taaM;
                g_k[k] += gAk * c.invM;
                p_taaM += gAk * X;
                float gcr = 2.f * er * gX, gci = 2.f * ei * gX;
                float gQ = gX;
                g_tr[k] -= gcr * c.inv_taa;
                g_ti[k] -= gci * c.inv_taa;
                p_invtaa -= gcr * tr[k] + gci * ti[k];
                const float gdr = 2.f * dr * gBk, gdi = 2.f * di * gBk;
                gQ += gBk * c.sab2;
                p_sab2 += gBk * Q;
                g_sr[k] += gdr;
                g_si[k] += gdi;
                gcr += -gdr * c.sab_re + gdi * c.sab_im;
                gci += -gdr * c.sab_im - gdi * c.sab_re;
                p_sre += -gdr * cr - gdi * ci;
                p_sim += -gdr * ci + gdi * cr;
                const float grhat = g_rh[k] * p.c_a2;
                gcr += 2.f * cr * grhat;
                gci += 2.f * ci * grhat;
                gQ += grhat;
                float gg = gQ * ru;
                gru += gQ * g_;
                gg += gcr * pr + gci * pi;
                const float gpr = gcr * g_, gpi = gci * g_;
                float grh = gg * rD;
                const float gD = -gg * rh * rD * rD;
                grh += gD * rtaa;
                gru += gD;
                pr_rtaa += gD * rh;
                g_tr[k] += gpr;
                g_ti[k] += gpi;
                g_sr[k] += gpr * slr + gpi * sli;
                g_si[k] += -gpr * sli + gpi * slr;
                pr_slr += gpr * sr[k] + gpi * si[k];
                pr_sli += -gpr * si[k] + gpi * sr[k];
                g_rh[k] = grh;
                g_ru[k] = gru;
            }
            float rv[3] = {pr_rtaa, pr_slr, pr_sli};
            block_sum_n<BLOCK, 3>(rv, reinterpret_cast<float (*)[BLOCK / 32][3]>(redn), (parity++) & 1);
            u_taa += rv[0];
            u_sab2 += rv[0] * il;
            u_sre += rv[1] * il;
            u_sim += rv[2] * il;
            const float gil = rv[0] * c.sab2 + rv[1] * c.sab_re + rv[2] * c.sab_im;
            g_lam = -gil * il * il;
        }
    }

    // ---- 3. invariants -> x; row sums staged in shared memory ----------------------------
    // kappa = tau_xx - |tau_ax|^2 / tau_aa: its tau_ax part joins g_tau (where it largely
    // cancels the pass's own tau_ax gradient) and its tau_aa part joins p_taa.  Roles of
    // the summing threads: C = sum g_txx x x^H (M*M), v_a = sum x conj(g_tau) (M),
    // v_b = sum x conj(g_sigma) (M), with compensated (Kahan) FP32 sums: they cancel
    // heavily in step 4, so plain FP32 accumulation would lose the result, and the
    // compensated sum keeps it at the rounding of the terms without the cost of FP64 (on
    // sm_103a FP64 runs at a small fraction of the FP32 rate).  Each role's slots are
    // split over n_groups threads (contiguous slot ranges of every staged block); their
    // partials are combined per role in group order as error-free FP32 pairs.
    const int n_roles = MM + 2 * M;
    const int n_groups = BLOCK / n_roles > 1 ? BLOCK / n_roles : 1;
    const int role = tid % n_roles, grp = tid / n_roles;
    const int span = (BLOCK + n_groups - 1) / n_groups;
    // Every role's term has one form, (o[ia] + i o[ia+1]) conj(o[ib] + i o[ib+1]) o[is] of a
    // staged record o (C_mn: x_m conj(x_n) g_txx; v_a: x_m conj(g_tau) 1; v_b: x_m conj(g_sigma) 1),
    // so the warps do not diverge; the record offsets are formed once (no division per term).
    int ia, ib, is;
    if (role < MM) {
        ia = 2 * (role / M);
        ib = 2 * (role % M);
        is = kGtxx;
    } else {
        ia = 2 * ((role - MM) % M);
        ib = role < MM + M ? kGtau : kGsig;
        is = kOne;
    }
    // four interleaved compensated sums per thread (independent chains), combined at the end
    float2 acc[4], comp[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = comp[u] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < NK; ++k) {                  // unrolled: the per-slot arrays stay in registers
        const int j = k * BLOCK + tid;
        float* my = stage + tid * kStage;
        if (valid[k]) {
            const float2* xj = rd->x + (int64_t)j * M;
            float2 xv[kMaxM];
#pragma unroll
            for (int m = 0; m < kMaxM; ++m) xv[m] = m < M ? xj[m] : make_float2(0.f, 0.f);
            const float gtxx = g_k[k];
            const float gtr = g_tr[k] - 2.f * tr[k] * gtxx * c.inv_taa;
            const float gti = g_ti[k] - 2.f * ti[k] * gtxx * c.inv_taa;
            p_taa += gtxx * (tr[k] * tr[k] + ti[k] * ti[k]) * c.inv_taa * c.inv_taa;
            const float2 gt = make_float2(gtr, gti), gs = make_float2(g_sr[k], g_si[k]);
            float2* gx = g.grad_x + rd->out_off + (int64_t)j * M;
#pragma unroll
            for (int m = 0; m < kMaxM; ++m) {
                if (m < M) {
                    float2 px = make_float2(0.f, 0.f);
#pragma unroll
                    for (int n = 0; n < kMaxM; ++n)
                        if (n < M) px = cfma(s_P[m * M + n], xv[n], px);
                    float2 v = cmul(s_Pa[m], gt);             // g_x = P a g_tau + b g_sigma + 2 g_txx P x
                    v = cfma(s_b[m], gs, v);
                    v = cadd(v, cscale(px, 2.f * gtxx));
                    gx[m] = v;
                    my[2 * m] = xv[m].x;
                    my[2 * m + 1] = xv[m].y;
                }
            }
            my[kGtau] = gtr;
            my[kGtau + 1] = gti;
            my[kGsig] = gs.x;
            my[kGsig + 1] = gs.y;
            my[kGtxx] = gtxx;
            my[kOne] = 1.f;
        } else {
            for (int i = 0; i < kStage; ++i) my[i] = 0.f;
        }
        __syncthreads();
        if (grp < n_groups) {
            const int sl0 = grp * span, sl1 = min(BLOCK, sl0 + span);
            auto term_at = [&](int sl) {
                const float* o = stage + sl * kStage;
                return cscale(cmul(make_float2(o[ia], o[ia + 1]), make_float2(o[ib], -o[ib + 1])), o[is]);
            };
            int sl = sl0;
            for (; sl + 4 <= sl1; sl += 4) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float2 t = term_at(sl + u);
                    kahan_add(acc[u].x, comp[u].x, t.x);
                    kahan_add(acc[u].y, comp[u].y, t.y);
                }
            }
            for (int u = 0; sl < sl1; ++sl, ++u) {
                const float2 t = term_at(sl);
                kahan_add(acc[u].x, comp[u].x, t.x);
                kahan_add(acc[u].y, comp[u].y, t.y);
            }
        }
        __syncthreads();
    }
    // this thread's four sums as one error-free pair each for re and im, then the groups'
    // partials of each role, combined in group order (stage is free again)
    float4 mine = make_float4(acc[0].x, -comp[0].x, acc[0].y, -comp[0].y);
#pragma unroll
    for (int u = 1; u < 4; ++u) {
        pair_add(mine.x, mine.y, acc[u].x, -comp[u].x);
        pair_add(mine.z, mine.w, acc[u].y, -comp[u].y);
    }
    float4* part = reinterpret_cast<float4*>(stage);
    if (grp < n_groups) part[grp * n_roles + role] = mine;
    // row-constant partials
    float pv[8] = {p_taa, p_taaM, p_invtaa, p_sab2, p_sre, p_sim, 0.f, 0.f};
    block_sum_n<BLOCK, 8>(pv, redn, (parity++) & 1);        // its barrier also publishes `part`
    float4 tot = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid < n_roles)
        for (int gi = 0; gi < n_groups; ++gi) {
            const float4 q = part[gi * n_roles + tid];
            pair_add(tot.x, tot.y, q.x, q.y);
            pair_add(tot.z, tot.w, q.z, q.w);
        }

    // ---- 4. the row's sums, for the setup adjoint (adjoint_setup_kernel) ------------------------
    // role sums in FP64 (the FP32 pairs added once), the total adjoints of tau_aa and sigma_ab
    // (FP64 from the FP32 sums) and the Wiener filter's gradient of a
    double* out = g.sums + (size_t)r * kAdjSums;
    if (tid < n_roles) {
        out[2 * tid] = (double)tot.x + (double)tot.y;
        out[2 * tid + 1] = (double)tot.z + (double)tot.w;
    }
    if (tid == 0) {
        const double taa = d.taa64[r];
        const double2 sab = d.sab64[r];
        out[kAdjGtaa] = (double)u_taa + (double)pv[0] + (double)pv[1] / M - (double)pv[2] / (taa * taa);
        out[kAdjGsab] = (double)u_sre + pv[4] + 2.0 * sab.x * ((double)u_sab2 + pv[3]);
        out[kAdjGsab + 1] = (double)u_sim + pv[5] + 2.0 * sab.y * ((double)u_sab2 + pv[3]);
        for (int i = 0; i < 2 * kMaxM; ++i) out[kAdjGaw + i] = (double)sh.ga_w[i];
    }
}

// Step 4, the setup adjoint in FP64, one row per warp (lanes own matrix entries): from the
// row kernel's sums it forms g_a and the gradient of R' through the eigenpairs of R'.  As
// its own kernel it runs many rows per SM at once, instead of holding a row kernel's CTA
// with one FP64 warp.
struct SetupAdjShared {
    double2 dP[kMaxM][kMaxM], dG[kMaxM][kMaxM], dT[kMaxM][kMaxM];
    double2 dva[kMaxM], dvb[kMaxM], dga[kMaxM], dgb[kMaxM], dGb[kMaxM];
    double2 dA_[kMaxM], dE[kMaxM][kMaxM];
    double dmu[kMaxM], dimu[kMaxM];
};
constexpr int kSetupAdjWarps = 4;

// LANES = 16 (M <= 4, two rows per warp) or 32: lanes per row.  A warp's rows run the same
// instruction stream, so the rows of a launch with M <= 4 take half the FP64 instructions.
template <int LANES>
__global__ void __launch_bounds__(kSetupAdjWarps * 32) adjoint_setup_kernel(DevState d, AdjointArgs g, int n_rows) {
    constexpr int kRowsPerCta = kSetupAdjWarps * 32 / LANES;
    __shared__ SetupAdjShared shw[kRowsPerCta];
    const int lane = threadIdx.x & (LANES - 1);
    SetupAdjShared& sh = shw[threadIdx.x / LANES];
    const int r0 = blockIdx.x * kRowsPerCta + (int)(threadIdx.x / LANES);
    const bool active = r0 < n_rows;                          // an idle row keeps its warp's syncs
    const int r = active ? r0 : n_rows - 1;
    const RowDesc* rd = d.rows + r;
    const int M = rd->M;
    const int MM = M * M;
    double2(*dP)[kMaxM] = sh.dP;
    double2(*dG)[kMaxM] = sh.dG;
    double2(*dT)[kMaxM] = sh.dT;
    double2 *dva = sh.dva, *dvb = sh.dvb, *dga = sh.dga, *dgb = sh.dgb, *dGb = sh.dGb, *dA_ = sh.dA_;
    double2(*dE)[kMaxM] = sh.dE;
    double* dmu = sh.dmu;
    double* dimu = sh.dimu;
    const double* in = g.sums + (size_t)r * kAdjSums;
    if (lane < M) {
        const double mu = d.mu[(size_t)r * kMaxM + lane];
        dmu[lane] = mu;
        dimu[lane] = lane >= 1 ? 1.0 / mu : 0.0;              // 1/mu_i of the nonzero eigenpairs
        dA_[lane] = rd->a[lane];
    }
    for (int e = lane; e < MM; e += LANES) dE[e / M][e % M] = d.evec64[(size_t)r * 64 + e];
    const int n_roles = MM + 2 * M;
    for (int t = lane; t < n_roles; t += LANES) {                // C, v_a, v_b of the row kernel
        const double2 v = make_double2(in[2 * t], in[2 * t + 1]);
        if (t < MM) dG[t / M][t % M] = v;
        else if (t < MM + M) dva[t - MM] = v;
        else dvb[t - MM - M] = v;
    }
    __syncwarp();
    for (int e = lane; e < MM; e += LANES) {                     // P = sum_{i>=2} e_i e_i^H / mu_i
        const int m = e / M, n = e % M;
        double2 v = make_double2(0.0, 0.0);
        for (int i = 1; i < M; ++i) v = zadd(v, zscale(zmulc(dE[n][i], dE[m][i]), dimu[i]));
        dP[m][n] = v;
    }
    __syncwarp();
    const double g_taa = in[kAdjGtaa];
    const double2 g_sab = make_double2(in[kAdjGsab], in[kAdjGsab + 1]);
    if (lane < M) {
        double2 pa = make_double2(0.0, 0.0), pva = make_double2(0.0, 0.0);
        for (int n = 0; n < M; ++n) {
            pa = zfma(pa, dP[lane][n], dA_[n]);
            pva = zfma(pva, dP[lane][n], dva[n]);
        }
        // g_a = g_a(Wiener) + P v_a + 2 g_taa P a + b conj(g_sab)
        double2 ga = make_double2(in[kAdjGaw + 2 * lane], in[kAdjGaw + 2 * lane + 1]);
        ga = zadd(ga, pva);
        ga = zadd(ga, zscale(pa, 2.0 * g_taa));
        ga = zadd(ga, zmul(dE[lane][0], zconj(g_sab)));
        dga[lane] = ga;
        dgb[lane] = zadd(dvb[lane], zmul(dA_[lane], g_sab));     // g_b = v_b + a g_sab
    }
    __syncwarp();
    // G = Hermitian part of (C + g_taa a a^H + a v_a^H)
    for (int e = lane; e < MM; e += LANES) {
        const int m = e / M, n = e % M;
        const double2 t1 = zadd(zscale(zmul(dA_[m], zconj(dA_[n])), g_taa), zmul(dA_[m], zconj(dva[n])));
        const double2 t2 = zadd(zscale(zmul(dA_[n], zconj(dA_[m])), g_taa), zmul(dA_[n], zconj(dva[m])));
        dT[m][n] = zscale(zadd(zadd(dG[m][n], t1), zconj(zadd(dG[n][m], t2))), 0.5);
    }
    __syncwarp();
    constexpr int kPer = (kMaxM * kMaxM + LANES - 1) / LANES;
    double2 tmp[kPer];                                        // at most kPer entries per lane
#pragma unroll
    for (int t = 0; t < kPer; ++t) {                          // G E
        const int e = lane + LANES * t;
        if (e < MM) {
            const int m = e / M, n = e % M;
            double2 v = make_double2(0.0, 0.0);
            for (int k = 0; k < M; ++k) v = zfma(v, dT[m][k], dE[k][n]);
            tmp[t] = v;
        }
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < kPer; ++t)
        if (lane + LANES * t < MM) dG[(lane + LANES * t) / M][(lane + LANES * t) % M] = tmp[t];
    __syncwarp();
    for (int e = lane; e < MM; e += LANES) {                     // G' = E^H (G E)
        const int i = e / M, k = e % M;
        double2 v = make_double2(0.0, 0.0);
        for (int m = 0; m < M; ++m) v = zfma_c(v, dE[m][i], dG[m][k]);
        dT[i][k] = v;
    }
    if (lane < M) {                                           // g' = E^H g_b
        double2 v = make_double2(0.0, 0.0);
        for (int m = 0; m < M; ++m) v = zfma_c(v, dE[m][lane], dgb[m]);
        dGb[lane] = v;
    }
    __syncwarp();
    const double mu1 = dmu[0];
    for (int e = lane; e < MM; e += LANES) {                     // F (eigenbasis)
        const int i = e / M, k = e % M;
        double2 f = make_double2(0.0, 0.0);
        if (i >= 1 && k >= 1) {
            f = zscale(dT[i][k], -(dimu[i] * dimu[k]));
        } else if (i >= 1 || k >= 1) {
            const int q = i >= 1 ? i : k;
            const double igap = 1.0 / (dmu[q] - mu1);
            f = zsub(zscale(dT[q][0], dimu[q] * igap), zscale(dGb[q], 0.5 * igap));
            if (i == 0) f = zconj(f);
        }
        dG[i][k] = f;
    }
    __syncwarp();
    for (int e = lane; e < MM; e += LANES) {                     // F E^H
        const int i = e / M, n = e % M;
        double2 v = make_double2(0.0, 0.0);
        for (int k = 0; k < M; ++k) v = zfma(v, dG[i][k], zconj(dE[n][k]));
        dT[i][n] = v;
    }
    __syncwarp();
    double2* gR = g.grad_Rp + rd->rp_off;
    for (int e = lane; e < MM && active; e += LANES) {           // E (F E^H)
        const int m = e / M, n = e % M;
        double2 v = make_double2(0.0, 0.0);
        for (int i = 0; i < M; ++i) v = zfma(v, dE[m][i], dT[i][n]);
        gR[e] = v;
    }
    if (active && lane < M) g.grad_a[rd->a_off + lane] = dga[lane];
}


// One CTA per row; the row's exact count of chunk pairs selects the body (as in the
// forward kernel, so the recomputed states equal the forward ones bit for bit).
// 128-thread rows are held to 4 CTAs per SM (128 registers; the row phases are latency
// chains, so residency pays more than the few spilled values cost).
template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK, BLOCK == 128 ? 4 : 1) adjoint_kernel(DevState d, AdjointArgs g, IterParams p, int seg_in_smem) {
    __shared__ AdjShared<BLOCK, SPT> sh;
    extern __shared__ float segsm[];
    float* seg = seg_in_smem ? segsm : nullptr;
    const int r = blockIdx.x;
    RCSCM_CTA_CHECK(row_ok(d, r, BLOCK * SPT), d.status);
    const int np = (d.rows[r].J + 2 * BLOCK - 1) / (2 * BLOCK);
    switch (np) {
        case 1: adjoint_row<BLOCK, 1, SPT>(d, g, p, r, sh, seg); break;
        case 2: if constexpr (SPT >= 4) adjoint_row<BLOCK, 2, SPT>(d, g, p, r, sh, seg); break;
        case 3: if constexpr (SPT >= 8) adjoint_row<BLOCK, 3, SPT>(d, g, p, r, sh, seg); break;
        case 4: if constexpr (SPT >= 8) adjoint_row<BLOCK, 4, SPT>(d, g, p, r, sh, seg); break;
        default: break;
    }
}

// The segment buffer goes to shared memory when it fits beside the kernel's static shared
// memory within the per-block limit (and leaves room for the CTAs the registers allow).
template <int BLOCK, int SPT>
cudaError_t launch_adjoint_t(const DevState& d, int n_rows, int max_m, const AdjointArgs& a, const IterParams& p,
                             cudaStream_t s) {
    const size_t bytes = ((size_t)2 * a.stride * SPT * BLOCK + (size_t)a.stride) * sizeof(float);
    static size_t limit = 0;
    static size_t static_bytes = 0;
    if (!limit) {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
            cudaFuncGetAttributes(&fa, adjoint_kernel<BLOCK, SPT>) == cudaSuccess) {
            static_bytes = fa.sharedSizeBytes;
            limit = (size_t)optin > static_bytes ? (size_t)optin - static_bytes : 1;
            if (cudaFuncSetAttribute(adjoint_kernel<BLOCK, SPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(limit > 1 ? limit : 0)) != cudaSuccess) {
                cudaGetLastError();
                limit = 1;
            }
        } else {
            cudaGetLastError();
            limit = 1;
        }
    }
    const bool in_smem = bytes <= 96 * 1024 && bytes <= limit;
    adjoint_kernel<BLOCK, SPT><<<n_rows, BLOCK, in_smem ? bytes : 0, s>>>(d, a, p, in_smem ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (max_m <= 4)
        adjoint_setup_kernel<16><<<(n_rows + 2 * kSetupAdjWarps - 1) / (2 * kSetupAdjWarps), kSetupAdjWarps * 32, 0, s>>>(
            d, a, n_rows);
    else
        adjoint_setup_kernel<32><<<(n_rows + kSetupAdjWarps - 1) / kSetupAdjWarps, kSetupAdjWarps * 32, 0, s>>>(d, a,
                                                                                                         n_rows);
    return cudaGetLastError();
}

}  // namespace

// Shapes (threads per row, slots per thread) follow the forward kernel's: the
// block of a context with checkpoints is adjoint_block(max_j).
cudaError_t launch_adjoint(const DevState& d, int n_rows, int max_j, int max_m, int block, const AdjointArgs& a,
                           const IterParams& p, cudaStream_t s) {
    const int need = (max_j + block - 1) / block;
    if (block == 128 && need <= 4) return launch_adjoint_t<128, 4>(d, n_rows, max_m, a, p, s);
    if (block == 256 && need <= 4) return launch_adjoint_t<256, 4>(d, n_rows, max_m, a, p, s);
    if (block == 256 && need <= 8) return launch_adjoint_t<256, 8>(d, n_rows, max_m, a, p, s);
    return cudaErrorInvalidValue;
}

}  // namespace rcscm
