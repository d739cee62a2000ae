// First-stage accelerated rule (Algorithm 1, Sec. III-C-1), sm_103a.
//
// The first stage inverts R_i = R'_i + lambda_i b_i b_i^H once per frequency
// bin and pass (Table I: O(I M^3 + I J M^2) per iteration) and evaluates the
// slot quantities rho_ax = a^H R^{-1} x and rho_xx = x^H R^{-1} x from x_ij at
// every pass (O(M^2) per slot); rho~ of a pass are the rho of the previous pass
// (Algorithm 1 copies them), so one inverse per row and pass suffices.  A pass:
//   pass A (per slot):  gamma~ = r~_h / (r~_u + r~_h rho~_aa)          Eq. (eq:tal)
//                       r_h <- (gamma~ (r~_u + gamma~ |rho~_ax|^2) + beta) / (alpha + 2)   (eq:1st_rh)
//                       ell = gamma~ |sigma_ab|^2 + |sigma_bx - gamma~ conj(sigma_ab) rho~_ax|^2 / r~_u
//   lambda <- (1/J) sum_j ell_j                                        Eq. (eq:1st_li)
//   per row:            R = R' + lambda b b^H = C C^H (Cholesky), so R^{-1} = C^-H C^-1;
//                       g = C^{-1} a, rho_aa = |g|^2                   Eq. (eq:raa)
//   pass B (per slot):  z = C^{-1} x (forward substitution), rho_ax = g^H z   Eq. (eq:rax)
//                       r_u <- (gamma~ rho_aa r~_u + |z - c g|^2) / M, c = gamma~ rho~_ax
// The last line is Eq. (eq:1st_ru): |C^{-1} (x - c a)|^2 = rho_xx - 2 gamma~ Re[rho~_ax conj(rho_ax)]
// + gamma~^2 |rho~_ax|^2 rho_aa (Eq. (eq:rxx) expanded), evaluated as a sum of squares so
// FP32 keeps r_u > 0.  The factorisation is done by M + 1 lanes of one warp on the
// augmented matrix [R a; a^H *]: its last factor row is (C^{-1} a)^H, so g and
// rho_aa come out of the same column sweep.  It runs in double-float arithmetic
// (about 48 significand bits, dfloat.cuh): the low bins' R_i have condition
// numbers of 1e3 to 1e4, where an FP32 factor would miss the 1e-5 agreement with
// the FP64 algorithm, and FP64 would put tens of cycles per instruction on the
// row's critical path.  The factor and g are rounded to FP32 once; the per-slot
// work is FP32.  sigma_bx = b^H x (Eq. (eq:spx)) is formed once before the
// loop, as Algorithm 1 does.
#include <float.h>

#include "accel_common.cuh"
#include "dfloat.cuh"

namespace rcscm {
namespace {

// Cholesky factor of R = R' + lambda b b^H for one row, with g = C^{-1} a, by lanes
// 0..M of the calling warp (all 32 lanes call; control flow around __syncwarp is
// warp-uniform).  Lane i < M owns row i of C, lane M the appended row a^H, whose
// factor row is conj(g).  Results rounded to FP32: sC (strictly lower triangle,
// row-major), sic (1 / C_kk), sg, *srho = |g|^2.
template <int M>
__device__ void row_factor(const dfc (*sRp)[M], const dfc* sb, const dfc* sa, float lam, dfc (*sL)[M + 1],
                           df* sinv, float2 (*sC)[M], float* sic, float2* sg, float* srho) {
    const int i = threadIdx.x & 31;
    const df lamd = df_make(lam);
    df gg = df_make(0.f);                                          // lane M: sum_k |C_Mk|^2
#pragma unroll
    for (int j = 0; j < M; ++j) {
        if (i == j) {                                            // C_jj = sqrt(R_jj - sum_k |C_jk|^2)
            df v = df_add(sRp[j][j].re, df_mul(lamd, dfc_abs2(sb[j])));
#pragma unroll
            for (int k = 0; k < j; ++k) v = df_sub(v, dfc_abs2(sL[j][k]));
            const df cjj = df_sqrt(v);
            sL[j][j] = dfc{cjj, df_make(0.f)};
            sinv[j] = df_div(df_make(1.f), cjj);
        }
        __syncwarp();
        if (i > j && i <= M) {                                   // C_ij = (A_ij - sum_k C_ik conj(C_jk)) / C_jj
            dfc v = i < M ? dfc_add(sRp[i][j], dfc_scale(dfc_mulc(sb[j], sb[i]), lamd))
                          : dfc{sa[j].re, df_neg(sa[j].im)};     // appended row: conj(a_j)
#pragma unroll
            for (int k = 0; k < j; ++k) v = dfc_sub(v, dfc_mulc(sL[j][k], sL[i][k]));
            v = dfc_scale(v, sinv[j]);
            sL[i][j] = v;
            if (i == M) gg = df_add(gg, dfc_abs2(v));
        }
        __syncwarp();
    }
    if (i < M) {
#pragma unroll
        for (int k = 0; k < M; ++k)
            if (k < i) sC[i][k] = dfc_to_float2(sL[i][k]);
        sic[i] = df_to_float(sinv[i]);
        const dfc gm = sL[M][i];                                 // g_i = conj(C_Mi)
        sg[i] = make_float2(df_to_float(gm.re), -df_to_float(gm.im));
    }
    if (i == M) *srho = df_to_float(gg);
}

// z = C^{-1} x by forward substitution (C in shared memory), rho_ax = g^H z.
template <int M>
__device__ __forceinline__ void apply_inverse(const float2 (*sC)[M], const float* sic, const float2* sg,
                                              const float2* __restrict__ xs, float2 (&z)[M], float2& rax) {
    rax = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < M; ++k) {
        float2 v = xs[k];
#pragma unroll
        for (int n = 0; n < k; ++n) {
            const float2 c = sC[k][n];
            v = make_float2(v.x - fmaf(c.x, z[n].x, -c.y * z[n].y), v.y - fmaf(c.x, z[n].y, c.y * z[n].x));
        }
        z[k] = cscale(v, sic[k]);
        rax = cfmac(sg[k], z[k], rax);
    }
}

template <int BLOCK, int SPT, int M>
__global__ void __launch_bounds__(BLOCK) accel1_kernel(DevState d, const int* __restrict__ rows, int n_iter,
                                                       IterParams p) {
    __shared__ __align__(16) float red[2][BLOCK / 32];
    __shared__ dfc sRp[M][M], sL[M + 1][M + 1];
    __shared__ dfc sb[M], sa[M];
    __shared__ df sinv[M];
    __shared__ float2 sC[M][M], sg[M], sb32[M];
    __shared__ float sic[M];
    __shared__ float s_rho;
    const int r = rows[blockIdx.x];
    RCSCM_CTA_CHECK(row_ok(d, r, SPT * BLOCK) && d.rows[r].M == M, d.status);
    const RowDesc* rd = d.rows + r;
    const int J = rd->J;
    const int64_t off = rd->slot_off;
    const int tid = threadIdx.x;
    // R' with its smallest eigenvalue set to zero (the model's R_i = R' + lambda b b^H), a, b
    const double mu1 = d.mu[(size_t)r * kMaxM];
    for (int e = tid; e < M * M; e += BLOCK) {
        const int m = e / M, n = e % M;
        const double2 amn = rp_entry(*rd, m * M + n), anm = rp_entry(*rd, n * M + m);
        const double2 bm = d.b64[(size_t)r * kMaxM + m], bn = d.b64[(size_t)r * kMaxM + n];
        const double2 bb = zmulc(bn, bm);                                 // b_m conj(b_n)
        const double hr = 0.5 * (amn.x + anm.x) - mu1 * bb.x, hi = 0.5 * (amn.y - anm.y) - mu1 * bb.y;
        sRp[m][n] = dfc{df_from_double(hr), df_from_double(hi)};
    }
    if (tid < M) {
        const double2 bv = d.b64[(size_t)r * kMaxM + tid], av = rd->a[tid];
        sb[tid] = dfc{df_from_double(bv.x), df_from_double(bv.y)};
        sa[tid] = dfc{df_from_double(av.x), df_from_double(av.y)};
        sb32[tid] = d.b32[(size_t)r * kMaxM + tid];
    }
    const RowConst rc = d.rc[r];
    float lam = d.lam[r];
    __syncthreads();
    if (tid < 32) row_factor<M>(sRp, sb, sa, lam, sL, sinv, sC, sic, sg, &s_rho);
    __syncthreads();

    // before the loop: sigma_bx (Eq. (eq:spx)) and rho_ax with the initial lambda (Eq. (eq:rax))
    const float2* xrow = rd->x;
    float sbr[SPT], sbi[SPT], rtr[SPT], rti[SPT], rh[SPT], ru[SPT], gm[SPT];
#pragma unroll
    for (int k = 0; k < SPT; ++k) {
        const int j = k * BLOCK + tid;
        if (j < J) {
            const float2* xs = xrow + (size_t)j * M;
            float2 sbx = make_float2(0.f, 0.f);
#pragma unroll
            for (int n = 0; n < M; ++n) sbx = cfmac(sb32[n], xs[n], sbx);
            float2 z[M], rax;
            apply_inverse<M>(sC, sic, sg, xs, z, rax);
            sbr[k] = sbx.x;
            sbi[k] = sbx.y;
            rtr[k] = rax.x;
            rti[k] = rax.y;
            rh[k] = d.rh[off + j];
            ru[k] = d.ru[off + j];
        } else {                                      // padding: contributes exactly zero
            sbr[k] = sbi[k] = rtr[k] = rti[k] = rh[k] = 0.f;
            ru[k] = 1.f;
        }
        gm[k] = 0.f;
    }
    float rtaa = s_rho;
    const float sabr = rc.sab_re, sabi = rc.sab_im, sab2 = rc.sab2;
    const float invM = 1.f / (float)M;
    bool clamped = false;
    for (int it = 0; it < n_iter; ++it) {
        float part = 0.f;
#pragma unroll
        for (int k = 0; k < SPT; ++k) {               // pass A
            const float g = rh[k] / fmaf(rh[k], rtaa, ru[k]);                       // Eq. (eq:tal)
            const float rt2 = fmaf(rtr[k], rtr[k], rti[k] * rti[k]);
            const float rhat = g * fmaf(g, rt2, ru[k]);
            // sigma_bx - gamma~ conj(sigma_ab) rho~_ax
            const float cr = g * rtr[k], ci = g * rti[k];
            const float dr = sbr[k] - fmaf(sabr, cr, sabi * ci);
            const float di = sbi[k] - fmaf(sabr, ci, -sabi * cr);
            part += fmaf(g, sab2, fmaf(dr, dr, di * di) / ru[k]);                   // Eq. (eq:1st_li) summand
            const int j = k * BLOCK + tid;
            rh[k] = j < J ? fmaf(rhat, p.c_a2, p.c_b) : 0.f;                          // Eq. (eq:1st_rh)
            gm[k] = g;
        }
        lam = block_sum<BLOCK>(part, red, it & 1) * (1.0f / (float)J);
        if (tid < 32) row_factor<M>(sRp, sb, sa, lam, sL, sinv, sC, sic, sg, &s_rho);
        __syncthreads();
        const float rho = s_rho;
#pragma unroll
        for (int k = 0; k < SPT; ++k) {               // pass B with the up-to-date R_i
            const int j = k * BLOCK + tid;
            if (j < J) {
                float2 z[M], rax;
                apply_inverse<M>(sC, sic, sg, xrow + (size_t)j * M, z, rax);
                const float cr = gm[k] * rtr[k], ci = gm[k] * rti[k];                // c = gamma~ rho~_ax
                float s = 0.f;
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    const float yr = z[m].x - fmaf(cr, sg[m].x, -ci * sg[m].y);
                    const float yi = z[m].y - fmaf(cr, sg[m].y, ci * sg[m].x);
                    s = fmaf(yr, yr, fmaf(yi, yi, s));
                }
                const float ru_new = fmaf(gm[k] * rho, ru[k], s) * invM;            // Eq. (eq:1st_ru)
                clamped |= !(ru_new > p.ru_floor);
                ru[k] = fmaxf(ru_new, p.ru_floor);
                rtr[k] = rax.x;                                                     // rho~_ax <- rho_ax
                rti[k] = rax.y;
            }
        }
        rtaa = rho;
    }
#pragma unroll
    for (int k = 0; k < SPT; ++k) {
        const int j = k * BLOCK + tid;
        if (j < J) {
            d.rh[off + j] = rh[k];
            d.ru[off + j] = ru[k];
        }
    }
    if (clamped) atomicOr(d.status, kFlagClamp);
    if (tid == 0) {
        d.lam[r] = lam;
        if (!(lam > 0.f) || !(lam <= FLT_MAX)) atomicOr(d.status, kFlagNonfinite);
    }
}

template <int BLOCK, int SPT>
cudaError_t launch_shape(const DevState& d, const int* rows_by_m, const int* count_by_m, const int* first_by_m,
                         int n_iter, const IterParams& p, cudaStream_t s) {
    for (int M = 2; M <= kMaxM; ++M) {
        const int n = count_by_m[M];
        if (n <= 0) continue;
        const int* rows = rows_by_m + first_by_m[M];
        switch (M) {
            case 2: accel1_kernel<BLOCK, SPT, 2><<<n, BLOCK, 0, s>>>(d, rows, n_iter, p); break;
            case 3: accel1_kernel<BLOCK, SPT, 3><<<n, BLOCK, 0, s>>>(d, rows, n_iter, p); break;
            case 4: accel1_kernel<BLOCK, SPT, 4><<<n, BLOCK, 0, s>>>(d, rows, n_iter, p); break;
            case 5: accel1_kernel<BLOCK, SPT, 5><<<n, BLOCK, 0, s>>>(d, rows, n_iter, p); break;
            case 6: accel1_kernel<BLOCK, SPT, 6><<<n, BLOCK, 0, s>>>(d, rows, n_iter, p); break;
            case 7: accel1_kernel<BLOCK, SPT, 7><<<n, BLOCK, 0, s>>>(d, rows, n_iter, p); break;
            default: accel1_kernel<BLOCK, SPT, 8><<<n, BLOCK, 0, s>>>(d, rows, n_iter, p); break;
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

// Rows of up to 512 frames run with 128 threads x 4 slots, up to 1024 with 128 x 8
// (several rows per SM hide each other's per-pass factorisation), up to 2048 with
// 256 x 8, up to 4096 with 512 x 8.
int accel1_block(int max_j) { return max_j <= 1024 ? 128 : (max_j <= 2048 ? 256 : (max_j <= 4096 ? 512 : 0)); }

cudaError_t launch_accel1(const DevState& d, const int* rows_by_m, const int* count_by_m, const int* first_by_m,
                          int max_j, int n_iter, const IterParams& p, cudaStream_t s) {
    if (max_j <= 512) return launch_shape<128, 4>(d, rows_by_m, count_by_m, first_by_m, n_iter, p, s);
    if (max_j <= 1024) return launch_shape<128, 8>(d, rows_by_m, count_by_m, first_by_m, n_iter, p, s);
    if (max_j <= 2048) return launch_shape<256, 8>(d, rows_by_m, count_by_m, first_by_m, n_iter, p, s);
    if (max_j <= 4096) return launch_shape<512, 8>(d, rows_by_m, count_by_m, first_by_m, n_iter, p, s);
    return cudaErrorInvalidValue;
}

}  // namespace rcscm
