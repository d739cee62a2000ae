// Naive EM rule of the rank-constrained SCM estimator (Sec. II-B-2), sm_103a.
//
// naive_kernel<T, M>: one CTA per row (utterance, frequency i), one slot per
// thread at a time, arithmetic in T (double: RCSCM_RULE_NAIVE_F64, float:
// RCSCM_RULE_NAIVE_PRINTED), in the coordinates the formulas are printed in.
// A pass:
//   R~_i    = R'_i + lambda~ b b^H
//   R~^(x)  = r~_h a a^H + r~_u R~_i                      Eq. (eq:rijx)
//   P       = (R~^(x))^{-1}  (explicit, Cholesky)
//   rhat_h  = r~_h - r~_h^2 a^H P a + |r~_h x^H P a|^2    Eq. (eq:E_hrh)
//   R^u     = r~_u R~ - r~_u^2 R~ P R~ + r~_u^2 R~ P x x^H P R~   Eq. (eq:E_hru)
//   r_h    <- (rhat_h + beta) / (alpha + 2)               Eq. (eq:M_rh)
//   lambda <- (1/J) sum_j b^H R^u b / r~_u                Eq. (eq:M_li)
//   R_i     = R'_i + lambda b b^H, explicit inverse
//   r_u    <- tr(R_i^{-1} R^u) / M                        Eq. (eq:M_ru)
// R^u (Hermitian M x M) is kept per slot in a global scratch array between the
// lambda reduction and the r_u update.
//
// The printed E-step forms are differences of nearly equal terms when
// r~_h rho~ >> r~_u; in exact arithmetic rhat_h >= 0 and b^H R^u b >= 0, and in
// FP32 they can come out negative.  Such values are held at zero (r_h at its
// exact-arithmetic bound beta/(alpha+2)) and reported as RCSCM_ECLAMP, so the
// model covariance stays positive definite.  In FP64 the bound is not reached
// on the workloads measured here.
//
// naive_white_kernel<M> (RCSCM_RULE_NAIVE): the same E-step and M-step in FP32,
// in the whitened coordinates of R~_i.  With R' = sum_{k>=1} mu_k e_k e_k^H
// (e_0 = b, mu_0 set to zero) the congruence G = diag(lambda~^-1/2, mu_1^-1/2,
// ...) E^H maps R~_i to I, and every quantity of the pass transforms exactly:
//   G R~^(x) G^H = r~_h a' a'^H + r~_u I  with a' = G a, x' = G x,
//   P' = (G R~^(x) G^H)^{-1} (explicit, Cholesky) and P = G^H P' G,
//   rhat_h = r~_h - r~_h^2 a'^H P' a' + |r~_h x'^H P' a'|^2            Eq. (eq:E_hrh)
//   G^-1 R^u G^-H = R' := r~_u I - r~_u^2 P' + r~_u^2 P' x' x'^H P'     Eq. (eq:E_hru)
//   b^H R^u b = lambda~ R'_00                                           Eq. (eq:M_li)
//   tr(R_i^{-1} R^u) = (lambda~ / lambda) R'_00 + sum_{k>=1} R'_kk       Eq. (eq:M_ru)
// (G^-H R_i^{-1} G^-1 = diag(lambda~/lambda, 1, ..., 1) with the new lambda).  G
// is formed per row in FP64 by the setup; only lambda~ changes between passes.
// In the printed coordinates the per-slot inverse inherits the condition number
// of R~_i (1e3 to 1e4 at the low bins of a small array) on top of the slot's
// signal-to-noise ratio, and FP32 leaves 1e-4 to 1e-2 relative error after one
// pass; here the matrix inverted is the identity plus a rank-one term, whose
// FP32 inverse is accurate to a few units of rounding in the directions the
// E-step uses.  The scratch holds two values per slot, R'_00 and
// sum_{k>=1} R'_kk.
#include <float.h>

#include <type_traits>

#include "rcscm_internal.cuh"

namespace rcscm {
namespace {

template <class T>
struct Cx {
    T re, im;
};
template <class T>
__device__ __forceinline__ Cx<T> cx(T r, T i) { return Cx<T>{r, i}; }
template <class T>
__device__ __forceinline__ Cx<T> operator+(Cx<T> a, Cx<T> b) { return cx(a.re + b.re, a.im + b.im); }
template <class T>
__device__ __forceinline__ Cx<T> operator-(Cx<T> a, Cx<T> b) { return cx(a.re - b.re, a.im - b.im); }
template <class T>
__device__ __forceinline__ Cx<T> operator*(Cx<T> a, Cx<T> b) {
    return cx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class T>
__device__ __forceinline__ Cx<T> operator*(Cx<T> a, T s) { return cx(a.re * s, a.im * s); }
template <class T>
__device__ __forceinline__ Cx<T> conj(Cx<T> a) { return cx(a.re, -a.im); }
template <class T>
__device__ __forceinline__ T abs2(Cx<T> a) { return a.re * a.re + a.im * a.im; }
template <class T>
__device__ __forceinline__ Cx<T> zero() { return cx(T(0), T(0)); }

template <class T>
__device__ __forceinline__ T rsqrt_t(T v);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float v) { return rsqrtf(v); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double v) { return rsqrt(v); }

// In-place inverse of a Hermitian positive definite matrix through its
// Cholesky factor: A = L L^H, W = L^{-1}, A^{-1} = W^H W.
template <class T, int M>
__device__ __forceinline__ void hpd_inverse(Cx<T> (&A)[M][M]) {
    Cx<T> L[M][M];
    T dinv[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        T s = A[j][j].re;
#pragma unroll
        for (int k = 0; k < j; ++k) s -= abs2(L[j][k]);
        dinv[j] = rsqrt_t<T>(s);
        L[j][j] = cx(s * dinv[j], T(0));
#pragma unroll
        for (int i = j + 1; i < M; ++i) {
            Cx<T> v = A[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) v = v - L[i][k] * conj(L[j][k]);
            L[i][j] = v * dinv[j];
        }
    }
    Cx<T> W[M][M];   // L^{-1} by forward substitution on L W = I
#pragma unroll
    for (int i = 0; i < M; ++i) {
        W[i][i] = cx(dinv[i], T(0));
#pragma unroll
        for (int j = 0; j < i; ++j) {
            Cx<T> v = zero<T>();
#pragma unroll
            for (int k = j; k < i; ++k) v = v + L[i][k] * W[k][j];
            W[i][j] = v * (-dinv[i]);
        }
    }
#pragma unroll
    for (int m = 0; m < M; ++m) {
#pragma unroll
        for (int n = m; n < M; ++n) {
            Cx<T> v = zero<T>();
#pragma unroll
            for (int k = (m > n ? m : n); k < M; ++k) v = v + conj(W[k][m]) * W[k][n];
            A[m][n] = v;
            A[n][m] = conj(v);
        }
        A[m][m].im = T(0);
    }
}

template <class T, int BLOCK>
__device__ __forceinline__ T block_sum_t(T v, T (*red)[BLOCK / 32], int parity) {
    constexpr int NW = BLOCK / 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31;
    if (lane == 0) red[parity][threadIdx.x >> 5] = v;
    __syncthreads();
    T t = red[parity][lane & (NW - 1)];
#pragma unroll
    for (int o = NW / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

constexpr int kNaiveBlock = 128;

template <class T, int M>
__global__ void __launch_bounds__(kNaiveBlock) naive_kernel(DevState d, const int* __restrict__ rows,
                                                             int n_iter, IterParams p) {
    constexpr bool kF64 = std::is_same<T, double>::value;
    // R^u scratch of the row: M*M values of T per slot (M real diagonal entries, then
    // the M(M-1)/2 complex upper entries), element q of slot j at [q * J + j].
    __shared__ Cx<T> sRp[M][M], sRt[M][M], sRi[M][M];
    __shared__ Cx<T> sa[M], sb[M];
    __shared__ T red[2][kNaiveBlock / 32];
    const int r = rows[blockIdx.x];
    RCSCM_CTA_CHECK(row_ok(d, r, 1 << 30) && d.rows[r].M == M, d.status);
    const RowDesc* rd = d.rows + r;
    const int J = rd->J;
    const int64_t off = rd->slot_off;
    T* scratch = static_cast<T*>(d.ru_hat) + rd->scratch_off;
    const float2* xrow = rd->x;
    const int tid = threadIdx.x;
    const T c_a2 = kF64 ? T(p.c_a2_f64) : T(p.c_a2);
    const T c_b = kF64 ? T(p.c_b_f64) : T(p.c_b);
    if (tid < M) {
        if constexpr (kF64) {
            const double2 av = rd->a[tid], bv = d.b64[(size_t)r * kMaxM + tid];
            sa[tid] = cx(av.x, av.y);
            sb[tid] = cx(bv.x, bv.y);
        } else {
            const float2 av = d.a32[(size_t)r * kMaxM + tid], bv = d.b32[(size_t)r * kMaxM + tid];
            sa[tid] = cx(av.x, av.y);
            sb[tid] = cx(bv.x, bv.y);
        }
    }
    __syncthreads();
    // R' with its smallest eigenvalue set to zero (so R' + lambda b b^H is the model's R_i)
    for (int e = tid; e < M * M; e += kNaiveBlock) {
        const int m = e / M, n = e % M;
        if constexpr (kF64) {
            const double2 amn = rp_entry(*rd, m * M + n), anm = rp_entry(*rd, n * M + m);
            const double mu1 = d.mu[(size_t)r * kMaxM];
            sRp[m][n] = cx(0.5 * (amn.x + anm.x), 0.5 * (amn.y - anm.y)) - (sb[m] * conj(sb[n])) * mu1;
        } else {
            const float2 v = d.rp32[(size_t)r * 64 + e];
            sRp[m][n] = cx(v.x, v.y);
        }
    }
    T lam = T(d.lam[r]);
    bool clamped = false;
    __syncthreads();

    for (int it = 0; it < n_iter; ++it) {
        for (int e = tid; e < M * M; e += kNaiveBlock) {            // R~_i = R'_i + lambda~ b b^H
            const int m = e / M, n = e % M;
            sRt[m][n] = sRp[m][n] + (sb[m] * conj(sb[n])) * lam;
        }
        __syncthreads();
        T part = T(0);
        for (int j = tid; j < J; j += kNaiveBlock) {
            const T rh_t = T(d.rh[off + j]);
            const T ru_t = T(d.ru[off + j]);
            Cx<T> xv[M];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const float2 v = xrow[(size_t)j * M + m];
                xv[m] = cx(T(v.x), T(v.y));
            }
            Cx<T> P[M][M];
#pragma unroll
            for (int m = 0; m < M; ++m)
#pragma unroll
                for (int n = 0; n < M; ++n) P[m][n] = (sa[m] * conj(sa[n])) * rh_t + sRt[m][n] * ru_t;
            hpd_inverse<T, M>(P);
            Cx<T> Pa[M];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                Cx<T> v = zero<T>();
#pragma unroll
                for (int n = 0; n < M; ++n) v = v + P[m][n] * sa[n];
                Pa[m] = v;
            }
            T aPa = T(0);
            Cx<T> xPa = zero<T>();
#pragma unroll
            for (int m = 0; m < M; ++m) {
                aPa += (conj(sa[m]) * Pa[m]).re;
                xPa = xPa + conj(xv[m]) * Pa[m];
            }
            const T rhat = rh_t - rh_t * rh_t * aPa + rh_t * rh_t * abs2(xPa);    // Eq. (eq:E_hrh)
            Cx<T> Tm[M][M];                                                        // R~ P
#pragma unroll
            for (int m = 0; m < M; ++m)
#pragma unroll
                for (int n = 0; n < M; ++n) {
                    Cx<T> v = zero<T>();
#pragma unroll
                    for (int k = 0; k < M; ++k) v = v + sRt[m][k] * P[k][n];
                    Tm[m][n] = v;
                }
            Cx<T> y[M];                                                            // R~ P x
#pragma unroll
            for (int m = 0; m < M; ++m) {
                Cx<T> v = zero<T>();
#pragma unroll
                for (int n = 0; n < M; ++n) v = v + Tm[m][n] * xv[n];
                y[m] = v;
            }
            const T ru2 = ru_t * ru_t;
            T* out = scratch + j;
            T bRb = T(0);
            int q = M;
#pragma unroll
            for (int m = 0; m < M; ++m) {
#pragma unroll
                for (int n = m; n < M; ++n) {
                    Cx<T> N = zero<T>();
#pragma unroll
                    for (int k = 0; k < M; ++k) N = N + Tm[m][k] * sRt[k][n];
                    const Cx<T> v = sRt[m][n] * ru_t - N * ru2 + (y[m] * conj(y[n])) * ru2;   // Eq. (eq:E_hru)
                    const T bvb = ((conj(sb[m]) * v) * sb[n]).re;
                    if (m == n) {
                        out[(size_t)m * J] = v.re;
                        bRb += bvb;
                    } else {
                        out[(size_t)q * J] = v.re;
                        out[(size_t)(q + 1) * J] = v.im;
                        q += 2;
                        bRb += T(2) * bvb;
                    }
                }
            }
            const bool ok_l = bRb >= T(0);
            const bool ok_h = rhat >= T(0);
            clamped |= !(ok_l && ok_h);
            part += ok_l ? bRb / ru_t : T(0);                                     // Eq. (eq:M_li) summand
            d.rh[off + j] = (float)(ok_h ? rhat * c_a2 + c_b : c_b);               // Eq. (eq:M_rh)
        }
        lam = block_sum_t<T, kNaiveBlock>(part, red, it & 1) / T(J);
        if (tid == 0) {                                                            // R_i^{-1}
            Cx<T> R[M][M];
#pragma unroll
            for (int m = 0; m < M; ++m)
#pragma unroll
                for (int n = 0; n < M; ++n) R[m][n] = sRp[m][n] + (sb[m] * conj(sb[n])) * lam;
            hpd_inverse<T, M>(R);
#pragma unroll
            for (int m = 0; m < M; ++m)
#pragma unroll
                for (int n = 0; n < M; ++n) sRi[m][n] = R[m][n];
        }
        __syncthreads();
        for (int j = tid; j < J; j += kNaiveBlock) {
            const T* in = scratch + j;
            T tr = T(0);   // Re tr(R^{-1} R^u) = sum_m Ri_mm Ru_mm + 2 sum_{m<n} Re(Ri_nm Ru_mn)
            int q = M;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                tr += sRi[m][m].re * in[(size_t)m * J];
#pragma unroll
                for (int n = m + 1; n < M; ++n) {
                    const Cx<T> v = cx(in[(size_t)q * J], in[(size_t)(q + 1) * J]);
                    q += 2;
                    tr += T(2) * (sRi[n][m] * v).re;
                }
            }
            const float ru_new = (float)(tr / T(M));                               // Eq. (eq:M_ru)
            clamped |= !(ru_new > p.ru_floor);
            d.ru[off + j] = fmaxf(ru_new, p.ru_floor);
        }
        __syncthreads();
    }
    if (clamped) atomicOr(d.status, kFlagClamp);
    if (tid == 0) {
        const float lf = (float)lam;
        d.lam[r] = lf;
        if (!(lf > 0.f) || !(lf <= FLT_MAX)) atomicOr(d.status, kFlagNonfinite);
    }
}

// Naive rule in FP32, whitened coordinates of R~_i (see the top of this file).
template <int M>
__global__ void __launch_bounds__(kNaiveBlock) naive_white_kernel(DevState d, const int* __restrict__ rows,
                                                                   int n_iter, IterParams p) {
    __shared__ Cx<float> sG[M][M];      // row 0: b^H; rows k >= 1: e_k^H / sqrt(mu_k)
    __shared__ Cx<float> saw[M];        // a' = G a of this pass
    __shared__ Cx<float> saa[M][M];     // a' a'^H of this pass
    __shared__ float s_g0;              // 1 / sqrt(lambda~)
    __shared__ float red[2][kNaiveBlock / 32];
    const int r = rows[blockIdx.x];
    RCSCM_CTA_CHECK(row_ok(d, r, 1 << 30) && d.rows[r].M == M, d.status);
    const RowDesc* rd = d.rows + r;
    const int J = rd->J;
    const int64_t off = rd->slot_off;
    float* scr0 = static_cast<float*>(d.ru_hat) + rd->scratch_off;   // R'_00 per slot
    float* scr1 = scr0 + J;                                          // sum_{k>=1} R'_kk per slot
    const float2* xrow = rd->x;
    const int tid = threadIdx.x;
    for (int e = tid; e < M * M; e += kNaiveBlock) {
        const float2 v = d.wht32[(size_t)r * 64 + e];
        sG[e / M][e % M] = cx(v.x, v.y);
    }
    const double2 sab = d.sab64[r];
    float lam = d.lam[r];
    bool clamped = false;
    for (int it = 0; it < n_iter; ++it) {
        if (tid < M) {   // a'_0 = b^H a / sqrt(lambda~) = conj(sigma_ab) / sqrt(lambda~); a'_k fixed
            const double g0 = 1.0 / sqrt((double)lam);
            const double2 w = tid == 0 ? make_double2(sab.x * g0, -sab.y * g0) : d.aw64[(size_t)r * kMaxM + tid];
            saw[tid] = cx((float)w.x, (float)w.y);
            if (tid == 0) s_g0 = (float)g0;
        }
        __syncthreads();
        for (int e = tid; e < M * M; e += kNaiveBlock) saa[e / M][e % M] = saw[e / M] * conj(saw[e % M]);
        __syncthreads();
        const float g0 = s_g0;
        float part = 0.f;
        for (int j = tid; j < J; j += kNaiveBlock) {
            const float rh_t = d.rh[off + j];
            const float ru_t = d.ru[off + j];
            Cx<float> xv[M], xw[M];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const float2 v = xrow[(size_t)j * M + m];
                xv[m] = cx(v.x, v.y);
            }
#pragma unroll
            for (int k = 0; k < M; ++k) {                                       // x' = G x
                Cx<float> v = zero<float>();
#pragma unroll
                for (int n = 0; n < M; ++n) v = v + sG[k][n] * xv[n];
                xw[k] = k == 0 ? v * g0 : v;
            }
            Cx<float> P[M][M];                                                  // G R~^(x) G^H, Eq. (eq:rijx)
#pragma unroll
            for (int m = 0; m < M; ++m)
#pragma unroll
                for (int n = 0; n < M; ++n) P[m][n] = saa[m][n] * rh_t + (m == n ? cx(ru_t, 0.f) : zero<float>());
            hpd_inverse<float, M>(P);
            Cx<float> Pa[M], Px[M];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                Cx<float> u = zero<float>(), v = zero<float>();
#pragma unroll
                for (int n = 0; n < M; ++n) {
                    u = u + P[m][n] * saw[n];
                    v = v + P[m][n] * xw[n];
                }
                Pa[m] = u;
                Px[m] = v;
            }
            float aPa = 0.f;
            Cx<float> xPa = zero<float>();
#pragma unroll
            for (int m = 0; m < M; ++m) {
                aPa += (conj(saw[m]) * Pa[m]).re;
                xPa = xPa + conj(xw[m]) * Pa[m];
            }
            const float rhat = rh_t - rh_t * rh_t * aPa + rh_t * rh_t * abs2(xPa);   // Eq. (eq:E_hrh)
            const float ru2 = ru_t * ru_t;
            float d0 = 0.f, drest = 0.f;                                         // diagonal of Eq. (eq:E_hru)
#pragma unroll
            for (int k = 0; k < M; ++k) {
                const float v = ru_t - ru2 * P[k][k].re + ru2 * abs2(Px[k]);
                if (k == 0) d0 = v; else drest += v;
            }
            const bool ok_l = d0 >= 0.f;
            const bool ok_h = rhat >= 0.f;
            clamped |= !(ok_l && ok_h);
            d0 = ok_l ? d0 : 0.f;
            part += lam * d0 / ru_t;                                             // Eq. (eq:M_li) summand
            scr0[j] = d0;
            scr1[j] = drest;
            d.rh[off + j] = ok_h ? fmaf(rhat, p.c_a2, p.c_b) : p.c_b;             // Eq. (eq:M_rh)
        }
        const float lam_new = block_sum_t<float, kNaiveBlock>(part, red, it & 1) / (float)J;
        const float ratio = lam / lam_new;
        const float invM = 1.f / (float)M;
        for (int j = tid; j < J; j += kNaiveBlock) {
            const float ru_new = fmaf(ratio, scr0[j], scr1[j]) * invM;           // Eq. (eq:M_ru)
            clamped |= !(ru_new > p.ru_floor);
            d.ru[off + j] = fmaxf(ru_new, p.ru_floor);
        }
        lam = lam_new;
        __syncthreads();
    }
    if (clamped) atomicOr(d.status, kFlagClamp);
    if (tid == 0) {
        d.lam[r] = lam;
        if (!(lam > 0.f) || !(lam <= FLT_MAX)) atomicOr(d.status, kFlagNonfinite);
    }
}

cudaError_t launch_naive_white(const DevState& d, const int* rows_by_m, const int* count_by_m, const int* first_by_m,
                               int n_iter, const IterParams& p, cudaStream_t s) {
    for (int M = 2; M <= kMaxM; ++M) {
        const int n = count_by_m[M];
        if (n <= 0) continue;
        const int* rows = rows_by_m + first_by_m[M];
        switch (M) {
            case 2: naive_white_kernel<2><<<n, kNaiveBlock, 0, s>>>(d, rows, n_iter, p); break;
            case 3: naive_white_kernel<3><<<n, kNaiveBlock, 0, s>>>(d, rows, n_iter, p); break;
            case 4: naive_white_kernel<4><<<n, kNaiveBlock, 0, s>>>(d, rows, n_iter, p); break;
            case 5: naive_white_kernel<5><<<n, kNaiveBlock, 0, s>>>(d, rows, n_iter, p); break;
            case 6: naive_white_kernel<6><<<n, kNaiveBlock, 0, s>>>(d, rows, n_iter, p); break;
            case 7: naive_white_kernel<7><<<n, kNaiveBlock, 0, s>>>(d, rows, n_iter, p); break;
            default: naive_white_kernel<8><<<n, kNaiveBlock, 0, s>>>(d, rows, n_iter, p); break;
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <class T>
cudaError_t launch_naive_t(const DevState& d, const int* rows_by_m, const int* count_by_m, const int* first_by_m,
                           int n_iter, const IterParams& p, cudaStream_t s) {
    for (int M = 2; M <= kMaxM; ++M) {
        const int n = count_by_m[M];
        if (n <= 0) continue;
        const int* rows = rows_by_m + first_by_m[M];
        switch (M) {
            case 2: naive_kernel<T, 2><<<n, kNaiveBlock, 0, s>>>(d, rows, n_iter, p); break;
            case 3: naive_kernel<T, 3><<<n, kNaiveBlock, 0, s>>>(d, rows, n_iter, p); break;
            case 4: naive_kernel<T, 4><<<n, kNaiveBlock, 0, s>>>(d, rows, n_iter, p); break;
            case 5: naive_kernel<T, 5><<<n, kNaiveBlock, 0, s>>>(d, rows, n_iter, p); break;
            case 6: naive_kernel<T, 6><<<n, kNaiveBlock, 0, s>>>(d, rows, n_iter, p); break;
            case 7: naive_kernel<T, 7><<<n, kNaiveBlock, 0, s>>>(d, rows, n_iter, p); break;
            default: naive_kernel<T, 8><<<n, kNaiveBlock, 0, s>>>(d, rows, n_iter, p); break;
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_naive(const DevState& d, const int* rows_by_m, const int* count_by_m, const int* first_by_m,
                         int n_iter, const IterParams& p, int rule, cudaStream_t s) {
    if (rule == RCSCM_RULE_NAIVE) return launch_naive_white(d, rows_by_m, count_by_m, first_by_m, n_iter, p, s);
    return rule == RCSCM_RULE_NAIVE_F64 ? launch_naive_t<double>(d, rows_by_m, count_by_m, first_by_m, n_iter, p, s)
                                        : launch_naive_t<float>(d, rows_by_m, count_by_m, first_by_m, n_iter, p, s);
}

}  // namespace rcscm
