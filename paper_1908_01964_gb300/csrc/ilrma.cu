// Estimator inputs from the outputs of the ILRMA stage (Sec. II-A, II-B-1,
// II-B-3), sm_103a.
//
// ILRMA gives, per frequency i, the demixing matrix W_i = (w_{i,1} ... w_{i,M})^H
// = A_i^{-1} (Sec. II-A) and, for the target source n_h, the NMF bases t_{ik}
// and activations v_{kj} of its low-rank model.  ilrma_init_kernel<M> turns one
// utterance's (x, W, T, V, n_h) into the estimator's inputs, one CTA per row i:
//
//   warp f      A_i = W_i^{-1} in FP64 (Gauss-Jordan elimination on [W_i | I]
//               with partial pivoting; lanes own entries) and a_i = column n_h
//               of A_i (the target's steering vector, Sec. II-B-1);
//   the others  the output powers d_n = (1/J) sum_j |w_{i,n}^H x_ij|^2 with
//               y = W_i x_ij in FP32 (W rounded once), compensated FP32
//               partial sums and a compensated block reduction; d_{n_h} = 0;
//   warp f      R'_i = A_i diag(d) A_i^H in FP64: the back-projection of the
//               M-1 noise outputs, Eq. (eq:rit) (upper triangle, mirrored);
//   all warps   r_u0_ij = (1/M) sum_{n != n_h} |w_{i,n}^H x_ij|^2 / d_n.
//
// r_h0_ij = sum_k t_ik v_kj (Eq. (eq:rhinit)) is a small product T V, made by
// CTAs of the same grid placed after the rows (tiles of 8 rows x 128 frames, t_ik
// staged in shared memory): they take the SM slots the rows leave free and those
// the rows release, so the product costs no launch and no wave of its own.
//
// The last line is Eq. (eq:ruinit) in closed form: R'_i = Q D Q^H with Q the
// columns n != n_h of A_i (full column rank) and D = diag(d_n), and the
// back-projected noise image is Q y_{-h}, so y^H (R'_i)^+ y = y_{-h}^H D^{-1}
// y_{-h}.  x is read twice (the second time mostly from L2).
//
// The FP64 warp f = i mod 4 rotates over the CTAs: warps map to the SM's
// sub-partitions by their slot, and with a fixed role every resident CTA's FP64
// work would queue on one sub-partition's FP64 pipe.
//
// A zero pivot (singular W_i) or a noise output with zero power sets the
// null-space bit of the status word (R'_i would not have rank M-1); a
// non-finite R'_i sets the non-finite bit.
#include <float.h>

#include "ilrma.cuh"

namespace rcscm {
namespace {

constexpr int kIlrmaBlock = 128;
constexpr int kIlrmaWarps = kIlrmaBlock / 32;

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Unevaluated FP32 pairs hi + lo: error-free sum (Knuth's TwoSum, 6 additions) and
// the sum of two pairs, renormalised (Dekker's FastTwoSum); no product, so no
// contraction into fused multiply-adds can change them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void pair_add(float& hi, float& lo, float hi2, float lo2) {
    float s, e;
    two_sum(hi, hi2, s, e);
    e += lo + lo2;
    hi = s + e;
    lo = e - (hi - s);
}

// Resident CTAs per SM the register budget is sized for: 7 x 152 SMs hold the
// 1025 rows of a 2048-point STFT in one wave at M <= 4.
constexpr int ilrma_min_blocks(int M) { return M <= 4 ? 7 : 2; }

// r_h0 = T V (Eq. (eq:rhinit)) as a tiled product, in CTAs of the same grid after
// the rows: a CTA makes kRhRows rows x kRhCols frames.  The K dimension goes in
// chunks of kRhK (24 keeps the tile role within the rows' 72-register budget):
// each thread loads its column of V into registers and its share of the rows'
// t_ik, both before the first barrier (one round trip per chunk); the t_ik are
// then read from shared memory four at a time as broadcasts.  Each output sums k
// in increasing order with fused multiply-adds.
constexpr int kRhRows = 8, kRhCols = kIlrmaBlock, kRhK = 24;
constexpr int kRhTPer = (kRhRows * kRhK + kRhCols - 1) / kRhCols;   // t_ik loaded per thread

__device__ void rh_tile(const IlrmaArgs& u, int tile) {
    __shared__ __align__(16) float sT[kRhRows][kRhK];
    const int nx = (u.J + kRhCols - 1) / kRhCols;
    const int i0 = (tile / nx) * kRhRows;
    const int j = (tile % nx) * kRhCols + threadIdx.x;
    float acc[kRhRows];
#pragma unroll
    for (int r = 0; r < kRhRows; ++r) acc[r] = 0.f;
    for (int k0 = 0; k0 < u.K; k0 += kRhK) {
        const int kn = min(kRhK, u.K - k0);
        float v[kRhK], t[kRhTPer];
#pragma unroll
        for (int q = 0; q < kRhTPer; ++q) {
            const int e = threadIdx.x + q * kRhCols;
            const int r = e / kRhK, k = e % kRhK;
            t[q] = (r < kRhRows && i0 + r < u.I && k < kn) ? u.T[(size_t)(i0 + r) * u.K + k0 + k] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < kRhK; ++k) v[k] = (k < kn && j < u.J) ? u.V[(size_t)(k0 + k) * u.J + j] : 0.f;
        __syncthreads();                              // the previous chunk of sT is consumed
#pragma unroll
        for (int q = 0; q < kRhTPer; ++q) {
            const int e = threadIdx.x + q * kRhCols;
            if (e < kRhRows * kRhK) sT[e / kRhK][e % kRhK] = t[q];
        }
        __syncthreads();
#pragma unroll
        for (int k4 = 0; k4 < kRhK; k4 += 4) {
            if (k4 < kn) {
#pragma unroll
                for (int r = 0; r < kRhRows; ++r) {
                    const float4 tr = *reinterpret_cast<const float4*>(&sT[r][k4]);
                    float a = acc[r];
                    a = fmaf(tr.x, v[k4], a);
                    if (k4 + 1 < kn) a = fmaf(tr.y, v[k4 + 1], a);
                    if (k4 + 2 < kn) a = fmaf(tr.z, v[k4 + 2], a);
                    if (k4 + 3 < kn) a = fmaf(tr.w, v[k4 + 3], a);
                    acc[r] = a;
                }
            }
        }
    }
    if (j < u.J) {
#pragma unroll
        for (int r = 0; r < kRhRows; ++r)
            if (i0 + r < u.I) u.rh0[(size_t)(i0 + r) * u.J + j] = acc[r];
    }
}


template <int M>
__global__ void __launch_bounds__(kIlrmaBlock, ilrma_min_blocks(M)) ilrma_init_kernel(IlrmaArgs u, int* status) {
    constexpr int W2 = 2 * M;                          // columns of [W | I]
    constexpr int NE = (M * W2 + 31) / 32;             // entries per lane
    __shared__ double2 aug[M][W2];
    __shared__ float2 w32[M][M];
    __shared__ float2 red[kIlrmaWarps][M];
    __shared__ float sinvd[M];
    __shared__ double sd[M];
    __shared__ int sbad;

    if ((int)blockIdx.x >= u.I) {                      // a T V tile (uniform over the CTA)
        rh_tile(u, (int)blockIdx.x - u.I);
        return;
    }
    const int i = blockIdx.x;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int fw = i & (kIlrmaWarps - 1);              // the FP64 warp of this CTA
    const int wt = tid - 32 * (warp > fw ? 1 : 0);     // index among the other warps' threads
    const int J = u.J, nh = u.n_h;
    const double2* Wi = u.W + (size_t)i * M * M;
    const float2* xi = u.x + (size_t)i * J * M;

    for (int e = tid; e < M * W2; e += kIlrmaBlock) {
        const int r = e / W2, c = e % W2;
        if (c < M) {
            const double2 w = Wi[r * M + c];
            aug[r][c] = w;
            w32[r][c] = make_float2((float)w.x, (float)w.y);
        } else {
            aug[r][c] = make_double2(c - M == r ? 1.0 : 0.0, 0.0);
        }
    }
    if (tid == 0) sbad = 0;
    __syncthreads();

    float ps[M], pc[M];                                // compensated partial sums of |y_n|^2
#pragma unroll
    for (int n = 0; n < M; ++n) ps[n] = pc[n] = 0.f;

    if (warp == fw) {
        // ---- A = W^{-1}: Gauss-Jordan on [W | I] with partial pivoting -----------
        bool singular = false;
        for (int k = 0; k < M; ++k) {
            // pivot: the largest |entry|^2 of column k in rows k..M-1, compared in FP32
            // (any well-sized pivot serves; the lowest row wins ties)
            float best = -1.f;
            int prow = k;
            if (lane >= k && lane < M) {
                best = (float)zabs2(aug[lane][k]);
                prow = lane;
            }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int orow = __shfl_xor_sync(0xffffffffu, prow, o);
                if (ob > best || (ob == best && orow < prow)) {
                    best = ob;
                    prow = orow;
                }
            }
            prow = __shfl_sync(0xffffffffu, prow, 0);
            if (prow != k && lane < W2) {              // swap rows k and prow
                const double2 t = aug[k][lane];
                aug[k][lane] = aug[prow][lane];
                aug[prow][lane] = t;
            }
            __syncwarp();
            const double2 piv = aug[k][k];
            const double pn = zabs2(piv);
            if (!(pn > 0.0)) singular = true;
            const double ipn = pn > 0.0 ? 1.0 / pn : 0.0;
            const double2 ipiv = make_double2(piv.x * ipn, -piv.y * ipn);   // 1 / piv
            double2 rowk[NE], fac[NE];
#pragma unroll
            for (int t = 0; t < NE; ++t) {
                const int e = lane + 32 * t;
                if (e < M * W2) {
                    const int r = e / W2, c = e % W2;
                    rowk[t] = zmul(aug[k][c], ipiv);   // normalised pivot row
                    fac[t] = aug[r][k];
                }
            }
            __syncwarp();
#pragma unroll
            for (int t = 0; t < NE; ++t) {
                const int e = lane + 32 * t;
                if (e < M * W2) {
                    const int r = e / W2, c = e % W2;
                    aug[r][c] = (r == k) ? rowk[t] : zsub(aug[r][c], zmul(fac[t], rowk[t]));
                }
            }
            __syncwarp();
        }
        if (singular && lane == 0) sbad = 1;
    } else {
        // ---- output powers d_n = (1/J) sum_j |w_n^H x_ij|^2 ------------------------
        // S2 frames per thread per round, all loads issued before the arithmetic
        constexpr int S2 = M <= 4 ? 4 : 2;
        constexpr int NT = kIlrmaBlock - 32;
        for (int j0 = wt; j0 < J; j0 += NT * S2) {
            float2 xv[S2][M];
#pragma unroll
            for (int q = 0; q < S2; ++q) {
                const int j = j0 + q * NT;
#pragma unroll
                for (int m = 0; m < M; ++m) xv[q][m] = j < J ? xi[(size_t)j * M + m] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < S2; ++q) {
#pragma unroll
                for (int n = 0; n < M; ++n) {
                    float2 y = make_float2(0.f, 0.f);
#pragma unroll
                    for (int m = 0; m < M; ++m) y = cfma(w32[n][m], xv[q][m], y);
                    kahan_add(ps[n], pc[n], cabs2(y));         // frames past J add exact zeros
                }
            }
        }
    }
    // block sum of the partial powers: compensated FP32 pairs down each warp and across
    // the warps (warp f contributes zeros), one conversion to FP64 at the end
#pragma unroll
    for (int n = 0; n < M; ++n) {
        float hi = ps[n], lo = -pc[n];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
            const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            pair_add(hi, lo, h2, l2);
        }
        if (lane == 0) red[warp][n] = make_float2(hi, lo);
    }
    __syncthreads();
    if (tid < M) {
        float hi = red[0][tid].x, lo = red[0][tid].y;
#pragma unroll
        for (int w = 1; w < kIlrmaWarps; ++w) pair_add(hi, lo, red[w][tid].x, red[w][tid].y);
        const double d = tid == nh ? 0.0 : ((double)hi + (double)lo) / (double)J;
        sd[tid] = d;
        sinvd[tid] = tid == nh ? 0.f : (float)(1.0 / d);
        if (tid != nh && !(d > 0.0)) atomicOr(&sbad, 1);
    }
    __syncthreads();

    if (warp == fw) {
        // ---- a_i and R'_i = A diag(d) A^H, Eq. (eq:rit) ------------------------------
        if (lane < M) u.a[(size_t)i * M + lane] = aug[lane][M + nh];
        bool nonfinite = false;
        for (int e = lane; e < M * M; e += 32) {
            const int r = e / M, c = e % M;
            if (r > c) continue;
            double2 acc = make_double2(0.0, 0.0);
#pragma unroll
            for (int n = 0; n < M; ++n) {          // acc += (d_n A_rn) conj(A_cn)
                const double2 t = zscale(aug[r][M + n], sd[n]);
                const double2 q = aug[c][M + n];
                acc = make_double2(fma(t.x, q.x, fma(t.y, q.y, acc.x)), fma(t.y, q.x, fma(-t.x, q.y, acc.y)));
            }
            if (r == c) acc.y = 0.0;
            nonfinite |= !(fabs(acc.x) <= DBL_MAX) || !(fabs(acc.y) <= DBL_MAX);
            u.Rp[(size_t)i * M * M + r * M + c] = acc;
            u.Rp[(size_t)i * M * M + c * M + r] = zconj(acc);
        }
        if (status) {
            if (__any_sync(0xffffffffu, nonfinite) && lane == 0) atomicOr(status, kFlagNonfinite);
            if (sbad && lane == 0) atomicOr(status, kFlagNullspace);
        }
    }

    // ---- r_u0_ij (Eq. (eq:ruinit), closed form) per frame: x again (mostly from L2),
    // SX frames per thread per round with every load issued before the arithmetic
    constexpr int SX = M <= 4 ? 4 : 2;
    const float invM = 1.f / (float)M;
    for (int j0 = tid; j0 < J; j0 += kIlrmaBlock * SX) {
        float2 xv[SX][M];
#pragma unroll
        for (int q = 0; q < SX; ++q) {
            const int j = j0 + q * kIlrmaBlock;
#pragma unroll
            for (int m = 0; m < M; ++m) xv[q][m] = j < J ? xi[(size_t)j * M + m] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < SX; ++q) {
            const int j = j0 + q * kIlrmaBlock;
            float ru = 0.f;
#pragma unroll
            for (int n = 0; n < M; ++n) {
                float2 y = make_float2(0.f, 0.f);
#pragma unroll
                for (int m = 0; m < M; ++m) y = cfma(w32[n][m], xv[q][m], y);
                ru = fmaf(cabs2(y), sinvd[n], ru);
            }
            if (j < J) u.ru0[(size_t)i * J + j] = ru * invM;
        }
    }
}

}  // namespace

cudaError_t launch_ilrma_init(const IlrmaArgs& u, int* status, cudaStream_t s) {
    if (u.I <= 0 || u.J <= 0) return cudaSuccess;
    const long long n_rh = (long long)((u.J + kRhCols - 1) / kRhCols) * ((u.I + kRhRows - 1) / kRhRows);
    const long long grid = (long long)u.I + n_rh;      // the rows, then the T V tiles
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const unsigned g = (unsigned)grid;
    switch (u.M) {
        case 2: ilrma_init_kernel<2><<<g, kIlrmaBlock, 0, s>>>(u, status); break;
        case 3: ilrma_init_kernel<3><<<g, kIlrmaBlock, 0, s>>>(u, status); break;
        case 4: ilrma_init_kernel<4><<<g, kIlrmaBlock, 0, s>>>(u, status); break;
        case 5: ilrma_init_kernel<5><<<g, kIlrmaBlock, 0, s>>>(u, status); break;
        case 6: ilrma_init_kernel<6><<<g, kIlrmaBlock, 0, s>>>(u, status); break;
        case 7: ilrma_init_kernel<7><<<g, kIlrmaBlock, 0, s>>>(u, status); break;
        case 8: ilrma_init_kernel<8><<<g, kIlrmaBlock, 0, s>>>(u, status); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace rcscm
