// Front end of rank-constrained SCM estimation on sm_103a (declarations and
// contracts in include/rcscm_frontend.h): STFT, inverse STFT and ILRMA.
//
// STFT / inverse STFT (Table II: 64 ms Hamming window, 32 ms shift): one CTA per
// frame; the windowed frames of two microphones are the real and imaginary parts
// of one complex sequence, transformed by an iterative radix-2 FFT in shared
// memory (decimation in time, input in bit-reversed order), and the two real
// spectra are separated with the conjugate symmetry of real signals:
//   A[k] = (Z[k] + conj(Z[N-k])) / 2,  B[k] = (Z[k] - conj(Z[N-k])) / (2 sqrt(-1)).
// The inverse runs the same FFT on Z = A + sqrt(-1) B (conjugate twiddles) and
// writes windowed frames; a second kernel gathers, for every output sample, the
// frames that cover it and divides by the sum of their squared windows (the
// least-squares inverse), in a fixed order, so results do not depend on timing.
//
// ILRMA (the published algorithm, see the header): a CTA per frequency for the
// sphering, the basis update T and the demixing update W; a CTA per tile of 32
// frames for the activation update V, whose sums run over all frequencies.
#include <float.h>
#include <math.h>

#include <algorithm>
#include <new>

#include "rcscm_internal.cuh"
#include "../../include/rcscm_frontend.h"

namespace rcscm {
namespace {

constexpr int kFftThreads = 256;
constexpr int kFrontMaxK = 16;
constexpr float kNmfFloor = 1e-6f;

// Periodic Hamming window (Table II: Hamming).
__device__ __forceinline__ float hamming_w(int n, int N) { return 0.54f - 0.46f * cospif(2.0f * (float)n / (float)N); }

// In-place radix-2 decimation-in-time FFT of buf[0..N) (N a power of two, already in
// bit-reversed order) by the whole CTA; sign = -1 forward, +1 inverse (no scaling).
__device__ void fft_pow2(float2* buf, int N, float sign) {
    for (int len = 2; len <= N; len <<= 1) {
        const int half = len >> 1;
        for (int b = threadIdx.x; b < (N >> 1); b += blockDim.x) {
            const int grp = b / half, pos = b - grp * half;
            const int i0 = grp * len + pos, i1 = i0 + half;
            float s, c;
            sincospif(sign * 2.0f * (float)pos / (float)len, &s, &c);
            const float2 u = buf[i0], v = buf[i1];
            const float2 t = make_float2(c * v.x - s * v.y, c * v.y + s * v.x);
            buf[i0] = make_float2(u.x + t.x, u.y + t.y);
            buf[i1] = make_float2(u.x - t.x, u.y - t.y);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int bitrev(int k, int log2n) { return (int)(__brev((unsigned)k) >> (32 - log2n)); }

// One CTA per frame j: X[i][j][m] for every microphone, two per complex FFT.
__global__ void __launch_bounds__(kFftThreads) stft_kernel(const float* __restrict__ sig, int M, int64_t T,
                                                           int N, int log2n, int shift, int J, float2* __restrict__ X) {
    extern __shared__ float2 zbuf[];
    const int j = blockIdx.x;
    const int I = N / 2 + 1;
    const int64_t t0 = (int64_t)j * shift;
    for (int p = 0; p < M; p += 2) {
        const float* sa = sig + (int64_t)p * T;
        const float* sb = p + 1 < M ? sig + (int64_t)(p + 1) * T : nullptr;
        for (int n = threadIdx.x; n < N; n += blockDim.x) {
            const int64_t t = t0 + n;
            const float w = hamming_w(n, N);
            const float a = t < T ? sa[t] : 0.f;
            const float b = (sb && t < T) ? sb[t] : 0.f;
            zbuf[bitrev(n, log2n)] = make_float2(w * a, w * b);
        }
        __syncthreads();
        fft_pow2(zbuf, N, -1.0f);
        for (int k = threadIdx.x; k < I; k += blockDim.x) {
            const float2 z = zbuf[k], zc = zbuf[(N - k) & (N - 1)];
            // A = (z + conj(zc)) / 2, B = (z - conj(zc)) / (2i)
            const float2 A = make_float2(0.5f * (z.x + zc.x), 0.5f * (z.y - zc.y));
            const float2 B = make_float2(0.5f * (z.y + zc.y), -0.5f * (z.x - zc.x));
            float2* out = X + ((int64_t)k * J + j) * M + p;
            out[0] = A;
            if (p + 1 < M) out[1] = B;
        }
        __syncthreads();
    }
}

// One CTA per frame j: the inverse transforms of two microphones at a time,
// windowed, into frames[m][j][n].
__global__ void __launch_bounds__(kFftThreads) istft_frames_kernel(const float2* __restrict__ X, int M, int N,
                                                                   int log2n, int J, float* __restrict__ frames) {
    extern __shared__ float2 zbuf[];
    const int j = blockIdx.x;
    const int half = N / 2;
    const float scale = 1.0f / (float)N;
    for (int p = 0; p < M; p += 2) {
        for (int k = threadIdx.x; k < N; k += blockDim.x) {
            // Hermitian extension of each real signal's spectrum: S[k] for k <= N/2,
            // conj(S[N-k]) above; the imaginary parts of bins 0 and N/2 are dropped
            const int kk = k <= half ? k : N - k;
            const float2* src = X + ((int64_t)kk * J + j) * M + p;
            float2 A = src[0];
            float2 B = p + 1 < M ? src[1] : make_float2(0.f, 0.f);
            if (kk == 0 || kk == half) {
                A.y = 0.f;
                B.y = 0.f;
            }
            if (k > half) {
                A.y = -A.y;
                B.y = -B.y;
            }
            zbuf[bitrev(k, log2n)] = make_float2(A.x - B.y, A.y + B.x);   // A + i B
        }
        __syncthreads();
        fft_pow2(zbuf, N, 1.0f);
        for (int n = threadIdx.x; n < N; n += blockDim.x) {
            const float w = hamming_w(n, N) * scale;
            const float2 z = zbuf[n];
            frames[((int64_t)p * J + j) * N + n] = w * z.x;
            if (p + 1 < M) frames[((int64_t)(p + 1) * J + j) * N + n] = w * z.y;
        }
        __syncthreads();
    }
}

// Overlap-add by gather: out[m][t] = sum_j frames[m][j][t - j shift] / sum_j w[t - j shift]^2.
__global__ void istft_ola_kernel(const float* __restrict__ frames, int M, int64_t T, int N, int shift, int J,
                                 float* __restrict__ out) {
    const int64_t total = (int64_t)M * T;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(e / T);
        const int64_t t = e - (int64_t)m * T;
        int64_t jlo = t - N + 1 > 0 ? (t - N + 1 + shift - 1) / shift : 0;
        int64_t jhi = t / shift;
        if (jhi > J - 1) jhi = J - 1;
        float acc = 0.f, den = 0.f;
        for (int64_t jj = jlo; jj <= jhi; ++jj) {
            const int n = (int)(t - jj * shift);
            const float w = hamming_w(n, N);
            acc += frames[((int64_t)m * J + jj) * N + n];
            den = fmaf(w, w, den);
        }
        out[e] = den > 0.f ? acc / den : 0.f;
    }
}

// ------------------------------------------------------------------ ILRMA: sphering

// Sum over a CTA of at most 8 warps of NV values per thread (FP64, fixed order): red holds
// 9 * NV doubles, the partials of each warp and then the totals at red[8 * NV + q].
template <int NV>
__device__ void block_sum_d(double (&v)[NV], double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) red[warp * NV + q] = v[q];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w * NV + threadIdx.x];
        red[8 * NV + threadIdx.x] = s;
    }
    __syncthreads();
}

// C_i = (1/J) sum_j x x^H (FP64 accumulation of FP32 products), one CTA per frequency.
template <int M>
__global__ void __launch_bounds__(256) cov_kernel(const float2* __restrict__ X, int J, double2* __restrict__ C) {
    constexpr int NU = M * (M + 1) / 2;
    __shared__ double red[9 * 2 * NU];
    const int i = blockIdx.x;
    double acc[2 * NU];
#pragma unroll
    for (int q = 0; q < 2 * NU; ++q) acc[q] = 0.0;
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        const float2* x = X + ((int64_t)i * J + j) * M;
        float2 xv[M];
#pragma unroll
        for (int m = 0; m < M; ++m) xv[m] = x[m];
        int q = 0;
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int n = m; n < M; ++n) {            // x_m conj(x_n)
                acc[2 * q] += (double)xv[m].x * xv[n].x + (double)xv[m].y * xv[n].y;
                acc[2 * q + 1] += (double)xv[m].y * xv[n].x - (double)xv[m].x * xv[n].y;
                ++q;
            }
    }
    block_sum_d<2 * NU>(acc, red);
    if (threadIdx.x == 0) {
        const double* tot = red + 8 * 2 * NU;
        int q = 0;
        for (int m = 0; m < M; ++m)
            for (int n = m; n < M; ++n) {
                const double2 v = make_double2(tot[2 * q] / J, tot[2 * q + 1] / J);
                C[(int64_t)i * M * M + m * M + n] = v;
                C[(int64_t)i * M * M + n * M + m] = make_double2(v.x, -v.y);
                ++q;
            }
    }
}

// Cyclic Jacobi on a Hermitian M x M matrix in FP64 (one thread): A <- G^H A G with
// the unitary rotation G = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] on (p, q), where
// a_pq = |a_pq| e^{i phi} and t = tan(theta) is the smaller root of
// t^2 + 2 tau t - 1 = 0, tau = (a_qq - a_pp) / (2 |a_pq|); V <- V G.  Sweeps until the
// off-diagonal mass is below 1e-30 of the total.
template <int M>
__device__ void herm_jacobi(double2 (&A)[M][M], double2 (&V)[M][M]) {
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int n = 0; n < M; ++n) V[m][n] = make_double2(m == n ? 1.0 : 0.0, 0.0);
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0, tot = 0.0;
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int n = 0; n < M; ++n) {
                const double v = zabs2(A[m][n]);
                tot += v;
                if (m != n) off += v;
            }
        if (!(off > 1e-30 * tot)) break;
#pragma unroll
        for (int p = 0; p < M - 1; ++p)
#pragma unroll
            for (int q = p + 1; q < M; ++q) {
                const double g2 = zabs2(A[p][q]);
                if (!(g2 > 1e-300)) continue;
                const double g = sqrt(g2);
                const double2 e = make_double2(A[p][q].x / g, A[p][q].y / g);   // e^{i phi}
                const double tau = (A[q][q].x - A[p][p].x) / (2.0 * g);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                const double2 ec = zconj(e);                                    // e^{-i phi}
                // columns: (A G)_kp = c a_kp - s e^{-i phi} a_kq, (A G)_kq = s a_kp + c e^{-i phi} a_kq
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    const double2 ap = A[k][p], aq = zmul(ec, A[k][q]);
                    A[k][p] = make_double2(c * ap.x - s * aq.x, c * ap.y - s * aq.y);
                    A[k][q] = make_double2(s * ap.x + c * aq.x, s * ap.y + c * aq.y);
                    const double2 vp = V[k][p], vq = zmul(ec, V[k][q]);
                    V[k][p] = make_double2(c * vp.x - s * vq.x, c * vp.y - s * vq.y);
                    V[k][q] = make_double2(s * vp.x + c * vq.x, s * vp.y + c * vq.y);
                }
                // rows: row p <- c row p - s e^{i phi} row q, row q <- s row p + c e^{i phi} row q
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    const double2 rp = A[p][k], rq = zmul(e, A[q][k]);
                    A[p][k] = make_double2(c * rp.x - s * rq.x, c * rp.y - s * rq.y);
                    A[q][k] = make_double2(s * rp.x + c * rq.x, s * rp.y + c * rq.y);
                }
                A[p][q] = make_double2(0.0, 0.0);
                A[q][p] = make_double2(0.0, 0.0);
                A[p][p].y = 0.0;
                A[q][q].y = 0.0;
            }
    }
}

// One thread per frequency: eigendecomposition of C_i, Q_i = diag(mu)^-1/2 E^H with mu
// descending (FP64 and FP32 copies), W_i = I.
template <int M>
__global__ void sphere_kernel(const double2* __restrict__ C, int I, double2* __restrict__ Q, float2* __restrict__ Q32,
                              double2* __restrict__ W, float2* __restrict__ W32, int* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I) return;
    double2 A[M][M], V[M][M];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int n = 0; n < M; ++n) A[m][n] = C[(int64_t)i * M * M + m * M + n];
    herm_jacobi<M>(A, V);
    int order[M];
#pragma unroll
    for (int k = 0; k < M; ++k) {                  // rank by descending eigenvalue (ties by index)
        int rank = 0;
#pragma unroll
        for (int l = 0; l < M; ++l) rank += (A[l][l].x > A[k][k].x) || (A[l][l].x == A[k][k].x && l < k);
        order[k] = rank;
    }
    bool bad = false;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        const double mu = A[k][k].x;
        bad |= !(mu > 0.0);
        const double rs = mu > 0.0 ? 1.0 / sqrt(mu) : 0.0;
#pragma unroll
        for (int n = 0; n < M; ++n) {                // row order[k] of Q: e_k^H / sqrt(mu_k)
            const double2 v = make_double2(V[n][k].x * rs, -V[n][k].y * rs);
            const int64_t o = (int64_t)i * M * M + order[k] * M + n;
            Q[o] = v;
            Q32[o] = make_float2((float)v.x, (float)v.y);
        }
    }
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
        for (int n = 0; n < M; ++n) {
            const int64_t o = (int64_t)i * M * M + m * M + n;
            W[o] = make_double2(m == n ? 1.0 : 0.0, 0.0);
            W32[o] = make_float2(m == n ? 1.f : 0.f, 0.f);
        }
    if (bad) atomicOr(status, kFlagNonfinite);
}

// x~ = Q_i x per slot, and P_n = |x~_n|^2 (the outputs of W = I).
template <int M>
__global__ void apply_sphere_kernel(const float2* __restrict__ X, const float2* __restrict__ Q32, int I, int J,
                                    float2* __restrict__ Xs, float* __restrict__ P) {
    const int64_t S = (int64_t)I * J;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(s / J);
        const float2* q = Q32 + (int64_t)i * M * M;
        float2 xv[M];
#pragma unroll
        for (int m = 0; m < M; ++m) xv[m] = X[s * M + m];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            float2 v = make_float2(0.f, 0.f);
#pragma unroll
            for (int n = 0; n < M; ++n) v = cfma(q[k * M + n], xv[n], v);
            Xs[s * M + k] = v;
            P[(int64_t)k * S + s] = cabs2(v);
        }
    }
}

// ------------------------------------------------------------------ ILRMA: updates

// FP32 sum over a CTA of at most 8 warps of NV values per thread, fixed order; red holds
// 9 * NV floats, totals at red[8 * NV + q].
template <int NV>
__device__ void block_sum_fv(float (&v)[NV], float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) red[warp * NV + q] = v[q];
    __syncthreads();
    if (threadIdx.x < NV) {
        float s = 0.f;
        for (int w = 0; w < nw; ++w) s += red[w * NV + threadIdx.x];
        red[8 * NV + threadIdx.x] = s;
    }
    __syncthreads();
}

// Bases of source n, one CTA per frequency i (MM update):
//   t_ik <- max(t_ik sqrt( sum_j p_ij v_kj / r_ij^2 / sum_j v_kj / r_ij ), floor).
__global__ void __launch_bounds__(256) t_update_kernel(const float* __restrict__ V, const float* __restrict__ P,
                                                       float* __restrict__ T, int J, int K) {
    __shared__ float sT[kFrontMaxK];
    __shared__ float red[9 * 2 * kFrontMaxK];
    const int i = blockIdx.x;
    if (threadIdx.x < K) sT[threadIdx.x] = T[(int64_t)i * K + threadIdx.x];
    __syncthreads();
    float acc[2 * kFrontMaxK];
#pragma unroll
    for (int q = 0; q < 2 * kFrontMaxK; ++q) acc[q] = 0.f;
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        float vk[kFrontMaxK];
        float r = 0.f;
#pragma unroll
        for (int k = 0; k < kFrontMaxK; ++k) {
            vk[k] = k < K ? V[(int64_t)k * J + j] : 0.f;
            if (k < K) r = fmaf(sT[k], vk[k], r);
        }
        const float ir = 1.0f / r;
        const float pr = P[(int64_t)i * J + j] * ir * ir;
#pragma unroll
        for (int k = 0; k < kFrontMaxK; ++k) {
            acc[k] = fmaf(pr, vk[k], acc[k]);
            acc[kFrontMaxK + k] = fmaf(ir, vk[k], acc[kFrontMaxK + k]);
        }
    }
    block_sum_fv<2 * kFrontMaxK>(acc, red);
    if (threadIdx.x < K) {
        const float* tot = red + 8 * 2 * kFrontMaxK;
        const int k = threadIdx.x;
        T[(int64_t)i * K + k] = fmaxf(sT[k] * sqrtf(tot[k] / tot[kFrontMaxK + k]), kNmfFloor);
    }
}

// Activations of source n in two kernels.  v_partial_kernel: a CTA of 8 warps per tile of
// 32 frames (lane = frame) and range of frequencies (blockIdx.y of nsplit), the warps
// splitting the range; it writes the range's sums
//   part[s][k][j] = sum_i p_ij t_ik / r_ij^2,  part[s][K + k][j] = sum_i t_ik / r_ij.
// v_finish_kernel adds the ranges in order and updates
//   v_kj <- max(v_kj sqrt( sum_s part[s][k][j] / sum_s part[s][K + k][j] ), floor).
__global__ void __launch_bounds__(256) v_partial_kernel(const float* __restrict__ T, const float* __restrict__ P,
                                                        const float* __restrict__ V, int I, int J, int K, int nsplit,
                                                        float* __restrict__ part) {
    __shared__ float sT[64 * kFrontMaxK];
    __shared__ float red[8 * 2 * kFrontMaxK * 32];
    const int s = blockIdx.y;
    const int i0 = (int)((int64_t)I * s / nsplit), i1 = (int)((int64_t)I * (s + 1) / nsplit);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane;
    const bool on = j < J;
    float vk[kFrontMaxK];
#pragma unroll
    for (int k = 0; k < kFrontMaxK; ++k) vk[k] = (on && k < K) ? V[(int64_t)k * J + j] : 0.f;
    float num[kFrontMaxK], den[kFrontMaxK];
#pragma unroll
    for (int k = 0; k < kFrontMaxK; ++k) num[k] = den[k] = 0.f;
    for (int c0 = i0; c0 < i1; c0 += 64) {           // stage up to 64 frequencies of T at a time
        const int c1 = min(i1, c0 + 64);
        __syncthreads();
        for (int e = threadIdx.x; e < (c1 - c0) * K; e += blockDim.x) sT[e] = T[(int64_t)c0 * K + e];
        __syncthreads();
        if (on) {
            for (int i = c0 + warp; i < c1; i += 8) {
                const float* t = sT + (size_t)(i - c0) * K;
                float r = 0.f;
#pragma unroll
                for (int k = 0; k < kFrontMaxK; ++k)
                    if (k < K) r = fmaf(t[k], vk[k], r);
                const float ir = 1.0f / r;
                const float pr = P[(int64_t)i * J + j] * ir * ir;
#pragma unroll
                for (int k = 0; k < kFrontMaxK; ++k)
                    if (k < K) {
                        num[k] = fmaf(pr, t[k], num[k]);
                        den[k] = fmaf(ir, t[k], den[k]);
                    }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kFrontMaxK; ++k)
        if (k < K) {
            red[((size_t)warp * 2 * K + k) * 32 + lane] = num[k];
            red[((size_t)warp * 2 * K + K + k) * 32 + lane] = den[k];
        }
    __syncthreads();
    if (on)
        for (int q = warp; q < 2 * K; q += 8) {
            float a = 0.f;
            for (int w = 0; w < 8; ++w) a += red[((size_t)w * 2 * K + q) * 32 + lane];
            part[((int64_t)s * 2 * K + q) * J + j] = a;
        }
}

__global__ void v_finish_kernel(const float* __restrict__ part, int J, int K, int nsplit, float* __restrict__ V) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)K * J) return;
    const int k = (int)(e / J), j = (int)(e % J);
    float a = 0.f, b = 0.f;
    for (int s = 0; s < nsplit; ++s) {
        a += part[((int64_t)s * 2 * K + k) * J + j];
        b += part[((int64_t)s * 2 * K + K + k) * J + j];
    }
    V[e] = fmaxf(V[e] * sqrtf(a / b), kNmfFloor);
}

// Demixing row n, one CTA per frequency i (iterative projection):
//   U = (1/J) sum_j x~ x~^H / r_ij (FP32 sums), then in FP64 w = (W_i U)^{-1} e_n,
//   w <- w / sqrt(w^H U w), row n of W_i = w^H; then p_ij = |w^H x~_ij|^2 and its row sum.
template <int M>
__global__ void __launch_bounds__(256) w_update_kernel(const float2* __restrict__ Xs, const float* __restrict__ T,
                                                       const float* __restrict__ V, int n, int J, int K,
                                                       double2* __restrict__ W, float2* __restrict__ W32,
                                                       float* __restrict__ P, double* __restrict__ sumP, int* status) {
    constexpr int NU = M * (M + 1) / 2;
    __shared__ float sT[kFrontMaxK];
    __shared__ float red[9 * 2 * NU];
    __shared__ float2 sw[M];
    __shared__ float redp[9];
    __shared__ double2 sU[M][M], sB[M][M + 1], sF[M];
    const int i = blockIdx.x;
    if (threadIdx.x < K) sT[threadIdx.x] = T[(int64_t)i * K + threadIdx.x];
    __syncthreads();
    float acc[2 * NU];
#pragma unroll
    for (int q = 0; q < 2 * NU; ++q) acc[q] = 0.f;
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        float r = 0.f;
        for (int k = 0; k < K; ++k) r = fmaf(sT[k], V[(int64_t)k * J + j], r);
        const float ir = 1.0f / r;
        const float2* x = Xs + ((int64_t)i * J + j) * M;
        float2 xv[M];
#pragma unroll
        for (int m = 0; m < M; ++m) xv[m] = x[m];
        int q = 0;
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
            for (int b = a; b < M; ++b) {              // x_a conj(x_b) / r
                acc[2 * q] = fmaf(ir, fmaf(xv[a].x, xv[b].x, xv[a].y * xv[b].y), acc[2 * q]);
                acc[2 * q + 1] = fmaf(ir, fmaf(xv[a].y, xv[b].x, -xv[a].x * xv[b].y), acc[2 * q + 1]);
                ++q;
            }
    }
    block_sum_fv<2 * NU>(acc, red);
    if (threadIdx.x < 32) {                           // FP64 solve by the lanes of warp 0
        const int lane = threadIdx.x;
        const float* tot = red + 8 * 2 * NU;
        if (lane < NU) {                              // U (Hermitian) from its upper triangle
            int a = 0, q = lane;
            while (q >= M - a) {
                q -= M - a;
                ++a;
            }
            const int b = a + q;
            const double2 v = make_double2((double)tot[2 * lane] / J, (double)tot[2 * lane + 1] / J);
            sU[a][b] = v;
            sU[b][a] = zconj(v);
        }
        __syncwarp();
        const double2* Wi = W + (int64_t)i * M * M;
        for (int e = lane; e < M * (M + 1); e += 32) {   // [W_i U | e_n]
            const int a = e / (M + 1), b = e % (M + 1);
            double2 v = make_double2(b == M && a == n ? 1.0 : 0.0, 0.0);
            if (b < M)
                for (int k = 0; k < M; ++k) v = zfma(v, Wi[a * M + k], sU[k][b]);
            sB[a][b] = v;
        }
        __syncwarp();
        bool bad = false;
        for (int c = 0; c < M; ++c) {                 // Gauss-Jordan with partial pivoting
            // pivot: the largest |B_rc| over r >= c (magnitudes compared in FP32 across lanes)
            float mag = lane >= c && lane < M ? (float)zabs2(sB[lane][c]) : -1.f;
            int idx = lane;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float om = __shfl_xor_sync(0xffffffffu, mag, o);
                const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
                if (om > mag || (om == mag && oi < idx)) {
                    mag = om;
                    idx = oi;
                }
            }
            const int piv = idx;
            if (piv != c)
                for (int b = lane; b <= M; b += 32) {
                    const double2 t = sB[c][b];
                    sB[c][b] = sB[piv][b];
                    sB[piv][b] = t;
                }
            __syncwarp();
            const double2 pv = sB[c][c];
            const double d2 = zabs2(pv);
            bad |= !(d2 > 0.0);
            const double2 inv = d2 > 0.0 ? make_double2(pv.x / d2, -pv.y / d2) : make_double2(0.0, 0.0);
            if (lane < M) sF[lane] = sB[lane][c];     // the column's factors, before it is cleared
            __syncwarp();
            for (int b = lane; b <= M; b += 32) sB[c][b] = zmul(sB[c][b], inv);
            __syncwarp();
            for (int e = lane; e < M * (M + 1); e += 32) {
                const int r = e / (M + 1), b = e % (M + 1);
                if (r != c && b >= c) sB[r][b] = zsub(sB[r][b], zmul(sF[r], sB[c][b]));
            }
            __syncwarp();
        }
        double qp = 0.0;                              // w^H U w
        if (lane < M) {
            double2 uw = make_double2(0.0, 0.0);
            for (int b = 0; b < M; ++b) uw = zfma(uw, sU[lane][b], sB[b][M]);
            qp = sB[lane][M].x * uw.x + sB[lane][M].y * uw.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) qp += __shfl_xor_sync(0xffffffffu, qp, o);
        bad |= !(qp > 0.0) || !(qp <= DBL_MAX);
        const double sc = qp > 0.0 ? 1.0 / sqrt(qp) : 0.0;
        if (lane < M) {                               // row n = w^H
            const double2 w = sB[lane][M];
            const double2 v = make_double2(w.x * sc, -w.y * sc);
            W[(int64_t)i * M * M + n * M + lane] = v;
            const float2 vf = make_float2((float)v.x, (float)v.y);
            W32[(int64_t)i * M * M + n * M + lane] = vf;
            sw[lane] = vf;
        }
        if (lane == 0 && bad) atomicOr(status, kFlagNonfinite);
    }
    __syncthreads();
    float ps = 0.f;
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        const float2* x = Xs + ((int64_t)i * J + j) * M;
        float2 y = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < M; ++m) y = cfma(sw[m], x[m], y);
        const float p = cabs2(y);
        P[(int64_t)i * J + j] = p;
        ps += p;
    }
    float pv[1] = {ps};
    block_sum_fv<1>(pv, redp);
    if (threadIdx.x == 0) sumP[i] = (double)redp[8];
}

// Scale factors of the normalisation: lam2[n] = (1/(IJ)) sum_ij p_ijn, from the row sums
// of the demixing update, one CTA, FP64 tree in a fixed order.
__global__ void __launch_bounds__(256) scale_kernel(const double* __restrict__ sumP, int N, int I, int J,
                                                    double* __restrict__ lam2, int* status) {
    __shared__ double red[256];
    for (int n = 0; n < N; ++n) {
        double v = 0.0;
        for (int i = threadIdx.x; i < I; i += blockDim.x) v += sumP[(int64_t)n * I + i];
        red[threadIdx.x] = v;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double l2 = red[0] / ((double)I * (double)J);
            lam2[n] = l2;
            if (!(l2 > 0.0) || !(l2 <= DBL_MAX)) atomicOr(status, kFlagNonfinite);
        }
        __syncthreads();
    }
}

// Scale normalisation after the iteration, one CTA per frequency:
//   w_in /= lambda_n, t_ikn /= lambda_n^2, p_ijn /= lambda_n^2.
template <int M>
__global__ void __launch_bounds__(256) normalise_kernel(const double* __restrict__ lam2, int I, int J, int K,
                                                        double2* __restrict__ W, float2* __restrict__ W32,
                                                        float* __restrict__ T, float* __restrict__ P) {
    const int i = blockIdx.x;
    if (threadIdx.x < M * M) {
        const int n = threadIdx.x / M;
        const double il = lam2[n] > 0.0 ? 1.0 / sqrt(lam2[n]) : 1.0;
        const int64_t o = (int64_t)i * M * M + threadIdx.x;
        const double2 v = zscale(W[o], il);
        W[o] = v;
        W32[o] = make_float2((float)v.x, (float)v.y);
    }
    const int64_t S = (int64_t)I * J;
    for (int n = 0; n < M; ++n) {
        const float il2 = lam2[n] > 0.0 ? (float)(1.0 / lam2[n]) : 1.f;
        if (threadIdx.x < K) T[((int64_t)n * I + i) * K + threadIdx.x] *= il2;
        for (int j = threadIdx.x; j < J; j += blockDim.x) P[(int64_t)n * S + (int64_t)i * J + j] *= il2;
    }
}

// W of the observation itself: W_i Q_i (FP64), complex128 output.
template <int M>
__global__ void demix_out_kernel(const double2* __restrict__ W, const double2* __restrict__ Q, int I,
                                 double2* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)I * M * M) return;
    const int i = (int)(e / (M * M)), a = (int)(e % (M * M)) / M, b = (int)(e % M);
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < M; ++k) s = zfma(s, W[(int64_t)i * M * M + a * M + k], Q[(int64_t)i * M * M + k * M + b]);
    out[e] = s;
}

}  // namespace
}  // namespace rcscm

// ------------------------------------------------------------------ C ABI

using namespace rcscm;

struct rcscm_front {
    int M = 0, K = 0, n_fft = 0, log2n = 0, shift = 0, I = 0, J = 0;
    int64_t T = 0;
    float* frames = nullptr;     // [M][J][n_fft] inverse-STFT frames
    float2* Xs = nullptr;        // [I][J][M] sphered observation
    double2* C = nullptr;        // [I][M][M] covariance
    double2* Q = nullptr;        // [I][M][M] sphering (FP64)
    float2* Q32 = nullptr;       // [I][M][M]
    double2* W = nullptr;        // [I][M][M] demixing in the sphered coordinates (FP64)
    float2* W32 = nullptr;       // [I][M][M]
    float* P = nullptr;          // [N][I][J] |y|^2
    double* sumP = nullptr;      // [N][I] row sums of P
    int* status = nullptr;       // [1] status word when the caller passes none
    double* lam2 = nullptr;      // [N] scale factors of the normalisation
    float* vpart = nullptr;      // [nsplit][2K][J] partial sums of the activation update
    int nsplit = 1;              // frequency ranges of the activation update
    // rcscm_front_ilrma's launches captured as a CUDA graph, replayed while its arguments
    // (addresses and iteration count) stay the same
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void* gkey[8] = {};
    int giter = -1;
};

namespace {

int front_view(const void* p, const void** out) { return caller_view(p, out); }

void front_free(rcscm_front* f) {
    if (!f) return;
    cudaFree(f->frames);
    cudaFree(f->Xs);
    cudaFree(f->C);
    cudaFree(f->Q);
    cudaFree(f->Q32);
    cudaFree(f->W);
    cudaFree(f->W32);
    cudaFree(f->P);
    cudaFree(f->sumP);
    cudaFree(f->status);
    cudaFree(f->lam2);
    cudaFree(f->vpart);
    if (f->gexec) cudaGraphExecDestroy(f->gexec);
    if (f->graph) cudaGraphDestroy(f->graph);
    if (f->cap) cudaStreamDestroy(f->cap);
    delete f;
}

template <int M>
cudaError_t ilrma_launches(rcscm_front* f, const float2* X, float* T, float* V, int n_iter, double2* Wout, int* st,
                           cudaStream_t s) {
    const int I = f->I, J = f->J, K = f->K;
    const int64_t S = (int64_t)I * J;
    cov_kernel<M><<<I, 256, 0, s>>>(X, J, f->C);
    sphere_kernel<M><<<(I + 31) / 32, 32, 0, s>>>(f->C, I, f->Q, f->Q32, f->W, f->W32, st);
    const int gs = (int)std::min<int64_t>((S + 255) / 256, 152 * 16);
    apply_sphere_kernel<M><<<gs, 256, 0, s>>>(X, f->Q32, I, J, f->Xs, f->P);
    cudaError_t e = cudaGetLastError();
    const int vt = (J + 31) / 32;
    for (int it = 0; it < n_iter && e == cudaSuccess; ++it) {
        for (int n = 0; n < M; ++n) {
            float* Tn = T + (int64_t)n * I * K;
            float* Vn = V + (int64_t)n * K * J;
            float* Pn = f->P + (int64_t)n * S;
            t_update_kernel<<<I, 256, 0, s>>>(Vn, Pn, Tn, J, K);
            v_partial_kernel<<<dim3(vt, f->nsplit), 256, 0, s>>>(Tn, Pn, Vn, I, J, K, f->nsplit, f->vpart);
            v_finish_kernel<<<(K * J + 255) / 256, 256, 0, s>>>(f->vpart, J, K, f->nsplit, Vn);
            w_update_kernel<M><<<I, 256, 0, s>>>(f->Xs, Tn, Vn, n, J, K, f->W, f->W32, Pn, f->sumP + (int64_t)n * I, st);
        }
        scale_kernel<<<1, 256, 0, s>>>(f->sumP, M, I, J, f->lam2, st);
        normalise_kernel<M><<<I, 256, 0, s>>>(f->lam2, I, J, K, f->W, f->W32, T, f->P);
        e = cudaGetLastError();
    }
    const int64_t nw = (int64_t)I * M * M;
    if (e == cudaSuccess) demix_out_kernel<M><<<(int)((nw + 255) / 256), 256, 0, s>>>(f->W, f->Q, I, Wout);
    return e == cudaSuccess ? cudaGetLastError() : e;
}

int map_err(cudaError_t e) {
    if (e == cudaSuccess) return RCSCM_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return RCSCM_ENOMEM;
    }
    return RCSCM_ECUDA;
}

int ilrma_enqueue(rcscm_front* f, const void* vx, const void* vt0, const void* vv0, int n_iter, const void* vw,
                  const void* vt, const void* vv, const void* vst, cudaStream_t s);

}  // namespace

extern "C" {

int rcscm_front_create(rcscm_front** out, int64_t M, int64_t n_samples, int n_fft, int shift, int K) {
    if (!out) return RCSCM_EINVAL;
    *out = nullptr;
    if (M < 2 || M > kMaxM || n_samples < 1 || n_fft < 16 || n_fft > 4096 || (n_fft & (n_fft - 1)) || shift < 1 ||
        shift > n_fft || K < 1 || K > kFrontMaxK)
        return RCSCM_EINVAL;
    const int64_t J64 = n_samples <= n_fft ? 1 : 1 + (n_samples - n_fft + shift - 1) / shift;
    if (J64 > INT32_MAX / 64) return RCSCM_EINVAL;
    rcscm_front* f = new (std::nothrow) rcscm_front();
    if (!f) return RCSCM_ENOMEM;
    f->M = (int)M;
    f->K = K;
    f->n_fft = n_fft;
    int lg = 0;
    while ((1 << lg) < n_fft) ++lg;
    f->log2n = lg;
    f->shift = shift;
    f->I = n_fft / 2 + 1;
    f->J = (int)J64;
    f->T = n_samples;
    const size_t I = f->I, J = f->J, Mz = (size_t)M, S = I * J;
    cudaError_t e = cudaMalloc(&f->frames, Mz * J * (size_t)n_fft * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&f->Xs, S * Mz * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&f->C, I * Mz * Mz * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&f->Q, I * Mz * Mz * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&f->Q32, I * Mz * Mz * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&f->W, I * Mz * Mz * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&f->W32, I * Mz * Mz * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&f->P, Mz * S * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&f->sumP, Mz * I * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&f->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&f->lam2, Mz * sizeof(double));
    // the activation update's frequency ranges: about two CTAs per SM of 152, at least 8
    // frequencies per range
    const int tiles = (int)((J + 31) / 32);
    f->nsplit = std::max(1, std::min((int)(I / 8), (304 + tiles - 1) / tiles));
    if (e == cudaSuccess) e = cudaMalloc(&f->vpart, (size_t)f->nsplit * 2 * K * J * sizeof(float));
    const size_t fft_smem = (size_t)n_fft * sizeof(float2);
    if (e == cudaSuccess && fft_smem > 48 * 1024) {
        e = cudaFuncSetAttribute(stft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(istft_frames_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_smem);
    }
    if (e != cudaSuccess) {
        front_free(f);
        return map_err(e);
    }
    *out = f;
    return RCSCM_OK;
}

int rcscm_front_shape(const rcscm_front* f, int64_t* I, int64_t* J) {
    if (!f) return RCSCM_EINVAL;
    if (I) *I = f->I;
    if (J) *J = f->J;
    return RCSCM_OK;
}

void rcscm_front_destroy(rcscm_front* f) {
    if (!f) return;
    cudaDeviceSynchronize();
    front_free(f);
}

int rcscm_front_stft(rcscm_front* f, const float* sig, void* X, void* stream) {
    const void *vs = nullptr, *vx = nullptr;
    if (!f || front_view(sig, &vs) || front_view(X, &vx)) return RCSCM_EINVAL;
    stft_kernel<<<f->J, kFftThreads, (size_t)f->n_fft * sizeof(float2), static_cast<cudaStream_t>(stream)>>>(
        static_cast<const float*>(vs), f->M, f->T, f->n_fft, f->log2n, f->shift, f->J,
        static_cast<float2*>(const_cast<void*>(vx)));
    return map_err(cudaGetLastError());
}

int rcscm_front_istft(rcscm_front* f, const void* X, float* out, void* stream) {
    const void *vx = nullptr, *vo = nullptr;
    if (!f || front_view(X, &vx) || front_view(out, &vo)) return RCSCM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    istft_frames_kernel<<<f->J, kFftThreads, (size_t)f->n_fft * sizeof(float2), s>>>(
        static_cast<const float2*>(vx), f->M, f->n_fft, f->log2n, f->J, f->frames);
    const int64_t total = (int64_t)f->M * f->T;
    const int g = (int)std::min<int64_t>((total + 255) / 256, 152 * 32);
    istft_ola_kernel<<<g, 256, 0, s>>>(f->frames, f->M, f->T, f->n_fft, f->shift, f->J,
                                       static_cast<float*>(const_cast<void*>(vo)));
    return map_err(cudaGetLastError());
}

int rcscm_front_ilrma(rcscm_front* f, const void* X, const float* T0, const float* V0, int n_iter, void* W,
                      float* T, float* V, int* status, void* stream) {
    const void *vx, *vt0, *vv0, *vw, *vt, *vv, *vst = nullptr;
    if (!f || n_iter < 0 || front_view(X, &vx) || front_view(T0, &vt0) || front_view(V0, &vv0) ||
        front_view(W, &vw) || front_view(T, &vt) || front_view(V, &vv) || (status && front_view(status, &vst)))
        return RCSCM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const void* key[8] = {vx, vt0, vv0, vw, vt, vv, vst, nullptr};
    bool same = f->gexec && f->giter == n_iter;
    for (int k = 0; k < 8 && same; ++k) same = f->gkey[k] == key[k];
    if (same) return map_err(cudaGraphLaunch(f->gexec, s));
    // capture the launches on the context's own stream, then replay the graph on `stream`
    cudaError_t e = cudaSuccess;
    if (!f->cap) e = cudaStreamCreateWithFlags(&f->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(f->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return map_err(e);
    const int st = ilrma_enqueue(f, vx, vt0, vv0, n_iter, vw, vt, vv, vst, f->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(f->cap, &g);
    if (st != RCSCM_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return st != RCSCM_OK ? st : map_err(e);
    }
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return map_err(e);
    }
    if (f->gexec) cudaGraphExecDestroy(f->gexec);
    if (f->graph) cudaGraphDestroy(f->graph);
    f->graph = g;
    f->gexec = x;
    f->giter = n_iter;
    for (int k = 0; k < 8; ++k) f->gkey[k] = key[k];
    return map_err(cudaGraphLaunch(f->gexec, s));
}

}  // extern "C"

namespace {

// The work of rcscm_front_ilrma on stream s (captured into the context's graph).
int ilrma_enqueue(rcscm_front* f, const void* vx, const void* vt0, const void* vv0, int n_iter, const void* vw,
                  const void* vt, const void* vv, const void* vst, cudaStream_t s) {
    const size_t nT = (size_t)f->M * f->I * f->K * sizeof(float), nV = (size_t)f->M * f->K * f->J * sizeof(float);
    cudaError_t e = cudaSuccess;
    if (vt != vt0) e = cudaMemcpyAsync(const_cast<void*>(vt), vt0, nT, cudaMemcpyDefault, s);
    if (e == cudaSuccess && vv != vv0) e = cudaMemcpyAsync(const_cast<void*>(vv), vv0, nV, cudaMemcpyDefault, s);
    int* st = vst ? static_cast<int*>(const_cast<void*>(vst)) : f->status;
    if (e == cudaSuccess && !vst) e = cudaMemsetAsync(f->status, 0, sizeof(int), s);
    if (e != cudaSuccess) return map_err(e);
    const float2* Xp = static_cast<const float2*>(vx);
    float* Tp = static_cast<float*>(const_cast<void*>(vt));
    float* Vp = static_cast<float*>(const_cast<void*>(vv));
    double2* Wp = static_cast<double2*>(const_cast<void*>(vw));
    switch (f->M) {
        case 2: e = ilrma_launches<2>(f, Xp, Tp, Vp, n_iter, Wp, st, s); break;
        case 3: e = ilrma_launches<3>(f, Xp, Tp, Vp, n_iter, Wp, st, s); break;
        case 4: e = ilrma_launches<4>(f, Xp, Tp, Vp, n_iter, Wp, st, s); break;
        case 5: e = ilrma_launches<5>(f, Xp, Tp, Vp, n_iter, Wp, st, s); break;
        case 6: e = ilrma_launches<6>(f, Xp, Tp, Vp, n_iter, Wp, st, s); break;
        case 7: e = ilrma_launches<7>(f, Xp, Tp, Vp, n_iter, Wp, st, s); break;
        default: e = ilrma_launches<8>(f, Xp, Tp, Vp, n_iter, Wp, st, s); break;
    }
    return map_err(e);
}

}  // namespace
