/*
 * rcscm_frontend.h -- the front end of rank-constrained SCM estimation on GB300
 * (sm_103a): STFT, ILRMA and inverse STFT, so that the library goes from a
 * multichannel time signal to the extracted target's time signal.
 *
 * The paper (Kubo et al., APSIPA 2019) runs the estimator on the STFT of the
 * observation (Sec. II-A) after ILRMA, whose outputs give a_i, R'_i, r^(h) and
 * r^(u) (Sec. II-B-1, II-B-3; rcscm_ilrma_init in rcscm.h), and fixes the
 * settings (Sec. IV-A, Table II): 16 kHz, a 64 ms Hamming window with a 32 ms
 * shift, K = 10 NMF bases per source, 50 ILRMA iterations, the observation
 * sphered by principal component analysis, W_i = I and non-negative random NMF
 * variables to start.  ILRMA's updates are those of its published algorithm
 * (Kitamura et al., IEEE/ACM TASLP 2016): multiplicative (majorisation-
 * minimisation) updates of the bases T and activations V of each source,
 * iterative-projection updates of each demixing row, then a per-source scale
 * normalisation; T and V are floored at 1e-6 (the normalisation keeps the
 * mean output power at 1, so r = T V stays above 1e-12).
 *
 * Conventions are those of rcscm.h: complex numbers interleaved, arrays dense and
 * row-major in the index order given, `stream` a cudaStream_t passed as void*,
 * pointers are device memory of the current device or page-locked host memory
 * (anything else: RCSCM_EINVAL before any launch), and calls enqueue work without
 * synchronising unless stated.  Status codes are the RCSCM_* codes of rcscm.h.
 */
#ifndef RCSCM_FRONTEND_H
#define RCSCM_FRONTEND_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rcscm_front rcscm_front;

/* A front end for signals of n_samples samples on M microphones (2 <= M <= 8),
 * frames of n_fft samples (a power of two, 16 <= n_fft <= 4096) every `shift`
 * samples (1 <= shift <= n_fft), and K NMF bases per source (1 <= K <= 16).
 * The STFT has I = n_fft / 2 + 1 bins and J frames, the frames starting at
 * j * shift from the first sample with zeros past the end (J = 1 if n_samples <=
 * n_fft, else 1 + ceil((n_samples - n_fft) / shift)).  The context allocates all
 * its working memory here.  Errors: EINVAL, ENOMEM, ECUDA. */
int rcscm_front_create(rcscm_front** f, int64_t M, int64_t n_samples, int n_fft, int shift, int K);
/* I and J of the context's STFT. */
int rcscm_front_shape(const rcscm_front* f, int64_t* I, int64_t* J);
void rcscm_front_destroy(rcscm_front* f);

/* STFT with the periodic Hamming window w[n] = 0.54 - 0.46 cos(2 pi n / n_fft):
 * X[i][j][m] = sum_n w[n] sig[m][j shift + n] exp(-2 pi sqrt(-1) i n / n_fft).
 * sig: float [M][n_samples]; X: complex64 [I][J][M] (the layout of x in
 * rcscm_problem).  FP32 arithmetic (radix-2 FFT in shared memory). */
int rcscm_front_stft(rcscm_front* f, const float* sig, void* X, void* stream);

/* Least-squares inverse STFT: every frame of X (complex64 [I][J][M]) is inverse
 * transformed (the imaginary parts of bins 0 and n_fft/2 are ignored), windowed
 * and overlap-added, and each sample is divided by the sum of the squared windows
 * covering it: out float [M][n_samples].  Applied to an unmodified STFT it
 * returns the signal (to FP32 rounding). */
int rcscm_front_istft(rcscm_front* f, const void* X, float* out, void* stream);

/* ILRMA on the observation X (complex64 [I][J][M]) with N = M sources: sphering
 * (per frequency, C_i = (1/J) sum_j x x^H = E diag(mu) E^H, Q_i = diag(mu)^-1/2 E^H
 * with mu descending; FP64), W_i = I, the caller's non-negative initial NMF
 * variables T0 (float [N][I][K]) and V0 (float [N][K][J]), then n_iter iterations;
 * in each, for n = 0..N-1: T_n, then V_n, then row n of W_i for every i; then the
 * scale normalisation.  Outputs: W (complex128 [I][M][M], the demixing matrices
 * of X itself, W_i Q_i, row n = w_{i,n}^H), T (float [N][I][K]) and V (float
 * [N][K][J]); T[n_h] and V[n_h] with W are the inputs rcscm_ilrma_init takes for
 * target source n_h (the caller chooses n_h; the paper does not say how the
 * target output is identified).  Per-slot sums and the NMF updates in FP32, the
 * covariance, the eigendecomposition and each M x M solve in FP64.  `status` (a
 * device int or NULL) receives RCSCM_ENONFINITE's bit if a non-finite or
 * non-positive value appears.  T, V may alias T0, V0.  The context captures the
 * call's launches into a CUDA graph and replays it while the arguments' addresses
 * and n_iter stay the same (new contents at the same addresses are read anew). */
int rcscm_front_ilrma(rcscm_front* f, const void* X, const float* T0, const float* V0, int n_iter, void* W,
                      float* T, float* V, int* status, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RCSCM_FRONTEND_H */
