/*
 * rcscm_probe.h -- measurement helper of the rank-constrained SCM library.  It has
 * no counterpart in the paper: the accelerated rule's kernels (Algorithm 2,
 * Sec. III-C-2) are bound by the FP32 fused multiply-add pipe, and this probe
 * measures that pipe's throughput on the running GPU, so the benchmark can state
 * their roofline against a measured peak.
 */
#ifndef RCSCM_PROBE_H
#define RCSCM_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Enqueue one launch of n_blocks blocks of 256 threads on `stream` (a
 * cudaStream_t as void*, NULL = legacy default stream); each thread runs n_loops
 * rounds of 16 independent FP32 fused multiply-adds: scalar FFMA when packed = 0,
 * or 8 packed f32x2 FMAs (two lanes each) when packed = 1.  *lane_ops (when not
 * NULL) receives the FP32 lane operations of the launch (one per FMA lane), the
 * numerator of a rate the caller forms with its own CUDA-event timing.  `sink` is
 * a device float array of n_blocks * 256 entries that the kernel may write (it
 * never does for finite inputs; the write keeps the computation from being
 * removed).  Returns RCSCM_OK (0), RCSCM_EINVAL (1) for a non-positive size or a
 * NULL sink, RCSCM_ECUDA (5) if the launch fails. */
int rcscm_probe_fma(int packed, int n_blocks, long long n_loops, float* sink, void* stream, double* lane_ops);

#ifdef __cplusplus
}
#endif
#endif /* RCSCM_PROBE_H */
