// Internal types and device helpers shared by the CUDA translation units of
// the rank-constrained SCM library (sm_103a).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rcscm.h"

namespace rcscm {

constexpr int kMaxM = RCSCM_MAX_M;
constexpr int kSlotBlock = 256;   // threads per block of the slot-parallel kernels

// Status bits (bit k-1 for status code k).
constexpr int kFlagNullspace = 1 << (RCSCM_ENULLSPACE - 1);
constexpr int kFlagNonfinite = 1 << (RCSCM_ENONFINITE - 1);
constexpr int kFlagClamp = 1 << (RCSCM_ECLAMP - 1);
constexpr int kFlagBounds = 1 << (RCSCM_EBOUNDS - 1);

// Index checks of the debug build (compiled with -DRCSCM_DEBUG; compute-sanitizer
// is not available).  RCSCM_CTA_CHECK takes a condition that is uniform over the
// CTA and is placed before the kernel's first barrier: on failure thread 0 sets the
// bounds bit of the status word and the whole CTA returns, so no buffer is touched
// out of range and nothing traps.  The normal build compiles the checks away.
#ifdef RCSCM_DEBUG
#define RCSCM_CTA_CHECK(cond, status)                                  \
    do {                                                               \
        if (!(cond)) {                                                 \
            if (threadIdx.x == 0) atomicOr((status), kFlagBounds);     \
            return;                                                    \
        }                                                              \
    } while (0)
#else
#define RCSCM_CTA_CHECK(cond, status) \
    do {                              \
    } while (0)
#endif

// One row = one (utterance, frequency bin i).  Rows share nothing in any rule.
struct RowDesc {
    int64_t slot_off;       // first slot of the row in the per-slot arrays
    int64_t out_off;        // first complex element of the row in the concatenated h_out
    int64_t scratch_off;    // naive rule: first float of the row's R^u scratch
    int64_t a_off;          // first element of the row in concatenated [I][M] arrays (grad_a)
    int64_t rp_off;         // first element of the row in concatenated [I][M][M] arrays (grad_Rp)
    const float2* x;        // row start in the caller's x  (J x M complex64)
    const double2* a;       // caller's a_i                 (M complex128)
    const double2* Rp;      // caller's R'_i                (M x M complex128), or nullptr
    const float2* Rp_c64;   // caller's R'_i given as complex64, or nullptr
    const double2* b_in;    // caller's b_i to validate (M complex128), or nullptr
    const double* lambda0;  // caller's lambda_i or nullptr
    const float* rh0;       // caller's r^(h)_i.  (J floats)
    const float* ru0;       // caller's r^(u)_i.  (J floats)
    int J, M, prob, freq;
};

// Per-row FP32 constants used by the slot kernels (derived in FP64 by setup).
struct __align__(16) RowConst {
    float taa;      // tau^(aa)_i                   Eq. (eq:taa)
    float taaM;     // tau^(aa)_i / M
    float inv_taa;  // 1 / tau^(aa)_i
    float sab2;     // |sigma^(ab)_i|^2
    float sab_re;   // sigma^(ab)_i                  Eq. (eq:sap)
    float sab_im;
    float invM;     // 1 / M
    float pad;
};

// A block of the slot-parallel kernels covers slots [j0, j0 + kSlotBlock) of one row.
struct BlockMap {
    int row;
    int j0;
};

// Device arrays owned by a context.
struct DevState {
    RowDesc* rows;         // [R]
    RowConst* rc;          // [R]
    BlockMap* bmap;        // [n_blocks]
    int* order;            // [R] rows by descending J (iterate launch order)
    // FP64 setup outputs, fixed stride kMaxM per row
    double2* b64;          // [R][8]
    double* mu;            // [R][8]
    double* lam0;          // [R]
    double* taa64;         // [R]
    double2* sab64;        // [R]
    // FP32 copies for the slot kernels
    float2* phi;           // [R][8][8]  rows: (R'^+ a)^H, Householder complement, b^H
    float2* a32;           // [R][8]
    float2* b32;           // [R][8]
    float2* rp32;          // [R][8][8]  (naive rule, printed coordinates)
    float2* wht32;         // [R][8][8]  whitening rows (naive rule): row 0 b^H, row k >= 1
                           //            e_k^H / sqrt(mu_k), e_k the eigenvectors of R' (ascending)
    double2* aw64;         // [R][8]     whitened steering vector a_k = e_k^H a / sqrt(mu_k), k >= 1
    double2* evec64;       // [R][64] eigenvectors of R', entry m * M + i = e_i[m], ascending (adjoint), or nullptr
    float* ckpt_rh;        // checkpoints written by the accelerated kernel when ckpt_stride > 0:
    float* ckpt_ru;        //   the state entering pass k * ckpt_stride, [k][S] and [k][R]
    float* ckpt_lam;
    int ckpt_stride;
    int64_t n_slots, n_rows;   // S and R of the context
    // per-slot invariants and EM state
    float4* inv4;          // [S] {tau_ax.re, tau_ax.im, sigma_bx.re, sigma_bx.im}
    float* kap;            // [S] kappa = tau_xx - |tau_ax|^2 / tau_aa
    float* rh;             // [S]
    float* ru;             // [S]
    float* lam;            // [R]
    void* ru_hat;          // naive rules: packed Hermitian R^u per slot (float or double)
    int* status;           // [1]
    int* counter;          // [1] row counter of the persistent accelerated kernel
    double* obj_part;      // [n_blocks] objective partial sums (per slot block)
    int n_sm;              // multiprocessors of the device
};

struct IterParams {
    float c_a2;      // 1 / (alpha + 2)
    float c_b;       // beta / (alpha + 2)
    float ru_floor;
    double c_a2_f64; // the same constants in FP64 (naive FP64 rule)
    double c_b_f64;
    int ckpt_first;        // index (since setup) of the first pass of this launch
};

// Entry e (row-major, m * M + n) of the caller's R'_i, in FP64 whatever its input type.
__device__ __forceinline__ double2 rp_entry(const RowDesc& q, int e) {
    if (q.Rp_c64) {
        const float2 v = q.Rp_c64[e];
        return make_double2((double)v.x, (double)v.y);
    }
    return q.Rp[e];
}

// Row r lies in the tables and its shape fits a kernel covering max_j frames (the
// debug build's row check).
__device__ __forceinline__ bool row_ok(const DevState& d, int r, int max_j) {
    if (r < 0 || r >= d.n_rows) return false;
    const RowDesc& q = d.rows[r];
    return q.M >= 1 && q.M <= kMaxM && q.J >= 1 && q.J <= max_j && q.slot_off >= 0 && q.slot_off + q.J <= d.n_slots;
}
// A slot block of a slot-parallel kernel starts inside its row.
__device__ __forceinline__ bool block_ok(const DevState& d, const BlockMap& bm) {
    return row_ok(d, bm.row, 1 << 30) && bm.j0 >= 0 && bm.j0 < d.rows[bm.row].J;
}

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // conj(a) * b
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
// acc += a * b
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}
// acc += conj(a) * b
__device__ __forceinline__ float2 cfmac(float2 a, float2 b, float2 acc) {
    return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zmulc(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double zabs2(double2 a) { return a.x * a.x + a.y * a.y; }
// acc + a b, acc + conj(a) b and acc - conj(a) b, two fused multiply-adds per component
// (every FP64 instruction counts on sm_103a).
__device__ __forceinline__ double2 zfma(double2 acc, double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 zfma_c(double2 acc, double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 zfms_c(double2 acc, double2 a, double2 b) {
    return make_double2(fma(-a.x, b.x, fma(-a.y, b.y, acc.x)), fma(-a.x, b.y, fma(a.y, b.x, acc.y)));
}

// Hardware reciprocal approximation (MUFU.RCP, relative error ~1 ulp); inputs
// here are positive normal numbers.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Per-slot invariants from the row's projection Phi (M x M, row-major, Phi x:
// row 0 gives tau_ax, row M-1 sigma_bx, rows 1..M-2 the components whose squared
// norm is kappa = tau_xx - |tau_ax|^2 / tau_aa).  out = {tau_ax, sigma_bx}.
template <int M>
__device__ __forceinline__ void project_vals(const float2* __restrict__ phi, const float2 (&xv)[M], float4& out,
                                             float& kappa) {
    float2 z0 = make_float2(0.f, 0.f), zb = make_float2(0.f, 0.f);
#pragma unroll
    for (int n = 0; n < M; ++n) {
        z0 = cfma(phi[n], xv[n], z0);
        zb = cfma(phi[(M - 1) * M + n], xv[n], zb);
    }
    float kap = 0.f;
#pragma unroll
    for (int k = 1; k <= M - 2; ++k) {
        float2 zk = make_float2(0.f, 0.f);
#pragma unroll
        for (int n = 0; n < M; ++n) zk = cfma(phi[k * M + n], xv[n], zk);
        kap += cabs2(zk);
    }
    out = make_float4(z0.x, z0.y, zb.x, zb.y);
    kappa = kap;
}
template <int M>
__device__ __forceinline__ void project_slot(const float2* __restrict__ phi, const float2* __restrict__ xs,
                                             float4& out, float& kappa) {
    float2 xv[M];
#pragma unroll
    for (int n = 0; n < M; ++n) xv[n] = xs[n];
    project_vals<M>(phi, xv, out, kappa);
}

// Projection of one slot for a runtime M (2..8).
__device__ __forceinline__ void project_slot_m(int M, const float2* __restrict__ phi, const float2* __restrict__ xs,
                                               float4& out, float& kappa) {
    switch (M) {
        case 2: project_slot<2>(phi, xs, out, kappa); break;
        case 3: project_slot<3>(phi, xs, out, kappa); break;
        case 4: project_slot<4>(phi, xs, out, kappa); break;
        case 5: project_slot<5>(phi, xs, out, kappa); break;
        case 6: project_slot<6>(phi, xs, out, kappa); break;
        case 7: project_slot<7>(phi, xs, out, kappa); break;
        default: project_slot<8>(phi, xs, out, kappa); break;
    }
}

// Wiener weight w of the posterior mean h = w a (Sec. II-A; Sherman-Morrison,
// Eq. (eq:rijxinv)): w = r_h rho_ax / (r_u + r_h rho_aa) with rho_ax = tau_ax +
// sigma_ab sigma_bx / lambda and rho_aa = tau_aa + |sigma_ab|^2 / lambda.
// Every operation is explicit (fmaf, IEEE division), so each kernel that calls it
// rounds identically.
__device__ __forceinline__ float2 wiener_weight(float taa, float sab2, float2 sab, float lam, float4 inv, float rh,
                                                float ru) {
    const float il = 1.0f / lam;
    const float ur = fmaf(sab.x, inv.z, -(sab.y * inv.w));      // sigma_ab sigma_bx
    const float ui = fmaf(sab.x, inv.w, sab.y * inv.z);
    const float raxr = fmaf(ur, il, inv.x), raxi = fmaf(ui, il, inv.y);
    const float raa = fmaf(sab2, il, taa);
    const float k = rh / fmaf(rh, raa, ru);
    return make_float2(raxr * k, raxi * k);
}

// w a_m with explicit fused multiply-adds (identical rounding in every kernel).
__device__ __forceinline__ float2 cmul_exact(float2 w, float2 a) {
    return make_float2(fmaf(w.x, a.x, -(w.y * a.y)), fmaf(w.x, a.y, w.y * a.x));
}


// Butterfly sum over a warp: every lane ends with the same, order-fixed value.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace rcscm

// Accelerated kernel shapes: threads per row (32 ... 1024) and the largest
// number of slots each thread keeps in registers for that block size.
__host__ __device__ constexpr int accel_max_spt(int block) { return block >= 1024 ? 4 : 8; }
// Default block for rows of up to max_j slots: the smallest block that keeps
// at most 8 slots per thread.
inline int accel_default_block(int max_j) {
    int b = 32;
    while (b < 512 && b * 8 < max_j) b *= 2;
    return b;
}
inline bool accel_block_ok(int block) {
    return block == 0 || block == 32 || block == 64 || block == 128 || block == 256 || block == 512 || block == 1024;
}
inline int accel_max_j(int block) { return block ? block * accel_max_spt(block) : 512 * 8; }
// Block of the adjoint kernel (and of the forward kernel of a context that keeps
// checkpoints): 128 threads for rows up to 512 frames, 256 up to 2048; 0 beyond.
inline int adjoint_block(int max_j) { return max_j <= 512 ? 128 : (max_j <= 2048 ? 256 : 0); }

// Per-row record handed from the adjoint's row kernel to its setup-adjoint kernel (doubles):
// the role sums C (M*M), v_a (M), v_b (M) as (re, im) pairs, then g_tau_aa, g_sigma_ab (re, im)
// and the Wiener filter's gradient of a (2 kMaxM).
constexpr int kAdjGtaa = 2 * (rcscm::kMaxM * rcscm::kMaxM + 2 * rcscm::kMaxM);
constexpr int kAdjGsab = kAdjGtaa + 1;
constexpr int kAdjGaw = kAdjGsab + 2;
constexpr int kAdjSums = kAdjGaw + 2 * rcscm::kMaxM;

struct AdjointArgs {
    const float2* grad_h;   // upstream gradient of h (concatenated, like h_out)
    float2* grad_x;         // like x, concatenated
    double2* grad_a;        // [rows][M] concatenated
    double2* grad_Rp;       // [rows][M][M] concatenated
    const float* ckpt_rh;   // [n_ckpt][S]: state entering pass k * stride
    const float* ckpt_ru;
    const float* ckpt_lam;  // [n_ckpt][R]
    float* seg_rh;          // [stride][S] states entering the passes of one segment (scratch)
    float* seg_ru;          // [stride][S]
    float* seg_lam;         // [stride][R]
    double* sums;           // [R][kAdjSums] each row's sums for the setup adjoint (scratch)
    int K;                  // passes run since setup
    int stride;             // passes between checkpoints
    int64_t S, R;
};

// Launchers (defined in the .cu files, called by the C ABI in api.cu).
namespace rcscm {
// The address under which the current device reaches caller memory p (api.cu): device
// or managed memory of this device as is, page-locked host memory through its device
// view.  RCSCM_EINVAL for anything else (pageable host memory, another device, an
// invalid address, NULL); allocates nothing.
int caller_view(const void* p, const void** out);
// Device status word of a context (api.cu), for the host pipeline's asynchronous status reads.
int* ctx_status_word(rcscm_ctx* c);
// The fused form (rcscm_run) on rows [first_row, first_row + n_rows) of a context in the
// fused configuration, on `s` (api.cu; for the host pipeline).  h is the output of the
// whole context: each row is written at its own offset in it.
int run_rows(rcscm_ctx* c, int first_row, int n_rows, int n_iter, float2* h, cudaStream_t s);
// Device state arrays of a context (r_h, r_u per slot, lambda per row; api.cu).
void ctx_state(rcscm_ctx* c, float** rh, float** ru, float** lam);
// True when rcscm_run applies to the context (accelerated rule, no checkpoints, all passes
// in one launch).
bool ctx_fused(const rcscm_ctx* c);
// max_m: the largest M among the rows (selects the kernel shape).
cudaError_t launch_setup(const DevState& d, int n_rows, int max_m, double null_tol, cudaStream_t s);
cudaError_t launch_invariants(const DevState& d, int n_blocks, cudaStream_t s);
// h != nullptr: the fused form (invariants from x, the passes, then the Wiener
// output into h), for a state freshly set by the setup kernel.
cudaError_t launch_accel(const DevState& d, int n_rows, int max_j, int block, int n_iter,
                         const IterParams& p, bool persistent, cudaStream_t s, float2* h = nullptr);
// Observed-data log posterior: per slot block partials, then per-utterance sums
// (block ranges [first_block[p], first_block[p + 1])) into out[p].
cudaError_t launch_objective(const DevState& d, int n_blocks, const IterParams& p, double alpha, double beta,
                             const int* first_block, int n_probs, double* out, cudaStream_t s);
// rows_by_m: device list of row indices grouped by M; count_by_m / first_by_m:
// host arrays indexed by M (size kMaxM + 1) giving each group's size and start.
// rule: RCSCM_RULE_NAIVE (FP32, whitened coordinates), RCSCM_RULE_NAIVE_F64 or
// RCSCM_RULE_NAIVE_PRINTED (FP64 / FP32 in the printed coordinates).
cudaError_t launch_naive(const DevState& d, const int* rows_by_m, const int* count_by_m,
                         const int* first_by_m, int n_iter, const IterParams& p, int rule, cudaStream_t s);
cudaError_t launch_extract(const DevState& d, int n_blocks, float2* h_out, cudaStream_t s);
// First-stage rule (accel1.cu): threads per row for rows of up to max_j frames (0: too long).
int accel1_block(int max_j);
// rows_by_m / count_by_m / first_by_m as for launch_naive.
cudaError_t launch_accel1(const DevState& d, const int* rows_by_m, const int* count_by_m, const int* first_by_m,
                          int max_j, int n_iter, const IterParams& p, cudaStream_t s);
cudaError_t launch_adjoint(const DevState& d, int n_rows, int max_j, int max_m, int block, const AdjointArgs& a,
                           const IterParams& p, cudaStream_t s);
}  // namespace rcscm
