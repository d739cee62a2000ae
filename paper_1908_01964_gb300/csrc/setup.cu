// Per-frequency setup (FP64 results) and per-slot invariants (FP32) of the
// rank-constrained SCM estimator, sm_103a.
//
// setup_kernel   one group of 16 lanes per row (utterance, frequency i):
//   R' <- (R' + R'^H)/2, Hermitian eigendecomposition (parallel FP32 Jacobi
//   sweeps, then iterative refinement of the eigenbasis to FP64 accuracy),
//   b_i = eigenvector of the smallest eigenvalue (Sec. II-B-1), lambda_i = the
//   next eigenvalue unless given (Sec. II-B-3), (R')^+ from the remaining pairs
//   (Eq. (eq:riinv)), tau^(aa)_i (Eq. (eq:taa)), sigma^(ab)_i (Eq. (eq:sap)),
//   and the per-frequency projection Phi_i (M x M) used by invariants_kernel:
//     row 0        (R'^+ a)^H                 -> z_0     = tau^(ax)_ij
//     rows 1..M-2  H_k L^H, R'^+ = L L^H       -> sum |z_k|^2 = kappa_ij
//     row M-1      b^H                        -> z_{M-1} = sigma^(bx)_ij
//   H is the Householder reflector that maps u = L^H a / |L^H a| to a multiple
//   of e_0, so the rows 1..M-2 span the whitened complement of u and
//   kappa = tau^(xx) - |tau^(ax)|^2 / tau^(aa) >= 0 is formed as a sum of
//   squares, without the cancellation of the difference.
//
//   The kernel is latency-bound on one row's chain of dependent operations, and
//   on sm_103a every FP64 instruction (conversions included) holds the FP64 pipe
//   of its SM sub-partition for tens of cycles per warp.  So FP64 is kept to the
//   quantities whose accuracy needs it: the refinement's residuals and the
//   FP64 outputs.  The Jacobi sweeps, the refinement's correction terms (of
//   order |E|, where FP32 rounding adds 6e-8 |E|) and the FP32 per-row
//   constants run on the FP32 pipe.
//
// invariants_kernel  one thread per slot: z = Phi_i x_ij, and initial state.
#include <float.h>

#include "rcscm_internal.cuh"

namespace rcscm {
namespace {

constexpr int kSetupWarps = 2;
constexpr int kGroupLanes = 16;                             // lanes per row
constexpr int kSetupRows = kSetupWarps * 32 / kGroupLanes;  // rows per block
// Matrix entries per lane: NE = 1 when every row of the launch has M <= 4 (the
// kernel is instantiated for NE = 1 and NE = kMaxEntries, so the common small-M
// launch carries neither the code nor the registers of the larger one).
constexpr int kMaxEntries = kMaxM * kMaxM / kGroupLanes;
constexpr int kJacobiMaxSweeps32 = 12;
constexpr int kRefineMaxSteps = 6;

__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2((float)v.x, (float)v.y); }

// Sum / maximum over the 16 lanes of a row group (xor offsets stay in the group).
__device__ __forceinline__ float group_sum_f(float v) {
#pragma unroll
    for (int o = kGroupLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// The same sum where only this row's group takes part (mask = the group's 16 lanes).
__device__ __forceinline__ float group_sum_masked(float v, unsigned mask) {
#pragma unroll
    for (int o = kGroupLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}
__device__ __forceinline__ float group_max_f(float v) {
#pragma unroll
    for (int o = kGroupLanes / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Integer key with the order of the doubles (negative values: low 63 bits flipped),
// so that ranks are a permutation for any input, NaN included.
__device__ __forceinline__ long long order_key(double v) {
    const long long b = __double_as_longlong(v);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}

// Partner of index x in round r (0 <= r < n - 1) of the circle schedule over n
// indices (n even): index 0 keeps position 0, the others advance one position per
// round, and the indices at positions k and n - 1 - k meet.  Over n - 1 rounds
// every pair meets once.
__device__ __forceinline__ int circle_partner(int x, int r, int n) {
    const int n1 = n - 1;
    int pos = x - 1 + r;
    pos = pos >= n1 ? pos - n1 : pos;
    pos = x == 0 ? 0 : pos + 1;
    const int P = n1 - pos;
    int v = P - 1 - r;
    v = v < 0 ? v + n1 : v;
    return P == 0 ? 0 : v + 1;
}

// Jacobi rotation of the pair (p, q), p < q, that zeroes A_pq.  With
// A_pq = m e^{i phi} and h = A_qq - A_pp, U = [[c, s], [-s e^{-i phi}, c e^{-i phi}]]
// on rows/columns (p, q), cos(2 theta) = |h| / sqrt(h^2 + 4 m^2), c = cos(theta),
// s = sign(h) sin(theta) (|theta| <= pi/4); c and s come from three reciprocal
// square roots.  The identity (on = false) when disabled, when p == q (an index
// without a partner this round) or when A_pq is negligible.
struct PairRot {
    float c, s, m, app, aqq;
    float2 ec;    // conj(e^{i phi})
    bool on;
};
__device__ __forceinline__ PairRot pair_rot(const float2 (*A)[kMaxM], int p, int q, bool enable, float skip2) {
    PairRot t;
    t.app = A[p][p].x;
    t.aqq = A[q][q].x;
    const float2 apq = A[p][q];
    const float m2 = cabs2(apq);
    const float h = t.aqq - t.app;
    const float inv_m = rsqrtf(m2);
    const float r = rsqrtf(fmaf(h, h, 4.f * m2));
    const float u = fmaf(0.5f * fabsf(h), r, 0.5f);
    const float ru = rsqrtf(u);
    // computed unconditionally (no branch between the two rotations of a round) and
    // replaced by the identity where the rotation does not apply
    t.on = enable && p != q && m2 > 0.f && m2 > skip2 * fabsf(t.app * t.aqq);
    t.m = t.on ? m2 * inv_m : 0.f;
    t.c = t.on ? u * ru : 1.f;
    t.s = t.on ? copysignf(t.m * r * ru, h) : 0.f;
    t.ec = t.on ? make_float2(apq.x * inv_m, -apq.y * inv_m) : make_float2(1.f, 0.f);
    return t;
}

// Column k of a pair's U: (U_pk, U_qk) = (c, -s conj(e)) for k = p, (s, c conj(e)) for
// k = q; (1, 0) for an index without a partner.
__device__ __forceinline__ void rot_column(const PairRot& t, bool k_is_p, float& up, float2& uq) {
    up = k_is_p ? t.c : t.s;
    uq = k_is_p ? cscale(t.ec, -t.s) : cscale(t.ec, t.c);
}

// Parallel cyclic Jacobi in FP32 on the Hermitian matrix of this lane's group.
// A sweep is n - 1 rounds of the circle schedule over n = M rounded up to even
// indices; in a round the disjoint pairs rotate together, A <- U^H A U and
// V <- V U, U the block-diagonal product of the pairs' rotations.  The warp runs
// the rounds of its largest n; a group whose own rounds, or sweeps, are done
// applies the identity (an exact copy), so each row's result does not depend on
// the row that shares its warp.  Lanes own matrix entries and form the new ones from the previous
// round's buffers (ping-pong), one warp synchronisation per round:
//   new A_ij = conj(U_{p_i i}) (A_{p_i p_j} U_{p_j j} + A_{p_i q_j} U_{q_j j})
//            + conj(U_{q_i i}) (A_{q_i p_j} U_{p_j j} + A_{q_i q_j} U_{q_j j})
// for i < j in different pairs (mirrored into A_ji, so A stays exactly Hermitian),
// A_pq = 0 and the closed-form 2 x 2 diagonal for the rotated pair's own entries.
// Sweeps stop when the off-diagonal mass is at most tol2 |A|_F^2 in every group of
// the warp.  Returns the buffer that holds the final A and V.  Control flow that
// contains warp-wide synchronisation is uniform over the warp.
template <int NE>
__device__ int jacobi_parallel(float2 (*Ab0)[kMaxM], float2 (*Ab1)[kMaxM], float2 (*Vb0)[kMaxM],
                               float2 (*Vb1)[kMaxM], int M, int l, float fro2, float tol2, float skip2,
                               int max_sweeps) {
    const int n = M + (M & 1);
    const int nw = __reduce_max_sync(0xffffffffu, n);
    const int MM = M * M;
    int ei[NE], ej[NE];                       // this lane's entries (i, j)
#pragma unroll
    for (int t = 0; t < NE; ++t) {
        const int e = l + kGroupLanes * t;
        ei[t] = e < MM ? e / M : 0;
        ej[t] = e < MM ? e - (e / M) * M : 0;
    }
    int cur = 0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        const float2(*A)[kMaxM] = cur ? Ab1 : Ab0;
        float off = 0.f;
#pragma unroll
        for (int t = 0; t < NE; ++t)
            if (l + kGroupLanes * t < MM && ei[t] < ej[t]) off += cabs2(A[ei[t]][ej[t]]);
        off = group_sum_f(off);
        const bool conv = !(off > tol2 * fro2);
        if (__all_sync(0xffffffffu, conv)) break;
        for (int rd = 0; rd < nw - 1; ++rd) {
            const bool rot = !conv && rd < n - 1;
            const float2(*Ac)[kMaxM] = cur ? Ab1 : Ab0;
            const float2(*Vc)[kMaxM] = cur ? Vb1 : Vb0;
            float2(*An)[kMaxM] = cur ? Ab0 : Ab1;
            float2(*Vn)[kMaxM] = cur ? Vb0 : Vb1;
#pragma unroll
            for (int t = 0; t < NE; ++t) {
                if (l + kGroupLanes * t < MM) {
                    const int i = ei[t], j = ej[t];
                    // partners only within this group's own rounds (past them the schedule
                    // formula leaves [0, n)); an index without a partner below M stays put
                    int pi = circle_partner(i, rd, n);
                    int pj = circle_partner(j, rd, n);
                    pi = (rd < n - 1 && pi >= 0 && pi < M) ? pi : i;
                    pj = (rd < n - 1 && pj >= 0 && pj < M) ? pj : j;
                    const int ip = min(i, pi), iq = max(i, pi), jp = min(j, pj), jq = max(j, pj);
                    // every operand first, then both rotations (independent chains)
                    const float2 vp = Vc[i][jp], vq = Vc[i][jq];
                    const float2 a00 = Ac[ip][jp], a01 = Ac[ip][jq], a10 = Ac[iq][jp], a11 = Ac[iq][jq];
                    const PairRot rj = pair_rot(Ac, jp, jq, rot, skip2);
                    const PairRot ri = pair_rot(Ac, ip, iq, rot, skip2);
                    float bp, ap;
                    float2 bq, aq;
                    rot_column(rj, j == jp, bp, bq);
                    rot_column(ri, i == ip, ap, aq);
                    Vn[i][j] = cadd(cscale(vp, bp), cmul(vq, bq));
                    if (i == j) {
                        float2 v = (i == ip) ? a00 : a11;             // A_ii (unrotated)
                        if (rj.on) {
                            const float cs2m = 2.f * rj.c * rj.s * rj.m;
                            v = (i == jp) ? make_float2(fmaf(rj.c * rj.c, rj.app, fmaf(rj.s * rj.s, rj.aqq, -cs2m)), 0.f)
                                          : make_float2(fmaf(rj.s * rj.s, rj.app, fmaf(rj.c * rj.c, rj.aqq, cs2m)), 0.f);
                        }
                        An[i][i] = v;
                    } else if (i < j) {
                        float2 v = make_float2(0.f, 0.f);           // the rotated pair's own entry
                        if (!(ip == jp && iq == jq && rj.on)) {
                            const float2 rp = cadd(cscale(a00, bp), cmul(a01, bq));
                            const float2 rq = cadd(cscale(a10, bp), cmul(a11, bq));
                            v = cadd(cscale(rp, ap), cmulc(aq, rq));
                        }
                        An[i][j] = v;
                        An[j][i] = cconj(v);
                    }
                }
            }
            __syncwarp();
            cur ^= 1;
        }
    }
    return cur;
}

// One row per group of 16 lanes (2 rows per warp).  The eigendecomposition of
// R' runs in two phases.  Phase 1: parallel Jacobi sweeps in FP32 give
// approximate eigenvectors X.  Phase 2: iterative refinement of the whole
// eigenbasis (Ogita and Aishima's method, written here for Hermitian matrices):
//   R = I - X^H X,  S = X^H R' X,  lambda_i = S_ii / (1 - R_ii),
//   E_ij = (S_ij + lambda_j R_ij) / (lambda_j - lambda_i)   (i != j, separated),
//   E_ij = R_ij / 2                                         (diagonal, clusters),
//   X <- X (I + E),
// which converges quadratically.  R, S and lambda are the residuals and take
// FP64; E and the product X E are corrections of order |E| and take FP32 (their
// rounding, 6e-8 |E|, is below the next step's |E|^2 until |E| reaches 1e-7),
// with X += X E accumulated in FP64.  1/(1 - R_ii) is the series
// 1 + R_ii + R_ii^2, whose error R_ii^3 is below FP64 rounding because the
// columns of X are unit vectors to FP32 accuracy (unitary rotations).  Lanes own
// matrix entries (at most 4 each).  Control flow that contains warp-wide
// synchronisation is uniform over the warp.
template <int NE>
__global__ void __launch_bounds__(kSetupWarps * 32)
setup_kernel(DevState d, int n_rows, double null_tol) {
    __shared__ double2 sA[kSetupRows][kMaxM][kMaxM];    // R' (symmetrised)
    __shared__ double2 sX[kSetupRows][kMaxM][kMaxM];    // eigenvectors (columns)
    __shared__ double2 sT[kSetupRows][kMaxM][kMaxM];    // R' X; later Householder data
    __shared__ float2 sJ[kSetupRows][4][kMaxM][kMaxM];  // Jacobi A, V (two buffers each); later E
    __shared__ float2 sX32[kSetupRows][kMaxM][kMaxM];   // FP32 copy of X for X E
    __shared__ float2 sA32[kSetupRows][kMaxM][kMaxM];   // FP32 copy of R'
    __shared__ double slam[kSetupRows][kMaxM];
    __shared__ double2 sa[kSetupRows][kMaxM];
    __shared__ double2 sc[kSetupRows][kMaxM];
    __shared__ double2 sf[kSetupRows][kMaxM];           // c_i / mu_i
    __shared__ double srs[kSetupRows][kMaxM];
    __shared__ float2 sb32[kSetupRows][kMaxM];
    __shared__ int sperm[kSetupRows][kMaxM];

    // the fused row kernel that follows may start now: it waits for this grid's results
    asm volatile("griddepcontrol.launch_dependents;");
    const int g = threadIdx.x / kGroupLanes;
    const int l = threadIdx.x % kGroupLanes;
    const int r = blockIdx.x * kSetupRows + g;
    bool active = r < n_rows;
    RowDesc rd;
    if (active) rd = d.rows[r];
#ifdef RCSCM_DEBUG
    if (active && !(rd.M >= 1 && rd.M <= kMaxM)) {    // the debug build's shape check (group-uniform)
        if (l == 0) atomicOr(d.status, kFlagBounds);
        active = false;
    }
#endif
    const int M = active ? rd.M : 0;
    const int MM = M * M;
    double2(*A)[kMaxM] = sA[g];
    double2(*X)[kMaxM] = sX[g];
    double2(*T)[kMaxM] = sT[g];
    float2(*X32)[kMaxM] = sX32[g];
    float2(*E32)[kMaxM] = sJ[g][0];

    float afro2 = 0.f;
    for (int e = l; e < MM; e += kGroupLanes) {
        const int m = e / M, n = e % M;
        const double2 amn = rp_entry(rd, m * M + n);
        const double2 anm = rp_entry(rd, n * M + m);
        const double2 h = make_double2(0.5 * (amn.x + anm.x), 0.5 * (amn.y - anm.y));
        A[m][n] = h;
        const float2 hf = to_f2(h);
        afro2 += cabs2(hf);
        sJ[g][0][m][n] = hf;
        sA32[g][m][n] = hf;
        sJ[g][2][m][n] = make_float2(m == n ? 1.f : 0.f, 0.f);
    }
    if (l < M) {
        const double2 av = rd.a[l];
        sa[g][l] = av;
        d.a32[(size_t)r * kMaxM + l] = to_f2(av);
    }
    afro2 = group_sum_f(afro2);
    const float afro = sqrtf(afro2);
    __syncwarp();

    // ---- phase 1: FP32 Jacobi sweeps ---------------------------------------------
    const int jc = jacobi_parallel<NE>(sJ[g][0], sJ[g][1], sJ[g][2], sJ[g][3], M, l, afro2, 1e-12f, 1e-14f,
                                   kJacobiMaxSweeps32);
    for (int e = l; e < MM; e += kGroupLanes) {
        const float2 v = sJ[g][2 + jc][e / M][e % M];
        X[e / M][e % M] = make_double2(v.x, v.y);
        X32[e / M][e % M] = v;
    }
    __syncwarp();

    // ---- phase 2: refinement of the eigenbasis ------------------------------------
    int ei[NE], ej[NE];                       // this lane's entries (i, j)
#pragma unroll
    for (int t = 0; t < NE; ++t) {
        const int e = l + kGroupLanes * t;
        ei[t] = e < MM ? e / M : 0;
        ej[t] = e < MM ? e - (e / M) * M : 0;
    }
    bool done = false;                  // this group's refinement has converged
    bool clustered = false;             // its last step treated some pair as a cluster
    for (int step = 0; step < kRefineMaxSteps; ++step) {
        double2 rv[NE], sv[NE];
#pragma unroll
        for (int t = 0; t < NE; ++t) {                     // R = I - X^H X, T = R' X (FP64)
            const int e = l + kGroupLanes * t;
            if (e < MM) {
                const int i = ei[t], j = ej[t];
                double2 rr = make_double2(i == j ? 1.0 : 0.0, 0.0), tt = make_double2(0.0, 0.0);
                for (int m = 0; m < M; ++m) {
                    rr = zfms_c(rr, X[m][i], X[m][j]);
                    tt = zfma(tt, A[i][m], X[m][j]);
                }
                rv[t] = rr;
                T[i][j] = tt;
                if (step > 0) X32[i][j] = to_f2(X[i][j]);
            }
        }
        __syncwarp();
        float so2 = 0.f, rr2 = 0.f;
#pragma unroll
        for (int t = 0; t < NE; ++t) {                     // S = X^H T (FP64), lambda
            const int e = l + kGroupLanes * t;
            if (e < MM) {
                const int i = ei[t], j = ej[t];
                double2 ss = make_double2(0.0, 0.0);
                for (int m = 0; m < M; ++m) ss = zfma_c(ss, X[m][i], T[m][j]);
                sv[t] = ss;
                if (i == j) {
                    const double rii = rv[t].x;
                    if (!done) slam[g][i] = fma(ss.x, rii * (1.0 + rii), ss.x);
                } else {
                    so2 += cabs2(to_f2(ss));
                }
                rr2 += cabs2(to_f2(rv[t]));
            }
        }
        so2 = group_sum_f(so2);
        rr2 = group_sum_f(rr2);
        const float delta = 2.f * (sqrtf(so2) + afro * sqrtf(rr2));
        __syncwarp();
        float emax = 0.f, clus = 0.f;
#pragma unroll
        for (int t = 0; t < NE; ++t) {                     // E (FP32)
            const int e = l + kGroupLanes * t;
            if (e < MM) {
                const int i = ei[t], j = ej[t];
                float2 ee;
                if (i == j) {
                    ee = make_float2(0.5f * (float)rv[t].x, 0.f);
                } else {
                    const double lj = slam[g][j];
                    const float dl = (float)(lj - slam[g][i]);
                    ee = fabsf(dl) > delta ? cscale(to_f2(zadd(sv[t], zscale(rv[t], lj))), 1.f / dl)
                                           : cscale(to_f2(rv[t]), 0.5f);
                    clus = fabsf(dl) > delta ? clus : 1.f;
                }
                E32[i][j] = ee;
                emax = fmaxf(emax, cabs2(ee));
            }
        }
        emax = group_max_f(emax);
        clus = group_max_f(clus);
        if (!done) clustered = clus > 0.f;                 // this group's last step treated a cluster
        __syncwarp();
#pragma unroll
        for (int t = 0; t < NE; ++t) {                     // X <- X + X E
            const int e = l + kGroupLanes * t;
            if (e < MM && !done) {
                const int i = ei[t], j = ej[t];
                float2 xe = make_float2(0.f, 0.f);
                for (int k = 0; k < M; ++k) xe = cadd(xe, cmul(X32[i][k], E32[k][j]));
                X[i][j] = zadd(X[i][j], make_double2(xe.x, xe.y));
            }
        }
        __syncwarp();
        // |E| <= 1e-6 was just applied: the remaining error is of order |E|^2 <= 1e-12 (scaled by
        // the eigenvalue gaps) plus the FP32 rounding of the correction, far below the FP32
        // outputs' rounding and the tolerances of the FP64 rule and the adjoint.  A converged
        // group leaves X and lambda alone while the other group of its warp continues.
        done = done || !(emax > 1e-12f);
        if (__all_sync(0xffffffffu, done)) break;
    }

    // ---- phase 3: exact rotations inside clusters (FP64) ---------------------------
    // The refinement's correction (S_ij + lambda_j R_ij) / (lambda_j - lambda_i) is a
    // first-order step, taken only for pairs whose eigenvalues are further apart than its
    // threshold delta; for closer pairs (a cluster) it restores orthogonality alone.  A
    // rotation inside such a pair that the FP32 Jacobi could not resolve -- two small
    // eigenvalues of R' a few FP32 units of |R'| apart, as ILRMA's noise estimate gives
    // at low frequencies, where the null vector b and the 1/mu_2 term of (R')^+ depend on
    // it -- is therefore never undone.  Here S = X^H R' X is formed again in FP64, and every
    // pair whose eigenvector angle |S_pq| / |S_pp - S_qq| is still above 1e-9 (a converged
    // pair sits near 1e-12, an unresolved cluster at 1e-7 to 1e-1) gets the exact 2 x 2
    // Jacobi rotation (applied to S and X) by lane 0 of its group, and the eigenvalues are
    // the Rayleigh quotients S_kk / |x_k|^2; rows without such a pair skip it.
    {
        // only rows whose refinement did not converge or ended with a cluster take part
        const bool redo = active && (clustered || !done);
#pragma unroll
        for (int t = 0; t < NE; ++t) {                     // T = R' X
            const int e = l + kGroupLanes * t;
            if (redo && e < MM) {
                const int i = ei[t], j = ej[t];
                double2 tt = make_double2(0.0, 0.0);
                for (int m = 0; m < M; ++m) tt = zfma(tt, A[i][m], X[m][j]);
                T[i][j] = tt;
            }
        }
        __syncwarp();
        double2 sv[NE];
#pragma unroll
        for (int t = 0; t < NE; ++t) {                     // S = X^H T
            const int e = l + kGroupLanes * t;
            sv[t] = make_double2(0.0, 0.0);
            if (redo && e < MM) {
                const int i = ei[t], j = ej[t];
                for (int m = 0; m < M; ++m) sv[t] = zfma_c(sv[t], X[m][i], T[m][j]);
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < NE; ++t)
            if (redo && l + kGroupLanes * t < MM) T[ei[t]][ej[t]] = sv[t];     // T now holds S
        __syncwarp();
        float couple = 0.f;
#pragma unroll
        for (int t = 0; t < NE; ++t) {
            const int e = l + kGroupLanes * t;
            if (redo && e < MM && ei[t] != ej[t]) {
                const float gap = (float)(T[ei[t]][ei[t]].x - T[ej[t]][ej[t]].x);
                const float off2 = cabs2(to_f2(sv[t]));
                couple = fmaxf(couple, off2 > 1e-18f * gap * gap ? 1.f : 0.f);
            }
        }
        couple = group_max_f(couple);
        if (redo && couple > 0.f && l == 0) {
            for (int p = 0; p < M - 1; ++p)
                for (int q = p + 1; q < M; ++q) {
                    const double g2 = zabs2(T[p][q]);
                    const double gap = T[q][q].x - T[p][p].x;
                    if (!(g2 > 1e-18 * gap * gap) || !(g2 > 0.0)) continue;
                    const double gm = sqrt(g2);
                    const double2 ep = make_double2(T[p][q].x / gm, T[p][q].y / gm);   // e^{i phi}
                    const double2 ec = zconj(ep);
                    const double tau = gap / (2.0 * gm);
                    const double tn = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    const double c = 1.0 / sqrt(1.0 + tn * tn), sn = tn * c;
                    for (int k = 0; k < M; ++k) {         // columns of S and X: S G, X G
                        const double2 sp = T[k][p], sq = zmul(ec, T[k][q]);
                        T[k][p] = make_double2(c * sp.x - sn * sq.x, c * sp.y - sn * sq.y);
                        T[k][q] = make_double2(sn * sp.x + c * sq.x, sn * sp.y + c * sq.y);
                        const double2 xp = X[k][p], xq = zmul(ec, X[k][q]);
                        X[k][p] = make_double2(c * xp.x - sn * xq.x, c * xp.y - sn * xq.y);
                        X[k][q] = make_double2(sn * xp.x + c * xq.x, sn * xp.y + c * xq.y);
                    }
                    for (int k = 0; k < M; ++k) {         // rows of S: G^H S
                        const double2 rp = T[p][k], rq = zmul(ep, T[q][k]);
                        T[p][k] = make_double2(c * rp.x - sn * rq.x, c * rp.y - sn * rq.y);
                        T[q][k] = make_double2(sn * rp.x + c * rq.x, sn * rp.y + c * rq.y);
                    }
                    T[p][q] = make_double2(0.0, 0.0);
                    T[q][p] = make_double2(0.0, 0.0);
                }
        }
        __syncwarp();
        if (redo && l < M) {                         // unit columns, Rayleigh quotients
            double n2 = 0.0;
            for (int m = 0; m < M; ++m) n2 += zabs2(X[m][l]);
            slam[g][l] = T[l][l].x / n2;
            const double rn = rsqrt(n2);
            for (int m = 0; m < M; ++m) X[m][l] = zscale(X[m][l], rn);
        }
        __syncwarp();
    }

    // ---- ascending order of the eigenvalues (ranks) --------------------------------
    if (l < M) {
        const long long kl = order_key(slam[g][l]);
        int rank = 0;
        for (int j = 0; j < M; ++j) {
            const long long kj = order_key(slam[g][j]);
            rank += (kj < kl) || (kj == kl && j < l);
        }
        sperm[g][rank] = l;
    }
    __syncwarp();
    if (!active) return;                       // only group-local synchronisation follows
    const unsigned gmask = 0xffffu << (threadIdx.x & 16);
    const int* perm = sperm[g];
    const double mu1 = slam[g][perm[0]];
    const double mu2 = slam[g][perm[1]];
    const double muM = slam[g][perm[M - 1]];
    const int k0 = perm[0];
    if (l < M) {
        d.mu[(size_t)r * kMaxM + l] = slam[g][perm[l]];
        const double2 bv = X[l][k0];
        const float2 bf = to_f2(bv);
        d.b64[(size_t)r * kMaxM + l] = bv;
        d.b32[(size_t)r * kMaxM + l] = bf;
        sb32[g][l] = bf;
    }
    if (d.evec64)                              // eigenbasis for the adjoint
        for (int e = l; e < MM; e += kGroupLanes) d.evec64[(size_t)r * 64 + e] = X[e / M][perm[e % M]];
    // c_i = e_i^H a, 1/sqrt(mu_i) and c_i / mu_i for the nonzero eigenpairs (sorted index i = 1..M-1)
    if (l >= 1 && l < M) {
        const int kk = perm[l];
        double2 acc = make_double2(0.0, 0.0);
        for (int m = 0; m < M; ++m) acc = zfma_c(acc, X[m][kk], sa[g][m]);
        const double rs = rsqrt(slam[g][kk]);
        sc[g][l] = acc;
        srs[g][l] = rs;
        sf[g][l] = zscale(acc, rs * rs);
    }
    __syncwarp(gmask);

    // whitening rows of R~_i = R' + lambda~ b b^H for the naive rule: G_0 = b^H (scaled by
    // 1/sqrt(lambda~) at each pass), G_k = e_k^H / sqrt(mu_k) (k >= 1), so G R~ G^H = I; and
    // the fixed part of the whitened steering vector, (G a)_k = c_k / sqrt(mu_k)
    if (d.wht32) {
        for (int e = l; e < MM; e += kGroupLanes) {
            const int kk = e / M, n = e % M;
            const double2 v = kk == 0 ? zconj(X[n][k0]) : zscale(zconj(X[n][perm[kk]]), srs[g][kk]);
            d.wht32[(size_t)r * 64 + e] = to_f2(v);
        }
        if (l < M) d.aw64[(size_t)r * kMaxM + l] = l == 0 ? make_double2(0.0, 0.0) : zscale(sc[g][l], srs[g][l]);
    }
    // a caller-supplied null vector b must be the eigenvector of the smallest eigenvalue
    // (Sec. II-B-1): |R' b| <= 1e-6 |R'|_F |b| and |b^H e_1| >= (1 - 1e-6) |b|
    bool bad_b = false;
    if (rd.b_in) {
        float rb2 = 0.f, bb2 = 0.f, ov_re = 0.f, ov_im = 0.f;
        if (l < M) {
            double2 rb = make_double2(0.0, 0.0);
            for (int n = 0; n < M; ++n) rb = zfma(rb, A[l][n], rd.b_in[n]);
            const double2 bl = rd.b_in[l];
            const double2 ov = zmulc(bl, X[l][k0]);
            rb2 = (float)zabs2(rb);
            bb2 = (float)zabs2(bl);
            ov_re = (float)ov.x;
            ov_im = (float)ov.y;
        }
        rb2 = group_sum_masked(rb2, gmask);
        bb2 = group_sum_masked(bb2, gmask);
        ov_re = group_sum_masked(ov_re, gmask);
        ov_im = group_sum_masked(ov_im, gmask);
        const float t = 1.f - 1e-6f;
        bad_b = !(bb2 > 0.f) || !(rb2 <= 1e-12f * afro2 * bb2) || !(ov_re * ov_re + ov_im * ov_im >= t * t * bb2);
    }

    double taa = 0.0;                          // tau^(aa) = sum_i |c_i|^2 / mu_i
    for (int i = 1; i < M; ++i) taa = fma(sc[g][i].x, sf[g][i].x, fma(sc[g][i].y, sf[g][i].y, taa));
    double2 sab = make_double2(0.0, 0.0);
    for (int m = 0; m < M; ++m) sab = zfma_c(sab, sa[g][m], X[m][k0]);

    const bool bad = !(mu2 > 0.0) || !(fabs(mu1) <= null_tol * muM) || !(taa > 0.0);
    if (l == 0 && (bad || bad_b)) atomicOr(d.status, kFlagNullspace);
    const double lam0 = rd.lambda0 ? rd.lambda0[0] : mu2;

    // Householder vector for u = v / |v|, v_i = c_{i+1} / sqrt(mu_{i+1}), i = 0..M-2
    const double inv_nv = taa > 0.0 ? rsqrt(taa) : 0.0;
    const double2 u0 = zscale(sc[g][1], srs[g][1] * inv_nv);
    const double au02 = zabs2(u0);
    const double inv_au0 = au02 > 0.0 ? rsqrt(au02) : 0.0;
    const double au0 = au02 * inv_au0;
    const double2 ph0 = au02 > 0.0 ? zscale(u0, inv_au0) : make_double2(1.0, 0.0);
    // w = u - alpha e_0 with alpha = -ph0 |u| -> w_0 = ph0 (|u_0| + 1); 2 / |w|^2 = 1 / (1 + |u_0|)
    const double two_over_wn2 = 1.0 / (1.0 + au0);

    // Householder data shared by the rows of Phi (in the refinement's T array, free by
    // now): w_i and conj(w_i) / sqrt(mu_i) (i = 1..M-1), then
    // q_n = sum_i conj(w_i e_i[n]) / sqrt(mu_i), once per n.
    double2* wd = &T[0][0];
    double2* hq = &T[1][0];
    double2* qd = &T[2][0];
    if (l >= 1 && l < M) {   // w = u - alpha e_0 in the whitened basis, u_i = c_{i+1} / (sqrt(mu_{i+1}) |v|)
        const double2 w = (l == 1) ? zscale(ph0, au0 + 1.0) : zscale(sc[g][l], inv_nv * srs[g][l]);
        wd[l] = w;
        hq[l] = zscale(zconj(w), srs[g][l]);
    }
    __syncwarp(gmask);
    if (l < M) {
        double2 q = make_double2(0.0, 0.0);
        for (int i = 1; i < M; ++i) q = zfma_c(q, X[l][perm[i]], hq[i]);
        qd[l] = q;
    }
    __syncwarp(gmask);
    // FP32 copy of R' with the smallest eigenvalue set to zero (R' + lambda b b^H is then
    // exactly the model's R_i); formed in FP32 (mu_1 b b^H is a rounding-level term)
    const float mu1f = (float)mu1;
    if (d.rp32)
        for (int e = l; e < MM; e += kGroupLanes) {
            const int m = e / M, n = e % M;
            d.rp32[(size_t)r * 64 + e] = csub(sA32[g][m][n], cscale(cmul(sb32[g][m], cconj(sb32[g][n])), mu1f));
        }
    // Phi entries (kk, n): row 0 (R'^+ a)^H, rows 1..M-2 H L^H, row M-1 b^H (FP64, rounded once)
    float2* phi = d.phi + (size_t)r * 64;
    for (int e = l; e < MM; e += kGroupLanes) {
        const int kk = e / M, n = e % M;
        double2 val;
        if (kk == 0) {                                   // conj(g_n), g = R'^+ a = sum_i e_i c_i / mu_i
            double2 gv = make_double2(0.0, 0.0);
            for (int i = 1; i < M; ++i) gv = zfma(gv, X[n][perm[i]], sf[g][i]);
            val = zconj(gv);
        } else if (kk == M - 1) {
            val = zconj(X[n][k0]);
        } else {                                         // H L^H entry, L = [e_i / sqrt(mu_i)]
            val = zsub(zscale(zconj(X[n][perm[kk + 1]]), srs[g][kk + 1]),
                       zscale(zmul(wd[kk + 1], qd[n]), two_over_wn2));
        }
        phi[e] = to_f2(val);
    }
    if (l == 0) {
        d.lam0[r] = lam0;
        d.taa64[r] = taa;
        d.sab64[r] = sab;
        RowConst c;                                      // FP32 per-row constants, formed in FP32
        const float taaf = (float)taa;
        const float2 sabf = to_f2(sab);
        const float invM = 1.f / (float)M;
        c.taa = taaf;
        c.taaM = taaf * invM;
        c.inv_taa = taa > 0.0 ? 1.f / taaf : 1.f;
        c.sab2 = cabs2(sabf);
        c.sab_re = sabf.x;
        c.sab_im = sabf.y;
        c.invM = invM;
        c.pad = 0.f;
        d.rc[r] = c;
        d.lam[r] = (float)lam0;
    }
}

__global__ void __launch_bounds__(kSlotBlock) invariants_kernel(DevState d) {
    __shared__ float2 sphi[kMaxM * kMaxM];
    __shared__ __align__(16) float2 sx[kSlotBlock * kMaxM];
    const BlockMap bm = d.bmap[blockIdx.x];
    RCSCM_CTA_CHECK(block_ok(d, bm), d.status);
    const RowDesc* rd = d.rows + bm.row;
    const int M = rd->M;
    const int J = rd->J;
    const int n = min(kSlotBlock, J - bm.j0);            // slots of this block
    const int t = threadIdx.x;
    const int j = bm.j0 + t;
    float rh0 = 0.f, ru0 = 0.f;                        // in flight while x is staged
    if (t < n) {
        rh0 = rd->rh0[j];
        ru0 = rd->ru0[j];
    }
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) sphi[e] = d.phi[(size_t)bm.row * 64 + e];
    // stage the block's x (n * M complex, contiguous) with coalesced 16-byte loads when aligned
    const float2* src = rd->x + (size_t)bm.j0 * M;
    const int nc = n * M;
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const float4* s4 = reinterpret_cast<const float4*>(src);
        float4* d4 = reinterpret_cast<float4*>(sx);
        for (int e = threadIdx.x; e < nc / 2; e += blockDim.x) d4[e] = s4[e];
        if ((nc & 1) && threadIdx.x == 0) sx[nc - 1] = src[nc - 1];
    } else {
        for (int e = threadIdx.x; e < nc; e += blockDim.x) sx[e] = src[e];
    }
    __syncthreads();
    if (t >= n) return;
    const float2* xs = sx + t * M;
    float4 o;
    float kap;
    project_slot_m(M, sphi, xs, o, kap);
    const int64_t s = rd->slot_off + j;
    d.inv4[s] = o;
    d.kap[s] = kap;
    d.rh[s] = rh0;
    d.ru[s] = ru0;
}

}  // namespace

cudaError_t launch_setup(const DevState& d, int n_rows, int max_m, double null_tol, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    const int grid = (n_rows + kSetupRows - 1) / kSetupRows;
    if (max_m * max_m <= kGroupLanes)
        setup_kernel<1><<<grid, kSetupWarps * 32, 0, s>>>(d, n_rows, null_tol);
    else
        setup_kernel<kMaxEntries><<<grid, kSetupWarps * 32, 0, s>>>(d, n_rows, null_tol);
    return cudaGetLastError();
}

cudaError_t launch_invariants(const DevState& d, int n_blocks, cudaStream_t s) {
    if (n_blocks <= 0) return cudaSuccess;
    invariants_kernel<<<n_blocks, kSlotBlock, 0, s>>>(d);
    return cudaGetLastError();
}

}  // namespace rcscm
