// Per-frequency setup (FP64) and per-slot invariants (FP32) of the
// rank-constrained SCM estimator, sm_103a.
//
// setup_kernel   one group of 8 lanes per row (utterance, frequency i):
//   R' <- (R' + R'^H)/2, cyclic complex Jacobi eigendecomposition,
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
// invariants_kernel  one thread per slot: z = Phi_i x_ij, and initial state.
#include <float.h>

#include "rcscm_internal.cuh"

namespace rcscm {
namespace {

constexpr int kSetupWarps = 4;
constexpr int kGroupLanes = 8;                            // lanes per row (M <= 8)
constexpr int kSetupRows = kSetupWarps * 32 / kGroupLanes; // rows per block
constexpr int kJacobiMaxSweeps = 30;

// One row per group of 8 lanes (4 rows per warp); lane k of a group owns index
// k of its row.  Control flow that contains __syncwarp is uniform over the warp;
// groups with less work (smaller M, converged, or past the last row) apply no
// rotation in a step.
__global__ void __launch_bounds__(kSetupWarps * 32)
setup_kernel(DevState d, int n_rows, double null_tol) {
    __shared__ double2 sA[kSetupRows][kMaxM][kMaxM];
    __shared__ double2 sV[kSetupRows][kMaxM][kMaxM];
    __shared__ double2 sa[kSetupRows][kMaxM];
    __shared__ double2 sc[kSetupRows][kMaxM];
    __shared__ int sperm[kSetupRows][kMaxM];

    const int g = threadIdx.x / kGroupLanes;
    const int k = threadIdx.x % kGroupLanes;
    const int r = blockIdx.x * kSetupRows + g;
    const bool active = r < n_rows;
    RowDesc rd;
    if (active) rd = d.rows[r];
    const int M = active ? rd.M : 0;
    double2(*A)[kMaxM] = sA[g];
    double2(*V)[kMaxM] = sV[g];

    for (int e = k; e < M * M; e += kGroupLanes) {
        const int m = e / M, n = e % M;
        const double2 amn = rd.Rp[m * M + n];
        const double2 anm = rd.Rp[n * M + m];
        const double2 h = make_double2(0.5 * (amn.x + anm.x), 0.5 * (amn.y - anm.y));
        A[m][n] = h;
        V[m][n] = make_double2(m == n ? 1.0 : 0.0, 0.0);
        d.rp32[(size_t)r * 64 + m * M + n] = make_float2((float)h.x, (float)h.y);
    }
    if (k < M) {
        const double2 av = rd.a[k];
        sa[g][k] = av;
        d.a32[(size_t)r * kMaxM + k] = make_float2((float)av.x, (float)av.y);
    }
    __syncwarp();
    const int Mw = __reduce_max_sync(0xffffffffu, M);

    double fro2 = 0.0;
    for (int m = 0; m < M; ++m)
        for (int n = 0; n < M; ++n) fro2 += zabs2(A[m][n]);

    // ---- cyclic Jacobi: the rotation in the (p, q) plane zeroes A[p][q] ------
    for (int sweep = 0; sweep < kJacobiMaxSweeps; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < M; ++p)
            for (int q = p + 1; q < M; ++q) off += zabs2(A[p][q]);
        const bool conv = !(off > 1e-32 * fro2);
        if (__all_sync(0xffffffffu, conv)) break;
        for (int p = 0; p < Mw - 1; ++p) {
            for (int q = p + 1; q < Mw; ++q) {
                double c = 1.0, s = 0.0;
                double2 e = make_double2(1.0, 0.0);
                bool rot = false;
                if (!conv && q < M) {
                    const double2 apq = A[p][q];
                    const double m2 = zabs2(apq);
                    const double app = A[p][p].x, aqq = A[q][q].x;
                    if (m2 > 0.0 && m2 > 1e-36 * fabs(app * aqq)) {
                        const double inv_mag = rsqrt(m2);
                        const double zeta = 0.5 * (aqq - app) * inv_mag;
                        const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
                        c = rsqrt(fma(t, t, 1.0));
                        s = t * c;
                        e = make_double2(apq.x * inv_mag, apq.y * inv_mag);   // exp(i phi)
                        rot = true;
                    }
                }
                __syncwarp();
                // A <- A U, V <- V U with U = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] on (p, q)
                if (rot && k < M) {
                    const double2 akp = A[k][p];
                    const double2 eq = zmulc(e, A[k][q]);
                    A[k][p] = zsub(zscale(akp, c), zscale(eq, s));
                    A[k][q] = zadd(zscale(akp, s), zscale(eq, c));
                    const double2 vkp = V[k][p];
                    const double2 veq = zmulc(e, V[k][q]);
                    V[k][p] = zsub(zscale(vkp, c), zscale(veq, s));
                    V[k][q] = zadd(zscale(vkp, s), zscale(veq, c));
                }
                __syncwarp();
                // A <- U^H A: rows p, q
                if (rot && k < M) {
                    const double2 apk = A[p][k];
                    const double2 eaq = zmul(e, A[q][k]);
                    A[p][k] = zsub(zscale(apk, c), zscale(eaq, s));
                    A[q][k] = zadd(zscale(apk, s), zscale(eaq, c));
                }
                __syncwarp();
                if (rot && k == 0) {
                    A[p][q] = make_double2(0.0, 0.0);
                    A[q][p] = make_double2(0.0, 0.0);
                    A[p][p].y = 0.0;
                    A[q][q].y = 0.0;
                }
                __syncwarp();
            }
        }
    }

    // ---- ascending order of the eigenvalues --------------------------------
    if (active && k == 0) {
        int perm[kMaxM];
        for (int i = 0; i < M; ++i) perm[i] = i;
        for (int i = 0; i < M; ++i) {
            int best = i;
            for (int l = i + 1; l < M; ++l)
                if (A[perm[l]][perm[l]].x < A[perm[best]][perm[best]].x) best = l;
            const int tmp = perm[i];
            perm[i] = perm[best];
            perm[best] = tmp;
        }
        for (int i = 0; i < M; ++i) sperm[g][i] = perm[i];
    }
    __syncwarp();
    if (!active) return;          // no warp-level synchronisation follows
    const int* perm = sperm[g];
    const double mu1 = A[perm[0]][perm[0]].x;
    const double mu2 = A[perm[1]][perm[1]].x;
    const double muM = A[perm[M - 1]][perm[M - 1]].x;
    if (k < M) d.mu[(size_t)r * kMaxM + k] = A[perm[k]][perm[k]].x;

    const int k0 = perm[0];
    if (k < M) {
        const double2 bv = V[k][k0];
        d.b64[(size_t)r * kMaxM + k] = bv;
        d.b32[(size_t)r * kMaxM + k] = make_float2((float)bv.x, (float)bv.y);
    }
    // c_i = e_i^H a for the nonzero eigenpairs (sorted index i = 1..M-1)
    if (k >= 1 && k < M) {
        const int kk = perm[k];
        double2 acc = make_double2(0.0, 0.0);
        for (int m = 0; m < M; ++m) acc = zadd(acc, zmulc(V[m][kk], sa[g][m]));
        sc[g][k] = acc;
    }
    __syncwarp(0xffu << (threadIdx.x & 24));   // this group's lanes only

    double taa = 0.0;
    for (int i = 1; i < M; ++i) taa += zabs2(sc[g][i]) / A[perm[i]][perm[i]].x;
    double2 sab = make_double2(0.0, 0.0);
    for (int m = 0; m < M; ++m) sab = zadd(sab, zmulc(sa[g][m], V[m][k0]));

    const bool bad = !(mu2 > 0.0) || !(fabs(mu1) <= null_tol * muM) || !(taa > 0.0);
    if (k == 0 && bad) atomicOr(d.status, kFlagNullspace);
    const double lam0 = rd.lambda0 ? rd.lambda0[0] : mu2;

    // Householder vector for u = v / |v|, v_i = c_{i+1} / sqrt(mu_{i+1}), i = 0..M-2
    const double nv = sqrt(taa);
    const double inv_nv = nv > 0.0 ? 1.0 / nv : 0.0;
    const double2 v0 = zscale(sc[g][1], rsqrt(A[perm[1]][perm[1]].x));
    const double2 u0 = zscale(v0, inv_nv);
    const double au0 = sqrt(zabs2(u0));
    const double2 ph0 = au0 > 0.0 ? zscale(u0, 1.0 / au0) : make_double2(1.0, 0.0);
    // w = u - alpha e_0 with alpha = -ph0 |u| -> w_0 = ph0 (|u_0| + 1); |w|^2 = 2 + 2|u_0|
    const double two_over_wn2 = 2.0 / (2.0 + 2.0 * au0);

    if (k < M) {
        const int n = k;
        float2* phi = d.phi + (size_t)r * 64;
        // row 0: conj(g_n), g = R'^+ a = sum_i e_i c_i / mu_i
        double2 gv = make_double2(0.0, 0.0);
        double2 qn = make_double2(0.0, 0.0);    // q_n = sum_l conj(w_l) conj(e_{l+1}[n]) / sqrt(mu_{l+1})
        for (int i = 1; i < M; ++i) {
            const double mui = A[perm[i]][perm[i]].x;
            const double rs = rsqrt(mui);
            const double2 ein = V[n][perm[i]];
            gv = zadd(gv, zscale(zmul(ein, sc[g][i]), rs * rs));
            const double2 vl = zscale(sc[g][i], inv_nv * rs);                          // u_{i-1}
            const double2 wl = (i == 1) ? zscale(ph0, au0 + 1.0) : vl;                 // w_{i-1}
            qn = zadd(qn, zscale(zconj(zmul(wl, ein)), rs));
        }
        phi[0 * M + n] = make_float2((float)gv.x, (float)-gv.y);
        for (int kk = 1; kk <= M - 2; ++kk) {
            const double rs = rsqrt(A[perm[kk + 1]][perm[kk + 1]].x);
            const double2 ekn = V[n][perm[kk + 1]];
            const double2 wk = zscale(sc[g][kk + 1], inv_nv * rs);                    // w_kk = u_kk
            double2 val = zscale(zconj(ekn), rs);
            val = zsub(val, zscale(zmul(wk, qn), two_over_wn2));
            phi[kk * M + n] = make_float2((float)val.x, (float)val.y);
        }
        const double2 bn = V[n][k0];
        phi[(M - 1) * M + n] = make_float2((float)bn.x, (float)-bn.y);
    }
    if (k == 0) {
        d.lam0[r] = lam0;
        d.taa64[r] = taa;
        d.sab64[r] = sab;
        RowConst c;
        const double tsafe = taa > 0.0 ? taa : 1.0;
        c.taa = (float)taa;
        c.taaM = (float)(taa / M);
        c.inv_taa = (float)(1.0 / tsafe);
        c.sab2 = (float)zabs2(sab);
        c.sab_re = (float)sab.x;
        c.sab_im = (float)sab.y;
        c.invM = (float)(1.0 / M);
        c.pad = 0.f;
        d.rc[r] = c;
        d.lam[r] = (float)lam0;
    }
}

template <int M>
__device__ __forceinline__ void project_slot(const float2* __restrict__ phi, const float2* __restrict__ xs,
                                             float4& out, float& kappa) {
    float2 xv[M];
#pragma unroll
    for (int n = 0; n < M; ++n) xv[n] = xs[n];
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

__global__ void __launch_bounds__(kSlotBlock) invariants_kernel(DevState d) {
    __shared__ float2 sphi[kMaxM * kMaxM];
    const BlockMap bm = d.bmap[blockIdx.x];
    const RowDesc* rd = d.rows + bm.row;
    const int M = rd->M;
    const int J = rd->J;
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) sphi[e] = d.phi[(size_t)bm.row * 64 + e];
    __syncthreads();
    const int j = bm.j0 + threadIdx.x;
    if (j >= J) return;
    const float2* xs = rd->x + (size_t)j * M;
    float4 o;
    float kap;
    switch (M) {
        case 2: project_slot<2>(sphi, xs, o, kap); break;
        case 3: project_slot<3>(sphi, xs, o, kap); break;
        case 4: project_slot<4>(sphi, xs, o, kap); break;
        case 5: project_slot<5>(sphi, xs, o, kap); break;
        case 6: project_slot<6>(sphi, xs, o, kap); break;
        case 7: project_slot<7>(sphi, xs, o, kap); break;
        default: project_slot<8>(sphi, xs, o, kap); break;
    }
    const int64_t s = rd->slot_off + j;
    d.inv4[s] = o;
    d.kap[s] = kap;
    d.rh[s] = rd->rh0[j];
    d.ru[s] = rd->ru0[j];
}

}  // namespace

cudaError_t launch_setup(const DevState& d, int n_rows, double null_tol, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    const int grid = (n_rows + kSetupRows - 1) / kSetupRows;
    setup_kernel<<<grid, kSetupWarps * 32, 0, s>>>(d, n_rows, null_tol);
    return cudaGetLastError();
}

cudaError_t launch_invariants(const DevState& d, int n_blocks, cudaStream_t s) {
    if (n_blocks <= 0) return cudaSuccess;
    invariants_kernel<<<n_blocks, kSlotBlock, 0, s>>>(d);
    return cudaGetLastError();
}

}  // namespace rcscm
