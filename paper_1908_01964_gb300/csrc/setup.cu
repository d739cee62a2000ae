// Per-frequency setup (FP64) and per-slot invariants (FP32) of the
// rank-constrained SCM estimator, sm_103a.
//
// setup_kernel   one warp per row (utterance, frequency i):
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
constexpr int kJacobiMaxSweeps = 30;

__global__ void __launch_bounds__(kSetupWarps * 32)
setup_kernel(DevState d, int n_rows, double null_tol) {
    __shared__ double2 sA[kSetupWarps][kMaxM][kMaxM];
    __shared__ double2 sV[kSetupWarps][kMaxM][kMaxM];
    __shared__ double2 sa[kSetupWarps][kMaxM];
    __shared__ double2 sc[kSetupWarps][kMaxM];
    __shared__ int sperm[kSetupWarps][kMaxM];

    const int w = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * kSetupWarps + w;
    if (r >= n_rows) return;            // whole warp leaves; only warp-level syncs below

    const RowDesc rd = d.rows[r];
    const int M = rd.M;
    double2(*A)[kMaxM] = sA[w];
    double2(*V)[kMaxM] = sV[w];

    for (int e = lane; e < M * M; e += 32) {
        const int m = e / M, n = e % M;
        const double2 amn = rd.Rp[m * M + n];
        const double2 anm = rd.Rp[n * M + m];
        const double2 h = make_double2(0.5 * (amn.x + anm.x), 0.5 * (amn.y - anm.y));
        A[m][n] = h;
        V[m][n] = make_double2(m == n ? 1.0 : 0.0, 0.0);
        d.rp32[(size_t)r * 64 + m * M + n] = make_float2((float)h.x, (float)h.y);
    }
    if (lane < M) {
        const double2 av = rd.a[lane];
        sa[w][lane] = av;
        d.a32[(size_t)r * kMaxM + lane] = make_float2((float)av.x, (float)av.y);
    }
    __syncwarp();

    double fro2 = 0.0;
    for (int m = 0; m < M; ++m)
        for (int n = 0; n < M; ++n) fro2 += zabs2(A[m][n]);

    // ---- cyclic Jacobi: rotations in the (p, q) plane zero A[p][q] --------
    for (int sweep = 0; sweep < kJacobiMaxSweeps; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < M; ++p)
            for (int q = p + 1; q < M; ++q) off += zabs2(A[p][q]);
        if (off <= 1e-32 * fro2) break;
        for (int p = 0; p < M - 1; ++p) {
            for (int q = p + 1; q < M; ++q) {
                const double2 apq = A[p][q];
                const double mag = sqrt(zabs2(apq));
                const double app = A[p][p].x, aqq = A[q][q].x;
                if (!(mag > 1e-300) || mag <= 1e-18 * sqrt(fabs(app * aqq))) continue;   // warp-uniform
                const double zeta = (aqq - app) / (2.0 * mag);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t);
                const double s = t * c;
                const double2 e = make_double2(apq.x / mag, apq.y / mag);   // exp(i phi)
                __syncwarp();
                // A <- A U, V <- V U with U = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] on (p, q)
                if (lane < M) {
                    const double2 akp = A[lane][p];
                    const double2 eq = zmulc(e, A[lane][q]);
                    A[lane][p] = zsub(zscale(akp, c), zscale(eq, s));
                    A[lane][q] = zadd(zscale(akp, s), zscale(eq, c));
                    const double2 vkp = V[lane][p];
                    const double2 veq = zmulc(e, V[lane][q]);
                    V[lane][p] = zsub(zscale(vkp, c), zscale(veq, s));
                    V[lane][q] = zadd(zscale(vkp, s), zscale(veq, c));
                }
                __syncwarp();
                // A <- U^H A: rows p, q
                if (lane < M) {
                    const double2 apk = A[p][lane];
                    const double2 eaq = zmul(e, A[q][lane]);
                    A[p][lane] = zsub(zscale(apk, c), zscale(eaq, s));
                    A[q][lane] = zadd(zscale(apk, s), zscale(eaq, c));
                }
                __syncwarp();
                if (lane == 0) {
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
    if (lane == 0) {
        int perm[kMaxM];
        for (int k = 0; k < M; ++k) perm[k] = k;
        for (int k = 0; k < M; ++k) {
            int best = k;
            for (int l = k + 1; l < M; ++l)
                if (A[perm[l]][perm[l]].x < A[perm[best]][perm[best]].x) best = l;
            const int tmp = perm[k];
            perm[k] = perm[best];
            perm[best] = tmp;
        }
        for (int k = 0; k < M; ++k) sperm[w][k] = perm[k];
    }
    __syncwarp();
    const int* perm = sperm[w];
    const double mu1 = A[perm[0]][perm[0]].x;
    const double mu2 = A[perm[1]][perm[1]].x;
    const double muM = A[perm[M - 1]][perm[M - 1]].x;
    if (lane < M) d.mu[(size_t)r * kMaxM + lane] = A[perm[lane]][perm[lane]].x;

    const int k0 = perm[0];
    if (lane < M) {
        const double2 bv = V[lane][k0];
        d.b64[(size_t)r * kMaxM + lane] = bv;
        d.b32[(size_t)r * kMaxM + lane] = make_float2((float)bv.x, (float)bv.y);
    }
    // c_k = e_k^H a for the nonzero eigenpairs (sorted index k = 1..M-1)
    if (lane >= 1 && lane < M) {
        const int kk = perm[lane];
        double2 acc = make_double2(0.0, 0.0);
        for (int m = 0; m < M; ++m) acc = zadd(acc, zmulc(V[m][kk], sa[w][m]));
        sc[w][lane] = acc;
    }
    __syncwarp();

    double taa = 0.0;
    for (int k = 1; k < M; ++k) taa += zabs2(sc[w][k]) / A[perm[k]][perm[k]].x;
    double2 sab = make_double2(0.0, 0.0);
    for (int m = 0; m < M; ++m) sab = zadd(sab, zmulc(sa[w][m], V[m][k0]));

    const bool bad = !(mu2 > 0.0) || !(fabs(mu1) <= null_tol * muM) || !(taa > 0.0);
    if (lane == 0 && bad) atomicOr(d.status, kFlagNullspace);
    const double lam0 = rd.lambda0 ? rd.lambda0[0] : mu2;

    // Householder vector for u = v / |v|, v_k = c_{k+1} / sqrt(mu_{k+1}), k = 0..M-2
    const double nv = sqrt(taa);
    const double inv_nv = nv > 0.0 ? 1.0 / nv : 0.0;
    const double2 v0 = zscale(sc[w][1], 1.0 / sqrt(A[perm[1]][perm[1]].x));
    const double2 u0 = zscale(v0, inv_nv);
    const double au0 = sqrt(zabs2(u0));
    const double2 ph0 = au0 > 0.0 ? zscale(u0, 1.0 / au0) : make_double2(1.0, 0.0);
    // w = u - alpha e_0 with alpha = -ph0 |u| -> w_0 = ph0 (|u_0| + 1); |w|^2 = 2 + 2|u_0|
    const double two_over_wn2 = 2.0 / (2.0 + 2.0 * au0);

    if (lane < M) {
        const int n = lane;
        float2* phi = d.phi + (size_t)r * 64;
        // row 0: conj(g_n), g = R'^+ a = sum_k e_k c_k / mu_k
        double2 g = make_double2(0.0, 0.0);
        double2 qn = make_double2(0.0, 0.0);    // q_n = sum_l conj(w_l) conj(e_{l+1}[n]) / sqrt(mu_{l+1})
        for (int k = 1; k < M; ++k) {
            const double muk = A[perm[k]][perm[k]].x;
            const double2 ekn = V[n][perm[k]];
            g = zadd(g, zscale(zmul(ekn, sc[w][k]), 1.0 / muk));
            const double2 vl = zscale(sc[w][k], inv_nv / sqrt(muk));                   // u_{k-1}
            const double2 wl = (k == 1) ? zscale(ph0, au0 + 1.0) : vl;                  // w_{k-1}
            qn = zadd(qn, zscale(zconj(zmul(wl, ekn)), 1.0 / sqrt(muk)));
        }
        phi[0 * M + n] = make_float2((float)g.x, (float)-g.y);
        for (int kk = 1; kk <= M - 2; ++kk) {
            const double muk = A[perm[kk + 1]][perm[kk + 1]].x;
            const double2 ekn = V[n][perm[kk + 1]];
            const double2 wk = zscale(sc[w][kk + 1], inv_nv / sqrt(muk));              // w_kk = u_kk
            double2 val = zscale(zconj(ekn), 1.0 / sqrt(muk));
            val = zsub(val, zscale(zmul(wk, qn), two_over_wn2));
            phi[kk * M + n] = make_float2((float)val.x, (float)val.y);
        }
        const double2 bn = V[n][k0];
        phi[(M - 1) * M + n] = make_float2((float)bn.x, (float)-bn.y);
    }
    if (lane == 0) {
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
    const int grid = (n_rows + kSetupWarps - 1) / kSetupWarps;
    setup_kernel<<<grid, kSetupWarps * 32, 0, s>>>(d, n_rows, null_tol);
    return cudaGetLastError();
}

cudaError_t launch_invariants(const DevState& d, int n_blocks, cudaStream_t s) {
    if (n_blocks <= 0) return cudaSuccess;
    invariants_kernel<<<n_blocks, kSlotBlock, 0, s>>>(d);
    return cudaGetLastError();
}

}  // namespace rcscm
