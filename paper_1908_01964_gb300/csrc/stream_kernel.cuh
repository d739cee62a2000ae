// Streaming kernel of the accelerated rule (one pass per launch).  Included by
// iterate_impl.cuh inside its namespaces; it uses the pass code of accel_common.cuh.
#pragma once

// Streaming form of a launch that runs exactly one pass: the row's pairs are
// loaded, updated and stored one at a time, with A/M and B of pass A kept in
// shared memory for pass B, so few registers are live (at most 64, so that
// 2048 threads of several rows stream through each SM).  Loading the next
// pair ahead of the current one's arithmetic was measured to make no
// difference.  Same operations in the same order and the same reduction as
// the register-resident form, so the results are bitwise equal.
// One pair of slots as loaded by the streaming kernel.
struct PairIn {
    float4 t0, t1;
    float k0, k1, rh0, rh1, ru0, ru1;
};

template <int BLOCK, int SPT>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) accel_stream_kernel(DevState d, IterParams p) {
    __shared__ __align__(16) float red[2][BLOCK / 32 > 0 ? BLOCK / 32 : 1];
    __shared__ f32x2 s_am[SPT / 2][BLOCK], s_b[SPT / 2][BLOCK];
    const int r = d.order[blockIdx.x];
    RCSCM_CTA_CHECK(row_ok(d, r, BLOCK * SPT), d.status);
    const RowDesc* rd = d.rows + r;
    const int J = rd->J;
    const int64_t off = rd->slot_off;
    const RowConst c = d.rc[r];
    const int tid = threadIdx.x;
    const int np = (J + 2 * BLOCK - 1) / (2 * BLOCK);     // 1..SPT/2 (checked by the host)
    const float lam0 = d.lam[r];
    const bool ckpt = d.ckpt_stride > 0 && p.ckpt_first % d.ckpt_stride == 0;
    const size_t kc = ckpt ? (size_t)(p.ckpt_first / d.ckpt_stride) : 0;
    const PassConsts k = pass_consts(c, p, rcp_refined(lam0));
    // loads of pair q (padding: zero invariants, r_h = 0, r_u = 1, kappa/M = 1)
    auto load_pair = [&](int q) {
        PairIn in;
        const int j0 = 2 * q * BLOCK + tid, j1 = j0 + BLOCK;
        const bool v0 = j0 < J, v1 = j1 < J;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        in.t0 = v0 ? d.inv4[off + j0] : z;
        in.t1 = v1 ? d.inv4[off + j1] : z;
        in.k0 = v0 ? d.kap[off + j0] : 0.f;
        in.k1 = v1 ? d.kap[off + j1] : 0.f;
        in.rh0 = v0 ? d.rh[off + j0] : 0.f;
        in.rh1 = v1 ? d.rh[off + j1] : 0.f;
        in.ru0 = v0 ? d.ru[off + j0] : 1.f;
        in.ru1 = v1 ? d.ru[off + j1] : 1.f;
        return in;
    };
    f32x2 part = dup(0.f);
    PairIn cur = load_pair(0);
    for (int q = 0; q < np; ++q) {
        if (q > 0) cur = load_pair(q);
        const int j0 = 2 * q * BLOCK + tid, j1 = j0 + BLOCK;
        const bool v0 = j0 < J, v1 = j1 < J;
        if (ckpt) {                                      // the state entering this pass
            float* crh = d.ckpt_rh + kc * d.n_slots + off;
            float* cru = d.ckpt_ru + kc * d.n_slots + off;
            if (v0) { crh[j0] = cur.rh0; cru[j0] = cur.ru0; }
            if (v1) { crh[j1] = cur.rh1; cru[j1] = cur.ru1; }
        }
        const float km0 = v0 ? fmaf(cur.k0, c.invM, p.ru_floor) : 1.f;
        const float km1 = v1 ? fmaf(cur.k1, c.invM, p.ru_floor) : 1.f;
        f32x2 rh = pk(cur.rh0, cur.rh1), ru = pk(cur.ru0, cur.ru1), B;
        const f32x2 cb = q == np - 1 ? pk(v0 ? p.c_b : 0.f, v1 ? p.c_b : 0.f) : k.CB;
        pass_a_pair(k, pk(cur.t0.x, cur.t1.x), pk(cur.t0.y, cur.t1.y), pk(cur.t0.z, cur.t1.z),
                    pk(cur.t0.w, cur.t1.w), pk(km0, km1), cb, rh, ru, B, part);
        if (v0) d.rh[off + j0] = lo_of(rh);
        if (v1) d.rh[off + j1] = hi_of(rh);
        s_am[q][tid] = ru;
        s_b[q][tid] = B;
    }
    if (ckpt && tid == 0) d.ckpt_lam[kc * d.n_rows + r] = lam0;
    const float lam = block_sum<BLOCK>(lo_of(part) + hi_of(part), red, 0) * (1.0f / (float)J);
    const f32x2 ILM = dup(rcp_refined(lam) * c.invM);
    bool clamp = false;
    for (int q = 0; q < np; ++q) {
        const f32x2 ru = fma2(s_b[q][tid], ILM, s_am[q][tid]);
        const int j0 = 2 * q * BLOCK + tid, j1 = j0 + BLOCK;
        if (j0 < J) {
            d.ru[off + j0] = lo_of(ru);
            clamp |= lo_of(ru) <= p.ru_floor;
        }
        if (j1 < J) {
            d.ru[off + j1] = hi_of(ru);
            clamp |= hi_of(ru) <= p.ru_floor;
        }
    }
    if (clamp) atomicOr(d.status, kFlagClamp);
    if (tid == 0) {
        d.lam[r] = lam;
        if (!(lam > 0.f) || !(lam <= FLT_MAX)) atomicOr(d.status, kFlagNonfinite);
    }
}

