// C ABI of the rank-constrained SCM library (declarations and contracts in
// include/rcscm.h).  Host code: validation, context memory, row tables and
// kernel launches.  Every numerical step runs in the CUDA kernels of setup.cu,
// iterate.cu and extract.cu.
#include <float.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "ilrma.cuh"
#include "rcscm_internal.cuh"

using namespace rcscm;

struct rcscm_ctx {
    rcscm_options opt;
    std::vector<rcscm_problem> probs;
    std::vector<int64_t> row0, slot0, out0;   // per utterance: first row, slot, output element
    int64_t R = 0, S = 0;
    int n_blocks = 0;
    int max_j = 0;
    int max_m = 0;
    DevState d;
    int* naive_rows = nullptr;
    int count_by_m[kMaxM + 1];
    int first_by_m[kMaxM + 1];
    std::vector<void*> allocs;
    int64_t bytes = 0;
    int* first_block = nullptr;      // [n_probs + 1] first slot block of each utterance
    double* obj_out = nullptr;       // [n_probs] objective per utterance (device)
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    // checkpoints for rcscm_backward (ckpt_stride > 0)
    int n_ckpt = 0;
    float* ckpt_rh = nullptr;        // [n_ckpt][S]
    float* ckpt_ru = nullptr;        // [n_ckpt][S]
    float* ckpt_lam = nullptr;       // [n_ckpt][R]
    float* seg_rh = nullptr;         // adjoint scratch: [stride][S], [stride][S], [stride][R]
    float* seg_ru = nullptr;
    float* seg_lam = nullptr;
    double* adj_sums = nullptr;      // [R][kAdjSums] row sums handed to the setup adjoint
    int* ident = nullptr;            // rows 0..R-1 in order (row ranges of the fused kernel)
    int iters_done = 0;              // passes since the last setup / set_state
    int iter_block = 0;              // block of those passes (-1: mixed)
};

namespace {

int map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return RCSCM_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return RCSCM_ENOMEM;
    }
    return RCSCM_ECUDA;
}

template <class T>
int dalloc(rcscm_ctx* c, T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    void* q = nullptr;
    const cudaError_t e = cudaMalloc(&q, n * sizeof(T));
    if (e != cudaSuccess) return map_cuda(e);
    c->allocs.push_back(q);
    c->bytes += (int64_t)(n * sizeof(T));
    *p = static_cast<T*>(q);
    return RCSCM_OK;
}

void free_all(rcscm_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    c->gexec = nullptr;
    c->graph = nullptr;
    c->cap_stream = nullptr;
    for (void* q : c->allocs) cudaFree(q);
    c->allocs.clear();
}

int valid_options(const rcscm_options* o) {
    if (o->rule != RCSCM_RULE_ACCEL && o->rule != RCSCM_RULE_NAIVE && o->rule != RCSCM_RULE_NAIVE_F64 &&
        o->rule != RCSCM_RULE_ACCEL1 && o->rule != RCSCM_RULE_NAIVE_PRINTED)
        return 0;
    if (!(o->alpha > -2.0) || !(o->beta >= 0.0)) return 0;
    if (!(o->null_tol > 0.0) || !(o->ru_floor >= 0.0f)) return 0;
    if (!accel_block_ok(o->block)) return 0;
    if (o->iters_per_launch < 0) return 0;
    if (o->persistent != 0 && o->persistent != 1) return 0;
    if (o->ckpt_stride < 0) return 0;
    if (o->ckpt_stride > 0) {
        if (o->rule != RCSCM_RULE_ACCEL || o->ckpt_max_iters < 1) return 0;
        if (o->block != 0 && o->block != 128 && o->block != 256) return 0;
    }
    return 1;
}

IterParams iter_params(const rcscm_options& o) {
    IterParams p;
    p.c_a2 = (float)(1.0 / (o.alpha + 2.0));
    p.c_b = (float)(o.beta / (o.alpha + 2.0));
    p.ru_floor = o.ru_floor;
    p.c_a2_f64 = 1.0 / (o.alpha + 2.0);
    p.c_b_f64 = o.beta / (o.alpha + 2.0);
    p.ckpt_first = 0;
    return p;
}

// The address under which the current device reaches caller memory `p`: device or
// managed memory of this device as is; page-locked host memory through its device
// view (with the coherent host link of this platform kernels read and write it
// directly).  Anything else -- pageable host memory, another device's memory, an
// invalid address -- is refused (nothing is launched on it).
template <class T>
int device_view(T* p, T** out) {
    *out = nullptr;
    if (!p) return RCSCM_EINVAL;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, (const void*)p) != cudaSuccess) {
        cudaGetLastError();
        return RCSCM_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RCSCM_ECUDA;
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
        if (at.type == cudaMemoryTypeDevice && at.device != dev) return RCSCM_EINVAL;
        *out = p;
        return RCSCM_OK;
    }
    if (at.type == cudaMemoryTypeHost && at.devicePointer) {
        *out = static_cast<T*>(at.devicePointer);
        return RCSCM_OK;
    }
    return RCSCM_EINVAL;
}

}  // namespace

int rcscm::caller_view(const void* p, const void** out) { return device_view(p, out); }

int* rcscm::ctx_status_word(rcscm_ctx* c) { return c ? c->d.status : nullptr; }

static bool fused_config(const rcscm_options& o) {
    return o.rule == RCSCM_RULE_ACCEL && o.iters_per_launch == 0 && o.ckpt_stride == 0;
}

bool rcscm::ctx_fused(const rcscm_ctx* c) { return c && fused_config(c->opt); }

void rcscm::ctx_state(rcscm_ctx* c, float** rh, float** ru, float** lam) {
    *rh = c->d.rh;
    *ru = c->d.ru;
    *lam = c->d.lam;
}

int rcscm::run_rows(rcscm_ctx* c, int first_row, int n_rows, int n_iter, float2* h, cudaStream_t s) {
    if (!c || !fused_config(c->opt) || first_row < 0 || n_rows < 0 || first_row + (int64_t)n_rows > c->R)
        return RCSCM_EINVAL;
    DevState d = c->d;                       // the same kernel over a contiguous range of rows
    d.order = c->ident + first_row;
    // one CTA per row: ranges may run concurrently on several streams, and the
    // persistent form's row counter is per context
    return map_cuda(launch_accel(d, n_rows, c->max_j, c->opt.block, n_iter, iter_params(c->opt), false, s, h));
}

extern "C" {

void rcscm_default_options(rcscm_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->rule = RCSCM_RULE_ACCEL;
    opt->alpha = 1.1;
    opt->beta = 1e-16;
    opt->ru_floor = FLT_MIN;
    opt->null_tol = 1e-6;
    opt->block = 0;
    opt->iters_per_launch = 0;
    opt->persistent = 0;
    opt->ckpt_stride = 0;
    opt->ckpt_max_iters = 0;
}

const char* rcscm_strerror(int code) {
    switch (code) {
        case RCSCM_OK: return "success";
        case RCSCM_EINVAL: return "invalid argument (shape, pointer, option or call order)";
        case RCSCM_ENULLSPACE: return "R' is not rank M-1 within the null-space tolerance (or a lies in its null space)";
        case RCSCM_ENONFINITE: return "non-finite or non-positive lambda produced";
        case RCSCM_ECLAMP: return "warning: a variance was held at its floor (r_u at ru_floor, or a negative FP32 naive-rule r_h estimate)";
        case RCSCM_ECUDA: return "CUDA runtime error";
        case RCSCM_ENOMEM: return "device memory allocation failed";
        case RCSCM_ETIMEOUT: return "bounded device wait gave up";
        case RCSCM_ECAPACITY: return "problem too large for the fixed scratch array of rcscm_solve_noalloc";
        case RCSCM_EBOUNDS: return "an index check of the debug build failed";
        default: return "unknown rcscm status code";
    }
}

int rcscm_create(rcscm_ctx** out, const rcscm_problem* probs, int n_probs, const rcscm_options* opt,
                 void* stream) {
    if (!out) return RCSCM_EINVAL;
    *out = nullptr;
    if (!probs || n_probs < 1 || !opt || !valid_options(opt)) return RCSCM_EINVAL;
    int64_t R = 0, S = 0, n_blocks = 0, naive_scratch = 0;
    int max_m = 0;
    int max_j = 0;
    for (int p = 0; p < n_probs; ++p) {
        const rcscm_problem& q = probs[p];
        if (q.I < 1 || q.J < 1 || q.M < 2 || q.M > kMaxM) return RCSCM_EINVAL;
        if (!q.x || !q.a || !q.Rp || !q.rh0 || !q.ru0) return RCSCM_EINVAL;
        if (q.rp_c64 != 0 && q.rp_c64 != 1) return RCSCM_EINVAL;
        const void* v;
        const double* vd;
        const float* vf;
        if (device_view(q.x, &v) || device_view(q.a, &v) || device_view(q.Rp, &v) || device_view(q.rh0, &vf) ||
            device_view(q.ru0, &vf) || (q.lambda0 && device_view(q.lambda0, &vd)) || (q.b && device_view(q.b, &v)))
            return RCSCM_EINVAL;
        if (q.J > INT32_MAX / 2) return RCSCM_EINVAL;
        if (opt->rule == RCSCM_RULE_ACCEL && q.J > accel_max_j(opt->block)) return RCSCM_EINVAL;
        if (opt->rule == RCSCM_RULE_ACCEL1 && accel1_block((int)q.J) == 0) return RCSCM_EINVAL;
        R += q.I;
        S += q.I * q.J;
        n_blocks += q.I * ((q.J + kSlotBlock - 1) / kSlotBlock);
        naive_scratch += q.I * q.J * q.M * q.M;
        max_j = std::max<int>(max_j, (int)q.J);
        max_m = std::max<int>(max_m, (int)q.M);
    }
    if (R > INT32_MAX || n_blocks > INT32_MAX) return RCSCM_EINVAL;
    rcscm_options eff = *opt;
    if (eff.ckpt_stride > 0) {               // the adjoint kernel's shapes: 128 x 4 or 256 x 8 slots
        if (eff.block == 0) eff.block = adjoint_block(max_j);
        if (eff.block == 0 || max_j > 8 * eff.block || (eff.block == 128 && max_j > 512)) return RCSCM_EINVAL;
    }

    rcscm_ctx* c = new (std::nothrow) rcscm_ctx();
    if (!c) return RCSCM_ENOMEM;
    c->opt = eff;
    c->probs.assign(probs, probs + n_probs);
    c->R = R;
    c->S = S;
    c->n_blocks = (int)n_blocks;
    c->max_j = max_j;
    c->max_m = max_m;

    // ---- host row tables ----------------------------------------------------
    std::vector<RowDesc> rows((size_t)R);
    std::vector<BlockMap> bmap((size_t)n_blocks);
    std::vector<int> jrow((size_t)R), mrow((size_t)R);
    int64_t r = 0, s = 0, o = 0, sc = 0, b = 0, ao = 0, po = 0;
    for (int p = 0; p < n_probs; ++p) {
        const rcscm_problem& q = probs[p];
        rcscm_problem qv = q;                  // the device views of the caller's buffers (checked above)
        device_view(q.x, &qv.x);
        device_view(q.a, &qv.a);
        device_view(q.Rp, &qv.Rp);
        device_view(q.rh0, &qv.rh0);
        device_view(q.ru0, &qv.ru0);
        if (q.lambda0) device_view(q.lambda0, &qv.lambda0);
        if (q.b) device_view(q.b, &qv.b);
        c->row0.push_back(r);
        c->slot0.push_back(s);
        c->out0.push_back(o);
        for (int64_t i = 0; i < q.I; ++i, ++r) {
            RowDesc& rd = rows[(size_t)r];
            rd.slot_off = s;
            rd.out_off = o;
            rd.scratch_off = sc;
            rd.a_off = ao;
            rd.rp_off = po;
            rd.x = static_cast<const float2*>(qv.x) + i * q.J * q.M;
            rd.a = static_cast<const double2*>(qv.a) + i * q.M;
            rd.Rp = q.rp_c64 ? nullptr : static_cast<const double2*>(qv.Rp) + i * q.M * q.M;
            rd.Rp_c64 = q.rp_c64 ? static_cast<const float2*>(qv.Rp) + i * q.M * q.M : nullptr;
            rd.b_in = qv.b ? static_cast<const double2*>(qv.b) + i * q.M : nullptr;
            rd.lambda0 = qv.lambda0 ? qv.lambda0 + i : nullptr;
            rd.rh0 = qv.rh0 + i * q.J;
            rd.ru0 = qv.ru0 + i * q.J;
            rd.J = (int)q.J;
            rd.M = (int)q.M;
            rd.prob = p;
            rd.freq = (int)i;
            jrow[(size_t)r] = (int)q.J;
            mrow[(size_t)r] = (int)q.M;
            for (int j0 = 0; j0 < q.J; j0 += kSlotBlock) bmap[(size_t)b++] = BlockMap{(int)r, j0};
            s += q.J;
            o += q.J * q.M;
            sc += q.J * q.M * q.M;
            ao += q.M;
            po += q.M * q.M;
        }
    }
    std::vector<int> first_block;
    {
        int64_t fb = 0;
        for (int p = 0; p < n_probs; ++p) {
            first_block.push_back((int)fb);
            fb += probs[p].I * ((probs[p].J + kSlotBlock - 1) / kSlotBlock);
        }
        first_block.push_back((int)fb);
    }
    std::vector<int> order((size_t)R);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return jrow[(size_t)x] > jrow[(size_t)y]; });
    std::vector<int> naive_rows;
    naive_rows.reserve((size_t)R);
    for (int M = 0; M <= kMaxM; ++M) {
        c->first_by_m[M] = (int)naive_rows.size();
        for (int64_t k = 0; k < R; ++k)
            if (mrow[(size_t)order[(size_t)k]] == M) naive_rows.push_back(order[(size_t)k]);
        c->count_by_m[M] = (int)naive_rows.size() - c->first_by_m[M];
    }

    // ---- device memory -------------------------------------------------------
    DevState& d = c->d;
    int st = RCSCM_OK;
    const size_t Rz = (size_t)R, Sz = (size_t)S;
    d.n_slots = S;
    d.n_rows = R;
    if (!st) st = dalloc(c, &d.rows, Rz);
    if (!st) st = dalloc(c, &d.rc, Rz);
    if (!st) st = dalloc(c, &d.bmap, (size_t)n_blocks);
    if (!st) st = dalloc(c, &d.order, Rz);
    if (!st) st = dalloc(c, &d.b64, Rz * kMaxM);
    if (!st) st = dalloc(c, &d.mu, Rz * kMaxM);
    if (!st) st = dalloc(c, &d.lam0, Rz);
    if (!st) st = dalloc(c, &d.taa64, Rz);
    if (!st) st = dalloc(c, &d.sab64, Rz);
    if (!st) st = dalloc(c, &d.phi, Rz * 64);
    if (!st) st = dalloc(c, &d.a32, Rz * kMaxM);
    if (!st) st = dalloc(c, &d.b32, Rz * kMaxM);
    // the naive rules' per-row inputs (the setup forms them only where they are allocated)
    const bool printed = opt->rule == RCSCM_RULE_NAIVE_F64 || opt->rule == RCSCM_RULE_NAIVE_PRINTED;
    if (!st && printed) st = dalloc(c, &d.rp32, Rz * 64);
    if (!st && opt->rule == RCSCM_RULE_NAIVE) st = dalloc(c, &d.wht32, Rz * 64);
    if (!st && opt->rule == RCSCM_RULE_NAIVE) st = dalloc(c, &d.aw64, Rz * kMaxM);
    if (!st) st = dalloc(c, &d.inv4, Sz);
    if (!st) st = dalloc(c, &d.kap, Sz);
    if (!st) st = dalloc(c, &d.rh, Sz);
    if (!st) st = dalloc(c, &d.ru, Sz);
    if (!st) st = dalloc(c, &d.lam, Rz);
    if (!st) st = dalloc(c, &d.status, 1);
    if (!st) st = dalloc(c, &c->naive_rows, Rz);
    if (!st) st = dalloc(c, &d.counter, 1);
    if (!st) st = dalloc(c, &d.obj_part, (size_t)n_blocks);
    if (!st) st = dalloc(c, &c->first_block, (size_t)n_probs + 1);
    if (!st) st = dalloc(c, &c->ident, Rz);
    if (!st) st = dalloc(c, &c->obj_out, (size_t)n_probs);
    if (!st) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&d.n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            st = RCSCM_ECUDA;
    }
    if (!st && eff.ckpt_stride > 0) {
        c->n_ckpt = (eff.ckpt_max_iters + eff.ckpt_stride - 1) / eff.ckpt_stride;
        st = dalloc(c, &d.evec64, Rz * 64);
        if (!st) st = dalloc(c, &c->ckpt_rh, Sz * (size_t)c->n_ckpt);
        if (!st) st = dalloc(c, &c->ckpt_ru, Sz * (size_t)c->n_ckpt);
        if (!st) st = dalloc(c, &c->ckpt_lam, Rz * (size_t)c->n_ckpt);
        d.ckpt_rh = c->ckpt_rh;
        d.ckpt_ru = c->ckpt_ru;
        d.ckpt_lam = c->ckpt_lam;
        d.ckpt_stride = eff.ckpt_stride;
        const size_t seg = (size_t)std::min(eff.ckpt_stride, eff.ckpt_max_iters);
        if (!st) st = dalloc(c, &c->seg_rh, Sz * seg);
        if (!st) st = dalloc(c, &c->seg_ru, Sz * seg);
        if (!st) st = dalloc(c, &c->seg_lam, Rz * seg);
        if (!st) st = dalloc(c, &c->adj_sums, Rz * kAdjSums);
    }
    if (!st && opt->rule == RCSCM_RULE_NAIVE) {            // two values per slot
        float* q = nullptr;
        st = dalloc(c, &q, (size_t)naive_scratch);
        d.ru_hat = q;
    } else if (!st && opt->rule == RCSCM_RULE_NAIVE_PRINTED) {
        float* q = nullptr;
        st = dalloc(c, &q, (size_t)naive_scratch);
        d.ru_hat = q;
    } else if (!st && opt->rule == RCSCM_RULE_NAIVE_F64) {
        double* q = nullptr;
        st = dalloc(c, &q, (size_t)naive_scratch);
        d.ru_hat = q;
    }
    if (st) {
        free_all(c);
        delete c;
        return st;
    }
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(d.rows, rows.data(), Rz * sizeof(RowDesc), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.bmap, bmap.data(), (size_t)n_blocks * sizeof(BlockMap), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.order, order.data(), Rz * sizeof(int), cudaMemcpyHostToDevice, cs);
    std::vector<int> ident((size_t)R);
    std::iota(ident.begin(), ident.end(), 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->ident, ident.data(), Rz * sizeof(int), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->naive_rows, naive_rows.data(), Rz * sizeof(int), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->first_block, first_block.data(), first_block.size() * sizeof(int),
                            cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.status, 0, sizeof(int), cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);    // host tables go out of scope
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return map_cuda(e);
    }
    *out = c;
    return RCSCM_OK;
}

int rcscm_setup(rcscm_ctx* c, void* stream) {
    if (!c) return RCSCM_EINVAL;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_setup(c->d, (int)c->R, c->max_m, c->opt.null_tol, cs);
    if (e == cudaSuccess) e = launch_invariants(c->d, c->n_blocks, cs);
    c->iters_done = 0;
    c->iter_block = 0;
    return map_cuda(e);
}

int rcscm_iterate(rcscm_ctx* c, int n_iter, void* stream) {
    if (!c || n_iter < 0) return RCSCM_EINVAL;
    if (n_iter == 0) return RCSCM_OK;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    const IterParams p = iter_params(c->opt);
    const int chunk = c->opt.iters_per_launch > 0 ? c->opt.iters_per_launch : n_iter;
    if (c->opt.ckpt_stride > 0 && n_iter > c->opt.ckpt_max_iters - c->iters_done) return RCSCM_EINVAL;
    for (int done = 0; done < n_iter;) {
        const int k = std::min(chunk, n_iter - done);
        IterParams pk = p;
        pk.ckpt_first = c->iters_done;        // the accelerated kernel writes checkpoints itself
        cudaError_t e;
        if (c->opt.rule == RCSCM_RULE_ACCEL)
            e = launch_accel(c->d, (int)c->R, c->max_j, c->opt.block, k, pk, c->opt.persistent != 0, cs);
        else if (c->opt.rule == RCSCM_RULE_ACCEL1)
            e = launch_accel1(c->d, c->naive_rows, c->count_by_m, c->first_by_m, c->max_j, k, p, cs);
        else
            e = launch_naive(c->d, c->naive_rows, c->count_by_m, c->first_by_m, k, p, c->opt.rule, cs);
        if (e != cudaSuccess) return map_cuda(e);
        const int blk = c->opt.block;
        c->iter_block = (c->iters_done == 0 || c->iter_block == blk) ? blk : -1;
        c->iters_done += k;
        done += k;
    }
    return RCSCM_OK;
}

int rcscm_setup_freq(rcscm_ctx* c, void* stream) {
    if (!c) return RCSCM_EINVAL;
    return map_cuda(launch_setup(c->d, (int)c->R, c->max_m, c->opt.null_tol, static_cast<cudaStream_t>(stream)));
}

int rcscm_run(rcscm_ctx* c, int n_iter, void* h_out, void* stream) {
    void* h = nullptr;
    if (!c || n_iter < 0 || !fused_config(c->opt) || device_view(h_out, &h)) return RCSCM_EINVAL;
    const cudaError_t e = launch_accel(c->d, (int)c->R, c->max_j, c->opt.block, n_iter, iter_params(c->opt),
                                       c->opt.persistent != 0, static_cast<cudaStream_t>(stream),
                                       static_cast<float2*>(h));
    c->iters_done = n_iter;
    c->iter_block = c->opt.block;
    return map_cuda(e);
}

int rcscm_solve(rcscm_ctx* c, int n_iter, void* h_out, void* stream) {
    if (!c || n_iter < 0 || !h_out) return RCSCM_EINVAL;
    if (!fused_config(c->opt)) {             // the same work as separate calls
        int st = rcscm_setup(c, stream);
        if (!st) st = rcscm_iterate(c, n_iter, stream);
        if (!st) st = rcscm_extract(c, h_out, stream);
        return st;
    }
    int st = rcscm_setup_freq(c, stream);
    if (!st) st = rcscm_run(c, n_iter, h_out, stream);
    return st;
}

int rcscm_extract(rcscm_ctx* c, void* h_out, void* stream) {
    void* h = nullptr;
    if (!c || device_view(h_out, &h)) return RCSCM_EINVAL;
    return map_cuda(launch_extract(c->d, c->n_blocks, static_cast<float2*>(h), static_cast<cudaStream_t>(stream)));
}

int rcscm_get_state(rcscm_ctx* c, int p, float* rh, float* ru, float* lambda, void* stream) {
    if (!c || p < 0 || p >= (int)c->probs.size()) return RCSCM_EINVAL;
    const rcscm_problem& q = c->probs[(size_t)p];
    const size_t n = (size_t)(q.I * q.J);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (rh) e = cudaMemcpyAsync(rh, c->d.rh + c->slot0[(size_t)p], n * sizeof(float), cudaMemcpyDeviceToDevice, cs);
    if (ru && e == cudaSuccess) e = cudaMemcpyAsync(ru, c->d.ru + c->slot0[(size_t)p], n * sizeof(float), cudaMemcpyDeviceToDevice, cs);
    if (lambda && e == cudaSuccess)
        e = cudaMemcpyAsync(lambda, c->d.lam + c->row0[(size_t)p], (size_t)q.I * sizeof(float), cudaMemcpyDeviceToDevice, cs);
    return map_cuda(e);
}

int rcscm_set_state(rcscm_ctx* c, int p, const float* rh, const float* ru, const float* lambda, void* stream) {
    if (!c || p < 0 || p >= (int)c->probs.size()) return RCSCM_EINVAL;
    const rcscm_problem& q = c->probs[(size_t)p];
    const size_t n = (size_t)(q.I * q.J);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (rh) e = cudaMemcpyAsync(c->d.rh + c->slot0[(size_t)p], rh, n * sizeof(float), cudaMemcpyDeviceToDevice, cs);
    if (ru && e == cudaSuccess) e = cudaMemcpyAsync(c->d.ru + c->slot0[(size_t)p], ru, n * sizeof(float), cudaMemcpyDeviceToDevice, cs);
    if (lambda && e == cudaSuccess)
        e = cudaMemcpyAsync(c->d.lam + c->row0[(size_t)p], lambda, (size_t)q.I * sizeof(float), cudaMemcpyDeviceToDevice, cs);
    c->iters_done = 0;                       // the set state is the new starting point of the passes
    c->iter_block = 0;
    return map_cuda(e);
}

int rcscm_get_setup(rcscm_ctx* c, int p, void* b, double* lambda0, double* tau_aa, void* sigma_ab,
                    double* mu, void* stream) {
    if (!c || p < 0 || p >= (int)c->probs.size()) return RCSCM_EINVAL;
    const rcscm_problem& q = c->probs[(size_t)p];
    const size_t r0 = (size_t)c->row0[(size_t)p], I = (size_t)q.I, M = (size_t)q.M;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (b) e = cudaMemcpy2DAsync(b, M * sizeof(double2), c->d.b64 + r0 * kMaxM, kMaxM * sizeof(double2),
                                 M * sizeof(double2), I, cudaMemcpyDeviceToDevice, cs);
    if (mu && e == cudaSuccess)
        e = cudaMemcpy2DAsync(mu, M * sizeof(double), c->d.mu + r0 * kMaxM, kMaxM * sizeof(double),
                              M * sizeof(double), I, cudaMemcpyDeviceToDevice, cs);
    if (lambda0 && e == cudaSuccess) e = cudaMemcpyAsync(lambda0, c->d.lam0 + r0, I * sizeof(double), cudaMemcpyDeviceToDevice, cs);
    if (tau_aa && e == cudaSuccess) e = cudaMemcpyAsync(tau_aa, c->d.taa64 + r0, I * sizeof(double), cudaMemcpyDeviceToDevice, cs);
    if (sigma_ab && e == cudaSuccess) e = cudaMemcpyAsync(sigma_ab, c->d.sab64 + r0, I * sizeof(double2), cudaMemcpyDeviceToDevice, cs);
    return map_cuda(e);
}

int rcscm_get_invariants(rcscm_ctx* c, int p, void* tau_ax, void* sigma_bx, float* kappa, void* stream) {
    if (!c || p < 0 || p >= (int)c->probs.size()) return RCSCM_EINVAL;
    const rcscm_problem& q = c->probs[(size_t)p];
    const size_t s0 = (size_t)c->slot0[(size_t)p], n = (size_t)(q.I * q.J);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    const char* base = reinterpret_cast<const char*>(c->d.inv4 + s0);
    if (tau_ax) e = cudaMemcpy2DAsync(tau_ax, sizeof(float2), base, sizeof(float4), sizeof(float2), n, cudaMemcpyDeviceToDevice, cs);
    if (sigma_bx && e == cudaSuccess)
        e = cudaMemcpy2DAsync(sigma_bx, sizeof(float2), base + sizeof(float2), sizeof(float4), sizeof(float2), n,
                              cudaMemcpyDeviceToDevice, cs);
    if (kappa && e == cudaSuccess) e = cudaMemcpyAsync(kappa, c->d.kap + s0, n * sizeof(float), cudaMemcpyDeviceToDevice, cs);
    return map_cuda(e);
}

int rcscm_ilrma_init(const rcscm_ilrma* u, int n_utt, int* status, void* stream) {
    using namespace rcscm;
    if (!u || n_utt < 1) return RCSCM_EINVAL;
    int* st = nullptr;
    if (status && device_view(status, &st)) return RCSCM_EINVAL;
    std::vector<IlrmaArgs> args((size_t)n_utt);
    for (int k = 0; k < n_utt; ++k) {               // validate every utterance before any launch
        const rcscm_ilrma& q = u[k];
        if (q.I < 1 || q.J < 1 || q.I > INT32_MAX || q.J > INT32_MAX || q.M < 2 || q.M > kMaxM || q.K < 1 ||
            q.K > kIlrmaMaxK || q.n_h < 0 || q.n_h >= q.M)
            return RCSCM_EINVAL;
        IlrmaArgs& g = args[(size_t)k];
        g.I = (int)q.I;
        g.J = (int)q.J;
        g.M = (int)q.M;
        g.K = (int)q.K;
        g.n_h = (int)q.n_h;
        const void *x, *W;
        const float *T, *V;
        void *a, *Rp;
        float *rh0, *ru0;
        if (device_view(q.x, &x) || device_view(q.W, &W) || device_view(q.T, &T) || device_view(q.V, &V) ||
            device_view(q.a, &a) || device_view(q.Rp, &Rp) || device_view(q.rh0, &rh0) || device_view(q.ru0, &ru0))
            return RCSCM_EINVAL;
        g.x = static_cast<const float2*>(x);
        g.W = static_cast<const double2*>(W);
        g.T = T;
        g.V = V;
        g.a = static_cast<double2*>(a);
        g.Rp = static_cast<double2*>(Rp);
        g.rh0 = rh0;
        g.ru0 = ru0;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (const IlrmaArgs& g : args) {
        const cudaError_t e = launch_ilrma_init(g, st, s);
        if (e != cudaSuccess) return map_cuda(e);
    }
    return RCSCM_OK;
}

int rcscm_status(rcscm_ctx* c, int* flags, void* stream) {
    if (!c) return RCSCM_EINVAL;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    int h = 0;
    cudaError_t e = cudaStreamSynchronize(cs);
    if (e == cudaSuccess) e = cudaMemcpy(&h, c->d.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(c->d.status, 0, sizeof(int));
    if (e != cudaSuccess) return map_cuda(e);
    if (flags) *flags = h;
    if (h & kFlagBounds) return RCSCM_EBOUNDS;
    if (h & kFlagNullspace) return RCSCM_ENULLSPACE;
    if (h & kFlagNonfinite) return RCSCM_ENONFINITE;
    if (h & kFlagClamp) return RCSCM_ECLAMP;
    return RCSCM_OK;
}

int rcscm_info(const rcscm_ctx* c, int64_t* rows, int64_t* slots, int64_t* device_bytes) {
    if (!c) return RCSCM_EINVAL;
    if (rows) *rows = c->R;
    if (slots) *slots = c->S;
    if (device_bytes) *device_bytes = c->bytes;
    return RCSCM_OK;
}

void rcscm_destroy(rcscm_ctx* c) {
    if (!c) return;
    cudaDeviceSynchronize();
    free_all(c);
    delete c;
}

int rcscm_objective(rcscm_ctx* c, double* value, void* stream) {
    if (!c || !value) return RCSCM_EINVAL;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_objective(c->d, c->n_blocks, iter_params(c->opt), c->opt.alpha, c->opt.beta,
                                     c->first_block, (int)c->probs.size(), c->obj_out, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(value, c->obj_out, c->probs.size() * sizeof(double), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    return map_cuda(e);
}

int rcscm_autotune(rcscm_ctx* c, int n_iter_probe, int* chosen_block, int* chosen_persistent, void* stream) {
    if (!c || n_iter_probe < 1) return RCSCM_EINVAL;
    if (c->opt.rule != RCSCM_RULE_ACCEL) return RCSCM_EINVAL;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    const size_t S = (size_t)c->S, R = (size_t)c->R;
    float *rh = nullptr, *ru = nullptr, *lam = nullptr;
    int* status = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&rh, S * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&ru, S * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&lam, R * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    auto copy_state = [&](bool save) {
        cudaError_t x = cudaMemcpyAsync(save ? rh : c->d.rh, save ? c->d.rh : rh, S * sizeof(float),
                                        cudaMemcpyDeviceToDevice, cs);
        if (x == cudaSuccess)
            x = cudaMemcpyAsync(save ? ru : c->d.ru, save ? c->d.ru : ru, S * sizeof(float), cudaMemcpyDeviceToDevice, cs);
        if (x == cudaSuccess)
            x = cudaMemcpyAsync(save ? lam : c->d.lam, save ? c->d.lam : lam, R * sizeof(float),
                                cudaMemcpyDeviceToDevice, cs);
        if (x == cudaSuccess)
            x = cudaMemcpyAsync(save ? status : c->d.status, save ? c->d.status : status, sizeof(int),
                                cudaMemcpyDeviceToDevice, cs);
        return x;
    };
    if (e == cudaSuccess) e = copy_state(true);
    const IterParams p = iter_params(c->opt);
    DevState dd = c->d;                      // probe passes must not overwrite checkpoints
    dd.ckpt_stride = 0;
    float best = 3.0e38f;
    const bool fixed_block = c->opt.ckpt_stride > 0;   // the adjoint needs the context's block
    int best_block = fixed_block ? c->opt.block : accel_default_block(c->max_j), best_pers = 0;
    const int blocks[] = {32, 64, 128, 256, 512, 1024};
    for (int bi = 0; bi < 6 && e == cudaSuccess; ++bi) {
        const int b = blocks[bi];
        if ((int64_t)b * accel_max_spt(b) < c->max_j) continue;
        if (fixed_block && b != c->opt.block) continue;
        for (int pers = 0; pers <= 1 && e == cudaSuccess; ++pers) {
            float t = 3.0e38f;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                e = copy_state(false);
                if (e == cudaSuccess) e = cudaEventRecord(e0, cs);
                if (e == cudaSuccess) e = launch_accel(dd, (int)c->R, c->max_j, b, n_iter_probe, p, pers != 0, cs);
                if (e == cudaSuccess) e = cudaEventRecord(e1, cs);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e == cudaSuccess && ms < t) t = ms;
            }
            if (e == cudaSuccess && t < best) {
                best = t;
                best_block = b;
                best_pers = pers;
            }
        }
    }
    if (e == cudaSuccess) e = copy_state(false);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e == cudaSuccess) {
        c->opt.block = best_block;
        c->opt.persistent = best_pers;
        if (chosen_block) *chosen_block = best_block;
        if (chosen_persistent) *chosen_persistent = best_pers;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(rh);
    cudaFree(ru);
    cudaFree(lam);
    cudaFree(status);
    return map_cuda(e);
}

int rcscm_graph_create(rcscm_ctx* c, int n_iter, void* h_out) {
    if (!c || n_iter < 0 || !h_out) return RCSCM_EINVAL;
    if (c->opt.ckpt_stride > 0) return RCSCM_EINVAL;   // checkpoint bookkeeping lives on the host
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    cudaError_t e = cudaSuccess;
    if (!c->cap_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return map_cuda(e);
    e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return map_cuda(e);
    int st = rcscm_solve(c, n_iter, h_out, c->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e2 != cudaSuccess) return map_cuda(e2);
    c->graph = g;
    return map_cuda(cudaGraphInstantiate(&c->gexec, g, 0));
}

int rcscm_backward(rcscm_ctx* c, const void* grad_h, void* grad_x, void* grad_a, void* grad_Rp, void* stream) {
    if (!c || !grad_h || !grad_x || !grad_a || !grad_Rp) return RCSCM_EINVAL;
    if (c->opt.ckpt_stride <= 0) return RCSCM_EINVAL;
    if (c->iters_done > 0 && c->iter_block != c->opt.block) return RCSCM_EINVAL;
    AdjointArgs g;
    g.grad_h = static_cast<const float2*>(grad_h);
    g.grad_x = static_cast<float2*>(grad_x);
    g.grad_a = static_cast<double2*>(grad_a);
    g.grad_Rp = static_cast<double2*>(grad_Rp);
    g.ckpt_rh = c->ckpt_rh;
    g.ckpt_ru = c->ckpt_ru;
    g.ckpt_lam = c->ckpt_lam;
    g.seg_rh = c->seg_rh;
    g.seg_ru = c->seg_ru;
    g.seg_lam = c->seg_lam;
    g.sums = c->adj_sums;
    g.K = c->iters_done;
    g.stride = c->opt.ckpt_stride;
    g.S = c->S;
    g.R = c->R;
    return map_cuda(launch_adjoint(c->d, (int)c->R, c->max_j, c->max_m, c->opt.block, g, iter_params(c->opt),
                                   static_cast<cudaStream_t>(stream)));
}

int rcscm_graph_launch(rcscm_ctx* c, void* stream) {
    if (!c || !c->gexec) return RCSCM_EINVAL;
    return map_cuda(cudaGraphLaunch(c->gexec, static_cast<cudaStream_t>(stream)));
}

int rcscm_solve_host(int64_t I, int64_t J, int64_t M, const void* x, const void* a, const void* Rp,
                     const double* lambda0, const float* rh0, const float* ru0, const rcscm_options* opt,
                     int n_iter, void* h_out, float* rh, float* ru, float* lambda) {
    if (!x || !a || !Rp || !rh0 || !ru0 || !h_out || !opt || n_iter < 0) return RCSCM_EINVAL;
    if (I < 1 || J < 1 || M < 2 || M > kMaxM) return RCSCM_EINVAL;
    const size_t nx = (size_t)(I * J * M), ns = (size_t)(I * J), ni = (size_t)I;
    void *dx = nullptr, *da = nullptr, *dR = nullptr, *dh = nullptr;
    double* dl = nullptr;
    float *drh = nullptr, *dru = nullptr;
    int st = RCSCM_OK;
    cudaError_t e = cudaMalloc(&dx, nx * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&da, ni * (size_t)M * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&dR, ni * (size_t)(M * M) * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&dh, nx * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&drh, ns * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dru, ns * sizeof(float));
    if (e == cudaSuccess && lambda0) e = cudaMalloc(&dl, ni * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(dx, x, nx * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(da, a, ni * (size_t)M * sizeof(double2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dR, Rp, ni * (size_t)(M * M) * sizeof(double2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(drh, rh0, ns * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dru, ru0, ns * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && lambda0) e = cudaMemcpy(dl, lambda0, ni * sizeof(double), cudaMemcpyHostToDevice);
    st = map_cuda(e);
    rcscm_ctx* c = nullptr;
    if (!st) {
        rcscm_problem q;
        memset(&q, 0, sizeof(q));
        q.I = I; q.J = J; q.M = M;
        q.x = dx; q.a = da; q.Rp = dR; q.lambda0 = dl; q.rh0 = drh; q.ru0 = dru;
        st = rcscm_create(&c, &q, 1, opt, nullptr);
    }
    if (!st) st = rcscm_solve(c, n_iter, dh, nullptr);
    if (!st) st = map_cuda(cudaMemcpy(h_out, dh, nx * sizeof(float2), cudaMemcpyDeviceToHost));
    if (!st && (rh || ru || lambda)) {
        // reuse the input state buffers as staging for the outputs
        float* dlam = nullptr;
        e = cudaMalloc(&dlam, ni * sizeof(float));
        if (e == cudaSuccess) st = rcscm_get_state(c, 0, drh, dru, dlam, nullptr);
        else st = map_cuda(e);
        if (!st && rh) st = map_cuda(cudaMemcpy(rh, drh, ns * sizeof(float), cudaMemcpyDeviceToHost));
        if (!st && ru) st = map_cuda(cudaMemcpy(ru, dru, ns * sizeof(float), cudaMemcpyDeviceToHost));
        if (!st && lambda) st = map_cuda(cudaMemcpy(lambda, dlam, ni * sizeof(float), cudaMemcpyDeviceToHost));
        if (dlam) cudaFree(dlam);
    }
    if (!st && c) {
        const int s2 = rcscm_status(c, nullptr, nullptr);
        if (s2 == RCSCM_ENULLSPACE || s2 == RCSCM_ENONFINITE) st = s2;
    }
    rcscm_destroy(c);
    cudaFree(dx); cudaFree(da); cudaFree(dR); cudaFree(dh); cudaFree(drh); cudaFree(dru);
    if (dl) cudaFree(dl);
    return st;
}

}  // extern "C"
