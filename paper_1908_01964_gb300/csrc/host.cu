// Host-memory pipeline for one utterance shape (declarations in include/rcscm.h).
//
// Accelerated rule (fused configuration): one context over all rows.  The
// per-frequency setup needs only a and R' (small), so they are copied first and
// rcscm_setup_freq runs once for every row while x, r_h0 and r_u0 are still in
// flight; the rows are split into contiguous chunks, each with its own stream:
// copy the chunk's x, r_h0, r_u0, wait for the setup, run the fused kernel on
// the chunk's rows, copy its h back.  Copies of one chunk overlap the kernels of
// another, and the setup's latency is paid once.
// Other rules and configurations: the same copies, then rcscm_solve on one
// stream (no overlap).
// Device buffers, the context, the streams and the event are created once per plan.
#include <algorithm>
#include <new>
#include <vector>

#include "rcscm_internal.cuh"

struct rcscm_host {
    int64_t I = 0, J = 0, M = 0;
    int n_chunks = 0;
    std::vector<int64_t> i0;                   // first row of each chunk (n_chunks + 1 entries)
    rcscm_ctx* ctx = nullptr;
    std::vector<cudaStream_t> streams;         // streams[0] also carries the setup
    cudaEvent_t setup_done = nullptr;
    std::vector<void*> allocs;
    float2* x = nullptr;
    double2* a = nullptr;
    double2* Rp = nullptr;
    float* rh0 = nullptr;
    float* ru0 = nullptr;
    float2* h = nullptr;
    int* hstatus = nullptr;                    // page-locked status word
};

namespace {

template <class T>
cudaError_t halloc(rcscm_host* p, T** q, size_t n) {
    void* v = nullptr;
    const cudaError_t e = cudaMalloc(&v, (n ? n : 1) * sizeof(T));
    if (e == cudaSuccess) {
        p->allocs.push_back(v);
        *q = static_cast<T*>(v);
    }
    return e;
}

void release(rcscm_host* p) {
    if (p->hstatus) cudaFreeHost(p->hstatus);
    if (p->ctx) rcscm_destroy(p->ctx);
    if (p->setup_done) cudaEventDestroy(p->setup_done);
    for (cudaStream_t s : p->streams) cudaStreamDestroy(s);
    for (void* v : p->allocs) cudaFree(v);
    delete p;
}

int code_of(cudaError_t e) {
    if (e == cudaSuccess) return RCSCM_OK;
    if (e == cudaErrorMemoryAllocation) return RCSCM_ENOMEM;
    return RCSCM_ECUDA;
}

}  // namespace

extern "C" int rcscm_host_create(rcscm_host** out, int64_t I, int64_t J, int64_t M, const rcscm_options* opt,
                                 int n_chunks) {
    if (!out || !opt) return RCSCM_EINVAL;
    *out = nullptr;
    if (I < 1 || J < 1 || M < 2 || M > rcscm::kMaxM || n_chunks < 1) return RCSCM_EINVAL;
    rcscm_host* p = new (std::nothrow) rcscm_host();
    if (!p) return RCSCM_ENOMEM;
    p->I = I;
    p->J = J;
    p->M = M;
    p->n_chunks = (int)std::min<int64_t>(n_chunks, I);
    const size_t nx = (size_t)(I * J * M), ns = (size_t)(I * J);
    cudaError_t e = halloc(p, &p->x, nx);
    if (e == cudaSuccess) e = halloc(p, &p->a, (size_t)(I * M));
    if (e == cudaSuccess) e = halloc(p, &p->Rp, (size_t)(I * M * M));
    if (e == cudaSuccess) e = halloc(p, &p->rh0, ns);
    if (e == cudaSuccess) e = halloc(p, &p->ru0, ns);
    if (e == cudaSuccess) e = halloc(p, &p->h, nx);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&p->hstatus), sizeof(int), 0);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->setup_done, cudaEventDisableTiming);
    for (int c = 0; c < p->n_chunks && e == cudaSuccess; ++c) {
        cudaStream_t s = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) p->streams.push_back(s);
    }
    if (e != cudaSuccess) {
        release(p);
        return code_of(e);
    }
    for (int c = 0; c <= p->n_chunks; ++c) p->i0.push_back(I * c / p->n_chunks);
    rcscm_problem q;
    q.I = I;
    q.J = J;
    q.M = M;
    q.x = p->x;
    q.a = p->a;
    q.Rp = p->Rp;
    q.lambda0 = nullptr;
    q.rh0 = p->rh0;
    q.ru0 = p->ru0;
    const int st = rcscm_create(&p->ctx, &q, 1, opt, p->streams[0]);
    if (st) {
        release(p);
        return st;
    }
    *out = p;
    return RCSCM_OK;
}

extern "C" int rcscm_host_run(rcscm_host* p, const void* x, const void* a, const void* Rp, const double* lambda0,
                              const float* rh0, const float* ru0, int n_iter, void* h_out, float* rh, float* ru,
                              float* lambda) {
    if (!p || !x || !a || !Rp || !rh0 || !ru0 || !h_out || n_iter < 0) return RCSCM_EINVAL;
    if (lambda0) return RCSCM_EINVAL;   // the plan's context takes lambda_i from R' (Sec. II-B-3)
    const int64_t I = p->I, J = p->J, M = p->M;
    const bool fused = rcscm::ctx_fused(p->ctx);
    float *d_rh = nullptr, *d_ru = nullptr, *d_lam = nullptr;
    rcscm::ctx_state(p->ctx, &d_rh, &d_ru, &d_lam);
    cudaStream_t s0 = p->streams[0];
    int st = RCSCM_OK;
    cudaError_t e = cudaMemcpyAsync(p->a, a, (size_t)(I * M) * 16, cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->Rp, Rp, (size_t)(I * M * M) * 16, cudaMemcpyHostToDevice, s0);
    if (e == cudaSuccess && fused) {
        st = rcscm_setup_freq(p->ctx, s0);
        if (!st) e = cudaEventRecord(p->setup_done, s0);
    }
    const int n_chunks = fused ? p->n_chunks : 1;
    for (int c = 0; c < n_chunks && e == cudaSuccess && !st; ++c) {
        cudaStream_t s = p->streams[(size_t)c];
        const int64_t r0 = fused ? p->i0[(size_t)c] : 0, r1 = fused ? p->i0[(size_t)c + 1] : I, nI = r1 - r0;
        const size_t bx = (size_t)(nI * J * M) * sizeof(float2), bs = (size_t)(nI * J) * sizeof(float);
        e = cudaMemcpyAsync(p->x + r0 * J * M, static_cast<const float2*>(x) + r0 * J * M, bx,
                            cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p->rh0 + r0 * J, rh0 + r0 * J, bs, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p->ru0 + r0 * J, ru0 + r0 * J, bs, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        if (fused) {
            e = cudaStreamWaitEvent(s, p->setup_done, 0);
            // the kernel writes row r at its offset r * J * M within the whole output
            if (e == cudaSuccess) st = rcscm::run_rows(p->ctx, (int)r0, (int)nI, n_iter, p->h, s);
        } else {
            st = rcscm_solve(p->ctx, n_iter, p->h, s);
        }
        if (st || e != cudaSuccess) break;
        // this chunk's rows only (one utterance: row r starts at slot r * J)
        e = cudaMemcpyAsync(static_cast<float2*>(h_out) + r0 * J * M, p->h + r0 * J * M, bx, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && rh) e = cudaMemcpyAsync(rh + r0 * J, d_rh + r0 * J, bs, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && ru) e = cudaMemcpyAsync(ru + r0 * J, d_ru + r0 * J, bs, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && lambda)
            e = cudaMemcpyAsync(lambda + r0, d_lam + r0, (size_t)nI * sizeof(float), cudaMemcpyDeviceToHost, s);
    }
    // always drain every stream before returning (the host buffers are in use)
    for (cudaStream_t s : p->streams) {
        const cudaError_t e2 = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = e2;
    }
    if (st) return st;
    if (e != cudaSuccess) return code_of(e);
    int* sw = rcscm::ctx_status_word(p->ctx);       // read and clear the status word
    e = cudaMemcpyAsync(p->hstatus, sw, sizeof(int), cudaMemcpyDeviceToHost, s0);
    if (e == cudaSuccess) e = cudaMemsetAsync(sw, 0, sizeof(int), s0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s0);
    if (e != cudaSuccess) return code_of(e);
    const int flags = *p->hstatus;
    if (flags & rcscm::kFlagNullspace) return RCSCM_ENULLSPACE;
    if (flags & rcscm::kFlagNonfinite) return RCSCM_ENONFINITE;
    if (flags & rcscm::kFlagClamp) return RCSCM_ECLAMP;
    return RCSCM_OK;
}

extern "C" void rcscm_host_destroy(rcscm_host* p) {
    if (!p) return;
    for (cudaStream_t s : p->streams) cudaStreamSynchronize(s);
    release(p);
}
