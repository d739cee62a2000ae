// Host-memory pipeline for one utterance shape (declarations in include/rcscm.h):
// the frequency rows are split into chunks, each with its own context and
// stream, so that the host-to-device copy of one chunk, the kernels of another
// and the device-to-host copy of a third overlap (rows are independent in
// every rule).  Device buffers and contexts are created once per plan.
#include <algorithm>
#include <new>
#include <vector>

#include "rcscm_internal.cuh"

struct rcscm_host {
    int64_t I = 0, J = 0, M = 0;
    int n_chunks = 0;
    std::vector<int64_t> i0;                   // first row of each chunk (n_chunks + 1 entries)
    std::vector<rcscm_ctx*> ctx;
    std::vector<cudaStream_t> streams;
    std::vector<void*> allocs;
    float2* x = nullptr;
    double2* a = nullptr;
    double2* Rp = nullptr;
    double* lam0 = nullptr;
    float* rh0 = nullptr;
    float* ru0 = nullptr;
    float2* h = nullptr;
    float* rh = nullptr;
    float* ru = nullptr;
    float* lam = nullptr;
    int* hstatus = nullptr;                    // page-locked, one status word per chunk
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
    for (rcscm_ctx* c : p->ctx) rcscm_destroy(c);
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
    if (e == cudaSuccess) e = halloc(p, &p->lam0, (size_t)I);
    if (e == cudaSuccess) e = halloc(p, &p->rh0, ns);
    if (e == cudaSuccess) e = halloc(p, &p->ru0, ns);
    if (e == cudaSuccess) e = halloc(p, &p->h, nx);
    if (e == cudaSuccess) e = halloc(p, &p->rh, ns);
    if (e == cudaSuccess) e = halloc(p, &p->ru, ns);
    if (e == cudaSuccess) e = halloc(p, &p->lam, (size_t)I);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&p->hstatus), sizeof(int) * p->n_chunks, 0);
    if (e != cudaSuccess) {
        release(p);
        return code_of(e);
    }
    for (int c = 0; c <= p->n_chunks; ++c) p->i0.push_back(I * c / p->n_chunks);
    for (int c = 0; c < p->n_chunks; ++c) {
        cudaStream_t s = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            release(p);
            return code_of(e);
        }
        p->streams.push_back(s);
        const int64_t r0 = p->i0[(size_t)c], nI = p->i0[(size_t)c + 1] - r0;
        rcscm_problem q;
        q.I = nI;
        q.J = J;
        q.M = M;
        q.x = p->x + r0 * J * M;
        q.a = p->a + r0 * M;
        q.Rp = p->Rp + r0 * M * M;
        q.lambda0 = nullptr;
        q.rh0 = p->rh0 + r0 * J;
        q.ru0 = p->ru0 + r0 * J;
        rcscm_ctx* ctx = nullptr;
        const int st = rcscm_create(&ctx, &q, 1, opt, s);
        if (st) {
            release(p);
            return st;
        }
        p->ctx.push_back(ctx);
    }
    *out = p;
    return RCSCM_OK;
}

extern "C" int rcscm_host_run(rcscm_host* p, const void* x, const void* a, const void* Rp, const double* lambda0,
                              const float* rh0, const float* ru0, int n_iter, void* h_out, float* rh, float* ru,
                              float* lambda) {
    if (!p || !x || !a || !Rp || !rh0 || !ru0 || !h_out || n_iter < 0) return RCSCM_EINVAL;
    if (lambda0) return RCSCM_EINVAL;   // the plan's contexts take lambda_i from R' (Sec. II-B-3)
    const int64_t J = p->J, M = p->M;
    int st = RCSCM_OK;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < p->n_chunks && e == cudaSuccess && !st; ++c) {
        cudaStream_t s = p->streams[(size_t)c];
        const int64_t r0 = p->i0[(size_t)c], nI = p->i0[(size_t)c + 1] - r0;
        const size_t bx = (size_t)(nI * J * M) * sizeof(float2), bs = (size_t)(nI * J) * sizeof(float);
        e = cudaMemcpyAsync(p->x + r0 * J * M, static_cast<const float2*>(x) + r0 * J * M, bx,
                            cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->a + r0 * M, static_cast<const double2*>(a) + r0 * M, (size_t)(nI * M) * 16,
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->Rp + r0 * M * M, static_cast<const double2*>(Rp) + r0 * M * M,
                                (size_t)(nI * M * M) * 16, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p->rh0 + r0 * J, rh0 + r0 * J, bs, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p->ru0 + r0 * J, ru0 + r0 * J, bs, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        rcscm_ctx* ctx = p->ctx[(size_t)c];
        st = rcscm_solve(ctx, n_iter, p->h + r0 * J * M, s);
        if (!st && (rh || ru || lambda))
            st = rcscm_get_state(ctx, 0, p->rh + r0 * J, p->ru + r0 * J, p->lam + r0, s);
        if (st) break;
        e = cudaMemcpyAsync(static_cast<float2*>(h_out) + r0 * J * M, p->h + r0 * J * M, bx, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && rh) e = cudaMemcpyAsync(rh + r0 * J, p->rh + r0 * J, bs, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && ru) e = cudaMemcpyAsync(ru + r0 * J, p->ru + r0 * J, bs, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && lambda)
            e = cudaMemcpyAsync(lambda + r0, p->lam + r0, (size_t)nI * sizeof(float), cudaMemcpyDeviceToHost, s);
        int* sw = rcscm::ctx_status_word(ctx);       // read and clear the status word, asynchronously
        if (e == cudaSuccess) e = cudaMemcpyAsync(p->hstatus + c, sw, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(sw, 0, sizeof(int), s);
    }
    // always drain every stream before returning (the host buffers are in use)
    for (cudaStream_t s : p->streams) {
        const cudaError_t e2 = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = e2;
    }
    if (st) return st;
    if (e != cudaSuccess) return code_of(e);
    int flags = 0;
    for (int c = 0; c < p->n_chunks; ++c) flags |= p->hstatus[c];
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
