// rcscm_solve_noalloc: a solve of one utterance that performs no device-memory
// allocation, for callers that cannot call cudaMalloc -- for example a
// real-time audio thread, where an allocation can synchronise the device and
// stall for an unbounded time, or a host application that gives each library a
// fixed GPU memory budget up front.  The paper has no counterpart; this is a
// deployment variant of the accelerated solve.
//
// All working memory the solve needs beyond the caller's inputs and outputs
// (row tables, per-frequency constants, per-slot invariants, status word)
// lives in one file-scope device array of kNoAllocScratchBytes.  Every GPU that
// loads this library's module reserves that array for the life of the process;
// with lazy module loading (the CUDA default) that happens at the first call on
// the device.  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress (with
// that device current; it loads the module if needed) and caches it; make that
// first call before any stream capture.
// Every call on a device shares the one array and leaves its contents behind;
// the parts that must start at zero are cleared by each call.  Calls whose work
// overlaps on the GPU (for example on two streams of the same device) race on
// the array and corrupt each other's results.
#include <float.h>

#include <mutex>

#include "rcscm_internal.cuh"

namespace rcscm {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_addr_mu;
void* g_addr[kNoAllocMaxDevices] = {};

int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RCSCM_ECUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return RCSCM_EINVAL;
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        // With lazy module loading the first lookup on a device also loads the module,
        // which places the array in device memory: running out of memory there is ENOMEM.
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return RCSCM_ENOMEM;
        }
        if (e != cudaSuccess || !p) return RCSCM_ECUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return RCSCM_OK;
}

// Bump allocator over the fixed array: only computes offsets.
struct Carve {
    size_t off = 0;
    template <class T>
    size_t take(size_t n) {
        off = (off + 255) & ~size_t(255);
        const size_t at = off;
        off += n * sizeof(T);
        return at;
    }
};

// Row tables of one utterance, written on the device (no host staging).
__global__ void fill_tables_kernel(DevState d, int I, int J, int M, int nbpr, const float2* x, const double2* a,
                                   const double2* Rp, const double* lambda0, const float* rh0, const float* ru0) {
    const int n = I * nbpr > I ? I * nbpr : I;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        if (t < I) {
            RowDesc rd;
            rd.slot_off = (int64_t)t * J;
            rd.out_off = (int64_t)t * J * M;
            rd.scratch_off = 0;
            rd.x = x + (int64_t)t * J * M;
            rd.a = a + (int64_t)t * M;
            rd.Rp = Rp + (int64_t)t * M * M;
            rd.Rp_c64 = nullptr;
            rd.b_in = nullptr;
            rd.lambda0 = lambda0 ? lambda0 + t : nullptr;
            rd.rh0 = rh0 + (int64_t)t * J;
            rd.ru0 = ru0 + (int64_t)t * J;
            rd.J = J;
            rd.M = M;
            rd.prob = 0;
            rd.freq = t;
            d.rows[t] = rd;
            d.order[t] = t;
        }
        if (t < I * nbpr) d.bmap[t] = BlockMap{t / nbpr, (t % nbpr) * kSlotBlock};
        if (t == 0) d.status[0] = 0;
    }
}

}  // namespace
}  // namespace rcscm

using namespace rcscm;

extern "C" int rcscm_solve_noalloc(int64_t I, int64_t J, int64_t M, const void* x, const void* a, const void* Rp,
                                   const double* lambda0, const float* rh0, const float* ru0,
                                   const rcscm_options* opt, int n_iter, float* rh, float* ru, float* lambda,
                                   void* h_out, int* status, void* stream) {
    if (!x || !a || !Rp || !rh0 || !ru0 || !opt || !rh || !ru || !lambda || !h_out || n_iter < 0)
        return RCSCM_EINVAL;
    if (opt->rule != RCSCM_RULE_ACCEL || opt->iters_per_launch < 0 || !(opt->alpha > -2.0) || !(opt->beta >= 0.0))
        return RCSCM_EINVAL;
    if (opt->persistent != 0 || opt->ckpt_stride != 0) return RCSCM_EINVAL;   // not offered here
    if (!accel_block_ok(opt->block)) return RCSCM_EINVAL;
    if (I < 1 || J < 1 || M < 2 || M > kMaxM) return RCSCM_EINVAL;
    if (J > accel_max_j(opt->block)) return RCSCM_EINVAL;

    // Layout of the fixed array for this call; reject what does not fit.
    if (I > (int64_t)kNoAllocScratchBytes || J > (int64_t)kNoAllocScratchBytes) return RCSCM_ECAPACITY;
    const size_t R = (size_t)I, S = (size_t)(I * J), nbpr = (size_t)((J + kSlotBlock - 1) / kSlotBlock);
    Carve cv;
    const size_t o_rows = cv.take<RowDesc>(R), o_rc = cv.take<RowConst>(R), o_bmap = cv.take<BlockMap>(R * nbpr);
    const size_t o_order = cv.take<int>(R), o_b64 = cv.take<double2>(R * kMaxM), o_mu = cv.take<double>(R * kMaxM);
    const size_t o_lam0 = cv.take<double>(R), o_taa = cv.take<double>(R), o_sab = cv.take<double2>(R);
    const size_t o_phi = cv.take<float2>(R * 64), o_a32 = cv.take<float2>(R * kMaxM);
    const size_t o_b32 = cv.take<float2>(R * kMaxM), o_rp32 = cv.take<float2>(R * 64);
    const size_t o_inv4 = cv.take<float4>(S), o_kap = cv.take<float>(S), o_status = cv.take<int>(1);
    if (cv.off > kNoAllocScratchBytes || R * nbpr > (size_t)INT32_MAX) return RCSCM_ECAPACITY;

    // Every caller address must be one this device can reach (the check allocates
    // nothing); a pageable host buffer or another device's memory is refused here
    // rather than faulting in a kernel.
    const void* in[6] = {x, a, Rp, rh0, ru0, lambda0};
    void* outp[5] = {rh, ru, lambda, h_out, status};
    const void* vin[6] = {};
    const void* vout[5] = {};
    for (int k = 0; k < 6; ++k)
        if ((in[k] || k < 5) && caller_view(in[k], &vin[k])) return RCSCM_EINVAL;
    for (int k = 0; k < 5; ++k)
        if ((outp[k] || k < 4) && caller_view(outp[k], &vout[k])) return RCSCM_EINVAL;
    x = vin[0];
    a = vin[1];
    Rp = vin[2];
    rh0 = static_cast<const float*>(vin[3]);
    ru0 = static_cast<const float*>(vin[4]);
    lambda0 = static_cast<const double*>(vin[5]);
    rh = static_cast<float*>(const_cast<void*>(vout[0]));
    ru = static_cast<float*>(const_cast<void*>(vout[1]));
    lambda = static_cast<float*>(const_cast<void*>(vout[2]));
    h_out = const_cast<void*>(vout[3]);
    status = static_cast<int*>(const_cast<void*>(vout[4]));

    void* base = nullptr;
    int st = scratch_address(&base);
    if (st) return st;
    unsigned char* b = static_cast<unsigned char*>(base);
    DevState d{};
    d.rows = reinterpret_cast<RowDesc*>(b + o_rows);
    d.n_rows = I;
    d.n_slots = I * J;
    d.rc = reinterpret_cast<RowConst*>(b + o_rc);
    d.bmap = reinterpret_cast<BlockMap*>(b + o_bmap);
    d.order = reinterpret_cast<int*>(b + o_order);
    d.b64 = reinterpret_cast<double2*>(b + o_b64);
    d.mu = reinterpret_cast<double*>(b + o_mu);
    d.lam0 = reinterpret_cast<double*>(b + o_lam0);
    d.taa64 = reinterpret_cast<double*>(b + o_taa);
    d.sab64 = reinterpret_cast<double2*>(b + o_sab);
    d.phi = reinterpret_cast<float2*>(b + o_phi);
    d.a32 = reinterpret_cast<float2*>(b + o_a32);
    d.b32 = reinterpret_cast<float2*>(b + o_b32);
    d.rp32 = reinterpret_cast<float2*>(b + o_rp32);
    d.inv4 = reinterpret_cast<float4*>(b + o_inv4);
    d.kap = reinterpret_cast<float*>(b + o_kap);
    d.status = reinterpret_cast<int*>(b + o_status);
    d.rh = rh;          // the caller's outputs hold the EM state
    d.ru = ru;
    d.lam = lambda;
    d.ru_hat = nullptr;

    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    const int nt = (int)(R * nbpr > R ? R * nbpr : R);
    fill_tables_kernel<<<(nt + 255) / 256, 256, 0, cs>>>(d, (int)I, (int)J, (int)M, (int)nbpr,
                                                         static_cast<const float2*>(x), static_cast<const double2*>(a),
                                                         static_cast<const double2*>(Rp), lambda0, rh0, ru0);
    cudaError_t e = cudaGetLastError();
    IterParams p;
    p.c_a2 = (float)(1.0 / (opt->alpha + 2.0));
    p.c_b = (float)(opt->beta / (opt->alpha + 2.0));
    p.ru_floor = opt->ru_floor;
    p.c_a2_f64 = 1.0 / (opt->alpha + 2.0);
    p.c_b_f64 = opt->beta / (opt->alpha + 2.0);
    p.ckpt_first = 0;
    if (e == cudaSuccess) e = launch_setup(d, (int)R, (int)M, opt->null_tol, cs);
    if (e == cudaSuccess) e = launch_invariants(d, (int)(R * nbpr), cs);
    const int chunk = opt->iters_per_launch > 0 ? opt->iters_per_launch : (n_iter > 0 ? n_iter : 1);
    for (int done = 0; e == cudaSuccess && done < n_iter; done += chunk) {
        const int k = n_iter - done < chunk ? n_iter - done : chunk;
        e = launch_accel(d, (int)R, (int)J, opt->block, k, p, false, cs);
    }
    if (e == cudaSuccess) e = launch_extract(d, (int)(R * nbpr), static_cast<float2*>(h_out), cs);
    if (e == cudaSuccess && status) e = cudaMemcpyAsync(status, d.status, sizeof(int), cudaMemcpyDeviceToDevice, cs);
    if (e == cudaErrorMemoryAllocation) return RCSCM_ENOMEM;
    return e == cudaSuccess ? RCSCM_OK : RCSCM_ECUDA;
}
