// vc_noalloc.cu -- one FP32 Bellman sweep of the implicit model that allocates nothing.
//
// Some callers cannot call cudaMalloc: code whose device memory is entirely reserved by
// another allocator (a framework's caching pool), code that must not risk the implicit
// device synchronisation an allocation can cause (latency-bound control loops), and code
// that runs while another library captures the stream.  For them this file keeps the
// sweep's scratch -- the post-decision value array U, a residual word and a control block
// whose error word the bounds-checking build reports through -- in file-scope __device__
// arrays of fixed size, loaded with the library on every GPU that loads it and held until
// the process exits.  The caller still passes V and V_out.
#include <math.h>

#include <mutex>

#include "vc_internal.cuh"

namespace vc {

constexpr int kNoAllocMaxStates = 1 << 20;  // 1,048,576 states: 4 MiB of float scratch

static __device__ __align__(256) float g_noalloc_U[kNoAllocMaxStates];
static __device__ __align__(256) unsigned int g_noalloc_res[64];
static __device__ __align__(256) Ctl g_noalloc_ctl;

// Device addresses of the static arrays and the SM count, looked up once per device by the
// first call there.  A later call makes no CUDA call but launches, an asynchronous memset and
// error queries, so it may run while the stream is being captured.  In host code the array
// names are host-side stand-ins, never device addresses: only these pointers are passed to
// kernels.
struct NoAllocScratch {
    bool ready = false;
    float* U = nullptr;
    unsigned int* res = nullptr;
    Ctl* ctl = nullptr;
    int num_sms = 0;
};

constexpr int kMaxDevices = 64;
static NoAllocScratch g_scratch[kMaxDevices];
static std::mutex g_scratch_mu;

static int noalloc_scratch(NoAllocScratch* out) {
    int dev = 0;
    VC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(VC_ERR_ARG, "device ordinal beyond the static scratch table");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    NoAllocScratch& s = g_scratch[dev];
    if (!s.ready) {
        void* p = nullptr;
        VC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_U));
        s.U = (float*)p;
        VC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_res));
        s.res = (unsigned int*)p;
        VC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_ctl));
        s.ctl = (Ctl*)p;
        VC_CUDA(cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev));
        s.ready = true;
    }
    *out = s;
    return VC_OK;
}

// max |V_out - V| over all states into *cell (non-negative float bits, order independent).
// A NaN difference counts as +infinity: fmaxf would drop it, and a sweep that produced a
// NaN must not report a finite residual.
__global__ void __launch_bounds__(kThreads) k_noalloc_residual(const float* __restrict__ V,
                                                               const float* __restrict__ V_out, int S,
                                                               unsigned int* cell) {
    float r = 0.0f;
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < S; s += gridDim.x * kThreads) {
        const float d = fabsf(V_out[s] - V[s]);
        r = (d != d) ? INFINITY : fmaxf(r, d);
    }
    r = block_max<float, kThreads>(r);
    if (threadIdx.x == 0) atomicMax(cell, __float_as_uint(r));
}

__global__ void k_noalloc_copy_residual(const unsigned int* cell, float* out) {
    *out = __uint_as_float(*cell);
}

}  // namespace vc

using namespace vc;

extern "C" int vc_bellman32_noalloc(const vc_params* p, const float* V, float* V_out, int32_t* pi, float* residual,
                                    void* stream) {
    set_error("");
    if (!V || !V_out) return fail(VC_ERR_ARG, "V / V_out is NULL");
    if (V == V_out) return fail(VC_ERR_ARG, "V and V_out must be different buffers");
    Mdp m;  // host-side descriptor only; owns no device memory here
    m.fmt = VC_IMPLICIT;
    int rc = build_model(p, &m);
    if (rc) return rc;
    if (m.S > kNoAllocMaxStates)
        return fail(VC_ERR_ARG, "S = " + std::to_string(m.S) + " exceeds the static scratch of " +
                                    std::to_string(kNoAllocMaxStates) + " states");
    NoAllocScratch sc;
    if ((rc = noalloc_scratch(&sc))) return rc;
    m.num_sms = sc.num_sms;
    m.U32 = sc.U;
    cudaStream_t st = (cudaStream_t)stream;
#ifdef VC_DEBUG_BOUNDS
    // bounds-checking build: the sweep raises its flags in the static control block, which
    // is cleared here and read back after the sweep (this build synchronises the stream)
    VC_CUDA(cudaMemsetAsync(&sc.ctl->error, 0, sizeof(int), st));
    SweepCtl none{sc.ctl, kModeNone, 0, nullptr};
#else
    SweepCtl none{nullptr, kModeNone, 0, nullptr};
#endif
    if ((rc = launch_sweep32(&m, V, V_out, pi, nullptr, none, st))) return rc;
    if (residual) {
        VC_CUDA(cudaMemsetAsync(sc.res, 0, sizeof(unsigned int), st));
        count_launches(2);
        k_noalloc_residual<<<state_grid(&m), kThreads, 0, st>>>(V, V_out, m.S, sc.res);
        k_noalloc_copy_residual<<<1, 1, 0, st>>>(sc.res, residual);
        VC_CUDA(cudaGetLastError());
    }
#ifdef VC_DEBUG_BOUNDS
    int err = 0;
    VC_CUDA(cudaMemcpyAsync(&err, &sc.ctl->error, sizeof(int), cudaMemcpyDeviceToHost, st));
    VC_CUDA(cudaStreamSynchronize(st));
    if (err & kErrBounds) return fail(VC_ERR_CUDA, "a device bounds check failed (bounds-checking build)");
#endif
    return VC_OK;
}
