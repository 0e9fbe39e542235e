// vc_api.cu -- the extern "C" entry points declared in include/vcmdp.h: handle
// construction, the value-iteration driver (Algorithm 3: FP32 Jacobi sweeps until the
// residual test of step 3, argmax policy of step 4) and the FP64 refinement and
// certification that follow it.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "vc_internal.cuh"
#include "vc_krylov.cuh"

namespace vc {

static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_err = msg; }

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? VC_ERR_OOM : VC_ERR_CUDA;
}

static void free_mdp(Mdp* m) {
    if (!m) return;
    void* ptrs[] = {m->row_ptr, m->col, m->val, m->scale, m->R, m->val64, m->R64, m->rate_tab, m->work,
                    m->sell_rec, m->sell_slab};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (m->work_host) cudaFreeHost(m->work_host);
    delete m;
}

// The handle's work buffers, one device allocation carved into 256-byte-aligned parts (a
// cudaMalloc per buffer costs tens of microseconds each), and the pinned mirrors of the two
// control blocks, one pinned allocation.
static int alloc_work(Mdp* m) {
    const size_t S = (size_t)m->S;
    const bool implicit = (m->fmt & 0xF) == VC_IMPLICIT;
    struct Part {
        void** p;
        size_t bytes;
    };
    const Part parts[] = {
        {(void**)&m->Vb, 4 * S},
        {(void**)&m->U32, implicit ? 4 * S : 0},
        {(void**)&m->U32s, implicit ? 4 * S : 0},
        {(void**)&m->U64, m->has_model ? 8 * S : 0},
        {(void**)&m->V64a, 8 * S},
        {(void**)&m->V64b, 8 * S},
        {(void**)&m->E0, 4 * S},
        {(void**)&m->E1, 4 * S},
        {(void**)&m->Rres, 4 * S},
        {(void**)&m->pi, 4 * S},
        {(void**)&m->pi2, 4 * S},
        {(void**)&m->kr, 20 * S},
        {(void**)&m->kr_part, 24 * (size_t)state_grid(m)},
        {(void**)&m->kctl, sizeof(KrylovCtl)},
        {(void**)&m->ctl, sizeof(Ctl)},
    };
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t total = 0;
    for (const Part& q : parts) total += up(q.bytes);
    int rc;
    if ((rc = alloc_dev(m, &m->work, total))) return rc;
    size_t off = 0;
    for (const Part& q : parts) {
        *q.p = q.bytes ? static_cast<void*>(static_cast<unsigned char*>(m->work) + off) : nullptr;
        off += up(q.bytes);
    }
    const size_t kbytes = up(sizeof(KrylovCtl));
    VC_CUDA(cudaMallocHost(&m->work_host, kbytes + sizeof(Ctl)));
    m->kctl_host = static_cast<KrylovCtl*>(m->work_host);
    m->ctl_host = reinterpret_cast<Ctl*>(static_cast<unsigned char*>(m->work_host) + kbytes);
    memset(m->ctl_host, 0, sizeof(Ctl));
    VC_CUDA(cudaMemset(m->ctl, 0, sizeof(Ctl)));
    return VC_OK;
}

namespace {
std::mutex g_cache_mu;
std::map<std::pair<int, const void*>, cudaFuncAttributes> g_attr_cache;
std::map<std::pair<int, const void*>, int> g_smem_cache;
std::map<std::tuple<int, const void*, int, size_t>, int> g_occ_cache;

int current_device() {
    int dev = 0;
    cudaGetDevice(&dev);
    return dev;
}
}  // namespace

cudaError_t cached_func_attributes(const void* fn, cudaFuncAttributes* fa) {
    const auto key = std::make_pair(current_device(), fn);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_attr_cache.find(key);
    if (it != g_attr_cache.end()) {
        *fa = it->second;
        return cudaSuccess;
    }
    const cudaError_t e = cudaFuncGetAttributes(fa, fn);
    if (e == cudaSuccess) g_attr_cache[key] = *fa;
    return e;
}

cudaError_t cached_set_max_dyn_smem(const void* fn, int bytes) {
    const auto key = std::make_pair(current_device(), fn);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_smem_cache.find(key);
    if (it != g_smem_cache.end() && it->second == bytes) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) {
        g_smem_cache[key] = bytes;
        // occupancy answers depend on the attribute: drop this kernel's cached ones
        for (auto o = g_occ_cache.begin(); o != g_occ_cache.end();)
            o = (std::get<0>(o->first) == key.first && std::get<1>(o->first) == fn) ? g_occ_cache.erase(o)
                                                                                      : std::next(o);
    }
    return e;
}

cudaError_t cached_occupancy(const void* fn, int threads, size_t smem, int* per_sm) {
    const auto key = std::make_tuple(current_device(), fn, threads, smem);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_occ_cache.find(key);
    if (it != g_occ_cache.end()) {
        *per_sm = it->second;
        return cudaSuccess;
    }
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, threads, smem);
    if (e == cudaSuccess) g_occ_cache[key] = *per_sm;
    return e;
}

static int device_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
    return n;
}

// ------------------------------------------------------------------ loop drivers
static void reset_ctl(Ctl& h, double tol, long long max_sweeps, long long spin_polls) {
    memset(&h, 0, sizeof(Ctl));
    h.tol = tol;
    h.max_sweeps = max_sweeps;
    h.best_res = INFINITY;
    h.spin_limit = spin_polls < 0 ? 0 : spin_polls + 1;
}

static int read_ctl(Mdp* m, cudaStream_t st) {
    VC_CUDA(cudaMemcpyAsync(m->ctl_host, m->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    VC_CUDA(cudaStreamSynchronize(st));
    return VC_OK;
}

// Sweeps still needed for a residual r to fall below tol at contraction rate gamma.
static long long predict_sweeps(double r, double tol, double gamma) {
    if (!(r > tol)) return 1;
    const double n = ceil(log(tol / r) / log(gamma));
    if (!(n < 1e6)) return 1000000;
    return (long long)n + 1;
}

// An FP32 fixed-point loop with device-side termination (value iteration, or the
// correction solve of the refinement).  Sweeps are enqueued in chunks sized from the
// observed residual; once the device flags termination the rest of a chunk returns
// immediately, so the sweep count is exactly the first sweep meeting the test.  On
// return buf[*final_idx] holds the iterate.
template <typename Launch>
static int loop32(Mdp* m, float* buf0, float* buf1, double tol, long long max_sweeps, cudaStream_t st,
                  int* final_idx, Launch&& launch) {
    Ctl& h = *m->ctl_host;
    reset_ctl(h, tol, max_sweeps, m->spin_polls);
    VC_CUDA(cudaMemcpyAsync(m->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    float* buf[2] = {buf0, buf1};
    long long launched = 0, chunk = 16;
    int rc;
    for (;;) {
        for (long long i = 0; i < chunk; i++) {
            const int in = (int)(launched & 1);
            SweepCtl sc{m->ctl, kModeLoop32, 1 - in, nullptr};
            if ((rc = launch(buf[in], buf[1 - in], sc))) return rc;
            launched++;
        }
        if ((rc = read_ctl(m, st))) return rc;
        if (h.error & kErrTimeout) return fail(VC_ERR_TIMEOUT, "a bounded device-side wait expired");
        if (h.error & kErrBounds) return fail(VC_ERR_CUDA, "a device bounds check failed (bounds-checking build)");
        if (h.error) return fail(VC_ERR_ARG, "a kernel flagged invalid input (infeasible policy)");
        if (h.done) break;
        const int slot = (int)((h.sweeps - 1) % kRing);
        float r, vm;
        memcpy(&r, &h.res32[slot], 4);
        memcpy(&vm, &h.vmax32[slot], 4);
        int e = 0;
        frexpf(vm, &e);
        const double tol_eff = std::max(tol, vm > 0 ? 4.0 * ldexp(1.0, e - 24) : 0.0);
        // sweeps still needed, from the contraction observed over the last sweeps (the
        // residual ring), else from gamma; most of them are enqueued at once and the rest
        // in exact small chunks, so few sweeps are launched past the device's stop
        double rate = m->gamma;
        const long long k = std::min<long long>(std::min<long long>(chunk, kRing / 2), h.sweeps - 1);
        if (k >= 4) {
            float r0;
            memcpy(&r0, &h.res32[(h.sweeps - 1 - k) % kRing], 4);
            if (r0 > 0.0f && r > 0.0f && r < r0) rate = pow((double)r / (double)r0, 1.0 / (double)k);
        }
        const long long n = predict_sweeps(r, tol_eff, rate);
        chunk = n > 16 ? n - n / 8 : n;
        chunk = std::min<long long>(std::max<long long>(chunk, 2), 1024);
        chunk = std::min<long long>(chunk, max_sweeps - h.sweeps + 1);
    }
    *final_idx = h.final_buf;
    return VC_OK;
}

// FP64 policy evaluation V <- R_pi + gamma P_pi V until the sweep change is below tol.
// One FP64 Bellman backup V_in -> V_out with argmax pi_out; returns max|V_out - V_in| and
// the number of states whose argmax differs from pi_ref (if given).
static int cert64(Mdp* m, const double* V_in, double* V_out, int32_t* pi_out, double* qgap,
                  const int32_t* pi_ref, cudaStream_t st, double* residual, unsigned long long* changes) {
    VC_CUDA(cudaMemsetAsync(&m->ctl->changes, 0, 2 * sizeof(unsigned long long), st));
    SweepCtl sc{m->ctl, kModeCert64, 0, pi_ref};
    int rc = launch_bellman64(m, V_in, V_out, pi_out, qgap, sc, st);
    if (rc) return rc;
    if ((rc = read_ctl(m, st))) return rc;
    memcpy(residual, &m->ctl_host->cert64, 8);
    if (changes) *changes = m->ctl_host->changes;
    return VC_OK;
}

// Correction solve of the refinement, (I - gamma P_pi) e = Rres until the recurrence
// residual max |Rres - (I - gamma P_pi) e| is below target: BiCGSTAB (unless `plain`),
// else, or when BiCGSTAB breaks down or reaches its iteration cap, fixed-point sweeps
// e <- Rres + gamma P_pi e from e = 0 (each sweep's change is that residual).  *e_out
// receives the buffer holding e, *products the products by P_pi spent.
constexpr long long kKrylovMaxIter = 1000;

static int correction_solve(Mdp* m, const int32_t* pi, double target, long long max_products, bool plain,
                            cudaStream_t st, float** e_out, long long* products) {
    *products = 0;
    int rc;
    if (!plain) {
        bool conv = false;
        long long prods = 0;
        const long long iters = std::min<long long>(kKrylovMaxIter, std::max<long long>(max_products / 2, 1));
        if ((rc = krylov_correct(m, pi, m->Rres, m->E0, target, iters, st, &prods, &conv))) return rc;
        *products = prods;
        if (conv) {
            *e_out = m->E0;
            return VC_OK;
        }
    }
    VC_CUDA(cudaMemsetAsync(m->E0, 0, 4 * (size_t)m->S, st));
    int efin = 0;
    rc = loop32(m, m->E0, m->E1, target, std::max<long long>(max_products - *products, 1), st, &efin,
                [&](const float* in, float* o, SweepCtl s2) { return launch_correct32(m, pi, m->Rres, in, o, s2, st); });
    if (rc) return rc;
    *products += m->ctl_host->sweeps;
    *e_out = efin == 1 ? m->E1 : m->E0;
    return VC_OK;
}

static float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

}  // namespace vc

using namespace vc;

// =================================================================== extern "C" ABI
extern "C" {

const char* vc_last_error(void) { return g_err.c_str(); }

int64_t vc_kernel_launches(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

// Builds the sliced copy and switches the FP32 sweep to it: the first pipelined tiling that
// fits, else (or for VC_DIRECT handles) the direct sliced kernel at 4 CTAs per SM.
static int use_sliced(Mdp* m, cudaStream_t st) {
    int rc = build_sliced(m, st);
    if (rc) return rc;
    std::vector<CsrPlan> cands;
    if (!(m->fmt & VC_DIRECT) && (rc = sell_plans(m, st, cands))) return rc;
    if (cands.empty()) {
        CsrPlan P;
        P.sliced = true;
        P.ctas_per_sm = 4;
        m->plan = P;
    } else {
        m->plan = cands.front();
    }
    return VC_OK;
}

int vc_build_mdp(const vc_params* p, int fmt, void* stream, vc_mdp** out) {
    NvtxRange nv("vc_build_mdp");
    g_err.clear();
    if (!out) return fail(VC_ERR_ARG, "out is NULL");
    *out = nullptr;
    const int base = fmt & 0xF;
    if (base != VC_IMPLICIT && base != VC_CSR_F32 && base != VC_CSR_BF16)
        return fail(VC_ERR_ARG, "unknown format");
    if ((fmt & ~(0xF | VC_PADDED | VC_DIRECT | VC_SLICED)) != 0) return fail(VC_ERR_ARG, "unknown format flag");
    if (base == VC_IMPLICIT && (fmt & (VC_PADDED | VC_DIRECT | VC_SLICED)))
        return fail(VC_ERR_ARG, "VC_PADDED / VC_DIRECT / VC_SLICED need a CSR format");
    Mdp* m = new Mdp();
    m->fmt = fmt;
    m->num_sms = device_sms();
    cudaStream_t st = (cudaStream_t)stream;
    int rc = build_model(p, m);
    if (!rc) rc = upload_rate_table(m, st);
    if (!rc && base != VC_IMPLICIT) rc = build_csr_from_model(m, st);
    if (!rc && base == VC_IMPLICIT) rc = count_model_rows(m, st);  // logical nnz, nothing stored
    if (!rc) rc = alloc_work(m);
    if (!rc && (fmt & VC_SLICED)) rc = use_sliced(m, st);
    if (rc) {
        free_mdp(m);
        return rc;
    }
    *out = (vc_mdp*)m;
    return VC_OK;
}

int vc_build_binary_mdp(const vc_binary_params* p, int fmt, void* stream, vc_mdp** out) {
    NvtxRange nv("vc_build_binary_mdp");
    g_err.clear();
    if (!out) return fail(VC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!p) return fail(VC_ERR_ARG, "params is NULL");
    const int base = fmt & 0xF;
    if (base != VC_CSR_F32 && base != VC_CSR_BF16) return fail(VC_ERR_ARG, "the binary model needs a CSR format");
    if ((fmt & ~(0xF | VC_DIRECT | VC_SLICED)) != 0) return fail(VC_ERR_ARG, "unknown or unsupported format flag");
    Mdp* m = new Mdp();
    m->fmt = fmt;
    m->has_model = false;
    m->num_sms = device_sms();
    cudaStream_t st = (cudaStream_t)stream;
    int rc = build_csr_binary(m, p, st);
    if (!rc) rc = alloc_work(m);
    if (!rc && (fmt & VC_SLICED)) rc = use_sliced(m, st);
    if (rc) {
        free_mdp(m);
        return rc;
    }
    *out = (vc_mdp*)m;
    return VC_OK;
}

int vc_build_mdp_csr(int64_t S, int32_t A, const int64_t* row_ptr, const int32_t* col, const void* val,
                     int val_dtype, const float* row_scale, const float* R, double gamma, void* stream,
                     vc_mdp** out) {
    g_err.clear();
    if (!out) return fail(VC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (S < 1 || S >= 2147483647LL || A < 1 || A > 1024 || S * (int64_t)A >= (1LL << 40))
        return fail(VC_ERR_ARG, "S must be in [1, 2^31) and A in [1, 1024]");
    if (!row_ptr || !R) return fail(VC_ERR_ARG, "row_ptr / R is NULL");
    if (val_dtype != VC_VAL_F32 && val_dtype != VC_VAL_BF16) return fail(VC_ERR_ARG, "unknown val_dtype");
    if (!(gamma > 0.0 && gamma < 1.0)) return fail(VC_ERR_ARG, "gamma must be in (0, 1)");
    Mdp* m = new Mdp();
    m->fmt = val_dtype == VC_VAL_BF16 ? VC_CSR_BF16 : VC_CSR_F32;
    m->has_model = false;
    m->S = (int)S;
    m->A = A;
    m->gamma = gamma;
    m->num_sms = device_sms();
    cudaStream_t st = (cudaStream_t)stream;
    int rc = build_csr_user(m, row_ptr, col, val, val_dtype, row_scale, R, st);
    if (!rc) rc = alloc_work(m);
    if (rc) {
        free_mdp(m);
        return rc;
    }
    *out = (vc_mdp*)m;
    return VC_OK;
}

int vc_mdp_info(const vc_mdp* mh, vc_info* out) {
    g_err.clear();
    if (!mh || !out) return fail(VC_ERR_ARG, "NULL argument");
    const Mdp* m = (const Mdp*)mh;
    memset(out, 0, sizeof(*out));
    out->S = m->S;
    out->A = m->A;
    out->fmt = m->fmt;
    out->nnz_logical = m->nnz_logical;
    out->nnz_stored = m->nnz_stored;
    out->feasible_rows = m->feasible_rows;
    out->device_bytes = m->device_bytes;
    out->has_model = m->has_model ? 1 : 0;
    out->csr_pipelined = m->plan.tma ? 1 : 0;
    out->csr_tile_states = m->plan.sliced ? 32 * (m->plan.tma ? m->plan.ts : 1) : m->plan.ts;
    out->csr_stages = m->plan.stages;
    out->csr_ctas_per_sm = m->plan.ctas_per_sm;
    out->csr_smem_bytes = m->plan.smem;
    out->csr_sliced = m->plan.sliced ? 1 : 0;
    out->nnz_sliced = m->nnz_sliced;
    const int64_t rows = (int64_t)m->S * m->A;
    const int base = m->fmt & 0xF;
    if (base == VC_IMPLICIT)
        out->sweep_bytes = 8 * (int64_t)m->S;
    else if (m->plan.sliced)
        out->sweep_bytes = sell_sweep_bytes(m);
    else
        out->sweep_bytes = m->nnz_stored * ((base == VC_CSR_BF16 ? 2 : 4) + 4) + rows * (8 + 4) +
                           (base == VC_CSR_BF16 ? rows * 4 : 0) + 8 * (int64_t)m->S;
    return VC_OK;
}

int vc_set_wait_limit(vc_mdp* mh, int64_t polls) {
    g_err.clear();
    if (!mh) return fail(VC_ERR_ARG, "NULL handle");
    Mdp* m = (Mdp*)mh;
    m->spin_polls = polls < 0 ? -1 : polls;
    // also the current control block, for sweeps launched outside a solve
    const long long v = polls < 0 ? 0 : polls + 1;
    VC_CUDA(cudaMemcpy(&m->ctl->spin_limit, &v, sizeof(v), cudaMemcpyHostToDevice));
    return VC_OK;
}

int vc_mdp_slice(vc_mdp* mh, void* stream) {
    NvtxRange nv("vc_mdp_slice");
    g_err.clear();
    if (!mh) return fail(VC_ERR_ARG, "NULL handle");
    Mdp* m = (Mdp*)mh;
    if ((m->fmt & 0xF) == VC_IMPLICIT) return fail(VC_ERR_ARG, "an implicit handle stores no matrix to slice");
    int rc = use_sliced(m, (cudaStream_t)stream);
    if (rc) return rc;
    m->fmt |= VC_SLICED;
    return VC_OK;
}

int vc_mdp_export_csr(const vc_mdp* mh, int64_t* row_ptr, int32_t* col, void* val, float* row_scale, float* R,
                      void* stream) {
    g_err.clear();
    if (!mh) return fail(VC_ERR_ARG, "NULL handle");
    const Mdp* m = (const Mdp*)mh;
    const int base = m->fmt & 0xF;
    if (base == VC_IMPLICIT) return fail(VC_ERR_ARG, "an implicit handle stores no CSR");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t rows = (size_t)m->S * m->A;
    const size_t nnz = (size_t)m->nnz_stored;
    if (row_ptr) VC_CUDA(cudaMemcpyAsync(row_ptr, m->row_ptr, 8 * (rows + 1), cudaMemcpyDeviceToDevice, st));
    if (col && nnz) VC_CUDA(cudaMemcpyAsync(col, m->col, 4 * nnz, cudaMemcpyDeviceToDevice, st));
    if (val && nnz)
        VC_CUDA(cudaMemcpyAsync(val, m->val, (base == VC_CSR_BF16 ? 2 : 4) * nnz, cudaMemcpyDeviceToDevice, st));
    if (row_scale && m->scale) VC_CUDA(cudaMemcpyAsync(row_scale, m->scale, 4 * rows, cudaMemcpyDeviceToDevice, st));
    if (R) VC_CUDA(cudaMemcpyAsync(R, m->R, 4 * rows, cudaMemcpyDeviceToDevice, st));
    return VC_OK;
}

int vc_value_grad(vc_mdp* mh, const double* V, const int32_t* pi, const double* rho, double* dJ_dtheta,
                  double* lambda_out, double tol, int64_t max_sweeps, vc_grad_stats* stats, void* stream) {
    NvtxRange nv("vc_value_grad");
    g_err.clear();
    if (!mh || !V || !pi || !rho || !dJ_dtheta) return fail(VC_ERR_ARG, "NULL argument");
    if (!(tol > 0.0) || max_sweeps < 1) return fail(VC_ERR_ARG, "tol must be > 0 and max_sweeps >= 1");
    Mdp* m = (Mdp*)mh;
    if (!m->has_model) return fail(VC_ERR_ARG, "the gradient needs a handle built from model parameters");
    cudaStream_t st = (cudaStream_t)stream;
    const int S = m->S;
    const int nt = 2 * m->md.H + 5;
    vc_grad_stats gs;
    memset(&gs, 0, sizeof(gs));

    // temporaries, stream-ordered; freed on every exit path
    int32_t* cnt = nullptr;
    int32_t* fillpos = nullptr;
    int64_t* rowT = nullptr;
    int32_t* colT = nullptr;
    float* valT = nullptr;
    double* valT64 = nullptr;
    float* rhoF = nullptr;
    double* partial = nullptr;
    double* out = nullptr;
    int* err = nullptr;
    auto release = [&]() {
        void* ps[] = {cnt, fillpos, rowT, colT, valT, valT64, rhoF, partial, out, err};
        for (void* p : ps)
            if (p) cudaFreeAsync(p, st);
    };
    auto bail = [&](int rc) {
        release();
        cudaStreamSynchronize(st);
        return rc;
    };
#define VC_TRY(call)                                                \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return bail(cuda_fail(e_, #call)); \
    } while (0)

    // ---- P_pi^T: in-degree count, exclusive scan, fill, per-row sort by source
    VC_TRY(cudaMallocAsync((void**)&cnt, 4 * (size_t)S, st));
    VC_TRY(cudaMallocAsync((void**)&fillpos, 4 * (size_t)S, st));
    VC_TRY(cudaMallocAsync((void**)&rowT, 8 * ((size_t)S + 3), st));
    VC_TRY(cudaMallocAsync((void**)&err, 16, st));
    VC_TRY(cudaMemsetAsync(cnt, 0, 4 * (size_t)S, st));
    VC_TRY(cudaMemsetAsync(fillpos, 0, 4 * (size_t)S, st));
    VC_TRY(cudaMemsetAsync(err, 0, 16, st));
    int rc = launch_adj_count(m, pi, cnt, err, st);
    if (rc) return bail(rc);
    if ((rc = exclusive_scan(m, cnt, S, rowT, st))) return bail(rc);
    int herr = 0;
    int64_t nnzT = 0;
    VC_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    VC_TRY(cudaMemcpyAsync(&nnzT, rowT + S, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    VC_TRY(cudaStreamSynchronize(st));
    if (herr) return bail(fail(VC_ERR_ARG, "the policy picks an infeasible action"));
    gs.nnz_transpose = nnzT;
    VC_TRY(cudaMallocAsync((void**)&colT, 4 * ((size_t)nnzT + 16), st));
    VC_TRY(cudaMallocAsync((void**)&valT, 4 * ((size_t)nnzT + 16), st));
    VC_TRY(cudaMallocAsync((void**)&valT64, 8 * ((size_t)nnzT + 16), st));
    if ((rc = launch_adj_fill(m, pi, rowT, fillpos, colT, valT, valT64, st))) return bail(rc);

    // ---- lam: the transposed system as a one-action stored MDP (reward rho, matrix P^T)
    VC_TRY(cudaMallocAsync((void**)&rhoF, 4 * ((size_t)S + 8), st));
    if ((rc = launch_f64_to_f32(rho, rhoF, S, st))) return bail(rc);
    Mdp T;
    T.fmt = VC_CSR_F32 | VC_DIRECT;
    T.has_model = false;
    T.S = S;
    T.A = 1;
    T.gamma = m->gamma;
    T.row_ptr = rowT;
    T.col = colT;
    T.val = valT;
    T.R = rhoF;
    T.ctl = m->ctl;
    T.ctl_host = m->ctl_host;
    T.num_sms = m->num_sms;
    T.kr = m->kr;  // BiCGSTAB work space of the handle
    T.kr_part = m->kr_part;
    T.kctl = m->kctl;
    T.kctl_host = m->kctl_host;
    auto sweep_T = [&](const float* in, float* o, SweepCtl sc) { return csr_sweep32(&T, in, o, nullptr, nullptr, sc, st); };
    // (I - gamma P_pi^T) x = b in FP32: BiCGSTAB, or fixed-point sweeps x <- b + gamma P^T x
    // from x = 0 (T.R = b) when it breaks down; *xo receives the buffer holding x
    auto solve_T = [&](float* b, double target, float** xo, long long* prods) -> int {
        bool conv = false;
        int r = krylov_correct(&T, nullptr, b, m->E0, target, std::min<long long>(kKrylovMaxIter, max_sweeps), st,
                               prods, &conv);
        if (r || conv) {
            *xo = m->E0;
            return r;
        }
        T.R = b;
        VC_CUDA(cudaMemsetAsync(m->E0, 0, 4 * (size_t)S, st));
        int fin = 0;
        if ((r = loop32(m, m->E0, m->E1, target, max_sweeps, st, &fin, sweep_T))) return r;
        *prods += m->ctl_host->sweeps;
        *xo = fin == 1 ? m->E1 : m->E0;
        return VC_OK;
    };
    float* lamF = nullptr;
    long long prods = 0;
    if ((rc = solve_T(rhoF, tol, &lamF, &prods))) return bail(rc);
    gs.sweeps = prods;
    double* lam = m->V64b;
    if ((rc = launch_f32_to_f64(lamF, lam, S, st))) return bail(rc);

    // ---- FP64 residual + FP32 correction rounds
    bool ok = false;
    for (int round = 0; round < 20; round++) {
        VC_TRY(cudaMemsetAsync(&m->ctl->changes, 0, 2 * sizeof(unsigned long long), st));
        SweepCtl sc{m->ctl, kModeCert64, 0, nullptr};
        if ((rc = launch_adj_resid64(m, rowT, colT, valT64, rho, lam, m->Rres, sc, st))) return bail(rc);
        VC_TRY(cudaMemcpyAsync(m->ctl_host, m->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        VC_TRY(cudaStreamSynchronize(st));
        double r64;
        memcpy(&r64, &m->ctl_host->cert64, 8);
        gs.residual64 = r64;
        if (r64 < tol) {
            ok = true;
            break;
        }
        gs.rounds++;
        // correction (I - gamma P^T) e = r
        float* e = nullptr;
        long long cp = 0;
        if ((rc = solve_T(m->Rres, 0.5 * tol, &e, &cp))) return bail(rc);
        gs.correction_sweeps += cp;
        if ((rc = launch_axpy64(lam, e, S, st))) return bail(rc);
    }

    // ---- contraction over states, reduced in a fixed order
    const int g = state_grid(m);
    VC_TRY(cudaMallocAsync((void**)&partial, 8 * (size_t)g * grad_partial_stride(m), st));
    VC_TRY(cudaMallocAsync((void**)&out, 8 * ((size_t)nt + 1), st));
    if ((rc = launch_grad_contract(m, pi, V, lam, rho, partial, out, st))) return bail(rc);
    VC_TRY(cudaMemcpyAsync(dJ_dtheta, out, 8 * (size_t)nt, cudaMemcpyDeviceToDevice, st));
    VC_TRY(cudaMemcpyAsync(&gs.J, out + nt, 8, cudaMemcpyDeviceToHost, st));
    if (lambda_out) VC_TRY(cudaMemcpyAsync(lambda_out, lam, 8 * (size_t)S, cudaMemcpyDeviceToDevice, st));
    release();
    VC_TRY(cudaStreamSynchronize(st));
#undef VC_TRY
    if (stats) *stats = gs;
    if (!ok) return fail(VC_ERR_NOT_CONVERGED, "adjoint residual above tol");
    return VC_OK;
}

int vc_autotune(vc_mdp* mh, int reps, double* best_us, void* stream) {
    NvtxRange nv("vc_autotune");
    g_err.clear();
    if (!mh) return fail(VC_ERR_ARG, "NULL handle");
    Mdp* m = (Mdp*)mh;
    if ((m->fmt & 0xF) == VC_IMPLICIT) {
        if (best_us) *best_us = 0.0;
        return VC_OK;
    }
    return autotune_csr(m, reps, (cudaStream_t)stream, best_us);
}

int vc_sweep_schedule(vc_mdp* mh, int32_t index, int32_t* count, void* stream) {
    g_err.clear();
    if (!mh) return fail(VC_ERR_ARG, "NULL handle");
    Mdp* m = (Mdp*)mh;
    if ((m->fmt & 0xF) == VC_IMPLICIT) return fail(VC_ERR_ARG, "an implicit handle has one sweep schedule");
    std::vector<CsrPlan> cands;
    int rc = csr_candidates(m, (cudaStream_t)stream, cands);
    if (rc) return rc;
    if (count) *count = (int32_t)cands.size();
    if (index < 0) return VC_OK;
    if (index >= (int32_t)cands.size()) return fail(VC_ERR_ARG, "schedule index out of range");
    m->plan = cands[(size_t)index];
    return VC_OK;
}

int64_t vc_autotune_report(const vc_mdp* mh, char* buf, int64_t len) {
    if (!mh) return 0;
    const std::string& r = ((const Mdp*)mh)->tune_report;
    if (buf && len > 0) {
        const int64_t n = std::min<int64_t>(len - 1, (int64_t)r.size());
        memcpy(buf, r.data(), (size_t)n);
        buf[n] = 0;
    }
    return (int64_t)r.size() + 1;
}

int vc_destroy(vc_mdp* mh) {
    g_err.clear();
    free_mdp((Mdp*)mh);
    return VC_OK;
}

int vc_extract_policy(vc_mdp* mh, const float* V, int32_t* pi, float* qgap, void* stream) {
    g_err.clear();
    if (!mh || !V || !pi) return fail(VC_ERR_ARG, "NULL argument");
    Mdp* m = (Mdp*)mh;
    SweepCtl sc{m->ctl, kModeNone, 0, nullptr};
    return launch_sweep32(m, V, nullptr, pi, qgap, sc, (cudaStream_t)stream);
}

int vc_set_block_iteration(vc_mdp* mh, int32_t inner_hosts, int32_t passes) {
    g_err.clear();
    if (!mh) return fail(VC_ERR_ARG, "NULL handle");
    Mdp* m = (Mdp*)mh;
    if ((m->fmt & 0xF) != VC_IMPLICIT) return fail(VC_ERR_ARG, "the in-block iteration needs a VC_IMPLICIT handle");
    if (passes < 1 || passes > 64) return fail(VC_ERR_ARG, "passes must be in 1..64");
    if (inner_hosts < -1 || inner_hosts > m->md.H) return fail(VC_ERR_ARG, "inner_hosts must be in -1..H");
    const int old_h = m->blk_h;
    m->blk_h = inner_hosts;
    int h = 0, B = 0;
    const int rc = block_shape(m, &h, &B);
    if (rc) {
        m->blk_h = old_h;
        return rc;
    }
    m->blk_passes = passes;
    m->blk_grid = 0;
    return VC_OK;
}

int vc_block_iteration_info(const vc_mdp* mh, int32_t* inner_hosts, int32_t* block_states, int32_t* passes) {
    g_err.clear();
    if (!mh) return fail(VC_ERR_ARG, "NULL handle");
    const Mdp* m = (const Mdp*)mh;
    if ((m->fmt & 0xF) != VC_IMPLICIT) return fail(VC_ERR_ARG, "the in-block iteration needs a VC_IMPLICIT handle");
    int h = 0, B = 0;
    const int rc = block_shape(m, &h, &B);
    if (rc) return rc;
    if (inner_hosts) *inner_hosts = h;
    if (block_states) *block_states = B;
    if (passes) *passes = m->blk_passes;
    return VC_OK;
}

int vc_bellman32(vc_mdp* mh, const float* V, float* V_out, int32_t* pi, float* qgap, void* stream) {
    g_err.clear();
    if (!mh || !V) return fail(VC_ERR_ARG, "NULL argument");
    Mdp* m = (Mdp*)mh;
    SweepCtl sc{m->ctl, kModeNone, 0, nullptr};
    return launch_sweep32(m, V, V_out, pi, qgap, sc, (cudaStream_t)stream);
}

int vc_bellman64(vc_mdp* mh, const double* V, double* V_out, int32_t* pi, double* qgap, double* residual,
                 void* stream) {
    g_err.clear();
    if (!mh || !V) return fail(VC_ERR_ARG, "NULL argument");
    Mdp* m = (Mdp*)mh;
    cudaStream_t st = (cudaStream_t)stream;
    if (residual) {
        double r = 0;
        int rc = cert64(m, V, V_out, pi, qgap, nullptr, st, &r, nullptr);
        if (rc) return rc;
        *residual = r;
        return VC_OK;
    }
    SweepCtl sc{m->ctl, kModeNone, 0, nullptr};
    return launch_bellman64(m, V, V_out, pi, qgap, sc, st);
}

int vc_greedy_policy(vc_mdp* mh, int32_t* pi, void* stream) {
    g_err.clear();
    if (!mh || !pi) return fail(VC_ERR_ARG, "NULL argument");
    Mdp* m = (Mdp*)mh;
    if (!m->has_model) return fail(VC_ERR_ARG, "the greedy heuristic needs a handle built from model parameters");
    return launch_greedy(m, pi, (cudaStream_t)stream);
}

int vc_evaluate_policy(vc_mdp* mh, const int32_t* pi, double* V_pi, double tol, int64_t max_sweeps,
                       int64_t* sweeps_out, void* stream) {
    NvtxRange nv("vc_evaluate_policy");
    g_err.clear();
    if (!mh || !pi || !V_pi) return fail(VC_ERR_ARG, "NULL argument");
    if (!(tol > 0.0) || max_sweeps < 1) return fail(VC_ERR_ARG, "tol must be > 0 and max_sweeps >= 1");
    Mdp* m = (Mdp*)mh;
    cudaStream_t st = (cudaStream_t)stream;
    // Mixed-precision iterative refinement of V_pi = R_pi + gamma P_pi V_pi: the policy
    // residual r = T_pi V - V and its maximum in FP64, the correction (I - gamma P_pi) e = r
    // in FP32 (BiCGSTAB, fixed-point sweeps as the fallback) until its residual is below
    // tol/2, V += e in FP64; stop when max|r| < tol (the FP64 Jacobi criterion: the next
    // sweep would change V by less than tol).  max_sweeps caps the products by P_pi.
    long long total = 0;
    int rc;
    for (int round = 0; round < 60; round++) {
        VC_CUDA(cudaMemsetAsync(&m->ctl->cert64, 0, sizeof(unsigned long long), st));
        VC_CUDA(cudaMemsetAsync(&m->ctl->error, 0, sizeof(int), st));
        SweepCtl sc{m->ctl, kModeCert64, 0, nullptr};
        if ((rc = launch_resid64(m, pi, V_pi, m->Rres, sc, st))) return rc;
        if ((rc = read_ctl(m, st))) return rc;
        if (m->ctl_host->error & kErrInfeasiblePolicy) return fail(VC_ERR_ARG, "the policy picks an infeasible action");
        double r;
        memcpy(&r, &m->ctl_host->cert64, 8);
        if (r < tol) {
            if (sweeps_out) *sweeps_out = total;
            return VC_OK;
        }
        if (total >= max_sweeps) break;
        float* e = nullptr;
        long long prods = 0;
        rc = correction_solve(m, pi, 0.5 * tol, max_sweeps - total, false, st, &e, &prods);
        total += prods;
        if (rc) return rc;
        if ((rc = launch_axpy64(V_pi, e, m->S, st))) return rc;
    }
    VC_CUDA(cudaStreamSynchronize(st));
    if (sweeps_out) *sweeps_out = total;
    return fail(VC_ERR_NOT_CONVERGED, "policy evaluation hit max_sweeps");
}

int vc_value_iterate(vc_mdp* mh, float* V, double* V64_out, int32_t* pi_out, double tol, int64_t max_sweeps,
                     int flags, vc_stats* stats, void* stream) {
    NvtxRange nv("vc_value_iterate");
    g_err.clear();
    if (!mh || !V) return fail(VC_ERR_ARG, "NULL argument");
    if (!(tol > 0.0) || max_sweeps < 1) return fail(VC_ERR_ARG, "tol must be > 0 and max_sweeps >= 1");
    Mdp* m = (Mdp*)mh;
    cudaStream_t st = (cudaStream_t)stream;
    vc_stats sx;
    memset(&sx, 0, sizeof(sx));
    cudaEvent_t ev[3];
    for (auto& e : ev) VC_CUDA(cudaEventCreate(&e));
    int rc = VC_OK;
    int fin = 0;
    const size_t S = (size_t)m->S;

    VC_CUDA(cudaEventRecord(ev[0], st));
    {
        NvtxRange nv32("fp32 sweeps");
        const int block = (flags & VC_ITER_BLOCK) ? 1 : 0;
        const int self_loop = ((flags & VC_ITER_SELF_LOOP) || block) ? 1 : 0;
        if (block && (m->fmt & 0xF) != VC_IMPLICIT) {
            rc = fail(VC_ERR_ARG, "VC_ITER_BLOCK needs a VC_IMPLICIT handle");
            goto out;
        }
        rc = loop32(m, V, m->Vb, tol, max_sweeps, st, &fin, [&](const float* in, float* o, SweepCtl sc) {
            sc.self_loop = self_loop;
            sc.block = block;
            return launch_sweep32(m, in, o, nullptr, nullptr, sc, st);
        });
    }
    if (rc) goto out;
    if (fin == 1) VC_CUDA(cudaMemcpyAsync(V, m->Vb, 4 * S, cudaMemcpyDeviceToDevice, st));
    VC_CUDA(cudaEventRecord(ev[1], st));
    sx.sweeps = m->ctl_host->sweeps;
    {
        float r;
        memcpy(&r, &m->ctl_host->res32[(sx.sweeps - 1) % kRing], 4);
        sx.residual = r;
    }
    {
        const int done32 = m->ctl_host->done;
        if (flags & VC_ITER_FP32_ONLY) {
            if (pi_out) {
                SweepCtl sc{m->ctl, kModeNone, 0, nullptr};
                if ((rc = launch_sweep32(m, V, nullptr, pi_out, nullptr, sc, st))) goto out;
            }
            if (V64_out) {
                if ((rc = launch_f32_to_f64(V, V64_out, m->S, st))) goto out;
            }
            VC_CUDA(cudaEventRecord(ev[2], st));
            VC_CUDA(cudaStreamSynchronize(st));
            if (done32 == 2) rc = fail(VC_ERR_NOT_CONVERGED, "max_sweeps reached before the FP32 tolerance");
            goto out;
        }
        // ---- refinement: the argmax policy of the FP32 values (Algorithm 3, step 4) is
        // evaluated by mixed-precision iterative refinement -- policy residual
        // r = T_pi V64 - V64 in FP64, correction (I - gamma P_pi) e = r solved in FP32 by
        // BiCGSTAB (or fixed-point sweeps: VC_ITER_PLAIN_CORRECTION, and the fallback),
        // V64 += e -- and certified by one FP64 Bellman backup whose residual is the
        // step-3 test.  If the backup's argmax differs, the loop repeats with it (a
        // policy-improvement step).  Since T_pi(V64 + e) - (V64 + e) = r - (I - gamma P_pi) e
        // is the correction's own residual, solving it to tol/2 leaves a policy residual
        // below tol (up to FP32 rounding of e).
        int32_t* pcur = m->pi;
        int32_t* pnew = m->pi2;
        if ((rc = launch_f32_to_f64(V, m->V64a, m->S, st))) goto out;
        if ((m->fmt & 0xF) == VC_CSR_BF16 && (m->has_model || m->val64)) {
            // BF16 storage: the FP32 iterate carries the BF16 matrix's modelling error, so
            // the first policy is the argmax of an FP64 backup of it with the exact model
            // (one policy-improvement step of the exact MDP from that iterate) rather than
            // the stored matrix's argmax, which would only be corrected by a later round
            SweepCtl sc{m->ctl, kModeNone, 0, nullptr};
            if ((rc = launch_bellman64(m, m->V64a, m->V64b, pcur, nullptr, sc, st))) goto out;
        } else {
            SweepCtl sc{m->ctl, kModeNone, 0, nullptr};
            if ((rc = launch_sweep32(m, V, nullptr, pcur, nullptr, sc, st))) goto out;
        }
        double* cur = m->V64a;
        double* other = m->V64b;
        const long long eval_max = std::max<long long>(100000, max_sweeps);
        // certificate target: Algorithm 3's residual test, or (VC_ITER_ACCURATE) the
        // residual that bounds max|V64 - V*| by tol/2 through gamma/(1-gamma)
        const double r_target = (flags & VC_ITER_ACCURATE) ? tol * (1.0 - m->gamma) / (2.0 * m->gamma) : tol;
        bool certified = false;
        double r64 = INFINITY;
        for (int round = 0; round < 50; round++) {
            {
                SweepCtl sc{m->ctl, kModeNone, 0, nullptr};
                VC_CUDA(cudaMemsetAsync(&m->ctl->error, 0, sizeof(int), st));
                if ((rc = launch_resid64(m, pcur, cur, m->Rres, sc, st))) goto out;
            }
            {
                float* e = nullptr;
                long long prods = 0;
                rc = correction_solve(m, pcur, 0.5 * r_target, eval_max, (flags & VC_ITER_PLAIN_CORRECTION) != 0, st,
                                      &e, &prods);
                sx.eval_sweeps += prods;
                if (rc) goto out;
                if ((rc = launch_axpy64(cur, e, m->S, st))) goto out;
            }
            unsigned long long changes = 0;
            if ((rc = cert64(m, cur, other, pnew, nullptr, pcur, st, &r64, &changes))) goto out;
            sx.bellman64++;
            sx.residual64 = r64;
            std::swap(cur, other);  // cur = T(previous), Algorithm 3's V^{k+1}
            std::swap(pcur, pnew);  // pcur = argmax of that backup
            if (r64 < r_target) {
                certified = true;
                break;
            }
            sx.policy_rounds++;
        }
        sx.certified = certified ? 1 : 0;
        if (V64_out) VC_CUDA(cudaMemcpyAsync(V64_out, cur, 8 * S, cudaMemcpyDeviceToDevice, st));
        if (pi_out) VC_CUDA(cudaMemcpyAsync(pi_out, pcur, 4 * S, cudaMemcpyDeviceToDevice, st));
        VC_CUDA(cudaEventRecord(ev[2], st));
        VC_CUDA(cudaStreamSynchronize(st));
        if (!certified) rc = fail(VC_ERR_NOT_CONVERGED, "FP64 certificate not reached");
    }
out:
    if (!rc || rc == VC_ERR_NOT_CONVERGED) {
        sx.ms_fp32 = elapsed(ev[0], ev[1]);
        sx.ms_fp64 = elapsed(ev[1], ev[2]);
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (stats) *stats = sx;
    return rc;
}

}  // extern "C"
