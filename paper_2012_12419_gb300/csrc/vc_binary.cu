// vc_binary.cu -- explicit CSR of the paper's binary-action model (Section V-B..V-E):
// state (busy VMs of each vehicular cloud, pending request) of Eq. 10, actions {-1, 1} of
// Eq. 11, reward k - g of Eqs. 14-16, one uniformised event per step.  Built on the device
// by a count pass, an exclusive scan and a fill pass; the fill also writes the exact FP64
// probabilities and rewards, which the FP64 refinement and certificate use.
#include <math.h>

#include <algorithm>

#include "vc_internal.cuh"

namespace vc {

struct BinModel {
    int H, C, J, E;  // clouds, VMs per cloud, largest request, request codes 1 + H J
    int S;
    int stride[VC_MAX_HOSTS];  // E (C+1)^k
    double arr;                // lambda / (H J): rate of each request kind
    double Lam;                // uniformisation constant
    double mu[VC_MAX_HOSTS], delta[VC_MAX_HOSTS];
    double bvc, btc, gvc;
};

// Row (s, a), entries emitted in ascending column order through emit(j, col, p); returns
// the number of entries or -1 if a is infeasible in s.  Column order: for cloud k from the
// highest stride down, its departure (u_k = 0) below its completion (u_k - 1), both below
// every target of cloud k-1 (u_{k-1} stride_{k-1} <= C stride_{k-1} < stride_k); then the
// post-decision state itself; then the request kinds x + 1 .. x + HJ (below x + stride_0).
template <typename F>
__device__ __forceinline__ int bin_row_emit(const BinModel& md, int s, int a, double* R, F&& emit) {
    const int e = s % md.E;
    int rest = s / md.E;
    int u[VC_MAX_HOSTS];
    for (int k = 0; k < md.H; k++) {
        u[k] = rest % (md.C + 1);
        rest /= (md.C + 1);
    }
    int x = s - e;
    if (a == 1) {
        if (e == 0) return -1;
        const int vc = (e - 1) / md.J, n = (e - 1) % md.J + 1;
        if (u[vc] + n > md.C) return -1;
        u[vc] += n;
        x += n * md.stride[vc];
        *R = md.bvc * n - md.gvc * (md.C - u[vc]);
    } else {
        if (e == 0) {
            *R = 0.0;
        } else {
            const int vc = (e - 1) / md.J, n = (e - 1) % md.J + 1;
            *R = -md.btc * n - md.gvc * (md.C - u[vc]);
        }
    }
    // probability of leaving x: every busy cloud's completion and departure, every request
    const double pa = md.arr / md.Lam;
    double moved = 0.0;
    for (int k = 0; k < md.H; k++) {
        if (u[k] > 0) moved += md.mu[k] * u[k] / md.Lam + md.delta[k] / md.Lam;
    }
    moved += (md.H * md.J) * pa;
    int j = 0;
    for (int k = md.H - 1; k >= 0; k--) {
        if (u[k] == 0) continue;  // no completion; a departure stays at x
        if (u[k] == 1) {
            emit(j++, x - md.stride[k], md.mu[k] / md.Lam + md.delta[k] / md.Lam);
        } else {
            if (md.delta[k] > 0.0) emit(j++, x - u[k] * md.stride[k], md.delta[k] / md.Lam);
            emit(j++, x - md.stride[k], md.mu[k] * u[k] / md.Lam);
        }
    }
    emit(j++, x, 1.0 - moved);
    for (int c = 1; c < md.E; c++) emit(j++, x + c, pa);
    return j;
}

__global__ void __launch_bounds__(kThreads) k_bin_count(BinModel md, int64_t nrows, int32_t* cnt,
                                                        unsigned long long* tallies) {
    unsigned long long feas = 0, nz = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x) {
        double R;
        const int n = bin_row_emit(md, (int)(r >> 1), (int)(r & 1), &R, [](int, int, double) {});
        cnt[r] = n < 0 ? 0 : n;
        if (n >= 0) {
            feas += 1;
            nz += (unsigned long long)n;
        }
    }
    block_tally<kThreads>(feas, nz, tallies);
}

// Nearest-even bfloat16 of a positive double through round-to-odd at float precision
// (Boldo & Melquiond, IEEE Trans. Computers 57(4), 2008), as the model CSR build does.
__device__ __forceinline__ uint16_t bin_bf16_rne(double x) {
    float t = __double2float_rz(x);
    uint32_t u = __float_as_uint(t);
    if ((double)t != x) u |= 1u;
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

template <bool kBf16>
__global__ void k_bin_fill(BinModel md, int64_t nrows, const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                           void* __restrict__ val, float* __restrict__ scale, float* __restrict__ R,
                           double* __restrict__ val64, double* __restrict__ R64) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const int64_t base = row_ptr[r];
    double Rv = 0.0, tot = 0.0;
    const int n = bin_row_emit(md, (int)(r >> 1), (int)(r & 1), &Rv, [&](int j, int c, double p) {
        col[base + j] = c;
        val64[base + j] = p;
        if (kBf16) {
            const uint16_t b = bin_bf16_rne(p);
            ((uint16_t*)val)[base + j] = b;
            tot += (double)__uint_as_float((uint32_t)b << 16);
        } else {
            ((float*)val)[base + j] = (float)p;
        }
    });
    if (n < 0) {
        R[r] = -INFINITY;
        R64[r] = -INFINITY;
        if (kBf16) scale[r] = 0.0f;
        return;
    }
    R[r] = (float)Rv;
    R64[r] = Rv;
    if (kBf16) scale[r] = (float)(1.0 / tot);
}

static int bin_model_of(const vc_binary_params* p, BinModel* md) {
    if (!p) return fail(VC_ERR_ARG, "params is NULL");
    if (p->H < 1 || p->H > VC_MAX_HOSTS) return fail(VC_ERR_ARG, "H must be in 1..16");
    if (p->J < 1 || p->J > 8) return fail(VC_ERR_ARG, "J must be in 1..8");
    if (p->C < 1) return fail(VC_ERR_ARG, "C must be >= 1");
    if (!(p->gamma > 0.0 && p->gamma < 1.0)) return fail(VC_ERR_ARG, "gamma must be in (0, 1)");
    if (!(p->lambda > 0.0) || !isfinite(p->lambda)) return fail(VC_ERR_ARG, "lambda must be > 0");
    if (!isfinite(p->beta_vc) || !isfinite(p->beta_tc) || !isfinite(p->gamma_vc))
        return fail(VC_ERR_ARG, "reward weights must be finite");
    if (!p->mu || !p->delta) return fail(VC_ERR_ARG, "mu / delta is NULL");
    md->H = p->H;
    md->C = p->C;
    md->J = p->J;
    md->E = 1 + p->H * p->J;
    double S = md->E;
    for (int k = 0; k < p->H; k++) {
        md->stride[k] = (int)S;
        S *= (p->C + 1);
        if (S >= 2147483647.0) return fail(VC_ERR_ARG, "S = (1 + H J)(C+1)^H must stay below 2^31");
    }
    md->S = (int)S;
    double smu = 0.0, sde = 0.0;
    for (int k = 0; k < p->H; k++) {
        if (!(p->mu[k] > 0.0) || !isfinite(p->mu[k])) return fail(VC_ERR_ARG, "every mu must be > 0");
        if (!(p->delta[k] >= 0.0) || !isfinite(p->delta[k])) return fail(VC_ERR_ARG, "every delta must be >= 0");
        md->mu[k] = p->mu[k];
        md->delta[k] = p->delta[k];
        smu += p->mu[k];
        sde += p->delta[k];
    }
    for (int k = p->H; k < VC_MAX_HOSTS; k++) md->mu[k] = md->delta[k] = 0.0, md->stride[k] = 0;
    md->Lam = p->lambda + p->C * smu + sde + 1.0;
    md->arr = p->lambda / (p->H * p->J);
    md->bvc = p->beta_vc;
    md->btc = p->beta_tc;
    md->gvc = p->gamma_vc;
    return VC_OK;
}

int build_csr_binary(Mdp* m, const vc_binary_params* p, cudaStream_t st) {
    BinModel md;
    int rc = bin_model_of(p, &md);
    if (rc) return rc;
    m->S = md.S;
    m->A = 2;
    m->gamma = p->gamma;
    const bool bf16 = (m->fmt & 0xF) == VC_CSR_BF16;
    const int64_t nrows = 2 * (int64_t)md.S;
    const int T = 256;
    const unsigned nb = (unsigned)((nrows + T - 1) / T);

    int32_t* cnt = nullptr;
    unsigned long long* tallies = nullptr;
    unsigned long long th[2] = {0, 0};
    VC_CUDA(cudaMallocAsync((void**)&tallies, sizeof(unsigned long long) * 2, st));
    VC_CUDA(cudaMemsetAsync(tallies, 0, sizeof(unsigned long long) * 2, st));
    VC_CUDA(cudaMallocAsync((void**)&cnt, sizeof(int32_t) * nrows, st));
    count_launches(1);
    k_bin_count<<<(unsigned)std::min<int64_t>(nb, (int64_t)m->num_sms * 16), kThreads, 0, st>>>(md, nrows, cnt, tallies);
    VC_CUDA(cudaGetLastError());
    VC_CUDA(cudaMemcpyAsync(th, tallies, sizeof(th), cudaMemcpyDeviceToHost, st));
    VC_CUDA(cudaStreamSynchronize(st));
    m->feasible_rows = (int64_t)th[0];
    m->nnz_logical = (int64_t)th[1];
    m->nnz_stored = m->nnz_logical;

    if ((rc = alloc_dev(m, (void**)&m->row_ptr, sizeof(int64_t) * (nrows + 3)))) return rc;
    if ((rc = alloc_dev(m, (void**)&m->col, sizeof(int32_t) * (m->nnz_stored + 16)))) return rc;
    if ((rc = alloc_dev(m, &m->val, (bf16 ? 2 : 4) * (size_t)(m->nnz_stored + 16)))) return rc;
    if ((rc = alloc_dev(m, (void**)&m->R, sizeof(float) * (nrows + 8)))) return rc;
    if (bf16 && (rc = alloc_dev(m, (void**)&m->scale, sizeof(float) * (nrows + 8)))) return rc;
    if ((rc = alloc_dev(m, (void**)&m->val64, sizeof(double) * (m->nnz_stored + 2)))) return rc;
    if ((rc = alloc_dev(m, (void**)&m->R64, sizeof(double) * nrows))) return rc;
    if ((rc = exclusive_scan(m, cnt, nrows, m->row_ptr, st))) return rc;
    count_launches(1);
    if (bf16)
        k_bin_fill<true><<<nb, T, 0, st>>>(md, nrows, m->row_ptr, m->col, m->val, m->scale, m->R, m->val64, m->R64);
    else
        k_bin_fill<false><<<nb, T, 0, st>>>(md, nrows, m->row_ptr, m->col, m->val, nullptr, m->R, m->val64, m->R64);
    VC_CUDA(cudaGetLastError());
    VC_CUDA(cudaFreeAsync(cnt, st));
    VC_CUDA(cudaFreeAsync(tallies, st));
    VC_CUDA(cudaStreamSynchronize(st));
    return plan_csr(m, st);
}

}  // namespace vc
