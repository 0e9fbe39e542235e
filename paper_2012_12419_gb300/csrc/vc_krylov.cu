// vc_krylov.cu -- BiCGSTAB for the correction equation (I - gamma P_pi) e = r of the
// mixed-precision refinement (single handle): the element-wise kernels of one iteration
// and the host driver.  The two products by the matrix are launch_apply32 (implicit model
// or stored rows).  Iterations are enqueued in chunks sized from the observed rate of
// decrease; the host reads the control block between chunks only.
#include <math.h>

#include <algorithm>

#include "vc_krylov.cuh"

namespace vc {

// r = b, x = 0, with <b, b> and max |b|.
__global__ void __launch_bounds__(kThreads) k_kr_init(KrylovArgs k) {
    if (kr_done(k)) return;
    float d0 = 0.0f, mx = 0.0f;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < k.n; i += gridDim.x * kThreads) {
        const float b = k.b[i];
        k.r[i] = b;
        k.x[i] = 0.0f;
        d0 = fmaf(b, b, d0);
        mx = fmaxf(mx, fabsf(b));
    }
    kr_finish<kThreads>(k, kKrInit, d0, 0.0f, mx);
}

// p = r (first iteration), else p = r + beta (p - omega v).
__global__ void __launch_bounds__(kThreads) k_kr_p(KrylovArgs k) {
    if (kr_done(k)) return;
    const bool first = k.kc->iter == 0;
    const float beta = (float)k.kc->beta, omega = (float)k.kc->omega;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < k.n; i += gridDim.x * kThreads)
        k.p[i] = first ? k.r[i] : fmaf(beta, fmaf(-omega, k.v[i], k.p[i]), k.r[i]);
}

// s = r - alpha v.
__global__ void __launch_bounds__(kThreads) k_kr_s(KrylovArgs k) {
    if (kr_done(k)) return;
    const float alpha = (float)k.kc->alpha;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < k.n; i += gridDim.x * kThreads)
        k.s[i] = fmaf(-alpha, k.v[i], k.r[i]);
}

// x += alpha p + omega s; r = s - omega t, with <b, r> and max |r|.
__global__ void __launch_bounds__(kThreads) k_kr_x(KrylovArgs k) {
    if (kr_done(k)) return;
    const float alpha = (float)k.kc->alpha, omega = (float)k.kc->omega;
    float d0 = 0.0f, mx = 0.0f;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < k.n; i += gridDim.x * kThreads) {
        const float s = k.s[i];
        k.x[i] += fmaf(alpha, k.p[i], omega * s);
        const float r = fmaf(-omega, k.t[i], s);
        k.r[i] = r;
        d0 = fmaf(k.b[i], r, d0);
        mx = fmaxf(mx, fabsf(r));
    }
    kr_finish<kThreads>(k, kKrX, d0, 0.0f, mx);
}

int krylov_correct(Mdp* m, const int32_t* pi, const float* b, float* x, double target, long long max_iter,
                   cudaStream_t st, long long* products, bool* converged) {
    *products = 0;
    *converged = false;
    const size_t S = (size_t)m->S;
    KrylovCtl& h = *m->kctl_host;
    memset(&h, 0, sizeof(KrylovCtl));
    h.target = target;
    h.max_iter = (int)std::min<long long>(std::max<long long>(max_iter, 1), 1 << 30);
    VC_CUDA(cudaMemcpyAsync(m->kctl, &h, sizeof(KrylovCtl), cudaMemcpyHostToDevice, st));
    KrylovArgs k;
    k.kc = m->kctl;
    k.ctl = m->ctl;
    k.part = m->kr_part;
    k.b = b;
    k.x = x;
    k.r = m->kr;
    k.p = m->kr + S;
    k.v = m->kr + 2 * S;
    k.s = m->kr + 3 * S;
    k.t = m->kr + 4 * S;
    k.n = m->S;
    const int g = state_grid(m);
    count_launches(1);
    k_kr_init<<<g, kThreads, 0, st>>>(k);
    VC_CUDA(cudaGetLastError());
    int rc;
    long long chunk = 4;
    float r_prev = -1.0f;
    for (;;) {
        for (long long i = 0; i < chunk; i++) {
            count_launches(3);
            k_kr_p<<<g, kThreads, 0, st>>>(k);
            if ((rc = launch_apply32(m, pi, k.p, k.v, b, kKrV, k, st))) return rc;
            k_kr_s<<<g, kThreads, 0, st>>>(k);
            if ((rc = launch_apply32(m, pi, k.s, k.t, k.s, kKrT, k, st))) return rc;
            k_kr_x<<<g, kThreads, 0, st>>>(k);
            VC_CUDA(cudaGetLastError());
        }
        VC_CUDA(cudaMemcpyAsync(&h, m->kctl, sizeof(KrylovCtl), cudaMemcpyDeviceToHost, st));
        VC_CUDA(cudaStreamSynchronize(st));
        if (h.done) break;
        // next chunk: the iterations the last chunk's rate of decrease predicts (2 .. 64)
        long long next = 2 * chunk;
        if (r_prev > 0.0f && h.rmax > 0.0f && h.rmax < r_prev) {
            const double rate = log((double)h.rmax / r_prev) / (double)chunk;  // < 0
            next = (long long)ceil(log(h.target / (double)h.rmax) / rate);
        }
        r_prev = h.rmax;
        chunk = std::min<long long>(std::max<long long>(next, 2), 64);
        chunk = std::min<long long>(chunk, (long long)h.max_iter - h.iter);
        if (chunk < 1) chunk = 1;
    }
    *products = 2LL * h.iter;
    *converged = (h.done == 1);
    return VC_OK;
}

}  // namespace vc
