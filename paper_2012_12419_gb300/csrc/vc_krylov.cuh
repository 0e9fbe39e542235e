// vc_krylov.cuh -- device side of the BiCGSTAB correction solve of the refinement.
//
// The mixed-precision refinement solves, for a fixed policy pi, the correction equation
// (I - gamma P_pi) e = r, where r = T_pi V64 - V64 is the FP64 policy residual stored in
// FP32.  Plain fixed-point sweeps e <- r + gamma P_pi e converge at rate gamma per sweep;
// BiCGSTAB (H. A. van der Vorst, SIAM J. Sci. Stat. Comput. 13(2), 1992), unpreconditioned,
// in FP32, reaches the same stopping test (max |r - (I - gamma P_pi) e| below the target)
// with fewer products by the matrix on these uniformised chains.
//
// One iteration is five kernels: p update, v = A p (with <b, v>), s = r - alpha v,
// t = A s (with <t, s>, <t, t>), and the x / r update (with <b, r> and max |r|).  Every
// reducing kernel writes one partial per block; the last block to arrive sums the
// partials in block order (deterministic) and advances the scalars in the control block,
// so the host only reads the control block between chunks of iterations.  Every kernel
// returns at once after the control block says done.
#pragma once

#include "vc_internal.cuh"

namespace vc {

struct KrylovCtl {
    double rho;       // <b, r> of the current residual (b is the shadow residual)
    double alpha, omega, beta;
    double target;    // stop once max |r| < target (raised to 2^-18 max |b| by the first kernel)
    double dots[2];   // dot products of the last reducing kernel
    float rmax;       // max |r| after the last iteration
    int done;         // 0 running, 1 converged, 2 iteration cap, 5 breakdown
    int iter, max_iter;
    unsigned int ticket;
    int pad_;
};

enum KrylovStage : int { kKrInit = 0, kKrV = 1, kKrT = 2, kKrX = 3 };

// Vectors of one solve (FP32, n entries each) and the reduction scratch.
struct KrylovArgs {
    KrylovCtl* kc;
    Ctl* ctl;         // the handle's control block (error flags of the bounds-checking build)
    double* part;     // [3][gridDim.x]: two partial sums and a partial max per block
    const float* b;   // right-hand side and shadow residual
    float *x, *r, *p, *v, *s, *t;
    int n;
};

__device__ __forceinline__ bool kr_done(const KrylovArgs& k) { return *((volatile int*)&k.kc->done) != 0; }

// Block-wide sum over NT threads in a fixed order; result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double part[NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) part[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (l < NT / 32) ? part[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

// Scalars of the stage, from the grid totals (thread 0 of the last block).
__device__ inline void kr_advance(KrylovCtl* c, int stage, double d0, double d1, double mx) {
    c->dots[0] = d0;
    c->dots[1] = d1;
    if (stage == kKrInit) {
        c->rho = d0;  // <b, r0> with r0 = b
        c->rmax = (float)mx;
        // one FP32 solve reduces the residual by 2^-18 at most (the refinement's next
        // FP64 round takes it further), so the target never asks for more
        c->target = fmax(c->target, ldexp(mx, -18));
        c->alpha = c->omega = 1.0;
        c->beta = 0.0;
        c->iter = 0;
        if (mx < c->target) c->done = 1;
        else if (!(d0 > 0.0)) c->done = 5;
    } else if (stage == kKrV) {
        // alpha = rho / <b, v>
        if (d0 == 0.0 || !isfinite(d0)) {
            c->done = 5;
        } else {
            c->alpha = c->rho / d0;
        }
    } else if (stage == kKrT) {
        // omega = <t, s> / <t, t>; t = 0 means s = 0 (A is non-singular): omega = 0 and
        // the x / r update below ends the solve with r = s = 0
        c->omega = (d1 > 0.0) ? d0 / d1 : 0.0;
        if (!isfinite(c->omega)) c->done = 5;
    } else {
        // after x += alpha p + omega s, r = s - omega t
        c->rmax = (float)mx;
        c->iter += 1;
        if (mx < c->target) {
            c->done = 1;
        } else if (c->iter >= c->max_iter) {
            c->done = 2;
        } else if (c->omega == 0.0 || c->rho == 0.0 || !isfinite(mx)) {
            c->done = 5;
        } else {
            c->beta = (d0 / c->rho) * (c->alpha / c->omega);
            c->rho = d0;
            if (!isfinite(c->beta) || d0 == 0.0) c->done = 5;
        }
    }
    c->ticket = 0;
    __threadfence();
}

// Every thread of every block calls this once at the end of a reducing kernel with its
// partial sums d0, d1 and partial max mx.
template <int NT>
__device__ void kr_finish(const KrylovArgs& k, int stage, float d0, float d1, float mx) {
    __shared__ int last;
    const double s0 = block_sum<NT>((double)d0);
    const double s1 = block_sum<NT>((double)d1);
    const float m = block_max<float, NT>(mx);
    const int G = (int)gridDim.x;
    if (threadIdx.x == 0) {
        k.part[blockIdx.x] = s0;
        k.part[G + blockIdx.x] = s1;
        k.part[2 * G + blockIdx.x] = (double)m;
        __threadfence();
        last = (atomicAdd(&k.kc->ticket, 1u) == (unsigned)G - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a0 = 0.0, a1 = 0.0, am = 0.0;
    for (int i = threadIdx.x; i < G; i += NT) {
        a0 += __ldcg(k.part + i);
        a1 += __ldcg(k.part + G + i);
        am = fmax(am, __ldcg(k.part + 2 * G + i));
    }
    a0 = block_sum<NT>(a0);
    a1 = block_sum<NT>(a1);
    am = block_max<double, NT>(am);
    if (threadIdx.x == 0) kr_advance(k.kc, stage, a0, a1, am);
}

// Product by the correction matrix, y = x - gamma P_pi x, fused with the partial sums
// <w, y> and <y, y> of `stage` (vc_sweep.cu: implicit model; vc_csr.cu: stored rows).
int launch_apply32(Mdp* m, const int32_t* pi, const float* x, float* y, const float* w, int stage,
                   const KrylovArgs& k, cudaStream_t st);
int csr_apply32(Mdp* m, const int32_t* pi, const float* x, float* y, const float* w, int stage,
                const KrylovArgs& k, cudaStream_t st);

// BiCGSTAB solve of (I - gamma P_pi) x = b from x = 0 until max |b - (I - gamma P_pi) x|
// (the recurrence residual) is below target or max_iter iterations; *products counts the
// products by the matrix, *converged reports whether the target was met (a breakdown or
// the iteration cap leave it false; the caller then falls back to fixed-point sweeps).
int krylov_correct(Mdp* m, const int32_t* pi, const float* b, float* x, double target, long long max_iter,
                   cudaStream_t st, long long* products, bool* converged);

}  // namespace vc
