// vc_grad.cu -- adjoint gradient of J = rho . V_pi with respect to the model parameters
// theta = (lambda, mu_1..mu_H, delta_1..delta_H, f, w_occ, w_loss, w_q).
//
// For a fixed policy pi, V = R_pi + gamma P_pi V, so
//     dJ/dtheta_i = lam . (dR_pi/dtheta_i + gamma (dP_pi/dtheta_i) V),
//     (I - gamma P_pi)^T lam = rho.
// lam is found by pull sweeps over an explicit transpose P_pi^T (rows = targets, entries
// sorted by source so every sweep sums in one fixed order), FP32 sweeps refined in FP64
// like the forward solve.  The contraction regenerates every event of each state's
// post-decision state and differentiates its probability rate/Lam analytically:
// d(rate/Lam) = drate/Lam - rate dLam/Lam^2, the self-loop taking minus the others, so
// sum_s' dP V = sum_e dp_e (V(y_e) - V(x)).  Partial sums reduce per block and then in
// block order, so the result is reproducible bit for bit.
#include <math.h>

#include "vc_internal.cuh"

namespace vc {

// ------------------------------------------------------------- transpose of P_pi
__global__ void k_adj_count(Model md, Rates rt, const int32_t* __restrict__ pi, int32_t* __restrict__ cnt, int* err) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < md.S; s += gridDim.x * blockDim.x) {
        int cols[kMaxRow];
        double probs[kMaxRow], R;
        const int n = model_row(md, rt, s, pi[s], cols, probs, &R);
        if (n < 0) {
            atomicOr(err, kErrInfeasiblePolicy);
            continue;
        }
        for (int j = 0; j < n; j++) atomicAdd(&cnt[cols[j]], 1);
    }
}

__global__ void k_adj_fill(Model md, Rates rt, const int32_t* __restrict__ pi, const int64_t* __restrict__ rowT,
                           int32_t* __restrict__ fillpos, int32_t* __restrict__ colT, float* __restrict__ valT,
                           double* __restrict__ valT64) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < md.S; s += gridDim.x * blockDim.x) {
        int cols[kMaxRow];
        double probs[kMaxRow], R;
        const int n = model_row(md, rt, s, pi[s], cols, probs, &R);
        for (int j = 0; j < n; j++) {
            const int y = cols[j];
            const int64_t slot = rowT[y] + atomicAdd(&fillpos[y], 1);
            colT[slot] = s;
            valT[slot] = (float)probs[j];
            valT64[slot] = probs[j];
        }
    }
}

// Orders each transposed row by source state (insertion sort; in-degrees are small).
__global__ void k_adj_sort(int S, const int64_t* __restrict__ rowT, int32_t* __restrict__ colT,
                           float* __restrict__ valT, double* __restrict__ valT64) {
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < S; y += gridDim.x * blockDim.x) {
        const int64_t lo = rowT[y], hi = rowT[y + 1];
        for (int64_t i = lo + 1; i < hi; i++) {
            const int c = colT[i];
            const float v = valT[i];
            const double v64 = valT64[i];
            int64_t j = i - 1;
            while (j >= lo && colT[j] > c) {
                colT[j + 1] = colT[j];
                valT[j + 1] = valT[j];
                valT64[j + 1] = valT64[j];
                j--;
            }
            colT[j + 1] = c;
            valT[j + 1] = v;
            valT64[j + 1] = v64;
        }
    }
}

// FP64 residual of the adjoint system r = rho + gamma P^T lam - lam (stored as float);
// max |r| into the control block's certificate slot.
__global__ void __launch_bounds__(kThreads) k_adj_resid64(int S, double gamma, const int64_t* __restrict__ rowT,
                                                          const int32_t* __restrict__ colT,
                                                          const double* __restrict__ valT64,
                                                          const double* __restrict__ rho,
                                                          const double* __restrict__ lam, float* __restrict__ r,
                                                          SweepCtl sc) {
    double res = 0.0;
    for (int y = blockIdx.x * kThreads + threadIdx.x; y < S; y += gridDim.x * kThreads) {
        double acc = 0.0;
        for (int64_t j = rowT[y]; j < rowT[y + 1]; j++) acc += valT64[j] * lam[colT[j]];
        const double v = rho[y] + gamma * acc - lam[y];
        r[y] = (float)v;
        res = fmax(res, fabs(v));
    }
    res = block_max<double, kThreads>(res);
    finish_block<double>(sc, res, 0.0, 0);
}

__global__ void k_f64_to_f32(const double* __restrict__ in, float* __restrict__ out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = (float)in[i];
}

// ------------------------------------------------------------------ contraction
// Per state s with x = x_pi(s): lam(s) * (dR(x)/dtheta + gamma sum_e dp_e (V(y_e) - V(x))),
// and rho(s) V(s) for J, in slots 0..2H+4 and 2*MH+5 of a per-block partial row.
template <int MH>
__global__ void __launch_bounds__(kThreads) k_grad_contract(Model md, Rates rt, double gamma,
                                                            const int32_t* __restrict__ pi,
                                                            const double* __restrict__ V,
                                                            const double* __restrict__ lam,
                                                            const double* __restrict__ rho,
                                                            double* __restrict__ partial) {
    constexpr int NT = 2 * MH + 6;  // theta slots (2H+5 used) + J
    double g[NT];
#pragma unroll
    for (int i = 0; i < NT; i++) g[i] = 0.0;
    const int H = md.H;
    const double Lam = rt.Lam, Lam2 = rt.Lam * rt.Lam;
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < md.S; s += gridDim.x * kThreads) {
        Digits d;
        decode<MH>(md, s, d);
        int x = s;
        if (!apply_action<MH>(md, s, pi[s], d, x)) continue;  // rejected by the count kernel
        const double vx = V[x];
        double dVc[MH], dVd[MH];
        double D = 0.0, L = 0.0;
        int occ_sum = 0;
#pragma unroll
        for (int k = 0; k < MH; k++) {
            dVc[k] = 0.0;
            dVd[k] = 0.0;
            if (k < H) {
                const int o = d.occ[k];
                if (o > 0) {
                    dVc[k] = V[x - md.stride[k]] - vx;
                    dVd[k] = V[x - o * md.stride[k]] - vx;
                }
                D += rt.mu[k] * o * dVc[k] + rt.delta[k] * dVd[k];
                L += rt.delta[k] * o;
                occ_sum += o;
            }
        }
        const bool full = d.q >= md.Q;
        const double dVa = full ? 0.0 : V[x + 2] - vx;
        D += rt.lambda * dVa;
        if (full) L += rt.lambda;
        const double dVf = V[d.ph ? x - 1 : x + 1] - vx;
        D += (d.ph ? 1.0 - rt.f : rt.f) * dVf;
        const double w = lam[s];
        // lambda
        g[0] += w * (rt.w_loss * ((full ? 1.0 : 0.0) / Lam - L / Lam2) + gamma * (dVa / Lam - D / Lam2));
#pragma unroll
        for (int k = 0; k < MH; k++) {
            if (k < H) {
                const int o = d.occ[k];
                g[1 + k] += w * (-rt.w_loss * L * md.C / Lam2 + gamma * (o * dVc[k] / Lam - md.C * D / Lam2));
                g[1 + MH + k] += w * (rt.w_loss * (o / Lam - L / Lam2) + gamma * (dVd[k] / Lam - D / Lam2));
            }
        }
        g[1 + 2 * MH] += w * gamma * (d.ph ? -dVf : dVf) / Lam;  // f
        g[2 + 2 * MH] += w * occ_sum;                            // w_occ
        g[3 + 2 * MH] += w * L / Lam;                            // w_loss
        g[4 + 2 * MH] += w * d.q;                                // w_q
        g[5 + 2 * MH] += rho[s] * V[s];                          // J
    }
    // block reduction, fixed order: warp shuffles, then warps in index order
    __shared__ double part[kThreads / 32][NT];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < NT; i++) {
        double v = g[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) part[wid][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < NT) {
        double v = 0.0;
        for (int w2 = 0; w2 < kThreads / 32; w2++) v += part[w2][threadIdx.x];
        partial[(size_t)blockIdx.x * NT + threadIdx.x] = v;
    }
}

// Sums the per-block rows in block order and maps the MH-strided slots to the packed
// theta order (lambda, mu_0..mu_{H-1}, delta_0..delta_{H-1}, f, w_occ, w_loss, w_q), J.
__global__ void k_grad_final(const double* __restrict__ partial, int nblocks, int MH, int H, double* __restrict__ out) {
    const int NT = 2 * MH + 6;
    const int i = threadIdx.x;
    if (i >= 2 * H + 6) return;
    int src;
    if (i == 0)
        src = 0;
    else if (i <= H)
        src = i;  // mu_{i-1}
    else if (i <= 2 * H)
        src = 1 + MH + (i - 1 - H);  // delta
    else
        src = 1 + 2 * MH + (i - 1 - 2 * H);  // f, w_occ, w_loss, w_q, J
    double v = 0.0;
    for (int b = 0; b < nblocks; b++) v += partial[(size_t)b * NT + src];
    out[i] = v;
}


// J = rho . V in FP64 by one block: each thread sums its strided states in index order,
// then the block halves the partials in a fixed tree, so the result is reproducible bit
// for bit (one block suffices: the objective is read once per solve).
__global__ void __launch_bounds__(1024) k_objective(const double* __restrict__ V, const double* __restrict__ rho,
                                                   long long S, double* __restrict__ J) {
    __shared__ double part[1024];
    double acc = 0.0;
    for (long long s = threadIdx.x; s < S; s += 1024) acc = fma(rho[s], V[s], acc);
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *J = part[0];
}

// ------------------------------------------------------------------------ launchers
int launch_adj_count(Mdp* m, const int32_t* pi, int32_t* cnt, int* err, cudaStream_t st) {
    count_launches(1);
    k_adj_count<<<state_grid(m), kThreads, 0, st>>>(m->md, m->rates, pi, cnt, err);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int launch_adj_fill(Mdp* m, const int32_t* pi, const int64_t* rowT, int32_t* fillpos, int32_t* colT, float* valT,
                    double* valT64, cudaStream_t st) {
    count_launches(2);
    k_adj_fill<<<state_grid(m), kThreads, 0, st>>>(m->md, m->rates, pi, rowT, fillpos, colT, valT, valT64);
    k_adj_sort<<<state_grid(m), kThreads, 0, st>>>(m->S, rowT, colT, valT, valT64);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int launch_adj_resid64(Mdp* m, const int64_t* rowT, const int32_t* colT, const double* valT64, const double* rho,
                       const double* lam, float* r, SweepCtl sc, cudaStream_t st) {
    count_launches(1);
    k_adj_resid64<<<state_grid(m), kThreads, 0, st>>>(m->S, m->gamma, rowT, colT, valT64, rho, lam, r, sc);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int launch_f64_to_f32(const double* in, float* out, int n, cudaStream_t st) {
    count_launches(1);
    const int b = (n + kThreads - 1) / kThreads;
    k_f64_to_f32<<<b < 4096 ? (b > 0 ? b : 1) : 4096, kThreads, 0, st>>>(in, out, n);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int grad_partial_stride(const Mdp* m) { return 2 * (m->md.H <= 4 ? 4 : m->md.H <= 8 ? 8 : 16) + 6; }

int launch_grad_contract(Mdp* m, const int32_t* pi, const double* V, const double* lam, const double* rho,
                         double* partial, double* out, cudaStream_t st) {
    const int g = state_grid(m);
    const int MH = m->md.H <= 4 ? 4 : m->md.H <= 8 ? 8 : 16;
    count_launches(2);
    if (MH == 4)
        k_grad_contract<4><<<g, kThreads, 0, st>>>(m->md, m->rates, m->gamma, pi, V, lam, rho, partial);
    else if (MH == 8)
        k_grad_contract<8><<<g, kThreads, 0, st>>>(m->md, m->rates, m->gamma, pi, V, lam, rho, partial);
    else
        k_grad_contract<16><<<g, kThreads, 0, st>>>(m->md, m->rates, m->gamma, pi, V, lam, rho, partial);
    k_grad_final<<<1, 64, 0, st>>>(partial, g, MH, m->md.H, out);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int launch_objective(const double* V, const double* rho, long long S, double* J, cudaStream_t st) {
    count_launches(1);
    k_objective<<<1, 1024, 0, st>>>(V, rho, S, J);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

}  // namespace vc

// The objective of the gradient entry point, exported on its own: J = rho . V.
extern "C" int vc_objective(const double* V, const double* rho, int64_t S, double* J, void* stream) {
    vc::set_error("");
    if (!V || !rho || !J) return vc::fail(VC_ERR_ARG, "vc_objective: NULL argument");
    if (S < 1) return vc::fail(VC_ERR_ARG, "vc_objective: S < 1");
    return vc::launch_objective(V, rho, (long long)S, J, (cudaStream_t)stream);
}
