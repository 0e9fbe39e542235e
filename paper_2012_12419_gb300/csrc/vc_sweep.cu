// vc_sweep.cu -- Bellman sweep kernels (Algorithm 3, step 2, with the Eq. 18 backup):
//
//  * implicit form: successors generated in registers from the mixed-radix state code.
//    A sweep is two passes over the state space.  Pass 1 evaluates, for every state x
//    read as a post-decision state, U(x) = R(x) + gamma * sum_e p_e V(y_e) over the at
//    most 2H+3 uniformised events (reward and probabilities depend on x only).  Pass 2
//    takes V'(s) = max over feasible a of U(x_a(s)), x_a the state after placing on
//    host a (or s itself for defer).  This is the same backup as Eq. 18 with
//    (2H+3) + A gathers per state instead of A * (2H+3).
//  * explicit CSR form: warp per state, G lanes per row, rows of a state reduced with
//    warp shuffles (sum within a row, top-2 max/argmax across rows).
//
// Every V-producing kernel fuses the residual max|V' - V| (warp -> block -> one atomicMax
// per block on the non-negative float bits, order independent) and, in loop mode, the
// convergence bookkeeping of the last block to finish (ticket counter), so the host
// never reads the residual per sweep.
#include <math.h>

#include "vc_internal.cuh"

namespace vc {

constexpr int kThreads = 256;

// ------------------------------------------------------------------ sweep bookkeeping
__device__ __forceinline__ bool loop_done(const SweepCtl& sc) {
    if (sc.mode != kModeLoop32 && sc.mode != kModeLoop64) return false;
    return *((volatile int*)&sc.ctl->done) != 0;
}

__device__ __forceinline__ long long loop_sweep(const SweepCtl& sc) {
    return *((volatile long long*)&sc.ctl->sweeps);
}

// Called by every block after its residual is known (res, vmax valid in thread 0).
template <typename T>
__device__ void finish_block(const SweepCtl& sc, T res, T vmax, long long sweep) {
    if (threadIdx.x != 0 || sc.mode == kModeNone) return;
    Ctl* c = sc.ctl;
    if (sc.mode == kModeCert64) {
        atomicMax(&c->cert64, dbits((double)res));
        return;
    }
    const int slot = (int)(sweep % kRing);
    if (sc.mode == kModeLoop32) {
        atomicMax(&c->res32[slot], fbits((float)res));
        atomicMax(&c->vmax32[slot], fbits((float)vmax));
    } else {
        atomicMax(&c->res64[slot], dbits((double)res));
    }
    __threadfence();
    const unsigned int t = atomicAdd(&c->ticket, 1u);
    if (t != gridDim.x - 1) return;
    // last block of this sweep: all residual atomics are visible
    __threadfence();
    const long long k = sweep + 1;
    c->ticket = 0;
    c->sweeps = k;
    c->final_buf = sc.out_index;
    const int next = (int)(k % kRing);
    int done = 0;
    if (sc.mode == kModeLoop32) {
        const float r = __uint_as_float(*((volatile unsigned int*)&c->res32[slot]));
        const float vm = __uint_as_float(*((volatile unsigned int*)&c->vmax32[slot]));
        c->res32[next] = 0u;
        c->vmax32[next] = 0u;
        int e = 0;
        frexpf(vm, &e);
        const double ulp = (vm > 0.0f) ? ldexp(1.0, e - 24) : 0.0;
        const double tol_eff = fmax(c->tol, 4.0 * ulp);
        if ((double)r < tol_eff) {
            done = 1;
        } else if (r < c->best_res) {
            c->best_res = r;
            c->since_best = 0;
        } else if (++c->since_best >= kStallSweeps) {
            done = 3;
        }
    } else {
        const double r = __longlong_as_double((long long)*((volatile unsigned long long*)&c->res64[slot]));
        c->res64[next] = 0ull;
        if (r < c->tol) done = 1;
    }
    if (!done && k >= c->max_sweeps) done = 2;
    c->done = done;
    __threadfence();
}

// ---------------------------------------------------------------- implicit: pass 1
// U(x) = R(x) + gamma * (V(x) + sum_e p_e (V(y_e) - V(x))): the self-loop probability is
// never formed, so rounding scales with the value differences, not with |V|.
template <typename T>
__device__ __forceinline__ T post_value(const Model& md, const Coef<T>& c, const T* __restrict__ V, int x,
                                        const Digits& d) {
    const T vx = V[x];
    T acc = T(0), loss = T(0);
    int occ_sum = 0;
#pragma unroll
    for (int k = 0; k < kMaxH; k++) {
        if (k < md.H) {
            const int o = d.occ[k];
            if (o > 0) {
                const T v1 = V[x - md.stride[k]];
                if (o == 1) {
                    acc += (c.pc[k] + c.pd[k]) * (v1 - vx);
                } else {
                    const T v0 = V[x - o * md.stride[k]];
                    acc += c.pc[k] * T(o) * (v1 - vx) + c.pd[k] * (v0 - vx);
                }
                occ_sum += o;
                loss += c.lossd[k] * T(o);
            }
        }
    }
    if (d.q < md.Q)
        acc += c.pa * (V[x + 2] - vx);
    else
        loss += c.lossa;
    const T vf = V[d.ph ? x - 1 : x + 1];
    acc += (d.ph ? c.pf1 : c.pf0) * (vf - vx);
    const T R = c.w_occ * T(occ_sum) + c.w_q * T(d.q) + loss;
    return R + c.gamma * (vx + acc);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_post(Model md, Coef<T> c, const T* __restrict__ V, T* __restrict__ U,
                                                   SweepCtl sc) {
    if (loop_done(sc)) return;
    const int x = blockIdx.x * kThreads + threadIdx.x;
    if (x >= md.S) return;
    Digits d;
    decode(md, x, d);
    U[x] = post_value(md, c, V, x, d);
}

// ---------------------------------------------------------------- implicit: pass 2
template <typename T>
__global__ void __launch_bounds__(kThreads) k_max(Model md, const T* __restrict__ U, const T* __restrict__ V_in,
                                                  T* __restrict__ V_out, int32_t* __restrict__ pi,
                                                  T* __restrict__ qgap, SweepCtl sc) {
    if (loop_done(sc)) return;
    const long long sweep = (sc.mode == kModeLoop32 || sc.mode == kModeLoop64) ? loop_sweep(sc) : 0;
    const int s = blockIdx.x * kThreads + threadIdx.x;
    T res = T(0), vabs = T(0);
    if (s < md.S) {
        Digits d;
        decode(md, s, d);
        T best = -INFINITY, second = -INFINITY;
        int arg = md.H;
        if (d.q >= 1) {
#pragma unroll
            for (int k = 0; k < kMaxH; k++) {
                if (k < md.H && d.occ[k] < md.C && (k == md.H - 1 || d.ph == 1)) {
                    const T u = U[s + md.stride[k] - 2];
                    if (u > best) {
                        second = best;
                        best = u;
                        arg = k;
                    } else if (u > second) {
                        second = u;
                    }
                }
            }
        }
        const T u = U[s];  // defer: the post-decision state is s itself
        if (u > best) {
            second = best;
            best = u;
            arg = md.H;
        } else if (u > second) {
            second = u;
        }
        if (V_out) V_out[s] = best;
        if (pi) pi[s] = arg;
        if (qgap) qgap[s] = (second == -INFINITY) ? T(INFINITY) : best - second;
        res = fabs(best - V_in[s]);
        vabs = fabs(best);
        if (sc.mode == kModeCert64 && sc.pi_ref && sc.pi_ref[s] != arg) atomicAdd(&sc.ctl->changes, 1ull);
    }
    if (sc.mode == kModeNone) return;
    res = block_max<T, kThreads>(res);
    __syncthreads();
    vabs = block_max<T, kThreads>(vabs);
    finish_block<T>(sc, res, vabs, sweep);
}

// --------------------------------------------------- implicit: policy evaluation sweep
template <typename T>
__global__ void __launch_bounds__(kThreads) k_eval(Model md, Coef<T> c, const int32_t* __restrict__ pi,
                                                   const T* __restrict__ V_in, T* __restrict__ V_out, SweepCtl sc) {
    if (loop_done(sc)) return;
    const long long sweep = (sc.mode == kModeLoop64) ? loop_sweep(sc) : 0;
    const int s = blockIdx.x * kThreads + threadIdx.x;
    T res = T(0);
    if (s < md.S) {
        Digits d;
        decode(md, s, d);
        const int a = pi[s];
        int x = s;
        bool ok = (a >= 0 && a <= md.H);
        if (ok && a < md.H) {
            ok = d.q >= 1 && d.occ[a] < md.C && (a == md.H - 1 || d.ph == 1);
            if (ok) {
                d.occ[a] += 1;
                d.q -= 1;
                x = s + md.stride[a] - 2;
            }
        }
        if (!ok) {
            atomicOr(&sc.ctl->error, kErrInfeasiblePolicy);
            V_out[s] = V_in[s];
        } else {
            const T v = post_value(md, c, V_in, x, d);
            V_out[s] = v;
            res = fabs(v - V_in[s]);
        }
    }
    if (sc.mode == kModeNone) return;
    res = block_max<T, kThreads>(res);
    finish_block<T>(sc, res, T(0), sweep);
}

// ----------------------------------------------------------------------- explicit CSR
template <typename VT>
__device__ __forceinline__ float load_val(const VT* __restrict__ v, int64_t j);
template <>
__device__ __forceinline__ float load_val<float>(const float* __restrict__ v, int64_t j) {
    return __ldg(v + j);
}
template <>
__device__ __forceinline__ float load_val<uint16_t>(const uint16_t* __restrict__ v, int64_t j) {
    return __uint_as_float((uint32_t)__ldg(v + j) << 16);
}

// Warp per state, G lanes per row, 32/G rows of the state in flight per step.  Row sums
// reduce within their G-lane group; Q values reduce across groups to (best, argmax with
// the lowest action on ties, second best).
template <typename VT, int G>
__global__ void __launch_bounds__(kThreads) k_csr32(int S, int A, float gamma, const int64_t* __restrict__ row_ptr,
                                                    const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                    const float* __restrict__ scale, const float* __restrict__ R,
                                                    const float* __restrict__ V_in, float* __restrict__ V_out,
                                                    int32_t* __restrict__ pi, float* __restrict__ qgap, SweepCtl sc) {
    if (loop_done(sc)) return;
    const long long sweep = (sc.mode == kModeLoop32) ? loop_sweep(sc) : 0;
    constexpr int RPI = 32 / G;
    const int lane = threadIdx.x & 31;
    const int sub = lane % G, grp = lane / G;
    const int warp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * kThreads) >> 5;
    float res = 0.0f, vabs = 0.0f;
    for (int s = warp; s < S; s += nwarps) {
        float best = -INFINITY, second = -INFINITY;
        int arg = -1;
        const int64_t rbase = (int64_t)s * A;
        for (int a0 = 0; a0 < A; a0 += RPI) {
            const int a = a0 + grp;
            float acc = 0.0f;
            int64_t r = rbase + a;
            if (a < A) {
                const int64_t lo = __ldg(row_ptr + r), hi = __ldg(row_ptr + r + 1);
                for (int64_t j = lo + sub; j < hi; j += G) acc += load_val<VT>(val, j) * __ldg(V_in + __ldg(col + j));
            }
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            float q = -INFINITY;
            if (a < A) {
                const float rr = __ldg(R + r);
                if (rr != -INFINITY) q = rr + gamma * (scale ? __ldg(scale + r) * acc : acc);
            }
            float b1 = q, b2 = -INFINITY;
            int ia = (a < A) ? a : 0x7fffffff;
#pragma unroll
            for (int o = G; o < 32; o <<= 1) {
                const float ob1 = __shfl_xor_sync(0xffffffffu, b1, o);
                const float ob2 = __shfl_xor_sync(0xffffffffu, b2, o);
                const int oia = __shfl_xor_sync(0xffffffffu, ia, o);
                const bool take = (ob1 > b1) || (ob1 == b1 && oia < ia);
                const float nb2 = fmaxf(fmaxf(b2, ob2), take ? b1 : ob1);
                b1 = take ? ob1 : b1;
                ia = take ? oia : ia;
                b2 = nb2;
            }
            // chunks arrive in increasing action order: strict > keeps the lowest action
            if (b1 > best) {
                second = fmaxf(best, b2);
                best = b1;
                arg = ia;
            } else {
                second = fmaxf(second, b1);
            }
        }
        if (lane == 0) {
            if (V_out) V_out[s] = best;
            if (pi) pi[s] = arg;
            if (qgap) qgap[s] = (second == -INFINITY) ? INFINITY : best - second;
        }
        res = fmaxf(res, fabsf(best - __ldg(V_in + s)));
        vabs = fmaxf(vabs, fabsf(best));
    }
    if (sc.mode == kModeNone) return;
    res = block_max<float, kThreads>(res);
    __syncthreads();
    vabs = block_max<float, kThreads>(vabs);
    finish_block<float>(sc, res, vabs, sweep);
}

// FP64 backups on a stored CSR (handles built from a user matrix): thread per state.
template <typename VT>
__device__ __forceinline__ double load_val64(const VT* __restrict__ v, int64_t j) {
    return (double)load_val<VT>(v, j);
}

template <typename VT>
__global__ void __launch_bounds__(kThreads) k_csr_bellman64(int S, int A, double gamma,
                                                            const int64_t* __restrict__ row_ptr,
                                                            const int32_t* __restrict__ col,
                                                            const VT* __restrict__ val, const float* __restrict__ scale,
                                                            const float* __restrict__ R, const double* __restrict__ V_in,
                                                            double* __restrict__ V_out, int32_t* __restrict__ pi,
                                                            double* __restrict__ qgap, SweepCtl sc) {
    const int s = blockIdx.x * kThreads + threadIdx.x;
    double res = 0.0;
    if (s < S) {
        double best = -INFINITY, second = -INFINITY;
        int arg = -1;
        for (int a = 0; a < A; a++) {
            const int64_t r = (int64_t)s * A + a;
            const float rr = R[r];
            if (rr == -INFINITY) continue;
            double acc = 0.0;
            for (int64_t j = row_ptr[r]; j < row_ptr[r + 1]; j++) acc += load_val64<VT>(val, j) * V_in[col[j]];
            if (scale) acc *= (double)scale[r];
            const double qv = (double)rr + gamma * acc;
            if (qv > best) {
                second = best;
                best = qv;
                arg = a;
            } else if (qv > second) {
                second = qv;
            }
        }
        if (V_out) V_out[s] = best;
        if (pi) pi[s] = arg;
        if (qgap) qgap[s] = (second == -INFINITY) ? INFINITY : best - second;
        res = fabs(best - V_in[s]);
        if (sc.mode == kModeCert64 && sc.pi_ref && sc.pi_ref[s] != arg) atomicAdd(&sc.ctl->changes, 1ull);
    }
    if (sc.mode == kModeNone) return;
    res = block_max<double, kThreads>(res);
    finish_block<double>(sc, res, 0.0, 0);
}

template <typename VT>
__global__ void __launch_bounds__(kThreads) k_csr_eval64(int S, int A, double gamma, const int64_t* __restrict__ row_ptr,
                                                         const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                         const float* __restrict__ scale, const float* __restrict__ R,
                                                         const int32_t* __restrict__ pi, const double* __restrict__ V_in,
                                                         double* __restrict__ V_out, SweepCtl sc) {
    if (loop_done(sc)) return;
    const long long sweep = (sc.mode == kModeLoop64) ? loop_sweep(sc) : 0;
    const int s = blockIdx.x * kThreads + threadIdx.x;
    double res = 0.0;
    if (s < S) {
        const int a = pi[s];
        const int64_t r = (int64_t)s * A + a;
        const float rr = (a >= 0 && a < A) ? R[r] : -INFINITY;
        if (rr == -INFINITY) {
            atomicOr(&sc.ctl->error, kErrInfeasiblePolicy);
            V_out[s] = V_in[s];
        } else {
            double acc = 0.0;
            for (int64_t j = row_ptr[r]; j < row_ptr[r + 1]; j++) acc += load_val64<VT>(val, j) * V_in[col[j]];
            if (scale) acc *= (double)scale[r];
            const double v = (double)rr + gamma * acc;
            V_out[s] = v;
            res = fabs(v - V_in[s]);
        }
    }
    if (sc.mode == kModeNone) return;
    res = block_max<double, kThreads>(res);
    finish_block<double>(sc, res, 0.0, sweep);
}

__global__ void k_f32_to_f64(const float* __restrict__ in, double* __restrict__ out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}

// ------------------------------------------------------------------------ launchers
static inline unsigned blocks_for(int n) { return (unsigned)((n + kThreads - 1) / kThreads); }

static int csr_grid(const Mdp* m) {
    // warp per state; enough resident warps to cover the machine several times
    const int per_block = kThreads / 32;
    const long long need = ((long long)m->S + per_block - 1) / per_block;
    const long long cap = (long long)(m->num_sms > 0 ? m->num_sms : 148) * 8 * 4;
    return (int)(need < cap ? need : cap);
}

int launch_sweep32(Mdp* m, const float* V_in, float* V_out, int32_t* pi, float* qgap, SweepCtl sc,
                   cudaStream_t st) {
    const int base = m->fmt & 0xF;
    if (base == VC_IMPLICIT) {
        SweepCtl sc1 = sc;
        if (sc1.mode != kModeLoop32) sc1.mode = kModeNone;
        count_launches(2);
        k_post<float><<<blocks_for(m->S), kThreads, 0, st>>>(m->md, m->c32, V_in, m->U32, sc1);
        k_max<float><<<blocks_for(m->S), kThreads, 0, st>>>(m->md, m->U32, V_in, V_out, pi, qgap, sc);
    } else if (base == VC_CSR_F32) {
        count_launches(1);
        k_csr32<float, 8><<<csr_grid(m), kThreads, 0, st>>>(m->S, m->A, (float)m->gamma, m->row_ptr, m->col,
                                                            (const float*)m->val, nullptr, m->R, V_in, V_out, pi,
                                                            qgap, sc);
    } else {
        count_launches(1);
        k_csr32<uint16_t, 8><<<csr_grid(m), kThreads, 0, st>>>(m->S, m->A, (float)m->gamma, m->row_ptr, m->col,
                                                               (const uint16_t*)m->val, m->scale, m->R, V_in, V_out,
                                                               pi, qgap, sc);
    }
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int launch_bellman64(Mdp* m, const double* V_in, double* V_out, int32_t* pi, double* qgap, SweepCtl sc,
                     cudaStream_t st) {
    if (m->has_model) {
        SweepCtl none = sc;
        none.mode = kModeNone;
        count_launches(2);
        k_post<double><<<blocks_for(m->S), kThreads, 0, st>>>(m->md, m->c64, V_in, m->U64, none);
        k_max<double><<<blocks_for(m->S), kThreads, 0, st>>>(m->md, m->U64, V_in, V_out, pi, qgap, sc);
    } else if ((m->fmt & 0xF) == VC_CSR_BF16) {
        count_launches(1);
        k_csr_bellman64<uint16_t><<<blocks_for(m->S), kThreads, 0, st>>>(m->S, m->A, m->gamma, m->row_ptr, m->col,
                                                                        (const uint16_t*)m->val, m->scale, m->R,
                                                                        V_in, V_out, pi, qgap, sc);
    } else {
        count_launches(1);
        k_csr_bellman64<float><<<blocks_for(m->S), kThreads, 0, st>>>(m->S, m->A, m->gamma, m->row_ptr, m->col,
                                                                     (const float*)m->val, nullptr, m->R, V_in,
                                                                     V_out, pi, qgap, sc);
    }
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int launch_eval64(Mdp* m, const int32_t* pi, const double* V_in, double* V_out, SweepCtl sc, cudaStream_t st) {
    if (m->has_model) {
        count_launches(1);
        k_eval<double><<<blocks_for(m->S), kThreads, 0, st>>>(m->md, m->c64, pi, V_in, V_out, sc);
    } else if ((m->fmt & 0xF) == VC_CSR_BF16) {
        count_launches(1);
        k_csr_eval64<uint16_t><<<blocks_for(m->S), kThreads, 0, st>>>(m->S, m->A, m->gamma, m->row_ptr, m->col,
                                                                     (const uint16_t*)m->val, m->scale, m->R, pi,
                                                                     V_in, V_out, sc);
    } else {
        count_launches(1);
        k_csr_eval64<float><<<blocks_for(m->S), kThreads, 0, st>>>(m->S, m->A, m->gamma, m->row_ptr, m->col,
                                                                  (const float*)m->val, nullptr, m->R, pi, V_in,
                                                                  V_out, sc);
    }
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int launch_f32_to_f64(const float* in, double* out, int n, cudaStream_t st) {
    count_launches(1);
    k_f32_to_f64<<<blocks_for(n), kThreads, 0, st>>>(in, out, n);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

}  // namespace vc
