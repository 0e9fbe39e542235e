// vc_sweep.cu -- implicit-form Bellman kernels (Algorithm 3, step 2, with the Eq. 18
// backup) and the dispatch between the implicit and the explicit CSR forms.
//
// Implicit form: successors generated in registers from the mixed-radix state code.  A
// sweep is two passes over the state space.  Pass 1 evaluates, for every state x read as
// a post-decision state, U(x) = R(x) + gamma * E[V(next) | x] over the at most 2H+3
// uniformised events (reward and probabilities depend on x only).  Pass 2 takes
// V'(s) = max over feasible a of U(x_a(s)), x_a the state after placing on host a (or s
// itself for defer).  This is the Eq. 18 backup with (2H+3) + A gathers per state
// instead of A * (2H+3).
//
// Every V-producing kernel fuses the residual max|V' - V| (warp -> block -> one atomicMax
// per block, order independent) and, in loop mode, the termination test of the last
// block (finish_block), so the host never reads the residual per sweep.  All grids are
// persistent (a few blocks per SM, grid-stride over states) to keep the per-sweep atomics
// on the control block few.  Kernels are instantiated for every H <= 8 and for H <= 16
// (MH) so the per-host loops issue no dead iterations up to 8 hosts.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "vc_internal.cuh"
#include "vc_krylov.cuh"

namespace vc {

int state_grid(const Mdp* m) {
    const long long need = ((long long)m->S + kThreads - 1) / kThreads;
    const long long cap = (long long)(m->num_sms > 0 ? m->num_sms : 148) * 8;
    return (int)(need < cap ? need : cap);
}

// ------------------------------------------------------------------ model arithmetic
// E[V(next) | x] = V(x) + sum_e p_e (V(y_e) - V(x)) from the gathered values (vx = V(x),
// v1 / v0 the completion / departure targets of each host, va the arrival, vf the phase
// flip): the self-loop probability is never formed, so rounding scales with value
// differences, not with |V|.  The sum runs in a fixed order.
template <int MH, typename T>
__device__ __forceinline__ T expect_from(const Model& md, const Coef<T>& c, const Digits& d, T vx, const T* v1,
                                         const T* v0, T va, T vf) {
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < MH; k++) {
        if (k < md.H) {
            const int o = d.occ[k];
            if (o > 0) {
                if (o == 1) {
                    acc += (c.pc[k] + c.pd[k]) * (v1[k] - vx);  // completion and departure both empty the host
                } else {
                    acc += c.pc[k] * T(o) * (v1[k] - vx) + c.pd[k] * (v0[k] - vx);
                }
            }
        }
    }
    if (d.q < md.Q) acc += c.pa * (va - vx);
    acc += (d.ph ? c.pf1 : c.pf0) * (vf - vx);
    return vx + acc;
}

template <int MH, typename T>
__device__ __forceinline__ T expect_next(const Model& md, const Coef<T>& c, const T* __restrict__ V, int x,
                                         const Digits& d) {
    // every gather first (independent loads in flight together), then the sum
    const T vx = V[x];
    T v1[MH], v0[MH];
#pragma unroll
    for (int k = 0; k < MH; k++) {
        const int o = d.occ[k];
        v1[k] = (k < md.H && o > 0) ? V[x - md.stride[k]] : T(0);
        v0[k] = (k < md.H && o > 1) ? V[x - o * md.stride[k]] : T(0);
    }
    const T va = (d.q < md.Q) ? V[x + 2] : T(0);
    const T vf = V[d.ph ? x - 1 : x + 1];
    return expect_from<MH, T>(md, c, d, vx, v1, v0, va, vf);
}

#ifdef VC_DEBUG_BOUNDS
// Every state expect_next reads from post-decision state x lies in [0, S).
template <int MH>
__device__ __forceinline__ bool successors_in_range(const Model& md, int x, const Digits& d, Ctl* ctl) {
    bool ok = x >= 0 && x < md.S && (d.ph ? x - 1 : x + 1) >= 0 && (d.ph ? x - 1 : x + 1) < md.S &&
              (d.q >= md.Q || x + 2 < md.S);
#pragma unroll
    for (int k = 0; k < MH; k++)
        if (k < md.H && d.occ[k] > 0) ok = ok && x - d.occ[k] * md.stride[k] >= 0 && x - md.stride[k] >= 0;
    return VC_IN_BOUNDS(ctl, ok);
}
#endif

// Expected one-step reward of the post-decision state: occupancy, queue and losses
// (departures lose their tasks, a full queue loses the arrival).
template <int MH, typename T>
__device__ __forceinline__ T post_reward(const Model& md, const Coef<T>& c, const Digits& d) {
    T loss = T(0);
    int occ_sum = 0;
#pragma unroll
    for (int k = 0; k < MH; k++) {
        if (k < md.H) {
            occ_sum += d.occ[k];
            loss += c.lossd[k] * T(d.occ[k]);
        }
    }
    if (d.q >= md.Q) loss += c.lossa;
    return c.w_occ * T(occ_sum) + c.w_q * T(d.q) + loss;
}

// Defer's backup with its self-transition solved, W of post_and_defer, computed on its
// own: in the single-instance pass 1 this form, next to the plain expect_next, timed
// faster (93 against 108 us per sweep of the 2.5 M-state instance) than the fused one,
// which the batched pass uses.
// (the same from gathered values, as expect_from)
template <int MH>
__device__ __forceinline__ float defer_from(const Model& md, const Coef<float>& c, const Digits& d, const float* v1,
                                           const float* v0, float va, float vf, float rx) {
    float sm = 0.0f, pm = 0.0f;
#pragma unroll
    for (int k = 0; k < MH; k++) {
        if (k < md.H) {
            const int o = d.occ[k];
            if (o == 1) {
                const float p = c.pc[k] + c.pd[k];
                sm = fmaf(p, v1[k], sm);
                pm += p;
            } else if (o > 1) {
                const float p1 = c.pc[k] * (float)o;
                sm = fmaf(p1, v1[k], sm);
                sm = fmaf(c.pd[k], v0[k], sm);
                pm += p1;
                pm += c.pd[k];
            }
        }
    }
    if (d.q < md.Q) {
        sm = fmaf(c.pa, va, sm);
        pm += c.pa;
    }
    const float pf = d.ph ? c.pf1 : c.pf0;
    sm = fmaf(pf, vf, sm);
    pm += pf;
    return __fdiv_rn(fmaf(c.gamma, sm, rx), fmaf(c.gamma, pm, 1.0f - c.gamma));
}

template <int MH>
__device__ __forceinline__ float defer_self_loop(const Model& md, const Coef<float>& c, const float* __restrict__ V,
                                                 int x, const Digits& d, float rx) {
    float v1[MH], v0[MH];
#pragma unroll
    for (int k = 0; k < MH; k++) {
        const int o = d.occ[k];
        v1[k] = (k < md.H && o > 0) ? V[x - md.stride[k]] : 0.0f;
        v0[k] = (k < md.H && o > 1) ? V[x - o * md.stride[k]] : 0.0f;
    }
    const float va = (d.q < md.Q) ? V[x + 2] : 0.0f;
    const float vf = V[d.ph ? x - 1 : x + 1];
    return defer_from<MH>(md, c, d, v1, v0, va, vf, rx);
}

// ---------------------------------------------------------------- implicit: pass 1
// SL (FP32 only): also U2(x) = defer's backup with the self-transition solved.
template <int MH, typename T, bool SL>
__global__ void __launch_bounds__(kThreads) k_post(Model md, Coef<T> c, const T* __restrict__ V, T* __restrict__ U,
                                                   T* __restrict__ U2, SweepCtl sc) {
    static_assert(!SL || std::is_same<T, float>::value, "self-transition solve in FP32 sweeps only");
    if (loop_done(sc)) return;
    for (int x = blockIdx.x * kThreads + threadIdx.x; x < md.S; x += gridDim.x * kThreads) {
        Digits d;
        decode<MH>(md, x, d);
#ifdef VC_DEBUG_BOUNDS
        if (!successors_in_range<MH>(md, x, d, sc.ctl)) continue;
#endif
        const T rx = post_reward<MH>(md, c, d);
        U[x] = rx + c.gamma * expect_next<MH>(md, c, V, x, d);
        if constexpr (SL) U2[x] = defer_self_loop<MH>(md, c, V, x, d, rx);
    }
}

// FP32 pass 1 over pairs of states: x (even, channel phase 0) and x + 1 (phase 1) share
// their digits and their reward (the phase does not enter it), and every value the two
// read comes in 8-byte-aligned pairs (the strides are even): V(x - o s_k) and
// V(x + 1 - o s_k) are adjacent, and each state's phase flip reads the other's V.  One
// decode, one reward and half the loads and stores per state; each state's arithmetic is
// expect_from's (and defer_from's), so U and W are those of k_post bit for bit.
template <int MH, bool SL>
__global__ void __launch_bounds__(kThreads) k_post_pair(Model md, Coef<float> c, const float* __restrict__ V,
                                                        float* __restrict__ U, float* __restrict__ U2, SweepCtl sc) {
    if (loop_done(sc)) return;
    const int npairs = md.S >> 1;  // S = 2 (Q + 1) (C + 1)^H is even
    for (int t = blockIdx.x * kThreads + threadIdx.x; t < npairs; t += gridDim.x * kThreads) {
        const int x = 2 * t;
        Digits d0;
        decode<MH>(md, x, d0);  // phase 0
        Digits d1 = d0;
        d1.ph = 1;
#ifdef VC_DEBUG_BOUNDS
        if (!successors_in_range<MH>(md, x, d0, sc.ctl) || !successors_in_range<MH>(md, x + 1, d1, sc.ctl)) continue;
#endif
        const float rx = post_reward<MH>(md, c, d0);
        const float2 vx = *reinterpret_cast<const float2*>(V + x);
        float v1a[MH], v1b[MH], v0a[MH], v0b[MH];
#pragma unroll
        for (int k = 0; k < MH; k++) {
            const int o = d0.occ[k];
            const float2 p1 = (k < md.H && o > 0) ? *reinterpret_cast<const float2*>(V + x - md.stride[k])
                                                  : make_float2(0.0f, 0.0f);
            const float2 p0 = (k < md.H && o > 1) ? *reinterpret_cast<const float2*>(V + x - o * md.stride[k])
                                                  : make_float2(0.0f, 0.0f);
            v1a[k] = p1.x;
            v1b[k] = p1.y;
            v0a[k] = p0.x;
            v0b[k] = p0.y;
        }
        const float2 va = (d0.q < md.Q) ? *reinterpret_cast<const float2*>(V + x + 2) : make_float2(0.0f, 0.0f);
        // the phase flip of x lands on x + 1, that of x + 1 on x
        const float e0 = expect_from<MH, float>(md, c, d0, vx.x, v1a, v0a, va.x, vx.y);
        const float e1 = expect_from<MH, float>(md, c, d1, vx.y, v1b, v0b, va.y, vx.x);
        *reinterpret_cast<float2*>(U + x) = make_float2(rx + c.gamma * e0, rx + c.gamma * e1);
        if constexpr (SL) {
            const float w0 = defer_from<MH>(md, c, d0, v1a, v0a, va.x, vx.y, rx);
            const float w1 = defer_from<MH>(md, c, d1, v1b, v0b, va.y, vx.x, rx);
            *reinterpret_cast<float2*>(U2 + x) = make_float2(w0, w1);
        }
    }
}

// ---------------------------------------------------------------- implicit: pass 2
// SL: defer takes U2(s) (its backup with the self-transition solved) instead of U(s).
template <int MH, typename T, bool SL>
__global__ void __launch_bounds__(kThreads) k_max(Model md, const T* __restrict__ U, const T* __restrict__ U2,
                                                  const T* __restrict__ V_in,
                                                  T* __restrict__ V_out, int32_t* __restrict__ pi,
                                                  T* __restrict__ qgap, SweepCtl sc) {
    if (loop_done(sc)) return;
    const long long sweep = loop_sweep(sc);
    T res = T(0), vabs = T(0);
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < md.S; s += gridDim.x * kThreads) {
        Digits d;
        decode<MH>(md, s, d);
        T best = -INFINITY, second = -INFINITY;
        int arg = md.H;
        // every gather first (infeasible actions read nothing and count as -inf), then the
        // max in action order
        T uk[MH];
#pragma unroll
        for (int k = 0; k < MH; k++) {
            const bool f = d.q >= 1 && k < md.H && d.occ[k] < md.C && (k == md.H - 1 || d.ph == 1) &&
                           VC_IN_BOUNDS(sc.ctl, s + md.stride[k] - 2 >= 0 && s + md.stride[k] - 2 < md.S);
            uk[k] = f ? U[s + md.stride[k] - 2] : T(-INFINITY);
        }
        const T u = SL ? U2[s] : U[s];  // defer: the post-decision state is s itself; highest index, so ties keep lower ones
#pragma unroll
        for (int k = 0; k < MH; k++) {
            if (uk[k] > best) {
                second = best;
                best = uk[k];
                arg = k;
            } else if (uk[k] > second) {
                second = uk[k];
            }
        }
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
        res = fmax(res, fabs(best - V_in[s]));
        vabs = fmax(vabs, fabs(best));
        if (sc.mode == kModeCert64 && sc.pi_ref && sc.pi_ref[s] != arg) atomicAdd(&sc.ctl->changes, 1ull);
    }
    if (sc.mode == kModeNone) return;
    res = block_max<T, kThreads>(res);
    vabs = block_max<T, kThreads>(vabs);
    finish_block<T>(sc, res, vabs, sweep);
}

// ------------------------------------------------------- implicit: in-block iteration
// (block_tile, the local passes over one tile of blocks, lives in vc_internal.cuh: the
// batched loop runs the same routine per instance.)
template <int MH, int HIN>
__global__ void __launch_bounds__(kBlockThreads, 3) k_block(Model md, Coef<float> c, int T, int passes,
                                                const float* __restrict__ Vin, const float* __restrict__ U,
                                                const float* __restrict__ W, float* __restrict__ V_out,
                                                SweepCtl sc) {
    extern __shared__ float blk_sm[];
    if (loop_done(sc)) return;
    const long long sweep = loop_sweep(sc);
    const int ntiles = (md.S + T - 1) / T;
    float res = 0.0f, vabs = 0.0f;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int start = t * T;
        block_tile<MH, HIN>(md, c, start, min(T, md.S - start), passes, Vin, U, W, V_out, blk_sm, sc.ctl, res, vabs);
    }
    if (sc.mode == kModeNone) return;
    res = block_max_dyn(res);
    vabs = block_max_dyn(vabs);
    finish_block<float>(sc, res, vabs, sweep);
}

// FP32 pass 2 with two states per thread and loop step: both states' gathers are issued
// before either maximum is taken, so twice as many independent loads are in flight per
// warp (the pass waits on the L2 latency of its gathers).  Same arithmetic and order as
// k_max, so the same results bit for bit.
template <int MH, bool SL>
__global__ void __launch_bounds__(kThreads) k_max2(Model md, const float* __restrict__ U, const float* __restrict__ U2,
                                                   const float* __restrict__ V_in, float* __restrict__ V_out,
                                                   int32_t* __restrict__ pi, float* __restrict__ qgap, SweepCtl sc) {
    if (loop_done(sc)) return;
    const long long sweep = loop_sweep(sc);
    float res = 0.0f, vabs = 0.0f;
    const int step = gridDim.x * kThreads;
    for (int s0 = blockIdx.x * kThreads + threadIdx.x; s0 < md.S; s0 += 2 * step) {
        float uk[2][MH], ud[2], vin[2];
        int sv[2];
        bool live[2];
#pragma unroll
        for (int t = 0; t < 2; t++) {
            const int s = s0 + t * step;
            sv[t] = s;
            live[t] = s < md.S;
            Digits d;
            decode<MH>(md, live[t] ? s : 0, d);
#pragma unroll
            for (int k = 0; k < MH; k++) {
                const bool f = live[t] && d.q >= 1 && k < md.H && d.occ[k] < md.C && (k == md.H - 1 || d.ph == 1) &&
                               VC_IN_BOUNDS(sc.ctl, s + md.stride[k] - 2 >= 0 && s + md.stride[k] - 2 < md.S);
                uk[t][k] = f ? U[s + md.stride[k] - 2] : -INFINITY;
            }
            ud[t] = live[t] ? (SL ? U2[s] : U[s]) : -INFINITY;
            vin[t] = live[t] ? V_in[s] : 0.0f;
        }
#pragma unroll
        for (int t = 0; t < 2; t++) {
            if (!live[t]) continue;
            float best = -INFINITY, second = -INFINITY;
            int arg = md.H;
#pragma unroll
            for (int k = 0; k < MH; k++) {
                if (uk[t][k] > best) {
                    second = best;
                    best = uk[t][k];
                    arg = k;
                } else if (uk[t][k] > second) {
                    second = uk[t][k];
                }
            }
            const float u = ud[t];
            if (u > best) {
                second = best;
                best = u;
                arg = md.H;
            } else if (u > second) {
                second = u;
            }
            const int s = sv[t];
            if (V_out) V_out[s] = best;
            if (pi) pi[s] = arg;
            if (qgap) qgap[s] = (second == -INFINITY) ? INFINITY : best - second;
            res = fmaxf(res, fabsf(best - vin[t]));
            vabs = fmaxf(vabs, fabsf(best));
        }
    }
    if (sc.mode == kModeNone) return;
    res = block_max<float, kThreads>(res);
    vabs = block_max<float, kThreads>(vabs);
    finish_block<float>(sc, res, vabs, sweep);
}

// Max over actions in order, lowest index on ties, for one state: its placements uk[] and
// defer's value u (the highest index).
template <int MH>
__device__ __forceinline__ void max_actions(const Model& md, const float* uk, float u, float& best, float& second,
                                            int& arg) {
    best = -INFINITY;
    second = -INFINITY;
    arg = md.H;
#pragma unroll
    for (int k = 0; k < MH; k++) {
        if (uk[k] > best) {
            second = best;
            best = uk[k];
            arg = k;
        } else if (uk[k] > second) {
            second = uk[k];
        }
    }
    if (u > best) {
        second = best;
        best = u;
        arg = md.H;
    } else if (u > second) {
        second = u;
    }
}

// Pass 2 over pairs of states s (even, channel phase 0) and s + 1 (phase 1): one decode,
// and one 8-byte load per action serves both, since their post-decision states of a
// placement are adjacent (s + s_k - 2 is even) and every placement feasible in phase 0
// (the RSU) is feasible in phase 1; outputs are written as pairs.  Each state's maximum,
// argmax and gap are k_max2's.
template <int MH, bool SL>
__global__ void __launch_bounds__(kThreads) k_max_pair(Model md, const float* __restrict__ U,
                                                       const float* __restrict__ U2, const float* __restrict__ V_in,
                                                       float* __restrict__ V_out, int32_t* __restrict__ pi,
                                                       float* __restrict__ qgap, SweepCtl sc) {
    if (loop_done(sc)) return;
    const long long sweep = loop_sweep(sc);
    float res = 0.0f, vabs = 0.0f;
    const int npairs = md.S >> 1;
    for (int t = blockIdx.x * kThreads + threadIdx.x; t < npairs; t += gridDim.x * kThreads) {
        const int s = 2 * t;
        Digits d;
        decode<MH>(md, s, d);  // phase 0; s + 1 has the same queue and occupancies
        float uk0[MH], uk1[MH];
#pragma unroll
        for (int k = 0; k < MH; k++) {
            // phase 1: every host with a free slot; phase 0: the RSU (host H - 1) only
            const bool f1 = d.q >= 1 && k < md.H && d.occ[k] < md.C &&
                            VC_IN_BOUNDS(sc.ctl, s + md.stride[k] - 2 >= 0 && s + md.stride[k] - 1 < md.S);
            const bool f0 = f1 && k == md.H - 1;
            const float2 u2 = f1 ? *reinterpret_cast<const float2*>(U + s + md.stride[k] - 2)
                                 : make_float2(-INFINITY, -INFINITY);
            uk0[k] = f0 ? u2.x : -INFINITY;
            uk1[k] = f1 ? u2.y : -INFINITY;
        }
        const float2 ud = *reinterpret_cast<const float2*>((SL ? U2 : U) + s);
        const float2 vin = *reinterpret_cast<const float2*>(V_in + s);
        float b0, c0, b1, c1;
        int a0, a1;
        max_actions<MH>(md, uk0, ud.x, b0, c0, a0);
        max_actions<MH>(md, uk1, ud.y, b1, c1, a1);
        if (V_out) *reinterpret_cast<float2*>(V_out + s) = make_float2(b0, b1);
        if (pi) *reinterpret_cast<int2*>(pi + s) = make_int2(a0, a1);
        if (qgap)
            *reinterpret_cast<float2*>(qgap + s) =
                make_float2(c0 == -INFINITY ? INFINITY : b0 - c0, c1 == -INFINITY ? INFINITY : b1 - c1);
        res = fmaxf(res, fmaxf(fabsf(b0 - vin.x), fabsf(b1 - vin.y)));
        vabs = fmaxf(vabs, fmaxf(fabsf(b0), fabsf(b1)));
    }
    if (sc.mode == kModeNone) return;
    res = block_max<float, kThreads>(res);
    vabs = block_max<float, kThreads>(vabs);
    finish_block<float>(sc, res, vabs, sweep);
}

// ------------------------------------------------ implicit: mixed-precision refinement
// Policy residual in FP64, r(s) = U64(x_pi(s)) - V64(s) with U64 = R + gamma E[V64(next) | x]
// from the FP64 pass-1 kernel over every post-decision state (coalesced: thread x gathers
// around x), so this kernel makes one gather per state.  r is stored as float (it is small
// once V64 is near V_pi, so FP32 keeps ~1e-7 of it).
template <int MH>
__global__ void __launch_bounds__(kThreads) k_resid64(Model md, const int32_t* __restrict__ pi,
                                                      const double* __restrict__ U, const double* __restrict__ V,
                                                      float* __restrict__ r, SweepCtl sc) {
    double mx = 0.0;
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < md.S; s += gridDim.x * kThreads) {
        Digits d;
        decode<MH>(md, s, d);
        int x = s;
        if (!apply_action<MH>(md, s, pi[s], d, x)) {
            atomicOr(&sc.ctl->error, kErrInfeasiblePolicy);
            r[s] = 0.0f;
            continue;
        }
#ifdef VC_DEBUG_BOUNDS
        if (!VC_IN_BOUNDS(sc.ctl, x >= 0 && x < md.S)) continue;
#endif
        const double rd = U[x] - V[s];
        r[s] = (float)rd;
        mx = fmax(mx, fabs(rd));
    }
    // kModeCert64: max |T_pi V - V| in FP64 into the control block
    if (sc.mode != kModeCert64) return;
    mx = block_max<double, kThreads>(mx);
    finish_block<double>(sc, mx, 0.0, 0);
}

// Correction sweep in FP32: e_out(s) = r(s) + gamma E[e_in(next) | x_pi(s)].  Its fixed
// point e solves (I - gamma P_pi) e = r, so V64 + e is the evaluation of pi.
template <int MH>
__global__ void __launch_bounds__(kThreads) k_correct32(Model md, Coef<float> c, const int32_t* __restrict__ pi,
                                                        const float* __restrict__ r, const float* __restrict__ e_in,
                                                        float* __restrict__ e_out, SweepCtl sc) {
    if (loop_done(sc)) return;
    const long long sweep = loop_sweep(sc);
    float res = 0.0f, vabs = 0.0f;
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < md.S; s += gridDim.x * kThreads) {
        Digits d;
        decode<MH>(md, s, d);
        int x = s;
        if (!apply_action<MH>(md, s, pi[s], d, x)) {
            atomicOr(&sc.ctl->error, kErrInfeasiblePolicy);
            e_out[s] = e_in[s];
            continue;
        }
#ifdef VC_DEBUG_BOUNDS
        if (!successors_in_range<MH>(md, x, d, sc.ctl)) continue;
#endif
        const float v = r[s] + c.gamma * expect_next<MH>(md, c, e_in, x, d);
        e_out[s] = v;
        res = fmaxf(res, fabsf(v - e_in[s]));
        vabs = fmaxf(vabs, fabsf(v));
    }
    if (sc.mode == kModeNone) return;
    res = block_max<float, kThreads>(res);
    vabs = block_max<float, kThreads>(vabs);
    finish_block<float>(sc, res, vabs, sweep);
}

// Product by the correction matrix for the BiCGSTAB solve: y(s) = x(s) - gamma
// E[x(next) | x_pi(s)], with the stage's partial sums <w, y> and <y, y>.  The policy was
// checked feasible by the residual pass; an infeasible entry would act as the identity.
template <int MH>
__global__ void __launch_bounds__(kThreads) k_apply32(Model md, Coef<float> c, const int32_t* __restrict__ pi,
                                                      const float* __restrict__ xin, float* __restrict__ y,
                                                      const float* __restrict__ w, int stage, KrylovArgs k) {
    if (kr_done(k)) return;
    float d0 = 0.0f, d1 = 0.0f;
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < md.S; s += gridDim.x * kThreads) {
        Digits d;
        decode<MH>(md, s, d);
        int x = s;
        float yv = xin[s];
        if (apply_action<MH>(md, s, pi[s], d, x)) {
#ifdef VC_DEBUG_BOUNDS
            if (successors_in_range<MH>(md, x, d, k.ctl))
#endif
                yv -= c.gamma * expect_next<MH>(md, c, xin, x, d);
        }
        y[s] = yv;
        d0 = fmaf(w[s], yv, d0);
        d1 = fmaf(yv, yv, d1);
    }
    kr_finish<kThreads>(k, stage, d0, d1, 0.0f);
}

__global__ void k_axpy64(double* __restrict__ V, const float* __restrict__ e, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) V[i] += (double)e[i];
}

__global__ void k_f32_to_f64(const float* __restrict__ in, double* __restrict__ out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = (double)in[i];
}

// ------------------------------------------------------------------------ dispatch
static inline bool implicit_sweeps(const Mdp* m) { return (m->fmt & 0xF) == VC_IMPLICIT; }

// Calls f with std::integral_constant<int, MH>: MH = H for H <= 8 (the per-host loops are
// unrolled to MH, so an exact bound issues no predicated-off iterations), else 16.
template <typename F>
static int by_h(const Mdp* m, F&& f) {
    switch (m->md.H) {
        case 1: return f(std::integral_constant<int, 1>());
        case 2: return f(std::integral_constant<int, 2>());
        case 3: return f(std::integral_constant<int, 3>());
        case 4: return f(std::integral_constant<int, 4>());
        case 5: return f(std::integral_constant<int, 5>());
        case 6: return f(std::integral_constant<int, 6>());
        case 7: return f(std::integral_constant<int, 7>());
        case 8: return f(std::integral_constant<int, 8>());
        default: return f(std::integral_constant<int, 16>());
    }
}

// Inner hosts and states of the blocks of the in-block iteration: h as set on the handle,
// else the largest h whose block of 2(Q+1)(C+1)^h states fits 1024 threads.
int block_shape(const Mdp* m, int* h_out, int* B_out) {
    int h = m->blk_h;
    if (h < 0) {
        h = 0;
        long long B = 2LL * (m->md.Q + 1);
        while (h < m->md.H && h < kBlockMaxInner && B * (m->md.C + 1) <= kBlockThreads) {
            B *= (m->md.C + 1);
            h++;
        }
    }
    long long B = 2LL * (m->md.Q + 1);
    for (int k = 0; k < h; k++) B *= (m->md.C + 1);
    if (h > m->md.H || h > kBlockMaxInner || B > kBlockThreads)
        return fail(VC_ERR_ARG, "a block of the in-block iteration needs at most 3 inner hosts and 512 states");
    *h_out = h;
    *B_out = (int)B;
    return VC_OK;
}

static int launch_block(Mdp* m, const float* V_in, float* V_out, SweepCtl sc, cudaStream_t st) {
    int h = 0, B = 0, rc;
    if ((rc = block_shape(m, &h, &B))) return rc;
    // tiles of whole blocks, at most kBlockThreads states
    const int T = B * (kBlockThreads / B);
    const int threads = (T + 31) / 32 * 32;
    const size_t smem = 4 * sizeof(float) * (size_t)threads;
    const int g = state_grid(m);
    SweepCtl sc1 = sc;
    if (sc1.mode != kModeLoop32) sc1.mode = kModeNone;
    count_launches(2);
    return by_h(m, [&](auto mh) {
        constexpr int MH = decltype(mh)::value;
        auto kern = h == 0 ? k_block<MH, 0> : h == 1 ? k_block<MH, 1> : h == 2 ? k_block<MH, 2> : k_block<MH, 3>;
        if (m->blk_grid <= 0) {
            int per_sm = 0;
            VC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared));
            VC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
            m->blk_grid = std::max(1, per_sm) * (m->num_sms > 0 ? m->num_sms : 148);
        }
        const int ntiles = (m->S + T - 1) / T;
        k_post_pair<MH, true><<<g, kThreads, 0, st>>>(m->md, m->c32, V_in, m->U32, m->U32s, sc1);
        kern<<<std::min(ntiles, m->blk_grid), threads, smem, st>>>(m->md, m->c32, T, m->blk_passes, V_in, m->U32,
                                                                   m->U32s, V_out, sc);
        VC_CUDA(cudaGetLastError());
        return (int)VC_OK;
    });
}

int launch_sweep32(Mdp* m, const float* V_in, float* V_out, int32_t* pi, float* qgap, SweepCtl sc,
                   cudaStream_t st) {
    if (!implicit_sweeps(m)) return csr_sweep32(m, V_in, V_out, pi, qgap, sc, st);
    if (sc.block) {
        if (pi || qgap) return fail(VC_ERR_ARG, "the in-block iteration returns values only");
        return launch_block(m, V_in, V_out, sc, st);
    }
    const int g = state_grid(m);
    SweepCtl sc1 = sc;
    if (sc1.mode != kModeLoop32) sc1.mode = kModeNone;
    count_launches(2);
    by_h(m, [&](auto mh) {
        constexpr int MH = decltype(mh)::value;
        if (sc.self_loop) {
            k_post_pair<MH, true><<<g, kThreads, 0, st>>>(m->md, m->c32, V_in, m->U32, m->U32s, sc1);
            k_max_pair<MH, true><<<g, kThreads, 0, st>>>(m->md, m->U32, m->U32s, V_in, V_out, pi, qgap, sc);
        } else {
            k_post_pair<MH, false><<<g, kThreads, 0, st>>>(m->md, m->c32, V_in, m->U32, nullptr, sc1);
            k_max_pair<MH, false><<<g, kThreads, 0, st>>>(m->md, m->U32, nullptr, V_in, V_out, pi, qgap, sc);
        }
        return 0;
    });
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int launch_bellman64(Mdp* m, const double* V_in, double* V_out, int32_t* pi, double* qgap, SweepCtl sc,
                     cudaStream_t st) {
    if (!m->has_model) return csr_bellman64(m, V_in, V_out, pi, qgap, sc, st);
    const int g = state_grid(m);
    SweepCtl none = sc;
    none.mode = kModeNone;
    count_launches(2);
    by_h(m, [&](auto mh) {
        constexpr int MH = decltype(mh)::value;
        k_post<MH, double, false><<<g, kThreads, 0, st>>>(m->md, m->c64, V_in, m->U64, nullptr, none);
        k_max<MH, double, false><<<g, kThreads, 0, st>>>(m->md, m->U64, nullptr, V_in, V_out, pi, qgap, sc);
        return 0;
    });
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int launch_resid64(Mdp* m, const int32_t* pi, const double* V64, float* r, SweepCtl sc, cudaStream_t st) {
    if (!m->has_model) return csr_resid64(m, pi, V64, r, sc, st);
    const int g = state_grid(m);
    SweepCtl none = sc;
    none.mode = kModeNone;
    count_launches(2);
    by_h(m, [&](auto mh) {
        constexpr int MH = decltype(mh)::value;
        k_post<MH, double, false><<<g, kThreads, 0, st>>>(m->md, m->c64, V64, m->U64, nullptr, none);
        k_resid64<MH><<<g, kThreads, 0, st>>>(m->md, pi, m->U64, V64, r, sc);
        return 0;
    });
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int launch_correct32(Mdp* m, const int32_t* pi, const float* r, const float* e_in, float* e_out, SweepCtl sc,
                     cudaStream_t st) {
    if (!m->has_model) return csr_correct32(m, pi, r, e_in, e_out, sc, st);
    count_launches(1);
    by_h(m, [&](auto mh) {
        k_correct32<decltype(mh)::value><<<state_grid(m), kThreads, 0, st>>>(m->md, m->c32, pi, r, e_in, e_out, sc);
        return 0;
    });
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int launch_apply32(Mdp* m, const int32_t* pi, const float* x, float* y, const float* w, int stage,
                   const KrylovArgs& k, cudaStream_t st) {
    if (!m->has_model) return csr_apply32(m, pi, x, y, w, stage, k, st);
    count_launches(1);
    by_h(m, [&](auto mh) {
        k_apply32<decltype(mh)::value><<<state_grid(m), kThreads, 0, st>>>(m->md, m->c32, pi, x, y, w, stage, k);
        return 0;
    });
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

static inline unsigned elementwise_grid(int n) {
    const int b = (n + kThreads - 1) / kThreads;
    return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

int launch_axpy64(double* V64, const float* e, int n, cudaStream_t st) {
    count_launches(1);
    k_axpy64<<<elementwise_grid(n), kThreads, 0, st>>>(V64, e, n);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int launch_f32_to_f64(const float* in, double* out, int n, cudaStream_t st) {
    count_launches(1);
    k_f32_to_f64<<<elementwise_grid(n), kThreads, 0, st>>>(in, out, n);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

// ------------------------------------------------------------- greedy heuristic policy
// Algorithm 2 read as a policy on this MDP: with a task waiting, place it on the feasible
// host with the largest service rate (ties to the lowest index), else defer.
struct ServiceRates {
    double mu[kMaxH];
};

template <int MH>
__global__ void __launch_bounds__(kThreads) k_greedy(Model md, ServiceRates r, int32_t* __restrict__ pi) {
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < md.S; s += gridDim.x * kThreads) {
        Digits d;
        decode<MH>(md, s, d);
        int best = md.H;
        double best_mu = -1.0;
        if (d.q >= 1) {
#pragma unroll
            for (int k = 0; k < MH; k++) {
                if (k < md.H && d.occ[k] < md.C && (k == md.H - 1 || d.ph == 1) && r.mu[k] > best_mu) {
                    best_mu = r.mu[k];
                    best = k;
                }
            }
        }
        pi[s] = best;
    }
}

int launch_greedy(Mdp* m, int32_t* pi, cudaStream_t st) {
    ServiceRates r;
    for (int k = 0; k < kMaxH; k++) r.mu[k] = m->rates.mu[k];
    count_launches(1);
    by_h(m, [&](auto mh) {
        k_greedy<decltype(mh)::value><<<state_grid(m), kThreads, 0, st>>>(m->md, r, pi);
        return 0;
    });
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

}  // namespace vc
