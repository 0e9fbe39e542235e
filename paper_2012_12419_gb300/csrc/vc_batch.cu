// vc_batch.cu -- batched value iteration: hundreds of independent uneven-sized instances
// of the placement MDP solved together (each by Algorithm 3 with its own gamma, its own
// convergence test and its own sweep count).
//
// Layout: the instances' state ranges are concatenated; a tile table cuts every range into
// tiles of at most `ts` states that never straddle two instances.  Every sweep kernel is
// persistent (a few CTAs per SM, grid-stride over the tile table); a tile of an instance
// that has terminated returns at once.  Per sweep and instance, each tile folds its
// residual max|V' - V| into the instance's slot (one atomicMax per tile) and takes a ticket;
// the instance's last tile closes its sweep (count, tolerance max(tol, 4 ulp(max|V|)),
// FP32 stall, max_sweeps) and retires the instance from the active count.  All active
// instances advance one sweep per launch, so a launch's parity names the ring slot.
//
// The FP32 loop is one CUDA graph: a conditional WHILE node whose body is two sweeps (the
// ping-pong pair) and a one-thread kernel that keeps the loop running while any instance is
// active and the sweep budget lasts.  There are no inter-CTA waits anywhere: instances only
// couple through their per-sweep tickets.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "vc_internal.cuh"
#include "vc_krylov.cuh"

namespace vc {

// Named check of the kernel launches just enqueued (a refused launch leaves its error
// pending; this reports it where it happened instead of at a later call).
#define VC_LAUNCHED(what)                                                  \
    do {                                                                   \
        const cudaError_t le_ = cudaGetLastError();                        \
        if (le_ != cudaSuccess) return vc::cuda_fail(le_, "launch: " what); \
    } while (0)

struct InstDesc {
    Model md;
    Coef<float> c32;
    Coef<double> c64;
    long long off;  // first state in the concatenated arrays
    int S;
    int blk_h;      // inner hosts of the in-block iteration's blocks (2(Q+1)(C+1)^blk_h states)
};

struct BatchTile {
    int inst;
    int start;  // first state, relative to the instance
    int count;
    int pad_;
};

// Device-side control of the batched loops (SoA over instances).
struct BatchCtl {
    int* done;                 // 0 running, 1 converged, 2 max sweeps, 3 FP32 stall
    int* sweeps;
    int* ticket;
    const int* tiles_of;       // tiles per instance (constant)
    int* final_buf;            // buffer of the last iterate (0: A, 1: B)
    int* since_best;
    float* best_res;
    unsigned int* res32;       // [2n] ring of two slots
    unsigned int* vmax32;      // [2n]
    unsigned long long* res64; // [n] FP64 residual of a certificate / residual pass
    int* active;               // instances still running
    long long* iters;          // sweeps launched by the graph loop
    const long long* max_sweeps; // loop parameters in device memory, so one captured graph
    const double* tol;           // serves every call
    const float* tol_scale;      // per-instance factor on tol (nullptr: 1)
};

// Instance descriptor of a tile, staged in shared memory once per tile.
__device__ __forceinline__ void load_desc(const InstDesc* __restrict__ descs, int inst, InstDesc& sd) {
    const int n = (int)(sizeof(InstDesc) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(descs + inst);
    int* dst = reinterpret_cast<int*>(&sd);
    for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

// Algorithm 3's step-3 test for one instance after sweep k: residual r below
// max(tol, 4 ulp(max|V|)) -> 1, no new best residual for kStallSweeps sweeps (the FP32
// floor) -> 3, k reaching max_sweeps -> 2, else 0 (best_res / since_best updated).
__device__ __forceinline__ int sweep_verdict(double tol, float r, float vm, long long k, long long max_sweeps,
                                             float& best_res, int& since_best) {
    int e = 0;
    frexpf(vm, &e);
    const double ulp = (vm > 0.0f) ? ldexp(1.0, e - 24) : 0.0;
    const double tol_eff = fmax(tol, 4.0 * ulp);
    int done = 0;
    if ((double)r < tol_eff) {
        done = 1;
    } else if (r < best_res) {
        best_res = r;
        since_best = 0;
    } else if (++since_best >= kStallSweeps) {
        done = 3;
    }
    if (!done && k >= max_sweeps) done = 2;
    return done;
}

// Closes an instance's sweep once its last tile arrives (thread 0 of that tile).
__device__ void close_instance(const BatchCtl& c, int i, float res, float vmax, int parity, int out_buf) {
    const double tol = *c.tol * (c.tol_scale ? (double)c.tol_scale[i] : 1.0);
    const int slot = 2 * i + parity, next = 2 * i + (parity ^ 1);
    atomicMax(&c.res32[slot], __float_as_uint(res));
    atomicMax(&c.vmax32[slot], __float_as_uint(vmax));
    __threadfence();
    const int t = atomicAdd(&c.ticket[i], 1);
    if (t != c.tiles_of[i] - 1) return;
    __threadfence();
    const float r = __uint_as_float(*((volatile unsigned int*)&c.res32[slot]));
    const float vm = __uint_as_float(*((volatile unsigned int*)&c.vmax32[slot]));
    c.ticket[i] = 0;
    c.res32[next] = 0u;
    c.vmax32[next] = 0u;
    const int k = c.sweeps[i] + 1;
    c.sweeps[i] = k;
    c.final_buf[i] = out_buf;
    float best = c.best_res[i];
    int since = c.since_best[i];
    const int done = sweep_verdict(tol, r, vm, k, *c.max_sweeps, best, since);
    c.best_res[i] = best;
    c.since_best[i] = since;
    if (done) {
        c.done[i] = done;
        atomicSub(c.active, 1);
    }
    __threadfence();
}

// Model arithmetic per instance (same formulas as the single-instance implicit kernels).
template <int MH, typename T>
__device__ __forceinline__ T b_expect(const Model& md, const Coef<T>& c, const T* __restrict__ V, int x,
                                      const Digits& d) {
    const T vx = V[x];
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < MH; k++) {
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
            }
        }
    }
    if (d.q < md.Q) acc += c.pa * (V[x + 2] - vx);
    const T vf = V[d.ph ? x - 1 : x + 1];
    acc += (d.ph ? c.pf1 : c.pf0) * (vf - vx);
    return vx + acc;
}

template <int MH, typename T>
__device__ __forceinline__ T b_reward(const Model& md, const Coef<T>& c, const Digits& d) {
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

template <typename T>
__device__ __forceinline__ const Coef<T>& coef_of(const InstDesc& d);
template <>
__device__ __forceinline__ const Coef<float>& coef_of<float>(const InstDesc& d) {
    return d.c32;
}
template <>
__device__ __forceinline__ const Coef<double>& coef_of<double>(const InstDesc& d) {
    return d.c64;
}

// Pass 1 over all active tiles: U(x) = R(x) + gamma E[V(next) | x] (per instance).
// done = nullptr processes every instance (extraction / certificate passes).  SL (FP32
// loop only): also U2(x) = defer's backup with its self-transition solved.
template <int MH, typename T, bool SL>
__global__ void k_bpost(const InstDesc* __restrict__ descs, const BatchTile* __restrict__ tiles, int ntiles,
                        const int* __restrict__ done, const T* __restrict__ V, T* __restrict__ U,
                        T* __restrict__ U2) {
    static_assert(!SL || std::is_same<T, float>::value, "self-transition solve in FP32 sweeps only");
    __shared__ InstDesc sd;
    __shared__ int skip;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        if (threadIdx.x == 0) skip = done ? (*((volatile int*)&done[tl.inst]) != 0) : 0;
        __syncthreads();
        if (!skip) {
            load_desc(descs, tl.inst, sd);
            __syncthreads();
            const T* Vi = V + sd.off;
            T* Ui = U + sd.off;
            for (int j = threadIdx.x; j < tl.count; j += blockDim.x) {
                const int x = tl.start + j;
                Digits d;
                decode<MH>(sd.md, x, d);
                const T rx = b_reward<MH>(sd.md, coef_of<T>(sd), d);
                if constexpr (SL) {
                    float u, w;
                    post_and_defer<MH>(sd.md, sd.c32, Vi, x, d, rx, u, w);
                    Ui[x] = u;
                    U2[sd.off + x] = w;
                } else {
                    Ui[x] = rx + coef_of<T>(sd).gamma * b_expect<MH>(sd.md, coef_of<T>(sd), Vi, x, d);
                }
            }
        }
        __syncthreads();
    }
}

// b_expect from gathered values (vx = V(x), v1 / v0 the completion / departure targets,
// va the arrival, vf the phase flip), the same operations in the same order.
template <int MH>
__device__ __forceinline__ float b_expect_from(const Model& md, const Coef<float>& c, const Digits& d, float vx,
                                               const float* v1, const float* v0, float va, float vf) {
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < MH; k++) {
        if (k < md.H) {
            const int o = d.occ[k];
            if (o > 0) {
                if (o == 1) {
                    acc += (c.pc[k] + c.pd[k]) * (v1[k] - vx);
                } else {
                    acc += c.pc[k] * float(o) * (v1[k] - vx) + c.pd[k] * (v0[k] - vx);
                }
            }
        }
    }
    if (d.q < md.Q) acc += c.pa * (va - vx);
    acc += (d.ph ? c.pf1 : c.pf0) * (vf - vx);
    return vx + acc;
}

// post_and_defer from gathered values: U and W of one post-decision state, the same
// operations in the same order (the self-transition loop's pass 1).
template <int MH>
__device__ __forceinline__ void b_post_defer_from(const Model& md, const Coef<float>& c, const Digits& d, float vx,
                                                  const float* v1, const float* v0, float va, float vf, float rx,
                                                  float& U, float& W) {
    float acc = 0.0f, sm = 0.0f, pm = 0.0f;
#pragma unroll
    for (int k = 0; k < MH; k++) {
        if (k < md.H) {
            const int o = d.occ[k];
            if (o == 1) {
                const float p = c.pc[k] + c.pd[k];
                acc += p * (v1[k] - vx);
                sm = fmaf(p, v1[k], sm);
                pm += p;
            } else if (o > 1) {
                const float p1 = c.pc[k] * (float)o;
                acc += p1 * (v1[k] - vx) + c.pd[k] * (v0[k] - vx);
                sm = fmaf(p1, v1[k], sm);
                sm = fmaf(c.pd[k], v0[k], sm);
                pm += p1;
                pm += c.pd[k];
            }
        }
    }
    if (d.q < md.Q) {
        acc += c.pa * (va - vx);
        sm = fmaf(c.pa, va, sm);
        pm += c.pa;
    }
    const float pf = d.ph ? c.pf1 : c.pf0;
    acc += pf * (vf - vx);
    sm = fmaf(pf, vf, sm);
    pm += pf;
    U = rx + c.gamma * (vx + acc);
    W = __fdiv_rn(fmaf(c.gamma, sm, rx), fmaf(c.gamma, pm, 1.0f - c.gamma));
}

// Pass 1 of Eq. 18's FP32 loop over pairs of states x (even, channel phase 0) and x + 1
// (phase 1), which share their digits and their reward; every value they read comes in
// 8-byte-aligned pairs (tile starts, tile lengths, instance sizes and offsets are even, and
// so are the strides).  One decode, one reward, paired loads and stores; each state's
// value is k_bpost's bit for bit.
// SL: the self-transition loop's pass 1, U and W (defer's value with its self-transition
// solved) of both states, as post_and_defer computes them.
template <int MH, bool SL>
__global__ void __launch_bounds__(kThreads, 3) k_bpost_pair(const InstDesc* __restrict__ descs, const BatchTile* __restrict__ tiles, int ntiles,
                             const int* __restrict__ done, const float* __restrict__ V, float* __restrict__ U,
                             float* __restrict__ U2) {
    __shared__ InstDesc sd;
    __shared__ int skip;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        if (threadIdx.x == 0) skip = done ? (*((volatile int*)&done[tl.inst]) != 0) : 0;
        __syncthreads();
        if (!skip) {
            load_desc(descs, tl.inst, sd);
            __syncthreads();
            const float* Vi = V + sd.off;
            float* Ui = U + sd.off;
            const Coef<float>& c = sd.c32;
            for (int jj = threadIdx.x; 2 * jj < tl.count; jj += blockDim.x) {
                const int x = tl.start + 2 * jj;  // even, and x + 1 < start + count (even tiles)
                Digits d0;
                decode<MH>(sd.md, x, d0);
                Digits d1 = d0;
                d1.ph = 1;
                const float rx = b_reward<MH>(sd.md, c, d0);  // the phase does not enter the reward
                const float2 vx = *reinterpret_cast<const float2*>(Vi + x);
                float v1a[MH], v1b[MH], v0a[MH], v0b[MH];
#pragma unroll
                for (int k = 0; k < MH; k++) {
                    const int o = d0.occ[k];
                    const float2 p1 = (k < sd.md.H && o > 0)
                                          ? *reinterpret_cast<const float2*>(Vi + x - sd.md.stride[k])
                                          : make_float2(0.0f, 0.0f);
                    const float2 p0 = (k < sd.md.H && o > 1)
                                          ? *reinterpret_cast<const float2*>(Vi + x - o * sd.md.stride[k])
                                          : make_float2(0.0f, 0.0f);
                    v1a[k] = p1.x;
                    v1b[k] = p1.y;
                    v0a[k] = p0.x;
                    v0b[k] = p0.y;
                }
                const float2 va = (d0.q < sd.md.Q) ? *reinterpret_cast<const float2*>(Vi + x + 2)
                                                   : make_float2(0.0f, 0.0f);
                // the phase flip of x lands on x + 1, that of x + 1 on x
                if constexpr (SL) {
                    float u0, w0, u1, w1;
                    b_post_defer_from<MH>(sd.md, c, d0, vx.x, v1a, v0a, va.x, vx.y, rx, u0, w0);
                    b_post_defer_from<MH>(sd.md, c, d1, vx.y, v1b, v0b, va.y, vx.x, rx, u1, w1);
                    *reinterpret_cast<float2*>(Ui + x) = make_float2(u0, u1);
                    *reinterpret_cast<float2*>(U2 + sd.off + x) = make_float2(w0, w1);
                } else {
                    const float e0 = b_expect_from<MH>(sd.md, c, d0, vx.x, v1a, v0a, va.x, vx.y);
                    const float e1 = b_expect_from<MH>(sd.md, c, d1, vx.y, v1b, v0b, va.y, vx.x);
                    *reinterpret_cast<float2*>(Ui + x) = make_float2(rx + c.gamma * e0, rx + c.gamma * e1);
                }
            }
        }
        __syncthreads();
    }
}

// Pass 2 of Eq. 18's FP32 loop over the same pairs: one decode, one 8-byte load per action
// for both states (phase 0's feasible placements are a subset of phase 1's), paired
// stores; each state's maximum is k_bmax's, and a tile's residual closes the instance as
// there.
// SL: defer takes U2 (its value with the self-transition solved), as in k_bmax.
template <int MH, bool SL>
__global__ void k_bmax_pair(const InstDesc* __restrict__ descs, const BatchTile* __restrict__ tiles, int ntiles,
                            BatchCtl c, int parity, const float* __restrict__ U, const float* __restrict__ U2,
                            const float* __restrict__ V_in, float* __restrict__ V_out) {
    __shared__ InstDesc sd;
    __shared__ int skip;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        if (threadIdx.x == 0) skip = (*((volatile int*)&c.done[tl.inst]) != 0);
        __syncthreads();
        if (skip) {
            __syncthreads();
            continue;
        }
        load_desc(descs, tl.inst, sd);
        __syncthreads();
        const float* Ui = U + sd.off;
        const float* Vi = V_in + sd.off;
        float* Vo = V_out + sd.off;
        float res = 0.0f, vabs = 0.0f;
        for (int jj = threadIdx.x; 2 * jj < tl.count; jj += blockDim.x) {
            const int s = tl.start + 2 * jj;  // even, and s + 1 < start + count (even tiles)
            Digits d;
            decode<MH>(sd.md, s, d);
            float uk0[MH], uk1[MH];
#pragma unroll
            for (int k = 0; k < MH; k++) {
                // s + 1 (phase 1): every host with a free slot; s (phase 0): the RSU only
                const bool f1 = d.q >= 1 && k < sd.md.H && d.occ[k] < sd.md.C;
                const bool f0 = f1 && k == sd.md.H - 1;
                const float2 u2 = f1 ? *reinterpret_cast<const float2*>(Ui + s + sd.md.stride[k] - 2)
                                     : make_float2(-INFINITY, -INFINITY);
                uk0[k] = f0 ? u2.x : -INFINITY;
                uk1[k] = f1 ? u2.y : -INFINITY;
            }
            const float2 ud = *reinterpret_cast<const float2*>(SL ? U2 + sd.off + s : Ui + s);
            const float2 vin = *reinterpret_cast<const float2*>(Vi + s);
            float b0 = -INFINITY, b1 = -INFINITY;
#pragma unroll
            for (int k = 0; k < MH; k++) {
                if (uk0[k] > b0) b0 = uk0[k];
                if (uk1[k] > b1) b1 = uk1[k];
            }
            if (ud.x > b0) b0 = ud.x;
            if (ud.y > b1) b1 = ud.y;
            *reinterpret_cast<float2*>(Vo + s) = make_float2(b0, b1);
            res = fmax(res, fabs(b0 - vin.x));
            res = fmax(res, fabs(b1 - vin.y));
            vabs = fmax(vabs, fabs(b0));
            vabs = fmax(vabs, fabs(b1));
        }
        res = block_max<float, kThreads>(res);
        vabs = block_max<float, kThreads>(vabs);
        if (threadIdx.x == 0) close_instance(c, tl.inst, res, vabs, parity, parity ^ 1);
        __syncthreads();
    }
}

// Pass 2: V'(s) = max_a U(x_a(s)); per-instance residual and close (loop mode, ctl given),
// or plain extraction with policy / FP64 certificate residual into res64 (ctl null).  SL:
// defer takes U2(s) (its backup with the self-transition solve).  Outside loop mode,
// instances with a non-zero entry in `skipped` (nullable) are left untouched.
template <int MH, typename T, bool SL>
__global__ void k_bmax(const InstDesc* __restrict__ descs, const BatchTile* __restrict__ tiles, int ntiles,
                       BatchCtl c, int loop, int parity, const T* __restrict__ U, const T* __restrict__ U2,
                       const T* __restrict__ V_in,
                       T* __restrict__ V_out, int32_t* __restrict__ pi, unsigned long long* __restrict__ res64,
                       const int* __restrict__ skipped = nullptr) {
    __shared__ InstDesc sd;
    __shared__ int skip;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        if (threadIdx.x == 0)
            skip = loop ? (*((volatile int*)&c.done[tl.inst]) != 0) : (skipped ? skipped[tl.inst] != 0 : 0);
        __syncthreads();
        if (skip) {
            __syncthreads();
            continue;
        }
        load_desc(descs, tl.inst, sd);
        __syncthreads();
        const T* Ui = U + sd.off;
        const T* Vi = V_in + sd.off;
        T res = T(0), vabs = T(0);
        // two states per thread and step: every gather of both is issued before either
        // maximum (more loads in flight); same arithmetic and order per state
        for (int j0 = threadIdx.x; j0 < tl.count; j0 += 2 * blockDim.x) {
            T uk[2][MH], ud[2], vin[2];
#pragma unroll
            for (int t = 0; t < 2; t++) {
                const int j = j0 + t * blockDim.x;
                const bool live = j < tl.count;
                const int s = tl.start + (live ? j : 0);
                Digits d;
                decode<MH>(sd.md, s, d);
#pragma unroll
                for (int k = 0; k < MH; k++) {
                    const bool f = live && d.q >= 1 && k < sd.md.H && d.occ[k] < sd.md.C &&
                                   (k == sd.md.H - 1 || d.ph == 1);
                    uk[t][k] = f ? Ui[s + sd.md.stride[k] - 2] : T(-INFINITY);
                }
                ud[t] = live ? (SL ? U2[sd.off + s] : Ui[s]) : T(-INFINITY);
                vin[t] = live ? Vi[s] : T(0);
            }
#pragma unroll
            for (int t = 0; t < 2; t++) {
                const int j = j0 + t * blockDim.x;
                if (j >= tl.count) continue;
                const int s = tl.start + j;
                T best = -INFINITY;
                int arg = sd.md.H;
#pragma unroll
                for (int k = 0; k < MH; k++) {
                    if (uk[t][k] > best) {
                        best = uk[t][k];
                        arg = k;
                    }
                }
                if (ud[t] > best) {
                    best = ud[t];
                    arg = sd.md.H;
                }
                if (V_out) V_out[sd.off + s] = best;
                if (pi) pi[sd.off + s] = arg;
                res = fmax(res, fabs(best - vin[t]));
                vabs = fmax(vabs, fabs(best));
            }
        }
        if (loop || res64) {
            res = block_max<T, kThreads>(res);
            vabs = block_max<T, kThreads>(vabs);
            if (threadIdx.x == 0) {
                if (loop)
                    close_instance(c, tl.inst, (float)res, (float)vabs, parity, parity ^ 1);
                else
                    atomicMax(&res64[tl.inst], dbits((double)res));
            }
        }
        __syncthreads();
    }
}

// Algorithm 4's in-block iteration for every active instance (VC_ITER_BLOCK).  The block
// tile table cuts each instance into chunks of whole sub-tiles; a sub-tile (tile.pad_
// states) is whole blocks of 2(Q_i+1)(C_i+1)^h_i states that block_tile iterates with one
// thread per state; a chunk loads its descriptor once and closes its share of the
// instance's sweep once.
template <int MH>
__global__ void __launch_bounds__(1024) k_bblock(const InstDesc* __restrict__ descs,
                                                 const BatchTile* __restrict__ tiles, int ntiles, BatchCtl c,
                                                 int parity, int passes, const float* __restrict__ U,
                                                 const float* __restrict__ U2, const float* __restrict__ V_in,
                                                 float* __restrict__ V_out) {
    extern __shared__ float bb_sm[];
    __shared__ InstDesc sd;
    __shared__ int skip;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        if (threadIdx.x == 0) skip = *((volatile int*)&c.done[tl.inst]) != 0;
        __syncthreads();
        if (skip) {
            __syncthreads();
            continue;
        }
        load_desc(descs, tl.inst, sd);
        __syncthreads();
        float res = 0.0f, vabs = 0.0f;
        const float* Vi = V_in + sd.off;
        const float* Ui = U + sd.off;
        const float* Wi = U2 + sd.off;
        float* Vo = V_out + sd.off;
        for (int s0 = tl.start; s0 < tl.start + tl.count; s0 += tl.pad_) {
            const int cnt = min(tl.pad_, tl.start + tl.count - s0);
            switch (sd.blk_h) {
                case 0: block_tile<MH, 0>(sd.md, sd.c32, s0, cnt, passes, Vi, Ui, Wi, Vo, bb_sm, nullptr, res, vabs); break;
                case 1: block_tile<MH, 1>(sd.md, sd.c32, s0, cnt, passes, Vi, Ui, Wi, Vo, bb_sm, nullptr, res, vabs); break;
                case 2: block_tile<MH, 2>(sd.md, sd.c32, s0, cnt, passes, Vi, Ui, Wi, Vo, bb_sm, nullptr, res, vabs); break;
                default: block_tile<MH, 3>(sd.md, sd.c32, s0, cnt, passes, Vi, Ui, Wi, Vo, bb_sm, nullptr, res, vabs); break;
            }
            __syncthreads();  // the next sub-tile reuses the shared arrays
        }
        res = block_max_dyn(res);
        vabs = block_max_dyn(vabs);
        if (threadIdx.x == 0) close_instance(c, tl.inst, res, vabs, parity, parity ^ 1);
        __syncthreads();
    }
}

// Whole-instance solve in one CTA for instances whose values fit in shared memory: the
// same Jacobi sweeps as the graph loop (k_bpost + k_bmax arithmetic, Eq. 18's backup or the
// self-transition solve) with V, U (and W) in shared memory, the instance's own step-3 test
// after every sweep (sweep_verdict, as close_instance applies it), and no kernel launch or
// grid-wide exchange per sweep: Algorithm 4's in-block iteration with the whole instance as
// the block.  Iterates and sweep counts are those of the graph loop bit for bit.  The
// result goes to Va (final_buf 0).  It runs on side streams concurrently with the graph
// loop, which skips these instances (k_bmark_small flags them before either starts and the
// loop's active count leaves them out).
template <int MH, bool SL>
__global__ void __launch_bounds__(512) k_bsmall(const InstDesc* __restrict__ descs, const int* __restrict__ list,
                                                 int nlist, BatchCtl c, float* __restrict__ Va) {
    extern __shared__ float sm_small[];
    __shared__ InstDesc sd;
    __shared__ int sh_done;
    for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
        const int inst = list[li];
        load_desc(descs, inst, sd);
        __syncthreads();
        const int S = sd.S;
        float* Vc = sm_small;          // current iterate
        float* Vn = sm_small + S;      // next iterate
        float* Us = sm_small + 2 * S;  // pass-1 values
        float* Ws = sm_small + 3 * S;  // defer's self-transition-solved values (SL)
        float* Vg = Va + sd.off;
        for (int j = threadIdx.x; j < S; j += blockDim.x) Vc[j] = Vg[j];
        const double tol = *c.tol * (c.tol_scale ? (double)c.tol_scale[inst] : 1.0);
        const long long max_sweeps = *c.max_sweeps;
        float best_res = INFINITY;
        int since_best = 0;
        long long k = 0;
        if (threadIdx.x == 0) sh_done = 0;
        __syncthreads();
        while (true) {
            for (int x = threadIdx.x; x < S; x += blockDim.x) {
                Digits d;
                decode<MH>(sd.md, x, d);
                const float rx = b_reward<MH>(sd.md, sd.c32, d);
                if constexpr (SL) {
                    float u, w;
                    post_and_defer<MH>(sd.md, sd.c32, Vc, x, d, rx, u, w);
                    Us[x] = u;
                    Ws[x] = w;
                } else {
                    Us[x] = rx + sd.c32.gamma * b_expect<MH>(sd.md, sd.c32, Vc, x, d);
                }
            }
            __syncthreads();
            float res = 0.0f, vabs = 0.0f;
            for (int s = threadIdx.x; s < S; s += blockDim.x) {
                Digits d;
                decode<MH>(sd.md, s, d);
                float best = -INFINITY;
                if (d.q >= 1) {
#pragma unroll
                    for (int kk = 0; kk < MH; kk++) {
                        if (kk < sd.md.H && d.occ[kk] < sd.md.C && (kk == sd.md.H - 1 || d.ph == 1)) {
                            const float u = Us[s + sd.md.stride[kk] - 2];
                            if (u > best) best = u;
                        }
                    }
                }
                const float u = SL ? Ws[s] : Us[s];
                if (u > best) best = u;
                Vn[s] = best;
                res = fmaxf(res, fabsf(best - Vc[s]));
                vabs = fmaxf(vabs, fabsf(best));
            }
            res = block_max_dyn(res);
            vabs = block_max_dyn(vabs);
            k++;
            if (threadIdx.x == 0) sh_done = sweep_verdict(tol, res, vabs, k, max_sweeps, best_res, since_best);
            __syncthreads();
            float* t = Vc;
            Vc = Vn;
            Vn = t;
            if (sh_done) break;
        }
        for (int j = threadIdx.x; j < S; j += blockDim.x) Vg[j] = Vc[j];
        if (threadIdx.x == 0) {
            c.sweeps[inst] = (int)k;
            c.final_buf[inst] = 0;
            c.done[inst] = sh_done;
        }
        __syncthreads();
    }
}

// Flags the instances of the whole-instance path so that the graph loop skips them.
__global__ void k_bmark_small(int* __restrict__ done, const int* __restrict__ list, int n) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) done[list[j]] = 5;
}

// Keeps the graph's while loop running while instances are active and budget remains.
__global__ void k_bcond(cudaGraphConditionalHandle h, BatchCtl c, int sweeps_per_body) {
    const long long it = *c.iters + sweeps_per_body;
    *c.iters = it;
    const int go = (*((volatile int*)c.active) > 0) && (it < *c.max_sweeps);
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Policy residual in FP64: r = U64(x_pi) - V64 (as float), U64 from the FP64 pass-1
// kernel over every post-decision state (one gather per state here).  Instances with a
// non-zero entry in `skipped` (nullable; already certified) get r = 0, so every correction
// solve retires them at its first step with a zero correction.
template <int MH>
__global__ void k_bresid64(const InstDesc* __restrict__ descs, const BatchTile* __restrict__ tiles, int ntiles,
                           const int32_t* __restrict__ pi, const double* __restrict__ U, const double* __restrict__ V,
                           float* __restrict__ r, int* err, const int* __restrict__ skipped) {
    __shared__ InstDesc sd;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        load_desc(descs, tl.inst, sd);
        __syncthreads();
        if (skipped && skipped[tl.inst]) {
            for (int j = threadIdx.x; j < tl.count; j += blockDim.x) r[sd.off + tl.start + j] = 0.0f;
            __syncthreads();
            continue;
        }
        const double* Ui = U + sd.off;
        const double* Vi = V + sd.off;
        for (int j = threadIdx.x; j < tl.count; j += blockDim.x) {
            const int s = tl.start + j;
            Digits d;
            decode<MH>(sd.md, s, d);
            int x = s;
            if (!apply_action<MH>(sd.md, s, pi[sd.off + s], d, x)) {
                atomicOr(err, kErrInfeasiblePolicy);
                r[sd.off + s] = 0.0f;
                continue;
            }
            r[sd.off + s] = (float)(Ui[x] - Vi[s]);
        }
        __syncthreads();
    }
}

// FP32 correction sweep e_out = r + gamma E[e_in(next) | x_pi] with per-instance close.
template <int MH>
__global__ void k_bcorr(const InstDesc* __restrict__ descs, const BatchTile* __restrict__ tiles, int ntiles,
                        BatchCtl c, int parity, const int32_t* __restrict__ pi, const float* __restrict__ r,
                        const float* __restrict__ e_in, float* __restrict__ e_out) {
    __shared__ InstDesc sd;
    __shared__ int skip;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        if (threadIdx.x == 0) skip = (*((volatile int*)&c.done[tl.inst]) != 0);
        __syncthreads();
        if (skip) {
            __syncthreads();
            continue;
        }
        load_desc(descs, tl.inst, sd);
        __syncthreads();
        const float* Ei = e_in + sd.off;
        float res = 0.0f, vabs = 0.0f;
        for (int j = threadIdx.x; j < tl.count; j += blockDim.x) {
            const int s = tl.start + j;
            Digits d;
            decode<MH>(sd.md, s, d);
            int x = s;
            apply_action<MH>(sd.md, s, pi[sd.off + s], d, x);  // feasibility checked by k_bresid64
            const float v = r[sd.off + s] + sd.c32.gamma * b_expect<MH>(sd.md, sd.c32, Ei, x, d);
            e_out[sd.off + s] = v;
            res = fmaxf(res, fabsf(v - Ei[s]));
            vabs = fmaxf(vabs, fabsf(v));
        }
        res = block_max<float, kThreads>(res);
        vabs = block_max<float, kThreads>(vabs);
        if (threadIdx.x == 0) close_instance(c, tl.inst, res, vabs, parity, parity ^ 1);
        __syncthreads();
    }
}

// ------------------------------------------------ batched BiCGSTAB correction solve
// The refinement's correction equations (I - gamma_i P_pi,i) e_i = r_i of every instance,
// solved together by BiCGSTAB (one iteration = five kernels over the tile table, one
// graph-loop pass).  Every reducing kernel writes one partial per tile; the instance's
// last tile (ticket) sums the instance's tile partials in tile order and advances the
// instance's scalars, and retires the instance once its residual is below its target.
struct BatchKrylov {
    double *rho, *alpha, *omega, *beta, *target;  // [n] per-instance scalars
    float* rmax;                                  // [n] max |r| after the last iteration
    int* done;                                    // [n] 0 running, 1 converged, 2 cap, 5 breakdown
    int* iter;                                    // [n] iterations completed
    unsigned int* ticket;                         // [n] arrivals of the current kernel
    const int* tiles_of;                          // [n] tiles per instance
    const int* tile_first;                        // [n] first tile of each instance
    double* part;                                 // [ntiles][3] tile partials
    int* active;                                  // instances still iterating
    long long* iters;                             // graph-loop passes
    const long long* max_iter;
    const float* b;                               // right-hand sides (policy residuals)
    float *x, *r, *p, *v, *s, *t;                 // concatenated vectors
};

// Scalars of instance i after `stage`, from its totals (one thread).
__device__ void bkr_advance(const BatchKrylov& K, int i, int stage, double d0, double d1, double mx) {
    int done = 0;
    if (stage == kKrInit) {
        K.rho[i] = d0;
        K.rmax[i] = (float)mx;
        K.alpha[i] = K.omega[i] = 1.0;
        K.beta[i] = 0.0;
        K.iter[i] = 0;
        K.target[i] = fmax(K.target[i], ldexp(mx, -18));  // the reach of one FP32 solve
        if (mx < K.target[i]) done = 1;
        else if (!(d0 > 0.0)) done = 5;
    } else if (stage == kKrV) {
        if (d0 == 0.0 || !isfinite(d0)) done = 5;
        else K.alpha[i] = K.rho[i] / d0;
    } else if (stage == kKrT) {
        const double om = (d1 > 0.0) ? d0 / d1 : 0.0;
        K.omega[i] = om;
        if (!isfinite(om)) done = 5;
    } else {
        K.rmax[i] = (float)mx;
        const int it = K.iter[i] + 1;
        K.iter[i] = it;
        if (mx < K.target[i]) {
            done = 1;
        } else if (it >= *K.max_iter) {
            done = 2;
        } else if (K.omega[i] == 0.0 || K.rho[i] == 0.0 || !isfinite(mx)) {
            done = 5;
        } else {
            const double be = (d0 / K.rho[i]) * (K.alpha[i] / K.omega[i]);
            K.beta[i] = be;
            K.rho[i] = d0;
            if (!isfinite(be) || d0 == 0.0) done = 5;
        }
    }
    K.ticket[i] = 0;
    if (done) {
        K.done[i] = done;
        atomicSub(K.active, 1);
    }
    __threadfence();
}

// Tile epilogue of a reducing kernel: every thread of the block calls it once per tile.
__device__ void bkr_tile_finish(const BatchKrylov& K, int tile, int inst, int stage, float d0, float d1, float mx) {
    __shared__ int last;
    const double s0 = block_sum<kThreads>((double)d0);
    const double s1 = block_sum<kThreads>((double)d1);
    const float m = block_max<float, kThreads>(mx);
    if (threadIdx.x == 0) {
        K.part[3 * (long long)tile] = s0;
        K.part[3 * (long long)tile + 1] = s1;
        K.part[3 * (long long)tile + 2] = (double)m;
        __threadfence();
        last = (atomicAdd(&K.ticket[inst], 1u) == (unsigned)K.tiles_of[inst] - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const long long t0 = K.tile_first[inst];
    const int nt = K.tiles_of[inst];
    double a0 = 0.0, a1 = 0.0, am = 0.0;
    for (int j = threadIdx.x; j < nt; j += kThreads) {
        a0 += __ldcg(K.part + 3 * (t0 + j));
        a1 += __ldcg(K.part + 3 * (t0 + j) + 1);
        am = fmax(am, __ldcg(K.part + 3 * (t0 + j) + 2));
    }
    a0 = block_sum<kThreads>(a0);
    a1 = block_sum<kThreads>(a1);
    am = block_max<double, kThreads>(am);
    if (threadIdx.x == 0) bkr_advance(K, inst, stage, a0, a1, am);
    __syncthreads();
}

__device__ __forceinline__ bool bkr_skip(const BatchKrylov& K, int inst) {
    __shared__ int skip;
    if (threadIdx.x == 0) skip = *((volatile int*)&K.done[inst]) != 0;
    __syncthreads();
    const bool r = skip != 0;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kThreads) k_bkr_init(const InstDesc* __restrict__ descs,
                                                       const BatchTile* __restrict__ tiles, int ntiles, BatchKrylov K) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        if (bkr_skip(K, tl.inst)) continue;
        const long long off = descs[tl.inst].off + tl.start;
        float d0 = 0.0f, mx = 0.0f;
        for (int j = threadIdx.x; j < tl.count; j += kThreads) {
            const float bv = K.b[off + j];
            K.r[off + j] = bv;
            K.x[off + j] = 0.0f;
            d0 = fmaf(bv, bv, d0);
            mx = fmaxf(mx, fabsf(bv));
        }
        bkr_tile_finish(K, t, tl.inst, kKrInit, d0, 0.0f, mx);
    }
}

__global__ void __launch_bounds__(kThreads) k_bkr_p(const InstDesc* __restrict__ descs,
                                                    const BatchTile* __restrict__ tiles, int ntiles, BatchKrylov K) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        if (bkr_skip(K, tl.inst)) continue;
        const long long off = descs[tl.inst].off + tl.start;
        const bool first = K.iter[tl.inst] == 0;
        const float be = (float)K.beta[tl.inst], om = (float)K.omega[tl.inst];
        for (int j = threadIdx.x; j < tl.count; j += kThreads)
            K.p[off + j] = first ? K.r[off + j] : fmaf(be, fmaf(-om, K.v[off + j], K.p[off + j]), K.r[off + j]);
    }
}

__global__ void __launch_bounds__(kThreads) k_bkr_s(const InstDesc* __restrict__ descs,
                                                    const BatchTile* __restrict__ tiles, int ntiles, BatchKrylov K) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        if (bkr_skip(K, tl.inst)) continue;
        const long long off = descs[tl.inst].off + tl.start;
        const float al = (float)K.alpha[tl.inst];
        for (int j = threadIdx.x; j < tl.count; j += kThreads) K.s[off + j] = fmaf(-al, K.v[off + j], K.r[off + j]);
    }
}

__global__ void __launch_bounds__(kThreads) k_bkr_x(const InstDesc* __restrict__ descs,
                                                    const BatchTile* __restrict__ tiles, int ntiles, BatchKrylov K) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        if (bkr_skip(K, tl.inst)) continue;
        const long long off = descs[tl.inst].off + tl.start;
        const float al = (float)K.alpha[tl.inst], om = (float)K.omega[tl.inst];
        float d0 = 0.0f, mx = 0.0f;
        for (int j = threadIdx.x; j < tl.count; j += kThreads) {
            const long long g = off + j;
            const float sv = K.s[g];
            K.x[g] += fmaf(al, K.p[g], om * sv);
            const float rv = fmaf(-om, K.t[g], sv);
            K.r[g] = rv;
            d0 = fmaf(K.b[g], rv, d0);
            mx = fmaxf(mx, fabsf(rv));
        }
        bkr_tile_finish(K, t, tl.inst, kKrX, d0, 0.0f, mx);
    }
}

// y = x - gamma_i E[x(next) | x_pi(s)] per instance, with the stage's partial sums <w, y>
// and <y, y>.  The policy was checked feasible by k_bresid64.
template <int MH>
__global__ void __launch_bounds__(kThreads) k_bkr_apply(const InstDesc* __restrict__ descs,
                                                        const BatchTile* __restrict__ tiles, int ntiles,
                                                        const int32_t* __restrict__ pi, const float* __restrict__ xin,
                                                        float* __restrict__ y, const float* __restrict__ w, int stage,
                                                        BatchKrylov K) {
    __shared__ InstDesc sd;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        if (bkr_skip(K, tl.inst)) continue;
        load_desc(descs, tl.inst, sd);
        __syncthreads();
        const float* Xi = xin + sd.off;
        float d0 = 0.0f, d1 = 0.0f;
        for (int j = threadIdx.x; j < tl.count; j += kThreads) {
            const int s = tl.start + j;
            const long long g = sd.off + s;
            Digits d;
            decode<MH>(sd.md, s, d);
            int x = s;
            float yv = Xi[s];
            if (apply_action<MH>(sd.md, s, pi[g], d, x)) yv -= sd.c32.gamma * b_expect<MH>(sd.md, sd.c32, Xi, x, d);
            y[g] = yv;
            d0 = fmaf(w[g], yv, d0);
            d1 = fmaf(yv, yv, d1);
        }
        bkr_tile_finish(K, t, tl.inst, stage, d0, d1, 0.0f);
    }
}

// Keeps the BiCGSTAB graph loop running while instances iterate and the budget lasts.
__global__ void k_bkr_cond(cudaGraphConditionalHandle h, BatchKrylov K) {
    const long long it = *K.iters + 1;
    *K.iters = it;
    const int go = (*((volatile int*)K.active) > 0) && (it < *K.max_iter);
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// Per-instance start of a solve: target (x tol_scale), counters cleared.
__global__ void k_bkr_reset(BatchKrylov K, int n, double target, const float* tol_scale) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        K.done[i] = 0;
        K.iter[i] = 0;
        K.ticket[i] = 0u;
        K.target[i] = target * (double)tol_scale[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *K.active = n;
        *K.iters = 0;
    }
}

// Per-instance selection of the final ping-pong buffer into out (float or double).
template <typename TI, typename TO>
__global__ void k_bselect(const InstDesc* __restrict__ descs, const BatchTile* __restrict__ tiles, int ntiles,
                          const int* __restrict__ final_buf, const TI* __restrict__ A, const TI* __restrict__ B,
                          TO* __restrict__ out) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        const long long off = descs[tl.inst].off;
        const TI* src = final_buf[tl.inst] ? B : A;
        for (int j = threadIdx.x; j < tl.count; j += blockDim.x) {
            const long long g = off + tl.start + j;
            out[g] = (TO)src[g];
        }
    }
}

__global__ void k_baxpy(const float* __restrict__ A, const float* __restrict__ B, const InstDesc* __restrict__ descs,
                        const BatchTile* __restrict__ tiles, int ntiles, const int* __restrict__ final_buf,
                        double* __restrict__ V64) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        const long long off = descs[tl.inst].off;
        const float* src = final_buf[tl.inst] ? B : A;
        for (int j = threadIdx.x; j < tl.count; j += blockDim.x) {
            const long long g = off + tl.start + j;
            V64[g] += (double)src[g];
        }
    }
}

__global__ void k_binit(BatchCtl c, int n, int active) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        c.done[i] = 0;
        c.sweeps[i] = 0;
        c.ticket[i] = 0;
        c.final_buf[i] = 0;
        c.since_best[i] = 0;
        c.best_res[i] = INFINITY;
        c.res32[2 * i] = c.res32[2 * i + 1] = 0u;
        c.vmax32[2 * i] = c.vmax32[2 * i + 1] = 0u;
        c.res64[i] = 0ull;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *c.active = active;
        *c.iters = 0;
    }
}

__global__ void k_f32_to_f64_n(const float* __restrict__ in, double* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

// Calls f with std::integral_constant<int, MH>: MH = the batch's largest H when it is at
// most 8 (per-host loops unrolled to exactly that bound), else 16.
template <typename F>
static void by_mh(int mh, F&& f) {
    switch (mh) {
        case 1: f(std::integral_constant<int, 1>()); break;
        case 2: f(std::integral_constant<int, 2>()); break;
        case 3: f(std::integral_constant<int, 3>()); break;
        case 4: f(std::integral_constant<int, 4>()); break;
        case 5: f(std::integral_constant<int, 5>()); break;
        case 6: f(std::integral_constant<int, 6>()); break;
        case 7: f(std::integral_constant<int, 7>()); break;
        case 8: f(std::integral_constant<int, 8>()); break;
        default: f(std::integral_constant<int, 16>()); break;
    }
}

// ------------------------------------------------------------------------ batch handle
struct Batch {
    int n = 0;
    long long total = 0;
    int mh = 8;
    int ts = 4096;    // states per tile (default: the fastest measured on the 512-instance batch)
    int bps = 8;      // blocks per SM of the persistent grid
    int grid = 0;
    int ntiles = 0;
    int num_sms = 0;
    std::vector<InstDesc> h_desc;
    std::vector<int> h_tiles_of;
    InstDesc* d_desc = nullptr;
    BatchTile* d_tiles = nullptr;
    float *Va = nullptr, *Vb = nullptr, *U = nullptr, *U2 = nullptr, *E0 = nullptr, *E1 = nullptr, *Rr = nullptr;
    double *V64 = nullptr, *V64b = nullptr, *U64 = nullptr;
    int32_t *pi = nullptr, *pi2 = nullptr;
    int *done = nullptr, *sweeps = nullptr, *ticket = nullptr, *tiles_of = nullptr, *final_buf = nullptr,
        *since_best = nullptr, *active = nullptr, *err = nullptr;
    float* best_res = nullptr;
    unsigned int *res32 = nullptr, *vmax32 = nullptr;
    unsigned long long* res64 = nullptr;
    long long* iters = nullptr;
    long long* max_d = nullptr;
    double* tol_d = nullptr;
    float* tol_scale = nullptr;  // per-instance factor of the correction loop's tolerance
    int* certified = nullptr;    // [n] 1: certified in an earlier refinement round (skipped)
    // BiCGSTAB correction solve: vectors r, p, v, s, t ([5][total]; x is E0), tile partials,
    // per-instance scalars
    float* kr = nullptr;
    double* kr_part = nullptr;  // [ntiles][3], sized with the tile table
    double *kr_rho = nullptr, *kr_alpha = nullptr, *kr_omega = nullptr, *kr_beta = nullptr, *kr_target = nullptr;
    float* kr_rmax = nullptr;
    int *kr_done = nullptr, *kr_iter = nullptr, *tile_first = nullptr;
    unsigned int* kr_ticket = nullptr;
    long long* kr_max_d = nullptr;
    // in-block iteration (VC_ITER_BLOCK): tiles of whole blocks of at most blk_threads states
    bool pairs = false;  // every tile of d_tiles starts and ends on an even state (paired loop kernels)
    int blk_threads = 512;
    int blk_passes = 4;
    int blk_grid = 0;
    int nbtiles = 0;
    std::vector<int> h_btiles_of;
    BatchTile* d_btiles = nullptr;
    int* btiles_of = nullptr;
    // instances solved whole in one CTA's shared memory (k_bsmall) before the graph loop
    int small_cap = 0;       // states that fit: (opt-in shared memory - reserve) / 16 bytes
    int small_max = 0;       // instances with S <= small_max take that path (0: none)
    int n_small = 0;
    int* d_small = nullptr;  // the instances, grouped by size class
    // size classes (largest S of a class at most small_cap / 8, / 4, / 2, / 1): each class
    // is one launch on its own side stream with shared memory for its largest instance
    static constexpr int kSmallClasses = 4;
    int cls_first[kSmallClasses] = {0, 0, 0, 0};
    int cls_count[kSmallClasses] = {0, 0, 0, 0};
    int cls_S[kSmallClasses] = {0, 0, 0, 0};
    cudaStream_t side[kSmallClasses] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kSmallClasses] = {nullptr, nullptr, nullptr, nullptr};
    cudaGraph_t g_vi = nullptr, g_vi_sl = nullptr, g_corr = nullptr, g_kry = nullptr, g_vi_blk = nullptr;
    cudaGraphExec_t x_vi = nullptr, x_vi_sl = nullptr, x_corr = nullptr, x_kry = nullptr, x_vi_blk = nullptr;
    std::vector<void*> owned;
    int64_t device_bytes = 0;
    std::string tune_report;
};

static int balloc(Batch* b, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(VC_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    b->owned.push_back(*p);
    b->device_bytes += (int64_t)bytes;
    return VC_OK;
}

static BatchCtl ctl_of(Batch* b, bool scaled = false) {
    BatchCtl c;
    c.tol_scale = scaled ? b->tol_scale : nullptr;
    c.done = b->done;
    c.sweeps = b->sweeps;
    c.ticket = b->ticket;
    c.tiles_of = b->tiles_of;
    c.final_buf = b->final_buf;
    c.since_best = b->since_best;
    c.best_res = b->best_res;
    c.res32 = b->res32;
    c.vmax32 = b->vmax32;
    c.res64 = b->res64;
    c.active = b->active;
    c.iters = b->iters;
    c.max_sweeps = b->max_d;
    c.tol = b->tol_d;
    return c;
}

static BatchKrylov kry_of(Batch* b) {
    BatchKrylov K;
    const size_t T = (size_t)b->total;
    K.rho = b->kr_rho;
    K.alpha = b->kr_alpha;
    K.omega = b->kr_omega;
    K.beta = b->kr_beta;
    K.target = b->kr_target;
    K.rmax = b->kr_rmax;
    K.done = b->kr_done;
    K.iter = b->kr_iter;
    K.ticket = b->kr_ticket;
    K.tiles_of = b->tiles_of;
    K.tile_first = b->tile_first;
    K.part = b->kr_part;
    K.active = b->active;
    K.iters = b->iters;
    K.max_iter = b->kr_max_d;
    K.b = b->Rr;
    K.x = b->E0;
    K.r = b->kr;
    K.p = b->kr + T;
    K.v = b->kr + 2 * T;
    K.s = b->kr + 3 * T;
    K.t = b->kr + 4 * T;
    return K;
}

// Destroys every captured loop graph.  The graphs hold the tile tables' device addresses,
// so they go before a table is freed or rebuilt: a failed rebuild then leaves no graph that
// could run on freed memory, and the solves refuse to start until build_graphs succeeds.
static std::string g_destroy_note;  // first failed destroy (diagnostics)

static void destroy_graphs(Batch* b) {
    cudaGraphExec_t* xs[] = {&b->x_vi, &b->x_vi_sl, &b->x_vi_blk, &b->x_corr, &b->x_kry};
    cudaGraph_t* gs[] = {&b->g_vi, &b->g_vi_sl, &b->g_vi_blk, &b->g_corr, &b->g_kry};
    int k = 0;
    for (auto* x : xs) {
        if (*x) {
            const cudaError_t e = cudaGraphExecDestroy(*x);
            if (e != cudaSuccess && g_destroy_note.empty())
                g_destroy_note = "exec " + std::to_string(k) + ": " + cudaGetErrorString(e);
        }
        *x = nullptr;
        k++;
    }
    k = 0;
    for (auto* g : gs) {
        if (*g) {
            const cudaError_t e = cudaGraphDestroy(*g);
            if (e != cudaSuccess && g_destroy_note.empty())
                g_destroy_note = "graph " + std::to_string(k) + ": " + cudaGetErrorString(e);
        }
        *g = nullptr;
        k++;
    }
}

static bool graphs_ready(const Batch* b) { return b->x_vi && b->x_vi_sl && b->x_vi_blk && b->x_corr && b->x_kry; }

// Tile table for tile size ts; tiles of an instance are contiguous in the table.
static int build_tiles(Batch* b, cudaStream_t st) {
    destroy_graphs(b);
    std::vector<BatchTile> tiles;
    b->h_tiles_of.assign(b->n, 0);
    for (int i = 0; i < b->n; i++) {
        const int S = b->h_desc[i].S;
        for (int s0 = 0; s0 < S; s0 += b->ts) {
            BatchTile t;
            t.inst = i;
            t.start = s0;
            t.count = std::min(b->ts, S - s0);
            t.pad_ = 0;
            tiles.push_back(t);
            b->h_tiles_of[i]++;
        }
    }
    b->ntiles = (int)tiles.size();
    // the paired loop kernels need every tile to start and end on an even state (tile sizes
    // and instance sizes 2(Q+1)(C+1)^H are even; checked rather than assumed)
    b->pairs = true;
    for (const BatchTile& t : tiles) b->pairs = b->pairs && (t.start % 2 == 0) && (t.count % 2 == 0);
    std::vector<int> first(b->n, 0);
    for (int i = 1; i < b->n; i++) first[i] = first[i - 1] + b->h_tiles_of[i - 1];
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->kr_part) cudaFree(b->kr_part);
    b->d_tiles = nullptr;
    b->kr_part = nullptr;
    VC_CUDA(cudaMalloc((void**)&b->d_tiles, sizeof(BatchTile) * tiles.size()));
    VC_CUDA(cudaMalloc((void**)&b->kr_part, 3 * sizeof(double) * tiles.size()));
    VC_CUDA(cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(BatchTile) * tiles.size(), cudaMemcpyHostToDevice, st));
    VC_CUDA(cudaMemcpyAsync(b->tiles_of, b->h_tiles_of.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, st));
    VC_CUDA(cudaMemcpyAsync(b->tile_first, first.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, st));
    VC_CUDA(cudaStreamSynchronize(st));
    b->grid = std::max(1, std::min(b->ntiles, b->num_sms * b->bps));
    return VC_OK;
}

constexpr int kBlockChunk = 2048;  // states per chunk of the batched in-block iteration

// Block tile table of the in-block iteration: per instance the largest h with a block of
// B = 2(Q+1)(C+1)^h <= blk_threads states, tiles of floor(blk_threads / B) whole blocks
// (the last one shorter), tiles of an instance contiguous.
static int build_block_tiles(Batch* b, cudaStream_t st) {
    destroy_graphs(b);
    std::vector<BatchTile> tiles;
    b->h_btiles_of.assign(b->n, 0);
    for (int i = 0; i < b->n; i++) {
        InstDesc& d = b->h_desc[i];
        int h = 0;
        long long B = 2LL * (d.md.Q + 1);
        while (h < d.md.H && h < kBlockMaxInner && B * (d.md.C + 1) <= b->blk_threads) {
            B *= (d.md.C + 1);
            h++;
        }
        if (B > b->blk_threads) return fail(VC_ERR_ARG, "an instance's smallest block exceeds the block threads");
        d.blk_h = h;
        const int T = (int)(B * (b->blk_threads / B));        // sub-tile: whole blocks
        const int chunk = T * std::max(1, kBlockChunk / T);    // chunk: whole sub-tiles
        for (int s0 = 0; s0 < d.S; s0 += chunk) {
            BatchTile t;
            t.inst = i;
            t.start = s0;
            t.count = std::min(chunk, d.S - s0);
            t.pad_ = T;
            tiles.push_back(t);
            b->h_btiles_of[i]++;
        }
    }
    b->nbtiles = (int)tiles.size();
    if (b->d_btiles) cudaFree(b->d_btiles);
    b->d_btiles = nullptr;
    VC_CUDA(cudaMalloc((void**)&b->d_btiles, sizeof(BatchTile) * tiles.size()));
    VC_CUDA(cudaMemcpyAsync(b->d_btiles, tiles.data(), sizeof(BatchTile) * tiles.size(), cudaMemcpyHostToDevice, st));
    VC_CUDA(cudaMemcpyAsync(b->btiles_of, b->h_btiles_of.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, st));
    VC_CUDA(cudaMemcpyAsync(b->d_desc, b->h_desc.data(), sizeof(InstDesc) * b->n, cudaMemcpyHostToDevice, st));
    VC_CUDA(cudaStreamSynchronize(st));
    b->blk_grid = 0;
    return VC_OK;
}

// List of the instances solved whole in one CTA (S <= small_max), grouped into size
// classes and uploaded for k_bsmall.
static int build_small_list(Batch* b, cudaStream_t st) {
    std::vector<int> list;
    b->n_small = 0;
    for (int c = 0; c < Batch::kSmallClasses; c++) {
        const int hi = b->small_cap >> (Batch::kSmallClasses - 1 - c);
        const int lo = c == 0 ? 0 : (b->small_cap >> (Batch::kSmallClasses - c));
        b->cls_first[c] = (int)list.size();
        b->cls_S[c] = 0;
        for (int i = 0; i < b->n; i++) {
            const int S = b->h_desc[i].S;
            if (S <= b->small_max && S > lo && S <= hi) {
                list.push_back(i);
                b->cls_S[c] = std::max(b->cls_S[c], S);
            }
        }
        b->cls_count[c] = (int)list.size() - b->cls_first[c];
    }
    b->n_small = (int)list.size();
    if (b->d_small) cudaFree(b->d_small);
    b->d_small = nullptr;
    if (list.empty()) return VC_OK;
    VC_CUDA(cudaMalloc((void**)&b->d_small, sizeof(int) * list.size()));
    VC_CUDA(cudaMemcpyAsync(b->d_small, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, st));
    VC_CUDA(cudaStreamSynchronize(st));
    return VC_OK;
}

// Starts the whole-instance solves (Eq. 18's backup, or the self-transition solve: SL,
// which the in-block iteration uses for a whole-instance block): flags them for the loop
// on `st`, then one launch per size class on its side stream, forked from `st`.
template <int MH>
static int launch_small(Batch* b, bool sl, cudaStream_t st) {
    if (b->n_small == 0) return VC_OK;
    count_launches(1);
    k_bmark_small<<<(b->n_small + 255) / 256, 256, 0, st>>>(b->done, b->d_small, b->n_small);
    VC_LAUNCHED("k_bmark_small");
    VC_CUDA(cudaEventRecord(b->fork_ev, st));
    auto kern = sl ? k_bsmall<MH, true> : k_bsmall<MH, false>;
    for (int c = 0; c < Batch::kSmallClasses; c++) {
        if (b->cls_count[c] == 0) continue;
        const size_t smem = 16 * (size_t)b->cls_S[c];
        const int threads = b->cls_S[c] <= 2048 ? 128 : b->cls_S[c] <= 4096 ? 256 : 512;
        VC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        VC_CUDA(cudaStreamWaitEvent(b->side[c], b->fork_ev, 0));
        count_launches(1);
        kern<<<b->cls_count[c], threads, smem, b->side[c]>>>(b->d_desc, b->d_small + b->cls_first[c],
                                                              b->cls_count[c], ctl_of(b), b->Va);
        VC_LAUNCHED("the whole-instance kernel");
        VC_CUDA(cudaEventRecord(b->join_ev[c], b->side[c]));
    }
    return VC_OK;
}

// Makes `st` wait for the whole-instance solves.
static int join_small(Batch* b, cudaStream_t st) {
    for (int c = 0; c < Batch::kSmallClasses; c++)
        if (b->n_small && b->cls_count[c]) VC_CUDA(cudaStreamWaitEvent(st, b->join_ev[c], 0));
    return VC_OK;
}

// Kernels in one pass of each loop body (two sweeps per pass); the launch counter adds
// passes x this after every graph launch, since the graph runs them without a host call.
// The paired loop kernels serve batches whose tiles are all even and whose largest H is
// at most 5 (above it pass 1's pair of states no longer fits its register budget).
template <int MH>
static bool pairs_ok(const Batch* b) {
    return b->pairs && MH <= 5;
}

constexpr int kViBodyKernels = 5;
constexpr int kCorrBodyKernels = 3;
constexpr int kKryBodyKernels = 6;      // one BiCGSTAB iteration per pass
constexpr long long kKrylovMaxIter = 1000;

template <int MH, bool SL>
static void enqueue_vi_body(Batch* b, cudaStream_t cs, cudaGraphConditionalHandle h) {
    const BatchCtl c = ctl_of(b);
    float* U2 = SL ? b->U2 : nullptr;
    if (pairs_ok<MH>(b)) {
        // the loop over pairs of states (every tile starts and ends on an even state)
        k_bpost_pair<MH, SL><<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, b->done, b->Va, b->U, U2);
        k_bmax_pair<MH, SL><<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, c, 0, b->U, U2, b->Va,
                                                          b->Vb);
        k_bpost_pair<MH, SL><<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, b->done, b->Vb, b->U, U2);
        k_bmax_pair<MH, SL><<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, c, 1, b->U, U2, b->Vb,
                                                          b->Va);
        k_bcond<<<1, 1, 0, cs>>>(h, c, 2);
        return;
    }
    k_bpost<MH, float, SL><<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, b->done, b->Va, b->U, U2);
    k_bmax<MH, float, SL><<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, c, 1, 0, b->U, U2, b->Va,
                                                         b->Vb, nullptr, nullptr);
    k_bpost<MH, float, SL><<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, b->done, b->Vb, b->U, U2);
    k_bmax<MH, float, SL><<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, c, 1, 1, b->U, U2, b->Vb,
                                                         b->Va, nullptr, nullptr);
    k_bcond<<<1, 1, 0, cs>>>(h, c, 2);
}

template <int MH>
static void enqueue_vi_blk_body(Batch* b, cudaStream_t cs, cudaGraphConditionalHandle h) {
    BatchCtl c = ctl_of(b);
    c.tiles_of = b->btiles_of;  // the block tiles close each instance's sweep
    const int threads = (b->blk_threads + 31) / 32 * 32;
    const size_t smem = 4 * sizeof(float) * (size_t)threads;
    k_bpost<MH, float, true><<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, b->done, b->Va, b->U,
                                                           b->U2);
    k_bblock<MH><<<b->blk_grid, threads, smem, cs>>>(b->d_desc, b->d_btiles, b->nbtiles, c, 0, b->blk_passes, b->U,
                                                    b->U2, b->Va, b->Vb);
    k_bpost<MH, float, true><<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, b->done, b->Vb, b->U,
                                                           b->U2);
    k_bblock<MH><<<b->blk_grid, threads, smem, cs>>>(b->d_desc, b->d_btiles, b->nbtiles, c, 1, b->blk_passes, b->U,
                                                    b->U2, b->Vb, b->Va);
    k_bcond<<<1, 1, 0, cs>>>(h, c, 2);
}

template <int MH>
static void enqueue_corr_body(Batch* b, cudaStream_t cs, cudaGraphConditionalHandle h) {
    const BatchCtl c = ctl_of(b, true);
    k_bcorr<MH><<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, c, 0, b->pi, b->Rr, b->E0, b->E1);
    k_bcorr<MH><<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, c, 1, b->pi, b->Rr, b->E1, b->E0);
    k_bcond<<<1, 1, 0, cs>>>(h, c, 2);
}

template <int MH>
static void enqueue_kry_body(Batch* b, cudaStream_t cs, cudaGraphConditionalHandle h) {
    const BatchKrylov K = kry_of(b);
    k_bkr_p<<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, K);
    k_bkr_apply<MH><<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, b->pi, K.p, K.v, K.b, kKrV, K);
    k_bkr_s<<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, K);
    k_bkr_apply<MH><<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, b->pi, K.s, K.t, K.s, kKrT, K);
    k_bkr_x<<<b->grid, kThreads, 0, cs>>>(b->d_desc, b->d_tiles, b->ntiles, K);
    k_bkr_cond<<<1, 1, 0, cs>>>(h, K);
}

// One graph: a WHILE node (default condition 1 at every launch) whose body is built by
// capturing `body` on a private stream.
template <typename Body>
static int make_loop_graph(cudaGraph_t* g, cudaGraphExec_t* x, const std::string& name, Body&& body) {
    if (*x) cudaGraphExecDestroy(*x);
    if (*g) cudaGraphDestroy(*g);
    *x = nullptr;
    *g = nullptr;
    VC_CUDA(cudaGraphCreate(g, 0));
    cudaGraphConditionalHandle h;
    VC_CUDA(cudaGraphConditionalHandleCreate(&h, *g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    VC_CUDA(cudaGraphAddNode(&node, *g, nullptr, nullptr, 0, &cp));
    cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
    cudaStream_t cs;
    VC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    VC_CUDA(cudaStreamBeginCaptureToGraph(cs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    body(cs, h);
    const cudaError_t le = cudaGetLastError();  // a launch refused while capturing
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (captured && captured != bodyg) cudaGraphDestroy(captured);
        cudaGraphDestroy(*g);
        *g = nullptr;
        if (le != cudaSuccess)
            return cuda_fail(le, ("kernel launch while capturing the batched loop body (" + name + ")").c_str());
        return cuda_fail(e, "cudaStreamEndCapture (batched loop body)");
    }
    VC_CUDA(cudaGraphInstantiate(x, *g, 0));
    return VC_OK;
}

// Resident grid of the batched in-block kernel for the current block threads (queried
// before any capture; a failed query falls back to one CTA per SM).
template <int MH>
static void block_grid_of(Batch* b) {
    const int threads = (b->blk_threads + 31) / 32 * 32;
    const size_t smem = 4 * sizeof(float) * (size_t)threads;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bblock<MH>, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    b->blk_grid = std::max(1, std::min(b->nbtiles, std::max(1, per_sm) * b->num_sms));
}

static int build_graphs_once(Batch* b);

// Captures every loop graph, all or nothing: after a failure no graph is left.
static int build_graphs(Batch* b) {
    destroy_graphs(b);
    const int rc = build_graphs_once(b);
    if (rc) destroy_graphs(b);
    return rc;
}

static int build_graphs_once(Batch* b) {
    int rc;
    {
        const cudaError_t pe = cudaGetLastError();
        if (pe != cudaSuccess)
            return cuda_fail(pe, ("pending before the graph captures; destroy note: " + g_destroy_note).c_str());
    }
    by_mh(b->mh, [&](auto m) { block_grid_of<decltype(m)::value>(b); });
    VC_LAUNCHED("pending after the block-kernel occupancy query");
    auto vi = [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
        by_mh(b->mh, [&](auto m) { enqueue_vi_body<decltype(m)::value, false>(b, cs, h); });
    };
    auto vi_sl = [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
        by_mh(b->mh, [&](auto m) { enqueue_vi_body<decltype(m)::value, true>(b, cs, h); });
    };
    auto corr = [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
        by_mh(b->mh, [&](auto m) { enqueue_corr_body<decltype(m)::value>(b, cs, h); });
    };
    auto kry = [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
        by_mh(b->mh, [&](auto m) { enqueue_kry_body<decltype(m)::value>(b, cs, h); });
    };
    if ((rc = make_loop_graph(&b->g_vi, &b->x_vi, "Eq. 18 loop", vi))) return rc;
    if ((rc = make_loop_graph(&b->g_vi_sl, &b->x_vi_sl, "self-transition loop", vi_sl))) return rc;
    auto vi_blk = [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
        by_mh(b->mh, [&](auto m) { enqueue_vi_blk_body<decltype(m)::value>(b, cs, h); });
    };
    const std::string blk = "in-block loop: grid " + std::to_string(b->blk_grid) + " threads " +
                            std::to_string((b->blk_threads + 31) / 32 * 32) + " tiles " + std::to_string(b->nbtiles);
    if ((rc = make_loop_graph(&b->g_vi_blk, &b->x_vi_blk, blk, vi_blk))) return rc;
    if ((rc = make_loop_graph(&b->g_corr, &b->x_corr, "correction loop", corr))) return rc;
    if ((rc = make_loop_graph(&b->g_kry, &b->x_kry, "BiCGSTAB loop", kry))) return rc;
    return VC_OK;
}

static void free_batch(Batch* b) {
    if (!b) return;
    destroy_graphs(b);
    for (int c = 0; c < Batch::kSmallClasses; c++) {
        if (b->side[c]) cudaStreamDestroy(b->side[c]);
        if (b->join_ev[c]) cudaEventDestroy(b->join_ev[c]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    if (b->d_btiles) cudaFree(b->d_btiles);
    if (b->d_small) cudaFree(b->d_small);
    for (void* p : b->owned) cudaFree(p);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->kr_part) cudaFree(b->kr_part);
    delete b;
}

static int reset_loop(Batch* b, double tol, long long max_sweeps, cudaStream_t st, int skipped = 0) {
    VC_CUDA(cudaMemcpyAsync(b->tol_d, &tol, sizeof(double), cudaMemcpyHostToDevice, st));
    VC_CUDA(cudaMemcpyAsync(b->max_d, &max_sweeps, sizeof(long long), cudaMemcpyHostToDevice, st));
    count_launches(1);
    k_binit<<<(b->n + 255) / 256, 256, 0, st>>>(ctl_of(b), b->n, b->n - skipped);
    VC_LAUNCHED("k_binit");
    // the parameters live in pageable host memory: make the copies complete before return
    VC_CUDA(cudaStreamSynchronize(st));
    return VC_OK;
}

template <int MH>
static void enqueue_extract(Batch* b, const float* V, int32_t* pi, cudaStream_t st) {
    if (pairs_ok<MH>(b))
        k_bpost_pair<MH, false><<<b->grid, kThreads, 0, st>>>(b->d_desc, b->d_tiles, b->ntiles, nullptr, V, b->U,
                                                              nullptr);
    else
        k_bpost<MH, float, false><<<b->grid, kThreads, 0, st>>>(b->d_desc, b->d_tiles, b->ntiles, nullptr, V, b->U,
                                                                nullptr);
    k_bmax<MH, float, false><<<b->grid, kThreads, 0, st>>>(b->d_desc, b->d_tiles, b->ntiles, ctl_of(b), 0, 0, b->U,
                                                           nullptr, V, nullptr, pi, nullptr);
}

// skipped (nullable): instances certified in an earlier round, left untouched.
template <int MH>
static void enqueue_cert(Batch* b, const int* skipped, cudaStream_t st) {
    k_bpost<MH, double, false><<<b->grid, kThreads, 0, st>>>(b->d_desc, b->d_tiles, b->ntiles, skipped, b->V64,
                                                             b->U64, nullptr);
    k_bmax<MH, double, false><<<b->grid, kThreads, 0, st>>>(b->d_desc, b->d_tiles, b->ntiles, ctl_of(b), 0, 0, b->U64,
                                                            nullptr, b->V64, b->V64b, b->pi2, b->res64, skipped);
}

template <int MH>
static void enqueue_resid(Batch* b, const int* skipped, cudaStream_t st) {
    k_bpost<MH, double, false><<<b->grid, kThreads, 0, st>>>(b->d_desc, b->d_tiles, b->ntiles, skipped, b->V64,
                                                             b->U64, nullptr);
    k_bresid64<MH><<<b->grid, kThreads, 0, st>>>(b->d_desc, b->d_tiles, b->ntiles, b->pi, b->U64, b->V64, b->Rr,
                                                 b->err, skipped);
}


}  // namespace vc

using namespace vc;

extern "C" {

int vc_build_batch(const vc_params* p, int32_t n, void* stream, vc_batch** out) {
    set_error("");
    if (!out || !p) return fail(VC_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (n < 1) return fail(VC_ERR_ARG, "n must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    Batch* b = new Batch();
    b->n = n;
    int rc = VC_OK;
    int maxH = 1;
    for (int i = 0; i < n && !rc; i++) {
        Mdp tmp;
        tmp.fmt = VC_IMPLICIT;
        rc = build_model(&p[i], &tmp);
        if (rc) {
            set_error("instance " + std::to_string(i) + ": " + vc_last_error());
            break;
        }
        InstDesc d;
        memset(&d, 0, sizeof(d));
        d.md = tmp.md;
        d.c32 = tmp.c32;
        d.c64 = tmp.c64;
        d.off = b->total;
        d.S = tmp.S;
        b->h_desc.push_back(d);
        b->total += tmp.S;
        maxH = std::max(maxH, tmp.md.H);
    }
    if (!rc && b->total >= (1LL << 31)) rc = fail(VC_ERR_ARG, "total states must be < 2^31");
    if (rc) {
        delete b;
        return rc;
    }
    b->mh = maxH <= 8 ? maxH : 16;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t T = (size_t)b->total, N = (size_t)n;
    void** f4[] = {(void**)&b->Va, (void**)&b->Vb, (void**)&b->U, (void**)&b->U2, (void**)&b->E0, (void**)&b->E1,
                   (void**)&b->Rr, (void**)&b->pi, (void**)&b->pi2};
    for (void** pp : f4)
        if (!rc) rc = balloc(b, pp, 4 * T);
    void** f8[] = {(void**)&b->V64, (void**)&b->V64b, (void**)&b->U64};
    for (void** pp : f8)
        if (!rc) rc = balloc(b, pp, 8 * T);
    void** fi[] = {(void**)&b->done, (void**)&b->sweeps, (void**)&b->ticket, (void**)&b->tiles_of,
                   (void**)&b->final_buf, (void**)&b->since_best, (void**)&b->best_res, (void**)&b->btiles_of};
    for (void** pp : fi)
        if (!rc) rc = balloc(b, pp, 4 * N);
    if (!rc) rc = balloc(b, (void**)&b->res32, 8 * N);
    if (!rc) rc = balloc(b, (void**)&b->vmax32, 8 * N);
    if (!rc) rc = balloc(b, (void**)&b->res64, 8 * N);
    if (!rc) rc = balloc(b, (void**)&b->active, 16);
    if (!rc) rc = balloc(b, (void**)&b->err, 16);
    if (!rc) rc = balloc(b, (void**)&b->iters, 16);
    if (!rc) rc = balloc(b, (void**)&b->max_d, 16);
    if (!rc) rc = balloc(b, (void**)&b->tol_d, 16);
    if (!rc) rc = balloc(b, (void**)&b->tol_scale, 4 * N);
    if (!rc) rc = balloc(b, (void**)&b->certified, 4 * N);
    if (!rc) rc = balloc(b, (void**)&b->kr, 20 * T);
    void** kd[] = {(void**)&b->kr_rho, (void**)&b->kr_alpha, (void**)&b->kr_omega, (void**)&b->kr_beta,
                   (void**)&b->kr_target};
    for (void** pp : kd)
        if (!rc) rc = balloc(b, pp, 8 * N);
    void** k4[] = {(void**)&b->kr_rmax, (void**)&b->kr_done, (void**)&b->kr_iter, (void**)&b->kr_ticket,
                   (void**)&b->tile_first};
    for (void** pp : k4)
        if (!rc) rc = balloc(b, pp, 4 * N);
    if (!rc) rc = balloc(b, (void**)&b->kr_max_d, 16);
    if (!rc) {
        const long long mi = kKrylovMaxIter;
        cudaError_t e = cudaMemcpy(b->kr_max_d, &mi, sizeof(mi), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpy(iteration cap)");
    }
    if (!rc) rc = balloc(b, (void**)&b->d_desc, sizeof(InstDesc) * N);
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(b->d_desc, b->h_desc.data(), sizeof(InstDesc) * N, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(descriptors)");
    }
    if (!rc) {
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        b->small_cap = std::max(0, (optin - 4096) / 16);
        b->small_max = b->small_cap;
        cudaError_t e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
        for (int c = 0; c < Batch::kSmallClasses && e == cudaSuccess; c++) {
            e = cudaStreamCreateWithFlags(&b->side[c], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev[c], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) rc = cuda_fail(e, "side streams of the whole-instance path");
    }
    if (!rc) rc = build_tiles(b, st);
    if (!rc) rc = build_block_tiles(b, st);
    if (!rc) rc = build_small_list(b, st);
    if (!rc) rc = build_graphs(b);
    if (rc) {
        free_batch(b);
        return rc;
    }
    *out = (vc_batch*)b;
    return VC_OK;
}

int vc_batch_info(const vc_batch* bh, vc_batch_info_t* out) {
    set_error("");
    if (!bh || !out) return fail(VC_ERR_ARG, "NULL argument");
    const Batch* b = (const Batch*)bh;
    out->n = b->n;
    out->total_states = b->total;
    out->tiles = b->ntiles;
    out->tile_states = b->ts;
    out->blocks_per_sm = b->bps;
    out->grid = b->grid;
    out->device_bytes = b->device_bytes;
    return VC_OK;
}

int vc_batch_offsets(const vc_batch* bh, int64_t* offsets) {
    set_error("");
    if (!bh || !offsets) return fail(VC_ERR_ARG, "NULL argument");
    const Batch* b = (const Batch*)bh;
    for (int i = 0; i < b->n; i++) offsets[i] = b->h_desc[i].off;
    offsets[b->n] = b->total;
    return VC_OK;
}

int vc_value_iterate_batch(vc_batch* bh, float* V, double* V64_out, int32_t* pi_out, double tol, int64_t max_sweeps,
                           int flags, vc_batch_stats* per_inst, void* stream) {
    NvtxRange nv("vc_value_iterate_batch");
    set_error("");
    if (!bh || !V) return fail(VC_ERR_ARG, "NULL argument");
    if (!(tol > 0.0) || max_sweeps < 1) return fail(VC_ERR_ARG, "tol must be > 0 and max_sweeps >= 1");
    Batch* b = (Batch*)bh;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t T = (size_t)b->total, N = (size_t)b->n;
    int rc;
    {
        const cudaError_t pe = cudaGetLastError();
        if (pe != cudaSuccess) return cuda_fail(pe, "an earlier CUDA call left an error pending");
    }
    if (!graphs_ready(b)) return fail(VC_ERR_CUDA, "the batch's loop graphs are not built (a schedule change failed)");
    // ---- FP32 value iteration of every instance: one graph launch
    VC_CUDA(cudaMemcpyAsync(b->Va, V, 4 * T, cudaMemcpyDeviceToDevice, st));
    if ((rc = reset_loop(b, tol, max_sweeps, st, b->n_small))) return rc;
    {
        const bool sl = (flags & (VC_ITER_SELF_LOOP | VC_ITER_BLOCK)) != 0;
        int rs = VC_OK;
        by_mh(b->mh, [&](auto m) { rs = launch_small<decltype(m)::value>(b, sl, st); });
        if (rs) return rs;
    }
    VC_CUDA(cudaGraphLaunch((flags & VC_ITER_BLOCK) ? b->x_vi_blk : (flags & VC_ITER_SELF_LOOP) ? b->x_vi_sl : b->x_vi,
                            st));
    {
        const cudaError_t ge = cudaGetLastError();
        if (ge != cudaSuccess) return cuda_fail(ge, "after the FP32 loop graph launch");
    }
    if ((rc = join_small(b, st))) return rc;
    long long vi_iters = 0, corr_iters = 0;
    VC_CUDA(cudaMemcpyAsync(&vi_iters, b->iters, 8, cudaMemcpyDeviceToHost, st));
    count_launches(1);
    k_bselect<float, float><<<b->grid, kThreads, 0, st>>>(b->d_desc, b->d_tiles, b->ntiles, b->final_buf, b->Va,
                                                          b->Vb, V);
    VC_LAUNCHED("k_bselect");
    std::vector<int> done(N), sweeps(N), csweeps(N, 0), cert(N, 0), rounds(N, 0);
    std::vector<double> r64(N, INFINITY);
    VC_CUDA(cudaMemcpyAsync(done.data(), b->done, 4 * N, cudaMemcpyDeviceToHost, st));
    VC_CUDA(cudaMemcpyAsync(sweeps.data(), b->sweeps, 4 * N, cudaMemcpyDeviceToHost, st));
    VC_CUDA(cudaStreamSynchronize(st));
    count_launches((int)(vi_iters / 2 * kViBodyKernels));
    bool all_cert = false;
    if (!(flags & VC_ITER_FP32_ONLY)) {
        // ---- refinement of every instance: argmax policy, FP64 residual, FP32 correction
        // by BiCGSTAB (one graph launch; fixed-point sweeps as the fallback), FP64 update,
        // FP64 Bellman certificate; repeat on failures.
        by_mh(b->mh, [&](auto m) { enqueue_extract<decltype(m)::value>(b, V, b->pi, st); });
        VC_LAUNCHED("policy extraction");
        count_launches(3);
        k_f32_to_f64_n<<<b->grid, kThreads, 0, st>>>(V, b->V64, (long long)T);
        VC_LAUNCHED("k_f32_to_f64_n");
        const long long eval_max = std::max<long long>(100000, max_sweeps);
        // Per-instance target of the FP64 residual: tol, or, in accuracy mode,
        // tol (1 - gamma_i) / (2 gamma_i), which bounds max|V64 - V*| by tol / 2.
        std::vector<float> scale(N, 1.0f);
        if (flags & VC_ITER_ACCURATE)
            for (size_t i = 0; i < N; i++) {
                const double g = b->h_desc[i].c64.gamma;
                scale[i] = (float)((1.0 - g) / (2.0 * g));
            }
        VC_CUDA(cudaMemcpyAsync(b->tol_scale, scale.data(), 4 * N, cudaMemcpyHostToDevice, st));
        const bool plain = (flags & VC_ITER_PLAIN_CORRECTION) != 0;
        // instances certified in an earlier round keep their values, policy and residual:
        // later rounds skip them in every pass
        std::vector<int> skip_h(N, 0);
        const int* skipped = nullptr;
        for (int round = 0; round < 20; round++) {
            VC_CUDA(cudaMemsetAsync(b->err, 0, 4, st));
            count_launches(2);
            by_mh(b->mh, [&](auto m) { enqueue_resid<decltype(m)::value>(b, skipped, st); });
            VC_LAUNCHED("FP64 policy residual");
            int herr = 0;
            VC_CUDA(cudaMemcpyAsync(&herr, b->err, 4, cudaMemcpyDeviceToHost, st));
            std::vector<int> cs(N, 0);
            bool solved = false;
            if (!plain) {
                // BiCGSTAB for every instance's correction equation: one graph launch
                const BatchKrylov K = kry_of(b);
                count_launches(2);
                k_bkr_reset<<<(b->n + 255) / 256, 256, 0, st>>>(K, b->n, 0.5 * tol, b->tol_scale);
                k_bkr_init<<<b->grid, kThreads, 0, st>>>(b->d_desc, b->d_tiles, b->ntiles, K);
                VC_LAUNCHED("BiCGSTAB start");
                VC_CUDA(cudaGraphLaunch(b->x_kry, st));
                long long kit = 0;
                std::vector<int> kd(N), ki(N);
                VC_CUDA(cudaMemcpyAsync(&kit, b->iters, 8, cudaMemcpyDeviceToHost, st));
                VC_CUDA(cudaMemcpyAsync(kd.data(), b->kr_done, 4 * N, cudaMemcpyDeviceToHost, st));
                VC_CUDA(cudaMemcpyAsync(ki.data(), b->kr_iter, 4 * N, cudaMemcpyDeviceToHost, st));
                VC_CUDA(cudaStreamSynchronize(st));
                count_launches((int)(kit * kKryBodyKernels));
                if (herr) return fail(VC_ERR_CUDA, "internal: batched refinement policy infeasible");
                solved = true;
                for (size_t i = 0; i < N; i++) {
                    cs[i] = 2 * ki[i];
                    solved = solved && kd[i] == 1;
                }
                if (solved && (rc = launch_axpy64(b->V64, b->E0, (int)T, st))) return rc;
            }
            if (!solved) {
                // fixed-point correction sweeps (VC_ITER_PLAIN_CORRECTION, or BiCGSTAB broke
                // down for an instance): e <- r + gamma P_pi e from e = 0 for every instance
                VC_CUDA(cudaMemsetAsync(b->E0, 0, 4 * T, st));
                if ((rc = reset_loop(b, 0.5 * tol, eval_max, st))) return rc;
                VC_CUDA(cudaGraphLaunch(b->x_corr, st));
                VC_CUDA(cudaMemcpyAsync(&corr_iters, b->iters, 8, cudaMemcpyDeviceToHost, st));
                count_launches(1);
                k_baxpy<<<b->grid, kThreads, 0, st>>>(b->E0, b->E1, b->d_desc, b->d_tiles, b->ntiles, b->final_buf,
                                                      b->V64);
                VC_LAUNCHED("k_baxpy");
                std::vector<int> cs2(N);
                VC_CUDA(cudaMemcpyAsync(cs2.data(), b->sweeps, 4 * N, cudaMemcpyDeviceToHost, st));
                VC_CUDA(cudaStreamSynchronize(st));
                count_launches((int)(corr_iters / 2 * kCorrBodyKernels));
                corr_iters = 0;
                for (size_t i = 0; i < N; i++) cs[i] += cs2[i];
            }
            VC_CUDA(cudaMemsetAsync(b->res64, 0, 8 * N, st));
            count_launches(2);
            by_mh(b->mh, [&](auto m) { enqueue_cert<decltype(m)::value>(b, skipped, st); });
            VC_LAUNCHED("FP64 certificate");
            std::vector<unsigned long long> rb(N);
            VC_CUDA(cudaMemcpyAsync(rb.data(), b->res64, 8 * N, cudaMemcpyDeviceToHost, st));
            VC_CUDA(cudaMemcpyAsync(b->V64, b->V64b, 8 * T, cudaMemcpyDeviceToDevice, st));
            VC_CUDA(cudaMemcpyAsync(b->pi, b->pi2, 4 * T, cudaMemcpyDeviceToDevice, st));
            VC_CUDA(cudaStreamSynchronize(st));
            if (herr) return fail(VC_ERR_CUDA, "internal: batched refinement policy infeasible");
            all_cert = true;
            for (size_t i = 0; i < N; i++) {
                csweeps[i] += cs[i];
                if (skip_h[i]) continue;
                double r;
                memcpy(&r, &rb[i], 8);
                r64[i] = r;
                cert[i] = r < tol * (double)scale[i];
                if (cert[i]) rounds[i] = round + 1;
                all_cert = all_cert && cert[i];
            }
            if (all_cert) break;
            for (size_t i = 0; i < N; i++) skip_h[i] = cert[i];
            VC_CUDA(cudaMemcpyAsync(b->certified, skip_h.data(), 4 * N, cudaMemcpyHostToDevice, st));
            skipped = b->certified;
        }
        if (V64_out) VC_CUDA(cudaMemcpyAsync(V64_out, b->V64, 8 * T, cudaMemcpyDeviceToDevice, st));
        if (pi_out) VC_CUDA(cudaMemcpyAsync(pi_out, b->pi, 4 * T, cudaMemcpyDeviceToDevice, st));
    } else {
        if (pi_out) by_mh(b->mh, [&](auto m) { enqueue_extract<decltype(m)::value>(b, V, pi_out, st); });
        VC_LAUNCHED("policy extraction (FP32 only)");
        if (V64_out) {
            count_launches(1);
            k_f32_to_f64_n<<<b->grid, kThreads, 0, st>>>(V, V64_out, (long long)T);
            VC_LAUNCHED("k_f32_to_f64_n (FP32 only)");
        }
    }
    VC_CUDA(cudaStreamSynchronize(st));
    VC_LAUNCHED("end of the batched solve");
    bool any_max = false;
    for (size_t i = 0; i < N; i++) {
        if (done[i] == 0 || done[i] == 2) any_max = true;
        if (per_inst) {
            per_inst[i].sweeps = sweeps[i];
            per_inst[i].correction_sweeps = csweeps[i];
            per_inst[i].residual64 = r64[i];
            per_inst[i].certified = cert[i];
            per_inst[i].termination = done[i];
            per_inst[i].rounds = rounds[i];
            per_inst[i].reserved = 0;
        }
    }
    if (flags & VC_ITER_FP32_ONLY) {
        if (any_max) return fail(VC_ERR_NOT_CONVERGED, "an instance reached max_sweeps");
        return VC_OK;
    }
    if (!all_cert) return fail(VC_ERR_NOT_CONVERGED, "an instance was not certified");
    return VC_OK;
}

int vc_batch_set_small_instances(vc_batch* bh, int32_t max_states, void* stream) {
    set_error("");
    if (!bh) return fail(VC_ERR_ARG, "NULL handle");
    Batch* b = (Batch*)bh;
    if (max_states < 0) return fail(VC_ERR_ARG, "max_states must be >= 0");
    b->small_max = std::min(max_states, b->small_cap);
    return build_small_list(b, (cudaStream_t)stream);
}

int vc_batch_small_instances(const vc_batch* bh, int32_t* count, int32_t* max_states) {
    set_error("");
    if (!bh) return fail(VC_ERR_ARG, "NULL handle");
    const Batch* b = (const Batch*)bh;
    if (count) *count = b->n_small;
    if (max_states) *max_states = b->small_max;
    return VC_OK;
}

int vc_batch_set_block_iteration(vc_batch* bh, int32_t threads, int32_t passes, void* stream) {
    set_error("");
    if (!bh) return fail(VC_ERR_ARG, "NULL handle");
    if (threads < 32 || threads > 512) return fail(VC_ERR_ARG, "threads must be in 32..512");
    if (passes < 1 || passes > 64) return fail(VC_ERR_ARG, "passes must be in 1..64");
    Batch* b = (Batch*)bh;
    cudaStream_t st = (cudaStream_t)stream;
    VC_LAUNCHED("pending before the block shape change");
    g_destroy_note.clear();
    {
        // the kernel's own limit (registers x threads) may be below 1024
        int lim = 1024;
        by_mh(b->mh, [&](auto m) {
            cudaFuncAttributes fa;
            if (cudaFuncGetAttributes(&fa, k_bblock<decltype(m)::value>) == cudaSuccess) lim = fa.maxThreadsPerBlock;
            else cudaGetLastError();
        });
        if (threads > lim)
            return fail(VC_ERR_ARG, "threads exceeds the in-block kernel's limit of " + std::to_string(lim));
    }
    VC_LAUNCHED("pending after the thread-limit query");
    const int old_t = b->blk_threads, old_p = b->blk_passes;
    b->blk_threads = threads;
    b->blk_passes = passes;
    int rc = build_block_tiles(b, st);
    if (!rc) {
        const cudaError_t pe = cudaGetLastError();
        if (pe != cudaSuccess)
            rc = cuda_fail(pe, ("pending after the block tile table; destroy note: " + g_destroy_note).c_str());
    }
    if (!rc) rc = build_graphs(b);
    if (rc) {
        // back to the previous shape; if even that cannot be rebuilt, the graphs stay
        // destroyed and the solves report it
        const std::string why = vc_last_error();
        b->blk_threads = old_t;
        b->blk_passes = old_p;
        if (!build_block_tiles(b, st)) build_graphs(b);
        return fail(rc, why);
    }
    return VC_OK;
}

// Times the FP32 loop graph for every (tile size, blocks per SM) schedule on this batch
// (a fixed number of sweeps from V = 0) and keeps the fastest.
int vc_batch_autotune(vc_batch* bh, int sweeps, double* best_ms, void* stream) {
    set_error("");
    if (!bh) return fail(VC_ERR_ARG, "NULL handle");
    Batch* b = (Batch*)bh;
    cudaStream_t st = (cudaStream_t)stream;
    if (sweeps < 2) sweeps = 2;
    const int tss[] = {256, 512, 1024, 2048, 4096, 8192};
    const int bpss[] = {2, 4, 8};
    cudaEvent_t e0, e1;
    VC_CUDA(cudaEventCreate(&e0));
    VC_CUDA(cudaEventCreate(&e1));
    double best = 1e300;
    int best_ts = b->ts, best_bps = b->bps;
    int rc;
    b->tune_report = "tile_states blocks_per_sm grid tiles ms\n";
    for (int ts : tss) {
        for (int bps : bpss) {
            b->ts = ts;
            b->bps = bps;
            if ((rc = build_tiles(b, st))) return rc;
            if ((rc = build_graphs(b))) return rc;
            float ms_best = 1e30f;
            for (int rep = 0; rep < 2; rep++) {
                VC_CUDA(cudaMemsetAsync(b->Va, 0, 4 * (size_t)b->total, st));
                if ((rc = reset_loop(b, 1e-30, sweeps, st))) return rc;
                VC_CUDA(cudaEventRecord(e0, st));
                count_launches((sweeps + 1) / 2 * kViBodyKernels);
                if (!graphs_ready(b)) return fail(VC_ERR_CUDA, "the batch's loop graphs are not built");
                VC_CUDA(cudaGraphLaunch(b->x_vi, st));
                VC_CUDA(cudaEventRecord(e1, st));
                VC_CUDA(cudaEventSynchronize(e1));
                float ms = 0.0f;
                VC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                ms_best = std::min(ms_best, ms);
            }
            char line[128];
            snprintf(line, sizeof(line), "%d %d %d %d %.3f\n", ts, bps, b->grid, b->ntiles, ms_best);
            b->tune_report += line;
            if (ms_best < best) {
                best = ms_best;
                best_ts = ts;
                best_bps = bps;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->ts = best_ts;
    b->bps = best_bps;
    if ((rc = build_tiles(b, st))) return rc;
    if ((rc = build_graphs(b))) return rc;
    if (best_ms) *best_ms = best;
    return VC_OK;
}

int64_t vc_batch_autotune_report(const vc_batch* bh, char* buf, int64_t len) {
    if (!bh) return 0;
    const std::string& r = ((const Batch*)bh)->tune_report;
    if (buf && len > 0) {
        const int64_t n = std::min<int64_t>(len - 1, (int64_t)r.size());
        memcpy(buf, r.data(), (size_t)n);
        buf[n] = 0;
    }
    return (int64_t)r.size() + 1;
}

int vc_batch_destroy(vc_batch* bh) {
    set_error("");
    free_batch((Batch*)bh);
    return VC_OK;
}

}  // extern "C"
