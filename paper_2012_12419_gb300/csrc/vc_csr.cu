// vc_csr.cu -- explicit-CSR Bellman sweep (Algorithm 3, step 2; Eq. 18 backup from stored
// rows r = s*A + a) and the FP64 / correction kernels of handles without a model.
//
// Main kernel, k_csr_tma: the CSR streams (row_ptr, R, scale, col, val) are the only
// HBM-bound data, so each CTA runs a producer/consumer pipeline over tiles of `ts`
// consecutive states.  One producer lane stages the tile's contiguous slices into shared
// memory with bulk asynchronous copies (cp.async.bulk, completion counted on an mbarrier,
// L2 evict-first so the streamed matrix does not push V out of L2); NW consumer warps
// compute from shared memory.  Consumer lanes map to rows: APAD lanes per state (APAD =
// next power of two >= A), lane a sums row (s, a) in column order and the state's Q values
// are reduced across its APAD lanes with xor shuffles to (max, lowest argmax, second max).
// Consecutive states of a tile share successor offsets, so the V gathers of one warp touch
// few cache lines.  Every wait is bounded: on expiry the kernel flags kErrTimeout, drains
// its own copies (again bounded) and returns normally.
//
// Fallback, k_csr_direct: the same row mapping reading rows straight from global memory,
// for tiles that do not fit in shared memory (very long rows) or A > 32.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "vc_internal.cuh"
#include "vc_krylov.cuh"
#include "vc_ptx.cuh"

namespace vc {

constexpr int kNW = 8;                      // consumer warps of the pipelined kernel
// ----------------------------------------------------------------------- tile layout
struct StageLayout {
    int off_rp, off_R, off_scale, off_col, off_val, bytes;
};

__host__ __device__ inline int round16(long long x) { return (int)((x + 15) & ~15LL); }

__host__ __device__ inline StageLayout stage_layout(int ts, int A, long long cap, int vt_size, bool has_scale) {
    StageLayout L;
    const long long rows = (long long)ts * A;
    L.off_rp = 0;
    L.off_R = L.off_rp + round16(8 * (rows + 2));
    L.off_scale = L.off_R + round16(4 * (rows + 4));
    L.off_col = L.off_scale + (has_scale ? round16(4 * (rows + 4)) : 0);
    L.off_val = L.off_col + round16(4 * (cap + 8));
    L.bytes = L.off_val + round16((long long)vt_size * (cap + 8));
    return L;
}

template <typename VT>
__device__ __forceinline__ float ldv(const VT* p, int j);
template <>
__device__ __forceinline__ float ldv<float>(const float* p, int j) {
    return p[j];
}
template <>
__device__ __forceinline__ float ldv<uint16_t>(const uint16_t* p, int j) {
    return __uint_as_float((uint32_t)p[j] << 16);
}
template <typename VT>
__device__ __forceinline__ float ldg_v(const VT* p, int64_t j);
template <>
__device__ __forceinline__ float ldg_v<float>(const float* p, int64_t j) {
    return __ldg(p + j);
}
template <>
__device__ __forceinline__ float ldg_v<uint16_t>(const uint16_t* p, int64_t j) {
    return __uint_as_float((uint32_t)__ldg(p + j) << 16);
}

// Top-2 merge over xor partners: (best, lowest index of best, second best).
template <int WIDTH>
__device__ __forceinline__ void top2_reduce(float& b1, int& ia, float& b2) {
#pragma unroll
    for (int o = 1; o < WIDTH; o <<= 1) {
        const float ob1 = __shfl_xor_sync(0xffffffffu, b1, o);
        const float ob2 = __shfl_xor_sync(0xffffffffu, b2, o);
        const int oia = __shfl_xor_sync(0xffffffffu, ia, o);
        const bool take = (ob1 > b1) || (ob1 == b1 && oia < ia);
        const float nb2 = fmaxf(fmaxf(b2, ob2), take ? b1 : ob1);
        b1 = take ? ob1 : b1;
        ia = take ? oia : ia;
        b2 = nb2;
    }
}

// Dot product of one stored row with V, fused multiply-adds in column order (the
// arithmetic of every CSR sweep kernel, so their results agree bitwise).  Entries go in
// batches of kBatch: every gather of a batch is issued before the first multiply-add, so
// a row of up to kBatch successors costs one memory round trip.
constexpr int kBatch = 16;

// SL: entries whose column is the row's own state `self` add their value to pss and
// nothing to the sum (fmaf with a zero operand leaves acc unchanged), so the result is
// the sum over the other successors, still in column order.
template <typename VT, bool SL>
__device__ __forceinline__ float row_dot_smem(const int32_t* cp, const VT* vp, int n, const float* __restrict__ V,
                                              int self, float& pss) {
    float acc = 0.0f;
    for (int j0 = 0; j0 < n; j0 += kBatch) {
        float w[kBatch], g[kBatch];
        uint32_t own = 0;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (j0 + u < n) {
                const int c = cp[j0 + u];
                w[u] = ldv<VT>(vp, j0 + u);
                g[u] = __ldg(V + c);
                if (SL) own |= (c == self ? 1u : 0u) << u;
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (j0 + u < n) {
                if (SL) {
                    const bool o = (own >> u) & 1u;
                    pss += o ? w[u] : 0.0f;
                    acc = fmaf(w[u], o ? 0.0f : g[u], acc);
                } else {
                    acc = fmaf(w[u], g[u], acc);
                }
            }
        }
    }
    return acc;
}

template <typename VT, bool SL>
__device__ __forceinline__ float row_dot_global(const int32_t* __restrict__ col, const VT* __restrict__ val, int64_t lo,
                                                int n, const float* __restrict__ V, int self, float& pss) {
    float acc = 0.0f;
    for (int j0 = 0; j0 < n; j0 += kBatch) {
        float w[kBatch], g[kBatch];
        uint32_t own = 0;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (j0 + u < n) {
                const int c = __ldg(col + lo + j0 + u);
                w[u] = ldg_v<VT>(val, lo + j0 + u);
                g[u] = __ldg(V + c);
                if (SL) own |= (c == self ? 1u : 0u) << u;
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (j0 + u < n) {
                if (SL) {
                    const bool o = (own >> u) & 1u;
                    pss += o ? w[u] : 0.0f;
                    acc = fmaf(w[u], o ? 0.0f : g[u], acc);
                } else {
                    acc = fmaf(w[u], g[u], acc);
                }
            }
        }
    }
    return acc;
}

// Q value of a stored row from its sum (and, SL, its self-transition probability).
template <bool SL>
__device__ __forceinline__ float row_q(float rr, float gamma, float acc, float pss, const float* sc) {
    if (SL) return q_self_loop(rr, gamma, sc ? *sc * acc : acc, sc ? *sc * pss : pss);
    return rr + gamma * (sc ? *sc * acc : acc);
}

struct CsrArgs {
    int S, A, ts, stages;
    int64_t ntiles;
    float gamma;
    StageLayout L;
    const int64_t* row_ptr;
    const int32_t* col;
    const void* val;
    const float* scale;
    const float* R;
    const float* V_in;
    float* V_out;
    int32_t* pi;
    float* qgap;
};

// ------------------------------------------------------------------ pipelined sweep
template <typename VT, int APAD, bool SL>
__global__ void __launch_bounds__((kNW + 1) * 32, 3) k_csr_tma(CsrArgs a, SweepCtl sc) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (loop_done(sc)) return;
    const long long sweep = loop_sweep(sc);
    const long long lim = wait_limit(sc);
    constexpr int SPW = 32 / APAD;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + a.stages;
    unsigned char* stage0 = smem + ((16 * a.stages + 127) & ~127);
    __shared__ int s_fail;
    __shared__ int s_consumed;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < a.stages; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kNW);
        }
        fence_mbar_init();
        s_fail = 0;
        s_consumed = 0x7fffffff;
    }
    __syncthreads();

    const VT* val = reinterpret_cast<const VT*>(a.val);
    float res = 0.0f, vabs = 0.0f;
    int issued = 0;
    if (warp == kNW) {
        // ---------------- producer: one lane issues the bulk copies of each tile
        if (lane == 0) {
            const uint64_t pol = l2_evict_first();
            // entry bounds of a tile; the next tile's are loaded one iteration ahead so
            // their latency overlaps the wait for a free stage
            auto bounds = [&](int64_t t, int64_t& e0, int64_t& e1) {
                const int64_t s0 = t * a.ts;
                const int64_t s1 = (s0 + a.ts < a.S) ? s0 + a.ts : a.S;
                e0 = a.row_ptr[s0 * a.A];
                e1 = a.row_ptr[s1 * a.A];
            };
            int64_t ne0 = 0, ne1 = 0;
            if (blockIdx.x < a.ntiles) bounds(blockIdx.x, ne0, ne1);
            int i = 0;
            for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++i) {
                const int64_t e0 = ne0, e1 = ne1;
                if (t + gridDim.x < a.ntiles) bounds(t + gridDim.x, ne0, ne1);
                const int stg = i % a.stages;
                if (i >= a.stages && !mbar_wait(&empty[stg], (uint32_t)(((i / a.stages) - 1) & 1), lim)) {
                    atomicExch(&s_fail, 1);
                    break;
                }
                if (*((volatile int*)&s_fail)) break;
                const int64_t s0 = t * a.ts;
                const int64_t s1 = (s0 + a.ts < a.S) ? s0 + a.ts : a.S;
                const int64_t r0 = s0 * a.A, r1 = s1 * a.A;
                unsigned char* base = stage0 + (size_t)stg * a.L.bytes;
                const uint32_t b_rp = (uint32_t)(((r1 - r0 + 1) + 1) & ~1LL) * 8u;
                const uint32_t b_R = (uint32_t)(((r1 - r0) + 3) & ~3LL) * 4u;
                const int64_t c0 = e0 & ~3LL, c1 = (e1 + 3) & ~3LL;
                const int64_t v0 = (sizeof(VT) == 4) ? c0 : (e0 & ~7LL);
                const int64_t v1 = (sizeof(VT) == 4) ? c1 : ((e1 + 7) & ~7LL);
                const uint32_t b_col = (uint32_t)(c1 - c0) * 4u;
                const uint32_t b_val = (uint32_t)(v1 - v0) * (uint32_t)sizeof(VT);
                const uint32_t total = b_rp + b_R + (a.scale ? b_R : 0u) + b_col + b_val;
                mbar_arrive_expect_tx(&full[stg], total);
                bulk_g2s(base + a.L.off_rp, a.row_ptr + r0, b_rp, &full[stg], pol);
                bulk_g2s(base + a.L.off_R, a.R + r0, b_R, &full[stg], pol);
                if (a.scale) bulk_g2s(base + a.L.off_scale, a.scale + r0, b_R, &full[stg], pol);
                if (b_col) bulk_g2s(base + a.L.off_col, a.col + c0, b_col, &full[stg], pol);
                if (b_val) bulk_g2s(base + a.L.off_val, val + v0, b_val, &full[stg], pol);
                issued = i + 1;
            }
        }
    } else {
        // ---------------- consumers: lanes = rows, APAD lanes per state.  Four consecutive
        // states x A actions per warp step keep the V gathers of one load instruction
        // within a few cache lines (same successor offsets, adjacent states).
        const int grp = lane / APAD, act = lane % APAD;
        int i = 0;
        for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++i) {
            const int stg = i % a.stages;
            if (!mbar_wait(&full[stg], (uint32_t)((i / a.stages) & 1), lim)) {
                atomicExch(&s_fail, 1);
                break;
            }
            const unsigned char* base = stage0 + (size_t)stg * a.L.bytes;
            const int64_t* rp = reinterpret_cast<const int64_t*>(base + a.L.off_rp);
            const float* Rs = reinterpret_cast<const float*>(base + a.L.off_R);
            const float* Ss = a.scale ? reinterpret_cast<const float*>(base + a.L.off_scale) : nullptr;
            const int32_t* cs = reinterpret_cast<const int32_t*>(base + a.L.off_col);
            const VT* vs = reinterpret_cast<const VT*>(base + a.L.off_val);
            const int64_t e0 = rp[0];
            const int64_t c0 = e0 & ~3LL;
            const int64_t v0 = (sizeof(VT) == 4) ? c0 : (e0 & ~7LL);
            const int s0 = (int)(t * a.ts);
            const int ns = (a.S - s0 < a.ts) ? a.S - s0 : a.ts;
            for (int sb = warp * SPW; sb < ns; sb += kNW * SPW) {
                const int sl = sb + grp;
                float q = -INFINITY;
                if (sl < ns && act < a.A) {
                    const int rl = sl * a.A + act;
                    const float rr = Rs[rl];
                    if (rr != -INFINITY) {
                        const int64_t lo = rp[rl], hi = rp[rl + 1];
                        bool ok = true;
#ifdef VC_DEBUG_BOUNDS
                        // the row lies inside the staged slices and its columns index V
                        ok = VC_IN_BOUNDS(sc.ctl, lo >= c0 && hi >= lo &&
                                                      (hi - c0) * 4 <= (int64_t)(a.L.off_val - a.L.off_col));
                        for (int64_t j = lo; ok && j < hi; ++j)
                            ok = VC_IN_BOUNDS(sc.ctl, cs[j - c0] >= 0 && cs[j - c0] < a.S);
#endif
                        if (ok) {
                            float pss = 0.0f;
                            const float acc = row_dot_smem<VT, SL>(cs + (lo - c0), vs + (lo - v0), (int)(hi - lo),
                                                                   a.V_in, s0 + sl, pss);
                            q = row_q<SL>(rr, a.gamma, acc, pss, Ss ? Ss + rl : nullptr);
                        }
                    }
                }
                float b1 = q, b2 = -INFINITY;
                int ia = (act < a.A) ? act : 0x7fffffff;
                top2_reduce<APAD>(b1, ia, b2);
                if (act == 0 && sl < ns) {
                    const int s = s0 + sl;
                    if (a.V_out) a.V_out[s] = b1;
                    if (a.pi) a.pi[s] = ia;
                    if (a.qgap) a.qgap[s] = (b2 == -INFINITY) ? INFINITY : b1 - b2;
                    res = fmaxf(res, fabsf(b1 - __ldg(a.V_in + s)));
                    vabs = fmaxf(vabs, fabsf(b1));
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[stg]);
        }
        if (lane == 0) atomicMin(&s_consumed, i);
    }
    __syncthreads();
    if (s_fail) {
        // drain this CTA's copies still in flight before shared memory is released
        if (warp == kNW && lane == 0) {
            for (int j = (s_consumed < issued ? s_consumed : issued); j < issued; ++j)
                mbar_wait(&full[j % a.stages], (uint32_t)((j / a.stages) & 1));
            atomicOr(&sc.ctl->error, kErrTimeout);
        }
    }
    if (sc.mode == kModeNone) return;
    res = block_max<float, (kNW + 1) * 32>(res);
    vabs = block_max<float, (kNW + 1) * 32>(vabs);
    finish_block<float>(sc, res, vabs, sweep);
}

// ------------------------------------------------------------------- direct fallback
// Same lane-per-row mapping, rows read from global memory; grid-stride over state groups.
template <typename VT, int APAD, bool SL>
__global__ void __launch_bounds__(kThreads) k_csr_direct(CsrArgs a, SweepCtl sc) {
    if (loop_done(sc)) return;
    const long long sweep = loop_sweep(sc);
    constexpr int SPW = 32 / APAD;
    const VT* val = reinterpret_cast<const VT*>(a.val);
    const int lane = threadIdx.x & 31;
    const int grp = lane / APAD, act = lane % APAD;
    const int warp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * kThreads) >> 5;
    float res = 0.0f, vabs = 0.0f;
    for (int sb = warp * SPW; sb < a.S; sb += nwarps * SPW) {
        const int s = sb + grp;
        float q = -INFINITY;
        if (s < a.S && act < a.A) {
            const int64_t r = (int64_t)s * a.A + act;
            const float rr = __ldg(a.R + r);
            if (rr != -INFINITY) {
                const int64_t lo = __ldg(a.row_ptr + r), hi = __ldg(a.row_ptr + r + 1);
                bool ok = true;
#ifdef VC_DEBUG_BOUNDS
                for (int64_t j = lo; ok && j < hi; ++j)
                    ok = VC_IN_BOUNDS(sc.ctl, a.col[j] >= 0 && a.col[j] < a.S);
#endif
                if (ok) {
                    float pss = 0.0f;
                    const float acc = row_dot_global<VT, SL>(a.col, val, lo, (int)(hi - lo), a.V_in, s, pss);
                    const float scv = a.scale ? __ldg(a.scale + r) : 1.0f;
                    q = row_q<SL>(rr, a.gamma, acc, pss, a.scale ? &scv : nullptr);
                }
            }
        }
        float b1 = q, b2 = -INFINITY;
        int ia = (act < a.A) ? act : 0x7fffffff;
        top2_reduce<APAD>(b1, ia, b2);
        if (act == 0 && s < a.S) {
            if (a.V_out) a.V_out[s] = b1;
            if (a.pi) a.pi[s] = ia;
            if (a.qgap) a.qgap[s] = (b2 == -INFINITY) ? INFINITY : b1 - b2;
            res = fmaxf(res, fabsf(b1 - __ldg(a.V_in + s)));
            vabs = fmaxf(vabs, fabsf(b1));
        }
    }
    if (sc.mode == kModeNone) return;
    res = block_max<float, kThreads>(res);
    vabs = block_max<float, kThreads>(vabs);
    finish_block<float>(sc, res, vabs, sweep);
}

// Very wide action sets (A > 32): warp per state, rows in sequence, warp-reduced sums.
template <typename VT, bool SL>
__global__ void __launch_bounds__(kThreads) k_csr_wide(CsrArgs a, SweepCtl sc) {
    if (loop_done(sc)) return;
    const long long sweep = loop_sweep(sc);
    const VT* val = reinterpret_cast<const VT*>(a.val);
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * kThreads) >> 5;
    float res = 0.0f, vabs = 0.0f;
    for (int s = warp; s < a.S; s += nwarps) {
        float best = -INFINITY, second = -INFINITY;
        int arg = -1;
        for (int act = 0; act < a.A; ++act) {
            const int64_t r = (int64_t)s * a.A + act;
            const int64_t lo = __ldg(a.row_ptr + r), hi = __ldg(a.row_ptr + r + 1);
            float acc = 0.0f, pss = 0.0f;
            for (int64_t j = lo + lane; j < hi; j += 32) {
                const int c = __ldg(a.col + j);
                const float v = ldg_v<VT>(val, j);
                if (SL && c == s)
                    pss += v;
                else
                    acc = fmaf(v, __ldg(a.V_in + c), acc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (SL) pss += __shfl_xor_sync(0xffffffffu, pss, o);
            }
            const float rr = __ldg(a.R + r);
            if (rr == -INFINITY) continue;
            const float scv = a.scale ? __ldg(a.scale + r) : 1.0f;
            const float q = row_q<SL>(rr, a.gamma, acc, pss, a.scale ? &scv : nullptr);
            if (q > best) {
                second = best;
                best = q;
                arg = act;
            } else if (q > second) {
                second = q;
            }
        }
        if (lane == 0) {
            if (a.V_out) a.V_out[s] = best;
            if (a.pi) a.pi[s] = arg;
            if (a.qgap) a.qgap[s] = (second == -INFINITY) ? INFINITY : best - second;
        }
        res = fmaxf(res, fabsf(best - __ldg(a.V_in + s)));
        vabs = fmaxf(vabs, fabsf(best));
    }
    if (sc.mode == kModeNone) return;
    res = block_max<float, kThreads>(res);
    vabs = block_max<float, kThreads>(vabs);
    finish_block<float>(sc, res, vabs, sweep);
}

// --------------------------------------------------- FP64 / correction kernels (no model)
template <typename VT>
__device__ __forceinline__ double row_dot64(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                            const VT* __restrict__ val, const float* __restrict__ scale, int64_t r,
                                            const double* __restrict__ V) {
    double acc = 0.0;
    for (int64_t j = row_ptr[r]; j < row_ptr[r + 1]; j++) acc += (double)ldg_v<VT>(val, j) * V[col[j]];
    if (scale) acc *= (double)scale[r];
    return acc;
}

// The same row with the exact FP64 probabilities a handle keeps beside its stored ones
// (handles built from a model's FP64 rows; val64 = nullptr: the stored values).
template <typename VT>
__device__ __forceinline__ double row_dot64x(const CsrArgs& a, const VT* __restrict__ val,
                                             const double* __restrict__ val64, int64_t r,
                                             const double* __restrict__ V) {
    if (!val64) return row_dot64<VT>(a.row_ptr, a.col, val, a.scale, r, V);
    double acc = 0.0;
    for (int64_t j = a.row_ptr[r]; j < a.row_ptr[r + 1]; j++) acc += val64[j] * V[a.col[j]];
    return acc;
}

template <typename VT>
__global__ void __launch_bounds__(kThreads) k_csr_bellman64(CsrArgs a, double gamma, const double* __restrict__ V_in,
                                                            double* __restrict__ V_out, int32_t* __restrict__ pi,
                                                            double* __restrict__ qgap, SweepCtl sc,
                                                            const double* __restrict__ val64,
                                                            const double* __restrict__ R64) {
    const VT* val = reinterpret_cast<const VT*>(a.val);
    double res = 0.0;
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < a.S; s += gridDim.x * kThreads) {
        double best = -INFINITY, second = -INFINITY;
        int arg = -1;
        for (int act = 0; act < a.A; act++) {
            const int64_t r = (int64_t)s * a.A + act;
            const float rr = a.R[r];
            if (rr == -INFINITY) continue;
            const double qv = (R64 ? R64[r] : (double)rr) + gamma * row_dot64x<VT>(a, val, val64, r, V_in);
            if (qv > best) {
                second = best;
                best = qv;
                arg = act;
            } else if (qv > second) {
                second = qv;
            }
        }
        if (V_out) V_out[s] = best;
        if (pi) pi[s] = arg;
        if (qgap) qgap[s] = (second == -INFINITY) ? INFINITY : best - second;
        res = fmax(res, fabs(best - V_in[s]));
        if (sc.mode == kModeCert64 && sc.pi_ref && sc.pi_ref[s] != arg) atomicAdd(&sc.ctl->changes, 1ull);
    }
    if (sc.mode == kModeNone) return;
    res = block_max<double, kThreads>(res);
    finish_block<double>(sc, res, 0.0, 0);
}

template <typename VT>
__global__ void __launch_bounds__(kThreads) k_csr_resid64(CsrArgs a, double gamma, const int32_t* __restrict__ pi,
                                                          const double* __restrict__ V, float* __restrict__ r_out,
                                                          SweepCtl sc, const double* __restrict__ val64,
                                                          const double* __restrict__ R64) {
    const VT* val = reinterpret_cast<const VT*>(a.val);
    double mx = 0.0;
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < a.S; s += gridDim.x * kThreads) {
        const int act = pi[s];
        const int64_t r = (int64_t)s * a.A + act;
        const float rr = (act >= 0 && act < a.A) ? a.R[r] : -INFINITY;
        if (rr == -INFINITY) {
            atomicOr(&sc.ctl->error, kErrInfeasiblePolicy);
            r_out[s] = 0.0f;
            continue;
        }
        const double rd = (R64 ? R64[r] : (double)rr) + gamma * row_dot64x<VT>(a, val, val64, r, V) - V[s];
        r_out[s] = (float)rd;
        mx = fmax(mx, fabs(rd));
    }
    // kModeCert64: max |T_pi V - V| in FP64 into the control block
    if (sc.mode != kModeCert64) return;
    mx = block_max<double, kThreads>(mx);
    finish_block<double>(sc, mx, 0.0, 0);
}

template <typename VT>
__global__ void __launch_bounds__(kThreads) k_csr_correct32(CsrArgs a, const int32_t* __restrict__ pi,
                                                            const float* __restrict__ rres,
                                                            const float* __restrict__ e_in, float* __restrict__ e_out,
                                                            SweepCtl sc) {
    if (loop_done(sc)) return;
    const long long sweep = loop_sweep(sc);
    const VT* val = reinterpret_cast<const VT*>(a.val);
    float res = 0.0f, vabs = 0.0f;
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < a.S; s += gridDim.x * kThreads) {
        const int act = pi[s];
        if (act < 0 || act >= a.A) {
            atomicOr(&sc.ctl->error, kErrInfeasiblePolicy);
            e_out[s] = e_in[s];
            continue;
        }
        const int64_t r = (int64_t)s * a.A + act;
        float acc = 0.0f;
        for (int64_t j = a.row_ptr[r]; j < a.row_ptr[r + 1]; j++) acc = fmaf(ldg_v<VT>(val, j), e_in[a.col[j]], acc);
        if (a.scale) acc *= a.scale[r];
        const float v = rres[s] + a.gamma * acc;
        e_out[s] = v;
        res = fmaxf(res, fabsf(v - e_in[s]));
        vabs = fmaxf(vabs, fabsf(v));
    }
    if (sc.mode == kModeNone) return;
    res = block_max<float, kThreads>(res);
    vabs = block_max<float, kThreads>(vabs);
    finish_block<float>(sc, res, vabs, sweep);
}

// Product by the correction matrix for the BiCGSTAB solve from the stored rows of pi
// (pi = nullptr: action 0, the one row of a single-action system such as the adjoint's):
// y(s) = x(s) - gamma (scale) sum_j val_j x[col_j], with the stage's partial sums.
template <typename VT>
__global__ void __launch_bounds__(kThreads) k_csr_apply32(CsrArgs a, const int32_t* __restrict__ pi,
                                                          const float* __restrict__ xin, float* __restrict__ y,
                                                          const float* __restrict__ w, int stage, KrylovArgs k) {
    if (kr_done(k)) return;
    const VT* val = reinterpret_cast<const VT*>(a.val);
    float d0 = 0.0f, d1 = 0.0f;
    for (int s = blockIdx.x * kThreads + threadIdx.x; s < a.S; s += gridDim.x * kThreads) {
        const int act = pi ? pi[s] : 0;
        float yv = xin[s];
        if (act >= 0 && act < a.A) {
            const int64_t r = (int64_t)s * a.A + act;
            float acc = 0.0f;
            for (int64_t j = a.row_ptr[r]; j < a.row_ptr[r + 1]; j++) acc = fmaf(ldg_v<VT>(val, j), xin[a.col[j]], acc);
            if (a.scale) acc *= a.scale[r];
            yv -= a.gamma * acc;
        }
        y[s] = yv;
        d0 = fmaf(w[s], yv, d0);
        d1 = fmaf(yv, yv, d1);
    }
    kr_finish<kThreads>(k, stage, d0, d1, 0.0f);
}

// ------------------------------------------------------------------------- planning
__global__ void k_tile_cap(const int64_t* __restrict__ row_ptr, int S, int A, int ts, int64_t ntiles,
                           unsigned long long* out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    const int64_t s0 = t * ts;
    const int64_t s1 = (s0 + ts < S) ? s0 + ts : S;
    atomicMax(out, (unsigned long long)(row_ptr[s1 * A] - row_ptr[s0 * A]));
}

static int pow2_at_least(int a) {
    int p = 1;
    while (p < a) p <<= 1;
    return p;
}

// Dynamic shared memory limit of a kernel instance, and how many CTAs fit on an SM.
// `bytes` is the per-block opt-in limit; the kernel's static shared memory comes off it.
// *dyn_limit receives the dynamic amount actually allowed.
// Both instantiations (Eq. 18's backup and the self-transition solve) get the same limit,
// and the occupancy is the smaller of the two, since one plan serves both.
template <typename VT, int APAD>
static cudaError_t set_tma_smem(int bytes, int* dyn_limit) {
    cudaFuncAttributes fa, fb;
    cudaError_t e = cached_func_attributes((const void*)k_csr_tma<VT, APAD, false>, &fa);
    if (e == cudaSuccess) e = cached_func_attributes((const void*)k_csr_tma<VT, APAD, true>, &fb);
    if (e != cudaSuccess) return e;
    *dyn_limit = bytes - (int)std::max(fa.sharedSizeBytes, fb.sharedSizeBytes);
    e = cached_set_max_dyn_smem((const void*)k_csr_tma<VT, APAD, false>, *dyn_limit);
    if (e != cudaSuccess) return e;
    return cached_set_max_dyn_smem((const void*)k_csr_tma<VT, APAD, true>, *dyn_limit);
}

template <typename VT, int APAD>
static cudaError_t tma_occupancy(int bytes, int* per_sm) {
    int a = 0, b = 0;
    cudaError_t e = cached_occupancy((const void*)k_csr_tma<VT, APAD, false>, (kNW + 1) * 32, bytes, &a);
    if (e == cudaSuccess) e = cached_occupancy((const void*)k_csr_tma<VT, APAD, true>, (kNW + 1) * 32, bytes, &b);
    *per_sm = std::min(a, b);
    return e;
}

template <typename VT>
static cudaError_t set_tma_smem_any(int apad, int bytes, int* dyn_limit) {
    switch (apad) {
        case 1: return set_tma_smem<VT, 1>(bytes, dyn_limit);
        case 2: return set_tma_smem<VT, 2>(bytes, dyn_limit);
        case 4: return set_tma_smem<VT, 4>(bytes, dyn_limit);
        case 8: return set_tma_smem<VT, 8>(bytes, dyn_limit);
        case 16: return set_tma_smem<VT, 16>(bytes, dyn_limit);
        default: return set_tma_smem<VT, 32>(bytes, dyn_limit);
    }
}

template <typename VT>
static cudaError_t tma_occupancy_any(int apad, int bytes, int* per_sm) {
    switch (apad) {
        case 1: return tma_occupancy<VT, 1>(bytes, per_sm);
        case 2: return tma_occupancy<VT, 2>(bytes, per_sm);
        case 4: return tma_occupancy<VT, 4>(bytes, per_sm);
        case 8: return tma_occupancy<VT, 8>(bytes, per_sm);
        case 16: return tma_occupancy<VT, 16>(bytes, per_sm);
        default: return tma_occupancy<VT, 32>(bytes, per_sm);
    }
}

// Candidate tilings of the pipelined sweep, in preference order: (CTAs per SM, stages)
// pairs with the most consumer warps and copies in flight first, largest tile first; the
// largest tile of each size is measured on the device so any CSR fits.
static int enumerate_plans(Mdp* m, cudaStream_t st, std::vector<CsrPlan>& out) {
    out.clear();
    if (m->A > 32 || (m->fmt & VC_DIRECT)) return VC_OK;
    const int apad = pow2_at_least(m->A);
    const int spw = 32 / apad;
    const bool bf16 = (m->fmt & 0xF) == VC_CSR_BF16;
    const int vt = bf16 ? 2 : 4;
    int dev = 0, smem_sm = 0, smem_blk = 0;
    VC_CUDA(cudaGetDevice(&dev));
    VC_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    VC_CUDA(cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    struct Cand {
        int ts;
        long long cap;
    };
    std::vector<Cand> cands;
    // tiles of 8, 4, 2, 1 and 1/2 state rows of the consumer warps (multiples of 4 states);
    // their largest entry counts, one kernel each, read back together
    std::vector<int> sizes;
    for (int k2 = 16; k2 >= 1; k2 >>= 1) {
        const int ts = k2 * kNW * spw / 2;
        if (ts >= 4 && ts % 4 == 0) sizes.push_back(ts);
    }
    unsigned long long* dcap = nullptr;
    unsigned long long hcap[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    VC_CUDA(cudaMallocAsync((void**)&dcap, sizeof(hcap), st));
    VC_CUDA(cudaMemsetAsync(dcap, 0, sizeof(hcap), st));
    for (size_t i = 0; i < sizes.size(); ++i) {
        const int64_t nt = ((int64_t)m->S + sizes[i] - 1) / sizes[i];
        count_launches(1);
        k_tile_cap<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(m->row_ptr, m->S, m->A, sizes[i], nt, dcap + i);
    }
    VC_CUDA(cudaGetLastError());
    VC_CUDA(cudaMemcpyAsync(hcap, dcap, sizeof(hcap), cudaMemcpyDeviceToHost, st));
    VC_CUDA(cudaFreeAsync(dcap, st));
    VC_CUDA(cudaStreamSynchronize(st));
    for (size_t i = 0; i < sizes.size(); ++i) cands.push_back({sizes[i], (long long)hcap[i] + 16});
    // one attribute per kernel instance: allow the largest request, launches ask for less
    int dyn_limit = 0;
    cudaError_t e = bf16 ? set_tma_smem_any<uint16_t>(apad, smem_blk, &dyn_limit)
                         : set_tma_smem_any<float>(apad, smem_blk, &dyn_limit);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_csr_tma)");
    smem_blk = dyn_limit;
    const int hdr = 128;  // barriers
    const int prefs[][2] = {{4, 3}, {4, 2}, {3, 3}, {3, 2}, {2, 3}, {2, 2}, {1, 4}, {1, 3}, {1, 2}};
    for (auto& pr : prefs) {
        const int ctas = pr[0], stages = pr[1];
        const int budget = (smem_sm - 1024 * ctas) / ctas;
        for (const Cand& c : cands) {
            const StageLayout L = stage_layout(c.ts, m->A, c.cap, vt, bf16);
            const long long need = hdr + (long long)stages * L.bytes;
            if (need > budget || need > smem_blk) continue;
            int per_sm = 0;
            e = bf16 ? tma_occupancy_any<uint16_t>(apad, (int)need, &per_sm)
                     : tma_occupancy_any<float>(apad, (int)need, &per_sm);
            if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
            if (per_sm < 1) continue;
            CsrPlan P;
            P.tma = true;
            P.apad = apad;
            P.ts = c.ts;
            P.cap = c.cap;
            P.stages = stages;
            P.ctas_per_sm = per_sm < ctas ? per_sm : ctas;
            P.smem = (int)need;
            P.ntiles = ((int64_t)m->S + P.ts - 1) / P.ts;
            out.push_back(P);
        }
    }
    return VC_OK;
}

// Default plan: the first candidate (the direct kernel if none fits).
int plan_csr(Mdp* m, cudaStream_t st) {
    // a handle built with its sliced copy takes its plan from the sliced layout
    if (m->fmt & VC_SLICED) {
        m->plan = CsrPlan();
        return VC_OK;
    }
    std::vector<CsrPlan> cands;
    int rc = enumerate_plans(m, st, cands);
    if (rc) return rc;
    m->plan = cands.empty() ? CsrPlan() : cands.front();
    return VC_OK;
}

// ------------------------------------------------------------------------ launchers
static CsrArgs args_of(const Mdp* m, const float* V_in, float* V_out, int32_t* pi, float* qgap) {
    CsrArgs a;
    a.S = m->S;
    a.A = m->A;
    a.ts = m->plan.ts;
    a.stages = m->plan.stages;
    a.ntiles = m->plan.ntiles;
    a.gamma = (float)m->gamma;
    a.L = stage_layout(m->plan.ts, m->A, m->plan.cap, (m->fmt & 0xF) == VC_CSR_BF16 ? 2 : 4,
                       (m->fmt & 0xF) == VC_CSR_BF16);
    a.row_ptr = m->row_ptr;
    a.col = m->col;
    a.val = m->val;
    a.scale = m->scale;
    a.R = m->R;
    a.V_in = V_in;
    a.V_out = V_out;
    a.pi = pi;
    a.qgap = qgap;
    return a;
}

template <typename VT, bool SL>
static void launch_tma(const Mdp* m, const CsrArgs& a, SweepCtl sc, cudaStream_t st) {
    const long long cap = (long long)m->num_sms * m->plan.ctas_per_sm;
    const int grid = (int)(m->plan.ntiles < cap ? m->plan.ntiles : cap);
    const dim3 blk((kNW + 1) * 32);
    switch (m->plan.apad) {
        case 1: k_csr_tma<VT, 1, SL><<<grid, blk, m->plan.smem, st>>>(a, sc); break;
        case 2: k_csr_tma<VT, 2, SL><<<grid, blk, m->plan.smem, st>>>(a, sc); break;
        case 4: k_csr_tma<VT, 4, SL><<<grid, blk, m->plan.smem, st>>>(a, sc); break;
        case 8: k_csr_tma<VT, 8, SL><<<grid, blk, m->plan.smem, st>>>(a, sc); break;
        case 16: k_csr_tma<VT, 16, SL><<<grid, blk, m->plan.smem, st>>>(a, sc); break;
        default: k_csr_tma<VT, 32, SL><<<grid, blk, m->plan.smem, st>>>(a, sc); break;
    }
}

template <typename VT, bool SL>
static void launch_direct(const Mdp* m, const CsrArgs& a, SweepCtl sc, cudaStream_t st) {
    const int g = state_grid(m);
    if (m->A > 32) {
        k_csr_wide<VT, SL><<<g, kThreads, 0, st>>>(a, sc);
        return;
    }
    switch (pow2_at_least(m->A)) {
        case 1: k_csr_direct<VT, 1, SL><<<g, kThreads, 0, st>>>(a, sc); break;
        case 2: k_csr_direct<VT, 2, SL><<<g, kThreads, 0, st>>>(a, sc); break;
        case 4: k_csr_direct<VT, 4, SL><<<g, kThreads, 0, st>>>(a, sc); break;
        case 8: k_csr_direct<VT, 8, SL><<<g, kThreads, 0, st>>>(a, sc); break;
        case 16: k_csr_direct<VT, 16, SL><<<g, kThreads, 0, st>>>(a, sc); break;
        default: k_csr_direct<VT, 32, SL><<<g, kThreads, 0, st>>>(a, sc); break;
    }
}

template <typename VT>
static void launch_sweep_form(const Mdp* m, const CsrArgs& a, SweepCtl sc, cudaStream_t st) {
    if (m->plan.tma) {
        if (sc.self_loop)
            launch_tma<VT, true>(m, a, sc, st);
        else
            launch_tma<VT, false>(m, a, sc, st);
    } else {
        if (sc.self_loop)
            launch_direct<VT, true>(m, a, sc, st);
        else
            launch_direct<VT, false>(m, a, sc, st);
    }
}

int csr_sweep32(Mdp* m, const float* V_in, float* V_out, int32_t* pi, float* qgap, SweepCtl sc, cudaStream_t st) {
    if (m->plan.sliced) return sell_sweep32(m, V_in, V_out, pi, qgap, sc, st);
    const CsrArgs a = args_of(m, V_in, V_out, pi, qgap);
    const bool bf16 = (m->fmt & 0xF) == VC_CSR_BF16;
    count_launches(1);
    if (bf16)
        launch_sweep_form<uint16_t>(m, a, sc, st);
    else
        launch_sweep_form<float>(m, a, sc, st);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int csr_bellman64(Mdp* m, const double* V_in, double* V_out, int32_t* pi, double* qgap, SweepCtl sc,
                  cudaStream_t st) {
    const CsrArgs a = args_of(m, nullptr, nullptr, nullptr, nullptr);
    count_launches(1);
    if ((m->fmt & 0xF) == VC_CSR_BF16)
        k_csr_bellman64<uint16_t><<<state_grid(m), kThreads, 0, st>>>(a, m->gamma, V_in, V_out, pi, qgap, sc,
                                                                       m->val64, m->R64);
    else
        k_csr_bellman64<float><<<state_grid(m), kThreads, 0, st>>>(a, m->gamma, V_in, V_out, pi, qgap, sc, m->val64,
                                                                    m->R64);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int csr_resid64(Mdp* m, const int32_t* pi, const double* V64, float* r, SweepCtl sc, cudaStream_t st) {
    const CsrArgs a = args_of(m, nullptr, nullptr, nullptr, nullptr);
    count_launches(1);
    if ((m->fmt & 0xF) == VC_CSR_BF16)
        k_csr_resid64<uint16_t><<<state_grid(m), kThreads, 0, st>>>(a, m->gamma, pi, V64, r, sc, m->val64, m->R64);
    else
        k_csr_resid64<float><<<state_grid(m), kThreads, 0, st>>>(a, m->gamma, pi, V64, r, sc, m->val64, m->R64);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int csr_apply32(Mdp* m, const int32_t* pi, const float* x, float* y, const float* w, int stage,
                const KrylovArgs& k, cudaStream_t st) {
    const CsrArgs a = args_of(m, nullptr, nullptr, nullptr, nullptr);
    count_launches(1);
    if ((m->fmt & 0xF) == VC_CSR_BF16)
        k_csr_apply32<uint16_t><<<state_grid(m), kThreads, 0, st>>>(a, pi, x, y, w, stage, k);
    else
        k_csr_apply32<float><<<state_grid(m), kThreads, 0, st>>>(a, pi, x, y, w, stage, k);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

int csr_correct32(Mdp* m, const int32_t* pi, const float* r, const float* e_in, float* e_out, SweepCtl sc,
                  cudaStream_t st) {
    const CsrArgs a = args_of(m, nullptr, nullptr, nullptr, nullptr);
    count_launches(1);
    if ((m->fmt & 0xF) == VC_CSR_BF16)
        k_csr_correct32<uint16_t><<<state_grid(m), kThreads, 0, st>>>(a, pi, r, e_in, e_out, sc);
    else
        k_csr_correct32<float><<<state_grid(m), kThreads, 0, st>>>(a, pi, r, e_in, e_out, sc);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

// Every candidate schedule of the FP32 sweep, in the autotuner's order: the CSR tilings,
// the direct CSR kernel, then (with a sliced copy) the ring sweep's shapes and the direct
// sliced kernel at 2, 4 and 8 CTAs per SM.
int csr_candidates(Mdp* m, cudaStream_t st, std::vector<CsrPlan>& cands) {
    int rc = enumerate_plans(m, st, cands);
    if (rc) return rc;
    cands.push_back(CsrPlan());  // direct kernel
    if (m->sell_slab) {
        std::vector<CsrPlan> sp;
        if ((rc = sell_plans(m, st, sp))) return rc;
        cands.insert(cands.end(), sp.begin(), sp.end());
        for (int bps : {2, 4, 8}) {
            CsrPlan P;
            P.sliced = true;
            P.ctas_per_sm = bps;
            cands.push_back(P);
        }
    }
    return VC_OK;
}

// Times every candidate schedule on this handle and keeps the fastest: reps FP32 sweeps
// each after two warm-up sweeps, CUDA events on `st`.
int autotune_csr(Mdp* m, int reps, cudaStream_t st, double* best_us) {
    std::vector<CsrPlan> cands;
    int rc = csr_candidates(m, st, cands);
    if (rc) return rc;
    if (reps < 1) reps = 1;
    float* A = m->Vb;
    float* B = m->E0;
    VC_CUDA(cudaMemsetAsync(A, 0, 4 * (size_t)m->S, st));
    cudaEvent_t e0, e1;
    VC_CUDA(cudaEventCreate(&e0));
    VC_CUDA(cudaEventCreate(&e1));
    double best = 1e300;
    CsrPlan chosen = cands.front();
    m->tune_report = "kernel tile_states stages ctas_per_sm smem_bytes us_per_sweep\n";
    for (const CsrPlan& P : cands) {
        m->plan = P;
        SweepCtl none{m->ctl, kModeNone, 0, nullptr};
        for (int w = 0; w < 2; w++)
            if ((rc = csr_sweep32(m, A, B, nullptr, nullptr, none, st))) return rc;
        VC_CUDA(cudaEventRecord(e0, st));
        for (int r = 0; r < reps; r++)
            if ((rc = csr_sweep32(m, (r & 1) ? B : A, (r & 1) ? A : B, nullptr, nullptr, none, st))) return rc;
        VC_CUDA(cudaEventRecord(e1, st));
        VC_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        VC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        const double us = 1e3 * ms / reps;
        char line[160];
        char kname[40];
        if (P.sliced && P.tma)
            snprintf(kname, sizeof(kname), "sliced-pipelined-w%d-r%d", P.warps, P.minb);
        else
            snprintf(kname, sizeof(kname), "%s", P.sliced ? "sliced-direct" : (P.tma ? "pipelined" : "direct"));
        snprintf(line, sizeof(line), "%s %d %d %d %d %.2f\n", kname, P.sliced ? 32 * (P.tma ? P.ts : 1) : P.ts,
                 P.stages, P.ctas_per_sm, P.smem, us);
        m->tune_report += line;
        if (us < best) {
            best = us;
            chosen = P;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    m->plan = chosen;
    if (best_us) *best_us = best;
    return VC_OK;
}

}  // namespace vc
