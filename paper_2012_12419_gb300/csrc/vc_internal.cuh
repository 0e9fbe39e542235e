// vc_internal.cuh -- shared device/host definitions of the vcmdp library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/vcmdp.h"

namespace vc {

constexpr int kMaxH = VC_MAX_HOSTS;
constexpr int kRing = 64;          // residual slots, indexed by sweep number mod kRing
constexpr int kStallSweeps = 64;   // FP32 sweeps without a new best residual = FP32 floor
constexpr int kThreads = 256;      // block size of the state-parallel kernels
constexpr int kBlockMaxInner = 3;  // inner hosts of an in-block iteration block (VC_ITER_BLOCK)
constexpr int kBlockThreads = 512; // states of a block, and of a tile of blocks, at most

// ------------------------------------------------------------------ error plumbing
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define VC_CUDA(call)                                           \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return vc::cuda_fail(e_, #call); \
    } while (0)

// ------------------------------------------------------- division by a runtime constant
// q = n / d for 0 <= n < 2^31 and 1 <= d < 2^16 as a multiply-high and a shift: with
// l = ceil(log2 d), sh = 31 + l and m = floor(2^sh / d) + 1, the error term
// m*d - 2^sh <= d <= 2^(sh-31) keeps floor(n*m / 2^sh) exact for every n < 2^31
// (Granlund & Montgomery, "Division by invariant integers using multiplication", 1994).
// For d >= 2, m < 2^32 and sh >= 32, so the quotient is the high word of the 32x32
// product shifted by sh - 32; d = 1 returns n.
struct FastDiv {
    uint32_t m;
    uint32_t sh;  // sh - 32
    uint32_t d;
};

inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d;
    if (d <= 1) {
        f.m = 0;
        f.sh = 0;
        return f;
    }
    uint32_t l = 0;
    while ((1u << l) < d) l++;
    const uint32_t sh = 31 + l;
    f.m = (uint32_t)((((uint64_t)1) << sh) / d + 1);
    f.sh = sh - 32;
    return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
    return f.d <= 1 ? n : (__umulhi(n, f.m) >> f.sh);
}

// --------------------------------------------------------------------- model descriptor
// Per-precision coefficients of the uniformised model (all probabilities already / Lam).
template <typename T>
struct Coef {
    T gamma;
    T pc[kMaxH];     // mu_k / Lam          (completion, times occ_k)
    T pd[kMaxH];     // delta_k / Lam       (departure)
    T lossd[kMaxH];  // w_loss * delta_k / Lam
    T pa;            // lambda / Lam        (arrival)
    T lossa;         // w_loss * lambda / Lam (blocked arrival)
    T pf0, pf1;      // f / Lam (CCHI -> SCHI), (1 - f) / Lam (SCHI -> CCHI)
    T w_occ, w_q;
};

struct Model {
    int H, C, Q, A;
    int S;
    int stride[kMaxH];  // 2 (Q+1) (C+1)^k: code step of occ_k
    FastDiv div_q;      // by Q+1
    FastDiv div_c;      // by C+1
};

// Raw FP64 rates, used where probabilities are formed once (explicit CSR construction).
struct Rates {
    double mu[kMaxH], delta[kMaxH];
    double lambda, f, Lam;
    double w_occ, w_loss, w_q;
    // probabilities formed once on the host with the same FP64 operations the rows use
    // (IEEE division and multiplication are correctly rounded, so the values are equal):
    double pdep[kMaxH];      // delta_k / Lam
    double parr;             // lambda / Lam
    double pflip[2];         // f / Lam, (1 - f) / Lam
    const double* occ_tab;   // device [2][kMaxH][C+1]: mu_k o / Lam, delta_k o / Lam (or null)
    int tab_c1;              // C + 1
    // The FP32 roundings (to nearest) of the probabilities the CSR rows hold, formed on the
    // host from the FP64 values above, and their non-zero tests taken on those FP64 values,
    // so the FP32 fill emits exactly the FP64 path's entries and their rounded values.
    float pdep32[kMaxH];            // (float) pdep[k]
    float p1_32[kMaxH];             // (float)(mu_k / Lam + pdep[k]): occ_k = 1 (completion and departure merged)
    float parr32, pflip32[2];
    uint32_t nz_pdep, nz_p1;        // bit k: pdep[k] != 0, mu_k / Lam + pdep[k] != 0
    int nz_parr, nz_pflip[2];
    const float* occ_tab32;         // device [kMaxH][C+1]: (float)(mu_k o / Lam)
    const unsigned char* occ_nz;    // device [kMaxH][C+1]: mu_k o / Lam != 0
};

// Digits of a state code.
struct Digits {
    int occ[kMaxH];
    int q, ph;
};

// MH: a compile-time bound on H (kernels are instantiated for H <= 4, 8, 16).
template <int MH = kMaxH>
__device__ __forceinline__ void decode(const Model& md, int s, Digits& d) {
    d.ph = s & 1;
    uint32_t rest = (uint32_t)s >> 1;
    uint32_t t = fdiv(rest, md.div_q);
    d.q = (int)(rest - t * md.div_q.d);
    rest = t;
#pragma unroll
    for (int k = 0; k < MH; k++) {
        if (k < md.H) {
            uint32_t t2 = fdiv(rest, md.div_c);
            d.occ[k] = (int)(rest - t2 * md.div_c.d);
            rest = t2;
        } else {
            d.occ[k] = 0;
        }
    }
}

// Post-decision state of action a in s (digits updated in place, static indexing only).
// Returns false if a is not feasible in s.
template <int MH = kMaxH>
__device__ __forceinline__ bool apply_action(const Model& md, int s, int a, Digits& d, int& x) {
    if (a == md.H) {
        x = s;
        return true;
    }
    if (a < 0 || a > md.H || d.q < 1) return false;
    bool ok = false;
    int step = 0;
#pragma unroll
    for (int k = 0; k < MH; k++) {
        if (k == a && k < md.H && d.occ[k] < md.C && (k == md.H - 1 || d.ph == 1)) {
            d.occ[k] += 1;
            step = md.stride[k];
            ok = true;
        }
    }
    if (!ok) return false;
    d.q -= 1;
    x = s + step - 2;
    return true;
}

// --------------------------------------------------------- device: one model row (FP64)
constexpr int kMaxRow = 2 * kMaxH + 3;

// Probability of host k's completion event at occupancy o (mu_k o / Lam).
__device__ __forceinline__ double p_comp(const Rates& rt, int k, int o) {
    return rt.occ_tab ? __ldg(rt.occ_tab + (size_t)k * rt.tab_c1 + o) : rt.mu[k] * o / rt.Lam;
}

// Successors of (s, a), merged, zero probabilities dropped, passed to emit(j, column, p)
// in ascending column order for j = 0, 1, ...: host k's entries x - o_k s_k (departure)
// and x - s_k (completion) lie above every entry of host k + 1, since o_k s_k <= C s_k <
// s_{k+1}, and below x - 1, since s_0 = 2(Q + 1) >= 2; then the phase flip (x - 1 or
// x + 1), the self-loop x and the arrival x + 2.  So no sort is needed.  Returns the count,
// or -1 if a is infeasible in s; R receives the expected reward.  The probabilities and
// the reward are summed host 0 first, in one fixed order.
// MH: a compile-time bound on H (loops unrolled, digits in registers).
template <int MH = kMaxH, typename Emit>
__device__ __forceinline__ int model_row_emit(const Model& md, const Rates& rt, int s, int a, double* R, Emit&& emit) {
    Digits d;
    decode<MH>(md, s, d);
    int x = s;
    if (a < md.H && !apply_action<MH>(md, s, a, d, x)) return -1;
    double total = 0.0, self_extra = 0.0, occ_sum = 0.0, lost = 0.0;
#pragma unroll
    for (int k = 0; k < MH; k++) {
        if (k < md.H) {
            const int o = d.occ[k];
            const double pcomp = p_comp(rt, k, o);
            const double pdep = rt.pdep[k];
            total += pcomp + pdep;
            occ_sum += o;
            lost += rt.occ_tab ? __ldg(rt.occ_tab + (size_t)(kMaxH + k) * rt.tab_c1 + o) : rt.delta[k] * o / rt.Lam;
            if (o == 0) self_extra += pdep;  // departure of an empty host changes nothing
        }
    }
    const double parr = rt.parr;
    total += parr;
    if (d.q >= md.Q) {
        self_extra += parr;  // blocked arrival
        lost += parr;
    }
    const double pflip = d.ph ? rt.pflip[1] : rt.pflip[0];
    total += pflip;
    const double pself = (1.0 - total) + self_extra;
    *R = rt.w_occ * occ_sum + rt.w_q * d.q + rt.w_loss * lost;
    int n = 0;
#pragma unroll
    for (int k = MH - 1; k >= 0; k--) {
        if (k < md.H) {
            const int o = d.occ[k];
            if (o == 1) {
                const double p = p_comp(rt, k, 1) + rt.pdep[k];  // completion and departure both empty the host
                if (p != 0.0) emit(n++, x - md.stride[k], p);
            } else if (o > 1) {
                if (rt.pdep[k] != 0.0) emit(n++, x - o * md.stride[k], rt.pdep[k]);
                const double pc = p_comp(rt, k, o);
                if (pc != 0.0) emit(n++, x - md.stride[k], pc);
            }
        }
    }
    if (d.ph) {
        if (pflip != 0.0) emit(n++, x - 1, pflip);
        if (pself != 0.0) emit(n++, x, pself);
    } else {
        if (pself != 0.0) emit(n++, x, pself);
        if (pflip != 0.0) emit(n++, x + 1, pflip);
    }
    if (d.q < md.Q && parr != 0.0) emit(n++, x + 2, parr);
    return n;
}

// The same row into arrays (cols, probs of at least kMaxRow entries).
__device__ __forceinline__ int model_row(const Model& md, const Rates& rt, int s, int a, int* cols, double* probs,
                                         double* R) {
    return model_row_emit(md, rt, s, a, R, [&](int j, int c, double p) {
        cols[j] = c;
        probs[j] = p;
    });
}

// --------------------------------------------------------------------------- control
// Device-side loop control shared by the sweep kernels of one handle.
struct Ctl {
    unsigned int res32[kRing];          // FP32 residual bits per sweep (atomicMax on >= 0 floats)
    unsigned int vmax32[kRing];         // max |V'| bits per sweep
    unsigned int ticket;                // arrival counter of the last-block pattern
    int done;                           // 0 running, 1 converged, 2 max sweeps, 3 stalled at the FP32 floor
    long long sweeps;                   // sweeps completed
    long long max_sweeps;
    int final_buf;                      // ping-pong buffer holding the latest iterate
    int since_best;
    float best_res;
    float pad_;
    double tol;
    unsigned long long changes;         // policy entries that differ from a reference policy
    unsigned long long cert64;          // FP64 residual bits of a standalone Bellman backup
    int error;                          // bit flags raised by kernels (infeasible policy, bad input)
    int pad2_;
    long long spin_limit;               // polls + 1 of each bounded pipeline wait (0 = the default)
};

// Error flags raised on the device.
constexpr int kErrInfeasiblePolicy = 1;
constexpr int kErrBadColumn = 2;
constexpr int kErrNegative = 4;
constexpr int kErrRowSum = 8;
constexpr int kErrNoFeasible = 16;
constexpr int kErrRowPtr = 32;
constexpr int kErrTimeout = 64;
constexpr int kErrBounds = 128;  // a bounds check of the VC_DEBUG_BOUNDS build failed

// Bounds checks of the VC_DEBUG_BOUNDS build (the library's stand-in for a memory checker):
// a failed check raises kErrBounds in the control block and the caller skips the access.
// In the normal build the check is compiled out (always true, condition unevaluated).
#ifdef VC_DEBUG_BOUNDS
__device__ __forceinline__ bool in_bounds(Ctl* ctl, bool ok) {
    if (!ok && ctl) atomicOr(&ctl->error, kErrBounds);
    return ok;
}
#define VC_IN_BOUNDS(ctl, cond) in_bounds((ctl), (cond))
#else
#define VC_IN_BOUNDS(ctl, cond) true
#endif

// Bookkeeping mode of a sweep kernel.
enum SweepMode : int {
    kModeNone = 0,     // plain backup (policy extraction)
    kModeLoop32 = 1,   // FP32 loop: skip when done, residual ring, tolerance / stall test
    kModeCert64 = 3,   // FP64 standalone backup: residual into cert64, policy changes vs pi_ref
};

struct SweepCtl {
    Ctl* ctl;
    int mode;
    int out_index;
    const int32_t* pi_ref;
    int self_loop;  // FP32 sweeps: solve each action's self-transition (q_self_loop)
    int block;      // FP32 sweeps of an implicit handle: Algorithm 4's in-block passes (k_block)
};

// Q value with the row's self-transition solved exactly: the fixed point in W of
// W = R + gamma (p_ss W + off), i.e. (R + gamma off) / (1 - gamma p_ss), where off is the
// row sum over the successors other than the state itself and p_ss the probability of
// staying (Puterman, Markov Decision Processes, 1994, Sec. 6.3.3; Algorithm 4's in-block
// iteration for a block of one state, run to its limit).  One rounding per operation in a
// fixed form, shared by every explicit sweep kernel so their results agree bitwise.
__device__ __forceinline__ float q_self_loop(float rr, float gamma, float off, float pss) {
    return __fdiv_rn(fmaf(gamma, off, rr), fmaf(-gamma, pss, 1.0f));
}

// Pass 1 of an implicit sweep at post-decision state x with defer's self-transition solved,
// from one set of gathers: U = R(x) + gamma E[V(next) | x] in the difference form of the
// plain pass (E = V(x) + sum_e p_e (V(y_e) - V(x)), the self-loop probability never
// formed), and W = defer's backup with its self-transition solved (the post-decision state
// of defer is s itself).  The events that leave x carry probability p_move and the sum
// sum_move of p_e V(y_e); the rest (uniformisation remainder, an arrival blocked by a full
// queue, the departure of an empty host) stays at x, so the fixed point of
// W = R(x) + gamma ((1 - p_move) W + sum_move) is
// W = (R(x) + gamma sum_move) / ((1 - gamma) + gamma p_move).  Both sums of W are formed
// directly (no differences), so W carries a relative rounding error of a few units.
template <int MH>
__device__ __forceinline__ void post_and_defer(const Model& md, const Coef<float>& c, const float* __restrict__ V,
                                               int x, const Digits& d, float rx, float& U, float& W) {
    const float vx = V[x];
    float v1[MH], v0[MH];
#pragma unroll
    for (int k = 0; k < MH; k++) {
        const int o = d.occ[k];
        v1[k] = (k < md.H && o > 0) ? V[x - md.stride[k]] : 0.0f;
        v0[k] = (k < md.H && o > 1) ? V[x - o * md.stride[k]] : 0.0f;
    }
    const float va = (d.q < md.Q) ? V[x + 2] : 0.0f;
    const float vf = V[d.ph ? x - 1 : x + 1];
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

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Adds a block's two tallies (feasible rows, non-zero successors) to tallies[0..1] with one
// atomic each (every thread of the block calls it).
template <int NT>
__device__ __forceinline__ void block_tally(unsigned long long feas, unsigned long long nz,
                                            unsigned long long* tallies) {
    __shared__ unsigned long long part[2][NT / 32];
    for (int o = 16; o > 0; o >>= 1) {
        feas += __shfl_xor_sync(0xffffffffu, feas, o);
        nz += __shfl_xor_sync(0xffffffffu, nz, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        part[0][w] = feas;
        part[1][w] = nz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long f = 0, z = 0;
        for (int i = 0; i < NT / 32; ++i) {
            f += part[0][i];
            z += part[1][i];
        }
        atomicAdd(&tallies[0], f);
        atomicAdd(&tallies[1], z);
    }
}

// Block-wide max of a non-negative value over NT threads; result valid in thread 0.
// Every thread of the block must call it.
template <typename T, int NT>
__device__ __forceinline__ T block_max(T v) {
    __shared__ T part[NT / 32];
    v = warp_max(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) part[w] = v;
    __syncthreads();
    T r = 0;
    if (threadIdx.x < 32) {
        r = (l < NT / 32) ? part[l] : T(0);
        r = warp_max(r);
    }
    __syncthreads();
    return r;
}

// Block-wide max of a non-negative float for any block size up to 1024 threads (a whole
// number of warps); result valid in thread 0.  Every thread of the block must call it.
__device__ __forceinline__ float block_max_dyn(float v) {
    __shared__ float part[32];
    v = warp_max(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int nw = (int)(blockDim.x >> 5);
    if (l == 0) part[w] = v;
    __syncthreads();
    float r = 0.0f;
    if (threadIdx.x < 32) {
        r = (l < nw) ? part[l] : 0.0f;
        r = warp_max(r);
    }
    __syncthreads();
    return r;
}

// Algorithm 4's in-block "episodes" (Section V-H) over one tile of whole blocks, with each
// action's self-transition solved.  A block is the 2(Q+1)(C+1)^h consecutive states that
// share the occupancies of hosts h..H-1: every queue length, phase and occupancy of the h
// inner hosts.  The events of the inner hosts, the arrivals and the phase flips of a state
// stay in its block, everything else leaves it, so a tile of whole blocks needs no block
// index at all.  Given the pass-1 values of the previous iterate V (U(x) = R(x) + gamma
// E[V(next) | x] and defer's self-transition-solved W(x), from k_post<SL> or k_bpost<SL>),
// the tile runs `passes` local Jacobi passes in shared memory in which a successor inside
// the state's block takes the block's previous local values Vl and every other successor
// V.  Each pass corrects the pass-1 values by the in-block terms only:
//   U_l(x) = U(x) + gamma ((1 - p_move(x)) (Vl(x) - V(x)) + D(x)),
//   W_l(x) = W(x) + gamma D(x) / ((1 - gamma) + gamma p_move(x)),
//   D(x) = sum over the in-block events e of x of p_e (Vl(y_e) - V(y_e));
// a placement on an outer host a leaves the block, and of its post-decision state's events
// only the completion on host a (merged with the departure when host a was empty) comes
// back, to s - 2.  The first pass therefore reproduces the plain self-transition sweep bit
// for bit; p passes over blocks of B states are the block iteration of the oracle's CSR
// routine with tile B (the sums differ only in rounding).  One thread per state (blockDim
// >= count); smem holds 4 x blockDim floats; res / vabs accumulate max|V' - V| and |V'|.
// HIN = h, the inner hosts, a compile-time constant so the inner loops are static and the
// outer hosts' digits die after the set-up.
template <int MH, int HIN>
__device__ __forceinline__ void block_tile(const Model& md, const Coef<float>& c, int start, int count,
                                           int passes, const float* __restrict__ Vin, const float* __restrict__ U,
                                           const float* __restrict__ W, float* __restrict__ V_out, float* smem,
                                           Ctl* ctl, float& res, float& vabs) {
    float* Vg = smem;                     // previous iterate on the tile
    float* Vl = smem + blockDim.x;        // local values, double-buffered across passes
    float* Vn = smem + 2 * blockDim.x;
    float* Ul = smem + 3 * blockDim.x;    // corrected pass-1 values of the current pass
    const int i = threadIdx.x;
    const bool act = i < count;
    const int s = start + i;
    Digits d;
    float ug = 0.0f, wg = 0.0f, vg = 0.0f, g1 = 0.0f, gd = 0.0f;
    float uo[MH], gp[MH];
    if (act) {
        decode<MH>(md, s, d);
        vg = Vin[s];
        ug = U[s];
        wg = W[s];
        Vg[i] = vg;
        Vl[i] = vg;
        // probability that an event leaves s read as a post-decision state (pass-1 order)
        float pm = 0.0f;
#pragma unroll
        for (int k = 0; k < MH; k++) {
            if (k < md.H) {
                const int o = d.occ[k];
                if (o == 1) {
                    pm += c.pc[k] + c.pd[k];
                } else if (o > 1) {
                    pm += c.pc[k] * (float)o;
                    pm += c.pd[k];
                }
            }
        }
        if (d.q < md.Q) pm += c.pa;
        pm += d.ph ? c.pf1 : c.pf0;
        g1 = c.gamma * (1.0f - pm);
        gd = __fdiv_rn(c.gamma, fmaf(c.gamma, pm, 1.0f - c.gamma));
        // placements on outer hosts: the pass-1 value of their post-decision state and
        // gamma times the probability of its one event back into the block
#pragma unroll
        for (int k = 0; k < MH; k++) {
            const bool f = k >= HIN && d.q >= 1 && k < md.H && d.occ[k] < md.C && (k == md.H - 1 || d.ph == 1) &&
                           VC_IN_BOUNDS(ctl, s + md.stride[k] - 2 < md.S);
            uo[k] = f ? U[s + md.stride[k] - 2] : -INFINITY;
            gp[k] = k < md.H ? c.gamma * (c.pc[k] * (float)(d.occ[k] + 1) + (d.occ[k] == 0 ? c.pd[k] : 0.0f)) : 0.0f;
        }
    }
    __syncthreads();
    float vnew = vg;
    for (int pass = 0; pass < passes; pass++) {
        float wl = wg;
        if (act) {
            float D = 0.0f;
#pragma unroll
            for (int k = 0; k < MH; k++) {
                if (k < HIN) {
                    const int o = d.occ[k];
                    const int j1 = i - md.stride[k];
                    if (o == 1) {
                        D = fmaf(c.pc[k] + c.pd[k], Vl[j1] - Vg[j1], D);
                    } else if (o > 1) {
                        const int j0 = i - o * md.stride[k];
                        D = fmaf(c.pc[k] * (float)o, Vl[j1] - Vg[j1], D);
                        D = fmaf(c.pd[k], Vl[j0] - Vg[j0], D);
                    }
                }
            }
            if (d.q < md.Q) D = fmaf(c.pa, Vl[i + 2] - Vg[i + 2], D);
            const int jf = d.ph ? i - 1 : i + 1;
            D = fmaf(d.ph ? c.pf1 : c.pf0, Vl[jf] - Vg[jf], D);
            Ul[i] = fmaf(g1, Vl[i] - Vg[i], fmaf(c.gamma, D, ug));
            wl = fmaf(gd, D, wg);
        }
        __syncthreads();
        if (act) {
            float best = -INFINITY;
            const float back = (d.q >= 1) ? Vl[i - 2] - Vg[i - 2] : 0.0f;
#pragma unroll
            for (int k = 0; k < MH; k++) {
                float u = -INFINITY;
                if (k < HIN) {
                    if (d.q >= 1 && k < md.H && d.occ[k] < md.C && (k == md.H - 1 || d.ph == 1))
                        u = Ul[i + md.stride[k] - 2];
                } else if (uo[k] != -INFINITY) {
                    u = fmaf(gp[k], back, uo[k]);
                }
                if (u > best) best = u;
            }
            if (wl > best) best = wl;  // defer last: ties keep the lower action
            vnew = best;
            Vn[i] = vnew;
        }
        __syncthreads();
        float* t = Vl;
        Vl = Vn;
        Vn = t;
    }
    if (act) {
        V_out[s] = vnew;
        res = fmaxf(res, fabsf(vnew - vg));
        vabs = fmaxf(vabs, fabsf(vnew));
    }
}

__device__ __forceinline__ unsigned int fbits(float x) { return __float_as_uint(x); }
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

__device__ __forceinline__ bool loop_done(const SweepCtl& sc) {
    if (sc.mode != kModeLoop32) return false;
    return *((volatile int*)&sc.ctl->done) != 0;
}

__device__ __forceinline__ long long loop_sweep(const SweepCtl& sc) {
    if (sc.mode != kModeLoop32) return 0;
    return *((volatile long long*)&sc.ctl->sweeps);
}

// Residual bookkeeping, called by thread 0 of every block once its block maximum is known.
// Loop mode: one atomicMax per block into the sweep's ring slot, then the last block to
// arrive (ticket counter) closes the sweep: advances the sweep count, records the output
// buffer, clears the next slot and decides termination (tolerance max(tol, 4 ulp(max|V|)),
// FP32 stall, or max_sweeps).  Order independent, so every run takes the same decisions.
// Standalone FP64 mode: the block maximum into cert64.
template <typename T>
__device__ void finish_block(const SweepCtl& sc, T res, T vmax, long long sweep) {
    if (threadIdx.x != 0 || sc.mode == kModeNone) return;
    Ctl* c = sc.ctl;
    if (sc.mode == kModeCert64) {
        atomicMax(&c->cert64, dbits((double)res));
        return;
    }
    const int slot = (int)(sweep % kRing);
    atomicMax(&c->res32[slot], fbits((float)res));
    atomicMax(&c->vmax32[slot], fbits((float)vmax));
    __threadfence();
    const unsigned int t = atomicAdd(&c->ticket, 1u);
    if (t != gridDim.x - 1) return;
    __threadfence();
    const long long k = sweep + 1;
    c->ticket = 0;
    c->sweeps = k;
    c->final_buf = sc.out_index;
    const int next = (int)(k % kRing);
    int done = 0;
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
    if (!done && k >= c->max_sweeps) done = 2;
    if (*((volatile int*)&c->error) & kErrTimeout) done = 4;
    c->done = done;
    __threadfence();
}

// ---------------------------------------------------------------------------- handle
// Tiling of the pipelined CSR sweep: tiles of `ts` consecutive states whose rows (and
// entries, at most `cap`) are staged in shared memory by bulk asynchronous copies.
struct CsrPlan {
    bool tma = false;
    bool sliced = false; // sweep the sliced layout (k_sell) instead of the CSR
    int apad = 8;        // lanes per state (power of two >= A)
    int ts = 0;          // states per tile
    int64_t cap = 0;     // max entries of a tile (+ alignment slack)
    int stages = 0;
    int ctas_per_sm = 0;
    int smem = 0;        // dynamic shared memory per CTA
    int64_t ntiles = 0;
    int warps = 0;       // consumer warps per CTA (sliced ring sweep)
    int minb = 1;        // register budget of the sliced ring kernel (1: 80 registers, 2: 60)
};

struct KrylovCtl;  // vc_krylov.cuh

struct Mdp {
    int fmt;              // VC_IMPLICIT / VC_CSR_F32 / VC_CSR_BF16 (| VC_PADDED)
    bool has_model;
    int S, A;
    double gamma;
    Model md;
    Rates rates;
    Coef<float> c32;
    Coef<double> c64;
    // explicit CSR (owned; col / val / R / scale carry 16-byte tail padding for bulk copies)
    int64_t nnz_stored = 0, nnz_logical = 0, feasible_rows = 0;
    int64_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    void* val = nullptr;        // float or uint16 (bf16)
    float* scale = nullptr;     // BF16 per-row scale
    float* R = nullptr;         // [S*A], -inf = infeasible
    double* val64 = nullptr;    // exact FP64 probabilities beside val (handles built from a model's
    double* R64 = nullptr;      // FP64 rows without a register generator); the FP64 steps use them
    double* rate_tab = nullptr; // rates.occ_tab (device, owned)
    CsrPlan plan;
    std::string tune_report;    // candidates and times of the last autotune
    // sliced copy of the stored matrix (SELL-C-sigma, C = 32 states per slice): one
    // 128-byte-aligned record per slice in a byte slab (header, state map, R / scale,
    // col / val rows lane-fastest)
    int64_t sell_slices = 0, nnz_sliced = 0, sell_bytes = 0;
    int64_t* sell_rec = nullptr;          // [G + 1] record offsets in units of 128 bytes
    unsigned char* sell_slab = nullptr;   // the records
    int64_t sell_max_tile[3] = {0, 0, 0};  // bytes of the largest tile of 1, 2, 4 slice records (planning)
    // work buffers: carved out of one owned allocation (work), the two pinned mirrors out
    // of one pinned allocation (work_host)
    void* work = nullptr;
    void* work_host = nullptr;
    float* Vb = nullptr;        // FP32 ping-pong partner
    float* U32 = nullptr;       // FP32 post-decision values (implicit)
    float* U32s = nullptr;      // FP32 defer values with the self-transition solved (implicit)
    double* U64 = nullptr;      // FP64 post-decision values
    double* V64a = nullptr;     // FP64 pair
    double* V64b = nullptr;
    float* E0 = nullptr;        // FP32 correction ping-pong
    float* E1 = nullptr;
    float* Rres = nullptr;      // FP32 copy of the FP64 policy residual
    int32_t* pi = nullptr;      // policy under refinement
    int32_t* pi2 = nullptr;
    float* kr = nullptr;        // BiCGSTAB vectors of the correction solve: r, p, v, s, t ([5][S])
    double* kr_part = nullptr;  // BiCGSTAB per-block partials ([3][grid])
    KrylovCtl* kctl = nullptr;  // BiCGSTAB scalars (device) and their pinned mirror
    KrylovCtl* kctl_host = nullptr;
    Ctl* ctl = nullptr;         // device control block
    Ctl* ctl_host = nullptr;    // pinned mirror
    int64_t device_bytes = 0;
    int num_sms = 0;
    long long spin_polls = -1;  // bounded-wait cap for the pipelined sweeps (-1 = the default)
    // in-block iteration of the implicit form (VC_ITER_BLOCK): blocks of the states of
    // blk_h inner hosts' occupancies (B = 2(Q+1)(C+1)^blk_h), blk_passes local passes
    int blk_h = -1;             // -1: the largest h with B <= 1024
    int blk_passes = 4;
    int blk_grid = 0;           // resident blocks of k_block (0: not yet queried)
};

// Process-wide count of kernels this library has enqueued.
void count_launches(int n);

// Scoped NVTX range: names the library's phases on a profiler's timeline (a no-op when no
// tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Kernels / launchers implemented in the .cu files.
int alloc_dev(Mdp* m, void** p, size_t bytes);
int build_model(const vc_params* p, Mdp* m);
int upload_rate_table(Mdp* m, cudaStream_t st);
int build_csr_from_model(Mdp* m, cudaStream_t st);
int count_model_rows(Mdp* m, cudaStream_t st);
int build_csr_user(Mdp* m, const int64_t* row_ptr, const int32_t* col, const void* val, int val_dtype,
                   const float* row_scale, const float* R, cudaStream_t st);
int plan_csr(Mdp* m, cudaStream_t st);
// CSR of the binary-action model (vc_binary.cu), with its exact FP64 values and rewards.
int build_csr_binary(Mdp* m, const vc_binary_params* p, cudaStream_t st);
// Sliced layout (vc_sell.cu): build from the stored CSR, sweep, sweep bytes.
int build_sliced(Mdp* m, cudaStream_t st);
int sell_plans(Mdp* m, cudaStream_t st, std::vector<CsrPlan>& out);
int sell_sweep32(Mdp* m, const float* V_in, float* V_out, int32_t* pi, float* qgap, SweepCtl sc, cudaStream_t st);
int64_t sell_sweep_bytes(const Mdp* m);
int csr_candidates(Mdp* m, cudaStream_t st, std::vector<CsrPlan>& cands);
// Per-process caches, keyed by device, of a kernel's attributes, of its dynamic
// shared-memory limit (set once) and of its occupancy for a launch shape: the queries cost
// microseconds each and every handle plans its launches again.
cudaError_t cached_func_attributes(const void* fn, cudaFuncAttributes* fa);
cudaError_t cached_set_max_dyn_smem(const void* fn, int bytes);
cudaError_t cached_occupancy(const void* fn, int threads, size_t smem, int* per_sm);
int autotune_csr(Mdp* m, int reps, cudaStream_t st, double* best_us);

// Grid of the persistent state-parallel kernels.
int state_grid(const Mdp* m);

// Inner hosts and block size of the in-block iteration of an implicit handle.
int block_shape(const Mdp* m, int* h_out, int* B_out);

// One FP32 Bellman backup V_in -> V_out (implicit or CSR), optional policy / gap.
int launch_sweep32(Mdp* m, const float* V_in, float* V_out, int32_t* pi, float* qgap, SweepCtl sc,
                   cudaStream_t st);
// One FP64 full Bellman backup (exact model when available, else the stored CSR in FP64).
int launch_bellman64(Mdp* m, const double* V_in, double* V_out, int32_t* pi, double* qgap, SweepCtl sc,
                     cudaStream_t st);
// r = (R_pi + gamma P_pi V64) - V64 in FP64, stored as float (policy residual).
int launch_resid64(Mdp* m, const int32_t* pi, const double* V64, float* r, SweepCtl sc, cudaStream_t st);
// One FP32 correction sweep e_out = r + gamma P_pi e_in.
int launch_correct32(Mdp* m, const int32_t* pi, const float* r, const float* e_in, float* e_out, SweepCtl sc,
                     cudaStream_t st);
// V64 += e (FP64 add of the FP32 correction).
int launch_axpy64(double* V64, const float* e, int n, cudaStream_t st);
int launch_f32_to_f64(const float* in, double* out, int n, cudaStream_t st);
// Greedy heuristic policy (Algorithm 2 read as a policy) of a model handle.
int launch_greedy(Mdp* m, int32_t* pi, cudaStream_t st);

// out[0..n] = exclusive prefix sums of cnt (int32 -> int64), out[n] = total.
int exclusive_scan(Mdp* m, const int32_t* cnt, int64_t n, int64_t* out, cudaStream_t st);

// Adjoint gradient kernels (vc_grad.cu).
int launch_adj_count(Mdp* m, const int32_t* pi, int32_t* cnt, int* err, cudaStream_t st);
int launch_adj_fill(Mdp* m, const int32_t* pi, const int64_t* rowT, int32_t* fillpos, int32_t* colT, float* valT,
                    double* valT64, cudaStream_t st);
int launch_adj_resid64(Mdp* m, const int64_t* rowT, const int32_t* colT, const double* valT64, const double* rho,
                       const double* lam, float* r, SweepCtl sc, cudaStream_t st);
int launch_f64_to_f32(const double* in, float* out, int n, cudaStream_t st);
int grad_partial_stride(const Mdp* m);
int launch_grad_contract(Mdp* m, const int32_t* pi, const double* V, const double* lam, const double* rho,
                         double* partial, double* out, cudaStream_t st);

// CSR kernels (vc_csr.cu).
int csr_sweep32(Mdp* m, const float* V_in, float* V_out, int32_t* pi, float* qgap, SweepCtl sc, cudaStream_t st);
int csr_bellman64(Mdp* m, const double* V_in, double* V_out, int32_t* pi, double* qgap, SweepCtl sc,
                  cudaStream_t st);
int csr_resid64(Mdp* m, const int32_t* pi, const double* V64, float* r, SweepCtl sc, cudaStream_t st);
int csr_correct32(Mdp* m, const int32_t* pi, const float* r, const float* e_in, float* e_out, SweepCtl sc,
                  cudaStream_t st);

}  // namespace vc
