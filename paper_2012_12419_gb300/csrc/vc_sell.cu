// vc_sell.cu -- sliced layout of the stored matrix and its FP32 Bellman sweep
// (Algorithm 3, step 2; Eq. 18 backup over the stored rows r = s*A + a).
//
// Layout: SELL-C-sigma (Kreutzer, Hager, Wellein, Fehske, Bishop, SIAM J. Sci. Comput.
// 36(5), 2014) with C = 32 and sigma = 4096.  States are sorted inside aligned windows of
// 4096 by (feasible-action mask, total row length descending, index), stable, so slices
// of 32 states group states with the same feasible actions (in the placement model: the
// same channel phase and queue-empty bit) in ascending state order.  Slice g holds, for
// each action a, a block of width(g, a) x 32 entries stored lane-fastest: entry j of the
// row of lane l sits at (off[g*A+a] + j)*32 + l.  width is the longest feasible row of the
// block; shorter rows are padded with (column = the lane's own state, value 0), which
// leaves every row sum bitwise unchanged.  Infeasible rows (R = -inf) store nothing.
//
// Sweeps keep the arithmetic of the CSR kernels (row sum in column order with fused
// multiply-adds in batches of 16, q = R + gamma (scale) sum, max over actions in order
// with the lowest maximising index), so both layouts give bitwise-equal results.
//
// k_sell_ring (pipelined): one producer lane stages tiles of consecutive slices -- the
// slices' block offsets, state map, R (and scale) and their contiguous col / val range --
// into a ring of shared memory with bulk asynchronous copies (every array of the layout
// starts each slice on a 128-byte boundary, so no realignment is needed), completion
// counted on an mbarrier, L2 evict-first.  Tiles take their actual size in the ring, so
// the buffering is not sized for the largest tile.  Consumer warps take (slice, action)
// blocks round-robin, one lane per state: shared-memory reads are lane-consecutive (no
// bank conflicts) and the V gathers of a warp fall on a few cache lines because the
// lanes' successors share offsets.  Q values go to a per-tile shared buffer; the warp
// that completes a tile's last block takes the max over actions and releases the tile.
//
// k_sell (direct): one warp per slice straight from global memory, for comparison and
// as the fallback when no tile fits in shared memory.
#include <math.h>
#include <stdio.h>

#include <vector>

#include "vc_internal.cuh"
#include "vc_ptx.cuh"

namespace vc {

constexpr int kSellC = 32;
constexpr int kSellSigma = 4096;
constexpr int kSellBatch = 16;
constexpr int kSellMaxA = 31;  // the slice's A + 1 block offsets live in one warp's lanes

// ------------------------------------------------------------------------ build
// Sort key of a state: feasible-action mask (bits 32..62), 2^20 - 1 - total row length
// (bits 12..31), index inside its window (bits 0..11).  Padding states past S get ~0.
__global__ void k_sell_keys(const int64_t* __restrict__ row_ptr, const float* __restrict__ R, int S, int A,
                            int64_t n_pad, uint64_t* __restrict__ keys) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_pad;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (s >= S) {
            keys[s] = ~0ull;
            continue;
        }
        uint32_t mask = 0;
        int64_t tot = 0;
        for (int a = 0; a < A; ++a) {
            const int64_t r = s * A + a;
            if (R[r] != -INFINITY) {
                mask |= 1u << (a < 30 ? a : 30);
                tot += row_ptr[r + 1] - row_ptr[r];
            }
        }
        const uint64_t len = (uint64_t)(tot < 0xFFFFF ? tot : 0xFFFFF);
        keys[s] = ((uint64_t)mask << 32) | ((0xFFFFFull - len) << 12) | (uint64_t)(s & (kSellSigma - 1));
    }
}

// One block per window: bitonic sort of the window's 4096 keys in shared memory, then
// perm = window start + index field (keys are distinct, so the order is deterministic).
__global__ void __launch_bounds__(1024) k_sell_sort(const uint64_t* __restrict__ keys, int32_t* __restrict__ perm) {
    __shared__ uint64_t k[kSellSigma];
    const int64_t base = (int64_t)blockIdx.x * kSellSigma;
    for (int i = threadIdx.x; i < kSellSigma; i += blockDim.x) k[i] = keys[base + i];
    __syncthreads();
    for (int size = 2; size <= kSellSigma; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < kSellSigma / 2; i += blockDim.x) {
                const int lo = (i / stride) * 2 * stride + (i % stride);
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const uint64_t x = k[lo], y = k[hi];
                if ((x > y) == up) {
                    k[lo] = y;
                    k[hi] = x;
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < kSellSigma; i += blockDim.x) {
        const uint64_t u = k[i];
        perm[base + i] = (u == ~0ull) ? -1 : (int32_t)(base + (int64_t)(u & (kSellSigma - 1)));
    }
}

// Warp per slice: width(g, a) = longest feasible row among the slice's lanes.
__global__ void k_sell_width(const int64_t* __restrict__ row_ptr, const float* __restrict__ R,
                             const int32_t* __restrict__ perm, int A, int64_t G, int32_t* __restrict__ width) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {
        const int s = perm[g * kSellC + lane];
        for (int a = 0; a < A; ++a) {
            int len = 0;
            if (s >= 0) {
                const int64_t r = (int64_t)s * A + a;
                if (R[r] != -INFINITY) len = (int)(row_ptr[r + 1] - row_ptr[r]);
            }
            const int w = __reduce_max_sync(0xffffffffu, len);
            if (lane == 0) width[g * A + a] = w;
        }
    }
}

// Warp per slice: copy rows into their blocks, pad, and lay R / scale out per block.
template <typename VT>
__global__ void k_sell_fill(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const VT* __restrict__ val, const float* __restrict__ R, const float* __restrict__ scale,
                            const int32_t* __restrict__ perm, int A, int64_t G, const int64_t* __restrict__ off,
                            int32_t* __restrict__ col_s, VT* __restrict__ val_s, float* __restrict__ R_s,
                            float* __restrict__ scale_s) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {
        const int s = perm[g * kSellC + lane];
        for (int a = 0; a < A; ++a) {
            const int64_t b = g * A + a;
            const int64_t o0 = off[b];
            const int w = (int)(off[b + 1] - o0);
            int64_t lo = 0;
            int len = 0;
            float rr = -INFINITY, sc = 1.0f;
            if (s >= 0) {
                const int64_t r = (int64_t)s * A + a;
                rr = R[r];
                if (scale) sc = scale[r];
                if (rr != -INFINITY) {
                    lo = row_ptr[r];
                    len = (int)(row_ptr[r + 1] - lo);
                }
            }
            for (int j = 0; j < w; ++j) {
                const int64_t e = (o0 + j) * kSellC + lane;
                if (j < len) {
                    col_s[e] = col[lo + j];
                    val_s[e] = val[lo + j];
                } else {
                    col_s[e] = s >= 0 ? s : 0;
                    val_s[e] = VT(0);
                }
            }
            R_s[b * kSellC + lane] = rr;
            if (scale_s) scale_s[b * kSellC + lane] = sc;
        }
    }
}

static unsigned warp_grid(int64_t warps, int sms) {
    const int64_t blocks = (warps * 32 + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sms * 16;
    return (unsigned)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

int build_sliced(Mdp* m, cudaStream_t st) {
    const int base = m->fmt & 0xF;
    if (base == VC_IMPLICIT) return fail(VC_ERR_ARG, "the sliced layout needs a stored (CSR) matrix");
    if (m->A > kSellMaxA) return fail(VC_ERR_ARG, "the sliced layout needs A <= 31");
    if (m->sell_perm) return VC_OK;  // already built
    const bool bf16 = base == VC_CSR_BF16;
    const int A = m->A;
    const int64_t S = m->S;
    const int64_t n_pad = (S + kSellSigma - 1) / kSellSigma * kSellSigma;
    const int64_t G = (S + kSellC - 1) / kSellC;
    int rc;
    // temporaries: keys, widths (freed below)
    uint64_t* keys = nullptr;
    int32_t* width = nullptr;
    VC_CUDA(cudaMalloc((void**)&keys, 8 * (size_t)n_pad));
    cudaError_t e = cudaMalloc((void**)&width, 4 * (size_t)(G * A + 1));
    if (e != cudaSuccess) {
        cudaFree(keys);
        return cuda_fail(e, "cudaMalloc(sliced widths)");
    }
    auto cleanup = [&]() {
        cudaFree(keys);
        cudaFree(width);
    };
    if ((rc = alloc_dev(m, (void**)&m->sell_perm, 4 * (size_t)n_pad)) ||
        (rc = alloc_dev(m, (void**)&m->sell_off, 8 * (size_t)(G * A + 2)))) {
        cleanup();
        return rc;
    }
    count_launches(4);
    k_sell_keys<<<warp_grid(n_pad / 32 + 1, m->num_sms), kThreads, 0, st>>>(m->row_ptr, m->R, (int)S, A, n_pad,
                                                                            keys);
    k_sell_sort<<<(unsigned)(n_pad / kSellSigma), 1024, 0, st>>>(keys, m->sell_perm);
    k_sell_width<<<warp_grid(G, m->num_sms), kThreads, 0, st>>>(m->row_ptr, m->R, m->sell_perm, A, G, width);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "sliced layout: key / sort / width kernels");
    }
    if ((rc = exclusive_scan(m, width, G * A, m->sell_off, st))) {
        cleanup();
        return rc;
    }
    int64_t rows32 = 0;
    e = cudaMemcpyAsync(&rows32, m->sell_off + G * A, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "sliced layout: size read-back");
    }
    const int64_t nnz = rows32 * kSellC;
    m->sell_slices = G;
    m->nnz_sliced = nnz;
    if ((rc = alloc_dev(m, (void**)&m->sell_col, 4 * (size_t)(nnz + 32))) ||
        (rc = alloc_dev(m, &m->sell_val, (bf16 ? 2 : 4) * (size_t)(nnz + 32))) ||
        (rc = alloc_dev(m, (void**)&m->sell_R, 4 * (size_t)(G * A * kSellC))) ||
        (bf16 && (rc = alloc_dev(m, (void**)&m->sell_scale, 4 * (size_t)(G * A * kSellC))))) {
        cleanup();
        return rc;
    }
    if (bf16)
        k_sell_fill<uint16_t><<<warp_grid(G, m->num_sms), kThreads, 0, st>>>(
            m->row_ptr, m->col, (const uint16_t*)m->val, m->R, m->scale, m->sell_perm, A, G, m->sell_off, m->sell_col,
            (uint16_t*)m->sell_val, m->sell_R, m->sell_scale);
    else
        k_sell_fill<float><<<warp_grid(G, m->num_sms), kThreads, 0, st>>>(
            m->row_ptr, m->col, (const float*)m->val, m->R, nullptr, m->sell_perm, A, G, m->sell_off, m->sell_col,
            (float*)m->sell_val, m->sell_R, nullptr);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "sliced layout: fill");
    count_launches(1);
    return VC_OK;
}

int64_t sell_sweep_bytes(const Mdp* m) {
    const bool bf16 = (m->fmt & 0xF) == VC_CSR_BF16;
    const int64_t blocks = m->sell_slices * m->A;
    return m->nnz_sliced * ((bf16 ? 2 : 4) + 4) + blocks * kSellC * (bf16 ? 8 : 4) + (blocks + 1) * 8 +
           m->sell_slices * kSellC * 4 + 8 * (int64_t)m->S;
}

// ------------------------------------------------------------------------ sweep
struct SellArgs {
    int64_t G;
    int A;
    float gamma;
    const int64_t* off;
    const int32_t* col;
    const void* val;
    const float* R;
    const float* scale;
    const int32_t* perm;
    const float* V_in;
    float* V_out;
    int32_t* pi;
    float* qgap;
};

template <typename VT>
__device__ __forceinline__ float ldcs_v(const VT* p);
template <>
__device__ __forceinline__ float ldcs_v<float>(const float* p) {
    return __ldcs(p);
}
template <>
__device__ __forceinline__ float ldcs_v<uint16_t>(const uint16_t* p) {
    return __uint_as_float((uint32_t)__ldcs(reinterpret_cast<const unsigned short*>(p)) << 16);
}

template <typename VT>
__device__ __forceinline__ float ldsv(const VT* p);
template <>
__device__ __forceinline__ float ldsv<float>(const float* p) {
    return *p;
}
template <>
__device__ __forceinline__ float ldsv<uint16_t>(const uint16_t* p) {
    return __uint_as_float((uint32_t)*p << 16);
}

template <typename VT>
__global__ void __launch_bounds__(kThreads) k_sell(SellArgs a, SweepCtl sc) {
    if (loop_done(sc)) return;
    const long long sweep = loop_sweep(sc);
    const VT* val = reinterpret_cast<const VT*>(a.val);
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * kThreads) >> 5;
    float res = 0.0f, vabs = 0.0f;
    for (int64_t g = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5; g < a.G; g += nw) {
        const int s = __ldcs(a.perm + g * kSellC + lane);
        // lane i < = A holds the offset of block (g, i); block a spans [off_a, off_{a+1})
        const int64_t offl = (lane <= a.A) ? __ldcs(a.off + g * a.A + lane) : 0;
        float b1 = -INFINITY, b2 = -INFINITY;
        int ia = 0;
        for (int act = 0; act < a.A; ++act) {
            const int64_t o0 = __shfl_sync(0xffffffffu, offl, act);
            const int w = (int)(__shfl_sync(0xffffffffu, offl, act + 1) - o0);
            const int64_t blk = (g * a.A + act) * kSellC + lane;
            const float rr = __ldcs(a.R + blk);
            float q = -INFINITY;
            if (rr != -INFINITY) {
                const int32_t* cp = a.col + o0 * kSellC + lane;
                const VT* vp = val + o0 * kSellC + lane;
                float acc = 0.0f;
                for (int j0 = 0; j0 < w; j0 += kSellBatch) {
                    float wv[kSellBatch], gv[kSellBatch];
#pragma unroll
                    for (int u = 0; u < kSellBatch; ++u) {
                        if (j0 + u < w) {
                            wv[u] = ldcs_v<VT>(vp + (int64_t)(j0 + u) * kSellC);
                            gv[u] = __ldg(a.V_in + __ldcs(cp + (int64_t)(j0 + u) * kSellC));
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kSellBatch; ++u)
                        if (j0 + u < w) acc = fmaf(wv[u], gv[u], acc);
                }
                q = rr + a.gamma * (a.scale ? __ldcs(a.scale + blk) * acc : acc);
            }
            // max with the lowest maximising action; second best counts ties
            if (act == 0 || q > b1) {
                b2 = (act == 0) ? -INFINITY : b1;
                b1 = q;
                ia = act;
            } else {
                b2 = fmaxf(b2, q);
            }
        }
        if (s >= 0) {
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

// ------------------------------------------------------------------ pipelined sweep
constexpr int kSlots = 12;      // tiles in flight per CTA
constexpr int kMaxRW = 24;      // most consumer warps per CTA
constexpr int kHead = 512;      // barriers and per-slot words at the start of shared memory
static_assert(kSlots * (8 + 8 + 4 + 4) <= 384 && 384 + 8 * kSlots <= kHead, "slot words exceed the header");

__host__ __device__ inline int round128(long long x) { return (int)((x + 127) & ~127LL); }

// Byte layout of one tile inside the ring: ns slices, nb = ns*A blocks, n_off staged
// offsets, rows rows of 32 entries.  Every region starts on a 128-byte boundary.
struct TileLayout {
    int off_perm, off_R, off_scale, off_col, off_val, bytes;
};

__host__ __device__ inline TileLayout tile_layout(int ns, int nb, int n_off, long long rows, int vt, bool has_scale) {
    TileLayout L;
    L.off_perm = round128(8LL * n_off);
    L.off_R = L.off_perm + 128 * ns;
    L.off_scale = L.off_R + 128 * nb;
    L.off_col = L.off_scale + (has_scale ? 128 * nb : 0);
    L.off_val = L.off_col + round128(128LL * rows);
    L.bytes = L.off_val + round128(32LL * vt * rows);
    return L;
}

struct SellRingArgs {
    int TS;           // slices per tile (the last tile may hold fewer)
    int64_t ntiles;
    int ring;         // bytes of the tile ring
    int qfloats;      // floats of one slot's Q buffer (TS * A * 32)
    int qoff;         // byte offset of the Q buffers
    int roff;         // byte offset of the ring
};

// Producer / consumer sweep over the sliced copy.  Tiles are placed back to back in a
// ring of shared memory at their actual size (a tile that would wrap starts over at the
// ring's base); the producer reuses bytes only after the tiles holding them are released,
// in order.  Consumer warps take the (slice, action) blocks of the CTA's tile sequence
// round-robin, so every warp has work whatever the number of blocks per tile; the warp
// completing a tile's last block takes the max over actions and releases the tile.
template <typename VT>
__global__ void __launch_bounds__((kMaxRW + 1) * 32, 1) k_sell_ring(SellArgs a, SellRingArgs t, SweepCtl sc) {
    extern __shared__ __align__(128) unsigned char smem[];
    if (loop_done(sc)) return;
    const long long sweep = loop_sweep(sc);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kSlots;
    int* done_cnt = reinterpret_cast<int*>(empty + kSlots);
    uint32_t* slot_pos = reinterpret_cast<uint32_t*>(done_cnt + kSlots);
    unsigned long long* slot_end = reinterpret_cast<unsigned long long*>(smem + 384);  // after 288 header bytes
    float* qbuf = reinterpret_cast<float*>(smem + t.qoff);
    unsigned char* ring = smem + t.roff;
    __shared__ int s_fail, s_consumed;
    const int nrw = (int)(blockDim.x >> 5) - 1;  // consumer warps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int A = a.A;
    const int nb_full = t.TS * A;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kSlots; i++) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
            done_cnt[i] = 0;
        }
        fence_mbar_init();
        s_fail = 0;
        s_consumed = 0x7fffffff;
    }
    __syncthreads();
    const VT* val = reinterpret_cast<const VT*>(a.val);
    constexpr int vt = (int)sizeof(VT);
    const bool has_scale = a.scale != nullptr;
    float res = 0.0f, vabs = 0.0f;
    int issued = 0;
    if (warp == nrw) {
        // ---------------- producer: the warp loads the entry bounds of its next 32 tiles at
        // once (one memory round trip per 32 tiles), then lane 0 places and issues them
        __shared__ long long s_bounds[2][32];
        const uint64_t pol = l2_evict_first();
        unsigned long long head = 0, rel = 0;  // monotonic ring bytes: allocated / free below
        int oldest = 0;                         // oldest tile not yet released
        int i = 0;
        int failed = 0;
        for (int64_t c0 = blockIdx.x; c0 < t.ntiles && !failed; c0 += 32LL * gridDim.x) {
            const int64_t tk = c0 + (int64_t)lane * gridDim.x;
            if (tk < t.ntiles) {
                const int64_t g0 = tk * t.TS;
                const int64_t g1 = (g0 + t.TS < a.G) ? g0 + t.TS : a.G;
                s_bounds[0][lane] = a.off[g0 * A];
                s_bounds[1][lane] = a.off[g1 * A];
            }
            __syncwarp();
            if (lane == 0) {
                for (int k = 0; k < 32; ++k, ++i) {
                    const int64_t tile = c0 + (int64_t)k * gridDim.x;
                    if (tile >= t.ntiles) break;
                    const int64_t e0 = s_bounds[0][k], e1 = s_bounds[1][k];
                    const int64_t g0 = tile * t.TS;
                    const int64_t g1 = (g0 + t.TS < a.G) ? g0 + t.TS : a.G;
                    const int ns = (int)(g1 - g0), nb = ns * A;
                    const int64_t b0a = (g0 * A) & ~1LL;
                    const int n_off = (int)((((g1 * A + 1) - b0a) + 1) & ~1LL);
                    const TileLayout L = tile_layout(ns, nb, n_off, e1 - e0, vt, has_scale);
                    unsigned long long pos = head % (unsigned long long)t.ring;
                    if (pos + (unsigned long long)L.bytes > (unsigned long long)t.ring) {
                        head += (unsigned long long)t.ring - pos;  // skip the ring's tail
                        pos = 0;
                    }
                    // reuse bytes (and the slot) only after the tiles holding them are released
                    while (oldest < i &&
                           (head + L.bytes - rel > (unsigned long long)t.ring || i - oldest >= kSlots)) {
                        const int os = oldest % kSlots;
                        if (!mbar_wait(&empty[os], (uint32_t)((oldest / kSlots) & 1))) {
                            failed = 1;
                            break;
                        }
                        rel = slot_end[os];
                        oldest++;
                    }
                    if (failed) {
                        atomicExch(&s_fail, 1);
                        break;
                    }
                    const int s = i % kSlots;
                    slot_end[s] = head + L.bytes;
                    slot_pos[s] = (uint32_t)pos;
                    head += L.bytes;
                    const uint32_t b_perm = (uint32_t)ns * 128u, b_R = (uint32_t)nb * 128u;
                    const uint32_t b_col = (uint32_t)(e1 - e0) * 128u;
                    const uint32_t b_val = (uint32_t)(e1 - e0) * (uint32_t)(32 * vt);
                    const uint32_t total =
                        (uint32_t)n_off * 8u + b_perm + b_R + (has_scale ? b_R : 0u) + b_col + b_val;
                    unsigned char* base = ring + pos;
                    mbar_arrive_expect_tx(&full[s], total);
                    bulk_g2s(base, a.off + b0a, (uint32_t)n_off * 8u, &full[s], pol);
                    bulk_g2s(base + L.off_perm, a.perm + g0 * kSellC, b_perm, &full[s], pol);
                    bulk_g2s(base + L.off_R, a.R + g0 * A * kSellC, b_R, &full[s], pol);
                    if (has_scale) bulk_g2s(base + L.off_scale, a.scale + g0 * A * kSellC, b_R, &full[s], pol);
                    if (b_col) {
                        bulk_g2s(base + L.off_col, a.col + e0 * kSellC, b_col, &full[s], pol);
                        bulk_g2s(base + L.off_val, val + e0 * kSellC, b_val, &full[s], pol);
                    }
                    issued = i + 1;
                }
            }
            failed = __shfl_sync(0xffffffffu, failed, 0);
            __syncwarp();
        }
    } else {
        // ---------------- consumers
        int i = 0;
        const int step = nb_full % nrw;
        int rot = 0;  // (i * nb_full) mod nrw, kept incrementally
        for (int64_t tile = blockIdx.x; tile < t.ntiles; tile += gridDim.x, ++i) {
            // this warp's blocks of the tile: global block index i*nb_full + b = warp (mod nrw)
            int b = warp - rot;
            if (b < 0) b += nrw;
            rot += step;
            if (rot >= nrw) rot -= nrw;
            if (b >= nb_full) continue;
            const int64_t g0 = tile * t.TS;
            const int ns = (int)(((g0 + t.TS < a.G) ? g0 + t.TS : a.G) - g0);
            const int nb = ns * A;
            if (b >= nb) continue;
            const int s = i % kSlots;
            if (!mbar_wait(&full[s], (uint32_t)((i / kSlots) & 1))) {
                atomicExch(&s_fail, 1);
                break;
            }
            const unsigned char* base = ring + *((volatile uint32_t*)&slot_pos[s]);
            const int64_t* offs = reinterpret_cast<const int64_t*>(base);
            const int delta = (int)(g0 * A - ((g0 * A) & ~1LL));
            const int64_t e0 = offs[delta];
            const int n_off = (int)((((g0 + ns) * A + 1 - ((g0 * A) & ~1LL)) + 1) & ~1LL);
            const TileLayout L = tile_layout(ns, nb, n_off, offs[delta + nb] - e0, vt, has_scale);
            const float* Rs = reinterpret_cast<const float*>(base + L.off_R);
            const float* Ss = has_scale ? reinterpret_cast<const float*>(base + L.off_scale) : nullptr;
            const int32_t* cs = reinterpret_cast<const int32_t*>(base + L.off_col);
            const VT* vs = reinterpret_cast<const VT*>(base + L.off_val);
            float* qb = qbuf + s * t.qfloats;
            bool last = false;
            for (; b < nb; b += nrw) {
                const float rr = Rs[b * kSellC + lane];
                float q = -INFINITY;
                if (rr != -INFINITY) {
                    const int o0 = (int)(offs[delta + b] - e0);
                    const int w = (int)(offs[delta + b + 1] - offs[delta + b]);
                    const int32_t* cp = cs + o0 * kSellC + lane;
                    const VT* vp = vs + o0 * kSellC + lane;
                    float acc = 0.0f;
                    for (int j0 = 0; j0 < w; j0 += kSellBatch) {
                        float wv[kSellBatch], gv[kSellBatch];
#pragma unroll
                        for (int u = 0; u < kSellBatch; ++u) {
                            if (j0 + u < w) {
                                wv[u] = ldsv<VT>(vp + (j0 + u) * kSellC);
                                gv[u] = __ldg(a.V_in + cp[(j0 + u) * kSellC]);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kSellBatch; ++u)
                            if (j0 + u < w) acc = fmaf(wv[u], gv[u], acc);
                    }
                    q = rr + a.gamma * (Ss ? Ss[b * kSellC + lane] * acc : acc);
                }
                qb[b * kSellC + lane] = q;
                __threadfence_block();
                __syncwarp();
                int l = 0;
                if (lane == 0) l = (atomicAdd(&done_cnt[s], 1) == nb - 1);
                last = __shfl_sync(0xffffffffu, l, 0) != 0;
            }
            if (last) {
                __threadfence_block();
                const int32_t* ps = reinterpret_cast<const int32_t*>(base + L.off_perm);
                for (int k = lane; k < ns * kSellC; k += 32) {
                    const int sl = k >> 5;
                    const int st = ps[k];
                    float b1 = -INFINITY, b2 = -INFINITY;
                    int ia = 0;
                    for (int act = 0; act < A; ++act) {
                        const float q = qb[(sl * A + act) * kSellC + lane];
                        if (act == 0 || q > b1) {
                            b2 = (act == 0) ? -INFINITY : b1;
                            b1 = q;
                            ia = act;
                        } else {
                            b2 = fmaxf(b2, q);
                        }
                    }
                    if (st >= 0) {
                        if (a.V_out) a.V_out[st] = b1;
                        if (a.pi) a.pi[st] = ia;
                        if (a.qgap) a.qgap[st] = (b2 == -INFINITY) ? INFINITY : b1 - b2;
                        res = fmaxf(res, fabsf(b1 - __ldg(a.V_in + st)));
                        vabs = fmaxf(vabs, fabsf(b1));
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    done_cnt[s] = 0;
                    __threadfence_block();
                    mbar_arrive(&empty[s]);
                }
            }
        }
        if (lane == 0) atomicMin(&s_consumed, i);
    }
    __syncthreads();
    if (s_fail) {
        // drain this CTA's copies still in flight before shared memory is released
        if (warp == nrw && lane == 0) {
            for (int j = (s_consumed < issued ? s_consumed : issued); j < issued; ++j)
                mbar_wait(&full[j % kSlots], (uint32_t)((j / kSlots) & 1));
            atomicOr(&sc.ctl->error, kErrTimeout);
        }
    }
    if (sc.mode == kModeNone) return;
    res = block_max_dyn(res);
    vabs = block_max_dyn(vabs);
    finish_block<float>(sc, res, vabs, sweep);
}

// Candidate launch shapes of the ring sweep, in preference order: (CTAs per SM, consumer
// warps per CTA, slices per tile); the ring takes the shared memory left after the Q
// buffers and must hold the largest tile.
int sell_plans(Mdp* m, cudaStream_t st, std::vector<CsrPlan>& out) {
    out.clear();
    if (!m->sell_perm) return VC_OK;
    const bool bf16 = (m->fmt & 0xF) == VC_CSR_BF16;
    const int vt = bf16 ? 2 : 4;
    const int A = m->A;
    int dev = 0, smem_sm = 0, smem_blk = 0;
    VC_CUDA(cudaGetDevice(&dev));
    VC_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    VC_CUDA(cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (m->sell_slice_rows.empty()) {
        const int64_t G = m->sell_slices;
        std::vector<int64_t> off((size_t)(G * A + 1));
        VC_CUDA(cudaMemcpyAsync(off.data(), m->sell_off, 8 * off.size(), cudaMemcpyDeviceToHost, st));
        VC_CUDA(cudaStreamSynchronize(st));
        m->sell_slice_rows.resize((size_t)G);
        for (int64_t g = 0; g < G; ++g) m->sell_slice_rows[g] = off[(g + 1) * A] - off[g * A];
    }
    const std::vector<int64_t>& rows = m->sell_slice_rows;
    // (CTAs per SM, consumer warps), preferred first
    const int shapes[][2] = {{2, 12}, {1, 24}, {2, 8}};
    for (int TS : {1, 2}) {
        // largest tile of TS slices
        long long max_tile = 0;
        for (int64_t g0 = 0; g0 < (int64_t)rows.size(); g0 += TS) {
            long long r = 0;
            const int ns = (int)std::min<int64_t>(TS, (int64_t)rows.size() - g0);
            for (int k = 0; k < ns; ++k) r += rows[g0 + k];
            const TileLayout L = tile_layout(ns, ns * A, ns * A + 3, r, vt, bf16);
            max_tile = std::max<long long>(max_tile, L.bytes);
        }
        for (auto& sh : shapes) {
            const int ctas = sh[0], nrw = sh[1];
            const void* fn = bf16 ? (const void*)k_sell_ring<uint16_t> : (const void*)k_sell_ring<float>;
            cudaFuncAttributes fa;
            VC_CUDA(cudaFuncGetAttributes(&fa, fn));
            const int dyn_max = smem_blk - (int)fa.sharedSizeBytes;
            VC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
            const int threads = (nrw + 1) * 32;
            if (threads > fa.maxThreadsPerBlock || (long long)threads * fa.numRegs * ctas > 65536) continue;
            const int qoff = kHead;
            const int qbytes = kSlots * round128(4LL * TS * A * kSellC);
            const int budget = std::min(dyn_max, (smem_sm - 1024 * ctas) / ctas - (int)fa.sharedSizeBytes);
            const int ring = ((budget - qoff - qbytes) / 128) * 128;
            if (ring < max_tile + 128) continue;
            const int need = qoff + qbytes + ring;
            int per_sm = 0;
            VC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, (size_t)need));
            if (per_sm < 1) continue;
            CsrPlan P;
            P.sliced = true;
            P.tma = true;
            P.ts = TS;
            P.cap = ring;
            P.stages = kSlots;
            P.warps = nrw;
            P.ctas_per_sm = per_sm < ctas ? per_sm : ctas;
            P.smem = need;
            P.ntiles = (m->sell_slices + TS - 1) / TS;
            out.push_back(P);
        }
    }
    return VC_OK;
}

int sell_sweep32(Mdp* m, const float* V_in, float* V_out, int32_t* pi, float* qgap, SweepCtl sc, cudaStream_t st) {
    SellArgs a;
    a.G = m->sell_slices;
    a.A = m->A;
    a.gamma = (float)m->gamma;
    a.off = m->sell_off;
    a.col = m->sell_col;
    a.val = m->sell_val;
    a.R = m->sell_R;
    a.scale = m->sell_scale;
    a.perm = m->sell_perm;
    a.V_in = V_in;
    a.V_out = V_out;
    a.pi = pi;
    a.qgap = qgap;
    const bool bf16 = (m->fmt & 0xF) == VC_CSR_BF16;
    if (m->plan.tma) {
        SellRingArgs t;
        t.TS = m->plan.ts;
        t.ntiles = m->plan.ntiles;
        t.ring = (int)m->plan.cap;
        t.qfloats = round128(4LL * t.TS * m->A * kSellC) / 4;
        t.qoff = kHead;
        t.roff = kHead + kSlots * round128(4LL * t.TS * m->A * kSellC);
        const long long cap = (long long)m->num_sms * m->plan.ctas_per_sm;
        const unsigned grid = (unsigned)(t.ntiles < cap ? t.ntiles : cap);
        const unsigned threads = (unsigned)(m->plan.warps + 1) * 32;
        count_launches(1);
        if (bf16)
            k_sell_ring<uint16_t><<<grid, threads, m->plan.smem, st>>>(a, t, sc);
        else
            k_sell_ring<float><<<grid, threads, m->plan.smem, st>>>(a, t, sc);
        VC_CUDA(cudaGetLastError());
        return VC_OK;
    }
    const int bps = m->plan.ctas_per_sm > 0 ? m->plan.ctas_per_sm : 4;
    const int64_t want = (a.G * kSellC + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)m->num_sms * bps;
    const unsigned grid = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
    count_launches(1);
    if (bf16)
        k_sell<uint16_t><<<grid, kThreads, 0, st>>>(a, sc);
    else
        k_sell<float><<<grid, kThreads, 0, st>>>(a, sc);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

}  // namespace vc
