// vc_sell.cu -- sliced layout of the stored matrix and its FP32 Bellman sweep
// (Algorithm 3, step 2; Eq. 18 backup over the stored rows r = s*A + a).
//
// Layout: SELL-C-sigma (Kreutzer, Hager, Wellein, Fehske, Bishop, SIAM J. Sci. Comput.
// 36(5), 2014) with C = 32 and sigma = 4096.  States are sorted inside aligned windows of
// 4096 by (feasible-action mask, total row length descending, index), stable, so slices
// of 32 states group states with the same feasible actions (in the placement model: the
// same channel phase and queue-empty bit) in ascending state order.  For each action a,
// slice g holds a block of width(g, a) rows of 32 entries stored lane-fastest; width is
// the longest feasible row of the block and shorter rows are padded with (column = the
// lane's own state, value 0), which leaves every row sum bitwise unchanged.  Infeasible
// rows (R = -inf) store nothing, and neither do a stored row's explicit zeros (a padded
// CSR's filler entries): a zero term leaves the row's fused multiply-add chain bitwise
// unchanged for finite V, so the row is its non-zero entries in column order.
//
// Everything one slice needs is one contiguous record in a byte slab, every region on a
// 128-byte boundary:
//   [0, 128)     int32 hdr[32]: hdr[a] = first row of action a's block, hdr[A] = rows
//   [128, 256)   int32 perm[32]: the state of each lane (-1 = padding lane)
//   [256, ...)   float R[A][32] (-inf = infeasible), then for BF16 float scale[A][32]
//   col base     int32 col[rows][32]
//   val base     float or bf16 val[rows][32]
// so a tile of consecutive slices is one contiguous byte range: one bulk copy.
//
// Sweeps keep the arithmetic of the CSR kernels (row sum in column order with fused
// multiply-adds in batches of 16, q = R + gamma (scale) sum, max over actions in order
// with the lowest maximising index), so both layouts give bitwise-equal results.
//
// k_sell_ring (pipelined): one producer lane stages tiles of consecutive slice records
// into a ring of shared memory, one cp.async.bulk per tile, completion counted on an
// mbarrier, L2 evict-first.  Tiles take their actual size in the ring (a tile that would
// wrap restarts at the ring base; bytes are reused only after the tiles holding them are
// released, in order).  Consumer warps take (slice, action) blocks of the CTA's tile
// sequence round-robin, one lane per state: shared-memory reads are lane-consecutive (no
// bank conflicts) and the V gathers of a warp fall on a few cache lines because the
// lanes' successors share offsets.  A block's Q values overwrite its own R row in the
// ring (read once, by the same lane), so no separate Q buffer takes shared memory from the
// ring; the warp that completes a tile's last block takes the max over actions from the
// tile's R rows and releases the tile.
// Sweeps are launched as programmatic dependents of the previous sweep: a CTA that starts
// while the previous grid drains stages its first tiles (the slab never changes), then
// waits for that grid (griddepcontrol.wait) before it reads V or the loop's control
// block; if the loop has ended by then it drains its copies and returns.
//
// k_sell (direct): one warp per slice straight from global memory, for comparison and
// as the fallback when no tile fits in shared memory.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "vc_internal.cuh"
#include "vc_ptx.cuh"

namespace vc {

constexpr int kSellC = 32;
constexpr int kSellSigma = 4096;
constexpr int kSellBatch = 16;  // gathers per batch of a row longer than kSellLast
constexpr int kSellLast = 24;   // rows (and remainders) up to this length: one batch
constexpr int kSellMaxA = 31;  // hdr holds A + 1 row offsets in 32 slots

__host__ __device__ inline long long round128(long long x) { return (x + 127) & ~127LL; }

// Byte offsets inside a slice record with `rows` rows of 32 entries.
struct RecLayout {
    int R, scale, col;
    long long val, bytes;
};

__host__ __device__ inline RecLayout rec_layout(int A, long long rows, int vt, bool has_scale) {
    RecLayout L;
    L.R = 256;
    L.scale = L.R + 128 * A;
    L.col = L.scale + (has_scale ? 128 * A : 0);
    L.val = L.col + 128LL * rows;
    L.bytes = L.val + round128(32LL * vt * rows);
    return L;
}

// ------------------------------------------------------------------------ build
__device__ __forceinline__ bool nonzero_val(float v) { return v != 0.0f; }
__device__ __forceinline__ bool nonzero_val(uint16_t b) { return (b & 0x7FFFu) != 0u; }

// Non-zero entries of stored row r (the entries the sliced layout keeps).
template <typename VT>
__device__ __forceinline__ int row_nonzeros(const int64_t* __restrict__ row_ptr, const VT* __restrict__ val,
                                            int64_t r) {
    int n = 0;
    for (int64_t j = row_ptr[r]; j < row_ptr[r + 1]; ++j) n += nonzero_val(val[j]) ? 1 : 0;
    return n;
}

// Sort key of a state: feasible-action mask (bits 32..62), 2^20 - 1 - total non-zero row
// length (bits 12..31), index inside its window (bits 0..11).  Padding states past S get ~0.
// Every row's non-zero count also goes to nzc (255: 255 or more, to be counted again),
// which the width pass reads instead of the values.
template <typename VT>
__global__ void k_sell_keys(const int64_t* __restrict__ row_ptr, const VT* __restrict__ val,
                            const float* __restrict__ R, int S, int A, int64_t n_pad, uint64_t* __restrict__ keys,
                            unsigned char* __restrict__ nzc) {
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
            int n = 0;
            if (R[r] != -INFINITY) {
                mask |= 1u << (a < 30 ? a : 30);
                n = row_nonzeros(row_ptr, val, r);
                tot += n;
            }
            nzc[r] = (unsigned char)(n < 255 ? n : 255);
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

// Warp per slice: width(g, a) = longest feasible row (non-zero entries, from nzc) among
// the slice's lanes; the record size of the slice in units of 128 bytes; the slice's rows
// added to stats[0].
template <typename VT>
__global__ void k_sell_width(const int64_t* __restrict__ row_ptr, const VT* __restrict__ val,
                             const float* __restrict__ R, const unsigned char* __restrict__ nzc,
                             const int32_t* __restrict__ perm, int A, int64_t G, int vt, int has_scale,
                             int32_t* __restrict__ width, int32_t* __restrict__ rec_units,
                             unsigned long long* __restrict__ stats) {
    __shared__ unsigned long long s_rows;
    if (threadIdx.x == 0) s_rows = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long warp_rows = 0;
    for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {
        const int s = perm[g * kSellC + lane];
        long long rows = 0;
        for (int a = 0; a < A; ++a) {
            int len = 0;
            if (s >= 0) {
                const int64_t r = (int64_t)s * A + a;
                if (R[r] != -INFINITY) {
                    len = nzc[r];
                    if (len == 255) len = row_nonzeros(row_ptr, val, r);
                }
            }
            const int w = __reduce_max_sync(0xffffffffu, len);
            if (lane == 0) width[g * A + a] = w;
            rows += w;
        }
        if (lane == 0) rec_units[g] = (int32_t)(rec_layout(A, rows, vt, has_scale != 0).bytes / 128);
        warp_rows += (unsigned long long)rows;
    }
    // the rows of the block's slices, one global atomic per block
    if (lane == 0) atomicAdd(&s_rows, warp_rows);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&stats[0], s_rows);
}

// Largest tile of TS = 1, 2 and 4 consecutive slice records, in bytes, from the record
// offsets (units of 128 bytes): stats[1..3] (the pipelined sweep's ring must hold it).
__global__ void k_sell_tile_max(const int64_t* __restrict__ rec, int64_t G, unsigned long long* __restrict__ stats) {
    // a tile of at most 4 records of at most 2^31 / 4 bytes each: 32-bit maxima per warp
    unsigned int m1 = 0, m2 = 0, m4 = 0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r0 = rec[g];
        // bytes of the tiles starting here, clamped to 32 bits (no ring holds 4 GB)
        auto bytes = [&](int64_t g1) {
            const long long b = (rec[g1 < G ? g1 : G] - r0) * 128LL;
            return (unsigned int)(b < 0xFFFFFFFFLL ? b : 0xFFFFFFFFLL);
        };
        m1 = max(m1, bytes(g + 1));
        if ((g & 1) == 0) m2 = max(m2, bytes(g + 2));
        if ((g & 3) == 0) m4 = max(m4, bytes(g + 4));
    }
    m1 = __reduce_max_sync(0xffffffffu, m1);
    m2 = __reduce_max_sync(0xffffffffu, m2);
    m4 = __reduce_max_sync(0xffffffffu, m4);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&stats[1], (unsigned long long)m1);
        atomicMax(&stats[2], (unsigned long long)m2);
        atomicMax(&stats[3], (unsigned long long)m4);
    }
}

// Warp per slice: write the slice's record (header, state map, R / scale, rows padded).
template <typename VT>
__global__ void k_sell_fill(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const VT* __restrict__ val, const float* __restrict__ R, const float* __restrict__ scale,
                            const int32_t* __restrict__ perm, const int32_t* __restrict__ width, int A, int64_t G,
                            const int64_t* __restrict__ rec_units, unsigned char* __restrict__ slab) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool has_scale = scale != nullptr;
    for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {
        unsigned char* rec = slab + rec_units[g] * 128;
        const int s = perm[g * kSellC + lane];
        // header: exclusive prefix of the block widths (lane a < A holds width a)
        const int wl = (lane < A) ? width[g * A + lane] : 0;
        int incl = wl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int rows = __shfl_sync(0xffffffffu, incl, 31);
        int32_t* hdr = reinterpret_cast<int32_t*>(rec);
        hdr[lane] = (lane < A) ? incl - wl : (lane == A ? rows : 0);
        reinterpret_cast<int32_t*>(rec + 128)[lane] = s;
        const RecLayout L = rec_layout(A, rows, (int)sizeof(VT), has_scale);
        float* Rr = reinterpret_cast<float*>(rec + L.R);
        float* Sr = reinterpret_cast<float*>(rec + L.scale);
        int32_t* cr = reinterpret_cast<int32_t*>(rec + L.col);
        VT* vr = reinterpret_cast<VT*>(rec + L.val);
        int row0 = 0;
        for (int a = 0; a < A; ++a) {
            const int w = __shfl_sync(0xffffffffu, wl, a);
            int64_t lo = 0, hi = 0;
            float rr = -INFINITY, sc = 1.0f;
            if (s >= 0) {
                const int64_t r = (int64_t)s * A + a;
                rr = R[r];
                if (has_scale) sc = scale[r];
                if (rr != -INFINITY) {
                    lo = row_ptr[r];
                    hi = row_ptr[r + 1];
                }
            }
            // the row's non-zero entries in column order, then padding
            int j = 0;
            for (int64_t k = lo; k < hi; ++k) {
                const VT v = val[k];
                if (!nonzero_val(v)) continue;
                const int64_t e = (int64_t)(row0 + j) * kSellC + lane;
                cr[e] = col[k];
                vr[e] = v;
                ++j;
            }
            for (; j < w; ++j) {
                const int64_t e = (int64_t)(row0 + j) * kSellC + lane;
                cr[e] = s >= 0 ? s : 0;
                vr[e] = VT(0);
            }
            Rr[a * kSellC + lane] = rr;
            if (has_scale) Sr[a * kSellC + lane] = sc;
            row0 += w;
        }
        // zero the alignment tail of the value region (BF16 blocks of odd row count)
        const long long vbytes = 32LL * (int)sizeof(VT) * rows;
        for (long long b = vbytes + lane * 4; b < L.bytes - L.val; b += 128)
            *reinterpret_cast<uint32_t*>(rec + L.val + b) = 0u;
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
    if (m->sell_slab) return VC_OK;  // already built
    const bool bf16 = base == VC_CSR_BF16;
    const int vt = bf16 ? 2 : 4;
    const int A = m->A;
    const int64_t S = m->S;
    const int64_t n_pad = (S + kSellSigma - 1) / kSellSigma * kSellSigma;
    const int64_t G = (S + kSellC - 1) / kSellC;
    int rc;
    // temporaries, one allocation (freed below): keys, state map, widths, record sizes,
    // per-row non-zero counts, and the statistics read back at the end
    const size_t o_keys = 0, o_perm = o_keys + 8 * (size_t)n_pad, o_width = o_perm + 4 * (size_t)n_pad;
    const size_t o_units = o_width + ((4 * (size_t)(G * A + 1) + 255) & ~(size_t)255);
    const size_t o_nzc = o_units + ((4 * (size_t)(G + 1) + 255) & ~(size_t)255);
    const size_t o_stats = o_nzc + (((size_t)S * A + 255) & ~(size_t)255);
    const size_t tmp_bytes = o_stats + 64;
    unsigned char* tmp = nullptr;
    cudaError_t e = cudaMalloc((void**)&tmp, tmp_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(sliced layout temporaries)");
    auto cleanup = [&]() { cudaFree(tmp); };
    uint64_t* keys = reinterpret_cast<uint64_t*>(tmp + o_keys);
    int32_t* perm = reinterpret_cast<int32_t*>(tmp + o_perm);
    int32_t* width = reinterpret_cast<int32_t*>(tmp + o_width);
    int32_t* units = reinterpret_cast<int32_t*>(tmp + o_units);
    unsigned char* nzc = tmp + o_nzc;
    unsigned long long* stats = reinterpret_cast<unsigned long long*>(tmp + o_stats);  // rows, max tiles (1, 2, 4)
    if ((e = cudaMemsetAsync(stats, 0, 64, st)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "sliced layout: statistics reset");
    }
    if ((rc = alloc_dev(m, (void**)&m->sell_rec, 8 * (size_t)(G + 2)))) {
        cleanup();
        return rc;
    }
    count_launches(3);
    if (bf16)
        k_sell_keys<uint16_t><<<warp_grid(n_pad / 32 + 1, m->num_sms), kThreads, 0, st>>>(
            m->row_ptr, (const uint16_t*)m->val, m->R, (int)S, A, n_pad, keys, nzc);
    else
        k_sell_keys<float><<<warp_grid(n_pad / 32 + 1, m->num_sms), kThreads, 0, st>>>(
            m->row_ptr, (const float*)m->val, m->R, (int)S, A, n_pad, keys, nzc);
    k_sell_sort<<<(unsigned)(n_pad / kSellSigma), 1024, 0, st>>>(keys, perm);
    if (bf16)
        k_sell_width<uint16_t><<<warp_grid(G, m->num_sms), kThreads, 0, st>>>(
            m->row_ptr, (const uint16_t*)m->val, m->R, nzc, perm, A, G, vt, 1, width, units, stats);
    else
        k_sell_width<float><<<warp_grid(G, m->num_sms), kThreads, 0, st>>>(
            m->row_ptr, (const float*)m->val, m->R, nzc, perm, A, G, vt, 0, width, units, stats);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "sliced layout: key / sort / width kernels");
    }
    if ((rc = exclusive_scan(m, units, G, m->sell_rec, st))) {
        cleanup();
        return rc;
    }
    int64_t total_units = 0;
    e = cudaMemcpyAsync(&total_units, m->sell_rec + G, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "sliced layout: size read-back");
    }
    m->sell_slices = G;
    m->sell_bytes = total_units * 128;
    if ((rc = alloc_dev(m, (void**)&m->sell_slab, (size_t)m->sell_bytes + 128))) {
        cleanup();
        return rc;
    }
    count_launches(2);
    if (bf16)
        k_sell_fill<uint16_t><<<warp_grid(G, m->num_sms), kThreads, 0, st>>>(
            m->row_ptr, m->col, (const uint16_t*)m->val, m->R, m->scale, perm, width, A, G, m->sell_rec,
            m->sell_slab);
    else
        k_sell_fill<float><<<warp_grid(G, m->num_sms), kThreads, 0, st>>>(
            m->row_ptr, m->col, (const float*)m->val, m->R, nullptr, perm, width, A, G, m->sell_rec, m->sell_slab);
    k_sell_tile_max<<<(unsigned)std::min<int64_t>((G + kThreads - 1) / kThreads, (int64_t)m->num_sms * 4), kThreads,
                      0, st>>>(m->sell_rec, G, stats);
    e = cudaGetLastError();
    // the rows of the copy and its largest tiles, for the entry count and the planner
    unsigned long long sh[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(sh, stats, sizeof(sh), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "sliced layout: fill");
    m->nnz_sliced = (int64_t)sh[0] * kSellC;
    for (int k = 0; k < 3; ++k) m->sell_max_tile[k] = (int64_t)sh[k + 1];
    return VC_OK;
}

// Algorithmic bytes of one sweep of the sliced copy: the slab, the record offsets, V in
// and out.
int64_t sell_sweep_bytes(const Mdp* m) { return m->sell_bytes + 8 * (m->sell_slices + 1) + 8 * (int64_t)m->S; }

// ------------------------------------------------------------------------ sweeps
struct SellArgs {
    int64_t G;
    int S;
    int A;
    float gamma;
    bool has_scale;
    const int64_t* rec;         // [G + 1] record offsets in units of 128 bytes
    const unsigned char* slab;
    const float* V_in;
    float* V_out;
    int32_t* pi;
    float* qgap;
};

template <typename VT>
__device__ __forceinline__ float ld_val(const VT* p);
template <>
__device__ __forceinline__ float ld_val<float>(const float* p) {
    return *p;
}
template <>
__device__ __forceinline__ float ld_val<uint16_t>(const uint16_t* p) {
    return __uint_as_float((uint32_t)*p << 16);
}

// W consecutive entries of a lane's row: all loads and gathers first, then the fused
// multiply-adds in column order onto acc.  SL: entries whose column is the lane's own
// state `self` add their value to pss and nothing to acc (fmaf with a zero operand leaves
// acc unchanged), so acc is the sum over the other successors, still in column order.
template <typename VT, int W, bool SL>
__device__ __forceinline__ float dot_fixed(const int32_t* cp, const VT* vp, const float* __restrict__ V, float acc,
                                           int self, float& pss) {
    float gv[W];
    uint32_t own = 0;
#pragma unroll
    for (int u = 0; u < W; ++u) {
        const int c = cp[u * kSellC];
        if (SL) {
            // an own-state entry is not gathered: it enters through pss
            const bool o = c == self;
            own |= (o ? 1u : 0u) << u;
            gv[u] = o ? 0.0f : __ldg(V + c);
        } else {
            gv[u] = __ldg(V + c);
        }
    }
    // the values are read from shared memory only once the gathers are in flight, so
    // they hold no registers meanwhile.  SL: the own-state entries' values are added to
    // pss in column order in the same pass, fmaf(v, 1, pss) = pss + v for them and
    // fmaf(v, 0, pss) = pss for the others (v >= 0), so pss is the plain column-order sum
#pragma unroll
    for (int u = 0; u < W; ++u) {
        const float v = ld_val<VT>(vp + u * kSellC);
        acc = fmaf(v, gv[u], acc);
        if (SL) pss = fmaf(v, ((own >> u) & 1u) ? 1.0f : 0.0f, pss);
    }
    return acc;
}

// Row sum of w entries in column order: rows of up to kSellLast entries in one exactly
// sized batch (every gather of the row in flight at once), longer rows in batches of 16
// until the rest fits one batch (no predicated slots).
template <typename VT, bool SL>
__device__ __forceinline__ float row_dot(const int32_t* cp, const VT* vp, int w, const float* __restrict__ V, int self,
                                         float& pss) {
    float acc = 0.0f;
    for (; w > kSellLast; w -= kSellBatch, cp += kSellBatch * kSellC, vp += kSellBatch * kSellC)
        acc = dot_fixed<VT, kSellBatch, SL>(cp, vp, V, acc, self, pss);
    switch (w) {
#define VC_DOT_CASE(n) \
    case n: return dot_fixed<VT, n, SL>(cp, vp, V, acc, self, pss);
        VC_DOT_CASE(1) VC_DOT_CASE(2) VC_DOT_CASE(3) VC_DOT_CASE(4) VC_DOT_CASE(5) VC_DOT_CASE(6) VC_DOT_CASE(7)
        VC_DOT_CASE(8) VC_DOT_CASE(9) VC_DOT_CASE(10) VC_DOT_CASE(11) VC_DOT_CASE(12) VC_DOT_CASE(13)
        VC_DOT_CASE(14) VC_DOT_CASE(15) VC_DOT_CASE(16) VC_DOT_CASE(17) VC_DOT_CASE(18) VC_DOT_CASE(19)
        VC_DOT_CASE(20) VC_DOT_CASE(21) VC_DOT_CASE(22) VC_DOT_CASE(23) VC_DOT_CASE(24)
#undef VC_DOT_CASE
        default: return acc;
    }
}
static_assert(kSellLast >= kSellBatch, "a remainder must fit one batch");

// Q value of lane `lane` in block `a` of a slice record (shared or global memory):
// R + gamma (scale) sum_j val_j V[col_j], the sum in column order; SL: the same row with
// its self-transition solved (q_self_loop).
template <typename VT, bool SL>
__device__ __forceinline__ float block_q(const unsigned char* rec, int A, int a, int lane, float gamma, bool has_scale,
                                         const float* __restrict__ V, int S, Ctl* ctl) {
    const int32_t* hdr = reinterpret_cast<const int32_t*>(rec);
    const float rr = reinterpret_cast<const float*>(rec + 256)[a * kSellC + lane];
    if (rr == -INFINITY) return -INFINITY;
    const int rows = hdr[A];
    const RecLayout L = rec_layout(A, rows, (int)sizeof(VT), has_scale);
    const int r0 = hdr[a], w = hdr[a + 1] - r0;
    const int32_t* cp = reinterpret_cast<const int32_t*>(rec + L.col) + r0 * kSellC + lane;
    const VT* vp = reinterpret_cast<const VT*>(rec + L.val) + r0 * kSellC + lane;
#ifdef VC_DEBUG_BOUNDS
    if (!VC_IN_BOUNDS(ctl, r0 >= 0 && w >= 0 && hdr[a + 1] <= rows)) return -INFINITY;
    for (int j = 0; j < w; ++j)
        if (!VC_IN_BOUNDS(ctl, cp[j * kSellC] >= 0 && cp[j * kSellC] < S)) return -INFINITY;
#else
    (void)S;
    (void)ctl;
#endif
    float pss = 0.0f;
    const int self = SL ? reinterpret_cast<const int32_t*>(rec + 128)[lane] : -1;
    const float acc = row_dot<VT, SL>(cp, vp, w, V, self, pss);
    const float sc = has_scale ? reinterpret_cast<const float*>(rec + L.scale)[a * kSellC + lane] : 1.0f;
    if (SL) {
        const float off = has_scale ? sc * acc : acc, ps = has_scale ? sc * pss : pss;
        // no self-transition (every placement row of the model): q_self_loop's denominator
        // is exactly 1 and its quotient the numerator, so the division is skipped
        if (ps == 0.0f) return fmaf(gamma, off, rr);
        return q_self_loop(rr, gamma, off, ps);
    }
    return rr + gamma * (has_scale ? sc * acc : acc);
}

// Max over actions in order (lowest maximising index; a tie counts as the second best).
__device__ __forceinline__ void top2_step(int act, float q, float& b1, float& b2, int& ia) {
    if (act == 0 || q > b1) {
        b2 = (act == 0) ? -INFINITY : b1;
        b1 = q;
        ia = act;
    } else {
        b2 = fmaxf(b2, q);
    }
}

__device__ __forceinline__ void write_state(const SellArgs& a, int s, float b1, float b2, int ia, float& res,
                                            float& vabs, Ctl* ctl) {
    if (s < 0 || !VC_IN_BOUNDS(ctl, s < a.S)) return;
    if (a.V_out) a.V_out[s] = b1;
    if (a.pi) a.pi[s] = ia;
    if (a.qgap) a.qgap[s] = (b2 == -INFINITY) ? INFINITY : b1 - b2;
    res = fmaxf(res, fabsf(b1 - __ldg(a.V_in + s)));
    vabs = fmaxf(vabs, fabsf(b1));
}

// Direct: one warp per slice, the record read from global memory.
template <typename VT, bool SL>
__global__ void __launch_bounds__(kThreads) k_sell(SellArgs a, SweepCtl sc) {
    if (loop_done(sc)) return;
    const long long sweep = loop_sweep(sc);
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * kThreads) >> 5;
    float res = 0.0f, vabs = 0.0f;
    for (int64_t g = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5; g < a.G; g += nw) {
        const unsigned char* rec = a.slab + a.rec[g] * 128;
        float b1 = -INFINITY, b2 = -INFINITY;
        int ia = 0;
        for (int act = 0; act < a.A; ++act)
            top2_step(act, block_q<VT, SL>(rec, a.A, act, lane, a.gamma, a.has_scale, a.V_in, a.S, sc.ctl), b1, b2, ia);
        write_state(a, reinterpret_cast<const int32_t*>(rec + 128)[lane], b1, b2, ia, res, vabs, sc.ctl);
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
constexpr int kMaxTS = 4;       // most slices per tile (the planner's tile sizes are 1, 2, 4)
static_assert(kSlots * (8 + 8 + 4 + 4) <= 384 && 384 + 8 * kSlots <= kHead, "slot words exceed the header");

struct SellRingArgs {
    FastDiv div_nb;   // division by TS * A (blocks per full tile)
    FastDiv div_A;    // division by A
    int TS;           // slices per tile (the last tile may hold fewer)
    int64_t ntiles;
    int ring;         // bytes of the tile ring
    int roff;         // byte offset of the ring (Q values live in the tiles' own R rows)
};

// MB = 1: up to 800 threads (24 consumer warps), 80 registers; MB = 2: two CTAs of up to
// 17 warps per SM, 60 registers.
template <typename VT, int MB, bool SL>
__global__ void __launch_bounds__(MB == 1 ? (kMaxRW + 1) * 32 : 17 * 32, MB) k_sell_ring(SellArgs a, SellRingArgs t,
                                                                                        SweepCtl sc) {
    extern __shared__ __align__(128) unsigned char smem[];
    // the next sweep may be scheduled now: it stages its first tiles (the slab does not
    // change) and waits for this grid before it reads V or the control block
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    long long sweep = 0;
    const long long lim = wait_limit(sc);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kSlots;
    int* done_cnt = reinterpret_cast<int*>(empty + kSlots);
    uint32_t* slot_pos = reinterpret_cast<uint32_t*>(done_cnt + kSlots);
    unsigned long long* slot_end = reinterpret_cast<unsigned long long*>(smem + 384);
    unsigned char* ring = smem + t.roff;
    __shared__ int s_fail, s_consumed, s_next, s_abort;
    __shared__ long long s_bounds[2][32];
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
        s_next = 0;
        s_abort = 0;
    }
    __syncthreads();
    float res = 0.0f, vabs = 0.0f;
    int issued = 0;
    if (warp == nrw) {
        // ---------------- producer: the warp loads the record bounds of its next 32 tiles
        // at once, then lane 0 places each tile in the ring and issues its one bulk copy
        const uint64_t pol = l2_evict_first();
        unsigned long long head = 0, rel = 0;  // monotonic ring bytes: allocated / free below
        int oldest = 0;                         // oldest tile not yet released
        int i = 0;
        int failed = 0;
        bool pre = true;  // before the wait for the previous grid (only tiles, no V read)
        for (int64_t c0 = blockIdx.x; c0 < t.ntiles && !failed; c0 += 32LL * gridDim.x) {
            const int64_t tk = c0 + (int64_t)lane * gridDim.x;
            if (tk < t.ntiles) {
                const int64_t g0 = tk * t.TS;
                const int64_t g1 = (g0 + t.TS < a.G) ? g0 + t.TS : a.G;
                s_bounds[0][lane] = a.rec[g0];
                s_bounds[1][lane] = a.rec[g1];
            }
            __syncwarp();
            if (lane == 0) {
                for (int k = 0; k < 32; ++k, ++i) {
                    const int64_t tile = c0 + (int64_t)k * gridDim.x;
                    if (tile >= t.ntiles) break;
                    const int64_t u0 = s_bounds[0][k];
                    const unsigned long long bytes = (unsigned long long)(s_bounds[1][k] - u0) * 128ull;
                    unsigned long long pos = head % (unsigned long long)t.ring;
                    if (pos + bytes > (unsigned long long)t.ring) {
                        head += (unsigned long long)t.ring - pos;  // skip the ring's tail
                        pos = 0;
                    }
                    if (!VC_IN_BOUNDS(sc.ctl, bytes <= (unsigned long long)t.ring)) {
                        failed = 1;
                        atomicExch(&s_fail, 1);
                        break;
                    }
                    // the first time the ring is full: wait for the previous grid, and stop
                    // if the loop has ended
                    if (pre && oldest < i && (head + bytes - rel > (unsigned long long)t.ring || i - oldest >= kSlots)) {
                        pre = false;
                        asm volatile("griddepcontrol.wait;" ::: "memory");
                        if (loop_done(sc)) {
                            atomicExch(&s_abort, 1);
                            failed = 1;
                            break;
                        }
                    }
                    // reuse bytes (and the slot) only after the tiles holding them are released
                    while (oldest < i && (head + bytes - rel > (unsigned long long)t.ring || i - oldest >= kSlots)) {
                        const int os = oldest % kSlots;
                        if (!mbar_wait(&empty[os], (uint32_t)((oldest / kSlots) & 1), lim)) {
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
                    slot_end[s] = head + bytes;
                    slot_pos[s] = (uint32_t)pos;
                    head += bytes;
                    mbar_arrive_expect_tx(&full[s], (uint32_t)bytes);
                    bulk_g2s(ring + pos, a.slab + u0 * 128, (uint32_t)bytes, &full[s], pol);
                    issued = i + 1;
                }
            }
            failed = __shfl_sync(0xffffffffu, failed, 0);
            __syncwarp();
        }
        if (lane == 0 && pre) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            if (loop_done(sc)) atomicExch(&s_abort, 1);
        }
    } else {
        // ---------------- consumers: every warp takes the CTA's next unclaimed block (a
        // shared counter over the blocks of the CTA's tile sequence), so blocks finish
        // roughly in tile order and the ring is released in order without waiting on a
        // slow warp's backlog.  The planner keeps nrw <= (kSlots - 2) blocks-per-tile
        // multiples, so claimed blocks never run kSlots tiles ahead of the oldest one.
        const int64_t nt_cta = (blockIdx.x < t.ntiles) ? (t.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
        int i = 0;
        asm volatile("griddepcontrol.wait;" ::: "memory");
        const bool ended = loop_done(sc);
        sweep = loop_sweep(sc);
        while (!ended) {
            int gb = 0;
            if (lane == 0) gb = atomicAdd(&s_next, 1);
            gb = __shfl_sync(0xffffffffu, gb, 0);
            i = (int)fdiv((uint32_t)gb, t.div_nb);
            const int b = gb - i * nb_full;
            if (i >= nt_cta) break;
            const int64_t tile = blockIdx.x + (int64_t)i * gridDim.x;
            const int64_t g0 = tile * t.TS;
            const int ns = (int)(((g0 + t.TS < a.G) ? g0 + t.TS : a.G) - g0);
            const int nb = ns * A;
            if (b >= nb) continue;  // the last tile may hold fewer slices
            const int s = i % kSlots;
            if (!mbar_wait(&full[s], (uint32_t)((i / kSlots) & 1), lim)) {
                atomicExch(&s_fail, 1);
                break;
            }
            unsigned char* base = ring + *((volatile uint32_t*)&slot_pos[s]);
            const int sl = (int)fdiv((uint32_t)b, t.div_A), act = b - sl * A;
            long long roff = 0;
            for (int k = 0; k < sl; ++k)
                roff += rec_layout(A, reinterpret_cast<const int32_t*>(base + roff)[A], (int)sizeof(VT), a.has_scale)
                            .bytes;
#ifdef VC_DEBUG_BOUNDS
            {
                const long long tile_bytes = (a.rec[(tile * t.TS + ns)] - a.rec[tile * t.TS]) * 128;
                const long long rb =
                    rec_layout(A, reinterpret_cast<const int32_t*>(base + roff)[A], (int)sizeof(VT), a.has_scale).bytes;
                if (!VC_IN_BOUNDS(sc.ctl, roff + rb <= tile_bytes)) roff = 0;
            }
#endif
            const float qv = block_q<VT, SL>(base + roff, A, act, lane, a.gamma, a.has_scale, a.V_in, a.S, sc.ctl);
            // the Q value replaces the block's own R entry in the ring (read above, by this lane
            // only); the proxy fence orders the write before the tile's next bulk copy
            reinterpret_cast<float*>(base + roff + 256)[act * kSellC + lane] = qv;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __threadfence_block();
            __syncwarp();
            int l = 0;
            if (lane == 0) l = (atomicAdd(&done_cnt[s], 1) == nb - 1);
            if (__shfl_sync(0xffffffffu, l, 0)) {
                // the tile's last block: the max over actions and the state map come out
                // of shared memory first, the tile is released, and only then the state
                // writes and the residual's read of V_in (global memory) follow, so the
                // ring slot is not held over a global-memory round trip
                __threadfence_block();
                float b1v[kMaxTS], b2v[kMaxTS];
                int iav[kMaxTS], sv[kMaxTS];
                long long ro = 0;
#pragma unroll
                for (int k = 0; k < kMaxTS; ++k) {
                    sv[k] = -1;
                    if (k < ns) {
                        const unsigned char* rec = base + ro;
                        float b1 = -INFINITY, b2 = -INFINITY;
                        int ia = 0;
                        const float* qrow = reinterpret_cast<const float*>(rec + 256);
                        for (int c = 0; c < A; ++c) top2_step(c, qrow[c * kSellC + lane], b1, b2, ia);
                        b1v[k] = b1;
                        b2v[k] = b2;
                        iav[k] = ia;
                        sv[k] = reinterpret_cast<const int32_t*>(rec + 128)[lane];
                        ro += rec_layout(A, reinterpret_cast<const int32_t*>(rec)[A], (int)sizeof(VT), a.has_scale).bytes;
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    done_cnt[s] = 0;
                    __threadfence_block();
                    mbar_arrive(&empty[s]);
                }
#pragma unroll
                for (int k = 0; k < kMaxTS; ++k)
                    if (k < ns) write_state(a, sv[k], b1v[k], b2v[k], iav[k], res, vabs, sc.ctl);
            }
        }
        if (lane == 0) atomicMin(&s_consumed, i);
    }
    __syncthreads();
    if (s_fail || s_abort) {
        // drain this CTA's copies still in flight before shared memory is released
        if (warp == nrw && lane == 0) {
            for (int j = (s_consumed < issued ? s_consumed : issued); j < issued; ++j)
                mbar_wait(&full[j % kSlots], (uint32_t)((j / kSlots) & 1));
            if (s_fail) atomicOr(&sc.ctl->error, kErrTimeout);
        }
    }
    if (s_abort || sc.mode == kModeNone) return;
    res = block_max_dyn(res);
    vabs = block_max_dyn(vabs);
    finish_block<float>(sc, res, vabs, sweep);
}

static const void* ring_fn(bool bf16, int mb, bool sl) {
    if (bf16) {
        if (mb == 2) return sl ? (const void*)k_sell_ring<uint16_t, 2, true> : (const void*)k_sell_ring<uint16_t, 2, false>;
        return sl ? (const void*)k_sell_ring<uint16_t, 1, true> : (const void*)k_sell_ring<uint16_t, 1, false>;
    }
    if (mb == 2) return sl ? (const void*)k_sell_ring<float, 2, true> : (const void*)k_sell_ring<float, 2, false>;
    return sl ? (const void*)k_sell_ring<float, 1, true> : (const void*)k_sell_ring<float, 1, false>;
}

// Candidate launch shapes of the ring sweep, in preference order: (CTAs per SM, consumer
// warps per CTA) x slices per tile; the ring takes the shared memory left after the
// header and must hold the largest tile.  A shape must fit both instantiations (Eq. 18's
// backup and the self-transition solve), since one plan serves both.
int sell_plans(Mdp* m, cudaStream_t st, std::vector<CsrPlan>& out) {
    (void)st;
    out.clear();
    if (!m->sell_slab) return VC_OK;
    const bool bf16 = (m->fmt & 0xF) == VC_CSR_BF16;
    const int A = m->A;
    int dev = 0, smem_sm = 0, smem_blk = 0;
    VC_CUDA(cudaGetDevice(&dev));
    VC_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    VC_CUDA(cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));

    // (CTAs per SM, consumer warps, register budget), preferred first
    const int shapes[][3] = {{2, 12, 1}, {2, 16, 2}, {3, 10, 2}, {1, 24, 1}, {2, 8, 1}, {3, 8, 1}};
    for (int TS : {1, 2, 4}) {
        static_assert(kMaxTS >= 4, "the last block's registers cover every planned tile size");
        const long long max_tile = m->sell_max_tile[TS == 1 ? 0 : (TS == 2 ? 1 : 2)];  // largest tile of TS records
        for (auto& sh : shapes) {
            const int ctas = sh[0], nrw = sh[1], mb = sh[2];
            const void* fn = ring_fn(bf16, mb, false);
            const void* fn_sl = ring_fn(bf16, mb, true);
            cudaFuncAttributes fa, fa_sl;
            VC_CUDA(cached_func_attributes(fn, &fa));
            VC_CUDA(cached_func_attributes(fn_sl, &fa_sl));
            fa.numRegs = std::max(fa.numRegs, fa_sl.numRegs);
            fa.sharedSizeBytes = std::max(fa.sharedSizeBytes, fa_sl.sharedSizeBytes);
            fa.maxThreadsPerBlock = std::min(fa.maxThreadsPerBlock, fa_sl.maxThreadsPerBlock);
            const int dyn_max = smem_blk - (int)fa.sharedSizeBytes;
            VC_CUDA(cached_set_max_dyn_smem(fn, dyn_max));
            VC_CUDA(cached_set_max_dyn_smem(fn_sl, dyn_max));
            const int threads = (nrw + 1) * 32;
            if (threads > fa.maxThreadsPerBlock || (long long)threads * fa.numRegs * ctas > 65536) continue;
            if (nrw > (kSlots - 2) * TS * A) continue;  // claimed blocks stay within kSlots tiles
            // the ring follows the header; Q values live in the tiles' own R rows
            const int budget = std::min(dyn_max, (smem_sm - 1024 * ctas) / ctas - (int)fa.sharedSizeBytes);
            const int ring = ((budget - kHead) / 128) * 128;
            if (ring < max_tile + 128) continue;
            const int need = kHead + ring;
            int per_sm = 0;
            int per_sm_sl = 0;
            VC_CUDA(cached_occupancy(fn, threads, (size_t)need, &per_sm));
            VC_CUDA(cached_occupancy(fn_sl, threads, (size_t)need, &per_sm_sl));
            per_sm = std::min(per_sm, per_sm_sl);
            if (per_sm < 1) continue;
            CsrPlan P;
            P.sliced = true;
            P.tma = true;
            P.ts = TS;
            P.cap = ring;
            P.stages = kSlots;
            P.warps = nrw;
            P.minb = mb;
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
    a.S = m->S;
    a.A = m->A;
    a.gamma = (float)m->gamma;
    a.has_scale = (m->fmt & 0xF) == VC_CSR_BF16;
    a.rec = m->sell_rec;
    a.slab = m->sell_slab;
    a.V_in = V_in;
    a.V_out = V_out;
    a.pi = pi;
    a.qgap = qgap;
    const bool bf16 = a.has_scale;
    if (m->plan.tma) {
        SellRingArgs t;
        t.div_nb = make_fastdiv((uint32_t)(m->plan.ts * m->A));
        t.div_A = make_fastdiv((uint32_t)m->A);
        t.TS = m->plan.ts;
        t.ntiles = m->plan.ntiles;
        t.ring = (int)m->plan.cap;
        t.roff = kHead;
        const long long cap = (long long)m->num_sms * m->plan.ctas_per_sm;
        const unsigned grid = (unsigned)(t.ntiles < cap ? t.ntiles : cap);
        const unsigned threads = (unsigned)(m->plan.warps + 1) * 32;
        count_launches(1);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = (size_t)m->plan.smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        void* args[] = {&a, &t, &sc};
        VC_CUDA(cudaLaunchKernelExC(&cfg, ring_fn(bf16, m->plan.minb, sc.self_loop != 0), args));
        return VC_OK;
    }
    const int bps = m->plan.ctas_per_sm > 0 ? m->plan.ctas_per_sm : 4;
    const int64_t want = (a.G * kSellC + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)m->num_sms * bps;
    const unsigned grid = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
    count_launches(1);
    if (bf16 && sc.self_loop)
        k_sell<uint16_t, true><<<grid, kThreads, 0, st>>>(a, sc);
    else if (bf16)
        k_sell<uint16_t, false><<<grid, kThreads, 0, st>>>(a, sc);
    else if (sc.self_loop)
        k_sell<float, true><<<grid, kThreads, 0, st>>>(a, sc);
    else
        k_sell<float, false><<<grid, kThreads, 0, st>>>(a, sc);
    VC_CUDA(cudaGetLastError());
    return VC_OK;
}

}  // namespace vc
