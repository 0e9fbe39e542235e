// vc_build.cu -- instance construction: model descriptor, explicit CSR from the model
// (count -> exclusive scan -> fill), and validation of user-supplied CSR matrices.
//
// The transition structure follows the uniformised model of Section V (Eq. 10-16 under
// the library's readings): from the post-decision state x one event fires -- completion
// on host k (mu_k occ_k), departure of host k (delta_k, host emptied), arrival (lambda,
// blocked at a full queue), phase flip (f or 1-f) -- all over Lam, the rest a self-loop.
#include <cuda_bf16.h>
#include <math.h>

#include <type_traits>
#include <algorithm>
#include <vector>

#include "vc_internal.cuh"

namespace vc {

int alloc_dev(Mdp* m, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(VC_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                    cudaGetErrorString(e));
    }
    m->device_bytes += (int64_t)bytes;
    return VC_OK;
}

// ------------------------------------------------------------------- host: descriptor
int build_model(const vc_params* p, Mdp* m) {
    if (!p) return fail(VC_ERR_ARG, "params is NULL");
    const int H = p->H, C = p->C, Q = p->Q;
    if (H < 1 || H > kMaxH) return fail(VC_ERR_ARG, "H must be in 1..16");
    if (C < 1 || C > 1000) return fail(VC_ERR_ARG, "C must be in 1..1000");
    if (Q < 0 || Q > 100000) return fail(VC_ERR_ARG, "Q must be in 0..100000");
    if (!p->mu || !p->delta) return fail(VC_ERR_ARG, "mu / delta is NULL");
    if (!(p->gamma > 0.0 && p->gamma < 1.0)) return fail(VC_ERR_ARG, "gamma must be in (0, 1)");
    if (!(p->f > 0.0 && p->f < 1.0)) return fail(VC_ERR_ARG, "f must be in (0, 1)");
    if (!(p->lambda > 0.0) || !isfinite(p->lambda)) return fail(VC_ERR_ARG, "lambda must be > 0");
    if (!isfinite(p->w_occ) || !isfinite(p->w_loss) || !isfinite(p->w_q)) return fail(VC_ERR_ARG, "weights must be finite");
    double S = 2.0 * (Q + 1);
    for (int k = 0; k < H; k++) {
        if (!(p->mu[k] > 0.0) || !isfinite(p->mu[k])) return fail(VC_ERR_ARG, "mu_k must be > 0");
        if (!(p->delta[k] >= 0.0) || !isfinite(p->delta[k])) return fail(VC_ERR_ARG, "delta_k must be >= 0");
        S *= (C + 1);
    }
    if (S >= 2147483647.0) return fail(VC_ERR_ARG, "S = 2(Q+1)(C+1)^H must be < 2^31");

    Model& md = m->md;
    md.H = H;
    md.C = C;
    md.Q = Q;
    md.A = H + 1;
    md.S = (int)S;
    int64_t st = 2 * (int64_t)(Q + 1);
    for (int k = 0; k < kMaxH; k++) {
        md.stride[k] = (k < H) ? (int)st : 0;
        if (k < H) st *= (C + 1);
    }
    md.div_q = make_fastdiv((uint32_t)(Q + 1));
    md.div_c = make_fastdiv((uint32_t)(C + 1));

    Rates& r = m->rates;
    double sum_mu = 0.0, sum_delta = 0.0;
    for (int k = 0; k < kMaxH; k++) {
        r.mu[k] = (k < H) ? p->mu[k] : 0.0;
        r.delta[k] = (k < H) ? p->delta[k] : 0.0;
        sum_mu += r.mu[k];
        sum_delta += r.delta[k];
    }
    r.lambda = p->lambda;
    r.f = p->f;
    r.Lam = p->lambda + C * sum_mu + sum_delta + 1.0;
    r.w_occ = p->w_occ;
    r.w_loss = p->w_loss;
    r.w_q = p->w_q;
    for (int k = 0; k < kMaxH; k++) r.pdep[k] = r.delta[k] / r.Lam;
    r.parr = r.lambda / r.Lam;
    r.pflip[0] = r.f / r.Lam;
    r.pflip[1] = (1.0 - r.f) / r.Lam;
    r.occ_tab = nullptr;  // upload_rate_table
    r.tab_c1 = C + 1;

    Coef<double>& c = m->c64;
    c.gamma = p->gamma;
    for (int k = 0; k < kMaxH; k++) {
        c.pc[k] = r.mu[k] / r.Lam;
        c.pd[k] = r.delta[k] / r.Lam;
        c.lossd[k] = p->w_loss * r.delta[k] / r.Lam;
    }
    c.pa = p->lambda / r.Lam;
    c.lossa = p->w_loss * p->lambda / r.Lam;
    c.pf0 = p->f / r.Lam;
    c.pf1 = (1.0 - p->f) / r.Lam;
    c.w_occ = p->w_occ;
    c.w_q = p->w_q;
    Coef<float>& c32 = m->c32;
    c32.gamma = (float)c.gamma;
    for (int k = 0; k < kMaxH; k++) {
        c32.pc[k] = (float)c.pc[k];
        c32.pd[k] = (float)c.pd[k];
        c32.lossd[k] = (float)c.lossd[k];
    }
    c32.pa = (float)c.pa;
    c32.lossa = (float)c.lossa;
    c32.pf0 = (float)c.pf0;
    c32.pf1 = (float)c.pf1;
    c32.w_occ = (float)c.w_occ;
    c32.w_q = (float)c.w_q;

    m->has_model = true;
    m->S = md.S;
    m->A = md.A;
    m->gamma = p->gamma;
    return VC_OK;
}

// Round a positive finite double to bfloat16, nearest-even: first to float with
// round-to-odd (truncate, then set the last bit if anything was lost), then float to
// bf16 with nearest-even.  Rounding to odd at 24 bits before rounding to 8 bits gives
// the correctly rounded result (Boldo & Melquiond, IEEE Trans. Computers 57(4), 2008).
__device__ __forceinline__ uint16_t bf16_rne_from_double(double x) {
    float t = __double2float_rz(x);
    uint32_t u = __float_as_uint(t);
    if ((double)t != x) u |= 1u;
    const uint32_t bias = 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)((u + bias) >> 16);
}

__device__ __forceinline__ double bf16_to_double(uint16_t b) { return (double)__uint_as_float((uint32_t)b << 16); }

// ------------------------------------------------------------------------- build kernels
// The per-occupancy probabilities mu_k o / Lam and delta_k o / Lam of every host, formed
// on the host (the same FP64 operations as the device formula) and placed in device
// memory, so the row kernels read them instead of dividing in FP64.
// Also the FP32 tables of the FP32 fill (their roundings and non-zero flags), one upload.
int upload_rate_table(Mdp* m, cudaStream_t st) {
    Rates& r = m->rates;
    const int c1 = r.tab_c1;
    const size_t n64 = (size_t)2 * kMaxH * c1, n32 = (size_t)kMaxH * c1;
    const size_t bytes = 8 * n64 + 4 * n32 + n32;
    std::vector<unsigned char> buf(bytes, 0);
    double* tab = reinterpret_cast<double*>(buf.data());
    float* tab32 = reinterpret_cast<float*>(buf.data() + 8 * n64);
    unsigned char* nz = buf.data() + 8 * n64 + 4 * n32;
    for (int k = 0; k < kMaxH; k++)
        for (int o = 0; o < c1; o++) {
            const double pc = r.mu[k] * (double)o / r.Lam;
            tab[(size_t)k * c1 + o] = pc;
            tab[(size_t)(kMaxH + k) * c1 + o] = r.delta[k] * (double)o / r.Lam;
            tab32[(size_t)k * c1 + o] = (float)pc;
            nz[(size_t)k * c1 + o] = pc != 0.0 ? 1 : 0;
        }
    r.nz_pdep = r.nz_p1 = 0u;
    for (int k = 0; k < kMaxH; k++) {
        const double p1 = tab[(size_t)k * c1 + 1] + r.pdep[k];
        r.pdep32[k] = (float)r.pdep[k];
        r.p1_32[k] = (float)p1;
        if (r.pdep[k] != 0.0) r.nz_pdep |= 1u << k;
        if (p1 != 0.0) r.nz_p1 |= 1u << k;
    }
    r.parr32 = (float)r.parr;
    r.nz_parr = r.parr != 0.0;
    for (int ph = 0; ph < 2; ph++) {
        r.pflip32[ph] = (float)r.pflip[ph];
        r.nz_pflip[ph] = r.pflip[ph] != 0.0;
    }
    int rc;
    if ((rc = alloc_dev(m, (void**)&m->rate_tab, bytes))) return rc;
    VC_CUDA(cudaMemcpyAsync(m->rate_tab, buf.data(), bytes, cudaMemcpyHostToDevice, st));
    VC_CUDA(cudaStreamSynchronize(st));  // buf is pageable host memory
    r.occ_tab = m->rate_tab;
    r.occ_tab32 = reinterpret_cast<const float*>(reinterpret_cast<const unsigned char*>(m->rate_tab) + 8 * n64);
    r.occ_nz = reinterpret_cast<const unsigned char*>(m->rate_tab) + 8 * n64 + 4 * n32;
    return VC_OK;
}

// Per-row entry counts (grid-stride), with the block's tallies of feasible rows and
// logical non-zeros added once per block.
template <int MH>
__global__ void __launch_bounds__(kThreads) k_row_count(Model md, Rates rt, int64_t nrows, int32_t* cnt,
                                                        unsigned long long* tallies) {
    unsigned long long feas = 0, nz = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(r / md.A), a = (int)(r % md.A);
        double R;
        const int n = model_row_emit<MH>(md, rt, s, a, &R, [](int, int, double) {});
        if (cnt) cnt[r] = n < 0 ? 0 : n;
        if (n >= 0) {
            feas += 1;
            nz += (unsigned long long)n;
        }
    }
    block_tally<kThreads>(feas, nz, tallies);
}

// One row of the CSR fill, written as the row's entries come (ascending columns); returns
// the row's non-zero successors (-1: infeasible).
template <int MH, bool kBf16>
__device__ __forceinline__ int fill_row(const Model& md, const Rates& rt, int64_t r, int padded,
                                        const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                                        void* __restrict__ val, float* __restrict__ scale, float* __restrict__ R) {
    const int s = (int)(r / md.A), a = (int)(r % md.A);
    const int64_t base = row_ptr[r];
    const int width = 2 * md.H + 3;
    double Rv, tot = 0.0;
    int last = s;
    const int n = model_row_emit<MH>(md, rt, s, a, &Rv, [&](int j, int c, double p) {
        col[base + j] = c;
        if (kBf16) {
            const uint16_t b = bf16_rne_from_double(p);
            ((uint16_t*)val)[base + j] = b;
            tot += bf16_to_double(b);
        } else {
            ((float*)val)[base + j] = (float)p;
        }
        last = c;
    });
    if (n < 0) {
        R[r] = -INFINITY;
        if (kBf16) scale[r] = 0.0f;
        if (padded) {
            for (int j = 0; j < width; j++) {
                col[base + j] = s;
                if (kBf16)
                    ((uint16_t*)val)[base + j] = 0;
                else
                    ((float*)val)[base + j] = 0.0f;
            }
        }
        return -1;
    }
    R[r] = (float)Rv;
    if (kBf16) scale[r] = (float)(1.0 / tot);
    if (padded) {
        for (int j = n; j < width; j++) {
            col[base + j] = last;
            if (kBf16)
                ((uint16_t*)val)[base + j] = 0;
            else
                ((float*)val)[base + j] = 0.0f;
        }
    }
    return n;
}

// Fills every row (BF16 values; grid-stride); with tallies (padded rows, where no count
// pass precedes the fill) it also adds up the feasible rows and their non-zero successors,
// once per block.
template <int MH, bool kBf16>
__global__ void __launch_bounds__(kThreads) k_row_fill(Model md, Rates rt, int64_t nrows, int padded,
                                                       const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                                                       void* __restrict__ val, float* __restrict__ scale,
                                                       float* __restrict__ R, unsigned long long* tallies) {
    unsigned long long feas = 0, nz = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x) {
        const int n = fill_row<MH, kBf16>(md, rt, r, padded, row_ptr, col, val, scale, R);
        if (n >= 0) {
            feas += 1;
            nz += (unsigned long long)n;
        }
    }
    if (tallies) block_tally<kThreads>(feas, nz, tallies);
}

// model_row_emit with FP32 values, for the FP32 fill: the same successors in the same order,
// each value the FP32 rounding of model_row_emit's FP64 probability.  The per-event values
// and their non-zero tests come from the host-formed tables of Rates; only what a row sums
// (the self-loop remainder and the reward) is formed here in FP64, with model_row_emit's
// operations in its order (the occupancy sum, exact in FP64, is kept as an integer).
template <int MH, typename Emit>
__device__ __forceinline__ int model_row_emit_f32(const Model& md, const Rates& rt, int s, int a, double* R,
                                                  Emit&& emit) {
    Digits d;
    decode<MH>(md, s, d);
    int x = s;
    if (a < md.H && !apply_action<MH>(md, s, a, d, x)) return -1;
    const int c1 = rt.tab_c1;
    double total = 0.0, self_extra = 0.0, lost = 0.0;
    int occ_sum = 0;
#pragma unroll
    for (int k = 0; k < MH; k++) {
        if (k < md.H) {
            const int o = d.occ[k];
            const double pdep = rt.pdep[k];
            total += __ldg(rt.occ_tab + (size_t)k * c1 + o) + pdep;
            occ_sum += o;
            lost += __ldg(rt.occ_tab + (size_t)(kMaxH + k) * c1 + o);
            if (o == 0) self_extra += pdep;
        }
    }
    const double parr = rt.parr;
    total += parr;
    if (d.q >= md.Q) {
        self_extra += parr;
        lost += parr;
    }
    total += d.ph ? rt.pflip[1] : rt.pflip[0];
    const double pself = (1.0 - total) + self_extra;
    *R = rt.w_occ * (double)occ_sum + rt.w_q * d.q + rt.w_loss * lost;
    int n = 0;
#pragma unroll
    for (int k = MH - 1; k >= 0; k--) {
        if (k < md.H) {
            const int o = d.occ[k];
            if (o == 1) {
                if ((rt.nz_p1 >> k) & 1u) emit(n++, x - md.stride[k], rt.p1_32[k]);
            } else if (o > 1) {
                if ((rt.nz_pdep >> k) & 1u) emit(n++, x - o * md.stride[k], rt.pdep32[k]);
                if (__ldg(rt.occ_nz + (size_t)k * c1 + o)) emit(n++, x - md.stride[k], __ldg(rt.occ_tab32 + (size_t)k * c1 + o));
            }
        }
    }
    const float pflip32 = d.ph ? rt.pflip32[1] : rt.pflip32[0];
    const int nzflip = d.ph ? rt.nz_pflip[1] : rt.nz_pflip[0];
    if (d.ph) {
        if (nzflip) emit(n++, x - 1, pflip32);
        if (pself != 0.0) emit(n++, x, (float)pself);
    } else {
        if (pself != 0.0) emit(n++, x, (float)pself);
        if (nzflip) emit(n++, x + 1, pflip32);
    }
    if (d.q < md.Q && rt.nz_parr) emit(n++, x + 2, rt.parr32);
    return n;
}

// FP32 fill: a warp's 32 consecutive rows occupy one contiguous range of the CSR, so each
// lane writes its row into the warp's shared-memory stage and the warp then stores the
// range lane-consecutively (coalesced) instead of each lane striding through its own row.
constexpr int kFillThreads = 128;

template <int MH>
__global__ void __launch_bounds__(kFillThreads) k_row_fill32(Model md, Rates rt, int64_t nrows, int padded,
                                                             const int64_t* __restrict__ row_ptr,
                                                             int32_t* __restrict__ col, float* __restrict__ val,
                                                             float* __restrict__ R, unsigned long long* tallies) {
    constexpr int kW = 2 * MH + 3;  // most entries of a row
    __shared__ int32_t s_col[kFillThreads / 32][32 * kW];
    __shared__ float s_val[kFillThreads / 32][32 * kW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int width = 2 * md.H + 3;
    unsigned long long feas = 0, nz = 0;
    // grid-stride over groups of 32 rows, one group per warp and step
    for (int64_t r0 = ((int64_t)blockIdx.x * (kFillThreads / 32) + warp) * 32; r0 < nrows;
         r0 += (int64_t)gridDim.x * kFillThreads) {
        const int64_t r = r0 + lane;
        const int64_t rend = (r0 + 32 < nrows) ? r0 + 32 : nrows;
        const int64_t b0 = row_ptr[r0];
        if (r < nrows) {
            const int s = (int)(r / md.A), a = (int)(r % md.A);
            const int off = (int)(row_ptr[r] - b0);
            int32_t* cs = &s_col[warp][off];
            float* vs = &s_val[warp][off];
            double Rv;
            int last = s;
            const int n = model_row_emit_f32<MH>(md, rt, s, a, &Rv, [&](int j, int c, float p) {
                cs[j] = c;
                vs[j] = p;
                last = c;
            });
            if (n < 0) {
                R[r] = -INFINITY;
                if (padded)
                    for (int j = 0; j < width; j++) {
                        cs[j] = s;
                        vs[j] = 0.0f;
                    }
            } else {
                R[r] = (float)Rv;
                if (padded)
                    for (int j = n; j < width; j++) {
                        cs[j] = last;
                        vs[j] = 0.0f;
                    }
                feas += 1;
                nz += (unsigned long long)n;
            }
        }
        __syncwarp();
        const int nent = (int)(row_ptr[rend] - b0);
        const bool fits = nent <= 32 * kW;  // always: a row holds at most 2H + 3 entries
        for (int i = lane; fits && i < nent; i += 32) {
            col[b0 + i] = s_col[warp][i];
            val[b0 + i] = s_val[warp][i];
        }
        __syncwarp();  // the stage is rewritten by the warp's next group
    }
    if (tallies) block_tally<kFillThreads>(feas, nz, tallies);
}

__global__ void k_padded_rowptr(int64_t nrows, int width, int64_t* row_ptr) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r <= nrows) row_ptr[r] = r * width;
}

// ------------------------------------------------------------- exclusive scan (int32 -> int64)
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* total) {
    __shared__ long long warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        long long ws = (lane < kScanThreads / 32) ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += y;
        }
        if (lane < kScanThreads / 32) warp_sums[lane] = ws;
    }
    __syncthreads();
    const long long warp_off = (w > 0) ? warp_sums[w - 1] : 0;
    *total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return warp_off + x - v;
}

__global__ void k_scan_tiles(const int32_t* __restrict__ cnt, int64_t n, long long* __restrict__ tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    long long v = 0;
    for (int i = 0; i < kScanItems; i++)
        if (base + i < n) v += cnt[base + i];
    long long total;
    block_exclusive_scan(v, &total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Single block: exclusive scan of the tile sums in place, grand total to *out_total.
__global__ void k_scan_top(long long* tile_sums, int64_t ntiles, long long* out_total) {
    long long carry = 0;
    for (int64_t b0 = 0; b0 < ntiles; b0 += kScanThreads) {
        const int64_t i = b0 + threadIdx.x;
        const long long v = (i < ntiles) ? tile_sums[i] : 0;
        long long total;
        const long long ex = block_exclusive_scan(v, &total);
        if (i < ntiles) tile_sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) *out_total = carry;
}

__global__ void k_scan_apply(const int32_t* __restrict__ cnt, int64_t n, const long long* __restrict__ tile_off,
                             const long long* __restrict__ grand, int64_t* __restrict__ out) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    long long loc[kScanItems];
    long long v = 0;
    for (int i = 0; i < kScanItems; i++) {
        loc[i] = (base + i < n) ? cnt[base + i] : 0;
        v += loc[i];
    }
    long long total;
    long long run = tile_off[blockIdx.x] + block_exclusive_scan(v, &total);
    for (int i = 0; i < kScanItems; i++) {
        if (base + i < n) out[base + i] = run;
        run += loc[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = *grand;
}

// out[0..n] = exclusive prefix sums of cnt[0..n-1], out[n] = total.  Scratch: tile sums.
int exclusive_scan(Mdp* m, const int32_t* cnt, int64_t n, int64_t* out, cudaStream_t st) {
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    long long* scratch = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&scratch, sizeof(long long) * (ntiles + 1), st);
    if (e != cudaSuccess) return fail(VC_ERR_OOM, "scan scratch allocation failed");
    count_launches(3);
    k_scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, st>>>(cnt, n, scratch);
    k_scan_top<<<1, kScanThreads, 0, st>>>(scratch, ntiles, scratch + ntiles);
    k_scan_apply<<<(unsigned)ntiles, kScanThreads, 0, st>>>(cnt, n, scratch, scratch + ntiles, out);
    VC_CUDA(cudaGetLastError());
    VC_CUDA(cudaFreeAsync(scratch, st));
    (void)m;
    return VC_OK;
}

// Feasible rows and logical successor count of a model without storing anything.
// Calls f with std::integral_constant<int, MH>: MH = H for H <= 8, else 16.
template <typename F>
static void by_h_build(int H, F&& f) {
    switch (H) {
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

int count_model_rows(Mdp* m, cudaStream_t st) {
    const int64_t nrows = (int64_t)m->S * m->A;
    const unsigned grid = (unsigned)std::min<int64_t>((nrows + kThreads - 1) / kThreads, (int64_t)m->num_sms * 16);
    unsigned long long* tallies = nullptr;
    VC_CUDA(cudaMallocAsync((void**)&tallies, sizeof(unsigned long long) * 2, st));
    VC_CUDA(cudaMemsetAsync(tallies, 0, sizeof(unsigned long long) * 2, st));
    count_launches(1);
    by_h_build(m->md.H, [&](auto mh) {
        k_row_count<decltype(mh)::value><<<grid, kThreads, 0, st>>>(m->md, m->rates, nrows, nullptr, tallies);
    });
    VC_CUDA(cudaGetLastError());
    unsigned long long th[2];
    VC_CUDA(cudaMemcpyAsync(th, tallies, sizeof(th), cudaMemcpyDeviceToHost, st));
    VC_CUDA(cudaFreeAsync(tallies, st));
    VC_CUDA(cudaStreamSynchronize(st));
    m->feasible_rows = (int64_t)th[0];
    m->nnz_logical = (int64_t)th[1];
    m->nnz_stored = 0;
    return VC_OK;
}

// ------------------------------------------------------------------ CSR from the model
int build_csr_from_model(Mdp* m, cudaStream_t st) {
    const int64_t nrows = (int64_t)m->S * m->A;
    const bool padded = (m->fmt & VC_PADDED) != 0;
    const bool bf16 = (m->fmt & 0xF) == VC_CSR_BF16;
    const int width = 2 * m->md.H + 3;
    const int T = 256;
    const unsigned nb = (unsigned)((nrows + T - 1) / T);
    int rc;

    // counts: canonical rows need them for the offsets (and give the logical nnz and the
    // feasible-row tally); padded rows have fixed offsets, so the fill tallies instead
    int32_t* cnt = nullptr;
    unsigned long long* tallies = nullptr;
    unsigned long long th[2] = {0, 0};
    VC_CUDA(cudaMallocAsync((void**)&tallies, sizeof(unsigned long long) * 2, st));
    VC_CUDA(cudaMemsetAsync(tallies, 0, sizeof(unsigned long long) * 2, st));
    if (!padded) {
        VC_CUDA(cudaMallocAsync((void**)&cnt, sizeof(int32_t) * nrows, st));
        count_launches(1);
        by_h_build(m->md.H, [&](auto mh) {
            k_row_count<decltype(mh)::value><<<(unsigned)std::min<int64_t>(nb, (int64_t)m->num_sms * 16), kThreads, 0,
                                                st>>>(m->md, m->rates, nrows, cnt, tallies);
        });
        VC_CUDA(cudaGetLastError());
        VC_CUDA(cudaMemcpyAsync(th, tallies, sizeof(th), cudaMemcpyDeviceToHost, st));
        VC_CUDA(cudaStreamSynchronize(st));
        m->feasible_rows = (int64_t)th[0];
        m->nnz_logical = (int64_t)th[1];
    }
    m->nnz_stored = padded ? nrows * width : m->nnz_logical;

    if ((rc = alloc_dev(m, (void**)&m->row_ptr, sizeof(int64_t) * (nrows + 3)))) return rc;
    if ((rc = alloc_dev(m, (void**)&m->col, sizeof(int32_t) * (m->nnz_stored + 16)))) return rc;
    if ((rc = alloc_dev(m, &m->val, (bf16 ? 2 : 4) * (size_t)(m->nnz_stored + 16)))) return rc;
    if ((rc = alloc_dev(m, (void**)&m->R, sizeof(float) * (nrows + 8)))) return rc;
    if (bf16 && (rc = alloc_dev(m, (void**)&m->scale, sizeof(float) * (nrows + 8)))) return rc;

    if (padded) {
        count_launches(1);
        k_padded_rowptr<<<(unsigned)((nrows + 1 + T - 1) / T), T, 0, st>>>(nrows, width, m->row_ptr);
    } else {
        if ((rc = exclusive_scan(m, cnt, nrows, m->row_ptr, st))) return rc;
    }
    unsigned long long* fill_tallies = padded ? tallies : nullptr;
    count_launches(1);
    by_h_build(m->md.H, [&](auto mh) {
        constexpr int MH = decltype(mh)::value;
        if (bf16)
            k_row_fill<MH, true><<<(unsigned)std::min<int64_t>(nb, (int64_t)m->num_sms * 16), kThreads, 0, st>>>(
                m->md, m->rates, nrows, padded, m->row_ptr, m->col, m->val,
                                                  m->scale, m->R, fill_tallies);
        else
            // one group of 32 rows per warp (the kernel strides further if the grid is capped)
            k_row_fill32<MH><<<(unsigned)((nrows + kFillThreads - 1) / kFillThreads), kFillThreads, 0, st>>>(
                m->md, m->rates, nrows, padded, m->row_ptr, m->col, (float*)m->val, m->R, fill_tallies);
    });
    VC_CUDA(cudaGetLastError());
    if (padded) {
        VC_CUDA(cudaMemcpyAsync(th, tallies, sizeof(th), cudaMemcpyDeviceToHost, st));
        VC_CUDA(cudaStreamSynchronize(st));
        m->feasible_rows = (int64_t)th[0];
        m->nnz_logical = (int64_t)th[1];
    }
    if (cnt) VC_CUDA(cudaFreeAsync(cnt, st));
    VC_CUDA(cudaFreeAsync(tallies, st));
    VC_CUDA(cudaStreamSynchronize(st));
    return plan_csr(m, st);
}

// ------------------------------------------------------------------------ user CSR
// Per row: columns in range, entries >= 0 and finite, feasible rows summing to 1 (after
// the scale) within 1e-5, row_ptr non-decreasing.  Per state: one feasible row at least.
__global__ void __launch_bounds__(kThreads) k_validate_rows(int S, int A, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const void* __restrict__ val, int bf16, float* __restrict__ scale,
                                int compute_scale, const float* __restrict__ R, int* err,
                                unsigned long long* tallies) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long feas = 0, nz = 0;
    if (s < S) {
        int flags = 0;
        bool any = false;
        for (int a = 0; a < A; a++) {
            const int64_t r = (int64_t)s * A + a;
            const int64_t lo = row_ptr[r], hi = row_ptr[r + 1];
            if (hi < lo || lo < 0) {
                flags |= kErrRowPtr;
                continue;
            }
            const float rr = R[r];
            const bool feasible = !(rr == -INFINITY);
            double sum = 0.0;
            for (int64_t j = lo; j < hi; j++) {
                const int c = col[j];
                if (c < 0 || c >= S) flags |= kErrBadColumn;
                const double v = bf16 ? bf16_to_double(((const uint16_t*)val)[j]) : (double)((const float*)val)[j];
                if (!(v >= 0.0) || !isfinite(v)) flags |= kErrNegative;
                sum += v;
            }
            if (bf16) {
                if (compute_scale) scale[r] = (sum > 0.0) ? (float)(1.0 / sum) : 0.0f;
                sum *= (double)scale[r];
            }
            if (feasible) {
                if (!isfinite(rr)) flags |= kErrNegative;
                if (fabs(sum - 1.0) > 1e-5) flags |= kErrRowSum;
                any = true;
                feas++;
                nz += (unsigned long long)(hi - lo);
            }
        }
        if (!any) flags |= kErrNoFeasible;
        if (flags) atomicOr(err, flags);
    }
    block_tally<kThreads>(feas, nz, tallies);
}

int build_csr_user(Mdp* m, const int64_t* row_ptr, const int32_t* col, const void* val, int val_dtype,
                   const float* row_scale, const float* R, cudaStream_t st) {
    const int64_t nrows = (int64_t)m->S * m->A;
    int64_t nnz = 0;
    VC_CUDA(cudaMemcpyAsync(&nnz, row_ptr + nrows, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    int64_t first = 0;
    VC_CUDA(cudaMemcpyAsync(&first, row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    VC_CUDA(cudaStreamSynchronize(st));
    if (first != 0 || nnz < 0) return fail(VC_ERR_ARG, "row_ptr[0] must be 0 and row_ptr[S*A] >= 0");
    const bool bf16 = val_dtype == VC_VAL_BF16;
    int rc;
    m->nnz_stored = nnz;
    if ((rc = alloc_dev(m, (void**)&m->row_ptr, sizeof(int64_t) * (nrows + 3)))) return rc;
    if ((rc = alloc_dev(m, (void**)&m->col, sizeof(int32_t) * (nnz + 16)))) return rc;
    if ((rc = alloc_dev(m, &m->val, (bf16 ? 2 : 4) * (size_t)(nnz + 16)))) return rc;
    if ((rc = alloc_dev(m, (void**)&m->R, sizeof(float) * (nrows + 8)))) return rc;
    if (bf16 && (rc = alloc_dev(m, (void**)&m->scale, sizeof(float) * (nrows + 8)))) return rc;
    VC_CUDA(cudaMemcpyAsync(m->row_ptr, row_ptr, sizeof(int64_t) * (nrows + 1), cudaMemcpyDeviceToDevice, st));
    if (nnz > 0) {
        VC_CUDA(cudaMemcpyAsync(m->col, col, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, st));
        VC_CUDA(cudaMemcpyAsync(m->val, val, (bf16 ? 2 : 4) * (size_t)nnz, cudaMemcpyDeviceToDevice, st));
    }
    VC_CUDA(cudaMemcpyAsync(m->R, R, sizeof(float) * nrows, cudaMemcpyDeviceToDevice, st));
    if (bf16 && row_scale)
        VC_CUDA(cudaMemcpyAsync(m->scale, row_scale, sizeof(float) * nrows, cudaMemcpyDeviceToDevice, st));

    int* err = nullptr;
    unsigned long long* tallies = nullptr;
    VC_CUDA(cudaMallocAsync((void**)&err, sizeof(int) + 2 * sizeof(unsigned long long) + 8, st));
    tallies = (unsigned long long*)((char*)err + 8);
    VC_CUDA(cudaMemsetAsync(err, 0, 8 + 2 * sizeof(unsigned long long), st));
    const int T = 256;
    count_launches(1);
    k_validate_rows<<<(m->S + T - 1) / T, T, 0, st>>>(m->S, m->A, m->row_ptr, m->col, m->val, bf16 ? 1 : 0,
                                                      m->scale, (bf16 && !row_scale) ? 1 : 0, m->R, err, tallies);
    VC_CUDA(cudaGetLastError());
    int herr = 0;
    unsigned long long th[2];
    VC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    VC_CUDA(cudaMemcpyAsync(th, tallies, sizeof(th), cudaMemcpyDeviceToHost, st));
    VC_CUDA(cudaFreeAsync(err, st));
    VC_CUDA(cudaStreamSynchronize(st));
    m->feasible_rows = (int64_t)th[0];
    m->nnz_logical = (int64_t)th[1];
    if (herr & kErrRowPtr) return fail(VC_ERR_ARG, "row_ptr is not non-decreasing");
    if (herr & kErrBadColumn) return fail(VC_ERR_ARG, "a column index is outside [0, S)");
    if (herr & kErrNegative) return fail(VC_ERR_NOT_STOCHASTIC, "negative or non-finite probability / reward");
    if (herr & kErrRowSum) return fail(VC_ERR_NOT_STOCHASTIC, "a feasible row does not sum to 1 (tolerance 1e-5)");
    if (herr & kErrNoFeasible) return fail(VC_ERR_NO_FEASIBLE_ACTION, "a state has no feasible action");
    return plan_csr(m, st);
}

}  // namespace vc
