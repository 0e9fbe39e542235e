/*
 * vcmdp.h -- C ABI of the GB300 value-iteration library for the vehicular-cloud
 * task-placement MDP of arxiv 2012.12419 (Section V).
 *
 * The method: value iteration (Algorithm 3) on the Bellman equation (Eq. 18), read as
 *     V(s) = max_{a feasible in s} [ R(s,a) + gamma * sum_s' P(s'|s,a) V(s') ],
 * Jacobi sweeps from V = 0 (or a warm start) until max_s |V^{k+1}(s) - V^k(s)| < tol,
 * then pi(s) = argmax_a (ties to the lowest action).
 *
 * The instance (Eq. 10-16 under the readings this library fixes):
 *   state  s = ph + 2*(q + (Q+1)*sum_k occ_k*(C+1)^k), S = 2(Q+1)(C+1)^H   (Eq. 10)
 *          occ_k in 0..C tasks on host k (hosts 0..H-2 vehicles, H-1 the RSU),
 *          q in 0..Q queued tasks, ph = 1 in the service-channel interval (SCHI)
 *   action a < H places the head task on host a (needs q >= 1, occ_a < C, and a == H-1
 *          or ph == 1); a = H defers.  A = H+1.                             (Eq. 11)
 *   one uniformised event then fires from the post-decision state, rates over
 *          Lam = lambda + C*sum(mu) + sum(delta) + 1: completion mu_k*occ_k, departure
 *          delta_k (host emptied, tasks lost), arrival lambda (blocked and lost when
 *          q == Q), phase flip f (CCHI->SCHI) / 1-f (SCHI->CCHI), self-loop the rest.
 *                                                                           (Eq. 12-13)
 *   reward R = w_occ*sum occ + w_q*q + w_loss*(sum_k delta_k occ_k + [q==Q] lambda)/Lam,
 *          all on the post-decision state.                                  (Eq. 14-16)
 *
 * Conventions for every entry point:
 *   - Returns VC_OK (0) or a VC_ERR_* code; vc_last_error() then describes the failure
 *     (thread-local string, valid until the next call on the same thread).
 *   - Array arguments are DEVICE pointers unless the comment says host.  They are
 *     borrowed for the duration of the call; the library never frees them.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is enqueued
 *     on it; calls that return statistics or a convergence outcome synchronise it.
 *   - The library allocates device memory only inside handles it owns (vc_mdp,
 *     vc_batch); vc_destroy / vc_batch_destroy release it.
 *   - States are indexed with int32 (S < 2^31); CSR offsets are int64.
 */
#ifndef VCMDP_H
#define VCMDP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VC_MAX_HOSTS 16

/* status codes */
#define VC_OK 0
#define VC_ERR_ARG 1                /* bad argument (size, pointer, range) */
#define VC_ERR_NOT_STOCHASTIC 2     /* a CSR row does not sum to 1 or has a negative entry */
#define VC_ERR_NO_FEASIBLE_ACTION 3 /* a state has no feasible action (R = -inf on all rows) */
#define VC_ERR_NOT_CONVERGED 4      /* max_sweeps ran out before the tolerance was met */
#define VC_ERR_TIMEOUT 5            /* a bounded device-side wait gave up */
#define VC_ERR_OOM 6                /* device allocation failed */
#define VC_ERR_CUDA 7               /* any other CUDA runtime error */

/* storage formats for vc_build_mdp (one of the first three, optionally | VC_PADDED) */
#define VC_IMPLICIT 0  /* successors generated in registers from the mixed-radix state code */
#define VC_CSR_F32 1   /* explicit CSR, FP32 probabilities, int32 columns, int64 row offsets */
#define VC_CSR_BF16 2  /* explicit CSR, BF16 probabilities + FP32 per-row renormalising scale */
#define VC_PADDED 16   /* CSR rows padded to exactly 2H+3 entries, infeasible rows included */
#define VC_DIRECT 32   /* CSR sweeps read rows straight from global memory (no shared-memory
                          pipeline); same arithmetic and results, for comparison */
#define VC_SLICED 64   /* also build the sliced copy of the matrix (vc_mdp_slice) and sweep it;
                          with VC_DIRECT the sliced sweep reads global memory directly */

/* value types for vc_build_mdp_csr */
#define VC_VAL_F32 0
#define VC_VAL_BF16 1

/* flags for vc_value_iterate */
#define VC_ITER_FP32_ONLY 1  /* stop after the FP32 sweeps: no FP64 refinement / certificate */
#define VC_ITER_ACCURATE 2   /* certify the error, not the residual: refine until the FP64
                                residual is below tol (1-gamma)/(2 gamma), so that
                                max|V64 - V*| <= gamma/(1-gamma) * residual <= tol/2 */
#define VC_ITER_PLAIN_CORRECTION 4  /* solve the refinement's correction equation by
                                       fixed-point sweeps instead of BiCGSTAB */
#define VC_ITER_SELF_LOOP 8  /* FP32 sweeps solve each action's self-transition exactly:
                                Q(s,a) = (R + gamma sum_{s' != s} P V) / (1 - gamma P(s|s,a))
                                (Puterman 1994, Sec. 6.3.3; Algorithm 4's in-block iteration
                                for a block of one state, run to its limit).  Same fixed point
                                V* and the same optimal actions as Eq. 18's backup, contraction
                                max gamma (1 - p_ss) / (1 - gamma p_ss) <= gamma per sweep, so
                                fewer sweeps; the sweep change, not Eq. 18's residual, is the
                                FP32 stopping test, and the FP64 refinement and certificate use
                                Eq. 18's backup as without the flag.  Every storage form. */

#define VC_ITER_BLOCK 16     /* implicit handles: FP32 sweeps run Algorithm 4's in-block iteration
                                (Section V-H) with the self-transition solve of VC_ITER_SELF_LOOP:
                                states are cut into blocks of B = 2(Q+1)(C+1)^h consecutive codes
                                (every queue length, phase and occupancy of the h inner hosts), and
                                in one global sweep each block runs `passes` local Jacobi passes in
                                which successors inside the block take the block's latest local
                                values and all others the previous global iterate
                                (vc_set_block_iteration).  Same fixed point V*; the stopping test
                                is the global sweep change; refinement and certificate unchanged.
                                VC_ERR_ARG for explicit handles. */

/* Model parameters (host struct; mu and delta are HOST arrays of length H). */
typedef struct vc_params {
    int32_t H, C, Q;      /* hosts, VM slots per host, queue capacity */
    int32_t reserved;
    double lambda;        /* task arrival rate */
    double f;             /* SCHI fraction of the sync interval (stationary phase law) */
    double gamma;         /* discount factor in (0, 1) */
    double w_occ, w_loss, w_q; /* reward weights */
    const double* mu;     /* host, [H] service rate per occupied slot */
    const double* delta;  /* host, [H] departure rate of each host */
} vc_params;

/* Sizes of a built instance. */
typedef struct vc_info {
    int64_t S;              /* states */
    int32_t A;              /* actions per state */
    int32_t fmt;            /* VC_IMPLICIT / VC_CSR_F32 / VC_CSR_BF16 (| VC_PADDED) */
    int64_t nnz_logical;    /* successor updates per sweep: non-zero entries of feasible rows */
    int64_t nnz_stored;     /* CSR entries streamed per sweep (0 for VC_IMPLICIT) */
    int64_t feasible_rows;  /* (s, a) pairs with a feasible */
    int64_t device_bytes;   /* device memory owned by the handle */
    int64_t sweep_bytes;    /* algorithmic HBM bytes of one FP32 sweep */
    int32_t has_model;      /* 1 if built from vc_params (exact FP64 P available) */
    int32_t csr_pipelined;  /* 1 if the FP32 sweep stages tiles through shared memory */
    int32_t csr_tile_states;/* states per staged tile (sliced: 32 x slices per tile) */
    int32_t csr_stages;     /* tiles in flight per CTA */
    int32_t csr_ctas_per_sm;/* resident CTAs per SM of the CSR sweep */
    int32_t csr_smem_bytes; /* dynamic shared memory per CTA */
    int32_t csr_sliced;     /* 1 if FP32 sweeps run on the sliced copy (vc_mdp_slice) */
    int32_t reserved;
    int64_t nnz_sliced;     /* entries of the sliced copy incl. padding (0 if none) */
} vc_info;

/* Statistics of vc_value_iterate (host struct, filled on return). */
typedef struct vc_stats {
    int64_t sweeps;         /* FP32 Bellman sweeps performed */
    double residual;        /* last FP32 residual max|V^{k+1}-V^k| */
    int64_t eval_sweeps;    /* FP32 products by P_pi in the refinement's correction solves */
    int64_t bellman64;      /* FP64 full Bellman backups (certification checks) */
    int32_t policy_rounds;  /* policy-improvement rounds inside the refinement */
    int32_t certified;      /* 1 if residual64 < tol */
    double residual64;      /* FP64 max|T V - V| of the returned V64 (Algorithm 3, step 3) */
    double ms_fp32;         /* device time of the FP32 sweeps (ms) */
    double ms_fp64;         /* device time of refinement + certification (ms) */
} vc_stats;

typedef struct vc_mdp vc_mdp;
typedef struct vc_batch vc_batch;

/* Description of the last failure on the calling thread ("" if none). */
const char* vc_last_error(void);

/* Number of CUDA kernels this library has enqueued since it was loaded (all threads). */
int64_t vc_kernel_launches(void);

/*
 * Build an instance from model parameters (Eq. 10-16).  fmt selects the storage of the
 * FP32/BF16 sweeps; VC_IMPLICIT stores nothing per transition.  CSR builds run a count,
 * an exclusive scan and a fill kernel on `stream`.  Rows hold the merged non-zero
 * successors sorted by column (VC_PADDED: exactly 2H+3 entries, zero-padded).  BF16
 * entries are bf16(p) rounded to nearest even from the FP64 probability; each row
 * carries scale = 1/sum_j bf16(p_j) (FP64 sum, rounded to FP32).  Every handle built
 * here also keeps the FP64 model for refinement, certification and gradients.
 * fmt | VC_SLICED also builds the sliced copy (vc_mdp_slice) before returning.
 * Errors: VC_ERR_ARG for H outside 1..16, C < 1, Q < 0, S >= 2^31, rates <= 0 (mu,
 * lambda; delta >= 0), f outside (0,1), gamma outside (0,1); VC_ERR_OOM.
 */
int vc_build_mdp(const vc_params* p, int fmt, void* stream, vc_mdp** out);

/*
 * Build an instance from an arbitrary explicit MDP in CSR form: the transition law
 * P(s'|s,a) and expected reward r(s,a) of the Bellman equation (Section V-G, Eq. 18) given
 * as data instead of generated from Eq. 10-16, so any finite MDP runs through the same
 * sweeps (device pointers, copied into the handle): row r = s*A + a spans [row_ptr[r], row_ptr[r+1]) of col/val; R[r]
 * is its expected reward, -INFINITY marking an infeasible action.  val_dtype is
 * VC_VAL_F32 (float) or VC_VAL_BF16 (uint16 bf16 bit patterns); row_scale (nullable,
 * [S*A] float) multiplies a row's sum (BF16 only; NULL = 1/sum of the stored values).
 * Validated on the device: columns in [0, S), entries >= 0, each feasible row summing
 * to 1 within 1e-5 after scaling (VC_ERR_NOT_STOCHASTIC), each state with at least one
 * feasible action (VC_ERR_NO_FEASIBLE_ACTION), row_ptr non-decreasing (VC_ERR_ARG).
 * The FP64 refinement of such a handle uses the stored (scaled) values in FP64.
 */
int vc_build_mdp_csr(int64_t S, int32_t A, const int64_t* row_ptr, const int32_t* col, const void* val,
                     int val_dtype, const float* row_scale, const float* R, double gamma, void* stream,
                     vc_mdp** out);

/*
 * Parameters of the paper's binary-action model (host struct; mu and delta are HOST arrays
 * of length H).  Section V-B..V-E: the state (n_1..n_TT, M, e) of Eq. 10 is read as the
 * busy VMs u_k of each of H vehicular clouds plus the pending request e; the actions are
 * A = {-1, 1} of Eq. 11; the reward is r = k - g of Eqs. 14-16.
 */
typedef struct vc_binary_params {
    int32_t H;            /* vehicular clouds (1..16) */
    int32_t C;            /* VMs per cloud */
    int32_t J;            /* largest request in VMs (1..8); sizes 1..J equally likely */
    int32_t reserved;
    double lambda;        /* request arrival rate */
    double gamma;         /* discount factor in (0, 1) */
    double beta_vc;       /* reward per VM placed on a vehicular cloud (Eq. 15) */
    double beta_tc;       /* cost per VM hosted in the paid traditional cloud (Eq. 16) */
    double gamma_vc;      /* penalty per idle VM of the requested cloud (Eq. 16) */
    const double* mu;     /* host, [H] completion rate of each busy VM */
    const double* delta;  /* host, [H] departure rate of each cloud */
} vc_binary_params;

/*
 * Build an explicit instance of the paper's binary-action model (Section V-B..V-E; the
 * transition law the paper leaves open is read as one uniformised event per step):
 *   state  s = e + E * sum_k u_k (C+1)^k, E = 1 + H J, S = E (C+1)^H; u_k in 0..C busy
 *          VMs of cloud k; e = 0 no request, e = 1 + i J + (n-1) a task of n VMs for cloud i
 *   action 0 ("-1"): the task goes to the paid traditional cloud, reward
 *          -beta_tc n - gamma_vc (C - u_i); with no request the no-op, reward 0
 *   action 1 ("+1"): the task is placed on cloud i, feasible iff a request is pending and
 *          u_i + n <= C, reward beta_vc n - gamma_vc (C - u_i - n)
 *   then from the post-decision state (request consumed) one event, rates over
 *          Lam = lambda + C sum(mu) + sum(delta) + 1: completion of a busy VM of cloud k
 *          (mu_k u_k, u_k - 1), departure of cloud k (delta_k, u_k = 0), a request of n VMs
 *          at cloud i (lambda / (H J) for each (i, n)), self-loop the rest.
 * Rows hold the merged non-zero successors sorted by column (at most 2H + 1 + HJ).  fmt is
 * VC_CSR_F32 or VC_CSR_BF16 (BF16 values rounded to nearest even from the FP64
 * probability, per-row FP32 scale 1/sum bf16(p)), optionally | VC_SLICED | VC_DIRECT.  The
 * handle keeps the exact FP64 probabilities and rewards beside the stored ones, so the
 * FP64 refinement and certificate of vc_value_iterate solve the exact model; the FP32
 * sweeps, products and autotuner run on the stored values.  It has no rate gradients
 * (vc_value_grad) and no greedy rule (vc_greedy_policy): both return VC_ERR_ARG.
 * Errors: VC_ERR_ARG for H outside 1..16, J outside 1..8, C < 1, S >= 2^31, lambda or a mu
 * not > 0, a delta < 0, gamma outside (0, 1), non-finite weights, other formats;
 * VC_ERR_OOM.
 */
int vc_build_binary_mdp(const vc_binary_params* p, int fmt, void* stream, vc_mdp** out);

/* Sizes of a handle (host struct out). */
int vc_mdp_info(const vc_mdp* m, vc_info* out);

/*
 * Copy the stored CSR of a handle out (device pointers, each nullable): row_ptr
 * [S*A+1] int64, col [nnz_stored] int32, val [nnz_stored] float (VC_CSR_F32) or uint16
 * bf16 bits (VC_CSR_BF16), row_scale [S*A] float (BF16 only), R [S*A] float.
 * VC_ERR_ARG for a VC_IMPLICIT handle, which stores no transitions.
 */
int vc_mdp_export_csr(const vc_mdp* m, int64_t* row_ptr, int32_t* col, void* val, float* row_scale, float* R,
                      void* stream);

/*
 * Add a sliced copy of the stored matrix to a CSR handle and make the FP32 sweeps use
 * it.  This is a storage layout for the Eq. 18 backup of the same rows, not an operation
 * of the paper: SELL-C-sigma (Kreutzer et al., SIAM J. Sci. Comput. 36(5), 2014) with 32
 * states per slice, states sorted inside windows of 4096 by feasible-action mask and row
 * length; each (slice, action) block stores its rows lane-fastest, padded to the block's
 * longest feasible row with zero-valued entries.  Infeasible rows store nothing.  The
 * sweep keeps the CSR kernels' arithmetic (FMA in column order, lowest-index argmax), so
 * V, pi and the residual are bitwise those of the CSR sweep.  The CSR stays (FP64
 * refinement of user matrices, export, autotuner candidates); the copy adds
 * nnz_sliced x (4 + value bytes) + 4 S A (+ 4 S A for BF16) bytes.  Runs on `stream`
 * and synchronises it.  The sweep stages tiles of slices through shared memory (the
 * direct-load sliced kernel on VC_DIRECT handles or when no tile fits).  Errors:
 * VC_ERR_ARG for a VC_IMPLICIT handle or A > 31; VC_ERR_OOM.  Idempotent.
 */
int vc_mdp_slice(vc_mdp* m, void* stream);

/*
 * Fault-injection hook for the bounded device waits (no paper counterpart).  The pipelined
 * sweeps (CSR and sliced) wait on shared-memory barriers for their staged tiles with an
 * iteration limit; polls >= 0 caps every such wait of this handle's later solves at that
 * many polls (0: give up at once), polls < 0 restores the default (2^22).  A wait that
 * gives up flags the sweep, the kernel drains its own copies in flight (with the default
 * limit) and returns, and vc_value_iterate returns VC_ERR_TIMEOUT; the handle and the
 * CUDA context stay usable.  Synchronous; applies to later launches on the handle.
 * VC_ERR_ARG for NULL.
 */
int vc_set_wait_limit(vc_mdp* m, int64_t polls);

/*
 * Value iteration (Algorithm 3).  V: [S] float, in: V^0 (zeros = the paper's step 1,
 * anything else = warm start / resume), out: the last FP32 iterate.  FP32 Jacobi sweeps
 * run until the sweep residual is below max(tol, 4 ulp(max|V|)), stops improving for
 * 64 sweeps (FP32 floor), or max_sweeps is reached.  Then, unless VC_ITER_FP32_ONLY,
 * the FP64 refinement: pi = argmax of the FP32 values, evaluated by mixed-precision
 * iterative refinement (FP64 policy residual, FP32 correction solve by BiCGSTAB -- or
 * fixed-point sweeps with VC_ITER_PLAIN_CORRECTION or when BiCGSTAB breaks down -- FP64
 * update) until the policy residual is below tol, and an FP64 full Bellman backup
 * V64 = T(V) whose residual max|T V - V| is the certificate (policy improvement repeats
 * if the backup changes pi).  V64_out ([S] double, nullable) receives that backup, pi_out
 * ([S] int32, nullable) its argmax.  Synchronises `stream`.
 * With VC_ITER_SELF_LOOP the FP32 sweeps use the self-transition-solved backup (see the
 * flag); the policy taken from the FP32 values and everything after it are unchanged.
 * Errors: VC_ERR_NOT_CONVERGED if max_sweeps ran out (outputs still written),
 * VC_ERR_ARG for tol <= 0 or max_sweeps < 1.
 */
int vc_value_iterate(vc_mdp* m, float* V, double* V64_out, int32_t* pi_out, double tol, int64_t max_sweeps,
                     int flags, vc_stats* stats, void* stream);

/*
 * Policy extraction from FP32 values (Algorithm 3, step 4): pi[s] = argmax_a Q(s,a)
 * (lowest action on ties, FP32 arithmetic), qgap[s] (nullable) = best Q minus the
 * second-best (+INFINITY with one feasible action).  V: [S] float.
 */
int vc_extract_policy(vc_mdp* m, const float* V, int32_t* pi, float* qgap, void* stream);

/*
 * One FP32 Bellman sweep (Algorithm 3, step 2) without bookkeeping: V_out[s] = max_a Q(s,a)
 * from V ([S] float), each output nullable (pi int32, qgap float).  Repeated calls give a
 * fixed number of Jacobi sweeps; kernels are only enqueued on `stream`.
 */
int vc_bellman32(vc_mdp* m, const float* V, float* V_out, int32_t* pi, float* qgap, void* stream);

/*
 * Shape of the in-block iteration of an implicit handle (VC_ITER_BLOCK; Algorithm 4's
 * "episodes" inside a block, Section V-H): inner_hosts = h (0..3) gives blocks of
 * B = 2(Q+1)(C+1)^h states (at most 512; -1 = the largest such h, the default), passes the
 * local passes per global sweep (1..64, default 4; 1 is the plain self-transition sweep).
 * Applies to later solves.  VC_ERR_ARG for explicit handles, passes outside 1..64, h above
 * 3 or H, or a block of more than 512 states.
 */
int vc_set_block_iteration(vc_mdp* m, int32_t inner_hosts, int32_t passes);

/* The current shape (host outputs, each nullable): inner hosts, states per block, passes. */
int vc_block_iteration_info(const vc_mdp* m, int32_t* inner_hosts, int32_t* block_states, int32_t* passes);

/*
 * One FP32 Bellman sweep of the model in *p (implicit form) that allocates no device
 * memory, for callers that cannot call cudaMalloc: code whose device memory is entirely
 * held by another allocator's pool, control loops that must not risk the device-wide
 * synchronisation an allocation can cause, or code running while another library captures
 * the stream.  The paper has no counterpart; it is an interface convenience.
 *   V: [S] float in; V_out: [S] float out (a different buffer); pi: [S] int32 argmax
 *   (nullable); residual: ONE float on the device (nullable) receiving max|V_out - V|
 *   (+INFINITY if any difference is NaN).
 * Results equal vc_bellman32 on a VC_IMPLICIT handle of the same model.
 * Scratch: the post-decision values live in a static device array of 1,048,576 floats
 * (4 MiB) plus a residual word and a 1.3 KB control block, present on every GPU that
 * loads the library until the process exits; S above 1,048,576 returns VC_ERR_ARG.  The
 * first call on each device looks up the arrays' device addresses (cudaGetSymbolAddress)
 * and the SM count with that device current: make that first call before any stream
 * capture.  Later calls only enqueue kernels and an asynchronous memset on `stream`, so
 * they may be captured into a CUDA graph (the bounds-checking build's read-back excepted);
 * a replay reads V and writes V_out, pi and residual at the addresses captured.  All
 * calls on a device share the
 * array, so calls that overlap on the GPU (different streams, or different host threads)
 * race and must be ordered by the caller.  The residual word is cleared on every call.
 * In the bounds-checking build (libvcmdp_debug.so) the call also synchronises `stream`
 * and returns VC_ERR_CUDA if a device bounds check failed.
 */
int vc_bellman32_noalloc(const vc_params* p, const float* V, float* V_out, int32_t* pi, float* residual,
                         void* stream);

/*
 * FP64 Bellman backup of V ([S] double): V_out[s] = max_a Q(s,a) in FP64 (nullable),
 * pi (nullable) the argmax, qgap (nullable, double) the gap, and *residual (host,
 * nullable) = max_s |V_out(s) - V(s)|, the check of Algorithm 3, step 3.  Synchronises
 * `stream` when residual is requested.
 */
int vc_bellman64(vc_mdp* m, const double* V, double* V_out, int32_t* pi, double* qgap, double* residual,
                 void* stream);

/*
 * The paper's greedy heuristic (Algorithm 2, "efficient VM first") read as a policy on this
 * MDP: pi[s] = the feasible host with the largest service rate mu_a when a task waits
 * (ties to the lowest host index), else defer (a = H).  pi: [S] int32 device, written on
 * `stream`.  Evaluating it with vc_evaluate_policy gives the heuristic's values, which
 * never exceed the optimum (the paper's MDP-versus-greedy comparison).  VC_ERR_ARG for a
 * handle built from a user CSR (no model to read rates from).
 */
int vc_greedy_policy(vc_mdp* m, int32_t* pi, void* stream);

/*
 * The AAA multichannel timer update (Section II, Algorithm 1 with Eqs. 1-9) over a trace of
 * synchronisation intervals (SIs): the SCHI fraction f it produces is the `f` of
 * vc_params.  Host routine (no device work, no handle).
 *   S_v, D_v, R_v: HOST arrays [n_si][n_vehicles], row j = SI j: BSMs each vehicle sent
 *       and had acknowledged (Eq. 2), the total end-to-end delay in ms of the BSMs it
 *       received (the numerator of Eq. 3), and how many it received (R_vhBSM).
 *   si_per_second: SIs per UTC second (10 for the standard's 100 ms SI); si_ms the SI,
 *       dcchi_ms + dschi_ms = si_ms the IEEE 1609.4 defaults (50 + 50 ms).
 *   In an SI that is not the last of its second: S_V2V <- (S_V2V + sum_h S_vh)/(1 + N_V),
 *   D_V2V <- (D_V2V + sum_h D_vh)/(1 + sum_h R_vh).  In the last SI of each second:
 *   U_CCH = S_V2V D_V2V, I_CCH = CCHI - U_CCH; if U_CCH < DCCHI then CCHI = U_CCH and
 *   SCHI = SCHI + I_CCH, else both return to the defaults; S_V2V = D_V2V = 0.
 *   cchi_out, schi_out ([n_si / si_per_second] doubles, host) receive the intervals after
 *   each second's update; f_out (nullable) SCHI / SI.  CCHI + SCHI stays equal to the SI.
 * VC_ERR_ARG for NULL arrays, sizes < 1, or defaults that do not sum to the SI.
 */
int vc_aaa_intervals(const double* S_v, const double* D_v, const double* R_v, int32_t n_vehicles, int32_t n_si,
                     int32_t si_per_second, double si_ms, double dcchi_ms, double dschi_ms, double* cchi_out,
                     double* schi_out, double* f_out);

/*
 * Policy evaluation V_pi = R_pi + gamma P_pi V_pi (Eq. 18 with the action fixed) over the
 * chosen rows only, by mixed-precision iterative refinement: the policy residual
 * r = T_pi V - V and its maximum in FP64, the correction (I - gamma P_pi) e = r solved in
 * FP32 by BiCGSTAB (fixed-point sweeps if it breaks down) until its residual is below
 * tol/2, V += e in FP64, until max|r| < tol (the point where an FP64 Jacobi sweep would
 * change V by less than tol).  pi: [S] int32 (feasible everywhere, else VC_ERR_ARG);
 * V_pi: [S] double, in: initial guess, out: the result.  *sweeps_out (host, nullable)
 * receives the FP32 products by P_pi spent.  VC_ERR_NOT_CONVERGED once max_sweeps such
 * products are spent.  Synchronises `stream`.
 */

int vc_evaluate_policy(vc_mdp* m, const int32_t* pi, double* V_pi, double tol, int64_t max_sweeps,
                       int64_t* sweeps_out, void* stream);

/*
 * Autotuner of the CSR sweep schedule: times every feasible shared-memory tiling (states
 * per tile, pipeline stages, CTAs per SM), the direct-load kernel and, when the handle
 * has a sliced copy, the sliced sweep at several CTAs per SM, reps sweeps each on
 * `stream`, and keeps the fastest for later sweeps.  *best_us (host,
 * nullable) receives its time per sweep.  No-op for VC_IMPLICIT handles.  The schedule
 * never changes results: every candidate does the same arithmetic in the same order.
 */
int vc_autotune(vc_mdp* m, int reps, double* best_us, void* stream);

/*
 * Text table of the last vc_autotune on this handle (one line per candidate: kernel,
 * states per tile, stages, CTAs per SM, shared memory bytes, microseconds per sweep)
 * copied into the host buffer buf of len bytes, NUL-terminated and truncated to fit.
 * Returns the length needed including the NUL (1 if the handle was never tuned).
 */
int64_t vc_autotune_report(const vc_mdp* m, char* buf, int64_t len);

/*
 * The autotuner's candidate schedules without timing: *count (host, nullable) receives the
 * number of candidates of this CSR handle, in the order of vc_autotune_report's rows (CSR
 * tilings, the direct CSR kernel, then with a sliced copy the ring sweep's launch shapes
 * and the direct sliced kernel); index >= 0 switches the handle to that candidate for later
 * sweeps, index < 0 only counts.  The schedule never changes results (see vc_autotune).
 * VC_ERR_ARG for an implicit handle or an index >= *count; the handle keeps its schedule.
 */
int vc_sweep_schedule(vc_mdp* m, int32_t index, int32_t* count, void* stream);

/* Statistics of vc_value_grad (host struct). */
typedef struct vc_grad_stats {
    int64_t sweeps;          /* FP32 products by P_pi^T in the first solve */
    int64_t correction_sweeps; /* FP32 products by P_pi^T in the FP64 refinement's corrections */
    int32_t rounds;          /* refinement rounds */
    int32_t reserved;
    double residual64;       /* FP64 max|rho + gamma P_pi^T lam - lam| of the returned lam */
    double J;                /* rho . V */
    int64_t nnz_transpose;   /* entries of P_pi^T */
} vc_grad_stats;

/*
 * Adjoint gradient of J = rho . V_pi for a handle built from model parameters.  The paper
 * differentiates nothing; this is Eq. 18 with the action fixed to pi (the policy-evaluation
 * equation V = R_pi + gamma P_pi V of Section V-G) differentiated in the model parameters
 * of Eq. 12-16 (rates and reward weights), by the adjoint method:
 *     dJ/dtheta_i = lam . (dR_pi/dtheta_i + gamma (dP_pi/dtheta_i) V),
 *     (I - gamma P_pi)^T lam = rho,
 * theta = (lambda, mu_1..mu_H, delta_1..delta_H, f, w_occ, w_loss, w_q), 2H+5 entries.
 * V is the policy's value ([S] double, e.g. V64 from vc_value_iterate, which equals the
 * optimum when pi is optimal: then this is the derivative of the optimal J wherever the
 * optimal action is unique), pi its
 * policy ([S] int32, feasible everywhere, else VC_ERR_ARG), rho [S] double weights.
 * lam is solved with products by an explicit transpose P_pi^T (one pull over its rows):
 * an FP32 BiCGSTAB solve (fixed-point sweeps lam <- rho + gamma P^T lam if it breaks
 * down), then FP64 residual + FP32 correction rounds until the FP64 residual is below tol.
 * dJ_dtheta: [2H+5] double on the device; lambda_out: [S] double (nullable).  Temporary
 * device memory for P_pi^T is stream-ordered (cudaMallocAsync) and released before
 * return.  Synchronises `stream`.  VC_ERR_ARG for a handle built from an explicit CSR.
 * Errors: VC_ERR_NOT_CONVERGED if the residual test is not met within max_sweeps.
 */
int vc_value_grad(vc_mdp* m, const double* V, const int32_t* pi, const double* rho, double* dJ_dtheta,
                  double* lambda_out, double tol, int64_t max_sweeps, vc_grad_stats* stats, void* stream);

/*
 * The objective of vc_value_grad, J = rho . V = sum_s rho[s] V[s], in FP64 on the device
 * (the initial-distribution-weighted value whose gradient vc_value_grad returns; the paper
 * has no objective of this form).  V, rho: [S] double device arrays; J: ONE double on the
 * device, written on `stream` (enqueued only).  One block sums in a fixed order, so the
 * result is reproducible bit for bit.  VC_ERR_ARG for NULL pointers or S < 1.
 */
int vc_objective(const double* V, const double* rho, int64_t S, double* J, void* stream);

/* ------------------------------------------------------------------ batched solves */

/* Sizes and schedule of a batch (host struct). */
typedef struct vc_batch_info_t {
    int32_t n;              /* instances */
    int32_t tiles;          /* tiles of the schedule */
    int64_t total_states;   /* sum of the instances' S (length of the concatenated arrays) */
    int32_t tile_states;    /* states per tile */
    int32_t blocks_per_sm;  /* persistent grid = SMs x blocks_per_sm (capped by the tile count) */
    int32_t grid;
    int32_t reserved;
    int64_t device_bytes;
} vc_batch_info_t;

/* Per-instance result of vc_value_iterate_batch (host struct array of length n). */
typedef struct vc_batch_stats {
    int64_t sweeps;            /* FP32 sweeps of this instance */
    int64_t correction_sweeps; /* FP32 products by P_pi in its refinement's correction solves */
    double residual64;         /* FP64 max|T V - V| of its certified values */
    int32_t certified;         /* residual64 < tol */
    int32_t termination;       /* FP32 loop: 1 tolerance, 2 max_sweeps, 3 FP32 floor stall */
    int32_t rounds;            /* refinement rounds until its certificate held (later rounds
                                  skip it; 0 with VC_ITER_FP32_ONLY or if never certified) */
    int32_t reserved;
} vc_batch_stats;

/*
 * Build a batch of n independent instances (p: HOST array of n vc_params, each validated
 * as in vc_build_mdp; implicit form).  Instance i occupies states [off_i, off_i + S_i) of
 * the concatenated arrays, off from vc_batch_offsets.  The schedule (tile size, persistent
 * grid) starts at 4096 states per tile and 8 blocks per SM; vc_batch_autotune picks one by
 * timing.  CUDA graphs are captured once per schedule: the FP32 value-iteration loop (with
 * Eq. 18's backup, and with each action's self-transition solved) and the refinement's
 * correction loops, each a device-side WHILE loop.  Algorithm 3 for
 * every instance, applied to many cells of a vehicular cloud at once (the paper's BSDI
 * partitions one state space into independent blocks; here the blocks are whole MDPs).
 */
int vc_build_batch(const vc_params* p, int32_t n, void* stream, vc_batch** out);

int vc_batch_info(const vc_batch* b, vc_batch_info_t* out);

/* Host array of n+1 int64: first state of each instance, then the total. */
int vc_batch_offsets(const vc_batch* b, int64_t* offsets);

/*
 * Value iteration of every instance (Algorithm 3), each with its own gamma, tolerance test
 * (max(tol, 4 ulp(max|V_i|)) or FP32 stall) and sweep count, in one graph launch; then,
 * unless VC_ITER_FP32_ONLY, every instance's argmax policy is evaluated by FP64 residual +
 * FP32 correction (BiCGSTAB for every instance in one graph launch; fixed-point sweeps with
 * VC_ITER_PLAIN_CORRECTION or if an instance breaks down) + FP64 update and certified by
 * one FP64 Bellman backup (repeated while an instance fails); VC_ITER_ACCURATE certifies
 * each instance's error
 * (residual below tol (1 - gamma_i) / (2 gamma_i)).  VC_ITER_SELF_LOOP runs the FP32 loop
 * with the self-transition-solved backup, as in vc_value_iterate; VC_ITER_BLOCK adds
 * Algorithm 4's in-block passes to it (vc_batch_set_block_iteration), each instance in its
 * own blocks.  V: [total] float in (warm start) / out (FP32
 * iterate); V64_out [total] double and pi_out [total] int32 nullable (pi is local to the
 * instance: 0..H_i); per_inst: HOST array of n stats (nullable).  Synchronises `stream`.
 * VC_ERR_NOT_CONVERGED if an instance is not certified (or, FP32 only, hit max_sweeps).
 */
int vc_value_iterate_batch(vc_batch* b, float* V, double* V64_out, int32_t* pi_out, double tol, int64_t max_sweeps,
                           int flags, vc_batch_stats* per_inst, void* stream);

/*
 * Instances solved whole inside one thread block (no paper counterpart; Algorithm 4's block
 * taken as the whole instance): before the FP32 graph loop, each instance with S <=
 * max_states (capped by the device's shared memory: 16 bytes per state for the iterate pair
 * and the pass-1 values; the default is that cap, about 14,000 states on GB300) is swept in
 * one CTA with its values in shared memory and its own step-3 test after every sweep --
 * the loop's arithmetic, so the iterate and the sweep count are the loop's bit for bit --
 * and the loop skips it.  With VC_ITER_BLOCK such an instance is one block iterated by the
 * self-transition sweeps to its test.  0 disables the path.  Synchronises `stream`.
 * VC_ERR_ARG for max_states < 0.
 */
int vc_batch_set_small_instances(vc_batch* b, int32_t max_states, void* stream);

/* Instances taking that path and the state limit in force (host outputs, nullable). */
int vc_batch_small_instances(const vc_batch* b, int32_t* count, int32_t* max_states);

/*
 * Shape of the batched in-block iteration (VC_ITER_BLOCK; Algorithm 4's "episodes", Section
 * V-H): each instance i is cut into blocks of 2(Q_i+1)(C_i+1)^h_i states with the largest
 * h_i <= 3 that fits `threads` (32..512, default 512), packed into tiles of whole blocks of
 * at most `threads` states, one thread per state; `passes` (1..64, default 4) local passes
 * per global sweep.  Rebuilds the tile table and recaptures the loop graphs on `stream`
 * (synchronised).  VC_ERR_ARG for out-of-range values or an instance whose smallest block
 * 2(Q_i+1) exceeds `threads` (the previous shape is kept).
 */
int vc_batch_set_block_iteration(vc_batch* b, int32_t threads, int32_t passes, void* stream);

/*
 * Autotuner of the batched schedule: times the FP32 loop graph for `sweeps` sweeps of every
 * (tile size in {256, 512, ..., 8192}, blocks per SM in {2, 4, 8}) and keeps the fastest,
 * recapturing the graphs.  *best_ms (host, nullable) receives its time.  Results do not
 * depend on the schedule.
 */
int vc_batch_autotune(vc_batch* b, int sweeps, double* best_ms, void* stream);

/* Text table of the last vc_batch_autotune (same contract as vc_autotune_report). */
int64_t vc_batch_autotune_report(const vc_batch* b, char* buf, int64_t len);

/* Release a batch and all device memory it owns (NULL is a no-op). */
int vc_batch_destroy(vc_batch* b);

/* Release a handle and all device memory it owns (NULL is a no-op). */
int vc_destroy(vc_mdp* m);

#ifdef __cplusplus
}
#endif

#endif /* VCMDP_H */
