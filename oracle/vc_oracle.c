/*
 * vc_oracle.c -- plain FP64 CPU oracle for value iteration on the vehicular-cloud
 * task-placement MDP (arxiv 2012.12419, Section V, Eq. 18 and Algorithm 3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the CUDA
 * path is checked against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or helper with the
 * CUDA library: it enumerates every successor with nested loops, merges duplicates
 * by linear search and runs plain Jacobi sweeps, all in double precision.
 *
 * Model (Section V-A..V-G; the paper leaves the concrete instance open, so the
 * readings below are the ones this project fixes and lists in its design notes):
 *   state  s = ph + 2*(q + (Q+1)*sum_k occ_k*(C+1)^k)            (Eq. 10, mixed radix)
 *          ph = 1 in the service-channel interval (SCHI), 0 in CCHI
 *   action a in 0..H-1 places the head task on host a, a = H defers (Eq. 11 widened)
 *          placement feasible iff q >= 1, occ_a < C and (a == H-1 (the RSU) or ph == 1)
 *   post-decision state x: occ_a + 1, q - 1 for a placement; x = s for defer
 *   one uniformised event fires from x (Eq. 12-13 read as a CTMC), all rates / Lam,
 *          Lam = lambda + C*sum(mu) + sum(delta) + 1:
 *          completion on host k   rate mu_k*occ_k     -> occ_k - 1
 *          departure of host k    rate delta_k        -> occ_k = 0 (its tasks are lost)
 *          arrival                rate lambda         -> q + 1, or blocked (lost) if q == Q
 *          phase flip             rate f (CCHI->SCHI), 1-f (SCHI->CCHI)
 *          self-loop              the remaining probability
 *   reward R(s,a) = w_occ*sum occ(x) + w_q*q(x)
 *                 + w_loss*(sum_k delta_k*occ_k(x)/Lam + [q(x)==Q]*lambda/Lam)   (Eq. 14-16 replaced)
 *   Bellman      V(s) = max_{a feasible} [ R(s,a) + gamma * sum_s' P(s'|s,a) V(s') ]  (Eq. 18,
 *                max taken over actions, expected reward, discount gamma)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXH 16
#define OR_MAXSUCC (2 * OR_MAXH + 4)
#define OR_NTHETA (2 * OR_MAXH + 5)

typedef struct {
    int32_t H, C, Q, pad_;
    double lambda, f, gamma, w_occ, w_loss, w_q;
    double mu[OR_MAXH];
    double delta[OR_MAXH];
} or_params;

/* ---------------------------------------------------------------- state codes */

int64_t or_num_states(const or_params* p) {
    int64_t n = 2 * (int64_t)(p->Q + 1);
    for (int k = 0; k < p->H; k++) n *= (p->C + 1);
    return n;
}

static void decode(const or_params* p, int64_t s, int* occ, int* q, int* ph) {
    *ph = (int)(s % 2);
    int64_t rest = s / 2;
    *q = (int)(rest % (p->Q + 1));
    rest = rest / (p->Q + 1);
    for (int k = 0; k < p->H; k++) {
        occ[k] = (int)(rest % (p->C + 1));
        rest = rest / (p->C + 1);
    }
}

static int64_t encode(const or_params* p, const int* occ, int q, int ph) {
    int64_t code = 0;
    for (int k = p->H - 1; k >= 0; k--) code = code * (p->C + 1) + occ[k];
    return ph + 2 * (q + (int64_t)(p->Q + 1) * code);
}

void or_decode(const or_params* p, int64_t s, int32_t* occ, int32_t* q, int32_t* ph) {
    int o[OR_MAXH], qq, pp;
    decode(p, s, o, &qq, &pp);
    for (int k = 0; k < p->H; k++) occ[k] = o[k];
    *q = qq;
    *ph = pp;
}

int64_t or_encode(const or_params* p, const int32_t* occ, int32_t q, int32_t ph) {
    int o[OR_MAXH];
    for (int k = 0; k < p->H; k++) o[k] = occ[k];
    return encode(p, o, q, ph);
}

double or_uniformisation(const or_params* p) {
    double sum_mu = 0.0, sum_delta = 0.0;
    for (int k = 0; k < p->H; k++) {
        sum_mu += p->mu[k];
        sum_delta += p->delta[k];
    }
    return p->lambda + p->C * sum_mu + sum_delta + 1.0;
}

/* Is action a allowed in state s?  (placement rule and defer, see header) */
int or_feasible(const or_params* p, int64_t s, int a) {
    int occ[OR_MAXH], q, ph;
    if (a < 0 || a > p->H) return 0;
    if (a == p->H) return 1;
    decode(p, s, occ, &q, &ph);
    if (q < 1) return 0;
    if (occ[a] >= p->C) return 0;
    if (a != p->H - 1 && ph != 1) return 0;
    return 1;
}

/* Adds probability pr for target t into a small merged list (linear search). */
static void add_succ(int64_t* cols, double* probs, int* n, int64_t t, double pr) {
    for (int i = 0; i < *n; i++) {
        if (cols[i] == t) {
            probs[i] += pr;
            return;
        }
    }
    cols[*n] = t;
    probs[*n] = pr;
    (*n)++;
}

/* Sorts the merged list by target index (insertion sort; lists are tiny). */
static void sort_succ(int64_t* cols, double* probs, int n) {
    for (int i = 1; i < n; i++) {
        int64_t c = cols[i];
        double v = probs[i];
        int j = i - 1;
        while (j >= 0 && cols[j] > c) {
            cols[j + 1] = cols[j];
            probs[j + 1] = probs[j];
            j--;
        }
        cols[j + 1] = c;
        probs[j + 1] = v;
    }
}

/*
 * Transition row of (s, a): merged successor list sorted by target, zero-probability
 * entries dropped, plus the expected one-step reward.  Returns the number of
 * successors, or -1 if a is not feasible in s.
 */
int or_transitions(const or_params* p, int64_t s, int a, int64_t* cols, double* probs, double* R) {
    int occ[OR_MAXH] = {0}, q = 0, ph = 0;
    if (!or_feasible(p, s, a)) return -1;
    decode(p, s, occ, &q, &ph);
    /* post-decision state */
    if (a < p->H) {
        occ[a] += 1;
        q -= 1;
    }
    const int64_t x = encode(p, occ, q, ph);
    const double Lam = or_uniformisation(p);

    int64_t ec[OR_MAXSUCC];
    double ep[OR_MAXSUCC];
    int ne = 0;
    double total = 0.0;
    for (int k = 0; k < p->H; k++) {
        /* completion on host k */
        if (occ[k] > 0) {
            int o2[OR_MAXH];
            memcpy(o2, occ, sizeof(int) * p->H);
            o2[k] -= 1;
            ec[ne] = encode(p, o2, q, ph);
            ep[ne] = p->mu[k] * occ[k] / Lam;
            total += ep[ne];
            ne++;
        }
        /* departure of host k: empties it */
        {
            int o2[OR_MAXH];
            memcpy(o2, occ, sizeof(int) * p->H);
            o2[k] = 0;
            ec[ne] = encode(p, o2, q, ph);
            ep[ne] = p->delta[k] / Lam;
            total += ep[ne];
            ne++;
        }
    }
    /* arrival: joins the queue, or is blocked (self-transition) when it is full */
    ec[ne] = (q < p->Q) ? encode(p, occ, q + 1, ph) : x;
    ep[ne] = p->lambda / Lam;
    total += ep[ne];
    ne++;
    /* phase flip */
    ec[ne] = encode(p, occ, q, 1 - ph);
    ep[ne] = (ph == 0 ? p->f : 1.0 - p->f) / Lam;
    total += ep[ne];
    ne++;
    /* self-loop: what is left */
    ec[ne] = x;
    ep[ne] = 1.0 - total;
    ne++;

    int n = 0;
    for (int e = 0; e < ne; e++) add_succ(cols, probs, &n, ec[e], ep[e]);
    /* drop exact zeros */
    int m = 0;
    for (int i = 0; i < n; i++) {
        if (probs[i] != 0.0) {
            cols[m] = cols[i];
            probs[m] = probs[i];
            m++;
        }
    }
    sort_succ(cols, probs, m);

    double occ_sum = 0.0, lost = 0.0;
    for (int k = 0; k < p->H; k++) {
        occ_sum += occ[k];
        lost += p->delta[k] * occ[k] / Lam;
    }
    if (q == p->Q) lost += p->lambda / Lam;
    *R = p->w_occ * occ_sum + p->w_q * q + p->w_loss * lost;
    return m;
}

/*
 * Derivatives of one transition row with respect to
 *   theta = (lambda, mu_0..mu_{H-1}, delta_0..delta_{H-1}, f, w_occ, w_loss, w_q),
 * nt = 2H+5 entries.  dprobs is n x nt (row-major, aligned with the merged, sorted
 * successor list that or_transitions returns for the same (s, a)); dR has nt entries.
 * Each event probability is rate/Lam, so d(rate/Lam) = drate/Lam - rate*dLam/Lam^2;
 * the self-loop takes minus the sum of the others.  Returns n, or -1 if infeasible.
 */
int or_transition_grads(const or_params* p, int64_t s, int a, int64_t* cols, double* dprobs, double* dR) {
    int occ[OR_MAXH] = {0}, q = 0, ph = 0;
    double probs_unused[OR_MAXSUCC], Rv;
    const int H = p->H, nt = 2 * H + 5;
    const int i_lam = 0, i_mu = 1, i_del = 1 + H, i_f = 1 + 2 * H;
    const int i_wocc = 2 + 2 * H, i_wloss = 3 + 2 * H, i_wq = 4 + 2 * H;

    int n = or_transitions(p, s, a, cols, probs_unused, &Rv);
    if (n < 0) return -1;
    decode(p, s, occ, &q, &ph);
    if (a < H) {
        occ[a] += 1;
        q -= 1;
    }
    const int64_t x = encode(p, occ, q, ph);
    const double Lam = or_uniformisation(p);
    double dLam[OR_NTHETA];
    for (int i = 0; i < nt; i++) dLam[i] = 0.0;
    dLam[i_lam] = 1.0;
    for (int k = 0; k < H; k++) {
        dLam[i_mu + k] = p->C;
        dLam[i_del + k] = 1.0;
    }

    /* unmerged events with rate and d(rate)/d(theta) */
    int64_t ec[OR_MAXSUCC];
    double er[OR_MAXSUCC];
    double edr[OR_MAXSUCC][OR_NTHETA];
    int ne = 0;
    memset(edr, 0, sizeof(edr));
    for (int k = 0; k < H; k++) {
        if (occ[k] > 0) {
            int o2[OR_MAXH];
            memcpy(o2, occ, sizeof(int) * H);
            o2[k] -= 1;
            ec[ne] = encode(p, o2, q, ph);
            er[ne] = p->mu[k] * occ[k];
            edr[ne][i_mu + k] = occ[k];
            ne++;
        }
        {
            int o2[OR_MAXH];
            memcpy(o2, occ, sizeof(int) * H);
            o2[k] = 0;
            ec[ne] = encode(p, o2, q, ph);
            er[ne] = p->delta[k];
            edr[ne][i_del + k] = 1.0;
            ne++;
        }
    }
    ec[ne] = (q < p->Q) ? encode(p, occ, q + 1, ph) : x;
    er[ne] = p->lambda;
    edr[ne][i_lam] = 1.0;
    ne++;
    ec[ne] = encode(p, occ, q, 1 - ph);
    er[ne] = (ph == 0) ? p->f : 1.0 - p->f;
    edr[ne][i_f] = (ph == 0) ? 1.0 : -1.0;
    ne++;

    for (int j = 0; j < n * nt; j++) dprobs[j] = 0.0;
    double dself[OR_NTHETA];
    for (int i = 0; i < nt; i++) dself[i] = 0.0;
    for (int e = 0; e < ne; e++) {
        int row = -1;
        for (int j = 0; j < n; j++)
            if (cols[j] == ec[e]) row = j;
        for (int i = 0; i < nt; i++) {
            double dp = edr[e][i] / Lam - er[e] * dLam[i] / (Lam * Lam);
            dself[i] -= dp;
            if (row >= 0) dprobs[row * nt + i] += dp;
        }
    }
    {
        int row = -1;
        for (int j = 0; j < n; j++)
            if (cols[j] == x) row = j;
        if (row >= 0)
            for (int i = 0; i < nt; i++) dprobs[row * nt + i] += dself[i];
    }

    /* reward derivatives */
    double occ_sum = 0.0, Lnum = 0.0;
    for (int k = 0; k < H; k++) {
        occ_sum += occ[k];
        Lnum += p->delta[k] * occ[k];
    }
    const int blocked = (q == p->Q);
    if (blocked) Lnum += p->lambda;
    for (int i = 0; i < nt; i++) dR[i] = 0.0;
    dR[i_wocc] = occ_sum;
    dR[i_wq] = q;
    dR[i_wloss] = Lnum / Lam;
    dR[i_lam] = p->w_loss * ((blocked ? 1.0 : 0.0) / Lam - Lnum / (Lam * Lam));
    for (int k = 0; k < H; k++) {
        dR[i_mu + k] = p->w_loss * (-Lnum * p->C / (Lam * Lam));
        dR[i_del + k] = p->w_loss * (occ[k] / Lam - Lnum / (Lam * Lam));
    }
    dR[i_f] = 0.0;
    return n;
}

/* ------------------------------------------------------------ explicit CSR form */

/*
 * Row r = s*A + a.  Canonical form (padded == 0): merged non-zero successors sorted by
 * column; infeasible rows are empty with R = -inf.  Padded form: every row holds exactly
 * 2H+3 entries: the successors, then probability-0 entries that repeat the row's last
 * column (so columns stay sorted); an infeasible row holds 2H+3 zeros at column s.
 * Returns nnz.  Pass NULL arrays to count only.
 */
int64_t or_build_csr(const or_params* p, int padded, int64_t* row_ptr, int32_t* col, double* val, double* R) {
    const int64_t S = or_num_states(p);
    const int A = p->H + 1;
    const int width = 2 * p->H + 3;
    int64_t nnz = 0;
    int64_t cols[OR_MAXSUCC];
    double probs[OR_MAXSUCC];
    if (row_ptr) row_ptr[0] = 0;
    for (int64_t s = 0; s < S; s++) {
        for (int a = 0; a < A; a++) {
            double Rv;
            int n = or_transitions(p, s, a, cols, probs, &Rv);
            int64_t r = s * A + a;
            if (n < 0) {
                if (R) R[r] = -INFINITY;
                if (padded) {
                    for (int j = 0; j < width; j++) {
                        if (col) col[nnz + j] = (int32_t)s;
                        if (val) val[nnz + j] = 0.0;
                    }
                    nnz += width;
                }
            } else {
                if (R) R[r] = Rv;
                for (int j = 0; j < n; j++) {
                    if (col) col[nnz + j] = (int32_t)cols[j];
                    if (val) val[nnz + j] = probs[j];
                }
                if (padded) {
                    for (int j = n; j < width; j++) {
                        if (col) col[nnz + j] = (int32_t)cols[n - 1];
                        if (val) val[nnz + j] = 0.0;
                    }
                    nnz += width;
                } else {
                    nnz += n;
                }
            }
            if (row_ptr) row_ptr[r + 1] = nnz;
        }
    }
    return nnz;
}

/* ------------------------------------------------------------- value iteration */

/* Q(s,a) = R(s,a) + gamma * sum_s' P(s'|s,a) V(s'); returns 0 and -inf if infeasible. */
static int q_value(const or_params* p, const double* V, int64_t s, int a, double* out) {
    int64_t cols[OR_MAXSUCC];
    double probs[OR_MAXSUCC], Rv;
    int n = or_transitions(p, s, a, cols, probs, &Rv);
    if (n < 0) {
        *out = -INFINITY;
        return 0;
    }
    double acc = 0.0;
    for (int j = 0; j < n; j++) acc += probs[j] * V[cols[j]];
    *out = Rv + p->gamma * acc;
    return 1;
}

/*
 * One Bellman backup of state s from V (Algorithm 3, step 2).  best = max over feasible
 * actions, arg = the lowest action attaining it, gap = best minus the second-largest
 * Q value (+inf when only one action is feasible).
 */
void or_backup(const or_params* p, const double* V, int64_t s, double* best, int32_t* arg, double* gap) {
    double b = -INFINITY, second = -INFINITY;
    int ba = -1;
    for (int a = 0; a <= p->H; a++) {
        double qv;
        if (!q_value(p, V, s, a, &qv)) continue;
        if (qv > b) {
            second = b;
            b = qv;
            ba = a;
        } else if (qv > second) {
            second = qv;
        }
    }
    *best = b;
    *arg = ba;
    *gap = (second == -INFINITY) ? INFINITY : b - second;
}

/*
 * Jacobi value iteration (Algorithm 3): V holds V^0 on entry (zeros for the paper's
 * step 1) and the last iterate on exit.  Stops after the first sweep with
 * max_s |V^{k+1}(s) - V^k(s)| < tol.  residuals (nullable, length max_sweeps) receives
 * every sweep's residual.  Returns 0 on convergence, 1 if max_sweeps ran out.
 */
int or_value_iteration(const or_params* p, double tol, int64_t max_sweeps, double* V, int64_t* sweeps_out,
                       double* residual_out, double* residuals) {
    const int64_t S = or_num_states(p);
    double* Vn = (double*)malloc(sizeof(double) * S);
    int64_t k = 0;
    double res = INFINITY;
    int status = 1;
    while (k < max_sweeps) {
        res = 0.0;
        for (int64_t s = 0; s < S; s++) {
            double b, g;
            int32_t a;
            or_backup(p, V, s, &b, &a, &g);
            Vn[s] = b;
            double d = fabs(Vn[s] - V[s]);
            if (d > res) res = d;
        }
        memcpy(V, Vn, sizeof(double) * S);
        if (residuals) residuals[k] = res;
        k++;
        if (res < tol) {
            status = 0;
            break;
        }
    }
    free(Vn);
    *sweeps_out = k;
    *residual_out = res;
    return status;
}

/* ----------------------------------- value iteration with self-transitions solved */

/*
 * Backup of state s with each action's own self-transition solved exactly: for a
 * feasible action a with P(s|s,a) = p_ss,
 *     Qs(s,a) = (R(s,a) + gamma * sum_{s' != s} P(s'|s,a) V(s')) / (1 - gamma * p_ss),
 * and the backup is the largest Qs.  This is the "Jacobi" value iteration of Puterman
 * (Markov Decision Processes, 1994, Sec. 6.3.3), and the in-block iteration of
 * Algorithm 4 taken to a block of a single state and iterated to its limit.  For each
 * action the map W -> R + gamma (p_ss W + rest) is affine with slope gamma p_ss < 1, so
 * the fixed point of their maximum is the maximum of their fixed points: Eq. 18's V*
 * is also the fixed point here, and at V* the same actions attain the maximum.
 */
static double sl_backup(const or_params* p, const double* V, int64_t s) {
    double b = -INFINITY;
    for (int a = 0; a <= p->H; a++) {
        int64_t cols[OR_MAXSUCC];
        double probs[OR_MAXSUCC], Rv;
        int n = or_transitions(p, s, a, cols, probs, &Rv);
        if (n < 0) continue;
        double off = 0.0, pss = 0.0;
        for (int j = 0; j < n; j++) {
            if (cols[j] == s)
                pss += probs[j];
            else
                off += probs[j] * V[cols[j]];
        }
        double qv = (Rv + p->gamma * off) / (1.0 - p->gamma * pss);
        if (qv > b) b = qv;
    }
    return b;
}

/*
 * Value iteration with sl_backup in place of Eq. 18's backup: Jacobi sweeps (every state
 * from the previous iterate) from V, stopping after the first sweep whose change
 * max_s |V^{k+1}(s) - V^k(s)| is below tol.  Same arguments and return value as
 * or_value_iteration.
 */
int or_value_iteration_sl(const or_params* p, double tol, int64_t max_sweeps, double* V, int64_t* sweeps_out,
                          double* residual_out, double* residuals) {
    const int64_t S = or_num_states(p);
    double* Vn = (double*)malloc(sizeof(double) * S);
    int64_t k = 0;
    double res = INFINITY;
    int status = 1;
    while (k < max_sweeps) {
        res = 0.0;
        for (int64_t s = 0; s < S; s++) {
            Vn[s] = sl_backup(p, V, s);
            double d = fabs(Vn[s] - V[s]);
            if (d > res) res = d;
        }
        memcpy(V, Vn, sizeof(double) * S);
        if (residuals) residuals[k] = res;
        k++;
        if (res < tol) {
            status = 0;
            break;
        }
    }
    free(Vn);
    *sweeps_out = k;
    *residual_out = res;
    return status;
}

/* Greedy policy of Algorithm 2 read on this MDP: place the head task on the feasible
 * host with the largest service rate (lowest index on ties), else defer. */
void or_greedy_policy(const or_params* p, int32_t* pi) {
    const int64_t S = or_num_states(p);
    for (int64_t s = 0; s < S; s++) {
        int best = p->H;
        double best_mu = -1.0;
        for (int a = 0; a < p->H; a++) {
            if (or_feasible(p, s, a) && p->mu[a] > best_mu) {
                best_mu = p->mu[a];
                best = a;
            }
        }
        pi[s] = best;
    }
}

/* Policy from V: pi(s) = argmax_a Q(s,a) (Algorithm 3, step 4), qgap as in or_backup. */
void or_policy(const or_params* p, const double* V, int32_t* pi, double* qgap) {
    const int64_t S = or_num_states(p);
    for (int64_t s = 0; s < S; s++) {
        double b, g;
        int32_t a;
        or_backup(p, V, s, &b, &a, &g);
        pi[s] = a;
        if (qgap) qgap[s] = g;
    }
}

/*
 * Backups of the states s0 .. s1-1 from V (Algorithm 3, steps 2 and 4 for a range of
 * states): Vn[s] (nullable) the best Q value, pi[s] (nullable) its lowest-index argmax,
 * gap[s] (nullable) the Q-gap, each state by or_backup.  Arrays are indexed like V, so
 * disjoint ranges can run on separate host threads.
 */
void or_backup_range(const or_params* p, const double* V, int64_t s0, int64_t s1, double* Vn, int32_t* pi,
                     double* gap) {
    for (int64_t s = s0; s < s1; s++) {
        double b, g;
        int32_t a;
        or_backup(p, V, s, &b, &a, &g);
        if (Vn) Vn[s] = b;
        if (pi) pi[s] = a;
        if (gap) gap[s] = g;
    }
}

/*
 * Policy evaluation by Jacobi iteration: V <- R_pi + gamma P_pi V until the sweep change
 * is below tol.  Returns 0 on convergence, 1 if max_sweeps ran out, 2 if pi is not
 * feasible somewhere.
 */
int or_policy_eval_iter(const or_params* p, const int32_t* pi, double tol, int64_t max_sweeps, double* V,
                        int64_t* sweeps_out) {
    const int64_t S = or_num_states(p);
    double* Vn = (double*)malloc(sizeof(double) * S);
    int64_t k = 0;
    int status = 1;
    while (k < max_sweeps) {
        double res = 0.0;
        for (int64_t s = 0; s < S; s++) {
            double qv;
            if (!q_value(p, V, s, pi[s], &qv)) {
                free(Vn);
                return 2;
            }
            Vn[s] = qv;
            double d = fabs(Vn[s] - V[s]);
            if (d > res) res = d;
        }
        memcpy(V, Vn, sizeof(double) * S);
        k++;
        if (res < tol) {
            status = 0;
            break;
        }
    }
    free(Vn);
    *sweeps_out = k;
    return status;
}

/* ------------------------------------------------------- generic explicit MDP */

/*
 * Jacobi value iteration on an explicit CSR MDP with S states and A actions per state:
 * row s*A+a spans [row_ptr[r], row_ptr[r+1]), R[r] = -inf marks an infeasible action.
 * Same stopping rule as or_value_iteration.  pi / qgap (nullable) receive the argmax
 * of the final backup.
 */
int or_vi_csr(int64_t S, int32_t A, const int64_t* row_ptr, const int32_t* col, const double* val,
              const double* R, double gamma, double tol, int64_t max_sweeps, double* V, int64_t* sweeps_out,
              double* residual_out) {
    double* Vn = (double*)malloc(sizeof(double) * S);
    int64_t k = 0;
    double res = INFINITY;
    int status = 1;
    while (k < max_sweeps) {
        res = 0.0;
        for (int64_t s = 0; s < S; s++) {
            double b = -INFINITY;
            for (int a = 0; a < A; a++) {
                int64_t r = s * A + a;
                if (R[r] == -INFINITY) continue;
                double acc = 0.0;
                for (int64_t j = row_ptr[r]; j < row_ptr[r + 1]; j++) acc += val[j] * V[col[j]];
                double qv = R[r] + gamma * acc;
                if (qv > b) b = qv;
            }
            Vn[s] = b;
            double d = fabs(Vn[s] - V[s]);
            if (d > res) res = d;
        }
        memcpy(V, Vn, sizeof(double) * S);
        k++;
        if (res < tol) {
            status = 0;
            break;
        }
    }
    free(Vn);
    *sweeps_out = k;
    *residual_out = res;
    return status;
}

/*
 * or_vi_csr with each row's self-transition solved exactly (the backup of sl_backup):
 * entries of row s*A+a whose column is s make up p_ss, the others the sum.
 */
int or_vi_csr_sl(int64_t S, int32_t A, const int64_t* row_ptr, const int32_t* col, const double* val,
                 const double* R, double gamma, double tol, int64_t max_sweeps, double* V, int64_t* sweeps_out,
                 double* residual_out) {
    double* Vn = (double*)malloc(sizeof(double) * S);
    int64_t k = 0;
    double res = INFINITY;
    int status = 1;
    while (k < max_sweeps) {
        res = 0.0;
        for (int64_t s = 0; s < S; s++) {
            double b = -INFINITY;
            for (int a = 0; a < A; a++) {
                int64_t r = s * A + a;
                if (R[r] == -INFINITY) continue;
                double off = 0.0, pss = 0.0;
                for (int64_t j = row_ptr[r]; j < row_ptr[r + 1]; j++) {
                    if (col[j] == s)
                        pss += val[j];
                    else
                        off += val[j] * V[col[j]];
                }
                double qv = (R[r] + gamma * off) / (1.0 - gamma * pss);
                if (qv > b) b = qv;
            }
            Vn[s] = b;
            double d = fabs(Vn[s] - V[s]);
            if (d > res) res = d;
        }
        memcpy(V, Vn, sizeof(double) * S);
        k++;
        if (res < tol) {
            status = 0;
            break;
        }
    }
    free(Vn);
    *sweeps_out = k;
    *residual_out = res;
    return status;
}

/*
 * Block iteration (Algorithm 4's in-block "episodes") on an explicit CSR MDP, with each
 * action's self-transition solved as in or_vi_csr_sl.  States are cut into consecutive
 * blocks of `tile` states.  In one global sweep every block runs `passes` local Jacobi
 * passes of the self-transition-solved backup: a successor inside the state's own block
 * takes the block's values from the previous local pass (the previous iterate in the first
 * pass), a successor outside it the previous global iterate.  passes = 1 is or_vi_csr_sl's
 * sweep; tile = 1 leaves only the state itself in its block, which the backup already
 * solves; one block of all S states with p passes is p sweeps of or_vi_csr_sl.  Stops
 * after the first global sweep whose change max_s |V^{k+1}(s) - V^k(s)| is below tol.
 */
int or_block_vi_csr_sl(int64_t S, int32_t A, const int64_t* row_ptr, const int32_t* col, const double* val,
                       const double* R, double gamma, int64_t tile, int32_t passes, double tol, int64_t max_sweeps,
                       double* V, int64_t* sweeps_out, double* residual_out) {
    double* Vold = (double*)malloc(sizeof(double) * S);
    double* W = (double*)malloc(sizeof(double) * S);
    double* Wn = (double*)malloc(sizeof(double) * S);
    int64_t k = 0;
    double res = INFINITY;
    int status = 1;
    if (tile < 1) tile = 1;
    if (passes < 1) passes = 1;
    while (k < max_sweeps) {
        memcpy(Vold, V, sizeof(double) * S);
        memcpy(W, V, sizeof(double) * S);
        for (int32_t pass = 0; pass < passes; pass++) {
            for (int64_t s = 0; s < S; s++) {
                const int64_t blk = s / tile;
                double b = -INFINITY;
                for (int a = 0; a < A; a++) {
                    int64_t r = s * A + a;
                    if (R[r] == -INFINITY) continue;
                    double off = 0.0, pss = 0.0;
                    for (int64_t j = row_ptr[r]; j < row_ptr[r + 1]; j++) {
                        const int64_t c = col[j];
                        if (c == s)
                            pss += val[j];
                        else
                            off += val[j] * (c / tile == blk ? W[c] : Vold[c]);
                    }
                    double qv = (R[r] + gamma * off) / (1.0 - gamma * pss);
                    if (qv > b) b = qv;
                }
                Wn[s] = b;
            }
            memcpy(W, Wn, sizeof(double) * S);
        }
        res = 0.0;
        for (int64_t s = 0; s < S; s++) {
            double d = fabs(W[s] - Vold[s]);
            if (d > res) res = d;
        }
        memcpy(V, W, sizeof(double) * S);
        k++;
        if (res < tol) {
            status = 0;
            break;
        }
    }
    free(Vold);
    free(W);
    free(Wn);
    *sweeps_out = k;
    *residual_out = res;
    return status;
}

void or_policy_csr(int64_t S, int32_t A, const int64_t* row_ptr, const int32_t* col, const double* val,
                   const double* R, double gamma, const double* V, int32_t* pi, double* qgap) {
    for (int64_t s = 0; s < S; s++) {
        double b = -INFINITY, second = -INFINITY;
        int ba = -1;
        for (int a = 0; a < A; a++) {
            int64_t r = s * A + a;
            if (R[r] == -INFINITY) continue;
            double acc = 0.0;
            for (int64_t j = row_ptr[r]; j < row_ptr[r + 1]; j++) acc += val[j] * V[col[j]];
            double qv = R[r] + gamma * acc;
            if (qv > b) {
                second = b;
                b = qv;
                ba = a;
            } else if (qv > second) {
                second = qv;
            }
        }
        pi[s] = ba;
        if (qgap) qgap[s] = (second == -INFINITY) ? INFINITY : b - second;
    }
}

/* ------------------------------------------------------------------- bfloat16 */

/*
 * Round a double to the nearest bfloat16 (8 exponent bits, 7 stored mantissa bits),
 * ties to even, directly from the double's bits (no intermediate float rounding).
 * Finite, non-negative inputs below the bf16 overflow threshold only (probabilities).
 * Returns the 16-bit pattern.
 */
uint16_t or_bf16_rne(double x) {
    if (x == 0.0) return 0;
    /* exact decomposition x = m * 2^e with m in [1, 2) */
    int e;
    double m = frexp(x, &e); /* m in [0.5, 1) */
    m *= 2.0;
    e -= 1;
    if (e < -126) {
        /* bf16 subnormal: value = k * 2^-133, k in [0, 127] */
        double k = ldexp(x, 133);
        double kr = nearbyint(k); /* default rounding mode: ties to even */
        return (uint16_t)kr;
    }
    /* normal: 7 fraction bits -> scale mantissa to [128, 256) and round */
    double t = ldexp(m, 7);
    double tr = nearbyint(t);
    if (tr == 256.0) {
        tr = 128.0;
        e += 1;
    }
    uint32_t frac = (uint32_t)tr - 128u;
    uint32_t bexp = (uint32_t)(e + 127);
    return (uint16_t)((bexp << 7) | frac);
}

double or_bf16_to_double(uint16_t b) {
    uint32_t exp = (b >> 7) & 0xFF;
    uint32_t frac = b & 0x7F;
    double sign = (b & 0x8000) ? -1.0 : 1.0;
    if (exp == 0) return sign * ldexp((double)frac, -133);
    return sign * ldexp(1.0 + frac / 128.0, (int)exp - 127);
}

/* Elementwise bf16 rounding of an array (bit patterns out). */
void or_bf16_round_array(int64_t n, const double* x, uint16_t* bits) {
    for (int64_t i = 0; i < n; i++) bits[i] = or_bf16_rne(x[i]);
}

/*
 * The matrix the BF16 storage form actually solves: each stored entry is bf16(p) and each
 * row is scaled by scale = 1 / sum_j bf16(p_j), the sum taken in FP64 in column order and
 * the reciprocal rounded to FP32.  Writes the bit patterns, the effective FP64 values
 * bf16(p_j) * scale and the FP32 scales (0 for an empty row).
 */
void or_bf16_renormalise_csr(int64_t nrows, const int64_t* row_ptr, const double* val, uint16_t* bits,
                             double* val_out, float* scale_out) {
    for (int64_t r = 0; r < nrows; r++) {
        double tot = 0.0;
        for (int64_t j = row_ptr[r]; j < row_ptr[r + 1]; j++) {
            bits[j] = or_bf16_rne(val[j]);
            tot += or_bf16_to_double(bits[j]);
        }
        float sc = (tot > 0.0) ? (float)(1.0 / tot) : 0.0f;
        scale_out[r] = sc;
        for (int64_t j = row_ptr[r]; j < row_ptr[r + 1]; j++) val_out[j] = or_bf16_to_double(bits[j]) * (double)sc;
    }
}

/*
 * One Jacobi backup (Algorithm 3, step 2) of the states s0, s0+step, ... < s1 from V into
 * Vn (Vn indexed like V).  Returns the number of successor terms summed (the logical
 * state-action-successor updates), used to time the oracle on a sample of a workload.
 */
int64_t or_sweep_states(const or_params* p, const double* V, double* Vn, int64_t s0, int64_t s1, int64_t step) {
    int64_t updates = 0;
    int64_t cols[OR_MAXSUCC];
    double probs[OR_MAXSUCC], Rv;
    for (int64_t s = s0; s < s1; s += step) {
        double b = -INFINITY;
        for (int a = 0; a <= p->H; a++) {
            int n = or_transitions(p, s, a, cols, probs, &Rv);
            if (n < 0) continue;
            double acc = 0.0;
            for (int j = 0; j < n; j++) acc += probs[j] * V[cols[j]];
            updates += n;
            double qv = Rv + p->gamma * acc;
            if (qv > b) b = qv;
        }
        Vn[s] = b;
    }
    return updates;
}

/*
 * Gradient contraction for a fixed policy: g_i = sum_s lam[s] * (dR(s,pi)/dtheta_i +
 * gamma * sum_j dP(j|s,pi)/dtheta_i * V[j]), theta as in or_transition_grads (2H+5
 * entries).  Returns 0, or 2 if pi is infeasible somewhere.
 */
int or_grad_contract(const or_params* p, const double* V, const int32_t* pi, const double* lam, double* g) {
    const int64_t S = or_num_states(p);
    const int nt = 2 * p->H + 5;
    int64_t cols[OR_MAXSUCC];
    double dprobs[OR_MAXSUCC * OR_NTHETA], dR[OR_NTHETA];
    for (int i = 0; i < nt; i++) g[i] = 0.0;
    for (int64_t s = 0; s < S; s++) {
        int n = or_transition_grads(p, s, pi[s], cols, dprobs, dR);
        if (n < 0) return 2;
        for (int i = 0; i < nt; i++) {
            double acc = 0.0;
            for (int j = 0; j < n; j++) acc += dprobs[j * nt + i] * V[cols[j]];
            g[i] += lam[s] * (dR[i] + p->gamma * acc);
        }
    }
    return 0;
}

/* out[y] = sum_s lam[s] * P(y | s, pi[s]): P_pi transposed applied to lam, by pushing
 * each row.  Returns 0, or 2 if pi is infeasible somewhere. */
int or_adjoint_apply(const or_params* p, const int32_t* pi, const double* lam, double* out) {
    const int64_t S = or_num_states(p);
    int64_t cols[OR_MAXSUCC];
    double probs[OR_MAXSUCC], Rv;
    for (int64_t y = 0; y < S; y++) out[y] = 0.0;
    for (int64_t s = 0; s < S; s++) {
        int n = or_transitions(p, s, pi[s], cols, probs, &Rv);
        if (n < 0) return 2;
        for (int j = 0; j < n; j++) out[cols[j]] += lam[s] * probs[j];
    }
    return 0;
}

/* =====================================================================================
 * The paper's binary-action model (Section V-B..V-E: state Eq. 10, actions A = {-1, 1}
 * of Eq. 11, reward r = k - g of Eqs. 14-16), with the transition law the paper leaves
 * open read as one uniformised event per step (the readings are in the design notes):
 *   state  s = e + E * sum_k u_k (C+1)^k,  E = 1 + H*J
 *          u_k in 0..C busy VMs of vehicular cloud k (Eq. 10's n_k), e the pending request:
 *          e = 0 none, e = 1 + i*J + (n-1) a task of n VMs (1 <= n <= J) asking VC i
 *   action index 0 = "-1": the task goes to the paid traditional cloud (TCC), always
 *          feasible; with no request it is the no-op (reward 0)
 *          index 1 = "+1": the task is placed on VC i, feasible iff a request is pending
 *          and u_i + n <= C
 *   reward index 1: beta_vc n - gamma_vc (C - u_i - n)       (k - g, free VMs after)
 *          index 0: -beta_tc n - gamma_vc (C - u_i)          (paid VMs, VC i stays idle)
 *   post-decision state: u (+ n on VC i for index 1), e = 0; then one event, rates over
 *          Lam = lambda + C sum(mu) + sum(delta) + 1:
 *          completion of one busy VM of VC k   mu_k u_k -> u_k - 1
 *          departure of VC k                   delta_k  -> u_k = 0 (self if u_k = 0)
 *          a request of n VMs at VC i          lambda / (H J) for each (i, n) -> e
 *          self-loop                           the rest
 * ===================================================================================== */

typedef struct {
    int32_t H, C, J, pad_;
    double lambda, gamma, beta_vc, beta_tc, gamma_vc;
    double mu[OR_MAXH];
    double delta[OR_MAXH];
} or_bin_params;

#define OR_BIN_MAXSUCC (2 * OR_MAXH + 2 + OR_MAXH * 8)

int64_t or_bin_num_states(const or_bin_params* p) {
    int64_t n = 1 + (int64_t)p->H * p->J;
    for (int k = 0; k < p->H; k++) n *= (p->C + 1);
    return n;
}

static void bin_decode(const or_bin_params* p, int64_t s, int* u, int* e) {
    const int64_t E = 1 + (int64_t)p->H * p->J;
    *e = (int)(s % E);
    int64_t rest = s / E;
    for (int k = 0; k < p->H; k++) {
        u[k] = (int)(rest % (p->C + 1));
        rest /= (p->C + 1);
    }
}

static int64_t bin_encode(const or_bin_params* p, const int* u, int e) {
    int64_t code = 0;
    for (int k = p->H - 1; k >= 0; k--) code = code * (p->C + 1) + u[k];
    return e + (1 + (int64_t)p->H * p->J) * code;
}

double or_bin_uniformisation(const or_bin_params* p) {
    double mu = 0.0, de = 0.0;
    for (int k = 0; k < p->H; k++) {
        mu += p->mu[k];
        de += p->delta[k];
    }
    return p->lambda + p->C * mu + de + 1.0;
}

/* Row of (s, a): merged successors sorted by target, zeros dropped, and the reward.
 * Returns the number of successors, or -1 if a is not feasible in s. */
int or_bin_transitions(const or_bin_params* p, int64_t s, int a, int64_t* cols, double* probs, double* R) {
    int u[OR_MAXH] = {0}, e = 0;
    bin_decode(p, s, u, &e);
    const int H = p->H, C = p->C, J = p->J;
    int vc = -1, n = 0;
    if (e > 0) {
        vc = (e - 1) / J;
        n = (e - 1) % J + 1;
    }
    if (a == 1) {
        if (e == 0 || u[vc] + n > C) return -1;
        u[vc] += n;
        *R = p->beta_vc * n - p->gamma_vc * (C - u[vc]);
    } else if (a == 0) {
        *R = (e == 0) ? 0.0 : -p->beta_tc * n - p->gamma_vc * (C - u[vc]);
    } else {
        return -1;
    }
    const int64_t x = bin_encode(p, u, 0);
    const double Lam = or_bin_uniformisation(p);

    int64_t ec[OR_BIN_MAXSUCC];
    double ep[OR_BIN_MAXSUCC];
    int ne = 0;
    double total = 0.0;
    for (int k = 0; k < H; k++) {
        if (u[k] > 0) {
            int u2[OR_MAXH];
            memcpy(u2, u, sizeof(int) * H);
            u2[k] -= 1;
            ec[ne] = bin_encode(p, u2, 0);
            ep[ne] = p->mu[k] * u[k] / Lam;
            total += ep[ne];
            ne++;
        }
        {
            int u2[OR_MAXH];
            memcpy(u2, u, sizeof(int) * H);
            u2[k] = 0;
            ec[ne] = bin_encode(p, u2, 0);
            ep[ne] = p->delta[k] / Lam;
            total += ep[ne];
            ne++;
        }
    }
    for (int i = 0; i < H; i++) {
        for (int m = 1; m <= J; m++) {
            ec[ne] = bin_encode(p, u, 1 + i * J + (m - 1));
            ep[ne] = p->lambda / (H * J) / Lam;
            total += ep[ne];
            ne++;
        }
    }
    ec[ne] = x;
    ep[ne] = 1.0 - total;
    ne++;

    int cnt = 0;
    for (int i = 0; i < ne; i++) add_succ(cols, probs, &cnt, ec[i], ep[i]);
    int m = 0;
    for (int i = 0; i < cnt; i++) {
        if (probs[i] != 0.0) {
            cols[m] = cols[i];
            probs[m] = probs[i];
            m++;
        }
    }
    sort_succ(cols, probs, m);
    return m;
}

/* CSR of the binary model (row r = 2 s + a); with NULL outputs returns the count only. */
int64_t or_bin_build_csr(const or_bin_params* p, int64_t* row_ptr, int32_t* col, double* val, double* R) {
    const int64_t S = or_bin_num_states(p);
    int64_t nnz = 0;
    int64_t cols[OR_BIN_MAXSUCC];
    double probs[OR_BIN_MAXSUCC];
    if (row_ptr) row_ptr[0] = 0;
    for (int64_t s = 0; s < S; s++) {
        for (int a = 0; a < 2; a++) {
            double Rv = 0.0;
            const int n = or_bin_transitions(p, s, a, cols, probs, &Rv);
            const int64_t r = 2 * s + a;
            if (R) R[r] = (n < 0) ? -INFINITY : Rv;
            for (int j = 0; j < n; j++) {
                if (col) col[nnz + j] = (int32_t)cols[j];
                if (val) val[nnz + j] = probs[j];
            }
            if (n > 0) nnz += n;
            if (row_ptr) row_ptr[r + 1] = nnz;
        }
    }
    return nnz;
}

/* Backups of the states s0 .. s1-1 of the binary-action model from V: Vn[s] the best Q
 * value, pi[s] its lowest-index argmax, gap[s] the Q-gap (+inf with one feasible action). */
void or_bin_backup_range(const or_bin_params* p, const double* V, int64_t s0, int64_t s1, double* Vn, int32_t* pi,
                         double* gap) {
    int64_t cols[OR_BIN_MAXSUCC];
    double probs[OR_BIN_MAXSUCC];
    for (int64_t s = s0; s < s1; s++) {
        double b = -INFINITY, second = -INFINITY;
        int ba = -1;
        for (int a = 0; a < 2; a++) {
            double Rv;
            const int n = or_bin_transitions(p, s, a, cols, probs, &Rv);
            if (n < 0) continue;
            double acc = 0.0;
            for (int j = 0; j < n; j++) acc += probs[j] * V[cols[j]];
            const double qv = Rv + p->gamma * acc;
            if (qv > b) {
                second = b;
                b = qv;
                ba = a;
            } else if (qv > second) {
                second = qv;
            }
        }
        Vn[s] = b;
        pi[s] = ba;
        gap[s] = (second == -INFINITY) ? INFINITY : b - second;
    }
}
