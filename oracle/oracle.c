/*
 * FP64 reference decoder for syndrome-based flooding sum-product belief
 * propagation (BP) on an LDPC / MET-LDPC Tanner graph.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA decoder is
 * checked against.  Only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it; the decoder never calls it, and
 * it shares no code, header or constant with the decoder.
 *
 * It follows the paper's Methods section ("Belief propagation decoding
 * algorithm of LDPC code", Steps 1-5, Eqs. 1-5) step by step, in the
 * log-likelihood-ratio (LLR) domain that the closing paragraph of that
 * section recommends, with these readings of points the paper leaves open:
 *
 *   - LLR convention: L = ln p(x=0)/p(x=1); for the BIAWGN observation
 *     y = (1-2x) + sigma z this is L = 2y/sigma^2.  The hard decision of
 *     Step 5 ("c_i = 1 iff q_i > 1" in the ratio q(1)/q(0)) is x = 1 iff L < 0,
 *     and L = 0 decides 0.
 *   - Eqs. 2-3 do not show Bob's syndrome although Step 1 sends it and Step 5
 *     compares against it: the check-to-variable message of check j carries
 *     the factor (1 - 2 s_j).
 *   - One iteration is a check update (Step 3) followed by a variable update
 *     (Step 4); the channel values feed the first check update.  The
 *     syndrome comparison (Step 5) happens after each iteration, so with
 *     early termination at least one iteration runs.
 *   - Clamps: channel LLRs, variable-to-check messages q and check-to-variable
 *     messages r are limited to [-LMAX, LMAX] (LMAX = 25 by default), and
 *     every argument of phi(x) = -ln tanh(x/2) is limited to
 *     [phi(LMAX), LMAX], the interval phi maps onto itself.  The posterior of
 *     Eq. 5 is not clamped.
 *   - Eq. 5 writes q_ij^0 where the channel term of VN i is meant.
 *
 * Per iteration (Eqs. 2-5 in the LLR domain, flooding schedule, full graph,
 * degree-1 VNs updated like every other VN):
 *   q_{v->c} = clamp( Lch(v) + sum_{c' in C_v \ c} r_{c'->v} )           (Eq. 4)
 *   r_{c->v} = clamp( (1-2 s_c) prod_{v' in R_c \ v} sgn q_{v'->c}
 *                     * phi( sum_{v' in R_c \ v} phi(|q_{v'->c}|) ) )     (Eqs. 2-3)
 *   L_v      = Lch(v) + sum_{c in C_v} r_{c->v},   xhat_v = [L_v < 0]    (Eq. 5)
 * The leave-one-out sums are formed directly over the other edges (no
 * total-minus-own shortcut).
 *
 * Also: weighted BP (a per-(iteration, edge type) scale on every
 * variable-to-check message) and its exact reverse-mode gradient, used to
 * check the decoder's adjoint.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

/* phi(x) = -ln tanh(x/2) = ln((e^x + 1)/(e^x - 1)) = log1p(2/expm1(x)), x > 0.
 * The last form keeps full relative precision at both ends of (0, inf). */
double oracle_phi(double x) { return log1p(2.0 / expm1(x)); }

static double clampd(double x, double lo, double hi) {
    return x < lo ? lo : (x > hi ? hi : x);
}

typedef struct {
    int32_t n_vn, n_cn;
    int64_t n_edges;
    const int32_t *edge_vn, *edge_cn;
    int64_t *cptr;   /* [n_cn+1]: edges of check c are cedge[cptr[c]..cptr[c+1]) */
    int64_t *cedge;
    int64_t *vptr;   /* [n_vn+1]: edges of VN v are vedge[vptr[v]..vptr[v+1]) */
    int64_t *vedge;
} adjacency;

static void adj_free(adjacency *a) {
    free(a->cptr); free(a->cedge); free(a->vptr); free(a->vedge);
}

static int adj_build(adjacency *a, int32_t n_vn, int32_t n_cn, int64_t n_edges,
                     const int32_t *edge_vn, const int32_t *edge_cn) {
    memset(a, 0, sizeof *a);
    a->n_vn = n_vn; a->n_cn = n_cn; a->n_edges = n_edges;
    a->edge_vn = edge_vn; a->edge_cn = edge_cn;
    for (int64_t e = 0; e < n_edges; ++e)
        if (edge_vn[e] < 0 || edge_vn[e] >= n_vn || edge_cn[e] < 0 || edge_cn[e] >= n_cn)
            return ORACLE_EINVAL;
    a->cptr = calloc((size_t)n_cn + 1, sizeof(int64_t));
    a->vptr = calloc((size_t)n_vn + 1, sizeof(int64_t));
    a->cedge = malloc(sizeof(int64_t) * (size_t)(n_edges > 0 ? n_edges : 1));
    a->vedge = malloc(sizeof(int64_t) * (size_t)(n_edges > 0 ? n_edges : 1));
    if (!a->cptr || !a->vptr || !a->cedge || !a->vedge) { adj_free(a); return ORACLE_ENOMEM; }
    for (int64_t e = 0; e < n_edges; ++e) { a->cptr[edge_cn[e] + 1]++; a->vptr[edge_vn[e] + 1]++; }
    for (int32_t c = 0; c < n_cn; ++c) a->cptr[c + 1] += a->cptr[c];
    for (int32_t v = 0; v < n_vn; ++v) a->vptr[v + 1] += a->vptr[v];
    int64_t *cfill = malloc(sizeof(int64_t) * ((size_t)n_cn + 1));
    int64_t *vfill = malloc(sizeof(int64_t) * ((size_t)n_vn + 1));
    if (!cfill || !vfill) { free(cfill); free(vfill); adj_free(a); return ORACLE_ENOMEM; }
    memcpy(cfill, a->cptr, sizeof(int64_t) * ((size_t)n_cn + 1));
    memcpy(vfill, a->vptr, sizeof(int64_t) * ((size_t)n_vn + 1));
    for (int64_t e = 0; e < n_edges; ++e) {
        a->cedge[cfill[edge_cn[e]]++] = e;
        a->vedge[vfill[edge_vn[e]]++] = e;
    }
    free(cfill); free(vfill);
    return ORACLE_OK;
}

/* Step 5: does the hard decision satisfy every check, H xhat = s (mod 2)? */
static int syndrome_ok(const adjacency *a, const uint8_t *xhat, const uint8_t *s) {
    for (int32_t c = 0; c < a->n_cn; ++c) {
        int parity = s[c] & 1;
        for (int64_t k = a->cptr[c]; k < a->cptr[c + 1]; ++k)
            parity ^= xhat[a->edge_vn[a->cedge[k]]];
        if (parity) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Plain BP, one codeword.                                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    const adjacency *a;
    const double *llr;       /* [batch][n_vn] */
    const uint8_t *syn;      /* [batch][n_cn] */
    int32_t batch, max_iters, early_term;
    double lmax;
    double *post;            /* [batch][n_vn] or NULL */
    uint8_t *bits;           /* [batch][n_vn] */
    uint8_t *converged;      /* [batch] */
    int32_t *iters_used;     /* [batch] */
    int next;                /* work counter (atomic) */
    int status;
    const int32_t *order;    /* layered schedule: the check order [n_cn] */
    double ms_offset;        /* offset min-sum: the offset subtracted from the minimum */
} decode_job;

static int decode_one(const decode_job *J, int b) {
    const adjacency *a = J->a;
    const int32_t n = a->n_vn;
    const int64_t E = a->n_edges;
    const double lmax = J->lmax;
    const double amin = oracle_phi(lmax);     /* phi maps [amin, lmax] onto itself */
    const double *llr = J->llr + (size_t)b * n;
    const uint8_t *s = J->syn + (size_t)b * a->n_cn;
    double *Lch = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *L = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *q = malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
    double *r = malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
    double *phiq = malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
    uint8_t *xhat = malloc((size_t)(n > 0 ? n : 1));
    if (!Lch || !L || !q || !r || !phiq || !xhat) {
        free(Lch); free(L); free(q); free(r); free(phiq); free(xhat);
        return ORACLE_ENOMEM;
    }
    /* Step 2 / Eq. 1: channel values; no check message has been sent yet. */
    for (int32_t v = 0; v < n; ++v) {
        Lch[v] = clampd(llr[v], -lmax, lmax);
        L[v] = Lch[v];
        xhat[v] = L[v] < 0.0;
    }
    for (int64_t e = 0; e < E; ++e) r[e] = 0.0;

    int used = 0, conv = 0;
    for (int l = 1; l <= J->max_iters; ++l) {
        /* Eq. 4: variable-to-check messages from the previous iteration's r. */
        for (int32_t v = 0; v < n; ++v) {
            for (int64_t k = a->vptr[v]; k < a->vptr[v + 1]; ++k) {
                double acc = Lch[v];
                for (int64_t k2 = a->vptr[v]; k2 < a->vptr[v + 1]; ++k2)
                    if (k2 != k) acc += r[a->vedge[k2]];
                q[a->vedge[k]] = clampd(acc, -lmax, lmax);
            }
        }
        /* Eqs. 2-3 with the syndrome sign: check-to-variable messages. */
        for (int64_t e = 0; e < E; ++e) phiq[e] = oracle_phi(clampd(fabs(q[e]), amin, lmax));
        for (int32_t c = 0; c < a->n_cn; ++c) {
            for (int64_t k = a->cptr[c]; k < a->cptr[c + 1]; ++k) {
                double sgn = (s[c] & 1) ? -1.0 : 1.0;
                double sum = 0.0;
                for (int64_t k2 = a->cptr[c]; k2 < a->cptr[c + 1]; ++k2) {
                    if (k2 == k) continue;
                    int64_t e2 = a->cedge[k2];
                    if (q[e2] < 0.0) sgn = -sgn;
                    sum += phiq[e2];
                }
                double mag = oracle_phi(clampd(sum, amin, lmax));
                r[a->cedge[k]] = clampd(sgn * mag, -lmax, lmax);
            }
        }
        /* Eq. 5: posterior and hard decision. */
        for (int32_t v = 0; v < n; ++v) {
            double acc = Lch[v];
            for (int64_t k = a->vptr[v]; k < a->vptr[v + 1]; ++k) acc += r[a->vedge[k]];
            L[v] = acc;
            xhat[v] = acc < 0.0;
        }
        used = l;
        /* Step 5: stop on a syndrome match when early termination is on. */
        if (J->early_term && syndrome_ok(a, xhat, s)) { conv = 1; break; }
    }
    if (!conv) conv = syndrome_ok(a, xhat, s);
    if (J->post) memcpy(J->post + (size_t)b * n, L, sizeof(double) * (size_t)n);
    memcpy(J->bits + (size_t)b * n, xhat, (size_t)n);
    J->converged[b] = (uint8_t)conv;
    J->iters_used[b] = used;
    free(Lch); free(L); free(q); free(r); free(phiq); free(xhat);
    return ORACLE_OK;
}

static void *decode_worker(void *arg) {
    decode_job *J = arg;
    for (;;) {
        int b = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (b >= J->batch) break;
        int st = decode_one(J, b);
        if (st != ORACLE_OK) __atomic_store_n(&J->status, st, __ATOMIC_RELAXED);
    }
    return NULL;
}

static int run_workers(void *(*fn)(void *), void *job, int32_t n_threads, int32_t batch) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > batch) n_threads = batch;
    if (n_threads <= 1) { fn(job); return ORACLE_OK; }
    pthread_t *th = malloc(sizeof(pthread_t) * (size_t)n_threads);
    if (!th) return ORACLE_ENOMEM;
    int started = 0;
    for (int i = 0; i < n_threads; ++i) {
        if (pthread_create(&th[i], NULL, fn, job) != 0) break;
        ++started;
    }
    if (started == 0) fn(job);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    free(th);
    return ORACLE_OK;
}

int oracle_decode(int32_t n_vn, int32_t n_cn, int64_t n_edges,
                  const int32_t *edge_vn, const int32_t *edge_cn,
                  int32_t batch, const double *llr, const uint8_t *syndrome,
                  int32_t max_iters, int32_t early_term, double lmax,
                  double *post, uint8_t *bits, uint8_t *converged,
                  int32_t *iters_used, int32_t n_threads) {
    if (n_vn < 0 || n_cn < 0 || n_edges < 0 || batch < 0 || max_iters < 0 || !(lmax > 0.0))
        return ORACLE_EINVAL;
    if (batch == 0) return ORACLE_OK;
    if (!llr || !syndrome || !bits || !converged || !iters_used) return ORACLE_EINVAL;
    adjacency a;
    int st = adj_build(&a, n_vn, n_cn, n_edges, edge_vn, edge_cn);
    if (st != ORACLE_OK) return st;
    decode_job J = {&a, llr, syndrome, batch, max_iters, early_term, lmax,
                    post, bits, converged, iters_used, 0, ORACLE_OK, NULL, 0.0};
    st = run_workers(decode_worker, &J, n_threads, batch);
    adj_free(&a);
    return st != ORACLE_OK ? st : J.status;
}

/* ------------------------------------------------------------------------- */
/* Layered (serial) schedule, one codeword.                                   */
/*                                                                           */
/* The checks are updated one at a time in the order `order`; each check      */
/* forms its incoming messages from the latest outgoing messages of the other */
/* checks (those already updated in this iteration included), then replaces   */
/* its own outgoing messages.  For check c, in order:                         */
/*   q_{v->c} = clamp( Lch(v) + sum_{c' in C_v \ c} r_{c'->v} )  (Eq. 4)      */
/*   r_{c->v} = clamp( (1-2 s_c) prod_{v' in R_c \ v} sgn q_{v'->c}           */
/*                     * phi( sum_{v' in R_c \ v} phi(|q_{v'->c}|) ) )        */
/*                                                            (Eqs. 2-3)     */
/* with the clamps and readings of the flooding decoder above.  After every  */
/* check has been updated once (one iteration), the posterior and decision   */
/* of Eq. 5 and the syndrome comparison of Step 5 follow as in flooding.     */
/* The schedule is not in the paper, which runs the flooding schedule of     */
/* Steps 3-4; it reorders the same Steps 3-4 per check.                      */
/* ------------------------------------------------------------------------- */
static int decode_one_layered(const decode_job *J, int b) {
    const adjacency *a = J->a;
    const int32_t n = a->n_vn;
    const int64_t E = a->n_edges;
    const double lmax = J->lmax;
    const double amin = oracle_phi(lmax);
    const double *llr = J->llr + (size_t)b * n;
    const uint8_t *s = J->syn + (size_t)b * a->n_cn;
    double *Lch = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *L = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *q = malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
    double *r = malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
    double *phiq = malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
    uint8_t *xhat = malloc((size_t)(n > 0 ? n : 1));
    if (!Lch || !L || !q || !r || !phiq || !xhat) {
        free(Lch); free(L); free(q); free(r); free(phiq); free(xhat);
        return ORACLE_ENOMEM;
    }
    for (int32_t v = 0; v < n; ++v) {
        Lch[v] = clampd(llr[v], -lmax, lmax);
        L[v] = Lch[v];
        xhat[v] = L[v] < 0.0;
    }
    for (int64_t e = 0; e < E; ++e) r[e] = 0.0;

    int used = 0, conv = 0;
    for (int l = 1; l <= J->max_iters; ++l) {
        for (int32_t k = 0; k < a->n_cn; ++k) {
            const int32_t c = J->order[k];
            /* Eq. 4 for the edges of c, from the current messages */
            for (int64_t k1 = a->cptr[c]; k1 < a->cptr[c + 1]; ++k1) {
                const int64_t e = a->cedge[k1];
                const int32_t v = a->edge_vn[e];
                double acc = Lch[v];
                for (int64_t k2 = a->vptr[v]; k2 < a->vptr[v + 1]; ++k2)
                    if (a->vedge[k2] != e) acc += r[a->vedge[k2]];
                q[e] = clampd(acc, -lmax, lmax);
                phiq[e] = oracle_phi(clampd(fabs(q[e]), amin, lmax));
            }
            /* Eqs. 2-3 with the syndrome sign for the edges of c */
            for (int64_t k1 = a->cptr[c]; k1 < a->cptr[c + 1]; ++k1) {
                double sgn = (s[c] & 1) ? -1.0 : 1.0;
                double sum = 0.0;
                for (int64_t k2 = a->cptr[c]; k2 < a->cptr[c + 1]; ++k2) {
                    if (k2 == k1) continue;
                    const int64_t e2 = a->cedge[k2];
                    if (q[e2] < 0.0) sgn = -sgn;
                    sum += phiq[e2];
                }
                r[a->cedge[k1]] = clampd(sgn * oracle_phi(clampd(sum, amin, lmax)), -lmax, lmax);
            }
        }
        /* Eq. 5: posterior and hard decision */
        for (int32_t v = 0; v < n; ++v) {
            double acc = Lch[v];
            for (int64_t k = a->vptr[v]; k < a->vptr[v + 1]; ++k) acc += r[a->vedge[k]];
            L[v] = acc;
            xhat[v] = acc < 0.0;
        }
        used = l;
        if (J->early_term && syndrome_ok(a, xhat, s)) { conv = 1; break; }
    }
    if (!conv) conv = syndrome_ok(a, xhat, s);
    if (J->post) memcpy(J->post + (size_t)b * n, L, sizeof(double) * (size_t)n);
    memcpy(J->bits + (size_t)b * n, xhat, (size_t)n);
    J->converged[b] = (uint8_t)conv;
    J->iters_used[b] = used;
    free(Lch); free(L); free(q); free(r); free(phiq); free(xhat);
    return ORACLE_OK;
}

static void *decode_layered_worker(void *arg) {
    decode_job *J = arg;
    for (;;) {
        int b = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (b >= J->batch) break;
        int st = decode_one_layered(J, b);
        if (st != ORACLE_OK) __atomic_store_n(&J->status, st, __ATOMIC_RELAXED);
    }
    return NULL;
}

/* Layered decoding; `order` lists every check exactly once. */
int oracle_decode_layered(int32_t n_vn, int32_t n_cn, int64_t n_edges,
                          const int32_t *edge_vn, const int32_t *edge_cn, const int32_t *order,
                          int32_t batch, const double *llr, const uint8_t *syndrome,
                          int32_t max_iters, int32_t early_term, double lmax,
                          double *post, uint8_t *bits, uint8_t *converged,
                          int32_t *iters_used, int32_t n_threads) {
    if (n_vn < 0 || n_cn < 0 || n_edges < 0 || batch < 0 || max_iters < 0 || !(lmax > 0.0))
        return ORACLE_EINVAL;
    if (batch == 0) return ORACLE_OK;
    if (!llr || !syndrome || !bits || !converged || !iters_used || (n_cn > 0 && !order))
        return ORACLE_EINVAL;
    uint8_t *seen = calloc((size_t)n_cn + 1, 1);
    if (!seen) return ORACLE_ENOMEM;
    for (int32_t k = 0; k < n_cn; ++k) {
        if (order[k] < 0 || order[k] >= n_cn || seen[order[k]]) { free(seen); return ORACLE_EINVAL; }
        seen[order[k]] = 1;
    }
    free(seen);
    adjacency a;
    int st = adj_build(&a, n_vn, n_cn, n_edges, edge_vn, edge_cn);
    if (st != ORACLE_OK) return st;
    decode_job J = {&a, llr, syndrome, batch, max_iters, early_term, lmax,
                    post, bits, converged, iters_used, 0, ORACLE_OK, order, 0.0};
    st = run_workers(decode_layered_worker, &J, n_threads, batch);
    adj_free(&a);
    return st != ORACLE_OK ? st : J.status;
}

/* ------------------------------------------------------------------------- */
/* Offset min-sum, one codeword (flooding schedule).                          */
/*                                                                           */
/* The approximation of the check update that keeps the sign rule of Eqs. 2-3 */
/* and replaces the magnitude phi(sum phi(|q|)) by the smallest magnitude     */
/* among the other incoming messages, reduced by an offset and floored at 0:  */
/*   r_{c->v} = (1-2 s_c) prod_{v' in R_c \ v} sgn q_{v'->c}                  */
/*              * max( min_{v' in R_c \ v} |q_{v'->c}| - offset, 0 )          */
/* (the paper's closing remark on simplifying the check update in the LLR     */
/* domain; the offset is a parameter).  Everything else (clamps, Eq. 4,       */
/* Eq. 5, Step 5) is as in the sum-product decoder above.                     */
/* ------------------------------------------------------------------------- */
static int decode_one_ms(const decode_job *J, int b) {
    const adjacency *a = J->a;
    const int32_t n = a->n_vn;
    const int64_t E = a->n_edges;
    const double lmax = J->lmax;
    const double *llr = J->llr + (size_t)b * n;
    const uint8_t *s = J->syn + (size_t)b * a->n_cn;
    double *Lch = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *L = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *q = malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
    double *r = malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
    uint8_t *xhat = malloc((size_t)(n > 0 ? n : 1));
    if (!Lch || !L || !q || !r || !xhat) {
        free(Lch); free(L); free(q); free(r); free(xhat);
        return ORACLE_ENOMEM;
    }
    for (int32_t v = 0; v < n; ++v) {
        Lch[v] = clampd(llr[v], -lmax, lmax);
        L[v] = Lch[v];
        xhat[v] = L[v] < 0.0;
    }
    for (int64_t e = 0; e < E; ++e) r[e] = 0.0;
    int used = 0, conv = 0;
    for (int l = 1; l <= J->max_iters; ++l) {
        /* Eq. 4 */
        for (int32_t v = 0; v < n; ++v)
            for (int64_t k = a->vptr[v]; k < a->vptr[v + 1]; ++k) {
                double acc = Lch[v];
                for (int64_t k2 = a->vptr[v]; k2 < a->vptr[v + 1]; ++k2)
                    if (k2 != k) acc += r[a->vedge[k2]];
                q[a->vedge[k]] = clampd(acc, -lmax, lmax);
            }
        /* offset min-sum check update */
        for (int32_t c = 0; c < a->n_cn; ++c)
            for (int64_t k = a->cptr[c]; k < a->cptr[c + 1]; ++k) {
                double sgn = (s[c] & 1) ? -1.0 : 1.0;
                double mn = lmax;   /* |q| <= lmax: the minimum of an empty set is lmax */
                for (int64_t k2 = a->cptr[c]; k2 < a->cptr[c + 1]; ++k2) {
                    if (k2 == k) continue;
                    const double qe = q[a->cedge[k2]];
                    if (qe < 0.0) sgn = -sgn;
                    if (fabs(qe) < mn) mn = fabs(qe);
                }
                const double mag = mn - J->ms_offset > 0.0 ? mn - J->ms_offset : 0.0;
                r[a->cedge[k]] = sgn * mag;
            }
        /* Eq. 5 */
        for (int32_t v = 0; v < n; ++v) {
            double acc = Lch[v];
            for (int64_t k = a->vptr[v]; k < a->vptr[v + 1]; ++k) acc += r[a->vedge[k]];
            L[v] = acc;
            xhat[v] = acc < 0.0;
        }
        used = l;
        if (J->early_term && syndrome_ok(a, xhat, s)) { conv = 1; break; }
    }
    if (!conv) conv = syndrome_ok(a, xhat, s);
    if (J->post) memcpy(J->post + (size_t)b * n, L, sizeof(double) * (size_t)n);
    memcpy(J->bits + (size_t)b * n, xhat, (size_t)n);
    J->converged[b] = (uint8_t)conv;
    J->iters_used[b] = used;
    free(Lch); free(L); free(q); free(r); free(xhat);
    return ORACLE_OK;
}

static void *decode_ms_worker(void *arg) {
    decode_job *J = arg;
    for (;;) {
        int b = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (b >= J->batch) break;
        int st = decode_one_ms(J, b);
        if (st != ORACLE_OK) __atomic_store_n(&J->status, st, __ATOMIC_RELAXED);
    }
    return NULL;
}

int oracle_decode_ms(int32_t n_vn, int32_t n_cn, int64_t n_edges,
                     const int32_t *edge_vn, const int32_t *edge_cn, double offset,
                     int32_t batch, const double *llr, const uint8_t *syndrome,
                     int32_t max_iters, int32_t early_term, double lmax,
                     double *post, uint8_t *bits, uint8_t *converged,
                     int32_t *iters_used, int32_t n_threads) {
    if (n_vn < 0 || n_cn < 0 || n_edges < 0 || batch < 0 || max_iters < 0 || !(lmax > 0.0) || !(offset >= 0.0))
        return ORACLE_EINVAL;
    if (batch == 0) return ORACLE_OK;
    if (!llr || !syndrome || !bits || !converged || !iters_used) return ORACLE_EINVAL;
    adjacency a;
    int st = adj_build(&a, n_vn, n_cn, n_edges, edge_vn, edge_cn);
    if (st != ORACLE_OK) return st;
    decode_job J = {&a, llr, syndrome, batch, max_iters, early_term, lmax,
                    post, bits, converged, iters_used, 0, ORACLE_OK, NULL, offset};
    st = run_workers(decode_ms_worker, &J, n_threads, batch);
    adj_free(&a);
    return st != ORACLE_OK ? st : J.status;
}

/* Check H xhat = s for a batch of hard decisions (uint8 0/1 per bit). */
int oracle_syndrome_ok(int32_t n_vn, int32_t n_cn, int64_t n_edges,
                       const int32_t *edge_vn, const int32_t *edge_cn,
                       int32_t batch, const uint8_t *bits, const uint8_t *syndrome,
                       uint8_t *ok) {
    adjacency a;
    int st = adj_build(&a, n_vn, n_cn, n_edges, edge_vn, edge_cn);
    if (st != ORACLE_OK) return st;
    for (int32_t b = 0; b < batch; ++b)
        ok[b] = (uint8_t)syndrome_ok(&a, bits + (size_t)b * n_vn, syndrome + (size_t)b * n_cn);
    adj_free(&a);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* Weighted BP and its exact gradient (reverse mode, full history).           */
/*                                                                           */
/* Weighted BP scales each variable-to-check message by a weight that depends */
/* on the iteration t and on the edge's type tau(e):                          */
/*   x_e^t = Lch(v) + sum_{c' in C_v \ c} r_{c'->v}^{t-1}                     */
/*   q_e^t = clamp(w[t][tau(e)] * x_e^t)                                      */
/*   r_e^t = check update of the q^t as in plain BP (Eqs. 2-3, syndrome sign) */
/*   L_v   = Lch(v) + sum_{c in C_v} r^T                                       */
/*   loss  = mean_{b,v} softplus(-(1 - 2 x_v) L_v)                            */
/* All weights equal to 1 is plain BP.  Derivatives of the clamps are 1      */
/* strictly inside and 0 outside; the sign factors have derivative 0;         */
/* phi'(x) = -1/sinh(x).                                                       */
/* ------------------------------------------------------------------------- */

static double softplus(double z) { return z > 0 ? z + log1p(exp(-z)) : log1p(exp(z)); }
static double sigmoid(double z) { return z >= 0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z)); }

typedef struct {
    const adjacency *a;
    const uint8_t *etype;  /* [E] */
    int32_t n_types;
    const double *llr;     /* [B][n] */
    const uint8_t *syn;    /* [B][m] */
    const uint8_t *xbits;  /* [B][n] */
    int32_t batch, T;
    const double *w;       /* [T][n_types] */
    double lmax;
    double *loss;          /* [B]: per-codeword sum of softplus terms */
    double *post;          /* [B][n] */
    double *dw;            /* [B][T][n_types] per-codeword partial */
    double *dllr;          /* [B][n] */
    int next, status;
} wbp_job;

static int wbp_one(const wbp_job *J, int b) {
    const adjacency *a = J->a;
    const int32_t n = a->n_vn;
    const int64_t E = a->n_edges;
    const int T = J->T, NT = J->n_types;
    const double lmax = J->lmax, amin = oracle_phi(lmax);
    const double *llr = J->llr + (size_t)b * n;
    const uint8_t *s = J->syn + (size_t)b * a->n_cn;
    const uint8_t *xb = J->xbits + (size_t)b * n;
    const size_t Es = (size_t)(E > 0 ? E : 1);
    double *Lch = calloc((size_t)n + 1, sizeof(double));
    double *gLch = calloc((size_t)n + 1, sizeof(double));
    double *r = calloc(Es * (size_t)(T + 1), sizeof(double));   /* r[t][e], r[0] = 0 */
    double *x = calloc(Es * (size_t)(T + 1), sizeof(double));   /* x[t][e] */
    double *gr = calloc(Es, sizeof(double));                     /* dloss/dr^t */
    double *gx = calloc(Es, sizeof(double));
    double *q = calloc(Es, sizeof(double)), *f = calloc(Es, sizeof(double));
    double *go = calloc(Es, sizeof(double));
    double *dw = J->dw + (size_t)b * T * NT;
    if (!Lch || !gLch || !r || !x || !gr || !gx || !q || !f || !go) {
        free(Lch); free(gLch); free(r); free(x); free(gr); free(gx); free(q); free(f); free(go);
        return ORACLE_ENOMEM;
    }
    for (int32_t v = 0; v < n; ++v) Lch[v] = clampd(llr[v], -lmax, lmax);

    /* forward, keeping x^t and r^t for every iteration */
    for (int t = 1; t <= T; ++t) {
        double *rp = r + (size_t)(t - 1) * Es, *rt = r + (size_t)t * Es, *xt = x + (size_t)t * Es;
        for (int32_t v = 0; v < n; ++v)
            for (int64_t k = a->vptr[v]; k < a->vptr[v + 1]; ++k) {
                double acc = Lch[v];
                for (int64_t k2 = a->vptr[v]; k2 < a->vptr[v + 1]; ++k2)
                    if (k2 != k) acc += rp[a->vedge[k2]];
                xt[a->vedge[k]] = acc;
            }
        for (int64_t e = 0; e < E; ++e) {
            q[e] = clampd(J->w[(size_t)(t - 1) * NT + J->etype[e]] * xt[e], -lmax, lmax);
            f[e] = oracle_phi(clampd(fabs(q[e]), amin, lmax));
        }
        for (int32_t c = 0; c < a->n_cn; ++c)
            for (int64_t k = a->cptr[c]; k < a->cptr[c + 1]; ++k) {
                double sgn = (s[c] & 1) ? -1.0 : 1.0, sum = 0.0;
                for (int64_t k2 = a->cptr[c]; k2 < a->cptr[c + 1]; ++k2) {
                    if (k2 == k) continue;
                    if (q[a->cedge[k2]] < 0.0) sgn = -sgn;
                    sum += f[a->cedge[k2]];
                }
                rt[a->cedge[k]] = clampd(sgn * oracle_phi(clampd(sum, amin, lmax)), -lmax, lmax);
            }
    }
    double lsum = 0.0;
    for (int32_t v = 0; v < n; ++v) {
        double L = Lch[v];
        for (int64_t k = a->vptr[v]; k < a->vptr[v + 1]; ++k) L += r[(size_t)T * Es + a->vedge[k]];
        if (J->post) J->post[(size_t)b * n + v] = L;
        const double y = 1.0 - 2.0 * (xb[v] & 1);
        lsum += softplus(-y * L);
        /* d softplus(-yL)/dL = -y sigmoid(-yL); the loss is a mean over B*n */
        const double g = -y * sigmoid(-y * L) / ((double)J->batch * (double)n);
        gLch[v] += g;
        for (int64_t k = a->vptr[v]; k < a->vptr[v + 1]; ++k) gr[a->vedge[k]] = g;
    }
    J->loss[b] = lsum;

    /* reverse sweep */
    for (int t = T; t >= 1; --t) {
        const double *rp = r + (size_t)(t - 1) * Es, *xt = x + (size_t)t * Es;
        (void)rp;
        for (int64_t e = 0; e < E; ++e) {
            q[e] = clampd(J->w[(size_t)(t - 1) * NT + J->etype[e]] * xt[e], -lmax, lmax);
            f[e] = oracle_phi(clampd(fabs(q[e]), amin, lmax));
        }
        /* r_e = sgn_e * phi(clamp(o_e)), o_e = sum of the other f */
        for (int32_t c = 0; c < a->n_cn; ++c)
            for (int64_t k = a->cptr[c]; k < a->cptr[c + 1]; ++k) {
                const int64_t e = a->cedge[k];
                double sgn = (s[c] & 1) ? -1.0 : 1.0, o = 0.0;
                for (int64_t k2 = a->cptr[c]; k2 < a->cptr[c + 1]; ++k2) {
                    if (k2 == k) continue;
                    if (q[a->cedge[k2]] < 0.0) sgn = -sgn;
                    o += f[a->cedge[k2]];
                }
                /* |r| = phi(clamp(o)) <= lmax: the outer clamp never binds */
                go[e] = (o > amin && o < lmax) ? sgn * gr[e] * (-1.0 / sinh(o)) : 0.0;
            }
        for (int64_t e = 0; e < E; ++e) gx[e] = 0.0;
        for (int32_t c = 0; c < a->n_cn; ++c)
            for (int64_t k = a->cptr[c]; k < a->cptr[c + 1]; ++k) {
                const int64_t e = a->cedge[k];
                double gf = 0.0;
                for (int64_t k2 = a->cptr[c]; k2 < a->cptr[c + 1]; ++k2)
                    if (k2 != k) gf += go[a->cedge[k2]];
                const double aq = fabs(q[e]);
                const double ga = (aq > amin && aq < lmax) ? gf * (-1.0 / sinh(aq)) : 0.0;
                const double gq = q[e] > 0 ? ga : (q[e] < 0 ? -ga : 0.0);
                const double wt = J->w[(size_t)(t - 1) * NT + J->etype[e]];
                const double p = wt * xt[e];
                const double gp = (p > -lmax && p < lmax) ? gq : 0.0;
                dw[(size_t)(t - 1) * NT + J->etype[e]] += gp * xt[e];
                gx[e] = gp * wt;
            }
        /* x_e = Lch(v) + sum of the other r^{t-1} at v */
        for (int64_t e = 0; e < E; ++e) gr[e] = 0.0;
        for (int32_t v = 0; v < n; ++v)
            for (int64_t k = a->vptr[v]; k < a->vptr[v + 1]; ++k) {
                const int64_t e = a->vedge[k];
                gLch[v] += gx[e];
                for (int64_t k2 = a->vptr[v]; k2 < a->vptr[v + 1]; ++k2)
                    if (k2 != k) gr[a->vedge[k2]] += gx[e];
            }
    }
    for (int32_t v = 0; v < n; ++v)
        J->dllr[(size_t)b * n + v] = (llr[v] > -lmax && llr[v] < lmax) ? gLch[v] : 0.0;
    free(Lch); free(gLch); free(r); free(x); free(gr); free(gx); free(q); free(f); free(go);
    return ORACLE_OK;
}

static void *wbp_worker(void *arg) {
    wbp_job *J = arg;
    for (;;) {
        int b = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (b >= J->batch) break;
        int st = wbp_one(J, b);
        if (st != ORACLE_OK) __atomic_store_n(&J->status, st, __ATOMIC_RELAXED);
    }
    return NULL;
}

/* loss (mean over B*n), posteriors, dloss/dw [T][n_types], dloss/dllr [B][n] */
int oracle_wbp(int32_t n_vn, int32_t n_cn, int64_t n_edges, const int32_t *edge_vn,
               const int32_t *edge_cn, const uint8_t *edge_type, int32_t n_types,
               int32_t batch, const double *llr, const uint8_t *syndrome, const uint8_t *xbits,
               int32_t T, const double *w, double lmax, double *loss, double *post,
               double *dw, double *dllr, int32_t n_threads) {
    if (n_vn < 0 || n_cn < 0 || n_edges < 0 || batch < 1 || T < 1 || n_types < 1 || !(lmax > 0.0))
        return ORACLE_EINVAL;
    for (int64_t e = 0; e < n_edges; ++e)
        if (edge_type[e] >= n_types) return ORACLE_EINVAL;
    adjacency a;
    int st = adj_build(&a, n_vn, n_cn, n_edges, edge_vn, edge_cn);
    if (st != ORACLE_OK) return st;
    double *lossb = calloc((size_t)batch, sizeof(double));
    double *dwb = calloc((size_t)batch * T * n_types, sizeof(double));
    if (!lossb || !dwb) { free(lossb); free(dwb); adj_free(&a); return ORACLE_ENOMEM; }
    wbp_job J = {&a, edge_type, n_types, llr, syndrome, xbits, batch, T, w, lmax,
                 lossb, post, dwb, dllr, 0, ORACLE_OK};
    st = run_workers(wbp_worker, &J, n_threads, batch);
    double l = 0.0;
    for (int32_t b = 0; b < batch; ++b) l += lossb[b];
    *loss = l / ((double)batch * (double)n_vn);
    for (int64_t i = 0; i < (int64_t)T * n_types; ++i) {
        double acc = 0.0;
        for (int32_t b = 0; b < batch; ++b) acc += dwb[(size_t)b * T * n_types + i];
        dw[i] = acc;
    }
    free(lossb); free(dwb);
    adj_free(&a);
    return st != ORACLE_OK ? st : J.status;
}
