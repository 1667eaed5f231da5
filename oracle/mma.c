/*
 * Oracle numeric core: min-sum passes, min-marginals and the deferred min-marginal
 * averaging (MMA) iteration on explicit BDD node graphs, in FP64, one BDD after another.
 *
 * TEST INFRASTRUCTURE ONLY: called by tests, by the smoke check and by the bench's CPU
 * baseline; the product path never links or loads it.
 *
 * Passages followed:
 *   - Lagrange decomposition dual (D): max_lambda sum_j min_{s in S_j} s^T lambda^j
 *     s.t. sum_{j in J_i} lambda^j_i = c_i (Sec. 2 "Dual Decomposition for ILPs", Eq. D).
 *   - shortest paths through each BDD (Sec. 3.2 "Constraint Splitting").
 *   - min-marginal differences M^j_i = min_{s_i=1} s^T lambda^j - min_{s_i=0} s^T lambda^j
 *     (App. A.5 "Coarse-to-fine solving strategy").
 *   - min-marginal averaging with deferred, parallel-across-subproblems updates
 *     (the first-order scheme the paper builds on, Sec. 2 and Alg. 1 "MMA").
 *
 * Reading of the iteration (the paper defers its details to the cited first-order
 * method): one half-pass visits every BDD's layers in order (forward) or in reverse
 * (backward); at each layer of variable i it
 *     lambda += pend_i            (mean of the previous half-pass's removed mass)
 *     M = m1 - m0                 (current f of this layer, b of the next)
 *     lambda -= omega * M
 *     acc_i += omega * M
 * and after the half-pass pend_i = acc_i / |J_i|.
 *
 * Graph layout: BDD j owns layers [blp[j], blp[j+1]); layer l tests variable lvar[l]
 * and owns nodes [lnp[l], lnp[l+1]); lo[u] / hi[u] is the global index of the child
 * node, -1 for the false terminal, -2 for the true terminal. The first node of a BDD's
 * first layer is its root. state[i]: 0 free, 1 fixed to 0, 2 fixed to 1.
 */
#include <math.h>
#include <stdint.h>

#define BOT (-1)
#define TOP (-2)

static double child_cost(const double *b, int64_t c)
{
    if (c == TOP) return 0.0;
    if (c == BOT) return INFINITY;
    return b[c];
}

static double dmin(double a, double b) { return a < b ? a : b; }

static void push(double *f, double *top, int64_t c, double v)
{
    if (c == TOP) { if (v < *top) *top = v; }
    else if (c != BOT) { if (v < f[c]) f[c] = v; }
}

/* f = cost of the cheapest path root -> node; returns per BDD the cheapest root -> TOP cost. */
void or_forward(int64_t nb, const int64_t *blp, const int64_t *lvar, const int64_t *lnp,
                const int64_t *lo, const int64_t *hi, const double *cost, const int8_t *state,
                double *f, double *out_min)
{
    for (int64_t j = 0; j < nb; ++j) {
        double top = INFINITY;
        f[lnp[blp[j]]] = 0.0;
        for (int64_t l = blp[j]; l < blp[j + 1]; ++l) {
            int8_t st = state ? state[lvar[l]] : 0;
            if (l + 1 < blp[j + 1])
                for (int64_t u = lnp[l + 1]; u < lnp[l + 2]; ++u) f[u] = INFINITY;
            for (int64_t u = lnp[l]; u < lnp[l + 1]; ++u) {
                if (f[u] == INFINITY) continue;
                if (st != 2) push(f, &top, lo[u], f[u]);
                if (st != 1) push(f, &top, hi[u], f[u] + cost[l]);
            }
        }
        out_min[j] = top;
    }
}

/* b = cost of the cheapest path node -> TOP; returns per BDD the root's value. */
void or_backward(int64_t nb, const int64_t *blp, const int64_t *lvar, const int64_t *lnp,
                 const int64_t *lo, const int64_t *hi, const double *cost, const int8_t *state,
                 double *b, double *out_min)
{
    for (int64_t j = 0; j < nb; ++j) {
        for (int64_t l = blp[j + 1] - 1; l >= blp[j]; --l) {
            int8_t st = state ? state[lvar[l]] : 0;
            for (int64_t u = lnp[l]; u < lnp[l + 1]; ++u) {
                double v0 = st != 2 ? child_cost(b, lo[u]) : INFINITY;
                double v1 = st != 1 ? cost[l] + child_cost(b, hi[u]) : INFINITY;
                b[u] = dmin(v0, v1);
            }
        }
        out_min[j] = b[lnp[blp[j]]];
    }
}

/* M per layer from f (root side) and b (terminal side) of one cost vector. */
void or_min_marginals(int64_t nl, const int64_t *lnp, const int64_t *lo, const int64_t *hi,
                      const double *cost, const double *f, const double *b, double *m0_out,
                      double *m1_out)
{
    for (int64_t l = 0; l < nl; ++l) {
        double m0 = INFINITY, m1 = INFINITY;
        for (int64_t u = lnp[l]; u < lnp[l + 1]; ++u) {
            m0 = dmin(m0, f[u] + child_cost(b, lo[u]));
            m1 = dmin(m1, f[u] + cost[l] + child_cost(b, hi[u]));
        }
        m0_out[l] = m0;
        m1_out[l] = m1;
    }
}

/*
 * One half-pass of deferred MMA. dir > 0: forward (reads b, writes f);
 * dir < 0: backward (reads f, writes b). pend is read, acc accumulates the removed
 * mass; the caller forms the next pend. Fixed variables (state != 0) are not updated.
 * Returns the number of layers whose min-marginal was not finite (0 when well posed).
 */
int64_t or_half_pass(int dir, int64_t nb, const int64_t *blp, const int64_t *lvar,
                     const int64_t *lnp, const int64_t *lo, const int64_t *hi, double *lam,
                     const double *pend, double *acc, const int8_t *state, double omega,
                     double *f, double *b)
{
    int64_t bad = 0;
    for (int64_t j = 0; j < nb; ++j) {
        int64_t first = blp[j], last = blp[j + 1] - 1;
        double top = INFINITY;
        if (dir > 0) f[lnp[first]] = 0.0;
        for (int64_t t = 0; t <= last - first; ++t) {
            int64_t l = dir > 0 ? first + t : last - t;
            int64_t i = lvar[l];
            int8_t st = state ? state[i] : 0;
            if (st == 0) {
                double m0 = INFINITY, m1 = INFINITY;
                lam[l] += pend[i];
                for (int64_t u = lnp[l]; u < lnp[l + 1]; ++u) {
                    m0 = dmin(m0, f[u] + child_cost(b, lo[u]));
                    m1 = dmin(m1, f[u] + lam[l] + child_cost(b, hi[u]));
                }
                if (isfinite(m0) && isfinite(m1)) {
                    double M = m1 - m0;
                    lam[l] -= omega * M;
                    acc[i] += omega * M;
                } else {
                    ++bad;
                }
            }
            if (dir > 0) {
                if (l < last)
                    for (int64_t u = lnp[l + 1]; u < lnp[l + 2]; ++u) f[u] = INFINITY;
                for (int64_t u = lnp[l]; u < lnp[l + 1]; ++u) {
                    if (f[u] == INFINITY) continue;
                    if (st != 2) push(f, &top, lo[u], f[u]);
                    if (st != 1) push(f, &top, hi[u], f[u] + lam[l]);
                }
            } else {
                for (int64_t u = lnp[l]; u < lnp[l + 1]; ++u) {
                    double v0 = st != 2 ? child_cost(b, lo[u]) : INFINITY;
                    double v1 = st != 1 ? lam[l] + child_cost(b, hi[u]) : INFINITY;
                    b[u] = dmin(v0, v1);
                }
            }
        }
    }
    return bad;
}

/*
 * Values each layer's variable can take on some root -> TOP path that respects the
 * fixings: sup0[l] / sup1[l] in {0, 1}. rf / rb are node scratch arrays.
 */
void or_supports(int64_t nb, const int64_t *blp, const int64_t *lvar, const int64_t *lnp,
                 const int64_t *lo, const int64_t *hi, const int8_t *state, int8_t *rf, int8_t *rb,
                 int8_t *sup0, int8_t *sup1)
{
    for (int64_t j = 0; j < nb; ++j) {
        int64_t first = blp[j], last = blp[j + 1] - 1;
        for (int64_t u = lnp[first]; u < lnp[last + 1]; ++u) rf[u] = 0;
        rf[lnp[first]] = 1;
        for (int64_t l = first; l <= last; ++l) {
            int8_t st = state[lvar[l]];
            for (int64_t u = lnp[l]; u < lnp[l + 1]; ++u) {
                if (!rf[u]) continue;
                if (st != 2 && lo[u] >= 0) rf[lo[u]] = 1;
                if (st != 1 && hi[u] >= 0) rf[hi[u]] = 1;
            }
        }
        for (int64_t l = last; l >= first; --l) {
            int8_t st = state[lvar[l]];
            int8_t s0 = 0, s1 = 0;
            for (int64_t u = lnp[l]; u < lnp[l + 1]; ++u) {
                int8_t ok0 = st != 2 && (lo[u] == TOP || (lo[u] >= 0 && rb[lo[u]]));
                int8_t ok1 = st != 1 && (hi[u] == TOP || (hi[u] >= 0 && rb[hi[u]]));
                rb[u] = ok0 || ok1;
                if (rf[u] && ok0) s0 = 1;
                if (rf[u] && ok1) s1 = 1;
            }
            sup0[l] = s0;
            sup1[l] = s1;
        }
    }
}
