/*
 * Reference oracle for bound propagation (BP), double probing and probe priority.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this code.  The GPU library never links, includes or calls it,
 * and this file includes nothing from the library.
 *
 * Plain sequential C over IEEE double, built with -ffp-contract=off (no fused
 * multiply-add, every product and sum rounded on its own), written from
 *   - the MILP statement of the paper's Section 1 (rows  sum_i a_ki x_i <= g_k,
 *     l <= x <= u, x_i integer for integer variables),
 *   - Section 2.1 (minimal activity L_min and the bound update formulas),
 *   - Section 2.2 (probe split of integer domains, probe priority keys),
 * with a stated reading for every point the paper leaves open:
 *   - only <= rows; equalities come as two rows;
 *   - an infinite bound is never summed: it is counted (ninf) and a residual activity
 *     is finite only when ninf == 0, or ninf == 1 and the variable is the infinite one;
 *   - Jacobi rounds: every candidate of round r is tested against the bounds at the start
 *     of round r; round r+1 processes the rows holding a variable changed in round r;
 *   - tolerance 1e-6 (Section 3's feasibility tolerance) for integer rounding
 *     (floor(c + tol), ceil(c - tol)), row infeasibility (L_min > g + tol) and the
 *     crossing of continuous bounds (l > u + tol);
 *   - continuous bounds move only when the improvement exceeds theta * max(1, |bound|),
 *     or the old bound is infinite (the "threshold" of Section 2.1);
 *   - |value| >= 1e20 means infinite; candidates with |c| >= 1e20 are dropped.
 *
 * Besides the result, the oracle counts "fragile" decisions: a rounding, acceptance or
 * infeasibility decision whose outcome would change somewhere inside an error window
 * around the computed value.  The window is twice the worst-case error of recursive
 * summation in any order (Higham, Accuracy and Stability of Numerical Algorithms,
 * Lemma 3.4: |error| <= gamma_{n} * sum |terms|, gamma_n = n u / (1 - n u), u = 2^-53)
 * plus the propagated uncertainty of continuous bounds computed in earlier rounds.
 * An implementation that sums in another order (or with fused multiply-add) may decide a
 * fragile case differently; it must agree on every decision that is not fragile.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define ORC_TOL 1e-6
#define ORC_INF 1e20
#define ORC_U 1.1102230246251565e-16 /* 2^-53, unit roundoff of binary64 */

static double gam(double k) { return k * ORC_U / (1.0 - k * ORC_U); }

/* ---------------------------------------------------------------- loading ---- */

/* Validates and copies the CSR matrix, builds its transpose.  Returns NULL when the input
 * is malformed; *err receives a code (1 row_ptr, 2 column range / order, 3 coefficient,
 * 4 right-hand side). */
orc_problem *orc_load(int32_t m, int32_t n, const int64_t *row_ptr, const int32_t *col,
                      const double *val, const double *g, const uint8_t *is_int, int32_t *err)
{
    *err = 0;
    if (m < 0 || n < 0 || row_ptr[0] != 0) { *err = 1; return NULL; }
    for (int32_t k = 0; k < m; ++k)
        if (row_ptr[k + 1] < row_ptr[k]) { *err = 1; return NULL; }
    int64_t nnz = row_ptr[m];
    for (int32_t k = 0; k < m; ++k) {
        for (int64_t p = row_ptr[k]; p < row_ptr[k + 1]; ++p) {
            if (col[p] < 0 || col[p] >= n) { *err = 2; return NULL; }
            if (p > row_ptr[k] && col[p] <= col[p - 1]) { *err = 2; return NULL; }
            double a = val[p];
            if (!(fabs(a) >= 1e-12) || !(fabs(a) < ORC_INF)) { *err = 3; return NULL; }
        }
        if (isnan(g[k]) || g[k] <= -ORC_INF) { *err = 4; return NULL; }
    }
    orc_problem *p = (orc_problem *)calloc(1, sizeof(orc_problem));
    p->m = m; p->n = n; p->nnz = nnz;
    p->row_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    p->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    p->val = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
    p->g = (double *)malloc(sizeof(double) * (size_t)(m ? m : 1));
    p->is_int = (uint8_t *)malloc((size_t)(n ? n : 1));
    memcpy(p->row_ptr, row_ptr, sizeof(int64_t) * (size_t)(m + 1));
    memcpy(p->col, col, sizeof(int32_t) * (size_t)nnz);
    memcpy(p->val, val, sizeof(double) * (size_t)nnz);
    for (int32_t k = 0; k < m; ++k) p->g[k] = (g[k] >= ORC_INF) ? INFINITY : g[k];
    memcpy(p->is_int, is_int, (size_t)n);
    /* transpose by counting */
    p->col_ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    p->row_idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz ? nnz : 1));
    p->col_val = (double *)malloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
    for (int64_t q = 0; q < nnz; ++q) p->col_ptr[col[q] + 1]++;
    for (int32_t j = 0; j < n; ++j) p->col_ptr[j + 1] += p->col_ptr[j];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    for (int32_t j = 0; j < n; ++j) fill[j] = p->col_ptr[j];
    for (int32_t k = 0; k < m; ++k)
        for (int64_t q = row_ptr[k]; q < row_ptr[k + 1]; ++q) {
            int64_t s = fill[col[q]]++;
            p->row_idx[s] = k;
            p->col_val[s] = val[q];
        }
    free(fill);
    return p;
}

void orc_free(orc_problem *p)
{
    if (!p) return;
    free(p->row_ptr); free(p->col); free(p->val); free(p->g); free(p->is_int);
    free(p->col_ptr); free(p->row_idx); free(p->col_val);
    free(p);
}

/* Bound normalisation: |b| >= 1e20 becomes infinite; an integer variable's finite bounds
 * are rounded inward with the tolerance: l = ceil(l - tol), u = floor(u + tol). */
void orc_normalize(const orc_problem *p, double *lb, double *ub)
{
    for (int32_t j = 0; j < p->n; ++j) {
        double l = lb[j], u = ub[j];
        if (l <= -ORC_INF) l = -INFINITY;
        if (u >= ORC_INF) u = INFINITY;
        if (p->is_int[j]) {
            if (isfinite(l)) l = ceil(l - ORC_TOL);
            if (isfinite(u)) u = floor(u + ORC_TOL);
        }
        lb[j] = l; ub[j] = u;
    }
}

/* ----------------------------------------------------------- propagation ---- */

/* A variable's bounds cross: integer l > u, continuous l > u + tol. */
static int crossed(int is_int, double l, double u)
{
    if (is_int) return l > u;
    return l > u + ORC_TOL;
}

/*
 * Bound propagation to a fixpoint (Section 2.1), Jacobi rounds driven by a worklist of
 * rows.  lb/ub: in = start bounds (normalised here), out = bounds after the last round.
 * dlb/dub (nullable): per-bound uncertainty of continuous bounds, in/out.
 * w0 (nullable): rows of round 0; NULL means every row.
 * mode: 0 worklist, 1 full sweep every round (same bounds and rounds, more work),
 *       2 Gauss-Seidel (candidates applied at once; only for the schedule-independence
 *       check on pure-integer problems).
 * trace_rows / trace_nnz (nullable, max_rounds entries): rows and nonzeros of each round.
 */
int orc_bp(const orc_problem *p, double *lb, double *ub, double *dlb, double *dub,
           const int32_t *w0, int32_t w0_len, double theta, int32_t max_rounds, int32_t mode,
           orc_bp_result *res, int64_t *trace_rows, int64_t *trace_nnz)
{
    const int32_t m = p->m, n = p->n;
    memset(res, 0, sizeof(*res));
    res->first_infeasible_row = -1;
    res->first_infeasible_var = -1;
    orc_normalize(p, lb, ub);

    double *l0 = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *u0 = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    memcpy(l0, lb, sizeof(double) * (size_t)n);
    memcpy(u0, ub, sizeof(double) * (size_t)n);
    double *dl = (double *)calloc((size_t)(n ? n : 1), sizeof(double));
    double *du = (double *)calloc((size_t)(n ? n : 1), sizeof(double));
    if (dlb) memcpy(dl, dlb, sizeof(double) * (size_t)n);
    if (dub) memcpy(du, dub, sizeof(double) * (size_t)n);

    /* entry check: a start box that already crosses is infeasible before any round */
    for (int32_t j = 0; j < n; ++j)
        if (crossed(p->is_int[j], lb[j], ub[j])) {
            res->status = ORC_INFEASIBLE;
            res->first_infeasible_var = j;
            break;
        }
    double *nl = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *nu = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *ndl = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *ndu = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    uint8_t *changed = (uint8_t *)calloc((size_t)(n ? n : 1), 1);
    uint8_t *inw = (uint8_t *)calloc((size_t)(m ? m : 1), 1);
    int32_t *w = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    int32_t wlen = 0;
    if (res->status == ORC_INFEASIBLE) goto done;

    if (w0) {
        for (int32_t i = 0; i < w0_len; ++i) inw[w0[i]] = 1;
    } else {
        for (int32_t k = 0; k < m; ++k) inw[k] = 1;
    }
    for (int32_t k = 0; k < m; ++k)
        if (inw[k]) w[wlen++] = k; /* ascending row order */

    for (int32_t r = 0;; ++r) {
        if (wlen == 0) { res->status = ORC_FIXPOINT; break; }
        if (r == max_rounds) { res->status = ORC_ROUND_LIMIT; break; }
        res->rounds = r + 1;
        if (trace_rows) {
            int64_t z = 0;
            for (int32_t wi = 0; wi < wlen; ++wi) z += p->row_ptr[w[wi] + 1] - p->row_ptr[w[wi]];
            trace_rows[r] = wlen;
            trace_nnz[r] = z;
        }
        memcpy(nl, lb, sizeof(double) * (size_t)n);
        memcpy(nu, ub, sizeof(double) * (size_t)n);
        memcpy(ndl, dl, sizeof(double) * (size_t)n);
        memcpy(ndu, du, sizeof(double) * (size_t)n);
        /* Gauss-Seidel reads and writes one set of bounds */
        double *rl = (mode == 2) ? nl : lb, *ru = (mode == 2) ? nu : ub;
        double *rdl = (mode == 2) ? ndl : dl, *rdu = (mode == 2) ? ndu : du;
        int any_row_infeasible = 0;

        for (int32_t wi = 0; wi < wlen; ++wi) {
            const int32_t k = w[wi];
            const int64_t beg = p->row_ptr[k], end = p->row_ptr[k + 1];
            const double gk = p->g[k];
            res->nnz_updates += end - beg;
            /* minimal activity: finite part, number of infinite contributions */
            double minfin = 0.0, mag = fabs(gk), upstream = 0.0;
            int32_t ninf = 0, infj = -1;
            for (int64_t q = beg; q < end; ++q) {
                const double a = p->val[q];
                const int32_t j = p->col[q];
                const double b = (a > 0) ? rl[j] : ru[j];
                if (isinf(b)) { ninf++; infj = j; continue; }
                const double t = a * b;
                minfin = minfin + t;
                mag += fabs(t);
                upstream += fabs(a) * ((a > 0) ? rdl[j] : rdu[j]);
            }
            const double L = (double)(end - beg);
            const double erow = 2.0 * (gam(L + 2.0) * mag + upstream);
            const double gt = gk + ORC_TOL;
            if (ninf == 0 && isfinite(gk) && fabs(minfin - gt) <= erow) res->fragile++;
            if (ninf == 0 && minfin > gt) {
                any_row_infeasible = 1;
                if (res->first_infeasible_row < 0 || k < res->first_infeasible_row)
                    res->first_infeasible_row = k;
                continue; /* an infeasible row proposes no bounds */
            }
            if (ninf >= 2) continue;
            for (int64_t q = beg; q < end; ++q) {
                const double a = p->val[q];
                const int32_t j = p->col[q];
                double resid;
                if (ninf == 1) {
                    if (j != infj) continue;
                    resid = minfin;
                } else {
                    const double b = (a > 0) ? rl[j] : ru[j];
                    const double t = a * b;
                    resid = minfin - t;
                }
                const double num = gk - resid;
                const double cand = num / a;
                if (!(fabs(cand) < ORC_INF)) continue;
                res->candidates++;
                const double ec = erow / fabs(a) + 2.0 * ORC_U * fabs(cand) * 2.0;
                const double own = ec / 2.0; /* this oracle's own error bound */
                if (a > 0) { /* upper bound candidate */
                    const double ur = ru[j];
                    if (p->is_int[j]) {
                        const double c = floor(cand + ORC_TOL);
                        const double lo = floor(cand - ec + ORC_TOL), hi = floor(cand + ec + ORC_TOL);
                        if (lo != hi && lo < ur) res->fragile++;
                        if (c < ur) {
                            if (c < nu[j]) nu[j] = c;
                            ndu[j] = 0.0;
                            changed[j] = 1;
                        }
                    } else {
                        int acc;
                        if (isinf(ur)) {
                            acc = 1;
                        } else {
                            const double thr = theta * fmax(1.0, fabs(ur));
                            acc = (ur - cand) > thr;
                            const int a1 = (ur - (cand - ec)) > thr, a2 = (ur - (cand + ec)) > thr;
                            if (a1 != a2) res->fragile++;
                        }
                        if (acc) {
                            if (cand < nu[j]) { nu[j] = cand; ndu[j] = own; }
                            else if (cand == nu[j] && own > ndu[j]) ndu[j] = own;
                            changed[j] = 1;
                        }
                    }
                } else { /* lower bound candidate */
                    const double lr = rl[j];
                    if (p->is_int[j]) {
                        const double c = ceil(cand - ORC_TOL);
                        const double lo = ceil(cand - ec - ORC_TOL), hi = ceil(cand + ec - ORC_TOL);
                        if (lo != hi && hi > lr) res->fragile++;
                        if (c > lr) {
                            if (c > nl[j]) nl[j] = c;
                            ndl[j] = 0.0;
                            changed[j] = 1;
                        }
                    } else {
                        int acc;
                        if (isinf(lr)) {
                            acc = 1;
                        } else {
                            const double thr = theta * fmax(1.0, fabs(lr));
                            acc = (cand - lr) > thr;
                            const int a1 = ((cand - ec) - lr) > thr, a2 = ((cand + ec) - lr) > thr;
                            if (a1 != a2) res->fragile++;
                        }
                        if (acc) {
                            if (cand > nl[j]) { nl[j] = cand; ndl[j] = own; }
                            else if (cand == nl[j] && own > ndl[j]) ndl[j] = own;
                            changed[j] = 1;
                        }
                    }
                }
            }
        }
        /* end of round: crossing check on the changed variables */
        int any_var_infeasible = 0;
        for (int32_t j = 0; j < n; ++j) {
            if (!changed[j]) continue;
            if (!p->is_int[j]) {
                const double ex = 2.0 * (ndl[j] + ndu[j]) + 4.0 * ORC_U * (fabs(nl[j]) + fabs(nu[j]));
                if (isfinite(nl[j]) && isfinite(nu[j]) && fabs((nl[j] - nu[j]) - ORC_TOL) <= ex)
                    res->fragile++;
            }
            if (crossed(p->is_int[j], nl[j], nu[j])) {
                any_var_infeasible = 1;
                if (res->first_infeasible_var < 0 || j < res->first_infeasible_var)
                    res->first_infeasible_var = j;
            }
        }
        memcpy(lb, nl, sizeof(double) * (size_t)n);
        memcpy(ub, nu, sizeof(double) * (size_t)n);
        memcpy(dl, ndl, sizeof(double) * (size_t)n);
        memcpy(du, ndu, sizeof(double) * (size_t)n);
        if (any_row_infeasible || any_var_infeasible) {
            res->status = ORC_INFEASIBLE;
            break;
        }
        /* next worklist: rows holding a variable changed in this round */
        int any_change = 0;
        memset(inw, 0, (size_t)m);
        for (int32_t j = 0; j < n; ++j) {
            if (!changed[j]) continue;
            any_change = 1;
            changed[j] = 0;
            for (int64_t s = p->col_ptr[j]; s < p->col_ptr[j + 1]; ++s) inw[p->row_idx[s]] = 1;
        }
        wlen = 0;
        if (mode == 1) {
            if (any_change)
                for (int32_t k = 0; k < m; ++k) w[wlen++] = k;
        } else {
            for (int32_t k = 0; k < m; ++k)
                if (inw[k]) w[wlen++] = k;
        }
    }
done:
    for (int32_t j = 0; j < n; ++j)
        if (lb[j] != l0[j] || ub[j] != u0[j]) res->n_changed++;
    if (dlb) memcpy(dlb, dl, sizeof(double) * (size_t)n);
    if (dub) memcpy(dub, du, sizeof(double) * (size_t)n);
    free(l0); free(u0); free(dl); free(du); free(nl); free(nu); free(ndl); free(ndu);
    free(changed); free(inw); free(w);
    return 0;
}

/* ---------------------------------------------------------------- probing ---- */

/* Probe split of an integer variable's domain (Section 2.2).  Boxed: c = ceil((l+u)/2),
 * down = [l, c-1], up = [c, u] (a binary gives [0,0] and [1,1]).  Only l finite: [l, l] and
 * [l+1, +inf).  Only u finite (the mirror case): [u, u] and (-inf, u-1].  Returns 0 for
 * continuous, fixed or free variables, which are not probed. */
int orc_probe_split(int32_t is_int, double l, double u, double *out4)
{
    if (!is_int || !(l < u)) return 0;
    if (isfinite(l) && isfinite(u)) {
        const double c = ceil((l + u) / 2.0);
        out4[0] = l; out4[1] = c - 1.0; out4[2] = c; out4[3] = u;
        return 1;
    }
    if (isfinite(l)) { out4[0] = l; out4[1] = l; out4[2] = l + 1.0; out4[3] = INFINITY; return 1; }
    if (isfinite(u)) { out4[0] = u; out4[1] = u; out4[2] = -INFINITY; out4[3] = u - 1.0; return 1; }
    return 0;
}

/*
 * Double probing (Section 2.2): for pair i, branch 0 runs BP from root ∩ [box_l0, box_u0]
 * of variable var[i], branch 1 from root ∩ [box_l1, box_u1]; round 0 processes the rows of
 * var[i].  Branch b of pair i is entry 2i+b.  The cache lists, for each feasible branch,
 * the variables whose bounds differ from the root, ascending, with their new bounds.
 * Infeasible branches list nothing.  Returns the number of cache entries needed; entries
 * beyond cap are not written (offsets are still complete).
 */
int64_t orc_probe_batch(const orc_problem *p, const double *root_l, const double *root_u,
                        int32_t npairs, const int32_t *var, const double *boxes /* 4 per pair */,
                        double theta, int32_t max_rounds,
                        int32_t *status, int32_t *rounds, int64_t *nnz_updates,
                        int64_t *offsets, int32_t *ent_var, double *ent_l, double *ent_u,
                        int64_t cap)
{
    const int32_t n = p->n;
    double *l = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *u = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    int32_t *w0 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(p->m ? p->m : 1));
    int64_t total = 0;
    offsets[0] = 0;
    for (int32_t i = 0; i < npairs; ++i) {
        const int32_t v = var[i];
        int32_t w0len = 0;
        for (int64_t s = p->col_ptr[v]; s < p->col_ptr[v + 1]; ++s) w0[w0len++] = p->row_idx[s];
        for (int b = 0; b < 2; ++b) {
            memcpy(l, root_l, sizeof(double) * (size_t)n);
            memcpy(u, root_u, sizeof(double) * (size_t)n);
            const double bl = boxes[4 * i + 2 * b], bu = boxes[4 * i + 2 * b + 1];
            if (bl > l[v]) l[v] = bl;
            if (bu < u[v]) u[v] = bu;
            orc_bp_result r;
            orc_bp(p, l, u, NULL, NULL, w0, w0len, theta, max_rounds, 0, &r, NULL, NULL);
            const int e = 2 * i + b;
            status[e] = r.status;
            rounds[e] = r.rounds;
            nnz_updates[e] = r.nnz_updates;
            if (r.status != ORC_INFEASIBLE) {
                for (int32_t j = 0; j < n; ++j) {
                    if (l[j] != root_l[j] || u[j] != root_u[j]) {
                        if (total < cap) { ent_var[total] = j; ent_l[total] = l[j]; ent_u[total] = u[j]; }
                        total++;
                    }
                }
            }
            offsets[e + 1] = total;
        }
    }
    free(l); free(u); free(w0);
    return total;
}

/*
 * Global bounds from a probing cache (Section 2.2: the cache gives early infeasibility
 * detection and bounds valid for every solution).  The two branch boxes of a pair cover the
 * probed variable's whole integer domain, so every feasible point lies in a feasible branch,
 * inside that branch's implied box (root bounds where the branch lists nothing).  For each
 * pair the bounds are therefore intersected with the hull of its feasible branches' boxes:
 *   - one branch infeasible: the variable is fixed to the other branch's box together with all
 *     of that branch's implied bounds;
 *   - both feasible: a variable listed by both branches gets (min of the lower bounds, max of the
 *     upper bounds); a variable listed by only one keeps its bounds;
 *   - both infeasible: the hull is empty and the problem has no feasible point.
 * lb/ub: in = the root bounds the cache was computed from (normalised here), out = the
 * intersection.  Afterwards a variable whose bounds cross (integer l > u, continuous
 * l > u + tol) also proves infeasibility.  Result: status (ORC_FIXPOINT or ORC_INFEASIBLE), the
 * first pair with both branches infeasible, the first crossing variable, the pairs with
 * exactly one infeasible branch, and the variables whose bounds changed.
 */
typedef struct {
    int32_t status;
    int32_t first_infeasible_pair;
    int32_t first_infeasible_var;
    int32_t fixed_pairs;
    int64_t tightened;
} orc_apply_result;

void orc_probe_cache_apply(const orc_problem *p, double *lb, double *ub, int32_t npairs, const int32_t *status,
                           const int64_t *offsets, const int32_t *ent_var, const double *ent_l,
                           const double *ent_u, orc_apply_result *res)
{
    const int32_t n = p->n;
    memset(res, 0, sizeof(*res));
    res->first_infeasible_pair = -1;
    res->first_infeasible_var = -1;
    orc_normalize(p, lb, ub);
    double *l0 = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *u0 = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    memcpy(l0, lb, sizeof(double) * (size_t)n);
    memcpy(u0, ub, sizeof(double) * (size_t)n);
    for (int32_t i = 0; i < npairs; ++i) {
        const int f0 = status[2 * i] != ORC_INFEASIBLE, f1 = status[2 * i + 1] != ORC_INFEASIBLE;
        if (!f0 && !f1) {
            if (res->first_infeasible_pair < 0) res->first_infeasible_pair = i;
            continue;
        }
        if (f0 != f1) {
            const int e = 2 * i + (f0 ? 0 : 1);
            res->fixed_pairs++;
            for (int64_t q = offsets[e]; q < offsets[e + 1]; ++q) {
                const int32_t w = ent_var[q];
                if (ent_l[q] > lb[w]) lb[w] = ent_l[q];
                if (ent_u[q] < ub[w]) ub[w] = ent_u[q];
            }
            continue;
        }
        /* both feasible: the variables listed by both branches (both lists ascend by variable) */
        int64_t a = offsets[2 * i], b = offsets[2 * i + 1];
        const int64_t ae = offsets[2 * i + 1], be = offsets[2 * i + 2];
        while (a < ae && b < be) {
            if (ent_var[a] < ent_var[b]) { a++; continue; }
            if (ent_var[b] < ent_var[a]) { b++; continue; }
            const int32_t w = ent_var[a];
            const double hl = ent_l[a] < ent_l[b] ? ent_l[a] : ent_l[b];
            const double hu = ent_u[a] > ent_u[b] ? ent_u[a] : ent_u[b];
            if (hl > lb[w]) lb[w] = hl;
            if (hu < ub[w]) ub[w] = hu;
            a++;
            b++;
        }
    }
    for (int32_t j = 0; j < n; ++j) {
        if (lb[j] != l0[j] || ub[j] != u0[j]) res->tightened++;
        if (res->first_infeasible_var < 0 && crossed(p->is_int[j], lb[j], ub[j])) res->first_infeasible_var = j;
    }
    res->status = (res->first_infeasible_pair >= 0 || res->first_infeasible_var >= 0) ? ORC_INFEASIBLE : ORC_FIXPOINT;
    free(l0);
    free(u0);
}

/* ------------------------------------------------------------ priority ---- */

/*
 * Probe priority keys (Section 2.2) under bounds (lb, ub), for every probeable integer
 * variable (l < u, at least one finite bound):
 *   key1 = number of rows whose minimal activity, with this variable's contribution flipped
 *          from its minimising to its maximising bound (L_min + |a| (u - l)), exceeds g + tol;
 *   key2 = the largest such excess (flipped activity - g);
 *   key3 = the smallest unit slack (g - L_min) / |a| over the variable's rows.
 * key1 and key2 are computed only for variables with coefficients of both signs, else 0.
 * Rows with an infinite minimal activity take no part; an infinite width counts as a
 * violation with infinite excess.  Writes keys for all n (non-probeable: key1 = -1).
 */
void orc_probe_priority(const orc_problem *p, const double *lb, const double *ub,
                        int32_t *key1, double *key2, double *key3)
{
    const int32_t m = p->m, n = p->n;
    double *minfin = (double *)malloc(sizeof(double) * (size_t)(m ? m : 1));
    int32_t *ninf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    for (int32_t k = 0; k < m; ++k) {
        double s = 0.0;
        int32_t c = 0;
        for (int64_t q = p->row_ptr[k]; q < p->row_ptr[k + 1]; ++q) {
            const double a = p->val[q];
            const double b = (a > 0) ? lb[p->col[q]] : ub[p->col[q]];
            if (isinf(b)) { c++; continue; }
            const double t = a * b;
            s = s + t;
        }
        minfin[k] = s;
        ninf[k] = c;
    }
    for (int32_t j = 0; j < n; ++j) {
        double box[4];
        if (!orc_probe_split(p->is_int[j], lb[j], ub[j], box)) {
            key1[j] = -1; key2[j] = 0.0; key3[j] = INFINITY;
            continue;
        }
        int pos = 0, neg = 0;
        for (int64_t s = p->col_ptr[j]; s < p->col_ptr[j + 1]; ++s) {
            if (p->col_val[s] > 0) pos = 1; else neg = 1;
        }
        const int mixed = pos && neg;
        int32_t cnt = 0;
        double exc = 0.0, unit = INFINITY;
        const double width = ub[j] - lb[j];
        for (int64_t s = p->col_ptr[j]; s < p->col_ptr[j + 1]; ++s) {
            const int32_t k = p->row_idx[s];
            if (ninf[k] != 0 || isinf(p->g[k])) continue;
            const double a = fabs(p->col_val[s]);
            const double slack = p->g[k] - minfin[k];
            const double us = slack / a;
            if (us < unit) unit = us;
            if (mixed) {
                const double flipped = minfin[k] + a * width;
                if (flipped > p->g[k] + ORC_TOL) {
                    cnt++;
                    const double e = flipped - p->g[k];
                    if (e > exc) exc = e;
                }
            }
        }
        key1[j] = cnt; key2[j] = exc; key3[j] = unit;
    }
    free(minfin); free(ninf);
}
