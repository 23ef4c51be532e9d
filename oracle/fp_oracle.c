/*
 * Oracle of bulk fix-and-propagate rounding (Section 2.3, Algorithm 1 "Bound Propagation
 * Rounding"; LP polish off, repair optional and off by default, as in the paper's experiments).
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests and the benchmark's CPU leg, never by the
 * library.  Plain sequential C over IEEE double (-ffp-contract=off).
 *
 * Steps, in the paper's order, with a stated reading wherever the paper leaves a point open:
 *  1. propagate the start bounds (every row);
 *  2. initial sort of the integer variables (Section 2.3): binary (u - l <= 1) before ternary
 *     (u - l = 2) before the rest, then ascending fractionality |x - round(x)|, then index;
 *  3. per bulk:
 *     - bulk size: ceil(sqrt(remaining)) or ceil(fraction * integer variables); one variable
 *       at a time for the last `last_single` (36 in the paper) and in recovery;
 *     - for bulks larger than one, a stable implied-slack sort of the unfixed variables:
 *       S_i = sum over rows with a finite minimal activity of (a / slack)^2,
 *       slack = max(g - L_min, tol), descending (Section 2.3 equation); with a learned order
 *       score (no counterpart in the paper) the score ranks the variables within their class
 *       instead and the implied-slack sort is skipped;
 *     - two candidate values per variable drawn from the rounding distribution (random near
 *       .5, nearest away from .5: P(up) = 0 for f <= .25, 1 for f >= .75, linear between);
 *       single-variable bulks try the drawn value and the other integer neighbour;
 *     - with a probing cache, a fixing is kept only if its value and the cached implications
 *       of the branch containing it agree with the fixings kept before it (Section 2.2), and
 *       the cached bounds tighten the start of the propagation (warm start);
 *     - both candidate vectors are propagated from the rows of the variables whose bounds
 *       they change; the first feasible result is kept (probe 0 first);
 *     - both infeasible: a bulk's variables are retried one by one (recovery); a single
 *       variable that fails both ways ends the search (repair disabled, as in the paper's
 *       experiments, Section 3): the remaining integer variables are rounded to the nearest
 *       value inside their bounds without propagation and the result is INFEASIBLE.  With
 *       repair on (repair_max > 0, no probing cache) it first tries up to repair_max times in
 *       the run to shift earlier fixings until a propagation from the start bounds is feasible
 *       (the repair branch of Algorithm 1; see repair() for the reading).
 *  4. FEASIBLE when every integer variable is fixed, the last propagation was feasible, and a
 *     propagation of the start bounds with every integer variable fixed at its value is not
 *     infeasible either (`refuted` otherwise: under the threshold of Section 2.1 an incremental
 *     propagation can stop short of a contradiction that one from the start bounds reaches).
 *
 * The random draws use splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) chained over (seed, bulk, variable, draw); the 53 high bits give a
 * uniform double in [0, 1).
 *
 * Fragile decisions (result field `fragile`): the propagations' own (bp_oracle.c), and the bulk
 * boundary of each implied-slack sort.  S_i depends on each row's minimal activity, whose sum
 * another implementation may round differently (any order, fused multiply-add) and whose
 * continuous bounds carry the uncertainty the propagations report; both are bounded per row
 * as in bp_oracle.c (twice the Higham bound plus the upstream uncertainty), and S_i's window
 * is the exact range of its terms a^2 / max(slack, tol)^2 over the slack's window.  A bulk is
 * fragile when a variable inside it and one outside could exchange places within their
 * windows (with a probing cache, also two variables inside it, whose order decides which
 * conflicting fixing is kept).  The draws need no window: their inputs (the fractional value
 * clamped to exact integer bounds, the generator's integers) are the same on any IEEE
 * implementation, and so is the comparison u < P(up).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define FP_TOL 1e-6
#define FP_U 1.1102230246251565e-16 /* 2^-53 */

static double fp_gam(double k) { return k * FP_U / (1.0 - k * FP_U); }

typedef struct {
    uint64_t seed;
    int32_t bulk_rule;      /* 0: ceil(sqrt(remaining)), 1: ceil(fraction * integer variables) */
    double fraction;
    int32_t last_single;
    double theta;
    int32_t max_rounds;
    const double *order_score;  /* optional: order by class, descending score, fractionality, index; no
                                 * per-bulk implied-slack sort */
    const double *up_prob;      /* optional: P(up) for fractions strictly inside (0.25, 0.75) */
    int32_t repair_max;         /* repairs a run may attempt (0: repair off, as in the paper's experiments) */
    int32_t repair_cycles;      /* propagations one repair may run */
} orc_fp_params;

typedef struct {
    int32_t status;         /* 0 feasible (all integers fixed, propagation feasible), 1 infeasible */
    int32_t bulks;
    int32_t bp_runs;
    int32_t recoveries;
    int32_t fixed_by_choice; /* kept fixings of the chosen candidate vectors, summed over bulks */
    int32_t refuted;         /* every integer fixed, but the final check from the start bounds failed */
    int64_t nnz_updates;
    int64_t fragile;
    int32_t repairs;         /* repairs that ended with a feasible propagation */
    int32_t repair_runs;     /* propagations run by repairs (also counted in bp_runs and nnz_updates) */
} orc_fp_result;

/* probing cache in the layout of bp_probe_batch */
typedef struct {
    int32_t npairs;
    const int32_t *var;
    const double *boxes;
    const int32_t *status;
    const int64_t *offsets;
    const int32_t *ent_var;
    const double *ent_l;
    const double *ent_u;
} orc_cache;

static uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64(uint64_t z) { return splitmix64(z); }

double orc_uniform(uint64_t seed, uint64_t bulk, uint64_t var, uint64_t draw)
{
    uint64_t h = splitmix64(seed);
    h = splitmix64(h ^ bulk);
    h = splitmix64(h ^ var);
    h = splitmix64(h ^ draw);
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

static double clampd(double x, double l, double u) { return x < l ? l : (x > u ? u : x); }

/* one draw from the rounding distribution of x (already inside the bounds) */
static double draw_value(double x, uint64_t seed, uint64_t bulk, int32_t j, int d, const double *up_prob)
{
    const double fl = floor(x);
    const double f = x - fl;
    if (f == 0.0) return x;
    double pup;
    if (f <= 0.25) pup = 0.0;
    else if (f >= 0.75) pup = 1.0;
    else pup = up_prob ? up_prob[j] : (f - 0.25) / 0.5;
    const double u = orc_uniform(seed, bulk, (uint64_t)j, (uint64_t)d);
    return u < pup ? fl + 1.0 : fl;
}

static uint64_t isqrt_ceil(uint64_t r)
{
    uint64_t s = (uint64_t)sqrt((double)r);
    while (s * s > r) --s;
    while ((s + 1) * (s + 1) <= r) ++s;
    return s * s == r ? s : s + 1;
}

/* sort helpers (stable merge sort over an index array with a key comparator) */
typedef struct {
    const int32_t *cls;
    const double *frac;
    const double *S;
    const double *score;
} sort_ctx;

static int cmp_initial(const sort_ctx *c, int32_t a, int32_t b)
{
    if (c->cls[a] != c->cls[b]) return c->cls[a] < c->cls[b] ? -1 : 1;
    if (c->score && c->score[a] != c->score[b]) return c->score[a] > c->score[b] ? -1 : 1;
    if (c->frac[a] != c->frac[b]) return c->frac[a] < c->frac[b] ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

static int cmp_slack(const sort_ctx *c, int32_t a, int32_t b)
{
    if (c->S[a] != c->S[b]) return c->S[a] > c->S[b] ? -1 : 1;   /* descending; ties keep order */
    return 0;
}

static void merge_sort(int32_t *v, int32_t *tmp, int64_t n, const sort_ctx *c, int (*cmp)(const sort_ctx *, int32_t, int32_t))
{
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) tmp[k++] = cmp(c, v[j], v[i]) < 0 ? v[j++] : v[i++];
            while (i < mid) tmp[k++] = v[i++];
            while (j < hi) tmp[k++] = v[j++];
        }
        memcpy(v, tmp, sizeof(int32_t) * (size_t)n);
    }
}

/* implied slack S_i of every variable under bounds (l, u) */
static void implied_slack(const orc_problem *p, const double *l, const double *u, double *S)
{
    for (int32_t j = 0; j < p->n; ++j) S[j] = 0.0;
    for (int32_t k = 0; k < p->m; ++k) {
        if (isinf(p->g[k])) continue;
        double minfin = 0.0;
        int ninf = 0;
        for (int64_t q = p->row_ptr[k]; q < p->row_ptr[k + 1]; ++q) {
            const double a = p->val[q];
            const double b = a > 0 ? l[p->col[q]] : u[p->col[q]];
            if (isinf(b)) { ninf++; continue; }
            const double t = a * b;
            minfin = minfin + t;
        }
        if (ninf) continue;
        double slack = p->g[k] - minfin;
        if (slack < FP_TOL) slack = FP_TOL;
        for (int64_t q = p->row_ptr[k]; q < p->row_ptr[k + 1]; ++q) {
            const double s = p->val[q] / slack;
            const double s2 = s * s;
            S[p->col[q]] = S[p->col[q]] + s2;
        }
    }
}

/* exported for the pins of the implied-slack equation (Section 2.3) */
void orc_implied_slack(const orc_problem *p, const double *l, const double *u, double *S)
{
    implied_slack(p, l, u, S);
}

/* Window E_i of every S_i (see the header): the range of sum_k a^2 / max(slack_k, tol)^2 when
 * each slack_k moves by its row's error bound; dl / du: uncertainty of the bounds. */
static void implied_slack_window(const orc_problem *p, const double *l, const double *u, const double *dl,
                                 const double *du, double *E)
{
    for (int32_t j = 0; j < p->n; ++j) E[j] = 0.0;
    for (int32_t k = 0; k < p->m; ++k) {
        if (isinf(p->g[k])) continue;
        double minfin = 0.0, mag = fabs(p->g[k]), upstream = 0.0;
        int ninf = 0, exact = p->g[k] == floor(p->g[k]);
        for (int64_t q = p->row_ptr[k]; q < p->row_ptr[k + 1]; ++q) {
            const double a = p->val[q];
            const int32_t j = p->col[q];
            const double b = a > 0 ? l[j] : u[j];
            if (isinf(b)) { ninf++; continue; }
            const double t = a * b;
            minfin = minfin + t;
            mag += fabs(t);
            upstream += fabs(a) * (a > 0 ? dl[j] : du[j]);
            exact = exact && a == floor(a) && b == floor(b);
        }
        if (ninf) continue;
        /* integer terms and right-hand side below 2^53 and exact bounds: every summation order
         * gives the same exact activity, so the slack has no window */
        if (exact && upstream == 0.0 && mag < 9007199254740992.0) continue;
        const double len = (double)(p->row_ptr[k + 1] - p->row_ptr[k]);
        const double err = 2.0 * (fp_gam(len + 2.0) * mag + upstream);
        if (err == 0.0) continue;
        const double slack = p->g[k] - minfin;
        const double lo = fmax(slack - err, FP_TOL), hi = fmax(slack + err, FP_TOL);
        if (lo == hi) continue;   /* the floor holds over the whole window */
        for (int64_t q = p->row_ptr[k]; q < p->row_ptr[k + 1]; ++q) {
            const double a = p->val[q];
            E[p->col[q]] += a * a * (1.0 / (lo * lo) - 1.0 / (hi * hi)) * (1.0 + 8.0 * FP_U);
        }
    }
}

/* Fragile bulk boundary: after the sort of work[0..nun) by decreasing S, can a variable of the
 * bulk work[0..bsize) and one after it exchange places within their windows [S - E, S + E]?
 * With `inside`, also two variables of the bulk.  Since the order is decreasing, a pair (a
 * before b) can exchange iff S_b + E_b >= S_a - E_a with a nonzero window on either side; two
 * zero windows overlap only in an exact tie, which every IEEE implementation reproduces and the
 * stable sort keeps in order.  Both tests are linear: against the lowest S - E before b (any
 * window, when E_b > 0; nonzero windows only, when E_b = 0). */
static int slack_sort_fragile(const int32_t *work, int64_t nun, int64_t bsize, const double *S, const double *E,
                              int inside)
{
    if (bsize >= nun) return 0;
    double lo_any = INFINITY, lo_wide = INFINITY;   /* over the bulk: min S - E, and over E > 0 only */
    for (int64_t i = 0; i < bsize; ++i) {
        const int32_t a = work[i];
        if (inside && i > 0) {
            const double top = S[a] + E[a];
            if ((E[a] > 0.0 && top >= lo_any) || top >= lo_wide) return 1;
        }
        lo_any = fmin(lo_any, S[a] - E[a]);
        if (E[a] > 0.0) lo_wide = fmin(lo_wide, S[a] - E[a]);
    }
    for (int64_t i = bsize; i < nun; ++i) {
        const int32_t b = work[i];
        const double top = S[b] + E[b];
        if ((E[b] > 0.0 && top >= lo_any) || top >= lo_wide) return 1;
    }
    return 0;
}

/* cache branch of (j, value): entry index 2*pair + b, or -1 */
static int64_t cache_branch(const orc_cache *c, const int32_t *pair_of, int32_t j, double val)
{
    if (!c) return -1;
    const int32_t i = pair_of[j];
    if (i < 0) return -1;
    for (int b = 0; b < 2; ++b) {
        const double lo = c->boxes[4 * i + 2 * b], hi = c->boxes[4 * i + 2 * b + 1];
        if (val >= lo && val <= hi) return 2 * (int64_t)i + b;
    }
    return -1;
}

static int var_cross(int is_i, double l, double u) { return is_i ? l > u : l > u + FP_TOL; }

/* Minimal activity of row k under (l, u): finite part (row order, separate multiply and add,
 * as in bp_oracle.c), number of infinite contributions, and the error bound of the finite part
 * (twice the Higham bound plus the continuous bounds' uncertainty; 0 when every term and
 * partial sum is an integer below 2^50, which makes the sum exact in any order). */
static double row_min_activity(const orc_problem *p, int32_t k, const double *l, const double *u, const double *dl,
                               const double *du, int32_t *ninf, double *err)
{
    const int64_t beg = p->row_ptr[k], end = p->row_ptr[k + 1];
    double minfin = 0.0, mag = fabs(p->g[k]), upstream = 0.0;
    int exact = p->g[k] == floor(p->g[k]);
    *ninf = 0;
    for (int64_t q = beg; q < end; ++q) {
        const double a = p->val[q];
        const int32_t j = p->col[q];
        const double b = (a > 0) ? l[j] : u[j];
        if (isinf(b)) { (*ninf)++; continue; }
        const double t = a * b;
        minfin = minfin + t;
        mag += fabs(t);
        const double ub = dl ? fabs(a) * ((a > 0) ? dl[j] : du[j]) : 0.0;
        upstream += ub;
        if (a != floor(a) || b != floor(b) || ub != 0.0) exact = 0;
    }
    *err = (exact && mag < 1125899906842624.0) ? 0.0 : 2.0 * (fp_gam((double)(end - beg) + 2.0) * mag + upstream);
    return minfin;
}

/* ceil(e / c) for e > 0, c > 0; exact when both are integers below 2^50 */
static double ceil_div(double e, double c)
{
    double d = ceil(e / c);
    if (e == floor(e) && c == floor(c)) {
        while (d > 1.0 && (d - 1.0) * c >= e) d -= 1.0;
        while (d * c < e) d += 1.0;
    }
    return d;
}

/* One repair step after an infeasible propagation whose final bounds are (l, u) (uncertainty dl,
 * du): the infeasible constraint (row k0, or the smallest violated row of the crossing variable
 * w0) and the move of one fixed variable, applied to cval.  Returns the moved variable, or -1
 * when no fixed variable of the row can move.  Fragile decisions are added to *fragile. */
static int32_t repair_step(const orc_problem *p, const double *l, const double *u, const double *dl, const double *du,
                           int32_t k0, int32_t w0, const double *lb0, const double *ub0, const uint8_t *chosen,
                           double *cval, int64_t *fragile)
{
    const double *tl = l, *tu = u, *tdl = dl, *tdu = du;
    int32_t k = k0;
    if (k < 0 && w0 >= 0) {
        const int32_t w = w0;
        for (int64_t s = p->col_ptr[w]; s < p->col_ptr[w + 1]; ++s) {
            const int32_t kk = p->row_idx[s];
            int32_t ninf;
            double err;
            const double mf = row_min_activity(p, kk, tl, tu, tdl, tdu, &ninf, &err);
            const double gt = p->g[kk] + FP_TOL;
            if (ninf || !isfinite(p->g[kk])) continue;
            if (fabs(mf - gt) <= err && err > 0.0) (*fragile)++;
            if (mf > gt && (k < 0 || kk < k)) k = kk;
        }
    }
    if (k < 0) return -1;
    int32_t ninf;
    double err;
    const double e = row_min_activity(p, k, tl, tu, tdl, tdu, &ninf, &err) - p->g[k];
    if (ninf || !(e > 0.0)) return -1;
    int32_t best = -1;
    double best_r = 0.0, best_d = 0.0, best_a = 0.0;
    for (int64_t q = p->row_ptr[k]; q < p->row_ptr[k + 1]; ++q) {
        const int32_t i = p->col[q];
        if (!chosen[i]) continue;
        const double a = p->val[q], aa = fabs(a);
        const double need = ceil_div(e, aa);
        if (err > 0.0 && ceil((e - err) / aa) != ceil((e + err) / aa)) (*fragile)++;
        const double room = a > 0 ? floor(cval[i] - lb0[i]) : floor(ub0[i] - cval[i]);   /* +inf when unbounded */
        const double d = need < room ? need : room;
        if (!(d > 0.0)) continue;
        const double rr = aa * d;
        if (rr > best_r || (rr == best_r && i < best)) {
            best = i;
            best_r = rr;
            best_d = d;
            best_a = a;
        }
    }
    if (best < 0) return -1;
    cval[best] = best_a > 0 ? cval[best] - best_d : cval[best] + best_d;
    return best;
}

/* repair_step for the tests (dl, du may be NULL: exact bounds) */
int32_t orc_repair_step(const orc_problem *p, const double *l, const double *u, int32_t k0, int32_t w0,
                        const double *lb0, const double *ub0, const uint8_t *chosen, double *cval, int64_t *fragile)
{
    *fragile = 0;
    return repair_step(p, l, u, NULL, NULL, k0, w0, lb0, ub0, chosen, cval, fragile);
}

/*
 * Repair (Section 2.3, the repair branch of Algorithm 1; the paper describes it in words only,
 * and this is the reading taken).
 * Called when a one-variable bulk fails both ways, with the variable j and its drawn value v.
 * Every variable fixed by choice so far (chosen, at cval) and j at v are taken as the fixings,
 * and up to `repair_cycles` times:
 *   - propagate the start bounds with the fixings; feasible: the repair succeeds and these
 *     bounds become the current ones;
 *   - else the infeasible constraint: the propagation's first infeasible row, or, when only a
 *     crossing variable is reported, the smallest row of that variable whose minimal activity
 *     under the propagation's final bounds exceeds g + tol;
 *   - for each fixed variable i of that row a shift that alone makes it feasible: its value
 *     moves against its coefficient by d_i = ceil((L_min - g) / |a_i|), at most down to its
 *     start lower bound (a > 0) or up to its start upper bound (a < 0);
 *   - the variable whose shift lowers the minimal activity most (|a_i| d_i, ties to the
 *     smallest index) is shifted, and the next cycle propagates again from the start bounds.
 * Fails when no variable of the row can move or the cycles run out.  Fragile decisions (the
 * violation test and the shift size within the activity's error bound) are counted.
 */
static int repair(const orc_problem *p, const double *lb0, const double *ub0, uint8_t *chosen, double *cval,
                  int32_t j, double v, const orc_fp_params *prm, double *l, double *u, double *dl, double *du,
                  double *tl, double *tu, double *tdl, double *tdu, orc_fp_result *res)
{
    const int32_t n = p->n;
    chosen[j] = 1;
    cval[j] = v;
    for (int32_t c = 0; c < prm->repair_cycles; ++c) {
        memcpy(tl, lb0, sizeof(double) * (size_t)n);
        memcpy(tu, ub0, sizeof(double) * (size_t)n);
        memset(tdl, 0, sizeof(double) * (size_t)n);
        memset(tdu, 0, sizeof(double) * (size_t)n);
        for (int32_t i = 0; i < n; ++i)
            if (chosen[i]) tl[i] = tu[i] = cval[i];
        orc_bp_result r;
        orc_bp(p, tl, tu, tdl, tdu, NULL, 0, prm->theta, prm->max_rounds, 0, &r, NULL, NULL);
        res->bp_runs++;
        res->repair_runs++;
        res->nnz_updates += r.nnz_updates;
        res->fragile += r.fragile;
        if (r.status != ORC_INFEASIBLE) {
            memcpy(l, tl, sizeof(double) * (size_t)n);
            memcpy(u, tu, sizeof(double) * (size_t)n);
            memcpy(dl, tdl, sizeof(double) * (size_t)n);
            memcpy(du, tdu, sizeof(double) * (size_t)n);
            return 1;
        }
        if (repair_step(p, tl, tu, tdl, tdu, r.first_infeasible_row, r.first_infeasible_var, lb0, ub0, chosen, cval,
                        &res->fragile) < 0)
            return 0;
    }
    return 0;
}

int orc_fix_and_propagate(const orc_problem *p, const double *x, const double *lb0, const double *ub0,
                          const orc_cache *cache, const orc_fp_params *prm, double *x_out, orc_fp_result *res)
{
    const int32_t n = p->n;
    memset(res, 0, sizeof(*res));
    if (cache && prm->repair_max > 0) return -1;   /* repair is defined without a probing cache */
    double *l = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *u = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *cl[2], *cu[2];
    for (int i = 0; i < 2; ++i) {
        cl[i] = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
        cu[i] = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    }
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int32_t *work = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    int32_t *cls = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    double *frac = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *S = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *E = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    /* uncertainty of the current bounds and of each candidate vector's (continuous bounds only;
     * the propagations report it, fixings and cached values are exact inputs) */
    double *dl = (double *)calloc((size_t)(n ? n : 1), sizeof(double));
    double *du = (double *)calloc((size_t)(n ? n : 1), sizeof(double));
    double *cdl[2], *cdu[2];
    for (int i = 0; i < 2; ++i) {
        cdl[i] = (double *)calloc((size_t)(n ? n : 1), sizeof(double));
        cdu[i] = (double *)calloc((size_t)(n ? n : 1), sizeof(double));
    }
    double *val[2];
    val[0] = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    val[1] = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    int32_t *recq = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    /* fixings by choice (the repair's fixings) and, per candidate, which bulk fixings were kept */
    uint8_t *chosen = (uint8_t *)calloc((size_t)(n ? n : 1), 1);
    double *cval = (double *)calloc((size_t)(n ? n : 1), sizeof(double));
    uint8_t *keptv[2];
    keptv[0] = (uint8_t *)calloc((size_t)(n ? n : 1), 1);
    keptv[1] = (uint8_t *)calloc((size_t)(n ? n : 1), 1);
    int32_t repairs_tried = 0;
    int32_t *w0 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(p->m ? p->m : 1));
    uint8_t *rowmark = (uint8_t *)calloc((size_t)(p->m ? p->m : 1), 1);
    int32_t *pair_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
    for (int32_t j = 0; j < n; ++j) pair_of[j] = -1;
    if (cache)
        for (int32_t i = cache->npairs - 1; i >= 0; --i) pair_of[cache->var[i]] = i;   /* first pair wins */

    memcpy(l, lb0, sizeof(double) * (size_t)n);
    memcpy(u, ub0, sizeof(double) * (size_t)n);
    orc_bp_result r;
    orc_bp(p, l, u, dl, du, NULL, 0, prm->theta, prm->max_rounds, 0, &r, NULL, NULL);
    res->bp_runs++;
    res->nnz_updates += r.nnz_updates;
    res->fragile += r.fragile;
    int infeasible = r.status == ORC_INFEASIBLE;

    /* initial order (under the propagated start bounds) */
    int64_t nint = 0;
    for (int32_t j = 0; j < n; ++j) {
        if (!p->is_int[j]) continue;
        const double w = u[j] - l[j];
        cls[j] = w <= 1.0 ? 0 : (w == 2.0 ? 1 : 2);
        const double xh = clampd(x[j], l[j], u[j]);
        const double f = xh - floor(xh);
        frac[j] = f < 1.0 - f ? f : 1.0 - f;
        order[nint++] = j;
    }
    sort_ctx ctx = {cls, frac, S, prm->order_score};
    merge_sort(order, tmp, nint, &ctx, cmp_initial);

    int rounding_infeasible = infeasible;
    int64_t nrec = 0, rec_pos = 0;
    uint64_t bulk_index = 0;
    while (!rounding_infeasible) {
        /* unfixed integer variables in the initial order */
        int64_t nun = 0;
        for (int64_t i = 0; i < nint; ++i)
            if (l[order[i]] < u[order[i]]) work[nun++] = order[i];
        if (nun == 0) break;
        int64_t bsize;
        int single = 0;
        int32_t *bulk = work;
        int32_t one;
        while (rec_pos < nrec && !(l[recq[rec_pos]] < u[recq[rec_pos]])) rec_pos++;
        if (rec_pos < nrec) {
            one = recq[rec_pos++];
            bulk = &one;
            bsize = 1;
            single = 1;
        } else {
            nrec = rec_pos = 0;
            if (nun <= prm->last_single) {
                bsize = 1;
            } else if (prm->bulk_rule == 0) {
                bsize = (int64_t)isqrt_ceil((uint64_t)nun);
            } else {
                bsize = (int64_t)ceil(prm->fraction * (double)nint);
                if (bsize < 1) bsize = 1;
            }
            if (bsize > nun) bsize = nun;
            /* a learned order score replaces the per-bulk implied-slack order: the bulks then
             * follow the initial order (class, score, fractionality, index) */
            if (bsize > 1 && !prm->order_score) {
                implied_slack(p, l, u, S);
                merge_sort(work, tmp, nun, &ctx, cmp_slack);
                implied_slack_window(p, l, u, dl, du, E);
                if (slack_sort_fragile(work, nun, bsize, S, E, cache != NULL)) res->fragile++;
            }
            single = bsize == 1;
        }
        /* candidate values */
        for (int64_t i = 0; i < bsize; ++i) {
            const int32_t j = bulk[i];
            const double xh = clampd(x[j], l[j], u[j]);
            const double v0 = clampd(draw_value(xh, prm->seed, bulk_index, j, 0, prm->up_prob), l[j], u[j]);
            double v1;
            if (single) {
                const double fl = floor(xh);
                v1 = clampd(v0 == fl ? fl + 1.0 : fl, l[j], u[j]);
            } else {
                v1 = clampd(draw_value(xh, prm->seed, bulk_index, j, 1, prm->up_prob), l[j], u[j]);
            }
            val[0][j] = v0;
            val[1][j] = v1;
        }
        /* start boxes: kept fixings and their cached implications */
        int kept[2] = {0, 0};
        for (int c = 0; c < 2; ++c) {
            memcpy(cl[c], l, sizeof(double) * (size_t)n);
            memcpy(cu[c], u, sizeof(double) * (size_t)n);
            memcpy(cdl[c], dl, sizeof(double) * (size_t)n);
            memcpy(cdu[c], du, sizeof(double) * (size_t)n);
            for (int64_t i = 0; i < bsize; ++i) {
                const int32_t j = bulk[i];
                const double v = val[c][j];
                keptv[c][i] = 0;
                if (!(v >= cl[c][j] && v <= cu[c][j])) continue;
                const int64_t e = cache_branch(cache, pair_of, j, v);
                int ok = 1;
                if (e >= 0) {
                    if (cache->status[e] == ORC_INFEASIBLE) ok = 0;
                    for (int64_t q = cache->offsets[e]; ok && q < cache->offsets[e + 1]; ++q) {
                        const int32_t w = cache->ent_var[q];
                        const double lo = cache->ent_l[q] > cl[c][w] ? cache->ent_l[q] : cl[c][w];
                        const double hi = cache->ent_u[q] < cu[c][w] ? cache->ent_u[q] : cu[c][w];
                        if (w == j ? !(v >= lo && v <= hi) : var_cross(p->is_int[w], lo, hi)) ok = 0;
                    }
                }
                if (!ok) continue;
                kept[c]++;
                keptv[c][i] = 1;
                cl[c][j] = v;
                cu[c][j] = v;
                cdl[c][j] = cdu[c][j] = 0.0;
                if (e >= 0)
                    for (int64_t q = cache->offsets[e]; q < cache->offsets[e + 1]; ++q) {
                        const int32_t w = cache->ent_var[q];
                        if (w == j) continue;
                        if (cache->ent_l[q] > cl[c][w]) { cl[c][w] = cache->ent_l[q]; cdl[c][w] = 0.0; }
                        if (cache->ent_u[q] < cu[c][w]) { cu[c][w] = cache->ent_u[q]; cdu[c][w] = 0.0; }
                    }
            }
        }
        /* double propagation */
        int feasible[2] = {0, 0};
        for (int c = 0; c < 2; ++c) {
            if (!kept[c]) continue;
            int32_t nw = 0;
            memset(rowmark, 0, (size_t)p->m);
            for (int32_t j = 0; j < n; ++j) {
                if (cl[c][j] == l[j] && cu[c][j] == u[j]) continue;
                for (int64_t s = p->col_ptr[j]; s < p->col_ptr[j + 1]; ++s) rowmark[p->row_idx[s]] = 1;
            }
            for (int32_t k = 0; k < p->m; ++k)
                if (rowmark[k]) w0[nw++] = k;
            orc_bp(p, cl[c], cu[c], cdl[c], cdu[c], w0, nw, prm->theta, prm->max_rounds, 0, &r, NULL, NULL);
            res->bp_runs++;
            res->nnz_updates += r.nnz_updates;
            res->fragile += r.fragile;
            feasible[c] = r.status != ORC_INFEASIBLE;
        }
        res->bulks++;
        bulk_index++;
        const int pick = feasible[0] ? 0 : (feasible[1] ? 1 : -1);
        if (pick >= 0) {
            res->fixed_by_choice += kept[pick];
            for (int64_t i = 0; i < bsize; ++i)
                if (keptv[pick][i]) {
                    chosen[bulk[i]] = 1;
                    cval[bulk[i]] = val[pick][bulk[i]];
                }
            memcpy(l, cl[pick], sizeof(double) * (size_t)n);
            memcpy(u, cu[pick], sizeof(double) * (size_t)n);
            memcpy(dl, cdl[pick], sizeof(double) * (size_t)n);
            memcpy(du, cdu[pick], sizeof(double) * (size_t)n);
        } else if (!single) {
            memcpy(recq, bulk, sizeof(int32_t) * (size_t)bsize);
            nrec = bsize;
            rec_pos = 0;
            res->recoveries++;
        } else if (repairs_tried < prm->repair_max) {
            /* a single variable failing both ways: repair (off unless repair_max > 0) */
            repairs_tried++;
            if (repair(p, lb0, ub0, chosen, cval, bulk[0], val[0][bulk[0]], prm, l, u, dl, du, cl[0], cu[0], cdl[0],
                       cdu[0], res))
                res->repairs++;
            else
                rounding_infeasible = 1;
        } else {
            rounding_infeasible = 1;
        }
    }
    /* remaining integer variables: nearest value inside the bounds, no propagation */
    for (int64_t i = 0; i < nint; ++i) {
        const int32_t j = order[i];
        if (l[j] < u[j]) {
            const double v = clampd(floor(clampd(x[j], l[j], u[j]) + 0.5), l[j], u[j]);
            l[j] = u[j] = v;
        }
    }
    for (int32_t j = 0; j < n; ++j) {
        if (p->is_int[j]) {
            x_out[j] = l[j];
        } else {
            x_out[j] = clampd(x[j], l[j], u[j]);
        }
    }
    /* final check: the start bounds with every integer variable fixed at its value */
    if (!rounding_infeasible) {
        memcpy(l, lb0, sizeof(double) * (size_t)n);
        memcpy(u, ub0, sizeof(double) * (size_t)n);
        for (int32_t j = 0; j < n; ++j)
            if (p->is_int[j]) l[j] = u[j] = x_out[j];
        orc_bp(p, l, u, NULL, NULL, NULL, 0, prm->theta, prm->max_rounds, 0, &r, NULL, NULL);
        res->fragile += r.fragile;
        if (r.status == ORC_INFEASIBLE) res->refuted = 1;
    }
    res->status = (rounding_infeasible || res->refuted) ? 1 : 0;
    for (int i = 0; i < 2; ++i) { free(cl[i]); free(cu[i]); free(val[i]); free(cdl[i]); free(cdu[i]); }
    free(l); free(u); free(order); free(work); free(tmp); free(cls); free(frac); free(S); free(E); free(dl); free(du);
    free(recq); free(w0); free(rowmark); free(pair_of);
    free(chosen); free(cval); free(keptv[0]); free(keptv[1]);
    return 0;
}
