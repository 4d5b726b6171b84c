/*
 * ara_oracle.c -- plain FP64 CPU oracle for aggregate risk analysis.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * execute this file: only the tests, the smoke check and the bench's CPU
 * baseline use it. It shares no code with the CUDA library.
 *
 * What it computes (Section II, Algorithm 1 of Bahl et al., "Achieving
 * Speedup in Aggregate Risk Analysis using Multiple GPUs"):
 *
 *   For layer j with ELT set E_j and trial t with events E_{t,1..K_t}
 *     x_d   = sum_{e in E_j} F_e(l_e[E_{t,d}])        (steps 1 and 2)
 *     o_d   = O_j(x_d)                                (step 3, occurrence)
 *     S     = sum_d o_d                               (cumulative sum)
 *     Y_t,j = A_j(S)                                  (step 4, aggregate)
 *   with XL(v; R, L) = min(max(v - R, 0), L),
 *     F_e = XL(m_e * y; D_e, Lim_e)   (per-ELT financial terms, a reading:
 *                                       the paper leaves the form open),
 *     O_j = XL(.; OccR_j, OccL_j), A_j = XL(.; AggR_j, AggL_j).
 *
 * The paper's Algorithm 1 carries the aggregate as a running form: cumulative
 * sums C_d, aggregate terms on each C_d, per-event differences, and the trial
 * loss lr as their sum. Because A(0) = 0 for AggR >= 0 the differences
 * telescope and lr = A(C_K) = A(S). ara_oracle_ylt evaluates the closed form;
 * ara_oracle_ylt_running follows the algorithm's step order and also returns
 * the per-event payouts p_d = A(C_d) - A(C_{d-1}).
 *
 * Everything is FP64. Losses arrive as the FP32 direct-access tables the
 * method stores (Section III); terms arrive as doubles so that tests can
 * perturb them by amounts FP32 cannot represent.
 *
 * Readings of the paper taken here (where it is silent or garbled):
 *   - the garbled lookup of Algorithm 1 step 1 reads "x_d is the loss, in
 *     ELT c, of the event at trial position d"; absent events have loss 0;
 *   - accumulators are indexed by trial position d, not by event id, so an
 *     event that occurs twice in a trial counts twice;
 *   - lo is reset per (layer, trial) and lr per (layer, trial);
 *   - the in-place difference uses the un-overwritten cumulative values,
 *     with C_0 = 0.
 *
 * PML and TVaR are named in Section I but not defined there. Reading: with
 * k = ceil((1-p) N) (at least 1), PML_p is the k-th largest trial loss and
 * TVaR_p the mean of the k largest. The expected layer loss is the mean.
 *
 * Gradients (for the pricing-sensitivity pattern; the paper has none): Y is
 * piecewise linear in every term; at a kink the derivative of the branch
 * with strict inequalities is taken (so "mid" means R < v < R + L).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1

/* XL(v; R, L) = min(max(v - R, 0), L): the excess-of-loss form shared by the
 * occurrence terms (Algorithm 1 step 3) and the aggregate terms (step 4). */
static double xl(double v, double ret, double lim)
{
    double w = v - ret;
    if (w < 0.0) w = 0.0;
    if (w > lim) w = lim;
    return w;
}

/* Branch of XL with strict inequalities: 0 below or at the retention,
 * 1 strictly between, 2 strictly above retention + limit. */
static int xl_branch(double v, double ret, double lim)
{
    double w = v - ret;
    if (!(w > 0.0)) return 0;
    if (w > lim) return 2;
    if (w < lim) return 1;
    return 0; /* exactly at the cap: treated like a flat piece */
}

typedef struct {
    int32_t catalogue_size;
    int32_t n_elt;
    const float *elt_losses;            /* [n_elt][catalogue_size] */
    const double *elt_mult, *elt_ded, *elt_lim;
    int32_t n_layers;
    const int32_t *layer_elt_off;       /* [n_layers + 1] */
    const int32_t *layer_elt_ids;
    const double *occ_ret, *occ_lim, *agg_ret, *agg_lim;
    const int32_t *event_ids;
    const int64_t *trial_off;           /* [n_trials + 1] or NULL (dense) */
    int32_t events_per_trial;           /* used when trial_off is NULL */
    int64_t n_trials;
} problem;

static int64_t trial_begin(const problem *p, int64_t t)
{
    return p->trial_off ? p->trial_off[t] : t * (int64_t)p->events_per_trial;
}
static int64_t trial_end(const problem *p, int64_t t)
{
    return p->trial_off ? p->trial_off[t + 1] : (t + 1) * (int64_t)p->events_per_trial;
}

static int validate(const problem *p, const int64_t *trials, int64_t n_out)
{
    if (p->catalogue_size < 0 || p->n_elt < 0 || p->n_layers < 0 || p->n_trials < 0) return ORACLE_EINVAL;
    if (p->n_layers > 0 && p->layer_elt_off[0] != 0) return ORACLE_EINVAL;
    for (int32_t j = 0; j < p->n_layers; ++j) {
        if (p->layer_elt_off[j + 1] < p->layer_elt_off[j]) return ORACLE_EINVAL;
        for (int32_t i = p->layer_elt_off[j]; i < p->layer_elt_off[j + 1]; ++i)
            if (p->layer_elt_ids[i] < 0 || p->layer_elt_ids[i] >= p->n_elt) return ORACLE_EINVAL;
    }
    for (int64_t i = 0; i < n_out; ++i) {
        int64_t t = trials ? trials[i] : i;
        if (t < 0 || t >= p->n_trials) return ORACLE_EINVAL;
        for (int64_t d = trial_begin(p, t); d < trial_end(p, t); ++d)
            if (p->event_ids[d] < 0 || p->event_ids[d] >= p->catalogue_size) return ORACLE_EINVAL;
    }
    return ORACLE_OK;
}

/* Steps 1-2 for one event: x = sum over the layer's ELTs of F_e(l_e[id]);
 * also the gross loss g = sum of m_e * l_e[id] before any terms. */
static double event_layer_loss(const problem *p, int32_t j, int32_t id, double *gross)
{
    double x = 0.0, g = 0.0;
    for (int32_t i = p->layer_elt_off[j]; i < p->layer_elt_off[j + 1]; ++i) {
        int32_t e = p->layer_elt_ids[i];
        double y = (double)p->elt_losses[(int64_t)e * p->catalogue_size + id];
        g += p->elt_mult[e] * y;
        x += xl(p->elt_mult[e] * y, p->elt_ded[e], p->elt_lim[e]);
    }
    if (gross) *gross = g;
    return x;
}

/* Closed form: Y = A(sum_d O(x_d)). Outputs are [n_layers][n_out]; row i
 * of the outputs is trial trials[i] (or trial i when trials is NULL). */
static int ylt_closed(const problem *p, const int64_t *trials, int64_t n_out,
                      double *ylt, double *gross, double *agg_sum)
{
    int rc = validate(p, trials, n_out);
    if (rc) return rc;
    int64_t n_work = (int64_t)p->n_layers * n_out;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t w = 0; w < n_work; ++w) {
        int32_t j = (int32_t)(w / n_out);
        int64_t i = w % n_out;
        int64_t t = trials ? trials[i] : i;
        double s = 0.0, g = 0.0;
        for (int64_t d = trial_begin(p, t); d < trial_end(p, t); ++d) {
            double gd;
            double x = event_layer_loss(p, j, p->event_ids[d], &gd);
            s += xl(x, p->occ_ret[j], p->occ_lim[j]);
            g += gd;
        }
        ylt[w] = xl(s, p->agg_ret[j], p->agg_lim[j]);
        if (gross) gross[w] = g;
        if (agg_sum) agg_sum[w] = s;
    }
    return ORACLE_OK;
}

int ara_oracle_ylt(int32_t catalogue_size, int32_t n_elt, const float *elt_losses,
                   const double *elt_mult, const double *elt_ded, const double *elt_lim,
                   int32_t n_layers, const int32_t *layer_elt_off, const int32_t *layer_elt_ids,
                   const double *occ_ret, const double *occ_lim,
                   const double *agg_ret, const double *agg_lim,
                   const int32_t *event_ids, const int64_t *trial_off, int32_t events_per_trial,
                   int64_t n_trials, const int64_t *trials, int64_t n_out,
                   double *ylt, double *gross, double *agg_sum)
{
    problem p = {catalogue_size, n_elt, elt_losses, elt_mult, elt_ded, elt_lim,
                 n_layers, layer_elt_off, layer_elt_ids, occ_ret, occ_lim, agg_ret, agg_lim,
                 event_ids, trial_off, events_per_trial, n_trials};
    return ylt_closed(&p, trials, n_out, ylt, gross, agg_sum);
}

/* Running form, in Algorithm 1's step order for one (layer, trial):
 *   per ELT: look up every event, apply the financial terms, accumulate;
 *   occurrence terms per event; cumulative sum; aggregate terms on each
 *   cumulative value; per-event difference; sum into lr.
 * payouts (optional) receives p_d for every event of every selected trial,
 * laid out [n_layers][sum of the selected trials' lengths], trials in the
 * order given. */
int ara_oracle_ylt_running(int32_t catalogue_size, int32_t n_elt, const float *elt_losses,
                           const double *elt_mult, const double *elt_ded, const double *elt_lim,
                           int32_t n_layers, const int32_t *layer_elt_off, const int32_t *layer_elt_ids,
                           const double *occ_ret, const double *occ_lim,
                           const double *agg_ret, const double *agg_lim,
                           const int32_t *event_ids, const int64_t *trial_off, int32_t events_per_trial,
                           int64_t n_trials, const int64_t *trials, int64_t n_out,
                           double *lr_out, double *payouts)
{
    problem p = {catalogue_size, n_elt, elt_losses, elt_mult, elt_ded, elt_lim,
                 n_layers, layer_elt_off, layer_elt_ids, occ_ret, occ_lim, agg_ret, agg_lim,
                 event_ids, trial_off, events_per_trial, n_trials};
    int rc = validate(&p, trials, n_out);
    if (rc) return rc;
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_out + 1));
    if (!pos) return ORACLE_EINVAL;
    pos[0] = 0;
    for (int64_t i = 0; i < n_out; ++i) {
        int64_t t = trials ? trials[i] : i;
        pos[i + 1] = pos[i] + (trial_end(&p, t) - trial_begin(&p, t));
    }
    int64_t total = pos[n_out];
    int64_t n_work = (int64_t)n_layers * n_out;
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : failed)
    for (int64_t w = 0; w < n_work; ++w) {
        int32_t j = (int32_t)(w / n_out);
        int64_t i = w % n_out;
        int64_t t = trials ? trials[i] : i;
        int64_t b = trial_begin(&p, t), k = trial_end(&p, t) - b;
        double *x = (double *)calloc((size_t)(k > 0 ? k : 1), sizeof(double));
        double *l = (double *)calloc((size_t)(k > 0 ? k : 1), sizeof(double));
        double *lo = (double *)calloc((size_t)(k > 0 ? k : 1), sizeof(double));
        double *cum = (double *)calloc((size_t)(k > 0 ? k : 1), sizeof(double));
        if (!x || !l || !lo || !cum) { failed = 1; free(x); free(l); free(lo); free(cum); continue; }
        /* steps 1-2, once per ELT of the layer */
        for (int32_t c = layer_elt_off[j]; c < layer_elt_off[j + 1]; ++c) {
            int32_t e = layer_elt_ids[c];
            for (int64_t d = 0; d < k; ++d)        /* look up each event's loss */
                x[d] = (double)elt_losses[(int64_t)e * catalogue_size + event_ids[b + d]];
            for (int64_t d = 0; d < k; ++d)        /* apply the financial terms */
                l[d] = xl(elt_mult[e] * x[d], elt_ded[e], elt_lim[e]);
            for (int64_t d = 0; d < k; ++d)        /* accumulate across ELTs */
                lo[d] += l[d];
        }
        /* step 3: occurrence terms */
        for (int64_t d = 0; d < k; ++d) lo[d] = xl(lo[d], occ_ret[j], occ_lim[j]);
        /* cumulative sum */
        for (int64_t d = 0; d < k; ++d) cum[d] = lo[d] + (d ? cum[d - 1] : 0.0);
        /* step 4: aggregate terms on every cumulative value */
        for (int64_t d = 0; d < k; ++d) cum[d] = xl(cum[d], agg_ret[j], agg_lim[j]);
        /* per-event difference, then the trial loss */
        double lr = 0.0;
        for (int64_t d = 0; d < k; ++d) {
            double pd = cum[d] - (d ? cum[d - 1] : 0.0); /* nothing is paid before the first event */
            if (payouts) payouts[(int64_t)j * total + pos[i] + d] = pd;
            lr += pd;
        }
        lr_out[w] = lr;
        free(x); free(l); free(lo); free(cum);
    }
    free(pos);
    return failed ? ORACLE_EINVAL : ORACLE_OK;
}

/* k = ceil((1 - p) N), at least 1 and at most N. (1 - p) N is computed in
 * FP64; when it lies within 1e-9 N of an integer that integer is taken, so
 * that 0.01 * 10000 (which FP64 evaluates a hair above 100) gives 100. */
int64_t ara_oracle_tail_count(double p, int64_t n)
{
    if (n <= 0) return 0;
    double q = (1.0 - p) * (double)n;
    double r = nearbyint(q);
    int64_t k = (fabs(q - r) <= 1e-9 * (double)n) ? (int64_t)r : (int64_t)ceil(q);
    if (k < 1) k = 1;
    if (k > n) k = n;
    return k;
}

static int cmp_desc(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) - (x > y);
}

/* Per layer: mean, PML_p (k-th largest) and TVaR_p (mean of the k largest),
 * by a full sort of the layer's trial losses. Outputs: mean [n_layers],
 * pml and tvar [n_layers][n_p]. */
int ara_oracle_metrics(const double *ylt, int64_t n_trials, int32_t n_layers,
                       const double *probs, int32_t n_p,
                       double *mean, double *pml, double *tvar)
{
    if (n_trials <= 0 || n_layers < 0 || n_p < 0) return ORACLE_EINVAL;
    for (int32_t q = 0; q < n_p; ++q)
        if (!(probs[q] > 0.0 && probs[q] < 1.0)) return ORACLE_EINVAL;
    double *buf = (double *)malloc(sizeof(double) * (size_t)n_trials);
    if (!buf) return ORACLE_EINVAL;
    for (int32_t j = 0; j < n_layers; ++j) {
        const double *y = ylt + (int64_t)j * n_trials;
        double s = 0.0;
        for (int64_t t = 0; t < n_trials; ++t) s += y[t];
        mean[j] = s / (double)n_trials;
        memcpy(buf, y, sizeof(double) * (size_t)n_trials);
        qsort(buf, (size_t)n_trials, sizeof(double), cmp_desc);
        for (int32_t q = 0; q < n_p; ++q) {
            int64_t k = ara_oracle_tail_count(probs[q], n_trials);
            double top = 0.0;
            for (int64_t i = 0; i < k; ++i) top += buf[i];
            pml[(int64_t)j * n_p + q] = buf[k - 1];
            tvar[(int64_t)j * n_p + q] = top / (double)k;
        }
    }
    free(buf);
    return ORACLE_OK;
}

/* Analytic gradient of sum_{t,j} g_{t,j} Y_{t,j} with respect to the layer
 * terms (OccR, OccL, AggR, AggL per layer) and the ELT multipliers m_e:
 *   dY/dAggR = -a,  dY/dAggL = c,  a = [AggR < S < AggR+AggL], c = [S > AggR+AggL]
 *   dY/dOccR = -a * #{d : OccR < x_d < OccR+OccL}
 *   dY/dOccL =  a * #{d : x_d > OccR+OccL}
 *   dY/dm_e  =  a * sum_d [o_d mid] [D_e < m_e l < D_e + Lim_e] l,  l = l_e[E_d]
 * grad_terms is [n_layers][4] (OccR, OccL, AggR, AggL), grad_mult [n_elt].
 * per_trial (optional) receives, for row w = j * n_out + i, the 4 + n_elt
 * partial derivatives of Y_{t,j} itself (unweighted).
 * pattern (optional) receives a 64-bit FNV-1a hash of every branch taken in
 * (layer j, trial t): F branch per (event, ELT), O branch per event, A branch.
 * Equal hashes at two parameter points mean the same linear piece. */
int ara_oracle_grad(int32_t catalogue_size, int32_t n_elt, const float *elt_losses,
                    const double *elt_mult, const double *elt_ded, const double *elt_lim,
                    int32_t n_layers, const int32_t *layer_elt_off, const int32_t *layer_elt_ids,
                    const double *occ_ret, const double *occ_lim,
                    const double *agg_ret, const double *agg_lim,
                    const int32_t *event_ids, const int64_t *trial_off, int32_t events_per_trial,
                    int64_t n_trials, const int64_t *trials, int64_t n_out,
                    const double *grad_ylt, double *grad_terms, double *grad_mult,
                    double *per_trial, uint64_t *pattern)
{
    problem p = {catalogue_size, n_elt, elt_losses, elt_mult, elt_ded, elt_lim,
                 n_layers, layer_elt_off, layer_elt_ids, occ_ret, occ_lim, agg_ret, agg_lim,
                 event_ids, trial_off, events_per_trial, n_trials};
    int rc = validate(&p, trials, n_out);
    if (rc) return rc;
    const int64_t width = 4 + (int64_t)n_elt;
    int64_t n_work = (int64_t)n_layers * n_out;
    double *rows = per_trial ? per_trial : (double *)calloc((size_t)(n_work > 0 ? n_work : 1) * (size_t)width, sizeof(double));
    if (!rows) return ORACLE_EINVAL;
    if (per_trial) memset(per_trial, 0, sizeof(double) * (size_t)n_work * (size_t)width);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t w = 0; w < n_work; ++w) {
        int32_t j = (int32_t)(w / n_out);
        int64_t i = w % n_out;
        int64_t t = trials ? trials[i] : i;
        double *row = rows + w * width;
        uint64_t h = 1469598103934665603ull;
        double s = 0.0, n_occ_mid = 0.0, n_occ_cap = 0.0;
        double *dm = row + 4;
        /* first pass: S and the per-event indicators (dm holds the sums of
         * [o_d mid][F mid] l before the factor a) */
        for (int64_t d = trial_begin(&p, t); d < trial_end(&p, t); ++d) {
            int32_t id = event_ids[d];
            double x = 0.0;
            for (int32_t c = layer_elt_off[j]; c < layer_elt_off[j + 1]; ++c) {
                int32_t e = layer_elt_ids[c];
                double y = (double)elt_losses[(int64_t)e * catalogue_size + id];
                x += xl(elt_mult[e] * y, elt_ded[e], elt_lim[e]);
                h = (h ^ (uint64_t)(xl_branch(elt_mult[e] * y, elt_ded[e], elt_lim[e]) + 1)) * 1099511628211ull;
            }
            int ob = xl_branch(x, occ_ret[j], occ_lim[j]);
            h = (h ^ (uint64_t)(ob + 7)) * 1099511628211ull;
            s += xl(x, occ_ret[j], occ_lim[j]);
            if (ob == 1) {
                n_occ_mid += 1.0;
                for (int32_t c = layer_elt_off[j]; c < layer_elt_off[j + 1]; ++c) {
                    int32_t e = layer_elt_ids[c];
                    double y = (double)elt_losses[(int64_t)e * catalogue_size + id];
                    if (xl_branch(elt_mult[e] * y, elt_ded[e], elt_lim[e]) == 1) dm[e] += y;
                }
            } else if (ob == 2) {
                n_occ_cap += 1.0;
            }
        }
        int ab = xl_branch(s, agg_ret[j], agg_lim[j]);
        h = (h ^ (uint64_t)(ab + 13)) * 1099511628211ull;
        double a = (ab == 1) ? 1.0 : 0.0, cc = (ab == 2) ? 1.0 : 0.0;
        row[0] = -a * n_occ_mid;
        row[1] = a * n_occ_cap;
        row[2] = -a;
        row[3] = cc;
        for (int32_t e = 0; e < n_elt; ++e) dm[e] *= a;
        if (pattern) pattern[w] = h;
    }
    /* weighted sums, in a fixed order */
    for (int32_t j = 0; j < n_layers; ++j)
        for (int q = 0; q < 4; ++q) grad_terms[j * 4 + q] = 0.0;
    for (int32_t e = 0; e < n_elt; ++e) grad_mult[e] = 0.0;
    for (int64_t w = 0; w < n_work; ++w) {
        int32_t j = (int32_t)(w / n_out);
        double g = grad_ylt[w];
        const double *row = rows + w * width;
        if (g == 0.0) continue;
        for (int q = 0; q < 4; ++q) grad_terms[j * 4 + q] += g * row[q];
        for (int32_t e = 0; e < n_elt; ++e) grad_mult[e] += g * row[4 + e];
    }
    if (!per_trial) free(rows);
    return ORACLE_OK;
}

int ara_oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
