/*
 * farm_oracle.c -- plain FP64 CPU oracle of FARM's query-time relational
 * retrieval ("Find Anything using Relational Spatial Memory").
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package's smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, helper or constant table with the CUDA path, and the product path
 * never calls it.
 *
 * It evaluates the method's plain definition over all N objects, with no
 * pruning, blocking or reordering beyond what the definition states:
 *
 *   score(e; q, M) = max over bindings eta with eta(x*) = e of Verify(eta),
 *   y_hat = TopK_e score(e)                                (Sec. 2.3; App. B)
 *
 * with Verify = Agg as given in App. D.2 step 5 ("Composite scoring") and in
 * the "Why soft, not hard?" paragraph:
 *
 *   s(e) = s_sem(e) * [(1 - w) + w * gbar(e)],   gbar = geometric mean of the
 *   predicate scores t_i(e),  w = 0.5, s_sem scaled by 0.3 on a class mismatch.
 *
 * Because Agg is non-decreasing in every t_i and the anchors of a star-shaped
 * query are independent once the target is fixed, the best binding takes each
 * anchor's best witness separately (App. B, "Query-time complexity"):
 * t_i(e) = max over a in L_i, a != e of r_rho_i(e, a).
 *
 * The steps, in the order the paper gives them (App. D.2 steps 3-5):
 *  1. cos_ij = <u_i/|u_i|, d_j/|d_j|> for the target row (i = 0) and every
 *     constraint's landmark row (App. D.2 step 3, one embedding channel).
 *  2. rank_i(j) = 1 + #{j' : cos_ij' > cos_ij, or equal and j' < j}.
 *  3. s_sem(j) = cf(j) / (mu + rank_0(j)), mu = 5, one reciprocal-rank-fusion
 *     channel of weight 1; cf = class_mis if the query names a target class
 *     and c_j differs from it, else 1 (App. D.2 steps 3 and 5).
 *  4. L_i = the K_a objects of smallest rank_i ("landmarks are bound greedily
 *     to their top-scoring candidates", App. D.2 step 4).
 *  5. Closed-form relation scores over the object geometry (App. D.2 step 4):
 *       above(e,a) = sig((z_e - z_a)/tau_v), below(e,a) = sig((z_a - z_e)/tau_v)
 *       near(e,a)  = exp(-|p_e - p_a|^2 / (2 sigma_near^2)), sigma_near = 0.5 m
 *       left_of / right_of: evaluated in the stored views of the target
 *       candidate e; per view the horizontal image-plane coordinate
 *       u = X/Z of each centre (X along the camera's right vector f x z_up,
 *       Z along the viewing direction f); a view counts when both depths
 *       exceed z_min; left_of = mean over counted views of
 *       sig((u_a - u_e)/tau_h), right_of = mean of sig((u_e - u_a)/tau_h);
 *       0.5 when no view counts.
 *       next_to(e,a) = exp(-|p_e - p_a|^2 / (2 sigma_next^2)), sigma_next = 1.0 m
 *       on(e,a) = gate * band: gate = sig((rho_a - d_xy)/on_gate) with rho_a
 *       half the landmark's larger horizontal size and d_xy the horizontal
 *       centre distance; band = exp(-g^2 / (2 on_band^2)) with g the gap
 *       between e's bottom and a's top.
 *       in_front_of / behind: in the same counted views of e,
 *       sig((Z_a - Z_e)/tau_d) (e nearer the camera) and sig((Z_e - Z_a)/tau_d);
 *       mean over counted views, 0.5 when none counts.
 *       closest / farthest: a rank within the candidate set C = the k_closest
 *       objects of smallest target rank (step 2): rank_d(e) = 1 + #{j in
 *       C \ {a} : |p_j - p_a| < |p_e - p_a|, or equal and j < e};
 *       closest = 1 / rank_d, farthest = 1 / (|C \ {a}| - rank_d + 1)
 *       (score = 1/(|rank - r*| + 1) with r* = 1 or |C \ {a}|); 0 when e is
 *       not in C.
 *       near_h: the Hellinger form of Near (Sec. 2.3): each object is the
 *       Gaussian whose mean is its box centre and whose covariance is the
 *       covariance of the uniform distribution over its box,
 *       diag(s_x^2, s_y^2, s_z^2) / 12; with the Bhattacharyya coefficient
 *       BC = integral of sqrt(N_e N_a), the Hellinger distance is
 *       H = sqrt(1 - BC) and near_h(e,a) = 1 - H (= BC / (1 + H)).  For diagonal Gaussians
 *       BC = prod_k sqrt(2 sd_ek sd_ak / (sd_ek^2 + sd_ak^2))
 *            * exp(-sum_k dp_k^2 / (4 (sd_ek^2 + sd_ak^2)))
 *       with sd the per-axis standard deviations and dp the centre offset
 *       (an axis on which both objects have zero extent contributes 1 when
 *       their centres agree on it, else 0).
 *       inside(e,a): the containment test of App. D.2 step 4 as the fraction
 *       of e's box volume that lies in a's box, the product over the three
 *       axes of |[e] cap [a]|_k / s_ek (an axis of zero extent contributes 1
 *       when e's coordinate lies in a's interval, else 0).
 *       between(e, a_p, a_q): the ternary relation of App. B ("Between
 *       couples only the variables it mentions"); the paper gives no
 *       evaluator, the reading taken is: with the segment from a_p's centre to
 *       a_q's, t = position of e's centre projected on it (0 at a_p, 1 at a_q)
 *       and d its distance from the line,
 *         between = sig(t / tau_b) sig((1 - t) / tau_b) exp(-d^2 / (2 sigma_near^2)),
 *       tau_b = 0.1; 0 when the two centres coincide.  A Between occupies two
 *       consecutive constraints (codes ORC_BETWEEN, ORC_BETWEEN_AND), each with
 *       its own landmark embedding and candidate list, and is one factor of
 *       the geometric mean of step 7; its witness is the best pair
 *       (a_p, a_q) in L_p x L_q with a_p != a_q, neither the target (exact
 *       bucket elimination of the pair, App. B), lower a_p then lower a_q on
 *       ties; both constraints report that score.
 *  6. t_i(e) = max_{a in L_i, a != e} r_rho_i(e, a), 0 without a witness; the
 *     bound anchor is the argmax (lower object index on ties).
 *  7. gbar = (prod_i t_i)^(1/m) (0 if some t_i = 0, 1 if m = 0);
 *     s = s_sem * ((1 - w) + w * gbar).
 *  8. TopK by s descending, lower object index first on ties.
 *
 * Readings where the paper is silent (the same list is kept with the design
 * notes): one retrieval channel; Near is the Gaussian of App. D.2, and the
 * Hellinger wording of Sec. 2.3 is the separate predicate near_h; box centres stand in for Gaussian means and
 * mask centroids; mean over views; the constants tau_v, tau_h, z_min are
 * parameters; a landmark may not be the target itself; ties go to the lower
 * object index.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_ABOVE 0
#define ORC_BELOW 1
#define ORC_LEFT_OF 2
#define ORC_RIGHT_OF 3
#define ORC_NEAR 4
#define ORC_NEXT_TO 5
#define ORC_ON 6
#define ORC_IN_FRONT_OF 7
#define ORC_BEHIND 8
#define ORC_CLOSEST 9
#define ORC_FARTHEST 10
#define ORC_NEAR_H 11
#define ORC_INSIDE 12
#define ORC_BETWEEN 13      /* first landmark of a Between pair: the next constraint is its second */
#define ORC_BETWEEN_AND 14  /* second landmark of a Between pair */

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2

typedef struct {
    double mu;          /* reciprocal-rank offset (5) */
    double w;           /* blend weight (0.5) */
    double class_mis;   /* class-mismatch factor (0.3) */
    double sigma_near;  /* Near Gaussian width, metres (0.5) */
    double tau_v;       /* Above/Below sigmoid scale, metres */
    double tau_h;       /* LeftOf/RightOf sigmoid scale, image units */
    double z_min;       /* minimum camera depth for a view to count, metres */
    int64_t k_anchor;   /* landmark candidates per constraint (K_a) */
    double sigma_next;  /* NextTo Gaussian width, metres (1.0) */
    double on_gate;     /* On: horizontal gate sigmoid scale, metres */
    double on_band;     /* On: vertical band width, metres */
    double tau_d;       /* InFrontOf/Behind depth sigmoid scale, metres */
    int64_t k_closest;  /* Closest/Farthest: target candidates ranked (the set C) */
} orc_params;

typedef struct {
    int64_t n;
    int64_t dim;
    const float *desc;   /* [n, dim] */
    const int32_t *cls;  /* [n] */
    const float *box;    /* [6, n]: cx, cy, cz, sx, sy, sz */
    int64_t n_views;
    const float *views;  /* [6, n_views, n]: ox, oy, oz, fx, fy, fz */
} orc_scene;

/* ------------------------------------------------------------------ */
/* Elementary pieces                                                   */
/* ------------------------------------------------------------------ */

double orc_sigmoid(double x)
{
    if (x >= 0.0) {
        return 1.0 / (1.0 + exp(-x));
    }
    double ex = exp(x);
    return ex / (1.0 + ex);
}

static double center(const orc_scene *s, int axis, int64_t j)
{
    return (double)s->box[(int64_t)axis * s->n + j];
}

static double view_comp(const orc_scene *s, int comp, int64_t v, int64_t j)
{
    return (double)s->views[((int64_t)comp * s->n_views + v) * s->n + j];
}

/* Left/right (depth = 0) or front/behind (depth = 1) in the stored views of
 * e (step 5).  sign = +1 for left_of / in_front_of, -1 for right_of / behind. */
static double viewpoint_rel(const orc_scene *s, const orc_params *p, int64_t e,
                            int64_t a, double sign, int depth)
{
    double acc = 0.0;
    int64_t counted = 0;
    for (int64_t v = 0; v < s->n_views; ++v) {
        double ox = view_comp(s, 0, v, e), oy = view_comp(s, 1, v, e), oz = view_comp(s, 2, v, e);
        double fx = view_comp(s, 3, v, e), fy = view_comp(s, 4, v, e), fz = view_comp(s, 5, v, e);
        double fn = sqrt(fx * fx + fy * fy + fz * fz);
        if (!(fn > 0.0)) continue;
        fx /= fn; fy /= fn; fz /= fn;
        /* right vector r = f x z_up = (fy, -fx, 0), normalised */
        double rx = fy, ry = -fx;
        double rn = sqrt(rx * rx + ry * ry);
        if (!(rn > 0.0)) continue;  /* camera looking straight up or down */
        rx /= rn; ry /= rn;
        double dex = center(s, 0, e) - ox, dey = center(s, 1, e) - oy, dez = center(s, 2, e) - oz;
        double dax = center(s, 0, a) - ox, day = center(s, 1, a) - oy, daz = center(s, 2, a) - oz;
        double Ze = dex * fx + dey * fy + dez * fz;
        double Za = dax * fx + day * fy + daz * fz;
        if (!(Ze > p->z_min && Za > p->z_min)) continue;
        if (depth) {
            acc += orc_sigmoid(sign * (Za - Ze) / p->tau_d);
        } else {
            double Xe = dex * rx + dey * ry;
            double Xa = dax * rx + day * ry;
            double ue = Xe / Ze, ua = Xa / Za;
            acc += orc_sigmoid(sign * (ua - ue) / p->tau_h);
        }
        counted += 1;
    }
    if (counted == 0) return 0.5;
    return acc / (double)counted;
}

static double box_size(const orc_scene *s, int axis, int64_t j)
{
    return (double)s->box[(int64_t)(3 + axis) * s->n + j];
}

static double dist2(const orc_scene *s, int64_t i, int64_t j)
{
    double dx = center(s, 0, i) - center(s, 0, j);
    double dy = center(s, 1, i) - center(s, 1, j);
    double dz = center(s, 2, i) - center(s, 2, j);
    return dx * dx + dy * dy + dz * dz;
}

/* Hellinger form of Near (step 5): 1 - H(N_e, N_a) with box-moment Gaussians.
 * With per-axis variances s^2 / 12 the factor 2 sd_e sd_a / (sd_e^2 + sd_a^2)
 * is 2 |s_e| |s_a| / (s_e^2 + s_a^2) and the exponent d^2 / (4 (sd_e^2 + sd_a^2))
 * is 3 d^2 / (s_e^2 + s_a^2). */
static double near_hellinger(const orc_scene *s, int64_t e, int64_t a)
{
    double bc = 1.0;
    for (int k = 0; k < 3; ++k) {
        double se = fabs(box_size(s, k, e)), sa = fabs(box_size(s, k, a));
        double d = center(s, k, e) - center(s, k, a);
        double q = se * se + sa * sa;
        if (q == 0.0) {
            if (d != 0.0) bc = 0.0;
            continue;
        }
        bc *= sqrt(2.0 * se * sa / q) * exp(-3.0 * d * d / q);
    }
    double h2 = 1.0 - bc;
    if (h2 < 0.0) h2 = 0.0;
    /* 1 - H written as BC / (1 + H) (the same number): 1 - sqrt(1 - BC)
     * would round to 0 once BC is below the FP64 epsilon, where the score is
     * still positive */
    return bc / (1.0 + sqrt(h2));
}

/* Inside (step 5): the fraction of e's box volume inside a's box. */
static double inside_fraction(const orc_scene *s, int64_t e, int64_t a)
{
    double frac = 1.0;
    for (int k = 0; k < 3; ++k) {
        double he = 0.5 * fabs(box_size(s, k, e)), ha = 0.5 * fabs(box_size(s, k, a));
        double ce = center(s, k, e), ca = center(s, k, a);
        if (he == 0.0) {
            if (!(fabs(ce - ca) <= ha)) return 0.0;
            continue;
        }
        double lo = ce - he > ca - ha ? ce - he : ca - ha;
        double hi = ce + he < ca + ha ? ce + he : ca + ha;
        double ov = hi - lo;
        if (!(ov > 0.0)) return 0.0;
        frac *= ov / (2.0 * he);
    }
    return frac;
}

/* Closest / farthest (step 5): rank of e by distance to a within the set
 * `set` (n_set objects; e and a may or may not be members). */
static double rank_relation(const orc_scene *s, int32_t pred, int64_t e, int64_t a,
                            const int64_t *set, int64_t n_set)
{
    int in = 0;
    for (int64_t k = 0; k < n_set; ++k) in |= set[k] == e;
    if (!in || e == a) return 0.0;
    double de = dist2(s, e, a);
    int64_t members = 0, closer = 0;
    for (int64_t k = 0; k < n_set; ++k) {
        int64_t j = set[k];
        if (j == a) continue;
        members += 1;
        double dj = dist2(s, j, a);
        if (dj < de || (dj == de && j < e)) closer += 1;
    }
    int64_t rank_d = 1 + closer;
    return pred == ORC_CLOSEST ? 1.0 / (double)rank_d : 1.0 / (double)(members - rank_d + 1);
}

/* r_rho(e, a): the soft relation score of predicate `pred` with e as the
 * target-side argument and a as the anchor (App. D.2 step 4).  Closest and
 * farthest need the query's candidate set: orc_relation_in. */
double orc_relation_in(const orc_scene *s, const orc_params *p, int32_t pred, int64_t e, int64_t a,
                       const int64_t *set, int64_t n_set)
{
    double dz = center(s, 2, e) - center(s, 2, a);
    switch (pred) {
    case ORC_NEXT_TO:
        return exp(-dist2(s, e, a) / (2.0 * p->sigma_next * p->sigma_next));
    case ORC_ON: {
        double dx = center(s, 0, e) - center(s, 0, a);
        double dy = center(s, 1, e) - center(s, 1, a);
        double sxa = box_size(s, 0, a), sya = box_size(s, 1, a);
        double rho = 0.5 * (sxa > sya ? sxa : sya);
        double gate = orc_sigmoid((rho - sqrt(dx * dx + dy * dy)) / p->on_gate);
        double gap = (center(s, 2, e) - 0.5 * box_size(s, 2, e)) - (center(s, 2, a) + 0.5 * box_size(s, 2, a));
        return gate * exp(-gap * gap / (2.0 * p->on_band * p->on_band));
    }
    case ORC_IN_FRONT_OF:
        return viewpoint_rel(s, p, e, a, +1.0, 1);
    case ORC_BEHIND:
        return viewpoint_rel(s, p, e, a, -1.0, 1);
    case ORC_CLOSEST:
    case ORC_FARTHEST:
        return rank_relation(s, pred, e, a, set, n_set);
    case ORC_NEAR_H:
        return near_hellinger(s, e, a);
    case ORC_INSIDE:
        return inside_fraction(s, e, a);
    case ORC_ABOVE:
        return orc_sigmoid(dz / p->tau_v);
    case ORC_BELOW:
        return orc_sigmoid(-dz / p->tau_v);
    case ORC_NEAR: {
        double dx = center(s, 0, e) - center(s, 0, a);
        double dy = center(s, 1, e) - center(s, 1, a);
        double d2 = dx * dx + dy * dy + dz * dz;
        return exp(-d2 / (2.0 * p->sigma_near * p->sigma_near));
    }
    case ORC_LEFT_OF:
        return viewpoint_rel(s, p, e, a, +1.0, 0);
    case ORC_RIGHT_OF:
        return viewpoint_rel(s, p, e, a, -1.0, 0);
    default:
        return NAN;
    }
}

/* Between (step 5): e on the segment from a_p to a_q. */
double orc_between(const orc_scene *s, const orc_params *p, int64_t e, int64_t ap, int64_t aq)
{
    double seg[3], rel[3], ss = 0.0, dot = 0.0;
    for (int k = 0; k < 3; ++k) {
        seg[k] = center(s, k, aq) - center(s, k, ap);
        rel[k] = center(s, k, e) - center(s, k, ap);
        ss += seg[k] * seg[k];
        dot += rel[k] * seg[k];
    }
    if (!(ss > 0.0)) return 0.0;
    double t = dot / ss, d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        double off = rel[k] - t * seg[k];
        d2 += off * off;
    }
    const double tau_b = 0.1;
    const double sg = p->sigma_near;
    return orc_sigmoid(t / tau_b) * orc_sigmoid((1.0 - t) / tau_b) * exp(-0.5 * d2 / (sg * sg));
}

/* Bounds of a Between pair's score for candidate e: the best pair among the
 * certain members (lists Dp, Dq: in_dp / in_dq flags over the possible
 * lists) and among the possible members (Pp, Pq). */
static void between_bounds(const orc_scene *s, const orc_params *p, int64_t e, const int64_t *Pp, int64_t np,
                           const int8_t *dp, const int64_t *Pq, int64_t nq, const int8_t *dq, double *lo,
                           double *hi)
{
    double l = 0.0, h = 0.0;
    for (int64_t x = 0; x < np; ++x) {
        int64_t ap = Pp[x];
        if (ap == e) continue;
        for (int64_t y = 0; y < nq; ++y) {
            int64_t aq = Pq[y];
            if (aq == e || aq == ap) continue;
            double r = orc_between(s, p, e, ap, aq);
            if (r > h) h = r;
            if (dp[ap] && dq[aq] && r > l) l = r;
        }
    }
    *lo = l;
    *hi = h;
}

/* A query's constraint predicates form valid Between pairs. */
static int pairs_ok(int32_t m, const int32_t *preds)
{
    for (int32_t i = 0; i < m; ++i) {
        if (preds[i] == ORC_BETWEEN && !(i + 1 < m && preds[i + 1] == ORC_BETWEEN_AND)) return 0;
        if (preds[i] == ORC_BETWEEN_AND && !(i > 0 && preds[i - 1] == ORC_BETWEEN)) return 0;
    }
    return 1;
}

/* The factors of step 7 from the per-constraint scores: a Between pair's two
 * constraints carry one score and count once.  Returns their number. */
static int32_t factors_of(int32_t m, const int32_t *preds, const double *t, double *f)
{
    int32_t k = 0;
    for (int32_t i = 0; i < m; ++i)
        if (preds[i] != ORC_BETWEEN_AND) f[k++] = t[i];
    return k;
}

/* Step 6 for the Between pair (i, i+1): the best (a_p, a_q) over Lp x Lq. */
static void between_witness(const orc_scene *s, const orc_params *p, int64_t e, const int64_t *Lp, int64_t np,
                            const int64_t *Lq, int64_t nq, double *t_out, int64_t *ap_out, int64_t *aq_out)
{
    double best = 0.0;
    int64_t bp = -1, bq = -1;
    for (int64_t x = 0; x < np; ++x) {
        int64_t ap = Lp[x];
        if (ap == e) continue;
        for (int64_t y = 0; y < nq; ++y) {
            int64_t aq = Lq[y];
            if (aq == e || aq == ap) continue;
            double r = orc_between(s, p, e, ap, aq);
            if (bp < 0 || r > best || (r == best && (ap < bp || (ap == bp && aq < bq)))) {
                best = r;
                bp = ap;
                bq = aq;
            }
        }
    }
    *t_out = bp < 0 ? 0.0 : best;
    *ap_out = bp;
    *aq_out = bq;
}

double orc_relation(const orc_scene *s, const orc_params *p, int32_t pred, int64_t e, int64_t a)
{
    return orc_relation_in(s, p, pred, e, a, NULL, 0);
}

/* Step 1: cosine of embedding u against every descriptor, all in FP64.
 * Returns ORC_EINVAL when u or a descriptor has zero or non-finite norm. */
int orc_cosines(const orc_scene *s, const float *u, double *out)
{
    double un = 0.0;
    for (int64_t k = 0; k < s->dim; ++k) un += (double)u[k] * (double)u[k];
    un = sqrt(un);
    if (!(un > 0.0) || !isfinite(un)) return ORC_EINVAL;
    for (int64_t j = 0; j < s->n; ++j) {
        const float *d = s->desc + j * s->dim;
        double dot = 0.0, dn = 0.0;
        for (int64_t k = 0; k < s->dim; ++k) {
            dot += (double)u[k] * (double)d[k];
            dn += (double)d[k] * (double)d[k];
        }
        dn = sqrt(dn);
        if (!(dn > 0.0) || !isfinite(dn)) return ORC_EINVAL;
        out[j] = dot / (un * dn);
    }
    return ORC_OK;
}

/* Order: larger value first, lower index first among equal values. */
static int before(const double *c, int64_t a, int64_t b)
{
    if (c[a] > c[b]) return 1;
    if (c[a] < c[b]) return 0;
    return a < b;
}

/* Stable merge sort of indices by `before`. */
static void sort_by_value(int64_t n, const double *c, int64_t *idx, int64_t *tmp)
{
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) tmp[k++] = before(c, idx[j], idx[i]) ? idx[j++] : idx[i++];
            while (i < mid) tmp[k++] = idx[i++];
            while (j < hi) tmp[k++] = idx[j++];
        }
        memcpy(idx, tmp, (size_t)n * sizeof(int64_t));
    }
}

/* Step 2: 1-based ranks.  rank[j] = 1 + #{j' : c[j'] > c[j] or (== and j' < j)}. */
int orc_ranks(int64_t n, const double *c, int64_t *rank)
{
    int64_t *idx = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *tmp = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!idx || !tmp) { free(idx); free(tmp); return ORC_ENOMEM; }
    sort_by_value(n, c, idx, tmp);
    for (int64_t r = 0; r < n; ++r) rank[idx[r]] = r + 1;
    free(idx);
    free(tmp);
    return ORC_OK;
}

/* Step 7 for one candidate. */
static double compose(const orc_params *p, double s_sem, int32_t m, const double *t)
{
    double gbar;
    if (m == 0) {
        gbar = 1.0;
    } else {
        double lsum = 0.0;
        int zero = 0;
        for (int32_t i = 0; i < m; ++i) {
            if (!(t[i] > 0.0)) { zero = 1; break; }
            lsum += log(t[i]);
        }
        gbar = zero ? 0.0 : exp(lsum / (double)m);
    }
    return s_sem * ((1.0 - p->w) + p->w * gbar);
}

static double class_factor(const orc_scene *s, const orc_params *p, int32_t c_t, int64_t j)
{
    return (c_t >= 0 && s->cls[j] != c_t) ? p->class_mis : 1.0;
}

/* ------------------------------------------------------------------ */
/* One query, every object: steps 1-7 with all intermediates exposed.  */
/* ------------------------------------------------------------------ */

/*
 * u0: target embedding [dim]; c_t: target class (-1 none); m constraints with
 * predicates preds[m] and landmark embeddings u_c[m, dim].
 * Outputs (all length n, or m*n for per-constraint arrays; any may be NULL):
 *   cos0, rank0, s_sem, t[i*n + e], anchor[i*n + e] (-1 without a witness),
 *   s (composite score).
 */
int orc_query_all(const orc_scene *s, const orc_params *p, const float *u0, int32_t c_t,
                  int32_t m, const int32_t *preds, const float *u_c,
                  double *cos0_out, int64_t *rank0_out, double *s_sem_out,
                  double *t_out, int64_t *anchor_out, double *s_out)
{
    int64_t n = s->n;
    if (n <= 0 || m < 0 || m > 64 || p->k_anchor < 1 || p->k_closest < 1) return ORC_EINVAL;
    if (!pairs_ok(m, preds)) return ORC_EINVAL;
    int rc = ORC_OK;
    double *cos = (double *)malloc((size_t)n * sizeof(double));
    int64_t *rank = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    double *t = (double *)malloc((size_t)(m > 0 ? m : 1) * (size_t)n * sizeof(double));
    int64_t *anc = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * (size_t)n * sizeof(int64_t));
    /* every constraint's L_i (a Between pair's second constraint needs the first's) */
    int64_t *lm_all = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * (size_t)p->k_anchor * sizeof(int64_t));
    int64_t n_lm_of[64];
    double *ssem = (double *)malloc((size_t)n * sizeof(double));
    int64_t kc = p->k_closest < n ? p->k_closest : n;
    int64_t *cset = (int64_t *)malloc((size_t)(kc > 0 ? kc : 1) * sizeof(int64_t));
    int64_t n_cset = 0;
    if (!cos || !rank || !t || !anc || !lm_all || !ssem || !cset) { rc = ORC_ENOMEM; goto done; }

    /* Steps 1-3 for the target row. */
    if ((rc = orc_cosines(s, u0, cos)) != ORC_OK) goto done;
    if ((rc = orc_ranks(n, cos, rank)) != ORC_OK) goto done;
    for (int64_t j = 0; j < n; ++j) {
        ssem[j] = class_factor(s, p, c_t, j) / (p->mu + (double)rank[j]);
        if (cos0_out) cos0_out[j] = cos[j];
        if (rank0_out) rank0_out[j] = rank[j];
        if (s_sem_out) s_sem_out[j] = ssem[j];
    }
    /* the candidate set of closest / farthest: target ranks 1..k_closest */
    for (int64_t r = 1; r <= kc; ++r)
        for (int64_t j = 0; j < n; ++j)
            if (rank[j] == r) { cset[n_cset++] = j; break; }

    /* Steps 1, 2, 4, 5, 6 for every constraint. */
    for (int32_t i = 0; i < m; ++i) {
        if ((rc = orc_cosines(s, u_c + (int64_t)i * s->dim, cos)) != ORC_OK) goto done;
        if ((rc = orc_ranks(n, cos, rank)) != ORC_OK) goto done;
        int64_t n_lm = 0;
        int64_t *lm = lm_all + (int64_t)i * p->k_anchor;
        /* L_i in rank order: walk ranks 1..K_a. */
        int64_t ka = p->k_anchor < n ? p->k_anchor : n;
        for (int64_t r = 1; r <= ka; ++r)
            for (int64_t j = 0; j < n; ++j)
                if (rank[j] == r) { lm[n_lm++] = j; break; }
        n_lm_of[i] = n_lm;
        if (preds[i] == ORC_BETWEEN) continue;     /* scored with its second constraint */
        if (preds[i] == ORC_BETWEEN_AND) {
            const int64_t *lp = lm_all + (int64_t)(i - 1) * p->k_anchor;
            for (int64_t e = 0; e < n; ++e) {
                double tb;
                int64_t ap, aq;
                between_witness(s, p, e, lp, n_lm_of[i - 1], lm, n_lm, &tb, &ap, &aq);
                t[(int64_t)(i - 1) * n + e] = t[(int64_t)i * n + e] = tb;
                anc[(int64_t)(i - 1) * n + e] = ap;
                anc[(int64_t)i * n + e] = aq;
            }
            continue;
        }
        for (int64_t e = 0; e < n; ++e) {
            double best = 0.0;
            int64_t arg = -1;
            for (int64_t l = 0; l < n_lm; ++l) {
                int64_t a = lm[l];
                if (a == e) continue;
                double r = orc_relation_in(s, p, preds[i], e, a, cset, n_cset);
                if (arg < 0 || r > best || (r == best && a < arg)) { best = r; arg = a; }
            }
            t[(int64_t)i * n + e] = arg < 0 ? 0.0 : best;
            anc[(int64_t)i * n + e] = arg;
        }
    }

    /* Step 7. */
    for (int64_t e = 0; e < n; ++e) {
        double ts[64], te[64];
        for (int32_t i = 0; i < m; ++i) ts[i] = t[(int64_t)i * n + e];
        int32_t mf = factors_of(m, preds, ts, te);
        double sc = compose(p, ssem[e], mf, te);
        if (s_out) s_out[e] = sc;
    }
    if (t_out) memcpy(t_out, t, (size_t)m * (size_t)n * sizeof(double));
    if (anchor_out) memcpy(anchor_out, anc, (size_t)m * (size_t)n * sizeof(int64_t));
done:
    free(cos); free(rank); free(t); free(anc); free(lm_all); free(ssem); free(cset);
    return rc;
}

/* Step 8: the k largest of s (lower index first on ties). */
int orc_topk(int64_t n, const double *s, int64_t k, int64_t *idx_out)
{
    if (k < 0 || k > n) return ORC_EINVAL;
    int64_t *idx = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *tmp = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!idx || !tmp) { free(idx); free(tmp); return ORC_ENOMEM; }
    sort_by_value(n, s, idx, tmp);
    for (int64_t r = 0; r < k; ++r) idx_out[r] = idx[r];
    free(idx);
    free(tmp);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* A batch of queries on one scene (OpenMP over queries).              */
/* ------------------------------------------------------------------ */

/*
 * Queries in CSR form: query q has constraints c_off[q] .. c_off[q+1]-1 with
 * predicates c_pred[] and landmark embeddings c_emb[c, dim].
 * Outputs per query (k entries): out_idx, out_score; per entry and constraint
 * slot (4 slots, -1 beyond m): out_t, out_anchor.  n_threads <= 0 uses the
 * OpenMP default.  Returns the first failing query's code.
 */
int orc_batch(const orc_scene *s, const orc_params *p, int64_t n_q, const float *tgt_emb,
              const int32_t *tgt_cls, const int32_t *c_off, const int32_t *c_pred,
              const float *c_emb, int64_t k, int64_t *out_idx, double *out_score,
              double *out_t, int64_t *out_anchor, int32_t n_threads)
{
    int64_t n = s->n;
    if (k < 1 || k > n) return ORC_EINVAL;
    for (int64_t q = 0; q < n_q; ++q) {
        int32_t m = c_off[q + 1] - c_off[q];
        if (m < 0 || m > 4) return ORC_EINVAL;
    }
    int rc_all = ORC_OK;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t q = 0; q < n_q; ++q) {
        int32_t m = c_off[q + 1] - c_off[q];
        double *sc = (double *)malloc((size_t)n * sizeof(double));
        double *t = (double *)malloc((size_t)(m > 0 ? m : 1) * (size_t)n * sizeof(double));
        int64_t *anc = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * (size_t)n * sizeof(int64_t));
        int64_t *top = (int64_t *)malloc((size_t)k * sizeof(int64_t));
        int rc = (sc && t && anc && top) ? ORC_OK : ORC_ENOMEM;
        if (rc == ORC_OK)
            rc = orc_query_all(s, p, tgt_emb + q * s->dim, tgt_cls[q], m, c_pred + c_off[q],
                               c_emb + (int64_t)c_off[q] * s->dim, NULL, NULL, NULL, t, anc, sc);
        if (rc == ORC_OK) rc = orc_topk(n, sc, k, top);
        if (rc == ORC_OK) {
            for (int64_t r = 0; r < k; ++r) {
                int64_t e = top[r];
                out_idx[q * k + r] = e;
                out_score[q * k + r] = sc[e];
                for (int32_t i = 0; i < 4; ++i) {
                    if (out_t) out_t[(q * k + r) * 4 + i] = i < m ? t[(int64_t)i * n + e] : -1.0;
                    if (out_anchor) out_anchor[(q * k + r) * 4 + i] = i < m ? anc[(int64_t)i * n + e] : -1;
                }
            }
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            if (rc != ORC_OK && rc_all == ORC_OK) rc_all = rc;
        }
        free(sc); free(t); free(anc); free(top);
    }
    return rc_all;
}

/* ------------------------------------------------------------------ */
/* Tie-tolerant bounds: what any valid result may score.               */
/* ------------------------------------------------------------------ */

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* #{v in sorted ascending a[0..n) : v > x} */
static int64_t count_greater(const double *a, int64_t n, double x)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] > x) hi = mid; else lo = mid + 1;
    }
    return n - lo;
}

/* #{v : v >= x} */
static int64_t count_geq(const double *a, int64_t n, double x)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] >= x) hi = mid; else lo = mid + 1;
    }
    return n - lo;
}

/* Bounds of closest / farthest for a candidate e that is certainly in the
 * candidate set `set` (n_set objects): distances within a relative dtol of
 * one another may be ordered either way. */
static void rank_relation_bounds(const orc_scene *s, int32_t pred, int64_t e, int64_t a,
                                 const int64_t *set, int64_t n_set, double dtol, double *lo, double *hi)
{
    double de = dist2(s, e, a);
    int64_t members = 0, c_lo = 0, c_hi = 0;
    for (int64_t k = 0; k < n_set; ++k) {
        int64_t j = set[k];
        if (j == a) continue;
        members += 1;
        if (j == e) continue;
        double dj = dist2(s, j, a);
        if (dj < de * (1.0 - dtol)) c_lo += 1;
        if (dj <= de * (1.0 + dtol)) c_hi += 1;
    }
    int64_t r_lo = 1 + c_lo, r_hi = 1 + c_hi;
    if (pred == ORC_CLOSEST) {
        *lo = 1.0 / (double)r_hi;
        *hi = 1.0 / (double)r_lo;
    } else {
        *lo = 1.0 / (double)(members - r_lo + 1);
        *hi = 1.0 / (double)(members - r_hi + 1);
    }
}

/*
 * When two cosines differ by at most tau, an implementation whose cosines are
 * within tau/2 of the exact ones may order them either way.  For every object
 * this gives the range of ranks it can take,
 *   rank_lo(j) = 1 + #{j' : c_j' > c_j + tau},  rank_hi(j) = #{j' : c_j' >= c_j - tau},
 * and from them, because every later step is monotone, bounds on what any
 * such implementation can return:
 *   s_sem in [cf/(mu + rank_hi), cf/(mu + rank_lo)];
 *   L_i contains D_i = {a : rank_hi_i(a) <= K_a} and lies in P_i = {a : rank_lo_i(a) <= K_a};
 *   t_i(e) in [max over D_i \ {e}, max over P_i \ {e}];  s in [s_lo, s_hi].
 * Closest / farthest depend on the candidate set C (target ranks up to
 * k_closest): when C is ambiguous (some object's rank range straddles
 * k_closest) their scores are only known to lie in [0, 1] for possible
 * members; otherwise squared distances within a relative 1e-5 may be
 * ordered either way.
 * With tau = 0 on tie-free data every interval is a single point equal to
 * orc_query_all's result.
 * Outputs (length n; per-constraint arrays m*n; any may be NULL):
 *   s_lo, s_hi, t_lo, t_hi, rank_lo0, rank_hi0, and in_p[i*n + a] = 1 when a
 *   lies in P_i (a valid bound anchor).
 */
int orc_query_bounds(const orc_scene *s, const orc_params *p, const float *u0, int32_t c_t,
                     int32_t m, const int32_t *preds, const float *u_c, double tau,
                     double *s_lo, double *s_hi, double *t_lo_out, double *t_hi_out,
                     int64_t *rank_lo0, int64_t *rank_hi0, int8_t *in_p_out)
{
    int64_t n = s->n;
    if (n <= 0 || m < 0 || m > 64 || !(tau >= 0.0)) return ORC_EINVAL;
    if (!pairs_ok(m, preds)) return ORC_EINVAL;
    int rc = ORC_OK;
    double *cos = (double *)malloc((size_t)n * sizeof(double));
    double *sorted = (double *)malloc((size_t)n * sizeof(double));
    double *slo = (double *)malloc((size_t)n * sizeof(double));
    double *shi = (double *)malloc((size_t)n * sizeof(double));
    double *tlo = (double *)malloc((size_t)(m > 0 ? m : 1) * (size_t)n * sizeof(double));
    double *thi = (double *)malloc((size_t)(m > 0 ? m : 1) * (size_t)n * sizeof(double));
    int8_t *in_d = (int8_t *)malloc((size_t)n);
    int8_t *in_p = (int8_t *)malloc((size_t)n);
    int64_t *plist = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int8_t *c_d = (int8_t *)malloc((size_t)n);     /* certainly in the candidate set C */
    int8_t *c_p = (int8_t *)malloc((size_t)n);     /* possibly in C */
    int64_t *cset = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *prev_plist = (int64_t *)malloc((size_t)n * sizeof(int64_t));   /* a Between pair's first list */
    int8_t *prev_in_d = (int8_t *)malloc((size_t)n);
    int64_t n_prev = 0, n_cset = 0, n_cp = 0;
    if (!cos || !sorted || !slo || !shi || !tlo || !thi || !in_d || !in_p || !plist || !c_d || !c_p || !cset ||
        !prev_plist || !prev_in_d) {
        rc = ORC_ENOMEM;
        goto done;
    }

    if ((rc = orc_cosines(s, u0, cos)) != ORC_OK) goto done;
    memcpy(sorted, cos, (size_t)n * sizeof(double));
    qsort(sorted, (size_t)n, sizeof(double), cmp_double);
    for (int64_t j = 0; j < n; ++j) {
        int64_t rlo = 1 + count_greater(sorted, n, cos[j] + tau);
        int64_t rhi = count_geq(sorted, n, cos[j] - tau);
        double cf = class_factor(s, p, c_t, j);
        slo[j] = cf / (p->mu + (double)rhi);
        shi[j] = cf / (p->mu + (double)rlo);
        if (rank_lo0) rank_lo0[j] = rlo;
        if (rank_hi0) rank_hi0[j] = rhi;
        c_d[j] = rhi <= p->k_closest;
        c_p[j] = rlo <= p->k_closest;
        if (c_d[j]) cset[n_cset++] = j;
        n_cp += c_p[j];
    }
    const int cset_certain = n_cset == n_cp;
    for (int32_t i = 0; i < m; ++i) {
        if ((rc = orc_cosines(s, u_c + (int64_t)i * s->dim, cos)) != ORC_OK) goto done;
        memcpy(sorted, cos, (size_t)n * sizeof(double));
        qsort(sorted, (size_t)n, sizeof(double), cmp_double);
        for (int64_t a = 0; a < n; ++a) {
            int64_t rlo = 1 + count_greater(sorted, n, cos[a] + tau);
            int64_t rhi = count_geq(sorted, n, cos[a] - tau);
            in_d[a] = rhi <= p->k_anchor;
            in_p[a] = rlo <= p->k_anchor;
            if (in_p_out) in_p_out[(int64_t)i * n + a] = in_p[a];
        }
        int64_t n_p = 0;
        for (int64_t a = 0; a < n; ++a)
            if (in_p[a]) plist[n_p++] = a;
        if (preds[i] == ORC_BETWEEN) {
            memcpy(prev_plist, plist, (size_t)n_p * sizeof(int64_t));
            memcpy(prev_in_d, in_d, (size_t)n);
            n_prev = n_p;
            continue;
        }
        if (preds[i] == ORC_BETWEEN_AND) {
            for (int64_t e = 0; e < n; ++e) {
                double lo, hi;
                between_bounds(s, p, e, prev_plist, n_prev, prev_in_d, plist, n_p, in_d, &lo, &hi);
                tlo[(int64_t)(i - 1) * n + e] = tlo[(int64_t)i * n + e] = lo;
                thi[(int64_t)(i - 1) * n + e] = thi[(int64_t)i * n + e] = hi;
            }
            continue;
        }
        for (int64_t e = 0; e < n; ++e) {
            double lo = 0.0, hi = 0.0;
            const int ranked = preds[i] == ORC_CLOSEST || preds[i] == ORC_FARTHEST;
            for (int64_t l = 0; l < n_p; ++l) {
                int64_t a = plist[l];
                if (a == e) continue;
                double r_lo, r_hi;
                if (!ranked) {
                    r_lo = r_hi = orc_relation(s, p, preds[i], e, a);
                } else if (!c_p[e]) {
                    r_lo = r_hi = 0.0;
                } else if (!cset_certain || !c_d[e]) {
                    r_lo = 0.0;
                    r_hi = 1.0;
                } else {
                    rank_relation_bounds(s, preds[i], e, a, cset, n_cset, 1e-5, &r_lo, &r_hi);
                }
                if (r_hi > hi) hi = r_hi;
                if (in_d[a] && r_lo > lo) lo = r_lo;
            }
            tlo[(int64_t)i * n + e] = lo;
            thi[(int64_t)i * n + e] = hi;
        }
    }
    for (int64_t e = 0; e < n; ++e) {
        double ts[64], te[64];
        for (int32_t i = 0; i < m; ++i) ts[i] = tlo[(int64_t)i * n + e];
        int32_t mf = factors_of(m, preds, ts, te);
        double a = compose(p, slo[e], mf, te);
        for (int32_t i = 0; i < m; ++i) ts[i] = thi[(int64_t)i * n + e];
        mf = factors_of(m, preds, ts, te);
        double b = compose(p, shi[e], mf, te);
        if (s_lo) s_lo[e] = a;
        if (s_hi) s_hi[e] = b;
    }
    if (t_lo_out) memcpy(t_lo_out, tlo, (size_t)m * (size_t)n * sizeof(double));
    if (t_hi_out) memcpy(t_hi_out, thi, (size_t)m * (size_t)n * sizeof(double));
done:
    free(cos); free(sorted); free(slo); free(shi); free(tlo); free(thi); free(in_d); free(in_p); free(plist);
    free(c_d); free(c_p); free(cset); free(prev_plist); free(prev_in_d);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Several retrieval channels: reciprocal-rank fusion (App. D.2 step 3) */
/* ------------------------------------------------------------------ */

/*
 * App. D.2 step 3 ranks the whole pool once per query channel -- four
 * channels over three embedding spaces, each channel contributing
 * w / (mu + rank) -- and takes the sum as the fused rank score; landmark
 * variables are retrieved the same way.  Here:
 *
 *   F(j)   = sum_c w_c / (mu + rank_c(j)),  rank_c over the cosines of
 *            channel c's embedding against every object's descriptor in
 *            channel c's space (steps 1-2 per channel);
 *   s_sem  = cf(j) * F(j);
 *   L_i    = the K_a objects of largest F_i (the landmark's channels),
 *            lower index first on equal F_i;
 *   the Closest / Farthest set C = the k_closest objects of largest F.
 * Steps 5-8 are unchanged.  With one channel of weight 1 this is
 * orc_query_all.
 *
 * spaces[s] = (dim_s, descriptors [n, dim_s]) for s < n_spaces; channel c
 * reads space ch_space[c] with weight ch_w[c].  u0 holds the target's
 * channel embeddings end to end (dim of channel 0's space, then channel 1's,
 * ...); u_c holds, channel after channel, the m landmark embeddings of that
 * channel ([m, dim] per channel).  Outputs as orc_query_all, with F of the
 * target in fused_out.
 */
typedef struct {
    int64_t dim;
    const float *desc;
} orc_space;

/* Fused score of every object for one variable (target or landmark):
 * emb holds its n_ch channel embeddings end to end. */
static int fused_scores(const orc_scene *s, const orc_space *spaces, int32_t n_spaces, const orc_params *p,
                        int32_t n_ch, const int32_t *ch_space, const double *ch_w, const float *const *emb,
                        double *F, double *cos, int64_t *rank)
{
    for (int64_t j = 0; j < s->n; ++j) F[j] = 0.0;
    for (int32_t c = 0; c < n_ch; ++c) {
        if (ch_space[c] < 0 || ch_space[c] >= n_spaces) return ORC_EINVAL;
        orc_scene sc = *s;
        sc.dim = spaces[ch_space[c]].dim;
        sc.desc = spaces[ch_space[c]].desc;
        int rc = orc_cosines(&sc, emb[c], cos);
        if (rc != ORC_OK) return rc;
        if ((rc = orc_ranks(s->n, cos, rank)) != ORC_OK) return rc;
        for (int64_t j = 0; j < s->n; ++j) F[j] += ch_w[c] / (p->mu + (double)rank[j]);
    }
    return ORC_OK;
}

int orc_query_mc(const orc_scene *s, const orc_space *spaces, int32_t n_spaces, const orc_params *p,
                 int32_t n_ch, const int32_t *ch_space, const double *ch_w, const float *u0, int32_t c_t,
                 int32_t m, const int32_t *preds, const float *u_c,
                 double *fused_out, double *s_sem_out, double *t_out, int64_t *anchor_out, double *s_out)
{
    int64_t n = s->n;
    if (n <= 0 || m < 0 || m > 64 || n_ch < 1 || n_ch > 16 || p->k_anchor < 1 || p->k_closest < 1)
        return ORC_EINVAL;
    if (!pairs_ok(m, preds)) return ORC_EINVAL;
    int rc = ORC_OK;
    double *F = (double *)malloc((size_t)n * sizeof(double));
    double *Fl = (double *)malloc((size_t)n * sizeof(double));
    double *cos = (double *)malloc((size_t)n * sizeof(double));
    int64_t *rank = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *tmp = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    double *ssem = (double *)malloc((size_t)n * sizeof(double));
    double *tt = (double *)malloc((size_t)(m > 0 ? m : 1) * (size_t)n * sizeof(double));
    int64_t *aa = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * (size_t)n * sizeof(int64_t));
    int64_t *prev_L = (int64_t *)malloc((size_t)n * sizeof(int64_t));     /* a Between pair's first list */
    const float *emb[16];
    if (!F || !Fl || !cos || !rank || !order || !tmp || !ssem || !tt || !aa || !prev_L) { rc = ORC_ENOMEM; goto out; }

    /* the target: fused score and s_sem */
    {
        int64_t off = 0;
        for (int32_t c = 0; c < n_ch; ++c) {
            emb[c] = u0 + off;
            off += spaces[ch_space[c] >= 0 && ch_space[c] < n_spaces ? ch_space[c] : 0].dim;
        }
    }
    if ((rc = fused_scores(s, spaces, n_spaces, p, n_ch, ch_space, ch_w, emb, F, cos, rank)) != ORC_OK) goto out;
    for (int64_t j = 0; j < n; ++j) ssem[j] = class_factor(s, p, c_t, j) * F[j];
    /* C: the k_closest objects of largest F */
    sort_by_value(n, F, order, tmp);
    int64_t kc = p->k_closest < n ? p->k_closest : n;
    int64_t cset[4096];
    if (kc > 4096) { rc = ORC_EINVAL; goto out; }
    for (int64_t r = 0; r < kc; ++r) cset[r] = order[r];

    for (int32_t i = 0; i < m; ++i) {
        /* the landmark's channel embeddings: row i of each channel's block */
        int64_t off = 0;
        for (int32_t c = 0; c < n_ch; ++c) {
            int64_t d = spaces[ch_space[c]].dim;
            emb[c] = u_c + off + (int64_t)i * d;
            off += (int64_t)m * d;
        }
        if ((rc = fused_scores(s, spaces, n_spaces, p, n_ch, ch_space, ch_w, emb, Fl, cos, rank)) != ORC_OK)
            goto out;
        sort_by_value(n, Fl, order, tmp);       /* order[0 .. K_a) is L_i */
        int64_t ka = p->k_anchor < n ? p->k_anchor : n;
        if (preds[i] == ORC_BETWEEN) {          /* scored with its second constraint */
            memcpy(prev_L, order, (size_t)ka * sizeof(int64_t));
            continue;
        }
        if (preds[i] == ORC_BETWEEN_AND) {
            for (int64_t e = 0; e < n; ++e) {
                double tb;
                int64_t ap, aq;
                between_witness(s, p, e, prev_L, ka, order, ka, &tb, &ap, &aq);
                tt[(int64_t)(i - 1) * n + e] = tt[(int64_t)i * n + e] = tb;
                aa[(int64_t)(i - 1) * n + e] = ap;
                aa[(int64_t)i * n + e] = aq;
            }
            continue;
        }
        for (int64_t e = 0; e < n; ++e) {
            double tbest = 0.0;
            int64_t abest = -1;
            for (int64_t l = 0; l < ka; ++l) {
                int64_t cand = order[l];
                if (cand == e) continue;
                double rv = orc_relation_in(s, p, preds[i], e, cand, cset, kc);
                if (abest < 0 || rv > tbest || (rv == tbest && cand < abest)) {
                    tbest = rv;
                    abest = cand;
                }
            }
            tt[(int64_t)i * n + e] = abest < 0 ? 0.0 : tbest;
            aa[(int64_t)i * n + e] = abest;
        }
    }
    for (int64_t e = 0; e < n; ++e) {
        double ts[64], te[64];
        for (int32_t i = 0; i < m; ++i) ts[i] = tt[(int64_t)i * n + e];
        int32_t mf = factors_of(m, preds, ts, te);
        if (s_out) s_out[e] = compose(p, ssem[e], mf, te);
        if (fused_out) fused_out[e] = F[e];
        if (s_sem_out) s_sem_out[e] = ssem[e];
    }
    if (t_out) memcpy(t_out, tt, (size_t)m * (size_t)n * sizeof(double));
    if (anchor_out) memcpy(anchor_out, aa, (size_t)m * (size_t)n * sizeof(int64_t));
out:
    free(F); free(Fl); free(cos); free(rank); free(order); free(tmp); free(ssem); free(tt); free(aa); free(prev_L);
    return rc;
}

/*
 * Tie-tolerant bounds for several channels (as orc_query_bounds for one):
 * each channel's rank range [rank_lo, rank_hi] at tie tolerance tau gives
 * F in [F_lo, F_hi] = [sum_c w_c / (mu + rank_hi_c), sum_c w_c / (mu + rank_lo_c)].
 * An object is certainly among the K largest F when fewer than K others can
 * reach its F_lo (#{j != a : F_hi(j) >= F_lo(a)} < K), possibly so when
 * fewer than K others certainly beat it (#{j != a : F_lo(j) > F_hi(a)} < K).
 * That decides L_i's certain (D_i) and possible (P_i) members and the
 * Closest / Farthest set; the rest follows orc_query_bounds.  Outputs:
 * s_lo, s_hi, t_lo, t_hi, F_lo, F_hi (target), in_p (m*n).
 */
static void fused_range(const orc_scene *s, const orc_space *spaces, const orc_params *p, int32_t n_ch,
                        const int32_t *ch_space, const double *ch_w, const float *const *emb, double tau,
                        double *Flo, double *Fhi, double *cos, double *sorted)
{
    int64_t n = s->n;
    for (int64_t j = 0; j < n; ++j) Flo[j] = Fhi[j] = 0.0;
    for (int32_t c = 0; c < n_ch; ++c) {
        orc_scene sc = *s;
        sc.dim = spaces[ch_space[c]].dim;
        sc.desc = spaces[ch_space[c]].desc;
        orc_cosines(&sc, emb[c], cos);
        memcpy(sorted, cos, (size_t)n * sizeof(double));
        qsort(sorted, (size_t)n, sizeof(double), cmp_double);
        for (int64_t j = 0; j < n; ++j) {
            int64_t rlo = 1 + count_greater(sorted, n, cos[j] + tau);
            int64_t rhi = count_geq(sorted, n, cos[j] - tau);
            Flo[j] += ch_w[c] / (p->mu + (double)rhi);
            Fhi[j] += ch_w[c] / (p->mu + (double)rlo);
        }
    }
}

/* certain[j] / possible[j]: j is certainly / possibly among the K largest. */
static void topk_membership(int64_t n, const double *lo, const double *hi, int64_t K, int8_t *certain,
                            int8_t *possible, double *sorted)
{
    memcpy(sorted, hi, (size_t)n * sizeof(double));
    qsort(sorted, (size_t)n, sizeof(double), cmp_double);
    for (int64_t j = 0; j < n; ++j) {
        /* others whose upper bound reaches lo[j] (j itself counts when hi[j] >= lo[j]) */
        int64_t reach = count_geq(sorted, n, lo[j]) - (hi[j] >= lo[j] ? 1 : 0);
        certain[j] = reach < K;
    }
    memcpy(sorted, lo, (size_t)n * sizeof(double));
    qsort(sorted, (size_t)n, sizeof(double), cmp_double);
    for (int64_t j = 0; j < n; ++j) {
        int64_t beat = count_greater(sorted, n, hi[j]) - (lo[j] > hi[j] ? 1 : 0);
        possible[j] = beat < K;
    }
}

int orc_query_bounds_mc(const orc_scene *s, const orc_space *spaces, int32_t n_spaces, const orc_params *p,
                        int32_t n_ch, const int32_t *ch_space, const double *ch_w, const float *u0,
                        int32_t c_t, int32_t m, const int32_t *preds, const float *u_c, double tau,
                        double *s_lo, double *s_hi, double *t_lo_out, double *t_hi_out,
                        double *F_lo_out, double *F_hi_out, int8_t *in_p_out)
{
    int64_t n = s->n;
    if (n <= 0 || m < 0 || m > 64 || n_ch < 1 || n_ch > 16 || !(tau >= 0.0)) return ORC_EINVAL;
    for (int32_t c = 0; c < n_ch; ++c)
        if (ch_space[c] < 0 || ch_space[c] >= n_spaces) return ORC_EINVAL;
    if (!pairs_ok(m, preds)) return ORC_EINVAL;
    int rc = ORC_OK;
    double *Flo = (double *)malloc((size_t)n * sizeof(double));
    double *Fhi = (double *)malloc((size_t)n * sizeof(double));
    double *Llo = (double *)malloc((size_t)n * sizeof(double));
    double *Lhi = (double *)malloc((size_t)n * sizeof(double));
    double *cos = (double *)malloc((size_t)n * sizeof(double));
    double *sorted = (double *)malloc((size_t)n * sizeof(double));
    double *tlo = (double *)malloc((size_t)(m > 0 ? m : 1) * (size_t)n * sizeof(double));
    double *thi = (double *)malloc((size_t)(m > 0 ? m : 1) * (size_t)n * sizeof(double));
    int8_t *c_d = (int8_t *)malloc((size_t)n), *c_p = (int8_t *)malloc((size_t)n);
    int8_t *l_d = (int8_t *)malloc((size_t)n), *l_p = (int8_t *)malloc((size_t)n);
    int64_t *cset = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *plist = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *prev_plist = (int64_t *)malloc((size_t)n * sizeof(int64_t));   /* a Between pair's first list */
    int8_t *prev_d = (int8_t *)malloc((size_t)n);
    int64_t n_prev = 0;
    const float *emb[16];
    int64_t n_cset = 0, n_cp = 0;
    if (!Flo || !Fhi || !Llo || !Lhi || !cos || !sorted || !tlo || !thi || !c_d || !c_p || !l_d || !l_p ||
        !cset || !plist || !prev_plist || !prev_d) {
        rc = ORC_ENOMEM;
        goto out;
    }
    {
        int64_t off = 0;
        for (int32_t c = 0; c < n_ch; ++c) { emb[c] = u0 + off; off += spaces[ch_space[c]].dim; }
    }
    fused_range(s, spaces, p, n_ch, ch_space, ch_w, emb, tau, Flo, Fhi, cos, sorted);
    topk_membership(n, Flo, Fhi, p->k_closest, c_d, c_p, sorted);
    for (int64_t j = 0; j < n; ++j) {
        if (c_d[j]) cset[n_cset++] = j;
        n_cp += c_p[j];
    }
    const int cset_certain = n_cset == n_cp;
    for (int32_t i = 0; i < m; ++i) {
        int64_t off = 0;
        for (int32_t c = 0; c < n_ch; ++c) {
            int64_t d = spaces[ch_space[c]].dim;
            emb[c] = u_c + off + (int64_t)i * d;
            off += (int64_t)m * d;
        }
        fused_range(s, spaces, p, n_ch, ch_space, ch_w, emb, tau, Llo, Lhi, cos, sorted);
        topk_membership(n, Llo, Lhi, p->k_anchor, l_d, l_p, sorted);
        int64_t n_p = 0;
        for (int64_t a = 0; a < n; ++a) {
            if (in_p_out) in_p_out[(int64_t)i * n + a] = l_p[a];
            if (l_p[a]) plist[n_p++] = a;
        }
        if (preds[i] == ORC_BETWEEN) {
            memcpy(prev_plist, plist, (size_t)n_p * sizeof(int64_t));
            memcpy(prev_d, l_d, (size_t)n);
            n_prev = n_p;
            continue;
        }
        if (preds[i] == ORC_BETWEEN_AND) {
            for (int64_t e = 0; e < n; ++e) {
                double lo, hi;
                between_bounds(s, p, e, prev_plist, n_prev, prev_d, plist, n_p, l_d, &lo, &hi);
                tlo[(int64_t)(i - 1) * n + e] = tlo[(int64_t)i * n + e] = lo;
                thi[(int64_t)(i - 1) * n + e] = thi[(int64_t)i * n + e] = hi;
            }
            continue;
        }
        const int ranked = preds[i] == ORC_CLOSEST || preds[i] == ORC_FARTHEST;
        for (int64_t e = 0; e < n; ++e) {
            double lo = 0.0, hi = 0.0;
            for (int64_t l = 0; l < n_p; ++l) {
                int64_t a = plist[l];
                if (a == e) continue;
                double r_lo, r_hi;
                if (!ranked) {
                    r_lo = r_hi = orc_relation(s, p, preds[i], e, a);
                } else if (!c_p[e]) {
                    r_lo = r_hi = 0.0;
                } else if (!cset_certain || !c_d[e]) {
                    r_lo = 0.0;
                    r_hi = 1.0;
                } else {
                    rank_relation_bounds(s, preds[i], e, a, cset, n_cset, 1e-5, &r_lo, &r_hi);
                }
                if (r_hi > hi) hi = r_hi;
                if (l_d[a] && r_lo > lo) lo = r_lo;
            }
            tlo[(int64_t)i * n + e] = lo;
            thi[(int64_t)i * n + e] = hi;
        }
    }
    for (int64_t e = 0; e < n; ++e) {
        double cf = class_factor(s, p, c_t, e), ts[64], te[64];
        for (int32_t i = 0; i < m; ++i) ts[i] = tlo[(int64_t)i * n + e];
        int32_t mf = factors_of(m, preds, ts, te);
        double a = compose(p, cf * Flo[e], mf, te);
        for (int32_t i = 0; i < m; ++i) ts[i] = thi[(int64_t)i * n + e];
        mf = factors_of(m, preds, ts, te);
        double b = compose(p, cf * Fhi[e], mf, te);
        if (s_lo) s_lo[e] = a;
        if (s_hi) s_hi[e] = b;
        if (F_lo_out) F_lo_out[e] = Flo[e];
        if (F_hi_out) F_hi_out[e] = Fhi[e];
    }
    if (t_lo_out) memcpy(t_lo_out, tlo, (size_t)m * (size_t)n * sizeof(double));
    if (t_hi_out) memcpy(t_hi_out, thi, (size_t)m * (size_t)n * sizeof(double));
out:
    free(Flo); free(Fhi); free(Llo); free(Lhi); free(cos); free(sorted); free(tlo); free(thi);
    free(c_d); free(c_p); free(l_d); free(l_p); free(cset); free(plist); free(prev_plist); free(prev_d);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Mapping-side association (App. D.1 steps 3-5)                      */
/* ------------------------------------------------------------------ */

/*
 * A batch of detections against the memory's entities, each a 3D Gaussian
 * (mean; covariance packed as xx, xy, xz, yy, yz, zz) with an appearance
 * feature and, for entities, a weight w (the detections fused so far) and an
 * active flag:
 *  3. neighbour search: for detection d, the active entities e with
 *     cos(f_d, f_e) >= tau_f, then the Hellinger distance
 *       H = sqrt(1 - BC),  BC = det(S_d)^(1/4) det(S_e)^(1/4) / det(S)^(1/2)
 *                               * exp(-(1/8) dmu' S^-1 dmu),  S = (S_d + S_e) / 2,
 *     keeping those with H <= h_max sorted by H (lower index on ties); the
 *     first max_m of them are the detection's matches;
 *  4. correspondence: the connected components of the graph whose edges join
 *     each detection to its matches (union-find); in a component holding
 *     entities the winner is the entity of largest w (lower index on ties),
 *     every other entity of it merges into the winner; a detection without a
 *     match starts a new entity (slot n_ent + d);
 *  5. fusion: the winner absorbs every member (entities with their w,
 *     detections with w = 1) by the sufficient-statistics merge
 *       w = sum w_i,  M1 = sum w_i mu_i,  M2 = sum w_i (S_i + mu_i mu_i'),
 *       mu = M1 / w,  S = M2 / w - mu mu',
 *     here evaluated in the equal form S = sum w_i (S_i + (mu_i - mu)(mu_i - mu)') / w,
 *     and the appearance feature by the w-weighted average sum w_i f_i / w.
 * Outputs over n_ent + n_det slots (entities, then one slot per detection):
 * parent (the slot a slot merges into; itself for a winner, an untouched
 * entity or a new entity), w (0 for a merged-away slot), mu [3, slots],
 * cov [6, slots], feat [slots, F]; per detection: match_cnt (matches within
 * the budget, before the max_m cap), match_idx / match_h [n_det, max_m]
 * (-1 / -1 past the count).
 */
static double det3(const double c[6])
{
    /* c = xx, xy, xz, yy, yz, zz */
    return c[0] * (c[3] * c[5] - c[4] * c[4]) - c[1] * (c[1] * c[5] - c[4] * c[2]) +
           c[2] * (c[1] * c[4] - c[3] * c[2]);
}

/* Hellinger distance between two Gaussians (packed covariances). */
double orc_hellinger(const double *mu1, const double *c1, const double *mu2, const double *c2)
{
    double S[6], d[3];
    for (int k = 0; k < 6; ++k) S[k] = 0.5 * (c1[k] + c2[k]);
    for (int k = 0; k < 3; ++k) d[k] = mu1[k] - mu2[k];
    double dS = det3(S), d1 = det3(c1), d2 = det3(c2);
    if (!(dS > 0.0) || !(d1 > 0.0) || !(d2 > 0.0)) return 1.0;
    /* S^-1 d by the adjugate */
    double a[6] = {S[3] * S[5] - S[4] * S[4], S[2] * S[4] - S[1] * S[5], S[1] * S[4] - S[2] * S[3],
                   S[0] * S[5] - S[2] * S[2], S[1] * S[2] - S[0] * S[4], S[0] * S[3] - S[1] * S[1]};
    double x0 = a[0] * d[0] + a[1] * d[1] + a[2] * d[2];
    double x1 = a[1] * d[0] + a[3] * d[1] + a[4] * d[2];
    double x2 = a[2] * d[0] + a[4] * d[1] + a[5] * d[2];
    double q = (d[0] * x0 + d[1] * x1 + d[2] * x2) / dS;
    double bc = pow(d1, 0.25) * pow(d2, 0.25) / sqrt(dS) * exp(-q / 8.0);
    double h2 = 1.0 - bc;
    return h2 > 0.0 ? sqrt(h2) : 0.0;
}

static int64_t uf_find(int64_t *par, int64_t x)
{
    while (par[x] != x) {
        par[x] = par[par[x]];     /* path halving */
        x = par[x];
    }
    return x;
}

int orc_associate(int64_t n_ent, const float *ent_mu, const float *ent_cov, const float *ent_feat,
                  const int32_t *ent_active, const float *ent_w, int64_t n_det, const float *det_mu,
                  const float *det_cov, const float *det_feat, int64_t F, double tau_f, double h_max,
                  int64_t max_m, int64_t *match_cnt, int64_t *match_idx, double *match_h, int64_t *parent,
                  double *out_w, double *out_mu, double *out_cov, double *out_feat)
{
    if (n_ent < 0 || n_det < 0 || F < 1 || max_m < 1) return ORC_EINVAL;
    const int64_t N = n_ent, B = n_det, T = N + B;
    int rc = ORC_OK;
    double *en = (double *)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
    int64_t *uf = (int64_t *)malloc((size_t)(T > 0 ? T : 1) * sizeof(int64_t));
    int64_t *win = (int64_t *)malloc((size_t)(T > 0 ? T : 1) * sizeof(int64_t));
    double *cand_h = (double *)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
    int64_t *cand_i = (int64_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int64_t));
    int64_t *tmp = (int64_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int64_t));
    double *key = (double *)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
    if (!en || !uf || !win || !cand_h || !cand_i || !tmp || !key) { rc = ORC_ENOMEM; goto out; }
    for (int64_t e = 0; e < N; ++e) {
        double ss = 0.0;
        for (int64_t k = 0; k < F; ++k) ss += (double)ent_feat[e * F + k] * ent_feat[e * F + k];
        en[e] = sqrt(ss);
    }
    /* slot accessors: entities 0..N-1, detections N..N+B-1 */
#define MU(x, k) ((x) < N ? (double)ent_mu[(int64_t)(k) * N + (x)] : (double)det_mu[(int64_t)(k) * B + (x) - N])
#define CV(x, k) ((x) < N ? (double)ent_cov[(int64_t)(k) * N + (x)] : (double)det_cov[(int64_t)(k) * B + (x) - N])
#define FT(x, k) ((x) < N ? (double)ent_feat[(x) * F + (k)] : (double)det_feat[((x) - N) * F + (k)])
#define WT(x) ((x) < N ? (double)ent_w[x] : 1.0)

    /* 3. neighbour search */
    for (int64_t t = 0; t < T; ++t) uf[t] = t;
    for (int64_t d = 0; d < B; ++d) {
        double dn = 0.0, mud[3], cd[6];
        for (int64_t k = 0; k < F; ++k) dn += (double)det_feat[d * F + k] * det_feat[d * F + k];
        dn = sqrt(dn);
        for (int k = 0; k < 3; ++k) mud[k] = det_mu[(int64_t)k * B + d];
        for (int k = 0; k < 6; ++k) cd[k] = det_cov[(int64_t)k * B + d];
        int64_t nc = 0;
        for (int64_t e = 0; e < N; ++e) {
            if (!ent_active[e]) continue;
            double dot = 0.0;
            for (int64_t k = 0; k < F; ++k) dot += (double)det_feat[d * F + k] * ent_feat[e * F + k];
            if (!(dn > 0.0 && en[e] > 0.0) || dot / (dn * en[e]) < tau_f) continue;
            double mue[3], ce[6];
            for (int k = 0; k < 3; ++k) mue[k] = ent_mu[(int64_t)k * N + e];
            for (int k = 0; k < 6; ++k) ce[k] = ent_cov[(int64_t)k * N + e];
            double h = orc_hellinger(mud, cd, mue, ce);
            if (h <= h_max) {
                cand_h[nc] = h;
                cand_i[nc] = e;
                ++nc;
            }
        }
        /* sort by H ascending, lower index on ties: sort_by_value orders by
         * larger value first and lower index first, so sort -H over positions */
        for (int64_t i = 0; i < nc; ++i) key[i] = -cand_h[i];
        sort_by_value(nc, key, tmp, win);
        match_cnt[d] = nc;
        for (int64_t j = 0; j < max_m; ++j) {
            if (j < nc) {
                int64_t e = cand_i[tmp[j]];
                match_idx[d * max_m + j] = e;
                match_h[d * max_m + j] = cand_h[tmp[j]];
                /* 4. union of the detection with its match */
                int64_t a = uf_find(uf, N + d), b = uf_find(uf, e);
                if (a != b) uf[a] = b;
            } else {
                match_idx[d * max_m + j] = -1;
                match_h[d * max_m + j] = -1.0;
            }
        }
    }
    /* 4. winners: per component root, the entity of largest w, lower index on ties */
    for (int64_t t = 0; t < T; ++t) win[t] = -1;
    for (int64_t e = 0; e < N; ++e) {
        int64_t r = uf_find(uf, e);
        if (win[r] < 0 || ent_w[e] > ent_w[win[r]] || (ent_w[e] == ent_w[win[r]] && e < win[r])) win[r] = e;
    }
    for (int64_t t = 0; t < T; ++t) {
        int64_t r = uf_find(uf, t);
        parent[t] = win[r] >= 0 ? win[r] : t;       /* a component without an entity: a lone detection */
    }
    /* 5. fusion: winners gather their members */
    for (int64_t t = 0; t < T; ++t) {
        out_w[t] = 0.0;
        for (int k = 0; k < 3; ++k) out_mu[(int64_t)k * T + t] = 0.0;
        for (int k = 0; k < 6; ++k) out_cov[(int64_t)k * T + t] = 0.0;
        for (int64_t k = 0; k < F; ++k) out_feat[t * F + k] = 0.0;
    }
    for (int64_t t = 0; t < T; ++t) {              /* w and w mu */
        int64_t g = parent[t];
        double w = WT(t);
        out_w[g] += w;
        for (int k = 0; k < 3; ++k) out_mu[(int64_t)k * T + g] += w * MU(t, k);
        for (int64_t k = 0; k < F; ++k) out_feat[g * F + k] += w * FT(t, k);
    }
    for (int64_t g = 0; g < T; ++g) {
        if (parent[g] != g) continue;
        if (!(out_w[g] > 0.0)) continue;
        for (int k = 0; k < 3; ++k) out_mu[(int64_t)k * T + g] /= out_w[g];
        for (int64_t k = 0; k < F; ++k) out_feat[g * F + k] /= out_w[g];
    }
    for (int64_t t = 0; t < T; ++t) {              /* w (S_i + (mu_i - mu)(mu_i - mu)') */
        int64_t g = parent[t];
        double w = WT(t), dm[3];
        for (int k = 0; k < 3; ++k) dm[k] = MU(t, k) - out_mu[(int64_t)k * T + g];
        const int ix[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
        for (int k = 0; k < 6; ++k)
            out_cov[(int64_t)k * T + g] += w * (CV(t, k) + dm[ix[k][0]] * dm[ix[k][1]]);
    }
    for (int64_t g = 0; g < T; ++g) {
        if (parent[g] != g || !(out_w[g] > 0.0)) continue;
        for (int k = 0; k < 6; ++k) out_cov[(int64_t)k * T + g] /= out_w[g];
    }
    /* merged-away slots keep w = 0 and zero statistics */
#undef MU
#undef CV
#undef FT
#undef WT
out:
    free(en); free(uf); free(win); free(cand_h); free(cand_i); free(tmp); free(key);
    return rc;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
