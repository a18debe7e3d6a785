/*
 * CPU oracle for the base-ranking + Tabu swap search of
 * "Algorithms for Optimizing Fleet Staging of Air Ambulances" (Tassone, Pond,
 * Choudhury, arXiv 2001.05291).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * Plain, slow, obviously correct: every function is a direct restatement of
 * the definition it cites, with no blocking or fusion.  Integer arithmetic
 * throughout; float64 appears only in the leg distance (one sqrt per leg).
 *
 * Model (Sec. 3, restated for identical vehicles and a coverage range R):
 *   c[b][m]  round-trip cost of mission m from base b: base -> pickup ->
 *            drop-off -> same base (Sec. 3 mission definition), each leg the
 *            ceiling of the Euclidean distance in metres (Sec. 3 allows a
 *            Euclidean metric for simulated data in place of Eq. 1).
 *   f(c)     (1, c) if c <= R, else (0, 0): covered flag and distance.
 *   F(O)     sum over missions of f(min over open bases o of c[o][m]); a
 *            placement is better when it covers more missions, then when its
 *            covered distance is smaller (Eq. 2 minimises total distance; the
 *            coverage goal is the paper's stated aim, Sec. 1).
 *
 * Parity status of each function is listed in its comment.  The whole-run Tabu
 * trajectory is "parity unpinned" beyond the checks in the test suite: the
 * paper gives no worked trajectory, so the trajectory's definition is the
 * reading of Alg. 3 written below.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_INF INT32_MAX

/* ------------------------------------------------------------------------ */
/* Leg distance (Sec. 3, Eq. 1 replaced by planar Euclidean distance).       */
/* ceil of the correctly rounded float64 square root of the exact integer    */
/* squared distance.                                                          */
/* ------------------------------------------------------------------------ */
int32_t oracle_leg(int32_t x1, int32_t y1, int32_t x2, int32_t y2)
{
    int64_t dx = (int64_t)x1 - (int64_t)x2;
    int64_t dy = (int64_t)y1 - (int64_t)y2;
    int64_t sq = dx * dx + dy * dy;
    double d = sqrt((double)sq);
    return (int32_t)ceil(d);
}

/* Eq. 1 (Haversine) between (latitude, longitude) points given in integer
 * microdegrees, on a sphere of radius 6,371,000 m, rounded up to metres:
 *   d = 2 r asin(sqrt(sin^2(dphi / 2) + cos(phi1) cos(phi2) sin^2(dpsi / 2))).
 * The argument of the square root is capped at 1 (antipodes under rounding). */
#define ORACLE_EARTH_RADIUS_M 6371000.0
#define ORACLE_UDEG_TO_RAD (3.14159265358979323846 / 180.0 * 1e-6)

int32_t oracle_leg_haversine(int32_t lat1, int32_t lon1, int32_t lat2, int32_t lon2)
{
    double phi1 = (double)lat1 * ORACLE_UDEG_TO_RAD, phi2 = (double)lat2 * ORACLE_UDEG_TO_RAD;
    double dphi = (double)(lat2 - lat1) * ORACLE_UDEG_TO_RAD;
    double dpsi = (double)(lon2 - lon1) * ORACLE_UDEG_TO_RAD;
    double sp = sin(0.5 * dphi), sl = sin(0.5 * dpsi);
    double h = sp * sp + (cos(phi1) * cos(phi2)) * (sl * sl);
    if (h > 1.0) h = 1.0;
    double d = (2.0 * ORACLE_EARTH_RADIUS_M) * asin(sqrt(h));
    return (int32_t)ceil(d);
}

/* Round-trip cost of mission m flown from base b: the three legs of the
 * mission of Sec. 3 (base -> pickup, pickup -> drop-off, drop-off -> base),
 * Euclidean on metres (metric 0) or Eq. 1's Haversine on microdegrees (1). */
int32_t oracle_mission_cost_metric(const int32_t *base_xy, const int32_t *pick_xy,
                                   const int32_t *drop_xy, int32_t b, int32_t m, int32_t metric)
{
    int32_t bx = base_xy[2 * b], by = base_xy[2 * b + 1];
    int32_t px = pick_xy[2 * m], py = pick_xy[2 * m + 1];
    int32_t qx = drop_xy[2 * m], qy = drop_xy[2 * m + 1];
    if (metric == 1)
        return oracle_leg_haversine(bx, by, px, py) + oracle_leg_haversine(px, py, qx, qy) +
               oracle_leg_haversine(qx, qy, bx, by);
    return oracle_leg(bx, by, px, py) + oracle_leg(px, py, qx, qy) + oracle_leg(qx, qy, bx, by);
}

int32_t oracle_mission_cost(const int32_t *base_xy, const int32_t *pick_xy,
                            const int32_t *drop_xy, int32_t b, int32_t m)
{
    return oracle_mission_cost_metric(base_xy, pick_xy, drop_xy, b, m, 0);
}

/* ------------------------------------------------------------------------ */
/* Distance table (Sec. 3 matrices D/E; Alg. 1 lines building Distances).   */
/* cost is B x M, row-major (row = base).                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t B, M, m0, m1, metric;
    const int32_t *base_xy, *pick_xy, *drop_xy;
    int32_t *cost;
} table_job;

static void *table_worker(void *p)
{
    table_job *t = (table_job *)p;
    for (int32_t b = 0; b < t->B; b++)
        for (int32_t m = t->m0; m < t->m1; m++)
            t->cost[(size_t)b * t->M + m] =
                oracle_mission_cost_metric(t->base_xy, t->pick_xy, t->drop_xy, b, m, t->metric);
    return NULL;
}

void oracle_cost_table_metric(int32_t B, int32_t M, const int32_t *base_xy, const int32_t *pick_xy,
                              const int32_t *drop_xy, int32_t *cost, int32_t nthreads, int32_t metric);

void oracle_cost_table(int32_t B, int32_t M, const int32_t *base_xy, const int32_t *pick_xy,
                       const int32_t *drop_xy, int32_t *cost, int32_t nthreads)
{
    oracle_cost_table_metric(B, M, base_xy, pick_xy, drop_xy, cost, nthreads, 0);
}

void oracle_cost_table_metric(int32_t B, int32_t M, const int32_t *base_xy, const int32_t *pick_xy,
                              const int32_t *drop_xy, int32_t *cost, int32_t nthreads, int32_t metric)
{
    if (nthreads < 1) nthreads = 1;
    pthread_t th[256];
    table_job jobs[256];
    if (nthreads > 256) nthreads = 256;
    for (int32_t t = 0; t < nthreads; t++) {
        jobs[t].B = B; jobs[t].M = M;
        jobs[t].m0 = (int32_t)((int64_t)M * t / nthreads);
        jobs[t].m1 = (int32_t)((int64_t)M * (t + 1) / nthreads);
        jobs[t].base_xy = base_xy; jobs[t].pick_xy = pick_xy; jobs[t].drop_xy = drop_xy;
        jobs[t].cost = cost;
        jobs[t].metric = metric;
        if (nthreads == 1) table_worker(&jobs[t]);
        else pthread_create(&th[t], NULL, table_worker, &jobs[t]);
    }
    if (nthreads > 1)
        for (int32_t t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------ */
/* Objective (Eq. 2 with coverage): f(c) and F(O).                           */
/* ------------------------------------------------------------------------ */
static void f_of(int32_t c, int32_t R, int64_t *cov, int64_t *dist)
{
    if (c <= R) { *cov = 1; *dist = c; }
    else        { *cov = 0; *dist = 0; }
}

/* 1 if (c1, d1) is strictly better than (c2, d2): more covered, then less distance. */
static int better(int64_t c1, int64_t d1, int64_t c2, int64_t d2)
{
    if (c1 != c2) return c1 > c2;
    return d1 < d2;
}

/* F(O) by its definition: each mission is flown from its nearest open base. */
void oracle_evaluate(int32_t B, int32_t M, const int32_t *cost, int32_t K, const int32_t *open,
                     int32_t R, int64_t *out_cov, int64_t *out_dist)
{
    (void)B;
    int64_t cov = 0, dist = 0;
    for (int32_t m = 0; m < M; m++) {
        int32_t best = ORACLE_INF;
        for (int32_t k = 0; k < K; k++) {
            int32_t c = cost[(size_t)open[k] * M + m];
            if (c < best) best = c;
        }
        int64_t fc, fd;
        f_of(best, R, &fc, &fd);
        cov += fc;
        dist += fd;
    }
    *out_cov = cov;
    *out_dist = dist;
}

/* ------------------------------------------------------------------------ */
/* Base Ranking (Alg. 1): sum each base's row of the distance table over all */
/* missions, then take the K bases with the smallest sums (ties: lower base  */
/* index first).  Unavailable bases are not ranked.  Returns 0, or -1 when   */
/* fewer than K bases are available.                                          */
/* ------------------------------------------------------------------------ */
static const int64_t *g_rank_sums;
static int rank_cmp(const void *pa, const void *pb)
{
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    if (g_rank_sums[a] != g_rank_sums[b]) return g_rank_sums[a] < g_rank_sums[b] ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

int32_t oracle_rank(int32_t B, int32_t M, const int32_t *cost, const uint8_t *avail, int32_t K,
                    int32_t *out_open, int64_t *out_rowsum)
{
    int64_t *S = (int64_t *)malloc(sizeof(int64_t) * (size_t)B);
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)B);
    int32_t n = 0;
    for (int32_t b = 0; b < B; b++) {
        int64_t s = 0;
        for (int32_t m = 0; m < M; m++) s += cost[(size_t)b * M + m];
        S[b] = s;
        if (out_rowsum) out_rowsum[b] = s;
        if (!avail || avail[b]) idx[n++] = b;
    }
    int32_t rc = 0;
    if (n < K) rc = -1;
    else {
        g_rank_sums = S;
        qsort(idx, (size_t)n, sizeof(int32_t), rank_cmp);
        for (int32_t k = 0; k < K; k++) out_open[k] = idx[k];
    }
    free(S);
    free(idx);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Ranking of the chosen bases for each mission (Alg. 1, "rank chosen bases  */
/* for each mission"): best b1 and second-best b2 open base of every mission,*/
/* ordered by (cost, base index).  b2 = -1 and b = INF when K = 1.           */
/* ------------------------------------------------------------------------ */
void oracle_best_two(int32_t B, int32_t M, const int32_t *cost, int32_t K, const int32_t *open,
                     int32_t *a, int32_t *b, int32_t *b1, int32_t *b2)
{
    (void)B;
    for (int32_t m = 0; m < M; m++) {
        int32_t i1 = -1, i2 = -1, c1 = ORACLE_INF, c2 = ORACLE_INF;
        for (int32_t k = 0; k < K; k++) {
            int32_t o = open[k];
            int32_t c = cost[(size_t)o * M + m];
            if (i1 < 0 || c < c1 || (c == c1 && o < i1)) {
                i2 = i1; c2 = c1;
                i1 = o; c1 = c;
            } else if (i2 < 0 || c < c2 || (c == c2 && o < i2)) {
                i2 = o; c2 = c;
            }
        }
        a[m] = c1; b[m] = c2; b1[m] = i1; b2[m] = i2;
    }
}

/* ------------------------------------------------------------------------ */
/* Objective of one swap (close i, open j), two independent ways.            */
/* ------------------------------------------------------------------------ */

/* (i) Full recomputation: F(O - i + j) by the definition. */
void oracle_swap_full(int32_t B, int32_t M, const int32_t *cost, int32_t K, const int32_t *open,
                      int32_t R, int32_t i, int32_t j, int64_t *cov, int64_t *dist)
{
    int32_t *o2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    for (int32_t k = 0; k < K; k++) o2[k] = (open[k] == i) ? j : open[k];
    oracle_evaluate(B, M, cost, K, o2, R, cov, dist);
    free(o2);
}

/* (ii) From each mission's best and second-best open base: after closing i
 * and opening j, the new best is min(a, x) when i was not the mission's best
 * base, else min(b, x), with x = c[j][m]. */
void oracle_swap_best_two(int32_t B, int32_t M, const int32_t *cost, int32_t K,
                          const int32_t *open, int32_t R, int32_t i, int32_t j,
                          int64_t *out_cov, int64_t *out_dist)
{
    int32_t *a = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    int32_t *b = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    int32_t *b1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    int32_t *b2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    oracle_best_two(B, M, cost, K, open, a, b, b1, b2);
    int64_t cov = 0, dist = 0;
    for (int32_t m = 0; m < M; m++) {
        int32_t x = cost[(size_t)j * M + m];
        int32_t keep = (b1[m] != i) ? a[m] : b[m];
        int32_t nb = x < keep ? x : keep;
        int64_t fc, fd;
        f_of(nb, R, &fc, &fd);
        cov += fc;
        dist += fd;
    }
    *out_cov = cov;
    *out_dist = dist;
    free(a); free(b); free(b1); free(b2);
}

/* ------------------------------------------------------------------------ */
/* (iii) The whole swap neighbourhood at once, by the fast-interchange      */
/* decomposition (Whitaker 1983; Resende and Werneck 2007):                  */
/*   F(i, j) = V0 + gain[j] + loss[i] + extra[i][j]                          */
/*   V0        = sum_m f(a_m)                                                 */
/*   gain[j]   = sum_m [x < a_m] (f(x) - f(a_m)),            x = c[j][m]     */
/*   loss[i]   = sum_{m: b1_m = i} (f(b_m) - f(a_m))                          */
/*   extra[i][j] = sum_{m: b1_m = i} [x < b_m] (f(max(x, a_m)) - f(b_m))      */
/* Outputs, for every open i and every closed available j, F(i, j) in        */
/* out_cov / out_dist indexed [i * B + j] (global base indices); other       */
/* entries are left untouched.  Loops per mission; threads split missions    */
/* and their integer partials are added in thread order.                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t B, M, m0, m1, R;
    const int32_t *cost;
    const uint8_t *closed_avail; /* 1 for a closed, available base */
    const int32_t *a, *b, *b1;
    int64_t v0c, v0d;
    int64_t *gc, *gd;   /* B */
    int64_t *lc, *ld;   /* B */
    int64_t *ec, *ed;   /* B * B */
} nbhd_job;

static void *nbhd_worker(void *p)
{
    nbhd_job *t = (nbhd_job *)p;
    const int32_t B = t->B, M = t->M, R = t->R;
    for (int32_t m = t->m0; m < t->m1; m++) {
        int32_t am = t->a[m], bm = t->b[m], i = t->b1[m];
        int64_t fac, fad, fbc, fbd;
        f_of(am, R, &fac, &fad);
        f_of(bm, R, &fbc, &fbd);
        t->v0c += fac;
        t->v0d += fad;
        t->lc[i] += fbc - fac;
        t->ld[i] += fbd - fad;
        for (int32_t j = 0; j < B; j++) {
            if (!t->closed_avail[j]) continue;
            int32_t x = t->cost[(size_t)j * M + m];
            if (x < am) {
                int64_t fxc, fxd;
                f_of(x, R, &fxc, &fxd);
                t->gc[j] += fxc - fac;
                t->gd[j] += fxd - fad;
            }
            if (x < bm) {
                int32_t y = x > am ? x : am;
                int64_t fyc, fyd;
                f_of(y, R, &fyc, &fyd);
                t->ec[(size_t)i * B + j] += fyc - fbc;
                t->ed[(size_t)i * B + j] += fyd - fbd;
            }
        }
    }
    return NULL;
}

void oracle_swap_table(int32_t B, int32_t M, const int32_t *cost, const uint8_t *avail,
                       int32_t K, const int32_t *open, int32_t R,
                       int64_t *out_cov, int64_t *out_dist, int32_t nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    int32_t *a = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    int32_t *b = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    int32_t *b1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    int32_t *b2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    oracle_best_two(B, M, cost, K, open, a, b, b1, b2);
    uint8_t *ca = (uint8_t *)calloc((size_t)B, 1);
    for (int32_t j = 0; j < B; j++) ca[j] = (!avail || avail[j]) ? 1 : 0;
    for (int32_t k = 0; k < K; k++) ca[open[k]] = 0;

    nbhd_job jobs[256];
    pthread_t th[256];
    for (int32_t t = 0; t < nthreads; t++) {
        nbhd_job *J = &jobs[t];
        memset(J, 0, sizeof(*J));
        J->B = B; J->M = M; J->R = R; J->cost = cost; J->closed_avail = ca;
        J->a = a; J->b = b; J->b1 = b1;
        J->m0 = (int32_t)((int64_t)M * t / nthreads);
        J->m1 = (int32_t)((int64_t)M * (t + 1) / nthreads);
        J->gc = (int64_t *)calloc((size_t)B, 8); J->gd = (int64_t *)calloc((size_t)B, 8);
        J->lc = (int64_t *)calloc((size_t)B, 8); J->ld = (int64_t *)calloc((size_t)B, 8);
        J->ec = (int64_t *)calloc((size_t)B * B, 8); J->ed = (int64_t *)calloc((size_t)B * B, 8);
        if (nthreads == 1) nbhd_worker(J);
        else pthread_create(&th[t], NULL, nbhd_worker, J);
    }
    if (nthreads > 1)
        for (int32_t t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    for (int32_t t = 1; t < nthreads; t++) {
        nbhd_job *J = &jobs[t];
        jobs[0].v0c += J->v0c; jobs[0].v0d += J->v0d;
        for (int32_t x = 0; x < B; x++) {
            jobs[0].gc[x] += J->gc[x]; jobs[0].gd[x] += J->gd[x];
            jobs[0].lc[x] += J->lc[x]; jobs[0].ld[x] += J->ld[x];
        }
        for (size_t x = 0; x < (size_t)B * B; x++) {
            jobs[0].ec[x] += J->ec[x]; jobs[0].ed[x] += J->ed[x];
        }
    }
    nbhd_job *S = &jobs[0];
    for (int32_t k = 0; k < K; k++) {
        int32_t i = open[k];
        for (int32_t j = 0; j < B; j++) {
            if (!ca[j]) continue;
            size_t ij = (size_t)i * B + j;
            out_cov[ij] = S->v0c + S->gc[j] + S->lc[i] + S->ec[ij];
            out_dist[ij] = S->v0d + S->gd[j] + S->ld[i] + S->ed[ij];
        }
    }
    for (int32_t t = 0; t < nthreads; t++) {
        free(jobs[t].gc); free(jobs[t].gd); free(jobs[t].lc); free(jobs[t].ld);
        free(jobs[t].ec); free(jobs[t].ed);
    }
    free(ca); free(a); free(b); free(b1); free(b2);
}

/* ------------------------------------------------------------------------ */
/* Tabu search over base exchanges (Alg. 3, read for identical vehicles):   */
/*  - the neighbourhood of a placement O is every swap (close i in O, open  */
/*    an available j not in O); with identical vehicles and no capacity the */
/*    mission assignment follows from O, so the three move kinds of Alg. 2/3 */
/*    reduce to these swaps;                                                 */
/*  - the tabu list holds bases: after a move at iteration t both bases are */
/*    tabu until iteration t + tenure (inclusive), i.e. expiry = t+tenure+1,*/
/*    and move (i, j) is tabu at t iff t < expiry[i] or t < expiry[j];      */
/*  - a tabu move is still admissible when it beats the best placement seen */
/*    so far (aspiration); when no move is admissible the best of all moves */
/*    is taken (fallback);                                                   */
/*  - among admissible moves the best is chosen: more covered, then less    */
/*    distance, then lower i, then lower j (global base indices);           */
/*  - accept_worsening = 0 is the paper's improving-only rule (Sec. 4.3):   */
/*    the search stops when the chosen move does not strictly improve.      */
/* eval_mode: 0 = neighbourhood table (iii), 1 = best/second-best per swap  */
/* (ii), 2 = full recomputation per swap (i).                               */
/* ------------------------------------------------------------------------ */
/* One trajectory entry: iteration, closed base, opened base, flags, and the
 * objective of the placement after the move. */
typedef struct {
    int32_t iter, i, j, flags;
    int64_t cov, dist;
} oracle_move;

enum { MOVE_FALLBACK = 1, MOVE_ASPIRATION = 2, MOVE_NEW_BEST = 4 };

typedef struct {
    /* inputs */
    int32_t iters, tenure, accept_worsening, eval_mode, nthreads;
    int32_t t0;                 /* iteration number of the first step (resume) */
    const int32_t *expiry_in;   /* B, or NULL for all zero */
    const int32_t *best_in;     /* K, or NULL: best-so-far starts at the start placement */
    int64_t best_cov_in, best_dist_in;
    int32_t best_iter_in;
    /* outputs */
    int32_t n_moves;
    int32_t best_iter;
    int64_t best_cov, best_dist;
    int64_t final_cov, final_dist;
} oracle_tabu_io;

int32_t oracle_tabu(int32_t B, int32_t M, const int32_t *cost, const uint8_t *avail, int32_t K,
                    int32_t R, const int32_t *start_open, oracle_tabu_io *io,
                    oracle_move *traj, int32_t *best_open, int32_t *final_open,
                    int32_t *expiry_out)
{
    int32_t *open = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    int32_t *expiry = (int32_t *)calloc((size_t)B, sizeof(int32_t));
    uint8_t *is_open = (uint8_t *)calloc((size_t)B, 1);
    int64_t *Fc = NULL, *Fd = NULL;
    memcpy(open, start_open, sizeof(int32_t) * (size_t)K);
    for (int32_t k = 0; k < K; k++) is_open[open[k]] = 1;
    if (io->expiry_in) memcpy(expiry, io->expiry_in, sizeof(int32_t) * (size_t)B);
    if (io->eval_mode == 0) {
        Fc = (int64_t *)malloc(sizeof(int64_t) * (size_t)B * B);
        Fd = (int64_t *)malloc(sizeof(int64_t) * (size_t)B * B);
    }

    int64_t cur_c, cur_d;
    oracle_evaluate(B, M, cost, K, open, R, &cur_c, &cur_d);
    int64_t best_c, best_d;
    int32_t best_iter;
    if (io->best_in) {
        memcpy(best_open, io->best_in, sizeof(int32_t) * (size_t)K);
        best_c = io->best_cov_in; best_d = io->best_dist_in; best_iter = io->best_iter_in;
    } else {
        memcpy(best_open, open, sizeof(int32_t) * (size_t)K);
        best_c = cur_c; best_d = cur_d; best_iter = -1;
    }

    int32_t n_moves = 0;
    for (int32_t step = 0; step < io->iters; step++) {
        int32_t t = io->t0 + step;
        if (io->eval_mode == 0)
            oracle_swap_table(B, M, cost, avail, K, open, R, Fc, Fd, io->nthreads);

        int have_adm = 0, have_any = 0;
        int32_t ai = 0, aj = 0, xi = 0, xj = 0, a_tabu = 0;
        int64_t ac = 0, ad = 0, xc = 0, xd = 0;
        for (int32_t k = 0; k < K; k++) {
            int32_t i = open[k];
            for (int32_t j = 0; j < B; j++) {
                if (is_open[j] || (avail && !avail[j])) continue;
                int64_t c, d;
                if (io->eval_mode == 0) { c = Fc[(size_t)i * B + j]; d = Fd[(size_t)i * B + j]; }
                else if (io->eval_mode == 1) oracle_swap_best_two(B, M, cost, K, open, R, i, j, &c, &d);
                else oracle_swap_full(B, M, cost, K, open, R, i, j, &c, &d);
                /* the order of the whole key: covered desc, distance asc, i asc, j asc */
                int tabu = (t < expiry[i]) || (t < expiry[j]);
                int admissible = !tabu || better(c, d, best_c, best_d);
                if (!have_any || better(c, d, xc, xd) ||
                    (c == xc && d == xd && (i < xi || (i == xi && j < xj)))) {
                    have_any = 1; xc = c; xd = d; xi = i; xj = j;
                }
                if (admissible && (!have_adm || better(c, d, ac, ad) ||
                                   (c == ac && d == ad && (i < ai || (i == ai && j < aj))))) {
                    have_adm = 1; ac = c; ad = d; ai = i; aj = j; a_tabu = tabu;
                }
            }
        }
        if (!have_any) break; /* no closed available base: nothing to swap */
        int32_t flags = 0;
        int32_t mi, mj;
        int64_t mc, md;
        if (have_adm) {
            mi = ai; mj = aj; mc = ac; md = ad;
            if (a_tabu) flags |= MOVE_ASPIRATION;
        } else {
            mi = xi; mj = xj; mc = xc; md = xd;
            flags |= MOVE_FALLBACK;
        }
        if (!io->accept_worsening && !better(mc, md, cur_c, cur_d)) break;

        for (int32_t k = 0; k < K; k++)
            if (open[k] == mi) open[k] = mj;
        is_open[mi] = 0;
        is_open[mj] = 1;
        expiry[mi] = t + io->tenure + 1;
        expiry[mj] = t + io->tenure + 1;
        cur_c = mc; cur_d = md;
        if (better(mc, md, best_c, best_d)) {
            best_c = mc; best_d = md; best_iter = t;
            memcpy(best_open, open, sizeof(int32_t) * (size_t)K);
            flags |= MOVE_NEW_BEST;
        }
        if (traj) {
            traj[n_moves].iter = t;
            traj[n_moves].i = mi; traj[n_moves].j = mj; traj[n_moves].flags = flags;
            traj[n_moves].cov = mc; traj[n_moves].dist = md;
        }
        n_moves++;
    }

    io->n_moves = n_moves;
    io->best_iter = best_iter;
    io->best_cov = best_c; io->best_dist = best_d;
    io->final_cov = cur_c; io->final_dist = cur_d;
    if (final_open) memcpy(final_open, open, sizeof(int32_t) * (size_t)K);
    if (expiry_out) memcpy(expiry_out, expiry, sizeof(int32_t) * (size_t)B);
    free(open); free(expiry); free(is_open); free(Fc); free(Fd);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact optimum by enumeration of every K-subset of the available bases,   */
/* in lexicographic order; the first subset with the best objective wins.   */
/* This is the homogeneous special case of the model of Eq. 2-11 with a     */
/* coverage range.  Returns the number of subsets evaluated.                */
/* ------------------------------------------------------------------------ */
int64_t oracle_bruteforce(int32_t B, int32_t M, const int32_t *cost, const uint8_t *avail,
                          int32_t K, int32_t R, int32_t *best_open, int64_t *best_cov,
                          int64_t *best_dist)
{
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)B);
    int32_t n = 0;
    for (int32_t b = 0; b < B; b++)
        if (!avail || avail[b]) ids[n++] = b;
    if (K > n || K < 1) { free(ids); return 0; }
    int32_t *sel = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    int32_t *open = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
    for (int32_t k = 0; k < K; k++) sel[k] = k;
    int64_t count = 0, bc = -1, bd = 0;
    for (;;) {
        for (int32_t k = 0; k < K; k++) open[k] = ids[sel[k]];
        int64_t c, d;
        oracle_evaluate(B, M, cost, K, open, R, &c, &d);
        count++;
        if (bc < 0 || better(c, d, bc, bd)) {
            bc = c; bd = d;
            memcpy(best_open, open, sizeof(int32_t) * (size_t)K);
        }
        int32_t k = K - 1;
        while (k >= 0 && sel[k] == n - K + k) k--;
        if (k < 0) break;
        sel[k]++;
        for (int32_t q = k + 1; q < K; q++) sel[q] = sel[q - 1] + 1;
    }
    *best_cov = bc;
    *best_dist = bd;
    free(ids); free(sel); free(open);
    return count;
}
