/*
 * stage.h -- C ABI of the GB300 fleet-staging engine.
 *
 * The engine places K identical vehicles at K of B candidate bases so that as
 * many round-trip missions as possible are within range R, and among those
 * placements the total round-trip distance is smallest.  It implements the
 * base ranking of Alg. 1 and the Tabu search of Alg. 3 of "Algorithms for
 * Optimizing Fleet Staging of Air Ambulances" (arXiv 2001.05291), read for
 * identical vehicles:
 *   - a mission goes base -> pickup -> drop-off -> same base (Sec. 3);
 *   - each leg costs ceil(Euclidean distance) in integer metres, the planar
 *     metric that Sec. 3 allows for simulated data in place of Eq. 1;
 *   - c[b][m] = leg(b, pickup_m) + leg(pickup_m, drop_m) + leg(drop_m, b);
 *   - f(c) = (1, c) if c <= R else (0, 0);  F(O) = sum_m f(min_{o in O} c[o][m]);
 *     more covered missions is better, then a smaller distance (Eq. 2 with
 *     the coverage aim of Sec. 1);
 *   - the Tabu neighbourhood is every swap (close i in O, open available j
 *     not in O), evaluated in full each iteration on the GPU.
 *
 * Conventions
 *   - Every function returns a stage_status: STAGE_OK (0), STAGE_PENDING (1)
 *     or a negative error.  stage_last_error() gives the message of the last
 *     error on a context.
 *   - Handles are opaque.  Input arrays are copied in (the caller keeps
 *     ownership); outputs go to caller-allocated HOST buffers unless a flag
 *     says otherwise.  Nothing returned points into library memory.
 *   - Coordinates are int32 metres with |x|, |y| <= STAGE_MAX_COORD, so that
 *     every squared leg length is below 2^52 and the float64 square root of
 *     the exact integer is correctly rounded to the right ceiling.
 *   - Base ids are 0-based indices into the instance's base array.
 *   - All results are integers and are bit-identical run to run.
 *   - Calls on one context are serialised internally (the batch engine's
 *     worker thread shares the context); STAGE_THREADSAFE is accepted for
 *     compatibility and changes nothing.
 *   - The library never falls back to the CPU: without a CUDA device every
 *     call that needs one returns STAGE_ERR_CUDA.
 */
#ifndef STAGE_H
#define STAGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define STAGE_API __attribute__((visibility("default")))
#else
#define STAGE_API
#endif

typedef int32_t stage_status;

#define STAGE_OK                0
#define STAGE_PENDING           1
#define STAGE_ERR_INVALID_ARG  (-1)  /* malformed argument (NULL, K > B, duplicate base, ...) */
#define STAGE_ERR_OUT_OF_RANGE (-2)  /* a size or coordinate beyond the limits below */
#define STAGE_ERR_NO_MEMORY    (-3)  /* device allocation failed */
#define STAGE_ERR_ADMISSION    (-4)  /* over the context's HBM budget, or no free slot */
#define STAGE_ERR_TIMEOUT      (-5)  /* a bounded device-side wait or a poll timed out */
#define STAGE_ERR_CUDA         (-6)  /* CUDA runtime error, or no device */
#define STAGE_ERR_INTERNAL     (-7)  /* a device self-check failed */
#define STAGE_ERR_NOT_FOUND    (-8)  /* unknown instance handle or ticket */

#define STAGE_MAX_COORD    (1 << 24)   /* |x|, |y| <= 16,777,216 m */
#define STAGE_MAX_BASES    65535
#define STAGE_MAX_MISSIONS (1 << 24)
#define STAGE_MAX_K        1024

/* context flags */
#define STAGE_THREADSAFE   1u   /* accepted; calls are always serialised */
#define STAGE_PROFILE      2u   /* time every kernel launch with CUDA events */
#define STAGE_AUTOTUNE     4u   /* tune the swap pass's tile the first time a shape is met */
#define STAGE_FULL_PASS    8u   /* Tabu searches (stage_tabu_run) re-evaluate the whole swap
                                   neighbourhood by a full pass over the cost table every
                                   iteration.  By default the neighbourhood's terms are kept
                                   across iterations and updated for the missions whose best or
                                   second-best open base changed (the same values exactly),
                                   the whole search in one cooperative launch, whenever that
                                   launch takes the shape (K <= 256, at most 2048 bases) and the
                                   search is not one small enough for a single block; with
                                   STAGE_NO_PERSIST, as per-iteration launches for tables well
                                   beyond the L2 cache (candidate rows x missions x 4 B >=
                                   256 MiB) and a full pass otherwise.  That form keeps a mission-major
                                   copy of the cost table with the instance (the table's size
                                   again, built on the first such search and again after
                                   stage_update_instance) and 32 bytes per mission; when the
                                   context's HBM budget has no room for them the search takes
                                   the full pass */
#define STAGE_INCREMENTAL 16u   /* that incremental update whatever the table's size */
#define STAGE_NO_PERSIST  32u   /* run the incremental update as three kernel launches per
                                   iteration; by default, where the shape allows (K <= 256,
                                   B <= 2048), the whole search is one persistent cooperative
                                   launch whose CTAs meet at grid-wide barriers, each wait
                                   bounded by spin_limit */

/* instance descriptor flags */
#define STAGE_DESC_DEVICE  1u   /* base_xy/pick_xy/drop_xy/base_available are device pointers */
#define STAGE_DESC_HAVERSINE 2u /* coordinates are (latitude, longitude) in integer microdegrees and
                                   every leg is the Haversine distance of Eq. 1 on a sphere of radius
                                   STAGE_EARTH_RADIUS_M, in metres, rounded up */
#define STAGE_EARTH_RADIUS_M 6371000.0
#define STAGE_MAX_LAT_UDEG  90000000    /* |latitude| <= 90 degrees */
#define STAGE_MAX_LON_UDEG  180000000   /* |longitude| <= 180 degrees */

/* trajectory flags */
#define STAGE_MOVE_FALLBACK   1  /* every move was tabu and none beat the best: best of all taken */
#define STAGE_MOVE_ASPIRATION 2  /* a tabu move admitted because it beats the best so far */
#define STAGE_MOVE_NEW_BEST   4  /* the move produced a new best placement */

typedef struct stage_ctx stage_ctx;
typedef uint64_t stage_inst;   /* instance handle; 0 is never a valid handle */

/* Optional device allocator (e.g. PyTorch's caching allocator).  alloc returns
 * a device pointer aligned to 256 bytes or NULL; free releases it. */
typedef void *(*stage_alloc_fn)(size_t bytes, void *user);
typedef void (*stage_free_fn)(void *ptr, size_t bytes, void *user);

typedef struct {
    int32_t device;            /* CUDA device ordinal */
    uint32_t flags;            /* STAGE_THREADSAFE | STAGE_PROFILE */
    uint64_t hbm_budget_bytes; /* cap on the context's device memory; 0 = device limit */
    int32_t max_slots;         /* batch/serving slots run concurrently; 0 = 8 */
    int32_t reserved0;
    int64_t spin_limit;        /* bound on every device-side wait (the persistent search's grid
                                  barriers and shared-memory ring), in polls; 0 = 1<<26.  A wait
                                  that gives up ends the kernel and the call returns
                                  STAGE_ERR_TIMEOUT; the context stays usable */
    stage_alloc_fn alloc;      /* NULL = cudaMalloc */
    stage_free_fn free;        /* must be set iff alloc is */
    void *alloc_user;
    void *stream;              /* cudaStream_t to run on; NULL = a stream the context owns */
} stage_config;

/* Problem data (Sec. 3): B candidate bases and M missions.  Coordinates are
 * interleaved (x0, y0, x1, y1, ...) int32 metres in a plane (Euclidean legs),
 * or, with STAGE_DESC_HAVERSINE, interleaved (latitude, longitude) pairs in
 * microdegrees (Haversine legs, Eq. 1).  base_available may be NULL (all
 * available); an unavailable base is never opened. */
typedef struct {
    int32_t B;
    int32_t M;
    uint32_t flags;            /* STAGE_DESC_DEVICE | STAGE_DESC_HAVERSINE */
    int32_t reserved0;
    const int32_t *base_xy;    /* [2*B] */
    const int32_t *pick_xy;    /* [2*M] pickup points */
    const int32_t *drop_xy;    /* [2*M] drop-off points */
    const uint8_t *base_available; /* [B] or NULL */
} stage_instance_desc;

/* One Tabu iteration: the swap applied and the objective after it. */
typedef struct {
    int32_t iter;   /* iteration number t */
    int32_t i;      /* base closed */
    int32_t j;      /* base opened */
    int32_t flags;  /* STAGE_MOVE_* */
    int64_t cov;    /* missions covered after the move */
    int64_t dist;   /* covered distance after the move (metres) */
} stage_move;

/* Resumable Tabu state (placement, tabu expiries, best so far).  All arrays
 * are caller-owned host buffers. */
typedef struct {
    int32_t t;              /* iteration number of the next step */
    int32_t best_iter;      /* iteration that produced the best (-1: the start) */
    int64_t best_cov;
    int64_t best_dist;
    int32_t *open;          /* [K] current placement */
    int32_t *best_open;     /* [K] best placement so far */
    int32_t *tabu_expiry;   /* [B] move (i, j) is tabu at t iff t < expiry[i] or t < expiry[j] */
} stage_tabu_state;

typedef struct {
    int32_t K;                /* vehicles, 1 <= K <= min(B, STAGE_MAX_K) */
    int32_t R;                /* range in metres, 0 <= R < INT32_MAX */
    int32_t iters;            /* iterations (Alg. 3 outer loop), >= 0 */
    int32_t tenure;           /* iterations a moved base stays tabu, >= 0 */
    int32_t accept_worsening; /* 1: best admissible move even if worse; 0: stop when no
                                 move improves (the improving-only rule of Sec. 4.3) */
    int32_t reserved0;
    const int32_t *start_open;        /* [K] start placement, or NULL: stage_rank_bases */
    const stage_tabu_state *resume;   /* continue from this state, or NULL */
} stage_tabu_params;

typedef struct {
    int32_t n_moves;        /* moves applied (== iterations unless the search stopped) */
    int32_t best_iter;
    int64_t best_cov;
    int64_t best_dist;
    int64_t final_cov;
    int64_t final_dist;
    int32_t *best_open;     /* [K] caller buffer or NULL; filled sorted ascending */
    int32_t *final_open;    /* [K] caller buffer or NULL; filled sorted ascending */
    stage_tabu_state *end_state; /* NULL, or filled (caller's arrays) to resume from */
} stage_tabu_result;

/* ------------------------------------------------------------------ context */

/* Create a context on cfg->device (cfg may be NULL: device 0, defaults).
 * Errors: STAGE_ERR_CUDA (no device), STAGE_ERR_INVALID_ARG. */
STAGE_API stage_status stage_create(const stage_config *cfg, stage_ctx **out);

/* Free every instance, slot and buffer of the context.  NULL is a no-op. */
STAGE_API stage_status stage_destroy(stage_ctx *ctx);

/* Copy the last error message (NUL-terminated, truncated to n) into buf. */
STAGE_API stage_status stage_last_error(const stage_ctx *ctx, char *buf, size_t n);

/* Library version as major*10000 + minor*100 + patch. */
STAGE_API int32_t stage_version(void);

/* Device memory currently held by the context, in bytes. */
STAGE_API stage_status stage_memory_used(const stage_ctx *ctx, uint64_t *out_bytes);

/* ----------------------------------------------------------------- instance */

/* Copy an instance in and build its B x M round-trip cost table on the device
 * (Sec. 3 distance matrices; the summed base-pickup-destination distance of
 * Alg. 1).  The table is int32 row-major, one row per base, missions padded
 * to a multiple of 64 with INT32_MAX.
 * Errors: STAGE_ERR_INVALID_ARG (NULL pointers, B < 1, M < 1),
 * STAGE_ERR_OUT_OF_RANGE (B, M or a coordinate beyond the limits),
 * STAGE_ERR_ADMISSION (over the HBM budget), STAGE_ERR_NO_MEMORY. */
STAGE_API stage_status stage_load_instance(stage_ctx *ctx, const stage_instance_desc *desc, stage_inst *out);

/* Release an instance and its device memory. */
STAGE_API stage_status stage_unload_instance(stage_ctx *ctx, stage_inst inst);

/* Base ranking (Alg. 1): S[b] = sum over missions of c[b][m] (int64), then the
 * K available bases with the smallest S, ties to the lower index.  out_open
 * [K] receives them in rank order; out_rowsum [B] (nullable) receives S.
 * Errors: STAGE_ERR_INVALID_ARG (K < 1, fewer than K available bases). */
STAGE_API stage_status stage_rank_bases(stage_ctx *ctx, stage_inst inst, int32_t K, int32_t *out_open,
                              int64_t *out_rowsum);

/* F(O) for the placement open[K] (distinct, available base ids) at range R:
 * missions covered and their summed distance (Eq. 2 with coverage).
 * Errors: STAGE_ERR_INVALID_ARG (duplicate, unknown or unavailable base). */
STAGE_API stage_status stage_evaluate_placement(stage_ctx *ctx, stage_inst inst, const int32_t *open,
                                      int32_t K, int32_t R, int64_t *out_cov, int64_t *out_dist);

/* The whole swap neighbourhood of the placement open[K] at range R: for every
 * slot k and every base j, out_cov[k*B + j], out_dist[k*B + j] = F(O - open[k]
 * + j) when j is closed and available, else -1.  (Alg. 3 evaluates these
 * moves one by one; here one streaming pass of the table computes all.) */
STAGE_API stage_status stage_evaluate_swaps(stage_ctx *ctx, stage_inst inst, const int32_t *open,
                                  int32_t K, int32_t R, int64_t *out_cov, int64_t *out_dist);

/* Tabu search (Alg. 3, read for identical vehicles):
 *   - start: params->start_open, or the ranking of Alg. 1, or params->resume;
 *   - each iteration evaluates every swap, takes the best admissible one
 *     (not tabu, or strictly better than the best so far), ordered by
 *     (covered desc, distance asc, i asc, j asc); when every move is tabu and
 *     none beats the best, the best of all moves is taken (STAGE_MOVE_FALLBACK);
 *   - both bases of the move become tabu for `tenure` iterations;
 *   - stops early when no closed available base exists, or, with
 *     accept_worsening = 0, when the chosen move does not improve.
 * traj (nullable) receives one stage_move per applied move ([iters]).
 * Errors: STAGE_ERR_INVALID_ARG, STAGE_ERR_OUT_OF_RANGE, STAGE_ERR_INTERNAL
 * (a device self-check failed: the incremental objective disagreed with the
 * chosen move's). */
STAGE_API stage_status stage_tabu_run(stage_ctx *ctx, stage_inst inst, const stage_tabu_params *params,
                            stage_tabu_result *result, stage_move *traj);

/* Many Tabu searches (Alg. 3, each exactly as stage_tabu_run computes it)
 * evaluated together: search k runs on the resident instance insts[k] with
 * params[k]; results[k] and trajs[k] (trajs nullable, and each entry nullable;
 * [params[k].iters] moves) receive what stage_tabu_run would return.  Every
 * search whose shape the persistent search takes (K <= 256, at most 2048
 * bases) and that has a move to make runs inside ONE cooperative launch:
 * each on a gang of CTAs sized by its estimated work, the gangs placed on the
 * GPU's CTAs largest first and run in one global order, so that their waits
 * on one another are bounded.  Those searches use the incremental
 * neighbourhood (one full pass, then the update of the swap terms from the
 * missions each move touched), so each instance gets its mission-major table
 * copy on first use, kept with it.  Before that launch, the rankings of the
 * searches that start from Alg. 1 run as one grouped launch, and so do the
 * searches' first full passes.  The other searches run one after another
 * afterwards.  An instance may appear once per call; the call returns when all
 * are done.
 * Errors: STAGE_ERR_NOT_FOUND (unknown instance), STAGE_ERR_INVALID_ARG (n < 0,
 * NULL arrays, an instance named twice, or a malformed params entry, checked
 * as stage_tabu_run checks it), STAGE_ERR_NO_MEMORY / STAGE_ERR_ADMISSION (no
 * room for the copies or scratch), STAGE_ERR_TIMEOUT (a wait between a
 * search's CTAs gave up after the context's spin limit), STAGE_ERR_INTERNAL
 * (a device self-check failed).  An error in checking or setting up a search
 * returns at once; errors of the searches themselves are reported once every
 * search has finished (the first of them). */
STAGE_API stage_status stage_tabu_batch(stage_ctx *ctx, int32_t n, const stage_inst *insts,
                              const stage_tabu_params *params, stage_tabu_result *results,
                              stage_move *const *trajs);

/* Local search (Alg. 2, read for identical vehicles): a first-improvement
 * scan of the swap neighbourhood in a randomised order.
 *   - the moves are the swaps (close the base in slot s, open the closed
 *     available base at candidate position c); the candidate positions 0 ..
 *     nC-1 start as the closed available bases in ascending id order, nC =
 *     (available bases) - K, and a swap puts the closed base at the opened
 *     base's position;
 *   - pass p scans the K x nC pairs in the order of its two permutations
 *     (Alg. 2 draws them at random; here the caller supplies them): outer
 *     loop over slots perm_slots[p*K + a], inner loop over positions
 *     perm_cands[p*nC + b];
 *   - each pair is judged against the current placement; the first strictly
 *     better one (more covered, then less distance) is applied at once and the
 *     scan goes on with the next pair;
 *   - a pass that applied a move is followed by the next pair of
 *     permutations; a pass without one ends the search at a local optimum of
 *     the whole swap neighbourhood; the search also ends when the passes or
 *     max_moves run out.
 * The GPU evaluates the whole neighbourhood for the current placement in one
 * streaming pass and picks the first improving pair at or after the scan
 * position, which is the pair the sequential scan would apply next. */
typedef struct {
    int32_t K;                   /* vehicles, 1 <= K <= min(B, STAGE_MAX_K) */
    int32_t R;                   /* range in metres, 0 <= R < INT32_MAX */
    int32_t n_passes;            /* permutation pairs supplied, >= 1 */
    int32_t max_moves;           /* move budget (trajectory capacity), >= 0 */
    const int32_t *perm_slots;   /* [n_passes * K]: each row a permutation of 0 .. K-1 */
    const int32_t *perm_cands;   /* [n_passes * nC]: each row a permutation of 0 .. nC-1 */
    const int32_t *start_open;   /* [K] start placement, or NULL: stage_rank_bases */
} stage_ls_params;

typedef struct {
    int32_t n_moves;             /* moves applied */
    int32_t passes;              /* passes started */
    int32_t local_optimum;       /* 1: the last pass found no improving swap */
    int32_t reserved0;
    int64_t final_cov;
    int64_t final_dist;
    int32_t *final_open;         /* [K] caller buffer or NULL; filled sorted ascending */
} stage_ls_result;

/* Run the local search on a resident instance.  traj (nullable) receives one
 * stage_move per applied move ([max_moves]; iter = move number, flags =
 * STAGE_MOVE_NEW_BEST).  All arrays are host memory, copied in.
 * Errors: STAGE_ERR_INVALID_ARG (bad K, a row that is not a permutation,
 * n_passes < 1, max_moves < 0), STAGE_ERR_OUT_OF_RANGE (R), STAGE_ERR_INTERNAL
 * (a device self-check failed). */
STAGE_API stage_status stage_local_search(stage_ctx *ctx, stage_inst inst, const stage_ls_params *params,
                                          stage_ls_result *result, stage_move *traj);

/* Tabu search with a heterogeneous fleet (the vehicle and base types of
 * Sec. 3 and Eq. 6-10, read for this model):
 *   - K_rotary rotary-wing vehicles may stand at any base; K_fixed fixed-wing
 *     vehicles only at aerodromes (base_helipad[b] = 0); one vehicle per base;
 *   - a mission with mission_rotary[m] = 1 may be flown by rotary-wing
 *     vehicles only, any other mission by either type; each mission is flown
 *     from its nearest compatible open base, and the objective is Eq. 2's with
 *     coverage (most covered, then least distance);
 *   - start: start_rotary / start_fixed, or the ranking of Alg. 1 with the
 *     helipad rule of its lines 14-16: bases by (row sum, id), a helipad taken
 *     only while fewer than K_rotary are taken, until K_rotary + K_fixed; the
 *     helipads and then the best-ranked aerodromes get the rotary-wing
 *     vehicles, the other aerodromes the fixed-wing ones;
 *   - a move takes one vehicle from its base i to a closed available base j
 *     (an aerodrome for a fixed-wing vehicle); the tabu, aspiration, fallback,
 *     tie-break and improving-only rules are stage_tabu_run's.
 * traj (nullable) receives one stage_move per applied move ([iters]).  Arrays
 * are host memory, copied in; mission ids are the caller's (load order, then
 * appended missions).
 * Errors: STAGE_ERR_INVALID_ARG (counts, a fixed-wing start at a helipad, a
 * start base repeated or unavailable, missing arrays), STAGE_ERR_OUT_OF_RANGE
 * (R), STAGE_ERR_INTERNAL (a device self-check failed). */
typedef struct {
    int32_t K_rotary;                 /* >= 0 */
    int32_t K_fixed;                  /* >= 0; 1 <= K_rotary + K_fixed <= min(B, STAGE_MAX_K) */
    int32_t R;                        /* range in metres, 0 <= R < INT32_MAX */
    int32_t iters;                    /* >= 0 */
    int32_t tenure;                   /* >= 0 */
    int32_t accept_worsening;         /* as stage_tabu_params */
    const uint8_t *base_helipad;      /* [B]: 1 helipad, 0 aerodrome */
    const uint8_t *mission_rotary;    /* [M]: 1 rotary-wing only */
    const int32_t *start_rotary;      /* [K_rotary] or NULL (with start_fixed NULL: the ranking) */
    const int32_t *start_fixed;       /* [K_fixed] or NULL */
} stage_fleet_params;

typedef struct {
    int32_t n_moves;
    int32_t best_iter;
    int64_t best_cov;
    int64_t best_dist;
    int64_t final_cov;
    int64_t final_dist;
    int32_t *best_rotary;             /* [K_rotary] caller buffer or NULL; sorted ascending */
    int32_t *best_fixed;              /* [K_fixed] */
    int32_t *final_rotary;            /* [K_rotary] */
    int32_t *final_fixed;             /* [K_fixed] */
} stage_fleet_result;

STAGE_API stage_status stage_fleet_tabu(stage_ctx *ctx, stage_inst inst, const stage_fleet_params *params,
                                        stage_fleet_result *result, stage_move *traj);

/* ---------------------------------------------------------- updates, batches */

/* Incremental change to a resident instance (re-staging after new demand,
 * cancelled missions or closed bases).  All arrays are host memory.
 *   add:      n_add missions appended; they receive the next mission ids
 *             (M, M+1, ... in the order given)
 *   remove:   n_remove mission ids withdrawn; their table columns become
 *             INT32_MAX, so they are never covered and add nothing to any sum
 *             or to the ranking; removing an id twice is a no-op
 *   unavail:  bases that may no longer be opened
 *   avail:    bases that may be opened again */
typedef struct {
    int32_t n_add;
    int32_t n_remove;
    int32_t n_unavail;
    int32_t n_avail;
    const int32_t *add_pick_xy;   /* [2*n_add] */
    const int32_t *add_drop_xy;   /* [2*n_add] */
    const int32_t *remove_ids;    /* [n_remove] */
    const int32_t *unavail_ids;   /* [n_unavail] */
    const int32_t *avail_ids;     /* [n_avail] */
} stage_update;

/* Apply an update to a resident instance (synchronous).  The table grows in
 * place (with slack) when missions are added.
 * Errors: STAGE_ERR_NOT_FOUND, STAGE_ERR_INVALID_ARG (id out of range),
 * STAGE_ERR_OUT_OF_RANGE (coordinates, or more than STAGE_MAX_MISSIONS ids),
 * STAGE_ERR_ADMISSION (the instance is in use by a batch request). */
STAGE_API stage_status stage_update_instance(stage_ctx *ctx, stage_inst inst, const stage_update *update);

/* One request of the batch engine: a Tabu search (Alg. 3, as stage_tabu_run)
 * on a resident instance, or on an instance given by value that is loaded for
 * this request only.  An optional update is applied to the resident instance
 * first.  Requests on the same instance run one after the other, in
 * submission order. */
typedef struct {
    stage_inst inst;                  /* resident instance, or 0 to use desc */
    const stage_instance_desc *desc;  /* host descriptor, copied at submit (inst == 0) */
    const stage_update *update;       /* applied to inst before the search, or NULL (copied at submit) */
    stage_tabu_params params;         /* K <= 256; params.resume is not used (see resume_resident);
                                         start_open copied at submit */
    stage_move *traj;                 /* [params.iters] host buffer or NULL; written before completion */
    int32_t *best_open;               /* [K] host buffer or NULL; sorted ascending */
    int32_t *final_open;              /* [K] host buffer or NULL; sorted ascending */
    /* 1 (resident instances only): continue from the instance's resident
     * state -- the end state (placement, tabu expiries, iteration number, best
     * so far) of the last request on it that set this flag with the same K --
     * and keep this search's end state as the new one.  With no resident state
     * the search starts as usual (start_open, else the ranking).  After an
     * update of the instance the best so far restarts from the resumed
     * placement (its objective changed), and every open base the update made
     * unavailable is first closed by a forced move (reading A15): it opens the
     * available closed base with the best swap objective (covered desc,
     * distance asc, base id asc), tabu ignored, the unavailable bases taken in
     * ascending id; a forced move takes no iteration, and both of its bases
     * are tabu for the next tenure iterations.  0: the resident state is
     * neither used nor changed. */
    int32_t resume_resident;
    int32_t reserved1;
} stage_request;

typedef struct {
    stage_status status;
    int32_t n_moves;
    int32_t best_iter;
    int32_t n_forced;      /* forced moves before the search (resume_resident after an update) */
    int64_t best_cov;
    int64_t best_dist;
    int64_t final_cov;
    int64_t final_dist;
    int64_t t_submit_ns;   /* steady clock: submission, admission to a slot, completion */
    int64_t t_start_ns;
    int64_t t_end_ns;
} stage_result;

/* Queue n requests; tickets[k] identifies request k.  Returns at once: a
 * worker thread admits requests into slots (at most cfg->max_slots at a time,
 * and only while the context's HBM budget allows) and advances all active
 * searches together, one grouped launch per kernel per step, replayed from a
 * CUDA graph; finished searches leave and waiting ones join between replays.
 * Each search computes exactly what stage_tabu_run computes alone.  The caller
 * keeps traj / best_open / final_open valid until stage_poll reports the
 * ticket done.  Errors: STAGE_ERR_INVALID_ARG (malformed request). */
STAGE_API stage_status stage_batch_submit(stage_ctx *ctx, const stage_request *reqs, int32_t n,
                                          uint64_t *tickets);

/* Wait up to timeout_us microseconds (0: do not wait, < 0: no limit) for a
 * ticket.  Returns STAGE_PENDING while it runs; otherwise fills *out, forgets
 * the ticket and returns its status (STAGE_OK, or the request's error, e.g.
 * STAGE_ERR_ADMISSION when it can never fit the HBM budget).
 * STAGE_ERR_NOT_FOUND for an unknown or already collected ticket. */
STAGE_API stage_status stage_poll(stage_ctx *ctx, uint64_t ticket, stage_result *out, int32_t timeout_us);

/* ----------------------------------------------------------------- autotuner */

/* Tile autotuner of the swap pass.  Times every candidate number of missions
 * per block (1024 ... 16384) on this instance with placement open[K] (NULL:
 * the ranking) and range R, and records the fastest for the instance's shape
 * bucket (ceil log2 of padded missions, of candidate rows, of K); every later
 * search of that bucket on this process uses it.  *out_missions_per_block
 * (nullable) receives the choice.  The choice changes no result. */
STAGE_API stage_status stage_autotune(stage_ctx *ctx, stage_inst inst, const int32_t *open, int32_t K, int32_t R,
                                      int32_t *out_missions_per_block);

/* ---------------------------------------------------------------- profiling */

/* Kernel timing (contexts created with STAGE_PROFILE): launches and summed
 * device milliseconds of the named kernel ("swap_eval", "select", "refresh",
 * "table", "rowsum", "topk", "init", "evaluate") since the last reset. */
STAGE_API stage_status stage_kernel_stats(stage_ctx *ctx, const char *kernel, int64_t *launches,
                                double *total_ms);
STAGE_API stage_status stage_reset_stats(stage_ctx *ctx);

/* ------------------------------------------------------------ test support */

/* Copy rows [b0, b0+nb) x missions [m0, m0+nm) of the cost table into out
 * (row-major nb x nm). */
STAGE_API stage_status stage_read_table(stage_ctx *ctx, stage_inst inst, int32_t b0, int32_t nb,
                              int32_t m0, int32_t nm, int32_t *out);

/* Best and second-best open base of every mission for placement open[K],
 * ordered by (cost, base id): a, b (INT32_MAX when K = 1), b1, b2 (-1 when
 * K = 1) -- the per-mission ranking of the chosen bases in Alg. 1.  With
 * tabu_steps > 0, first runs that many Tabu iterations (params as in
 * stage_tabu_run, start open) and returns the arrays as the GPU's incremental
 * refresh left them. */
STAGE_API stage_status stage_best_two(stage_ctx *ctx, stage_inst inst, const int32_t *open, int32_t K,
                            int32_t R, int32_t tabu_steps, int32_t tenure, int32_t *a,
                            int32_t *b, int32_t *b1, int32_t *b2);

/* One bounded device-side wait on a flag that nothing sets, polled at most
 * the context's spin_limit times (the same wait the persistent search's grid
 * barriers use).  Returns STAGE_ERR_TIMEOUT when the wait gave up -- the
 * expected outcome -- with no trap and no hang; the context stays usable. */
STAGE_API stage_status stage_test_wait_timeout(stage_ctx *ctx);

/* The placement stage_tabu_batch uses (host logic only; no device, no context):
 * n searches, search k estimated at us[k] microseconds on gang[k] CTAs (1 <=
 * gang[k] <= P), placed largest first (by gang x time) on the gang[k] CTAs
 * that are free first, from the latest of their finish times.  out_off [P+1]
 * receives each CTA's first entry in out_entries [2 * sum(gang)], entries
 * (search k, its rank among the search's CTAs) in the order the CTA runs them
 * -- one global order of the searches for every CTA.  *out_makespan_us
 * receives the latest estimated finish.  Errors: STAGE_ERR_INVALID_ARG (NULL
 * arrays, n < 0, P < 1, a gang outside [1, P]). */
STAGE_API stage_status stage_test_batch_schedule(int32_t n, const double *us, const int32_t *gang, int32_t P,
                                       int32_t *out_off, int32_t *out_entries, double *out_makespan_us);

/* ------------------------------------------------------- allocation-free call */

/* Every GPU that loads this library keeps a STAGE_NOALLOC_SCRATCH_MB MiB device
 * array for stage_evaluate_swaps_noalloc until the process exits. */
#define STAGE_NOALLOC_SCRATCH_MB 8
#define STAGE_NOALLOC_MAX_BASES  8192

/* stage_evaluate_swaps for callers that cannot allocate device memory.  The
 * paper has no counterpart: this is a deployment variant of the swap
 * neighbourhood evaluation, not a step of the method.
 *
 * Who needs it: a re-staging service embedded in a host application that owns
 * all device memory through its own fixed pool, and dispatch loops that must
 * not block on cudaMalloc (it can synchronise the device) or meet an
 * out-of-memory failure halfway through a request.  The call makes no
 * cudaMalloc, cudaFree, cudaMallocHost or other allocating call; the caller
 * passes every input and output as DEVICE memory, and the scratch of the
 * computation (per-mission best / second-best arrays, objective accumulators,
 * candidate list) lives in a file-scope device array of fixed size.
 *
 *   cost             B x M_pad int32, row-major, one row per base (the layout
 *                    stage_load_instance builds): columns M .. M_pad-1 must hold
 *                    INT32_MAX, M_pad a multiple of 4, base 16-byte aligned
 *   base_available   [B] uint8, or NULL for all available
 *   open             [K] distinct available base ids in [0, B).  They are
 *                    device memory, so the host cannot check them; the first
 *                    kernel does: with an id outside [0, B), a repeated id or
 *                    an unavailable base, no objective is computed and every
 *                    output entry stays -1 (the call still returns STAGE_OK,
 *                    since it only enqueues the work)
 *   R                range in metres, 0 <= R < INT32_MAX
 *   out_cov/out_dist [K*B] int64: entry k*B + j = F(O - open[k] + j) for a
 *                    closed available j, else -1, exactly as stage_evaluate_swaps
 *   stream           cudaStream_t to enqueue on (NULL = the legacy default stream)
 *   errbuf, errlen   optional host buffer that receives an error message
 *
 * Limits: B <= STAGE_NOALLOC_MAX_BASES, K <= STAGE_MAX_K, and the scratch,
 * about 12 bytes per padded mission plus 12 bytes per (K, B) pair, must fit in
 * STAGE_NOALLOC_SCRATCH_MB MiB (e.g. M_pad up to about 560,000 with K = 64,
 * B = 2000).  Larger sizes return STAGE_ERR_OUT_OF_RANGE before any work runs.
 * Other errors: STAGE_ERR_INVALID_ARG, STAGE_ERR_CUDA.
 *
 * The call only enqueues work on `stream`; the results are ready when the
 * stream reaches that point.  All calls share the one scratch array, which
 * keeps the last call's contents (each call clears what must start at zero):
 * calls whose work overlaps on the GPU -- on different streams or from
 * different threads -- race on it and corrupt each other's results, so
 * serialise them.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture begins. */
STAGE_API stage_status stage_evaluate_swaps_noalloc(const int32_t *cost, int32_t B, int32_t M,
                                                    int32_t M_pad, const uint8_t *base_available,
                                                    const int32_t *open, int32_t K, int32_t R,
                                                    int64_t *out_cov, int64_t *out_dist,
                                                    void *stream, char *errbuf, size_t errlen);

#ifdef __cplusplus
}
#endif

#endif /* STAGE_H */
