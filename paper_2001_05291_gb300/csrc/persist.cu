// Persistent Tabu search over the incremental neighbourhood (Alg. 3's outer
// loop on the device): one cooperative launch runs every iteration of a
// search, its CTAs resident on their SMs and meeting at three grid-wide
// barriers per iteration.
//
// Missions are owned in blocks of kBlockMissions consecutive columns (the
// table's columns are in a spatial order), block q by CTA q mod G: a move's
// work -- the missions it touches lie near the bases it exchanges -- spreads
// over every CTA, and each CTA's share stays spatially coherent.
//
// One iteration, for the move u:
//   barrier A   every CTA has published its best admissible and best overall
//               key over its share of the swaps; each CTA reduces the same
//               keys to the same move and applies it to its copy of the
//               placement, candidate list and tabu expiries (a5, a6);
//   refresh     each CTA updates the best / second-best state of its missions
//               (a7), records those whose terms changed, adds their changes of
//               V0 and loss (kept across moves like gain and extra) and every
//               mission's terms of the closed base's column to a few global
//               sums, and appends its records to the move's list (one atomic
//               per CTA: each CTA's records stay together, in spatial order);
//   barrier B   the list is complete;
//   update      each CTA takes an equal contiguous share of the list (the
//               records lie near the move, so a CTA's own would leave most
//               CTAs idle) and moves each one's old terms out of, and its new
//               terms into, every other base's column (a4).  The copy's bases
//               are in spatial order, so a record's terms fall in few cells of
//               32 positions; the exact minimum of each cell of each row
//               (built with the copy) shows which cells of a record have any
//               term, and only those pieces of its row (128 bytes) are read.
//               The (cell, records) work is cut into items dealt to the warps
//               in turn (the cells near the move carry most of it); the
//               records are ordered by slot, so gain terms add up in
//               registers and extra terms in runs of one slot, flushed to the
//               global columns with atomics;
//   barrier C   the columns are complete; each CTA scores its share of the
//               swaps F(s, j) = V0 + gain[j] + loss[s] + extra[s][j] -- the
//               closed base's column taken from the refresh's sums, which CTA
//               0 also writes back -- for the next move.
//
// The terms are integers, so the columns equal what a full pass over the
// table would give for each new placement (the fast-interchange
// decomposition of Whitaker 1983 / Resende and Werneck 2007, kept across
// moves), and every move is the one the oracle chooses.
//
// Sums that one step fills and a later one reads are double-buffered by move
// parity (V0 / loss, the closed column, the list's length), each reset by CTA
// 0 in a phase where no CTA reads or writes it (V0 / loss to the previous
// move's values, the others to zero).  The grid barriers give up after the
// context's spin limit: the CTA sets an error word and leaves the loop, the
// others give up at their next barrier, and the host reports STAGE_ERR_TIMEOUT.
#include <cuda_runtime.h>

#include <climits>
#include <stdint.h>

#include "stage_internal.h"
#include "device_common.cuh"

namespace stg {

// CTA shapes (NT threads per CTA, REC records staged per round of the
// update): 1024 threads and 256 records, one CTA per SM, for a single search
// and for a batch.  (A batch of 256-thread CTAs, four per SM staging 128
// records, took as much SM time for the batched workload's update, on 608
// CTAs less evenly loaded: 612 ms against 517 ms per batch.)
constexpr int kPerThreads = 1024;
constexpr int kBatchThreads = 1024;
constexpr int kBatchRec = 256;
constexpr int kBlockMissions = 32;     // missions per ownership block (one warp chunk)
constexpr int kRecCap = 256;           // records staged in shared memory per round of a single search's update
constexpr int kUpdBatch = 8;           // listed records whose costs a warp loads at once
constexpr int kUpdItem = 16;           // listed records of one cell per work item of a warp
constexpr int kMaxLd = 2048;           // longest table-copy row (its 64 cells fit the item scan)
constexpr size_t kPerSmemLimit = 220 * 1024;
constexpr int kMaxGrid = 256;          // CTAs of a search (the update's count prefix and sums: 8 per lane)
static_assert(kMaxGrid + 1 <= kRefQ, "the count prefix fits in the refresh's queue");

// Per-CTA clocks (ns, summed over the search): choosing and applying the move,
// the refresh, the wait at the barrier after it, the update, the wait at the
// barrier after it, the selection, the wait at the barrier before the next
// move; the first seven cover the whole time, the others split the refresh
// and the update.
enum : int {
    kClkMove = 0, kClkRefresh, kClkWaitB, kClkUpdate, kClkWaitC, kClkSelect, kClkWaitA,
    // parts of the refresh and the update (thread 0's view): the update's
    // record staging, its wait for the CTA's slowest warp, and warp 0's walk
    // over the records
    kClkRefLoop, kClkRefRescan, kClkRefSums, kClkUpdIssue, kClkUpdWait, kClkUpdCompute, kClocks
};
static_assert(kClocks == kPersistClocks, "clock layout shared with the host");

__device__ __forceinline__ long long gtimer()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Records (two int4 per mission whose terms changed), clamped at R + 1 as the
// terms use them: (column, hi = max(old b, new b), old a, old b),
// (old slot, new a, new b, new slot).  No term of a base with cost >= hi changes.

// Shared-memory layout (byte offsets).
struct PerLayout {
    size_t recs, raw, cnt, cells, wlist, cand, expiry, cidx, open, lc, ic, ld, id, q, total;
};

__host__ __device__ inline size_t per_align(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline PerLayout per_layout(int K, int B, int ldT, int rec)
{
    PerLayout L{};
    size_t o = 0;
    L.recs = o;   o = per_align(o + (size_t)rec * 32, 16);
    L.raw = o;    o = per_align(o + (size_t)rec * 32, 16);
    L.cnt = o;    o = per_align(o + (size_t)kPipeMaxK * 4, 16);
    L.cells = o;  o = per_align(o + (size_t)rec * (ldT / 32) * 4, 16);
    L.wlist = o;  o = per_align(o + (size_t)(ldT / 32) * rec * 2, 16);
    L.cand = o;   o = per_align(o + (size_t)B * 4, 16);
    L.expiry = o; o = per_align(o + (size_t)B * 4, 16);
    L.cidx = o;   o = per_align(o + (size_t)B * 4, 16);
    L.open = o;   o = per_align(o + (size_t)K * 4, 16);
    L.lc = o;     o = per_align(o + (size_t)K * 4, 16);
    L.ic = o;     o = per_align(o + (size_t)K * 4, 16);
    L.ld = o;     o = per_align(o + (size_t)K * 8, 16);
    L.id = o;     o = per_align(o + (size_t)K * 8, 16);
    L.q = o;      o = per_align(o + (size_t)kRefQ * 4, 16);
    L.total = o;
    return L;
}

// ---------------------------------------------------------------- primitives

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Poll *flag until it differs from `seen`; false after `limit` polls.
__device__ __forceinline__ bool wait_change(const unsigned *flag, unsigned seen, long long limit)
{
    for (long long k = 0; k < limit; k++) {
        if (ld_acquire_u32(flag) != seen) return true;
        if (k > 64) __nanosleep(64);
    }
    return false;
}

// Barrier of the G CTAs that run one search (the launch is cooperative, so
// every CTA is resident).  Arrivals count up without reset: barrier number g
// (from 0) is passed once the count reaches G * (g + 1).  Thread 0 of each CTA adds its
// arrival with release semantics (the CTA's writes, ordered before it by the
// CTA barrier, become visible first), a reduction that returns nothing, and
// polls the count with acquire loads (the first poll sees its own arrival:
// same thread, same address), at most `limit` times, then sets the timeout
// bit in *err and gives up.
// Returns false when this CTA gave up or another CTA has reported an error:
// the caller then leaves the loop.  (The count wraps after 2^32 arrivals:
// 9 million iterations of three barriers on 152 CTAs.)
__device__ __forceinline__ bool grid_sync(unsigned *bar, unsigned &gen, int G, long long limit, int *err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 0;
        const unsigned target = (unsigned)G * (gen + 1u);
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" : : "l"(bar) : "memory");
        for (long long k = 0; k < limit; k++) {
            if ((int)(ld_acquire_u32(bar) - target) >= 0) {
                ok = 1;
                break;
            }
            if (k > 256) __nanosleep(32);
        }
        if (!ok) atomicOr(err, kErrPipelineTimeout);
        if (ok && *reinterpret_cast<volatile int *>(err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    gen += 1u;
    return s_ok != 0;
}

// A read-only cost of the table copy (unchanged during the search), not
// kept in L1 and first to leave L2: each row is read once per move.
__device__ __forceinline__ int ld_stream(const int32_t *p, unsigned long long policy)
{
    int v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(policy));
    return v;
}

// Add (c, d) into the shared per-slot sums of the lanes with `has`: lanes
// with the same slot are summed first, one atomic per slot per warp.  Every
// lane of the warp calls it; |d| < 2^31 (as group_sum_small needs).
__device__ __forceinline__ void slot_add_warp(bool has, int slot, int c, long long d, int *s_c,
                                              unsigned long long *s_d)
{
    const unsigned full = 0xffffffffu;
    if (!__ballot_sync(full, has)) return;
    const unsigned peers = __match_any_sync(full, has ? slot : -1);
    const int sc = (int)__reduce_add_sync(peers, has ? (unsigned)c : 0u);
    const long long sd = group_sum_small(peers, has ? d : 0ll);
    if (has && (int)(threadIdx.x & 31) == __ffs(peers) - 1 && (sc | (sd != 0))) {
        atomicAdd(&s_c[slot], sc);
        atomicAdd(&s_d[slot], (unsigned long long)sd);
    }
}

// ---------------------------------------------------------------- kernel

struct PersistArgs {
    TabuBuffers w;                  // search buffers; costT, border, ldT set
    const int32_t *cost;            // the table, row-major
    unsigned long long *acc;        // [2][2 + 2K]: V0 (covered, distance), loss_c[K], loss_d[K]
    unsigned long long *col;        // [2][2 + 2K]: closed column: gain (c, d), extra_c[K], extra_d[K]
    // per-CTA arrays are indexed by the CTA's rank g in the G CTAs of the search
    MoveKey *part;                  // [2 * G] best admissible, best overall per CTA
    unsigned *bar;                  // arrivals at the grid barriers
    int *err;                       // error word (kErr*)
    long long *info;                // [2] CTAs, records over the search
    int *nrec;                      // [G] records in each CTA's region for the move
    long long *psum;                // [2 * (2 + 2K)][G] each CTA's parts of the move's sums
    long long *cta_ns;              // [G][kClocks] per-CTA time of each step, ns
    int4 *region;                   // [G * region_cap * 2] each CTA's records of a move
    long long spin_limit;
    int region_cap;                 // records per CTA region
    int G;                          // CTAs of the search
    const int *rank_slot;           // local search: [passes][K] each slot's place in a pass's scan order
    const int *rank_cand;           // local search: [passes][nC] each candidate position's place
};

// Search scalars, the same in every CTA (each applies the same moves).
struct PerState {
    long long cur_c, cur_d, best_c, best_d, v0c, v0d;
    int t, n_moves, best_iter, done, mv_s, mv_i, mv_j, recn, qn, prev_i;
    int ls_pass, ls_pos, ls_moved, ls_optimum, ls_passes;   // local search (Alg. 2)
};

// The local search's pick (Alg. 2 as read: the first strictly improving swap
// of a scan order): the swap's objective, its place u in the order.
struct LsPick {
    long long cov, dist;
    int u, i, j, s, c, valid;
};
static_assert(sizeof(LsPick) <= sizeof(MoveKey), "picks use the per-CTA key slots");

__device__ __forceinline__ LsPick no_pick()
{
    LsPick k;
    k.cov = 0; k.dist = 0; k.u = INT_MAX; k.i = 0; k.j = 0; k.s = 0; k.c = 0; k.valid = 0;
    return k;
}

// The warp's pick with the smallest place (places are distinct), in every lane.
__device__ __forceinline__ void warp_first_pick(LsPick &k)
{
    const unsigned full = 0xffffffffu;
    const unsigned v = k.valid ? (unsigned)k.u : 0xffffffffu;
    const unsigned m = __reduce_min_sync(full, v);
    if (m == 0xffffffffu) {   // the same on the warp
        k = no_pick();
        return;
    }
    const int src = __ffs(__ballot_sync(full, v == m)) - 1;
    LsPick o;
    o.cov = __shfl_sync(full, k.cov, src);
    o.dist = __shfl_sync(full, k.dist, src);
    o.u = (int)m;
    o.i = __shfl_sync(full, k.i, src);
    o.j = __shfl_sync(full, k.j, src);
    o.s = __shfl_sync(full, k.s, src);
    o.c = __shfl_sync(full, k.c, src);
    o.valid = 1;
    k = o;
}

// The CTA's first picks a and b: in warp 0 (to_all false) or in every thread.
template <int NT>
__device__ __forceinline__ void block_first_picks(LsPick &a, LsPick &b, LsPick *sa, LsPick *sb, bool to_all)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    warp_first_pick(a);
    warp_first_pick(b);
    if (lane == 0) {
        sa[wid] = a;
        sb[wid] = b;
    }
    __syncthreads();
    if (wid == 0) {
        a = lane < NT / 32 ? sa[lane] : no_pick();
        b = lane < NT / 32 ? sb[lane] : no_pick();
        warp_first_pick(a);
        warp_first_pick(b);
        if (to_all && lane == 0) {
            sa[0] = a;
            sb[0] = b;
        }
    }
    if (to_all) {
        __syncthreads();
        a = sa[0];
        b = sb[0];
        __syncthreads();
    }
}

__device__ __forceinline__ LsPick load_pick_cg(const LsPick *p)
{
    LsPick k;
    k.cov = __ldcg(&p->cov);
    k.dist = __ldcg(&p->dist);
    k.u = __ldcg(&p->u);
    k.i = __ldcg(&p->i);
    k.j = __ldcg(&p->j);
    k.s = __ldcg(&p->s);
    k.c = __ldcg(&p->c);
    k.valid = __ldcg(&p->valid);
    return k;
}

// The best admissible and best overall key over this CTA's share of the
// K x nC swaps, for the placement of iteration st.t, whose V0 and loss are
// `acc` (V0 returned in v0c, v0d).  The base closed by the previous move
// (st.prev_i, -1 at the start) takes its column from the move's sums `cl`.
// Every load of a swap's terms (V0, loss, gain, extra) is issued together.
template <int NT>
__device__ __forceinline__ void persist_select(const TabuBuffers &w, const PerState &st, int nC, const int *s_open,
                                               const int *s_cand, const int *s_exp, const unsigned long long *acc,
                                               const unsigned long long *cl, MoveKey &adm, MoveKey &all,
                                               long long &v0c, long long &v0d, int gr, int G)
{
    const int K = w.K, t = st.t;
    v0c = (long long)__ldcg(&acc[0]);
    v0d = (long long)__ldcg(&acc[1]);
    const int total = K * nC;   // K <= 256, nC <= 2048
    const int q0 = (int)((long long)total * gr / G);
    const int q1 = (int)((long long)total * (gr + 1) / G);
    for (int q = q0 + (int)threadIdx.x; q < q1; q += NT) {
        const int s = q / nC, c = q - s * nC;
        const int i = s_open[s], j = s_cand[c];
        long long gc, gd, ec, ed;
        if (j == st.prev_i) {
            gc = (long long)__ldcg(&cl[0]);
            gd = (long long)__ldcg(&cl[1]);
            ec = (long long)__ldcg(&cl[2 + s]);
            ed = (long long)__ldcg(&cl[2 + K + s]);
        } else {
            const size_t sj = (size_t)s * w.B + j;
            gc = __ldcg(&w.gain_c[j]);
            gd = (long long)__ldcg(&w.gain_d[j]);
            ec = __ldcg(&w.extra_c[sj]);
            ed = (long long)__ldcg(&w.extra_d[sj]);
        }
        const long long lc = (long long)__ldcg(&acc[2 + s]), ld = (long long)__ldcg(&acc[2 + K + s]);
        MoveKey k;
        k.cov = v0c + gc + lc + ec;
        k.dist = v0d + gd + ld + ed;
        k.i = i; k.j = j; k.s = s; k.c = c; k.valid = 1;
        k.tabu = (t < s_exp[i]) || (t < s_exp[j]);
        if (key_better(k, all)) all = k;
        if ((!k.tabu || obj_better(k.cov, k.dist, st.best_c, st.best_d)) && key_better(k, adm)) adm = k;
    }
}

// The local search's picks over this CTA's share of the K x nC swaps, for
// the placement of move st.t (V0 and loss in `acc`, returned in v0c, v0d):
// the first strictly improving swap at or after place st.ls_pos of pass
// st.ls_pass's scan order (p1), and the first of the next pass's order (p2,
// taken when the current pass has none left after a move).  A swap's place
// is rank_slot[s] * nC + rank_cand[c] for its slot s and candidate position c.
template <int NT>
__device__ __forceinline__ void persist_local_select(const TabuBuffers &w, const PerState &st, int nC,
                                                     const int *s_open, const int *s_cand, const int *rank_slot,
                                                     const int *rank_cand, const unsigned long long *acc,
                                                     const unsigned long long *cl, LsPick &p1, LsPick &p2,
                                                     long long &v0c, long long &v0d, int gr, int G)
{
    const int K = w.K;
    v0c = (long long)__ldcg(&acc[0]);
    v0d = (long long)__ldcg(&acc[1]);
    const int pass = st.ls_pass, pos0 = st.ls_pos;
    const bool next = pass + 1 < st.ls_passes;
    const int *ra = rank_slot + (size_t)pass * K, *rb = rank_cand + (size_t)pass * nC;
    const int *ra2 = next ? ra + K : ra, *rb2 = next ? rb + nC : rb;
    const int total = K * nC;
    const int q0 = (int)((long long)total * gr / G);
    const int q1 = (int)((long long)total * (gr + 1) / G);
    for (int q = q0 + (int)threadIdx.x; q < q1; q += NT) {
        const int s = q / nC, c = q - s * nC;
        const int i = s_open[s], j = s_cand[c];
        long long gc, gd, ec, ed;
        if (j == st.prev_i) {
            gc = (long long)__ldcg(&cl[0]);
            gd = (long long)__ldcg(&cl[1]);
            ec = (long long)__ldcg(&cl[2 + s]);
            ed = (long long)__ldcg(&cl[2 + K + s]);
        } else {
            const size_t sj = (size_t)s * w.B + j;
            gc = __ldcg(&w.gain_c[j]);
            gd = (long long)__ldcg(&w.gain_d[j]);
            ec = __ldcg(&w.extra_c[sj]);
            ed = (long long)__ldcg(&w.extra_d[sj]);
        }
        const int u1 = __ldg(&ra[s]) * nC + __ldg(&rb[c]);
        const int u2 = __ldg(&ra2[s]) * nC + __ldg(&rb2[c]);
        const long long lc = (long long)__ldcg(&acc[2 + s]), ld = (long long)__ldcg(&acc[2 + K + s]);
        const long long cov = v0c + gc + lc + ec, dist = v0d + gd + ld + ed;
        if (!obj_better(cov, dist, st.cur_c, st.cur_d)) continue;
        if (u1 >= pos0 && u1 < p1.u) {
            p1.cov = cov; p1.dist = dist; p1.u = u1; p1.i = i; p1.j = j; p1.s = s; p1.c = c; p1.valid = 1;
        }
        if (next && u2 < p2.u) {
            p2.cov = cov; p2.dist = dist; p2.u = u2; p2.i = i; p2.j = j; p2.s = s; p2.c = c; p2.valid = 1;
        }
    }
}

// Best admissible and best overall key of the CTA, valid in warp 0 only
// (block_best2 without handing the result to every thread).
template <int NT>
__device__ __forceinline__ void block_best2_warp0(MoveKey &adm, MoveKey &all, MoveKey *s_adm, MoveKey *s_all)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    warp_best_key(adm);
    warp_best_key(all);
    if (lane == 0) {
        s_adm[wid] = adm;
        s_all[wid] = all;
    }
    __syncthreads();
    if (wid == 0) {
        adm = lane < NT / 32 ? s_adm[lane] : invalid_key();
        all = lane < NT / 32 ? s_all[lane] : invalid_key();
        warp_best_key(adm);
        warp_best_key(all);
    }
}

// One whole search, run by the G CTAs of ranks gr = 0 .. G-1 (all resident,
// each calling this with the same arguments); the lead CTA (rank 0) hands the
// state back.  LOCAL: Alg. 2's local search (first improvement over the scan
// orders of A.rank_slot / A.rank_cand) instead of the Tabu search; the
// refresh and the update are the same.  max_steps > 0: at most that many
// iterations this launch (the search goes on in a later launch from the state
// handed back); a search already done makes none.
template <int NT, int REC, bool LOCAL = false>
__device__ __forceinline__ void persist_search(const PersistArgs &A, const int gr, const int G, int max_steps = 0)
{
    constexpr int kPerWarps = NT / 32;
    static_assert(REC <= NT && REC % 32 == 0, "one staged record per thread");
    const TabuBuffers &w = A.w;
    extern __shared__ __align__(128) unsigned char smem[];
    const int K = w.K, B = w.B, R = w.R, ldT = w.ldT;
    const PerLayout L = per_layout(K, B, ldT, REC);
    int4 *s_recs = reinterpret_cast<int4 *>(smem + L.recs);
    int32_t *s_cells = reinterpret_cast<int32_t *>(smem + L.cells);
    int4 *s_raw = reinterpret_cast<int4 *>(smem + L.raw);
    int *s_cnt = reinterpret_cast<int *>(smem + L.cnt);
    uint16_t *s_clist = reinterpret_cast<uint16_t *>(smem + L.wlist);   // [cell][REC]
    __shared__ int s_ccnt[kMaxLd / 32], s_ipre[kMaxLd / 32 + 1];
    int *s_cand = reinterpret_cast<int *>(smem + L.cand);
    int *s_exp = reinterpret_cast<int *>(smem + L.expiry);
    int *s_cidx = reinterpret_cast<int *>(smem + L.cidx);
    int *s_open = reinterpret_cast<int *>(smem + L.open);
    int *s_lc = reinterpret_cast<int *>(smem + L.lc);
    int *s_ic = reinterpret_cast<int *>(smem + L.ic);
    unsigned long long *s_ld = reinterpret_cast<unsigned long long *>(smem + L.ld);
    unsigned long long *s_id = reinterpret_cast<unsigned long long *>(smem + L.id);
    int *s_q = reinterpret_cast<int *>(smem + L.q);
    __shared__ MoveKey s_adm[kPerWarps], s_all[kPerWarps];
    __shared__ PerState S;
    __shared__ long long s_clk[kClocks + 1];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool lead_cta = gr == 0;
    const int nA = 2 + 2 * K;
    TabuDevState *st = w.st;
    const int t_end0 = st->t_end, tenure = st->tenure, aw = st->accept_worsening, nC = st->nC;
    const int t_end = st->done ? st->t : max_steps > 0 ? min(t_end0, st->t + max_steps) : t_end0;
    const int traj_cap = st->traj_cap;
    int4 *region = A.region + (size_t)gr * A.region_cap * 2;
    long long rec_total = 0;   // records of this CTA over the search
    // the update's (record, base) pairs with a term, and the (record, warp
    // cell) passes with at least one: the update's work and how densely it
    // fills the warps
    __shared__ unsigned long long s_terms[4];
    if (tid < 4) s_terms[tid] = 0;

    if (tid == 0) {
        S.t = st->t;
        S.n_moves = st->n_moves;
        S.best_iter = st->best_iter;
        S.done = st->done;
        S.mv_s = st->mv_s; S.mv_i = st->mv_i; S.mv_j = st->mv_j;
        S.prev_i = -1;
        S.cur_c = st->cur_cov; S.cur_d = st->cur_dist;
        S.best_c = st->best_cov; S.best_d = st->best_dist;
        S.ls_pass = st->ls_pass; S.ls_pos = st->ls_pos; S.ls_moved = st->ls_moved;
        S.ls_optimum = st->ls_optimum; S.ls_passes = st->ls_passes;
        const unsigned long long *acc = A.acc + (size_t)(S.t & 1) * nA;
        S.v0c = (long long)acc[0];
        S.v0d = (long long)acc[1];
        for (int k = 0; k < kClocks; k++) s_clk[k] = 0;
        s_clk[kClocks] = gtimer();
    }
    for (int k = tid; k < K; k += NT) s_open[k] = w.open[k];
    for (int b = tid; b < B; b += NT) {
        s_exp[b] = w.expiry[b];
        s_cidx[b] = -1;
    }
    __syncthreads();
    for (int c = tid; c < nC; c += NT) {
        const int b = w.cand[c];
        s_cand[c] = b;
        s_cidx[b] = c;
    }
    __syncthreads();
    unsigned gen = 0;
    const unsigned long long evict_first = evict_first_policy();
    __shared__ long long s_sub;   // thread 0: the last mark inside a step
    auto lap = [&](int which) {
        if (tid == 0) {
            const long long now = gtimer();
            s_clk[which] += now - s_clk[kClocks];
            s_clk[kClocks] = now;
            s_sub = now;
        }
    };
    auto sub = [&](int which) {
        if (tid == 0) {
            const long long now = gtimer();
            s_clk[which] += now - s_sub;
            s_sub = now;
        }
    };
    // the scores of this CTA's share of the swaps for the move of iteration
    // S.t; CTA 0 also writes the previous move's closed column back
    auto select = [&]() {
        const int u = S.t;
        const unsigned long long *clp = A.col + (size_t)((u + 1) & 1) * nA;   // the previous move's sums
        const unsigned long long *acc = A.acc + (size_t)(u & 1) * nA;         // V0 and loss of this placement
        long long v0c, v0d;
        if constexpr (LOCAL) {
            LsPick p1 = no_pick(), p2 = no_pick();
            persist_local_select<NT>(w, S, nC, s_open, s_cand, A.rank_slot, A.rank_cand, acc, clp, p1, p2, v0c,
                                     v0d, gr, G);
            block_first_picks<NT>(p1, p2, reinterpret_cast<LsPick *>(s_adm), reinterpret_cast<LsPick *>(s_all),
                                  false);
            if (tid == 0) {
                reinterpret_cast<LsPick *>(A.part)[2 * gr] = p1;
                reinterpret_cast<LsPick *>(A.part)[2 * gr + 1] = p2;
            }
        } else {
            MoveKey adm = invalid_key(), all = invalid_key();
            persist_select<NT>(w, S, nC, s_open, s_cand, s_exp, acc, clp, adm, all, v0c, v0d, gr, G);
            block_best2_warp0<NT>(adm, all, s_adm, s_all);
            if (tid == 0) {
                A.part[2 * gr] = adm;
                A.part[2 * gr + 1] = all;
            }
        }
        if (tid == 0) {
            S.v0c = v0c;   // for the check of the chosen move's objective
            S.v0d = v0d;
        }
        if (lead_cta && S.prev_i >= 0) {
            // the closed column, now in the sums, into the global columns
            // (every CTA reads it from the sums until the next barrier)
            const int ip = S.prev_i;
            if (tid == 0) {
                w.gain_c[ip] = (int)(long long)__ldcg(&clp[0]);
                w.gain_d[ip] = __ldcg(&clp[1]);
            }
            for (int k = tid; k < K; k += NT) {
                w.extra_c[(size_t)k * B + ip] = (int)(long long)__ldcg(&clp[2 + k]);
                w.extra_d[(size_t)k * B + ip] = __ldcg(&clp[2 + K + k]);
            }
        }
        lap(kClkSelect);
    };

    select();   // the first move's keys

    while (S.t < t_end) {   // S.t is read after a CTA barrier on every path: the same on every thread
        if (!grid_sync(A.bar, gen, G, A.spin_limit, A.err)) break;
        lap(kClkWaitA);
        const int u = S.t;   // the move of this iteration
        // ------------------------------------------------ choose and apply the move (a5, a6)
        if constexpr (LOCAL) {
            // Alg. 2 (readings L3, L4): the first improving swap of the pass
            // at or after the scan position; none left after a move in this
            // pass: the next pass's first from its start; none: stop (a local
            // optimum unless the pass had moved and no pass is left)
            LsPick p1 = no_pick(), p2 = no_pick();
            for (int b = tid; b < G; b += NT) {
                const LsPick a1 = load_pick_cg(reinterpret_cast<const LsPick *>(A.part) + 2 * b);
                const LsPick a2 = load_pick_cg(reinterpret_cast<const LsPick *>(A.part) + 2 * b + 1);
                if (a1.valid && a1.u < p1.u) p1 = a1;
                if (a2.valid && a2.u < p2.u) p2 = a2;
            }
            block_first_picks<NT>(p1, p2, reinterpret_cast<LsPick *>(s_adm), reinterpret_cast<LsPick *>(s_all),
                                  true);
            if (S.cur_c != S.v0c || S.cur_d != S.v0d) {
                if (lead_cta && tid == 0) atomicOr(A.err, kErrObjectiveMismatch);
                if (tid == 0) S.done = 1;
                break;
            }
            const int lpass = S.ls_pass, lmoved = S.ls_moved, lpasses = S.ls_passes;
            const bool take2 = !p1.valid && lmoved && lpass + 1 < lpasses;
            const LsPick Pm = p1.valid ? p1 : p2;
            __syncthreads();   // every thread has read S before thread 0 changes it
            if (!p1.valid && !(take2 && p2.valid)) {
                if (tid == 0) {
                    if (take2) S.ls_pass = lpass + 1;   // the new pass has no improving swap
                    S.ls_optimum = (take2 || !lmoved) ? 1 : 0;
                    S.done = 1;
                }
                break;
            }
            if (tid == 0) {
                S.best_c = Pm.cov;   // every applied move is strictly better
                S.best_d = Pm.dist;
                S.best_iter = u;
                S.cur_c = Pm.cov;
                S.cur_d = Pm.dist;
                S.mv_s = Pm.s; S.mv_i = Pm.i; S.mv_j = Pm.j;
                s_open[Pm.s] = Pm.j;
                s_cand[Pm.c] = Pm.i;
                s_cidx[Pm.i] = Pm.c;
                s_cidx[Pm.j] = -1;
                if (lead_cta) {
                    if (S.n_moves < traj_cap) {
                        stage_move mv;
                        mv.iter = u; mv.i = Pm.i; mv.j = Pm.j; mv.flags = STAGE_MOVE_NEW_BEST;
                        mv.cov = Pm.cov; mv.dist = Pm.dist;
                        w.traj[S.n_moves] = mv;
                    }
                    for (int k = 0; k < K; k++) w.best_open[k] = s_open[k];
                }
                if (take2) S.ls_pass = lpass + 1;
                S.ls_pos = Pm.u + 1;
                S.ls_moved = 1;
                S.n_moves += 1;
                S.recn = 0;
                S.qn = 0;
            }
        } else {
        MoveKey adm = invalid_key(), all = invalid_key();
        for (int b = tid; b < G; b += NT) {
            const MoveKey pa = load_key_cg(&A.part[2 * b]), px = load_key_cg(&A.part[2 * b + 1]);
            if (key_better(pa, adm)) adm = pa;
            if (key_better(px, all)) all = px;
        }
        block_best2<NT>(adm, all, s_adm, s_all);
        if (!all.valid) {
            if (tid == 0) S.done = 1;   // no closed available base
            break;
        }
        if (S.cur_c != S.v0c || S.cur_d != S.v0d) {
            // the refresh's objective disagrees with the chosen move's
            if (lead_cta && tid == 0) atomicOr(A.err, kErrObjectiveMismatch);
            if (tid == 0) S.done = 1;
            break;
        }
        const MoveKey Pm = adm.valid ? adm : all;
        if (!aw && !obj_better(Pm.cov, Pm.dist, S.cur_c, S.cur_d)) {
            if (tid == 0) S.done = 1;   // improving-only rule: no improving move
            break;
        }
        __syncthreads();   // every thread has read S before thread 0 changes it
        if (tid == 0) {
            int flags = adm.valid ? (adm.tabu ? STAGE_MOVE_ASPIRATION : 0) : STAGE_MOVE_FALLBACK;
            if (obj_better(Pm.cov, Pm.dist, S.best_c, S.best_d)) {
                S.best_c = Pm.cov;
                S.best_d = Pm.dist;
                S.best_iter = u;
                flags |= STAGE_MOVE_NEW_BEST;
            }
            S.cur_c = Pm.cov;
            S.cur_d = Pm.dist;
            S.mv_s = Pm.s; S.mv_i = Pm.i; S.mv_j = Pm.j;
            s_open[Pm.s] = Pm.j;
            s_cand[Pm.c] = Pm.i;
            s_cidx[Pm.i] = Pm.c;
            s_cidx[Pm.j] = -1;
            s_exp[Pm.i] = u + tenure + 1;
            s_exp[Pm.j] = u + tenure + 1;
            if (lead_cta) {
                if (S.n_moves < traj_cap) {
                    stage_move mv;
                    mv.iter = u; mv.i = Pm.i; mv.j = Pm.j; mv.flags = flags;
                    mv.cov = Pm.cov; mv.dist = Pm.dist;
                    w.traj[S.n_moves] = mv;
                }
                if (flags & STAGE_MOVE_NEW_BEST)
                    for (int k = 0; k < K; k++) w.best_open[k] = s_open[k];
            }
            S.n_moves += 1;
            S.recn = 0;
            S.qn = 0;
        }
        }   // the Tabu move
        for (int k = tid; k < K; k += NT) {
            s_lc[k] = 0;
            s_ld[k] = 0;
            s_ic[k] = 0;
            s_id[k] = 0;
        }
        __syncthreads();
        lap(kClkMove);

        const int ss = S.mv_s, jj = S.mv_j, ic = S.mv_i;
        // ------------------------------------------------ refresh this CTA's missions (a7)
        {
            const size_t M_pad = w.M_pad;
            const int32_t *rowj = A.cost + (size_t)jj * M_pad;
            const int32_t *rowi = A.cost + (size_t)ic * M_pad;
            long long gic = 0, gid = 0, rv0c = 0, rv0d = 0;
            int *rcount = &S.recn;
            // a changed mission: its record, in this CTA's region (clamped as
            // the update reads it), and its change of V0 (f(a) new minus old)
            // and of loss (f(b) - f(a) out of its old best slot, into its new
            // one); every lane of the warp calls it
            auto record = [&](bool ch, int m, int ao, int bo, int so, int an, int bn, int sn) {
                const unsigned cm = __ballot_sync(0xffffffffu, ch);
                if (!cm) return;
                const int lead = __ffs(cm) - 1;
                int q0 = 0;
                if (lane == lead) q0 = atomicAdd(rcount, __popc(cm));
                q0 = __shfl_sync(0xffffffffu, q0, lead);
                int oc = 0, nc = 0;
                long long od = 0, nd = 0;
                if (ch) {
                    const int ao1 = min(ao, R + 1), bo1 = min(bo, R + 1), an1 = min(an, R + 1), bn1 = min(bn, R + 1);
                    int4 *r = region + 2 * (size_t)(q0 + __popc(cm & ((1u << lane) - 1u)));
                    r[0] = make_int4(m, max(bo1, bn1), ao1, bo1);
                    r[1] = make_int4(so, an1, bn1, sn);
                    const int cao = ao1 <= R, cbo = bo1 <= R, can = an1 <= R, cbn = bn1 <= R;
                    const long long fao = cao ? ao1 : 0, fbo = cbo ? bo1 : 0, fan = can ? an1 : 0,
                                    fbn = cbn ? bn1 : 0;
                    rv0c += can - cao;
                    rv0d += fan - fao;
                    oc = cbo - cao; od = fbo - fao;   // the old loss term, taken out
                    nc = cbn - can; nd = fbn - fan;   // the new one
                }
                slot_add_warp(ch && (oc | (od != 0)), so, -oc, -od, s_lc, s_ld);
                slot_add_warp(ch && (nc | (nd != 0)), sn, nc, nd, s_lc, s_ld);
            };
            // one chunk of 32 missions per warp step, values loaded beforehand.
            // The search keeps each mission's best and second-best cost exact
            // up to R and R + 1 above it (an uncovered cost adds no term, so no
            // term depends on its value or its slot): a mission loses a base
            // only if that base covered it, and only those are rescanned.
            auto chunk = [&](int m, bool in, int a, int b, int k1, int k2, int x, int xi) {
                bool term = false;
                a = min(a, R + 1);
                b = min(b, R + 1);
                const bool lost = in && ((a <= R && k1 == ss) || (b <= R && k2 == ss));
                const int ao = a, bo = b, so = k1;   // the state before the move
                if (in && !lost) {
                    const int x1 = min(x, R + 1);
                    if (x1 < a || (x1 == a && a <= R && jj < s_open[k1])) {
                        k2 = k1; b = a;
                        k1 = ss; a = x1;
                        w.a[m] = a; w.b[m] = b; w.s1[m] = (int16_t)k1; w.s2[m] = (int16_t)k2;
                    } else if (x1 < b || (x1 == b && b <= R && jj < s_open[k2])) {
                        k2 = ss; b = x1;
                        w.b[m] = b; w.s2[m] = (int16_t)k2;
                    }
                    term = true;
                }
                // missions that lost their best or second best: rescanned by
                // the whole CTA after the loop (past the queue's capacity, in place)
                const unsigned lm = __ballot_sync(0xffffffffu, lost);
                if (lm) {
                    int q0 = 0;
                    if (lane == __ffs(lm) - 1) q0 = atomicAdd(&S.qn, __popc(lm));
                    q0 = __shfl_sync(0xffffffffu, q0, __ffs(lm) - 1);
                    if (lost) {
                        const int pos = q0 + __popc(lm & ((1u << lane) - 1u));
                        if (pos < kRefQ) {
                            s_q[pos] = m;
                        } else {
                            const int2 ab = refresh_scan_one(w, A.cost, m, s_open, k1);
                            a = ab.x; b = ab.y;
                            term = true;
                        }
                    }
                }
                if (term) closed_column_terms(xi, a, b, k1, R, gic, gid, s_ic, s_id);
                record(term && terms_changed(ao, bo, so, a, b, k1, R), m, ao, bo, so, a, b, k1);
            };
            // this CTA's chunks: chunk r of block b is missions (b * CPB + r)
            // * 32 .. +31, blocks gr, gr + G, gr + 2G, ...; warp w takes the
            // CTA's chunks w, w + 32, ..., kStep per step (their loads in
            // flight together)
            constexpr int CPB = kBlockMissions / 32;   // chunks per block
            const int nch = (w.M + 31) >> 5;
            const int nblk = (nch + CPB - 1) / CPB;
            const int mine_blocks = nblk > gr ? (nblk - gr + G - 1) / G : 0;
            const int mine_chunks = mine_blocks * CPB;
            auto chunk_of = [&](int k) { return (gr + (k / CPB) * G) * CPB + (k % CPB); };
            constexpr int kStep = 2;
            for (int k = warp; k < mine_chunks; k += kStep * kPerWarps) {   // the same on every lane
                int ch[kStep], mm[kStep], va[kStep], vb[kStep], v1[kStep], v2[kStep], vx[kStep], vxi[kStep];
#pragma unroll
                for (int e = 0; e < kStep; e++) {
                    const int kk = k + e * kPerWarps;
                    ch[e] = kk < mine_chunks ? chunk_of(kk) : nch;
                    mm[e] = ch[e] * 32 + lane;
                    const bool in = ch[e] < nch && mm[e] < w.M;
                    va[e] = in ? w.a[mm[e]] : 0;
                    vb[e] = in ? w.b[mm[e]] : 0;
                    v1[e] = in ? w.s1[mm[e]] : 0;
                    v2[e] = in ? w.s2[mm[e]] : 0;
                    vx[e] = in ? __ldcs(rowj + mm[e]) : 0;
                    vxi[e] = in ? __ldcs(rowi + mm[e]) : 0;
                }
#pragma unroll
                for (int e = 0; e < kStep; e++)
                    if (ch[e] < nch) chunk(mm[e], mm[e] < w.M, va[e], vb[e], v1[e], v2[e], vx[e], vxi[e]);
            }
            __syncthreads();
            sub(kClkRefLoop);
            const int nq = min(S.qn, kRefQ);   // no thread changes the count after the barrier
            if (nq > 0)   // (their V0 and loss changes go with their records)
                refresh_rescans(w, A.cost, s_open, s_q, nq, rowi, gic, gid, s_ic, s_id, [](int, int, int) {},
                                record);
            __syncthreads();
            sub(kClkRefRescan);
            // this CTA's parts of the move's sums -- the closed base's column
            // (gain, extra per slot) and the changes of V0 and loss per slot --
            // and its record count, stored in entries of its own (value v of
            // CTA g at psum[v][g]); the update adds each value's parts up, so
            // no address takes an atomic from every CTA
            {
                __shared__ long long s_p4[4][kPerWarps];
                const long long p4[4] = {warp_sum_ll(gic), warp_sum_ll(gid), warp_sum_ll(rv0c), warp_sum_ll(rv0d)};
                if (lane == 0)
                    for (int e = 0; e < 4; e++) s_p4[e][warp] = p4[e];
                __syncthreads();
                const int g = gr;
                long long *P = A.psum;
                if (tid < 4) {
                    long long v = 0;
                    for (int k = 0; k < kPerWarps; k++) v += s_p4[tid][k];
                    const int at = tid < 2 ? tid : nA + tid - 2;   // gain (c, d); V0 (c, d)
                    P[(size_t)at * G + g] = v;
                }
                if (tid == 0) A.nrec[g] = S.recn;
                for (int k = tid; k < K; k += NT) {
                    P[(size_t)(2 + k) * G + g] = (long long)s_ic[k];
                    P[(size_t)(2 + K + k) * G + g] = (long long)s_id[k];
                    P[(size_t)(nA + 2 + k) * G + g] = (long long)s_lc[k];
                    P[(size_t)(nA + 2 + K + k) * G + g] = (long long)s_ld[k];
                }
            }
            sub(kClkRefSums);
        }
        lap(kClkRefresh);
        if (!grid_sync(A.bar, gen, G, A.spin_limit, A.err)) break;
        lap(kClkWaitB);

        // ------------------------------------------------ update every column with this CTA's records (a4)
        {
            // This CTA's share of the list: records r0 .. r0+nshare-1 (the
            // list is in spatial order, so a share is spatially compact),
            // staged in shared memory in rounds of at most REC, ordered by
            // their new slot (a base's terms in a row then mostly go to one
            // slot's column and add up in one run), with the cell minima of
            // each record's row.  Per cell of the row (32 positions, one per
            // lane) the records whose minimum over the cell is below their
            // threshold are listed (a cell at or above it has no term); the
            // lists, cut into items of at most kUpdItem records, are dealt to
            // the warps in turn, and a warp loads an item's costs in the cell
            // (32 costs, 128 bytes per record) kUpdBatch records at a time and
            // compares each lane's cost with the threshold.  Each item adds
            // its sums to the columns by itself.
            // Every CTA's record count and their exclusive prefix s_pre (in
            // the refresh's queue, unused until the next refresh): record r of
            // the move's list is record r - s_pre[g] of CTA g's region, for
            // the last g with s_pre[g] <= r.  Meanwhile warp k of CTA g adds up
            // the parts of value v = g + k * G of the move's sums: the closed
            // base's column (into the column sums), and V0 and loss of the new
            // placement (this placement's plus the changes).
            int *s_pre = s_q;
            if (tid < G) s_pre[tid] = __ldcg(&A.nrec[tid]);
            {
                const unsigned long long *cu = A.acc + (size_t)(u & 1) * nA;
                unsigned long long *nx = A.acc + (size_t)((u + 1) & 1) * nA;
                unsigned long long *cl = A.col + (size_t)(u & 1) * nA;
                for (int v = gr + warp * G; v < 2 * nA; v += kPerWarps * G) {   // the same on the warp
                    const unsigned long long was = (v >= nA && lane == 0) ? __ldcg(&cu[v - nA]) : 0ull;
                    long long sum = 0;
#pragma unroll
                    for (int e = 0; e < kMaxGrid / 32; e++) {
                        const int g = lane + 32 * e;
                        if (g < G) sum += __ldcg(&A.psum[(size_t)v * G + g]);
                    }
                    sum = warp_sum_ll(sum);
                    if (lane == 0) {
                        if (v < nA) cl[v] = (unsigned long long)sum;
                        else nx[v - nA] = was + (unsigned long long)sum;
                    }
                }
            }
            __syncthreads();
            if (warp == 0) {   // the prefix in place (G <= kMaxGrid: 8 counts per lane); s_pre[G] = the total
                constexpr int PL = kMaxGrid / 32;
                int v[PL], sum = 0;
#pragma unroll
                for (int e = 0; e < PL; e++) {
                    const int g = lane * PL + e;
                    v[e] = g < G ? s_pre[g] : 0;
                    sum += v[e];
                }
                int incl = sum;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, d);
                    if (lane >= d) incl += y;
                }
                int run = incl - sum;
#pragma unroll
                for (int e = 0; e < PL; e++) {
                    const int g = lane * PL + e;
                    if (g < G) s_pre[g] = run;
                    run += v[e];
                }
                if (lane == 31) s_pre[G] = incl;
            }
            __syncthreads();
            const int ntot = min(s_pre[G], w.M);
            const int r0 = (int)((long long)ntot * gr / G);
            const int nshare = (int)((long long)ntot * (gr + 1) / G) - r0;
            if (lead_cta) rec_total += ntot;
            const int nCell = ldT >> 5;
            const int *srec = reinterpret_cast<const int *>(s_recs);
            unsigned lanes = 0, passes = 0;   // this warp's pairs with a term, (record, cell) passes
            unsigned flushes = 0;             // this thread's runs written to the columns
            for (int base = 0; base < nshare; base += REC) {   // the same on every thread
                const int n = min(REC, nshare - base);
                __syncthreads();   // the previous round's records are used
                for (int q = tid; q < 2 * n; q += NT) {
                    const int r = r0 + base + (q >> 1);   // < ntot
                    int lo = 0, hi = G - 1;               // the region holding record r
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_pre[mid] <= r) lo = mid;
                        else hi = mid - 1;
                    }
                    s_raw[q] = __ldcg(&A.region[((size_t)lo * A.region_cap + (r - s_pre[lo])) * 2 + (q & 1)]);
                }
                for (int k = tid; k < K; k += NT) s_cnt[k] = 0;
                __syncthreads();
                // counting sort by new slot (the order within a slot is free:
                // the sums are integers)
                int key = tid < n ? s_raw[2 * tid + 1].w : 0;
                key = (unsigned)key < (unsigned)K ? key : 0;   // an index; only the order depends on it
                const int pos = tid < n ? atomicAdd(&s_cnt[key], 1) : 0;
                __syncthreads();
                if (tid < 32) {   // exclusive scan of the K counts (K <= 256: 8 per lane)
                    int v[8], sum = 0;
#pragma unroll
                    for (int e = 0; e < 8; e++) {
                        const int k = tid * 8 + e;
                        v[e] = k < K ? s_cnt[k] : 0;
                        sum += v[e];
                    }
                    int incl = sum;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, incl, d);
                        if (tid >= d) incl += y;
                    }
                    int run = incl - sum;
#pragma unroll
                    for (int e = 0; e < 8; e++) {
                        const int k = tid * 8 + e;
                        if (k < K) s_cnt[k] = run;
                        run += v[e];
                    }
                }
                __syncthreads();
                if (tid < n) {
                    const int dst = s_cnt[key] + pos;
                    s_recs[2 * dst] = s_raw[2 * tid];
                    s_recs[2 * dst + 1] = s_raw[2 * tid + 1];
                }
                __syncthreads();
                {
                    const int lane = tid & 31;
#pragma unroll 4
                    for (int r = tid >> 5; r < n; r += kPerWarps) {   // a warp per record
                        const size_t row = (size_t)srec[8 * r] * cell_ld(ldT);
                        for (int c = lane; c < nCell; c += 32) s_cells[r * nCell + c] = __ldcg(&w.cellmin[row + c]);
                    }
                }
                __syncthreads();
                sub(kClkUpdIssue);
                // per cell (32 positions of the row): the records whose minimum
                // over the cell is below their threshold, in order (a cell at
                // or above it has no term)
                const int lane = tid & 31, warp = tid >> 5;
                for (int cell = warp; cell < nCell; cell += kPerWarps) {   // the same on the warp
                    uint16_t *cl = s_clist + cell * REC;
                    int cnt = 0;
                    for (int rb = 0; rb < n; rb += 32) {   // the same on the warp
                        const int r = rb + lane;
                        const bool need = r < n && s_cells[r * nCell + cell] < srec[8 * r + 1];
                        const unsigned bm = __ballot_sync(0xffffffffu, need);
                        if (need) cl[cnt + __popc(bm & ((1u << lane) - 1u))] = (uint16_t)r;
                        cnt += __popc(bm);
                    }
                    if (lane == 0) {
                        s_ccnt[cell] = cnt;
                        atomicAdd(&s_terms[3], (unsigned long long)cnt);   // cells read (128 bytes each)
                    }
                }
                __syncthreads();
                // work items: each cell's list in pieces of at most kUpdItem
                // records, dealt to the warps in turn (the cells near the move
                // have the longest lists); s_ipre = first item of each cell
                static_assert(kMaxLd / 32 <= 64, "two cells per lane");
                if (tid < 32) {
                    const int c0 = 2 * tid, c1 = c0 + 1;
                    const int n0 = c0 < nCell ? (s_ccnt[c0] + kUpdItem - 1) / kUpdItem : 0;
                    const int n1 = c1 < nCell ? (s_ccnt[c1] + kUpdItem - 1) / kUpdItem : 0;
                    int incl = n0 + n1;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, incl, d);
                        if (tid >= d) incl += y;
                    }
                    const int ex = incl - n0 - n1;
                    if (c0 < nCell) s_ipre[c0] = ex;
                    if (c1 < nCell) s_ipre[c1] = ex + n0;
                    if (tid == 31) s_ipre[kMaxLd / 32] = incl;
                }
                __syncthreads();
                const int nitems = s_ipre[kMaxLd / 32];
                for (int it = warp; it < nitems; it += kPerWarps) {   // the same on the warp
                    int lo = 0, hc = nCell - 1;   // the item's cell: the last with s_ipre <= it
                    while (lo < hc) {
                        const int mid = (lo + hc + 1) >> 1;
                        if (s_ipre[mid] <= it) lo = mid;
                        else hc = mid - 1;
                    }
                    const int cell = lo;
                    const int e0 = (it - s_ipre[cell]) * kUpdItem, e1 = min(e0 + kUpdItem, s_ccnt[cell]);
                    const uint16_t *cl = s_clist + cell * REC;
                    const int pos = cell * 32 + lane;   // < ldT
                    const int j = w.border[pos];
                    const bool mine = j >= 0 && j != ic;
                    // the listed records' costs in this cell (the warp's 32
                    // consecutive entries of each row, 128 bytes), kUpdBatch
                    // records' at a time, every load of a batch in flight together
                    const int32_t *Tp = w.costT + pos;
                    long long gd = 0;
                    int gc = 0;
                    DeltaRun rn{-1, 0, 0}, ro{-1, 0, 0};
                    for (int q0 = e0; q0 < e1; q0 += kUpdBatch) {   // the same on the warp
                        int xs[kUpdBatch];
#pragma unroll
                        for (int v = 0; v < kUpdBatch; v++) {
                            const int q = q0 + v;
                            xs[v] = (q < e1 && mine) ? ld_stream(Tp + (size_t)srec[8 * cl[q]] * ldT, evict_first)
                                                     : INT_MAX;
                        }
#pragma unroll
                        for (int v = 0; v < kUpdBatch; v++) {
                            const int q = q0 + v;
                            if (q >= e1) break;   // the same on the warp
                            const int r = cl[q];
                            const int x = xs[v];
                            const int hi = srec[8 * r + 1];
                            const unsigned bm = __ballot_sync(0xffffffffu, x < hi);
                            lanes += __popc(bm);
                            passes += bm != 0u;
                            if (x >= hi) continue;
                            const int4 q0r = s_recs[2 * r];       // (column, hi, old a, old b)
                            const int4 q1r = s_recs[2 * r + 1];   // (old slot, new a, new b, new slot)
                            const int ao = q0r.z, bo = q0r.w, so = q1r.x, an = q1r.y, bn = q1r.z, sn = q1r.w;
                            const int cao = ao <= R, cbo = bo <= R, can = an <= R, cbn = bn <= R;
                            if (x < an) { gc += 1 - can; gd += (long long)x - (can ? an : 0); }
                            if (x < ao) { gc -= 1 - cao; gd -= (long long)x - (cao ? ao : 0); }
                            // extra: the new state's term into the new slot's
                            // column, the old one's out of the old slot's (one
                            // run when the slot is kept)
                            int nc = 0, nd = 0, oc = 0, od = 0;
                            if (x < bn) { nc = can - cbn; nd = (can ? max(x, an) : 0) - (cbn ? bn : 0); }
                            if (x < bo) { oc = cao - cbo; od = (cao ? max(x, ao) : 0) - (cbo ? bo : 0); }
                            if (sn == so) {
                                nc -= oc;
                                nd -= od;
                                oc = od = 0;
                            }
                            if (nc | nd) {
                                flushes += sn != rn.s && rn.s >= 0 && (rn.c | (rn.d != 0));
                                delta_run_add(rn, sn, nc, nd, w, j);
                            }
                            if (oc | od) {
                                flushes += so != ro.s && ro.s >= 0 && (ro.c | (ro.d != 0));
                                delta_run_add(ro, so, -oc, -od, w, j);
                            }
                        }
                    }
                    if (mine) {
                        flushes += (rn.s >= 0 && (rn.c | (rn.d != 0))) + (ro.s >= 0 && (ro.c | (ro.d != 0)));
                        delta_run_add(rn, -1, 0, 0, w, j);   // flush
                        delta_run_add(ro, -1, 0, 0, w, j);
                        if (gc) atomicAdd(&w.gain_c[j], gc);
                        if (gd) atomicAdd(&w.gain_d[j], (unsigned long long)gd);
                    }
                }
                sub(kClkUpdCompute);
            }
            if ((tid & 31) == 0 && passes) {
                atomicAdd(&s_terms[0], (unsigned long long)lanes);
                atomicAdd(&s_terms[1], (unsigned long long)passes);
            }
            {
                const unsigned f = __reduce_add_sync(0xffffffffu, flushes);
                if ((tid & 31) == 0 && f) atomicAdd(&s_terms[2], (unsigned long long)f);
            }
            __syncthreads();   // the CTA's slowest warp
            sub(kClkUpdWait);
        }
        lap(kClkUpdate);
        if (tid == 0) {
            S.t = u + 1;
            S.prev_i = ic;
        }
        if (!grid_sync(A.bar, gen, G, A.spin_limit, A.err)) break;
        lap(kClkWaitC);
        select();   // the next move's keys (and the closed column written back)
    }

    // ------------------------------------------------ hand the state back (CTA 0)
    __syncthreads();
    if (tid < 4) atomicAdd(reinterpret_cast<unsigned long long *>(&A.info[2 + tid]), s_terms[tid]);
    if (tid == 0) {
        for (int k = 0; k < kClocks; k++) A.cta_ns[(size_t)gr * kClocks + k] = s_clk[k];
        if (lead_cta) A.info[1] = rec_total;
    }
    if (!lead_cta) return;
    const int t = S.t;
    const unsigned long long *acc = A.acc + (size_t)(t & 1) * nA;
    for (int k = tid; k < K; k += NT) {
        w.open[k] = s_open[k];
        w.loss_c[k] = __ldcg(&acc[2 + k]);
        w.loss_d[k] = __ldcg(&acc[2 + K + k]);
    }
    for (int c = tid; c < nC; c += NT) w.cand[c] = s_cand[c];
    for (int b = tid; b < B; b += NT) w.expiry[b] = s_exp[b];
    if (tid == 0) {
        w.v0[0] = __ldcg(&acc[0]);
        w.v0[1] = __ldcg(&acc[1]);
        st->t = t;
        st->n_moves = S.n_moves;
        st->done = S.done;
        st->cur_cov = S.cur_c;
        st->cur_dist = S.cur_d;
        st->best_cov = S.best_c;
        st->best_dist = S.best_d;
        st->best_iter = S.best_iter;
        st->mv_s = S.mv_s;
        st->mv_i = S.mv_i;
        st->mv_j = S.mv_j;
        st->chg_n = 0;
        st->err |= *reinterpret_cast<volatile int *>(A.err);
        if constexpr (LOCAL) {
            st->ls_pass = S.ls_pass;
            st->ls_pos = S.ls_pos;
            st->ls_moved = S.ls_moved;
            st->ls_optimum = S.ls_optimum;
        }
        A.info[0] = G;
    }
}

__global__ void __launch_bounds__(kPerThreads, 1) k_tabu_persist(PersistArgs A)
{
    persist_search<kPerThreads, kRecCap>(A, (int)blockIdx.x, (int)gridDim.x);
}

// Alg. 2's local search in one cooperative launch (the same body, LOCAL).
__global__ void __launch_bounds__(kPerThreads, 1) k_local_persist(PersistArgs A)
{
    persist_search<kPerThreads, kRecCap, true>(A, (int)blockIdx.x, (int)gridDim.x);
}

// Many searches in one cooperative launch: CTA b runs the entries
// sched[off[b]] .. sched[off[b+1]-1], each (search, its rank among the
// search's G CTAs), in order.  The host gives every CTA its entries in one
// global order of the searches, so the lowest-numbered unfinished search has
// every one of its CTAs at it or done with it, and each barrier wait ends
// (bounded by the spin limit in any case).  A search's arguments are staged
// in shared memory.
__global__ void __launch_bounds__(kBatchThreads, 1024 / kBatchThreads) k_tabu_batch(int max_steps,
                                                                                       const PersistArgs *__restrict__ args,
                                                               const int2 *__restrict__ sched,
                                                               const int *__restrict__ off)
{
    __shared__ __align__(16) PersistArgs sA;
    static_assert(sizeof(PersistArgs) % 4 == 0, "copied as 32-bit words");
    const int e0 = off[blockIdx.x], e1 = off[blockIdx.x + 1];
    for (int e = e0; e < e1; e++) {
        const int2 it = sched[e];
        const int *src = reinterpret_cast<const int *>(args + it.x);
        int *dst = reinterpret_cast<int *>(&sA);
        for (int q = threadIdx.x; q < (int)(sizeof(PersistArgs) / 4); q += kBatchThreads) dst[q] = __ldg(src + q);
        __syncthreads();
        persist_search<kBatchThreads, kBatchRec>(sA, it.y, sA.G, max_steps);
        __syncthreads();   // every thread is done with this search's arguments
    }
}

// Test support: one block waits on a flag that nothing sets, with the same
// bounded poll as the grid barrier; the error word records the give-up.
__global__ void k_wait_unset_flag(const unsigned *flag, long long limit, int *err)
{
    if (threadIdx.x == 0 && !wait_change(flag, *flag, limit)) atomicOr(err, kErrPipelineTimeout);
}

// ---------------------------------------------------------------- host side

static size_t persist_smem(int K, int B, int ldT) { return per_layout(K, B, ldT, kRecCap).total; }
static size_t batch_smem(int K, int B, int ldT) { return per_layout(K, B, ldT, kBatchRec).total; }

// CTAs of a persistent search: up to one per SM (the cooperative launch needs
// them all resident), no more than the mission blocks; 0 when the shape is
// not supported (K > 256, more than 2048 bases, or the per-CTA arrays do not
// fit in shared memory).
int persist_grid(int K, int B, int ldT, int M_pad)
{
    if (K > kPipeMaxK || (ldT & 31) || ldT > kMaxLd) return 0;
    const size_t sm = persist_smem(K, B, ldT);
    if (sm > kPerSmemLimit) return 0;
    int nb = 0, dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)k_tabu_persist, kPerThreads, sm) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int blocks = (M_pad + kBlockMissions - 1) / kBlockMissions;
    int g = nb * sms;
    if (g > blocks) g = blocks;
    if (g > kMaxGrid) g = kMaxGrid;
    return g > 0 ? g : 0;
}

static size_t region_cap(int M_pad, int grid)
{
    const int nblk = (M_pad + kBlockMissions - 1) / kBlockMissions;
    return (size_t)((nblk + grid - 1) / grid) * kBlockMissions;
}

size_t persist_scratch_bytes(int K, int grid, int M_pad)
{
    const size_t nA = 2 + 2 * (size_t)K;
    return per_align(2 * nA * 8, 256) * 2 + 256 + per_align((size_t)2 * grid * sizeof(MoveKey), 256) +
           per_align((size_t)grid * 4, 256) + per_align(2 * nA * grid * 8, 256) +
           per_align(region_cap(M_pad, grid) * grid * 32, 256) + per_align((size_t)grid * kClocks * 8, 256);
}

size_t persist_clock_offset(int K, int grid, int M_pad)
{
    return persist_scratch_bytes(K, grid, M_pad) - per_align((size_t)grid * kClocks * 8, 256);
}

size_t persist_info_offset(int K)
{
    const size_t nA = 2 + 2 * (size_t)K;
    return per_align(2 * nA * 8, 256) * 2 + 64;
}

cudaError_t persist_init()
{
    cudaError_t e = cudaFuncSetAttribute(k_tabu_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPerSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tabu_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPerSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_local_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPerSmemLimit);
    return e;
}


// The arguments of one search on `grid` CTAs over its scratch (laid out as
// persist_scratch_bytes counts it); with `clear`, the scratch's sums, counters
// and barrier are cleared and the start placement's V0 and loss put in both
// buffers (asynchronously, on s; a batch does this with k_batch_prep).
static cudaError_t persist_args(const TabuBuffers &w, const int32_t *cost, void *scratch, int grid,
                                long long spin_limit, cudaStream_t s, PersistArgs &A, bool clear = true)
{
    const size_t nA = 2 + 2 * (size_t)w.K;
    if (grid < 1 || grid > kMaxGrid || w.ldT > kMaxLd || (w.ldT & 31)) return cudaErrorInvalidValue;
    char *p = static_cast<char *>(scratch);
    A = PersistArgs{};
    A.G = grid;
    A.w = w;
    A.cost = cost;
    A.acc = reinterpret_cast<unsigned long long *>(p);
    p += per_align(2 * nA * 8, 256);
    A.col = reinterpret_cast<unsigned long long *>(p);
    p += per_align(2 * nA * 8, 256);
    A.bar = reinterpret_cast<unsigned *>(p + 16);
    A.err = reinterpret_cast<int *>(p + 32);
    A.info = reinterpret_cast<long long *>(p + 64);
    p += 256;
    const size_t cleared = (size_t)(p - static_cast<char *>(scratch));
    A.part = reinterpret_cast<MoveKey *>(p);
    p += per_align((size_t)2 * grid * sizeof(MoveKey), 256);
    A.nrec = reinterpret_cast<int *>(p);   // each written by its CTA before it is read
    p += per_align((size_t)grid * 4, 256);
    A.psum = reinterpret_cast<long long *>(p);
    p += per_align(2 * nA * grid * 8, 256);
    A.region_cap = (int)region_cap(w.M_pad, grid);
    A.region = reinterpret_cast<int4 *>(p);
    p += per_align((size_t)A.region_cap * grid * 32, 256);
    A.cta_ns = reinterpret_cast<long long *>(p);
    A.spin_limit = spin_limit > 0 ? spin_limit : (1ll << 26);
    if (!clear) return cudaSuccess;
    // clear the sums, counters and barrier, then put the start placement's
    // V0 and loss (the per-mission initialisation's) in both buffers (the
    // first move's update writes the other one again)
    cudaError_t e = cudaMemsetAsync(scratch, 0, cleared, s);
    for (int b = 0; b < 2 && e == cudaSuccess; b++) {
        unsigned long long *a0 = A.acc + (size_t)b * nA;
        e = cudaMemcpyAsync(a0, w.v0, 16, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(a0 + 2, w.loss_c, (size_t)w.K * 8, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(a0 + 2 + w.K, w.loss_d, (size_t)w.K * 8, cudaMemcpyDeviceToDevice, s);
    }
    return e;
}

cudaError_t launch_tabu_persist(const TabuBuffers &w, const int32_t *cost, void *scratch, int grid,
                                long long spin_limit, cudaStream_t s)
{
    PersistArgs A;
    cudaError_t e = persist_args(w, cost, scratch, grid, spin_limit, s, A);
    if (e != cudaSuccess) return e;
    void *args[] = {&A};
    return cudaLaunchCooperativeKernel((const void *)k_tabu_persist, dim3(grid), dim3(kPerThreads), args,
                                       persist_smem(w.K, w.B, w.ldT), s);
}

cudaError_t launch_local_persist(const TabuBuffers &w, const int32_t *cost, void *scratch, int grid,
                                 long long spin_limit, const int *rank_slot, const int *rank_cand, cudaStream_t s)
{
    PersistArgs A;
    cudaError_t e = persist_args(w, cost, scratch, grid, spin_limit, s, A);
    if (e != cudaSuccess) return e;
    A.rank_slot = rank_slot;
    A.rank_cand = rank_cand;
    void *args[] = {&A};
    return cudaLaunchCooperativeKernel((const void *)k_local_persist, dim3(grid), dim3(kPerThreads), args,
                                       persist_smem(w.K, w.B, w.ldT), s);
}

size_t persist_args_bytes() { return sizeof(PersistArgs); }

cudaError_t persist_args_host(const TabuBuffers &w, const int32_t *cost, void *scratch, int gang,
                              long long spin_limit, cudaStream_t s, void *out)
{
    PersistArgs A;
    cudaError_t e = persist_args(w, cost, scratch, gang, spin_limit, s, A, false);
    if (e == cudaSuccess) *static_cast<PersistArgs *>(out) = A;
    return e;
}

// Block k readies search k of a batch: clears its sums, counters and barrier
// (the scratch's head, as persist_args clears it) and puts its start
// placement's V0 and loss in both buffers.
__global__ void k_batch_prep(const PersistArgs *__restrict__ args)
{
    const PersistArgs &A = args[blockIdx.x];
    const int K = A.w.K;
    const size_t nA = 2 + 2 * (size_t)K;
    const size_t words = (2 * per_align(2 * nA * 8, 256) + 256) / 8;
    for (size_t q = threadIdx.x; q < words; q += blockDim.x) A.acc[q] = 0ull;
    __syncthreads();
    for (size_t q = threadIdx.x; q < 2 * nA; q += blockDim.x) {
        const size_t k = q % nA;
        A.acc[q] = k < 2 ? A.w.v0[k] : k < 2 + (size_t)K ? A.w.loss_c[k - 2] : A.w.loss_d[k - 2 - K];
    }
}

cudaError_t launch_batch_prep(const void *d_args, int n, cudaStream_t s)
{
    if (n < 1) return cudaSuccess;
    k_batch_prep<<<n, 256, 0, s>>>(static_cast<const PersistArgs *>(d_args));
    return cudaGetLastError();
}

size_t persist_search_smem(int K, int B, int ldT) { return batch_smem(K, B, ldT); }

// CTAs of a batch launch with `smem` bytes of dynamic shared memory: as many
// as the device holds at once (one per SM for 1024-thread CTAs); 0 when none
// fits.  (Each search of the batch takes at most kMaxGrid of them.)
int persist_batch_grid(size_t smem)
{
    if (smem > kPerSmemLimit) return 0;
    int nb = 0, dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void *)k_tabu_batch, kBatchThreads, smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb * sms;
}

// Searches whose shape the persistent body takes (K <= 256, at most 2048
// bases, its per-CTA arrays within the shared-memory limit).
bool persist_shape_ok(int K, int B, int ldT)
{
    return K <= kPipeMaxK && !(ldT & 31) && ldT <= kMaxLd && batch_smem(K, B, ldT) <= kPerSmemLimit;
}

int persist_max_gang() { return kMaxGrid; }

cudaError_t launch_tabu_batch(const void *d_args, const int2 *d_sched, const int *d_off, int grid, size_t smem,
                              cudaStream_t s, int max_steps)
{
    const PersistArgs *a = static_cast<const PersistArgs *>(d_args);
    void *args[] = {(void *)&max_steps, (void *)&a, (void *)&d_sched, (void *)&d_off};
    return cudaLaunchCooperativeKernel((const void *)k_tabu_batch, dim3(grid), dim3(kBatchThreads), args, smem, s);
}

cudaError_t launch_wait_unset_flag(unsigned *flag, long long limit, int *err, cudaStream_t s)
{
    k_wait_unset_flag<<<1, 32, 0, s>>>(flag, limit > 0 ? limit : (1ll << 26), err);
    return cudaGetLastError();
}

}  // namespace stg
