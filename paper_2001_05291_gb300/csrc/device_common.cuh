// Device helpers shared by the staging engine's kernels (kernels.cu) and the
// persistent Tabu kernel (persist.cu): warp and block reductions, the move
// order of the Tabu selection, the per-mission terms of the objective
// decomposition, the refresh's rescans and change records.  Included by the
// .cu files only.
#pragma once

#include <cuda_runtime.h>
#include <climits>
#include <stdint.h>

#include "stage_internal.h"

namespace stg {

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// Warp sum of per-lane int64 values that each fit in int32, over the lanes of
// `mask` (all of which call this with the same mask): biased 16-bit halves,
// three 32-bit reductions.
__device__ __forceinline__ long long group_sum_small(unsigned mask, long long v)
{
    const unsigned u = (unsigned)(v + 2147483648ll);
    const unsigned lo = __reduce_add_sync(mask, u & 0xffffu);
    const unsigned hi = __reduce_add_sync(mask, u >> 16);
    return ((long long)hi << 16) + (long long)lo - ((long long)__popc(mask) << 31);
}

// L2 cache policy for data read once per pass: evict it before other lines.
__device__ __forceinline__ unsigned long long evict_first_policy()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ int warp_sum_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of two int64 values; the result is valid in thread 0.
template <int NT>
__device__ __forceinline__ void block_sum2(long long &x, long long &y)
{
    __shared__ long long sx[NT / 32], sy[NT / 32];
    x = warp_sum_ll(x);
    y = warp_sum_ll(y);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sx[wid] = x; sy[wid] = y; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long a = 0, b = 0;
#pragma unroll
        for (int k = 0; k < NT / 32; k++) { a += sx[k]; b += sy[k]; }
        x = a; y = b;
    }
}

__device__ __forceinline__ void add_ull(unsigned long long *p, long long v)
{
    atomicAdd(p, (unsigned long long)v);
}

__device__ __forceinline__ bool obj_better(long long c1, long long d1, long long c2, long long d2)
{
    return c1 != c2 ? c1 > c2 : d1 < d2;
}

__device__ __forceinline__ bool key_better(const MoveKey &a, const MoveKey &b)
{
    if (!a.valid) return false;
    if (!b.valid) return true;
    if (a.cov != b.cov) return a.cov > b.cov;
    if (a.dist != b.dist) return a.dist < b.dist;
    if (a.i != b.i) return a.i < b.i;
    return a.j < b.j;
}

__device__ __forceinline__ void mission_terms(int a, int b, int R, long long &v0c, long long &v0d,
                                              int *s_lc, unsigned long long *s_ld, int s1)
{
    const int ca = a <= R, cb = b <= R;
    const long long da = ca ? a : 0, db = cb ? b : 0;
    v0c += ca;
    v0d += da;
    const int dc = cb - ca;
    const long long dd = db - da;
    // lanes with the same best slot add their terms first (neighbouring
    // columns share slots often), so a slot takes one shared atomic per warp
    // instead of one per lane; |dd| <= R < 2^31, as group_sum_small needs
    const unsigned peers = __match_any_sync(__activemask(), s1);
    const int sc = (int)__reduce_add_sync(peers, (unsigned)dc);
    const long long sd = group_sum_small(peers, dd);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) {
        if (sc) atomicAdd(&s_lc[s1], sc);
        if (sd) atomicAdd(&s_ld[s1], (unsigned long long)sd);
    }
}

__device__ __forceinline__ void scan_best_two(const int32_t *__restrict__ cost, size_t M_pad, int m,
                                              const int *s_open, int K, int &a, int &b, int &k1,
                                              int &k2)
{
    int c1 = kInf, c2 = kInf, i1 = 0x7fffffff, i2 = 0x7fffffff;
    k1 = -1;
    k2 = -1;
    for (int k0 = 0; k0 < K; k0 += 8) {
        int cv[8];
#pragma unroll
        for (int u = 0; u < 8; u++)
            cv[u] = (k0 + u < K) ? __ldg(cost + (size_t)s_open[k0 + u] * M_pad + m) : kInf;
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int k = k0 + u;
            if (k >= K) break;
            const int o = s_open[k];
            const int c = cv[u];
            if (k1 < 0 || c < c1 || (c == c1 && o < i1)) {
                k2 = k1; c2 = c1; i2 = i1;
                k1 = k; c1 = c; i1 = o;
            } else if (k2 < 0 || c < c2 || (c == c2 && o < i2)) {
                k2 = k; c2 = c; i2 = o;
            }
        }
    }
    a = c1;
    b = c2;
}

__device__ __forceinline__ MoveKey invalid_key()
{
    MoveKey k;
    k.cov = 0; k.dist = 0; k.i = 0; k.j = 0; k.s = 0; k.c = 0; k.valid = 0; k.tabu = 0;
    return k;
}

__device__ __forceinline__ MoveKey load_key_cg(const MoveKey *p)
{
    MoveKey k;
    k.cov = __ldcg(&p->cov);
    k.dist = __ldcg(&p->dist);
    k.i = __ldcg(&p->i);
    k.j = __ldcg(&p->j);
    k.s = __ldcg(&p->s);
    k.c = __ldcg(&p->c);
    k.valid = __ldcg(&p->valid);
    k.tabu = __ldcg(&p->tabu);
    return k;
}

// The best key of a warp under key_better's order (valid first; covered desc,
// distance asc, i asc, j asc), left in every lane: one 32-bit warp reduction per
// field of the order on the lanes still tied, then the winner's key is read
// from its lane.  Covered counts fit 31 bits, distances are non-negative and
// base ids fit 16 bits.
__device__ __forceinline__ void warp_best_key(MoveKey &k)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned tied = __ballot_sync(full, k.valid);
    if (!tied) return;
    const bool in1 = (tied >> lane) & 1u;
    const int cv = in1 ? (int)k.cov : -1;
    const int bc = __reduce_max_sync(full, cv);
    tied = __ballot_sync(full, in1 && cv == bc);
    const bool in2 = (tied >> lane) & 1u;
    const unsigned dh = in2 ? (unsigned)((unsigned long long)k.dist >> 32) : 0xffffffffu;
    const unsigned bdh = __reduce_min_sync(full, dh);
    tied = __ballot_sync(full, in2 && dh == bdh);
    const bool in3 = (tied >> lane) & 1u;
    const unsigned dl = in3 ? (unsigned)(unsigned long long)k.dist : 0xffffffffu;
    const unsigned bdl = __reduce_min_sync(full, dl);
    tied = __ballot_sync(full, in3 && dl == bdl);
    const bool in4 = (tied >> lane) & 1u;
    const unsigned ij = in4 ? (((unsigned)k.i << 16) | (unsigned)k.j) : 0xffffffffu;
    const unsigned bij = __reduce_min_sync(full, ij);
    tied = __ballot_sync(full, in4 && ij == bij);
    const int src = __ffs(tied) - 1;
    MoveKey o;
    o.cov = __shfl_sync(full, k.cov, src);
    o.dist = __shfl_sync(full, k.dist, src);
    o.i = __shfl_sync(full, k.i, src);
    o.j = __shfl_sync(full, k.j, src);
    o.s = __shfl_sync(full, k.s, src);
    o.c = __shfl_sync(full, k.c, src);
    o.valid = __shfl_sync(full, k.valid, src);
    o.tabu = __shfl_sync(full, k.tabu, src);
    k = o;
}

// Best admissible and best overall key of a block: warp reductions, then one
// warp over the warps' winners.  Every thread receives the results.
template <int NT>
__device__ __forceinline__ void block_best2(MoveKey &adm, MoveKey &all, MoveKey *s_adm, MoveKey *s_all)
{
    static_assert(NT % 32 == 0 && NT <= 1024, "block of whole warps");
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
        if (lane == 0) {
            s_adm[0] = adm;
            s_all[0] = all;
        }
    }
    __syncthreads();
    adm = s_adm[0];
    all = s_all[0];
    __syncthreads();
}

constexpr int kRefQ = 2048;
// Whether a mission's terms in the swap neighbourhood changed: they depend on
// its clamped best and second-best costs and, while it is covered, on its
// best slot (an uncovered mission adds no extra term to any slot).
__device__ __forceinline__ bool terms_changed(int ao, int bo, int so, int an, int bn, int sn, int R)
{
    const int ao1 = min(ao, R + 1), bo1 = min(bo, R + 1), an1 = min(an, R + 1), bn1 = min(bn, R + 1);
    return ao1 != an1 || bo1 != bn1 || (an1 <= R && so != sn);
}

// Append the lanes' changed missions to the record list, two int4 per
// record: (column, old a, old b, old best slot), (new a, new b, new best
// slot, 0); `count` is the list's length.  One global atomic per warp; every
// lane of the warp calls it.
__device__ __forceinline__ void record_changes(const TabuBuffers &w, int *count, bool ch, int m, int ao, int bo,
                                               int so, int an, int bn, int sn)
{
    const unsigned full = 0xffffffffu;
    const unsigned cm = __ballot_sync(full, ch);
    if (!cm) return;
    const int lane = threadIdx.x & 31, lead = __ffs(cm) - 1;
    int q0 = 0;
    if (lane == lead) q0 = atomicAdd(count, __popc(cm));
    q0 = __shfl_sync(full, q0, lead);
    if (ch) {
        int4 *r = w.chg + 2 * (size_t)(q0 + __popc(cm & ((1u << lane) - 1u)));
        r[0] = make_int4(m, ao, bo, so);
        r[1] = make_int4(an, bn, sn, 0);
    }
}

// A mission's terms in the column of a base x away (the closed base, a
// candidate again), for its state after the move: the gain term into
// (gc, gd), the extra term at its best slot into the block's accumulators.
// Lanes with the same best slot add their extra terms first (neighbouring
// columns share slots often, so a slot takes one shared atomic per warp, not
// one per lane); |term| <= R + 1 < 2^31, as group_sum_small needs.  Every
// lane that reaches the call takes part.
__device__ __forceinline__ void closed_column_terms(int x, int a, int b, int s1, int R, long long &gc, long long &gd,
                                                    int *s_ic, unsigned long long *s_id)
{
    const int a1 = min(a, R + 1), b1 = min(b, R + 1);
    int dc = 0;
    long long dd = 0;
    if (x < b1) {   // a <= b
        const int ca = a1 <= R, cb = b1 <= R;
        dc = ca - cb;
        dd = (ca ? (long long)max(x, a1) : 0ll) - (cb ? (long long)b1 : 0ll);
        if (x < a1) {
            gc += 1 - ca;
            gd += (long long)x - (ca ? (long long)a1 : 0ll);
        }
    }
    const unsigned active = __activemask();
    if (!__ballot_sync(active, dc != 0 || dd != 0)) return;
    const unsigned peers = __match_any_sync(active, s1);
    const int sc = (int)__reduce_add_sync(peers, (unsigned)dc);
    const long long sd = group_sum_small(peers, dd);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1 && (sc | (sd != 0))) {
        atomicAdd(&s_ic[s1], sc);
        atomicAdd(&s_id[s1], (unsigned long long)sd);
    }
}

// Best and second-best open base of the missions queued for a rescan (their
// best or second best was the closed base), G threads per mission with G
// chosen from the queue length so that a short queue still has every thread
// loading: a thread scans every G-th slot, 8 independent loads at a time,
// with keys (cost, base id) ordered as in scan_best_two; the G partial pairs
// are merged by butterfly shuffles within the group.  The mission's terms (V0,
// loss of its best slot) are added as mission_terms adds them.
// `terms(a, b, k1)` takes a rescanned mission's new state (the lanes that
// hold one call it together); `record(ch, m, ao, bo, so, an, bn, sn)`
// appends a changed mission's record, every lane of every warp calling it (ch
// false where nothing changed).
template <class Terms, class Record>
__device__ __forceinline__ void refresh_rescans(const TabuBuffers &w, const int32_t *__restrict__ cost,
                                                const int *s_open, const int *s_q, int nq,
                                                const int32_t *rowi, long long &gic, long long &gid, int *s_ic,
                                                unsigned long long *s_id, Terms terms, Record record)
{
    constexpr int L = 8;
    const unsigned full = 0xffffffffu;
    const int K = w.K;
    const size_t M_pad = w.M_pad;
    // threads per mission: as many as keep every thread of the block loading
    // (the same on every thread)
    const int nt = (int)blockDim.x;
    const int G = nq * 8 <= nt ? 8 : nq * 4 <= nt ? 4 : nq * 2 <= nt ? 2 : 1;
    const int per = blockDim.x / G;
    const int sub = threadIdx.x & (G - 1);
    for (int q0 = 0; q0 < nq; q0 += per) {
        const int qi = q0 + (int)threadIdx.x / G;
        const bool has = qi < nq;
        const int m = has ? s_q[qi] : 0;
        unsigned long long e1 = ~0ull, e2 = ~0ull;
        int k1 = -1, k2 = -1;
        int ao = 0, bo = 0, so = 0, xi = 0;   // the state before the move (recorded if it changes)
        if (has && sub == 0 && w.chg) {
            ao = w.a[m]; bo = w.b[m]; so = w.s1[m];
            xi = __ldcs(rowi + m);
        }
        if (has) {
            for (int k0 = sub; k0 < K; k0 += L * G) {
                int cv[L];
#pragma unroll
                for (int u = 0; u < L; u++) {
                    const int k = k0 + u * G;
                    cv[u] = k < K ? __ldg(cost + (size_t)s_open[k] * M_pad + m) : 0;
                }
#pragma unroll
                for (int u = 0; u < L; u++) {
                    const int k = k0 + u * G;
                    if (k < K) {
                        const unsigned long long e = ((unsigned long long)(unsigned)cv[u] << 32) | (unsigned)s_open[k];
                        if (e < e1) {
                            e2 = e1; k2 = k1;
                            e1 = e; k1 = k;
                        } else if (e < e2) {
                            e2 = e; k2 = k;
                        }
                    }
                }
            }
        }
        // every lane takes part (lanes without a mission carry empty pairs)
        for (int off = 1; off < G; off <<= 1) {
            const unsigned long long f1 = __shfl_xor_sync(full, e1, off), f2 = __shfl_xor_sync(full, e2, off);
            const int g1 = __shfl_xor_sync(full, k1, off), g2 = __shfl_xor_sync(full, k2, off);
            if (f1 < e1) {
                if (f2 < e1) { e2 = f2; k2 = g2; } else { e2 = e1; k2 = k1; }
                e1 = f1; k1 = g1;
            } else if (f1 < e2) {
                e2 = f1; k2 = g1;
            }
        }
        const bool lead = has && sub == 0;
        const int a = (int)(e1 >> 32);
        const int b = e2 == ~0ull ? kInf : (int)(e2 >> 32);
        if (lead) {
            w.a[m] = a; w.b[m] = b; w.s1[m] = (int16_t)k1; w.s2[m] = (int16_t)k2;
            terms(a, b, k1);
            if (w.chg) closed_column_terms(xi, a, b, k1, w.R, gic, gid, s_ic, s_id);
        }
        if (w.chg) record(lead && terms_changed(ao, bo, so, a, b, k1, w.R), m, ao, bo, so, a, b, k1);
    }
}

// One mission's rescan by its own thread, past the queue's capacity (out of
// line: a rare path kept out of the unrolled loop's registers).  Writes the
// mission's state; returns (a, b) and the best slot in k1.
static __device__ __noinline__ int2 refresh_scan_one(const TabuBuffers &w, const int32_t *__restrict__ cost, int m,
                                              const int *s_open, int &k1)
{
    int a, b, k2;
    scan_best_two(cost, w.M_pad, m, s_open, w.K, a, b, k1, k2);
    w.a[m] = a; w.b[m] = b; w.s1[m] = (int16_t)k1; w.s2[m] = (int16_t)k2;
    return make_int2(a, b);
}

// One run of extra terms of one row at one slot, added when the slot changes.
struct DeltaRun {
    int s, c;
    long long d;
};

__device__ __forceinline__ void delta_run_add(DeltaRun &run, int s, int c, int d, const TabuBuffers &w, int j)
{
    if (s != run.s) {
        if (run.s >= 0 && (run.c | (run.d != 0))) {
            atomicAdd(&w.extra_c[(size_t)run.s * w.B + j], run.c);
            atomicAdd(&w.extra_d[(size_t)run.s * w.B + j], (unsigned long long)run.d);
        }
        run.s = s;
        run.c = 0;
        run.d = 0;
    }
    run.c += c;
    run.d += d;
}

}  // namespace stg
