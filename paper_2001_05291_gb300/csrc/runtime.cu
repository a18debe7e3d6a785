// Host runtime of the staging engine: contexts, instances, device memory,
// validation and the Tabu driver loop behind the C ABI of include/stage.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "stage_internal.h"

using namespace stg;

#include "runtime_internal.h"

namespace stg_rt {

constexpr int kGraphIters = 16;   // iterations per captured graph of a single search

struct Guard {
    stage_ctx *c;
    bool locked;
    // every call is serialised on the context's mutex: the batch engine's
    // thread shares the context with the caller's thread
    explicit Guard(stage_ctx *ctx) : c(ctx), locked(ctx != nullptr)
    {
        if (locked) c->mu.lock();
    }
    ~Guard()
    {
        if (locked) c->mu.unlock();
    }
};

stage_status set_err(stage_ctx *c, stage_status code, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return set_err(c, STAGE_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

stage_status dev_alloc(stage_ctx *c, size_t bytes, DevBuf &out)
{
    bytes = round_up(bytes ? bytes : 256, 256);
    if (c->budget && c->used + bytes > c->budget)
        return set_err(c, STAGE_ERR_ADMISSION, "allocation of %zu bytes exceeds the HBM budget (%llu of %llu used)",
                       bytes, (unsigned long long)c->used, (unsigned long long)c->budget);
    void *p = nullptr;
    if (c->alloc) {
        p = c->alloc(bytes, c->alloc_user);
    } else if (c->pool) {
        // stream-ordered on the context stream: every user of the memory is
        // ordered after that stream (the callers synchronise it before another
        // stream touches the buffer)
        cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, c->pool, c->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    if (!p) return set_err(c, STAGE_ERR_NO_MEMORY, "device allocation of %zu bytes failed", bytes);
    out.p = p;
    out.bytes = bytes;
    c->used += bytes;
    return STAGE_OK;
}

void dev_free(stage_ctx *c, DevBuf &b)
{
    if (!b.p) return;
    // the pool's free is ordered on the context stream and does not wait for
    // the device (cudaFree would); callers free only memory no stream still uses
    if (c->free) c->free(b.p, b.bytes, c->alloc_user);
    else if (c->pool) cudaFreeAsync(b.p, c->stream);
    else cudaFree(b.p);
    c->used -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
}

cudaEvent_t get_event(stage_ctx *c)
{
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch through `f`, counting launches and (with STAGE_PROFILE) timing them.
template <class F>
cudaError_t timed(stage_ctx *c, const char *name, int n_kernels, F &&f)
{
    KernelStat &ks = c->stats[name];
    ks.launches += n_kernels;
    if (!(c->flags & STAGE_PROFILE)) return f();
    cudaEvent_t e0 = get_event(c), e1 = get_event(c);
    cudaEventRecord(e0, c->stream);
    cudaError_t r = f();
    cudaEventRecord(e1, c->stream);
    ks.pending.emplace_back(e0, e1);
    return r;
}

void fold_stats(stage_ctx *c)
{
    for (auto &kv : c->stats) {
        for (auto &pr : kv.second.pending) {
            float ms = 0.f;
            if (cudaEventSynchronize(pr.second) == cudaSuccess &&
                cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess)
                kv.second.ms += ms;
            c->event_pool.push_back(pr.first);
            c->event_pool.push_back(pr.second);
        }
        kv.second.pending.clear();
    }
}

Instance *find_inst(stage_ctx *c, stage_inst h)
{
    auto it = c->insts.find(h);
    return it == c->insts.end() ? nullptr : it->second;
}

void free_instance(stage_ctx *c, Instance *in)
{
    dev_free(c, in->mem_table);
    dev_free(c, in->mem_coords);
    dev_free(c, in->mem_ws);
    dev_free(c, in->mem_scratch);
    dev_free(c, in->mem_chg);
    dev_free(c, in->mem_costT);
    dev_free(c, in->mem_persist);
    dev_free(c, in->mem_rowsum);
    delete in;
}

stage_status ensure_scratch(stage_ctx *c, Instance *in, size_t bytes)
{
    if (in->mem_scratch.p && in->scratch_bytes >= bytes) return STAGE_OK;
    dev_free(c, in->mem_scratch);
    stage_status s = dev_alloc(c, bytes, in->mem_scratch);
    if (s != STAGE_OK) return s;
    in->scratch_bytes = in->mem_scratch.bytes;
    return STAGE_OK;
}

// Sub-allocation of one workspace chunk (256-byte aligned pieces).
struct Carver {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t n)
    {
        off = round_up(off, 256);
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += n * sizeof(T);
        return p;
    }
};

size_t carve_ws(char *base, int K, int B, int M_pad, int traj, TabuBuffers &tb)
{
    Carver cv{base};
    tb.a = cv.take<int32_t>(M_pad);
    tb.b = cv.take<int32_t>(M_pad);
    tb.s1 = cv.take<int16_t>(M_pad);
    tb.s2 = cv.take<int16_t>(M_pad);
    tb.v0 = cv.take<unsigned long long>(2);
    tb.loss_c = cv.take<unsigned long long>(K);
    tb.loss_d = cv.take<unsigned long long>(K);
    tb.gain_c = cv.take<int>(B);
    tb.gain_d = cv.take<unsigned long long>(B);
    tb.extra_c = cv.take<int>((size_t)K * B);
    tb.extra_d = cv.take<unsigned long long>((size_t)K * B);
    tb.open = cv.take<int32_t>(K);
    tb.best_open = cv.take<int32_t>(K);
    tb.cand = cv.take<int32_t>(B);
    tb.expiry = cv.take<int32_t>(B);
    tb.st = cv.take<TabuDevState>(1);
    tb.partials = cv.take<MoveKey>(2 * kSelectBlocks);
    tb.traj = cv.take<stage_move>(traj > 0 ? traj : 1);
    return round_up(cv.off, 256);
}

stage_status ensure_ws(stage_ctx *c, Instance *in, int K, int traj)
{
    if (in->mem_ws.p && in->ws_K == K && in->ws_traj >= traj && in->ws_M_pad == in->M_pad) return STAGE_OK;
    dev_free(c, in->mem_ws);
    TabuBuffers tb{};
    size_t bytes = carve_ws(nullptr, K, in->B, in->M_pad, traj, tb);
    stage_status s = dev_alloc(c, bytes, in->mem_ws);
    if (s != STAGE_OK) return s;
    carve_ws(static_cast<char *>(in->mem_ws.p), K, in->B, in->M_pad, traj, tb);
    tb.K = K;
    tb.B = in->B;
    tb.M = in->M;
    tb.M_pad = in->M_pad;
    in->tb = tb;
    in->ws_K = K;
    in->ws_traj = traj;
    in->ws_M_pad = in->M_pad;
    return STAGE_OK;
}

// Coordinate block of an instance with room for `cap` missions.
size_t carve_coords(char *base, int B, int cap, Instance *in)
{
    Carver cv{base};
    int2 *b = cv.take<int2>(B);
    int2 *p = cv.take<int2>(cap);
    int2 *d = cv.take<int2>(cap);
    int2 *pi = cv.take<int2>(cap);
    int2 *di = cv.take<int2>(cap);
    int32_t *pd = cv.take<int32_t>(cap);
    int32_t *perm = cv.take<int32_t>(cap);
    int32_t *inv = cv.take<int32_t>(cap);
    uint8_t *av = cv.take<uint8_t>(B);
    if (base && in) {
        in->base = b; in->pick = p; in->drop = d; in->pick_in = pi; in->drop_in = di;
        in->pd = pd; in->perm = perm; in->inv = inv; in->avail = av;
    }
    return round_up(cv.off, 256);
}

stage_status check_placement(stage_ctx *c, Instance *in, const int32_t *open, int K)
{
    if (!open) return set_err(c, STAGE_ERR_INVALID_ARG, "placement pointer is NULL");
    if (K < 1 || K > in->B || K > STAGE_MAX_K)
        return set_err(c, STAGE_ERR_INVALID_ARG, "K=%d outside [1, min(B=%d, %d)]", K, in->B, STAGE_MAX_K);
    std::vector<uint8_t> seen(in->B, 0);
    for (int k = 0; k < K; k++) {
        int o = open[k];
        if (o < 0 || o >= in->B) return set_err(c, STAGE_ERR_INVALID_ARG, "base id %d out of range", o);
        if (seen[o]) return set_err(c, STAGE_ERR_INVALID_ARG, "base %d appears twice in the placement", o);
        if (!in->h_avail[o]) return set_err(c, STAGE_ERR_INVALID_ARG, "base %d is unavailable", o);
        seen[o] = 1;
    }
    return STAGE_OK;
}

// The ranking's checks of K and its row sums (Alg. 1), queued on the
// context's stream (kept with the instance once computed, until an update).
stage_status rank_sums(stage_ctx *c, Instance *in, int K)
{
    if (K < 1 || K > in->B || K > STAGE_MAX_K)
        return set_err(c, STAGE_ERR_INVALID_ARG, "K=%d outside [1, min(B=%d, %d)]", K, in->B, STAGE_MAX_K);
    if (K > in->n_avail)
        return set_err(c, STAGE_ERR_INVALID_ARG, "K=%d exceeds the %d available bases", K, in->n_avail);
    if (!in->rowsum_ok) {
        stage_status s;
        if (!in->mem_rowsum.p || in->mem_rowsum.bytes < (size_t)in->B * 8) {
            dev_free(c, in->mem_rowsum);
            s = dev_alloc(c, (size_t)in->B * 8, in->mem_rowsum);
            if (s != STAGE_OK) return s;
        }
        auto *S = static_cast<unsigned long long *>(in->mem_rowsum.p);
        CK(cudaMemsetAsync(S, 0, (size_t)in->B * 8, c->stream));
        CK(timed(c, "rowsum", 1, [&] { return launch_rowsum(in->cost, in->B, in->M, in->M_pad, S, c->stream); }));
        in->rowsum_ok = true;
    }
    return STAGE_OK;
}

// The ranking (Alg. 1) queued on the context's stream: the row sums, the K
// smallest, their ids copied to out_open (host memory; pinned memory is
// filled when the stream gets there, pageable memory before this returns)
// and, if asked, the sums.
stage_status rank_queue(stage_ctx *c, Instance *in, int K, int32_t *out_open, int64_t *out_rowsum)
{
    stage_status s = rank_sums(c, in, K);
    if (s != STAGE_OK) return s;
    s = ensure_scratch(c, in, round_up((size_t)K * 4, 256));
    if (s != STAGE_OK) return s;
    auto *d_open = static_cast<int32_t *>(in->mem_scratch.p);
    const auto *S = static_cast<const unsigned long long *>(in->mem_rowsum.p);
    CK(timed(c, "topk", 1, [&] { return launch_topk(S, in->avail, in->B, K, d_open, c->stream); }));
    CK(cudaMemcpyAsync(out_open, d_open, (size_t)K * 4, cudaMemcpyDeviceToHost, c->stream));
    if (out_rowsum)
        CK(cudaMemcpyAsync(out_rowsum, S, (size_t)in->B * 8, cudaMemcpyDeviceToHost, c->stream));
    return STAGE_OK;
}

stage_status do_rank(stage_ctx *c, Instance *in, int K, int32_t *out_open, int64_t *out_rowsum)
{
    stage_status s = rank_queue(c, in, K, out_open, out_rowsum);
    if (s != STAGE_OK) return s;
    CK(cudaStreamSynchronize(c->stream));
    return STAGE_OK;
}

// Set up the workspace for placement `open` (host ids), zero the accumulators,
// and run the per-mission initialisation.  Returns the number of candidates.
// sync = false: return without waiting for the copies and kernels it queued
// (its host arrays are pageable, and a copy from pageable host memory is
// staged before cudaMemcpyAsync returns, so they may go out of scope).
stage_status setup_search(stage_ctx *c, Instance *in, const int32_t *open, int K, int R,
                          int traj_cap, int tenure, int accept_worsening, int t0,
                          const int32_t *expiry_in, int *out_nC, bool sync)
{
    stage_status s = ensure_ws(c, in, K, traj_cap);
    if (s != STAGE_OK) return s;
    TabuBuffers &tb = in->tb;
    tb.R = R;
    std::vector<uint8_t> is_open(in->B, 0);
    for (int k = 0; k < K; k++) is_open[open[k]] = 1;
    std::vector<int32_t> cand;
    cand.reserve(in->B);
    for (int b = 0; b < in->B; b++)
        if (in->h_avail[b] && !is_open[b]) cand.push_back(b);
    const int nC = (int)cand.size();
    TabuDevState st{};
    st.t = t0;
    st.tenure = tenure;
    st.accept_worsening = accept_worsening;
    st.nC = nC;
    st.traj_cap = traj_cap;
    st.best_iter = -1;
    st.t_end = t0 + traj_cap;
    std::vector<int32_t> expiry(in->B, 0);
    if (expiry_in) std::copy(expiry_in, expiry_in + in->B, expiry.begin());
    CK(cudaMemcpyAsync(tb.open, open, (size_t)K * 4, cudaMemcpyHostToDevice, c->stream));
    if (nC) CK(cudaMemcpyAsync(tb.cand, cand.data(), (size_t)nC * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(tb.expiry, expiry.data(), (size_t)in->B * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(tb.st, &st, sizeof st, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(tb.v0, 0, 16, c->stream));
    CK(cudaMemsetAsync(tb.loss_c, 0, (size_t)K * 8, c->stream));
    CK(cudaMemsetAsync(tb.loss_d, 0, (size_t)K * 8, c->stream));
    CK(cudaMemsetAsync(tb.gain_c, 0, (size_t)in->B * 4, c->stream));
    CK(cudaMemsetAsync(tb.gain_d, 0, (size_t)in->B * 8, c->stream));
    CK(cudaMemsetAsync(tb.extra_c, 0, (size_t)K * in->B * 4, c->stream));
    CK(cudaMemsetAsync(tb.extra_d, 0, (size_t)K * in->B * 8, c->stream));
    CK(timed(c, "init", 1, [&] { return launch_init(tb, in->cost, c->stream); }));
    if (sync) CK(cudaStreamSynchronize(c->stream));
    *out_nC = nC;
    return STAGE_OK;
}

std::vector<int32_t> spatial_order(const std::vector<int2> &xy, int ld);

stage_status ensure_costT(stage_ctx *c, Instance *in);

// The change records and the mission-major copy for a search on `in`, set in
// tw; false (and tw unchanged) when there is no room for them (the context's
// HBM budget): the search then takes the full pass.
bool use_incremental(stage_ctx *c, Instance *in, TabuBuffers &tw)
{
    const size_t need = (size_t)in->M_pad * 2 * sizeof(int4);
    if (!in->mem_chg.p || in->mem_chg.bytes < need) {
        dev_free(c, in->mem_chg);
        if (dev_alloc(c, need, in->mem_chg) != STAGE_OK) {
            set_err(c, STAGE_OK, "");   // a refused allocation here is not an error of the search
            return false;
        }
    }
    if (ensure_costT(c, in) != STAGE_OK) {
        set_err(c, STAGE_OK, "");
        return false;
    }
    tw.chg = static_cast<int4 *>(in->mem_chg.p);
    tw.costT = static_cast<const int32_t *>(in->mem_costT.p);
    tw.border = tw.costT + (size_t)in->M_pad * in->ldT;
    tw.cellmin = tw.border + in->ldT;
    tw.ldT = in->ldT;
    return true;
}

// The instance's mission-major copy with its position order and cell minima
// (built once per table by a tiled transpose when the load did not build it).
// STAGE_ERR_NO_MEMORY / STAGE_ERR_ADMISSION when there is no room for it.
stage_status ensure_costT(stage_ctx *c, Instance *in)
{
    if (in->costT_ok) return STAGE_OK;
    const int ldT = table_ldT(in->B);
    const size_t needT = costT_bytes(in->M_pad, ldT);
    if (!in->mem_costT.p || in->mem_costT.bytes < needT) {
        dev_free(c, in->mem_costT);
        stage_status s = dev_alloc(c, needT, in->mem_costT);
        if (s != STAGE_OK) return s;
    }
    // bases in Morton order of their coordinates (either metric: planar
    // metres or latitude / longitude), so that bases near one another take
    // neighbouring positions
    std::vector<int2> bxy(in->B);
    CK(cudaMemcpyAsync(bxy.data(), in->base, (size_t)in->B * sizeof(int2), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::vector<int32_t> border = spatial_order(bxy, ldT);
    int32_t *costT = static_cast<int32_t *>(in->mem_costT.p);
    int32_t *d_border = costT + (size_t)in->M_pad * ldT;
    int32_t *d_cellmin = d_border + ldT;
    CK(cudaMemcpyAsync(d_border, border.data(), (size_t)ldT * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    CK(timed(c, "transpose", 1, [&] {
        return launch_transpose_table(in->cost, in->B, in->M_pad, d_border, costT, d_cellmin, c->stream);
    }));
    CK(cudaStreamSynchronize(c->stream));   // the host order vector goes out of scope
    in->ldT = ldT;
    in->costT_ok = true;
    return STAGE_OK;
}

// A15 (reading): every open base of `open` that the instance no longer has
// available is closed by a forced move, the unavailable ones in ascending id:
// it opens the available closed base j with the best objective of the swap
// (a4: F(O - i + j) by covered desc, distance asc, then j asc), tabu ignored.
// A forced move takes no iteration; both bases become tabu for the next
// `tenure` iterations from t (expiry = t + tenure).  Each move evaluates the
// whole swap neighbourhood of the current placement once on the device.
stage_status forced_moves(stage_ctx *c, Instance *in, int32_t *open, int K, int R, int t, int tenure,
                          int32_t *expiry, int *n_forced)
{
    *n_forced = 0;
    const int B = in->B;
    const size_t n = (size_t)K * B;
    std::vector<long long> cov, dist;
    for (;;) {
        int k_out = -1;
        for (int k = 0; k < K; k++)
            if (!in->h_avail[open[k]] && (k_out < 0 || open[k] < open[k_out])) k_out = k;
        if (k_out < 0) return STAGE_OK;
        int nC = 0;
        stage_status s = setup_search(c, in, open, K, R, 0, 0, 1, 0, nullptr, &nC);
        if (s != STAGE_OK) return s;
        s = ensure_scratch(c, in, 2 * round_up(n * 8, 256));
        if (s != STAGE_OK) return s;
        auto *oc = static_cast<long long *>(in->mem_scratch.p);
        auto *od = reinterpret_cast<long long *>(static_cast<char *>(in->mem_scratch.p) + round_up(n * 8, 256));
        CK(cudaMemsetAsync(oc, 0xff, n * 8, c->stream));
        CK(cudaMemsetAsync(od, 0xff, n * 8, c->stream));
        CK(timed(c, "swap_eval", 1, [&] { return launch_swap_eval(in->tb, in->cost, nC, 1, c->stream); }));
        CK(launch_swap_table(in->tb, nC, oc, od, c->stream));
        cov.resize(B);
        dist.resize(B);
        CK(cudaMemcpyAsync(cov.data(), oc + (size_t)k_out * B, (size_t)B * 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(dist.data(), od + (size_t)k_out * B, (size_t)B * 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        int jb = -1;
        for (int j = 0; j < B; j++) {
            if (cov[j] < 0) continue;   // open or unavailable
            if (jb < 0 || cov[j] > cov[jb] || (cov[j] == cov[jb] && dist[j] < dist[jb])) jb = j;
        }
        if (jb < 0) return set_err(c, STAGE_ERR_INVALID_ARG, "no available closed base for a forced move");
        const int i = open[k_out];
        open[k_out] = jb;
        expiry[i] = expiry[jb] = t + tenure;
        *n_forced += 1;
    }
}

// Time the swap pass for each candidate missions-per-block and record the
// fastest for this shape bucket.  Runs on a scratch search state that is
// discarded (every search sets its state up afresh).
stage_status autotune_shape(stage_ctx *c, Instance *in, const int32_t *open, int K, int R, int *out_seg)
{
    std::vector<int32_t> start(K);
    if (open) {
        stage_status s = check_placement(c, in, open, K);
        if (s != STAGE_OK) return s;
        std::copy(open, open + K, start.begin());
    } else {
        stage_status s = do_rank(c, in, K, start.data(), nullptr);
        if (s != STAGE_OK) return s;
    }
    int nC = 0;
    stage_status s = setup_search(c, in, start.data(), K, R, 0, 0, 1, 0, nullptr, &nC);
    if (s != STAGE_OK) return s;
    if (nC == 0 || K > 256) {
        if (out_seg) *out_seg = swap_segment_heuristic(in->M_pad, nC);
        return STAGE_OK;
    }
    cudaEvent_t e0 = get_event(c), e1 = get_event(c);
    float best_ms = 0.f;
    int best = 0;
    for (int seg = 1024; seg <= 16384; seg <<= 1) {
        if (seg > 1024 && (seg >> 1) >= in->M_pad) break;   // one block already covers every mission
        CK(launch_swap_direct_seg(in->tb, in->cost, nC, seg, c->stream));
        CK(cudaEventRecord(e0, c->stream));
        for (int r = 0; r < 3; r++) CK(launch_swap_direct_seg(in->tb, in->cost, nC, seg, c->stream));
        CK(cudaEventRecord(e1, c->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (!best || ms < best_ms) {
            best_ms = ms;
            best = seg;
        }
    }
    c->event_pool.push_back(e0);
    c->event_pool.push_back(e1);
    c->stats["autotune"].launches += 1;
    swap_segment_record(in->M_pad, nC, K, best);
    if (out_seg) *out_seg = best;
    return STAGE_OK;
}

// Positions of the bases in the mission-major table copy: Morton order of
// their coordinates (16 bits per axis over the bounding box), ties by id;
// positions past B hold -1.
std::vector<int32_t> spatial_order(const std::vector<int2> &xy, int ld)
{
    const int B = (int)xy.size();
    long long x0 = LLONG_MAX, y0 = LLONG_MAX, x1 = LLONG_MIN, y1 = LLONG_MIN;
    for (const int2 &q : xy) {
        x0 = std::min<long long>(x0, q.x); x1 = std::max<long long>(x1, q.x);
        y0 = std::min<long long>(y0, q.y); y1 = std::max<long long>(y1, q.y);
    }
    auto spread16 = [](uint32_t v) {
        v &= 0xffffu;
        v = (v | (v << 8)) & 0x00ff00ffu;
        v = (v | (v << 4)) & 0x0f0f0f0fu;
        v = (v | (v << 2)) & 0x33333333u;
        v = (v | (v << 1)) & 0x55555555u;
        return v;
    };
    std::vector<std::pair<uint32_t, int32_t>> key(B);
    for (int b = 0; b < B; b++) {
        const uint32_t qx = (uint32_t)(((long long)xy[b].x - x0) * 65535 / std::max(1ll, x1 - x0));
        const uint32_t qy = (uint32_t)(((long long)xy[b].y - y0) * 65535 / std::max(1ll, y1 - y0));
        key[b] = {spread16(qx) | (spread16(qy) << 1), b};
    }
    std::sort(key.begin(), key.end());
    std::vector<int32_t> order(ld, -1);
    for (int p = 0; p < B; p++) order[p] = key[p].second;
    return order;
}

// The start of one Tabu search: the parameters checked, the start placement
// (given, resumed or ranked), the workspace set up and initialised for it,
// the resumed best so far restored (t0 and nC out).  ranked (nullable): the
// ranking's start placement, already computed; sync = false: return with the
// set-up still queued on the stream (setup_search).
stage_status tabu_prepare(stage_ctx *c, Instance *in, const stage_tabu_params *p, int *out_t0, int *out_nC,
                          const int32_t *ranked = nullptr, bool sync = true)
{
    if (!p) return set_err(c, STAGE_ERR_INVALID_ARG, "params is NULL");
    const int K = p->K;
    if (K < 1 || K > in->B || K > STAGE_MAX_K)
        return set_err(c, STAGE_ERR_INVALID_ARG, "K=%d outside [1, min(B=%d, %d)]", K, in->B, STAGE_MAX_K);
    if (K > in->n_avail)
        return set_err(c, STAGE_ERR_INVALID_ARG, "K=%d exceeds the %d available bases", K, in->n_avail);
    if (p->R < 0 || p->R == INT32_MAX)
        return set_err(c, STAGE_ERR_OUT_OF_RANGE, "R=%d outside [0, INT32_MAX)", p->R);
    if (p->iters < 0 || p->tenure < 0)
        return set_err(c, STAGE_ERR_INVALID_ARG, "iters and tenure must be >= 0");
    std::vector<int32_t> start(K);
    const stage_tabu_state *rs = p->resume;
    if (rs) {
        if (!rs->open || !rs->best_open || !rs->tabu_expiry || rs->t < 0)
            return set_err(c, STAGE_ERR_INVALID_ARG, "resume state is incomplete");
        stage_status s = check_placement(c, in, rs->open, K);
        if (s != STAGE_OK) return s;
        s = check_placement(c, in, rs->best_open, K);
        if (s != STAGE_OK) return s;
        std::copy(rs->open, rs->open + K, start.begin());
    } else if (p->start_open) {
        stage_status s = check_placement(c, in, p->start_open, K);
        if (s != STAGE_OK) return s;
        std::copy(p->start_open, p->start_open + K, start.begin());
    } else if (ranked) {
        std::copy(ranked, ranked + K, start.begin());
    } else {
        stage_status s = do_rank(c, in, K, start.data(), nullptr);
        if (s != STAGE_OK) return s;
    }
    const int iters = p->iters;
    const int t0 = rs ? rs->t : 0;
    if (c->flags & STAGE_AUTOTUNE) {
        int nc0 = 0;
        for (int b = 0; b < in->B; b++) nc0 += in->h_avail[b];
        nc0 -= K;
        if (!swap_segment_known(in->M_pad, nc0, K)) {
            stage_status s = autotune_shape(c, in, start.data(), K, p->R, nullptr);
            if (s != STAGE_OK) return s;
        }
    }
    int nC = 0;
    stage_status s = setup_search(c, in, start.data(), K, p->R, iters, p->tenure,
                                  p->accept_worsening ? 1 : 0, t0, rs ? rs->tabu_expiry : nullptr, &nC,
                                  sync || rs);
    if (s != STAGE_OK) return s;
    TabuBuffers &tb = in->tb;
    if (rs) {
        TabuDevState st{};
        CK(cudaMemcpy(&st, tb.st, sizeof st, cudaMemcpyDeviceToHost));
        st.best_cov = rs->best_cov;
        st.best_dist = rs->best_dist;
        st.best_iter = rs->best_iter;
        CK(cudaMemcpyAsync(tb.st, &st, sizeof st, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(tb.best_open, rs->best_open, (size_t)K * 4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    CK(timed(c, "begin", 1, [&] { return launch_begin(tb, rs ? 1 : 0, c->stream); }));
    *out_t0 = t0;
    *out_nC = nC;
    return STAGE_OK;
}

stage_status tabu_result(stage_ctx *c, const stage_tabu_params *p, bool count_records, const TabuDevState &st,
                         const int32_t *fin_in, const int32_t *best_in, const int32_t *expiry_in, int B,
                         stage_tabu_result *res);

// The end of one Tabu search: the device's error word checked, the
// trajectory and the result (best and final placements, end state) read back;
// exp_* (nullable) receive the per-mission best / second-best state.
stage_status tabu_finish(stage_ctx *c, Instance *in, const stage_tabu_params *p, bool count_records,
                         stage_tabu_result *res, stage_move *traj, int32_t *exp_a, int32_t *exp_b,
                         int32_t *exp_b1, int32_t *exp_b2)
{
    const int K = p->K, iters = p->iters;
    TabuBuffers &tb = in->tb;
    stage_status s = STAGE_OK;
    if (exp_a) {
        size_t per = round_up((size_t)in->M * 4, 256);
        s = ensure_scratch(c, in, 4 * per);
        if (s != STAGE_OK) return s;
        char *sc = static_cast<char *>(in->mem_scratch.p);
        auto *da = reinterpret_cast<int32_t *>(sc);
        auto *db = reinterpret_cast<int32_t *>(sc + per);
        auto *db1 = reinterpret_cast<int32_t *>(sc + 2 * per);
        auto *db2 = reinterpret_cast<int32_t *>(sc + 3 * per);
        CK(launch_export_best_two(tb, in->perm, da, db, db1, db2, c->stream));
        CK(cudaMemcpyAsync(exp_a, da, (size_t)in->M * 4, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(exp_b, db, (size_t)in->M * 4, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(exp_b1, db1, (size_t)in->M * 4, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaMemcpyAsync(exp_b2, db2, (size_t)in->M * 4, cudaMemcpyDeviceToHost, c->stream));
    }
    TabuDevState st{};
    std::vector<int32_t> fin(K), best(K), expiry(in->B);
    CK(cudaMemcpyAsync(&st, tb.st, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(fin.data(), tb.open, (size_t)K * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(best.data(), tb.best_open, (size_t)K * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(expiry.data(), tb.expiry, (size_t)in->B * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int n = std::min(st.n_moves, iters);
    if (traj && n > 0 && !st.err)
        CK(cudaMemcpy(traj, tb.traj, (size_t)n * sizeof(stage_move), cudaMemcpyDeviceToHost));
    return tabu_result(c, p, count_records, st, fin.data(), best.data(), expiry.data(), in->B, res);
}

// A search's result from host copies of its end state, placement, best
// placement and expiries (the trajectory already copied): the device's error
// word checked, the result and end state filled in.
stage_status tabu_result(stage_ctx *c, const stage_tabu_params *p, bool count_records, const TabuDevState &st,
                         const int32_t *fin_in, const int32_t *best_in, const int32_t *expiry_in, int B,
                         stage_tabu_result *res)
{
    const int K = p->K;
    if (st.err & kErrPipelineTimeout)
        return set_err(c, STAGE_ERR_TIMEOUT, "a device-side wait gave up after %lld polls at iteration %d",
                       (long long)c->spin_limit, st.t);
    if (st.err)
        return set_err(c, STAGE_ERR_INTERNAL, "device self-check failed (code %d) at iteration %d", st.err, st.t);
    if (count_records) {
        // missions the incremental passes took (traffic accounting)
        std::lock_guard<std::recursive_mutex> g(c->mu);
        c->stats["swap_delta_records"].launches += st.chg_total + st.chg_n;
    }
    if (res) {
        std::vector<int32_t> fin(fin_in, fin_in + K), best(best_in, best_in + K);
        res->n_moves = st.n_moves;
        res->best_iter = st.best_iter;
        res->best_cov = st.best_cov;
        res->best_dist = st.best_dist;
        res->final_cov = st.cur_cov;
        res->final_dist = st.cur_dist;
        if (res->end_state) {
            stage_tabu_state *es = res->end_state;
            es->t = st.t;
            es->best_iter = st.best_iter;
            es->best_cov = st.best_cov;
            es->best_dist = st.best_dist;
            if (es->open) std::copy(fin.begin(), fin.end(), es->open);
            if (es->best_open) std::copy(best.begin(), best.end(), es->best_open);
            if (es->tabu_expiry) std::copy(expiry_in, expiry_in + B, es->tabu_expiry);
        }
        std::sort(fin.begin(), fin.end());
        std::sort(best.begin(), best.end());
        if (res->best_open) std::copy(best.begin(), best.end(), res->best_open);
        if (res->final_open) std::copy(fin.begin(), fin.end(), res->final_open);
    }
    return STAGE_OK;
}

stage_status run_tabu(stage_ctx *c, Instance *in, const stage_tabu_params *p,
                      stage_tabu_result *res, stage_move *traj, int32_t *exp_a, int32_t *exp_b,
                      int32_t *exp_b1, int32_t *exp_b2)
{
    int t0 = 0, nC = 0;
    stage_status s = tabu_prepare(c, in, p, &t0, &nC);
    if (s != STAGE_OK) return s;
    const int K = p->K, iters = p->iters;
    TabuBuffers &tb = in->tb;
    volatile int *done_flag = static_cast<volatile int *>(c->pinned);
    const bool profiling = (c->flags & STAGE_PROFILE) != 0;
    // Incremental neighbourhood: one full pass, then each iteration selects
    // and applies a move, refreshes the per-mission state (recording the
    // missions whose terms changed, rebuilding the closed base's column) and
    // updates the other columns from those records.  STAGE_FULL_PASS: a full
    // pass every iteration instead.  The whole loop runs in one cooperative
    // launch where the shape fits and the device can hold the grid (not with
    // STAGE_NO_PERSIST, nor for the test-support export of the per-mission
    // state, which the persistent search keeps exact only up to R); that form
    // is taken whenever it can run.  The per-iteration launches of the
    // incremental form are taken only for tables well beyond the L2 cache: an
    // L2-resident table is streamed faster than their scattered columns.
    TabuBuffers tw = tb;   // the buffers of this run's multi-kernel launches
    const bool multi = nC > 0 && iters > 0 && !(tabu_resident_fits(K, in->B, in->M_pad, nC)) &&
                       !(tabu_small_fits(nC, in->M_pad, K));
    const bool persist_ok = multi && !(c->flags & STAGE_NO_PERSIST) && tw.mask == nullptr && exp_a == nullptr;
    const int pgrid = persist_ok ? persist_grid(K, in->B, table_ldT(in->B), in->M_pad) : 0;
    bool inc = !(c->flags & STAGE_FULL_PASS) && swap_delta_fits(K) &&
               ((c->flags & STAGE_INCREMENTAL) || pgrid > 0 ||
                (size_t)nC * in->M_pad * sizeof(int32_t) >= kIncrementalMinTableBytes);
    bool persist = inc && pgrid > 0;
    if (inc) inc = use_incremental(c, in, tw);
    // one Tabu iteration of the multi-kernel path
    auto step = [&](bool time_each) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        auto run = [&](const char *nm, auto &&f) {
            if (e != cudaSuccess) return;
            e = time_each ? timed(c, nm, 1, f) : f();
        };
        if (!inc) run("swap_eval", [&] { return launch_swap_eval(tw, in->cost, nC, 0, c->stream); });
        run("select", [&] { return launch_select(tw, nC, c->stream); });
        run("refresh", [&] { return launch_refresh(tw, in->cost, c->stream); });
        if (inc) run("swap_delta", [&] { return launch_swap_delta(tw, c->stream); });
        return e;
    };
    if (!inc) persist = false;   // no room for the incremental form's buffers
    if (persist) {
        const size_t need = persist_scratch_bytes(K, pgrid, in->M_pad);
        if (pgrid < 1) {
            persist = false;
        } else if (!in->mem_persist.p || in->mem_persist.bytes < need) {
            dev_free(c, in->mem_persist);
            if (dev_alloc(c, need, in->mem_persist) != STAGE_OK) {
                persist = false;
                set_err(c, STAGE_OK, "");   // a refused allocation here is not an error of the search
            }
        }
    }
    if (inc && multi) CK(timed(c, "swap_eval", 1, [&] { return launch_swap_eval(tw, in->cost, nC, 0, c->stream); }));
    if (nC > 0 && iters > 0 && tabu_resident_fits(K, in->B, in->M_pad, nC)) {
        // small instance: the whole search in one block, its arrays in shared memory
        CK(timed(c, "tabu_small", 1, [&] { return launch_tabu_resident(tb, in->cost, nC, iters, c->stream); }));
    } else if (nC > 0 && iters > 0 && tabu_small_fits(nC, in->M_pad, K)) {
        // small instance: the whole search in one resident block
        CK(timed(c, "tabu_small", 1, [&] { return launch_tabu_small(tb, in->cost, iters, c->stream); }));
    } else if (persist) {
        CK(timed(c, "persist", 1, [&] {
            return launch_tabu_persist(tw, in->cost, in->mem_persist.p, pgrid, c->spin_limit, c->stream);
        }));
        // the records over the search (the traffic accounting), the
        // (record, base) pairs with a term and the warps' passes over them
        long long info[6] = {0, 0, 0, 0, 0, 0};
        CK(cudaMemcpyAsync(info, static_cast<const char *>(in->mem_persist.p) + persist_info_offset(K), sizeof info,
                           cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        {
            std::lock_guard<std::recursive_mutex> g(c->mu);
            c->stats["swap_delta_records"].launches += info[1];
            c->stats["persist_ctas"].launches = info[0];
            c->stats["swap_delta_term_pairs"].launches += info[2];
            c->stats["swap_delta_warp_passes"].launches += info[3];
            c->stats["swap_delta_run_writes"].launches += info[4];
            c->stats["swap_delta_cells_read"].launches += info[5];
        }
        if (profiling) {
            // the kernel's own clocks: per step the mean over the CTAs and the
            // slowest CTA ("_max"), with the moves applied as the count
            std::vector<long long> clk((size_t)pgrid * kPersistClocks);
            const char *base = static_cast<const char *>(in->mem_persist.p);
            TabuDevState sd{};
            CK(cudaMemcpyAsync(&sd, tb.st, sizeof sd, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(clk.data(), base + persist_clock_offset(K, pgrid, in->M_pad),
                               clk.size() * sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            const char *nm[kPersistClocks] = {"persist_move",          "persist_refresh",
                                              "persist_wait_refresh",  "persist_update",
                                              "persist_wait_update",   "persist_select",
                                              "persist_wait_select",   "persist_refresh_loop",
                                              "persist_refresh_rescan", "persist_refresh_sums",
                                              "persist_update_issue",  "persist_update_wait",
                                              "persist_update_compute"};
            const long long moves = sd.t - t0;
            for (int k = 0; k < kPersistClocks; k++) {
                double sum = 0.0, mx = 0.0;
                for (int g = 0; g < pgrid; g++) {
                    const double v = clk[(size_t)g * kPersistClocks + k] * 1e-6;
                    sum += v;
                    mx = std::max(mx, v);
                }
                KernelStat &mean = c->stats[nm[k]];
                mean.launches += moves;
                mean.ms += sum / pgrid;
                KernelStat &top = c->stats[std::string(nm[k]) + "_max"];
                top.launches += moves;
                top.ms += mx;
            }
        }
    } else if (nC > 0 && iters >= kGraphIters && !profiling) {
        // replay kGraphIters iterations at a time from a CUDA graph
        cudaGraph_t gr = nullptr;
        cudaGraphExec_t ge = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        for (int k = 0; e == cudaSuccess && k < kGraphIters; k++) e = step(false);
        cudaError_t e2 = cudaStreamEndCapture(c->stream, &gr);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, gr, 0);
        if (gr) cudaGraphDestroy(gr);
        if (e != cudaSuccess) {
            if (ge) cudaGraphExecDestroy(ge);
            return set_err(c, STAGE_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
        }
        int it = 0;
        for (; it + kGraphIters <= iters; it += kGraphIters) {
            if (inc) {
                for (const char *nm : {"select", "refresh", "swap_delta"})
                    c->stats[nm].launches += kGraphIters;
            } else {
                for (const char *nm : {"swap_eval", "select", "refresh"}) c->stats[nm].launches += kGraphIters;
            }
            e = cudaGraphLaunch(ge, c->stream);
            if (e != cudaSuccess) break;
            if (!p->accept_worsening && ((it / kGraphIters) & 1)) {
                e = cudaMemcpyAsync(c->pinned, &tb.st->done, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
                if (e != cudaSuccess || *done_flag) break;
            }
        }
        cudaGraphExecDestroy(ge);
        CK(e);
        // the remaining iterations (iterations past the budget do nothing)
        for (; it < iters && !(!p->accept_worsening && *done_flag); it++) CK(step(true));
    } else {
        for (int it = 0; it < iters && nC > 0; it++) {
            CK(step(true));
            // the improving-only rule usually stops early: poll the device flag now and then
            if (!p->accept_worsening && (it & 31) == 31) {
                CK(cudaMemcpyAsync(c->pinned, &tb.st->done, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
                CK(cudaStreamSynchronize(c->stream));
                if (*done_flag) break;
            }
        }
    }
    return tabu_finish(c, in, p, inc && multi && !persist, res, traj, exp_a, exp_b, exp_b1, exp_b2);
}

// ----------------------------------------------------------- many searches, one launch
// Every search of a batch whose shape the persistent body takes runs inside
// one cooperative launch (k_tabu_batch), on a gang of CTAs sized by its
// estimated work; the others (no move to make, or a shape the body does not
// take) run alone afterwards.  Each search computes what stage_tabu_run
// computes for it.
namespace {

struct BatchItem {
    Instance *in = nullptr;
    int t0 = 0, nC = 0;
    bool fused = false;   // runs inside the batch launch
    int gang = 1;
    double us_per_iter = 0.0;   // estimated on one CTA (without the fixed part)
    TabuBuffers tw{};
};

}  // namespace

double persist_iter_us_estimate(const Instance *in, int K, int nC, double cov)
{
    const double M = in->M_pad, cells = 0.386 * table_ldT(in->B) / 32.0;
    const double records = 2.0 * cov * M / K;
    return (2.2 * M + records * (20.0 + 28.0 * cells) + 2.05 * K * nC) * 1e-3;
}

namespace {

// Estimated device time of one iteration of the persistent body on one CTA,
// beyond its fixed part, in us, before any measurement of the instance: 2.2 ns
// per mission (the refresh), 2 cov M / K records per move (the covered
// missions whose best or second-best base is the closed one; cov = the start
// placement's covered fraction) at 20 ns each plus 28 ns per cell of the row
// read (0.386 of the row's 32-position cells on average), 2.05 ns per swap
// (the selection).  The costs are the batched workload's measured per-CTA
// totals (512 searches on a GB300) over these counts.  Once an instance has
// run in a batch launch, its measured time replaces the estimate.
double batch_iter_us(const Instance *in, int K, int R, int nC, double cov)
{
    if (in->batch_K == K && in->batch_R == R && in->batch_version == in->version && in->batch_work_us > 0.0)
        return in->batch_work_us;
    return persist_iter_us_estimate(in, K, nC, cov);
}

constexpr double kBatchFixedUs = 5.0;    // an iteration's move, barriers and reductions on one CTA
constexpr double kBatchGangUs = 4.0;     // more per iteration once the search spans several CTAs

double batch_search_us(const BatchItem &it, int iters, int g)
{
    return iters * (kBatchFixedUs + (g > 1 ? kBatchGangUs : 0.0) + it.us_per_iter / g);
}

}  // namespace

// Placement of a batch's searches on P CTAs: search k takes gang[k] CTAs for
// work[k] (its estimated time on them); largest first by gang x time, each on
// the gang of CTAs that are free first, starting at the latest of their finish
// times.  lists[q]: CTA q's (search, rank) entries in placement order, so
// every CTA runs the searches in one global order; returns the latest finish.
double batch_place(int n, const double *work, const int *gang, int P, std::vector<std::vector<int2>> &lists,
                   std::vector<int> &order)
{
    order.resize(n);
    for (int k = 0; k < n; k++) order[k] = k;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        const double wa = work[a] * gang[a], wb = work[b] * gang[b];
        return wa != wb ? wa > wb : a < b;
    });
    std::vector<double> fin(P, 0.0);
    lists.assign(P, {});
    std::vector<int> idx(P);
    double makespan = 0.0;
    for (int pos = 0; pos < n; pos++) {
        const int k = order[pos], g = gang[k];
        for (int q = 0; q < P; q++) idx[q] = q;
        std::partial_sort(idx.begin(), idx.begin() + g, idx.end(), [&](int a, int b) {
            return fin[a] != fin[b] ? fin[a] < fin[b] : a < b;
        });
        double start = 0.0;
        for (int r = 0; r < g; r++) start = std::max(start, fin[idx[r]]);
        const double end = start + work[k];
        makespan = std::max(makespan, end);
        for (int r = 0; r < g; r++) {
            fin[idx[r]] = end;
            lists[idx[r]].push_back(make_int2(pos, r));   // pos: the search's place in the placement order
        }
    }
    return makespan;
}

// Pinned host staging of a batch call's copies, at least `bytes` (kept with
// the context; every copy into it has completed when a call returns).
static char *batch_staging(stage_ctx *c, size_t bytes)
{
    if (c->batch_pinned_bytes < bytes) {
        if (c->batch_pinned) cudaFreeHost(c->batch_pinned);
        c->batch_pinned = nullptr;
        c->batch_pinned_bytes = 0;
        if (cudaMallocHost(&c->batch_pinned, bytes) != cudaSuccess) {
            c->batch_pinned = nullptr;
            return nullptr;
        }
        c->batch_pinned_bytes = bytes;
    }
    return static_cast<char *>(c->batch_pinned);
}

stage_status run_tabu_batch(stage_ctx *c, int n, const stage_inst *hs, const stage_tabu_params *ps,
                            stage_tabu_result *res, stage_move *const *trajs)
{
    // host time of the call's phases (set-up, launch and read-back, results)
    auto host_ms = [t = std::chrono::steady_clock::now()]() mutable {
        const auto now = std::chrono::steady_clock::now();
        const double ms = std::chrono::duration<double, std::milli>(now - t).count();
        t = now;
        return ms;
    };
    std::vector<BatchItem> items(n);
    for (int i = 0; i < n; i++) {
        items[i].in = find_inst(c, hs[i]);
        if (!items[i].in) return set_err(c, STAGE_ERR_NOT_FOUND, "request %d: unknown instance %llu", i,
                                         (unsigned long long)hs[i]);
        for (int k = 0; k < i; k++)
            if (items[k].in == items[i].in)
                return set_err(c, STAGE_ERR_INVALID_ARG, "requests %d and %d name the same instance", k, i);
    }
    // 1. the ranking of every search that starts from it: the row sums an
    //    instance lacks, then every search's K smallest in one grouped launch
    //    and one read-back of the start placements to pinned staging, one wait
    // (an early return first waits for the work already queued, whose
    // buffers a later call may reallocate)
    auto fail = [&](stage_status s) {
        cudaStreamSynchronize(c->stream);
        return s;
    };
    std::vector<size_t> at_rank(n, 0);
    std::vector<int> ranked;   // the searches that start from the ranking
    size_t rank_bytes = 0, rank_blocks = 0;
    for (int i = 0; i < n; i++) {
        if (ps[i].resume || ps[i].start_open) continue;
        stage_status s = rank_sums(c, items[i].in, ps[i].K);
        if (s != STAGE_OK) return fail(s);
        ranked.push_back(i);
        at_rank[i] = rank_bytes;
        rank_bytes += round_up((size_t)ps[i].K * 4, 16);
        rank_blocks += topk_blocks(items[i].in->B);
    }
    // the staging: the start placements, then every search's V0 (phase 2)
    const size_t v0_at = round_up(rank_bytes, 16);
    const size_t bytes = v0_at + 16 * (size_t)n;
    char *stage = batch_staging(c, bytes);
    if (!stage)
        return fail(set_err(c, STAGE_ERR_NO_MEMORY, "no pinned host memory for the batch (%zu bytes)", bytes));
    if (!ranked.empty()) {
        const size_t off_map = round_up(ranked.size() * sizeof(TopkSlot), 256),
                     off_open = off_map + round_up(rank_blocks * sizeof(int2), 256);
        DevBuf rbuf;
        stage_status s = dev_alloc(c, off_open + rank_bytes, rbuf);
        if (s != STAGE_OK) return fail(s);
        char *d = static_cast<char *>(rbuf.p);
        std::vector<TopkSlot> ts(ranked.size());
        std::vector<int2> tmap;
        tmap.reserve(rank_blocks);
        for (size_t k = 0; k < ranked.size(); k++) {
            const int i = ranked[k];
            const Instance *in = items[i].in;
            ts[k] = TopkSlot{static_cast<const unsigned long long *>(in->mem_rowsum.p), in->avail,
                             reinterpret_cast<int32_t *>(d + off_open + at_rank[i]), in->B, ps[i].K};
            for (int b = 0; b < topk_blocks(in->B); b++) tmap.push_back(make_int2((int)k, b));
        }
        // (copies from pageable host memory are staged before they return)
        cudaError_t e = cudaMemcpyAsync(d, ts.data(), ts.size() * sizeof(TopkSlot), cudaMemcpyHostToDevice,
                                        c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d + off_map, tmap.data(), tmap.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                c->stream);
        if (e == cudaSuccess)
            e = timed(c, "topk", 1, [&] {
                return launch_topk_group(reinterpret_cast<const TopkSlot *>(d),
                                         reinterpret_cast<const int2 *>(d + off_map), (int)tmap.size(), c->stream);
            });
        if (e == cudaSuccess) e = cudaMemcpyAsync(stage, d + off_open, rank_bytes, cudaMemcpyDeviceToHost, c->stream);
        const cudaError_t se = cudaStreamSynchronize(c->stream);
        dev_free(c, rbuf);   // after the wait: the launch and the copy have read it
        if (e == cudaSuccess) e = se;
        if (e != cudaSuccess) return set_err(c, STAGE_ERR_CUDA, "batch ranking failed: %s", cudaGetErrorString(e));
    }
    const double rank_ms = host_ms();
    double prep_ms = 0.0;   // host time in the searches' set-up (the rest of phase 2: their full passes)
    // 2. the start of every search, queued (no wait per search); the full
    //    passes that start the incremental form, all in one grouped launch; the
    //    start placements' covered counts (the estimate of an unmeasured
    //    search), one read-back and one wait
    size_t smem = 0;
    std::vector<int> full;   // the searches the launch takes, each with its full pass
    for (int i = 0; i < n; i++) {
        BatchItem &it = items[i];
        Instance *in = it.in;
        const stage_tabu_params *p = &ps[i];
        const bool ranked = !p->resume && !p->start_open;
        const auto tp0 = std::chrono::steady_clock::now();
        stage_status s = tabu_prepare(c, in, p, &it.t0, &it.nC,
                                      ranked ? reinterpret_cast<const int32_t *>(stage + at_rank[i]) : nullptr, false);
        prep_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tp0).count();
        if (s != STAGE_OK) return fail(s);
        const int K = p->K, ldT = table_ldT(in->B);
        it.fused = it.nC > 0 && p->iters > 0 && persist_shape_ok(K, in->B, ldT) &&
                   !(c->flags & (STAGE_FULL_PASS | STAGE_NO_PERSIST));
        if (!it.fused) continue;
        it.tw = in->tb;
        if (!use_incremental(c, in, it.tw)) {
            it.fused = false;
            continue;
        }
        full.push_back(i);
        smem = std::max(smem, persist_search_smem(K, in->B, ldT));
    }
    {
        // every full pass in one grouped launch (the searches' descriptors and
        // its block map uploaded first), then every start's V0 gathered into
        // one read-back
        const int nf = (int)full.size();
        std::vector<int> mp(nf), nc(nf);
        for (int k = 0; k < nf; k++) {
            mp[k] = items[full[k]].in->M_pad;
            nc[k] = items[full[k]].nC;
        }
        const int common = group_common_segment(mp.data(), nc.data(), nf);
        std::vector<GroupSlot> gs(nf);
        std::vector<int2> map;
        size_t pass_smem = 0;
        for (int k = 0; k < nf; k++) {
            const BatchItem &it = items[full[k]];
            gs[k] = GroupSlot{};
            gs[k].w = it.tw;
            gs[k].cost = it.in->cost;
            gs[k].swap_blocks = group_swap_blocks(mp[k], nc[k], it.tw.K, common, &gs[k].swap_bx, &gs[k].swap_seg);
            for (int b = 0; b < gs[k].swap_blocks; b++) map.push_back(make_int2(k, b));
            pass_smem = std::max(pass_smem, swap_direct_smem(it.tw.K));
        }
        const size_t off_map = round_up(gs.size() * sizeof(GroupSlot), 256),
                     off_v0 = off_map + round_up(map.size() * sizeof(int2), 256);
        DevBuf gbuf;
        cudaError_t e = cudaSuccess;
        if (nf > 0) {
            stage_status s = dev_alloc(c, off_v0 + 16 * (size_t)nf, gbuf);
            if (s != STAGE_OK) return fail(s);
            char *d = static_cast<char *>(gbuf.p);
            // (copies from pageable host memory are staged before they return)
            e = cudaMemcpyAsync(d, gs.data(), gs.size() * sizeof(GroupSlot), cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d + off_map, map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                    c->stream);
            if (e == cudaSuccess)
                e = timed(c, "group_swap", 1, [&] {
                    return launch_group_swap(reinterpret_cast<const GroupSlot *>(d),
                                             reinterpret_cast<const int2 *>(d + off_map), (int)map.size(), pass_smem,
                                             c->stream);
                });
            if (e == cudaSuccess)
                e = launch_group_v0(reinterpret_cast<const GroupSlot *>(d), nf,
                                    reinterpret_cast<unsigned long long *>(d + off_v0), c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(stage + v0_at, d + off_v0, 16 * (size_t)nf, cudaMemcpyDeviceToHost, c->stream);
        }
        const cudaError_t se = cudaStreamSynchronize(c->stream);
        dev_free(c, gbuf);   // after the wait: the launch has read it
        if (e == cudaSuccess) e = se;
        if (e != cudaSuccess) return set_err(c, STAGE_ERR_CUDA, "batch set-up failed: %s", cudaGetErrorString(e));
    }
    double total_us = 0.0;
    for (size_t k = 0; k < full.size(); k++) {
        const int i = full[k];
        BatchItem &it = items[i];
        const unsigned long long covered = *reinterpret_cast<const unsigned long long *>(stage + v0_at + 16 * k);
        const double cov = it.in->M > 0 ? std::min(1.0, (double)covered / it.in->M) : 0.0;
        it.us_per_iter = batch_iter_us(it.in, ps[i].K, ps[i].R, it.nC, cov);
        total_us += batch_search_us(it, ps[i].iters, 1);
    }
    const int P = smem ? persist_batch_grid(smem) : 0;
    {
        // set-up: the rankings, the searches' set-up, their full passes and covered counts
        const double ms = host_ms();
        c->stats["batch_host_setup"].ms += rank_ms + ms;
        c->stats["batch_host_setup_rank"].ms += rank_ms;
        c->stats["batch_host_setup_prepare"].ms += prep_ms;
        c->stats["batch_host_setup_pass"].ms += ms - prep_ms;
    }
    std::vector<int> order;
    for (int i = 0; i < n; i++)
        if (items[i].fused) {
            if (P < 1) items[i].fused = false;
            else order.push_back(i);
        }
    stage_status first = STAGE_OK;
    if (!order.empty()) {
        // 3. gang sizes: the smallest power of two that brings a search under
        //    half of the ideal per-CTA time (at most the search's 32-mission
        //    chunks)
        const double ideal = total_us / P;
        for (int i : order) {
            BatchItem &it = items[i];
            const int gmax = std::min({persist_max_gang(), P, (int)((it.in->M_pad + 31) / 32)});
            int g = 1;
            while (g * 2 <= gmax && batch_search_us(it, ps[i].iters, g) > 0.5 * ideal) g *= 2;
            it.gang = g;
        }
        // placement (batch_place); `order` becomes the placement order, which
        // is also the order of the searches' arguments on the device
        const int ns = (int)order.size();
        std::vector<double> work(ns);
        std::vector<int> gangs(ns), place;
        for (int k = 0; k < ns; k++) {
            work[k] = batch_search_us(items[order[k]], ps[order[k]].iters, items[order[k]].gang);
            gangs[k] = items[order[k]].gang;
        }
        std::vector<std::vector<int2>> lists;
        batch_place(ns, work.data(), gangs.data(), P, lists, place);
        {
            std::vector<int> placed(ns);
            for (int pos = 0; pos < ns; pos++) placed[pos] = order[place[pos]];
            order = placed;
        }
        // per search its scratch and arguments; the schedule
        const size_t ab = persist_args_bytes();
        std::vector<unsigned char> h_args(ab * ns);
        for (int k = 0; k < ns; k++) {
            BatchItem &it = items[order[k]];
            Instance *in = it.in;
            const size_t need = persist_scratch_bytes(ps[order[k]].K, it.gang, in->M_pad);
            if (!in->mem_persist.p || in->mem_persist.bytes < need) {
                dev_free(c, in->mem_persist);
                stage_status s = dev_alloc(c, need, in->mem_persist);
                if (s != STAGE_OK) return s;
            }
            CK(persist_args_host(it.tw, in->cost, in->mem_persist.p, it.gang, c->spin_limit, c->stream,
                                 h_args.data() + ab * k));
        }
        std::vector<int2> h_sched;
        std::vector<int> h_off(P + 1, 0);
        for (int q = 0; q < P; q++) {
            h_off[q] = (int)h_sched.size();
            h_sched.insert(h_sched.end(), lists[q].begin(), lists[q].end());
        }
        h_off[P] = (int)h_sched.size();
        const size_t off_args = 0, off_sched = round_up(h_args.size(), 256),
                     off_off = off_sched + round_up(h_sched.size() * sizeof(int2), 256),
                     dbytes = off_off + round_up(h_off.size() * sizeof(int), 256);
        DevBuf buf;
        stage_status s = dev_alloc(c, dbytes, buf);
        if (s != STAGE_OK) return s;
        char *d = static_cast<char *>(buf.p);
        // (copies from pageable host memory are staged before they return)
        cudaError_t e = cudaMemcpyAsync(d + off_args, h_args.data(), h_args.size(), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d + off_sched, h_sched.data(), h_sched.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d + off_off, h_off.data(), h_off.size() * sizeof(int), cudaMemcpyHostToDevice,
                                c->stream);
        // every search's scratch readied, then the launch, timed by CUDA events
        // on its stream whether or not the context profiles (one launch per call)
        if (e == cudaSuccess) e = launch_batch_prep(d + off_args, ns, c->stream);
        cudaEvent_t ev0 = get_event(c), ev1 = get_event(c);
        if (e == cudaSuccess) e = cudaEventRecord(ev0, c->stream);
        if (e == cudaSuccess)
            e = launch_tabu_batch(d + off_args, reinterpret_cast<const int2 *>(d + off_sched),
                                  reinterpret_cast<const int *>(d + off_off), P, smem, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev1, c->stream);
        // 4. every search's clocks, end state, counters, placements, expiries
        //    and trajectory to pinned staging, one wait
        std::vector<size_t> at_clk(ns), at_st(ns), at_info(ns), at_open(ns), at_best(ns), at_exp(ns), at_traj(ns);
        size_t rb = 0;
        for (int k = 0; k < ns; k++) {
            const BatchItem &it = items[order[k]];
            const int K = ps[order[k]].K;
            at_clk[k] = rb; rb += round_up((size_t)it.gang * kPersistClocks * 8, 16);
            at_st[k] = rb; rb += round_up(sizeof(TabuDevState), 16);
            at_info[k] = rb; rb += 48;
            at_open[k] = rb; rb += round_up((size_t)K * 4, 16);
            at_best[k] = rb; rb += round_up((size_t)K * 4, 16);
            at_exp[k] = rb; rb += round_up((size_t)it.in->B * 4, 16);
            at_traj[k] = rb; rb += round_up((size_t)ps[order[k]].iters * sizeof(stage_move), 16);
        }
        if (e == cudaSuccess) {
            stage = batch_staging(c, rb);   // the earlier staging is consumed
            if (!stage) e = cudaErrorMemoryAllocation;
        }
        for (int k = 0; k < ns && e == cudaSuccess; k++) {
            const BatchItem &it = items[order[k]];
            const int K = ps[order[k]].K;
            const char *base = static_cast<const char *>(it.in->mem_persist.p);
            const TabuBuffers &tb = it.in->tb;
            auto cp = [&](size_t at, const void *src, size_t nb) {
                if (e == cudaSuccess) e = cudaMemcpyAsync(stage + at, src, nb, cudaMemcpyDeviceToHost, c->stream);
            };
            cp(at_clk[k], base + persist_clock_offset(K, it.gang, it.in->M_pad),
               (size_t)it.gang * kPersistClocks * 8);
            cp(at_st[k], tb.st, sizeof(TabuDevState));
            cp(at_info[k], base + persist_info_offset(K), 48);
            cp(at_open[k], tb.open, (size_t)K * 4);
            cp(at_best[k], tb.best_open, (size_t)K * 4);
            cp(at_exp[k], tb.expiry, (size_t)it.in->B * 4);
            if (trajs && trajs[order[k]] && ps[order[k]].iters > 0)
                cp(at_traj[k], tb.traj, (size_t)ps[order[k]].iters * sizeof(stage_move));
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        float kms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&kms, ev0, ev1);
        c->event_pool.push_back(ev0);
        c->event_pool.push_back(ev1);
        if (e != cudaSuccess) cudaStreamSynchronize(c->stream);   // nothing of this call left in flight
        dev_free(c, buf);
        CK(e);
        c->stats["batch_host_launch"].ms += host_ms();
        // Each search's measured work (its CTAs' time outside the waits, per
        // iteration) sizes its gang in the next batch; the batch's statistics:
        // every CTA's busy time (the sum of its searches' steps), each step's
        // total, the longest search, the records and cell pieces the updates
        // read; then each search's result.
        auto clk_of = [&](int k) { return reinterpret_cast<const long long *>(stage + at_clk[k]); };
        std::vector<double> busy(P, 0.0), step(7, 0.0);
        double est = 0.0, longest = 0.0;
        int longest_i = -1;
        long long records = 0, cells = 0, cellmin_bytes = 0, moves = 0, refresh_bytes = 0, select_bytes = 0;
        for (int k = 0; k < ns; k++) {
            BatchItem &it = items[order[k]];
            const stage_tabu_params &pk = ps[order[k]];
            const TabuDevState &sd = *reinterpret_cast<const TabuDevState *>(stage + at_st[k]);
            const long long *info = reinterpret_cast<const long long *>(stage + at_info[k]);
            const int done = sd.t - it.t0;
            double work = 0.0, dur = 0.0;
            for (int r = 0; r < it.gang; r++) {
                const long long *q = clk_of(k) + (size_t)r * kPersistClocks;
                work += (double)(q[0] + q[1] + q[3] + q[5]);   // move, refresh, update, select
                double dd = 0.0;
                for (int q2 = 0; q2 < 7; q2++) {
                    step[q2] += q[q2] * 1e-6;
                    dd += q[q2] * 1e-6;
                }
                dur = std::max(dur, dd);
            }
            if (dur > longest) {
                longest = dur;
                longest_i = order[k];
            }
            est += batch_search_us(it, pk.iters, it.gang) * 1e-3 * it.gang;
            if (done >= 1 && !sd.err) {
                const double fixed = kBatchFixedUs * it.gang;   // counted in the move and select
                it.in->batch_work_us = std::max(0.0, work * 1e-3 / done - fixed);
                it.in->batch_K = pk.K;
                it.in->batch_R = pk.R;
                it.in->batch_version = it.in->version;
            }
            records += info[1];
            cells += info[5];
            cellmin_bytes += info[1] * 4 * (table_ldT(it.in->B) / 32);
            moves += std::max(0, done);
            refresh_bytes += (long long)std::max(0, done) * 20 * it.in->M;
            select_bytes += (long long)std::max(0, done) * 12 * pk.K * it.nC;
            // the result
            const int i = order[k];
            stage_move *tr = trajs ? trajs[i] : nullptr;
            const int nm = std::min(sd.n_moves, pk.iters);
            if (tr && nm > 0 && !sd.err) std::memcpy(tr, stage + at_traj[k], (size_t)nm * sizeof(stage_move));
            s = tabu_result(c, &pk, false, sd, reinterpret_cast<const int32_t *>(stage + at_open[k]),
                            reinterpret_cast<const int32_t *>(stage + at_best[k]),
                            reinterpret_cast<const int32_t *>(stage + at_exp[k]), it.in->B, &res[i]);
            if (s != STAGE_OK && first == STAGE_OK) first = s;
        }
        for (int q = 0; q < P; q++)
            for (int ee = h_off[q]; ee < h_off[q + 1]; ee++) {
                const long long *cq = clk_of(h_sched[ee].x) + (size_t)h_sched[ee].y * kPersistClocks;
                for (int q2 = 0; q2 < 7; q2++) busy[q] += cq[q2] * 1e-6;
            }
        std::lock_guard<std::recursive_mutex> g(c->mu);
        KernelStat &ks = c->stats["tabu_batch"];
        ks.launches += 1;
        ks.ms += kms;
        c->stats["batch_records"].launches += records;
        c->stats["batch_cells_read"].launches += cells;
        // the method's bytes: the refreshes' 20 per mission, the updates' 32
        // per record, its row of cell minima and 128 per cell piece, the
        // selections' 12 per swap
        c->stats["batch_bytes"].launches += refresh_bytes + records * 32 + cellmin_bytes + cells * 128 + select_bytes;
        c->stats["batch_moves"].launches += moves;
        c->stats["batch_searches"].launches += ns;
        c->stats["batch_ctas"].launches = P;
        int gmax = 1;
        for (int i : order) gmax = std::max(gmax, items[i].gang);
        c->stats["batch_gang_max"].launches = gmax;
        double mx = 0.0, sum = 0.0;
        for (double b : busy) { mx = std::max(mx, b); sum += b; }
        c->stats["batch_cta_busy_max"].ms += mx;
        c->stats["batch_cta_busy_mean"].ms += sum / P;
        c->stats["batch_cta_estimate"].ms += est / P;
        if (longest_i >= 0) {
            // the longest search: its time, request index and gang; its estimate
            KernelStat &ls = c->stats["batch_longest"];
            ls.ms = longest;
            ls.launches = longest_i;
            KernelStat &le = c->stats["batch_longest_estimate"];
            le.ms = batch_search_us(items[longest_i], ps[longest_i].iters, items[longest_i].gang) * 1e-3;
            le.launches = items[longest_i].gang;
        }
        const char *nm[7] = {"batch_move", "batch_refresh", "batch_wait_refresh", "batch_update",
                             "batch_wait_update", "batch_select", "batch_wait_select"};
        for (int q = 0; q < 7; q++) c->stats[nm[q]].ms += step[q];
    }
    // the searches the launch did not take, alone
    for (int i = 0; i < n; i++) {
        if (items[i].fused) continue;
        stage_status s;
        if (items[i].nC == 0 || ps[i].iters == 0)
            s = tabu_finish(c, items[i].in, &ps[i], false, &res[i], trajs ? trajs[i] : nullptr, nullptr, nullptr,
                            nullptr, nullptr);
        else
            s = run_tabu(c, items[i].in, &ps[i], &res[i], trajs ? trajs[i] : nullptr, nullptr, nullptr, nullptr,
                         nullptr);
        if (s != STAGE_OK && first == STAGE_OK) first = s;
    }
    c->stats["batch_host_results"].ms += host_ms();
    return first;
}

// ----------------------------------------------------------- heterogeneous fleet
// Two searches over the one table (see k_fleet_select): A over every vehicle
// and the missions any vehicle may fly, B over the rotary-wing vehicles and
// the rotary-only missions; the other search's missions are masked out.
namespace {

struct FleetSide {
    DevBuf ws;
    TabuBuffers tb{};
    std::vector<int32_t> cand;
    int nC = 0;
};

// Workspace, placement, candidates and per-mission initialisation of one side.
stage_status fleet_side(stage_ctx *c, Instance *in, FleetSide &f, const std::vector<int32_t> &open, int R,
                        int traj_cap, const uint8_t *d_mask)
{
    const int K = (int)open.size();
    TabuBuffers tb{};
    const size_t bytes = carve_ws(nullptr, K, in->B, in->M_pad, traj_cap, tb);
    stage_status s = dev_alloc(c, bytes, f.ws);
    if (s != STAGE_OK) return s;
    carve_ws(static_cast<char *>(f.ws.p), K, in->B, in->M_pad, traj_cap, tb);
    tb.K = K; tb.B = in->B; tb.M = in->M; tb.M_pad = in->M_pad; tb.R = R;
    tb.mask = d_mask;
    std::vector<uint8_t> is_open(in->B, 0);
    for (int b : open) is_open[b] = 1;
    f.cand.clear();
    for (int b = 0; b < in->B; b++)
        if (in->h_avail[b] && !is_open[b]) f.cand.push_back(b);
    f.nC = (int)f.cand.size();
    f.tb = tb;
    std::vector<int32_t> zeros(in->B, 0);
    CK(cudaMemcpyAsync(tb.open, open.data(), (size_t)K * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(tb.best_open, open.data(), (size_t)K * 4, cudaMemcpyHostToDevice, c->stream));
    if (f.nC) CK(cudaMemcpyAsync(tb.cand, f.cand.data(), (size_t)f.nC * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(tb.expiry, zeros.data(), (size_t)in->B * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(tb.st, 0, sizeof(TabuDevState), c->stream));
    CK(cudaMemsetAsync(tb.v0, 0, 16, c->stream));
    CK(cudaMemsetAsync(tb.loss_c, 0, (size_t)K * 8, c->stream));
    CK(cudaMemsetAsync(tb.loss_d, 0, (size_t)K * 8, c->stream));
    CK(cudaMemsetAsync(tb.gain_c, 0, (size_t)in->B * 4, c->stream));
    CK(cudaMemsetAsync(tb.gain_d, 0, (size_t)in->B * 8, c->stream));
    CK(cudaMemsetAsync(tb.extra_c, 0, (size_t)K * in->B * 4, c->stream));
    CK(cudaMemsetAsync(tb.extra_d, 0, (size_t)K * in->B * 8, c->stream));
    CK(timed(c, "init", 1, [&] { return launch_init(tb, in->cost, c->stream); }));
    CK(cudaStreamSynchronize(c->stream));   // host vectors above
    return STAGE_OK;
}

}  // namespace

stage_status run_fleet(stage_ctx *c, Instance *in, const stage_fleet_params *p, stage_fleet_result *res,
                       stage_move *traj)
{
    if (!p) return set_err(c, STAGE_ERR_INVALID_ARG, "params is NULL");
    const int Kr = p->K_rotary, Kf = p->K_fixed, K = Kr + Kf;
    if (Kr < 0 || Kf < 0 || K < 1 || K > in->B || K > STAGE_MAX_K)
        return set_err(c, STAGE_ERR_INVALID_ARG, "K_rotary=%d, K_fixed=%d: need 1 <= K <= min(B=%d, %d)", Kr, Kf,
                       in->B, STAGE_MAX_K);
    if (K > in->n_avail) return set_err(c, STAGE_ERR_INVALID_ARG, "%d vehicles, %d available bases", K, in->n_avail);
    if (p->R < 0 || p->R == INT32_MAX) return set_err(c, STAGE_ERR_OUT_OF_RANGE, "R=%d outside [0, INT32_MAX)", p->R);
    if (p->iters < 0 || p->tenure < 0) return set_err(c, STAGE_ERR_INVALID_ARG, "iters and tenure must be >= 0");
    if (!p->base_helipad || !p->mission_rotary)
        return set_err(c, STAGE_ERR_INVALID_ARG, "base_helipad and mission_rotary are required");
    const int B = in->B;
    std::vector<uint8_t> heli(p->base_helipad, p->base_helipad + B);
    for (auto &h : heli) h = h ? 1 : 0;
    // ---- start: given, or ranking with the helipad rule
    std::vector<int32_t> rot, fix;
    if (p->start_rotary || p->start_fixed) {
        if ((Kr && !p->start_rotary) || (Kf && !p->start_fixed))
            return set_err(c, STAGE_ERR_INVALID_ARG, "give both start_rotary and start_fixed, or neither");
        if (Kr) rot.assign(p->start_rotary, p->start_rotary + Kr);
        if (Kf) fix.assign(p->start_fixed, p->start_fixed + Kf);
        std::vector<int32_t> all(rot);
        all.insert(all.end(), fix.begin(), fix.end());
        stage_status s = check_placement(c, in, all.data(), K);
        if (s != STAGE_OK) return s;
        for (int b : fix)
            if (heli[b]) return set_err(c, STAGE_ERR_INVALID_ARG, "fixed-wing start at helipad %d", b);
    } else {
        std::vector<int64_t> S(B);
        int32_t one = 0;
        stage_status s = do_rank(c, in, 1, &one, S.data());
        if (s != STAGE_OK) return s;
        std::vector<int32_t> order;
        for (int b = 0; b < B; b++)
            if (in->h_avail[b]) order.push_back(b);
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return S[x] != S[y] ? S[x] < S[y] : x < y; });
        std::vector<int32_t> chosen;
        int nh = 0;
        for (int b : order) {
            if ((int)chosen.size() == K) break;
            if (heli[b]) {
                if (nh < Kr) {
                    chosen.push_back(b);
                    nh++;
                }
            } else {
                chosen.push_back(b);
            }
        }
        int aer_avail = 0;
        for (int b : chosen) aer_avail += !heli[b];
        if ((int)chosen.size() < K || aer_avail < Kf)
            return set_err(c, STAGE_ERR_INVALID_ARG, "too few available aerodromes for %d fixed-wing vehicles", Kf);
        for (int b : chosen)
            if (heli[b]) rot.push_back(b);
        for (int b : chosen)
            if (!heli[b]) {
                if ((int)rot.size() < Kr) rot.push_back(b);
                else fix.push_back(b);
            }
    }
    std::vector<int32_t> open(rot);
    open.insert(open.end(), fix.begin(), fix.end());
    // ---- per-column mission masks of the two searches
    std::vector<int32_t> perm(in->M);
    CK(cudaMemcpy(perm.data(), in->perm, (size_t)in->M * 4, cudaMemcpyDeviceToHost));
    std::vector<uint8_t> host(3 * (size_t)in->M_pad + B, 0);
    uint8_t *mA = host.data(), *mB = host.data() + in->M_pad;
    bool anyB = false;
    for (int col = 0; col < in->M; col++) {
        const int m = perm[col];
        if (m < 0) continue;   // removed mission
        const bool r = p->mission_rotary[m] != 0;
        mA[col] = !r;
        mB[col] = r;
        anyB |= r;
    }
    std::copy(heli.begin(), heli.end(), host.data() + 2 * (size_t)in->M_pad);
    const int hasB = (Kr >= 1 && anyB) ? 1 : 0;
    DevBuf dm, dpos, chgB;
    stage_status s = dev_alloc(c, host.size(), dm);
    if (s != STAGE_OK) return s;
    s = dev_alloc(c, (size_t)B * 4, dpos);
    if (s != STAGE_OK) {
        dev_free(c, dm);
        return s;
    }
    auto *d_m = static_cast<uint8_t *>(dm.p);
    int *d_pos = static_cast<int *>(dpos.p);
    FleetSide A, Bs;
    auto cleanup = [&]() {
        dev_free(c, A.ws);
        dev_free(c, Bs.ws);
        dev_free(c, dm);
        dev_free(c, dpos);
        dev_free(c, chgB);
    };
    cudaError_t e = cudaMemcpyAsync(d_m, host.data(), host.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cleanup();
        return set_err(c, STAGE_ERR_CUDA, "fleet set-up failed: %s", cudaGetErrorString(e));
    }
    s = fleet_side(c, in, A, open, p->R, p->iters, d_m);
    if (s == STAGE_OK && hasB) s = fleet_side(c, in, Bs, rot, p->R, 1, d_m + in->M_pad);
    if (s != STAGE_OK) {
        cleanup();
        return s;
    }
    // beyond L2 (or with STAGE_INCREMENTAL) both searches keep their terms
    // across moves: one full pass each, then per iteration the records of the
    // missions a move touched (B, held after a fixed-wing move, skips its
    // refresh and update as it skips its pass); B's candidates are every base
    // outside its placement, so its columns stay whole while fixed-wing
    // vehicles come and go
    bool inc = !(c->flags & STAGE_FULL_PASS) && swap_delta_fits(K) && A.nC > 0 &&
               ((c->flags & STAGE_INCREMENTAL) ||
                (size_t)A.nC * in->M_pad * sizeof(int32_t) >= kIncrementalMinTableBytes);
    if (inc) inc = use_incremental(c, in, A.tb);
    if (inc && hasB) {
        if (dev_alloc(c, (size_t)in->M_pad * 2 * sizeof(int4), chgB) == STAGE_OK) {
            Bs.tb.chg = static_cast<int4 *>(chgB.p);
            Bs.tb.costT = A.tb.costT;
            Bs.tb.border = A.tb.border;
            Bs.tb.cellmin = A.tb.cellmin;
            Bs.tb.ldT = A.tb.ldT;
        } else {
            set_err(c, STAGE_OK, "");   // no room: both searches take the full pass
            inc = false;
            A.tb.chg = nullptr;
        }
    }
    // state: A carries the search; B only its hold / done flags and last move
    unsigned long long v0a[2] = {0, 0}, v0b[2] = {0, 0};
    std::vector<int32_t> pos(B, -1);
    for (int q = 0; q < Bs.nC; q++) pos[Bs.cand[q]] = q;
    e = cudaMemcpy(v0a, A.tb.v0, 16, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && hasB) e = cudaMemcpy(v0b, Bs.tb.v0, 16, cudaMemcpyDeviceToHost);
    TabuDevState st{}, sb{};
    st.tenure = p->tenure;
    st.accept_worsening = p->accept_worsening ? 1 : 0;
    st.nC = A.nC;
    st.traj_cap = p->iters;
    st.t_end = p->iters;
    st.best_iter = -1;
    st.cur_cov = st.best_cov = (long long)(v0a[0] + v0b[0]);
    st.cur_dist = st.best_dist = (long long)(v0a[1] + v0b[1]);
    sb.nC = Bs.nC;
    sb.t_end = INT32_MAX;
    if (e == cudaSuccess) e = cudaMemcpyAsync(A.tb.st, &st, sizeof st, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && hasB) e = cudaMemcpyAsync(Bs.tb.st, &sb, sizeof sb, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_pos, pos.data(), (size_t)B * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    volatile int *done_flag = static_cast<volatile int *>(c->pinned);
    *done_flag = 0;
    const uint8_t *d_heli = d_m + 2 * (size_t)in->M_pad;
    for (int it = 0; e == cudaSuccess && it < p->iters && A.nC > 0; it++) {
        const bool full = !inc || it == 0;
        if (full)
            e = timed(c, "swap_eval", 1, [&] { return launch_swap_eval(A.tb, in->cost, A.nC, 0, c->stream); });
        if (e == cudaSuccess && full && hasB && Bs.nC > 0)
            e = timed(c, "swap_eval", 1, [&] { return launch_swap_eval(Bs.tb, in->cost, Bs.nC, 0, c->stream); });
        if (e == cudaSuccess)
            e = timed(c, "fleet_select", 1,
                      [&] { return launch_fleet_select(A.tb, Bs.tb, Kr, hasB, d_heli, d_pos, c->stream); });
        if (e == cudaSuccess) e = timed(c, "refresh", 1, [&] { return launch_refresh(A.tb, in->cost, c->stream); });
        if (e == cudaSuccess && hasB)
            e = timed(c, "refresh", 1, [&] { return launch_refresh(Bs.tb, in->cost, c->stream); });
        if (e == cudaSuccess && inc)
            e = timed(c, "swap_delta", 1, [&] { return launch_swap_delta(A.tb, c->stream); });
        if (e == cudaSuccess && inc && hasB)
            e = timed(c, "swap_delta", 1, [&] { return launch_swap_delta(Bs.tb, c->stream); });
        if (e == cudaSuccess && (it & 31) == 31) {
            e = cudaMemcpyAsync(c->pinned, &A.tb.st->done, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (*done_flag) break;
        }
    }
    std::vector<int32_t> fin(K), best(K);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, A.tb.st, sizeof st, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fin.data(), A.tb.open, (size_t)K * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(best.data(), A.tb.best_open, (size_t)K * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    const int n = std::min(st.n_moves, p->iters);
    if (e == cudaSuccess && traj && n > 0)
        e = cudaMemcpy(traj, A.tb.traj, (size_t)n * sizeof(stage_move), cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) return set_err(c, STAGE_ERR_CUDA, "fleet search failed: %s", cudaGetErrorString(e));
    if (st.err & kErrPipelineTimeout)
        return set_err(c, STAGE_ERR_TIMEOUT, "a device-side wait gave up after %lld polls at iteration %d",
                       (long long)c->spin_limit, st.t);
    if (st.err)
        return set_err(c, STAGE_ERR_INTERNAL, "device self-check failed (code %d) at iteration %d", st.err, st.t);
    if (res) {
        res->n_moves = st.n_moves;
        res->best_iter = st.best_iter;
        res->best_cov = st.best_cov;
        res->best_dist = st.best_dist;
        res->final_cov = st.cur_cov;
        res->final_dist = st.cur_dist;
        auto put = [](std::vector<int32_t> v, int32_t *dst) {
            std::sort(v.begin(), v.end());
            if (dst) std::copy(v.begin(), v.end(), dst);
        };
        put(std::vector<int32_t>(best.begin(), best.begin() + Kr), res->best_rotary);
        put(std::vector<int32_t>(best.begin() + Kr, best.end()), res->best_fixed);
        put(std::vector<int32_t>(fin.begin(), fin.begin() + Kr), res->final_rotary);
        put(std::vector<int32_t>(fin.begin() + Kr, fin.end()), res->final_fixed);
    }
    return STAGE_OK;
}

// Local search (Alg. 2 as read for identical vehicles): iterations of
// (swap pass, first-improvement selection, refresh) until the device state
// says done; a pass change skips the swap pass and the refresh of the next step.
stage_status run_local_search(stage_ctx *c, Instance *in, const stage_ls_params *p, stage_ls_result *res,
                              stage_move *traj)
{
    if (!p) return set_err(c, STAGE_ERR_INVALID_ARG, "params is NULL");
    const int K = p->K;
    if (K < 1 || K > in->B || K > STAGE_MAX_K)
        return set_err(c, STAGE_ERR_INVALID_ARG, "K=%d outside [1, min(B=%d, %d)]", K, in->B, STAGE_MAX_K);
    if (K > in->n_avail)
        return set_err(c, STAGE_ERR_INVALID_ARG, "K=%d exceeds the %d available bases", K, in->n_avail);
    if (p->R < 0 || p->R == INT32_MAX)
        return set_err(c, STAGE_ERR_OUT_OF_RANGE, "R=%d outside [0, INT32_MAX)", p->R);
    if (p->n_passes < 1 || p->max_moves < 0 || !p->perm_slots || (!p->perm_cands && in->n_avail > K))
        return set_err(c, STAGE_ERR_INVALID_ARG, "local search needs n_passes >= 1, max_moves >= 0 and permutations");
    const int nC0 = in->n_avail - K;
    const int P = p->n_passes;
    // positions of every slot and candidate in each pass's scan order
    std::vector<int32_t> rank((size_t)P * (K + nC0), -1);
    for (int q = 0; q < P; q++) {
        int32_t *rs = rank.data() + (size_t)q * K;
        int32_t *rc = rank.data() + (size_t)P * K + (size_t)q * nC0;
        for (int a = 0; a < K; a++) {
            const int v = p->perm_slots[(size_t)q * K + a];
            if (v < 0 || v >= K || rs[v] >= 0)
                return set_err(c, STAGE_ERR_INVALID_ARG, "perm_slots row %d is not a permutation of 0..%d", q, K - 1);
            rs[v] = a;
        }
        for (int b = 0; b < nC0; b++) {
            const int v = p->perm_cands[(size_t)q * nC0 + b];
            if (v < 0 || v >= nC0 || rc[v] >= 0)
                return set_err(c, STAGE_ERR_INVALID_ARG, "perm_cands row %d is not a permutation of 0..%d", q,
                               nC0 - 1);
            rc[v] = b;
        }
    }
    std::vector<int32_t> start(K);
    if (p->start_open) {
        stage_status s = check_placement(c, in, p->start_open, K);
        if (s != STAGE_OK) return s;
        std::copy(p->start_open, p->start_open + K, start.begin());
    } else {
        stage_status s = do_rank(c, in, K, start.data(), nullptr);
        if (s != STAGE_OK) return s;
    }
    int nC = 0;
    stage_status s = setup_search(c, in, start.data(), K, p->R, p->max_moves, 0, 1, 0, nullptr, &nC);
    if (s != STAGE_OK) return s;
    if (nC != nC0) return set_err(c, STAGE_ERR_INTERNAL, "candidate count %d, expected %d", nC, nC0);
    // The terms are kept across moves (one full pass, then per step the
    // records of the missions a move touched; a pass change holds the terms,
    // as in the full-pass form): the whole search in one cooperative launch
    // for tables of 2^18 entries or more (or with STAGE_INCREMENTAL) where
    // that launch takes the shape (not with STAGE_NO_PERSIST; smaller tables
    // stream faster than its fixed cost per move), else per-step launches for
    // tables beyond L2 (or with STAGE_INCREMENTAL), else a full pass per step.
    TabuBuffers tb = in->tb;
    const bool big = (size_t)nC * in->M_pad >= (1u << 18) || (c->flags & STAGE_INCREMENTAL);
    const int pgrid = nC > 0 && p->max_moves > 0 && big && !(c->flags & STAGE_NO_PERSIST) && tb.mask == nullptr
                          ? persist_grid(K, in->B, table_ldT(in->B), in->M_pad)
                          : 0;
    bool inc = !(c->flags & STAGE_FULL_PASS) && swap_delta_fits(K) && nC > 0 &&
               ((c->flags & STAGE_INCREMENTAL) || pgrid > 0 ||
                (size_t)nC * in->M_pad * sizeof(int32_t) >= kIncrementalMinTableBytes);
    if (inc) inc = use_incremental(c, in, tb);
    bool persist = inc && pgrid > 0;
    if (persist) {
        const size_t need = persist_scratch_bytes(K, pgrid, in->M_pad);
        if (!in->mem_persist.p || in->mem_persist.bytes < need) {
            dev_free(c, in->mem_persist);
            if (dev_alloc(c, need, in->mem_persist) != STAGE_OK) {
                persist = false;
                set_err(c, STAGE_OK, "");   // a refused allocation here is not an error of the search
            }
        }
    }
    DevBuf dr;
    s = dev_alloc(c, rank.size() * 4 + 4, dr);
    if (s != STAGE_OK) return s;
    const int *d_rank_slot = static_cast<const int *>(dr.p);
    const int *d_rank_cand = d_rank_slot + (size_t)P * K;
    cudaError_t e = cudaMemcpyAsync(dr.p, rank.data(), rank.size() * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&tb.st->ls_passes, &P, sizeof(int), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_begin(tb, 0, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // host vectors above
    c->stats["begin"].launches += 1;
    // every step applies a move, changes pass or stops
    const long long max_steps = (long long)p->max_moves + P + 1;
    volatile int *done_flag = static_cast<volatile int *>(c->pinned);
    *done_flag = 0;
    const bool profiling = (c->flags & STAGE_PROFILE) != 0;
    if (e == cudaSuccess && inc)
        e = timed(c, "swap_eval", 1, [&] { return launch_swap_eval(tb, in->cost, nC, 0, c->stream); });
    auto step = [&]() {
        cudaError_t r = inc ? cudaSuccess : launch_swap_eval(tb, in->cost, nC, 0, c->stream);
        if (r == cudaSuccess) r = launch_ls_select(tb, nC, d_rank_slot, d_rank_cand, c->stream);
        if (r == cudaSuccess) r = launch_refresh(tb, in->cost, c->stream);
        if (r == cudaSuccess && inc) r = launch_swap_delta(tb, c->stream);
        return r;
    };
    auto poll = [&]() {
        cudaError_t r = cudaMemcpyAsync(c->pinned, &tb.st->done, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (r == cudaSuccess) r = cudaStreamSynchronize(c->stream);
        return r;
    };
    if (e == cudaSuccess && persist)
        e = timed(c, "local_persist", 1, [&] {
            return launch_local_persist(tb, in->cost, in->mem_persist.p, pgrid, c->spin_limit, d_rank_slot,
                                        d_rank_cand, c->stream);
        });
    cudaGraphExec_t ge = nullptr;
    if (e == cudaSuccess && nC > 0 && !persist && !profiling && max_steps >= kGraphIters) {
        cudaGraph_t gr = nullptr;
        e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        for (int k = 0; e == cudaSuccess && k < kGraphIters; k++) e = step();
        cudaError_t e2 = cudaStreamEndCapture(c->stream, &gr);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, gr, 0);
        if (gr) cudaGraphDestroy(gr);
    }
    long long it = 0;
    while (e == cudaSuccess && nC > 0 && !persist && it < max_steps) {
        if (ge) {
            for (const char *nm : {"ls_select", "refresh"}) c->stats[nm].launches += kGraphIters;
            c->stats[inc ? "swap_delta" : "swap_eval"].launches += kGraphIters;
            e = cudaGraphLaunch(ge, c->stream);
            it += kGraphIters;
        } else {
            for (int k = 0; e == cudaSuccess && k < kGraphIters && it < max_steps; k++, it++) {
                if (!inc)
                    e = timed(c, "swap_eval", 1, [&] { return launch_swap_eval(tb, in->cost, nC, 0, c->stream); });
                if (e == cudaSuccess)
                    e = timed(c, "ls_select", 1,
                              [&] { return launch_ls_select(tb, nC, d_rank_slot, d_rank_cand, c->stream); });
                if (e == cudaSuccess)
                    e = timed(c, "refresh", 1, [&] { return launch_refresh(tb, in->cost, c->stream); });
                if (e == cudaSuccess && inc)
                    e = timed(c, "swap_delta", 1, [&] { return launch_swap_delta(tb, c->stream); });
            }
        }
        if (e == cudaSuccess) e = poll();
        if (*done_flag) break;
    }
    if (ge) cudaGraphExecDestroy(ge);
    TabuDevState st{};
    std::vector<int32_t> fin(K);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, tb.st, sizeof st, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fin.data(), tb.open, (size_t)K * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    const int n = std::min(st.n_moves, p->max_moves);
    if (e == cudaSuccess && traj && n > 0)
        e = cudaMemcpy(traj, tb.traj, (size_t)n * sizeof(stage_move), cudaMemcpyDeviceToHost);
    dev_free(c, dr);
    if (e != cudaSuccess) return set_err(c, STAGE_ERR_CUDA, "local search failed: %s", cudaGetErrorString(e));
    if (st.err & kErrPipelineTimeout)
        return set_err(c, STAGE_ERR_TIMEOUT, "a device-side wait gave up after %lld polls after %d moves",
                       (long long)c->spin_limit, st.n_moves);
    if (st.err)
        return set_err(c, STAGE_ERR_INTERNAL, "device self-check failed (code %d) after %d moves", st.err, st.n_moves);
    if (nC > 0 && !st.done && st.n_moves < p->max_moves)
        return set_err(c, STAGE_ERR_INTERNAL, "local search did not finish in %lld steps", max_steps);
    if (res) {
        res->n_moves = st.n_moves;
        res->passes = nC > 0 ? st.ls_pass + 1 : 0;
        res->local_optimum = nC > 0 ? st.ls_optimum : 1;
        res->final_cov = st.cur_cov;
        res->final_dist = st.cur_dist;
        std::sort(fin.begin(), fin.end());
        if (res->final_open) std::copy(fin.begin(), fin.end(), res->final_open);
    }
    return STAGE_OK;
}

}  // namespace stg_rt

using namespace stg_rt;

// ============================================================== C ABI

extern "C" {

int32_t stage_version(void) { return 1 * 10000 + 0 * 100 + 0; }

stage_status stage_create(const stage_config *cfg, stage_ctx **out)
{
    if (!out) return STAGE_ERR_INVALID_ARG;
    *out = nullptr;
    stage_config d{};
    if (cfg) d = *cfg;
    if ((d.alloc == nullptr) != (d.free == nullptr)) return STAGE_ERR_INVALID_ARG;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        return STAGE_ERR_CUDA;
    }
    if (d.device < 0 || d.device >= n) return STAGE_ERR_INVALID_ARG;
    if (cudaSetDevice(d.device) != cudaSuccess) return STAGE_ERR_CUDA;
    if (kernels_init() != cudaSuccess) return STAGE_ERR_CUDA;
    stage_ctx *c = new stage_ctx();
    c->device = d.device;
    c->flags = d.flags;
    c->budget = d.hbm_budget_bytes;
    c->max_slots = d.max_slots > 0 ? d.max_slots : 8;
    c->spin_limit = d.spin_limit > 0 ? d.spin_limit : (1ll << 26);
    c->alloc = d.alloc;
    c->free = d.free;
    c->alloc_user = d.alloc_user;
    if (d.stream) {
        c->stream = static_cast<cudaStream_t>(d.stream);
    } else {
        // the context's own stream takes the highest priority: set-up work of
        // requests joining the batch engine (whose stream has the lowest)
        // then waits for free SMs, not for the whole running step
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (cudaStreamCreateWithPriority(&c->stream, cudaStreamNonBlocking, greatest) != cudaSuccess) {
            delete c;
            return STAGE_ERR_CUDA;
        }
        c->own_stream = true;
    }
    if (cudaMallocHost(&c->pinned, 256) != cudaSuccess) {
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return STAGE_ERR_CUDA;
    }
    int pools = 0;
    if (!c->alloc && cudaDeviceGetAttribute(&pools, cudaDevAttrMemoryPoolsSupported, c->device) == cudaSuccess &&
        pools) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = c->device;
        if (cudaMemPoolCreate(&c->pool, &props) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;   // freed blocks stay with the pool for reuse
            cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        } else {
            cudaGetLastError();
            c->pool = nullptr;
        }
    }
    *out = c;
    return STAGE_OK;
}

stage_status stage_destroy(stage_ctx *c)
{
    if (!c) return STAGE_OK;
    engine_destroy(c);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto &kv : c->insts) free_instance(c, kv.second);
    c->insts.clear();
    fold_stats(c);
    if (c->pool) {
        cudaStreamSynchronize(c->stream);
        cudaMemPoolDestroy(c->pool);
    }
    for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->batch_pinned) cudaFreeHost(c->batch_pinned);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return STAGE_OK;
}

stage_status stage_last_error(const stage_ctx *c, char *buf, size_t n)
{
    if (!c || !buf || n == 0) return STAGE_ERR_INVALID_ARG;
    snprintf(buf, n, "%s", c->err.c_str());
    return STAGE_OK;
}

stage_status stage_memory_used(const stage_ctx *c, uint64_t *out)
{
    if (!c || !out) return STAGE_ERR_INVALID_ARG;
    *out = c->used;
    return STAGE_OK;
}

stage_status stage_load_instance(stage_ctx *c, const stage_instance_desc *d, stage_inst *out)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    if (!d || !out) return set_err(c, STAGE_ERR_INVALID_ARG, "desc or out is NULL");
    if (!d->base_xy || !d->pick_xy || !d->drop_xy)
        return set_err(c, STAGE_ERR_INVALID_ARG, "coordinate pointer is NULL");
    if (d->B < 1 || d->M < 1) return set_err(c, STAGE_ERR_INVALID_ARG, "B and M must be >= 1");
    if (d->B > STAGE_MAX_BASES) return set_err(c, STAGE_ERR_OUT_OF_RANGE, "B=%d > %d", d->B, STAGE_MAX_BASES);
    if (d->M > STAGE_MAX_MISSIONS) return set_err(c, STAGE_ERR_OUT_OF_RANGE, "M=%d > %d", d->M, STAGE_MAX_MISSIONS);
    CK(cudaSetDevice(c->device));
    const bool on_dev = (d->flags & STAGE_DESC_DEVICE) != 0;
    const int metric = (d->flags & STAGE_DESC_HAVERSINE) ? 1 : 0;
    // coordinate bounds: metres in a plane, or latitude / longitude in microdegrees
    const int lim_x = metric ? STAGE_MAX_LAT_UDEG : STAGE_MAX_COORD;
    const int lim_y = metric ? STAGE_MAX_LON_UDEG : STAGE_MAX_COORD;
    const int B = d->B, M = d->M;
    const int M_pad = (int)round_up((size_t)M, kPadMissions);
    std::vector<uint8_t> avail(B, 1);
    if (on_dev) {
        // device inputs: range check on the device, availability read back
        if (d->base_available) CK(cudaMemcpy(avail.data(), d->base_available, B, cudaMemcpyDeviceToHost));
        int *flag = static_cast<int *>(c->pinned) + 16;
        *flag = 0;
        DevBuf fb;
        stage_status s0 = dev_alloc(c, 256, fb);
        if (s0 != STAGE_OK) return s0;
        int *dflag = static_cast<int *>(fb.p);
        cudaError_t e0 = cudaMemsetAsync(dflag, 0, 4, c->stream);
        if (e0 == cudaSuccess) e0 = launch_check_coords(d->base_xy, 2 * (size_t)B, lim_x, lim_y, dflag, c->stream);
        if (e0 == cudaSuccess) e0 = launch_check_coords(d->pick_xy, 2 * (size_t)M, lim_x, lim_y, dflag, c->stream);
        if (e0 == cudaSuccess) e0 = launch_check_coords(d->drop_xy, 2 * (size_t)M, lim_x, lim_y, dflag, c->stream);
        if (e0 == cudaSuccess) e0 = cudaMemcpyAsync(flag, dflag, 4, cudaMemcpyDeviceToHost, c->stream);
        if (e0 == cudaSuccess) e0 = cudaStreamSynchronize(c->stream);
        dev_free(c, fb);
        if (e0 != cudaSuccess) return set_err(c, STAGE_ERR_CUDA, "input check failed: %s", cudaGetErrorString(e0));
        if (*flag) return set_err(c, STAGE_ERR_OUT_OF_RANGE, "a coordinate is outside [-%d, %d] x [-%d, %d]", lim_x,
                                  lim_x, lim_y, lim_y);
    } else {
        if (d->base_available) std::copy(d->base_available, d->base_available + B, avail.begin());
        auto bad = [&](const int32_t *v, size_t n) {
            for (size_t k = 0; k < n; k++) {
                const int lim = (k & 1) ? lim_y : lim_x;
                if (v[k] > lim || v[k] < -lim) return true;
            }
            return false;
        };
        if (bad(d->base_xy, 2 * (size_t)B) || bad(d->pick_xy, 2 * (size_t)M) || bad(d->drop_xy, 2 * (size_t)M))
            return set_err(c, STAGE_ERR_OUT_OF_RANGE, "a coordinate is outside [-%d, %d] x [-%d, %d]", lim_x, lim_x,
                           lim_y, lim_y);
    }
    for (auto &a : avail) a = a ? 1 : 0;
    Instance *in = new Instance();
    in->B = B; in->M = M; in->M_pad = M_pad;
    in->metric = metric;
    in->h_avail = avail;
    in->n_avail = (int)std::count(avail.begin(), avail.end(), (uint8_t)1);
    size_t coords = carve_coords(nullptr, B, M_pad, nullptr);
    stage_status s = dev_alloc(c, coords, in->mem_coords);
    if (s == STAGE_OK) s = dev_alloc(c, (size_t)B * M_pad * 4, in->mem_table);
    if (s != STAGE_OK) {
        free_instance(c, in);
        return s;
    }
    carve_coords(static_cast<char *>(in->mem_coords.p), B, M_pad, in);
    in->cost = static_cast<int32_t *>(in->mem_table.p);
    DevBuf order_tmp;
    s = dev_alloc(c, order_scratch_bytes(M), order_tmp);
    if (s != STAGE_OK) {
        free_instance(c, in);
        return s;
    }
    const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(in->base, d->base_xy, (size_t)B * 8, kind, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(in->pick_in, d->pick_xy, (size_t)M * 8, kind, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(in->drop_in, d->drop_xy, (size_t)M * 8, kind, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(in->avail, in->h_avail.data(), B, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = timed(c, "order", 10, [&] {
            return launch_order(M, in->pick_in, in->drop_in, order_tmp.p, in->perm, in->inv, in->pick,
                                in->drop, c->stream);
        });
    // where the search will take the incremental form, the table, its row
    // sums, its mission-major copy and the copy's cell minima in one pass
    // (with no room for the copy, the table alone; the copy follows when a
    // search needs it)
    const int ldT = table_ldT(B);
    const bool want_copy = !c->load_without_copy && !(c->flags & STAGE_FULL_PASS) &&
                           ((c->flags & STAGE_INCREMENTAL) || (size_t)B * M_pad * 4 >= kIncrementalMinTableBytes);
    bool fused = false;
    if (e == cudaSuccess && want_copy) {
        fused = dev_alloc(c, costT_bytes(M_pad, ldT), in->mem_costT) == STAGE_OK &&
                dev_alloc(c, (size_t)B * 8, in->mem_rowsum) == STAGE_OK;
        if (!fused) {
            dev_free(c, in->mem_costT);
            dev_free(c, in->mem_rowsum);
            set_err(c, STAGE_OK, "");   // a refused allocation here is not an error of the load
        }
    }
    if (e == cudaSuccess && fused) {
        std::vector<int2> bxy(B);
        if (on_dev) e = cudaMemcpy(bxy.data(), d->base_xy, (size_t)B * sizeof(int2), cudaMemcpyDeviceToHost);
        else std::memcpy(bxy.data(), d->base_xy, (size_t)B * sizeof(int2));
        const std::vector<int32_t> border = spatial_order(bxy, ldT);
        int32_t *costT = static_cast<int32_t *>(in->mem_costT.p);
        int32_t *d_border = costT + (size_t)M_pad * ldT;
        int32_t *d_cellmin = d_border + ldT;
        auto *S = static_cast<unsigned long long *>(in->mem_rowsum.p);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_border, border.data(), (size_t)ldT * sizeof(int32_t), cudaMemcpyHostToDevice,
                                c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(S, 0, (size_t)B * 8, c->stream);
        if (e == cudaSuccess)
            e = timed(c, "table", 2, [&] {
                return launch_table_fused(B, M, M_pad, ldT, in->base, in->pick, in->drop, in->pd, d_border,
                                          in->cost, costT, d_cellmin, S, metric, c->stream);
            });
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // the host order goes out of scope
        if (e == cudaSuccess) {
            in->ldT = ldT;
            in->costT_ok = true;
            in->rowsum_ok = true;
        }
    } else if (e == cudaSuccess) {
        e = timed(c, "table", 2, [&] {
            return launch_table(B, M, M_pad, in->base, in->pick, in->drop, in->pd, in->cost, metric, c->stream);
        });
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, order_tmp);
    if (e != cudaSuccess) {
        free_instance(c, in);
        return set_err(c, STAGE_ERR_CUDA, "building the cost table failed: %s", cudaGetErrorString(e));
    }
    uint64_t id = c->next_id++;
    c->insts[id] = in;
    *out = id;
    return STAGE_OK;
}

stage_status stage_unload_instance(stage_ctx *c, stage_inst h)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    Instance *in = find_inst(c, h);
    if (!in) return set_err(c, STAGE_ERR_NOT_FOUND, "unknown instance %llu", (unsigned long long)h);
    if (in->busy) return set_err(c, STAGE_ERR_ADMISSION, "instance %llu is in use by a batch request",
                                 (unsigned long long)h);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    c->insts.erase(h);
    free_instance(c, in);
    return STAGE_OK;
}

// Grow an instance's table and mission arrays to hold at least M_new columns.
static stage_status grow_instance(stage_ctx *c, Instance *in, int M_new)
{
    const int cap = (int)round_up((size_t)M_new + (size_t)M_new / 8 + 64, kPadMissions);
    DevBuf coords, table;
    stage_status s = dev_alloc(c, carve_coords(nullptr, in->B, cap, nullptr), coords);
    if (s == STAGE_OK) s = dev_alloc(c, (size_t)in->B * cap * 4, table);
    if (s != STAGE_OK) {
        dev_free(c, coords);
        return s;
    }
    Instance nw;
    carve_coords(static_cast<char *>(coords.p), in->B, cap, &nw);
    int32_t *cost = static_cast<int32_t *>(table.p);
    const int M = in->M, B = in->B;
    cudaStream_t st = c->stream;
    cudaError_t e = launch_fill_i32(cost, (size_t)B * cap, kInf, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(cost, (size_t)cap * 4, in->cost, (size_t)in->M_pad * 4, (size_t)M * 4, B,
                              cudaMemcpyDeviceToDevice, st);
    auto cp = [&](void *dst, const void *src, size_t n) {
        if (e == cudaSuccess && n) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, st);
    };
    cp(nw.base, in->base, (size_t)B * 8);
    cp(nw.pick, in->pick, (size_t)M * 8);
    cp(nw.drop, in->drop, (size_t)M * 8);
    cp(nw.pick_in, in->pick_in, (size_t)M * 8);
    cp(nw.drop_in, in->drop_in, (size_t)M * 8);
    cp(nw.pd, in->pd, (size_t)M * 4);
    cp(nw.perm, in->perm, (size_t)M * 4);
    cp(nw.inv, in->inv, (size_t)M * 4);
    cp(nw.avail, in->avail, (size_t)B);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        dev_free(c, coords);
        dev_free(c, table);
        return set_err(c, STAGE_ERR_CUDA, "growing the table failed: %s", cudaGetErrorString(e));
    }
    dev_free(c, in->mem_coords);
    dev_free(c, in->mem_table);
    in->mem_coords = coords;
    in->mem_table = table;
    in->base = nw.base; in->pick = nw.pick; in->drop = nw.drop; in->pick_in = nw.pick_in;
    in->drop_in = nw.drop_in; in->pd = nw.pd; in->perm = nw.perm; in->inv = nw.inv; in->avail = nw.avail;
    in->cost = cost;
    in->M_pad = cap;
    return STAGE_OK;
}

stage_status stage_update_instance(stage_ctx *c, stage_inst h, const stage_update *u)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    Instance *in = find_inst(c, h);
    if (!in) return set_err(c, STAGE_ERR_NOT_FOUND, "unknown instance %llu", (unsigned long long)h);
    if (!u) return set_err(c, STAGE_ERR_INVALID_ARG, "update is NULL");
    if (in->busy) return set_err(c, STAGE_ERR_ADMISSION, "instance %llu is in use by a batch request",
                                 (unsigned long long)h);
    if (u->n_add < 0 || u->n_remove < 0 || u->n_unavail < 0 || u->n_avail < 0 ||
        (u->n_add && (!u->add_pick_xy || !u->add_drop_xy)) || (u->n_remove && !u->remove_ids) ||
        (u->n_unavail && !u->unavail_ids) || (u->n_avail && !u->avail_ids))
        return set_err(c, STAGE_ERR_INVALID_ARG, "malformed update");
    for (int k = 0; k < u->n_unavail; k++)
        if (u->unavail_ids[k] < 0 || u->unavail_ids[k] >= in->B)
            return set_err(c, STAGE_ERR_INVALID_ARG, "base id %d out of range", u->unavail_ids[k]);
    for (int k = 0; k < u->n_avail; k++)
        if (u->avail_ids[k] < 0 || u->avail_ids[k] >= in->B)
            return set_err(c, STAGE_ERR_INVALID_ARG, "base id %d out of range", u->avail_ids[k]);
    for (int k = 0; k < u->n_remove; k++)
        if (u->remove_ids[k] < 0 || u->remove_ids[k] >= in->M)
            return set_err(c, STAGE_ERR_INVALID_ARG, "mission id %d out of range", u->remove_ids[k]);
    for (size_t k = 0; k < 2 * (size_t)u->n_add; k++) {
        const int32_t x = u->add_pick_xy[k], y = u->add_drop_xy[k];
        const int lim = in->metric ? ((k & 1) ? STAGE_MAX_LON_UDEG : STAGE_MAX_LAT_UDEG) : STAGE_MAX_COORD;
        if (x > lim || x < -lim || y > lim || y < -lim)
            return set_err(c, STAGE_ERR_OUT_OF_RANGE, "an added coordinate is outside [-%d, %d]", lim, lim);
    }
    if ((int64_t)in->M + u->n_add > STAGE_MAX_MISSIONS)
        return set_err(c, STAGE_ERR_OUT_OF_RANGE, "more than %d mission ids", STAGE_MAX_MISSIONS);
    CK(cudaSetDevice(c->device));
    // bases
    if (u->n_unavail || u->n_avail) {
        for (int k = 0; k < u->n_unavail; k++) in->h_avail[u->unavail_ids[k]] = 0;
        for (int k = 0; k < u->n_avail; k++) in->h_avail[u->avail_ids[k]] = 1;
        in->n_avail = (int)std::count(in->h_avail.begin(), in->h_avail.end(), (uint8_t)1);
        CK(cudaMemcpyAsync(in->avail, in->h_avail.data(), in->B, cudaMemcpyHostToDevice, c->stream));
    }
    // removed missions
    if (u->n_remove) {
        DevBuf ids;
        stage_status s = dev_alloc(c, (size_t)u->n_remove * 4, ids);
        if (s != STAGE_OK) return s;
        cudaError_t e = cudaMemcpyAsync(ids.p, u->remove_ids, (size_t)u->n_remove * 4, cudaMemcpyHostToDevice,
                                        c->stream);
        if (e == cudaSuccess)
            e = timed(c, "update", 1, [&] {
                return launch_tombstone(static_cast<int32_t *>(ids.p), u->n_remove, in->inv, in->perm, in->cost,
                                        in->B, in->M_pad, c->stream);
            });
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        dev_free(c, ids);
        if (e != cudaSuccess) return set_err(c, STAGE_ERR_CUDA, "removing missions failed: %s", cudaGetErrorString(e));
    }
    // appended missions: next ids, next columns (id == column for appended missions)
    if (u->n_add) {
        const int M0 = in->M, M1 = in->M + u->n_add;
        if (M1 > in->M_pad) {
            stage_status s = grow_instance(c, in, M1);
            if (s != STAGE_OK) return s;
        }
        std::vector<int32_t> ident(u->n_add);
        for (int k = 0; k < u->n_add; k++) ident[k] = M0 + k;
        const size_t n8 = (size_t)u->n_add * 8, n4 = (size_t)u->n_add * 4;
        CK(cudaMemcpyAsync(in->pick_in + M0, u->add_pick_xy, n8, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(in->drop_in + M0, u->add_drop_xy, n8, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(in->pick + M0, u->add_pick_xy, n8, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(in->drop + M0, u->add_drop_xy, n8, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(in->perm + M0, ident.data(), n4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(in->inv + M0, ident.data(), n4, cudaMemcpyHostToDevice, c->stream));
        CK(timed(c, "update", 1, [&] {
            return launch_table_columns(in->B, M0, u->n_add, in->M_pad, in->base, in->pick, in->drop, in->pd,
                                        in->cost, in->metric, c->stream);
        }));
        CK(cudaStreamSynchronize(c->stream));
        in->M = M1;
    }
    // the single-run workspace is sized for the old table; the mission-major
    // copy is stale
    dev_free(c, in->mem_ws);
    in->ws_K = 0;
    in->costT_ok = false;
    in->rowsum_ok = false;
    in->version += 1;
    return STAGE_OK;
}

stage_status stage_rank_bases(stage_ctx *c, stage_inst h, int32_t K, int32_t *out_open, int64_t *out_rowsum)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    Instance *in = find_inst(c, h);
    if (!in) return set_err(c, STAGE_ERR_NOT_FOUND, "unknown instance %llu", (unsigned long long)h);
    if (!out_open) return set_err(c, STAGE_ERR_INVALID_ARG, "out_open is NULL");
    CK(cudaSetDevice(c->device));
    return do_rank(c, in, K, out_open, out_rowsum);
}

stage_status stage_evaluate_placement(stage_ctx *c, stage_inst h, const int32_t *open, int32_t K,
                                      int32_t R, int64_t *out_cov, int64_t *out_dist)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    Instance *in = find_inst(c, h);
    if (!in) return set_err(c, STAGE_ERR_NOT_FOUND, "unknown instance %llu", (unsigned long long)h);
    if (!out_cov || !out_dist) return set_err(c, STAGE_ERR_INVALID_ARG, "output pointer is NULL");
    stage_status s = check_placement(c, in, open, K);
    if (s != STAGE_OK) return s;
    if (R < 0 || R == INT32_MAX) return set_err(c, STAGE_ERR_OUT_OF_RANGE, "R=%d outside [0, INT32_MAX)", R);
    CK(cudaSetDevice(c->device));
    s = ensure_scratch(c, in, 256 + round_up((size_t)K * 4, 256));
    if (s != STAGE_OK) return s;
    auto *acc = static_cast<unsigned long long *>(in->mem_scratch.p);
    auto *d_open = reinterpret_cast<int32_t *>(static_cast<char *>(in->mem_scratch.p) + 256);
    unsigned long long h_acc[2];
    CK(cudaMemcpyAsync(d_open, open, (size_t)K * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(acc, 0, 16, c->stream));
    CK(timed(c, "evaluate", 1, [&] { return launch_evaluate(in->cost, in->M, in->M_pad, d_open, K, R, acc, c->stream); }));
    CK(cudaMemcpyAsync(h_acc, acc, 16, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *out_cov = (int64_t)h_acc[0];
    *out_dist = (int64_t)h_acc[1];
    return STAGE_OK;
}

stage_status stage_evaluate_swaps(stage_ctx *c, stage_inst h, const int32_t *open, int32_t K,
                                  int32_t R, int64_t *out_cov, int64_t *out_dist)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    Instance *in = find_inst(c, h);
    if (!in) return set_err(c, STAGE_ERR_NOT_FOUND, "unknown instance %llu", (unsigned long long)h);
    if (!out_cov || !out_dist) return set_err(c, STAGE_ERR_INVALID_ARG, "output pointer is NULL");
    stage_status s = check_placement(c, in, open, K);
    if (s != STAGE_OK) return s;
    if (R < 0 || R == INT32_MAX) return set_err(c, STAGE_ERR_OUT_OF_RANGE, "R=%d outside [0, INT32_MAX)", R);
    CK(cudaSetDevice(c->device));
    int nC = 0;
    s = setup_search(c, in, open, K, R, 0, 0, 1, 0, nullptr, &nC);
    if (s != STAGE_OK) return s;
    const size_t n = (size_t)K * in->B;
    s = ensure_scratch(c, in, 2 * round_up(n * 8, 256));
    if (s != STAGE_OK) return s;
    auto *oc = static_cast<long long *>(in->mem_scratch.p);
    auto *od = reinterpret_cast<long long *>(static_cast<char *>(in->mem_scratch.p) + round_up(n * 8, 256));
    CK(cudaMemsetAsync(oc, 0xff, n * 8, c->stream));
    CK(cudaMemsetAsync(od, 0xff, n * 8, c->stream));
    CK(timed(c, "swap_eval", 1, [&] { return launch_swap_eval(in->tb, in->cost, nC, 1, c->stream); }));
    CK(launch_swap_table(in->tb, nC, oc, od, c->stream));
    CK(cudaMemcpyAsync(out_cov, oc, n * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(out_dist, od, n * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return STAGE_OK;
}

stage_status stage_fleet_tabu(stage_ctx *c, stage_inst h, const stage_fleet_params *p, stage_fleet_result *res,
                              stage_move *traj)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    Instance *in = find_inst(c, h);
    if (!in) return set_err(c, STAGE_ERR_NOT_FOUND, "unknown instance %llu", (unsigned long long)h);
    CK(cudaSetDevice(c->device));
    return run_fleet(c, in, p, res, traj);
}

stage_status stage_local_search(stage_ctx *c, stage_inst h, const stage_ls_params *p, stage_ls_result *res,
                                stage_move *traj)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    Instance *in = find_inst(c, h);
    if (!in) return set_err(c, STAGE_ERR_NOT_FOUND, "unknown instance %llu", (unsigned long long)h);
    CK(cudaSetDevice(c->device));
    return run_local_search(c, in, p, res, traj);
}

stage_status stage_tabu_run(stage_ctx *c, stage_inst h, const stage_tabu_params *p,
                            stage_tabu_result *res, stage_move *traj)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    Instance *in = find_inst(c, h);
    if (!in) return set_err(c, STAGE_ERR_NOT_FOUND, "unknown instance %llu", (unsigned long long)h);
    CK(cudaSetDevice(c->device));
    return run_tabu(c, in, p, res, traj, nullptr, nullptr, nullptr, nullptr);
}

stage_status stage_tabu_batch(stage_ctx *c, int32_t n, const stage_inst *insts, const stage_tabu_params *params,
                              stage_tabu_result *results, stage_move *const *trajs)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    if (n < 0) return set_err(c, STAGE_ERR_INVALID_ARG, "n=%d < 0", n);
    if (n == 0) return STAGE_OK;
    if (!insts || !params || !results) return set_err(c, STAGE_ERR_INVALID_ARG, "insts, params or results is NULL");
    CK(cudaSetDevice(c->device));
    return run_tabu_batch(c, n, insts, params, results, trajs);
}

stage_status stage_autotune(stage_ctx *c, stage_inst h, const int32_t *open, int32_t K, int32_t R, int32_t *out)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    Instance *in = find_inst(c, h);
    if (!in) return set_err(c, STAGE_ERR_NOT_FOUND, "unknown instance %llu", (unsigned long long)h);
    if (K < 1 || K > in->B || K > STAGE_MAX_K || K > in->n_avail)
        return set_err(c, STAGE_ERR_INVALID_ARG, "K=%d outside [1, min(B, %d, available bases)]", K, STAGE_MAX_K);
    if (R < 0 || R == INT32_MAX) return set_err(c, STAGE_ERR_OUT_OF_RANGE, "R=%d outside [0, INT32_MAX)", R);
    CK(cudaSetDevice(c->device));
    int seg = 0;
    stage_status s = autotune_shape(c, in, open, K, R, &seg);
    if (s == STAGE_OK && out) *out = seg;
    return s;
}

stage_status stage_best_two(stage_ctx *c, stage_inst h, const int32_t *open, int32_t K, int32_t R,
                            int32_t tabu_steps, int32_t tenure, int32_t *a, int32_t *b, int32_t *b1,
                            int32_t *b2)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    Instance *in = find_inst(c, h);
    if (!in) return set_err(c, STAGE_ERR_NOT_FOUND, "unknown instance %llu", (unsigned long long)h);
    if (!a || !b || !b1 || !b2) return set_err(c, STAGE_ERR_INVALID_ARG, "output pointer is NULL");
    CK(cudaSetDevice(c->device));
    stage_tabu_params p{};
    p.K = K;
    p.R = R;
    p.iters = tabu_steps < 0 ? 0 : tabu_steps;
    p.tenure = tenure;
    p.accept_worsening = 1;
    p.start_open = open;
    return run_tabu(c, in, &p, nullptr, nullptr, a, b, b1, b2);
}

stage_status stage_read_table(stage_ctx *c, stage_inst h, int32_t b0, int32_t nb, int32_t m0,
                              int32_t nm, int32_t *out)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    Instance *in = find_inst(c, h);
    if (!in) return set_err(c, STAGE_ERR_NOT_FOUND, "unknown instance %llu", (unsigned long long)h);
    if (!out || b0 < 0 || nb < 0 || m0 < 0 || nm < 0 || b0 + nb > in->B || m0 + nm > in->M_pad)
        return set_err(c, STAGE_ERR_INVALID_ARG, "table window out of range");
    if (nb == 0 || nm == 0) return STAGE_OK;
    CK(cudaSetDevice(c->device));
    // columns are stored in the engine's mission order: gather the window back
    DevBuf win;
    stage_status s = dev_alloc(c, (size_t)nb * nm * 4, win);
    if (s != STAGE_OK) return s;
    cudaError_t e = launch_gather_window(in->cost, in->M, in->M_pad, in->inv, b0, nb, m0, nm,
                                         static_cast<int32_t *>(win.p), c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, win.p, (size_t)nb * nm * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, win);
    if (e != cudaSuccess) return set_err(c, STAGE_ERR_CUDA, "reading the table failed: %s", cudaGetErrorString(e));
    return STAGE_OK;
}

stage_status stage_test_batch_schedule(int32_t n, const double *us, const int32_t *gang, int32_t P,
                                       int32_t *out_off, int32_t *out_entries, double *out_makespan_us)
{
    if (n < 0 || P < 1 || (n > 0 && (!us || !gang || !out_entries)) || !out_off) return STAGE_ERR_INVALID_ARG;
    std::vector<int> g(n);
    for (int k = 0; k < n; k++) {
        if (gang[k] < 1 || gang[k] > P) return STAGE_ERR_INVALID_ARG;
        g[k] = gang[k];
    }
    std::vector<std::vector<int2>> lists;
    std::vector<int> order;
    const double mk = n > 0 ? batch_place(n, us, g.data(), P, lists, order) : 0.0;
    if (n == 0) lists.assign(P, {});
    int at = 0;
    for (int q = 0; q < P; q++) {
        out_off[q] = at;
        for (const int2 &e : lists[q]) {
            out_entries[2 * at] = order[e.x];   // the caller's search index
            out_entries[2 * at + 1] = e.y;
            at++;
        }
    }
    out_off[P] = at;
    if (out_makespan_us) *out_makespan_us = mk;
    return STAGE_OK;
}

stage_status stage_test_wait_timeout(stage_ctx *c)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    if (cudaSetDevice(c->device) != cudaSuccess) return set_err(c, STAGE_ERR_CUDA, "cudaSetDevice failed");
    DevBuf buf;
    stage_status s = dev_alloc(c, 256, buf);
    if (s != STAGE_OK) return s;
    unsigned *flag = static_cast<unsigned *>(buf.p);
    int *err = reinterpret_cast<int *>(static_cast<char *>(buf.p) + 64);
    int h_err = 0;
    cudaError_t e = cudaMemsetAsync(buf.p, 0, 256, c->stream);
    if (e == cudaSuccess) e = launch_wait_unset_flag(flag, c->spin_limit, err, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof h_err, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, buf);
    if (e != cudaSuccess) return set_err(c, STAGE_ERR_CUDA, "bounded-wait test failed: %s", cudaGetErrorString(e));
    if (h_err & kErrPipelineTimeout)
        return set_err(c, STAGE_ERR_TIMEOUT, "the device-side wait gave up after %lld polls", (long long)c->spin_limit);
    return STAGE_OK;
}

stage_status stage_kernel_stats(stage_ctx *c, const char *kernel, int64_t *launches, double *total_ms)
{
    if (!c || !kernel) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    cudaSetDevice(c->device);
    fold_stats(c);
    auto it = c->stats.find(kernel);
    if (launches) *launches = it == c->stats.end() ? 0 : it->second.launches;
    if (total_ms) *total_ms = it == c->stats.end() ? 0.0 : it->second.ms;
    return STAGE_OK;
}

stage_status stage_reset_stats(stage_ctx *c)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    Guard g(c);
    cudaSetDevice(c->device);
    fold_stats(c);
    c->stats.clear();
    return STAGE_OK;
}

}  // extern "C"
