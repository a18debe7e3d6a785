// Batch engine: stage_batch_submit / stage_poll.
//
// Requests (one Tabu search each, on a resident instance or on an instance
// given inline) wait in a FIFO.  A worker thread admits them into slots while
// slots and device memory are free, and advances every active slot together:
// one grouped launch of the swap evaluation, one of the move selection (a block
// per slot) and one of the refresh per Tabu step, captured as a CUDA graph of
// kStepsPerGraph steps and replayed while the set of slots is unchanged.
// Between replays finished slots retire (results copied to the caller's
// buffers, memory released) and waiting requests join: continuous batching.
// Slots whose shape the persistent search takes (K <= 256, at most 2048 bases;
// not with STAGE_NO_PERSIST or STAGE_FULL_PASS) run their first full pass at
// admission and are then advanced, every round, by one cooperative launch of
// the persistent batch body (each on a gang of CTAs placed when the slot set
// changes), kPersistRoundSteps iterations per launch; the others by the grouped
// launches.
// Every slot runs exactly the search stage_tabu_run would run alone, so each
// result is independent of what else is in the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <unordered_set>

#include "runtime_internal.h"

using namespace stg;

namespace stg_rt {

namespace {

constexpr int kStepsPerGraph = 8;
constexpr int kPersistRoundSteps = 16;  // iterations of the persistent slots per round (8: the same latency, 543 inst/s batched; 32: p99 223 ms)
constexpr int kLanes = 2;   // lanes of slots advanced on their own streams (see Engine::Lane)

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Ticket {
    uint64_t id = 0;
    stage_request req{};
    std::vector<int32_t> start;            // copy of params.start_open
    bool has_update = false;
    std::vector<int32_t> add_pick, add_drop, remove_ids, unavail_ids, avail_ids;
    bool inline_inst = false;              // instance given by value: loaded and unloaded here
    std::vector<int32_t> d_base, d_pick, d_drop;
    std::vector<uint8_t> d_avail;
    uint32_t d_flags = 0;                  // STAGE_DESC_HAVERSINE of the inline instance
    stage_inst inst = 0;
    stage_result res{};
    int state = 0;                         // 0 pending, 1 running, 2 done
    bool released = false;                 // came back from waiting on its busy instance: goes first
};

struct Slot {
    Ticket *tk = nullptr;
    Instance *in = nullptr;
    DevBuf ws;
    DevBuf chg;               // incremental slots: the refresh's change records
    TabuBuffers tb{};
    int nC = 0;
    bool first_done = false;  // incremental slots: the first full pass has run
    bool persist = false;     // advanced by the persistent batch launch
    DevBuf pscratch;          // its scratch for that launch (sized for its gang)
    double cov = 0.5;         // covered fraction of the start placement (its gang's estimate)
};

// Slots whose candidate rows x missions reach this many table bytes keep the
// swap terms across steps (the incremental neighbourhood of a single search:
// one full pass, then per step the records of the missions a move touched);
// smaller ones stream their table every step.  Lower than the single search's
// threshold: a batch's tables share L2 and are streamed from HBM anyway.
constexpr size_t kEngineIncrementalMinBytes = 8ull << 20;

}  // namespace

struct Engine {
    stage_ctx *c = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Ticket *> pending;
    std::unordered_map<uint64_t, std::unique_ptr<Ticket>> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    cudaStream_t stream = nullptr;
    std::vector<Slot> active;
    DevBuf d_slots, d_map, d_states;
    int cap = 0;
    size_t map_cap = 0;       // int2 entries of d_map
    TabuDevState *h_states = nullptr;      // pinned
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t ev_round[2] = {nullptr, nullptr};   // brackets each round on the engine stream
    bool dirty = true;        // slot set changed: device arrays must be rebuilt
    int stable = 0;           // rounds since the last change (the graph is captured once stable)
    // Lanes: the active slots are split into kLanes sets of about equal swap
    // work, each advanced by its own launches on its own stream, so one lane's
    // latency-bound selection and refresh overlap another's streaming swap
    // pass instead of leaving SMs idle between kernels.
    struct Lane {
        int n_swap = 0, n_sel = 0, n_ref = 0, n_delta = 0, maxK = 1;
        size_t swap_smem = 0;
        size_t map_off = 0;   // first entry of this lane's block maps in d_map
    };
    Lane lane[kLanes];
    // the persistent slots' launch: their arguments, the schedule and the
    // per-CTA offsets (device), the grid and its dynamic shared memory
    DevBuf d_pbuf;
    const void *p_args = nullptr;
    const int2 *p_sched = nullptr;
    const int *p_off = nullptr;
    int p_n = 0, p_grid = 0;
    size_t p_smem = 0;
    cudaEvent_t ev_p[2] = {nullptr, nullptr};
    cudaStream_t lane_stream[kLanes] = {};   // lane_stream[0] is `stream`
    cudaEvent_t ev_fork = nullptr, ev_join[kLanes] = {};
    int lane_begin[kLanes + 1] = {};         // active[lane_begin[l], lane_begin[l + 1]) is lane l

    // requests waiting for their instance's current search to finish, per instance, in order
    std::unordered_map<stage_inst, std::deque<Ticket *>> parked;
    // instances whose next request was released from `parked` and waits in
    // `pending`: until it is admitted (or fails for good) later requests on the
    // instance park behind it, so requests on one instance keep their order
    std::unordered_map<stage_inst, int> releasing;
    void unrelease(stage_inst h)
    {
        auto it = releasing.find(h);
        if (it != releasing.end() && --it->second <= 0) releasing.erase(it);
    }
    std::vector<struct Retiring> retiring;   // finished in the last round, released during the next
    void retire_pending();

    void run();
    void release_streams()
    {
        for (int l = 0; l < kLanes; l++) {
            if (lane_stream[l]) cudaStreamDestroy(lane_stream[l]);
            if (ev_join[l]) cudaEventDestroy(ev_join[l]);
            lane_stream[l] = nullptr;
            ev_join[l] = nullptr;
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        ev_fork = nullptr;
        stream = nullptr;
    }
    cudaError_t launch_steps(int steps);
    bool admit(Ticket *tk, bool &transient, stage_inst &busy_on);
    void complete(Ticket *tk, stage_status st);
    void retire_copy(struct Retiring &r);
    void retire_finish(struct Retiring &r, bool copies_ok);
    stage_status rebuild();
};

namespace {

stage_status copy_update(Ticket *tk, const stage_update *u)
{
    if (!u) return STAGE_OK;
    auto take = [](std::vector<int32_t> &dst, const int32_t *src, int32_t n, int per) {
        if (n < 0 || (n > 0 && !src)) return false;
        dst.assign(src, src + (size_t)n * per);
        return true;
    };
    if (!take(tk->add_pick, u->add_pick_xy, u->n_add, 2) || !take(tk->add_drop, u->add_drop_xy, u->n_add, 2) ||
        !take(tk->remove_ids, u->remove_ids, u->n_remove, 1) ||
        !take(tk->unavail_ids, u->unavail_ids, u->n_unavail, 1) || !take(tk->avail_ids, u->avail_ids, u->n_avail, 1))
        return STAGE_ERR_INVALID_ARG;
    tk->has_update = true;
    return STAGE_OK;
}

}  // namespace

void Engine::complete(Ticket *tk, stage_status st)
{
    std::lock_guard<std::mutex> lk(mu);
    tk->res.status = st;
    tk->res.t_end_ns = now_ns();
    tk->state = 2;
    cv_done.notify_all();
}

// Admit one request into a new slot.  On a memory shortage returns false with
// transient = true; when its instance is busy in another slot, returns false
// with busy_on = that instance (the request then waits on the instance).
bool Engine::admit(Ticket *tk, bool &transient, stage_inst &busy_on)
{
    transient = false;
    busy_on = 0;
    std::lock_guard<std::recursive_mutex> g(c->mu);
    stage_status s = STAGE_OK;
    if (!tk->inst) {
        if (tk->inline_inst) {
            stage_instance_desc d{};
            d.B = (int32_t)(tk->d_base.size() / 2);
            d.M = (int32_t)(tk->d_pick.size() / 2);
            d.base_xy = tk->d_base.data();
            d.pick_xy = tk->d_pick.data();
            d.drop_xy = tk->d_drop.data();
            d.base_available = tk->d_avail.empty() ? nullptr : tk->d_avail.data();
            d.flags = tk->d_flags;
            stage_inst h = 0;
            c->load_without_copy = true;   // (the context lock is held)
            s = stage_load_instance(c, &d, &h);
            c->load_without_copy = false;
            if (s == STAGE_ERR_ADMISSION || s == STAGE_ERR_NO_MEMORY) {
                transient = !active.empty();
                if (!transient) complete(tk, s);
                return false;
            }
            if (s != STAGE_OK) {
                complete(tk, s);
                return false;
            }
            tk->inst = h;
        }
    }
    Instance *in = find_inst(c, tk->inst);
    if (!in) {
        set_err(c, STAGE_ERR_NOT_FOUND, "unknown instance %llu", (unsigned long long)tk->inst);
        complete(tk, STAGE_ERR_NOT_FOUND);
        return false;
    }
    if (in->busy || (!tk->released && (parked.count(tk->inst) || releasing.count(tk->inst)))) {
        busy_on = tk->inst;   // one request per instance at a time: updates and searches stay ordered
        return false;
    }
    auto fail = [&](stage_status st) {
        if (tk->inline_inst) {
            stage_unload_instance(c, tk->inst);
            tk->inst = 0;
        }
        complete(tk, st);
        return false;
    };
    if (tk->has_update) {
        stage_update u{};
        u.n_add = (int32_t)(tk->add_pick.size() / 2);
        u.add_pick_xy = tk->add_pick.data();
        u.add_drop_xy = tk->add_drop.data();
        u.n_remove = (int32_t)tk->remove_ids.size();
        u.remove_ids = tk->remove_ids.data();
        u.n_unavail = (int32_t)tk->unavail_ids.size();
        u.unavail_ids = tk->unavail_ids.data();
        u.n_avail = (int32_t)tk->avail_ids.size();
        u.avail_ids = tk->avail_ids.data();
        s = stage_update_instance(c, tk->inst, &u);
        if (s != STAGE_OK) return fail(s);
        tk->has_update = false;   // applied once, even if admission is retried
    }
    const stage_tabu_params &p = tk->req.params;
    const int K = p.K;
    if (K < 1 || K > in->B || K > kGroupMaxK || K > in->n_avail) {
        set_err(c, STAGE_ERR_INVALID_ARG, "K=%d outside [1, min(B, %d, available bases)] for a batch request",
                K, kGroupMaxK);
        return fail(STAGE_ERR_INVALID_ARG);
    }
    if (p.R < 0 || p.R == INT32_MAX || p.iters < 0 || p.tenure < 0 || p.resume) {
        set_err(c, STAGE_ERR_INVALID_ARG, "batch request: bad R / iters / tenure, or resume given");
        return fail(STAGE_ERR_INVALID_ARG);
    }
    std::vector<int32_t> start(K);
    // the instance's resident state (A15 forced moves after an update)
    const ResidentState &rsd = in->resident;
    const bool from_resident = tk->req.resume_resident && !tk->inline_inst && rsd.valid && rsd.K == K &&
                               (int)rsd.expiry.size() == in->B && (int)rsd.open.size() == K;
    std::vector<int32_t> expiry0(in->B, 0);
    int t0 = 0, n_forced = 0;
    const bool keep_best = from_resident && rsd.version == in->version;
    if (from_resident) {
        start = rsd.open;
        expiry0 = rsd.expiry;
        t0 = rsd.t;
        s = forced_moves(c, in, start.data(), K, p.R, t0, p.tenure, expiry0.data(), &n_forced);
        if (s != STAGE_OK) return fail(s);
    } else if (!tk->start.empty()) {
        s = check_placement(c, in, tk->start.data(), K);
        if (s != STAGE_OK) return fail(s);
        start = tk->start;
    } else {
        s = do_rank(c, in, K, start.data(), nullptr);
        if (s != STAGE_OK) return fail(s);
    }
    if (c->flags & STAGE_AUTOTUNE) {
        const int nc0 = in->n_avail - K;
        if (!swap_segment_known(in->M_pad, nc0, K)) {
            s = autotune_shape(c, in, start.data(), K, p.R, nullptr);
            if (s != STAGE_OK) return fail(s);
        }
    }
    Slot sl;
    sl.tk = tk;
    sl.in = in;
    TabuBuffers tb{};
    const size_t bytes = carve_ws(nullptr, K, in->B, in->M_pad, p.iters, tb);
    s = dev_alloc(c, bytes, sl.ws);
    if (s != STAGE_OK) {
        if (s == STAGE_ERR_ADMISSION || s == STAGE_ERR_NO_MEMORY) {
            transient = !active.empty();
            if (!transient) return fail(s);
            return false;
        }
        return fail(s);
    }
    carve_ws(static_cast<char *>(sl.ws.p), K, in->B, in->M_pad, p.iters, tb);
    tb.K = K;
    tb.B = in->B;
    tb.M = in->M;
    tb.M_pad = in->M_pad;
    tb.R = p.R;
    // the incremental form where the table is large enough and there is room
    // for the mission-major copy and the records (else a full pass per step)
    bool pmode = false;
    {
        int nc_est = 0;
        for (int b = 0; b < in->B; b++) nc_est += in->h_avail[b];
        nc_est -= K;
        pmode = !(c->flags & (STAGE_FULL_PASS | STAGE_NO_PERSIST)) && swap_delta_fits(K) && nc_est > 0 &&
                p.iters > 0 && persist_shape_ok(K, in->B, table_ldT(in->B));
        const bool want = !(c->flags & STAGE_FULL_PASS) && swap_delta_fits(K) && nc_est > 0 &&
                          (pmode || (c->flags & STAGE_INCREMENTAL) ||
                           (size_t)nc_est * in->M_pad * sizeof(int32_t) >= kEngineIncrementalMinBytes);
        // a persistent slot's scratch, for the largest gang it can be given (so
        // that placing it later allocates nothing)
        if (pmode) {
            const int ldT = table_ldT(in->B);
            const int gcap = std::min({persist_max_gang(), persist_batch_grid(persist_search_smem(K, in->B, ldT)),
                                       (in->M_pad + 31) / 32});
            size_t need = 0;   // over the gangs it can be given: powers of two up to gcap
            for (int g = 1; g <= gcap; g *= 2) need = std::max(need, persist_scratch_bytes(K, g, in->M_pad));
            if (gcap < 1 || dev_alloc(c, need, sl.pscratch) != STAGE_OK) {
                pmode = false;
                dev_free(c, sl.pscratch);
                set_err(c, STAGE_OK, "");   // a refused buffer only means the grouped launches
            }
        }
        if (want && ensure_costT(c, in) == STAGE_OK &&
            dev_alloc(c, (size_t)in->M_pad * 2 * sizeof(int4), sl.chg) == STAGE_OK) {
            tb.chg = static_cast<int4 *>(sl.chg.p);
            tb.costT = static_cast<const int32_t *>(in->mem_costT.p);
            tb.border = tb.costT + (size_t)in->M_pad * in->ldT;
            tb.cellmin = tb.border + in->ldT;
            tb.ldT = in->ldT;
        } else {
            dev_free(c, sl.chg);
            dev_free(c, sl.pscratch);
            pmode = false;
            set_err(c, STAGE_OK, "");   // a refused buffer only means the full pass
        }
        if (!pmode) dev_free(c, sl.pscratch);
    }
    std::vector<uint8_t> is_open(in->B, 0);
    for (int k = 0; k < K; k++) is_open[start[k]] = 1;
    std::vector<int32_t> cand;
    for (int b = 0; b < in->B; b++)
        if (in->h_avail[b] && !is_open[b]) cand.push_back(b);
    sl.nC = (int)cand.size();
    TabuDevState st{};
    st.t = t0;
    st.tenure = p.tenure;
    st.accept_worsening = p.accept_worsening ? 1 : 0;
    st.nC = sl.nC;
    st.traj_cap = p.iters;
    st.best_iter = -1;
    st.t_end = t0 + p.iters;
    if (keep_best) {   // resumed with no update since: the best so far carries over
        st.best_iter = rsd.best_iter;
        st.best_cov = rsd.best_cov;
        st.best_dist = rsd.best_dist;
    }
    // set-up runs on the context's stream: the engine's stream may be busy
    // with the current step, which this slot is not part of
    cudaStream_t stream = c->stream;
    cudaError_t e = cudaMemcpyAsync(tb.open, start.data(), (size_t)K * 4, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && sl.nC)
        e = cudaMemcpyAsync(tb.cand, cand.data(), (size_t)sl.nC * 4, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tb.expiry, expiry0.data(), (size_t)in->B * 4, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && keep_best)
        e = cudaMemcpyAsync(tb.best_open, rsd.best_open.data(), (size_t)K * 4, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tb.st, &st, sizeof st, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.v0, 0, 16, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.loss_c, 0, (size_t)K * 8, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.loss_d, 0, (size_t)K * 8, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.gain_c, 0, (size_t)in->B * 4, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.gain_d, 0, (size_t)in->B * 8, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.extra_c, 0, (size_t)K * in->B * 4, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.extra_d, 0, (size_t)K * in->B * 8, stream);
    if (e == cudaSuccess) e = timed_on(c, stream, "init", 1, [&] { return launch_init(tb, in->cost, stream); });
    if (e == cudaSuccess)
        e = timed_on(c, stream, "begin", 1, [&] { return launch_begin(tb, keep_best ? 1 : 0, stream); });
    // a persistent slot's first full pass (its swap terms, then kept move by move)
    // and its start placement's covered count
    unsigned long long v0h[2] = {0, 0};
    if (e == cudaSuccess && pmode && sl.nC > 0) {
        e = timed_on(c, stream, "swap_eval", 1, [&] { return launch_swap_eval(tb, in->cost, sl.nC, 0, stream); });
        if (e == cudaSuccess) e = cudaMemcpyAsync(v0h, tb.v0, 16, cudaMemcpyDeviceToHost, stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);   // host vectors above go out of scope
    if (in->M > 0) sl.cov = std::min(1.0, (double)v0h[0] / in->M);
    if (e != cudaSuccess) {
        dev_free(c, sl.ws);
        dev_free(c, sl.chg);
        dev_free(c, sl.pscratch);
        set_err(c, STAGE_ERR_CUDA, "batch slot set-up failed: %s", cudaGetErrorString(e));
        return fail(STAGE_ERR_CUDA);
    }
    sl.tb = tb;
    sl.persist = pmode && sl.nC > 0;
    if (!sl.persist) dev_free(c, sl.pscratch);
    sl.first_done = sl.first_done || sl.persist;
    in->busy += 1;
    tk->res.n_forced = n_forced;
    {
        std::lock_guard<std::mutex> lk(mu);
        tk->state = 1;
        tk->res.t_start_ns = now_ns();
    }
    active.push_back(sl);
    dirty = true;
    return true;
}

stage_status Engine::rebuild()
{
    const int n = (int)active.size();
    if (graph) {
        cudaGraphExecDestroy(graph);
        graph = nullptr;
    }
    if (n > cap) {
        std::lock_guard<std::recursive_mutex> g(c->mu);
        dev_free(c, d_slots);
        dev_free(c, d_states);
        if (h_states) cudaFreeHost(h_states);
        h_states = nullptr;
        cap = std::max(n, std::max(cap * 2, 16));
        stage_status s = dev_alloc(c, sizeof(GroupSlot) * (size_t)cap, d_slots);
        if (s == STAGE_OK) s = dev_alloc(c, sizeof(TabuDevState) * (size_t)cap, d_states);
        if (s != STAGE_OK) return s;
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return STAGE_ERR_CUDA;   // allocations ordered there
        if (cudaMallocHost(&h_states, sizeof(TabuDevState) * (size_t)cap) != cudaSuccess) return STAGE_ERR_CUDA;
    }
    // split into lanes by swap work (largest first, to the lightest lane);
    // lane l's slots are contiguous in `active`
    {
        std::vector<int> order(n);
        for (int k = 0; k < n; k++) order[k] = k;
        auto work = [&](int k) { return (double)active[k].nC * active[k].tb.M_pad; };
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
        double load[kLanes] = {};
        std::vector<int> side(n, 0);
        for (int k : order) {
            int l = 0;
            for (int q = 1; q < kLanes; q++)
                if (load[q] < load[l]) l = q;
            side[k] = l;
            load[l] += work(k);
        }
        std::vector<Slot> re;
        re.reserve(n);
        for (int l = 0; l < kLanes; l++) {
            lane_begin[l] = (int)re.size();
            for (int k = 0; k < n; k++)
                if (side[k] == l) re.push_back(active[k]);
        }
        lane_begin[kLanes] = n;
        active.swap(re);
    }
    std::vector<GroupSlot> gs(n);
    std::vector<int> mp(n), nc(n);
    for (int k = 0; k < n; k++) {
        mp[k] = active[k].tb.M_pad;
        nc[k] = active[k].nC;
    }
    const int common = group_common_segment(mp.data(), nc.data(), n);
    for (int k = 0; k < n; k++) {
        const Slot &sl = active[k];
        gs[k].w = sl.tb;
        gs[k].cost = sl.in->cost;
        gs[k].swap_blocks =
            group_swap_blocks(sl.tb.M_pad, sl.nC, sl.tb.K, common, &gs[k].swap_bx, &gs[k].swap_seg);
        gs[k].delta_bx = gs[k].delta_by = 0;
        if (sl.tb.chg) {
            group_delta_blocks(sl.tb.ldT, sl.tb.M, sl.tb.K, &gs[k].delta_bx, &gs[k].delta_by);
            if (sl.first_done) gs[k].swap_blocks = 0;   // its terms are kept by the delta step
        }
        gs[k].sel_blocks = select_blocks(sl.tb.K, sl.nC);
        gs[k].ref_blocks = group_ref_blocks(sl.tb.M_pad);
        if (sl.persist) {   // advanced by the persistent launch only
            gs[k].swap_blocks = gs[k].sel_blocks = gs[k].ref_blocks = 0;
            gs[k].delta_bx = gs[k].delta_by = 0;
        }
    }
    std::vector<int2> map;   // per lane: swap blocks, then select blocks, then refresh blocks
    for (int l = 0; l < kLanes; l++) {
        Lane &ln = lane[l];
        const int k0 = lane_begin[l], k1 = lane_begin[l + 1];
        ln = Lane{};
        ln.map_off = map.size();
        for (int k = k0; k < k1; k++) {
            for (int b = 0; b < gs[k].swap_blocks; b++) map.push_back(make_int2(k, b));
            ln.swap_smem = std::max(ln.swap_smem, swap_direct_smem(active[k].tb.K));
            ln.maxK = std::max(ln.maxK, active[k].tb.K);
        }
        ln.n_swap = (int)(map.size() - ln.map_off);
        for (int k = k0; k < k1; k++)
            for (int b = 0; b < gs[k].sel_blocks; b++) map.push_back(make_int2(k, b));
        ln.n_sel = (int)(map.size() - ln.map_off) - ln.n_swap;
        for (int k = k0; k < k1; k++)
            for (int b = 0; b < gs[k].ref_blocks; b++) map.push_back(make_int2(k, b));
        ln.n_ref = (int)(map.size() - ln.map_off) - ln.n_swap - ln.n_sel;
        for (int k = k0; k < k1; k++)
            for (int b = 0; b < gs[k].delta_bx * gs[k].delta_by; b++) map.push_back(make_int2(k, b));
        ln.n_delta = (int)(map.size() - ln.map_off) - ln.n_swap - ln.n_sel - ln.n_ref;
    }
    if (map.size() > map_cap) {
        std::lock_guard<std::recursive_mutex> g(c->mu);
        dev_free(c, d_map);
        map_cap = std::max(map.size(), 2 * map_cap);
        if (dev_alloc(c, sizeof(int2) * map_cap, d_map) != STAGE_OK) {
            map_cap = 0;
            return STAGE_ERR_NO_MEMORY;
        }
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return STAGE_ERR_CUDA;
    }
    cudaError_t e = cudaMemcpyAsync(d_slots.p, gs.data(), sizeof(GroupSlot) * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_map.p, map.data(), sizeof(int2) * map.size(), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return STAGE_ERR_CUDA;
    // the persistent slots: gang sizes (the smallest power of two that brings
    // a slot's round under half of the ideal per-CTA time, from the estimate of
    // the one-launch batch), placement, scratch and arguments
    p_n = 0;
    std::vector<int> pk;
    for (int k = 0; k < n; k++)
        if (active[k].persist) pk.push_back(k);
    if (!pk.empty()) {
        const int np = (int)pk.size();
        size_t smem = 0;
        std::vector<double> us(np);
        double total = 0.0;
        for (int i = 0; i < np; i++) {
            const Slot &sl = active[pk[i]];
            smem = std::max(smem, persist_search_smem(sl.tb.K, sl.in->B, sl.tb.ldT));
            // the instance's measured work in a batch launch for this K and R,
            // else the estimate from the start placement's covered fraction
            const Instance *in = sl.in;
            us[i] = in->batch_K == sl.tb.K && in->batch_R == sl.tb.R && in->batch_version == in->version &&
                            in->batch_work_us > 0.0
                        ? in->batch_work_us
                        : persist_iter_us_estimate(in, sl.tb.K, sl.nC, sl.cov);
            total += kPersistRoundSteps * (5.0 + us[i]);
        }
        const int P = persist_batch_grid(smem);
        if (P < 1) return STAGE_ERR_INTERNAL;
        const double ideal = total / P;
        std::vector<int> gang(np, 1);
        std::vector<double> work(np);
        auto round_us = [&](int i, int g) { return kPersistRoundSteps * (5.0 + (g > 1 ? 4.0 : 0.0) + us[i] / g); };
        for (int i = 0; i < np; i++) {
            const Slot &sl = active[pk[i]];
            const int gmax = std::min({persist_max_gang(), P, (sl.tb.M_pad + 31) / 32});
            while (gang[i] * 2 <= gmax && round_us(i, gang[i]) > 0.5 * ideal) gang[i] *= 2;
            work[i] = round_us(i, gang[i]);
        }
        std::vector<std::vector<int2>> lists;
        std::vector<int> order;
        batch_place(np, work.data(), gang.data(), P, lists, order);
        const size_t ab = persist_args_bytes();
        std::vector<unsigned char> h_args(ab * np);
        for (int pos = 0; pos < np; pos++) {
            const int i = order[pos];
            Slot &sl = active[pk[i]];
            const size_t need = persist_scratch_bytes(sl.tb.K, gang[i], sl.tb.M_pad);
            if (!sl.pscratch.p || sl.pscratch.bytes < need) {
                std::lock_guard<std::recursive_mutex> g(c->mu);
                dev_free(c, sl.pscratch);
                stage_status st = dev_alloc(c, need, sl.pscratch);
                if (st != STAGE_OK) return st;
            }
            if (persist_args_host(sl.tb, sl.in->cost, sl.pscratch.p, gang[i], c->spin_limit, stream,
                                  h_args.data() + ab * pos) != cudaSuccess)
                return STAGE_ERR_CUDA;
        }
        std::vector<int2> h_sched;
        std::vector<int> h_off(P + 1, 0);
        for (int q = 0; q < P; q++) {
            h_off[q] = (int)h_sched.size();
            h_sched.insert(h_sched.end(), lists[q].begin(), lists[q].end());
        }
        h_off[P] = (int)h_sched.size();
        const size_t off_sched = round_up(h_args.size(), 256),
                     off_off = off_sched + round_up(h_sched.size() * sizeof(int2), 256),
                     bytes = off_off + round_up(h_off.size() * sizeof(int), 256);
        if (!d_pbuf.p || d_pbuf.bytes < bytes) {
            std::lock_guard<std::recursive_mutex> g(c->mu);
            dev_free(c, d_pbuf);
            stage_status st = dev_alloc(c, bytes, d_pbuf);
            if (st != STAGE_OK) return st;
        }
        // new buffers are allocated in order on the context stream: finish it
        // before the engine's stream uses them
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return STAGE_ERR_CUDA;
        char *d = static_cast<char *>(d_pbuf.p);
        e = cudaMemcpyAsync(d, h_args.data(), h_args.size(), cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d + off_sched, h_sched.data(), h_sched.size() * sizeof(int2), cudaMemcpyHostToDevice,
                                stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d + off_off, h_off.data(), h_off.size() * sizeof(int), cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);   // the host arrays above
        if (e != cudaSuccess) return STAGE_ERR_CUDA;
        p_args = d;
        p_sched = reinterpret_cast<const int2 *>(d + off_sched);
        p_off = reinterpret_cast<const int *>(d + off_off);
        p_n = np;
        p_grid = P;
        p_smem = smem;
    }
    dirty = false;
    stable = 0;
    return STAGE_OK;
}

// kStepsPerGraph grouped steps of every lane (lanes 1.. forked onto their
// streams and joined back): launched directly while the slot set keeps
// changing, replayed from a captured CUDA graph once it has been stable.
cudaError_t Engine::launch_steps(int steps)
{
    const GroupSlot *ds = static_cast<const GroupSlot *>(d_slots.p);
    auto enqueue_lane = [&](const Lane &ln, cudaStream_t s) {
        const int2 *map_swap = static_cast<const int2 *>(d_map.p) + ln.map_off;
        const int2 *map_sel = map_swap + ln.n_swap;
        const int2 *map_ref = map_sel + ln.n_sel;
        const int2 *map_delta = map_ref + ln.n_ref;
        cudaError_t e = cudaSuccess;
        for (int k = 0; e == cudaSuccess && k < steps; k++) {
            e = launch_group_swap(ds, map_swap, ln.n_swap, ln.swap_smem, s);
            if (e == cudaSuccess) e = launch_group_select(ds, map_sel, ln.n_sel, s);
            if (e == cudaSuccess) e = launch_group_refresh(ds, map_ref, ln.n_ref, ln.maxK, s);
            if (e == cudaSuccess) e = launch_group_delta(ds, map_delta, ln.n_delta, s);
        }
        return e;
    };
    auto used = [&](int l) { return lane[l].n_swap + lane[l].n_sel + lane[l].n_ref + lane[l].n_delta > 0; };
    {
        bool any = false;
        for (int l = 0; l < kLanes; l++) any = any || used(l);
        if (!any) return cudaSuccess;   // every slot is advanced by the persistent launch
    }
    auto enqueue = [&]() {
        cudaError_t e = cudaEventRecord(ev_fork, stream);
        for (int l = 1; e == cudaSuccess && l < kLanes; l++)
            if (used(l)) e = cudaStreamWaitEvent(lane_stream[l], ev_fork, 0);
        for (int l = 0; e == cudaSuccess && l < kLanes; l++)
            if (used(l)) e = enqueue_lane(lane[l], lane_stream[l]);
        for (int l = 1; e == cudaSuccess && l < kLanes; l++)
            if (used(l)) {
                e = cudaEventRecord(ev_join[l], lane_stream[l]);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev_join[l], 0);
            }
        return e;
    };
    if (stable < 1) return enqueue();
    if (!graph) {
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = enqueue();
        cudaError_t e2 = cudaStreamEndCapture(stream, &gr);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&graph, gr, 0);
        if (gr) cudaGraphDestroy(gr);
        if (e != cudaSuccess) {
            cudaGetLastError();
            graph = nullptr;
            return enqueue();
        }
    }
    return cudaGraphLaunch(graph, stream);
}

// Retiring slots: a slot that finished in round N leaves the active set before
// round N+1 is launched, and its read-backs (retire_copy, on the context
// stream, all waited for once) and release (retire_finish) run on the host
// while round N+1 runs on the device.
struct Retiring {
    Slot sl;
    TabuDevState s;
    stage_status status;
    std::vector<int32_t> fin, best, expiry;   // fin and best in slot order until published
};

void Engine::retire_copy(Retiring &r)
{
    Slot &sl = r.sl;
    Ticket *tk = sl.tk;
    const int K = sl.tb.K;
    r.fin.assign(K, 0);
    r.best.assign(K, 0);
    // on the context stream: the engine's streams already run the next round
    cudaStream_t cs = c->stream;
    cudaError_t e = cudaMemcpyAsync(r.fin.data(), sl.tb.open, (size_t)K * 4, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r.best.data(), sl.tb.best_open, (size_t)K * 4, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess && tk->req.resume_resident && !tk->inline_inst) {   // kept as the resident state
        r.expiry.assign(sl.in->B, 0);
        e = cudaMemcpyAsync(r.expiry.data(), sl.tb.expiry, (size_t)sl.in->B * 4, cudaMemcpyDeviceToHost, cs);
    }
    const int n = std::min(r.s.n_moves, tk->req.params.iters);
    if (e == cudaSuccess && tk->req.traj && n > 0)
        e = cudaMemcpyAsync(tk->req.traj, sl.tb.traj, (size_t)n * sizeof(stage_move), cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess && r.status == STAGE_OK) r.status = STAGE_ERR_CUDA;
}

void Engine::retire_finish(Retiring &r, bool copies_ok)
{
    Slot &sl = r.sl;
    Ticket *tk = sl.tk;
    stage_status status = r.status;
    if (!copies_ok && status == STAGE_OK) status = STAGE_ERR_CUDA;
    if (r.s.err && status == STAGE_OK) status = STAGE_ERR_INTERNAL;
    if (tk->req.resume_resident && !tk->inline_inst) {
        ResidentState &rs = sl.in->resident;
        rs.valid = status == STAGE_OK && (int)r.expiry.size() == sl.in->B;
        rs.K = sl.tb.K;
        rs.t = r.s.t;
        rs.best_iter = r.s.best_iter;
        rs.best_cov = r.s.best_cov;
        rs.best_dist = r.s.best_dist;
        rs.version = sl.in->version;
        rs.open = r.fin;
        rs.best_open = r.best;
        rs.expiry = r.expiry;
    }
    std::sort(r.fin.begin(), r.fin.end());
    std::sort(r.best.begin(), r.best.end());
    if (tk->req.best_open) std::copy(r.best.begin(), r.best.end(), tk->req.best_open);
    if (tk->req.final_open) std::copy(r.fin.begin(), r.fin.end(), tk->req.final_open);
    tk->res.n_moves = r.s.n_moves;
    tk->res.best_iter = r.s.best_iter;
    tk->res.best_cov = r.s.best_cov;
    tk->res.best_dist = r.s.best_dist;
    tk->res.final_cov = r.s.cur_cov;
    tk->res.final_dist = r.s.cur_dist;
    const stage_inst inst = tk->inst;
    {
        std::lock_guard<std::recursive_mutex> g(c->mu);
        dev_free(c, sl.ws);
        dev_free(c, sl.chg);
        dev_free(c, sl.pscratch);
        sl.in->busy -= 1;
        if (tk->inline_inst) stage_unload_instance(c, tk->inst);
    }
    // the next request waiting on this instance goes to the head of the queue
    auto it = tk->inline_inst ? parked.end() : parked.find(inst);
    if (it != parked.end()) {
        Ticket *nx = it->second.front();
        it->second.pop_front();
        if (it->second.empty()) parked.erase(it);
        nx->released = true;
        releasing[inst] += 1;
        std::lock_guard<std::mutex> lk(mu);
        pending.push_front(nx);
    }
    complete(tk, status);
}

void Engine::retire_pending()
{
    if (retiring.empty()) return;
    for (Retiring &r : retiring) retire_copy(r);
    const bool copies_ok = cudaStreamSynchronize(c->stream) == cudaSuccess;
    for (Retiring &r : retiring) retire_finish(r, copies_ok);
    retiring.clear();
}

// Host-side phases of the worker loop, reported through stage_kernel_stats
// under engine_* names (calls, milliseconds): where a round's wall time goes.
struct PhaseClock {
    stage_ctx *c;
    const char *name;
    int64_t t0;
    PhaseClock(stage_ctx *c_, const char *n) : c(c_), name(n), t0(now_ns()) {}
    ~PhaseClock()
    {
        const double ms = (now_ns() - t0) / 1e6;
        std::lock_guard<std::recursive_mutex> g(c->mu);
        KernelStat &k = c->stats[name];
        k.launches += 1;
        k.ms += ms;
    }
};

void Engine::run()
{
    cudaSetDevice(c->device);
    for (;;) {
        PhaseClock round_clock(c, "engine_round");
        std::vector<Ticket *> take;
        int64_t idle_ns = 0;   // added after the engine lock is released (lock order: context, then engine)
        {
            std::unique_lock<std::mutex> lk(mu);
            if (!(stop || !pending.empty() || !active.empty())) {
                const int64_t t0 = now_ns();
                cv_work.wait(lk, [&] { return stop || !pending.empty() || !active.empty(); });
                idle_ns = now_ns() - t0;
            }
            if (stop) break;
            const size_t room = (size_t)c->max_slots > active.size() ? c->max_slots - active.size() : 0;
            while (!pending.empty() && take.size() < room) {
                take.push_back(pending.front());
                pending.pop_front();
            }
        }
        if (idle_ns) {
            std::lock_guard<std::recursive_mutex> g(c->mu);
            KernelStat &k = c->stats["engine_idle"];
            k.launches += 1;
            k.ms += idle_ns / 1e6;
        }
        // 1. advance the current slots (asynchronous)
        cudaError_t e = cudaSuccess;
        const int n = (int)active.size();
        if (n > 0) {
            if (dirty) {
                PhaseClock pc(c, "engine_rebuild");
                if (rebuild() != STAGE_OK) e = cudaErrorUnknown;
            }
            if (e == cudaSuccess) {
                {
                    std::lock_guard<std::recursive_mutex> g(c->mu);
                    for (const char *nm : {"group_swap", "group_select", "group_refresh"})
                        c->stats[nm].launches += kStepsPerGraph;
                    int n_delta = 0;
                    for (int l = 0; l < kLanes; l++) n_delta += lane[l].n_delta;
                    if (n_delta > 0) c->stats["group_delta"].launches += kStepsPerGraph;
                    c->stats["group_steps"].launches += kStepsPerGraph;
                }
                if (!ev_round[0]) {
                    cudaEventCreate(&ev_round[0]);
                    cudaEventCreate(&ev_round[1]);
                }
                cudaEventRecord(ev_round[0], stream);
                e = launch_steps(kStepsPerGraph);
                if (e == cudaSuccess && p_n > 0) {
                    // the persistent slots: kPersistRoundSteps iterations each, in one launch
                    if (!ev_p[0]) {
                        cudaEventCreate(&ev_p[0]);
                        cudaEventCreate(&ev_p[1]);
                    }
                    e = launch_batch_prep(p_args, p_n, stream);
                    if (e == cudaSuccess) e = cudaEventRecord(ev_p[0], stream);
                    if (e == cudaSuccess)
                        e = launch_tabu_batch(p_args, p_sched, p_off, p_grid, p_smem, stream, kPersistRoundSteps);
                    if (e == cudaSuccess) e = cudaEventRecord(ev_p[1], stream);
                }
                if (e == cudaSuccess)
                    e = launch_gather_states(static_cast<const GroupSlot *>(d_slots.p), n,
                                             static_cast<TabuDevState *>(d_states.p), stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(h_states, d_states.p, sizeof(TabuDevState) * n, cudaMemcpyDeviceToHost,
                                        stream);
                cudaEventRecord(ev_round[1], stream);
            }
        }
        // 2. meanwhile release the slots that finished in the previous round
        //    and admit waiting requests (their set-up runs on the context's stream)
        if (!retiring.empty()) {
            PhaseClock pc(c, "engine_retire");
            retire_pending();
        }
        const size_t before = active.size();
        std::vector<Ticket *> retry;
        std::unordered_set<stage_inst> held;   // instances with a request sent back to the queue
        for (Ticket *tk : take) {
            if (tk->inst && held.count(tk->inst)) {
                retry.push_back(tk);   // keeps requests on one instance in submission order
                continue;
            }
            PhaseClock pc(c, "engine_admit");
            bool transient = false;
            stage_inst busy_on = 0;
            const bool was_released = tk->released;
            const stage_inst h0 = tk->inst;
            if (admit(tk, transient, busy_on)) {
                if (was_released) unrelease(h0);
                continue;
            }
            if (busy_on) {
                if (was_released) {   // back to the head of its instance's queue
                    unrelease(h0);
                    tk->released = false;
                    parked[busy_on].push_front(tk);
                } else {
                    parked[busy_on].push_back(tk);
                }
            } else if (transient) {
                retry.push_back(tk);   // a released request stays released (and counted)
                if (tk->inst && !tk->inline_inst) held.insert(tk->inst);
            } else if (was_released) {
                unrelease(h0);         // failed for good
            }
        }
        if (!retry.empty()) {
            std::lock_guard<std::mutex> lk(mu);
            for (auto it = retry.rbegin(); it != retry.rend(); ++it) pending.push_front(*it);
        }
        // 3. finish the step and retire finished slots (only the first n slots took part)
        if (n > 0) {
            if (e == cudaSuccess) {
                PhaseClock pc(c, "engine_wait");
                e = cudaStreamSynchronize(stream);
            }
            float gpu_ms = 0.f;
            if (e == cudaSuccess && cudaEventElapsedTime(&gpu_ms, ev_round[0], ev_round[1]) == cudaSuccess) {
                std::lock_guard<std::recursive_mutex> g(c->mu);
                KernelStat &k = c->stats["engine_gpu_round"];   // device time of the round's launches
                k.launches += 1;
                k.ms += gpu_ms;
                float pms = 0.f;
                if (p_n > 0 && cudaEventElapsedTime(&pms, ev_p[0], ev_p[1]) == cudaSuccess) {
                    KernelStat &kp = c->stats["engine_persist"];   // the persistent launch's device time
                    kp.launches += 1;
                    kp.ms += pms;
                }
            }
            int erased = 0;
            for (size_t k = n; k-- > 0;) {   // descending: erasing keeps the lower indices
                TabuDevState z{};
                const TabuDevState &s = e == cudaSuccess ? h_states[k] : z;
                const bool fin = e != cudaSuccess || s.done || s.t >= s.t_end || s.err;
                if (!fin) continue;
                retiring.push_back(Retiring{active[k], s, e != cudaSuccess ? STAGE_ERR_CUDA : STAGE_OK, {}, {}});
                active.erase(active.begin() + k);
                erased += 1;
                dirty = true;
            }
            // incremental slots that took part ran their first full pass: the
            // next map leaves out their swap blocks (the round's remaining
            // slots are the first n - erased; slots admitted meanwhile follow)
            for (int k = 0; k < n - erased; k++)
                if (active[k].tb.chg && !active[k].first_done) {
                    active[k].first_done = true;
                    dirty = true;
                }
            // nothing left to run: release now rather than after a next round
            if (active.empty() && !retiring.empty()) {
                PhaseClock pc(c, "engine_retire");
                retire_pending();
            }
        }
        if (active.size() != before) dirty = true;
        if (!dirty) stable += 1;
        if (active.empty() && !retry.empty()) std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    // stopping: release what is still held; unfinished tickets report a timeout
    retire_pending();
    for (size_t k = active.size(); k-- > 0;) {
        Retiring r{active[k], TabuDevState{}, STAGE_ERR_TIMEOUT, {}, {}};
        r.fin.assign(r.sl.tb.K, 0);
        r.best.assign(r.sl.tb.K, 0);
        retire_finish(r, true);
    }
    active.clear();
    {
        // requests still waiting on an instance go back to the queue, which is
        // answered with a timeout when the engine is destroyed
        std::lock_guard<std::mutex> lk(mu);
        for (auto &kv : parked)
            for (Ticket *tk : kv.second) pending.push_back(tk);
        parked.clear();
    }
}

void engine_destroy(stage_ctx *c)
{
    Engine *E = c->engine.load();
    if (!E) return;
    {
        std::lock_guard<std::mutex> lk(E->mu);
        E->stop = true;
    }
    E->cv_work.notify_all();
    if (E->th.joinable()) E->th.join();
    {
        std::lock_guard<std::mutex> lk(E->mu);
        for (Ticket *tk : E->pending) {
            tk->res.status = STAGE_ERR_TIMEOUT;
            tk->state = 2;
        }
        E->pending.clear();
    }
    if (E->graph) cudaGraphExecDestroy(E->graph);
    for (cudaEvent_t ev : E->ev_round)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : E->ev_p)
        if (ev) cudaEventDestroy(ev);
    dev_free(c, E->d_pbuf);
    dev_free(c, E->d_slots);
    dev_free(c, E->d_map);
    dev_free(c, E->d_states);
    if (E->h_states) cudaFreeHost(E->h_states);
    E->release_streams();
    delete E;
    c->engine.store(nullptr);
}

}  // namespace stg_rt

using namespace stg_rt;

extern "C" {

stage_status stage_batch_submit(stage_ctx *c, const stage_request *reqs, int32_t n, uint64_t *tickets)
{
    if (!c) return STAGE_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!reqs || !tickets))) return set_err(c, STAGE_ERR_INVALID_ARG, "bad request array");
    Engine *E = c->engine.load();
    if (!E) {
        std::lock_guard<std::recursive_mutex> g(c->mu);
        if (!c->engine.load()) {
            cudaSetDevice(c->device);
            E = new Engine();
            E->c = c;
            int least = 0, greatest = 0;
            cudaDeviceGetStreamPriorityRange(&least, &greatest);
            bool ok = cudaEventCreateWithFlags(&E->ev_fork, cudaEventDisableTiming) == cudaSuccess;
            for (int l = 0; ok && l < kLanes; l++)
                ok = cudaStreamCreateWithPriority(&E->lane_stream[l], cudaStreamNonBlocking, least) == cudaSuccess &&
                     cudaEventCreateWithFlags(&E->ev_join[l], cudaEventDisableTiming) == cudaSuccess;
            E->stream = E->lane_stream[0];
            if (!ok) {
                E->release_streams();
                delete E;
                return set_err(c, STAGE_ERR_CUDA, "engine stream creation failed");
            }
            c->engine.store(E);
            E->th = std::thread([E] { E->run(); });
        }
        E = c->engine.load();
    }
    std::vector<std::unique_ptr<Ticket>> made;
    for (int32_t k = 0; k < n; k++) {
        const stage_request &r = reqs[k];
        auto tk = std::make_unique<Ticket>();
        tk->req = r;
        tk->inst = r.inst;
        if (r.params.start_open && r.params.K > 0) tk->start.assign(r.params.start_open, r.params.start_open + r.params.K);
        tk->req.params.start_open = nullptr;
        if (!r.inst) {
            const stage_instance_desc *d = r.desc;
            if (!d || !d->base_xy || !d->pick_xy || !d->drop_xy || d->B < 1 || d->M < 1 ||
                (d->flags & STAGE_DESC_DEVICE))
                return set_err(c, STAGE_ERR_INVALID_ARG, "request %d: needs an instance handle or a host descriptor", k);
            tk->inline_inst = true;
            tk->d_base.assign(d->base_xy, d->base_xy + 2 * (size_t)d->B);
            tk->d_pick.assign(d->pick_xy, d->pick_xy + 2 * (size_t)d->M);
            tk->d_drop.assign(d->drop_xy, d->drop_xy + 2 * (size_t)d->M);
            if (d->base_available) tk->d_avail.assign(d->base_available, d->base_available + d->B);
            tk->d_flags = d->flags & STAGE_DESC_HAVERSINE;
        }
        if (copy_update(tk.get(), r.update) != STAGE_OK)
            return set_err(c, STAGE_ERR_INVALID_ARG, "request %d: malformed update", k);
        made.push_back(std::move(tk));
    }
    {
        std::lock_guard<std::mutex> lk(E->mu);
        const int64_t t = now_ns();
        for (int32_t k = 0; k < n; k++) {
            Ticket *tk = made[k].get();
            tk->id = E->next_ticket++;
            tk->res.t_submit_ns = t;
            tickets[k] = tk->id;
            E->pending.push_back(tk);
            E->tickets[tk->id] = std::move(made[k]);
        }
    }
    E->cv_work.notify_all();
    return STAGE_OK;
}

stage_status stage_poll(stage_ctx *c, uint64_t ticket, stage_result *out, int32_t timeout_us)
{
    if (!c || !out) return STAGE_ERR_INVALID_ARG;
    Engine *E = c->engine.load();
    if (!E) return STAGE_ERR_NOT_FOUND;
    std::unique_lock<std::mutex> lk(E->mu);
    auto it = E->tickets.find(ticket);
    if (it == E->tickets.end()) return STAGE_ERR_NOT_FOUND;
    Ticket *tk = it->second.get();
    if (tk->state != 2 && timeout_us != 0) {
        auto pred = [&] { return tk->state == 2; };
        if (timeout_us < 0) E->cv_done.wait(lk, pred);
        else E->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred);
    }
    if (tk->state != 2) return STAGE_PENDING;
    *out = tk->res;
    const stage_status st = tk->res.status;
    E->tickets.erase(it);
    return st;
}

}  // extern "C"
