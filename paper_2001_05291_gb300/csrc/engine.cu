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
// Every slot runs exactly the search stage_tabu_run would run alone, so each
// result is independent of what else is in the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>

#include "runtime_internal.h"

using namespace stg;

namespace stg_rt {

namespace {

constexpr int kStepsPerGraph = 8;

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
    stage_inst inst = 0;
    stage_result res{};
    int state = 0;                         // 0 pending, 1 running, 2 done
};

struct Slot {
    Ticket *tk = nullptr;
    Instance *in = nullptr;
    DevBuf ws;
    TabuBuffers tb{};
    int nC = 0;
};

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
    bool dirty = true;        // slot set changed: device arrays must be rebuilt
    int stable = 0;           // rounds since the last change (the graph is captured once stable)
    int n_swap_blocks = 0, n_sel_blocks = 0, n_ref_blocks = 0, maxK = 1;
    size_t swap_smem = 0;

    void run();
    cudaError_t launch_steps(int steps);
    bool admit(Ticket *tk, bool &transient);
    void complete(Ticket *tk, stage_status st);
    void retire(size_t k, const TabuDevState &s, stage_status status);
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

// Admit one request into a new slot.  On a transient shortage (memory, or its
// instance busy in another slot) returns false with transient = true.
bool Engine::admit(Ticket *tk, bool &transient)
{
    transient = false;
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
            stage_inst h = 0;
            s = stage_load_instance(c, &d, &h);
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
    if (in->busy) {
        transient = true;   // one request per instance at a time: updates and searches stay ordered
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
    if (!tk->start.empty()) {
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
    std::vector<uint8_t> is_open(in->B, 0);
    for (int k = 0; k < K; k++) is_open[start[k]] = 1;
    std::vector<int32_t> cand;
    for (int b = 0; b < in->B; b++)
        if (in->h_avail[b] && !is_open[b]) cand.push_back(b);
    sl.nC = (int)cand.size();
    TabuDevState st{};
    st.tenure = p.tenure;
    st.accept_worsening = p.accept_worsening ? 1 : 0;
    st.nC = sl.nC;
    st.traj_cap = p.iters;
    st.best_iter = -1;
    st.t_end = p.iters;
    std::vector<int32_t> zeros(in->B, 0);
    // set-up runs on the context's stream: the engine's stream may be busy
    // with the current step, which this slot is not part of
    cudaStream_t stream = c->stream;
    cudaError_t e = cudaMemcpyAsync(tb.open, start.data(), (size_t)K * 4, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && sl.nC)
        e = cudaMemcpyAsync(tb.cand, cand.data(), (size_t)sl.nC * 4, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tb.expiry, zeros.data(), (size_t)in->B * 4, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tb.st, &st, sizeof st, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.v0, 0, 16, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.loss_c, 0, (size_t)K * 8, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.loss_d, 0, (size_t)K * 8, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.gain_c, 0, (size_t)in->B * 4, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.gain_d, 0, (size_t)in->B * 8, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.extra_c, 0, (size_t)K * in->B * 4, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tb.extra_d, 0, (size_t)K * in->B * 8, stream);
    if (e == cudaSuccess) e = timed_on(c, stream, "init", 1, [&] { return launch_init(tb, in->cost, stream); });
    if (e == cudaSuccess) e = timed_on(c, stream, "begin", 1, [&] { return launch_begin(tb, 0, stream); });
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);   // host vectors above go out of scope
    if (e != cudaSuccess) {
        dev_free(c, sl.ws);
        set_err(c, STAGE_ERR_CUDA, "batch slot set-up failed: %s", cudaGetErrorString(e));
        return fail(STAGE_ERR_CUDA);
    }
    sl.tb = tb;
    in->busy += 1;
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
        if (cudaMallocHost(&h_states, sizeof(TabuDevState) * (size_t)cap) != cudaSuccess) return STAGE_ERR_CUDA;
    }
    std::vector<GroupSlot> gs(n);
    std::vector<int> mp(n), nc(n);
    for (int k = 0; k < n; k++) {
        mp[k] = active[k].tb.M_pad;
        nc[k] = active[k].nC;
    }
    const int common = group_common_segment(mp.data(), nc.data(), n);
    maxK = 1;
    swap_smem = 0;
    std::vector<int2> map;   // swap blocks, then select blocks, then refresh blocks
    for (int k = 0; k < n; k++) {
        const Slot &sl = active[k];
        gs[k].w = sl.tb;
        gs[k].cost = sl.in->cost;
        gs[k].swap_blocks =
            group_swap_blocks(sl.tb.M_pad, sl.nC, sl.tb.K, common, &gs[k].swap_bx, &gs[k].swap_seg);
        swap_smem = std::max(swap_smem, swap_direct_smem(sl.tb.K));
        gs[k].sel_blocks = select_blocks(sl.tb.K, sl.nC);
        gs[k].ref_blocks = group_ref_blocks(sl.tb.M_pad);
        for (int b = 0; b < gs[k].swap_blocks; b++) map.push_back(make_int2(k, b));
        maxK = std::max(maxK, sl.tb.K);
    }
    n_swap_blocks = (int)map.size();
    for (int k = 0; k < n; k++)
        for (int b = 0; b < gs[k].sel_blocks; b++) map.push_back(make_int2(k, b));
    n_sel_blocks = (int)map.size() - n_swap_blocks;
    for (int k = 0; k < n; k++)
        for (int b = 0; b < gs[k].ref_blocks; b++) map.push_back(make_int2(k, b));
    n_ref_blocks = (int)map.size() - n_swap_blocks - n_sel_blocks;
    if (map.size() > map_cap) {
        std::lock_guard<std::recursive_mutex> g(c->mu);
        dev_free(c, d_map);
        map_cap = std::max(map.size(), 2 * map_cap);
        if (dev_alloc(c, sizeof(int2) * map_cap, d_map) != STAGE_OK) {
            map_cap = 0;
            return STAGE_ERR_NO_MEMORY;
        }
    }
    cudaError_t e = cudaMemcpyAsync(d_slots.p, gs.data(), sizeof(GroupSlot) * n, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_map.p, map.data(), sizeof(int2) * map.size(), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return STAGE_ERR_CUDA;
    dirty = false;
    stable = 0;
    return STAGE_OK;
}

// kStepsPerGraph grouped steps: launched directly while the slot set keeps
// changing, replayed from a captured CUDA graph once it has been stable.
cudaError_t Engine::launch_steps(int steps)
{
    const GroupSlot *ds = static_cast<const GroupSlot *>(d_slots.p);
    const int2 *map_swap = static_cast<const int2 *>(d_map.p);
    const int2 *map_sel = map_swap + n_swap_blocks;
    const int2 *map_ref = map_sel + n_sel_blocks;
    auto enqueue = [&]() {
        cudaError_t e = cudaSuccess;
        for (int k = 0; e == cudaSuccess && k < steps; k++) {
            e = launch_group_swap(ds, map_swap, n_swap_blocks, swap_smem, stream);
            if (e == cudaSuccess) e = launch_group_select(ds, map_sel, n_sel_blocks, stream);
            if (e == cudaSuccess) e = launch_group_refresh(ds, map_ref, n_ref_blocks, maxK, stream);
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

void Engine::retire(size_t k, const TabuDevState &s, stage_status status)
{
    Slot &sl = active[k];
    Ticket *tk = sl.tk;
    const int K = sl.tb.K;
    std::vector<int32_t> fin(K), best(K);
    cudaError_t e = cudaMemcpyAsync(fin.data(), sl.tb.open, (size_t)K * 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(best.data(), sl.tb.best_open, (size_t)K * 4, cudaMemcpyDeviceToHost, stream);
    const int n = std::min(s.n_moves, tk->req.params.iters);
    if (e == cudaSuccess && tk->req.traj && n > 0)
        e = cudaMemcpyAsync(tk->req.traj, sl.tb.traj, (size_t)n * sizeof(stage_move), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess && status == STAGE_OK) status = STAGE_ERR_CUDA;
    if (s.err && status == STAGE_OK) status = STAGE_ERR_INTERNAL;
    std::sort(fin.begin(), fin.end());
    std::sort(best.begin(), best.end());
    if (tk->req.best_open) std::copy(best.begin(), best.end(), tk->req.best_open);
    if (tk->req.final_open) std::copy(fin.begin(), fin.end(), tk->req.final_open);
    tk->res.n_moves = s.n_moves;
    tk->res.best_iter = s.best_iter;
    tk->res.best_cov = s.best_cov;
    tk->res.best_dist = s.best_dist;
    tk->res.final_cov = s.cur_cov;
    tk->res.final_dist = s.cur_dist;
    {
        std::lock_guard<std::recursive_mutex> g(c->mu);
        dev_free(c, sl.ws);
        sl.in->busy -= 1;
        if (tk->inline_inst) stage_unload_instance(c, tk->inst);
    }
    complete(tk, status);
}

void Engine::run()
{
    cudaSetDevice(c->device);
    for (;;) {
        std::vector<Ticket *> take;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_work.wait(lk, [&] { return stop || !pending.empty() || !active.empty(); });
            if (stop) break;
            const size_t room = (size_t)c->max_slots > active.size() ? c->max_slots - active.size() : 0;
            while (!pending.empty() && take.size() < room) {
                take.push_back(pending.front());
                pending.pop_front();
            }
        }
        // 1. advance the current slots (asynchronous)
        cudaError_t e = cudaSuccess;
        const int n = (int)active.size();
        if (n > 0) {
            if (dirty && rebuild() != STAGE_OK) e = cudaErrorUnknown;
            if (e == cudaSuccess) {
                {
                    std::lock_guard<std::recursive_mutex> g(c->mu);
                    for (const char *nm : {"group_swap", "group_select", "group_refresh"})
                        c->stats[nm].launches += kStepsPerGraph;
                    c->stats["group_steps"].launches += kStepsPerGraph;
                }
                e = launch_steps(kStepsPerGraph);
                if (e == cudaSuccess)
                    e = launch_gather_states(static_cast<const GroupSlot *>(d_slots.p), n,
                                             static_cast<TabuDevState *>(d_states.p), stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(h_states, d_states.p, sizeof(TabuDevState) * n, cudaMemcpyDeviceToHost,
                                        stream);
            }
        }
        // 2. meanwhile admit waiting requests (their set-up runs on the context's stream)
        const size_t before = active.size();
        std::vector<Ticket *> retry;
        for (Ticket *tk : take) {
            bool transient = false;
            if (!admit(tk, transient) && transient) retry.push_back(tk);
        }
        if (!retry.empty()) {
            std::lock_guard<std::mutex> lk(mu);
            for (auto it = retry.rbegin(); it != retry.rend(); ++it) pending.push_front(*it);
        }
        // 3. finish the step and retire finished slots (only the first n slots took part)
        if (n > 0) {
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
            for (size_t k = n; k-- > 0;) {
                TabuDevState z{};
                const TabuDevState &s = e == cudaSuccess ? h_states[k] : z;
                const bool fin = e != cudaSuccess || s.done || s.t >= s.t_end || s.err;
                if (!fin) continue;
                retire(k, s, e != cudaSuccess ? STAGE_ERR_CUDA : STAGE_OK);
                active.erase(active.begin() + k);
                dirty = true;
            }
        }
        if (active.size() != before) dirty = true;
        if (!dirty) stable += 1;
        if (active.empty() && !retry.empty()) std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    // stopping: release what is still held; unfinished tickets report a timeout
    for (size_t k = active.size(); k-- > 0;) {
        TabuDevState z{};
        retire(k, z, STAGE_ERR_TIMEOUT);
    }
    active.clear();
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
    dev_free(c, E->d_slots);
    dev_free(c, E->d_map);
    dev_free(c, E->d_states);
    if (E->h_states) cudaFreeHost(E->h_states);
    if (E->stream) cudaStreamDestroy(E->stream);
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
            if (cudaStreamCreateWithFlags(&E->stream, cudaStreamNonBlocking) != cudaSuccess) {
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
