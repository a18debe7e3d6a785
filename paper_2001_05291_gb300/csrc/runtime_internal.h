// Internal declarations of the host runtime shared by runtime.cu (single
// instance calls) and engine.cu (batch engine).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "stage_internal.h"

namespace stg_rt {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct KernelStat {
    int64_t launches = 0;
    double ms = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};

// The end state of the last batch search on a resident instance that asked
// to keep it (stage_request.resume_resident): the next such request resumes
// from it.  `version` is the instance's update count when it was saved.
struct ResidentState {
    bool valid = false;
    int K = 0, t = 0, best_iter = -1;
    int64_t best_cov = 0, best_dist = 0;
    uint64_t version = 0;
    std::vector<int32_t> open, best_open, expiry;
};

struct Instance {
    int B = 0, M = 0, M_pad = 0;   // M: table columns in use (live + removed); M_pad: allocated columns
    int metric = 0;                // 0: Euclidean legs on metres, 1: Haversine legs on microdegrees (Eq. 1)
    int n_avail = 0;
    std::vector<uint8_t> h_avail;
    DevBuf mem_coords;   // base, pick, drop (caller order and column order), pd, perm, inv, avail
    DevBuf mem_table;    // B x M_pad int32, columns in mission order `perm`
    int2 *base = nullptr, *pick = nullptr, *drop = nullptr;   // column order
    int2 *pick_in = nullptr, *drop_in = nullptr;              // caller order
    int32_t *pd = nullptr;
    int32_t *perm = nullptr;   // column -> caller's mission index
    int32_t *inv = nullptr;    // caller's mission index -> column
    uint8_t *avail = nullptr;
    int32_t *cost = nullptr;
    // Tabu workspace, sized for ws_K / ws_traj
    DevBuf mem_ws;
    int ws_K = 0, ws_traj = -1, ws_M_pad = 0;
    stg::TabuBuffers tb{};
    DevBuf mem_scratch;  // rank sums, evaluation outputs, exports
    DevBuf mem_chg;      // change records of the incremental neighbourhood ([2 * M_pad] int4)
    DevBuf mem_costT;    // the table mission-major for the incremental neighbourhood (M_pad x ldT)
    DevBuf mem_persist;  // accumulators, counters and barrier of the persistent search
    DevBuf mem_rowsum;   // [B] uint64 row sums of the table, built with it (the ranking's key)
    int ldT = 0;
    bool costT_ok = false;   // mem_costT holds the current table
    bool rowsum_ok = false;  // mem_rowsum holds the current table's row sums
    size_t scratch_bytes = 0;
    int busy = 0;        // batch requests referring to this instance
    uint64_t version = 0;      // stage_update_instance calls so far
    ResidentState resident;    // kept between batch requests (resume_resident)
    // the measured device work of this instance's last search in a batch
    // launch (CTA time per iteration outside the waits, us), for that K, R and
    // version: the next batch sizes its gang from it
    double batch_work_us = 0.0;
    int batch_K = 0, batch_R = -1;
    uint64_t batch_version = 0;
};

struct Engine;   // batch engine (engine.cu)

}  // namespace stg_rt

struct stage_ctx {
    int device = 0;
    uint32_t flags = 0;
    uint64_t budget = 0;
    int max_slots = 8;
    int64_t spin_limit = 1ll << 26;
    // set by the batch engine around its loads of instances given by value:
    // its grouped searches never read a mission-major copy, so none is built
    bool load_without_copy = false;
    stage_alloc_fn alloc = nullptr;
    stage_free_fn free = nullptr;
    void *alloc_user = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaMemPool_t pool = nullptr;   // stream-ordered pool behind dev_alloc when no allocator hook is given
    uint64_t used = 0;
    std::unordered_map<uint64_t, stg_rt::Instance *> insts;
    uint64_t next_id = 1;
    std::string err;
    std::recursive_mutex mu;
    std::unordered_map<std::string, stg_rt::KernelStat> stats;
    std::vector<cudaEvent_t> event_pool;
    void *pinned = nullptr;       // small pinned host buffer for early-stop polls
    void *batch_pinned = nullptr; // pinned staging of stage_tabu_batch's copies, grown as needed
    size_t batch_pinned_bytes = 0;
    std::atomic<stg_rt::Engine *> engine{nullptr};
};

namespace stg_rt {

stage_status set_err(stage_ctx *c, stage_status code, const char *fmt, ...);
size_t round_up(size_t x, size_t a);
stage_status dev_alloc(stage_ctx *c, size_t bytes, DevBuf &out);
void dev_free(stage_ctx *c, DevBuf &b);
Instance *find_inst(stage_ctx *c, stage_inst h);
void free_instance(stage_ctx *c, Instance *in);
stage_status ensure_ws(stage_ctx *c, Instance *in, int K, int traj);
size_t carve_ws(char *base, int K, int B, int M_pad, int traj, stg::TabuBuffers &tb);
stage_status check_placement(stage_ctx *c, Instance *in, const int32_t *open, int K);
stage_status do_rank(stage_ctx *c, Instance *in, int K, int32_t *out_open, int64_t *out_rowsum);
void engine_destroy(stage_ctx *c);
stage_status autotune_shape(stage_ctx *c, Instance *in, const int32_t *open, int K, int R, int *out_seg);
stage_status setup_search(stage_ctx *c, Instance *in, const int32_t *open, int K, int R, int traj_cap, int tenure,
                          int accept_worsening, int t0, const int32_t *expiry_in, int *out_nC, bool sync = true);
stage_status rank_queue(stage_ctx *c, Instance *in, int K, int32_t *out_open, int64_t *out_rowsum);
stage_status rank_sums(stage_ctx *c, Instance *in, int K);   // its checks and row sums only
// The persistent batch launch's host logic (runtime.cu): the estimated work of
// one iteration of a search on one CTA (us; cov = covered fraction), and the
// placement of n searches (work[k] on gang[k] CTAs) on P CTAs -- lists[q] =
// CTA q's (placement position, rank) entries, order[pos] = the search placed
// at pos; returns the latest estimated finish.
double persist_iter_us_estimate(const Instance *in, int K, int nC, double cov);
double batch_place(int n, const double *work, const int *gang, int P, std::vector<std::vector<int2>> &lists,
                   std::vector<int> &order);
stage_status ensure_costT(stage_ctx *c, Instance *in);
stage_status forced_moves(stage_ctx *c, Instance *in, int32_t *open, int K, int R, int t, int tenure,
                          int32_t *expiry, int *n_forced);

// Launch through `f`, counting launches and (with STAGE_PROFILE) timing them
// on `stream`.
cudaEvent_t get_event(stage_ctx *c);
template <class F>
cudaError_t timed_on(stage_ctx *c, cudaStream_t stream, const char *name, int n_kernels, F &&f)
{
    KernelStat &ks = c->stats[name];
    ks.launches += n_kernels;
    if (!(c->flags & STAGE_PROFILE)) return f();
    cudaEvent_t e0 = get_event(c), e1 = get_event(c);
    cudaEventRecord(e0, stream);
    cudaError_t r = f();
    cudaEventRecord(e1, stream);
    ks.pending.emplace_back(e0, e1);
    return r;
}

}  // namespace stg_rt
