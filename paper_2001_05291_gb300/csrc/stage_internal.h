// Internal declarations shared by the kernels and the host runtime of the
// staging engine.  Nothing here is part of the C ABI (include/stage.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "stage.h"

namespace stg {

constexpr int32_t kInf = INT32_MAX;
constexpr int kPadMissions = 64;     // table rows are padded to a multiple of 64 missions

// Candidate-move key of the Tabu selection: more covered first, then less
// distance, then lower closed base i, then lower opened base j.
struct MoveKey {
    long long cov;
    long long dist;
    int i, j;       // global base ids
    int s, c;       // slot of i in the placement, position of j in the candidate list
    int valid;      // 0 = no candidate
    int tabu;       // the move is tabu (admitted by aspiration when chosen)
};

// Device-resident state of one Tabu run.  Written by the select kernel,
// read by the evaluation and refresh kernels; the host reads it at the end.
struct TabuDevState {
    int t;                // iteration number of the next step
    int n_moves;          // moves applied (trajectory length)
    int done;             // 1 once the search has stopped
    int err;              // nonzero: a self-check failed (see kErr*)
    int tenure;
    int accept_worsening;
    int nC;               // closed available bases (candidate rows)
    int traj_cap;         // trajectory capacity (entries)
    long long cur_cov, cur_dist;     // F of the current placement
    long long best_cov, best_dist;   // best so far
    int best_iter;
    int mv_s, mv_i, mv_j; // last applied move: slot, closed base, opened base
    unsigned int ticket;  // last-block counter of the select kernel
    unsigned int work;    // work-unit counter of the streaming swap pass
    int t_end;            // iteration budget: no step at t >= t_end
    // local search (Alg. 2): scan position in the current pass, pass index,
    // whether the pass applied a move, passes supplied, "accumulators still
    // valid, skip evaluation and refresh" (after a pass change), local optimum
    int ls_pos, ls_pass, ls_moved, ls_passes, ls_hold, ls_optimum;
    // incremental neighbourhood: missions the last refresh recorded, and the
    // running total over the search (for the traffic accounting)
    int chg_n;
    long long chg_total;
};

enum : int { kErrObjectiveMismatch = 1, kErrBadSlot = 2, kErrPipelineTimeout = 4 };

// Device buffers of one Tabu run (or one neighbourhood evaluation).
struct TabuBuffers {
    int K, B, M, M_pad, R;
    // per mission (M_pad): best / second-best cost and their slots
    int32_t *a, *b;
    int16_t *s1, *s2;
    // objective decomposition F(i, j) = V0 + gain[j] + loss[i] + extra[i][j]
    unsigned long long *v0;      // [2]: covered, distance (two's complement)
    unsigned long long *loss_c;  // [K]
    unsigned long long *loss_d;  // [K]
    int *gain_c;                 // [B]
    unsigned long long *gain_d;  // [B]
    int *extra_c;                // [K * B]
    unsigned long long *extra_d; // [K * B]
    // placement
    int32_t *open;               // [K] slot -> base
    int32_t *best_open;          // [K]
    int32_t *cand;               // [B] closed available bases (first nC entries)
    int32_t *expiry;             // [B]
    TabuDevState *st;
    MoveKey *partials;           // [2 * kSelectBlocks]
    stage_move *traj;            // [traj_cap]
    // missions of this search, per column (the heterogeneous fleet splits the
    // missions into two searches); NULL = every mission.  A mission outside
    // has thresholds INT_MIN: no hit, no term, untouched by the refresh.
    const uint8_t *mask;
    // incremental neighbourhood: [2 * M_pad] records, two int4 per mission
    // whose terms the last refresh changed: (column, old a, old b, old best
    // slot), (new a, new b, new best slot, 0); the gain / extra terms are then
    // kept across iterations and updated from these records.  NULL = the
    // refresh clears the terms and a full pass rebuilds them every iteration.
    int4 *chg;
    // incremental neighbourhood: the cost table mission-major with the bases
    // in a spatial order, costT[m * ldT + p] = cost of base border[p] for m
    const int32_t *costT;
    const int32_t *border;   // [ldT] position -> base id (-1 past B)
    // [M_pad][cell_ld(ldT)]: each mission's least cost over each 32
    // consecutive positions of its costT row
    const int32_t *cellmin;
    int ldT;
};

constexpr int kPipeMaxK = 256;   // most slots of the direct swap pass and of the incremental form
constexpr int kSelectBlocks = 148;
constexpr int kSelectThreads = 256;

// ----------------------------------------------------------------- launchers
// Every launcher enqueues on `stream` and returns the launch error.
cudaError_t launch_fill_i32(int32_t *p, size_t n, int32_t v, cudaStream_t s);
cudaError_t launch_table_columns(int B, int col0, int n, int M_pad, const int2 *base, const int2 *pick,
                                 const int2 *drop, int32_t *pd, int32_t *cost, int metric, cudaStream_t s);
cudaError_t launch_tombstone(const int32_t *ids, int n, int32_t *inv, int32_t *perm, int32_t *cost, int B,
                             int M_pad, cudaStream_t s);
cudaError_t launch_check_coords(const int32_t *v, size_t n, int lim_x, int lim_y, int *bad, cudaStream_t s);
cudaError_t launch_table(int B, int M, int M_pad, const int2 *base, const int2 *pick,
                         const int2 *drop, int32_t *pd_scratch, int32_t *cost, int metric, cudaStream_t s);
cudaError_t launch_rowsum(const int32_t *cost, int B, int M, int M_pad, unsigned long long *S,
                          cudaStream_t s);
cudaError_t launch_topk(const unsigned long long *S, const uint8_t *avail, int B, int K,
                        int32_t *open, cudaStream_t s);
// many rankings in one launch (one descriptor each; map[b] = (ranking, block))
struct TopkSlot {
    const unsigned long long *S;   // row sums [B]
    const uint8_t *avail;          // [B]
    int32_t *open;                 // out: [K] base ids in rank order
    int B, K;
};
int topk_blocks(int B);
cudaError_t launch_topk_group(const TopkSlot *slots, const int2 *map, int total_blocks, cudaStream_t s);
cudaError_t launch_evaluate(const int32_t *cost, int M, int M_pad, const int32_t *open, int K,
                            int R, unsigned long long *out2, cudaStream_t s);
cudaError_t launch_init(const TabuBuffers &w, const int32_t *cost, cudaStream_t s);
cudaError_t launch_begin(const TabuBuffers &w, int resumed, cudaStream_t s);
cudaError_t launch_swap_eval(const TabuBuffers &w, const int32_t *cost, int nC, int ignore_done,
                             cudaStream_t s);
cudaError_t launch_select(const TabuBuffers &w, int nC, cudaStream_t s);
cudaError_t launch_refresh(const TabuBuffers &w, const int32_t *cost, cudaStream_t s);
// Incremental neighbourhood (w.chg set): every base's column over the
// missions the refresh recorded (the refresh itself rebuilds the column of
// the base the move closed).
bool swap_delta_fits(int K);
constexpr size_t kIncrementalMinTableBytes = 256ull << 20;   // candidate rows x missions, int32
cudaError_t launch_swap_delta(const TabuBuffers &w, cudaStream_t s);
// The B x M_pad table copied mission-major (M_pad x ldT, ldT = B rounded up to
// 32), the bases in the order border (position -> base id, -1 past B).
int table_ldT(int B);
// row stride of the cell minima (cells of 32 positions of a mission-major row),
// a multiple of 8 cells (32 bytes)
__host__ __device__ inline int cell_ld(int ldT) { return ((ldT >> 5) + 7) & ~7; }
// bytes of the mission-major copy with its position order and cell minima:
// [M_pad][ldT] costs, [ldT] positions, [M_pad][cell_ld(ldT)] minima
inline size_t costT_bytes(int M_pad, int ldT)
{
    return ((size_t)M_pad * ldT + (size_t)ldT + (size_t)M_pad * cell_ld(ldT)) * sizeof(int32_t);
}
// the table, its row sums (added to S, zeroed by the caller), the mission-major
// copy (bases in the order border, row length ldT) and its cell minima, in one
// pass; pd receives the pickup-to-drop-off legs
cudaError_t launch_table_fused(int B, int M, int M_pad, int ldT, const int2 *base, const int2 *pick,
                               const int2 *drop, int32_t *pd, const int32_t *border, int32_t *cost, int32_t *costT,
                               int32_t *cellmin, unsigned long long *S, int metric, cudaStream_t s);
cudaError_t launch_transpose_table(const int32_t *cost, int B, int M_pad, const int32_t *border, int32_t *costT,
                                   int32_t *cellmin,
                                   cudaStream_t s);
cudaError_t launch_export_best_two(const TabuBuffers &w, const int *perm, int32_t *a, int32_t *b,
                                   int32_t *b1, int32_t *b2, cudaStream_t s);
// mission order (Morton order of pickup/drop-off midpoints) and readback in caller order
size_t order_scratch_bytes(int M);
cudaError_t launch_order(int M, const int2 *pick, const int2 *drop, void *scratch, int *perm, int *inv,
                         int2 *pick_s, int2 *drop_s, cudaStream_t s);
cudaError_t launch_gather_window(const int32_t *cost, int M, int M_pad, const int *inv, int b0, int nb,
                                 int m0, int nm, int32_t *out, cudaStream_t s);
cudaError_t launch_swap_table(const TabuBuffers &w, int nC, long long *out_c, long long *out_d,
                              cudaStream_t s);
// Persistent search (persist.cu): the incremental neighbourhood's whole loop
// in one cooperative launch.  persist_grid: the CTAs a search of this shape
// takes on the current device (0 when the shape is not supported: K > 256,
// more than 2048 bases, or the per-CTA arrays do not fit in shared memory).
// The scratch (persist_scratch_bytes) holds the sums, barrier, error word,
// per-CTA keys and record regions; at byte offset persist_info_offset(K) six
// int64 -- the CTAs, the records over the search, the update's (record, base)
// pairs with a term, its (record, cell) passes with a term, the extra-column
// runs it wrote, and the (record, cell) pieces it read -- and at persist_clock_offset(K, grid, M_pad) [grid][kPersistClocks] int64:
// each CTA's time in ns of each step (choose and apply the move, refresh, wait
// at the barrier after it, update the columns, wait at the barrier after it,
// select, wait at the barrier before the next move; then parts of the refresh
// -- the mission loop, the rescans, the sums -- and of the update -- staging
// the records, waiting for the CTA's slowest warp, warp 0's walk over the
// records), summed over the search.
constexpr int kPersistClocks = 13;
int persist_grid(int K, int B, int ldT, int M_pad);
size_t persist_scratch_bytes(int K, int grid, int M_pad);
size_t persist_info_offset(int K);
size_t persist_clock_offset(int K, int grid, int M_pad);
cudaError_t launch_tabu_persist(const TabuBuffers &w, const int32_t *cost, void *scratch, int grid,
                                long long spin_limit, cudaStream_t s);
// Many searches in one cooperative launch (k_tabu_batch): search k runs on
// `gang` CTAs with the arguments persist_args_host wrote (persist_args_bytes
// each, copied to the device as one array d_args), its scratch laid out for
// that gang; d_sched / d_off give each CTA its (search, rank) entries in one
// global order of the searches.  persist_search_smem: the dynamic shared
// memory a search of this shape needs (the launch takes the largest);
// persist_batch_grid: the CTAs the device holds at once with that much.
size_t persist_args_bytes();
cudaError_t persist_args_host(const TabuBuffers &w, const int32_t *cost, void *scratch, int gang,
                              long long spin_limit, cudaStream_t s, void *out);
// readies every search's scratch of a batch (clears, start V0 and loss):
// one block per search, before the batch launch
cudaError_t launch_batch_prep(const void *d_args, int n, cudaStream_t s);
size_t persist_search_smem(int K, int B, int ldT);
int persist_batch_grid(size_t smem);
bool persist_shape_ok(int K, int B, int ldT);
int persist_max_gang();
// max_steps > 0: each search makes at most that many iterations in this launch
// and goes on from its handed-back state in a later one (engine rounds).
cudaError_t launch_tabu_batch(const void *d_args, const int2 *d_sched, const int *d_off, int grid, size_t smem,
                              cudaStream_t s, int max_steps = 0);
// Alg. 2's local search with the incremental neighbourhood in one cooperative
// launch (the persistent body with its first-improvement selection): the
// scan orders' ranks rank_slot [passes][K], rank_cand [passes][nC] on the
// device, passes in w.st->ls_passes; grid and scratch as for the Tabu search.
cudaError_t launch_local_persist(const TabuBuffers &w, const int32_t *cost, void *scratch, int grid,
                                 long long spin_limit, const int *rank_slot, const int *rank_cand, cudaStream_t s);
cudaError_t persist_init();
// Test support: a wait on a flag that nothing sets, bounded by `limit` polls;
// it sets kErrPipelineTimeout in *err when it gives up.
cudaError_t launch_wait_unset_flag(unsigned *flag, long long limit, int *err, cudaStream_t s);
cudaError_t kernels_init();   // one-time function attributes (dynamic shared memory)

// ------------------------------------------------------- grouped (batched) launches
// One descriptor per active slot of the batch engine; one launch covers all of
// them.  Each launch gets a block map: (slot, block within the slot) per block.
struct GroupSlot {
    TabuBuffers w;
    const int32_t *cost;
    int swap_bx;      // swap blocks along the missions of this slot
    int swap_blocks;  // swap blocks of this slot (swap_bx x row chunks)
    int ref_blocks;   // refresh blocks of this slot
    int swap_seg;     // missions per swap block
    int sel_blocks;   // select blocks of this slot
    int delta_bx;     // incremental slots (w.chg set): delta blocks along the copy's positions
    int delta_by;     // ... and along the record chunks (0: a full pass every step)
};
constexpr int kGroupMaxK = 256;
int group_swap_blocks(int M_pad, int nC, int K, int seg_override, int *bx, int *seg);
void group_delta_blocks(int ldT, int M, int K, int *bx, int *by);
cudaError_t launch_group_delta(const GroupSlot *slots, const int2 *map, int total_blocks, cudaStream_t s);
int group_common_segment(const int *M_pad, const int *nC, int n);
size_t swap_direct_smem(int K);   // dynamic shared memory of the direct swap pass
bool tabu_small_fits(int nC, int M_pad, int K);
cudaError_t launch_tabu_small(const TabuBuffers &w, const int32_t *cost, int iters, cudaStream_t s);
// small instances, every per-iteration array in shared memory (one block)
bool tabu_resident_fits(int K, int B, int M_pad, int nC);
cudaError_t launch_tabu_resident(const TabuBuffers &w, const int32_t *cost, int nC, int iters, cudaStream_t s);
// heterogeneous fleet: the best move over both searches (A: every vehicle,
// every mission a vehicle of any type may fly; B: the rotary-wing vehicles,
// the rotary-only missions); B's slots are A's first Kr slots
cudaError_t launch_fleet_select(const TabuBuffers &A, const TabuBuffers &B, int Kr, int hasB,
                                const uint8_t *helipad, int *b_pos, cudaStream_t s);
// local search: first improving swap at or after the scan position of the
// current pass (rank_slot / rank_cand: [passes][K] / [passes][nC] positions)
cudaError_t launch_ls_select(const TabuBuffers &w, int nC, const int *rank_slot, const int *rank_cand,
                             cudaStream_t s);
int select_blocks(int K, int nC);
// missions per block of the direct swap pass, per shape (measured choice or heuristic)
int swap_segment_for(int M_pad, int nC, int K);
int swap_segment_heuristic(int M_pad, int nC);
void swap_segment_record(int M_pad, int nC, int K, int seg);
bool swap_segment_known(int M_pad, int nC, int K);
cudaError_t launch_swap_direct_seg(const TabuBuffers &w, const int32_t *cost, int nC, int seg, cudaStream_t s);
int group_ref_blocks(int M_pad);
cudaError_t launch_group_swap(const GroupSlot *slots, const int2 *map, int total_blocks, size_t smem,
                              cudaStream_t s);
// out[2k .. 2k + 1] = slots[k].w.v0[0 .. 1] for k < n
cudaError_t launch_group_v0(const GroupSlot *slots, int n, unsigned long long *out, cudaStream_t s);
cudaError_t launch_group_select(const GroupSlot *slots, const int2 *map, int total_blocks, cudaStream_t s);
cudaError_t launch_group_refresh(const GroupSlot *slots, const int2 *map, int total_blocks, int maxK,
                                 cudaStream_t s);
cudaError_t launch_gather_states(const GroupSlot *slots, int n, TabuDevState *out, cudaStream_t s);

}  // namespace stg
