// Allocation-free variant of the swap-neighbourhood evaluation
// (stage_evaluate_swaps_noalloc).  Its scratch -- per-mission best and
// second-best arrays, the objective accumulators and the candidate list -- lives
// in one file-scope device array of fixed size, so the call itself never
// allocates device or pinned host memory.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "stage_internal.h"

namespace stg {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)STAGE_NOALLOC_SCRATCH_MB << 20;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch layout for (K, B, M_pad); returns the bytes needed.  With base ==
// nullptr only the size is computed.
size_t layout(unsigned char *base, int K, int B, int M_pad, TabuBuffers &tb)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = align256(off);
        unsigned char *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    tb.a = reinterpret_cast<int32_t *>(take((size_t)M_pad * 4));
    tb.b = reinterpret_cast<int32_t *>(take((size_t)M_pad * 4));
    tb.s1 = reinterpret_cast<int16_t *>(take((size_t)M_pad * 2));
    tb.s2 = reinterpret_cast<int16_t *>(take((size_t)M_pad * 2));
    tb.v0 = reinterpret_cast<unsigned long long *>(take(16));
    tb.loss_c = reinterpret_cast<unsigned long long *>(take((size_t)K * 8));
    tb.loss_d = reinterpret_cast<unsigned long long *>(take((size_t)K * 8));
    tb.gain_c = reinterpret_cast<int *>(take((size_t)B * 4));
    tb.gain_d = reinterpret_cast<unsigned long long *>(take((size_t)B * 8));
    tb.extra_c = reinterpret_cast<int *>(take((size_t)K * B * 4));
    tb.extra_d = reinterpret_cast<unsigned long long *>(take((size_t)K * B * 8));
    tb.open = reinterpret_cast<int32_t *>(take((size_t)K * 4));
    tb.cand = reinterpret_cast<int32_t *>(take((size_t)B * 4));
    tb.st = reinterpret_cast<TabuDevState *>(take(sizeof(TabuDevState)));
    tb.best_open = nullptr;
    tb.expiry = nullptr;
    tb.partials = nullptr;
    tb.traj = nullptr;
    return align256(off);
}

// One block: copy the placement, list the closed available bases in ascending
// order, clear the accumulators and the state.  Earlier calls' contents are
// overwritten here, so nothing stale survives into this call.  A placement
// with an id outside [0, B), a repeated id or an unavailable base is refused
// on the device: every slot is pointed at base 0 (so the per-mission pass
// reads inside the table), the candidate list is left empty and the state's
// err word is set, so no objective is written and the outputs keep the -1
// the call filled them with.
__global__ void k_noalloc_prepare(TabuBuffers w, const int32_t *__restrict__ open,
                                  const uint8_t *__restrict__ avail)
{
    __shared__ unsigned is_open[(STAGE_NOALLOC_MAX_BASES + 31) / 32];
    __shared__ int s_count, s_bad;
    const int B = w.B, K = w.K;
    for (int q = threadIdx.x; q < (B + 31) / 32; q += blockDim.x) is_open[q] = 0;
    if (threadIdx.x == 0) {
        s_count = 0;
        s_bad = 0;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const int o = open[k];
        bool bad = o < 0 || o >= B;
        if (!bad) {
            const unsigned bit = 1u << (o & 31);
            bad = (atomicOr(&is_open[o >> 5], bit) & bit) != 0 || (avail != nullptr && avail[o] == 0);
        }
        if (bad) s_bad = 1;
        w.loss_c[k] = 0;
        w.loss_d[k] = 0;
    }
    __syncthreads();
    const bool bad = s_bad != 0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) w.open[k] = bad ? 0 : open[k];
    // ordered compaction, one warp-sized chunk of bases at a time
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32 && !bad) {
        for (int b0 = 0; b0 < B; b0 += 32) {
            const int b = b0 + lane;
            const bool take = b < B && !((is_open[b >> 5] >> (b & 31)) & 1u) && (avail == nullptr || avail[b] != 0);
            const unsigned mask = __ballot_sync(0xffffffffu, take);
            if (take) w.cand[s_count + __popc(mask & ((1u << lane) - 1u))] = b;
            __syncwarp();
            if (lane == 0) s_count += __popc(mask);
            __syncwarp();
        }
    }
    for (size_t q = threadIdx.x; q < (size_t)K * B; q += blockDim.x) {
        w.extra_c[q] = 0;
        w.extra_d[q] = 0;
    }
    for (int q = threadIdx.x; q < B; q += blockDim.x) {
        w.gain_c[q] = 0;
        w.gain_d[q] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        w.v0[0] = 0;
        w.v0[1] = 0;
        TabuDevState st;
        memset(&st, 0, sizeof st);
        st.nC = s_count;
        st.best_iter = -1;
        st.err = bad ? kErrBadSlot : 0;
        *w.st = st;
    }
}

stage_status fail(char *errbuf, size_t errlen, stage_status code, const char *msg)
{
    if (errbuf && errlen) snprintf(errbuf, errlen, "%s", msg);
    return code;
}

}  // namespace
}  // namespace stg

using namespace stg;

extern "C" stage_status stage_evaluate_swaps_noalloc(const int32_t *cost, int32_t B, int32_t M,
                                                     int32_t M_pad, const uint8_t *base_available,
                                                     const int32_t *open, int32_t K, int32_t R,
                                                     int64_t *out_cov, int64_t *out_dist,
                                                     void *stream, char *errbuf, size_t errlen)
{
    char msg[256];
    if (!cost || !open || !out_cov || !out_dist)
        return fail(errbuf, errlen, STAGE_ERR_INVALID_ARG, "a required device pointer is NULL");
    if (B < 1 || M < 1 || K < 1 || K > B)
        return fail(errbuf, errlen, STAGE_ERR_INVALID_ARG, "need B >= 1, M >= 1 and 1 <= K <= B");
    if (M_pad < M || (M_pad & 3) || (reinterpret_cast<uintptr_t>(cost) & 15))
        return fail(errbuf, errlen, STAGE_ERR_INVALID_ARG,
                    "the table needs M_pad >= M, M_pad a multiple of 4 and a 16-byte aligned base");
    if (R < 0 || R == INT32_MAX) return fail(errbuf, errlen, STAGE_ERR_OUT_OF_RANGE, "R outside [0, INT32_MAX)");
    if (B > STAGE_NOALLOC_MAX_BASES || K > STAGE_MAX_K) {
        snprintf(msg, sizeof msg, "B=%d or K=%d beyond the allocation-free limits (B <= %d, K <= %d)", B, K,
                 STAGE_NOALLOC_MAX_BASES, STAGE_MAX_K);
        return fail(errbuf, errlen, STAGE_ERR_OUT_OF_RANGE, msg);
    }
    TabuBuffers tb{};
    const size_t need = layout(nullptr, K, B, M_pad, tb);
    if (need > kNoAllocScratchBytes) {
        snprintf(msg, sizeof msg,
                 "scratch for M_pad=%d, K=%d, B=%d needs %zu bytes; the static scratch holds %zu "
                 "(about 12 bytes per mission plus 12 per (K, B) pair)",
                 M_pad, K, B, need, kNoAllocScratchBytes);
        return fail(errbuf, errlen, STAGE_ERR_OUT_OF_RANGE, msg);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fail(errbuf, errlen, STAGE_ERR_CUDA, "no current CUDA device");
    }
    unsigned char *base = nullptr;
    {
        // first call on this device: look up the scratch array's device address
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                snprintf(msg, sizeof msg, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                return fail(errbuf, errlen, STAGE_ERR_CUDA, msg);
            }
            // function attributes and the SM count, once per device
            e = kernels_init();
            if (e != cudaSuccess) {
                cudaGetLastError();
                snprintf(msg, sizeof msg, "kernel set-up failed: %s", cudaGetErrorString(e));
                return fail(errbuf, errlen, STAGE_ERR_CUDA, msg);
            }
            g_scratch_addr[dev] = static_cast<unsigned char *>(p);
        }
        base = g_scratch_addr[dev];
    }
    layout(base, K, B, M_pad, tb);
    tb.K = K;
    tb.B = B;
    tb.M = M;
    tb.M_pad = M_pad;
    tb.R = R;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)K * B;
    cudaError_t e = cudaMemsetAsync(out_cov, 0xff, n * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(out_dist, 0xff, n * 8, s);
    if (e == cudaSuccess) {
        k_noalloc_prepare<<<1, 1024, 0, s>>>(tb, open, base_available);
        e = cudaGetLastError();
    }
    // the candidate count is known on the device only: launch for B - K rows;
    // blocks past the real count find no rows and do nothing
    if (e == cudaSuccess) e = launch_init(tb, cost, s);
    if (e == cudaSuccess) e = launch_swap_eval(tb, cost, B - K, 1, s);
    if (e == cudaSuccess) e = launch_swap_table(tb, B - K, reinterpret_cast<long long *>(out_cov),
                                                reinterpret_cast<long long *>(out_dist), s);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "launch failed: %s", cudaGetErrorString(e));
        return fail(errbuf, errlen, STAGE_ERR_CUDA, msg);
    }
    return STAGE_OK;
}
