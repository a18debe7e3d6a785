// sm_103a kernels of the staging engine: cost table, ranking, evaluation and
// the Tabu loop (per-mission best/second-best, swap neighbourhood, move
// selection, incremental refresh).  Integer arithmetic throughout; float64 only
// for the one square root per leg.
#include <cuda_runtime.h>
#include <stdint.h>

#include "stage_internal.h"

namespace stg {

// --------------------------------------------------------------------------
// helpers
// --------------------------------------------------------------------------

// Leg cost (Sec. 3; Euclidean in place of Eq. 1): ceil of the correctly rounded
// float64 square root of the exact squared distance.  |coord| <= 2^24 keeps the
// square below 2^52, where int64 -> float64 is exact and the ceiling of the
// rounded root equals the exact integer ceiling.
__device__ __forceinline__ int32_t leg_ceil(int x1, int y1, int x2, int y2)
{
    long long dx = (long long)x1 - (long long)x2;
    long long dy = (long long)y1 - (long long)y2;
    double r = __dsqrt_rn(__ll2double_rn(dx * dx + dy * dy));
    return (int32_t)ceil(r);
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

// --------------------------------------------------------------------------
// a1: cost table.  c[b][m] = leg(b, p_m) + leg(p_m, d_m) + leg(d_m, b).
// --------------------------------------------------------------------------

__global__ void k_pickup_drop_leg(int M, const int2 *__restrict__ pick,
                                  const int2 *__restrict__ drop, int32_t *__restrict__ pd)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        int2 p = pick[m], d = drop[m];
        pd[m] = leg_ceil(p.x, p.y, d.x, d.y);
    }
}

constexpr int kTableBasesPerBlock = 8;

// Each thread owns 4 consecutive missions and writes them for 8 bases (one
// 16-byte store per base row); pads (m >= M) hold INT32_MAX.
__global__ void __launch_bounds__(256) k_build_table(int B, int M, int M_pad,
                                                     const int2 *__restrict__ base,
                                                     const int2 *__restrict__ pick,
                                                     const int2 *__restrict__ drop,
                                                     const int32_t *__restrict__ pd,
                                                     int32_t *__restrict__ cost)
{
    const int b0 = blockIdx.y * kTableBasesPerBlock;
    const int n4 = M_pad >> 2;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += gridDim.x * blockDim.x) {
        const int m = q << 2;
        int2 p[4], d[4];
        int l[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            if (m + e < M) { p[e] = pick[m + e]; d[e] = drop[m + e]; l[e] = pd[m + e]; }
            else { p[e] = make_int2(0, 0); d[e] = make_int2(0, 0); l[e] = -1; }
        }
#pragma unroll 1
        for (int bb = 0; bb < kTableBasesPerBlock; bb++) {
            const int b = b0 + bb;
            if (b >= B) break;
            const int2 o = base[b];
            int v[4];
#pragma unroll
            for (int e = 0; e < 4; e++)
                v[e] = (l[e] >= 0) ? leg_ceil(o.x, o.y, p[e].x, p[e].y) + l[e] +
                                         leg_ceil(d[e].x, d[e].y, o.x, o.y)
                                   : kInf;
            reinterpret_cast<int4 *>(cost + (size_t)b * M_pad)[q] = make_int4(v[0], v[1], v[2], v[3]);
        }
    }
}

// Input check: flag |coordinate| > STAGE_MAX_COORD (device-resident inputs).
__global__ void k_check_coords(const int32_t *__restrict__ v, size_t n, int *__restrict__ bad)
{
    int found = 0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int x = v[k];
        found |= (x > STAGE_MAX_COORD) | (x < -STAGE_MAX_COORD);
    }
    if (__syncthreads_or(found) && threadIdx.x == 0) atomicOr(bad, 1);
}

cudaError_t launch_check_coords(const int32_t *v, size_t n, int *bad, cudaStream_t s)
{
    size_t g = (n + 255) / 256;
    if (g > 1024) g = 1024;
    if (g == 0) return cudaSuccess;
    k_check_coords<<<(int)g, 256, 0, s>>>(v, n, bad);
    return cudaGetLastError();
}

cudaError_t launch_table(int B, int M, int M_pad, const int2 *base, const int2 *pick,
                         const int2 *drop, int32_t *pd, int32_t *cost, cudaStream_t s)
{
    int g1 = (M + 255) / 256;
    if (g1 > 4096) g1 = 4096;
    k_pickup_drop_leg<<<g1, 256, 0, s>>>(M, pick, drop, pd);
    int n4 = M_pad / 4;
    int gx = (n4 + 255) / 256;
    int gy = (B + kTableBasesPerBlock - 1) / kTableBasesPerBlock;
    // enough blocks for every SM even when B is small
    if (gx > 1024) gx = 1024;
    k_build_table<<<dim3(gx, gy), 256, 0, s>>>(B, M, M_pad, base, pick, drop, pd, cost);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// a2: base ranking (Alg. 1).  S[b] = sum_m c[b][m]; top K by (S asc, b asc).
// --------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_row_sums(const int32_t *__restrict__ cost, int M,
                                                  int M_pad, unsigned long long *__restrict__ S)
{
    const int b = blockIdx.y;
    const int4 *row = reinterpret_cast<const int4 *>(cost + (size_t)b * M_pad);
    const int n4 = M_pad >> 2;
    long long acc = 0, dummy = 0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += gridDim.x * blockDim.x) {
        int4 v = __ldcs(row + q);
        int m = q << 2;
        acc += (m + 0 < M ? (long long)v.x : 0) + (m + 1 < M ? (long long)v.y : 0) +
               (m + 2 < M ? (long long)v.z : 0) + (m + 3 < M ? (long long)v.w : 0);
    }
    block_sum2<256>(acc, dummy);
    if (threadIdx.x == 0) add_ull(&S[b], acc);
}

cudaError_t launch_rowsum(const int32_t *cost, int B, int M, int M_pad, unsigned long long *S,
                          cudaStream_t s)
{
    int n4 = M_pad / 4;
    int gx = (n4 + 256 * 8 - 1) / (256 * 8);   // ~8 int4 per thread
    if (gx < 1) gx = 1;
    k_row_sums<<<dim3(gx, B), 256, 0, s>>>(cost, M, M_pad, S);
    return cudaGetLastError();
}

// rank(b) = number of available b' with (S[b'], b') < (S[b], b); the K with
// rank < K are written in rank order.
__global__ void __launch_bounds__(256) k_topk(const unsigned long long *__restrict__ S,
                                              const uint8_t *__restrict__ avail, int B, int K,
                                              int32_t *__restrict__ open)
{
    __shared__ long long sS[1024];
    __shared__ uint8_t sA[1024];
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const bool mine = b < B && avail[b];
    const long long s = mine ? (long long)S[b] : 0;
    int rank = 0;
    for (int t0 = 0; t0 < B; t0 += 1024) {
        __syncthreads();
        for (int k = threadIdx.x; k < 1024; k += blockDim.x) {
            int bb = t0 + k;
            sS[k] = bb < B ? (long long)S[bb] : 0;
            sA[k] = bb < B ? avail[bb] : 0;
        }
        __syncthreads();
        if (mine) {
            const int n = min(1024, B - t0);
            for (int k = 0; k < n; k++) {
                const int bb = t0 + k;
                rank += (sA[k] && (sS[k] < s || (sS[k] == s && bb < b))) ? 1 : 0;
            }
        }
    }
    if (mine && rank < K) open[rank] = b;
}

cudaError_t launch_topk(const unsigned long long *S, const uint8_t *avail, int B, int K,
                        int32_t *open, cudaStream_t s)
{
    k_topk<<<(B + 255) / 256, 256, 0, s>>>(S, avail, B, K, open);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// F(O): every mission flown from its nearest open base (Eq. 2 with coverage).
// --------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_evaluate(const int32_t *__restrict__ cost, int M, int M_pad,
                                                  const int32_t *__restrict__ open, int K, int R,
                                                  unsigned long long *__restrict__ out)
{
    extern __shared__ int s_open[];
    for (int k = threadIdx.x; k < K; k += blockDim.x) s_open[k] = open[k];
    __syncthreads();
    long long cov = 0, dist = 0;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        int best = kInf;
        for (int k = 0; k < K; k++) best = min(best, __ldg(cost + (size_t)s_open[k] * M_pad + m));
        if (best <= R) { cov += 1; dist += best; }
    }
    block_sum2<256>(cov, dist);
    if (threadIdx.x == 0) { add_ull(&out[0], cov); add_ull(&out[1], dist); }
}

cudaError_t launch_evaluate(const int32_t *cost, int M, int M_pad, const int32_t *open, int K,
                            int R, unsigned long long *out2, cudaStream_t s)
{
    int g = (M + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    k_evaluate<<<g, 256, K * sizeof(int), s>>>(cost, M, M_pad, open, K, R, out2);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// a3: per-mission best and second-best open base (Alg. 1, ranking of the
// chosen bases for each mission), ordered by (cost, base id), with
// V0 = sum f(a) and loss[s] = sum_{m: b1 = s} f(b) - f(a).
// --------------------------------------------------------------------------

// Accumulate f(b) - f(a) of one mission into the shared loss of its best slot.
__device__ __forceinline__ void mission_terms(int a, int b, int R, long long &v0c, long long &v0d,
                                              int *s_lc, unsigned long long *s_ld, int s1)
{
    const int ca = a <= R, cb = b <= R;
    const long long da = ca ? a : 0, db = cb ? b : 0;
    v0c += ca;
    v0d += da;
    const int dc = cb - ca;
    const long long dd = db - da;
    if (dc) atomicAdd(&s_lc[s1], dc);
    if (dd) atomicAdd(&s_ld[s1], (unsigned long long)dd);
}

// Shared layout used by init and refresh: open ids [K], loss cov [K], loss dist [K].
__device__ __forceinline__ void flush_loss_v0(const TabuBuffers &w, int *s_lc,
                                              unsigned long long *s_ld, long long v0c,
                                              long long v0d)
{
    block_sum2<256>(v0c, v0d);
    if (threadIdx.x == 0) {
        if (v0c) add_ull(&w.v0[0], v0c);
        if (v0d) add_ull(&w.v0[1], v0d);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < w.K; k += blockDim.x) {
        if (s_lc[k]) add_ull(&w.loss_c[k], s_lc[k]);
        if (s_ld[k]) atomicAdd(&w.loss_d[k], s_ld[k]);
    }
}

__device__ __forceinline__ void scan_best_two(const int32_t *__restrict__ cost, size_t M_pad, int m,
                                              const int *s_open, int K, int &a, int &b, int &k1,
                                              int &k2)
{
    int c1 = kInf, c2 = kInf, i1 = 0x7fffffff, i2 = 0x7fffffff;
    k1 = -1;
    k2 = -1;
    for (int k = 0; k < K; k++) {
        const int o = s_open[k];
        const int c = __ldg(cost + (size_t)o * M_pad + m);
        if (k1 < 0 || c < c1 || (c == c1 && o < i1)) {
            k2 = k1; c2 = c1; i2 = i1;
            k1 = k; c1 = c; i1 = o;
        } else if (k2 < 0 || c < c2 || (c == c2 && o < i2)) {
            k2 = k; c2 = c; i2 = o;
        }
    }
    a = c1;
    b = c2;
}

__global__ void __launch_bounds__(256) k_init(TabuBuffers w, const int32_t *__restrict__ cost)
{
    extern __shared__ unsigned long long sm_init[];
    unsigned long long *s_ld = sm_init;
    int *s_lc = reinterpret_cast<int *>(s_ld + w.K);
    int *s_open = s_lc + w.K;
    for (int k = threadIdx.x; k < w.K; k += blockDim.x) {
        s_open[k] = w.open[k];
        s_lc[k] = 0;
        s_ld[k] = 0;
    }
    __syncthreads();
    long long v0c = 0, v0d = 0;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < w.M_pad; m += gridDim.x * blockDim.x) {
        if (m >= w.M) {
            w.a[m] = kInf; w.b[m] = kInf; w.s1[m] = 0; w.s2[m] = -1;
            continue;
        }
        int a, b, k1, k2;
        scan_best_two(cost, w.M_pad, m, s_open, w.K, a, b, k1, k2);
        w.a[m] = a; w.b[m] = b; w.s1[m] = (int16_t)k1; w.s2[m] = (int16_t)k2;
        mission_terms(a, b, w.R, v0c, v0d, s_lc, s_ld, k1);
    }
    __syncthreads();
    flush_loss_v0(w, s_lc, s_ld, v0c, v0d);
}

static int grid_missions(int M_pad)
{
    int g = (M_pad + 255) / 256;
    return g > 152 * 8 ? 152 * 8 : g;
}

cudaError_t launch_init(const TabuBuffers &w, const int32_t *cost, cudaStream_t s)
{
    size_t sm = (size_t)w.K * (8 + 4 + 4);
    k_init<<<grid_missions(w.M_pad), 256, sm, s>>>(w, cost);
    return cudaGetLastError();
}

// Current objective = V0 of the start placement; best so far = start unless resumed.
__global__ void k_begin(TabuBuffers w, int resumed)
{
    TabuDevState *st = w.st;
    if (threadIdx.x == 0) {
        st->cur_cov = (long long)w.v0[0];
        st->cur_dist = (long long)w.v0[1];
        if (!resumed) {
            st->best_cov = st->cur_cov;
            st->best_dist = st->cur_dist;
            st->best_iter = -1;
        }
    }
    if (!resumed)
        for (int k = threadIdx.x; k < w.K; k += blockDim.x) w.best_open[k] = w.open[k];
}

cudaError_t launch_begin(const TabuBuffers &w, int resumed, cudaStream_t s)
{
    k_begin<<<1, 256, 0, s>>>(w, resumed);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// a4: the swap neighbourhood.  For every closed available j (a candidate row)
// and every mission m, with x = c[j][m], a = best, b = second best, s1 = slot
// of the best base:
//     x < b :  extra[s1][j] += f(max(x, a)) - f(b)
//     x < a :  gain[j]      += f(x) - f(a)
// so that F(close slot s, open j) = V0 + gain[j] + loss[s] + extra[s][j]
// (fast interchange: Whitaker 1983; Resende and Werneck 2007).
//
// Grid: x = mission segments, y = chunks of J candidate rows.  A thread owns 4
// consecutive missions at a time (one 16-byte load per row); the best /
// second-best values stay in registers across the J rows.  extra is
// accumulated per block in shared memory and flushed with one global atomic
// per nonzero (slot, row); gain in registers, reduced per warp at the end.
// --------------------------------------------------------------------------

constexpr int kSwapJ = 8;
constexpr int kSwapThreads = 256;
constexpr int kSwapSegment = 16384;   // missions per block (multiple of 4 * kSwapThreads)

template <int J>
__device__ __forceinline__ void swap_element(int x, int a, int b, int s, int r, int R,
                                             int *ex_c, unsigned long long *ex_d, int (&gc)[J],
                                             long long (&gd)[J])
{
    if (x < b) {
        const int y = max(x, a);
        const int cy = y <= R, cb = b <= R;
        const int dc = cy - cb;
        const long long dd = (cy ? (long long)y : 0ll) - (cb ? (long long)b : 0ll);
        if (dc | (dd != 0)) {
            atomicAdd(&ex_c[s * J + r], dc);
            atomicAdd(&ex_d[s * J + r], (unsigned long long)dd);
        }
        if (x < a) {
            const int cx = x <= R, ca = a <= R;
            gc[r] += cx - ca;
            gd[r] += (cx ? (long long)x : 0ll) - (ca ? (long long)a : 0ll);
        }
    }
}

template <int J>
__global__ void __launch_bounds__(kSwapThreads, 2)
k_swap_eval(TabuBuffers w, const int32_t *__restrict__ cost, int ignore_done)
{
    if (!ignore_done && w.st->done) return;
    extern __shared__ unsigned long long sm_swap[];
    const int K = w.K;
    unsigned long long *ex_d = sm_swap;                         // [K * J]
    int *ex_c = reinterpret_cast<int *>(ex_d + K * J);          // [K * J]
    __shared__ int rows[J];
    __shared__ int g_c[J];
    __shared__ unsigned long long g_d[J];
    const int nC = w.st->nC;
    const int c0 = blockIdx.y * J;
    for (int k = threadIdx.x; k < K * J; k += blockDim.x) { ex_d[k] = 0; ex_c[k] = 0; }
    if (threadIdx.x < J) {
        rows[threadIdx.x] = (c0 + threadIdx.x < nC) ? w.cand[c0 + threadIdx.x] : -1;
        g_c[threadIdx.x] = 0;
        g_d[threadIdx.x] = 0;
    }
    __syncthreads();

    int gc[J];
    long long gd[J];
    const int4 *rowp[J];
#pragma unroll
    for (int r = 0; r < J; r++) {
        gc[r] = 0;
        gd[r] = 0;
        rowp[r] = rows[r] >= 0 ? reinterpret_cast<const int4 *>(cost + (size_t)rows[r] * w.M_pad)
                               : nullptr;
    }
    const int R = w.R;
    const int m_begin = blockIdx.x * kSwapSegment;
    const int m_end = min(m_begin + kSwapSegment, w.M_pad);
    for (int m = m_begin + 4 * threadIdx.x; m < m_end; m += 4 * kSwapThreads) {
        const int q = m >> 2;
        const int4 a4 = __ldg(reinterpret_cast<const int4 *>(w.a) + q);
        const int4 b4 = __ldg(reinterpret_cast<const int4 *>(w.b) + q);
        const uint2 sp = __ldg(reinterpret_cast<const uint2 *>(w.s1) + q);
        const int s_0 = (int)(int16_t)(sp.x & 0xffff), s_1 = (int)(int16_t)(sp.x >> 16);
        const int s_2 = (int)(int16_t)(sp.y & 0xffff), s_3 = (int)(int16_t)(sp.y >> 16);
        int4 x[J];
#pragma unroll
        for (int r = 0; r < J; r++)
            x[r] = rowp[r] ? __ldcs(rowp[r] + q) : make_int4(kInf, kInf, kInf, kInf);
#pragma unroll
        for (int r = 0; r < J; r++) {
            swap_element<J>(x[r].x, a4.x, b4.x, s_0, r, R, ex_c, ex_d, gc, gd);
            swap_element<J>(x[r].y, a4.y, b4.y, s_1, r, R, ex_c, ex_d, gc, gd);
            swap_element<J>(x[r].z, a4.z, b4.z, s_2, r, R, ex_c, ex_d, gc, gd);
            swap_element<J>(x[r].w, a4.w, b4.w, s_3, r, R, ex_c, ex_d, gc, gd);
        }
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < J; r++) {
        const int v = warp_sum_i(gc[r]);
        const long long u = warp_sum_ll(gd[r]);
        if (lane == 0 && (v | (u != 0))) {
            atomicAdd(&g_c[r], v);
            atomicAdd(&g_d[r], (unsigned long long)u);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K * J; k += blockDim.x) {
        const int r = k % J, s = k / J;
        const int j = rows[r];
        if (j < 0) continue;
        const int c = ex_c[k];
        const unsigned long long d = ex_d[k];
        if (c | (d != 0)) {
            atomicAdd(&w.extra_c[(size_t)s * w.B + j], c);
            atomicAdd(&w.extra_d[(size_t)s * w.B + j], d);
        }
    }
    if (threadIdx.x < J && rows[threadIdx.x] >= 0) {
        const int j = rows[threadIdx.x];
        if (g_c[threadIdx.x]) atomicAdd(&w.gain_c[j], g_c[threadIdx.x]);
        if (g_d[threadIdx.x]) atomicAdd(&w.gain_d[j], g_d[threadIdx.x]);
    }
}

cudaError_t launch_swap_eval(const TabuBuffers &w, const int32_t *cost, int nC, int ignore_done,
                             cudaStream_t s)
{
    if (nC <= 0) return cudaSuccess;
    dim3 grid((w.M_pad + kSwapSegment - 1) / kSwapSegment, (nC + kSwapJ - 1) / kSwapJ);
    size_t sm = (size_t)w.K * kSwapJ * (8 + 4);
    k_swap_eval<kSwapJ><<<grid, kSwapThreads, sm, s>>>(w, cost, ignore_done);
    return cudaGetLastError();
}

// F(s, j) = V0 + gain[j] + loss[s] + extra[s][j] for every slot and candidate.
__global__ void k_swap_table(TabuBuffers w, long long *__restrict__ out_c, long long *__restrict__ out_d)
{
    const int nC = w.st->nC;
    const long long v0c = (long long)w.v0[0], v0d = (long long)w.v0[1];
    const long long total = (long long)w.K * nC;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(q / nC), c = (int)(q % nC);
        const int j = w.cand[c];
        const size_t sj = (size_t)s * w.B + j;
        out_c[sj] = v0c + w.gain_c[j] + (long long)w.loss_c[s] + w.extra_c[sj];
        out_d[sj] = v0d + (long long)w.gain_d[j] + (long long)w.loss_d[s] + (long long)w.extra_d[sj];
    }
}

cudaError_t launch_swap_table(const TabuBuffers &w, int nC, long long *out_c, long long *out_d,
                              cudaStream_t s)
{
    long long total = (long long)w.K * nC;
    if (total <= 0) return cudaSuccess;
    long long g = (total + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    k_swap_table<<<(int)g, 256, 0, s>>>(w, out_c, out_d);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// a5 + a6: choose the move and apply it (Alg. 3 as read for identical
// vehicles).  Each block reduces its share of the K x nC candidates to the
// best admissible and the best overall key; the last block to finish reduces
// the block results, applies the move, updates the tabu expiries, the best so
// far and the trajectory, and clears V0 / loss for the refresh kernel.
// --------------------------------------------------------------------------

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

template <int NT>
__device__ __forceinline__ void block_best2(MoveKey &adm, MoveKey &all, MoveKey *s_adm, MoveKey *s_all)
{
    s_adm[threadIdx.x] = adm;
    s_all[threadIdx.x] = all;
    __syncthreads();
    for (int h = NT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            if (key_better(s_adm[threadIdx.x + h], s_adm[threadIdx.x])) s_adm[threadIdx.x] = s_adm[threadIdx.x + h];
            if (key_better(s_all[threadIdx.x + h], s_all[threadIdx.x])) s_all[threadIdx.x] = s_all[threadIdx.x + h];
        }
        __syncthreads();
    }
    adm = s_adm[0];
    all = s_all[0];
}

__global__ void __launch_bounds__(kSelectThreads) k_select(TabuBuffers w)
{
    TabuDevState *st = w.st;
    if (st->done) return;
    __shared__ MoveKey s_adm[kSelectThreads], s_all[kSelectThreads];
    __shared__ int s_last, s_newbest;
    const int t = st->t;
    const int nC = st->nC;
    const int B = w.B;
    const long long v0c = (long long)w.v0[0], v0d = (long long)w.v0[1];
    const long long bc = st->best_cov, bd = st->best_dist;
    MoveKey adm = invalid_key(), all = invalid_key();
    const long long total = (long long)w.K * nC;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(q / nC), c = (int)(q % nC);
        const int i = w.open[s], j = w.cand[c];
        const size_t sj = (size_t)s * B + j;
        MoveKey k;
        k.cov = v0c + w.gain_c[j] + (long long)w.loss_c[s] + w.extra_c[sj];
        k.dist = v0d + (long long)w.gain_d[j] + (long long)w.loss_d[s] + (long long)w.extra_d[sj];
        k.i = i; k.j = j; k.s = s; k.c = c; k.valid = 1;
        k.tabu = (t < w.expiry[i]) || (t < w.expiry[j]);
        if (key_better(k, all)) all = k;
        if ((!k.tabu || obj_better(k.cov, k.dist, bc, bd)) && key_better(k, adm)) adm = k;
    }
    block_best2<kSelectThreads>(adm, all, s_adm, s_all);
    if (threadIdx.x == 0) {
        w.partials[2 * blockIdx.x] = adm;
        w.partials[2 * blockIdx.x + 1] = all;
        __threadfence();
        const unsigned int ticket = atomicAdd(&st->ticket, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    adm = invalid_key();
    all = invalid_key();
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        MoveKey pa = load_key_cg(&w.partials[2 * b]);
        MoveKey px = load_key_cg(&w.partials[2 * b + 1]);
        if (key_better(pa, adm)) adm = pa;
        if (key_better(px, all)) all = px;
    }
    __syncthreads();
    block_best2<kSelectThreads>(adm, all, s_adm, s_all);
    if (threadIdx.x == 0) {
        st->ticket = 0;
        s_newbest = 0;
        if (!all.valid) {
            st->done = 1;                       // no closed available base
        } else if (st->cur_cov != v0c || st->cur_dist != v0d) {
            st->err |= kErrObjectiveMismatch;   // refresh disagreed with the chosen move
            st->done = 1;
        } else {
            const MoveKey P = adm.valid ? adm : all;
            int flags = adm.valid ? (adm.tabu ? STAGE_MOVE_ASPIRATION : 0) : STAGE_MOVE_FALLBACK;
            if (!st->accept_worsening && !obj_better(P.cov, P.dist, st->cur_cov, st->cur_dist)) {
                st->done = 1;                   // improving-only rule: no improving move
            } else {
                w.open[P.s] = P.j;
                w.cand[P.c] = P.i;
                w.expiry[P.i] = t + st->tenure + 1;
                w.expiry[P.j] = t + st->tenure + 1;
                st->cur_cov = P.cov;
                st->cur_dist = P.dist;
                if (obj_better(P.cov, P.dist, st->best_cov, st->best_dist)) {
                    st->best_cov = P.cov;
                    st->best_dist = P.dist;
                    st->best_iter = t;
                    flags |= STAGE_MOVE_NEW_BEST;
                    s_newbest = 1;
                }
                if (st->n_moves < st->traj_cap) {
                    stage_move mv;
                    mv.iter = t; mv.i = P.i; mv.j = P.j; mv.flags = flags;
                    mv.cov = P.cov; mv.dist = P.dist;
                    w.traj[st->n_moves] = mv;
                }
                st->n_moves += 1;
                st->t = t + 1;
                st->mv_s = P.s; st->mv_i = P.i; st->mv_j = P.j;
                w.v0[0] = 0;
                w.v0[1] = 0;
            }
        }
    }
    __syncthreads();
    if (st->done) return;
    for (int k = threadIdx.x; k < w.K; k += blockDim.x) {
        w.loss_c[k] = 0;
        w.loss_d[k] = 0;
        if (s_newbest) w.best_open[k] = w.open[k];
    }
}

cudaError_t launch_select(const TabuBuffers &w, cudaStream_t s)
{
    k_select<<<kSelectBlocks, kSelectThreads, 0, s>>>(w);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// a7: incremental refresh after move (slot s*, opened j*).  A mission whose
// best and second best do not use slot s* only has to consider j*; the others
// rescan the K open bases.  V0 and loss are rebuilt from the new arrays, and
// gain / extra are cleared for the next evaluation.
// --------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_refresh(TabuBuffers w, const int32_t *__restrict__ cost)
{
    TabuDevState *st = w.st;
    if (st->done) return;
    extern __shared__ unsigned long long sm_ref[];
    unsigned long long *s_ld = sm_ref;
    int *s_lc = reinterpret_cast<int *>(s_ld + w.K);
    int *s_open = s_lc + w.K;
    for (int k = threadIdx.x; k < w.K; k += blockDim.x) {
        s_open[k] = w.open[k];
        s_lc[k] = 0;
        s_ld[k] = 0;
    }
    __syncthreads();
    const int ss = st->mv_s, jj = st->mv_j;
    const size_t M_pad = w.M_pad;
    const int32_t *rowj = cost + (size_t)jj * M_pad;
    long long v0c = 0, v0d = 0;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < w.M; m += gridDim.x * blockDim.x) {
        int a = w.a[m], b = w.b[m];
        int k1 = w.s1[m], k2 = w.s2[m];
        if (k1 != ss && k2 != ss) {
            const int x = __ldcs(rowj + m);
            const int id1 = s_open[k1];
            const int id2 = k2 >= 0 ? s_open[k2] : 0x7fffffff;
            if (x < a || (x == a && jj < id1)) {
                k2 = k1; b = a;
                k1 = ss; a = x;
                w.a[m] = a; w.b[m] = b; w.s1[m] = (int16_t)k1; w.s2[m] = (int16_t)k2;
            } else if (k2 < 0 || x < b || (x == b && jj < id2)) {
                k2 = ss; b = x;
                w.b[m] = b; w.s2[m] = (int16_t)k2;
            }
        } else {
            scan_best_two(cost, M_pad, m, s_open, w.K, a, b, k1, k2);
            w.a[m] = a; w.b[m] = b; w.s1[m] = (int16_t)k1; w.s2[m] = (int16_t)k2;
        }
        mission_terms(a, b, w.R, v0c, v0d, s_lc, s_ld, k1);
    }
    // clear the neighbourhood accumulators for the next evaluation
    const size_t nE = (size_t)w.K * w.B;
    const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    for (size_t q = tid; q < nE; q += nth) { w.extra_c[q] = 0; w.extra_d[q] = 0; }
    for (size_t q = tid; q < (size_t)w.B; q += nth) { w.gain_c[q] = 0; w.gain_d[q] = 0; }
    __syncthreads();
    flush_loss_v0(w, s_lc, s_ld, v0c, v0d);
}

cudaError_t launch_refresh(const TabuBuffers &w, const int32_t *cost, cudaStream_t s)
{
    size_t sm = (size_t)w.K * (8 + 4 + 4);
    k_refresh<<<grid_missions(w.M_pad), 256, sm, s>>>(w, cost);
    return cudaGetLastError();
}

__global__ void k_export_best_two(TabuBuffers w, int32_t *__restrict__ a, int32_t *__restrict__ b,
                                  int32_t *__restrict__ b1, int32_t *__restrict__ b2)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < w.M; m += gridDim.x * blockDim.x) {
        a[m] = w.a[m];
        b[m] = w.b[m];
        const int k1 = w.s1[m], k2 = w.s2[m];
        b1[m] = w.open[k1];
        b2[m] = k2 >= 0 ? w.open[k2] : -1;
    }
}

cudaError_t launch_export_best_two(const TabuBuffers &w, int32_t *a, int32_t *b, int32_t *b1,
                                   int32_t *b2, cudaStream_t s)
{
    k_export_best_two<<<grid_missions(w.M_pad), 256, 0, s>>>(w, a, b, b1, b2);
    return cudaGetLastError();
}

cudaError_t kernels_init()
{
    cudaError_t e = cudaFuncSetAttribute(k_swap_eval<kSwapJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(STAGE_MAX_K * kSwapJ * 12));
    if (e != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace stg
