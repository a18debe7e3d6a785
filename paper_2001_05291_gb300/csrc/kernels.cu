// sm_103a kernels of the staging engine: cost table, ranking, evaluation and
// the Tabu loop (per-mission best/second-best, swap neighbourhood, move
// selection, incremental refresh).  Integer arithmetic throughout; the only
// floating point is a float32 first guess of each leg's square root, corrected
// to the exact integer.
#include <cuda_runtime.h>
#include <climits>
#include <cstdlib>
#include <mutex>
#include <stdint.h>

#include "stage_internal.h"
#include "device_common.cuh"

namespace stg {

// SMs per device, filled by kernels_init (once per device); launchers size
// their grids for the current device
constexpr int kMaxDevices = 64;
static int g_sms_of[kMaxDevices] = {};
static std::mutex g_init_mu;

static int sm_count()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 152;
    return g_sms_of[dev] > 0 ? g_sms_of[dev] : 152;
}
int swap_segment_for(int M_pad, int nC, int K);

// --------------------------------------------------------------------------
// helpers
// --------------------------------------------------------------------------

// Leg cost (Sec. 3; Euclidean in place of Eq. 1): the ceiling of the square
// root of the exact squared distance n.  |coord| <= 2^24 keeps n below 2^52,
// where the ceiling of the correctly rounded float64 root is exactly the
// integer ceiling square root; that integer is computed here without float64
// (GB300's float64 rate is low): a float32 estimate s from the 32-bit
// differences, the exact remainder r = n - s^2 (one 32 x 32 -> 64-bit
// product), then steps of s by one that keep r exact by additions alone
// ((s - 1)^2 = s^2 - (2s - 1), (s + 1)^2 = s^2 + (2s + 1)) to the floor root
// (0 <= r <= 2s), then s + [r != 0].  Exact whatever the estimate's error.
__device__ __forceinline__ int32_t leg_ceil(int x1, int y1, int x2, int y2)
{
    const int dx = x1 - x2, dy = y1 - y2;   // |.| <= 2^25
    const long long n = (long long)dx * dx + (long long)dy * dy;
    const float fx = (float)dx, fy = (float)dy;
    const float fn = __fmaf_rn(fx, fx, __fmul_rn(fy, fy));   // n to a few parts in 2^24
    int s = fn > 0.0f ? (int)__fmul_rn(fn, rsqrtf(fn)) : 0;   // within a few tens of units of sqrt(n)
    long long r = n - (long long)s * s;
    while (r < 0) {
        r += 2 * s - 1;
        --s;
    }
    while (r > 2 * (long long)s) {
        ++s;
        r -= 2 * s - 1;
    }
    return s + (r != 0 ? 1 : 0);
}

// Leg cost of Eq. 1 (Haversine) for points given as (latitude, longitude) in
// microdegrees, in metres on a sphere of radius STAGE_EARTH_RADIUS_M, rounded
// up; c1, c2 are the cosines of the two latitudes (computed once per point).
// The products and sums use explicit round-to-nearest operations (no fused
// multiply-add), in the order the CPU oracle uses, so that only the sine,
// cosine and arcsine implementations can differ between the two.
constexpr double kMicroDegToRad = 3.14159265358979323846 / 180.0 * 1e-6;

__device__ __forceinline__ double lat_cos(int lat)
{
    return cos(__dmul_rn((double)lat, kMicroDegToRad));
}

__device__ __forceinline__ int32_t leg_haversine(int lat1, int lon1, double c1, int lat2, int lon2, double c2)
{
    const double dp = __dmul_rn((double)(lat2 - lat1), kMicroDegToRad);
    const double dl = __dmul_rn((double)(lon2 - lon1), kMicroDegToRad);
    const double sp = sin(__dmul_rn(0.5, dp)), sl = sin(__dmul_rn(0.5, dl));
    double h = __dadd_rn(__dmul_rn(sp, sp), __dmul_rn(__dmul_rn(c1, c2), __dmul_rn(sl, sl)));
    h = fmin(h, 1.0);
    const double d = __dmul_rn(2.0 * STAGE_EARTH_RADIUS_M, asin(sqrt(h)));
    return (int32_t)ceil(d);
}

// Leg by metric: 0 = Euclidean on integer metres, 1 = Haversine.
template <int Metric>
__device__ __forceinline__ int32_t leg_of(int2 u, double cu, int2 v, double cv)
{
    if (Metric == 0) return leg_ceil(u.x, u.y, v.x, v.y);
    return leg_haversine(u.x, u.y, cu, v.x, v.y, cv);
}

template <int Metric>
__device__ __forceinline__ double point_cos(int2 u)
{
    return Metric == 0 ? 0.0 : lat_cos(u.x);
}








// --------------------------------------------------------------------------
// Mission order.  The table's columns are laid out in Morton order of the
// missions' pickup/drop-off midpoints, so neighbouring columns hold missions
// with similar cost rows: the rare "closer than the second-best" hits of the
// swap pass bunch into few warps, and refresh rescans bunch into few blocks.
// Every quantity the engine returns is an integer sum over missions, so the
// column order changes no result.  The order is a stable LSD radix sort of a
// 16-bit key (two 8-bit digits), ties kept in mission-index order.
// --------------------------------------------------------------------------

__global__ void k_mid_bbox(int M, const int2 *__restrict__ pick, const int2 *__restrict__ drop,
                           int *__restrict__ bbox /* minx, miny, maxx, maxy */)
{
    int mnx = INT_MAX, mny = INT_MAX, mxx = INT_MIN, mxy = INT_MIN;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        const int2 p = pick[m], d = drop[m];
        const int x = (p.x + d.x) >> 1, y = (p.y + d.y) >> 1;   // |sum| < 2^29 (metres or microdegrees)
        mnx = min(mnx, x); mny = min(mny, y); mxx = max(mxx, x); mxy = max(mxy, y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mnx = min(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mny = min(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mxx = max(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mxy = max(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&bbox[0], mnx); atomicMin(&bbox[1], mny);
        atomicMax(&bbox[2], mxx); atomicMax(&bbox[3], mxy);
    }
}

__device__ __forceinline__ unsigned spread8(unsigned v)
{
    v &= 0xffu;
    v = (v | (v << 4)) & 0x0f0fu;
    v = (v | (v << 2)) & 0x3333u;
    v = (v | (v << 1)) & 0x5555u;
    return v;
}

__global__ void k_morton_keys(int M, const int2 *__restrict__ pick, const int2 *__restrict__ drop,
                              const int *__restrict__ bbox, unsigned *__restrict__ key,
                              int *__restrict__ val)
{
    const long long x0 = bbox[0], y0 = bbox[1];
    const long long wx = (long long)bbox[2] - x0 + 1, wy = (long long)bbox[3] - y0 + 1;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        const int2 p = pick[m], d = drop[m];
        const long long x = (p.x + d.x) >> 1, y = (p.y + d.y) >> 1;
        const unsigned qx = (unsigned)(((x - x0) << 8) / wx), qy = (unsigned)(((y - y0) << 8) / wy);
        key[m] = spread8(qx) | (spread8(qy) << 1);
        val[m] = m;
    }
}

constexpr int kSortThreads = 256;
constexpr int kSortTile = kSortThreads * 16;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(int n, const unsigned *__restrict__ key,
                                                             int shift, int nBlocks, int *__restrict__ counts)
{
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int t0 = blockIdx.x * kSortTile;
    for (int e = t0 + threadIdx.x; e < min(n, t0 + kSortTile); e += kSortThreads)
        atomicAdd(&h[(key[e] >> shift) & 255u], 1);
    __syncthreads();
    counts[threadIdx.x * nBlocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of `n` ints in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_exclusive(int n, int *__restrict__ v)
{
    __shared__ int part[1024];
    const int per = (n + 1023) / 1024;
    const int b = threadIdx.x * per, e = min(n, b + per);
    int s = 0;
    for (int k = b; k < e; k++) s += v[k];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int add = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    int run = part[threadIdx.x] - s;
    for (int k = b; k < e; k++) {
        const int x = v[k];
        v[k] = run;
        run += x;
    }
}

// Stable scatter: rounds of 256 elements in index order; within a round, lower
// warps first and lower lanes first.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(int n, const unsigned *__restrict__ key_in,
                                                                const int *__restrict__ val_in, int shift,
                                                                int nBlocks, const int *__restrict__ offsets,
                                                                unsigned *__restrict__ key_out,
                                                                int *__restrict__ val_out)
{
    constexpr int W = kSortThreads / 32;
    __shared__ int s_base[256], s_run[256];
    __shared__ int s_wc[W][257];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    s_base[threadIdx.x] = offsets[threadIdx.x * nBlocks + blockIdx.x];
    s_run[threadIdx.x] = 0;
    for (int w = 0; w < W; w++) s_wc[w][threadIdx.x] = 0;
    __syncthreads();
    const int t0 = blockIdx.x * kSortTile;
    for (int r = 0; r < kSortTile / kSortThreads; r++) {
        const int e = t0 + r * kSortThreads + threadIdx.x;
        const bool ok = e < n;
        const unsigned k = ok ? key_in[e] : 0u;
        const int d = ok ? (int)((k >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (ok && rank == 0) s_wc[wid][d] = __popc(peers);
        __syncthreads();
        if (ok) {
            int prior = 0;
            for (int w = 0; w < wid; w++) prior += s_wc[w][d];
            const int pos = s_base[d] + s_run[d] + prior + rank;
            key_out[pos] = k;
            val_out[pos] = val_in[e];
        }
        __syncthreads();
        int tot = 0;
        for (int w = 0; w < W; w++) { tot += s_wc[w][threadIdx.x]; s_wc[w][threadIdx.x] = 0; }
        s_run[threadIdx.x] += tot;
        __syncthreads();
    }
}

__global__ void k_apply_order(int M, const int *__restrict__ perm, const int2 *__restrict__ pick,
                              const int2 *__restrict__ drop, int2 *__restrict__ pick_s,
                              int2 *__restrict__ drop_s, int *__restrict__ inv)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < M; q += gridDim.x * blockDim.x) {
        const int m = perm[q];
        pick_s[q] = pick[m];
        drop_s[q] = drop[m];
        inv[m] = q;
    }
}

size_t order_scratch_bytes(int M)
{
    const size_t nB = (size_t)(M + kSortTile - 1) / kSortTile;
    return 4 * ((size_t)M * 4 + 256) + 256 * nB * 4 + 512;
}

cudaError_t launch_order(int M, const int2 *pick, const int2 *drop, void *scratch, int *perm,
                         int *inv, int2 *pick_s, int2 *drop_s, cudaStream_t s)
{
    const int nB = (M + kSortTile - 1) / kSortTile;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char *p = static_cast<char *>(scratch);
    int *bbox = reinterpret_cast<int *>(p);                 p += 256;
    unsigned *k0 = reinterpret_cast<unsigned *>(p);         p += al((size_t)M * 4);
    unsigned *k1 = reinterpret_cast<unsigned *>(p);         p += al((size_t)M * 4);
    int *v0 = reinterpret_cast<int *>(p);                   p += al((size_t)M * 4);
    int *v1 = perm;                                          // second pass lands in perm
    int *counts = reinterpret_cast<int *>(p);
    const int init[4] = {INT_MAX, INT_MAX, INT_MIN, INT_MIN};
    cudaError_t e = cudaMemcpyAsync(bbox, init, sizeof init, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    int g = (M + 255) / 256;
    if (g > 1024) g = 1024;
    k_mid_bbox<<<g, 256, 0, s>>>(M, pick, drop, bbox);
    k_morton_keys<<<g, 256, 0, s>>>(M, pick, drop, bbox, k0, v0);
    // pass 1: low digit  (k0, v0) -> (k1, perm as temporary values)
    k_radix_hist<<<nB, kSortThreads, 0, s>>>(M, k0, 0, nB, counts);
    k_scan_exclusive<<<1, 1024, 0, s>>>(256 * nB, counts);
    k_radix_scatter<<<nB, kSortThreads, 0, s>>>(M, k0, v0, 0, nB, counts, k1, v1);
    // pass 2: high digit (k1, perm) -> (k0, v0); then v0 is the order
    k_radix_hist<<<nB, kSortThreads, 0, s>>>(M, k1, 8, nB, counts);
    k_scan_exclusive<<<1, 1024, 0, s>>>(256 * nB, counts);
    k_radix_scatter<<<nB, kSortThreads, 0, s>>>(M, k1, v1, 8, nB, counts, k0, v0);
    e = cudaMemcpyAsync(perm, v0, (size_t)M * 4, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    k_apply_order<<<g, 256, 0, s>>>(M, perm, pick, drop, pick_s, drop_s, inv);
    return cudaGetLastError();
}

// Table window in the caller's mission order: out[r][q] = cost[b0 + r][inv[m0 + q]].
__global__ void k_gather_window(const int32_t *__restrict__ cost, int M, int M_pad, const int *__restrict__ inv,
                                int b0, int nb, int m0, int nm, int32_t *__restrict__ out)
{
    const size_t n = (size_t)nb * nm;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(q / nm), c = (int)(q % nm);
        const int m = m0 + c;
        const int col = m < M ? inv[m] : m;    // pads keep their position; removed ids have none
        out[q] = col >= 0 ? cost[(size_t)(b0 + r) * M_pad + col] : kInf;
    }
}

cudaError_t launch_gather_window(const int32_t *cost, int M, int M_pad, const int *inv, int b0, int nb,
                                 int m0, int nm, int32_t *out, cudaStream_t s)
{
    size_t n = (size_t)nb * nm;
    size_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    if (g == 0) return cudaSuccess;
    k_gather_window<<<(int)g, 256, 0, s>>>(cost, M, M_pad, inv, b0, nb, m0, nm, out);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// a1: cost table.  c[b][m] = leg(b, p_m) + leg(p_m, d_m) + leg(d_m, b).
// --------------------------------------------------------------------------

template <int Metric>
__global__ void k_pickup_drop_leg(int M, const int2 *__restrict__ pick,
                                  const int2 *__restrict__ drop, int32_t *__restrict__ pd)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        const int2 p = pick[m], d = drop[m];
        pd[m] = leg_of<Metric>(p, point_cos<Metric>(p), d, point_cos<Metric>(d));
    }
}

constexpr int kTableBasesPerBlock = 8;

// Each thread owns 4 consecutive missions and writes them for 8 bases (one
// 16-byte store per base row); pads (m >= M) hold INT32_MAX.
template <int Metric>
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
        double cp[4], cd[4];
        int l[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            if (m + e < M) { p[e] = pick[m + e]; d[e] = drop[m + e]; l[e] = pd[m + e]; }
            else { p[e] = make_int2(0, 0); d[e] = make_int2(0, 0); l[e] = -1; }
            cp[e] = point_cos<Metric>(p[e]);
            cd[e] = point_cos<Metric>(d[e]);
        }
#pragma unroll 1
        for (int bb = 0; bb < kTableBasesPerBlock; bb++) {
            const int b = b0 + bb;
            if (b >= B) break;
            const int2 o = base[b];
            const double co = point_cos<Metric>(o);
            int v[4];
#pragma unroll
            for (int e = 0; e < 4; e++)
                v[e] = (l[e] >= 0) ? leg_of<Metric>(o, co, p[e], cp[e]) + l[e] + leg_of<Metric>(d[e], cd[e], o, co)
                                   : kInf;
            reinterpret_cast<int4 *>(cost + (size_t)b * M_pad)[q] = make_int4(v[0], v[1], v[2], v[3]);
        }
    }
}

// Input check (device-resident inputs): flag an interleaved (x, y) value
// outside [-lim_x, lim_x] x [-lim_y, lim_y].
__global__ void k_check_coords(const int32_t *__restrict__ v, size_t n, int lim_x, int lim_y,
                               int *__restrict__ bad)
{
    int found = 0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int x = v[k], lim = (k & 1) ? lim_y : lim_x;
        found |= (x > lim) | (x < -lim);
    }
    if (__syncthreads_or(found) && threadIdx.x == 0) atomicOr(bad, 1);
}

cudaError_t launch_check_coords(const int32_t *v, size_t n, int lim_x, int lim_y, int *bad, cudaStream_t s)
{
    size_t g = (n + 255) / 256;
    if (g > 1024) g = 1024;
    if (g == 0) return cudaSuccess;
    k_check_coords<<<(int)g, 256, 0, s>>>(v, n, lim_x, lim_y, bad);
    return cudaGetLastError();
}

// Instance updates: appended columns, removed columns, fills.
__global__ void k_fill_i32(int32_t *__restrict__ p, size_t n, int32_t v)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) p[q] = v;
}

cudaError_t launch_fill_i32(int32_t *p, size_t n, int32_t v, cudaStream_t s)
{
    size_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    if (g == 0) return cudaSuccess;
    k_fill_i32<<<(int)g, 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

// Costs of columns [col0, col0 + n) for every base (missions appended at the end).
template <int Metric>
__global__ void k_table_columns(int B, int col0, int n, int M_pad, const int2 *__restrict__ base,
                                const int2 *__restrict__ pick, const int2 *__restrict__ drop,
                                int32_t *__restrict__ pd, int32_t *__restrict__ cost)
{
    const size_t total = (size_t)B * n;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(q / n), col = col0 + (int)(q % n);
        const int2 p = pick[col], d = drop[col], o = base[b];
        const double cp = point_cos<Metric>(p), cd = point_cos<Metric>(d), co = point_cos<Metric>(o);
        const int l = leg_of<Metric>(p, cp, d, cd);
        if (b == 0) pd[col] = l;
        cost[(size_t)b * M_pad + col] = leg_of<Metric>(o, co, p, cp) + l + leg_of<Metric>(d, cd, o, co);
    }
}

cudaError_t launch_table_columns(int B, int col0, int n, int M_pad, const int2 *base, const int2 *pick,
                                 const int2 *drop, int32_t *pd, int32_t *cost, int metric, cudaStream_t s)
{
    size_t total = (size_t)B * n;
    size_t g = (total + 255) / 256;
    if (g > 8192) g = 8192;
    if (g == 0) return cudaSuccess;
    if (metric == 1)
        k_table_columns<1><<<(int)g, 256, 0, s>>>(B, col0, n, M_pad, base, pick, drop, pd, cost);
    else
        k_table_columns<0><<<(int)g, 256, 0, s>>>(B, col0, n, M_pad, base, pick, drop, pd, cost);
    return cudaGetLastError();
}

// Removed missions: their columns become INT32_MAX (one block per id).
__global__ void k_tombstone(const int32_t *__restrict__ ids, int n, int32_t *__restrict__ inv,
                            int32_t *__restrict__ perm, int32_t *__restrict__ cost, int B, int M_pad)
{
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int col = inv[ids[k]];
        __syncthreads();
        if (col < 0) continue;
        for (int b = threadIdx.x; b < B; b += blockDim.x) cost[(size_t)b * M_pad + col] = kInf;
        __syncthreads();
        if (threadIdx.x == 0) {
            inv[ids[k]] = -1;
            perm[col] = -1;
        }
    }
}

cudaError_t launch_tombstone(const int32_t *ids, int n, int32_t *inv, int32_t *perm, int32_t *cost, int B,
                             int M_pad, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_tombstone<<<n < 1024 ? n : 1024, 256, 0, s>>>(ids, n, inv, perm, cost, B, M_pad);
    return cudaGetLastError();
}

cudaError_t launch_table(int B, int M, int M_pad, const int2 *base, const int2 *pick,
                         const int2 *drop, int32_t *pd, int32_t *cost, int metric, cudaStream_t s)
{
    int g1 = (M + 255) / 256;
    if (g1 > 4096) g1 = 4096;
    int n4 = M_pad / 4;
    int gx = (n4 + 255) / 256;
    int gy = (B + kTableBasesPerBlock - 1) / kTableBasesPerBlock;
    // enough blocks for every SM even when B is small
    if (gx > 1024) gx = 1024;
    if (metric == 1) {
        k_pickup_drop_leg<1><<<g1, 256, 0, s>>>(M, pick, drop, pd);
        k_build_table<1><<<dim3(gx, gy), 256, 0, s>>>(B, M, M_pad, base, pick, drop, pd, cost);
    } else {
        k_pickup_drop_leg<0><<<g1, 256, 0, s>>>(M, pick, drop, pd);
        k_build_table<0><<<dim3(gx, gy), 256, 0, s>>>(B, M, M_pad, base, pick, drop, pd, cost);
    }
    return cudaGetLastError();
}

// The table, its row sums, its mission-major copy and the copy's cell minima
// in one pass (no second read of the table).  A block covers 8 cells of the
// copy (256 positions, base border[p] at position p) and walks tiles of 32
// missions: warp w computes cell 8 g + w of the tile, lane = mission, writes
// each base's 32 costs of the tile to the table (128 bytes per base row),
// transposes them through its own shared tile and writes each mission's 32
// costs of the cell to the copy (128 bytes), the lane of position p adding
// its base's costs to the row sum and the warp taking each mission's minimum
// over the cell.  Pads (m >= M) and positions past B hold INT32_MAX and add
// nothing to a row sum.
constexpr int kFusedCells = 8;

template <int Metric>
__global__ void __launch_bounds__(256) k_build_table_fused(int B, int M, int M_pad, int ldT,
                                                           const int2 *__restrict__ base,
                                                           const int2 *__restrict__ pick,
                                                           const int2 *__restrict__ drop,
                                                           const int32_t *__restrict__ pd,
                                                           const int32_t *__restrict__ border,
                                                           int32_t *__restrict__ cost, int32_t *__restrict__ costT,
                                                           int32_t *__restrict__ cellmin,
                                                           unsigned long long *__restrict__ S)
{
    __shared__ int32_t tile[kFusedCells][32][33];
    __shared__ int32_t smin[2][32][kFusedCells];
    __shared__ int2 sxy[kFusedCells * 32];
    __shared__ double scos[kFusedCells * 32];
    __shared__ int32_t sid[kFusedCells * 32];
    const int nCell = ldT >> 5, ldC = cell_ld(ldT);
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int cell = blockIdx.y * kFusedCells + wq;
    const int p0 = blockIdx.y * kFusedCells * 32;
    {
        const int p = p0 + threadIdx.x;
        const int b = p < ldT ? border[p] : -1;
        sid[threadIdx.x] = b;
        sxy[threadIdx.x] = b >= 0 ? base[b] : make_int2(0, 0);
        scos[threadIdx.x] = b >= 0 ? point_cos<Metric>(base[b]) : 0.0;
    }
    __syncthreads();
    const bool live = cell < nCell;   // the same on the warp
    const int mb = sid[wq * 32 + lane];   // the base of this lane's position (transposed phase)
    long long rs = 0;
    const int nTiles = M_pad >> 5;
    int buf = 0;
    for (int t = blockIdx.x; t < nTiles; t += gridDim.x) {   // the same on the block
        const int m = t * 32 + lane;
        if (live) {
            int2 pm = make_int2(0, 0), dm = make_int2(0, 0);
            int l = -1;
            if (m < M) { pm = pick[m]; dm = drop[m]; l = pd[m]; }
            const double cpm = point_cos<Metric>(pm), cdm = point_cos<Metric>(dm);
#pragma unroll 4
            for (int k = 0; k < 32; k++) {
                const int q = wq * 32 + k;
                const int b = sid[q];
                int32_t v = kInf;
                if (b >= 0 && l >= 0) {
                    const int2 o = sxy[q];
                    const double co = scos[q];
                    v = leg_of<Metric>(o, co, pm, cpm) + l + leg_of<Metric>(dm, cdm, o, co);
                }
                if (b >= 0) cost[(size_t)b * M_pad + m] = v;
                tile[wq][k][lane] = v;
            }
            __syncwarp();
            int32_t mymin = kInf;
#pragma unroll 4
            for (int mm = 0; mm < 32; mm++) {
                const int32_t v = tile[wq][lane][mm];   // position lane, mission mm
                costT[(size_t)(t * 32 + mm) * ldT + cell * 32 + lane] = v;
                if (mb >= 0 && v != kInf) rs += v;
                const int32_t mn = __reduce_min_sync(0xffffffffu, v);
                if (lane == mm) mymin = mn;
            }
            smin[buf][lane][wq] = mymin;
            __syncwarp();
        }
        __syncthreads();
        {   // the tile's cell minima: 32 missions x 8 cells, 32 bytes per mission
            const int mm = threadIdx.x >> 3, c = threadIdx.x & 7;
            if (blockIdx.y * kFusedCells + c < nCell)
                cellmin[(size_t)(t * 32 + mm) * ldC + blockIdx.y * kFusedCells + c] = smin[buf][mm][c];
        }
        buf ^= 1;
    }
    if (live && mb >= 0 && rs) atomicAdd(&S[mb], (unsigned long long)rs);
}

cudaError_t launch_table_fused(int B, int M, int M_pad, int ldT, const int2 *base, const int2 *pick,
                               const int2 *drop, int32_t *pd, const int32_t *border, int32_t *cost, int32_t *costT,
                               int32_t *cellmin, unsigned long long *S, int metric, cudaStream_t s)
{
    const int sms = sm_count();
    int g1 = (M + 255) / 256;
    if (g1 > 4096) g1 = 4096;
    const int gy = (ldT / 32 + kFusedCells - 1) / kFusedCells;
    // one wave of as many resident blocks as the SMs hold (each block walks an
    // equal share of the mission tiles)
    int per_sm = 0;
    if ((metric == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_table_fused<1>, 256, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_table_fused<0>, 256, 0)) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 4;
    int gx = (sms * per_sm + gy - 1) / gy;
    if (gx > M_pad / 32) gx = M_pad / 32;
    if (gx < 1) gx = 1;
    if (metric == 1) {
        k_pickup_drop_leg<1><<<g1, 256, 0, s>>>(M, pick, drop, pd);
        k_build_table_fused<1><<<dim3(gx, gy), 256, 0, s>>>(B, M, M_pad, ldT, base, pick, drop, pd, border, cost,
                                                             costT, cellmin, S);
    } else {
        k_pickup_drop_leg<0><<<g1, 256, 0, s>>>(M, pick, drop, pd);
        k_build_table_fused<0><<<dim3(gx, gy), 256, 0, s>>>(B, M, M_pad, ldT, base, pick, drop, pd, border, cost,
                                                             costT, cellmin, S);
    }
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
        // columns >= M are pads; INT32_MAX inside [0, M) marks a removed mission
        acc += (m + 0 < M && v.x != kInf ? (long long)v.x : 0) + (m + 1 < M && v.y != kInf ? (long long)v.y : 0) +
               (m + 2 < M && v.z != kInf ? (long long)v.z : 0) + (m + 3 < M && v.w != kInf ? (long long)v.w : 0);
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
// rank < K are written in rank order.  Block `blk` ranks bases blk*256 ...
__device__ __forceinline__ void topk_body(const unsigned long long *__restrict__ S,
                                          const uint8_t *__restrict__ avail, int B, int K,
                                          int32_t *__restrict__ open, int blk)
{
    __shared__ long long sS[1024];
    __shared__ uint8_t sA[1024];
    const int b = blk * blockDim.x + threadIdx.x;
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

__global__ void __launch_bounds__(256) k_topk(const unsigned long long *__restrict__ S,
                                              const uint8_t *__restrict__ avail, int B, int K,
                                              int32_t *__restrict__ open)
{
    topk_body(S, avail, B, K, open, blockIdx.x);
}

// Many rankings in one launch: map[b] = (ranking, block within it).
__global__ void __launch_bounds__(256) k_topk_group(const TopkSlot *__restrict__ slots,
                                                    const int2 *__restrict__ map)
{
    const int2 e = map[blockIdx.x];
    const TopkSlot g = slots[e.x];
    topk_body(g.S, g.avail, g.B, g.K, g.open, e.y);
}

int topk_blocks(int B)
{
    return (B + 255) / 256;
}

cudaError_t launch_topk_group(const TopkSlot *slots, const int2 *map, int total_blocks, cudaStream_t s)
{
    if (total_blocks <= 0) return cudaSuccess;
    k_topk_group<<<total_blocks, 256, 0, s>>>(slots, map);
    return cudaGetLastError();
}

cudaError_t launch_topk(const unsigned long long *S, const uint8_t *avail, int B, int K,
                        int32_t *open, cudaStream_t s)
{
    k_topk<<<topk_blocks(B), 256, 0, s>>>(S, avail, B, K, open);
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


// Body shared by the single-instance and the grouped launch: block `bid` of
// `nb` blocks working on one instance.
__device__ __forceinline__ void init_body(const TabuBuffers &w, const int32_t *__restrict__ cost, int bid, int nb)
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
    for (int m = bid * blockDim.x + threadIdx.x; m < w.M_pad; m += nb * blockDim.x) {
        if (m >= w.M) {
            w.a[m] = kInf; w.b[m] = kInf; w.s1[m] = 0; w.s2[m] = -1;
            continue;
        }
        if (w.mask && !w.mask[m]) {   // not a mission of this search: never a hit, no term
            w.a[m] = INT_MIN; w.b[m] = INT_MIN; w.s1[m] = 0; w.s2[m] = -1;
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

__global__ void __launch_bounds__(256) k_init(TabuBuffers w, const int32_t *__restrict__ cost)
{
    init_body(w, cost, blockIdx.x, gridDim.x);
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
    if (!ignore_done && (w.st->done || w.st->ls_hold)) return;
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

// --------------------------------------------------------------------------
// a4, direct form: non-persistent grid (the block scheduler balances dense and
// sparse regions), 16 candidate rows per block, one thread per 4 consecutive
// missions, 4 independent 16-byte table loads in flight per thread and 4
// blocks (32 warps) per SM: the hit path's latency is hidden by other warps,
// not by deeper per-thread batches.  Same clamped thresholds and
// warp-aggregated accumulation as the streaming form.
// --------------------------------------------------------------------------
constexpr int kDirJ = 16;      // candidate rows per block (at most; fewer when the grid is small)
constexpr int kStages = 2;     // batches of 4 rows in flight per thread

constexpr int kDirThreads = 256;
// Dynamic shared memory of the direct swap pass: [K][J] accumulators, then the
// per-thread staging slots.
size_t swap_direct_smem(int K)
{
    return (size_t)K * kDirJ * 12 + 16 + (size_t)kStages * 4 * kDirThreads * 16;
}

// Hit path of one row for one warp: called (out of line, so the kernel body
// stays small enough for the instruction cache) only when some lane of the
// warp has a hit in the row; every lane of the warp takes part.
template <int J>
__device__ __noinline__ void dir_row(const int4 x, const int4 ap, const int4 bp, const int s0, const int s1,
                                     const int s2, const int s3, const bool uni, const int r, const int R,
                                     int *ex_c, unsigned long long *ex_d, int *g_c, unsigned long long *g_d,
                                     const int lane)
{
    int ec = 0, gc = 0;
    long long ed = 0, gd = 0;
    if (x.x < bp.x || x.y < bp.y || x.z < bp.z || x.w < bp.w) {
        const int xv[4] = {x.x, x.y, x.z, x.w}, av[4] = {ap.x, ap.y, ap.z, ap.w},
                  bv[4] = {bp.x, bp.y, bp.z, bp.w}, sv[4] = {s0, s1, s2, s3};
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int xe = xv[e], a = av[e], b = bv[e];
            if (xe < b) {
                const int ca = a <= R, cb = b <= R;
                const int dc = ca - cb;
                const long long dd = (ca ? (long long)max(xe, a) : 0ll) - (cb ? (long long)b : 0ll);
                if (uni) {
                    ec += dc;
                    ed += dd;
                } else if (dc | (dd != 0)) {
                    atomicAdd(&ex_c[sv[e] * J + r], dc);
                    atomicAdd(&ex_d[sv[e] * J + r], (unsigned long long)dd);
                }
                if (xe < a) {
                    gc += 1 - ca;
                    gd += (long long)xe - (ca ? (long long)a : 0ll);
                }
            }
        }
    }
    if (uni && (ec | (ed != 0))) {
        const unsigned am = __activemask();
        const unsigned peers = __match_any_sync(am, s0);
        const int sc = (int)__reduce_add_sync(peers, (unsigned)ec);
        const long long sd = group_sum_small(peers, ed);
        if (lane == __ffs(peers) - 1 && (sc | (sd != 0))) {
            atomicAdd(&ex_c[s0 * J + r], sc);
            atomicAdd(&ex_d[s0 * J + r], (unsigned long long)sd);
        }
    }
    if (__any_sync(0xffffffffu, gc | (gd != 0))) {
        const int sc = (int)__reduce_add_sync(0xffffffffu, (unsigned)gc);
        const long long sd = group_sum_small(0xffffffffu, gd);
        if (lane == 0 && (sc | (sd != 0))) {
            atomicAdd(&g_c[r], sc);
            atomicAdd(&g_d[r], (unsigned long long)sd);
        }
    }
}

template <int J>
__device__ __forceinline__ void swap_direct_body(const TabuBuffers &w, const int32_t *__restrict__ cost,
                                                 int bx, int by, int seg)
{
    extern __shared__ unsigned long long sm_dir[];
    const int K = w.K;
    unsigned long long *ex_d = sm_dir;                               // [K * J]
    int *ex_c = reinterpret_cast<int *>(ex_d + K * J);           // [K * J]
    __shared__ int rows[J];
    __shared__ int g_c[J];
    __shared__ unsigned long long g_d[J];
    const int nC = w.st->nC;
    const int c0 = by * J;
    for (int k = threadIdx.x; k < K * J; k += blockDim.x) { ex_d[k] = 0; ex_c[k] = 0; }
    if (threadIdx.x < J) {
        rows[threadIdx.x] = (c0 + threadIdx.x < nC) ? w.cand[c0 + threadIdx.x] : -1;
        g_c[threadIdx.x] = 0;
        g_d[threadIdx.x] = 0;
    }
    __syncthreads();
    const int R = w.R, lane = threadIdx.x & 31;
    const size_t M_pad = w.M_pad;
    const int nrows = min(J, nC - c0);
    const int m_begin = bx * seg;
    const int m_end = min(m_begin + seg, w.M_pad);
    // Table loads are staged through shared memory with per-thread async
    // copies (cp.async, L2 only), kStages batches of 4 rows ahead, so they keep
    // streaming while the warp works on hits.  Each thread reads back only the
    // slots it copied into, after waiting on its own copy groups.  Every lane of
    // a warp runs every batch (the warp-collective calls in dir_row need all 32
    // lanes); lanes past the segment end see thresholds nothing can beat.
    int4 *stg = reinterpret_cast<int4 *>(ex_c + K * J + ((K * J) & 3 ? 4 - ((K * J) & 3) : 0));
    const int wbase = 4 * (threadIdx.x & ~31);
    const int first = m_begin + wbase;
    const int npass = first < m_end ? (m_end - first + 4 * kDirThreads - 1) / (4 * kDirThreads) : 0;
    const int nbatch = npass * (J / 4);
    // the table streams through once per iteration: evict it first from L2, so
    // the per-mission thresholds (re-read by every row chunk) stay resident
    const unsigned long long policy = evict_first_policy();
    auto issue = [&](int i) {
        const int p = i / (J / 4), h = (i % (J / 4)) * 4;
        const int m = first + p * 4 * kDirThreads + 4 * lane;
        if (m < m_end) {
            const int q = m >> 2;
#pragma unroll
            for (int r = 0; r < 4; r++)
                if (h + r < nrows) {
                    const int4 *src = reinterpret_cast<const int4 *>(cost + (size_t)rows[h + r] * M_pad) + q;
                    const unsigned dst = (unsigned)__cvta_generic_to_shared(&stg[((i % kStages) * 4 + r) * kDirThreads + threadIdx.x]);
                    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                                 "l"(policy)
                                 : "memory");
                }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
#pragma unroll 1
    for (int i = 0; i < kStages - 1; i++) {
        if (i < nbatch) issue(i);
        else asm volatile("cp.async.commit_group;" ::: "memory");
    }
    int4 ap = make_int4(0, 0, 0, 0), bp = make_int4(INT_MIN, INT_MIN, INT_MIN, INT_MIN);
    int s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    bool uni = false, act = false;
#pragma unroll 1
    for (int b = 0; b < nbatch; b++) {
        if (b + kStages - 1 < nbatch) issue(b + kStages - 1);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        const int hb = b % (J / 4), h = hb * 4;
        if (hb == 0) {
            const int m = first + (b / (J / 4)) * 4 * kDirThreads + 4 * lane;
            act = m < m_end;
            const int q = act ? (m >> 2) : 0;
            ap = __ldg(reinterpret_cast<const int4 *>(w.a) + q);
            bp = __ldg(reinterpret_cast<const int4 *>(w.b) + q);
            const uint2 sp = __ldg(reinterpret_cast<const uint2 *>(w.s1) + q);
            ap.x = min(ap.x, R + 1); ap.y = min(ap.y, R + 1); ap.z = min(ap.z, R + 1); ap.w = min(ap.w, R + 1);
            bp.x = min(bp.x, R + 1); bp.y = min(bp.y, R + 1); bp.z = min(bp.z, R + 1); bp.w = min(bp.w, R + 1);
            if (!act) bp = make_int4(INT_MIN, INT_MIN, INT_MIN, INT_MIN);
            s0 = (int)(int16_t)(sp.x & 0xffff); s1 = (int)(int16_t)(sp.x >> 16);
            s2 = (int)(int16_t)(sp.y & 0xffff); s3 = (int)(int16_t)(sp.y >> 16);
            uni = (s0 == s1) && (s1 == s2) && (s2 == s3);
        }
        asm volatile("cp.async.wait_group %0;" ::"n"(kStages - 1) : "memory");
        int4 x[4];
#pragma unroll
        for (int r = 0; r < 4; r++)
            x[r] = (act && h + r < nrows) ? stg[((b % kStages) * 4 + r) * kDirThreads + threadIdx.x]
                                          : make_int4(INT_MAX, INT_MAX, INT_MAX, INT_MAX);
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const bool hit = x[r].x < bp.x || x[r].y < bp.y || x[r].z < bp.z || x[r].w < bp.w;
            if (__any_sync(0xffffffffu, hit))
                dir_row<J>(x[r], ap, bp, s0, s1, s2, s3, uni, h + r, R, ex_c, ex_d, g_c, g_d, lane);
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    for (int k = threadIdx.x; k < K * J; k += blockDim.x) {
        const int r = k % J, sidx = k / J;
        const int j = rows[r];
        if (j < 0) continue;
        const int c = ex_c[k];
        const unsigned long long d = ex_d[k];
        if (c | (d != 0)) {
            atomicAdd(&w.extra_c[(size_t)sidx * w.B + j], c);
            atomicAdd(&w.extra_d[(size_t)sidx * w.B + j], d);
        }
    }
    if (threadIdx.x < J && rows[threadIdx.x] >= 0) {
        const int j = rows[threadIdx.x];
        if (g_c[threadIdx.x]) atomicAdd(&w.gain_c[j], g_c[threadIdx.x]);
        if (g_d[threadIdx.x]) atomicAdd(&w.gain_d[j], g_d[threadIdx.x]);
    }
}

template <int J>
__global__ void __launch_bounds__(kDirThreads, 4)
k_swap_direct(TabuBuffers w, const int32_t *__restrict__ cost, int ignore_done, int seg)
{
    if (!ignore_done && (w.st->done || w.st->ls_hold)) return;
    swap_direct_body<J>(w, cost, blockIdx.x, blockIdx.y, seg);
}

// Missions per block of the direct swap pass: the largest power of two in
// [1024, 16384] that still gives at least two waves of blocks (4 per SM), so
// mid-size instances fill the GPU and large ones keep the per-block flush
// rare.  A measured choice (stage_autotune) overrides it per shape bucket.
int swap_segment_heuristic(int M_pad, int nC)
{
    const int chunks = (nC + kDirJ - 1) / kDirJ;   // judged at the default 16 rows per block
    const long long target = 2ll * 4 * sm_count();
    int seg = 16384;
    while (seg > 1024 && (long long)((M_pad + seg - 1) / seg) * chunks < target) seg >>= 1;
    return seg;
}

// Tile cache: missions per block chosen by measurement, per shape bucket
// (ceil log2 of padded missions, of candidate rows, and of K).  0 = unset.
static int g_seg_cache[26][18][12];

static inline int ilog2_ceil(long long v)
{
    int r = 0;
    while ((1ll << r) < v) r++;
    return r;
}

int swap_segment_for(int M_pad, int nC, int K)
{
    const int a = min(25, ilog2_ceil(M_pad)), b = min(17, ilog2_ceil(nC > 0 ? nC : 1)), c = min(11, ilog2_ceil(K));
    const int v = g_seg_cache[a][b][c];
    return v ? v : swap_segment_heuristic(M_pad, nC);
}

void swap_segment_record(int M_pad, int nC, int K, int seg)
{
    const int a = min(25, ilog2_ceil(M_pad)), b = min(17, ilog2_ceil(nC > 0 ? nC : 1)), c = min(11, ilog2_ceil(K));
    g_seg_cache[a][b][c] = seg;
}

bool swap_segment_known(int M_pad, int nC, int K)
{
    const int a = min(25, ilog2_ceil(M_pad)), b = min(17, ilog2_ceil(nC > 0 ? nC : 1)), c = min(11, ilog2_ceil(K));
    return g_seg_cache[a][b][c] != 0;
}

// Launch the direct swap pass with an explicit segment (autotuning).
cudaError_t launch_swap_direct_seg(const TabuBuffers &w, const int32_t *cost, int nC, int seg, cudaStream_t s)
{
    if (nC <= 0) return cudaSuccess;
    dim3 grid((w.M_pad + seg - 1) / seg, (nC + kDirJ - 1) / kDirJ);
    k_swap_direct<kDirJ><<<grid, kDirThreads, swap_direct_smem(w.K), s>>>(w, cost, 1, seg);
    return cudaGetLastError();
}

cudaError_t launch_swap_eval(const TabuBuffers &w, const int32_t *cost, int nC, int ignore_done,
                             cudaStream_t s)
{
    if (nC <= 0) return cudaSuccess;
    if (w.K <= kPipeMaxK) {
        const int seg = swap_segment_for(w.M_pad, nC, w.K);
        const int bx = (w.M_pad + seg - 1) / seg;
        // latency-bound small grids: fewer rows per block, more blocks and
        // shorter per-warp chains, until the grid reaches two waves
        const long long waves2 = 2ll * 4 * sm_count();
        const size_t sm = swap_direct_smem(w.K);
        if ((long long)bx * ((nC + 15) / 16) >= waves2) {
            k_swap_direct<16><<<dim3(bx, (nC + 15) / 16), kDirThreads, sm, s>>>(w, cost, ignore_done, seg);
        } else if ((long long)bx * ((nC + 7) / 8) >= waves2) {
            k_swap_direct<8><<<dim3(bx, (nC + 7) / 8), kDirThreads, sm, s>>>(w, cost, ignore_done, seg);
        } else {
            k_swap_direct<4><<<dim3(bx, (nC + 3) / 4), kDirThreads, sm, s>>>(w, cost, ignore_done, seg);
        }
        return cudaGetLastError();
    }
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





// Scan candidates [q0, total) with stride `step` into the best admissible and
// the best overall key.
__device__ __forceinline__ void select_scan(const TabuBuffers &w, int t, int nC, long long v0c, long long v0d,
                                            long long bc, long long bd, long long q0, long long step,
                                            MoveKey &adm, MoveKey &all)
{
    const int B = w.B;
    const long long total = (long long)w.K * nC;
    for (long long q = q0; q < total; q += step) {
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
}

// Apply the chosen move (called by every thread of one block, with the block's
// final keys): tabu expiries, best so far, trajectory, and clearing V0 / loss
// for the refresh.  Also stops the search when there is no candidate, when the
// improving-only rule says so, or when the iteration budget is used up.
__device__ __forceinline__ void select_apply(const TabuBuffers &w, const MoveKey &adm, const MoveKey &all,
                                             long long v0c, long long v0d)
{
    TabuDevState *st = w.st;
    __shared__ int s_newbest;
    if (threadIdx.x == 0) {
        const int t = st->t;
        st->ticket = 0;
        st->work = 0;
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
                st->chg_total += st->chg_n;     // the records the last incremental pass took
                st->chg_n = 0;
                if (w.chg) {
                    // the closed base is a candidate again: its column of the
                    // terms is rebuilt from zero by the refresh
                    w.gain_c[P.i] = 0;
                    w.gain_d[P.i] = 0;
                }
                w.v0[0] = 0;
                w.v0[1] = 0;
            }
        }
    }
    __syncthreads();
    if (st->done) return;
    const int ic = st->mv_i;
    for (int k = threadIdx.x; k < w.K; k += blockDim.x) {
        w.loss_c[k] = 0;
        w.loss_d[k] = 0;
        if (s_newbest) w.best_open[k] = w.open[k];
        if (w.chg) {
            w.extra_c[(size_t)k * w.B + ic] = 0;
            w.extra_d[(size_t)k * w.B + ic] = 0;
        }
    }
}

// Multi-block selection: block `bid` of `nb` scans its share, the last block
// of the instance to finish (ticket) reduces the block results and applies.
__device__ __forceinline__ void select_body(const TabuBuffers &w, int bid, int nb)
{
    TabuDevState *st = w.st;
    __shared__ MoveKey s_adm[kSelectThreads / 32], s_all[kSelectThreads / 32];
    __shared__ int s_last;
    const int t = st->t;
    const int nC = st->nC;
    const long long v0c = (long long)w.v0[0], v0d = (long long)w.v0[1];
    const long long bc = st->best_cov, bd = st->best_dist;
    MoveKey adm = invalid_key(), all = invalid_key();
    select_scan(w, t, nC, v0c, v0d, bc, bd, bid * (long long)blockDim.x + threadIdx.x, (long long)nb * blockDim.x,
                adm, all);
    block_best2<kSelectThreads>(adm, all, s_adm, s_all);
    if (threadIdx.x == 0) {
        w.partials[2 * bid] = adm;
        w.partials[2 * bid + 1] = all;
        __threadfence();
        const unsigned int ticket = atomicAdd(&st->ticket, 1u);
        s_last = (ticket == (unsigned)nb - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    adm = invalid_key();
    all = invalid_key();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        MoveKey pa = load_key_cg(&w.partials[2 * b]);
        MoveKey px = load_key_cg(&w.partials[2 * b + 1]);
        if (key_better(pa, adm)) adm = pa;
        if (key_better(px, all)) all = px;
    }
    __syncthreads();
    block_best2<kSelectThreads>(adm, all, s_adm, s_all);
    select_apply(w, adm, all, v0c, v0d);
}

__global__ void __launch_bounds__(kSelectThreads) k_select(TabuBuffers w)
{
    TabuDevState *st = w.st;
    if (st->done || st->t >= st->t_end) return;
    select_body(w, blockIdx.x, gridDim.x);
}

// Blocks for K x nC candidates: about 2 candidates per thread (each one is a
// chain of dependent loads), at most kSelectBlocks.
int select_blocks(int K, int nC)
{
    const long long n = (long long)K * nC;
    long long b = (n + kSelectThreads * 2 - 1) / (kSelectThreads * 2);
    if (b < 1) b = 1;
    if (b > kSelectBlocks) b = kSelectBlocks;
    return (int)b;
}

cudaError_t launch_select(const TabuBuffers &w, int nC, cudaStream_t s)
{
    k_select<<<select_blocks(w.K, nC), kSelectThreads, 0, s>>>(w);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// a7: incremental refresh after move (slot s*, opened j*).  A mission whose
// best and second best do not use slot s* only has to consider j*; the others
// rescan the K open bases.  V0 and loss are rebuilt from the new arrays, and
// gain / extra are cleared for the next evaluation.
// --------------------------------------------------------------------------

   // missions queued for a cooperative rescan per block

// Dynamic shared memory of the refresh: per slot the loss (distance, count),
// the closed base's column terms (distance, count) and the base id.
size_t refresh_smem(int K) { return (size_t)K * (8 + 8 + 4 + 4 + 4); }






// a7: incremental refresh after the move (close slot mv_s, open base mv_j in
// it).  A thread loads a mission's state and the new base's cost together
// (one round trip, not two dependent ones).  A mission whose best and second
// best both stay open compares only the new base's cost.  One that lost either
// needs a rescan of the K open bases: with one mission per thread its own
// thread does it at once; with several (large instances, grouped searches) it
// is queued, and after the loop the whole block rescans the queue
// (refresh_rescans), so the long scans neither serialise behind a thread's
// other missions nor hold the block's other warps.  Past the queue's capacity
// a thread scans the mission itself.
__device__ __forceinline__ void refresh_body(const TabuBuffers &w, const int32_t *__restrict__ cost, int bid,
                                             int nb)
{
    TabuDevState *st = w.st;
    if (st->done || st->ls_hold) return;
    extern __shared__ unsigned long long sm_ref[];
    __shared__ int s_q[kRefQ];
    __shared__ int s_qn;
    unsigned long long *s_ld = sm_ref;
    unsigned long long *s_id = s_ld + w.K;                     // closed base's column: extra, distance
    int *s_lc = reinterpret_cast<int *>(s_id + w.K);
    int *s_ic = s_lc + w.K;                                    // closed base's column: extra, count
    int *s_open = s_ic + w.K;
    for (int k = threadIdx.x; k < w.K; k += blockDim.x) {
        s_open[k] = w.open[k];
        s_lc[k] = 0;
        s_ld[k] = 0;
        s_ic[k] = 0;
        s_id[k] = 0;
    }
    if (threadIdx.x == 0) s_qn = 0;
    __syncthreads();
    const int ss = st->mv_s, jj = st->mv_j, ic = st->mv_i;
    const size_t M_pad = w.M_pad;
    const int32_t *rowj = cost + (size_t)jj * M_pad;
    // incremental form: the closed base is a candidate again, its column of
    // the terms (zeroed with the move) is rebuilt here over every mission
    const bool inc = w.chg != nullptr;
    const int32_t *rowi = cost + (size_t)ic * M_pad;
    long long gic = 0, gid = 0;
    long long v0c = 0, v0d = 0;
    const int base = bid * (int)blockDim.x, stride = nb * (int)blockDim.x;
    const int rounds = w.M > base ? (w.M - base + stride - 1) / stride : 0;   // the same on every thread
    const bool queue = rounds > 1;
    const int lane = threadIdx.x & 31;
    for (int rd = 0; rd < rounds; rd++) {
        const int m = base + rd * stride + (int)threadIdx.x;
        int a = 0, b = 0, k1 = 0, k2 = 0, x = 0, xi = 0;
        bool in = m < w.M;
        if (in) {
            a = w.a[m]; b = w.b[m];
            k1 = w.s1[m]; k2 = w.s2[m];
            x = __ldcs(rowj + m);
            if (inc) xi = __ldcs(rowi + m);
            if (w.mask) in = w.mask[m] != 0;
        }
        bool term = false;
        const bool lost = in && (k1 == ss || k2 == ss);
        const int ao = a, bo = b, so = k1;   // the state before the move
        if (in && !lost) {
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
            term = true;
        }
        // queue the missions that lost their best or second best: one shared
        // atomic per warp, positions in lane order
        const unsigned lm = __ballot_sync(0xffffffffu, lost);
        if (lm) {
            int q0 = kRefQ;   // not queued: scanned in place
            if (queue) {
                if (lane == __ffs(lm) - 1) q0 = atomicAdd(&s_qn, __popc(lm));
                q0 = __shfl_sync(0xffffffffu, q0, __ffs(lm) - 1);
            }
            if (lost) {
                const int pos = q0 + __popc(lm & ((1u << lane) - 1u));
                if (pos < kRefQ) {
                    s_q[pos] = m;
                } else {
                    const int2 ab = refresh_scan_one(w, cost, m, s_open, k1);
                    a = ab.x; b = ab.y;
                    term = true;
                }
            }
        }
        if (term) {
            mission_terms(a, b, w.R, v0c, v0d, s_lc, s_ld, k1);
            if (inc) closed_column_terms(xi, a, b, k1, w.R, gic, gid, s_ic, s_id);
        }
        if (inc) record_changes(w, &st->chg_n, term && terms_changed(ao, bo, so, a, b, k1, w.R), m, ao, bo, so, a, b, k1);
    }
    __syncthreads();
    const int nq = min(s_qn, kRefQ);   // no thread changes the count after the barrier
    if (nq > 0)
        refresh_rescans(
            w, cost, s_open, s_q, nq, rowi, gic, gid, s_ic, s_id,
            [&](int a, int b, int k1) { mission_terms(a, b, w.R, v0c, v0d, s_lc, s_ld, k1); },
            [&](bool ch, int m, int ao, int bo, int so, int an, int bn, int sn) {
                record_changes(w, &st->chg_n, ch, m, ao, bo, so, an, bn, sn);
            });
    if (inc) {
        // the other terms stay; the closed base's column goes out
        block_sum2<256>(gic, gid);
        if (threadIdx.x == 0) {
            if (gic) atomicAdd(&w.gain_c[ic], (int)gic);
            if (gid) atomicAdd(&w.gain_d[ic], (unsigned long long)gid);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < w.K; k += blockDim.x) {
            if (s_ic[k]) atomicAdd(&w.extra_c[(size_t)k * w.B + ic], s_ic[k]);
            if (s_id[k]) atomicAdd(&w.extra_d[(size_t)k * w.B + ic], s_id[k]);
        }
    } else {
        // clear the neighbourhood accumulators for the next full evaluation
        const size_t nE = (size_t)w.K * w.B;
        const size_t tid = bid * (size_t)blockDim.x + threadIdx.x;
        const size_t nth = (size_t)nb * blockDim.x;
        for (size_t q = tid; q < nE; q += nth) { w.extra_c[q] = 0; w.extra_d[q] = 0; }
        for (size_t q = tid; q < (size_t)w.B; q += nth) { w.gain_c[q] = 0; w.gain_d[q] = 0; }
    }
    __syncthreads();
    flush_loss_v0(w, s_lc, s_ld, v0c, v0d);
}

__global__ void __launch_bounds__(256, 4) k_refresh(TabuBuffers w, const int32_t *__restrict__ cost)
{
    refresh_body(w, cost, blockIdx.x, gridDim.x);
}

cudaError_t launch_refresh(const TabuBuffers &w, const int32_t *cost, cudaStream_t s)
{
    const size_t sm = refresh_smem(w.K);
    k_refresh<<<grid_missions(w.M_pad), 256, sm, s>>>(w, cost);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// a4, incremental form.  With the gain and extra terms kept across
// iterations, a move changes them only through the missions whose clamped
// best / second-best cost or best slot changed (recorded by the refresh) and
// through the closed base, which is a candidate again.  k_swap_delta takes
// each recorded mission's old terms out of, and its new terms into, every
// other base's column; the refresh rebuilds the closed base's column over
// all missions.  Afterwards gain and extra equal what a full pass over the table
// would give for the new placement (integer sums: exactly), so the
// selection still scores every swap of the neighbourhood.
// --------------------------------------------------------------------------
constexpr int kDeltaRows = 256;    // positions of the mission-major copy (bases) per block, one per thread
constexpr int kDeltaChunk = 32;    // recorded missions staged per block step
constexpr int kDeltaBatch = 8;     // cost loads in flight per thread

bool swap_delta_fits(int K) { return K <= kPipeMaxK; }



// Thread = one position p of the mission-major copy, i.e. base border[p]
// (every base but the one the move closed: a column that is not a
// candidate's is never read, and is rebuilt by the refresh when its base
// closes); the block walks chunks of the record list, staged in shared
// memory, and a warp reads 32 consecutive positions of one mission (one
// 128-byte line).  The positions follow a spatial order of the bases, so the
// few bases near enough to a mission to carry a term sit in few warps and
// the others pass the mission together.  The gain terms of the base add up
// in registers; the extra terms go out in runs of one slot (the records come
// in runs of neighbouring missions, which share slots).
// Block (bx, by) of a gx x gy grid: positions bx * kDeltaRows .. +255, record
// chunks by, by + gy, ...
__device__ __forceinline__ void swap_delta_body(const TabuBuffers &w, int bx, int by, int gy)
{
    TabuDevState *st = w.st;
    if (st->done || st->ls_hold) return;
    __shared__ int4 s_old[kDeltaChunk];   // column, clamped a, clamped b, best slot: before the move
    __shared__ int4 s_new[kDeltaChunk];   // clamped a, clamped b, best slot: after
    __shared__ long long s_off[kDeltaChunk];   // the mission's row in the mission-major copy
    __shared__ int s_hi[kDeltaChunk];          // the larger clamped second best: no term from x >= it
    // the minima of the block's cells (a warp's 32 positions each) in each
    // staged mission's row: a warp whose cell minimum is at or above the
    // threshold has no term there and loads nothing (rows of 16 cells or more)
    __shared__ int s_cm[kDeltaChunk][kDeltaRows / 32];
    const int ic = st->mv_i, R = w.R;
    const int nrec = min(st->chg_n, w.M);
    const int p = bx * kDeltaRows + (int)threadIdx.x;
    const int j = p < w.ldT ? w.border[p] : -1;
    const bool row = j >= 0 && j != ic;   // the closed base's column: the refresh
    const int32_t *colp = w.costT + (row ? p : 0);
    const size_t ld = (size_t)w.ldT;
    // skipping cells pays only on long rows: the staging of the minima costs a
    // barrier and a scattered load per (record, cell) of each chunk
    const bool use_cm = (ld >> 5) >= 16;
    long long gc = 0, gd = 0;
    DeltaRun rn{-1, 0, 0}, ro{-1, 0, 0};   // the new state's terms, the old state's (taken out)
    for (int e0 = by * kDeltaChunk; e0 < nrec; e0 += gy * kDeltaChunk) {   // the same on every thread
        const int n = min(kDeltaChunk, nrec - e0);
        __syncthreads();   // the previous chunk is consumed
        if ((int)threadIdx.x < n) {
            const int4 ro = w.chg[2 * (size_t)(e0 + threadIdx.x)], rq = w.chg[2 * (size_t)(e0 + threadIdx.x) + 1];
            const int bo1 = min(ro.z, R + 1), bn1 = min(rq.y, R + 1);
            s_old[threadIdx.x] = make_int4(ro.x, min(ro.y, R + 1), bo1, ro.w);
            s_new[threadIdx.x] = make_int4(min(rq.x, R + 1), bn1, rq.z, 0);
            s_off[threadIdx.x] = (long long)ro.x * (long long)ld;
            s_hi[threadIdx.x] = max(bo1, bn1);
        }
        __syncthreads();
        if (use_cm) {   // the same on the block
            static_assert(kDeltaChunk * (kDeltaRows / 32) == kDeltaRows, "one cell minimum per thread");
            const int r = threadIdx.x / (kDeltaRows / 32), cw = threadIdx.x % (kDeltaRows / 32);
            const int cell = bx * (kDeltaRows / 32) + cw, nCell = (int)(ld >> 5);
            s_cm[r][cw] = (r < n && cell < nCell) ? __ldg(&w.cellmin[(size_t)s_old[r].x * cell_ld((int)ld) + cell])
                                                  : INT_MAX;
            __syncthreads();
        }
        if (!row) continue;
        const int cw = (int)threadIdx.x >> 5;   // this warp's cell of the block
        for (int k0 = 0; k0 < n; k0 += kDeltaBatch) {
            int xv[kDeltaBatch];
#pragma unroll
            for (int u = 0; u < kDeltaBatch; u++)
                xv[u] = (k0 + u < n && (!use_cm || s_cm[k0 + u][cw] < s_hi[k0 + u])) ? __ldg(colp + s_off[k0 + u])
                                                                                     : INT_MAX;
#pragma unroll
            for (int u = 0; u < kDeltaBatch; u++) {
                const int x = xv[u];
                if (k0 + u >= n) break;
                if (x >= s_hi[k0 + u]) continue;   // no term in either state (a <= b)
                const int4 o = s_old[k0 + u], q = s_new[k0 + u];
                const int ao = o.y, bo = o.z, so = o.w, an = q.x, bn = q.y, sn = q.z;
                const int cao = ao <= R, cbo = bo <= R, can = an <= R, cbn = bn <= R;
                if (x < an) { gc += 1 - can; gd += (long long)x - (can ? an : 0); }
                if (x < ao) { gc -= 1 - cao; gd -= (long long)x - (cao ? ao : 0); }
                if (x < bn) {
                    const int nc = can - cbn, nd = (can ? max(x, an) : 0) - (cbn ? bn : 0);
                    if (nc | nd) delta_run_add(rn, sn, nc, nd, w, j);
                }
                if (x < bo) {
                    const int oc = cao - cbo, od = (cao ? max(x, ao) : 0) - (cbo ? bo : 0);
                    if (oc | od) delta_run_add(ro, so, -oc, -od, w, j);
                }
            }
        }
    }
    if (!row) return;
    delta_run_add(rn, -1, 0, 0, w, j);   // flush
    delta_run_add(ro, -1, 0, 0, w, j);
    if (gc) atomicAdd(&w.gain_c[j], (int)gc);
    if (gd) atomicAdd(&w.gain_d[j], (unsigned long long)gd);
}

__global__ void __launch_bounds__(kDeltaRows) k_swap_delta(TabuBuffers w)
{
    swap_delta_body(w, blockIdx.x, blockIdx.y, gridDim.y);
}

cudaError_t launch_swap_delta(const TabuBuffers &w, cudaStream_t s)
{
    const int gx = (w.ldT + kDeltaRows - 1) / kDeltaRows;
    // about two waves of resident blocks over the record chunks (their count
    // is known only on the device), no more than the missions could fill
    const int sms = sm_count();
    const int max_y = (w.M + kDeltaChunk - 1) / kDeltaChunk;
    int gy = (2 * 6 * sms + gx - 1) / gx;
    if (gy > max_y) gy = max_y;
    if (gy < 1) gy = 1;
    k_swap_delta<<<dim3(gx, gy), kDeltaRows, 0, s>>>(w);
    return cudaGetLastError();
}

int table_ldT(int B) { return (B + 31) / 32 * 32; }

// Tiled transpose through shared memory: reads and writes both coalesced;
// position p of a mission's row holds base border[p] (INT32_MAX past B).  Each
// tile also gives, per mission, the least cost of its 32 positions (the cell
// minimum, cellmin[m * cell_ld(ldT) + cell]): exact, and enough to skip a cell
// with no cost below a threshold.
__global__ void __launch_bounds__(256) k_transpose_table(const int32_t *__restrict__ cost, int M_pad, int ldT,
                                                         const int32_t *__restrict__ border,
                                                         int32_t *__restrict__ costT, int32_t *__restrict__ cellmin)
{
    __shared__ int32_t tile[32][33];
    const int m0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int k = ty; k < 32; k += 8) {
        const int b = border[b0 + k], m = m0 + tx;
        tile[k][tx] = (b >= 0 && m < M_pad) ? cost[(size_t)b * M_pad + m] : INT_MAX;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {   // a warp: one mission's 32 positions of the cell
        const int m = m0 + k, b = b0 + tx;
        const int32_t v = tile[tx][k];
        if (m < M_pad && b < ldT) costT[(size_t)m * ldT + b] = v;
        const int32_t mn = __reduce_min_sync(0xffffffffu, v);
        if (tx == 0 && m < M_pad) cellmin[(size_t)m * cell_ld(ldT) + blockIdx.y] = mn;
    }
}

cudaError_t launch_transpose_table(const int32_t *cost, int B, int M_pad, const int32_t *border, int32_t *costT,
                                   int32_t *cellmin, cudaStream_t s)
{
    const int ldT = table_ldT(B);
    k_transpose_table<<<dim3((M_pad + 31) / 32, ldT / 32), 256, 0, s>>>(cost, M_pad, ldT, border, costT,
                                                                           cellmin);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Local search (Alg. 2 as read for identical vehicles): with the accumulators
// of the current placement, find the first strictly improving (slot,
// candidate position) pair at or after the scan position in the current
// pass's order, u = rank_slot[s] * nC + rank_cand[c].  Each block keeps its
// smallest improving u; the last block to finish reduces them and applies the
// move, changes pass (accumulators stay valid: evaluation and refresh skip the
// next step), or stops.
// --------------------------------------------------------------------------
struct LsKey {
    long long cov, dist;
    int u, s, c, i, j, valid;
};
static_assert(sizeof(LsKey) <= sizeof(MoveKey), "local-search keys reuse the partials buffer");

__device__ __forceinline__ bool ls_first(const LsKey &a, const LsKey &b)
{
    return a.valid && (!b.valid || a.u < b.u);
}

// Smallest scan position of a block (every thread receives the key): a warp
// minimum, then one warp over the warps' winners.  Positions are unique.
__device__ __forceinline__ void ls_block_first(LsKey &k, LsKey *sh)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned u = k.valid ? (unsigned)k.u : 0xffffffffu;
    unsigned bu = __reduce_min_sync(full, u);
    if (lane == __ffs(__ballot_sync(full, u == bu)) - 1) sh[wid] = k;
    __syncthreads();
    if (wid == 0) {
        LsKey c;
        c.valid = 0;
        c.u = 0x7fffffff;
        if (lane < kSelectThreads / 32) c = sh[lane];
        u = c.valid ? (unsigned)c.u : 0xffffffffu;
        bu = __reduce_min_sync(full, u);
        const int src = __ffs(__ballot_sync(full, u == bu)) - 1;
        __syncwarp();
        if (lane == src) sh[0] = c;
    }
    __syncthreads();
    k = sh[0];
    __syncthreads();
}

__global__ void __launch_bounds__(kSelectThreads) k_ls_select(TabuBuffers w, const int *__restrict__ rank_slot,
                                                             const int *__restrict__ rank_cand)
{
    TabuDevState *st = w.st;
    if (st->done) return;
    __shared__ LsKey sh[kSelectThreads / 32];
    __shared__ int s_last, s_moved;
    const int nC = st->nC, K = w.K, pass = st->ls_pass, u0 = st->ls_pos;
    const int *ra = rank_slot + (size_t)pass * K;
    const int *rb = rank_cand + (size_t)pass * nC;
    const long long v0c = (long long)w.v0[0], v0d = (long long)w.v0[1];
    const long long cc = st->cur_cov, cd = st->cur_dist;
    const bool budget_left = st->n_moves < st->traj_cap;
    LsKey best;
    best.valid = 0;
    best.u = 0x7fffffff;
    const long long total = (long long)K * nC;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; budget_left && q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(q / nC), c = (int)(q % nC);
        const int u = ra[s] * nC + rb[c];
        if (u < u0 || (best.valid && u >= best.u)) continue;
        const int j = w.cand[c];
        const size_t sj = (size_t)s * w.B + j;
        const long long cov = v0c + w.gain_c[j] + (long long)w.loss_c[s] + w.extra_c[sj];
        const long long dist = v0d + (long long)w.gain_d[j] + (long long)w.loss_d[s] + (long long)w.extra_d[sj];
        if (obj_better(cov, dist, cc, cd)) {
            best.cov = cov; best.dist = dist; best.u = u; best.s = s; best.c = c;
            best.i = w.open[s]; best.j = j; best.valid = 1;
        }
    }
    ls_block_first(best, sh);
    LsKey *part = reinterpret_cast<LsKey *>(w.partials);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = best;
        __threadfence();
        const unsigned int ticket = atomicAdd(&st->ticket, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    best.valid = 0;
    best.u = 0x7fffffff;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        LsKey k;
        k.cov = __ldcg(&part[b].cov);
        k.dist = __ldcg(&part[b].dist);
        k.u = __ldcg(&part[b].u);
        k.s = __ldcg(&part[b].s);
        k.c = __ldcg(&part[b].c);
        k.i = __ldcg(&part[b].i);
        k.j = __ldcg(&part[b].j);
        k.valid = __ldcg(&part[b].valid);
        if (ls_first(k, best)) best = k;
    }
    ls_block_first(best, sh);
    if (threadIdx.x == 0) {
        st->ticket = 0;
        s_moved = 0;
        if (st->cur_cov != v0c || st->cur_dist != v0d) {
            st->err |= kErrObjectiveMismatch;   // refresh disagreed with the applied move
            st->done = 1;
        } else if (!budget_left) {
            st->done = 1;                        // move budget used up
        } else if (best.valid) {
            const int t = st->t;
            w.open[best.s] = best.j;
            w.cand[best.c] = best.i;
            st->cur_cov = best.cov;
            st->cur_dist = best.dist;
            st->best_cov = best.cov;             // every applied move is strictly better
            st->best_dist = best.dist;
            st->best_iter = t;
            stage_move mv;
            mv.iter = t; mv.i = best.i; mv.j = best.j; mv.flags = STAGE_MOVE_NEW_BEST;
            mv.cov = best.cov; mv.dist = best.dist;
            w.traj[st->n_moves] = mv;
            st->n_moves += 1;
            st->t = t + 1;
            st->mv_s = best.s; st->mv_i = best.i; st->mv_j = best.j;
            st->ls_pos = best.u + 1;
            st->ls_moved = 1;
            st->ls_hold = 0;
            st->chg_total += st->chg_n;          // the records the last incremental pass took
            st->chg_n = 0;
            if (w.chg) {
                // the closed base is a candidate again: its column of the terms
                // is rebuilt from zero by the refresh
                w.gain_c[best.i] = 0;
                w.gain_d[best.i] = 0;
            }
            w.v0[0] = 0;
            w.v0[1] = 0;
            s_moved = 1;
        } else if (st->ls_moved && st->ls_pass + 1 < st->ls_passes) {
            st->ls_pass += 1;                    // next pair of permutations, same placement
            st->ls_pos = 0;
            st->ls_moved = 0;
            st->ls_hold = 1;
        } else {
            st->ls_optimum = st->ls_moved ? 0 : 1;
            st->done = 1;
        }
    }
    __syncthreads();
    if (!s_moved) return;
    const int ic = st->mv_i;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        w.loss_c[k] = 0;
        w.loss_d[k] = 0;
        w.best_open[k] = w.open[k];
        if (w.chg) {
            w.extra_c[(size_t)k * w.B + ic] = 0;
            w.extra_d[(size_t)k * w.B + ic] = 0;
        }
    }
}

cudaError_t launch_ls_select(const TabuBuffers &w, int nC, const int *rank_slot, const int *rank_cand,
                             cudaStream_t s)
{
    k_ls_select<<<select_blocks(w.K, nC), kSelectThreads, 0, s>>>(w, rank_slot, rank_cand);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Heterogeneous fleet (the vehicle and base types of Sec. 3, Eq. 6-10, as read
// for this model): Kr rotary-wing vehicles in slots 0 .. Kr-1 (any base) and
// fixed-wing vehicles in the other slots (aerodromes only); rotary-only
// missions may be flown by rotary-wing vehicles only.  Two searches share the
// table: A (all vehicles, the missions any vehicle may fly) and B (the
// rotary-wing vehicles, the rotary-only missions).  Moving a rotary-wing
// vehicle from i to j changes both, F = F_A(s, j) + F_B(s, j); moving a
// fixed-wing vehicle changes only A, F = F_A(s, j) + V0_B, and then B's
// accumulators stay valid (B holds: its next swap pass and refresh are
// skipped).  Same admissibility, aspiration, fallback, tie-break and
// improving-only rule as k_select, over A's candidate list.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(kSelectThreads) k_fleet_select(TabuBuffers A, TabuBuffers B, int Kr, int hasB,
                                                                const uint8_t *__restrict__ helipad,
                                                                int *__restrict__ b_pos)
{
    TabuDevState *st = A.st;
    if (st->done || st->t >= st->t_end) return;
    __shared__ MoveKey s_adm[kSelectThreads / 32], s_all[kSelectThreads / 32];
    __shared__ int s_last, s_moved, s_newbest, s_rot;
    const int t = st->t;
    const int nC = st->nC, K = A.K, Bn = A.B;
    const long long v0c = (long long)A.v0[0] + (hasB ? (long long)B.v0[0] : 0ll);
    const long long v0d = (long long)A.v0[1] + (hasB ? (long long)B.v0[1] : 0ll);
    const long long bc = st->best_cov, bd = st->best_dist;
    MoveKey adm = invalid_key(), all = invalid_key();
    const long long total = (long long)K * nC;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int sl = (int)(q / nC), c = (int)(q % nC);
        const int j = A.cand[c];
        const bool rot = sl < Kr;
        if (!rot && helipad[j]) continue;   // a fixed-wing vehicle needs an aerodrome
        const size_t sj = (size_t)sl * Bn + j;
        MoveKey k;
        k.cov = v0c + A.gain_c[j] + (long long)A.loss_c[sl] + A.extra_c[sj];
        k.dist = v0d + (long long)A.gain_d[j] + (long long)A.loss_d[sl] + (long long)A.extra_d[sj];
        if (rot && hasB) {
            k.cov += B.gain_c[j] + (long long)B.loss_c[sl] + B.extra_c[sj];
            k.dist += (long long)B.gain_d[j] + (long long)B.loss_d[sl] + (long long)B.extra_d[sj];
        }
        k.i = A.open[sl]; k.j = j; k.s = sl; k.c = c; k.valid = 1;
        k.tabu = (t < A.expiry[k.i]) || (t < A.expiry[j]);
        if (key_better(k, all)) all = k;
        if ((!k.tabu || obj_better(k.cov, k.dist, bc, bd)) && key_better(k, adm)) adm = k;
    }
    block_best2<kSelectThreads>(adm, all, s_adm, s_all);
    if (threadIdx.x == 0) {
        A.partials[2 * blockIdx.x] = adm;
        A.partials[2 * blockIdx.x + 1] = all;
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
        MoveKey pa = load_key_cg(&A.partials[2 * b]);
        MoveKey px = load_key_cg(&A.partials[2 * b + 1]);
        if (key_better(pa, adm)) adm = pa;
        if (key_better(px, all)) all = px;
    }
    __syncthreads();
    block_best2<kSelectThreads>(adm, all, s_adm, s_all);
    if (threadIdx.x == 0) {
        st->ticket = 0;
        s_moved = 0;
        s_newbest = 0;
        s_rot = 0;
        if (!all.valid) {
            st->done = 1;                       // no move at all
        } else if (st->cur_cov != v0c || st->cur_dist != v0d) {
            st->err |= kErrObjectiveMismatch;   // the refreshes disagreed with the chosen move
            st->done = 1;
        } else {
            const MoveKey P = adm.valid ? adm : all;
            int flags = adm.valid ? (adm.tabu ? STAGE_MOVE_ASPIRATION : 0) : STAGE_MOVE_FALLBACK;
            if (!st->accept_worsening && !obj_better(P.cov, P.dist, st->cur_cov, st->cur_dist)) {
                st->done = 1;
            } else {
                A.open[P.s] = P.j;
                A.cand[P.c] = P.i;
                A.expiry[P.i] = t + st->tenure + 1;
                A.expiry[P.j] = t + st->tenure + 1;
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
                    A.traj[st->n_moves] = mv;
                }
                st->n_moves += 1;
                st->t = t + 1;
                st->mv_s = P.s; st->mv_i = P.i; st->mv_j = P.j;
                st->chg_total += st->chg_n;     // the records the last incremental pass took
                st->chg_n = 0;
                if (A.chg) {   // the closed base's column is rebuilt from zero by the refresh
                    A.gain_c[P.i] = 0;
                    A.gain_d[P.i] = 0;
                }
                A.v0[0] = 0;
                A.v0[1] = 0;
                s_moved = 1;
                if (hasB) {
                    TabuDevState *sb = B.st;
                    if (P.s < Kr) {
                        // the rotary-wing vehicle moved: B's placement and candidates follow
                        const int pos = b_pos[P.j];
                        B.open[P.s] = P.j;
                        B.cand[pos] = P.i;
                        b_pos[P.i] = pos;
                        b_pos[P.j] = -1;
                        sb->mv_s = P.s; sb->mv_i = P.i; sb->mv_j = P.j;
                        sb->ls_hold = 0;
                        sb->chg_total += sb->chg_n;
                        sb->chg_n = 0;
                        if (B.chg) {
                            B.gain_c[P.i] = 0;
                            B.gain_d[P.i] = 0;
                        }
                        B.v0[0] = 0;
                        B.v0[1] = 0;
                        s_rot = 1;
                    } else {
                        sb->ls_hold = 1;                // B unchanged: skip its swap pass and refresh
                    }
                }
            }
        }
        if (st->done && hasB) B.st->done = 1;
    }
    __syncthreads();
    if (!s_moved) return;
    const int ic = st->mv_i;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        A.loss_c[k] = 0;
        A.loss_d[k] = 0;
        if (s_newbest) A.best_open[k] = A.open[k];
        if (A.chg) {
            A.extra_c[(size_t)k * A.B + ic] = 0;
            A.extra_d[(size_t)k * A.B + ic] = 0;
        }
    }
    if (s_rot)
        for (int k = threadIdx.x; k < B.K; k += blockDim.x) {
            B.loss_c[k] = 0;
            B.loss_d[k] = 0;
            if (B.chg) {
                B.extra_c[(size_t)k * B.B + ic] = 0;
                B.extra_d[(size_t)k * B.B + ic] = 0;
            }
        }
}

cudaError_t launch_fleet_select(const TabuBuffers &A, const TabuBuffers &B, int Kr, int hasB,
                                const uint8_t *helipad, int *b_pos, cudaStream_t s)
{
    // A's state holds the candidate count
    k_fleet_select<<<kSelectBlocks, kSelectThreads, 0, s>>>(A, B, Kr, hasB, helipad, b_pos);
    return cudaGetLastError();
}

// Per-mission arrays back in the caller's mission order (perm: column -> mission).
__global__ void k_export_best_two(TabuBuffers w, const int *__restrict__ perm, int32_t *__restrict__ a,
                                  int32_t *__restrict__ b, int32_t *__restrict__ b1, int32_t *__restrict__ b2)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < w.M; q += gridDim.x * blockDim.x) {
        const int m = perm ? perm[q] : q;
        if (m < 0) continue;   // removed mission
        a[m] = w.a[q];
        b[m] = w.b[q];
        const int k1 = w.s1[q], k2 = w.s2[q];
        b1[m] = w.open[k1];
        b2[m] = k2 >= 0 ? w.open[k2] : -1;
    }
}

// --------------------------------------------------------------------------
// Small instances: the whole search in one resident block.  Each iteration
// runs every swap tile, the selection and the refresh back to back, separated
// by block barriers, so a search costs one launch instead of three per
// iteration.  Same bodies, same arithmetic, same results as the multi-kernel
// path.
// --------------------------------------------------------------------------
constexpr long long kSmallElems = 1ll << 18;   // (candidates) x (padded missions)

bool tabu_small_fits(int nC, int M_pad, int K)
{
    return (long long)nC * M_pad <= kSmallElems && K <= kPipeMaxK;
}

__global__ void __launch_bounds__(kDirThreads) k_tabu_small(TabuBuffers w, const int32_t *__restrict__ cost,
                                                            int iters)
{
    TabuDevState *st = w.st;
    const int seg = ((w.M_pad + 1023) / 1024) * 1024;   // one segment covers every mission
    for (int it = 0; it < iters; it++) {
        if (st->done || st->t >= st->t_end) break;
        const int nC = st->nC;
        for (int by = 0; by * kDirJ < nC; by++) {
            swap_direct_body<kDirJ>(w, cost, 0, by, seg);
            __syncthreads();
        }
        select_body(w, 0, 1);
        __syncthreads();
        refresh_body(w, cost, 0, 1);
        __syncthreads();
    }
}

cudaError_t launch_tabu_small(const TabuBuffers &w, const int32_t *cost, int iters, cudaStream_t s)
{
    const size_t sm = swap_direct_smem(w.K) > refresh_smem(w.K) ? swap_direct_smem(w.K) : refresh_smem(w.K);
    k_tabu_small<<<1, kDirThreads, sm, s>>>(w, cost, iters);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Small instances, resident form: the whole Tabu search in one block of 1024
// threads with every per-iteration array in shared memory -- best / second
// best per mission, gain and extra per candidate position, loss, the
// placement, the candidate list and the tabu expiries.  Only the cost table
// (L2-resident at these sizes) and the trajectory live in global memory.  One
// iteration: the swap pass (a warp per candidate position, so each gain and
// extra entry has a single writer), the selection (warp-shuffle then one
// warp), the move by one thread, the refresh.  Same rules and tie-breaks as
// the multi-kernel path; the state is written back at the end.
// --------------------------------------------------------------------------
constexpr int kResThreads = 1024;
constexpr int kResWarps = kResThreads / 32;

struct ResLayout {
    size_t gain_d, extra_d, loss_d, gain_c, extra_c, loss_c, a, b, s1, s2, open, cand, expiry, bytes;
};

__host__ __device__ inline ResLayout res_layout(int K, int B, int M_pad, int nC)
{
    ResLayout L;
    size_t o = 0;
    auto take = [&](size_t n, size_t al) {
        o = (o + al - 1) / al * al;
        const size_t at = o;
        o += n;
        return at;
    };
    L.gain_d = take((size_t)nC * 8, 8);
    L.extra_d = take((size_t)K * nC * 8, 8);
    L.loss_d = take((size_t)K * 8, 8);
    L.gain_c = take((size_t)nC * 4, 4);
    L.extra_c = take((size_t)K * nC * 4, 4);
    L.loss_c = take((size_t)K * 4, 4);
    L.a = take((size_t)M_pad * 4, 16);
    L.b = take((size_t)M_pad * 4, 16);
    L.s1 = take((size_t)M_pad * 2, 16);
    L.s2 = take((size_t)M_pad * 2, 16);
    L.open = take((size_t)K * 4, 4);
    L.cand = take((size_t)nC * 4, 4);
    L.expiry = take((size_t)B * 4, 4);
    L.bytes = (o + 15) / 16 * 16;
    return L;
}

// Bytes of the resident kernel's shared memory with the cost table staged in
// it too (0 when it does not fit: the table is then read from global memory).
__host__ __device__ inline size_t res_bytes_with_table(int K, int B, int M_pad, int nC)
{
    const size_t base = res_layout(K, B, M_pad, nC).bytes;
    const size_t all = base + (size_t)B * M_pad * 4;
    return all <= 160 * 1024 ? all : 0;
}

constexpr size_t kResMaxSmem = 160 * 1024;

bool tabu_resident_fits(int K, int B, int M_pad, int nC)
{
    return (long long)nC * M_pad <= kSmallElems && K <= kPipeMaxK &&
           res_layout(K, B, M_pad, nC).bytes <= kResMaxSmem;
}

__global__ void __launch_bounds__(kResThreads, 1) k_tabu_resident(TabuBuffers w, const int32_t *__restrict__ cost,
                                                                 int iters)
{
    extern __shared__ __align__(16) unsigned char sm_res[];
    TabuDevState *gst = w.st;
    const int K = w.K, B = w.B, M = w.M, R = w.R;
    const size_t M_pad = w.M_pad;
    const int nC = gst->nC;
    const ResLayout L = res_layout(K, B, (int)M_pad, nC);
    long long *gain_d = reinterpret_cast<long long *>(sm_res + L.gain_d);
    long long *extra_d = reinterpret_cast<long long *>(sm_res + L.extra_d);
    long long *loss_d = reinterpret_cast<long long *>(sm_res + L.loss_d);
    int *gain_c = reinterpret_cast<int *>(sm_res + L.gain_c);
    int *extra_c = reinterpret_cast<int *>(sm_res + L.extra_c);
    int *loss_c = reinterpret_cast<int *>(sm_res + L.loss_c);
    int *sa = reinterpret_cast<int *>(sm_res + L.a);
    int *sb = reinterpret_cast<int *>(sm_res + L.b);
    int16_t *ss1 = reinterpret_cast<int16_t *>(sm_res + L.s1);
    int16_t *ss2 = reinterpret_cast<int16_t *>(sm_res + L.s2);
    int *open = reinterpret_cast<int *>(sm_res + L.open);
    int *cand = reinterpret_cast<int *>(sm_res + L.cand);
    int *expiry = reinterpret_cast<int *>(sm_res + L.expiry);
    // the cost table: a shared-memory copy when it fits, else global memory
    // (plain loads below, valid for both)
    const bool staged = res_bytes_with_table(K, B, (int)M_pad, nC) != 0;
    const int32_t *tab = cost;
    if (staged) {
        int4 *dst = reinterpret_cast<int4 *>(sm_res + L.bytes);
        const int4 *src = reinterpret_cast<const int4 *>(cost);
        const size_t n4 = (size_t)B * M_pad / 4;
        for (size_t q = threadIdx.x; q < n4; q += kResThreads) dst[q] = __ldg(src + q);
        tab = reinterpret_cast<const int32_t *>(sm_res + L.bytes);
    }
    __shared__ MoveKey w_adm[kResWarps], w_all[kResWarps];
    __shared__ long long s_v0c, s_v0d, s_curc, s_curd, s_bestc, s_bestd;
    __shared__ long long r_c[kResWarps], r_d[kResWarps];
    __shared__ int s_t, s_nmoves, s_done, s_err, s_best_iter, s_mv_s, s_mv_j, s_moved, s_newbest;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---- load the state set up by the init / begin kernels
    for (int m = tid; m < M; m += kResThreads) {
        sa[m] = w.a[m];
        sb[m] = w.b[m];
        ss1[m] = w.s1[m];
        ss2[m] = w.s2[m];
    }
    for (int k = tid; k < K; k += kResThreads) {
        open[k] = w.open[k];
        loss_c[k] = (int)(long long)w.loss_c[k];
        loss_d[k] = (long long)w.loss_d[k];
    }
    for (int c = tid; c < nC; c += kResThreads) cand[c] = w.cand[c];
    for (int b = tid; b < B; b += kResThreads) expiry[b] = w.expiry[b];
    if (tid == 0) {
        s_v0c = (long long)w.v0[0];
        s_v0d = (long long)w.v0[1];
        s_curc = gst->cur_cov;
        s_curd = gst->cur_dist;
        s_bestc = gst->best_cov;
        s_bestd = gst->best_dist;
        s_best_iter = gst->best_iter;
        s_t = gst->t;
        s_nmoves = gst->n_moves;
        s_done = gst->done;
        s_err = 0;
        s_mv_s = gst->mv_s;
        s_mv_j = gst->mv_j;
    }
    __syncthreads();
    const int tenure = gst->tenure, accept_worsening = gst->accept_worsening, traj_cap = gst->traj_cap;
    const int t_end = gst->t_end;

    for (int it = 0; it < iters; it++) {
        if (s_done || s_t >= t_end) break;
        // ---- swap pass
        for (int q = tid; q < K * nC; q += kResThreads) {
            extra_c[q] = 0;
            extra_d[q] = 0;
        }
        __syncthreads();
        for (int c = warp; c < nC; c += kResWarps) {
            const int32_t *row = tab + (size_t)cand[c] * M_pad;
            int gc = 0;
            long long gd = 0;
            for (int m0 = 0; m0 < M; m0 += 32) {
                const int m = m0 + lane;
                const bool act = m < M;
                const int x = act ? row[m] : INT_MAX;
                const int ap = act ? min(sa[m], R + 1) : 0;
                const int bp = act ? min(sb[m], R + 1) : INT_MIN;
                const bool hb = x < bp;
                if (!__any_sync(0xffffffffu, hb)) continue;
                const int ca = ap <= R, cb = bp <= R;
                const int dc = hb ? ca - cb : 0;
                const long long dd = hb ? (ca ? (long long)max(x, ap) : 0ll) - (cb ? (long long)bp : 0ll) : 0ll;
                const int key = (dc | (dd != 0)) ? (int)ss1[m] : -1;
                const unsigned peers = __match_any_sync(0xffffffffu, key);
                const int sc = (int)__reduce_add_sync(peers, (unsigned)dc);
                const long long sd = group_sum_small(peers, dd);
                if (key >= 0 && lane == __ffs(peers) - 1) {
                    extra_c[key * nC + c] += sc;   // this warp is the only writer of column c
                    extra_d[key * nC + c] += sd;
                }
                if (x < ap) {
                    gc += 1 - ca;
                    gd += (long long)x - (ca ? (long long)ap : 0ll);
                }
            }
            gc = (int)__reduce_add_sync(0xffffffffu, (unsigned)gc);
            gd = warp_sum_ll(gd);
            if (lane == 0) {
                gain_c[c] = gc;
                gain_d[c] = gd;
            }
        }
        __syncthreads();
        // ---- selection (same keys and rules as k_select)
        {
            const int t = s_t;
            const long long v0c = s_v0c, v0d = s_v0d, bc = s_bestc, bd = s_bestd;
            MoveKey adm = invalid_key(), all = invalid_key();
            for (int q = tid; q < K * nC; q += kResThreads) {
                const int sl = q / nC, c = q % nC;
                MoveKey k;
                k.i = open[sl];
                k.j = cand[c];
                k.s = sl;
                k.c = c;
                k.cov = v0c + gain_c[c] + loss_c[sl] + extra_c[q];
                k.dist = v0d + gain_d[c] + loss_d[sl] + extra_d[q];
                k.valid = 1;
                k.tabu = (t < expiry[k.i]) || (t < expiry[k.j]);
                if (key_better(k, all)) all = k;
                if ((!k.tabu || obj_better(k.cov, k.dist, bc, bd)) && key_better(k, adm)) adm = k;
            }
            warp_best_key(adm);
            warp_best_key(all);
            if (lane == 0) {
                w_adm[warp] = adm;
                w_all[warp] = all;
            }
            __syncthreads();
            if (warp == 0) {
                adm = w_adm[lane];
                all = w_all[lane];
                warp_best_key(adm);
                warp_best_key(all);
                if (lane == 0) {
                    s_moved = 0;
                    s_newbest = 0;
                    if (!all.valid) {
                        s_done = 1;
                    } else if (s_curc != v0c || s_curd != v0d) {
                        s_err |= kErrObjectiveMismatch;
                        s_done = 1;
                    } else {
                        const MoveKey P = adm.valid ? adm : all;
                        int flags = adm.valid ? (adm.tabu ? STAGE_MOVE_ASPIRATION : 0) : STAGE_MOVE_FALLBACK;
                        if (!accept_worsening && !obj_better(P.cov, P.dist, s_curc, s_curd)) {
                            s_done = 1;
                        } else {
                            open[P.s] = P.j;
                            cand[P.c] = P.i;
                            expiry[P.i] = t + tenure + 1;
                            expiry[P.j] = t + tenure + 1;
                            s_curc = P.cov;
                            s_curd = P.dist;
                            if (obj_better(P.cov, P.dist, s_bestc, s_bestd)) {
                                s_bestc = P.cov;
                                s_bestd = P.dist;
                                s_best_iter = t;
                                flags |= STAGE_MOVE_NEW_BEST;
                                s_newbest = 1;
                            }
                            if (s_nmoves < traj_cap) {
                                stage_move mv;
                                mv.iter = t; mv.i = P.i; mv.j = P.j; mv.flags = flags;
                                mv.cov = P.cov; mv.dist = P.dist;
                                w.traj[s_nmoves] = mv;
                            }
                            s_nmoves += 1;
                            s_t = t + 1;
                            s_mv_s = P.s;
                            s_mv_j = P.j;
                            s_moved = 1;
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (!s_moved) continue;   // stopped: the loop condition ends the search
        if (s_newbest)
            for (int k = tid; k < K; k += kResThreads) w.best_open[k] = open[k];
        // ---- refresh (slot s* now holds j*)
        for (int k = tid; k < K; k += kResThreads) {
            loss_c[k] = 0;
            loss_d[k] = 0;
        }
        __syncthreads();
        {
            const int ssl = s_mv_s, jj = s_mv_j;
            const int32_t *rowj = tab + (size_t)jj * M_pad;
            long long v0c = 0, v0d = 0;
            for (int m0 = 0; m0 < M; m0 += kResThreads) {
                const int m = m0 + tid;
                const bool act = m < M;
                int a = 0, b = 0, k1 = -1, k2 = -1;
                if (act) {
                    a = sa[m]; b = sb[m]; k1 = ss1[m]; k2 = ss2[m];
                    if (k1 != ssl && k2 != ssl) {
                        const int x = rowj[m];
                        const int id1 = open[k1];
                        const int id2 = k2 >= 0 ? open[k2] : 0x7fffffff;
                        if (x < a || (x == a && jj < id1)) {
                            k2 = k1; b = a;
                            k1 = ssl; a = x;
                        } else if (k2 < 0 || x < b || (x == b && jj < id2)) {
                            k2 = ssl; b = x;
                        }
                    } else {
                        // best two over the open bases by (cost, base id)
                        int c1 = kInf, c2 = kInf, i1 = 0x7fffffff, i2 = 0x7fffffff;
                        k1 = -1;
                        k2 = -1;
                        for (int k = 0; k < K; k++) {
                            const int o = open[k];
                            const int cv = tab[(size_t)o * M_pad + m];
                            if (k1 < 0 || cv < c1 || (cv == c1 && o < i1)) {
                                k2 = k1; c2 = c1; i2 = i1;
                                k1 = k; c1 = cv; i1 = o;
                            } else if (k2 < 0 || cv < c2 || (cv == c2 && o < i2)) {
                                k2 = k; c2 = cv; i2 = o;
                            }
                        }
                        a = c1;
                        b = c2;
                    }
                    sa[m] = a; sb[m] = b; ss1[m] = (int16_t)k1; ss2[m] = (int16_t)k2;
                }
                const int ca = act && a <= R, cb = act && b <= R;
                const long long da = ca ? a : 0, db = cb ? b : 0;
                v0c += ca;
                v0d += da;
                const int dc = cb - ca;
                const long long dd = db - da;
                const int key = act && (dc | (dd != 0)) ? k1 : -1;
                const unsigned peers = __match_any_sync(0xffffffffu, key);
                const int sc = (int)__reduce_add_sync(peers, (unsigned)dc);
                const long long sd = group_sum_small(peers, dd);
                if (key >= 0 && lane == __ffs(peers) - 1) {
                    atomicAdd(&loss_c[key], sc);
                    atomicAdd(reinterpret_cast<unsigned long long *>(&loss_d[key]), (unsigned long long)sd);
                }
            }
            v0c = warp_sum_ll(v0c);
            v0d = warp_sum_ll(v0d);
            if (lane == 0) {
                r_c[warp] = v0c;
                r_d[warp] = v0d;
            }
            __syncthreads();
            if (tid == 0) {
                long long x = 0, y = 0;
                for (int k = 0; k < kResWarps; k++) {
                    x += r_c[k];
                    y += r_d[k];
                }
                s_v0c = x;
                s_v0d = y;
            }
            __syncthreads();
        }
    }
    // ---- write the state back
    __syncthreads();
    for (int m = tid; m < M; m += kResThreads) {
        w.a[m] = sa[m];
        w.b[m] = sb[m];
        w.s1[m] = ss1[m];
        w.s2[m] = ss2[m];
    }
    for (int k = tid; k < K; k += kResThreads) {
        w.open[k] = open[k];
        w.loss_c[k] = (unsigned long long)(long long)loss_c[k];
        w.loss_d[k] = (unsigned long long)loss_d[k];
    }
    for (int c = tid; c < nC; c += kResThreads) w.cand[c] = cand[c];
    for (int b = tid; b < B; b += kResThreads) w.expiry[b] = expiry[b];
    if (tid == 0) {
        w.v0[0] = (unsigned long long)s_v0c;
        w.v0[1] = (unsigned long long)s_v0d;
        gst->t = s_t;
        gst->n_moves = s_nmoves;
        gst->done = s_done;
        gst->err |= s_err;
        gst->cur_cov = s_curc;
        gst->cur_dist = s_curd;
        gst->best_cov = s_bestc;
        gst->best_dist = s_bestd;
        gst->best_iter = s_best_iter;
        gst->mv_s = s_mv_s;
        gst->mv_j = s_mv_j;
    }
}

cudaError_t launch_tabu_resident(const TabuBuffers &w, const int32_t *cost, int nC, int iters, cudaStream_t s)
{
    const size_t with_table = res_bytes_with_table(w.K, w.B, w.M_pad, nC);
    const size_t sm = with_table ? with_table : res_layout(w.K, w.B, w.M_pad, nC).bytes;
    k_tabu_resident<<<1, kResThreads, sm, s>>>(w, cost, iters);
    return cudaGetLastError();
}

cudaError_t launch_export_best_two(const TabuBuffers &w, const int *perm, int32_t *a, int32_t *b,
                                   int32_t *b1, int32_t *b2, cudaStream_t s)
{
    k_export_best_two<<<grid_missions(w.M_pad), 256, 0, s>>>(w, perm, a, b, b1, b2);
    return cudaGetLastError();
}

__global__ void k_group_swap(const GroupSlot *__restrict__ slots, const int2 *__restrict__ map);
__global__ void k_tabu_small(TabuBuffers w, const int32_t *__restrict__ cost, int iters);
__global__ void k_tabu_resident(TabuBuffers w, const int32_t *__restrict__ cost, int iters);

// Function attributes (dynamic shared memory limits) and the SM count, once
// per device: later calls on an initialised device return at once.
cudaError_t kernels_init()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_init_mu);
    if (g_sms_of[dev] > 0) return cudaSuccess;
    e = cudaFuncSetAttribute(k_swap_eval<kSwapJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(STAGE_MAX_K * kSwapJ * 12));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_swap_direct<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)swap_direct_smem(kPipeMaxK));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_swap_direct<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)swap_direct_smem(kPipeMaxK));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_swap_direct<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)swap_direct_smem(kPipeMaxK));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tabu_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)swap_direct_smem(kPipeMaxK));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_group_swap, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)swap_direct_smem(kGroupMaxK));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tabu_resident, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kResMaxSmem);
    if (e != cudaSuccess) return e;
    e = persist_init();
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_sms_of[dev] = n;
    return cudaSuccess;
}


// --------------------------------------------------------------------------
// Grouped launches of the batch engine.  Every active slot is one instance in
// its own Tabu run; one launch of each kernel advances every slot by one step.
// A slot whose search has stopped, or whose iteration budget is used up,
// returns at once.
// --------------------------------------------------------------------------

// seg_override > 0: the batch's common segment (a whole batch fills the GPU
// with far fewer, larger blocks than each instance would want alone).
int group_swap_blocks(int M_pad, int nC, int K, int seg_override, int *bx, int *seg)
{
    *seg = seg_override > 0 ? seg_override : swap_segment_for(M_pad, nC, K);
    *bx = (M_pad + *seg - 1) / *seg;
    return nC > 0 ? *bx * ((nC + kDirJ - 1) / kDirJ) : 0;
}

// The largest power-of-two segment in [1024, 16384] for which the whole batch
// still has two waves of blocks; 0 when even 1024 leaves the GPU short (then
// every slot keeps its own choice).
int group_common_segment(const int *M_pad, const int *nC, int n)
{
    const long long target = 2ll * 4 * sm_count();
    for (int seg = 16384; seg >= 1024; seg >>= 1) {
        long long total = 0;
        for (int k = 0; k < n; k++)
            if (nC[k] > 0) total += (long long)((M_pad[k] + seg - 1) / seg) * ((nC[k] + kDirJ - 1) / kDirJ);
        if (total >= target) return seg;
    }
    return 0;
}

int group_ref_blocks(int M_pad)
{
    const int g = (M_pad + 255) / 256;
    return g < 64 ? g : 64;
}

// Copy one slot descriptor into shared memory, one 4-byte word per thread.
__device__ __forceinline__ void load_slot(const GroupSlot *slots, int slot, GroupSlot &dst)
{
    static_assert(sizeof(GroupSlot) % 4 == 0, "slot descriptor must be word-sized");
    constexpr int words = sizeof(GroupSlot) / 4;
    const int *src = reinterpret_cast<const int *>(slots + slot);
    int *d = reinterpret_cast<int *>(&dst);
    for (int k = threadIdx.x; k < words; k += blockDim.x) d[k] = __ldg(src + k);
    __syncthreads();
}

// map[b] = (slot, block within the slot) for every block of a grouped launch.
__global__ void __launch_bounds__(kDirThreads, 4)
k_group_swap(const GroupSlot *__restrict__ slots, const int2 *__restrict__ map)
{
    __shared__ GroupSlot g;
    const int2 e = map[blockIdx.x];
    load_slot(slots, e.x, g);
    const TabuDevState *st = g.w.st;
    if (st->done || st->t >= st->t_end) return;
    if (g.w.chg && st->n_moves > 0) return;   // incremental slot: its terms are kept by the delta step
    swap_direct_body<kDirJ>(g.w, g.cost, e.y % g.swap_bx, e.y / g.swap_bx, g.swap_seg);
}

cudaError_t launch_group_swap(const GroupSlot *slots, const int2 *map, int total_blocks, size_t smem,
                              cudaStream_t s)
{
    if (total_blocks <= 0) return cudaSuccess;
    k_group_swap<<<total_blocks, kDirThreads, smem, s>>>(slots, map);
    return cudaGetLastError();
}

// out[2k], out[2k + 1] = slot k's V0 (covered, distance): every slot's start
// objective gathered for one read-back.
__global__ void k_group_v0(const GroupSlot *__restrict__ slots, int n, unsigned long long *__restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const unsigned long long *v0 = slots[k].w.v0;
    out[2 * k] = v0[0];
    out[2 * k + 1] = v0[1];
}

cudaError_t launch_group_v0(const GroupSlot *slots, int n, unsigned long long *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_group_v0<<<(n + 127) / 128, 128, 0, s>>>(slots, n, out);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kSelectThreads) k_group_select(const GroupSlot *__restrict__ slots,
                                                                const int2 *__restrict__ map)
{
    __shared__ GroupSlot g;
    const int2 e = map[blockIdx.x];
    load_slot(slots, e.x, g);
    TabuDevState *st = g.w.st;
    if (st->done || st->t >= st->t_end) return;
    select_body(g.w, e.y, g.sel_blocks);
}

cudaError_t launch_group_select(const GroupSlot *slots, const int2 *map, int total_blocks, cudaStream_t s)
{
    if (total_blocks <= 0) return cudaSuccess;
    k_group_select<<<total_blocks, kSelectThreads, 0, s>>>(slots, map);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256, 4) k_group_refresh(const GroupSlot *__restrict__ slots,
                                                          const int2 *__restrict__ map)
{
    __shared__ GroupSlot g;
    const int2 e = map[blockIdx.x];
    load_slot(slots, e.x, g);
    refresh_body(g.w, g.cost, e.y, g.ref_blocks);
}

cudaError_t launch_group_refresh(const GroupSlot *slots, const int2 *map, int total_blocks, int maxK,
                                 cudaStream_t s)
{
    if (total_blocks <= 0) return cudaSuccess;
    k_group_refresh<<<total_blocks, 256, refresh_smem(maxK), s>>>(slots, map);
    return cudaGetLastError();
}

// The incremental slots' update of their kept terms from the missions the
// refresh recorded (the per-search k_swap_delta, one slot's grid per slot).
__global__ void __launch_bounds__(kDeltaRows) k_group_delta(const GroupSlot *__restrict__ slots,
                                                            const int2 *__restrict__ map)
{
    __shared__ GroupSlot g;
    const int2 e = map[blockIdx.x];
    load_slot(slots, e.x, g);
    if (!g.w.chg) return;
    swap_delta_body(g.w, e.y % g.delta_bx, e.y / g.delta_bx, g.delta_by);
}

cudaError_t launch_group_delta(const GroupSlot *slots, const int2 *map, int total_blocks, cudaStream_t s)
{
    if (total_blocks <= 0) return cudaSuccess;
    k_group_delta<<<total_blocks, kDeltaRows, 0, s>>>(slots, map);
    return cudaGetLastError();
}

// Delta grid of one incremental slot in a grouped launch: the copy's
// positions in blocks of kDeltaRows, and the record chunks over blocks sized
// for the records a move can make (known only on the device): a move changes
// the state of about 2 M / K missions (those near the two bases, K bases
// sharing the missions), so about one block per eight chunks of 4 M / K.
void group_delta_blocks(int ldT, int M, int K, int *bx, int *by)
{
    *bx = (ldT + kDeltaRows - 1) / kDeltaRows;
    const long long rec = 4ll * M / (K > 0 ? K : 1);
    long long y = (rec + 8 * kDeltaChunk - 1) / (8 * kDeltaChunk);
    if (y > 256) y = 256;
    *by = y < 1 ? 1 : (int)y;
}

__global__ void k_gather_states(const GroupSlot *__restrict__ slots, int n, TabuDevState *__restrict__ out)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) out[k] = *slots[k].w.st;
}

cudaError_t launch_gather_states(const GroupSlot *slots, int n, TabuDevState *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_gather_states<<<(n + 127) / 128, 128, 0, s>>>(slots, n, out);
    return cudaGetLastError();
}
}  // namespace stg
