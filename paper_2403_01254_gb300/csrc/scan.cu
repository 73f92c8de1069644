// Device-wide exclusive scan (int64) and a stable LSD radix sort (uint32 keys,
// int32 payload).  Both are the plumbing of the grid build (Sec. VI-time
// analysis: the pair sum needs a spatial index; the paper names GPU voxel
// hashing as future work) and of the per-evaluation query binning.
#include "common.cuh"

namespace rk {

namespace {
constexpr int SCAN_T = 512;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_IPT;     // 4096 items per block

constexpr int RAD_T = 256;
constexpr int RAD_IPT = 8;
constexpr int RAD_TILE = RAD_T * RAD_IPT;        // 2048 items per block
constexpr int RAD_WARPS = RAD_T / 32;

__device__ __forceinline__ long long warp_incl_scan(long long v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// exclusive scan of one value per thread over the block; returns the block total
template <int T>
__device__ __forceinline__ long long block_excl_scan(long long v, long long* s_warp, long long& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long inc = warp_incl_scan(v, lane);
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < T / 32 ? s_warp[lane] : 0;
        long long wi = warp_incl_scan(w, lane);
        if (lane < T / 32) s_warp[lane] = wi - w;
        if (lane == 31) s_warp[T / 32] = wi;
    }
    __syncthreads();
    long long res = s_warp[warp] + inc - v;
    total = s_warp[T / 32];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const long long* __restrict__ in, long long n,
                                                        long long* __restrict__ bsum) {
    __shared__ long long s_warp[SCAN_T / 32 + 1];
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    long long s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        long long i = base + (long long)k * SCAN_T + threadIdx.x;
        if (i < n) s += in[i];
    }
    long long tot;
    block_excl_scan<SCAN_T>(s, s_warp, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// single block: exclusive scan of the block sums in place, total to *total
__global__ void __launch_bounds__(1024) k_scan_top(long long* bsum, long long nb, long long* total) {
    __shared__ long long s_warp[1024 / 32 + 1];
    __shared__ long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (long long base = 0; base < nb; base += 1024) {
        long long i = base + threadIdx.x;
        long long v = i < nb ? bsum[i] : 0;
        long long tot;
        long long ex = block_excl_scan<1024>(v, s_warp, tot);
        if (i < nb) bsum[i] = ex + s_carry;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = s_carry;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_down(const long long* in, long long* out, long long n,
                                                      const long long* __restrict__ boff) {
    __shared__ long long tile[SCAN_TILE];
    __shared__ long long s_warp[SCAN_T / 32 + 1];
    const long long base = (long long)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        long long i = base + (long long)k * SCAN_T + threadIdx.x;
        tile[k * SCAN_T + threadIdx.x] = i < n ? in[i] : 0;
    }
    __syncthreads();
    long long loc[SCAN_IPT];
    long long s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        loc[k] = s;
        s += tile[threadIdx.x * SCAN_IPT + k];
    }
    long long tot;
    long long ex = block_excl_scan<SCAN_T>(s, s_warp, tot) + boff[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) tile[threadIdx.x * SCAN_IPT + k] = ex + loc[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        long long i = base + (long long)k * SCAN_T + threadIdx.x;
        if (i < n) out[i] = tile[k * SCAN_T + threadIdx.x];
    }
}

__global__ void __launch_bounds__(RAD_T) k_radix_hist(const uint32_t* __restrict__ keys, long long n,
                                                      int shift, long long* __restrict__ hist, int nb) {
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * RAD_TILE;
#pragma unroll
    for (int k = 0; k < RAD_IPT; ++k) {
        long long i = base + (long long)k * RAD_T + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: items are taken in input order in rounds of 256; inside a
// round the rank of an item among equal digits counts lower lanes of its warp
// (match.any) plus the equal digits of lower warps.
__global__ void __launch_bounds__(RAD_T) k_radix_scatter(const uint32_t* __restrict__ kin,
                                                         const int* __restrict__ vin,
                                                         uint32_t* __restrict__ kout,
                                                         int* __restrict__ vout, long long n, int shift,
                                                         const long long* __restrict__ hist, int nb) {
    __shared__ long long run[256];
    __shared__ int wcnt[RAD_WARPS][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run[threadIdx.x] = hist[(long long)threadIdx.x * nb + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    const long long base = (long long)blockIdx.x * RAD_TILE;
    for (int r = 0; r < RAD_IPT; ++r) {
#pragma unroll
        for (int w = 0; w < RAD_WARPS; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        long long i = base + (long long)r * RAD_T + threadIdx.x;
        bool valid = i < n;
        uint32_t key = valid ? kin[i] : 0u;
        int digit = valid ? (int)((key >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, digit);
        int rank = __popc(peers & lt);
        if (valid && (peers & lt) == 0) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        if (valid) {
            long long off = run[digit] + rank;
            for (int w = 0; w < warp; ++w) off += wcnt[w][digit];
            kout[off] = key;
            vout[off] = vin[i];
        }
        __syncthreads();
        long long add = 0;
#pragma unroll
        for (int w = 0; w < RAD_WARPS; ++w) add += wcnt[w][threadIdx.x];
        run[threadIdx.x] += add;
        __syncthreads();
    }
}
}  // namespace

size_t scan_ws_elems(long long n) {
    long long nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    return (size_t)(nb + 2);
}

void scan_exclusive_i64(const long long* in, long long* out, long long n, long long* total,
                        long long* ws, cudaStream_t st) {
    if (n <= 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(long long), st);
        return;
    }
    long long nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_reduce<<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, ws);
    k_scan_top<<<1, 1024, 0, st>>>(ws, nb, total);
    k_scan_down<<<(unsigned)nb, SCAN_T, 0, st>>>(in, out, n, ws);
    count_launch(3);
}

size_t radix_hist_elems(long long n) {
    long long nb = (n + RAD_TILE - 1) / RAD_TILE;
    return (size_t)(256 * (nb > 0 ? nb : 1));
}

void radix_sort_u32(uint32_t* keys, int* vals, uint32_t* keys_alt, int* vals_alt, long long n,
                    int nbits, long long* hist, long long* ws, cudaStream_t st, bool* in_alt) {
    *in_alt = false;
    if (n <= 0) return;
    const int nb = (int)((n + RAD_TILE - 1) / RAD_TILE);
    uint32_t* ki = keys;
    int* vi = vals;
    uint32_t* ko = keys_alt;
    int* vo = vals_alt;
    for (int shift = 0; shift < nbits; shift += 8) {
        k_radix_hist<<<nb, RAD_T, 0, st>>>(ki, n, shift, hist, nb);
        count_launch();
        scan_exclusive_i64(hist, hist, 256LL * nb, nullptr, ws, st);
        k_radix_scatter<<<nb, RAD_T, 0, st>>>(ki, vi, ko, vo, n, shift, hist, nb);
        count_launch();
        uint32_t* tk = ki; ki = ko; ko = tk;
        int* tv = vi; vi = vo; vo = tv;
        *in_alt = !*in_alt;
    }
}

}  // namespace rk
