// Stable LSD radix sort of uint32 keys with an int32 payload: the plumbing of
// the grid build (points by cell) and of the per-evaluation query binning
// (queries by home cell).  The pair sum needs a spatial index (the paper
// names GPU voxel hashing as future work); this one is rebuilt by sorting.
//
// One counting kernel reads the keys once and histograms every 8-bit digit;
// each pass is then a single kernel ("one sweep"): a block takes the next
// tile of 2048 keys (tiles are handed out in order by an atomic counter),
// ranks its keys stably (match.any inside a warp, per-warp digit counts
// across warps, rounds of 256 keys in input order), publishes its per-digit
// counts, and obtains the counts of all earlier tiles by looking back over
// their published records (decoupled look-back): a record holds a flag
// (aggregate of the tile / inclusive prefix up to the tile) and a count in
// one 64-bit word.  Every wait is bounded; a wait that gives up sets an error
// word and the kernel finishes with what it has.
#include "common.cuh"

#include <vector>

namespace rk {

namespace {
constexpr int RAD_T = 256;
constexpr int RAD_IPT = 8;
constexpr int RAD_TILE = RAD_T * RAD_IPT;        // 2048 keys per tile
constexpr int RAD_WARPS = RAD_T / 32;
constexpr int MAX_PASS = 4;
constexpr unsigned long long ST_AGG = 1ull << 62;      // count = this tile's
constexpr unsigned long long ST_PRE = 2ull << 62;      // count = tiles 0..t inclusive
constexpr unsigned long long ST_CNT = (1ull << 62) - 1ull;
constexpr int SPIN_LIMIT = 1 << 22;         // polls of one look-back wait before it gives up

__global__ void __launch_bounds__(RAD_T) k_radix_counts(const uint32_t* __restrict__ keys, long long n,
                                                        int npass, unsigned long long* __restrict__ counts) {
    __shared__ int c[MAX_PASS][256];
#pragma unroll
    for (int p = 0; p < MAX_PASS; ++p) c[p][threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * RAD_TILE;
#pragma unroll
    for (int k = 0; k < RAD_IPT; ++k) {
        const long long i = base + (long long)k * RAD_T + threadIdx.x;
        if (i < n) {
            const uint32_t key = keys[i];
            for (int p = 0; p < npass; ++p) atomicAdd(&c[p][(key >> (8 * p)) & 255u], 1);
        }
    }
    __syncthreads();
    for (int p = 0; p < npass; ++p)
        if (c[p][threadIdx.x]) atomicAdd(&counts[256 * p + threadIdx.x], (unsigned long long)c[p][threadIdx.x]);
}

// exclusive scan of one value per thread over a 256-thread block
__device__ __forceinline__ long long block_excl_scan256(long long v, long long* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    long long before = 0;
    for (int w = 0; w < warp; ++w) before += s_warp[w];
    __syncthreads();
    return before + inc - v;
}

__global__ void __launch_bounds__(RAD_T) k_onesweep(const uint32_t* __restrict__ kin,
                                                    const int* __restrict__ vin,
                                                    uint32_t* __restrict__ kout, int* __restrict__ vout,
                                                    long long n, int shift,
                                                    const unsigned long long* __restrict__ counts,
                                                    unsigned long long* status, int* tile_ctr, int* err,
                                                    int spin_limit) {
    __shared__ int s_tile;
    __shared__ int run[256];
    __shared__ int wcnt[RAD_WARPS][256];
    __shared__ long long s_base[256];
    __shared__ long long s_warp[RAD_WARPS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(tile_ctr, 1);
    run[tid] = 0;
#pragma unroll
    for (int w = 0; w < RAD_WARPS; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    const int t = s_tile;
    const long long base = (long long)t * RAD_TILE;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t key[RAD_IPT];
    int val[RAD_IPT], dig[RAD_IPT], rank[RAD_IPT];
    // all loads of the tile first (independent), then the ranking rounds
#pragma unroll
    for (int r = 0; r < RAD_IPT; ++r) {
        const long long i = base + (long long)r * RAD_T + tid;
        key[r] = i < n ? kin[i] : 0u;
        val[r] = i < n ? vin[i] : 0;
    }
    // stable ranks inside the tile: round r holds keys base + 256 r + tid
#pragma unroll
    for (int r = 0; r < RAD_IPT; ++r) {
        const long long i = base + (long long)r * RAD_T + tid;
        const bool valid = i < n;
        const int d = valid ? (int)((key[r] >> shift) & 255u) : 256;
        dig[r] = d;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int lr = __popc(peers & lt);
        if (valid && lr == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        rank[r] = 0;
        if (valid) {
            int off = run[d] + lr;
            for (int w = 0; w < warp; ++w) off += wcnt[w][d];
            rank[r] = off;
        }
        __syncthreads();
        int add = 0;
#pragma unroll
        for (int w = 0; w < RAD_WARPS; ++w) {
            add += wcnt[w][tid];
            wcnt[w][tid] = 0;
        }
        run[tid] += add;
        __syncthreads();
    }
    // publish this tile's count of digit tid, then look back for the prefix
    const int d = tid;
    const long long cnt = run[d];
    volatile unsigned long long* st = status + (long long)t * 256 + d;
    long long excl = 0;
    if (t == 0) {
        *st = ST_PRE | (unsigned long long)cnt;
    } else {
        *st = ST_AGG | (unsigned long long)cnt;
        bool gave_up = false;
        for (int p = t - 1; p >= 0 && !gave_up; --p) {
            volatile unsigned long long* sp = status + (long long)p * 256 + d;
            unsigned long long v = *sp;
            int spins = 0;
            while ((v >> 62) == 0ull) {
                if (++spins > spin_limit) {   // give up: the prefix stays short, writes stay in bounds
                    atomicOr(err, 1);
                    gave_up = true;
                    break;
                }
                __nanosleep(32);
                v = *sp;
            }
            excl += (long long)(v & ST_CNT);
            if ((v >> 62) == 2ull) break;
        }
        *st = ST_PRE | (unsigned long long)(excl + cnt);
    }
    s_base[d] = block_excl_scan256((long long)counts[d], s_warp) + excl;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RAD_IPT; ++r) {
        const long long i = base + (long long)r * RAD_T + tid;
        if (i < n) {
            const long long o = s_base[dig[r]] + rank[r];
            kout[o] = key[r];
            vout[o] = val[r];
        }
    }
}
}  // namespace

size_t scan_ws_elems(long long) { return (size_t)(MAX_PASS * 256 + 2 * MAX_PASS); }

size_t radix_hist_elems(long long n) {
    const long long nb = (n + RAD_TILE - 1) / RAD_TILE;
    return (size_t)(MAX_PASS * 256 * (nb > 0 ? nb : 1));
}

void radix_sort_u32(uint32_t* keys, int* vals, uint32_t* keys_alt, int* vals_alt, long long n,
                    int nbits, long long* hist, long long* ws, int* err, cudaStream_t st, bool* in_alt) {
    *in_alt = false;
    if (n <= 0 || nbits <= 0) return;
    const int nb = (int)((n + RAD_TILE - 1) / RAD_TILE);
    const int npass = (nbits + 7) / 8;
    unsigned long long* status = reinterpret_cast<unsigned long long*>(hist);
    unsigned long long* counts = reinterpret_cast<unsigned long long*>(ws);
    int* ctr = reinterpret_cast<int*>(ws + MAX_PASS * 256);
    cudaMemsetAsync(status, 0, sizeof(unsigned long long) * 256 * (size_t)nb * npass, st);
    cudaMemsetAsync(ws, 0, sizeof(long long) * scan_ws_elems(n), st);
    k_radix_counts<<<nb, RAD_T, 0, st>>>(keys, n, npass, counts);
    count_launch();
    uint32_t* ki = keys;
    int* vi = vals;
    uint32_t* ko = keys_alt;
    int* vo = vals_alt;
    for (int p = 0; p < npass; ++p) {
        k_onesweep<<<nb, RAD_T, 0, st>>>(ki, vi, ko, vo, n, 8 * p, counts + 256 * p,
                                         status + (size_t)256 * nb * p, ctr + p, err, SPIN_LIMIT);
        count_launch();
        uint32_t* tk = ki; ki = ko; ko = tk;
        int* tv = vi; vi = vo; vo = tv;
        *in_alt = !*in_alt;
    }
}

}  // namespace rk

// Failure-detection self-test of the look-back's bounded wait (declared in
// include/rkhsba.h).  Two tiles of keys; tile_ctr starts at 1, so the single
// launched block takes tile 1 while the record of tile 0 is never published.
// Every thread of the block then polls a record that stays zero, gives up
// after spin_limit polls, raises the error word and finishes with a short
// prefix (zero): each output index is the digit's base from the global counts
// plus the key's rank inside tile 1, below n, so all writes land inside the
// output arrays.  Guard words on both sides of the outputs are checked.
extern "C" rkhsba_status rkhsba_selftest_lookback_timeout(int32_t spin_limit, int32_t* writes_in_bounds) {
    using namespace rk;
    if (writes_in_bounds) *writes_in_bounds = 0;
    if (spin_limit < 1 || spin_limit > (1 << 20)) {
        set_thread_error("rkhsba_selftest_lookback_timeout: spin_limit must be in [1, 2^20]");
        return RKHSBA_EINVAL;
    }
    const long long n = 2LL * RAD_TILE;
    const long long G = 256;                        // guard words on each side of the outputs
    uint32_t* kin = nullptr;
    uint32_t* kout = nullptr;
    int* vin = nullptr;
    int* vout = nullptr;
    unsigned long long* status = nullptr;
    unsigned long long* counts = nullptr;
    int* ctl = nullptr;                              // [0] tile counter, [1] error word
    auto release = [&] {
        cudaFree(kin); cudaFree(kout); cudaFree(vin); cudaFree(vout);
        cudaFree(status); cudaFree(counts); cudaFree(ctl);
    };
    auto cuda_fail = [&](cudaError_t e) {
        release();
        cudaGetLastError();
        set_thread_error(cudaGetErrorString(e));
        return RKHSBA_ECUDA;
    };
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc(&kin, sizeof(uint32_t) * n)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMalloc(&vin, sizeof(int) * n)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMalloc(&kout, sizeof(uint32_t) * (n + 2 * G))) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMalloc(&vout, sizeof(int) * (n + 2 * G))) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMalloc(&status, sizeof(unsigned long long) * 2 * 256)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMalloc(&counts, sizeof(unsigned long long) * 256)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMalloc(&ctl, sizeof(int) * 2)) != cudaSuccess) return cuda_fail(e);
    std::vector<uint32_t> hk(n);
    std::vector<int> hv(n);
    for (long long i = 0; i < n; ++i) {
        hk[i] = (uint32_t)((unsigned long long)(i + 1) * 2654435761ull);
        hv[i] = (int)i;
    }
    const int ctl0[2] = {1, 0};
    if ((e = cudaMemcpy(kin, hk.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemcpy(vin, hv.data(), sizeof(int) * n, cudaMemcpyHostToDevice)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemset(kout, 0xAB, sizeof(uint32_t) * (n + 2 * G))) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemset(vout, 0xAB, sizeof(int) * (n + 2 * G))) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemset(status, 0, sizeof(unsigned long long) * 2 * 256)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemset(counts, 0, sizeof(unsigned long long) * 256)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemcpy(ctl, ctl0, sizeof(ctl0), cudaMemcpyHostToDevice)) != cudaSuccess) return cuda_fail(e);
    k_radix_counts<<<2, RAD_T>>>(kin, n, 1, counts);
    count_launch();
    k_onesweep<<<1, RAD_T>>>(kin, vin, kout + G, vout + G, n, 0, counts, status, ctl, ctl + 1, spin_limit);
    count_launch();
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
    int ctl1[2] = {0, 0};
    std::vector<uint32_t> gk(n + 2 * G);
    std::vector<int> gv(n + 2 * G);
    if ((e = cudaMemcpy(ctl1, ctl, sizeof(ctl1), cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e);
    if ((e = cudaMemcpy(gk.data(), kout, sizeof(uint32_t) * (n + 2 * G), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e);
    if ((e = cudaMemcpy(gv.data(), vout, sizeof(int) * (n + 2 * G), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e);
    release();
    bool guards = true;
    for (long long i = 0; i < G; ++i) {
        guards = guards && gk[i] == 0xABABABABu && gk[n + G + i] == 0xABABABABu;
        guards = guards && gv[i] == (int)0xABABABABu && gv[n + G + i] == (int)0xABABABABu;
    }
    if (writes_in_bounds) *writes_in_bounds = guards ? 1 : 0;
    if (ctl1[1]) {
        set_thread_error("a bounded wait of the radix sort's look-back gave up (self-test)");
        return RKHSBA_ETIMEOUT;
    }
    set_thread_error("");
    return RKHSBA_OK;
}
