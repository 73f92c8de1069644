// Grid step of the hot path: per-frame uniform grids over frame-local points.
//
// The paper evaluates the double sum of Eq. (inner_product_actual_ba) only
// over nearby point pairs (Sec. III-B: the sum is sparse because most point
// pairs are far apart) and names GPU voxel hashing as future work.  Here every
// frame gets a dense grid of cells of size h = r_c (1 + 2^-10) over its own
// bounding box plus a one-cell margin; points are sorted by (frame, cell),
// stable in the input order, and stored as FP32 offsets from their cell
// centre.  Because points stay in frame-local coordinates the grid never
// moves with the poses: only the queries of the other frame do.
#include "common.cuh"

#include <cuda_bf16.h>

namespace rk {

namespace {
constexpr int GT = 256;

__device__ __forceinline__ int frame_of(const long long* __restrict__ off, int K, long long g) {
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// floor(x / h) computed as floor(x * h_inv) in FP64; identical in every kernel
__device__ __forceinline__ double cell_q(double x, double h_inv) { return floor(x * h_inv); }

// Cell-coordinate bounds and label-norm maximum per frame, plus input checks.
// A warp whose points all belong to one frame reduces its bounds with
// shuffles and makes one set of atomics; a warp across a frame boundary
// falls back to per-point atomics.
__global__ void k_bbox(const double* __restrict__ xyz, const float* __restrict__ sem,
                       const float* __restrict__ rgb, long long N, int K,
                       const long long* __restrict__ pt_off, int sem_dim, double h_inv,
                       int* cmin, int* cmax, unsigned* sem_norm_bits, int* err) {
    const double lim = 536870912.0;   // 2^29
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long w0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); w0 < N; w0 += stride) {
        const long long g = w0 + lane;
        const bool valid = g < N;
        const int f = valid ? frame_of(pt_off, K, g) : -1;
        int bad = 0;
        int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {(int)0x80000000, (int)0x80000000,
                                                                (int)0x80000000};
        unsigned nrm_bits = 0u;
        if (valid) {
            int c[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                double x = xyz[3 * g + k];
                if (!isfinite(x)) { bad |= 1; c[k] = 0; continue; }
                double q = cell_q(x, h_inv);
                if (!(fabs(q) < lim)) { bad |= 2; c[k] = 0; continue; }
                c[k] = (int)q;
            }
            if (!bad) {
#pragma unroll
                for (int k = 0; k < 3; ++k) lo[k] = hi[k] = c[k];
            }
            if (sem_dim > 0) {
                float s = 0.f;
                for (int k = 0; k < sem_dim; ++k) {
                    float v = sem[g * sem_dim + k];
                    if (!isfinite(v)) bad |= 4;
                    s = fmaf(v, v, s);
                }
                nrm_bits = __float_as_uint(isfinite(s) ? sqrtf(s) : 0.f);
            }
            if (rgb) {
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    if (!isfinite(rgb[3 * g + k])) bad |= 8;
            }
        }
        const int f0 = __shfl_sync(0xffffffffu, f, 0);
        if (__all_sync(0xffffffffu, !valid || f == f0)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
                    hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
                }
                nrm_bits = max(nrm_bits, __shfl_xor_sync(0xffffffffu, nrm_bits, o));
                bad |= __shfl_xor_sync(0xffffffffu, bad, o);
            }
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    if (lo[k] <= hi[k]) {
                        atomicMin(&cmin[3 * f0 + k], lo[k]);
                        atomicMax(&cmax[3 * f0 + k], hi[k]);
                    }
                }
                if (sem_dim > 0) atomicMax(&sem_norm_bits[f0], nrm_bits);
                if (bad) atomicOr(err, bad);
            }
        } else if (valid) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (lo[k] <= hi[k]) {
                    atomicMin(&cmin[3 * f + k], lo[k]);
                    atomicMax(&cmax[3 * f + k], hi[k]);
                }
            }
            if (sem_dim > 0) atomicMax(&sem_norm_bits[f], nrm_bits);
            if (bad) atomicOr(err, bad);
        }
    }
}

__global__ void k_keys(const double* __restrict__ xyz, long long N, int K,
                       const long long* __restrict__ pt_off, const FrameDev* __restrict__ frames,
                       double h_inv, uint32_t* __restrict__ keys, int* __restrict__ vals) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N;
         g += (long long)gridDim.x * blockDim.x) {
        const FrameDev& F = frames[frame_of(pt_off, K, g)];
        int l[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) l[k] = (int)cell_q(xyz[3 * g + k], h_inv) - F.lo[k];
        long long key = F.cell_off + ((long long)l[2] * F.dim[1] + l[1]) * F.dim[0] + l[0];
        keys[g] = (uint32_t)key;
        vals[g] = (int)g;
    }
}

__global__ void k_gather(const double* __restrict__ xyz, const float* __restrict__ sem,
                         const float* __restrict__ rgb, long long N, int K,
                         const long long* __restrict__ pt_off, const uint32_t* __restrict__ keys,
                         const int* __restrict__ perm, GridParams gp, long long C_total,
                         float4* __restrict__ pts4, void* __restrict__ sem_sorted,
                         float4* __restrict__ col4, int* __restrict__ perm_local,
                         int* __restrict__ cell_start, long long* __restrict__ run_flag) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const long long g = perm[s];
        const int f = frame_of(pt_off, K, s);
        float o[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double x = xyz[3 * g + k];
            double ctr = (cell_q(x, gp.h_inv) + 0.5) * gp.h;
            o[k] = (float)(x - ctr);
        }
        pts4[s] = make_float4(o[0], o[1], o[2], 0.f);
        perm_local[s] = (int)(g - pt_off[f]);
        if (gp.sem_pad > 0) {
            if (gp.sem_bf16) {
                __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(sem_sorted) + s * gp.sem_pad;
                for (int k = 0; k < gp.sem_pad; ++k)
                    dst[k] = __float2bfloat16_rn(k < gp.sem_dim ? sem[g * gp.sem_dim + k] : 0.f);
            } else {
                float* dst = reinterpret_cast<float*>(sem_sorted) + s * gp.sem_pad;
                for (int k = 0; k < gp.sem_pad; ++k) dst[k] = k < gp.sem_dim ? sem[g * gp.sem_dim + k] : 0.f;
            }
        }
        if (gp.color) col4[s] = make_float4(rgb[3 * g], rgb[3 * g + 1], rgb[3 * g + 2], 0.f);
        const long long key = keys[s];
        run_flag[s] = ((s == 0) || ((long long)keys[s - 1] != key)) ? 1 : 0;
    }
}

// cell_start[c] = first sorted point whose cell key is >= c, for c in
// [0, C_total] (a lower bound in the sorted keys; empty cells get the start
// of the next occupied one, the end entry N).
__global__ void k_cell_start(const uint32_t* __restrict__ keys, long long N, long long C_total,
                             int* __restrict__ cell_start) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c <= C_total;
         c += (long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = N;
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if ((long long)keys[mid] < c) lo = mid + 1;
            else hi = mid;
        }
        cell_start[c] = (int)lo;
    }
}

inline unsigned grid_for(long long n) {
    long long b = (n + GT - 1) / GT;
    if (b < 1) b = 1;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return (unsigned)b;
}
}  // namespace

void launch_bbox(const double* xyz, const float* sem, const float* rgb, long long N, int K,
                 const long long* pt_off, int sem_dim, double h_inv, int* cmin, int* cmax,
                 unsigned* sem_norm_bits, int* err, cudaStream_t st) {
    if (N <= 0) return;
    k_bbox<<<grid_for(N), GT, 0, st>>>(xyz, sem, rgb, N, K, pt_off, sem_dim, h_inv, cmin, cmax,
                                       sem_norm_bits, err);
    count_launch();
}

void launch_keys(const double* xyz, long long N, int K, const long long* pt_off,
                 const FrameDev* frames, double h_inv, uint32_t* keys, int* vals, cudaStream_t st) {
    if (N <= 0) return;
    k_keys<<<grid_for(N), GT, 0, st>>>(xyz, N, K, pt_off, frames, h_inv, keys, vals);
    count_launch();
}

void launch_gather(const double* xyz, const float* sem, const float* rgb, long long N, int K,
                   const long long* pt_off, const uint32_t* keys, const int* perm, GridParams gp,
                   long long C_total, float4* pts4, void* sem_sorted, float4* col4,
                   int* perm_local, int* cell_start, long long* run_flag, cudaStream_t st) {
    if (N <= 0) return;
    k_gather<<<grid_for(N), GT, 0, st>>>(xyz, sem, rgb, N, K, pt_off, keys, perm, gp, C_total,
                                         pts4, sem_sorted, col4, perm_local, cell_start, run_flag);
    k_cell_start<<<grid_for(C_total + 1), GT, 0, st>>>(keys, N, C_total, cell_start);
    count_launch(2);
}

}  // namespace rk
