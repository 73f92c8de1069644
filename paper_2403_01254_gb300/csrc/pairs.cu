// Candidate search and pair kernel of the hot path.
//
// For every edge (a, b) of the pose graph, every point y_j of frame b is moved
// into frame a (y' = T_ab y, T_ab = T_a^-1 T_b; the relative transform of
// Eq. inner_product_actual_ba written in frame a, where |T_a x - T_b y| =
// |x - T_ab y| because SE(3) acts by isometries) and binned by the frame-a
// grid cell that contains it.  A warp then takes <= 32 queries of one home
// cell and walks the 27 cells around it together: candidates are read once
// per warp (broadcast loads) and each lane tests its own query.  For every
// pair inside r_c the lane forms the weight
//     w = <l_i, l_j> * k_c(c_i, c_j) * exp(-|d|^2 / (2 ell^2))      Eq. (irls_weight)
// and accumulates W = sum w, D = sum w d, Q = sum w d d^T with d = x - y'.
// Per query these become the 28 edge moments (see common.cuh) in frame-a
// coordinates, which fix the loss, the gradient of Eq. (inner_product_reformat)
// and the Gauss-Newton blocks of Eq. (irls_final) exactly.
//
// Every per-query contribution is rounded to 64-bit fixed point (power-of-two
// scale per moment class and edge) before any cross-query sum, so the edge
// totals are exact integer sums: independent of the order in which warps run,
// of the binning order and of which other problems share the launch.
#include "common.cuh"

namespace rk {

namespace {
constexpr unsigned FULL = 0xffffffffu;

__global__ void k_edge_setup(const double* __restrict__ poses, const EdgeDev* __restrict__ edges,
                             int E, EdgeXf* __restrict__ xf, const int* done) {
    if (done && *done) return;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const double* Ta = poses + 16 * edges[e].a;
    const double* Tb = poses + 16 * edges[e].b;
    EdgeXf X;
    // R_ab = R_a^T R_b,  t_ab = R_a^T (t_b - t_a)
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Ta[4 * k + r] * Tb[4 * k + c];
            X.R[3 * r + c] = s;
            X.Rf[3 * r + c] = (float)s;
        }
    double dt[3] = {Tb[3] - Ta[3], Tb[7] - Ta[7], Tb[11] - Ta[11]};
    for (int r = 0; r < 3; ++r) X.t[r] = Ta[r] * dt[0] + Ta[4 + r] * dt[1] + Ta[8 + r] * dt[2];
    xf[e] = X;
}

__device__ __forceinline__ int find_edge_wi(const EdgeDev* __restrict__ edges, int E, long long it) {
    int lo = 0, hi = E - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (edges[mid].wi_off <= it) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_edge_bin(const EdgeDev* __restrict__ edges, int E, long long bin) {
    int lo = 0, hi = E - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (edges[mid].bin_off <= bin) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One warp per (edge, occupied cell of frame b).  Lane 0 moves the cell centre
// into frame a in FP64 and splits it into an integer cell K and an FP32
// remainder F; each lane then moves its points in FP32 relative to K, so no
// large coordinate ever enters FP32 arithmetic.
template <int PASS>
__global__ void __launch_bounds__(256) k_bin(const EdgeDev* __restrict__ edges, int E,
                                             const FrameDev* __restrict__ frames,
                                             const EdgeXf* __restrict__ xf,
                                             const long long* __restrict__ occ_key,
                                             const int* __restrict__ cell_start,
                                             const float4* __restrict__ pts4, GridParams gp,
                                             int* __restrict__ bin_count,
                                             const long long* __restrict__ bin_packed,
                                             int* __restrict__ bin_cursor, Slot* __restrict__ slots,
                                             long long n_items, const int* done) {
    if (done && *done) return;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long it = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < n_items;
         it += nwarps) {
        const int e = find_edge_wi(edges, E, it);
        const EdgeDev& Ed = edges[e];
        const FrameDev& Fa = frames[Ed.a];
        const FrameDev& Fb = frames[Ed.b];
        const long long key = occ_key[Fb.occ_off + (it - Ed.wi_off)];
        const int beg = cell_start[key], end = cell_start[key + 1];
        int Kx = 0, Ky = 0, Kz = 0;
        float Fx = 0.f, Fy = 0.f, Fz = 0.f;
        if (lane == 0) {
            long long loc = key - Fb.cell_off;
            int cx = (int)(loc % Fb.dim[0]);
            long long r = loc / Fb.dim[0];
            int cy = (int)(r % Fb.dim[1]);
            int cz = (int)(r / Fb.dim[1]);
            double o[3] = {((double)(cx + Fb.lo[0]) + 0.5) * gp.h, ((double)(cy + Fb.lo[1]) + 0.5) * gp.h,
                           ((double)(cz + Fb.lo[2]) + 0.5) * gp.h};
            const EdgeXf& X = xf[e];
            double P[3];
            for (int k = 0; k < 3; ++k)
                P[k] = fma(X.R[3 * k + 2], o[2], fma(X.R[3 * k + 1], o[1], fma(X.R[3 * k], o[0], X.t[k])));
            double Kd[3];
            // clamp keeps the int conversion defined for any pose; a clamped
            // cell lies far outside every grid and is dropped below
            for (int k = 0; k < 3; ++k) Kd[k] = fmin(fmax(floor(P[k] * gp.h_inv), -1073741824.0), 1073741824.0);
            Kx = (int)Kd[0]; Ky = (int)Kd[1]; Kz = (int)Kd[2];
            Fx = (float)(P[0] - (Kd[0] + 0.5) * gp.h);
            Fy = (float)(P[1] - (Kd[1] + 0.5) * gp.h);
            Fz = (float)(P[2] - (Kd[2] + 0.5) * gp.h);
        }
        Kx = __shfl_sync(FULL, Kx, 0); Ky = __shfl_sync(FULL, Ky, 0); Kz = __shfl_sync(FULL, Kz, 0);
        Fx = __shfl_sync(FULL, Fx, 0); Fy = __shfl_sync(FULL, Fy, 0); Fz = __shfl_sync(FULL, Fz, 0);
        const float* R = xf[e].Rf;
        const float r0 = R[0], r1 = R[1], r2 = R[2], r3 = R[3], r4 = R[4], r5 = R[5], r6 = R[6],
                    r7 = R[7], r8 = R[8];
        for (int s = beg + lane; s < end; s += 32) {
            const float4 p = pts4[s];
            const float vx = fmaf(r2, p.z, fmaf(r1, p.y, fmaf(r0, p.x, Fx)));
            const float vy = fmaf(r5, p.z, fmaf(r4, p.y, fmaf(r3, p.x, Fy)));
            const float vz = fmaf(r8, p.z, fmaf(r7, p.y, fmaf(r6, p.x, Fz)));
            const float mx = floorf(fmaf(vx, gp.hf_inv, 0.5f));
            const float my = floorf(fmaf(vy, gp.hf_inv, 0.5f));
            const float mz = floorf(fmaf(vz, gp.hf_inv, 0.5f));
            const int hx = Kx + (int)mx - Fa.lo[0];
            const int hy = Ky + (int)my - Fa.lo[1];
            const int hz = Kz + (int)mz - Fa.lo[2];
            if (hx < 0 || hy < 0 || hz < 0 || hx >= Fa.dim[0] || hy >= Fa.dim[1] || hz >= Fa.dim[2])
                continue;   // no frame-a point within one cell: no neighbour possible
            const long long bin = Ed.bin_off + ((long long)hz * Fa.dim[1] + hy) * Fa.dim[0] + hx;
            if (PASS == 0) {
                atomicAdd(&bin_count[bin], 1);
            } else {
                const int qstart = (int)(bin_packed[bin] & 0xffffffffLL);
                const int r = atomicAdd(&bin_cursor[bin], 1);
                if (r >= bin_count[bin]) continue;   // never past the counted range
                const int pos = qstart + r;
                Slot q;
                q.s = s;
                q.vx = fmaf(-mx, gp.hf, vx);
                q.vy = fmaf(-my, gp.hf, vy);
                q.vz = fmaf(-mz, gp.hf, vz);
                slots[pos] = q;
            }
        }
    }
}

// count -> packed (count | warp tasks << 32) for one scan of both prefix sums
__global__ void k_make_bins(const int* __restrict__ cnt, long long* __restrict__ val, long long n,
                            const int* done) {
    if (done && *done) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        long long c = cnt[i];
        val[i] = c | (((c + 31) >> 5) << 32);
    }
}

__global__ void k_emit_tasks(const int* __restrict__ cnt, const long long* __restrict__ packed,
                             const EdgeDev* __restrict__ edges, int E, long long n_bins,
                             const long long* __restrict__ total, Task* __restrict__ tasks,
                             int* __restrict__ n_tasks, const int* done) {
    if (done && *done) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_tasks = (int)(*total >> 32);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_bins;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = cnt[i];
        if (c == 0) continue;
        const long long p = packed[i];
        const int qs = (int)(p & 0xffffffffLL);
        const int ts = (int)(p >> 32);
        const int e = find_edge_bin(edges, E, i);
        const int cell = (int)(i - edges[e].bin_off);
        for (int k = 0; 32 * k < c; ++k) {
            Task t;
            t.edge = e;
            t.cell = cell;
            t.qstart = qs + 32 * k;
            t.qcount = min(32, c - 32 * k);
            tasks[ts + k] = t;
        }
    }
}

__device__ __forceinline__ long long to_fixed(float v, float scale) { return __float2ll_rn(v * scale); }

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

template <int DP, bool BF16>
struct Sem;

template <int DP>
struct Sem<DP, false> {   // FP32 rows of DP floats
    float q[DP > 0 ? DP : 1];
    __device__ __forceinline__ void load(const void* base, int s, bool valid) {
        const float4* row = reinterpret_cast<const float4*>(base) + (size_t)s * (DP / 4);
#pragma unroll
        for (int k = 0; k < DP / 4; ++k) {
            float4 v = valid ? __ldg(row + k) : make_float4(0.f, 0.f, 0.f, 0.f);
            q[4 * k] = v.x; q[4 * k + 1] = v.y; q[4 * k + 2] = v.z; q[4 * k + 3] = v.w;
        }
    }
    __device__ __forceinline__ float dot(const void* base, int i) const {
        if (DP == 0) return 1.f;
        const float4* row = reinterpret_cast<const float4*>(base) + (size_t)i * (DP / 4);
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int k = 0; k < DP / 4; ++k) {
            float4 v = __ldg(row + k);
            s0 = fmaf(q[4 * k], v.x, s0);
            s1 = fmaf(q[4 * k + 1], v.y, s1);
            s0 = fmaf(q[4 * k + 2], v.z, s0);
            s1 = fmaf(q[4 * k + 3], v.w, s1);
        }
        return s0 + s1;
    }
};

__device__ __forceinline__ float bf_lo(unsigned u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(unsigned u) { return __uint_as_float(u & 0xffff0000u); }

template <int DP>
struct Sem<DP, true> {    // BF16 rows of DP values (DP % 8 == 0), FP32 products
    float q[DP];
    __device__ __forceinline__ void load(const void* base, int s, bool valid) {
        const uint4* row = reinterpret_cast<const uint4*>(base) + (size_t)s * (DP / 8);
#pragma unroll
        for (int k = 0; k < DP / 8; ++k) {
            uint4 v = valid ? __ldg(row + k) : make_uint4(0u, 0u, 0u, 0u);
            q[8 * k + 0] = bf_lo(v.x); q[8 * k + 1] = bf_hi(v.x);
            q[8 * k + 2] = bf_lo(v.y); q[8 * k + 3] = bf_hi(v.y);
            q[8 * k + 4] = bf_lo(v.z); q[8 * k + 5] = bf_hi(v.z);
            q[8 * k + 6] = bf_lo(v.w); q[8 * k + 7] = bf_hi(v.w);
        }
    }
    __device__ __forceinline__ float dot(const void* base, int i) const {
        const uint4* row = reinterpret_cast<const uint4*>(base) + (size_t)i * (DP / 8);
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int k = 0; k < DP / 8; ++k) {
            uint4 v = __ldg(row + k);
            s0 = fmaf(q[8 * k + 0], bf_lo(v.x), s0); s1 = fmaf(q[8 * k + 1], bf_hi(v.x), s1);
            s0 = fmaf(q[8 * k + 2], bf_lo(v.y), s0); s1 = fmaf(q[8 * k + 3], bf_hi(v.y), s1);
            s0 = fmaf(q[8 * k + 4], bf_lo(v.z), s0); s1 = fmaf(q[8 * k + 5], bf_hi(v.z), s1);
            s0 = fmaf(q[8 * k + 6], bf_lo(v.w), s0); s1 = fmaf(q[8 * k + 7], bf_hi(v.w), s1);
        }
        return s0 + s1;
    }
};

constexpr int PAIR_T = 256;

template <int DP, bool BF16, bool COLOR>
__global__ void __launch_bounds__(PAIR_T, 2)
k_pairs(const Task* __restrict__ tasks, const int* __restrict__ n_tasks, int* task_counter,
        const Slot* __restrict__ slots, const EdgeDev* __restrict__ edges,
        const FrameDev* __restrict__ frames, const int* __restrict__ cell_start,
        const float4* __restrict__ pts4, const void* __restrict__ sem_sorted,
        const float4* __restrict__ col4, GridParams gp, long long* __restrict__ acc, const int* done) {
    if (done && *done) return;
    const int lane = threadIdx.x & 31;
    const int ntask = *n_tasks;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(task_counter, 1);
        t = __shfl_sync(FULL, t, 0);
        if (t >= ntask) break;
        const Task T = tasks[t];
        const EdgeDev& Ed = edges[T.edge];
        const FrameDev& Fa = frames[Ed.a];
        const int dx0 = Fa.dim[0], dy0 = Fa.dim[1], dz0 = Fa.dim[2];
        const long long coff = Fa.cell_off;
        const bool valid = lane < T.qcount;
        Slot q;
        if (valid) q = slots[T.qstart + lane];
        else { q.s = 0; q.vx = q.vy = q.vz = 0.f; }
        Sem<DP, BF16> qs;
        if (DP > 0) qs.load(sem_sorted, q.s, valid);
        float4 qc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (COLOR && valid) qc = col4[q.s];
        const int hx = T.cell % dx0;
        const int hy = (T.cell / dx0) % dy0;
        const int hz = T.cell / (dx0 * dy0);

        float W = 0.f, Dx = 0.f, Dy = 0.f, Dz = 0.f;
        float Qxx = 0.f, Qxy = 0.f, Qxz = 0.f, Qyy = 0.f, Qyz = 0.f, Qzz = 0.f;
        int cnt = 0;
        for (int dz = -1; dz <= 1; ++dz) {
            const int nz = hz + dz;
            if (nz < 0 || nz >= dz0) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                const int ny = hy + dy;
                if (ny < 0 || ny >= dy0) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int nx = hx + dx;
                    if (nx < 0 || nx >= dx0) continue;
                    const long long g = coff + ((long long)nz * dy0 + ny) * dx0 + nx;
                    const int beg = cell_start[g], end = cell_start[g + 1];
                    // query relative to the centre of the neighbour cell
                    const float qx = fmaf(-(float)dx, gp.hf, q.vx);
                    const float qy = fmaf(-(float)dy, gp.hf, q.vy);
                    const float qz = fmaf(-(float)dz, gp.hf, q.vz);
                    for (int i = beg; i < end; ++i) {
                        const float4 p = __ldg(pts4 + i);
                        const float ex = p.x - qx, ey = p.y - qy, ez = p.z - qz;
                        const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                        if (valid && d2 < gp.rc2) {
                            float arg = d2 * gp.kg;
                            if (COLOR) {
                                const float4 c = __ldg(col4 + i);
                                const float cr = c.x - qc.x, cg = c.y - qc.y, cb = c.z - qc.z;
                                arg = fmaf(fmaf(cr, cr, fmaf(cg, cg, cb * cb)), gp.kc, arg);
                            }
                            const float k = exp2f(arg);
                            const float s = (DP > 0) ? qs.dot(sem_sorted, i) : 1.f;
                            const float w = s * k;
                            const float wx = w * ex, wy = w * ey, wz = w * ez;
                            W += w;
                            Dx += wx; Dy += wy; Dz += wz;
                            Qxx = fmaf(wx, ex, Qxx); Qxy = fmaf(wx, ey, Qxy); Qxz = fmaf(wx, ez, Qxz);
                            Qyy = fmaf(wy, ey, Qyy); Qyz = fmaf(wy, ez, Qyz); Qzz = fmaf(wz, ez, Qzz);
                            ++cnt;
                        }
                    }
                }
            }
        }
        // query position y' in frame-a coordinates
        const float yx = fmaf((float)(hx + Fa.lo[0]) + 0.5f, gp.hf, q.vx);
        const float yy = fmaf((float)(hy + Fa.lo[1]) + 0.5f, gp.hf, q.vy);
        const float yz = fmaf((float)(hz + Fa.lo[2]) + 0.5f, gp.hf, q.vz);
        const float Wx = W * yx, Wy = W * yy, Wz = W * yz;
        const float* sc = Ed.scale;
        long long v[N_MOM];
        v[0] = to_fixed(W, sc[MC_W]);
        v[1] = to_fixed(Dx, sc[MC_D]); v[2] = to_fixed(Dy, sc[MC_D]); v[3] = to_fixed(Dz, sc[MC_D]);
        v[4] = to_fixed(Wx, sc[MC_SY]); v[5] = to_fixed(Wy, sc[MC_SY]); v[6] = to_fixed(Wz, sc[MC_SY]);
        v[7] = to_fixed(Wx * yx, sc[MC_MYY]); v[8] = to_fixed(Wx * yy, sc[MC_MYY]);
        v[9] = to_fixed(Wx * yz, sc[MC_MYY]); v[10] = to_fixed(Wy * yy, sc[MC_MYY]);
        v[11] = to_fixed(Wy * yz, sc[MC_MYY]); v[12] = to_fixed(Wz * yz, sc[MC_MYY]);
        v[13] = to_fixed(Dx * yx, sc[MC_MDY]); v[14] = to_fixed(Dx * yy, sc[MC_MDY]);
        v[15] = to_fixed(Dx * yz, sc[MC_MDY]); v[16] = to_fixed(Dy * yx, sc[MC_MDY]);
        v[17] = to_fixed(Dy * yy, sc[MC_MDY]); v[18] = to_fixed(Dy * yz, sc[MC_MDY]);
        v[19] = to_fixed(Dz * yx, sc[MC_MDY]); v[20] = to_fixed(Dz * yy, sc[MC_MDY]);
        v[21] = to_fixed(Dz * yz, sc[MC_MDY]);
        v[22] = to_fixed(Qxx, sc[MC_Q]); v[23] = to_fixed(Qxy, sc[MC_Q]); v[24] = to_fixed(Qxz, sc[MC_Q]);
        v[25] = to_fixed(Qyy, sc[MC_Q]); v[26] = to_fixed(Qyz, sc[MC_Q]); v[27] = to_fixed(Qzz, sc[MC_Q]);
        v[28] = cnt;
        long long* dst = acc + (long long)T.edge * ACC_N;
#pragma unroll
        for (int k = 0; k < N_MOM; ++k) {
            const long long tot = warp_sum_ll(v[k]);
            if (lane == k && tot != 0) atomicAdd(reinterpret_cast<unsigned long long*>(dst + k),
                                                 (unsigned long long)tot);
        }
    }
}

// Same search, geometry only: writes the pair list of one edge (verification).
__global__ void __launch_bounds__(PAIR_T)
k_emit_pairs(const Task* __restrict__ tasks, const int* __restrict__ n_tasks, int* task_counter,
             const Slot* __restrict__ slots, const EdgeDev* __restrict__ edges,
             const FrameDev* __restrict__ frames, const int* __restrict__ cell_start,
             const float4* __restrict__ pts4, GridParams gp, int edge_sel,
             const int* __restrict__ perm_local, long long capacity, int* __restrict__ i_out,
             int* __restrict__ j_out, unsigned long long* n_out) {
    const int lane = threadIdx.x & 31;
    const int ntask = *n_tasks;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(task_counter, 1);
        t = __shfl_sync(FULL, t, 0);
        if (t >= ntask) break;
        const Task T = tasks[t];
        if (T.edge != edge_sel) continue;
        const FrameDev& Fa = frames[edges[T.edge].a];
        const int dx0 = Fa.dim[0], dy0 = Fa.dim[1], dz0 = Fa.dim[2];
        const bool valid = lane < T.qcount;
        Slot q;
        if (valid) q = slots[T.qstart + lane];
        else { q.s = 0; q.vx = q.vy = q.vz = 0.f; }
        const int hx = T.cell % dx0, hy = (T.cell / dx0) % dy0, hz = T.cell / (dx0 * dy0);
        const int jq = valid ? perm_local[q.s] : 0;
        for (int dz = -1; dz <= 1; ++dz) {
            const int nz = hz + dz;
            if (nz < 0 || nz >= dz0) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                const int ny = hy + dy;
                if (ny < 0 || ny >= dy0) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int nx = hx + dx;
                    if (nx < 0 || nx >= dx0) continue;
                    const long long g = Fa.cell_off + ((long long)nz * dy0 + ny) * dx0 + nx;
                    const int beg = cell_start[g], end = cell_start[g + 1];
                    const float qx = fmaf(-(float)dx, gp.hf, q.vx);
                    const float qy = fmaf(-(float)dy, gp.hf, q.vy);
                    const float qz = fmaf(-(float)dz, gp.hf, q.vz);
                    for (int i = beg; i < end; ++i) {
                        const float4 p = __ldg(pts4 + i);
                        const float ex = p.x - qx, ey = p.y - qy, ez = p.z - qz;
                        const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                        if (valid && d2 < gp.rc2) {
                            unsigned long long k = atomicAdd(n_out, 1ULL);
                            if ((long long)k < capacity) {
                                i_out[k] = perm_local[i];
                                j_out[k] = jq;
                            }
                        }
                    }
                }
            }
        }
    }
}

inline unsigned blocks_for(long long n, int t) {
    long long b = (n + t - 1) / t;
    if (b < 1) b = 1;
    if (b > 1048560) b = 1048560;
    return (unsigned)b;
}

template <int DP, bool BF16, bool COLOR>
void run_pairs(unsigned grid, cudaStream_t st, const Task* tasks, const int* n_tasks,
               int* task_counter, const Slot* slots, const EdgeDev* edges, const FrameDev* frames,
               const int* cell_start, const float4* pts4, const void* sem, const float4* col4,
               GridParams gp, long long* acc, const int* done) {
    k_pairs<DP, BF16, COLOR><<<grid, PAIR_T, 0, st>>>(tasks, n_tasks, task_counter, slots, edges,
                                                      frames, cell_start, pts4, sem, col4, gp, acc,
                                                      done);
}

template <bool COLOR>
bool dispatch_pairs(unsigned grid, cudaStream_t st, const Task* tasks, const int* n_tasks,
                    int* task_counter, const Slot* slots, const EdgeDev* edges,
                    const FrameDev* frames, const int* cell_start, const float4* pts4,
                    const void* sem, const float4* col4, GridParams gp, long long* acc,
                    const int* done) {
#define RK_P(DPV, BFV) \
    run_pairs<DPV, BFV, COLOR>(grid, st, tasks, n_tasks, task_counter, slots, edges, frames, \
                               cell_start, pts4, sem, col4, gp, acc, done); return true
    if (gp.sem_pad == 0) { RK_P(0, false); }
    if (gp.sem_bf16) {
        switch (gp.sem_pad) {
            case 8: RK_P(8, true);
            case 16: RK_P(16, true);
            case 24: RK_P(24, true);
            case 32: RK_P(32, true);
            default: return false;
        }
    }
    switch (gp.sem_pad) {
        case 4: RK_P(4, false);
        case 8: RK_P(8, false);
        case 12: RK_P(12, false);
        case 16: RK_P(16, false);
        case 20: RK_P(20, false);
        case 24: RK_P(24, false);
        case 32: RK_P(32, false);
        default: return false;
    }
#undef RK_P
}
}  // namespace

void launch_edge_setup(const double* poses, const EdgeDev* edges, int E, EdgeXf* xf,
                       const int* done, cudaStream_t st) {
    k_edge_setup<<<(E + 127) / 128, 128, 0, st>>>(poses, edges, E, xf, done);
    count_launch();
}

void launch_bin(int pass, const EdgeDev* edges, int E, const FrameDev* frames, const EdgeXf* xf,
                const long long* occ_key, const int* cell_start, const float4* pts4, GridParams gp,
                int* bin_count, const long long* bin_packed, int* bin_cursor, Slot* slots,
                long long n_items, const int* done, int num_sms, cudaStream_t st) {
    if (n_items <= 0) return;
    long long want = (n_items + 7) / 8;   // 8 warps per block
    long long cap = (long long)num_sms * 8;
    unsigned grid = (unsigned)(want < cap ? want : cap);
    if (pass == 0)
        k_bin<0><<<grid, 256, 0, st>>>(edges, E, frames, xf, occ_key, cell_start, pts4, gp, bin_count,
                                       bin_packed, bin_cursor, slots, n_items, done);
    else
        k_bin<1><<<grid, 256, 0, st>>>(edges, E, frames, xf, occ_key, cell_start, pts4, gp, bin_count,
                                       bin_packed, bin_cursor, slots, n_items, done);
    count_launch();
}

void launch_make_bins(const int* bin_count, long long* bin_val, long long n_bins, const int* done,
                      cudaStream_t st) {
    if (n_bins <= 0) return;
    k_make_bins<<<blocks_for(n_bins, 256), 256, 0, st>>>(bin_count, bin_val, n_bins, done);
    count_launch();
}

void launch_emit_tasks(const int* bin_count, const long long* bin_packed, const EdgeDev* edges,
                       int E, long long n_bins, const long long* total_packed, Task* tasks,
                       int* n_tasks, const int* done, cudaStream_t st) {
    k_emit_tasks<<<blocks_for(n_bins, 256), 256, 0, st>>>(bin_count, bin_packed, edges, E, n_bins,
                                                          total_packed, tasks, n_tasks, done);
    count_launch();
}

void launch_pairs(const Task* tasks, const int* n_tasks, int* task_counter, const Slot* slots,
                  const EdgeDev* edges, const FrameDev* frames, const int* cell_start,
                  const float4* pts4, const void* sem_sorted, const float4* col4, GridParams gp,
                  long long* acc, const int* done, int num_sms, cudaStream_t st) {
    unsigned grid = (unsigned)(num_sms * 2);
    bool ok = gp.color ? dispatch_pairs<true>(grid, st, tasks, n_tasks, task_counter, slots, edges,
                                              frames, cell_start, pts4, sem_sorted, col4, gp, acc, done)
                       : dispatch_pairs<false>(grid, st, tasks, n_tasks, task_counter, slots, edges,
                                               frames, cell_start, pts4, sem_sorted, col4, gp, acc, done);
    if (ok) count_launch();
}

void launch_emit_pairs(const Task* tasks, const int* n_tasks, int* task_counter, const Slot* slots,
                       const EdgeDev* edges, const FrameDev* frames, const int* cell_start,
                       const float4* pts4, GridParams gp, int edge_sel, const int* perm_local,
                       long long capacity, int* i_out, int* j_out, unsigned long long* n_out,
                       int num_sms, cudaStream_t st) {
    k_emit_pairs<<<num_sms * 2, PAIR_T, 0, st>>>(tasks, n_tasks, task_counter, slots, edges, frames,
                                                 cell_start, pts4, gp, edge_sel, perm_local,
                                                 capacity, i_out, j_out, n_out);
    count_launch();
}

}  // namespace rk
