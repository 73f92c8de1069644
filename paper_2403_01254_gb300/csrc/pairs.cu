// Candidate search and pair kernel of the hot path.
//
// For every edge (a, b) of the pose graph the points y_j of frame b are the
// queries: each is moved into frame a (y' = T_ab y, T_ab = T_a^-1 T_b; the
// pair distance of Eq. inner_product_actual_ba written in frame a, since
// |T_a x - T_b y| = |x - T_ab y|) and keyed by the frame-a grid cell holding
// it.  A stable radix sort groups the queries by home cell (order inside a
// cell = frame-b order, so results do not depend on thread timing), and the
// groups are cut into units of <= 32 (or 64) queries.  A warp takes one unit,
// stages its queries in shared memory and streams the candidates of the 27
// surrounding cells, 32 at a time, through a box test against the unit's
// queries.  For every candidate x query pair inside r_c the weight
//     w = <l_i, l_j> * k_c(c_i, c_j) * exp(-|d|^2 / (2 ell^2))      Eq. (irls_weight)
// enters the sums that fix the 28 edge moments (layout in common.cuh), and
// through them the loss, the gradient of Eq. (inner_product_reformat) and the
// Gauss-Newton blocks of Eq. (irls_final).  Two unit bodies do this:
//   * the dense tile unit (no colour, no pruning): every element of the
//     32-candidate x unit tile in MMA fragment layout, label products and
//     per-query moment sums on the tensor cores (see "dense tile path");
//   * the bit-walk unit (colour, semantic pruning): lane = candidate, a bit
//     mask of its pairs inside r_c, each lane walking its own set bits and
//     folding W = sum w, D = sum w d, Q = sum w d d^T (d = x - y') per
//     candidate.
// Each lane's moments are rounded to 64-bit fixed point before any
// cross-lane sum, so edge totals are exact integer sums, independent of which
// warp ran which unit.
//
// No FP64 arithmetic runs per query: the frame-a position of a frame-b cell
// centre comes from a per-edge affine map held as double-float pairs, evaluated
// with error-free transformations (Dekker product, Knuth sum) on the FP32 pipe.
#include "common.cuh"

#include <type_traits>

namespace rk {

namespace {
constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t NO_KEY = 0xffffffffu;

// ---------------------------------------------------------- double-float --
struct df { float hi, lo; };

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ df df_add(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + a.lo + b.lo);
}
// (hi + lo) * c for a float c holding a small integer or half-integer
__device__ __forceinline__ df df_mul_f(float hi, float lo, float c) {
    const float p = hi * c;
    const float e = fmaf(hi, c, -p);
    return fast_two_sum(p, fmaf(lo, c, e));
}

__global__ void k_edge_setup(const double* __restrict__ poses, const EdgeDev* __restrict__ edges,
                             int E, const FrameDev* __restrict__ frames, double h,
                             EdgeXf* __restrict__ xf, const int* done) {
    if (done && *done) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const double* Ta = poses + 16 * edges[e].a;
    const double* Tb = poses + 16 * edges[e].b;
    const FrameDev& Fb = frames[edges[e].b];
    EdgeXf X;
    // R_ab = R_a^T R_b,  t_ab = R_a^T (t_b - t_a)
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Ta[4 * k + r] * Tb[4 * k + c];
            X.R[3 * r + c] = s;
            X.Rf[3 * r + c] = (float)s;
        }
    const double dt[3] = {Tb[3] - Ta[3], Tb[7] - Ta[7], Tb[11] - Ta[11]};
    for (int r = 0; r < 3; ++r) X.t[r] = Ta[r] * dt[0] + Ta[4 + r] * dt[1] + Ta[8 + r] * dt[2];
    // P(l) = h R l + [R (lo_b + 1/2) h + t]
    for (int r = 0; r < 3; ++r) {
        double B = X.t[r];
        for (int c = 0; c < 3; ++c) {
            const double A = h * X.R[3 * r + c];
            X.Ahi[3 * r + c] = (float)A;
            X.Alo[3 * r + c] = (float)(A - (double)(float)A);
            B += X.R[3 * r + c] * ((double)Fb.lo[c] + 0.5) * h;
        }
        X.Bhi[r] = (float)B;
        X.Blo[r] = (float)(B - (double)(float)B);
    }
    xf[e] = X;
}

__device__ __forceinline__ int find_edge_q(const EdgeDev* __restrict__ edges, int E, long long q) {
    int lo = 0, hi = E - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (edges[mid].q_off <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_edge_bin(const EdgeDev* __restrict__ edges, int E, long long bin) {
    int lo = 0, hi = E - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (edges[mid].bin_off <= bin) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One thread per query: frame-a home cell key and the query's FP32 offset
// from that cell's centre.
__global__ void k_query_keys(const EdgeDev* __restrict__ edges, int E, const FrameDev* __restrict__ frames,
                             const EdgeXf* __restrict__ xf, const uint32_t* __restrict__ pt_cell,
                             const float4* __restrict__ pts4, GridParams gp, long long Q,
                             uint32_t* __restrict__ qkey, int* __restrict__ qval,
                             float4* __restrict__ qrec, const int* done) {
    if (done && *done) return;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < Q;
         q += (long long)gridDim.x * blockDim.x) {
        const int e = find_edge_q(edges, E, q);
        const EdgeDev& Ed = edges[e];
        const FrameDev& Fa = frames[Ed.a];
        const FrameDev& Fb = frames[Ed.b];
        const int s = (int)(Fb.pt_off + (q - Ed.q_off));
        const int l = (int)((long long)pt_cell[s] - Fb.cell_off);
        const float lf[3] = {(float)(l % Fb.dim[0]), (float)((l / Fb.dim[0]) % Fb.dim[1]),
                             (float)(l / (Fb.dim[0] * Fb.dim[1]))};
        const EdgeXf& X = xf[e];
        float K[3], F[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            df P = {X.Bhi[r], X.Blo[r]};
#pragma unroll
            for (int c = 0; c < 3; ++c) P = df_add(P, df_mul_f(X.Ahi[3 * r + c], X.Alo[3 * r + c], lf[c]));
            float k = floorf(P.hi * gp.hf_inv);
            k = fminf(fmaxf(k, -4194304.f), 4194304.f);
            df C = df_mul_f(gp.hf, gp.hf_lo, k + 0.5f);
            df Rm = df_add(P, {-C.hi, -C.lo});
            float f = Rm.hi + Rm.lo;
            if (f < -0.5f * gp.hf) { k -= 1.f; C = df_mul_f(gp.hf, gp.hf_lo, k + 0.5f);
                                     Rm = df_add(P, {-C.hi, -C.lo}); f = Rm.hi + Rm.lo; }
            else if (f >= 0.5f * gp.hf) { k += 1.f; C = df_mul_f(gp.hf, gp.hf_lo, k + 0.5f);
                                          Rm = df_add(P, {-C.hi, -C.lo}); f = Rm.hi + Rm.lo; }
            K[r] = k;
            F[r] = f;
        }
        const float4 p = pts4[s];
        const float* R = X.Rf;
        const float vx = fmaf(R[2], p.z, fmaf(R[1], p.y, fmaf(R[0], p.x, F[0])));
        const float vy = fmaf(R[5], p.z, fmaf(R[4], p.y, fmaf(R[3], p.x, F[1])));
        const float vz = fmaf(R[8], p.z, fmaf(R[7], p.y, fmaf(R[6], p.x, F[2])));
        const float mx = floorf(fmaf(vx, gp.hf_inv, 0.5f));
        const float my = floorf(fmaf(vy, gp.hf_inv, 0.5f));
        const float mz = floorf(fmaf(vz, gp.hf_inv, 0.5f));
        const int hx = (int)(K[0] + mx) - Fa.lo[0];
        const int hy = (int)(K[1] + my) - Fa.lo[1];
        const int hz = (int)(K[2] + mz) - Fa.lo[2];
        const float ox = fmaf(-mx, gp.hf, vx), oy = fmaf(-my, gp.hf, vy), oz = fmaf(-mz, gp.hf, vz);
        uint32_t key = NO_KEY;
        if (hx >= 0 && hy >= 0 && hz >= 0 && hx < Fa.dim[0] && hy < Fa.dim[1] && hz < Fa.dim[2]) {
            key = (uint32_t)(Ed.bin_off + ((long long)hz * Fa.dim[1] + hy) * Fa.dim[0] + hx);
            // with key_sub = 3 the low bits hold the query's octant of its home
            // cell, so a cell's queries sort by octant and a unit's are close
            if (gp.key_sub)
                key = (key << 3) | (ox >= 0.f ? 1u : 0u) | (oy >= 0.f ? 2u : 0u) | (oz >= 0.f ? 4u : 0u);
        }
        qkey[q] = key;
        qval[q] = (int)q;
        qrec[q] = make_float4(ox, oy, oz, __int_as_float(s));
    }
}

// sorted query records, and the first sorted query of every home cell (keys
// >> sub are home-cell keys)
__global__ void k_query_gather(const uint32_t* __restrict__ key, const int* __restrict__ val,
                               const float4* __restrict__ qrec, long long Q, int sub, float4* __restrict__ slots,
                               int* __restrict__ bin_first, const int* done) {
    if (done && *done) return;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < Q;
         k += (long long)gridDim.x * blockDim.x) {
        slots[k] = qrec[val[k]];
        const uint32_t kk = key[k];
        if (kk != NO_KEY && (k == 0 || (key[k - 1] >> sub) != (kk >> sub))) bin_first[kk >> sub] = (int)k;
    }
}

// a unit starts at the first query of a home cell and every uq queries
// after (uq <= 32); one atomic per block reserves the block's slots in the
// unit list
__global__ void __launch_bounds__(256) k_units(const uint32_t* __restrict__ key, const int* __restrict__ bin_first,
                                               long long Q, int uq, int sub, int* __restrict__ unit_start,
                                               int* __restrict__ n_units, const int* done) {
    if (done && *done) return;
    __shared__ int s_cnt[8];
    __shared__ int s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < Q; base += (long long)gridDim.x * blockDim.x) {
        const long long k = base + threadIdx.x;
        bool st = false;
        if (k < Q) {
            const uint32_t kk = key[k];
            st = kk != NO_KEY && ((k - bin_first[kk >> sub]) % uq) == 0;
        }
        const unsigned m = __ballot_sync(FULL, st);
        if (lane == 0) s_cnt[warp] = __popc(m);
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < 8; ++w) { const int c = s_cnt[w]; s_cnt[w] = tot; tot += c; }
            s_base = tot ? atomicAdd(n_units, tot) : 0;
        }
        __syncthreads();
        if (st) unit_start[s_base + s_cnt[warp] + __popc(m & ((1u << lane) - 1u))] = (int)k;
        __syncthreads();
    }
}

// round(v * scale) to the nearest integer (ties to even) as int64, for
// |v * scale| < 2^62, with FP32 adds and integer operations only.  Below 2^22
// adding 2^23 leaves the rounded magnitude in the mantissa bits; from 2^22 up
// the value is m * 2^(e - 150) with a 24-bit mantissa m.
__device__ __forceinline__ long long to_fixed(float v, float scale) {
    const float x = v * scale;
    const int b = __float_as_int(x);
    const int ex = (b >> 23) & 0xff;
    long long mag;
    if (ex < 149) {
        const float t = fabsf(x) + 8388608.0f;
        mag = __float_as_int(t) & 0x7fffff;
    } else {
        const long long m = (b & 0x7fffff) | 0x800000;
        mag = (ex == 149) ? ((m >> 1) + (m & (m >> 1) & 1)) : (m << (ex - 150));
    }
    return b < 0 ? -mag : mag;
}

// ---------------------------------------------------- paired FP32 ops ----
// Two FP32 lanes in one 64-bit register: fma/mul/add .f32x2 issue one
// instruction for two IEEE FP32 operations (each rounded as its scalar form).
typedef unsigned long long u64;
__device__ __forceinline__ u64 f2(float a, float b) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 f2_split(u64 v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 fmul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fadd2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

template <int DP, bool BF16>
struct Sem;

template <int DP>
struct Sem<DP, false> {   // FP32 label row of DP floats, as DP/2 pairs
    u64 q2[DP > 0 ? DP / 2 : 1];
    __device__ __forceinline__ void load(const void* base, int s, bool valid) {
        const ulonglong2* row = reinterpret_cast<const ulonglong2*>(base) + (size_t)s * (DP / 4);
#pragma unroll
        for (int k = 0; k < DP / 4; ++k) {
            const ulonglong2 v = valid ? __ldg(row + k) : make_ulonglong2(0ull, 0ull);
            q2[2 * k] = v.x;
            q2[2 * k + 1] = v.y;
        }
    }
};

__device__ __forceinline__ float bf_lo(unsigned u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(unsigned u) { return __uint_as_float(u & 0xffff0000u); }
__device__ __forceinline__ u64 bf_pair(unsigned u) { return f2(bf_lo(u), bf_hi(u)); }

template <int DP>
struct Sem<DP, true> {    // BF16 label row of DP values (DP % 8 == 0), widened to FP32 pairs
    u64 q2[DP / 2];
    __device__ __forceinline__ void load(const void* base, int s, bool valid) {
        const uint4* row = reinterpret_cast<const uint4*>(base) + (size_t)s * (DP / 8);
#pragma unroll
        for (int k = 0; k < DP / 8; ++k) {
            const uint4 v = valid ? __ldg(row + k) : make_uint4(0u, 0u, 0u, 0u);
            q2[4 * k + 0] = bf_pair(v.x);
            q2[4 * k + 1] = bf_pair(v.y);
            q2[4 * k + 2] = bf_pair(v.z);
            q2[4 * k + 3] = bf_pair(v.w);
        }
    }
};

// Label rows staged in shared memory (FP32 or BF16 rows) and their dot
// product with a row held in registers: even and odd terms summed in the
// two halves of a pair, then added.
template <int DP, bool BF16>
struct SemRow;
template <int DP>
struct SemRow<DP, false> {
    static constexpr int WORDS = DP;          // 32-bit words per row
    __device__ __forceinline__ static void stage(float* dst, const void* base, int i) {
        const float4* src = reinterpret_cast<const float4*>(base) + (size_t)i * (DP / 4);
        float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
        for (int k = 0; k < DP / 4; ++k) d[k] = __ldg(src + k);
    }
    __device__ __forceinline__ static float dot(const Sem<DP, false>& q, const float* row) {
        const ulonglong2* r = reinterpret_cast<const ulonglong2*>(row);
        u64 acc = 0ull;
#pragma unroll
        for (int k = 0; k < DP / 4; ++k) {
            const ulonglong2 v = r[k];
            acc = ffma2(q.q2[2 * k], v.x, acc);
            acc = ffma2(q.q2[2 * k + 1], v.y, acc);
        }
        const float2 s = f2_split(acc);
        return s.x + s.y;
    }
};
template <int DP>
struct SemRow<DP, true> {
    static constexpr int WORDS = DP / 2;
    __device__ __forceinline__ static void stage(float* dst, const void* base, int i) {
        const uint4* src = reinterpret_cast<const uint4*>(base) + (size_t)i * (DP / 8);
        uint4* d = reinterpret_cast<uint4*>(dst);
#pragma unroll
        for (int k = 0; k < DP / 8; ++k) d[k] = __ldg(src + k);
    }
    __device__ __forceinline__ static float dot(const Sem<DP, true>& q, const float* row) {
        const uint4* r = reinterpret_cast<const uint4*>(row);
        u64 acc = 0ull;
#pragma unroll
        for (int k = 0; k < DP / 8; ++k) {
            const uint4 v = r[k];
            acc = ffma2(q.q2[4 * k + 0], bf_pair(v.x), acc);
            acc = ffma2(q.q2[4 * k + 1], bf_pair(v.y), acc);
            acc = ffma2(q.q2[4 * k + 2], bf_pair(v.z), acc);
            acc = ffma2(q.q2[4 * k + 3], bf_pair(v.w), acc);
        }
        const float2 s = f2_split(acc);
        return s.x + s.y;
    }
};
template <>
struct SemRow<0, false> {
    static constexpr int WORDS = 0;
    __device__ __forceinline__ static void stage(float*, const void*, int) {}
    __device__ __forceinline__ static float dot(const Sem<0, false>&, const float*) { return 1.f; }
};


constexpr int PAIR_T = 256;
#ifndef RK_PAIR_MINB
#define RK_PAIR_MINB 2              // resident CTAs per SM the register budget targets
#endif
// Resident CTAs per SM the register budget of a dense tile kernel targets:
// three for BF16 rows of <= 24 values and units of <= 32 queries (75 KB of
// shared memory per CTA, so three fit; 80 registers with a few bytes of
// spills: window workload 1.85 -> 1.73 ms per evaluation), else two (the
// larger layouts fit only two CTAs' shared memory).
template <int DP, bool BF16, int DENSE>
__host__ __device__ constexpr int dense_min_blocks() {
    return (BF16 && DENSE == 1 && DP <= 24) ? 3 : 2;
}
constexpr int UQ = UNIT_Q;          // queries per unit: one 32-bit mask word
static_assert(UQ == 32, "units hold 32 queries");

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Per-warp shared memory, queries kept as m = -2 y and |y|^2 so that the
// cutoff test of a candidate x is |y|^2 - 2 x.y < r_c^2 - |x|^2 (three FMA)
// and d = x - y = x + m/2:
//   walk  [UQ]    float4 (m_x, m_y, m_z, m_x): pairs (m_x, m_y), (m_z, m_x)
//   test  [UQ/2]  8 floats per query pair (j, j+1):
//                 (m_x j, m_x j+1, m_y j, m_y j+1, m_z j, m_z j+1, |y|^2 j, |y|^2 j+1)
//   colours [UQ] float4, labels [UQ][row words], stencil rows [40] ints,
//   per-lane unit sums [32][N_ACC] (kept in shared memory to free registers),
//   candidate queue [CQ_N] float4 (x relative to the home centre, point index),
//   with BF16 labels the batch's label Gram [32 queries][GRAM_LD] floats.
// Per-lane sums over a unit, in this order: W, D (3), Q (6), sum w0 x (3),
// sum w0 x x^T (6), sum x dc^T (9), with w0 = sum w, dc = sum w d of one
// candidate over its queries.
constexpr int N_ACC = 28;
constexpr int CQ_N = 64;            // ring of candidates that survived the unit's box test
constexpr int GRAM_LD = 32;         // row stride (floats) of the BF16 label Gram tile, stored
                                    // [query][candidate]: the walk's lane c reads column c,
                                    // one bank per lane
constexpr int A_W = 0, A_D = 1, A_Q = 4, A_SWX = 10, A_SWXX = 13, A_SXD = 19;

template <int DP, bool BF16, bool COLOR>
__host__ __device__ constexpr int warp_smem_words() {
    return UQ * 4 + UQ * 4 + (COLOR ? UQ * 4 : 0) + UQ * SemRow<DP, BF16>::WORDS + 4 * 10 + 32 * N_ACC +
           4 * CQ_N + ((BF16 && DP > 0) ? 32 * GRAM_LD : 0);
}

struct Rows {
    int* rb;    // [9] first point of the row (three x-adjacent cells)
    int* b1;    // [9] first point of the home-x cell
    int* b2;    // [9] first point of the x+1 cell
    int* pre;   // [10] prefix of row lengths
};

// Rows of the 3x3x3 stencil around home cell (hx, hy, hz): lanes 0..8 fill one
// row each; returns the total candidate count.
__device__ __forceinline__ int build_rows(const Rows& R, const int* __restrict__ cell_start, long long coff,
                                          int dx0, int dy0, int dz0, int hx, int hy, int hz, int lane) {
    int len = 0, rb = 0, b1 = 0, b2 = 0;
    if (lane < 9) {
        const int ny = hy + (lane % 3) - 1, nz = hz + (lane / 3) - 1;
        if (ny >= 0 && ny < dy0 && nz >= 0 && nz < dz0) {
            const long long g0 = coff + ((long long)nz * dy0 + ny) * dx0;
            const int xlo = max(hx - 1, 0), xhi = min(hx + 1, dx0 - 1);
            rb = cell_start[g0 + xlo];
            len = cell_start[g0 + xhi + 1] - rb;
            b1 = cell_start[g0 + hx];
            b2 = cell_start[g0 + hx + 1];
        }
    }
    int inc = len;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const int u = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane < 9) {
        R.rb[lane] = rb;
        R.b1[lane] = b1;
        R.b2[lane] = b2;
        R.pre[lane] = inc - len;
    }
    const int total = __shfl_sync(FULL, inc, 8);
    if (lane == 9) R.pre[9] = total;
    __syncwarp();
    return total;
}

// Candidate v of the unit's stream: point index and offset (dx, dy, dz) of
// its cell from the home cell.
__device__ __forceinline__ int stream_point(const Rows& R, int v, int& dx, int& dy, int& dz) {
    int r = 0;
#pragma unroll
    for (int k = 1; k < 9; ++k) r += (R.pre[k] <= v) ? 1 : 0;
    const int i = R.rb[r] + (v - R.pre[r]);
    dx = (i >= R.b1[r]) + (i >= R.b2[r]) - 1;
    dy = (r % 3) - 1;
    dz = (r / 3) - 1;
    return i;
}

// The same with the row prefix held in registers (pre[0] = 0).
__device__ __forceinline__ int stream_point_r(const Rows& R, const int (&pre)[9], int v, int& dx, int& dy, int& dz) {
    int r = 0;
#pragma unroll
    for (int k = 1; k < 9; ++k) r += (pre[k] <= v) ? 1 : 0;
    int base = pre[0];
#pragma unroll
    for (int k = 1; k < 9; ++k) base = (r == k) ? pre[k] : base;
    const int i = R.rb[r] + (v - base);
    dx = (i >= R.b1[r]) + (i >= R.b2[r]) - 1;
    dy = (r % 3) - 1;
    dz = (r / 3) - 1;
    return i;
}

// Unit header shared by the pair and the pair-list kernels: home cell of the
// unit starting at sorted query k0, and the number of its queries (<= UQ).
__device__ __forceinline__ int unit_queries(const uint32_t* __restrict__ qkey, long long Q, int k0,
                                            uint32_t key0, int lane, int uq, int sub) {
    // units start every uq queries of a home cell, so a unit holds at most uq
    // of them even when the cell continues past k0 + uq
    const long long k1 = (long long)k0 + lane;
    const bool m1 = k1 < Q && (qkey[k1] >> sub) == (key0 >> sub);
    const int n = __popc(__ballot_sync(FULL, m1));
    return n < uq ? n : uq;
}

// The same for units of up to 64 queries (the dense tile unit and the
// pair-list kernel).
__device__ __forceinline__ int unit_queries64(const uint32_t* __restrict__ qkey, long long Q, int k0,
                                              uint32_t key0, int lane, int uq, int sub) {
    int n = unit_queries(qkey, Q, k0, key0, lane, uq, sub);
    if (n == 32 && uq > 32) {
        const long long k1 = (long long)k0 + 32 + lane;
        const bool m1 = k1 < Q && (qkey[k1] >> sub) == (key0 >> sub);
        n = 32 + __popc(__ballot_sync(FULL, m1));
        n = n < uq ? n : uq;
    }
    return n;
}

// One step of the moment reduce-scatter: lanes whose bit `o` is clear keep
// the lower half of their values, the others the upper half, and each adds
// the half its partner sends.
template <int N>
__device__ __forceinline__ void reduce_half(long long (&v)[32], int lane) {
    const bool up = (lane & N) != 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const long long send = up ? v[k] : v[k + N];
        const long long keep = up ? v[k + N] : v[k];
        v[k] = keep + __shfl_xor_sync(FULL, send, N);
    }
}

// Unit end, shared by the pair kernels: the lane's moments about the home
// cell centre move to frame-a coordinates (y' += o), are rounded to 64-bit
// fixed point and reduce-scattered over the warp (lane k ends with the warp
// total of moment k), and added to the edge's accumulators with one integer
// atomic per moment.
__device__ __forceinline__ void store_moments(float W, const float (&Dv)[3], float (&Sy)[3], float (&Myy)[6],
                                              float (&Mdy)[9], const float* Qm, int cnt, const FrameDev& Fa,
                                              int hx, int hy, int hz, const GridParams& gp,
                                              const float* __restrict__ scl, long long* __restrict__ acc_e,
                                              int lane) {
    const float o[3] = {((float)(hx + Fa.lo[0]) + 0.5f) * gp.hf, ((float)(hy + Fa.lo[1]) + 0.5f) * gp.hf,
                        ((float)(hz + Fa.lo[2]) + 0.5f) * gp.hf};
    {
        int t6 = 0;
#pragma unroll
        for (int mm = 0; mm < 3; ++mm)
#pragma unroll
            for (int l = mm; l < 3; ++l, ++t6)
                Myy[t6] += Sy[mm] * o[l] + o[mm] * Sy[l] + W * o[mm] * o[l];
#pragma unroll
        for (int mm = 0; mm < 3; ++mm)
#pragma unroll
            for (int l = 0; l < 3; ++l) Mdy[3 * mm + l] = fmaf(Dv[mm], o[l], Mdy[3 * mm + l]);
#pragma unroll
        for (int mm = 0; mm < 3; ++mm) Sy[mm] = fmaf(W, o[mm], Sy[mm]);
    }
    long long vals[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        float val = 0.f;
        if (k == 0) val = W;
        else if (k < 4) val = Dv[k - 1];
        else if (k < 7) val = Sy[k - 4];
        else if (k < 13) val = Myy[k - 7];
        else if (k < 22) val = Mdy[k - 13];
        else if (k < 28) val = Qm[k - 22];
        vals[k] = (k == N_MOM - 1) ? (long long)cnt
                : (k < N_MOM ? to_fixed(val, __ldg(scl + moment_class(k))) : 0ll);
    }
    reduce_half<16>(vals, lane);
    reduce_half<8>(vals, lane);
    reduce_half<4>(vals, lane);
    reduce_half<2>(vals, lane);
    reduce_half<1>(vals, lane);
    if (lane < N_MOM && vals[0] != 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(acc_e + lane), (unsigned long long)vals[0]);
}

// BF16 labels: the candidate x query label products of a batch come from the
// tensor cores (mma.sync m16n8k16, BF16 in, FP32 accumulate; BF16 products
// are exact in FP32) into a shared-memory tile; the walk reads one float per
// pair instead of forming the dot product.
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Query-side (B) fragments of the Gram MMAs: lane (g, t4) holds words
// 8 ks + t4 and 8 ks + t4 + 4 of query row 8 nt + g; the unit's queries do
// not change from batch to batch, so they are loaded once per unit.
template <int DP>
struct GramB {
    static constexpr int KS = (DP + 15) / 16;   // k16 steps; words beyond DP are zero
    unsigned b[4][KS][2];
    __device__ __forceinline__ void load(const float* ssq, int lane) {
        constexpr int RW = DP / 2;
        const int g = lane >> 2, t4 = lane & 3;
        const unsigned* qw = reinterpret_cast<const unsigned*>(ssq);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int ks = 0; ks < KS; ++ks) {
                const unsigned* qrow = qw + (8 * nt + g) * RW;
                const int w0 = 8 * ks + t4, w1 = w0 + 4;
                b[nt][ks][0] = (w0 < RW) ? qrow[w0] : 0u;
                b[nt][ks][1] = (w1 < RW) ? qrow[w1] : 0u;
            }
    }
};

// Column of candidate c in row q of the Gram tile: XOR-swizzled by q so that
// the MMA fragment stores (four query rows of one candidate per instruction)
// hit 32 different banks.
__device__ __forceinline__ int gram_col(int q, int c) { return c ^ (((q >> 1) & 3) << 3); }

template <int DP>
__device__ __forceinline__ void label_gram_bf16(const unsigned* __restrict__ semw, const GramB<DP>& B, int cand_i,
                                                unsigned has_mask, int lane, float* G) {
    constexpr int KS = GramB<DP>::KS;
    constexpr int RW = DP / 2;           // 32-bit words per label row
    const int g = lane >> 2, t4 = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[mt][nt][k] = 0.f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int r0 = 16 * mt + g, r1 = r0 + 8;                 // candidate rows of this lane
        const int i0 = __shfl_sync(FULL, cand_i, r0), i1 = __shfl_sync(FULL, cand_i, r1);
        const bool v0 = (has_mask >> r0) & 1u, v1 = (has_mask >> r1) & 1u;
        const unsigned* row0 = semw + (size_t)i0 * RW;
        const unsigned* row1 = semw + (size_t)i1 * RW;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            const int w0 = 8 * ks + t4, w1 = w0 + 4;             // words of k = 16 ks + 2 t, + 8
            unsigned a[4];
            a[0] = (v0 && w0 < RW) ? __ldg(row0 + w0) : 0u;
            a[1] = (v1 && w0 < RW) ? __ldg(row1 + w0) : 0u;
            a[2] = (v0 && w1 < RW) ? __ldg(row0 + w1) : 0u;
            a[3] = (v1 && w1 < RW) ? __ldg(row1 + w1) : 0u;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) mma_bf16_16816(acc[mt][nt], a, B.b[nt][ks][0], B.b[nt][ks][1]);
        }
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int c = 16 * mt + g, q = 8 * nt + 2 * t4;      // candidate row, query column
            G[q * GRAM_LD + gram_col(q, c)] = acc[mt][nt][0];
            G[(q + 1) * GRAM_LD + gram_col(q + 1, c)] = acc[mt][nt][1];
            G[q * GRAM_LD + gram_col(q, c + 8)] = acc[mt][nt][2];
            G[(q + 1) * GRAM_LD + gram_col(q + 1, c + 8)] = acc[mt][nt][3];
        }
}

// ------------------------------------------------------ dense tile path ----
// Labels without colour or pruning.  On the LiDAR workloads half to two
// thirds of a batch's candidate x query tests pass the cutoff after the box
// cull, so instead of walking each lane's set bits the warp evaluates the
// whole tile in MMA fragment layout and moves the moment sums onto the tensor
// cores:
//   1. S = L_q L_c^T, the tile's label products (rows are the unit's queries
//      in m tiles of 16, columns the batch's 32 candidates): BF16 labels as
//      stored; FP32 labels scaled by a power of two and split into FP16
//      hi + lo parts, S = hi*hi + hi*lo + lo*hi;
//   2. per element: the exact cutoff test of the bit-walk kernel (same FP32
//      formula, so the same pair set), w = s 2^(kg |d|^2) (one ex2), and 0
//      outside r_c; |d|^2 = |y|^2 - 2 x.y + |x|^2;
//   3. the weights, now an A operand in registers (the accumulator layout of
//      step 1 is the A-fragment layout of the next MMA), split into FP16
//      hi + lo, times the candidate features f(x) = (1, x, x x^T), also
//      split: per query q the sums k_q = sum_c w, X1_q = sum_c w x_c and
//      X2_q = sum_c w x_c x_c^T accumulate over the unit's batches
//      (hi*hi + hi*lo + lo*hi: products of 22-bit operands, FP32 sums,
//      added into FP32 running sums once per batch);
//   4. at the unit's end each lane takes one query and forms, with y = y_q,
//      W = k, D = X1 - k y, sum w y = k y, sum w y y^T = k y y^T,
//      sum w d y^T = D y^T and Q = X2 - X1 y^T - y X1^T + k y y^T, which
//      enter the same fixed-point reduction as the bit-walk kernel.
// Scaling: w is carried as w 2^KW with 2^KW |l|max^2 <= 2^14 and the
// features as x 2^-EX with 2^EX >= h, so every FP16 operand stays inside
// its range; both are powers of two and undone exactly at the unit's end.

// ldmatrix: four / two / one 8x8 b16 matrices from shared memory; lanes
// 8m..8m+7 give the row addresses of matrix m.
__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(unsigned& r0, unsigned& r1, const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(a));
}
__device__ __forceinline__ void ldsm_x1(unsigned& r0, const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x1.shared.b16 {%0}, [%1];" : "=r"(r0) : "r"(a));
}

__device__ __forceinline__ void mma_bf16_1688(float (&d)[4], unsigned a0, unsigned a1, unsigned b0) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}
__device__ __forceinline__ void mma_bf16_16816_r(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                                 unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_f16_16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// (lo, hi) rounded to FP16 (nearest even), lo in the low half
__device__ __forceinline__ unsigned f16x2_rn(float lo, float hi) {
    unsigned r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}
__device__ __forceinline__ float2 f16x2_to_f32(unsigned v) {
    float2 r;
    asm("{\n\t.reg .f16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "r"(v));
    return r;
}
// v0 ~ hi.lo + lo.lo, v1 ~ hi.hi + lo.hi: two FP16 pieces per value (22 bits)
__device__ __forceinline__ void split_f16x2(float v0, float v1, unsigned& hi, unsigned& lo) {
    hi = f16x2_rn(v0, v1);
    const float2 h = f16x2_to_f32(hi);
    lo = f16x2_rn(v0 - h.x, v1 - h.y);
}

// w when t < thr (the pair is inside r_c), counted in cnt; else 0
__device__ __forceinline__ float inside_count(float t, float thr, float w, int& cnt) {
    float r;
    asm("{\n\t.reg .pred p;\n\tsetp.lt.f32 p, %2, %3;\n\tselp.f32 %0, %4, 0f00000000, p;\n\t@p add.s32 %1, %1, 1;\n\t}"
        : "=f"(r), "+r"(cnt) : "f"(t), "f"(thr), "f"(w));
    return r;
}

// Per-warp shared memory of the dense path, in 32-bit words.  Label rows:
// BF16 rows as stored (DP values); FP32 rows (SPLIT) as an FP16 hi part and an
// FP16 lo part of DPH values each (DP rounded up to 8), scaled by a power of two.
template <int DP, bool SPLIT, int MQ = 32>
struct DenseSmem {
    static constexpr int DPH = SPLIT ? ((DP + 7) / 8) * 8 : DP;    // values per part
    static constexpr int PW = DPH / 2;                            // words per part
    static constexpr int RW = SPLIT ? 2 * PW : PW;                // words per staged row
    static constexpr int LW = (RW % 8 == 0) ? RW + 4 : RW;        // row stride: 4 x odd, conflict-free ldmatrix
    static constexpr int MAXQ = SPLIT ? 32 : MQ;                  // queries per unit (m tiles of 16: MAXQ / 16)
    static constexpr int QGW = SPLIT ? 4 : 8;                     // query geometry words:
                                                                  //   (mx mx my my mz mz yy yy) or (mx my mz yy), m = -2y
    static constexpr int QG = 0;                                  // [MAXQ][QGW]
    static constexpr int QL = QG + MAXQ * QGW;                    // [MAXQ][LW] query label rows
    static constexpr int CL = QL + MAXQ * LW;                     // [32][LW] the batch's candidate label rows
    static constexpr int CG = CL + 32 * LW;                       // [16][12] candidate pairs (2p, 2p+1):
                                                                  //   x0 x0' x1 x1' | x2 x2' thr thr' | xk xk' - -
    static constexpr int CF = CG + 16 * 12;                       // [32][16] features: FP16 hi (8 words), lo (8);
                                                                  //   16-byte chunks XOR-swizzled by (c >> 1) & 3;
                                                                  //   at the unit's end [32 queries][16] FP32 sums
    // running per-query sums of the moment MMAs, in the accumulator layout:
    // feature tile 0 as [m tile][lane] float4; feature tile 1 holds only
    // features 8 and 9 (lanes with t4 = 0), as [m tile][g] float4
    static constexpr int RUN = CF + 32 * 16;
    static constexpr int RUN1 = RUN + (MAXQ / 16) * 32 * 4;
    static constexpr int RING = RUN1 + (MAXQ / 16) * 8 * 4;      // [CQ_N] float4 candidate ring
    static constexpr int ROWS = RING + 4 * CQ_N;                  // [40] stencil rows
    static constexpr int WORDS = ROWS + 40;
};

// Stage one label row into shared memory: BF16 rows copied; FP32 rows scaled
// by ls and split into FP16 hi and lo parts (zeros beyond DP); a zero row when
// !valid.
template <int DP, bool SPLIT>
__device__ __forceinline__ void stage_label_row(unsigned* row, const void* base, int i, float ls, bool valid) {
    using L = DenseSmem<DP, SPLIT>;
    uint4* dst = reinterpret_cast<uint4*>(row);
    if constexpr (!SPLIT) {
        const uint4* src = reinterpret_cast<const uint4*>(base) + (size_t)i * (L::PW / 4);
#pragma unroll
        for (int k = 0; k < L::PW / 4; ++k) dst[k] = valid ? __ldg(src + k) : make_uint4(0u, 0u, 0u, 0u);
    } else {
        float v[L::DPH];
        const float4* src = reinterpret_cast<const float4*>(base) + (size_t)i * (DP / 4);
#pragma unroll
        for (int k = 0; k < DP / 4; ++k) {
            const float4 t = valid ? __ldg(src + k) : make_float4(0.f, 0.f, 0.f, 0.f);
            v[4 * k] = t.x * ls;
            v[4 * k + 1] = t.y * ls;
            v[4 * k + 2] = t.z * ls;
            v[4 * k + 3] = t.w * ls;
        }
#pragma unroll
        for (int k = DP; k < L::DPH; ++k) v[k] = 0.f;
        unsigned hw[L::PW], lw[L::PW];
#pragma unroll
        for (int j = 0; j < L::PW; ++j) split_f16x2(v[2 * j], v[2 * j + 1], hw[j], lw[j]);
#pragma unroll
        for (int k = 0; k < L::PW / 4; ++k) {
            dst[k] = make_uint4(hw[4 * k], hw[4 * k + 1], hw[4 * k + 2], hw[4 * k + 3]);
            dst[L::PW / 4 + k] = make_uint4(lw[4 * k], lw[4 * k + 1], lw[4 * k + 2], lw[4 * k + 3]);
        }
    }
}

// The 8-wide chunks [0, NKC) of one part of the staged rows as MMA fragments:
// query side (A, rows 16 mt .. + 15; two registers per chunk) and candidate
// side (B, candidates 8 nt .. + 7; one register per chunk).
template <int NKC>
__device__ __forceinline__ void load_a_chunks(unsigned (&qa)[2 * NKC], const unsigned* rowp) {
    // rowp: this lane's row (16 mt + (lane & 7) + 8 ((lane >> 3) & 1)) at the part's first word
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int kc = 0; kc + 1 < NKC; kc += 2) {
        unsigned r[4];
        ldsm_x4(r, rowp + 4 * (kc + (lane >> 4)));
        qa[2 * kc] = r[0];
        qa[2 * kc + 1] = r[1];
        qa[2 * kc + 2] = r[2];
        qa[2 * kc + 3] = r[3];
    }
    if constexpr (NKC & 1) ldsm_x2(qa[2 * (NKC - 1)], qa[2 * (NKC - 1) + 1], rowp + 4 * (NKC - 1));
}
template <int NKC>
__device__ __forceinline__ void load_b_chunks(unsigned (&cb)[NKC], const unsigned* rowp) {
    // rowp: row of candidate 8 nt + (lane & 7) at the part's first word
    const int lane = threadIdx.x & 31;
    if constexpr (NKC == 4) {
        unsigned r[4];
        ldsm_x4(r, rowp + 4 * (lane >> 3));
#pragma unroll
        for (int k = 0; k < 4; ++k) cb[k] = r[k];
    } else if constexpr (NKC == 3) {
        ldsm_x2(cb[0], cb[1], rowp + 4 * ((lane >> 3) & 1));
        ldsm_x1(cb[2], rowp + 8);
    } else if constexpr (NKC == 2) {
        ldsm_x2(cb[0], cb[1], rowp + 4 * ((lane >> 3) & 1));
    } else {
        ldsm_x1(cb[0], rowp);
    }
}

__device__ __forceinline__ void mma_f16_1688(float (&d)[4], unsigned a0, unsigned a1, unsigned b0) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(b0));
}
__device__ __forceinline__ void mma_f16_16816_r(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                                unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// s += A B over NKC chunks: BF16 (F16 false) or FP16 operands.
template <int NKC, bool F16>
__device__ __forceinline__ void gram_chunks(float (&s)[4], const unsigned (&qa)[2 * NKC], const unsigned (&cb)[NKC]) {
#pragma unroll
    for (int kc = 0; kc + 1 < NKC; kc += 2) {
        if constexpr (F16) mma_f16_16816_r(s, qa[2 * kc], qa[2 * kc + 1], qa[2 * kc + 2], qa[2 * kc + 3], cb[kc], cb[kc + 1]);
        else mma_bf16_16816_r(s, qa[2 * kc], qa[2 * kc + 1], qa[2 * kc + 2], qa[2 * kc + 3], cb[kc], cb[kc + 1]);
    }
    if constexpr (NKC & 1) {
        if constexpr (F16) mma_f16_1688(s, qa[2 * (NKC - 1)], qa[2 * (NKC - 1) + 1], cb[NKC - 1]);
        else mma_bf16_1688(s, qa[2 * (NKC - 1)], qa[2 * (NKC - 1) + 1], cb[NKC - 1]);
    }
}

template <int DP, bool SPLIT, int MQ>
__device__ __forceinline__ void pair_unit_dense(const PairArgs& A, int k0, float* wb, int lane) {
    using L = DenseSmem<DP, SPLIT, MQ>;
    constexpr int LW = L::LW, PW = L::PW;
    constexpr int NKC = L::DPH / 8;             // 8-wide chunks of a label row part (1..4)
    const GridParams& gp = A.gp;
    float* qg = wb + L::QG;
    unsigned* ql = reinterpret_cast<unsigned*>(wb + L::QL);
    unsigned* cl = reinterpret_cast<unsigned*>(wb + L::CL);
    float* cg = wb + L::CG;
    unsigned* cf = reinterpret_cast<unsigned*>(wb + L::CF);
    float4* cq = reinterpret_cast<float4*>(wb + L::RING);
    int* ri = reinterpret_cast<int*>(wb + L::ROWS);
    const Rows R{ri, ri + 9, ri + 18, ri + 27};
    const int g = lane >> 2, t4 = lane & 3;
    const float INF = __int_as_float(0x7f800000);

    const uint32_t kq0 = A.qkey[k0];
    const int qcount = unit_queries64(A.qkey, A.Q, k0, kq0, lane, L::MAXQ < A.uq ? L::MAXQ : A.uq, gp.key_sub);
    const uint32_t key0 = kq0 >> gp.key_sub;
    const int e = find_edge_bin(A.edges, A.E, key0);
    const FrameDev& Fa = A.frames[A.edges[e].a];
    const FrameDev& Fb = A.frames[A.edges[e].b];
    const int dx0 = Fa.dim[0], dy0 = Fa.dim[1], dz0 = Fa.dim[2];
    const int cell = (int)(key0 - A.edges[e].bin_off);
    const int hx = cell % dx0, hy = (cell / dx0) % dy0, hz = cell / (dx0 * dy0);
    // power-of-two scales of the FP16 operands
    int ew, ex;
    frexpf(Fa.sem_norm_max * Fb.sem_norm_max, &ew);
    frexpf(gp.hf, &ex);
    const int KW = min(max(14 - ew, -100), 100);
    // FP32 labels enter the FP16 parts scaled by ls = 2^-el (|l| ls < 1), so
    // the products carry 2^-2el, which the exponent offset undoes
    int el = 0;
    if constexpr (SPLIT) {
        frexpf(fmaxf(Fa.sem_norm_max, Fb.sem_norm_max), &el);
        el = min(max(el, -60), 60);
    }
    const float ls = ldexpf(1.f, -el);
    const float kwf = (float)(KW + 2 * el);
    const float xs = ldexpf(1.f, -ex);
    __syncwarp();
    // stage the unit's queries: geometry, label rows (zero rows for absent
    // queries, whose |y|^2 = inf fails every test), bounding box
    float blo0 = INF, blo1 = INF, blo2 = INF, bhi0 = -INF, bhi1 = -INF, bhi2 = -INF;
#pragma unroll
    for (int h = 0; h < L::MAXQ / 32; ++h) {
        const int q = lane + 32 * h;
        float4* q4 = reinterpret_cast<float4*>(qg) + (L::QGW / 4) * q;
        const bool qv = q < qcount;
        int s = 0;
        if (qv) {
            const float4 r = A.slots[(long long)k0 + q];
            blo0 = fminf(blo0, r.x);
            bhi0 = fmaxf(bhi0, r.x);
            blo1 = fminf(blo1, r.y);
            bhi1 = fmaxf(bhi1, r.y);
            blo2 = fminf(blo2, r.z);
            bhi2 = fmaxf(bhi2, r.z);
            s = __float_as_int(r.w);
            const float mx = -2.f * r.x, my = -2.f * r.y, mz = -2.f * r.z;
            const float yy = fmaf(r.x, r.x, fmaf(r.y, r.y, r.z * r.z));
            if constexpr (SPLIT) {
                q4[0] = make_float4(mx, my, mz, yy);
            } else {
                q4[0] = make_float4(mx, mx, my, my);
                q4[1] = make_float4(mz, mz, yy, yy);
            }
        } else {
            if constexpr (SPLIT) {
                q4[0] = make_float4(0.f, 0.f, 0.f, INF);
            } else {
                q4[0] = make_float4(0.f, 0.f, 0.f, 0.f);
                q4[1] = make_float4(0.f, 0.f, INF, INF);
            }
        }
        stage_label_row<DP, SPLIT>(ql + q * LW, A.sem_sorted, s, ls, qv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        blo0 = fminf(blo0, __shfl_xor_sync(FULL, blo0, o));
        blo1 = fminf(blo1, __shfl_xor_sync(FULL, blo1, o));
        blo2 = fminf(blo2, __shfl_xor_sync(FULL, blo2, o));
        bhi0 = fmaxf(bhi0, __shfl_xor_sync(FULL, bhi0, o));
        bhi1 = fmaxf(bhi1, __shfl_xor_sync(FULL, bhi1, o));
        bhi2 = fmaxf(bhi2, __shfl_xor_sync(FULL, bhi2, o));
    }
    const int C = build_rows(R, A.cell_start, Fa.cell_off, dx0, dy0, dz0, hx, hy, hz, lane);
    const float box_thr = gp.rc2 * 1.0001f;
    const int n_mt = (qcount + 15) >> 4;        // m tiles of 16 queries that hold queries
    const u64 KG2 = f2(gp.kg, gp.kg);
    // this lane's running sums (feature tile 0 for every lane, tile 1 for
    // the lanes holding features 8 and 9), in shared memory
    float4* run0 = reinterpret_cast<float4*>(wb + L::RUN) + lane;       // [mt * 32]
    float4* run1 = reinterpret_cast<float4*>(wb + L::RUN1) + g;         // [mt * 8], t4 == 0
#pragma unroll
    for (int mt = 0; mt < L::MAXQ / 16; ++mt) {
        run0[32 * mt] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t4 == 0) run1[8 * mt] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    int cnt = 0;
    int c_s = 0, qhead = 0, qlen = 0;
    while (c_s < C || qlen > 0) {
        while (qlen < 32 && c_s < C) {
            const int v = c_s + lane;
            bool keep = false;
            float4 ent = make_float4(0.f, 0.f, 0.f, 0.f);
            if (v < C) {
                int dx, dy, dz;
                const int i = stream_point(R, v, dx, dy, dz);
                const float4 p = __ldg(A.pts4 + i);
                ent.x = fmaf((float)dx, gp.hf, p.x);
                ent.y = fmaf((float)dy, gp.hf, p.y);
                ent.z = fmaf((float)dz, gp.hf, p.z);
                ent.w = __int_as_float(i);
                const float e0 = fmaxf(fmaxf(blo0 - ent.x, ent.x - bhi0), 0.f);
                const float e1 = fmaxf(fmaxf(blo1 - ent.y, ent.y - bhi1), 0.f);
                const float e2 = fmaxf(fmaxf(blo2 - ent.z, ent.z - bhi2), 0.f);
                keep = fmaf(e0, e0, fmaf(e1, e1, e2 * e2)) < box_thr;
            }
            const unsigned bal = __ballot_sync(FULL, keep);
            if (keep) cq[(qhead + qlen + __popc(bal & ((1u << lane) - 1u))) & (CQ_N - 1)] = ent;
            qlen += __popc(bal);
            c_s += 32;
        }
        __syncwarp();
        const int nb = qlen < 32 ? qlen : 32;
        if (nb == 0) break;
        // lane c stages candidate c of the batch (absent ones: zero rows,
        // zero features, thr = -inf)
        {
            const bool has = lane < nb;
            const float4 ent = has ? cq[(qhead + lane) & (CQ_N - 1)] : make_float4(0.f, 0.f, 0.f, 0.f);
            const int i = __float_as_int(ent.w);
            stage_label_row<DP, SPLIT>(cl + lane * LW, A.sem_sorted, i, ls, has);
            const float x0 = ent.x, x1 = ent.y, x2 = ent.z;
            const float xx = fmaf(x0, x0, fmaf(x1, x1, x2 * x2));
            float* cgp = cg + 12 * (lane >> 1) + (lane & 1);
            cgp[0] = x0;
            cgp[2] = x1;
            cgp[4] = x2;
            cgp[6] = has ? gp.rc2 - xx : -INF;
            cgp[8] = fmaf(xx, gp.kg, kwf);
            const float u0 = x0 * xs, u1 = x1 * xs, u2 = x2 * xs;
            unsigned h0, h1, h2, h3, h4, l0, l1, l2, l3, l4;
            split_f16x2(has ? 1.f : 0.f, u0, h0, l0);
            split_f16x2(u1, u2, h1, l1);
            split_f16x2(u0 * u0, u0 * u1, h2, l2);
            split_f16x2(u0 * u2, u1 * u1, h3, l3);
            split_f16x2(u1 * u2, u2 * u2, h4, l4);
            const int sw = (lane >> 1) & 3;
            uint4* frow = reinterpret_cast<uint4*>(cf + 16 * lane);
            frow[0 ^ sw] = make_uint4(h0, h1, h2, h3);
            frow[1 ^ sw] = make_uint4(h4, 0u, 0u, 0u);
            frow[2 ^ sw] = make_uint4(l0, l1, l2, l3);
            frow[3 ^ sw] = make_uint4(l4, 0u, 0u, 0u);
        }
        qhead = (qhead + nb) & (CQ_N - 1);
        qlen -= nb;
        __syncwarp();
        // m tiles one after another, not unrolled: the smaller loop body ran
        // faster (LiDAR 0.344 -> 0.284 ms, window 2.00 -> 1.85 ms, mapping
        // within 1%)
#pragma unroll 1
        for (int mt = 0; mt < L::MAXQ / 16; ++mt) {
            if (mt >= n_mt) break;
            // query-side A fragments of the label products: rows 16 mt ..
            // 16 mt + 15 (FP32 labels: hi and lo parts)
            const unsigned* qrowp = ql + (16 * mt + (lane & 7) + 8 * ((lane >> 3) & 1)) * LW;
            unsigned qa[2 * NKC];
            load_a_chunks<NKC>(qa, qrowp);
            unsigned qal[SPLIT ? 2 * NKC : 1];
            if constexpr (SPLIT) load_a_chunks<NKC>(qal, qrowp + PW);
            // per candidate tile nt (8 candidates): label products, then the
            // weights of rows q0 = 16 mt + g, q0 + 8 and columns 8 nt + 2 t4,
            // + 1, split into the FP16 A operands of the moment MMAs
            unsigned ah[2][4], al[2][4];
            const ulonglong2* q2 = reinterpret_cast<const ulonglong2*>(qg);
            const float4* qg4 = reinterpret_cast<const float4*>(qg);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const unsigned* crowp = cl + (8 * nt + (lane & 7)) * LW;
                unsigned cb[NKC];
                load_b_chunks<NKC>(cb, crowp);
                float s[4] = {0.f, 0.f, 0.f, 0.f};
                if constexpr (SPLIT) {
                    // FP32 labels: hi*hi + hi*lo + lo*hi of the FP16 parts
                    unsigned cbl[NKC];
                    load_b_chunks<NKC>(cbl, crowp + PW);
                    gram_chunks<NKC, true>(s, qa, cb);
                    gram_chunks<NKC, true>(s, qa, cbl);
                    gram_chunks<NKC, true>(s, qal, cb);
                } else {
                    gram_chunks<NKC, false>(s, qa, cb);
                }
                const int p = 4 * nt + t4;
                const ulonglong2 c01 = *reinterpret_cast<const ulonglong2*>(cg + 12 * p);
                const ulonglong2 c2t = *reinterpret_cast<const ulonglong2*>(cg + 12 * p + 4);
                const u64 XK = *reinterpret_cast<const u64*>(cg + 12 * p + 8);
                const float2 thr = f2_split(c2t.y);
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int q = 16 * mt + g + 8 * i;
                    ulonglong2 QA, QB;
                    if constexpr (SPLIT) {
                        const float4 qv = qg4[q];
                        QA = make_ulonglong2(f2(qv.x, qv.x), f2(qv.y, qv.y));
                        QB = make_ulonglong2(f2(qv.z, qv.z), f2(qv.w, qv.w));
                    } else {
                        QA = q2[2 * q];
                        QB = q2[2 * q + 1];
                    }
                    const u64 T = ffma2(c01.x, QA.x, ffma2(c01.y, QA.y, ffma2(c2t.x, QB.x, QB.y)));
                    const float2 t = f2_split(T);
                    const float2 a = f2_split(ffma2(T, KG2, XK));
                    const float w0 = s[2 * i] * ex2_approx(a.x), w1 = s[2 * i + 1] * ex2_approx(a.y);
                    split_f16x2(inside_count(t.x, thr.x, w0, cnt), inside_count(t.y, thr.y, w1, cnt),
                                ah[nt >> 1][2 * (nt & 1) + i], al[nt >> 1][2 * (nt & 1) + i]);
                }
            }
            // per query: sum over the batch's candidates of w (1, x, x x^T);
            // feature B fragments (FP16 hi and lo) of each 16-candidate k step
            float t[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                unsigned fh[4], fl[4];
                const int c = 16 * ks + (lane & 7) + 8 * ((lane >> 3) & 1);
                const int sw = (c >> 1) & 3;
                const unsigned* rowp = cf + 16 * c;
                ldsm_x4_t(fh, rowp + 4 * ((lane >> 4) ^ sw));
                ldsm_x4_t(fl, rowp + 4 * ((2 + (lane >> 4)) ^ sw));
#pragma unroll
                for (int n2 = 0; n2 < 2; ++n2) {
                    mma_f16_16816(t[n2], ah[ks], fh[2 * n2], fh[2 * n2 + 1]);
                    mma_f16_16816(t[n2], ah[ks], fl[2 * n2], fl[2 * n2 + 1]);
                    mma_f16_16816(t[n2], al[ks], fh[2 * n2], fh[2 * n2 + 1]);
                }
            }
            {
                float4 r = run0[32 * mt];
                r.x += t[0][0];
                r.y += t[0][1];
                r.z += t[0][2];
                r.w += t[0][3];
                run0[32 * mt] = r;
                if (t4 == 0) {     // features 8, 9 (the other columns of tile 1 are zero)
                    float4 r1 = run1[8 * mt];
                    r1.x += t[1][0];
                    r1.y += t[1][1];
                    r1.z += t[1][2];
                    r1.w += t[1][3];
                    run1[8 * mt] = r1;
                }
            }
        }
    }
    // unit end: per-query sums through shared memory to one lane per query
    // (32 queries at a time), formed into this lane's moments
    float W = 0.f, Dv[3] = {0.f, 0.f, 0.f}, Sy[3] = {0.f, 0.f, 0.f}, Myy[6], Mdy[9], Qm[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) Myy[k] = Qm[k] = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) Mdy[k] = 0.f;
    const float s0 = ldexpf(1.f, -KW), s1 = ldexpf(1.f, ex - KW), s2 = ldexpf(1.f, 2 * ex - KW);
    float* sq = reinterpret_cast<float*>(cf);    // [32][16] (features 0..9 used)
#pragma unroll
    for (int h = 0; h < L::MAXQ / 32; ++h) {
        __syncwarp();
#pragma unroll
        for (int m2 = 0; m2 < 2; ++m2) {
            const int mt = 2 * h + m2;
            const int q0 = 16 * m2 + g;
            const float4 r = run0[32 * mt];
            *reinterpret_cast<float2*>(sq + 16 * q0 + 2 * t4) = make_float2(r.x, r.y);
            *reinterpret_cast<float2*>(sq + 16 * (q0 + 8) + 2 * t4) = make_float2(r.z, r.w);
            if (t4 == 0) {
                const float4 r1 = run1[8 * mt];
                *reinterpret_cast<float2*>(sq + 16 * q0 + 8) = make_float2(r1.x, r1.y);
                *reinterpret_cast<float2*>(sq + 16 * (q0 + 8) + 8) = make_float2(r1.z, r1.w);
            }
        }
        __syncwarp();
        const int q = lane + 32 * h;
        const float4* rq = reinterpret_cast<const float4*>(sq + 16 * lane);
        const float4 r0 = rq[0], r1 = rq[1];
        const float2 r2 = *reinterpret_cast<const float2*>(sq + 16 * lane + 8);
        float y[3];
        if constexpr (SPLIT) {
            const float4 qm = reinterpret_cast<const float4*>(qg)[q];
            y[0] = -0.5f * qm.x;
            y[1] = -0.5f * qm.y;
            y[2] = -0.5f * qm.z;
        } else {
            const float4 qm = reinterpret_cast<const float4*>(qg)[2 * q];
            y[0] = -0.5f * qm.x;
            y[1] = -0.5f * qm.z;
            y[2] = -0.5f * qg[8 * q + 4];
        }
        const float k = r0.x * s0;
        const float X1[3] = {r0.y * s1, r0.z * s1, r0.w * s1};
        const float X2[6] = {r1.x * s2, r1.y * s2, r1.z * s2, r1.w * s2, r2.x * s2, r2.y * s2};
        float ky[3], D[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            ky[m] = k * y[m];
            D[m] = X1[m] - ky[m];
        }
        W += k;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            Sy[m] += ky[m];
            Dv[m] += D[m];
        }
        int t6 = 0;
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int l = m; l < 3; ++l, ++t6) {
                const float kyy = ky[m] * y[l];
                Myy[t6] += kyy;
                Qm[t6] += X2[t6] - X1[m] * y[l] - y[m] * X1[l] + kyy;
            }
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int l = 0; l < 3; ++l) Mdy[3 * m + l] = fmaf(D[m], y[l], Mdy[3 * m + l]);
    }
    store_moments(W, Dv, Sy, Myy, Mdy, Qm, cnt, Fa, hx, hy, hz, gp, A.edges[e].scale,
                  A.acc + (long long)e * ACC_N, lane);
}

// One unit (<= A.uq queries of one frame-a home cell, starting at sorted
// query k0) of the pair sum: stage the queries, stream the candidates of the
// 27-cell stencil, test, walk and fold, and add the unit's moments to its
// edge.  wb is the warp's shared-memory block.
template <int DP, bool BF16, bool COLOR>
__device__ __forceinline__ void pair_unit(const PairArgs& A, int k0, float* wb, int lane) {
    const uint32_t* __restrict__ qkey = A.qkey;
    const float4* __restrict__ slots = A.slots;
    const long long Q = A.Q;
    const EdgeDev* __restrict__ edges = A.edges;
    const int E = A.E;
    const FrameDev* __restrict__ frames = A.frames;
    const int* __restrict__ cell_start = A.cell_start;
    const float4* __restrict__ pts4 = A.pts4;
    const void* __restrict__ sem_sorted = A.sem_sorted;
    const float4* __restrict__ col4 = A.col4;
    long long* __restrict__ acc = A.acc;
    const GridParams& gp = A.gp;
    constexpr int SW = SemRow<DP, BF16>::WORDS;
    float4* smw = reinterpret_cast<float4*>(wb);                      // [UQ] walk records
    float* smt = wb + 4 * UQ;                                         // [UQ/2][8] test records
    float4* scq = reinterpret_cast<float4*>(wb + 8 * UQ);             // [UQ] query colours
    float* ssq = wb + (COLOR ? 12 : 8) * UQ;                          // [UQ][SW] query labels
    int* ri = reinterpret_cast<int*>(ssq + UQ * SW);
    const Rows R{ri, ri + 9, ri + 18, ri + 27};
    float4* sacc = reinterpret_cast<float4*>(ri + 40) + lane * (N_ACC / 4);   // this lane's unit sums
    float4* cq = reinterpret_cast<float4*>(ri + 40) + 32 * (N_ACC / 4);       // candidate ring
    float* gram = reinterpret_cast<float*>(cq + CQ_N);                        // [query][candidate] (BF16)
    const ulonglong2* walk2 = reinterpret_cast<const ulonglong2*>(smw);
    const ulonglong2* test2 = reinterpret_cast<const ulonglong2*>(smt);
    const u64 H2 = f2(0.5f, 0.5f);
    const uint32_t kq0 = qkey[k0];
    const int qcount = unit_queries(qkey, Q, k0, kq0, lane, A.uq, gp.key_sub);
    const uint32_t key0 = kq0 >> gp.key_sub;                 // home-cell key
    const int e = find_edge_bin(edges, E, key0);
    const FrameDev& Fa = frames[edges[e].a];
    const int dx0 = Fa.dim[0], dy0 = Fa.dim[1], dz0 = Fa.dim[2];
    const int cell = (int)(key0 - edges[e].bin_off);
    const int hx = cell % dx0, hy = (cell / dx0) % dy0, hz = cell / (dx0 * dy0);
    __syncwarp();
    // bounding box of the unit's queries (home-centre coordinates)
    float blo0 = __int_as_float(0x7f800000), blo1 = blo0, blo2 = blo0;
    float bhi0 = -blo0, bhi1 = -blo0, bhi2 = -blo0;
    {
        const int q = lane;
        float* tq = smt + 8 * (q >> 1) + (q & 1);
        if (q < qcount) {
            const float4 r = slots[(long long)k0 + q];
            blo0 = bhi0 = r.x;
            blo1 = bhi1 = r.y;
            blo2 = bhi2 = r.z;
            const int s = __float_as_int(r.w);
            const float mx = -2.f * r.x, my = -2.f * r.y, mz = -2.f * r.z;
            smw[q] = make_float4(mx, my, mz, mx);
            tq[0] = mx;
            tq[2] = my;
            tq[4] = mz;
            tq[6] = fmaf(r.x, r.x, fmaf(r.y, r.y, r.z * r.z));
            if (COLOR) scq[q] = __ldg(col4 + s);
            SemRow<DP, BF16>::stage(ssq + q * SW, sem_sorted, s);
        } else if (q == qcount && (q & 1)) {
            // odd count: the partner slot of the last pair never passes
            tq[0] = 0.f;
            tq[2] = 0.f;
            tq[4] = 0.f;
            tq[6] = __int_as_float(0x7f800000);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        blo0 = fminf(blo0, __shfl_xor_sync(FULL, blo0, o));
        blo1 = fminf(blo1, __shfl_xor_sync(FULL, blo1, o));
        blo2 = fminf(blo2, __shfl_xor_sync(FULL, blo2, o));
        bhi0 = fmaxf(bhi0, __shfl_xor_sync(FULL, bhi0, o));
        bhi1 = fmaxf(bhi1, __shfl_xor_sync(FULL, bhi1, o));
        bhi2 = fmaxf(bhi2, __shfl_xor_sync(FULL, bhi2, o));
    }
    const int C = build_rows(R, cell_start, Fa.cell_off, dx0, dy0, dz0, hx, hy, hz, lane);
    const int np = (qcount + 1) >> 1;
    // a candidate farther than r_c from the query box pairs with none of
    // the queries; the margin keeps every candidate the exact test passes
    const float box_thr = gp.rc2 * 1.0001f;
    // BF16 labels: the Gram path leaves registers free, so the stencil row
    // prefix, the query-side MMA fragments and the per-lane unit sums live
    // in registers instead of shared memory
    constexpr bool REG = BF16 && DP > 0;
    int pre[9];
    if constexpr (REG) {
#pragma unroll
        for (int k = 0; k < 9; ++k) pre[k] = R.pre[k];
    }
    GramB<(BF16 && DP > 0) ? DP : 16> gb;
    if constexpr (REG) gb.load(ssq, lane);

    // per lane, over its candidates x with sums w0 = sum w, dc = sum w d,
    // qc = sum w d d^T: W, D, Q and sum w0 x, sum w0 x x^T, sum x dc^T
    float racc[REG ? N_ACC : 1];
    if constexpr (REG) {
#pragma unroll
        for (int k = 0; k < N_ACC; ++k) racc[k] = 0.f;
    } else {
#pragma unroll
        for (int k = 0; k < N_ACC / 4; ++k) sacc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    int cnt = 0;
    int c_s = 0, qhead = 0, qlen = 0;            // stream position, ring head and fill
    while (c_s < C || qlen > 0) {
        // stream the 27-cell candidates through the box test into the
        // ring until it holds a full batch (or the stream ends)
        while (qlen < 32 && c_s < C) {
            const int v = c_s + lane;
            bool keep = false;
            float4 ent = make_float4(0.f, 0.f, 0.f, 0.f);
            if (v < C) {
                int dx, dy, dz;
                int i;
                if constexpr (REG) i = stream_point_r(R, pre, v, dx, dy, dz);
                else i = stream_point(R, v, dx, dy, dz);
                const float4 p = __ldg(pts4 + i);
                ent.x = fmaf((float)dx, gp.hf, p.x);
                ent.y = fmaf((float)dy, gp.hf, p.y);
                ent.z = fmaf((float)dz, gp.hf, p.z);
                ent.w = __int_as_float(i);
                const float e0 = fmaxf(fmaxf(blo0 - ent.x, ent.x - bhi0), 0.f);
                const float e1 = fmaxf(fmaxf(blo1 - ent.y, ent.y - bhi1), 0.f);
                const float e2 = fmaxf(fmaxf(blo2 - ent.z, ent.z - bhi2), 0.f);
                keep = fmaf(e0, e0, fmaf(e1, e1, e2 * e2)) < box_thr;
            }
            const unsigned bal = __ballot_sync(FULL, keep);
            if (keep) cq[(qhead + qlen + __popc(bal & ((1u << lane) - 1u))) & (CQ_N - 1)] = ent;
            qlen += __popc(bal);
            c_s += 32;
        }
        __syncwarp();
        const int nb = qlen < 32 ? qlen : 32;
        if (nb == 0) break;                      // stream ended with the ring empty
        const bool has = lane < nb;
        const float4 ent = has ? cq[(qhead + lane) & (CQ_N - 1)] : make_float4(0.f, 0.f, 0.f, 0.f);
        qhead = (qhead + nb) & (CQ_N - 1);
        qlen -= nb;
        __syncwarp();
        const int i = __float_as_int(ent.w);
        // candidate relative to the home cell centre
        const float x0 = ent.x, x1 = ent.y, x2 = ent.z;
        const float xx = fmaf(x0, x0, fmaf(x1, x1, x2 * x2));
        const float thr = gp.rc2 - xx;
        Sem<DP, BF16> cs;
        if (DP > 0 && !BF16) cs.load(sem_sorted, i, has);
        float4 cc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (COLOR && has) cc = __ldg(col4 + i);
        // cutoff test against query pairs: bit j set when |x - y_j| < r_c
        unsigned mk = 0u;
        {
            const u64 X0 = f2(x0, x0), X1 = f2(x1, x1), X2 = f2(x2, x2);
#pragma unroll 4
            for (int pj = 0; pj < np; ++pj) {
                const ulonglong2 a = test2[2 * pj], b = test2[2 * pj + 1];
                const float2 t = f2_split(ffma2(X0, a.x, ffma2(X1, a.y, ffma2(X2, b.x, b.y))));
                mk |= ((t.x < thr ? 1u : 0u) | (t.y < thr ? 2u : 0u)) << (2 * pj);
            }
        }
        if (!has) mk = 0u;
        if constexpr (BF16 && DP > 0) {
            label_gram_bf16<DP>(reinterpret_cast<const unsigned*>(sem_sorted), gb, i, __ballot_sync(FULL, has),
                                lane, gram);
            __syncwarp();
        }
        const u64 XA = f2(x0, x1), XB = f2(x2, x0);
        float w0 = 0.f, dz_s = 0.f, q12 = 0.f, q22 = 0.f;
        u64 D01 = 0ull, Q0011 = 0ull, Q0201 = 0ull;
        // the bit walk, compiled twice: with the semantic-pruning test
        // only when pruning is on (a uniform branch per batch).  Each
        // iteration takes 4 of the lane's pairs as independent dependency
        // chains (missing ones weigh zero); at 2 CTAs per SM the registers
        // for them are there, and the ILP hides more latency than a third
        // CTA's warps did.
        auto walk = [&](auto prune) {
            constexpr bool PRUNE = decltype(prune)::value;
            auto pair_w = [&](int j, u64& E01, u64& E20, float& ez, bool& kept) -> float {
                const ulonglong2 m = walk2[j];
                E01 = ffma2(H2, m.x, XA);
                E20 = ffma2(H2, m.y, XB);
                const float2 exy = f2_split(E01);
                ez = f2_split(E20).x;
                const float dd = fmaf(exy.x, exy.x, fmaf(exy.y, exy.y, ez * ez));
                float arg = dd * gp.kg;
                if (COLOR) {
                    const float4 qc = scq[j];
                    const float cr = cc.x - qc.x, cg = cc.y - qc.y, cb = cc.z - qc.z;
                    arg = fmaf(fmaf(cr, cr, fmaf(cg, cg, cb * cb)), gp.kc, arg);
                }
                float s;
                if constexpr (BF16 && DP > 0) s = gram[j * GRAM_LD + gram_col(j, lane)];
                else s = SemRow<DP, BF16>::dot(cs, ssq + j * SW);
                kept = true;
                if constexpr (PRUNE) kept = s >= gp.sem_min;
                return kept ? s * ex2_approx(arg) : 0.f;
            };
            auto add = [&](float w, u64 E01, u64 E20, float ez, bool kept) {
                const u64 WXY = fmul2(f2(w, w), E01);
                const float wz = w * ez;
                w0 += w;
                D01 = fadd2(D01, WXY);
                dz_s += wz;
                Q0011 = ffma2(WXY, E01, Q0011);
                Q0201 = ffma2(WXY, E20, Q0201);
                q12 = fmaf(f2_split(WXY).y, ez, q12);
                q22 = fmaf(wz, ez, q22);
                cnt += kept ? 1 : 0;
            };
            constexpr int U = 4;   // pairs per iteration
            while (__any_sync(FULL, mk != 0u)) {
                if (mk) {
                    int jj[U];
                    bool hv[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        hv[u] = mk != 0u;
                        jj[u] = hv[u] ? __ffs(mk) - 1 : 0;
                        if (hv[u]) mk &= mk - 1u;
                    }
                    u64 Ea[U], Eb[U];
                    float ez[U], w[U];
                    bool kp[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) w[u] = pair_w(jj[u], Ea[u], Eb[u], ez[u], kp[u]);
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (!hv[u]) { w[u] = 0.f; kp[u] = false; }
                        add(w[u], Ea[u], Eb[u], ez[u], kp[u]);
                    }
                }
            }
        };
        if (DP > 0 && gp.sem_min > -__int_as_float(0x7f800000)) walk(std::true_type{});
        else walk(std::false_type{});
        const float2 dxy = f2_split(D01), q0011 = f2_split(Q0011), q0201 = f2_split(Q0201);
        const float x[3] = {x0, x1, x2};
        const float dc[3] = {dxy.x, dxy.y, dz_s};
        const float qc[6] = {q0011.x, q0201.y, q0201.x, q0011.y, q12, q22};
        float a_s[REG ? 1 : N_ACC];
        float* a = REG ? racc : a_s;
        if constexpr (!REG) {
#pragma unroll
            for (int k = 0; k < N_ACC / 4; ++k) {
                const float4 t = sacc[k];
                a[4 * k] = t.x; a[4 * k + 1] = t.y; a[4 * k + 2] = t.z; a[4 * k + 3] = t.w;
            }
        }
        a[A_W] += w0;
#pragma unroll
        for (int t6 = 0; t6 < 6; ++t6) a[A_Q + t6] += qc[t6];
#pragma unroll
        for (int mm = 0; mm < 3; ++mm) {
            a[A_D + mm] += dc[mm];
            const float wx = w0 * x[mm];
            a[A_SWX + mm] += wx;
#pragma unroll
            for (int l = 0; l < 3; ++l) a[A_SXD + 3 * mm + l] = fmaf(x[mm], dc[l], a[A_SXD + 3 * mm + l]);
#pragma unroll
            for (int l = mm; l < 3; ++l) {
                const int t6 = mm == 0 ? l : (mm == 1 ? 2 + l : 5);
                a[A_SWXX + t6] = fmaf(wx, x[l], a[A_SWXX + t6]);
            }
        }
        if constexpr (!REG) {
#pragma unroll
            for (int k = 0; k < N_ACC / 4; ++k)
                sacc[k] = make_float4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
        }
    }
    float a_s[REG ? 1 : N_ACC];
    float* a = REG ? racc : a_s;
    if constexpr (!REG) {
#pragma unroll
        for (int k = 0; k < N_ACC / 4; ++k) {
            const float4 t = sacc[k];
            a[4 * k] = t.x; a[4 * k + 1] = t.y; a[4 * k + 2] = t.z; a[4 * k + 3] = t.w;
        }
    }
    const float W = a[A_W];
    const float Dv[3] = {a[A_D], a[A_D + 1], a[A_D + 2]};
    const float* Qm = a + A_Q;
    const float* Swx = a + A_SWX;
    const float* Swxx = a + A_SWXX;
    const float* Sxd = a + A_SXD;
    // y' = x - d:  sum w y' = sum w0 x - D;  sum w y'y'^T = sum w0 x x^T -
    // sum (x dc^T + dc x^T) + Q;  sum w d y'^T = sum dc x^T - Q
    float Sy[3], Myy[6], Mdy[9];
#pragma unroll
    for (int mm = 0; mm < 3; ++mm) Sy[mm] = Swx[mm] - Dv[mm];
#pragma unroll
    for (int mm = 0; mm < 3; ++mm)
#pragma unroll
        for (int l = mm; l < 3; ++l) {
            const int t6 = mm == 0 ? l : (mm == 1 ? 2 + l : 5);
            Myy[t6] = Swxx[t6] - (Sxd[3 * mm + l] + Sxd[3 * l + mm]) + Qm[t6];
        }
#pragma unroll
    for (int mm = 0; mm < 3; ++mm)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const int qi = (mm <= l) ? (mm == 0 ? l : (mm == 1 ? 2 + l : 5))
                                     : (l == 0 ? mm : (l == 1 ? 2 + mm : 5));
            Mdy[3 * mm + l] = Sxd[3 * l + mm] - Qm[qi];
        }
    store_moments(W, Dv, Sy, Myy, Mdy, Qm, cnt, Fa, hx, hy, hz, gp, edges[e].scale,
                  acc + (long long)e * ACC_N, lane);

}

// Shared-memory words per warp of the bit-walk (DENSE false) or the dense
// tile unit (BF16 labels, no colour).
// DENSE: 0 bit walk, 1 dense tile with units of <= 32 queries, 2 dense tile
// with units of <= 64 queries (BF16 labels).
template <int DP, bool BF16, bool COLOR, int DENSE>
__host__ __device__ constexpr int unit_smem_words() {
    if constexpr (DENSE > 0) return DenseSmem<(DP > 0 ? DP : 8), !BF16, DENSE == 2 ? 64 : 32>::WORDS;
    else return warp_smem_words<DP, BF16, COLOR>();
}

template <int DP, bool BF16, bool COLOR, int DENSE>
__device__ __forceinline__ void run_unit(const PairArgs& A, int k0, float* wb, int lane) {
    if constexpr (DENSE > 0 && DP > 0 && !COLOR) pair_unit_dense<DP, !BF16, DENSE == 2 ? 64 : 32>(A, k0, wb, lane);
    else pair_unit<DP, BF16, COLOR>(A, k0, wb, lane);
}

template <int DP, bool BF16, bool COLOR, int DENSE>
__global__ void __launch_bounds__(PAIR_T, DENSE ? dense_min_blocks<DP, BF16, DENSE>()
                                                  : ((BF16 && DP > 0) ? 2 : RK_PAIR_MINB))
k_pairs(const int* __restrict__ unit_start, const int* __restrict__ n_units, int* unit_counter,
        const PairArgs A, const int* done) {
    if (done && *done) return;
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float* wb = reinterpret_cast<float*>(smem4) + warp * unit_smem_words<DP, BF16, COLOR, DENSE>();
    const int nu = *n_units;
    for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(unit_counter, 1);
        u = __shfl_sync(FULL, u, 0);
        if (u >= nu) break;
        run_unit<DP, BF16, COLOR, DENSE>(A, unit_start[u], wb, lane);
    }
}

// The pair stage of several problems in one persistent launch: the units of
// job j are numbered after those of jobs 0..j-1 (a job whose solve is done
// contributes none), warps take global unit numbers from one counter, find
// the job by binary search over the prefix, and run the unit with that
// job's arrays.  Every job adds into its own fixed-point accumulators, so a
// problem's results do not depend on which other problems share the launch.
template <int DP, bool BF16, bool COLOR, int DENSE>
__global__ void __launch_bounds__(PAIR_T, DENSE ? dense_min_blocks<DP, BF16, DENSE>()
                                                  : ((BF16 && DP > 0) ? 2 : RK_PAIR_MINB))
k_pairs_multi(const PairJob* __restrict__ jobs, int n_jobs, int* unit_counter) {
    __shared__ int s_pref[MAX_PAIR_JOBS + 1];
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        int carry = 0;
        for (int base = 0; base < n_jobs; base += 32) {
            const int j = base + lane;
            int n = 0;
            if (j < n_jobs) {
                const int* dn = jobs[j].done;
                n = (dn && *dn) ? 0 : *jobs[j].n_units;
            }
            int inc = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULL, inc, o);
                if (lane >= o) inc += v;
            }
            if (j < n_jobs) s_pref[j] = carry + inc - n;
            carry += __shfl_sync(FULL, inc, 31);
        }
        if (lane == 0) s_pref[n_jobs] = carry;
    }
    __syncthreads();
    const int total = s_pref[n_jobs];
    float* wb = reinterpret_cast<float*>(smem4) + warp * unit_smem_words<DP, BF16, COLOR, DENSE>();
    for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(unit_counter, 1);
        u = __shfl_sync(FULL, u, 0);
        if (u >= total) break;
        int lo = 0, hi = n_jobs - 1;                 // last job with s_pref[j] <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_pref[mid] <= u) lo = mid; else hi = mid - 1;
        }
        const PairJob* J = jobs + lo;
        run_unit<DP, BF16, COLOR, DENSE>(J->a, J->unit_start[u - s_pref[lo]], wb, lane);
    }
}

// Neighbour-limited variant (top_k > 0): the same candidate stream, cutoff
// test and weight, with lanes over the unit's queries.  Each lane keeps the
// TOPK_MAX pairs of largest w of its query (candidates broadcast from shared
// memory in stream order; a later candidate displaces only a strictly smaller
// w), then sums its first top_k: W, D = sum w d, Q = sum w d d^T, and with
// y' the query itself sum w y' = W y, sum w y'y'^T = W y y^T,
// sum w d y'^T = D y^T.
template <int DP, bool BF16, bool COLOR>
__host__ __device__ constexpr int warp_smem_words_topk() {
    return 32 * 4 + 32 * SemRow<DP, BF16>::WORDS + (COLOR ? 32 * 4 : 0) + 4 * CQ_N + 4 * 10;
}

template <int DP, bool BF16, bool COLOR>
__global__ void __launch_bounds__(PAIR_T, 2)
k_pairs_topk(const int* __restrict__ unit_start, const int* __restrict__ n_units, int* unit_counter,
             const uint32_t* __restrict__ qkey, const float4* __restrict__ slots, long long Q,
             const EdgeDev* __restrict__ edges, int E, const FrameDev* __restrict__ frames,
             const int* __restrict__ cell_start, const float4* __restrict__ pts4,
             const void* __restrict__ sem_sorted, const float4* __restrict__ col4, GridParams gp,
             long long* __restrict__ acc, int uq, const int* done) {
    if (done && *done) return;
    extern __shared__ float4 smem4[];
    constexpr int SW = SemRow<DP, BF16>::WORDS;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float* wb = reinterpret_cast<float*>(smem4) + warp * warp_smem_words_topk<DP, BF16, COLOR>();
    float4* scx = reinterpret_cast<float4*>(wb);                      // [32] staged candidates (x, index)
    float* srow = wb + 4 * 32;                                        // [32][SW] their label rows
    float4* scc = reinterpret_cast<float4*>(srow + 32 * SW);          // [32] their colours
    float4* cq = reinterpret_cast<float4*>(wb + 4 * 32 + 32 * SW + (COLOR ? 4 * 32 : 0));   // ring
    int* ri = reinterpret_cast<int*>(cq + CQ_N);
    const Rows R{ri, ri + 9, ri + 18, ri + 27};
    const float NEG_INF = -__int_as_float(0x7f800000);
    const int nu = *n_units;
    for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(unit_counter, 1);
        u = __shfl_sync(FULL, u, 0);
        if (u >= nu) break;
        const int k0 = unit_start[u];
        const uint32_t kq0 = qkey[k0];
        const int qcount = unit_queries(qkey, Q, k0, kq0, lane, uq, gp.key_sub);
        const uint32_t key0 = kq0 >> gp.key_sub;
        const int e = find_edge_bin(edges, E, key0);
        const FrameDev& Fa = frames[edges[e].a];
        const int dx0 = Fa.dim[0], dy0 = Fa.dim[1], dz0 = Fa.dim[2];
        const int cell = (int)(key0 - edges[e].bin_off);
        const int hx = cell % dx0, hy = (cell / dx0) % dy0, hz = cell / (dx0 * dy0);
        // this lane's query
        const bool qv = lane < qcount;
        const float4 r = qv ? slots[(long long)k0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int sidx = __float_as_int(r.w);
        const float mx = -2.f * r.x, my = -2.f * r.y, mz = -2.f * r.z;
        const float mw = fmaf(r.x, r.x, fmaf(r.y, r.y, r.z * r.z));
        Sem<DP, BF16> qs;
        if (DP > 0) qs.load(sem_sorted, sidx, qv);
        float4 qc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (COLOR && qv) qc = __ldg(col4 + sidx);
        float blo0 = qv ? r.x : -NEG_INF, blo1 = qv ? r.y : -NEG_INF, blo2 = qv ? r.z : -NEG_INF;
        float bhi0 = qv ? r.x : NEG_INF, bhi1 = qv ? r.y : NEG_INF, bhi2 = qv ? r.z : NEG_INF;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            blo0 = fminf(blo0, __shfl_xor_sync(FULL, blo0, o));
            blo1 = fminf(blo1, __shfl_xor_sync(FULL, blo1, o));
            blo2 = fminf(blo2, __shfl_xor_sync(FULL, blo2, o));
            bhi0 = fmaxf(bhi0, __shfl_xor_sync(FULL, bhi0, o));
            bhi1 = fmaxf(bhi1, __shfl_xor_sync(FULL, bhi1, o));
            bhi2 = fmaxf(bhi2, __shfl_xor_sync(FULL, bhi2, o));
        }
        __syncwarp();
        const int C = build_rows(R, cell_start, Fa.cell_off, dx0, dy0, dz0, hx, hy, hz, lane);
        const float box_thr = gp.rc2 * 1.0001f;
        float tw[TOPK_MAX], t0[TOPK_MAX], t1[TOPK_MAX], t2[TOPK_MAX];   // w descending, d = x - y
#pragma unroll
        for (int k = 0; k < TOPK_MAX; ++k) {
            tw[k] = NEG_INF;
            t0[k] = t1[k] = t2[k] = 0.f;
        }
        int c_s = 0, qhead = 0, qlen = 0;
        while (c_s < C || qlen > 0) {
            while (qlen < 32 && c_s < C) {
                const int v = c_s + lane;
                bool keep = false;
                float4 ent = make_float4(0.f, 0.f, 0.f, 0.f);
                if (v < C) {
                    int dx, dy, dz;
                    const int i = stream_point(R, v, dx, dy, dz);
                    const float4 p = __ldg(pts4 + i);
                    ent.x = fmaf((float)dx, gp.hf, p.x);
                    ent.y = fmaf((float)dy, gp.hf, p.y);
                    ent.z = fmaf((float)dz, gp.hf, p.z);
                    ent.w = __int_as_float(i);
                    const float e0 = fmaxf(fmaxf(blo0 - ent.x, ent.x - bhi0), 0.f);
                    const float e1 = fmaxf(fmaxf(blo1 - ent.y, ent.y - bhi1), 0.f);
                    const float e2 = fmaxf(fmaxf(blo2 - ent.z, ent.z - bhi2), 0.f);
                    keep = fmaf(e0, e0, fmaf(e1, e1, e2 * e2)) < box_thr;
                }
                const unsigned bal = __ballot_sync(FULL, keep);
                if (keep) cq[(qhead + qlen + __popc(bal & ((1u << lane) - 1u))) & (CQ_N - 1)] = ent;
                qlen += __popc(bal);
                c_s += 32;
            }
            __syncwarp();
            const int nb = qlen < 32 ? qlen : 32;
            if (nb == 0) break;
            if (lane < nb) {
                const float4 ent = cq[(qhead + lane) & (CQ_N - 1)];
                const int i = __float_as_int(ent.w);
                scx[lane] = ent;
                SemRow<DP, BF16>::stage(srow + lane * SW, sem_sorted, i);
                if (COLOR) scc[lane] = __ldg(col4 + i);
            }
            qhead = (qhead + nb) & (CQ_N - 1);
            qlen -= nb;
            __syncwarp();
            for (int c = 0; c < nb; ++c) {
                const float4 xe = scx[c];
                const float thr = gp.rc2 - fmaf(xe.x, xe.x, fmaf(xe.y, xe.y, xe.z * xe.z));
                const float t = fmaf(xe.x, mx, fmaf(xe.y, my, fmaf(xe.z, mz, mw)));
                if (qv && t < thr) {
                    const float ex = fmaf(0.5f, mx, xe.x), ey = fmaf(0.5f, my, xe.y), ez = fmaf(0.5f, mz, xe.z);
                    const float dd = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                    float arg = dd * gp.kg;
                    if (COLOR) {
                        const float4 cc = scc[c];
                        const float cr = cc.x - qc.x, cg = cc.y - qc.y, cb = cc.z - qc.z;
                        arg = fmaf(fmaf(cr, cr, fmaf(cg, cg, cb * cb)), gp.kc, arg);
                    }
                    const float s = SemRow<DP, BF16>::dot(qs, srow + c * SW);
                    if (s >= gp.sem_min) {
                        float cw = s * ex2_approx(arg);
                        if (cw > tw[TOPK_MAX - 1]) {
                            float c0 = ex, c1 = ey, c2 = ez;
#pragma unroll
                            for (int k = 0; k < TOPK_MAX; ++k) {
                                const bool sw = cw > tw[k];
                                const float a = tw[k], b0 = t0[k], b1 = t1[k], b2 = t2[k];
                                tw[k] = sw ? cw : a;
                                t0[k] = sw ? c0 : b0;
                                t1[k] = sw ? c1 : b1;
                                t2[k] = sw ? c2 : b2;
                                cw = sw ? a : cw;
                                c0 = sw ? b0 : c0;
                                c1 = sw ? b1 : c1;
                                c2 = sw ? b2 : c2;
                            }
                        }
                    }
                }
            }
            __syncwarp();
        }
        float W = 0.f, Dv[3] = {0.f, 0.f, 0.f}, Qm[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < TOPK_MAX; ++k) {
            if (k < gp.top_k && tw[k] > NEG_INF) {
                const float w = tw[k];
                const float wx = w * t0[k], wy = w * t1[k], wz = w * t2[k];
                W += w;
                Dv[0] += wx; Dv[1] += wy; Dv[2] += wz;
                Qm[0] = fmaf(wx, t0[k], Qm[0]); Qm[1] = fmaf(wx, t1[k], Qm[1]); Qm[2] = fmaf(wx, t2[k], Qm[2]);
                Qm[3] = fmaf(wy, t1[k], Qm[3]); Qm[4] = fmaf(wy, t2[k], Qm[4]); Qm[5] = fmaf(wz, t2[k], Qm[5]);
                ++cnt;
            }
        }
        const float y[3] = {r.x, r.y, r.z};
        float Sy[3], Myy[6], Mdy[9];
        int t6 = 0;
#pragma unroll
        for (int mm = 0; mm < 3; ++mm) {
            Sy[mm] = W * y[mm];
#pragma unroll
            for (int l = 0; l < 3; ++l) Mdy[3 * mm + l] = Dv[mm] * y[l];
#pragma unroll
            for (int l = mm; l < 3; ++l, ++t6) Myy[t6] = W * y[mm] * y[l];
        }
        store_moments(W, Dv, Sy, Myy, Mdy, Qm, cnt, Fa, hx, hy, hz, gp, edges[e].scale,
                      acc + (long long)e * ACC_N, lane);
    }
}

// Same search and the same cutoff test, geometry only: writes the pair list
// of one edge (verification).
__global__ void __launch_bounds__(PAIR_T)
k_emit_pairs(const int* __restrict__ unit_start, const int* __restrict__ n_units, int* unit_counter,
             const uint32_t* __restrict__ qkey, const float4* __restrict__ slots, long long Q,
             const EdgeDev* __restrict__ edges, int E, const FrameDev* __restrict__ frames,
             const int* __restrict__ cell_start, const float4* __restrict__ pts4, GridParams gp,
             int edge_sel, const int* __restrict__ perm_local, long long capacity, int uq,
             int* __restrict__ i_out, int* __restrict__ j_out, unsigned long long* n_out) {
    __shared__ float4 s_m[PAIR_T / 32][64];
    __shared__ int s_j[PAIR_T / 32][64];
    __shared__ int s_rows[PAIR_T / 32][40];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float4* sm = s_m[warp];
    const Rows R{s_rows[warp], s_rows[warp] + 9, s_rows[warp] + 18, s_rows[warp] + 27};
    const int nu = *n_units;
    for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(unit_counter, 1);
        u = __shfl_sync(FULL, u, 0);
        if (u >= nu) break;
        const int k0 = unit_start[u];
        const uint32_t kq0 = qkey[k0];
        const uint32_t key0 = kq0 >> gp.key_sub;
        const int e = find_edge_bin(edges, E, key0);
        if (e != edge_sel) continue;
        const int qcount = unit_queries64(qkey, Q, k0, kq0, lane, uq, gp.key_sub);
        const FrameDev& Fa = frames[edges[e].a];
        const int dx0 = Fa.dim[0], dy0 = Fa.dim[1], dz0 = Fa.dim[2];
        const int cell = (int)(key0 - edges[e].bin_off);
        const int hx = cell % dx0, hy = (cell / dx0) % dy0, hz = cell / (dx0 * dy0);
        __syncwarp();
        for (int h = 0; h < 2; ++h) {
            const int q = lane + 32 * h;
            if (q < qcount) {
                const float4 r = slots[(long long)k0 + q];
                sm[q] = make_float4(-2.f * r.x, -2.f * r.y, -2.f * r.z, fmaf(r.x, r.x, fmaf(r.y, r.y, r.z * r.z)));
                s_j[warp][q] = perm_local[__float_as_int(r.w)];
            }
        }
        const int C = build_rows(R, cell_start, Fa.cell_off, dx0, dy0, dz0, hx, hy, hz, lane);
        for (int c0 = 0; c0 < C; c0 += 32) {
            const int v = c0 + lane;
            if (v >= C) continue;
            int dx, dy, dz;
            const int i = stream_point(R, v, dx, dy, dz);
            const float4 p = __ldg(pts4 + i);
            const float x0 = fmaf((float)dx, gp.hf, p.x), x1 = fmaf((float)dy, gp.hf, p.y),
                        x2 = fmaf((float)dz, gp.hf, p.z);
            const float thr = gp.rc2 - fmaf(x0, x0, fmaf(x1, x1, x2 * x2));
            for (int j = 0; j < qcount; ++j) {
                const float4 m = sm[j];
                const float t = fmaf(x0, m.x, fmaf(x1, m.y, fmaf(x2, m.z, m.w)));
                if (t < thr) {
                    const unsigned long long k = atomicAdd(n_out, 1ULL);
                    if ((long long)k < capacity) {
                        i_out[k] = perm_local[i];
                        j_out[k] = s_j[warp][j];
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

// Resident CTAs per SM of a pair kernel at its shared-memory size (queried
// once per instantiation; the dynamic shared memory opt-in is set then).
template <typename KernelT>
int pair_blocks_per_sm(KernelT kernel, size_t smem, int* cache) {
    if (!*cache) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, PAIR_T, smem);
        *cache = b < 1 ? 1 : b;
    }
    return *cache;
}

inline unsigned pair_grid(int num_sms, int resident, int ctas_per_sm) {
    const int per_sm = (ctas_per_sm > 0 && ctas_per_sm < resident) ? ctas_per_sm : resident;
    return (unsigned)(num_sms * per_sm);
}

// The dense tile unit serves BF16 labels without colour and without
// semantic pruning (top_k has its own kernel); RK_NO_DENSE builds the
// bit-walk kernel for every layout.
inline bool dense_path(const GridParams& gp) {
#ifdef RK_NO_DENSE
    (void)gp;
    return false;
#else
    return gp.sem_pad > 0 && !gp.color && !(gp.sem_min > -__builtin_huge_valf()) && gp.top_k == 0;
#endif
}

template <int DP, bool BF16, bool COLOR, int DENSE>
void launch_k_pairs(const PairLaunch& L, const PairArgs& A) {
    const size_t smem = sizeof(float) * (PAIR_T / 32) * unit_smem_words<DP, BF16, COLOR, DENSE>();
    static int resident = 0;   // opt in to > 48 KB and size the persistent grid, once per instantiation
    const int r = pair_blocks_per_sm(k_pairs<DP, BF16, COLOR, DENSE>, smem, &resident);
    k_pairs<DP, BF16, COLOR, DENSE><<<pair_grid(L.num_sms, r, L.ctas_per_sm), PAIR_T, smem, L.stream>>>(
        L.unit_start, L.n_units, L.unit_counter, A, L.done);
}

template <int DP, bool BF16, bool COLOR>
void run_pairs(const PairLaunch& L, const PairArgs& A) {
    if (A.gp.top_k > 0) {
        const size_t smem = sizeof(float) * (PAIR_T / 32) * warp_smem_words_topk<DP, BF16, COLOR>();
        static int resident = 0;
        const int r = pair_blocks_per_sm(k_pairs_topk<DP, BF16, COLOR>, smem, &resident);
        k_pairs_topk<DP, BF16, COLOR><<<pair_grid(L.num_sms, r, L.ctas_per_sm), PAIR_T, smem, L.stream>>>(
            L.unit_start, L.n_units, L.unit_counter, A.qkey, A.slots, A.Q, A.edges, A.E, A.frames, A.cell_start,
            A.pts4, A.sem_sorted, A.col4, A.gp, A.acc, A.uq, L.done);
        return;
    }
    if constexpr (DP > 0 && !COLOR) {
        if (dense_path(A.gp)) {
            if constexpr (BF16) {
                if (A.uq > 32) {
                    launch_k_pairs<DP, BF16, COLOR, 2>(L, A);
                    return;
                }
            }
            launch_k_pairs<DP, BF16, COLOR, 1>(L, A);
            return;
        }
    }
    launch_k_pairs<DP, BF16, COLOR, 0>(L, A);
}

template <int DP, bool BF16, bool COLOR, int DENSE>
void launch_k_pairs_multi(const PairJob* jobs, int n_jobs, int* counter, int num_sms, int ctas_per_sm,
                          cudaStream_t st) {
    const size_t smem = sizeof(float) * (PAIR_T / 32) * unit_smem_words<DP, BF16, COLOR, DENSE>();
    static int resident = 0;   // opt in to > 48 KB and size the persistent grid, once per instantiation
    const int r = pair_blocks_per_sm(k_pairs_multi<DP, BF16, COLOR, DENSE>, smem, &resident);
    k_pairs_multi<DP, BF16, COLOR, DENSE><<<pair_grid(num_sms, r, ctas_per_sm), PAIR_T, smem, st>>>(
        jobs, n_jobs, counter);
}

// max_uq: the largest unit size among the jobs
template <int DP, bool BF16, bool COLOR>
void run_pairs_multi(const PairJob* jobs, int n_jobs, int* counter, int num_sms, int ctas_per_sm, bool dense,
                     int max_uq, cudaStream_t st) {
    if constexpr (DP > 0 && !COLOR) {
        if (dense) {
            if constexpr (BF16) {
                if (max_uq > 32) {
                    launch_k_pairs_multi<DP, BF16, COLOR, 2>(jobs, n_jobs, counter, num_sms, ctas_per_sm, st);
                    return;
                }
            }
            launch_k_pairs_multi<DP, BF16, COLOR, 1>(jobs, n_jobs, counter, num_sms, ctas_per_sm, st);
            return;
        }
    }
    launch_k_pairs_multi<DP, BF16, COLOR, 0>(jobs, n_jobs, counter, num_sms, ctas_per_sm, st);
}

// Calls F.template operator()<DP, BF16>() for the label layout of gp
// (padded width, FP32 or BF16 rows); false for a layout without kernels.
template <typename F>
bool with_label_layout(const GridParams& gp, const F& f) {
    if (gp.sem_pad == 0) { f.template operator()<0, false>(); return true; }
    if (gp.sem_bf16) {
        switch (gp.sem_pad) {
            case 8: f.template operator()<8, true>(); return true;
            case 16: f.template operator()<16, true>(); return true;
            case 24: f.template operator()<24, true>(); return true;
            case 32: f.template operator()<32, true>(); return true;
            default: return false;
        }
    }
    switch (gp.sem_pad) {
        case 4: f.template operator()<4, false>(); return true;
        case 8: f.template operator()<8, false>(); return true;
        case 12: f.template operator()<12, false>(); return true;
        case 16: f.template operator()<16, false>(); return true;
        case 20: f.template operator()<20, false>(); return true;
        case 24: f.template operator()<24, false>(); return true;
        case 32: f.template operator()<32, false>(); return true;
        default: return false;
    }
}
}  // namespace

void launch_edge_setup(const double* poses, const EdgeDev* edges, int E, const FrameDev* frames,
                       double h, EdgeXf* xf, const int* done, cudaStream_t st) {
    k_edge_setup<<<(E + 127) / 128, 128, 0, st>>>(poses, edges, E, frames, h, xf, done);
    count_launch();
}

void launch_query_keys(const EdgeDev* edges, int E, const FrameDev* frames, const EdgeXf* xf,
                       const uint32_t* pt_cell, const float4* pts4, GridParams gp, long long Q,
                       uint32_t* qkey, int* qval, float4* qrec, const int* done, cudaStream_t st) {
    if (Q <= 0) return;
    k_query_keys<<<blocks_for(Q, 256), 256, 0, st>>>(edges, E, frames, xf, pt_cell, pts4, gp, Q, qkey, qval,
                                                    qrec, done);
    count_launch();
}

void launch_query_gather(const uint32_t* qkey_sorted, const int* qval_sorted, const float4* qrec,
                         long long Q, int sub, float4* slots, int* bin_first, const int* done,
                         cudaStream_t st) {
    if (Q <= 0) return;
    k_query_gather<<<blocks_for(Q, 256), 256, 0, st>>>(qkey_sorted, qval_sorted, qrec, Q, sub, slots, bin_first,
                                                      done);
    count_launch();
}

void launch_units(const uint32_t* qkey_sorted, const int* bin_first, long long Q, int uq, int sub, int* unit_start,
                  int* n_units, const int* done, cudaStream_t st) {
    if (Q <= 0) return;
    if (uq < 1 || uq > 64) uq = UQ;
    k_units<<<blocks_for(Q, 256), 256, 0, st>>>(qkey_sorted, bin_first, Q, uq, sub, unit_start, n_units, done);
    count_launch();
}

namespace {
struct SingleLaunch {
    const PairLaunch& L;
    const PairArgs& A;
    template <int DP, bool BF16>
    void operator()() const {
        if (A.gp.color) run_pairs<DP, BF16, true>(L, A);
        else run_pairs<DP, BF16, false>(L, A);
    }
};
struct MultiLaunch {
    const PairJob* jobs;
    int n_jobs;
    bool color;
    bool dense;
    int max_uq;
    int* counter;
    int num_sms, ctas_per_sm;
    cudaStream_t st;
    template <int DP, bool BF16>
    void operator()() const {
        if (color) run_pairs_multi<DP, BF16, true>(jobs, n_jobs, counter, num_sms, ctas_per_sm, dense, max_uq, st);
        else run_pairs_multi<DP, BF16, false>(jobs, n_jobs, counter, num_sms, ctas_per_sm, dense, max_uq, st);
    }
};
}  // namespace

int pair_unit_max(const GridParams& gp) { return (dense_path(gp) && gp.sem_bf16) ? 64 : UQ; }

void launch_pairs(const PairLaunch& L, const PairArgs& A) {
    if (A.Q <= 0) return;
    if (with_label_layout(A.gp, SingleLaunch{L, A})) count_launch();
}

bool launch_pairs_multi(const PairJob* jobs, int n_jobs, const GridParams& layout, int max_uq, int* counter,
                        int num_sms, int ctas_per_sm, cudaStream_t st) {
    if (n_jobs <= 0 || n_jobs > MAX_PAIR_JOBS || layout.top_k > 0) return false;
    const bool ok = with_label_layout(layout, MultiLaunch{jobs, n_jobs, layout.color != 0, dense_path(layout),
                                                          max_uq, counter, num_sms, ctas_per_sm, st});
    if (ok) count_launch();
    return ok;
}

void launch_emit_pairs(const int* unit_start, const int* n_units, int* unit_counter,
                       const uint32_t* qkey, const float4* slots, long long Q, const EdgeDev* edges,
                       int E, const FrameDev* frames, const int* cell_start, const float4* pts4,
                       GridParams gp, int edge_sel, const int* perm_local, long long capacity, int uq,
                       int* i_out, int* j_out, unsigned long long* n_out, int num_sms,
                       cudaStream_t st) {
    if (Q <= 0) return;
    if (uq < 1 || uq > 64) uq = UQ;
    k_emit_pairs<<<num_sms * 2, PAIR_T, 0, st>>>(unit_start, n_units, unit_counter, qkey, slots, Q, edges, E,
                                                 frames, cell_start, pts4, gp, edge_sel, perm_local, capacity, uq,
                                                 i_out, j_out, n_out);
    count_launch();
}

}  // namespace rk
