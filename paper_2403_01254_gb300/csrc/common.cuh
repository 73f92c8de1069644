// Shared types and launchers of the RKHS-BA CUDA library (sm_103a).
//
// Data layout in HBM (one problem):
//   * points of all frames sorted by (frame, uniform-grid cell), stable in the
//     input order inside a cell; per point a float4 of its offset from its own
//     cell centre (cell-local FP32 coordinates keep |x~| <= h/2, so differences
//     of nearby points lose nothing even 50 m from the sensor);
//   * labels in the same order, FP32 rows padded to a multiple of 4 floats or
//     BF16 rows padded to a multiple of 8 (16-byte aligned rows);
//   * cell_start[] over dense per-frame grids that carry a one-cell margin, so
//     every cell of a 3x3x3 stencil around a cell that can hold a neighbour is
//     addressable without a hash;
//   * per evaluation: queries (points of frame b moved into frame a) sorted
//     stably by their home cell of frame a and cut into units of <= 32
//     queries of one home cell; a warp takes a unit and streams the
//     candidates of the 27 surrounding cells through its lanes.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <atomic>

namespace rk {

extern std::atomic<long long> g_launches;      // kernels launched by the library (process)
extern thread_local long long t_launches;      // the same, counted per host thread
inline void count_launch(long long n = 1) {
    g_launches.fetch_add(n, std::memory_order_relaxed);
    t_launches += n;
}

constexpr int MAX_SEM = 32;     // label floats per point
constexpr int ACC_N = 32;       // int64 accumulator slots per edge
constexpr int N_MOM = 29;       // used slots (see MomentIndex)
#ifndef RK_UNIT_Q
#define RK_UNIT_Q 32
#endif
constexpr int UNIT_Q = RK_UNIT_Q;   // queries of one home cell per warp unit (32 or 64)

// Fixed-point accumulator layout per edge.  All sums are over the pairs of the
// edge, in frame-a coordinates: d = x - y', y' = T_ab y.
//   0 W = sum w            1..3 D = sum w d       4..6 Sy = sum w y'
//   7..12 Myy = sum w y'y'^T (xx xy xz yy yz zz)
//   13..21 Mdy = sum w d y'^T (row-major [m][l] = sum w d_m y'_l)
//   22..27 Q = sum w d d^T (xx xy xz yy yz zz)      28 pair count
enum MomentClass { MC_W = 0, MC_D = 1, MC_SY = 2, MC_MYY = 3, MC_MDY = 4, MC_Q = 5, MC_CNT = 6, MC_N = 8 };

__host__ __device__ inline int moment_class(int k) {
    return k == 0 ? MC_W : k < 4 ? MC_D : k < 7 ? MC_SY : k < 13 ? MC_MYY
         : k < 22 ? MC_MDY : k < 28 ? MC_Q : MC_CNT;
}

struct FrameDev {
    long long pt_off;     // first point (input order == sorted order range)
    int n_pts;
    int lo[3];            // absolute cell coordinates of grid cell (0,0,0)
    int dim[3];           // grid extent including a one-cell margin on each side
    long long cell_off;   // offset of this frame's cells in cell_start[]
    float sem_norm_max;   // max |l| over the frame (bounds of the fixed point)
};

struct EdgeDev {
    int a, b;             // a < b
    long long bin_off;    // first bin (bins = cells of frame a's grid)
    long long q_off;      // first query (queries = points of frame b)
    float scale[MC_N];    // fixed-point scale per moment class (power of two)
    double inv_scale[MC_N];
};

// T_ab = T_a^-1 T_b for one evaluation, plus the map from frame-b grid
// indices l (cell c = lo_b + l) to frame-a positions of cell centres,
//   P(l) = A l + B,  A = h R_ab,  B = R_ab (lo_b + 1/2) h + t_ab,
// as double-float pairs (hi + lo) so that queries need no FP64.
struct EdgeXf {
    double R[9];
    double t[3];
    float Rf[9];
    float Ahi[9], Alo[9];
    float Bhi[3], Blo[3];
};

struct EdgeOut {          // FP64 per-edge results of one evaluation
    double F;             // sigma^2 sum w
    double E;             // sum w |d|^2
    long long n;          // pair-terms
    long long pad;
    double b[12];         // sum w J^T d, [rho_a phi_a rho_b phi_b]
    double H[144];        // sum w J^T J, same ordering
};

struct GridParams {
    double h, h_inv;      // cell size h = r_c (1 + 2^-10) and its inverse
    float hf, hf_inv, hf_lo;  // FP32 h, 1/h and the remainder h - hf
    float rc2;            // r_c^2 in FP32
    float kg;             // -log2(e) / (2 ell^2)
    float kc;             // -log2(e) / (2 ell_c^2), 0 without colour
    int sem_dim, sem_pad, sem_bf16, color;
    int top_k;            // 0: every pair; else the top_k pairs of largest w per query
    float sem_min;        // pairs with <l_i, l_j> below this are dropped (-inf: off)
    int key_sub;          // low bits of a query key below its home-cell key (3: octant, 0: none)
};

constexpr int TOPK_MAX = 8;   // largest top_k of the neighbour-limited variant

// What the pair kernel reads of one problem for one evaluation: the sorted
// queries of every edge, the problem's grids and labels, and its per-edge
// fixed-point accumulators.
struct PairArgs {
    const uint32_t* qkey;     // sorted home-cell keys of the queries
    const float4* slots;      // sorted query records (offset from the home centre, point index)
    long long Q;              // queries over all edges
    const EdgeDev* edges;
    const FrameDev* frames;
    const int* cell_start;
    const float4* pts4;       // points, cell-local, sorted by (frame, cell)
    const void* sem_sorted;   // label rows in the same order (FP32 or BF16), or NULL
    const float4* col4;       // colours in the same order, or NULL
    long long* acc;           // [E][ACC_N] fixed-point moments
    int E;
    int uq;                   // queries per unit (1..32; up to 64 for the dense kernel with BF16 labels)
    GridParams gp;
};

// One problem of a batched pair launch: its unit list and LM state flag
// (a job whose solve is done contributes no units).
struct PairJob {
    const int* unit_start;
    const int* n_units;
    const int* done;
    PairArgs a;
};
constexpr int MAX_PAIR_JOBS = 64;   // problems in one batched pair launch

// Launch state of a single-problem pair launch.
struct PairLaunch {
    const int* unit_start;
    const int* n_units;
    int* unit_counter;        // zeroed by the caller
    const int* done;          // LM state flag or NULL
    int num_sms;
    int ctas_per_sm;          // 0: as many as fit
    cudaStream_t stream;
};

struct LMState {
    double lambda;
    double F_cur, F_cand;
    double step_inf;
    double tol_step, tol_rel_f;
    long long pair_terms;     // summed over evaluations of the solve
    long long n_cand;         // pair-terms of the last evaluation
    int iters, max_iters;
    int done, status;         // status: 0 converged, 4 not converged
    int first, chol_fail, accepted;
    int n_accepted;           // accepted steps after the first evaluation
};

// ------------------------------------------------------------ launchers ----
// scan.cu
size_t scan_ws_elems(long long n);   // long longs of the radix sort's small workspace
// Stable LSD sort of the low nbits of keys (payload vals); ends in the *_alt
// buffers when *in_alt.  hist: radix_hist_elems(n) long longs; ws:
// scan_ws_elems(n); *err |= 1 if a bounded wait of the look-back gave up.
void radix_sort_u32(uint32_t* keys, int* vals, uint32_t* keys_alt, int* vals_alt, long long n,
                    int nbits, long long* hist, long long* ws, int* err, cudaStream_t st, bool* in_alt);
size_t radix_hist_elems(long long n);

// grid.cu
void launch_bbox(const double* xyz, const float* sem, const float* rgb, long long N, int K,
                 const long long* pt_off, int sem_dim, double h_inv, int* cmin, int* cmax,
                 unsigned* sem_norm_bits, int* err, cudaStream_t st);
void launch_keys(const double* xyz, long long N, int K, const long long* pt_off,
                 const FrameDev* frames, double h_inv, uint32_t* keys, int* vals, cudaStream_t st);
void launch_gather(const double* xyz, const float* sem, const float* rgb, long long N, int K,
                   const long long* pt_off, const uint32_t* keys, const int* perm, GridParams gp,
                   long long C_total, float4* pts4, void* sem_sorted, float4* col4,
                   int* perm_local, int* cell_start, long long* run_flag, cudaStream_t st);

// pairs.cu
void launch_edge_setup(const double* poses, const EdgeDev* edges, int E, const FrameDev* frames,
                       double h, EdgeXf* xf, const int* done, cudaStream_t st);
void launch_query_keys(const EdgeDev* edges, int E, const FrameDev* frames, const EdgeXf* xf,
                       const uint32_t* pt_cell, const float4* pts4, GridParams gp, long long Q,
                       uint32_t* qkey, int* qval, float4* qrec, const int* done, cudaStream_t st);
void launch_query_gather(const uint32_t* qkey_sorted, const int* qval_sorted, const float4* qrec,
                         long long Q, int sub, float4* slots, int* bin_first, const int* done,
                         cudaStream_t st);
void launch_units(const uint32_t* qkey_sorted, const int* bin_first, long long Q, int uq, int sub, int* unit_start,
                  int* n_units, const int* done, cudaStream_t st);
void launch_pairs(const PairLaunch& L, const PairArgs& A);
// Largest unit (queries of one home cell per warp) the pair kernel of this
// layout takes: 64 for the dense tile kernel with BF16 labels, else 32.
int pair_unit_max(const GridParams& gp);
// One persistent launch over the units of n_jobs problems (device array
// `jobs`) that share the label layout, colour use and variant of `layout`,
// with units of at most max_uq queries; false when the layout has no batched
// kernel (top_k variant) or n_jobs is out of range.  *counter must be zero.
bool launch_pairs_multi(const PairJob* jobs, int n_jobs, const GridParams& layout, int max_uq, int* counter,
                        int num_sms, int ctas_per_sm, cudaStream_t st);
void launch_emit_pairs(const int* unit_start, const int* n_units, int* unit_counter,
                       const uint32_t* qkey, const float4* slots, long long Q, const EdgeDev* edges,
                       int E, const FrameDev* frames, const int* cell_start, const float4* pts4,
                       GridParams gp, int edge_sel, const int* perm_local, long long capacity, int uq,
                       int* i_out, int* j_out, unsigned long long* n_out, int num_sms,
                       cudaStream_t st);

// solve.cu
void launch_edge_assemble(const EdgeDev* edges, int E, const EdgeXf* xf, const long long* acc,
                          double sigma2, EdgeOut* out, const int* done, cudaStream_t st);
void launch_frame_assemble(const EdgeDev* edges, int E, int K, const int* inc_off,
                           const int* inc_list, const EdgeOut* eout, double* H, double* b,
                           double* F, long long* npairs, const int* done, cudaStream_t st);
void launch_lm_solve(int K, const double* H_cur, const double* b_cur, const double* poses_cur,
                     double* poses_cand, LMState* st_dev, double* ws, cudaStream_t st);
void launch_lm_accept(int K, LMState* st_dev, const double* F_cand, const long long* n_cand,
                      double* poses_cur, const double* poses_cand, double* b_cur,
                      const double* b_cand, cudaStream_t st);
void launch_copy_if_accepted(const LMState* st_dev, double* dst, const double* src,
                             long long n, cudaStream_t st);

}  // namespace rk

#include "rkhsba.h"

namespace rk {
// api.cu: sets the message returned by rkhsba_last_error(NULL) on this thread
void set_thread_error(const char* msg);

// api.cu: asynchronous LM stepping of a context (used by the request server)
rkhsba_status ctx_begin_solve(rkhsba_ctx* c, const double* host_poses);
void ctx_iterate(rkhsba_ctx* c, int n);
cudaStream_t ctx_stream(const rkhsba_ctx* c);
const void* ctx_state_dev(const rkhsba_ctx* c);
const double* ctx_poses_dev(const rkhsba_ctx* c);
size_t ctx_bytes(const rkhsba_ctx* c);
int ctx_max_iters(const rkhsba_ctx* c);
int ctx_state_bytes();
// batched serving: the LM iteration split around the pair stage
void ctx_iter_pre(rkhsba_ctx* c);
void ctx_iter_post(rkhsba_ctx* c);
PairJob ctx_pair_job(const rkhsba_ctx* c);
GridParams ctx_layout(const rkhsba_ctx* c);
int ctx_num_sms(const rkhsba_ctx* c);
int ctx_tune_ctas(const rkhsba_ctx* c);
int ctx_tune_uq(const rkhsba_ctx* c);
}  // namespace rk
