// C ABI of the RKHS-BA hot path (declared in include/rkhsba.h).
//
// A context owns one problem on one GPU: the raw frame-local points, the
// per-frame grids (grid step), the per-evaluation binning buffers, the FP64
// Gauss-Newton system and the LM state.  Host code here only validates
// arguments, sizes buffers and issues kernels; every step of the objective,
// its derivatives and the solve runs on the device.
#include "context.cuh"
#include "layout.cuh"
#include "rkhsba.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <set>
#include <string>
#include <utility>
#include <vector>

namespace rk {
std::atomic<long long> g_launches{0};
thread_local long long t_launches = 0;
}

using namespace rk;

namespace {
thread_local std::string t_err;

rkhsba_status fail(rkhsba_ctx* ctx, rkhsba_status s, const std::string& msg) {
    t_err = msg;
    if (ctx) ctx->err = msg;
    return s;
}


template <typename T>
rkhsba_status alloc(rkhsba_ctx* ctx, T** out, long long count) {
    size_t bytes = (size_t)std::max<long long>(count, 1) * sizeof(T);
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, RKHSBA_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                            cudaGetErrorString(e));
    }
    ctx->bufs.push_back({p, bytes});
    ctx->bytes += bytes;
    *out = static_cast<T*>(p);
    return RKHSBA_OK;
}

rkhsba_status normalize_params(rkhsba_ctx* ctx, const rkhsba_params* in) {
    if (!in) return fail(ctx, RKHSBA_EINVAL, "params is NULL");
    rkhsba_params p = *in;
    if (!(p.ell > 0.0) || !std::isfinite(p.ell)) return fail(ctx, RKHSBA_EINVAL, "params.ell must be > 0");
    if (p.cutoff_mult == 0.0) p.cutoff_mult = 3.0;
    if (!(p.cutoff_mult > 0.0) || !std::isfinite(p.cutoff_mult))
        return fail(ctx, RKHSBA_EINVAL, "params.cutoff_mult must be finite and > 0");
    if (p.sigma == 0.0) p.sigma = 1.0;
    if (!std::isfinite(p.sigma)) return fail(ctx, RKHSBA_EINVAL, "params.sigma must be finite");
    if (p.sem_dim < 0 || p.sem_dim > MAX_SEM)
        return fail(ctx, RKHSBA_EINVAL, "params.sem_dim must be in [0, 32]");
    if (p.max_iters == 0) p.max_iters = 100;
    if (p.max_iters < 0) return fail(ctx, RKHSBA_EINVAL, "params.max_iters must be >= 0");
    if (p.lambda0 == 0.0) p.lambda0 = 1e-4;
    if (p.tol_step == 0.0) p.tol_step = 1e-10;
    if (p.tol_rel_f == 0.0) p.tol_rel_f = 1e-12;
    if (p.top_k < 0 || p.top_k > TOPK_MAX) return fail(ctx, RKHSBA_EINVAL, "params.top_k must be in [0, 8]");
    if (!(p.sem_min >= 0.0) || !std::isfinite(p.sem_min))
        return fail(ctx, RKHSBA_EINVAL, "params.sem_min must be finite and >= 0");
    if (p.cell_scale == 0.0) p.cell_scale = 1.0;
    if (!(p.cell_scale >= 1.0 && p.cell_scale <= 4.0))
        return fail(ctx, RKHSBA_EINVAL, "params.cell_scale must be in [1, 4]");
    ctx->p = p;
    ctx->gp = grid_params_for(p);
    const GridParams& g = ctx->gp;
    if (p.sem_dim > 0 && g.sem_pad == 0) return fail(ctx, RKHSBA_EINVAL, "unsupported sem_dim");
    return RKHSBA_OK;
}

rkhsba_status check_shape(rkhsba_ctx* ctx, int32_t n_frames, const int64_t* n_points, int32_t n_edges,
                          const int32_t* edges, bool allow_self = false) {
    if (n_frames < 1 || n_frames > 4096) return fail(ctx, RKHSBA_EINVAL, "n_frames must be in [1, 4096]");
    if (!n_points) return fail(ctx, RKHSBA_EINVAL, "n_points is NULL");
    if (n_edges < 1) return fail(ctx, RKHSBA_EINVAL, "the pose graph needs at least one edge");
    if (!edges) return fail(ctx, RKHSBA_EINVAL, "edges is NULL");
    ctx->K = n_frames;
    ctx->pt_off.assign(n_frames + 1, 0);
    for (int m = 0; m < n_frames; ++m) {
        if (n_points[m] < 0) return fail(ctx, RKHSBA_EINVAL, "negative point count");
        ctx->pt_off[m + 1] = ctx->pt_off[m] + n_points[m];
        if (ctx->pt_off[m + 1] >= (1LL << 31) - 64) return fail(ctx, RKHSBA_EINVAL, "more than 2^31 points");
    }
    ctx->N = ctx->pt_off[n_frames];
    std::set<std::pair<int, int>> seen;
    ctx->E = n_edges;
    ctx->edges_h.assign(n_edges, EdgeDev{});
    ctx->edge_in.clear();
    for (int e = 0; e < n_edges; ++e) {
        int a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= n_frames || b >= n_frames)
            return fail(ctx, RKHSBA_EINVAL, "edge " + std::to_string(e) + " names a missing frame");
        if (a == b && !allow_self)
            return fail(ctx, RKHSBA_EINVAL, "edge " + std::to_string(e) + " is a self-edge");
        ctx->edge_in.push_back({a, b});
        if (a > b) std::swap(a, b);
        if (!seen.insert({a, b}).second)
            return fail(ctx, RKHSBA_EINVAL, "edge " + std::to_string(e) + " duplicates an earlier edge");
        ctx->edges_h[e].a = a;
        ctx->edges_h[e].b = b;
    }
    return RKHSBA_OK;
}

void grid_fill(rkhsba_ctx* c, bool* keys_in_alt) {
    cudaStream_t st = c->stream;
    launch_keys(c->d_xyz, c->N, c->K, c->d_pt_off, c->d_frames, c->gp.h_inv, c->d_keys, c->d_vals, st);
    int nbits = 0;
    while ((1LL << nbits) < c->C_total) ++nbits;
    bool alt = false;
    radix_sort_u32(c->d_keys, c->d_vals, c->d_keys_alt, c->d_vals_alt, c->N, nbits, c->d_hist,
                   c->d_scan_ws, c->d_err + 1, st, &alt);
    const uint32_t* keys = alt ? c->d_keys_alt : c->d_keys;
    const int* perm = alt ? c->d_vals_alt : c->d_vals;
    launch_gather(c->d_xyz, c->d_sem_in, c->d_rgb_in, c->N, c->K, c->d_pt_off, keys, perm, c->gp,
                  c->C_total, c->d_pts4, c->d_sem, c->d_col4, c->d_perm_local, c->d_cell_start,
                  c->d_run, st);
    c->d_pt_cell = keys;
    *keys_in_alt = alt;
}

// Freed context memory stays in the device's default pool for the next
// context instead of going back to the driver (set once per device).
void keep_pool_warm(int dev) {
    static std::once_flag flags[64];
    if (dev < 0 || dev >= 64) return;
    std::call_once(flags[dev], [dev] {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            unsigned long long thr = ~0ULL;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

rkhsba_status build(rkhsba_ctx* c, const double* xyz, const float* sem, const float* rgb, bool on_device,
                    void* stream) {
    const long long N = c->N;
    const int K = c->K, E = c->E;
    int dev = 0;
    RK_CUDA(c, cudaGetDevice(&dev));
    RK_CUDA(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
    keep_pool_warm(dev);
    if (const char* ng = std::getenv("RKHSBA_NO_GRAPHS")) c->use_graph = ng[0] == '0';
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        RK_CUDA(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    cudaStream_t st = c->stream;
    const bool has_sem = c->p.sem_dim > 0;
    if (has_sem != (sem != nullptr))
        return fail(c, RKHSBA_EINVAL, "sem must be given exactly when params.sem_dim > 0");
    grid_params_color(c->gp, rgb != nullptr && c->p.ell_color > 0.0, c->p.ell_color);
    const float* rgb_used = c->gp.color ? rgb : nullptr;

    // raw inputs
    RK_TRY(alloc(c, &c->d_xyz, 3 * N));
    RK_CUDA(c, cudaMemcpyAsync(c->d_xyz, xyz, sizeof(double) * 3 * N,
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (has_sem) {
        RK_TRY(alloc(c, &c->d_sem_in, (long long)c->p.sem_dim * N));
        RK_CUDA(c, cudaMemcpyAsync(c->d_sem_in, sem, sizeof(float) * c->p.sem_dim * N,
                                   on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    }
    if (rgb_used) {
        RK_TRY(alloc(c, &c->d_rgb_in, 3 * N));
        RK_CUDA(c, cudaMemcpyAsync(c->d_rgb_in, rgb_used, sizeof(float) * 3 * N,
                                   on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    }
    RK_TRY(alloc(c, &c->d_pt_off, K + 1));
    RK_CUDA(c, cudaMemcpyAsync(c->d_pt_off, c->pt_off.data(), sizeof(long long) * (K + 1),
                               cudaMemcpyHostToDevice, st));
    RK_TRY(alloc(c, &c->d_cmin, 3 * K));
    RK_TRY(alloc(c, &c->d_cmax, 3 * K));
    RK_TRY(alloc(c, &c->d_semnorm, K));
    RK_TRY(alloc(c, &c->d_err, 4));
    std::vector<int> big(3 * K, 0x7fffffff), small(3 * K, (int)0x80000000);
    RK_CUDA(c, cudaMemcpyAsync(c->d_cmin, big.data(), sizeof(int) * 3 * K, cudaMemcpyHostToDevice, st));
    RK_CUDA(c, cudaMemcpyAsync(c->d_cmax, small.data(), sizeof(int) * 3 * K, cudaMemcpyHostToDevice, st));
    RK_CUDA(c, cudaMemsetAsync(c->d_semnorm, 0, sizeof(unsigned) * K, st));
    RK_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(int) * 4, st));
    launch_bbox(c->d_xyz, c->d_sem_in, c->d_rgb_in, N, K, c->d_pt_off, c->p.sem_dim, c->gp.h_inv,
                c->d_cmin, c->d_cmax, c->d_semnorm, c->d_err, st);
    std::vector<int> cmin(3 * K), cmax(3 * K);
    std::vector<unsigned> semn(K);
    int errbits = 0;
    RK_CUDA(c, cudaMemcpyAsync(cmin.data(), c->d_cmin, sizeof(int) * 3 * K, cudaMemcpyDeviceToHost, st));
    RK_CUDA(c, cudaMemcpyAsync(cmax.data(), c->d_cmax, sizeof(int) * 3 * K, cudaMemcpyDeviceToHost, st));
    RK_CUDA(c, cudaMemcpyAsync(semn.data(), c->d_semnorm, sizeof(unsigned) * K, cudaMemcpyDeviceToHost, st));
    RK_CUDA(c, cudaMemcpyAsync(&errbits, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RK_CUDA(c, cudaStreamSynchronize(st));
    if (errbits & 1) return fail(c, RKHSBA_EINVAL, "non-finite point coordinate");
    if (errbits & 2) return fail(c, RKHSBA_EINVAL, "point coordinate beyond 2^29 grid cells");
    if (errbits & 4) return fail(c, RKHSBA_EINVAL, "non-finite label value");
    if (errbits & 8) return fail(c, RKHSBA_EINVAL, "non-finite colour value");

    // grid layout per frame (dense, one-cell margin)
    c->frames_h.assign(K, FrameDev{});
    if (const char* msg = layout_frames(c->frames_h.data(), K, c->pt_off.data(), cmin.data(), cmax.data(),
                                        semn.data(), has_sem, 1LL << 20, 1LL << 30, (1LL << 31) - 2,
                                        &c->C_total))
        return fail(c, RKHSBA_EINVAL, std::string(msg) + " (2^20 per axis, 2^30 per frame, 2^31 in all)");
    RK_TRY(alloc(c, &c->d_frames, K));
    RK_CUDA(c, cudaMemcpyAsync(c->d_frames, c->frames_h.data(), sizeof(FrameDev) * K,
                               cudaMemcpyHostToDevice, st));

    // grid buffers
    const int sp = c->gp.sem_pad;
    RK_TRY(alloc(c, &c->d_keys, N));
    RK_TRY(alloc(c, &c->d_keys_alt, N));
    RK_TRY(alloc(c, &c->d_vals, N));
    RK_TRY(alloc(c, &c->d_vals_alt, N));
    RK_TRY(alloc(c, &c->d_hist, (long long)radix_hist_elems(N)));
    RK_TRY(alloc(c, &c->d_cell_start, c->C_total + 1));
    RK_TRY(alloc(c, &c->d_pts4, N));
    if (sp > 0) {
        char* p = nullptr;
        RK_TRY(alloc(c, &p, (long long)N * sp * (c->gp.sem_bf16 ? 2 : 4)));
        c->d_sem = p;
    }
    if (c->gp.color) RK_TRY(alloc(c, &c->d_col4, N));
    RK_TRY(alloc(c, &c->d_perm_local, N));
    RK_TRY(alloc(c, &c->d_run, N));
    RK_TRY(alloc(c, &c->d_total, 4));

    // per-edge sizes (bins = cells of frame a's grid, queries = points of
    // frame b) and fixed-point scales
    const double rc = c->p.cutoff_mult * c->p.ell;
    layout_edges(c->edges_h.data(), E, c->frames_h.data(), c->gp, rc, &c->total_bins, &c->Q_total);
    if (c->total_bins >= (1LL << 31) - 2) return fail(c, RKHSBA_EINVAL, "total home cells exceed 2^31");
    if (c->Q_total >= (1LL << 31) - 64) return fail(c, RKHSBA_EINVAL, "more than 2^31 queries over all edges");
    c->qbits = 1;
    while ((1LL << c->qbits) <= c->total_bins) ++c->qbits;   // invalid key sorts last
    // three more key bits order a home cell's queries by octant, when they fit
    c->gp.key_sub = (c->qbits + 3 <= 31) ? 3 : 0;
    c->qbits += c->gp.key_sub;
    long long scan_n = std::max<long long>((long long)radix_hist_elems(N),
                                           (long long)radix_hist_elems(c->Q_total));
    RK_TRY(alloc(c, &c->d_scan_ws, (long long)scan_ws_elems(scan_n) + 64));
    RK_CUDA(c, cudaMemsetAsync(c->d_cell_start, 0, sizeof(int) * (c->C_total + 1), st));
    bool alt = false;
    grid_fill(c, &alt);
    RK_CUDA(c, cudaGetLastError());

    RK_TRY(alloc(c, &c->d_edges, E));
    RK_CUDA(c, cudaMemcpyAsync(c->d_edges, c->edges_h.data(), sizeof(EdgeDev) * E,
                               cudaMemcpyHostToDevice, st));
    // incidence lists (frame -> edges), edge order kept
    std::vector<int> inc_off(K + 1, 0), inc_list(2 * (size_t)E + 1, 0);
    inc_list.resize(incidence_lists(c->edges_h.data(), E, K, inc_off.data(), inc_list.data()));
    RK_TRY(alloc(c, &c->d_inc_off, K + 1));
    RK_TRY(alloc(c, &c->d_inc_list, (long long)inc_list.size()));
    RK_CUDA(c, cudaMemcpyAsync(c->d_inc_off, inc_off.data(), sizeof(int) * (K + 1), cudaMemcpyHostToDevice, st));
    RK_CUDA(c, cudaMemcpyAsync(c->d_inc_list, inc_list.data(), sizeof(int) * inc_list.size(),
                               cudaMemcpyHostToDevice, st));

    // evaluation buffers
    const long long Q = c->Q_total;
    RK_TRY(alloc(c, &c->d_xf, E));
    RK_TRY(alloc(c, &c->d_qkey, Q));
    RK_TRY(alloc(c, &c->d_qkey_alt, Q));
    RK_TRY(alloc(c, &c->d_qval, Q));
    RK_TRY(alloc(c, &c->d_qval_alt, Q));
    RK_TRY(alloc(c, &c->d_qhist, (long long)radix_hist_elems(Q)));
    RK_TRY(alloc(c, &c->d_qrec, Q));
    RK_TRY(alloc(c, &c->d_slots, Q));
    RK_TRY(alloc(c, &c->d_bin_first, c->total_bins));
    RK_TRY(alloc(c, &c->d_unit_start, Q));
    RK_TRY(alloc(c, &c->d_ucount, 4));
    RK_TRY(alloc(c, &c->d_acc, (long long)E * ACC_N));
    RK_TRY(alloc(c, &c->d_eout, E));
    const long long n6 = 6LL * K;
    RK_TRY(alloc(c, &c->d_H_cand, n6 * n6));
    RK_TRY(alloc(c, &c->d_H_cur, n6 * n6));
    RK_TRY(alloc(c, &c->d_b_cand, n6));
    RK_TRY(alloc(c, &c->d_b_cur, n6));
    RK_TRY(alloc(c, &c->d_F_cand, 1));
    RK_TRY(alloc(c, &c->d_n_cand, 1));
    RK_TRY(alloc(c, &c->d_poses_cur, 16LL * K));
    RK_TRY(alloc(c, &c->d_poses_cand, 16LL * K));
    RK_TRY(alloc(c, &c->d_state, 1));
    const long long nf = 6LL * (K - 1);
    RK_TRY(alloc(c, &c->d_lm_ws, nf * nf + 2 * nf + 16));
    RK_CUDA(c, cudaMemsetAsync(c->d_state, 0, sizeof(LMState), st));
    RK_CUDA(c, cudaStreamSynchronize(st));
    RK_CUDA(c, cudaGetLastError());
    return RKHSBA_OK;
}

// Transform and bin the queries of every edge at the device poses `poses`:
// sorted home-cell keys, sorted query records and the unit list.
void run_binning(rkhsba_ctx* c, const double* poses, const int* done) {
    cudaStream_t st = c->stream;
    launch_edge_setup(poses, c->d_edges, c->E, c->d_frames, c->gp.h, c->d_xf, done, st);
    cudaMemsetAsync(c->d_ucount, 0, sizeof(int) * 4, st);
    launch_query_keys(c->d_edges, c->E, c->d_frames, c->d_xf, c->d_pt_cell, c->d_pts4, c->gp, c->Q_total,
                      c->d_qkey, c->d_qval, c->d_qrec, done, st);
    bool alt = false;
    radix_sort_u32(c->d_qkey, c->d_qval, c->d_qkey_alt, c->d_qval_alt, c->Q_total, c->qbits, c->d_qhist,
                   c->d_scan_ws, c->d_err + 1, st, &alt);
    c->q_sorted_key = alt ? c->d_qkey_alt : c->d_qkey;
    const int* qv = alt ? c->d_qval_alt : c->d_qval;
    launch_query_gather(c->q_sorted_key, qv, c->d_qrec, c->Q_total, c->gp.key_sub, c->d_slots, c->d_bin_first, done,
                        st);
    launch_units(c->q_sorted_key, c->d_bin_first, c->Q_total, c->tune_uq, c->gp.key_sub, c->d_unit_start,
                 c->d_ucount, done, st);
}

// One evaluation at the device poses `poses`, results into the cand
// buffers, in three parts: binning (queries keyed, sorted and cut into
// units; accumulators cleared), the pair stage, and the FP64 assembly.
void eval_pre(rkhsba_ctx* c, const double* poses, const int* done) {
    c->phase_begin(1);
    run_binning(c, poses, done);
    cudaMemsetAsync(c->d_acc, 0, sizeof(long long) * c->E * ACC_N, c->stream);
    c->phase_end();
}

void eval_pairs(rkhsba_ctx* c, const int* done) {
    c->phase_begin(2);
    launch_pairs(PairLaunch{c->d_unit_start, c->d_ucount, c->d_ucount + 1, done, c->num_sms, c->tune_ctas,
                            c->stream},
                 c->pair_args());
    c->phase_end();
}

void eval_post(rkhsba_ctx* c, const int* done) {
    cudaStream_t st = c->stream;
    c->phase_begin(3);
    launch_edge_assemble(c->d_edges, c->E, c->d_xf, c->d_acc, c->p.sigma * c->p.sigma, c->d_eout, done, st);
    cudaMemsetAsync(c->d_H_cand, 0, sizeof(double) * 36LL * c->K * c->K, st);
    launch_frame_assemble(c->d_edges, c->E, c->K, c->d_inc_off, c->d_inc_list, c->d_eout, c->d_H_cand,
                          c->d_b_cand, c->d_F_cand, c->d_n_cand, done, st);
    c->phase_end();
}

void run_eval(rkhsba_ctx* c, const double* poses, const int* done) {
    eval_pre(c, poses, done);
    eval_pairs(c, done);
    eval_post(c, done);
}

rkhsba_status check_poses(rkhsba_ctx* c, const double* poses) {
    if (!poses) return fail(c, RKHSBA_EINVAL, "poses is NULL");
    for (int m = 0; m < c->K; ++m) {
        const double* T = poses + 16 * m;
        for (int k = 0; k < 16; ++k)
            if (!std::isfinite(T[k])) return fail(c, RKHSBA_EINVAL, "non-finite pose entry");
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += T[4 * k + i] * T[4 * k + j];
                if (std::fabs(s - (i == j ? 1.0 : 0.0)) > 1e-9)
                    return fail(c, RKHSBA_EINVAL, "pose " + std::to_string(m) + " has a non-orthonormal rotation");
            }
        if (T[12] != 0.0 || T[13] != 0.0 || T[14] != 0.0 || T[15] != 1.0)
            return fail(c, RKHSBA_EINVAL, "pose " + std::to_string(m) + " last row is not [0 0 0 1]");
    }
    return RKHSBA_OK;
}

void reset_state(rkhsba_ctx* c) {
    LMState s{};
    s.lambda = c->p.lambda0;
    s.tol_step = c->p.tol_step;
    s.tol_rel_f = c->p.tol_rel_f;
    s.max_iters = c->p.max_iters;
    s.first = 1;
    s.status = 4;
    cudaMemcpyAsync(c->d_state, &s, sizeof(LMState), cudaMemcpyHostToDevice, c->stream);
    c->need_initial = true;
}

void lm_initial(rkhsba_ctx* c) {
    const int* done = &c->d_state->done;
    run_eval(c, c->d_poses_cand, done);
    c->phase_begin(4);
    launch_lm_accept(c->K, c->d_state, c->d_F_cand, c->d_n_cand, c->d_poses_cur, c->d_poses_cand,
                     c->d_b_cur, c->d_b_cand, c->stream);
    launch_copy_if_accepted(c->d_state, c->d_H_cur, c->d_H_cand, 36LL * c->K * c->K, c->stream);
    c->phase_end();
    c->need_initial = false;
}

// One LM iteration in two halves around the pair stage: the damped solve
// and the binning at the candidate poses; then the assembly and the
// accept/reject of the candidate.
void lm_iter_pre(rkhsba_ctx* c) {
    const int* done = &c->d_state->done;
    c->phase_begin(4);
    launch_lm_solve(c->K, c->d_H_cur, c->d_b_cur, c->d_poses_cur, c->d_poses_cand, c->d_state,
                    c->d_lm_ws, c->stream);
    c->phase_end();
    eval_pre(c, c->d_poses_cand, done);
}

void lm_iter_post(rkhsba_ctx* c) {
    const int* done = &c->d_state->done;
    eval_post(c, done);
    c->phase_begin(4);
    launch_lm_accept(c->K, c->d_state, c->d_F_cand, c->d_n_cand, c->d_poses_cur, c->d_poses_cand,
                     c->d_b_cur, c->d_b_cand, c->stream);
    launch_copy_if_accepted(c->d_state, c->d_H_cur, c->d_H_cand, 36LL * c->K * c->K, c->stream);
    c->phase_end();
}

void lm_iteration(rkhsba_ctx* c) {
    lm_iter_pre(c);
    eval_pairs(c, &c->d_state->done);
    lm_iter_post(c);
}

// Captures fn (kernels on the context stream) into *exec once; false when
// capture is not possible (the caller then launches fn directly).
template <typename Fn>
bool capture_graph(rkhsba_ctx* c, cudaGraphExec_t* exec, long long* kernels, Fn fn) {
    cudaGraph_t g = nullptr;
    const long long before = t_launches;
    bool ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        fn();
        ok = cudaStreamEndCapture(c->stream, &g) == cudaSuccess && g != nullptr;
    }
    if (ok) ok = cudaGraphInstantiate(exec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    const long long n = t_launches - before;   // captured, not run
    g_launches.fetch_sub(n);
    t_launches = before;
    if (!ok) {
        cudaGetLastError();
        *exec = nullptr;
        return false;
    }
    *kernels = n;
    return true;
}

// n LM iterations.  After the first evaluation has run (kernel attributes and
// occupancy are then settled), one iteration is captured into a CUDA graph
// and replayed, which removes the per-kernel launch cost of the ~30 small
// launches of an iteration.  With the phase profiler on, or when capture is
// not possible, the iterations are launched one kernel at a time.
void lm_iterate(rkhsba_ctx* c, int n) {
    if (n <= 0) return;
    if (c->prof || !c->use_graph) {
        for (int i = 0; i < n; ++i) lm_iteration(c);
        return;
    }
    if (!c->iter_graph) {
        if (!capture_graph(c, &c->iter_graph, &c->iter_launches, [&] { lm_iteration(c); })) {
            c->use_graph = false;
            for (int i = 0; i < n; ++i) lm_iteration(c);
            return;
        }
    }
    for (int i = 0; i < n; ++i) {
        cudaGraphLaunch(c->iter_graph, c->stream);
        count_launch(c->iter_launches);
    }
}

rkhsba_status create_impl(rkhsba_ctx** out, int32_t n_frames, const int64_t* n_points,
                          const double* xyz, const float* sem, const float* rgb, int32_t n_edges,
                          const int32_t* edges, const rkhsba_params* params, void* stream,
                          bool on_device, bool allow_self = false) {
    if (!out) return fail(nullptr, RKHSBA_EINVAL, "out is NULL");
    *out = nullptr;
    rkhsba_ctx* c = new rkhsba_ctx();
    rkhsba_status s = normalize_params(c, params);
    if (s == RKHSBA_OK) s = check_shape(c, n_frames, n_points, n_edges, edges, allow_self);
    if (s == RKHSBA_OK && c->N > 0 && !xyz) s = fail(c, RKHSBA_EINVAL, "xyz is NULL");
    if (s == RKHSBA_OK) s = build(c, xyz, sem, rgb, on_device, stream);
    if (s != RKHSBA_OK) {
        std::string msg = c->err;
        delete c;
        t_err = msg;
        return s;
    }
    *out = c;
    return RKHSBA_OK;
}
}  // namespace

// Internal stepping interface for the request server (server.cu): the same
// device-resident LM loop as rkhsba_solve, issued asynchronously.
namespace rk {
rkhsba_status ctx_fail(rkhsba_ctx* ctx, rkhsba_status s, const std::string& msg) { return fail(ctx, s, msg); }
void ctx_run_eval(rkhsba_ctx* c, const double* d_poses) { run_eval(c, d_poses, nullptr); }
rkhsba_status ctx_create(rkhsba_ctx** out, int32_t n_frames, const int64_t* n_points, const double* xyz,
                         const float* sem, const float* rgb, int32_t n_edges, const int32_t* edges,
                         const rkhsba_params* params, void* stream, bool on_device, bool allow_self) {
    return create_impl(out, n_frames, n_points, xyz, sem, rgb, n_edges, edges, params, stream, on_device,
                       allow_self);
}
rkhsba_status ctx_check_poses(rkhsba_ctx* c, const double* poses) { return check_poses(c, poses); }

rkhsba_status ctx_begin_solve(rkhsba_ctx* c, const double* host_poses) {
    RK_TRY(check_poses(c, host_poses));
    RK_CUDA(c, cudaMemcpyAsync(c->d_poses_cand, host_poses, sizeof(double) * 16 * c->K, cudaMemcpyHostToDevice,
                               c->stream));
    reset_state(c);
    lm_initial(c);
    RK_CUDA(c, cudaGetLastError());
    return RKHSBA_OK;
}
void ctx_iterate(rkhsba_ctx* c, int n) { lm_iterate(c, n); }

// The two halves of one LM iteration for the batched server, each replayed
// from a CUDA graph captured on first use; the pair stage between them runs
// in the server's batched launch.
void ctx_iter_pre(rkhsba_ctx* c) {
    if (c->use_graph && !c->prof) {
        if (c->pre_graph || capture_graph(c, &c->pre_graph, &c->pre_launches, [&] { lm_iter_pre(c); })) {
            cudaGraphLaunch(c->pre_graph, c->stream);
            count_launch(c->pre_launches);
            return;
        }
    }
    lm_iter_pre(c);
}
void ctx_iter_post(rkhsba_ctx* c) {
    if (c->use_graph && !c->prof) {
        if (c->post_graph || capture_graph(c, &c->post_graph, &c->post_launches, [&] { lm_iter_post(c); })) {
            cudaGraphLaunch(c->post_graph, c->stream);
            count_launch(c->post_launches);
            return;
        }
    }
    lm_iter_post(c);
}
PairJob ctx_pair_job(const rkhsba_ctx* c) {
    PairJob j{};
    j.unit_start = c->d_unit_start;
    j.n_units = c->d_ucount;
    j.done = &c->d_state->done;
    j.a = c->pair_args();
    return j;
}
GridParams ctx_layout(const rkhsba_ctx* c) { return c->gp; }
int ctx_num_sms(const rkhsba_ctx* c) { return c->num_sms; }
int ctx_tune_ctas(const rkhsba_ctx* c) { return c->tune_ctas; }
int ctx_tune_uq(const rkhsba_ctx* c) { return c->tune_uq; }
cudaStream_t ctx_stream(const rkhsba_ctx* c) { return c->stream; }
const void* ctx_state_dev(const rkhsba_ctx* c) { return c->d_state; }
const double* ctx_poses_dev(const rkhsba_ctx* c) { return c->d_poses_cur; }
size_t ctx_bytes(const rkhsba_ctx* c) { return c->bytes; }
int ctx_max_iters(const rkhsba_ctx* c) { return c->p.max_iters; }
int ctx_state_bytes() { return (int)sizeof(LMState); }
}  // namespace rk

extern "C" {

rkhsba_status rkhsba_create(rkhsba_ctx** out, int32_t n_frames, const int64_t* n_points,
                            const double* xyz, const float* sem, const float* rgb, int32_t n_edges,
                            const int32_t* edges, const rkhsba_params* params, void* cuda_stream) {
    return create_impl(out, n_frames, n_points, xyz, sem, rgb, n_edges, edges, params, cuda_stream, false);
}

rkhsba_status rkhsba_create_device(rkhsba_ctx** out, int32_t n_frames, const int64_t* n_points,
                                   const double* d_xyz, const float* d_sem, const float* d_rgb,
                                   int32_t n_edges, const int32_t* edges, const rkhsba_params* params,
                                   void* cuda_stream) {
    return create_impl(out, n_frames, n_points, d_xyz, d_sem, d_rgb, n_edges, edges, params, cuda_stream,
                       true);
}

void rkhsba_destroy(rkhsba_ctx* ctx) { delete ctx; }

rkhsba_status rkhsba_eval(rkhsba_ctx* c, const double* poses, double* loss, double* grad, double* H_full,
                          double* H_blocks, int64_t* edge_pairs) {
    if (!c) return fail(nullptr, RKHSBA_EINVAL, "ctx is NULL");
    RK_TRY(check_poses(c, poses));
    cudaStream_t st = c->stream;
    RK_CUDA(c, cudaMemcpyAsync(c->d_poses_cand, poses, sizeof(double) * 16 * c->K, cudaMemcpyHostToDevice, st));
    run_eval(c, c->d_poses_cand, nullptr);
    RK_CUDA(c, cudaGetLastError());
    double F = 0.0;
    int sort_err = 0;
    RK_CUDA(c, cudaMemcpyAsync(&sort_err, c->d_err + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    RK_CUDA(c, cudaMemcpyAsync(&F, c->d_F_cand, sizeof(double), cudaMemcpyDeviceToHost, st));
    std::vector<double> b;
    if (grad) {
        b.resize(6 * c->K);
        RK_CUDA(c, cudaMemcpyAsync(b.data(), c->d_b_cand, sizeof(double) * 6 * c->K, cudaMemcpyDeviceToHost, st));
    }
    if (H_full)
        RK_CUDA(c, cudaMemcpyAsync(H_full, c->d_H_cand, sizeof(double) * 36LL * c->K * c->K,
                                   cudaMemcpyDeviceToHost, st));
    std::vector<EdgeOut> eo;
    if (H_blocks || edge_pairs) {
        eo.resize(c->E);
        RK_CUDA(c, cudaMemcpyAsync(eo.data(), c->d_eout, sizeof(EdgeOut) * c->E, cudaMemcpyDeviceToHost, st));
    }
    RK_CUDA(c, cudaStreamSynchronize(st));
    if (sort_err) return fail(c, RKHSBA_ETIMEOUT, "a bounded wait of the radix sort gave up");
    if (loss) *loss = -F;
    if (grad) {
        const double scale = c->p.sigma * c->p.sigma / (c->p.ell * c->p.ell);
        for (int i = 0; i < 6 * c->K; ++i) grad[i] = scale * b[i];
    }
    for (int e = 0; e < c->E; ++e) {
        if (H_blocks) std::memcpy(H_blocks + 144LL * e, eo[e].H, sizeof(double) * 144);
        if (edge_pairs) edge_pairs[e] = eo[e].n;
    }
    return RKHSBA_OK;
}

rkhsba_status rkhsba_set_poses_device(rkhsba_ctx* c, const double* d_poses) {
    if (!c || !d_poses) return fail(c, RKHSBA_EINVAL, "NULL argument");
    RK_CUDA(c, cudaMemcpyAsync(c->d_poses_cand, d_poses, sizeof(double) * 16 * c->K,
                               cudaMemcpyDeviceToDevice, c->stream));
    reset_state(c);
    return RKHSBA_OK;
}

rkhsba_status rkhsba_rebuild(rkhsba_ctx* c) {
    if (!c) return fail(nullptr, RKHSBA_EINVAL, "ctx is NULL");
    bool alt = false;
    c->phase_begin(0);
    cudaMemsetAsync(c->d_cell_start, 0, sizeof(int) * (c->C_total + 1), c->stream);
    grid_fill(c, &alt);
    c->phase_end();
    RK_CUDA(c, cudaGetLastError());
    return RKHSBA_OK;
}

rkhsba_status rkhsba_iterate(rkhsba_ctx* c, int32_t n_iters) {
    if (!c) return fail(nullptr, RKHSBA_EINVAL, "ctx is NULL");
    if (c->need_initial) lm_initial(c);
    lm_iterate(c, n_iters);
    RK_CUDA(c, cudaGetLastError());
    return RKHSBA_OK;
}

rkhsba_status rkhsba_get_state(rkhsba_ctx* c, double* poses, rkhsba_solve_info* info) {
    if (!c) return fail(nullptr, RKHSBA_EINVAL, "ctx is NULL");
    LMState s{};
    int sort_err = 0;
    RK_CUDA(c, cudaMemcpyAsync(&s, c->d_state, sizeof(LMState), cudaMemcpyDeviceToHost, c->stream));
    RK_CUDA(c, cudaMemcpyAsync(&sort_err, c->d_err + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    if (poses)
        RK_CUDA(c, cudaMemcpyAsync(poses, c->d_poses_cur, sizeof(double) * 16 * c->K,
                                   cudaMemcpyDeviceToHost, c->stream));
    RK_CUDA(c, cudaStreamSynchronize(c->stream));
    if (sort_err) return fail(c, RKHSBA_ETIMEOUT, "a bounded wait of the radix sort gave up");
    if (info) {
        info->iters = s.iters;
        info->status = s.done ? s.status : RKHSBA_ENOTCONV;
        info->final_loss = -s.F_cur;
        info->lambda = s.lambda;
        info->pair_terms = s.pair_terms;
    }
    return RKHSBA_OK;
}

rkhsba_status rkhsba_solve(rkhsba_ctx* c, double* poses, rkhsba_solve_info* info) {
    if (!c) return fail(nullptr, RKHSBA_EINVAL, "ctx is NULL");
    RK_TRY(check_poses(c, poses));
    RK_CUDA(c, cudaMemcpyAsync(c->d_poses_cand, poses, sizeof(double) * 16 * c->K, cudaMemcpyHostToDevice,
                               c->stream));
    reset_state(c);
    lm_initial(c);
    // iterations are issued in small batches between reads of the device
    // state; once the device marks the solve done the remaining launches of a
    // batch return at once
    LMState s{};
    int issued = 0;
    while (issued < c->p.max_iters) {
        const int chunk = std::min(4, c->p.max_iters - issued);
        lm_iterate(c, chunk);
        issued += chunk;
        RK_CUDA(c, cudaMemcpyAsync(&s, c->d_state, sizeof(LMState), cudaMemcpyDeviceToHost, c->stream));
        RK_CUDA(c, cudaStreamSynchronize(c->stream));
        if (s.done) break;
    }
    RK_CUDA(c, cudaGetLastError());
    rkhsba_solve_info tmp{};
    RK_TRY(rkhsba_get_state(c, poses, &tmp));
    if (info) *info = tmp;
    return tmp.status == RKHSBA_OK ? RKHSBA_OK : RKHSBA_ENOTCONV;
}

rkhsba_status rkhsba_edge_pairs(rkhsba_ctx* c, const double* poses, int32_t edge, int64_t capacity,
                                int32_t* i_out, int32_t* j_out, int64_t* n_out) {
    if (!c) return fail(nullptr, RKHSBA_EINVAL, "ctx is NULL");
    if (edge < 0 || edge >= c->E) return fail(c, RKHSBA_EINVAL, "edge out of range");
    if (capacity < 0 || (capacity > 0 && (!i_out || !j_out)) || !n_out)
        return fail(c, RKHSBA_EINVAL, "bad output buffers");
    RK_TRY(check_poses(c, poses));
    cudaStream_t st = c->stream;
    RK_CUDA(c, cudaMemcpyAsync(c->d_poses_cand, poses, sizeof(double) * 16 * c->K, cudaMemcpyHostToDevice, st));
    run_binning(c, c->d_poses_cand, nullptr);
    int* di = nullptr;
    int* dj = nullptr;
    unsigned long long* dn = nullptr;
    cudaError_t e1 = cudaMalloc(&di, sizeof(int) * std::max<int64_t>(capacity, 1));
    cudaError_t e2 = cudaMalloc(&dj, sizeof(int) * std::max<int64_t>(capacity, 1));
    cudaError_t e3 = cudaMalloc(&dn, sizeof(unsigned long long));
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        cudaFree(di); cudaFree(dj); cudaFree(dn);
        cudaGetLastError();
        return fail(c, RKHSBA_ENOMEM, "pair list buffers");
    }
    cudaMemsetAsync(dn, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(c->d_ucount + 1, 0, sizeof(int), st);
    launch_emit_pairs(c->d_unit_start, c->d_ucount, c->d_ucount + 1, c->q_sorted_key, c->d_slots, c->Q_total,
                      c->d_edges, c->E, c->d_frames, c->d_cell_start, c->d_pts4, c->gp, edge, c->d_perm_local,
                      capacity, c->tune_uq, di, dj, dn, c->num_sms, st);
    unsigned long long n = 0;
    cudaMemcpyAsync(&n, dn, sizeof(n), cudaMemcpyDeviceToHost, st);
    cudaError_t es = cudaStreamSynchronize(st);
    long long m = std::min<long long>((long long)n, capacity);
    if (es == cudaSuccess && m > 0) {
        cudaMemcpy(i_out, di, sizeof(int) * m, cudaMemcpyDeviceToHost);
        cudaMemcpy(j_out, dj, sizeof(int) * m, cudaMemcpyDeviceToHost);
    }
    cudaFree(di); cudaFree(dj); cudaFree(dn);
    if (es != cudaSuccess) return fail(c, RKHSBA_ECUDA, cudaGetErrorString(es));
    // frame a of the device pair list is min(edge); report (a-index, b-index)
    *n_out = (int64_t)n;
    return RKHSBA_OK;
}

rkhsba_status rkhsba_profile(rkhsba_ctx* c, int32_t enable, double* ms, int64_t* launches) {
    if (!c) return fail(nullptr, RKHSBA_EINVAL, "ctx is NULL");
    if (ms || launches) {
        RK_CUDA(c, cudaStreamSynchronize(c->stream));
        double acc_ms[rkhsba_ctx::NPH] = {0, 0, 0, 0, 0};
        int64_t acc_n[rkhsba_ctx::NPH] = {0, 0, 0, 0, 0};
        for (auto& r : c->ev_rec) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, c->ev_pool[r.second.first], c->ev_pool[r.second.second]) ==
                cudaSuccess) {
                acc_ms[r.first] += t;
                acc_n[r.first] += 1;
            }
        }
        for (int i = 0; i < rkhsba_ctx::NPH; ++i) {
            if (ms) ms[i] = acc_ms[i];
            if (launches) launches[i] = acc_n[i];
        }
    }
    if (enable) {
        c->ev_rec.clear();
        c->prof = true;
    } else {
        c->prof = false;
    }
    return RKHSBA_OK;
}

rkhsba_status rkhsba_info(const rkhsba_ctx* c, int32_t* n_frames, int32_t* n_edges, int64_t* n_points_total,
                          int64_t* device_bytes) {
    if (!c) return fail(nullptr, RKHSBA_EINVAL, "ctx is NULL");
    if (n_frames) *n_frames = c->K;
    if (n_edges) *n_edges = c->E;
    if (n_points_total) *n_points_total = c->N;
    if (device_bytes) *device_bytes = (int64_t)c->bytes;
    return RKHSBA_OK;
}

const char* rkhsba_last_error(const rkhsba_ctx* c) {
    if (c) return c->err.c_str();
    return t_err.c_str();
}

int64_t rkhsba_launch_count(void) { return g_launches.load(); }

rkhsba_status rkhsba_set_tuning(rkhsba_ctx* c, int32_t unit_queries, int32_t ctas_per_sm) {
    if (!c) return fail(nullptr, RKHSBA_EINVAL, "ctx is NULL");
    if (unit_queries < 1 || unit_queries > pair_unit_max(c->gp))
        return fail(c, RKHSBA_EINVAL, "unit_queries must be in [1, 32] (up to 64 for BF16 labels without "
                                      "colour, pruning or top_k)");
    if (ctas_per_sm < 0 || ctas_per_sm > 32) return fail(c, RKHSBA_EINVAL, "ctas_per_sm must be in [0, 32]");
    c->tune_uq = unit_queries;
    c->tune_ctas = ctas_per_sm;
    c->drop_graphs();
    return RKHSBA_OK;
}

rkhsba_status rkhsba_get_tuning(const rkhsba_ctx* c, rkhsba_tuning* out) {
    if (!c || !out) return fail(nullptr, RKHSBA_EINVAL, "NULL argument");
    out->cell_scale = c->p.cell_scale;
    out->unit_queries = c->tune_uq;
    out->ctas_per_sm = c->tune_ctas;
    out->ms = 0.0;
    return RKHSBA_OK;
}

// The autotuner: for every candidate cell size a context is built over the
// caller's inputs (grid build at that cell size), and for every unit size
// and CTA count the evaluation at `poses` (binning, pair stage, FP64
// assembly) is timed with CUDA events on the stream after one untimed run,
// over at least `reps` evaluations and at least 20 ms.  The default setting
// (the first candidate) is kept unless another is faster by more than 3%,
// so timing noise on small problems does not move it.
rkhsba_status rkhsba_autotune(int32_t n_frames, const int64_t* n_points, const double* xyz, const float* sem,
                              const float* rgb, int32_t n_edges, const int32_t* edges,
                              const rkhsba_params* params, int32_t inputs_on_device, const double* poses,
                              void* cuda_stream, int32_t reps, rkhsba_tuning* best, rkhsba_tuning* table,
                              int32_t table_cap, int32_t* n_table) {
    if (!params || !poses || !best) return fail(nullptr, RKHSBA_EINVAL, "NULL argument");
    if (reps < 1 || reps > 100) return fail(nullptr, RKHSBA_EINVAL, "reps must be in [1, 100]");
    if (table_cap < 0 || (table_cap > 0 && !table)) return fail(nullptr, RKHSBA_EINVAL, "bad table");
    // the default setting (cell_scale 1, 32 queries per unit, all CTAs that
    // fit) is timed first
    static const double scales[] = {1.0, 1.25, 1.5};
    static const int uqs_all[] = {32, 16, 64};   // 64 only where the pair kernel takes it
    static const int ctas[] = {0, 1};
    int n = 0;
    best->ms = -1.0;
    rkhsba_tuning dflt{};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return fail(nullptr, RKHSBA_ECUDA, "event creation failed");
    }
    rkhsba_status st = RKHSBA_OK;
    for (double sc : scales) {
        rkhsba_params p = *params;
        p.cell_scale = sc;
        rkhsba_ctx* c = nullptr;
        st = create_impl(&c, n_frames, n_points, xyz, sem, rgb, n_edges, edges, &p, cuda_stream,
                         inputs_on_device != 0);
        if (st != RKHSBA_OK) break;
        st = check_poses(c, poses);
        if (st == RKHSBA_OK) {
            cudaMemcpyAsync(c->d_poses_cand, poses, sizeof(double) * 16 * c->K, cudaMemcpyHostToDevice, c->stream);
            for (int uq : uqs_all)
                for (int ct : ctas) {
                    if (uq > pair_unit_max(c->gp)) continue;
                    c->tune_uq = uq;
                    c->tune_ctas = ct;
                    float ms = 0.f, ms0 = 0.f;
                    cudaEventRecord(e0, c->stream);
                    run_eval(c, c->d_poses_cand, nullptr);     // untimed: its duration sizes the repeats
                    cudaEventRecord(e1, c->stream);
                    int nrep = reps;
                    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms0, e0, e1) == cudaSuccess &&
                        ms0 > 0.f)
                        nrep = std::max(reps, std::min(100, (int)std::ceil(20.0 / ms0)));
                    cudaEventRecord(e0, c->stream);
                    for (int r = 0; r < nrep; ++r) run_eval(c, c->d_poses_cand, nullptr);
                    cudaEventRecord(e1, c->stream);
                    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        st = fail(c, RKHSBA_ECUDA, "autotune timing failed");
                        break;
                    }
                    rkhsba_tuning t{sc, uq, ct, (double)ms / nrep};
                    if (n < table_cap) table[n] = t;
                    if (n == 0) dflt = t;
                    ++n;
                    if (best->ms < 0.0 || t.ms < best->ms) *best = t;
                }
        }
        if (st != RKHSBA_OK) {
            std::string msg = c->err;
            delete c;
            t_err = msg;
            break;
        }
        delete c;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_table) *n_table = n;
    if (st == RKHSBA_OK && n > 0 && !(best->ms < 0.97 * dflt.ms)) *best = dflt;
    return st;
}

}  // extern "C"

namespace rk {
// Message of the last context-free failure on this thread (read back through
// rkhsba_last_error(NULL)); used by entry points defined in other files.
void set_thread_error(const char* msg) { t_err = msg ? msg : ""; }
}  // namespace rk
