// Internal: the context of one problem and the host helpers shared by the
// translation units that drive it (api.cu, init.cu).  Not part of the C ABI.
#pragma once
#include "common.cuh"

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

using rk::EdgeDev;
using rk::EdgeOut;
using rk::EdgeXf;
using rk::FrameDev;
using rk::GridParams;
using rk::LMState;

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct rkhsba_ctx {
    int K = 0, E = 0;
    long long N = 0;
    rkhsba_params p{};
    GridParams gp{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 1;
    std::string err;
    std::vector<DevBuf> bufs;
    size_t bytes = 0;

    std::vector<long long> pt_off;        // K+1
    std::vector<FrameDev> frames_h;
    std::vector<EdgeDev> edges_h;
    std::vector<std::pair<int, int>> edge_in;   // as given by the caller (a, b)

    // device
    long long* d_pt_off = nullptr;
    FrameDev* d_frames = nullptr;
    EdgeDev* d_edges = nullptr;
    double* d_xyz = nullptr;
    float* d_sem_in = nullptr;
    float* d_rgb_in = nullptr;
    int* d_cmin = nullptr;
    int* d_cmax = nullptr;
    unsigned* d_semnorm = nullptr;
    int* d_err = nullptr;

    long long C_total = 0;
    uint32_t* d_keys = nullptr;
    uint32_t* d_keys_alt = nullptr;
    int* d_vals = nullptr;
    int* d_vals_alt = nullptr;
    long long* d_hist = nullptr;
    int* d_cell_start = nullptr;
    float4* d_pts4 = nullptr;
    void* d_sem = nullptr;
    float4* d_col4 = nullptr;
    int* d_perm_local = nullptr;
    long long* d_run = nullptr;       // cell run starts of the sorted points
    const uint32_t* d_pt_cell = nullptr;  // grid cell key of every sorted point
    long long* d_total = nullptr;      // scratch totals [4]
    long long* d_scan_ws = nullptr;

    long long total_bins = 0, Q_total = 0;
    int qbits = 0;                     // radix bits of the query keys
    EdgeXf* d_xf = nullptr;
    uint32_t* d_qkey = nullptr;        // home-cell key per query (then sorted)
    uint32_t* d_qkey_alt = nullptr;
    int* d_qval = nullptr;             // query index (then sorted)
    int* d_qval_alt = nullptr;
    long long* d_qhist = nullptr;
    float4* d_qrec = nullptr;          // per query: offset from home centre, point index
    float4* d_slots = nullptr;         // the same in sorted order
    int* d_bin_first = nullptr;        // first sorted query of each home cell
    int* d_unit_start = nullptr;       // units of <= tune_uq queries of one home cell
    int* d_ucount = nullptr;           // [2]: number of units, unit counter
    const uint32_t* q_sorted_key = nullptr;
    long long* d_acc = nullptr;
    EdgeOut* d_eout = nullptr;
    int* d_inc_off = nullptr;
    int* d_inc_list = nullptr;

    double* d_H_cand = nullptr;
    double* d_H_cur = nullptr;
    double* d_b_cand = nullptr;
    double* d_b_cur = nullptr;
    double* d_F_cand = nullptr;
    long long* d_n_cand = nullptr;
    double* d_poses_cur = nullptr;
    double* d_poses_cand = nullptr;
    LMState* d_state = nullptr;
    double* d_lm_ws = nullptr;
    bool need_initial = true;
    cudaGraphExec_t iter_graph = nullptr;   // one LM iteration, replayed
    bool use_graph = true;
    long long iter_launches = 0;            // kernels in one iteration
    cudaGraphExec_t pre_graph = nullptr;    // LM solve + binning of one iteration (batched serving)
    cudaGraphExec_t post_graph = nullptr;   // assembly + accept of one iteration (batched serving)
    long long pre_launches = 0, post_launches = 0;

    // pair-kernel tuning (rkhsba_set_tuning / the autotuner)
    int tune_uq = 32;                       // queries per unit
    int tune_ctas = 0;                      // CTAs per SM of the pair launch (0: as many as fit)

    // drop captured graphs (their kernels' arguments changed)
    void drop_graphs() {
        if (iter_graph) cudaGraphExecDestroy(iter_graph);
        if (pre_graph) cudaGraphExecDestroy(pre_graph);
        if (post_graph) cudaGraphExecDestroy(post_graph);
        iter_graph = pre_graph = post_graph = nullptr;
    }

    rk::PairArgs pair_args() const {
        rk::PairArgs a{};
        a.qkey = q_sorted_key;
        a.slots = d_slots;
        a.Q = Q_total;
        a.edges = d_edges;
        a.frames = d_frames;
        a.cell_start = d_cell_start;
        a.pts4 = d_pts4;
        a.sem_sorted = d_sem;
        a.col4 = d_col4;
        a.acc = d_acc;
        a.E = E;
        a.uq = tune_uq;
        a.gp = gp;
        return a;
    }

    // phase profiler (CUDA events on the context stream)
    static constexpr int NPH = 5;
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<int, int>>> ev_rec;   // phase, (start, end) pool index
    int cur_phase = -1, cur_start = -1;
    int ev_take() {
        if (ev_rec.size() * 2 + 2 > ev_pool.size()) {
            for (int i = 0; i < 64; ++i) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) return -1;
                ev_pool.push_back(e);
            }
        }
        return -2;
    }
    void phase_begin(int ph) {
        if (!prof) return;
        if (ev_take() == -1) return;
        int idx = (int)(ev_rec.size() * 2);
        cudaEventRecord(ev_pool[idx], stream);
        cur_phase = ph;
        cur_start = idx;
    }
    void phase_end() {
        if (!prof || cur_phase < 0) return;
        cudaEventRecord(ev_pool[cur_start + 1], stream);
        ev_rec.push_back({cur_phase, {cur_start, cur_start + 1}});
        cur_phase = -1;
    }

    rkhsba_ctx* self_ctx = nullptr;         // self-edge context (inner products)

    ~rkhsba_ctx() {
        delete self_ctx;                    // runs on this context's stream
        // stream-ordered frees: no device-wide synchronisation, so contexts
        // ending while others run (the request server) do not stall them
        for (auto& b : bufs) cudaFreeAsync(b.p, stream);
        if (stream) cudaStreamSynchronize(stream);
        for (auto e : ev_pool) cudaEventDestroy(e);
        if (iter_graph) cudaGraphExecDestroy(iter_graph);
        if (pre_graph) cudaGraphExecDestroy(pre_graph);
        if (post_graph) cudaGraphExecDestroy(post_graph);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace rk {
// records msg as the context's (and this thread's) last error; returns s
rkhsba_status ctx_fail(rkhsba_ctx* ctx, rkhsba_status s, const std::string& msg);
// one evaluation at device poses (16 K doubles); per-edge results land in d_eout
void ctx_run_eval(rkhsba_ctx* c, const double* d_poses);
// a context on `stream` from host or device inputs; allow_self admits edges
// (m, m), whose inner products are the self terms <f_m, f_m>
rkhsba_status ctx_create(rkhsba_ctx** out, int32_t n_frames, const int64_t* n_points, const double* xyz,
                         const float* sem, const float* rgb, int32_t n_edges, const int32_t* edges,
                         const rkhsba_params* params, void* stream, bool on_device, bool allow_self);
rkhsba_status ctx_check_poses(rkhsba_ctx* c, const double* poses);
}  // namespace rk

#define RK_CUDA(ctx, call)                                                                          \
    do {                                                                                            \
        cudaError_t _e = (call);                                                                    \
        if (_e != cudaSuccess)                                                                      \
            return rk::ctx_fail(ctx, RKHSBA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)

#define RK_TRY(expr)                        \
    do {                                    \
        rkhsba_status _s = (expr);          \
        if (_s != RKHSBA_OK) return _s;     \
    } while (0)
