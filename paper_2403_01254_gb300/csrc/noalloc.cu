// rkhsba_eval_static: one evaluation with no device allocation.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// runtime which owns every device byte through its own pool, and plug-ins or
// real-time loops that must not take the allocator's locks or risk an
// allocation failure mid-run.  For them this entry point evaluates a small
// problem with the same kernels as rkhsba_eval, but every temporary buffer is
// carved out of one file-scope device array, g_scratch, of fixed size.  The
// caller passes device pointers to the points and labels and host buffers
// for the results.  The host-side layout (grids, edge offsets, fixed-point
// scales, incidence lists) comes from the same helpers as the context path
// (layout.cuh).
//
// g_scratch is held by every GPU that loads the library, for as long as the
// library stays loaded.  Its device address is obtained once per device with
// cudaGetSymbolAddress (in host code the symbol names a host-side stand-in,
// not device memory); that happens in the first call on each device, so the
// first call on a device must not be made while a stream is being captured.
// The call waits on its stream (bounding boxes, results), so it refuses a
// stream under capture.  Every call uses the same array: two calls whose work
// overlaps on the GPU (different streams, or different host threads)
// overwrite each other's temporaries, so calls must be serialised by the
// caller.
#include "common.cuh"
#include "layout.cuh"
#include "rkhsba.h"

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

namespace {
using namespace rk;

constexpr size_t SCRATCH_BYTES = size_t(32) << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_K = 16;
constexpr int MAX_E = 64;
constexpr long long MAX_N = 32768;
constexpr long long MAX_Q = 131072;
constexpr long long MAX_CELLS = 1LL << 20;
constexpr long long MAX_BINS = 1LL << 20;
constexpr int MAX_DEVICES = 64;

void* g_scratch_dev[MAX_DEVICES] = {};
std::mutex g_scratch_mu;

rkhsba_status fail(rkhsba_status s, const std::string& msg) {
    set_thread_error(msg.c_str());
    return s;
}

// device address of g_scratch on the current device, looked up once
rkhsba_status scratch_base(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(RKHSBA_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(RKHSBA_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fail(RKHSBA_ECUDA, std::string("cudaGetSymbolAddress(g_scratch): ") + cudaGetErrorString(e));
        g_scratch_dev[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_dev[dev]);
    return RKHSBA_OK;
}

// bump allocator over the static array (256-byte aligned pieces)
struct Carve {
    unsigned char* base;
    size_t off = 0;
    bool ok = true;
    template <typename T>
    T* take(long long count) {
        size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
        bytes = (bytes + 255) & ~size_t(255);
        if (off + bytes > SCRATCH_BYTES) {
            ok = false;
            return nullptr;
        }
        T* p = reinterpret_cast<T*>(base + off);
        off += bytes;
        return p;
    }
};

#define SCK(call)                                                                              \
    do {                                                                                       \
        cudaError_t _e = (call);                                                               \
        if (_e != cudaSuccess) return fail(RKHSBA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)
}  // namespace

extern "C" rkhsba_status rkhsba_eval_static(int32_t n_frames, const int64_t* n_points, const double* d_xyz,
                                            const float* d_sem, const float* d_rgb, int32_t n_edges,
                                            const int32_t* edges, const rkhsba_params* params,
                                            const double* poses, double* loss, double* grad,
                                            double* H_full, void* cuda_stream) {
    // ---- arguments (host side, fixed-size arrays only) ----
    if (!params || !n_points || !edges || !poses) return fail(RKHSBA_EINVAL, "NULL argument");
    if (n_frames < 1 || n_frames > MAX_K) return fail(RKHSBA_EINVAL, "rkhsba_eval_static: 1 <= n_frames <= 16");
    if (n_edges < 1 || n_edges > MAX_E) return fail(RKHSBA_EINVAL, "rkhsba_eval_static: 1 <= n_edges <= 64");
    rkhsba_params p = *params;
    if (!(p.ell > 0.0) || !std::isfinite(p.ell)) return fail(RKHSBA_EINVAL, "params.ell must be > 0");
    if (p.cutoff_mult == 0.0) p.cutoff_mult = 3.0;
    if (p.sigma == 0.0) p.sigma = 1.0;
    if (!(p.cutoff_mult > 0.0) || !std::isfinite(p.cutoff_mult) || !std::isfinite(p.sigma))
        return fail(RKHSBA_EINVAL, "bad cutoff_mult or sigma");
    if (p.sem_dim < 0 || p.sem_dim > MAX_SEM || (p.sem_dim > 0) != (d_sem != nullptr))
        return fail(RKHSBA_EINVAL, "sem must be given exactly when 0 < sem_dim <= 32");
    const int K = n_frames, E = n_edges;
    long long pt_off[MAX_K + 1];
    pt_off[0] = 0;
    for (int m = 0; m < K; ++m) {
        if (n_points[m] < 0) return fail(RKHSBA_EINVAL, "negative point count");
        pt_off[m + 1] = pt_off[m] + n_points[m];
    }
    const long long N = pt_off[K];
    if (N > MAX_N) return fail(RKHSBA_EINVAL, "rkhsba_eval_static: more than 32768 points (static scratch limit)");
    if (N > 0 && !d_xyz) return fail(RKHSBA_EINVAL, "xyz is NULL");
    EdgeDev eh[MAX_E];
    std::memset(eh, 0, sizeof(eh));
    for (int e = 0; e < E; ++e) {
        int a = edges[2 * e], b = edges[2 * e + 1];
        if (a < 0 || b < 0 || a >= K || b >= K || a == b) return fail(RKHSBA_EINVAL, "bad edge");
        if (a > b) { int t = a; a = b; b = t; }
        for (int f = 0; f < e; ++f)
            if (eh[f].a == a && eh[f].b == b) return fail(RKHSBA_EINVAL, "duplicate edge");
        eh[e].a = a;
        eh[e].b = b;
    }
    for (int m = 0; m < K; ++m)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += poses[16 * m + 4 * k + i] * poses[16 * m + 4 * k + j];
                if (!(std::fabs(s - (i == j ? 1.0 : 0.0)) <= 1e-9)) return fail(RKHSBA_EINVAL, "non-orthonormal pose");
            }

    if (p.top_k < 0 || p.top_k > TOPK_MAX) return fail(RKHSBA_EINVAL, "params.top_k must be in [0, 8]");
    if (!(p.sem_min >= 0.0) || !std::isfinite(p.sem_min))
        return fail(RKHSBA_EINVAL, "params.sem_min must be finite and >= 0");
    if (p.cell_scale == 0.0) p.cell_scale = 1.0;
    if (!(p.cell_scale >= 1.0 && p.cell_scale <= 4.0)) return fail(RKHSBA_EINVAL, "params.cell_scale must be in [1, 4]");
    const double rc = p.cutoff_mult * p.ell;
    GridParams gp = grid_params_for(p);
    grid_params_color(gp, d_rgb != nullptr && p.ell_color > 0.0, p.ell_color);
    if (p.sem_dim > 0 && gp.sem_pad == 0) return fail(RKHSBA_EINVAL, "unsupported sem_dim");

    // the call waits on its stream for the bounding boxes and the results;
    // on a stream under capture those waits would fail and end the caller's
    // capture, so such a stream is refused before anything is issued on it
    cudaStream_t st = (cudaStream_t)cuda_stream;
    {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        SCK(cudaStreamIsCapturing(st, &cap));
        if (cap != cudaStreamCaptureStatusNone)
            return fail(RKHSBA_EINVAL, "rkhsba_eval_static waits on its stream and cannot run on a stream under capture");
    }

    unsigned char* base = nullptr;
    rkhsba_status st0 = scratch_base(&base);
    if (st0 != RKHSBA_OK) return st0;
    int dev = 0, num_sms = 1;
    SCK(cudaGetDevice(&dev));
    SCK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));

    // ---- small arrays and the bounding boxes ----
    Carve cv{base};
    long long* d_pt_off = cv.take<long long>(K + 1);
    int* d_cmin = cv.take<int>(3 * K);
    int* d_cmax = cv.take<int>(3 * K);
    unsigned* d_semn = cv.take<unsigned>(K);
    int* d_err = cv.take<int>(4);
    FrameDev* d_frames = cv.take<FrameDev>(K);
    EdgeDev* d_edges = cv.take<EdgeDev>(E);
    EdgeXf* d_xf = cv.take<EdgeXf>(E);
    int* d_inc_off = cv.take<int>(K + 1);
    int* d_inc_list = cv.take<int>(2 * E);
    double* d_poses = cv.take<double>(16 * K);
    long long* d_total = cv.take<long long>(4);
    if (!cv.ok) return fail(RKHSBA_EINVAL, "static scratch too small");
    int cmin[3 * MAX_K], cmax[3 * MAX_K], errbits = 0;
    unsigned semn[MAX_K];
    for (int i = 0; i < 3 * K; ++i) { cmin[i] = 0x7fffffff; cmax[i] = (int)0x80000000; }
    SCK(cudaMemcpyAsync(d_pt_off, pt_off, sizeof(long long) * (K + 1), cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(d_cmin, cmin, sizeof(int) * 3 * K, cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(d_cmax, cmax, sizeof(int) * 3 * K, cudaMemcpyHostToDevice, st));
    SCK(cudaMemsetAsync(d_semn, 0, sizeof(unsigned) * K, st));
    SCK(cudaMemsetAsync(d_err, 0, sizeof(int) * 4, st));
    launch_bbox(d_xyz, d_sem, gp.color ? d_rgb : nullptr, N, K, d_pt_off, p.sem_dim, gp.h_inv, d_cmin, d_cmax,
                d_semn, d_err, st);
    SCK(cudaMemcpyAsync(cmin, d_cmin, sizeof(int) * 3 * K, cudaMemcpyDeviceToHost, st));
    SCK(cudaMemcpyAsync(cmax, d_cmax, sizeof(int) * 3 * K, cudaMemcpyDeviceToHost, st));
    SCK(cudaMemcpyAsync(semn, d_semn, sizeof(unsigned) * K, cudaMemcpyDeviceToHost, st));
    SCK(cudaMemcpyAsync(&errbits, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    if (errbits) return fail(RKHSBA_EINVAL, "non-finite or out-of-range input values");

    // ---- grid layout, edges, fixed-point scales (host) ----
    FrameDev fh[MAX_K];
    long long C = 0;
    if (const char* msg = layout_frames(fh, K, pt_off, cmin, cmax, semn, p.sem_dim > 0, MAX_CELLS, MAX_CELLS,
                                        MAX_CELLS + 1, &C))
        return fail(RKHSBA_EINVAL, std::string("rkhsba_eval_static: ") + msg + " (2^20 grid cells at most)");
    long long bins = 0, Q = 0;
    layout_edges(eh, E, fh, gp, rc, &bins, &Q);
    if (bins > MAX_BINS) return fail(RKHSBA_EINVAL, "rkhsba_eval_static: more than 2^20 home cells over all edges");
    if (Q > MAX_Q) return fail(RKHSBA_EINVAL, "rkhsba_eval_static: more than 131072 queries over all edges");
    int qbits = 1;
    while ((1LL << qbits) <= bins) ++qbits;
    gp.key_sub = (qbits + 3 <= 31) ? 3 : 0;
    qbits += gp.key_sub;
    int cbits = 0;
    while ((1LL << cbits) < C) ++cbits;
    int inc_off[MAX_K + 1], inc_list[2 * MAX_E];
    const int ninc = incidence_lists(eh, E, K, inc_off, inc_list);

    // ---- large arrays ----
    const int sp = gp.sem_pad;
    const long long hist_n = (long long)(radix_hist_elems(N) > radix_hist_elems(Q) ? radix_hist_elems(N)
                                                                                   : radix_hist_elems(Q));
    uint32_t* d_keys = cv.take<uint32_t>(N);
    uint32_t* d_keys_alt = cv.take<uint32_t>(N);
    int* d_vals = cv.take<int>(N);
    int* d_vals_alt = cv.take<int>(N);
    long long* d_hist = cv.take<long long>(hist_n);
    long long* d_ws = cv.take<long long>((long long)scan_ws_elems(hist_n) + 64);
    int* d_cell_start = cv.take<int>(C + 1);
    float4* d_pts4 = cv.take<float4>(N);
    void* d_sem_sorted = sp > 0 ? (void*)cv.take<unsigned char>(N * sp * (gp.sem_bf16 ? 2 : 4)) : nullptr;
    float4* d_col4 = gp.color ? cv.take<float4>(N) : nullptr;
    int* d_perm_local = cv.take<int>(N);
    long long* d_run = cv.take<long long>(N);
    uint32_t* d_qkey = cv.take<uint32_t>(Q);
    uint32_t* d_qkey_alt = cv.take<uint32_t>(Q);
    int* d_qval = cv.take<int>(Q);
    int* d_qval_alt = cv.take<int>(Q);
    float4* d_qrec = cv.take<float4>(Q);
    float4* d_slots = cv.take<float4>(Q);
    int* d_bin_first = cv.take<int>(bins);
    int* d_units = cv.take<int>(Q);
    int* d_ucount = cv.take<int>(4);
    long long* d_acc = cv.take<long long>((long long)E * ACC_N);
    EdgeOut* d_eout = cv.take<EdgeOut>(E);
    double* d_H = cv.take<double>(36LL * K * K);
    double* d_b = cv.take<double>(6 * K);
    double* d_F = cv.take<double>(1);
    long long* d_n = cv.take<long long>(1);
    if (!cv.ok) return fail(RKHSBA_EINVAL, "rkhsba_eval_static: problem does not fit the 32 MiB static scratch");

    SCK(cudaMemcpyAsync(d_frames, fh, sizeof(FrameDev) * K, cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(d_edges, eh, sizeof(EdgeDev) * E, cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(d_inc_off, inc_off, sizeof(int) * (K + 1), cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(d_inc_list, inc_list, sizeof(int) * (ninc > 0 ? ninc : 1), cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(d_poses, poses, sizeof(double) * 16 * K, cudaMemcpyHostToDevice, st));

    // ---- grid step (all temporaries that must start at zero are cleared) ----
    SCK(cudaMemsetAsync(d_cell_start, 0, sizeof(int) * (C + 1), st));
    launch_keys(d_xyz, N, K, d_pt_off, d_frames, gp.h_inv, d_keys, d_vals, st);
    bool alt = false;
    radix_sort_u32(d_keys, d_vals, d_keys_alt, d_vals_alt, N, cbits, d_hist, d_ws, d_err + 1, st, &alt);
    const uint32_t* pt_cell = alt ? d_keys_alt : d_keys;
    launch_gather(d_xyz, d_sem, gp.color ? d_rgb : nullptr, N, K, d_pt_off, pt_cell, alt ? d_vals_alt : d_vals,
                  gp, C, d_pts4, d_sem_sorted, d_col4, d_perm_local, d_cell_start, d_run, st);

    // ---- evaluation ----
    launch_edge_setup(d_poses, d_edges, E, d_frames, gp.h, d_xf, nullptr, st);
    SCK(cudaMemsetAsync(d_ucount, 0, sizeof(int) * 4, st));
    SCK(cudaMemsetAsync(d_acc, 0, sizeof(long long) * E * ACC_N, st));
    launch_query_keys(d_edges, E, d_frames, d_xf, pt_cell, d_pts4, gp, Q, d_qkey, d_qval, d_qrec, nullptr, st);
    bool qalt = false;
    radix_sort_u32(d_qkey, d_qval, d_qkey_alt, d_qval_alt, Q, qbits, d_hist, d_ws, d_err + 1, st, &qalt);
    const uint32_t* qk = qalt ? d_qkey_alt : d_qkey;
    launch_query_gather(qk, qalt ? d_qval_alt : d_qval, d_qrec, Q, gp.key_sub, d_slots, d_bin_first, nullptr, st);
    launch_units(qk, d_bin_first, Q, UNIT_Q, gp.key_sub, d_units, d_ucount, nullptr, st);
    {
        PairArgs a{};
        a.qkey = qk;
        a.slots = d_slots;
        a.Q = Q;
        a.edges = d_edges;
        a.frames = d_frames;
        a.cell_start = d_cell_start;
        a.pts4 = d_pts4;
        a.sem_sorted = d_sem_sorted;
        a.col4 = d_col4;
        a.acc = d_acc;
        a.E = E;
        a.uq = UNIT_Q;
        a.gp = gp;
        launch_pairs(PairLaunch{d_units, d_ucount, d_ucount + 1, nullptr, num_sms, 0, st}, a);
    }
    launch_edge_assemble(d_edges, E, d_xf, d_acc, p.sigma * p.sigma, d_eout, nullptr, st);
    SCK(cudaMemsetAsync(d_H, 0, sizeof(double) * 36LL * K * K, st));
    launch_frame_assemble(d_edges, E, K, d_inc_off, d_inc_list, d_eout, d_H, d_b, d_F, d_n, nullptr, st);

    // ---- results to the caller's host buffers ----
    double F = 0.0;
    double bvec[6 * MAX_K];
    int sort_err = 0;
    SCK(cudaMemcpyAsync(&sort_err, d_err + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCK(cudaMemcpyAsync(&F, d_F, sizeof(double), cudaMemcpyDeviceToHost, st));
    SCK(cudaMemcpyAsync(bvec, d_b, sizeof(double) * 6 * K, cudaMemcpyDeviceToHost, st));
    if (H_full) SCK(cudaMemcpyAsync(H_full, d_H, sizeof(double) * 36LL * K * K, cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    SCK(cudaGetLastError());
    if (sort_err) return fail(RKHSBA_ETIMEOUT, "a bounded wait of the radix sort gave up");
    if (loss) *loss = -F;
    if (grad) {
        const double scale = p.sigma * p.sigma / (p.ell * p.ell);
        for (int i = 0; i < 6 * K; ++i) grad[i] = scale * bvec[i];
    }
    return RKHSBA_OK;
}
