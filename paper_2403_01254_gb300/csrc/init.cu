// Function-space distance, cosine and their use around the pose solve:
//   * rkhsba_inner_products   self terms <f_m, f_m>, per-edge <f_a, f_b>,
//                             |f_a - f_b|^2, cosine, d(sum dist)/d ell
//                             (Sec. III-A, Eq. dist_rkhs)
//   * rkhsba_rotation_search  60 icosahedral rotations of one frame against
//                             another, ranked by the cosine (Sec. IV-A)
//   * rkhsba_solve_ell_decay  outer loop over ell around the LM solve
//                             (Sec. V-C)
// Every inner product is the objective's own evaluation (grid, binning, pair
// kernel, assembly) over a suitable edge list: self terms are edges (m, m) at
// identity poses; the 60 rotation candidates are 60 edges of one batched
// evaluation against 60 copies of the moving frame.
#include "context.cuh"
#include "rkhsba.h"

#include <array>
#include <cmath>
#include <memory>
#include <mutex>

using namespace rk;

namespace {

constexpr int N_ROT = 60;

// ------------------------------------------------------------- kernels -----

// Block-wide sum of per-thread FP64 values in a fixed order (deterministic).
__device__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Candidate poses of the rotation search: pose 0 = T_a, pose 1 + k =
// T_a [R_k | mu_a - R_k mu_b], mu the frame-local centroids.  One block.
__global__ void k_rot_candidates(const double* __restrict__ xyz, long long off_a, long long n_a,
                                 long long off_b, long long n_b, const double* __restrict__ Ta,
                                 const double* __restrict__ R, double* __restrict__ poses) {
    __shared__ double sh[256];
    __shared__ double mu[6];
    for (int f = 0; f < 2; ++f) {
        const long long off = f ? off_b : off_a;
        const long long n = f ? n_b : n_a;
        double s[3] = {0.0, 0.0, 0.0};
        for (long long i = threadIdx.x; i < n; i += blockDim.x)
            for (int k = 0; k < 3; ++k) s[k] += xyz[3 * (off + i) + k];
        for (int k = 0; k < 3; ++k) {
            const double t = block_sum(s[k], sh);
            if (threadIdx.x == 0) mu[3 * f + k] = t / (double)n;
        }
    }
    __syncthreads();
    const int k = threadIdx.x;
    if (k < 16) poses[k] = Ta[k];
    if (k >= N_ROT) return;
    const double* Rk = R + 9 * k;
    double C[12];
    for (int i = 0; i < 3; ++i) {
        double rm = 0.0;
        for (int j = 0; j < 3; ++j) {
            C[4 * i + j] = Rk[3 * i + j];
            rm += Rk[3 * i + j] * mu[3 + j];
        }
        C[4 * i + 3] = mu[i] - rm;
    }
    double* P = poses + 16 * (1 + k);
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 4; ++j) {
            double v = (j == 3) ? Ta[4 * i + 3] : 0.0;
            for (int l = 0; l < 3; ++l) v += Ta[4 * i + l] * C[4 * l + j];
            P[4 * i + j] = v;
        }
    }
    P[12] = 0.0;
    P[13] = 0.0;
    P[14] = 0.0;
    P[15] = 1.0;
}

// cos_k = <f_a, f_{b,k}> / sqrt(<f_a,f_a> <f_b,f_b>); best = first maximum.
// out: [60] cosines, [16] best pose, [1] best index (as double).  One block.
__global__ void k_rot_select(const EdgeOut* __restrict__ cross, const EdgeOut* __restrict__ self_a,
                             const EdgeOut* __restrict__ self_b, const double* __restrict__ poses,
                             double* __restrict__ out) {
    __shared__ int s_best;
    const double den = self_a->F * self_b->F;
    const int k = threadIdx.x;
    if (k < N_ROT) out[k] = den > 0.0 ? cross[k].F / sqrt(den) : 0.0;
    __syncthreads();
    if (k == 0) {
        int best = 0;
        for (int j = 1; j < N_ROT; ++j)
            if (out[j] > out[best]) best = j;
        s_best = best;
        out[N_ROT + 16] = (double)best;
    }
    __syncthreads();
    if (k < 16) out[N_ROT + k] = poses[16 * (1 + s_best) + k];
}

// Per edge: cross term, distance and cosine; the self terms; and
// dD/dell = sigma^2/ell^3 sum_e (E_aa + E_bb - 2 E_ab).  One block; out holds
// [K] self, [E] cross, [E] dist, [E] cosine, [1] dD/dell.
__global__ void k_ip_metrics(const EdgeDev* __restrict__ edges, int E, int K,
                             const EdgeOut* __restrict__ cross, const EdgeOut* __restrict__ self,
                             double sigma2, double ell, double* __restrict__ out) {
    __shared__ double sh[256];
    double* o_self = out;
    double* o_cross = out + K;
    double* o_dist = o_cross + E;
    double* o_cos = o_dist + E;
    for (int m = threadIdx.x; m < K; m += blockDim.x) o_self[m] = self[m].F;
    double part = 0.0;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int a = edges[e].a, b = edges[e].b;
        const double Sa = self[a].F, Sb = self[b].F, X = cross[e].F;
        o_cross[e] = X;
        o_dist[e] = Sa + Sb - 2.0 * X;
        o_cos[e] = (Sa > 0.0 && Sb > 0.0) ? X / sqrt(Sa * Sb) : 0.0;
        part += self[a].E + self[b].E - 2.0 * cross[e].E;
    }
    const double tot = block_sum(part, sh);
    if (threadIdx.x == 0) o_cross[3 * E] = sigma2 / (ell * ell * ell) * tot;
}

// --------------------------------------------------- icosahedral group -----

using Mat3 = std::array<double, 9>;

Mat3 mul(const Mat3& A, const Mat3& B) {
    Mat3 C{};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
    return C;
}

// Rotation by `angle` about the unit axis u (Rodrigues).
Mat3 axis_angle(double ux, double uy, double uz, double angle) {
    const double n = std::sqrt(ux * ux + uy * uy + uz * uz);
    ux /= n;
    uy /= n;
    uz /= n;
    const double c = std::cos(angle), s = std::sin(angle), v = 1.0 - c;
    return Mat3{c + ux * ux * v,      ux * uy * v - uz * s, ux * uz * v + uy * s,
                uy * ux * v + uz * s, c + uy * uy * v,      uy * uz * v - ux * s,
                uz * ux * v - uy * s, uz * uy * v + ux * s, c + uz * uz * v};
}

// The rotation group of the icosahedron whose vertices are the cyclic
// permutations of (0, +-1, +-phi): generated by the 2pi/5 turn about the
// vertex (0, 1, phi) and the half turn about the z axis (through the
// midpoint of the edge (0, +-1, phi)), closed under products.  Ordered as
// the paper lists the classes: identity, the 15 half turns, the 20 turns by
// 2pi/3 or 4pi/3, the 24 turns by multiples of 2pi/5; lexicographic inside a
// class.
const std::vector<Mat3>& icosahedral_group() {
    static std::vector<Mat3> G;
    static std::once_flag once;
    std::call_once(once, [] {
        const double phi = (1.0 + std::sqrt(5.0)) / 2.0;
        const double pi = 3.14159265358979323846;
        const Mat3 g5 = axis_angle(0.0, 1.0, phi, 2.0 * pi / 5.0);
        const Mat3 g2 = axis_angle(0.0, 0.0, 1.0, pi);
        auto same = [](const Mat3& A, const Mat3& B) {
            for (int i = 0; i < 9; ++i)
                if (std::fabs(A[i] - B[i]) > 1e-9) return false;
            return true;
        };
        std::vector<Mat3> out{Mat3{1, 0, 0, 0, 1, 0, 0, 0, 1}};
        for (size_t i = 0; i < out.size() && out.size() < 200; ++i)
            for (const Mat3* g : {&g5, &g2}) {
                const Mat3 P = mul(out[i], *g);
                bool found = false;
                for (const Mat3& Q : out) found = found || same(P, Q);
                if (!found) out.push_back(P);
            }
        // class by trace = 1 + 2 cos(angle): 3 (identity), -1 (pi), 0 (2pi/3),
        // 1 +- 2 cos(2pi/5) ... (fifth turns)
        auto cls = [](const Mat3& A) {
            const double t = A[0] + A[4] + A[8];
            if (t > 2.5) return 0;
            if (std::fabs(t + 1.0) < 1e-6) return 1;
            if (std::fabs(t) < 1e-6) return 2;
            return 3;
        };
        std::sort(out.begin(), out.end(), [&](const Mat3& A, const Mat3& B) {
            const int ca = cls(A), cb = cls(B);
            if (ca != cb) return ca < cb;
            for (int i = 0; i < 9; ++i)
                if (std::fabs(A[i] - B[i]) > 1e-9) return A[i] < B[i];
            return false;
        });
        G = out;
    });
    return G;
}

// ------------------------------------------------------------- helpers -----

struct TmpBuf {                       // stream-ordered scratch
    void* p = nullptr;
    cudaStream_t st = nullptr;
    ~TmpBuf() {
        if (p) cudaFreeAsync(p, st);
    }
};

template <typename T>
rkhsba_status tmp_alloc(rkhsba_ctx* c, TmpBuf& b, T** out, long long count) {
    b.st = c->stream;
    cudaError_t e = cudaMallocAsync(&b.p, (size_t)std::max<long long>(count, 1) * sizeof(T), c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return ctx_fail(c, RKHSBA_ENOMEM, std::string("scratch allocation failed: ") + cudaGetErrorString(e));
    }
    *out = static_cast<T*>(b.p);
    return RKHSBA_OK;
}

std::vector<int64_t> frame_sizes(const rkhsba_ctx* c) {
    std::vector<int64_t> n(c->K);
    for (int m = 0; m < c->K; ++m) n[m] = c->pt_off[m + 1] - c->pt_off[m];
    return n;
}

// Self terms <f_m, f_m>: a context over the same device inputs with the
// edges (m, m), evaluated once at identity poses; its per-edge outputs stay
// in its d_eout.
rkhsba_status ensure_self(rkhsba_ctx* c) {
    if (c->self_ctx) return RKHSBA_OK;
    std::vector<int32_t> edges(2 * c->K);
    for (int m = 0; m < c->K; ++m) edges[2 * m] = edges[2 * m + 1] = m;
    const std::vector<int64_t> n = frame_sizes(c);
    rkhsba_ctx* s = nullptr;
    rkhsba_status r = ctx_create(&s, c->K, n.data(), c->d_xyz, c->d_sem_in, c->d_rgb_in, c->K, edges.data(),
                                 &c->p, c->stream, true, true);
    if (r != RKHSBA_OK) return ctx_fail(c, r, std::string("self-term context: ") + rkhsba_last_error(nullptr));
    std::vector<double> eye(16 * (size_t)c->K, 0.0);
    for (int m = 0; m < c->K; ++m)
        for (int i = 0; i < 4; ++i) eye[16 * m + 5 * i] = 1.0;
    cudaError_t e = cudaMemcpyAsync(s->d_poses_cand, eye.data(), sizeof(double) * eye.size(),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        ctx_run_eval(s, s->d_poses_cand);
        e = cudaStreamSynchronize(c->stream);   // eye is read before it goes out of scope
    }
    if (e != cudaSuccess) {
        delete s;
        return ctx_fail(c, RKHSBA_ECUDA, std::string("self terms: ") + cudaGetErrorString(e));
    }
    c->self_ctx = s;
    return RKHSBA_OK;
}

}  // namespace

extern "C" {

rkhsba_status rkhsba_inner_products(rkhsba_ctx* c, const double* poses, double* self_ip, double* cross_ip,
                                    double* dist, double* cosine, double* dD_dell) {
    if (!c) return ctx_fail(nullptr, RKHSBA_EINVAL, "ctx is NULL");
    RK_TRY(ctx_check_poses(c, poses));
    RK_TRY(ensure_self(c));
    cudaStream_t st = c->stream;
    RK_CUDA(c, cudaMemcpyAsync(c->d_poses_cand, poses, sizeof(double) * 16 * c->K, cudaMemcpyHostToDevice, st));
    ctx_run_eval(c, c->d_poses_cand);
    const int K = c->K, E = c->E;
    TmpBuf tb;
    double* d_out = nullptr;
    RK_TRY(tmp_alloc(c, tb, &d_out, (long long)K + 3LL * E + 1));
    k_ip_metrics<<<1, 256, 0, st>>>(c->d_edges, E, K, c->d_eout, c->self_ctx->d_eout, c->p.sigma * c->p.sigma,
                                    c->p.ell, d_out);
    count_launch();
    std::vector<double> h((size_t)K + 3 * (size_t)E + 1);
    RK_CUDA(c, cudaMemcpyAsync(h.data(), d_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
    RK_CUDA(c, cudaStreamSynchronize(st));
    RK_CUDA(c, cudaGetLastError());
    if (self_ip) std::copy(h.begin(), h.begin() + K, self_ip);
    if (cross_ip) std::copy(h.begin() + K, h.begin() + K + E, cross_ip);
    if (dist) std::copy(h.begin() + K + E, h.begin() + K + 2 * E, dist);
    if (cosine) std::copy(h.begin() + K + 2 * E, h.begin() + K + 3 * E, cosine);
    if (dD_dell) *dD_dell = h[K + 3 * E];
    return RKHSBA_OK;
}

rkhsba_status rkhsba_rotation_search(rkhsba_ctx* c, int32_t a, int32_t b, const double* poses, double* cosine,
                                     double* rotations, double* best_pose, int32_t* best) {
    if (!c) return ctx_fail(nullptr, RKHSBA_EINVAL, "ctx is NULL");
    if (a < 0 || b < 0 || a >= c->K || b >= c->K || a == b)
        return ctx_fail(c, RKHSBA_EINVAL, "rotation search needs two different frames of the context");
    RK_TRY(ctx_check_poses(c, poses));
    const long long na = c->pt_off[a + 1] - c->pt_off[a], nb = c->pt_off[b + 1] - c->pt_off[b];
    if (na == 0 || nb == 0) return ctx_fail(c, RKHSBA_EINVAL, "rotation search on an empty frame");
    const long long n_child = na + (long long)N_ROT * nb;
    if (n_child >= (1LL << 31) - 64)
        return ctx_fail(c, RKHSBA_EINVAL, "rotation search: 1 + 60 copies exceed 2^31 points");
    RK_TRY(ensure_self(c));
    cudaStream_t st = c->stream;

    // inputs of the batch: frame a, then 60 copies of frame b
    const int sd = c->p.sem_dim;
    TmpBuf bx, bs, bc, bp;
    double* d_xyz = nullptr;
    float* d_sem = nullptr;
    float* d_rgb = nullptr;
    RK_TRY(tmp_alloc(c, bx, &d_xyz, 3 * n_child));
    if (c->d_sem_in) RK_TRY(tmp_alloc(c, bs, &d_sem, (long long)sd * n_child));
    if (c->d_rgb_in) RK_TRY(tmp_alloc(c, bc, &d_rgb, 3 * n_child));
    for (int f = 0; f <= N_ROT; ++f) {
        const int src = f == 0 ? a : b;
        const long long n = f == 0 ? na : nb;
        const long long dst = f == 0 ? 0 : na + (long long)(f - 1) * nb;
        const long long so = c->pt_off[src];
        RK_CUDA(c, cudaMemcpyAsync(d_xyz + 3 * dst, c->d_xyz + 3 * so, sizeof(double) * 3 * n,
                                   cudaMemcpyDeviceToDevice, st));
        if (d_sem)
            RK_CUDA(c, cudaMemcpyAsync(d_sem + (long long)sd * dst, c->d_sem_in + (long long)sd * so,
                                       sizeof(float) * sd * n, cudaMemcpyDeviceToDevice, st));
        if (d_rgb)
            RK_CUDA(c, cudaMemcpyAsync(d_rgb + 3 * dst, c->d_rgb_in + 3 * so, sizeof(float) * 3 * n,
                                       cudaMemcpyDeviceToDevice, st));
    }
    std::vector<int64_t> n_pts(1 + N_ROT, nb);
    n_pts[0] = na;
    std::vector<int32_t> edges(2 * N_ROT);
    for (int k = 0; k < N_ROT; ++k) {
        edges[2 * k] = 0;
        edges[2 * k + 1] = 1 + k;
    }
    rkhsba_ctx* child = nullptr;
    rkhsba_status r = ctx_create(&child, 1 + N_ROT, n_pts.data(), d_xyz, d_sem, d_rgb, N_ROT, edges.data(), &c->p,
                                 st, true, false);
    if (r != RKHSBA_OK) return ctx_fail(c, r, std::string("rotation batch: ") + rkhsba_last_error(nullptr));
    std::unique_ptr<rkhsba_ctx> hold(child);

    // rotation table and T_a
    const std::vector<Mat3>& G = icosahedral_group();
    if (G.size() != (size_t)N_ROT) return ctx_fail(c, RKHSBA_EINVAL, "icosahedral group construction failed");
    std::vector<double> hin(9 * N_ROT + 16);
    for (int k = 0; k < N_ROT; ++k) std::copy(G[k].begin(), G[k].end(), hin.begin() + 9 * k);
    std::copy(poses + 16 * a, poses + 16 * a + 16, hin.begin() + 9 * N_ROT);
    double* d_in = nullptr;
    RK_TRY(tmp_alloc(c, bp, &d_in, (long long)hin.size() + N_ROT + 17));
    double* d_out = d_in + hin.size();
    RK_CUDA(c, cudaMemcpyAsync(d_in, hin.data(), sizeof(double) * hin.size(), cudaMemcpyHostToDevice, st));
    k_rot_candidates<<<1, 256, 0, st>>>(c->d_xyz, c->pt_off[a], na, c->pt_off[b], nb, d_in + 9 * N_ROT, d_in,
                                        child->d_poses_cand);
    count_launch();
    ctx_run_eval(child, child->d_poses_cand);
    k_rot_select<<<1, 64, 0, st>>>(child->d_eout, c->self_ctx->d_eout + a, c->self_ctx->d_eout + b,
                                   child->d_poses_cand, d_out);
    count_launch();
    std::vector<double> h(N_ROT + 17);
    RK_CUDA(c, cudaMemcpyAsync(h.data(), d_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
    RK_CUDA(c, cudaStreamSynchronize(st));
    RK_CUDA(c, cudaGetLastError());
    if (cosine) std::copy(h.begin(), h.begin() + N_ROT, cosine);
    if (rotations) std::copy(hin.begin(), hin.begin() + 9 * N_ROT, rotations);
    if (best_pose) std::copy(h.begin() + N_ROT, h.begin() + N_ROT + 16, best_pose);
    if (best) *best = (int32_t)h[N_ROT + 16];
    return RKHSBA_OK;
}

rkhsba_status rkhsba_solve_ell_decay(rkhsba_ctx* c, const rkhsba_ell_schedule* sched, double* poses,
                                     double* ell_levels, double* dD_levels, rkhsba_ell_info* info) {
    if (!c) return ctx_fail(nullptr, RKHSBA_EINVAL, "ctx is NULL");
    if (!sched) return ctx_fail(c, RKHSBA_EINVAL, "schedule is NULL");
    if (!(sched->decay > 0.0 && sched->decay < 1.0))
        return ctx_fail(c, RKHSBA_EINVAL, "schedule.decay must be in (0, 1)");
    if (!(sched->ell_min >= 0.0) || !std::isfinite(sched->ell_min))
        return ctx_fail(c, RKHSBA_EINVAL, "schedule.ell_min must be finite and >= 0");
    if (sched->max_outer < 1) return ctx_fail(c, RKHSBA_EINVAL, "schedule.max_outer must be >= 1");
    if (sched->reserved != 0) return ctx_fail(c, RKHSBA_EINVAL, "schedule.reserved must be 0");
    RK_TRY(ctx_check_poses(c, poses));
    const std::vector<int64_t> n = frame_sizes(c);
    std::vector<int32_t> edges(2 * c->E);
    for (int e = 0; e < c->E; ++e) {
        edges[2 * e] = c->edges_h[e].a;
        edges[2 * e + 1] = c->edges_h[e].b;
    }
    rkhsba_ell_info out{};
    double ell = c->p.ell;
    for (int t = 0; t < sched->max_outer; ++t) {
        rkhsba_params q = c->p;
        q.ell = ell;
        rkhsba_ctx* L = nullptr;
        rkhsba_status r = ctx_create(&L, c->K, n.data(), c->d_xyz, c->d_sem_in, c->d_rgb_in, c->E, edges.data(),
                                     &q, c->stream, true, false);
        if (r != RKHSBA_OK) return ctx_fail(c, r, std::string("level context: ") + rkhsba_last_error(nullptr));
        std::unique_ptr<rkhsba_ctx> hold(L);
        rkhsba_solve_info si{};
        r = rkhsba_solve(L, poses, &si);
        if (r != RKHSBA_OK && r != RKHSBA_ENOTCONV) return ctx_fail(c, r, L->err);
        LMState s{};
        RK_CUDA(c, cudaMemcpyAsync(&s, L->d_state, sizeof(LMState), cudaMemcpyDeviceToHost, c->stream));
        double g = 0.0;
        r = rkhsba_inner_products(L, poses, nullptr, nullptr, nullptr, nullptr, &g);
        if (r != RKHSBA_OK) return ctx_fail(c, r, L->err);
        if (ell_levels) ell_levels[t] = ell;
        if (dD_levels) dD_levels[t] = g;
        out.levels = t + 1;
        out.status = si.status;
        out.ell_final = ell;
        out.final_loss = si.final_loss;
        out.iters += si.iters;
        out.pair_terms += si.pair_terms;
        if (s.n_accepted == 0) break;
        const double sgn = g > 0.0 ? 1.0 : (g < 0.0 ? -1.0 : 0.0);
        const double nxt = std::max(ell * (1.0 - sched->decay * sgn), sched->ell_min);
        if (!(nxt > 0.0)) break;
        if (nxt == ell) break;
        ell = nxt;
    }
    if (info) *info = out;
    return RKHSBA_OK;
}

}  // extern "C"
