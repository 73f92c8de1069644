// FP64 assembly of the Gauss-Newton system and the damped pose solve.
//
// Per edge the 28 fixed-point moments become, in FP64,
//   loss term  F_ab = sigma^2 sum w                      Eq. (inner_product_actual_ba)
//   b = sum w J^T d  (gradient of Eq. inner_product_reformat up to -sigma^2/ell^2)
//   H = sum w J^T J  (normal matrix of the IRLS cost, Eq. irls_final)
// with J_a = R_a [I | -[x]x], J_b = -R_b [I | -[y]x] (right perturbation,
// rho before phi as in the wedge operator of Sec. V-A).  The frame blocks are
// then summed into the 6K x 6K system, frame 0 is held fixed, and one
// Levenberg-Marquardt step (H_ff + lambda diag) delta = -b_f is solved by
// Cholesky; poses move by T <- T exp(delta^).  A step is kept when the
// original cost F increases (Sec. V-C); the weights are recomputed at the new
// poses by the next evaluation (Sec. V-A, last paragraph).
#include "common.cuh"

#include <algorithm>

namespace rk {

namespace {

__device__ __forceinline__ void skew(const double* v, double S[3][3]) {
    S[0][0] = 0.0;   S[0][1] = -v[2]; S[0][2] = v[1];
    S[1][0] = v[2];  S[1][1] = 0.0;   S[1][2] = -v[0];
    S[2][0] = -v[1]; S[2][1] = v[0];  S[2][2] = 0.0;
}

__global__ void k_edge_assemble(const EdgeDev* __restrict__ edges, int E, const EdgeXf* __restrict__ xf,
                                const long long* __restrict__ acc, double sigma2,
                                EdgeOut* __restrict__ out, const int* done) {
    if (done && *done) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    const long long* a = acc + (long long)e * ACC_N;
    const EdgeDev& Ed = edges[e];
    double m[28];
    for (int k = 0; k < 28; ++k) m[k] = (double)a[k] * Ed.inv_scale[moment_class(k)];
    const double W = m[0];
    const double D[3] = {m[1], m[2], m[3]};
    const double Sy[3] = {m[4], m[5], m[6]};
    const double Myy[3][3] = {{m[7], m[8], m[9]}, {m[8], m[10], m[11]}, {m[9], m[11], m[12]}};
    const double Mdy[3][3] = {{m[13], m[14], m[15]}, {m[16], m[17], m[18]}, {m[19], m[20], m[21]}};
    const double Q[3][3] = {{m[22], m[23], m[24]}, {m[23], m[25], m[26]}, {m[24], m[26], m[27]}};
    const EdgeXf& X = xf[e];
    const double* R = X.R;
    const double* t = X.t;

    double Sx[3], St[3], Gx[3], Gt[3];
    double Mxx[3][3], Mxt[3][3], Mtt[3][3];
    for (int i = 0; i < 3; ++i) {
        Sx[i] = Sy[i] + D[i];
        St[i] = Sy[i] - W * t[i];
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const double Mxy = Myy[i][j] + Mdy[i][j];                 // sum w x y'^T
            Mxx[i][j] = Myy[i][j] + Mdy[i][j] + Mdy[j][i] + Q[i][j];   // sum w x x^T
            Mxt[i][j] = Mxy - Sx[i] * t[j];                             // sum w x y~^T
            Mtt[i][j] = Myy[i][j] - Sy[i] * t[j] - t[i] * Sy[j] + W * t[i] * t[j];
        }
    // sum w x (x) d = sum w y' (x) d
    Gx[0] = Mdy[2][1] - Mdy[1][2];
    Gx[1] = Mdy[0][2] - Mdy[2][0];
    Gx[2] = Mdy[1][0] - Mdy[0][1];
    // sum w y~ (x) d, y~ = y' - t_ab
    Gt[0] = Gx[0] - (t[1] * D[2] - t[2] * D[1]);
    Gt[1] = Gx[1] - (t[2] * D[0] - t[0] * D[2]);
    Gt[2] = Gx[2] - (t[0] * D[1] - t[1] * D[0]);

    EdgeOut o;
    o.F = sigma2 * W;
    o.E = Q[0][0] + Q[1][1] + Q[2][2];
    o.n = a[28];
    o.pad = 0;
    // b_a = [D; Gx],  b_b = -[R^T D; R^T Gt]
    for (int i = 0; i < 3; ++i) {
        o.b[i] = D[i];
        o.b[3 + i] = Gx[i];
        o.b[6 + i] = -(R[i] * D[0] + R[3 + i] * D[1] + R[6 + i] * D[2]);
        o.b[9 + i] = -(R[i] * Gt[0] + R[3 + i] * Gt[1] + R[6 + i] * Gt[2]);
    }
    double* H = o.H;
    for (int k = 0; k < 144; ++k) H[k] = 0.0;
    double Kx[3][3], Kt[3][3], Kb[3][3];
    skew(Sx, Kx);
    skew(St, Kt);
    // frame-b quantities in b's own axes: Sb = R^T St, Mb = R^T Mtt R
    double Sb[3], Mb[3][3], T1[3][3];
    for (int i = 0; i < 3; ++i) Sb[i] = R[i] * St[0] + R[3 + i] * St[1] + R[6 + i] * St[2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T1[i][j] = Mtt[i][0] * R[j] + Mtt[i][1] * R[3 + j] + Mtt[i][2] * R[6 + j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Mb[i][j] = R[i] * T1[0][j] + R[3 + i] * T1[1][j] + R[6 + i] * T1[2][j];
    skew(Sb, Kb);
    const double trx = Mxx[0][0] + Mxx[1][1] + Mxx[2][2];
    const double trb = Mb[0][0] + Mb[1][1] + Mb[2][2];
    const double trxt = Mxt[0][0] + Mxt[1][1] + Mxt[2][2];
    // right factors of the a-b block: [S~]x R, [Sx]x R, (Mxt^T - tr I) R
    double KtR[3][3], KxR[3][3], NR[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s1 = 0.0, s2 = 0.0, s3 = 0.0;
            for (int k = 0; k < 3; ++k) {
                s1 += Kt[i][k] * R[3 * k + j];
                s2 += Kx[i][k] * R[3 * k + j];
                const double Nik = Mxt[k][i] - (i == k ? trxt : 0.0);
                s3 += Nik * R[3 * k + j];
            }
            KtR[i][j] = s1; KxR[i][j] = s2; NR[i][j] = s3;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const double id = (i == j) ? 1.0 : 0.0;
            // H_aa
            H[12 * i + j] = W * id;
            H[12 * i + 3 + j] = -Kx[i][j];
            H[12 * (3 + i) + j] = Kx[i][j];
            H[12 * (3 + i) + 3 + j] = trx * id - Mxx[i][j];
            // H_bb
            H[12 * (6 + i) + 6 + j] = W * id;
            H[12 * (6 + i) + 9 + j] = -Kb[i][j];
            H[12 * (9 + i) + 6 + j] = Kb[i][j];
            H[12 * (9 + i) + 9 + j] = trb * id - Mb[i][j];
            // H_ab and its transpose
            const double ab00 = -W * R[3 * i + j];
            const double ab01 = KtR[i][j];
            const double ab10 = -KxR[i][j];
            const double ab11 = NR[i][j];
            H[12 * i + 6 + j] = ab00;
            H[12 * i + 9 + j] = ab01;
            H[12 * (3 + i) + 6 + j] = ab10;
            H[12 * (3 + i) + 9 + j] = ab11;
            H[12 * (6 + j) + i] = ab00;
            H[12 * (9 + j) + i] = ab01;
            H[12 * (6 + j) + 3 + i] = ab10;
            H[12 * (9 + j) + 3 + i] = ab11;
        }
    out[e] = o;
}

// blocks [0, K): diagonal 6x6 block and gradient of frame m (sum over its
// edges in edge order); [K, K+E): the off-diagonal block of edge e;
// K+E: totals.  Every entry has one writer and a fixed summation order.
__global__ void k_frame_assemble(const EdgeDev* __restrict__ edges, int E, int K,
                                 const int* __restrict__ inc_off, const int* __restrict__ inc_list,
                                 const EdgeOut* __restrict__ eo, double* __restrict__ H,
                                 double* __restrict__ b, double* __restrict__ F,
                                 long long* __restrict__ npairs, const int* done) {
    if (done && *done) return;
    const int ld = 6 * K;
    const int tid = threadIdx.x;
    const int blk = blockIdx.x;
    if (blk < K) {
        const int m = blk;
        if (tid < 36) {
            const int r = tid / 6, c = tid % 6;
            double s = 0.0;
            for (int k = inc_off[m]; k < inc_off[m + 1]; ++k) {
                const int e = inc_list[k] >> 1, off = 6 * (inc_list[k] & 1);
                s += eo[e].H[12 * (off + r) + off + c];
            }
            H[(long long)(6 * m + r) * ld + 6 * m + c] = s;
        } else if (tid < 42) {
            const int r = tid - 36;
            double s = 0.0;
            for (int k = inc_off[m]; k < inc_off[m + 1]; ++k) {
                const int e = inc_list[k] >> 1, off = 6 * (inc_list[k] & 1);
                s += eo[e].b[off + r];
            }
            b[6 * m + r] = s;
        }
    } else if (blk < K + E) {
        const int e = blk - K;
        if (tid < 36) {
            const int r = tid / 6, c = tid % 6;
            const int a = edges[e].a, bb = edges[e].b;
            const double v = eo[e].H[12 * r + 6 + c];
            H[(long long)(6 * a + r) * ld + 6 * bb + c] = v;
            H[(long long)(6 * bb + c) * ld + 6 * a + r] = v;
        }
    } else if (tid == 0) {
        double s = 0.0;
        long long n = 0;
        for (int e = 0; e < E; ++e) {
            s += eo[e].F;
            n += eo[e].n;
        }
        *F = s;
        *npairs = n;
    }
}

__device__ void se3_exp_dev(const double* xi, double T[12]) {
    const double* rho = xi;
    const double* phi = xi + 3;
    const double th2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
    const double th = sqrt(th2);
    double A, B, C;
    if (th < 1e-5) {
        A = 1.0 - th2 / 6.0;
        B = 0.5 - th2 / 24.0;
        C = 1.0 / 6.0 - th2 / 120.0;
    } else {
        const double s = sin(th), c = cos(th);
        A = s / th;
        B = (1.0 - c) / th2;
        C = (th - s) / (th2 * th);
    }
    double P[3][3], P2[3][3];
    skew(phi, P);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P2[i][j] = P[i][0] * P[0][j] + P[i][1] * P[1][j] + P[i][2] * P[2][j];
    for (int i = 0; i < 3; ++i) {
        double tv = 0.0;
        for (int j = 0; j < 3; ++j) {
            const double id = (i == j) ? 1.0 : 0.0;
            T[4 * i + j] = id + A * P[i][j] + B * P2[i][j];
            tv += (id + B * P[i][j] + C * P2[i][j]) * rho[j];
        }
        T[4 * i + 3] = tv;
    }
}

__device__ __forceinline__ double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double w = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) w = fmax(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (lane == 0) red[32] = w;
    }
    __syncthreads();
    const double r = red[32];
    __syncthreads();
    return r;
}

// 1/sqrt(d) for d > 0: FP32 estimate refined by two Newton-Raphson steps
// r <- r (3 - d r^2) / 2 in FP64 (each step doubles the correct bits:
// ~2^-22 -> 2^-44 -> FP64 rounding).  Outside the FP32 range the estimate
// falls back to the FP64 square root.
__device__ __forceinline__ double rsqrt_nr(double d) {
    const float f = (float)d;
    double r;
    if (f > 1e-37f && f < 1e37f) r = (double)rsqrtf(f);
    else r = 1.0 / sqrt(d);
    r = r * fma(-0.5 * d * r, r, 1.5);
    r = r * fma(-0.5 * d * r, r, 1.5);
    return r;
}

constexpr int LM_T = 512;
constexpr int LM_SMEM_N = 160;   // n <= 160 keeps the factor in shared memory

// Tail of the LM step, after the damped system is factored (L in the lower
// triangle of A, row-major n x n, with 1 / L_kk in rinv): forward and back
// substitution of y = -b in one warp, the step's infinity norm, and the
// candidate poses T_m exp(delta_m^) (frame 0 fixed).  A failed factorization
// gives a zero step.  Called by every thread of the block.
__device__ void lm_finish(int K, int n, const double* __restrict__ A, double* __restrict__ y,
                          const double* __restrict__ rinv, int fail, const double* __restrict__ Tcur,
                          double* __restrict__ Tcand, LMState* S, double* red) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nt = blockDim.x;
    if (!fail) {
        if (warp == 0) {                          // substitutions in one warp
            for (int k = 0; k < n; ++k) {         // L z = -b
                const double yk = y[k] * rinv[k];
                __syncwarp();
                if (lane == 0) y[k] = yk;
                for (int i = k + 1 + lane; i < n; i += 32) y[i] = fma(-A[(long long)i * n + k], yk, y[i]);
                __syncwarp();
            }
            for (int k = n - 1; k >= 0; --k) {    // L^T delta = z
                const double yk = y[k] * rinv[k];
                __syncwarp();
                if (lane == 0) y[k] = yk;
                for (int i = lane; i < k; i += 32) y[i] = fma(-A[(long long)k * n + i], yk, y[i]);
                __syncwarp();
            }
        }
        __syncthreads();
    } else {
        for (int i = tid; i < n; i += nt) y[i] = 0.0;
        __syncthreads();
    }
    double st = 0.0;
    for (int i = tid; i < n; i += nt) st = fmax(st, fabs(y[i]));
    st = block_max(st, red);
    // candidate poses: frame 0 fixed, T_m exp(delta_m^) otherwise
    for (int m = tid; m < K; m += nt) {
        const double* T = Tcur + 16 * m;
        double* O = Tcand + 16 * m;
        if (m == 0) {
            for (int k = 0; k < 16; ++k) O[k] = T[k];
            continue;
        }
        double E12[12];
        se3_exp_dev(y + 6 * (m - 1), E12);
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 4; ++j) {
                double s = (j == 3) ? T[4 * i + 3] : 0.0;
                for (int k = 0; k < 3; ++k) s += T[4 * i + k] * E12[4 * k + j];
                O[4 * i + j] = s;
            }
        }
        O[12] = 0.0; O[13] = 0.0; O[14] = 0.0; O[15] = 1.0;
    }
    if (tid == 0) {
        S->step_inf = st;
        S->chol_fail = fail;
    }
}

__global__ void __launch_bounds__(LM_T) k_lm_solve(int K, const double* __restrict__ Hc,
                                                   const double* __restrict__ bc,
                                                   const double* __restrict__ Tcur,
                                                   double* __restrict__ Tcand, LMState* S,
                                                   double* __restrict__ ws) {
    extern __shared__ double sm[];
    __shared__ double red[33];
    __shared__ int fail;
    if (S->done) return;
    const int n = 6 * (K - 1);
    const int ld = 6 * K;
    const int tid = threadIdx.x;
    double* A = (n <= LM_SMEM_N) ? sm : ws;
    double* y = A + (long long)n * n;
    const double lam = S->lambda;
    if (tid == 0) fail = 0;
    for (long long idx = tid; idx < (long long)n * n; idx += LM_T) {
        const int i = (int)(idx / n), j = (int)(idx % n);
        A[idx] = Hc[(long long)(6 + i) * ld + 6 + j];
    }
    double dmax = 0.0;
    for (int i = tid; i < n; i += LM_T) dmax = fmax(dmax, Hc[(long long)(6 + i) * ld + 6 + i]);
    for (int i = tid; i < n; i += LM_T) y[i] = -bc[6 + i];
    dmax = block_max(dmax, red);
    const double floor_d = 1e-9 * (dmax > 0.0 ? dmax : 1e-300);
    for (int i = tid; i < n; i += LM_T) {
        const double hii = Hc[(long long)(6 + i) * ld + 6 + i];
        A[(long long)i * n + i] = hii + lam * fmax(hii, floor_d);
    }
    __syncthreads();
    // right-looking Cholesky, lower triangle in place; the pivot's reciprocal
    // square root is kept in rinv[] so that no FP64 division or square root
    // sits on the sequential path
    double* rinv = y + n;
    const int warp = tid >> 5, lane = tid & 31;
    constexpr int NW = LM_T / 32;
    // pivot k: thread 0 (for k > 0 right after its own update of A_kk,
    // which row k + 1 of warp 0, lane 0 holds, so the pivot's chain overlaps
    // the other warps' updates instead of costing a barrier of its own)
    auto pivot = [&](int k) {
        const double d = A[(long long)k * n + k];
        const double r = rsqrt_nr(d);
        if (!(d > 0.0) || !(r > 0.0) || !isfinite(r)) fail = 1;
        else {
            A[(long long)k * n + k] = d * r;   // sqrt(d)
            rinv[k] = r;
        }
    };
    if (tid == 0 && n > 0) pivot(0);
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (fail) break;
        const double r = rinv[k];
        for (int i = k + 1 + tid; i < n; i += LM_T) A[(long long)i * n + k] *= r;
        __syncthreads();
        // rows over warps, columns j <= i over lanes
        for (int i = k + 1 + warp; i < n; i += NW) {
            const double lik = A[(long long)i * n + k];
            for (int j = k + 1 + lane; j <= i; j += 32)
                A[(long long)i * n + j] = fma(-lik, A[(long long)j * n + k], A[(long long)i * n + j]);
        }
        if (tid == 0 && k + 1 < n) pivot(k + 1);
        __syncthreads();
    }
    lm_finish(K, n, A, y, rinv, fail, Tcur, Tcand, S, red);
}

// ---- blocked Cholesky over many blocks, for large systems -----------------
// For n = 6(K-1) >= LM_BLOCKED_N the single-block factorization is bound by
// one SM reading the trailing matrix from L2; the blocked right-looking form
// spreads it over the GPU: for each tile column k (tiles of CT = 32 rows) the
// diagonal tile is factored, the tile column below it solved (one block per
// tile), and L_ik L_jk^T subtracted from every trailing tile (i, j),
// k < j <= i (one block per tile).  A sits in the workspace (row-major n x n,
// lower triangle used); rows and columns beyond n are padded as the identity.
constexpr int CT = 32;
constexpr int CH_T = 256;
constexpr int LM_BLOCKED_N = 192;

// the damped system A = H_ff + lambda Dm and y = -b_f (as k_lm_solve builds them)
__global__ void __launch_bounds__(CH_T) k_lm_prep(int K, const double* __restrict__ Hc, const double* __restrict__ bc,
                                                  const LMState* S, double* __restrict__ ws) {
    __shared__ double red[33];
    if (S->done) return;
    const int n = 6 * (K - 1), ld = 6 * K;
    double* A = ws;
    double* y = A + (long long)n * n;
    double dmax = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) dmax = fmax(dmax, Hc[(long long)(6 + i) * ld + 6 + i]);
    dmax = block_max(dmax, red);
    const double floor_d = 1e-9 * (dmax > 0.0 ? dmax : 1e-300);
    const double lam = S->lambda;
    const long long nn = (long long)n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nn;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / n), j = (int)(idx % n);
        double v = Hc[(long long)(6 + i) * ld + 6 + j];
        if (i == j) v += lam * fmax(v, floor_d);
        A[idx] = v;
    }
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = -bc[6 + i];
}

// tile (ti, tj) of A into T[CT][CT + 1]; outside n: identity on the diagonal
__device__ __forceinline__ void load_tile(const double* __restrict__ A, int n, int ti, int tj, double (*T)[CT + 1]) {
    for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) {
        const int r = e / CT, c = e % CT;
        const int gi = ti * CT + r, gj = tj * CT + c;
        T[r][c] = (gi < n && gj < n) ? A[(long long)gi * n + gj] : (gi == gj ? 1.0 : 0.0);
    }
}

// diagonal tile k: factored in shared memory by one block, written back with
// the pivot reciprocals
__global__ void __launch_bounds__(CH_T) k_chol_diag(int K, int k, LMState* S, double* __restrict__ ws) {
    __shared__ double L[CT][CT + 1];
    __shared__ int bad;
    if (S->done || S->chol_fail) return;
    const int n = 6 * (K - 1);
    double* A = ws;
    double* rinv = A + (long long)n * n + n;
    if (threadIdx.x == 0) bad = 0;
    load_tile(A, n, k, k, L);
    __syncthreads();
    for (int c = 0; c < CT; ++c) {
        if (threadIdx.x == 0) {
            const double d = L[c][c];
            if (!(d > 0.0) || !isfinite(d)) bad = 1;
            else L[c][c] = sqrt(d);
        }
        __syncthreads();
        if (bad) break;
        const double inv = 1.0 / L[c][c];
        for (int r = c + 1 + threadIdx.x; r < CT; r += blockDim.x) L[r][c] *= inv;
        __syncthreads();
        for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) {
            const int r = e / CT, j = e % CT;
            if (j > c && j <= r) L[r][j] = fma(-L[r][c], L[j][c], L[r][j]);
        }
        __syncthreads();
    }
    if (bad) {
        if (threadIdx.x == 0) S->chol_fail = 1;
        return;
    }
    for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) {
        const int r = e / CT, c = e % CT;
        const int gi = k * CT + r, gj = k * CT + c;
        if (c <= r && gi < n && gj < n) A[(long long)gi * n + gj] = L[r][c];
    }
    for (int r = threadIdx.x; r < CT; r += blockDim.x)
        if (k * CT + r < n) rinv[k * CT + r] = 1.0 / L[r][r];
}

// tile column below diagonal tile k: X L_kk^T = A_ik for tile row i = k + 1 +
// block, one row of X per thread of the first warp
__global__ void __launch_bounds__(CH_T) k_chol_panel(int K, int k, const LMState* S, double* __restrict__ ws) {
    __shared__ double L[CT][CT + 1];
    __shared__ double X[CT][CT + 1];
    if (S->done || S->chol_fail) return;
    const int n = 6 * (K - 1);
    double* A = ws;
    const int ti = k + 1 + blockIdx.x;
    load_tile(A, n, k, k, L);
    load_tile(A, n, ti, k, X);
    __syncthreads();
    if (threadIdx.x < CT) {
        const int r = threadIdx.x;
        for (int c = 0; c < CT; ++c) {
            double v = X[r][c];
            for (int j = 0; j < c; ++j) v = fma(-X[r][j], L[c][j], v);
            X[r][c] = v / L[c][c];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) {
        const int r = e / CT, c = e % CT;
        const int gi = ti * CT + r, gj = k * CT + c;
        if (gi < n && gj < n) A[(long long)gi * n + gj] = X[r][c];
    }
}

__global__ void __launch_bounds__(CH_T) k_chol_update(int K, int k, const LMState* S, double* __restrict__ ws) {
    __shared__ double Li[CT][CT + 1];
    __shared__ double Lj[CT][CT + 1];
    if (S->done || S->chol_fail) return;
    const int n = 6 * (K - 1);
    double* A = ws;
    // block b -> trailing tile (i, j), k < j <= i, rows of the lower triangle in order
    int b = blockIdx.x, i = 0;
    while (b > i) {
        b -= i + 1;
        ++i;
    }
    const int ti = k + 1 + i, tj = k + 1 + b;
    load_tile(A, n, ti, k, Li);
    load_tile(A, n, tj, k, Lj);
    __syncthreads();
    for (int e = threadIdx.x; e < CT * CT; e += blockDim.x) {
        const int r = e / CT, c = e % CT;
        const int gi = ti * CT + r, gj = tj * CT + c;
        if (gi >= n || gj >= n || gj > gi) continue;
        double v = A[(long long)gi * n + gj];
#pragma unroll 8
        for (int q = 0; q < CT; ++q) v = fma(-Li[r][q], Lj[c][q], v);
        A[(long long)gi * n + gj] = v;
    }
}

// substitutions and candidate poses after the blocked factorization
__global__ void __launch_bounds__(LM_T) k_lm_subst(int K, const double* __restrict__ Tcur,
                                                   double* __restrict__ Tcand, LMState* S,
                                                   double* __restrict__ ws) {
    __shared__ double red[33];
    if (S->done) return;
    const int n = 6 * (K - 1);
    double* A = ws;
    double* y = A + (long long)n * n;
    double* rinv = y + n;
    lm_finish(K, n, A, y, rinv, S->chol_fail, Tcur, Tcand, S, red);
}

__global__ void k_lm_accept(int K, LMState* S, const double* __restrict__ Fc,
                            const long long* __restrict__ nc, double* __restrict__ Tcur,
                            const double* __restrict__ Tcand, double* __restrict__ bcur,
                            const double* __restrict__ bcand) {
    __shared__ int s_acc;
    if (S->done) return;
    if (threadIdx.x == 0) {
        const double F = *Fc;
        const long long n = *nc;
        S->pair_terms += n;
        S->n_cand = n;
        int acc;
        if (S->first) {
            acc = 1;
            S->first = 0;
            S->F_cur = F;
        } else {
            S->iters += 1;
            const double step = S->step_inf;
            if (F > S->F_cur) {
                const double rel = (F - S->F_cur) / fmax(fabs(S->F_cur), 1e-300);
                acc = 1;
                S->F_cur = F;
                S->n_accepted += 1;
                S->lambda = fmax(S->lambda * 0.1, 1e-12);
                if (step < S->tol_step || rel < S->tol_rel_f) { S->done = 1; S->status = 0; }
            } else {
                acc = 0;
                S->lambda *= 10.0;
                if (step < S->tol_step || S->lambda > 1e10) { S->done = 1; S->status = 0; }
            }
            if (!S->done && S->iters >= S->max_iters) { S->done = 1; S->status = 4; }
        }
        S->F_cand = F;
        S->accepted = acc;
        S->chol_fail = 0;
        s_acc = acc;
    }
    __syncthreads();
    if (s_acc) {
        for (int i = threadIdx.x; i < 16 * K; i += blockDim.x) Tcur[i] = Tcand[i];
        for (int i = threadIdx.x; i < 6 * K; i += blockDim.x) bcur[i] = bcand[i];
    }
}

__global__ void k_copy_if(const LMState* S, double* __restrict__ dst, const double* __restrict__ src,
                          long long n) {
    if (!S->accepted) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
}  // namespace

void launch_edge_assemble(const EdgeDev* edges, int E, const EdgeXf* xf, const long long* acc,
                          double sigma2, EdgeOut* out, const int* done, cudaStream_t st) {
    k_edge_assemble<<<(E + 63) / 64, 64, 0, st>>>(edges, E, xf, acc, sigma2, out, done);
    count_launch();
}

void launch_frame_assemble(const EdgeDev* edges, int E, int K, const int* inc_off,
                           const int* inc_list, const EdgeOut* eout, double* H, double* b,
                           double* F, long long* npairs, const int* done, cudaStream_t st) {
    k_frame_assemble<<<K + E + 1, 64, 0, st>>>(edges, E, K, inc_off, inc_list, eout, H, b, F, npairs,
                                              done);
    count_launch();
}

void launch_lm_solve(int K, const double* H_cur, const double* b_cur, const double* poses_cur,
                     double* poses_cand, LMState* st_dev, double* ws, cudaStream_t st) {
    const int n = 6 * (K - 1);
    // factor A (n x n), right-hand side y (n) and pivot reciprocals rinv (n)
    size_t smem = (n <= LM_SMEM_N) ? (size_t)(n * n + 2 * n) * sizeof(double) : 0;
    // opt in once to the largest factor kept in shared memory (not a stream
    // operation, so it must not happen while an iteration is being captured;
    // the first call of any context runs before capture)
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_lm_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)(LM_SMEM_N * LM_SMEM_N + 2 * LM_SMEM_N) * sizeof(double)));
        attr_set = true;
    }
    if (n >= LM_BLOCKED_N) {
        const int nt = (n + CT - 1) / CT;
        const long long nn = (long long)n * n;
        k_lm_prep<<<(unsigned)std::min<long long>((nn + CH_T - 1) / CH_T, 4096), CH_T, 0, st>>>(K, H_cur, b_cur,
                                                                                            st_dev, ws);
        count_launch();
        for (int k = 0; k < nt; ++k) {
            k_chol_diag<<<1, CH_T, 0, st>>>(K, k, st_dev, ws);
            count_launch();
            const int m = nt - k - 1;
            if (m > 0) {
                k_chol_panel<<<m, CH_T, 0, st>>>(K, k, st_dev, ws);
                k_chol_update<<<m * (m + 1) / 2, CH_T, 0, st>>>(K, k, st_dev, ws);
                count_launch(2);
            }
        }
        k_lm_subst<<<1, LM_T, 0, st>>>(K, poses_cur, poses_cand, st_dev, ws);
        count_launch();
        return;
    }
    k_lm_solve<<<1, LM_T, smem, st>>>(K, H_cur, b_cur, poses_cur, poses_cand, st_dev, ws);
    count_launch();
}

void launch_lm_accept(int K, LMState* st_dev, const double* F_cand, const long long* n_cand,
                      double* poses_cur, const double* poses_cand, double* b_cur,
                      const double* b_cand, cudaStream_t st) {
    k_lm_accept<<<1, 128, 0, st>>>(K, st_dev, F_cand, n_cand, poses_cur, poses_cand, b_cur, b_cand);
    count_launch();
}

void launch_copy_if_accepted(const LMState* st_dev, double* dst, const double* src, long long n,
                             cudaStream_t st) {
    long long blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    k_copy_if<<<(unsigned)blocks, 256, 0, st>>>(st_dev, dst, src, n);
    count_launch();
}

}  // namespace rk
