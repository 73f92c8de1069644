// Host-side layout of one problem, shared by the context path (api.cu) and
// the allocation-free evaluation (noalloc.cu), so the two cannot drift apart:
// kernel constants, the per-frame uniform grids, the per-edge query and
// home-cell offsets with their fixed-point scales, and the frame -> edge
// incidence lists.  Plain arrays only (the allocation-free path keeps every
// host array on the stack).
#pragma once

#include "common.cuh"

#include <cmath>
#include <cstring>

namespace rk {

// Label row padding: the pair kernel is instantiated for these widths only
// (FP32 rows of 4..32 floats, BF16 rows of 8..32 values; 16-byte rows).
inline int sem_pad_for(int dim, bool bf16) {
    if (dim <= 0) return 0;
    static const int pads_f32[] = {4, 8, 12, 16, 20, 24, 32};
    static const int pads_bf16[] = {8, 16, 24, 32};
    if (bf16) {
        for (int pd : pads_bf16)
            if (dim <= pd) return pd;
        return 0;
    }
    for (int pd : pads_f32)
        if (dim <= pd) return pd;
    return 0;
}

// Kernel constants of Eq. kernel for validated parameters: cell size
// h = cell_scale r_c (1 + 2^-10) (cell_scale >= 1, so the 27-cell stencil
// covers every pair closer than r_c), r_c^2, the exponent scale
// -log2(e) / (2 ell^2), the label variants.
// The colour factor is set by grid_params_color once the inputs are known.
inline GridParams grid_params_for(const rkhsba_params& p) {
    GridParams g{};
    const double rc = p.cutoff_mult * p.ell;
    g.h = (p.cell_scale >= 1.0 ? p.cell_scale : 1.0) * rc * (1.0 + 1.0 / 1024.0);
    g.h_inv = 1.0 / g.h;
    g.hf = (float)g.h;
    g.hf_inv = (float)g.h_inv;
    g.hf_lo = (float)(g.h - (double)g.hf);
    g.rc2 = (float)(rc * rc);
    const double log2e = 1.4426950408889634;
    g.kg = (float)(-log2e / (2.0 * p.ell * p.ell));
    g.color = 0;
    g.kc = 0.f;
    g.sem_dim = p.sem_dim;
    g.sem_bf16 = p.sem_bf16 ? 1 : 0;
    g.sem_pad = sem_pad_for(p.sem_dim, g.sem_bf16);
    g.top_k = p.top_k;
    g.sem_min = (p.sem_min > 0.0 && p.sem_dim > 0) ? (float)p.sem_min : -__builtin_huge_valf();
    return g;
}

inline void grid_params_color(GridParams& g, bool color, double ell_color) {
    g.color = color ? 1 : 0;
    if (color) {
        const double log2e = 1.4426950408889634;
        g.kc = (float)(-log2e / (2.0 * ell_color * ell_color));
    } else {
        g.kc = 0.f;
    }
}

// Power-of-two fixed-point scale for sums bounded by `bound`: values times
// *scale stay below 2^61.  Returns 1 / *scale in FP64.
inline double bound_exp_scale(double bound, float* scale) {
    if (!(bound > 0.0) || !std::isfinite(bound)) bound = 1.0;
    int e = 61 - (int)std::ceil(std::log2(bound));
    e = e < -120 ? -120 : (e > 120 ? 120 : e);
    *scale = std::ldexp(1.0f, e);
    return std::ldexp(1.0, -e);
}

// Per-frame dense grid with a one-cell margin from the frames' cell
// bounding boxes (cmin/cmax, 3 ints per frame) and label-norm bounds
// (semn_bits: FP32 bit patterns).  Limits: max_axis cells per axis,
// max_frame_cells per frame, max_total cells over all frames (exclusive).
// Returns nullptr, or the message of the first limit that is exceeded.
inline const char* layout_frames(FrameDev* F, int K, const long long* pt_off, const int* cmin,
                                 const int* cmax, const unsigned* semn_bits, bool has_sem,
                                 long long max_axis, long long max_frame_cells, long long max_total,
                                 long long* C_total) {
    long long coff = 0;
    for (int m = 0; m < K; ++m) {
        FrameDev& f = F[m];
        f = FrameDev{};
        f.pt_off = pt_off[m];
        f.n_pts = (int)(pt_off[m + 1] - pt_off[m]);
        long long cells = 1;
        for (int k = 0; k < 3; ++k) {
            if (f.n_pts > 0) {
                f.lo[k] = cmin[3 * m + k] - 1;
                const long long d = (long long)cmax[3 * m + k] - cmin[3 * m + k] + 3;
                if (d > max_axis) return "frame extent exceeds the grid's cells per axis";
                f.dim[k] = (int)d;
            } else {
                f.lo[k] = 0;
                f.dim[k] = 1;
            }
            cells *= f.dim[k];
            if (cells > max_frame_cells) return "frame grid has more cells than allowed";
        }
        f.cell_off = coff;
        coff += cells;
        float nrm;
        std::memcpy(&nrm, &semn_bits[m], sizeof(float));
        f.sem_norm_max = has_sem ? nrm : 1.0f;
    }
    if (coff >= max_total) return "total grid cells exceed the limit";
    *C_total = coff;
    return nullptr;
}

// Per edge (a, b): its home cells (frame a's grid) and queries (frame b's
// points) in the flat per-evaluation arrays, and the fixed-point scale of
// each moment class from bounds known before any evaluation: W <= n_a n_b
// |l|max^2, |d| <= r_c, |y'| <= R (frame a's grid extent from its origin).
inline void layout_edges(EdgeDev* eh, int E, const FrameDev* fh, const GridParams& gp, double rc,
                         long long* total_bins, long long* total_q) {
    long long bins = 0, q = 0;
    for (int e = 0; e < E; ++e) {
        EdgeDev& Ed = eh[e];
        const FrameDev& Fa = fh[Ed.a];
        const FrameDev& Fb = fh[Ed.b];
        Ed.bin_off = bins;
        Ed.q_off = q;
        bins += (long long)Fa.dim[0] * Fa.dim[1] * Fa.dim[2];
        q += Fb.n_pts;
        const double smax = (double)Fa.sem_norm_max * (double)Fb.sem_norm_max * (1.0 + 1e-6) + 1e-30;
        const double Wb = (double)(Fa.n_pts > 0 ? Fa.n_pts : 1) * (double)(Fb.n_pts > 0 ? Fb.n_pts : 1) * smax;
        double R2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double lo = Fa.lo[k] * gp.h, hi = (Fa.lo[k] + Fa.dim[k]) * gp.h;
            const double mm = std::fabs(lo) > std::fabs(hi) ? std::fabs(lo) : std::fabs(hi);
            R2 += mm * mm;
        }
        const double R = std::sqrt(R2) + gp.h;
        const double bounds[MC_N] = {Wb, Wb * rc, Wb * R, Wb * R * R, Wb * rc * R, Wb * rc * rc, 1.0, 1.0};
        for (int k = 0; k < MC_N; ++k) Ed.inv_scale[k] = bound_exp_scale(bounds[k], &Ed.scale[k]);
        Ed.scale[MC_CNT] = 1.0f;
        Ed.inv_scale[MC_CNT] = 1.0;
    }
    *total_bins = bins;
    *total_q = q;
}

// Frame -> edge incidence in edge order: frame m's entries are 2e when m is
// edge e's first frame and 2e + 1 when it is the second.  inc_off [K + 1],
// inc_list [2 E]; returns the number of entries.
inline int incidence_lists(const EdgeDev* eh, int E, int K, int* inc_off, int* inc_list) {
    int n = 0;
    inc_off[0] = 0;
    for (int m = 0; m < K; ++m) {
        for (int e = 0; e < E; ++e) {
            if (eh[e].a == m) inc_list[n++] = 2 * e;
            if (eh[e].b == m) inc_list[n++] = 2 * e + 1;
        }
        inc_off[m + 1] = n;
    }
    return n;
}

}  // namespace rk
