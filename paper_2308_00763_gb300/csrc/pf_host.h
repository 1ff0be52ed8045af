// pf_host.h -- host-side helpers shared by the runtime, the allocation-free entry point and
// the server: configuration checks, the tracker descriptor's constants, the initial state.
#pragma once
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include "pf.h"
#include "pf_internal.h"

namespace pfk {

// NVTX range over an entry point (visible to Nsight tools; a no-op without one attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// bytes of one stored position / likelihood value
inline size_t pos_bytes(int prec) { return prec == PF_REF64 ? 8 : prec == PF_F32 ? 4 : 2; }

// floor(v) + (v - floor(v) >= 1/2): the pixel / anchor rounding (reading C3)
inline double round_half_up(double v) { return floor(v) + ((v - floor(v)) >= 0.5 ? 1.0 : 0.0); }

// |D|: lattice points with dx^2 + dy^2 <= r^2 (Eq. 3's template, reading C2)
inline int disk_count(int r) {
    int n = 0;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx)
            if (dx * dx + dy * dy <= r * r) ++n;
    return n;
}

inline pf_status check_config(const pf_config *c) {
    if (!c) return PF_ERR_ARG;
    if (c->width < 1 || c->width > 65535 || c->height < 1 || c->height > 65535) return PF_ERR_ARG;
    if (c->num_particles < 1 || c->num_particles > 2147483647ll) return PF_ERR_ARG;
    if (c->disk_radius < 0 || c->disk_radius > kMaxRadius) return PF_ERR_ARG;
    if (c->precision < PF_REF64 || c->precision > PF_BF16) return PF_ERR_ARG;
    if (!(c->sigma_x >= 0) || !(c->sigma_y >= 0)) return PF_ERR_ARG;
    if (!isfinite(c->init_x) || !isfinite(c->init_y) || !isfinite(c->drift_x) || !isfinite(c->drift_y))
        return PF_ERR_ARG;
    if (!isfinite(c->bg_level) || !isfinite(c->fg_level) || !isfinite(c->sigma_x) || !isfinite(c->sigma_y))
        return PF_ERR_ARG;
    if (fabs(c->init_x) > 1.0e6 || fabs(c->init_y) > 1.0e6) return PF_ERR_ARG;
    if (c->est_capacity < 0) return PF_ERR_ARG;
    if (c->resampler < PF_RESAMPLE_SYSTEMATIC || c->resampler > PF_RESAMPLE_REJECTION) return PF_ERR_ARG;
    // Gumbel-max draws N^2 variates a frame
    if (c->resampler == PF_RESAMPLE_GUMBEL && c->num_particles > kGumbelMaxN) return PF_ERR_ARG;
    if (c->resampler == PF_RESAMPLE_METROPOLIS || c->resampler == PF_RESAMPLE_REJECTION) {
        if (c->num_particles > kMetropolisMaxN) return PF_ERR_ARG;   // offspring index in the draw tag
        const int cap = c->resampler == PF_RESAMPLE_METROPOLIS ? kMetropolisMaxSteps : kRejectionMaxTries;
        if (c->resampler_steps < 0 || c->resampler_steps > cap) return PF_ERR_ARG;
    } else if (c->resampler_steps != 0) {
        return PF_ERR_ARG;
    }
    if (c->reserved != 0) return PF_ERR_ARG;
    // stratified points in FP32 are ordered only while (float)j is exact
    if (c->resampler == PF_RESAMPLE_STRATIFIED && c->precision != PF_REF64 && c->num_particles > (1ll << 24))
        return PF_ERR_ARG;
    if (c->flags & ~(PF_FLAG_DEBUG_ARRAYS | PF_FLAG_ACCUM32 | PF_FLAG_TUNED)) return PF_ERR_ARG;
    return PF_OK;
}

// Fill the FP32 / integer copies of the state scalars from the FP64 ones.
inline void state_copies(TrackerState &s) {
    s.M_f = static_cast<float>(s.M);
    s.invS_f = static_cast<float>(s.invS);
    s.axi = static_cast<int32_t>(s.ax);
    s.ayi = static_cast<int32_t>(s.ay);
    s.nxi = static_cast<int32_t>(s.nx);
    s.nyi = static_cast<int32_t>(s.ny);
}

// The descriptor's constants of a tracker (everything but its buffers and tiles).
inline void fill_tracker_constants(const pf_config &c, TrackerDev &T) {
    T.N = c.num_particles;
    T.W = c.width;
    T.H = c.height;
    T.r = c.disk_radius;
    T.D = disk_count(c.disk_radius);
    T.key_lo = static_cast<uint32_t>(c.seed & 0xffffffffu);
    T.key_hi = static_cast<uint32_t>(c.seed >> 32);
    T.tracker_id = c.tracker_id;
    T.flags = c.flags;
    T.c1 = c.fg_level - c.bg_level;
    T.c2 = c.bg_level + c.fg_level;
    T.den = 50.0 * T.D;
    T.kappa = static_cast<float>(1.0 / sqrt(50.0 * T.D));
    T.bg_f = static_cast<float>(c.bg_level);
    T.fg_f = static_cast<float>(c.fg_level);
    T.init_x = c.init_x; T.init_y = c.init_y;
    T.sigma_x = c.sigma_x; T.sigma_y = c.sigma_y;
    T.drift_x = c.drift_x; T.drift_y = c.drift_y;
    T.inv_n = 1.0 / static_cast<double>(c.num_particles);
    T.inv_n_f = 1.0f / static_cast<float>(c.num_particles);
    T.resampler = c.resampler;
    T.steps = c.resampler == PF_RESAMPLE_METROPOLIS   ? (c.resampler_steps ? c.resampler_steps : kMetropolisDefaultSteps)
              : c.resampler == PF_RESAMPLE_REJECTION ? (c.resampler_steps ? c.resampler_steps : kRejectionDefaultTries)
                                                     : 0;
    T.init_xf = static_cast<float>(c.init_x); T.init_yf = static_cast<float>(c.init_y);
    T.drift_xf = static_cast<float>(c.drift_x); T.drift_yf = static_cast<float>(c.drift_y);
    T.sigma_xf = static_cast<float>(c.sigma_x); T.sigma_yf = static_cast<float>(c.sigma_y);
    T.c1f = static_cast<float>(T.c1);
    T.c2Df = static_cast<float>(T.c2 * T.D);
    T.denf = static_cast<float>(T.den);
}

// The state of a fresh tracker: every particle at the initial position (reading C12).
inline TrackerState initial_state(const pf_config &c) {
    TrackerState s;
    memset(&s, 0, sizeof s);
    s.t = 0;
    s.epoch = 1;
    s.M = 0.0;
    s.S = 1.0;
    s.invS = 1.0;
    s.ax = s.nx = round_half_up(c.init_x);
    s.ay = s.ny = round_half_up(c.init_y);
    s.est_x = c.init_x;
    s.est_y = c.init_y;
    // every particle starts at the initial position
    s.bb_x0 = s.bb_x1 = static_cast<float>(c.init_x);
    s.bb_y0 = s.bb_y1 = static_cast<float>(c.init_y);
    state_copies(s);
    return s;
}

// Mark the bounding box of the stored positions unknown (the next step builds its
// likelihood tables per tile).
inline void bbox_unknown(TrackerState &s) {
    s.bb_x0 = s.bb_x1 = s.bb_y0 = s.bb_y1 = nanf("");
}

}  // namespace pfk
