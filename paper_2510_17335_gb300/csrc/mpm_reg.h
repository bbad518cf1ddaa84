// Factors of the gradient regularisers of Sec. III-E (DDBot, arXiv
// 2510.17335), for the host and the device.
#pragma once
#include <math.h>

#if defined(__CUDACC__)
#define MPM_REG_HD __host__ __device__
#else
#define MPM_REG_HD
#endif

namespace mpm {

// ---------------------------------------------------------------------------
// Regularisers of whole adjoint vectors (Sec. III-E). A vector's statistic is
// its largest magnitude (mode 1, dynamic scaling) or its sum of squares
// (mode 2, normalisation); the factor divides the vector by 10^doom + delta
// (doom = round(log10 max) - oom, only when positive) or by its norm + delta.
// ---------------------------------------------------------------------------
MPM_REG_HD inline double reg_factor(int mode, double stat, double oom, double delta) {
    if (mode == 1) {
        if (!(stat > 0.0)) return 1.0;
        const double doom = round(log10(stat)) - oom;
        return doom > 0.0 ? 1.0 / (pow(10.0, doom) + delta) : 1.0;
    }
    if (mode == 2) return 1.0 / (sqrt(stat) + delta);
    return 1.0;
}

// the statistic of a vector scaled by f, from the statistic of the vector
MPM_REG_HD inline double reg_scaled(int mode, double stat, double f) {
    return mode == 2 ? stat * f * f : stat * f;
}

// factors of the grid adjoints of one substep from their raw statistics
// (the grid reversal is linear in its input): the velocity-after-contact
// vector by s0, then the velocity-before-contact by s1, the mass by s2.
// Returns m-bar's factor s0 s1 s2 in fm and the momentum's s0 s1 in fv.
MPM_REG_HD inline void reg_grid_factors(int mode, const double* gst, double oom, double delta, float& s0out,
                                             float& fm, float& fv) {
    const double s0 = reg_factor(mode, gst[0], oom, delta);
    const double s1 = reg_factor(mode, reg_scaled(mode, gst[1], s0), oom, delta);
    const double s2 = reg_factor(mode, reg_scaled(mode, gst[2], s0 * s1), oom, delta);
    s0out = (float)s0;
    fv = (float)(s0 * s1);
    fm = (float)(s0 * s1 * s2);
}

}  // namespace mpm
