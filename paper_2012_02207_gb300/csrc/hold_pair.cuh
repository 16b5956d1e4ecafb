// The pair step size of the HOLD integrator (Appendix A), shared by the
// step-size kernel (timestep.cu) and the device-resident recursion
// (hold.cu). Both translation units are compiled with -fmad=false, so the
// value is the same plain function of the pair's FP64 data in both, and the
// same as the oracle's.
#pragma once

#include <math_constants.h>

namespace gbfmm {

// Step size of body i against body j: the smaller of the free-fall time
// eta sqrt(r / a), a = G (m_i + m_j) / r^2, and the fly-by time eta r / v.
// sym: each divided by (1 - tau'/2) (Eq. step_symm), tau' its derivative
// along the two-body motion (1.5 tau (r.v)/r^2 for the free-fall time,
// tau ((r.v)/r^2 - (v.a_rel)/v^2) for the fly-by time, a_rel the two-body
// relative acceleration), capped at 1.
__device__ __forceinline__ double tau_pair(double rx, double ry, double rz, double ux, double uy, double uz,
                                           double mij, double G, double eta, bool sym) {
    const double r2 = rx * rx + ry * ry + rz * rz;
    const double r = sqrt(r2);
    const double v2 = ux * ux + uy * uy + uz * uz;
    const double v = sqrt(v2);
    const double gm = G * mij;
    double tff = eta * sqrt(r2 * r / gm);
    double tfl = v > 0.0 ? eta * r / v : CUDART_INF;
    if (sym) {
        const double rv = rx * ux + ry * uy + rz * uz;
        double dff = 1.5 * tff * rv / r2;
        if (dff > 1.0) dff = 1.0;
        tff = tff / (1.0 - 0.5 * dff);
        if (v > 0.0) {
            const double va = -gm * rv / (r2 * r);
            double dfl = tfl * (rv / r2 - va / v2);
            if (dfl > 1.0) dfl = 1.0;
            tfl = tfl / (1.0 - 0.5 * dfl);
        }
    }
    return tff < tfl ? tff : tfl;
}

}  // namespace gbfmm
