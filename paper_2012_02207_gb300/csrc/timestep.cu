// Per-body step sizes of the HOLD integrator (Appendix A).
//
// Compiled with -fmad=false: every step size is a plain function of the
// pair's FP64 data (one IEEE operation per source operation), so the split
// of a set into fast and slow bodies is reproducible bit for bit.
#include <math_constants.h>

#include "gbfmm_internal.cuh"

namespace gbfmm {

namespace {

// Step size of body i against body j: the smaller of the free-fall time
// eta sqrt(r / a), a = G (m_i + m_j) / r^2, and the fly-by time eta r / v.
// sym: each divided by (1 - tau'/2) (Eq. step_symm), tau' its derivative
// along the two-body motion (1.5 tau (r.v)/r^2 for the free-fall time,
// tau ((r.v)/r^2 - (v.a_rel)/v^2) for the fly-by time, a_rel the two-body
// relative acceleration), capped at 1.
__device__ double tau_pair(double rx, double ry, double rz, double ux, double uy, double uz, double mij, double G,
                           double eta, bool sym) {
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

// tau_i = min over j != i; one thread per body, sources staged in shared memory
__global__ void __launch_bounds__(256) k_timesteps(int n, const double* __restrict__ x, const double* __restrict__ y,
                                                   const double* __restrict__ z, const double* __restrict__ vx,
                                                   const double* __restrict__ vy, const double* __restrict__ vz,
                                                   const double* __restrict__ m, double G, double eta, int sym,
                                                   double* __restrict__ tau) {
    __shared__ double sh[7][256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = i < n;
    const int ii = act ? i : 0;
    const double xi = x[ii], yi = y[ii], zi = z[ii], ui = vx[ii], vi = vy[ii], wi = vz[ii], mi = m[ii];
    double t = CUDART_INF;
    for (int j0 = 0; j0 < n; j0 += 256) {
        const int j = j0 + threadIdx.x;
        if (j < n) {
            sh[0][threadIdx.x] = x[j]; sh[1][threadIdx.x] = y[j]; sh[2][threadIdx.x] = z[j];
            sh[3][threadIdx.x] = vx[j]; sh[4][threadIdx.x] = vy[j]; sh[5][threadIdx.x] = vz[j];
            sh[6][threadIdx.x] = m[j];
        }
        __syncthreads();
        const int cnt = n - j0 < 256 ? n - j0 : 256;
        for (int k = 0; k < cnt; ++k) {
            if (j0 + k == i) continue;
            const double tij = tau_pair(sh[0][k] - xi, sh[1][k] - yi, sh[2][k] - zi, sh[3][k] - ui, sh[4][k] - vi,
                                        sh[5][k] - wi, mi + sh[6][k], G, eta, sym != 0);
            t = tij < t ? tij : t;
        }
        __syncthreads();
    }
    if (act) tau[i] = t;
}

}  // namespace

void timesteps_f64(int n, const double* x, const double* y, const double* z, const double* vx, const double* vy,
                   const double* vz, const double* m, double G, double eta, bool sym, double* tau, cudaStream_t st) {
    if (n > 0)
        (k_timesteps<<<(n + 255) / 256, 256, 0, st>>>(n, x, y, z, vx, vy, vz, m, G, eta, sym ? 1 : 0, tau),
         note_launch());
}

}  // namespace gbfmm
