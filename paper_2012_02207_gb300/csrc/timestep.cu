// Per-body step sizes of the HOLD integrator (Appendix A).
//
// Compiled with -fmad=false: every step size is a plain function of the
// pair's FP64 data (one IEEE operation per source operation), so the split
// of a set into fast and slow bodies is reproducible bit for bit.
#include "gbfmm_internal.cuh"
#include "hold_pair.cuh"

namespace gbfmm {

namespace {

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
