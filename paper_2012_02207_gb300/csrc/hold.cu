// Set operations of the HOLD integrator (Appendix A): gathers of a set's
// bodies into compact arrays, the stable split of a set into slow and fast
// bodies, kicks and drifts of a set. The recursion and the force solves are
// driven from the host (api.cu, fmm_hold).
//
// Compiled with -fmad=false: a drift x + dt v and a kick v + h a round as
// two operations, as the oracle does.
#include "gbfmm_internal.cuh"

namespace gbfmm {

namespace {

inline int grid_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

// out[c][a] = field c of body idx[a]: x, y, z, vx, vy, vz, m (7 arrays of k);
// zero_from >= 0 zeroes the masses of a >= zero_from
__global__ void k_hold_gather(int k, const int* __restrict__ idx, const double* __restrict__ x,
                              const double* __restrict__ y, const double* __restrict__ z,
                              const double* __restrict__ vx, const double* __restrict__ vy,
                              const double* __restrict__ vz, const double* __restrict__ m, double* __restrict__ out,
                              int stride, int zero_from) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= k) return;
    const int i = idx[a];
    out[a] = x[i];
    out[stride + a] = y[i];
    out[2 * (size_t)stride + a] = z[i];
    out[3 * (size_t)stride + a] = vx[i];
    out[4 * (size_t)stride + a] = vy[i];
    out[5 * (size_t)stride + a] = vz[i];
    out[6 * (size_t)stride + a] = (zero_from >= 0 && a >= zero_from) ? 0.0 : m[i];
}

__global__ void k_hold_flags(int k, const double* __restrict__ tau, double dt, uint32_t* __restrict__ flag) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < k) flag[a] = tau[a] < dt ? 1u : 0u;
}

// stable split by an exclusive scan of the fast flags
__global__ void k_hold_compact(int k, const int* __restrict__ idx, const uint32_t* __restrict__ flag,
                               const uint32_t* __restrict__ scan, int* __restrict__ S, int* __restrict__ F) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= k) return;
    const uint32_t f = scan[a];
    if (flag[a]) F[f] = idx[a];
    else S[a - f] = idx[a];
}

// v[idx[a]] += h (acc[a] - sub[a]) (sub may be NULL); acc: 3 arrays of stride
__global__ void k_hold_kick(int k, const int* __restrict__ idx, const double* __restrict__ acc,
                            const double* __restrict__ sub, int stride, int sub_stride, double h,
                            double* __restrict__ vx, double* __restrict__ vy, double* __restrict__ vz) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= k) return;
    const int i = idx[a];
    double ax = acc[a], ay = acc[stride + a], az = acc[2 * (size_t)stride + a];
    if (sub) {
        ax = ax - sub[a];
        ay = ay - sub[sub_stride + a];
        az = az - sub[2 * (size_t)sub_stride + a];
    }
    vx[i] = vx[i] + h * ax;
    vy[i] = vy[i] + h * ay;
    vz[i] = vz[i] + h * az;
}

__global__ void k_hold_drift(int k, const int* __restrict__ idx, double dt, double* __restrict__ x,
                             double* __restrict__ y, double* __restrict__ z, const double* __restrict__ vx,
                             const double* __restrict__ vy, const double* __restrict__ vz) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= k) return;
    const int i = idx[a];
    x[i] = x[i] + dt * vx[i];
    y[i] = y[i] + dt * vy[i];
    z[i] = z[i] + dt * vz[i];
}

__global__ void k_hold_iota(int n, int* __restrict__ idx) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n) idx[a] = a;
}

}  // namespace

void hold_iota(int n, int* idx, cudaStream_t st) {
    if (n > 0) (k_hold_iota<<<grid_for(n, 256), 256, 0, st>>>(n, idx), note_launch());
}

void hold_gather(int k, const int* idx, const double* x, const double* y, const double* z, const double* vx,
                 const double* vy, const double* vz, const double* m, double* out, int stride, int zero_from,
                 cudaStream_t st) {
    if (k > 0)
        (k_hold_gather<<<grid_for(k, 256), 256, 0, st>>>(k, idx, x, y, z, vx, vy, vz, m, out, stride, zero_from),
         note_launch());
}

void hold_split(int k, const int* idx, const double* tau, double dt, uint32_t* flag, uint32_t* scan, int* S, int* F,
                uint32_t* nfast, uint32_t* scratch, cudaStream_t st) {
    if (k <= 0) return;
    (k_hold_flags<<<grid_for(k, 256), 256, 0, st>>>(k, tau, dt, flag), note_launch());
    cudaMemcpyAsync(scan, flag, 4 * (size_t)k, cudaMemcpyDeviceToDevice, st);
    scan_exclusive_u32_large(scan, k, nfast, scratch, st);
    (k_hold_compact<<<grid_for(k, 256), 256, 0, st>>>(k, idx, flag, scan, S, F), note_launch());
}

void hold_kick(int k, const int* idx, const double* acc, const double* sub, int stride, int sub_stride, double h,
               double* vx, double* vy, double* vz, cudaStream_t st) {
    if (k > 0)
        (k_hold_kick<<<grid_for(k, 256), 256, 0, st>>>(k, idx, acc, sub, stride, sub_stride, h, vx, vy, vz),
         note_launch());
}

void hold_drift(int k, const int* idx, double dt, double* x, double* y, double* z, const double* vx,
                const double* vy, const double* vz, cudaStream_t st) {
    if (k > 0) (k_hold_drift<<<grid_for(k, 256), 256, 0, st>>>(k, idx, dt, x, y, z, vx, vy, vz), note_launch());
}

}  // namespace gbfmm
