// Set operations of the HOLD integrator (Appendix A): gathers of a set's
// bodies into compact arrays, the stable split of a set into slow and fast
// bodies, kicks and drifts of a set. The recursion over large sets and
// their force solves are driven from the host (api.cu, fmm_hold); a small set
// evolves entirely inside one block (k_hold_small), recursion included.
//
// Compiled with -fmad=false: a drift x + dt v and a kick v + h a round as
// two operations, as the oracle does.
#include "gbfmm_internal.cuh"
#include "hold_pair.cuh"

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

// ---------------------------------------------------------------------------
// Device-resident HOLD for a small set: evolve(P, dt) of Appendix A for the k
// bodies idx[0..k), recursion included, in one block. The set's positions,
// velocities and masses are copied into shared memory; every subset of the
// recursion is a segment of the index array ix, split in place (stable: slow
// bodies first, then fast ones). A frame's split is kept as a bit mask and
// undone when the frame ends, so the parent sees its fast set in its own
// order again, as the oracle (fresh S and F arrays per level) does. Forces
// are the oracle's FP64 direct sum in the oracle's order and operations
// (r = sqrt(r^2), m / (r^2 r), no contraction), the step sizes the same
// tau_pair: the trajectory is the oracle's bit for bit.

struct HoldFrame {
    double dt;
    int lo, hi;   // the set: ix[lo..hi)
    int ns;       // slow bodies ix[lo..lo+ns) after the split; fast ones after them
    int phase;    // 0: split and evolve the fast set; 1: kick-drift-kick, fast again; 2: undo the split
    int depth;
    int pad;
};

constexpr int kHoldThreads = 256;

// accelerations of the sinks ix[s0..s1) from the sources ix[q0..q1) (a body
// does not act on itself), each sink kicked at once: v <- v + h G sum
__device__ __forceinline__ void hold_kick_from(const int* ix, int s0, int s1, int q0, int q1, const double* px,
                                               const double* py, const double* pz, const double* pm, double* pvx,
                                               double* pvy, double* pvz, double G, double soft2, double h) {
    for (int t = s0 + (int)threadIdx.x; t < s1; t += kHoldThreads) {
        const int i = ix[t];
        const double xi = px[i], yi = py[i], zi = pz[i];
        double sx = 0.0, sy = 0.0, sz = 0.0;
        for (int q = q0; q < q1; ++q) {
            const int j = ix[q];
            if (j == i) continue;
            const double dx = px[j] - xi, dy = py[j] - yi, dz = pz[j] - zi;
            double r2 = dx * dx + dy * dy + dz * dz;
            if (soft2 > 0.0) r2 = r2 + soft2;
            const double r = sqrt(r2);
            const double mr3 = pm[j] / (r2 * r);
            sx += mr3 * dx;
            sy += mr3 * dy;
            sz += mr3 * dz;
        }
        pvx[i] += h * (G * sx);
        pvy[i] += h * (G * sy);
        pvz[i] += h * (G * sz);
    }
}

// stats: {slow-system kicks, FMM solves (none here), direct solves, deepest level, splits}
__global__ void __launch_bounds__(kHoldThreads) k_hold_small(int k, const int* __restrict__ idx, double* x,
                                                             double* y, double* z, double* vx, double* vy,
                                                             double* vz, const double* __restrict__ m, double G,
                                                             double soft2, double eta, int sym, double dt,
                                                             double dt_min, int depth0,
                                                             unsigned long long* __restrict__ stats) {
    extern __shared__ __align__(16) double hsm[];
    const int W = (k + 31) >> 5;  // mask words per level
    double* px = hsm;
    double* py = px + k;
    double* pz = py + k;
    double* pvx = pz + k;
    double* pvy = pvx + k;
    double* pvz = pvy + k;
    double* pm = pvz + k;
    double* tau = pm + k;
    HoldFrame* stack = reinterpret_cast<HoldFrame*>(tau + k);  // kHoldMaxLevels frames
    int* ix = reinterpret_cast<int*>(stack + kHoldMaxLevels);
    int* tmp = ix + k;
    unsigned* fbits = reinterpret_cast<unsigned*>(tmp + k);  // kHoldMaxLevels x W
    __shared__ int s_sp, s_nf;
    const int tid = threadIdx.x;
    for (int a = tid; a < k; a += kHoldThreads) {
        const int i = idx[a];
        px[a] = x[i]; py[a] = y[i]; pz[a] = z[i];
        pvx[a] = vx[i]; pvy[a] = vy[i]; pvz[a] = vz[i];
        pm[a] = m[i];
        ix[a] = a;
    }
    unsigned long long kicks = 0, direct = 0, splits = 0, deepest = 0;
    if (tid == 0) {
        stack[0] = HoldFrame{dt, 0, k, k, 0, depth0, 0};
        s_sp = 0;
    }
    __syncthreads();
    for (;;) {
        const int sp = s_sp;
        if (sp < 0) break;
        const HoldFrame f = stack[sp];
        __syncthreads();  // every thread has its copy before thread 0 edits the stack
        const int n = f.hi - f.lo;
        unsigned* bits = fbits + (size_t)sp * W;
        if (f.phase == 0) {
            if ((unsigned long long)f.depth > deepest) deepest = (unsigned long long)f.depth;
            int ns = n;
            if (n > 1 && f.dt > dt_min && f.depth < kHoldMaxDepth && sp + 1 < kHoldMaxLevels) {
                // tau of every member within the set, then the fast flags as a mask
                for (int t = tid; t < n; t += kHoldThreads) {
                    const int i = ix[f.lo + t];
                    double tt = CUDART_INF;
                    for (int q = f.lo; q < f.hi; ++q) {
                        const int j = ix[q];
                        if (j == i) continue;
                        const double tij = tau_pair(px[j] - px[i], py[j] - py[i], pz[j] - pz[i], pvx[j] - pvx[i],
                                                    pvy[j] - pvy[i], pvz[j] - pvz[i], pm[i] + pm[j], G, eta,
                                                    sym != 0);
                        if (tij < tt) tt = tij;
                    }
                    tau[t] = tt;
                }
                __syncthreads();
                for (int t0 = 0; t0 < n; t0 += kHoldThreads) {
                    const int t = t0 + tid;
                    const unsigned b = __ballot_sync(0xffffffffu, t < n && tau[t] < f.dt);
                    if ((tid & 31) == 0 && t < n) bits[t >> 5] = b;
                }
                if (tid == 0) s_nf = 0;
                __syncthreads();
                if (tid < ((n + 31) >> 5)) atomicAdd(&s_nf, __popc(bits[tid]));
                __syncthreads();
                const int nf = s_nf;
                ns = n - nf;
                // stable split into tmp, back into the segment
                for (int t = tid; t < n; t += kHoldThreads) {
                    int before = 0;
                    for (int w = 0; w < (t >> 5); ++w) before += __popc(bits[w]);
                    const unsigned word = bits[t >> 5];
                    before += __popc(word & ((1u << (t & 31)) - 1u));
                    const bool fast = (word >> (t & 31)) & 1u;
                    tmp[fast ? ns + before : t - before] = ix[f.lo + t];
                }
                __syncthreads();
                for (int t = tid; t < n; t += kHoldThreads) ix[f.lo + t] = tmp[t];
                ++splits;
            }
            if (tid == 0) {
                stack[sp].ns = ns;
                stack[sp].phase = 1;
                if (ns < n) {
                    stack[sp + 1] = HoldFrame{0.5 * f.dt, f.lo + ns, f.hi, f.hi - f.lo - ns, 0, f.depth + 1, 0};
                    s_sp = sp + 1;
                }
            }
            __syncthreads();
            continue;
        }
        if (f.phase == 1) {
            const int s1 = f.lo + f.ns;
            if (f.ns > 0) {
                // slow bodies feel all of P, fast ones the slow ones; drift the slow ones
                const double h = 0.5 * f.dt;
                hold_kick_from(ix, f.lo, s1, f.lo, f.hi, px, py, pz, pm, pvx, pvy, pvz, G, soft2, h);
                hold_kick_from(ix, s1, f.hi, f.lo, s1, px, py, pz, pm, pvx, pvy, pvz, G, soft2, h);
                __syncthreads();
                for (int t = f.lo + tid; t < s1; t += kHoldThreads) {
                    const int i = ix[t];
                    px[i] += f.dt * pvx[i];
                    py[i] += f.dt * pvy[i];
                    pz[i] += f.dt * pvz[i];
                }
                __syncthreads();
                hold_kick_from(ix, f.lo, s1, f.lo, f.hi, px, py, pz, pm, pvx, pvy, pvz, G, soft2, h);
                hold_kick_from(ix, s1, f.hi, f.lo, s1, px, py, pz, pm, pvx, pvy, pvz, G, soft2, h);
                kicks += 2;
                direct += (f.ns < n) ? 4 : 2;
            }
            __syncthreads();
            if (tid == 0) {
                stack[sp].phase = 2;
                if (f.ns < n) {
                    stack[sp + 1] = HoldFrame{0.5 * f.dt, s1, f.hi, f.hi - s1, 0, f.depth + 1, 0};
                    s_sp = sp + 1;
                }
            }
            __syncthreads();
            continue;
        }
        // phase 2: undo this frame's split (its children undid theirs), then return
        if (f.ns < n) {
            for (int t = tid; t < n; t += kHoldThreads) {
                int before = 0;
                for (int w = 0; w < (t >> 5); ++w) before += __popc(bits[w]);
                const unsigned word = bits[t >> 5];
                before += __popc(word & ((1u << (t & 31)) - 1u));
                const bool fast = (word >> (t & 31)) & 1u;
                tmp[t] = ix[f.lo + (fast ? f.ns + before : t - before)];
            }
            __syncthreads();
            for (int t = tid; t < n; t += kHoldThreads) ix[f.lo + t] = tmp[t];
        }
        if (tid == 0) s_sp = sp - 1;
        __syncthreads();
    }
    for (int a = tid; a < k; a += kHoldThreads) {
        const int i = idx[a];
        x[i] = px[a]; y[i] = py[a]; z[i] = pz[a];
        vx[i] = pvx[a]; vy[i] = pvy[a]; vz[i] = pvz[a];
    }
    if (tid == 0) {
        atomicAdd(stats + 0, kicks);
        atomicAdd(stats + 2, direct);
        atomicMax(stats + 3, deepest);
        atomicAdd(stats + 4, splits);
    }
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

size_t hold_small_smem(int k) {
    const size_t W = (size_t)(k + 31) / 32;
    return 8 * sizeof(double) * (size_t)k + sizeof(HoldFrame) * kHoldMaxLevels + 2 * sizeof(int) * (size_t)k +
           sizeof(unsigned) * W * kHoldMaxLevels;
}

void hold_small(int k, const int* idx, double* x, double* y, double* z, double* vx, double* vy, double* vz,
                const double* m, double G, double soft, double eta, bool sym, double dt, double dt_min, int depth,
                unsigned long long* stats, cudaStream_t st) {
    if (k <= 0) return;
    const size_t sh = hold_small_smem(k);
    ensure_dyn_smem((const void*)k_hold_small, (int)hold_small_smem(kHoldSmallMax));
    (k_hold_small<<<1, kHoldThreads, sh, st>>>(k, idx, x, y, z, vx, vy, vz, m, G, soft * soft, eta, sym ? 1 : 0, dt,
                                               dt_min, depth, stats),
     note_launch());
}

}  // namespace gbfmm
