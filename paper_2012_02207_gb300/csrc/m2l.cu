// Rotation-accelerated M2L (Sec. 2.4).
//
// For a source cell A and a target cell B with R = z_A - z_B, the source's
// hat multipole is rotated so that R points along +z:
//     Rz(pi/2 - phi), swap x<->z, Rz(-theta), swap x<->z
// (phi, theta the angles of R; swap-Rz-swap is a rotation about x), then
// translated along z in O(p^3):
//     Fhat'_n^m = sum_{k=m}^{p-n} (-1)^{k+m} (n+k)!/(w_n^m w_k^m) Mhat'_k^m u^k v^n / rho,
// with u = s_A/rho, v = s_B/rho, and rotated back with the inverse sequence
//     swap, Rz(theta), swap, Rz(phi - pi/2).
// z-rotations are diagonal (coefficient m times e^{i m angle}); the swap
// matrices of the hat basis are exact tables (cosine and sine blocks, half of
// each block is zero by parity).
//
// One warp per target cell gathers over the target's sources (sorted by
// index); lane l takes sources l, l+32, ... and accumulates its own partial
// local expansion; the 32 partials are summed in a fixed order in FP64, so
// the result does not depend on scheduling.
#include "gbfmm_internal.cuh"

namespace gbfmm {

namespace {

__host__ __device__ constexpr int cos_off(int n) { return n * (n + 1) * (2 * n + 1) / 6; }
__host__ __device__ constexpr int sin_off(int n) { return (n - 1) * n * (2 * n - 1) / 6; }
constexpr int kSwapCos32 = cos_off(kMaxPF32 + 1);
constexpr int kSwapSin32 = sin_off(kMaxPF32 + 1);

__constant__ float c_swc[kSwapCos32];
__constant__ float c_sws[kSwapSin32];
__constant__ float c_tz[kMaxPF32 + 1][kMaxPF32 + 1][kMaxPF32 + 1];  // (n+k)!/(w_n^m w_k^m) at [n][k][m]

// ------------------------------------------------------------------------
// FP32, compile-time order P: coefficients live in registers.

template <int P>
__device__ __forceinline__ void rotz32(float* a, float c, float s) {
    float pr = 1.0f, pi = 0.0f;
#pragma unroll
    for (int m = 1; m <= P; ++m) {
        const float t = pr * c - pi * s;
        pi = pr * s + pi * c;
        pr = t;
#pragma unroll
        for (int n = m; n <= P; ++n) {
            const float re = a[hre(n, m)], im = a[him(n, m)];
            a[hre(n, m)] = re * pr - im * pi;
            a[him(n, m)] = re * pi + im * pr;
        }
    }
}

template <int P>
__device__ __forceinline__ void swap32(float* a) {
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        float tc[P + 1], ts[P + 1];
#pragma unroll
        for (int m = 0; m <= n; ++m) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j <= n; ++j)
                if (((j + m + n) & 1) == 0) acc += c_swc[cos_off(n) + m * (n + 1) + j] * a[hre(n, j)];
            tc[m] = acc;
        }
#pragma unroll
        for (int m = 1; m <= n; ++m) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 1; j <= n; ++j)
                if (((j + m + n) & 1) == 1) acc += c_sws[sin_off(n) + (m - 1) * n + (j - 1)] * a[him(n, j)];
            ts[m] = acc;
        }
#pragma unroll
        for (int m = 0; m <= n; ++m) a[hre(n, m)] = tc[m];
#pragma unroll
        for (int m = 1; m <= n; ++m) a[him(n, m)] = ts[m];
    }
}

template <int P>
__device__ __forceinline__ void ztrans32(float* a, float u, float v, float irho) {
    float up[P + 1], vp[P + 1];
    up[0] = 1.0f;
    vp[0] = irho;
#pragma unroll
    for (int k = 1; k <= P; ++k) { up[k] = up[k - 1] * u; vp[k] = vp[k - 1] * v; }
#pragma unroll
    for (int m = 0; m <= P; ++m) {
        float tr[P + 1], ti[P + 1];
#pragma unroll
        for (int k = m; k <= P; ++k) {
            const float sg = ((k + m) & 1) ? -up[k] : up[k];
            tr[k] = sg * a[hre(k, m)];
            ti[k] = m ? sg * a[him(k, m)] : 0.0f;
        }
#pragma unroll
        for (int n = m; n <= P; ++n) {
            float sr = 0.0f, si = 0.0f;
#pragma unroll
            for (int k = m; k <= P - n; ++k) {
                sr += c_tz[n][k][m] * tr[k];
                si += c_tz[n][k][m] * ti[k];
            }
            a[hre(n, m)] = vp[n] * sr;
            if (m) a[him(n, m)] = vp[n] * si;
        }
    }
}

template <int P>
__global__ void __launch_bounds__(128) k_m2l32(int nnodes, const uint64_t* __restrict__ keys,
                                                const uint32_t* __restrict__ off, int nb,
                                                const float* __restrict__ mult, int stride,
                                                const double* __restrict__ zc,
                                                const double* __restrict__ rr,
                                                float* __restrict__ loc) {
    constexpr int NR = (P + 1) * (P + 1);
    extern __shared__ float sh_acc[];  // [warp][NR][32]
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float* acc = sh_acc + (size_t)wib * NR * 32;
    const uint64_t mask = (1ull << nb) - 1ull;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int b = blockIdx.x * (blockDim.x >> 5) + wib; b < nnodes; b += nwarps) {
#pragma unroll
        for (int j = 0; j < NR; ++j) acc[j * 32 + lane] = 0.0f;
        const uint32_t q0 = off[b], q1 = off[b + 1];
        const double bx = zc[3 * b], by = zc[3 * b + 1], bz = zc[3 * b + 2];
        const float sb = (float)hat_scale(rr[b]);
        for (uint32_t q = q0 + lane; q < q1; q += 32) {
            const int a = (int)(keys[q] & mask);
            const float rx = (float)(zc[3 * a] - bx), ry = (float)(zc[3 * a + 1] - by),
                        rz = (float)(zc[3 * a + 2] - bz);
            const float sa = (float)hat_scale(rr[a]);
            float c[NR];
            const float* src = mult + (size_t)stride * a;
#pragma unroll
            for (int j = 0; j < NR; ++j) c[j] = __ldg(src + j);
            const float rxy2 = rx * rx + ry * ry;
            const float rho = sqrtf(rxy2 + rz * rz);
            const float rxy = sqrtf(rxy2);
            float cp = 1.0f, sp = 0.0f;
            if (rxy > 0.0f) { cp = rx / rxy; sp = ry / rxy; }
            const float ct = rz / rho, st = rxy / rho;
            const float irho = 1.0f / rho;
            rotz32<P>(c, sp, cp);      // Rz(pi/2 - phi)
            swap32<P>(c);
            rotz32<P>(c, ct, -st);     // Rz(-theta)
            swap32<P>(c);
            ztrans32<P>(c, sa * irho, sb * irho, irho);
            swap32<P>(c);
            rotz32<P>(c, ct, st);      // Rz(theta)
            swap32<P>(c);
            rotz32<P>(c, sp, -cp);     // Rz(phi - pi/2)
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[j * 32 + lane] += c[j];
        }
        __syncwarp();
        float* out = loc + (size_t)stride * b;
        for (int j = 0; j < NR; ++j) {
            double v = (double)acc[j * 32 + lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) out[j] = (float)v;
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------
// FP64, runtime order p <= 30: coefficients in per-thread local arrays.

struct Swap64 {
    const double* cosb;
    const double* sinb;
};

__device__ void rotz64(double* a, int p, double c, double s) {
    double pr = 1.0, pi = 0.0;
    for (int m = 1; m <= p; ++m) {
        const double t = pr * c - pi * s;
        pi = pr * s + pi * c;
        pr = t;
        for (int n = m; n <= p; ++n) {
            const double re = a[hre(n, m)], im = a[him(n, m)];
            a[hre(n, m)] = re * pr - im * pi;
            a[him(n, m)] = re * pi + im * pr;
        }
    }
}

template <int PM>
__device__ void swap64(double* a, int p, const Swap64& sw) {
    double tc[PM + 1], ts[PM + 1];
    for (int n = 1; n <= p; ++n) {
        const double* A = sw.cosb + cos_off(n);
        const double* B = sw.sinb + sin_off(n);
        for (int m = 0; m <= n; ++m) {
            double acc = 0.0;
            for (int j = (m + n) & 1; j <= n; j += 2) acc += __ldg(A + m * (n + 1) + j) * a[hre(n, j)];
            tc[m] = acc;
        }
        for (int m = 1; m <= n; ++m) {
            double acc = 0.0;
            for (int j = ((m + n + 1) & 1) ? 1 : 2; j <= n; j += 2)
                acc += __ldg(B + (m - 1) * n + (j - 1)) * a[him(n, j)];
            ts[m] = acc;
        }
        for (int m = 0; m <= n; ++m) a[hre(n, m)] = tc[m];
        for (int m = 1; m <= n; ++m) a[him(n, m)] = ts[m];
    }
}

template <int PM>
__device__ void ztrans64(double* a, int p, double u, double v, double irho, const double* fact,
                         const double* iw) {
    double up[PM + 1], vp[PM + 1], tr[PM + 1], ti[PM + 1];
    up[0] = 1.0;
    vp[0] = irho;
    for (int k = 1; k <= p; ++k) { up[k] = up[k - 1] * u; vp[k] = vp[k - 1] * v; }
    for (int m = 0; m <= p; ++m) {
        for (int k = m; k <= p; ++k) {
            const double sg = ((k + m) & 1) ? -up[k] : up[k];
            tr[k] = sg * a[hre(k, m)];
            ti[k] = m ? sg * a[him(k, m)] : 0.0;
        }
        for (int n = m; n <= p; ++n) {
            double sr = 0.0, si = 0.0;
            const double iwn = __ldg(iw + n * (kMaxP + 2) + m);
            for (int k = m; k <= p - n; ++k) {
                const double cz = __ldg(fact + n + k) * iwn * __ldg(iw + k * (kMaxP + 2) + m);
                sr += cz * tr[k];
                si += cz * ti[k];
            }
            a[hre(n, m)] = vp[n] * sr;
            if (m) a[him(n, m)] = vp[n] * si;
        }
    }
}

// PM bounds the per-thread arrays: p <= PM.
template <int PM>
__global__ void __launch_bounds__(64) k_m2l64(int nnodes, int p, const uint64_t* __restrict__ keys,
                                               const uint32_t* __restrict__ off, int nb,
                                               const double* __restrict__ mult,
                                               const double* __restrict__ zc,
                                               const double* __restrict__ rr,
                                               double* __restrict__ loc, Swap64 sw,
                                               const double* __restrict__ fact,
                                               const double* __restrict__ iw) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nr = ncoef_real(p);
    const uint64_t mask = (1ull << nb) - 1ull;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    double c[ncoef_real(PM)], acc[ncoef_real(PM)];
    for (int b = blockIdx.x * (blockDim.x >> 5) + wib; b < nnodes; b += nwarps) {
        for (int j = 0; j < nr; ++j) acc[j] = 0.0;
        const uint32_t q0 = off[b], q1 = off[b + 1];
        const double bx = zc[3 * b], by = zc[3 * b + 1], bz = zc[3 * b + 2];
        const double sb = hat_scale(rr[b]);
        for (uint32_t q = q0 + lane; q < q1; q += 32) {
            const int a = (int)(keys[q] & mask);
            const double rx = zc[3 * a] - bx, ry = zc[3 * a + 1] - by, rz = zc[3 * a + 2] - bz;
            const double sa = hat_scale(rr[a]);
            const double* src = mult + (size_t)nr * a;
            for (int j = 0; j < nr; ++j) c[j] = src[j];
            const double rxy2 = rx * rx + ry * ry;
            const double rho = sqrt(rxy2 + rz * rz);
            const double rxy = sqrt(rxy2);
            double cp = 1.0, sp = 0.0;
            if (rxy > 0.0) { cp = rx / rxy; sp = ry / rxy; }
            const double ct = rz / rho, st = rxy / rho;
            const double irho = 1.0 / rho;
            rotz64(c, p, sp, cp);
            swap64<PM>(c, p, sw);
            rotz64(c, p, ct, -st);
            swap64<PM>(c, p, sw);
            ztrans64<PM>(c, p, sa * irho, sb * irho, irho, fact, iw);
            swap64<PM>(c, p, sw);
            rotz64(c, p, ct, st);
            swap64<PM>(c, p, sw);
            rotz64(c, p, sp, -cp);
            for (int j = 0; j < nr; ++j) acc[j] += c[j];
        }
        double* out = loc + (size_t)nr * b;
        for (int j = 0; j < nr; ++j) {
            double v = acc[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) out[j] = v;
        }
    }
}

template <int P>
void launch_m2l32(int nnodes, const uint64_t* keys, const uint32_t* off, int nb, const float* mult,
                  int stride, const double* zc, const double* r, float* loc, cudaStream_t st) {
    const size_t sh = (size_t)4 * (P + 1) * (P + 1) * 32 * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_m2l32<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        attr = true;
    }
    (k_m2l32<P><<<152 * 4, 128, sh, st>>>(nnodes, keys, off, nb, mult, stride, zc, r, loc), note_launch());
}
}  // namespace

void upload_m2l_tables(const HostTables& h, const double* swap_cos, const double* swap_sin) {
    static float swc[kSwapCos32], sws[kSwapSin32];
    for (int i = 0; i < kSwapCos32; ++i) swc[i] = (float)swap_cos[i];
    for (int i = 0; i < kSwapSin32; ++i) sws[i] = (float)swap_sin[i];
    static float tz[kMaxPF32 + 1][kMaxPF32 + 1][kMaxPF32 + 1];
    for (int n = 0; n <= kMaxPF32; ++n)
        for (int k = 0; k <= kMaxPF32; ++k)
            for (int m = 0; m <= kMaxPF32; ++m)
                tz[n][k][m] = (m <= n && m <= k) ? (float)(h.fact[n + k] * h.iw[n][m] * h.iw[k][m]) : 0.0f;
    cudaMemcpyToSymbol(c_swc, swc, sizeof(swc));
    cudaMemcpyToSymbol(c_sws, sws, sizeof(sws));
    cudaMemcpyToSymbol(c_tz, tz, sizeof(tz));
}

void m2l_f64(int nnodes, int p, const uint64_t* keys, const uint32_t* off, int nb,
             const double* mult, const double* zc, const double* r, double* loc,
             const DevTables& tb, cudaStream_t st) {
    const Swap64 sw{tb.swap_cos, tb.swap_sin};
    if (p <= 8) {
        (k_m2l64<8><<<152 * 16, 64, 0, st>>>(nnodes, p, keys, off, nb, mult, zc, r, loc, sw, tb.fact, tb.iw), note_launch());
    } else if (p <= 16) {
        (k_m2l64<16><<<152 * 16, 64, 0, st>>>(nnodes, p, keys, off, nb, mult, zc, r, loc, sw, tb.fact, tb.iw), note_launch());
    } else {
        // ~17 KB of local arrays per thread: a 48 KB shared-memory request caps
        // residency at 4 blocks (256 threads) per SM to bound the local-memory reservation
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_m2l64<kMaxP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024);
            attr = true;
        }
        (k_m2l64<kMaxP><<<152 * 4, 64, 48 * 1024, st>>>(nnodes, p, keys, off, nb, mult, zc, r, loc, sw, tb.fact, tb.iw), note_launch());
    }
}

void m2l_f32(int nnodes, int p, const uint64_t* keys, const uint32_t* off, int nb,
             const float* mult, const double* zc, const double* r, float* loc, cudaStream_t st) {
    const int stride = ncoef_real(p);
    switch (p) {
        case 4: launch_m2l32<4>(nnodes, keys, off, nb, mult, stride, zc, r, loc, st); break;
        case 6: launch_m2l32<6>(nnodes, keys, off, nb, mult, stride, zc, r, loc, st); break;
        case 8: launch_m2l32<8>(nnodes, keys, off, nb, mult, stride, zc, r, loc, st); break;
        case 10: launch_m2l32<10>(nnodes, keys, off, nb, mult, stride, zc, r, loc, st); break;
        case 12: launch_m2l32<12>(nnodes, keys, off, nb, mult, stride, zc, r, loc, st); break;
        case 14: launch_m2l32<14>(nnodes, keys, off, nb, mult, stride, zc, r, loc, st); break;
        default: break;  // other orders run the FP64 kernel (the caller checks m2l32_supported)
    }
}

bool m2l32_supported(int p) { return p == 4 || p == 6 || p == 8 || p == 10 || p == 12 || p == 14; }

}  // namespace gbfmm
