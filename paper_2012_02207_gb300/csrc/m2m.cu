// Rotation-accelerated M2M (Sec. 2.1 translation, done with the rotations of
// Sec. 2.4) in FP64, one warp per child cell.
#include "gbfmm_internal.cuh"
#include "swap_tables.cuh"

namespace gbfmm {

namespace {

// ------------------------------------------------------------------------
// Rotation-accelerated M2M (FP64). With b = z_C - z_P rotated onto +z, the
// shift of a multipole is diagonal in m:
//     Mhat_n^m(P) = sum_k sqrt(C(n+m,k) C(n-m,k)) (rho/s_P)^k (s_C/s_P)^{n-k} Mhat_{n-k}^m(C),
// the hat form of M_n^m(P) = sum_k rho^k/k! M_{n-k}^m(C). One warp per child
// (lanes over coefficients, the vector in shared memory: FP64 arithmetic is
// slow per instruction, so the chain per child must be short) writes the
// rotated-and-shifted contribution; k_m2m_sum adds the children of each parent
// in child order.

// coefficient q of the real layout -> (n, m, imaginary part?)
__device__ __forceinline__ void decode_q(int q, int& n, int& m, bool& im) {
    n = (int)sqrtf((float)q + 0.5f);
    while (n * n > q) --n;
    while ((n + 1) * (n + 1) <= q) ++n;
    const int r = q - n * n;
    if (r == 0) { m = 0; im = false; }
    else { m = (r + 1) >> 1; im = (r & 1) == 0; }
}

// shared doubles per warp: vector, scratch, two power tables, u^k and (s_C/s_P)^k
__host__ __device__ inline int m2m_warp_doubles(int p) { return 2 * ncoef_real(p) + 6 * (p + 1); }

struct WarpVec {
    double* v;    // (p+1)^2
    double* t;    // (p+1)^2 scratch
};

// pw[2m], pw[2m+1] = (c + i s)^m for m = 0..p, lane m by binary powering
// (FP64 costs the same per warp instruction however few lanes are active,
// so a short chain on every lane beats a long chain on one).
__device__ void wpowers(double* pw, int p, double c, double s, int lane) {
    if (lane <= p) {
        double pr = 1.0, pi = 0.0, br = c, bi = s;
        for (int e = lane; e > 0; e >>= 1) {
            if (e & 1) { const double tq = pr * br - pi * bi; pi = pr * bi + pi * br; pr = tq; }
            const double tb = br * br - bi * bi;
            bi = 2.0 * br * bi;
            br = tb;
        }
        pw[2 * lane] = pr;
        pw[2 * lane + 1] = pi;
    }
    __syncwarp();
}

// v <- Rz: coefficient m times pw_m (or its conjugate)
__device__ void wrotz(WarpVec& w, int p, const double* pw, bool conj, int lane) {
    const int ncx = p * (p + 1) / 2;  // complex coefficients with m >= 1
    for (int q = lane; q < ncx; q += 32) {
        int n = (int)((sqrtf(8.0f * q + 1.0f) - 1.0f) * 0.5f);  // q = n(n-1)/2 + (m-1), n >= 1
        while (n * (n + 1) / 2 <= q) ++n;
        while ((n - 1) * n / 2 > q) --n;
        const int mm = q - (n - 1) * n / 2 + 1;
        const double re = w.v[hre(n, mm)], im = w.v[him(n, mm)];
        const double pr = pw[2 * mm], pi = conj ? -pw[2 * mm + 1] : pw[2 * mm + 1];
        w.v[hre(n, mm)] = re * pr - im * pi;
        w.v[him(n, mm)] = re * pi + im * pr;
    }
    __syncwarp();
}

__device__ void wswap(WarpVec& w, int p, const Swap64& sw, int lane) {
    const int nr = ncoef_real(p);
    for (int q = lane; q < nr; q += 32) {
        int n, mm;
        bool im;
        decode_q(q, n, mm, im);
        double acc = 0.0;
        if (!im) {
            const double* A = sw.cosb + cos_off(n) + mm * (n + 1);
            for (int j = (mm + n) & 1; j <= n; j += 2) acc += __ldg(A + j) * w.v[hre(n, j)];
        } else {
            const double* B = sw.sinb + sin_off(n) + (mm - 1) * n;
            for (int j = ((mm + n + 1) & 1) ? 1 : 2; j <= n; j += 2) acc += __ldg(B + j - 1) * w.v[him(n, j)];
        }
        w.t[q] = acc;
    }
    __syncwarp();
    double* tq = w.v; w.v = w.t; w.t = tq;
}

__global__ void __launch_bounds__(128) k_m2m_rot(TreeView t, int k0, int k1, int p,
                                                  const double* __restrict__ zc,
                                                  const double* __restrict__ hs,
                                                  const double* __restrict__ mult,
                                                  double* __restrict__ contrib, Swap64 sw,
                                                  const double* __restrict__ zsh) {
    extern __shared__ double sh_m2m[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nr = ncoef_real(p);
    double* base = sh_m2m + (size_t)wib * m2m_warp_doubles(p);
    WarpVec wv{base, base + nr};
    double* pwa = base + 2 * nr;        // (sin phi + i cos phi)^m: Rz(pi/2 - phi), conjugate for Rz(phi - pi/2)
    double* pwb = pwa + 2 * (p + 1);    // (cos theta - i sin theta)^m: Rz(-theta), conjugate for Rz(theta)
    double* upow = pwb + 2 * (p + 1);   // u^k
    double* spow = upow + (p + 1);      // (s_C/s_P)^k
    const int C = k0 + blockIdx.x * (blockDim.x >> 5) + wib;
    if (C >= k1) return;
    const int P = t.parent[C];
    const double* src = mult + (size_t)nr * C;
    for (int q = lane; q < nr; q += 32) wv.v[q] = src[q];
    const double bx = zc[3 * C] - zc[3 * P], by = zc[3 * C + 1] - zc[3 * P + 1], bz = zc[3 * C + 2] - zc[3 * P + 2];
    const double rxy2 = bx * bx + by * by;
    const double rho = sqrt(rxy2 + bz * bz);
    const double rxy = sqrt(rxy2);
    double cp = 1.0, sp = 0.0, ct = 1.0, st = 0.0;
    if (rxy > 0.0) { cp = bx / rxy; sp = by / rxy; }
    if (rho > 0.0) { ct = bz / rho; st = rxy / rho; }
    const double sP = hs[P];
    const double u = rho / sP, sg = hs[C] / sP;
    wpowers(pwa, p, sp, cp, lane);
    wpowers(pwb, p, ct, -st, lane);
    // u^k and (s_C/s_P)^k, lane k by binary powering
    if (lane <= p) {
        double a = 1.0, b = 1.0, ba = u, bb = sg;
        for (int e = lane; e > 0; e >>= 1) {
            if (e & 1) { a *= ba; b *= bb; }
            ba *= ba;
            bb *= bb;
        }
        upow[lane] = a;
        spow[lane] = b;
    }
    __syncwarp();
    wrotz(wv, p, pwa, false, lane);  // Rz(pi/2 - phi)
    wswap(wv, p, sw, lane);
    wrotz(wv, p, pwb, false, lane);  // Rz(-theta)
    wswap(wv, p, sw, lane);
    // z-shift into the scratch vector
    for (int q = lane; q < nr; q += 32) {
        int n, mm;
        bool im;
        decode_q(q, n, mm, im);
        const double* cz = zsh + zshift_offset(n, mm);
        double acc = 0.0;
        for (int k = 0; k <= n - mm; ++k)
            acc += (__ldg(cz + k) * upow[k]) * (spow[n - k] * wv.v[im ? him(n - k, mm) : hre(n - k, mm)]);
        wv.t[q] = acc;
    }
    __syncwarp();
    { double* tq = wv.v; wv.v = wv.t; wv.t = tq; }
    wswap(wv, p, sw, lane);
    wrotz(wv, p, pwb, true, lane);   // Rz(theta)
    wswap(wv, p, sw, lane);
    wrotz(wv, p, pwa, true, lane);   // Rz(phi - pi/2)
    double* dst = contrib + (size_t)nr * C;
    for (int q = lane; q < nr; q += 32) dst[q] = wv.v[q];
}

__global__ void k_m2m_sum(TreeView t, int k0, int k1, int nr, const double* __restrict__ contrib,
                          double* __restrict__ mult) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int P = k0 + (int)(q / nr), j = (int)(q % nr);
    if (P >= k1 || t.nchild[P] == 0) return;
    const int c0 = t.first_child[P];
    double s = 0.0;
    for (int c = c0; c < c0 + t.nchild[P]; ++c) s += contrib[(size_t)nr * c + j];
    mult[(size_t)nr * P + j] = s;
}

}  // namespace

void m2m_level_f64(const TreeView& t, int parent0, int parent1, int child0, int child1, int p,
                   const double* zc, const double* hs, double* mult, double* contrib, const DevTables& tb,
                   cudaStream_t st) {
    if (child1 <= child0) return;
    const Swap64 sw{tb.swap_cos, tb.swap_sin};
    const int nr = ncoef_real(p);
    const size_t sh = (size_t)4 * m2m_warp_doubles(p) * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_m2m_rot, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
        attr = true;
    }
    const int nblk = (child1 - child0 + 3) / 4;
    (k_m2m_rot<<<nblk, 128, sh, st>>>(t, child0, child1, p, zc, hs, mult, contrib, sw, tb.zshift), note_launch());
    const int64_t work = (int64_t)(parent1 - parent0) * nr;
    (k_m2m_sum<<<(int)((work + 127) / 128), 128, 0, st>>>(t, parent0, parent1, nr, contrib, mult), note_launch());
}

}  // namespace gbfmm
