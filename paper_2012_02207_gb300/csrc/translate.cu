// Rotation-accelerated M2M and L2L (the translations of Sec. 2.1, done with
// the rotations of Sec. 2.4), one warp per child cell. M2M runs in FP64 (FP64
// mode) or double-word FP32 (mixed precision; see dword.cuh); L2L in FP64 or
// FP32.
#include "dword.cuh"
#include "gbfmm_internal.cuh"
#include "swap_tables.cuh"

namespace gbfmm {

namespace {

// With b = z_C - z_P rotated onto +z, the shift of a multipole is diagonal in m:
//     Mhat_n^m(P) = sum_k sqrt(C(n+m,k) C(n-m,k)) (rho/s_P)^k (s_C/s_P)^{n-k} Mhat_{n-k}^m(C),
// the hat form of M_n^m(P) = sum_k rho^k/k! M_{n-k}^m(C). One warp per child
// (lanes over coefficients, the vector in shared memory) writes the
// rotated-and-shifted contribution; k_m2m_sum adds the children of each parent
// in child order. GB300 runs a warp's FP64 instruction for about 64 cycles
// however few lanes are active, so every step keeps all lanes busy and no
// step divides.

// arithmetic of the two precisions
__device__ __forceinline__ double ar_add(double a, double b) { return a + b; }
__device__ __forceinline__ double ar_sub(double a, double b) { return a - b; }
__device__ __forceinline__ double ar_mul(double a, double b) { return a * b; }
__device__ __forceinline__ double ar_neg(double a) { return -a; }
__device__ __forceinline__ float ar_add(float a, float b) { return a + b; }
__device__ __forceinline__ float ar_sub(float a, float b) { return a - b; }
__device__ __forceinline__ float ar_mul(float a, float b) { return a * b; }
__device__ __forceinline__ float ar_neg(float a) { return -a; }
__device__ __forceinline__ dw ar_add(dw a, dw b) { return dw_add(a, b); }
__device__ __forceinline__ dw ar_sub(dw a, dw b) { return dw_sub(a, b); }
__device__ __forceinline__ dw ar_mul(dw a, dw b) { return dw_mul(a, b); }
__device__ __forceinline__ dw ar_neg(dw a) { return dw_neg(a); }
template <typename T> __device__ __forceinline__ T ar_from(double x);
template <> __device__ __forceinline__ double ar_from<double>(double x) { return x; }
template <> __device__ __forceinline__ dw ar_from<dw>(double x) { return dw_from(x); }
template <> __device__ __forceinline__ float ar_from<float>(double x) { return (float)x; }
__device__ __forceinline__ double ar_to(double x) { return x; }
__device__ __forceinline__ double ar_to(float x) { return (double)x; }
__device__ __forceinline__ double ar_to(dw x) { return dw_to(x); }

// tables in the working precision: swap blocks (cos_off/sin_off layout) and
// the z-shift coefficients (zshift_offset layout); FP32 and double-word read
// the (hi, lo) pair tables, FP32 their hi part
template <typename T>
struct RotTables;
template <>
struct RotTables<double> {
    const double *cosb, *sinb, *zsh;
    __device__ double c(int i) const { return __ldg(cosb + i); }
    __device__ double s(int i) const { return __ldg(sinb + i); }
    __device__ double z(int i) const { return __ldg(zsh + i); }
};
template <>
struct RotTables<dw> {
    const float2 *cosb, *sinb, *zsh;
    __device__ dw c(int i) const { const float2 v = __ldg(cosb + i); return dw{v.x, v.y}; }
    __device__ dw s(int i) const { const float2 v = __ldg(sinb + i); return dw{v.x, v.y}; }
    __device__ dw z(int i) const { const float2 v = __ldg(zsh + i); return dw{v.x, v.y}; }
};
template <>
struct RotTables<float> {
    const float2 *cosb, *sinb, *zsh;
    __device__ float c(int i) const { return __ldg(cosb + i).x; }
    __device__ float s(int i) const { return __ldg(sinb + i).x; }
    __device__ float z(int i) const { return __ldg(zsh + i).x; }
};

// coefficient q of the real layout -> (n, m, imaginary part?)
__device__ __forceinline__ void decode_q(int q, int& n, int& m, bool& im) {
    n = (int)sqrtf((float)q + 0.5f);
    while (n * n > q) --n;
    while ((n + 1) * (n + 1) <= q) ++n;
    const int r = q - n * n;
    if (r == 0) { m = 0; im = false; }
    else { m = (r + 1) >> 1; im = (r & 1) == 0; }
}

template <typename T>
struct WarpVec {
    T* v;    // (p+1)^2
    T* t;    // (p+1)^2 scratch
};

// The G threads (a warp, or a block of 128 for the few nodes of the upper
// levels) that evolve one node's vector synchronise with gsync<G>.
template <int G>
__device__ __forceinline__ void gsync() {
    if constexpr (G == 32) __syncwarp();
    else __syncthreads();
}

// pw[2m], pw[2m+1] = (c + i s)^m for m = 0..p, thread m by binary powering
template <int G, typename T>
__device__ void wpowers(T* pw, int p, T c, T s, int lane) {
    if (lane <= p) {
        T pr = ar_from<T>(1.0), pi = ar_from<T>(0.0), br = c, bi = s;
        for (int e = lane; e > 0; e >>= 1) {
            if (e & 1) {
                const T tq = ar_sub(ar_mul(pr, br), ar_mul(pi, bi));
                pi = ar_add(ar_mul(pr, bi), ar_mul(pi, br));
                pr = tq;
            }
            const T tb = ar_sub(ar_mul(br, br), ar_mul(bi, bi));
            const T tm = ar_mul(br, bi);
            bi = ar_add(tm, tm);
            br = tb;
        }
        pw[2 * lane] = pr;
        pw[2 * lane + 1] = pi;
    }
    gsync<G>();
}

// v <- Rz: coefficient m times pw_m (or its conjugate)
template <int G, typename T>
__device__ void wrotz(WarpVec<T>& w, int p, const T* pw, bool conj, int lane) {
    const int ncx = p * (p + 1) / 2;  // complex coefficients with m >= 1
    for (int q = lane; q < ncx; q += G) {
        int n = (int)((sqrtf(8.0f * q + 1.0f) - 1.0f) * 0.5f);  // q = n(n-1)/2 + (m-1), n >= 1
        while (n * (n + 1) / 2 <= q) ++n;
        while ((n - 1) * n / 2 > q) --n;
        const int mm = q - (n - 1) * n / 2 + 1;
        const T re = w.v[hre(n, mm)], im = w.v[him(n, mm)];
        const T pr = pw[2 * mm], pi = conj ? ar_neg(pw[2 * mm + 1]) : pw[2 * mm + 1];
        w.v[hre(n, mm)] = ar_sub(ar_mul(re, pr), ar_mul(im, pi));
        w.v[him(n, mm)] = ar_add(ar_mul(re, pi), ar_mul(im, pr));
    }
    gsync<G>();
}

template <int G, typename T>
__device__ void wswap(WarpVec<T>& w, int p, const RotTables<T>& tb, int lane) {
    const int nr = ncoef_real(p);
    for (int q = lane; q < nr; q += G) {
        int n, mm;
        bool im;
        decode_q(q, n, mm, im);
        T acc = ar_from<T>(0.0);
        if (!im) {
            const int a0 = cos_off(n) + mm * (n + 1);
            for (int j = (mm + n) & 1; j <= n; j += 2) acc = ar_add(acc, ar_mul(tb.c(a0 + j), w.v[hre(n, j)]));
        } else {
            const int b0 = sin_off(n) + (mm - 1) * n;
            for (int j = ((mm + n + 1) & 1) ? 1 : 2; j <= n; j += 2) acc = ar_add(acc, ar_mul(tb.s(b0 + j - 1), w.v[him(n, j)]));
        }
        w.t[q] = acc;
    }
    gsync<G>();
    T* tq = w.v; w.v = w.t; w.t = tq;
}

// The M2M z-shift gives output (n, m) n - m + 1 terms, from 1 to n + 1, so a
// lane per output leaves most lanes idle while the longest finish. Outputs
// are paired into units of n + 1 terms each: (n, 0) alone; (n, m) with
// (n, n + 1 - m) for 1 <= m <= n/2, real parts together and imaginary parts
// together; for odd n the real and imaginary parts of m = (n + 1)/2. Unit u
// counts down from degree p, so the units a warp takes at once have nearly
// equal lengths. Output A takes the first len_a terms of the unit; output B
// (absent when len_a = n + 1) the rest.
__device__ __forceinline__ void m2m_zshift_unit(int p, int u, int& n, int& ma, bool& ia, int& mb, bool& ib,
                                                int& len_a) {
    n = p;
    while (u > n) {  // degree n owns n + 1 units
        u -= n + 1;
        --n;
    }
    if (u == 0) {
        ma = mb = 0;
        ia = ib = false;
        len_a = n + 1;
        return;
    }
    if ((n & 1) && u == n) {  // odd n: both parts of m = (n + 1)/2
        ma = mb = (n + 1) >> 1;
        ia = false;
        ib = true;
        len_a = n - ma + 1;
        return;
    }
    ma = ((u - 1) >> 1) + 1;
    mb = n + 1 - ma;
    ia = ib = ((u - 1) & 1) != 0;
    len_a = n - ma + 1;
}

// shared values per warp: vector, scratch, two power tables, u^k and (s_C/s_P)^k
__host__ __device__ inline int m2m_warp_values(int p) { return 2 * ncoef_real(p) + 6 * (p + 1); }

// The geometry of the shift from node C's centre to its parent P's, one
// thread per node: with b = z_C - z_P, the angles of b (cos and sin of phi
// and theta), u = |b| / s_P and s_C / s_P. The warps of the M2M and L2L
// kernels read these instead of each evaluating the FP64 square roots and
// divisions on all of their lanes (a warp's FP64 instruction occupies the
// FP64 pipe about as long whether one lane or 32 need the value).
__global__ void k_shift_geometry(TreeView t, const double* __restrict__ zc, const double* __restrict__ hs,
                                 double* __restrict__ geo) {
    const int C = blockIdx.x * blockDim.x + threadIdx.x;
    if (C >= *t.dnn) return;
    const int P = t.parent[C];
    if (P < 0) return;  // a root shifts nowhere
    const double bx = zc[3 * C] - zc[3 * P], by = zc[3 * C + 1] - zc[3 * P + 1], bz = zc[3 * C + 2] - zc[3 * P + 2];
    const double rxy2 = bx * bx + by * by;
    const double rho = sqrt(rxy2 + bz * bz);
    const double rxy = sqrt(rxy2);
    double cp = 1.0, sp = 0.0, ct = 1.0, st = 0.0;
    if (rxy > 0.0) { cp = bx / rxy; sp = by / rxy; }
    if (rho > 0.0) { ct = bz / rho; st = rxy / rho; }
    const double sP = hs[P];
    double* g = geo + kShiftGeo * (size_t)C;
    g[0] = cp; g[1] = sp; g[2] = ct; g[3] = st;
    g[4] = rho / sP;
    g[5] = hs[C] / sP;
}

template <typename T, int G>
__global__ void __launch_bounds__(128) k_m2m_rot(TreeView t, int Lc, int p,
                                                  const double* __restrict__ geo,
                                                  const double* __restrict__ mult,
                                                  double* __restrict__ contrib, RotTables<T> tb) {
    extern __shared__ __align__(16) unsigned char sh_m2m_raw[];
    T* sh_m2m = reinterpret_cast<T*>(sh_m2m_raw);
    const int lane = threadIdx.x % G, wib = threadIdx.x / G;
    const int nr = ncoef_real(p);
    T* base = sh_m2m + (size_t)wib * m2m_warp_values(p);
    WarpVec<T> wv{base, base + nr};
    T* pwa = base + 2 * nr;        // (sin phi + i cos phi)^m: Rz(pi/2 - phi), conjugate for Rz(phi - pi/2)
    T* pwb = pwa + 2 * (p + 1);    // (cos theta - i sin theta)^m: Rz(-theta), conjugate for Rz(theta)
    T* upow = pwb + 2 * (p + 1);   // u^k
    T* spow = upow + (p + 1);      // (s_C/s_P)^k
    const int C = t.dls[Lc] + blockIdx.x * (blockDim.x / G) + wib;
    if (C >= t.dls[Lc + 1]) return;
    const int P = t.parent[C];
    const double* src = mult + (size_t)nr * C;
    for (int q = lane; q < nr; q += G) wv.v[q] = ar_from<T>(src[q]);
    (void)P;
    const double* gc = geo + kShiftGeo * (size_t)C;  // the shift's geometry (k_shift_geometry)
    const double cp = gc[0], sp = gc[1], ct = gc[2], st = gc[3], u = gc[4], sg = gc[5];
    wpowers<G, T>(pwa, p, ar_from<T>(sp), ar_from<T>(cp), lane);
    wpowers<G, T>(pwb, p, ar_from<T>(ct), ar_from<T>(-st), lane);
    // u^k and (s_C/s_P)^k, lane k by binary powering
    if (lane <= p) {
        T a = ar_from<T>(1.0), b = ar_from<T>(1.0), ba = ar_from<T>(u), bb = ar_from<T>(sg);
        for (int e = lane; e > 0; e >>= 1) {
            if (e & 1) { a = ar_mul(a, ba); b = ar_mul(b, bb); }
            ba = ar_mul(ba, ba);
            bb = ar_mul(bb, bb);
        }
        upow[lane] = a;
        spow[lane] = b;
    }
    gsync<G>();
    wrotz<G>(wv, p, pwa, false, lane);  // Rz(pi/2 - phi)
    wswap<G>(wv, p, tb, lane);
    wrotz<G>(wv, p, pwb, false, lane);  // Rz(-theta)
    wswap<G>(wv, p, tb, lane);
    // z-shift into the scratch vector, over balanced units (m2m_zshift_unit):
    // each output's terms in the same order as a plain loop over k
    const int nunits = (p + 1) * (p + 2) / 2;
    for (int u = lane; u < nunits; u += G) {
        int n, ma, mb, len_a;
        bool ia, ib;
        m2m_zshift_unit(p, u, n, ma, ia, mb, ib, len_a);
        const int cza = zshift_offset(n, ma), czb = zshift_offset(n, mb);
        T acc_a = ar_from<T>(0.0), acc_b = ar_from<T>(0.0);
        for (int s = 0; s <= n; ++s) {
            const bool in_a = s < len_a;
            const int k = in_a ? s : s - len_a;
            const int mm = in_a ? ma : mb;
            const bool im = in_a ? ia : ib;
            const T term = ar_mul(ar_mul(tb.z((in_a ? cza : czb) + k), upow[k]),
                                  ar_mul(spow[n - k], wv.v[im ? him(n - k, mm) : hre(n - k, mm)]));
            const T sum = ar_add(in_a ? acc_a : acc_b, term);  // one add on every lane, no divergence
            acc_a = in_a ? sum : acc_a;
            acc_b = in_a ? acc_b : sum;
        }
        wv.t[ia ? him(n, ma) : hre(n, ma)] = acc_a;
        if (len_a <= n) wv.t[ib ? him(n, mb) : hre(n, mb)] = acc_b;
    }
    gsync<G>();
    { T* tq = wv.v; wv.v = wv.t; wv.t = tq; }
    wswap<G>(wv, p, tb, lane);
    wrotz<G>(wv, p, pwb, true, lane);   // Rz(theta)
    wswap<G>(wv, p, tb, lane);
    wrotz<G>(wv, p, pwa, true, lane);   // Rz(phi - pi/2)
    double* dst = contrib + (size_t)nr * C;
    for (int q = lane; q < nr; q += G) dst[q] = ar_to(wv.v[q]);
}

// Rotation-accelerated L2L: with b = z_C - z_P rotated onto +z,
//     Fhat_n^m(C) += sigma^n sum_{k=0}^{p-n} sqrt(C(n+k+m,k) C(n+k-m,k)) u^k Fhat_{n+k}^m(P),
// u = rho/s_P, sigma = s_C/s_P (the hat form of F_n^m(C) = sum_k rho^k/k! F_{n+k}^m(P)
// on the axis), between the same rotations as M2M. The local coefficients
// (T = float or double) are added to the child's, which the M2L wrote.
template <typename T, int G>
__global__ void __launch_bounds__(128) k_l2l_rot(TreeView t, int L, int p,
                                                  const double* __restrict__ geo,
                                                  T* __restrict__ loc, RotTables<T> tb) {
    extern __shared__ __align__(16) unsigned char sh_l2l_raw[];
    T* sh = reinterpret_cast<T*>(sh_l2l_raw);
    const int lane = threadIdx.x % G, wib = threadIdx.x / G;
    const int nr = ncoef_real(p);
    T* base = sh + (size_t)wib * m2m_warp_values(p);
    WarpVec<T> wv{base, base + nr};
    T* pwa = base + 2 * nr;
    T* pwb = pwa + 2 * (p + 1);
    T* upow = pwb + 2 * (p + 1);
    T* spow = upow + (p + 1);
    const int C = t.dls[L] + blockIdx.x * (blockDim.x / G) + wib;
    if (C >= t.dls[L + 1]) return;
    const int P = t.parent[C];
    const T* src = loc + (size_t)nr * P;
    for (int q = lane; q < nr; q += G) wv.v[q] = src[q];
    const double* gc = geo + kShiftGeo * (size_t)C;  // the shift's geometry (k_shift_geometry)
    const double cp = gc[0], sp = gc[1], ct = gc[2], st = gc[3], u = gc[4], sg = gc[5];
    wpowers<G, T>(pwa, p, ar_from<T>(sp), ar_from<T>(cp), lane);
    wpowers<G, T>(pwb, p, ar_from<T>(ct), ar_from<T>(-st), lane);
    if (lane <= p) {
        T a = ar_from<T>(1.0), b = ar_from<T>(1.0), ba = ar_from<T>(u), bb = ar_from<T>(sg);
        for (int e = lane; e > 0; e >>= 1) {
            if (e & 1) { a = ar_mul(a, ba); b = ar_mul(b, bb); }
            ba = ar_mul(ba, ba);
            bb = ar_mul(bb, bb);
        }
        upow[lane] = a;
        spow[lane] = b;
    }
    gsync<G>();
    wrotz<G>(wv, p, pwa, false, lane);  // Rz(pi/2 - phi)
    wswap<G>(wv, p, tb, lane);
    wrotz<G>(wv, p, pwb, false, lane);  // Rz(-theta)
    wswap<G>(wv, p, tb, lane);
    for (int q = lane; q < nr; q += G) {
        int n, mm;
        bool im;
        decode_q(q, n, mm, im);
        T acc = ar_from<T>(0.0);
        for (int k = 0; k <= p - n; ++k)
            acc = ar_add(acc, ar_mul(ar_mul(tb.z(zshift_offset(n + k, mm) + k), upow[k]),
                                     wv.v[im ? him(n + k, mm) : hre(n + k, mm)]));
        wv.t[q] = ar_mul(spow[n], acc);
    }
    gsync<G>();
    { T* tq = wv.v; wv.v = wv.t; wv.t = tq; }
    wswap<G>(wv, p, tb, lane);
    wrotz<G>(wv, p, pwb, true, lane);   // Rz(theta)
    wswap<G>(wv, p, tb, lane);
    wrotz<G>(wv, p, pwa, true, lane);   // Rz(phi - pi/2)
    T* dst = loc + (size_t)nr * C;
    for (int q = lane; q < nr; q += G) dst[q] = ar_add(dst[q], wv.v[q]);
}

__global__ void k_m2m_sum(TreeView t, int L, int nr, const double* __restrict__ contrib,
                          double* __restrict__ mult) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int P = t.dls[L] + (int)(q / nr), j = (int)(q % nr);
    if (P >= t.dls[L + 1] || t.nchild[P] == 0) return;
    const int c0 = t.first_child[P];
    double s = 0.0;
    for (int c = c0; c < c0 + t.nchild[P]; ++c) s += contrib[(size_t)nr * c + j];
    mult[(size_t)nr * P + j] = s;
}

// Levels with fewer nodes than kSmallLevel give each node a block of 128
// threads: the steps of one node then take a quarter of the passes, which
// is what bounds the time of a launch that leaves most SMs idle.
constexpr int kSmallLevel = 2048;

template <typename T>
void launch_m2m(const TreeView& t, int Lc, int p, const double* geo,
                const double* mult, double* contrib, const RotTables<T>& tb, cudaStream_t st) {
    const size_t per = (size_t)m2m_warp_values(p) * sizeof(T);
    const int cnt = t.lvl_cnt[Lc];
    if (cnt < kSmallLevel) {
        ensure_dyn_smem((const void*)k_m2m_rot<T, 128>, 100 * 1024);
        (k_m2m_rot<T, 128><<<cnt, 128, per, st>>>(t, Lc, p, geo, mult, contrib, tb), note_launch());
        return;
    }
    ensure_dyn_smem((const void*)k_m2m_rot<T, 32>, 100 * 1024);
    (k_m2m_rot<T, 32><<<(cnt + 3) / 4, 128, 4 * per, st>>>(t, Lc, p, geo, mult, contrib, tb), note_launch());
}

template <typename T>
void launch_l2l(const TreeView& t, int L, int p, const double* geo, T* loc,
                const RotTables<T>& tb, cudaStream_t st) {
    const size_t per = (size_t)m2m_warp_values(p) * sizeof(T);
    const int cnt = t.lvl_cnt[L];
    if (cnt < kSmallLevel) {
        ensure_dyn_smem((const void*)k_l2l_rot<T, 128>, 100 * 1024);
        (k_l2l_rot<T, 128><<<cnt, 128, per, st>>>(t, L, p, geo, loc, tb), note_launch());
        return;
    }
    ensure_dyn_smem((const void*)k_l2l_rot<T, 32>, 100 * 1024);
    (k_l2l_rot<T, 32><<<(cnt + 3) / 4, 128, 4 * per, st>>>(t, L, p, geo, loc, tb), note_launch());
}

}  // namespace

void shift_geometry(const TreeView& t, const double* zc, const double* hs, double* geo, cudaStream_t st) {
    if (t.nnodes > 0)
        (k_shift_geometry<<<(t.nnodes + 127) / 128, 128, 0, st>>>(t, zc, hs, geo), note_launch());
}

void l2l_level(const TreeView& t, int L, int p, const double* geo, void* loc, const DevTables& tb, bool fp32,
               cudaStream_t st) {
    if (t.lvl_cnt[L] <= 0) return;
    if (fp32)
        launch_l2l<float>(t, L, p, geo, static_cast<float*>(loc),
                          RotTables<float>{tb.swap_cos_dw, tb.swap_sin_dw, tb.zshift_dw}, st);
    else
        launch_l2l<double>(t, L, p, geo, static_cast<double*>(loc),
                           RotTables<double>{tb.swap_cos, tb.swap_sin, tb.zshift}, st);
}

void m2m_level(const TreeView& t, int L, int p, const double* geo, double* mult, double* contrib,
               const DevTables& tb, bool dword, cudaStream_t st) {
    if (t.lvl_cnt[L + 1] <= 0) return;
    const int nr = ncoef_real(p);
    if (dword)
        launch_m2m<dw>(t, L + 1, p, geo, mult, contrib,
                       RotTables<dw>{tb.swap_cos_dw, tb.swap_sin_dw, tb.zshift_dw}, st);
    else
        launch_m2m<double>(t, L + 1, p, geo, mult, contrib,
                           RotTables<double>{tb.swap_cos, tb.swap_sin, tb.zshift}, st);
    const int64_t work = (int64_t)t.lvl_cnt[L] * nr;
    (k_m2m_sum<<<(int)((work + 127) / 128), 128, 0, st>>>(t, L, nr, contrib, mult), note_launch());
}

}  // namespace gbfmm
