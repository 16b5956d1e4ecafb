// Upward and downward passes on hat-normalised expansions.
//
// The library stores multipoles and locals in the basis
//   Shat_n^m(r) = sqrt((n+m)!(n-m)!) Upsilon_n^m(r)   (Schmidt semi-normalised r^n Y_n^m)
// scaled by the cell size s (its radius r_A, Sec. 2.3):
//   Mhat_n^m = sum_i m_i Shat_n^m((x_i - z_A)/s_A)        = M_n^m w_n^m / s_A^n
//   Fhat_n^m = F_n^m s_B^n / w_n^m
// with M, F the moments and local coefficients of Sec. 2.2 and w_n^m =
// sqrt((n+m)!(n-m)!). Every hat coefficient is bounded by the cell mass (or
// the local field), so the same code runs in FP32 without overflow.
// The degree norms of Sec. 2.3 become P_n = s_A^n sqrt(sum_m |Mhat_n^m|^2).
//
// Real layout of a vector: degree n at offset n^2 as [Re m=0, Re 1, Im 1, ...].
#include "gbfmm_internal.cuh"
#include "dword.cuh"

namespace gbfmm {

namespace {

__constant__ float c_w32[kMaxPF32 + 2][kMaxPF32 + 2];
__constant__ float c_iw32[kMaxPF32 + 2][kMaxPF32 + 2];
__constant__ float c_rec_a32[kMaxPF32 + 1][kMaxPF32 + 1];
__constant__ float c_rec_b32[kMaxPF32 + 1][kMaxPF32 + 1];
__constant__ float c_diag32[kMaxPF32 + 1];
__constant__ float c_sub32[kMaxPF32 + 1];

__host__ __device__ constexpr int tri(int n, int m) { return n * (n + 1) / 2 + m; }

template <typename T>
struct Cx { T re, im; };

template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// Table access for both precisions: FP64 from global tables, FP32 from constants.
struct TabF64 {
    const double *w, *iw, *rec_a, *rec_b, *diag, *sub;
    __device__ double W(int n, int m) const { return w[n * (kMaxP + 2) + m]; }
    __device__ double IW(int n, int m) const { return iw[n * (kMaxP + 2) + m]; }
    __device__ double A(int n, int m) const { return rec_a[n * (kMaxP + 1) + m]; }
    __device__ double B(int n, int m) const { return rec_b[n * (kMaxP + 1) + m]; }
    __device__ double D(int m) const { return diag[m]; }
    __device__ double Sb(int m) const { return sub[m]; }
};
struct TabF32 {
    __device__ float W(int n, int m) const { return c_w32[n][m]; }
    __device__ float IW(int n, int m) const { return c_iw32[n][m]; }
    __device__ float A(int n, int m) const { return c_rec_a32[n][m]; }
    __device__ float B(int n, int m) const { return c_rec_b32[n][m]; }
    __device__ float D(int m) const { return c_diag32[m]; }
    __device__ float Sb(int m) const { return c_sub32[m]; }
};

// double-word copies of the recurrence constants (mixed-precision P2M)
__constant__ dw c_dw_a[kMaxP + 1][kMaxP + 1];
__constant__ dw c_dw_b[kMaxP + 1][kMaxP + 1];
__constant__ dw c_dw_d[kMaxP + 1];
__constant__ dw c_dw_s[kMaxP + 1];

// All Shat_n^m(x,y,z), 0 <= m <= n <= p, into out[tri(n,m)] (sequential).
template <typename T, typename Tab>
__device__ void shat_all(int p, T x, T y, T z, const Tab& tb, Cx<T>* out) {
    const T r2 = x * x + y * y + z * z;
    Cx<T> d{T(1), T(0)};
    const Cx<T> xp{x, y};
    for (int m = 0; m <= p; ++m) {
        if (m > 0) {
            d = cmul(d, xp);
            d.re *= tb.D(m);
            d.im *= tb.D(m);
        }
        out[tri(m, m)] = d;
        if (m + 1 <= p) out[tri(m + 1, m)] = {tb.Sb(m) * z * d.re, tb.Sb(m) * z * d.im};
        for (int n = m + 2; n <= p; ++n) {
            const T a = tb.A(n, m) * z, b = tb.B(n, m) * r2;
            const Cx<T> u = out[tri(n - 1, m)], v = out[tri(n - 2, m)];
            out[tri(n, m)] = {a * u.re - b * v.re, a * u.im - b * v.im};
        }
    }
}

// conjugate-symmetric access X_n^m, m in [-n, n], to a tri-stored vector
template <typename T>
__device__ __forceinline__ Cx<T> tri_get(const Cx<T>* a, int n, int m) {
    if (m >= 0) return a[tri(n, m)];
    Cx<T> v = a[tri(n, -m)];
    return ((-m) & 1) ? Cx<T>{-v.re, v.im} : Cx<T>{v.re, -v.im};
}
// same for the real layout
template <typename T>
__device__ __forceinline__ Cx<T> real_get(const T* a, int n, int m) {
    const int am = m < 0 ? -m : m;
    Cx<T> v{a[hre(n, am)], am ? a[him(n, am)] : T(0)};
    if (m >= 0) return v;
    return (am & 1) ? Cx<T>{-v.re, v.im} : Cx<T>{v.re, -v.im};
}

// ---- P2M (FP64): one warp per leaf, one lane per body. Column by column
// (order m), each lane runs the hat recurrence for its body and writes
// m_i Shat_n^m((x_i - z)/s), n = m..p, to a per-warp shared tile
// [entry][lane]; lane e then adds entry e over the 32 bodies. The body order
// of every sum is fixed (chunks of 32 in order, lanes in order).
template <int PM, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_p2m(TreeView t, int p, TabF64 tb,
                                              const double* __restrict__ xs,
                                              const double* __restrict__ ys,
                                              const double* __restrict__ zs,
                                              const double* __restrict__ ms,
                                              const double* __restrict__ zc,
                                              const double* __restrict__ hs,
                                              double* __restrict__ mult) {
    __shared__ double sh_tile[WARPS][2 * (PM + 1)][33];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double (*tile)[33] = sh_tile[wib];
    const int nr = ncoef_real(p);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int k = blockIdx.x * (blockDim.x >> 5) + wib, nnodes = *t.dnn; k < nnodes; k += nwarps) {
        if (t.nchild[k] != 0) continue;
        const double is = 1.0 / hs[k];
        const double cx = zc[3 * k], cy = zc[3 * k + 1], cz = zc[3 * k + 2];
        // lane e owns entries e and e + 32 of every column (a column has 2(p-m+1) <= 62 reals)
        double acc[PM + 1][2];
#pragma unroll
        for (int m = 0; m <= PM; ++m) { acc[m][0] = 0.0; acc[m][1] = 0.0; }
        for (int i0 = t.begin[k]; i0 < t.end[k]; i0 += 32) {
            const int i = i0 + lane;
            const bool act = i < t.end[k];
            const int nact = t.end[k] - i0 < 32 ? t.end[k] - i0 : 32;  // bodies in this chunk
            const double x = act ? (xs[i] - cx) * is : 0.0, y = act ? (ys[i] - cy) * is : 0.0,
                         z = act ? (zs[i] - cz) * is : 0.0, w = act ? ms[i] : 0.0;
            const double r2 = x * x + y * y + z * z;
            double dre = w, dim = 0.0;  // w * Shat_m^m
#pragma unroll
            for (int m = 0; m <= PM; ++m) {
                if (m <= p) {
                    if (m > 0) {
                        const double tq = dre * x - dim * y;
                        dim = (dre * y + dim * x) * tb.D(m);
                        dre = tq * tb.D(m);
                    }
                    double s1r = dre, s1i = dim, s2r = 0.0, s2i = 0.0;
                    tile[0][lane] = dre;
                    tile[1][lane] = dim;
                    for (int n = m + 1; n <= p; ++n) {
                        double vr, vi;
                        if (n == m + 1) {
                            vr = tb.Sb(m) * z * s1r;
                            vi = tb.Sb(m) * z * s1i;
                        } else {
                            const double a = tb.A(n, m) * z, b = tb.B(n, m) * r2;
                            vr = a * s1r - b * s2r;
                            vi = a * s1i - b * s2i;
                        }
                        tile[2 * (n - m)][lane] = vr;
                        tile[2 * (n - m) + 1][lane] = vi;
                        s2r = s1r; s2i = s1i; s1r = vr; s1i = vi;
                    }
                    __syncwarp();
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int ent = lane + 32 * h;
                        if (ent < 2 * (p - m + 1)) {
                            double s = acc[m][h];
                            for (int l = 0; l < nact; ++l) s += tile[ent][l];  // the rest are zeros
                            acc[m][h] = s;
                        }
                    }
                    __syncwarp();
                }
            }
        }
        double* out = mult + (size_t)nr * k;
#pragma unroll
        for (int m = 0; m <= PM; ++m) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ent = lane + 32 * h;
                if (m <= p && ent < 2 * (p - m + 1)) {
                    const int n = m + (ent >> 1);
                    if (ent & 1) { if (m) out[him(n, m)] = acc[m][h]; }
                    else out[hre(n, m)] = acc[m][h];
                }
            }
        }
    }
}

// The same P2M in double-word FP32 arithmetic (mixed precision): the
// positions relative to the leaf centre are formed in FP64, split into
// double words, and every recurrence step and tile sum runs on the FP32
// pipes in the same order as k_p2m. The result is stored in FP64; its
// relative error is of order 1e-13 instead of 1e-16, far below what the
// FP32 translations downstream add.
// Shared memory per warp: the tile of one chunk's harmonics, 2(p+1) rows of
// 33 (one per body, padded), and the sums, p+1 columns of 2(p+1) entries.
__host__ __device__ inline int p2m_dw_warp_values(int p) { return 2 * (p + 1) * 33 + (p + 1) * 2 * (p + 1); }

template <int PM, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_p2m_dw(TreeView t, int p,
                                                 const double* __restrict__ xs,
                                                 const double* __restrict__ ys,
                                                 const double* __restrict__ zs,
                                                 const double* __restrict__ ms,
                                                 const double* __restrict__ zc,
                                                 const double* __restrict__ hs,
                                                 double* __restrict__ mult) {
    extern __shared__ __align__(16) unsigned char sh_p2m_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int np1 = p + 1, ne = 2 * (p + 1);
    dw* tile_base = reinterpret_cast<dw*>(sh_p2m_raw) + (size_t)wib * p2m_dw_warp_values(p);
    dw* acc_base = tile_base + ne * 33;
    // tile[row][body], acc[column m][entry]
    auto tile = [&](int r) { return tile_base + r * 33; };
    auto acc = [&](int m) { return acc_base + m * ne; };
    (void)np1;
    const int nr = ncoef_real(p);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const dw zero = dw_make(0.f, 0.f);
    for (int k = blockIdx.x * (blockDim.x >> 5) + wib, nnodes = *t.dnn; k < nnodes; k += nwarps) {
        if (t.nchild[k] != 0) continue;
        const double is = 1.0 / hs[k];
        const double cx = zc[3 * k], cy = zc[3 * k + 1], cz = zc[3 * k + 2];
        for (int e = lane; e < np1 * ne; e += 32) acc_base[e] = zero;
        for (int i0 = t.begin[k]; i0 < t.end[k]; i0 += 32) {
            const int i = i0 + lane;
            const bool act = i < t.end[k];
            const int nact = t.end[k] - i0 < 32 ? t.end[k] - i0 : 32;
            const dw x = act ? dw_from((xs[i] - cx) * is) : zero, y = act ? dw_from((ys[i] - cy) * is) : zero,
                     z = act ? dw_from((zs[i] - cz) * is) : zero, w = act ? dw_from(ms[i]) : zero;
            const dw r2 = dw_add(dw_add(dw_mul(x, x), dw_mul(y, y)), dw_mul(z, z));
            dw dre = w, dim = zero;  // w * Shat_m^m
            // one code path for every column m (a rolled loop keeps the code small)
#pragma unroll 1
            for (int m = 0; m <= p; ++m) {
                if (m > 0) {
                    const dw tq = dw_sub(dw_mul(dre, x), dw_mul(dim, y));
                    dim = dw_mul(dw_add(dw_mul(dre, y), dw_mul(dim, x)), c_dw_d[m]);
                    dre = dw_mul(tq, c_dw_d[m]);
                }
                dw s1r = dre, s1i = dim, s2r = zero, s2i = zero;
                tile(0)[lane] = dre;
                tile(1)[lane] = dim;
                for (int n = m + 1; n <= p; ++n) {
                    dw vr, vi;
                    if (n == m + 1) {
                        const dw sz = dw_mul(c_dw_s[m], z);
                        vr = dw_mul(sz, s1r);
                        vi = dw_mul(sz, s1i);
                    } else {
                        const dw a = dw_mul(c_dw_a[n][m], z), b = dw_mul(c_dw_b[n][m], r2);
                        vr = dw_sub(dw_mul(a, s1r), dw_mul(b, s2r));
                        vi = dw_sub(dw_mul(a, s1i), dw_mul(b, s2i));
                    }
                    tile(2 * (n - m))[lane] = vr;
                    tile(2 * (n - m) + 1)[lane] = vi;
                    s2r = s1r; s2i = s1i; s1r = vr; s1i = vi;
                }
                __syncwarp();
                for (int ent = lane; ent < 2 * (p - m + 1); ent += 32) {
                    dw sacc = acc(m)[ent];
                    for (int l = 0; l < nact; ++l) sacc = dw_add(sacc, tile(ent)[l]);
                    acc(m)[ent] = sacc;
                }
                __syncwarp();
            }
        }
        double* out = mult + (size_t)nr * k;
        for (int m = 0; m <= p; ++m)
            for (int ent = lane; ent < 2 * (p - m + 1); ent += 32) {
                const int n = m + (ent >> 1);
                if (ent & 1) { if (m) out[him(n, m)] = dw_to(acc(m)[ent]); }
                else out[hre(n, m)] = dw_to(acc(m)[ent]);
            }
        __syncwarp();
    }
}

// a grid of as many blocks as fit on the SMs (warps stride over the leaves)
template <int PM, int WARPS>
void launch_p2m_dw(const TreeView& t, int p, const double* xs, const double* ys, const double* zs, const double* w,
                   const double* zc, const double* hs, double* mult, cudaStream_t st) {
    const int sh = (int)(WARPS * p2m_dw_warp_values(p) * sizeof(dw));
    ensure_dyn_smem((const void*)k_p2m_dw<PM, WARPS>, sh);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2m_dw<PM, WARPS>, WARPS * 32, sh) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    (k_p2m_dw<PM, WARPS><<<device_sm_count() * per_sm, WARPS * 32, sh, st>>>(t, p, xs, ys, zs, w, zc, hs, mult),
     note_launch());
}

// P_n = s^n sqrt(sum_{m=-n}^{n} |Mhat_n^m|^2)  (Sec. 2.3)
// (also the FP32 copies used by the walk's screen: Phat_n = P_n / s^n and r)
__global__ void k_pnorm(const int* __restrict__ dnn, int p, const double* __restrict__ mult,
                        const double* __restrict__ rr, const double* __restrict__ hs,
                        double* __restrict__ Pk, float* __restrict__ Phat,
                        float* __restrict__ r32) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *dnn) return;
    const double* M = mult + (size_t)ncoef_real(p) * k;
    const double s = hs[k];
    double sp = 1.0;
    for (int n = 0; n <= p; ++n) {
        double acc = M[hre(n, 0)] * M[hre(n, 0)];
        for (int m = 1; m <= n; ++m) acc += 2.0 * (M[hre(n, m)] * M[hre(n, m)] + M[him(n, m)] * M[him(n, m)]);
        const double nrm = sqrt(acc);
        Pk[(size_t)(p + 1) * k + n] = sp * nrm;
        Phat[(size_t)(p + 1) * k + n] = (float)nrm;
        sp *= s;
    }
    r32[k] = (float)rr[k];
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, const int* __restrict__ dnn, int nr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (int64_t)*dnn * nr) b[i] = (float)a[i];
}

// ---- L2L: one block per child, one thread per output (n, m >= 0)
//   Fhat_n^m(C) += sum_{k<=p-n} sum_l conj(Shat_k^l(b)) beta' sigma^n Fhat_{n+k}^{m+l}(P),
//   b = (z_C - z_P)/s_P, sigma = s_C/s_P, beta' = w_{n+k}^{m+l} / (w_k^l w_n^m).
template <typename T, typename Tab>
__global__ void k_l2l(TreeView t, int L, int p, Tab tb, const double* __restrict__ zc,
                      const double* __restrict__ hs, T* __restrict__ loc) {
    extern __shared__ __align__(16) unsigned char sh_l2l_raw[];
    const int C = t.dls[L] + blockIdx.x;
    if (C >= t.dls[L + 1]) return;
    const int P = t.parent[C];
    const int nc = tri(p + 1, 0), nr = ncoef_real(p);
    Cx<T>* S = reinterpret_cast<Cx<T>*>(sh_l2l_raw);
    T* Fp = reinterpret_cast<T*>(S + nc);
    T* sig = Fp + nr;
    const double sP = hs[P];
    if (threadIdx.x == 0) {
        const T bx = (T)((zc[3 * C] - zc[3 * P]) / sP), by = (T)((zc[3 * C + 1] - zc[3 * P + 1]) / sP),
                bz = (T)((zc[3 * C + 2] - zc[3 * P + 2]) / sP);
        shat_all<T>(p, bx, by, bz, tb, S);
        const T sg = (T)(hs[C] / sP);
        T pw = T(1);
        for (int j = 0; j <= p; ++j) { sig[j] = pw; pw *= sg; }
    }
    for (int i = threadIdx.x; i < nr; i += blockDim.x) Fp[i] = loc[(size_t)nr * P + i];
    __syncthreads();
    for (int q = threadIdx.x; q < nc; q += blockDim.x) {
        int n = 0;
        while (tri(n + 1, 0) <= q) ++n;
        const int m = q - tri(n, 0);
        T are = T(0), aim = T(0);
        for (int k = 0; k <= p - n; ++k) {
            for (int l = -k; l <= k; ++l) {
                const int ml = m + l;
                const T beta = tb.W(n + k, ml < 0 ? -ml : ml) * tb.IW(k, l < 0 ? -l : l) * tb.IW(n, m);
                Cx<T> sv = tri_get(S, k, l);
                sv.im = -sv.im;
                const Cx<T> prod = cmul(sv, real_get(Fp, n + k, ml));
                are += beta * prod.re;
                aim += beta * prod.im;
            }
        }
        T* out = loc + (size_t)nr * C;
        out[hre(n, m)] += sig[n] * are;
        if (m) out[him(n, m)] += sig[n] * aim;
    }
}

__global__ void k_hat_scales(const int* __restrict__ dnn, const int* __restrict__ parent,
                             const double* __restrict__ r, double* __restrict__ hs) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *dnn) return;
    int root = k;
    while (parent[root] >= 0) root = parent[root];
    const double floor_s = kHatFloor * (r[root] > 0.0 ? r[root] : 1.0);
    hs[k] = r[k] > floor_s ? r[k] : floor_s;
}

__global__ void k_node_centres(const int* __restrict__ dnn, const double* __restrict__ zc, const double* __restrict__ hs,
                               float4* __restrict__ zhi, float4* __restrict__ zlo) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *dnn) return;
    float h[3], l[3];
    for (int d = 0; d < 3; ++d) {
        const double z = zc[3 * k + d];
        h[d] = (float)z;
        l[d] = (float)(z - (double)h[d]);
    }
    zhi[k] = make_float4(h[0], h[1], h[2], (float)hs[k]);
    zlo[k] = make_float4(l[0], l[1], l[2], 0.0f);
}

inline int blocks_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

TabF64 tab64(const DevTables& tb) { return TabF64{tb.w, tb.iw, tb.rec_a, tb.rec_b, tb.diag, tb.sub}; }

// Hat multipoles of the point dipoles D_i = m_i v_i of a leaf (the jerk's
// chi field): M_n^m = -sum_i D_i . grad Upsilon_n^m(x_i - z). With the ladder
// relations d_z U_n^m = U_{n-1}^m, (d_x + i d_y) U_n^m = -U_{n-1}^{m+1},
// (d_x - i d_y) U_n^m = U_{n-1}^{m-1}, this is
//   M_n^m = -[ Z_{n-1}^m + (X + iY)_{n-1}^{m-1} / 2 + (-X + iY)_{n-1}^{m+1} / 2 ]
// with X, Y, Z the order p-1 moments of the weights D_x, D_y, D_z. In the hat
// basis (Xhat = X w / s^n) the degree ratios become
// w_n^m / w_{n-1}^{m'} = sqrt((n+m)(n-m)), sqrt((n+m)(n+m-1)), sqrt((n-m)(n-m-1))
// for m' = m, m-1, m+1, and one factor 1/s. One thread per leaf.
__global__ void k_dipole_moments(TreeView t, int p, const double* __restrict__ X, const double* __restrict__ Y,
                                 const double* __restrict__ Z, const double* __restrict__ hs,
                                 double* __restrict__ mult) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *t.dnn || t.nchild[k] != 0) return;
    const int nr = ncoef_real(p), nq = ncoef_real(p - 1);
    const double* x = X + (size_t)nq * k;
    const double* y = Y + (size_t)nq * k;
    const double* z = Z + (size_t)nq * k;
    const double is = 1.0 / hs[k];
    double* out = mult + (size_t)nr * k;
    out[0] = 0.0;  // a dipole has no monopole
    for (int n = 1; n <= p; ++n) {
        for (int m = 0; m <= n; ++m) {
            double re = 0.0, im = 0.0;
            if (m <= n - 1) {  // Z_{n-1}^m
                const double c = sqrt((double)((n + m) * (n - m)));
                re += c * z[hre(n - 1, m)];
                im += c * (m ? z[him(n - 1, m)] : 0.0);
            }
            if (m >= 1 || n >= 2) {  // (X + iY)_{n-1}^{m-1} / 2
                const int ml = m - 1, am = ml < 0 ? -ml : ml;
                double xr = x[hre(n - 1, am)], xi = am ? x[him(n - 1, am)] : 0.0;
                double yr = y[hre(n - 1, am)], yi = am ? y[him(n - 1, am)] : 0.0;
                if (ml < 0) { xr = -xr; yr = -yr; }  // X^{-1} = -conj(X^1): (-re, +im)
                const double c = 0.5 * sqrt((double)((n + m) * (n + m - 1)));
                re += c * (xr - yi);
                im += c * (xi + yr);
            }
            if (m + 1 <= n - 1) {  // (-X + iY)_{n-1}^{m+1} / 2
                const double xr = x[hre(n - 1, m + 1)], xi = x[him(n - 1, m + 1)];
                const double yr = y[hre(n - 1, m + 1)], yi = y[him(n - 1, m + 1)];
                const double c = 0.5 * sqrt((double)((n - m) * (n - m - 1)));
                re += c * (-xr - yi);
                im += c * (-xi + yr);
            }
            out[hre(n, m)] = -re * is;
            if (m) out[him(n, m)] = -im * is;
        }
    }
}
}  // namespace

void upload_expansion_tables(const HostTables& h) {
    float w[kMaxPF32 + 2][kMaxPF32 + 2], iw[kMaxPF32 + 2][kMaxPF32 + 2];
    float a[kMaxPF32 + 1][kMaxPF32 + 1], b[kMaxPF32 + 1][kMaxPF32 + 1];
    float d[kMaxPF32 + 1], s[kMaxPF32 + 1];
    for (int n = 0; n < kMaxPF32 + 2; ++n)
        for (int m = 0; m < kMaxPF32 + 2; ++m) { w[n][m] = (float)h.w[n][m]; iw[n][m] = (float)h.iw[n][m]; }
    for (int n = 0; n <= kMaxPF32; ++n) {
        for (int m = 0; m <= kMaxPF32; ++m) { a[n][m] = (float)h.rec_a[n][m]; b[n][m] = (float)h.rec_b[n][m]; }
        d[n] = (float)h.diag[n];
        s[n] = (float)h.sub[n];
    }
    cudaMemcpyToSymbol(c_w32, w, sizeof(w));
    cudaMemcpyToSymbol(c_iw32, iw, sizeof(iw));
    cudaMemcpyToSymbol(c_rec_a32, a, sizeof(a));
    cudaMemcpyToSymbol(c_rec_b32, b, sizeof(b));
    cudaMemcpyToSymbol(c_diag32, d, sizeof(d));
    cudaMemcpyToSymbol(c_sub32, s, sizeof(s));
    // double words: hi = the float nearest x, lo = the float nearest x - hi
    static dw da[kMaxP + 1][kMaxP + 1], db[kMaxP + 1][kMaxP + 1], dd[kMaxP + 1], ds[kMaxP + 1];
    auto split = [](double x) { const float hi = (float)x; return dw{hi, (float)(x - (double)hi)}; };
    for (int n = 0; n <= kMaxP; ++n) {
        for (int m = 0; m <= kMaxP; ++m) { da[n][m] = split(h.rec_a[n][m]); db[n][m] = split(h.rec_b[n][m]); }
        dd[n] = split(h.diag[n]);
        ds[n] = split(h.sub[n]);
    }
    cudaMemcpyToSymbol(c_dw_a, da, sizeof(da));
    cudaMemcpyToSymbol(c_dw_b, db, sizeof(db));
    cudaMemcpyToSymbol(c_dw_d, dd, sizeof(dd));
    cudaMemcpyToSymbol(c_dw_s, ds, sizeof(ds));
}

void upward_pass(const TreeView& t, const int* h_level_start, int p, const double* xs,
                 const double* ys, const double* zs, const double* ms, const double* zc,
                 const double* r, const double* hs, const double* geo, double* mult, double* Pk, float* Phat,
                 float* r32, double* contrib, const DevTables& tbl, bool dword, cudaStream_t st) {
    const TabF64 tb = tab64(tbl);
    if (dword && p <= 16)
        launch_p2m_dw<16, 4>(t, p, xs, ys, zs, ms, zc, hs, mult, st);
    else if (dword)
        launch_p2m_dw<kMaxP, 2>(t, p, xs, ys, zs, ms, zc, hs, mult, st);
    else if (p <= 16)
        (k_p2m<16, 4><<<device_sm_count() * 8, 128, 0, st>>>(t, p, tb, xs, ys, zs, ms, zc, hs, mult), note_launch());
    else
        (k_p2m<kMaxP, 2><<<device_sm_count() * 16, 64, 0, st>>>(t, p, tb, xs, ys, zs, ms, zc, hs, mult), note_launch());
    const int nr = ncoef_real(p);
    (void)nr;
    (void)h_level_start;
    for (int L = t.nlevels - 2; L >= 0; --L) m2m_level(t, L, p, geo, mult, contrib, tbl, dword, st);
    (k_pnorm<<<blocks_for(t.nnodes, 128), 128, 0, st>>>(t.dnn, p, mult, r, hs, Pk, Phat, r32), note_launch());
}

void p2m_weights(const TreeView& t, int p, const double* xs, const double* ys, const double* zs, const double* w,
                 const double* zc, const double* hs, double* mult, const DevTables& tbl, bool dword, cudaStream_t st) {
    const TabF64 tb = tab64(tbl);
    if (dword && p <= 16)
        launch_p2m_dw<16, 4>(t, p, xs, ys, zs, w, zc, hs, mult, st);
    else if (dword)
        launch_p2m_dw<kMaxP, 2>(t, p, xs, ys, zs, w, zc, hs, mult, st);
    else if (p <= 16)
        (k_p2m<16, 4><<<device_sm_count() * 8, 128, 0, st>>>(t, p, tb, xs, ys, zs, w, zc, hs, mult), note_launch());
    else
        (k_p2m<kMaxP, 2><<<device_sm_count() * 16, 64, 0, st>>>(t, p, tb, xs, ys, zs, w, zc, hs, mult), note_launch());
}

void dipole_moments(const TreeView& t, int p, const double* X, const double* Y, const double* Z, const double* hs,
                    double* mult, cudaStream_t st) {
    (k_dipole_moments<<<blocks_for(t.nnodes, 128), 128, 0, st>>>(t, p, X, Y, Z, hs, mult), note_launch());
}

void hat_scales(const TreeView& t, const int* parent, const double* r, double* hs, cudaStream_t st) {
    (k_hat_scales<<<blocks_for(t.nnodes, 128), 128, 0, st>>>(t.dnn, parent, r, hs), note_launch());
}

void node_centres_f32(const TreeView& t, const double* zc, const double* hs, float4* zhi, float4* zlo,
                      cudaStream_t st) {
    (k_node_centres<<<blocks_for(t.nnodes, 128), 128, 0, st>>>(t.dnn, zc, hs, zhi, zlo), note_launch());
}

__global__ void k_to_f32_strided(const double* __restrict__ a, float* __restrict__ b, const int* __restrict__ dnn,
                                 int nr, int stride) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)*dnn * stride) return;
    const int64_t k = q / stride;
    const int j = (int)(q - k * stride);
    b[q] = j < nr ? (float)a[k * nr + j] : 0.0f;
}

void multipoles_to_f32_padded(const double* mult, float* mult32, const TreeView& t, int nr, int stride,
                              cudaStream_t st) {
    const int64_t n = (int64_t)t.nnodes * stride;
    if (n > 0) (k_to_f32_strided<<<(int)((n + 255) / 256), 256, 0, st>>>(mult, mult32, t.dnn, nr, stride), note_launch());
}

void multipoles_to_f32(const double* mult, float* mult32, const TreeView& t, int nr, cudaStream_t st) {
    const int64_t count = (int64_t)t.nnodes * nr;
    if (count > 0) (k_to_f32<<<blocks_for(count, 256), 256, 0, st>>>(mult, mult32, t.dnn, nr), note_launch());
}

// L2L level by level: the rotation form (translate.cu) unless GBFMM_L2L_DIRECT
// selects the direct O(p^4) kernel above.
#ifndef GBFMM_L2L_DIRECT
#define GBFMM_L2L_DIRECT 0
#endif

void downward_pass_f64(const TreeView& t, const int* h_level_start, int p, const double* zc,
                       const double* hs, const double* geo, double* loc, const DevTables& tbl, cudaStream_t st) {
    const TabF64 tb = tab64(tbl);
    const int nc = tri(p + 1, 0), nr = ncoef_real(p);
    const size_t sh = (size_t)(2 * nc + nr + p + 1) * sizeof(double);
    if (GBFMM_L2L_DIRECT) ensure_dyn_smem((const void*)k_l2l<double, TabF64>, 100 * 1024);
    (void)h_level_start;
    for (int L = 1; L < t.nlevels; ++L) {
        if (t.lvl_cnt[L] <= 0) continue;
        if (GBFMM_L2L_DIRECT) (k_l2l<double, TabF64><<<t.lvl_cnt[L], 64, sh, st>>>(t, L, p, tb, zc, hs, loc), note_launch());
        else l2l_level(t, L, p, geo, loc, tbl, false, st);
    }
}

void downward_pass_f32(const TreeView& t, const int* h_level_start, int p, const double* zc,
                       const double* hs, const double* geo, float* loc, const DevTables& tbl, cudaStream_t st) {
    const int nc = tri(p + 1, 0), nr = ncoef_real(p);
    const size_t sh = (size_t)(2 * nc + nr + p + 1) * sizeof(float);
    (void)h_level_start;
    for (int L = 1; L < t.nlevels; ++L) {
        if (t.lvl_cnt[L] <= 0) continue;
        if (GBFMM_L2L_DIRECT) (k_l2l<float, TabF32><<<t.lvl_cnt[L], 64, sh, st>>>(t, L, p, TabF32{}, zc, hs, loc), note_launch());
        else l2l_level(t, L, p, geo, loc, tbl, true, st);
    }
}

}  // namespace gbfmm
