// Leaf evaluation: far field by L2P, near field by P2P (Sec. 2.1), plus the
// plain FP64 direct sum used to measure force errors (Sec. 3.1.1).
//
// One warp per target leaf; lane l owns target body l of each 32-body chunk
// of the leaf. The leaf's local expansion is evaluated at the body (L2P),
// then the sources of every leaf in the target's P2P list (sorted by index)
// are summed directly, all lanes reading the same source at a time. The
// result times G is written to the caller's order through the sort
// permutation.
//
// Mixed precision: bodies are stored relative to their own leaf centre in
// FP32; a source leaf A is moved into the target leaf B's frame by the
// FP32-rounded offset z_A - z_B (computed in FP64). Terms are FP32 (rsqrtf);
// each source leaf's partial sum is folded into an FP64 accumulator.
#include "gbfmm_internal.cuh"

namespace gbfmm {

namespace {

__constant__ float c_w32l[kMaxPF32 + 2][kMaxPF32 + 2];
__constant__ float c_iw32l[kMaxPF32 + 2][kMaxPF32 + 2];
__constant__ float c_rec_a32l[kMaxPF32 + 1][kMaxPF32 + 1];
__constant__ float c_rec_b32l[kMaxPF32 + 1][kMaxPF32 + 1];
__constant__ float c_diag32l[kMaxPF32 + 1];
__constant__ float c_sub32l[kMaxPF32 + 1];

struct TabL64 {
    const double *w, *iw, *rec_a, *rec_b, *diag, *sub;
    __device__ double W(int n, int m) const { return __ldg(w + n * (kMaxP + 2) + m); }
    __device__ double IW(int n, int m) const { return __ldg(iw + n * (kMaxP + 2) + m); }
    __device__ double A(int n, int m) const { return __ldg(rec_a + n * (kMaxP + 1) + m); }
    __device__ double B(int n, int m) const { return __ldg(rec_b + n * (kMaxP + 1) + m); }
    __device__ double D(int m) const { return __ldg(diag + m); }
    __device__ double Sb(int m) const { return __ldg(sub + m); }
};
struct TabL32 {
    __device__ float W(int n, int m) const { return c_w32l[n][m]; }
    __device__ float IW(int n, int m) const { return c_iw32l[n][m]; }
    __device__ float A(int n, int m) const { return c_rec_a32l[n][m]; }
    __device__ float B(int n, int m) const { return c_rec_b32l[n][m]; }
    __device__ float D(int m) const { return c_diag32l[m]; }
    __device__ float Sb(int m) const { return c_sub32l[m]; }
};

// L2P on a hat local expansion F at dhat = d / s (|dhat| <= 1):
//   phi = -sum_{n,m} conj(Shat_n^m(dhat)) Fhat_n^m
//   F_1^m(x) = (1/s) sum_{k,l} conj(Shat_k^l) w_{1+k}^{m+l}/w_k^l Fhat_{1+k}^{m+l}, m = 0, 1
//   a = (Re F_1^1, Im F_1^1, F_1^0)        (all without G)
template <typename T, typename Tab>
__device__ void l2p_hat(int p, const T* __restrict__ F, T x, T y, T z, T inv_s, const Tab& tb,
                        T& phi, T& ax, T& ay, T& az) {
    const T r2 = x * x + y * y + z * z;
    T pot = T(0), g0 = T(0), g1r = T(0), g1i = T(0);
    T dre = T(1), dim = T(0);  // Shat_l^l
    for (int l = 0; l <= p; ++l) {
        if (l > 0) {
            const T t = dre * x - dim * y;
            dim = dre * y + dim * x;
            dre = t;
            dre *= tb.D(l);
            dim *= tb.D(l);
        }
        T s1r = dre, s1i = dim, s2r = T(0), s2i = T(0);  // Shat_k^l, Shat_{k-1}^l
        for (int k = l; k <= p; ++k) {
            T sr, si;
            if (k == l) { sr = dre; si = dim; }
            else if (k == l + 1) { sr = tb.Sb(l) * z * s1r; si = tb.Sb(l) * z * s1i; }
            else {
                const T a = tb.A(k, l) * z, b = tb.B(k, l) * r2;
                sr = a * s1r - b * s2r;
                si = a * s1i - b * s2i;
            }
            if (k > l) { s2r = s1r; s2i = s1i; s1r = sr; s1i = si; }
            // potential: Re(conj(S) F) counted twice for l > 0
            const T fr = F[hre(k, l)], fi = l ? F[him(k, l)] : T(0);
            const T re = sr * fr + si * fi;
            pot += l ? T(2) * re : re;
            if (k < p) {
                const T iwkl = tb.IW(k, l);
                // F_1^0
                const T g0r = F[hre(k + 1, l)], g0i = l ? F[him(k + 1, l)] : T(0);
                const T c0 = tb.W(k + 1, l) * iwkl;
                const T re0 = sr * g0r + si * g0i;
                g0 += l ? T(2) * c0 * re0 : c0 * re0;
                // F_1^1, +l part: conj(S_k^l) alpha Fhat_{1+k}^{1+l}
                const T al = tb.W(k + 1, l + 1) * iwkl;
                const T hr = F[hre(k + 1, l + 1)], hi = F[him(k + 1, l + 1)];
                g1r += al * (sr * hr + si * hi);
                g1i += al * (sr * hi - si * hr);
                // -l part (l >= 1): -S_k^l gamma conj(Fhat_{1+k}^{l-1})
                if (l >= 1) {
                    const T ga = tb.W(k + 1, l - 1) * iwkl;
                    const T er = F[hre(k + 1, l - 1)], ei = (l - 1) ? F[him(k + 1, l - 1)] : T(0);
                    g1r -= ga * (sr * er + si * ei);
                    g1i -= ga * (si * er - sr * ei);
                }
            }
        }
    }
    phi = -pot;
    ax = g1r * inv_s;
    ay = g1i * inv_s;
    az = g0 * inv_s;
}

__global__ void __launch_bounds__(128) k_leaf_f32(LeafArgs a) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const uint64_t mask = (1ull << a.nb) - 1ull;
    const int nr = ncoef_real(a.p);
    const float* locs = reinterpret_cast<const float*>(a.loc);
    const TabL32 tb;
    for (int b = blockIdx.x * (blockDim.x >> 5) + wib; b < a.t.nnodes; b += nwarps) {
        if (a.t.nchild[b] != 0) continue;
        const int b0 = a.t.begin[b], b1 = a.t.end[b];
        const double zbx = a.zc[3 * b], zby = a.zc[3 * b + 1], zbz = a.zc[3 * b + 2];
        const float inv_s = (float)(1.0 / hat_scale(a.r[b]));
        const float* F = locs + (size_t)nr * b;
        const uint32_t q0 = a.p2p_off[b], q1 = a.p2p_off[b + 1];
        for (int t0 = b0; t0 < b1; t0 += 32) {
            const int i = t0 + lane;
            const bool act = i < b1;
            const float4 ti = act ? a.prel[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            float phi = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
            if (act) l2p_hat<float>(a.p, F, ti.x * inv_s, ti.y * inv_s, ti.z * inv_s, inv_s, tb, phi, fx, fy, fz);
            double sx = fx, sy = fy, sz = fz, sp = phi;
            for (uint32_t q = q0; q < q1; ++q) {
                const int src = (int)(a.p2p_keys[q] & mask);
                const float ox = (float)(a.zc[3 * src] - zbx), oy = (float)(a.zc[3 * src + 1] - zby),
                            oz = (float)(a.zc[3 * src + 2] - zbz);
                const int j0 = a.t.begin[src], j1 = a.t.end[src];
                float px = 0.f, py = 0.f, pz = 0.f, pp = 0.f;
                for (int j = j0; j < j1; ++j) {
                    const float4 s = a.prel[j];
                    const float dx = (s.x + ox) - ti.x, dy = (s.y + oy) - ti.y, dz = (s.z + oz) - ti.z;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    const float rinv = (r2 > 0.f) ? rsqrtf(r2) : 0.f;
                    const float mr = s.w * rinv;
                    const float mr3 = mr * rinv * rinv;
                    px += mr3 * dx;
                    py += mr3 * dy;
                    pz += mr3 * dz;
                    pp += mr;
                }
                sx += px; sy += py; sz += pz; sp -= pp;
            }
            if (act) {
                const uint32_t o = a.perm[i];
                a.ax[o] = a.G * sx;
                a.ay[o] = a.G * sy;
                a.az[o] = a.G * sz;
                if (a.pot) a.pot[o] = a.G * sp;
            }
        }
    }
}

__global__ void __launch_bounds__(64) k_leaf_f64(LeafArgs a) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const uint64_t mask = (1ull << a.nb) - 1ull;
    const int nr = ncoef_real(a.p);
    const double* locs = reinterpret_cast<const double*>(a.loc);
    const TabL64 tb{a.tb.w, a.tb.iw, a.tb.rec_a, a.tb.rec_b, a.tb.diag, a.tb.sub};
    for (int b = blockIdx.x * (blockDim.x >> 5) + wib; b < a.t.nnodes; b += nwarps) {
        if (a.t.nchild[b] != 0) continue;
        const int b0 = a.t.begin[b], b1 = a.t.end[b];
        const double zbx = a.zc[3 * b], zby = a.zc[3 * b + 1], zbz = a.zc[3 * b + 2];
        const double inv_s = 1.0 / hat_scale(a.r[b]);
        const double* F = locs + (size_t)nr * b;
        const uint32_t q0 = a.p2p_off[b], q1 = a.p2p_off[b + 1];
        for (int t0 = b0; t0 < b1; t0 += 32) {
            const int i = t0 + lane;
            const bool act = i < b1;
            const double xi = act ? a.xs[i] : 0.0, yi = act ? a.ys[i] : 0.0, zi = act ? a.zs[i] : 0.0;
            double phi = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
            if (act) l2p_hat<double>(a.p, F, (xi - zbx) * inv_s, (yi - zby) * inv_s, (zi - zbz) * inv_s, inv_s, tb, phi, sx, sy, sz);
            double sp = phi;
            for (uint32_t q = q0; q < q1; ++q) {
                const int src = (int)(a.p2p_keys[q] & mask);
                const int j0 = a.t.begin[src], j1 = a.t.end[src];
                for (int j = j0; j < j1; ++j) {
                    const double dx = a.xs[j] - xi, dy = a.ys[j] - yi, dz = a.zs[j] - zi;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 > 0.0) {
                        const double r = sqrt(r2);
                        const double mr = a.ms[j] / r;
                        const double mr3 = mr / r2;
                        sx += mr3 * dx;
                        sy += mr3 * dy;
                        sz += mr3 * dz;
                        sp -= mr;
                    }
                }
            }
            if (act) {
                const uint32_t o = a.perm[i];
                a.ax[o] = a.G * sx;
                a.ay[o] = a.G * sy;
                a.az[o] = a.G * sz;
                if (a.pot) a.pot[o] = a.G * sp;
            }
        }
    }
}

__global__ void k_leaf_relative(TreeView t, const double* __restrict__ xs, const double* __restrict__ ys,
                                const double* __restrict__ zs, const double* __restrict__ ms,
                                const double* __restrict__ zc, float4* __restrict__ prel) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= t.nnodes || t.nchild[k] != 0) return;
    const double cx = zc[3 * k], cy = zc[3 * k + 1], cz = zc[3 * k + 2];
    for (int i = t.begin[k]; i < t.end[k]; ++i)
        prel[i] = make_float4((float)(xs[i] - cx), (float)(ys[i] - cy), (float)(zs[i] - cz), (float)ms[i]);
}

// Direct FP64 sum, one thread per target, source tiles staged in shared memory.
__global__ void __launch_bounds__(256) k_direct(int64_t n, const double* __restrict__ x,
                                                const double* __restrict__ y,
                                                const double* __restrict__ z,
                                                const double* __restrict__ m, double G, int64_t ntgt,
                                                const int64_t* __restrict__ tgt, double* ax, double* ay,
                                                double* az, double* pot) {
    __shared__ double4 tile[256];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = t < ntgt;
    const int64_t i = act ? (tgt ? tgt[t] : t) : 0;
    const double xi = act ? x[i] : 0.0, yi = act ? y[i] : 0.0, zi = act ? z[i] : 0.0;
    double sx = 0.0, sy = 0.0, sz = 0.0, sp = 0.0;
    for (int64_t j0 = 0; j0 < n; j0 += 256) {
        const int64_t j = j0 + threadIdx.x;
        tile[threadIdx.x] = (j < n) ? make_double4(x[j], y[j], z[j], m[j]) : make_double4(0, 0, 0, 0);
        __syncthreads();
        const int cnt = (int)((n - j0) < 256 ? (n - j0) : 256);
        for (int k = 0; k < cnt; ++k) {
            if (j0 + k == i) continue;
            const double4 s = tile[k];
            const double dx = s.x - xi, dy = s.y - yi, dz = s.z - zi;
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double r = sqrt(r2);
            const double mr = s.w / r;
            const double mr3 = mr / r2;
            sx += mr3 * dx;
            sy += mr3 * dy;
            sz += mr3 * dz;
            sp += mr;
        }
        __syncthreads();
    }
    if (act) {
        ax[t] = G * sx;
        ay[t] = G * sy;
        az[t] = G * sz;
        if (pot) pot[t] = -G * sp;
    }
}

// directed body-body interactions of the P2P list (self pairs without i = j)
__global__ void k_count_p2p(const uint64_t* __restrict__ keys, int64_t nk, int nb,
                            const int* __restrict__ begin, const int* __restrict__ end,
                            unsigned long long* out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = 0;
    if (q < nk) {
        const int t = (int)(keys[q] >> nb), s = (int)(keys[q] & ((1ull << nb) - 1ull));
        const unsigned long long nt = (unsigned long long)(end[t] - begin[t]);
        const unsigned long long ns = (unsigned long long)(end[s] - begin[s]);
        c = nt * ns - (t == s ? nt : 0ull);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

inline int blocks_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }
}  // namespace

void count_p2p_interactions(const uint64_t* keys, int64_t nk, int nb, const int* begin, const int* end,
                            unsigned long long* out, cudaStream_t st) {
    if (nk > 0) (k_count_p2p<<<blocks_for(nk, 256), 256, 0, st>>>(keys, nk, nb, begin, end, out), note_launch());
}

void upload_leaf_tables(const HostTables& h) {
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
    cudaMemcpyToSymbol(c_w32l, w, sizeof(w));
    cudaMemcpyToSymbol(c_iw32l, iw, sizeof(iw));
    cudaMemcpyToSymbol(c_rec_a32l, a, sizeof(a));
    cudaMemcpyToSymbol(c_rec_b32l, b, sizeof(b));
    cudaMemcpyToSymbol(c_diag32l, d, sizeof(d));
    cudaMemcpyToSymbol(c_sub32l, s, sizeof(s));
}

void leaf_eval_f64(const LeafArgs& a, cudaStream_t st) { (k_leaf_f64<<<152 * 16, 64, 0, st>>>(a), note_launch()); }
void leaf_eval_f32(const LeafArgs& a, cudaStream_t st) { (k_leaf_f32<<<152 * 8, 128, 0, st>>>(a), note_launch()); }

void leaf_relative_f32(const TreeView& t, const double* xs, const double* ys, const double* zs,
                       const double* ms, const double* zc, float4* prel, cudaStream_t st) {
    (k_leaf_relative<<<blocks_for(t.nnodes, 128), 128, 0, st>>>(t, xs, ys, zs, ms, zc, prel), note_launch());
}

void direct_sum_f64(int64_t n, const double* x, const double* y, const double* z, const double* m,
                    double G, int64_t ntgt, const int64_t* tgt, double* ax, double* ay, double* az,
                    double* pot, cudaStream_t st) {
    if (ntgt > 0) (k_direct<<<blocks_for(ntgt, 256), 256, 0, st>>>(n, x, y, z, m, G, ntgt, tgt, ax, ay, az, pot), note_launch());
}

}  // namespace gbfmm
