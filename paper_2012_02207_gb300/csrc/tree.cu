// Bounding cube, Morton keys, octree and cell geometry.
//
// Compiled with -fmad=false: every floating-point operation here is one IEEE
// operation in program order (no fused multiply-add), so the centres, sizes
// and keys are exactly those of a plain sequential evaluation of the same
// formulas.
//
// Octree (Fig. 1, Sec. 2.1): a node is split while it holds
// more than leaf_size bodies and is above level 21; empty children are
// omitted; nodes are numbered level by level, in key order inside a level.
// The build needs no per-level loop: with lcp_i the number of leading 3-bit
// digits shared by keys i-1 and i, and D_i the deepest level at which some
// window of leaf_size+1 consecutive keys containing i shares its prefix, a
// node of level L starts at body i exactly when lcp_i < L <= min(D_i+1, 21)
// (the root at i = 0, L = 0). Counting those starts per chunk of bodies and
// scanning the (level, chunk) table gives every node its index directly.
//
// Several independent clusters (an ensemble) are built as one forest: each
// cluster gets its own cube and keys, the bodies are sorted by (cluster, key),
// and lcp_i = -1 where a cluster begins, so every cluster has its own root at
// level 0 and no node spans two clusters. Nodes stay level-major, then
// (cluster, key) inside a level; a one-cluster forest is the plain octree.
#include "gbfmm_internal.cuh"

namespace gbfmm {

namespace {
constexpr int kChunk = 256;  // bodies per thread in the node enumeration
constexpr int kBboxBlocks = 304;  // bounding-cube partials (2 blocks per SM)

// block (c, s) of a grid of nclusters * slices blocks reduces slice s of cluster c
__global__ void k_bbox_partial(const double* __restrict__ x, const double* __restrict__ y,
                               const double* __restrict__ z, const double* __restrict__ m,
                               const int* __restrict__ coff, int slices, double* __restrict__ part,
                               unsigned* err) {
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    const int c = blockIdx.x / slices, sl = blockIdx.x - c * slices;
    const int64_t b = coff[c], e = coff[c + 1];
    for (int64_t i = b + (int64_t)sl * blockDim.x + threadIdx.x; i < e; i += (int64_t)slices * blockDim.x) {
        const double v[3] = {x[i], y[i], z[i]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (!isfinite(v[d])) bad = true;
            mn[d] = fmin(mn[d], v[d]);
            mx[d] = fmax(mx[d], v[d]);
        }
        const double mi = m[i];
        if (!(mi > 0.0) || !isfinite(mi)) bad = true;
    }
    __shared__ double s[6][256];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        s[d][threadIdx.x] = mn[d];
        s[3 + d][threadIdx.x] = mx[d];
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                s[d][threadIdx.x] = fmin(s[d][threadIdx.x], s[d][threadIdx.x + w]);
                s[3 + d][threadIdx.x] = fmax(s[3 + d][threadIdx.x], s[3 + d][threadIdx.x + w]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[6 * blockIdx.x + threadIdx.x] = s[threadIdx.x][0];
    if (bad) atomicOr(err, kErrNonfinite);
}

// Cube of each cluster: centre c = (min+max)/2 per axis,
// half-size h = the largest (max-min)/2 (h = 1 if all its bodies coincide,
// e.g. one body). box[8c ..]: cx, cy, cz, h, lox, loy, loz, size.
__global__ void k_bbox_final(const double* __restrict__ part, int nclusters, int slices,
                             double* __restrict__ box) {
    // one warp per cluster; min and max are exact, so the order does not matter
    const int c = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (c >= nclusters) return;
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = c * slices + lane; b < (c + 1) * slices; b += 32)
        for (int d = 0; d < 3; ++d) {
            mn[d] = fmin(mn[d], part[6 * b + d]);
            mx[d] = fmax(mx[d], part[6 * b + 3 + d]);
        }
    for (int o = 16; o > 0; o >>= 1)
        for (int d = 0; d < 3; ++d) {
            mn[d] = fmin(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmax(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
    if (lane != 0) return;
    double* bx = box + 8 * c;
    double h = 0.0;
    for (int d = 0; d < 3; ++d) {
        bx[d] = 0.5 * (mn[d] + mx[d]);
        const double hd = 0.5 * (mx[d] - mn[d]);
        if (hd > h) h = hd;
    }
    if (h == 0.0) h = 1.0;
    bx[3] = h;
    for (int d = 0; d < 3; ++d) bx[4 + d] = bx[d] - h;
    bx[7] = 2.0 * h;
}

// cluster of body i (coff: nclusters + 1 ascending offsets)
__device__ __forceinline__ int cluster_of(const int* __restrict__ coff, int nclusters, int64_t i) {
    int lo = 0, hi = nclusters;  // last c with coff[c] <= i
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (coff[mid] <= i) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint64_t spread3(uint64_t v) {  // 21 bits -> every third bit
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__device__ __forceinline__ uint64_t quantise(double v, double lo, double size) {
    const double t = (v - lo) / size;
    double f = floor(t * 2097152.0);
    f = f < 0.0 ? 0.0 : (f > 2097151.0 ? 2097151.0 : f);
    return (uint64_t)f;
}

// Morton key: x in the high bit of each 3-bit digit, then y, then z.
__global__ void k_keys(const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, int64_t n, const int* __restrict__ coff,
                       int nclusters, const double* __restrict__ box, uint64_t* __restrict__ keys,
                       uint32_t* __restrict__ idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* bx = box + 8 * cluster_of(coff, nclusters, i);
    const double size = bx[7];
    const uint64_t qx = quantise(x[i], bx[4], size);
    const uint64_t qy = quantise(y[i], bx[5], size);
    const uint64_t qz = quantise(z[i], bx[6], size);
    keys[i] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    idx[i] = (uint32_t)i;
}

// cluster pass of the (cluster, key) sort: the cluster of each key-sorted
// body as the sort key, its key-sorted position as the value
__global__ void k_cluster_keys(const uint32_t* __restrict__ perm, int64_t n, const int* __restrict__ coff,
                               int nclusters, uint64_t* __restrict__ ckey, uint32_t* __restrict__ cval) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ckey[i] = (uint64_t)cluster_of(coff, nclusters, perm[i]);
    cval[i] = (uint32_t)i;
}

__global__ void k_cluster_apply(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ perm,
                                const uint64_t* __restrict__ ckey, const uint32_t* __restrict__ cval,
                                int64_t n, uint64_t* __restrict__ keys_out, uint32_t* __restrict__ perm_out,
                                uint32_t* __restrict__ cid) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = cval[i];
    keys_out[i] = keys[j];
    perm_out[i] = perm[j];
    cid[i] = (uint32_t)ckey[i];
}

__global__ void k_gather(const double* __restrict__ x, const double* __restrict__ y,
                         const double* __restrict__ z, const double* __restrict__ m,
                         const uint32_t* __restrict__ perm, int64_t n, const uint32_t* __restrict__ cid,
                         const double* __restrict__ box, double* __restrict__ xs,
                         double* __restrict__ ys, double* __restrict__ zs, double* __restrict__ ms,
                         float4* __restrict__ xf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = perm[i];
    const double* bx = box + 8 * (cid ? cid[i] : 0u);
    const double a = x[j], b = y[j], c = z[j], w = m[j];
    xs[i] = a; ys[i] = b; zs[i] = c; ms[i] = w;
    xf[i] = make_float4((float)(a - bx[0]), (float)(b - bx[1]), (float)(c - bx[2]), (float)w);
}

// lcp_i (levels shared by keys i-1 and i; -1 where a cluster begins) and
// the coincident-body check (within a cluster).
constexpr int kRunScan = 4096;
__global__ void k_lcp(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ cid,
                      const double* __restrict__ xs, const double* __restrict__ ys,
                      const double* __restrict__ zs, int64_t n, int8_t* __restrict__ lcp, unsigned* err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t ci = cid ? cid[i] : 0u;
    if (i == 0 || (cid && cid[i - 1] != ci)) { lcp[i] = -1; return; }
    const uint64_t k = keys[i];
    const uint64_t d = k ^ keys[i - 1];
    lcp[i] = d ? (int8_t)((__clzll((long long)d) - 1) / 3) : (int8_t)kMaxLevel;
    if (d == 0) {
        // equal keys: compare with the earlier bodies of the run, at most
        // kRunScan back; a longer run is flagged for coincident_exact
        const double a = xs[i], b = ys[i], c = zs[i];
        int steps = 0;
        int64_t j = i - 1;
        for (; j >= 0 && keys[j] == k && (!cid || cid[j] == ci) && steps < kRunScan; --j, ++steps)
            if (xs[j] == a && ys[j] == b && zs[j] == c) { atomicOr(err, kErrCoincident); return; }
        if (steps == kRunScan && j >= 0 && keys[j] == k && (!cid || cid[j] == ci)) atomicOr(err, kErrLongRun);
    }
}

// 64-bit mix of a body's cluster and position (-0.0 counted as +0.0, so
// bodies equal under == hash alike): the finaliser of SplitMix64 over the
// combined words
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
__global__ void k_pos_hash(const double* __restrict__ xs, const double* __restrict__ ys,
                           const double* __restrict__ zs, const uint32_t* __restrict__ cid, int64_t n,
                           uint64_t* __restrict__ h, uint32_t* __restrict__ idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t z = mix64((uint64_t)__double_as_longlong(xs[i] + 0.0) ^ 0x9e3779b97f4a7c15ull);
    z = mix64(z ^ (uint64_t)__double_as_longlong(ys[i] + 0.0));
    z = mix64(z ^ (uint64_t)__double_as_longlong(zs[i] + 0.0));
    h[i] = mix64(z ^ (uint64_t)(cid ? cid[i] : 0u));
    idx[i] = (uint32_t)i;
}
// bodies with equal hashes: compare positions and clusters exactly, each
// with the earlier bodies of its hash run (a run of distinct positions
// needs a 64-bit hash collision)
__global__ void k_pos_equal(const uint64_t* __restrict__ h, const uint32_t* __restrict__ idx,
                            const double* __restrict__ xs, const double* __restrict__ ys,
                            const double* __restrict__ zs, const uint32_t* __restrict__ cid, int64_t n,
                            unsigned* err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || i == 0 || h[i] != h[i - 1]) return;
    const uint32_t bi = idx[i];
    for (int64_t j = i - 1; j >= 0 && h[j] == h[i]; --j) {
        const uint32_t bj = idx[j];
        if (xs[bi] == xs[bj] && ys[bi] == ys[bj] && zs[bi] == zs[bj] && (!cid || cid[bi] == cid[bj])) {
            atomicOr(err, kErrCoincident);
            return;
        }
    }
}

// W_a = min(lcp[a+1 .. a+leaf]) for a in [0, n-1-leaf].
// (a window that crosses into another cluster has W_a = -1)
__global__ void k_window_min(const int8_t* __restrict__ lcp, int64_t n, int leaf,
                             int8_t* __restrict__ win) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a > n - 1 - leaf) return;
    int8_t w = kMaxLevel;
    for (int k = 1; k <= leaf; ++k) { const int8_t v = lcp[a + k]; w = v < w ? v : w; }
    win[a] = w;
}

// hi_i = min(D_i + 1, 21) with D_i the max of W over the windows holding i.
__global__ void k_window_max(const int8_t* __restrict__ win, int64_t n, int leaf,
                             uint8_t* __restrict__ hi) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (n <= leaf) { hi[i] = 0; return; }
    const int64_t a0 = i - leaf > 0 ? i - leaf : 0;
    const int64_t a1 = i < n - 1 - leaf ? i : n - 1 - leaf;
    int d = -1;
    for (int64_t a = a0; a <= a1; ++a) d = win[a] > d ? win[a] : d;
    hi[i] = (uint8_t)(d + 1 < kMaxLevel ? d + 1 : kMaxLevel);
}

__device__ __forceinline__ int start_lo(const int8_t* lcp, int64_t i) { return (int)lcp[i]; }

// per (level, chunk) node-start counts, level-major
__global__ void k_level_count(const int8_t* __restrict__ lcp, const uint8_t* __restrict__ hi,
                              int64_t n, int nchunks, uint32_t* __restrict__ cnt) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchunks) return;
    uint32_t local[kMaxLevel + 1];
#pragma unroll
    for (int L = 0; L <= kMaxLevel; ++L) local[L] = 0;
    const int64_t b = (int64_t)c * kChunk;
    const int64_t e = b + kChunk < n ? b + kChunk : n;
    for (int64_t i = b; i < e; ++i) {
        const int lo = start_lo(lcp, i), h = hi[i];
#pragma unroll
        for (int L = 0; L <= kMaxLevel; ++L) local[L] += (L > lo && L <= h) ? 1u : 0u;
    }
#pragma unroll
    for (int L = 0; L <= kMaxLevel; ++L) cnt[(int64_t)L * nchunks + c] = local[L];
}

__global__ void k_level_emit(const int8_t* __restrict__ lcp, const uint8_t* __restrict__ hi,
                             int64_t n, int nchunks, const uint32_t* __restrict__ off,
                             int* __restrict__ level, int* __restrict__ begin, int64_t node_cap,
                             unsigned* err) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchunks) return;
    uint32_t next[kMaxLevel + 1];
#pragma unroll
    for (int L = 0; L <= kMaxLevel; ++L) next[L] = off[(int64_t)L * nchunks + c];
    const int64_t b = (int64_t)c * kChunk;
    const int64_t e = b + kChunk < n ? b + kChunk : n;
    for (int64_t i = b; i < e; ++i) {
        const int lo = start_lo(lcp, i), h = hi[i];
#pragma unroll
        for (int L = 0; L <= kMaxLevel; ++L) {
            if (L > lo && L <= h) {
                const uint32_t k = next[L]++;
                if ((int64_t)k < node_cap) { level[k] = L; begin[k] = (int)i; }
                else atomicOr(err, kErrCapacity);
            }
        }
    }
}

// (more nodes than node_cap, the size of the node arrays, raise the capacity
// error and clamp the counts, so that no later kernel indexes past the arrays)
__global__ void k_level_starts(const uint32_t* __restrict__ off, int nchunks, const uint32_t* total,
                               int node_cap, DevScalars* ds) {
    const int L = threadIdx.x;
    const uint32_t cap = (uint32_t)node_cap;
    if (L <= kMaxLevel) {
        const uint32_t v = off[(int64_t)L * nchunks];
        ds->level_start[L] = (int)(v < cap ? v : cap);
    }
    if (L == 0) {
        const uint32_t tot = *total;
        ds->level_start[kMaxLevel + 1] = (int)(tot < cap ? tot : cap);
        ds->nnodes = (int)(tot < cap ? tot : cap);
        if (tot > cap) atomicOr(&ds->err, kErrCapacity);
    }
}

// end, parent and children of every node by binary searches.
__global__ void k_finalize(const uint64_t* __restrict__ keys, int64_t n, int leaf, int nnodes,
                           const uint32_t* __restrict__ cid, const int* __restrict__ coff,
                           const DevScalars* __restrict__ ds, const int* __restrict__ level,
                           const int* __restrict__ begin, int* __restrict__ end,
                           int* __restrict__ parent, int* __restrict__ first_child,
                           int* __restrict__ nchild) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ds->nnodes) return;
    const int L = level[k];
    const int b = begin[k];
    const int cend = cid ? coff[cid[b] + 1] : (int)n;  // end of the node's cluster
    int e = cend;
    if (L > 0) {
        const int shift = 3 * (kMaxLevel - L);
        const uint64_t pre = keys[b] >> shift;
        int lo = b + 1, hi = cend;  // first index with a larger prefix
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((keys[mid] >> shift) > pre) hi = mid; else lo = mid + 1;
        }
        e = lo;
        int plo = ds->level_start[L - 1], phi = ds->level_start[L];  // last parent begin <= b
        while (phi - plo > 1) {
            const int mid = (plo + phi) >> 1;
            if (begin[mid] <= b) plo = mid; else phi = mid;
        }
        parent[k] = plo;
    } else {
        parent[k] = -1;
    }
    end[k] = e;
    if (e - b > leaf && L < kMaxLevel) {
        const int c0 = ds->level_start[L + 1], c1 = ds->level_start[L + 2];
        int lo = c0, hi = c1;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (begin[mid] < b) lo = mid + 1; else hi = mid; }
        const int f = lo;
        hi = c1;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (begin[mid] < e) lo = mid + 1; else hi = mid; }
        first_child[k] = f;
        nchild[k] = lo - f;
    } else {
        first_child[k] = -1;
        nchild[k] = 0;
    }
}

// Leaf geometry: sums over the leaf's bodies in sorted order.
__global__ void k_geometry_leaves(TreeView t, const double* __restrict__ xs,
                                  const double* __restrict__ ys, const double* __restrict__ zs,
                                  const double* __restrict__ ms, double* __restrict__ M,
                                  double* __restrict__ S, double* __restrict__ zc,
                                  double* __restrict__ r) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *t.dnn || t.nchild[k] != 0) return;
    double Mk = 0.0, Sx = 0.0, Sy = 0.0, Sz = 0.0;
    const int b = t.begin[k], e = t.end[k];
    for (int i = b; i < e; ++i) {
        const double mi = ms[i];
        Mk = Mk + mi;
        Sx = Sx + mi * xs[i];
        Sy = Sy + mi * ys[i];
        Sz = Sz + mi * zs[i];
    }
    const double zx = Sx / Mk, zy = Sy / Mk, zz = Sz / Mk;
    // the largest distance: a correctly rounded square root is monotonic, so
    // the root of the largest squared distance equals the largest root (one
    // FP64 square root per leaf instead of one per body)
    double rr2 = 0.0;
    for (int i = b; i < e; ++i) {
        const double dx = xs[i] - zx, dy = ys[i] - zy, dz = zs[i] - zz;
        const double d2 = dx * dx + dy * dy + dz * dz;
        if (d2 > rr2) rr2 = d2;
    }
    const double rr = sqrt(rr2);
    M[k] = Mk;
    S[3 * k] = Sx; S[3 * k + 1] = Sy; S[3 * k + 2] = Sz;
    zc[3 * k] = zx; zc[3 * k + 1] = zy; zc[3 * k + 2] = zz;
    r[k] = rr;
}

// Internal geometry of one level: sums over children in order.
__global__ void k_geometry_internal(TreeView t, int L, double* __restrict__ M,
                                    double* __restrict__ S, double* __restrict__ zc,
                                    double* __restrict__ r) {
    const int k = t.dls[L] + blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= t.dls[L + 1] || t.nchild[k] == 0) return;
    const int c0 = t.first_child[k], c1 = c0 + t.nchild[k];
    double Mk = 0.0, Sx = 0.0, Sy = 0.0, Sz = 0.0;
    for (int c = c0; c < c1; ++c) {
        Mk = Mk + M[c];
        Sx = Sx + S[3 * c];
        Sy = Sy + S[3 * c + 1];
        Sz = Sz + S[3 * c + 2];
    }
    const double zx = Sx / Mk, zy = Sy / Mk, zz = Sz / Mk;
    double rr = 0.0;
    for (int c = c0; c < c1; ++c) {
        const double dx = zc[3 * c] - zx, dy = zc[3 * c + 1] - zy, dz = zc[3 * c + 2] - zz;
        const double d = sqrt(dx * dx + dy * dy + dz * dz) + r[c];
        if (d > rr) rr = d;
    }
    M[k] = Mk;
    S[3 * k] = Sx; S[3 * k + 1] = Sy; S[3 * k + 2] = Sz;
    zc[3 * k] = zx; zc[3 * k + 1] = zy; zc[3 * k + 2] = zz;
    r[k] = rr;
}

inline int blocks_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }
}  // namespace

int tree_nchunks(int64_t n) { return (int)((n + kChunk - 1) / kChunk); }

int bbox_partials(int nclusters) { return nclusters >= kBboxBlocks ? nclusters : 2 * kBboxBlocks; }

void tree_build_count(TreeBuffers& b, int* sorted_in_1, cudaStream_t st) {
    const int64_t n = b.n;
    const int nc = b.nclusters;
    const int slices = nc >= kBboxBlocks ? 1 : (kBboxBlocks + nc - 1) / nc;
    (k_bbox_partial<<<nc * slices, 256, 0, st>>>(b.x, b.y, b.z, b.m, b.coff, slices, b.bbox_part, &b.ds->err),
     note_launch());
    (k_bbox_final<<<blocks_for((int64_t)nc * 32, 128), 128, 0, st>>>(b.bbox_part, nc, slices, b.box), note_launch());
    (k_keys<<<blocks_for(n, 256), 256, 0, st>>>(b.x, b.y, b.z, n, b.coff, nc, b.box, b.k0, b.v0), note_launch());
    int in1 = radix_sort(b.k0, b.v0, b.k1, b.v1, n, 63, b.hist, st);
    const uint64_t* keys = in1 ? b.k1 : b.k0;
    const uint32_t* perm = in1 ? b.v1 : b.v0;
    const uint32_t* cid = nullptr;
    if (nc > 1) {
        // stable pass on the cluster: (cluster, key) order
        (k_cluster_keys<<<blocks_for(n, 256), 256, 0, st>>>(perm, n, b.coff, nc, b.ck0, b.cv0), note_launch());
        int bits = 0;
        while ((1 << bits) < nc) ++bits;
        const int cin1 = radix_sort(b.ck0, b.cv0, b.ck1, b.cv1, n, bits, b.hist, st);
        uint64_t* kout = in1 ? b.k0 : b.k1;
        uint32_t* vout = in1 ? b.v0 : b.v1;
        (k_cluster_apply<<<blocks_for(n, 256), 256, 0, st>>>(keys, perm, cin1 ? b.ck1 : b.ck0, cin1 ? b.cv1 : b.cv0,
                                                            n, kout, vout, b.cid), note_launch());
        in1 ^= 1;
        keys = kout;
        perm = vout;
        cid = b.cid;
    }
    *sorted_in_1 = in1;
    (k_gather<<<blocks_for(n, 256), 256, 0, st>>>(b.x, b.y, b.z, b.m, perm, n, cid, b.box, b.xs, b.ys, b.zs,
                                                 b.ms, b.xf), note_launch());
    (k_lcp<<<blocks_for(n, 256), 256, 0, st>>>(keys, cid, b.xs, b.ys, b.zs, n, b.lcp, &b.ds->err), note_launch());
    if (n > b.leaf_size)
        (k_window_min<<<blocks_for(n - b.leaf_size, 256), 256, 0, st>>>(b.lcp, n, b.leaf_size, b.win), note_launch());
    (k_window_max<<<blocks_for(n, 256), 256, 0, st>>>(b.win, n, b.leaf_size, b.hi), note_launch());
    const int nchunks = tree_nchunks(n);
    (k_level_count<<<blocks_for(nchunks, 128), 128, 0, st>>>(b.lcp, b.hi, n, nchunks, b.chunk_cnt), note_launch());
    const int64_t cells = (int64_t)(kMaxLevel + 1) * nchunks;
    scan_exclusive_u32(b.chunk_cnt, cells, b.chunk_cnt + cells, st);
}

void tree_build_emit(TreeBuffers& b, cudaStream_t st) {
    const int64_t n = b.n;
    const int nchunks = tree_nchunks(n);
    const int64_t cells = (int64_t)(kMaxLevel + 1) * nchunks;
    (k_level_emit<<<blocks_for(nchunks, 128), 128, 0, st>>>(b.lcp, b.hi, n, nchunks, b.chunk_cnt,
                                                           b.level, b.begin, b.node_cap, &b.ds->err), note_launch());
    (k_level_starts<<<1, 32, 0, st>>>(b.chunk_cnt, nchunks, b.chunk_cnt + cells, (int)b.node_cap, b.ds), note_launch());
}

void tree_build_phase2(TreeBuffers& b, const uint64_t* keys, int nnodes, const int* h_level_start,
                       int nlevels, cudaStream_t st) {
    (void)h_level_start;
    (void)nlevels;
    (k_finalize<<<blocks_for(nnodes, 128), 128, 0, st>>>(keys, b.n, b.leaf_size, nnodes,
                                                        b.nclusters > 1 ? b.cid : nullptr, b.coff, b.ds, b.level,
                                                        b.begin, b.end, b.parent, b.first_child,
                                                        b.nchild), note_launch());
}

void cell_geometry(const TreeView& t, const double* xs, const double* ys, const double* zs,
                   const double* ms, const int* h_level_start, double* M, double* S, double* zc,
                   double* r, cudaStream_t st) {
    (void)h_level_start;
    (k_geometry_leaves<<<blocks_for(t.nnodes, 128), 128, 0, st>>>(t, xs, ys, zs, ms, M, S, zc, r), note_launch());
    for (int L = t.nlevels - 2; L >= 0; --L)
        if (t.lvl_cnt[L] > 0)
            (k_geometry_internal<<<blocks_for(t.lvl_cnt[L], 128), 128, 0, st>>>(t, L, M, S, zc, r), note_launch());
}

void coincident_exact(const TreeBuffers& b, uint64_t* hk0, uint32_t* hv0, uint64_t* hk1, uint32_t* hv1,
                      cudaStream_t st) {
    const int64_t n = b.n;
    if (n < 2) return;
    const uint32_t* cid = b.nclusters > 1 ? b.cid : nullptr;
    (k_pos_hash<<<blocks_for(n, 256), 256, 0, st>>>(b.xs, b.ys, b.zs, cid, n, hk0, hv0), note_launch());
    const int in1 = radix_sort(hk0, hv0, hk1, hv1, n, 64, b.hist, st);
    (k_pos_equal<<<blocks_for(n, 256), 256, 0, st>>>(in1 ? hk1 : hk0, in1 ? hv1 : hv0, b.xs, b.ys, b.zs, cid, n,
                                                     &b.ds->err), note_launch());
}

}  // namespace gbfmm
