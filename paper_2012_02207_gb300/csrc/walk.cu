// Dual-tree walks and the scalar-force estimate.
//
// Compiled with -fmad=false: the MAC and the estimate f are evaluated with
// one IEEE operation per source operation, in program order, so the
// decisions are a plain function of the cell data.
//
// The walk (Sec. 2.1) runs level-synchronously: each launch classifies
// every pair of the current frontier and appends the accepted pairs, the
// leaf pairs and the child pairs of the next frontier. The error-controlled
// walk appends in frontier order: blocks take tiles of kWalkTile pairs by
// ticket, and a tile's output offsets come from a block scan and a
// decoupled look-back over the earlier tiles' published totals, so its
// lists come out in one fixed order and are then sorted by target only
// (keeping the walk order within a target). The theta-walk appends with
// warp-aggregated atomics; its lists are sorted by (target, source), the
// order the scalar estimate sums in.
#include "gbfmm_internal.cuh"

namespace gbfmm {

namespace {

struct WalkCells {
    int nnodes;
    const int* nchild;
    const int* first_child;
    const double* zc;
    const double* r;
    const double* P;
    const float* fmin;
    const double* binom;  // C(p, k), k = 0..p
    int p;
    double eps;
    // FP32 screen: double-float centres (zhi.w = hat scale s), sizes, and the
    // scaled degree norms Phat_k = P_k / s^k
    const float4* zhi;
    const float4* zlo;
    const float* r32;
    const float* Phat;
    // Plummer softening (Appendix B): the MAC adds 1.5 M_A soft^2 / d_min^4,
    // d_min = r - r_A - r_B, the bound on what the Newtonian far field leaves
    // out; soft2 = 0 skips it
    const double* M;
    double soft2;
    float soft2f;
};

// Relative margins of the FP32 screen. Its error is below 1e-5 (positive
// terms only, at most ~3(p+2) roundings of 2^-24 each plus the inputs'
// rounding), so outside the margin the FP32 decision equals the FP64 one.
constexpr float kThetaMargin = 1e-5f * 4.0f;
constexpr float kMacMargin = 1e-4f;

// FP32 estimate of E_{A->B} M_A / r^2: pre/r^2 sum_k C(p,k) Phat_k x^k y^{p-k}
// with x = s_A / r and y = r_B / r (Horner over k ascending).
__device__ __forceinline__ float mac_lhs32(const WalkCells& c, int a, float ra, float rb, float sa,
                                           float r, const float* binom32) {
    const float sum = ra + rb;
    const float pre = (sum > 0.0f) ? 8.0f * fmaxf(ra, rb) / sum : 4.0f;
    const float ir = 1.0f / r;
    const float x = sa * ir, y = rb * ir;
    const float* Pa = c.Phat + (size_t)(c.p + 1) * a;
    float h = 0.0f, xk = 1.0f;
    for (int k = 0; k <= c.p; ++k) {
        h = h * y + binom32[k] * Pa[k] * xk;
        xk *= x;
    }
    return pre * h * ir * ir;
}

// E_{A->B} M_A / r^2 of Sec. 2.3, Horner over k ascending.
__device__ double mac_lhs(const WalkCells& c, int a, double ra, double rb, double r, double r2) {
    const double sum = ra + rb;
    const double pre = (sum > 0.0) ? 8.0 * (ra > rb ? ra : rb) / sum : 4.0;
    const double* Pa = c.P + (size_t)(c.p + 1) * a;
    double h = 0.0;
    for (int k = 0; k <= c.p; ++k) h = h * rb + c.binom[k] * Pa[k];
    double rp = 1.0;
    for (int k = 0; k < c.p; ++k) rp = rp * r;
    return pre * h / (rp * r2);
}

// Device-scope accesses of the look-back records that bypass L1 (a relaxed
// load; an acquire load would invalidate the SM's L1, which the walk's node
// gathers live in).
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long walk_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Look-back records: one 64-bit word per counter and tile holding the kind
// (bits 63-62; 1: the tile's own count, 2: its inclusive prefix), the step
// (bits 61-54) and the value (bits 53-0), so one load reads a consistent
// record. The records a walk used are cleared before the next walk
// (k_walk_clear), and the step field tells this step's records from the
// earlier steps' of the same walk. Waits are bounded: after kLookbackNs the
// block raises kErrTimeout and goes on with a zero prefix (the host then
// fails the solve), so no wait can hang.
constexpr unsigned long long kLookbackNs = 1000000000ull;
constexpr unsigned long long kKindAgg = 1ull, kKindIncl = 2ull;
constexpr unsigned long long kValueMask = (1ull << 54) - 1ull;
__device__ __forceinline__ unsigned long long walk_record(unsigned long long kind, int it, unsigned long long v) {
    return (kind << 62) | ((unsigned long long)(it & 0xff) << 54) | (v & kValueMask);
}

// Exclusive prefix of one counter over the tiles before `tile`, by one warp:
// lane l reads tile j - l, waiting until that tile has published for this
// step; the nearest tile with an inclusive prefix ends the walk back.
__device__ unsigned long long lookback(const unsigned long long* rec, int64_t tile, int it, unsigned* err,
                                       int stall) {
    const int lane = threadIdx.x & 31;
    // (stall: a step no record carries, so every wait runs out)
    const unsigned long long step_bits = (unsigned long long)((stall ? it + 0x80 : it) & 0xff);
    unsigned long long excl = 0;
    const unsigned long long t0 = walk_ns();
    for (int64_t j = tile - 1;; j -= 32) {
        const int64_t idx = j - lane;
        unsigned long long kind = kKindIncl, v = 0;
        bool late = false;
        if (idx >= 0) {
            unsigned long long w = ld_relaxed(rec + idx);
            while ((w >> 62) == 0ull || ((w >> 54) & 0xffull) != step_bits) {
                // give up after kLookbackNs, or at once when some wait already ran out
                if (walk_ns() - t0 > kLookbackNs || (ld_relaxed_u32(err) & kErrTimeout)) {
                    late = true;
                    break;
                }
                w = ld_relaxed(rec + idx);
            }
            kind = late ? kKindIncl : (w >> 62);
            v = late ? 0ull : (w & kValueMask);
        }
        if (__any_sync(0xffffffffu, late)) {
            if (lane == 0) atomicOr(err, kErrTimeout);
        }
        const unsigned incl = __ballot_sync(0xffffffffu, kind == kKindIncl);
        const int first = incl ? __ffs(incl) - 1 : 32;
        unsigned long long c = lane <= first ? v : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        excl += c;
        if (incl) break;
    }
    return excl;
}

// inclusive scan of v over the warp
__device__ __forceinline__ unsigned warp_incl(unsigned v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Classify frontier pair q (of nin): accepted (n_acc = 1), a leaf pair
// (n_leaf = 1), or split into n_next child pairs (split_kind 1: the children
// pairs of a self pair, 2: split a, 3: split b). Pairs past nin count nothing.
template <int MODE>
__device__ __forceinline__ void classify_pair(const WalkCells& c, const int2* __restrict__ fin, int64_t nin,
                                              int64_t q, const float* binom32, float eps32, unsigned* err,
                                              int& a, int& b, int& split_kind, unsigned& n_next, unsigned& n_acc,
                                              unsigned& n_leaf) {
    a = 0;
    b = 0;
    n_next = n_acc = n_leaf = 0;
    split_kind = 0;
    const int2 pr = q < nin ? fin[q] : make_int2(0, 0);
    if (q < nin && ((unsigned)pr.x >= (unsigned)c.nnodes || (unsigned)pr.y >= (unsigned)c.nnodes)) {
        atomicOr(err, kErrIndex);  // never expected: a frontier entry that no step wrote
    } else if (q < nin) {
        a = pr.x;
        b = pr.y;
        const int nca = c.nchild[a], ncb = c.nchild[b];
        if (a == b) {
            if (nca == 0) n_leaf = 1;
            else { split_kind = 1; n_next = (unsigned)(nca * (nca + 1) / 2); }
        } else {
            // FP32 screen first
            const float4 ah = c.zhi[a], al = c.zlo[a], bh = c.zhi[b], bl = c.zlo[b];
            const float fx = (bh.x - ah.x) + (bl.x - al.x), fy = (bh.y - ah.y) + (bl.y - al.y),
                        fz = (bh.z - ah.z) + (bl.z - al.z);
            const float fr = sqrtf(fx * fx + fy * fy + fz * fz);
            const float fra = c.r32[a], frb = c.r32[b];
            int theta = 2;  // 0: fails, 1: passes, 2: undecided
            if (fra + frb < fr * (1.0f - kThetaMargin)) theta = 1;
            else if (fra + frb > fr * (1.0f + kThetaMargin)) theta = 0;
            bool accept;
            double r2 = 0.0, r = 0.0;
            bool have64 = false;
            if (theta == 2) {
                // theta = (r_A + r_B)/r < 1 in FP64
                const double* za = c.zc + 3 * a;
                const double* zb = c.zc + 3 * b;
                const double dx = zb[0] - za[0], dy = zb[1] - za[1], dz = zb[2] - za[2];
                r2 = dx * dx + dy * dy + dz * dz;
                r = sqrt(r2);
                have64 = true;
                accept = c.r[a] + c.r[b] < r;
            } else {
                accept = theta == 1;
            }
            if (MODE == 1 && accept) {
                float lab32 = mac_lhs32(c, a, fra, frb, ah.w, fr, binom32);
                float lba32 = mac_lhs32(c, b, frb, fra, bh.w, fr, binom32);
                const float rb32 = eps32 * c.fmin[b], ra32 = eps32 * c.fmin[a];
                // softening term in FP32 only well inside theta < 1, where
                // d_min = r - r_A - r_B > r/4 keeps its relative error near 1e-5
                bool screen = true;
                if (c.soft2 > 0.0) {
                    const float dmin32 = fr - fra - frb;
                    if (dmin32 > 0.25f * fr) {
                        const float d2 = dmin32 * dmin32;
                        const float d4 = d2 * d2;
                        lab32 = lab32 + 1.5f * (float)c.M[a] * c.soft2f / d4;
                        lba32 = lba32 + 1.5f * (float)c.M[b] * c.soft2f / d4;
                    } else {
                        screen = false;
                    }
                }
                if (screen && lab32 < rb32 * (1.0f - kMacMargin) && lba32 < ra32 * (1.0f - kMacMargin)) {
                    accept = true;
                } else if (screen && (lab32 > rb32 * (1.0f + kMacMargin) || lba32 > ra32 * (1.0f + kMacMargin))) {
                    accept = false;
                } else {
                    if (!have64) {
                        const double* za = c.zc + 3 * a;
                        const double* zb = c.zc + 3 * b;
                        const double dx = zb[0] - za[0], dy = zb[1] - za[1], dz = zb[2] - za[2];
                        r2 = dx * dx + dy * dy + dz * dz;
                        r = sqrt(r2);
                    }
                    const double ra = c.r[a], rb = c.r[b];
                    double lab = mac_lhs(c, a, ra, rb, r, r2);
                    double lba = mac_lhs(c, b, rb, ra, r, r2);
                    if (c.soft2 > 0.0) {
                        const double dab = r - ra - rb, dba = r - rb - ra;
                        const double qab = dab * dab, qba = dba * dba;
                        lab = lab + 1.5 * c.M[a] * c.soft2 / (qab * qab);
                        lba = lba + 1.5 * c.M[b] * c.soft2 / (qba * qba);
                    }
                    accept = lab < c.eps * (double)c.fmin[b] && lba < c.eps * (double)c.fmin[a];
                }
            }
            const double ra = c.r[a], rb = c.r[b];
            if (accept) n_acc = 1;
            else if (nca == 0 && ncb == 0) n_leaf = 1;
            else {
                const bool split_a = (ncb == 0) ? true : ((nca == 0) ? false : (ra >= rb));
                split_kind = split_a ? 2 : 3;
                n_next = (unsigned)(split_a ? nca : ncb);
            }
        }
    }
}

// the child pairs of a split pair, from fout[o] on
__device__ __forceinline__ void emit_children(const WalkCells& c, int2* __restrict__ fout, unsigned long long o,
                                              int split_kind, int a, int b) {
    if (split_kind == 1) {
        const int c0 = c.first_child[a], nc = c.nchild[a];
        for (int i = 0; i < nc; ++i)
            for (int j = i; j < nc; ++j) fout[o++] = make_int2(c0 + i, c0 + j);
    } else if (split_kind == 2) {
        const int c0 = c.first_child[a], nc = c.nchild[a];
        for (int i = 0; i < nc; ++i) fout[o++] = make_int2(c0 + i, b);
    } else {
        const int c0 = c.first_child[b], nc = c.nchild[b];
        for (int i = 0; i < nc; ++i) fout[o++] = make_int2(a, c0 + i);
    }
}

// Append cnt items per lane to a list; returns the lane's first slot. All
// 32 lanes of the warp must call it.
__device__ __forceinline__ unsigned long long warp_alloc(unsigned long long* counter, unsigned cnt) {
    const int lane = threadIdx.x & 31;
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + (incl - cnt);
}

// One step of the theta-walk (mode 0), appending with warp-aggregated
// atomics: its lists are sorted by (target, source) afterwards, so the order
// of the appends does not matter, and the atomics cost less than the
// ordered appends' look-back.
__global__ void __launch_bounds__(256) k_walk_step_any_order(WalkCells c, const int2* __restrict__ fin,
                                                             const unsigned long long* cnt_in,
                                                             int2* __restrict__ fout,
                                                             unsigned long long* cnt_out, int64_t cap_out,
                                                             int2* __restrict__ acc_list,
                                                             unsigned long long* cnt_acc, int64_t cap_acc,
                                                             int2* __restrict__ leaf_list,
                                                             unsigned long long* cnt_leaf, int64_t cap_leaf,
                                                             unsigned* err) {
    __shared__ float binom32[kMaxP + 1];
    if (threadIdx.x <= (unsigned)c.p) binom32[threadIdx.x] = (float)c.binom[threadIdx.x];
    __syncthreads();
    const float eps32 = (float)c.eps;
    const int64_t nin = (int64_t)*cnt_in;
    if (nin > cap_out) {  // an incomplete input frontier: the host grows the buffers
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, kErrCapacity);
        return;
    }
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp0 * 32; base < nin; base += nwarps * 32) {
        int a, b, split_kind;
        unsigned n_next, n_acc, n_leaf;
        classify_pair<0>(c, fin, nin, base + lane, binom32, eps32, err, a, b, split_kind, n_next, n_acc, n_leaf);
        const unsigned long long so = warp_alloc(cnt_out, n_next);
        const unsigned long long sa = warp_alloc(cnt_acc, n_acc);
        const unsigned long long sl = warp_alloc(cnt_leaf, n_leaf);
        if (n_acc) {
            if ((int64_t)sa < cap_acc) acc_list[sa] = make_int2(a, b); else atomicOr(err, kErrCapacity);
        }
        if (n_leaf) {
            if ((int64_t)sl < cap_leaf) leaf_list[sl] = make_int2(a, b); else atomicOr(err, kErrCapacity);
        }
        if (n_next) {
            if ((int64_t)(so + n_next) > cap_out) atomicOr(err, kErrCapacity);
            else emit_children(c, fout, so, split_kind, a, b);
        }
    }
}

// One step of the walk: the pairs fin[0..*cnt_in) become the next frontier
// fout (count into *cnt_out), accepted pairs appended to acc_list from
// position acc_hist[it] and leaf pairs to leaf_list from leaf_hist[it], in
// frontier order; the list lengths after the step go to acc_hist[it + 1],
// leaf_hist[it + 1] and list_cnt. Counts keep counting past a capacity
// (kErrCapacity, nothing written out of bounds), so the host can grow the
// buffers to what was asked for.
template <int MODE>
__global__ void __launch_bounds__(kWalkThreads) k_walk_step(WalkCells c, int it, const int2* __restrict__ fin,
                                                         const unsigned long long* cnt_in,
                                                         int2* __restrict__ fout,
                                                         unsigned long long* cnt_out, int64_t cap_out,
                                                         int2* __restrict__ acc_list, int64_t cap_acc,
                                                         int2* __restrict__ leaf_list, int64_t cap_leaf,
                                                         DevScalars* ds, int list_acc, int list_leaf,
                                                         unsigned long long* scan, int64_t scan_tiles,
                                                         int stall, unsigned* err) {
    __shared__ float binom32[kMaxP + 1];
    __shared__ unsigned s_tile;
    __shared__ unsigned s_wsum[3][kWalkThreads / 32];
    __shared__ unsigned long long s_excl[3];
    if (threadIdx.x <= (unsigned)c.p) binom32[threadIdx.x] = (float)c.binom[threadIdx.x];
    const float eps32 = (float)c.eps;
    const int64_t nin = (int64_t)*cnt_in;
    // An input frontier that outgrew its buffer is incomplete (the pairs past
    // the end were never written): do no work, the host sees the capacity
    // error and grows the buffers.
    if (nin > cap_out) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, kErrCapacity);
        return;
    }
    const unsigned long long acc_base = ds->acc_hist[it], leaf_base = ds->leaf_hist[it];
    const int64_t ntiles = (nin + kWalkTile - 1) / kWalkTile;  // kWalkTile pairs per tile, kWalkIPT per thread
    if (ntiles > scan_tiles) {  // never expected: the records are sized by the frontier capacity
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, kErrCapacity);
        return;
    }
    if (ntiles == 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *cnt_out = 0ull;
            ds->acc_hist[it + 1] = acc_base;
            ds->leaf_hist[it + 1] = leaf_base;
        }
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(&ds->walk_tiles, (unsigned long long)ntiles);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        __syncthreads();  // binom32 ready; the previous tile's shared state consumed
        if (threadIdx.x == 0) s_tile = atomicAdd(&ds->ticket[it], 1u);
        __syncthreads();
        const int64_t tile = (int64_t)s_tile;
        if (tile >= ntiles) break;
        const int64_t q0 = tile * kWalkTile + (int64_t)kWalkIPT * threadIdx.x;
        int a[kWalkIPT], b[kWalkIPT], split_kind[kWalkIPT];
        unsigned n_next[kWalkIPT], n_acc[kWalkIPT], n_leaf[kWalkIPT];
#pragma unroll
        for (int k = 0; k < kWalkIPT; ++k)
            classify_pair<MODE>(c, fin, nin, q0 + k, binom32, eps32, err, a[k], b[k], split_kind[k], n_next[k],
                                n_acc[k], n_leaf[k]);
        // offsets inside the tile, the tile's totals, then its place among the tiles
        unsigned own[3] = {0u, 0u, 0u};
#pragma unroll
        for (int k = 0; k < kWalkIPT; ++k) {
            own[0] += n_next[k];
            own[1] += n_acc[k];
            own[2] += n_leaf[k];
        }
        unsigned incl[3], wpre[3] = {0u, 0u, 0u}, tot[3] = {0u, 0u, 0u};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            incl[k] = warp_incl(own[k]);
            if (lane == 31) s_wsum[k][warp] = incl[k];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 3; ++k)
            for (int w = 0; w < kWalkThreads / 32; ++w) {
                const unsigned v = s_wsum[k][w];
                wpre[k] += w < warp ? v : 0u;
                tot[k] += v;
            }
        if (warp < 3) {
            unsigned long long* rec = scan + (size_t)warp * scan_tiles;
            if (tile == 0) {
                if (lane == 0) {
                    st_relaxed(rec + tile, walk_record(kKindIncl, it, tot[warp]));
                    s_excl[warp] = 0ull;
                }
            } else {
                if (lane == 0) st_relaxed(rec + tile, walk_record(kKindAgg, it, tot[warp]));
                const unsigned long long ex = lookback(rec, tile, it, err, stall);
                if (lane == 0) {
                    st_relaxed(rec + tile, walk_record(kKindIncl, it, ex + tot[warp]));
                    s_excl[warp] = ex;
                }
            }
        }
        __syncthreads();
        if (tile == ntiles - 1 && threadIdx.x == 0) {
            const unsigned long long an = acc_base + s_excl[1] + tot[1], ln = leaf_base + s_excl[2] + tot[2];
            *cnt_out = s_excl[0] + tot[0];
            ds->acc_hist[it + 1] = an;
            ds->leaf_hist[it + 1] = ln;
            ds->list_cnt[list_acc] = an;
            ds->list_cnt[list_leaf] = ln;
        }
        unsigned long long so = s_excl[0] + (incl[0] - own[0]) + wpre[0];
        unsigned long long sa = acc_base + s_excl[1] + (incl[1] - own[1]) + wpre[1];
        unsigned long long sl = leaf_base + s_excl[2] + (incl[2] - own[2]) + wpre[2];
#pragma unroll
        for (int k = 0; k < kWalkIPT; ++k) {
            if (n_acc[k]) {
                if ((int64_t)sa < cap_acc) acc_list[sa] = make_int2(a[k], b[k]); else atomicOr(err, kErrCapacity);
                ++sa;
            }
            if (n_leaf[k]) {
                if ((int64_t)sl < cap_leaf) leaf_list[sl] = make_int2(a[k], b[k]); else atomicOr(err, kErrCapacity);
                ++sl;
            }
            if (n_next[k]) {
                if ((int64_t)(so + n_next[k]) > cap_out) {
                    atomicOr(err, kErrCapacity);
                } else {
                    unsigned long long o = so;
                    if (split_kind[k] == 1) {
                        const int c0 = c.first_child[a[k]], nc = c.nchild[a[k]];
                        for (int i = 0; i < nc; ++i)
                            for (int j = i; j < nc; ++j) fout[o++] = make_int2(c0 + i, c0 + j);
                    } else if (split_kind[k] == 2) {
                        const int c0 = c.first_child[a[k]], nc = c.nchild[a[k]];
                        for (int i = 0; i < nc; ++i) fout[o++] = make_int2(c0 + i, b[k]);
                    } else {
                        const int c0 = c.first_child[b[k]], nc = c.nchild[b[k]];
                        for (int i = 0; i < nc; ++i) fout[o++] = make_int2(a[k], c0 + i);
                    }
                }
                so += n_next[k];
            }
        }
    }
}

// clear the look-back records the previous walk used (walk_tiles tiles)
__global__ void k_walk_clear(DevScalars* ds, unsigned long long* scan, int64_t scan_tiles) {
    const unsigned long long used = ds->walk_tiles < (unsigned long long)scan_tiles ? ds->walk_tiles
                                                                                     : (unsigned long long)scan_tiles;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < used;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        scan[i] = 0ull;
        scan[scan_tiles + i] = 0ull;
        scan[2 * scan_tiles + i] = 0ull;
    }
}

// the walk starts from the self pair (root, root) of every tree of the forest
__global__ void k_walk_init(int2* f0, const int* __restrict__ dls, DevScalars* ds, int iters, int mode) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nroots = dls[1];  // the nodes of level 0
    if (i < nroots) f0[i] = make_int2(i, i);
    if (i < iters) {
        ds->cnt[i] = (i == 0) ? (unsigned long long)nroots : 0ull;
        ds->ticket[i] = 0u;
        ds->acc_hist[i] = 0ull;
        ds->leaf_hist[i] = 0ull;
    }
    if (i < 2) ds->list_cnt[2 * mode + i] = 0ull;
    if (i == 0) ds->walk_tiles = 0ull;
}

// directed keys target << nb | source
// (pairs past the device count *np, up to the grid's npcap, become two
// markers: a list read back by the host has npcap == *np)
__global__ void k_directed(const int2* __restrict__ pairs, const unsigned long long* __restrict__ np,
                           int64_t npcap, int nb, uint64_t* __restrict__ keys, unsigned long long* count,
                           unsigned long long* nkeys) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t npr = (int64_t)*np < npcap ? (int64_t)*np : npcap;
    if (q == 0) *nkeys = 2ull * (unsigned long long)npr;
    // two slots per pair; self pairs fill one and leave a marker that sorts last
    if (q >= npr) return;
    const int2 pr = pairs[q];
    const uint64_t a = (uint64_t)pr.x, b = (uint64_t)pr.y;
    keys[2 * q] = (b << nb) | a;
    keys[2 * q + 1] = (pr.x == pr.y) ? ~0ull : ((a << nb) | b);
    if (pr.x == pr.y) atomicAdd(count, 1ull);
}

// 32-bit form of k_directed (when 2 nb <= 32): marker 0xffffffff
__global__ void k_directed32(const int2* __restrict__ pairs, const unsigned long long* __restrict__ np,
                             int64_t npcap, int nb, uint32_t* __restrict__ keys, unsigned long long* count,
                             unsigned long long* nkeys) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t npr = (int64_t)*np < npcap ? (int64_t)*np : npcap;
    if (q == 0) *nkeys = 2ull * (unsigned long long)npr;
    if (q >= npr) return;
    const int2 pr = pairs[q];
    const uint32_t a = (uint32_t)pr.x, b = (uint32_t)pr.y;
    keys[2 * q] = (b << nb) | a;
    keys[2 * q + 1] = (pr.x == pr.y) ? 0xffffffffu : ((a << nb) | b);
    if (pr.x == pr.y) atomicAdd(count, 1ull);
}

// sorted 32-bit keys -> the source index of every entry (what the consumers
// read) and the CSR offsets per target
__global__ void k_offsets_src32(const uint32_t* __restrict__ k32, int64_t nk,
                                const unsigned long long* __restrict__ dnk, int nb, const int* __restrict__ dnn,
                                uint32_t* __restrict__ src, uint32_t* __restrict__ off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((int64_t)*dnk < nk) nk = (int64_t)*dnk;
    if (i > nk) return;
    const int nnodes = *dnn;
    const uint32_t k = i < nk ? k32[i] : 0xffffffffu;
    if (i < nk) src[i] = k == 0xffffffffu ? 0xffffffffu : (k & ((1u << nb) - 1u));
    int64_t t = (i < nk) ? (int64_t)(k >> nb) : (int64_t)nnodes;
    int64_t tp = (i > 0) ? (int64_t)(k32[i - 1] >> nb) : -1;
    t = t < nnodes ? t : nnodes;
    tp = tp < nnodes ? tp : nnodes;
    for (int64_t u = tp + 1; u <= t && u <= nnodes; ++u) off[u] = (uint32_t)i;
}

__global__ void k_offsets(const uint64_t* __restrict__ keys, int64_t nk, const unsigned long long* __restrict__ dnk,
                          int nb, const int* __restrict__ dnn, uint32_t* __restrict__ src, uint32_t* __restrict__ off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((int64_t)*dnk < nk) nk = (int64_t)*dnk;
    if (i > nk) return;
    const int nnodes = *dnn;
    if (i < nk) src[i] = keys[i] == ~0ull ? 0xffffffffu : (uint32_t)(keys[i] & ((1ull << nb) - 1ull));
    // marker keys (all ones, from self pairs) sort last and count as "past the end"
    int64_t t = (i < nk) ? (int64_t)(keys[i] >> nb) : (int64_t)nnodes;
    int64_t tp = (i > 0) ? (int64_t)(keys[i - 1] >> nb) : -1;
    t = t < nnodes ? t : nnodes;
    tp = tp < nnodes ? tp : nnodes;
    for (int64_t u = tp + 1; u <= t && u <= nnodes; ++u) off[u] = (uint32_t)i;
}

// far part of the estimate: per cell, M_A / r^2 summed over theta-partners in
// ascending order, r^2 from the FP32-rounded centre offsets. One warp per
// cell: the lanes form the terms of 32 partners at a time, then the terms are
// added one after the other in partner order (the same sequence of FP32
// additions as a single thread walking the list).
__global__ void k_far_f(const int* __restrict__ dnn, const double* __restrict__ zc, const double* __restrict__ M,
                        const uint32_t* __restrict__ src, const uint32_t* __restrict__ off,
                        float* __restrict__ farf) {
    const int b = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= *dnn) return;
    const double bx = zc[3 * b], by = zc[3 * b + 1], bz = zc[3 * b + 2];
    float acc = 0.0f;
    const uint32_t q0 = off[b], q1 = off[b + 1];
    for (uint32_t qb = q0; qb < q1; qb += 32) {
        const uint32_t q = qb + lane;
        float term = 0.0f;
        if (q < q1) {
            const int a = (int)src[q];
            const float dx = (float)(zc[3 * a] - bx), dy = (float)(zc[3 * a + 1] - by),
                        dz = (float)(zc[3 * a + 2] - bz);
            const float r2 = dx * dx + dy * dy + dz * dz;
            term = (float)M[a] / r2;
        }
        const int cnt = q1 - qb < 32u ? (int)(q1 - qb) : 32;
        for (int k = 0; k < cnt; ++k) acc = acc + __shfl_sync(0xffffffffu, term, k);
    }
    if (lane == 0) farf[b] = acc;
}

// g(k) = g(parent) + far(k), accumulated from the root down the ancestor chain
__global__ void k_push_down(TreeView t, const float* __restrict__ farf, float* __restrict__ g) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *t.dnn) return;
    int chain[kMaxLevel + 1];
    int len = 0;
    for (int a = k; a >= 0; a = t.parent[a]) chain[len++] = a;
    float acc = farf[chain[len - 1]];
    for (int i = len - 2; i >= 0; --i) acc = acc + farf[chain[i]];
    g[k] = acc;
}

// near part per body: partner leaves ascending, their bodies in order, j != i
// (one thread per body; a warp's bodies share their leaf's partners, so most
// loads are broadcasts)
__global__ void k_near_f(TreeView t, const float4* __restrict__ xf, const uint32_t* __restrict__ src,
                         const uint32_t* __restrict__ off, const int* __restrict__ leaf_of,
                         const float* __restrict__ g, float soft2f, float* __restrict__ f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= t.n) return;
    const int b = leaf_of[i];
    const float4 pi = xf[i];
    float acc = 0.0f;
    for (uint32_t q = off[b]; q < off[b + 1]; ++q) {
        const int a = (int)src[q];
        const int j0 = t.begin[a], j1 = t.end[a];
        for (int j = j0; j < j1; ++j) {
            if (j == i) continue;
            const float4 pj = xf[j];
            const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 > 0.0f)) continue;
            if (soft2f > 0.0f) {
                // softened magnitude m r / (r^2 + soft^2)^{3/2}
                const float s2 = r2 + soft2f;
                acc = acc + pj.w * sqrtf(r2) / (s2 * sqrtf(s2));
            } else {
                acc = acc + pj.w / r2;
            }
        }
    }
    f[i] = g[b] + acc;
}

__global__ void k_leaf_of(TreeView t, int* __restrict__ leaf_of) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *t.dnn || t.nchild[k] != 0) return;
    for (int i = t.begin[k]; i < t.end[k]; ++i) leaf_of[i] = k;
}

// fmin of a leaf over its bodies; of an internal cell over its children
// (a minimum, so the order does not matter)
__global__ void k_fmin_leaves(TreeView t, const float* __restrict__ f, float* __restrict__ fmin) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *t.dnn || t.nchild[k] != 0) return;
    const int b = t.begin[k], e = t.end[k];
    float mn = f[b];
    for (int i = b + 1; i < e; ++i) mn = f[i] < mn ? f[i] : mn;
    fmin[k] = mn;
}

__global__ void k_fmin_internal(TreeView t, int L, float* __restrict__ fmin) {
    const int k = t.dls[L] + blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= t.dls[L + 1] || t.nchild[k] == 0) return;
    const int c0 = t.first_child[k], c1 = c0 + t.nchild[k];
    float mn = fmin[c0];
    for (int c = c0 + 1; c < c1; ++c) mn = fmin[c] < mn ? fmin[c] : mn;
    fmin[k] = mn;
}

inline int blocks_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }
}  // namespace

int dual_tree_walk(int mode, const TreeView& t, const double* zc, const double* r, const double* P,
                   const float* fmin, int p, double eps, const double* binom_row, const float4* zhi,
                   const float4* zlo, const float* r32, const float* Phat, const double* M, double soft,
                   WalkBuffers& wb, DevScalars* ds, DevScalars* h_ds, int fixed_iters, cudaStream_t st) {
    WalkCells c{t.nnodes, t.nchild, t.first_child, zc, r, P, fmin, binom_row, p, eps, zhi, zlo, r32, Phat,
                M, soft * soft, (float)(soft * soft)};
    const int nroots = t.nroots;
    const int ninit = nroots > kMaxWalkIters + 2 ? nroots : kMaxWalkIters + 2;
    (k_walk_clear<<<device_sm_count() * 4, 256, 0, st>>>(ds, wb.scan, wb.scan_tiles), note_launch());
    (k_walk_init<<<blocks_for(ninit, 256), 256, 0, st>>>(wb.front0, t.dls, ds, kMaxWalkIters + 2, mode),
     note_launch());
    const int la = mode == 0 ? 0 : 2, ll = mode == 0 ? 1 : 3;
    int2* acc_list = wb.out[la];
    int2* leaf_list = wb.out[ll];
    const int64_t cap_acc = wb.out_cap[la];
    const int64_t cap_leaf = wb.out_cap[ll];
    const int grid = device_sm_count() * 8;
    auto step = [&](int it, const int2* fi, int2* fo) {
        if (mode == 0)
            (k_walk_step_any_order<<<grid, 256, 0, st>>>(c, fi, ds->cnt + it, fo, ds->cnt + it + 1, wb.front_cap,
                                                          acc_list, ds->list_cnt + la, cap_acc, leaf_list,
                                                          ds->list_cnt + ll, cap_leaf, &ds->err), note_launch());
        else
            (k_walk_step<1><<<grid, kWalkThreads, 0, st>>>(c, it, fi, ds->cnt + it, fo, ds->cnt + it + 1, wb.front_cap,
                                                        acc_list, cap_acc, leaf_list, cap_leaf, ds, la, ll, wb.scan,
                                                        wb.scan_tiles, wb.stall_lookback, &ds->err), note_launch());
    };
    if (fixed_iters > 0) {
        // a planned number of steps with no read-back (a captured solve): steps
        // past the end of the walk find an empty frontier and return at once;
        // an overflow or a walk longer than planned shows in ds->err and in
        // the count of the step after the last
        const int nit = fixed_iters < kMaxWalkIters ? fixed_iters : kMaxWalkIters;
        for (int it = 0; it < nit; ++it)
            step(it, (it & 1) ? wb.front1 : wb.front0, (it & 1) ? wb.front0 : wb.front1);
        return nit;
    }
    int it = 0;
    const int kCheck = 6;
    while (it < kMaxWalkIters) {
        for (int s = 0; s < kCheck && it < kMaxWalkIters; ++s, ++it)
            step(it, (it & 1) ? wb.front1 : wb.front0, (it & 1) ? wb.front0 : wb.front1);
        unsigned long long nxt = 0;
        unsigned err = 0;
        if (cudaMemcpyAsync(&nxt, ds->cnt + it, sizeof(nxt), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&err, &ds->err, sizeof(err), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return FMM_ERR_CUDA;
        if (err & kErrIndex) return kWalkBadIndex;
        if (err & kErrTimeout) return FMM_ERR_TIMEOUT;
        if (err & kErrCapacity) return FMM_ERR_CAPACITY;
        if (nxt == 0) break;
    }
    if (it >= kMaxWalkIters) return FMM_ERR_CAPACITY;
    (void)h_ds;
    return it;
}

__global__ void k_walk_check(DevScalars* ds, int nit) {
    if (threadIdx.x == 0 && ds->cnt[nit] != 0) atomicOr(&ds->err, kErrCapacity);
}

void walk_check_finished(DevScalars* ds, int nit, cudaStream_t st) {
    (k_walk_check<<<1, 32, 0, st>>>(ds, nit), note_launch());
}

void pairs_to_directed(const int2* pairs, const unsigned long long* np, int64_t npcap, int nb, uint64_t* keys,
                       unsigned long long* count, unsigned long long* nkeys, cudaStream_t st) {
    (k_directed<<<blocks_for(npcap > 0 ? npcap : 1, 256), 256, 0, st>>>(pairs, np, npcap, nb, keys, count, nkeys),
     note_launch());
}

void pairs_to_directed32(const int2* pairs, const unsigned long long* np, int64_t npcap, int nb, uint32_t* keys,
                         unsigned long long* count, unsigned long long* nkeys, cudaStream_t st) {
    (k_directed32<<<blocks_for(npcap > 0 ? npcap : 1, 256), 256, 0, st>>>(pairs, np, npcap, nb, keys, count, nkeys),
     note_launch());
}

void directed_offsets_src32(const uint32_t* k32, int64_t nkeys, const unsigned long long* dnk, int nb,
                            const int* dnn, uint32_t* src, uint32_t* off, cudaStream_t st) {
    (k_offsets_src32<<<blocks_for(nkeys + 1, 256), 256, 0, st>>>(k32, nkeys, dnk, nb, dnn, src, off), note_launch());
}

void directed_offsets(const uint64_t* keys, int64_t nkeys, const unsigned long long* dnk, int nb, const int* dnn,
                      uint32_t* src, uint32_t* off, cudaStream_t st) {
    (k_offsets<<<blocks_for(nkeys + 1, 256), 256, 0, st>>>(keys, nkeys, dnk, nb, dnn, src, off), note_launch());
}

void scalar_force(const TreeView& t, const double* zc, const double* M, const float4* xf,
                  const uint32_t* far_src, const uint32_t* far_off, const uint32_t* near_src,
                  const uint32_t* near_off, const int* h_level_start, double soft, float* farf,
                  float* f, float* fmin, cudaStream_t st) {
    // farf doubles as scratch: [0, nnodes) far sums, [nnodes, 2 nnodes) pushed-down g,
    // and the leaf index of every body after that.
    float* g = farf + t.nnodes;
    int* leaf_of = reinterpret_cast<int*>(farf + 2 * (size_t)t.nnodes);
    (k_far_f<<<blocks_for(32 * (int64_t)t.nnodes, 128), 128, 0, st>>>(t.dnn, zc, M, far_src, far_off, farf),
     note_launch());
    (k_push_down<<<blocks_for(t.nnodes, 128), 128, 0, st>>>(t, farf, g), note_launch());
    (k_leaf_of<<<blocks_for(t.nnodes, 128), 128, 0, st>>>(t, leaf_of), note_launch());
    (k_near_f<<<blocks_for(t.n, 128), 128, 0, st>>>(t, xf, near_src, near_off, leaf_of, g, (float)(soft * soft), f),
     note_launch());
    (k_fmin_leaves<<<blocks_for(t.nnodes, 128), 128, 0, st>>>(t, f, fmin), note_launch());
    (void)h_level_start;
    for (int L = t.nlevels - 2; L >= 0; --L)
        if (t.lvl_cnt[L] > 0) (k_fmin_internal<<<blocks_for(t.lvl_cnt[L], 128), 128, 0, st>>>(t, L, fmin), note_launch());
}

}  // namespace gbfmm
