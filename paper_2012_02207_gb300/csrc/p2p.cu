// Leaf evaluation: far field by L2P, near field by P2P (Sec. 2.1), plus the
// plain FP64 direct sum used to measure force errors (Sec. 3.1.1).
//
// P2P runs over work items: a target leaf and at most kLeavesPerItem of the
// source leaves in its (sorted) P2P list, taken by warps from a counter.
// The default kernel (k_p2p_tiles) stages the item's source bodies in shared
// memory, by bulk copies or plain loads, puts the sources across the lanes
// and keeps a group of target bodies in every lane's registers, so one
// shared-memory load serves several interactions and every lane is busy
// whatever the leaf sizes; a fixed transpose reduction then sums the lanes.
// The alternative kernel (k_p2p_lanes, GBFMM_P2P_TILES=0) gives each target
// G = 32 / nt lanes that split the sources between them. Each item writes
// one partial per target body. k_leaf_reduce then evaluates the leaf's local
// expansion at the body (L2P), adds the body's partials in item order, and
// writes the result to the caller's order through the sort permutation.
// Every sum runs in a fixed order.
//
// Mixed precision: bodies are stored relative to their own leaf centre in
// FP32; a source leaf A is moved into the target leaf B's frame by the
// FP32-rounded offset z_A - z_B (computed from double-float centres). Terms
// are FP32 (rsqrtf); each staged pack's sum is accumulated in FP64.
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
// PC > 0: the order is the compile-time PC (loops unrolled); PC = 0: p.
template <typename T, typename Tab, int PC = 0>
__device__ __forceinline__ void l2p_hat(int p_rt, const T* __restrict__ F, T x, T y, T z, T inv_s, const Tab& tb,
                                        T& phi, T& ax, T& ay, T& az) {
    const int p = PC > 0 ? PC : p_rt;
    const T r2 = x * x + y * y + z * z;
    T pot = T(0), g0 = T(0), g1r = T(0), g1i = T(0);
    T dre = T(1), dim = T(0);  // Shat_l^l
#pragma unroll
    for (int l = 0; l <= p; ++l) {
        if (l > 0) {
            const T t = dre * x - dim * y;
            dim = dre * y + dim * x;
            dre = t;
            dre *= tb.D(l);
            dim *= tb.D(l);
        }
        T s1r = dre, s1i = dim, s2r = T(0), s2i = T(0);  // Shat_k^l, Shat_{k-1}^l
#pragma unroll
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

// ---------------------------------------------------------------------------
// P2P over work items. Item (B, j) covers the sources q in
// [off[B] + j*kLeavesPerItem, ...) of target leaf B (at most kLeavesPerItem
// source leaves), so no warp carries more than a bounded share of a dense
// leaf's work. Warps fetch items dynamically. Each item writes one partial
// sum per target body; k_leaf_reduce adds the partials of a body in item
// order (deterministic) together with the L2P far field.

// Knuth's two-sum: (hi, lo) += b with the rounding error kept in lo.
__device__ __forceinline__ void two_sum(float& hi, float& lo, float b) {
    const float s = hi + b;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (b - bb);
    hi = s;
    lo += err;
}

// a body (position, mass) as one 16-byte (FP32) or 32-byte (FP64) aligned record,
// so that shared-memory reads and writes take one vector access
template <typename T>
struct alignas(4 * sizeof(T)) Body4 { T x, y, z, w; };

constexpr int kStageCap = 256;  // bodies staged per pack (source leaves packed back to back)

// Accumulators of one target: FP32 runs of at most kRun terms are folded
// into (hi, lo) two-sum pairs (FP64 sums in FP64 mode), so the FP32 rounding
// of near-field terms that cancel stays at the level of a short run.
constexpr int kRun = 16;

template <typename T>
struct NearAcc {
    float hx = 0.f, hy = 0.f, hz = 0.f, hp = 0.f, lx = 0.f, ly = 0.f, lz = 0.f, lp = 0.f;
    double dx = 0.0, dy = 0.0, dz = 0.0, dp = 0.0;
    __device__ __forceinline__ void add(T px, T py, T pz, T pp) {
        if (sizeof(T) == 4) {
            two_sum(hx, lx, (float)px);
            two_sum(hy, ly, (float)py);
            two_sum(hz, lz, (float)pz);
            two_sum(hp, lp, (float)pp);
        } else {
            dx += (double)px; dy += (double)py; dz += (double)pz; dp += (double)pp;
        }
    }
};

// 1/sqrt(x) in FP64 without the long FP64 divide and square root: an FP32
// seed refined by two Newton steps y <- y (3 - x y^2) / 2 (each squares the
// relative error: about 2^-22 -> 2^-44 -> the FP64 rounding level). Outside
// the FP32 range of the seed (and for x = 0) it falls back to 1 / sqrt(x).
__device__ __forceinline__ double rsqrt_nr(double x) {
    if (!(x > 1e-30 && x < 1e30)) return x > 0.0 ? 1.0 / sqrt(x) : 0.0;
    double y = (double)rsqrtf((float)x);
    const double hx = 0.5 * x;
    y = y * fma(-hx * y, y, 1.5);
    y = y * fma(-hx * y, y, 1.5);
    return y;
}

// ---------------------------------------------------------------------------
// P2P force over work items, sources across lanes and targets in registers.
//
// A warp stages the item's source bodies (moved into the target leaf B's
// frame) in shared memory, up to TileCfg::kCap at a time. The targets of B
// are taken in groups of TG (8 in FP32, 4 in FP64; a last group of TG/2 when
// at most TG/2 remain). For a group, lane l runs over the staged sources
// l, l + 32, l + 64, ... and keeps TG four-component partial sums (ax, ay,
// az, sum m/r) in registers: one shared-memory load serves TG interactions
// and every lane is busy whatever the leaf sizes. The 32 lanes' partials of
// the group are then summed by a transpose reduction across the warp (a
// fixed tree: lane l ends with component l % 4 of target l / 4), and added
// in FP64 to the group's totals in shared memory. So the order of every sum
// is fixed and the result does not depend on scheduling.
//
// FP32 terms are summed per lane over at most kCap / 32 = 16 sources of a
// staged pack, the cross-lane tree adds five levels, and each pack's total is
// accumulated in FP64.
//
// SOFT: Plummer softening (Appendix B), 1/r -> 1/sqrt(r^2 + s2); the body
// itself (r2 = 0; coincident bodies are rejected) still contributes nothing.

template <typename T>
struct TileCfg;
#ifndef GBFMM_P2P_CAP32
#define GBFMM_P2P_CAP32 512
#endif
// blocks per SM the tile kernel's registers are cut for: 4 (128 registers, no
// spill) measured 5.74 ms against 5.82 ms for 5 (96 registers, a small spill)
#ifndef GBFMM_P2P_MINB
#define GBFMM_P2P_MINB 4
#endif
#ifndef GBFMM_P2P_TG
#define GBFMM_P2P_TG 8
#endif
template <>
struct TileCfg<float> {
    static constexpr int TG = GBFMM_P2P_TG;  // targets per group
    static constexpr int kCap = GBFMM_P2P_CAP32;  // staged source bodies per warp (512: 8 KB, at most 16 per lane)
};
template <>
struct TileCfg<double> {
    static constexpr int TG = 4;
    static constexpr int kCap = 256;          // 8 KB per warp
};
constexpr int kTargetChunk = 64;  // targets whose totals a warp keeps in shared memory per pass

// per warp: staged sources, the target chunk's positions, its FP64 totals, an mbarrier
template <typename T>
constexpr size_t p2p_tile_smem_per_warp() {
    return sizeof(Body4<T>) * TileCfg<T>::kCap + sizeof(Body4<T>) * kTargetChunk + sizeof(double) * 4 * kTargetChunk +
           4 * sizeof(Body4<T>);
}

// Bulk-copy staging (BULK, FP32; the default, FMM_FLAG_P2P_LOADS turns it off):
// the bodies of every staged
// source leaf come into shared memory by one cp.async.bulk (the tensor memory
// accelerator's 1-D copy, 16-byte aligned, a multiple of 16 bytes) that
// completes on the warp's mbarrier; the leaf-centre offsets are then added in
// shared memory. Waits are bounded: after kBulkWaitNs the warp raises
// kErrTimeout and leaves the kernel (every issued copy has completed by then
// unless the copy engine itself stalled).
constexpr unsigned long long kBulkWaitNs = 1000000000ull;  // one second

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// generic-proxy accesses of shared memory before this are ordered before later bulk copies into it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// wait (all lanes) for the phase of the warp's mbarrier; false: the wait ran out
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
    const unsigned long long t0 = global_ns();
    bool done = mbar_test(bar, phase);
    while (!done) {
        if (global_ns() - t0 > kBulkWaitNs) break;
        done = mbar_test(bar, phase);
    }
    return __all_sync(0xffffffffu, done) != 0;
}

// Stage whole source leaves src[q], src[q+1], ... (below q1) of target leaf
// B into sm, moved into B's frame, as many as fit in kCap bodies; returns the
// body count, advances q and sets selfin if B itself is among them. The lanes
// read 32 leaves' ranges and centres at once and copy their bodies with
// independent loads, so the latency of the index, range and body loads is paid
// once per 32 leaves rather than once per leaf. A leaf larger than kCap (a
// level-21 leaf can exceed the leaf size) goes in pieces of kCap bodies, soff
// being the next body of it.
template <typename T, int kCap, bool BULK>
__device__ __forceinline__ int stage_leaves(const LeafArgs& a, int B, float4 bh, float4 bl, uint32_t& q,
                                            uint32_t q1, int& soff, Body4<T>* __restrict__ sm, bool& selfin,
                                            int lane, uint64_t* bar, uint32_t& phase, bool& timed_out) {
    int cnt = 0;
    selfin = false;
    {
        // the next leaf does not fit in an empty stage, or a piece of it is already staged
        const int A = (int)a.p2p_src[q];
        const int a0 = a.t.begin[A], nA = a.t.end[A] - a0;
        if (soff > 0 || nA > kCap) {
            const int take = nA - soff < kCap ? nA - soff : kCap;
            float ox = 0.f, oy = 0.f, oz = 0.f;
            if (sizeof(T) == 4) {
                const float4 ah = a.zhi[A], al = a.zlo[A];
                ox = (ah.x - bh.x) + (al.x - bl.x);
                oy = (ah.y - bh.y) + (al.y - bl.y);
                oz = (ah.z - bh.z) + (al.z - bl.z);
            }
            for (int l = lane; l < take; l += 32) {
                const int jj = a0 + soff + l;
                Body4<T> v;
                if (sizeof(T) == 4) {
                    const float4 u = a.prel[jj];
                    v = {(T)(u.x + ox), (T)(u.y + oy), (T)(u.z + oz), (T)u.w};
                } else {
                    v = {(T)a.xs[jj], (T)a.ys[jj], (T)a.zs[jj], (T)a.ms[jj]};
                }
                sm[l] = v;
            }
            selfin = A == B;
            soff += take;
            if (soff >= nA) {
                soff = 0;
                ++q;
            }
            return take;
        }
    }
    while (q < q1) {
        const int nl = q1 - q < 32u ? (int)(q1 - q) : 32;
        int A = -1, a0 = 0, nA = 0;
        float ox = 0.f, oy = 0.f, oz = 0.f;
        if (lane < nl) {
            A = (int)a.p2p_src[q + lane];
            a0 = a.t.begin[A];
            nA = a.t.end[A] - a0;
            if (sizeof(T) == 4) {
                const float4 ah = a.zhi[A], al = a.zlo[A];
                ox = (ah.x - bh.x) + (al.x - bl.x);
                oy = (ah.y - bh.y) + (al.y - bl.y);
                oz = (ah.z - bh.z) + (al.z - bl.z);
            }
        }
        int incl = nA;  // inclusive prefix sum of the leaf sizes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const unsigned fits = __ballot_sync(0xffffffffu, lane < nl && cnt + incl <= kCap);
        // (an empty stage always takes the first leaf: one larger than kCap went the piecewise way above,
        // and this loop stops before such a leaf once anything is staged)
        const int fit = __popc(fits);  // a prefix of the leaves, since incl grows
        selfin |= __any_sync(0xffffffffu, lane < fit && A == B) != 0;
        if (BULK && sizeof(T) == 4 && fit > 0) {
            // one bulk copy per leaf (lane j for leaf j), then the offsets in shared memory
            const uint32_t bytes = (uint32_t)__shfl_sync(0xffffffffu, incl, fit - 1) * (uint32_t)sizeof(Body4<T>);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive_expect(bar, bytes + a.tx_extra);
            __syncwarp();
            if (lane < fit)
                bulk_to_smem(sm + cnt + incl - nA, a.prel + a0, (uint32_t)nA * (uint32_t)sizeof(Body4<T>), bar);
            const bool ok = mbar_wait_bounded(bar, phase);
            phase ^= 1u;
            if (!ok) {
                timed_out = true;
                return cnt;
            }
#pragma unroll 4
            for (int j = 0; j < fit; ++j) {
                const int nj = __shfl_sync(0xffffffffu, nA, j);
                const int dst = cnt + __shfl_sync(0xffffffffu, incl, j) - nj;
                const float oxj = __shfl_sync(0xffffffffu, ox, j), oyj = __shfl_sync(0xffffffffu, oy, j),
                            ozj = __shfl_sync(0xffffffffu, oz, j);
                for (int l = lane; l < nj; l += 32) {
                    Body4<T>& v = sm[dst + l];
                    v.x = (T)(v.x + oxj);
                    v.y = (T)(v.y + oyj);
                    v.z = (T)(v.z + ozj);
                }
            }
            cnt += __shfl_sync(0xffffffffu, incl, fit - 1);
            q += (uint32_t)fit;
            if (fit < nl) break;
            continue;
        }
#pragma unroll 4
        for (int j = 0; j < fit; ++j) {
            const int aj = __shfl_sync(0xffffffffu, a0, j), nj = __shfl_sync(0xffffffffu, nA, j);
            const int dst = cnt + __shfl_sync(0xffffffffu, incl, j) - nj;
            const float oxj = __shfl_sync(0xffffffffu, ox, j), oyj = __shfl_sync(0xffffffffu, oy, j),
                        ozj = __shfl_sync(0xffffffffu, oz, j);
            for (int l = lane; l < nj; l += 32) {
                Body4<T> v;
                if (sizeof(T) == 4) {
                    const float4 u = a.prel[aj + l];
                    v = {(T)(u.x + oxj), (T)(u.y + oyj), (T)(u.z + ozj), (T)u.w};
                } else {
                    v = {(T)a.xs[aj + l], (T)a.ys[aj + l], (T)a.zs[aj + l], (T)a.ms[aj + l]};
                }
                sm[dst + l] = v;
            }
        }
        if (fit > 0) cnt += __shfl_sync(0xffffffffu, incl, fit - 1);
        q += (uint32_t)fit;
        if (fit < nl) break;  // the stage is full
    }
    return cnt;
}

// Halving step of the transpose reduction: C values per lane become C/2;
// a lane with bit o set keeps the upper half and receives its partner's.
template <int C, typename T>
__device__ __forceinline__ void halve(T* v, int lane, int o) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < C / 2; ++i) {
        const T send = up ? v[i] : v[i + C / 2];
        const T keep = up ? v[i + C / 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
}

// The same step for a lane whose halves are already swapped when bit o is
// set (slot s of such a lane holds value s ^ (C/2)): every lane keeps the
// lower slots and sends the upper ones, with no selects.
template <int C, typename T>
__device__ __forceinline__ void halve_swapped(T* v, int o) {
#pragma unroll
    for (int i = 0; i < C / 2; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i + C / 2], o);
}

// v[0..V-1] on every lane (V = 32, 16 or 8), value j = 4 t + c (target t,
// component c), with lane l holding target t ^ ((l >> 2) & (V/4 - 1)) in
// slot t (the target order p2p_group gives each lane). On return v[0] of
// lane l holds the sum over the 32 lanes of value l % V. The steps over the
// target bits (lane bits 4..2) need no selects; the two over the components
// (lane bits 1, 0) do.
template <int V, typename T>
__device__ __forceinline__ T transpose_reduce(T* v, int lane) {
    static_assert(V == 32 || V == 16 || V == 8, "V");
    if constexpr (V <= 16) {
#pragma unroll
        for (int i = 0; i < V; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], 16);
    }
    if constexpr (V == 8) {
#pragma unroll
        for (int i = 0; i < V; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], 8);
    }
    if constexpr (V == 32) halve_swapped<32>(v, 16);
    if constexpr (V >= 16) halve_swapped<16>(v, 8);
    halve_swapped<8>(v, 4);
    halve<4>(v, lane, 2);
    halve<2>(v, lane, 1);
    return v[0];
}

// One group of NT targets (b0 + t0 .. b0 + t0 + NT - 1, clamped to the last
// target; clamped duplicates are computed and discarded) against the cnt
// staged sources; adds the group's totals to tot[4 * (t0 + t) + c]. Lane l
// keeps target t ^ g, g = (l >> 2) & (NT - 1), in its slot t: the order the
// select-free steps of transpose_reduce expect. A lane's FP32 sums run over
// at most kCap / 32 terms.
template <typename T, int NT, bool GUARD, bool SOFT>
__device__ __forceinline__ void p2p_group(const Body4<T>* __restrict__ sm, int cnt, const Body4<T>* __restrict__ tg,
                                          int t0, int nt, T s2, double* tot, int lane) {
    const int g = (lane >> 2) & (NT - 1);
    T tx[NT], ty[NT], tz[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const int i = t0 + (t ^ g);
        const Body4<T> v = tg[i < nt ? i : nt - 1];
        tx[t] = v.x; ty[t] = v.y; tz[t] = v.z;
    }
    T run[NT * 4];
#pragma unroll
    for (int e = 0; e < NT * 4; ++e) run[e] = T(0);
    // the stage is padded to a multiple of 32 with massless far bodies (pad_stage)
    const int per_lane = (cnt + 31) >> 5;
    for (int u = 0; u < per_lane; ++u) {
        const Body4<T> s = sm[lane + 32 * u];
        const T mj = s.w;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const T dx = s.x - tx[t], dy = s.y - ty[t], dz = s.z - tz[t];
            const T r2 = dx * dx + dy * dy + dz * dz;
            T rinv;
            if constexpr (sizeof(T) == 4) rinv = rsqrtf(SOFT ? r2 + s2 : r2);
            else rinv = (T)rsqrt_nr((double)(SOFT ? r2 + s2 : r2));
            if (GUARD && !(r2 > T(0))) rinv = T(0);  // the body itself
            const T mr = mj * rinv;
            const T mr3 = mr * rinv * rinv;
            run[4 * t] += mr3 * dx;
            run[4 * t + 1] += mr3 * dy;
            run[4 * t + 2] += mr3 * dz;
            run[4 * t + 3] += mr;
        }
    }
    const T v = transpose_reduce<NT * 4>(run, lane);
    if (lane < NT * 4 && 4 * t0 + lane < 4 * nt) tot[4 * t0 + lane] += (double)v;
}

// Fill the stage from cnt up to the next multiple of 32 with massless bodies
// at x = 1e18: their terms are exactly zero (r^2 ~ 1e36 stays finite in FP32,
// 0 * r^-1 = 0), so the lanes' loops need no bounds test. kCap is a multiple
// of 32, so the padding stays inside the stage.
template <typename T>
__device__ __forceinline__ void pad_stage(Body4<T>* sm, int cnt, int lane) {
    const int k = cnt + lane;
    if (k < ((cnt + 31) & ~31)) sm[k] = {T(1e18), T(0), T(0), T(0)};
}

template <typename T, bool GUARD, bool SOFT>
__device__ __forceinline__ void p2p_groups(const Body4<T>* __restrict__ sm, int cnt, const Body4<T>* __restrict__ tg,
                                           int nt, T s2, double* tot, int lane) {
    constexpr int TG = TileCfg<T>::TG;
    int t0 = 0;
    for (; nt - t0 > TG / 2; t0 += TG) p2p_group<T, TG, GUARD, SOFT>(sm, cnt, tg, t0, nt, s2, tot, lane);
    if (t0 < nt) p2p_group<T, TG / 2, GUARD, SOFT>(sm, cnt, tg, t0, nt, s2, tot, lane);
}

template <typename T, bool SOFT, bool BULK>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 4 : GBFMM_P2P_MINB) k_p2p_tiles(LeafArgs a, const int* __restrict__ item_leaf,
                                                    const uint32_t* __restrict__ item_first,
                                                    const uint32_t* __restrict__ slot_first,
                                                    const uint32_t* __restrict__ nitems_p, unsigned* __restrict__ work) {
    constexpr int kCap = TileCfg<T>::kCap;
    static_assert(kCap % 32 == 0, "the padded stage must fit in kCap");
    extern __shared__ __align__(16) unsigned char p2p_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char* wbase = p2p_smem + (size_t)wib * p2p_tile_smem_per_warp<T>();
    Body4<T>* sm = reinterpret_cast<Body4<T>*>(wbase);
    Body4<T>* tg = sm + kCap;
    double* tot = reinterpret_cast<double*>(tg + kTargetChunk);
    uint64_t* bar = reinterpret_cast<uint64_t*>(tot + 4 * kTargetChunk);  // the warp's mbarrier (bulk staging)
    uint32_t phase = 0;
    bool timed_out = false;
    if (BULK && sizeof(T) == 4) {
        if (lane == 0) mbar_init(bar);
        __syncwarp();
    }
    const int nitems = (int)*nitems_p;
    const T s2 = SOFT ? (sizeof(T) == 4 ? (T)a.soft2f : (T)a.soft2) : T(0);
    for (;;) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(work, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if ((int)it >= nitems) break;
        const int B = item_leaf[it];
        const int j = (int)(it - item_first[B]);
        const uint32_t q0 = a.p2p_off[B] + (uint32_t)j * kLeavesPerItem;
        const uint32_t qe = a.p2p_off[B + 1];
        const uint32_t q1 = q0 + kLeavesPerItem < qe ? q0 + kLeavesPerItem : qe;
        const int b0 = a.t.begin[B], nB = a.t.end[B] - b0;
        const uint32_t slot0 = slot_first[B] + (uint32_t)j * (uint32_t)nB;
        const float4 bh = a.zhi[B], bl = a.zlo[B];
        unsigned long long nsrc = 0;  // source bodies of this item (for the interaction count)
        bool self_item = false;
        for (int tc = 0; tc < nB; tc += kTargetChunk) {
            const int nt = nB - tc < kTargetChunk ? nB - tc : kTargetChunk;
            __syncwarp();
            for (int e = lane; e < 4 * nt; e += 32) tot[e] = 0.0;
            for (int t = lane; t < nt; t += 32) {
                const int i = b0 + tc + t;
                if (sizeof(T) == 4) {
                    const float4 v = a.prel[i];
                    tg[t] = {(T)v.x, (T)v.y, (T)v.z, (T)v.w};
                } else {
                    tg[t] = {(T)a.xs[i], (T)a.ys[i], (T)a.zs[i], (T)a.ms[i]};
                }
            }
            uint32_t q = q0;
            int soff = 0;
            while (q < q1) {
                __syncwarp();
                bool selfin = false;
                const int cnt = stage_leaves<T, kCap, BULK>(a, B, bh, bl, q, q1, soff, sm, selfin, lane, bar, phase,
                                                            timed_out);
                if (timed_out) {
                    if (lane == 0) atomicOr(a.err, kErrTimeout);
                    return;
                }
                pad_stage<T>(sm, cnt, lane);
                __syncwarp();
                if (tc == 0) { nsrc += (unsigned long long)cnt; self_item |= selfin; }
                if (selfin) p2p_groups<T, true, SOFT>(sm, cnt, tg, nt, s2, tot, lane);
                else p2p_groups<T, false, SOFT>(sm, cnt, tg, nt, s2, tot, lane);
            }
            __syncwarp();
            // totals to the item's partial slots: (ax, ay) in part_hi, (az, sum m/r) in part_lo
            double* hi = reinterpret_cast<double*>(a.part_hi);
            double* lo = reinterpret_cast<double*>(a.part_lo);
            for (int e = lane; e < 4 * nt; e += 32) {
                const size_t slot = (size_t)slot0 + (size_t)(tc + (e >> 2));
                const int c = e & 3;
                (c < 2 ? hi : lo)[2 * slot + (c & 1)] = tot[e];
            }
        }
        // directed body-body interactions of the item (a body never acts on itself)
        if (lane == 0)
            atomicAdd(a.interactions, (unsigned long long)nB * nsrc - (self_item ? (unsigned long long)nB : 0ull));
    }
}

// ---------------------------------------------------------------------------
// P2P force over work items, targets across lanes (the alternative layout,
// selected by GBFMM_P2P_TILES = 0): a warp stages the item's sources in
// shared memory 256 at a time and gives each of the nt targets of a chunk of
// 32 G = 32 / nt lanes that split the sources between them; FP32 runs of
// kRun terms are folded into two-sum pairs; one partial per target body.
// SOFT: Plummer softening (Appendix B), 1/r -> 1/sqrt(r^2 + s2); the body
// itself (r2 = 0; coincident bodies are rejected) still contributes nothing.
template <typename T, bool GUARD, int GC, bool SOFT>
__device__ __forceinline__ void p2p_pack_g(const Body4<T>* __restrict__ sm, int cnt, int sub, int Gr, T tx, T ty,
                                           T tz, T s2, NearAcc<T>& acc) {
    const int G = GC > 0 ? GC : Gr;  // lanes per target (compile-time when GC > 0)
    auto term = [&](int k, T& px, T& py, T& pz, T& pp) {
        const Body4<T> sv = sm[k];
        const T dx = sv.x - tx, dy = sv.y - ty, dz = sv.z - tz;
        const T r2 = dx * dx + dy * dy + dz * dz;
        T rinv;
        if (sizeof(T) == 4) {
            rinv = (T)rsqrtf((float)(SOFT ? r2 + s2 : r2));
            if (GUARD && !(r2 > T(0))) rinv = T(0);  // the body itself
        } else {
            rinv = (T)rsqrt_nr((double)(SOFT ? r2 + s2 : r2));
            if (SOFT && GUARD && !(r2 > T(0))) rinv = T(0);
        }
        const T mr = sv.w * rinv;
        const T mr3 = mr * rinv * rinv;
        px += mr3 * dx;
        py += mr3 * dy;
        pz += mr3 * dz;
        pp += mr;
    };
    int k0 = sub;
    if (GC > 0) {
        // full runs of kRun terms, unrolled (constant shared-memory offsets, no loop control)
        for (; k0 + kRun * GC <= cnt; k0 += kRun * GC) {
            T px = T(0), py = T(0), pz = T(0), pp = T(0);
#pragma unroll
            for (int u = 0; u < kRun; ++u) term(k0 + u * GC, px, py, pz, pp);
            acc.add(px, py, pz, pp);
        }
    }
    for (; k0 < cnt; k0 += kRun * G) {
        const int k1 = k0 + kRun * G < cnt ? k0 + kRun * G : cnt;
        T px = T(0), py = T(0), pz = T(0), pp = T(0);
#pragma unroll 4
        for (int k = k0; k < k1; k += G) term(k, px, py, pz, pp);
        acc.add(px, py, pz, pp);
    }
}

template <typename T, bool GUARD, bool SOFT>
__device__ __forceinline__ void p2p_pack(const Body4<T>* __restrict__ sm, int cnt, int sub, int G, T tx, T ty,
                                         T tz, T s2, NearAcc<T>& acc) {
    if (G == 1) p2p_pack_g<T, GUARD, 1, SOFT>(sm, cnt, sub, G, tx, ty, tz, s2, acc);
    else if (G == 2) p2p_pack_g<T, GUARD, 2, SOFT>(sm, cnt, sub, G, tx, ty, tz, s2, acc);
    else if (G == 4) p2p_pack_g<T, GUARD, 4, SOFT>(sm, cnt, sub, G, tx, ty, tz, s2, acc);
    else p2p_pack_g<T, GUARD, 0, SOFT>(sm, cnt, sub, G, tx, ty, tz, s2, acc);
}

template <typename T, bool SOFT>
__global__ void __launch_bounds__(128) k_p2p_lanes(LeafArgs a, const int* __restrict__ item_leaf,
                                                    const uint32_t* __restrict__ item_first,
                                                    const uint32_t* __restrict__ slot_first,
                                                    const uint32_t* __restrict__ nitems_p, unsigned* __restrict__ work) {
    __shared__ Body4<T> stage[4][kStageCap];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    Body4<T>* sm = stage[wib];
    const int nitems = (int)*nitems_p;
    for (;;) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(work, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if ((int)it >= nitems) break;
        const int B = item_leaf[it];
        const int j = (int)(it - item_first[B]);
        const uint32_t q0 = a.p2p_off[B] + (uint32_t)j * kLeavesPerItem;
        const uint32_t qe = a.p2p_off[B + 1];
        const uint32_t q1 = q0 + kLeavesPerItem < qe ? q0 + kLeavesPerItem : qe;
        const int b0 = a.t.begin[B], nB = a.t.end[B] - b0;
        const uint32_t slot0 = slot_first[B] + (uint32_t)j * (uint32_t)nB;
        const float4 bh = a.zhi[B], bl = a.zlo[B];
        unsigned long long nsrc = 0;  // source bodies of this item (for the interaction count)
        bool self_item = false;
        for (int tc = 0; tc < nB; tc += 32) {
            const int nt = nB - tc < 32 ? nB - tc : 32;
            const int G = 32 / nt;            // lanes per target
            const int t = lane / G, sub = lane - t * G;
            const bool act = t < nt;
            T tx = T(0), ty = T(0), tz = T(0);
            if (act) {
                if (sizeof(T) == 4) {
                    const float4 v = a.prel[b0 + tc + t];
                    tx = (T)v.x; ty = (T)v.y; tz = (T)v.z;
                } else {
                    tx = (T)a.xs[b0 + tc + t]; ty = (T)a.ys[b0 + tc + t]; tz = (T)a.zs[b0 + tc + t];
                }
            }
            NearAcc<T> acc;
            uint32_t q = q0;
            int soff = 0;
            while (q < q1) {
                // pack source leaves (or a piece of an oversized one) into the stage
                __syncwarp();
                int cnt = 0;
                bool selfin = false;
                while (q < q1) {
                    const int A = (int)a.p2p_src[q];
                    const int a0 = a.t.begin[A], nA = a.t.end[A] - a0;
                    const int rem = nA - soff;
                    int take = rem;
                    if (cnt + take > kStageCap) {
                        if (cnt > 0) break;
                        take = kStageCap;
                    }
                    float ox = 0.f, oy = 0.f, oz = 0.f;
                    if (sizeof(T) == 4) {
                        const float4 ah = a.zhi[A], al = a.zlo[A];
                        ox = (ah.x - bh.x) + (al.x - bl.x);
                        oy = (ah.y - bh.y) + (al.y - bl.y);
                        oz = (ah.z - bh.z) + (al.z - bl.z);
                    }
                    for (int l = lane; l < take; l += 32) {
                        const int jj = a0 + soff + l;
                        Body4<T> v;
                        if (sizeof(T) == 4) {
                            const float4 u = a.prel[jj];
                            v = {(T)(u.x + ox), (T)(u.y + oy), (T)(u.z + oz), (T)u.w};
                        } else {
                            v = {(T)a.xs[jj], (T)a.ys[jj], (T)a.zs[jj], (T)a.ms[jj]};
                        }
                        sm[cnt + l] = v;
                    }
                    selfin |= (A == B);
                    if (tc == 0) { nsrc += (unsigned long long)take; self_item |= (A == B); }
                    cnt += take;
                    if (take < rem) { soff += take; break; }
                    soff = 0;
                    ++q;
                }
                __syncwarp();
                if (!act) continue;
                const T s2 = SOFT ? (sizeof(T) == 4 ? (T)a.soft2f : (T)a.soft2) : T(0);
                if (selfin) p2p_pack<T, true, SOFT>(sm, cnt, sub, G, tx, ty, tz, s2, acc);
                else p2p_pack<T, false, SOFT>(sm, cnt, sub, G, tx, ty, tz, s2, acc);
            }
            float &hx = acc.hx, &hy = acc.hy, &hz = acc.hz, &hp = acc.hp;
            float &lx = acc.lx, &ly = acc.ly, &lz = acc.lz, &lp = acc.lp;
            double &dx64 = acc.dx, &dy64 = acc.dy, &dz64 = acc.dz, &dp64 = acc.dp;
            // combine the G sub-lanes of each target in sub-lane order
            const int leader = t * G;
            for (int s = 1; s < G; ++s) {
                const int src = leader + s < 32 ? leader + s : 31;
                if (sizeof(T) == 4) {
                    const float vx = __shfl_sync(0xffffffffu, hx, src), vy = __shfl_sync(0xffffffffu, hy, src),
                                vz = __shfl_sync(0xffffffffu, hz, src), vp = __shfl_sync(0xffffffffu, hp, src);
                    const float wx = __shfl_sync(0xffffffffu, lx, src), wy = __shfl_sync(0xffffffffu, ly, src),
                                wz = __shfl_sync(0xffffffffu, lz, src), wp = __shfl_sync(0xffffffffu, lp, src);
                    if (sub == 0 && act) {
                        two_sum(hx, lx, vx); lx += wx;
                        two_sum(hy, ly, vy); ly += wy;
                        two_sum(hz, lz, vz); lz += wz;
                        two_sum(hp, lp, vp); lp += wp;
                    }
                } else {
                    const double vx = __shfl_sync(0xffffffffu, dx64, src), vy = __shfl_sync(0xffffffffu, dy64, src),
                                 vz = __shfl_sync(0xffffffffu, dz64, src), vp = __shfl_sync(0xffffffffu, dp64, src);
                    if (sub == 0 && act) { dx64 += vx; dy64 += vy; dz64 += vz; dp64 += vp; }
                }
            }
            if (act && sub == 0) {
                const uint32_t slot = slot0 + (uint32_t)(tc + t);
                if (sizeof(T) == 4) {
                    a.part_hi[slot] = make_double2((double)hx + (double)lx, (double)hy + (double)ly);
                    a.part_lo[slot] = make_double2((double)hz + (double)lz, (double)hp + (double)lp);
                } else {
                    a.part_hi[slot] = make_double2(dx64, dy64);
                    a.part_lo[slot] = make_double2(dz64, dp64);
                }
            }
        }
        // directed body-body interactions of the item (a body never acts on itself)
        if (lane == 0)
            atomicAdd(a.interactions, (unsigned long long)nB * nsrc - (self_item ? (unsigned long long)nB : 0ull));
    }
}

// One thread per body: L2P of its leaf's local expansion plus the P2P
// partials of its leaf's items in item order; G-scaled, to the caller's order.
template <typename T, int PC>
__global__ void __launch_bounds__(128) k_leaf_reduce(LeafArgs a, const int* __restrict__ leaf_of,
                                                      const uint32_t* __restrict__ item_first,
                                                      const uint32_t* __restrict__ slot_first) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.t.n) return;
    const int B = leaf_of[i];
    const int b0 = a.t.begin[B], nB = a.t.end[B] - b0;
    const int nr = ncoef_real(a.p);
    double sx, sy, sz, sp;
    if (sizeof(T) == 4) {
        const TabL32 tb;
        const float4 bh = a.zhi[B];
        const float inv_s = 1.0f / bh.w;
        const float4 v = a.prel[i];
        float phi, fx, fy, fz;
        l2p_hat<float, TabL32, PC>(a.p, reinterpret_cast<const float*>(a.loc) + (size_t)nr * B, v.x * inv_s,
                                   v.y * inv_s, v.z * inv_s, inv_s, tb, phi, fx, fy, fz);
        sx = fx; sy = fy; sz = fz; sp = phi;
    } else {
        const TabL64 tb{a.tb.w, a.tb.iw, a.tb.rec_a, a.tb.rec_b, a.tb.diag, a.tb.sub};
        const double inv_s = 1.0 / a.hs[B];
        double phi, fx, fy, fz;
        l2p_hat<double>(a.p, reinterpret_cast<const double*>(a.loc) + (size_t)nr * B,
                        (a.xs[i] - a.zc[3 * B]) * inv_s, (a.ys[i] - a.zc[3 * B + 1]) * inv_s,
                        (a.zs[i] - a.zc[3 * B + 2]) * inv_s, inv_s, tb, phi, fx, fy, fz);
        sx = fx; sy = fy; sz = fz; sp = phi;
    }
    const uint32_t i0 = item_first[B], i1 = item_first[B + 1];
    const uint32_t s0 = slot_first[B] + (uint32_t)(i - b0);
    // the body's item partials in item order; four items' loads are issued
    // before they are added, so their latencies overlap
    uint32_t it = i0;
    for (; it + 4 <= i1; it += 4) {
        double2 u[4], w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t slot = s0 + (it + k - i0) * (uint32_t)nB;
            if (slot >= a.slots_cap) slot = 0;  // only after a capacity error (the result is discarded)
            u[k] = a.part_hi[slot];
            w[k] = a.part_lo[slot];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) { sx += u[k].x; sy += u[k].y; sz += w[k].x; sp -= w[k].y; }
    }
    for (; it < i1; ++it) {
        const uint32_t slot = s0 + (it - i0) * (uint32_t)nB;
        if (slot >= a.slots_cap) break;  // only after a capacity error (the result is discarded)
        const double2 u = a.part_hi[slot], w = a.part_lo[slot];
        sx += u.x; sy += u.y; sz += w.x; sp -= w.y;
    }
    const uint32_t o = a.perm[i];
    a.ax[o] = a.G * sx;
    a.ay[o] = a.G * sy;
    a.az[o] = a.G * sz;
    if (a.pot) a.pot[o] = a.G * sp;
}

// work items per leaf: ceil(#source leaves / kLeavesPerItem); slots = items * n_B
__global__ void k_items_count(TreeView t, const uint32_t* __restrict__ off, uint32_t* __restrict__ nitems,
                              uint32_t* __restrict__ nslots) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= t.nnodes) return;  // the grid's nodes; those past *dnn get no items
    uint32_t ni = 0;
    if (b < *t.dnn && t.nchild[b] == 0) {
        const uint32_t deg = off[b + 1] - off[b];
        ni = (deg + kLeavesPerItem - 1) / kLeavesPerItem;
    }
    nitems[b] = ni;
    nslots[b] = ni ? ni * (uint32_t)(t.end[b] - t.begin[b]) : 0u;
}

__global__ void k_items_fill(const int* __restrict__ dnn, const uint32_t* __restrict__ item_first,
                             int* __restrict__ item_leaf, uint32_t items_cap) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= *dnn) return;
    for (uint32_t it = item_first[b]; it < item_first[b + 1] && it < items_cap; ++it) item_leaf[it] = b;
}

// work items or partial slots past the buffers (a replayed solve whose lists
// grew): raise the capacity error and run no item
__global__ void k_check_items(uint32_t* totals, uint32_t items_cap, uint32_t slots_cap, unsigned* err) {
    if (threadIdx.x != 0) return;
    if (totals[0] > items_cap || totals[1] > slots_cap) {
        atomicOr(err, kErrCapacity);
        totals[0] = 0;
    }
}

__global__ void k_leaf_of_bodies(TreeView t, int* __restrict__ leaf_of) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *t.dnn || t.nchild[k] != 0) return;
    for (int i = t.begin[k]; i < t.end[k]; ++i) leaf_of[i] = k;
}

__global__ void k_leaf_relative(TreeView t, const double* __restrict__ xs, const double* __restrict__ ys,
                                const double* __restrict__ zs, const double* __restrict__ ms,
                                const double* __restrict__ zc, float4* __restrict__ prel) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *t.dnn || t.nchild[k] != 0) return;
    const double cx = zc[3 * k], cy = zc[3 * k + 1], cz = zc[3 * k + 2];
    for (int i = t.begin[k]; i < t.end[k]; ++i)
        prel[i] = make_float4((float)(xs[i] - cx), (float)(ys[i] - cy), (float)(zs[i] - cz), (float)ms[i]);
}

// Direct FP64 sum, one thread per target, source tiles staged in shared memory
// (1/r by the Newton-refined rsqrt above, to FP64 rounding).
__global__ void __launch_bounds__(256) k_direct(int64_t n, const double* __restrict__ x,
                                                const double* __restrict__ y,
                                                const double* __restrict__ z,
                                                const double* __restrict__ m, double G, double soft2,
                                                int64_t ntgt, const int64_t* __restrict__ tgt, double* ax,
                                                double* ay, double* az, double* pot) {
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
            const double r2 = dx * dx + dy * dy + dz * dz + soft2;  // soft2 = 0: Newtonian
            const double rinv = rsqrt_nr(r2);
            const double mr = s.w * rinv;
            const double mr3 = mr * rinv * rinv;
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

inline int blocks_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

// ---------------------------------------------------------------------------
// Jerks (the time derivative of the acceleration). With Psi = sum_j m_j /
// |x_j - x| (-phi without G), chi = sum_j m_j v_j . grad_x (1/|x_j - x|)
// (the potential of point dipoles m_j v_j) and H the Hessian of Psi,
//   j_i = G [ -grad chi(x_i) + H(x_i) v_i + near_i ],
// near_i the direct jerk over the P2P leaf pairs. The far part of chi is one
// more expansion through the same tree and lists; its gradient comes from
// l2p_hat like the acceleration. H comes from the degree-2 coefficients of
// the solve's own local expansion shifted to the body.

// Fhat_n^m for m in [-n, n] from the real layout (X^{-m} = (-1)^m conj(X^m)).
template <typename T>
__device__ __forceinline__ void fget(const T* __restrict__ F, int n, int m, T& re, T& im) {
    const int am = m < 0 ? -m : m;
    re = F[hre(n, am)];
    im = am ? F[him(n, am)] : T(0);
    if (m < 0) {
        if (am & 1) re = -re;
        else im = -im;
    }
}

// Hessian of Psi at dhat = d / s from a hat local F:
//   F_2^m(x) = (1/s^2) sum_{k, l} conj(Shat_k^l(dhat)) w_{2+k}^{m+l} / w_k^l Fhat_{2+k}^{m+l}, m = 0, 1, 2
// (the shift of the local to the body, degree 2), then
//   xx = (Re F_2^2 - F_2^0)/2, yy = -(Re F_2^2 + F_2^0)/2, zz = F_2^0,
//   xy = Im F_2^2 / 2, xz = Re F_2^1, yz = Im F_2^1.
// h = {xx, yy, zz, xy, xz, yz}.
template <typename T, typename Tab>
__device__ void l2p_hess_hat(int p, const T* __restrict__ F, T x, T y, T z, T inv_s, const Tab& tb, T* h) {
    const T r2 = x * x + y * y + z * z;
    T gr[3] = {T(0), T(0), T(0)}, gi[3] = {T(0), T(0), T(0)};
    T dre = T(1), dim = T(0);  // Shat_l^l
    for (int l = 0; l <= p - 2; ++l) {
        if (l > 0) {
            const T t = dre * x - dim * y;
            dim = dre * y + dim * x;
            dre = t;
            dre *= tb.D(l);
            dim *= tb.D(l);
        }
        T s1r = dre, s1i = dim, s2r = T(0), s2i = T(0);
        for (int k = l; k <= p - 2; ++k) {
            T sr, si;
            if (k == l) { sr = dre; si = dim; }
            else if (k == l + 1) { sr = tb.Sb(l) * z * s1r; si = tb.Sb(l) * z * s1i; }
            else {
                const T a = tb.A(k, l) * z, b = tb.B(k, l) * r2;
                sr = a * s1r - b * s2r;
                si = a * s1i - b * s2i;
            }
            if (k > l) { s2r = s1r; s2i = s1i; s1r = sr; s1i = si; }
            const T iw = tb.IW(k, l);
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                // +l: conj(S) w_{2+k}^{m+l} Fhat_{2+k}^{m+l}
                T fr, fi;
                fget(F, 2 + k, m + l, fr, fi);
                const T c = tb.W(2 + k, m + l) * iw;
                gr[m] += c * (sr * fr + si * fi);
                gi[m] += c * (sr * fi - si * fr);
                if (l > 0) {
                    // -l: conj(Shat_k^{-l}) = (-1)^l Shat_k^l, times w_{2+k}^{|m-l|} Fhat_{2+k}^{m-l}
                    fget(F, 2 + k, m - l, fr, fi);
                    const int am = m - l < 0 ? l - m : m - l;
                    const T c2 = (l & 1 ? -tb.W(2 + k, am) : tb.W(2 + k, am)) * iw;
                    gr[m] += c2 * (sr * fr - si * fi);
                    gi[m] += c2 * (sr * fi + si * fr);
                }
            }
        }
    }
    const T q = inv_s * inv_s;
    const T f20 = gr[0] * q, f21r = gr[1] * q, f21i = gi[1] * q, f22r = gr[2] * q, f22i = gi[2] * q;
    h[0] = T(0.5) * (f22r - f20);
    h[1] = T(-0.5) * (f22r + f20);
    h[2] = f20;
    h[3] = T(0.5) * f22i;
    h[4] = f21r;
    h[5] = f21i;
}

// Sorted-order jerk inputs: velocities (FP64, and an FP32 copy for the mixed
// near field) and the dipole weights m_i v_i.
__global__ void k_jerk_inputs(int n, const uint32_t* __restrict__ perm, const double* __restrict__ ms,
                              const double* __restrict__ vx, const double* __restrict__ vy,
                              const double* __restrict__ vz, double* __restrict__ vs, double* __restrict__ w,
                              float4* __restrict__ v32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t o = perm[i];
    const double a = vx[o], b = vy[o], c = vz[o], m = ms[i];
    vs[i] = a; vs[n + i] = b; vs[2 * (size_t)n + i] = c;
    w[i] = m * a; w[n + i] = m * b; w[2 * (size_t)n + i] = m * c;
    v32[i] = make_float4((float)a, (float)b, (float)c, 0.0f);
}

// Near jerk over the same bounded work items as the P2P (a target leaf and
// at most kLeavesPerItem of its source leaves, fetched dynamically): source
// positions and velocities staged per warp in shared memory, G lanes per
// target, runs of kRun terms folded into the accumulators (two-sum pairs in
// FP32), one partial per (item, body) in part_hi = (jx, jy), part_lo.x = jz.
// k_jerk_reduce adds a body's partials in item order.
template <typename T, bool SOFT>
__device__ __forceinline__ void jerk_pack(const Body4<T>* __restrict__ sm, const Body4<T>* __restrict__ su, int cnt,
                                          int sub, int G, T tx, T ty, T tz, T tvx, T tvy, T tvz, T s2,
                                          NearAcc<T>& acc) {
    for (int k0 = sub; k0 < cnt; k0 += kRun * G) {
        const int k1 = k0 + kRun * G < cnt ? k0 + kRun * G : cnt;
        T px = T(0), py = T(0), pz = T(0);
#pragma unroll 4
        for (int k = k0; k < k1; k += G) {
            const Body4<T> sv = sm[k], uv = su[k];
            const T dx = sv.x - tx, dy = sv.y - ty, dz = sv.z - tz;
            const T wx = uv.x - tvx, wy = uv.y - tvy, wz = uv.z - tvz;
            const T r2 = dx * dx + dy * dy + dz * dz;
            T rinv;
            if constexpr (sizeof(T) == 4) rinv = rsqrtf(SOFT ? r2 + s2 : r2);
            else rinv = rsqrt_nr(SOFT ? r2 + s2 : r2);
            if (!(r2 > T(0))) rinv = T(0);  // the body itself
            const T ri2 = rinv * rinv;
            const T mr3 = sv.w * rinv * ri2;
            const T c = T(3) * (dx * wx + dy * wy + dz * wz) * ri2;
            px += mr3 * (wx - c * dx);
            py += mr3 * (wy - c * dy);
            pz += mr3 * (wz - c * dz);
        }
        acc.add(px, py, pz, T(0));
    }
}

template <typename T, bool SOFT>
__global__ void __launch_bounds__(128) k_jerk_items(LeafArgs a, const double* __restrict__ vs,
                                                     const float4* __restrict__ v32, const int* __restrict__ item_leaf,
                                                     const uint32_t* __restrict__ item_first,
                                                     const uint32_t* __restrict__ slot_first,
                                                     const uint32_t* __restrict__ nitems_p,
                                                     unsigned* __restrict__ work) {
    constexpr int kCap = sizeof(T) == 8 ? kStageCap / 2 : kStageCap;  // 32 KB of staging per block
    __shared__ Body4<T> stage[4][kCap];
    __shared__ Body4<T> vstage[4][kCap];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    Body4<T>* sm = stage[wib];
    Body4<T>* su = vstage[wib];
    const int nitems = (int)*nitems_p;
    const size_t n = (size_t)a.t.n;
    const T s2 = sizeof(T) == 4 ? (T)a.soft2f : (T)a.soft2;
    for (;;) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(work, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if ((int)it >= nitems) break;
        const int B = item_leaf[it];
        const int j = (int)(it - item_first[B]);
        const uint32_t q0 = a.p2p_off[B] + (uint32_t)j * kLeavesPerItem;
        const uint32_t qe = a.p2p_off[B + 1];
        const uint32_t q1 = q0 + kLeavesPerItem < qe ? q0 + kLeavesPerItem : qe;
        const int b0 = a.t.begin[B], nB = a.t.end[B] - b0;
        const uint32_t slot0 = slot_first[B] + (uint32_t)j * (uint32_t)nB;
        const float4 bh = a.zhi[B], bl = a.zlo[B];
        for (int tc = 0; tc < nB; tc += 32) {
            const int nt = nB - tc < 32 ? nB - tc : 32;
            const int G = 32 / nt;
            const int t = lane / G, sub = lane - t * G;
            const bool act = t < nt;
            T tx = T(0), ty = T(0), tz = T(0), tvx = T(0), tvy = T(0), tvz = T(0);
            if (act) {
                const int ib = b0 + tc + t;
                if constexpr (sizeof(T) == 4) {
                    const float4 v = a.prel[ib], u = v32[ib];
                    tx = v.x; ty = v.y; tz = v.z;
                    tvx = u.x; tvy = u.y; tvz = u.z;
                } else {
                    tx = a.xs[ib]; ty = a.ys[ib]; tz = a.zs[ib];
                    tvx = vs[ib]; tvy = vs[n + ib]; tvz = vs[2 * n + ib];
                }
            }
            NearAcc<T> acc;
            uint32_t q = q0;
            int soff = 0;
            while (q < q1) {
                __syncwarp();
                int cnt = 0;
                while (q < q1) {
                    const int A = (int)a.p2p_src[q];
                    const int a0 = a.t.begin[A], nA = a.t.end[A] - a0;
                    const int rem = nA - soff;
                    int take = rem;
                    if (cnt + take > kCap) {
                        if (cnt > 0) break;
                        take = kCap;
                    }
                    float ox = 0.f, oy = 0.f, oz = 0.f;
                    if constexpr (sizeof(T) == 4) {
                        const float4 ah = a.zhi[A], al = a.zlo[A];
                        ox = (ah.x - bh.x) + (al.x - bl.x);
                        oy = (ah.y - bh.y) + (al.y - bl.y);
                        oz = (ah.z - bh.z) + (al.z - bl.z);
                    }
                    for (int l = lane; l < take; l += 32) {
                        const int jj = a0 + soff + l;
                        if constexpr (sizeof(T) == 4) {
                            const float4 u = a.prel[jj], w = v32[jj];
                            sm[cnt + l] = {u.x + ox, u.y + oy, u.z + oz, u.w};
                            su[cnt + l] = {w.x, w.y, w.z, 0.0f};
                        } else {
                            sm[cnt + l] = {a.xs[jj], a.ys[jj], a.zs[jj], a.ms[jj]};
                            su[cnt + l] = {vs[jj], vs[n + jj], vs[2 * n + jj], 0.0};
                        }
                    }
                    cnt += take;
                    if (take < rem) { soff += take; break; }
                    soff = 0;
                    ++q;
                }
                __syncwarp();
                if (act) jerk_pack<T, SOFT>(sm, su, cnt, sub, G, tx, ty, tz, tvx, tvy, tvz, s2, acc);
            }
            // combine the G sub-lanes of each target in sub-lane order
            const int leader = t * G;
            for (int s = 1; s < G; ++s) {
                const int src = leader + s < 32 ? leader + s : 31;
                if constexpr (sizeof(T) == 4) {
                    const float vx = __shfl_sync(0xffffffffu, acc.hx, src), vy = __shfl_sync(0xffffffffu, acc.hy, src),
                                vz = __shfl_sync(0xffffffffu, acc.hz, src);
                    const float wx = __shfl_sync(0xffffffffu, acc.lx, src), wy = __shfl_sync(0xffffffffu, acc.ly, src),
                                wz = __shfl_sync(0xffffffffu, acc.lz, src);
                    if (sub == 0 && act) {
                        two_sum(acc.hx, acc.lx, vx); acc.lx += wx;
                        two_sum(acc.hy, acc.ly, vy); acc.ly += wy;
                        two_sum(acc.hz, acc.lz, vz); acc.lz += wz;
                    }
                } else {
                    const double vx = __shfl_sync(0xffffffffu, acc.dx, src), vy = __shfl_sync(0xffffffffu, acc.dy, src),
                                 vz = __shfl_sync(0xffffffffu, acc.dz, src);
                    if (sub == 0 && act) { acc.dx += vx; acc.dy += vy; acc.dz += vz; }
                }
            }
            if (act && sub == 0) {
                const uint32_t slot = slot0 + (uint32_t)(tc + t);
                if constexpr (sizeof(T) == 4) {
                    a.part_hi[slot] = make_double2((double)acc.hx + (double)acc.lx, (double)acc.hy + (double)acc.ly);
                    a.part_lo[slot] = make_double2((double)acc.hz + (double)acc.lz, 0.0);
                } else {
                    a.part_hi[slot] = make_double2(acc.dx, acc.dy);
                    a.part_lo[slot] = make_double2(acc.dz, 0.0);
                }
            }
        }
    }
}

// One thread per body: -grad chi from the dipole locals and the Hessian of
// the mass locals times v_i, plus the near partials of its leaf's items in
// item order; G-scaled, to the caller's order.
template <typename T>
__global__ void __launch_bounds__(128) k_jerk_reduce(LeafArgs a, const void* __restrict__ locj,
                                                      const double* __restrict__ vs, const int* __restrict__ leaf_of,
                                                      const uint32_t* __restrict__ item_first,
                                                      const uint32_t* __restrict__ slot_first,
                                                      double* __restrict__ jx, double* __restrict__ jy,
                                                      double* __restrict__ jz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.t.n) return;
    const int n = a.t.n;
    const int B = leaf_of[i];
    const int b0 = a.t.begin[B], nB = a.t.end[B] - b0;
    const int nr = ncoef_real(a.p);
    T h[6];
    T gx, gy, gz, phi;
    if constexpr (sizeof(T) == 4) {
        const TabL32 tb;
        const float inv_s = 1.0f / a.zhi[B].w;
        const float4 v = a.prel[i];
        const float ux = v.x * inv_s, uy = v.y * inv_s, uz = v.z * inv_s;
        l2p_hat<float>(a.p, reinterpret_cast<const float*>(locj) + (size_t)nr * B, ux, uy, uz, inv_s, tb, phi, gx,
                       gy, gz);
        l2p_hess_hat<float>(a.p, reinterpret_cast<const float*>(a.loc) + (size_t)nr * B, ux, uy, uz, inv_s, tb, h);
    } else {
        const TabL64 tb{a.tb.w, a.tb.iw, a.tb.rec_a, a.tb.rec_b, a.tb.diag, a.tb.sub};
        const double inv_s = 1.0 / a.hs[B];
        const double ux = (a.xs[i] - a.zc[3 * B]) * inv_s, uy = (a.ys[i] - a.zc[3 * B + 1]) * inv_s,
                     uz = (a.zs[i] - a.zc[3 * B + 2]) * inv_s;
        l2p_hat<double>(a.p, reinterpret_cast<const double*>(locj) + (size_t)nr * B, ux, uy, uz, inv_s, tb, phi, gx,
                        gy, gz);
        l2p_hess_hat<double>(a.p, reinterpret_cast<const double*>(a.loc) + (size_t)nr * B, ux, uy, uz, inv_s, tb, h);
    }
    (void)phi;
    const double vix = vs[i], viy = vs[n + i], viz = vs[2 * (size_t)n + i];
    double fx = -(double)gx + (double)h[0] * vix + (double)h[3] * viy + (double)h[4] * viz;
    double fy = -(double)gy + (double)h[3] * vix + (double)h[1] * viy + (double)h[5] * viz;
    double fz = -(double)gz + (double)h[4] * vix + (double)h[5] * viy + (double)h[2] * viz;
    const uint32_t i0 = item_first[B], i1 = item_first[B + 1];
    const uint32_t s0 = slot_first[B] + (uint32_t)(i - b0);
    for (uint32_t it = i0; it < i1; ++it) {
        const uint32_t slot = s0 + (it - i0) * (uint32_t)nB;
        if (slot >= a.slots_cap) break;
        const double2 u = a.part_hi[slot], w = a.part_lo[slot];
        fx += u.x; fy += u.y; fz += w.x;
    }
    const uint32_t o = a.perm[i];
    jx[o] = a.G * fx;
    jy[o] = a.G * fy;
    jz[o] = a.G * fz;
}
}  // namespace

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

void leaf_items_plan(const TreeView& t, const uint32_t* p2p_off, uint32_t* item_first, uint32_t* slot_first,
                     uint32_t* totals, cudaStream_t st) {
    (k_items_count<<<blocks_for(t.nnodes, 128), 128, 0, st>>>(t, p2p_off, item_first, slot_first), note_launch());
    scan_exclusive_u32(item_first, t.nnodes, item_first + t.nnodes, st);
    scan_exclusive_u32(slot_first, t.nnodes, slot_first + t.nnodes, st);
    cudaMemcpyAsync(totals, item_first + t.nnodes, 4, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(totals + 1, slot_first + t.nnodes, 4, cudaMemcpyDeviceToDevice, st);
}

void leaf_items_check(uint32_t* totals, uint32_t items_cap, uint32_t slots_cap, unsigned* err, cudaStream_t st) {
    (k_check_items<<<1, 32, 0, st>>>(totals, items_cap, slots_cap, err), note_launch());
}

void leaf_items_fill(const TreeView& t, const uint32_t* item_first, int* item_leaf, uint32_t items_cap,
                     int* leaf_of, cudaStream_t st) {
    (k_items_fill<<<blocks_for(t.nnodes, 128), 128, 0, st>>>(t.dnn, item_first, item_leaf, items_cap), note_launch());
    (k_leaf_of_bodies<<<blocks_for(t.nnodes, 128), 128, 0, st>>>(t, leaf_of), note_launch());
}

#ifndef GBFMM_P2P_TILES
#define GBFMM_P2P_TILES 1
#endif

namespace {
// persistent grid: as many blocks as fit on every SM (warps take items from a counter)
template <typename T, bool SOFT, bool BULK>
void launch_tiles(const LeafArgs& a, const int* item_leaf, const uint32_t* item_first, const uint32_t* slot_first,
                  const uint32_t* nitems, unsigned* work, cudaStream_t st) {
    const int sh = (int)(4 * p2p_tile_smem_per_warp<T>());
    ensure_dyn_smem((const void*)k_p2p_tiles<T, SOFT, BULK>, sh);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2p_tiles<T, SOFT, BULK>, 128, sh) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    (k_p2p_tiles<T, SOFT, BULK><<<device_sm_count() * per_sm, 128, sh, st>>>(a, item_leaf, item_first, slot_first,
                                                                             nitems, work),
     note_launch());
}

template <typename T, bool SOFT>
void launch_p2p_tiles(const LeafArgs& a, const int* item_leaf, const uint32_t* item_first, const uint32_t* slot_first,
                      const uint32_t* nitems, unsigned* work, cudaStream_t st) {
    if (!GBFMM_P2P_TILES) {
        (k_p2p_lanes<T, SOFT><<<device_sm_count() * 16, 128, 0, st>>>(a, item_leaf, item_first, slot_first, nitems,
                                                                     work),
         note_launch());
        return;
    }
    if (sizeof(T) == 4 && a.bulk) launch_tiles<T, SOFT, true>(a, item_leaf, item_first, slot_first, nitems, work, st);
    else launch_tiles<T, SOFT, false>(a, item_leaf, item_first, slot_first, nitems, work, st);
}
}  // namespace

void leaf_eval(const LeafArgs& a, bool p2p32, bool l2p32, const int* item_leaf, const uint32_t* item_first,
               const uint32_t* slot_first, const uint32_t* nitems, unsigned* work, const int* leaf_of,
               cudaStream_t st) {
    cudaMemsetAsync(work, 0, sizeof(unsigned), st);
    const bool soft = a.soft2 > 0.0;
    if (p2p32) {
        if (soft) launch_p2p_tiles<float, true>(a, item_leaf, item_first, slot_first, nitems, work, st);
        else launch_p2p_tiles<float, false>(a, item_leaf, item_first, slot_first, nitems, work, st);
    } else {
        if (soft) launch_p2p_tiles<double, true>(a, item_leaf, item_first, slot_first, nitems, work, st);
        else launch_p2p_tiles<double, false>(a, item_leaf, item_first, slot_first, nitems, work, st);
    }
    const int nb = blocks_for(a.t.n, 128);
    if (l2p32) {
        switch (a.p) {
            case 4: (k_leaf_reduce<float, 4><<<nb, 128, 0, st>>>(a, leaf_of, item_first, slot_first), note_launch()); break;
            case 6: (k_leaf_reduce<float, 6><<<nb, 128, 0, st>>>(a, leaf_of, item_first, slot_first), note_launch()); break;
            case 8: (k_leaf_reduce<float, 8><<<nb, 128, 0, st>>>(a, leaf_of, item_first, slot_first), note_launch()); break;
            case 10: (k_leaf_reduce<float, 10><<<nb, 128, 0, st>>>(a, leaf_of, item_first, slot_first), note_launch()); break;
            case 12: (k_leaf_reduce<float, 12><<<nb, 128, 0, st>>>(a, leaf_of, item_first, slot_first), note_launch()); break;
            case 14: (k_leaf_reduce<float, 14><<<nb, 128, 0, st>>>(a, leaf_of, item_first, slot_first), note_launch()); break;
            default: (k_leaf_reduce<float, 0><<<nb, 128, 0, st>>>(a, leaf_of, item_first, slot_first), note_launch()); break;
        }
    } else {
        (k_leaf_reduce<double, 0><<<nb, 128, 0, st>>>(a, leaf_of, item_first, slot_first), note_launch());
    }
}

void jerk_inputs(int n, const uint32_t* perm, const double* ms, const double* vx, const double* vy,
                 const double* vz, double* vs, double* w, float4* v32, cudaStream_t st) {
    if (n > 0) (k_jerk_inputs<<<blocks_for(n, 256), 256, 0, st>>>(n, perm, ms, vx, vy, vz, vs, w, v32), note_launch());
}

void jerk_leaves(const LeafArgs& a, bool fp32, const void* locj, const double* vs, const float4* v32,
                 const int* item_leaf, const uint32_t* item_first, const uint32_t* slot_first, const uint32_t* nitems,
                 unsigned* work, const int* leaf_of, double* jx, double* jy, double* jz, cudaStream_t st) {
    cudaMemsetAsync(work, 0, sizeof(unsigned), st);
    const bool soft = a.soft2 > 0.0;
    if (fp32) {
        if (soft) (k_jerk_items<float, true><<<device_sm_count() * 16, 128, 0, st>>>(a, vs, v32, item_leaf, item_first, slot_first, nitems, work), note_launch());
        else (k_jerk_items<float, false><<<device_sm_count() * 16, 128, 0, st>>>(a, vs, v32, item_leaf, item_first, slot_first, nitems, work), note_launch());
        (k_jerk_reduce<float><<<blocks_for(a.t.n, 128), 128, 0, st>>>(a, locj, vs, leaf_of, item_first, slot_first, jx, jy, jz), note_launch());
    } else {
        if (soft) (k_jerk_items<double, true><<<device_sm_count() * 16, 128, 0, st>>>(a, vs, v32, item_leaf, item_first, slot_first, nitems, work), note_launch());
        else (k_jerk_items<double, false><<<device_sm_count() * 16, 128, 0, st>>>(a, vs, v32, item_leaf, item_first, slot_first, nitems, work), note_launch());
        (k_jerk_reduce<double><<<blocks_for(a.t.n, 128), 128, 0, st>>>(a, locj, vs, leaf_of, item_first, slot_first, jx, jy, jz), note_launch());
    }
}

void leaf_relative_f32(const TreeView& t, const double* xs, const double* ys, const double* zs,
                       const double* ms, const double* zc, float4* prel, cudaStream_t st) {
    (k_leaf_relative<<<blocks_for(t.nnodes, 128), 128, 0, st>>>(t, xs, ys, zs, ms, zc, prel), note_launch());
}

void direct_sum_f64(int64_t n, const double* x, const double* y, const double* z, const double* m,
                    double G, double soft, int64_t ntgt, const int64_t* tgt, double* ax, double* ay, double* az,
                    double* pot, cudaStream_t st) {
    if (ntgt > 0)
        (k_direct<<<blocks_for(ntgt, 256), 256, 0, st>>>(n, x, y, z, m, G, soft * soft, ntgt, tgt, ax, ay, az, pot),
         note_launch());
}

}  // namespace gbfmm
