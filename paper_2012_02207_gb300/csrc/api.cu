// C ABI of the gbfmm library: context, workspace and the solve pipeline.
//
// One solve (Sec. 2.1, Fig. 1 of Mukherjee et al. 2021):
//   bounding cube -> Morton keys -> radix sort -> octree -> cell geometry
//   -> P2M / M2M (FP64 hat multipoles) and degree norms P_n
//   -> theta < 1 walk -> scalar-force estimate f (Sec. 2.3)
//   -> error-controlled walk -> M2L (rotation, Sec. 2.4) -> L2L
//   -> per leaf: L2P + P2P, written to the caller's order.
// The host reads back three small things (node count, level starts, list
// sizes); everything else stays on the device.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "gbfmm_internal.cuh"
#include "swap_table.inc"

namespace gbfmm {
namespace {
thread_local int64_t g_launches = 0;
constexpr int kMaxDevices = 64;
std::mutex g_dev_mu;
int g_sm_count[kMaxDevices] = {};
std::vector<std::pair<const void*, int>> g_smem_set[kMaxDevices];  // (function, bytes) set per device
int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return 0;
    }
    return dev;
}
}  // namespace
void note_launch() { ++g_launches; }

int device_sm_count() {
    const int dev = current_device();
    std::lock_guard<std::mutex> lock(g_dev_mu);
    if (g_sm_count[dev] == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
            cudaGetLastError();
            sms = 1;  // a launch then still covers the work (grid-stride loops), only slower
        }
        g_sm_count[dev] = sms;
    }
    return g_sm_count[dev];
}

cudaError_t ensure_dyn_smem(const void* func, int bytes) {
    const int dev = current_device();
    std::lock_guard<std::mutex> lock(g_dev_mu);
    for (auto& e : g_smem_set[dev])
        if (e.first == func) {
            if (e.second >= bytes) return cudaSuccess;
            const cudaError_t rc = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (rc == cudaSuccess) e.second = bytes;
            return rc;
        }
    const cudaError_t rc = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (rc == cudaSuccess) g_smem_set[dev].emplace_back(func, bytes);
    return rc;
}
bool m2l32_supported(int p);
void tree_build_count(TreeBuffers& b, int* sorted_in_1, cudaStream_t st);
void tree_build_emit(TreeBuffers& b, cudaStream_t st);
}  // namespace gbfmm

using namespace gbfmm;

namespace {

std::string g_create_error = "no error";

struct Buf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

template <typename T>
T* as(Buf& b) { return reinterpret_cast<T*>(b.ptr); }

}  // namespace

namespace gbfmm {
// message returned by fmm_last_error(NULL) (also used by the no-allocation entry point)
void set_global_error(const char* msg) { g_create_error = msg; }
}  // namespace gbfmm

// A captured solve (fmm_solve_graph): the capacities it was captured for,
// taken from an ordinary solve of the same problem with headroom, and the
// arguments its launches are bound to.
struct GraphPlan {
    bool valid = false;
    int64_t n = 0;
    std::vector<int64_t> offs;
    const void* ptrs[8] = {};
    cudaStream_t st = nullptr;
    int64_t gen = -1;                     // buffer generation it was captured with
    int node_cap = 0, nlevels = 0, nroots = 0, nb = 1;
    int lvl_cap[kMaxLevel + 2] = {};
    int walk_iters[2] = {0, 0};
    int64_t pair_cap[4] = {0, 0, 0, 0};
    uint32_t items_cap = 0, slots_cap = 0;
    int* h_coff = nullptr;                // pinned copy of the cluster offsets (a memcpy node)
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
};

struct fmm_ctx {
    fmm_config cfg{};
    int device = 0;
    std::string err = "no error";
    fmm_stats stats{};
    HostTables ht{};
    DevTables tb{};
    Buf tables, tables_dw;
    DevScalars* ds = nullptr;
    DevScalars* h_ds = nullptr;  // pinned
    cudaEvent_t ev[10] = {};
    // per-body
    Buf k0, k1, v0, v1, hist, xs, ys, zs, ms, xf, prel, lcp, win, hi, chunk, f, bbox;
    // clusters of a forest (an ensemble solve)
    Buf coff, box, ck0, ck1, cv0, cv1, cid;
    std::vector<int> h_coff;
    // per-node
    Buf level, begin, end, parent, first_child, nchild, M, S, zc, r, hs, Pk, mult, mult32, loc, loc32,
        fmin, fscratch, zhi, zlo, contrib, Phat, r32;
    // P2P work items
    Buf item_first, slot_first, item_leaf, leaf_of, part_hi, part_lo, work;
    // jerks: sorted velocities (FP64, FP32), dipole weights, order p-1 moments,
    // dipole multipoles and locals (FP64 and FP32)
    Buf jv, jv32, jw, jmom, jmult, jmult32, jloc, jloc32;
    // HOLD integrator: all-body list, compact gathers, accelerations, step
    // sizes, split flags and scan, the fast count; per-depth slow/fast lists
    Buf h_all, h_gat, h_acc, h_acc2, h_tau, h_flag, h_scan, h_scr, h_nf;
    std::vector<Buf> h_S, h_F;
    // walk and lists
    // per list: sorted directed keys, the sort's second buffer (its own, so a
    // buffer never moves to a list of another size), CSR offsets
    Buf front0, front1, lists[4], dkeys[4], dalt[4], dsrc[4], doff[4], dcount, geo;
    Buf walk_scan;  // look-back records of the walk's ordered appends (zeroed when allocated)
    int64_t front_cap = 0, list_cap[4] = {0, 0, 0, 0};
    // host staging for fmm_solve_host
    Buf hin[4], hout[4];
    // last solve
    int64_t n = 0;
    int nnodes = 0, nlevels = 0, nb = 1, sorted_in_1 = 0, nclusters = 1;
    int h_level_start[kMaxLevel + 3] = {};
    int64_t npairs[4] = {0, 0, 0, 0}, ndirected[4] = {0, 0, 0, 0};
    int dk_in_alt[4] = {0, 0, 0, 0};
    // workspace generation: bumped by every reallocation (a captured graph
    // holds the old addresses and must be captured again)
    int64_t gen = 0;
    GraphPlan plan;
    const GraphPlan* gmode = nullptr;     // set while the solve runs in graph form
    cudaStream_t gstream = nullptr;       // stream of the captured solve (capture needs a non-default one)
    int walk_steps[2] = {0, 0};           // steps of the last ordinary solve's walks
    uint32_t items_total[2] = {0, 0};     // and its P2P work items and partial slots
    cudaEvent_t gev[2] = {nullptr, nullptr};
};

void drop_plan(GraphPlan& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.h_coff) cudaFreeHost(g.h_coff);
    g = GraphPlan{};
}

namespace {

int fail(fmm_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, FMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int ensure(fmm_ctx* ctx, Buf& b, size_t bytes) {
    if (b.bytes >= bytes) return FMM_OK;
    ctx->gen++;
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    size_t want = bytes + bytes / 4 + 256;
    if (cudaMalloc(&b.ptr, want) != cudaSuccess) {
        cudaGetLastError();
        b.ptr = nullptr;
        return fail(ctx, FMM_ERR_OOM, "device allocation of " + std::to_string(want) + " bytes failed");
    }
    b.bytes = want;
    return FMM_OK;
}

// ensure, and zero the buffer whenever it is (re)allocated
int ensure_zeroed(fmm_ctx* ctx, Buf& b, size_t bytes, cudaStream_t st) {
    const void* old = b.ptr;
    int rc = ensure(ctx, b, bytes);
    if (rc != FMM_OK) return rc;
    if (b.ptr != old && cudaMemsetAsync(b.ptr, 0, b.bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, FMM_ERR_CUDA, "clearing the walk's look-back records failed");
    }
    return FMM_OK;
}

int ensure_walk_scan(fmm_ctx* ctx, WalkBuffers& wb, cudaStream_t st) {
    wb.stall_lookback = (ctx->cfg.fault_inject & 4u) ? 1 : 0;
    const int64_t tiles = walk_scan_tiles(ctx->front_cap);
    const int rc = ensure_zeroed(ctx, ctx->walk_scan, sizeof(unsigned long long) * kWalkScanWords * (size_t)tiles, st);
    if (rc != FMM_OK) return rc;
    wb.scan = as<unsigned long long>(ctx->walk_scan);
    // the records' stride is fixed by the capacity they were sized for
    wb.scan_tiles = (int64_t)(ctx->walk_scan.bytes / (sizeof(unsigned long long) * kWalkScanWords));
    return FMM_OK;
}

void release(Buf& b) {
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
}

void build_host_tables(HostTables& h) {
    h.fact[0] = 1.0;
    for (int k = 1; k < 2 * kMaxP + 4; ++k) h.fact[k] = h.fact[k - 1] * (double)k;
    for (int n = 0; n < kMaxP + 2; ++n)
        for (int m = 0; m < kMaxP + 2; ++m) {
            if (m <= n) {
                h.w[n][m] = std::sqrt(h.fact[n + m] * h.fact[n - m]);
                h.iw[n][m] = 1.0 / h.w[n][m];
            } else {
                h.w[n][m] = 0.0;
                h.iw[n][m] = 0.0;
            }
        }
    for (int n = 0; n <= kMaxP; ++n) {
        h.binom[n][0] = 1.0;
        h.binom[n][n] = 1.0;
        for (int k = 1; k < n; ++k) h.binom[n][k] = h.binom[n - 1][k - 1] + h.binom[n - 1][k];
        for (int m = 0; m <= kMaxP; ++m) {
            if (m < n - 1 || (m == n - 1 && n >= 1)) {
                const double a = (double)(n + m), b = (double)(n - m);
                h.rec_a[n][m] = (2.0 * n - 1.0) / std::sqrt(a * b);
                h.rec_b[n][m] = (n - m >= 2) ? std::sqrt((a - 1.0) * (b - 1.0) / (a * b)) : 0.0;
            } else {
                h.rec_a[n][m] = 0.0;
                h.rec_b[n][m] = 0.0;
            }
        }
        h.diag[n] = n == 0 ? 1.0 : std::sqrt((2.0 * n - 1.0) / (2.0 * n));
        h.sub[n] = std::sqrt(2.0 * n + 1.0);
    }
}

int bit_length(int64_t v) {
    int b = 0;
    while (v > 0) { ++b; v >>= 1; }
    return b;
}

TreeView view(fmm_ctx* ctx) {
    TreeView t;
    t.n = (int)ctx->n;
    t.nnodes = ctx->nnodes;
    t.nlevels = ctx->nlevels;
    t.leaf_size = ctx->cfg.leaf_size;
    t.level = as<int>(ctx->level);
    t.begin = as<int>(ctx->begin);
    t.end = as<int>(ctx->end);
    t.parent = as<int>(ctx->parent);
    t.first_child = as<int>(ctx->first_child);
    t.nchild = as<int>(ctx->nchild);
    t.nroots = ctx->nnodes > 0 ? ctx->h_level_start[1] : 0;
    for (int L = 0; L <= kMaxLevel; ++L)
        t.lvl_cnt[L] = ctx->nnodes > 0 ? ctx->h_level_start[L + 1] - ctx->h_level_start[L] : 0;
    t.lvl_cnt[kMaxLevel + 1] = 0;
    if (const GraphPlan* g = ctx->gmode) {  // grids sized by the planned capacities
        t.nroots = g->nroots;
        for (int L = 0; L <= kMaxLevel + 1; ++L) t.lvl_cnt[L] = g->lvl_cap[L];
    }
    t.dnn = &ctx->ds->nnodes;
    t.dls = ctx->ds->level_start;
    return t;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

// directed, sorted, CSR-indexed form of pair list `which`: every unordered
// pair (A, B) gives the keys B<<nb|A and A<<nb|B; a self pair gives one key
// and an all-ones marker that sorts last and is ignored. The key count lives on
// the device (dcount[8 + which]): a captured solve sizes the grids for its
// planned capacity but sorts only the keys present.
int build_directed(fmm_ctx* ctx, int which, cudaStream_t st) {
    const int64_t np = ctx->npairs[which];
    const size_t keys_bytes = sizeof(uint64_t) * (size_t)(2 * np + 1);
    int rc;
    if ((rc = ensure(ctx, ctx->dkeys[which], keys_bytes)) != FMM_OK) return rc;
    if ((rc = ensure(ctx, ctx->dalt[which], keys_bytes)) != FMM_OK) return rc;
    if ((rc = ensure(ctx, ctx->doff[which], sizeof(uint32_t) * (size_t)(ctx->nnodes + 2))) != FMM_OK) return rc;
    if ((rc = ensure(ctx, ctx->dsrc[which], sizeof(uint32_t) * (size_t)(2 * np + 1))) != FMM_OK) return rc;
    if ((rc = ensure(ctx, ctx->hist, sizeof(uint32_t) * radix_hist_words(2 * np + 1))) != FMM_OK) return rc;
    ctx->ndirected[which] = 2 * np;
    unsigned long long* nkeys = as<unsigned long long>(ctx->dcount) + 8 + which;
    // The error-controlled walk's lists (M2L, P2P) come out of the walk in a
    // fixed order: sorting by target alone keeps that order within a target.
    // The theta-walk's lists are sorted by (target, source), the order the
    // scalar estimate sums in.
    const int lo_bit = which >= 2 ? ctx->nb : 0;
    if (2 * ctx->nb <= 32) {
        // 32-bit keys: half the bytes per radix pass; both ping-pong halves fit in dalt
        uint32_t* ka = as<uint32_t>(ctx->dalt[which]);
        uint32_t* kb = ka + (2 * np + 1);
        pairs_to_directed32(as<int2>(ctx->lists[which]), ctx->ds->list_cnt + which, np, ctx->nb, ka,
                            as<unsigned long long>(ctx->dcount) + 2 + which, nkeys, st);
        const int in1 = radix_sort32(ka, kb, 2 * np, 2 * ctx->nb, as<uint32_t>(ctx->hist), st, nkeys, lo_bit);
        directed_offsets_src32(in1 ? kb : ka, 2 * np, nkeys, ctx->nb, &ctx->ds->nnodes,
                               as<uint32_t>(ctx->dsrc[which]), as<uint32_t>(ctx->doff[which]), st);
        return FMM_OK;
    }
    pairs_to_directed(as<int2>(ctx->lists[which]), ctx->ds->list_cnt + which, np, ctx->nb,
                      as<uint64_t>(ctx->dkeys[which]), as<unsigned long long>(ctx->dcount) + 2 + which, nkeys, st);
    const int in1 = radix_sort(as<uint64_t>(ctx->dkeys[which]), nullptr, as<uint64_t>(ctx->dalt[which]), nullptr,
                               2 * np, 2 * ctx->nb, as<uint32_t>(ctx->hist), st, nkeys, lo_bit);
    directed_offsets(as<uint64_t>(in1 ? ctx->dalt[which] : ctx->dkeys[which]), 2 * np, nkeys, ctx->nb,
                     &ctx->ds->nnodes, as<uint32_t>(ctx->dsrc[which]), as<uint32_t>(ctx->doff[which]), st);
    return FMM_OK;
}

int run_walk(fmm_ctx* ctx, int mode, cudaStream_t st) {
    TreeView t = view(ctx);
    const int p = ctx->cfg.p;
    const double* binom_row0 = ctx->tb.sub + (kMaxP + 1);
    if (const GraphPlan* g = ctx->gmode) {
        // graph form: planned capacities and steps, no read-back; overflows and
        // an unfinished walk raise kErrCapacity for the check after the replay
        int rc;
        if ((rc = ensure(ctx, ctx->front0, sizeof(int2) * (size_t)ctx->front_cap)) != FMM_OK) return rc;
        if ((rc = ensure(ctx, ctx->front1, sizeof(int2) * (size_t)ctx->front_cap)) != FMM_OK) return rc;
        WalkBuffers wb;
        wb.front0 = as<int2>(ctx->front0);
        wb.front1 = as<int2>(ctx->front1);
        wb.front_cap = ctx->front_cap;
        for (int l = 0; l < 4; ++l) {
            wb.out[l] = as<int2>(ctx->lists[l]);
            wb.out_cap[l] = g->pair_cap[l];
        }
        if ((rc = ensure_walk_scan(ctx, wb, st)) != FMM_OK) return rc;
        for (int l = 2 * mode; l < 2 * mode + 2; ++l) {
            if ((rc = ensure(ctx, ctx->lists[l], sizeof(int2) * (size_t)g->pair_cap[l])) != FMM_OK) return rc;
            wb.out[l] = as<int2>(ctx->lists[l]);
            ctx->npairs[l] = g->pair_cap[l];
        }
        dual_tree_walk(mode, t, as<double>(ctx->zc), as<double>(ctx->r), as<double>(ctx->Pk),
                       as<float>(ctx->fmin), p, ctx->cfg.eps, binom_row0, as<float4>(ctx->zhi),
                       as<float4>(ctx->zlo), as<float>(ctx->r32), as<float>(ctx->Phat), as<double>(ctx->M),
                       ctx->cfg.soft, wb, ctx->ds, ctx->h_ds, g->walk_iters[mode], st);
        walk_check_finished(ctx->ds, g->walk_iters[mode], st);
        CK(cudaGetLastError());
        return FMM_OK;
    }
    for (int attempt = 0; attempt < 12; ++attempt) {
        int rc;
        if ((rc = ensure(ctx, ctx->front0, sizeof(int2) * (size_t)ctx->front_cap)) != FMM_OK) return rc;
        if ((rc = ensure(ctx, ctx->front1, sizeof(int2) * (size_t)ctx->front_cap)) != FMM_OK) return rc;
        for (int l = 2 * mode; l < 2 * mode + 2; ++l)
            if ((rc = ensure(ctx, ctx->lists[l], sizeof(int2) * (size_t)ctx->list_cap[l])) != FMM_OK) return rc;
        WalkBuffers wb;
        wb.front0 = as<int2>(ctx->front0);
        wb.front1 = as<int2>(ctx->front1);
        wb.front_cap = ctx->front_cap;
        for (int l = 0; l < 4; ++l) {
            wb.out[l] = as<int2>(ctx->lists[l]);
            wb.out_cap[l] = ctx->list_cap[l];
        }
        if ((rc = ensure_walk_scan(ctx, wb, st)) != FMM_OK) return rc;
        // the binomial row C(p, k) follows the sub-diagonal table (see fmm_create)
        const double* binom_row = ctx->tb.sub + (kMaxP + 1);
        CK(cudaMemsetAsync(&ctx->ds->err, 0, sizeof(unsigned), st));
        const int it = dual_tree_walk(mode, t, as<double>(ctx->zc), as<double>(ctx->r), as<double>(ctx->Pk),
                                      as<float>(ctx->fmin), p, ctx->cfg.eps, binom_row, as<float4>(ctx->zhi),
                                      as<float4>(ctx->zlo), as<float>(ctx->r32), as<float>(ctx->Phat),
                                      as<double>(ctx->M), ctx->cfg.soft, wb, ctx->ds, ctx->h_ds, 0, st);
        if (it == FMM_ERR_CAPACITY) {
            // the counters kept counting past the capacity: grow to what was asked for
            CK(cudaMemcpyAsync(ctx->h_ds, ctx->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            unsigned long long fmax = 0;
            for (int i = 0; i < kMaxWalkIters + 2; ++i) fmax = ctx->h_ds->cnt[i] > fmax ? ctx->h_ds->cnt[i] : fmax;
            ctx->front_cap = std::max<int64_t>(4 * ctx->front_cap, 2 * (int64_t)fmax);
            for (int l = 2 * mode; l < 2 * mode + 2; ++l)
                ctx->list_cap[l] = std::max<int64_t>(4 * ctx->list_cap[l], 2 * (int64_t)ctx->h_ds->list_cnt[l]);
            ctx->stats.regrows++;
            continue;
        }
        if (it == kWalkBadIndex) return fail(ctx, FMM_ERR_CUDA, "dual-tree walk read an out-of-range cell index");
        if (it == FMM_ERR_TIMEOUT) return fail(ctx, it, "a bounded wait of the walk's ordered appends ran out");
        if (it == FMM_ERR_CUDA)
            return fail(ctx, it, std::string("dual-tree walk failed: ") + cudaGetErrorString(cudaGetLastError()));
        if (it < 0) return fail(ctx, it, "dual-tree walk failed");
        ctx->stats.walk_iters += it;
        ctx->walk_steps[mode] = it;
        unsigned long long cnt[4];
        CK(cudaMemcpyAsync(cnt, ctx->ds->list_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        bool over = false;
        for (int l = 2 * mode; l < 2 * mode + 2; ++l) {
            if ((int64_t)cnt[l] > ctx->list_cap[l]) over = true;
            ctx->npairs[l] = (int64_t)cnt[l];
        }
        if (over) {
            for (int l = 2 * mode; l < 2 * mode + 2; ++l)
                while (ctx->list_cap[l] < ctx->npairs[l]) ctx->list_cap[l] *= 2;
            ctx->stats.regrows++;
            continue;
        }
        return FMM_OK;
    }
    return fail(ctx, FMM_ERR_CAPACITY, "interaction lists outgrew their capacity");
}

// One pipeline pass over a forest of nclusters independent clusters (bodies
// offsets[c] .. offsets[c+1]-1 of cluster c; offsets == nullptr: one cluster).
int solve_device(fmm_ctx* ctx, int64_t n, int nclusters, const int64_t* offsets, const double* x,
                 const double* y, const double* z, const double* m, double* ax, double* ay, double* az,
                 double* pot, cudaStream_t st) {
    const int p = ctx->cfg.p;
    const bool mixed = ctx->cfg.precision == FMM_PRECISION_MIXED;
    // FP32 far field (M2L, L2L, L2P on hat FP32 coefficients) unless the flag asks for FP64 locals
    const bool far32 = mixed && !(ctx->cfg.flags & FMM_FLAG_FP64_LOCALS);
    const GraphPlan* gp = ctx->gmode;  // non-null: the graph form (planned sizes, no read-back)
    // phase events; while capturing they become event-record nodes (the external
    // flag is only accepted then), so a replay times its phases too
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (gp) CK(cudaStreamIsCapturing(st, &cap));
    const unsigned ev_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    auto rec = [&](int i) { return cudaEventRecordWithFlags(ctx->ev[i], st, ev_flags); };
    std::memset(&ctx->stats, 0, sizeof(ctx->stats));
    g_launches = 0;
    ctx->stats.n = n;
    ctx->n = n;
    ctx->nnodes = 0;
    if (n == 0) return FMM_OK;
    int rc;
    if (!offsets) nclusters = 1;
    ctx->nclusters = nclusters;
    ctx->h_coff.resize((size_t)nclusters + 1);
    for (int c = 0; c <= nclusters; ++c) ctx->h_coff[c] = offsets ? (int)offsets[c] : (c ? (int)n : 0);
    // ---- per-body workspace
    const size_t N = (size_t)n;
    const int nchunks = tree_nchunks(n);
    if ((rc = ensure(ctx, ctx->k0, 8 * N)) || (rc = ensure(ctx, ctx->k1, 8 * N)) ||
        (rc = ensure(ctx, ctx->v0, 4 * N)) || (rc = ensure(ctx, ctx->v1, 4 * N)) ||
        (rc = ensure(ctx, ctx->hist, 4 * radix_hist_words(n))) || (rc = ensure(ctx, ctx->xs, 8 * N)) ||
        (rc = ensure(ctx, ctx->ys, 8 * N)) || (rc = ensure(ctx, ctx->zs, 8 * N)) ||
        (rc = ensure(ctx, ctx->ms, 8 * N)) || (rc = ensure(ctx, ctx->xf, 16 * N)) ||
        (rc = ensure(ctx, ctx->prel, 16 * N)) || (rc = ensure(ctx, ctx->lcp, N)) ||
        (rc = ensure(ctx, ctx->win, N)) || (rc = ensure(ctx, ctx->hi, N)) ||
        (rc = ensure(ctx, ctx->chunk, 4 * ((size_t)(kMaxLevel + 1) * nchunks + 2))) ||
        (rc = ensure(ctx, ctx->f, 4 * N)) || (rc = ensure(ctx, ctx->bbox, 8 * 6 * (size_t)bbox_partials(nclusters))) ||
        (rc = ensure(ctx, ctx->coff, 4 * ((size_t)nclusters + 1))) || (rc = ensure(ctx, ctx->box, 64 * (size_t)nclusters)))
        return rc;
    if (nclusters > 1 &&
        ((rc = ensure(ctx, ctx->ck0, 8 * N)) || (rc = ensure(ctx, ctx->ck1, 8 * N)) ||
         (rc = ensure(ctx, ctx->cv0, 4 * N)) || (rc = ensure(ctx, ctx->cv1, 4 * N)) ||
         (rc = ensure(ctx, ctx->cid, 4 * N))))
        return rc;
    CK(rec(0));
    CK(cudaMemsetAsync(&ctx->ds->err, 0, sizeof(unsigned), st));
    CK(cudaMemcpyAsync(ctx->coff.ptr, gp ? gp->h_coff : ctx->h_coff.data(), 4 * ((size_t)nclusters + 1),
                       cudaMemcpyHostToDevice, st));
    TreeBuffers tb{};
    tb.x = x; tb.y = y; tb.z = z; tb.m = m; tb.n = n; tb.leaf_size = ctx->cfg.leaf_size;
    tb.nclusters = nclusters; tb.coff = as<int>(ctx->coff); tb.box = as<double>(ctx->box);
    tb.ck0 = as<uint64_t>(ctx->ck0); tb.ck1 = as<uint64_t>(ctx->ck1);
    tb.cv0 = as<uint32_t>(ctx->cv0); tb.cv1 = as<uint32_t>(ctx->cv1); tb.cid = as<uint32_t>(ctx->cid);
    tb.bbox_part = as<double>(ctx->bbox);
    tb.k0 = as<uint64_t>(ctx->k0); tb.k1 = as<uint64_t>(ctx->k1);
    tb.v0 = as<uint32_t>(ctx->v0); tb.v1 = as<uint32_t>(ctx->v1);
    tb.hist = as<uint32_t>(ctx->hist);
    tb.xs = as<double>(ctx->xs); tb.ys = as<double>(ctx->ys); tb.zs = as<double>(ctx->zs);
    tb.ms = as<double>(ctx->ms); tb.xf = as<float4>(ctx->xf);
    tb.lcp = as<int8_t>(ctx->lcp); tb.win = as<int8_t>(ctx->win); tb.hi = as<uint8_t>(ctx->hi);
    tb.chunk_cnt = as<uint32_t>(ctx->chunk);
    tb.ds = ctx->ds;
    int in1 = 0;
    tree_build_count(tb, &in1, st);
    ctx->sorted_in_1 = in1;
    uint32_t total = 0;
    unsigned err = 0;
    if (gp) {
        total = (uint32_t)gp->node_cap;
    } else {
        CK(cudaMemcpyAsync(&total, as<uint32_t>(ctx->chunk) + (size_t)(kMaxLevel + 1) * nchunks, 4,
                           cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&err, &ctx->ds->err, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (err & kErrNonfinite) return fail(ctx, FMM_ERR_NONFINITE, "non-finite position or mass, or a mass <= 0");
        if (err & kErrCoincident) return fail(ctx, FMM_ERR_COINCIDENT, "two bodies share the same position");
        if (err & kErrLongRun) {
            // a run of equal keys longer than the bounded scan: check every body exactly
            // (the cluster pass's sort buffers are free again here)
            if ((rc = ensure(ctx, ctx->ck0, 8 * N)) || (rc = ensure(ctx, ctx->ck1, 8 * N)) ||
                (rc = ensure(ctx, ctx->cv0, 4 * N)) || (rc = ensure(ctx, ctx->cv1, 4 * N)))
                return rc;
            coincident_exact(tb, as<uint64_t>(ctx->ck0), as<uint32_t>(ctx->cv0), as<uint64_t>(ctx->ck1),
                             as<uint32_t>(ctx->cv1), st);
            CK(cudaMemcpyAsync(&err, &ctx->ds->err, 4, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (err & kErrCoincident) return fail(ctx, FMM_ERR_COINCIDENT, "two bodies share the same position");
            CK(cudaMemsetAsync(&ctx->ds->err, 0, sizeof(unsigned), st));
        }
    }
    const int nnodes = (int)total;  // the node arrays' size (the planned capacity in graph form)
    ctx->nnodes = nnodes;
    const size_t K = (size_t)nnodes;
    const size_t nr = (size_t)ncoef_real(p);
    if ((rc = ensure(ctx, ctx->level, 4 * K)) || (rc = ensure(ctx, ctx->begin, 4 * K)) ||
        (rc = ensure(ctx, ctx->end, 4 * K)) || (rc = ensure(ctx, ctx->parent, 4 * K)) ||
        (rc = ensure(ctx, ctx->first_child, 4 * K)) || (rc = ensure(ctx, ctx->nchild, 4 * K)) ||
        (rc = ensure(ctx, ctx->M, 8 * K)) || (rc = ensure(ctx, ctx->S, 24 * K)) ||
        (rc = ensure(ctx, ctx->zc, 24 * K)) || (rc = ensure(ctx, ctx->r, 8 * K)) || (rc = ensure(ctx, ctx->hs, 8 * K)) ||
        (rc = ensure(ctx, ctx->Pk, 8 * K * (p + 1))) || (rc = ensure(ctx, ctx->mult, 8 * K * nr)) ||
        (rc = ensure(ctx, ctx->fmin, 4 * K)) || (rc = ensure(ctx, ctx->fscratch, 4 * (2 * K + N))) ||
        (rc = ensure(ctx, ctx->zhi, 16 * K)) || (rc = ensure(ctx, ctx->zlo, 16 * K)) ||
        (rc = ensure(ctx, ctx->contrib, 8 * K * nr)) || (rc = ensure(ctx, ctx->Phat, 4 * K * (p + 1))) ||
        (rc = ensure(ctx, ctx->r32, 4 * K)) || (rc = ensure(ctx, ctx->geo, sizeof(double) * kShiftGeo * K)) ||
        (rc = ensure(ctx, ctx->item_first, 4 * (K + 2))) || (rc = ensure(ctx, ctx->slot_first, 4 * (K + 2))) ||
        (rc = ensure(ctx, ctx->leaf_of, 4 * N)) || (rc = ensure(ctx, ctx->work, 64)))
        return rc;
    if (far32) {
        if ((rc = ensure(ctx, ctx->mult32, 4 * K * ((nr + 3) & ~(size_t)3))) || (rc = ensure(ctx, ctx->loc32, 4 * K * nr)))
            return rc;
        if (!m2l32_supported(p) && (rc = ensure(ctx, ctx->loc, 8 * K * nr))) return rc;
    } else {
        if ((rc = ensure(ctx, ctx->loc, 8 * K * nr))) return rc;
    }
    tb.level = as<int>(ctx->level); tb.begin = as<int>(ctx->begin); tb.end = as<int>(ctx->end);
    tb.parent = as<int>(ctx->parent); tb.first_child = as<int>(ctx->first_child);
    tb.nchild = as<int>(ctx->nchild); tb.node_cap = nnodes;
    tree_build_emit(tb, st);
    int nl = 1;
    if (gp) {
        nl = gp->nlevels;
        ctx->nb = gp->nb;
    } else {
        CK(cudaMemcpyAsync(ctx->h_ds, ctx->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        std::memcpy(ctx->h_level_start, ctx->h_ds->level_start, sizeof(ctx->h_level_start));
        for (int L = 1; L <= kMaxLevel; ++L)
            if (ctx->h_level_start[L] < nnodes) nl = L + 1;
        ctx->nb = bit_length(nnodes);
    }
    ctx->nlevels = nl;
    TreeView t = view(ctx);
    const uint64_t* keys = as<uint64_t>(in1 ? ctx->k1 : ctx->k0);
    tree_build_phase2(tb, keys, nnodes, ctx->h_level_start, nl, st);
    cell_geometry(t, as<double>(ctx->xs), as<double>(ctx->ys), as<double>(ctx->zs), as<double>(ctx->ms),
                  ctx->h_level_start, as<double>(ctx->M), as<double>(ctx->S), as<double>(ctx->zc),
                  as<double>(ctx->r), st);
    hat_scales(t, as<int>(ctx->parent), as<double>(ctx->r), as<double>(ctx->hs), st);
    shift_geometry(t, as<double>(ctx->zc), as<double>(ctx->hs), as<double>(ctx->geo), st);
    node_centres_f32(t, as<double>(ctx->zc), as<double>(ctx->hs), as<float4>(ctx->zhi), as<float4>(ctx->zlo), st);
    CK(rec(1));
    // ---- upward pass
    upward_pass(t, ctx->h_level_start, p, as<double>(ctx->xs), as<double>(ctx->ys), as<double>(ctx->zs),
                as<double>(ctx->ms), as<double>(ctx->zc), as<double>(ctx->r), as<double>(ctx->hs),
                as<double>(ctx->geo), as<double>(ctx->mult), as<double>(ctx->Pk), as<float>(ctx->Phat), as<float>(ctx->r32), as<double>(ctx->contrib), ctx->tb,
                mixed, st);
    CK(rec(2));
    // ---- scalar-force estimate
    if (ctx->front_cap == 0) {
        const int64_t base = 64 * (int64_t)nnodes + 4096;
        ctx->front_cap = base;
        ctx->list_cap[0] = ctx->list_cap[1] = base;
        ctx->list_cap[2] = ctx->list_cap[3] = 4 * base;
        if (ctx->cfg.fault_inject & 1u) {
            ctx->front_cap = 16;
            for (int l = 0; l < 4; ++l) ctx->list_cap[l] = 16;
        }
    }
    if ((rc = ensure(ctx, ctx->dcount, 128))) return rc;  // [1] P2P interactions, [2..5] self pairs, [8..11] keys
    CK(cudaMemsetAsync(ctx->dcount.ptr, 0, 128, st));
    if ((rc = run_walk(ctx, 0, st))) return rc;
    if ((rc = build_directed(ctx, 0, st)) || (rc = build_directed(ctx, 1, st))) return rc;
    scalar_force(t, as<double>(ctx->zc), as<double>(ctx->M), as<float4>(ctx->xf), as<uint32_t>(ctx->dsrc[0]),
                 as<uint32_t>(ctx->doff[0]), as<uint32_t>(ctx->dsrc[1]), as<uint32_t>(ctx->doff[1]),
                 ctx->h_level_start, ctx->cfg.soft, as<float>(ctx->fscratch), as<float>(ctx->f),
                 as<float>(ctx->fmin), st);
    CK(rec(3));
    // ---- error-controlled walk
    if ((rc = run_walk(ctx, 1, st))) return rc;
    if ((rc = build_directed(ctx, 2, st)) || (rc = build_directed(ctx, 3, st))) return rc;
    CK(rec(4));
    // ---- far field
    const uint32_t* mk = as<uint32_t>(ctx->dsrc[2]);
    const uint32_t* mo = as<uint32_t>(ctx->doff[2]);
    if (far32 && m2l32_supported(p)) {
        multipoles_to_f32_padded(as<double>(ctx->mult), as<float>(ctx->mult32), t, (int)nr,
                                 (int)((nr + 3) & ~(size_t)3), st);
        m2l_f32(t.dnn, p, mk, mo, as<float>(ctx->mult32), as<float4>(ctx->zhi), as<float4>(ctx->zlo),
                as<float>(ctx->loc32), &ctx->ds->queue, st);
    } else {
        m2l_f64(t.dnn, p, mk, mo, as<double>(ctx->mult), as<double>(ctx->zc), as<double>(ctx->hs),
                as<double>(ctx->loc), ctx->tb, &ctx->ds->queue, st);
        if (far32) multipoles_to_f32(as<double>(ctx->loc), as<float>(ctx->loc32), t, (int)nr, st);
    }
    CK(rec(5));
    if (far32)
        downward_pass_f32(t, ctx->h_level_start, p, as<double>(ctx->zc), as<double>(ctx->hs), as<double>(ctx->geo),
                          as<float>(ctx->loc32),
                          ctx->tb, st);
    else
        downward_pass_f64(t, ctx->h_level_start, p, as<double>(ctx->zc), as<double>(ctx->hs), as<double>(ctx->geo),
                          as<double>(ctx->loc),
                          ctx->tb, st);
    CK(rec(6));
    // ---- leaves: P2P work items, then L2P + partials per body
    uint32_t* item_first = as<uint32_t>(ctx->item_first);
    uint32_t* slot_first = as<uint32_t>(ctx->slot_first);
    uint32_t* totals = as<uint32_t>(ctx->work) + 4;
    leaf_items_plan(t, as<uint32_t>(ctx->doff[3]), item_first, slot_first, totals, st);
    uint32_t htot[2] = {0, 0};
    if (gp) {
        htot[0] = gp->items_cap;
        htot[1] = gp->slots_cap;
        leaf_items_check(totals, gp->items_cap, gp->slots_cap, &ctx->ds->err, st);
    } else {
        CK(cudaMemcpyAsync(htot, totals, 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        ctx->items_total[0] = htot[0];
        ctx->items_total[1] = htot[1];
    }
    if ((rc = ensure(ctx, ctx->item_leaf, 4 * (size_t)(htot[0] + 1))) ||
        (rc = ensure(ctx, ctx->part_hi, 16 * (size_t)(htot[1] + 1))) ||
        (rc = ensure(ctx, ctx->part_lo, 16 * (size_t)(htot[1] + 1))))
        return rc;
    leaf_items_fill(t, item_first, as<int>(ctx->item_leaf), htot[0], as<int>(ctx->leaf_of), st);
    LeafArgs la{};
    la.t = t; la.p = p; la.G = ctx->cfg.G;
    la.soft2 = ctx->cfg.soft * ctx->cfg.soft;
    la.soft2f = (float)la.soft2;
    la.xs = as<double>(ctx->xs); la.ys = as<double>(ctx->ys); la.zs = as<double>(ctx->zs); la.ms = as<double>(ctx->ms);
    la.zc = as<double>(ctx->zc); la.hs = as<double>(ctx->hs);
    la.zhi = as<float4>(ctx->zhi); la.zlo = as<float4>(ctx->zlo);
    la.p2p_src = as<uint32_t>(ctx->dsrc[3]); la.p2p_off = as<uint32_t>(ctx->doff[3]);
    la.perm = as<uint32_t>(in1 ? ctx->v1 : ctx->v0);
    la.ax = ax; la.ay = ay; la.az = az; la.pot = pot;
    la.part_hi = as<double2>(ctx->part_hi); la.part_lo = as<double2>(ctx->part_lo);
    la.tb = ctx->tb;
    la.interactions = as<unsigned long long>(ctx->dcount) + 1;
    la.err = &ctx->ds->err;
    la.bulk = (ctx->cfg.flags & FMM_FLAG_P2P_LOADS) == 0;
    la.tx_extra = (ctx->cfg.fault_inject & 2u) ? 16u : 0u;
    la.slots_cap = htot[1];
    if (mixed) {
        leaf_relative_f32(t, la.xs, la.ys, la.zs, la.ms, la.zc, as<float4>(ctx->prel), st);
        la.prel = as<float4>(ctx->prel);
    }
    la.loc = far32 ? ctx->loc32.ptr : ctx->loc.ptr;
    leaf_eval(la, mixed, far32, as<int>(ctx->item_leaf), item_first, slot_first, totals,
              as<unsigned>(ctx->work), as<int>(ctx->leaf_of), st);
    CK(rec(7));
    CK(cudaGetLastError());
    if (gp) return FMM_OK;  // the caller checks the status block after the replay
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpy(&err, &ctx->ds->err, 4, cudaMemcpyDeviceToHost));
    if (err & kErrCapacity) return fail(ctx, FMM_ERR_CAPACITY, "an internal list overflowed");
    if (err & kErrTimeout)
        return fail(ctx, FMM_ERR_TIMEOUT, "a bounded wait ran out (the walk's ordered appends or the P2P staging)");
    unsigned long long inter = 0;
    CK(cudaMemcpy(&inter, as<unsigned long long>(ctx->dcount) + 1, 8, cudaMemcpyDeviceToHost));
    ctx->stats.p2p_interactions = (int64_t)inter;
    // stats
    fmm_stats& s = ctx->stats;
    s.nnodes = nnodes;
    s.nlevels = nl;
    s.n_far = ctx->npairs[0];
    s.n_near = ctx->npairs[1];
    s.n_m2l = ctx->npairs[2];
    s.n_p2p = ctx->npairs[3];
    s.ms_tree = elapsed(ctx->ev[0], ctx->ev[1]);
    s.ms_upward = elapsed(ctx->ev[1], ctx->ev[2]);
    s.ms_estimate = elapsed(ctx->ev[2], ctx->ev[3]);
    s.ms_walk = elapsed(ctx->ev[3], ctx->ev[4]);
    s.ms_m2l = elapsed(ctx->ev[4], ctx->ev[5]);
    s.ms_downward = elapsed(ctx->ev[5], ctx->ev[6]);
    s.ms_leaf = elapsed(ctx->ev[6], ctx->ev[7]);
    s.ms_total = elapsed(ctx->ev[0], ctx->ev[7]);
    s.kernel_launches = g_launches;
    return FMM_OK;
}

// Jerks on the tree, lists and locals of the solve that just ran (see
// jerk_leaves): the dipole field chi of the weights m_i v_i goes through an
// order p - 1 P2M of each component, the dipole moments, M2M, M2L over the
// same directed list and L2L, in the solve's precision (P2M and M2M in
// double-word FP32 in mixed precision, as for the mass multipoles).
int jerk_pass(fmm_ctx* ctx, const double* vx, const double* vy, const double* vz, double* jx, double* jy,
              double* jz, cudaStream_t st) {
    const int p = ctx->cfg.p;
    const bool mixed = ctx->cfg.precision == FMM_PRECISION_MIXED;
    const bool m2l32 = mixed && m2l32_supported(p);
    const size_t N = (size_t)ctx->n, K = (size_t)ctx->nnodes;
    const size_t nr = ncoef_real(p), nq = ncoef_real(p - 1), pad = (nr + 3) & ~(size_t)3;
    if (ctx->cfg.flags & FMM_FLAG_FP64_LOCALS)
        return fail(ctx, FMM_ERR_ARG, "jerks are not available with FMM_FLAG_FP64_LOCALS");
    int rc;
    if ((rc = ensure(ctx, ctx->jv, 24 * N)) || (rc = ensure(ctx, ctx->jw, 24 * N)) ||
        (rc = ensure(ctx, ctx->jv32, 16 * N)) || (rc = ensure(ctx, ctx->jmom, 24 * K * nq)) ||
        (rc = ensure(ctx, ctx->jmult, 8 * K * nr)))
        return rc;
    if (!m2l32 && (rc = ensure(ctx, ctx->jloc, 8 * K * nr))) return rc;
    if (mixed && ((rc = ensure(ctx, ctx->jloc32, 4 * K * nr)) || (m2l32 && (rc = ensure(ctx, ctx->jmult32, 4 * K * pad)))))
        return rc;
    TreeView t = view(ctx);
    const uint32_t* perm = as<uint32_t>(ctx->sorted_in_1 ? ctx->v1 : ctx->v0);
    const double *xs = as<double>(ctx->xs), *ys = as<double>(ctx->ys), *zs = as<double>(ctx->zs);
    const double *zc = as<double>(ctx->zc), *hs = as<double>(ctx->hs);
    double* w = as<double>(ctx->jw);
    double* mom = as<double>(ctx->jmom);
    CK(cudaEventRecord(ctx->ev[8], st));
    jerk_inputs((int)N, perm, as<double>(ctx->ms), vx, vy, vz, as<double>(ctx->jv), w, as<float4>(ctx->jv32), st);
    for (int c = 0; c < 3; ++c)
        p2m_weights(t, p - 1, xs, ys, zs, w + c * N, zc, hs, mom + c * K * nq, ctx->tb, mixed, st);
    dipole_moments(t, p, mom, mom + K * nq, mom + 2 * K * nq, hs, as<double>(ctx->jmult), st);
    for (int L = t.nlevels - 2; L >= 0; --L)
        m2m_level(t, L, p, as<double>(ctx->geo), as<double>(ctx->jmult), as<double>(ctx->contrib), ctx->tb, mixed, st);
    const uint32_t* mk = as<uint32_t>(ctx->dsrc[2]);
    const uint32_t* mo = as<uint32_t>(ctx->doff[2]);
    if (m2l32) {
        multipoles_to_f32_padded(as<double>(ctx->jmult), as<float>(ctx->jmult32), t, (int)nr, (int)pad, st);
        m2l_f32(t.dnn, p, mk, mo, as<float>(ctx->jmult32), as<float4>(ctx->zhi), as<float4>(ctx->zlo),
                as<float>(ctx->jloc32), &ctx->ds->queue, st);
    } else {
        m2l_f64(t.dnn, p, mk, mo, as<double>(ctx->jmult), zc, hs, as<double>(ctx->jloc), ctx->tb,
                &ctx->ds->queue, st);
        if (mixed) multipoles_to_f32(as<double>(ctx->jloc), as<float>(ctx->jloc32), t, (int)nr, st);
    }
    if (mixed) downward_pass_f32(t, ctx->h_level_start, p, zc, hs, as<double>(ctx->geo), as<float>(ctx->jloc32), ctx->tb, st);
    else downward_pass_f64(t, ctx->h_level_start, p, zc, hs, as<double>(ctx->geo), as<double>(ctx->jloc), ctx->tb, st);
    LeafArgs la{};
    la.err = &ctx->ds->err;
    la.t = t; la.p = p; la.G = ctx->cfg.G;
    la.soft2 = ctx->cfg.soft * ctx->cfg.soft;
    la.soft2f = (float)la.soft2;
    la.xs = xs; la.ys = ys; la.zs = zs; la.ms = as<double>(ctx->ms);
    la.zc = zc; la.hs = hs;
    la.zhi = as<float4>(ctx->zhi); la.zlo = as<float4>(ctx->zlo);
    la.p2p_src = as<uint32_t>(ctx->dsrc[3]); la.p2p_off = as<uint32_t>(ctx->doff[3]);
    la.perm = perm;
    la.tb = ctx->tb;
    la.prel = as<float4>(ctx->prel);
    la.loc = mixed ? ctx->loc32.ptr : ctx->loc.ptr;
    la.part_hi = as<double2>(ctx->part_hi); la.part_lo = as<double2>(ctx->part_lo);
    la.slots_cap = ctx->items_total[1];
    jerk_leaves(la, mixed, mixed ? ctx->jloc32.ptr : ctx->jloc.ptr, as<double>(ctx->jv), as<float4>(ctx->jv32),
                as<int>(ctx->item_leaf), as<uint32_t>(ctx->item_first), as<uint32_t>(ctx->slot_first),
                as<uint32_t>(ctx->work) + 4, as<unsigned>(ctx->work), as<int>(ctx->leaf_of), jx, jy, jz, st);
    CK(cudaEventRecord(ctx->ev[9], st));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    unsigned err = 0;
    CK(cudaMemcpy(&err, &ctx->ds->err, 4, cudaMemcpyDeviceToHost));
    if (err) return fail(ctx, FMM_ERR_CAPACITY, "an internal list overflowed");
    ctx->stats.ms_jerk = elapsed(ctx->ev[8], ctx->ev[9]);
    return FMM_OK;
}

// ---------------------------------------------------------------- HOLD
// The HOLD integrator of Appendix A (after Pelupessy et al. 2012), driven
// from the host: evolve(P, dt) splits the set P by the step sizes of its
// pairs into fast bodies (tau < dt) and slow ones, evolves the fast system
// for dt/2, kicks, drifts and kicks the slow system (H_S = T_S + V_SS +
// V_FS: slow bodies feel all of P, fast bodies the slow ones), and evolves
// the fast system for dt/2 again. Sets of fewer than direct_below bodies use
// the FP64 direct sum (the fast-from-slow force then with the fast masses
// zeroed), larger ones the FMM solve (fast from slow as the difference of the
// solves over P and over F).
struct HoldRun {
    fmm_ctx* ctx;
    cudaStream_t st;
    double *x, *y, *z, *vx, *vy, *vz;
    const double* m;
    double eta, dt_min;
    bool sym;
    int64_t direct_below;
    int64_t device_below;                   // sets of at most this many bodies evolve in one block
    unsigned long long* dstats = nullptr;   // the device-resident evolutions' counters (device)
    int64_t kicks = 0, fmm_solves = 0, direct_solves = 0, max_depth = 0, splits = 0;
};

// accelerations of the first ntgt of k compact bodies (columns of g, stride k)
// from all k, into acc (3 columns of stride k; a 4th column is scratch)
int hold_force(HoldRun& R, int k, const double* g, int ntgt, double* acc, bool force_direct) {
    fmm_ctx* ctx = R.ctx;
    const size_t K = (size_t)k;
    if (force_direct || k < R.direct_below) {
        direct_sum_f64(k, g, g + K, g + 2 * K, g + 6 * K, ctx->cfg.G, ctx->cfg.soft, ntgt, nullptr, acc, acc + K,
                       acc + 2 * K, acc + 3 * K, R.st);
        CK(cudaGetLastError());
        R.direct_solves++;
        return FMM_OK;
    }
    R.fmm_solves++;
    return solve_device(ctx, k, 1, nullptr, g, g + K, g + 2 * K, g + 6 * K, acc, acc + K, acc + 2 * K, acc + 3 * K,
                        R.st);
}

int hold_kick_sets(HoldRun& R, const int* S, int ns, const int* F, int nf, double h) {
    fmm_ctx* ctx = R.ctx;
    const int k = ns + nf;
    double* g = as<double>(ctx->h_gat);
    double* acc = as<double>(ctx->h_acc);
    double* acc2 = as<double>(ctx->h_acc2);
    hold_gather(ns, S, R.x, R.y, R.z, R.vx, R.vy, R.vz, R.m, g, k, -1, R.st);
    hold_gather(nf, F, R.x, R.y, R.z, R.vx, R.vy, R.vz, R.m, g + ns, k, -1, R.st);
    int rc;
    if ((rc = hold_force(R, k, g, k, acc, false)) != FMM_OK) return rc;
    hold_kick(ns, S, acc, nullptr, k, 0, h, R.vx, R.vy, R.vz, R.st);
    if (nf > 0) {
        if (k < R.direct_below) {
            // fast bodies first, their masses zeroed: the force of the slow ones alone
            hold_gather(nf, F, R.x, R.y, R.z, R.vx, R.vy, R.vz, R.m, g, k, 0, R.st);
            hold_gather(ns, S, R.x, R.y, R.z, R.vx, R.vy, R.vz, R.m, g + nf, k, -1, R.st);
            if ((rc = hold_force(R, k, g, nf, acc2, true)) != FMM_OK) return rc;
            hold_kick(nf, F, acc2, nullptr, k, 0, h, R.vx, R.vy, R.vz, R.st);
        } else {
            hold_gather(nf, F, R.x, R.y, R.z, R.vx, R.vy, R.vz, R.m, g, nf, -1, R.st);
            if ((rc = hold_force(R, nf, g, nf, acc2, false)) != FMM_OK) return rc;
            hold_kick(nf, F, acc + ns, acc2, k, nf, h, R.vx, R.vy, R.vz, R.st);
        }
    }
    CK(cudaGetLastError());
    R.kicks++;
    return FMM_OK;
}

int hold_evolve(HoldRun& R, const int* P, int k, double dt, int depth) {
    if (k == 0) return FMM_OK;
    fmm_ctx* ctx = R.ctx;
    if (k <= R.device_below && k <= kHoldSmallMax && k < R.direct_below) {
        // the whole recursion below here inside one block (direct forces, as this path would use)
        hold_small(k, P, R.x, R.y, R.z, R.vx, R.vy, R.vz, R.m, ctx->cfg.G, ctx->cfg.soft, R.eta, R.sym, dt, R.dt_min,
                   depth, R.dstats, R.st);
        CK(cudaGetLastError());
        return FMM_OK;
    }
    if (depth > R.max_depth) R.max_depth = depth;
    const int* S = P;
    const int* F = nullptr;
    int ns = k, nf = 0, rc;
    if (k > 1 && dt > R.dt_min && depth < kHoldMaxDepth) {
        if ((int)ctx->h_S.size() <= depth) {
            ctx->h_S.resize(depth + 1);
            ctx->h_F.resize(depth + 1);
        }
        if ((rc = ensure(ctx, ctx->h_S[depth], 4 * (size_t)k)) || (rc = ensure(ctx, ctx->h_F[depth], 4 * (size_t)k)))
            return rc;
        double* g = as<double>(ctx->h_gat);
        hold_gather(k, P, R.x, R.y, R.z, R.vx, R.vy, R.vz, R.m, g, k, -1, R.st);
        const size_t K = (size_t)k;
        timesteps_f64(k, g, g + K, g + 2 * K, g + 3 * K, g + 4 * K, g + 5 * K, g + 6 * K, ctx->cfg.G, R.eta, R.sym,
                      as<double>(ctx->h_tau), R.st);
        hold_split(k, P, as<double>(ctx->h_tau), dt, as<uint32_t>(ctx->h_flag), as<uint32_t>(ctx->h_scan),
                   as<int>(ctx->h_S[depth]), as<int>(ctx->h_F[depth]), as<uint32_t>(ctx->h_nf),
                   as<uint32_t>(ctx->h_scr), R.st);
        uint32_t hnf = 0;
        CK(cudaMemcpyAsync(&hnf, ctx->h_nf.ptr, 4, cudaMemcpyDeviceToHost, R.st));
        CK(cudaStreamSynchronize(R.st));
        nf = (int)hnf;
        ns = k - nf;
        S = as<int>(ctx->h_S[depth]);
        F = as<int>(ctx->h_F[depth]);
        R.splits++;
    }
    if (nf > 0 && (rc = hold_evolve(R, F, nf, 0.5 * dt, depth + 1)) != FMM_OK) return rc;
    if (ns > 0) {
        if ((rc = hold_kick_sets(R, S, ns, F, nf, 0.5 * dt)) != FMM_OK) return rc;
        hold_drift(ns, S, dt, R.x, R.y, R.z, R.vx, R.vy, R.vz, R.st);
        if ((rc = hold_kick_sets(R, S, ns, F, nf, 0.5 * dt)) != FMM_OK) return rc;
    }
    if (nf > 0 && (rc = hold_evolve(R, F, nf, 0.5 * dt, depth + 1)) != FMM_OK) return rc;
    return FMM_OK;
}

int check_cfg(const fmm_config* c, std::string& why) {
    if (!c) { why = "cfg is NULL"; return FMM_ERR_ARG; }
    if (c->p < 1 || c->p > kMaxP) { why = "p must be in [1, 30]"; return FMM_ERR_ARG; }
    if (!(c->eps >= 0.0) || !std::isfinite(c->eps)) { why = "eps must be finite and >= 0"; return FMM_ERR_ARG; }
    if (c->leaf_size < 1 || c->leaf_size > kMaxLeaf) { why = "leaf_size must be in [1, 256]"; return FMM_ERR_ARG; }
    if (c->precision != FMM_PRECISION_FP64 && c->precision != FMM_PRECISION_MIXED) { why = "unknown precision"; return FMM_ERR_ARG; }
    if (c->precision == FMM_PRECISION_MIXED && c->p > kMaxPF32) { why = "mixed precision supports p <= 16"; return FMM_ERR_ARG; }
    if (!std::isfinite(c->G)) { why = "G must be finite"; return FMM_ERR_ARG; }
    if (!(c->soft >= 0.0) || !std::isfinite(c->soft)) { why = "soft must be finite and >= 0"; return FMM_ERR_ARG; }
    if (c->flags & ~(FMM_FLAG_FP64_LOCALS | FMM_FLAG_P2P_LOADS)) { why = "unknown flag bits"; return FMM_ERR_ARG; }
    if ((c->flags & FMM_FLAG_FP64_LOCALS) && c->precision != FMM_PRECISION_MIXED) {
        why = "FMM_FLAG_FP64_LOCALS applies to mixed precision only";
        return FMM_ERR_ARG;
    }
    return FMM_OK;
}

}  // namespace

extern "C" {

int fmm_create(fmm_ctx** out, const fmm_config* cfg) {
    if (!out) { g_create_error = "out is NULL"; return FMM_ERR_ARG; }
    *out = nullptr;
    std::string why;
    int rc = check_cfg(cfg, why);
    if (rc != FMM_OK) { g_create_error = why; return rc; }
    fmm_ctx* ctx = new fmm_ctx();
    ctx->cfg = *cfg;
    if (cudaGetDevice(&ctx->device) != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "no CUDA device";
        delete ctx;
        return FMM_ERR_CUDA;
    }
    build_host_tables(ctx->ht);
    // global-memory tables: swap cos, swap sin, w, iw, fact, rec_a, rec_b, diag, sub, binom row
    const size_t ncos = sizeof(kSwapCos) / sizeof(double), nsin = sizeof(kSwapSin) / sizeof(double);
    const size_t nw = (size_t)(kMaxP + 2) * (kMaxP + 2), nrec = (size_t)(kMaxP + 1) * (kMaxP + 1);
    const size_t nfact = 2 * kMaxP + 4, nd = kMaxP + 1;
    std::vector<double> blob;
    blob.insert(blob.end(), kSwapCos, kSwapCos + ncos);
    blob.insert(blob.end(), kSwapSin, kSwapSin + nsin);
    blob.insert(blob.end(), &ctx->ht.w[0][0], &ctx->ht.w[0][0] + nw);
    blob.insert(blob.end(), &ctx->ht.iw[0][0], &ctx->ht.iw[0][0] + nw);
    blob.insert(blob.end(), ctx->ht.fact, ctx->ht.fact + nfact);
    blob.insert(blob.end(), &ctx->ht.rec_a[0][0], &ctx->ht.rec_a[0][0] + nrec);
    blob.insert(blob.end(), &ctx->ht.rec_b[0][0], &ctx->ht.rec_b[0][0] + nrec);
    blob.insert(blob.end(), ctx->ht.diag, ctx->ht.diag + nd);
    blob.insert(blob.end(), ctx->ht.sub, ctx->ht.sub + nd);
    blob.insert(blob.end(), &ctx->ht.binom[cfg->p][0], &ctx->ht.binom[cfg->p][0] + nd);
    // z-shift coefficients sqrt(C(n+m,k) C(n-m,k)) from exact binomials
    // (every C(a, k) with a <= 2 kMaxP is below 2^63; long double keeps them exact)
    const size_t zsh_at = blob.size();
    blob.resize(blob.size() + kZShiftSize);
    for (int n = 0; n <= kMaxP; ++n)
        for (int m = 0; m <= n; ++m)
            for (int k = 0; k <= n - m; ++k) {
                long double c1 = 1.0L, c2 = 1.0L;
                for (int i = 1; i <= k; ++i) {
                    c1 = c1 * (long double)(n + m - k + i) / (long double)i;
                    c2 = c2 * (long double)(n - m - k + i) / (long double)i;
                }
                blob[zsh_at + zshift_offset(n, m) + k] = (double)sqrtl(c1 * c2);
            }
    if (ensure(ctx, ctx->tables, blob.size() * sizeof(double)) != FMM_OK ||
        cudaMemcpy(ctx->tables.ptr, blob.data(), blob.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMalloc(&ctx->ds, sizeof(DevScalars)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_ds, sizeof(DevScalars)) != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "device allocation failed in fmm_create";
        fmm_destroy(ctx);
        return FMM_ERR_OOM;
    }
    cudaMemset(ctx->ds, 0, sizeof(DevScalars));
    const double* base = reinterpret_cast<const double*>(ctx->tables.ptr);
    size_t o = 0;
    ctx->tb.swap_cos = base + o; o += ncos;
    ctx->tb.swap_sin = base + o; o += nsin;
    ctx->tb.w = base + o; o += nw;
    ctx->tb.iw = base + o; o += nw;
    ctx->tb.fact = base + o; o += nfact;
    ctx->tb.rec_a = base + o; o += nrec;
    ctx->tb.rec_b = base + o; o += nrec;
    ctx->tb.diag = base + o; o += nd;
    ctx->tb.sub = base + o; o += nd;
    ctx->tb.zshift = base + zsh_at;
    // double-word copies: hi = the float nearest x, lo = the float nearest x - hi
    {
        std::vector<float2> dwb;
        auto put = [&dwb](const double* src, size_t cnt) {
            for (size_t i = 0; i < cnt; ++i) {
                const float hi = (float)src[i];
                dwb.push_back(make_float2(hi, (float)(src[i] - (double)hi)));
            }
        };
        put(kSwapCos, ncos);
        put(kSwapSin, nsin);
        put(blob.data() + zsh_at, kZShiftSize);
        if (ensure(ctx, ctx->tables_dw, dwb.size() * sizeof(float2)) != FMM_OK ||
            cudaMemcpy(ctx->tables_dw.ptr, dwb.data(), dwb.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            g_create_error = "device allocation failed in fmm_create";
            fmm_destroy(ctx);
            return FMM_ERR_OOM;
        }
        const float2* b2 = reinterpret_cast<const float2*>(ctx->tables_dw.ptr);
        ctx->tb.swap_cos_dw = b2;
        ctx->tb.swap_sin_dw = b2 + ncos;
        ctx->tb.zshift_dw = b2 + ncos + nsin;
    }
    upload_expansion_tables(ctx->ht);
    upload_leaf_tables(ctx->ht);
    for (auto& e : ctx->ev) cudaEventCreate(&e);
    if (cudaGetLastError() != cudaSuccess) {
        g_create_error = "CUDA error while uploading tables";
        fmm_destroy(ctx);
        return FMM_ERR_CUDA;
    }
    *out = ctx;
    return FMM_OK;
}

void fmm_destroy(fmm_ctx* ctx) {
    if (!ctx) return;
    Buf* all[] = {&ctx->tables, &ctx->tables_dw, &ctx->k0, &ctx->k1, &ctx->v0, &ctx->v1, &ctx->hist, &ctx->xs, &ctx->ys,
                  &ctx->zs, &ctx->ms, &ctx->xf, &ctx->prel, &ctx->lcp, &ctx->win, &ctx->hi, &ctx->chunk,
                  &ctx->f, &ctx->bbox, &ctx->level, &ctx->begin, &ctx->end, &ctx->parent,
                  &ctx->first_child, &ctx->nchild, &ctx->M, &ctx->S, &ctx->zc, &ctx->r, &ctx->hs, &ctx->Pk,
                  &ctx->mult, &ctx->mult32, &ctx->loc, &ctx->loc32, &ctx->fmin, &ctx->fscratch,
                  &ctx->front0, &ctx->front1, &ctx->walk_scan, &ctx->dcount, &ctx->zhi, &ctx->zlo, &ctx->contrib, &ctx->Phat, &ctx->r32,
                  &ctx->item_first, &ctx->slot_first, &ctx->item_leaf, &ctx->leaf_of, &ctx->part_hi,
                  &ctx->part_lo, &ctx->work, &ctx->coff, &ctx->box, &ctx->ck0, &ctx->ck1, &ctx->cv0,
                  &ctx->cv1, &ctx->cid, &ctx->jv, &ctx->jv32, &ctx->jw, &ctx->jmom, &ctx->jmult,
                  &ctx->jmult32, &ctx->jloc, &ctx->jloc32, &ctx->h_all, &ctx->h_gat, &ctx->h_acc, &ctx->h_acc2,
                  &ctx->h_tau, &ctx->h_flag, &ctx->h_scan, &ctx->h_scr, &ctx->h_nf, &ctx->geo};
    for (Buf* b : all) release(*b);
    for (Buf& b : ctx->h_S) release(b);
    for (Buf& b : ctx->h_F) release(b);
    drop_plan(ctx->plan);
    if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
    if (ctx->gev[0]) cudaEventDestroy(ctx->gev[0]);
    if (ctx->gev[1]) cudaEventDestroy(ctx->gev[1]);
    for (int l = 0; l < 4; ++l) {
        release(ctx->lists[l]);
        release(ctx->dkeys[l]);
        release(ctx->dalt[l]);
        release(ctx->dsrc[l]);
        release(ctx->doff[l]);
        release(ctx->hin[l]);
        release(ctx->hout[l]);
    }
    if (ctx->ds) cudaFree(ctx->ds);
    if (ctx->h_ds) cudaFreeHost(ctx->h_ds);
    for (auto& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    delete ctx;
}

int fmm_solve(fmm_ctx* ctx, int64_t n, const double* x, const double* y, const double* z, const double* m,
              double* ax, double* ay, double* az, double* pot, void* cuda_stream) {
    if (!ctx) return FMM_ERR_ARG;
    if (n < 0 || n > (int64_t)1 << 30) return fail(ctx, FMM_ERR_ARG, "n must be in [0, 2^30]");
    if (n > 0 && (!x || !y || !z || !m || !ax || !ay || !az))
        return fail(ctx, FMM_ERR_ARG, "NULL input or output pointer");
    cudaSetDevice(ctx->device);
    return solve_device(ctx, n, 1, nullptr, x, y, z, m, ax, ay, az, pot, (cudaStream_t)cuda_stream);
}

int fmm_solve_jerk(fmm_ctx* ctx, int64_t n, const double* x, const double* y, const double* z, const double* vx,
                   const double* vy, const double* vz, const double* m, double* ax, double* ay, double* az,
                   double* pot, double* jx, double* jy, double* jz, void* cuda_stream) {
    if (!ctx) return FMM_ERR_ARG;
    if (n < 0 || n > (int64_t)1 << 30) return fail(ctx, FMM_ERR_ARG, "n must be in [0, 2^30]");
    if (n > 0 && (!x || !y || !z || !vx || !vy || !vz || !m || !ax || !ay || !az || !jx || !jy || !jz))
        return fail(ctx, FMM_ERR_ARG, "NULL input or output pointer");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc = solve_device(ctx, n, 1, nullptr, x, y, z, m, ax, ay, az, pot, st);
    if (rc != FMM_OK || n == 0) return rc;
    return jerk_pass(ctx, vx, vy, vz, jx, jy, jz, st);
}

int fmm_solve_host(fmm_ctx* ctx, int64_t n, const double* x, const double* y, const double* z,
                   const double* m, double* ax, double* ay, double* az, double* pot, void* cuda_stream) {
    if (!ctx) return FMM_ERR_ARG;
    if (n < 0 || n > (int64_t)1 << 30) return fail(ctx, FMM_ERR_ARG, "n must be in [0, 2^30]");
    if (n == 0) return FMM_OK;
    if (!x || !y || !z || !m || !ax || !ay || !az) return fail(ctx, FMM_ERR_ARG, "NULL input or output pointer");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t bytes = 8 * (size_t)n;
    int rc;
    for (int i = 0; i < 4; ++i)
        if ((rc = ensure(ctx, ctx->hin[i], bytes)) || (rc = ensure(ctx, ctx->hout[i], bytes))) return rc;
    const double* in[4] = {x, y, z, m};
    for (int i = 0; i < 4; ++i) CK(cudaMemcpyAsync(ctx->hin[i].ptr, in[i], bytes, cudaMemcpyHostToDevice, st));
    rc = solve_device(ctx, n, 1, nullptr, as<double>(ctx->hin[0]), as<double>(ctx->hin[1]), as<double>(ctx->hin[2]),
                      as<double>(ctx->hin[3]), as<double>(ctx->hout[0]), as<double>(ctx->hout[1]),
                      as<double>(ctx->hout[2]), pot ? as<double>(ctx->hout[3]) : nullptr, st);
    if (rc != FMM_OK) return rc;
    double* outp[4] = {ax, ay, az, pot};
    for (int i = 0; i < 4; ++i)
        if (outp[i]) CK(cudaMemcpyAsync(outp[i], ctx->hout[i].ptr, bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return FMM_OK;
}

int fmm_solve_graph(fmm_ctx* ctx, int32_t nclusters, const int64_t* offsets, int64_t n, const double* x,
                    const double* y, const double* z, const double* m, double* ax, double* ay, double* az,
                    double* pot, void* cuda_stream) {
    if (!ctx) return FMM_ERR_ARG;
    if (n < 0 || n > (int64_t)1 << 30) return fail(ctx, FMM_ERR_ARG, "n must be in [0, 2^30]");
    if (offsets) {
        if (nclusters < 1 || offsets[0] != 0 || offsets[nclusters] != n)
            return fail(ctx, FMM_ERR_ARG, "offsets must run from 0 to n");
        for (int32_t c = 0; c < nclusters; ++c)
            if (offsets[c + 1] < offsets[c]) return fail(ctx, FMM_ERR_ARG, "offsets must be non-decreasing");
    } else {
        nclusters = 1;
    }
    if (n == 0) return solve_device(ctx, 0, nclusters, offsets, x, y, z, m, ax, ay, az, pot, nullptr);
    if (!x || !y || !z || !m || !ax || !ay || !az) return fail(ctx, FMM_ERR_ARG, "NULL input or output pointer");
    cudaSetDevice(ctx->device);
    if (!ctx->gstream) {
        CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
        CK(cudaEventCreate(&ctx->gev[0]));
        CK(cudaEventCreate(&ctx->gev[1]));
    }
    cudaStream_t gs = ctx->gstream;
    CK(cudaStreamSynchronize((cudaStream_t)cuda_stream));  // the inputs are ready
    GraphPlan& g = ctx->plan;
    const void* ptrs[8] = {x, y, z, m, ax, ay, az, pot};
    std::vector<int64_t> offs(offsets ? offsets : nullptr, offsets ? offsets + nclusters + 1 : nullptr);
    const bool same = g.valid && g.n == n && g.offs == offs && g.gen == ctx->gen &&
                      std::equal(ptrs, ptrs + 8, g.ptrs);
    if (same) {
        // replay, then read one status block: any overflow or a tree deeper than
        // planned sends this call to the ordinary solve and the next to a new plan
        CK(cudaEventRecord(ctx->gev[0], gs));
        CK(cudaGraphLaunch(g.exec, gs));
        CK(cudaEventRecord(ctx->gev[1], gs));
        CK(cudaMemcpyAsync(ctx->h_ds, ctx->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost, gs));
        unsigned long long cnt[6] = {};
        CK(cudaMemcpyAsync(cnt, ctx->dcount.ptr, sizeof(cnt), cudaMemcpyDeviceToHost, gs));
        CK(cudaStreamSynchronize(gs));
        const DevScalars& d = *ctx->h_ds;
        bool ok = d.err == 0;
        int nl = 1;
        for (int L = 0; L <= kMaxLevel && ok; ++L) {
            const int cntL = d.level_start[L + 1] - d.level_start[L];
            if (cntL > g.lvl_cap[L]) ok = false;
            if (cntL > 0) nl = L + 1;
        }
        if (nl > g.nlevels) ok = false;
        if (ok) {
            ctx->nnodes = d.nnodes;
            ctx->nlevels = nl;
            std::memcpy(ctx->h_level_start, d.level_start, sizeof(ctx->h_level_start));
            std::memset(&ctx->stats, 0, sizeof(ctx->stats));
            fmm_stats& st = ctx->stats;
            st.n = n;
            st.nnodes = d.nnodes;
            st.nlevels = nl;
            st.n_far = (int64_t)d.list_cnt[0];
            st.n_near = (int64_t)d.list_cnt[1];
            st.n_m2l = (int64_t)d.list_cnt[2];
            st.n_p2p = (int64_t)d.list_cnt[3];
            st.p2p_interactions = (int64_t)cnt[1];
            st.walk_iters = g.walk_iters[0] + g.walk_iters[1];
            st.kernel_launches = g.launches;
            st.ms_tree = elapsed(ctx->ev[0], ctx->ev[1]);
            st.ms_upward = elapsed(ctx->ev[1], ctx->ev[2]);
            st.ms_estimate = elapsed(ctx->ev[2], ctx->ev[3]);
            st.ms_walk = elapsed(ctx->ev[3], ctx->ev[4]);
            st.ms_m2l = elapsed(ctx->ev[4], ctx->ev[5]);
            st.ms_downward = elapsed(ctx->ev[5], ctx->ev[6]);
            st.ms_leaf = elapsed(ctx->ev[6], ctx->ev[7]);
            st.ms_total = elapsed(ctx->gev[0], ctx->gev[1]);
            st.graph_replays = 1;
            return FMM_OK;
        }
        g.valid = false;
    }
    // an ordinary solve gives this call's result and the sizes to plan from
    int rc = solve_device(ctx, n, nclusters, offsets, x, y, z, m, ax, ay, az, pot, gs);
    if (rc != FMM_OK) return rc;
    const fmm_stats eager = ctx->stats;
    drop_plan(g);
    g.n = n;
    g.offs = offs;
    std::copy(ptrs, ptrs + 8, g.ptrs);
    const auto grow = [](int64_t v, double f, int64_t pad) { return (int64_t)(v * f) + pad; };
    // node headroom, but not past the index width of the ordinary solve when that
    // still leaves 6%: one more bit can turn the 32-bit directed keys into 64-bit
    // ones (a 2^16-node tree) or add a radix pass
    int64_t node_cap = grow(ctx->nnodes, 1.25, 64);
    const int64_t same_width = ((int64_t)1 << bit_length(ctx->nnodes)) - 1;
    if (node_cap > same_width && same_width >= ctx->nnodes + ctx->nnodes / 16 + 16) node_cap = same_width;
    g.node_cap = (int)std::min<int64_t>(node_cap, INT32_MAX / 2);
    g.nb = bit_length(g.node_cap);
    g.nlevels = std::min(ctx->nlevels + 1, kMaxLevel + 1);
    g.nroots = nclusters;
    for (int L = 0; L <= kMaxLevel + 1; ++L) {
        const int cntL = L <= kMaxLevel ? ctx->h_level_start[L + 1] - ctx->h_level_start[L] : 0;
        g.lvl_cap[L] = L < g.nlevels ? (int)std::min<int64_t>(grow(cntL, 1.5, 64), g.node_cap) : 0;
    }
    for (int l = 0; l < 4; ++l) g.pair_cap[l] = grow(ctx->npairs[l], 1.3, 4096);
    // walk steps: the ordinary solve's count of each walk plus a margin
    g.walk_iters[0] = std::min(ctx->walk_steps[0] + 4, kMaxWalkIters);
    g.walk_iters[1] = std::min(ctx->walk_steps[1] + 4, kMaxWalkIters);
    g.items_cap = (uint32_t)grow(ctx->items_total[0], 1.3, 1024);
    g.slots_cap = (uint32_t)grow(ctx->items_total[1], 1.3, 65536);
    CK(cudaMallocHost(&g.h_coff, 4 * ((size_t)nclusters + 1)));
    std::memcpy(g.h_coff, ctx->h_coff.data(), 4 * ((size_t)nclusters + 1));
    // the graph form once without capture: allocates every buffer at its planned
    // size (nothing may allocate while capturing) and checks that it runs clean
    ctx->gmode = &g;
    rc = solve_device(ctx, n, nclusters, offsets, x, y, z, m, ax, ay, az, pot, gs);
    ctx->gmode = nullptr;
    unsigned err = 1;
    if (rc == FMM_OK) {
        CK(cudaMemcpyAsync(&err, &ctx->ds->err, 4, cudaMemcpyDeviceToHost, gs));
        CK(cudaStreamSynchronize(gs));
    }
    if (rc == FMM_OK && err == 0) {
        cudaGraph_t graph = nullptr;
        const int64_t gen0 = ctx->gen;
        if (cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            ctx->gmode = &g;
            rc = solve_device(ctx, n, nclusters, offsets, x, y, z, m, ax, ay, az, pot, gs);
            ctx->gmode = nullptr;
            g.launches = g_launches;
            const cudaError_t ec = cudaStreamEndCapture(gs, &graph);
            if (rc == FMM_OK && ec == cudaSuccess && graph && ctx->gen == gen0 &&
                cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess) {
                g.valid = true;
                g.gen = ctx->gen;
            }
            if (graph) cudaGraphDestroy(graph);
        }
        cudaGetLastError();
    }
    // this call's result is the ordinary solve's (the graph form wrote the same)
    ctx->stats = eager;
    ctx->stats.graph_replays = 0;
    return rc == FMM_OK || g.valid ? FMM_OK : rc;
}

int fmm_solve_batch(fmm_ctx* ctx, int32_t nclusters, const int64_t* offsets, const double* x,
                    const double* y, const double* z, const double* m, double* ax, double* ay, double* az,
                    double* pot, void* cuda_stream) {
    if (!ctx) return FMM_ERR_ARG;
    if (nclusters < 0 || (nclusters > 0 && !offsets)) return fail(ctx, FMM_ERR_ARG, "bad cluster offsets");
    if (nclusters > 0 && offsets[0] != 0) return fail(ctx, FMM_ERR_ARG, "offsets[0] must be 0");
    for (int32_t c = 0; c < nclusters; ++c)
        if (offsets[c + 1] < offsets[c]) return fail(ctx, FMM_ERR_ARG, "offsets must be non-decreasing");
    const int64_t n = nclusters > 0 ? offsets[nclusters] : 0;
    if (n > (int64_t)1 << 30) return fail(ctx, FMM_ERR_ARG, "the clusters hold more than 2^30 bodies");
    if (n > 0 && (!x || !y || !z || !m || !ax || !ay || !az))
        return fail(ctx, FMM_ERR_ARG, "NULL input or output pointer");
    cudaSetDevice(ctx->device);
    return solve_device(ctx, n, nclusters, offsets, x, y, z, m, ax, ay, az, pot, (cudaStream_t)cuda_stream);
}

int fmm_hold(fmm_ctx* ctx, int64_t n, double* x, double* y, double* z, double* vx, double* vy, double* vz,
             const double* m, double dt, int64_t nsteps, double eta, int32_t symmetrize, double dt_min,
             int64_t direct_below, int64_t device_below, int64_t* stats, void* cuda_stream) {
    if (!ctx) return FMM_ERR_ARG;
    if (n < 0 || n > (int64_t)1 << 30) return fail(ctx, FMM_ERR_ARG, "n must be in [0, 2^30]");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, FMM_ERR_ARG, "dt must be finite and > 0");
    if (!(eta > 0.0) || !std::isfinite(eta)) return fail(ctx, FMM_ERR_ARG, "eta must be finite and > 0");
    if (!(dt_min >= 0.0) || nsteps < 0) return fail(ctx, FMM_ERR_ARG, "dt_min >= 0 and nsteps >= 0 required");
    if (device_below < 0 || device_below > kHoldSmallMax)
        return fail(ctx, FMM_ERR_ARG, "device_below must be in [0, 1024]");
    if (n > 0 && (!x || !y || !z || !vx || !vy || !vz || !m)) return fail(ctx, FMM_ERR_ARG, "NULL pointer");
    cudaSetDevice(ctx->device);
    HoldRun R{ctx, (cudaStream_t)cuda_stream, x, y, z, vx, vy, vz, m, eta, dt_min, symmetrize != 0, direct_below,
              device_below};
    const size_t N = (size_t)(n > 0 ? n : 1);
    int rc;
    if ((rc = ensure(ctx, ctx->h_all, 4 * N)) || (rc = ensure(ctx, ctx->h_gat, 56 * N)) ||
        (rc = ensure(ctx, ctx->h_acc, 32 * N)) || (rc = ensure(ctx, ctx->h_acc2, 32 * N)) ||
        (rc = ensure(ctx, ctx->h_tau, 8 * N)) || (rc = ensure(ctx, ctx->h_flag, 4 * N)) ||
        (rc = ensure(ctx, ctx->h_scan, 4 * N)) || (rc = ensure(ctx, ctx->h_scr, 4 * scan_scratch_words((int64_t)N))) ||
        (rc = ensure(ctx, ctx->h_nf, 64)))
        return rc;
    R.dstats = as<unsigned long long>(ctx->h_nf) + 1;  // words 1..5 (word 0 holds the split's fast count)
    CK(cudaMemsetAsync(R.dstats, 0, 5 * sizeof(unsigned long long), R.st));
    hold_iota((int)n, as<int>(ctx->h_all), R.st);
    for (int64_t s = 0; s < nsteps && n > 0; ++s)
        if ((rc = hold_evolve(R, as<int>(ctx->h_all), (int)n, dt, 0)) != FMM_OK) return rc;
    unsigned long long dst[5] = {0, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(dst, R.dstats, sizeof(dst), cudaMemcpyDeviceToHost, R.st));
    CK(cudaStreamSynchronize(R.st));
    R.kicks += (int64_t)dst[0];
    R.direct_solves += (int64_t)dst[2];
    if ((int64_t)dst[3] > R.max_depth) R.max_depth = (int64_t)dst[3];
    R.splits += (int64_t)dst[4];
    if (stats) {
        stats[0] = R.kicks;
        stats[1] = R.fmm_solves;
        stats[2] = R.direct_solves;
        stats[3] = R.max_depth;
        stats[4] = R.splits;
    }
    return FMM_OK;
}

int fmm_timesteps(fmm_ctx* ctx, int64_t n, const double* x, const double* y, const double* z, const double* vx,
                  const double* vy, const double* vz, const double* m, double eta, int32_t symmetrize, double* tau,
                  void* cuda_stream) {
    if (!ctx) return FMM_ERR_ARG;
    if (n < 0 || n > INT32_MAX) return fail(ctx, FMM_ERR_ARG, "n must be in [0, 2^31)");
    if (!(eta > 0.0) || !std::isfinite(eta)) return fail(ctx, FMM_ERR_ARG, "eta must be finite and > 0");
    if (n == 0) return FMM_OK;
    if (!x || !y || !z || !vx || !vy || !vz || !m || !tau) return fail(ctx, FMM_ERR_ARG, "NULL pointer");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    timesteps_f64((int)n, x, y, z, vx, vy, vz, m, ctx->cfg.G, eta, symmetrize != 0, tau, st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return FMM_OK;
}

int fmm_direct(fmm_ctx* ctx, int64_t n, const double* x, const double* y, const double* z, const double* m,
               int64_t ntargets, const int64_t* targets, double* ax, double* ay, double* az, double* pot,
               void* cuda_stream) {
    if (!ctx) return FMM_ERR_ARG;
    if (n < 0 || ntargets < 0) return fail(ctx, FMM_ERR_ARG, "negative size");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    direct_sum_f64(n, x, y, z, m, ctx->cfg.G, ctx->cfg.soft, targets ? ntargets : n, targets, ax, ay, az, pot, st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return FMM_OK;
}

int fmm_get_stats(const fmm_ctx* ctx, fmm_stats* out) {
    if (!ctx || !out) return FMM_ERR_ARG;
    *out = ctx->stats;
    return FMM_OK;
}

int fmm_export_tree(const fmm_ctx* cctx, uint64_t* keys, int64_t* perm, int32_t* level, int32_t* begin,
                    int32_t* end, int32_t* parent, int32_t* first_child, int32_t* nchild) {
    fmm_ctx* ctx = const_cast<fmm_ctx*>(cctx);
    if (!ctx) return FMM_ERR_ARG;
    const size_t n = (size_t)ctx->n, K = (size_t)ctx->nnodes;
    if (keys) CK(cudaMemcpy(keys, (ctx->sorted_in_1 ? ctx->k1 : ctx->k0).ptr, 8 * n, cudaMemcpyDeviceToHost));
    if (perm) {
        std::vector<uint32_t> p32(n);
        CK(cudaMemcpy(p32.data(), (ctx->sorted_in_1 ? ctx->v1 : ctx->v0).ptr, 4 * n, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) perm[i] = p32[i];
    }
    struct { int32_t* dst; Buf* src; } arr[] = {{level, &ctx->level}, {begin, &ctx->begin}, {end, &ctx->end},
                                                {parent, &ctx->parent}, {first_child, &ctx->first_child},
                                                {nchild, &ctx->nchild}};
    for (auto& a : arr)
        if (a.dst) CK(cudaMemcpy(a.dst, a.src->ptr, 4 * K, cudaMemcpyDeviceToHost));
    return FMM_OK;
}

int fmm_export_geometry(const fmm_ctx* cctx, double* M, double* z, double* r, double* P, float* fmin, float* f) {
    fmm_ctx* ctx = const_cast<fmm_ctx*>(cctx);
    if (!ctx) return FMM_ERR_ARG;
    const size_t K = (size_t)ctx->nnodes;
    if (M) CK(cudaMemcpy(M, ctx->M.ptr, 8 * K, cudaMemcpyDeviceToHost));
    if (z) CK(cudaMemcpy(z, ctx->zc.ptr, 24 * K, cudaMemcpyDeviceToHost));
    if (r) CK(cudaMemcpy(r, ctx->r.ptr, 8 * K, cudaMemcpyDeviceToHost));
    if (P) CK(cudaMemcpy(P, ctx->Pk.ptr, 8 * K * (size_t)(ctx->cfg.p + 1), cudaMemcpyDeviceToHost));
    if (fmin) CK(cudaMemcpy(fmin, ctx->fmin.ptr, 4 * K, cudaMemcpyDeviceToHost));
    if (f) CK(cudaMemcpy(f, ctx->f.ptr, 4 * (size_t)ctx->n, cudaMemcpyDeviceToHost));
    return FMM_OK;
}

int fmm_export_pairs(const fmm_ctx* cctx, int which, int64_t* count, int32_t* pairs) {
    fmm_ctx* ctx = const_cast<fmm_ctx*>(cctx);
    if (!ctx || which < 0 || which > 3 || !count) return FMM_ERR_ARG;
    *count = ctx->npairs[which];
    if (pairs && ctx->npairs[which] > 0)
        CK(cudaMemcpy(pairs, ctx->lists[which].ptr, 8 * (size_t)ctx->npairs[which], cudaMemcpyDeviceToHost));
    return FMM_OK;
}

int fmm_export_swap(int64_t* ncos, int64_t* nsin, double* cos_blocks, double* sin_blocks) {
    const int64_t nc = (int64_t)(sizeof(kSwapCos) / sizeof(double)), ns = (int64_t)(sizeof(kSwapSin) / sizeof(double));
    if (ncos) *ncos = nc;
    if (nsin) *nsin = ns;
    if (cos_blocks) std::memcpy(cos_blocks, kSwapCos, sizeof(kSwapCos));
    if (sin_blocks) std::memcpy(sin_blocks, kSwapSin, sizeof(kSwapSin));
    return FMM_OK;
}

const char* fmm_last_error(const fmm_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
