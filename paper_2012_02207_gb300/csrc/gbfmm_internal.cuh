// Internal declarations of the gbfmm GPU library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "gbfmm.h"

namespace gbfmm {

constexpr int kMaxLevel = 21;   // 21 bits per axis in a 63-bit Morton key
constexpr int kMaxP = 30;       // swap matrices are tabulated to p = 30 (Sec. 2.4)
constexpr int kMaxPF32 = 16;    // largest order of the FP32 expansion kernels
constexpr int kMaxLeaf = 256;
constexpr int kMaxWalkIters = 192;

// error bits raised by kernels (never a trap)
enum : unsigned {
    kErrCapacity = 1u,
    kErrCoincident = 2u,
    kErrNonfinite = 4u,
    kErrTimeout = 8u,
    kErrIndex = 16u,  // a cell index out of range (an internal error)
    kErrLongRun = 32u,  // a run of equal keys longer than the bounded coincidence scan (not an error)
};

// real layout of a hat coefficient vector: degree n starts at n*n with
// [Re m=0, Re m=1, Im m=1, ..., Re m=n, Im m=n]; (p+1)^2 reals in all.
__host__ __device__ constexpr int hre(int n, int m) { return n * n + (m == 0 ? 0 : 2 * m - 1); }
__host__ __device__ constexpr int him(int n, int m) { return n * n + 2 * m; }
__host__ __device__ constexpr int ncoef_real(int p) { return (p + 1) * (p + 1); }

// Device-resident scalars of one context (counters, box, tree sizes).
struct DevScalars {
    double box[8];                 // cx, cy, cz, h, lox, loy, loz, size
    unsigned err;                  // kErr* bits
    unsigned queue;                // work counter of the M2L kernels (zeroed before each launch)
    unsigned long long cnt[kMaxWalkIters + 2];  // walk frontier sizes per iteration
    unsigned long long list_cnt[4];             // far, near, m2l, p2p
    // the walk's ordered appends: the most tiles a step of the current walk
    // used (records to clear before the next walk), per step the tile ticket
    // and the accepted and leaf list lengths so far
    unsigned long long walk_tiles;
    unsigned ticket[kMaxWalkIters + 2];
    unsigned long long acc_hist[kMaxWalkIters + 2];
    unsigned long long leaf_hist[kMaxWalkIters + 2];
    int nnodes;
    int level_start[kMaxLevel + 3];
};

// Host tables of normalisation constants for hat-normalised harmonics
// Shat_n^m = sqrt((n+m)!(n-m)!) Upsilon_n^m.
struct HostTables {
    double w[kMaxP + 2][kMaxP + 2];    // sqrt((n+m)!(n-m)!)
    double iw[kMaxP + 2][kMaxP + 2];   // 1 / w
    double fact[2 * kMaxP + 4];
    double binom[kMaxP + 1][kMaxP + 1];
    double rec_a[kMaxP + 1][kMaxP + 1];  // (2n-1)/sqrt((n+m)(n-m))
    double rec_b[kMaxP + 1][kMaxP + 1];  // sqrt((n+m-1)(n-m-1)/((n+m)(n-m)))
    double diag[kMaxP + 1];              // sqrt((2m-1)/(2m))
    double sub[kMaxP + 1];               // sqrt(2m+1)
};

// Device pointers of the global-memory tables (FP64, p <= 30).
struct DevTables {
    const double* swap_cos;   // generator layout
    const double* swap_sin;
    const double* w;          // (kMaxP+2)^2
    const double* iw;
    const double* fact;
    const double* rec_a;      // (kMaxP+1)^2
    const double* rec_b;
    const double* diag;
    const double* sub;
    const double* zshift;     // sqrt(C(n+m,k) C(n-m,k)) at zshift_offset(n, m) + k, k <= n-m
    // double-word (hi, lo float pairs) copies of the swap and z-shift tables
    const float2* swap_cos_dw;
    const float2* swap_sin_dw;
    const float2* zshift_dw;
};

// offset of (n, m) in the z-shift coefficient table (n <= kMaxP, 0 <= m <= n)
__host__ __device__ constexpr int zshift_offset(int n, int m) {
    return n * (n + 1) * (n + 2) / 6 + m * (n + 1) - m * (m - 1) / 2;
}
constexpr int kZShiftSize = zshift_offset(kMaxP + 1, 0);

inline size_t swap_cos_offset(int n) { return (size_t)n * (n + 1) * (2 * n + 1) / 6; }  // sum_{k<n}(k+1)^2
inline size_t swap_sin_offset(int n) { return (size_t)(n - 1) * n * (2 * n - 1) / 6; }  // sum_{k<n} k^2

// Tree arrays (device), nodes numbered level by level, key order inside a level.
// Kernels take the node count and the level ranges from device memory (dnn,
// dls: written by the tree build), so one launch sequence serves any tree up
// to the sizes the host used for the grids: the exact sizes of this tree in
// an ordinary solve, planned capacities when the solve is replayed from a
// captured CUDA graph.
struct TreeView {
    int n;
    int nnodes;   // grid size of per-node launches (>= *dnn)
    int nlevels;  // levels launched by per-level loops (>= the tree's)
    int leaf_size;
    int nroots;   // grid size for the roots (>= the number of trees)
    int lvl_cnt[kMaxLevel + 2];  // grid size of per-level launches, level L
    const int* dnn;  // device: number of nodes
    const int* dls;  // device: level_start[0 .. kMaxLevel + 1]
    const int* level;
    const int* begin;
    const int* end;
    const int* parent;
    const int* first_child;
    const int* nchild;
};

// Every kernel launch of the library calls note_launch(); fmm_get_stats
// reports the count of the last solve.
void note_launch();

// Streaming multiprocessors of the current device (queried once per device).
// Persistent and grid-stride kernels size their grids as a multiple of it.
int device_sm_count();

// Raise func's dynamic shared-memory limit to `bytes` on the current device.
// cudaFuncSetAttribute acts on the current device only, so this is done once
// per (device, function) pair, under a lock, and remembered.
cudaError_t ensure_dyn_smem(const void* func, int bytes);

// Message returned by fmm_last_error(NULL) (entry points without a context).
void set_global_error(const char* msg);

// ---------------------------------------------------------------- sort.cu
// Stable LSD radix sort of 64-bit keys (optionally with 32-bit values) on
// bits [lo_bit, bits): keys equal there keep their input order. Ping-pongs
// between buffers; returns 1 if the sorted data ends in (k1, v1), 0 if in
// (k0, v0). hist needs radix_hist_words(n) words. dn (device, may be NULL):
// the grid covers n keys but only the first min(n, *dn) are sorted (a count
// known on the device only, in a captured solve).
size_t radix_hist_words(int64_t n);
int radix_sort(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n, int bits,
               uint32_t* hist, cudaStream_t st, const unsigned long long* dn = nullptr, int lo_bit = 0);
// The same for 32-bit keys without payload.
int radix_sort32(uint32_t* k0, uint32_t* k1, int64_t n, int bits, uint32_t* hist, cudaStream_t st,
                 const unsigned long long* dn = nullptr, int lo_bit = 0);
// single-block exclusive scan of count uint32 values in place; total -> *total (device)
void scan_exclusive_u32(uint32_t* data, int64_t count, uint32_t* total, cudaStream_t st);
// the same for large tables (multi-block); scratch: scan_scratch_words(count) words
size_t scan_scratch_words(int64_t count);
void scan_exclusive_u32_large(uint32_t* data, int64_t count, uint32_t* total, uint32_t* scratch,
                              cudaStream_t st);

// ---------------------------------------------------------------- tree.cu
struct TreeBuffers {
    // inputs
    const double *x, *y, *z, *m;
    int64_t n;
    int leaf_size;
    int nclusters;               // independent clusters (a forest); 1 for one cluster
    const int* coff;             // device, nclusters + 1 body offsets of the clusters
    // scratch / outputs
    double* bbox_part;           // 6 * bbox_partials(nclusters)
    double* box;                 // 8 per cluster: centre, h, lower corner, size
    uint64_t *k0, *k1;
    uint32_t *v0, *v1;
    uint64_t *ck0, *ck1;         // cluster pass of the sort (nclusters > 1)
    uint32_t *cv0, *cv1;
    uint32_t* cid;               // cluster of every sorted body (nclusters > 1)
    uint32_t* hist;
    double *xs, *ys, *zs, *ms;   // sorted bodies
    float4* xf;                  // cube-centred FP32 coordinates + mass (scalar-force estimate)
    int8_t *lcp, *win;           // per body
    uint8_t* hi;
    uint32_t* chunk_cnt;         // 23 * nchunks (+1 total)
    int *level, *begin, *end, *parent, *first_child, *nchild;
    int64_t node_cap;
    DevScalars* ds;
};
// keys -> sort -> gather -> node-start counts and their scan; the node
// total lands at chunk_cnt[22 * nchunks]. sorted_in_1 tells where the sorted
// keys/perm ended up.
void tree_build_count(TreeBuffers& b, int* sorted_in_1, cudaStream_t st);
// Exact coincidence check of all n sorted bodies (for key runs longer than
// the bounded scan of k_lcp): sorts a 64-bit hash of (cluster, position) with
// the body index through (hk0, hv0) / (hk1, hv1) and compares bodies with
// equal hashes exactly; sets kErrCoincident in ds->err.
void coincident_exact(const TreeBuffers& b, uint64_t* hk0, uint32_t* hv0, uint64_t* hk1, uint32_t* hv1,
                      cudaStream_t st);
// doubles (times 6) of the bounding-cube partials for nclusters clusters
int bbox_partials(int nclusters);
// node level/begin arrays and ds->level_start, ds->nnodes
void tree_build_emit(TreeBuffers& b, cudaStream_t st);
int tree_nchunks(int64_t n);
void tree_build_phase2(TreeBuffers& b, const uint64_t* keys, int nnodes, const int* h_level_start,
                       int nlevels, cudaStream_t st);
// Cell geometry (Sec. 2.3 readings): M, S, z (centre of mass), r (size).
void cell_geometry(const TreeView& t, const double* xs, const double* ys, const double* zs,
                   const double* ms, const int* h_level_start, double* M, double* S, double* zc,
                   double* r, cudaStream_t st);

// ---------------------------------------------------------------- walk.cu
struct WalkBuffers {
    int2 *front0, *front1;
    int64_t front_cap;
    int2* out[4];          // far, near, m2l, p2p
    int64_t out_cap[4];
    // look-back records of the ordered appends, zeroed when allocated; each
    // walk first clears those the previous walk used. kWalkScanWords words
    // per tile of the largest frontier
    unsigned long long* scan;
    int64_t scan_tiles;
    int stall_lookback = 0;  // test hook: the look-back waits for records no tile writes
};
constexpr int kWalkThreads = 256;    // threads of a walk block
#ifndef GBFMM_WALK_IPT
#define GBFMM_WALK_IPT 4
#endif
constexpr int kWalkIPT = GBFMM_WALK_IPT;  // frontier pairs per thread
constexpr int kWalkTile = kWalkThreads * kWalkIPT;  // frontier pairs per tile (one block)
constexpr int kWalkScanWords = 3;    // per tile: one record per counter (next frontier, accepted, leaf)
inline int64_t walk_scan_tiles(int64_t front_cap) { return front_cap / kWalkTile + 2; }
// Dual-tree walk from (root, root). mode 0: theta < 1 (lists far/near);
// mode 1: the error-controlled MAC (lists m2l/p2p). Returns iterations or a
// negative fmm_status. Counts land in ds->list_cnt.
constexpr int kWalkBadIndex = -100;  // dual_tree_walk: a frontier entry out of range
// M: cell masses, soft: Plummer softening length (0: Newtonian MAC)
int dual_tree_walk(int mode, const TreeView& t, const double* zc, const double* r, const double* P,
                   const float* fmin, int p, double eps, const double* binom_row, const float4* zhi,
                   const float4* zlo, const float* r32, const float* Phat, const double* M, double soft,
                   WalkBuffers& wb, DevScalars* ds, DevScalars* h_ds, int fixed_iters, cudaStream_t st);
// a walk run for a planned nit steps must have an empty frontier after them
// (else kErrCapacity)
void walk_check_finished(DevScalars* ds, int nit, cudaStream_t st);
// Scalar-force estimate f (Sec. 2.3) from the theta-walk lists given as
// per-target CSR (source cell of every entry, sources ascending per target).
void scalar_force(const TreeView& t, const double* zc, const double* M, const float4* xf,
                  const uint32_t* far_src, const uint32_t* far_off, const uint32_t* near_src,
                  const uint32_t* near_off, const int* h_level_start, double soft, float* farf,
                  float* f, float* fmin, cudaStream_t st);
// directed entries of a pair list: (B<-A) and (A<-B), a self pair once and a
// marker that sorts last; np: the device count of pairs, npcap >= *np the
// pairs the grid covers; *nkeys (device) <- 2 min(*np, npcap), the keys written.
void pairs_to_directed(const int2* pairs, const unsigned long long* np, int64_t npcap, int nb, uint64_t* keys,
                       unsigned long long* count, unsigned long long* nkeys, cudaStream_t st);
// 32-bit keys (when 2 nb <= 32); directed_offsets_src32 turns the sorted keys
// into source indices and CSR offsets.
void pairs_to_directed32(const int2* pairs, const unsigned long long* np, int64_t npcap, int nb, uint32_t* keys,
                         unsigned long long* count, unsigned long long* nkeys, cudaStream_t st);
// Sorted directed keys -> src (the source cell of every entry; 0xffffffff for
// the markers past the end) and the CSR offsets per target (nnodes + 1,
// nnodes = *dnn). dnk (device): the keys present, of the nkeys the grid covers.
void directed_offsets_src32(const uint32_t* k32, int64_t nkeys, const unsigned long long* dnk, int nb,
                            const int* dnn, uint32_t* src, uint32_t* off, cudaStream_t st);
void directed_offsets(const uint64_t* keys, int64_t nkeys, const unsigned long long* dnk, int nb, const int* dnn,
                      uint32_t* src, uint32_t* off, cudaStream_t st);

// ---------------------------------------------------------- expansions.cu
void upload_expansion_tables(const HostTables& h);
// Hat scale s_k of every node: its size r_k, floored at kHatFloor times the
// size of its tree's root so that no cell (a single body has r = 0) gets a scale so small
// that its FP32 local coefficients F s^n fall into the denormal range.
constexpr double kHatFloor = 0x1p-40;
void hat_scales(const TreeView& t, const int* parent, const double* r, double* hs, cudaStream_t st);
// Hat multipoles in FP64: P2M at leaves, M2M level by level; P_k per node.
// dword: the P2M and M2M arithmetic runs in double-word FP32 (mixed precision).
// r: node sizes (the walk's FP32 copy r32 is written from them); hs: hat scales.
void upward_pass(const TreeView& t, const int* h_level_start, int p, const double* xs,
                 const double* ys, const double* zs, const double* ms, const double* zc,
                 const double* r, const double* hs, const double* geo, double* mult, double* Pk, float* Phat,
                 float* r32, double* contrib, const DevTables& tb, bool dword, cudaStream_t st);
// hat P2M of the leaves with per-body weights w (in place of masses); dword:
// double-word FP32 arithmetic (mixed precision) instead of FP64
void p2m_weights(const TreeView& t, int p, const double* xs, const double* ys, const double* zs, const double* w,
                 const double* zc, const double* hs, double* mult, const DevTables& tb, bool dword, cudaStream_t st);
// hat multipoles (order p) of the point dipoles of each leaf from the order
// p - 1 hat moments X, Y, Z of their x, y, z components (the jerk's chi field)
void dipole_moments(const TreeView& t, int p, const double* X, const double* Y, const double* Z, const double* hs,
                    double* mult, cudaStream_t st);
// The geometry of every node's shift to its parent, kShiftGeo doubles per
// node: cos phi, sin phi, cos theta, sin theta of b = z_C - z_P, |b| / s_P and
// s_C / s_P (FP64, one thread per node); read by the M2M and L2L kernels.
constexpr int kShiftGeo = 6;
void shift_geometry(const TreeView& t, const double* zc, const double* hs, double* geo, cudaStream_t st);
// rotation-accelerated M2M of one level: the children (level L + 1) into their
// parents (level L); contrib: (p+1)^2 doubles per node (scratch); dword:
// double-word FP32 arithmetic instead of FP64
void m2m_level(const TreeView& t, int L, int p, const double* geo, double* mult, double* contrib,
               const DevTables& tb, bool dword, cudaStream_t st);
// rotation-accelerated L2L of one level: the locals of the nodes of level L
// gain their parents' shifted locals; loc: FP32 (fp32) or FP64 (p+1)^2 per node
void l2l_level(const TreeView& t, int L, int p, const double* geo, void* loc, const DevTables& tb, bool fp32,
               cudaStream_t st);
void multipoles_to_f32(const double* mult, float* mult32, const TreeView& t, int nr, cudaStream_t st);
// FP32 copy with each node's vector padded to `stride` floats (zeros after nr)
void multipoles_to_f32_padded(const double* mult, float* mult32, const TreeView& t, int nr, int stride,
                              cudaStream_t st);
// double-float node centres (hi, lo) and the FP32 hat scale in zhi.w
void node_centres_f32(const TreeView& t, const double* zc, const double* hs, float4* zhi, float4* zlo,
                      cudaStream_t st);
// per-node minimum of the scalar-force estimate (leaves over bodies, then levels upward)

// L2L level by level (FP64 or FP32 locals).
void downward_pass_f64(const TreeView& t, const int* h_level_start, int p, const double* zc,
                       const double* hs, const double* geo, double* loc, const DevTables& tb, cudaStream_t st);
void downward_pass_f32(const TreeView& t, const int* h_level_start, int p, const double* zc,
                       const double* hs, const double* geo, float* loc, const DevTables& tb, cudaStream_t st);

// ----------------------------------------------------------------- m2l.cu
// Rotation-accelerated M2L (Sec. 2.4), gathered per target over the sorted
// directed list; writes the locals of every node (zero without sources).
// queue: a device counter, zeroed here; warps take target cells (below *dnn) from it.
void m2l_f64(const int* dnn, int p, const uint32_t* src, const uint32_t* off,
             const double* mult, const double* zc, const double* hs, double* loc,
             const DevTables& tb, unsigned* queue, cudaStream_t st);
void m2l_f32(const int* dnn, int p, const uint32_t* src, const uint32_t* off,
             const float* mult, const float4* zhi, const float4* zlo, float* loc, unsigned* queue,
             cudaStream_t st);
bool m2l32_supported(int p);

// ----------------------------------------------------------------- p2p.cu
#ifndef GBFMM_LEAVES_PER_ITEM
#define GBFMM_LEAVES_PER_ITEM 128
#endif
constexpr int kLeavesPerItem = GBFMM_LEAVES_PER_ITEM;  // source leaves per P2P work item
void upload_leaf_tables(const HostTables& h);
// Leaf evaluation: P2P over bounded work items (target leaf, up to
// kLeavesPerItem source leaves) written as per-body partials, then per body
// L2P of its leaf's local expansion plus its partials in item order; G-scaled
// results go to the caller's arrays through perm.
struct LeafArgs {
    TreeView t;
    int p;
    double G;
    const double *xs, *ys, *zs, *ms;
    const double *zc, *hs;  // node centres and hat scales
    const float4 *zhi, *zlo;  // double-float node centres; zhi.w = hat scale
    const uint32_t* p2p_src;  // source leaf of every directed P2P entry, ascending per target
    const uint32_t* p2p_off;
    const uint32_t* perm;
    double *ax, *ay, *az, *pot;
    const void* loc;   // FP64 or FP32 locals
    unsigned long long* interactions;  // directed body-body interactions (added by the P2P kernel)
    uint32_t slots_cap;                // partial slots the buffers hold
    const float4* prel;  // leaf-relative FP32 bodies (mixed)
    double2 *part_hi, *part_lo;  // P2P partials: (ax, ay), (az, pot)
    DevTables tb;
    double soft2;  // squared Plummer softening length (0: Newtonian P2P)
    float soft2f;  // the same, rounded to FP32 (mixed P2P)
    unsigned* err;      // kErr* bits (a bounded wait that ran out: kErrTimeout)
    bool bulk;          // FP32 P2P: stage source leaves by bulk copies (unless FMM_FLAG_P2P_LOADS)
    uint32_t tx_extra;  // test hook: bytes a bulk-copy wait expects beyond those copied (0)
};
void leaf_items_plan(const TreeView& t, const uint32_t* p2p_off, uint32_t* item_first, uint32_t* slot_first,
                     uint32_t* totals, cudaStream_t st);
// raise kErrCapacity (and run no item) when the item or slot totals exceed the buffers
void leaf_items_check(uint32_t* totals, uint32_t items_cap, uint32_t slots_cap, unsigned* err, cudaStream_t st);
void leaf_items_fill(const TreeView& t, const uint32_t* item_first, int* item_leaf, uint32_t items_cap,
                     int* leaf_of, cudaStream_t st);
// nitems: device count of work items; p2p32: FP32 P2P on leaf-relative
// bodies (else FP64); l2p32: FP32 L2P on FP32 hat locals (else FP64)
void leaf_eval(const LeafArgs& a, bool p2p32, bool l2p32, const int* item_leaf, const uint32_t* item_first,
               const uint32_t* slot_first, const uint32_t* nitems, unsigned* work, const int* leaf_of,
               cudaStream_t st);
void leaf_relative_f32(const TreeView& t, const double* xs, const double* ys, const double* zs,
                       const double* ms, const double* zc, float4* prel, cudaStream_t st);
// Jerk inputs in sorted order: velocities vs (3n, FP64) and v32 (FP32), and
// the dipole weights w = m v (3n).
void jerk_inputs(int n, const uint32_t* perm, const double* ms, const double* vx, const double* vy,
                 const double* vz, double* vs, double* w, float4* v32, cudaStream_t st);
// Jerk of every body: -grad chi from the dipole locals locj, the Hessian of
// the mass locals a.loc times v_i, and the direct jerk over the P2P list (on
// the solve's P2P work items, partials in a.part_hi/part_lo); G-scaled, to
// the caller's order through a.perm.
void jerk_leaves(const LeafArgs& a, bool fp32, const void* locj, const double* vs, const float4* v32,
                 const int* item_leaf, const uint32_t* item_first, const uint32_t* slot_first, const uint32_t* nitems,
                 unsigned* work, const int* leaf_of, double* jx, double* jy, double* jz, cudaStream_t st);
// ------------------------------------------------------------- timestep.cu
// HOLD step sizes: tau_i = min over j != i of the pair step (Appendix A)
void timesteps_f64(int n, const double* x, const double* y, const double* z, const double* vx, const double* vy,
                   const double* vz, const double* m, double G, double eta, bool sym, double* tau, cudaStream_t st);
// ----------------------------------------------------------------- hold.cu
constexpr int kHoldMaxDepth = 60;                  // no set is split below this level
constexpr int kHoldMaxLevels = kHoldMaxDepth + 1;  // frames of the device-resident recursion
constexpr int kHoldSmallMax = 1024;                // largest set evolved inside one block
// set operations of the HOLD integrator (index lists of bodies)
void hold_iota(int n, int* idx, cudaStream_t st);
// out[c * stride + a] = field c of body idx[a] (x, y, z, vx, vy, vz, m);
// masses of a >= zero_from are zeroed (zero_from < 0: none)
void hold_gather(int k, const int* idx, const double* x, const double* y, const double* z, const double* vx,
                 const double* vy, const double* vz, const double* m, double* out, int stride, int zero_from,
                 cudaStream_t st);
// stable split of idx by tau < dt into S (slow) and F (fast); *nfast (device) <- |F|
void hold_split(int k, const int* idx, const double* tau, double dt, uint32_t* flag, uint32_t* scan, int* S, int* F,
                uint32_t* nfast, uint32_t* scratch, cudaStream_t st);
// v[idx[a]] += h (acc[c * stride + a] - sub[c * sub_stride + a]) (sub may be NULL)
void hold_kick(int k, const int* idx, const double* acc, const double* sub, int stride, int sub_stride, double h,
               double* vx, double* vy, double* vz, cudaStream_t st);
void hold_drift(int k, const int* idx, double dt, double* x, double* y, double* z, const double* vx,
                const double* vy, const double* vz, cudaStream_t st);
// evolve(P, dt) of the k <= kHoldSmallMax bodies idx[0..k) at recursion
// level depth, recursion included, in one block with direct FP64 forces (the
// oracle's operations and order); adds its counters to stats (device,
// {kicks, -, direct solves, deepest level (max), splits})
size_t hold_small_smem(int k);
void hold_small(int k, const int* idx, double* x, double* y, double* z, double* vx, double* vy, double* vz,
                const double* m, double G, double soft, double eta, bool sym, double dt, double dt_min, int depth,
                unsigned long long* stats, cudaStream_t st);
// soft: Plummer softening length (0: Newtonian)
void direct_sum_f64(int64_t n, const double* x, const double* y, const double* z, const double* m,
                    double G, double soft, int64_t ntgt, const int64_t* tgt, double* ax, double* ay, double* az,
                    double* pot, cudaStream_t st);

}  // namespace gbfmm
