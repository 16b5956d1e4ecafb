/*
 * gbfmm: GPU fast multipole force solve for collisional star systems.
 *
 * The method is that of Mukherjee, Zhu, Trac & Rodriguez (2021), "Fast
 * Multipole Methods for N-body Simulations of Collisional Star Systems",
 * Section 2: an octree, multipole moments in solid spherical harmonics
 * (Sec. 2.2, Eq. moments), an error-controlled multipole-acceptance
 * criterion built on a scalar-force estimate (Sec. 2.3), a dual-tree walk
 * (Sec. 2.1) emitting M2L and P2P interaction lists, the rotation-accelerated
 * M2L (Sec. 2.4), L2L/L2P, and direct summation for the near field.
 *
 * Problem (Sec. 2.3, Sec. 3.1.1): given N bodies with positions x_i and masses
 * m_i, compute a_i = G sum_{j != i} m_j (x_j - x_i)/|x_j - x_i|^3 and
 * phi_i = -G sum_{j != i} m_j/|x_j - x_i|, approximately, with the expansion
 * order p and the tolerance eps of the MAC. Optionally with Plummer softening
 * (Appendix B): |x_j - x_i|^2 -> |x_j - x_i|^2 + soft^2 in both sums.
 *
 * Conventions for every call:
 *  - All array arguments of fmm_solve/fmm_solve_batch are DEVICE pointers
 *    (cudaMalloc'd or from a tensor on the current device), FP64, one value
 *    per body, in the caller's order; outputs are written in the same order.
 *    The caller owns them; the library never frees or keeps them.
 *  - The library owns its workspace inside the context, grows it on demand
 *    and frees it in fmm_destroy.
 *  - All GPU work is issued on the caller's stream (NULL = legacy default).
 *    Calls return when the outputs are complete on that stream's timeline:
 *    the library synchronises the stream internally (it reads back tree and
 *    list sizes).
 *  - Every call returns an fmm_status; fmm_last_error() gives a message. On
 *    error the outputs are unspecified and the context stays usable. The
 *    library never aborts and never traps on the device.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef GBFMM_H
#define GBFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FMM_OK = 0,
    FMM_ERR_ARG = -1,        /* invalid argument (n < 0, p outside [1, 30], eps < 0, ...) */
    FMM_ERR_CUDA = -2,       /* a CUDA runtime call failed */
    FMM_ERR_OOM = -3,        /* device allocation failed */
    FMM_ERR_NONFINITE = -4,  /* a position or mass is NaN or infinite, or a mass is <= 0 */
    FMM_ERR_COINCIDENT = -5, /* two bodies share exactly the same position */
    FMM_ERR_CAPACITY = -6,   /* an internal list outgrew its capacity after one regrow */
    FMM_ERR_TIMEOUT = -7     /* a bounded device-side wait ran out (the P2P's bulk-copy
                                staging); the context stays usable */
} fmm_status;

typedef enum {
    FMM_PRECISION_FP64 = 0,  /* every expansion and pair sum in FP64 */
    FMM_PRECISION_MIXED = 1  /* M2L, L2L, L2P and P2P in FP32 on scaled / cell-relative
                                values with compensated or FP64 accumulation; tree,
                                multipoles for the MAC and the walk in FP64 */
} fmm_precision;

/* fmm_config.flags bits */
#define FMM_FLAG_FP64_LOCALS 1u /* mixed precision only: M2L, L2L and L2P run in FP64 on FP64
                                   multipole and local coefficients, P2P stays FP32 (the split
                                   "FP64 coefficients for the high orders"); slower */
#define FMM_FLAG_P2P_LOADS 2u   /* FP32 P2P: stage the source bodies into shared memory by per-lane
                                   loads instead of the default, one bulk copy (cp.async.bulk) per
                                   source leaf completing on an mbarrier. Same results. The bulk
                                   copies' waits are bounded (about one second); one that runs out
                                   makes the call return FMM_ERR_TIMEOUT. */

typedef struct {
    int p;                 /* expansion order, 1..30 (swap matrices are tabulated to 30, Sec. 2.4) */
    double eps;            /* MAC tolerance epsilon of Sec. 2.3, >= 0 (0: never accept, all P2P) */
    int leaf_size;         /* split a cell while it holds more than leaf_size bodies, 1..256 */
    int precision;         /* fmm_precision */
    double G;              /* gravitational constant (Henon units: 1) */
    unsigned flags;        /* FMM_FLAG_* bits (0: none); unknown bits are rejected */
    unsigned fault_inject; /* test hook, 0 in production: bit 0 forces tiny list capacities
                              so the capacity-regrow path runs; bit 1 makes every bulk-copy wait
                              of the FP32 P2P expect 16 bytes that never come, so it runs out
                              and the call returns FMM_ERR_TIMEOUT; bit 2 makes the walk's
                              look-back wait for records no tile writes, with the same outcome */
    double soft;           /* Plummer softening length eps_soft >= 0 (Appendix B; 0: Newtonian).
                              P2P, fmm_direct and the near part of the scalar-force estimate
                              use the softened kernel; the far field stays the expansion of
                              1/r, and the MAC adds the bound 1.5 M_A soft^2 / d_min^4
                              (d_min = r - r_A - r_B) on what that leaves out, so accepted
                              pairs keep the error within eps. Coincident bodies are still
                              rejected (the octree cannot separate them). */
} fmm_config;

typedef struct {
    int64_t n;              /* bodies in the last solve */
    int32_t nnodes, nleaves, nlevels;
    int64_t n_far, n_near;  /* pair counts of the theta < 1 walk (scalar-force estimate) */
    int64_t n_m2l, n_p2p;   /* pair counts of the eps walk (unordered pairs, self pairs in P2P) */
    int64_t p2p_interactions; /* directed body-body interactions evaluated */
    double ms_tree, ms_upward, ms_estimate, ms_walk, ms_m2l, ms_downward, ms_leaf, ms_total;
    int32_t walk_iters, regrows;
    int64_t kernel_launches;  /* kernels the library launched in the last solve */
    int32_t graph_replays;    /* 1 if the last fmm_solve_graph call replayed its captured graph */
    int32_t reserved;
    double ms_jerk;           /* the jerk pass of the last fmm_solve_jerk (0 otherwise) */
} fmm_stats;

typedef struct fmm_ctx fmm_ctx;

/* Create a context for the current CUDA device. Validates cfg (FMM_ERR_ARG)
 * and uploads the swap matrices and coefficient tables. *out is NULL on error. */
int fmm_create(fmm_ctx** out, const fmm_config* cfg);

/* Release every device and host resource of the context. NULL is allowed. */
void fmm_destroy(fmm_ctx* ctx);

/* One force solve (Sec. 2.1, Fig. 1): tree, P2M/M2M, scalar-force estimate,
 * error-controlled walk, M2L/L2L/L2P and P2P. x, y, z, m: n device FP64
 * values each; ax, ay, az, pot: n device FP64 outputs (pot may be NULL).
 * n = 0 is a no-op. */
int fmm_solve(fmm_ctx* ctx, int64_t n, const double* x, const double* y, const double* z,
              const double* m, double* ax, double* ay, double* az, double* pot, void* cuda_stream);

/* The same solve from HOST buffers: copies the inputs in, solves, copies the
 * outputs back, all on cuda_stream; returns when the host outputs are final.
 * Host buffers may be pageable or pinned. */
int fmm_solve_host(fmm_ctx* ctx, int64_t n, const double* x, const double* y, const double* z,
                   const double* m, double* ax, double* ay, double* az, double* pot, void* cuda_stream);

/* Independent solves of nclusters clusters stored back to back: cluster c
 * holds bodies [offsets[c], offsets[c+1]) (offsets: HOST array of
 * nclusters + 1 non-decreasing values, offsets[0] = 0; empty clusters are
 * allowed; at most 2^30 bodies in all). Bodies of different clusters do not
 * interact. Device arrays as in fmm_solve. The ensemble is solved as one
 * forest in a single pipeline pass (one launch of each kernel for all
 * clusters); each cluster's tree, interaction lists and forces are exactly
 * those of a separate fmm_solve of that cluster with the same config.
 * Statistics and exports then describe the whole forest. The paper's tests
 * (Sec. 3) average over many independent realizations of a cluster, each a
 * separate run; the single pass over all of them is this library's addition. Errors: FMM_ERR_ARG for bad offsets or NULL pointers,
 * otherwise as fmm_solve (a coincidence is only checked inside a cluster). */
int fmm_solve_batch(fmm_ctx* ctx, int32_t nclusters, const int64_t* offsets, const double* x,
                    const double* y, const double* z, const double* m, double* ax, double* ay,
                    double* az, double* pot, void* cuda_stream);

/* The solve of fmm_solve (offsets == NULL) or fmm_solve_batch (nclusters
 * clusters, HOST offsets as there) replayed from a captured CUDA graph. The
 * first call for a set of arguments is an ordinary solve (its result is
 * returned), which also plans capacities from the sizes it met (nodes, nodes
 * per level and levels, walk steps, list lengths, P2P work items, each with
 * headroom) and captures the whole solve, with no read-back, into one CUDA
 * graph on an internal stream. Later calls with the same n, offsets and
 * pointers replay the graph: one launch, then one read of a status block.
 * If the bodies moved enough that a planned capacity is exceeded (or the
 * tree got deeper), that call falls back to an ordinary solve and the next
 * call plans and captures again; the result is always that of fmm_solve.
 * Any reallocation of the context's workspace (another solve of a larger
 * problem on the same context) also forces a new capture.
 * cuda_stream is synchronised before the solve; the call returns with the
 * outputs complete. The paper has no counterpart (it is a CPU code); this is
 * the GPU way to remove per-phase launch and read-back costs from repeated
 * solves of the same bodies (time steps) or ensembles. Statistics after a
 * replay carry the counts from the status block and graph_replays = 1;
 * the per-phase times come from event nodes inside the graph and ms_total
 * is the whole replay. Exports after a
 * replay are not supported. Errors as fmm_solve and fmm_solve_batch. */
int fmm_solve_graph(fmm_ctx* ctx, int32_t nclusters, const int64_t* offsets, int64_t n, const double* x,
                    const double* y, const double* z, const double* m, double* ax, double* ay,
                    double* az, double* pot, void* cuda_stream);

/* The solve of fmm_solve plus the jerk, the time derivative of the
 * acceleration for bodies moving with velocities (vx, vy, vz):
 * j_i = G sum_{j != i} m_j [v_ij / r^3 - 3 (r_ij . v_ij) r_ij / r^5],
 * r_ij = x_j - x_i, v_ij = v_j - v_i (Plummer-softened like P2P when soft > 0).
 * The paper (Sec. 6) computes jerks within the FMM after Dehnen (2014) for
 * Hermite integrators; the form here: j_i = G [-grad chi(x_i) + H(x_i) v_i
 * + near_i], with chi the potential of point dipoles m_j v_j, expanded on
 * the same tree and interaction lists (one more P2M/M2M/M2L/L2L pass, in
 * the context's precision), H the Hessian of the solve's own local
 * expansion, and near_i the direct jerk over the P2P leaf pairs. The lists
 * come from the acceleration's MAC, so the jerk's error is not controlled
 * by eps directly (measured: it tracks eps within a small factor).
 * All arrays are device pointers of n FP64 values in the caller's order
 * (pot may be NULL). Errors as fmm_solve. */
int fmm_solve_jerk(fmm_ctx* ctx, int64_t n, const double* x, const double* y, const double* z, const double* vx,
                   const double* vy, const double* vz, const double* m, double* ax, double* ay, double* az,
                   double* pot, double* jx, double* jy, double* jz, void* cuda_stream);

/* Plain FP64 O(N * ntargets) direct sum at the given target indices (a
 * device int64 array, or NULL for all n bodies): the exact quantity the FMM
 * approximates (Sec. 3.1.1), used to measure force errors. 1/r comes from an
 * FP32 seed refined by two Newton steps, to FP64 rounding; a body exactly on
 * top of the target contributes nothing. */
int fmm_direct(fmm_ctx* ctx, int64_t n, const double* x, const double* y, const double* z,
               const double* m, int64_t ntargets, const int64_t* targets, double* ax, double* ay,
               double* az, double* pot, void* cuda_stream);

/* Step sizes of the HOLD integrator (Appendix A) for n bodies (device FP64
 * arrays): tau_i = min over j != i of min(eta sqrt(r^3 / (G (m_i + m_j))),
 * eta r / v), r and v the pair's separation and relative speed (the
 * free-fall and fly-by times). symmetrize != 0: each time is divided by
 * (1 - tau'/2) (Eq. step_symm), tau' its time derivative along the two-body
 * motion, capped at 1. O(n^2), FP64, reproducible bit for bit. A single body
 * gets +infinity. Errors: FMM_ERR_ARG for n out of range, eta <= 0 or NULL
 * pointers. */
int fmm_timesteps(fmm_ctx* ctx, int64_t n, const double* x, const double* y, const double* z, const double* vx,
                  const double* vy, const double* vz, const double* m, double eta, int32_t symmetrize, double* tau,
                  void* cuda_stream);

/* nsteps steps of the HOLD integrator (Appendix A, after Pelupessy et al.
 * 2012) on n bodies, positions and velocities updated in place (device FP64
 * arrays; masses m). evolve(P, dt): split the set P into fast bodies (their
 * fmm_timesteps step size within P below dt) and slow ones; evolve the fast
 * system for dt/2; kick (dt/2), drift (dt) and kick (dt/2) the slow system
 * H_S = T_S + V_SS + V_FS (slow bodies feel all of P, fast ones the slow
 * ones); evolve the fast system for dt/2. Below dt_min (or 60 levels) a set
 * is not split further. Forces: FP64 direct sum for sets of fewer than
 * direct_below bodies, else the context's FMM solve; G and the softening
 * from the context. A set of at most device_below bodies (0..1024; and
 * fewer than direct_below) evolves inside one GPU block, its whole recursion
 * included, with no host round trip: its direct forces are the oracle's
 * (1 / (r^2 sqrt(r^2)), no fused multiply-add, sources in set order), so
 * such runs reproduce the oracle's trajectory bit for bit; 0 keeps every
 * level on the host-driven path. stats (host, may be NULL): {slow-system
 * kicks, FMM solves, direct solves, deepest level, splits}. Errors as
 * fmm_solve, and FMM_ERR_ARG for dt <= 0, eta <= 0, dt_min < 0, nsteps < 0
 * or device_below outside [0, 1024]. */
int fmm_hold(fmm_ctx* ctx, int64_t n, double* x, double* y, double* z, double* vx, double* vy, double* vz,
             const double* m, double dt, int64_t nsteps, double eta, int32_t symmetrize, double dt_min,
             int64_t direct_below, int64_t device_below, int64_t* stats, void* cuda_stream);

/* Statistics of the last solve. */
int fmm_get_stats(const fmm_ctx* ctx, fmm_stats* out);

/* Export the octree of the last solve to HOST buffers, for parity tests.
 * keys/perm: n values (Morton keys in sorted order; perm[i] = caller index of
 * the i-th sorted body). Node arrays: nnodes values each, nodes numbered level
 * by level and in key order within a level. Any pointer may be NULL. */
int fmm_export_tree(const fmm_ctx* ctx, uint64_t* keys, int64_t* perm, int32_t* level,
                    int32_t* begin, int32_t* end, int32_t* parent, int32_t* first_child,
                    int32_t* nchild);

/* Export per-node geometry of the last solve to HOST buffers (any may be NULL):
 * M (nnodes), z (3*nnodes, centre of mass), r (nnodes, cell size), P
 * (nnodes*(p+1), degree norms of Sec. 2.3), fmin (nnodes, minimum scalar-force
 * estimate), f (n, per sorted body). */
int fmm_export_geometry(const fmm_ctx* ctx, double* M, double* z, double* r, double* P,
                        float* fmin, float* f);

/* Export an interaction list of the last solve to HOST memory: which = 0 far
 * pairs and 1 near pairs of the theta < 1 walk, 2 M2L pairs and 3 P2P pairs of
 * the eps walk; pairs: 2*count int32 (A, B), in the library's own order.
 * *count receives the number of pairs; pairs may be NULL to query it. */
int fmm_export_pairs(const fmm_ctx* ctx, int which, int64_t* count, int32_t* pairs);

/* Export the swap-matrix table (degrees 0..30, layout of the generator: cosine
 * blocks then sine blocks) to HOST memory; ncos/nsin receive the counts. */
int fmm_export_swap(int64_t* ncos, int64_t* nsin, double* cos_blocks, double* sin_blocks);

/* Bounding cube, Morton keys and their sort for up to 262144 bodies, with
 * no device allocation: the paper has no counterpart (it is a service for
 * callers that cannot call cudaMalloc, e.g. under a device-memory budget owned
 * by another allocator, or in a loop where an allocation's latency or failure
 * is not acceptable).
 * x, y, z: n device FP64 positions. The inputs, the outputs and the stream
 * must belong to the current CUDA device: the call takes its scratch and
 * launches its kernels there. Outputs (device): keys[n] sorted Morton
 * keys, perm[n] the caller index of each sorted body (ties keep input order),
 * box[4] (may be NULL) the cube centre and half-size. These are exactly the
 * keys and permutation fmm_solve builds its octree from.
 * Scratch: a static device array of about 4.3 MB in the library, held by every
 * GPU that loads it until the process exits. The first call on a device looks
 * up the array's address (cudaGetSymbolAddress), so make that first call
 * before any stream capture. All calls share the array: calls that overlap on
 * the GPU (other streams, other host threads) race. The call synchronises its
 * stream before returning.
 * Errors: FMM_ERR_ARG for n outside [0, 262144] or NULL pointers,
 * FMM_ERR_NONFINITE for a NaN or infinite position, FMM_ERR_CUDA; the message
 * is fmm_last_error(NULL). */
int fmm_morton_sort_noalloc(int64_t n, const double* x, const double* y, const double* z,
                            uint64_t* keys, int64_t* perm, double* box, void* cuda_stream);

/* Measured FMA throughput of the current device, the denominator of the
 * arithmetic rooflines of the solve's kernels (M2L and P2P run on the FP32
 * pipe in mixed precision and on the FP64 pipe in FP64 mode). The paper has
 * no counterpart: it is a measurement utility. precision: FMM_PRECISION_MIXED
 * times FP32 FMAs, FMM_PRECISION_FP64 FP64 FMAs; independent FMA chains on
 * every lane of a full grid, one launch grown to last about target_ms
 * (0 < target_ms <= 10000), the best of three such launches timed with CUDA
 * events on cuda_stream. *tflops receives 2 x FMAs / s / 1e12. Allocates and
 * frees a small device buffer; synchronises the stream. Errors: FMM_ERR_ARG,
 * FMM_ERR_OOM, FMM_ERR_CUDA (message in fmm_last_error(NULL)). */
int fmm_fma_peak(int precision, double target_ms, double* tflops, void* cuda_stream);

/* Message of the last error on this context (or of the last failed
 * fmm_create when ctx is NULL). Never NULL. */
const char* fmm_last_error(const fmm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GBFMM_H */
