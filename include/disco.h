/*
 * disco.h - C ABI of the GB300 (sm_103a) DiscoMatch dual / primal solver.
 *
 * Problem (Sec. 3.1, Eq. P): match two closed, consistently oriented triangle meshes X and
 * Y by a binary ILP over product triangles ("matching elements": triangle-triangle,
 * triangle-edge, triangle-vertex), min c^T x s.t. closedness rows A^d x = 0 and projection
 * rows A^X x = 1, A^Y x = 1. Each row becomes a BDD (Sec. 3.2, App. A.3); the solver runs
 * the Lagrange-decomposition dual (Eq. D) by deferred min-marginal averaging on the GPU and
 * rounds a feasible x from min-marginal signs (App. A.5, Sec. 3 pipeline).
 *
 * Conventions for every entry point:
 *   - Return value: DISCO_OK (0) or a negative DISCO_ERR_*; no exceptions cross the ABI and
 *     no call aborts the process. disco_strerror() names a code; disco_last_error() gives
 *     the calling thread's most recent message.
 *   - Pointers documented "host or device" may be either; the library asks the CUDA driver
 *     which (cudaPointerGetAttributes) and copies as needed. Pointers documented "device"
 *     must be device memory of the handle's device. All arrays are dense and row-major.
 *   - Inputs are caller-owned and only read during the call. Outputs are caller-allocated.
 *     Device state is owned by the handle and released by disco_free().
 *   - Work is issued on the handle's stream (disco_opts.stream, a cudaStream_t; 0 = a stream
 *     the library creates). Calls documented "synchronises" wait for that stream.
 *   - A handle must not be used from two threads at once.
 */
#ifndef DISCO_H
#define DISCO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DISCO_ABI_VERSION 1

enum {
    DISCO_OK = 0,
    DISCO_ERR_INVALID_ARG = -1,   /* bad pointer, size or option */
    DISCO_ERR_NONMANIFOLD = -2,   /* a mesh is not a closed, consistently oriented 2-manifold */
    DISCO_ERR_GENUS_MISMATCH = -3,/* Euler characteristics differ: (P) has no solution (Sec. 4) */
    DISCO_ERR_INFEASIBLE = -4,    /* a row of (P) has no solution after presolve */
    DISCO_ERR_PRIMAL_FAILED = -5, /* rounding used all its rounds without a feasible x */
    DISCO_ERR_TIMEOUT = -6,       /* a bounded device or host loop hit its limit */
    DISCO_ERR_CUDA = -7,          /* a CUDA runtime call failed (message in disco_last_error) */
    DISCO_ERR_OOM = -8,           /* device or host allocation failed */
    DISCO_ERR_NOT_READY = -9,     /* call order violated (e.g. primal before any dual pass) */
    DISCO_ERR_RANGE = -10,        /* a mass removed by a dual update left the range of the
                                     fixed-point averaging sums (see disco_dual): costs far too
                                     large for normalize_costs = 0, or a diverging dual */
    DISCO_ERR_INTERNAL = -11      /* bounds-checking build only: a kernel index fell outside its
                                     array; the access was skipped and the results are void */
};

/* A triangle mesh: nv vertices (V: nv*3 float, may be NULL: positions are not used by the
 * solver) and nt triangles (T: nt*3 int32 vertex indices, counter-clockwise). Host memory. */
typedef struct {
    int32_t nv;
    int32_t nt;
    const float *V;
    const int32_t *T;
} disco_mesh;

/* Solver options; disco_default_opts() fills the defaults given in brackets. */
typedef struct {
    float omega;              /* [0.5] damping of the min-marginal averaging step */
    int32_t split_chunk;      /* [0] App. A.3 splitting: rows longer than this many layers are
                                 cut into balanced segments; 0 disables */
    int32_t lb_every;         /* [20] iterations between lower-bound checks in disco_converge */
    double conv_rel_tol;      /* [1e-6] disco_converge stops when the bound moved less than
                                 this, relative, over lb_every iterations */
    int32_t primal_rounds;    /* [100] rounding rounds before DISCO_ERR_PRIMAL_FAILED */
    int32_t primal_inner_iters; /* [20] dual iterations between rounding rounds */
    float perturb_delta0;     /* [1e-3] first perturbation of undecided variables */
    float perturb_growth;     /* [2] perturbation growth per round */
    float tie_tau;            /* [1e-6] |M| at or below this counts as undecided */
    int32_t propagate_limit;  /* [10000] max propagation sweeps per rounding round */
    int32_t device;           /* [0] CUDA device ordinal */
    void *stream;             /* [NULL] cudaStream_t to issue work on; NULL = own stream */
    int32_t host_threads;     /* [0] threads for the host compiler; 0 = hardware concurrency */
    int32_t split_max_segments; /* [8] at most this many segments per row when splitting (0 = no
                                 cap): a one-hot chain carries cost information across one cut
                                 per half-pass, so very long rows are cut into longer segments */
    int32_t graph_iters;      /* [10] dual iterations captured once into a CUDA graph and replayed
                                 as a block; 0 = one launch per half-pass and width class. If the
                                 stream cannot be captured the library launches plainly. */
    int32_t autotune;         /* [1] time the launch geometries of the half-pass kernels on the
                                 first dual iterations and keep the fastest; every geometry gives
                                 bit-identical results, so the trial iterations count as normal
                                 iterations. 0 = the default geometry. */
    int32_t normalize_costs;  /* [1] divide the element costs by the largest one (c in [0, 1]);
                                 0 = raw means of the three pair costs (then the bound is linear
                                 in the pair costs' scale) */
    int32_t qn_memory;        /* [0] disco_converge interleaves quasi-Newton steps (Alg. 1) with
                                 its lb_every MMA iterations, keeping this many L-BFGS pairs;
                                 0 = MMA only */
    int32_t cost_model;       /* [0] element costs from the pair costs: 0 = mean of the three pair
                                 costs; 1 = Eq. 2: sum over the corners of (A_X(m_v) + A_Y(n_v))
                                 d(m_v, n_v) with A the mixed vertex areas (Meyer et al. 2003;
                                 needs the meshes' V) and d the pair distances
                                 (disco_pair_distances) */
    int32_t tile_order;       /* [0] order of the warp tiles in the device store (results are the
                                 same, up to the order of the bound's FP64 tile sums): 0 = the
                                 default, which is 1; 1 = width class, then length, over each instance; 2 = blocks
                                 of 4096 segments in mesh-region order (table locality), each
                                 by width class and length */
} disco_opts;

typedef struct {
    int64_t nvars;            /* |P|: matching elements kept by the candidate mask */
    int64_t nrows;            /* rows of (P) */
    int64_t nvars_free;       /* variables left after presolve */
    int64_t nvars_aux;        /* auxiliary variables added by splitting */
    int64_t nbdds;            /* BDD segments */
    int64_t nslots;           /* (BDD, variable) pairs = layers over all BDDs */
    int64_t nnodes;           /* BDD nodes over all layers */
    int64_t max_layers;       /* longest BDD segment (sequential depth of a half-pass) */
    int64_t max_width;        /* widest layer */
    int64_t ntiles;           /* warp tiles of 32 BDD segments */
    int64_t device_bytes;     /* device memory held by the handle */
    int64_t iterations;       /* dual iterations run so far */
    double constant;          /* cost of variables fixed to 1 by presolve */
    double build_ms;          /* host time of disco_build */
    int64_t bytes_per_iter;   /* algorithmic bytes of one iteration (two half-passes) */
    double upload_ms;         /* disco_build time after the host compiler: device store, upload */
    int64_t launch_geometry;  /* warps per block of the half-pass kernels (chosen by the autotuner
                                 or the default) */
    int64_t reserved[3];
} disco_info_t;

typedef struct disco_handle disco_handle;

/* Fills *opts with the defaults. Returns DISCO_OK, or INVALID_ARG for NULL. */
int disco_default_opts(disco_opts *opts);

/*
 * Pair costs (Eq. 2 variant used by the workloads): d[m*nvy + n] = (1/dim) * sum_k
 * (FX[m,k] - FY[n,k])^2, FP32. FX: nvx*dim and FY: nvy*dim, host or device (host arrays are
 * copied in on `stream` through a buffer from the library's device pool; pinned host memory
 * makes the copy asynchronous); d: nvx*nvy, a DEVICE pointer. Asynchronous on `stream`
 * (cudaStream_t, NULL = legacy default stream). Errors: INVALID_ARG, CUDA.
 */
int disco_pair_costs(const float *FX, const float *FY, int32_t nvx, int32_t nvy, int32_t dim,
                     float *d, void *stream);

/* d[m, n] = ||FX[m, :] - FY[n, :]|| (Euclidean; the feature distance of Eq. 2), FP32,
 * row-major nvx x nvy. Same arguments, layout and errors as disco_pair_costs. */
int disco_pair_distances(const float *FX, const float *FY, int32_t nvx, int32_t nvy, int32_t dim, float *d,
                         void *stream);

/*
 * Candidate mask of the top-k pruned product space (Sec. 4 pruning to neighbourhoods of
 * vertex matches): allowed[m*nvy + n] = 1 iff n lies in the closed 1-ring (on Y) of one of
 * the k smallest d[m, .] (ties to the lower index), or m lies in the closed 1-ring (on X)
 * of one of the k smallest d[., n]. Only finite entries are ranked: a row or column with
 * fewer than k finite entries (the rest +inf or NaN) contributes just those. d and allowed
 * are DEVICE pointers; X and Y are host meshes (only T is read). 1 <= k <= 64.
 * Asynchronous on `stream`.
 */
int disco_candidates(const float *d, int32_t nvx, int32_t nvy, int32_t k, const disco_mesh *X,
                     const disco_mesh *Y, uint8_t *allowed, void *stream);

/*
 * disco_candidates without any allocation. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate memory while they run (a fixed device
 * budget owned by another allocator, latency-critical loops that cannot afford an
 * allocation's synchronisation). Same inputs and output as disco_candidates; every
 * temporary lives in one fixed library-owned device array of 3.75 MiB that each device
 * loading the library holds until the process exits. Limits: at most 16384 vertices and
 * 32768 triangles per mesh, 1 <= k <= 32 (and k <= both vertex counts); larger sizes return
 * DISCO_ERR_INVALID_ARG before any GPU work. The first call on a device resolves the
 * array's address (make it before any stream capture) and caches it; a cudaDeviceReset
 * invalidates the cached address, so the entry point must not be called again in that
 * process after one. All calls on a device share the array: calls whose GPU work overlaps
 * race and must be serialised by the caller. Each call clears what it needs and
 * synchronises `stream` before returning.
 */
int disco_candidates_noalloc(const float *d, int32_t nvx, int32_t nvy, int32_t k, const disco_mesh *X,
                             const disco_mesh *Y, uint8_t *allowed, void *stream);

/*
 * Builds the problem and the device BDD store (host compiler + one upload):
 * product space restricted to `allowed` (nvx*nvy uint8, host or device; NULL = full
 * product space), costs c_p = mean of the three pair costs d (nvx*nvy float, host or
 * device) normalised by the largest kept c_p, closedness and projection rows, presolve,
 * BDDs (split per opts->split_chunk), dual initialised at lambda = c / |J_i|.
 * On success *out receives a new handle. Synchronises. Errors: INVALID_ARG, NONMANIFOLD,
 * GENUS_MISMATCH, INFEASIBLE, OOM, CUDA.
 */
int disco_build(const disco_mesh *X, const disco_mesh *Y, const float *d, const uint8_t *allowed,
                const disco_opts *opts, disco_handle **out);

/*
 * Host-only compilation, for inspection (no CUDA call): runs the same compiler as
 * disco_build (split options as in disco_opts) on host arrays d and allowed (allowed may be
 * NULL) and fills *info (iterations,
 * ntiles, device_bytes = 0). Optional outputs, each ignored when NULL or too small:
 *   slot_var[nslots]   variable of every slot in canonical order: a matching-element id,
 *                      or nvars + k for the k-th auxiliary variable of splitting;
 *   slot_width[nslots] node count of every slot's layer;
 *   fixed[nvars]       presolve: -1 free, 0 or 1 fixed.
 * Call once with NULL outputs to learn the sizes. Errors as disco_build.
 */
int disco_compile_host(const disco_mesh *X, const disco_mesh *Y, const float *d, const uint8_t *allowed,
                       int32_t split_chunk, int32_t split_max_segments, disco_info_t *info,
                       int32_t *slot_var, int32_t *slot_width, int64_t nslots, int8_t *fixed,
                       int64_t nvars);

/*
 * Batched build (a serving pattern beside the plain solver; the paper solves one pair at a time): n
 * independent shape pairs in ONE handle and one device store, so that every half-pass of
 * every pair runs in the same kernel launches. X, Y: n meshes each (host); d[i], allowed[i]:
 * per pair as in disco_build (allowed may be NULL, or hold NULL entries). The pairs are
 * compiled on the host side by side. On a batch handle the single-instance calls act on all
 * pairs: disco_dual iterates all of them, disco_lower_bound returns the sum of their bounds,
 * disco_min_marginals / disco_get_state / disco_set_state concatenate the pairs' canonical
 * slots (and variables) in pair order, disco_primal writes the pairs' x one after another
 * (disco_instance_info gives each pair's sizes) and returns the summed cost; disco_info
 * reports totals. Errors as disco_build (the message names the failing pair).
 */
int disco_build_batch(int32_t n, const disco_mesh *X, const disco_mesh *Y, const float *const *d,
                      const uint8_t *const *allowed, const disco_opts *opts, disco_handle **out);

/* Number of pairs in the handle (1 for disco_build). */
int disco_batch_size(disco_handle *h, int32_t *n);

/* Per-pair lower bounds (as disco_lower_bound) into lb[0 .. n). Synchronises. */
int disco_lower_bounds(disco_handle *h, double *lb, int32_t n);

/* Sizes of pair i of the handle (ntiles = its warp tiles). */
int disco_instance_info(disco_handle *h, int32_t i, disco_info_t *info);

/*
 * Rounding of all pairs (as disco_primal). x_out: sum of the pairs' nvars bytes, pair after
 * pair; costs[i] (may be NULL): pair i's c^T x; status[i] (may be NULL): DISCO_OK or
 * DISCO_ERR_PRIMAL_FAILED for pair i. Returns DISCO_OK iff every pair is feasible.
 */
int disco_primal_batch(disco_handle *h, uint8_t *x_out, int64_t nvars, double *costs, int32_t *status,
                       int32_t n);

/* Runs `iters` dual iterations (forward + backward half-pass of deferred min-marginal
 * averaging, Alg. 1 "MMA"). Asynchronous on the handle's stream. */
int disco_dual(disco_handle *h, int32_t iters);

/* Runs `calls` executions of the quasi-Newton powered iteration (Alg. 1): move the deferred
 * means into lambda; subgradient g = per BDD the minimising assignment (per slot 1 iff its
 * min-marginal difference is negative, App. A.5); direction H g by the L-BFGS two-loop
 * recursion (Alg. 5) over the stored pairs, projected so that every variable's entries sum
 * to 0 (Alg. 1, dual feasibility); step size by FindStepSize (Alg. 6, bound evaluations,
 * the step is taken only if it raises the bound); then `mma_iters` MMA iterations; then
 * the pair (s, y) enters the memory if s^T y >= 1e-8 (Alg. 4). Memory size: opts.qn_memory,
 * or 5 if that is 0. The bound never decreases. Synchronises (the step search reads
 * bounds on the host). Errors: DISCO_ERR_INVALID_ARG for negative counts, DISCO_ERR_OOM. */
int disco_dual_qn(disco_handle *h, int32_t calls, int32_t mma_iters);

/* Point map of a matching (triangle matching -> vertex pairs): the distinct vertex pairs
 * (m, n) at the corners of the elements set to 1 in x (x as written by disco_primal, one byte
 * per element of a single-instance handle), sorted by (m, n), written as pairs[2k] = m,
 * pairs[2k+1] = n (host pointer). *count receives the number of pairs; if it exceeds
 * `capacity` nothing is written and DISCO_ERR_INVALID_ARG is returned. */
int disco_point_map(disco_handle *h, const uint8_t *x, int64_t nvars, int32_t *pairs, int64_t capacity,
                    int64_t *count);

/* Coarse-to-fine candidate mask (Sec. 4, coarse-to-fine: fine matchings are kept near the
 * coarse solution): allowed[m', n'] = 1 iff some coarse pair (m, n) of `pairs` (npairs pairs,
 * layout of disco_point_map) has m' within `rings` edges of fine vertex c2f_x[m] on the fine
 * mesh X and n' within `rings` edges of c2f_y[n] on the fine mesh Y. c2f_x / c2f_y map coarse
 * vertex ids to fine ones (host arrays, lengths ncx / ncy). Out: Xf->nv * Yf->nv bytes,
 * row-major, host or device pointer. Host computation; synchronises. Errors:
 * DISCO_ERR_INVALID_ARG (ids out of range, rings < 0). */
int disco_candidates_coarse_to_fine(const int32_t *pairs, int64_t npairs, const int32_t *c2f_x, int32_t ncx,
                                    const int32_t *c2f_y, int32_t ncy, int32_t rings, const disco_mesh *Xf,
                                    const disco_mesh *Yf, uint8_t *allowed);

/* Lower bound E(lambda + pend) + presolve constant of Eq. D, FP64 sum. Synchronises. */
int disco_lower_bound(disco_handle *h, double *lb);

/*
 * Iterates until the lower bound changed by less than opts.conv_rel_tol (relative) over
 * opts.lb_every iterations, or max_iters iterations. Outputs (host, may be NULL): iterations
 * run by this call and the final bound. Synchronises. TIMEOUT if max_iters was reached.
 */
int disco_converge(disco_handle *h, int32_t max_iters, int32_t *iters_done, double *lb);

/*
 * Min-marginal differences M^j_i = min_{s_i=1} s^T l~^j - min_{s_i=0} s^T l~^j (App. A.5) on
 * l~ = lambda + pend, one per slot in canonical order: BDD segments by row of (P) (closedness
 * rows by product edge, then X-, then Y-projection rows) and segment, layers in order.
 * out: n >= nslots floats, host or device. Synchronises.
 */
int disco_min_marginals(disco_handle *h, float *out, int64_t n);

/*
 * Rounds a feasible x (min-marginal agreement, propagation, perturbation; Sec. 3 pipeline,
 * App. A.5). x_out: nvars uint8 (host or device) indexed by canonical matching-element id;
 * cost (host, may be NULL): c^T x in FP64 on the normalised costs. The dual state continues
 * from where it is and is modified. Synchronises. PRIMAL_FAILED leaves the best partial x.
 */
int disco_primal(disco_handle *h, uint8_t *x_out, int64_t nvars, double *cost);

/* Copies the per-slot dual variables lambda (canonical slot order, host or device floats,
 * n >= nslots) and the per-variable deferred mean (n_pend >= nvars_free + nvars_aux, may be
 * NULL) out of / into the handle: checkpoint and warm restart. Synchronises. */
int disco_get_state(disco_handle *h, float *lam, int64_t n, float *pend, int64_t n_pend);
int disco_set_state(disco_handle *h, const float *lam, int64_t n, const float *pend, int64_t n_pend);

/* Problem and store statistics. */
int disco_info(disco_handle *h, disco_info_t *info);

/* Differentiation of the dual bound (the bound after T iterations of Eq. D's first-order
 * method, Alg. 1 "MMA", is a piecewise linear function of the costs; this gives its gradient
 * wherever it is differentiable, and a subgradient choice at ties).
 *
 * disco_record: restarts the dual at lambda^0 = c / |J| (pend = 0, b from one backward
 * pass), runs `iters` iterations (as disco_dual would) and keeps a copy of the dual state
 * every `checkpoint_every` iterations on the device (lambda, the averaging sectors and the
 * backward node costs: about 8 B per slot + 32 B per variable + 4 B per node each).
 * Errors: DISCO_ERR_INVALID_ARG for iters < 0 or checkpoint_every < 1, DISCO_ERR_OOM. */
int disco_record(disco_handle *h, int32_t iters, int32_t checkpoint_every);

/* d(bound after the recorded iterations) / d(pair costs), by reverse mode through the
 * recorded iterations: every block of checkpoint_every iterations is replayed from its
 * checkpoint recording each half-pass's inputs and stored node costs (2 * checkpoint_every
 * copies of the state), then each half-pass is reversed by an adjoint kernel. Out: for every
 * instance nvx * nvy floats (row-major, the layout of disco_build's pair costs),
 * concatenated over a batch; host or device pointer, n >= that count. The chain rule follows
 * the handle's cost model (the mean of the three pair costs, or Eq. 2's area-weighted sum).
 * The bound includes the presolve constant (gradient 1 for elements fixed to 1) and, with
 * normalize_costs, the dependence on the largest element cost. The candidate mask and
 * presolve are held fixed. The handle's state is left at the recorded final state.
 * Synchronises.
 * Errors: DISCO_ERR_INVALID_ARG (no record, output too small), DISCO_ERR_OOM. */
int disco_grad(disco_handle *h, float *dlb_dpair_costs, int64_t n);

/* Releases the handle (NULL is allowed). A handle built on a caller's stream must be freed
 * before that stream is destroyed (its device memory is returned on that stream). */
void disco_free(disco_handle *h);

/* Static string for a return code. */
const char *disco_strerror(int code);

/* Most recent error message of the calling thread ("" if none). */
const char *disco_last_error(void);

/* Number of CUDA kernel launches this library has issued in the process so far (all
 * handles and devices): a caller can difference it around a region to count its launches. */
int64_t disco_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* DISCO_H */
