/*
 * hpm.h - C ABI of a GB300 (sm_103a) solver for the Hierarchical
 * Particle-Mesh fast multipole method (Gnedin 2019, "Hierarchical
 * Particle-Mesh: an FFT-accelerated Fast Multipole Method").
 *
 * Problem (Sec. 1): N bodies in a cubic domain, gravity as potential and
 * acceleration. The domain is the level-0 cell of a cubic oct-tree whose cells
 * split into 8 children; the tree may be adaptive. The solve follows the
 * paper's four steps (Sec. 1): leaf parameterisation by gridlets of effective
 * masses (Sec. 2.2), child-to-parent transformation (Sec. 2.3),
 * source-to-target transformation by one FFT convolution per target cell
 * over its interaction zone (Sec. 2.1), parent-to-child transformation and
 * evaluation (Sec. 2.4); the near zone is summed directly (Sec. 1, item 1).
 *
 * Kernel: a radial Green function g(r) (hpm_green below; the default is
 * g(r) = 1/sqrt(r^2 + eps^2)) with G = 1 (the 1/(4 pi) of Eq. gf is not
 * used). Outputs:
 *   phi_i = -sum_{j != i} m_j g(|x_i - x_j|)   (self term excluded)
 *   a_i   = -grad phi_i
 * approximated by the method (exact for pairs in the near zone).
 *
 * Conventions for every call:
 *  - Pointers named d_* are device pointers on the current CUDA device; h_*
 *    pointers are host memory. The caller owns every buffer it passes; the
 *    library never frees or keeps a caller pointer past the call.
 *  - The library owns the plan, the tree, the gridlets and all scratch
 *    memory, and frees them in hpm_destroy.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Calls are
 *    stream ordered; a call returns after its work is enqueued except where a
 *    host read-back is documented.
 *  - Errors are returned as hpm_status; nothing is thrown across the ABI.
 *    After HPM_ERR_CUDA the CUDA context may be unusable.
 *  - Arrays of particles are in the caller's order; outputs come back in the
 *    caller's order.
 *  - A plan is not thread safe: one host thread at a time per plan.
 */
#ifndef HPM_H
#define HPM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hpm_plan_s *hpm_plan_t;

typedef enum {
  HPM_OK = 0,
  HPM_ERR_INVALID_ARG = -1,   /* bad argument (null pointer, range, size)          */
  HPM_ERR_OUT_OF_DOMAIN = -2, /* a position outside [o, o+S]^3 or not a number      */
  HPM_ERR_OOM = -3,           /* device allocation failed                           */
  HPM_ERR_CUDA = -4,          /* a CUDA runtime error; see hpm_last_cuda_error()    */
  HPM_ERR_TIMEOUT = -5,       /* a bounded device wait gave up                      */
  HPM_ERR_NOT_BUILT = -6,     /* hpm_solve before hpm_build_tree, or N mismatch     */
  HPM_ERR_BUSY = -7,          /* no free slot (serving)                             */
  HPM_ERR_UNSUPPORTED = -8    /* a valid request this build does not implement      */
} hpm_status;

/* Cubic domain [origin, origin + side)^3 with open (non-periodic) boundaries
 * (Sec. 1: only a cubic domain and cubic cells are considered). A particle at
 * exactly origin + side on an axis is placed in the last cell. */
typedef struct {
  double origin[3];
  double side;
} hpm_domain;

/* Green function g(r), radial (Sec. 4: the method only convolves with the
 * Green function, so any kernel serves; Sec. 2.1 tabulates it exactly on the
 * gridlet lattice). phi_i = -sum_{j != i} m_j g(r_ij), a_i = -grad phi_i.
 *   HPM_GREEN_PLUMMER  g = 1 / sqrt(r^2 + eps^2)                 (eps >= 0)
 *   HPM_GREEN_NEWTON   g = 1 / r                                  (eps ignored)
 *   HPM_GREEN_YUKAWA   g = exp(-s / lambda) / s, s = sqrt(r^2 + eps^2)
 *                      (eps >= 0, lambda > 0)
 *   HPM_GREEN_USER     g = user_g(r, ctx), any radial kernel: called on the
 *                      calling thread during hpm_plan (and hpm_server_create)
 *                      only, never kept; it must return finite values for
 *                      r >= side * 2^-32. The library evaluates it in FP64 on
 *                      the lattice of every level (the far-field tables) and
 *                      tabulates g and -g'(r)/r (g' by fourth-order central
 *                      differences at step r/512) for the near field as
 *                      piecewise cubics, 32 per octave of (r/side)^2 over
 *                      [2^-64, 4) side^2 (relative interpolation error about
 *                      1e-7); pairs closer than side * 2^-32 take the values
 *                      at that distance. The value at r = 0 is never used.
 * Values that are not finite at the points the plan needs make hpm_plan
 * return HPM_ERR_INVALID_ARG. */
enum { HPM_GREEN_PLUMMER = 0, HPM_GREEN_NEWTON = 1, HPM_GREEN_YUKAWA = 2, HPM_GREEN_USER = 3 };
typedef struct {
  int kind;                                 /* HPM_GREEN_*                          */
  double eps;                               /* softening length (Plummer, Yukawa)   */
  double lambda;                            /* screening length (Yukawa)            */
  double (*user_g)(double r, void *ctx);    /* HPM_GREEN_USER                       */
  void *ctx;                                /* passed to user_g                     */
} hpm_green;

/* Tree options (Sec. 1: the tree "may or may not be of uniform depth").
 * leaf_max = 0: uniform tree, every nonempty cell above max_depth splits.
 * leaf_max > 0: a cell splits iff it holds more than leaf_max particles and
 * its level is below max_depth. */
typedef struct {
  int leaf_max;
  int flags;   /* HPM_FLAG_* bits */
} hpm_plan_opts;

enum {
  HPM_FLAG_TIMINGS = 1,        /* record per-stage CUDA-event timings (hpm_get_stats)   */
  HPM_FLAG_GENERIC_M2L = 2,    /* use the any-order convolution kernel for every Ng   */
  HPM_FLAG_XTRANSFORM_M2L = 4, /* Ng = 4: evaluate the convolution with the transform
                                  along x and direct (y, z) sums (Ng = 2, 3, 5, 6
                                  always do)                                          */
  HPM_FLAG_FFT_M2L = 8,        /* Ng = 4: evaluate the convolution by the FFT method of
                                  Sec. 2.1 (register FFT-32 kernel) instead of the
                                  default dense tensor-core product, which computes
                                  the same convolution over each parent's 6^3 block
                                  with three FP16 products per term (hi*hi, hi*lo,
                                  lo*hi of FP16 pairs; same result up to FP32
                                  rounding; needs 28.3 MB of device tables per level
                                  2..max_depth, built by hpm_plan)                   */
  HPM_FLAG_EXTENDED_GRIDLET = 16 /* target gridlets widened by one node on each side
                                  (Sec. 2.5): the source-to-target values are taken
                                  at the (Ng + 2)^3 nodes x_j = (j + 1/2)/Ng - 1/2,
                                  j = -1 .. Ng, which the (8 Ng)^3 convolution still
                                  gives exactly (every node within 4 Ng = P/2 grid
                                  points of every zone source), and the local
                                  expansion is the degree-(Ng + 1) interpolant
                                  through them; effective masses stay Ng^3. Uses
                                  the any-order FFT-form kernel; Ng <= 6
                                  (HPM_ERR_UNSUPPORTED above). Stage buffers of the
                                  source-to-target and local values then hold
                                  (Ng + 2)^3 values per target                       */
};

/*
 * hpm_plan - geometry-only set-up, outside any timed region (Sec. 4: the
 * exact Green function and the matrices A, B, T are tabulated before timing).
 *   dom           domain (host struct, copied)
 *   max_depth     deepest tree level, 0..21
 *   gridlet_order Ng, gridlet points per dimension, 1..8 (Sec. 2.2 uses
 *                 Ng^3 effective masses at x_p = (p + 1/2)/Ng - 1/2)
 *   green         kernel (host struct, copied)
 *   opts          may be NULL (uniform tree, no timings)
 *   out           receives the plan handle
 * Precomputes, on the current device: the 1-D child-to-parent matrices
 * T^{+-} (Sec. 2.3) and, for every level 2..max_depth, the transform of the
 * exact Green function on the (8 Ng)^3 periodic grid (Sec. 2.1, Eq. gf),
 * evaluated in FP64 and stored in FP32. Synchronises the device.
 * Errors: HPM_ERR_INVALID_ARG, HPM_ERR_OOM, HPM_ERR_CUDA.
 */
hpm_status hpm_plan(const hpm_domain *dom, int max_depth, int gridlet_order,
                    const hpm_green *green, const hpm_plan_opts *opts, hpm_plan_t *out);

/*
 * hpm_build_tree - the oct-tree and its lists for N particles (Sec. 1).
 *   d_pos  N x 3 FP64 positions, array of structs (x0 y0 z0 x1 ...), device
 *   n      N >= 0 (N < 2^31)
 * Builds Morton keys from the FP64 positions, sorts the particles by their
 * level-max_depth key (ties by index), the per-level cell tables, the near
 * zone of every leaf and the interaction-zone occupancy of every cell at
 * level >= 2. Reads back the per-level box counts and then the work-list
 * sizes (two host synchronisations on `stream`). Errors: HPM_ERR_INVALID_ARG,
 * HPM_ERR_OUT_OF_DOMAIN, HPM_ERR_OOM, HPM_ERR_CUDA, HPM_ERR_TIMEOUT.
 */
hpm_status hpm_build_tree(hpm_plan_t plan, const double *d_pos, int64_t n, void *stream);

/*
 * hpm_solve - potential and acceleration of every particle (Sec. 1, steps
 * 1-4 plus the near zone).
 *   d_pos   N x 3 FP64 positions, the same values given to hpm_build_tree
 *   d_mass  N FP64 masses
 *   d_phi   N FP32 output potentials (may be NULL)
 *   d_acc   N x 3 FP32 output accelerations, AoS (may be NULL)
 * Stream ordered, no host synchronisation. Errors: HPM_ERR_NOT_BUILT,
 * HPM_ERR_INVALID_ARG, HPM_ERR_CUDA. Every device wait of the solve is
 * bounded; one that runs out marks the plan, and the next synchronising call
 * on it (hpm_build_tree, hpm_solve_host, hpm_get_stats) returns
 * HPM_ERR_TIMEOUT once (the outputs of that solve are then not valid).
 */
hpm_status hpm_solve(hpm_plan_t plan, const double *d_pos, const double *d_mass, float *d_phi,
                     float *d_acc, void *stream);

/*
 * hpm_build_tree_batch - trees of P independent problems at once, with the
 * same launches as one problem: particle i of problem p lies in
 * [h_offsets[p], h_offsets[p+1]) of the packed arrays. All problems share the
 * plan's domain, depth, gridlet order, kernel and split rule. hpm_solve then
 * solves every problem of the batch in one pass over the packed arrays (masses
 * and outputs packed the same way). Problems may be empty. Needs 3 max_depth +
 * ceil(log2 P) <= 63. Reads back the number of nonempty problems, the
 * per-level box counts and the work-list sizes (three host synchronisations).
 * Errors as hpm_build_tree.
 */
hpm_status hpm_build_tree_batch(hpm_plan_t plan, const double *d_pos, const int64_t *h_offsets, int n_problems,
                                void *stream);

/* One problem of hpm_solve_batch: caller-owned device buffers, layouts as for
 * hpm_solve (d_phi / d_acc may be NULL). */
typedef struct {
  const double *d_pos;
  const double *d_mass;
  int64_t n;
  float *d_phi;
  float *d_acc;
} hpm_problem;

/*
 * hpm_solve_batch - P independent problems (h_problems, host array of P
 * descriptors) solved together: the particles are gathered into library-owned
 * packed buffers by one kernel, the batch tree is built, one solve covers all
 * problems and one kernel scatters the results back to each problem's buffers.
 * Each problem's result equals its solve alone (same lists, same arithmetic in
 * the same order). Host synchronisation as hpm_build_tree_batch.
 */
hpm_status hpm_solve_batch(hpm_plan_t plan, const hpm_problem *h_problems, int n_problems, void *stream);

/*
 * hpm_solve_host - the same solve from and to host memory: copies the
 * positions in and builds the tree while the masses are copied in on a stream
 * of the plan's own (ordered after the positions' copy; the solve waits for
 * it), solves, copies phi and acc back, then synchronises `stream`. No copy
 * from the caller's buffers outlives the call, error paths included.
 * h_phi / h_acc may be NULL.
 */
hpm_status hpm_solve_host(hpm_plan_t plan, const double *h_pos, const double *h_mass, int64_t n,
                          float *h_phi, float *h_acc, void *stream);

/* Counts of the built tree (host). */
typedef struct {
  int64_t n_particles;
  int64_t n_cells;      /* real tree cells, all levels                    */
  int64_t n_targets;    /* cells at level >= 2 (one FFT convolution each)  */
  int64_t n_leaves;
  int64_t n_boxes;      /* cells plus the virtual source boxes             */
  int max_depth;
  int depth_reached;    /* deepest level holding a cell                     */
} hpm_lists_info;

hpm_status hpm_get_lists_info(hpm_plan_t plan, hpm_lists_info *info);

/*
 * hpm_get_lists - the tree and its lists in canonical form, for parity checks
 * against an independent implementation. All arrays are host memory sized from
 * hpm_get_lists_info; any pointer may be NULL to skip it. Synchronises.
 *   level, key, begin, end, leaf   per cell, cells ordered by (level, Morton key):
 *        level; Morton key at that level (bit k of x, y, z -> bits 3k, 3k+1,
 *        3k+2); particle range [begin, end) in the sorted order; leaf flag
 *   iz   n_targets x 4 words, for the cells at level >= 2 in the same order:
 *        bit j (word j/64) set iff box j = bx + 6 by + 36 bz of the 6^3 block
 *        2 (parent - 1) + (bx, by, bz) is a nonempty box of the target's
 *        interaction zone (Sec. 1: in the parent's near zone, not in the
 *        target's)
 *   near n_leaves words, leaves in cell order: bit (dx+1) + 3(dy+1) + 9(dz+1)
 *        set iff the box at offset (dx, dy, dz) is nonempty (itself included)
 *   perm N: sorted position -> caller index
 */
hpm_status hpm_get_lists(hpm_plan_t plan, int32_t *level, uint64_t *key, int64_t *begin,
                         int64_t *end, uint8_t *leaf, uint64_t *iz, uint32_t *near,
                         int64_t *perm);

/*
 * hpm_get_boxes - every box of the built tree (cells and the virtual source
 * boxes inside coarser leaves that some interaction zone needs), level-major,
 * Morton order within a level. Host arrays of n_boxes (hpm_get_lists_info);
 * NULL skips. flags: bit 0 cell, bit 1 internal cell, bit 2 leaf.
 * Synchronises.
 */
hpm_status hpm_get_boxes(hpm_plan_t plan, int32_t *level, uint64_t *key, uint8_t *flags);

/*
 * hpm_get_stage - intermediate results of the last hpm_solve, for stage-by-
 * stage parity checks. Host output, FP32, Ng^3 values per row with node
 * p = i + Ng j + Ng^2 k (Sec. 2.2). Synchronises. `count` is the number of
 * floats the caller provides; HPM_ERR_INVALID_ARG if it is too small.
 *   HPM_STAGE_MASSES  effective masses of every box at level >= 2, rows in
 *                     hpm_get_boxes order starting at the first level-2 box
 *                     (Sec. 2.2 for leaves and virtual boxes, Sec. 2.3 for
 *                     internal cells)
 *   HPM_STAGE_M2L     source-to-target values of every target (cells at level
 *                     >= 2 in cell order), Ng^3 values ((Ng + 2)^3 with
 *                     HPM_FLAG_EXTENDED_GRIDLET) then one constant per
 *                     target: Phi_p = row_p + const (Sec. 2.1)
 *   HPM_STAGE_LOCAL   local gridlet after the parent-to-child pass (Sec. 2.4),
 *                     same layout: deviations then one constant per target
 */
enum { HPM_STAGE_MASSES = 1, HPM_STAGE_M2L = 2, HPM_STAGE_LOCAL = 3 };
hpm_status hpm_get_stage(hpm_plan_t plan, int stage, float *h_out, int64_t count);

/* Per-stage device times of the last solve (flags bit 0), milliseconds, and
 * launch counts. */
typedef struct {
  float ms_tree, ms_p2g, ms_m2m, ms_m2l, ms_l2l, ms_g2p, ms_p2p, ms_total;
  int64_t launches;        /* kernels launched by the last build + solve */
  int64_t m2l_launches;    /* of which source-to-target                  */
  int64_t m2l_targets;     /* target cells convolved by the last solve    */
  float ms_m2l_kernel;     /* Ng = 4 tensor-core path: the dense product
                              kernel alone (0 on the other paths)         */
  int64_t m2l_parents;     /* parents whose 6^3 blocks that kernel
                              multiplied (0 on the other paths)           */
  int64_t p2p_pairs;       /* near-zone pairs (i, j), j != i, summed by
                              the near field of the last solve            */
  int64_t table_bytes;     /* device bytes of the plan's tables (Green
                              transforms and lattice, W, near-field table),
                              held from hpm_plan to hpm_destroy           */
  int64_t work_bytes;      /* device bytes the last build and solve needed
                              in the plan's other buffers (each buffer is
                              kept at its largest size so far, so the plan
                              may hold more)                              */
} hpm_stats;

hpm_status hpm_get_stats(hpm_plan_t plan, hpm_stats *stats);

/* ------------------------------------------------------------------------
 * Launch shapes and their autotuner (an implementation choice; the paper
 * has none). Every shape here changes only how the work is spread over the
 * GPU: results are bit for bit the same for every value.
 * ------------------------------------------------------------------------ */
typedef struct {
  int level_blocks_per_sm; /* tree build: CTAs per SM of the cooperative level
                              kernel, 1..4 (0 = 2; capped at what fits)          */
  int gridlet_warps;       /* Ng = 4 child-to-parent and parent-to-child: warps
                              (one gridlet each) per CTA, 2, 4 or 8 (0 = 8)      */
  int m2l_ctas_per_sm;     /* FFT-form source-to-target kernels (HPM_FLAG_FFT_M2L,
                              HPM_FLAG_XTRANSFORM_M2L, other orders): persistent
                              CTAs per SM, 1 or 2 (0 = the most that fit)        */
  int m2l_block_order;     /* dense tensor-core source-to-target (Ng = 4, 6): the
                              order of its CTAs, 1 tile-major (the row blocks of
                              W for one tile of parents run together), 2 row-
                              block-major (one pair of row blocks runs over every
                              tile first: that part of W stays in L2 while the
                              parents' gridlets stream); 0 = 1                   */
  int m2l_tile_parents;    /* dense tensor-core source-to-target at Ng = 4:
                              parents per tile (the MMA's N), 256, 224, 208 or
                              192 (0 = 256); a narrower tile spreads each
                              level's parents over more CTA pairs. Applies from
                              the next hpm_build_tree (the tiles are built
                              there) */
} hpm_tuning;

/* Sets the plan's launch shapes (values outside the ranges above are
 * HPM_ERR_INVALID_ARG); they apply from the next build / solve. */
hpm_status hpm_set_tuning(hpm_plan_t plan, const hpm_tuning *tuning);
hpm_status hpm_get_tuning(hpm_plan_t plan, hpm_tuning *tuning);

/* Autotuner: builds and solves the given input (device positions and masses,
 * N x 3 and N FP64, as hpm_solve) for each candidate value of one shape at a
 * time, the others fixed, timing the stage the shape drives with CUDA events
 * on `stream` (best of three runs per candidate), and keeps the fastest in
 * the plan; `out` (may be null) receives the result. Shapes that do not apply
 * to the plan (m2l_ctas_per_sm on the Ng = 4 tensor-core path, gridlet_warps
 * at Ng != 4) keep their current value. Uses plan-owned output buffers,
 * synchronises the stream, leaves the plan built for this input.
 * Errors: those of hpm_build_tree and hpm_solve. */
hpm_status hpm_tune(hpm_plan_t plan, const double *d_pos, const double *d_mass, int64_t n, void *stream,
                    hpm_tuning *out);

/* Failure test hook. With `on` set, the source-to-target kernel of the
 * Ng = 4 tensor-core path first waits on a barrier that nothing arrives at;
 * every wait of that kernel is bounded by wait_limit_cycles (0 = the default,
 * about 2^32 cycles), so the kernel gives up, records the timeout and returns
 * (no GPU fault), and the next synchronising call on the plan returns
 * HPM_ERR_TIMEOUT. on = 0 restores normal operation (wait_limit_cycles also
 * applies then). Errors: HPM_ERR_INVALID_ARG. */
hpm_status hpm_test_stall(hpm_plan_t plan, int on, long long wait_limit_cycles);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of independent solves (no counterpart in the
 * paper; it serves the same solve to a stream of requests).
 * ------------------------------------------------------------------------ */
typedef struct hpm_server_s *hpm_server_t;

typedef struct {
  hpm_domain dom;           /* shared by every request                          */
  int max_depth;
  int gridlet_order;
  hpm_green green;
  int leaf_max;
  int workers;              /* worker threads, each with its own plan and stream
                               (>= 2 lets batches overlap on the device; 0 admits
                               requests but never runs them)                      */
  int max_batch;            /* requests per batch, >= 1                          */
  int64_t hbm_budget_bytes; /* admission bound on the estimated device memory of
                               all batches in flight; the worker plans' tables
                               are outside it                                     */
  double bytes_per_particle;/* the estimate's rate: a request of N particles is
                               taken to need rate x N + 8 MiB. 0: calibrated,
                               1.25 x the largest per-particle need beyond the
                               8 MiB measured on a completed batch (512 until
                               the first one);
                               > 0: this fixed rate. A queued request whose
                               estimate exceeds the whole budget (after a
                               recalibration) runs alone when nothing else is
                               in flight                                          */
  int64_t max_batch_particles;/* particles per batch (0: no bound, plain FIFO
                               batches); a batch's solve time grows with its
                               particles, and every request in it waits for all
                               of them. A request larger than the bound is large:
                               it runs alone, and one large request at a time;
                               while one runs, small requests queued behind a
                               waiting large one go ahead of it               */
} hpm_server_opts;

/* One request. pos (N x 3 FP64) and mass (N FP64) are read, phi (N FP32) and
 * acc (N x 3 FP32) written; each may be host or device memory (copies use
 * unified addressing). The buffers must stay valid until the request is done
 * or cancelled. */
typedef struct {
  const double *pos;
  const double *mass;
  int64_t n;
  float *phi;
  float *acc;
} hpm_request;

typedef struct {
  int64_t submitted, completed, rejected, cancelled, failed, batches, queued;
  int64_t in_flight_bytes;  /* estimated device bytes of the batches in flight */
  int64_t particles;        /* particles of completed requests                 */
  double p50_ms, p99_ms;    /* submit -> results in the caller's buffers, over the
                               last 65,536 completions                           */
  double mean_ms;           /* the same, over all completions since the last reset */
  double particles_per_s;   /* completed particles / (last completion - first submit) */
  double bytes_per_particle;/* device bytes per particle beyond 8 MiB that
                               completed batches needed (largest seen; 0
                               before the first)                                */
} hpm_server_stats;

/* Creates the worker plans (hpm_plan, synchronises) and starts the workers.
 * Errors: HPM_ERR_INVALID_ARG, and those of hpm_plan. */
hpm_status hpm_server_create(const hpm_server_opts *opts, hpm_server_t *out);
/* Queues a request; *ticket identifies it. A request whose estimated footprint
 * (hpm_server_opts.bytes_per_particle) exceeds the whole budget is refused
 * with HPM_ERR_OOM. Never blocks on the GPU. */
hpm_status hpm_server_submit(hpm_server_t server, const hpm_request *req, uint64_t *ticket);
/* *done: 1 finished, 0 pending, -1 cancelled or failed; latency in ms once done.
 * Once a call reports a final state (*done != 0) the server forgets the
 * request: the ticket is then unknown (HPM_ERR_INVALID_ARG). */
hpm_status hpm_server_poll(hpm_server_t server, uint64_t ticket, int *done, double *latency_ms);
/* Waits at most timeout_ms (bounded wait): HPM_ERR_TIMEOUT if still pending,
 * HPM_ERR_INVALID_ARG if it was cancelled, HPM_ERR_BUSY if the server is
 * being destroyed meanwhile. A return with the final state (HPM_OK, a failed
 * solve's status, or cancelled) ends the ticket as for hpm_server_poll. */
hpm_status hpm_server_wait(hpm_server_t server, uint64_t ticket, int timeout_ms, double *latency_ms);
/* Cancels a request that is still queued; HPM_ERR_BUSY once it runs or ran. */
hpm_status hpm_server_cancel(hpm_server_t server, uint64_t ticket);
hpm_status hpm_server_get_stats(hpm_server_t server, hpm_server_stats *stats);
hpm_status hpm_server_reset_stats(hpm_server_t server);
/* Stops the workers after their current batch and frees everything. Threads
 * blocked in hpm_server_wait are woken first and return HPM_ERR_BUSY; no
 * other call on the server may run concurrently with, or follow, this one. */
hpm_status hpm_server_destroy(hpm_server_t server);

/*
 * hpm_sort_particles_static - the Morton keys of N positions and their stable
 * sort, the first step of hpm_build_tree, without allocating any memory. The
 * paper has no counterpart: it is a service for callers that cannot call
 * cudaMalloc or any other allocator, for example code that runs under a
 * fixed device-memory budget set by a host application that owns all
 * allocation, or that must not allocate between set-up and shutdown.
 *   dom, max_depth  as for hpm_plan; keys are taken at level max_depth
 *   d_pos           N x 3 FP64 positions (device), AoS
 *   n               0 <= N <= HPM_STATIC_SORT_MAX_N
 *   d_keys          N u64 (device, caller-owned): the level-max_depth Morton
 *                   keys in ascending order (ties kept in caller order)
 *   d_perm          N u32 (device, caller-owned): sorted position -> caller
 *                   index, the same permutation hpm_get_lists reports
 * Scratch lives in one static device array of about 12.6 MiB that every GPU
 * loading the library holds until the process exits; it limits N to
 * HPM_STATIC_SORT_MAX_N and a larger N returns HPM_ERR_INVALID_ARG without
 * touching the device. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, once per device, under a lock); make that
 * first call before any stream capture on that device. All calls share the
 * array and each call overwrites it, so calls that overlap on the GPU (other
 * streams, other threads) race and must be serialised by the caller. Reads
 * back one error word and synchronises `stream`.
 * Errors: HPM_ERR_INVALID_ARG, HPM_ERR_OUT_OF_DOMAIN, HPM_ERR_CUDA,
 * HPM_ERR_TIMEOUT (a bounded wait of the sort's scan gave up),
 * HPM_ERR_UNSUPPORTED (a device index of 64 or more).
 */
#define HPM_STATIC_SORT_MAX_N 1048576
hpm_status hpm_sort_particles_static(const hpm_domain *dom, int max_depth, const double *d_pos, int64_t n,
                                     uint64_t *d_keys, uint32_t *d_perm, void *stream);

/* ------------------------------------------------------------------------
 * Measured arithmetic peaks of the current device (no counterpart in the
 * paper): the denominators of the rooflines of the kernels bound by CUDA-core
 * arithmetic. Each rate comes from a kernel of independent dependent-FMA (or
 * rsqrt) chains filling every SM, best of three launches of several
 * milliseconds timed with CUDA events on `stream` (synchronised). Scratch:
 * 64 bytes from the library's pool. Errors: HPM_ERR_INVALID_ARG,
 * HPM_ERR_CUDA, HPM_ERR_OOM.
 * ------------------------------------------------------------------------ */
typedef struct {
  double fp32_tflops;   /* FFMA, 2 FLOP per lane and instruction      */
  double fp64_tflops;   /* DFMA, 2 FLOP per lane and instruction      */
  double rsqrt_gops;    /* FP32 reciprocal square roots per second / 1e9 */
  double ms_fp32, ms_fp64, ms_rsqrt;  /* best launch durations         */
  int sm_count;
} hpm_alu_peaks;
hpm_status hpm_measure_alu_peaks(hpm_alu_peaks *out, void *stream);

/* ------------------------------------------------------------------------
 * Self-check of the float <-> double conversions the library does by
 * IEEE 754 bit manipulation on the integer units (in the gather of the
 * sorted particles: exact float -> double; double -> float rounded to
 * nearest, ties to even): converts the n_d doubles at d_in and the n_f
 * floats at f_in (device memory, either may be empty) both ways, its own and
 * the hardware's, and returns in *mismatches the number of inputs whose
 * results differ in any bit (NaNs compared by class). Synchronises `stream`.
 * Errors: HPM_ERR_INVALID_ARG, HPM_ERR_CUDA, HPM_ERR_OOM.
 * ------------------------------------------------------------------------ */
hpm_status hpm_check_conversions(const double *d_in, int64_t n_d, const float *f_in, int64_t n_f,
                                 int64_t *mismatches, void *stream);

/* Frees the plan and everything it owns. NULL is allowed. */
hpm_status hpm_destroy(hpm_plan_t plan);

/* Static strings. */
const char *hpm_status_str(hpm_status s);
const char *hpm_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HPM_H */
